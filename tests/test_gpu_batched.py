"""Batched persistent launch (trevr_compute_flux_batched): many independent boxes of
uneven sizes in one launch, bit-identical to one plain call per box, under every
launch shape, and when replayed from a CUDA graph; plus the autotuner."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boxes():
    return workloads.batched_boxes()  # 64 boxes, 2^12 .. 2^17 particles


@pytest.fixture(scope="module")
def trees(boxes):
    return [gpu_tree(P) for P in boxes]


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_batched_equals_sequential_bitwise(boxes, trees, variant):
    import torch
    from paper_1902_08083_gb300 import trevr
    th, tr = boxes[0]["theta"], boxes[0]["tau_ref"]
    seq = [trevr.compute_flux(t, th, tr, walk_variant=variant) for t in trees]
    seq_stats = [trevr.compute_flux(t, th, tr, stats=True, walk_variant=variant)[1]
                 for t in trees]
    B = trevr.Batch(trees)
    for item, bs in ((64, 128), (32, 64), (256, 256), (96, 128)):
        st = B.run(th, tr, stats=True, sinks_per_warp=item, block_size=bs, walk_variant=variant)
        for b in range(len(trees)):
            assert torch.equal(B.flux[b], seq[b]), (item, bs, b)
        for k in ("interactions", "segments", "src_nodes_visited", "refine_expansions"):
            assert st[k] == sum(s[k] for s in seq_stats)
    B.free()


def test_batched_graph_replay(boxes, trees):
    import torch
    from paper_1902_08083_gb300 import trevr
    th, tr = boxes[0]["theta"], boxes[0]["tau_ref"]
    seq = [trevr.compute_flux(t, th, tr) for t in trees]
    B = trevr.Batch(trees)
    B.capture(th, tr, sinks_per_warp=64, block_size=128)
    for f in B.flux:
        f.fill_(-1.0)
    for _ in range(3):
        B.replay()
    torch.cuda.synchronize()
    B.check()
    for b in range(len(trees)):
        assert torch.equal(B.flux[b], seq[b])
    B.free()


def test_batched_small_boxes_vs_oracle():
    # ragged: boxes of 1, 33 and 5000 particles, one with no sources
    from paper_1902_08083_gb300 import trevr
    Ps = [workloads.uniform_box(n_gas=n, n_src=s, seed=60 + n) for n, s in
          ((1, 1), (33, 2), (5000, 40))]
    Ps.append(workloads.uniform_box(n_gas=700, n_src=1, seed=9))
    Ps[-1]["src_lum"][:] = 0.0
    trees = [gpu_tree(P) for P in Ps]
    B = trevr.Batch(trees)
    B.run(0.75, 0.1, sinks_per_warp=32)
    B.check()
    for P, f in zip(Ps, B.flux):
        ref = oracle_tree(P).flux(0.75, 0.1)
        if np.all(ref == 0):
            assert float(f.abs().max()) == 0.0
        else:
            assert_flux_parity(f.cpu().numpy(), ref, P["name"])
    B.free()


def test_autotuner_picks_a_valid_shape(boxes, trees, tmp_path):
    from paper_1902_08083_gb300 import autotune, trevr
    B = trevr.Batch(trees[:16])
    res = autotune.tune(B, boxes[0]["theta"], boxes[0]["tau_ref"],
                        cache_path=str(tmp_path / "tune.json"), repeats=1)
    assert res["sinks_per_warp"] in autotune.ITEM_SIZES
    assert res["block_size"] in autotune.BLOCK_SIZES
    assert res["walk_variant"] in autotune.VARIANTS
    assert not res["cached"] and len(res["table"]) == 36
    again = autotune.tune(B, boxes[0]["theta"], boxes[0]["tau_ref"],
                          cache_path=str(tmp_path / "tune.json"))
    assert again["cached"] and again["sinks_per_warp"] == res["sinks_per_warp"]
    B.free()
