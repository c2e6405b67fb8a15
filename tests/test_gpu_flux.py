"""GPU flux vs the FP64 oracle (Eq. simpint over the pseudo-sources of the
opening-angle walk, with tau_ref refinement), element by element on the same
seeded inputs; per-sink counters (rays, segments, visited cells, refinements)
must match exactly because both sides take the decisions in the same fp32 steps."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, clumpy_problem, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def _run(P, theta, tau_ref, sinks=None, **tuning):
    import torch
    from paper_1902_08083_gb300 import trevr
    G = gpu_tree(P)
    sidx = None if sinks is None else torch.from_numpy(np.asarray(sinks, np.int64)).cuda()
    f, c, st = trevr.compute_flux(G, theta, tau_ref, sink_idx=sidx, counters=True, stats=True,
                                  **tuning)
    return G, f.cpu().numpy(), c.cpu().numpy(), st


def _lognormal(P, sigma=2.0, seed=1, corr=0.05):
    rng = np.random.default_rng(seed)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, sigma, corr, n_modes=128)
    return P


VARIANTS = [1, 2, 3]  # per-lane walk, warp-shared walk, warp-shared with merged rays


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("theta,tau_ref", [(0.75, 0.1), (0.0, 0.1), (0.75, 0.0), (0.4, 1e6)])
def test_uniform_box_4096(theta, tau_ref, variant):
    P = workloads.uniform_box(n_gas=4096, n_src=64, seed=0)
    G, f, c, st = _run(P, theta, tau_ref, walk_variant=variant)
    T = oracle_tree(P)
    ref, rc, margin = T.flux(theta, tau_ref, with_counters=True)
    assert_flux_parity(f, ref, f"uniform theta={theta} tau_ref={tau_ref}")
    np.testing.assert_array_equal(c, rc.astype(np.int32))
    assert st["interactions"] == rc[:, 0].sum() and st["segments"] == rc[:, 1].sum()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("theta,tau_ref", [(0.75, 0.1), (0.6, 0.01), (0.75, 0.0), (0.0, 0.3)])
def test_lognormal_refinement(theta, tau_ref, variant):
    P = _lognormal(workloads.uniform_box(n_gas=12000, n_src=200, seed=21), sigma=2.0)
    G, f, c, st = _run(P, theta, tau_ref, walk_variant=variant)
    T = oracle_tree(P)
    ref, rc, margin = T.flux(theta, tau_ref, with_counters=True)
    assert_flux_parity(f, ref, f"lognormal theta={theta} tau_ref={tau_ref}")
    assert rc[:, 3].sum() > 0  # refinement happened
    mism = np.nonzero(np.any(c != rc, axis=1))[0]
    assert len(mism) <= max(1, len(f) // 1000), f"{len(mism)} sinks with other decisions"


@pytest.mark.parametrize("variant", VARIANTS)
def test_weighted_cells_and_sink_subset(variant):
    P = _lognormal(workloads.uniform_box(n_gas=7777, n_src=100, seed=22), sigma=1.0)
    P["weight"] = np.random.default_rng(3).uniform(0.1, 4.0, 7777).astype(np.float32)
    sinks = np.random.default_rng(4).choice(7777, 1001, replace=False)
    sinks[5] = sinks[6]  # a repeated sink is allowed
    G, f, c, _ = _run(P, 0.75, 0.1, sinks=sinks, walk_variant=variant)
    T = oracle_tree(P)
    ref, rc, _ = T.flux(0.75, 0.1, sinks=sinks, with_counters=True)
    assert_flux_parity(f, ref, "weighted subset")
    np.testing.assert_array_equal(c, rc.astype(np.int32))


def _clumpy():
    return clumpy_problem()


@pytest.mark.parametrize("tau_ref", [0.01, 0.1, 0.5])
def test_stromgren_closed_form(tau_ref):
    # one source of L=1 at the centre, alpha=20: F = exp(-20 r) / (4 pi r^2) exactly
    P = workloads.stromgren(n_gas=1 << 18, seed=1, tau_ref=tau_ref)
    G, f, c, st = _run(P, P["theta"], tau_ref)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    ref = np.exp(-20.0 * r) / (4 * np.pi * r * r)
    assert_flux_parity(f, ref, f"stromgren tau_ref={tau_ref}")
    assert np.all(c[:, 0] == 1) and st["refine_expansions"] == 0
    # the oracle agrees on a sample, counters included
    sinks = workloads.sink_sample(1 << 18, 2048)
    T = oracle_tree(P)
    o, oc, _ = T.flux(P["theta"], tau_ref, sinks=sinks, with_counters=True)
    assert_flux_parity(f[sinks], o, "stromgren vs oracle")
    np.testing.assert_array_equal(c[sinks], oc.astype(np.int32))


@pytest.mark.parametrize("variant", VARIANTS)
def test_clumpy_full_size_sampled(variant):
    # 2^22 gas, 2^14 clustered sources, lognormal absorption with a dense occluder;
    # the GPU computes every sink in the benchmark's launch shape, the oracle a sample
    P = _clumpy()
    G, f, c, st = _run(P, P["theta"], P["tau_ref"], walk_variant=variant)
    assert np.all(np.isfinite(f)) and np.all(f >= 0)
    sinks = workloads.sink_sample(P["gas_xyz"].shape[1], 1024)
    T = oracle_tree(P)
    ref, rc, margin = T.flux(P["theta"], P["tau_ref"], sinks=sinks, with_counters=True)
    assert_flux_parity(f[sinks], ref, "clumpy sampled")
    mism = np.nonzero(np.any(c[sinks] != rc, axis=1))[0]
    assert len(mism) <= 2
    assert st["refine_expansions"] > 0


def test_empty_and_degenerate_calls():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=500, n_src=3, seed=2)
    G = gpu_tree(P)
    out = trevr.compute_flux(G, 0.75, 0.1, sink_idx=torch.empty(0, dtype=torch.int64,
                                                                 device="cuda"))
    assert out.numel() == 0
    # no sources at all: zero flux everywhere
    P0 = workloads.uniform_box(n_gas=300, n_src=1, seed=3)
    P0["src_xyz"] = np.zeros((3, 0), np.float32)
    P0["src_lum"] = np.zeros(0, np.float32)
    f = trevr.compute_flux(gpu_tree(P0), 0.75, 0.1)
    assert torch.all(f == 0)
    # zero-luminosity sources are skipped
    P1 = workloads.uniform_box(n_gas=300, n_src=4, seed=3)
    P1["src_lum"][:] = 0
    f, c = trevr.compute_flux(gpu_tree(P1), 0.75, 0.1, counters=True)
    assert torch.all(f == 0) and torch.all(c == 0)


def test_error_status_without_fault():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=4096, n_src=64, seed=0)
    G = gpu_tree(P)
    for variant in VARIANTS:
        with pytest.raises(trevr.TrevrError) as ei:
            trevr.compute_flux(G, 0.75, 0.1, stats=True, stack_depth=2, walk_variant=variant)
        assert ei.value.code == 3  # stack overflow reported, no trap
    with pytest.raises(trevr.TrevrError) as ei:
        trevr.compute_flux(G, -1.0, 0.1)
    assert ei.value.code == 1
    with pytest.raises(ValueError):
        trevr.compute_flux(G, 0.75, 0.1, sink_idx=None, out=torch.empty(1, device="cuda"))
    bad = torch.tensor([0, 4096], dtype=torch.int64, device="cuda")  # index out of range
    with pytest.raises(trevr.TrevrError) as ei:
        trevr.compute_flux(G, 0.75, 0.1, sink_idx=bad, stats=True)
    assert ei.value.code == 1
    # the tree and context still work after the reported errors
    f = trevr.compute_flux(G, 0.75, 0.1, stats=True)[0]
    T = oracle_tree(P)
    assert_flux_parity(f.cpu().numpy(), T.flux(0.75, 0.1), "after errors")
