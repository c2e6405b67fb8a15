"""The single-tree walk's autotuner on the GPU: it times every walk shape on the
caller's tree, the shape it picks gives the same decisions (per-sink counters) as
the default walk and fluxes within rounding of them, and a repeated call is
answered from its cache."""
import numpy as np
import pytest

import workloads
from _parity import gpu_tree

pytestmark = pytest.mark.gpu


def test_tune_walk_on_a_tree(tmp_path):
    from paper_1902_08083_gb300 import autotune, trevr
    P = workloads.uniform_box(n_gas=1 << 16, n_src=512, seed=41)
    rng = np.random.default_rng(42)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, 1.5, 0.1, n_modes=64)
    G = gpu_tree(P)
    cache = str(tmp_path / "walk.json")
    r = autotune.tune_walk(G, 0.6, 0.1, cache_path=cache, repeats=1)
    assert (r["walk_variant"], r["sinks_per_warp"]) in autotune.WALK_SHAPES
    assert not r["cached"] and len(r["table"]) == len(autotune.WALK_SHAPES)
    assert all(t > 0 for t in r["table"].values())
    f0, c0 = trevr.compute_flux(G, 0.6, 0.1, counters=True)
    f1, c1 = trevr.compute_flux(G, 0.6, 0.1, counters=True, walk_variant=r["walk_variant"],
                                sinks_per_warp=r["sinks_per_warp"])
    np.testing.assert_array_equal(c0.cpu().numpy(), c1.cpu().numpy())
    np.testing.assert_allclose(f1.cpu().numpy(), f0.cpu().numpy(), rtol=2e-6)
    again = autotune.tune_walk(G, 0.6, 0.1, cache_path=cache)
    assert again["cached"] and again["walk_variant"] == r["walk_variant"]
    G.free()
