"""Domains far from the origin. Positions, centres and cell planes are kept relative
to the domain's lower corner on both sides (planes g * h), so their fp32 rounding
depends on the domain's size only. In world coordinates a domain at 1000 with a side
that is not a power of two would round deep cell planes by up to 3e-5, and
distinct planes would merge.

Against the FP64 oracle (whose values use the planes lo + g * h exactly), on seeded
sinks: 2^20 particles in [1000, 1001)^3; and 2^18 particles in a domain of side
0.75 at (1000.3, 999.7, 1000.1) with a quarter of them in a clump of width 3e-4 of
the side, where the tree's cells reach below the fp32 spacing of the coordinates."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["unit_side_at_1000", "clump_at_1000.3_side_0.75"])
def test_far_domain_parity(case):
    from paper_1902_08083_gb300 import trevr
    if case == "unit_side_at_1000":
        P = workloads.far_domain()
    else:
        P = workloads.far_domain(n_gas=1 << 18, n_src=256, seed=11,
                                 lo=(1000.3, 999.7, 1000.1), side=0.75, clump_frac=0.25)
    G = gpu_tree(P)
    f, c = trevr.compute_flux(G, P["theta"], P["tau_ref"], counters=True)
    n = P["gas_xyz"].shape[1]
    sinks = np.concatenate([workloads.sink_sample(n, 3072, seed=3), np.arange(0, 1024)])
    T = oracle_tree(P)
    ref, rc, _ = T.flux(P["theta"], P["tau_ref"], sinks=sinks, with_counters=True)
    assert_flux_parity(f.cpu().numpy()[sinks], ref, case)
    mism = np.count_nonzero(np.any(c.cpu().numpy()[sinks] != rc.astype(np.int32), axis=1))
    assert mism <= 4, f"{mism} sinks with other decisions"
    G.free()
