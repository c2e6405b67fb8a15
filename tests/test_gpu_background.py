"""Background radiation on the GPU (Sec. 2.2.4): sources on a spiral sphere around
the volume. GPU vs oracle at theta = 0.75, and at theta = 0 vs the shell formula
L/(8 pi R r) ln((R+r)/(R-r)) (Eq. cosmof read with its missing 1/r)."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def test_background_shell_gpu():
    from paper_1902_08083_gb300 import trevr
    P = workloads.background_shell(n_gas=1 << 15, n_bg=20000, radius=0.45)
    G = gpu_tree(P)
    T = oracle_tree(P)
    for theta in (0.75, 0.3):
        f = trevr.compute_flux(G, theta, 0.1).cpu().numpy()
        sinks = workloads.sink_sample(1 << 15, 1024, seed=90)
        assert_flux_parity(f[sinks], T.flux(theta, 0.1, sinks=sinks), f"background theta={theta}")
    f0 = trevr.compute_flux(G, 0.0, 0.1).cpu().numpy().astype(np.float64)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    inner = r < 0.35
    ref = 1.0 / (8 * np.pi * 0.45 * r[inner]) * np.log((0.45 + r[inner]) / (0.45 - r[inner]))
    np.testing.assert_allclose(f0[inner], ref, rtol=2e-3)


@pytest.mark.parametrize("alpha,theta", [(0.0, 0.75), (3.0, 0.6), (3.0, 0.0)])
def test_background_projection_gpu(alpha, theta):
    # merged background sources moved onto the sphere (Sec. 2.2.4): same fluxes and
    # counters as the oracle, rays ending in the leaf that holds the moved point
    from paper_1902_08083_gb300 import trevr
    P = workloads.background_shell(n_gas=1 << 14, n_bg=8000, radius=0.45, alpha=alpha)
    G = gpu_tree(P)
    T = oracle_tree(P)
    f, c = trevr.compute_flux(G, theta, 0.1, counters=True, bg_radius=0.45)
    of, oc = T.flux_background(theta, 0.1, 0.45, with_counters=True)
    assert_flux_parity(f.cpu().numpy(), of, f"background projection alpha={alpha}")
    mism = np.nonzero(np.any(c.cpu().numpy() != oc.astype(np.int32), axis=1))[0]
    assert len(mism) <= 2


def test_background_projection_only_for_the_plain_flux():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.background_shell(n_gas=2000, n_bg=500, radius=0.45)
    G = gpu_tree(P)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_moments(G, 0.75, 0.1, bg_radius=0.45)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_backward(G, torch.ones(2000, device="cuda"), 0.75, 0.1,
                                    bg_radius=0.45)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux(G, 0.75, 0.1, bg_radius=-1.0)
