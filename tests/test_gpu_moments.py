"""GPU flux vector and radiation-pressure moment (trevr_compute_flux_moments) vs the
oracle: sum f n (Eq. simpflux) and sum f n n^T from the same walk as the flux; plus
rays that run exactly along cut planes (boxes half-open along a still axis)."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def _moments_close(gv, ov, F, label):
    # components can cancel: compare them on the scale of the scalar flux
    err = np.abs(np.asarray(gv, np.float64) - ov) / F[:, None]
    assert np.median(err) <= 1e-5, f"{label}: median {np.median(err):.3e}"
    assert err.max() <= 1e-3, f"{label}: max {err.max():.3e}"


@pytest.mark.parametrize("theta,tau_ref", [(0.75, 0.1), (0.0, 0.0)])
def test_moments_vs_oracle(theta, tau_ref):
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=8000, n_src=150, seed=80)
    rng = np.random.default_rng(81)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, 1.5, 0.05, n_modes=128)
    G = gpu_tree(P)
    f, v, m = trevr.compute_flux_moments(G, theta, tau_ref)
    f, v, m = f.cpu().numpy(), v.cpu().numpy().T, m.cpu().numpy().T
    T = oracle_tree(P)
    of, ov, om = T.flux_moments(theta, tau_ref)
    assert_flux_parity(f, of, "moments flux")
    _moments_close(v, ov, of, "flux vector")
    _moments_close(m, om, of, "pressure")
    tr = m[:, 0] + m[:, 1] + m[:, 2]
    np.testing.assert_allclose(tr, f, rtol=1e-5)
    # the scalar equals the plain flux call
    np.testing.assert_allclose(f, trevr.compute_flux(G, theta, tau_ref).cpu().numpy(), rtol=1e-6)


def test_moments_single_source_direction():
    from paper_1902_08083_gb300 import trevr
    P = workloads.stromgren(n_gas=1 << 16, seed=82)
    f, v, _ = trevr.compute_flux_moments(gpu_tree(P), 0.75, 0.1, pressure=False)
    f, v = f.cpu().numpy().astype(np.float64), v.cpu().numpy().T
    d = P["gas_xyz"].astype(np.float64).T - 0.5
    r = np.linalg.norm(d, axis=1)
    _moments_close(v, f[:, None] * d / r[:, None], f, "single source")


def test_rays_along_cut_planes():
    # six sources at +-1/4 around a sink at the centre: the rays run along the planes
    # x, y, z = 1/2 that cut the tree; each face cell counts once (half-open boxes)
    from paper_1902_08083_gb300 import trevr
    rng = np.random.default_rng(73)
    gas = rng.random((3, 500)).astype(np.float32)
    gas[:, 0] = 0.5
    src = np.array([[0.75, 0.25, 0.5, 0.5, 0.5, 0.5], [0.5, 0.5, 0.75, 0.25, 0.5, 0.5],
                    [0.5, 0.5, 0.5, 0.5, 0.75, 0.25]], np.float32)
    P = dict(gas_xyz=gas, alpha=np.full(500, 3.0, np.float32), src_xyz=src,
             src_lum=np.full(6, 2.0, np.float32), lo=(0.0, 0.0, 0.0), side=1.0, bucket=4)
    G = gpu_tree(P)
    T = oracle_tree(P)
    for theta, tau_ref in ((0.0, 0.0), (0.0, 0.1), (0.8, 0.1)):
        f, c = trevr.compute_flux(G, theta, tau_ref, counters=True)
        of, oc, _ = T.flux(theta, tau_ref, with_counters=True)
        assert_flux_parity(f.cpu().numpy(), of, "cut planes")
        np.testing.assert_array_equal(c.cpu().numpy(), oc.astype(np.int32))
    f1 = 2.0 * np.exp(-0.75) / (4 * np.pi * 0.0625)
    f0, v0, m0 = trevr.compute_flux_moments(G, 0.0, 0.1)
    assert abs(float(f0[0]) - 6 * f1) <= 1e-5 * 6 * f1
    assert float(v0[:, 0].abs().max()) <= 1e-5 * 6 * f1


def test_moments_clumpy_sampled():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.clumpy(n_gas=1 << 20, n_src=1 << 12, seed=83)
    sinks = workloads.sink_sample(1 << 20, 1024, seed=84)
    G = gpu_tree(P)
    f, v, m = trevr.compute_flux_moments(G, P["theta"], P["tau_ref"],
                                         sink_idx=torch.from_numpy(sinks).cuda())
    T = oracle_tree(P)
    of, ov, om = T.flux_moments(P["theta"], P["tau_ref"], sinks=sinks)
    assert_flux_parity(f.cpu().numpy(), of, "clumpy moments flux")
    _moments_close(v.cpu().numpy().T, ov, of, "clumpy flux vector")
    _moments_close(m.cpu().numpy().T, om, of, "clumpy pressure")
