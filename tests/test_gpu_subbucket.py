"""Sub-bucket particle trace on the GPU (Sec. 2.2.3, 3.1.3): GPU vs the oracle's
SPH-field integral (its closed-form kernel integrals against the kernel's
pre-computed integral table, bilinear on a 1025 x 1025 grid), with the counters of
the walk; the opaque sink that does not shadow itself; the argument checks."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity

pytestmark = pytest.mark.gpu


def _gpu(P):
    import torch
    from paper_1902_08083_gb300 import trevr
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    G = trevr.build_tree(t(P["gas_xyz"]), t(P["alpha"]), t(P["src_xyz"]), t(P["src_lum"]),
                         weight=t(P["weight"]), bucket=P["bucket"])
    G.set_smoothing(t(P["hsml"]))
    return G


def _oracle(oracle_lib, P):
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"],
                              bucket=P["bucket"], weight=P["weight"])
    T.set_smoothing(P["hsml"])
    return T


@pytest.mark.parametrize("theta,tau_ref,n_gas", [(0.6, 0.05, 1 << 14), (0.75, 0.0, 1 << 13)])
def test_sub_bucket_parity(oracle_lib, theta, tau_ref, n_gas):
    from paper_1902_08083_gb300 import trevr
    P = workloads.sub_bucket_problem(n_gas=n_gas, n_src=64, seed=80)
    G = _gpu(P)
    T = _oracle(oracle_lib, P)
    f, c, st = trevr.compute_flux(G, theta, tau_ref, sub_bucket=1, counters=True, stats=True)
    sinks = workloads.sink_sample(n_gas, 300 if tau_ref > 0 else 80, seed=81)
    of, oc = T.flux_sub(theta, tau_ref, sinks=sinks, with_counters=True)
    assert oc[:, 4].sum() > 0
    assert_flux_parity(f.cpu().numpy()[sinks], of, f"sub-bucket theta={theta} tau_ref={tau_ref}")
    mism = np.nonzero(np.any(c.cpu().numpy()[sinks] != oc[:, :4].astype(np.int32), axis=1))[0]
    assert len(mism) <= 2
    assert st["sub_bucket_segments"] > 0
    # the trace differs from the cell means where buckets are mixed
    plain = trevr.compute_flux(G, theta, tau_ref).cpu().numpy()[sinks]
    assert np.max(np.abs(plain - of) / of) > 1e-3


def test_opaque_sink_does_not_shadow_itself_gpu():
    import torch
    from paper_1902_08083_gb300 import trevr
    rng = np.random.default_rng(82)
    n = 4000
    gas = np.minimum(rng.random((3, n)), workloads.ONE_BELOW).astype(np.float32)
    gas[:, 0] = (0.4987, 0.5013, 0.50071)
    a = np.zeros(n, np.float32)
    a[0] = 1e6
    src = rng.random((3, 16)).astype(np.float32)
    lum = np.ones(16, np.float32)
    w = np.full(n, 1.0 / n, np.float32)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    G = trevr.build_tree(t(gas), t(a), t(src), t(lum), weight=t(w))
    G.set_smoothing(t(np.full(n, 0.03, np.float32)))
    G0 = trevr.build_tree(t(gas), t(np.zeros_like(a)), t(src), t(lum), weight=t(w))
    free = trevr.compute_flux(G0, 0.0, 0.05).cpu().numpy()[0]
    traced = trevr.compute_flux(G, 0.0, 0.05, sub_bucket=1).cpu().numpy()[0]
    np.testing.assert_allclose(traced, free, rtol=1e-6)
    assert trevr.compute_flux(G, 0.0, 0.05).cpu().numpy()[0] < 1e-3 * free


def test_sub_bucket_argument_checks():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.sub_bucket_problem(n_gas=2000, n_src=8, seed=83)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    G = trevr.build_tree(t(P["gas_xyz"]), t(P["alpha"]), t(P["src_xyz"]), t(P["src_lum"]),
                         weight=t(P["weight"]))
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux(G, 0.75, 0.1, sub_bucket=1)  # no smoothing lengths yet
    bad = P["hsml"].copy()
    bad[5] = -1.0
    with pytest.raises(trevr.TrevrError):
        G.set_smoothing(t(bad))
    G.set_smoothing(t(P["hsml"]))
    trevr.compute_flux(G, 0.75, 0.1, sub_bucket=1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux(G, 0.75, 0.1, sub_bucket=1, tau_stop=3.0)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_moments(G, 0.75, 0.1, sub_bucket=1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_backward(G, torch.ones(2000, device="cuda"), 0.75, 0.1, sub_bucket=1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux(G, 0.75, 0.1, sub_bucket=2)
