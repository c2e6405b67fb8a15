"""Several bands on the GPU (Sec. 4): the bands share the walk and the rays, each
band sums its own optical depth, and a cell refines when any band asks. GPU vs the
oracle's band flux per band, with the counters of the shared walk; one band equal
to the plain flux; proportional bands equal to scaled copies of the plain flux."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity

pytestmark = pytest.mark.gpu


def _problem(n_bands, n_gas=1 << 15, n_src=400, seed=60):
    P = workloads.uniform_box(n_gas=n_gas, n_src=n_src, seed=seed)
    rng = np.random.default_rng(seed + 1)
    A = np.stack([workloads.lognormal_alpha(rng, P["gas_xyz"], 3.0 / (b + 1), 1.0 + 0.5 * b,
                                            0.05 + 0.05 * b) for b in range(n_bands)])
    Lb = np.stack([rng.lognormal(0.0, 1.0, n_src) for _ in range(n_bands)]).astype(np.float32)
    return P, A, Lb


def _gpu(P, A, Lb):
    import torch
    from paper_1902_08083_gb300 import trevr
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return trevr.build_tree(t(P["gas_xyz"]), t(A), t(P["src_xyz"]), t(Lb), bucket=P["bucket"])


def _oracle(oracle_lib, P, A, Lb):
    return oracle_lib.OracleTree(P["gas_xyz"], A, P["src_xyz"], Lb, bucket=P["bucket"])


@pytest.mark.parametrize("n_bands", [2, 3, 4])
def test_bands_parity(oracle_lib, n_bands):
    from paper_1902_08083_gb300 import trevr
    P, A, Lb = _problem(n_bands)
    G = _gpu(P, A, Lb)
    T = _oracle(oracle_lib, P, A, Lb)
    f, c = trevr.compute_flux_bands(G, 0.6, 0.1, counters=True)
    sinks = workloads.sink_sample(1 << 15, 1500, seed=62)
    of, oc = T.flux_bands(0.6, 0.1, sinks=sinks, with_counters=True)
    f = f.cpu().numpy()
    for b in range(n_bands):
        assert_flux_parity(f[b, sinks], of[b], f"band {b} of {n_bands}")
    mism = np.nonzero(np.any(c.cpu().numpy()[sinks] != oc.astype(np.int32), axis=1))[0]
    assert len(mism) <= 2


def test_sink_list_and_zero_sinks(oracle_lib):
    import torch
    from paper_1902_08083_gb300 import trevr
    P, A, Lb = _problem(3, n_gas=6000, n_src=100, seed=63)
    G = _gpu(P, A, Lb)
    T = _oracle(oracle_lib, P, A, Lb)
    sinks = workloads.sink_sample(6000, 777, seed=64)
    f = trevr.compute_flux_bands(G, 0.75, 0.1, sink_idx=torch.from_numpy(sinks).cuda())
    of = T.flux_bands(0.75, 0.1, sinks=sinks)
    for b in range(3):
        assert_flux_parity(f.cpu().numpy()[b], of[b], f"band {b}, sink list")
    e = trevr.compute_flux_bands(G, 0.75, 0.1, sink_idx=torch.empty(0, dtype=torch.int64,
                                                                     device="cuda"))
    assert tuple(e.shape) == (3, 0)


def test_one_band_and_proportional_bands_match_the_plain_flux():
    import torch
    from paper_1902_08083_gb300 import trevr
    P, A, Lb = _problem(1, seed=65)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plain = trevr.build_tree(t(P["gas_xyz"]), t(A[0]), t(P["src_xyz"]), t(Lb[0]))
    F = trevr.compute_flux(plain, 0.6, 0.1).cpu().numpy()
    one = _gpu(P, A, Lb)
    np.testing.assert_array_equal(trevr.compute_flux_bands(one, 0.6, 0.1).cpu().numpy()[0], F)
    # luminosity factors that are powers of two with a sum of one: the summed light,
    # every decision and every ray are the plain ones, and band b is c_b times the flux
    c = np.array([0.5, 0.25, 0.125, 0.125], np.float32)
    G = _gpu(P, np.stack([A[0]] * 4), (c[:, None] * Lb[0][None, :]).astype(np.float32))
    fb = trevr.compute_flux_bands(G, 0.6, 0.1).cpu().numpy()
    for b in range(4):
        np.testing.assert_allclose(fb[b], c[b] * F, rtol=1e-6)


def test_band_trees_only_for_the_band_flux():
    import torch
    from paper_1902_08083_gb300 import trevr
    P, A, Lb = _problem(2, n_gas=3000, n_src=50, seed=66)
    G = _gpu(P, A, Lb)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux(G, 0.75, 0.1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_moments(G, 0.75, 0.1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_backward(G, torch.ones(3000, device="cuda"), 0.75, 0.1)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_bands(G, 0.75, 0.1, tau_stop=2.0)
    with pytest.raises(trevr.TrevrError):
        trevr.Batch([G])
    bad = Lb.copy()
    bad[1, 7] = -1.0
    with pytest.raises(trevr.TrevrError):
        _gpu(P, A, bad)
    badA = A.copy()
    badA[1, 11] = np.nan
    with pytest.raises(trevr.TrevrError):
        _gpu(P, badA, Lb)
