"""Several bands (Sec. 4: many bands for a constant factor in cost). Reading: the
bands share the walk and the rays. The tree's centres of luminosity come from the
band-summed luminosity. A cell is refined when any band asks for it, and each band
sums its own optical depth along the shared segments.

Pins:
- one band is the plain method, bit for bit;
- bands with proportional luminosities and equal absorption are scaled copies of
  the plain flux;
- at full refinement (tau_ref = 0) each band is the plain flux of its own field;
- with a transparent second band, band 0 is the plain flux of its field and band 1
  the unabsorbed flux;
- the shared refinement is at least as fine as each band's own.

The luminosity factors are powers of two, so the scaled luminosities, their sums and
the centres of luminosity are exact in fp32 and the decisions cannot move."""
import numpy as np
import pytest

import workloads

C = np.array([0.5, 0.25, 0.25])


def _base(seed=50, n_gas=3000, n_src=200):
    P = workloads.uniform_box(n_gas=n_gas, n_src=n_src, seed=seed)
    rng = np.random.default_rng(seed + 1)
    a0 = workloads.lognormal_alpha(rng, P["gas_xyz"], 3.0, 1.5, 0.08)
    a1 = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, 2.0, 0.05)
    a2 = workloads.lognormal_alpha(rng, P["gas_xyz"], 6.0, 0.5, 0.2)
    return P, np.stack([a0, a1, a2])


def _tree(oracle_lib, P, alpha, lum):
    return oracle_lib.OracleTree(P["gas_xyz"], alpha, P["src_xyz"], lum, bucket=P["bucket"])


def test_one_band_is_the_plain_method(oracle_lib):
    P, A = _base()
    T1 = _tree(oracle_lib, P, A[:1], P["src_lum"][None, :])
    T = _tree(oracle_lib, P, A[0], P["src_lum"])
    sinks = workloads.sink_sample(3000, 200, seed=52)
    fb, cb = T1.flux_bands(0.6, 0.1, sinks=sinks, with_counters=True)
    f, c, _ = T.flux(0.6, 0.1, sinks=sinks, with_counters=True)
    np.testing.assert_array_equal(fb[0], f)
    np.testing.assert_array_equal(cb, c)


def test_proportional_bands_scale_the_plain_flux(oracle_lib):
    P, A = _base()
    lum = (C[:, None] * P["src_lum"][None, :]).astype(np.float32)
    TB = _tree(oracle_lib, P, np.stack([A[0]] * 3), lum)
    T = _tree(oracle_lib, P, A[0], P["src_lum"])
    sinks = workloads.sink_sample(3000, 200, seed=53)
    fb, cb = TB.flux_bands(0.6, 0.1, sinks=sinks, with_counters=True)
    f, c, _ = T.flux(0.6, 0.1, sinks=sinks, with_counters=True)
    for b in range(3):
        np.testing.assert_allclose(fb[b], C[b] * f, rtol=1e-13)
    np.testing.assert_array_equal(cb, c)


def test_full_refinement_gives_each_band_its_own_field(oracle_lib):
    P, A = _base(n_gas=2000, n_src=100)
    lum = (C[:, None] * P["src_lum"][None, :]).astype(np.float32)
    TB = _tree(oracle_lib, P, A, lum)
    sinks = workloads.sink_sample(2000, 120, seed=54)
    fb = TB.flux_bands(0.75, 0.0, sinks=sinks)
    for b in range(3):
        Tb = _tree(oracle_lib, P, A[b], P["src_lum"])
        np.testing.assert_allclose(fb[b], C[b] * Tb.flux(0.75, 0.0, sinks=sinks), rtol=1e-12)


def test_transparent_band(oracle_lib):
    P, A = _base()
    lum = np.stack([0.5 * P["src_lum"], 0.5 * P["src_lum"]]).astype(np.float32)
    TB = _tree(oracle_lib, P, np.stack([A[0], np.zeros_like(A[0])]), lum)
    T = _tree(oracle_lib, P, A[0], P["src_lum"])
    T0 = _tree(oracle_lib, P, np.zeros_like(A[0]), P["src_lum"])
    sinks = workloads.sink_sample(3000, 200, seed=55)
    fb, cb = TB.flux_bands(0.6, 0.1, sinks=sinks, with_counters=True)
    f, c, _ = T.flux(0.6, 0.1, sinks=sinks, with_counters=True)
    np.testing.assert_allclose(fb[0], 0.5 * f, rtol=1e-13)
    np.testing.assert_allclose(fb[1], 0.5 * T0.flux(0.6, 0.1, sinks=sinks), rtol=1e-12)
    np.testing.assert_array_equal(cb, c)


def test_shared_refinement_is_the_finest(oracle_lib):
    P, A = _base()
    lum = (C[:, None] * P["src_lum"][None, :]).astype(np.float32)
    TB = _tree(oracle_lib, P, A, lum)
    sinks = workloads.sink_sample(3000, 200, seed=56)
    _, cb = TB.flux_bands(0.6, 0.1, sinks=sinks, with_counters=True)
    finer = np.zeros(len(sinks), bool)
    for b in range(3):
        Tb = _tree(oracle_lib, P, A[b], P["src_lum"])
        _, c, _ = Tb.flux(0.6, 0.1, sinks=sinks, with_counters=True)
        assert np.all(cb[:, 1] >= c[:, 1]) and np.all(cb[:, 3] >= c[:, 3])
        np.testing.assert_array_equal(cb[:, 0], c[:, 0])  # same walk
        finer |= cb[:, 1] > c[:, 1]
    assert finer.any()


def test_band_trees_reject_the_single_band_calls(oracle_lib):
    P, A = _base(n_gas=500, n_src=20)
    lum = np.stack([P["src_lum"], P["src_lum"]])
    TB = _tree(oracle_lib, P, A[:2], lum)
    with pytest.raises(oracle_lib.OracleError):
        TB.flux(0.75, 0.1)
    with pytest.raises(oracle_lib.OracleError):
        _tree(oracle_lib, P, np.zeros((9, 500), np.float32), np.ones((9, 20), np.float32))
