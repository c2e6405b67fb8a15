"""Pins for the oracle's top-down ray walk (Sec. 3.1.3, last paragraph of "Refinement
Criterion"; Sec. 4, Discussion): the ray starts as one segment in the lowest common
ancestor of the sink's bucket and the source cell, and the refinement criterion
(Eq. refcrit) alone splits it.

Fixed by: the tiling of the ray by its segments; the brute-force cell-by-cell optical
depth at tau_ref <= 0 (full refinement, where both walks reach the buckets); the
uniform-medium closed form with exactly one segment per ray (no cell has any spread
of absorption, so nothing refines); one segment per ray when tau_ref never refines;
the source walk, which the ray walk does not touch; the segment set being a
coarsening of the bottom-up walk's; the paper's accuracy statement that the RMS
error stays below tau_ref; and the shadow behind an opaque occluder.
"""
import numpy as np
import pytest

import workloads
from test_oracle_flux import _clip_all, _leaf_boxes, _tree


def _lognormal(seed, n=4000, ns=60, sigma=1.5, corr=0.1):
    P = workloads.uniform_box(n_gas=n, n_src=ns, seed=seed)
    rng = np.random.default_rng(seed + 1)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, sigma, corr, n_modes=64)
    return P


@pytest.mark.parametrize("tau_ref", [0.0, 0.05, 1e6])
def test_topdown_segments_tile_the_ray(oracle_lib, tau_ref):
    P = _lognormal(12)
    T = _tree(oracle_lib, P)
    for sink in (5, 1234, 3999):
        I = T.interactions(sink, 0.75, tau_ref)
        p = P["gas_xyz"][:, sink].astype(np.float64)
        for k in range(len(I["node"])):
            q = I["q"][k].astype(np.float32)
            tau, ls, ns = T.ray_tau(sink, I["node"][k], q, tau_ref, topdown=True)
            assert abs(ls - np.linalg.norm(q.astype(np.float64) - p)) <= 1e-12 * max(1.0, ls)
            assert ns >= 1 and tau >= 0.0


@pytest.mark.parametrize("theta", [0.0, 0.6])
def test_topdown_full_refinement_is_cell_by_cell(oracle_lib, theta):
    P = _lognormal(8, n=3000, ns=40)
    T = _tree(oracle_lib, P)
    lo, hi, abar = _leaf_boxes(T)
    for sink in (0, 17, 999, 2998):
        I = T.interactions(sink, theta, 0.0)
        p = P["gas_xyz"][:, sink].astype(np.float64)
        for k in range(len(I["tau"])):
            q = I["q"][k].astype(np.float32)
            tau, _, _ = T.ray_tau(sink, I["node"][k], q, 0.0, topdown=True)
            tau_bf = float(np.sum(abar * _clip_all(lo, hi, p, q.astype(np.float64))))
            assert abs(tau - tau_bf) <= 1e-9 * max(1.0, tau_bf)


@pytest.mark.parametrize("theta,tau_ref", [(0.3, 0.01), (0.75, 0.1), (1.0, 0.5)])
def test_topdown_uniform_medium_one_segment_per_ray(oracle_lib, theta, tau_ref):
    # one source of L=1 at the centre, alpha=20: F = exp(-20 r) / (4 pi r^2), and no
    # cell has a spread of absorption, so every ray is the single segment A
    P = workloads.stromgren(n_gas=4096, seed=1, theta=theta, tau_ref=tau_ref)
    T = _tree(oracle_lib, P)
    f, cnt = T.flux_topdown(theta, tau_ref, with_counters=True)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    np.testing.assert_allclose(f, np.exp(-20.0 * r) / (4 * np.pi * r * r), rtol=1e-12)
    assert np.all(cnt[:, 0] == 1) and np.all(cnt[:, 1] == 1) and np.all(cnt[:, 3] == 0)


def test_topdown_never_refining_is_one_segment_per_ray(oracle_lib):
    P = _lognormal(3, sigma=2.0)
    T = _tree(oracle_lib, P)
    sinks = np.arange(0, 4000, 37)
    _, cnt = T.flux_topdown(0.75, 1e6, sinks=sinks, with_counters=True)
    assert np.all(cnt[:, 1] == cnt[:, 0]) and np.all(cnt[:, 3] == 0)


@pytest.mark.parametrize("tau_ref", [0.0, 0.03, 0.1, 1.0])
def test_topdown_coarsens_the_bottom_up_walk(oracle_lib, tau_ref):
    # the source walk is unchanged; the top-down segments are unions of bottom-up
    # segments, so no ray has more of them (equal at full refinement)
    P = _lognormal(21, sigma=2.0)
    T = _tree(oracle_lib, P)
    sinks = np.arange(0, 4000, 7)
    fb, cb, _ = T.flux(0.75, tau_ref, sinks=sinks, with_counters=True)
    ft, ct = T.flux_topdown(0.75, tau_ref, sinks=sinks, with_counters=True)
    np.testing.assert_array_equal(ct[:, 0], cb[:, 0])  # interactions
    np.testing.assert_array_equal(ct[:, 2], cb[:, 2])  # source cells visited
    assert np.all(ct[:, 1] <= cb[:, 1])
    if tau_ref <= 0.0:
        np.testing.assert_array_equal(ct[:, 1], cb[:, 1])
        np.testing.assert_allclose(ft, fb, rtol=1e-12)
    else:
        assert ct[:, 1].sum() < cb[:, 1].sum()


def test_topdown_error_below_tau_ref(oracle_lib):
    # Sec. 3.1.3 / Eq. reffrac: the RMS fractional error against a fully refined
    # reference lies below tau_ref, and tightening tau_ref costs more segments
    P = _lognormal(13, n=6000, ns=200, sigma=2.0, corr=0.05)
    T = _tree(oracle_lib, P)
    sinks = np.arange(0, 6000, 10)
    ref = T.flux_topdown(0.75, 1e-8, sinks=sinks)
    prev = None
    for tau_ref in (1.0, 0.3, 0.1, 0.03):
        f, cnt = T.flux_topdown(0.75, tau_ref, sinks=sinks, with_counters=True)
        rms = np.sqrt(np.mean(((f - ref) / ref) ** 2))
        assert rms <= tau_ref
        if prev is not None:
            assert cnt[:, 1].sum() >= prev
        prev = cnt[:, 1].sum()


def test_topdown_shadow_behind_occluder(oracle_lib):
    rng = np.random.default_rng(30)
    n = 20000
    gas = rng.random((3, n)).astype(np.float32)
    alpha = np.ones(n, np.float32)
    inside = np.all((gas >= 0.45) & (gas <= 0.55), axis=0)
    alpha[inside] *= 1e3
    src = np.array([[0.2], [0.5], [0.5]], np.float32)
    lum = np.ones(1, np.float32)
    T = oracle_lib.OracleTree(gas, alpha, src, lum, bucket=8)
    T0 = oracle_lib.OracleTree(gas, np.ones(n, np.float32), src, lum, bucket=8)
    behind = np.nonzero((gas[0] > 0.65) & (gas[0] < 0.9) & (np.abs(gas[1] - 0.5) < 0.02)
                        & (np.abs(gas[2] - 0.5) < 0.02))[0]
    assert len(behind) > 5
    f = T.flux_topdown(0.75, 0.1, sinks=behind)
    f0 = T0.flux_topdown(0.75, 0.1, sinks=behind)
    assert np.all(f <= np.exp(-30.0) * f0)


def test_topdown_starts_at_the_common_ancestor(oracle_lib):
    # with refinement off the single segment is A, the lowest common ancestor of the
    # sink's leaf S and the source cell C: tau = abar_A |q - p|
    P = _lognormal(5, sigma=2.0)
    T = _tree(oracle_lib, P)
    N = T.nodes()
    parent, depth = N["parent"], N["depth"]
    leaf_of = T.particles()["leaf_of"]
    rank = np.argsort(T.particles()["perm"])
    for sink in (1, 2020, 3777):
        I = T.interactions(sink, 0.75, 1e6)
        p = P["gas_xyz"][:, sink].astype(np.float64)
        for k in range(len(I["node"])):
            u, v = leaf_of[rank[sink]], I["node"][k]
            while depth[u] > depth[v]:
                u = parent[u]
            while depth[v] > depth[u]:
                v = parent[v]
            while u != v:
                u, v = parent[u], parent[v]
            q = I["q"][k].astype(np.float32)
            tau, _, ns = T.ray_tau(sink, I["node"][k], q, 1e6, topdown=True)
            assert ns == 1
            expect = N["abar"][u] * np.linalg.norm(q.astype(np.float64) - p)
            assert abs(tau - expect) <= 1e-12 * max(1.0, expect)
