"""Pins for the oracle's flux vector (Eq. simpflux: sum f n, n the unit vector from the
source to the sink) and second moment (radiation pressure tensor sum f n n^T), the
'higher moments by simple summation' of Sec. 2.1.

Fixed by: the brute-force direct sums at theta=0 without absorption; the trace
identity tr(sum f n n^T) = sum f (n is a unit vector); the symmetric six-source
cross, whose vector flux vanishes at its centre and whose tensor is isotropic; and the
uniform-medium single source, whose vector is F (p - q)/|p - q| exactly."""
import numpy as np

import workloads


def test_direct_sums_theta0_no_absorption(oracle_lib):
    P = workloads.uniform_box(n_gas=1200, n_src=40, seed=70, alpha=0.0)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    sinks = np.arange(0, 1200, 7)
    F, V, M = T.flux_moments(0.0, 0.1, sinks=sinks)
    p = P["gas_xyz"][:, sinks].astype(np.float64).T[:, None, :]   # (n, 1, 3)
    y = P["src_xyz"].astype(np.float64).T[None, :, :]             # (1, s, 3)
    L = P["src_lum"].astype(np.float64)[None, :]
    d = p - y
    r = np.linalg.norm(d, axis=2)
    f = L / (4 * np.pi * r * r)
    n = d / r[:, :, None]
    np.testing.assert_allclose(F, f.sum(1), rtol=1e-12)
    np.testing.assert_allclose(V, (f[:, :, None] * n).sum(1), rtol=1e-10, atol=1e-12 * F.max())
    ref = np.stack([(f * n[:, :, a] * n[:, :, b]).sum(1)
                    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))], axis=1)
    np.testing.assert_allclose(M, ref, rtol=1e-10, atol=1e-12 * F.max())


def test_trace_and_bound(oracle_lib):
    P = workloads.uniform_box(n_gas=3000, n_src=120, seed=71)
    rng = np.random.default_rng(72)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, 1.5, 0.1, n_modes=64)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    F, V, M = T.flux_moments(0.7, 0.1)
    np.testing.assert_allclose(M[:, 0] + M[:, 1] + M[:, 2], F, rtol=1e-12)
    assert np.all(np.linalg.norm(V, axis=1) <= F * (1 + 1e-12))
    np.testing.assert_array_equal(F, T.flux(0.7, 0.1))  # the scalar is the same sum


def test_symmetric_cross_cancels(oracle_lib):
    # six equal sources at +-0.25 along each axis around a sink at the centre
    rng = np.random.default_rng(73)
    gas = rng.random((3, 500)).astype(np.float32)
    gas[:, 0] = 0.5
    src = np.array([[0.75, 0.25, 0.5, 0.5, 0.5, 0.5], [0.5, 0.5, 0.75, 0.25, 0.5, 0.5],
                    [0.5, 0.5, 0.5, 0.5, 0.75, 0.25]], np.float32)
    lum = np.full(6, 2.0, np.float32)
    T = oracle_lib.OracleTree(gas, np.full(500, 3.0, np.float32), src, lum, bucket=4)
    F, V, M = T.flux_moments(0.0, 0.1, sinks=np.array([0]))
    f1 = 2.0 * np.exp(-3.0 * 0.25) / (4 * np.pi * 0.25 ** 2)
    np.testing.assert_allclose(F[0], 6 * f1, rtol=1e-12)
    assert np.all(np.abs(V[0]) <= 1e-12 * F[0])
    np.testing.assert_allclose(M[0, :3], [2 * f1] * 3, rtol=1e-12)
    assert np.all(np.abs(M[0, 3:]) <= 1e-12 * F[0])
    # these rays run along cut planes (y = z = 1/2 ...): a ray lying in a face belongs
    # to the cell above it only, so at full refinement the segments are exactly the
    # leaves whose half-open boxes the ray crosses, each once
    I = T.interactions(0, 0.0, 0.0)
    np.testing.assert_allclose(I["len_sum"], 0.25, rtol=1e-14)
    N = T.nodes()
    leaf = np.nonzero(N["split_bit"] < 0)[0]
    lo = N["glo"][leaf] / 2.0 ** 21
    hi = N["ghi"][leaf] / 2.0 ** 21
    p = np.array([0.5, 0.5, 0.5])
    order = T.sources()["order"]  # sorted source -> caller index
    assert len(I["src"]) == 6
    for k in range(6):
        q = src[:, order[I["src"][k]]].astype(np.float64)
        axis = int(np.nonzero(q != p)[0][0])
        still = [a for a in range(3) if a != axis]
        inside = np.all((lo[:, still] <= 0.5) & (0.5 < hi[:, still]), axis=1)
        a0, a1 = min(p[axis], q[axis]), max(p[axis], q[axis])
        crosses = inside & (np.minimum(hi[:, axis], a1) > np.maximum(lo[:, axis], a0))
        assert I["nseg"][k] == np.count_nonzero(crosses)


def test_uniform_single_source_direction(oracle_lib):
    P = workloads.stromgren(n_gas=3000, seed=74)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    F, V, M = T.flux_moments(0.75, 0.1)
    d = P["gas_xyz"].astype(np.float64).T - 0.5
    r = np.linalg.norm(d, axis=1)
    np.testing.assert_allclose(V, F[:, None] * d / r[:, None], rtol=1e-12, atol=1e-14 * F.max())
