"""Pins for the oracle's adjoint (gradients of sum_p w_p log F_p with respect to the
source luminosities and the particle absorption coefficients, decisions frozen).

Fixed by: central finite differences of the replayed loss (the forward pass
re-evaluated with the recorded interactions and segment cells, a separate code
path that takes no derivatives); Euler's identity for the luminosities (F is
homogeneous of degree one in L once the decisions are frozen, so
sum_j L_j dF/dL_j = F); the linearity of tau in alpha (sum_i alpha_i dF/dalpha_i =
-sum_C f_C tau_C); and the uniform-medium closed form dF/dalpha = -r F.
"""
import numpy as np
import pytest

import workloads


def _problem(seed=40, n=3000, ns=60, sigma=1.0):
    P = workloads.uniform_box(n_gas=n, n_src=ns, seed=seed)
    rng = np.random.default_rng(seed + 1)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, sigma, 0.1, n_modes=64)
    return P


def _tree(oracle_lib, P):
    return oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"],
                                 bucket=P["bucket"], weight=P.get("weight"))


@pytest.mark.parametrize("theta,tau_ref,weighted", [(0.75, 0.1, False), (0.5, 0.0, False),
                                                   (0.75, 0.1, True)])
def test_adjoint_matches_replay_finite_differences(oracle_lib, theta, tau_ref, weighted):
    P = _problem()
    if weighted:  # volume weights w = m/rho enter d(abar)/d(alpha) = w_i / W_X
        P["weight"] = np.random.default_rng(7).uniform(0.2, 3.0, P["gas_xyz"].shape[1]).astype(
            np.float32)
    T = _tree(oracle_lib, P)
    n = P["gas_xyz"].shape[1]
    w = np.random.default_rng(5).standard_normal(n)
    F = T.flux(theta, tau_ref)
    gl, ga = T.adjoint(theta, tau_ref, w / F)
    R = T.replay(theta, tau_ref)
    assert abs(R.loss(w) - np.sum(w * np.log(F))) <= 1e-10 * np.sum(np.abs(w * np.log(F)))
    rng = np.random.default_rng(6)
    coords = [(0, j, float(P["src_lum"][j])) for j in rng.choice(P["src_xyz"].shape[1], 8,
                                                                   replace=False)]
    coords += [(1, i, float(P["alpha"][i])) for i in rng.choice(n, 8, replace=False)]
    for kind, idx, val in coords:
        ref = gl[idx] if kind == 0 else ga[idx]
        assert fd_agrees(R, w, kind, idx, val, ref), (kind, idx, ref)
        # with every segment's bounding planes frozen too the loss is analytic, so
        # the step of 1e-3 itself must agree: no retries at smaller steps
        h = 1e-3 * val
        fd = (R.loss(w, kind, idx, h, frozen_planes=True) -
              R.loss(w, kind, idx, -h, frozen_planes=True)) / (2 * h)
        assert abs(fd - ref) <= 1e-3 * abs(ref) + 1e-9, (kind, idx, fd, ref)


def fd_agrees(R, w, kind, idx, val, ref, rel=1e-3, tol=1e-3):
    """Central difference of the frozen-decision loss with step rel*val agrees with ref
    to tol (relative). That loss is piecewise smooth: a ray's entry or exit plane in a
    cell can switch inside the step (a kink). A step that fails must straddle such a
    switch (the replay counts them), and a smaller step (down to 1e-6) must agree."""
    for r in (rel, rel / 10, rel / 100, rel / 1000):
        h = r * val
        fd = (R.loss(w, kind, idx, h) - R.loss(w, kind, idx, -h)) / (2 * h)
        if abs(fd - ref) <= tol * abs(ref) + 1e-9:
            return True
        if R.kinks(kind, idx, h) == 0:
            return False  # no plane switch inside the step: a real disagreement
    return False


def test_replay_planes_and_kinks(oracle_lib):
    # the frozen-plane loss equals the re-clipped loss wherever no bounding plane
    # switches inside the step, and both equal the forward loss at h = 0
    P = _problem(seed=47, n=2000, ns=30)
    T = _tree(oracle_lib, P)
    n = P["gas_xyz"].shape[1]
    w = np.random.default_rng(2).standard_normal(n)
    R = T.replay(0.75, 0.1)
    base = R.loss(w)
    assert abs(R.loss(w, frozen_planes=True) - base) <= 1e-13 * abs(base)
    seen_kink = seen_clean = False
    for j in range(P["src_xyz"].shape[1]):
        for r in (1e-1, 1e-4):
            h = r * float(P["src_lum"][j])
            k = R.kinks(0, j, h)
            a, b = R.loss(w, 0, j, h), R.loss(w, 0, j, h, frozen_planes=True)
            if k == 0:
                seen_clean = True
                assert abs(a - b) <= 1e-12 * abs(base), (j, r)
            else:
                seen_kink = True
    assert seen_kink and seen_clean
    # an absorption coefficient moves no ray: no kinks, and both losses agree
    for i in (0, 77, 1999):
        h = 0.5 * float(P["alpha"][i])
        assert R.kinks(1, i, h) == 0
        assert abs(R.loss(w, 1, i, h) - R.loss(w, 1, i, h, frozen_planes=True)) <= 1e-13 * abs(base)


def test_adjoint_euler_identities(oracle_lib):
    P = _problem(seed=44, n=2500, ns=40)
    T = _tree(oracle_lib, P)
    n = P["gas_xyz"].shape[1]
    g = np.random.default_rng(9).standard_normal(n)
    F = T.flux(0.7, 0.1)
    gl, ga = T.adjoint(0.7, 0.1, g)
    # luminosities: sum_j L_j dLoss/dL_j = sum_p g_p F_p
    lhs = np.sum(P["src_lum"].astype(np.float64) * gl)
    rhs = np.sum(g * F)
    assert abs(lhs - rhs) <= 1e-9 * np.sum(np.abs(g * F))
    # absorption: sum_i alpha_i dLoss/dalpha_i = -sum_p g_p sum_C f_C tau_C
    lhs = np.sum(P["alpha"].astype(np.float64) * ga)
    rhs = 0.0
    for p in range(n):
        I = T.interactions(p, 0.7, 0.1)
        rhs -= g[p] * np.sum(I["flux"] * I["tau"])
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))


def test_adjoint_uniform_closed_form(oracle_lib):
    # one source (L=1) in a uniform medium alpha=20: F = exp(-20 r)/(4 pi r^2), so
    # dF/dL = F and the total derivative along alpha -> alpha + h (all particles)
    # is dF/dalpha = -r F
    P = workloads.stromgren(n_gas=3000, seed=3)
    T = _tree(oracle_lib, P)
    n = P["gas_xyz"].shape[1]
    for p in (0, 1234, 2999):
        g = np.zeros(n)
        g[p] = 1.0
        gl, ga = T.adjoint(0.75, 0.1, g)
        r = np.linalg.norm(P["gas_xyz"][:, p].astype(np.float64) - 0.5)
        Fp = np.exp(-20 * r) / (4 * np.pi * r * r)
        assert abs(gl[0] - Fp) <= 1e-10 * Fp
        assert abs(ga.sum() - (-r * Fp)) <= 1e-9 * r * Fp
