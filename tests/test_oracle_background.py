"""Background radiation (Sec. 2.2.4): sources on a spiral sphere around the volume.

Pin: inside an optically thin shell of radius R and total luminosity L, the
angle-averaged intensity at radius r is L/(8 pi R r) ln((R+r)/(R-r)) (the integral of
L/(4 pi R^2) dA / (4 pi d^2) over the sphere; the printed Eq. cosmof lacks the 1/r and
is read with it, so that F -> L/(4 pi R^2) at the centre). The oracle's direct sum over
the spiral sources (theta = 0) converges to it; merging (theta > 0) over-estimates the
flux (merged centroids lie inside the sphere), and moving merged sources onto the
sphere, the paper's remedy, removes that bias."""
import numpy as np

import workloads


def shell_flux(r, R, L):
    r = np.asarray(r, np.float64)
    return L / (8 * np.pi * R * r) * np.log((R + r) / (R - r))


def test_spiral_is_on_the_sphere_and_balanced():
    pts = workloads.spiral_sphere(5000, 0.45)
    d = pts - 0.5
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), 0.45, rtol=1e-12)
    assert np.all(np.abs(d.mean(axis=1)) < 1e-3 * 0.45)  # no net dipole


def test_shell_formula_theta0(oracle_lib):
    P = workloads.background_shell(n_gas=3000, n_bg=20000, radius=0.45)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    sinks = np.nonzero(r < 0.35)[0][:400]
    f = T.flux(0.0, 0.1, sinks=sinks)
    ref = shell_flux(r[sinks], 0.45, 1.0)
    np.testing.assert_allclose(f, ref, rtol=2e-3)
    # near the centre the flux is flat at L / (4 pi R^2)
    c = sinks[r[sinks] < 0.05]
    np.testing.assert_allclose(T.flux(0.0, 0.1, sinks=c), 1.0 / (4 * np.pi * 0.45 ** 2), rtol=2e-3)


def test_merging_overestimates_near_the_shell(oracle_lib):
    P = workloads.background_shell(n_gas=3000, n_bg=20000, radius=0.45)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    outer = np.nonzero((r > 0.35) & (r < 0.4))[0][:200]
    f0 = T.flux(0.0, 0.1, sinks=outer)
    f1 = T.flux(0.75, 0.1, sinks=outer)
    assert np.mean(f1 / f0) > 1.0  # merged centroids sit inside the sphere, closer


def test_projection_moves_merged_sources_onto_the_sphere(oracle_lib):
    P = workloads.background_shell(n_gas=3000, n_bg=20000, radius=0.45)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    # theta = 0 merges nothing: the projection changes nothing
    s0 = np.arange(0, 3000, 11)
    np.testing.assert_array_equal(T.flux_background(0.0, 0.1, 0.45, sinks=s0),
                                  T.flux(0.0, 0.1, sinks=s0))
    for sink in (0, 777, 2999):
        I = T.interactions(sink, 0.75, 0.1, bg_radius=0.45)
        merged = I["src"] < 0
        assert merged.any()
        R32 = float(np.float32(0.45))  # the radius is an fp32 parameter
        np.testing.assert_allclose(np.linalg.norm(I["q"][merged] - 0.5, axis=1), R32, rtol=1e-12)
        p = P["gas_xyz"][:, sink].astype(np.float64)
        np.testing.assert_allclose(I["len_sum"], np.linalg.norm(I["q"] - p, axis=1), rtol=1e-12)
    # Sec. 2.2.4: merged centroids lie inside the sphere, nearer the sink, so plain
    # merging over-estimates the flux; moving them onto the sphere removes that bias
    inner = np.nonzero(r < 0.3)[0][:400]
    ref = shell_flux(r[inner], 0.45, 1.0)
    e_plain = np.mean(T.flux(0.75, 0.1, sinks=inner) / ref - 1)
    e_proj = np.mean(T.flux_background(0.75, 0.1, 0.45, sinks=inner) / ref - 1)
    assert e_plain > 0.005 and abs(e_proj) < 0.5 * e_plain


def test_projection_in_an_absorbing_medium(oracle_lib):
    # uniform absorption: the ray to a moved source still tiles exactly, so tau = alpha |q - p|
    P = workloads.background_shell(n_gas=2000, n_bg=5000, radius=0.45, alpha=3.0)
    T = oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], bucket=8)
    for sink in (1, 1000):
        I = T.interactions(sink, 0.6, 0.1, bg_radius=0.45)
        p = P["gas_xyz"][:, sink].astype(np.float64)
        np.testing.assert_allclose(I["tau"], 3.0 * np.linalg.norm(I["q"] - p, axis=1), rtol=1e-12)
