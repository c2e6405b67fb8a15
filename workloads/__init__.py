"""Seeded synthetic inputs for the TREVR hot path.

This module holds no arithmetic of the method itself: it only draws particle
positions, absorption coefficients and source luminosities. Both the FP64
oracle and the CUDA library are fed from here, so the two always see the same
fp32 inputs. Every array is generated in FP64 by ``numpy.random.default_rng``
and cast to fp32; positions lie in the unit cube [0, 1)^3.

The workloads stand in for the paper's tests (Sec. 3): the paper's glass
initial conditions are not available, so uniform random particles with a
lognormal absorption field replace them.
"""
from __future__ import annotations

import os

import numpy as np

ONE_BELOW = np.nextafter(np.float32(1.0), np.float32(0.0))


def _unit_positions(rng, n):
    x = rng.random((3, n)).astype(np.float32)
    return np.minimum(x, ONE_BELOW)


def gaussian_field(rng, xyz, corr_len, n_modes=512, chunk=1 << 16):
    """Unit-variance Gaussian random field g(x) = sqrt(2/M) sum_m cos(k_m.x + phi_m),
    k_m ~ N(0, corr_len^-2 I), phi_m ~ U[0, 2pi), evaluated at the points xyz (3, N)."""
    k = rng.normal(0.0, 1.0 / corr_len, size=(n_modes, 3))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    n = xyz.shape[1]
    g = np.empty(n, dtype=np.float64)
    pts = xyz.astype(np.float64)
    amp = np.sqrt(2.0 / n_modes)
    for s in range(0, n, chunk):
        arg = pts[:, s:s + chunk].T @ k.T + phi
        g[s:s + chunk] = amp * np.cos(arg).sum(axis=1)
    return g


def lognormal_alpha(rng, xyz, alpha0, sigma, corr_len, n_modes=512):
    """alpha_i = alpha0 * exp(sigma g(x_i) - sigma^2/2): lognormal with mean alpha0."""
    g = gaussian_field(rng, xyz, corr_len, n_modes)
    return (alpha0 * np.exp(sigma * g - 0.5 * sigma * sigma)).astype(np.float32)


def _problem(name, gas_xyz, alpha, src_xyz, src_lum, theta, tau_ref, bucket=8, weight=None,
             seed=None, **extra):
    d = dict(name=name, gas_xyz=np.ascontiguousarray(gas_xyz, dtype=np.float32),
             alpha=np.ascontiguousarray(alpha, dtype=np.float32),
             weight=None if weight is None else np.ascontiguousarray(weight, np.float32),
             src_xyz=np.ascontiguousarray(np.asarray(src_xyz, np.float32).reshape(3, -1)),
             src_lum=np.ascontiguousarray(src_lum, dtype=np.float32), lo=(0.0, 0.0, 0.0),
             side=1.0, theta=float(theta), tau_ref=float(tau_ref), bucket=int(bucket), seed=seed)
    d.update(extra)
    return d


def uniform_box(n_gas=4096, n_src=64, seed=0, alpha=1.0, theta=0.75, tau_ref=0.1, bucket=8):
    """Uniform random gas and sources, uniform absorption (tau across the box = alpha),
    lognormal(0, 1) luminosities. Default: 4096 gas / 64 sources."""
    rng = np.random.default_rng(seed)
    gas = _unit_positions(rng, n_gas)
    src = _unit_positions(rng, n_src)
    lum = rng.lognormal(0.0, 1.0, n_src).astype(np.float32)
    a = np.full(n_gas, alpha, dtype=np.float32)
    return _problem(f"uniform_{n_gas}_{n_src}", gas, a, src, lum, theta, tau_ref, bucket,
                    seed=seed)


def stromgren(n_gas=1 << 18, seed=1, alpha=20.0, theta=0.75, tau_ref=0.1, bucket=8):
    """Stromgren-like test: one source of L=1 at the centre of a uniform medium
    with alpha=20 (tau=10 from the centre to a face)."""
    rng = np.random.default_rng(seed)
    gas = _unit_positions(rng, n_gas)
    src = np.full((3, 1), 0.5, dtype=np.float32)
    lum = np.ones(1, dtype=np.float32)
    a = np.full(n_gas, alpha, dtype=np.float32)
    return _problem(f"stromgren_{n_gas}", gas, a, src, lum, theta, tau_ref, bucket, seed=seed)


def clumpy(n_gas=1 << 22, n_src=1 << 14, n_clumps=16, seed=2, sigma=2.0, corr_len=0.05,
           alpha0=1.0, occluder=(0.45, 0.55), occluder_factor=1e3, clump_width=0.02,
           theta=0.6, tau_ref=0.1, bucket=8, n_modes=512):
    """Clumpy medium with a shadow: lognormal absorption (sigma_ln=2, correlation length
    0.05), a dense cube occluder (x1e3) over [0.45, 0.55]^3, sources in Gaussian clumps."""
    rng = np.random.default_rng(seed)
    gas = _unit_positions(rng, n_gas)
    a = lognormal_alpha(rng, gas, alpha0, sigma, corr_len, n_modes)
    lo, hi = occluder
    inside = np.all((gas >= lo) & (gas <= hi), axis=0)
    a[inside] *= np.float32(occluder_factor)
    centres = rng.uniform(0.1, 0.9, size=(n_clumps, 3))
    per = n_src // n_clumps
    pts = []
    for c in range(n_clumps):
        m = per if c < n_clumps - 1 else n_src - per * (n_clumps - 1)
        pts.append(centres[c][:, None] + clump_width * rng.standard_normal((3, m)))
    src = np.clip(np.concatenate(pts, axis=1), 0.0, 1.0).astype(np.float32)
    src = np.minimum(src, ONE_BELOW)
    lum = rng.lognormal(0.0, 1.0, n_src).astype(np.float32)
    return _problem(f"clumpy_{n_gas}_{n_src}", gas, a, src, lum, theta, tau_ref, bucket,
                    seed=seed)


def far_domain(n_gas=1 << 20, n_src=1024, seed=10, lo=(1000.0, 1000.0, 1000.0), side=1.0,
               clump_frac=0.0, clump_width=3e-4, sigma=1.0, corr_len=0.05, theta=0.75,
               tau_ref=0.1, bucket=8, n_modes=256):
    """A domain far from the origin: gas and sources uniform in [lo, lo + side)^3 (fp32),
    a fraction clump_frac of the gas in a Gaussian clump of the given width (in units of
    side) at the domain's centre, a lognormal absorption field (sigma_ln = sigma, given
    in the domain's unit coordinates) and lognormal(0, 1) luminosities."""
    rng = np.random.default_rng(seed)
    u = rng.random((3, n_gas))
    m = int(clump_frac * n_gas)
    if m:
        u[:, :m] = np.clip(0.5 + clump_width * rng.standard_normal((3, m)), 0.0, 1.0)
    us = rng.random((3, n_src))
    lo32 = np.asarray(lo, np.float32)[:, None]
    side32 = np.float32(side)
    hi32 = (lo32 + side32).astype(np.float32)

    def place(v):
        x = (lo32 + (v * float(side32)).astype(np.float32)).astype(np.float32)
        x = np.maximum(x, lo32)
        return np.minimum(x, np.nextafter(hi32, np.float32(-np.inf))).astype(np.float32)

    gas, src = place(u), place(us)
    a = lognormal_alpha(rng, u.astype(np.float32), 1.0, sigma, corr_len, n_modes)
    lum = rng.lognormal(0.0, 1.0, n_src).astype(np.float32)
    P = _problem(f"far_{n_gas}_{n_src}", gas, a, src, lum, theta, tau_ref, bucket, seed=seed)
    P["lo"], P["side"] = tuple(float(v) for v in lo32[:, 0]), float(side32)
    return P


def batched_boxes(n_boxes=64, seed=3, lo_exp=12, hi_exp=17, theta=0.75, tau_ref=0.1, bucket=8,
                  n_modes=512):
    """Independent boxes with log-uniform particle counts in [2^12, 2^17], N/64 sources
    each; even boxes uniform alpha=1, odd boxes a lognormal field (sigma_ln=1)."""
    rng = np.random.default_rng(seed)
    counts = np.floor(2.0 ** rng.uniform(lo_exp, hi_exp, n_boxes)).astype(np.int64)
    boxes = []
    for b in range(n_boxes):
        n = int(counts[b])
        s = max(1, n // 64)
        gas = _unit_positions(rng, n)
        if b % 2 == 0:
            a = np.ones(n, dtype=np.float32)
        else:
            a = lognormal_alpha(rng, gas, 1.0, 1.0, 0.05, n_modes)
        src = _unit_positions(rng, s)
        lum = rng.lognormal(0.0, 1.0, s).astype(np.float32)
        boxes.append(_problem(f"box{b}_{n}", gas, a, src, lum, theta, tau_ref, bucket,
                              seed=seed))
    return boxes


def adjoint_problem(n_gas=1 << 21, n_src=1024, seed=4, sigma=1.0, corr_len=0.05, theta=0.75,
                    tau_ref=0.1, bucket=8, loss_seed=5, fd_seed=6, n_fd=64, n_modes=512):
    """Differentiation workload: lognormal absorption (sigma_ln=1), uniform sources with
    lognormal luminosities; loss weights w_i ~ N(0, 1); 64 finite-difference coordinates
    (half luminosities, half absorption coefficients)."""
    rng = np.random.default_rng(seed)
    gas = _unit_positions(rng, n_gas)
    a = lognormal_alpha(rng, gas, 1.0, sigma, corr_len, n_modes)
    src = _unit_positions(rng, n_src)
    lum = rng.lognormal(0.0, 1.0, n_src).astype(np.float32)
    lw = np.random.default_rng(loss_seed).standard_normal(n_gas).astype(np.float32)
    frng = np.random.default_rng(fd_seed)
    fd_src = frng.choice(n_src, size=n_fd // 2, replace=False)
    fd_gas = frng.choice(n_gas, size=n_fd - n_fd // 2, replace=False)
    return _problem(f"adjoint_{n_gas}_{n_src}", gas, a, src, lum, theta, tau_ref, bucket,
                    seed=seed, loss_weight=lw, fd_src=fd_src, fd_gas=fd_gas)


def spiral_sphere(n, radius, centre=(0.5, 0.5, 0.5)):
    """n points spread over a sphere along a golden-angle spiral (equal-area bands in z,
    azimuth advancing by pi (3 - sqrt 5) per point): the background-source layout."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    u = np.stack([rho * np.cos(phi), rho * np.sin(phi), z])
    return np.asarray(centre, np.float64)[:, None] + radius * u


def background_shell(n_gas=1 << 14, n_bg=20000, radius=0.45, l_total=1.0, seed=9, alpha=0.0,
                     theta=0.75, tau_ref=0.1, bucket=8):
    """Background radiation: n_bg equal sources on a spiral sphere of the given radius
    around the box centre (total luminosity l_total), gas uniform inside the sphere."""
    rng = np.random.default_rng(seed)
    # gas uniform in the ball of radius 0.95 * radius (rejection sampling)
    pts = []
    need = n_gas
    while need > 0:
        c = rng.random((3, 2 * need)) - 0.5
        keep = np.sum(c * c, axis=0) < (0.95 * radius) ** 2
        pts.append(c[:, keep][:, :need])
        need -= pts[-1].shape[1]
    gas = (np.concatenate(pts, axis=1) + 0.5).astype(np.float32)
    src = spiral_sphere(n_bg, radius).astype(np.float32)
    lum = np.full(n_bg, l_total / n_bg, dtype=np.float32)
    a = np.full(n_gas, alpha, dtype=np.float32)
    return _problem(f"background_{n_gas}_{n_bg}", gas, a, src, lum, theta, tau_ref, bucket,
                    seed=seed, radius=radius, l_total=l_total)


def knn_smoothing(xyz, k=32):
    """SPH-style smoothing lengths: h_j = half the distance from particle j to its k-th
    nearest neighbour, so that the kernel support 2h holds about k particles."""
    from scipy.spatial import cKDTree
    pts = np.asarray(xyz, np.float64).T
    d, _ = cKDTree(pts).query(pts, k=k + 1)
    return (0.5 * d[:, -1]).astype(np.float32)


def sub_bucket_problem(n_gas=1 << 12, n_src=32, seed=11, alpha0=2.0, sigma=1.5, k=32,
                       theta=0.6, tau_ref=0.05, bucket=8):
    """Sub-bucket particle trace test: uniform particles of equal volume 1/N (the
    weights m/rho), lognormal absorption (sigma_ln=1.5, correlation length 0.05) so
    that buckets hold very different particles, smoothing lengths from the 32nd
    neighbour, uniform sources."""
    rng = np.random.default_rng(seed)
    gas = _unit_positions(rng, n_gas)
    a = lognormal_alpha(rng, gas, alpha0, sigma, 0.05)
    src = _unit_positions(rng, n_src)
    lum = rng.lognormal(0.0, 1.0, n_src).astype(np.float32)
    w = np.full(n_gas, 1.0 / n_gas, dtype=np.float32)
    return _problem(f"subbucket_{n_gas}_{n_src}", gas, a, src, lum, theta, tau_ref, bucket,
                    weight=w, seed=seed, hsml=knn_smoothing(gas, k))


_GLASS_MODES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "glass_modes.txt")


def glass_modes():
    """The 24 (k_x, k_y, k_z, phi) modes of the perturbed glass (Appendix A, Table
    "modes" of the paper), shape (24, 4)."""
    return np.loadtxt(_GLASS_MODES, comments="#")[:, 1:]


def perturbed_glass(n_side=64, seed=13, jitter=0.25, k=32, theta=0.75, tau_ref=0.1, bucket=8):
    """Stand-in for the sinusoidally perturbed glass of the accuracy tests (Sec. 3.1.1,
    Appendix A). The glass file is not available, so a cubic lattice of n_side^3
    points with seeded uniform jitter of +-jitter spacings replaces it. Each point
    moves by (1/275) sin(k_i . r0 + phi_i) along the unit vector of k_i for each of
    the 24 tabulated modes, and wraps into the unit box (the printed Eq. manfft adds
    a scalar to a vector; this is its reading). The stars are the gas points with
    their coordinates cycled (x_s = y_g, y_s = z_g, z_s = x_g), each of luminosity 1.
    The gas has total mass 1 and opacity 1, so alpha = rho, with the density from the
    distance to the k-th neighbour, rho_i = k m / ((4/3) pi d_k^3), and the volume
    weights w_i = m / rho_i."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    g = (np.arange(n_side) + 0.5) / n_side
    r0 = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, n)
    r0 = r0 + rng.uniform(-jitter, jitter, (3, n)) / n_side
    modes = glass_modes()
    r = r0.copy()
    for kx, ky, kz, phi in modes:
        kv = np.array([kx, ky, kz])
        r += (np.sin(kv @ r0 + phi) / 275.0) * (kv / np.linalg.norm(kv))[:, None]
    r = np.mod(r, 1.0)
    gas = np.minimum(r.astype(np.float32), ONE_BELOW)
    m = 1.0 / n
    d, _ = cKDTree(np.mod(r, 1.0).T, boxsize=1.0).query(np.mod(r, 1.0).T, k=k + 1)
    rho = k * m / (4.0 / 3.0 * np.pi * d[:, -1] ** 3)
    alpha = rho.astype(np.float32)
    w = (m / rho).astype(np.float32)
    src = np.ascontiguousarray(gas[[1, 2, 0]])
    lum = np.ones(n, np.float32)
    return _problem(f"glass_{n_side}", gas, alpha, src, lum, theta, tau_ref, bucket, weight=w,
                    seed=seed)


def sink_sample(n_gas, n_sample, seed=7):
    """A seeded sample of sink indices (sorted, without repetition)."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_gas)
    return np.sort(rng.choice(n_gas, size=n_sample, replace=False)).astype(np.int64)
