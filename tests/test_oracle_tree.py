"""Pins for the oracle's tree: Morton keys, sort order, topology and cell moments.

Each check is fixed by something other than the oracle's own code: hand-worked
examples, a string-based bit interleave, numpy's stable sort, numpy sums and
the space-filling invariants of the radiation tree (Sec. 2.2.2 and 2.3 of
Grond et al. 2019).
"""
import numpy as np
import pytest

import workloads

G = 1 << 21  # grid cells per axis


def _tree(oracle_lib, gas, alpha, src=None, lum=None, bucket=8, weight=None):
    gas = np.asarray(gas, np.float32).reshape(3, -1)
    if src is None:
        src = np.full((3, 1), 0.5, np.float32)
        lum = np.ones(1, np.float32)
    return oracle_lib.OracleTree(gas, np.asarray(alpha, np.float32), src,
                                 np.asarray(lum, np.float32), bucket=bucket, weight=weight)


# ---------------------------------------------------------------- keys
def test_morton_keys_hand_values(oracle_lib):
    # x is the most significant axis: its top bit is key bit 62, then y (61), z (60)
    pts = np.array([[0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5], [0.75, 0.0, 0.0],
                    [0.0, 0.0, 0.0]], np.float32).T
    keys = oracle_lib.morton_keys(pts, (0, 0, 0), 1.0)
    assert [int(k) for k in keys] == [1 << 62, 1 << 61, 1 << 60, (1 << 62) | (1 << 59), 0]
    top = np.nextafter(np.float32(1), np.float32(0))
    k = oracle_lib.morton_keys(np.full((3, 1), top, np.float32), (0, 0, 0), 1.0)
    assert int(k[0]) == (1 << 63) - 1  # every grid bit set: clamped to 2^21-1


def test_morton_keys_out_of_domain(oracle_lib):
    for bad in (1.0, -1e-9, np.nan):
        pts = np.array([[0.1, 0.2, 0.3], [bad, 0.5, 0.5]], np.float32).T
        with pytest.raises(oracle_lib.OracleError):
            oracle_lib.morton_keys(pts, (0, 0, 0), 1.0)


def test_morton_keys_match_string_interleave(oracle_lib):
    rng = np.random.default_rng(11)
    lo = np.array([-2.0, 0.5, 3.0], np.float32)
    side = np.float32(3.7)
    pts = (lo[:, None] + rng.random((3, 500)).astype(np.float32) * side).astype(np.float32)
    pts = np.minimum(pts, np.nextafter(lo[:, None] + side, lo[:, None]).astype(np.float32))
    keys = oracle_lib.morton_keys(pts, lo, side)
    scale = np.float32(2097152.0) / side
    for i in range(pts.shape[1]):
        q = []
        for d in range(3):
            t = (pts[d, i] - lo[d]) * scale  # two rounded fp32 operations
            q.append(min(int(np.floor(t)), G - 1))
        bits = [format(v, "021b") for v in q]
        s = "".join(bits[0][b] + bits[1][b] + bits[2][b] for b in range(21))
        assert int(keys[i]) == int(s, 2)


# ---------------------------------------------------------------- sort + topology
def test_sort_is_numpy_stable_sort(oracle_lib):
    P = workloads.uniform_box(n_gas=3000, n_src=8, seed=5)
    gas = P["gas_xyz"].copy()
    gas[:, 100:140] = gas[:, 7:8]  # 41 identical positions: ties must keep caller order
    T = _tree(oracle_lib, gas, P["alpha"], P["src_xyz"], P["src_lum"])
    keys = oracle_lib.morton_keys(gas, (0, 0, 0), 1.0)
    part = T.particles()
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(part["perm"], order)
    np.testing.assert_array_equal(part["key"], keys[order])


def _coords(keys):
    """Grid coordinates of Morton keys, de-interleaved bit by bit."""
    out = np.zeros((len(keys), 3), np.int64)
    for i, k in enumerate(keys):
        k = int(k)
        for d in range(3):
            g = 0
            for b in range(20, -1, -1):
                g = (g << 1) | ((k >> (3 * b + 2 - d)) & 1)
            out[i, d] = g
    return out


@pytest.mark.parametrize("case", ["uniform", "clustered"])
def test_tree_invariants(oracle_lib, case):
    rng = np.random.default_rng(3)
    if case == "uniform":
        gas = rng.random((3, 2000)).astype(np.float32)
    else:
        gas = (0.3 + 0.01 * rng.standard_normal((3, 2000))).astype(np.float32)
        gas[:, :30] = gas[:, 30:31]  # 31 coincident particles > bucket
    gas = np.clip(gas, 0, np.nextafter(np.float32(1), np.float32(0)))
    bucket = 6
    T = _tree(oracle_lib, gas, np.ones(gas.shape[1]), bucket=bucket)
    N = T.nodes()
    part = T.particles()
    keys = part["key"]
    q = _coords(keys)
    n = T.n_nodes
    leaf = N["split_bit"] < 0
    # leaves fill the domain: their integer volumes add up to the whole grid
    vol = sum(int(np.prod((N["ghi"][X] - N["glo"][X]).astype(object))) for X in np.nonzero(leaf)[0])
    assert vol == G ** 3
    # every particle lies in its leaf's box; leaves respect the bucket size
    lf = part["leaf_of"]
    assert np.all(leaf[lf])
    assert np.all((q >= N["glo"][lf]) & (q < N["ghi"][lf]))
    for X in np.nonzero(leaf)[0]:
        a, c = N["first"][X], N["count"][X]
        assert c <= bucket or keys[a] == keys[a + c - 1]
    if case == "clustered":
        assert N["count"][leaf].max() >= 31
    # internal nodes: preorder, children partition the range and the box at one plane
    for X in np.nonzero(~leaf)[0]:
        lo_c, up_c = N["lower"][X], N["upper"][X]
        assert lo_c == X + 1 and N["parent"][lo_c] == X and N["parent"][up_c] == X
        a, c = N["first"][X], N["count"][X]
        assert N["first"][lo_c] == a and N["first"][up_c] == a + N["count"][lo_c]
        assert N["count"][lo_c] + N["count"][up_c] == c
        b = int(N["split_bit"][X])
        kk = [int(k) for k in keys[a:a + c]]
        assert all(((k >> b) & 1) == 0 for k in kk[:N["count"][lo_c]])
        assert all(((k >> b) & 1) == 1 for k in kk[N["count"][lo_c]:])
        assert len({k >> (b + 1) for k in kk}) == 1  # common prefix above the split bit
        axis = (62 - b) % 3
        plane = N["ghi"][lo_c][axis]
        assert N["glo"][up_c][axis] == plane
        assert N["glo"][X][axis] < plane < N["ghi"][X][axis]
        level = (62 - b) // 3
        cell = 1 << (21 - level)  # the Morton cell of the prefix, halved by the plane
        assert plane % cell == cell // 2
        for d in range(3):
            if d != axis:
                for ch in (lo_c, up_c):
                    assert N["glo"][ch][d] == N["glo"][X][d] and N["ghi"][ch][d] == N["ghi"][X][d]


def test_tree_hand_example_column(oracle_lib):
    # four particles along x at y=z=0.1, bucket 1: cuts at x=1/2, then 1/4 and 3/4
    gas = np.array([[0.1, 0.3, 0.6, 0.8], [0.1] * 4, [0.1] * 4], np.float32)
    T = _tree(oracle_lib, gas, [1, 1, 1, 1], bucket=1)
    N = T.nodes()
    leaves = [X for X in range(T.n_nodes) if N["split_bit"][X] < 0]
    boxes = sorted((N["glo"][X][0], N["ghi"][X][0]) for X in leaves)
    q = G // 4
    assert boxes == [(0, q), (q, 2 * q), (2 * q, 3 * q), (3 * q, 4 * q)]
    for X in leaves:  # no cut on y or z: full extent
        assert list(N["glo"][X][1:]) == [0, 0] and list(N["ghi"][X][1:]) == [G, G]


def test_tree_hand_example_skipped_level(oracle_lib):
    # x = 1/8 and 3/8 share x's top bit: the first cut is at x = 1/4 and the upper
    # child keeps the empty volume up to x = 1 (space filling with a skipped level)
    gas = np.array([[0.125, 0.375], [0.5, 0.5], [0.5, 0.5]], np.float32)
    T = _tree(oracle_lib, gas, [2, 6], bucket=1)
    N = T.nodes()
    assert T.n_nodes == 3
    assert (N["glo"][1][0], N["ghi"][1][0]) == (0, G // 4)
    assert (N["glo"][2][0], N["ghi"][2][0]) == (G // 4, G)
    # alpha_min/max along x add optical depths across the cut and divide by the width:
    # (2 * 1/4 + 6 * 3/4) / 1 = 5; across the cut (y, z) take min / max of the children
    amin, amax = T.directional()
    assert amin[0, 0] == 5.0 and amax[0, 0] == 5.0
    assert list(amin[0, 1:]) == [2.0, 2.0] and list(amax[0, 1:]) == [6.0, 6.0]
    N = T.nodes()
    assert N["amin"][0] == 2.0 and N["amax"][0] == 6.0


def test_alpha_min_max_hand_octants(oracle_lib):
    # eight particles at the octant centres, bucket 1: cuts x, then y, then z.
    # alpha(ix,iy,iz): worked by hand from Sec. 2.2.3 (sum across a cut along the
    # cut axis divided by the width, min/max otherwise):
    #   x: mean(min over ix=0 leaves, min over ix=1 leaves) = mean(1, 2) = 1.5
    #   y: min over ix of mean over iy of min over iz = min(mean(1,3), mean(2,4)) = 2
    #   z: min over ix of min over iy of mean over iz = min(4, 4.5) = 4
    #   => alpha_min(root) = 1.5 ; likewise alpha_max(root) = max(8.5, 7.5, 6) = 8.5
    vals = {(0, 0, 0): 1, (0, 0, 1): 9, (0, 1, 0): 3, (0, 1, 1): 5,
            (1, 0, 0): 7, (1, 0, 1): 2, (1, 1, 0): 8, (1, 1, 1): 4}
    pts, al = [], []
    for (ix, iy, iz), v in vals.items():
        pts.append([0.25 + 0.5 * ix, 0.25 + 0.5 * iy, 0.25 + 0.5 * iz])
        al.append(v)
    T = _tree(oracle_lib, np.array(pts, np.float32).T, al, bucket=1)
    N = T.nodes()
    amin, amax = T.directional()
    assert list(amin[0]) == [1.5, 2.0, 4.0]
    assert list(amax[0]) == [8.5, 7.5, 6.0]
    assert N["amin"][0] == 1.5 and N["amax"][0] == 8.5
    assert N["abar"][0] == 39.0 / 8.0
    assert T.n_nodes == 15
    # the refinement test uses the spread alpha_max - alpha_min (Eq. refcrit)
    d32 = T.nodes32()["dalpha"]
    assert d32[0] == 7.0
    # node 1 is the x<1/2 half (cut on y): min over directions 1 (x: min of its
    # four leaves), max 9 (x: max of its four leaves)
    assert N["amin"][1] == 1.0 and N["amax"][1] == 9.0 and d32[1] == 8.0


def test_uniform_alpha_gives_no_spread(oracle_lib):
    P = workloads.uniform_box(n_gas=2000, n_src=4, seed=9, alpha=20.0)
    T = _tree(oracle_lib, P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"])
    N = T.nodes()
    assert np.all(N["abar"] == 20.0)
    assert np.all(N["amin"] == 20.0) and np.all(N["amax"] == 20.0)
    assert np.all(T.nodes32()["dalpha"] == 0.0)


def test_cell_density_is_volume_weighted(oracle_lib):
    # Sec. 2.3: rho_cell = sum m / sum (m / rho). With alpha = kappa*rho (kappa=1)
    # and weight w = m/rho the cell's mean absorption is exactly that density.
    rng = np.random.default_rng(21)
    n = 1500
    gas = rng.random((3, n)).astype(np.float32)
    m = rng.uniform(0.5, 2.0, n).astype(np.float32)
    rho = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    w = (m / rho).astype(np.float32)
    T = _tree(oracle_lib, gas, rho, weight=w)
    N = T.nodes()
    perm = T.particles()["perm"]
    for X in range(0, T.n_nodes, 7):
        idx = perm[N["first"][X]:N["first"][X] + N["count"][X]]
        ref = np.sum(w[idx].astype(np.float64) * rho[idx]) / np.sum(w[idx].astype(np.float64))
        assert abs(N["abar"][X] - ref) <= 1e-13 * ref
        assert abs(N["W"][X] - np.sum(w[idx].astype(np.float64))) <= 1e-12 * N["W"][X]


def test_source_deposit_and_moments(oracle_lib):
    P = workloads.uniform_box(n_gas=2500, n_src=300, seed=4)
    T = _tree(oracle_lib, P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"])
    N = T.nodes()
    S = T.sources()
    src = P["src_xyz"].astype(np.float64)
    lum = P["src_lum"].astype(np.float64)
    keys = oracle_lib.morton_keys(P["src_xyz"], (0, 0, 0), 1.0)
    q = _coords(keys)
    # each source sits in the leaf whose box holds its grid point
    for s in range(T.n_src):
        o, X = S["order"][s], S["leaf"][s]
        assert N["split_bit"][X] < 0
        assert np.all(q[o] >= N["glo"][X]) and np.all(q[o] < N["ghi"][X])
    # root: total luminosity and centre of luminosity
    assert abs(N["L"][0] - lum.sum()) <= 1e-12 * lum.sum()
    np.testing.assert_allclose(N["cen"][0], (src * lum).sum(1) / lum.sum(), rtol=1e-12)
    # every node: L and centroid over the sources in its subtree; l = furthest vertex
    h = 1.0 / G
    for X in range(T.n_nodes):
        a, c = N["src_first"][X], N["src_count"][X]
        idx = S["order"][a:a + c]
        assert abs(N["L"][X] - lum[idx].sum()) <= 1e-12 * max(lum[idx].sum(), 1e-300)
        if c:
            verts = np.array([[N[("glo", "ghi")[(v >> d) & 1]][X][d] * h for d in range(3)]
                              for v in range(8)])
            lref = np.max(np.linalg.norm(verts - N["cen"][X], axis=1))
            assert abs(N["lrad"][X] - lref) <= 1e-12
    assert N["src_count"][0] == T.n_src
