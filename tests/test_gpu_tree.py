"""GPU tree build vs the oracle: keys, sort order and topology bit-exact; cell
values equal to the oracle's fp32 values (Sec. 2.2, 2.3)."""
import numpy as np
import pytest

import workloads
from _parity import canonical_nodes_gpu, canonical_nodes_oracle, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(5)
    P0 = workloads.uniform_box(n_gas=4096, n_src=64, seed=0)
    P1 = workloads.uniform_box(n_gas=20000, n_src=300, seed=9)
    P1["alpha"] = workloads.lognormal_alpha(rng, P1["gas_xyz"], 1.0, 2.0, 0.05, n_modes=64)
    P1["weight"] = rng.uniform(0.2, 3.0, 20000).astype(np.float32)
    # clustered with exact duplicates (an over-full leaf) and a ragged bucket
    P2 = workloads.uniform_box(n_gas=5001, n_src=7, seed=3, bucket=3)
    g = (0.3 + 0.01 * rng.standard_normal((3, 5001))).astype(np.float32)
    g[:, :40] = g[:, 40:41]
    P2["gas_xyz"] = np.ascontiguousarray(np.clip(g, 0, workloads.ONE_BELOW))
    # shifted, non-unit domain
    P3 = workloads.uniform_box(n_gas=3000, n_src=20, seed=4)
    P3["gas_xyz"] = (P3["gas_xyz"] * np.float32(2.5) - np.float32(1.0)).astype(np.float32)
    P3["src_xyz"] = (P3["src_xyz"] * np.float32(2.5) - np.float32(1.0)).astype(np.float32)
    P3["lo"], P3["side"] = (-1.0, -1.0, -1.0), 2.5
    # a single particle
    P4 = workloads.uniform_box(n_gas=1, n_src=1, seed=8)
    return [("uniform4096", P0), ("lognormal_weighted", P1), ("clustered_dups", P2),
            ("shifted_domain", P3), ("single", P4), ("deep", deep_problem())]


def deep_problem():
    """A comb of 64 particles whose Morton keys are 0 and every single bit 2^b
    (the point with only grid bit m of one axis set), in buckets of one: each
    level of the tree splits off one particle, down to depth 63."""
    P = workloads.uniform_box(n_gas=64, n_src=40, seed=12, bucket=1)
    g = np.zeros((3, 64), np.float32)
    k = 1
    for m in range(21):
        for axis in range(3):
            g[axis, k] = np.float32(2.0 ** (m - 21))
            k += 1
    P["gas_xyz"] = g
    return P


@pytest.mark.parametrize("name,P", _cases(), ids=[c[0] for c in _cases()])
def test_tree_bit_exact(name, P):
    T = oracle_tree(P)
    G = gpu_tree(P)
    E = G.export()
    part = T.particles()
    np.testing.assert_array_equal(E["key"].cpu().numpy().view(np.uint64), part["key"])
    np.testing.assert_array_equal(E["perm"].cpu().numpy(), part["perm"])
    N = T.nodes()
    assert G.n_nodes == T.n_nodes
    assert G.max_depth == int(N["depth"].max())
    gi = canonical_nodes_gpu(E)
    oi = canonical_nodes_oracle(N)
    for gk, ok in (("first", "first"), ("count", "count"), ("depth", "depth")):
        np.testing.assert_array_equal(E[gk].cpu().numpy()[gi], N[ok][oi], err_msg=gk)
    np.testing.assert_array_equal(E["child"].cpu().numpy()[gi] < 0, N["split_bit"][oi] < 0)
    np.testing.assert_array_equal(E["glo"].cpu().numpy()[gi], N["glo"][oi])
    np.testing.assert_array_equal(E["ghi"].cpu().numpy()[gi], N["ghi"][oi])
    np.testing.assert_array_equal(E["src_count"].cpu().numpy()[gi], N["src_count"][oi])
    # leaf of every sorted particle: same cell (compared through its range)
    lf_g = E["leaf_of"].cpu().numpy()
    lf_o = part["leaf_of"]
    np.testing.assert_array_equal(E["first"].cpu().numpy()[lf_g], N["first"][lf_o])
    # sources in the same order
    np.testing.assert_array_equal(E["src_order"].cpu().numpy(), T.sources()["order"])
    # cell values: the alpha spread takes the same FP64 steps on both sides (bit-exact);
    # means and centroids are FP64 sums in another association, rounded to fp32
    N32 = T.nodes32()
    np.testing.assert_array_equal(E["dalpha"].cpu().numpy()[gi], N32["dalpha"][oi])
    for gk, ok in (("abar", "abar"), ("lum", "L"), ("cen", "cen"), ("l2", "l2")):
        a = E[gk].cpu().numpy()[gi].astype(np.float64)
        b = N32[ok][oi].astype(np.float64)
        np.testing.assert_allclose(a, b, rtol=2.5e-7, atol=0, err_msg=gk)
    G.free()


def test_out_of_domain_and_invalid_inputs():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=1000, n_src=5, seed=1)
    for mutate, code in ((lambda P: P["gas_xyz"].__setitem__((0, 17), 1.0), 2),
                         (lambda P: P["src_xyz"].__setitem__((2, 1), -0.5), 2),
                         (lambda P: P["alpha"].__setitem__(3, np.nan), 1),
                         (lambda P: P["alpha"].__setitem__(3, -1.0), 1),
                         (lambda P: P["src_lum"].__setitem__(0, np.inf), 1)):
        Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
        mutate(Q)
        with pytest.raises(trevr.TrevrError) as ei:
            gpu_tree(Q)
        assert ei.value.code == code
    torch.cuda.synchronize()
    # the context is still usable afterwards
    G = gpu_tree(P)
    assert G.n_nodes > 0


def test_deep_tree_flux():
    # the walk and the rays at the full tree depth (cells 63 levels down)
    from paper_1902_08083_gb300 import trevr
    from _parity import assert_flux_parity
    P = deep_problem()
    G = gpu_tree(P)
    T = oracle_tree(P)
    assert G.max_depth == 63
    for theta, tau_ref in ((0.75, 0.1), (0.0, 0.0)):
        f, c = trevr.compute_flux(G, theta, tau_ref, counters=True)
        of, oc, _ = T.flux(theta, tau_ref, with_counters=True)
        assert_flux_parity(f.cpu().numpy(), of, f"deep tree theta={theta}")
        assert np.count_nonzero(np.any(c.cpu().numpy() != oc.astype(np.int32), axis=1)) <= 2
