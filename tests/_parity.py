"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them."""
import numpy as np

# flux tolerance (fp32 path vs FP64 oracle), per sink relative error
MEDIAN_TOL = 1e-5
MAX_TOL = 1e-3
TINY = 1e-30  # below this the oracle flux underflows fp32's useful range


def to_gpu(P, device="cuda"):
    import torch
    g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(device)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
    g["weight"] = None if P.get("weight") is None else torch.from_numpy(P["weight"]).to(device)
    return g


def gpu_tree(P, device="cuda"):
    from paper_1902_08083_gb300 import trevr
    g = to_gpu(P, device)
    return trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"],
                            weight=g["weight"], lo=P["lo"], side=P["side"], bucket=P["bucket"])


def oracle_tree(P):
    import oracle
    return oracle.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], lo=P["lo"],
                             side=P["side"], bucket=P["bucket"], weight=P.get("weight"))


def flux_errors(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    big = ref >= TINY
    rel = np.abs(gpu[big] - ref[big]) / ref[big]
    tiny_ok = bool(np.all(gpu[~big] < 1e-29))
    return rel, tiny_ok


def assert_flux_parity(gpu, ref, label=""):
    rel, tiny_ok = flux_errors(gpu, ref)
    assert rel.size > 0
    med, mx = float(np.median(rel)), float(rel.max())
    assert med <= MEDIAN_TOL, f"{label}: median rel err {med:.3e} > {MEDIAN_TOL}"
    assert mx <= MAX_TOL, f"{label}: max rel err {mx:.3e} > {MAX_TOL}"
    assert tiny_ok, f"{label}: fluxes below {TINY} not reproduced as underflow"
    return med, mx


def canonical_nodes_gpu(E):
    """GPU cells (breadth-first numbering) as rows sorted by (first, -count): the
    preorder of the tree, independent of the numbering."""
    child = E["child"].cpu().numpy()
    n = child.shape[0]
    ids = np.arange(1, n)
    first = E["first"].cpu().numpy()[ids]
    count = E["count"].cpu().numpy()[ids]
    order = np.lexsort((-count, first))
    return ids[order]


def canonical_nodes_oracle(N):
    order = np.lexsort((-N["count"], N["first"]))
    return order


_CLUMPY = {}


def clumpy_problem():
    """The clumpy workload at the benchmark's size (2^22 gas, 2^14 sources), generated
    once per test process (it takes tens of seconds on the host)."""
    import workloads
    if "P" not in _CLUMPY:
        _CLUMPY["P"] = workloads.clumpy()
    return _CLUMPY["P"]
