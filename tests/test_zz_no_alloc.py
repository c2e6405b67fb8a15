"""The allocation-free Morton sort entry point (trevr_morton_sort_noalloc).

It serves callers that cannot allocate device memory while they run (a host
code that reserves its memory up front, a plug-in handed buffers by the
application that owns the GPU). It must give exactly the keys and the
permutation that trevr_build_tree computes, call after call, although every
call reuses the same fixed scratch array. This file is collected last so that
a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads
from _parity import gpu_tree

pytestmark = pytest.mark.gpu


def _existing(P):
    E = gpu_tree(P).export()
    return E["key"].cpu().numpy(), E["perm"].cpu().numpy()


def test_noalloc_sort_matches_build_tree_twice():
    import torch
    from paper_1902_08083_gb300 import trevr
    cases = [workloads.uniform_box(n_gas=300001, n_src=4, seed=31),
             workloads.uniform_box(n_gas=70000, n_src=4, seed=32)]
    # second case: a shifted domain and repeated positions (ties keep caller order)
    P = cases[1]
    P["gas_xyz"][:, 10:50] = P["gas_xyz"][:, 5:6]
    P["gas_xyz"] = (P["gas_xyz"] * np.float32(3.0) - np.float32(1.5)).astype(np.float32)
    P["lo"], P["side"] = (-1.5, -1.5, -1.5), 3.0
    for P in cases:  # two calls in a row on the shared scratch
        key_ref, perm_ref = _existing(P)
        g = torch.from_numpy(P["gas_xyz"]).cuda()
        keys, perm = trevr.morton_sort_noalloc(g, lo=P["lo"], side=P["side"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(keys.cpu().numpy(), key_ref)
        np.testing.assert_array_equal(perm.cpu().numpy(), perm_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1902_08083_gb300 import trevr
    g = torch.rand(3, trevr.NOALLOC_MAX_N + 1, device="cuda") * 0.5
    with pytest.raises(trevr.TrevrError) as ei:
        trevr.morton_sort_noalloc(g)
    assert ei.value.code == 1
    bad = torch.rand(3, 1000, device="cuda")
    bad[1, 7] = 2.0
    with pytest.raises(trevr.TrevrError) as ei:
        trevr.morton_sort_noalloc(bad)
    assert ei.value.code == 2
    # the scratch is still usable after the reported errors
    ok = torch.rand(3, 5000, device="cuda") * 0.999
    keys, perm = trevr.morton_sort_noalloc(ok)
    assert torch.all(keys[1:] >= keys[:-1])
