"""Host-side argument checks of the allocation-free Morton sort binding: a bad shape,
a short output tensor or tensors on different devices are rejected before the
library is called, so no kernel can read or write outside the caller's buffers."""
import pytest
import torch

from paper_1902_08083_gb300 import trevr


def test_rejects_wrong_shape():
    with pytest.raises(ValueError):
        trevr.morton_sort_noalloc(torch.zeros(2, 100))
    with pytest.raises(ValueError):
        trevr.morton_sort_noalloc(torch.zeros(300))


def test_rejects_short_outputs():
    g = torch.zeros(3, 100)
    with pytest.raises(ValueError):
        trevr.morton_sort_noalloc(g, keys_out=torch.zeros(99, dtype=torch.int64))
    with pytest.raises(ValueError):
        trevr.morton_sort_noalloc(g, perm_out=torch.zeros(50, dtype=torch.int32))


def test_rejects_outputs_on_another_device():
    g = torch.zeros(3, 100)
    with pytest.raises(ValueError):
        trevr.morton_sort_noalloc(g, keys_out=torch.empty(100, dtype=torch.int64,
                                                          device="meta"))


def test_rejects_host_tensors():
    with pytest.raises(TypeError):
        trevr.morton_sort_noalloc(torch.zeros(3, 100))
