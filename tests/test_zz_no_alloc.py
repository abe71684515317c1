"""The allocation-free compaction entry point against the context-based one.

sparseoit_compact_active_static serves callers that cannot allocate device
memory (code that must not trigger the synchronisation of cudaMalloc /
cudaFree, plug-ins whose host runtime owns the device memory budget,
deployments that forbid allocation after start-up).  Its scratch is a fixed
device array shared by every call, so this test makes two calls in a row
with different masks (the second reuses the scratch the first left behind)
and compares each with the index list of sparseoit_set_active /
sparseoit_get_active; index lists must match exactly, from the largest mask
the scratch allows down to small ones.  It also checks that a mask longer than
the static maximum is rejected.  Run last: it must pass both
alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_13855_gb300 import _lib, scenes
from paper_2605_13855_gb300.renderer import Renderer

pytestmark = pytest.mark.gpu


def _static_compact(lib, mask: torch.Tensor, stream):
    n = mask.numel()
    idx = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = lib.sparseoit_compact_active_static(ctypes.c_void_p(mask.data_ptr()), n, ctypes.c_void_p(idx.data_ptr()),
                                             ctypes.c_void_p(count.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.OK
    stream.synchronize()
    k = int(count.item())
    return idx[:k].cpu().numpy(), k


def test_static_compaction_matches_set_active():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    lib = _lib.load()
    stream = torch.cuda.Stream()
    # largest first: the scratch left by a larger call must not leak into the smaller ones; the first
    # two masks take more than one 1024-block chunk of the block-count scan (n > 4,194,304), the first
    # is the largest mask the static scratch allows
    cases = [(_lib.STATIC_MAX_SPLATS, 0.05, 3), (5_000_011, 0.2, 4), (300_017, 0.05, 1), (70_001, 0.5, 2)]
    for n, frac, seed in cases:
        m = scenes.random_active_mask(n, frac, seed)
        mask = torch.as_tensor(m, device="cuda")
        got, k = _static_compact(lib, mask, stream)
        r = Renderer(n, [(16, 16)])
        r.set_active(mask)
        want = r.active_indices().cpu().numpy()
        r.close()
        assert k == want.size == int(m.sum())
        assert np.array_equal(got, want)
    # a mask larger than the static scratch allows is rejected before any work
    too_big = _lib.STATIC_MAX_SPLATS + 1
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.sparseoit_compact_active_static(ctypes.c_void_p(count.data_ptr()), too_big,
                                             ctypes.c_void_p(count.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                                             ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.ERR_INVALID_ARG
