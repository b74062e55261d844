"""The allocation-free sort entry point against the allocating one.

rc_sort_accesses_noalloc serves callers that may not allocate device
memory (fixed memory budgets reserved at start-up, pipelines that cannot
take an allocation's synchronisation): its scratch is a fixed device array
inside the library.  This file is collected last so that a run that stops
at the first failure has run every other test first; it also passes on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    return racecheck.load()


def records(n, seed):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, 1 << 20, n).astype(np.uint32)
    cell[rng.random(n) < 0.25] = 7
    item = rng.integers(0, 1 << 18, n).astype(np.uint32) | ((rng.random(n) < 0.5).astype(np.uint32) << 31)
    return np.stack([cell, item, rng.integers(0, 99, n).astype(np.uint32), np.arange(n, dtype=np.uint32)], axis=1)


def call(fn, src, dst, cell_bits, item_bits):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    return fn(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), ctypes.c_uint64(src.shape[0]),
              ctypes.c_uint32(cell_bits), ctypes.c_uint32(item_bits), ctypes.c_void_p(stream))


def test_noalloc_sort_matches_allocating_sort_twice(lib):
    import torch
    vp = ctypes.c_void_p
    for f in (lib.rc_sort_accesses, lib.rc_sort_accesses_noalloc):
        f.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp]
        f.restype = ctypes.c_int
    # two calls in a row; the second is smaller and reuses the array's stale contents
    for n, seed in ((1 << 18, 1), (70_001, 2)):
        src = torch.from_numpy(records(n, seed).view(np.int32)).cuda()
        want = torch.full_like(src, -1)
        got = torch.full_like(src, -2)
        assert call(lib.rc_sort_accesses, src, want, 20, 18) == 0
        assert call(lib.rc_sort_accesses_noalloc, src, got, 20, 18) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_sort_rejects_inputs_beyond_its_array(lib):
    import torch
    vp = ctypes.c_void_p
    lib.rc_sort_accesses_noalloc.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp]
    src = torch.zeros(((1 << 18) + 1, 4), dtype=torch.int32, device="cuda")
    assert call(lib.rc_sort_accesses_noalloc, src, src.clone(), 20, 18) == 3  # RC_E_CAPACITY
