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


def records(n, seed, cell_bits=20, item_bits=18):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, 1 << cell_bits, n).astype(np.uint32)
    cell[rng.random(n) < 0.25] = 7 % (1 << cell_bits)
    item = rng.integers(0, 1 << item_bits, n).astype(np.uint32) | ((rng.random(n) < 0.5).astype(np.uint32) << 31)
    return np.stack([cell, item, rng.integers(0, 99, n).astype(np.uint32), np.arange(n, dtype=np.uint32)], axis=1)


def call(fn, src, dst, cell_bits, item_bits):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    return fn(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), ctypes.c_uint64(src.shape[0]),
              ctypes.c_uint32(cell_bits), ctypes.c_uint32(item_bits), ctypes.c_void_p(stream))


def declare(lib):
    vp = ctypes.c_void_p
    for f in (lib.rc_sort_accesses, lib.rc_sort_accesses_noalloc):
        f.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp]
        f.restype = ctypes.c_int
    lib.rc_release_workspace.restype = ctypes.c_int
    lib.rc_last_error.restype = ctypes.c_char_p


def compare(lib, n, seed, cell_bits, item_bits):
    import torch
    src = torch.from_numpy(records(n, seed, cell_bits, item_bits).view(np.int32)).cuda()
    want = torch.full_like(src, -1)
    got = torch.full_like(src, -2)
    assert call(lib.rc_sort_accesses, src, want, cell_bits, item_bits) == 0
    assert call(lib.rc_sort_accesses_noalloc, src, got, cell_bits, item_bits) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_sort_matches_allocating_sort_twice(lib):
    declare(lib)
    # two calls in a row; the second is smaller and reuses the array's stale contents
    # (38 key bits: five 8-bit passes, the last one writing the output)
    for n, seed in ((1 << 18, 1), (70_001, 2)):
        compare(lib, n, seed, 20, 18)


def test_noalloc_sort_every_pass_count(lib):
    """Two passes (the first writes the fixed array, the second the output),
    one pass (straight to the output) and a single record (a plain copy)."""
    declare(lib)
    for n, seed, cb, ib in ((50_000, 3, 8, 8), (33_333, 4, 4, 4), (1, 5, 8, 8), (2, 6, 4, 4)):
        compare(lib, n, seed, cb, ib)


def test_noalloc_sort_allocates_nothing(lib):
    """With the library's workspace released, a call after the set-up call
    leaves the device's free memory as it was: the scratch is the fixed array,
    not the workspace (which would grow) and not a fresh allocation."""
    import torch
    declare(lib)
    src = torch.from_numpy(records(1 << 17, 8).view(np.int32)).cuda()
    dst = torch.empty_like(src)
    assert call(lib.rc_sort_accesses_noalloc, src, dst, 20, 18) == 0  # set-up call
    torch.cuda.synchronize()
    assert lib.rc_release_workspace() == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call(lib.rc_sort_accesses_noalloc, src, dst, 20, 18) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    want = np.lexsort((records(1 << 17, 8)[:, 1] & 0x7FFFFFFF, records(1 << 17, 8)[:, 0]))
    np.testing.assert_array_equal(dst.cpu().numpy().view(np.uint32), records(1 << 17, 8)[want])


def test_noalloc_sort_rejects_inputs_beyond_its_array(lib):
    import torch
    declare(lib)
    src = torch.zeros(((1 << 18) + 1, 4), dtype=torch.int32, device="cuda")
    assert call(lib.rc_sort_accesses_noalloc, src, src.clone(), 20, 18) == 3  # RC_E_CAPACITY
    assert b"2^18" in lib.rc_last_error()
