"""GPU radix sort of access records (rc_sort_accesses) against a stable
sort by (cell, work-item) -- the definition of the grouping the exact
classifier relies on."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


def random_records(n, cell_bits, item_bits, seed):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, 1 << cell_bits, n, dtype=np.uint64).astype(np.uint32)
    if n and cell_bits > 3:  # some heavy cells
        cell[rng.random(n) < 0.3] = rng.integers(0, 4)
    item = rng.integers(0, 1 << item_bits, n, dtype=np.uint64).astype(np.uint32)
    write = (rng.random(n) < 0.4).astype(np.uint32) << 31
    rec = np.stack([cell, item | write, rng.integers(-9, 9, n).astype(np.int64).astype(np.uint32),
                    np.arange(n, dtype=np.uint32)], axis=1)
    return rec


def expected(rec):
    cell = rec[:, 0].astype(np.uint64)
    item = (rec[:, 1] & 0x7FFFFFFF).astype(np.uint64)
    order = np.lexsort((item, cell))  # stable: ties keep input order
    return rec[order]


@pytest.mark.parametrize("n,cell_bits,item_bits", [
    (0, 8, 8), (1, 8, 8), (2047, 8, 4), (2049, 12, 6), (100_003, 23, 18), (1 << 20, 26, 26),
    (50_000, 0, 31), (50_000, 27, 0)])
def test_sort_accesses_matches_stable_sort(rc, n, cell_bits, item_bits):
    import torch
    rec = random_records(n, cell_bits, item_bits, n + cell_bits)
    src = torch.from_numpy(rec.view(np.int32)).cuda()
    dst = torch.full_like(src, -1)
    rc.sort_accesses(src, dst, cell_bits, item_bits)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dst.cpu().numpy().view(np.uint32), expected(rec))
    np.testing.assert_array_equal(src.cpu().numpy().view(np.uint32), rec)  # input untouched


def test_sort_accesses_rejects_bad_sizes(rc):
    import torch
    a = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(rc.RaceCheckError):
        rc.sort_accesses(a, a.clone(), 40, 31)
    with pytest.raises(rc.RaceCheckError):
        rc.sort_accesses(a, a.clone(), 8, 32)
