"""Full-size workloads on the GPU: the 10,000-kernel batch (reports of
sampled kernels against the oracle) and the 2^26-work-item stress instance
(properties that hold at any size, and the oracle's full-size report by
digest; its shapes up to 16 x 1024 are compared with the oracle record by
record in test_gpu_parity.py)."""
import os
import time

import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.test_gpu_parity import same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    racecheck.set_strategy(0)
    return racecheck


@pytest.mark.parametrize("strategy", [0, 3])
def test_batch_of_10000_kernels(rc, oracle, strategy):
    """10,000 kernels of uneven shape in one rc_check_batch call, in
    lock-step rounds (autotuned) and resident (every round of a sub-batch in
    one launch): 12 sampled kernels against the oracle record by record,
    every kernel against the oracle's report by digest."""
    insts = W.batch_kernels(0, 10_000, processes=min(16, os.cpu_count() or 1))
    bcs = [rc.compile(i.src) for i in insts]
    rc.set_strategy(strategy)
    t0 = time.perf_counter()
    try:
        got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)],
                             want_final=False)
    finally:
        rc.set_strategy(0)
    dt = time.perf_counter() - t0
    total = sum(g["n_access"] for g in got)
    print(f"batch: {len(insts)} kernels, {total} accesses in {dt:.2f} s")
    assert total > 1e9
    rng = np.random.default_rng(7)
    small = [k for k, i in enumerate(insts) if i.n_threads <= 20_000]
    for k in rng.choice(small, 12, replace=False):
        i = insts[int(k)]
        want = oracle.check(i.src, i.groups, i.group_size, i.globals)
        same(got[int(k)], want, i.name)
    for g, i in zip(got, insts):
        r = g["records"]
        if len(r):
            assert (r[:, 0] < g["n_intervals"]).all()
    # every kernel against the oracle's report, by digest
    # (tests/golden/make_batch_oracle.py wrote them from oracle runs)
    import hashlib
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch10000_oracle.json")
    if os.path.exists(path):
        want = json.load(open(path))["kernels"]
        assert len(want) == len(got)
        bad = []
        for k, (g, w) in enumerate(zip(got, want)):
            digest = hashlib.sha256(np.ascontiguousarray(g["records"].astype(np.uint32)).tobytes()).hexdigest()[:16]
            if [g["status"], g["n_intervals"], g["n_access"], len(g["records"]), digest] != w:
                bad.append(k)
        assert not bad, f"{len(bad)} kernels differ from the oracle, first {bad[:5]}"


def test_stress_instance_full_size(rc):
    """65,536 groups x 1024 work-items, 16 barriers, 512 statements, a 2^26
    cell array: the run completes and its report is well formed."""
    inst = W.stress_kernel(0)
    bc = rc.compile(inst.src)
    r = rc.check(bc, inst.groups, inst.group_size, inst.globals, want_final=False)
    N = inst.n_threads
    assert r["n_access"] == r["n_global"] + r["n_local"] and r["n_access"] > 5e9
    assert r["n_intervals"] <= 17
    rec = r["records"]
    races = rec[rec[:, 4] < 16]
    if len(races):
        assert (races[:, 5] < N).all() and (races[:, 6] < N).all()
        assert (races[:, 5] != races[:, 6]).all()
        key = races[:, 0].astype(np.uint64) << 40 | races[:, 3].astype(np.uint64) << 4 | races[:, 4]
        assert (np.diff(key.astype(np.int64)) > 0).all()  # canonical order, no duplicates
    assert r["status"] in (0, 1, 2)


def test_stress_instance_full_size_against_the_oracle(rc):
    """The full 2^26-work-item report against the oracle's, from the digests
    tests/golden/make_config5_oracle.py wrote (an address-sharded oracle run):
    counters, every record (2,359,294 of them) and the final memory."""
    import hashlib
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config5_oracle.json")
    if not os.path.exists(path):
        pytest.skip("no oracle digest of the full instance")
    g = json.load(open(path))
    inst = W.stress_kernel(0)
    r = rc.check(rc.compile(inst.src), inst.groups, inst.group_size, inst.globals, want_final=True)
    for k in ("status", "n_intervals", "n_access", "n_global", "n_local"):
        assert r[k] == g[k], (k, r[k], g[k])
    recs = np.ascontiguousarray(r["records"].astype(np.uint32))
    assert len(recs) == g["n_race_records"] + g["n_error_records"]
    assert hashlib.sha256(recs.tobytes()).hexdigest() == g["records_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(r["final"]).tobytes()).hexdigest() == g["final_sha256"]
    # every class the classifier decides is present at full size (WW_RACE,
    # WW_BENIGN, RW_RACE): the digests above compare each of them
    classes = set(np.unique(recs[:, 4]).tolist()) if len(recs) else set()
    assert {1, 2, 3} <= classes, classes
