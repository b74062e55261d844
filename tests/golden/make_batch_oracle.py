"""Writes tests/golden/batch10000_oracle.json: for every kernel of the
10,000-kernel batch workload (seed 0), the oracle's status, interval and
access counters and a SHA-256 of its records.  Calls only the oracle and the
seeded input generator.

    python tests/golden/make_batch_oracle.py [--processes 8]
"""
import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def records_digest(recs) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(recs.astype(np.uint32)).tobytes()).hexdigest()


def _job(params):
    from oracle import oracle
    from paper_1308_3203_gb300 import workloads as W
    out = []
    for p in params:
        inst = W._batch_one(p)
        r = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
        out.append([int(r["status"]), int(r["n_intervals"]), int(r["n_access"]), int(len(r["records"])),
                    records_digest(r["records"])[:16]])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--processes", type=int, default=8)
    args = ap.parse_args()
    import multiprocessing as mp
    from oracle import oracle
    from paper_1308_3203_gb300 import workloads as W
    oracle.build()
    params = W._batch_params(0, 10000)
    chunks = [params[k:k + 25] for k in range(0, len(params), 25)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.processes) as pool:
        parts = pool.map(_job, chunks, chunksize=1)
    rows = [row for part in parts for row in part]
    out = {"workload": "10,000 kernels, seed 0 (the batch workload)",
           "fields": ["status", "n_intervals", "n_access", "n_records", "records_sha256_prefix16"],
           "kernels": rows, "wall_seconds": time.time() - t0, "processes": args.processes,
           "host": f"{os.cpu_count()} cores, {os.uname().machine}"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch10000_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(len(rows), out["wall_seconds"])


if __name__ == "__main__":
    main()
