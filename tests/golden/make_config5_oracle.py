"""Writes tests/golden/config5_oracle.json: the oracle's report of the config-5
instance (stress kernel, seed 0, 65,536 groups x 1024 work-items, 16
barriers, global int32[2^26]) from an address-sharded run, with how long it
took.  Calls only the oracle and the seeded input generator.

    python tests/golden/make_config5_oracle.py [--shards 8] [--processes 4]

About 33 minutes of one core per shard and about 12 GB of memory per
running shard.
"""
import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def _job(args):
    p, n_shards, groups = args
    from oracle import oracle
    from paper_1308_3203_gb300 import workloads as W
    st = W.stress_kernel(0, groups=groups)
    t0 = time.time()
    r = oracle.check(st.src, st.groups, st.group_size, st.globals, shard=(p, n_shards))
    dt = time.time() - t0
    out = {k: (int(r[k]) if k != "records" else r[k]) for k in ("status", "n_intervals", "n_access", "n_global",
                                                               "n_local", "records")}
    out["final_sha256"] = hashlib.sha256(r["final"].tobytes()).hexdigest()
    out["seconds"] = dt
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shards", type=int, default=8)
    ap.add_argument("--processes", type=int, default=4)
    ap.add_argument("--groups", type=int, default=65536, help="fewer: a trial run, nothing written")
    args = ap.parse_args()
    import multiprocessing as mp
    import numpy as np
    from oracle import oracle
    oracle.build()
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.processes) as pool:
        parts = pool.map(_job, [(p, args.shards, args.groups) for p in range(args.shards)], chunksize=1)
    wall = time.time() - t0
    finals = set(x["final_sha256"] for x in parts)
    assert len(finals) == 1, "every shard commits every cell: the final memories agree"
    races = np.concatenate([x["records"][x["records"][:, 4] < 16] for x in parts])
    if len(races):  # report order: (interval, space, wg, addr, cls)
        races = races[np.lexsort(tuple(races[:, k] for k in (4, 3, 2, 1, 0)))]
    errs = parts[0]["records"][parts[0]["records"][:, 4] >= 16]
    out = {
        "workload": f"stress kernel seed 0: {args.groups} groups x 1024 work-items, 16 barriers, "
                    f"global int32[{args.groups * 1024}]",
        "status": 1 if len(races) and bool(set(int(c) for c in races[:, 4]) & {1, 3, 4, 6}) else parts[0]["status"],
        "n_intervals": parts[0]["n_intervals"],
        "n_access": parts[0]["n_access"],
        "n_global": parts[0]["n_global"],
        "n_local": parts[0]["n_local"],
        "n_race_records": int(len(races)),
        "n_error_records": int(len(errs)),
        "records_sha256": hashlib.sha256(np.ascontiguousarray(
            np.concatenate([races.reshape(-1, 10), errs.reshape(-1, 10)]).astype(np.uint32)).tobytes()).hexdigest(),
        "final_sha256": finals.pop(),
        "shards": args.shards,
        "processes": args.processes,
        "wall_seconds": wall,
        "cpu_seconds": sum(x["seconds"] for x in parts),
        "host": f"{os.cpu_count()} cores, {os.uname().machine}",
    }
    if args.groups == 65536:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config5_oracle.json"), "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
