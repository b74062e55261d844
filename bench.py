"""Benchmark: race-checked accesses per second on one GB300.

One step = one full race check (every barrier interval: interpreter, access
logs, classification, commit, barrier agreement, report) of the stress
instance: 65,536 work-groups x 1024 work-items (2^26), 16 barriers, 512
statements with nested loops of up to 32 trips and branches on loaded
values, one global int32[2^26] array (seed = rank).  Timed with CUDA events
on the launching stream, each step bracketed by a barrier and a
synchronize, L2 flushed between steps.  The same JSON line carries the
1024 x 256 large instance, the instance checked with every access logged,
a batch of uneven kernels and the learned proposal as secondary objects.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload stress|large]

Under torchrun (N > 1) every rank checks its own instance (replicas: the
single-instance path has no exchange step); value = all ranks' accesses /
the slowest rank's time.  --impl reference times the CPU oracle on a bounded
sample of the same instance (first groups only) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "race-checked accesses/s"
UNIT = "accesses/s"
WORKLOADS = {
    "stress": ("stress instance: 65,536 groups x 1024 work-items, 16 barriers, 512 statements "
               "(nested loops of up to 32 trips, branches on loaded values), global int32[2^26]; "
               "each writing interval ends with a benign cell, a racy cell and reads of it in every group"),
    "large": ("large instance: 1024 groups x 256 work-items, 8 barriers, 200 statements "
              "(loops of 1-16 trips), global int32[4M], local int32[4096] per group, "
              "~5%+5% planted racy/benign stores"),
}
# oracle sample: the same program and input, first groups only
SAMPLE_GROUPS = {"stress": 128, "large": 96}

# DRAM traffic of interp_kernel per launch (dram__bytes_read.sum +
# dram__bytes_write.sum), from an ncu capture of the stress program at
# 4,096 x 1024 work-items, every interval launch of one check, scaled by 16
# to the 65,536-group instance (an interval's traffic grows with its
# work-items: same program, same per-work-item work):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
#       --clock-control none -k regex:interp_kernel --csv \
#       python bench.py --workload stress --groups 4096 --steps 1 --warmup 1 --secondary none
# It holds only for the kernel sources and the stress program it was taken
# on; a change to either reports null.
INTERP_TRAFFIC = {"sources_sha256": None, "program_sha256": None, "bytes_per_launch": None}
INTERP_SOURCES = ("paper_1308_3203_gb300/csrc/interp_kernel.cuh", "paper_1308_3203_gb300/csrc/jit_engine.cuh",
                  "paper_1308_3203_gb300/csrc/kernel_types.cuh", "paper_1308_3203_gb300/csrc/semantics.cuh",
                  "paper_1308_3203_gb300/csrc/translate.cpp", "paper_1308_3203_gb300/csrc/jit.cu")


def interp_sources_sha256() -> str:
    h = hashlib.sha256()
    for f in INTERP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="stress", choices=sorted(WORKLOADS))
    p.add_argument("--groups", type=int, default=0, help="work-groups of the instance (0: its full size)")
    p.add_argument("--strategy", type=int, default=0, help="0 auto, 1 sort, 2 shadow, 3 resident")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--secondary", default="all", choices=["all", "none", "small", "batch", "proposal"],
                   help="none: only the headline instance; small / batch / proposal: the headline and that "
                        "leg alone (profiling runs)")
    p.add_argument("--batch-kernels", type=int, default=10_000,
                   help="size of the batched-checking measurement (0 skips it)")
    p.add_argument("--proposal-kernels", type=int, default=2000,
                   help="training kernels of the learned-proposal measurement (0 skips it)")
    return p.parse_args()


def make_instance(W, workload: str, seed: int, groups: int = 0):
    if workload == "stress":
        return W.stress_kernel(seed, **({"groups": groups} if groups else {}))
    return W.large_kernel(seed, **({"groups": groups} if groups else {}))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler for the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(1.0)  # nvidia-smi takes a moment before its first sample
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(workload: str, seed: int = 0):
    """The oracle's bounded sample of the workload: the same program text and
    input, only the first SAMPLE_GROUPS work-groups launched."""
    from paper_1308_3203_gb300 import workloads as W
    inst = make_instance(W, workload, seed)
    g = SAMPLE_GROUPS[workload]
    return inst, g, (f"same program and input, first {g} of {inst.groups} groups, single-threaded")


def run_reference(args, world, rank):
    """CPU oracle on the host cores, bounded sample of the same workload."""
    if rank != 0:
        return
    from oracle import oracle
    inst, g, sample = oracle_sample(args.workload)
    oracle.build()
    times, acc = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.check(inst.src, g, inst.group_size, inst.globals)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            acc += r["n_access"]
    v = acc / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample} ({r['n_access']} accesses per step)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(workload: str):
    from oracle import oracle
    inst, g, sample = oracle_sample(workload)
    oracle.build()
    t0 = time.perf_counter()
    acc, n = 0, 0
    while time.perf_counter() - t0 < 12.0 or n == 0:
        r = oracle.check(inst.src, g, inst.group_size, inst.globals)
        acc += r["n_access"]
        n += 1
    dt = time.perf_counter() - t0
    return {"value": acc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample}: {n} run(s) of {r['n_access']} accesses in {dt:.1f} s"}


SMALL_KERNELS = 200


def small_leg(rc, W, n=SMALL_KERNELS):
    """Latency of one check of a small kernel (1 group x 64 work-items, one
    barrier, 32 statements over A[256]): n kernels, each checked from host
    inputs through rc_check, host wall clock per check (report on the host
    included); the automatic strategy takes the one-CTA path."""
    import torch
    insts = [W.small_kernel(s) for s in range(n)]
    bcs = [rc.compile(i.src) for i in insts]
    for b, i in zip(bcs[:10], insts[:10]):
        rc.check(b, i.groups, i.group_size, i.globals, want_final=False)
    torch.cuda.synchronize()
    l0 = rc.kernel_launches()
    t0 = time.perf_counter()
    acc = 0
    for b, i in zip(bcs, insts):
        acc += rc.check(b, i.groups, i.group_size, i.globals, want_final=False)["n_access"]
    dt = time.perf_counter() - t0
    launches = (rc.kernel_launches() - l0) / n
    # the same kernels in one rc_check_batch call: the time per kernel when
    # many small kernels are checked at once
    items = [(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)]
    rc.check_batch(items, want_final=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc.check_batch(items, want_final=False)
    dtb = time.perf_counter() - t0
    return {"workload": f"{n} small kernels: 1 group x 64 work-items, 1 barrier, 32 statements, global int32[256]",
            "us_per_check": 1e6 * dt / n, "launches_per_check": launches,
            "accesses_per_check": acc / n,
            "batched_us_per_kernel": 1e6 * dtb / n,
            "timing": "host wall clock around each rc_check (host inputs, H2D and report included); "
                      "batched: around one rc_check_batch of the same kernels"}


def small_oracle_ms(n=SMALL_KERNELS):
    """The oracle's time per small kernel (the same n kernels), one core."""
    from oracle import oracle
    from paper_1308_3203_gb300 import workloads as W
    insts = [W.small_kernel(s) for s in range(n)]
    oracle.build()
    t0 = time.perf_counter()
    for i in insts:
        oracle.check(i.src, i.groups, i.group_size, i.globals)
    return 1e3 * (time.perf_counter() - t0) / n


def shard(n: int, rank: int, world: int) -> range:
    """The units rank `rank` of `world` takes: every world-th, from rank."""
    return range(rank, n, world)


def combine(values, dist, op: str):
    """Reduce a list of floats over the ranks ("max" or "sum"); identity
    without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


def batch_leg(rc, W, n_kernels, rank=0, world=1, dist=None, hbm=6800.0):
    """Batched checking of n uneven kernels: each rank checks its shard in
    one rc_check_batch call (independent problems: no exchange); kernels/s
    = all kernels / the slowest rank's time."""
    params = W._batch_params(0, n_kernels)
    mine = [params[i] for i in shard(n_kernels, rank, world)]
    if len(mine) > 64 and (os.cpu_count() or 1) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(16, os.cpu_count())) as pool:
            insts = pool.map(W._batch_one, mine, chunksize=64)
    else:
        insts = [W._batch_one(p) for p in mine]
    import torch
    # inputs in page-locked host memory (as the headline's end-to-end figure
    # takes them); the call copies them to the device inside the timed region
    items = [(rc.compile(i.src), i.groups, i.group_size, [torch.from_numpy(g).pin_memory().numpy() for g in i.globals])
             for i in insts]

    def timed(strategy):
        rc.set_strategy(strategy)
        try:
            rc.check_batch(items[:64], want_final=False)  # warm-up (and autotuner exploration)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            got = rc.check_batch(items, want_final=False)
            dt = time.perf_counter() - t0
        finally:
            rc.set_strategy(0)
        return got, dt

    def line(got, dt):
        acc = sum(g["n_access"] for g in got)
        logged_g = sum(g["n_global"] * g["n_logged"] // max(g["n_access"], 1) for g in got)
        dt_max, = combine([dt], dist, "max")
        acc_all, n_all, lg_all = combine([acc, len(items), logged_g], dist, "sum")
        gbs = 24.0 * lg_all / dt_max / 1e9
        return {"kernels_per_s": n_all / dt_max, "accesses_per_s": acc_all / dt_max, "seconds": dt_max,
                "accesses": int(acc_all), "logged_global_accesses": int(lg_all),
                "hbm": {"what": "24 B per logged global access (log write + classification read) over the "
                                "call's wall time", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                        "frac": gbs / hbm}}

    out = {"workload": f"{n_kernels} kernels: group size log-uniform 32-1024, 1-64 groups, "
                       "16-512 statements, 0-8 barriers, global int32 arrays 1K-1M",
           "run": "lock-step rounds, strategy and block shape autotuned"}
    out.update(line(*timed(0)))
    out["resident"] = dict(run="every round of a sub-batch in one cooperative launch (strategy 3)",
                           **line(*timed(3)))
    out["timing"] = ("host wall clock around rc_check_batch (inputs in page-locked host memory: their copy "
                     "to the device and the reports' copy back included), slowest rank")
    return out


def proposal_leg(rc, n_train, n_eval=200, epochs=20):
    """Learned proposal: label every candidate of n_train kernels with the
    checker, train the ranking network on the GPU, then compare ranked search
    with plain enumeration on n_eval held-out kernels."""
    import torch
    from paper_1308_3203_gb300 import proposal
    t0 = time.perf_counter()
    X, y, _ = proposal.dataset(range(n_train))
    t_data = time.perf_counter() - t0
    m = rc.MLP(seed=0, capacity=8192)
    xt = torch.from_numpy(X).cuda()
    yt = torch.from_numpy(y).cuda()
    batch = 2048
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = m.train(xt, yt, epochs=epochs, batch=batch, lr=2e-3, seed=1)
    t_train = time.perf_counter() - t0
    # multiply-adds x 2 per example: forward 3 GEMM layers + head; backward
    # weight gradients of 3 layers + head, data gradients of layers 2 and 3
    fwd = 2 * (128 * 256 + 2 * 256 * 256 + 256)
    flops = 3 * fwd - 2 * 128 * 256
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        m.forward(xt)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t0) / 5
    res = proposal.compare_search(m, range(10**6, 10**6 + n_eval))
    res.pop("rows")
    fam = batch_family_leg(rc, proposal)
    return {"workload": f"{n_train} training kernels x 64 candidates (group size 32..1024 step 32, "
                        f"1..64 groups, input seed), {n_eval} held-out kernels",
            "train_examples": int(len(y)), "racy_fraction": float(y.mean()),
            "label_and_feature_seconds": t_data, "epochs": epochs, "batch": batch,
            "train_seconds": t_train, "train_examples_per_s": epochs * len(y) / t_train,
            "train_tflops": epochs * len(y) * flops / t_train / 1e12,
            "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
            "inference_examples_per_s": len(y) / t_inf,
            "search": res, "config3_family": fam}


def batch_family_leg(rc, proposal, n_train=300, n_eval=100, epochs=20):
    """The same pipeline on kernels of the config-3 generator (program fixed
    per kernel, 64 candidate launch shapes and inputs each): how many
    candidates are racy, whether the first one already is, and the searches
    with a network trained on this family."""
    import torch
    t0 = time.perf_counter()
    X, y, kid = proposal.dataset(range(2 * 10**6, 2 * 10**6 + n_train), family="batch")
    t_data = time.perf_counter() - t0
    per = [y[kid == k] for k in range(n_train)]
    racy_k = [p for p in per if p.max() > 0]
    m = rc.MLP(seed=0, capacity=8192)
    losses = m.train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), epochs=epochs, batch=2048,
                     lr=2e-3, seed=1)
    res = proposal.compare_search(m, range(3 * 10**6, 3 * 10**6 + n_eval), family="batch")
    res.pop("rows")
    return {"workload": f"{n_train} training kernels of the config-3 generator (16-512 statements, 0-8 barriers, "
                        f"A[1K..1M]) x 64 candidates, {n_eval} held-out kernels",
            "label_and_feature_seconds": t_data, "racy_fraction": float(y.mean()),
            "racy_kernels_fraction": len(racy_k) / n_train,
            "racy_candidates_per_racy_kernel": float(np.mean([p.mean() for p in racy_k])) if racy_k else 0.0,
            "first_candidate_racy_fraction": float(np.mean([p[0] > 0 for p in racy_k])) if racy_k else 0.0,
            "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]), "search": res}


def measure(rc, inst, bc, *, steps, warmup, dist, flush, log_every=False, host=True, prof_steps=None):
    """Check `inst` steps times with device-resident inputs (CUDA events on
    the launching stream), then with host inputs through the C ABI (e2e),
    then once more with per-launch profiling for the roofline."""
    import torch
    dev_in = [torch.from_numpy(a).cuda() for a in inst.globals]
    host_np = [torch.from_numpy(a).pin_memory().numpy() for a in inst.globals] if host else None
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(inputs, k):
        tot, last = 0.0, None
        for _ in range(k):
            flush.zero_()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            last = rc.check(bc, inst.groups, inst.group_size, inputs, stream=stream.cuda_stream,
                            want_final=False, log_every_access=log_every)
            b.record(stream)
            barrier()
            tot += a.elapsed_time(b)
        return tot, last

    for _ in range(warmup):
        rc.check(bc, inst.groups, inst.group_size, dev_in, want_final=False, log_every_access=log_every)
    torch.cuda.synchronize()
    l0 = rc.kernel_launches()
    ms, rep = timed(dev_in, steps)
    launches = rc.kernel_launches() - l0
    out = {"ms": ms, "rep": rep, "launches": launches, "steps": steps}
    if host:
        out["ms_e2e"], out["rep_e2e"] = timed(host_np, steps)
        out["h2d"] = int(sum(a.nbytes for a in host_np))
    ps = prof_steps or steps
    rc.profile_reset()
    rc.profile_enable(True)
    timed(dev_in, ps)
    rc.profile_enable(False)
    out["prof"] = [rc.profile_get(k) for k in range(2)]
    out["prof_steps"] = ps
    del dev_in, host_np
    return out


def interval_kernel(rc, n_items: int) -> str:
    """The interval kernel the automatic engine runs for an instance of
    n_items work-items: compiled intervals from 2^17 work-items (when this
    process compiled any), else the interpreter."""
    return "rc_jit_kernel" if n_items >= (1 << 17) and rc.jit_stats()["compiles"] else "interp_kernel"


def roofline(m, peak, peak_source, traffic=None, kernel="interp_kernel") -> dict:
    """Roofline of the interval kernel (the dominant kernel: it runs the
    work-items and writes the access logs; rc_jit_kernel under compiled
    intervals, interp_kernel under the interpreter).  Algorithmic bytes per launch: 12 B (cell, work-item and
    read/write bit, value) for every access it wrote to a log; accesses the
    pre-filter proved private are not written and not credited."""
    rep, p0, p1 = m["rep"], m["prof"][0], m["prof"][1]
    launches_per_check = p0["launches"] / max(m["prof_steps"], 1)
    interp_ms = p0["ms"] / max(p0["launches"], 1)
    classify_ms_per_check = p1["ms"] / max(m["prof_steps"], 1)
    logged = rep["n_logged"]
    bytes_per_launch = 12.0 * logged / max(launches_per_check, 1e-9)
    achieved = bytes_per_launch / (interp_ms / 1e3) / 1e9 if interp_ms else 0.0
    path_ms = interp_ms * launches_per_check + classify_ms_per_check
    path_gbs = 24.0 * logged / (path_ms / 1e3) / 1e9 if path_ms else 0.0
    credited = 12.0 * rep["n_access"] / max(launches_per_check, 1e-9) / (interp_ms / 1e3) / 1e9 if interp_ms else 0.0
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "bytes_rule": "12 B per logged access (written once by the interpreter)",
            "peak_source": peak_source, "avg_launch_ms": interp_ms,
            "launches_per_check": launches_per_check,
            "path": {"what": "log/classify path: 24 B per logged access (log write + classification read) over "
                             "interpreter + classification time per check",
                     "ms_per_check": path_ms, "achieved": path_gbs, "frac": path_gbs / peak,
                     "classify_ms_per_check": classify_ms_per_check},
            "private_credit": {"what": "12 B for every access, private ones included (not moved bytes)",
                               "achieved": credited, "frac": credited / peak}}


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1308_3203_gb300 import build as gpu_build
    from paper_1308_3203_gb300 import racecheck as rc
    from paper_1308_3203_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gpu_build.build()
    rc.load()
    rc.set_strategy(args.strategy)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_source = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6800 GB/s"
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    inst = make_instance(W, args.workload, rank, args.groups)
    full_size = args.groups == 0
    prof_steps = min(args.steps, 5)

    # cold end to end: the process's first check of the program, from host
    # inputs: rc_compile, the pre-filter's analysis of the launch shape and
    # the compile of its interval kernel (NVRTC) included, all of which later
    # checks of the program reuse
    host_np = [torch.from_numpy(a).pin_memory().numpy() for a in inst.globals]
    torch.cuda.synchronize()
    jit0 = rc.jit_stats()
    t0 = time.perf_counter()
    bc = rc.compile(inst.src)
    r_cold = rc.check(bc, inst.groups, inst.group_size, host_np, want_final=False)
    t_cold = time.perf_counter() - t0
    jit1 = rc.jit_stats()
    t0 = time.perf_counter()
    rc.check(bc, inst.groups, inst.group_size, host_np, want_final=False)
    t_warm = time.perf_counter() - t0
    del host_np

    clocks = Clocks(local)
    clocks.start()
    m = measure(rc, inst, bc, steps=args.steps, warmup=args.warmup, dist=dist, flush=flush, prof_steps=prof_steps)
    clk = clocks.stop()

    rep = m["rep"]
    acc_step = rep["n_access"]
    t_max, ms_e2e = combine([m["ms"], m["ms_e2e"]], dist, "max")
    acc_all, = combine([acc_step], dist, "sum")
    value = acc_all * args.steps / (t_max / 1e3)
    e2e = acc_all * args.steps / (ms_e2e / 1e3)

    same_kernel = (args.workload == "stress" and full_size and rank == 0 and
                   INTERP_TRAFFIC["sources_sha256"] == interp_sources_sha256() and
                   INTERP_TRAFFIC["program_sha256"] == hashlib.sha256(inst.src.encode()).hexdigest())
    kname = interval_kernel(rc, inst.groups * inst.group_size)
    roof = roofline(m, hbm, peak_source, INTERP_TRAFFIC["bytes_per_launch"] if same_kernel else None, kname)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + ("" if full_size else f" (reduced to {inst.groups} groups)"),
                   "work_items": inst.groups * inst.group_size,
                   "accesses_per_step": acc_step, "global_accesses_per_step": rep["n_global"],
                   "logged_accesses_per_step": rep["n_logged"],
                   "private_accesses_per_step": acc_step - rep["n_logged"],
                   "race_records_per_step": int((rep["records"][:, 4] < 16).sum()) if len(rep["records"]) else 0,
                   "status": rep["status"], "intervals": rep["n_intervals"],
                   "strategy": {0: "auto", 1: "sort", 2: "shadow", 3: "resident"}[args.strategy],
                   "run": "resident: one cooperative launch per check" if roof["launches_per_check"] == 1
                          else "interval by interval",
                   "private_accesses": "counted and committed, not logged (two-work-item pre-filter); "
                                       "see full_logging for every access logged",
                   "l2": "flushed between steps (256 MiB write); the 256 MiB input exceeds L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": m["h2d"],
                "d2h_bytes_per_step": int(m["rep_e2e"]["records"].nbytes)},
        "e2e_cold": {"what": "the process's first rc_compile + rc_check of the program from host inputs "
                             "(pre-filter analysis and interval-kernel compile included)",
                     "value": r_cold["n_access"] / t_cold, "unit": UNIT, "seconds": t_cold,
                     "warm_seconds": t_warm, "kernel_compiles": jit1["compiles"] - jit0["compiles"]},
        "engine": "compiled intervals" if rc.jit_stats()["compiles"] else "interpreter",
        "gpu_launches": int(m["launches"]),
        "clocks": clk,
    }
    if args.secondary == "all":
        # the same instance with every access logged (no pre-filter)
        f = measure(rc, inst, bc, steps=min(args.steps, 3), warmup=1, dist=dist, flush=flush,
                    log_every=True, host=False, prof_steps=2)
        fr = f["rep"]
        assert fr["n_logged"] == fr["n_access"] and fr["status"] == rep["status"]
        assert np.array_equal(fr["records"], rep["records"]), "the pre-filter changed the report"
        t_f, = combine([f["ms"]], dist, "max")
        acc_f, = combine([fr["n_access"]], dist, "sum")
        out["full_logging"] = {"what": "same instance, every access logged (RC_LOG_EVERY_ACCESS)",
                               "value": acc_f * f["steps"] / (t_f / 1e3), "unit": UNIT,
                               "ms_per_step": t_f / f["steps"], "logged_accesses_per_step": fr["n_logged"],
                               "roofline": roofline(f, hbm, peak_source,
                                                    kernel=interval_kernel(rc, inst.groups * inst.group_size))}
        del f
        if args.workload == "stress":
            # the 1024 x 256 large instance
            li = W.large_kernel(rank)
            lbc = rc.compile(li.src)
            lm = measure(rc, li, lbc, steps=args.steps, warmup=args.warmup, dist=dist, flush=flush,
                         prof_steps=prof_steps)
            t_l, t_le = combine([lm["ms"], lm["ms_e2e"]], dist, "max")
            acc_l, = combine([lm["rep"]["n_access"]], dist, "sum")
            out["large"] = {"workload": WORKLOADS["large"], "value": acc_l * lm["steps"] / (t_l / 1e3),
                            "unit": UNIT, "ms_per_step": t_l / lm["steps"],
                            "e2e": acc_l * lm["steps"] / (t_le / 1e3),
                            "logged_accesses_per_step": lm["rep"]["n_logged"],
                            "accesses_per_step": lm["rep"]["n_access"],
                            "roofline": roofline(lm, hbm, peak_source,
                                                 kernel=interval_kernel(rc, li.groups * li.group_size))}
    if args.secondary in ("all", "small"):
        out["small"] = small_leg(rc, W)
    if args.secondary in ("all", "batch") and args.batch_kernels > 0:
        out["batch"] = batch_leg(rc, W, args.batch_kernels, rank, world, dist, hbm)
    if args.secondary in ("all", "proposal") and args.proposal_kernels > 0:
        out["proposal"] = proposal_leg(rc, args.proposal_kernels)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
        if "small" in out:
            ms = small_oracle_ms()
            out["cpu_baseline"]["small"] = {"ms_per_kernel": ms, "kernels": SMALL_KERNELS, "cores": 1}
            out["small"]["oracle_over_gpu"] = ms * 1e3 / out["small"]["us_per_check"]
            out["small"]["oracle_over_gpu_batched"] = ms * 1e3 / out["small"]["batched_us_per_kernel"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
