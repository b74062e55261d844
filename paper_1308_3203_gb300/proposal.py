"""Learned proposal: rank a kernel's candidate instances so that the exact
checker meets a racy one sooner.

Pipeline (every computation in the library; this module only moves arrays):
  1. candidates of each kernel: (groups, group_size, input seed) instances;
  2. labels: the exact checker's verdict on every training candidate
     (rc_check_batch; racy = report status RC_RACY);
  3. features: rc_features_batch (host C++ in the library);
  4. training: rc_mlp_train (BF16 tensor-core forward/backward, Adam);
  5. search: scores from rc_mlp_forward, then rc_search checks candidates in
     descending score order until the first racy report.  Plain enumeration
     is rc_search without scores.  A race is claimed only from a checker
     report, so the precision of every flag is that of the checker.
"""
from __future__ import annotations

import numpy as np

from . import racecheck as rc
from . import workloads as W


def kernel_candidates(seed: int, n_cand: int = 64):
    """(bytecode, candidate items) of proposal kernel `seed`."""
    pk = W.proposal_kernel(seed)
    bc = rc.compile(pk.src)
    items = [(bc, G, S, pk.instance(G, S, i).globals) for (G, S, i) in W.proposal_candidates(seed, n_cand)]
    return bc, items


def label(items, chunk: int = 4096) -> np.ndarray:
    """1 where the checker reports a race, else 0."""
    out = []
    for i in range(0, len(items), chunk):
        reps = rc.check_batch(items[i:i + chunk], want_final=False)
        out += [1.0 if r["status"] == rc.RACY else 0.0 for r in reps]
    return np.asarray(out, dtype=np.float32)


def dataset(seeds, n_cand: int = 64):
    """Features [n, 128], labels [n], kernel index [n] for every candidate of
    the given kernels."""
    items, kid = [], []
    for k, s in enumerate(seeds):
        _, it = kernel_candidates(s, n_cand)
        items += it
        kid += [k] * len(it)
    return rc.features(items), label(items), np.asarray(kid, dtype=np.int64)


def scores(model: rc.MLP, X: np.ndarray) -> np.ndarray:
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    return model.forward(x).cpu().numpy()


# Feature columns the rule-based ranking reads (rc_features' layout): some
# access of the kernel must put two work-items of the candidate's launch
# shape on one cell with a store whose value varies (108); a race among the
# sampled work-items' accesses (107); sampled write/write and read/write
# collisions (104, 105).
F_PREDICTED, F_SAMPLED, F_WW, F_RW = 108, 107, 104, 105


def rule_scores(X: np.ndarray) -> np.ndarray:
    """The ranking without a network: candidates whose features predict a
    race first, then those with sampled collisions, more collisions first;
    ties keep the index order."""
    return 4.0 * X[:, F_PREDICTED] + 2.0 * X[:, F_SAMPLED] + 0.1 * (X[:, F_WW] + X[:, F_RW])


def compare_search(model: rc.MLP, seeds, n_cand: int = 64) -> dict:
    """Three searches of each kernel's candidates on the same GPU with the
    same checker: ranked by the trained network, ranked by the rule above
    (no network), and plain enumeration (index order).  Per search: checks
    and seconds to the first racy candidate, and whether it found a race
    where exhaustive enumeration does; `*_total_s` adds the cost of ranking
    (feature extraction, and the network's inference for the network)."""
    import time
    import torch
    rows = []
    for s in seeds:
        _, items = kernel_candidates(s, n_cand)
        t0 = time.perf_counter()
        X = rc.features(items)
        t_feat = time.perf_counter() - t0
        t0 = time.perf_counter()
        sc = scores(model, X)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        enum = rc.search(items)                   # index order = enumeration
        ranked = rc.search(items, scores=sc)
        rule = rc.search(items, scores=rule_scores(X))
        rows.append(dict(seed=s, racy=enum["first"] >= 0, enum_checks=enum["checks"],
                         enum_s=enum["seconds"], ranked_checks=ranked["checks"], ranked_s=ranked["seconds"],
                         ranked_first=ranked["first"], enum_first=enum["first"],
                         ranked_found=ranked["first"] >= 0,
                         ranked_total_s=ranked["seconds"] + t_feat + t_inf,
                         rule_checks=rule["checks"], rule_s=rule["seconds"], rule_found=rule["first"] >= 0,
                         rule_total_s=rule["seconds"] + t_feat, features_s=t_feat, inference_s=t_inf))
    return summarize(rows)


def summarize(rows) -> dict:
    racy = [r for r in rows if r["racy"]]
    out = dict(kernels=len(rows), racy_kernels=len(racy), rows=rows)
    if racy:
        te = sum(r["enum_s"] for r in racy)
        tr = sum(r["ranked_s"] for r in racy)
        out.update(enum_seconds=te, ranked_seconds=tr, speedup=te / tr if tr > 0 else float("inf"),
                   enum_checks_mean=float(np.mean([r["enum_checks"] for r in racy])),
                   ranked_checks_mean=float(np.mean([r["ranked_checks"] for r in racy])),
                   recall=float(np.mean([r["ranked_found"] for r in racy])))
        for k in (1, 2, 4, 8):
            out[f"recall_at_{k}"] = float(np.mean([r["ranked_found"] and r["ranked_checks"] <= k for r in racy]))
        if "rule_checks" in racy[0]:
            tt = sum(r["ranked_total_s"] for r in racy)
            tu = sum(r["rule_total_s"] for r in racy)
            out.update(ranked_total_seconds=tt, speedup_total=te / tt if tt > 0 else float("inf"),
                       features_seconds=sum(r["features_s"] for r in racy),
                       inference_seconds=sum(r["inference_s"] for r in racy),
                       rule_seconds=sum(r["rule_s"] for r in racy), rule_total_seconds=tu,
                       rule_speedup_total=te / tu if tu > 0 else float("inf"),
                       rule_checks_mean=float(np.mean([r["rule_checks"] for r in racy])),
                       rule_recall=float(np.mean([r["rule_found"] for r in racy])))
            for k in (1, 2, 4, 8):
                out[f"rule_recall_at_{k}"] = float(np.mean([r["rule_found"] and r["rule_checks"] <= k
                                                            for r in racy]))
    return out
