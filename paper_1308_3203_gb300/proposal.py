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


def compare_search(model: rc.MLP, seeds, n_cand: int = 64) -> dict:
    """Ranked search vs plain enumeration on each kernel (the same GPU, the
    same checker): checks and seconds to the first racy candidate, and
    whether each search found a race where exhaustive enumeration does."""
    rows = []
    for s in seeds:
        _, items = kernel_candidates(s, n_cand)
        sc = scores(model, rc.features(items))
        enum = rc.search(items)                   # index order = enumeration
        ranked = rc.search(items, scores=sc)
        rows.append(dict(seed=s, racy=enum["first"] >= 0, enum_checks=enum["checks"],
                         enum_s=enum["seconds"], ranked_checks=ranked["checks"], ranked_s=ranked["seconds"],
                         ranked_first=ranked["first"], enum_first=enum["first"],
                         ranked_found=ranked["first"] >= 0))
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
    return out
