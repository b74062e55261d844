"""Learned proposal: rank a kernel's candidate instances so that the exact
checker meets a racy one sooner.

Pipeline (every computation in the library; this module only moves arrays):
  1. candidates of each kernel: (groups, group_size, input seed) instances;
  2. labels: the exact checker's verdict on every training candidate
     (rc_check_batch; racy = report status RC_RACY);
  3. features: rc_features_batch (host C++ in the library);
  4. training: rc_mlp_train (BF16 tensor-core forward/backward, Adam);
  5. search: rc_search_ranked computes the features, scores them with
     rc_mlp_forward and checks candidates in descending score order until
     the first racy report (optionally checking in index order while the
     ranking is computed).  Plain enumeration is rc_search without scores.
     A race is claimed only from a checker report, so the precision of
     every flag is that of the checker.
"""
from __future__ import annotations

import numpy as np

from . import racecheck as rc
from . import workloads as W


FAMILIES = {"proposal": W.proposal_kernel, "batch": W.batch_proposal_kernel}


def kernel_candidates(seed: int, n_cand: int = 64, family: str = "proposal"):
    """(bytecode, candidate items) of kernel `seed` of a family: "proposal"
    (races that depend on the candidate) or "batch" (the config-3 generator's
    programs)."""
    pk = FAMILIES[family](seed)
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


def dataset(seeds, n_cand: int = 64, family: str = "proposal", chunk_kernels: int = 256):
    """Features [n, 128], labels [n], kernel index [n] for every candidate of
    the given kernels, built `chunk_kernels` kernels at a time (a chunk's
    inputs are dropped once its features and labels exist, so the host holds
    one chunk of inputs at most)."""
    seeds = list(seeds)
    Xs, ys, kids = [], [], []
    for c0 in range(0, len(seeds), chunk_kernels):
        items, kid = [], []
        for k in range(c0, min(len(seeds), c0 + chunk_kernels)):
            _, it = kernel_candidates(seeds[k], n_cand, family)
            items += it
            kid += [k] * len(it)
        Xs.append(rc.features(items))
        ys.append(label(items))
        kids.append(np.asarray(kid, dtype=np.int64))
        del items
    if not Xs:
        return np.zeros((0, rc.N_FEATURES), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int64)
    return np.concatenate(Xs), np.concatenate(ys), np.concatenate(kids)


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
    """The ranking rc_search_ranked uses without a network, in the same
    float32 arithmetic: candidates whose features predict a race first, then
    those with sampled collisions, more collisions first; ties keep the
    index order."""
    X = np.asarray(X, dtype=np.float32)
    return (np.float32(4) * X[:, F_PREDICTED] + np.float32(2) * X[:, F_SAMPLED]
            + (X[:, F_WW] + X[:, F_RW]) / np.float32(10))


def compare_search(model: rc.MLP, seeds, n_cand: int = 64, warmup_seed: int = 10**9,
                   family: str = "proposal") -> dict:
    """Searches of each kernel's candidates on the same GPU with the same
    checker, in this order:
      enum      plain enumeration (index order, rc_search without scores);
      ranked    rc_search_ranked with the trained network: features on the
                host threads, then network scores, then checks in order;
      overlap   the same with RC_RANK_OVERLAP (index-order checks while the
                ranking is computed);
      rule      rc_search_ranked without a network (the rule ranking);
      rule_overlap  the rule with RC_RANK_OVERLAP.
    Per search: checks and seconds to the first racy candidate (for the
    ranked searches the whole call: features, scores and checks; `*_check_s`
    the checks alone), and whether it found a race where exhaustive
    enumeration does.  One kernel outside `seeds` is searched first, every
    way, untimed (thread pool and workspace set-up)."""
    kinds = dict(ranked=(model, False), overlap=(model, True), rule=(None, False), rule_overlap=(None, True))
    _, items = kernel_candidates(warmup_seed, n_cand, family)
    rc.search(items)
    for m, ov in kinds.values():
        rc.search_ranked(items, m, overlap=ov)
    rows = []
    for s in seeds:
        _, items = kernel_candidates(s, n_cand, family)
        enum = rc.search(items)                   # index order = enumeration
        row = dict(seed=s, racy=enum["first"] >= 0, enum_checks=enum["checks"], enum_s=enum["seconds"],
                   enum_first=enum["first"])
        for k, (m, ov) in kinds.items():
            r = rc.search_ranked(items, m, overlap=ov)
            row.update({f"{k}_checks": r["checks"], f"{k}_s": r["seconds"], f"{k}_check_s": r["check_seconds"],
                        f"{k}_features_s": r["features_seconds"], f"{k}_scoring_s": r["scoring_seconds"],
                        f"{k}_unranked": r["checks_unranked"], f"{k}_first": r["first"],
                        f"{k}_found": r["first"] >= 0})
        rows.append(row)
    return summarize(rows)


def summarize(rows) -> dict:
    """Totals over the kernels enumeration finds racy: seconds and speed-up
    against enumeration per search, mean checks, recall and recall@k (a race
    within k checks)."""
    racy = [r for r in rows if r["racy"]]
    out = dict(kernels=len(rows), racy_kernels=len(racy), rows=rows)
    if not racy:
        return out
    te = sum(r["enum_s"] for r in racy)
    out.update(enum_seconds=te, enum_checks_mean=float(np.mean([r["enum_checks"] for r in racy])))
    for k in ("ranked", "overlap", "rule", "rule_overlap"):
        t = sum(r[f"{k}_s"] for r in racy)
        tc = sum(r[f"{k}_check_s"] for r in racy)
        out[k] = dict(seconds=t, speedup=te / t if t > 0 else float("inf"),
                      check_seconds=tc, check_speedup=te / tc if tc > 0 else float("inf"),
                      features_seconds=sum(r[f"{k}_features_s"] for r in racy),
                      scoring_seconds=sum(r[f"{k}_scoring_s"] for r in racy),
                      checks_mean=float(np.mean([r[f"{k}_checks"] for r in racy])),
                      unranked_checks_mean=float(np.mean([r[f"{k}_unranked"] for r in racy])),
                      recall=float(np.mean([r[f"{k}_found"] for r in racy])))
        for j in (1, 2, 4, 8):
            out[k][f"recall_at_{j}"] = float(np.mean([r[f"{k}_found"] and r[f"{k}_checks"] <= j for r in racy]))
    return out
