"""Reader for the hand-derived golden fixtures in this folder.

Each fixture holds a kernel, its launch shape, its global inputs and the
report the concrete semantics of the paper gives for it, derived by hand
(the derivation and the paper passage are in the fixture's header).
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    sections, cur = {}, None
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            if line.startswith("#"):
                continue
            s = line.rstrip("\n")
            if s.startswith("[") and s.endswith("]"):
                cur = s[1:-1]
                sections[cur] = []
            elif cur is not None and s.strip():
                sections[cur].append(s)
    groups, group_size = map(int, sections["launch"][0].split())
    glob = [np.array([int(x) for x in l.split()], dtype=np.int64).astype(np.int32)
            for l in sections["global"]]
    expect = {k: int(v) for k, v in (l.split() for l in sections["expect"])}
    recs = np.array([[int(x) for x in l.split()] for l in sections.get("records", [])],
                    dtype=np.uint64).astype(np.uint32).reshape(-1, 10)
    final = np.array([int(x) for x in " ".join(sections["final"]).split()],
                     dtype=np.int64).astype(np.int32)
    return dict(src="\n".join(sections["src"]) + "\n", groups=groups, group_size=group_size,
                globals=glob, expect=expect, records=recs, final=final)


def names() -> list:
    return sorted(n for n in os.listdir(HERE) if n.endswith(".txt"))
