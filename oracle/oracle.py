"""ORACLE wrapper (test infrastructure only).

Builds and loads the sequential C++ reference checker (oracle.cpp) and the
brute-force interleaving explorer (explore.cpp).  Only the test suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline leg may import this
module.  It imports nothing from the GPU package and the GPU package imports
nothing from here.

Reports use the same record layout as the GPU library (ten uint32 fields:
interval, space, wg, addr, cls, t_a, t_b, n_readers, n_writers, n_accesses) so
the two can be compared element by element; the layout is restated here, not
shared.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["oracle.cpp", "explore.cpp"]
_HDRS = ["kl_frontend.hpp"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RECORD_FIELDS = ("interval", "space", "wg", "addr", "cls", "t_a", "t_b",
                 "n_readers", "n_writers", "n_accesses")
WW_RACE, WW_BENIGN, RW_RACE = 1, 2, 3
OOB, ASSERT_FAIL, DIVERGENCE = 16, 17, 18
RACE_FREE, RACY, ERROR_OOB, ERROR_ASSERT, ERROR_DIVERGENCE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (plain -O2, no target-specific flags).

    If the environment names a prebuilt library in ``RC_ORACLE_LIB``, that
    library is used as it is: the mutation tests build copies of these
    sources with one planted mistake each and run the pins against them.
    """
    override = os.environ.get("RC_ORACLE_LIB")
    if override:
        return override
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDRS]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp] + srcs
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
        lib.oracle_check.restype = ctypes.c_int
        lib.oracle_check.argtypes = [ctypes.c_char_p, u32, u32, u32, ctypes.POINTER(u64),
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                     ctypes.POINTER(vp), ctypes.c_char_p, ctypes.c_size_t]
        for name, rt in [("oracle_status", i32), ("oracle_n_intervals", u32),
                         ("oracle_n_access", u64), ("oracle_n_global", u64),
                         ("oracle_n_local", u64), ("oracle_n_records", u64),
                         ("oracle_max_acc", u64), ("oracle_max_wr", u64),
                         ("oracle_records", vp), ("oracle_final_len", u64),
                         ("oracle_final", vp), ("oracle_trace_len", u64), ("oracle_trace", vp),
                         ("oracle_n_sites", u64), ("oracle_sites", vp)]:
            getattr(lib, name).restype = rt
            getattr(lib, name).argtypes = [vp]
        lib.oracle_free.argtypes = [vp]
        lib.oracle_free.restype = None
        lib.explore_check.restype = ctypes.c_int
        lib.explore_check.argtypes = [ctypes.c_char_p, u32, u32, u32, ctypes.POINTER(u64),
                                      ctypes.POINTER(ctypes.c_void_p), u64,
                                      ctypes.POINTER(vp), ctypes.c_char_p, ctypes.c_size_t]
        for name, rt, extra in [("explore_n_intervals", u32, []), ("explore_end_states", u32, [u32]),
                                ("explore_deviated", ctypes.c_int, [u32]),
                                ("explore_n_final", u32, []), ("explore_finals", vp, []),
                                ("explore_diverged", ctypes.c_int, []),
                                ("explore_overflow", ctypes.c_int, [])]:
            getattr(lib, name).restype = rt
            getattr(lib, name).argtypes = [vp] + extra
        lib.explore_pairs_check.restype = ctypes.c_int
        lib.explore_pairs_check.argtypes = lib.explore_check.argtypes
        lib.explore_n_pairs.restype = u32
        lib.explore_n_pairs.argtypes = [vp, u32]
        lib.explore_pairs.restype = vp
        lib.explore_pairs.argtypes = [vp, u32]
        lib.explore_free.argtypes = [vp]
        lib.explore_free.restype = None
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _marshal(globals_):
    arrs = [np.ascontiguousarray(np.asarray(g, dtype=np.int32)) for g in globals_]
    n = len(arrs)
    lens = (ctypes.c_uint64 * max(n, 1))(*[a.size for a in arrs])
    ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in arrs])
    return arrs, n, lens, ptrs


def check(src: str, groups: int, group_size: int, globals_, reverse: bool = False,
          group_barriers: bool = False, shard: tuple = (0, 1), trace: bool = False) -> dict:
    """Run the reference checker on one instance.

    ``globals_`` is one int32 array per ``global`` declaration, in order.
    ``group_barriers`` takes barriers as work-group scoped (per-group barrier
    agreement, cross-group records of the whole run).  ``shard = (p, P)``
    logs and classifies only the cells of address shard p of P (the run is
    the full one; only shard 0 reports errors); ``check_sharded`` merges.
    Returns dict(status, n_intervals, n_access, n_global, n_local,
    records (uint32 [n, 10]), final (int32, all global arrays concatenated)).
    ``trace`` adds every performed shared access, trace (uint32 [n, 8]:
    interval, gtid, space, wg, addr, write, site, value stored or loaded as
    uint32), and sites (uint32 [k, 2]: write, memory object of the k-th
    load/store command in text order).
    """
    lib = _load()
    arrs, n, lens, ptrs = _marshal(globals_)
    h = ctypes.c_void_p()
    err = ctypes.create_string_buffer(512)
    rc = lib.oracle_check(src.encode(), groups, group_size, n, lens, ptrs,
                          (1 if reverse else 0) | (2 if group_barriers else 0) | (4 if trace else 0) |
                          ((shard[0] << 8) | (shard[1] << 20) if shard[1] > 1 else 0),
                          ctypes.byref(h), err, 512)
    if rc != 0:
        raise OracleError(f"oracle rc={rc}: {err.value.decode()}")
    try:
        nrec = lib.oracle_n_records(h)
        recs = np.zeros((nrec, 10), dtype=np.uint32)
        if nrec:
            ctypes.memmove(recs.ctypes.data, lib.oracle_records(h), nrec * 40)
        nfin = lib.oracle_final_len(h)
        fin = np.zeros(nfin, dtype=np.int32)
        if nfin:
            ctypes.memmove(fin.ctypes.data, lib.oracle_final(h), nfin * 4)
        out = dict(status=lib.oracle_status(h), n_intervals=lib.oracle_n_intervals(h),
                   n_access=lib.oracle_n_access(h), n_global=lib.oracle_n_global(h),
                   n_local=lib.oracle_n_local(h), records=recs, final=fin,
                   max_acc=lib.oracle_max_acc(h), max_wr=lib.oracle_max_wr(h))
        if trace:
            nt, ns = lib.oracle_trace_len(h), lib.oracle_n_sites(h)
            out["trace"] = np.zeros((nt, 8), dtype=np.uint32)
            out["sites"] = np.zeros((ns, 2), dtype=np.uint32)
            if nt:
                ctypes.memmove(out["trace"].ctypes.data, lib.oracle_trace(h), nt * 32)
            if ns:
                ctypes.memmove(out["sites"].ctypes.data, lib.oracle_sites(h), ns * 8)
        return out
    finally:
        lib.oracle_free(h)


def explore(src: str, groups: int, group_size: int, globals_, max_states: int = 2_000_000) -> dict:
    """Enumerate every schedule of a tiny instance (true shared memory).

    Returns dict(end_states [per interval], deviated [per interval],
    finals (list of int32 arrays), diverged, overflow).
    """
    lib = _load()
    arrs, n, lens, ptrs = _marshal(globals_)
    h = ctypes.c_void_p()
    err = ctypes.create_string_buffer(512)
    rc = lib.explore_check(src.encode(), groups, group_size, n, lens, ptrs, max_states,
                           ctypes.byref(h), err, 512)
    if rc != 0:
        raise OracleError(f"explorer rc={rc}: {err.value.decode()}")
    try:
        k = lib.explore_n_intervals(h)
        ends = [lib.explore_end_states(h, i) for i in range(k)]
        dev = [bool(lib.explore_deviated(h, i)) for i in range(k)]
        nf = lib.explore_n_final(h)
        tot = sum(a.size for a in arrs)
        fin = np.zeros(nf * tot, dtype=np.int32)
        if nf * tot:
            ctypes.memmove(fin.ctypes.data, lib.explore_finals(h), nf * tot * 4)
        finals = [fin[i * tot:(i + 1) * tot] for i in range(nf)]
        return dict(end_states=ends, deviated=dev, finals=finals,
                    diverged=bool(lib.explore_diverged(h)), overflow=bool(lib.explore_overflow(h)))
    finally:
        lib.explore_free(h)


def explore_pairs(src: str, groups: int, group_size: int, globals_, max_states: int = 2_000_000) -> list:
    """The interleaving product of every two work-items i < j (all others
    frozen), per interval that starts from a single state: a list per
    interval, None where the interval starts from several states, else one
    (end_states, deviated) tuple per pair in (i, j) order."""
    lib = _load()
    arrs, n, lens, ptrs = _marshal(globals_)
    h = ctypes.c_void_p()
    err = ctypes.create_string_buffer(512)
    rc = lib.explore_pairs_check(src.encode(), groups, group_size, n, lens, ptrs, max_states,
                                 ctypes.byref(h), err, 512)
    if rc != 0:
        raise OracleError(f"explorer rc={rc}: {err.value.decode()}")
    try:
        if lib.explore_overflow(h):
            raise OracleError("explorer state budget exceeded")
        out = []
        for k in range(lib.explore_n_intervals(h)):
            m = lib.explore_n_pairs(h, k)
            if m == 0:
                out.append(None)
                continue
            v = np.zeros(m, dtype=np.uint32)
            ctypes.memmove(v.ctypes.data, lib.explore_pairs(h, k), m * 4)
            out.append([(int(x & 0x7FFFFFFF), bool(x >> 31)) for x in v])
        return out
    finally:
        lib.explore_free(h)


def _shard_job(args):
    src, groups, group_size, globals_, group_barriers, p, n_shards = args
    return check(src, groups, group_size, globals_, group_barriers=group_barriers, shard=(p, n_shards))


def check_sharded(src: str, groups: int, group_size: int, globals_, n_shards: int,
                  group_barriers: bool = False, processes: int = 1) -> dict:
    """The report of an address-sharded run: the P shards run one after the
    other, or in `processes` spawn-started processes, their race records
    merged in report order, shard 0's error records after them, the status
    from the merged records."""
    jobs = [(src, groups, group_size, [np.asarray(g) for g in globals_], group_barriers, p, n_shards)
            for p in range(n_shards)]
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(processes, n_shards)) as pool:
            parts = pool.map(_shard_job, jobs)
    else:
        parts = [_shard_job(j) for j in jobs]
    races = np.concatenate([r["records"][r["records"][:, 4] < 16] for r in parts])
    if len(races):
        order = np.lexsort(tuple(races[:, k] for k in (4, 3, 2, 1, 0)))
        races = races[order]
    errs = parts[0]["records"][parts[0]["records"][:, 4] >= 16]
    cls = set(int(c) for c in races[:, 4]) if len(races) else set()
    ecl = set(int(c) for c in errs[:, 4]) if len(errs) else set()
    status = 1 if cls & {1, 3, 4, 6} else 4 if 18 in ecl else 3 if 17 in ecl else 2 if 16 in ecl else 0
    out = dict(parts[0])
    out["records"] = np.concatenate([races.reshape(-1, 10), errs.reshape(-1, 10)]).astype(np.uint32)
    out["status"] = status
    return out
