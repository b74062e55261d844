"""Python binding of libracecheck.so (argument marshalling only).

Every step of a check runs in the CUDA library; this module converts numpy
arrays or torch tensors to the pointers and lengths of the C ABI declared in
include/racecheck.h and turns reports into numpy arrays.  If the library has
not been built, importing functions here raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libracecheck.so")

RECORD_FIELDS = ("interval", "space", "wg", "addr", "cls", "t_a", "t_b",
                 "n_readers", "n_writers", "n_accesses")
WW_RACE, WW_BENIGN, RW_RACE = 1, 2, 3
XG_WW_RACE, XG_WW_BENIGN, XG_RW_RACE = 4, 5, 6
OOB, ASSERT_FAIL, DIVERGENCE = 16, 17, 18
RACE_FREE, RACY, ERROR_OOB, ERROR_ASSERT, ERROR_DIVERGENCE = 0, 1, 2, 3, 4
STRATEGY_AUTO, STRATEGY_SORT, STRATEGY_SHADOW, STRATEGY_RESIDENT = 0, 1, 2, 3
RC_WANT_FINAL_MEMORY = 1
RC_GROUP_BARRIERS = 2
RC_LOG_EVERY_ACCESS = 4


class RaceCheckError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rc error {code}: {msg}")
        self.code = code


class _Input(ctypes.Structure):
    _fields_ = [("n_global", ctypes.c_uint32),
                ("global_len", ctypes.POINTER(ctypes.c_uint64)),
                ("global_init", ctypes.POINTER(ctypes.c_void_p)),
                ("on_device", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p),
                ("flags", ctypes.c_uint32)]


class _Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_intervals", ctypes.c_uint32),
                ("n_access", ctypes.c_uint64), ("n_global", ctypes.c_uint64),
                ("n_local", ctypes.c_uint64), ("n_records", ctypes.c_uint64),
                ("records", ctypes.c_void_p), ("final_len", ctypes.c_uint64),
                ("final_global", ctypes.c_void_p), ("n_logged", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("n_insn", "n_regs", "n_vars", "n_mems", "n_global", "n_barriers", "n_asserts",
                 "local_cells")] + [("max_access_per_interval", ctypes.c_uint64),
                                    ("max_write_per_interval", ctypes.c_uint64)]


class _ExploreInterval(ctypes.Structure):
    _fields_ = [("interval", ctypes.c_uint32), ("n_end_states", ctypes.c_uint32), ("deviated", ctypes.c_uint32),
                ("complete", ctypes.c_uint32), ("n_states", ctypes.c_uint64)]


class _PairInterval(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("interval", "n_pairs", "n_racy", "n_deviated", "first_i",
                                               "first_j", "complete", "reserved")] + [("n_states", ctypes.c_uint64)]


class _ProveResult(ctypes.Structure):
    _fields_ = [("race_free", ctypes.c_int32), ("in_bounds", ctypes.c_int32), ("first_pc_a", ctypes.c_uint32),
                ("first_pc_b", ctypes.c_uint32), ("n_pairs", ctypes.c_uint32), ("n_unresolved", ctypes.c_uint32)]


class _SearchResult(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("checks", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("seconds", ctypes.c_double)]


class _RankedResult(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("checks", ctypes.c_uint32), ("checks_unranked", ctypes.c_uint32),
                ("seconds", ctypes.c_double), ("features_seconds", ctypes.c_double),
                ("scoring_seconds", ctypes.c_double), ("check_seconds", ctypes.c_double)]


RC_RANK_OVERLAP = 1


N_FEATURES = 128
MLP_PARAMS = 164865

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libracecheck.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1308_3203_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, c_int = ctypes.c_void_p, ctypes.c_int
        lib.rc_compile.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(vp),
                                   ctypes.c_char_p, ctypes.c_size_t]
        lib.rc_bytecode_info_get.argtypes = [vp, ctypes.POINTER(_Info)]
        lib.rc_check.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input),
                                 ctypes.POINTER(ctypes.POINTER(_Report))]
        lib.rc_check_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_Input),
                                       ctypes.c_size_t, ctypes.POINTER(ctypes.POINTER(_Report))]
        lib.rc_bytecode_free.argtypes = [vp]
        lib.rc_bytecode_free.restype = None
        lib.rc_report_free.argtypes = [ctypes.POINTER(_Report)]
        lib.rc_report_free.restype = None
        lib.rc_strerror.argtypes = [c_int]
        lib.rc_strerror.restype = ctypes.c_char_p
        lib.rc_last_error.argtypes = []
        lib.rc_last_error.restype = ctypes.c_char_p
        lib.rc_set_strategy.argtypes = [c_int]
        lib.rc_set_engine.argtypes = [c_int]
        lib.rc_set_engine.restype = c_int
        lib.rc_jit_compile.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input), c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]
        lib.rc_jit_compile.restype = c_int
        lib.rc_jit_stats.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]
        lib.rc_jit_stats.restype = c_int
        lib.rc_profile_enable.argtypes = [c_int]
        lib.rc_profile_get.argtypes = [c_int, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        lib.rc_sort_accesses.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp]
        lib.rc_sort_accesses.restype = c_int
        lib.rc_sort_accesses_noalloc.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vp]
        lib.rc_sort_accesses_noalloc.restype = c_int
        lib.rc_autotune_config.argtypes = [ctypes.c_char_p]
        lib.rc_autotune_config.restype = c_int
        lib.rc_autotune_reset.argtypes = []
        lib.rc_autotune_reset.restype = c_int
        lib.rc_autotune_lookup.argtypes = [c_int, ctypes.c_uint64, ctypes.c_uint64]
        lib.rc_autotune_lookup.restype = c_int
        lib.rc_kernel_launches.argtypes = []
        lib.rc_kernel_launches.restype = ctypes.c_uint64
        fp = ctypes.POINTER(ctypes.c_float)
        lib.rc_features_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint32),
                                          ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_Input),
                                          ctypes.c_size_t, fp, c_int]
        lib.rc_mlp_create.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(vp)]
        lib.rc_mlp_free.argtypes = [vp]
        lib.rc_mlp_free.restype = None
        lib.rc_mlp_get_params.argtypes = [vp, fp]
        lib.rc_mlp_set_params.argtypes = [vp, fp]
        lib.rc_mlp_forward.argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
        lib.rc_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_uint32, fp, fp, vp]
        lib.rc_mlp_train.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_float, ctypes.c_uint64, fp, vp]
        lib.rc_search.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_Input), ctypes.c_size_t,
                                  fp, ctypes.c_uint32, ctypes.POINTER(_SearchResult),
                                  ctypes.POINTER(ctypes.POINTER(_Report))]
        lib.rc_search_ranked.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_Input), ctypes.c_size_t,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_RankedResult),
                                         ctypes.POINTER(ctypes.POINTER(_Report))]
        lib.rc_explore.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input), ctypes.c_uint64,
                                   ctypes.POINTER(_ExploreInterval), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        lib.rc_explore_pairs.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input),
                                         ctypes.c_uint64, ctypes.POINTER(_PairInterval), ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]
        lib.rc_mlp_set_backend.argtypes = [vp, c_int]
        lib.rc_mlp_backend_error.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
        lib.rc_prove.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input),
                                 ctypes.POINTER(_ProveResult)]
        lib.rc_prove_private.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_Input),
                                         ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_uint32)]
        lib.rc_access_sites.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint8),
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint32)]
        lib.rc_translate.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_size_t)]
        for f in ("rc_prove", "rc_prove_private", "rc_access_sites", "rc_translate", "rc_mlp_set_backend", "rc_mlp_backend_error", "rc_explore", "rc_explore_pairs", "rc_features_batch", "rc_mlp_create", "rc_mlp_get_params", "rc_mlp_set_params",
                  "rc_mlp_forward", "rc_mlp_grad", "rc_mlp_train", "rc_search", "rc_search_ranked"):
            getattr(lib, f).restype = c_int
        for f in ("rc_compile", "rc_bytecode_info_get", "rc_check", "rc_check_batch",
                  "rc_set_strategy", "rc_profile_enable", "rc_profile_reset", "rc_profile_get",
                  "rc_release_workspace"):
            getattr(lib, f).restype = c_int
        _lib = lib
        return lib


def _raise(code: int):
    lib = load()
    raise RaceCheckError(code, lib.rc_last_error().decode(errors="replace")
                         or lib.rc_strerror(code).decode())


class Bytecode:
    """A compiled kernel (library-owned bytecode)."""

    def __init__(self, handle, src: str):
        self._h = handle
        self.src = src

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _Info()
        rc = load().rc_bytecode_info_get(self._h, ctypes.byref(i))
        if rc:
            _raise(rc)
        return {n: getattr(i, n) for n, _ in _Info._fields_}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rc_bytecode_free(self._h)
            self._h = None


def compile(src: str) -> Bytecode:  # noqa: A001 - the paper's rc_compile
    lib = load()
    h = ctypes.c_void_p()
    err = ctypes.create_string_buffer(1024)
    b = src.encode()
    rc = lib.rc_compile(b, len(b), ctypes.byref(h), err, 1024)
    if rc:
        raise RaceCheckError(rc, err.value.decode(errors="replace"))
    return Bytecode(h, src)


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _marshal(globals_, stream, want_final):
    keep = []
    lens, ptrs = [], []
    on_device = bool(globals_) and all(_is_torch_cuda(g) for g in globals_)
    for g in globals_:
        if on_device:
            if str(g.dtype) != "torch.int32" or not g.is_contiguous():
                raise ValueError("device inputs must be contiguous int32 tensors")
            keep.append(g)
            lens.append(g.numel())
            ptrs.append(g.data_ptr())
        else:
            a = np.ascontiguousarray(np.asarray(g.cpu() if hasattr(g, "cpu") else g, dtype=np.int32))
            keep.append(a)
            lens.append(a.size)
            ptrs.append(a.ctypes.data if a.size else None)
    n = len(keep)
    clens = (ctypes.c_uint64 * max(n, 1))(*lens)
    cptrs = (ctypes.c_void_p * max(n, 1))(*ptrs)
    if stream is None and on_device:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    inp = _Input(n, clens, cptrs, 1 if on_device else 0,
                 ctypes.c_void_p(int(stream) if stream else 0),
                 RC_WANT_FINAL_MEMORY if want_final else 0)
    return inp, (keep, clens, cptrs)


class _ReportMemory:
    """Owns an rc_report: the record and final-memory arrays of the Python
    report are views of the library's own arrays (no copy), and the report
    is freed when the last of them is gone."""

    def __init__(self, lib, p):
        self.lib, self.p = lib, p

    def __del__(self):
        if self.p is not None:
            try:
                self.lib.rc_report_free(self.p)
            except Exception:  # the library already unloaded at interpreter exit
                pass
            self.p = None


class _ArrayView:
    """numpy's array interface over n values of dtype at addr; the array made
    from it keeps this object, and so the report, alive."""
    __slots__ = ("_owner", "__array_interface__")

    def __init__(self, owner: _ReportMemory, addr: int, n: int, dtype):
        self._owner = owner
        self.__array_interface__ = {"data": (addr, False), "shape": (n,), "typestr": np.dtype(dtype).str,
                                    "version": 3}


def _view(owner: _ReportMemory, addr: int, n: int, dtype) -> np.ndarray:
    return np.asarray(_ArrayView(owner, addr, n, dtype))


def _report(p) -> dict:
    r = p.contents
    owner = _ReportMemory(load(), p)
    if r.n_records:
        recs = _view(owner, r.records, r.n_records * 10, np.uint32).reshape(r.n_records, 10)
    else:
        recs = np.zeros((0, 10), dtype=np.uint32)
    fin = _view(owner, r.final_global, r.final_len, np.int32) if r.final_global else None
    return dict(status=r.status, n_intervals=r.n_intervals, n_access=r.n_access,
                n_global=r.n_global, n_local=r.n_local, n_logged=r.n_logged, records=recs, final=fin)


def check(bc: Bytecode, groups: int, group_size: int, globals_, stream=None,
          want_final: bool = True, group_barriers: bool = False, log_every_access: bool = False) -> dict:
    """Check one instance.  ``globals_``: one int32 array per ``global``
    declaration (numpy / host tensors, or contiguous int32 CUDA tensors).
    ``group_barriers``: barriers are work-group scoped (RC_GROUP_BARRIERS).
    ``log_every_access``: no access is taken as private (RC_LOG_EVERY_ACCESS)."""
    lib = load()
    inp, keep = _marshal(globals_, stream, want_final)
    if group_barriers:
        inp.flags |= RC_GROUP_BARRIERS
    if log_every_access:
        inp.flags |= RC_LOG_EVERY_ACCESS
    out = ctypes.POINTER(_Report)()
    rc = lib.rc_check(bc.handle, groups, group_size, ctypes.byref(inp), ctypes.byref(out))
    del keep
    if rc:
        _raise(rc)
    return _report(out)


def check_batch(items, want_final: bool = True) -> list:
    """Check many instances: items = [(bytecode, groups, group_size, globals)]."""
    lib = load()
    n = len(items)
    hs = (ctypes.c_void_p * max(n, 1))(*[it[0].handle.value for it in items])
    gs = (ctypes.c_uint32 * max(n, 1))(*[it[1] for it in items])
    ss = (ctypes.c_uint32 * max(n, 1))(*[it[2] for it in items])
    inputs = (_Input * max(n, 1))()
    keep = []
    for i, it in enumerate(items):
        inp, k = _marshal(it[3], None, want_final)
        inputs[i] = inp
        keep.append(k)
    outs = (ctypes.POINTER(_Report) * max(n, 1))()
    rc = lib.rc_check_batch(hs, gs, ss, inputs, n, outs)
    if rc:
        _raise(rc)
    return [_report(outs[i]) for i in range(n)]


def set_strategy(k: int) -> None:
    rc = load().rc_set_strategy(k)
    if rc:
        _raise(rc)


ENGINES = {"auto": 0, "interpreter": 1, "compiled": 2}


def set_engine(engine) -> None:
    """Engine of the interval kernels: "auto", "interpreter" or "compiled"
    (or 0, 1, 2)."""
    rc = load().rc_set_engine(ENGINES.get(engine, engine) if isinstance(engine, str) else engine)
    if rc:
        _raise(rc)


def jit_compile(bc: Bytecode, groups: int, group_size: int, globals_, resident: bool = False) -> dict:
    """Compile (without loading) the interval kernel of an instance: a check
    of the generated source that needs no GPU."""
    lib = load()
    inp, keep = _marshal(globals_, None, False)
    sec, nb = ctypes.c_double(), ctypes.c_uint64()
    rc = lib.rc_jit_compile(bc.handle, groups, group_size, ctypes.byref(inp), 1 if resident else 0,
                            ctypes.byref(sec), ctypes.byref(nb))
    del keep
    if rc:
        _raise(rc)
    return {"seconds": sec.value, "cubin_bytes": nb.value}


def jit_stats() -> dict:
    n, sec = ctypes.c_uint64(), ctypes.c_double()
    rc = load().rc_jit_stats(ctypes.byref(n), ctypes.byref(sec))
    if rc:
        _raise(rc)
    return {"compiles": n.value, "seconds": sec.value}


def profile_enable(on: bool = True) -> None:
    load().rc_profile_enable(1 if on else 0)


def profile_reset() -> None:
    load().rc_profile_reset()


def profile_get(kind: int) -> dict:
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    rc = load().rc_profile_get(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
    if rc:
        _raise(rc)
    return dict(launches=n.value, ms=ms.value, bytes=by.value)


def release_workspace() -> None:
    load().rc_release_workspace()


def diag_grid_barrier(limit_us: int) -> tuple:
    """Run the resident runs' failure-path diagnostic: a grid barrier that
    cannot complete must give up after limit_us; returns (timed_out, seconds)."""
    lib = load()
    lib.rc_diag_grid_barrier.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.rc_diag_grid_barrier.restype = ctypes.c_int
    t, sec = ctypes.c_int32(), ctypes.c_double()
    rc = lib.rc_diag_grid_barrier(limit_us, ctypes.byref(t), ctypes.byref(sec))
    if rc:
        _raise(rc)
    return bool(t.value), sec.value


def kernel_launches() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(load().rc_kernel_launches())


def sort_accesses(records_in, records_out, cell_bits: int, item_bits: int, stream=None) -> None:
    """Sort device access records (int32 CUDA tensors of shape [n, 4]: cell,
    item|write<<31, value, seq) by (cell, work-item) into records_out."""
    n = records_in.shape[0]
    if records_out.shape != records_in.shape:
        raise ValueError("records_out must have the shape of records_in")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    rc = load().rc_sort_accesses(ctypes.c_void_p(records_in.data_ptr()), ctypes.c_void_p(records_out.data_ptr()),
                                 n, cell_bits, item_bits, ctypes.c_void_p(int(stream) if stream else 0))
    if rc:
        _raise(rc)


def sort_accesses_noalloc(records_in, records_out, cell_bits: int, item_bits: int, stream=None) -> None:
    """sort_accesses without any device allocation: scratch comes from the
    library's fixed device array (at most 2^18 records).  For callers that may
    not allocate device memory; concurrent calls on the GPU share that array
    and must be serialised by the caller."""
    n = records_in.shape[0]
    if records_out.shape != records_in.shape:
        raise ValueError("records_out must have the shape of records_in")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    rc = load().rc_sort_accesses_noalloc(ctypes.c_void_p(records_in.data_ptr()),
                                         ctypes.c_void_p(records_out.data_ptr()), n, cell_bits, item_bits,
                                         ctypes.c_void_p(int(stream) if stream else 0))
    if rc:
        raise RaceCheckError(rc, load().rc_strerror(rc).decode())


def autotune_config(cache_path=None) -> None:
    """Autotuner cache file (None: default location, "": keep decisions in memory only)."""
    load().rc_autotune_config(None if cache_path is None else cache_path.encode())


def autotune_reset() -> None:
    load().rc_autotune_reset()


def autotune_lookup(kind: int, a: int, b: int) -> int:
    """The autotuner's decision for a size class (kind 0 single, 1 batch:
    strategy 1 sort / 2 shadow; kind 2 batch block shape in threads per CTA;
    kind 3 batch log capacity in permille of the static bound; 0 undecided)."""
    return int(load().rc_autotune_lookup(kind, a, b))


def prove(bc: Bytecode, groups: int, group_size: int, globals_) -> dict:
    """Two-work-item NoRace pre-filter for this launch shape (host only):
    race_free / in_bounds are proofs when True and say nothing when False."""
    inp, keep = _marshal(globals_, None, False)
    res = _ProveResult()
    rc = load().rc_prove(bc.handle, groups, group_size, ctypes.byref(inp), ctypes.byref(res))
    del keep
    if rc:
        _raise(rc)
    return dict(race_free=bool(res.race_free), in_bounds=bool(res.in_bounds),
                first=(res.first_pc_a, res.first_pc_b) if not res.race_free else None,
                n_pairs=res.n_pairs, n_unresolved=res.n_unresolved)


def prove_private(bc: Bytecode, groups: int, group_size: int, globals_) -> np.ndarray:
    """Per bytecode instruction: 1 where the pre-filter proves the load or
    store private for this launch shape (its cells carry no race or benign
    record in its interval: no other work-item touches a private store's
    cells, none writes a private load's cells, and no other work-item reads
    a private load's cell that a different one writes), else 0 (host only)."""
    inp, keep = _marshal(globals_, None, False)
    n_insn = bc.info()["n_insn"]
    flags = np.zeros(max(n_insn, 1), np.uint8)
    n = ctypes.c_uint32()
    rc = load().rc_prove_private(bc.handle, groups, group_size, ctypes.byref(inp),
                                 flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n_insn, ctypes.byref(n))
    del keep
    if rc:
        _raise(rc)
    return flags[:n_insn]


def access_sites(bc: Bytecode) -> np.ndarray:
    """The kernel's shared-access instructions in bytecode (= text) order:
    uint32 [n, 3] rows (pc, is_store, memory object) (host only)."""
    lib = load()
    n = ctypes.c_uint32()
    rc = lib.rc_access_sites(bc.handle, None, None, None, 0, ctypes.byref(n))
    if rc:
        _raise(rc)
    pc = np.zeros(max(n.value, 1), np.uint32)
    st = np.zeros(max(n.value, 1), np.uint8)
    mem = np.zeros(max(n.value, 1), np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib.rc_access_sites(bc.handle, pc.ctypes.data_as(u32p), st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                             mem.ctypes.data_as(u32p), n.value, ctypes.byref(n))
    if rc:
        _raise(rc)
    k = n.value
    return np.stack([pc[:k], st[:k].astype(np.uint32), mem[:k]], axis=1)


def translate(bc: Bytecode, fn_name: str = "rc_jit_run") -> str:
    """The kernel as C++ source text: one function that runs one work-item
    to its next barrier, exit or end (host only)."""
    lib = load()
    n = ctypes.c_size_t()
    rc = lib.rc_translate(bc.handle, fn_name.encode(), None, 0, ctypes.byref(n))
    if rc:
        _raise(rc)
    buf = ctypes.create_string_buffer(n.value + 1)
    rc = lib.rc_translate(bc.handle, fn_name.encode(), buf, n.value + 1, ctypes.byref(n))
    if rc:
        _raise(rc)
    return buf.value.decode()


def explore(bc: Bytecode, groups: int, group_size: int, globals_, max_states: int = 0,
            max_intervals: int = 64) -> list:
    """Every schedule of each interval of a small instance (<= 16 work-items),
    from the checker's state at the interval's start: per interval
    n_end_states (distinct shared memories at its closing barrier), deviated
    (some read depends on the schedule), complete, n_states."""
    inp, keep = _marshal(globals_, None, False)
    out = (_ExploreInterval * max(max_intervals, 1))()
    n = ctypes.c_uint32()
    rc = load().rc_explore(bc.handle, groups, group_size, ctypes.byref(inp), max_states, out, max_intervals,
                           ctypes.byref(n))
    del keep
    if rc:
        _raise(rc)
    return [dict(interval=o.interval, n_end_states=o.n_end_states, deviated=bool(o.deviated),
                 complete=bool(o.complete), n_states=int(o.n_states)) for o in out[:n.value]]


def explore_pairs(bc: Bytecode, groups: int, group_size: int, globals_, max_states: int = 0,
                  max_intervals: int = 64, detail: bool = False) -> list:
    """The interleaving product of every pair of work-items i < j (the others
    do not run), per interval from the checker's state at its start: n_pairs,
    n_racy (pairs reaching >= 2 shared memories), n_deviated, first racy pair,
    complete, n_states; with detail, per pair (end memories, deviated)."""
    inp, keep = _marshal(globals_, None, False)
    out = (_PairInterval * max(max_intervals, 1))()
    n = ctypes.c_uint32()
    N = groups * group_size
    P = N * (N - 1) // 2
    det = np.zeros(max(max_intervals * P, 1), dtype=np.uint32) if detail else None
    rc = load().rc_explore_pairs(bc.handle, groups, group_size, ctypes.byref(inp), max_states, out, max_intervals,
                                 ctypes.byref(n),
                                 det.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if detail else None)
    del keep
    if rc:
        _raise(rc)
    res = []
    for k, o in enumerate(out[:n.value]):
        d = dict(interval=o.interval, n_pairs=o.n_pairs, n_racy=o.n_racy, n_deviated=o.n_deviated,
                 first=(o.first_i, o.first_j) if o.n_racy else None, complete=bool(o.complete),
                 n_states=int(o.n_states))
        if detail:
            d["pairs"] = [(int(x & 0x7FFFFFFF), bool(x >> 31)) for x in det[k * P:(k + 1) * P]]
        res.append(d)
    return res


# ---------------------------------------------------------------- learned proposal


def _items_arrays(items, want_final=False):
    n = len(items)
    hs = (ctypes.c_void_p * max(n, 1))(*[it[0].handle.value for it in items])
    gs = (ctypes.c_uint32 * max(n, 1))(*[it[1] for it in items])
    ss = (ctypes.c_uint32 * max(n, 1))(*[it[2] for it in items])
    inputs = (_Input * max(n, 1))()
    keep = []
    for i, it in enumerate(items):
        inp, k = _marshal(it[3], None, want_final)
        inputs[i] = inp
        keep.append(k)
    return hs, gs, ss, inputs, keep


def features(items, n_threads: int = 0) -> np.ndarray:
    """Feature vectors [n, 128] of candidate instances items = [(bytecode,
    groups, group_size, host globals)]."""
    n = len(items)
    out = np.zeros((max(n, 1), N_FEATURES), dtype=np.float32)
    hs, gs, ss, inputs, keep = _items_arrays(items)
    rc = load().rc_features_batch(hs, gs, ss, inputs, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                  n_threads)
    del keep
    if rc:
        _raise(rc)
    return out[:n]


def search(items, scores=None, max_checks: int = 0) -> dict:
    """Check candidates in descending score order (or as given when scores is
    None) until one is racy; returns first (index or -1), checks, seconds and
    the racy candidate's report."""
    n = len(items)
    hs, gs, ss, inputs, keep = _items_arrays(items)
    sc = None
    if scores is not None:
        sc = np.ascontiguousarray(np.asarray(scores, dtype=np.float32))
        if sc.shape != (n,):
            raise ValueError("one score per candidate")
    res = _SearchResult()
    found = ctypes.POINTER(_Report)()
    rc = load().rc_search(hs, gs, ss, inputs, n,
                          sc.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if sc is not None else None,
                          max_checks, ctypes.byref(res), ctypes.byref(found))
    del keep
    if rc:
        _raise(rc)
    return dict(first=int(res.first), checks=int(res.checks), seconds=float(res.seconds),
                report=_report(found) if found else None)


def search_ranked(items, model=None, overlap: bool = False, max_checks: int = 0) -> dict:
    """Ranked search in one native call (rc_search_ranked): features on the
    library's host threads, scores from `model` (an MLP) or, with None, the
    rule ranking, then exact checks in score order; with overlap the GPU
    checks candidates in index order until the ranking exists.  Returns
    first, checks, checks_unranked, seconds (whole call), features_seconds,
    scoring_seconds, check_seconds and the racy candidate's report."""
    n = len(items)
    hs, gs, ss, inputs, keep = _items_arrays(items)
    res = _RankedResult()
    found = ctypes.POINTER(_Report)()
    rc = load().rc_search_ranked(model._h if model is not None else None, hs, gs, ss, inputs, n, max_checks,
                                 RC_RANK_OVERLAP if overlap else 0, ctypes.byref(res), ctypes.byref(found))
    del keep
    if rc:
        _raise(rc)
    out = {k: getattr(res, k) for k, _ in _RankedResult._fields_}
    out = {k: (int(v) if isinstance(v, int) else float(v)) for k, v in out.items()}
    out["report"] = _report(found) if found else None
    return out


class MLP:
    """Ranking network (128 -> 256 -> 256 -> 256 -> 1) on the GPU.  Inputs
    are CUDA float32 tensors: features [n, 128], labels [n]."""

    def __init__(self, seed: int = 0, capacity: int = 65536):
        self._h = ctypes.c_void_p()
        rc = load().rc_mlp_create(seed, capacity, ctypes.byref(self._h))
        if rc:
            _raise(rc)
        self.capacity = capacity

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rc_mlp_free(self._h)
            self._h = None

    @staticmethod
    def _dev(t, cols=None):
        if not (_is_torch_cuda(t) and str(t.dtype) == "torch.float32" and t.is_contiguous()):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
            raise ValueError(f"expected shape [n, {cols}]")
        return ctypes.c_void_p(t.data_ptr())

    @staticmethod
    def _stream():
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def set_backend(self, backend: int) -> None:
        """Every product on tcgen05 with TMEM accumulators -- forward layers in
        one launch (1, the default) or one per layer (2) -- or on mma.sync (0)."""
        rc = load().rc_mlp_set_backend(self._h, backend)
        if rc:
            _raise(rc)

    def backend_error(self) -> int:
        """Nonzero if a tcgen05 launch gave up waiting for its MMAs."""
        v = ctypes.c_uint32()
        rc = load().rc_mlp_backend_error(self._h, ctypes.byref(v))
        if rc:
            _raise(rc)
        return int(v.value)

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        rc = load().rc_mlp_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc:
            _raise(rc)
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if p.shape != (MLP_PARAMS,):
            raise ValueError("parameter vector of the wrong size")
        rc = load().rc_mlp_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc:
            _raise(rc)

    def forward(self, x):
        import torch
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        rc = load().rc_mlp_forward(self._h, self._dev(x, N_FEATURES), x.shape[0], ctypes.c_void_p(out.data_ptr()),
                                   self._stream())
        if rc:
            _raise(rc)
        return out

    def grad(self, x, y):
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        rc = load().rc_mlp_grad(self._h, self._dev(x, N_FEATURES), self._dev(y), x.shape[0],
                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss), self._stream())
        if rc:
            _raise(rc)
        return g, float(loss.value)

    def train(self, x, y, epochs: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0) -> np.ndarray:
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        rc = load().rc_mlp_train(self._h, self._dev(x, N_FEATURES), self._dev(y), x.shape[0], epochs, batch, lr,
                                 seed, losses.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self._stream())
        if rc:
            _raise(rc)
        return losses[:epochs]
