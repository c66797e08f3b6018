"""Thin ctypes binding of libsuffstats (include/stats.h), same names as the C ABI.

Argument marshalling only: every step of the pass runs in the library's CUDA
kernels.  PyTorch is used for device memory and streams (plumbing).  If the
compiled library is missing the import of this module fails loudly; there is
no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import itertools
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

# ----------------------------------------------------------------------------- constants (stats.h)
(STATS_OK, STATS_EINVAL, STATS_ENOMEM, STATS_ECUDA, STATS_EOVERFLOW, STATS_ETIMEOUT, STATS_ESTATE, STATS_ERANGE,
 STATS_EIO, STATS_EFORMAT, STATS_EMISMATCH) = range(11)
STATS_I16, STATS_I32, STATS_I64, STATS_F32, STATS_F64 = range(5)
STATS_EXACT, STATS_FP64, STATS_FP64_SHIFTED, STATS_BF16X3, STATS_BF16X4, STATS_FP32 = range(6)
STATS_T1_L32, STATS_T1_L16 = 0, 1
STATS_T1_P = 12
STATS_MAX_P = 256

_NAMES = {STATS_OK: "STATS_OK", STATS_EINVAL: "STATS_EINVAL", STATS_ENOMEM: "STATS_ENOMEM",
          STATS_ECUDA: "STATS_ECUDA", STATS_EOVERFLOW: "STATS_EOVERFLOW", STATS_ETIMEOUT: "STATS_ETIMEOUT",
          STATS_ESTATE: "STATS_ESTATE", STATS_ERANGE: "STATS_ERANGE", STATS_EIO: "STATS_EIO",
          STATS_EFORMAT: "STATS_EFORMAT", STATS_EMISMATCH: "STATS_EMISMATCH"}
# stats_file.h
STATS_FILE_HEADER_BYTES = 4096
STATS_FILE_ALIGN = 4096
STATS_FILE_MAX_P = 256

DTYPE_BYTES = {STATS_I16: 2, STATS_I32: 4, STATS_I64: 8, STATS_F32: 4, STATS_F64: 8}
T1_NAMES = ("A", "B", "C", "D", "E", "F", "G", "H", "cotC", "I", "J", "K")


class StatsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_NAMES.get(code, code)} ({stats_strerror(code)})")


class _Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("dtypes", ctypes.POINTER(ctypes.c_int32)),
                ("is_identifier", ctypes.POINTER(ctypes.c_uint8)), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double)), ("mode", ctypes.c_int32)]


class _I128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_int64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libsuffstats.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libsuffstats.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.stats_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Config)]
    L.stats_accumulate.argtypes = [vp, ctypes.POINTER(vp), i64, vp]
    L.stats_accumulate_host.argtypes = [vp, ctypes.POINTER(vp), i64, i64, vp]
    L.stats_merge.argtypes = [vp, vp]
    L.stats_sync.argtypes = [vp]
    L.stats_reset.argtypes = [vp]
    L.stats_raw.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I128), ctypes.POINTER(_I128)]
    L.stats_finalize.argtypes = [vp] + [ctypes.POINTER(ctypes.c_double)] * 5 + [i32]
    L.stats_finalize_warm.argtypes = [vp] + [ctypes.POINTER(ctypes.c_double)] * 5 + [i32, vp, ctypes.POINTER(i32)]
    L.stats_export.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.stats_import.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_size_t]
    L.stats_destroy.argtypes = [vp]
    L.stats_destroy.restype = None
    L.stats_strerror.argtypes = [ctypes.c_int]
    L.stats_strerror.restype = ctypes.c_char_p
    L.stats_num_analysis_columns.argtypes = [vp]
    L.stats_num_analysis_columns.restype = i32
    L.stats_set_grid.argtypes = [vp, i32]
    L.stats_table1_config.argtypes = [i32, i64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.stats_gen_table1.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i64, i32, ctypes.POINTER(vp), vp]
    L.stats_table1_row_bytes.argtypes = [i32]
    L.stats_table1_row_bytes.restype = i32
    cp = ctypes.c_char_p
    L.stats_file_write.argtypes = [cp, i32, ctypes.POINTER(i32), i64, ctypes.POINTER(vp)]
    L.stats_file_write_table1.argtypes = [cp, ctypes.c_uint64, ctypes.c_uint64, i64, i32, i64]
    L.stats_file_info.argtypes = [cp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.stats_file_read_rows.argtypes = [cp, i64, i64, ctypes.POINTER(vp)]
    L.stats_file_check_table1.argtypes = [cp, ctypes.c_uint64, ctypes.c_uint64, i32, i64, ctypes.POINTER(i64)]
    L.stats_accumulate_file.argtypes = [vp, cp, i64, i64, i64, vp]
    L.stats_csv_write.argtypes = [cp, i32, ctypes.POINTER(i32), i64, ctypes.POINTER(vp), cp]
    L.stats_csv_write_table1.argtypes = [cp, ctypes.c_uint64, ctypes.c_uint64, i64, i32, i64]
    L.stats_csv_parse.argtypes = [vp, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(vp), i64,
                                  ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    L.stats_accumulate_csv.argtypes = [vp, cp, i64, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    for name in ("stats_init", "stats_accumulate", "stats_accumulate_host", "stats_merge", "stats_sync",
                 "stats_reset", "stats_raw", "stats_finalize", "stats_finalize_warm", "stats_export", "stats_import", "stats_set_grid",
                 "stats_table1_config", "stats_gen_table1", "stats_file_write", "stats_file_write_table1",
                 "stats_file_info", "stats_file_read_rows", "stats_file_check_table1", "stats_accumulate_file",
                 "stats_csv_write", "stats_csv_write_table1", "stats_csv_parse", "stats_accumulate_csv"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code: int, where: str):
    if code != STATS_OK:
        raise StatsError(code, where)


def stats_strerror(code: int) -> str:
    return load().stats_strerror(code).decode()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> int:
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _ptr_array(cols: Sequence) -> ctypes.Array:
    return (ctypes.c_void_p * len(cols))(*[_ptr(c) for c in cols])


# ----------------------------------------------------------------------------- configuration
@dataclass
class Config:
    """Mirror of stats_config."""
    dtypes: Sequence[int]
    mode: int = STATS_EXACT
    is_identifier: Optional[Sequence[int]] = None
    lo: Optional[Sequence[float]] = None
    hi: Optional[Sequence[float]] = None
    _keep: list = field(default_factory=list, repr=False)

    @property
    def p(self) -> int:
        return len(self.dtypes)

    def c_struct(self) -> _Config:
        p = self.p
        dt = (ctypes.c_int32 * p)(*self.dtypes)
        ident = (ctypes.c_uint8 * p)(*self.is_identifier) if self.is_identifier is not None else None
        lo = (ctypes.c_double * p)(*self.lo) if self.lo is not None else None
        hi = (ctypes.c_double * p)(*self.hi) if self.hi is not None else None
        self._keep = [dt, ident, lo, hi]
        return _Config(p, dt, ident, lo, hi, self.mode)


def stats_table1_config(layout: int = STATS_T1_L32, max_rows: int = 10**10, mode: int = STATS_EXACT) -> Config:
    """The Table 1 configuration (12 columns, identifier A) of a layout."""
    dt = (ctypes.c_int32 * 12)()
    ident = (ctypes.c_uint8 * 12)()
    lo = (ctypes.c_double * 12)()
    hi = (ctypes.c_double * 12)()
    _check(load().stats_table1_config(layout, max_rows, dt, ident, lo, hi), "stats_table1_config")
    return Config(list(dt), mode, list(ident), list(lo), list(hi))


def stats_table1_row_bytes(layout: int) -> int:
    return load().stats_table1_row_bytes(layout)


# ----------------------------------------------------------------------------- context
class Ctx:
    """Owning handle of a stats_ctx (destroyed on close / garbage collection)."""

    def __init__(self, handle: int, p: int, mode: int):
        self.handle = ctypes.c_void_p(handle)
        self.p = p
        self.mode = mode

    def close(self):
        if self.handle:
            load().stats_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stats_init(cfg: Config) -> Ctx:
    h = ctypes.c_void_p()
    s = cfg.c_struct()
    _check(load().stats_init(ctypes.byref(h), ctypes.byref(s)), "stats_init")
    return Ctx(h.value, cfg.p, cfg.mode)


def stats_accumulate(ctx: Ctx, dcols: Sequence, nrows: int, stream=None):
    """Add nrows device-resident rows (dcols: tensors or device addresses)."""
    arr = _ptr_array(dcols)
    _check(load().stats_accumulate(ctx.handle, arr, nrows, _stream_handle(stream)), "stats_accumulate")


def stats_accumulate_host(ctx: Ctx, hcols: Sequence, nrows: int, chunk_rows: int = 0, stream=None):
    """Add nrows host-resident rows (hcols: pinned tensors / numpy arrays / host addresses)."""
    arr = _ptr_array(hcols)
    _check(load().stats_accumulate_host(ctx.handle, arr, nrows, chunk_rows, _stream_handle(stream)),
           "stats_accumulate_host")


class BatchArgs:
    """The argument arrays of one stats_accumulate_batched call, built once (the marshalling of
    thousands of column pointers costs milliseconds in Python) and reusable for later calls on
    the same contexts and column addresses."""

    def __init__(self, ctxs: Sequence[Ctx], dcols: Sequence[Sequence], nrows: Sequence[int]):
        n = len(ctxs)
        self.ctxs = list(ctxs)
        self.handles = np.fromiter((c.handle.value for c in ctxs), dtype=np.uint64, count=n)
        if n and dcols[0] and isinstance(dcols[0][0], int):
            self.flat = np.fromiter(itertools.chain.from_iterable(dcols), dtype=np.uint64)
        else:
            self.flat = np.fromiter((_ptr(x) for cols in dcols for x in cols), dtype=np.uint64)
        counts = np.fromiter((len(cols) for cols in dcols), dtype=np.int64, count=n)
        starts = np.concatenate(([0], np.cumsum(counts)[:-1])) if n else np.zeros(0, np.int64)
        # one flat array of column pointers and, per table, the address of its first entry
        self.outer = (self.flat.ctypes.data + 8 * starts).astype(np.uint64)
        self.rows = np.asarray(nrows, dtype=np.int64)
        self.n = n


def stats_accumulate_batched(ctxs, dcols: Sequence[Sequence] = None, nrows: Sequence[int] = None, stream=None):
    """Add table t (dcols[t]: its device columns, nrows[t] rows) to ctxs[t], all in one pass;
    ctxs may instead be a prepared BatchArgs."""
    L = load()
    L.stats_accumulate_batched.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
    L.stats_accumulate_batched.restype = ctypes.c_int
    b = ctxs if isinstance(ctxs, BatchArgs) else BatchArgs(ctxs, dcols, nrows)
    _check(L.stats_accumulate_batched(b.handles.ctypes.data, b.n, b.outer.ctypes.data, b.rows.ctypes.data,
                                      _stream_handle(stream)), "stats_accumulate_batched")


def stats_merge(dst: Ctx, src: Ctx):
    _check(load().stats_merge(dst.handle, src.handle), "stats_merge")


def stats_sync(ctx: Ctx):
    _check(load().stats_sync(ctx.handle), "stats_sync")


def stats_reset(ctx: Ctx):
    _check(load().stats_reset(ctx.handle), "stats_reset")


def stats_set_grid(ctx: Ctx, blocks: int):
    _check(load().stats_set_grid(ctx.handle, blocks), "stats_set_grid")


def stats_set_flush_rows(ctx: Ctx, rows: int):
    L = load()
    L.stats_set_flush_rows.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.stats_set_flush_rows.restype = ctypes.c_int
    _check(L.stats_set_flush_rows(ctx.handle, rows), "stats_set_flush_rows")


class _BatchTuning(ctypes.Structure):
    _fields_ = [("narrow_units_per_cta", ctypes.c_int32), ("gram32_chunks_per_cta", ctypes.c_int32),
                ("gram32_min_chunk", ctypes.c_int32)]


def stats_set_batch_tuning(width: int, mode: int, t: dict):
    """How batched launches of a width class (1-8, 9-16, 17-32, 33-64 columns) and split mode
    deal their stages to CTAs (stats.h); t has the three stats_batch_tuning fields."""
    L = load()
    L.stats_set_batch_tuning.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_BatchTuning)]
    L.stats_set_batch_tuning.restype = ctypes.c_int
    v = _BatchTuning(int(t["narrow_units_per_cta"]), int(t["gram32_chunks_per_cta"]), int(t["gram32_min_chunk"]))
    _check(L.stats_set_batch_tuning(width, mode, ctypes.byref(v)), "stats_set_batch_tuning")


def stats_get_batch_tuning(width: int, mode: int) -> dict:
    L = load()
    L.stats_get_batch_tuning.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_BatchTuning)]
    L.stats_get_batch_tuning.restype = ctypes.c_int
    v = _BatchTuning()
    _check(L.stats_get_batch_tuning(width, mode, ctypes.byref(v)), "stats_get_batch_tuning")
    return {f: getattr(v, f) for f, _ in _BatchTuning._fields_}


def stats_set_wide_pairs(ctx: Ctx, pairs: int):
    """129..256 FP32 columns in a [p, ld] block: 1 = the paired-CTA pass, 0 = one CTA per output block."""
    L = load()
    L.stats_set_wide_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.stats_set_wide_pairs.restype = ctypes.c_int
    _check(L.stats_set_wide_pairs(ctx.handle, pairs), "stats_set_wide_pairs")


def stats_set_exact_shape(ctx: Ctx, shape: int):
    """Launch shape of the STATS_EXACT pass (-1: default; 0, 1, 2: see stats.h)."""
    L = load()
    L.stats_set_exact_shape.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.stats_set_exact_shape.restype = ctypes.c_int
    _check(L.stats_set_exact_shape(ctx.handle, shape), "stats_set_exact_shape")


def stats_set_grid_wait(ctx: Ctx, wait_ns: int = 0, absent_block: int = -1):
    """Limit of the eigen-solver's bounded grid-wide waits (0: 2 s), and optionally a block that
    leaves before arriving, so that the other blocks' waits run out (stats.h)."""
    L = load()
    L.stats_set_grid_wait.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]
    L.stats_set_grid_wait.restype = ctypes.c_int
    _check(L.stats_set_grid_wait(ctx.handle, wait_ns, absent_block), "stats_set_grid_wait")


def stats_num_analysis_columns(ctx: Ctx) -> int:
    return load().stats_num_analysis_columns(ctx.handle)


def _i128(v: _I128) -> int:
    return (int(v.hi) << 64) + int(v.lo)


@dataclass
class Raw:
    n: int
    s: np.ndarray           # p, rounded once to double
    S: np.ndarray           # p x p symmetric, rounded once to double
    s_exact: list           # p Python ints (exact for integer-valued columns in STATS_EXACT)
    S_exact: list           # p x p Python ints (exact where both columns are integer-valued)
    status: int


def stats_raw(ctx: Ctx, allow_overflow: bool = False) -> Raw:
    p = ctx.p
    T = p * (p + 1) // 2
    n = ctypes.c_int64()
    s = np.zeros(p)
    Su = np.zeros(T)
    se = (_I128 * p)()
    Se = (_I128 * T)()
    rc = load().stats_raw(ctx.handle, ctypes.byref(n), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          Su.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), se, Se)
    if rc != STATS_OK and not (allow_overflow and rc == STATS_EOVERFLOW):
        raise StatsError(rc, "stats_raw")
    S = np.zeros((p, p))
    SE = [[0] * p for _ in range(p)]
    t = 0
    for j in range(p):
        for k in range(j, p):
            S[j, k] = S[k, j] = Su[t]
            SE[j][k] = SE[k][j] = _i128(Se[t])
            t += 1
    return Raw(int(n.value), s, S, [_i128(v) for v in se], SE, rc)


@dataclass
class Analysis:
    mean: np.ndarray
    cov: np.ndarray
    corr: np.ndarray
    evals: np.ndarray
    evecs: np.ndarray   # row k = eigenvector k
    sweeps: int = -1    # Jacobi sweeps taken (stats_finalize_warm only; -1: not reported)


def stats_finalize(ctx: Ctx, pca_on: int = 0) -> Analysis:
    pa = stats_num_analysis_columns(ctx)
    mean = np.zeros(pa)
    cov = np.zeros((pa, pa))
    corr = np.zeros((pa, pa))
    ev = np.zeros(pa)
    V = np.zeros((pa, pa))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    _check(load().stats_finalize(ctx.handle, dp(mean), dp(cov), dp(corr), dp(ev), dp(V), pca_on), "stats_finalize")
    return Analysis(mean, cov, corr, ev, V)


def stats_finalize_warm(ctx: Ctx, pca_on: int = 0, evecs_prev=None) -> Analysis:
    """stats_finalize with the eigen-solver seeded by evecs_prev (rows = eigenvectors, e.g. the
    evecs of an earlier snapshot), or cold when None; the result carries the sweep count."""
    pa = stats_num_analysis_columns(ctx)
    mean = np.zeros(pa)
    cov = np.zeros((pa, pa))
    corr = np.zeros((pa, pa))
    ev = np.zeros(pa)
    V = np.zeros((pa, pa))
    sw = ctypes.c_int32(-1)
    seed = None
    if evecs_prev is not None:
        seed = np.ascontiguousarray(evecs_prev, dtype=np.float64)
        if seed.shape != (pa, pa):
            raise ValueError(f"evecs_prev must be {pa} x {pa}")
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    _check(load().stats_finalize_warm(ctx.handle, dp(mean), dp(cov), dp(corr), dp(ev), dp(V), pca_on,
                                      None if seed is None else seed.ctypes.data, ctypes.byref(sw)),
           "stats_finalize_warm")
    return Analysis(mean, cov, corr, ev, V, int(sw.value))


class StreamingAnalysis:
    """Snapshots of a growing table: accumulate chunks with update(), and after any of them
    take snapshot(), whose eigen-solve is seeded by the previous snapshot's eigenvectors."""

    def __init__(self, cfg: "Config", pca_on: int = 0):
        self.ctx = stats_init(cfg)
        self.pca_on = pca_on
        self.prev = None

    def update(self, dcols: Sequence, nrows: int, stream=None):
        stats_accumulate(self.ctx, dcols, nrows, stream)

    def snapshot(self) -> Analysis:
        an = stats_finalize_warm(self.ctx, self.pca_on, self.prev)
        if np.all(np.isfinite(an.evecs)):
            self.prev = an.evecs
        return an

    def close(self):
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stats_finalize_batched(ctxs: Sequence[Ctx], pca_on: int = 0) -> list:
    """stats_finalize for every context in one launch; returns one Analysis per context."""
    L = load()
    L.stats_finalize_batched.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 5
    L.stats_finalize_batched.restype = ctypes.c_int
    n = len(ctxs)
    outs = []
    for c in ctxs:
        pa = stats_num_analysis_columns(c)
        outs.append(Analysis(np.zeros(pa), np.zeros((pa, pa)), np.zeros((pa, pa)), np.zeros(pa), np.zeros((pa, pa))))
    handles = np.fromiter((c.handle.value for c in ctxs), dtype=np.uint64, count=n)
    ptrs = [np.fromiter((getattr(a, f).ctypes.data for a in outs), dtype=np.uint64, count=n)
            for f in ("mean", "cov", "corr", "evals", "evecs")]
    _check(L.stats_finalize_batched(handles.ctypes.data, n, pca_on, *[x.ctypes.data for x in ptrs]),
           "stats_finalize_batched")
    return outs


def stats_export(ctx: Ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(load().stats_export(ctx.handle, None, ctypes.byref(n)), "stats_export(size)")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().stats_export(ctx.handle, buf, ctypes.byref(n)), "stats_export")
    return buf.raw[: n.value]


def stats_import(blob: bytes, p: int, mode: int) -> Ctx:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().stats_import(ctypes.byref(h), buf, len(blob)), "stats_import")
    return Ctx(h.value, p, mode)


def stats_destroy(ctx: Ctx):
    ctx.close()


def stats_gen_table1(seed: int, row0: int, nrows: int, layout: int, dcols: Sequence, stream=None):
    arr = _ptr_array(dcols)
    _check(load().stats_gen_table1(seed, row0, nrows, layout, arr, _stream_handle(stream)), "stats_gen_table1")


# ----------------------------------------------------------------------------- Table 1 buffers
def table1_torch_dtypes(layout: int):
    import torch
    m = {STATS_I16: torch.int16, STATS_I32: torch.int32, STATS_I64: torch.int64, STATS_F32: torch.float32,
         STATS_F64: torch.float64}
    cfg = stats_table1_config(layout, 1)
    return [m[d] for d in cfg.dtypes]


def alloc_table1(nrows: int, layout: int = STATS_T1_L32, device="cuda", pin_memory: bool = False):
    """Twelve column tensors of a Table 1 layout (torch provides the memory)."""
    import torch
    return [torch.empty(max(nrows, 1), dtype=dt, device=device, pin_memory=pin_memory and device == "cpu")
            for dt in table1_torch_dtypes(layout)]


def gen_table1(seed: int, nrows: int, layout: int = STATS_T1_L32, row0: int = 0, cols=None, stream=None):
    """Generate Table 1 rows on the current device; returns the column tensors."""
    if cols is None:
        cols = alloc_table1(nrows, layout)
    stats_gen_table1(seed, row0, nrows, layout, cols, stream)
    return cols


# ----------------------------------------------------------------------------- record checks
def identifier_checks(raw: Raw, first: int, count: int, col: int = 0) -> dict:
    """Closed-form checks that every record of a row range was processed exactly once.

    The paper validates its pipeline by the identifier column's sum ("Validation and
    Infrastructure Testing"): a column holding first, first + 1, ..., first + count - 1
    (Table 1's A is the 1-based row index) must give n = count, its sum
    count (first + last) / 2 and its sum of squares sum_{v <= last} v^2 - sum_{v < first} v^2,
    with v^2 sums k (k + 1) (2k + 1) / 6.  A dropped, repeated or displaced chunk changes at
    least one of them.  raw must hold exact sums (STATS_EXACT, integer identifier column)."""
    last = first + count - 1
    sq = lambda k: k * (k + 1) * (2 * k + 1) // 6  # noqa: E731
    return {"n": raw.n == count,
            "sum": raw.s_exact[col] == count * (first + last) // 2,
            "sum_sq": raw.S_exact[col][col] == sq(last) - sq(first - 1)}


# ----------------------------------------------------------------------------- no-allocation variant
def noalloc_result_bytes(p: int) -> int:
    """STATS_NOALLOC_RESULT_BYTES(p) of stats.h."""
    return 8 * (9 + 3 * p + 3 * (p * (p + 1) // 2))


def stats_pass_noalloc(cfg: Config, dcols: Sequence, nrows: int, d_result, stream=None):
    """The exact pass without a context or any device allocation; writes (n, s, S)
    into the caller's device buffer d_result (noalloc_result_bytes(p) bytes)."""
    L = load()
    if not hasattr(L, "_noalloc_ready"):
        L.stats_pass_noalloc.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.stats_pass_noalloc.restype = ctypes.c_int
        L._noalloc_ready = True
    s = cfg.c_struct()
    arr = _ptr_array(dcols) if nrows > 0 else None
    _check(L.stats_pass_noalloc(ctypes.byref(s), arr, nrows, _ptr(d_result), _stream_handle(stream)),
           "stats_pass_noalloc")


def parse_noalloc_result(buf: bytes, p: int) -> Raw:
    """Decode a host copy of the stats_pass_noalloc result buffer."""
    T = p * (p + 1) // 2
    w = np.frombuffer(buf, dtype=np.int64)
    d = np.frombuffer(buf, dtype=np.float64)
    n = int(w[0])
    s = d[1:1 + p].copy()
    Su = d[1 + p:1 + p + T]
    off = 1 + p + T
    s_ex = [(int(w[off + 2 * j + 1]) << 64) + (int(w[off + 2 * j]) & 0xFFFFFFFFFFFFFFFF) for j in range(p)]
    off += 2 * p
    S_ex_u = [(int(w[off + 2 * t + 1]) << 64) + (int(w[off + 2 * t]) & 0xFFFFFFFFFFFFFFFF) for t in range(T)]
    off += 2 * T
    flags = off
    status = int(np.frombuffer(buf[8 * (flags + 4):8 * (flags + 4) + 4], dtype=np.uint32)[0])
    S = np.zeros((p, p))
    SE = [[0] * p for _ in range(p)]
    t = 0
    for j in range(p):
        for k in range(j, p):
            S[j, k] = S[k, j] = Su[t]
            SE[j][k] = SE[k][j] = S_ex_u[t]
            t += 1
    # the order of the regular entry points: an expired wait first, then a range error
    code = STATS_ETIMEOUT if status & 2 else STATS_ERANGE if status & 1 else \
        STATS_EOVERFLOW if d[flags] != 0.0 else STATS_OK
    return Raw(n, s, S, s_ex, SE, code)


# ----------------------------------------------------------------------------- table files (stats_file.h)
def _path(path) -> bytes:
    return os.fsencode(path)


def stats_file_write(path, dtypes: Sequence[int], nrows: int, hcols: Sequence):
    """Write an n x p table from host columns (numpy arrays / pinned tensors / addresses)."""
    p = len(dtypes)
    dt = (ctypes.c_int32 * p)(*dtypes)
    _check(load().stats_file_write(_path(path), p, dt, nrows, _ptr_array(hcols)), "stats_file_write")


def stats_file_write_table1(path, seed: int, nrows: int, layout: int = STATS_T1_L32, row0: int = 0,
                            chunk_rows: int = 0):
    """Write Table 1 rows [row0, row0 + nrows), generated on the current device, to a table file."""
    _check(load().stats_file_write_table1(_path(path), seed, row0, nrows, layout, chunk_rows),
           "stats_file_write_table1")


def stats_file_info(path):
    """(p, nrows, dtypes) of a validated table file."""
    p = ctypes.c_int32(0)
    n = ctypes.c_int64(0)
    dt = (ctypes.c_int32 * STATS_FILE_MAX_P)()
    _check(load().stats_file_info(_path(path), ctypes.byref(p), ctypes.byref(n), dt), "stats_file_info")
    return p.value, n.value, [dt[j] for j in range(p.value)]


_NP_DTYPES = {STATS_I16: np.int16, STATS_I32: np.int32, STATS_I64: np.int64, STATS_F32: np.float32,
              STATS_F64: np.float64}


def stats_file_read_rows(path, row0: int, nrows: int):
    """Rows [row0, row0 + nrows) of every column, as numpy arrays."""
    _, _, dts = stats_file_info(path)
    cols = [np.empty(nrows, dtype=_NP_DTYPES[d]) for d in dts]
    _check(load().stats_file_read_rows(_path(path), row0, nrows, _ptr_array(cols)), "stats_file_read_rows")
    return cols


def stats_file_check_table1(path, seed: int, layout: int = STATS_T1_L32, rows_per_region: int = 4096,
                            row0: int = 0) -> int:
    """The conversion check of a Table 1 file; returns -1, raises StatsError(STATS_EMISMATCH) with
    .bad_row set to the first differing file row."""
    bad = ctypes.c_int64(-1)
    code = load().stats_file_check_table1(_path(path), seed, row0, layout, rows_per_region, ctypes.byref(bad))
    if code != STATS_OK:
        err = StatsError(code, "stats_file_check_table1")
        err.bad_row = bad.value
        raise err
    return bad.value


def stats_accumulate_file(ctx: Ctx, path, row0: int = 0, nrows: int = -1, chunk_rows: int = 0, stream=None):
    """Add file rows [row0, row0 + nrows) (nrows < 0: to the end) to ctx through pinned chunks."""
    _check(load().stats_accumulate_file(ctx.handle, _path(path), row0, nrows, chunk_rows, _stream_handle(stream)),
           "stats_accumulate_file")


# ----------------------------------------------------------------------------- CSV text (stats_csv.h)
T1_CSV_HEADER = "A,B,C,D,E,F,G,H,cotC,I,J,K"


def _csv_error(code, where, bad):
    err = StatsError(code, where)
    err.bad_line = bad
    return err


def stats_csv_write(path, dtypes: Sequence[int], nrows: int, hcols: Sequence, header: str | None = None):
    """Write an n x p table from host columns as CSV text (optional header line)."""
    p = len(dtypes)
    dt = (ctypes.c_int32 * p)(*dtypes)
    _check(load().stats_csv_write(_path(path), p, dt, nrows, _ptr_array(hcols),
                                  None if header is None else header.encode()), "stats_csv_write")


def stats_csv_write_table1(path, seed: int, nrows: int, layout: int = STATS_T1_L32, row0: int = 0,
                           chunk_rows: int = 0):
    """Write Table 1 rows [row0, row0 + nrows), generated on the current device, as CSV with a header."""
    _check(load().stats_csv_write_table1(_path(path), seed, row0, nrows, layout, chunk_rows),
           "stats_csv_write_table1")


def stats_csv_parse(d_text, nbytes: int, dtypes: Sequence[int], d_cols: Sequence, max_rows: int, stream=None) -> int:
    """Parse the first len(dtypes) fields of every line of device text into device columns; returns
    the number of lines, raises StatsError with .bad_line on a parse error."""
    k = len(dtypes)
    dt = (ctypes.c_int32 * k)(*dtypes)
    n = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    code = load().stats_csv_parse(_ptr(d_text) if nbytes else None, nbytes, k, dt, _ptr_array(d_cols), max_rows,
                                  ctypes.byref(n), ctypes.byref(bad), _stream_handle(stream))
    if code != STATS_OK:
        raise _csv_error(code, "stats_csv_parse", bad.value)
    return n.value


def stats_accumulate_csv(ctx: Ctx, path, skip_lines: int = 1, chunk_bytes: int = 0, stream=None) -> int:
    """Stream a CSV file's first ctx.p fields into ctx (after skip_lines header lines); returns the
    records added, raises StatsError with .bad_line (the file line) on a parse error."""
    n = ctypes.c_int64(0)
    bad = ctypes.c_int64(-1)
    code = load().stats_accumulate_csv(ctx.handle, _path(path), skip_lines, chunk_bytes, ctypes.byref(n),
                                       ctypes.byref(bad), _stream_handle(stream))
    if code != STATS_OK:
        err = _csv_error(code, "stats_accumulate_csv", bad.value)
        err.rows_added = n.value
        raise err
    return n.value
