"""CPU oracle for the fused sufficient-statistics pass (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` import this package.  It wraps ``oracle.c`` (plain C, built
with gcc by ``oracle/build.py``) through ctypes and returns exact Python
integers for integer-valued entries and (hi, lo) double-double pairs, folded
to ``float`` or ``fractions.Fraction``, for real-valued ones.

Paper: arxiv 2604.23826, Table 1 (the generator), "Data Representation and
Sufficient Statistics" (n, column sums, X^T X in one pass), "Numerical
Considerations" (exact / compensated accumulation, identifier exclusion),
"Principal Component Analysis Results" (eigenpairs of the p x p matrix).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

from . import build as _build

T1_P = 12
T1_NAMES = ("A", "B", "C", "D", "E", "F", "G", "H", "cotC", "I", "J", "K")
T1_REAL = (8, 10)          # cotC and J are real-valued (double) columns
T1_IDENTIFIER = 0          # A is the row identifier

_lib = None


def lib():
    """Load (building first if needed) liboracle.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_table1_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, i64p, f64p]
        for name in ("orc_stats_table1", "orc_stats_table1_hist"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, i64p, i64p, f64p,
                          i64p, f64p]
            f.restype = ctypes.c_int
        L.orc_stats_columns.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_int64, ctypes.c_int, i64p, i64p, f64p, i64p, f64p]
        L.orc_stats_columns.restype = ctypes.c_int
        L.orc_hist_table1.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, i64p, i64p,
                                      i64p]
        L.orc_hist_table1.restype = ctypes.c_int
        L.orc_cov_twopass_table1.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, f64p]
        L.orc_cov_twopass_table1.restype = ctypes.c_int
        L.orc_cov_twopass_columns.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int, f64p]
        L.orc_cov_twopass_columns.restype = ctypes.c_int
        L.orc_corr_from_cov.argtypes = [ctypes.c_int, f64p, f64p]
        L.orc_jacobi.argtypes = [ctypes.c_int, f64p, f64p, f64p, ctypes.c_int]
        L.orc_jacobi.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------- Philox / Table 1
def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return [int(x) for x in out]


def table1_rows(seed: int, row0: int, n: int):
    """Rows [row0, row0+n) of Table 1: (ints n x 12 int64, reals n x 12 float64).

    Integer-valued columns are exact in ``ints`` (and mirrored as floats in
    ``reals``); the real-valued columns cotC and J are valid in ``reals`` only.
    """
    iv = np.zeros((n, T1_P), dtype=np.int64)
    rv = np.zeros((n, T1_P), dtype=np.float64)
    lib().orc_table1_rows(seed, row0, n, _p(iv, ctypes.c_int64), _p(rv, ctypes.c_double))
    return iv, rv


# --------------------------------------------------------------------------- exact sums
def _i128(lo, hi) -> int:
    return (int(hi) << 64) + (int(lo) & 0xFFFFFFFFFFFFFFFF)


@dataclass
class Stats:
    """Exact sufficient statistics.

    ``s[j]`` and ``S[j][k]`` (full symmetric p x p lists) are Python ints where
    both columns are integer-valued, else ``Fraction`` values equal to the
    double-double result (error below n * 2^-104 relative).
    """
    p: int
    n: int
    kinds: tuple
    s: list
    S: list

    def s_float(self):
        return np.array([float(v) for v in self.s])

    def S_float(self):
        return np.array([[float(v) for v in row] for row in self.S])


def _unpack(p, kinds, n, s_int, s_dd, S_int, S_dd) -> Stats:
    s = []
    for j in range(p):
        if kinds[j] == 0:
            s.append(_i128(s_int[2 * j], s_int[2 * j + 1]))
        else:
            s.append(Fraction(float(s_dd[2 * j])) + Fraction(float(s_dd[2 * j + 1])))
    S = [[None] * p for _ in range(p)]
    t = 0
    for j in range(p):
        for k in range(j, p):
            if kinds[j] == 0 and kinds[k] == 0:
                v = _i128(S_int[2 * t], S_int[2 * t + 1])
            else:
                v = Fraction(float(S_dd[2 * t])) + Fraction(float(S_dd[2 * t + 1]))
            S[j][k] = v
            S[k][j] = v
            t += 1
    return Stats(p, int(n), tuple(kinds), s, S)


def _alloc(p):
    T = p * (p + 1) // 2
    return (np.zeros(1, np.int64), np.zeros(2 * p, np.int64), np.zeros(2 * p, np.float64),
            np.zeros(2 * T, np.int64), np.zeros(2 * T, np.float64))


def _ptrs(bufs):
    n, si, sd, Si, Sd = bufs
    return (_p(n, ctypes.c_int64), _p(si, ctypes.c_int64), _p(sd, ctypes.c_double), _p(Si, ctypes.c_int64),
            _p(Sd, ctypes.c_double))


T1_KINDS = tuple(1 if j in T1_REAL else 0 for j in range(T1_P))


def stats_table1(seed: int, n: int, row0: int = 0, threads: int | None = None) -> Stats:
    """Per-row exact (n, s, S) of Table 1 rows [row0, row0+n)."""
    bufs = _alloc(T1_P)
    rc = lib().orc_stats_table1(seed, row0, n, threads or default_threads(), *_ptrs(bufs))
    if rc < 0:
        raise RuntimeError(f"orc_stats_table1 failed: {rc}")
    return _unpack(T1_P, T1_KINDS, bufs[0][0], *bufs[1:])


def stats_table1_hist(seed: int, n: int, row0: int = 0, threads: int | None = None) -> Stats:
    """(n, s, S) of Table 1 rows [row0, row0+n) through the 6000-cell histogram."""
    bufs = _alloc(T1_P)
    rc = lib().orc_stats_table1_hist(seed, row0, n, threads or default_threads(), *_ptrs(bufs))
    if rc < 0:
        raise RuntimeError(f"orc_stats_table1_hist failed: {rc}")
    return _unpack(T1_P, T1_KINDS, bufs[0][0], *bufs[1:])


def hist_table1(seed: int, n: int, row0: int = 0, threads: int | None = None):
    """(count[6,10,100], sumA[6,10,100] as Python ints, sum of A^2)."""
    count = np.zeros(6000, np.int64)
    sumA = np.zeros(12000, np.int64)
    a2 = np.zeros(2, np.int64)
    lib().orc_hist_table1(seed, row0, n, threads or default_threads(), _p(count, ctypes.c_int64),
                          _p(sumA, ctypes.c_int64), _p(a2, ctypes.c_int64))
    sa = [_i128(sumA[2 * c], sumA[2 * c + 1]) for c in range(6000)]
    return count.reshape(6, 10, 100), sa, _i128(a2[0], a2[1])


def _columns(cols):
    """cols: list of 1-D arrays; int arrays -> kind 0 (as int64), float arrays -> kind 1 (as float64)."""
    kinds, keep = [], []
    for c in cols:
        a = np.asarray(c)
        if np.issubdtype(a.dtype, np.integer):
            kinds.append(0)
            keep.append(np.ascontiguousarray(a, dtype=np.int64))
        else:
            kinds.append(1)
            keep.append(np.ascontiguousarray(a, dtype=np.float64))
    n = len(keep[0]) if keep else 0
    for a in keep:
        if len(a) != n:
            raise ValueError("columns differ in length")
    ptrs = (ctypes.c_void_p * len(keep))(*[a.ctypes.data for a in keep])
    karr = (ctypes.c_int * len(kinds))(*kinds)
    return kinds, keep, ptrs, karr, n


def stats_columns(cols, threads: int | None = None) -> Stats:
    """Exact (n, s, S) of typed columns (integer arrays exact, float arrays in double-double)."""
    kinds, keep, ptrs, karr, n = _columns(cols)
    p = len(keep)
    bufs = _alloc(p)
    rc = lib().orc_stats_columns(p, karr, ptrs, n, threads or default_threads(), *_ptrs(bufs))
    if rc < 0:
        raise RuntimeError(f"orc_stats_columns failed: {rc}")
    if rc == 1:
        raise ValueError("an integer value paired with a real column exceeds 2^53")
    if rc == 2:
        raise OverflowError("an integer sum exceeds the __int128 range")
    return _unpack(p, kinds, bufs[0][0], *bufs[1:])


# --------------------------------------------------------------------------- covariance / PCA
def cov_twopass_table1(seed: int, n: int, row0: int = 0, threads: int | None = None):
    """Full 12 x 12 two-pass covariance (divisor n-1) of Table 1 rows."""
    cov = np.zeros((T1_P, T1_P), np.float64)
    rc = lib().orc_cov_twopass_table1(seed, row0, n, threads or default_threads(), _p(cov, ctypes.c_double))
    if rc < 0:
        raise RuntimeError(f"orc_cov_twopass_table1 failed: {rc}")
    return cov


def cov_twopass_columns(cols, threads: int | None = None):
    kinds, keep, ptrs, karr, n = _columns(cols)
    p = len(keep)
    cov = np.zeros((p, p), np.float64)
    rc = lib().orc_cov_twopass_columns(p, karr, ptrs, n, threads or default_threads(), _p(cov, ctypes.c_double))
    if rc < 0:
        raise RuntimeError(f"orc_cov_twopass_columns failed: {rc}")
    return cov


def corr_from_cov(cov):
    cov = np.ascontiguousarray(cov, dtype=np.float64)
    p = cov.shape[0]
    out = np.zeros_like(cov)
    lib().orc_corr_from_cov(p, _p(cov, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def jacobi(A, max_sweeps: int = 60):
    """Eigenpairs of symmetric A: (evals descending, evecs with row k = eigenvector k)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    p = A.shape[0]
    ev = np.zeros(p, np.float64)
    V = np.zeros((p, p), np.float64)
    sweeps = lib().orc_jacobi(p, _p(A, ctypes.c_double), _p(ev, ctypes.c_double), _p(V, ctypes.c_double),
                              max_sweeps)
    if sweeps < 0:
        raise RuntimeError("orc_jacobi failed")
    return ev, V


def analysis_from_stats(st: Stats, exclude=(T1_IDENTIFIER,)):
    """mean, cov, corr over the non-excluded columns from exact (n, s, S).

    Integer-exact centering: cov_jk = (n S_jk - s_j s_k) / (n (n-1)) in exact
    rationals, rounded once to double.  Used as the exact definition that the
    two-pass form and the GPU's finalize are both compared with.
    """
    keep = [j for j in range(st.p) if j not in exclude]
    n = st.n
    mean = np.array([float(Fraction(st.s[j]) / n) for j in keep])
    pa = len(keep)
    cov = np.zeros((pa, pa))
    for a, j in enumerate(keep):
        for b, k in enumerate(keep):
            num = Fraction(n) * Fraction(st.S[j][k]) - Fraction(st.s[j]) * Fraction(st.s[k])
            cov[a, b] = float(num / (n * (n - 1)))
    corr = corr_from_cov(cov)
    return mean, cov, corr
