"""Pins of the CPU oracle against facts other than the oracle itself.

Each test names the fact it pins: published known-answer vectors, closed
forms, identities of the Table 1 formulas, correctly rounded values from an
independent 60-digit evaluation, brute force with exact rationals, an
independent (histogram) formulation, the paper's own Table 2 -> Table 3 worked
example, and a library eigensolver.  No expected value here comes from the
CUDA path.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    """Philox4x32-10 reproduces the generator's published known-answer vectors."""
    assert O.philox4x32_10(ctr, key) == expect


# --------------------------------------------------------------------------- Table 1 generator
def test_table1_identifier_and_ranges():
    """A = 1..n; B in [3,8], C in [1,10], D in [1,100] and every value occurs (Table 1)."""
    n = 200_000
    iv, rv = O.table1_rows(7, 0, n)
    assert np.array_equal(iv[:, 0], np.arange(1, n + 1))
    for col, lo, hi in ((1, 3, 8), (2, 1, 10), (3, 1, 100)):
        vals = np.unique(iv[:, col])
        assert vals.min() == lo and vals.max() == hi and len(vals) == hi - lo + 1
    # ranges of the derived integer columns, from the formulas
    E, F, G, H, I, K = (iv[:, j] for j in (4, 5, 6, 7, 9, 11))
    assert E.min() >= 0 and E.max() <= 209
    assert F.min() >= 0 and F.max() <= 41918
    assert G.min() >= 0 and G.max() <= 100 and H.min() >= 0 and H.max() <= 100
    assert I.min() >= 147 and I.max() <= 7015
    assert K.min() >= 0 and K.max() <= 100
    assert len(np.unique(rv[:, 8])) == 10 and len(np.unique(rv[:, 10])) == 100


def test_table1_uniform_draws_chi_square():
    """randBetween draws are uniform: chi-square of B, C, D counts within 6 sigma."""
    n = 600_000
    iv, _ = O.table1_rows(11, 0, n)
    for col, lo, hi in ((1, 3, 8), (2, 1, 10), (3, 1, 100)):
        k = hi - lo + 1
        counts = np.bincount(iv[:, col] - lo, minlength=k)
        chi2 = float(((counts - n / k) ** 2 / (n / k)).sum())
        assert abs(chi2 - (k - 1)) < 6 * math.sqrt(2 * (k - 1)), (col, chi2)


def test_table1_rows_independent_of_chunking():
    """Row i depends only on (seed, i): a window of rows equals the same rows of a longer run."""
    iv_a, rv_a = O.table1_rows(3, 0, 5000)
    iv_b, rv_b = O.table1_rows(3, 1234, 100)
    assert np.array_equal(iv_a[1234:1334], iv_b)
    assert np.array_equal(rv_a[1234:1334], rv_b)


def _cr(x):
    """Correctly rounded double of an mpmath value."""
    return float(x)


def test_table1_formulas_against_60_digit_evaluation():
    """E..K equal the Table 1 formulas evaluated with correctly rounded log/sin/cos/tan.

    The transcendental values come from mpmath at 60 digits, rounded once to
    double; the remaining IEEE double operations are the ones Table 1 prints.
    Every (B, C, D) cell is covered.
    """
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    iv, rv = O.table1_rows(5, 0, 400_000)
    seen = {}
    for r in range(iv.shape[0]):
        key = (int(iv[r, 1]), int(iv[r, 2]), int(iv[r, 3]))
        if key not in seen:
            seen[key] = r
    assert len(seen) == 6000
    logs = {v: _cr(mpmath.log(v)) for v in range(1, 101)}
    for (B, C, D), r in seen.items():
        E = math.trunc(logs[C] / logs[B] * 100.0)
        F = round_half_away(logs[D] / logs[B] * 10000.0)
        G = math.trunc(abs(_cr(mpmath.cos(C))) * 100.0)
        H = math.trunc(abs(_cr(mpmath.sin(D))) * 100.0)
        cot = 1.0 / _cr(mpmath.tan(C))
        I = round_half_away(abs(cot) * 1000.0)
        J = abs(_cr(mpmath.tan(D)))
        K = D // C
        assert (iv[r, 4], iv[r, 5], iv[r, 6], iv[r, 7], iv[r, 9], iv[r, 11]) == (E, F, G, H, I, K), (B, C, D)
        assert rv[r, 8] == cot and rv[r, 10] == J, (B, C, D)


def round_half_away(x: float) -> int:
    """C's round(): nearest integer, halves away from zero (never Python's round)."""
    f = math.floor(abs(x) + 0.5)
    return int(math.copysign(f, x))


def test_table1_identities():
    """Identities of the Table 1 formulas that hold in exact and in IEEE arithmetic.

    E(B, 1) = 0, E(B, B) = 100, F(B, 1) = 0, F(B, B) = 10000 (log 1 = 0, x/x = 1);
    E(4, 2) = 50 and E(3, 9) = 200 (log 4 = 2 log 2 and log 9 = 2 log 3 are exact
    doublings); I(C) for C = 1..10 from |cot C| * 1000.
    """
    iv, rv = O.table1_rows(9, 0, 300_000)
    B, C, D, E, F, I = (iv[:, j] for j in (1, 2, 3, 4, 5, 9))
    assert np.all(E[C == 1] == 0) and np.all(E[C == B] == 100)
    assert np.all(F[D == 1] == 0) and np.all(F[D == B] == 10000)
    assert np.all(E[(B == 4) & (C == 2)] == 50) and np.all(E[(B == 3) & (C == 9)] == 200)
    assert np.all(E[(B == 4) & (C == 8)] == 150)
    expect_I = {1: 642, 2: 458, 3: 7015, 4: 864, 5: 296, 6: 3436, 7: 1148, 8: 147, 9: 2211, 10: 1542}
    for c, v in expect_I.items():
        assert np.all(I[C == c] == v), c
    cot = rv[:, 8]
    assert np.all(np.sign(cot[C == 3]) < 0) and np.all(np.sign(cot[C == 1]) > 0)


# --------------------------------------------------------------------------- exact sums
@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 123_457])
def test_identifier_closed_forms(n):
    """Sum A = n(n+1)/2 and Sum A^2 = n(n+1)(2n+1)/6 exactly (the paper's column-sum check)."""
    st = O.stats_table1(1, n)
    assert st.n == n
    assert st.s[0] == n * (n + 1) // 2
    assert st.S[0][0] == n * (n + 1) * (2 * n + 1) // 6


def test_identifier_closed_forms_offset_window():
    """Rows [r0, r0+n) give Sum A = sum of r0+1..r0+n (chunking of the identifier)."""
    r0, n = 10**9 + 7, 5000
    st = O.stats_table1(2, n, row0=r0)
    assert st.s[0] == (r0 + n) * (r0 + n + 1) // 2 - r0 * (r0 + 1) // 2


@pytest.mark.parametrize("n", [1, 5, 64, 100])
def test_brute_force_exact_rationals(n):
    """(n, s, S) of Table 1 equal a brute-force sum in exact rationals over the same rows."""
    iv, rv = O.table1_rows(13, 0, n)
    st = O.stats_table1(13, n, threads=3)
    x = [[Fraction(float(rv[r, j])) if j in O.T1_REAL else Fraction(int(iv[r, j])) for j in range(12)]
         for r in range(n)]
    for j in range(12):
        s = sum(x[r][j] for r in range(n))
        assert Fraction(st.s[j]) == s if j not in O.T1_REAL else abs(Fraction(st.s[j]) - s) <= abs(s) * Fraction(1, 2**100)
        for k in range(j, 12):
            S = sum(x[r][j] * x[r][k] for r in range(n))
            got = Fraction(st.S[j][k])
            if j in O.T1_REAL or k in O.T1_REAL:
                assert abs(got - S) <= abs(S) * Fraction(1, 2**100) + Fraction(1, 2**200), (j, k)
            else:
                assert got == S, (j, k)


def test_histogram_formulation_agrees():
    """The per-row oracle equals the 6000-cell histogram formulation (a different algorithm)."""
    n = 300_001
    a = O.stats_table1(21, n, row0=17)
    b = O.stats_table1_hist(21, n, row0=17)
    assert a.n == b.n
    for j in range(12):
        for k in range(12):
            if j in O.T1_REAL or k in O.T1_REAL:
                assert abs(float(a.S[j][k] - b.S[j][k])) <= 1e-24 * abs(float(a.S[j][k])), (j, k)
            else:
                assert a.S[j][k] == b.S[j][k], (j, k)
        if j in O.T1_REAL:
            assert abs(float(a.s[j] - b.s[j])) <= 1e-24 * abs(float(a.s[j]))
        else:
            assert a.s[j] == b.s[j]


def test_thread_count_invariance():
    """Integer-valued entries do not depend on how rows are split over threads."""
    a = O.stats_table1(4, 50_001, threads=1)
    b = O.stats_table1(4, 50_001, threads=7)
    for j in range(12):
        for k in range(12):
            if j not in O.T1_REAL and k not in O.T1_REAL:
                assert a.S[j][k] == b.S[j][k]


def test_merge_of_disjoint_ranges():
    """stats(X1 u X2) = stats(X1) + stats(X2), exact for integer entries (the paper's partial sums)."""
    a = O.stats_table1(6, 70_000)
    b1 = O.stats_table1(6, 30_000)
    b2 = O.stats_table1(6, 40_000, row0=30_000)
    assert a.n == b1.n + b2.n
    for j in range(12):
        for k in range(12):
            if j not in O.T1_REAL and k not in O.T1_REAL:
                assert a.S[j][k] == b1.S[j][k] + b2.S[j][k]
            else:
                assert abs(float(a.S[j][k] - b1.S[j][k] - b2.S[j][k])) <= 1e-25 * abs(float(a.S[j][k]))


def test_population_means():
    """Sample means lie within 6 standard errors of the exact population means over the 6000 cells."""
    n = 1_000_000
    st = O.stats_table1(0, n)
    iv, rv = O.table1_rows(99, 0, 2_000_000)  # any rows: collect one value per cell
    cell = {}
    for r in range(iv.shape[0]):
        key = (int(iv[r, 1]), int(iv[r, 2]), int(iv[r, 3]))
        if key not in cell:
            cell[key] = rv[r]
        if len(cell) == 6000:
            break
    vals = np.array(list(cell.values()))  # each cell equally likely
    mu = vals.mean(axis=0)
    sd = vals.std(axis=0)
    for j in range(1, 12):
        m = float(st.s[j]) / n
        assert abs(m - mu[j]) < 6 * sd[j] / math.sqrt(n) + 1e-12, (O.T1_NAMES[j], m, mu[j])


def test_stats_columns_brute_force_signed_and_large():
    """Typed columns with negative and large integers, and reals, against exact rationals."""
    rng = np.random.default_rng(3)
    n = 257
    a = rng.integers(-2**40, 2**40, n, dtype=np.int64)
    b = rng.integers(-2**58, 2**58, n, dtype=np.int64)
    c = rng.standard_normal(n) * 1e3
    d = rng.integers(-5, 5, n, dtype=np.int64)
    st = O.stats_columns([a, b, d])  # integer only (b exceeds 2^53, allowed without reals)
    cols = [a, b, d]
    for j in range(3):
        assert st.s[j] == sum(int(v) for v in cols[j])
        for k in range(j, 3):
            assert st.S[j][k] == sum(int(x) * int(y) for x, y in zip(cols[j], cols[k]))
    st2 = O.stats_columns([a, c, d])
    cols2 = [[Fraction(int(v)) for v in a], [Fraction(float(v)) for v in c], [Fraction(int(v)) for v in d]]
    for j in range(3):
        for k in range(j, 3):
            S = sum(x * y for x, y in zip(cols2[j], cols2[k]))
            assert abs(Fraction(st2.S[j][k]) - S) <= abs(S) * Fraction(1, 2**100) + Fraction(1, 2**120)
    with pytest.raises(ValueError):
        O.stats_columns([b, c])  # int beyond 2^53 paired with a real column is refused
    big = np.full(300, 2**62, dtype=np.int64)
    with pytest.raises(OverflowError):
        O.stats_columns([big])  # 300 * 2^124 leaves the __int128 range: reported, not wrapped


# --------------------------------------------------------------------------- covariance / correlation
def test_twopass_cov_matches_exact_centering():
    """Two-pass covariance equals (n S - s s^T) / (n(n-1)) from exact sums, to a few ulps."""
    n = 200_000
    st = O.stats_table1(8, n)
    _, cov_exact, _ = O.analysis_from_stats(st, exclude=())
    cov2 = O.cov_twopass_table1(8, n)
    rel = np.abs(cov2 - cov_exact) / np.maximum(np.abs(cov_exact), 1e-300)
    assert rel.max() < 1e-13, rel.max()


def test_cov_shift_and_constant_invariants():
    """cov(X + c) = cov(X); a constant column has zero variance; diag(corr) = 1, |corr| <= 1."""
    rng = np.random.default_rng(1)
    n = 4000
    x = rng.standard_normal(n)
    y = 0.5 * x + rng.standard_normal(n)
    k = np.full(n, 3.25)
    cov = O.cov_twopass_columns([x, y, k])
    cov_s = O.cov_twopass_columns([x + 1e6, y - 1e6, k])
    assert np.allclose(cov[:2, :2], cov_s[:2, :2], rtol=1e-9, atol=0)
    assert cov[2, 2] == 0.0 and cov[0, 2] == 0.0
    ref = np.cov(np.vstack([x, y]))
    assert np.allclose(cov[:2, :2], ref, rtol=1e-12)
    corr = O.corr_from_cov(cov[:2, :2])
    assert corr[0, 0] == 1.0 and corr[1, 1] == 1.0 and abs(corr[0, 1]) <= 1.0
    assert np.isclose(corr[0, 1], np.corrcoef(x, y)[0, 1], rtol=1e-12)
    c3 = O.corr_from_cov(cov)
    assert math.isnan(c3[0, 2]) and math.isnan(c3[2, 2])


# --------------------------------------------------------------------------- eigensolver
def _paper_tables():
    T2 = np.loadtxt(os.path.join(GOLDEN, "paper_table2.txt"))
    ev, load = [], []
    with open(os.path.join(GOLDEN, "paper_table3.txt")) as f:
        for line in f:
            if line.startswith("eigen"):
                ev.append(float(line.split()[1]))
            elif line.startswith("load"):
                load.append([float(x) for x in line.split()[1:]])
    return T2, np.array(ev), np.array(load)


def test_jacobi_reproduces_paper_table3():
    """Jacobi on the paper's Table 2 gives Table 3: eigenvalues within 5e-6, loadings within 1e-6."""
    T2, ev3, load3 = _paper_tables()
    ev, V = O.jacobi(T2)
    assert np.all(np.diff(ev) <= 0)
    assert np.abs(ev - ev3).max() < 5e-6
    assert abs(ev.sum() - 10.0) < 1e-12  # trace of a correlation matrix
    for k in range(10):
        sg = 1.0 if V[k] @ load3[k] > 0 else -1.0
        assert np.abs(sg * V[k] - load3[k]).max() < 1e-6, k
    # variance % column of Table 3
    pct = 100.0 * ev / ev.sum()
    assert np.abs(pct - np.array([10.00010, 10.00010, 10.0, 10.0, 10.0, 9.99999, 9.99997, 9.99996, 9.99994,
                                  9.99993])).max() < 6e-5


@pytest.mark.parametrize("p", [2, 5, 11, 40, 129, 256])
def test_jacobi_against_lapack(p):
    """Eigenvalues equal numpy.linalg.eigh (LAPACK); V is orthonormal; A V^T = V^T diag(ev)."""
    rng = np.random.default_rng(p)
    M = rng.standard_normal((p, p))
    A = M @ M.T + np.diag(np.arange(p, dtype=float))
    ev, V = O.jacobi(A)
    ref = np.linalg.eigh(A)[0][::-1]
    assert np.allclose(ev, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert np.abs(V @ V.T - np.eye(p)).max() < 1e-12
    assert np.abs(A @ V.T - V.T * ev).max() < 1e-10 * np.abs(ev).max()
    for k in range(p):  # sign convention: largest component positive
        assert V[k, np.argmax(np.abs(V[k]))] > 0


def test_jacobi_repeated_eigenvalues_as_subspaces():
    """A spectrum with a triple and a double eigenvalue (Q diag(...) Q^T, Q Haar): the
    eigenvalues match to rounding, and the eigenvectors span the same subspaces (projectors)."""
    rng = np.random.default_rng(21)
    q, r = np.linalg.qr(rng.standard_normal((9, 9)))
    q = q * np.sign(np.diag(r))
    lam = np.array([5.0, 3.0, 3.0, 3.0, 2.0, 1.0, 1.0, 0.5, 0.25])
    A = (q * lam) @ q.T
    A = 0.5 * (A + A.T)
    ev, V = O.jacobi(A)
    assert np.allclose(ev, lam, rtol=0, atol=1e-13)
    for lo, hi in ((1, 4), (5, 7)):
        P = V[lo:hi].T @ V[lo:hi]
        Pq = q[:, lo:hi] @ q[:, lo:hi].T
        assert np.abs(P - Pq).max() < 1e-12
    for k in (0, 4, 7, 8):  # simple eigenvalues: the vector itself, up to the sign convention
        assert abs(abs(V[k] @ q[:, k]) - 1.0) < 1e-13


def test_corr_from_cov_definition():
    """corr_jk = cov_jk / sqrt(cov_jj cov_kk), unit diagonal, NaN rows and columns for a zero
    variance (the paper's undefined correlations), on a covariance of known correlations."""
    sd = np.array([2.0, 0.5, 3.0, 1.0])
    R = np.array([[1.0, 0.3, -0.2, 0.0], [0.3, 1.0, 0.5, 0.1], [-0.2, 0.5, 1.0, -0.4], [0.0, 0.1, -0.4, 1.0]])
    C = R * np.outer(sd, sd)
    assert np.allclose(O.corr_from_cov(C), R, rtol=0, atol=1e-15)
    C0 = C.copy()
    C0[2, :] = C0[:, 2] = 0.0
    K = O.corr_from_cov(C0)
    assert np.all(np.isnan(K[2, [0, 1, 3]])) and np.all(np.isnan(K[[0, 1, 3], 2]))
    assert K[0, 0] == 1.0 and abs(K[0, 1] - 0.3) < 1e-15
