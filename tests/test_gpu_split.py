"""FP32 tables through the bf16-split tensor-core modes (BF16x3, BF16x4), against
the double-double oracle on the same float32 values.

Inputs follow the shapes of the batched-tables and wide-table workloads:
independent columns x ~ N(mu_j, sigma_j^2) with mu_j ~ U[1e3, 1e5] and
sigma_j ~ U[0.1, 10] (a mean-to-spread ratio up to 1e6 stresses centering), and
a correlated table X = Z L^T + mu with eigenvalues 1/k.  Generated on the host
with numpy (seeded) and handed to both sides.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")


def independent_table(seed, n, p):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(1e3, 1e5, p)
    sd = rng.uniform(0.1, 10.0, p)
    return (mu + sd * rng.standard_normal((n, p))).astype(np.float32)


def correlated_table(seed, n, p):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    cov = (q * (1.0 / np.arange(1, p + 1))) @ q.T
    L = np.linalg.cholesky(cov)
    mu = rng.uniform(0.0, 1e3, p)
    return (rng.standard_normal((n, p)) @ L.T + mu).astype(np.float32)


def run_mode(X, mode, flush_rows=None):
    n, p = X.shape
    cols = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    cfg = G.Config([G.STATS_F32] * p, mode, [0] * p)
    with G.stats_init(cfg) as ctx:
        if flush_rows:
            G.stats_set_flush_rows(ctx, flush_rows)
        G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx)
    return raw, an


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sums_within_fp32_bound(s, X):
    """Column sums of the FP32 split passes: each value enters as r = fl32(x - c) and r is
    summed in FP32 a few values at a time into (hi, lo) pairs, so the error of column j is at
    most a few units in the last place of the |x - c| it sums: 2^-22 sum_i |x_ij - mean_j|
    (a relative test would fail on a column whose values cross zero, where the sum is small
    next to the values)."""
    X64 = X.astype(np.float64)
    exact = np.array([float(np.sum(X64[:, j])) for j in range(X.shape[1])])
    bound = 2.0 ** -22 * np.abs(X64 - X64.mean(axis=0)).sum(axis=0) + 1e-12 * np.abs(exact)
    return bool(np.all(np.abs(s - exact) <= bound)), float(np.max(np.abs(s - exact) / bound))


@pytest.mark.parametrize("p", [8, 16, 32, 64])
@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
def test_split_independent_columns(p, mode):
    n = 200_003
    X = independent_table(100 + p, n, p)
    raw, an = run_mode(X, mode)
    cols = [X[:, j].astype(np.float64) for j in range(p)]
    cov = O.cov_twopass_columns(cols)
    st = O.stats_columns(cols)
    assert raw.n == n
    err = rel_fro(an.cov, cov)
    mean_err = float(np.max(np.abs(an.mean - st.s_float() / n) / np.abs(st.s_float() / n)))
    print(f"\nmode={mode} p={p}: cov rel-Frobenius error {err:.3e}, mean rel error {mean_err:.3e}")
    assert mean_err < 1e-9
    # both meet 2e-6: BF16x3 drops the off-diagonal of L^T L (sums of products of rounding
    # residuals, which cancel) and adds its diagonal (a positive bias ~2^-16 relative otherwise)
    assert err < 2e-6


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
def test_split_correlated_wide(mode):
    n, p = 40_000, 256
    X = correlated_table(4, n, p)
    raw, an = run_mode(X, mode)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    err = rel_fro(an.cov, cov)
    ev_ref = np.linalg.eigvalsh(cov)[::-1][:10]
    ev_err = float(np.max(np.abs(an.evals[:10] - ev_ref) / ev_ref))
    print(f"\nmode={mode} p=256: cov rel-Frobenius error {err:.3e}, top-10 eigenvalue rel error {ev_err:.3e}")
    assert err < 2e-6
    assert ev_err < 1e-4


@pytest.mark.parametrize("flush", [16, 32, 64, 256])
def test_split_flush_interval_sweep(flush):
    """Error of both modes against the flush interval of the FP32 tensor accumulators (reported)."""
    n, p = 200_003, 8
    X = independent_table(108, n, p)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    for mode in (G.STATS_BF16X3, G.STATS_BF16X4):
        _, an = run_mode(X, mode, flush)
        print(f"\nflush={flush} mode={mode} p={p}: cov rel-Frobenius error {rel_fro(an.cov, cov):.3e}")


# --------------------------------------------------------------------------- CUDA-core comparators, any width
@pytest.mark.parametrize("p", [13, 40, 256])
def test_wide_fp64_modes(p):
    """FP64 (raw and shifted) on tables wider than the row-parallel kernel: the tiled pass."""
    n = 30_011 if p == 256 else 100_003
    X = correlated_table(7 + p, n, p).astype(np.float64)
    cols64 = [np.ascontiguousarray(X[:, j]) for j in range(p)]
    st = O.stats_columns(cols64)
    cov = O.cov_twopass_columns(cols64)
    S = st.S_float()
    for mode in (G.STATS_FP64, G.STATS_FP64_SHIFTED):
        dev = [torch.from_numpy(c).cuda() for c in cols64]
        cfg = G.Config([G.STATS_F64] * p, mode, [0] * p)
        with G.stats_init(cfg) as ctx:
            G.stats_accumulate(ctx, dev, n)
            raw = G.stats_raw(ctx)
            an = G.stats_finalize(ctx)
        assert raw.n == n
        assert rel_fro(raw.S, S) < 1e-13, mode
        assert np.max(np.abs(raw.s - st.s_float()) / np.abs(st.s_float())) < 1e-13
        err = rel_fro(an.cov, cov)
        print(f"\nFP64 mode={mode} p={p}: cov rel-Frobenius error {err:.3e}")
        # raw moments (S - s s^T / n) cancel: with mean/spread up to 1e3 the paper's formula
        # loses ~6 digits to rounding; the shifted pass keeps full precision
        assert err < (1e-6 if mode == G.STATS_FP64 else 1e-12)


@pytest.mark.parametrize("p", [8, 64, 256])
def test_fp32_core_mode(p):
    """The FP32 CUDA-core comparator (shifted): error reported against the oracle."""
    n = 40_000 if p == 256 else 200_003
    X = correlated_table(11, n, p) if p == 256 else independent_table(200 + p, n, p)
    raw, an = run_mode(X, G.STATS_FP32)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    err = rel_fro(an.cov, cov)
    print(f"\nFP32-core p={p}: cov rel-Frobenius error {err:.3e}")
    assert raw.n == n
    assert err < 1e-4


# --------------------------------------------------------------------------- batched tables
def test_batched_many_tables_one_pass():
    """Independent FP32 tables of uneven sizes and widths in one batched call (two calls in a row),
    each table against the oracle; p in {8, 16, 32, 64}, rows log-uniform."""
    rng = np.random.default_rng(3)
    ntab = 48
    ps = rng.choice([8, 16, 32, 64], ntab)
    ns = np.exp(rng.uniform(np.log(1e3), np.log(1.2e5), ntab)).astype(np.int64)
    tables = [independent_table(1000 + t, int(ns[t]), int(ps[t])) for t in range(ntab)]
    ctxs = [G.stats_init(G.Config([G.STATS_F32] * int(ps[t]), G.STATS_BF16X4, [0] * int(ps[t])))
            for t in range(ntab)]
    halves = []
    for part in range(2):  # the first and second halves of every table, in two batched calls
        dev, rows = [], []
        for t, X in enumerate(tables):
            h = X.shape[0] // 2
            Xp = X[:h] if part == 0 else X[h:]
            dev.append([torch.from_numpy(np.ascontiguousarray(Xp[:, j])).cuda() for j in range(Xp.shape[1])])
            rows.append(Xp.shape[0])
        halves.append(dev)
        G.stats_accumulate_batched(ctxs, dev, rows)
    worst = 0.0
    for t, X in enumerate(tables):
        an = G.stats_finalize(ctxs[t])
        raw = G.stats_raw(ctxs[t])
        assert raw.n == X.shape[0]
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(X.shape[1])])
        worst = max(worst, rel_fro(an.cov, cov))
        ctxs[t].close()
    print(f"\nbatched BF16x4, {ntab} tables: worst cov rel-Frobenius error {worst:.3e}")
    assert worst < 2e-6


# --------------------------------------------------------------------------- register-fragment pass (p <= 64)
def run_cols(cols, n, mode, batched=False):
    p = len(cols)
    cfg = G.Config([G.STATS_F32] * p, mode, [0] * p)
    with G.stats_init(cfg) as ctx:
        if batched:
            G.stats_accumulate_batched([ctx], [cols], [n])
        else:
            G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx) if n >= 2 else None  # covariance needs two rows
    return raw, an


@pytest.mark.parametrize("p", [1, 5, 11, 19, 40, 63])
@pytest.mark.parametrize("n", [1, 15, 17, 1000, 100_003])
def test_fragment_pass_widths_and_ragged_rows(p, n):
    """Widths padded to 8/16/32/64 and row counts that end inside a K block, a chunk or a unit;
    columns cut from one [p, n] tensor (16-byte aligned only when n is a multiple of 4)."""
    X = independent_table(300 + p, n, p)
    dev = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    cols = [dev[j] for j in range(p)]
    raw, an = run_cols(cols, n, G.STATS_BF16X4)
    st = O.stats_columns([X[:, j].astype(np.float64) for j in range(p)])
    assert raw.n == n
    if n == 1:  # one row: the shifted sums are zero and S' = 0; raw moments are the row itself
        assert np.allclose(raw.s, X[0].astype(np.float64), rtol=1e-12, atol=0)
        return
    assert np.allclose(an.mean, st.s_float() / n, rtol=1e-9, atol=0)
    if n >= 2:
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
        scale = np.linalg.norm(cov)
        if scale > 0:
            assert rel_fro(an.cov, cov) < 2e-6, (p, n)


def test_fragment_pass_aligned_and_unaligned_agree():
    """The same table through 16-byte aligned columns (bulk 16-byte copies) and through
    columns offset by one float (4-byte copies): identical statistics."""
    n, p = 50_001, 32
    X = independent_table(77, n, p)
    a = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    ld = (n + 1 + 3) // 4 * 4  # row stride a multiple of 4 floats: every column starts 4 bytes past 16
    buf = torch.zeros((p, ld), dtype=torch.float32, device="cuda")
    for j in range(p):
        buf[j, 1:n + 1] = a[j]
    u = [buf[j, 1:n + 1] for j in range(p)]
    assert all(c.data_ptr() % 16 == 0 for c in a) and all(c.data_ptr() % 16 == 4 for c in u)
    ra, aa = run_cols(a, n, G.STATS_BF16X4)
    ru, au = run_cols(u, n, G.STATS_BF16X4)
    assert np.array_equal(ra.S, ru.S) and np.array_equal(ra.s, ru.s)
    assert np.array_equal(aa.cov, au.cov)


def test_fragment_pass_reproducible_bits():
    """Two runs of the same call give bit-identical results (fixed order of every addition)."""
    n, p = 300_007, 64
    X = independent_table(78, n, p)
    cols = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    r1, a1 = run_cols(cols, n, G.STATS_BF16X3)
    r2, a2 = run_cols(cols, n, G.STATS_BF16X3)
    assert np.array_equal(r1.S, r2.S) and np.array_equal(r1.s, r2.s)
    assert np.array_equal(a1.cov, a2.cov)


def test_fragment_pass_batched_equals_single_within_rounding():
    """One table through the batched entry point and through the single-table entry point
    (different unit splits): equal to rounding."""
    n, p = 200_003, 16
    X = independent_table(79, n, p)
    cols = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    _, a1 = run_cols(cols, n, G.STATS_BF16X4)
    _, a2 = run_cols(cols, n, G.STATS_BF16X4, batched=True)
    assert rel_fro(a1.cov, a2.cov) < 1e-7


@pytest.mark.parametrize("p", [33, 64])
def test_fragment_pass_tensor_copy_and_column_copies_agree(p):
    """Columns of one [p, ld] block (ld a multiple of 4: one 2D tensor copy per stage) and the
    same columns as separate allocations (one bulk copy per column): bit-identical statistics."""
    n = 100_003
    X = independent_table(81 + p, n, p)
    ld = (n + 3) // 4 * 4
    blk = torch.zeros((p, ld), dtype=torch.float32, device="cuda")
    blk[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    strided = [blk[j, :n] for j in range(p)]
    separate = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    r1, a1 = run_cols(strided, n, G.STATS_BF16X4)
    r2, a2 = run_cols(separate, n, G.STATS_BF16X4)
    assert np.array_equal(r1.S, r2.S) and np.array_equal(r1.s, r2.s)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    assert rel_fro(a1.cov, cov) < 2e-6


# --------------------------------------------------------------------------- merging shifted contexts
@pytest.mark.parametrize("mode", [G.STATS_FP64_SHIFTED, G.STATS_FP32, G.STATS_BF16X3, G.STATS_BF16X4])
@pytest.mark.parametrize("p", [16, 64, 96])
def test_merge_shifted_modes(mode, p):
    """Two disjoint row ranges in two contexts (different pivots: each its own first row), merged,
    against one context over all rows and against the oracle; the merged context then takes more rows."""
    n = 60_011
    X = independent_table(500 + p, n, p)
    if mode == G.STATS_FP64_SHIFTED:
        dt, Xd = G.STATS_F64, X.astype(np.float64)
    else:
        dt, Xd = G.STATS_F32, X
    h1, h2 = 20_000, 45_000
    def ctx_on(rows):
        c = G.stats_init(G.Config([dt] * p, mode, [0] * p))
        if rows.shape[0]:
            G.stats_accumulate(c, [torch.from_numpy(np.ascontiguousarray(rows[:, j])).cuda() for j in range(p)],
                               rows.shape[0])
        return c
    a, b, c = ctx_on(Xd[:h1]), ctx_on(Xd[h1:h2]), ctx_on(Xd[h2:])
    G.stats_merge(a, b)
    G.stats_merge(a, c)
    raw = G.stats_raw(a)
    an = G.stats_finalize(a)
    st = O.stats_columns([Xd[:, j].astype(np.float64) for j in range(p)])
    cov = O.cov_twopass_columns([Xd[:, j].astype(np.float64) for j in range(p)])
    assert raw.n == n
    # column sums: the tiled kernel (p > 64) sums h + l, which carries each value to ~2^-17
    assert np.max(np.abs(raw.s - st.s_float()) / np.abs(st.s_float())) < (1e-12 if mode == G.STATS_FP64_SHIFTED
                                                                         else 1e-10)
    tol = {G.STATS_FP64_SHIFTED: 1e-12, G.STATS_FP32: 1e-4, G.STATS_BF16X4: 2e-6, G.STATS_BF16X3: 2e-6}[mode]
    err = rel_fro(an.cov, cov)
    print(f"\nmerge mode={mode} p={p}: cov rel-Frobenius error {err:.3e}")
    assert err < tol
    for x in (a, b, c):
        x.close()


def test_merge_into_empty_and_export_import_shifted():
    """An empty context takes the other's pivot on merge; export/import keeps the pivot, and the
    imported context can take more rows of the same table."""
    n, p = 40_000, 32
    X = independent_table(600, n, p)
    cols = lambda R: [torch.from_numpy(np.ascontiguousarray(R[:, j])).cuda() for j in range(p)]
    cfg = G.Config([G.STATS_F32] * p, G.STATS_BF16X4, [0] * p)
    full = G.stats_init(cfg)
    G.stats_accumulate(full, cols(X), n)
    part = G.stats_init(cfg)
    G.stats_accumulate(part, cols(X[:25_000]), 25_000)
    empty = G.stats_init(cfg)
    G.stats_merge(empty, part)
    blob = G.stats_export(empty)
    imp = G.stats_import(blob, p, G.STATS_BF16X4)
    G.stats_accumulate(imp, cols(X[25_000:]), n - 25_000)
    a1 = G.stats_finalize(full)
    a2 = G.stats_finalize(imp)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    assert rel_fro(a2.cov, cov) < 2e-6 and rel_fro(a1.cov, cov) < 2e-6
    assert G.stats_raw(imp).n == n
    for x in (full, part, empty, imp):
        x.close()


# --------------------------------------------------------------------------- wide tables on tcgen05
def block_cols(X):
    """Columns of X as rows of one [p, ld] device block (ld a multiple of 4 floats): the layout
    that the wide tcgen05 pass reads with 2D tensor copies."""
    n, p = X.shape
    ld = (n + 3) // 4 * 4
    blk = torch.zeros((p, ld), dtype=torch.float32, device="cuda")
    blk[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    return blk, [blk[j, :n] for j in range(p)]


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
@pytest.mark.parametrize("p,n", [(96, 40_000), (128, 33), (200, 100_003), (256, 40_000), (160, 20_011),
                                 (256, 32_007), (130, 64 * 77 + 32)])
def test_wide_tcgen05_pass(mode, p, n):
    """p > 64 from a [p, ld] block (the tcgen05 pass): against the oracle, and against the tiled
    kernel on the same values (separate column allocations)."""
    X = correlated_table(9 + p, n, p) if p >= 200 else independent_table(900 + p, n, p)
    blk, cols = block_cols(X)
    raw, an = run_cols(cols, n, mode)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    st = O.stats_columns([X[:, j].astype(np.float64) for j in range(p)])
    err = rel_fro(an.cov, cov)
    print(f"\nwide tcgen05 mode={mode} p={p} n={n}: cov rel-Frobenius error {err:.3e}")
    assert raw.n == n
    ok, worst = sums_within_fp32_bound(raw.s, X)
    assert ok, worst
    # BF16x3 drops the off-diagonal of L^T L, sums of products of rounding residuals that cancel
    # only as 1/sqrt(n); below 64 p rows a BF16x3 context forms all four products instead
    tol = 2e-6
    assert err < tol
    sep = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    _, an2 = run_cols(sep, n, mode)
    assert rel_fro(an.cov, an2.cov) < tol


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
@pytest.mark.parametrize("p,n", [(64, (1 << 20) + 7), (33, (1 << 20) + 45), (48, (1 << 20) + 63),
                                 (40, (1 << 20) + 64 * 77 + 32), (64, 3_000_001)])
def test_narrow_tcgen05_pass(mode, p, n):
    """33..64 columns from a [p, ld] block, calls of at least 2^20 rows (the tcgen05 pass with h and
    l stacked into one M = 128 operand), ragged tails in either 32-row chunk of the last stage:
    against the oracle, and against the register-fragment pass on the same values (separate
    column allocations)."""
    X = independent_table(700 + p, n, p)
    blk, cols = block_cols(X)
    raw, an = run_cols(cols, n, mode)
    st = O.stats_columns([X[:, j].astype(np.float64) for j in range(p)])
    assert raw.n == n
    assert np.max(np.abs(raw.s - st.s_float()) / np.abs(st.s_float())) < 1e-9
    if n >= 2:
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
        err = rel_fro(an.cov, cov)
        print(f"\nnarrow tcgen05 mode={mode} p={p} n={n}: cov rel-Frobenius error {err:.3e}")
        tol = 2e-6
        assert err < tol
        sep = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
        _, an2 = run_cols(sep, n, mode)
        assert rel_fro(an.cov, an2.cov) < tol


def test_narrow_in_a_batch_and_across_calls():
    """A batch mixing a large 64-column block with small tables (one register-fragment launch); the
    large table also split into two calls of different paths (fragment pass, then tcgen05)."""
    rng = np.random.default_rng(8)
    big = independent_table(801, 1_200_001, 64)
    small = [independent_table(810 + t, int(rng.integers(1000, 50_000)), int(rng.choice([8, 40, 64])))
             for t in range(6)]
    tabs = [big] + small
    blocks = [block_cols(X) for X in tabs]
    ctxs = [G.stats_init(G.Config([G.STATS_F32] * X.shape[1], G.STATS_BF16X3, [0] * X.shape[1])) for X in tabs]
    G.stats_accumulate_batched(ctxs, [b[1] for b in blocks], [X.shape[0] for X in tabs])
    for X, c in zip(tabs, ctxs):
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(X.shape[1])])
        assert rel_fro(G.stats_finalize(c).cov, cov) < 2e-6
        c.close()
    # two calls: rows [0, 4) through the fragment pass (too few rows for a tensor copy), the
    # rest through tcgen05; the pivot of the first call serves both
    X = big
    blk, _ = block_cols(X)
    with G.stats_init(G.Config([G.STATS_F32] * 64, G.STATS_BF16X4, [0] * 64)) as c:
        G.stats_accumulate(c, [blk[j, 0:4] for j in range(64)], 4)
        G.stats_accumulate(c, [blk[j, 4:X.shape[0]] for j in range(64)], X.shape[0] - 4)
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(64)])
        assert rel_fro(G.stats_finalize(c).cov, cov) < 2e-6


def test_wide_tcgen05_long_paced():
    """Enough 64-row stages per CTA that the units pace one another: against the oracle, and
    chunked into three calls of uneven length (ragged tails inside a stage each time)."""
    n, p = 300_003, 160
    X = independent_table(960, n, p)
    blk, cols = block_cols(X)
    raw, an = run_cols(cols, n, G.STATS_BF16X3)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    assert rel_fro(an.cov, cov) < 2e-6
    ctx = G.stats_init(G.Config([G.STATS_F32] * p, G.STATS_BF16X3, [0] * p))
    for a, b in ((0, 100_004), (100_004, 100_036), (100_036, n)):  # 16-byte aligned starts
        G.stats_accumulate(ctx, [blk[j, a:b] for j in range(p)], b - a)
    an2 = G.stats_finalize(ctx)
    ctx.close()
    assert rel_fro(an2.cov, cov) < 2e-6


def test_wide_tcgen05_reproducible_and_ragged():
    """Two identical calls give identical bits; a row count ending inside a stage."""
    n, p = 70_001, 160
    X = independent_table(950, n, p)
    blk, cols = block_cols(X)
    r1, _ = run_cols(cols, n, G.STATS_BF16X3)
    r2, _ = run_cols(cols, n, G.STATS_BF16X3)
    assert np.array_equal(r1.S, r2.S) and np.array_equal(r1.s, r2.s)


# --------------------------------------------------------------------------- batched finalize
def test_finalize_batched_matches_single():
    """Many contexts of different widths and modes finalized in one launch: mean, cov and corr
    identical to finalizing each alone, and so are the eigenpairs below 24 analysis columns;
    from 24 columns a single finalize takes the grid-wide eigen-solver and the batched one the
    one-block solver, which agree to rounding.  A context with one row is reported and skipped."""
    rng = np.random.default_rng(5)
    ctxs, singles = [], []
    for t, (p, mode) in enumerate([(8, G.STATS_BF16X4), (16, G.STATS_BF16X3), (33, G.STATS_BF16X4),
                                   (64, G.STATS_BF16X3), (96, G.STATS_BF16X4), (12, G.STATS_FP64_SHIFTED),
                                   (40, G.STATS_FP32)] * 3):
        n = int(rng.integers(1_000, 20_000))
        X = independent_table(2000 + t, n, p)
        dt = G.STATS_F64 if mode == G.STATS_FP64_SHIFTED else G.STATS_F32
        Xd = X.astype(np.float64) if dt == G.STATS_F64 else X
        c = G.stats_init(G.Config([dt] * p, mode, [0] * p))
        G.stats_accumulate(c, [torch.from_numpy(np.ascontiguousarray(Xd[:, j])).cuda() for j in range(p)], n)
        ctxs.append(c)
    for pca_on in (0, 1):
        singles = [G.stats_finalize(c, pca_on) for c in ctxs]
        batched = G.stats_finalize_batched(ctxs, pca_on)
        for a, b in zip(singles, batched):
            for f in ("mean", "cov", "corr"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), f
            pa = len(a.evals)
            if pa < 24:
                assert np.array_equal(a.evals, b.evals) and np.array_equal(a.evecs, b.evecs)
                continue
            scale = np.abs(b.evals).max()
            assert np.abs(a.evals - b.evals).max() <= 2e-15 * pa * scale
            gaps = np.abs(np.diff(b.evals))
            for k in range(pa):
                sep = min(gaps[k - 1] if k > 0 else np.inf, gaps[k] if k < len(gaps) else np.inf)
                if sep > 1e-6 * scale:
                    assert np.abs(a.evecs[k] - b.evecs[k]).max() <= 1e-8, k
    one = G.stats_init(G.Config([G.STATS_F32] * 8, G.STATS_BF16X4, [0] * 8))
    G.stats_accumulate(one, [torch.ones(1, device="cuda") for _ in range(8)], 1)
    with pytest.raises(G.StatsError):
        G.stats_finalize_batched(ctxs[:2] + [one])
    for c in ctxs + [one]:
        c.close()


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
def test_narrow_batch_persistent_launch(mode):
    """Tables of 33..64 columns in one batched call share one persistent tcgen05 launch (units of
    at most 2^20 rows, dealt largest first, one slot each, merged per table in row order):
    every table against the oracle, against its own single-table call, and the batch rerun
    bit for bit.  Sizes: several units per table with a ragged tail, one unit, just above the
    batch threshold."""
    specs = [(2_100_003, 64), (300_001, 40), (4_096, 33), (70_000, 64), (1_048_577, 48)]
    tabs = [independent_table(1200 + t, n, p) for t, (n, p) in enumerate(specs)]
    blocks = [block_cols(X) for X in tabs]
    mk = lambda X: G.stats_init(G.Config([G.STATS_F32] * X.shape[1], mode, [0] * X.shape[1]))  # noqa: E731
    ctxs = [mk(X) for X in tabs]
    again = [mk(X) for X in tabs]
    rows = [X.shape[0] for X in tabs]
    G.stats_accumulate_batched(ctxs, [b[1] for b in blocks], rows)
    G.stats_accumulate_batched(again, [b[1] for b in blocks], rows)
    for X, c, c2, (blk, cols) in zip(tabs, ctxs, again, blocks):
        p = X.shape[1]
        cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
        a = G.stats_finalize(c)
        assert rel_fro(a.cov, cov) < 2e-6
        r1, r2 = G.stats_raw(c), G.stats_raw(c2)
        assert np.array_equal(r1.S, r2.S) and np.array_equal(r1.s, r2.s) and r1.n == r2.n == X.shape[0]
        _, single = run_cols(cols, X.shape[0], mode)
        assert rel_fro(a.cov, single.cov) < 1e-6
        c.close()
        c2.close()


# --------------------------------------------------------------------------- BF16x3 at small row counts
def _cols_of(X, layout):
    if layout == "block":
        return block_cols(X)[1]
    return [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(X.shape[1])]


@pytest.mark.parametrize("p,n,layout", [(8, 17, "sep"), (16, 1000, "sep"), (40, 33, "sep"), (64, 33, "block"),
                                        (64, 4095, "block"), (96, 40, "sep"), (128, 33, "block"),
                                        (256, 100, "block"), (256, 16_383, "block")])
def test_bf16x3_small_tables_meet_tolerance(p, n, layout):
    """A BF16x3 context below 64 p rows forms all four products (its dropped off-diagonal L^T L
    would otherwise leave ~2.6e-6 sqrt(p / n)): the same bits as BF16x4 on the same call, and the
    stated 2e-6 against the oracle on every path (fragment pass, tcgen05 wide pass, tiled kernel)."""
    X = independent_table(3000 + p + n, n, p)
    cols = _cols_of(X, layout)
    r3, a3 = run_cols(cols, n, G.STATS_BF16X3)
    r4, a4 = run_cols(cols, n, G.STATS_BF16X4)
    assert np.array_equal(r3.S, r4.S) and np.array_equal(r3.s, r4.s)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    err = rel_fro(a3.cov, cov)
    print(f"\nBF16x3 p={p} n={n} {layout}: cov rel-Frobenius error {err:.3e}")
    assert err < 2e-6


@pytest.mark.parametrize("p,layout", [(64, "block"), (96, "sep"), (160, "block")])
def test_bf16x3_stream_of_small_calls(p, layout):
    """A stream of small BF16x3 calls crossing the 64 p row threshold (the first calls with four
    products, later ones with three): every snapshot within 2e-6 of the oracle on the rows so far."""
    n = 100 * p
    X = independent_table(4000 + p, n, p)
    blk = block_cols(X)[0] if layout == "block" else None
    bounds = [0, 33, 70, 64 * p - 5, 64 * p + 100, n]
    with G.stats_init(G.Config([G.STATS_F32] * p, G.STATS_BF16X3, [0] * p)) as ctx:
        for a, b in zip(bounds[:-1], bounds[1:]):
            if layout == "block":
                cols = [blk[j, a:b] for j in range(p)]
            else:
                cols = [torch.from_numpy(np.ascontiguousarray(X[a:b, j])).cuda() for j in range(p)]
            G.stats_accumulate(ctx, cols, b - a)
            an = G.stats_finalize(ctx) if b >= 2 else None
            cov = O.cov_twopass_columns([X[:b, j].astype(np.float64) for j in range(p)])
            err = rel_fro(an.cov, cov)
            print(f"\nBF16x3 stream p={p}: rows {b}: cov rel-Frobenius error {err:.3e}")
            assert err < 2e-6, b


def test_bf16x3_small_tables_batched():
    """Small BF16x3 tables of every path in one batched call, and a second call on the same
    contexts that takes them past the row threshold: each table within 2e-6 of the oracle."""
    rng = np.random.default_rng(17)
    specs = [(int(rng.integers(2, 3000)), int(rng.choice([8, 16, 40, 64, 96]))) for _ in range(24)]
    specs += [(4096, 40), (5000, 64), (2000, 130)]
    tabs = [independent_table(5000 + t, 2 * n + 999, p) for t, (n, p) in enumerate(specs)]
    ctxs = [G.stats_init(G.Config([G.STATS_F32] * X.shape[1], G.STATS_BF16X3, [0] * X.shape[1])) for X in tabs]
    blocks = [block_cols(X)[0] for X in tabs]
    cut = [n for n, _ in specs]
    for part in range(2):
        cols, rows = [], []
        for X, blk, h in zip(tabs, blocks, cut):
            a, b = (0, h) if part == 0 else (h, X.shape[0])
            cols.append([blk[j, a:b] for j in range(X.shape[1])])
            rows.append(b - a)
        G.stats_accumulate_batched(ctxs, cols, rows)
        worst = 0.0
        for X, c, h in zip(tabs, ctxs, cut):
            b = h if part == 0 else X.shape[0]
            cov = O.cov_twopass_columns([X[:b, j].astype(np.float64) for j in range(X.shape[1])])
            worst = max(worst, rel_fro(G.stats_finalize(c).cov, cov))
        print(f"\nBF16x3 batched small tables, call {part}: worst cov rel-Frobenius error {worst:.3e}")
        assert worst < 2e-6
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("mode", [G.STATS_BF16X3, G.STATS_BF16X4])
@pytest.mark.parametrize("p,n", [(130, 64 * 77 + 32), (200, 100_003), (256, 40_000), (256, 300_007), (129, 5_000),
                                 (160, 33)])
def test_wide_pairs_against_oracle_and_unit_kernel(mode, p, n):
    """129..256 columns in a [p, ld] block: the paired-CTA pass (each CTA of a pair converts one
    128-column block, cta_group::2 MMAs over both) against the oracle, and against the pass with
    one CTA per output block on the same values; ragged tails in either chunk of a stage, and a
    second call on the same context."""
    X = correlated_table(19 + p, n, p) if p >= 200 else independent_table(1900 + p, n, p)
    blk, cols = block_cols(X)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(p)])
    res = {}
    for pairs in (1, 0):
        with G.stats_init(G.Config([G.STATS_F32] * p, mode, [0] * p)) as ctx:
            G.stats_set_wide_pairs(ctx, pairs)
            G.stats_accumulate(ctx, cols, n)
            raw = G.stats_raw(ctx)
            res[pairs] = (raw, G.stats_finalize(ctx))
    (r1, a1), (r0, a0) = res[1], res[0]
    err = rel_fro(a1.cov, cov)
    print(f"\nwide pairs mode={mode} p={p} n={n}: cov rel-Frobenius error {err:.3e} (one CTA per block: "
          f"{rel_fro(a0.cov, cov):.3e})")
    assert r1.n == n
    assert err < 2e-6
    assert rel_fro(a1.cov, a0.cov) < 2e-6
    ok, worst = sums_within_fp32_bound(r1.s, X)
    assert ok, worst
    if n > 1000:  # two calls: rows [0, h) then [h, n), h a multiple of 4 (16-byte aligned views)
        h = (n // 3) // 4 * 4
        with G.stats_init(G.Config([G.STATS_F32] * p, mode, [0] * p)) as ctx:
            G.stats_accumulate(ctx, [blk[j, :h] for j in range(p)], h)
            G.stats_accumulate(ctx, [blk[j, h:n] for j in range(p)], n - h)
            assert rel_fro(G.stats_finalize(ctx).cov, cov) < 2e-6


def test_wide_pairs_reproducible():
    """The paired-CTA pass gives the same bits on two identical calls."""
    n, p = 120_001, 256
    X = correlated_table(77, n, p)
    _, cols = block_cols(X)
    r1, _ = run_cols(cols, n, G.STATS_BF16X3)
    r2, _ = run_cols(cols, n, G.STATS_BF16X3)
    assert np.array_equal(r1.S, r2.S) and np.array_equal(r1.s, r2.s)
