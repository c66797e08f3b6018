"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer-valued entries of s and S must be bit-exact; entries involving the real
columns (cotC, J) within 1e-12 relative (the fixed-point field of the exact pass
quantises each value to 2^-52 of its declared range or better).  Inputs are
generated independently on both sides from the same seed (Philox counter =
row index), never copied from the device to the oracle.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")

REAL = O.T1_REAL
TOL_REAL = 1e-12


def _ctx(layout=G.STATS_T1_L32, max_rows=10**10, mode=G.STATS_EXACT):
    return G.stats_init(G.stats_table1_config(layout, max_rows, mode))


def _check_exact(raw, st, tol_real=TOL_REAL):
    assert raw.n == st.n
    for j in range(12):
        if j in REAL:
            ref = float(st.s[j])
            assert abs(raw.s[j] - ref) <= tol_real * max(abs(ref), 1e-300), (j, raw.s[j], ref)
        else:
            assert raw.s_exact[j] == st.s[j], (O.T1_NAMES[j], raw.s_exact[j], st.s[j])
            assert raw.s[j] == float(st.s[j])
        for k in range(j, 12):
            if j in REAL or k in REAL:
                ref = float(st.S[j][k])
                assert abs(raw.S[j, k] - ref) <= tol_real * abs(ref), (O.T1_NAMES[j], O.T1_NAMES[k], raw.S[j, k], ref)
            else:
                assert raw.S_exact[j][k] == st.S[j][k], (O.T1_NAMES[j], O.T1_NAMES[k])
                assert raw.S[j, k] == float(st.S[j][k])


# --------------------------------------------------------------------------- generator (a1)
@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
@pytest.mark.parametrize("row0,n", [(0, 100_003), (10**9 + 5, 4099), (2**33 - 3, 17)])
def test_generator_matches_oracle(layout, row0, n):
    """Device Table 1 rows equal the oracle's rows bit for bit (both from Philox at the row index)."""
    cols = G.gen_table1(seed=0, nrows=n, layout=layout, row0=row0)
    torch.cuda.synchronize()
    iv, rv = O.table1_rows(0, row0, n)
    for j in range(12):
        dev = cols[j][:n].cpu().numpy()
        if j in REAL:
            assert np.array_equal(dev, rv[:, j]), O.T1_NAMES[j]
        else:
            assert np.array_equal(dev.astype(np.int64), iv[:, j]), O.T1_NAMES[j]


# --------------------------------------------------------------------------- exact pass (a2-a5)
@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 31, 959, 960, 961, 1919, 12_345, 100_003])
def test_exact_ragged_sizes(n):
    """Exact pass over ragged row counts (tails < 8 rows, partial stages, several tiles)."""
    cols = G.gen_table1(seed=3, nrows=n)
    with _ctx() as ctx:
        G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
    _check_exact(raw, O.stats_table1(3, n))


def test_exact_empty():
    with _ctx() as ctx:
        G.stats_accumulate(ctx, [0] * 12, 0)
        raw = G.stats_raw(ctx)
    assert raw.n == 0 and all(v == 0 for v in raw.s_exact) and not raw.S.any()


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
def test_exact_1e6_seed0(layout):
    """The small Table 1 workload (n = 1e6, seed 0) in both layouts against the per-row oracle."""
    n = 10**6
    cols = G.gen_table1(seed=0, nrows=n, layout=layout)
    with _ctx(layout) as ctx:
        G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
    _check_exact(raw, O.stats_table1(0, n))
    assert raw.s_exact[0] == n * (n + 1) // 2
    assert raw.S_exact[0][0] == n * (n + 1) * (2 * n + 1) // 6


def test_exact_grid_chunk_and_repeat_invariance():
    """Bit-identical results for any grid size, any chunking, and on repeated runs."""
    n = 250_007
    cols = G.gen_table1(seed=5, nrows=n)
    outs = []
    for grid in (0, 1, 3, 152, 600):
        with _ctx() as ctx:
            G.stats_set_grid(ctx, grid)
            G.stats_accumulate(ctx, cols, n)
            outs.append(G.stats_raw(ctx))
    with _ctx() as ctx:  # chunked: uneven pieces, each a separate call
        edges = [0, 1, 9, 1000, 77_777, 77_778, 200_000, n]
        for a, b in zip(edges[:-1], edges[1:]):
            G.stats_accumulate(ctx, [c[a:] for c in cols], b - a)
        outs.append(G.stats_raw(ctx))
    ref = outs[0]
    for o in outs[1:]:
        assert o.n == ref.n and o.S_exact == ref.S_exact and np.array_equal(o.S, ref.S) and np.array_equal(o.s, ref.s)
    _check_exact(ref, O.stats_table1(5, n))


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
@pytest.mark.parametrize("n", [5, 17, 607, 608, 737, 895, 897, 100_003, 1_000_003])
def test_exact_launch_shapes_agree_with_oracle(layout, n):
    """Every launch shape of the exact pass (warps x rows per stage) against the oracle, ragged
    sizes around the shapes' stage lengths (608, 736, 896, 960 rows): bit-identical integer results."""
    cols = G.gen_table1(seed=11, nrows=n, layout=layout)
    st = O.stats_table1(11, n)
    raws = []
    for shape in (0, 1, 2, 3):
        with _ctx(layout) as ctx:
            G.stats_set_exact_shape(ctx, shape)
            G.stats_accumulate(ctx, cols, n)
            raws.append(G.stats_raw(ctx))
        _check_exact(raws[-1], st)
    for r in raws[1:]:
        assert r.S_exact == raws[0].S_exact and np.array_equal(r.S, raws[0].S) and np.array_equal(r.s, raws[0].s)


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
def test_exact_tcgen05_shape_grids_chunks_and_int32_flushes(layout):
    """The tcgen05 shape (3) on one block (about 1100 stages: ~980 accumulation chains, so the
    readers' int32 partial sums go to the int64 accumulator 15 times), on 3 and on 152 blocks,
    and in uneven chunks, each a separate call: bit-identical to the oracle and to shape 0."""
    n = 1_000_003
    cols = G.gen_table1(seed=21, nrows=n, layout=layout)
    st = O.stats_table1(21, n)
    raws = []
    for grid in (1, 3, 152):
        with _ctx(layout) as ctx:
            G.stats_set_exact_shape(ctx, 3)
            G.stats_set_grid(ctx, grid)
            G.stats_accumulate(ctx, cols, n)
            raws.append(G.stats_raw(ctx))
    with _ctx(layout) as ctx:
        G.stats_set_exact_shape(ctx, 3)
        edges = [0, 3, 899, 900, 17_000, 17_921, 500_000, n]
        for a, b in zip(edges[:-1], edges[1:]):
            G.stats_accumulate(ctx, [c[a:] for c in cols], b - a)
        raws.append(G.stats_raw(ctx))
    with _ctx(layout) as ctx:
        G.stats_set_exact_shape(ctx, 0)
        G.stats_accumulate(ctx, cols, n)
        raws.append(G.stats_raw(ctx))
    _check_exact(raws[0], st)
    for r in raws[1:]:
        assert r.n == raws[0].n and r.S_exact == raws[0].S_exact and np.array_equal(r.s, raws[0].s)


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_exact_launch_shapes_generic_and_unaligned(shape):
    """The generic converter in every shape, on aligned and unaligned columns (plain loads)."""
    rng = np.random.default_rng(13)
    n = 90_001
    vals = [rng.integers(-30000, 30000, n + 1, dtype=np.int16), rng.integers(-2**20, 2**20, n + 1, dtype=np.int32),
            rng.integers(-2**30, 2**30, n + 1, dtype=np.int64), (rng.standard_normal(n + 1) * 3.0)]
    cfg = G.Config([G.STATS_I16, G.STATS_I32, G.STATS_I64, G.STATS_F64], G.STATS_EXACT, [0, 0, 0, 0],
                   [-30000, -2**20, -2**30, -64.0], [30000, 2**20, 2**30, 64.0])
    whole = [torch.from_numpy(x).cuda() for x in vals]
    aligned = [torch.from_numpy(np.ascontiguousarray(x[1:])).cuda() for x in vals]
    unaligned = [d[1:] for d in whole]  # 2, 4 or 8 bytes past a 16-byte boundary
    st = O.stats_columns([v[1:].astype(np.int64) if v.dtype != np.float64 else v[1:] for v in vals])
    for cols in (aligned, unaligned):
        res = []
        for sh in (0, shape):
            with G.stats_init(cfg) as ctx:
                G.stats_set_exact_shape(ctx, sh)
                G.stats_accumulate(ctx, cols, n)
                res.append(G.stats_raw(ctx))
        assert res[0].S_exact == res[1].S_exact and np.array_equal(res[0].S, res[1].S)
        for j in range(3):
            for k in range(j, 3):
                assert res[1].S_exact[j][k] == st.S[j][k]
    with G.stats_init(cfg) as ctx:
        with pytest.raises(G.StatsError):
            G.stats_set_exact_shape(ctx, 4)


def test_exact_merge_export_import():
    """merge(stats(X1), stats(X2)) = stats(X1 u X2); an exported image re-imports unchanged."""
    n1, n2 = 123_456, 654_321
    a = G.gen_table1(seed=9, nrows=n1)
    b = G.gen_table1(seed=9, nrows=n2, row0=n1)
    with _ctx() as c1, _ctx() as c2:
        G.stats_accumulate(c1, a, n1)
        G.stats_accumulate(c2, b, n2)
        G.stats_merge(c1, c2)
        blob = G.stats_export(c1)
        r1 = G.stats_raw(c1)
    with G.stats_import(blob, 12, G.STATS_EXACT) as c3:
        r3 = G.stats_raw(c3)
    assert r1.S_exact == r3.S_exact and np.array_equal(r1.S, r3.S)
    _check_exact(r1, O.stats_table1(9, n1 + n2))


def test_exact_host_streamed():
    """stats_accumulate_host (double-buffered chunks from pinned memory) equals the device pass."""
    n = 300_001
    cols = G.gen_table1(seed=11, nrows=n)
    host = [c[:n].cpu().pin_memory() for c in cols]
    with _ctx() as ctx:
        G.stats_accumulate_host(ctx, host, n, chunk_rows=65_536)
        raw = G.stats_raw(ctx)
    _check_exact(raw, O.stats_table1(11, n))


def test_exact_range_error_rejects_call():
    """A value outside its digit field gives STATS_ERANGE and leaves the accumulator unchanged."""
    n = 5000
    cols = G.gen_table1(seed=2, nrows=n)
    with _ctx() as ctx:
        G.stats_accumulate(ctx, cols, n)
        good = G.stats_raw(ctx)
        bad = [c.clone() for c in cols]
        bad[1][77] = 300  # B is declared in [3, 8]: its one-byte field cannot carry 300
        G.stats_accumulate(ctx, bad, n)
        with pytest.raises(G.StatsError) as e:
            G.stats_sync(ctx)
        assert e.value.code == G.STATS_ERANGE
        G.stats_reset(ctx)
        G.stats_accumulate(ctx, cols, n)
        again = G.stats_raw(ctx)
    assert again.S_exact == good.S_exact


def _l16_host_columns(seed, n):
    """Table 1 rows from the oracle's generator, typed as the L16 layout (int16 / int32 / int64 / f64)."""
    iv, rv = O.table1_rows(seed, 0, n)
    out = []
    for j, dt in enumerate(G.table1_torch_dtypes(G.STATS_T1_L16)):
        src = rv[:, j] if j in REAL else iv[:, j]
        out.append(np.ascontiguousarray(src.astype(torch.empty(0, dtype=dt).numpy().dtype)))
    return out


@pytest.mark.parametrize("n", [9, 961, 100_003])
def test_exact_l16_int16_top_of_range(n):
    """L16 through the Table 1 converter: ragged sizes, and I (int16, declared [0, 65535]) at 32767,
    the largest value its dtype holds, against the oracle's exact sums of the same columns."""
    host = _l16_host_columns(13, n)
    host[9][n // 2] = 32767
    host[9][0] = 32000
    with _ctx(G.STATS_T1_L16) as ctx:
        G.stats_accumulate(ctx, [torch.from_numpy(c).cuda() for c in host], n)
        raw = G.stats_raw(ctx)
    _check_exact(raw, O.stats_columns(host))


def test_exact_l16_negative_int16_rejected():
    """A negative int16 in a column declared non-negative gives STATS_ERANGE (the sign-extended
    value spills past the two-byte field) and leaves the accumulator unchanged."""
    n = 4099
    host = _l16_host_columns(14, n)
    with _ctx(G.STATS_T1_L16) as ctx:
        G.stats_accumulate(ctx, [torch.from_numpy(c).cuda() for c in host], n)
        good = G.stats_raw(ctx)
        host[9][n - 3] = -1
        G.stats_accumulate(ctx, [torch.from_numpy(c).cuda() for c in host], n)
        with pytest.raises(G.StatsError) as e:
            G.stats_sync(ctx)
        assert e.value.code == G.STATS_ERANGE
        G.stats_reset(ctx)
        G.stats_accumulate(ctx, [torch.from_numpy(c).cuda() for c in _l16_host_columns(14, n)], n)
        again = G.stats_raw(ctx)
    assert again.S_exact == good.S_exact


# --------------------------------------------------------------------------- generic plan
def test_exact_generic_columns_signed_and_real():
    """A non-Table-1 configuration (signed int16/32/64, a real column) through the generic converter."""
    rng = np.random.default_rng(7)
    n = 70_001
    a = rng.integers(-30000, 30000, n, dtype=np.int16)
    b = rng.integers(-2**20, 2**20, n, dtype=np.int32)
    c = rng.integers(-2**30, 2**30, n, dtype=np.int64)
    d = (rng.standard_normal(n) * 3.0).astype(np.float64)
    cfg = G.Config([G.STATS_I16, G.STATS_I32, G.STATS_I64, G.STATS_F64], G.STATS_EXACT, [0, 0, 0, 0],
                   [-30000, -2**20, -2**30, -64.0], [30000, 2**20, 2**30, 64.0])
    dev = [torch.from_numpy(x).cuda() for x in (a, b, c, d)]
    with G.stats_init(cfg) as ctx:
        G.stats_accumulate(ctx, dev, n)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx)
    st = O.stats_columns([a.astype(np.int64), b.astype(np.int64), c, d])
    for j in range(4):
        for k in range(j, 4):
            if j == 3 or k == 3:
                ref = float(st.S[j][k])
                assert abs(raw.S[j, k] - ref) <= 1e-12 * abs(ref), (j, k)
            else:
                assert raw.S_exact[j][k] == st.S[j][k], (j, k)
    cov = O.cov_twopass_columns([a.astype(np.int64), b.astype(np.int64), c, d])
    assert np.abs(an.cov - cov).max() <= 1e-12 * np.abs(cov).max()


# --------------------------------------------------------------------------- finalize (a6)
def test_finalize_against_twopass_oracle():
    """mean / cov / corr / eigenpairs over the 11 analysis columns (identifier A excluded)."""
    n = 10**6
    cols = G.gen_table1(seed=0, nrows=n)
    with _ctx() as ctx:
        G.stats_accumulate(ctx, cols, n)
        an = G.stats_finalize(ctx, pca_on=0)
        anc = G.stats_finalize(ctx, pca_on=1)
    cov_full = O.cov_twopass_table1(0, n)
    keep = [j for j in range(12) if j != 0]
    cov = cov_full[np.ix_(keep, keep)]
    assert np.abs(an.cov - cov).max() <= 1e-12 * np.abs(cov).max()
    rel = np.abs(an.cov - cov) / np.abs(cov)
    assert rel.max() <= 1e-11
    corr = O.corr_from_cov(cov)
    assert np.abs(an.corr - corr).max() <= 1e-13
    assert np.allclose(np.diag(an.corr), 1.0, rtol=0, atol=0)
    st = O.stats_table1(0, n)
    assert np.allclose(an.mean, [float(st.s[j]) / n for j in keep], rtol=1e-15)
    for (res, M) in ((an, cov), (anc, corr)):
        ev, V = O.jacobi(M)
        assert np.abs(res.evals - ev).max() <= 1e-11 * np.abs(ev).max()
        assert abs(res.evals.sum() - np.trace(M)) <= 1e-11 * abs(np.trace(M))
        # eigenvectors: same sign convention; compare where eigenvalues are separated
        gaps = np.abs(np.diff(ev))
        for k in range(len(ev)):
            sep = min(gaps[k - 1] if k > 0 else np.inf, gaps[k] if k < len(gaps) else np.inf)
            if sep > 1e-6 * abs(ev).max():
                assert np.abs(res.evecs[k] - V[k]).max() <= 1e-8, k
        assert np.abs(res.evecs @ res.evecs.T - np.eye(11)).max() <= 1e-12


def test_finalize_zero_variance_and_small_n():
    """A constant column gives NaN correlations; n < 2 has no covariance (STATS_EINVAL)."""
    n = 1000
    a = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    b = torch.arange(n, dtype=torch.int32, device="cuda")
    cfg = G.Config([G.STATS_I32, G.STATS_I32], G.STATS_EXACT, [0, 0], [0, 0], [255, 65535])
    with G.stats_init(cfg) as ctx:
        G.stats_accumulate(ctx, [a, b], n)
        an = G.stats_finalize(ctx)
        assert an.cov[0, 0] == 0.0 and an.cov[0, 1] == 0.0
        assert math.isnan(an.corr[0, 1]) and an.corr[1, 1] == 1.0
        assert abs(an.cov[1, 1] - n * (n + 1) / 12.0) <= 1e-12 * an.cov[1, 1]
    with G.stats_init(cfg) as ctx:
        G.stats_accumulate(ctx, [a, b], 1)
        with pytest.raises(G.StatsError) as e:
            G.stats_finalize(ctx)
        assert e.value.code == G.STATS_EINVAL


# --------------------------------------------------------------------------- FP64 comparator (a8)
@pytest.mark.parametrize("mode", [G.STATS_FP64, G.STATS_FP64_SHIFTED])
def test_fp64_modes_against_oracle(mode):
    """The FP64 CUDA-core kernels: raw sums within FP64 accumulation error of the exact oracle."""
    n = 200_003
    cols = G.gen_table1(seed=4, nrows=n)
    with _ctx(mode=mode) as ctx:
        G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx)
    st = O.stats_table1(4, n)
    assert raw.n == n
    S = st.S_float()
    assert np.abs(raw.S - S).max() <= 1e-12 * np.abs(S).max()
    for j in range(12):
        assert abs(raw.s[j] - float(st.s[j])) <= 1e-12 * abs(float(st.s[j]))
    cov = O.cov_twopass_table1(4, n)[1:, 1:]
    tol = 1e-9 if mode == G.STATS_FP64 else 1e-12
    assert np.abs(an.cov - cov).max() <= tol * np.abs(cov).max()


# --------------------------------------------------------------------------- full-size workloads
def test_exact_table1_1e9_against_histogram_oracle():
    """Table 1 at n = 1e9 (seed 1, 60 GB, the launch configuration the benchmark times):
    every entry against the exact 6000-cell histogram oracle."""
    n = 10**9
    free, _ = torch.cuda.mem_get_info()
    if free < 70e9:
        pytest.skip("needs ~64 GB of device memory")
    cols = G.gen_table1(seed=1, nrows=n)
    with _ctx(max_rows=n) as ctx:
        G.stats_accumulate(ctx, cols, n)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx)
    del cols
    torch.cuda.empty_cache()
    st = O.stats_table1_hist(1, n)
    _check_exact(raw, st)
    assert raw.s_exact[0] == n * (n + 1) // 2
    assert raw.S_exact[0][0] == n * (n + 1) * (2 * n + 1) // 6
    _, cov, corr = O.analysis_from_stats(st)
    assert np.abs(an.cov - cov).max() <= 1e-12 * np.abs(cov).max()
    assert np.abs(an.corr - corr).max() <= 1e-12


def test_exact_table1_1e10_chunked_closed_forms():
    """The paper-scale workload: n = 1e10 rows in 2^28-row device chunks into one accumulator (seed 2);
    identifier sums against the closed forms, every entry against the histogram oracle."""
    n = 10**10
    chunk = 2**28
    cols = G.alloc_table1(chunk)
    with _ctx(max_rows=n) as ctx:
        r0 = 0
        while r0 < n:
            m = min(chunk, n - r0)
            G.stats_gen_table1(2, r0, m, G.STATS_T1_L32, cols)
            G.stats_accumulate(ctx, cols, m)
            r0 += m
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx)
    del cols
    torch.cuda.empty_cache()
    assert raw.s_exact[0] == 50000000005000000000
    assert raw.S_exact[0][0] == 333333333383333333335000000000
    st = O.stats_table1_hist(2, n)
    _check_exact(raw, st)
    _, cov, _ = O.analysis_from_stats(st)
    assert np.abs(an.cov - cov).max() <= 1e-12 * np.abs(cov).max()
    assert np.all(np.diff(an.evals) <= 0)
