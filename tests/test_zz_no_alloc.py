"""The no-allocation entry point (stats_pass_noalloc) against the regular one.

Some callers cannot allocate device memory: a serving process or framework that reserves
the GPU's memory up front in its own pool and lets no library call cudaMalloc outside it,
or code that must not block the device (cudaFree synchronises it).  stats_pass_noalloc
serves them with its scratch in a fixed device array inside the library.  This file is
collected last so that a failure here does not stop the rest of a run that halts on the
first failure.

Each case makes two calls in a row on different rows (the shared scratch must not carry
the first call's sums) and compares each with stats_accumulate + stats_raw on the same
rows: integer-valued entries exactly, real-valued ones within 1e-12 relative.  The cases
cover both Table 1 converters (L32, L16), the generic converter with signed, unsigned and
real columns, columns that are not 16-byte aligned (plain loads instead of bulk copies),
ragged tails, and a value outside its declared range (status slot bit 1, as the regular
entry point's ERANGE).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")


def _regular(cfg, cols, n, allow_range=False):
    with G.stats_init(cfg) as ctx:
        G.stats_accumulate(ctx, cols, n)
        try:
            return G.stats_raw(ctx)
        except G.StatsError as e:
            if allow_range and e.code == G.STATS_ERANGE:
                return None
            raise


def _noalloc(cfg, cols, n):
    out = torch.zeros(G.noalloc_result_bytes(cfg.p), dtype=torch.uint8, device="cuda")
    G.stats_pass_noalloc(cfg, cols, n, out)
    torch.cuda.synchronize()
    return G.parse_noalloc_result(out.cpu().numpy().tobytes(), cfg.p)


def _same(a, b, real):
    assert a.n == b.n
    p = len(a.s)
    for j in range(p):
        for k in range(j, p):
            if j in real or k in real:
                assert abs(a.S[j, k] - b.S[j, k]) <= 1e-12 * abs(b.S[j, k]), (j, k)
            else:
                assert a.S_exact[j][k] == b.S_exact[j][k], (j, k)
        if j not in real:
            assert a.s_exact[j] == b.s_exact[j], j
        else:
            assert abs(a.s[j] - b.s[j]) <= 1e-12 * abs(b.s[j]), j


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
def test_noalloc_table1_two_calls_in_a_row(layout):
    cfg = G.stats_table1_config(layout, 10**10)
    n1, n2 = 300_007, 123_451
    a = G.gen_table1(seed=0, nrows=n1, layout=layout)
    b = G.gen_table1(seed=5, nrows=n2, layout=layout, row0=10**9)
    first = _noalloc(cfg, a, n1)
    second = _noalloc(cfg, b, n2)
    assert first.status == G.STATS_OK and second.status == G.STATS_OK
    _same(first, _regular(cfg, a, n1), (8, 10))
    _same(second, _regular(cfg, b, n2), (8, 10))
    assert first.s_exact[0] == n1 * (n1 + 1) // 2
    lo, hi = 10**9, 10**9 + n2
    assert second.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2


def _generic_cfg():
    # unsigned int32, signed int32, float64 (signed range), signed int16, signed int64, float32:
    # 1 + 3 + 3 + 7 + 2 + 6 + 7 = 29 digits
    dt = [G.STATS_I32, G.STATS_I32, G.STATS_F64, G.STATS_I16, G.STATS_I64, G.STATS_F32]
    lo = [0, -70_000, -1e3, -300, -2.0**40, 0]
    hi = [1_000_000, 70_000, 1e3, 300, 2.0**40, 64]
    return G.Config(dt, G.STATS_EXACT, None, lo, hi)


def _generic_cols(seed, n, offset=0, bad=False):
    """Device columns of the generic configuration, each starting `offset` elements into its
    allocation (offset 1: not 16-byte aligned)."""
    rng = np.random.default_rng(seed)
    vals = [rng.integers(0, 1_000_001, n).astype(np.int32), rng.integers(-70_000, 70_001, n).astype(np.int32),
            rng.uniform(-1e3, 1e3, n), rng.integers(-300, 301, n).astype(np.int16),
            rng.integers(-2**40, 2**40 + 1, n, dtype=np.int64), rng.uniform(0, 64, n).astype(np.float32)]
    if bad:
        vals[1][n // 2] = 2**30  # outside the 3-byte field of [-70000, 70000]
    cols = []
    for v in vals:
        buf = torch.from_numpy(np.concatenate([np.zeros(offset, v.dtype), v])).cuda()
        cols.append(buf[offset:])
    return cols


@pytest.mark.parametrize("offset", [0, 1])
def test_noalloc_generic_config_two_calls_in_a_row(offset):
    cfg = _generic_cfg()
    n1, n2 = 200_003, 77_777  # ragged tails: neither a multiple of a stage nor of 8 rows
    a = _generic_cols(1, n1, offset)
    b = _generic_cols(2, n2, offset)
    if offset:
        assert all(c.data_ptr() % 16 != 0 for c in a)
    first = _noalloc(cfg, a, n1)
    second = _noalloc(cfg, b, n2)
    assert first.status == G.STATS_OK and second.status == G.STATS_OK
    _same(first, _regular(cfg, a, n1), (2, 5))
    _same(second, _regular(cfg, b, n2), (2, 5))


def test_noalloc_range_violation_sets_the_status_slot():
    cfg = _generic_cfg()
    n = 50_001
    bad = _generic_cols(3, n, bad=True)
    res = _noalloc(cfg, bad, n)
    assert res.status == G.STATS_ERANGE
    assert _regular(cfg, bad, n, allow_range=True) is None  # the regular entry point: ERANGE too
    # the next call on good rows starts from a cleared status word
    good = _generic_cols(4, n)
    res2 = _noalloc(cfg, good, n)
    assert res2.status == G.STATS_OK
    _same(res2, _regular(cfg, good, n), (2, 5))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    cfg = G.stats_table1_config(G.STATS_T1_L32, 10**10)
    out = torch.zeros(G.noalloc_result_bytes(12), dtype=torch.uint8, device="cuda")
    a = G.gen_table1(seed=0, nrows=16)
    with pytest.raises(G.StatsError) as e:
        G.stats_pass_noalloc(cfg, a, (1 << 46) + 1, out)
    assert e.value.code == G.STATS_EINVAL
    wide = G.Config([G.STATS_I64] * 5, G.STATS_EXACT)  # 1 + 5 * 8 digits > 32
    with pytest.raises(G.StatsError) as e:
        G.stats_pass_noalloc(wide, [a[0]] * 5, 16, out)
    assert e.value.code == G.STATS_EINVAL
