"""The no-allocation entry point (stats_pass_noalloc) against the regular one.

Some callers cannot allocate device memory (a stream being captured into a CUDA
graph in the global capture mode, or an application holding a fixed device
budget).  stats_pass_noalloc serves them with scratch in a device array inside
the library.  This file is collected last so that a failure here does not stop
the rest of a run that halts on the first failure.  Two calls in a row, on
different tables, must each match stats_accumulate + stats_raw exactly for the
integer-valued entries and within 1e-12 relative for the real-valued ones.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")

REAL = (8, 10)


def _regular(cols, n):
    with G.stats_init(G.stats_table1_config(G.STATS_T1_L32, 10**10)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        return G.stats_raw(ctx)


def _noalloc(cols, n):
    cfg = G.stats_table1_config(G.STATS_T1_L32, 10**10)
    out = torch.zeros(G.noalloc_result_bytes(12), dtype=torch.uint8, device="cuda")
    G.stats_pass_noalloc(cfg, cols, n, out)
    torch.cuda.synchronize()
    return G.parse_noalloc_result(out.cpu().numpy().tobytes(), 12)


def _same(a, b):
    assert a.n == b.n
    for j in range(12):
        for k in range(j, 12):
            if j in REAL or k in REAL:
                assert abs(a.S[j, k] - b.S[j, k]) <= 1e-12 * abs(b.S[j, k]), (j, k)
            else:
                assert a.S_exact[j][k] == b.S_exact[j][k], (j, k)
        if j not in REAL:
            assert a.s_exact[j] == b.s_exact[j], j
        else:
            assert abs(a.s[j] - b.s[j]) <= 1e-12 * abs(b.s[j]), j


def test_noalloc_two_calls_in_a_row_match_regular_entry_point():
    n1, n2 = 300_007, 123_451
    a = G.gen_table1(seed=0, nrows=n1)
    b = G.gen_table1(seed=5, nrows=n2, row0=10**9)
    first = _noalloc(a, n1)
    second = _noalloc(b, n2)  # the shared scratch must not carry the first call's sums
    assert first.status == G.STATS_OK and second.status == G.STATS_OK
    _same(first, _regular(a, n1))
    _same(second, _regular(b, n2))
    assert first.s_exact[0] == n1 * (n1 + 1) // 2
    lo, hi = 10**9, 10**9 + n2
    assert second.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2


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
