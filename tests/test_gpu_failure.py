"""Failure detection without a device fault.

Device: the grid-wide waits of the eigen-solver are bounded.  A test-only knob shortens the
limit and keeps one block from arriving at the first barrier (a generation word that nothing
advances), so every other block's wait runs out; the call must return STATS_ETIMEOUT and the
context must stay usable: the next finalize gives the same bits as a context that never saw
the timeout.

Host: the paper checks that every record was processed exactly once by the identifier
column's closed forms ("Validation and Infrastructure Testing").  A host-streamed Table 1
pass with one chunk dropped, repeated or displaced must fail at least one of n, sum A and
sum A^2, while the intact stream passes all three.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")


def _table(seed, n, p):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1e3, 1e3, p) + rng.uniform(0.5, 5.0, p) * rng.standard_normal((n, p))
    return X


@pytest.mark.parametrize("p,absent", [(32, 0), (64, 3), (200, 1)])
def test_grid_wait_runs_out_and_ctx_stays_usable(p, absent):
    n = 20_000
    X = _table(70 + p, n, p)
    cols = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
    cfg = G.Config([G.STATS_F64] * p, G.STATS_FP64_SHIFTED, [0] * p)
    with G.stats_init(cfg) as ctx, G.stats_init(cfg) as clean:
        for c in (ctx, clean):
            G.stats_accumulate(c, cols, n)
        ref = G.stats_finalize(clean)
        G.stats_set_grid_wait(ctx, 50_000_000, absent)  # 50 ms per wait, block `absent` never arrives
        with pytest.raises(G.StatsError) as e:
            G.stats_finalize(ctx)
        assert e.value.code == G.STATS_ETIMEOUT
        with pytest.raises(G.StatsError) as e:  # the seeded path waits at the same barriers
            G.stats_finalize_warm(ctx, 0, ref.evecs)
        assert e.value.code == G.STATS_ETIMEOUT
        G.stats_set_grid_wait(ctx, 0, -1)
        an = G.stats_finalize(ctx)
        for f in ("mean", "cov", "corr", "evals", "evecs"):
            assert np.array_equal(getattr(an, f), getattr(ref, f)), f
        cov = O.cov_twopass_columns([X[:, j] for j in range(p)])
        assert np.linalg.norm(an.cov - cov) <= 1e-12 * np.linalg.norm(cov)
        # a block index past the grid changes nothing
        G.stats_set_grid_wait(ctx, 50_000_000, 100_000)
        assert np.array_equal(G.stats_finalize(ctx).evals, ref.evals)


def test_grid_wait_knob_rejects_bad_values():
    with G.stats_init(G.Config([G.STATS_F64] * 4, G.STATS_FP64, [0] * 4)) as ctx:
        for wait, absent in ((-1, -1), (61 * 10**9, -1), (0, -2)):
            with pytest.raises(G.StatsError) as e:
                G.stats_set_grid_wait(ctx, wait, absent)
            assert e.value.code == G.STATS_EINVAL


def _host_stream(host, chunks, n_cfg):
    """Stream the given (row0, rows) ranges of the pinned host columns into one exact context."""
    with G.stats_init(G.stats_table1_config(G.STATS_T1_L32, n_cfg)) as ctx:
        for r0, rows in chunks:
            G.stats_accumulate_host(ctx, [h[r0:r0 + rows] for h in host], rows, 1 << 16)
        return G.stats_raw(ctx)


def test_dropped_repeated_or_displaced_chunk_fails_closed_forms():
    n, k = 1_000_000, 1 << 17
    dev = G.gen_table1(seed=31, nrows=n)
    host = [torch.empty(n, dtype=c.dtype, pin_memory=True) for c in dev]
    for h, c in zip(host, dev):
        h.copy_(c)
    chunks = [(r, min(k, n - r)) for r in range(0, n, k)]
    ok = G.identifier_checks(_host_stream(host, chunks, n), 1, n)
    assert all(ok.values()), ok
    dropped = G.identifier_checks(_host_stream(host, chunks[:3] + chunks[4:], n), 1, n)
    repeated = G.identifier_checks(_host_stream(host, chunks[:4] + chunks[3:], n), 1, n)
    # the same number of rows, but chunk 3 replaced by a copy of chunk 2: n passes, the sums do not
    displaced = G.identifier_checks(_host_stream(host, chunks[:3] + [chunks[2]] + chunks[4:], n), 1, n)
    print(f"\nintact {ok}\ndropped {dropped}\nrepeated {repeated}\ndisplaced {displaced}")
    for bad in (dropped, repeated):
        assert not bad["n"] and not bad["sum"] and not bad["sum_sq"]
    assert displaced["n"] and not displaced["sum"] and not displaced["sum_sq"]
    # the intact stream also equals the oracle's exact statistics
    raw = _host_stream(host, chunks, n)
    st = O.stats_table1(31, n)
    for j in range(12):
        if j not in O.T1_REAL:
            assert raw.s_exact[j] == st.s[j]
