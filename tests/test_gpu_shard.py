"""Row sharding through the library across processes: two gloo ranks, each with its own
context on the one GPU, accumulate disjoint row ranges (weak and strong splits), exchange
their stats_export images, and combine them with stats_import + stats_merge in rank order
(shard.combine_contexts).  Every rank's combined context must equal the oracle over the
whole table: bit-exact integer entries and 1e-12 on the real ones for STATS_EXACT, the
stated tolerances for the shifted modes.  The ranks' kernels never wait on one another;
only the host-side gather is collective."""
import os
import socket

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _f32_table(n, p):
    rng = np.random.default_rng(41)
    mu = rng.uniform(1e3, 1e5, p)
    sd = rng.uniform(0.1, 10.0, p)
    return (mu + sd * rng.standard_normal((n, p))).astype(np.float32)


def _worker(rank, world, port, split, kind, total, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2604_23826_gb300 as G
        from paper_2604_23826_gb300 import shard
        torch.cuda.set_device(0)
        r0, n = shard.weak_range(total, rank) if split == "weak" else shard.strong_range(total, world, rank)
        if kind == "exact":
            cfg = G.stats_table1_config(G.STATS_T1_L32, 10**10)
            cols = G.gen_table1(seed=23, nrows=n, row0=r0)
        else:
            mode, dt = {"bf16x4": (G.STATS_BF16X4, np.float32), "fp64s": (G.STATS_FP64_SHIFTED, np.float64)}[kind]
            p = 40
            X = _f32_table(total * (world if split == "weak" else 1), p).astype(dt)[r0:r0 + n]
            cfg = G.Config([G.STATS_F32 if dt == np.float32 else G.STATS_F64] * p, mode, [0] * p)
            cols = [torch.from_numpy(np.ascontiguousarray(X[:, j])).cuda() for j in range(p)]
        with G.stats_init(cfg) as ctx:
            G.stats_accumulate(ctx, cols, n)
            G.stats_sync(ctx)
            merged = shard.combine_contexts(ctx)
        raw = G.stats_raw(merged)
        an = G.stats_finalize(merged)
        merged.close()
        out_q.put((rank, raw.n, raw.s, raw.S, [str(v) for v in raw.s_exact],
                   [[str(v) for v in row] for row in raw.S_exact], an.cov))
    finally:
        dist.destroy_process_group()


def _run(split, kind, total, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, split, kind, total, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("split", ["weak", "strong"])
def test_two_ranks_exact_contexts_combined(split):
    total = 300_007
    res = _run(split, "exact", total)
    n_all = total * 2 if split == "weak" else total
    ref = O.stats_table1(23, n_all)
    for rank, n, s, S, s_ex, S_ex, cov in res:
        assert n == n_all
        assert int(s_ex[0]) == n_all * (n_all + 1) // 2
        for j in range(12):
            for k in range(j, 12):
                if j in O.T1_REAL or k in O.T1_REAL:
                    r = float(ref.S[j][k])
                    assert abs(S[j, k] - r) <= 1e-12 * abs(r), (rank, j, k)
                else:
                    assert int(S_ex[j][k]) == ref.S[j][k], (rank, j, k)
    # every rank holds the same combination, bit for bit
    assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][6], res[1][6])


@pytest.mark.parametrize("kind,tol", [("bf16x4", 2e-6), ("fp64s", 1e-12)])
def test_two_ranks_shifted_contexts_combined(kind, tol):
    total = 120_011
    res = _run("strong", kind, total)
    X = _f32_table(total, 40).astype(np.float64 if kind == "fp64s" else np.float32)
    cov = O.cov_twopass_columns([X[:, j].astype(np.float64) for j in range(40)])
    for rank, n, s, S, s_ex, S_ex, c in res:
        assert n == total
        err = float(np.linalg.norm(c - cov) / np.linalg.norm(cov))
        print(f"\n{kind} rank {rank}: combined cov rel-Frobenius error {err:.3e}")
        assert err < tol
    assert np.array_equal(res[0][6], res[1][6])
