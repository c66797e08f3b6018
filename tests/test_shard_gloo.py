"""The multi-rank path on CPU: two gloo ranks shard Table 1 by global row index,
each reduces its block (here with the CPU oracle standing in for a GPU context),
the partials are gathered and combined in rank order, and the result equals
the statistics of the whole table.  No GPU is used."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2604_23826_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _exact_tuple(st):
    return (st.n, tuple(st.s), tuple(tuple(r) for r in st.S))


def _worker(rank, world, port, mode, total, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if mode == "weak":
            r0, n = shard.weak_range(total, rank)
        else:
            r0, n = shard.strong_range(total, world, rank)
        st = O.stats_table1(17, n, row0=r0, threads=1)
        part = {"rank": rank, "row0": r0, "n": st.n, "s": st.s, "S": st.S}
        parts = shard.gather_in_rank_order(part)
        order = [p["rank"] for p in parts]

        def load(p):
            return {"n": p["n"], "s": list(p["s"]), "S": [list(r) for r in p["S"]], "ranges": [(p["row0"], p["n"])]}

        def merge(acc, other):
            acc["n"] += other["n"]
            acc["s"] = [a + b for a, b in zip(acc["s"], other["s"])]
            acc["S"] = [[a + b for a, b in zip(ra, rb)] for ra, rb in zip(acc["S"], other["S"])]
            acc["ranges"] += other["ranges"]

        merged = shard.combine_in_rank_order(parts, load, merge)
        if rank == 0:
            out_q.put((order, merged["n"], merged["ranges"], merged["s"][0], merged["S"][0][0],
                       [[merged["S"][j][k] for k in range(12)] for j in range(12)]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_rank_shard_and_rank_ordered_merge(mode):
    world = 2
    total = 20_001 if mode == "strong" else 10_000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, total, q)) for r in range(world)]
    for p in procs:
        p.start()
    order, n, ranges, sA, sAA, S = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert order == [0, 1]
    n_all = total * world if mode == "weak" else total
    assert n == n_all
    # disjoint, contiguous cover of [0, n_all)
    assert ranges[0][0] == 0 and ranges[0][0] + ranges[0][1] == ranges[1][0] and sum(r[1] for r in ranges) == n_all
    assert sA == n_all * (n_all + 1) // 2 and sAA == n_all * (n_all + 1) * (2 * n_all + 1) // 6
    ref = O.stats_table1(17, n_all)
    for j in range(12):
        for k in range(12):
            if j in O.T1_REAL or k in O.T1_REAL:
                assert abs(float(S[j][k] - ref.S[j][k])) <= 1e-25 * abs(float(ref.S[j][k]))
            else:
                assert S[j][k] == ref.S[j][k]


def test_ranges_partition():
    for total in (0, 1, 7, 1000, 10**10 + 3):
        for world in (1, 2, 3, 8):
            rs = [shard.strong_range(total, world, r) for r in range(world)]
            assert rs[0][0] == 0 and sum(n for _, n in rs) == total
            for (a0, an), (b0, _) in zip(rs[:-1], rs[1:]):
                assert a0 + an == b0
    assert shard.weak_range(5, 3) == (15, 5)
    with pytest.raises(ValueError):
        shard.strong_range(10, 0, 0)


def _worker_leaves(rank, world, port, out_q):
    """Rank 1 fails between steps (an exception before the gather, nothing in flight); rank 0
    must learn of it from its next collective, which ends with an error instead of hanging."""
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    r0, n = shard.strong_range(2_000, world, rank)
    st = O.stats_table1(17, n, row0=r0, threads=1)
    if rank == 1:
        raise SystemExit(3)  # the failing rank leaves without joining the gather
    t0 = __import__("time").monotonic()
    try:
        shard.gather_in_rank_order({"n": st.n})
        out_q.put(("no error", 0.0))
    except Exception as e:  # noqa: BLE001 - the collective's own error type varies by transport
        out_q.put((type(e).__name__, __import__("time").monotonic() - t0))


def test_rank_that_leaves_is_detected_by_the_next_collective():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_leaves, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    kind, secs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert kind != "no error"
    assert secs < 60
    assert procs[1].exitcode == 3
