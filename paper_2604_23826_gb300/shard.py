"""Row sharding of the pass across ranks and the rank-ordered combination of
their partial statistics.

The paper runs its pass data-parallel: each GPU takes a disjoint subset of the
rows and the partial sums are combined on the host (arxiv 2604.23826,
"Validation and Infrastructure Testing" and "Data Representation and
Sufficient Statistics").  Here each rank owns a contiguous block of global row
indices (the generator is counter-based on the global row index, so a rank
generates or reads exactly its block), accumulates it into its own context,
and the exported accumulators are combined in rank order with stats_merge.
The exchange is one small gather (a few KB per rank) after the pass; the pass
itself has no collective.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple


def weak_range(rows_per_rank: int, rank: int) -> Tuple[int, int]:
    """(first global row, row count) of `rank` when every rank holds rows_per_rank rows."""
    if rows_per_rank < 0 or rank < 0:
        raise ValueError("negative size or rank")
    return rank * rows_per_rank, rows_per_rank


def strong_range(total_rows: int, world: int, rank: int) -> Tuple[int, int]:
    """(first global row, row count) of `rank` in a near-equal contiguous split of total_rows."""
    if world < 1 or not 0 <= rank < world or total_rows < 0:
        raise ValueError("bad world / rank / size")
    lo = total_rows * rank // world
    hi = total_rows * (rank + 1) // world
    return lo, hi - lo


def gather_in_rank_order(obj, group=None) -> List:
    """All-gather a picklable object; element r of the result is rank r's object."""
    import torch.distributed as dist
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def combine_in_rank_order(parts: Sequence, load: Callable, merge: Callable):
    """load(parts[0]), then merge(acc, load(part)) for ranks 1, 2, ... in order."""
    if not parts:
        raise ValueError("nothing to combine")
    acc = load(parts[0])
    for part in parts[1:]:
        merge(acc, load(part))
    return acc


def combine_contexts(ctx, group=None):
    """The global statistics of every rank's context, on every rank.

    Each rank exports its accumulator (stats_export: a few KB, the single exchange of
    the data-parallel pass), the images are all-gathered in rank order, and each rank
    imports them and merges them with stats_merge in rank order, so every rank holds
    the same combination (bit-identical for STATS_EXACT; the shifted modes re-express
    each image about the first one's pivot in double-double).  Returns a new context
    owned by the caller."""
    from . import binding as G

    parts = gather_in_rank_order(G.stats_export(ctx), group)

    def merge(acc, other):
        G.stats_merge(acc, other)
        G.stats_sync(acc)
        other.close()

    return combine_in_rank_order(parts, lambda blob: G.stats_import(blob, ctx.p, ctx.mode), merge)
