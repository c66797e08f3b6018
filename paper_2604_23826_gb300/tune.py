"""Autotuner of the batched pass: how stats_accumulate_batched deals the stages of its
FP32 split-mode tables to the persistent CTAs of a launch.

The batched launches group tables by width class (1-8, 9-16, 17-32 and 33-64 columns) and
mode (BF16x3, BF16x4).  Two settings per group decide the launch's load balance against its
per-CTA partial sums: the units per CTA of the persistent tcgen05 launch (33-64 columns in
[p, ld] blocks) and the chunking of the register-fragment launch (chunks per CTA, smallest
chunk).  For every group present in a sample batch the tuner times that group's tables
alone through stats_accumulate_batched under each candidate setting -- CUDA events on the
call's stream, best of `reps`, on scratch contexts with the tables' own configurations --
and keeps the fastest (the library defaults are among the candidates, so the choice is
never slower on the sample).  Choices are cached in a JSON file keyed by the device (name,
SM count), the library build (hash of libsuffstats.so) and a workload tag, and applied
with stats_set_batch_tuning.

The setting regroups rows into partial sums, so results move within rounding only; every
setting keeps the stated tolerance.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional, Sequence

from . import binding as G

NARROW_UNITS = (4, 6, 8, 12, 16, 24, 32, 48, 64, 96)
GRAM32_CHUNKING = ((32, 32), (8, 32), (16, 32), (64, 32), (32, 8), (32, 128), (16, 128), (64, 8))
DEFAULT = {"narrow_units_per_cta": 12, "gram32_chunks_per_cta": 32, "gram32_min_chunk": 32}


def width_class(p: int) -> int:
    return 8 if p <= 8 else 16 if p <= 16 else 32 if p <= 32 else 64


def default_cache_path() -> str:
    return os.environ.get("STATS_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2604_23826_gb300", "batch_tuning.json"))


def library_hash() -> str:
    h = hashlib.sha256()
    with open(G.lib_path(), "rb") as f:
        for block in iter(lambda: f.read(1 << 20), b""):
            h.update(block)
    return h.hexdigest()[:16]


def device_key(workload: str = "default") -> str:
    import torch
    d = torch.cuda.current_device()
    prop = torch.cuda.get_device_properties(d)
    return f"{prop.name}|sm{prop.multi_processor_count}|lib{library_hash()}|{workload}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cache_get(key: str, path: Optional[str] = None) -> Optional[dict]:
    return _load(path or default_cache_path()).get(key)


def cache_put(key: str, value: dict, path: Optional[str] = None) -> None:
    path = path or default_cache_path()
    data = _load(path)
    data[key] = value
    _save(path, data)


def apply(choice: Dict[str, dict]) -> None:
    """Set the library's tuning from a {"w<P>_<mode>": setting} mapping."""
    for name, t in choice.items():
        w, mode = name.split("_")
        G.stats_set_batch_tuning(int(w[1:]), int(mode), t)


def apply_cached(workload: str = "default", path: Optional[str] = None) -> Optional[dict]:
    """Apply a cached choice for this device and library build, if there is one."""
    entry = cache_get(device_key(workload), path)
    if entry:
        apply(entry["choice"])
    return entry


def _time_group(ctxs, cols, rows, stream, reps: int) -> float:
    import torch
    batch = G.BatchArgs(ctxs, cols, rows)
    best = float("inf")
    for _ in range(reps + 1):  # the first call warms up (pivots, workspaces)
        for c in ctxs:
            G.stats_reset(c)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.stats_accumulate_batched(batch, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune_batched(ctxs: Sequence, dcols: Sequence[Sequence], nrows: Sequence[int], stream=None, reps: int = 3,
                     workload: str = "default", path: Optional[str] = None, force: bool = False) -> dict:
    """Tune every (width class, mode) group of a sample batch, apply the result and cache it.

    ctxs / dcols / nrows describe the sample as for stats_accumulate_batched; only their
    configurations, columns and row counts are used (the contexts are not modified).
    Groups already in the cache for this device, library build and workload are applied
    without measuring (force=True measures them again).  Returns {"choice": {...},
    "measured": {...}} where measured holds, per group, the default's and the choice's time
    in ms."""
    import torch
    key = device_key(workload)
    cached = (None if force else cache_get(key, path)) or {"choice": {}, "measured": {}}
    stream = stream or torch.cuda.current_stream()
    groups: Dict[str, List[int]] = {}
    for t, c in enumerate(ctxs):
        if c.mode in (G.STATS_BF16X3, G.STATS_BF16X4) and c.p <= 64 and nrows[t] > 0:
            groups.setdefault(f"w{width_class(c.p)}_{c.mode}", []).append(t)
    choice, measured = dict(cached["choice"]), dict(cached["measured"])
    todo = {name: idx for name, idx in groups.items() if name not in choice}
    apply({name: choice[name] for name in groups if name in choice})
    if not todo:
        return {"choice": choice, "measured": measured}
    for name, idx in sorted(todo.items()):
        mode = ctxs[idx[0]].mode
        scratch = [G.stats_init(G.Config([G.STATS_F32] * ctxs[t].p, mode, [0] * ctxs[t].p)) for t in idx]
        cols = [dcols[t] for t in idx]
        rows = [nrows[t] for t in idx]
        try:
            best = dict(DEFAULT)
            apply({name: best})
            t_default = _time_group(scratch, cols, rows, stream, reps)
            t_best = t_default
            if name.startswith("w64"):
                for u in NARROW_UNITS:
                    cand = dict(best, narrow_units_per_cta=u)
                    apply({name: cand})
                    t = _time_group(scratch, cols, rows, stream, reps)
                    if t < t_best:
                        best, t_best = cand, t
            for cpc, mc in GRAM32_CHUNKING:
                cand = dict(best, gram32_chunks_per_cta=cpc, gram32_min_chunk=mc)
                apply({name: cand})
                t = _time_group(scratch, cols, rows, stream, reps)
                if t < t_best:
                    best, t_best = cand, t
        finally:
            for c in scratch:
                c.close()
        apply({name: best})
        choice[name] = best
        measured[name] = {"tables": len(idx), "default_ms": t_default, "chosen_ms": t_best}
    entry = {"choice": choice, "measured": measured}
    cache_put(key, entry, path)
    return entry
