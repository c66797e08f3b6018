"""The batched-launch autotuner's host side (no GPU): the C-ABI tuning table and the cache."""
import json

import pytest

import paper_2604_23826_gb300 as G
from paper_2604_23826_gb300 import tune


def test_tuning_table_roundtrip_and_validation():
    before = G.stats_get_batch_tuning(40, G.STATS_BF16X4)
    try:
        G.stats_set_batch_tuning(40, G.STATS_BF16X4, {"narrow_units_per_cta": 24, "gram32_chunks_per_cta": 16,
                                                       "gram32_min_chunk": 128})
        # one width class: every width of 33..64 columns shares the setting
        assert G.stats_get_batch_tuning(64, G.STATS_BF16X4) == {"narrow_units_per_cta": 24,
                                                                 "gram32_chunks_per_cta": 16,
                                                                 "gram32_min_chunk": 128}
        assert G.stats_get_batch_tuning(64, G.STATS_BF16X3) == tune.DEFAULT  # the other mode untouched
        assert G.stats_get_batch_tuning(32, G.STATS_BF16X4) == tune.DEFAULT  # the other classes too
        for bad in ({"narrow_units_per_cta": 0, "gram32_chunks_per_cta": 16, "gram32_min_chunk": 1},
                    {"narrow_units_per_cta": 1, "gram32_chunks_per_cta": 2000, "gram32_min_chunk": 1},
                    {"narrow_units_per_cta": 1, "gram32_chunks_per_cta": 1, "gram32_min_chunk": 0}):
            with pytest.raises(G.StatsError):
                G.stats_set_batch_tuning(40, G.STATS_BF16X4, bad)
        for width, mode in ((0, G.STATS_BF16X4), (65, G.STATS_BF16X4), (8, G.STATS_EXACT)):
            with pytest.raises(G.StatsError):
                G.stats_set_batch_tuning(width, mode, tune.DEFAULT)
    finally:
        G.stats_set_batch_tuning(40, G.STATS_BF16X4, before)


def test_width_classes():
    assert [tune.width_class(p) for p in (1, 8, 9, 16, 17, 32, 33, 64)] == [8, 8, 16, 16, 32, 32, 64, 64]


def test_cache_roundtrip_and_apply(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert tune.cache_get("k", path) is None
    entry = {"choice": {f"w16_{G.STATS_BF16X3}": {"narrow_units_per_cta": 12, "gram32_chunks_per_cta": 64,
                                                  "gram32_min_chunk": 8}},
             "measured": {}}
    tune.cache_put("k", entry, path)
    tune.cache_put("other", {"choice": {}, "measured": {}}, path)
    assert tune.cache_get("k", path) == entry
    assert set(json.load(open(path))) == {"k", "other"}
    try:
        tune.apply(entry["choice"])
        assert G.stats_get_batch_tuning(16, G.STATS_BF16X3)["gram32_chunks_per_cta"] == 64
    finally:
        G.stats_set_batch_tuning(16, G.STATS_BF16X3, tune.DEFAULT)
    assert len(tune.library_hash()) == 16
