"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
the headers under include/ declare.  Host-only entry points are exercised without a GPU;
no compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def _declared():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(stats_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_23826_gb300 import build
    build.build()
    import paper_2604_23826_gb300 as G
    return G.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("stats_init", "stats_accumulate", "stats_accumulate_host", "stats_merge", "stats_raw",
                 "stats_finalize", "stats_export", "stats_import", "stats_destroy", "stats_strerror",
                 "stats_gen_table1", "stats_table1_config", "stats_file_info", "stats_file_check_table1",
                 "stats_accumulate_file"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_sm103a_only():
    from paper_2604_23826_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_strerror_and_table1_config(lib):
    import paper_2604_23826_gb300 as G
    for code in range(8):
        assert isinstance(G.stats_strerror(code), str) and G.stats_strerror(code)
    cfg = G.stats_table1_config(G.STATS_T1_L32, 10**9)
    assert cfg.dtypes == [G.STATS_I64] + [G.STATS_I32] * 7 + [G.STATS_F64, G.STATS_I32, G.STATS_F64, G.STATS_I32]
    assert cfg.is_identifier == [1] + [0] * 11
    assert cfg.lo[1] == 3 and cfg.hi[1] == 8 and cfg.lo[3] == 1 and cfg.hi[3] == 100
    assert cfg.hi[0] == 10**9
    cfg16 = G.stats_table1_config(G.STATS_T1_L16, 10**9)
    assert cfg16.dtypes[5] == G.STATS_I32 and cfg16.dtypes[1] == G.STATS_I16
    assert G.stats_table1_row_bytes(G.STATS_T1_L32) == 60 and G.stats_table1_row_bytes(G.STATS_T1_L16) == 44
    assert G.stats_table1_row_bytes(9) == 0
    with pytest.raises(G.StatsError):
        G.stats_table1_config(5, 10)


def test_bad_arguments_rejected_without_device(lib):
    import paper_2604_23826_gb300 as G
    h = ctypes.c_void_p()
    assert lib.stats_init(ctypes.byref(h), None) == G.STATS_EINVAL
    bad = G.Config([G.STATS_I32] * 0)
    assert lib.stats_init(ctypes.byref(h), ctypes.byref(bad.c_struct())) == G.STATS_EINVAL
    assert lib.stats_set_grid(None, 4) == G.STATS_EINVAL
    assert lib.stats_sync(None) == G.STATS_EINVAL
    lib.stats_destroy(None)  # no-op
