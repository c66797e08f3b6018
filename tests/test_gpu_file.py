"""Table files on the GPU: the Table 1 writer, the paper's sampled-row conversion check, and the
streaming pass from file against the device pass and the CPU oracle."""
import os
import struct

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")


def _ctx(layout=G.STATS_T1_L32, max_rows=10**10):
    return G.stats_init(G.stats_table1_config(layout, max_rows, G.STATS_EXACT))


def _col_offset(path, j):
    with open(path, "rb") as f:
        return struct.unpack_from("<Q", f.read(4096), 1056 + 8 * j)[0]


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
def test_write_check_and_read_back(tmp_path, layout):
    """Written rows equal the generator's; the beginning / middle / end check passes."""
    n = 100_003
    path = tmp_path / "t1.sscol"
    G.stats_file_write_table1(path, seed=7, nrows=n, layout=layout, chunk_rows=30_000)
    p, nrows, dts = G.stats_file_info(path)
    assert (p, nrows) == (12, n) and dts == G.stats_table1_config(layout, 1).dtypes
    assert G.stats_file_check_table1(path, 7, layout, rows_per_region=1000) == -1
    iv, rv = O.table1_rows(7, 40_000, 64)
    cols = G.stats_file_read_rows(path, 40_000, 64)
    for j in range(12):
        ref = rv[:, j] if j in O.T1_REAL else iv[:, j]
        assert np.array_equal(cols[j].astype(ref.dtype), ref), O.T1_NAMES[j]


def test_check_finds_an_altered_row(tmp_path):
    """One value changed in the middle region: STATS_EMISMATCH at that file row; a wrong seed
    fails at row 0; a row outside the sampled regions goes unseen (the check samples)."""
    n, k = 50_000, 512
    path = tmp_path / "t1.sscol"
    G.stats_file_write_table1(path, seed=11, nrows=n, layout=G.STATS_T1_L32)
    with pytest.raises(G.StatsError) as e:
        G.stats_file_check_table1(path, 12, G.STATS_T1_L32, rows_per_region=k)
    assert e.value.code == G.STATS_EMISMATCH and e.value.bad_row == 0
    bad = n // 2 + 3
    off = _col_offset(path, 5) + 4 * bad  # F, int32
    with open(path, "r+b") as f:
        f.seek(off)
        v = struct.unpack("<i", f.read(4))[0]
        f.seek(off)
        f.write(struct.pack("<i", v + 1))
    with pytest.raises(G.StatsError) as e:
        G.stats_file_check_table1(path, 11, G.STATS_T1_L32, rows_per_region=k)
    assert e.value.code == G.STATS_EMISMATCH and e.value.bad_row == bad
    with open(path, "r+b") as f:  # restore, then alter a row no region covers
        f.seek(off)
        f.write(struct.pack("<i", v))
        f.seek(_col_offset(path, 5) + 4 * (n // 4))
        f.write(struct.pack("<i", 123456))
    assert G.stats_file_check_table1(path, 11, G.STATS_T1_L32, rows_per_region=k) == -1


def test_check_rejects_a_wrong_layout(tmp_path):
    path = tmp_path / "t1.sscol"
    G.stats_file_write_table1(path, seed=1, nrows=1000, layout=G.STATS_T1_L16)
    with pytest.raises(G.StatsError) as e:
        G.stats_file_check_table1(path, 1, G.STATS_T1_L32)
    assert e.value.code == G.STATS_EFORMAT


@pytest.mark.parametrize("layout", [G.STATS_T1_L32, G.STATS_T1_L16])
def test_accumulate_file_matches_device_and_oracle(tmp_path, layout):
    """The pass from file (many small chunks, both pinned buffers in turn) equals the device pass
    bit for bit and the oracle; three row ranges in separate calls equal one call."""
    n = 100_003
    path = tmp_path / "t1.sscol"
    G.stats_file_write_table1(path, seed=5, nrows=n, layout=layout)
    with _ctx(layout) as c_file, _ctx(layout) as c_dev, _ctx(layout) as c_split:
        G.stats_accumulate_file(c_file, path, chunk_rows=4096)
        cols = G.gen_table1(seed=5, nrows=n, layout=layout)
        G.stats_accumulate(c_dev, cols, n)
        for r0, m in ((0, 33_337), (33_337, 8), (33_345, -1)):
            G.stats_accumulate_file(c_split, path, row0=r0, nrows=m, chunk_rows=10_000)
        a, b, c = G.stats_raw(c_file), G.stats_raw(c_dev), G.stats_raw(c_split)
    assert a.n == b.n == c.n == n
    assert a.S_exact == b.S_exact == c.S_exact and a.s_exact == b.s_exact == c.s_exact
    assert np.array_equal(a.S, b.S) and np.array_equal(a.S, c.S)
    st = O.stats_table1(5, n)
    for j in range(12):
        if j not in O.T1_REAL:
            assert a.s_exact[j] == st.s[j]


def test_accumulate_file_rejects_mismatched_columns(tmp_path):
    path = tmp_path / "t1.sscol"
    G.stats_file_write_table1(path, seed=1, nrows=1000, layout=G.STATS_T1_L16)
    with _ctx(G.STATS_T1_L32) as ctx:
        with pytest.raises(G.StatsError) as e:
            G.stats_accumulate_file(ctx, path)
        assert e.value.code == G.STATS_EINVAL
        with pytest.raises(G.StatsError) as e:
            G.stats_accumulate_file(ctx, tmp_path / "absent.sscol")
        assert e.value.code == G.STATS_EIO
