"""Columnar table files (include/stats_file.h) on the host: the on-disk layout, round trips,
and the validation that rejects truncated, extended or altered files.  No GPU is used."""
import os
import struct

import numpy as np
import pytest

G = pytest.importorskip("paper_2604_23826_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2604_23826_gb300 import build
    build.build()
    G.load()


def _columns(n, seed=3):
    rng = np.random.default_rng(seed)
    return [rng.integers(-30000, 30000, n, dtype=np.int16), rng.integers(-2**31, 2**31 - 1, n, dtype=np.int32),
            rng.integers(-2**62, 2**62, n, dtype=np.int64), rng.standard_normal(n).astype(np.float32),
            rng.standard_normal(n) * 1e6]


DTYPES = [G.STATS_I16, G.STATS_I32, G.STATS_I64, G.STATS_F32, G.STATS_F64]


def _fnv1a(b: bytes) -> int:
    h = 14695981039346656037
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _rehash(path):
    with open(path, "r+b") as f:
        hdr = bytearray(f.read(4096))
        hdr[3104:3112] = struct.pack("<Q", _fnv1a(bytes(hdr[:3104])))
        f.seek(0)
        f.write(hdr)


def _patch(path, off, data, rehash=True):
    with open(path, "r+b") as f:
        f.seek(off)
        f.write(data)
    if rehash:
        _rehash(path)


def test_layout_on_disk(tmp_path):
    """The header fields and column placement follow the documented format, parsed here
    independently of the library: magic, version, p, nrows, size, dtypes, 4096-aligned
    column offsets in order, FNV-1a of the first 3104 bytes, the column bytes themselves."""
    n = 1001
    cols = _columns(n)
    path = tmp_path / "t.sscol"
    G.stats_file_write(path, DTYPES, n, cols)
    raw = path.read_bytes()
    assert raw[:8] == b"SSCOL01\0"
    version, p, nrows, fbytes = struct.unpack_from("<IiqQ", raw, 8)
    assert (version, p, nrows, fbytes) == (1, 5, n, len(raw))
    dts = struct.unpack_from("<256i", raw, 32)
    offs = struct.unpack_from("<256Q", raw, 1056)
    assert list(dts[:5]) == DTYPES and not any(dts[5:]) and not any(offs[5:])
    assert struct.unpack_from("<Q", raw, 3104)[0] == _fnv1a(raw[:3104])
    end = 4096
    for j, c in enumerate(cols):
        assert offs[j] == (end + 4095) // 4096 * 4096
        assert raw[offs[j]:offs[j] + c.nbytes] == c.tobytes()
        end = offs[j] + c.nbytes
    assert end == len(raw)


@pytest.mark.parametrize("n", [0, 1, 7, 4096, 100_003])
def test_round_trip(tmp_path, n):
    cols = _columns(n, seed=n)
    path = tmp_path / "t.sscol"
    G.stats_file_write(path, DTYPES, n, cols)
    assert G.stats_file_info(path) == (5, n, DTYPES)
    back = G.stats_file_read_rows(path, 0, n)
    for a, b in zip(cols, back):
        assert np.array_equal(a, b)
    if n > 10:
        part = G.stats_file_read_rows(path, n // 3, n // 2)
        for a, b in zip(cols, part):
            assert np.array_equal(a[n // 3:n // 3 + n // 2], b)


def test_large_columns_span_io_pieces(tmp_path):
    """Columns longer than one parallel I/O piece (32 MB) read back whole and in a window that
    crosses a piece boundary."""
    n = 9_000_000  # int64: 72 MB
    a = np.arange(n, dtype=np.int64) * 3 - 7
    path = tmp_path / "big.sscol"
    G.stats_file_write(path, [G.STATS_I64], n, [a])
    (back,) = G.stats_file_read_rows(path, 0, n)
    assert np.array_equal(a, back)
    r0 = (32 << 20) // 8 - 5
    (win,) = G.stats_file_read_rows(path, r0, 11)
    assert np.array_equal(win, a[r0:r0 + 11])


def _expect(path, code):
    with pytest.raises(G.StatsError) as e:
        G.stats_file_info(path)
    assert e.value.code == code


@pytest.mark.parametrize("how", ["truncate", "extend", "flip_header", "magic", "version", "p_zero", "dtype",
                                 "offset_gap", "offset_overlap", "nrows", "stray_entry"])
def test_validation_rejects(tmp_path, how):
    n = 5000
    path = tmp_path / "t.sscol"
    G.stats_file_write(path, DTYPES, n, _columns(n))
    size = os.path.getsize(path)
    if how == "truncate":
        os.truncate(path, size - 1)
    elif how == "extend":
        with open(path, "ab") as f:
            f.write(b"\0")
    elif how == "flip_header":          # hash no longer matches
        _patch(path, 20, b"\x01", rehash=False)
    elif how == "magic":
        _patch(path, 0, b"SSCOL02\0")
    elif how == "version":
        _patch(path, 8, struct.pack("<I", 2))
    elif how == "p_zero":
        _patch(path, 12, struct.pack("<i", 0))
    elif how == "dtype":
        _patch(path, 32 + 4 * 2, struct.pack("<i", 9))
    elif how == "offset_gap":            # column 1 moved one alignment unit later
        off = struct.unpack_from("<Q", open(path, "rb").read(4096), 1056 + 8)[0]
        _patch(path, 1056 + 8, struct.pack("<Q", off + 4096))
    elif how == "offset_overlap":        # column 1 starts inside column 0
        _patch(path, 1056 + 8, struct.pack("<Q", 4096))
    elif how == "nrows":                 # one row more than the columns hold
        _patch(path, 16, struct.pack("<q", n + 1))
    elif how == "stray_entry":           # a dtype entry past p
        _patch(path, 32 + 4 * 10, struct.pack("<i", 1))
    _expect(path, G.STATS_EFORMAT)


def test_missing_file_and_bad_ranges(tmp_path):
    with pytest.raises(G.StatsError) as e:
        G.stats_file_info(tmp_path / "absent.sscol")
    assert e.value.code == G.STATS_EIO
    path = tmp_path / "t.sscol"
    n = 100
    G.stats_file_write(path, DTYPES, n, _columns(n))
    for r0, m in ((95, 6), (-1, 2), (101, 0)):
        with pytest.raises(G.StatsError) as e:
            G.stats_file_read_rows(path, r0, m)
        assert e.value.code == G.STATS_EINVAL
    with pytest.raises(G.StatsError) as e:
        G.stats_file_write(path, [G.STATS_I32, 42], n, _columns(n)[:2])
    assert e.value.code == G.STATS_EINVAL
