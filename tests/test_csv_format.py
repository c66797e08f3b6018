"""CSV text written by the library (include/stats_csv.h), checked on the host without a GPU:
the line format, round-trip precision of the printed reals, header and argument errors."""
import numpy as np
import pytest

G = pytest.importorskip("paper_2604_23826_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2604_23826_gb300 import build
    build.build()
    G.load()


def _cols(n, seed=1):
    rng = np.random.default_rng(seed)
    return [rng.integers(-32768, 32768, n).astype(np.int16), rng.integers(-2**31, 2**31, n).astype(np.int32),
            rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64), (rng.standard_normal(n) * 1e3).astype(np.float32),
            rng.standard_normal(n) * 10.0 ** rng.integers(-30, 30, n)]


DT = [G.STATS_I16, G.STATS_I32, G.STATS_I64, G.STATS_F32, G.STATS_F64]


@pytest.mark.parametrize("n", [0, 1, 7, 50_000])
def test_lines_match_an_independent_formatter(tmp_path, n):
    """Every line equals the fields formatted here by Python (integers in decimal, FP32 with 9 and
    FP64 with 17 significant digits), and the printed reals read back to the same values."""
    cols = _cols(n, seed=n)
    path = tmp_path / "t.csv"
    G.stats_csv_write(path, DT, n, cols, header="a,b,c,d,e")
    lines = path.read_text().split("\n")
    assert lines[0] == "a,b,c,d,e" and lines[-1] == "" and len(lines) == n + 2
    for i in range(n):
        want = ",".join([str(int(cols[0][i])), str(int(cols[1][i])), str(int(cols[2][i])),
                         "%.9g" % float(cols[3][i]), "%.17g" % float(cols[4][i])])
        assert lines[i + 1] == want, i
        f = lines[i + 1].split(",")
        assert np.float32(float(f[3])) == cols[3][i] and float(f[4]) == cols[4][i]


def test_no_header_and_errors(tmp_path):
    path = tmp_path / "t.csv"
    a = np.array([1, 2], np.int32)
    G.stats_csv_write(path, [G.STATS_I32], 2, [a])
    assert path.read_text() == "1\n2\n"
    with pytest.raises(G.StatsError) as e:
        G.stats_csv_write(path, [G.STATS_F64], 2, [np.array([1.0, np.nan])])
    assert e.value.code == G.STATS_EINVAL
    with pytest.raises(G.StatsError) as e:
        G.stats_csv_write(path, [9], 2, [a])
    assert e.value.code == G.STATS_EINVAL
    with pytest.raises(G.StatsError) as e:
        G.stats_csv_write(tmp_path / "missing_dir" / "t.csv", [G.STATS_I32], 2, [a])
    assert e.value.code == G.STATS_EIO
