"""CSV text parsed on the GPU (include/stats_csv.h).

Reals: every accepted field must give the correctly rounded value of its decimal text,
checked against Python's float() (correctly rounded) for FP64 and against exact rational
rounding written here for FP32, on seeded random decimals in many spellings plus the
round-half-to-even boundaries.  Table 1 through a CSV file: the records and the exact
statistics equal the oracle's; the paper's first-column check (sum of the row index
1..n in closed form) on the first field alone.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")


def _dev_text(s: str):
    b = s.encode()
    t = torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda() if b else torch.empty(0, dtype=torch.uint8,
                                                                                      device="cuda")
    return t, len(b)


def _parse(text: str, dtypes, max_rows=None):
    t, nb = _dev_text(text)
    n_lines = text.count("\n") + (1 if text and not text.endswith("\n") else 0)
    cap = max(1, n_lines if max_rows is None else max_rows)
    tdt = {G.STATS_I16: torch.int16, G.STATS_I32: torch.int32, G.STATS_I64: torch.int64,
           G.STATS_F32: torch.float32, G.STATS_F64: torch.float64}
    cols = [torch.zeros(cap, dtype=tdt[d], device="cuda") for d in dtypes]
    n = G.stats_csv_parse(t, nb, dtypes, cols, cap)
    return n, [c[:n].cpu().numpy() for c in cols]


def _f32_bits(fr: Fraction) -> int:
    """Nearest float32 (ties to even) of a nonzero rational in the normal range, as bits."""
    neg = fr < 0
    a = -fr if neg else fr
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    scaled = a / Fraction(2) ** (e - 23)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    if m == 2 ** 24:
        m //= 2
        e += 1
    assert -126 <= e <= 127
    return (int(neg) << 31) | ((e + 127) << 23) | (m - 2 ** 23)


def _spellings(rng, M: int, E: int):
    """Decimal strings of M * 10^E in the grammar's forms (M > 0)."""
    D = str(M)
    nd = len(D)
    sign = rng.choice(["", "", "+", "-"])
    forms = []
    forms.append(f"{D}e{E}")
    i = int(rng.integers(0, nd + 1))
    ex = E + (nd - i)
    mant = (D[:i] or "") + "." + (D[i:] or "")
    if mant == ".":
        mant = "0."
    forms.append(mant + ("" if ex == 0 else f"E{'+' if ex > 0 and rng.integers(2) else ''}{ex}"))
    z = int(rng.integers(0, 4))
    forms.append("0." + "0" * z + D + f"e{E + nd + z}")
    if E >= -35:  # the point's zeros become significant digits: the exponent stays >= -38
        forms.append("00" + D + ".000" + f"e{E}")
    return [sign + f for f in forms], sign == "-"


def test_reals_round_correctly():
    rng = np.random.default_rng(2024)
    lines, want64, want32 = [], [], []
    while len(lines) < 40_000:
        nd = int(rng.integers(1, 20))
        M = int(rng.integers(10 ** (nd - 1), 10 ** nd, dtype=np.uint64)) if nd < 19 else \
            int(rng.integers(10 ** 18, 10 ** 19 - 1, dtype=np.uint64))
        E = int(rng.integers(-38, 20))
        v = Fraction(M) * Fraction(10) ** E
        if not (Fraction(2) ** -126 <= v < Fraction(2) ** 127):
            continue
        forms, neg = _spellings(rng, M, E)
        for f in forms:
            lines.append(f"{f},{f}")
            want64.append(float(f))
            want32.append(_f32_bits(-v if neg else v))
    n, (c64, c32) = _parse("\n".join(lines) + "\n", [G.STATS_F64, G.STATS_F32])
    assert n == len(lines)
    assert np.array_equal(c64.view(np.uint64), np.array(want64).view(np.uint64))
    assert np.array_equal(c32.view(np.uint32), np.array(want32, dtype=np.uint32))


def test_round_half_even_boundaries():
    """Exact ties and their neighbours at the 53- and 24-bit boundaries, zeros, signs."""
    cases = []
    for base in (2 ** 53, 2 ** 54 + 2 ** 10):
        for d in range(-3, 4):
            cases.append(str(base + d))
    for d in range(-3, 4):
        cases.append(str(2 ** 24 + d))
    # 2^-1074-free decimals just around a tie: (2^53 + 1) / 2^k written exactly with <= 19 digits
    for k in (1, 2, 3, 10):
        fr = Fraction(2 ** 53 + 1, 2 ** k)
        s = str(fr.numerator * 5 ** k)  # = fr * 10^k
        if len(s) <= 19:
            cases.append(f"{s}e-{k}")
    cases += ["0", "-0", "0.0", "-0.000e5", "1", "-1", "1.5", "9999999999999999999", "0.1", "1e-37", "1e19",
              "123456789012345678.9", "3402823466385288598e19", "2e-38",
              "2.000000000000000000e-38", "1e20", "0.000500e-33"]
    text = "\n".join(f"{c},{c}" for c in cases) + "\n"
    n, (c64, c32) = _parse(text, [G.STATS_F64, G.STATS_F32])
    assert n == len(cases)
    for i, c in enumerate(cases):
        assert c64[i].view(np.uint64) == np.float64(float(c)).view(np.uint64), c
        fr = Fraction(c)
        want = (0x80000000 if c.startswith("-") else 0) if fr == 0 else _f32_bits(fr)
        assert int(c32[i].view(np.uint32)) == want, c


def test_integers_bounds_and_fields_past_k():
    rows = [("32767", "2147483647", "9223372036854775807"), ("-32768", "-2147483648", "-9223372036854775808"),
            ("+7", "007", "-0"), ("0", "1", "12")]
    text = "".join(",".join(r) + ",ignored field,x\n" for r in rows)
    n, (a, b, c) = _parse(text, [G.STATS_I16, G.STATS_I32, G.STATS_I64])
    assert n == 4
    assert a.tolist() == [32767, -32768, 7, 0]
    assert b.tolist() == [2147483647, -2147483648, 7, 1]
    assert c.tolist() == [2 ** 63 - 1, -2 ** 63, 0, 12]


@pytest.mark.parametrize("bad,code", [
    ("1,x", G.STATS_EFORMAT), ("1", G.STATS_EFORMAT), ("", G.STATS_EFORMAT), ("1,", G.STATS_EFORMAT),
    ("1.5,2", G.STATS_EFORMAT), ("32768,1", G.STATS_ERANGE), ("-32769,1", G.STATS_ERANGE),
    ("1,1e-39", G.STATS_EFORMAT), ("1,1e40", G.STATS_EFORMAT), ("1,12345678901234567891", G.STATS_EFORMAT),
    ("1,1e-38", G.STATS_ERANGE), ("1,1.2.3", G.STATS_EFORMAT), ("1,1e", G.STATS_EFORMAT),
    ("1,1e12345", G.STATS_EFORMAT), ("1,.", G.STATS_EFORMAT), ("1,--1", G.STATS_EFORMAT),
    ("12345678901234567890,1", G.STATS_EFORMAT)])
def test_errors_name_the_first_bad_line(bad, code):
    good = "5,0.25\n"
    text = good * 7 + bad + "\n" + good * 3 + "1,x\n"
    with pytest.raises(G.StatsError) as e:
        _parse(text, [G.STATS_I16, G.STATS_F32])
    assert e.value.code == code and e.value.bad_line == 7


def test_crlf_no_final_newline_and_too_many_lines():
    n, (a, b) = _parse("1,2.5\r\n3,-4\r\n5,6e1", [G.STATS_I32, G.STATS_F64])
    assert n == 3 and a.tolist() == [1, 3, 5] and b.tolist() == [2.5, -4.0, 60.0]
    with pytest.raises(G.StatsError) as e:
        _parse("1\n2\n3\n", [G.STATS_I32], max_rows=2)
    assert e.value.code == G.STATS_EINVAL
    assert _parse("", [G.STATS_I32])[0] == 0


@pytest.mark.parametrize("layout,chunk", [(G.STATS_T1_L32, 100_000), (G.STATS_T1_L16, 0), (G.STATS_T1_L32, 4099)])
def test_table1_csv_stream_matches_oracle(tmp_path, layout, chunk):
    """Table 1 written as CSV and streamed back (chunks that cut lines) gives the same records as
    the generator and exactly the oracle's statistics."""
    n = 60_001
    path = tmp_path / "t1.csv"
    G.stats_csv_write_table1(path, seed=3, nrows=n, layout=layout, chunk_rows=25_000)
    cfg = G.stats_table1_config(layout, 10 ** 6, G.STATS_EXACT)
    with G.stats_init(cfg) as c_csv, G.stats_init(cfg) as c_dev:
        assert G.stats_accumulate_csv(c_csv, path, skip_lines=1, chunk_bytes=chunk) == n
        G.stats_accumulate(c_dev, G.gen_table1(seed=3, nrows=n, layout=layout), n)
        a, b = G.stats_raw(c_csv), G.stats_raw(c_dev)
    assert a.n == b.n == n
    assert a.S_exact == b.S_exact and a.s_exact == b.s_exact and np.array_equal(a.S, b.S)
    st = O.stats_table1(3, n)
    for j in range(12):
        if j not in O.T1_REAL:
            assert a.s_exact[j] == st.s[j]
    # the parsed records themselves, against the oracle's rows
    text = path.read_text().split("\n", 1)[1]
    k = 12
    t, nb = _dev_text(text)
    tdt = {G.STATS_I16: torch.int16, G.STATS_I32: torch.int32, G.STATS_I64: torch.int64, G.STATS_F64: torch.float64}
    cols = [torch.empty(n, dtype=tdt[d], device="cuda") for d in cfg.dtypes]
    assert G.stats_csv_parse(t, nb, cfg.dtypes[:k], cols, n) == n
    iv, rv = O.table1_rows(3, 0, n)
    for j in range(12):
        ref = rv[:, j] if j in O.T1_REAL else iv[:, j]
        assert np.array_equal(cols[j].cpu().numpy().astype(ref.dtype), ref), O.T1_NAMES[j]


def test_first_column_closed_form(tmp_path):
    """The paper's first validation step: only the first field (the row index A = 1..n) is parsed
    from each line; its sum and sum of squares equal n(n+1)/2 and n(n+1)(2n+1)/6."""
    n = 250_003
    path = tmp_path / "t1.csv"
    G.stats_csv_write_table1(path, seed=1, nrows=n)
    with G.stats_init(G.Config([G.STATS_I64], G.STATS_EXACT, [0], [1], [n])) as ctx:
        assert G.stats_accumulate_csv(ctx, path, skip_lines=1, chunk_bytes=1 << 20) == n
        raw = G.stats_raw(ctx)
    assert raw.n == n and raw.s_exact[0] == n * (n + 1) // 2
    assert raw.S_exact[0][0] == n * (n + 1) * (2 * n + 1) // 6


def test_stream_errors(tmp_path):
    """A bad field reports its file line (header counted) and leaves the chunks before it added;
    a line longer than a chunk is EFORMAT."""
    path = tmp_path / "t.csv"
    good = "".join(f"{i},{i}.5\n" for i in range(1000))
    path.write_text("a,b\n" + good + "7,oops\n" + good)
    with G.stats_init(G.Config([G.STATS_I32, G.STATS_F64], G.STATS_FP64, [0, 0])) as ctx:
        with pytest.raises(G.StatsError) as e:
            G.stats_accumulate_csv(ctx, path, skip_lines=1, chunk_bytes=4096)
        assert e.value.code == G.STATS_EFORMAT and e.value.bad_line == 1001
        assert 0 < e.value.rows_added <= 1000
    path.write_text("1," + "1" * 200 + "\n")
    with G.stats_init(G.Config([G.STATS_I32, G.STATS_F64], G.STATS_FP64, [0, 0])) as ctx:
        with pytest.raises(G.StatsError) as e:
            G.stats_accumulate_csv(ctx, path, skip_lines=0, chunk_bytes=64)
        assert e.value.code == G.STATS_EFORMAT
