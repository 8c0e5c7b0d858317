"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test ties the oracle to something the method or mathematics fixes:
hand-derived streams (tests/golden), the closed form of the stream length,
exact rational arithmetic for the quantizer, the elementwise error bound of an
error-bounded compressor (gZCCL Sec. 2 / 3.3.2), exact integer round trips,
special inputs whose streams follow by hand, and the compositions that define
the ring step (Sec. 3.2.3) and the scatter pack (Sec. 3.3.4).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import GOLDEN, load_golden


def _parse_x(spec):
    vals = []
    for tok in spec.split(","):
        if "*" in tok:
            v, k = tok.split("*")
            vals += [float(v)] * int(k)
        else:
            vals.append(float(tok))
    return np.array(vals, np.float32)


GOLDEN_FILES = sorted(f for f in os.listdir(GOLDEN) if f.startswith("stream_"))


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_golden_streams(name):
    meta, expect, decoded = load_golden(name)
    x = _parse_x(meta["x"])
    eb = float(meta["eb"])
    log2L = int(meta["log2L"])
    got = oracle.compress(x, eb, log2L)
    assert got == expect, "stream differs from the hand-derived bytes"
    back = oracle.decompress(expect, x.size)
    np.testing.assert_array_equal(back, np.array(decoded, np.float32))


def _width_bytes(stream, nb):
    return np.frombuffer(stream[32:32 + nb], np.uint8)


def closed_form_len(widths, L):
    pad = lambda v: (v + 15) // 16 * 16
    nb = len(widths)
    payload = sum((int(w) + 1) * L // 8 for w in widths if w > 0)
    return 32 + pad(nb) + pad(payload), payload


@pytest.mark.parametrize("log2L", [4, 5, 6, 7])
@pytest.mark.parametrize("n", [1, 15, 16, 17, 100, 1000, 4099])
def test_stream_length_closed_form(log2L, n):
    rng = np.random.default_rng(n * 10 + log2L)
    x = np.cumsum(rng.normal(0, 0.05, n)).astype(np.float32)
    s = oracle.compress(x, 1e-3, log2L)
    L = 1 << log2L
    nb = (n + L - 1) // L
    h = oracle.header(s)
    assert h["nb"] == nb and h["n"] == n and h["log2L"] == log2L
    length, payload = closed_form_len(_width_bytes(s, nb), L)
    assert len(s) == length and h["payload"] == payload


def _exact_round_half_even(fr: Fraction) -> int:
    fl = math.floor(fr)
    rem = fr - fl
    if rem > Fraction(1, 2):
        return fl + 1
    if rem < Fraction(1, 2):
        return fl
    return fl if fl % 2 == 0 else fl + 1


@pytest.mark.parametrize("eb", [1e-4, 1e-3, 0.1, 0.3, 1.7e-5, 3.3])
def test_quantizer_is_exact_round_half_even(eb):
    """q is the integer nearest to x / (2 eb) in exact rational arithmetic,
    ties to even, for random values and for values planted on and beside
    half-integer ties; |x - q 2eb| <= eb then holds exactly, and the FP32
    reconstruction fl(q * 2eb) adds at most half an ulp of itself."""
    rng = np.random.default_rng(int(eb * 1e6) + 7)
    eb_f, two_eb = oracle.qparams(eb)
    assert eb_f == np.float32(eb) and two_eb == np.float32(2) * np.float32(eb_f)
    x = (rng.uniform(-1, 1, 4000) * rng.choice([1, 10, 1e3, 1e5, 3e6], 4000) * eb).astype(np.float32)
    k = rng.integers(-5000, 5000, 2000)
    ties = ((k + 0.5) * np.float64(two_eb)).astype(np.float32)
    x = np.concatenate([x, ties, np.nextafter(ties, np.float32(np.inf)),
                        np.nextafter(ties, np.float32(-np.inf)),
                        np.float32([0.0, -0.0, 1e-40, -1e-40, eb_f, -eb_f])])
    e = Fraction(float(eb_f))
    ok = []
    for xi in x.tolist():
        qe = _exact_round_half_even(Fraction(xi) / (2 * e))
        ok.append(abs(qe) <= 2 ** 22)
    ok = np.array(ok)
    q = oracle.quantize(x[ok], eb)
    for xi, qi in zip(x[ok].tolist(), q.tolist()):
        assert qi == _exact_round_half_even(Fraction(xi) / (2 * e))
        assert abs(Fraction(xi) - qi * 2 * e) <= e
        xh = np.float32(np.float32(qi) * np.float32(two_eb))
        half_ulp = Fraction(float(np.spacing(np.abs(xh)))) / 2
        assert abs(Fraction(xi) - Fraction(float(xh))) <= e + half_ulp
    for xi in x[~ok]:
        with pytest.raises(oracle.OracleError) as err:
            oracle.quantize(np.float32([xi]), eb)
        assert err.value.status == oracle.ERR_RANGE


def test_quantizer_midpoint_case():
    """A value whose exact quotient sits within half an FP32 ulp of a
    half-integer: both neighbouring levels round away in FP32, so the FP32
    reconstruction can exceed eb by at most half an ulp -- while the exact
    quantization error stays within eb."""
    eb = 1e-4
    x = np.float32(-9.4879)
    eb_f, two_eb = oracle.qparams(eb)
    q = int(oracle.quantize(np.array([x]), eb)[0])
    e = Fraction(float(eb_f))
    assert q == _exact_round_half_even(Fraction(float(x)) / (2 * e)) == -47440
    assert abs(Fraction(float(x)) - q * 2 * e) <= e
    for cand in (q - 1, q, q + 1):
        xh = np.float32(np.float32(cand) * np.float32(two_eb))
        assert abs(Fraction(float(x)) - Fraction(float(xh))) > e


@pytest.mark.parametrize("log2L", [4, 5, 6, 7])
def test_integer_round_trip_exact(log2L):
    """Any q whose deltas fit the format decodes back exactly, at every width."""
    rng = np.random.default_rng(log2L)
    L = 1 << log2L
    parts = []
    for w in range(0, 24):
        lim = 1 << w
        parts.append(rng.integers(-lim // 2, lim // 2 + 1, 3 * L + 5))
    q = np.concatenate(parts).astype(np.int32)
    q = np.clip(np.cumsum(q), -(1 << 22), 1 << 22).astype(np.int32)
    s = oracle.encode_q(q, 0.5, log2L)
    np.testing.assert_array_equal(oracle.decode_q(s, q.size), q)


def test_width_is_bit_length_of_max_delta():
    """Widths follow by hand for planted blocks: block j gets deltas with
    max |d| = 2^j - 1 (or exactly 2^j) -> width j (or j + 1)."""
    L = 32
    q = np.zeros(L * 48, np.int64)
    expect = []
    for j in range(24):
        m = (1 << j) - 1
        d = np.zeros(L, np.int64)
        d[5], d[6] = m, -m
        q[j * L:(j + 1) * L] = np.cumsum(d)
        expect.append(0 if m == 0 else int(m).bit_length())
    for j in range(24):
        b = 24 + j
        d = np.zeros(L, np.int64)
        d[0] = -(1 << j)  # head predicted from 0: q_head itself is the delta
        q[b * L:(b + 1) * L] = np.cumsum(d)
        expect.append(j + 1)
    s = oracle.encode_q(q.astype(np.int32), 0.5, 5)
    np.testing.assert_array_equal(_width_bytes(s, 48), np.array(expect, np.uint8))


CONFIG_SIGNALS = ["sin", "walk", "tdist", "const", "zeros", "ramp"]


def _signal(kind, n, rng):
    if kind == "sin":
        i = np.arange(n)
        return (np.sin(2 * np.pi * 3.3 * i / n) + rng.normal(0, 1e-3, n)).astype(np.float32)
    if kind == "walk":
        return np.cumsum(rng.normal(0, 0.01, n)).astype(np.float32)
    if kind == "tdist":
        return (rng.standard_t(3, n) * 0.01).astype(np.float32)
    if kind == "const":
        return np.full(n, 0.7371, np.float32)
    if kind == "zeros":
        return np.zeros(n, np.float32)
    return (np.arange(n) * 0.002).astype(np.float32)


@pytest.mark.parametrize("kind", CONFIG_SIGNALS)
@pytest.mark.parametrize("log2L", [4, 5, 6, 7])
def test_error_bound_and_q_round_trip(kind, log2L):
    rng = np.random.default_rng(abs(hash((kind, log2L))) % 2 ** 32)
    n = 5003
    x = _signal(kind, n, rng)
    eb = 1e-3
    s = oracle.compress(x, eb, log2L)
    eb_f = np.float64(np.float32(eb))
    y = oracle.decompress(s, n)
    err = np.abs(x.astype(np.float64) - y.astype(np.float64))
    assert np.all(err <= eb_f + np.spacing(np.abs(y)).astype(np.float64) / 2)
    q = oracle.decode_q(s, n)
    np.testing.assert_array_equal(q, oracle.quantize(x, eb))
    exact = np.abs(x.astype(np.float64) - q.astype(np.float64) * (2 * eb_f))
    assert np.all(exact <= eb_f * (1 + 2 ** -40))


def test_special_case_zeros():
    """All-zero input: every width 0, payload empty."""
    for log2L in (4, 5, 6, 7):
        n = 10000
        s = oracle.compress(np.zeros(n, np.float32), 1e-4, log2L)
        nb = (n + (1 << log2L) - 1) >> log2L
        assert len(s) == 32 + (nb + 15) // 16 * 16
        assert oracle.header(s)["payload"] == 0


def test_special_case_constant():
    """Constant c: every block holds d = (q_c, 0, ..., 0), width = bit length of q_c."""
    c, eb = np.float32(0.7371), 1e-3
    qc = _exact_round_half_even(Fraction(float(c)) / (2 * Fraction(float(np.float32(eb)))))
    for log2L in (4, 5, 6, 7):
        L = 1 << log2L
        s = oracle.compress(np.full(10 * L, c, np.float32), eb, log2L)
        w = abs(qc).bit_length()
        np.testing.assert_array_equal(_width_bytes(s, 10), np.full(10, w, np.uint8))
        assert len(s) == 32 + 16 + (10 * (w + 1) * L // 8 + 15) // 16 * 16


def test_special_case_ramp():
    """x_i = i * 2eb: q_i = i, so block j holds d = (jL, 1, 1, ...): width
    max(bit length of jL, 1)."""
    eb = 0.5
    for log2L in (4, 5, 6, 7):
        L = 1 << log2L
        nb = 9
        x = np.arange(nb * L, dtype=np.float32)
        s = oracle.compress(x, eb, log2L)
        expect = [max((j * L).bit_length(), 1) for j in range(nb)]
        np.testing.assert_array_equal(_width_bytes(s, nb), np.array(expect, np.uint8))


def test_bf16_input_matches_widened_fp32():
    """BF16 input is the FP32 value with the low mantissa bits zero: same
    stream except the dtype byte."""
    rng = np.random.default_rng(5)
    x32 = (rng.standard_t(3, 3000) * 0.05).astype(np.float32)
    bits = (x32.view(np.uint32) >> 16).astype(np.uint16)
    widened = (bits.astype(np.uint32) << 16).view(np.float32)
    s16 = oracle.compress(bits, 1e-4, 5)
    s32 = bytearray(oracle.compress(widened, 1e-4, 5))
    s32[4] = 1
    assert s16 == bytes(s32)
    # BF16 output: round-to-nearest-even of the FP32 reconstruction
    y32 = oracle.decompress(s16, 3000, oracle.F32)
    y16 = oracle.decompress(s16, 3000, oracle.BF16)
    u = y32.view(np.uint32).astype(np.uint64)
    rne = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    np.testing.assert_array_equal(y16, rne)


def test_relative_bound_resolution():
    """eb_abs = rel * (max - min) in FP64 from the FP32 extremes; a constant
    input uses max(|c|, 1)."""
    rng = np.random.default_rng(9)
    x = rng.normal(0, 3, 1001).astype(np.float32)
    mn, mx = oracle.minmax(x)
    assert mn == x.min() and mx == x.max()
    for rel in (1e-2, 1e-3, 1e-4):
        assert oracle.eb_from_rel(rel, mn, mx) == rel * (float(x.max()) - float(x.min()))
    assert oracle.eb_from_rel(1e-3, 0.25, 0.25) == 1e-3
    assert oracle.eb_from_rel(1e-3, -7.5, -7.5) == 1e-3 * 7.5
    # a range FP32 cannot hold: 2^24 + 2 - 1 = 2^24 + 1 is exact only in FP64
    assert oracle.eb_from_rel(1.0, 1.0, 16777218.0) == 16777217.0
    # extremes of one-signed inputs (neither is 0)
    pos = np.float32([5.0, 3.0, 7.0, 4.5])
    assert oracle.minmax(pos) == (3.0, 7.0)
    assert oracle.minmax(-pos) == (-7.0, -3.0)
    assert oracle.minmax(np.float32([2.5])) == (2.5, 2.5)


def test_error_codes():
    x = np.linspace(-1, 1, 100).astype(np.float32)
    bad = x.copy()
    bad[17] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(bad, 1e-3)
    assert e.value.status == oracle.ERR_NONFINITE
    bad[17] = np.inf
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(bad, 1e-3)
    assert e.value.status == oracle.ERR_NONFINITE
    big = x.copy()
    big[3] = 8e3  # 8e3 / 2e-3 = 4e6 <= 2^22: fine; 9e3 / 2e-3 > 2^22: range
    oracle.compress(big, 1e-3)
    big[3] = 9e3
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(big, 1e-3)
    assert e.value.status == oracle.ERR_RANGE
    # |q| = 2^22 is the last level in range, on both sides (2 eb = 2^-9)
    edge = np.float32([8192.0, -8192.0, 0.0])
    np.testing.assert_array_equal(oracle.quantize(edge, 2.0 ** -10), [1 << 22, -(1 << 22), 0])
    for v in (8192.001953125, -8192.001953125):
        with pytest.raises(oracle.OracleError) as e:
            oracle.quantize(np.float32([v]), 2.0 ** -10)
        assert e.value.status == oracle.ERR_RANGE
    for eb in (0.0, -1.0, float("nan"), float("inf"), 1e-300):
        with pytest.raises(oracle.OracleError) as e:
            oracle.compress(x, eb)
        assert e.value.status == oracle.ERR_ARG


def test_format_errors():
    x = np.linspace(-1, 1, 100).astype(np.float32)
    s = bytearray(oracle.compress(x, 1e-3, 5))
    for mutate in (
        lambda b: b.__setitem__(0, ord("X")),          # magic
        lambda b: b.__setitem__(4, 7),                 # dtype
        lambda b: b.__setitem__(5, 9),                 # log2L
        lambda b: b.__setitem__(32, 25),               # width beyond 24
        lambda b: b.__setitem__(20, 9),                # nb inconsistent with n
        lambda b: b.__setitem__(24, b[24] ^ 4),        # payload size
        lambda b: b.__setitem__(24, b[24] - 16),       # payload 16 short: still fits the stream
        lambda b: b.__setitem__(32, b[32] + 1),        # a width that the payload size disagrees with
    ):
        b = bytearray(s)
        mutate(b)
        with pytest.raises(oracle.OracleError) as e:
            oracle.decompress(bytes(b), 100)
        assert e.value.status == oracle.ERR_FORMAT
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress(bytes(s[:-16]), 100)           # truncated
    assert e.value.status == oracle.ERR_FORMAT
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress(bytes(s), 99)                  # n mismatch
    assert e.value.status == oracle.ERR_FORMAT


def test_empty_input_is_header_only():
    s = oracle.compress(np.zeros(0, np.float32), 1e-3, 5)
    assert len(s) == 32 and oracle.header(s)["nb"] == 0
    assert oracle.decompress(s, 0).size == 0


def test_raw_stream_round_trip():
    rng = np.random.default_rng(3)
    x = rng.normal(size=77).astype(np.float32)
    s = oracle.compress_raw(x)
    assert len(s) == 32 + (77 * 4 + 15) // 16 * 16 and oracle.header(s)["flags"] == 1
    np.testing.assert_array_equal(oracle.decompress(s, 77), x)


def test_reduce_step_is_decode_add_encode():
    """The fused ring step equals its definition: decode, add (FP32, one
    rounding, decoded + local), re-encode with the same fixed bound."""
    rng = np.random.default_rng(11)
    n, eb = 3001, 1e-3
    a = np.cumsum(rng.normal(0, 0.01, n)).astype(np.float32)
    b = np.cumsum(rng.normal(0, 0.01, n)).astype(np.float32)
    cin = oracle.compress(a, eb, 5)
    out, sm = oracle.reduce_step(cin, b, eb, 5, want_stream=True, want_sum=True)
    ref_sum = (oracle.decompress(cin, n) + b).astype(np.float32)
    np.testing.assert_array_equal(sm, ref_sum)
    assert out == oracle.compress(ref_sum, eb, 5)
    first, _ = oracle.reduce_step(None, b, eb, 5)
    assert first == oracle.compress(b, eb, 5)


@pytest.mark.parametrize("P", [2, 3, 4, 8])
def test_ring_error_bound_and_unbiased(P):
    """After the ring reduce-scatter each reduced chunk carries P-1
    quantizations (Sec. 3.3.3): |sum - exact| <= (P-1) eb + FP32 add
    rounding, and the mean error is close to 0 (Sec. 3.3.3, accuracy)."""
    rng = np.random.default_rng(P)
    n, eb = 4096 * P, 1e-3
    base = np.sin(np.arange(n) * 0.001).astype(np.float32)
    ranks = [(base + rng.normal(0, 0.01, n)).astype(np.float32) for _ in range(P)]
    result, history = oracle.ring_reduce_scatter(ranks, eb, 5)
    assert len(history) == P - 1
    exact = np.sum([r.astype(np.float64) for r in ranks], axis=0)
    bounds = oracle.chunk_bounds(n, P)
    eb_f = float(np.float32(eb))
    abs_sum = np.sum([np.abs(r.astype(np.float64)) for r in ranks], axis=0)
    errs = []
    for r in range(P):
        c = (r + 1) % P
        got = result[r].astype(np.float64)
        ex = exact[bounds[c]:bounds[c + 1]]
        lim = (P - 1) * eb_f + (P - 1) * 2.0 ** -24 * (abs_sum[bounds[c]:bounds[c + 1]] + P * eb_f)
        assert np.all(np.abs(got - ex) <= lim)
        errs.append(got - ex)
    e = np.concatenate(errs)
    assert abs(e.mean()) < 0.05 * eb_f * math.sqrt(P - 1) + 4 * e.std() / math.sqrt(e.size)


def test_scatter_pack_is_concatenation():
    """Sec. 3.3.4: each destination's block is compressed on its own and the
    streams are packed back to back; seg_off holds their offsets."""
    rng = np.random.default_rng(2)
    x = np.cumsum(rng.normal(0, 0.01, 10000)).astype(np.float32)
    counts = [1000, 0, 2500, 33, 6467]
    displs = list(np.cumsum([0] + counts[:-1]))
    packed, seg = oracle.scatter_pack(x, counts, displs, 1e-3, 5)
    parts = [oracle.compress(x[d:d + c], 1e-3, 5) for c, d in zip(counts, displs)]
    assert packed == b"".join(parts)
    np.testing.assert_array_equal(seg, np.cumsum([0] + [len(p) for p in parts]))
    assert all(int(o) % 16 == 0 for o in seg)


def test_brute_force_tiny_round_trips():
    """Every tiny input (n <= 40, every L, small integers in units of 2eb,
    including ragged tails) reconstructs exactly: q = x / (2 eb)."""
    rng = np.random.default_rng(4)
    for log2L in (4, 5, 6, 7):
        for n in range(0, 41):
            for _ in range(3):
                qv = rng.integers(-40, 41, n)
                x = (qv * 0.5).astype(np.float32)  # eb = 0.25 -> 2eb = 0.5
                s = oracle.compress(x, 0.25, log2L)
                np.testing.assert_array_equal(oracle.decode_q(s, n), qv.astype(np.int32))
                np.testing.assert_array_equal(oracle.decompress(s, n), x)


def _payload(stream, nb):
    """Width bytes and the unpadded payload of a stream with nb blocks."""
    h = oracle.header(stream)
    wb = (nb + 15) // 16 * 16
    s = np.frombuffer(stream, np.uint8)
    return s[32:32 + nb], s[32 + wb:32 + wb + h["payload"]]


@pytest.mark.parametrize("log2L", [4, 5, 6, 7])
def test_blocks_are_independent(log2L):
    """Blockwise Lorenzo (Sec. 3.3.2: cuSZp's blocks; head predicted from 0):
    a stream's width bytes and payload are the concatenation of those of its
    blocks compressed one by one, ragged last block included."""
    L = 1 << log2L
    rng = np.random.default_rng(40 + log2L)
    n = 7 * L + L // 2 + 3
    x = (np.cumsum(rng.normal(0, 0.02, n)) + rng.standard_t(3, n) * 1e-3).astype(np.float32)
    eb = 1e-3
    nb = (n + L - 1) // L
    widths, payload = _payload(oracle.compress(x, eb, log2L), nb)
    parts_w, parts_p = [], []
    for b in range(nb):
        wb, pb = _payload(oracle.compress(x[b * L:(b + 1) * L], eb, log2L), 1)
        parts_w.append(wb)
        parts_p.append(pb)
    np.testing.assert_array_equal(widths, np.concatenate(parts_w))
    np.testing.assert_array_equal(payload, np.concatenate(parts_p))


@pytest.mark.parametrize("log2L", [4, 5, 7])
def test_negation_symmetry(log2L):
    """Round-half-even is odd-symmetric, so -x quantizes to -q: the widths are
    the same, the decoded values are exactly negated."""
    rng = np.random.default_rng(50 + log2L)
    n = 3001
    x = (rng.standard_t(3, n) * 0.05).astype(np.float32)
    x[::97] = (rng.integers(-50, 51, x[::97].size) * 2e-3 + 1e-3).astype(np.float32)  # near ties
    eb = 1e-3
    nb = (n + (1 << log2L) - 1) >> log2L
    sp, sn = oracle.compress(x, eb, log2L), oracle.compress(-x, eb, log2L)
    np.testing.assert_array_equal(_width_bytes(sp, nb), _width_bytes(sn, nb))
    assert len(sp) == len(sn)
    np.testing.assert_array_equal(oracle.decode_q(sn, n), -oracle.decode_q(sp, n))
    np.testing.assert_array_equal(oracle.decompress(sn, n), -oracle.decompress(sp, n))


@pytest.mark.parametrize("k", [-3, 5])
def test_power_of_two_scaling(k):
    """x / (2 eb) is unchanged when x and eb are both scaled by 2^k (exact in
    binary floating point): the streams differ only in the bound's header
    field."""
    rng = np.random.default_rng(60 + k)
    n = 2500
    x = (rng.standard_t(3, n) * 0.1).astype(np.float32)
    eb = float(np.float32(1e-3))
    xs = (x * np.float32(2.0 ** k)).astype(np.float32)
    ebs = float(np.float32(eb) * np.float32(2.0 ** k))
    for log2L in (4, 5, 6, 7):
        a = oracle.compress(x, eb, log2L)
        b = oracle.compress(xs, ebs, log2L)
        assert len(a) == len(b)
        assert a[:16] == b[:16] and a[20:] == b[20:]
        assert oracle.header(b)["eb"] == ebs
