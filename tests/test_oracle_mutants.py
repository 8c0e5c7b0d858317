"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of the oracle (a dropped
term, a wrong sign, index or bit order, an off-by-one, the wrong rounding, the
wrong ring neighbour or chunk, a dropped derivative): codec mistakes in a
copy of oracle/zc_oracle.c, built with the oracle's own flags, collective and
selector mistakes in copies of oracle/__init__.py and oracle/selector.py
loaded as modules of their own.  The copy is
swapped in for the real oracle and a battery of pins runs against it: at
least one pin must fail.  The real oracle passes the same batteries."""
import contextlib
import ctypes
import os
import subprocess
import types

import pytest

import oracle
import test_oracle_collectives as coll
import test_oracle_heads as heads
import test_oracle_pins as pins
import test_oracle_selector as tsel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "zc_oracle.c")
PKG = os.path.join(ROOT, "oracle", "__init__.py")
# what a failing pin raises: an assertion, an oracle status error, or
# pytest's own failure (pytest.raises that saw nothing raised)
FAILURES = (Exception, pytest.fail.Exception)
SEL = os.path.join(ROOT, "oracle", "selector.py")

MUTANTS = {
    # block head predicted from the previous block's last value, not from 0
    "head_from_previous_block": [(
        "    if (i == 0) return heads ? 0 : q[e];",
        "    if (i == 0) return heads ? 0 : (e ? q[e] - q[e - 1] : q[e]);")],
    # ties rounded away from zero instead of to even
    "round_half_away": [("    double r = rint(t);", "    double r = round(t);")],
    # width one plane too many
    "width_off_by_one": [("        int w = bit_length(maxabs);",
                          "        int w = bit_length(maxabs) + (maxabs != 0);")],
    # sign plane set for positive deltas
    "sign_flipped": [("            if (di < 0) out[off + i / 8] |= (uint8_t)(1u << (i % 8));",
                      "            if (di > 0) out[off + i / 8] |= (uint8_t)(1u << (i % 8));")],
    # element i at bit 7 - i mod 8 of its plane byte (encoder and decoder alike)
    "plane_bits_msb_first": [
        ("            if (di < 0) out[off + i / 8] |= (uint8_t)(1u << (i % 8));",
         "            if (di < 0) out[off + i / 8] |= (uint8_t)(0x80u >> (i % 8));"),
        ("                    out[off + (uint64_t)(k + 1) * plane_bytes + i / 8] |= (uint8_t)(1u << (i % 8));",
         "                    out[off + (uint64_t)(k + 1) * plane_bytes + i / 8] |= (uint8_t)(0x80u >> (i % 8));"),
        ("                    if ((s[off + (uint64_t)(k + 1) * plane_bytes + i / 8] >> (i % 8)) & 1u)",
         "                    if ((s[off + (uint64_t)(k + 1) * plane_bytes + i / 8] >> (7 - i % 8)) & 1u)"),
        ("                int neg = (s[off + i / 8] >> (i % 8)) & 1u;",
         "                int neg = (s[off + i / 8] >> (7 - i % 8)) & 1u;")],
    # block offsets that leave out the sign plane (encoder and decoder alike)
    "offset_without_sign_plane": [
        ("        off += (uint64_t)(w + 1) * plane_bytes;\n    }\n    free(width);",
         "        off += (uint64_t)w * plane_bytes;\n    }\n    free(width);"),
        ("        if (w > 0) off += (uint64_t)(w + 1) * plane_bytes;",
         "        if (w > 0) off += (uint64_t)w * plane_bytes;")],
    # exclusive instead of inclusive prefix sum of the deltas
    "exclusive_scan": [(
        "            acc += di;\n            uint64_t e = j * L + i;\n            if (e < n) q[e] = acc;",
        "            uint64_t e = j * L + i;\n            if (e < n) q[e] = acc;\n            acc += di;")],
    # reconstruction with eb instead of 2 eb
    "reconstruct_with_eb": [("        float two_eb = h.eb + h.eb;", "        float two_eb = h.eb;")],
    # heads apart: a stored head read back without its 24-bit sign
    "head_field_unsigned": [(
        "            acc = (int32_t)v - ((v & 0x800000u) ? (int32_t)(1 << 24) : 0);  /* 24-bit signed */",
        "            acc = (int32_t)v;")],
    # heads apart: the head's own delta kept in the planes as well
    "head_delta_kept": [("    if (i == 0) return heads ? 0 : q[e];",
                         "    if (i == 0) return q[e];")],
    # ring step: the received chunk decoded but not added
    "reduce_drops_decoded": [("        for (uint64_t i = 0; i < n; ++i) acc[i] = acc[i] + local[i];",
                              "        for (uint64_t i = 0; i < n; ++i) acc[i] = local[i];")],
    # scatter pack: every segment read from the first displacement
    "scatter_wrong_displacement": [(
        "        const uint8_t* base = (const uint8_t*)x + displs[p] * (uint64_t)es;",
        "        const uint8_t* base = (const uint8_t*)x + displs[0] * (uint64_t)es;")],
    # range in FP32 instead of FP64 from the FP32 extremes
    "range_in_fp32": [("    return rel * ((double)mx - (double)mn);",
                       "    return rel * (double)(mx - mn);")],
    # the running minimum seeded with 0 instead of the first element
    "minmax_seeded_with_zero": [("        if (i == 0 || v < lo) lo = v;", "        if (v < lo) lo = v;")],
    # BF16 output truncated instead of rounded to nearest even
    "bf16_output_truncated": [("    u += 0x7fffu + lsb;", "    u += 0u * lsb;")],
    # |q| = 2^22 rejected although it is in range
    "range_limit_exclusive": [("    if (fabs(r) > 4194304.0) return O_ERR_RANGE;",
                               "    if (fabs(r) >= 4194304.0) return O_ERR_RANGE;")],
    # non-finite input not rejected
    "nonfinite_unchecked": [("    if (!isfinite(x)) return O_ERR_NONFINITE;\n    double t",
                             "    double t")],
    # a stream whose width bytes disagree with its payload length accepted
    "payload_sum_unchecked": [("    if (sum != h->payload) return O_ERR_FORMAT;", "")],
    # quotient taken in FP32 (a second rounding before rint)
    "quotient_in_fp32": [("    double t = (double)x / (double)two_eb;",
                          "    double t = (double)(x / two_eb);")],
    # raw stream not padded to 16 bytes
    "raw_unpadded": [("    uint64_t total = O_HEADER + pad16(payload);\n    *out_len = total;\n    if (total > cap) return O_ERR_CAPACITY;\n    memset(out, 0, total);\n    write_header(out, dtype, 5, 1,",
                      "    uint64_t total = O_HEADER + payload;\n    *out_len = total;\n    if (total > cap) return O_ERR_CAPACITY;\n    memset(out, 0, total);\n    write_header(out, dtype, 5, 1,")],
    # heads apart: head field written big-endian
    "head_field_big_endian": [("            p[0] = (uint8_t)h;\n            p[1] = (uint8_t)(h >> 8);\n            p[2] = (uint8_t)(h >> 16);",
                               "            p[2] = (uint8_t)h;\n            p[1] = (uint8_t)(h >> 8);\n            p[0] = (uint8_t)(h >> 16);")],
    # the block count recorded one too high
    "block_count_plus_one": [("    put_u32(out + 20, nb);", "    put_u32(out + 20, nb + (nb > 0));")],
    # scatter pack: each offset recorded after its own stream
    "scatter_offset_after_stream": [
        ("        seg_off[p] = pos;\n        uint64_t len = 0;", "        uint64_t len = 0;"),
        ("        pos += len;\n    }", "        pos += len;\n        seg_off[p] = pos;\n    }")],
}


def battery():
    """The pins each mutant is run against; returns the names that failed."""
    checks = [("golden_" + g, lambda g=g: pins.test_golden_streams(g)) for g in pins.GOLDEN_FILES]
    checks += [
        ("closed_form", lambda: pins.test_stream_length_closed_form(5, 1000)),
        ("quantizer", lambda: pins.test_quantizer_is_exact_round_half_even(1e-3)),
        ("widths", pins.test_width_is_bit_length_of_max_delta),
        ("blocks_independent", lambda: pins.test_blocks_are_independent(5)),
        ("brute_force", pins.test_brute_force_tiny_round_trips),
        ("error_bound", lambda: pins.test_error_bound_and_q_round_trip("tdist", 5)),
        ("heads_hand_stream", heads.test_hand_stream_l16),
        ("heads_extremes", heads.test_negative_and_extreme_heads_round_trip),
        ("heads_closed_form", lambda: heads.test_length_closed_form_and_same_values_as_plain(5)),
        ("heads_constant_blocks", heads.test_constant_blocks_store_only_heads),
        ("reduce_step", pins.test_reduce_step_is_decode_add_encode),
        ("relative_bound", pins.test_relative_bound_resolution),
        ("bf16_input", pins.test_bf16_input_matches_widened_fp32),
        ("error_codes", pins.test_error_codes),
        ("raw_stream", pins.test_raw_stream_round_trip),
        ("format_errors", pins.test_format_errors),
        ("scatter_pack", pins.test_scatter_pack_is_concatenation),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except FAILURES:
            failed.append(name)
    return failed


@contextlib.contextmanager
def oracle_built_from(path):
    saved = oracle._lib
    lib = ctypes.CDLL(path)
    oracle._declare(lib)
    oracle._lib = lib
    try:
        yield
    finally:
        oracle._lib = saved


def build_mutant(tmp_path, edits):
    src = open(SRC).read()
    for a, b in edits:
        assert src.count(a) == 1, a
        src = src.replace(a, b)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    return str(so)


def test_real_oracle_passes_the_battery():
    assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    with oracle_built_from(build_mutant(tmp_path, MUTANTS[name])):
        failed = battery()
    assert failed, "no pin caught the mutant %s" % name


# ---- the simulated collectives ------------------------------------------------

PY_MUTANTS = {
    # ring step on the wrong chunk: (r - t) instead of (r - 1 - t) mod P
    "ring_wrong_chunk": [(
        "            c = (r - 1 - t) % P\n            s, sm = reduce_step(sent[(r - 1) % P], chunk(r, c), eb_abs, log2L, want_stream=True,",
        "            c = (r - t) % P\n            s, sm = reduce_step(sent[(r - 1) % P], chunk(r, c), eb_abs, log2L, want_stream=True,")],
    # stream taken from the right-hand neighbour
    "ring_wrong_neighbour": [(
        "reduce_step(sent[(r - 1) % P], chunk(r, c), eb_abs, log2L, want_stream=True,",
        "reduce_step(sent[(r + 1) % P], chunk(r, c), eb_abs, log2L, want_stream=True,")],
    # the absorbing rank adds the sender's buffer to the sender's own
    "redoub_fold_adds_sender_buffer": [(
        "cur[i + 1] = reduce_step(s, cur[i + 1], eb_abs",
        "cur[i + 1] = reduce_step(s, cur[i], eb_abs")],
    # the bound drops the absorbed neighbours' quantization
    "redoub_bound_without_fold_term": [("    e0 = eb if r > 0 else 0.0", "    e0 = 0.0")],
    # the bound drops the returned result's quantization
    "redoub_bound_without_return_term": [("        e += eb\n    return e",
                                          "        e += 0.0\n    return e")],
}


def collective_battery():
    checks = [
        ("redoub_2", coll.test_redoub_two_ranks_closed_form),
        ("redoub_3", coll.test_redoub_three_ranks_closed_form),
        ("redoub_schedule", coll.test_redoub_schedule),
        ("redoub_bound_closed_form", coll.test_redoub_bound_closed_form),
        ("ring_2", coll.test_ring_two_ranks_closed_form),
    ]
    checks += [("redoub_bound_%d" % N, lambda N=N: coll.test_redoub_error_bound(N))
               for N in (3, 6, 8)]
    checks += [("ring_bound_%d" % P, lambda P=P: coll.test_ring_allreduce_bound_and_agreement(P))
               for P in (3, 5)]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except FAILURES:
            failed.append(name)
    return failed


@contextlib.contextmanager
def oracle_module_from(edits):
    src = open(PKG).read()
    for a, b in edits:
        assert src.count(a) == 1, a
        src = src.replace(a, b)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = PKG
    exec(compile(src, PKG, "exec"), mod.__dict__)
    saved = coll.oracle
    coll.oracle = mod
    try:
        yield
    finally:
        coll.oracle = saved


def test_real_oracle_passes_the_collective_battery():
    with oracle_module_from([]):
        assert collective_battery() == []


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_collective_mutant_fails_a_pin(name):
    with oracle_module_from(PY_MUTANTS[name]):
        failed = collective_battery()
    assert failed, "no pin caught the mutant %s" % name


# ---- the learned selector ----------------------------------------------------------

SEL_MUTANTS = {
    # the second ReLU's derivative left out of backpropagation
    "relu_derivative_dropped": [('    dA2 = (dY @ P["W3"]) * (A2 > 0)', '    dA2 = (dY @ P["W3"])')],
    # a transposed weight in backpropagation (square, so no shape error)
    "transposed_weight": [('    dA1 = (dA2 @ P["W2"]) * (A1 > 0)',
                           '    dA1 = (dA2 @ P["W2"].T) * (A1 > 0)')],
    # a bias gradient lost
    "bias_gradient_lost": [('    g["b1"] = dA1.sum(0)', '    g["b1"] = 0.0 * dA1.sum(0)')],
    # the factor 2 of the squared error's derivative dropped
    "loss_derivative_halved": [("    dY = 2.0 * R / (B * N_OUT)", "    dY = R / (B * N_OUT)")],
    # the update climbs the gradient
    "sgd_wrong_sign": [("    return np.asarray(p, np.float64) - lr * v, v",
                        "    return np.asarray(p, np.float64) + lr * v, v")],
    # the judge never rejects a prediction
    "judge_ignored": [('    if abs(float(y[k]) - math.log2(f[k])) > cfg["judge_log2"]:',
                       "    if False:")],
    # statistics: sampled spans spaced from the wrong count
    "span_spacing": [("    return [(SPAN * ((j * (m - 1)) // (S - 1)), SPAN) for j in range(S)]",
                      "    return [(SPAN * ((j * m) // S), SPAN) for j in range(S)]")],
    # statistics: spread of the spans' bits as a sample standard deviation
    "spread_with_ddof1": [("    f[13] = float(np.sqrt(np.mean((per_span - per_span.mean()) ** 2)))",
                           "    f[13] = float(np.std(per_span, ddof=1)) if len(per_span) > 1 else 0.0")],
    # statistics: sign changes that count zero deltas too
    "sign_changes_with_zeros": [("        f[11] = sum(int((v[1:] * v[:-1] < 0).sum()) for v in d) / nd2",
                                 "        f[11] = sum(int((v[1:] * v[:-1] <= 0).sum()) for v in d) / nd2")],
    # statistics: block heads taken every 16 elements instead of every 32
    "head_stride": [("    heads = [bitlen(abs(int(q[b0]))) for q in qs for b0 in range(0, len(q), 32)]",
                     "    heads = [bitlen(abs(int(q[b0]))) for q in qs for b0 in range(0, len(q), 16)]")],
    # statistics: zero-delta share over the second differences' count
    "zero_delta_share": [("        f[7] = sum(int((v == 0).sum()) for v in d) / nd",
                          "        f[7] = sum(int((v == 0).sum()) for v in d) / max(nd - len(d), 1)")],
    # statistics: share of nonzero instead of zero levels
    "zero_level_share": [("    f[8] = int((allq == 0).sum()) / tot", "    f[8] = int((allq != 0).sum()) / tot")],
    # statistics: raw bits of FP32 and BF16 swapped
    "raw_bits_swapped": [("    raw_bits = 32 if x.dtype == np.float32 else 16",
                          "    raw_bits = 16 if x.dtype == np.float32 else 32")],
    # statistics: natural instead of binary logarithm of the chunk length
    "length_natural_log": [("    f[15] = math.log2(n_c) / 16.0", "    f[15] = math.log(n_c) / 16.0")],
    # statistics: the level range without its +1
    "range_without_one": [("    f[4] = math.log2(1 + int(allq.max()) - int(allq.min()))",
                           "    f[4] = math.log2(max(int(allq.max()) - int(allq.min()), 1))")],
    # the time network's rates never judged against the measured ones
    "time_judge_ignored": [('        ok = math.isfinite(t) and abs(t - math.log2(c)) <= cfg["judge_time_log2"]',
                            "        ok = math.isfinite(t)")],
    # a time prediction read as ns per byte instead of its log2
    "time_not_exponentiated": [("        out.append(2.0 ** t if ok else c)",
                                "        out.append(t if ok else c)")],
    # the predicted rates charged to raw storage instead of the coded options
    "time_rates_ignored": [('    rate = cfg["ns_per_byte"] if rates is None else rates',
                            '    rate = cfg["ns_per_byte"]')],
    # a raw chunk's header not charged on the link
    "raw_header_free": [('    raw = bytes_in * cfg["raw_ns_per_byte"] + (32.0 + bytes_in) / link',
                         '    raw = bytes_in * cfg["raw_ns_per_byte"] + bytes_in / link')],
}


def selector_battery():
    names = [n for n in dir(tsel) if n.startswith("test_")]
    failed = []
    for name in names:
        fn = getattr(tsel, name)
        args = [("f32",), ("bf16",)] if name == "test_sampled_bits_equal_the_codec_oracle_on_the_spans" else [()]
        for a in args:
            try:
                fn(*a)
            except FAILURES:
                failed.append(name)
                break
    return failed


@contextlib.contextmanager
def selector_module_from(edits):
    src = open(SEL).read()
    for a, b in edits:
        assert src.count(a) == 1, a
        src = src.replace(a, b)
    mod = types.ModuleType("oracle.selector_mutant")
    mod.__file__ = SEL
    mod.__package__ = "oracle"
    exec(compile(src, SEL, "exec"), mod.__dict__)
    saved = tsel.S
    tsel.S = mod
    try:
        yield
    finally:
        tsel.S = saved


def test_real_selector_oracle_passes_the_selector_battery():
    with selector_module_from([]):
        assert selector_battery() == []


@pytest.mark.parametrize("name", sorted(SEL_MUTANTS))
def test_selector_mutant_fails_a_pin(name):
    with selector_module_from(SEL_MUTANTS[name]):
        failed = selector_battery()
    assert failed, "no pin caught the mutant %s" % name
