"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of oracle/zc_oracle.c (a
dropped term, a wrong sign, index or bit order, an off-by-one, the wrong
rounding), builds it with the oracle's own flags, swaps it in for the real
oracle and runs a battery of the pins from test_oracle_pins.py: at least one
pin must fail.  The real oracle passes the same battery."""
import contextlib
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "zc_oracle.c")

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
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:  # an assertion or an oracle status error
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
