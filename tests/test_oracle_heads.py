"""Pins of the heads-apart stream format (flag bit 1): a hand-derived
stream, the closed form of its length, agreement of its decoding with the
plain format's, and the saving on data with a large offset."""
import numpy as np
import pytest

import oracle

EB = 2.0 ** -10  # 2 eb = 2^-9


def test_hand_stream_l16():
    # q = 1000, 1001, 1001, 999 (then the tail): head 1000 stored apart,
    # deltas 0, 1, 0, -2 -> width 2, planes sign/0/1 of 2 bytes each
    q = np.array([1000, 1001, 1001, 999], np.int32)
    s = oracle.encode_q_heads(q, EB, 4)
    assert len(s) == 32 + 16 + 16 + 16
    h = oracle.header(s)
    assert h["flags"] == 2 and h["nb"] == 1 and h["payload"] == 6 and h["log2L"] == 4
    assert s[32] == 2 and s[33:48] == bytes(15)                  # width byte, padding
    assert s[48:51] == bytes([0xe8, 0x03, 0x00]) and s[51:64] == bytes(13)  # head 1000
    # sign plane: element 3 negative; plane 0: element 1; plane 1: element 3 (|-2| = 2)
    assert s[64:70] == bytes([0x08, 0x00, 0x02, 0x00, 0x08, 0x00])
    assert s[70:80] == bytes(10)
    np.testing.assert_array_equal(oracle.decode_q(s, 4), q)


def test_negative_and_extreme_heads_round_trip():
    q = np.array([-(1 << 22), 5, 1 << 22, -1, 0, 7, -8388608 // 2], np.int32)
    for lg in (4, 5, 6, 7):
        s = oracle.encode_q_heads(np.repeat(q, 40), EB, lg)
        np.testing.assert_array_equal(oracle.decode_q(s, q.size * 40), np.repeat(q, 40))


@pytest.mark.parametrize("lg", [4, 5, 6, 7])
def test_length_closed_form_and_same_values_as_plain(lg):
    r = np.random.default_rng(lg)
    x = (np.cumsum(r.normal(0, 0.01, 10007)) + 37.0).astype(np.float32)
    eb = 1e-3
    s2 = oracle.compress_heads(x, eb, lg)
    s1 = oracle.compress(x, eb, lg)
    n = x.size
    np.testing.assert_array_equal(oracle.decompress(s2, n), oracle.decompress(s1, n))
    q = oracle.quantize(x, eb).astype(np.int64)
    L = 1 << lg
    nb = (n + L - 1) // L
    payload = 0
    for j in range(nb):
        blk = q[j * L:(j + 1) * L]
        w = int(np.abs(np.diff(blk)).max()).bit_length() if blk.size > 1 else 0
        payload += (w + 1) * L // 8 if w else 0
    assert len(s2) == 32 + oracle.pad16(nb) + oracle.pad16(3 * nb) + oracle.pad16(payload)
    # the offset of 37 costs the plain format its bit length on every element
    assert len(s2) < 0.6 * len(s1)


def test_constant_blocks_store_only_heads():
    x = np.full(4096, 1.5, np.float32)
    s = oracle.compress_heads(x, 1e-3, 5)
    assert oracle.header(s)["payload"] == 0
    assert len(s) == 32 + 128 + oracle.pad16(3 * 128)


def test_flag_combinations_rejected():
    s = bytearray(oracle.compress_heads(np.arange(64, dtype=np.float32), 1e-2, 5))
    s[6] = 3
    with pytest.raises(oracle.OracleError):
        oracle.header(bytes(s))
    s = bytearray(oracle.compress_heads(np.arange(64, dtype=np.float32), 1e-2, 5))
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bytes(s[:-16]), 64)  # heads or payload cut off
