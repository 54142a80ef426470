"""Pins of the oracle's relative-bound codec (Sec. 4.3, Eq. 1-2, Algorithm 2), all on the CPU: the shift
against its defining inequality, the point-wise relative bound on every normal value (binade edges
included), exact zeros and signs, the sign-bitmap pre-scan (all-0 / all-1 chunks stored as a type only), the
lossless run coding of the remaining sign words, streams assembled by hand from the format description,
idempotence and corrupt-stream rejection."""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4, 2.0 ** -10, 0.3, 1e-6])
def test_shift_is_the_largest_admissible(rel):
    k = oracle.qszr_shift(rel)
    r = Fraction(rel) / (1 + Fraction(rel))
    assert Fraction(2) ** (k - 24) <= r < Fraction(2) ** (k - 23)


def test_shift_rejects_out_of_range():
    for rel in (0.0, -1e-3, 1.0, 2.0, float("nan"), 1e-9):
        with pytest.raises(oracle.OracleError):
            oracle.qszr_shift(rel)


def test_eq2_log_transform_bound():
    # Eq. 2 for the exact log2: moving log2|x| by b_a = log2(1 + b_r) changes |x| by a factor 1 + b_r
    for rel in (1e-2, 1e-3):
        ba = math.log2(1 + rel)
        for x in (1e-9, 0.37, 3.0):
            assert abs(2 ** (math.log2(x) + ba) - x) / x == pytest.approx(rel, rel=1e-9)


def edge_values(rng, n):
    """Log-uniform magnitudes over 40 binades, powers of two and their float neighbours, random signs."""
    mags = 2.0 ** rng.uniform(-40, 0, n)
    pw = 2.0 ** rng.integers(-40, 1, n // 4)
    below = np.nextafter(pw.astype(np.float32), np.float32(0))
    above = np.nextafter(pw.astype(np.float32), np.float32(1))
    x = np.concatenate([mags, pw, below, above]).astype(np.float32)
    x *= np.where(rng.random(x.size) < 0.5, -1, 1).astype(np.float32)
    return x


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-5])
def test_pointwise_relative_bound(rel):
    rng = np.random.default_rng(7)
    m = 11
    x = edge_values(rng, 3000)
    x = np.resize(x, 2 << m)
    x[::13] = 0.0
    x[5::17] = -0.0
    y = oracle.qszr_decode(oracle.qszr_encode(x, m, rel), m)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    nz = xd != 0
    assert np.all(np.abs(yd[nz] - xd[nz]) <= rel * np.abs(xd[nz]))
    assert np.all(yd[~nz] == 0)
    assert np.all(np.signbit(y[nz]) == np.signbit(x[nz]))
    assert not np.any(np.signbit(y[~nz]))  # a value that reconstructs to zero keeps sign 0


def test_subnormal_absolute_bound():
    rel = 1e-3
    k = oracle.qszr_shift(rel)
    m = 5
    x = np.zeros(2 << m, np.float32)
    x[:40] = (np.arange(40) + 1) * np.float32(2.0 ** -140) * np.where(np.arange(40) % 3 == 0, -1, 1)
    y = oracle.qszr_decode(oracle.qszr_encode(x, m, rel), m)
    assert np.all(np.abs(y.astype(np.float64) - x) <= 2.0 ** (k - 150))


def test_idempotent_and_deterministic():
    rng = np.random.default_rng(3)
    m = 12
    x = (rng.standard_normal(2 << m) * 2.0 ** -6).astype(np.float32)
    s1 = oracle.qszr_encode(x, m, 1e-3)
    y1 = oracle.qszr_decode(s1, m)
    s2 = oracle.qszr_encode(y1, m, 1e-3)
    assert s1 == s2
    assert np.array_equal(oracle.qszr_decode(s2, m).view(np.uint32), y1.view(np.uint32))


def hand_stream(m, k, frames):
    """A QSZR stream written straight from the format description. frames: list of bytes per frame."""
    nframes = len(frames)
    pad = lambda b: b + bytes((-len(b)) % 16)
    data_start = 32 + len(pad(bytes(4 * (nframes + 1))))
    offs, pos = [], data_start
    for fr in frames:
        offs.append(pos)
        pos += len(fr)
    offs.append(pos)
    hdr = struct.pack("<IHHBBbBIQQ", 0x525A5351, 1, 0, m, min(m, 12), k, 0, nframes, pos, 0)
    return hdr + pad(struct.pack("<%dI" % (nframes + 1), *offs)) + b"".join(frames)


def unit_frame(widths, types, mixed, planes, runs=()):
    """widths: 2 bytes (C = 1); types: 2-bit codes of the Re and Im chunk; mixed: stored sign words (u32);
    runs: run records (u16), after the stored words in the same 16-byte padded section; planes: u32 words."""
    pad = lambda b: b + bytes((-len(b)) % 16)
    t = bytes([types[0] | (types[1] << 2)])
    return (pad(bytes(widths)) + pad(t) +
            pad(struct.pack("<%dI" % len(mixed), *mixed) + struct.pack("<%dH" % len(runs), *runs)) +
            pad(struct.pack("<%dI" % len(planes), *planes)))


def test_hand_assembled_streams():
    # m = 5: one frame of 32 amplitudes, one chunk per plane; b_r = 1e-3 gives k = 14
    m, rel, k = 5, 1e-3, 14
    assert oracle.qszr_shift(rel) == k
    # 1.0 has bits 0x3F800000: code (0x3F800000 + 2^13) >> 14 = 0xFE00; 2.0: 0x40000000 >> 14 = 0x10000
    # Re all 1.0, Im all 0: d_0 = 0xFE00, d_j = 0; zigzag 0x1FC00 (bits 10..16): width 17, planes 10..16 = 1
    re_planes = [1 if 10 <= b <= 16 else 0 for b in range(17)]
    x = np.zeros(64, np.float32)
    x[0::2] = 1.0
    want = hand_stream(m, k, [unit_frame([17, 0], [0, 0], [], re_planes)])
    assert oracle.qszr_encode(x, m, rel) == want
    # alternating signs on Re: the chunk's sign word 0xAAAAAAAA is mixed (type 2) and stored;
    # Im all -2.0: code 0x10000, zigzag 0x20000, width 18 (only plane 17 set), signs all 1 (type 1)
    x[0::2] = np.where(np.arange(32) % 2 == 1, -1.0, 1.0)  # Re value j is -1 for odd j
    x[1::2] = -2.0
    im_planes = [1 if b == 17 else 0 for b in range(18)]
    want = hand_stream(m, k, [unit_frame([17, 18], [2, 1], [0xAAAAAAAA], re_planes + im_planes)])
    assert oracle.qszr_encode(x, m, rel) == want
    y = oracle.qszr_decode(want, m)
    assert np.array_equal(y, x)  # +-1 and -2 are on the grid
    # all-zero block: every frame has length 0
    z = np.zeros(64, np.float32)
    assert oracle.qszr_encode(z, m, rel) == hand_stream(m, k, [b""])


def test_hand_assembled_run_coded_signs():
    # the lossless step on the sign words left by the pre-scan: a chunk whose signs change 1 to 3 times
    # between neighbours is stored as a 2-byte run record (bit 15 = sign of value 0, 5-bit boundaries)
    m, rel, k = 5, 1e-3, 14
    re_planes = [1 if 10 <= b <= 16 else 0 for b in range(17)]  # every |Re| = 1.0 (see above)
    im_planes = [1 if b == 17 else 0 for b in range(18)]        # every |Im| = 2.0
    x = np.zeros(64, np.float32)
    # Re: values 0..9 negative -> word 0x000003FF, one boundary at 10: record 0x8000 | 10
    x[0::2] = np.where(np.arange(32) < 10, -1.0, 1.0)
    # Im: values 4..7 and 20..31 negative -> boundaries 4, 8, 20: record 4 | 8 << 5 | 20 << 10 = 0x5104
    im_neg = ((np.arange(32) >= 4) & (np.arange(32) < 8)) | (np.arange(32) >= 20)
    x[1::2] = np.where(im_neg, -2.0, 2.0)
    want = hand_stream(m, k, [unit_frame([17, 18], [3, 3], [], re_planes + im_planes, runs=[0x800A, 0x5104])])
    assert oracle.qszr_encode(x, m, rel) == want
    assert np.array_equal(oracle.qszr_decode(want, m), x)
    # Re alternating (31 boundaries): stored word first, then Im's run record, in one padded section
    x[0::2] = np.where(np.arange(32) % 2 == 1, -1.0, 1.0)
    want = hand_stream(m, k, [unit_frame([17, 18], [2, 3], [0xAAAAAAAA], re_planes + im_planes, runs=[0x5104])])
    assert oracle.qszr_encode(x, m, rel) == want
    assert np.array_equal(oracle.qszr_decode(want, m), x)
    # four boundaries are not run-coded: Im negative at 4..7 and 20..23 keeps its raw word
    im4 = ((np.arange(32) >= 4) & (np.arange(32) < 8)) | ((np.arange(32) >= 20) & (np.arange(32) < 24))
    x[1::2] = np.where(im4, -2.0, 2.0)
    want = hand_stream(m, k, [unit_frame([17, 18], [2, 2], [0xAAAAAAAA, 0x00F000F0], re_planes + im_planes)])
    assert oracle.qszr_encode(x, m, rel) == want


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 7])
def test_run_coding_sizes_and_round_trip(nb):
    # blocks whose chunks all have nb sign boundaries: 2 bytes per chunk for nb <= 3, 4 bytes otherwise,
    # against the same magnitudes with constant signs; the signs come back exactly
    rng = np.random.default_rng(40 + nb)
    m = 12
    mag = (rng.random(2 << m) * 0.5 + 0.25).astype(np.float32)
    sign = np.ones(2 << m, np.float32)
    for plane in range(2):
        for ch in range((1 << m) // 32):
            cuts = np.sort(rng.choice(np.arange(1, 32), nb, replace=False))
            s = np.ones(32, np.float32)
            for p in cuts:
                s[p:] *= -1
            sign[plane + 2 * 32 * ch: plane + 2 * 32 * (ch + 1): 2] = s
    x = mag * sign
    base = len(oracle.qszr_encode(mag, m, 1e-3))
    got = oracle.qszr_encode(x, m, 1e-3)
    per_chunk = 2 if nb <= 3 else 4
    assert len(got) == base + per_chunk * 256  # 2C = 256 chunks per 4096-amplitude frame, one frame
    y = oracle.qszr_decode(got, m)
    assert np.array_equal(np.signbit(y), np.signbit(x))


def test_sign_chunks_elided():
    # the sign words of all-positive and all-negative chunks are not stored: same length either way
    rng = np.random.default_rng(5)
    m = 12
    mag = (rng.random(2 << m) * 0.5 + 0.25).astype(np.float32)
    pos_len = len(oracle.qszr_encode(mag, m, 1e-3))
    assert len(oracle.qszr_encode(-mag, m, 1e-3)) == pos_len
    mixed = mag * np.where(rng.random(mag.size) < 0.5, -1, 1).astype(np.float32)
    # every chunk mixed: one extra 4-byte word per chunk (2C = 256 per 4096-amplitude frame)
    assert len(oracle.qszr_encode(mixed, m, 1e-3)) == pos_len + 4 * 256


def test_worst_case_and_capacity():
    rng = np.random.default_rng(11)
    m = 12
    x = (rng.standard_normal(2 << m) * 10.0 ** rng.uniform(-12, 0, 2 << m)).astype(np.float32)
    s = oracle.qszr_encode(x, m, 1e-5)
    assert len(s) <= oracle.qszr_worst_case_bytes(m)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qszr_encode(x, m, 1e-5, cap=len(s) - 1)
    assert ei.value.code == oracle.E_CAPACITY and ei.value.needed == len(s)


def test_range_and_invalid_inputs():
    m = 5
    x = np.zeros(64, np.float32)
    x[3] = np.float32(2.0 ** 64)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qszr_encode(x, m, 1e-3)
    assert ei.value.code == oracle.E_RANGE
    x[3] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qszr_encode(x, m, 1e-3)
    assert ei.value.code == oracle.E_INVALID


def test_corrupt_streams_rejected():
    m, rel = 5, 1e-3
    x = np.zeros(64, np.float32)
    x[0::2] = 1.0
    good = bytearray(oracle.qszr_encode(x, m, rel))
    frame = 48  # data_start for one frame
    bad_type = bytearray(good)
    bad_type[frame + 16] = 3  # a run-coded chunk, but the frame holds no run record: lengths disagree
    bad_magic = bytearray(good)
    bad_magic[0] ^= 1
    # run records no encoder writes: no boundary, and boundaries out of order
    x[0::2] = np.where(np.arange(32) < 10, -1.0, 1.0)
    runs = bytearray(oracle.qszr_encode(x, m, rel))
    rec_at = frame + 32  # widths (16) + types (16), then the sign section
    assert runs[rec_at:rec_at + 2] == bytes([0x0A, 0x80])
    no_boundary = bytearray(runs)
    no_boundary[rec_at:rec_at + 2] = bytes([0x00, 0x80])
    out_of_order = bytearray(runs)
    out_of_order[rec_at:rec_at + 2] = (10 | (4 << 5) | 0x8000).to_bytes(2, "little")
    for s in (bytes(bad_type), bytes(bad_magic), bytes(good[:-16]), bytes(no_boundary), bytes(out_of_order)):
        with pytest.raises(oracle.OracleError) as ei:
            oracle.qszr_decode(s, m)
        assert ei.value.code == oracle.E_CORRUPT
