"""Pins for the scalar QSZ1 codec oracle: hand-derived streams, the
point-wise bound on every value, exact round trip, the size formula and
validation of corrupt streams."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs
from tests.golden.fixtures import load_stream_fixture, load_ties

FIXTURES = ["qsz1_m5_unit.txt", "qsz1_m5_small.txt", "qsz1_m5_zero.txt"]


@pytest.mark.parametrize("name", FIXTURES)
def test_hand_derived_streams(name):
    m, eb, block, stream = load_stream_fixture(name)
    got = oracle.qsz_encode(block, m, eb)
    assert got == stream
    back = oracle.qsz_decode(stream, m)
    np.testing.assert_array_equal(back, block)


def test_step_exponent_values():
    # largest e with 2^e <= 2 eb
    assert oracle.qsz_step_exponent(0.5) == 0
    assert oracle.qsz_step_exponent(0.49) == -1
    assert oracle.qsz_step_exponent(2.0 ** -20) == -19
    for n, eps in [(16, 1e-3), (28, 1e-3), (35, 1e-2), (35, 1e-3)]:
        eb = eps * 2.0 ** (-n / 2)
        e = oracle.qsz_step_exponent(eb)
        assert 2.0 ** e <= 2 * eb < 2.0 ** (e + 1)


def test_ties_to_even():
    e, rows = load_ties()
    x = np.array([a * 2.0 ** e for a, _ in rows], dtype=np.float32)
    q = oracle.qsz_quantize(x, e)
    assert list(q) == [b for _, b in rows]


@pytest.mark.parametrize("m,n_equiv,eps", [(5, 10, 1e-3), (10, 16, 1e-3), (12, 16, 1e-2),
                                           (13, 20, 1e-3), (14, 28, 1e-3)])
def test_pointwise_bound_and_roundtrip(m, n_equiv, eps):
    eb = eps * 2.0 ** (-n_equiv / 2)
    e = oracle.qsz_step_exponent(eb)
    for seed, gen in [(1, inputs.gaussian_block), (2, inputs.smooth_block)]:
        x = gen(m, n_equiv, seed)
        s = oracle.qsz_encode(x, m, eb)
        y = oracle.qsz_decode(s, m)
        # every reconstructed value within eb (point-wise absolute bound)
        assert np.max(np.abs(y.astype(np.float64) - x.astype(np.float64))) <= eb
        # exact: decode(encode(x)) is the quantised input, q * 2^e
        q = np.rint(x.astype(np.float64) / 2.0 ** e)  # numpy rint: ties to even
        np.testing.assert_array_equal(y.astype(np.float64), q * 2.0 ** e)
        assert len(s) <= oracle.qsz_worst_case_bytes(m)


def test_zero_block_is_header_plus_offsets():
    for m in (5, 10, 12, 16):
        s = oracle.qsz_encode(np.zeros(2 << m, np.float32), m, 1e-6)
        nframes = max(1, (1 << m) // 4096)
        assert len(s) == 32 + ((4 * (nframes + 1) + 15) // 16) * 16


def test_constant_block_size():
    # every chunk: d_0 = q, the rest 0 -> width = bit length of zigzag(q)
    m, e = 13, -10
    x = np.zeros(2 << m, np.float32)
    x[0::2] = 37 * 2.0 ** e   # q = 37 -> zigzag 74 -> 7 bits
    x[1::2] = -5 * 2.0 ** e   # q = -5 -> zigzag 9 -> 4 bits
    s = oracle.qsz_encode(x, m, 2.0 ** (e - 1))
    nframes, C = 2, 128
    frame = 256 + ((4 * C * (7 + 4) + 15) // 16) * 16
    assert len(s) == 32 + 16 + nframes * frame


def test_worst_case_reached():
    # alternating +-(2^30 - 1) codes give deltas of magnitude 2^31 - 2 -> 32-bit widths
    m, e = 12, 0
    x = np.empty(2 << m, np.float32)
    big = float(2 ** 30 - 64)  # representable in float32, |q| < 2^30
    x[0::2] = np.where(np.arange(1 << m) % 2 == 0, big, -big)
    x[1::2] = np.where(np.arange(1 << m) % 2 == 0, -big, big)
    s = oracle.qsz_encode(x, m, 0.5)
    assert len(s) == oracle.qsz_worst_case_bytes(m)
    np.testing.assert_array_equal(oracle.qsz_decode(s, m), x)


def test_capacity_reports_needed():
    m = 10
    x = inputs.gaussian_block(m, 16, 3)
    full = oracle.qsz_encode(x, m, 1e-5)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qsz_encode(x, m, 1e-5, cap=len(full) - 16)
    assert ei.value.code == oracle.E_CAPACITY and ei.value.needed == len(full)


def test_range_and_invalid():
    m = 5
    x = np.zeros(2 << m, np.float32)
    x[3] = 2.0 ** 30  # q = 2^30 with e = 0
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qsz_encode(x, m, 0.5)
    assert ei.value.code == oracle.E_RANGE
    x[3] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.qsz_encode(x, m, 0.5)
    assert ei.value.code == oracle.E_INVALID


def test_corrupt_streams_rejected():
    m, eb, block, stream = load_stream_fixture("qsz1_m5_small.txt")
    bad = []
    b = bytearray(stream); b[0] ^= 1; bad.append(bytes(b))            # magic
    b = bytearray(stream); b[8] = 6; bad.append(bytes(b))             # m
    bad.append(stream[:-16])                                          # truncated
    b = bytearray(stream); b[48] = 33; bad.append(bytes(b))           # width > 32
    b = bytearray(stream); b[48] = 8; bad.append(bytes(b))            # widths vs length
    b = bytearray(stream); b[32] = 0x40; bad.append(bytes(b))         # first offset
    b = bytearray(stream); b[36] = 0x50; bad.append(bytes(b))         # last offset != total
    for s in bad:
        with pytest.raises(oracle.OracleError) as ei:
            oracle.qsz_decode(s, m)
        assert ei.value.code == oracle.E_CORRUPT


def test_compression_ratio_porter_thomas():
    # complex Gaussian amplitudes at eps=1e-3: about 12-13 bits per value
    m, n = 14, 16
    eb = 1e-3 * 2.0 ** (-n / 2)
    x = inputs.gaussian_block(m, n, 11)
    s = oracle.qsz_encode(x, m, eb)
    cr = (8 << m) / len(s)
    assert 2.2 < cr < 3.0
