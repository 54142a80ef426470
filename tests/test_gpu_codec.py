"""GPU QSZ1 codec vs the scalar oracle: byte-identical streams, exact decode,
the point-wise bound, capacity/corruption/range errors. Calls go through the
C ABI (qsim_compress_block / qsim_decompress_block)."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim
from tests.golden.fixtures import load_stream_fixture

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_encode(block, m, eb):
    out, nb = qsim.compress_block(dev(block), m, eb)
    torch.cuda.synchronize()
    return out[:nb].cpu().numpy().tobytes()


def gpu_decode(stream, m):
    buf = torch.zeros(max(16, len(stream) + 16), dtype=torch.uint8, device="cuda")
    buf[: len(stream)] = torch.frombuffer(bytearray(stream), dtype=torch.uint8).cuda()
    out = qsim.decompress_block(buf, m, nbytes=len(stream))
    return out.cpu().numpy().view(np.float32)


@pytest.mark.parametrize("name", ["qsz1_m5_unit.txt", "qsz1_m5_small.txt", "qsz1_m5_zero.txt"])
def test_hand_derived_streams(name):
    m, eb, block, stream = load_stream_fixture(name)
    assert gpu_encode(block, m, eb) == stream
    np.testing.assert_array_equal(gpu_decode(stream, m), block)


BLOCKS = [
    ("gauss", 5, 10, 1e-3), ("gauss", 10, 16, 1e-3), ("gauss", 12, 16, 1e-2), ("gauss", 13, 20, 1e-3),
    ("gauss", 16, 28, 1e-3), ("smooth", 14, 28, 1e-3), ("smooth", 17, 20, 1e-2), ("sparse", 15, 0, 1e-4),
    ("gauss", 22, 28, 1e-3),
]


def make_block(kind, m, n_equiv, seed):
    if kind == "gauss":
        return inputs.gaussian_block(m, n_equiv, seed)
    if kind == "smooth":
        return inputs.smooth_block(m, n_equiv, seed)
    return inputs.sparse_block(m, 37, seed)


@pytest.mark.parametrize("kind,m,n_equiv,eps", BLOCKS)
def test_bit_exact_vs_oracle(kind, m, n_equiv, eps):
    x = make_block(kind, m, n_equiv, 1000 + m)
    eb = eps * 2.0 ** (-max(n_equiv, 10) / 2)
    want = oracle.qsz_encode(x, m, eb)
    got = gpu_encode(x, m, eb)
    assert len(got) == len(want)
    assert got == want
    y = gpu_decode(got, m)
    np.testing.assert_array_equal(y, oracle.qsz_decode(want, m))
    assert np.max(np.abs(y.astype(np.float64) - x.astype(np.float64))) <= eb


def test_worst_case_and_zero_blocks():
    m = 12
    x = np.empty(2 << m, np.float32)
    big = float(2 ** 30 - 64)
    x[0::2] = np.where(np.arange(1 << m) % 2 == 0, big, -big)
    x[1::2] = -x[0::2]
    s = gpu_encode(x, m, 0.5)
    assert s == oracle.qsz_encode(x, m, 0.5) and len(s) == qsim.worst_case_bytes(m)
    z = np.zeros(2 << 20, np.float32)
    s = gpu_encode(z, 20, 1e-6)
    assert s == oracle.qsz_encode(z, 20, 1e-6)
    np.testing.assert_array_equal(gpu_decode(s, 20), z)


def test_capacity_error_reports_needed():
    m = 14
    x = inputs.gaussian_block(m, 20, 5)
    want = oracle.qsz_encode(x, m, 1e-6)
    rc, needed = qsim.compress_block_needed(dev(x), m, 1e-6, len(want) - 16)
    assert rc == qsim.E_CAPACITY and needed == len(want)
    rc, needed = qsim.compress_block_needed(dev(x), m, 1e-6, 64)  # smaller than the offsets table
    assert rc == qsim.E_CAPACITY and needed == len(want)


def test_range_and_invalid():
    m = 8
    x = np.zeros(2 << m, np.float32)
    x[7] = 2.0 ** 30
    rc, _ = qsim.compress_block_needed(dev(x), m, 0.5, qsim.worst_case_bytes(m))
    assert rc == qsim.E_RANGE
    x[7] = np.inf
    rc, _ = qsim.compress_block_needed(dev(x), m, 0.5, qsim.worst_case_bytes(m))
    assert rc == qsim.E_INVALID
    # the context stays usable
    y = inputs.gaussian_block(m, 12, 1)
    assert gpu_encode(y, m, 1e-4) == oracle.qsz_encode(y, m, 1e-4)


def test_corrupt_streams_rejected():
    m, eb, block, stream = load_stream_fixture("qsz1_m5_small.txt")
    cases = []
    b = bytearray(stream); b[0] ^= 1; cases.append(bytes(b))
    b = bytearray(stream); b[8] = 6; cases.append(bytes(b))
    cases.append(stream[:-16])
    b = bytearray(stream); b[48] = 33; cases.append(bytes(b))
    b = bytearray(stream); b[48] = 8; cases.append(bytes(b))
    b = bytearray(stream); b[36] = 0x50; cases.append(bytes(b))
    for s in cases:
        buf = torch.zeros(256, dtype=torch.uint8, device="cuda")
        buf[: len(s)] = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
        assert qsim.decompress_block_rc(buf, m, len(s)) == qsim.E_CORRUPT
    # valid stream still decodes afterwards
    np.testing.assert_array_equal(gpu_decode(stream, m), block)
