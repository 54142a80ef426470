"""GPU relative-bound codec (QSZR: Sec. 4.3, Eq. 1-2, Algorithm 2) vs the scalar oracle, through the C ABI:
byte-identical streams and exact decodes for blocks of several sizes and value mixes (run-coded sign chunks
included), the point-wise relative
bound, range / capacity / corruption errors, and the stage loop (stream engine, persistent kernel, batch)
storing QSZR blocks that re-encode exactly."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_encode(block, m, rel):
    out, nb = qsim.compress_block_rel(dev(block), m, rel)
    torch.cuda.synchronize()
    return out[:nb].cpu().numpy().tobytes()


def gpu_decode(stream, m):
    buf = torch.zeros(max(16, len(stream) + 16), dtype=torch.uint8, device="cuda")
    buf[: len(stream)] = torch.frombuffer(bytearray(stream), dtype=torch.uint8).cuda()
    out = qsim.decompress_block(buf, m, nbytes=len(stream))
    return out.cpu().numpy().view(np.float32)


def block(kind, m, seed):
    rng = np.random.default_rng(seed)
    n = 2 << m
    if kind == "gauss":
        return (rng.standard_normal(n) * 2.0 ** -8).astype(np.float32)
    if kind == "binades":  # magnitudes over 40 binades, powers of two and their neighbours, zeros, both signs
        x = (2.0 ** rng.uniform(-40, 0, n)).astype(np.float32)
        pw = (2.0 ** rng.integers(-40, 1, n)).astype(np.float32)
        x[1::5] = pw[1::5]
        x[2::5] = np.nextafter(pw[2::5], np.float32(0))
        x[::11] = 0.0
        x *= np.where(rng.random(n) < 0.5, -1, 1).astype(np.float32)
        return x
    if kind == "negative":
        return -(rng.random(n) * 0.5 + 0.01).astype(np.float32)
    if kind == "alternating":
        return (np.where(np.arange(n) % 4 < 2, 1, -1) * (rng.random(n) + 0.5) * 2.0 ** -6).astype(np.float32)
    if kind == "subnormal":
        return (rng.integers(-2000, 2000, n) * np.float32(2.0 ** -149)).astype(np.float32)
    if kind == "zero":
        return np.zeros(n, np.float32)
    if kind == "runs":  # every 32-value chunk of each plane changes sign 0..5 times: run-coded and stored words
        x = (rng.random(n) * 0.5 + 0.25).astype(np.float32)
        for plane in range(2):
            for ch in range(n // 64):
                nb = int(rng.integers(0, 6))
                s = np.ones(32, np.float32) * (1 if rng.random() < 0.5 else -1)
                for p in np.sort(rng.choice(np.arange(1, 32), nb, replace=False)):
                    s[p:] *= -1
                x[plane + 64 * ch: plane + 64 * (ch + 1): 2] *= s
        return x
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["gauss", "binades", "negative", "alternating", "subnormal", "zero", "runs"])
@pytest.mark.parametrize("m", [5, 8, 12, 14])
@pytest.mark.parametrize("rel", [1e-3, 1e-2])
def test_bit_exact_vs_oracle(kind, m, rel):
    x = block(kind, m, 100 * m + len(kind))
    want = oracle.qszr_encode(x, m, rel)
    got = gpu_encode(x, m, rel)
    assert got == want
    y = gpu_decode(got, m)
    assert np.array_equal(y.view(np.uint32), oracle.qszr_decode(want, m).view(np.uint32))
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    normal = np.abs(xd) >= 2.0 ** -126
    assert np.all(np.abs(yd[normal] - xd[normal]) <= rel * np.abs(xd[normal]))


def test_capacity_range_invalid():
    m, rel = 9, 1e-3
    x = block("gauss", m, 1)
    want = oracle.qszr_encode(x, m, rel)
    rc, needed = qsim.compress_block_rel_rc(dev(x), m, rel, len(want) - 16)
    assert rc == qsim.E_CAPACITY and needed == len(want)
    y = x.copy()
    y[7] = np.float32(2.0 ** 64)
    assert qsim.compress_block_rel_rc(dev(y), m, rel, 1 << 16)[0] == qsim.E_RANGE
    y[7] = np.inf
    assert qsim.compress_block_rel_rc(dev(y), m, rel, 1 << 16)[0] == qsim.E_INVALID
    assert qsim.compress_block_rel_rc(dev(x), m, 1.5, 1 << 16)[0] == qsim.E_INVALID


def test_corrupt_streams_rejected():
    m, rel = 5, 1e-3
    x = np.zeros(64, np.float32)
    x[0::2] = 1.0
    good = bytearray(oracle.qszr_encode(x, m, rel))
    bad_type = bytearray(good)
    bad_type[48 + 16] = 3  # first frame at 48: widths (16 B), then the sign chunk types
    bad_k = bytearray(good)
    bad_k[10] = 30
    for s in (bytes(bad_type), bytes(bad_k), bytes(good[:-16])):
        buf = torch.zeros(256, dtype=torch.uint8, device="cuda")
        buf[: len(s)] = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
        assert qsim.decompress_block_rc(buf, m, len(s)) == qsim.E_CORRUPT


@pytest.mark.parametrize("m", [9, 12])
def test_stage_loop_stores_relative_streams(m):
    n = 15
    c = inputs.random_brick(n, 6, 9)
    st = qsim.run(qsim.plan_stages(c, m=m, inner=2, k=4, eps=1e-3, codec=qsim.CODEC_QSZR))
    amps = st.decompress().cpu().numpy()
    f = oracle.fidelity(oracle.simulate(c), amps)
    assert f >= 0.999
    flat = amps.view(np.float32)
    for b in range(1 << (n - m)):
        blk = flat[(b << (m + 1)):((b + 1) << (m + 1))]
        assert st.block_stream(b) == oracle.qszr_encode(blk, m, 1e-3), b
    # the run's statistics come from the same encoder
    assert st.stats.fidelity_lower_bound >= 0.99 and st.stats.nstages >= 1


@pytest.mark.parametrize("prec", [qsim.PREC_FP32, qsim.PREC_TF32], ids=["fp32", "tf32"])
@pytest.mark.parametrize("graph", [0, 1])
def test_relative_codec_persistent_matches_streams(prec, graph):
    # the persistent stage kernel's in-place encoder and frame copy store the stream engine's bytes
    c = inputs.random_brick(16, 8, 2)
    kw = dict(m=10, inner=2, k=5, eps=1e-3, prec=prec, codec=qsim.CODEC_QSZR)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=graph, **kw))
    for b in range(64):
        assert per.block_stream(b) == ref.block_stream(b)
    assert per.fidelity(oracle.simulate(c)) >= 0.999


def test_relative_codec_persistent_qft_and_batch():
    # 2^22-amplitude working vectors with leading phase ops, then a uniform relative-codec batch in one launch
    c = inputs.qft_rz_cx(24, 2, 5)
    kw = dict(m=20, inner=2, k=5, eps=1e-3, codec=qsim.CODEC_QSZR)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=1, **kw))
    for b in range(16):
        assert per.block_stream(b) == ref.block_stream(b)
    circuits = [inputs.random_brick(13, 6, 31), inputs.qft_rz_cx(12, 1, 4), inputs.ghz(11)]
    plans = [qsim.plan_stages(x, m=x.n - 3, inner=2, k=4, eps=1e-3, codec=qsim.CODEC_QSZR) for x in circuits]
    states, launch = qsim.run_batch(plans)
    assert launch["launches"] == 1
    for x, p, st in zip(circuits, plans, states):
        one = qsim.run(p)
        for b in range(8):
            assert st.block_stream(b) == one.block_stream(b), x.family
    mixed = [plans[0], qsim.plan_stages(circuits[1], m=9, inner=2, k=4, eps=1e-3)]
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch(mixed)  # one codec per batch
    assert ei.value.code == qsim.E_INVALID


def test_relative_codec_with_learned_sizing():
    # rows logged by relative-bound runs train the predictor; predicted slots store the same streams as exact
    # sizing, and a forced under-estimate re-reserves exactly
    kw = dict(m=10, inner=2, k=4, eps=1e-3, codec=qsim.CODEC_QSZR)
    rows = np.concatenate([qsim.run(qsim.plan_stages(inputs.random_brick(14, 6, 300 + s), collect=1, **kw))
                           .training_data() for s in range(3)])
    qsim.predictor_train(rows, epochs=30, batch=64, lr=3e-3, seed=5)
    c = inputs.random_brick(14, 8, 4)
    exact = qsim.run(qsim.plan_stages(c, **kw))
    for margin in (0.25, -0.9):
        pred = qsim.run(qsim.plan_stages(c, sizing=qsim.SIZING_PREDICT, predictor_margin=margin, **kw))
        for b in range(16):
            assert pred.block_stream(b) == exact.block_stream(b)
        if margin < 0:
            assert pred.stats.overflow_blocks > 0
    for margin in (0.25, -0.9):  # the persistent kernel keeps fitting predicted slots the same way
        per = qsim.run(qsim.plan_stages(c, sizing=qsim.SIZING_PREDICT, predictor_margin=margin,
                                        mode=qsim.MODE_PERSISTENT, **kw))
        for b in range(16):
            assert per.block_stream(b) == exact.block_stream(b)
        if margin < 0:
            assert per.stats.overflow_blocks > 0


def test_relative_streams_in_host_tier_and_readout():
    # device tier capped: blocks land in pinned host memory, same streams; amplitude readout decodes QSZR
    c = inputs.qaoa_maxcut(16, 2, 6)
    kw = dict(m=10, inner=2, k=4, eps=1e-3, codec=qsim.CODEC_QSZR)
    base = qsim.run(qsim.plan_stages(c, **kw))
    capped = qsim.run(qsim.plan_stages(c, device_tier_cap_bytes=1 << 16, **kw))
    assert capped.stats.host_tier_peak_bytes > 0
    for b in range(0, 1 << 6, 5):
        assert base.block_stream(b) == capped.block_stream(b)
    full = base.decompress().cpu().numpy()
    idx = np.array([0, 3, 999, (1 << 16) - 1, 40000], dtype=np.uint64)
    np.testing.assert_array_equal(capped.amplitudes(idx), full[idx.astype(np.int64)])
    ideal = oracle.simulate(c)
    assert oracle.fidelity(ideal, full) >= 0.999


@pytest.mark.parametrize("rel", [None, 1e-3])
def test_largest_block_both_codecs(rel):
    # m = 26, the largest block: 2^26 amplitudes (512 MiB), 16384 frames; streams byte-identical to the oracle
    m = 26
    rng = np.random.default_rng(26)
    x = (rng.standard_normal(2 << m, dtype=np.float32) * np.float32(2.0 ** -13))
    x[: 1 << 20] = 0.0  # a run of zero frames at the start
    if rel is None:
        eb = 1e-3 * 2.0 ** -13
        out, nb = qsim.compress_block(dev(x), m, eb)
        want = oracle.qsz_encode(x, m, eb)
    else:
        out, nb = qsim.compress_block_rel(dev(x), m, rel)
        want = oracle.qszr_encode(x, m, rel)
    torch.cuda.synchronize()
    got = out[:nb].cpu().numpy().tobytes()
    assert got == want
    y = qsim.decompress_block(out, m, nbytes=nb).cpu().numpy().view(np.float32)
    ref = oracle.qsz_decode(want, m) if rel is None else oracle.qszr_decode(want, m)
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))
