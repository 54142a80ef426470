"""Dense ops on the 5th-generation tensor cores (tcgen05.mma in TF32 or split BF16, both operands in shared
memory, the FP32 accumulator in tensor memory) against the FP64 oracle and the warp-level mma.sync path,
uncompressed and through the compressed stage loop: width 5 natively, widths 3 and 4 as width-5 ops (the
matrix times the identity on tile bits the op does not touch), width 6 in TF32 with a 64 KB B operand."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dense5(p):
    return sum(1 for s in range(p.nstages) for o in p.stage_ops(s) if o["type"] == 0 and o["nq"] == 5)


@pytest.mark.parametrize("prec", [qsim.PREC_TF32, qsim.PREC_BF16X3], ids=["tf32", "bf16x3"])
@pytest.mark.parametrize("family", ["qft", "brick", "qaoa"])
def test_tcgen05_matches_fp64_and_warp_mma(family, prec):
    if family == "qft":
        n = 20
        c = inputs.Circuit(n, inputs.qft_gates(n), 0x5A5A5)
        kw = dict(m=14, inner=4, k=5)
    elif family == "brick":
        n = 18
        c = inputs.random_brick(n, 10, 5)
        kw = dict(m=12, inner=2, k=5)
    else:
        n = 18
        c = inputs.qaoa_maxcut(n, 2, 3)
        kw = dict(m=13, inner=2, k=5)
    plans = [qsim.plan_stages(c, codec=qsim.CODEC_NONE, prec=prec, tcgen05=t, **kw) for t in (0, 1)]
    assert dense5(plans[1]) > 0
    warp, tc = (qsim.run(p).decompress().cpu().numpy() for p in plans)
    want = cf.qft_basis_state(n, 0x5A5A5) if family == "qft" else oracle.simulate(c)
    # TF32: both operands of every dense op rounded to TF32 (unit roundoff 2^-11), so the state's relative
    # 2-norm error grows by at most about 2^-10 per op. Split BF16: three parts of 8 bits each and the six
    # products of order <= 2 leave about 2^-22 per op, below the FP32 rounding of the other ops; bound at 2^-20
    # per op. Either way tcgen05 stays as close to FP64 as the warp-level path.
    nops = sum(1 for s in range(plans[1].nstages) for o in plans[1].stage_ops(s) if o["type"] == 0)
    err_tc = np.linalg.norm(tc - want) / np.linalg.norm(want)
    err_warp = np.linalg.norm(warp - want) / np.linalg.norm(want)
    per_op = 2.0 ** -10 if prec == qsim.PREC_TF32 else 2.0 ** -20
    assert err_tc <= nops * per_op
    assert err_tc <= 1.5 * err_warp + 1e-6
    if prec == qsim.PREC_TF32:
        assert np.max(np.abs(tc - want)) <= 2e-2 * 2 ** (-n / 2)
    else:
        assert np.max(np.abs(tc - want)) <= 1e-5  # the FP32 paths' bound
    # the norm drifts with TF32 rounding as much as on the warp-level path
    assert abs(np.vdot(tc, tc).real - np.vdot(warp, warp).real) < 1e-3


def test_tcgen05_compressed_runs():
    c = inputs.qft_rz_cx(22, 2, 3)
    kw = dict(m=16, inner=4, k=5, eps=1e-3, prec=qsim.PREC_TF32)
    ideal = oracle.simulate(c)
    for streams in (1, 2):
        st = qsim.run(qsim.plan_stages(c, tcgen05=1, streams=streams, **kw))
        assert st.fidelity(ideal) >= 0.999
    st = qsim.run(qsim.plan_stages(c, tcgen05=1, **dict(kw, prec=qsim.PREC_BF16X3)))
    assert st.fidelity(ideal) >= 0.999
    # the persistent stage kernel runs the same TF32 MMAs on tcgen05 (128-thread CTAs, one thread per index group):
    # the same streams as the stream engine, byte for byte
    a = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, tcgen05=1, **kw))
    b = qsim.run(qsim.plan_stages(c, tcgen05=1, **kw))
    for blk in range(64):
        assert a.block_stream(blk) == b.block_stream(blk)


def test_tcgen05_bounded_wait_reports_timeout():
    # test hook: no MMA is issued or committed to the mbarrier, so every tile's wait runs out (1 s) and the run
    # ends with QSIM_E_TIMEOUT instead of hanging; the context stays usable
    c = inputs.random_brick(12, 4, 1)
    kw = dict(m=12, inner=2, k=5, prec=qsim.PREC_TF32, tcgen05=1, codec=qsim.CODEC_NONE)
    cfg = qsim.default_config(**kw)
    cfg.reserved[0] = 2
    stalled = qsim.Plan(c.n, c.gates, cfg)
    assert dense5(stalled) > 0
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run(stalled)
    assert ei.value.code == qsim.E_TIMEOUT
    got = qsim.run(qsim.plan_stages(c, **kw)).decompress().cpu().numpy()
    want = oracle.simulate(c)
    assert np.linalg.norm(got - want) <= stalled.stats()["dense_ops"] * 2.0 ** -10


def test_bench_configuration_full_size_sampled():
    # the default bench line's launch configuration: 28-qubit QFT of a random basis state + 4 x (RZ layer, CX
    # ladder), m = 22, inner 4, k = 5, TF32 on tcgen05, 2 streams, compressed; 4096 sampled amplitudes against
    # the closed form
    c = inputs.qft_rz_cx(28, 4, 1)
    st = qsim.run(qsim.plan_stages(c, m=22, inner=4, k=5, eps=1e-3, prec=qsim.PREC_TF32, tcgen05=1, streams=2))
    assert st.stats.fidelity_lower_bound >= 0.99
    idx = (inputs.splitmix64_array(78, 4096) >> np.uint64(36)).astype(np.uint64)
    got = st.amplitudes(idx).astype(np.complex128)
    want = cf.qft_rz_cx_amplitudes(28, c.meta["x"], c.meta["rz_angles"], idx)
    eb = 1e-3 * 2.0 ** -14
    # codec error <= eb per component per stage, plus the TF32 gate error (2 % of the amplitude scale bound)
    assert np.max(np.abs(got - want)) <= 2 * eb * st.nstages + 2e-2 * 2.0 ** -14
    fs = abs(np.vdot(want, got)) / (np.linalg.norm(want) * np.linalg.norm(got))
    assert fs >= 0.99


@pytest.mark.parametrize("prec,rel_tol", [(qsim.PREC_TF32, 2e-2), (qsim.PREC_BF16X3, 1e-4)], ids=["tf32", "bf16x3"])
def test_full_size_gate_error_vs_fp64(prec, rel_tol):
    # the 28-qubit workload with the codec off: the tcgen05 gate arithmetic against the exact state, with the
    # warp-level path's bounds
    c = inputs.qft_rz_cx(28, 4, 1)
    st = qsim.run(qsim.plan_stages(c, m=22, inner=4, k=5, codec=qsim.CODEC_NONE, prec=prec, tcgen05=1))
    idx = (inputs.splitmix64_array(91, 4096) >> np.uint64(36)).astype(np.uint64)
    got = st.amplitudes(idx).astype(np.complex128)
    want = cf.qft_rz_cx_amplitudes(28, c.meta["x"], c.meta["rz_angles"], idx)
    err = float(np.max(np.abs(got - want)))
    assert err / 2.0 ** -14 <= rel_tol
    if prec == qsim.PREC_BF16X3:
        assert err <= 1e-5


@pytest.mark.parametrize("prec", [qsim.PREC_TF32, qsim.PREC_BF16X3], ids=["tf32", "bf16x3"])
@pytest.mark.parametrize("k", [3, 4])
def test_tcgen05_widths_3_and_4(k, prec):
    # fused to at most k qubits: every dense op of width 3 or 4 in a 4096-amplitude tile pass runs on tcgen05
    # as a width-5 op; against FP64 with the per-op bounds above, and no worse than the warp-level path
    cases = [(inputs.qft_rz_cx(14, 2, 7), dict(m=9, inner=3)), (inputs.random_brick(16, 8, 2), dict(m=10, inner=2))]
    for c, kw in cases:
        plans = [qsim.plan_stages(c, codec=qsim.CODEC_NONE, prec=prec, k=k, tcgen05=t, **kw) for t in (0, 1)]
        nk = sum(1 for s in range(plans[1].nstages) for o in plans[1].stage_ops(s) if o["type"] == 0 and o["nq"] == k)
        assert nk > 0
        warp, tc = (qsim.run(p).decompress().cpu().numpy() for p in plans)
        want = oracle.simulate(c)
        nops = sum(1 for s in range(plans[1].nstages) for o in plans[1].stage_ops(s) if o["type"] == 0)
        err_tc = np.linalg.norm(tc - want) / np.linalg.norm(want)
        err_warp = np.linalg.norm(warp - want) / np.linalg.norm(want)
        per_op = 2.0 ** -10 if prec == qsim.PREC_TF32 else 2.0 ** -20
        print(f"\nk={k} prec={prec} n={c.n}: tcgen05 {err_tc:.3e}, warp/cuda-core {err_warp:.3e}, {nops} dense ops")
        assert err_tc <= nops * per_op
        assert err_tc <= 1.5 * err_warp + 1e-6
        if prec == qsim.PREC_BF16X3:
            assert np.max(np.abs(tc - want)) <= 1e-5
        else:
            assert np.max(np.abs(tc - want)) <= 2e-2 * 2 ** (-c.n / 2)


def test_tcgen05_width_6_tf32():
    # fused to 6 qubits: width-6 dense ops run on tcgen05 in TF32 (M = 128 with 64 live rows, K = N = 128);
    # against the FP32 CUDA-core run of the same plan the tcgen05 run shows TF32-sized errors (the tensor-core
    # path ran), within the per-op bound, and stays close to FP64
    cases = [(inputs.qft_rz_cx(14, 2, 7), dict(m=9, inner=3)), (inputs.random_brick(16, 8, 2), dict(m=10, inner=2))]
    for c, kw in cases:
        plans = [qsim.plan_stages(c, codec=qsim.CODEC_NONE, k=6, **kw),
                 qsim.plan_stages(c, codec=qsim.CODEC_NONE, prec=qsim.PREC_TF32, k=6, tcgen05=1, **kw)]
        n6 = sum(1 for s in range(plans[1].nstages) for o in plans[1].stage_ops(s) if o["type"] == 0 and o["nq"] == 6)
        assert n6 > 0
        fp32, tc = (qsim.run(p).decompress().cpu().numpy() for p in plans)  # FP32 CUDA cores, TF32 tcgen05
        want = oracle.simulate(c)
        nops = sum(1 for s in range(plans[1].nstages) for o in plans[1].stage_ops(s) if o["type"] == 0)
        err_tc = np.linalg.norm(tc - want) / np.linalg.norm(want)
        err_fp32 = np.linalg.norm(fp32 - want) / np.linalg.norm(want)
        print(f"\nk=6 tf32 n={c.n}: tcgen05 {err_tc:.3e}, cuda cores {err_fp32:.3e}, {n6} width-6 of {nops} dense ops")
        assert err_tc <= nops * 2.0 ** -10
        assert err_tc > 10 * err_fp32  # TF32 operands: the tensor-core path ran
        assert np.max(np.abs(tc - want)) <= 2e-2 * 2 ** (-c.n / 2)
        assert oracle.fidelity(want, tc) >= 0.9999
