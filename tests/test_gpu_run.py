"""End-to-end GPU runs through the C ABI vs the oracle: uncompressed runs
within 1e-5 of FP64, compressed runs on the quantisation grid with fidelity
>= 0.99, closed forms, determinism across stream counts, the initial store,
the pinned-host tier and readout calls."""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def state_c64(st):
    return st.decompress().cpu().numpy()


def test_config0_uncompressed_matches_fp64():
    c = inputs.random_brick(16, 8, 0)
    p = qsim.plan_stages(c, m=10, inner=2, k=4, codec=qsim.CODEC_NONE)
    st = qsim.run(p)
    got = state_c64(st)
    want = oracle.simulate(c)
    assert np.max(np.abs(got - want)) <= 1e-5


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_fused_widths_uncompressed(k):
    c = inputs.qft_rz_cx(14, 2, 7) if k > 1 else inputs.qaoa_maxcut(14, 2, 3)
    kk = max(k, 1)
    p = qsim.plan_stages(c, m=9, inner=3, k=kk, codec=qsim.CODEC_NONE, tile_bits=10)
    got = state_c64(qsim.run(p))
    assert np.max(np.abs(got - oracle.simulate(c))) <= 1e-5


def test_config0_compressed():
    c = inputs.random_brick(16, 8, 0)
    p = qsim.plan_stages(c, m=10, inner=2, k=4, eps=1e-3)
    st = qsim.run(p)
    got = state_c64(st)
    ideal = oracle.simulate(c)
    f = oracle.fidelity(ideal, got)
    assert f >= 0.99
    # every stored amplitude is on the codec grid q * 2^e
    eb = 1e-3 * 2.0 ** -8
    e = oracle.qsz_step_exponent(eb)
    q = got.view(np.float32).astype(np.float64) / 2.0 ** e
    assert np.all(q == np.rint(q))
    # close to the oracle's staged + quantised simulation
    staged, stages, _ = oracle.simulate_staged(c, 10, 2, 1e-3)
    assert len(stages) == p.nstages
    bound = len(stages) * math.sqrt(2 * (1 << 16)) * 2.0 ** e
    assert np.linalg.norm(got - staged) <= bound
    # element by element: both sides store grid values. Where the FP32 and FP64 gate results of a stage fall on
    # opposite sides of a rounding boundary the stored values differ by one grid step, and the next stage's
    # gates spread that difference over many amplitudes (so later boundaries flip too); each stage adds at most
    # one step to any component
    gv, sv = got.view(np.float32).astype(np.float64), staged.view(np.float64)
    d = np.abs(gv - sv)
    print(f"\nconfig 0 vs staged oracle: max {d.max() / 2.0 ** e:.2f} steps, {np.mean(d == 0):.3f} equal")
    assert np.max(d) <= len(stages) * 2.0 ** e
    # GPU fidelity reduction and the run's rigorous bound
    assert abs(st.fidelity(ideal) - f) < 1e-9
    assert st.stats.fidelity_lower_bound <= f + 1e-9
    assert st.stats.fidelity_lower_bound >= 0.99
    # the run statistic sums FP32 per-thread partials (FP64 across threads): relative 1e-6
    assert abs(st.norm_sq() - st.stats.norm_sq) < 1e-6


@pytest.mark.parametrize("m,eps,mode", [(6, 1e-3, qsim.MODE_STREAMS), (9, 1e-6, qsim.MODE_STREAMS),
                                         (13, 1e-3, qsim.MODE_STREAMS), (13, 1e-6, qsim.MODE_STREAMS),
                                         (13, 1e-6, qsim.MODE_PERSISTENT)])
def test_stored_streams_reencode_exactly(m, eps, mode):
    # every block stream the stage loop stored equals the oracle's encoding of the block's decoded amplitudes
    # (decoded values lie on the grid, so re-quantising them is exact); eps 1e-6 gives chunk widths above 16
    # bits (two bit-plane transposes per chunk pair; the step 2^-27 still keeps |x| = 1 of the initial basis
    # state below 2^30 steps), m 6 and 9 frames shorter than 4096 amplitudes
    n = 15
    c = inputs.random_brick(n, 4, 7)
    st = qsim.run(qsim.plan_stages(c, m=m, inner=2, k=4, eps=eps, mode=mode))
    amps = state_c64(st).view(np.float32)
    eb = eps * 2.0 ** (-n / 2)
    for b in range(1 << (n - m)):
        blk = amps[(b << (m + 1)):((b + 1) << (m + 1))]
        assert st.block_stream(b) == oracle.qsz_encode(blk, m, eb), b


def test_streams_are_deterministic():
    c = inputs.random_brick(16, 6, 4)
    streams = []
    for ns in (1, 2, 4):
        st = qsim.run(qsim.plan_stages(c, m=10, inner=2, k=4, streams=ns))
        streams.append([st.block_stream(b) for b in range(64)])
    assert streams[0] == streams[1] == streams[2]


def test_initial_store_shortcut():
    # identity circuit: the store is the basis block plus identical zero streams
    n, m, basis = 14, 8, 5000
    c = inputs.Circuit(n, [inputs.RZ(0, 0.0)], basis)
    st = qsim.run(qsim.plan_stages(c, m=m, inner=2, k=2))
    blocks = [st.block_stream(b) for b in range(1 << (n - m))]
    b0 = basis >> m
    zero = oracle.qsz_encode(np.zeros(2 << m, np.float32), m, 1e-3 * 2 ** (-n / 2))
    for b, s in enumerate(blocks):
        if b != b0:
            assert s == zero
    one = np.zeros(2 << m, np.float32)
    one[2 * (basis & ((1 << m) - 1))] = np.float32(np.exp(-0.0j).real)
    assert blocks[b0] == oracle.qsz_encode(one, m, 1e-3 * 2 ** (-n / 2))


@pytest.mark.parametrize("m,inner", [(20, 0), (14, 2), (12, 4)])
def test_ghz_closed_form(m, inner):
    n = 20
    st = qsim.run(qsim.plan_stages(inputs.ghz(n), m=m, inner=inner, k=3, eps=1e-3))
    got = state_c64(st)
    assert np.max(np.abs(got - cf.ghz_state(n))) <= 1e-3 * 2 ** (-n / 2) * st.nstages


def test_qft_basis_closed_form():
    n, x = 18, 12345
    c = inputs.Circuit(n, inputs.qft_gates(n), x)
    st = qsim.run(qsim.plan_stages(c, m=12, inner=3, k=5, eps=1e-3))
    want = cf.qft_basis_state(n, x)
    assert st.fidelity(want) >= 0.99
    got = state_c64(st)
    assert np.max(np.abs(got - want)) <= 2 * st.nstages * 1e-3 * 2 ** (-n / 2) + 1e-5


@pytest.mark.parametrize("prec", [qsim.PREC_FP32, qsim.PREC_TF32], ids=["fp32", "tf32"])
@pytest.mark.parametrize("mode", [qsim.MODE_STREAMS, qsim.MODE_PERSISTENT], ids=["streams", "persistent"])
def test_qft_separable_phase_ops(prec, mode):
    # a 20-qubit QFT folds its far controlled phases into controlled-separable ops (targets inside and
    # outside the tiles, control inside and outside); uncompressed result against the FP64 closed form
    n, x = 20, 0x5A5A5
    c = inputs.Circuit(n, inputs.qft_gates(n), x)
    p = qsim.plan_stages(c, m=14, inner=4, k=5, codec=qsim.CODEC_NONE, prec=prec, mode=qsim.MODE_STREAMS)
    assert any(o["type"] == 3 for s in range(p.nstages) for o in p.stage_ops(s))
    if mode == qsim.MODE_PERSISTENT:  # persistent mode runs a compressed store
        st = qsim.run(qsim.plan_stages(c, m=14, inner=4, k=5, eps=1e-4, prec=prec, mode=mode))
        assert st.fidelity(cf.qft_basis_state(n, x)) >= 0.999
        return
    got = state_c64(qsim.run(p))
    tol = 1e-5 if prec == qsim.PREC_FP32 else 1e-2 * 2 ** (-n / 2)  # TF32: 1 % of the amplitude scale
    assert np.max(np.abs(got - cf.qft_basis_state(n, x))) <= tol


def test_grover_closed_form():
    n, t, marked = 16, 4, 4321
    st = qsim.run(qsim.plan_stages(inputs.grover(n, t, marked), m=10, inner=2, k=4, eps=1e-3))
    assert st.fidelity(cf.grover_state(n, t, marked)) >= 0.99


def test_amplitudes_and_host_tier():
    c = inputs.qaoa_maxcut(18, 2, 6)
    base = qsim.run(qsim.plan_stages(c, m=11, inner=2, k=4))
    capped = qsim.run(qsim.plan_stages(c, m=11, inner=2, k=4, device_tier_cap_bytes=1 << 16))
    assert capped.stats.host_tier_peak_bytes > 0
    for b in range(0, 1 << 7, 9):
        assert base.block_stream(b) == capped.block_stream(b)
    full = state_c64(base)
    idx = np.array([0, 1, 77, 5000, (1 << 18) - 1, 131072], dtype=np.uint64)
    np.testing.assert_array_equal(capped.amplitudes(idx), full[idx.astype(np.int64)])


@pytest.mark.parametrize("m,codec", [(13, qsim.CODEC_QSZ1), (14, qsim.CODEC_QSZR), (9, qsim.CODEC_QSZ1),
                                     (15, qsim.CODEC_NONE)])
def test_amplitudes_equal_full_decompress(m, codec):
    # the readout decodes only the frames (4096 amplitudes, or the whole block below 2^12) holding the requested
    # indices: bit-equal to the same amplitudes of the fully decompressed state, repeated and unsorted indices included
    c = inputs.random_brick(18, 6, 4)
    st = qsim.run(qsim.plan_stages(c, m=m, inner=2, k=4, codec=codec))
    full = state_c64(st)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 1 << 18, size=3000).astype(np.uint64)
    idx = np.concatenate([idx, idx[:100], np.array([0, (1 << 18) - 1, 4095, 4096], dtype=np.uint64)])
    np.testing.assert_array_equal(st.amplitudes(idx), full[idx.astype(np.int64)])


def test_single_block_and_phaseflip_edges():
    # m = n: one block, no global qubits; phase flips on several blocks
    n = 12
    c = inputs.grover(n, 2, 3001)
    st = qsim.run(qsim.plan_stages(c, m=12, inner=0, k=3, codec=qsim.CODEC_NONE))
    assert np.max(np.abs(state_c64(st) - oracle.simulate(c))) <= 1e-5
    st = qsim.run(qsim.plan_stages(c, m=6, inner=2, k=3, codec=qsim.CODEC_NONE))
    assert np.max(np.abs(state_c64(st) - oracle.simulate(c))) <= 1e-5


def test_config1_full_size_sampled():
    # 28-qubit QFT of a random basis state + 4 x (RZ layer, CX ladder), m = 22
    c = inputs.qft_rz_cx(28, 4, 1)
    p = qsim.plan_stages(c, m=22, inner=2, k=5, eps=1e-3)
    st = qsim.run(p)
    assert st.stats.fidelity_lower_bound >= 0.99
    idx = (inputs.splitmix64_array(77, 4096) >> np.uint64(36)).astype(np.uint64)
    got = st.amplitudes(idx).astype(np.complex128)
    want = cf.qft_rz_cx_amplitudes(28, c.meta["x"], c.meta["rz_angles"], idx)
    eb = 1e-3 * 2.0 ** -14
    # codec error per stage is <= eb per component; fp32 gate error is far smaller
    assert np.max(np.abs(got - want)) <= 2 * eb * st.nstages
    # sampled fidelity estimate
    fs = abs(np.vdot(want, got)) / (np.linalg.norm(want) * np.linalg.norm(got))
    assert fs >= 0.99


# TF32 keeps 10 mantissa bits: its error scales with the amplitudes, 2^(-n/2) = 2^-7 here; allow 2 % of that
@pytest.mark.parametrize("prec,tol", [(qsim.PREC_TF32, 2e-2 * 2.0 ** -7), (qsim.PREC_BF16X3, 1e-5)],
                         ids=["tf32", "bf16x3"])
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_tensor_core_gates_uncompressed(prec, tol, k):
    # 12 working bits -> 4096-amplitude tiles, the tensor-core shape; codec off so only gate error remains
    c = inputs.qft_rz_cx(14, 2, 7)
    p = qsim.plan_stages(c, m=9, inner=3, k=k, codec=qsim.CODEC_NONE, prec=prec)
    got = state_c64(qsim.run(p))
    want = oracle.simulate(c)
    err = np.max(np.abs(got - want))
    print(f"\nk={k} prec={prec}: max-abs {err:.3e} = {err / 2.0 ** -7:.3e} of the amplitude scale")
    assert err <= tol, err
    assert oracle.fidelity(want, got) >= 0.9999


def test_tensor_core_compressed_run():
    c = inputs.random_brick(16, 8, 0)
    ideal = oracle.simulate(c)
    for prec in (qsim.PREC_TF32, qsim.PREC_BF16X3):
        st = qsim.run(qsim.plan_stages(c, m=10, inner=2, k=5, eps=1e-3, prec=prec))
        assert st.fidelity(ideal) >= 0.99


@pytest.mark.parametrize("prec,rel_tol", [(qsim.PREC_FP32, 1e-4), (qsim.PREC_TF32, 2e-2), (qsim.PREC_BF16X3, 1e-4)],
                         ids=["fp32", "tf32", "bf16x3"])
def test_config1_gate_error_vs_fp64(prec, rel_tol):
    # the 28-qubit QFT + RZ/CX workload, codec off: only the gate arithmetic differs from the exact state
    c = inputs.qft_rz_cx(28, 4, 1)
    st = qsim.run(qsim.plan_stages(c, m=22, inner=4, k=5, codec=qsim.CODEC_NONE, prec=prec))
    idx = (inputs.splitmix64_array(91, 4096) >> np.uint64(36)).astype(np.uint64)
    got = st.amplitudes(idx).astype(np.complex128)
    want = cf.qft_rz_cx_amplitudes(28, c.meta["x"], c.meta["rz_angles"], idx)
    err = float(np.max(np.abs(got - want)))
    rel = err / 2.0 ** -14
    print(f"\ngate error vs FP64, 28-qubit QFT+RZ/CX, prec={prec}: max-abs {err:.3e}, relative to 2^-14: {rel:.3e}")
    assert err <= 1e-5 or prec == qsim.PREC_TF32
    assert rel <= rel_tol


@pytest.mark.parametrize("family", ["qft", "qaoa", "random"])
def test_reordered_partition_runs(family):
    # the commutation-aware partition: fewer stages, same state up to the codec error, and the persistent
    # kernel stores the same streams as the streams engine
    c = {"qft": inputs.qft_rz_cx(16, 2, 5), "qaoa": inputs.qaoa_maxcut(16, 2, 7),
         "random": inputs.random_brick(16, 6, 8)}[family]
    kw = dict(m=11, inner=2, k=4, eps=1e-3, reorder=1)
    st = qsim.run(qsim.plan_stages(c, **kw))
    assert st.stats.nstages <= qsim.plan_stages(c, m=11, inner=2, k=4, eps=1e-3).nstages
    assert oracle.fidelity(oracle.simulate(c), state_c64(st)) >= 0.99
    pst = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, **kw))
    for b in range(1 << (16 - 11)):
        assert pst.block_stream(b) == st.block_stream(b)
    # the reordered plan's arithmetic with the codec off: the exact final state within 1e-5
    raw = state_c64(qsim.run(qsim.plan_stages(c, codec=qsim.CODEC_NONE, **kw)))
    assert np.max(np.abs(raw - oracle.simulate(c))) <= 1e-5


@pytest.mark.parametrize("mode,codec", [(qsim.MODE_STREAMS, qsim.CODEC_QSZ1), (qsim.MODE_PERSISTENT, qsim.CODEC_QSZ1),
                                        (qsim.MODE_STREAMS, qsim.CODEC_QSZR), (qsim.MODE_STREAMS, qsim.CODEC_NONE)])
def test_empty_circuit_returns_the_initial_state(mode, codec):
    # no gates: no stage; the stored state is the initial basis state, exactly (1.0 is on both codecs' grids)
    c = inputs.Circuit(12, [], 1234, "empty")
    p = qsim.plan_stages(c, m=8, inner=2, k=4, eps=1e-3, mode=mode, codec=codec)
    assert p.nstages == 0
    st = qsim.run(p)
    want = np.zeros(1 << 12, np.complex64)
    want[1234] = 1.0
    assert np.array_equal(state_c64(st), want)
    assert st.stats.nstages == 0


def test_repeated_runs_store_identical_streams():
    # every CTA of the in-place encoder must finish its frames' records before it counts as arrived; a run
    # repeated many times stores the same bytes (collect mode adds the training-row kernels to the stream)
    circuits = list(inputs.batch_circuits(100, count=6, nmin=18, nmax=21))
    ref = {}
    for rep in range(4):
        for i, c in enumerate(circuits):
            for collect in (0, 1):
                p = qsim.plan_stages(c, m=c.n - 4, inner=2, k=5, eps=1e-3, prec=qsim.PREC_TF32, collect=collect)
                st = qsim.run(p)
                got = [st.block_stream(b) for b in range(16)]
                if (i, collect) in ref:
                    assert got == ref[(i, collect)], (i, collect, rep)
                else:
                    ref[(i, collect)] = got


def test_bench_configuration_qaoa32_mirror():
    # the default bench line's launch configuration at its full size (32 qubits, m = 25, inner 3, k = 5, TF32 on
    # tcgen05, commutation-aware partition with diagonal gates exempt, 2 streams, compressed), on the QAOA circuit
    # followed by its inverse: the ideal final state is |0...0>, so the simulated fidelity is |a_0| / ||b||
    c = inputs.qaoa_maxcut(32, 3, 1)
    mirror = inputs.Circuit(32, list(c.gates) + [inputs.dagger(g) for g in reversed(c.gates)], 0, "qaoa-mirror")
    st = qsim.run(qsim.plan_stages(mirror, m=25, inner=3, k=5, eps=1e-3, prec=qsim.PREC_TF32, tcgen05=1,
                                   reorder=1, diag_exempt=1, streams=2))
    assert st.stats.fidelity_lower_bound >= 0.99
    a0 = complex(st.amplitudes(np.array([0], dtype=np.uint64))[0])
    f = abs(a0) / math.sqrt(st.norm_sq())
    print(f"\n32-qubit QAOA mirror: |a0| / ||b|| = {f:.6f}, {st.stats.nstages} stages")
    assert f >= 0.99
    # every sampled amplitude other than |0> is at most the distance to the ideal state: the run's total codec
    # error (unitary stages keep it) plus the TF32 gate error, which spread over 2^32 amplitudes is far smaller
    idx = (inputs.splitmix64_array(5, 4096) >> np.uint64(32)).astype(np.uint64)
    idx = idx[idx != 0]
    rest = np.abs(st.amplitudes(idx).astype(np.complex128))
    assert np.max(rest) <= st.stats.err_norm_sum + 1e-6
    # sampled stored blocks re-encode byte for byte with the oracle (decoded values lie on the grid)
    eb = 1e-3 * 2.0 ** -16
    for b in (0, 1, 77, 127):
        s_ = st.block_stream(b)
        assert s_ == oracle.qsz_encode(oracle.qsz_decode(s_, 25), 25, eb), b


@pytest.mark.parametrize("prec,tc", [(qsim.PREC_FP32, 0), (qsim.PREC_TF32, 1)], ids=["fp32", "tf32-tcgen05"])
@pytest.mark.parametrize("family", ["qft", "qaoa", "random"])
def test_pass_aware_order_runs(family, prec, tc):
    # reorder = 3 (each stage's gates gathered into tile passes and fused pass by pass, in every stage; mode 2 picks
    # per stage between this layout and the partition order's, which the other tests cover): 20 qubits, working
    # vectors of 2^17 amplitudes, so every stage takes several 4096-amplitude passes. Uncompressed, the final state
    # against FP64 element by element: FP32 within 1e-5; TF32 within its per-op bound (relative 2-norm error
    # 2^-10 per dense op) and, element by element, within twice the TF32 error of the same stages fused in
    # partition order (reorder = 1), so the pass-aware order costs no accuracy; compressed, fidelity >= 0.99 and the
    # persistent kernel stores the same streams as the stream engine
    n = 20
    c = {"qft": inputs.qft_rz_cx(n, 2, 5), "qaoa": inputs.qaoa_maxcut(n, 3, 7),
         "random": inputs.random_brick(n, 8, 8)}[family]
    kw = dict(m=14, inner=3, k=5, eps=1e-3, prec=prec, tcgen05=tc, reorder=3, diag_exempt=1)
    want = oracle.simulate(c)
    p = qsim.plan_stages(c, codec=qsim.CODEC_NONE, **kw)
    assert p.stats()["passes"] > p.nstages
    assert p.stats()["passes"] < qsim.plan_stages(c, codec=qsim.CODEC_NONE, **dict(kw, reorder=1)).stats()["passes"]
    raw = state_c64(qsim.run(p))
    if prec == qsim.PREC_FP32:
        assert np.max(np.abs(raw - want)) <= 1e-5
    else:
        nops = sum(1 for s in range(p.nstages) for o in p.stage_ops(s) if o["type"] == 0)
        assert np.linalg.norm(raw - want) / np.linalg.norm(want) <= nops * 2.0 ** -10
        inorder = state_c64(qsim.run(qsim.plan_stages(c, codec=qsim.CODEC_NONE, **dict(kw, reorder=1))))
        err, err_inorder = np.max(np.abs(raw - want)), np.max(np.abs(inorder - want))
        print(f"\nTF32 max-abs error vs FP64, {family}: pass-aware {err:.3e}, partition order {err_inorder:.3e}")
        assert err <= 2.0 * err_inorder
    st = qsim.run(qsim.plan_stages(c, **kw))
    assert oracle.fidelity(want, state_c64(st)) >= 0.99
    pst = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, **kw))
    for b in range(1 << (n - 14)):
        assert pst.block_stream(b) == st.block_stream(b)
