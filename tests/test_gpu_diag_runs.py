"""Runs of diagonal ops inside the tile passes: long chains of diagonal gates
(RZZ, RZ, CZ, CP) between dense layers, so that the passes carry runs of up
to four fused diagonal ops applied in one sweep (4096-amplitude tiles and
1024-amplitude tiles). Checked per element against the FP64 oracle with the
codec off, and streams = persistent byte for byte with the codec on."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu


def diag_heavy(n: int, layers: int, seed: int) -> inputs.Circuit:
    """H on every qubit, then `layers` x (a chain of 3n diagonal gates on random qubits, then U3 on every
    qubit); angles and qubits from the seeded generator."""
    rng = inputs.SplitMix64(seed)
    gates = [inputs.H(q) for q in range(n)]

    def pick(k):
        return rng.below(k)

    for _ in range(layers):
        for _ in range(3 * n):
            kind = pick(4)
            a = pick(n)
            b = (a + 1 + pick(n - 1)) % n
            th = 2 * math.pi * rng.uniform()
            if kind == 0:
                gates.append(inputs.RZZ(a, b, th))
            elif kind == 1:
                gates.append(inputs.RZ(a, th))
            elif kind == 2:
                gates.append(inputs.CZ(a, b))
            else:
                gates.append(inputs.CP(a, b, th))
        for q in range(n):
            gates.append(inputs.U3(q, math.pi * rng.uniform(), 2 * math.pi * rng.uniform(), 2 * math.pi * rng.uniform()))
    return inputs.Circuit(n, gates, 0, "diag-heavy", {"seed": seed})


@pytest.mark.parametrize("tile_bits", [0, 10])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_diag_runs_match_fp64(seed, tile_bits):
    c = diag_heavy(16, 3, seed)
    want = oracle.simulate(c)
    kw = dict(m=13, inner=3, k=5, codec=qsim.CODEC_NONE, prec=qsim.PREC_FP32)
    if tile_bits:
        kw["tile_bits"] = tile_bits
    plan = qsim.plan_stages(c, **kw)
    assert plan.stats()["diag_ops"] > 0
    got = qsim.run(plan).decompress().cpu().numpy().astype(np.complex128)
    # FP32 arithmetic: every amplitude within 1e-5 of the amplitude scale 2^(-n/2) of the exact state
    assert np.max(np.abs(got - want)) <= 1e-5 * 2.0 ** -8


def test_diag_runs_tcgen05_and_persistent():
    c = diag_heavy(18, 3, 7)
    kw = dict(m=12, inner=3, k=5, eps=1e-3, prec=qsim.PREC_TF32, tcgen05=1)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=1, **kw))
    for b in range(64):
        assert ref.block_stream(b) == per.block_stream(b)
    assert ref.fidelity(oracle.simulate(c)) >= 0.999


def ccz_mix(n: int, layers: int, seed: int) -> inputs.Circuit:
    """Diagonal chains that mix degree-2 phases (RZZ, CP) with doubly controlled Z gates (a degree-3 phase), so that
    a pass holds runs applied as phase polynomials next to runs applied from phase tables."""
    rng = inputs.SplitMix64(seed)
    ccz = np.diag([1, 1, 1, 1, 1, 1, 1, -1]).astype(complex)
    gates = [inputs.H(q) for q in range(n)]
    for _ in range(layers):
        for _ in range(2 * n):
            a = rng.below(n)
            b = (a + 1 + rng.below(n - 1)) % n
            kind = rng.below(3)
            if kind == 0:
                gates.append(inputs.RZZ(a, b, 2 * math.pi * rng.uniform()))
            elif kind == 1:
                gates.append(inputs.CP(a, b, 2 * math.pi * rng.uniform()))
            else:
                c3 = (b + 1 + rng.below(n - 2)) % n
                if c3 == a:
                    c3 = (c3 + 1) % n
                gates.append(inputs.Gate("ccz", (a, b, c3), (), ccz))
        for q in range(n):
            gates.append(inputs.U3(q, math.pi * rng.uniform(), 2 * math.pi * rng.uniform(), 2 * math.pi * rng.uniform()))
    return inputs.Circuit(n, gates, 0, "ccz-mix", {"seed": seed})


@pytest.mark.parametrize("seed", [1, 2])
def test_phase_polynomial_and_table_runs_match_fp64(seed):
    # 4096-amplitude passes whose diagonal ops are partly degree-2 (a run applied as one phase polynomial) and partly
    # not (CCZ products, applied from their phase tables): FP32 per element against FP64, and streams = persistent
    c = ccz_mix(16, 3, seed)
    kw = dict(m=13, inner=3, k=5, prec=qsim.PREC_FP32)
    plan = qsim.plan_stages(c, codec=qsim.CODEC_NONE, **kw)
    flags = [o["quadratic"] for s in range(plan.nstages) for o in plan.stage_ops(s) if o["type"] == 1]
    assert any(flags) and not all(flags), flags
    got = qsim.run(plan).decompress().cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - oracle.simulate(c))) <= 1e-5 * 2.0 ** -8
    ref = qsim.run(qsim.plan_stages(c, eps=1e-3, **kw))
    per = qsim.run(qsim.plan_stages(c, eps=1e-3, mode=qsim.MODE_PERSISTENT, **kw))
    for b in range(8):
        assert ref.block_stream(b) == per.block_stream(b)
