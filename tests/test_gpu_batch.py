"""A batch of independent circuits in one persistent launch (qsim_run_batch):
every circuit's compressed state is byte-identical to the same plan run on its
own, each circuit reaches fidelity >= 0.99 against the FP64 oracle, exact and
learned sizing mix in one batch, a stalled dependency ends the launch with
QSIM_E_TIMEOUT, and malformed batches are rejected."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu


def streams_of(st, nblocks):
    return [st.block_stream(b) for b in range(nblocks)]


def batch_plans(seed, count, prec, **extra):
    """Uneven circuits (GHZ, QFT, random brick, Grover; n in 10..14) with per-circuit m and k."""
    plans = []
    for i, c in enumerate(inputs.batch_circuits(seed, count=count, nmin=10, nmax=14)):
        m = c.n - 3 - (i % 2)
        k = 3 + (i % 3)
        plans.append((c, qsim.plan_stages(c, m=m, inner=2, k=k, eps=1e-3, prec=prec, **extra)))
    return plans


@pytest.mark.parametrize("prec", [qsim.PREC_FP32, qsim.PREC_TF32], ids=["fp32", "tf32"])
def test_batch_matches_single_runs(prec):
    plans = batch_plans(11, 8, prec)
    states, launch = qsim.run_batch([p for _, p in plans])
    assert launch["launches"] == 1 and launch["seconds"] > 0 and launch["alg_bytes"] > 0
    for (c, p), st in zip(plans, states):
        nblocks = 1 << (c.n - p.cfg.m)
        ref = qsim.run(p)  # the streams engine, one circuit
        assert streams_of(ref, nblocks) == streams_of(st, nblocks), c.family
        assert st.stats.nstages == ref.stats.nstages
        assert abs(st.stats.norm_sq - ref.stats.norm_sq) < 1e-6  # FP32 partial sums, another order
        assert st.fidelity(oracle.simulate(c)) >= 0.99


def test_batch_single_circuit_and_repeat():
    # a batch of one, then the same batch twice in a row (queue counters and epochs reset by the launch)
    c, p = batch_plans(3, 1, qsim.PREC_FP32)[0]
    nblocks = 1 << (c.n - p.cfg.m)
    ref = streams_of(qsim.run(p), nblocks)
    for _ in range(2):
        states, _ = qsim.run_batch([p])
        assert streams_of(states[0], nblocks) == ref


def test_batch_mixed_sizing_with_learned_predictor():
    kw = dict(m=10, inner=2, k=4, eps=1e-3)
    rows = np.concatenate([qsim.run(qsim.plan_stages(inputs.random_brick(14, 6, 300 + s), collect=1, **kw))
                           .training_data() for s in range(3)])
    qsim.predictor_train(rows, epochs=30, batch=64, lr=3e-3, seed=5)
    circuits = [inputs.random_brick(14, 8, 21), inputs.qft_rz_cx(13, 1, 4), inputs.ghz(12),
                inputs.random_brick(13, 6, 22)]
    plans = []
    for i, c in enumerate(circuits):
        if i % 2 == 0:  # learned sizing; the first margin forces every block through the exact re-encode
            plans.append(qsim.plan_stages(c, sizing=qsim.SIZING_PREDICT, predictor_margin=(-0.9, 0.25)[i // 2],
                                          **kw))
        else:
            plans.append(qsim.plan_stages(c, **kw))
    states, _ = qsim.run_batch(plans)
    for c, p, st in zip(circuits, plans, states):
        nblocks = 1 << (c.n - p.cfg.m)
        ref = qsim.run(qsim.plan_stages(c, **kw))
        assert streams_of(ref, nblocks) == streams_of(st, nblocks)
    assert states[0].stats.overflow_blocks > 0


def test_batch_bounded_wait_reports_timeout():
    plans = [p for _, p in batch_plans(5, 3, qsim.PREC_FP32)]
    c = inputs.random_brick(12, 4, 1)
    cfg = qsim.default_config(m=9, inner=2, k=4)
    cfg.reserved[0] = 1  # one dependency wait of this circuit is never satisfied
    stalled = qsim.Plan(c.n, c.gates, cfg)
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch(plans + [stalled])
    assert ei.value.code == qsim.E_TIMEOUT
    states, _ = qsim.run_batch(plans)  # the context is still usable
    assert len(states) == len(plans)


def test_batch_rejects_malformed():
    a = qsim.plan_stages(inputs.ghz(10), m=8, k=4)
    b = qsim.plan_stages(inputs.ghz(11), m=8, k=4, prec=qsim.PREC_TF32)
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch([a, b])  # mixed precision
    assert ei.value.code == qsim.E_INVALID
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch([])
    assert ei.value.code == qsim.E_INVALID
    wide = qsim.plan_stages(inputs.random_brick(12, 2, 1), m=9, k=6)
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch([a, wide])  # the persistent kernel fuses at most 5 qubits
    assert ei.value.code == qsim.E_INVALID
    raw = qsim.plan_stages(inputs.ghz(10), m=8, k=4, codec=qsim.CODEC_NONE)
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run_batch([raw])
    assert ei.value.code == qsim.E_INVALID
