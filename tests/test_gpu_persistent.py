"""Persistent stage kernel (one launch per stage over a queue of work items,
optionally the stage loop captured into one CUDA graph): byte-identical
compressed state to the stream engine, with exact and learned sizing, all
gate precisions, dense ops on tcgen05 (TF32 widths 3-6, split BF16 widths
3-5), and a bounded
dependency wait that ends the run with QSIM_E_TIMEOUT instead of hanging."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu


def streams_of(st, nblocks):
    return [st.block_stream(b) for b in range(nblocks)]


@pytest.mark.parametrize("prec", [qsim.PREC_FP32, qsim.PREC_TF32, qsim.PREC_BF16X3], ids=["fp32", "tf32", "bf16x3"])
@pytest.mark.parametrize("graph", [0, 1])
def test_persistent_matches_streams(prec, graph):
    c = inputs.random_brick(18, 8, 2)
    kw = dict(m=11, inner=2, k=5, eps=1e-3, prec=prec)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=graph, **kw))
    assert streams_of(ref, 128) == streams_of(per, 128)
    assert per.fidelity(oracle.simulate(c)) >= 0.99
    assert abs(per.stats.norm_sq - ref.stats.norm_sq) < 1e-6


def test_persistent_qft_large_groups():
    # 2^22-amplitude working vectors (several tiles per pass), leading phase ops, diagonal-only stages
    c = inputs.qft_rz_cx(24, 2, 5)
    kw = dict(m=20, inner=2, k=5, eps=1e-3)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=1, **kw))
    assert streams_of(ref, 16) == streams_of(per, 16)


def test_persistent_with_learned_sizing():
    kw = dict(m=10, inner=2, k=4, eps=1e-3)
    rows = np.concatenate([qsim.run(qsim.plan_stages(inputs.random_brick(16, 6, 200 + s), collect=1, **kw))
                           .training_data() for s in range(3)])
    qsim.predictor_train(rows, epochs=30, batch=64, lr=3e-3, seed=7)
    c = inputs.random_brick(16, 8, 3)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    for margin in (0.25, -0.9):  # the second forces every block through the exact re-encode
        per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, sizing=qsim.SIZING_PREDICT,
                                        predictor_margin=margin, **kw))
        assert streams_of(ref, 64) == streams_of(per, 64)
    assert per.stats.overflow_blocks > 0


def test_persistent_bounded_wait_reports_timeout():
    c = inputs.random_brick(16, 4, 1)
    cfg = qsim.default_config(m=10, inner=2, k=4, mode=qsim.MODE_PERSISTENT)
    cfg.reserved[0] = 1
    with pytest.raises(qsim.QsimError) as ei:
        qsim.run(qsim.Plan(c.n, c.gates, cfg))
    assert ei.value.code == qsim.E_TIMEOUT
    # the context is still usable
    st = qsim.run(qsim.plan_stages(c, m=10, inner=2, k=4, mode=qsim.MODE_PERSISTENT))
    assert st.fidelity(oracle.simulate(c)) >= 0.99


def test_persistent_k6_only_on_tcgen05_tf32():
    # width-6 ops in the persistent kernel exist only in the TF32 tcgen05 form; the others are rejected at planning
    c = inputs.random_brick(16, 2, 1)
    for kw in (dict(), dict(prec=qsim.PREC_TF32), dict(prec=qsim.PREC_BF16X3, tcgen05=1)):
        with pytest.raises(qsim.QsimError) as ei:
            qsim.plan_stages(c, m=10, k=6, mode=qsim.MODE_PERSISTENT, **kw)
        assert ei.value.code == qsim.E_INVALID
    qsim.plan_stages(c, m=10, k=6, mode=qsim.MODE_PERSISTENT, prec=qsim.PREC_TF32, tcgen05=1)


def test_persistent_tcgen05_width6_matches_streams():
    # TF32 width-6 ops on tcgen05 inside the persistent kernel: the stream engine's MMAs, the same streams
    c = inputs.random_brick(18, 8, 3)
    kw = dict(m=12, inner=2, k=6, eps=1e-3, prec=qsim.PREC_TF32, tcgen05=1)
    plan = qsim.plan_stages(c, **kw)
    assert any(op["type"] == 0 and op["nq"] == 6 for s in range(plan.nstages) for op in plan.stage_ops(s))
    ref = qsim.run(plan)
    for graph in (0, 1):
        per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=graph, **kw))
        assert streams_of(ref, 64) == streams_of(per, 64)
    assert per.fidelity(oracle.simulate(c)) >= 0.99


@pytest.mark.parametrize("k", [3, 4, 5])
def test_persistent_tcgen05_bf16x3_matches_streams(k):
    # split-BF16 dense ops (widths 3-5) on tcgen05 inside the persistent kernel: the same streams as the stream engine
    c = inputs.random_brick(18, 8, 4)
    kw = dict(m=11, inner=2, k=k, eps=1e-3, prec=qsim.PREC_BF16X3, tcgen05=1)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=1, **kw))
    assert streams_of(ref, 128) == streams_of(per, 128)
    assert per.fidelity(oracle.simulate(c)) >= 0.99


@pytest.mark.parametrize("k", [3, 4, 5])
def test_persistent_tcgen05_matches_streams(k):
    # TF32 dense ops of width 3..5 on tcgen05 inside the persistent kernel (TMEM and the MMA mbarrier held per CTA
    # for the launch): the same MMAs as the stream engine's tcgen05 form, so the same streams byte for byte
    c = inputs.random_brick(18, 8, 2)
    kw = dict(m=11, inner=2, k=k, eps=1e-3, prec=qsim.PREC_TF32, tcgen05=1)
    ref = qsim.run(qsim.plan_stages(c, **kw))
    for graph in (0, 1):
        per = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, graph=graph, **kw))
        assert streams_of(ref, 128) == streams_of(per, 128)
        assert per.fidelity(oracle.simulate(c)) >= 0.99
    # and it differs from the warp-level MMA run only by TF32 rounding (both within the codec's grid of each other)
    warp = qsim.run(qsim.plan_stages(c, mode=qsim.MODE_PERSISTENT, **dict(kw, tcgen05=0)))
    assert abs(warp.fidelity(oracle.simulate(c)) - per.fidelity(oracle.simulate(c))) < 1e-3
