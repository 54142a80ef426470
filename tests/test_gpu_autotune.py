"""Autotuner: searches (m, k, inner, streams) by timing a circuit prefix,
returns a configuration inside the search space that runs the full circuit
correctly, and answers a repeated query from its cache without timing."""
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu


def test_autotune_space_cache_and_result():
    c = inputs.qft_rz_cx(20, 2, 3)
    qsim.autotune_cache_clear()
    kw = dict(m=(12, 14), k=(3, 5), inner=(2, 3), streams=(1, 2), prefix_gates=150, reps=1)
    best, secs, cand = qsim.autotune(c, **kw)
    assert 12 <= best.m <= 14 and 3 <= best.k <= 5 and 2 <= best.inner <= 3 and best.streams in (1, 2)
    assert cand >= 7 and secs > 0
    best2, _, cand2 = qsim.autotune(c, **kw)
    assert cand2 == 0
    assert (best2.m, best2.k, best2.inner, best2.streams) == (best.m, best.k, best.inner, best.streams)
    st = qsim.run(qsim.Plan(c.n, c.gates, best))
    assert st.fidelity(oracle.simulate(c)) >= 0.99


def test_autotune_rejects_empty_space():
    c = inputs.ghz(12)
    with pytest.raises(qsim.QsimError):
        qsim.autotune(c, m=(9, 8))


def test_autotune_working_vector_limit():
    # candidates whose working vector (m + inner bits) exceeds the limit are not timed
    c = inputs.qft_rz_cx(18, 1, 4)
    qsim.autotune_cache_clear()
    best, _, cand = qsim.autotune(c, m=(10, 16), k=(3, 5), inner=(2, 4), streams=(1,), prefix_gates=120, reps=1,
                                  max_working_log2=c.n - 2)
    assert best.m + best.inner <= c.n - 2 and cand >= 1
    with pytest.raises(qsim.QsimError):
        qsim.autotune(c, m=(12, 14), inner=(3, 4), max_working_log2=10)
