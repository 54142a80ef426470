"""Learned size predictor on the GPU: forward, loss gradient and Adam kernels
against the float64 CPU oracle; training on sizes logged by exact-sizing
runs; predictor sizing gives byte-identical final streams, including when
every reservation is forced too small (overflow re-encode path); and the
trained predictor's reservations against the exact sizes and the worst case."""
import numpy as np
import pytest

import oracle
from paper_2410_14088_gb300 import inputs, qsim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rand_params(seed, scale=0.3):
    return ((inputs.uniform_array(seed, qsim.MLP_PARAMS) - 0.5) * scale)


def test_forward_matches_oracle():
    p = rand_params(1)
    x = inputs.uniform_array(2, 300 * 41).reshape(300, 41)
    want = oracle.mlp_forward(p, x)
    pd = torch.tensor(p, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    got = qsim.mlp_forward(pd, xd).cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-4 * max(1.0, np.max(np.abs(want)))
    got16 = qsim.mlp_forward(pd, xd, bf16=True).cpu().numpy()
    assert np.max(np.abs(got16 - want)) <= 2e-2 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("batch", [1, 37, 64, 200])
def test_gradient_matches_oracle(batch):
    p = rand_params(3)
    x = inputs.uniform_array(4, batch * 41).reshape(batch, 41)
    t = inputs.uniform_array(5, batch) * 2 - 1
    loss_w, g_w = oracle.mlp_loss_grad(p, x, t)
    pd = torch.tensor(p, dtype=torch.float32, device="cuda")
    loss, g = qsim.mlp_loss_grad(pd, torch.tensor(x, dtype=torch.float32, device="cuda"),
                                 torch.tensor(t, dtype=torch.float32, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_w) <= 1e-4 * max(1.0, abs(loss_w))
    assert np.linalg.norm(g - g_w) <= 1e-4 * max(1e-3, np.linalg.norm(g_w))


def test_adam_matches_oracle():
    p = rand_params(6)
    g = rand_params(7)
    pd = torch.tensor(p, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    md, vd = torch.zeros_like(pd), torch.zeros_like(pd)
    m, v = np.zeros_like(p), np.zeros_like(p)
    for t in (1, 2, 3):
        qsim.adam_step(pd, gd, md, vd, t, lr=1e-2)
        oracle.adam_step(p, g, m, v, t, lr=1e-2)
    assert np.max(np.abs(pd.cpu().numpy() - p)) <= 1e-5


def collect_rows(circuits, **kw):
    rows = []
    for c in circuits:
        st = qsim.run(qsim.plan_stages(c, collect=1, **kw))
        rows.append(st.training_data())
    return np.concatenate(rows)


def test_train_and_predict_identical_streams():
    kw = dict(m=10, inner=2, k=4, eps=1e-3)
    train = [inputs.random_brick(16, 6, 100 + s) for s in range(3)] + [inputs.qft_rz_cx(16, 2, 101)]
    rows = collect_rows(train, **kw)
    assert rows.shape[1] == qsim.TRAIN_ROW and rows.shape[0] > 100
    assert np.all(np.isfinite(rows))
    loss = qsim.predictor_train(rows, epochs=40, batch=64, lr=3e-3, seed=100)
    assert loss < 0.05  # 0.5 * mean squared log2-size residual
    c = inputs.random_brick(16, 8, 0)  # evaluation seed, not in training
    exact = qsim.run(qsim.plan_stages(c, **kw))
    pred = qsim.run(qsim.plan_stages(c, sizing=qsim.SIZING_PREDICT, predictor_margin=0.25, **kw))
    for b in range(64):
        assert exact.block_stream(b) == pred.block_stream(b)
    # forced under-estimate: every block overflows and is re-encoded exactly
    under = qsim.run(qsim.plan_stages(c, sizing=qsim.SIZING_PREDICT, predictor_margin=-0.9, **kw))
    assert under.stats.overflow_blocks > 0
    for b in range(64):
        assert exact.block_stream(b) == under.block_stream(b)
    # what the prediction buys, against exact sizing: each slot is reserved before its block is encoded, and the
    # reservation stays within 1.6x of the exact stream sizes (exact sizing learns them only from a pass over the
    # block); against the paper's reactive answer, reserving the worst case, it saves most of the space
    worst = qsim.worst_case_bytes(10) * 64
    exact_store = exact.stats.peak_store_bytes
    assert exact.stats.peak_reserved_bytes >= exact_store
    print(f"\nreserved: predicted {pred.stats.peak_reserved_bytes / exact_store:.3f}x the exact store, worst case "
          f"{worst / exact_store:.3f}x; overflows {pred.stats.overflow_blocks} of {pred.stats.blocks_encoded}")
    assert pred.stats.peak_reserved_bytes <= 1.6 * exact_store
    assert pred.stats.peak_reserved_bytes < 0.6 * worst
    assert pred.stats.overflow_blocks <= 0.2 * pred.stats.blocks_encoded


def test_predictor_set_get_roundtrip():
    p = rand_params(9).astype(np.float32)
    qsim.predictor_set(p)
    np.testing.assert_array_equal(qsim.predictor_get(), p)
