"""Group sharding across ranks on the CPU (gloo): the planner's rank qubits (qsim_plan_shards) and the routing
of compressed block streams between stages (paper_2410_14088_gb300.shard), driven by an oracle stage runner.

Each rank holds the QSZ1 streams of the blocks it owns; per stage it decodes each of its SV groups, applies the
stage's gates in FP64 (the oracle's update on the group's working vector) and encodes the blocks again with the
oracle's encoder; where the rank qubits change it sends the blocks that change owner. The gathered store must
equal, byte for byte, the same procedure on one rank and the oracle's staged simulation (Algorithm 1 stages,
quantised after every stage) encoded block by block: the routing loses, duplicates or misplaces no block.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (family, n, m, inner, log2 ranks)
CASES = [("random", 12, 6, 2, 1), ("qft", 12, 6, 2, 1), ("qaoa", 12, 5, 2, 2), ("random", 11, 5, 3, 2)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _circuit(family, n):
    from paper_2410_14088_gb300 import inputs
    return {"random": lambda: inputs.random_brick(n, 6, 5), "qft": lambda: inputs.qft_rz_cx(n, 2, 3),
            "qaoa": lambda: inputs.qaoa_maxcut(n, 2, 4)}[family]()


def run_sharded(case, rank, world, dist_mod):
    """The staged run on this rank's groups; returns {block id: QSZ1 stream} of the blocks it holds at the end
    and the number of blocks it sent."""
    import oracle
    from paper_2410_14088_gb300 import inputs, qsim, shard

    family, n, m, inner, r = case
    c = _circuit(family, n)
    eps = 1e-2
    eb = eps * 2.0 ** (-n / 2)
    plan = qsim.plan_stages(c, m=m, inner=inner, k=4, eps=eps)
    rq = shard.rank_qubits(plan, r) if world > 1 else np.zeros((plan.nstages, 0), np.uint32)
    nblocks = 1 << (n - m)
    # initial store (Sec. 4.2): the block holding the basis state, zero blocks elsewhere
    store = {}
    for b in shard.owned_blocks(nblocks, rq[0], m, rank):
        blk = np.zeros(2 << m, np.float32)
        if int(b) == c.init_basis >> m:
            blk[2 * (c.init_basis & ((1 << m) - 1))] = 1.0
        store[int(b)] = oracle.qsz_encode(blk, m, eb)
    sent = 0
    for s, (first, count, inner_q) in enumerate(plan.stages()):
        if s > 0 and world > 1 and list(rq[s]) != list(rq[s - 1]):
            out = shard.outgoing(sorted(store), rq[s - 1], rq[s], m, rank)
            send = {d: [(int(b), torch.frombuffer(bytearray(store.pop(int(b))), dtype=torch.uint8)) for b in ids]
                    for d, ids in out.items()}
            sent += sum(len(v) for v in send.values())
            for bid, t in shard.exchange(send, dist_mod, world):
                assert bid not in store
                store[bid] = t.numpy().tobytes()
        # every group of the stage this rank holds: blocks sharing their outer bits
        inner_mask = sum(1 << (q - m) for q in inner_q)
        W = m + len(inner_q)
        qmap = {q: q for q in range(m)}
        qmap.update({q: m + t for t, q in enumerate(inner_q)})
        gates = [inputs.Gate(g.name, tuple(qmap[q] for q in g.qubits), g.params, g.matrix)
                 for g in c.gates[first:first + count]]
        for base in sorted({b & ~inner_mask for b in store}):
            ids = [base | sum(((v >> t) & 1) << (q - m) for t, q in enumerate(inner_q))
                   for v in range(1 << len(inner_q))]
            psi = np.concatenate([oracle.qsz_decode(store[b], m) for b in ids]).astype(np.float64)
            for g in gates:
                oracle.apply_gate(psi, W, g)
            for v, b in enumerate(ids):
                store[b] = oracle.qsz_encode(psi[(2 * v) << m:(2 * (v + 1)) << m].astype(np.float32), m, eb)
    return store, sent


def _worker(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        store, sent = run_sharded(case, rank, world, dist)
        q.put((rank, store, sent))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, repr(e), -1))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-n%d-m%d-i%d-r%d" % c)
def test_sharded_store_equals_single_rank_and_oracle(case):
    import oracle
    family, n, m, inner, r = case
    world = 1 << r
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(rk, world, port, case, q)) for rk in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    merged, total_sent = {}, 0
    for rank, store, sent in got:
        assert sent >= 0, store
        total_sent += sent
        assert not (set(store) & set(merged)), "a block held by two ranks"
        merged.update(store)
    nblocks = 1 << (n - m)
    assert sorted(merged) == list(range(nblocks))
    assert total_sent > 0  # the case's stages do move blocks
    single, _ = run_sharded(case, 0, 1, None)
    assert merged == single
    # and the staged oracle (Algorithm 1 stages, FP64 gates, quantised after every stage) block by block
    c = _circuit(family, n)
    staged, _, _ = oracle.simulate_staged(c, m, inner, 1e-2)
    flat = staged.astype(np.complex64).view(np.float32)
    eb = 1e-2 * 2.0 ** (-n / 2)
    for b in range(nblocks):
        assert merged[b] == oracle.qsz_encode(flat[(2 * b) << m:(2 * (b + 1)) << m], m, eb), b


def test_rank_qubits_stay_outside_inner_sets():
    from paper_2410_14088_gb300 import inputs, qsim
    c = inputs.qaoa_maxcut(20, 3, 2)
    for m, inner, r in ((12, 2, 1), (12, 3, 3), (14, 2, 4)):
        plan = qsim.plan_stages(c, m=m, inner=inner, k=4, eps=1e-3)
        rq = plan.shards(r)
        changes = 0
        for s, (_, _, inner_q) in enumerate(plan.stages()):
            assert len(set(rq[s])) == r
            assert all(m <= q < 20 and q not in inner_q for q in rq[s])
            if s:
                # a slot changes only when the stage takes its qubit as inner
                for j in range(r):
                    if rq[s][j] != rq[s - 1][j]:
                        assert rq[s - 1][j] in inner_q
                        changes += 1
        assert changes < plan.nstages * r


def test_too_many_ranks_rejected():
    from paper_2410_14088_gb300 import inputs, qsim
    plan = qsim.plan_stages(inputs.random_brick(10, 4, 1), m=7, inner=2, k=4, eps=1e-3)
    with pytest.raises(qsim.QsimError):
        plan.shards(2)  # 3 global qubits, 2 inner: one left
