"""Sharded runs through the C ABI (qsim_shard_*) on one GPU: the ranks of a 2- or 4-rank run are emulated one
after another in this process (each rank's stage is a separate set of launches; no kernel waits on another
rank), blocks that change owner are exported from one rank's store and imported into another's, and after the
last stage every block is gathered on rank 0. Each block's stream must equal, byte for byte, the stream the
unsharded qsim_run stores: sharding changes where an SV group is run, not what it computes. Also: a stage run
with blocks out of place is refused, and blocks not on a rank read as missing."""
import numpy as np
import pytest

from paper_2410_14088_gb300 import inputs, qsim, shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [("random", 16, 9, 2, 1), ("qaoa", 16, 9, 2, 2), ("qft", 15, 8, 3, 2), ("random", 18, 10, 2, 2)]


def circuit(family, n):
    return {"random": lambda: inputs.random_brick(n, 8, 3), "qaoa": lambda: inputs.qaoa_maxcut(n, 3, 5),
            "qft": lambda: inputs.qft_rz_cx(n, 2, 9)}[family]()


def emulate(plan, r):
    """All 2^r ranks in turn; returns the rank runs, the blocks each holds and the number of blocks moved."""
    m = plan.cfg.m
    nblocks = 1 << (plan.n - m)
    rq = plan.shards(r)
    world = 1 << r
    runs = [qsim.ShardRun(plan, rq, r, k) for k in range(world)]
    held = [set(int(b) for b in shard.owned_blocks(nblocks, rq[0], m, k)) for k in range(world)]
    moved = 0
    for s in range(plan.nstages):
        if s and list(rq[s]) != list(rq[s - 1]):
            packets = []
            for k in range(world):
                for d, ids in shard.outgoing(sorted(held[k]), rq[s - 1], rq[s], m, k).items():
                    sizes, buf = runs[k].export(ids)
                    packets.append((d, ids, sizes, buf))
                    held[k] -= set(int(b) for b in ids)
                    moved += len(ids)
            for d, ids, sizes, buf in packets:
                runs[d].import_(ids, sizes, buf)
                held[d] |= set(int(b) for b in ids)
        for k in range(world):
            runs[k].stage(s)
    return runs, held, moved


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-n%d-m%d-i%d-r%d" % c)
def test_emulated_ranks_store_the_unsharded_streams(case):
    family, n, m, inner, r = case
    c = circuit(family, n)
    plan = qsim.plan_stages(c, m=m, inner=inner, k=4, eps=1e-3)
    ref = qsim.run(plan)
    runs, held, moved = emulate(plan, r)
    assert moved > 0
    for k in range(1, len(runs)):  # gather on rank 0
        ids = np.array(sorted(held[k]), dtype=np.uint64)
        sizes, buf = runs[k].export(ids)
        runs[0].import_(ids, sizes, buf)
    st = runs[0].finish()
    for b in range(1 << (n - m)):
        assert st.block_stream(b) == ref.block_stream(b), b
    idx = np.array([0, 5, (1 << n) - 1, 12345 % (1 << n)], dtype=np.uint64)
    np.testing.assert_array_equal(st.amplitudes(idx), ref.amplitudes(idx))


def test_stage_refused_with_blocks_out_of_place_and_missing_blocks_unreadable():
    c = circuit("random", 16)
    plan = qsim.plan_stages(c, m=9, inner=2, k=4, eps=1e-3)
    rq = plan.shards(1)
    changes = [s for s in range(1, plan.nstages) if list(rq[s]) != list(rq[s - 1])]
    assert changes
    run = qsim.ShardRun(plan, rq, 1, 0)
    for s in range(changes[0]):
        run.stage(s)
    with pytest.raises(qsim.QsimError):
        run.stage(changes[0])  # the exchange before this stage was skipped
    # a one-stage run on rank 1 of 2: blocks of rank 0 are not readable from rank 1's state
    one = qsim.plan_stages(inputs.Circuit(16, [inputs.H(0), inputs.H(9), inputs.CZ(9, 10)]), m=9, inner=2, k=4,
                           eps=1e-3)
    assert one.nstages == 1
    q = int(one.shards(1)[0][0])
    run = qsim.ShardRun(one, one.shards(1), 1, 1)
    run.stage(0)
    st = run.finish()
    assert st.block_stream(0) == b""                    # block 0 has bit 0 at the rank qubit: rank 0's
    assert len(st.block_stream(1 << (q - 9))) > 0       # rank 1's
