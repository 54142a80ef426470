"""Group sharding of the staged simulation over several ranks (one GPU each).

The SV groups of a stage are independent (Sec. 4.2), which is what lets the
paper spread a run over several GPUs (Sec. 5.8). With 2^r ranks, stage s deals
its groups by r rank qubits, global qubits outside the stage's inner set chosen
by the planner (qsim_plan_shards): block b belongs to the rank whose bit j is
the block's bit at rank qubit j, so a whole SV group sits on one rank and the
stage needs no communication. Between two stages whose rank qubits differ, each
rank sends the compressed streams of the blocks that change owner to their new
ranks: one all-to-all of variable-sized compressed blocks per such boundary
(sizes first, then the bytes), over torch.distributed — NCCL for device
tensors, gloo for host tensors.

This module holds the routing only: who owns which block when, which blocks move
at a boundary, and the exchange itself. It does no arithmetic on amplitudes.
"""
from typing import Dict, List, Sequence, Tuple

import numpy as np


def rank_qubits(plan, log2_ranks: int) -> np.ndarray:
    """Rank qubits of every stage, shape (nstages, log2_ranks) (qsim_plan_shards)."""
    return plan.shards(log2_ranks)


def block_owner(blocks, qubits: Sequence[int], m: int) -> np.ndarray:
    """Owner rank of each block id under the rank qubits `qubits` (bit j of the rank = the block's bit at
    qubit qubits[j]; a block id holds the index bits m.. of its amplitudes)."""
    b = np.asarray(blocks, dtype=np.uint64)
    owner = np.zeros(b.shape, dtype=np.int64)
    for j, q in enumerate(qubits):
        owner |= (((b >> np.uint64(int(q) - m)) & np.uint64(1)).astype(np.int64)) << j
    return owner


def owned_blocks(nblocks: int, qubits: Sequence[int], m: int, rank: int) -> np.ndarray:
    """Block ids that `rank` holds under the rank qubits `qubits`, ascending."""
    ids = np.arange(nblocks, dtype=np.uint64)
    return ids[block_owner(ids, qubits, m) == rank]


def outgoing(my_blocks, q_prev: Sequence[int], q_next: Sequence[int], m: int, rank: int) -> Dict[int, np.ndarray]:
    """Blocks this rank holds under q_prev that another rank holds under q_next: {destination: block ids}."""
    b = np.asarray(my_blocks, dtype=np.uint64)
    dst = block_owner(b, q_next, m)
    out = {}
    for d in np.unique(dst):
        if int(d) != rank:
            out[int(d)] = np.sort(b[dst == d])
    return out


def exchange(send: Dict[int, List[Tuple[int, "object"]]], dist, world: int, device="cpu") -> List[Tuple[int, "object"]]:
    """All-to-all of compressed block streams. send: {destination rank: [(block id, uint8 tensor), ...]};
    returns [(block id, uint8 tensor), ...] received from every other rank (tensors on `device`).
    Three all_to_all_single calls: block counts, (block id, bytes) headers, then the concatenated bytes."""
    import torch

    rank = dist.get_rank()
    counts = torch.zeros(world, dtype=torch.int64, device=device)
    for d, items in send.items():
        if d != rank:
            counts[d] = len(items)
    rcounts = torch.empty_like(counts)
    dist.all_to_all_single(rcounts, counts)
    sc, rc = counts.tolist(), rcounts.tolist()
    # headers: (block id, stream bytes) per block, in destination order
    hdr = []
    for d in range(world):
        for bid, t in (send.get(d, []) if d != rank else []):
            hdr += [int(bid), int(t.numel())]
    hsend = torch.tensor(hdr if hdr else [0], dtype=torch.int64, device=device)[: len(hdr)]
    hrecv = torch.empty(2 * sum(rc), dtype=torch.int64, device=device)
    dist.all_to_all_single(hrecv, hsend, [2 * x for x in rc], [2 * x for x in sc])
    hr = hrecv.view(-1, 2).tolist() if hrecv.numel() else []
    # payload
    parts, sbytes = [], []
    for d in range(world):
        items = send.get(d, []) if d != rank else []
        nb = 0
        for _, t in items:
            parts.append(t.reshape(-1).to(device=device, dtype=torch.uint8))
            nb += int(t.numel())
        sbytes.append(nb)
    psend = torch.cat(parts) if parts else torch.empty(0, dtype=torch.uint8, device=device)
    rbytes, k = [], 0
    for d in range(world):
        rbytes.append(sum(h[1] for h in hr[k:k + rc[d]]))
        k += rc[d]
    precv = torch.empty(sum(rbytes), dtype=torch.uint8, device=device)
    dist.all_to_all_single(precv, psend, rbytes, sbytes)
    out, pos = [], 0
    for bid, nb in hr:
        out.append((int(bid), precv[pos:pos + nb]))
        pos += nb
    return out


def run_sharded(plan, log2_ranks: int, dist=None, stream=None):
    """This rank's part of a sharded run: one process per GPU, torch.distributed initialised (NCCL for the
    device tensors exchanged here), world size 2^log2_ranks; with dist None, one rank (log2_ranks 0).
    Stages run over this rank's SV groups (qsim_shard_stage); before a stage whose rank qubits differ from the
    previous stage's, the blocks that change owner are exported, exchanged and imported. Returns (the state
    handle of the blocks on this rank after the last stage, the number of blocks this rank sent)."""
    import torch

    from . import qsim

    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    if world != 1 << log2_ranks:
        raise ValueError("world size %d is not 2^%d" % (world, log2_ranks))
    m = plan.cfg.m
    nblocks = 1 << (plan.n - m)
    rq = plan.shards(log2_ranks) if log2_ranks else np.zeros((plan.nstages, 0), np.uint32)
    run = qsim.ShardRun(plan, rq, log2_ranks, rank, stream)
    held = set(int(b) for b in owned_blocks(nblocks, rq[0], m, rank)) if plan.nstages else set()
    sent = 0
    for s in range(plan.nstages):
        if s and list(rq[s]) != list(rq[s - 1]):
            send = {}
            for d, ids in outgoing(sorted(held), rq[s - 1], rq[s], m, rank).items():
                sizes, buf = run.export(ids)
                parts, o = [], 0
                for b, nb in zip(ids, sizes):
                    parts.append((int(b), buf[o:o + int(nb)]))
                    o += int(nb)
                send[d] = parts
                held -= set(int(b) for b in ids)
                sent += len(ids)
            recv = exchange(send, dist, world, device="cuda")
            if recv:
                ids = [b for b, _ in recv]
                run.import_(ids, [int(t.numel()) for _, t in recv], torch.cat([t for _, t in recv]))
                held |= set(ids)
        run.stage(s)
    return run.finish(), sent
