"""Pins for the Algorithm 1 oracle (Sec. 4.1): hand-worked cuts and the
invariants the algorithm guarantees."""
import pytest

from oracle.partition import UnsupportedGate, partition
from paper_2410_14088_gb300 import inputs


def idx(stages):
    return [s.gate_indices for s in stages]


def test_hand_worked_cuts():
    # n = 6, m = 2 (local qubits 0, 1; global 2..5), inner 2 -> threshold 2.
    H, CX = inputs.H, inputs.CX
    g = [H(0), H(3), CX(3, 5), H(1), CX(2, 4), H(4), CX(0, 1), CX(5, 2), H(2)]
    st = partition(g, 6, 2, 2)
    # {3}, {3,5} ok, H(1) local, CX(2,4) -> {2,3,4,5} cut; {2,4}; H(4) ok; CX(0,1) local;
    # CX(5,2) -> {2,4,5} cut; {2,5}; H(2) ok
    assert idx(st) == [[0, 1, 2, 3], [4, 5, 6], [7, 8]]
    assert [s.inner for s in st] == [[3, 5], [2, 4], [2, 5]]


def test_threshold_is_at_least_two():
    H, CX = inputs.H, inputs.CX
    g = [CX(4, 5), H(4), H(3)]
    st0 = partition(g, 6, 2, 0)
    st1 = partition(g, 6, 2, 1)
    assert idx(st0) == idx(st1) == [[0, 1], [2]]
    st3 = partition(g, 6, 2, 3)
    assert idx(st3) == [[0, 1, 2]]


def test_local_only_circuit_is_one_stage():
    c = inputs.random_brick(8, 5, 1)
    st = partition(c.gates, 8, 8, 2)
    assert len(st) == 1 and st[0].inner == []


def test_unsupported_and_diagonal_exemption():
    big = inputs.Gate("ccx_like", (3, 4, 5), (), inputs.np.kron(inputs.np.eye(4), inputs.mat_x()))
    with pytest.raises(UnsupportedGate):
        partition([big], 6, 2, 2)
    pf = inputs.PHASEFLIP(5, 6)  # n-qubit diagonal: always block-local
    st = partition([inputs.H(2), pf, inputs.H(3)], 6, 2, 2)
    assert idx(st) == [[0, 1, 2]] and st[0].inner == [2, 3]
    # a 2-qubit diagonal counts its globals unless diag_exempt
    g = [inputs.CZ(2, 3), inputs.CZ(4, 5)]
    assert len(partition(g, 6, 2, 2)) == 2
    assert len(partition(g, 6, 2, 2, diag_exempt=True)) == 1


@pytest.mark.parametrize("circ,m,inner", [
    (inputs.qft_rz_cx(12, 2, 3), 8, 2),
    (inputs.random_brick(12, 6, 4), 7, 3),
    (inputs.qaoa_maxcut(12, 2, 5), 6, 4),
])
def test_invariants(circ, m, inner):
    st = partition(circ.gates, circ.n, m, inner)
    flat = [i for s in st for i in s.gate_indices]
    assert flat == list(range(len(circ.gates)))            # order preserved, nothing lost
    thr = max(inner, 2)
    for s in st:
        assert s.gate_indices and len(s.inner) <= thr
        for i in s.gate_indices:
            assert {q for q in circ.gates[i].qubits if q >= m} <= set(s.inner)
    # greedy maximality: the first gate of every later stage would overflow the previous one
    for a, b in zip(st, st[1:]):
        first = {q for q in circ.gates[b.gate_indices[0]].qubits if q >= m}
        assert len(set(a.inner) | first) > thr


def test_qft33_stage_count_monotone_in_inner():
    g = inputs.qft_gates(33)
    counts = [len(partition(g, 33, 24, i)) for i in (2, 3, 4, 5)]
    assert all(x >= y for x, y in zip(counts, counts[1:]))
