"""Circuit partition of Algorithm 1 (Sec. 4.1) — oracle (test infrastructure).

Greedy in-order scan: a gate joins the current stage unless the number of
distinct global qubits (qubits >= m, the paper's global index bits) used by
the stage plus the gate would exceed threshold = max(inner size, 2); then the
current stage is closed and a new one begins with the gate.

Readings where the paper is silent:
  * the gate counter starts at 0 and an empty stage is never emitted;
  * a non-diagonal gate whose own global qubits exceed the threshold cannot be
    placed in any stage: UnsupportedGate;
  * a diagonal gate only rescales amplitudes by a phase that depends on index
    bits, so it is block-local whatever its qubits; with diag_exempt it counts
    no global qubit, and without it, it counts its global qubits unless those
    alone exceed the threshold (then it is exempt, e.g. an n-qubit phase flip).
"""
from dataclasses import dataclass, field
from typing import List


class UnsupportedGate(ValueError):
    pass


@dataclass
class Stage:
    gate_indices: List[int] = field(default_factory=list)
    inner: List[int] = field(default_factory=list)  # ascending global qubits


def counted_global_qubits(gate, m, threshold, diag_exempt):
    glob = {q for q in gate.qubits if q >= m}
    if gate.is_diagonal and (diag_exempt or len(glob) > threshold):
        return set()
    if len(glob) > threshold:
        raise UnsupportedGate(f"gate {gate.name} on {gate.qubits} touches {len(glob)} global qubits")
    return glob


def partition(gates, n, m, inner_size, diag_exempt=False) -> List[Stage]:
    threshold = max(inner_size, 2)
    stages: List[Stage] = []
    cur: List[int] = []
    cur_glob = set()
    for i, g in enumerate(gates):
        gq = counted_global_qubits(g, m, threshold, diag_exempt)
        if cur and len(cur_glob | gq) > threshold:
            stages.append(Stage(cur, sorted(cur_glob)))
            cur, cur_glob = [], set()
        cur.append(i)
        cur_glob |= gq
    if cur:
        stages.append(Stage(cur, sorted(cur_glob)))
    return stages
