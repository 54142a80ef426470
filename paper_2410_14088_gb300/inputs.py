"""Seeded synthetic inputs: circuits (as gate lists with their unitaries) and
amplitude blocks.

This module is shared by the CPU oracle and the CUDA path. It holds no part of
the simulator's method (no partitioning, fusion, codec or state update): only
the pseudo-random draws and the textbook definitions of the gates that make up
the input circuits.

Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles as (u >> 11) * 2^-53. Draw
order is documented per generator below so the circuits are reproducible from
their seed alone.

Conventions (qubit q <-> bit q of the amplitude index, little-endian, as in the
paper's state-vector description, Sec. 2.1):
  * a gate acts on qubits q[0..nq-1]; q[0] is the least-significant bit of the
    gate matrix's row/column index;
  * U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]];
  * RZ(a) = diag(e^{-ia/2}, e^{ia/2}); RX(b) = exp(-i b X / 2);
  * RZZ(g) = exp(-i g Z(x)Z / 2); CP(f) = diag(1, 1, 1, e^{if});
  * CX(c -> t) is given with q = (c, t); CZ, H, X standard;
  * PHASEFLIP(basis) multiplies the single amplitude |basis> by -1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """splitmix64 stream; `next_u64` advances the state by the golden gamma."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, bound: int) -> int:
        """Integer in [0, bound) by rejection (no modulo bias)."""
        if bound <= 0:
            raise ValueError("bound must be positive")
        limit = (1 << 64) - ((1 << 64) % bound)
        while True:
            u = self.next_u64()
            if u < limit:
                return u % bound


def splitmix64_array(seed: int, count: int) -> np.ndarray:
    """`count` consecutive splitmix64 outputs as uint64, vectorised (same
    sequence as `SplitMix64(seed).next_u64()` called `count` times)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_array(seed: int, count: int) -> np.ndarray:
    return (splitmix64_array(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# --------------------------------------------------------------------------
# Gate definitions (textbook unitaries; inputs to the simulator)
# --------------------------------------------------------------------------

@dataclass
class Gate:
    name: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = None  # 2^nq x 2^nq complex128, None for PHASEFLIP
    phaseflip: bool = False
    basis: int = 0

    @property
    def nq(self) -> int:
        return len(self.qubits)

    @property
    def is_diagonal(self) -> bool:
        if self.phaseflip:
            return True
        m = self.matrix
        return bool(np.all(m[~np.eye(m.shape[0], dtype=bool)] == 0))


def mat_h():
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)


def mat_x():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def mat_u3(t, p, l):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -np.exp(1j * l) * s],
                     [np.exp(1j * p) * s, np.exp(1j * (p + l)) * c]], dtype=np.complex128)


def mat_rz(a):
    return np.diag([np.exp(-0.5j * a), np.exp(0.5j * a)]).astype(np.complex128)


def mat_rx(b):
    c, s = math.cos(b / 2), math.sin(b / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def mat_rzz(g):
    e0, e1 = np.exp(-0.5j * g), np.exp(0.5j * g)
    return np.diag([e0, e1, e1, e0]).astype(np.complex128)


def mat_cz():
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def mat_cp(f):
    return np.diag([1, 1, 1, np.exp(1j * f)]).astype(np.complex128)


def mat_cx():
    # qubits (control, target); index r = c + 2 t; swap |c=1,t=0> <-> |c=1,t=1>
    m = np.eye(4, dtype=np.complex128)
    m[[1, 3]] = m[[3, 1]]
    return m


def H(q):
    return Gate("h", (q,), (), mat_h())


def X(q):
    return Gate("x", (q,), (), mat_x())


def U3(q, t, p, l):
    return Gate("u3", (q,), (t, p, l), mat_u3(t, p, l))


def RZ(q, a):
    return Gate("rz", (q,), (a,), mat_rz(a))


def RX(q, b):
    return Gate("rx", (q,), (b,), mat_rx(b))


def RZZ(a, b, g):
    return Gate("rzz", (a, b), (g,), mat_rzz(g))


def CZ(a, b):
    return Gate("cz", (a, b), (), mat_cz())


def CP(a, b, f):
    return Gate("cp", (a, b), (f,), mat_cp(f))


def CX(c, t):
    return Gate("cx", (c, t), (), mat_cx())


def PHASEFLIP(basis, n):
    return Gate("phaseflip", tuple(range(n)), (), None, True, int(basis))


def dagger(g: Gate) -> Gate:
    if g.phaseflip:
        return g
    return Gate(g.name + "_dg", g.qubits, g.params, g.matrix.conj().T.copy())


# --------------------------------------------------------------------------
# Circuits
# --------------------------------------------------------------------------

@dataclass
class Circuit:
    n: int
    gates: List[Gate]
    init_basis: int = 0
    family: str = ""
    meta: dict = field(default_factory=dict)


def brick_pairs(n: int, layer: int):
    """Neighbour pairs of layer `layer` (0-based): even -> (0,1),(2,3),...;
    odd -> (1,2),(3,4),...; open chain."""
    start = layer % 2
    return [(a, a + 1) for a in range(start, n - 1, 2)]


def random_brick(n: int, depth: int, seed: int) -> Circuit:
    """Each layer: U3 on qubits 0..n-1 (angles drawn theta, phi, lambda per
    qubit, each uniform [0, 2pi)), then CZ on the layer's neighbour pairs."""
    rng = SplitMix64(seed)
    gates = []
    for layer in range(depth):
        for q in range(n):
            t = 2 * math.pi * rng.uniform()
            p = 2 * math.pi * rng.uniform()
            l = 2 * math.pi * rng.uniform()
            gates.append(U3(q, t, p, l))
        for a, b in brick_pairs(n, layer):
            gates.append(CZ(a, b))
    return Circuit(n, gates, 0, "random", {"depth": depth, "seed": seed})


def mirror_brick(n: int, half_depth: int, seed: int) -> Circuit:
    """`half_depth` random layers followed by their exact inverse; the ideal
    final state is |0...0>."""
    c = random_brick(n, half_depth, seed)
    inv = [dagger(g) for g in reversed(c.gates)]
    return Circuit(n, c.gates + inv, 0, "mirror", {"half_depth": half_depth, "seed": seed})


def qft_gates(n: int) -> List[Gate]:
    """QFT without the final swaps: for j = n-1 .. 0: H(j), then CP(pi/2^(j-k))
    on (k, j) for k = j-1 .. 0. Output amplitude index is bit-reversed."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(H(j))
        for k in range(j - 1, -1, -1):
            gates.append(CP(k, j, math.pi / (1 << (j - k))))
    return gates


def cx_ladder(n: int) -> List[Gate]:
    return [CX(a, a + 1) for a in range(n - 1)]


def qft_rz_cx(n: int, layers: int, seed: int) -> Circuit:
    """QFT of a seeded random basis state |x>, then `layers` x (RZ on every
    qubit, then a CX ladder). Draws: x = first u64 >> (64-n); then the RZ
    angles layer by layer, qubit 0..n-1, uniform [0, 2pi)."""
    rng = SplitMix64(seed)
    x = rng.next_u64() >> (64 - n)
    gates = qft_gates(n)
    angles = []
    for _ in range(layers):
        row = []
        for q in range(n):
            a = 2 * math.pi * rng.uniform()
            row.append(a)
            gates.append(RZ(q, a))
        angles.append(row)
        gates.extend(cx_ladder(n))
    return Circuit(n, gates, x, "qft_rz_cx", {"layers": layers, "seed": seed, "x": x,
                                                "rz_angles": angles})


def random_regular_graph(nv: int, degree: int, rng: SplitMix64):
    """Configuration model with restarts until the pairing is simple."""
    if (nv * degree) % 2:
        raise ValueError("nv * degree must be even")
    while True:
        stubs = [v for v in range(nv) for _ in range(degree)]
        # Fisher-Yates with splitmix draws
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for a, b in zip(stubs[0::2], stubs[1::2]):
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)


def qaoa_maxcut(nv: int, p: int, seed: int) -> Circuit:
    """QAOA MaxCut on a seeded random 3-regular graph: H on every qubit, then p
    x (RZZ(gamma) on every edge, RX(beta) on every qubit). Draws: the graph,
    then per layer gamma then beta, each uniform [0, pi]."""
    rng = SplitMix64(seed)
    edges = random_regular_graph(nv, 3, rng)
    gates = [H(q) for q in range(nv)]
    params = []
    for _ in range(p):
        gamma = math.pi * rng.uniform()
        beta = math.pi * rng.uniform()
        params.append((gamma, beta))
        gates.extend(RZZ(a, b, gamma) for a, b in edges)
        gates.extend(RX(q, beta) for q in range(nv))
    return Circuit(nv, gates, 0, "qaoa", {"edges": edges, "params": params, "seed": seed})


def ghz(n: int) -> Circuit:
    return Circuit(n, [H(0)] + cx_ladder(n), 0, "ghz", {})


def grover(n: int, iterations: int, marked: int) -> Circuit:
    """H on all qubits, then `iterations` x (PHASEFLIP(marked), H on all,
    PHASEFLIP(0), H on all). Each iteration is -(2|s><s| - I)(I - 2|w><w|)."""
    gates = [H(q) for q in range(n)]
    for _ in range(iterations):
        gates.append(PHASEFLIP(marked, n))
        gates.extend(H(q) for q in range(n))
        gates.append(PHASEFLIP(0, n))
        gates.extend(H(q) for q in range(n))
    return Circuit(n, gates, 0, "grover", {"iterations": iterations, "marked": marked})


def batch_circuits(seed: int, count: int = 64, nmin: int = 20, nmax: int = 30) -> List[Circuit]:
    """Batch of independent circuits: per circuit draw n ~ U{nmin..nmax}, a
    family in (ghz, qft, random depth 8, grover), then the family's own seed or
    parameters from the same stream."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = nmin + rng.below(nmax - nmin + 1)
        fam = rng.below(4)
        sub = rng.next_u64()
        if fam == 0:
            out.append(ghz(n))
        elif fam == 1:
            c = qft_rz_cx(n, 0, sub)
            c.family = "qft"
            out.append(c)
        elif fam == 2:
            out.append(random_brick(n, 8, sub))
        else:
            t = 3 + rng.below(4)
            marked = sub >> (64 - n)
            out.append(grover(n, t, marked))
    return out


# --------------------------------------------------------------------------
# Amplitude blocks for codec tests
# --------------------------------------------------------------------------

def gaussian_block(m: int, n_equiv: int, seed: int) -> np.ndarray:
    """2^m complex64 amplitudes, interleaved (re, im) float32, drawn complex
    Gaussian with variance 2^-n_equiv per amplitude (Porter-Thomas statistics
    of an n_equiv-qubit random state). Box-Muller on splitmix64 uniforms."""
    N = 1 << m
    u = uniform_array(seed, 2 * N)
    u1 = np.maximum(u[0::2], 1e-300)
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    sigma = math.sqrt(0.5 * 2.0 ** (-n_equiv))
    re = sigma * r * np.cos(2 * math.pi * u2)
    im = sigma * r * np.sin(2 * math.pi * u2)
    out = np.empty(2 * N, dtype=np.float32)
    out[0::2] = re
    out[1::2] = im
    return out


def smooth_block(m: int, n_equiv: int, seed: int) -> np.ndarray:
    """Flat magnitude 2^-n_equiv/2 with a slowly varying phase (QFT-like
    structure)."""
    N = 1 << m
    u = uniform_array(seed, 2)
    j = np.arange(N, dtype=np.float64)
    ph = 2 * math.pi * (u[0] + u[1] * j / N * 7.0)
    a = 2.0 ** (-n_equiv / 2)
    out = np.empty(2 * N, dtype=np.float32)
    out[0::2] = a * np.cos(ph)
    out[1::2] = a * np.sin(ph)
    return out


def sparse_block(m: int, nnz: int, seed: int) -> np.ndarray:
    """Mostly zero block with `nnz` random unit-scale amplitudes."""
    N = 1 << m
    rng = SplitMix64(seed)
    out = np.zeros(2 * N, dtype=np.float32)
    for _ in range(nnz):
        i = rng.below(N)
        out[2 * i] = rng.uniform() - 0.5
        out[2 * i + 1] = rng.uniform() - 0.5
    return out
