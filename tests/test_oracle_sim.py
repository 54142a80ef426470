"""Pins for the complex128 state-vector oracle (Sec. 2.1): full 2^n x 2^n
operators built from Kronecker products, closed forms (GHZ, QFT via FFT, the
QFT+RZ+CX phase formula, Grover) and norm preservation."""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_2410_14088_gb300 import inputs

I2 = np.eye(2, dtype=np.complex128)


def elementary(r, c):
    e = np.zeros((2, 2), dtype=np.complex128)
    e[r, c] = 1.0
    return e


def full_operator(gate, n):
    """sum_{r,c} U[r,c] (x)_{qubits high..low} (E_{r_j c_j} on gate qubit q[j], I elsewhere)."""
    N = 1 << n
    if gate.phaseflip:
        op = np.eye(N, dtype=np.complex128)
        op[gate.basis, gate.basis] = -1
        return op
    U = gate.matrix
    k = gate.nq
    op = np.zeros((N, N), dtype=np.complex128)
    for r in range(1 << k):
        for c in range(1 << k):
            if U[r, c] == 0:
                continue
            factors = []
            for qb in range(n - 1, -1, -1):
                if qb in gate.qubits:
                    j = gate.qubits.index(qb)
                    factors.append(elementary((r >> j) & 1, (c >> j) & 1))
                else:
                    factors.append(I2)
            t = factors[0]
            for f in factors[1:]:
                t = np.kron(t, f)
            op += U[r, c] * t
    return op


def dense_simulate(circuit):
    n = circuit.n
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[circuit.init_basis] = 1
    for g in circuit.gates:
        psi = full_operator(g, n) @ psi
    return psi


SMALL = [
    inputs.random_brick(6, 4, 7),
    inputs.qft_rz_cx(6, 2, 5),
    inputs.qaoa_maxcut(6, 2, 3),
    inputs.grover(5, 2, 19),
    inputs.ghz(7),
]


@pytest.mark.parametrize("circ", SMALL, ids=lambda c: c.family)
def test_against_kronecker_unitaries(circ):
    got = oracle.simulate(circ)
    want = dense_simulate(circ)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_reversed_qubit_order_matters():
    # a CX with swapped control/target must differ: the q[0] = low-bit convention is pinned
    n = 3
    c1 = inputs.Circuit(n, [inputs.H(0), inputs.CX(0, 2)])
    c2 = inputs.Circuit(n, [inputs.H(0), inputs.CX(2, 0)])
    a, b = oracle.simulate(c1), oracle.simulate(c2)
    assert np.max(np.abs(a - dense_simulate(c1))) <= 1e-12
    assert np.max(np.abs(a - b)) > 0.5
    assert abs(a[0b101] - 1 / math.sqrt(2)) < 1e-12


def test_u3_convention():
    # U3(pi/2, 0, pi) = H ; U3(pi, 0, pi) = X ; U3(0, 0, l) = diag(1, e^{il})
    np.testing.assert_allclose(inputs.mat_u3(math.pi / 2, 0, math.pi), inputs.mat_h(), atol=1e-15)
    np.testing.assert_allclose(inputs.mat_u3(math.pi, 0, math.pi), inputs.mat_x(), atol=1e-15)
    np.testing.assert_allclose(inputs.mat_u3(0, 0, 0.3), np.diag([1, np.exp(0.3j)]), atol=1e-15)


def test_ghz_closed_form():
    n = 14
    got = oracle.simulate(inputs.ghz(n))
    assert np.max(np.abs(got - cf.ghz_state(n))) <= 1e-12


@pytest.mark.parametrize("n,x", [(8, 0), (10, 613), (12, 4011)])
def test_qft_basis_closed_form(n, x):
    c = inputs.Circuit(n, inputs.qft_gates(n), x)
    got = oracle.simulate(c)
    assert np.max(np.abs(got - cf.qft_basis_state(n, x))) <= 1e-12


def test_qft_arbitrary_state_fft():
    n = 10
    u = inputs.uniform_array(99, 2 << n)
    start = (u[0::2] - 0.5) + 1j * (u[1::2] - 0.5)
    start /= np.linalg.norm(start)
    psi = start.astype(np.complex128).view(np.float64).copy()
    got = oracle.simulate(inputs.Circuit(n, inputs.qft_gates(n)), psi)
    assert np.max(np.abs(got - cf.qft_of_state(start))) <= 1e-12


def test_gate_count_qft33():
    # 33-qubit QFT: 33 H + 528 controlled phases; the paper's 2,673 gates
    # (Sec. 4.1) correspond to each controlled phase decomposed into 5 gates.
    g = inputs.qft_gates(33)
    nh = sum(1 for x in g if x.name == "h")
    ncp = len(g) - nh
    assert (nh, ncp) == (33, 528)
    assert nh + 5 * ncp == 2673


def test_qft_rz_cx_closed_form_full():
    n = 12
    c = inputs.qft_rz_cx(n, 4, 21)
    got = oracle.simulate(c)
    want = cf.qft_rz_cx_amplitudes(n, c.meta["x"], c.meta["rz_angles"], np.arange(1 << n))
    assert np.max(np.abs(got - want)) <= 1e-12


def test_qft_rz_cx_gate_count():
    c = inputs.qft_rz_cx(28, 4, 1)
    assert len(c.gates) == 626


def test_random_brick_gate_count():
    assert len(inputs.random_brick(16, 8, 0).gates) == 188
    assert len(inputs.random_brick(35, 14, 0).gates) == 728


def test_qaoa_gate_count_and_graph():
    c = inputs.qaoa_maxcut(32, 3, 0)
    assert len(c.gates) == 272
    deg = np.zeros(32, int)
    for a, b in c.meta["edges"]:
        deg[a] += 1
        deg[b] += 1
    assert np.all(deg == 3) and len(set(c.meta["edges"])) == 48


@pytest.mark.parametrize("n,t,marked", [(8, 3, 77), (10, 6, 1000)])
def test_grover_closed_form(n, t, marked):
    got = oracle.simulate(inputs.grover(n, t, marked))
    assert np.max(np.abs(got - cf.grover_state(n, t, marked))) <= 1e-12


def test_norm_preserved_and_mirror_identity():
    c = inputs.mirror_brick(12, 5, 4)
    got = oracle.simulate(c)
    assert abs(oracle.norm_sq(got) - 1.0) <= 1e-12
    assert abs(abs(got[0]) - 1.0) <= 1e-12
    c2 = inputs.random_brick(14, 6, 8)
    assert abs(oracle.norm_sq(oracle.simulate(c2)) - 1.0) <= 1e-12


def test_fidelity_definition():
    n = 8
    a = oracle.simulate(inputs.random_brick(n, 3, 1))
    b = (2.0 * a).astype(np.complex64)
    assert abs(oracle.fidelity(a, b) - 1.0) < 1e-6
    c = oracle.simulate(inputs.random_brick(n, 3, 2)).astype(np.complex64)
    f = oracle.fidelity(a, c)
    assert abs(f - abs(np.vdot(a, c.astype(np.complex128)))) < 1e-6


def test_staged_quantised_simulation_bound():
    # stage-wise quantisation error: ||psi_staged - psi|| <= sum over stages of
    # the per-component bound sqrt(2 * 2^n) * eb (unitary steps keep norms).
    c = inputs.random_brick(12, 6, 3)
    exact = oracle.simulate(c)
    staged, stages, e = oracle.simulate_staged(c, m=6, inner_size=2, eps=1e-2)
    eb = 1e-2 * 2.0 ** (-12 / 2)
    bound = len(stages) * math.sqrt(2 * (1 << 12)) * eb
    assert np.linalg.norm(staged - exact) <= bound
    assert oracle.fidelity(exact, staged.astype(np.complex64)) >= 0.99


def test_staged_hand_worked_two_stages():
    # n = 5, m = 2, inner 2: the global qubits are 2, 3, 4 and a stage may hold two of them, so
    # [U3(pi/3, 0, 0) on 2, H on 3] is stage 1 and [H on 4] stage 2 (Algorithm 1).
    # eps = 0.5: eb = 0.5 * 2^(-5/2) = 0.0884, 2 eb = 0.177, so e = -3 and the grid step is 1/8.
    # Stage 1 exact: cos(pi/6)/sqrt2 = 0.61237 at |0>, |8>; sin(pi/6)/sqrt2 = 0.35355 at |4>, |12>;
    #   stored: rint(4.899)/8 = 0.625 and rint(2.828)/8 = 0.375.
    # Stage 2 from the stored state: 0.625/sqrt2 * 8 = 3.536 -> 0.5, 0.375/sqrt2 * 8 = 2.121 -> 0.25.
    # Without the stage-1 quantisation the first value would be rint(3.464)/8 = 0.375, with a step of 1/16
    # it would be 0.4375 and with none 0.4330, so each of those mistakes changes the result.
    c = inputs.Circuit(5, [inputs.U3(2, math.pi / 3, 0.0, 0.0), inputs.H(3), inputs.H(4)])
    staged, stages, e = oracle.simulate_staged(c, m=2, inner_size=2, eps=0.5)
    assert e == -3
    assert [s.gate_indices for s in stages] == [[0, 1], [2]]
    want = np.zeros(32, np.complex128)
    want[[0, 8, 16, 24]] = 0.5
    want[[4, 12, 20, 28]] = 0.25
    assert np.array_equal(staged, want)


def test_staged_output_on_grid_and_not_the_exact_state():
    c = inputs.random_brick(10, 6, 12)
    staged, stages, e = oracle.simulate_staged(c, m=5, inner_size=2, eps=1e-2)
    assert len(stages) >= 2
    q = staged.view(np.float64) / 2.0 ** e
    assert np.array_equal(q, np.rint(q))
    exact = oracle.simulate(c)
    d = np.abs(staged - exact)
    assert d.max() > 0
    # each stage moves every component by at most half a step; the unitary stages keep 2-norms
    assert np.linalg.norm(staged - exact) <= len(stages) * math.sqrt(2 << 10) * 2.0 ** (e - 1)
