"""Closed-form final states (test infrastructure): independent of the
gate-by-gate update, used to pin the oracle and, at sampled indices, the CUDA
path at full size.
"""
import math

import numpy as np


def bit_reverse(y: np.ndarray, n: int) -> np.ndarray:
    y = np.asarray(y, dtype=np.uint64)
    r = np.zeros_like(y)
    for b in range(n):
        r |= ((y >> np.uint64(b)) & np.uint64(1)) << np.uint64(n - 1 - b)
    return r


def ghz_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = psi[-1] = 1 / math.sqrt(2)
    return psi


def qft_basis_state(n: int, x: int) -> np.ndarray:
    """QFT of |x> without the final swaps: amplitude at rev(y) is
    2^(-n/2) exp(2 pi i x y / 2^n). Uses numpy's FFT: sum_y w^{xy}|y> is
    N * ifft of the unit vector e_x."""
    N = 1 << n
    e = np.zeros(N, dtype=np.complex128)
    e[x] = 1.0
    amp_y = np.fft.ifft(e) * N / math.sqrt(N)
    out = np.empty(N, dtype=np.complex128)
    out[bit_reverse(np.arange(N, dtype=np.uint64), n).astype(np.int64)] = amp_y
    return out


def qft_of_state(psi: np.ndarray) -> np.ndarray:
    """QFT (no swaps) of an arbitrary state: sqrt(N) * ifft, then bit reversal."""
    N = psi.size
    n = int(round(math.log2(N)))
    amp_y = np.fft.ifft(psi) * math.sqrt(N)
    out = np.empty(N, dtype=np.complex128)
    out[bit_reverse(np.arange(N, dtype=np.uint64), n).astype(np.int64)] = amp_y
    return out


def qft_rz_cx_amplitudes(n: int, x: int, rz_angles, idx: np.ndarray) -> np.ndarray:
    """Final amplitudes at indices `idx` of QFT|x> followed by layers of
    (RZ(a_l,q) on every qubit, then the CX ladder CX(0,1), CX(1,2), ...).

    The ladder maps basis |z> to |z'> with z'_j = z_0 xor ... xor z_j, so it
    is undone by z_j = z'_j xor z'_{j-1}. RZ(a) on qubit q multiplies by
    exp(i a (z_q - 1/2)). Walking the layers backwards from the final index
    accumulates the phases; the remaining index is rev(y) of the QFT output,
    whose amplitude is 2^(-n/2) exp(2 pi i x y / 2^n)."""
    z = np.asarray(idx, dtype=np.uint64).copy()
    phase = np.zeros(z.shape, dtype=np.float64)
    for angles in reversed(rz_angles):
        prev = z ^ ((z << np.uint64(1)) & np.uint64((1 << n) - 1))  # undo ladder
        for q in range(n):
            bit = ((prev >> np.uint64(q)) & np.uint64(1)).astype(np.float64)
            phase += angles[q] * (bit - 0.5)
        z = prev
    y = bit_reverse(z, n)
    # x*y mod 2^n in exact integers (Python ints for n up to 62)
    xy = np.array([(x * int(v)) % (1 << n) for v in y], dtype=np.float64)
    phase += 2 * math.pi * xy / float(1 << n)
    return np.exp(1j * phase) / math.sqrt(float(1 << n))


def grover_state(n: int, iterations: int, marked: int) -> np.ndarray:
    """After H^n and t iterations of -(2|s><s| - I)(I - 2|w><w|):
    (-1)^t [sin((2t+1)th) |w> + cos((2t+1)th)/sqrt(N-1) sum_{x != w} |x>],
    th = asin(N^-1/2)."""
    N = 1 << n
    th = math.asin(1 / math.sqrt(N))
    a = (2 * iterations + 1) * th
    sign = -1.0 if iterations % 2 else 1.0
    psi = np.full(N, sign * math.cos(a) / math.sqrt(N - 1), dtype=np.complex128)
    psi[marked] = sign * math.sin(a)
    return psi
