"""CPU ORACLE — test infrastructure only.

A plain, slow, obviously-correct CPU restatement of what the simulator
computes, used to check the CUDA path. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package. It shares no code with
the CUDA path; the two meet only in the seeded input generators
(`paper_2410_14088_gb300.inputs`), which hold none of the method's arithmetic.

Modules:
  * this file    — ctypes front end of qsim_oracle.c (state update, QSZ1 and
                   QSZR codecs, MLP) and the circuit-level drivers built on it;
  * partition.py — the paper's circuit partition (Algorithm 1, Sec. 4.1);
  * closed_forms.py — closed-form final states used as pins.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  simulate            pinned: Kronecker-product unitaries (n <= 8), GHZ, QFT via
                      FFT, the QFT+RZ+CX closed form, Grover closed form, norm.
  qsz_encode/decode   pinned: point-wise bound on every value, round trip equals
                      the quantised input, hand-assembled streams of the format
                      (tests/golden/), worst-case size formula, corruption checks.
  qszr_encode/decode  pinned: point-wise relative bound on every normal value
                      (Eq. 1-2), exact zeros and signs, the shift against its
                      defining inequality, a stream assembled by hand in the
                      test, sign-chunk elision lengths, idempotence, corruption.
  partition           pinned: invariants of Algorithm 1 plus hand-worked cases.
  mlp_*               pinned: central finite differences, closed-form linear case,
                      a closed form whose value needs the ReLU of both hidden
                      layers (|x| from relu(x) + relu(-x), rows with negative
                      pre-activations cleared, their gradients zero), Adam
                      against its published recurrence on a scalar.
  simulate_staged     pinned: a two-stage 5-qubit case worked by hand (stage cut,
                      grid step, the state stored after each stage), output on
                      the 2^e grid and different from simulate, the norm bound.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_apply_matrix.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
        L.oracle_apply_matrix.restype = ctypes.c_int
        L.oracle_apply_phaseflip.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
        L.oracle_apply_phaseflip.restype = ctypes.c_int
        L.oracle_init_basis.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
        L.oracle_init_basis.restype = None
        L.oracle_norm_sq.argtypes = [dp, ctypes.c_int]
        L.oracle_norm_sq.restype = ctypes.c_double
        L.oracle_inner_mixed.argtypes = [dp, fp, ctypes.c_int64, dp, dp]
        L.oracle_inner_mixed.restype = None
        L.oracle_qsz_step_exponent.argtypes = [ctypes.c_double, ip]
        L.oracle_qsz_step_exponent.restype = ctypes.c_int
        L.oracle_qsz_worst_case_bytes.argtypes = [ctypes.c_int]
        L.oracle_qsz_worst_case_bytes.restype = ctypes.c_uint64
        L.oracle_qsz_quantize.argtypes = [fp, ctypes.c_int64, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int32)]
        L.oracle_qsz_quantize.restype = ctypes.c_int
        L.oracle_qsz_encode.argtypes = [fp, ctypes.c_int, ctypes.c_double, u8p, ctypes.c_uint64, u64p]
        L.oracle_qsz_encode.restype = ctypes.c_int
        L.oracle_qsz_decode.argtypes = [u8p, ctypes.c_uint64, ctypes.c_int, fp]
        L.oracle_qsz_decode.restype = ctypes.c_int
        L.oracle_qszr_shift.argtypes = [ctypes.c_double, ip]
        L.oracle_qszr_shift.restype = ctypes.c_int
        L.oracle_qszr_worst_case_bytes.argtypes = [ctypes.c_int]
        L.oracle_qszr_worst_case_bytes.restype = ctypes.c_uint64
        L.oracle_qszr_quantize.argtypes = [fp, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), u8p]
        L.oracle_qszr_quantize.restype = ctypes.c_int
        L.oracle_qszr_encode.argtypes = [fp, ctypes.c_int, ctypes.c_double, u8p, ctypes.c_uint64, u64p]
        L.oracle_qszr_encode.restype = ctypes.c_int
        L.oracle_qszr_decode.argtypes = [u8p, ctypes.c_uint64, ctypes.c_int, fp]
        L.oracle_qszr_decode.restype = ctypes.c_int
        L.oracle_mlp_nparams.argtypes = []
        L.oracle_mlp_nparams.restype = ctypes.c_int
        L.oracle_mlp_forward.argtypes = [dp, dp, ctypes.c_int, dp]
        L.oracle_mlp_forward.restype = None
        L.oracle_mlp_loss_grad.argtypes = [dp, dp, dp, ctypes.c_int, dp]
        L.oracle_mlp_loss_grad.restype = ctypes.c_double
        L.oracle_adam_step.argtypes = [dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_adam_step.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


E_INVALID, E_CAPACITY, E_CORRUPT, E_RANGE = -1, -3, -4, -5

# --------------------------------------------------------------------------
# State-vector simulation (Sec. 2.1)
# --------------------------------------------------------------------------


def basis_state(n: int, basis: int = 0) -> np.ndarray:
    psi = np.empty(2 << n, dtype=np.float64)
    lib().oracle_init_basis(_ptr(psi, ctypes.c_double), n, basis)
    return psi


def apply_gate(psi: np.ndarray, n: int, gate) -> None:
    """Apply one inputs.Gate in place to psi (interleaved complex128)."""
    L = lib()
    if gate.phaseflip:
        rc = L.oracle_apply_phaseflip(_ptr(psi, ctypes.c_double), n, gate.basis)
    else:
        q = np.asarray(gate.qubits, dtype=np.int32)
        u = np.ascontiguousarray(gate.matrix, dtype=np.complex128).view(np.float64)
        rc = L.oracle_apply_matrix(_ptr(psi, ctypes.c_double), n, len(q),
                                   _ptr(q, ctypes.c_int), _ptr(u, ctypes.c_double))
    if rc:
        raise OracleError(rc, "apply_gate")


def simulate(circuit, psi: Optional[np.ndarray] = None) -> np.ndarray:
    """Final state (complex128, shape 2^n) of `circuit` from |init_basis>,
    gates applied one by one in circuit order."""
    n = circuit.n
    if psi is None:
        psi = basis_state(n, circuit.init_basis)
    for g in circuit.gates:
        apply_gate(psi, n, g)
    return psi.view(np.complex128)


def norm_sq(psi_c128: np.ndarray) -> float:
    p = np.ascontiguousarray(psi_c128).view(np.float64)
    n = int(round(math.log2(p.size // 2)))
    return lib().oracle_norm_sq(_ptr(p, ctypes.c_double), n)


def inner(a_c128: np.ndarray, b_c64: np.ndarray):
    """<a|b> with a complex128 and b complex64 (sum conj(a_i) b_i, FP64)."""
    a = np.ascontiguousarray(a_c128).view(np.float64)
    b = np.ascontiguousarray(b_c64).view(np.float32)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_inner_mixed(_ptr(a, ctypes.c_double), _ptr(b, ctypes.c_float), a.size // 2,
                             ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def fidelity(ideal_c128: np.ndarray, sim_c64: np.ndarray) -> float:
    """|<ideal|sim>| / (||ideal|| ||sim||): the fidelity of Sec. 5.3, taken
    un-squared and normalised (the paper leaves normalisation unstated)."""
    ip = inner(ideal_c128, sim_c64)
    na = math.sqrt(norm_sq(ideal_c128))
    nb = math.sqrt(float(np.sum(np.abs(sim_c64.astype(np.complex128)) ** 2)))
    return abs(ip) / (na * nb)


# --------------------------------------------------------------------------
# QSZ1 codec (scalar)
# --------------------------------------------------------------------------


def qsz_step_exponent(eb: float) -> int:
    e = ctypes.c_int()
    rc = lib().oracle_qsz_step_exponent(eb, ctypes.byref(e))
    if rc:
        raise OracleError(rc, "step_exponent")
    return e.value


def qsz_worst_case_bytes(m: int) -> int:
    return int(lib().oracle_qsz_worst_case_bytes(m))


def qsz_quantize(x: np.ndarray, e: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.empty(x.size, dtype=np.int32)
    rc = lib().oracle_qsz_quantize(_ptr(x, ctypes.c_float), x.size, e, _ptr(q, ctypes.c_int32))
    if rc:
        raise OracleError(rc, "quantize")
    return q


def qsz_encode(amps: np.ndarray, m: int, eb: float, cap: Optional[int] = None) -> bytes:
    """Encode 2^m interleaved complex64 amplitudes (float32 array of 2^(m+1))."""
    a = np.ascontiguousarray(amps, dtype=np.float32)
    if a.size != 2 << m:
        raise ValueError("block size mismatch")
    cap = qsz_worst_case_bytes(m) if cap is None else cap
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nb = ctypes.c_uint64()
    rc = lib().oracle_qsz_encode(_ptr(a, ctypes.c_float), m, eb, _ptr(out, ctypes.c_uint8), cap,
                                 ctypes.byref(nb))
    if rc:
        err = OracleError(rc, "encode")
        err.needed = nb.value
        raise err
    return out[: nb.value].tobytes()


def qsz_decode(stream: bytes, m: int) -> np.ndarray:
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    if buf.size == 0:
        buf = np.zeros(1, dtype=np.uint8)
    out = np.empty(2 << m, dtype=np.float32)
    rc = lib().oracle_qsz_decode(_ptr(buf, ctypes.c_uint8), len(stream), m, _ptr(out, ctypes.c_float))
    if rc:
        raise OracleError(rc, "decode")
    return out


def qsz_reconstruct(amps: np.ndarray, e: int) -> np.ndarray:
    """x' = q * 2^e for every component (what decode(encode(x)) returns)."""
    q = qsz_quantize(amps, e)
    return (q.astype(np.float64) * 2.0 ** e).astype(np.float32)


def qszr_shift(rel: float) -> int:
    """Quantisation shift k of the relative-bound codec (largest k with 2^(k-24) <= b_r / (1 + b_r))."""
    k = ctypes.c_int()
    rc = lib().oracle_qszr_shift(rel, ctypes.byref(k))
    if rc:
        raise OracleError(rc, "qszr_shift")
    return k.value


def qszr_worst_case_bytes(m: int) -> int:
    return int(lib().oracle_qszr_worst_case_bytes(m))


def qszr_quantize(x: np.ndarray, k: int):
    """(codes, signs) of every component under shift k."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.empty(x.size, dtype=np.int32)
    s = np.empty(x.size, dtype=np.uint8)
    rc = lib().oracle_qszr_quantize(_ptr(x, ctypes.c_float), x.size, k, _ptr(q, ctypes.c_int32),
                                    _ptr(s, ctypes.c_uint8))
    if rc:
        raise OracleError(rc, "qszr_quantize")
    return q, s


def qszr_encode(amps: np.ndarray, m: int, rel: float, cap: Optional[int] = None) -> bytes:
    """Encode 2^m interleaved complex64 amplitudes under the point-wise relative bound rel."""
    a = np.ascontiguousarray(amps, dtype=np.float32)
    if a.size != 2 << m:
        raise ValueError("block size mismatch")
    cap = qszr_worst_case_bytes(m) if cap is None else cap
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nb = ctypes.c_uint64()
    rc = lib().oracle_qszr_encode(_ptr(a, ctypes.c_float), m, rel, _ptr(out, ctypes.c_uint8), cap,
                                  ctypes.byref(nb))
    if rc:
        err = OracleError(rc, "qszr_encode")
        err.needed = nb.value
        raise err
    return out[: nb.value].tobytes()


def qszr_decode(stream: bytes, m: int) -> np.ndarray:
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    if buf.size == 0:
        buf = np.zeros(1, dtype=np.uint8)
    out = np.empty(2 << m, dtype=np.float32)
    rc = lib().oracle_qszr_decode(_ptr(buf, ctypes.c_uint8), len(stream), m, _ptr(out, ctypes.c_float))
    if rc:
        raise OracleError(rc, "qszr_decode")
    return out


# --------------------------------------------------------------------------
# Staged compressed simulation: Algorithm 1 stages, the stage's gates in FP64,
# then every block quantised with the codec step (what the compressed store
# holds after each stage).
# --------------------------------------------------------------------------


def simulate_staged(circuit, m: int, inner_size: int, eps: float, diag_exempt: bool = False):
    from .partition import partition
    n = circuit.n
    eb = eps * 2.0 ** (-n / 2.0)
    e = qsz_step_exponent(eb)
    stages = partition(circuit.gates, n, m, inner_size, diag_exempt)
    psi = basis_state(n, circuit.init_basis)
    # the initial store holds the basis state exactly (0 and 1 are on the grid)
    for st in stages:
        for gi in st.gate_indices:
            apply_gate(psi, n, circuit.gates[gi])
        f32 = psi.astype(np.float32)
        psi = qsz_reconstruct(f32, e).astype(np.float64)
    return psi.view(np.complex128), stages, e


# --------------------------------------------------------------------------
# MLP (float64)
# --------------------------------------------------------------------------

MLP_IN, MLP_H = 41, 64


def mlp_nparams() -> int:
    return lib().oracle_mlp_nparams()


def mlp_forward(p: np.ndarray, x: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    y = np.empty(x.shape[0], dtype=np.float64)
    lib().oracle_mlp_forward(_ptr(p, ctypes.c_double), _ptr(x, ctypes.c_double), x.shape[0],
                             _ptr(y, ctypes.c_double))
    return y


def mlp_loss_grad(p: np.ndarray, x: np.ndarray, t: np.ndarray):
    p = np.ascontiguousarray(p, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.empty_like(p)
    loss = lib().oracle_mlp_loss_grad(_ptr(p, ctypes.c_double), _ptr(x, ctypes.c_double),
                                      _ptr(t, ctypes.c_double), x.shape[0], _ptr(g, ctypes.c_double))
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays (t is 1-based)."""
    lib().oracle_adam_step(_ptr(p, ctypes.c_double), _ptr(np.ascontiguousarray(g), ctypes.c_double),
                           _ptr(m, ctypes.c_double), _ptr(v, ctypes.c_double), p.size, t, lr, beta1,
                           beta2, eps)
