"""Python binding of libqsim (include/qsim.h): argument marshalling only.

Every step of the simulation runs inside libqsim's CUDA kernels; this module
converts Python gate lists, numpy arrays and torch CUDA tensors into the C
structs and pointers the library takes. PyTorch is used for device memory and
the current CUDA stream only. If the library is missing the import fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsim.so")

OK = 0
E_INVALID, E_NOMEM, E_CAPACITY, E_CORRUPT, E_RANGE, E_UNSUPPORTED, E_TIMEOUT, E_CUDA = -1, -2, -3, -4, -5, -6, -7, -8
ERROR_NAMES = {-1: "INVALID", -2: "NOMEM", -3: "CAPACITY", -4: "CORRUPT", -5: "RANGE", -6: "UNSUPPORTED",
               -7: "TIMEOUT", -8: "CUDA"}

GATE_DIAG, GATE_PHASEFLIP = 1, 2
PREC_FP32, PREC_TF32, PREC_BF16X3 = 0, 1, 2
MODE_STREAMS, MODE_PERSISTENT = 0, 1
CODEC_QSZ1, CODEC_NONE, CODEC_QSZR = 0, 1, 2
SIZING_EXACT, SIZING_PREDICT = 0, 1
REORDER_NONE, REORDER_STAGES, REORDER_PASSES, REORDER_PASSES_ALL = 0, 1, 2, 3


class QsimError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func}: QSIM_E_{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Gate(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("q", ctypes.c_uint32 * 6),
                ("basis", ctypes.c_uint64), ("u", ctypes.POINTER(ctypes.c_double))]


class Config(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint32), ("inner", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("prec", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("streams", ctypes.c_uint32),
                ("sizing", ctypes.c_uint32), ("diag_exempt", ctypes.c_uint32), ("codec", ctypes.c_uint32),
                ("graph", ctypes.c_uint32), ("tile_bits", ctypes.c_uint32), ("collect", ctypes.c_uint32),
                ("eps", ctypes.c_double), ("device_tier_cap_bytes", ctypes.c_uint64),
                ("init_basis", ctypes.c_uint64), ("predictor_margin", ctypes.c_double),
                ("reorder", ctypes.c_uint32), ("tcgen05", ctypes.c_uint32), ("reserved", ctypes.c_uint64 * 5)]


class PlanStats(ctypes.Structure):
    _fields_ = [("nstages", ctypes.c_uint64), ("ngates", ctypes.c_uint64), ("dense_ops", ctypes.c_uint64),
                ("diag_ops", ctypes.c_uint64), ("phaseflip_ops", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("max_working_log2", ctypes.c_uint64), ("plan_seconds", ctypes.c_double)]


class OpInfo(ctypes.Structure):
    _fields_ = [("type", ctypes.c_uint32), ("nq", ctypes.c_uint32), ("qubits", ctypes.c_uint32 * 8),
                ("ngates", ctypes.c_uint32), ("pass_", ctypes.c_uint32), ("quadratic", ctypes.c_uint32),
                ("reserved_", ctypes.c_uint32), ("basis", ctypes.c_uint64),
                ("u", ctypes.POINTER(ctypes.c_double)), ("qlist", ctypes.POINTER(ctypes.c_uint32))]


class Stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("err_norm_sum", ctypes.c_double), ("err_sq_total", ctypes.c_double),
                ("norm_sq", ctypes.c_double), ("nstages", ctypes.c_uint64), ("groups", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("peak_store_bytes", ctypes.c_uint64),
                ("peak_reserved_bytes", ctypes.c_uint64), ("final_store_bytes", ctypes.c_uint64),
                ("host_tier_peak_bytes", ctypes.c_uint64), ("overflow_blocks", ctypes.c_uint64),
                ("blocks_encoded", ctypes.c_uint64), ("fidelity_lower_bound", ctypes.c_double),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("seconds", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("alg_flops", ctypes.c_double)]


class TrainConfig(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("bf16_inference", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class TuneSpace(ctypes.Structure):
    _fields_ = [("m_min", ctypes.c_uint32), ("m_max", ctypes.c_uint32), ("k_min", ctypes.c_uint32),
                ("k_max", ctypes.c_uint32), ("inner_min", ctypes.c_uint32), ("inner_max", ctypes.c_uint32),
                ("streams_mask", ctypes.c_uint32), ("prefix_gates", ctypes.c_uint32), ("reps", ctypes.c_uint32),
                ("max_working_log2", ctypes.c_uint32)]


MLP_INPUTS, MLP_PARAMS, TRAIN_ROW = 41, 6913, 42

# every symbol include/qsim.h declares, with its ctypes signature
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_U32, _U64 = ctypes.c_uint32, ctypes.c_uint64
SIGNATURES = {
    "qsim_config_default": (None, [ctypes.POINTER(Config)]),
    "qsim_plan_stages": (ctypes.c_int, [_U32, ctypes.POINTER(Gate), _SZ, ctypes.POINTER(Config), ctypes.POINTER(_VP)]),
    "qsim_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(_SZ), ctypes.POINTER(_U32)]),
    "qsim_plan_stage_gates": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "qsim_plan_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(PlanStats)]),
    "qsim_plan_stage_ops": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(OpInfo)]),
    "qsim_plan_free": (None, [_VP]),
    "qsim_run": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_VP), ctypes.POINTER(Stats)]),
    "qsim_state_stage_stats": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                              ctypes.POINTER(ctypes.c_double)]),
    "qsim_amplitudes": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), _SZ, ctypes.POINTER(ctypes.c_float)]),
    "qsim_fidelity": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "qsim_state_norm": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "qsim_state_decompress": (ctypes.c_int, [_VP, _VP, _VP]),
    "qsim_state_block_stream": (ctypes.c_int, [_VP, _U64, _VP, _SZ, ctypes.POINTER(_SZ)]),
    "qsim_state_free": (None, [_VP]),
    "qsim_worst_case_bytes": (_SZ, [_U32]),
    "qsim_compress_block": (ctypes.c_int, [_VP, _U32, ctypes.c_double, _VP, _SZ, ctypes.POINTER(_SZ), _VP]),
    "qsim_plan_shards": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(_U32)]),
    "qsim_shard_begin": (ctypes.c_int, [_VP, ctypes.POINTER(_U32), _U32, _U32, _VP, ctypes.POINTER(_VP)]),
    "qsim_shard_stage": (ctypes.c_int, [_VP, _SZ]),
    "qsim_shard_block_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), _SZ, ctypes.POINTER(_U64)]),
    "qsim_shard_export": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), _SZ, _VP, _SZ]),
    "qsim_shard_import": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64), _SZ, _VP]),
    "qsim_shard_finish": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(Stats)]),
    "qsim_shard_free": (None, [_VP]),
    "qsim_compress_block_noalloc": (ctypes.c_int, [_VP, _U32, ctypes.c_double, _VP, _SZ, ctypes.POINTER(_SZ), _VP]),
    "qsim_decompress_block": (ctypes.c_int, [_VP, _SZ, _VP, _U32, _VP]),
    "qsim_compress_block_rel": (ctypes.c_int, [_VP, _U32, ctypes.c_double, _VP, _SZ, ctypes.POINTER(_SZ), _VP]),
    "qsim_worst_case_bytes_rel": (_SZ, [_U32]),
    "qsim_mlp_forward": (ctypes.c_int, [_VP, _VP, _SZ, _VP, ctypes.c_int, _VP]),
    "qsim_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, ctypes.POINTER(ctypes.c_float), _VP]),
    "qsim_adam_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _SZ, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_float, _VP]),
    "qsim_predictor_train": (ctypes.c_int, [_VP, _SZ, ctypes.POINTER(TrainConfig), ctypes.POINTER(ctypes.c_double)]),
    "qsim_predictor_set": (ctypes.c_int, [_VP, _SZ, ctypes.c_int]),
    "qsim_predictor_get": (ctypes.c_int, [_VP, _SZ]),
    "qsim_state_training_data": (ctypes.c_int, [_VP, _VP, _SZ, ctypes.POINTER(_SZ)]),
    "qsim_autotune": (ctypes.c_int, [_U32, ctypes.POINTER(Gate), _SZ, ctypes.POINTER(Config), ctypes.POINTER(TuneSpace),
                                     ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_U32)]),
    "qsim_autotune_cache_clear": (None, []),
    "qsim_profile_enable": (None, [ctypes.c_int]),
    "qsim_state_kernel_stats": (ctypes.c_int, [_VP, ctypes.POINTER(KernelStat), _SZ, ctypes.POINTER(_SZ)]),
    "qsim_run_batch": (ctypes.c_int, [ctypes.POINTER(_VP), _SZ, _VP, ctypes.POINTER(_VP), ctypes.POINTER(Stats),
                                      ctypes.POINTER(KernelStat)]),
    "qsim_last_error": (ctypes.c_char_p, []),
    "qsim_kernel_launch_count": (_U64, []),
    "qsim_alloc_count": (_U64, []),
    "qsim_release_cached_memory": (None, []),
}

_lib = None


def lib():
    """Load libqsim.so (built by paper_2410_14088_gb300.build). Raises if it
    is missing: the CUDA library is the only implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with paper_2410_14088_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, func: str):
    if rc != 0:
        raise QsimError(rc, func, lib().qsim_last_error().decode(errors="replace"))


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def profile_enable(on: bool = True):
    lib().qsim_profile_enable(1 if on else 0)


def launch_count() -> int:
    return int(lib().qsim_kernel_launch_count())


def alloc_count() -> int:
    """qsim_alloc_count: the library's device and pinned-host allocations in this process so far."""
    return int(lib().qsim_alloc_count())


def worst_case_bytes(m: int) -> int:
    return int(lib().qsim_worst_case_bytes(m))


def release_cached_memory():
    lib().qsim_release_cached_memory()


def default_config(**kw) -> Config:
    c = Config()
    lib().qsim_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


# --------------------------------------------------------------------------
# planning
# --------------------------------------------------------------------------

def marshal_gates(gates):
    """qsim_gate array for a list of inputs.Gate (matrices kept alive in the second return value)."""
    arr = (Gate * max(1, len(gates)))()
    mats = []
    for i, g in enumerate(gates):
        ga = arr[i]
        if getattr(g, "phaseflip", False):
            ga.nq = 0
            ga.flags = GATE_PHASEFLIP
            ga.basis = int(g.basis)
            ga.u = ctypes.POINTER(ctypes.c_double)()
        else:
            ga.nq = len(g.qubits)
            ga.flags = 0
            for j, q in enumerate(g.qubits):
                ga.q[j] = q
            u = np.ascontiguousarray(g.matrix, dtype=np.complex128).view(np.float64).ravel()
            mats.append(u)
            ga.u = u.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return arr, mats


class Plan:
    """Owns a qsim_plan handle (plus the gate matrices it was built from)."""

    def __init__(self, n: int, gates: Sequence, cfg: Config):
        self.n = n
        self.cfg = cfg
        arr, self._mats = marshal_gates(gates)
        h = ctypes.c_void_p()
        _check(lib().qsim_plan_stages(n, arr, len(gates), ctypes.byref(cfg), ctypes.byref(h)), "qsim_plan_stages")
        self.handle = h
        self.ngates = len(gates)

    def __del__(self):
        if getattr(self, "handle", None):
            lib().qsim_plan_free(self.handle)
            self.handle = None

    @property
    def nstages(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().qsim_plan_info(self.handle, ctypes.byref(n), None), "qsim_plan_info")
        return n.value

    def stages(self):
        """[(first_gate, count, inner_qubits)] per stage."""
        ns = self.nstages
        masks = (ctypes.c_uint32 * max(1, ns))()
        n = ctypes.c_size_t()
        _check(lib().qsim_plan_info(self.handle, ctypes.byref(n), masks), "qsim_plan_info")
        out = []
        for s in range(ns):
            f, c = ctypes.c_size_t(), ctypes.c_size_t()
            _check(lib().qsim_plan_stage_gates(self.handle, s, ctypes.byref(f), ctypes.byref(c)), "stage_gates")
            inner = [self.cfg.m + j for j in range(32) if (masks[s] >> j) & 1]
            out.append((f.value, c.value, inner))
        return out

    def stage_ops(self, stage: int):
        cnt = ctypes.c_size_t(0)
        _check(lib().qsim_plan_stage_ops(self.handle, stage, ctypes.byref(cnt), None), "qsim_plan_stage_ops")
        arr = (OpInfo * max(1, cnt.value))()
        _check(lib().qsim_plan_stage_ops(self.handle, stage, ctypes.byref(cnt), arr), "qsim_plan_stage_ops")
        ops = []
        for o in arr[: cnt.value]:
            d = {"type": o.type, "nq": o.nq, "qubits": tuple(o.qubits[: o.nq]), "ngates": o.ngates,
                 "pass": o.pass_, "quadratic": bool(o.quadratic), "basis": o.basis, "u": None}
            if o.type == 0:
                D = 1 << o.nq
                d["u"] = np.ctypeslib.as_array(o.u, shape=(2 * D * D,)).copy().view(np.complex128).reshape(D, D)
            elif o.type == 1:
                D = 1 << o.nq
                d["u"] = np.ctypeslib.as_array(o.u, shape=(2 * D,)).copy().view(np.complex128)
            elif o.type == 3:
                d["qubits"] = tuple(int(x) for x in np.ctypeslib.as_array(o.qlist, shape=(o.nq,)))
                d["u"] = np.ctypeslib.as_array(o.u, shape=(2 * (2 + 4 * (o.nq - 1)),)).copy().view(np.complex128)
            ops.append(d)
        return ops

    def shards(self, log2_ranks: int) -> np.ndarray:
        """qsim_plan_shards: rank qubits per stage, shape (nstages, log2_ranks)."""
        ns = self.nstages
        out = np.zeros((max(1, ns), max(1, log2_ranks)), dtype=np.uint32)
        _check(lib().qsim_plan_shards(self.handle, log2_ranks, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
               "qsim_plan_shards")
        return out[:ns, :log2_ranks]

    def stats(self) -> dict:
        s = PlanStats()
        _check(lib().qsim_plan_get_stats(self.handle, ctypes.byref(s)), "qsim_plan_get_stats")
        return {name: getattr(s, name) for name, _ in s._fields_}


def plan_stages(circuit_or_n, gates=None, cfg: Optional[Config] = None, **kw) -> Plan:
    if gates is None:
        c = circuit_or_n
        n, gates = c.n, c.gates
        kw.setdefault("init_basis", c.init_basis)
    else:
        n = circuit_or_n
    cfg = cfg if cfg is not None else default_config()
    for k, v in kw.items():
        setattr(cfg, k, v)
    return Plan(n, gates, cfg)


# --------------------------------------------------------------------------
# simulation and readout
# --------------------------------------------------------------------------

class State:
    def __init__(self, handle, n, m, stats: Stats, nstages: int):
        self.handle = handle
        self.n = n
        self.m = m
        self.stats = stats
        self.nstages = nstages

    def __del__(self):
        if getattr(self, "handle", None):
            lib().qsim_state_free(self.handle)
            self.handle = None

    def amplitudes(self, idx) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.uint64)
        out = np.empty(2 * idx.size, dtype=np.float32)
        _check(lib().qsim_amplitudes(self.handle, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), idx.size,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "qsim_amplitudes")
        return out.view(np.complex64)

    def fidelity(self, ref) -> float:
        """ref: numpy complex128 (host) or a torch complex128 CUDA tensor."""
        f = ctypes.c_double()
        if isinstance(ref, np.ndarray):
            r = np.ascontiguousarray(ref, dtype=np.complex128)
            ptr = ctypes.c_void_p(r.ctypes.data)
        else:
            r = ref.contiguous()
            ptr = ctypes.c_void_p(r.data_ptr())
        _check(lib().qsim_fidelity(self.handle, ptr, ctypes.byref(f)), "qsim_fidelity")
        return f.value

    def norm_sq(self) -> float:
        v = ctypes.c_double()
        _check(lib().qsim_state_norm(self.handle, ctypes.byref(v)), "qsim_state_norm")
        return v.value

    def decompress(self, out=None):
        """Whole state as a torch complex64 CUDA tensor (2^n amplitudes)."""
        import torch
        if out is None:
            out = torch.empty(1 << self.n, dtype=torch.complex64, device="cuda")
        _check(lib().qsim_state_decompress(self.handle, ctypes.c_void_p(out.data_ptr()), _stream_ptr()),
               "qsim_state_decompress")
        return out

    def block_stream(self, block: int) -> bytes:
        nb = ctypes.c_size_t()
        rc = lib().qsim_state_block_stream(self.handle, block, None, 0, ctypes.byref(nb))
        if rc not in (0, E_CAPACITY):
            _check(rc, "qsim_state_block_stream")
        buf = np.empty(max(1, nb.value), dtype=np.uint8)
        _check(lib().qsim_state_block_stream(self.handle, block, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                             ctypes.byref(nb)), "qsim_state_block_stream")
        return buf[: nb.value].tobytes()

    def training_data(self) -> np.ndarray:
        """Rows (features[41], target) logged by a run with collect=1."""
        n = ctypes.c_size_t()
        _check(lib().qsim_state_training_data(self.handle, None, 0, ctypes.byref(n)), "qsim_state_training_data")
        out = np.empty((max(1, n.value), TRAIN_ROW), dtype=np.float32)
        _check(lib().qsim_state_training_data(self.handle, ctypes.c_void_p(out.ctypes.data), n.value,
                                              ctypes.byref(n)), "qsim_state_training_data")
        return out[: n.value]

    def kernel_stats(self):
        cnt = ctypes.c_size_t()
        _check(lib().qsim_state_kernel_stats(self.handle, None, 0, ctypes.byref(cnt)), "qsim_state_kernel_stats")
        arr = (KernelStat * max(1, cnt.value))()
        _check(lib().qsim_state_kernel_stats(self.handle, arr, cnt.value, ctypes.byref(cnt)),
               "qsim_state_kernel_stats")
        return {k.name.decode(): {"launches": k.launches, "seconds": k.seconds, "alg_bytes": k.alg_bytes,
                                  "alg_flops": k.alg_flops} for k in arr[: cnt.value]}

    def stage_stats(self, stage: int):
        sb, rb, es = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
        _check(lib().qsim_state_stage_stats(self.handle, stage, ctypes.byref(sb), ctypes.byref(rb),
                                            ctypes.byref(es)), "qsim_state_stage_stats")
        return sb.value, rb.value, es.value


def run(plan: Plan, stream=None) -> State:
    h = ctypes.c_void_p()
    st = Stats()
    _check(lib().qsim_run(plan.handle, _stream_ptr(stream), ctypes.byref(h), ctypes.byref(st)), "qsim_run")
    return State(h, plan.n, plan.cfg.m, st, plan.nstages)


def run_batch(plans, stream=None):
    """Run several plans in one persistent launch (qsim_run_batch). Returns
    (states, launch) where launch is the persistent launch's kernel statistic."""
    n = len(plans)
    handles = (_VP * n)(*[p.handle for p in plans])
    outs = (_VP * n)()
    stats = (Stats * n)()
    ks = KernelStat()
    _check(lib().qsim_run_batch(handles, n, _stream_ptr(stream), outs, stats, ctypes.byref(ks)), "qsim_run_batch")
    states = [State(_VP(outs[i]), plans[i].n, plans[i].cfg.m, stats[i], plans[i].nstages) for i in range(n)]
    launch = {"name": ks.name.decode(), "launches": ks.launches, "seconds": ks.seconds, "alg_bytes": ks.alg_bytes,
              "alg_flops": ks.alg_flops}
    return states, launch


# --------------------------------------------------------------------------
# sharded runs (one rank's SV groups)
# --------------------------------------------------------------------------

class ShardRun:
    """qsim_shard_*: rank `rank` of 2^log2_ranks running its SV groups stage by stage; blocks move between
    ranks through export (packed into a uint8 CUDA tensor) and import."""

    def __init__(self, plan: Plan, rank_qubits, log2_ranks: int, rank: int, stream=None):
        self.plan = plan
        rq = np.ascontiguousarray(rank_qubits, dtype=np.uint32).reshape(-1)
        h = ctypes.c_void_p()
        _check(lib().qsim_shard_begin(plan.handle, rq.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), log2_ranks,
                                      rank, _stream_ptr(stream), ctypes.byref(h)), "qsim_shard_begin")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            lib().qsim_shard_free(self.handle)
            self.handle = None

    def stage(self, s: int):
        _check(lib().qsim_shard_stage(self.handle, s), "qsim_shard_stage")

    def block_bytes(self, blocks) -> np.ndarray:
        b = np.ascontiguousarray(blocks, dtype=np.uint64)
        out = np.zeros(max(1, b.size), dtype=np.uint64)
        _check(lib().qsim_shard_block_bytes(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), b.size,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
               "qsim_shard_block_bytes")
        return out[: b.size]

    def export(self, blocks):
        """(sizes, packed uint8 CUDA tensor) of the blocks, which leave this rank."""
        import torch
        b = np.ascontiguousarray(blocks, dtype=np.uint64)
        sizes = self.block_bytes(b)
        buf = torch.empty(max(16, int(sizes.sum())), dtype=torch.uint8, device="cuda")
        _check(lib().qsim_shard_export(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), b.size,
                                       ctypes.c_void_p(buf.data_ptr()), buf.numel()), "qsim_shard_export")
        return sizes, buf[: int(sizes.sum())]

    def import_(self, blocks, sizes, packed):
        b = np.ascontiguousarray(blocks, dtype=np.uint64)
        sz = np.ascontiguousarray(sizes, dtype=np.uint64)
        if b.size == 0:
            return
        packed = packed.contiguous()
        _check(lib().qsim_shard_import(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       sz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), b.size,
                                       ctypes.c_void_p(packed.data_ptr())), "qsim_shard_import")

    def finish(self) -> "State":
        h = ctypes.c_void_p()
        st = Stats()
        _check(lib().qsim_shard_finish(self.handle, ctypes.byref(h), ctypes.byref(st)), "qsim_shard_finish")
        return State(h, self.plan.n, self.plan.cfg.m, st, self.plan.nstages)


# --------------------------------------------------------------------------
# single-block codec
# --------------------------------------------------------------------------

def compress_block(amps, m: int, eb: float, out=None, cap: Optional[int] = None, stream=None):
    """amps: torch CUDA tensor of 2^m complex64 (or 2^(m+1) float32). Returns
    (out_tensor_uint8, nbytes)."""
    import torch
    if out is None:
        cap = worst_case_bytes(m) if cap is None else cap
        out = torch.empty(max(cap, 16), dtype=torch.uint8, device=amps.device)
    cap = out.numel() if cap is None else cap
    nb = ctypes.c_size_t()
    _check(lib().qsim_compress_block(ctypes.c_void_p(amps.data_ptr()), m, eb, ctypes.c_void_p(out.data_ptr()), cap,
                                     ctypes.byref(nb), _stream_ptr(stream)), "qsim_compress_block")
    return out, nb.value


def qszr_worst_case_bytes(m: int) -> int:
    """qsim_worst_case_bytes_rel: largest QSZR stream of a 2^m-amplitude block."""
    return int(lib().qsim_worst_case_bytes_rel(m))


def compress_block_rel(amps, m: int, rel: float, out=None, cap: Optional[int] = None, stream=None):
    """qsim_compress_block_rel: a QSZR stream under the point-wise relative bound rel. Returns
    (out_tensor_uint8, nbytes)."""
    import torch
    if out is None:
        cap = qszr_worst_case_bytes(m) if cap is None else cap
        out = torch.empty(max(cap, 16), dtype=torch.uint8, device=amps.device)
    cap = out.numel() if cap is None else cap
    nb = ctypes.c_size_t()
    _check(lib().qsim_compress_block_rel(ctypes.c_void_p(amps.data_ptr()), m, rel, ctypes.c_void_p(out.data_ptr()),
                                         cap, ctypes.byref(nb), _stream_ptr(stream)), "qsim_compress_block_rel")
    return out, nb.value


def compress_block_rel_rc(amps, m, rel, cap, stream=None):
    """Returns (rc, needed_bytes) without raising (for capacity and range tests)."""
    import torch
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=amps.device)
    nb = ctypes.c_size_t()
    rc = lib().qsim_compress_block_rel(ctypes.c_void_p(amps.data_ptr()), m, rel, ctypes.c_void_p(out.data_ptr()), cap,
                                       ctypes.byref(nb), _stream_ptr(stream))
    return rc, nb.value


def compress_block_needed(amps, m, eb, cap, stream=None):
    """Returns (rc, needed_bytes) without raising (for capacity tests)."""
    import torch
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=amps.device)
    nb = ctypes.c_size_t()
    rc = lib().qsim_compress_block(ctypes.c_void_p(amps.data_ptr()), m, eb, ctypes.c_void_p(out.data_ptr()), cap,
                                   ctypes.byref(nb), _stream_ptr(stream))
    return rc, nb.value


NOALLOC_MAX_M = 24


def compress_block_noalloc(amps, m: int, eb: float, out, cap: Optional[int] = None, stream=None):
    """qsim_compress_block_noalloc: same stream as compress_block, but the
    library allocates nothing (its scratch is a fixed device array). `out` is
    the caller's uint8 CUDA tensor. Returns (rc, nbytes) without raising."""
    import torch
    nfloat = amps.numel() * (2 if amps.dtype == torch.complex64 else 1)
    if not (amps.is_cuda and amps.dtype in (torch.complex64, torch.float32) and amps.is_contiguous()
            and nfloat >= (2 << m)):
        raise ValueError("amps must be a contiguous CUDA tensor of 2^m complex64 (or 2^(m+1) float32) values")
    if not (out.is_cuda and out.dtype == torch.uint8 and out.is_contiguous()):
        raise ValueError("out must be a contiguous uint8 CUDA tensor")
    cap = out.numel() if cap is None else cap
    if cap > out.numel():
        raise ValueError("cap exceeds the bytes of out")
    nb = ctypes.c_size_t()
    rc = lib().qsim_compress_block_noalloc(ctypes.c_void_p(amps.data_ptr()), m, eb, ctypes.c_void_p(out.data_ptr()),
                                           cap, ctypes.byref(nb), _stream_ptr(stream))
    return rc, nb.value


def decompress_block(stream_bytes, m: int, out=None, nbytes: Optional[int] = None, stream=None):
    """stream_bytes: torch uint8 CUDA tensor holding a QSZ1 stream."""
    import torch
    if out is None:
        out = torch.empty(1 << m, dtype=torch.complex64, device=stream_bytes.device)
    nb = stream_bytes.numel() if nbytes is None else nbytes
    _check(lib().qsim_decompress_block(ctypes.c_void_p(stream_bytes.data_ptr()), nb, ctypes.c_void_p(out.data_ptr()),
                                       m, _stream_ptr(stream)), "qsim_decompress_block")
    return out


def decompress_block_rc(stream_bytes, m: int, nbytes: int, stream=None) -> int:
    import torch
    out = torch.empty(1 << m, dtype=torch.complex64, device=stream_bytes.device)
    return lib().qsim_decompress_block(ctypes.c_void_p(stream_bytes.data_ptr()), nbytes, ctypes.c_void_p(out.data_ptr()),
                                       m, _stream_ptr(stream))


# --------------------------------------------------------------------------
# learned size predictor
# --------------------------------------------------------------------------

def mlp_forward(params, x, bf16=False, stream=None):
    """params: CUDA float32 (6913); x: CUDA float32 (B, 41). Returns y (B)."""
    import torch
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().qsim_mlp_forward(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                  ctypes.c_void_p(y.data_ptr()), 1 if bf16 else 0, _stream_ptr(stream)),
           "qsim_mlp_forward")
    return y


def mlp_loss_grad(params, x, t, stream=None):
    import torch
    g = torch.empty_like(params)
    loss = ctypes.c_float()
    _check(lib().qsim_mlp_loss_grad(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(t.data_ptr()), x.shape[0], ctypes.c_void_p(g.data_ptr()),
                                    ctypes.byref(loss), _stream_ptr(stream)), "qsim_mlp_loss_grad")
    return loss.value, g


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().qsim_adam_step(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), params.numel(), t, lr,
                                beta1, beta2, eps, _stream_ptr(stream)), "qsim_adam_step")


def predictor_train(rows: np.ndarray, epochs=60, batch=64, lr=3e-3, seed=100, bf16=False) -> float:
    rows = np.ascontiguousarray(rows, dtype=np.float32).reshape(-1, TRAIN_ROW)
    tc = TrainConfig(epochs, batch, lr, 1 if bf16 else 0, seed)
    loss = ctypes.c_double()
    _check(lib().qsim_predictor_train(ctypes.c_void_p(rows.ctypes.data), rows.shape[0], ctypes.byref(tc),
                                      ctypes.byref(loss)), "qsim_predictor_train")
    return loss.value


def predictor_set(params: np.ndarray, bf16=False):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().qsim_predictor_set(ctypes.c_void_p(p.ctypes.data), p.size, 1 if bf16 else 0), "qsim_predictor_set")


def predictor_get() -> np.ndarray:
    p = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(lib().qsim_predictor_get(ctypes.c_void_p(p.ctypes.data), p.size), "qsim_predictor_get")
    return p


# --------------------------------------------------------------------------
# autotuner
# --------------------------------------------------------------------------

def autotune(circuit, base: Optional[Config] = None, m=(18, 24), k=(3, 6), inner=(2, 4), streams=(1, 2, 4),
             prefix_gates=0, reps=1, max_working_log2=0):
    """Returns (best Config, prefix seconds, candidates timed; 0 = cache hit)."""
    base = base if base is not None else default_config(init_basis=circuit.init_basis)
    mask = 0
    for sc in streams:
        mask |= 1 << sc
    sp = TuneSpace(m[0], m[1], k[0], k[1], inner[0], inner[1], mask, prefix_gates, reps, max_working_log2)
    arr, mats = marshal_gates(circuit.gates)
    best = Config()
    secs = ctypes.c_double()
    cand = ctypes.c_uint32()
    _check(lib().qsim_autotune(circuit.n, arr, len(circuit.gates), ctypes.byref(base), ctypes.byref(sp),
                               ctypes.byref(best), ctypes.byref(secs), ctypes.byref(cand)), "qsim_autotune")
    return best, secs.value, cand.value


def autotune_cache_clear():
    lib().qsim_autotune_cache_clear()
