#!/usr/bin/env python
"""Benchmark of the compressed staged state-vector loop on GB300.

Workload (default): QAOA MaxCut with p = 3 on a seeded random 3-regular graph
of 32 vertices — an H layer, then 3 x (RZZ(gamma) on all 48 edges, RX(beta) on
every qubit), 272 gates, complex64 state (32 GiB raw), eps = 1e-3
(eb = eps * 2^-16 per real/imaginary part), SV blocks of 2^25 amplitudes,
inner size 3 (working vectors of 2^28 amplitudes), gates fused to k = 5, commutation-aware partition with diagonal
gates exempt. The timed form is the tensor-core one with learned sizing: fused
k-qubit gates as TF32 GEMMs on tcgen05, slots reserved by the trained size
predictor. Beside it, on the same circuit ("forms"): the plain FP32 form
(CUDA-core gates, exact sizing), the tensor-core form with exact sizing, and
the tensor-core form with Algorithm 1 over the gates in circuit order.

One step = one qsim_run of the whole circuit through the C ABI: initial
store, then per stage decompress -> fused gate passes -> sizing ->
reservation -> compress for every SV group. Metric: amplitude-gate updates/s
= 2^n * (gates before fusion) / time, with the compression ratio
8 * 2^n / (peak compressed store over stages) and the fidelity bound reported
beside it.

  value  — K steps, plan and inputs already resident, CUDA events on the
           caller's stream (the library joins its streams back to it);
  e2e    — K steps from host data through the public API: plan from the host
           gate list (matrices uploaded), run, read sampled amplitudes and
           the statistics back to the host.
The working set (32 GiB state, ~12 GB compressed) is larger than L2 (129 MB),
so no explicit flush is done between steps.

`--impl reference` times the CPU oracle (complex128 staged simulation + scalar
codec) on a bounded sample of the same workload on the host cores.

For N > 1 (torchrun), every rank runs an independent replica (weak scaling);
the per-rank times are reduced with MAX and rank 0 prints the line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128
NUM_SMS = 152


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--m", type=int, default=25)
    ap.add_argument("--inner", type=int, default=3)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--streams", type=int, default=2)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle sample")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--mode", default="streams", choices=["streams", "persistent"])
    ap.add_argument("--graph", action="store_true", help="persistent mode: capture the stage loop in a CUDA graph")
    ap.add_argument("--sizing", default="predict", choices=["exact", "predict"])
    ap.add_argument("--margin", type=float, default=0.25, help="predictor reservation margin")
    ap.add_argument("--diag-exempt", action=argparse.BooleanOptionalAction, default=True,
                    help="diagonal gates never count as global qubits in the partition (Algorithm 1's option for "
                         "QAOA and Grover; --no-diag-exempt counts them as the paper does)")
    ap.add_argument("--mma", default="tcgen05", choices=["warp", "tcgen05"],
                    help="TF32 / split-BF16 dense ops of width 5: warp-level mma.sync, or tcgen05 with the accumulator in TMEM")
    ap.add_argument("--reorder", action=argparse.BooleanOptionalAction, default=True,
                    help="commutation-aware partition: gates may move before earlier gates they commute with "
                         "(--no-reorder: Algorithm 1 in circuit order)")
    ap.add_argument("--pack", action=argparse.BooleanOptionalAction, default=True,
                    help="with --reorder: each stage's gates gathered into tile passes and fused pass by pass where "
                         "the planner's pass-time model gains 5 %% (reorder mode 2; --no-pack keeps each stage's "
                         "gates in partition order)")
    ap.add_argument("--pack-all", action="store_true",
                    help="with --reorder: the pass-aware order in every stage, without the model (reorder mode 3)")
    ap.add_argument("--train-n", type=int, default=0, help="qubits of the predictor's training circuits (0 = n)")
    ap.add_argument("--workload", default="qaoa", choices=["qft", "qaoa", "random", "mirror", "batch"],
                    help="qft: QFT + 4 x (RZ, CX ladder) on n qubits; qaoa: MaxCut p=3 on a random 3-regular "
                         "graph of n vertices; random: U3 + CZ brick of depth --depth; mirror: depth/2 random "
                         "layers then their inverse (ideal final state |0...0>); batch: --batch independent "
                         "circuits (GHZ, QFT, random depth 8, Grover 3-6 iterations; n ~ U{20..30}) in one "
                         "persistent launch")
    ap.add_argument("--batch", type=int, default=64, help="batch workload: number of circuits")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: fixed m, k instead of the autotuner")
    ap.add_argument("--tune", action="store_true",
                    help="single-circuit workloads: pick m, k, inner (and streams) with the autotuner first "
                         "(not timed; m in 18..24, k in 3..6: 3..5 in persistent mode unless TF32 on tcgen05)")
    ap.add_argument("--depth", type=int, default=14)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement (long workloads)")
    ap.add_argument("--cap-gib", type=float, default=0.0, help="device tier cap (pinned host holds the rest)")
    ap.add_argument("--forms", type=int, default=3,
                    help="timed runs of each comparison form (plain FP32 + exact sizing; the timed precision with "
                         "exact sizing); 0 skips them")
    ap.add_argument("--shard", action="store_true",
                    help="run the circuit sharded over the ranks (qsim_shard_*: each rank runs its SV groups, "
                         "compressed blocks exchanged between stages); the default for N > 1, and at N = 1 a "
                         "single-rank sharded run")
    ap.add_argument("--codec", default="abs", choices=["abs", "rel"],
                    help="abs: point-wise absolute bound eps*2^(-n/2) (QSZ1); rel: point-wise relative bound eps "
                         "(QSZR, the paper's Sec. 4.3 mode)")
    return ap.parse_args()


def batch_workload(args, seed=None):
    from paper_2410_14088_gb300 import inputs
    return inputs.batch_circuits(args.seed if seed is None else seed, count=args.batch, nmin=20, nmax=30)


def workload(args, seed=None, n=None):
    from paper_2410_14088_gb300 import inputs
    seed = args.seed if seed is None else seed
    n = args.n if n is None else n
    if args.workload == "batch":
        # the oracle sample of the batch: its first random circuit (per-amplitude cost does not depend on n)
        cs = batch_workload(args, seed)
        return next((c for c in cs if c.family == "random"), cs[0])
    if args.workload == "qaoa":
        return inputs.qaoa_maxcut(n, 3, seed)
    if args.workload == "random":
        return inputs.random_brick(n, args.depth, seed)
    if args.workload == "mirror":
        return inputs.mirror_brick(n, args.depth // 2, seed)
    return inputs.qft_rz_cx(n, 4, seed)


def max_over_ranks(x, dist, device="cuda"):
    """The largest of the ranks' values (every rank gets it); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, units_per_step, max_ms):
    """Whole-job throughput: every rank runs `steps` steps of `units_per_step` units (weak scaling), timed by the
    slowest rank."""
    return world * steps * units_per_step / (max_ms * 1e-3)


def cpu_model():
    """The host CPU's model name (lscpu on Arm, /proc/cpuinfo on x86), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


# --------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline key)
# --------------------------------------------------------------------------
class OracleSampler:
    """Bounded sample of the CPU oracle on the benchmark workload: complex128
    gate updates on the full state in circuit order (continuing across
    calls), plus QSZ1 encode + decode of SV blocks. The full-run time is
    modelled as (time per gate) x gates + (time per block) x blocks x stages."""

    MAX_SAMPLE_QUBITS = 28  # a 2^28 complex128 state is 4 GiB of host memory; 32 qubits would need 64 GiB

    def __init__(self, args):
        import numpy as np

        import oracle
        from oracle.partition import partition

        self.np, self.oracle = np, oracle
        full = workload(args)
        self.n, self.m = full.n, min(args.m, full.n - 4)
        # gates are timed on the same family's circuit at min(n, 28) qubits (same seed) and scaled by
        # 2^(n - n_sample): the per-gate work of the plain update is proportional to the state size
        self.n_sample = min(self.n, self.MAX_SAMPLE_QUBITS)
        if args.workload == "batch" or self.n_sample == self.n:
            self.n_sample = self.n
            self.circ = full
        else:
            self.circ = workload(args, n=self.n_sample)
        self.full_gates = len(full.gates)
        self.rel = getattr(args, "codec", "abs") == "rel"
        self.eb = args.eps if self.rel else args.eps * 2.0 ** (-self.n / 2)
        self.codec = "QSZR" if self.rel else "QSZ1"
        self.stages = partition(full.gates, self.n, self.m, args.inner)
        self.psi = oracle.basis_state(self.n_sample, self.circ.init_basis)
        self.next_gate = 0
        self.next_block = 0
        self.t_gates = self.t_codec = 0.0
        self.gates_done = self.blocks_done = 0

    def step(self, budget_s, record=True):
        t0 = time.perf_counter()
        g = b = 0
        while time.perf_counter() - t0 < 0.7 * budget_s or g == 0:
            gi = self.next_gate % len(self.circ.gates)
            self.oracle.apply_gate(self.psi, self.n_sample, self.circ.gates[gi])
            self.next_gate += 1
            g += 1
        t1 = time.perf_counter()
        nblocks = 1 << (self.n_sample - self.m)
        while time.perf_counter() - t1 < 0.3 * budget_s or b == 0:
            j = self.next_block % nblocks
            blk = self.psi[2 * (j << self.m): 2 * ((j + 1) << self.m)].astype(self.np.float32)
            if self.rel:
                self.oracle.qszr_decode(self.oracle.qszr_encode(blk, self.m, self.eb), self.m)
            else:
                self.oracle.qsz_decode(self.oracle.qsz_encode(blk, self.m, self.eb), self.m)
            self.next_block += 1
            b += 1
        t2 = time.perf_counter()
        if record:
            self.t_gates += t1 - t0
            self.t_codec += t2 - t1
            self.gates_done += g
            self.blocks_done += b

    def result(self):
        scale = float(1 << (self.n - self.n_sample))
        per_gate = self.t_gates / max(1, self.gates_done) * scale
        per_block = self.t_codec / max(1, self.blocks_done)
        nblocks = 1 << (self.n - self.m)
        total = per_gate * self.full_gates + per_block * nblocks * len(self.stages)
        ups = (1 << self.n) * self.full_gates / total
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        where = (f"the full 2^{self.n} state" if self.n_sample == self.n else
                 f"a 2^{self.n_sample} state of the same circuit family and seed (per-gate time x "
                 f"2^{self.n - self.n_sample} for 2^{self.n} amplitudes)")
        sample = (f"{self.gates_done} complex128 gate updates of {where} "
                  f"({self.t_gates:.1f} s) and {self.blocks_done} {self.codec} encode+decode of 2^{self.m}-amplitude "
                  f"blocks ({self.t_codec:.1f} s); full run modelled as per-gate time x {self.full_gates} "
                  f"gates + per-block codec time x {nblocks} blocks x {len(self.stages)} stages")
        return ups, sample, threads, total


def run_reference(args, rank, world):
    if rank != 0:
        return
    smp = OracleSampler(args)
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        smp.step(0.5, record=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.step(per_step)
    wall = time.perf_counter() - t0
    ups, sample, threads, total = smp.result()
    line = {
        "impl": "reference", "metric": "amplitude-gate updates/s incl. codec & compression ratio at fidelity>=0.99",
        "value": ups, "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        # each step is a bounded sample of the workload (its wall time here); the rate is the full run's,
        # modelled from the sample's per-gate and per-block times (modelled_full_run_ms)
        "ms_per_step": wall * 1e3 / max(1, args.steps), "modelled_full_run_ms": total * 1e3,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args),
        "cpu_baseline": {"value": ups, "unit": "updates/s", "cores": threads, "cpu_model": cpu_model(),
                         "nproc": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": ups, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reorder_mode(args):
    """qsim_config.reorder: 0 Algorithm 1 in circuit order, 1 commutation-aware stages, 2 and the pass-aware order
    where the planner's model gains, 3 the pass-aware order in every stage."""
    return (3 if args.pack_all else 2) if args.reorder and (args.pack or args.pack_all) else 1 if args.reorder else 0


def partition_name(args):
    return ("Algorithm 1 in circuit order" if not args.reorder else
            "commutation-aware (reorder), pass-aware order in every stage" if args.pack_all else
            "commutation-aware (reorder), pass-aware order where modelled faster" if args.pack else
            "commutation-aware (reorder)")


def config_dict(args):
    if args.workload == "batch":
        cs = batch_workload(args)
        return {"workload": f"batch of {args.batch} circuits (ghz, qft, random u3+cz depth 8, grover 3-6 "
                            f"iterations; n~U{{20..30}}, seed {args.seed}), one persistent launch, eps={args.eps:g}, "
                            f"prec={args.prec}, sizing={args.sizing}, m/k/inner "
                            f"{'fixed' if args.no_tune else 'autotuned per circuit'}",
                "circuits": len(cs), "n_qubits": [min(c.n for c in cs), max(c.n for c in cs)],
                "gates": sum(len(c.gates) for c in cs), "eps": args.eps, "prec": args.prec,
                "mode": "persistent (one launch for the batch)", "sizing": args.sizing,
                "partition": partition_name(args),
                "raw_state_gib": sum(8 << c.n for c in cs) / 2**30,
                "l2_policy": "working set (all circuits' compressed stores) > L2 (129 MB); no flush"}
    name = {"qft": f"qft{args.n}+4x(rz,cx-ladder)", "qaoa": f"qaoa-maxcut p=3, 3-regular n={args.n}",
            "random": f"random u3+cz brick n={args.n} depth={args.depth}",
            "mirror": f"mirror u3+cz brick n={args.n} depth={args.depth}"}[args.workload]
    raw = 8 << args.n
    bound = "" if args.codec == "abs" else ", codec=relative (QSZR)"
    return {"workload": f"{name}, m={args.m}, inner={args.inner}, k={args.k}, eps={args.eps:g}, prec={args.prec}, "
                        f"mode={args.mode}{'+graph' if args.graph else ''}, sizing={args.sizing}{bound}"
                        f"{', mma=tcgen05' if args.mma == 'tcgen05' and args.prec != 'fp32' and args.mode == 'streams' else ''}",
            "error_bound": ("absolute eps*2^(-n/2) per component" if args.codec == "abs"
                            else "relative eps per component"),
            "partition": partition_name(args) +
                         (", diagonal gates exempt" if args.diag_exempt else ""),
            "n_qubits": args.n, "gates": len(workload(args).gates), "block_log2": args.m, "inner": args.inner,
            "k": args.k, "eps": args.eps, "prec": args.prec,
            "mma": ("fp32 cuda cores" if args.prec == "fp32" else args.mma if args.mode == "streams" else "warp"),
            "streams": args.streams,
            "mode": args.mode,
            "graph": bool(args.graph), "sizing": args.sizing, "device_tier_cap_gib": args.cap_gib,
            "l2_policy": f"working set ({raw / 2**30:.3g} GiB state, compressed ~{raw / 2.8 / 2**30:.2g} GiB) "
                         f"> L2 (129 MB); no flush"}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_2410_14088_gb300 import qsim

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    prec = {"fp32": qsim.PREC_FP32, "tf32": qsim.PREC_TF32, "bf16x3": qsim.PREC_BF16X3}[args.prec]
    circ = workload(args)
    G = len(circ.gates)
    n = circ.n
    kw = dict(m=args.m, inner=args.inner, k=args.k, eps=args.eps, prec=prec, streams=args.streams,
              mode=qsim.MODE_PERSISTENT if args.mode == "persistent" else qsim.MODE_STREAMS,
              graph=1 if args.graph else 0,
              sizing=qsim.SIZING_PREDICT if args.sizing == "predict" else qsim.SIZING_EXACT,
              predictor_margin=args.margin, diag_exempt=1 if args.diag_exempt else 0,
              reorder=reorder_mode(args), tcgen05=1 if args.mma == "tcgen05" else 0,
              device_tier_cap_bytes=int(args.cap_gib * (1 << 30)),
              codec=qsim.CODEC_QSZR if args.codec == "rel" else qsim.CODEC_QSZ1)
    train_info = None
    if args.sizing == "predict":
        # training rows from exact-sizing runs of training seeds (100+) of the same family, not timed
        import numpy as np
        t0 = time.perf_counter()
        rows = []
        tkw = dict(kw, mode=qsim.MODE_STREAMS, sizing=qsim.SIZING_EXACT, graph=0)
        for sd in (100, 101):
            st = qsim.run(qsim.plan_stages(workload(args, sd, args.train_n or None), collect=1, **tkw))
            rows.append(st.training_data())
            del st
        rows = np.concatenate(rows)
        loss = qsim.predictor_train(rows, epochs=40, batch=64, lr=3e-3, seed=100)
        train_info = {"rows": int(rows.shape[0]), "loss": loss, "seconds": time.perf_counter() - t0}
    tune_info = None
    if args.tune:
        t0 = time.perf_counter()
        base = qsim.default_config(init_basis=circ.init_basis, **kw)
        # the persistent kernel fuses width 6 only as TF32 on tcgen05
        kmax = 6 if args.mode == "streams" or (args.prec == "tf32" and args.mma == "tcgen05") else 5
        best, secs, cand = qsim.autotune(circ, base, m=(18, min(24, n - 2)), k=(3, kmax), inner=(2, 5),
                                         streams=(1, 2) if args.mode == "streams" else (1,),
                                         prefix_gates=min(len(circ.gates), 160), reps=1, max_working_log2=n - 2)
        for f in ("m", "k", "inner", "streams"):
            kw[f] = getattr(best, f)
        args.m, args.k, args.inner, args.streams = best.m, best.k, best.inner, best.streams
        tune_info = {"seconds": time.perf_counter() - t0, "candidates_timed": cand, "prefix_seconds": secs,
                     "m": best.m, "k": best.k, "inner": best.inner, "streams": best.streams}
    plan = qsim.plan_stages(circ, **kw)
    stream = torch.cuda.current_stream()
    # sharded over the ranks (strong scaling: one circuit, its SV groups dealt to the ranks, compressed blocks
    # exchanged between stages), or one replica of the whole circuit per rank (weak scaling)
    sharded = args.shard or world > 1
    log2w = world.bit_length() - 1
    if sharded and world != 1 << log2w:
        raise SystemExit("sharded runs need a power-of-two number of ranks")
    jobs = 1 if sharded else world  # circuits the job runs per step

    def run_once():
        if sharded:
            from paper_2410_14088_gb300 import shard
            return shard.run_sharded(plan, log2w, dist)[0]
        return qsim.run(plan)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up ----
    for _ in range(args.warmup):
        st = run_once()
        del st
    barrier()

    # ---- timed: value (inputs resident) ----
    qsim.profile_enable(not args.no_profile)
    sampler = ClockSampler(dev)
    sampler.start()
    launches0 = qsim.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    kstats_acc = {}
    stats = []
    for _ in range(args.steps):
        st = run_once()
        stats.append(st.stats.as_dict())
        for k, v in st.kernel_stats().items():
            a = kstats_acc.setdefault(k, {"launches": 0, "seconds": 0.0, "alg_bytes": 0.0, "alg_flops": 0.0})
            for f in a:
                a[f] += v[f]
        del st
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    qsim.profile_enable(False)
    launches = qsim.launch_count() - launches0
    t_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(t_ms, dist)
    ups = job_rate(jobs, args.steps, (1 << n) * G, t_max)

    # ---- timed: e2e through the public API from host data ----
    idx = np.arange(0, 1 << n, (1 << n) // 4096, dtype=np.uint64)[:4096]
    if sharded and plan.nstages:
        # each rank reads the sampled amplitudes that lie in the blocks it holds after the last stage
        from paper_2410_14088_gb300 import shard
        last_q = plan.shards(log2w)[-1] if log2w else []
        own = shard.block_owner(idx >> np.uint64(args.m), last_q, args.m) == rank
        idx = idx[own]
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d = d2h = 0
    for _ in range(0 if args.no_e2e else args.steps):
        p2 = qsim.plan_stages(circ, **kw)
        if sharded:
            from paper_2410_14088_gb300 import shard
            st = shard.run_sharded(p2, log2w, dist)[0]
        else:
            st = qsim.run(p2)
        amps = st.amplitudes(idx)
        h2d += st.stats.h2d_bytes + idx.nbytes
        d2h += st.stats.d2h_bytes + amps.nbytes
        del st, p2
    e1.record(stream)
    barrier()
    te_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    e2e = job_rate(jobs, args.steps, (1 << n) * G, te_ms) if not args.no_e2e else None

    # ---- per-kernel times without the other stream's kernels beside them (roofline context) ----
    kstats_serial = None
    if not args.no_profile and args.mode == "streams" and args.streams > 1 and not sharded:
        plan1 = qsim.plan_stages(circ, **dict(kw, streams=1))
        st = qsim.run(plan1)
        del st
        qsim.profile_enable(True)
        st = qsim.run(plan1)
        kstats_serial = st.kernel_stats()
        qsim.profile_enable(False)
        del st, plan1

    # ---- the comparison forms on the same circuit and partition: plain FP32 CUDA-core gates with exact sizing
    # (the method without either addition), and the timed precision with exact sizing (without the predictor) ----
    forms = None
    if args.forms > 0 and args.codec == "abs" and not sharded:
        headline = f"{args.prec}{'_tcgen05' if args.mma == 'tcgen05' and args.prec != 'fp32' else ''}_{args.sizing}_sizing"
        forms = {headline: {"value": ups, "ms_per_step": t_max / args.steps, "steps": args.steps,
                            "stages": stats[-1]["nstages"], "fidelity_lower_bound": stats[-1]["fidelity_lower_bound"],
                            "timed_form": True}}
        variants = []
        if not (args.prec == "fp32" and args.sizing == "exact"):
            variants.append(("fp32_exact_sizing", dict(kw, prec=qsim.PREC_FP32, sizing=qsim.SIZING_EXACT, tcgen05=0)))
        if args.sizing == "predict":
            variants.append((headline.replace("_predict_sizing", "_exact_sizing"), dict(kw, sizing=qsim.SIZING_EXACT)))
        if args.reorder and (args.pack or args.pack_all):
            # the same partition with each stage's gates fused and laid out in partition order
            variants.append((headline.replace("_predict_sizing", "_exact_sizing") + "_without_pass_order",
                             dict(kw, sizing=qsim.SIZING_EXACT, reorder=1)))
        if args.reorder or args.diag_exempt:
            # the paper's partition: Algorithm 1 over the gates in circuit order, every gate counted
            variants.append((headline.replace("_predict_sizing", "_exact_sizing") + "_algorithm1_in_order",
                             dict(kw, sizing=qsim.SIZING_EXACT, reorder=0, diag_exempt=0)))
        for name, fk in variants:
            pl = qsim.plan_stages(circ, **fk)
            del_st = qsim.run(pl)  # warm-up (plan upload, arenas)
            del del_st
            barrier()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            fst = None
            for _ in range(args.forms):
                st = qsim.run(pl)
                fst = st.stats.as_dict()
                del st
            f1.record(stream)
            barrier()
            fms = max_over_ranks(f0.elapsed_time(f1), dist)
            forms[name] = {"value": job_rate(world, args.forms, (1 << n) * G, fms), "ms_per_step": fms / args.forms,
                           "steps": args.forms, "stages": fst["nstages"],
                           "fidelity_lower_bound": fst["fidelity_lower_bound"],
                           "compression_ratio": 8.0 * (1 << n) / max(1, fst["peak_store_bytes"]),
                           "overflow_blocks": fst["overflow_blocks"]}
            del pl
        if "fp32_exact_sizing" in forms:
            forms["speedup_vs_fp32_exact_sizing"] = ups / forms["fp32_exact_sizing"]["value"]

    if rank != 0:
        return
    last = stats[-1]
    peaks, peaks_kind = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # dominant kernel by event-timed total
    roofline = None
    kernels = {}
    if kstats_acc:
        dom = max(kstats_acc, key=lambda k: kstats_acc[k]["seconds"])
        for k, v in kstats_acc.items():
            kernels[k] = {"launches": v["launches"], "ms_per_launch": 1e3 * v["seconds"] / max(1, v["launches"]),
                          "share": v["seconds"] / max(1e-12, sum(x["seconds"] for x in kstats_acc.values())),
                          "GBps": v["alg_bytes"] / max(1e-12, v["seconds"]) / 1e9,
                          "TFLOPps": v["alg_flops"] / max(1e-12, v["seconds"]) / 1e12}
        d = kstats_acc[dom]
        per_launch_s = d["seconds"] / max(1, d["launches"])
        gbps = d["alg_bytes"] / max(1e-12, d["seconds"]) / 1e9
        tflops = d["alg_flops"] / max(1e-12, d["seconds"]) / 1e12
        hbm_frac = gbps / peaks["hbm_gbs"]
        cands = [{"bound": "hbm", "achieved": gbps, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "peak_source": f"{peaks_kind} hbm_gbs (copy)"}]
        if d["alg_flops"] > 0:
            if args.prec == "fp32":
                cands.append({"bound": "alu", "achieved": tflops, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                              "peak_source": f"derived: {NUM_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                             f"{sm_max:.0f} MHz"})
            else:
                key = "bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks else "bf16_tflops"
                ratio = 1.1 / 2.25 if args.prec == "tf32" else 1.0
                cands.append({"bound": "tensor", "achieved": tflops, "peak": peaks[key] * ratio, "unit": "TFLOP/s",
                              "peak_source": f"{peaks_kind} {key}" + (" x 1.1/2.25 (nominal TF32/BF16)"
                                                                      if args.prec == "tf32" else "")})
        for c in cands:
            c["frac"] = c["achieved"] / c["peak"]
        roofline = dict(max(cands, key=lambda c: c["frac"]))
        roofline["kernel"] = dom
        roofline["other_bounds"] = [{k: c[k] for k in ("bound", "frac")} for c in cands if c["bound"] != roofline["bound"]]
        roofline["traffic"] = traffic_for(dom, d["alg_bytes"] / max(1, d["launches"]))
        roofline["ms_per_launch"] = per_launch_s * 1e3
        if kstats_serial and dom in kstats_serial:
            # the same kernel in one more run on a single stream: its launches then share the GPU with nothing
            ds = kstats_serial[dom]
            secs = max(1e-12, ds["seconds"])
            ach = (ds["alg_bytes"] if roofline["unit"] == "GB/s" else ds["alg_flops"]) / secs / (
                1e9 if roofline["unit"] == "GB/s" else 1e12)
            roofline["one_stream"] = {"achieved": ach, "frac": ach / roofline["peak"],
                                      "ms_per_launch": 1e3 * ds["seconds"] / max(1, ds["launches"]),
                                      "note": "one extra run of the plan on 1 stream after the timed region; "
                                              "with 2 streams each launch shares the GPU with the other "
                                              "stream's kernels, which lengthens its event-timed duration"}
    cr = 8.0 * (1 << n) / max(1, last["peak_store_bytes"])
    mirror_fidelity = None
    if args.workload == "mirror":
        st = qsim.run(plan)
        a0 = st.amplitudes(np.array([0], dtype=np.uint64))[0]
        mirror_fidelity = float(abs(a0) / math.sqrt(st.norm_sq()))
        del st
    line = {
        "metric": "amplitude-gate updates/s incl. codec & compression ratio at fidelity>=0.99",
        "value": ups, "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "strong" if sharded else "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": dict(config_dict(args), parallelism=(f"sharded over {world} rank(s): SV groups dealt by rank "
                                                     f"qubits, compressed blocks exchanged between stages")
                       if sharded else f"{world} independent replica(s)"),
        "compression_ratio": cr, "compression_ratio_vs_complex128": 2 * cr,
        "fidelity_lower_bound": last["fidelity_lower_bound"], "norm_sq": last["norm_sq"],
        "stages": last["nstages"], "plan_seconds": plan.stats()["plan_seconds"],
        "overflow_blocks": last["overflow_blocks"], "peak_reserved_bytes": last["peak_reserved_bytes"],
        "host_tier_peak_bytes": last["host_tier_peak_bytes"], "predictor_training": train_info,
        "autotune": tune_info,
        "mirror_fidelity": mirror_fidelity,
        "forms": forms,
        "e2e": {"value": e2e, "unit": "updates/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps} if e2e is not None else None,
        "gpu_launches": launches,
        "launches_before_timed": launches0,
        "roofline": roofline,
        "kernels": kernels,
        "clocks": clocks,
        "peaks": peaks_kind,
    }
    if not args.no_cpu_baseline:
        smp = OracleSampler(args)
        smp.step(0.5, record=False)
        for _ in range(3):
            smp.step(args.cpu_seconds / 3)
        cups, sample, threads, _ = smp.result()
        line["cpu_baseline"] = {"value": cups, "unit": "updates/s", "cores": threads, "cpu_model": cpu_model(),
                                "nproc": os.cpu_count(), "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)


def run_batch_bench(args, rank, world, dist):
    """Config of a batch of independent circuits: one qsim_run_batch per step."""
    import numpy as np
    import torch

    from paper_2410_14088_gb300 import inputs, qsim

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    prec = {"fp32": qsim.PREC_FP32, "tf32": qsim.PREC_TF32, "bf16x3": qsim.PREC_BF16X3}[args.prec]
    circuits = batch_workload(args)
    base = dict(eps=args.eps, prec=prec, mode=qsim.MODE_PERSISTENT,
                sizing=qsim.SIZING_PREDICT if args.sizing == "predict" else qsim.SIZING_EXACT,
                predictor_margin=args.margin, reorder=reorder_mode(args))
    train_info = None
    if args.sizing == "predict":
        # training rows from exact-sizing runs of a training batch (seed 100+), not timed
        t0 = time.perf_counter()
        rows = []
        for c in inputs.batch_circuits(100, count=8, nmin=20, nmax=24):
            st = qsim.run(qsim.plan_stages(c, m=min(20, c.n - 4), inner=2, k=5, eps=args.eps, prec=prec, collect=1))
            rows.append(st.training_data())
            del st
        rows = np.concatenate(rows)
        loss = qsim.predictor_train(rows, epochs=40, batch=64, lr=3e-3, seed=100)
        train_info = {"rows": int(rows.shape[0]), "loss": loss, "seconds": time.perf_counter() - t0}
    t0 = time.perf_counter()
    cfgs, timed_candidates = [], 0
    for c in circuits:
        if args.no_tune:
            cfgs.append(dict(m=min(args.m, c.n - 4), inner=2, k=min(args.k, 5)))
            continue
        bc = qsim.default_config(init_basis=c.init_basis, **base)
        best, _, cand = qsim.autotune(c, bc, m=(max(12, c.n - 12), min(24, c.n - 4)), k=(3, 5), inner=(2, 4),
                                      streams=(1,), prefix_gates=min(len(c.gates), 96), reps=1,
                                      max_working_log2=c.n - 2)
        timed_candidates += cand
        cfgs.append(dict(m=best.m, inner=best.inner, k=best.k))
    tune_info = None if args.no_tune else {"seconds": time.perf_counter() - t0, "candidates_timed": timed_candidates,
                                           "m": sorted(set(c["m"] for c in cfgs)),
                                           "k": sorted(set(c["k"] for c in cfgs)),
                                           "inner": sorted(set(c["inner"] for c in cfgs))}
    plans = [qsim.plan_stages(c, **cfg, **base) for c, cfg in zip(circuits, cfgs)]
    updates = sum((1 << c.n) * len(c.gates) for c in circuits)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        states, _ = qsim.run_batch(plans)
        del states
    barrier()
    qsim.profile_enable(not args.no_profile)
    sampler = ClockSampler(dev)
    sampler.start()
    launches0 = qsim.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    launch_acc = {"launches": 0, "seconds": 0.0, "alg_bytes": 0.0, "alg_flops": 0.0}
    for _ in range(args.steps):
        states, launch = qsim.run_batch(plans)
        for f in launch_acc:
            launch_acc[f] += launch[f]
        stats = [st.stats.as_dict() for st in states]
        del states
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    qsim.profile_enable(False)
    launches = qsim.launch_count() - launches0
    t_max = max_over_ranks(ev0.elapsed_time(ev1), dist)
    ups = job_rate(world, args.steps, updates, t_max)

    # e2e: plans from the host gate lists, the batch, 64 sampled amplitudes of every circuit read back
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d = d2h = 0
    for _ in range(args.steps):
        ps = [qsim.plan_stages(c, **cfg, **base) for c, cfg in zip(circuits, cfgs)]
        sts, _ = qsim.run_batch(ps)
        for c, st in zip(circuits, sts):
            idx = np.arange(0, 1 << c.n, (1 << c.n) // 64, dtype=np.uint64)[:64]
            a = st.amplitudes(idx)
            h2d += st.stats.h2d_bytes + idx.nbytes
            d2h += st.stats.d2h_bytes + a.nbytes
        del sts, ps
    e1.record(stream)
    barrier()
    te_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    e2e = job_rate(world, args.steps, updates, te_ms)
    if rank != 0:
        return
    peaks, peaks_kind = load_peaks()
    roofline = None
    if launch_acc["launches"]:
        gbps = launch_acc["alg_bytes"] / max(1e-12, launch_acc["seconds"]) / 1e9
        roofline = {"bound": "hbm", "achieved": gbps, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "peak_source": f"{peaks_kind} hbm_gbs (copy)", "frac": gbps / peaks["hbm_gbs"],
                    "kernel": "stage_persistent (whole batch)", "traffic": None,
                    "ms_per_launch": 1e3 * launch_acc["seconds"] / launch_acc["launches"],
                    "tflops": launch_acc["alg_flops"] / max(1e-12, launch_acc["seconds"]) / 1e12}
    raw = sum(8.0 * (1 << c.n) for c in circuits)
    line = {
        "metric": "amplitude-gate updates/s incl. codec & compression ratio at fidelity>=0.99",
        "value": ups, "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3"}[args.prec], "data": "synthetic",
        "config": config_dict(args),
        "compression_ratio": raw / max(1, sum(s["peak_store_bytes"] for s in stats)),
        "fidelity_lower_bound_min": min(s["fidelity_lower_bound"] for s in stats),
        "fidelity_lower_bound_per_circuit": [round(s["fidelity_lower_bound"], 6) for s in stats],
        "stages_total": sum(s["nstages"] for s in stats),
        "overflow_blocks": sum(s["overflow_blocks"] for s in stats),
        "host_tier_peak_bytes": sum(s["host_tier_peak_bytes"] for s in stats),
        "predictor_training": train_info, "autotune": tune_info,
        "e2e": {"value": e2e, "unit": "updates/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": launches,
        "roofline": roofline,
        "clocks": clocks,
        "peaks": peaks_kind,
    }
    if not args.no_cpu_baseline:
        smp = OracleSampler(args)
        smp.step(0.5, record=False)
        for _ in range(3):
            smp.step(args.cpu_seconds / 3)
        cups, sample, threads, _ = smp.result()
        line["cpu_baseline"] = {"value": cups, "unit": "updates/s", "cores": threads, "cpu_model": cpu_model(),
                                "nproc": os.cpu_count(), "kind": "oracle",
                                "sample": "per-amplitude-gate rate of the batch's first random circuit: " + sample}
    print(json.dumps(line), flush=True)


def code_digest(path):
    """sha256[:16] of a source file's code: // comments, trailing blanks and
    empty lines removed, so that a comment edit keeps a capture valid."""
    import hashlib
    import re
    lines = []
    with open(path) as f:
        for line in f:
            line = re.sub(r"//.*$", "", line.rstrip("\n")).rstrip()
            if line:
                lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def traffic_for(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch size; None when no capture matches the kernel's current code."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) < 5 or parts[0] != kernel:
                continue
            src, digest, dram_bytes, alg_bytes = parts[1], parts[2], float(parts[3]), float(parts[4])
            sp = os.path.join(ROOT, src)
            if not os.path.exists(sp):
                return None
            if code_digest(sp) != digest:
                return None  # kernel changed since the counters were taken
            return dram_bytes / alg_bytes * alg_bytes_per_launch
    return None


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    if args.workload == "batch":
        run_batch_bench(args, rank, world, dist)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
