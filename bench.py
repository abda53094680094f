#!/usr/bin/env python3
"""Benchmark of the implicit-midpoint Lindblad path on GB300.

One bench step = one forward sweep plus the checkpointed discrete-adjoint
gradient (Appendix A-B) of the 2-transmon CNOT workload: two 3-level
transmons (N = 9, vec length 81), 16 essential-basis initial states,
10000 implicit-midpoint steps over T = 200 ns, 20 splines x 2 carriers per
transmon.  Metric: state-steps/s of forward + adjoint (16 x 10000 per step).

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm); under torchrun each rank runs its own replica (weak scaling)
and rank 0 prints the line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Lindblad state-steps/s (fwd+adjoint, FP64)"
UNIT = "state-steps/s"
WORKLOAD = ("cnot_2x3: 2 transmons x 3 levels (N=9, vec 81), 16 essential-basis states |i><j|, "
            "10000 IMR steps, T=200 ns, 2x20 splines x 2 carriers, J_Frob to CNOT, "
            "forward + adjoint gradient (stage vectors kept when the tape fits 8 GiB, else checkpoints)")
# other workloads (--workload), measured the same way; the default line is cnot_2x3
WORKLOADS = {
    "cnot_2x3": WORKLOAD,
    "cnot_3states": ("cnot_3states: the cnot_2x3 system and controls with the three-state gate objective "
                     "(Sec. III-C: 3 Hermitian states, weights 20, 1, 1), 10000 steps, fwd + adjoint"),
    "reset_2x2x20": ("reset_2x2x20: 2 qubits + 20-level cavity (vec 6400) from the ensemble state, J_N0, "
                     "dt=0.05 ns, first {n} of 100000 steps, 100 splines, fwd + adjoint, grid-wide sweep"),
    "qubit_x": "qubit_x: 1 qubit (vec 4), 4 states |i><j|, 1000 steps, T=100 ns, X gate, fwd + adjoint",
    "batch256": ("batch256: 256 independent problems, Q in {1,2,3}, 2-4 levels (vec 4..4096), 3 random pure states "
                 "each, 5000 steps, T=100 ns, fwd + adjoint, one persistent launch per sweep captured in a CUDA graph"),
    "qudits_4x4": ("qudits_4x4: 4 qudits x 4 levels (vec 65536), 3 random pure states, dt=0.0125 ns, "
                   "first {n} of 40000 steps, fwd + adjoint with checkpoints every 100 steps, grid-wide sweep"),
    "qutrits_6x3": ("qutrits_6x3: 6 qutrits (vec 531441), {m} random pure states, dt=0.015 ns, "
                    "first {n} of 20000 steps, fwd + adjoint with checkpoints every 10 steps, grid-wide sweep"),
    "apply_6x3": ("apply_6x3: y = M(t) x, the matrix-free Lindblad apply (lb_apply, one thread per element) on "
                  "{n} states of 6 qutrits (vec 531441, 8.5 MB each), x and y in HBM"),
    "cnot_penalty": ("cnot_penalty: the cnot_2x3 workload with the running penalty gamma1 int beta(t) J dt "
                     "(gamma1 = 0.1, a = 20 ns: Sec. III, eq. optimproblem), one CTA per state, fwd + adjoint"),
    "cnot_jc": ("cnot_jc: the cnot_2x3 workload with a Jaynes-Cummings coupling of the two transmons "
                "(g = 5 MHz, rotating frequencies 4.80 and 4.86 GHz: the coupling rotates at 60 MHz), "
                "one CTA per state, fwd + adjoint"),
    "fock_lbfgs": ("fock_lbfgs: one 4-level qudit |0> -> (|0>+|3>)/sqrt 2, J_Frob, 10 splines x 2 carriers, "
                   "T=200 ns, 10000 steps; one bench step = one L-BFGS run (lb_optimize, memory 10, "
                   "at most 150 iterations, gtol 1e-9) from the seeded controls"),
}
PREFIX = {"qudits_4x4": 2000, "qutrits_6x3": 40, "reset_2x2x20": 2000}
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_PER_SM = 4.0  # 2 FP64 FMA lanes per SM per clock, 2 flops each
CPU_SAMPLE_STEPS = 8000  # oracle sample for the CPU baseline (same dt, 16 states)
REF_SAMPLE_STEPS = 400  # oracle sample per reference-arm step


def problem(n_steps=None, workload="cnot_2x3", states=0):
    import workloads as W

    if workload == "qubit_x":
        p = W.config1()
    elif workload == "cnot_3states":
        p = W.cnot_three_states()
    elif workload == "reset_2x2x20":
        p = W.reset_ensemble()
        n_steps = n_steps or PREFIX[workload]
    elif workload == "qudits_4x4":
        p = W.config4()
        n_steps = n_steps or PREFIX[workload]
    elif workload == "qutrits_6x3":
        p = W.config5(n_states=states or 64)
        p.ckpt_every = 10
        n_steps = n_steps or PREFIX[workload]
    elif workload == "cnot_penalty":
        p = W.config2()
        p.gamma1, p.penalty_a = 0.1, 20.0
    elif workload == "cnot_jc":
        import numpy as np

        p = W.config2()
        p.system.jc_ghz = np.array([[0.0, 0.005], [0.0, 0.0]])
        p.system.rot_ghz = np.array([4.80, 4.86])
    else:
        p = W.config2()
    if n_steps is not None:
        # a prefix of the horizon at the same step size dt = 0.02 ns
        p.system.T_ns = p.system.T_ns * n_steps / p.system.n_steps
        p.system.n_steps = n_steps
    return p


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)


def oracle_sample(n_steps: int) -> dict:
    from oracle import imr

    p = problem(n_steps)
    t0 = time.perf_counter()
    imr.gradient(p)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "state_steps": p.M * n_steps}


def oracle_subprocess(n_steps: int, reps: int = 1) -> dict:
    """Run the oracle sample in a fresh single-threaded process (BLAS pinned to
    one thread) and return the best of ``reps`` runs."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    best = None
    for _ in range(reps):
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_steps)],
                             capture_output=True, text=True, env=env, check=True)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        if best is None or r["seconds"] < best["seconds"]:
            best = r
    return best


# ----------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        else:
            self.lines = []

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ----------------------------------------------------------------------------
# algorithmic FP64 work of the sweep kernels


def fp64_flops(V: int, Q: int, n_decay: int, st: dict, phase_set) -> float:
    """FP64 flops (FMA = 2) of the Jacobi sweeps, from the iteration counts.

    Per element and inner iteration: per subsystem 24 flops for the control
    term (two real-weighted neighbour pairs P, R and the complex control
    factor) plus 4 for the decay sandwich when T1 is finite; 6 for the
    multiplication by (I - dt/2 D)^-1 and 2 for the convergence difference.
    Per element and step: 6 for the initial guess, 4 for q <- 2z - q, and for
    adjoint steps 28 per subsystem for the gradient pieces.  ``V`` is the
    number of elements a state's sweep computes: N^2, or N (N + 1) / 2 when
    the Hermitian symmetry leaves the others as mirrored copies."""
    per_it = 24 * Q + 4 * n_decay + 8
    f = 0.0
    for ph in phase_set:
        f += V * (10 * st["phase_steps"][ph] + per_it * st["phase_iterations"][ph])
        if ph == 2:
            f += V * 28 * Q * st["phase_steps"][ph]
    return f


def traffic_record(kernel: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2110_10310_gb300", "csrc", "lb_kernels.cu")
    if rec.get("code_sha256") != kernel_source_digest(src):
        return None
    return rec.get("dram_bytes_per_launch")


def kernel_source_digest(path: str) -> str:
    """SHA-256 of the kernel source with its // comments and blank lines
    removed: the counters stay valid across comment edits, not across code
    edits.  (The kernel source has no block comments and no // inside string
    literals.)"""
    lines = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


# ----------------------------------------------------------------------------


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(REF_SAMPLE_STEPS)
    tot_s, tot_ss = 0.0, 0
    for _ in range(args.steps):
        r = oracle_sample(REF_SAMPLE_STEPS)
        tot_s += r["seconds"]
        tot_ss += r["state_steps"]
    value = tot_ss / tot_s
    cores = 1
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"first {REF_SAMPLE_STEPS} of 10000 steps per bench step, all 16 states"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"dense-LU oracle gradient, 16 states x {REF_SAMPLE_STEPS} steps per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measured_peaks() -> dict:
    """The machine's measured copy bandwidth and GEMM rates (MEASURED_PEAKS.json
    at the repository root), or {} when absent."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def run_apply(args, rank, world, dev):
    """Workload apply_6x3: the Lindblad apply kernel alone at the largest state
    size, timed per launch with CUDA events; reports its algorithmic HBM
    bandwidth and FP64 rate against the measured copy bandwidth and the
    derived FP64 peak."""
    import ctypes

    import numpy as np
    import torch

    import workloads as W
    from paper_2110_10310_gb300 import _lib
    from paper_2110_10310_gb300.system import LindbladSystem, colmajor

    n = args.states or 64
    p = W.config5(n_steps=40, n_states=n)
    p.system.T_ns = 300.0 * 40 / 20000
    p.ckpt_every = 10
    s = LindbladSystem(p, device=dev)
    lib = _lib.load()
    V = s.N * s.N
    x = torch.from_numpy(colmajor(p.rho0)).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    h = ctypes.c_void_p(stream.cuda_stream)

    def launch():
        _lib.check(lib.lb_apply(s.h, h, 0, 17, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), n))

    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    ms = []
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    with ClockSampler(gpu_id) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) * 1e-3
    Q = len(p.system.levels)
    n_decay = int(sum(1 for v in p.system.t1_us if np.isfinite(v) and v > 0))
    flops = n * V * (24 * Q + 4 * n_decay + 10)
    nbytes = n * V * 32
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    fp64_peak = FP64_FLOP_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
    if rank == 0:
        line = {
            "metric": "Lindblad apply state-applies/s (FP64)",
            "value": world * n / t,
            "unit": "state-applies/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["apply_6x3"].format(n=n),
                       "l2": "inputs ({:.0f} MB in, {:.0f} MB out) larger than L2".format(nbytes / 2e6, nbytes / 2e6),
                       "flops_per_element": 24 * Q + 4 * n_decay + 10, "bytes_per_element": 32},
            "roofline": {
                "kernel": "k_apply",
                "bound": "alu",
                "achieved": flops / t / 1e12,
                "peak": fp64_peak,
                "unit": "TFLOP/s",
                "frac": flops / t / 1e12 / fp64_peak,
                "hbm_achieved_gbs": nbytes / t / 1e9,
                "hbm_peak_gbs": hbm_peak,
                "hbm_frac": nbytes / t / 1e9 / hbm_peak,
                "traffic": None,
            },
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_optimize(args, rank, world, dev):
    """Workload fock_lbfgs: the L-BFGS loop above the gradient.  Every bench
    step runs the whole optimisation from the same seeded controls (the runs
    are identical); the metric counts the state-steps of every gradient
    evaluation (forward + adjoint) over the wall time of the run."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2110_10310_gb300.system import LindbladSystem

    p = W.fock_superposition()
    s = LindbladSystem(p, device=dev)
    a0 = np.array(p.controls.alpha)
    for _ in range(args.warmup):
        s.gradient()
    torch.cuda.synchronize()
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    secs, res = [], None
    with ClockSampler(gpu_id) as clk:
        for _ in range(args.steps):
            s.set_alpha(a0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = s.optimize(max_iter=150, memory=10, gtol=1e-9, step0=1e-2)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
    st = s.stats()
    state_steps = res["evaluations"] * p.M * p.system.n_steps
    value = world * state_steps * args.steps / sum(secs)
    h = res["history"]
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {
                "workload": WORKLOADS["fock_lbfgs"],
                "l2": "not flushed: the optimisation reuses the same workspace every evaluation",
                "iterations": res["iterations"],
                "gradient_evaluations": res["evaluations"],
                "J_start": float(h[0, 0]),
                "J_final": float(h[-1, 0]),
                "grad_max_start": float(h[0, 1]),
                "grad_max_final": float(h[-1, 1]),
                "ms_per_evaluation": 1e3 * sum(secs) / args.steps / res["evaluations"],
                "sweep": st["sweep"],
                "symmetry": st["symmetry"],
            },
            "gpu_launches": st["kernel_launches"] * res["evaluations"] * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_batch(args, rank, world, dev):
    """Workload batch256: one persistent launch per sweep over 256 uneven
    problems (captured in a CUDA graph), beside the plain form with one
    lb_gradient (its own launches) per problem on one stream."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2110_10310_gb300 import _lib
    from paper_2110_10310_gb300.system import LindbladBatch, LindbladSystem

    probs = W.config3()
    systems = [LindbladSystem(p, sweep=_lib.LB_SWEEP_RESIDENT, device=dev) for p in probs]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        batch = LindbladBatch(systems, stream=stream)
        for _ in range(args.warmup):
            batch.gradient(stream=stream)
        batch.capture(1, stream=stream)
        batch.gradient(stream=stream)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    state_steps = sum(p.M * p.system.n_steps for p in probs)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    ms = []
    with ClockSampler(gpu_id) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                batch.gradient(stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    st = batch.stats()
    total_ms = sum(ms)
    value = world * state_steps * args.steps / (total_ms * 1e-3)
    # plain: every problem on its own launch sequence (best single-problem sweep), one stream
    plain_sys = [LindbladSystem(p, device=dev) for p in probs]
    for s_ in plain_sys[:4]:
        s_.gradient()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s_ in plain_sys:
        s_.gradient()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_value = state_steps / plain_s
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {
                "workload": WORKLOADS["batch256"],
                "problems": len(probs),
                "state_steps_per_step": state_steps,
                "l2": "flushed between timed steps (256 MiB write)",
                "plain_value": plain_value,
                "plain_form": "one lb_gradient per problem, its own launches, one stream, sweep chosen per problem",
                "batched_over_plain": value / plain_value,
                "inner_iters_per_step": st["inner_iterations"] / max(1, st["state_steps"]),
            },
            "gpu_launches": st["kernel_launches"] * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="cnot_2x3", choices=sorted(WORKLOADS))
    ap.add_argument("--states", type=int, default=0,
                    help="initial states of qutrits_6x3 / apply_6x3 (default 64; smaller for ncu captures)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_sample or args.impl == "reference":
        # the oracle runs single-threaded: BLAS pinned to one thread before numpy loads
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            os.environ[k] = "1"
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample)))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2110_10310_gb300 import _lib
    from paper_2110_10310_gb300.system import LindbladSystem, colmajor

    assert args.warmup >= 3 or os.environ.get("LB_BENCH_ALLOW_SHORT_WARMUP"), "need >= 3 warm-up steps"
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    _lib.load(build_if_missing=True)
    dev = torch.device("cuda", local_rank)
    if args.workload == "batch256":
        return run_batch(args, rank, world, dev)
    if args.workload == "fock_lbfgs":
        return run_optimize(args, rank, world, dev)
    if args.workload == "apply_6x3":
        return run_apply(args, rank, world, dev)
    p = problem(workload=args.workload, states=args.states)
    s = LindbladSystem(p, device=dev)
    s.set_timing(True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        s.gradient()
    torch.cuda.synchronize()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None

    state_steps = p.M * p.system.n_steps
    ms_steps, ms_bwd, ms_fwd, launches = [], [], [], 0
    sts = []
    with ClockSampler(gpu_id) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.gradient()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
            st = s.stats()
            sts.append(st)
            ms_bwd.append(st["ms_backward"])
            ms_fwd.append(st["ms_forward"])
            launches += st["kernel_launches"]
    total_ms = sum(ms_steps)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * state_steps * args.steps / (total_ms * 1e-3)

    # end to end through the public API with host buffers: pinned states and
    # controls uploaded every step, G and the gradient read back every step
    pinned = torch.from_numpy(colmajor(p.rho0)).pin_memory()
    alpha = np.ascontiguousarray(p.controls.alpha)
    e2e_s = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        s.set_states_host(pinned, p.weights)
        s.set_alpha(alpha)
        G, g = s.gradient()
        t1 = time.perf_counter()
        if i:
            e2e_s.append(t1 - t0)
    e2e_tot = sum(e2e_s)
    if dist is not None:
        t = torch.tensor([e2e_tot], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = world * state_steps * args.steps / e2e_tot
    h2d = pinned.numel() * 8 + alpha.size * 8
    d2h = 8 + 8 * s.n_params + 64  # G, gradient, status block

    # roofline of the dominant kernel (the backward sweep: recompute + adjoint)
    Q = len(p.system.levels)
    V = s.N * s.N
    n_decay = int(sum(1 for t in p.system.t1_us if np.isfinite(t) and t > 0))
    st = sts[-1]
    Ve = s.N * (s.N + 1) // 2 if st["symmetry"] == "hermitian" else V
    bwd_flops = fp64_flops(Ve, Q, n_decay, st, (1, 2))
    fwd_flops = fp64_flops(Ve, Q, n_decay, st, (0,))
    bwd_ms = statistics.median(ms_bwd)
    peak = FP64_FLOP_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
    achieved = bwd_flops / (bwd_ms * 1e-3) / 1e12
    kernel_name = {"grid": "k_backward_grid", "cluster": "k_backward_cl"}.get(st["sweep"], "k_backward_res")
    traffic = traffic_record(kernel_name)
    clocks = clk.summary()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "cnot_2x3":
        r = oracle_subprocess(CPU_SAMPLE_STEPS)
        cpu = {"value": r["state_steps"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"dense-LU oracle gradient (forward + adjoint), 16 states x {CPU_SAMPLE_STEPS} of the "
                         f"10000 steps at the same dt, one thread, {r['seconds']:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {
                "workload": WORKLOADS[args.workload].format(n=p.system.n_steps, m=p.M),
                "states": p.M,
                "n_steps": p.system.n_steps,
                "ckpt_every": st["ckpt_every"],
                "tape_bytes": (p.M * p.system.n_steps * V * 16 if st["ckpt_every"] == 0
                               else p.M * (-(-p.system.n_steps // st["ckpt_every"]) + st["ckpt_every"]) * V * 16),
                "solver": f"{st['solver']} fixed point, rtol 1e-15",
                "sweep": st["sweep"],
                "symmetry": st["symmetry"],
                "workspace_bytes": s.workspace_bytes,
                "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev)),
                "l2": "flushed between timed steps (256 MiB write)",
                "parallelism": f"replicas{world}" if world > 1 else "single",
                "inner_iters_per_step": st["inner_iterations"] / max(1, st["state_steps"]),
                "ms_forward_kernel": statistics.median(ms_fwd),
                "ms_backward_kernel": bwd_ms,
                "fwd_fp64_tflops": fwd_flops / (statistics.median(ms_fwd) * 1e-3) / 1e12,
            },
            "roofline": {
                "kernel": kernel_name,
                "bound": "alu",
                "achieved": achieved,
                "peak": peak,
                "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic,
                "peak_source": "FP64 pipe: 2 FMA lanes/SM/clk x 2 flops x 152 SMs x 2070 MHz (derived)",
            },
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
