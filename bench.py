#!/usr/bin/env python3
"""Benchmark of the implicit-midpoint Lindblad path on GB300.

Default workload (the largest single-GPU configuration of the method's
targets): 6 qutrits (N = 729, vec(rho) of length 531441, complex FP64),
64 random pure initial states, ring cross-Kerr, dt = 0.015 ns, 40 splines x 2
carriers per qutrit, J_Frob to a random pure target, checkpoints every 100
steps.  One bench step = one forward sweep plus the checkpointed discrete
adjoint gradient (Appendices A-B) over the first 200 of the 20000 steps, so
that two checkpoint segments, their recompute and the adjoint all run in the
timed region.  Metric: state-steps/s of forward + adjoint (64 x 200 per step);
the line also gives the forward-only rate.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm).  Under torchrun the initial states are split over the ranks
(the paper's first level of parallelism) and (G, dG/dalpha) are summed with one
all-reduce, the path's only exchange.
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
DEFAULT_WORKLOAD = "qutrits_6x3"
WORKLOADS = {
    "qutrits_6x3": ("qutrits_6x3: 6 qutrits (N=729, vec 531441), {m} random pure states, ring cross-Kerr 0.003 GHz, "
                    "T1 in [40,80] us, T2=T1/2, dt=0.015 ns, first {n} of 20000 steps, 6 controls x 2 carriers x "
                    "40 splines, J_Frob to a random pure target, fwd + adjoint gradient with checkpoints every "
                    "{k} steps, grid-wide sweep"),
    "cnot_2x3": ("cnot_2x3: 2 transmons x 3 levels (N=9, vec 81), 16 essential-basis states |i><j|, "
                 "10000 IMR steps, T=200 ns, 2x20 splines x 2 carriers, J_Frob to CNOT, "
                 "forward + adjoint gradient (stage vectors kept when the tape fits 8 GiB, else checkpoints)"),
    "cnot_3states": ("cnot_3states: the cnot_2x3 system and controls with the three-state gate objective "
                     "(Sec. III-C: 3 Hermitian states, weights 20, 1, 1), 10000 steps, fwd + adjoint"),
    "reset_2x2x20": ("reset_2x2x20: 2 qubits + 20-level cavity (vec 6400) from the ensemble state, J_N0, "
                     "dt=0.05 ns, first {n} of 100000 steps, 100 splines, fwd + adjoint, grid-wide sweep"),
    "qubit_x": "qubit_x: 1 qubit (vec 4), 4 states |i><j|, 1000 steps, T=100 ns, X gate, fwd + adjoint",
    "batch256": ("batch256: 256 independent problems, Q in {1,2,3}, 2-4 levels (vec 4..4096), 3 random pure states "
                 "each, 5000 steps, T=100 ns, fwd + adjoint, one persistent launch per sweep captured in a CUDA graph"),
    "qudits_4x4": ("qudits_4x4: 4 qudits x 4 levels (vec 65536), 3 random pure states, dt=0.0125 ns, "
                   "first {n} of 40000 steps, fwd + adjoint with checkpoints every {k} steps, grid-wide sweep"),
    "apply_6x3": ("apply_6x3: y = M(t) x, the matrix-free Lindblad apply (lb_apply, one thread per element) on "
                  "{n} states of 6 qutrits (vec 531441, 8.5 MB each), x and y in HBM"),
    "cnot_penalty": ("cnot_penalty: the cnot_2x3 workload with the running penalty gamma1 int beta(t) J dt "
                     "(gamma1 = 0.1, a = 20 ns: Sec. III, eq. optimproblem), fwd + adjoint"),
    "cnot_jc": ("cnot_jc: the cnot_2x3 workload with a Jaynes-Cummings coupling of the two transmons "
                "(g = 5 MHz, rotating frequencies 4.80 and 4.86 GHz: the coupling rotates at 60 MHz), "
                "fwd + adjoint"),
    "fock_lbfgs": ("fock_lbfgs: one 4-level qudit |0> -> (|0>+|3>)/sqrt 2, J_Frob, 10 splines x 2 carriers, "
                   "T=200 ns, 10000 steps; one bench step = one L-BFGS run (lb_optimize, memory 10, "
                   "at most 150 iterations, gtol 1e-9) from the seeded controls"),
}
PREFIX = {"qudits_4x4": 2000, "qutrits_6x3": 200, "reset_2x2x20": 2000}
FP64_FLOP_PER_CLK_PER_SM = 4.0  # 2 FP64 FMA lanes per SM per clock, 2 flops each
E2E_STEPS = 3  # end-to-end steps through host buffers (each re-uploads every state)
CPU_SAMPLE_STEPS = 8000  # cnot_2x3 oracle sample (same dt, 16 states)
REF_SAMPLE_STEPS = 400  # cnot_2x3 oracle sample per reference-arm step
REDUCED_LEVELS = (2, 2, 2, 2, 2, 2)  # qutrits_6x3 reduced to qubits for the dense oracle (vec 4096)
REDUCED_STEPS = 1  # oracle steps per reduced-shape sample


def problem(n_steps=None, workload=DEFAULT_WORKLOAD, states=0, levels=None):
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
        p = W.config5(n_states=states or 64, levels=levels or (3,) * 6)
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
        # the first n_steps steps of the workload at its step size dt; the
        # controls stay those of the whole horizon
        W.prefix(p, n_steps)
    return p


def static_config(workload: str, p) -> dict:
    """The workload as both arms name it (the reference arm prints the same)."""
    K = p.ckpt_every
    c = {"workload": WORKLOADS[workload].format(n=p.system.n_steps, m=p.M, k=K), "states": p.M,
         "n_steps": p.system.n_steps, "ckpt_every": K,
         "l2": "flushed between timed steps (256 MiB write)"}
    return c


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)


def oracle_sample(workload: str, n_steps: int, states: int = 0) -> dict:
    """One oracle gradient (forward + adjoint, dense LU steps) on the sample
    shape of ``workload``: the workload's first n_steps steps, or for
    qutrits_6x3 its structure reduced to 2 levels per subsystem (vec 4096)."""
    from oracle import imr

    if workload == "qutrits_6x3":
        p = problem(n_steps, workload, states=states, levels=REDUCED_LEVELS)
    else:
        p = problem(n_steps, workload)
    t0 = time.perf_counter()
    imr.gradient(p)
    dt = time.perf_counter() - t0
    N = 1
    for n in p.system.levels:
        N *= n
    return {"seconds": dt, "state_steps": p.M * n_steps, "vec": N * N}


def _thread_env(threads: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def oracle_subprocess(workload: str, n_steps: int, threads: int, states: int = 0) -> dict:
    """Run one oracle sample in a fresh process with BLAS pinned to ``threads``
    threads (spawned, never forked from a process that touched the GPU)."""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_steps),
                          "--workload", workload, "--states", str(states)],
                         capture_output=True, text=True, env=_thread_env(threads), check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def extrapolate_dense(rate: float, vec_sample: int, vec_full: int) -> float:
    """State-steps/s of the dense-LU oracle extrapolated from a sample of vec
    length vec_sample to vec_full: a step's cost is dominated by the LU
    factorisation of the vec x vec matrix, which grows as vec^3."""
    return rate * (vec_sample / vec_full) ** 3


def cpu_baseline(workload: str, p) -> dict | None:
    cores = os.cpu_count() or 1
    if workload == "qutrits_6x3":
        r1 = oracle_subprocess(workload, REDUCED_STEPS, 1, states=p.M)
        rn = oracle_subprocess(workload, REDUCED_STEPS, cores, states=p.M)
        vfull = 729 * 729
        v1 = r1["state_steps"] / r1["seconds"]
        vn = rn["state_steps"] / rn["seconds"]
        return {"value": extrapolate_dense(vn, rn["vec"], vfull), "unit": UNIT, "cores": cores, "kind": "oracle",
                "extrapolated": True,
                "sample": (f"dense-LU oracle gradient (forward + adjoint) on the workload's structure reduced to "
                           f"2 levels per subsystem (6 qubits, vec {rn['vec']}), {p.M} states x {REDUCED_STEPS} step "
                           f"at dt = 0.015 ns: {vn:.3g} state-steps/s on {cores} threads ({rn['seconds']:.1f} s), "
                           f"{v1:.3g} on 1 thread ({r1['seconds']:.1f} s); value extrapolated to vec 531441 by the "
                           f"vec^3 cost of the dense LU (a dense 531441^2 matrix is 4.5 TB)"),
                "measured_reduced_all_cores": vn, "measured_reduced_one_thread": v1,
                "one_thread_extrapolated": extrapolate_dense(v1, r1["vec"], vfull), "nproc": cores}
    if workload == "cnot_2x3":
        r1 = oracle_subprocess(workload, CPU_SAMPLE_STEPS, 1)
        return {"value": r1["state_steps"] / r1["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "nproc": cores,
                "sample": f"dense-LU oracle gradient (forward + adjoint), 16 states x {CPU_SAMPLE_STEPS} of the "
                          f"10000 steps at the same dt, one thread, {r1['seconds']:.1f} s"}
    return None


# ----------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id
        self.lines = []

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


def gpu_uuid(dev):
    import torch

    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


# ----------------------------------------------------------------------------
# algorithmic work of the sweep kernels


def fp64_iterations(st: dict, ph: int) -> int:
    """Inner iterations of phase ``ph`` computed in FP64: all but the
    single-precision difference iterations of the grid sweeps."""
    return st["phase_iterations"][ph] - st.get("phase_diff_iterations", [0, 0, 0])[ph]


def fp64_flops(V: int, Q: int, n_decay: int, st: dict, phase_set) -> float:
    """FP64 flops (FMA = 2) of the Jacobi sweeps as the kernels compute them,
    from the iteration counts.

    Per element and FP64 inner iteration: per subsystem 24 flops for the
    control term (two real-weighted neighbour pairs P, R and the complex
    control factor) plus 4 for the decay sandwich when T1 is finite; 6 for
    the multiplication by (I - dt/2 D)^-1 and 2 for the convergence
    difference.  Per element and difference iteration: 4 (the single-precision
    changes added to the FP64 iterate and correction).  Per element and step:
    6 for the initial guess, 4 for q <- 2z - q, and for adjoint steps per
    subsystem 28 flops for the gradient pieces (24 under the Hermitian
    symmetry, which sums the g_ad piece as the conjugate of the g_a piece).
    ``V`` is the number of elements a state's sweep computes: N^2, or
    N (N + 1) / 2 when the Hermitian symmetry leaves the others as mirrored
    copies."""
    per_it = 24 * Q + 4 * n_decay + 8
    herm = st.get("symmetry") == "hermitian"
    f = 0.0
    for ph in phase_set:
        dits = st["phase_iterations"][ph] - fp64_iterations(st, ph)
        f += V * (10 * st["phase_steps"][ph] + per_it * fp64_iterations(st, ph) + 4 * dits)
        if ph == 2:
            f += V * (24 if herm else 28) * Q * st["phase_steps"][ph]
    return f


def method_flops(V: int, Q: int, st: dict, phase_set) -> float:
    """Algorithmic FP64 flops by the method's own count: one Lindblad apply
    costs 8 + 36 Q flops per element (a complex diagonal term and, per
    subsystem, the decay sandwich and the four control neighbours with their
    complex factors), one per FP64 inner iteration (the single-precision
    difference iterations of the grid sweeps are not counted); every adjoint
    step adds the gradient pieces of eq. reducedgradient, 28 Q per element
    (the two commutator combinations of each subsystem and their two complex
    dot products).  ``V``: elements the sweep computes (see fp64_flops)."""
    f = 0.0
    for ph in phase_set:
        f += V * (8 + 36 * Q) * fp64_iterations(st, ph)
        if ph == 2:
            f += V * 28 * Q * st["phase_steps"][ph]
    return f


BYTES_PER_ELEMENT_ITERATION = 48  # read the iterate and the right-hand side, write the new iterate


def kernel_source_digest(path: str) -> str:
    """SHA-256 of a kernel source with its // comments and blank lines
    removed: the counters stay valid across comment edits, not across code
    edits.  (The kernel sources have no block comments and no // inside
    string literals.)"""
    lines = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


KERNEL_SOURCES = {
    "k_backward_grid": ("lb_grid.cu", "lb_device.cuh"),
    "k_sweep_grid": ("lb_grid.cu", "lb_device.cuh"),
    # the paired-single instantiations (lb_set_precision LB_PREC_F32X2)
    "k_backward_grid_f32x2": ("lb_grid.cu", "lb_device.cuh"),
    "k_sweep_grid_f32x2": ("lb_grid.cu", "lb_device.cuh"),
    "k_backward_cl": ("lb_cluster.cu", "lb_device.cuh"),
    "k_forward_cl": ("lb_cluster.cu", "lb_device.cuh"),
    "k_backward_res": ("lb_resident.cu", "lb_device.cuh"),
    "k_forward_res": ("lb_resident.cu", "lb_device.cuh"),
}


def kernel_digest(kernel: str) -> str:
    csrc = os.path.join(ROOT, "paper_2110_10310_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel] + ("lb_internal.h",):
        h.update(kernel_source_digest(os.path.join(csrc, f)).encode())
    return h.hexdigest()


def traffic_record(kernel: str, workload: str):
    """The committed ncu DRAM record of ``kernel`` on ``workload``, or None
    when there is none or the kernel code changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel}@{workload}")
    if not rec or rec.get("code_sha256") != kernel_digest(kernel):
        return None
    return rec


# ----------------------------------------------------------------------------


def run_reference(args, rank: int, world: int):
    """The reference arm: the dense-LU CPU oracle, timed as it stands on the
    host cores, on a bounded sample of the same workload per step."""
    if rank != 0:
        return
    wl = args.workload
    p = problem(workload=wl, states=args.states)
    cores = os.cpu_count() or 1
    if wl == "qutrits_6x3":
        def sample():
            return oracle_sample(wl, REDUCED_STEPS, states=p.M)
        sdesc = (f"per step: dense-LU oracle gradient on the workload reduced to 2 levels per subsystem "
                 f"(6 qubits, vec 4096), {p.M} states x {REDUCED_STEPS} step, all {cores} threads; the value is "
                 f"extrapolated to vec 531441 by the vec^3 cost of the dense LU")
    else:
        def sample():
            return oracle_sample(wl, REF_SAMPLE_STEPS)
        sdesc = f"per step: dense-LU oracle gradient, first {REF_SAMPLE_STEPS} steps of the workload, 1 thread"
    for _ in range(args.warmup):
        sample()
    tot_s, tot_ss, vec = 0.0, 0, 0
    for _ in range(args.steps):
        r = sample()
        tot_s += r["seconds"]
        tot_ss += r["state_steps"]
        vec = r["vec"]
    rate = tot_ss / tot_s
    value = extrapolate_dense(rate, vec, 729 * 729) if wl == "qutrits_6x3" else rate
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
        "scaling": "strong" if wl == "qutrits_6x3" else "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": static_config(wl, p),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores if wl == "qutrits_6x3" else 1,
                         "kind": "oracle", "sample": sdesc, "measured_sample_rate": rate,
                         "extrapolated": wl == "qutrits_6x3"},
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


def fp64_peak_tflops(dev, sm_mhz: float | None) -> tuple[float, str]:
    """FP64 pipe peak of this GPU: 4 flops per SM per clock x the SM count
    the device reports x the median SM clock sampled during the timed region
    (the maximum clock when no sample was taken)."""
    import torch

    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or measured_peaks().get("sm_max_mhz") or 2070.0
    src = (f"FP64 pipe: 2 FMA lanes/SM/clk x 2 flops x {nsm} SMs (queried) x {mhz:.0f} MHz "
           f"({'median sampled in the timed region' if sm_mhz else 'maximum clock'}); derived")
    return FP64_FLOP_PER_CLK_PER_SM * nsm * mhz * 1e6 / 1e12, src


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
    p = W.prefix(W.config5(n_states=n), 40)
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
    with ClockSampler(gpu_uuid(dev)) as clk:
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
    clocks = clk.summary()
    fp64_peak, src = fp64_peak_tflops(dev, clocks["sm_mhz"] if clocks else None)
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
                "peak_source": src,
                "hbm_achieved_gbs": nbytes / t / 1e9,
                "hbm_peak_gbs": hbm_peak,
                "hbm_frac": nbytes / t / 1e9 / hbm_peak,
                "traffic": None,
            },
            "gpu_launches": args.steps,
            "clocks": clocks,
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
    secs, res = [], None
    with ClockSampler(gpu_uuid(dev)) as clk:
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
    ms = []
    with ClockSampler(gpu_uuid(dev)) as clk:
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


def run_gradient(args, rank, world, dev, dist):
    """Workloads timed as one lb_gradient per bench step (the default and the
    single-problem ones).  With several ranks each rank holds its share of
    the initial states and the per-rank (G, dG/dalpha) are summed."""
    import numpy as np
    import torch

    from paper_2110_10310_gb300 import _lib
    from paper_2110_10310_gb300 import dist as D
    from paper_2110_10310_gb300.system import LindbladSystem, colmajor

    wl = args.workload
    full = problem(n_steps=args.n_steps, workload=wl, states=args.states)
    if args.ckpt is not None:
        full.ckpt_every = args.ckpt
    p = D.shard_problem(full, rank, world) if world > 1 else full
    s = LindbladSystem(p, device=dev, predictor=args.predictor, pred_order=args.pred_order,
                       difference_iterations=1 if args.diff_iterations == "on" else 0,
                       precision=_lib.LB_PREC_F32X2 if args.precision == "f32x2" else _lib.LB_PREC_F64)
    tuned = None
    if args.autotune == "on" or (args.autotune == "auto" and wl in ("qutrits_6x3", "qudits_4x4") and not args.pred_order):
        # the library's autotuner (outside the timed region): sweep, inner
        # solver and, on grid sweeps, the predictor's order
        tuned = s.autotune()
    s.set_timing(True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()

    def step():
        G, g = s.gradient()
        if dist is not None:
            G, g = D.allreduce_objective(G, g)
        return G, g

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    state_steps = full.M * full.system.n_steps
    ms_steps, ms_bwd, ms_fwd, launches, sts = [], [], [], 0, []
    with ClockSampler(gpu_uuid(dev)) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
            st = s.stats()
            sts.append(st)
            ms_bwd.append(st["ms_backward"])
            ms_fwd.append(st["ms_forward"])
            launches += st["kernel_launches"]
    clocks = clk.summary()

    def maxrank(x):
        if dist is None:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    total_ms = maxrank(sum(ms_steps))
    value = state_steps * args.steps / (total_ms * 1e-3)
    fwd_ms = maxrank(statistics.median(ms_fwd))
    bwd_ms = statistics.median(ms_bwd)

    # end to end through the public API with host buffers: pinned states and
    # controls uploaded every step, G and the gradient read back every step
    pinned = torch.from_numpy(colmajor(p.rho0)).pin_memory()
    alpha = np.ascontiguousarray(p.controls.alpha)
    e2e_n = 0 if args.no_e2e else min(args.steps, E2E_STEPS)
    e2e_s = []
    for i in range(e2e_n + 1 if e2e_n else 0):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        s.set_states_host(pinned, p.weights)
        s.set_alpha(alpha)
        step()
        t1 = time.perf_counter()
        if i:
            e2e_s.append(t1 - t0)
    e2e_tot = maxrank(sum(e2e_s))
    e2e_value = state_steps * e2e_n / e2e_tot if e2e_n else None
    h2d = pinned.numel() * 8 + alpha.size * 8 + (0 if p.weights is None else 8 * p.M)
    d2h = 8 + 8 * s.n_params + 64  # G, gradient, status block

    # roofline of the dominant kernel, the backward sweep (recompute + adjoint)
    Q = len(p.system.levels)
    V = s.N * s.N
    n_decay = int(sum(1 for t in p.system.t1_us if np.isfinite(t) and t > 0))
    st = sts[-1]
    Ve = s.N * (s.N + 1) // 2 if st["symmetry"] == "hermitian" else V
    kernel_name = {"grid": "k_backward_grid", "cluster": "k_backward_cl"}.get(st["sweep"], "k_backward_res")
    bwd_method = method_flops(Ve, Q, st, (1, 2))
    bwd_impl = fp64_flops(Ve, Q, n_decay, st, (1, 2))
    fwd_method = method_flops(Ve, Q, st, (0,))
    fp64_peak, peak_src = fp64_peak_tflops(dev, clocks["sm_mhz"] if clocks else None)
    achieved = bwd_method / (bwd_ms * 1e-3) / 1e12
    elem_iters = Ve * (st["phase_iterations"][1] + st["phase_iterations"][2])
    hbm_alg = BYTES_PER_ELEMENT_ITERATION * elem_iters
    hbm_peak = measured_peaks().get("hbm_gbs") or 6800.0
    # the DRAM record of the instantiation that ran (FP64 or paired-single apply)
    trec = traffic_record(kernel_name + ("_f32x2" if args.precision == "f32x2" and kernel_name.endswith("grid") else ""),
                          wl)
    traffic = None
    if trec:
        # DRAM bytes of the capture scaled to this launch by the element-iterations
        traffic = trec["dram_bytes"] / trec["element_iterations"] * elem_iters
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, p)

    if rank == 0:
        inner = {ph: st["phase_iterations"][i] / max(1, st["phase_steps"][i])
                 for i, ph in enumerate(("forward", "recompute", "adjoint"))}
        diff = {ph: st["phase_diff_iterations"][i] / max(1, st["phase_steps"][i])
                for i, ph in enumerate(("forward", "recompute", "adjoint"))}
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == "f64" else "f64+f32x2",
            "data": "synthetic",
            "config": static_config(wl, full),
            "fwd_value": full.M * full.system.n_steps / (fwd_ms * 1e-3),
            "fwd_unit": "state-steps/s (forward sweep kernel alone, device-timed inside lb_gradient)",
            "detail": {
                "parallelism": f"states sharded over {world} ranks, (G, grad) all-reduced" if world > 1 else "single",
                "sweep": st["sweep"],
                "symmetry": st["symmetry"],
                "solver": f"{st['solver']} fixed point, rtol 1e-15",
                "ckpt_every": st["ckpt_every"],
                "predictor": args.predictor,
                "pred_order": (tuned or {}).get("pred_order", args.pred_order or 8),
                "autotune": tuned,
                "inner_iters_per_step": inner,
                "diff_iters_per_step": diff,
                "precision": ("FP64 states, corrections, objective, gradient and stopping rule; inner iterations "
                              "after the first of a step apply O to the single-precision change of the iterate "
                              "once it is below 2^-32 max|q| (lb_set_difference_iterations)"
                              if args.diff_iterations == "on" else "FP64 throughout")
                             + ("; the other inner iterations apply O in pairs of single-precision numbers "
                                "(about 48 significant bits, lb_set_precision LB_PREC_F32X2)"
                                if args.precision == "f32x2" else ""),
                "ms_forward_kernel": statistics.median(ms_fwd),
                "ms_backward_kernel": bwd_ms,
                "workspace_bytes": s.workspace_bytes,
                "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev)),
                "fwd_fp64_tflops_method_count": fwd_method / (statistics.median(ms_fwd) * 1e-3) / 1e12,
            },
            "roofline": {
                "kernel": kernel_name,
                "bound": "alu",
                "achieved": achieved,
                "peak": fp64_peak,
                "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "peak_source": peak_src,
                "flop_count": ("method count: (8 + 36 Q) per element per FP64 inner iteration (difference "
                               "iterations not counted) + 28 Q per element per adjoint step (gradient pieces), "
                               "over the elements the sweep computes "
                               f"({Ve} per state: {'k <= l under the Hermitian symmetry' if Ve != V else 'all'})"),
                "frac_instruction_count": bwd_impl / (bwd_ms * 1e-3) / 1e12 / fp64_peak,
                "hbm_achieved_gbs": hbm_alg / (bwd_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": hbm_peak,
                "hbm_frac": hbm_alg / (bwd_ms * 1e-3) / 1e9 / hbm_peak,
                "hbm_bytes_count": f"{BYTES_PER_ELEMENT_ITERATION} B per element per inner iteration",
                "traffic": traffic,
                "traffic_source": (trec or {}).get("command"),
            },
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_n},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (long single runs)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--states", type=int, default=0,
                    help="initial states of qutrits_6x3 / apply_6x3 (default 64; fewer for ncu captures)")
    ap.add_argument("--ckpt", type=int, default=None, help="checkpoint interval (default: the workload's)")
    ap.add_argument("--n-steps", type=int, default=None,
                    help="steps of the prefix (default: the workload's; smaller for ncu captures)")
    ap.add_argument("--predictor", type=int, default=-1,
                    help="forward predictor restart period (lb_set_predictor; -1 auto, -2 none)")
    ap.add_argument("--pred-order", type=int, default=0, help="predictor order (lb_set_predictor; 0: default)")
    ap.add_argument("--diff-iterations", default="on", choices=["on", "off"],
                    help="single-precision difference iterations of the grid sweeps (lb_set_difference_iterations)")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32x2"],
                    help="arithmetic of the grid sweeps' FP64 inner iterations (lb_set_precision)")
    ap.add_argument("--autotune", default="auto", choices=["auto", "on", "off"],
                    help="run lb_autotune before timing (auto: on for the grid-sweep workloads)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.workload, args.oracle_sample, states=args.states)))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.workload != "qutrits_6x3":
            # the short-horizon samples run on one thread: BLAS pinned before numpy loads
            os.environ.update({k: v for k, v in _thread_env(1).items() if k.endswith("_NUM_THREADS")})
        run_reference(args, rank, world)
        return

    import torch

    from paper_2110_10310_gb300 import _lib

    assert args.warmup >= 3 or os.environ.get("LB_BENCH_ALLOW_SHORT_WARMUP"), "need >= 3 warm-up steps"
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    _lib.load(build_if_missing=True)
    dev = torch.device("cuda", local_rank)
    try:
        if args.workload == "batch256":
            run_batch(args, rank, world, dev)
        elif args.workload == "fock_lbfgs":
            run_optimize(args, rank, world, dev)
        elif args.workload == "apply_6x3":
            run_apply(args, rank, world, dev)
        else:
            run_gradient(args, rank, world, dev, dist)
    finally:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
