"""Host-side pieces of bench.py that need no GPU: the kernel-code digest that
keys the ncu traffic records, the algorithmic FP64 counts, the oracle
extrapolation and the workload table."""

import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_digest_ignores_comments_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\n__global__ void k(double* x) {\n  x[0] = 1.0;  // one\n}\n")
    b.write_text("__global__ void k(double* x) {\n\n  // a new comment\n  x[0] = 1.0;\n}\n")
    c.write_text("__global__ void k(double* x) {\n  x[0] = 2.0;\n}\n")
    assert bench.kernel_source_digest(str(a)) == bench.kernel_source_digest(str(b))
    assert bench.kernel_source_digest(str(a)) != bench.kernel_source_digest(str(c))


def test_traffic_records_are_keyed_on_the_kernel_code():
    path = os.path.join(ROOT, "profiles", "traffic.json")
    recs = json.load(open(path))
    for key, rec in recs.items():
        kernel, workload = key.split("@")
        assert kernel in bench.KERNEL_SOURCES and workload in bench.WORKLOADS
        assert rec["dram_bytes"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
        assert rec["element_iterations"] > 0
        got = bench.traffic_record(kernel, workload)
        # the record applies exactly when it was taken on the current kernel code
        assert (got is not None) == (rec["code_sha256"] == bench.kernel_digest(kernel))


def test_fp64_counts_match_their_definitions():
    """Instruction count: per element and inner iteration 24 flops per
    subsystem, 4 per decaying subsystem and 8 more; per element and step 10;
    the adjoint adds 28 per subsystem per step.  Method count: 8 + 36 Q per
    element and inner iteration, 28 Q per element and adjoint step."""
    st = {"phase_steps": [5, 0, 5], "phase_iterations": [7, 0, 9]}
    V, Q, nd = 81, 2, 2
    per_it = 24 * Q + 4 * nd + 8
    assert bench.fp64_flops(V, Q, nd, st, (0,)) == V * (10 * 5 + per_it * 7)
    assert bench.fp64_flops(V, Q, nd, st, (1, 2)) == V * (10 * 5 + per_it * 9) + V * 28 * Q * 5
    assert bench.method_flops(V, Q, st, (0,)) == V * 80 * 7
    assert bench.method_flops(V, Q, st, (1, 2)) == V * 80 * 9 + V * 56 * 5


def test_difference_iterations_are_not_counted_as_fp64_applies():
    """A single-precision difference iteration adds 4 FP64 flops per element
    to the instruction count and nothing to the method count; the Hermitian
    symmetry's gradient pieces take 24 flops per subsystem."""
    st = {"phase_steps": [5, 0, 5], "phase_iterations": [7, 0, 9], "phase_diff_iterations": [2, 0, 3],
          "symmetry": "hermitian"}
    V, Q, nd = 81, 2, 2
    per_it = 24 * Q + 4 * nd + 8
    assert bench.fp64_flops(V, Q, nd, st, (0,)) == V * (10 * 5 + per_it * 5 + 4 * 2)
    assert bench.fp64_flops(V, Q, nd, st, (2,)) == V * (10 * 5 + per_it * 6 + 4 * 3) + V * 24 * Q * 5
    assert bench.method_flops(V, Q, st, (0,)) == V * 80 * 5
    assert bench.method_flops(V, Q, st, (1, 2)) == V * 80 * 6 + V * 56 * 5


def test_dense_oracle_extrapolation_is_cubic():
    assert bench.extrapolate_dense(8.0, 4096, 8192) == 1.0
    assert abs(bench.extrapolate_dense(2.0, 4096, 531441) - 2.0 / (531441 / 4096) ** 3) < 1e-20


def test_every_workload_has_a_description_and_builds():
    for w in bench.WORKLOADS:
        assert bench.WORKLOADS[w].startswith(w + ":")
    for w in ("cnot_2x3", "qubit_x", "cnot_3states", "cnot_penalty", "cnot_jc"):
        p = bench.problem(workload=w)
        assert p.M > 0 and p.system.n_steps > 0
    p = bench.problem(workload="qudits_4x4")
    assert p.system.n_steps == bench.PREFIX["qudits_4x4"]
    # the default line: the six-qutrit workload at its stated shape over a
    # prefix of two checkpoint segments
    assert bench.DEFAULT_WORKLOAD == "qutrits_6x3"
    p = bench.problem(workload="qutrits_6x3", states=2)
    assert p.system.levels == (3,) * 6 and p.ckpt_every == 100
    assert p.system.n_steps == 200 and abs(p.system.T_ns / p.system.n_steps - 0.015) < 1e-15
    c = bench.static_config("qutrits_6x3", p)
    assert "first 200 of 20000 steps" in c["workload"] and "every 100 steps" in c["workload"]
