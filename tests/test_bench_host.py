"""Host-side pieces of bench.py that need no GPU: the kernel-code digest that
keys the ncu traffic record, the algorithmic FP64 count, and the workload
table."""

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


def test_traffic_record_is_keyed_on_the_kernel_code():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_backward_cl"]
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    src = os.path.join(ROOT, "paper_2110_10310_gb300", "csrc", "lb_kernels.cu")
    got = bench.traffic_record("k_backward_cl")
    # the record applies exactly when it was taken on the current kernel code
    assert (got is not None) == (rec["code_sha256"] == bench.kernel_source_digest(src))


def test_fp64_count_matches_its_definition():
    """Per element and inner iteration 24 flops per subsystem, 4 per decaying
    subsystem and 8 more; per element and step 10; the adjoint adds 28 per
    subsystem per step."""
    st = {"phase_steps": [5, 0, 5], "phase_iterations": [7, 0, 9]}
    V, Q, nd = 81, 2, 2
    per_it = 24 * Q + 4 * nd + 8
    assert bench.fp64_flops(V, Q, nd, st, (0,)) == V * (10 * 5 + per_it * 7)
    assert bench.fp64_flops(V, Q, nd, st, (1, 2)) == V * (10 * 5 + per_it * 9) + V * 28 * Q * 5


def test_every_workload_has_a_description_and_builds():
    for w in bench.WORKLOADS:
        assert bench.WORKLOADS[w].startswith(w + ":")
    for w in ("cnot_2x3", "qubit_x", "cnot_3states", "cnot_penalty", "cnot_jc"):
        p = bench.problem(workload=w)
        assert p.M > 0 and p.system.n_steps > 0
    p = bench.problem(workload="qudits_4x4")
    assert p.system.n_steps == bench.PREFIX["qudits_4x4"]
