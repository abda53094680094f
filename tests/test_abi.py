"""The C-ABI library loads, exports every symbol the header declares, and its
host-side validation behaves as documented.  No device call is made."""

import ctypes
import os
import re
from ctypes import POINTER, byref, c_double, c_int32, c_size_t, c_void_p

import numpy as np
import pytest

import workloads as W
from paper_2110_10310_gb300 import _lib as L
from paper_2110_10310_gb300.system import colmajor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lindblad_gb300.h")


@pytest.fixture(scope="module")
def lib():
    return L.load(build_if_missing=True)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, n
    assert set(L.SIGNATURES) == set(names)
    assert b"sm_103a" in lib.lb_version()


def _desc(sysm, keep):
    def arr(x, ct, dt):
        a = np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep.append(a)
        return a.ctypes.data_as(POINTER(ct))

    Q = len(sysm.levels)
    d = L.lb_system_desc()
    d.Q = Q
    d.levels = arr(sysm.levels, c_int32, np.int32)
    d.essential = arr(sysm.essential, c_int32, np.int32) if sysm.essential is not None else None
    d.detuning_ghz = arr(sysm.detuning_ghz, c_double, np.float64)
    d.selfkerr_ghz = arr(sysm.selfkerr_ghz, c_double, np.float64)
    d.crosskerr_ghz = arr(np.asarray(sysm.crosskerr_ghz).reshape(-1), c_double, np.float64)
    d.t1_us = arr(sysm.t1_us, c_double, np.float64)
    d.t2_us = arr(sysm.t2_us, c_double, np.float64)
    d.T_ns = sysm.T_ns
    d.n_steps = sysm.n_steps
    return d


def _make(lib, prob, K=100):
    keep = []
    d = _desc(prob.system, keep)
    h = c_void_p()
    L.check(lib.lb_system_create(byref(d), byref(h)))
    c = prob.controls
    nf = np.array([len(x) for x in c.carriers_ghz], dtype=np.int32)
    car = np.concatenate(c.carriers_ghz).astype(np.float64)
    L.check(lib.lb_controls_define(h, c.n_splines, nf.ctypes.data_as(POINTER(c_int32)),
                                   car.ctypes.data_as(POINTER(c_double))))
    a = np.ascontiguousarray(c.alpha)
    L.check(lib.lb_controls_set(h, a.ctypes.data_as(POINTER(c_double)), a.size))
    r = colmajor(prob.rho0)
    L.check(lib.lb_states_set(h, prob.M, r.ctypes.data_as(c_void_p), None))
    L.check(lib.lb_solver_set(h, 0, 1e-15, 200, K))
    return h


def test_create_validation(lib):
    p = W.config2(n_steps=10)
    keep = []
    h = c_void_p()
    d = _desc(p.system, keep)
    d.Q = 0
    assert lib.lb_system_create(byref(d), byref(h)) == L.LB_EINVAL
    assert b"Q" in lib.lb_last_error()
    d = _desc(p.system, keep)
    d.n_steps = 0
    assert lib.lb_system_create(byref(d), byref(h)) == L.LB_EINVAL
    d = _desc(p.system, keep)
    d.T_ns = -1.0
    assert lib.lb_system_create(byref(d), byref(h)) == L.LB_EINVAL
    bad = np.array([3, 1], dtype=np.int32)
    d = _desc(p.system, keep)
    d.levels = bad.ctypes.data_as(POINTER(c_int32))
    assert lib.lb_system_create(byref(d), byref(h)) == L.LB_EINVAL
    big = np.array([16, 16, 16, 16], dtype=np.int32)
    p4 = W.config4(n_steps=10)
    d = _desc(p4.system, keep)
    d.levels = big.ctypes.data_as(POINTER(c_int32))
    assert lib.lb_system_create(byref(d), byref(h)) == L.LB_EINVAL  # N > 2^15


def test_controls_and_states_validation(lib):
    p = W.config1(n_steps=10)
    h = _make(lib, p)
    try:
        a = np.zeros(7)
        assert lib.lb_controls_set(h, a.ctypes.data_as(POINTER(c_double)), 7) == L.LB_EINVAL
        a = np.zeros(20)
        a[3] = np.nan
        assert lib.lb_controls_set(h, a.ctypes.data_as(POINTER(c_double)), 20) == L.LB_EINVAL
        assert b"non-finite" in lib.lb_last_error()
        nf = np.array([1], dtype=np.int32)
        car = np.zeros(1)
        assert lib.lb_controls_define(h, 2, nf.ctypes.data_as(POINTER(c_int32)),
                                      car.ctypes.data_as(POINTER(c_double))) == L.LB_EINVAL
        r = colmajor(p.rho0)
        assert lib.lb_states_set(h, 0, r.ctypes.data_as(c_void_p), None) == L.LB_EINVAL
        assert lib.lb_objective_set(h, 7, r.ctypes.data_as(c_void_p), 0.0) == L.LB_EINVAL
        assert lib.lb_objective_set(h, 0, r.ctypes.data_as(c_void_p), -1.0) == L.LB_EINVAL
        assert lib.lb_solver_set(h, 9, 1e-15, 200, 100) == L.LB_EINVAL
        assert lib.lb_solver_set(h, 0, 0.0, 200, 100) == L.LB_EINVAL
        assert lib.lb_solver_set(h, 0, 1e-15, 0, 100) == L.LB_EINVAL
        assert lib.lb_solver_set(h, 0, 1e-15, 200, -2) == L.LB_EINVAL
        # compute before binding a workspace is refused on the host
        G = c_double()
        assert lib.lb_forward(h, None, byref(G), None) == L.LB_EINVAL
        assert b"workspace" in lib.lb_last_error()
    finally:
        lib.lb_system_destroy(h)


@pytest.mark.parametrize("K", [0, 1, 7, 100])
def test_workspace_size_accounts_for_checkpoints(lib, K):
    p = W.config2(n_steps=250)
    h = _make(lib, p, K=K)
    try:
        V = np.asarray(p.gate.T, dtype=np.complex128)
        Vb = np.ascontiguousarray(V).view(np.float64)
        L.check(lib.lb_objective_set_gate(h, 0, Vb.ctypes.data_as(c_void_p), 0.0))
        n = c_size_t()
        L.check(lib.lb_workspace_bytes(h, byref(n)))
        # the 16 states |i><j| of the essential basis form 6 conjugate pairs:
        # 10 states are integrated (lb_set_pairing)
        M, Vl, NT = 10, 81, 250
        state = 16 * M * Vl
        if K == 0:
            tape = NT * state
        else:
            Kc = min(K, NT)
            tape = -(-NT // Kc) * state + Kc * state
        # per-warp gradient pieces of every state, enough for either lane
        # layout of the cluster sweep (2Q = 4 or 4Q = 8 lanes per element),
        # and their sum over the slots
        per = 0
        for lanes in (4, 8):
            C = -(-Vl * lanes // 128)  # CTAs per state
            nw = -(-(-(-Vl // C)) * lanes // 32)  # warps per CTA
            per = max(per, C * nw)
        gproj = M * per * NT * 2 * 2 * 16 + NT * 2 * 2 * 16
        # q0, tar, qT and the ten-slot ring of the first-iterate predictor
        # with the powers g^m, g^-m of its anchor frame; with checkpoints the
        # recompute's forward predictor has a ring (and powers) of its own
        rings = 12 if K == 0 else 24
        assert n.value >= tape + gproj + (3 + rings) * state
        assert n.value <= tape + gproj + (3 + rings) * state + 64 * 1024
    finally:
        lib.lb_system_destroy(h)


def test_conjugate_pairs_shrink_the_workspace(lib):
    """|i><j| and |j><i| = (|i><j|)^+ are integrated once: the gate workload's
    16 states need the workspace of 10; with pairing off, of 16; a target set
    that is not conjugate-paired like the states splits the pairs."""
    p = W.config2(n_steps=250)
    sizes = {}
    for on in (1, 0):
        h = _make(lib, p, K=0)
        try:
            V = np.ascontiguousarray(np.asarray(p.gate.T, dtype=np.complex128)).view(np.float64)
            L.check(lib.lb_objective_set_gate(h, 0, V.ctypes.data_as(c_void_p), 0.0))
            L.check(lib.lb_set_pairing(h, on))
            n = c_size_t()
            L.check(lib.lb_workspace_bytes(h, byref(n)))
            sizes[on] = n.value
        finally:
            lib.lb_system_destroy(h)
    tape_state = 16 * 81 * 250  # stage tape bytes per state (K = 0)
    # every per-state array (tape, states, targets, predictor ring, gradient
    # slots) holds 10 states instead of 16
    assert 0.6 < sizes[1] / sizes[0] < 0.66
    assert lib.lb_set_pairing(None, 1) == L.LB_EINVAL
    # explicit targets that are all the same Hermitian matrix do not pair like
    # the states |i><j| and |j><i| (tar_j != tar_i^+ unless tar is Hermitian:
    # a non-Hermitian common target splits every pair)
    h = _make(lib, p, K=0)
    try:
        rng = np.random.default_rng(5)
        t = rng.standard_normal((16, 9, 9)) + 1j * rng.standard_normal((16, 9, 9))
        tb = colmajor(t)
        L.check(lib.lb_objective_set(h, 0, tb.ctypes.data_as(c_void_p), 0.0))
        n = c_size_t()
        L.check(lib.lb_workspace_bytes(h, byref(n)))
        assert abs(n.value - sizes[0]) < 0.1 * tape_state
    finally:
        lib.lb_system_destroy(h)


def test_grid_sweep_workspace_and_sweep_choice(lib):
    """N^2 > 4096 selects the grid-wide sweep; its workspace adds the four
    iteration buffers, and one CTA per state cannot be forced."""
    p = W.config4(n_steps=40, levels=(3, 3, 3, 3), n_states=2)
    h = _make(lib, p, K=10)
    try:
        t = colmajor(p.targets)
        L.check(lib.lb_objective_set(h, 0, t.ctypes.data_as(c_void_p), 0.0))
        assert lib.lb_set_sweep(h, L.LB_SWEEP_RESIDENT) == L.LB_EINVAL
        assert lib.lb_set_sweep(h, 7) == L.LB_EINVAL
        L.check(lib.lb_set_sweep(h, L.LB_SWEEP_GRID))
        n = c_size_t()
        L.check(lib.lb_set_symmetry(h, L.LB_SYM_NONE))
        L.check(lib.lb_workspace_bytes(h, byref(n)))
        V, M = 81 * 81, 2
        state = 16 * M * V
        # q0, tar, qT, 4 checkpoints, 10-step segment tape, zA, zB, lam, qf,
        # the ten-slot rings of the adjoint's and the recompute's first-iterate
        # predictors, the powers g^m, g^-m of each ring's frame and the two
        # single-precision difference buffers (8 bytes per element each)
        assert n.value >= (3 + 4 + 10 + 4 + 20 + 4 + 1) * state
        assert n.value <= (3 + 4 + 10 + 4 + 20 + 4 + 1) * state + 2 * 1024 * 1024
        # Hermitian states and targets: the 14 tape slabs hold k <= l only
        L.check(lib.lb_set_symmetry(h, L.LB_SYM_HERMITIAN))
        npk = c_size_t()
        L.check(lib.lb_workspace_bytes(h, byref(npk)))
        Vh = 81 * 82 // 2
        assert n.value - npk.value == 14 * 16 * M * (V - Vh)
    finally:
        lib.lb_system_destroy(h)


def test_gmres_is_accepted_and_never_grid(lib):
    """GMRES is a valid solver; with it a system that AUTO would give grid
    sweeps (N^2 = 1024, two states) keeps the one-CTA-per-state layout."""
    p = W.random_problem(31, levels=(4, 4, 2), n_states=2, n_steps=20)
    sizes = {}
    for method in (L.LB_SOLVER_JACOBI, L.LB_SOLVER_GMRES):
        h = _make(lib, p, K=10)
        try:
            L.check(lib.lb_solver_set(h, method, 1e-15, 200, 10))
            t = colmajor(p.targets)
            L.check(lib.lb_objective_set(h, 0, t.ctypes.data_as(c_void_p), 0.0))
            n = c_size_t()
            L.check(lib.lb_workspace_bytes(h, byref(n)))
            sizes[method] = n.value
        finally:
            lib.lb_system_destroy(h)
    V, M = 1024, 2
    # grid sweeps add the four iteration buffers of M states each
    assert sizes[L.LB_SOLVER_JACOBI] - sizes[L.LB_SOLVER_GMRES] >= 4 * 16 * M * V


def test_cluster_sweep_rules_for_coupled_pairs(lib):
    """A Jaynes-Cummings pair adds a half pair to the cluster sweep's lane
    plan: two subsystems with one pair (three half pairs) may choose it,
    three subsystems with all three pairs (six) may not; the choice is made
    on the host, before any device work."""
    ok = W.random_problem(41, levels=(2, 3), n_states=2, n_steps=10, jc=0.05)
    bad = W.random_problem(42, levels=(2, 2, 2), n_states=2, n_steps=10, jc=0.05)
    for prob, want in ((ok, L.LB_OK), (bad, L.LB_EINVAL)):
        h = _make(lib, prob, K=10)
        try:
            Q = len(prob.system.levels)
            g = np.ascontiguousarray(np.asarray(prob.system.jc_ghz, dtype=np.float64).reshape(Q * Q))
            r = np.ascontiguousarray(np.asarray(prob.system.rot_ghz, dtype=np.float64))
            L.check(lib.lb_system_set_coupling(h, g.ctypes.data_as(POINTER(c_double)),
                                               r.ctypes.data_as(POINTER(c_double))))
            assert lib.lb_set_sweep(h, L.LB_SWEEP_CLUSTER) == want
            if want != L.LB_OK:
                assert b"pairs" in lib.lb_last_error()
            # without the coupling the same three qubits fit the cluster sweep
            zero = np.zeros(Q * Q)
            L.check(lib.lb_system_set_coupling(h, zero.ctypes.data_as(POINTER(c_double)), None))
            assert lib.lb_set_sweep(h, L.LB_SWEEP_CLUSTER) == L.LB_OK
        finally:
            lib.lb_system_destroy(h)
