"""lb_gradient_static: the gradient for callers that cannot allocate device
memory, with all device scratch in the library's static array.

Runs last (file name) so that a failure here stops a -x run only after every
other test has run; it also passes alone in a fresh process."""

import gc
from ctypes import POINTER, byref, c_double, c_int32, c_size_t, c_void_p

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _unbound_handle(lib, L, prob, K):
    """A handle with controls, states, objective and solver set and no workspace."""
    from paper_2110_10310_gb300.system import colmajor

    keep = []

    def arr(x, ct, dt):
        a = np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep.append(a)
        return a.ctypes.data_as(POINTER(ct))

    sysm = prob.system
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
    w = None if prob.weights is None else np.ascontiguousarray(prob.weights, dtype=np.float64)
    L.check(lib.lb_states_set(h, prob.M, r.ctypes.data_as(c_void_p),
                              None if w is None else w.ctypes.data_as(POINTER(c_double))))
    kind = L.LB_J_FROB if prob.objective == "frob" else L.LB_J_TR
    if prob.targets is not None:
        t = colmajor(prob.targets)
        L.check(lib.lb_objective_set(h, kind, t.ctypes.data_as(c_void_p), prob.gamma2))
    else:
        V = np.ascontiguousarray(np.asarray(prob.gate, dtype=np.complex128).T).view(np.float64)
        L.check(lib.lb_objective_set_gate(h, kind, V.ctypes.data_as(c_void_p), prob.gamma2))
    L.check(lib.lb_solver_set(h, 0, 1e-15, 200, K))
    return h


@pytest.mark.parametrize("name", ["cnot", "random", "hermitian"])
def test_static_scratch_gradient_matches_workspace_gradient(name):
    """Two calls in a row through the static-scratch entry point agree with
    lb_gradient on a caller-allocated workspace (states and objectives to
    1e-10, gradients to 1e-9, relative)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10310_gb300 import _lib as L
    from paper_2110_10310_gb300.system import LindbladSystem

    lib = L.load(build_if_missing=True)
    if name == "cnot":
        prob = W.config2(n_steps=400)
    else:
        prob = W.random_problem(301, levels=(3, 2), n_states=3, n_steps=60, T_ns=1.2, amp=0.1,
                                objective="trace", gamma2=0.1, ckpt_every=7, hermitian=name == "hermitian")
    ref = LindbladSystem(prob, ckpt_every=prob.ckpt_every)
    G_ref, g_ref = ref.gradient()
    h = _unbound_handle(lib, L, prob, prob.ckpt_every)
    try:
        stream = c_void_p(torch.cuda.current_stream().cuda_stream)
        for call in range(2):
            G = c_double()
            g = np.zeros(len(g_ref))
            if call == 1:
                # the first call has loaded the module; the second allocates
                # nothing (the collector is held off so that tensors of earlier
                # tests are not freed in between)
                gc.collect()
                gc.disable()
                torch.cuda.synchronize()
                used0 = torch.cuda.memory_allocated()
                free0 = torch.cuda.mem_get_info()[0]
            try:
                L.check(lib.lb_gradient_static(h, stream, byref(G), g.ctypes.data_as(POINTER(c_double))))
                if call == 1:
                    torch.cuda.synchronize()
                    assert torch.cuda.memory_allocated() == used0
                    assert torch.cuda.mem_get_info()[0] == free0
            finally:
                gc.enable()
            assert abs(G.value - G_ref) <= 1e-10 * abs(G_ref)
            assert np.max(np.abs(g - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))
        # the handle is left unbound and still usable
        n = c_size_t()
        L.check(lib.lb_workspace_bytes(h, byref(n)))
        assert n.value <= L.LB_STATIC_SCRATCH_BYTES
    finally:
        lib.lb_system_destroy(h)


def test_static_scratch_rejects_oversized_problem():
    """A problem needing more than the static array is refused on the host."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10310_gb300 import _lib as L

    lib = L.load(build_if_missing=True)
    prob = W.config2()  # with K = 0 the full stage tape is ~207 MB
    h = _unbound_handle(lib, L, prob, 0)
    try:
        G = c_double()
        rc = lib.lb_gradient_static(h, None, byref(G), None)
        assert rc == L.LB_ENOMEM
        assert b"static scratch" in lib.lb_last_error()
    finally:
        lib.lb_system_destroy(h)


def test_static_scratch_refuses_the_cluster_sweep():
    """The entry point runs one CTA per state; an explicit cluster-sweep
    request is refused on the host rather than silently dropped."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10310_gb300 import _lib as L

    lib = L.load(build_if_missing=True)
    prob = W.config2(n_steps=50)
    h = _unbound_handle(lib, L, prob, 10)
    try:
        L.check(lib.lb_set_sweep(h, L.LB_SWEEP_CLUSTER))
        G = c_double()
        rc = lib.lb_gradient_static(h, None, byref(G), None)
        assert rc == L.LB_EINVAL
        assert b"cluster" in lib.lb_last_error().lower()
    finally:
        lib.lb_system_destroy(h)
