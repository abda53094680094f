"""Python front end of the C ABI: marshal a problem into a ``lb_system``,
give it a PyTorch-allocated device workspace, and call the library.

PyTorch provides device memory and streams only; every step of the method
runs in the CUDA library.  Density matrices cross the boundary as M x N x N
complex FP64 arrays, column-major per matrix (vec(rho) of Appendix A).
"""

from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int32, c_size_t, c_void_p

import numpy as np
import torch

from . import _lib as L


def colmajor(rho) -> np.ndarray:
    """(M, N, N) complex -> contiguous float64 array in the ABI layout."""
    r = np.asarray(rho, dtype=np.complex128)
    if r.ndim == 2:
        r = r[None]
    return np.ascontiguousarray(np.transpose(r, (0, 2, 1))).view(np.float64)


def from_colmajor(t: torch.Tensor, M: int, N: int) -> torch.Tensor:
    """Device buffer of M column-major N x N matrices -> (M, N, N) complex tensor [i, k, l]."""
    return t.view(torch.complex128).reshape(M, N, N).transpose(1, 2)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _stats_dict(s) -> dict:
    return {"state_steps": s.state_steps, "inner_iterations": s.inner_iterations,
            "max_iterations": s.max_iterations, "kernel_launches": s.kernel_launches,
            "phase_steps": list(s.phase_steps), "phase_iterations": list(s.phase_iterations),
            "ms_forward": s.ms_forward, "ms_backward": s.ms_backward,
            "sweep": {1: "resident", 2: "grid", 3: "cluster"}.get(s.sweep, s.sweep),
            "solver": {1: "jacobi", 2: "neumann", 3: "gmres"}.get(s.solver, s.solver),
            "symmetry": "hermitian" if s.symmetry == L.LB_SYM_HERMITIAN else "none",
            "ckpt_every": s.ckpt_every, "states_integrated": s.states_integrated,
            "phase_diff_iterations": list(s.phase_diff_iterations)}


def _stream_handle(stream) -> c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


class LindbladSystem:
    """One composite system with its controls, initial states and objective.

    ``problem`` is any object with the attributes of ``workloads.Problem``
    (system, controls, rho0, objective, targets or gate, weights, gamma2,
    ckpt_every)."""

    def __init__(self, problem, *, solver: int = L.LB_SOLVER_AUTO, rtol: float = 1e-15, max_iter: int = 200,
                 ckpt_every: int | None = None, sweep: int = L.LB_SWEEP_AUTO, symmetry: int = L.LB_SYM_AUTO,
                 predictor: int = L.LB_PRED_AUTO, pred_order: int = 0, pairing: int = 1,
                 difference_iterations: int = 1, precision: int = L.LB_PREC_F64, device=None, stream=None):
        self.lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        sysm = problem.system
        Q = len(sysm.levels)
        self.Q = Q
        self.N = int(np.prod(sysm.levels))
        self.M = int(np.asarray(problem.rho0).shape[0])
        self.n_steps = int(sysm.n_steps)
        self._keep = []  # ctypes buffers referenced by the descriptor

        def arr(x, ct, dt):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self._keep.append(a)
            return a.ctypes.data_as(POINTER(ct))

        desc = L.lb_system_desc()
        desc.Q = Q
        desc.levels = arr(sysm.levels, c_int32, np.int32)
        desc.essential = arr(sysm.essential, c_int32, np.int32) if sysm.essential is not None else None
        desc.detuning_ghz = arr(sysm.detuning_ghz, c_double, np.float64)
        desc.selfkerr_ghz = arr(sysm.selfkerr_ghz, c_double, np.float64)
        desc.crosskerr_ghz = arr(np.asarray(sysm.crosskerr_ghz, dtype=np.float64).reshape(Q * Q), c_double, np.float64)
        desc.t1_us = arr(sysm.t1_us, c_double, np.float64)
        desc.t2_us = arr(sysm.t2_us, c_double, np.float64)
        desc.T_ns = float(sysm.T_ns)
        desc.n_steps = int(sysm.n_steps)
        h = c_void_p()
        L.check(self.lib.lb_system_create(byref(desc), byref(h)))
        self.h = h
        jc = getattr(sysm, "jc_ghz", None)
        if jc is not None and np.any(np.asarray(jc) != 0.0):
            rot = getattr(sysm, "rot_ghz", None)
            L.check(self.lib.lb_system_set_coupling(
                h, arr(np.asarray(jc, dtype=np.float64).reshape(Q * Q), c_double, np.float64),
                None if rot is None else arr(rot, c_double, np.float64)))
        ctrl = problem.controls
        nf = np.array([len(c) for c in ctrl.carriers_ghz], dtype=np.int32)
        car = np.concatenate([np.asarray(c, dtype=np.float64) for c in ctrl.carriers_ghz])
        L.check(self.lib.lb_controls_define(h, int(ctrl.n_splines), nf.ctypes.data_as(POINTER(c_int32)), _dptr(car)))
        if getattr(ctrl, "horizon_ns", None):
            L.check(self.lib.lb_controls_set_horizon(h, float(ctrl.horizon_ns)))
        self.n_params = 2 * int(ctrl.n_splines) * int(nf.sum())
        self.set_alpha(ctrl.alpha)
        rho = colmajor(problem.rho0)
        w = None if problem.weights is None else np.ascontiguousarray(problem.weights, dtype=np.float64)
        L.check(self.lib.lb_states_set(h, self.M, rho.ctypes.data_as(c_void_p), None if w is None else _dptr(w)))
        kind = L.LB_J_FROB if problem.objective == "frob" else L.LB_J_TR
        g2 = float(getattr(problem, "gamma2", 0.0))
        if problem.objective == "nm":
            L.check(self.lib.lb_objective_set_measure(h, int(problem.meta["m"]), g2))
        elif problem.targets is not None:
            tar = colmajor(problem.targets)
            L.check(self.lib.lb_objective_set(h, kind, tar.ctypes.data_as(c_void_p), g2))
        else:
            V = np.ascontiguousarray(np.asarray(problem.gate, dtype=np.complex128).T).view(np.float64)
            L.check(self.lib.lb_objective_set_gate(h, kind, V.ctypes.data_as(c_void_p), g2))
        g1 = float(getattr(problem, "gamma1", 0.0))
        if g1 != 0.0:
            L.check(self.lib.lb_objective_set_penalty(h, g1, float(problem.penalty_a)))
        K = int(getattr(problem, "ckpt_every", 100)) if ckpt_every is None else int(ckpt_every)
        L.check(self.lib.lb_solver_set(h, int(solver), float(rtol), int(max_iter), K))
        L.check(self.lib.lb_set_sweep(h, int(sweep)))
        L.check(self.lib.lb_set_symmetry(h, int(symmetry)))
        L.check(self.lib.lb_set_predictor(h, int(predictor), int(pred_order)))
        L.check(self.lib.lb_set_pairing(h, int(pairing)))
        L.check(self.lib.lb_set_difference_iterations(h, int(difference_iterations)))
        L.check(self.lib.lb_set_precision(h, int(precision)))
        nbytes = c_size_t()
        L.check(self.lib.lb_workspace_bytes(h, byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        L.check(self.lib.lb_bind_workspace(h, c_void_p(self.workspace.data_ptr()), nbytes, _stream_handle(stream)))

    # -- inputs --------------------------------------------------------------
    def set_alpha(self, alpha):
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
        if a.size != self.n_params:
            raise ValueError(f"alpha has {a.size} entries, expected {self.n_params}")
        L.check(self.lib.lb_controls_set(self.h, _dptr(a), a.size))

    def set_states_host(self, rho_host, weights=None):
        """rho_host: numpy (M, N, N) complex, or a (pinned) torch float64 CPU
        tensor already in the ABI layout."""
        if isinstance(rho_host, torch.Tensor):
            ptr = c_void_p(rho_host.data_ptr())
            keep = rho_host
        else:
            keep = colmajor(rho_host)
            ptr = keep.ctypes.data_as(c_void_p)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        L.check(self.lib.lb_states_set(self.h, self.M, ptr, None if w is None else _dptr(w)))
        return keep

    # -- the method ------------------------------------------------------------
    def forward(self, want_states: bool = False, stream=None):
        G = c_double()
        out = None
        if want_states:
            out = torch.empty(2 * self.M * self.N * self.N, dtype=torch.float64, device=self.device)
        L.check(self.lib.lb_forward(self.h, _stream_handle(stream), byref(G),
                                    c_void_p(out.data_ptr()) if out is not None else None))
        if want_states:
            return G.value, from_colmajor(out, self.M, self.N)
        return G.value

    def gradient(self, stream=None):
        G = c_double()
        g = np.zeros(self.n_params, dtype=np.float64)
        L.check(self.lib.lb_gradient(self.h, _stream_handle(stream), byref(G), _dptr(g)))
        return G.value, g

    def optimize(self, max_iter: int = 50, memory: int = 10, gtol: float = 1e-8, step0: float = 1e-2, stream=None):
        """L-BFGS on G(alpha) from the current controls (``lb_optimize``); the
        final alpha stays set.  Returns a dict with G, alpha, iterations,
        gradient evaluations and the (G, max|grad|) history."""
        G = c_double()
        a = np.zeros(self.n_params, dtype=np.float64)
        it = c_int32()
        ev = c_int32()
        hist = np.zeros((int(max_iter) + 1, 2), dtype=np.float64)
        L.check(self.lib.lb_optimize(self.h, _stream_handle(stream), int(max_iter), int(memory), float(gtol),
                                     float(step0), byref(G), _dptr(a), byref(it), byref(ev), _dptr(hist)))
        return {"G": G.value, "alpha": a, "iterations": it.value, "evaluations": ev.value,
                "history": hist[: it.value + 1].copy()}

    def gradient_async(self, G_dev: torch.Tensor, grad_dev: torch.Tensor, stream=None):
        L.check(self.lib.lb_gradient_async(self.h, _stream_handle(stream), c_void_p(G_dev.data_ptr()),
                                           c_void_p(grad_dev.data_ptr())))

    def propagate(self, x: torch.Tensor, j0: int, j1: int, adjoint: bool = False, stream=None):
        """x: (n, N, N) complex128 CUDA tensor [i, k, l]; returns the propagated copy."""
        n = x.shape[0]
        buf = x.transpose(1, 2).contiguous().view(torch.float64).reshape(-1).clone()
        L.check(self.lib.lb_propagate(self.h, _stream_handle(stream), int(adjoint), int(j0), int(j1),
                                      c_void_p(buf.data_ptr()), n))
        return from_colmajor(buf, n, self.N)

    def apply(self, x: torch.Tensor, step: int, adjoint: bool = False, stream=None):
        """y = M^{step+1/2} x (or its adjoint) for x: (n, N, N) complex128 CUDA tensor."""
        n = x.shape[0]
        xb = x.transpose(1, 2).contiguous().view(torch.float64).reshape(-1)
        yb = torch.empty_like(xb)
        L.check(self.lib.lb_apply(self.h, _stream_handle(stream), int(adjoint), int(step),
                                  c_void_p(xb.data_ptr()), c_void_p(yb.data_ptr()), n))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return from_colmajor(yb, n, self.N)

    def stats(self) -> dict:
        s = L.lb_stats()
        L.check(self.lib.lb_get_stats(self.h, byref(s)))
        return _stats_dict(s)

    def autotune(self, probe_steps: int = 20, stream=None) -> dict:
        """Time the candidate sweep kinds and inner solvers on a short probe and
        keep the fastest (lb_autotune)."""
        out = (c_int32 * 3)()
        L.check(self.lib.lb_autotune(self.h, _stream_handle(stream), int(probe_steps), out))
        names = {L.LB_SWEEP_RESIDENT: "resident", L.LB_SWEEP_GRID: "grid", L.LB_SWEEP_CLUSTER: "cluster"}
        solvers = {L.LB_SOLVER_JACOBI: "jacobi", L.LB_SOLVER_NEUMANN: "neumann", L.LB_SOLVER_GMRES: "gmres"}
        r, o = c_int32(), c_int32()
        L.check(self.lib.lb_get_predictor(self.h, byref(r), byref(o)))
        return {"sweep": names.get(out[0], out[0]), "solver": solvers.get(out[1], out[1]), "shape": out[2],
                "pred_order": o.value}

    def set_timing(self, on: bool = True):
        L.check(self.lib.lb_set_timing(self.h, int(on)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lb_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LindbladBatch:
    """Independent systems advanced together, one persistent launch per sweep.

    Every member must use one CTA per state (create it with
    ``sweep=LB_SWEEP_RESIDENT``; N^2 <= 4096)."""

    def __init__(self, systems, stream=None):
        self.lib = L.load()
        self.systems = list(systems)
        arr = (c_void_p * len(self.systems))(*[s.h.value for s in self.systems])
        b = c_void_p()
        L.check(self.lib.lb_batch_create(arr, len(self.systems), byref(b)))
        self.h = b
        nbytes = c_size_t()
        L.check(self.lib.lb_batch_workspace_bytes(b, byref(nbytes)))
        dev = self.systems[0].device
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
        L.check(self.lib.lb_batch_bind_workspace(b, c_void_p(self.workspace.data_ptr()), nbytes,
                                                 _stream_handle(stream)))
        self.n_grad = sum(s.n_params for s in self.systems)

    def forward(self, stream=None):
        G = np.zeros(len(self.systems))
        L.check(self.lib.lb_batch_forward(self.h, _stream_handle(stream), _dptr(G)))
        return G

    def gradient(self, stream=None):
        G = np.zeros(len(self.systems))
        g = np.zeros(self.n_grad)
        L.check(self.lib.lb_batch_gradient(self.h, _stream_handle(stream), _dptr(G), _dptr(g)))
        return G, g

    def capture(self, mode: int, stream=None):
        L.check(self.lib.lb_batch_capture_graph(self.h, _stream_handle(stream), int(mode)))

    def stats(self) -> dict:
        s = L.lb_stats()
        L.check(self.lib.lb_batch_get_stats(self.h, byref(s)))
        return _stats_dict(s)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LindbladObjective(torch.autograd.Function):
    """alpha -> G through the library; backward returns dG/dalpha from the
    discrete adjoint sweep (Appendix B), scaled by the incoming gradient."""

    @staticmethod
    def forward(ctx, alpha: torch.Tensor, system: LindbladSystem):
        system.set_alpha(alpha.detach().to("cpu", torch.float64).numpy())
        if alpha.requires_grad:
            G, g = system.gradient()
            ctx.save_for_backward(torch.from_numpy(g).to(alpha.device, alpha.dtype))
        else:
            G = system.forward()
        return alpha.new_tensor(G)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout * g, None


def objective(alpha: torch.Tensor, system: LindbladSystem) -> torch.Tensor:
    return LindbladObjective.apply(alpha, system)
