"""Dense operators of the composite open quantum system (Sec. II, Appendix A).

Test infrastructure only (see ``oracle/__init__.py``).  Units: inputs are
frequencies/2pi in GHz and times in ns (T1, T2 in microseconds); every
frequency is multiplied by 2pi here, so operators are in rad/ns.
"""

from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# single-subsystem operators and their embedding (Sec. II)


def lowering(n: int) -> np.ndarray:
    """Lowering operator a of an n-level subsystem: a|m> = sqrt(m)|m-1>."""
    a = np.zeros((n, n), dtype=np.complex128)
    for m in range(1, n):
        a[m - 1, m] = math.sqrt(m)
    return a


def embed(op: np.ndarray, q: int, levels) -> np.ndarray:
    """I x ... x op x ... x I with ``op`` on subsystem q; subsystem 0 is the
    leftmost Kronecker factor, i.e. the most significant digit of an index."""
    out = np.ones((1, 1), dtype=np.complex128)
    for p, n in enumerate(levels):
        out = np.kron(out, op if p == q else np.eye(n, dtype=np.complex128))
    return out


def a_op(q: int, levels) -> np.ndarray:
    return embed(lowering(levels[q]), q, levels)


# ----------------------------------------------------------------------------
# Hamiltonian and collapse operators (Sec. II, H_sys and the Lindbladian)


def system_hamiltonian(sysm) -> np.ndarray:
    """H_sys = sum_q [(w_q - w_q^rot) a_q^+ a_q - xi_q/2 a_q^+ a_q^+ a_q a_q]
    - sum_{p<q} xi_pq a_p^+ a_p a_q^+ a_q   (Sec. II, cross-Kerr model; the
    Jaynes-Cummings coupling is time dependent in the rotating frame and
    added by ``jc_hamiltonian``)."""
    levels = sysm.levels
    N = int(np.prod(levels))
    H = np.zeros((N, N), dtype=np.complex128)
    a = [a_op(q, levels) for q in range(len(levels))]
    ad = [x.conj().T for x in a]
    for q in range(len(levels)):
        H += TWO_PI * sysm.detuning_ghz[q] * (ad[q] @ a[q])
        H -= TWO_PI * sysm.selfkerr_ghz[q] / 2.0 * (ad[q] @ ad[q] @ a[q] @ a[q])
    for p in range(len(levels)):
        for q in range(p + 1, len(levels)):
            xi = sysm.crosskerr_ghz[p][q]
            if xi != 0.0:
                H -= TWO_PI * xi * (ad[p] @ a[p] @ ad[q] @ a[q])
    return H


def collapse_operators(sysm) -> list:
    """L_1q = a_q / sqrt(T1_q) (decay), L_2q = a_q^+ a_q / sqrt(T2_q)
    (dephasing), Sec. II.  T in microseconds -> ns; an infinite time, or a
    time printed as 0 (the cavity's T2 in the reset example of Sec. III-B),
    drops the operator."""
    levels = sysm.levels
    out = []
    for q in range(len(levels)):
        a = a_op(q, levels)
        t1, t2 = float(sysm.t1_us[q]), float(sysm.t2_us[q])
        if math.isfinite(t1) and t1 > 0.0:
            out.append(a / math.sqrt(1000.0 * t1))
        if math.isfinite(t2) and t2 > 0.0:
            out.append((a.conj().T @ a) / math.sqrt(1000.0 * t2))
    return out


# ----------------------------------------------------------------------------
# B-spline x carrier controls (Sec. II, eq. rotctrl)


def bspline_basis(s: int, t: float, n_splines: int, T: float) -> float:
    """Quadratic B-spline S_s(t), s = 0..n_splines-1 (Sec. II).

    Reading of the paper: wavelets on a uniform grid with knot spacing
    dtau = T/(n_splines - 2); centre of (1-based) spline s is (s - 3/2) dtau,
    i.e. (s - 1/2) dtau for the 0-based s used here.  With B2 the centred
    uniform quadratic B-spline of support 3 dtau, the basis is a partition of
    unity on [0, T]."""
    dtau = T / (n_splines - 2)
    x = abs((t - (s - 0.5) * dtau) / dtau)
    if x < 0.5:
        return 0.75 - x * x
    if x < 1.5:
        return 0.5 * (x - 1.5) ** 2
    return 0.0


def alpha_index(ctrl, q: int, f: int, s: int) -> int:
    """Offset of Re(alpha_q^{s,f}) in the flat layout [q][f][s][re, im]."""
    off = 0
    for p in range(q):
        off += 2 * ctrl.n_splines * len(ctrl.carriers_ghz[p])
    return off + 2 * (f * ctrl.n_splines + s)


def control_horizon(ctrl, sysm) -> float:
    """The interval [0, T_c] the B-splines of eq. rotctrl span: the final
    time T of the problem, or the longer horizon of which the problem
    integrates the first steps (its controls are then that problem's)."""
    hz = getattr(ctrl, "horizon_ns", None)
    return float(hz) if hz else float(sysm.T_ns)


def control_amplitudes(ctrl, t: float, T: float) -> np.ndarray:
    """d_q(t) = sum_s S_s(t) sum_f alpha_q^{s,f} exp(i t Omega_q^f), eq.
    rotctrl, in rad/ns (alpha and Omega given /2pi in GHz)."""
    Q = len(ctrl.carriers_ghz)
    d = np.zeros(Q, dtype=np.complex128)
    for q in range(Q):
        for f, om in enumerate(ctrl.carriers_ghz[q]):
            carrier = np.exp(1j * TWO_PI * om * t)
            for s in range(ctrl.n_splines):
                S = bspline_basis(s, t, ctrl.n_splines, T)
                if S == 0.0:
                    continue
                i = alpha_index(ctrl, q, f, s)
                d[q] += TWO_PI * S * complex(ctrl.alpha[i], ctrl.alpha[i + 1]) * carrier
    return d


def jc_hamiltonian(sysm, t: float) -> np.ndarray:
    """Jaynes-Cummings coupling of H_sys in its general rotating-frame form
    (Sec. II): sum_{p<q} g_pq (e^{i eta t} a_p^+ a_q + e^{-i eta t} a_p a_q^+),
    eta = omega_p^rot - omega_q^rot (rad/ns from GHz)."""
    levels = tuple(sysm.levels)
    N = int(np.prod(levels))
    H = np.zeros((N, N), dtype=np.complex128)
    g = getattr(sysm, "jc_ghz", None)
    if g is None:
        return H
    rot = getattr(sysm, "rot_ghz", None)
    Q = len(levels)
    for p in range(Q):
        for q in range(p + 1, Q):
            if g[p][q] == 0.0:
                continue
            eta = TWO_PI * ((rot[p] - rot[q]) if rot is not None else 0.0)
            ap, aq = a_op(p, levels), a_op(q, levels)
            ph = np.exp(1j * eta * t)
            H += TWO_PI * g[p][q] * (ph * (ap.conj().T @ aq) + np.conj(ph) * (ap @ aq.conj().T))
    return H


def control_hamiltonian(d: np.ndarray, levels) -> np.ndarray:
    """H_c = sum_q d_q a_q + conj(d_q) a_q^+ (Sec. II, rotating frame)."""
    N = int(np.prod(levels))
    H = np.zeros((N, N), dtype=np.complex128)
    for q in range(len(levels)):
        a = a_op(q, levels)
        H += d[q] * a + np.conj(d[q]) * a.conj().T
    return H


# ----------------------------------------------------------------------------
# vectorised Lindbladian (Appendix A, eq. mastereq_vectorized)


def vec(X: np.ndarray) -> np.ndarray:
    """Column stacking: vec(X)[k + N l] = X[k, l] (Appendix A); a stack of
    matrices gives a stack of vectors."""
    if X.ndim == 2:
        return X.reshape(-1, order="F")
    return np.stack([vec(x) for x in X])


def unvec(q: np.ndarray, N: int) -> np.ndarray:
    return q.reshape((N, N), order="F")


def hamiltonian_part(H: np.ndarray) -> np.ndarray:
    """-i (I_N x H - H^T x I_N), the Hamiltonian part of M (Appendix A)."""
    N = H.shape[0]
    I = np.eye(N, dtype=np.complex128)
    return -1j * (np.kron(I, H) - np.kron(H.T, I))


def dissipator_part(Ls: list, N: int) -> np.ndarray:
    """sum_l conj(L) x L - 1/2 (I x L^+L + (L^+L)^T x I) (Appendix A; for the
    real collapse operators of this model conj(L) = L, which is the paper's
    L x L)."""
    I = np.eye(N, dtype=np.complex128)
    D = np.zeros((N * N, N * N), dtype=np.complex128)
    for L in Ls:
        LdL = L.conj().T @ L
        D += np.kron(L.conj(), L) - 0.5 * (np.kron(I, LdL) + np.kron(LdL.T, I))
    return D


def vectorized_lindbladian(H: np.ndarray, Ls: list) -> np.ndarray:
    """M = -i(I x H - H^T x I) + sum (L x L - 1/2(I x L^T L + L^T L x I))."""
    return hamiltonian_part(H) + dissipator_part(Ls, H.shape[0])


def lindblad_matrix_form(H: np.ndarray, Ls: list, X: np.ndarray) -> np.ndarray:
    """-i[H, X] + sum_l (L X L^+ - 1/2 {L^+ L, X}), the master equation of
    Sec. II written on N x N matrices (no vectorisation)."""
    Y = -1j * (H @ X - X @ H)
    for L in Ls:
        LdL = L.conj().T @ L
        Y = Y + L @ X @ L.conj().T - 0.5 * (LdL @ X + X @ LdL)
    return Y


def adjoint_matrix_form(H: np.ndarray, Ls: list, X: np.ndarray) -> np.ndarray:
    """The Hilbert-Schmidt adjoint of the Lindbladian on N x N matrices,
    +i[H, X] + sum_l (L^+ X L - 1/2 {L^+ L, X}); its vectorisation is M^+
    (conjugate transpose of the Appendix A matrix)."""
    Y = 1j * (H @ X - X @ H)
    for L in Ls:
        LdL = L.conj().T @ L
        Y = Y + L.conj().T @ X @ L - 0.5 * (LdL @ X + X @ LdL)
    return Y


class Model:
    """Time-independent pieces of one system, built once (Sec. II)."""

    def __init__(self, sysm, ctrl):
        self.sys = sysm
        self.ctrl = ctrl
        self.levels = tuple(sysm.levels)
        self.N = int(np.prod(self.levels))
        self.H_sys = system_hamiltonian(sysm)
        self.Ls = collapse_operators(sysm)
        self._D = None
        self.h = sysm.T_ns / sysm.n_steps

    @property
    def D(self) -> np.ndarray:
        """Dense dissipator part of M, built on first use (N^2 x N^2)."""
        if self._D is None:
            self._D = dissipator_part(self.Ls, self.N)
        return self._D

    def t_half(self, j: int) -> float:
        """t_j + dt/2, where M^{j+1/2} is evaluated (Appendix A)."""
        return (j + 0.5) * self.h

    def d(self, t: float) -> np.ndarray:
        return control_amplitudes(self.ctrl, t, control_horizon(self.ctrl, self.sys))

    def H(self, t: float) -> np.ndarray:
        return self.H_sys + jc_hamiltonian(self.sys, t) + control_hamiltonian(self.d(t), self.levels)

    def M(self, t: float) -> np.ndarray:
        """Dense N^2 x N^2 vectorised Lindbladian at time t (Appendix A)."""
        return hamiltonian_part(self.H(t)) + self.D
