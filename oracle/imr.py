"""Implicit midpoint forward sweep, objective and discrete adjoint gradient.

Test infrastructure only (see ``oracle/__init__.py``).  Every step is a dense
LU solve (``numpy.linalg.solve``) with the dense N^2 x N^2 matrix of
``model.Model.M``; states of a problem are the columns of a (N^2, M) matrix.
"""

from __future__ import annotations

import numpy as np

from .model import Model, TWO_PI, a_op, alpha_index, bspline_basis, control_horizon, hamiltonian_part, unvec, vec


# ----------------------------------------------------------------------------
# targets (Sec. III-C for gates)


def embedding(levels, essential) -> np.ndarray:
    """Isometry P from the essential product basis into the full basis: column
    i is the full basis vector whose digits equal the essential digits of i.
    The paper does not discuss essential levels; a gate acts on the essential
    subspace and is zero on guard levels."""
    levels = tuple(levels)
    ess = tuple(essential) if essential is not None else levels
    Ne = int(np.prod(ess))
    N = int(np.prod(levels))
    P = np.zeros((N, Ne))
    for i in range(Ne):
        rem, digits = i, []
        for r in reversed(ess):
            digits.append(rem % r)
            rem //= r
        digits = digits[::-1]
        k = 0
        for dgt, n in zip(digits, levels):
            k = k * n + dgt
        P[k, i] = 1.0
    return P


def targets_of(prob) -> np.ndarray:
    """rho_i^tar: given explicitly, or V rho_i(0) V^+ with V lifted to the
    full space, V_full = P V P^T (Sec. III-C, gate optimisation)."""
    if prob.objective == "nm":
        N = int(np.prod(prob.system.levels))
        return np.stack([observable_nm(N, int(prob.meta["m"]))] * prob.M)
    if prob.targets is not None:
        return np.asarray(prob.targets, dtype=np.complex128)
    P = embedding(prob.system.levels, prob.system.essential)
    V = P @ prob.gate @ P.T
    return np.stack([V @ r @ V.conj().T for r in prob.rho0])


def weights_of(prob) -> np.ndarray:
    return np.ones(prob.M) if prob.weights is None else np.asarray(prob.weights, dtype=np.float64)


# ----------------------------------------------------------------------------
# forward sweep (Appendix A, eqs. IMR and linsystem_primal)


def imr_step(model: Model, j: int, Qm: np.ndarray):
    """One implicit midpoint step: (I - dt/2 M^{j+1/2}) z = q^j, then
    q^{j+1} = q^j + dt M^{j+1/2} z.  Returns (q^{j+1}, z)."""
    h = model.h
    M = model.M(model.t_half(j))
    A = np.eye(M.shape[0], dtype=np.complex128) - 0.5 * h * M
    Z = np.linalg.solve(A, Qm)
    return Qm + h * (M @ Z), Z


def forward(prob, n_steps: int | None = None, keep: bool = True):
    """Integrate all initial states of ``prob`` over ``n_steps`` steps (default:
    the whole horizon).  Returns dict with the final states (M, N, N) and,
    when ``keep``, every q^j and z^j as (N^2, M) matrices."""
    model = Model(prob.system, prob.controls)
    NT = prob.system.n_steps if n_steps is None else n_steps
    Qm = vec(np.asarray(prob.rho0, dtype=np.complex128)).T.copy()
    qs, zs = ([Qm], []) if keep else (None, None)
    for j in range(NT):
        Qm, Z = imr_step(model, j, Qm)
        if keep:
            qs.append(Qm)
            zs.append(Z)
    rhoT = np.stack([unvec(Qm[:, i], model.N) for i in range(Qm.shape[1])])
    return {"model": model, "rhoT": rhoT, "q": qs, "z": zs}


# ----------------------------------------------------------------------------
# objective (Sec. III, eq. optimproblem and the merit functionals)


def observable_nm(N: int, m: int) -> np.ndarray:
    """N_m = diag(|l - m|), l = 0..N-1 over the full basis index (Sec. III-B,
    eq. Jmeasure): J_Nm(rho) = Tr(N_m rho) vanishes only at |m><m|."""
    return np.diag(np.abs(np.arange(N) - m).astype(np.float64)).astype(np.complex128)


def merit(kind: str, tar: np.ndarray, rho: np.ndarray) -> float:
    """J_Frob = 1/2 ||rho_tar - rho||_F^2, J_Tr = 1 - Re Tr(rho_tar^+ rho)
    (Sec. III, eq. Jmeasure), and J_Nm = Re Tr(N_m rho) with ``tar`` = N_m."""
    if kind == "frob":
        return 0.5 * float(np.sum(np.abs(tar - rho) ** 2))
    if kind == "trace":
        return 1.0 - float(np.real(np.trace(tar.conj().T @ rho)))
    if kind == "nm":
        return float(np.real(np.trace(tar @ rho)))
    raise ValueError(kind)


def objective(prob, rhoT: np.ndarray) -> float:
    """G = 1/M sum_i beta_i J(rho_i^tar, rho_i(T)) + gamma2/2 ||alpha||^2
    (gamma1 = 0)."""
    tars = targets_of(prob)
    w = weights_of(prob)
    G = sum(w[i] * merit(prob.objective, tars[i], rhoT[i]) for i in range(prob.M)) / prob.M
    return G + 0.5 * prob.gamma2 * float(np.dot(prob.controls.alpha, prob.controls.alpha))


def terminal_adjoint(prob, rhoT: np.ndarray) -> np.ndarray:
    """q^_i(N_T) = beta_i/M * g_i (Appendix B), with g the gradient of J with
    respect to conj(q) under <a, b> = Re(a^H b): g = q - q_tar for J_Frob and
    g = -q_tar for J_Tr and g = vec(N_m) for J_Nm."""
    tars = targets_of(prob)
    w = weights_of(prob)
    cols = []
    for i in range(prob.M):
        if prob.objective == "frob":
            g = vec(rhoT[i]) - vec(tars[i])
        elif prob.objective == "nm":
            g = vec(tars[i])
        else:
            g = -vec(tars[i])
        cols.append(w[i] / prob.M * g)
    return np.stack(cols, axis=1)


def penalty_weights(prob, NT: int | None = None) -> np.ndarray:
    """dt beta(t_j), j = 0..N_T-1, beta(t) = exp(-((t - T)/a)^2)/a: the
    running penalty gamma1 int_0^T beta(t) J(rho_tar, rho(t)) dt of eq.
    optimproblem by the left rectangle rule on the time grid."""
    NT = prob.system.n_steps if NT is None else NT
    h = prob.system.T_ns / prob.system.n_steps
    t = np.arange(NT) * h
    a = float(prob.penalty_a)
    return h * np.exp(-(((t - prob.system.T_ns) / a) ** 2)) / a


def penalty(prob, qs) -> float:
    """gamma1/M sum_i beta_i sum_j dt beta(t_j) J(rho_i^tar, q_i^j) (the
    running penalty per state, weighted like the final-time term)."""
    g1 = float(getattr(prob, "gamma1", 0.0))
    if g1 == 0.0:
        return 0.0
    tars = targets_of(prob)
    w = weights_of(prob)
    pw = penalty_weights(prob, len(qs) - 1)
    N = tars.shape[1]
    tot = 0.0
    for i in range(prob.M):
        for j in range(len(qs) - 1):
            tot += w[i] * pw[j] * merit(prob.objective, tars[i], unvec(qs[j][:, i], N))
    return g1 * tot / prob.M


def merit_gradient(prob, tar: np.ndarray, q: np.ndarray) -> np.ndarray:
    """2 dJ/dconj(q) of the merit functional at q (vectors): q - q_tar,
    -q_tar or vec(N_m)."""
    if prob.objective == "frob":
        return q - tar
    if prob.objective == "nm":
        return tar
    return -tar


def value(prob) -> float:
    if float(getattr(prob, "gamma1", 0.0)) != 0.0:
        fw = forward(prob, keep=True)
        return objective(prob, fw["rhoT"]) + penalty(prob, fw["q"])
    return objective(prob, forward(prob, keep=False)["rhoT"])


# ----------------------------------------------------------------------------
# discrete adjoint and reduced gradient (Appendix B)


def dd_dalpha(ctrl, T: float, t: float):
    """Nonzero derivatives of d_q(t) (eq. rotctrl) with respect to the real
    control parameters: list of (flat index, q, dd/dalpha in rad/ns)."""
    out = []
    for q, carriers in enumerate(ctrl.carriers_ghz):
        for f, om in enumerate(carriers):
            carrier = np.exp(1j * TWO_PI * om * t)
            for s in range(ctrl.n_splines):
                S = bspline_basis(s, t, ctrl.n_splines, T)
                if S == 0.0:
                    continue
                i = alpha_index(ctrl, q, f, s)
                out.append((i, q, TWO_PI * S * carrier))  # d/dRe alpha
                out.append((i + 1, q, 1j * TWO_PI * S * carrier))  # d/dIm alpha
    return out


def gradient(prob, n_steps: int | None = None):
    """Objective G and its exact discrete gradient (Appendix B), with the
    running penalty's source gamma1 beta_i/M dt beta(t_j) g(q^j) added to
    qhat^j when gamma1 != 0.

    Backward sweep for j = N_T-1..0:
      (I - dt/2 (M^{j+1/2})^+) zhat^j = qhat^{j+1}     (eq. linsystem_adjoint)
      grad += dt Re((dM/dalpha z^j)^+ zhat^j)         (eq. reducedgradient)
      qhat^j = qhat^{j+1} + dt (M^{j+1/2})^+ zhat^j
    then grad += gamma2 alpha.  Because M is linear in H and H_c is linear in
    d_q, dM/dalpha_k = dd_q/dalpha_k (-i)(I x a_q - a_q^T x I)
    + conj(dd_q/dalpha_k) (-i)(I x a_q^+ - conj(a_q) x I).
    Returns (G, grad, forward result)."""
    fw = forward(prob, n_steps=n_steps, keep=True)
    model = fw["model"]
    h = model.h
    NT = len(fw["z"])
    G = objective(prob, fw["rhoT"]) + penalty(prob, fw["q"])
    Lam = terminal_adjoint(prob, fw["rhoT"])
    g1 = float(getattr(prob, "gamma1", 0.0))
    if g1 != 0.0:
        tars = np.stack([vec(t) for t in targets_of(prob)], axis=1)
        wts = weights_of(prob)
        pw = penalty_weights(prob, NT)
    levels = model.levels
    Ma = [hamiltonian_part(a_op(q, levels)) for q in range(len(levels))]
    Mad = [hamiltonian_part(a_op(q, levels).conj().T) for q in range(len(levels))]
    grad = np.zeros_like(prob.controls.alpha, dtype=np.float64)
    I = np.eye(model.N * model.N, dtype=np.complex128)
    for j in range(NT - 1, -1, -1):
        t = model.t_half(j)
        MH = model.M(t).conj().T
        Zh = np.linalg.solve(I - 0.5 * h * MH, Lam)
        Z = fw["z"][j]
        Ca = [np.sum(Zh.conj() * (Ma[q] @ Z)) for q in range(len(levels))]
        Cad = [np.sum(Zh.conj() * (Mad[q] @ Z)) for q in range(len(levels))]
        for k, q, dd in dd_dalpha(prob.controls, control_horizon(prob.controls, prob.system), t):
            grad[k] += h * np.real(dd * Ca[q] + np.conj(dd) * Cad[q])
        Lam = Lam + h * (MH @ Zh)
        if g1 != 0.0:
            # source of the running penalty at q^j (Appendix B)
            for i in range(prob.M):
                Lam[:, i] += g1 * wts[i] / prob.M * pw[j] * merit_gradient(prob, tars[:, i], fw["q"][j][:, i])
    grad += prob.gamma2 * prob.controls.alpha
    return G, grad, fw


def fd_gradient(prob, eps: float = 1e-6, indices=None, n_steps: int | None = None):
    """Central differences (G(alpha + eps e_k) - G(alpha - eps e_k)) / 2eps."""
    import copy

    idx = range(len(prob.controls.alpha)) if indices is None else indices
    out = {}
    for k in idx:
        vals = []
        for sgn in (+1, -1):
            p = copy.deepcopy(prob)
            p.controls.alpha = prob.controls.alpha.copy()
            p.controls.alpha[k] += sgn * eps
            if float(getattr(p, "gamma1", 0.0)) != 0.0:
                fw = forward(p, n_steps=n_steps, keep=True)
                vals.append(objective(p, fw["rhoT"]) + penalty(p, fw["q"]))
            else:
                vals.append(objective(p, forward(p, n_steps=n_steps, keep=False)["rhoT"]))
        out[k] = (vals[0] - vals[1]) / (2 * eps)
    return out


def adjoint_states(prob, n_steps: int | None = None):
    """All adjoint states qhat^j (j = N_T..0) of the backward sweep, as (N^2, M)
    matrices, for parity of the adjoint path (Appendix B)."""
    fw = forward(prob, n_steps=n_steps, keep=True)
    model = fw["model"]
    h = model.h
    NT = len(fw["z"])
    Lam = terminal_adjoint(prob, fw["rhoT"])
    out = [Lam]
    I = np.eye(model.N * model.N, dtype=np.complex128)
    for j in range(NT - 1, -1, -1):
        MH = model.M(model.t_half(j)).conj().T
        Zh = np.linalg.solve(I - 0.5 * h * MH, Lam)
        Lam = Lam + h * (MH @ Zh)
        out.append(Lam)
    return out
