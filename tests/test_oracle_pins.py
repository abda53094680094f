"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
solutions of the master equation and of the discrete implicit midpoint rule,
structural invariants of a Lindblad generator, the identities the paper
states, brute force, and central differences.  A dropped term, a wrong sign,
a wrong index ordering or a transposed operand in the oracle fails at least
one of them.
"""

import copy
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import imr, model

TWO_PI = 2 * math.pi
INF = float("inf")


def _undriven(levels, detuning, selfkerr, t1, t2, T=50.0, n_steps=500, crosskerr=None):
    Q = len(levels)
    ck = np.zeros((Q, Q)) if crosskerr is None else np.asarray(crosskerr, dtype=float)
    sysm = W.SystemSpec(
        levels=tuple(levels),
        detuning_ghz=np.asarray(detuning, float),
        selfkerr_ghz=np.asarray(selfkerr, float),
        crosskerr_ghz=ck,
        t1_us=np.asarray(t1, float),
        t2_us=np.asarray(t2, float),
        T_ns=T,
        n_steps=n_steps,
    )
    ctrl = W.ControlSpec(4, [np.array([0.0]) for _ in range(Q)], np.zeros(2 * 4 * Q))
    return sysm, ctrl


def _problem(sysm, ctrl, rho0):
    return W.Problem("pin", sysm, ctrl, np.asarray(rho0, dtype=np.complex128)[None], "frob",
                     targets=np.asarray(rho0, dtype=np.complex128)[None])


def _cayley(lam, h, n):
    """Amplification of the implicit midpoint rule for y' = lam y after n steps."""
    return ((1 + h * lam / 2) / (1 - h * lam / 2)) ** n


# ----------------------------------------------------------------------------
# closed forms of an undriven qubit / qudit


def test_qubit_t1_decay_and_t2_dephasing_closed_form():
    """Undriven qubit: rho11 decays at 1/T1 and rho01 at 1/(2T1) + 1/(2T2) while
    rotating at the detuning.  The discrete IMR values are the Cayley factors of
    those scalar rates; the continuous ones are exp(-t/T1) (Sec. II collapse
    operators)."""
    delta, T1, T2 = 0.013, 0.7, 0.45  # GHz, us, us  (strong so the decay is visible)
    sysm, ctrl = _undriven((2,), [delta], [0.0], [T1], [T2], T=200.0, n_steps=2000)
    h = sysm.T_ns / sysm.n_steps
    plus = 0.5 * np.ones((2, 2), dtype=np.complex128)
    one = np.diag([0.0, 1.0]).astype(np.complex128)
    rT_one = imr.forward(_problem(sysm, ctrl, one), keep=False)["rhoT"][0]
    rT_plus = imr.forward(_problem(sysm, ctrl, plus), keep=False)["rhoT"][0]
    g1 = 1.0 / (1000 * T1)
    g2 = 1.0 / (1000 * T2)
    n = sysm.n_steps
    assert abs(rT_one[1, 1] - _cayley(-g1, h, n)) < 1e-13
    assert abs(rT_one[0, 0] - (1 - _cayley(-g1, h, n))) < 1e-13
    # coherence <0|rho|1>: d/dt rho01 = (-i(E0 - E1) - g1/2 - g2/2) rho01, E1 = 2 pi delta
    lam01 = 1j * TWO_PI * delta - 0.5 * g1 - 0.5 * g2
    assert abs(rT_plus[0, 1] - 0.5 * _cayley(lam01, h, n)) < 1e-13
    assert abs(rT_plus[1, 0] - 0.5 * np.conj(_cayley(lam01, h, n))) < 1e-13
    # against the exact continuous solution, within the IMR truncation error
    t = sysm.T_ns
    err_bound = t * g1 ** 3 * h ** 2 / 12 * 1.01 + 1e-15
    assert abs(rT_one[1, 1] - math.exp(-t * g1)) < err_bound
    assert abs(rT_one[1, 1] - math.exp(-t * g1)) > 0  # the bound is not vacuous


def test_qudit_top_level_decay_and_kerr_phase():
    """4-level qudit: |3><3| decays at 3/T1; the coherence <0|rho|m> evolves at
    -i(E_0 - E_m) - m^2/(2T2) - m/(2T1) with E_m = delta m - xi/2 m(m-1)."""
    delta, xi, T1, T2 = 0.05, 0.2, 0.9, 0.6
    sysm, ctrl = _undriven((4,), [delta], [xi], [T1], [T2], T=20.0, n_steps=400)
    h = sysm.T_ns / sysm.n_steps
    n = sysm.n_steps
    g1, g2 = 1 / (1000 * T1), 1 / (1000 * T2)
    top = np.zeros((4, 4), dtype=np.complex128)
    top[3, 3] = 1.0
    rT = imr.forward(_problem(sysm, ctrl, top), keep=False)["rhoT"][0]
    assert abs(rT[3, 3] - _cayley(-3 * g1, h, n)) < 1e-13
    assert abs(np.trace(rT) - 1) < 1e-13
    for m in (1, 2, 3):
        X = np.zeros((4, 4), dtype=np.complex128)
        X[0, m] = 1.0
        rT = imr.forward(_problem(sysm, ctrl, X), keep=False)["rhoT"][0]
        Em = TWO_PI * (delta * m - xi / 2 * m * (m - 1))
        lam = -1j * (0.0 - Em) - m * m * g2 / 2 - m * g1 / 2
        assert abs(rT[0, m] - _cayley(lam, h, n)) < 1e-12
        others = rT.copy()
        others[0, m] = 0
        assert np.max(np.abs(others)) < 1e-14


def test_cross_kerr_and_subsystem_order():
    """Two qubits with different detunings and a cross-Kerr term: |10> (index 2)
    rotates with subsystem 0's detuning, |01> (index 1) with subsystem 1's,
    and |11> picks up -xi_01 (Sec. II H_sys, subsystem 0 most significant)."""
    d0, d1, xi, T1, T2 = 0.031, -0.017, 0.011, [0.8, 0.5], [0.7, 0.3]
    sysm, ctrl = _undriven((2, 2), [d0, d1], [0.0, 0.0], T1, T2, T=30.0, n_steps=300,
                           crosskerr=[[0, xi], [0, 0]])
    h = sysm.T_ns / sysm.n_steps
    n = sysm.n_steps
    g1 = [1 / (1000 * t) for t in T1]
    g2 = [1 / (1000 * t) for t in T2]
    E = {0: 0.0, 1: TWO_PI * d1, 2: TWO_PI * d0, 3: TWO_PI * (d0 + d1 - xi)}
    digits = {0: (0, 0), 1: (0, 1), 2: (1, 0), 3: (1, 1)}
    for k in (1, 2, 3):
        X = np.zeros((4, 4), dtype=np.complex128)
        X[k, 0] = 1.0
        rT = imr.forward(_problem(sysm, ctrl, X), keep=False)["rhoT"][0]
        gam = sum(digits[k][q] ** 2 * g2[q] / 2 + digits[k][q] * g1[q] / 2 for q in range(2))
        lam = -1j * (E[k] - E[0]) - gam
        assert abs(rT[k, 0] - _cayley(lam, h, n)) < 1e-12, k


# ----------------------------------------------------------------------------
# the implicit midpoint rule for a constant generator (Appendix A)


def test_cayley_transform_for_constant_generator():
    """With Omega = 0 and every spline coefficient equal, d_q(t) is constant, so
    M is constant and n IMR steps equal [(I - h/2 M)^-1 (I + h/2 M)]^n, which we
    evaluate through the eigendecomposition of M."""
    p = W.random_problem(11, levels=(2, 3), n_states=2, n_steps=25, T_ns=3.0, n_carriers=1)
    c = np.array([0.21, -0.13])
    p.controls.alpha = np.tile(c, len(p.controls.alpha) // 2)
    m = model.Model(p.system, p.controls)
    ts = np.linspace(0.0, p.system.T_ns, 7)
    d_all = np.array([m.d(t) for t in ts])
    assert np.allclose(d_all, TWO_PI * complex(*c), atol=1e-13, rtol=0)
    M = m.M(0.37)
    lam, V = sla.eig(M)
    h = m.h
    mu = (1 + h * lam / 2) / (1 - h * lam / 2)
    q0 = model.vec(p.rho0).T
    expect = V @ np.diag(mu ** p.system.n_steps) @ np.linalg.solve(V, q0)
    got = model.vec(imr.forward(p, keep=False)["rhoT"]).T
    assert np.max(np.abs(got - expect)) < 1e-11


def test_stage_identity():
    """q^{j+1} = q^j + dt M z^j with (I - dt/2 M) z^j = q^j gives z^j = (q^j + q^{j+1})/2."""
    p = W.random_problem(12, levels=(3, 2), n_states=2, n_steps=10)
    fw = imr.forward(p)
    for j in range(10):
        assert np.max(np.abs(fw["z"][j] - 0.5 * (fw["q"][j] + fw["q"][j + 1]))) < 1e-14


# ----------------------------------------------------------------------------
# B-spline controls (Sec. II, eq. rotctrl)


def test_bspline_partition_of_unity_and_shape():
    T, Ns = 7.0, 9
    dtau = T / (Ns - 2)
    for t in np.linspace(0.0, T, 101):
        assert abs(sum(model.bspline_basis(s, t, Ns, T) for s in range(Ns)) - 1.0) < 1e-14
        assert sum(model.bspline_basis(s, t, Ns, T) > 0 for s in range(Ns)) <= 3
    # centred values of the uniform quadratic B-spline: 3/4 at the centre, 1/2 at +-dtau/2, 1/8 at +-dtau
    s = 4
    c = (s - 0.5) * dtau
    assert abs(model.bspline_basis(s, c, Ns, T) - 0.75) < 1e-15
    assert abs(model.bspline_basis(s, c + dtau / 2, Ns, T) - 0.5) < 1e-15
    assert abs(model.bspline_basis(s, c - dtau, Ns, T) - 0.125) < 1e-15
    assert model.bspline_basis(s, c + 1.5 * dtau, Ns, T) == 0.0
    # unit area (times dtau) and C1 continuity at a knot
    xs = np.linspace(c - 1.5 * dtau, c + 1.5 * dtau, 30001)
    area = np.trapezoid([model.bspline_basis(s, x, Ns, T) for x in xs], xs)
    assert abs(area - dtau) < 1e-6
    e = 1e-7
    k = c + dtau / 2
    dl = (model.bspline_basis(s, k, Ns, T) - model.bspline_basis(s, k - e, Ns, T)) / e
    dr = (model.bspline_basis(s, k + e, Ns, T) - model.bspline_basis(s, k, Ns, T)) / e
    assert abs(dl - dr) < 1e-5


def test_control_amplitude_single_coefficient():
    """One nonzero coefficient alpha_q^{s,f}: d_q(t) = 2pi alpha S_s(t) e^{i 2pi Omega t}
    and the other subsystems see no drive."""
    p = W.random_problem(13, levels=(2, 2), n_splines=6, n_carriers=2)
    p.controls.alpha[:] = 0
    k = model.alpha_index(p.controls, 1, 1, 3)
    p.controls.alpha[k] = 0.3
    p.controls.alpha[k + 1] = -0.2
    om = p.controls.carriers_ghz[1][1]
    T = p.system.T_ns
    for t in (0.1, 1.3, 2.2, 3.9):
        d = model.control_amplitudes(p.controls, t, T)
        expect = TWO_PI * (0.3 - 0.2j) * model.bspline_basis(3, t, 6, T) * np.exp(1j * TWO_PI * om * t)
        assert abs(d[1] - expect) < 1e-14 and d[0] == 0


# ----------------------------------------------------------------------------
# structure of the vectorised Lindbladian (Appendix A)


@pytest.mark.parametrize("levels", [(2,), (3,), (2, 3), (3, 2, 2)])
def test_lindbladian_structure(levels):
    p = W.random_problem(21, levels=levels)
    m = model.Model(p.system, p.controls)
    t = 1.234
    M = m.M(t)
    H = m.H(t)
    N = m.N
    rng = np.random.default_rng(5)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    # Kronecker (vectorised) form equals the matrix form of the master equation
    assert np.allclose(M @ model.vec(X), model.vec(model.lindblad_matrix_form(H, m.Ls, X)), atol=1e-12, rtol=0)
    assert np.allclose(M.conj().T @ model.vec(X), model.vec(model.adjoint_matrix_form(H, m.Ls, X)),
                       atol=1e-12, rtol=0)
    # trace preserving generator: vec(I)^H M = 0
    assert np.max(np.abs(model.vec(np.eye(N)).conj() @ M)) < 1e-12
    # Hermiticity preserving: L(X^+) = L(X)^+
    Y = model.unvec(M @ model.vec(X), N)
    Yd = model.unvec(M @ model.vec(X.conj().T), N)
    assert np.allclose(Yd, Y.conj().T, atol=1e-12, rtol=0)
    # a Hamiltonian is Hermitian
    assert np.allclose(H, H.conj().T)
    # without collapse operators M is skew-Hermitian (Appendix A)
    p0 = W.random_problem(21, levels=levels, dissipation=False)
    m0 = model.Model(p0.system, p0.controls)
    M0 = m0.M(t)
    assert np.max(np.abs(M0 + M0.conj().T)) < 1e-12


def test_lindbladian_matches_textbook_qubit_generator():
    """Brute force for one qubit: the 4x4 generator written out by hand from
    rho' = -i[H, rho] + D[a]/T1 + D[n]/T2 with H = w n + d a + conj(d) a^+."""
    p = W.random_problem(22, levels=(2,))
    m = model.Model(p.system, p.controls)
    t = 0.77
    d = m.d(t)[0]
    w = TWO_PI * p.system.detuning_ghz[0]
    g1 = 1 / (1000 * p.system.t1_us[0])
    g2 = 1 / (1000 * p.system.t2_us[0])

    def gen(X):
        r00, r01, r10, r11 = X[0, 0], X[0, 1], X[1, 0], X[1, 1]
        # H = [[0, d], [conj d, w]]; [H, X] elementwise
        c00 = d * r10 - r01 * np.conj(d)
        c01 = d * r11 - (r00 * d + r01 * w)
        c10 = (np.conj(d) * r00 + w * r10) - r11 * np.conj(d)
        c11 = (np.conj(d) * r01 + w * r11) - (r10 * d + r11 * w)
        return np.array([
            [-1j * c00 + g1 * r11, -1j * c01 - (g1 / 2 + g2 / 2) * r01],
            [-1j * c10 - (g1 / 2 + g2 / 2) * r10, -1j * c11 - g1 * r11],
        ])

    M = m.M(t)
    for k in range(4):
        e = np.zeros(4, dtype=np.complex128)
        e[k] = 1
        assert np.allclose(M @ e, model.vec(gen(model.unvec(e, 2))), atol=1e-14, rtol=0)


# ----------------------------------------------------------------------------
# invariants of the discrete evolution


def test_closed_system_is_unitary():
    """No collapse operators: the IMR propagator is the Cayley transform of a
    skew-Hermitian matrix, hence unitary; ||q||_2 and Tr rho^2 are preserved."""
    p = W.random_problem(31, levels=(3, 2), n_states=2, n_steps=60, dissipation=False, hermitian=False)
    fw = imr.forward(p)
    for j in (0, 17, 60):
        assert np.allclose(np.linalg.norm(fw["q"][j], axis=0), np.linalg.norm(fw["q"][0], axis=0), atol=1e-13)


def test_trace_and_hermiticity_preserved():
    p = W.random_problem(32, levels=(2, 3), n_states=3, n_steps=80)
    rT = imr.forward(p, keep=False)["rhoT"]
    for r in rT:
        assert abs(np.trace(r) - 1) < 1e-13
        assert np.max(np.abs(r - r.conj().T)) < 1e-14


def test_linearity_over_initial_states():
    """The solution is linear in the initial state (Sec. III-B): evolving the
    mean equals the mean of the evolutions."""
    p = W.random_problem(33, levels=(2, 2), n_states=4, n_steps=30, hermitian=False)
    rT = imr.forward(p, keep=False)["rhoT"]
    pm = copy.deepcopy(p)
    pm.rho0 = p.rho0.mean(axis=0)[None]
    pm.targets = p.targets[:1]
    pm.weights = None
    rTm = imr.forward(pm, keep=False)["rhoT"][0]
    assert np.max(np.abs(rTm - rT.mean(axis=0))) < 1e-14


def test_frobenius_trace_identity():
    """J_Frob = J_Tr - 1/2 (1 - Tr rho_tar^2) - 1/2 (1 - Tr rho^2) (Sec. III-C)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        A = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
        rho = A @ A.conj().T
        rho /= np.trace(rho)
        tar = W.synthetic.pure_density(W.random_pure_state(rng, 5))
        jf = imr.merit("frob", tar, rho)
        jt = imr.merit("trace", tar, rho)
        pur_t = np.real(np.trace(tar @ tar))
        pur = np.real(np.trace(rho @ rho))
        assert abs(jf - (jt - 0.5 * (1 - pur_t) - 0.5 * (1 - pur))) < 1e-14


def test_gate_targets_brute_force():
    """CNOT (control = subsystem 0) on the 2-level essential subspace of two
    3-level transmons, and X on a qubit."""
    p = W.config2(n_steps=10)
    tars = imr.targets_of(p)
    # initial state |i><j| over essential indices, ordered i-major
    def full(i):
        return {0: 0, 1: 1, 2: 3, 3: 4}[i]
    cnot = {0: 0, 1: 1, 2: 3, 3: 2}
    for i in range(4):
        for j in range(4):
            r = tars[4 * i + j]
            e = np.zeros((9, 9))
            e[full(cnot[i]), full(cnot[j])] = 1
            assert np.array_equal(r, e)
            assert np.array_equal(p.rho0[4 * i + j], np.eye(9)[full(i)][:, None] * np.eye(9)[full(j)][None, :])
    p1 = W.config1(n_steps=10)
    t1 = imr.targets_of(p1)
    assert np.array_equal(t1[0], np.diag([0.0, 1.0])) and np.array_equal(t1[3], np.diag([1.0, 0.0]))
    assert np.array_equal(t1[1], np.array([[0, 0], [1, 0]]))


# ----------------------------------------------------------------------------
# discrete adjoint (Appendix B)


def test_adjoint_dot_product_identity():
    """The discrete adjoint is the exact transpose of the linearised forward
    map: Re <qhat^0, dq^0> = Re <qhat^N, dq^N> for any perturbation dq^0."""
    p = W.random_problem(41, levels=(2, 3), n_states=2, n_steps=15, hermitian=False)
    lams = imr.adjoint_states(p)
    rng = np.random.default_rng(9)
    N = 6
    dq0 = rng.standard_normal((N * N, 2)) + 1j * rng.standard_normal((N * N, 2))
    pd = copy.deepcopy(p)
    pd.rho0 = np.stack([model.unvec(dq0[:, i], N) for i in range(2)])
    dqN = model.vec(imr.forward(pd, keep=False)["rhoT"]).T
    lhs = np.real(np.sum(lams[-1].conj() * dq0))
    rhs = np.real(np.sum(lams[0].conj() * dqN))
    assert abs(lhs - rhs) < 1e-13 * max(1, abs(lhs))


@pytest.mark.parametrize("objective,hermitian,gamma2", [("frob", False, 0.0), ("trace", True, 0.3), ("frob", True, 0.1)])
def test_gradient_matches_central_differences(objective, hermitian, gamma2):
    """Exactness of the discrete adjoint gradient for finite dt (Sec. III):
    every component against central differences to 1e-6 relative."""
    p = W.random_problem(42, levels=(2, 3), n_states=2, n_steps=12, objective=objective,
                         hermitian=hermitian, gamma2=gamma2, n_splines=5, n_carriers=2)
    G, g, _ = imr.gradient(p)
    assert abs(G - imr.value(p)) < 1e-15
    fd = imr.fd_gradient(p, eps=1e-6)
    scale = max(np.max(np.abs(g)), 1e-3)
    for k, v in fd.items():
        assert abs(g[k] - v) <= 1e-6 * scale, (k, g[k], v)


def test_control_horizon_prefix_is_the_longer_problem_truncated():
    """A problem that integrates the first steps of a longer horizon with the
    longer horizon's controls (eq. rotctrl, splines on [0, T_c]) steps
    exactly like the longer problem's first steps, and its adjoint gradient
    -- whose spline factors come from the same horizon -- matches central
    differences; spline coefficients whose support starts after the prefix
    get no gradient."""
    p = W.random_problem(71, levels=(2, 2), n_states=2, n_steps=40, T_ns=0.8, amp=0.1, n_splines=8)
    full = imr.forward(p, keep=True)
    pre = copy.deepcopy(p)
    pre.controls.horizon_ns = p.system.T_ns
    pre.system.n_steps = 10
    pre.system.T_ns = 0.2
    fp = imr.forward(pre, keep=True)
    for j in range(11):
        assert np.max(np.abs(fp["q"][j] - full["q"][j])) <= 1e-14
    G, g, _ = imr.gradient(pre)
    idx = [0, 1, 2, 3, 9, 10]
    fd = imr.fd_gradient(pre, eps=1e-6, indices=idx)
    scale = max(np.max(np.abs(g)), 1e-3)
    for k in idx:
        assert abs(g[k] - fd[k]) <= 1e-6 * scale, (k, g[k], fd[k])
    # spline s is supported on ((s - 2) dtau, (s + 1) dtau), dtau = 0.8/6: the
    # 0.2 ns prefix meets splines 0..3 only
    ctrl = pre.controls
    for q, car in enumerate(ctrl.carriers_ghz):
        for f in range(len(car)):
            for sp in range(4, ctrl.n_splines):
                k = model.alpha_index(ctrl, q, f, sp)
                assert g[k] == 0.0 and g[k + 1] == 0.0


def test_gradient_matches_fd_for_config_shapes():
    """The workload conventions (essential levels, CNOT, two carriers) under
    central differences, on a 100-step prefix of the 2 x 3-level workload."""
    p = W.config2(n_steps=100)
    p.system.T_ns = 2.0
    p.controls.alpha *= 20
    G, g, _ = imr.gradient(p)
    idx = list(range(0, len(g), 11))
    fd = imr.fd_gradient(p, eps=1e-5, indices=idx)
    scale = np.max(np.abs(g))
    for k in idx:
        assert abs(g[k] - fd[k]) <= 1e-6 * scale, (k, g[k], fd[k])


def test_jnm_values_and_gradient():
    """J_Nm (Sec. III-B, eq. Jmeasure): Tr(N_m |l><l|) = |l - m|, J_Nm >= 0 on
    density matrices with equality only at |m><m|; the adjoint gradient of
    the reset problem from the ensemble state agrees with central
    differences."""
    N, m = 6, 2
    Nm = imr.observable_nm(N, m)
    for l in range(N):
        e = np.zeros((N, N), dtype=np.complex128)
        e[l, l] = 1.0
        assert imr.merit("nm", Nm, e) == abs(l - m)
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
        rho = A @ A.conj().T
        rho /= np.trace(rho).real
        assert imr.merit("nm", Nm, rho) > 0.0
    p = W.reset_ensemble(levels=(2, 3), n_steps=12, T_ns=1.0, n_splines=5, amp=0.2)
    assert abs(np.trace(p.rho0[0]) - 1.0) < 1e-15 and np.min(np.linalg.eigvalsh(p.rho0[0])) > 0.0
    G, g, _ = imr.gradient(p)
    fd = imr.fd_gradient(p, eps=1e-6)
    scale = np.max(np.abs(g))
    for k, v in fd.items():
        assert abs(g[k] - v) <= 1e-6 * scale, (k, g[k], v)


def test_basis_matrices_are_pure_states():
    """The N^2 basis matrices B^kj (Sec. III-B) are density matrices of pure
    states (Hermitian, unit trace, rank one), as the paper states -- which
    pins the reading of the garbled k > j case."""
    B = W.basis_matrices(4).reshape(-1, 4, 4)
    for b in B:
        assert np.allclose(b, b.conj().T, atol=0)
        assert abs(np.trace(b) - 1.0) < 1e-15
        ev = np.linalg.eigvalsh(b)
        assert abs(ev[-1] - 1.0) < 1e-14 and np.max(np.abs(ev[:-1])) < 1e-14


def _jc_pair(g, eta, T, n_steps, levels=(2, 2)):
    sysm, ctrl = _undriven(levels, [0.0, 0.0], [0.0, 0.0], [INF, INF], [INF, INF], T=T, n_steps=n_steps)
    jc = np.zeros((2, 2))
    jc[0, 1] = g
    sysm.jc_ghz = jc
    sysm.rot_ghz = np.array([eta, 0.0])
    return sysm, ctrl


def test_jaynes_cummings_resonant_swap_discrete_closed_form():
    """Resonant Jaynes-Cummings coupling of two qubits (Sec. II), |10> at
    t = 0: the eigenstates (|01> +- |10>)/sqrt 2 of the one-excitation block
    have energies +-omega, omega = 2 pi g, so their coherence turns by
    2 atan(omega dt) per implicit-midpoint step and P(|01>) after n steps is
    (1 - cos(2 n atan(omega dt)))/2 exactly."""
    g, T, n = 0.0123, 37.0, 300
    sysm, ctrl = _jc_pair(g, 0.0, T, n)
    rho = np.zeros((4, 4), dtype=np.complex128)
    rho[2, 2] = 1.0
    rT = imr.forward(_problem(sysm, ctrl, rho), keep=False)["rhoT"][0]
    om, h = TWO_PI * g, T / n
    p01 = 0.5 * (1 - math.cos(2 * n * math.atan(om * h)))
    assert abs(rT[1, 1].real - p01) < 1e-13
    assert abs(rT[2, 2].real - (1 - p01)) < 1e-13
    assert abs(np.trace(rT) - 1) < 1e-14


def test_jaynes_cummings_detuned_phases_against_schrodinger():
    """Detuned coupling (omega_0^rot - omega_1^rot = eta): the state of the
    closed system is a pure state whose one-excitation amplitudes obey
    i c' = H(t) c with H = g [[0, e^{-i eta t}], [e^{i eta t}, 0]] in the
    basis (|01>, |10>); the IMR density matrix matches the outer product of a
    tight Runge-Kutta solution to the method's O(dt^2) error, phases
    included (which fixes the sign of eta)."""
    from scipy.integrate import solve_ivp

    g, eta, T, n = 0.02, 0.031, 20.0, 4000
    sysm, ctrl = _jc_pair(g, eta, T, n)
    rho = np.zeros((4, 4), dtype=np.complex128)
    rho[2, 2] = 1.0
    rT = imr.forward(_problem(sysm, ctrl, rho), keep=False)["rhoT"][0]
    w, e = TWO_PI * g, TWO_PI * eta

    def rhs(t, y):
        c = y[:2] + 1j * y[2:]
        Hm = np.array([[0, w * np.exp(-1j * e * t)], [w * np.exp(1j * e * t), 0]])
        dc = -1j * Hm @ c
        return np.concatenate([dc.real, dc.imag])

    sol = solve_ivp(rhs, (0, T), [0.0, 1.0, 0.0, 0.0], rtol=1e-12, atol=1e-13)
    c = sol.y[:2, -1] + 1j * sol.y[2:, -1]
    ref = np.outer(c, c.conj())  # rows/columns: |01> (index 1), |10> (index 2)
    sub = rT[np.ix_([1, 2], [1, 2])]
    assert np.max(np.abs(sub - ref)) < 2e-5
    assert abs(ref[0, 1]) > 0.01  # a coherence large enough for its phase to matter


def test_running_penalty_closed_form_and_gradient():
    """The running penalty gamma1 int beta(t) J dt (Sec. III, eq.
    optimproblem), by the left rectangle rule: for an undriven qubit from
    |1><1| with J_Frob to |0><0|, J(q^j) = (1 - c^j)^2 with c the Cayley
    factor of the T1 decay, so the penalty is a closed-form sum; and with
    controls on, the adjoint gradient (sources included) matches central
    differences for every merit functional."""
    sysm, ctrl = _undriven((2,), [0.0], [0.0], [0.4], [INF], T=30.0, n_steps=300)
    one = np.diag([0.0, 1.0]).astype(np.complex128)
    zero = np.diag([1.0, 0.0]).astype(np.complex128)
    p = W.Problem("pen", sysm, ctrl, one[None], "frob", targets=zero[None], gamma1=0.7, penalty_a=8.0)
    h = sysm.T_ns / sysm.n_steps
    g1 = 1.0 / 400.0
    c = (1 - h * g1 / 2) / (1 + h * g1 / 2)
    expect = 0.0
    for j in range(sysm.n_steps):
        pop1 = c ** j
        J = pop1 ** 2  # |rho - |0><0||_F^2 / 2 with rho = diag(1 - pop1, pop1)
        t = j * h
        expect += h * math.exp(-(((t - sysm.T_ns) / 8.0) ** 2)) / 8.0 * J
    G = imr.value(p)
    GT = c ** (2 * sysm.n_steps)
    assert abs(G - (GT + 0.7 * expect)) < 1e-13
    for objective in ("frob", "trace"):
        q = W.random_problem(43, levels=(2, 3), n_states=2, n_steps=12, objective=objective, n_splines=5)
        q.gamma1, q.penalty_a = 0.8, 0.3
        Gq, g, _ = imr.gradient(q)
        assert abs(Gq - imr.value(q)) < 1e-15
        fd = imr.fd_gradient(q, eps=1e-6)
        scale = np.max(np.abs(g))
        for k, v in fd.items():
            assert abs(g[k] - v) <= 1e-6 * scale, (objective, k, g[k], v)
