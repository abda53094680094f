"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (stated by the method's accuracy targets): states and objectives
1e-10 relative, gradients 1e-9 relative to the oracle's adjoint gradient and
1e-6 to central differences; a single Lindbladian apply or IMR step agrees to
a few units of FP64 rounding (1e-13 relative)."""

import copy

import numpy as np
import pytest

import workloads as W
from oracle import imr, model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10310_gb300 import _lib as L

    L.load(build_if_missing=True)


def _sys(prob, **kw):
    from paper_2110_10310_gb300.system import LindbladSystem

    return LindbladSystem(prob, **kw)


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rand_states(rng, n, N):
    x = rng.standard_normal((n, N, N)) + 1j * rng.standard_normal((n, N, N))
    return x


SHAPES = [(2,), (3,), (2, 3), (4, 3), (2, 2, 2), (3, 2, 4), (4, 4, 4)]


@pytest.mark.parametrize("levels", SHAPES)
def test_apply_matches_dense_lindbladian(levels):
    """y = M^{j+1/2} x and (M^{j+1/2})^+ x against the dense Kronecker M."""
    p = W.random_problem(101, levels=levels, n_states=1, n_steps=10)
    s = _sys(p)
    m = model.Model(p.system, p.controls)
    N = m.N
    rng = np.random.default_rng(1)
    X = _rand_states(rng, 3, N)
    xt = torch.from_numpy(X).cuda()
    for j in (0, 7):
        Md = m.M(m.t_half(j))
        for adj in (False, True):
            A = Md.conj().T if adj else Md
            y = s.apply(xt, j, adjoint=adj).cpu().numpy()
            ref = np.stack([model.unvec(A @ model.vec(X[b]), N) for b in range(3)])
            scale = np.max(np.abs(A).sum(axis=1)) * np.max(np.abs(X))
            assert np.max(np.abs(y - ref)) <= 1e-14 * scale, (levels, j, adj)


@pytest.mark.parametrize("levels,sweep", [((2, 3), "cluster"), ((2, 3), "resident"), ((3, 2, 2), "auto"),
                                          ((4, 4), "auto"), ((3, 3, 3), "grid")])
def test_steps_match_oracle(levels, sweep):
    """lb_propagate over a few forward and adjoint IMR steps from random states,
    on each sweep kind."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"auto": L.LB_SWEEP_AUTO, "cluster": L.LB_SWEEP_CLUSTER, "resident": L.LB_SWEEP_RESIDENT,
          "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.random_problem(102, levels=levels, n_states=2, n_steps=12, T_ns=0.24, amp=0.1)
    s = _sys(p, sweep=sw)
    mdl = model.Model(p.system, p.controls)
    N = mdl.N
    rng = np.random.default_rng(2)
    X = _rand_states(rng, 2, N)
    got = s.propagate(torch.from_numpy(X).cuda(), 3, 8).cpu().numpy()
    Q = model.vec(X).T.copy()
    for j in range(3, 8):
        Q, _ = imr.imr_step(mdl, j, Q)
    ref = np.stack([model.unvec(Q[:, i], N) for i in range(2)])
    assert _rel(got, ref) < 1e-13
    # adjoint steps j = 7..3: (I - h/2 M^+) zh = lam, lam <- lam + h M^+ zh
    got = s.propagate(torch.from_numpy(X).cuda(), 3, 8, adjoint=True).cpu().numpy()
    lam = model.vec(X).T.copy()
    I = np.eye(N * N)
    for j in range(7, 2, -1):
        MH = mdl.M(mdl.t_half(j)).conj().T
        zh = np.linalg.solve(I - 0.5 * mdl.h * MH, lam)
        lam = lam + mdl.h * (MH @ zh)
    ref = np.stack([model.unvec(lam[:, i], N) for i in range(2)])
    assert _rel(got, ref) < 1e-13


def _check_problem(p, state_tol=1e-10, grad_tol=1e-9, **kw):
    s = _sys(p, **kw)
    G, rhoT = s.forward(want_states=True)
    Gg, g = s.gradient()
    Go, go, fw = imr.gradient(p)
    assert abs(G - Go) <= state_tol * abs(Go)
    assert abs(Gg - Go) <= state_tol * abs(Go)
    assert _rel(rhoT.cpu().numpy(), fw["rhoT"]) < state_tol
    assert _rel(g, go) < grad_tol
    return s, g


def test_config1_full_horizon():
    """1 qubit, 1000 steps, X-gate objective: states, G and gradient."""
    _check_problem(W.config1())


@pytest.mark.slow
def test_config2_full_horizon():
    """2 transmons x 3 levels, 10000 steps, CNOT on the essential subspace."""
    s, _ = _check_problem(W.config2())
    st = s.stats()
    # 16 states |i><j|, 6 conjugate pairs: 10 integrated; forward and adjoint
    # sweeps, plus the recompute sweep when checkpointing
    assert st["states_integrated"] == 10
    assert st["state_steps"] == 10 * 10000 * (3 if st["ckpt_every"] > 0 else 2)


@pytest.mark.parametrize("seed,objective,hermitian,gamma2,diss", [
    (201, "frob", False, 0.0, True),
    (202, "trace", True, 0.2, True),
    (203, "frob", True, 0.0, False),
    (204, "trace", False, 0.05, False),
])
def test_random_problems_match_oracle(seed, objective, hermitian, gamma2, diss):
    p = W.random_problem(seed, levels=(2, 3), n_states=3, n_steps=40, T_ns=0.8, amp=0.1, objective=objective,
                         hermitian=hermitian, gamma2=gamma2, dissipation=diss, ckpt_every=7)
    _check_problem(p)


@pytest.mark.parametrize("sweep", ["auto", "resident", "grid"])
def test_conjugate_pairs_match_oracle_and_unpaired_run(sweep):
    """|i><j| and |j><i| integrated once (lb_set_pairing): all 16 final states,
    the objective and the gradient of the gate workload against the oracle,
    and against the run that integrates every state; explicit targets that
    pair like the states (J_Tr) too."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"auto": L.LB_SWEEP_AUTO, "resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.prefix(W.config2(), 300)
    s, g = _check_problem(p, sweep=sw)
    assert s.stats()["states_integrated"] == 10
    s0 = _sys(p, sweep=sw, pairing=0)
    G0, g0 = s0.gradient()
    G1, g1 = s.gradient()
    assert s0.stats()["states_integrated"] == 16
    assert abs(G1 - G0) <= 1e-13 * abs(G0)
    assert _rel(g1, g0) < 1e-12
    # explicit targets in the same conjugate pairs as the states
    rng = np.random.default_rng(8)
    q = W.random_problem(417, levels=(3, 2), n_states=4, n_steps=30, T_ns=0.6, amp=0.1, objective="trace")
    X = rng.standard_normal((2, 6, 6)) + 1j * rng.standard_normal((2, 6, 6))
    T = rng.standard_normal((2, 6, 6)) + 1j * rng.standard_normal((2, 6, 6))
    q.rho0 = np.stack([X[0], X[0].conj().T, X[1], X[1].conj().T])
    q.targets = np.stack([T[0], T[0].conj().T, T[1], T[1].conj().T])
    sq, _ = _check_problem(q, sweep=sw)
    assert sq.stats()["states_integrated"] == 2
    # a workspace bound with these pairs refuses states that pair otherwise
    with pytest.raises(L.LBError) as e:
        sq.set_states_host(np.stack([X[0], X[1], X[0].conj().T, X[1].conj().T]), q.weights)
    assert e.value.code == L.LB_EINVAL


def test_gradient_matches_central_differences_on_gpu():
    """Central differences of the GPU objective against the GPU adjoint gradient."""
    p = W.random_problem(205, levels=(3, 2), n_states=2, n_steps=30, T_ns=0.6, amp=0.1, n_splines=6)
    s = _sys(p)
    G, g = s.gradient()
    a0 = p.controls.alpha.copy()
    eps = 1e-6
    scale = np.max(np.abs(g))
    for k in range(0, len(a0), 5):
        a = a0.copy()
        a[k] += eps
        s.set_alpha(a)
        gp = s.forward()
        a[k] -= 2 * eps
        s.set_alpha(a)
        gm = s.forward()
        assert abs((gp - gm) / (2 * eps) - g[k]) <= 1e-6 * scale, k
    s.set_alpha(a0)


def test_checkpoint_interval_bitwise_identical():
    """Without a forward predictor, checkpoint intervals K = 1, 7 and 100 give
    bit-identical gradients; the full tape (K = 0, whose forward sweep
    predicts its first iterates) agrees to rounding."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(206, levels=(2, 2), n_states=2, n_steps=45, T_ns=0.9, amp=0.1)
    res = []
    for K in (1, 7, 100):
        s = _sys(p, ckpt_every=K, predictor=L.LB_PRED_NONE)
        res.append(s.gradient())
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    G0, g0 = _sys(p, ckpt_every=0).gradient()
    assert abs(G0 - res[0][0]) <= 1e-13 * abs(res[0][0])
    assert _rel(g0, res[0][1]) < 1e-12


@pytest.mark.parametrize("sweep", ["auto", "cluster", "resident", "grid"])
def test_neumann_solver_agrees_with_jacobi(sweep):
    from paper_2110_10310_gb300 import _lib as L

    sw = {"auto": L.LB_SWEEP_AUTO, "cluster": L.LB_SWEEP_CLUSTER, "resident": L.LB_SWEEP_RESIDENT,
          "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.random_problem(207, levels=(3, 3), n_states=2, n_steps=60, T_ns=1.2, amp=0.05)
    Gj, gj = _sys(p, solver=L.LB_SOLVER_JACOBI, sweep=sw).gradient()
    Gn, gn = _sys(p, solver=L.LB_SOLVER_NEUMANN, sweep=sw).gradient()
    assert abs(Gj - Gn) <= 1e-12 * abs(Gj)
    assert _rel(gn, gj) < 1e-10


def test_batch_matches_plain_and_oracle():
    """Independent problems of uneven size in one launch (and as a CUDA graph)
    against one launch sequence per problem, and against the oracle."""
    from paper_2110_10310_gb300 import _lib as L
    from paper_2110_10310_gb300.system import LindbladBatch

    probs = W.config3(n_problems=12, n_steps=60)
    systems = [_sys(p, sweep=L.LB_SWEEP_RESIDENT) for p in probs]
    plain = [s.gradient() for s in systems]
    b = LindbladBatch(systems)
    Gb, gb = b.gradient()
    off = 0
    for i, (G, g) in enumerate(plain):
        assert abs(Gb[i] - G) <= 1e-12 * abs(G)
        assert _rel(gb[off:off + len(g)], g) < 1e-10
        off += len(g)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.capture(1, stream=stream)
        Gc, gc = b.gradient(stream=stream)
    assert np.array_equal(Gc, Gb) and np.array_equal(gc, gb)
    for i in (0, 5, 11):
        Go, go, _ = imr.gradient(probs[i])
        assert abs(Gb[i] - Go) <= 1e-10 * abs(Go)
        off = sum(len(plain[k][1]) for k in range(i))
        assert _rel(gb[off:off + len(go)], go) < 1e-9


def test_autograd_function():
    from paper_2110_10310_gb300.system import objective

    p = W.random_problem(208, levels=(2, 2), n_states=2, n_steps=20, T_ns=0.4, amp=0.1)
    s = _sys(p)
    a = torch.tensor(p.controls.alpha, dtype=torch.float64, requires_grad=True)
    G = objective(a, s)
    (3.0 * G).backward()
    G0, g0 = s.gradient()
    assert abs(G.item() - G0) == 0.0
    assert np.allclose(a.grad.numpy(), 3.0 * g0, rtol=0, atol=0)


def test_errors_are_reported_and_recoverable():
    """Non-convergence is a host-visible status, and the handle stays usable."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(209, levels=(2, 3), n_states=1, n_steps=10)
    s = _sys(p, max_iter=1)
    with pytest.raises(L.LBError) as e:
        s.forward()
    assert e.value.code == L.LB_ENOTCONV
    assert "time step 0" in str(e.value)
    # a step so large that the fixed point diverges
    p2 = W.random_problem(210, levels=(3, 3), n_states=1, n_steps=1, T_ns=400.0, amp=3.0)
    s2 = _sys(p2, max_iter=500)
    with pytest.raises(L.LBError) as e2:
        s2.forward()
    assert e2.value.code in (L.LB_ENOTCONV, L.LB_ENAN)
    # the same process and context continue to work
    s3 = _sys(W.random_problem(211, levels=(2,), n_states=1, n_steps=5, T_ns=0.1, amp=0.1))
    s3.forward()


@pytest.mark.parametrize("sweep", ["grid", "resident", "cluster"])
def test_overflowing_input_reports_nan_with_its_step(sweep):
    """Failure detection by input, not by a device fault: control coefficients
    of 1e300 GHz make the first step's fixed point overflow to Inf, and a NaN
    entry in an initial state is caught by the first solve; both come back as
    LB_ENAN naming time step 0, and the same handle then computes the oracle's
    gradient."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID, "cluster": L.LB_SWEEP_CLUSTER}[sweep]
    p = W.random_problem(213, levels=(3, 2), n_states=2, n_steps=6, T_ns=0.12, amp=0.1)
    s = _sys(p, sweep=sw)
    a0 = p.controls.alpha.copy()
    s.set_alpha(np.full_like(a0, 1e300))
    with pytest.raises(L.LBError) as e:
        s.gradient()
    assert e.value.code == L.LB_ENAN
    assert "time step 0" in str(e.value)
    s.set_alpha(a0)
    bad = p.rho0.copy()
    bad[1, 2, 2] = np.nan
    s.set_states_host(bad, p.weights)
    with pytest.raises(L.LBError) as e:
        s.forward()
    assert e.value.code == L.LB_ENAN
    assert "time step 0" in str(e.value)
    s.set_states_host(p.rho0, p.weights)
    G, g = s.gradient()
    Go, go, _ = imr.gradient(p)
    assert abs(G - Go) <= 1e-10 * abs(Go)
    assert _rel(g, go) < 1e-9


def test_grid_barrier_wait_that_gives_up_is_reported_and_recovered():
    """A grid-barrier wait bounded to one poll gives up (the other blocks have
    not arrived yet): every block returns, the call reports LB_ECUDA with the
    time step, and after the default bound is restored the same handle
    computes the oracle's gradient."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(214, levels=(3, 3), n_states=2, n_steps=8, T_ns=0.16, amp=0.1)
    s = _sys(p, sweep=L.LB_SWEEP_GRID)
    lib = L.load()
    L.check(lib.lb_set_wait_limit(s.h, 1))
    with pytest.raises(L.LBError) as e:
        s.gradient()
    assert e.value.code == L.LB_ECUDA
    assert "grid barrier wait gave up at time step" in str(e.value)
    L.check(lib.lb_set_wait_limit(s.h, 0))
    G, g = s.gradient()
    Go, go, _ = imr.gradient(p)
    assert abs(G - Go) <= 1e-10 * abs(Go)
    assert _rel(g, go) < 1e-9
    assert lib.lb_set_wait_limit(s.h, -1) == L.LB_EINVAL


def test_host_buffers_roundtrip():
    """States set from pinned host memory through the ABI give the same result."""
    p = W.random_problem(212, levels=(2, 3), n_states=2, n_steps=15, T_ns=0.3, amp=0.1)
    s = _sys(p)
    G0 = s.forward()
    from paper_2110_10310_gb300.system import colmajor

    pinned = torch.from_numpy(colmajor(p.rho0)).pin_memory()
    s.set_states_host(pinned, p.weights)
    torch.cuda.synchronize()
    assert s.forward() == G0


# ----------------------------------------------------------------------------
# grid-wide sweeps (one cooperative launch over all SMs and states)


@pytest.mark.parametrize("levels,K,herm", [((2, 3), 7, False), ((3, 2, 2), 0, True), ((4, 3), 100, False)])
def test_grid_sweep_matches_oracle(levels, K, herm):
    """The grid sweep forced on small states: oracle parity, and agreement with
    the one-CTA-per-state sweep."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(401, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, ckpt_every=K,
                         hermitian=herm)
    _, g = _check_problem(p, sweep=L.LB_SWEEP_GRID)
    Gr, gr = _sys(p, sweep=L.LB_SWEEP_RESIDENT).gradient()
    Gg, gg = _sys(p, sweep=L.LB_SWEEP_GRID).gradient()
    assert abs(Gg - Gr) <= 1e-12 * abs(Gr)
    assert _rel(gg, gr) < 1e-11


@pytest.mark.parametrize("levels,K,herm,coupled", [((3, 3), 7, True, False), ((2, 3), 0, False, False),
                                                  ((3, 2, 2), 10, True, True)])
def test_difference_iterations_match_oracle_and_fp64_iterations(levels, K, herm, coupled):
    """Grid sweeps with single-precision difference iterations (the default)
    against every iteration in FP64 and against the oracle.  A coarse step
    without a predictor needs ~10 inner iterations per step, the last third
    of them difference iterations: states and objective to 1e-10 of the oracle,
    gradient to 1e-9, and the two iteration schemes to 1e-12 (both stop at
    rtol 1e-15 of |q|; they differ by rounding)."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(411, levels=levels, n_states=3, n_steps=30, T_ns=1.2, amp=0.1, ckpt_every=K,
                         hermitian=herm, jc=0.05 if coupled else 0.0)
    kw = dict(sweep=L.LB_SWEEP_GRID, predictor=L.LB_PRED_NONE)
    s, g = _check_problem(p, **kw)
    st = s.stats()
    assert st["sweep"] == "grid"
    assert st["symmetry"] == ("hermitian" if herm else "none")
    its = np.array(st["phase_iterations"])
    dits = np.array(st["phase_diff_iterations"])
    steps = np.array(st["phase_steps"])
    assert its[0] >= 6 * steps[0]                   # a coarse step: many inner iterations
    assert dits[0] >= 0.2 * its[0] and dits[2] >= 0.2 * its[2]
    assert np.all(dits <= its - steps)              # the first iteration of every step is FP64
    G1, rho1 = s.forward(want_states=True)
    s0 = _sys(p, difference_iterations=0, **kw)
    G0, rho0 = s0.forward(want_states=True)
    Gg0, g0 = s0.gradient()
    assert s0.stats()["phase_diff_iterations"] == [0, 0, 0]
    assert abs(G1 - G0) <= 1e-12 * abs(G0)
    assert _rel(rho1.cpu().numpy(), rho0.cpu().numpy()) < 1e-12
    assert _rel(g, g0) < 1e-12


@pytest.mark.parametrize("levels,K,herm,objective", [((3, 3), 7, True, "frob"), ((2, 3), 0, False, "trace"),
                                                    ((3, 2, 2), 10, True, "trace"), ((2, 2, 2, 2), 5, False, "frob")])
def test_paired_single_apply_matches_oracle_and_fp64(levels, K, herm, objective):
    """lb_set_precision(LB_PREC_F32X2): the grid sweeps' FP64 iterations apply
    O in pairs of single-precision numbers.  States and objective within
    1e-10 of the oracle, gradient within 1e-9, and within 1e-11 of the FP64
    apply (the two differ by a few FP64 roundings of z per step); with
    checkpoints the recompute repeats the forward sweep bit for bit (the
    same paired-single iterates), so K and the full tape agree to rounding
    and two K give the same gradient."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(421, levels=levels, n_states=3, n_steps=40, T_ns=1.2, amp=0.1, ckpt_every=K,
                         hermitian=herm, objective=objective)
    kw = dict(sweep=L.LB_SWEEP_GRID, precision=L.LB_PREC_F32X2)
    s, g = _check_problem(p, **kw)
    assert s.stats()["sweep"] == "grid"
    G1, rho1 = s.forward(want_states=True)
    s0 = _sys(p, sweep=L.LB_SWEEP_GRID)
    G0, rho0 = s0.forward(want_states=True)
    _, g0 = s0.gradient()
    assert abs(G1 - G0) <= 1e-11 * abs(G0)
    assert _rel(rho1.cpu().numpy(), rho0.cpu().numpy()) < 1e-11
    assert _rel(g, g0) < 1e-10
    if K > 0:
        Ga, ga = _sys(p, ckpt_every=K, predictor=L.LB_PRED_NONE, **kw).gradient()
        Gb, gb = _sys(p, ckpt_every=1, predictor=L.LB_PRED_NONE, **kw).gradient()
        assert Ga == Gb and np.array_equal(ga, gb)


def test_paired_single_apply_keeps_fp64_with_couplings_and_full_size():
    """Systems with Jaynes-Cummings couplings run the FP64 apply under
    LB_PREC_F32X2 (bitwise the default); the paired-single apply on the full
    six-qutrit state (vec 531441, 2 states, 12 steps) agrees with the FP64
    apply to 1e-11."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(422, levels=(3, 2, 2), n_states=2, n_steps=30, T_ns=0.6, amp=0.1, jc=0.05)
    a = _sys(p, sweep=L.LB_SWEEP_GRID, precision=L.LB_PREC_F32X2).gradient()
    b = _sys(p, sweep=L.LB_SWEEP_GRID).gradient()
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    q = W.prefix(W.config5(n_states=2), 12)
    q.ckpt_every = 6
    Gf, gf = _sys(q, precision=L.LB_PREC_F32X2).gradient()
    Gd, gd = _sys(q).gradient()
    assert abs(Gf - Gd) <= 1e-11 * abs(Gd)
    assert _rel(gf, gd) < 1e-10


def test_difference_iterations_keep_recompute_bitwise():
    """The decision to take a difference iteration depends only on the
    iterates, so a recompute repeats it: without a forward predictor the
    gradient is bitwise the same for K = 1, 5, 30 with difference iterations
    on, and the switch may be flipped on a bound handle."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(412, levels=(3, 3), n_states=2, n_steps=30, T_ns=1.2, amp=0.1, hermitian=True)
    res = []
    for K in (1, 5, 30):
        s = _sys(p, ckpt_every=K, sweep=L.LB_SWEEP_GRID, predictor=L.LB_PRED_NONE)
        res.append(s.gradient())
        assert s.stats()["phase_diff_iterations"][1] > 0
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    L.check(s.lib.lb_set_difference_iterations(s.h, 0))
    G0, g0 = s.gradient()
    assert s.stats()["phase_diff_iterations"] == [0, 0, 0]
    assert abs(G0 - res[0][0]) <= 1e-12 * abs(res[0][0]) and _rel(g0, res[0][1]) < 1e-12
    assert s.lib.lb_set_difference_iterations(s.h, 2) == L.LB_EINVAL


def test_packed_tapes_need_hermitian_states():
    """A workspace bound while the states and targets are Hermitian holds the
    grid sweeps' checkpoint and segment tapes packed (N (N + 1) / 2 entries
    per state): the gradient matches the oracle; after non-Hermitian states
    are set the call is refused on the host (LB_EINVAL) instead of
    overrunning the tapes, and Hermitian states run again on the same
    workspace."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(431, levels=(3, 3), n_states=2, n_steps=30, T_ns=0.6, amp=0.1, ckpt_every=7,
                         hermitian=True)
    s, g = _check_problem(p, sweep=L.LB_SWEEP_GRID)
    q = W.random_problem(432, levels=(3, 3), n_states=2, n_steps=30, T_ns=0.6, amp=0.1, ckpt_every=7,
                         hermitian=False)
    s.set_states_host(q.rho0, q.weights)
    with pytest.raises(L.LBError) as err:
        s.gradient()
    assert err.value.code == L.LB_EINVAL and "packed" in str(err.value)
    s.set_states_host(p.rho0, p.weights)
    G2, g2 = s.gradient()
    assert _rel(g2, g) < 1e-13


def test_grid_checkpoint_interval_bitwise_identical():
    """Grid sweeps without a forward predictor: K = 1, 7, 100 bit-identical;
    the full tape (K = 0, whose forward sweep predicts its first iterates)
    agrees to rounding."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(402, levels=(3, 3), n_states=2, n_steps=45, T_ns=0.9, amp=0.1)
    res = [_sys(p, ckpt_every=K, sweep=L.LB_SWEEP_GRID, predictor=L.LB_PRED_NONE).gradient() for K in (1, 7, 100)]
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    G0, g0 = _sys(p, ckpt_every=0, sweep=L.LB_SWEEP_GRID).gradient()
    assert abs(G0 - res[0][0]) <= 1e-13 * abs(res[0][0])
    assert _rel(g0, res[0][1]) < 1e-12


@pytest.mark.parametrize("sweep,solver", [("resident", "jacobi"), ("grid", "jacobi"), ("resident", "gmres"),
                                          ("cluster", "jacobi")])
def test_recompute_repeats_the_forward_predictor_bitwise(sweep, solver):
    """The forward predictor restarts at every checkpoint, so with
    checkpoints every K steps the gradient is bitwise that of the full stage
    tape whose forward predictor restarts every K steps (the recompute
    repeats every forward iterate), different K agree to rounding, and both
    match the oracle.  The cluster sweep predicts forward solves only with the
    full tape, so there every K >= 1 is bitwise the run without the
    predictor."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID, "cluster": L.LB_SWEEP_CLUSTER}[sweep]
    sv = {"jacobi": L.LB_SOLVER_JACOBI, "gmres": L.LB_SOLVER_GMRES}[solver]
    p = W.random_problem(411, levels=(3, 2), n_states=2, n_steps=45, T_ns=0.9, amp=0.1, ckpt_every=0)
    Go, go, _ = imr.gradient(p)
    out = {}
    for K in (5, 9):
        s = _sys(p, ckpt_every=K, sweep=sw, solver=sv)
        G, g = s.gradient()
        out[K] = (G, g, s.stats())
        R = L.LB_PRED_NONE if sweep == "cluster" else K
        G0, g0 = _sys(p, ckpt_every=0 if sweep != "cluster" else K, sweep=sw, solver=sv, predictor=R).gradient()
        assert G == G0
        assert np.array_equal(g, g0)
        assert abs(G - Go) <= 1e-10 * abs(Go)
        assert _rel(g, go) < 1e-9
    assert abs(out[5][0] - out[9][0]) <= 1e-13 * abs(out[5][0])
    assert _rel(out[5][1], out[9][1]) < 1e-11
    if sweep != "cluster":
        s0 = _sys(p, ckpt_every=9, sweep=sw, solver=sv, predictor=L.LB_PRED_NONE)
        s0.gradient()
        st0 = s0.stats()
        for ph in (0, 1):
            assert out[9][2]["phase_iterations"][ph] < st0["phase_iterations"][ph]


@pytest.mark.parametrize("sweep", ["resident", "grid"])
def test_anchored_predictor_keeps_iterations_low_across_anchor_moves(sweep):
    """The first-iterate predictor keeps its ring in the frame of an anchor
    step and moves the anchor every 256 steps.  Over the first 1200 steps of
    the CNOT workload at its dt (four anchor moves, no restarts) forward and
    adjoint solves converge in about one inner iteration per step, the
    forward ones far fewer than from the unpredicted first iterate
    (LB_PRED_NONE switches the forward predictor off; the adjoint's stays),
    and the gradient is that of the run without the forward predictor."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.prefix(W.config2(), 1200)
    s = _sys(p, ckpt_every=0, sweep=sw)
    G, g = s.gradient()
    st = s.stats()
    s0 = _sys(p, ckpt_every=0, sweep=sw, predictor=L.LB_PRED_NONE)
    G0, g0 = s0.gradient()
    st0 = s0.stats()
    per = [st["phase_iterations"][ph] / st["phase_steps"][ph] for ph in (0, 2)]
    per0 = [st0["phase_iterations"][ph] / st0["phase_steps"][ph] for ph in (0, 2)]
    assert max(per) < 1.3, (per, per0)
    assert per[0] < 0.6 * per0[0], (per, per0)
    assert abs(G - G0) <= 1e-12 * abs(G0)
    assert _rel(g, g0) < 1e-10


@pytest.mark.parametrize("sweep", ["resident", "grid", "cluster"])
def test_control_horizon_longer_than_the_run_matches_oracle(sweep):
    """A run over the first steps of a longer horizon keeps that horizon's
    B-splines (lb_controls_set_horizon): states, objective and gradient
    against the oracle on the same prefix problem."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID, "cluster": L.LB_SWEEP_CLUSTER}[sweep]
    p = W.prefix(W.random_problem(415, levels=(3, 2), n_states=2, n_steps=160, T_ns=3.2, amp=0.1, n_splines=8), 30)
    assert p.controls.horizon_ns == 3.2 and p.system.n_steps == 30
    _check_problem(p, sweep=sw, ckpt_every=7)


def test_autotune_chooses_the_predictor_order_on_grid_sweeps():
    """On a grid sweep the autotuner also times the predictor orders 6..10 and
    keeps one; the gradient afterwards still matches the oracle."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(416, levels=(3, 3), n_states=2, n_steps=60, T_ns=1.2, amp=0.1, ckpt_every=20)
    s = _sys(p, sweep=L.LB_SWEEP_GRID)
    choice = s.autotune(probe_steps=30)
    assert choice["sweep"] == "grid" and 6 <= choice["pred_order"] <= 10
    G, g = s.gradient()
    Go, go, _ = imr.gradient(p)
    assert abs(G - Go) <= 1e-10 * abs(Go)
    assert _rel(g, go) < 1e-9


def test_predictor_restart_rules():
    """A predictor that never restarts needs the full tape; a restart period
    must divide the checkpoint interval."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(412, levels=(2, 2), n_states=1, n_steps=20, T_ns=0.4, amp=0.1)
    with pytest.raises(L.LBError) as e:
        _sys(p, ckpt_every=10, predictor=0)
    assert e.value.code == L.LB_EINVAL
    with pytest.raises(L.LBError) as e:
        _sys(p, ckpt_every=10, predictor=3)
    assert e.value.code == L.LB_EINVAL
    _sys(p, ckpt_every=10, predictor=5).gradient()
    _sys(p, ckpt_every=0, predictor=0).gradient()


def _imr_residual(mdl, j, q0, q1, adjoint=False):
    """max |q1 - q0 - dt L(z)| with z = (q0 + q1)/2, L the (adjoint) Lindbladian
    at t_j + dt/2 in matrix form (any size)."""
    t = mdl.t_half(j)
    H = mdl.H(t)
    f = model.adjoint_matrix_form if adjoint else model.lindblad_matrix_form
    out = 0.0
    for a, b in zip(q0, q1):
        Z = 0.5 * (a + b)
        out = max(out, float(np.max(np.abs(b - a - mdl.h * f(H, mdl.Ls, Z)))))
    return out


@pytest.mark.parametrize("which", ["qudits_4x4", "qutrits_6x3"])
def test_full_size_steps_satisfy_imr(which):
    """At full workload size (N^2 = 65536 and 531441), forward and adjoint steps
    taken by the grid sweep satisfy the implicit midpoint relation
    q^{j+1} - q^j = dt L((q^j + q^{j+1})/2) with the oracle's matrix-form
    Lindbladian, to FP64 rounding."""
    if which == "qudits_4x4":
        p = W.config4(n_states=3)
    else:
        p = W.config5(n_states=2)
    s = _sys(p, ckpt_every=10)
    mdl = model.Model(p.system, p.controls)
    rng = np.random.default_rng(7)
    x0 = torch.from_numpy(p.rho0).cuda()
    j = 1234
    x1 = s.propagate(x0, j, j + 1)
    r = _imr_residual(mdl, j, p.rho0, x1.cpu().numpy())
    assert r <= 1e-13 * np.max(np.abs(p.rho0)), r
    lam = rng.standard_normal(p.rho0.shape) * 1e-2 + 0j
    l1 = s.propagate(torch.from_numpy(lam).cuda(), j, j + 1, adjoint=True)
    r = _imr_residual(mdl, j, lam, l1.cpu().numpy(), adjoint=True)
    assert r <= 1e-13 * np.max(np.abs(lam)), r
    # trace preserved by the forward step
    tr0 = np.trace(p.rho0, axis1=1, axis2=2)
    tr1 = np.trace(x1.cpu().numpy(), axis1=1, axis2=2)
    assert np.max(np.abs(tr1 - tr0)) < 1e-13


def test_qudits_4x4_full_size_checkpoints_bitwise():
    """Full-size workload 4 states (N^2 = 65536) over 200 steps at its dt:
    without a forward predictor, checkpoint intervals 1 and 100 give
    bit-identical objective and gradient; with it (restarted every 100
    steps), checkpoints every 100 steps give bitwise the gradient of the full
    stage tape with the same restarts -- the recompute repeats the forward
    sweep exactly -- and the two agree to rounding."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.prefix(W.config4(), 200)
    G1, g1 = _sys(p, ckpt_every=1, predictor=L.LB_PRED_NONE).gradient()
    G2, g2 = _sys(p, ckpt_every=100, predictor=L.LB_PRED_NONE).gradient()
    assert G1 == G2
    assert np.array_equal(g1, g2)
    s = _sys(p, ckpt_every=100)
    G3, g3 = s.gradient()
    st = s.stats()
    G4, g4 = _sys(p, ckpt_every=0, predictor=100).gradient()
    assert G3 == G4
    assert np.array_equal(g3, g4)
    assert abs(G3 - G1) <= 1e-12 * abs(G1)
    assert _rel(g3, g1) < 1e-10
    # predicted first iterates: forward and recompute converge in fewer inner iterations
    s0 = _sys(p, ckpt_every=100, predictor=L.LB_PRED_NONE)
    s0.gradient()
    st0 = s0.stats()
    for ph in (0, 1):
        assert st["phase_iterations"][ph] < st0["phase_iterations"][ph], (ph, st, st0)


# ----------------------------------------------------------------------------
# cluster-split sweeps (one cluster per state, 2Q lanes per element)


@pytest.mark.parametrize("levels,K,herm", [((2,), 7, False), ((2, 3), 0, True), ((2, 2, 2), 100, False),
                                            ((3, 2), 5, True), ((3, 3), 7, False), ((4, 4), 0, True)])
def test_cluster_sweep_matches_oracle(levels, K, herm):
    """The cluster sweep against the oracle (1e-10 / 1e-9) and against the
    one-CTA-per-state sweep.  N^2 4Q <= 1024 runs 4Q lanes per element (one
    per half and component); (4, 4) only fits 2Q lanes."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(601, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, ckpt_every=K,
                         hermitian=herm, objective="trace" if herm else "frob", gamma2=0.05)
    _check_problem(p, sweep=L.LB_SWEEP_CLUSTER)
    Gc, gc = _sys(p, sweep=L.LB_SWEEP_CLUSTER).gradient()
    Gr, gr = _sys(p, sweep=L.LB_SWEEP_RESIDENT).gradient()
    assert abs(Gc - Gr) <= 1e-12 * abs(Gr)
    assert _rel(gc, gr) < 1e-11


def test_cluster_lane_layouts_agree():
    """Forty states of N^2 = 81: 4Q lanes would need 240 SMs, so the sweep
    binds with 2Q lanes; the autotuner times both layouts, and all agree."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(603, levels=(3, 3), n_states=40, n_steps=30, T_ns=0.6, amp=0.1)
    s = _sys(p, sweep=L.LB_SWEEP_CLUSTER)
    G2, g2 = s.gradient()
    q = copy.deepcopy(p)
    q.rho0 = p.rho0[:3]
    q.targets = p.targets[:3]
    s4 = _sys(q, sweep=L.LB_SWEEP_CLUSTER)
    G4, g4 = s4.gradient()
    s2 = _sys(q, sweep=L.LB_SWEEP_RESIDENT)
    Gr, gr = s2.gradient()
    assert abs(G4 - Gr) <= 1e-12 * abs(Gr) and _rel(g4, gr) < 1e-11
    Go, go, _ = imr.gradient(p)
    assert abs(G2 - Go) <= 1e-10 * abs(Go) and _rel(g2, go) < 1e-9
    choice = s.autotune(probe_steps=5)
    G3, g3 = s.gradient()
    assert abs(G3 - Go) <= 1e-10 * abs(Go) and _rel(g3, go) < 1e-9


def test_cluster_steps_and_bitwise_checkpoints():
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(602, levels=(3, 3), n_states=2, n_steps=45, T_ns=0.9, amp=0.1)
    res = [_sys(p, ckpt_every=K, sweep=L.LB_SWEEP_CLUSTER).gradient() for K in (1, 7, 100)]
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    G0, g0 = _sys(p, ckpt_every=0, sweep=L.LB_SWEEP_CLUSTER).gradient()
    assert abs(G0 - res[0][0]) <= 1e-13 * abs(res[0][0])
    assert _rel(g0, res[0][1]) < 1e-12
    s = _sys(p, sweep=L.LB_SWEEP_CLUSTER)
    mdl = model.Model(p.system, p.controls)
    X = _rand_states(np.random.default_rng(3), 2, mdl.N)
    got = s.propagate(torch.from_numpy(X).cuda(), 5, 9).cpu().numpy()
    Q = model.vec(X).T.copy()
    for j in range(5, 9):
        Q, _ = imr.imr_step(mdl, j, Q)
    assert _rel(got, np.stack([model.unvec(Q[:, i], mdl.N) for i in range(2)])) < 1e-13


def test_autotune_keeps_results():
    """The autotuner picks a converging candidate; the gradient after tuning
    still matches the oracle."""
    p = W.random_problem(701, levels=(2, 3), n_states=3, n_steps=40, T_ns=0.8, amp=0.1)
    s = _sys(p)
    choice = s.autotune(probe_steps=10)
    assert choice["sweep"] in ("resident", "cluster", "grid")
    assert choice["solver"] in ("jacobi", "neumann", "gmres")
    G, g = s.gradient()
    Go, go, _ = imr.gradient(p)
    assert abs(G - Go) <= 1e-10 * abs(Go)
    assert _rel(g, go) < 1e-9


# ----------------------------------------------------------------------------
# GMRES inner solve (one CTA per state, Krylov basis in shared memory)


@pytest.mark.parametrize("levels,K,herm", [((2,), 7, False), ((2, 3), 0, True), ((3, 3), 100, False),
                                            ((2, 2, 2, 2), 5, True), ((4, 4, 2), 10, False)])
def test_gmres_matches_oracle(levels, K, herm):
    """GMRES against the oracle (1e-10 / 1e-9) and against Jacobi, for one to
    eight elements per thread ((4, 4, 2): N^2 = 1024)."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(801, levels=levels, n_states=2, n_steps=30, T_ns=0.6, amp=0.1, ckpt_every=K,
                         hermitian=herm, objective="trace" if herm else "frob", gamma2=0.05)
    s, g = _check_problem(p, solver=L.LB_SOLVER_GMRES)
    st = s.stats()
    assert st["solver"] == "gmres" and st["sweep"] == "resident"
    Gj, gj = _sys(p, solver=L.LB_SOLVER_JACOBI, sweep=L.LB_SWEEP_RESIDENT).gradient()
    assert _rel(g, gj) < 1e-11


def _stiff_problem():
    # dt = 0.2 ns with 0.3 GHz amplitudes: the Jacobi iteration matrix has
    # spectral radius above 1 on the later steps, GMRES(20) converges
    return W.random_problem(802, levels=(3, 3), n_states=2, n_steps=10, T_ns=2.0, amp=0.3, ckpt_every=3)


def test_gmres_converges_where_fixed_point_diverges():
    from paper_2110_10310_gb300 import _lib as L

    p = _stiff_problem()
    with pytest.raises(L.LBError) as e:
        _sys(p, solver=L.LB_SOLVER_JACOBI, max_iter=400, sweep=L.LB_SWEEP_RESIDENT).forward()
    assert e.value.code in (L.LB_ENOTCONV, L.LB_ENAN)
    s, _ = _check_problem(p, solver=L.LB_SOLVER_GMRES, max_iter=400)
    st = s.stats()
    assert st["max_iterations"] < 400


def test_gmres_checkpoints_bitwise_and_steps():
    """Deterministic reductions: checkpoint intervals give bit-identical
    gradients; lb_propagate steps match the oracle's dense LU."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(803, levels=(3, 2), n_states=2, n_steps=24, T_ns=0.5, amp=0.1)
    res = [_sys(p, ckpt_every=K, solver=L.LB_SOLVER_GMRES, predictor=L.LB_PRED_NONE).gradient() for K in (1, 5, 100)]
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    p2 = _stiff_problem()
    s = _sys(p2, solver=L.LB_SOLVER_GMRES, max_iter=400)
    mdl = model.Model(p2.system, p2.controls)
    X = _rand_states(np.random.default_rng(4), 2, mdl.N)
    got = s.propagate(torch.from_numpy(X).cuda(), 6, 10).cpu().numpy()
    Q = model.vec(X).T.copy()
    for j in range(6, 10):
        Q, _ = imr.imr_step(mdl, j, Q)
    assert _rel(got, np.stack([model.unvec(Q[:, i], mdl.N) for i in range(2)])) < 1e-12


def test_batch_with_gmres_members():
    """A batch whose members mix GMRES and Jacobi runs the GMRES-capable
    kernels for all of them and matches the per-problem launches."""
    from paper_2110_10310_gb300 import _lib as L
    from paper_2110_10310_gb300.system import LindbladBatch

    shapes = [(2,), (2, 3), (3, 3), (2, 2, 2), (4,), (3, 2)]
    probs = [W.random_problem(810 + i, levels=lv, n_states=2, n_steps=30, T_ns=0.6, amp=0.1)
             for i, lv in enumerate(shapes)]
    systems = [_sys(p, sweep=L.LB_SWEEP_RESIDENT,
                    solver=L.LB_SOLVER_GMRES if i % 2 else L.LB_SOLVER_JACOBI) for i, p in enumerate(probs)]
    plain = [s.gradient() for s in systems]
    Gb, gb = LindbladBatch(systems).gradient()
    off = 0
    for i, (G, g) in enumerate(plain):
        assert abs(Gb[i] - G) <= 1e-12 * abs(G)
        assert _rel(gb[off:off + len(g)], g) < 1e-10
        off += len(g)
    for i in (1, 2):
        Go, go, _ = imr.gradient(probs[i])
        off = sum(len(plain[k][1]) for k in range(i))
        assert abs(Gb[i] - Go) <= 1e-10 * abs(Go)
        assert _rel(gb[off:off + len(go)], go) < 1e-9


# ----------------------------------------------------------------------------
# L-BFGS on top of the gradient (lb_optimize)


def test_lbfgs_trajectory_matches_oracle():
    """lb_optimize against the oracle's L-BFGS driven by the oracle gradient,
    on the Fock-superposition problem at 1000 steps: the same accepted
    iterates (G to 1e-9, alpha to 1e-7) and the same number of evaluations."""
    from oracle import lbfgs

    p = W.fock_superposition(n_steps=1000)
    s = _sys(p)
    res = s.optimize(max_iter=8, memory=5, gtol=0.0, step0=1e-2)

    def fg(x):
        q = copy.deepcopy(p)
        q.controls.alpha = np.array(x)
        G, g, _ = imr.gradient(q)
        return G, g

    x, f, hist = lbfgs.minimize(fg, p.controls.alpha, memory=5, max_iter=8, gtol=0.0, step0=1e-2)
    assert res["iterations"] == len(hist) - 1 == 8
    assert res["evaluations"] == hist.evals
    Gh = np.array([h[0] for h in hist])
    assert np.max(np.abs(res["history"][:, 0] - Gh) / Gh) < 1e-9
    assert _rel(res["alpha"], x) < 1e-7
    assert all(res["history"][k + 1, 0] <= res["history"][k, 0] for k in range(8))
    # the final iterate stays set: a plain gradient call reproduces the final G
    G, _ = s.gradient()
    assert G == res["G"]


def test_autotune_picks_gmres_when_the_fixed_points_diverge():
    """On the stiff problem only GMRES converges: the autotuner keeps it, and
    the gradient after tuning matches the oracle."""
    p = _stiff_problem()
    s = _sys(p, max_iter=400)
    choice = s.autotune(probe_steps=10)
    assert choice["solver"] == "gmres" and choice["sweep"] == "resident"
    G, g = s.gradient()
    Go, go, _ = imr.gradient(p)
    assert abs(G - Go) <= 1e-10 * abs(Go)
    assert _rel(g, go) < 1e-9


@pytest.mark.parametrize("objective", ["frob", "trace"])
def test_three_state_gate_objective_matches_oracle(objective):
    """The CNOT workload with the three-state gate objective (Sec. III-C:
    weights 20, 1, 1, purity-scaled for J_Tr) over its full 10000 steps."""
    p = W.cnot_three_states(objective=objective)
    _check_problem(p)


# ----------------------------------------------------------------------------
# Hermitian symmetry of the grid sweeps


@pytest.mark.parametrize("levels,K,objective", [((3, 2, 2), 0, "frob"), ((3, 3), 7, "trace"), ((2, 2, 2), 100, "frob")])
def test_grid_hermitian_symmetry_matches_oracle(levels, K, objective):
    """Hermitian states and targets on the grid sweep: the half-element
    iteration agrees with the full one (1e-12) and with the oracle."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(901, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, ckpt_every=K,
                         hermitian=True, objective=objective, gamma2=0.05)
    s_h, g_h = _check_problem(p, sweep=L.LB_SWEEP_GRID)
    G_h = s_h.gradient()[0]
    assert s_h.stats()["symmetry"] == "hermitian"
    s_f = _sys(p, sweep=L.LB_SWEEP_GRID, symmetry=L.LB_SYM_NONE)
    G_f, g_f = s_f.gradient()
    assert s_f.stats()["symmetry"] == "none"
    assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
    assert _rel(g_h, g_f) < 1e-11


def test_grid_hermitian_symmetry_with_gate_targets():
    """The three Hermitian gate states (targets V rho V^+ formed on the
    device) on the grid sweep, against the oracle."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.cnot_three_states(n_steps=200)
    p.system.T_ns = 200.0 * 200 / 10000
    s_h, _ = _check_problem(p, sweep=L.LB_SWEEP_GRID)
    assert s_h.stats()["symmetry"] == "hermitian"
    G_h, g_h = s_h.gradient()
    G_f, g_f = _sys(p, sweep=L.LB_SWEEP_GRID, symmetry=L.LB_SYM_NONE).gradient()
    assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
    assert _rel(g_h, g_f) < 1e-11


# ----------------------------------------------------------------------------
# J_Nm from the ensemble state (ground-state reset)


@pytest.mark.parametrize("levels,sweep", [((2, 2, 3), "auto"), ((2, 3), "cluster"), ((2, 2, 3), "grid")])
def test_reset_from_ensemble_state_matches_oracle(levels, sweep):
    """J_N0 of the qubit-qubit-cavity reset (reduced cavity) from the single
    ensemble state, on each sweep kind, against the oracle."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"auto": L.LB_SWEEP_AUTO, "cluster": L.LB_SWEEP_CLUSTER, "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.reset_ensemble(levels=levels, n_steps=400, T_ns=20.0, n_splines=8, amp=0.05)
    _check_problem(p, sweep=sw)


# ----------------------------------------------------------------------------
# Jaynes-Cummings coupling


@pytest.mark.parametrize("levels", [(2, 3), (2, 2, 2), (3, 2, 4)])
def test_apply_with_jaynes_cummings_matches_dense(levels):
    """y = M x and M^+ x with time-dependent Jaynes-Cummings pairs against
    the dense Kronecker M."""
    p = W.random_problem(111, levels=levels, n_states=1, n_steps=10, jc=0.05)
    s = _sys(p)
    m = model.Model(p.system, p.controls)
    N = m.N
    X = _rand_states(np.random.default_rng(9), 2, N)
    xt = torch.from_numpy(X).cuda()
    for j in (0, 6):
        Md = m.M(m.t_half(j))
        for adj in (False, True):
            A = Md.conj().T if adj else Md
            y = s.apply(xt, j, adjoint=adj).cpu().numpy()
            ref = np.stack([model.unvec(A @ model.vec(X[b]), N) for b in range(2)])
            scale = np.max(np.abs(A).sum(axis=1)) * np.max(np.abs(X))
            assert np.max(np.abs(y - ref)) <= 1e-14 * scale, (levels, j, adj)


@pytest.mark.parametrize("levels,sweep,solver", [((2, 3), "resident", "jacobi"), ((3, 2, 2), "grid", "jacobi"),
                                                  ((2, 3), "resident", "gmres"), ((2, 3), "cluster", "jacobi"),
                                                  ((3, 3), "cluster", "neumann")])
def test_jaynes_cummings_gradient_matches_oracle(levels, sweep, solver):
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(112, levels=levels, n_states=2, n_steps=40, T_ns=0.8, amp=0.1, jc=0.05, ckpt_every=7)
    sw = {"resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID, "cluster": L.LB_SWEEP_CLUSTER}[sweep]
    sv = {"jacobi": L.LB_SOLVER_JACOBI, "gmres": L.LB_SOLVER_GMRES, "neumann": L.LB_SOLVER_NEUMANN}[solver]
    s, g = _check_problem(p, sweep=sw, solver=sv)
    assert s.stats()["sweep"] == sweep


def test_jaynes_cummings_on_the_cluster_sweep():
    """A coupled pair adds two halves to the cluster sweep's lane plan: the
    cluster result agrees with the one-CTA sweep (1e-12 / 1e-11) with and
    without checkpoints, AUTO picks the cluster for it, and three pairs on
    three subsystems (six half pairs) are refused."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(113, levels=(2, 3), n_states=3, n_steps=30, T_ns=0.6, amp=0.1, jc=0.05)
    for K in (0, 7):
        Gc, gc = _sys(p, sweep=L.LB_SWEEP_CLUSTER, ckpt_every=K).gradient()
        Gr, gr = _sys(p, sweep=L.LB_SWEEP_RESIDENT, ckpt_every=K).gradient()
        assert abs(Gc - Gr) <= 1e-12 * abs(Gr)
        assert _rel(gc, gr) < 1e-11
    s = _sys(p)
    s.gradient()
    assert s.stats()["sweep"] == "cluster"
    q = W.random_problem(114, levels=(2, 2, 2), n_states=2, n_steps=10, T_ns=0.2, amp=0.1, jc=0.05)
    with pytest.raises(L.LBError):
        _sys(q, sweep=L.LB_SWEEP_CLUSTER)


# ----------------------------------------------------------------------------
# running penalty gamma1 int beta(t) J dt


@pytest.mark.parametrize("levels,objective,K,solver", [((2, 3), "frob", 0, "jacobi"), ((3, 3), "trace", 7, "jacobi"),
                                                        ((2, 3), "frob", 5, "gmres")])
def test_running_penalty_matches_oracle(levels, objective, K, solver):
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(121, levels=levels, n_states=2, n_steps=40, T_ns=0.8, amp=0.1, objective=objective,
                         ckpt_every=K, gamma2=0.05)
    p.gamma1, p.penalty_a = 0.6, 0.3
    sv = {"jacobi": L.LB_SOLVER_JACOBI, "gmres": L.LB_SOLVER_GMRES}[solver]
    s, _ = _check_problem(p, solver=sv)
    assert s.stats()["sweep"] == ("resident" if solver == "gmres" else "cluster")
    if solver != "gmres":
        # the one-CTA sweep computes the same penalty
        s_r, _ = _check_problem(p, solver=sv, sweep=L.LB_SWEEP_RESIDENT)
        assert s_r.stats()["sweep"] == "resident"


def test_running_penalty_with_jnm_and_sweep_rules():
    from paper_2110_10310_gb300 import _lib as L

    p = W.reset_ensemble(levels=(2, 3), n_steps=300, T_ns=15.0, n_splines=8, amp=0.05)
    p.gamma1, p.penalty_a = 0.4, 5.0
    for sweep in (L.LB_SWEEP_AUTO, L.LB_SWEEP_CLUSTER, L.LB_SWEEP_RESIDENT, L.LB_SWEEP_GRID):
        _check_problem(p, sweep=sweep)


@pytest.mark.parametrize("levels,objective,K,herm", [((3, 3), "frob", 7, True), ((2, 3), "trace", 0, False),
                                                     ((3, 2, 2), "frob", 100, False)])
def test_running_penalty_on_the_grid_sweep_matches_oracle(levels, objective, K, herm):
    """The grid sweep sums the running penalty's merit per step over blocks
    in a fixed order and adds its adjoint source from q^j rebuilt backwards:
    objective and gradient against the oracle, the same with and without
    checkpoints, and bitwise across checkpoint intervals with the same
    predictor restarts."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(123, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, objective=objective,
                         ckpt_every=K, gamma2=0.05, hermitian=herm)
    p.gamma1, p.penalty_a = 0.6, 0.3
    s, g = _check_problem(p, sweep=L.LB_SWEEP_GRID)
    assert s.stats()["sweep"] == "grid"
    assert s.stats()["symmetry"] == ("hermitian" if herm else "none")
    if K:
        G0, g0 = _sys(p, sweep=L.LB_SWEEP_GRID, ckpt_every=0, predictor=K).gradient()
        G1, g1 = s.gradient()
        assert G0 == G1 and np.array_equal(g0, g1)


def test_running_penalty_cluster_checkpoints_bitwise():
    """With the penalty, the cluster sweep's gradient is still bit-identical
    across checkpoint intervals K >= 1 and agrees with K = 0."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(122, levels=(3, 3), n_states=2, n_steps=45, T_ns=0.9, amp=0.1, gamma2=0.05)
    p.gamma1, p.penalty_a = 0.6, 0.3
    res = [_sys(p, ckpt_every=K, sweep=L.LB_SWEEP_CLUSTER).gradient() for K in (1, 7, 100)]
    for G, g in res[1:]:
        assert G == res[0][0]
        assert np.array_equal(g, res[0][1])
    G0, g0 = _sys(p, ckpt_every=0, sweep=L.LB_SWEEP_CLUSTER).gradient()
    assert abs(G0 - res[0][0]) <= 1e-13 * abs(res[0][0])
    assert _rel(g0, res[0][1]) < 1e-12


# ----------------------------------------------------------------------------
# Hermitian symmetry of the one-CTA sweeps


@pytest.mark.parametrize("levels,K,objective,solver", [
    ((2, 3), 0, "frob", "jacobi"),
    ((3, 3), 7, "trace", "neumann"),
    ((2, 2, 2), 100, "frob", "jacobi"),
    ((4, 3), 5, "trace", "jacobi"),
    ((3, 2, 4), 9, "frob", "jacobi"),
    ((2, 3), 0, "frob", "gmres"),
    ((3, 3), 7, "trace", "gmres"),
    ((3, 2, 2), 9, "frob", "gmres"),
])
def test_resident_hermitian_symmetry_matches_oracle(levels, K, objective, solver):
    """Hermitian states and targets on the one-CTA sweep (fixed points and
    GMRES, whose inner products become real sums over k <= l with weight 2 off
    the diagonal): the half-element iteration agrees with the full one (1e-12)
    and with the oracle."""
    from paper_2110_10310_gb300 import _lib as L

    sv = {"jacobi": L.LB_SOLVER_JACOBI, "neumann": L.LB_SOLVER_NEUMANN, "gmres": L.LB_SOLVER_GMRES}[solver]
    p = W.random_problem(905, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, ckpt_every=K,
                         hermitian=True, objective=objective, gamma2=0.05)
    s_h, g_h = _check_problem(p, sweep=L.LB_SWEEP_RESIDENT, solver=sv)
    assert s_h.stats()["symmetry"] == "hermitian"
    G_h = s_h.gradient()[0]
    s_f = _sys(p, sweep=L.LB_SWEEP_RESIDENT, solver=sv, symmetry=L.LB_SYM_NONE)
    G_f, g_f = s_f.gradient()
    assert s_f.stats()["symmetry"] == "none"
    assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
    assert _rel(g_h, g_f) < 1e-11


def test_resident_hermitian_symmetry_with_gate_targets_penalty_and_coupling():
    """The three Hermitian gate states, a running penalty and
    Jaynes-Cummings pairs on the one-CTA sweep, each against the oracle and
    the full-element iteration."""
    from paper_2110_10310_gb300 import _lib as L

    p1 = W.cnot_three_states(n_steps=200)
    p1.system.T_ns = 200.0 * 200 / 10000
    p2 = W.random_problem(906, levels=(2, 3), n_states=2, n_steps=40, T_ns=0.8, amp=0.1, hermitian=True,
                          gamma2=0.05, ckpt_every=6)
    p2.gamma1, p2.penalty_a = 0.6, 0.3
    p3 = W.random_problem(907, levels=(3, 2, 2), n_states=2, n_steps=40, T_ns=0.8, amp=0.1, hermitian=True,
                          jc=0.05, ckpt_every=7)
    for p in (p1, p2, p3):
        s_h, g_h = _check_problem(p, sweep=L.LB_SWEEP_RESIDENT)
        assert s_h.stats()["symmetry"] == "hermitian"
        G_h = s_h.gradient()[0]
        G_f, g_f = _sys(p, sweep=L.LB_SWEEP_RESIDENT, symmetry=L.LB_SYM_NONE).gradient()
        assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
        assert _rel(g_h, g_f) < 1e-11


@pytest.mark.parametrize("levels,K,objective,penalty,coupled", [
    ((2, 3), 0, "frob", False, False), ((3, 3), 7, "trace", False, False), ((2, 2, 2), 10, "frob", True, False),
    ((2, 3), 5, "frob", False, True)])
def test_cluster_hermitian_symmetry_matches_oracle(levels, K, objective, penalty, coupled):
    """Hermitian states and targets on the cluster sweep: the lanes take the
    elements k <= l and push each value to its mirror as well; oracle parity,
    and agreement with the full-element cluster sweep (1e-12 / 1e-11), with
    checkpoints, the running penalty and a Jaynes-Cummings pair."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(921, levels=levels, n_states=3, n_steps=40, T_ns=0.8, amp=0.1, ckpt_every=K,
                         hermitian=True, objective=objective, gamma2=0.05, jc=0.05 if coupled else 0.0)
    if penalty:
        p.gamma1, p.penalty_a = 0.2, 5.0
    s_h, g_h = _check_problem(p, sweep=L.LB_SWEEP_CLUSTER, symmetry=L.LB_SYM_HERMITIAN)
    st = s_h.stats()
    assert st["sweep"] == "cluster" and st["symmetry"] == "hermitian"
    G_h = s_h.gradient()[0]
    s_f = _sys(p, sweep=L.LB_SWEEP_CLUSTER, symmetry=L.LB_SYM_NONE)
    G_f, g_f = s_f.gradient()
    assert s_f.stats()["symmetry"] == "none"
    assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
    assert _rel(g_h, g_f) < 1e-11


def test_cluster_hermitian_symmetry_three_gate_states():
    """The three Hermitian gate states (workload cnot_3states) on the cluster
    sweep with the symmetry, against the oracle and the full-element sweep."""
    from paper_2110_10310_gb300 import _lib as L

    p = W.cnot_three_states(n_steps=200)
    p.system.T_ns = 200.0 * 200 / 10000
    s_h, g_h = _check_problem(p, sweep=L.LB_SWEEP_CLUSTER, symmetry=L.LB_SYM_HERMITIAN)
    assert s_h.stats()["symmetry"] == "hermitian"
    G_h = s_h.gradient()[0]
    # LB_SYM_AUTO (the default) leaves the cluster sweep on every element
    s_a = _sys(p, sweep=L.LB_SWEEP_CLUSTER)
    s_a.gradient()
    assert s_a.stats()["symmetry"] == "none"
    G_f, g_f = _sys(p, sweep=L.LB_SWEEP_CLUSTER, symmetry=L.LB_SYM_NONE).gradient()
    assert abs(G_h - G_f) <= 1e-12 * abs(G_f)
    assert _rel(g_h, g_f) < 1e-11


def test_resident_hermitian_symmetry_not_taken_for_general_states():
    from paper_2110_10310_gb300 import _lib as L

    p = W.random_problem(908, levels=(2, 3), n_states=2, n_steps=20, T_ns=0.4, amp=0.1, hermitian=True)
    s = _sys(p, sweep=L.LB_SWEEP_RESIDENT, solver=L.LB_SOLVER_GMRES)
    s.gradient()
    assert s.stats()["symmetry"] == "hermitian"
    q = W.random_problem(909, levels=(2, 3), n_states=2, n_steps=20, T_ns=0.4, amp=0.1, hermitian=False)
    s = _sys(q, sweep=L.LB_SWEEP_RESIDENT)
    s.gradient()
    assert s.stats()["symmetry"] == "none"


# ----------------------------------------------------------------------------
# horizons of one and two steps on every sweep kind


@pytest.mark.parametrize("n_steps,K", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 2)])
@pytest.mark.parametrize("sweep", ["cluster", "resident", "grid"])
def test_short_horizons_match_oracle(n_steps, K, sweep):
    """The first and last steps of a sweep are special (no predictor history,
    no next step to prepare, segment boundaries): horizons of one to three
    steps against the oracle on each sweep kind."""
    from paper_2110_10310_gb300 import _lib as L

    sw = {"cluster": L.LB_SWEEP_CLUSTER, "resident": L.LB_SWEEP_RESIDENT, "grid": L.LB_SWEEP_GRID}[sweep]
    p = W.random_problem(950 + n_steps, levels=(2, 3), n_states=2, n_steps=n_steps, T_ns=0.02 * n_steps, amp=0.1,
                         ckpt_every=K, gamma2=0.05)
    _check_problem(p, sweep=sw)
