"""Pins of the oracle's L-BFGS (the minimisation of G(alpha) by L-BFGS
updates, Sec. III; two-loop recursion of Nocedal & Wright, Algorithm 7.4)
against closed forms: the minimiser of a convex quadratic is A^-1 b, the
Rosenbrock function's is (1, 1); and against planted mistakes."""

import numpy as np
import pytest

from oracle import lbfgs


def _quadratic(n=12, seed=3, cond=100.0):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Qm @ np.diag(np.geomspace(1.0, cond, n)) @ Qm.T
    b = rng.standard_normal(n)
    return A, b, lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)


def _rosenbrock(x):
    f = (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2
    g = np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
    return f, g


def test_quadratic_minimiser_is_the_linear_solve():
    A, b, fg = _quadratic()
    x, f, hist = lbfgs.minimize(fg, np.zeros(len(b)), memory=5, max_iter=200, gtol=1e-11, step0=1.0)
    xs = np.linalg.solve(A, b)
    # the sufficient-decrease test compares values of f, which resolve x only
    # to about sqrt(machine epsilon) near the minimum
    assert np.max(np.abs(x - xs)) <= 1e-7 * np.max(np.abs(xs))
    assert abs(f - (-0.5 * b @ xs)) <= 1e-13 * abs(b @ xs)
    fs = [h[0] for h in hist]
    assert all(fs[k + 1] <= fs[k] for k in range(len(fs) - 1))


def test_rosenbrock_minimiser():
    x, f, hist = lbfgs.minimize(_rosenbrock, np.array([-1.2, 1.0]), memory=6, max_iter=500, gtol=1e-10,
                                step0=0.1)
    assert np.max(np.abs(x - 1.0)) < 1e-7
    assert f < 1e-14
    assert hist[-1][1] <= 1e-10


def test_first_step_and_armijo_rule():
    """The first trial point is x - step0 g/||g||_inf; on a quadratic whose
    first trial overshoots, the step is halved until the Armijo condition
    holds."""
    A = np.diag([1.0, 100.0])
    b = np.zeros(2)
    seen = []

    def fg(x):
        seen.append(x.copy())
        return 0.5 * x @ A @ x - b @ x, A @ x - b

    x0 = np.array([1.0, 1.0])
    lbfgs.minimize(fg, x0, memory=3, max_iter=1, gtol=0.0, step0=1.0)
    g0 = A @ x0
    d = -g0 / np.max(np.abs(g0))
    assert np.allclose(seen[1], x0 + d, rtol=0, atol=1e-15)
    f0 = 0.5 * x0 @ A @ x0
    t = 1.0
    k = 1
    while 0.5 * (x0 + t * d) @ A @ (x0 + t * d) > f0 + lbfgs.C1 * t * (g0 @ d):
        t *= 0.5
        k += 1
        assert np.allclose(seen[k], x0 + t * d, rtol=0, atol=1e-15)
    assert len(seen) == k + 1


def test_two_loop_equals_explicit_inverse_hessian_update():
    """The two-loop recursion applies H_k = V^T H_{k-1} V + rho s s^T
    (V = I - rho y s^T, rho = 1/y^T s) over the stored pairs, oldest first,
    from H^0 = (s^T y / y^T y) I of the newest pair: compare with that
    product of explicit matrices."""
    rng = np.random.default_rng(11)
    n = 7
    A = np.diag(np.geomspace(1.0, 30.0, n))
    S = [rng.standard_normal(n) for _ in range(3)]
    Y = [A @ s + 0.1 * rng.standard_normal(n) for s in S]
    assert all(s @ y > 0 for s, y in zip(S, Y))
    g = rng.standard_normal(n)
    H = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]) * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        Vm = np.eye(n) - rho * np.outer(y, s)
        H = Vm.T @ H @ Vm + rho * np.outer(s, s)
    d = lbfgs._direction(g, S, Y, 1.0)
    assert np.max(np.abs(d - (-H @ g))) <= 1e-12 * np.max(np.abs(H @ g))


def _broken_direction(kind):
    orig = lbfgs._direction

    def f(g, S, Y, step0):
        if not S:
            return orig(g, S, Y, step0)
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(S), reversed(Y)):
            rho = 1.0 / float(np.dot(y, s))
            a = rho * float(np.dot(s, q))
            q = q - a * y
            alphas.append((rho, a))
        s, y = S[-1], Y[-1]
        gamma = float(np.dot(s, y)) / float(np.dot(y, y))
        if kind == "gamma":
            gamma = 1.0
        r = gamma * q
        pairs = list(zip(zip(S, Y), reversed(alphas)))
        if kind == "order":
            pairs = list(zip(zip(S, Y), alphas))
        for (s, y), (rho, a) in pairs:
            b = rho * float(np.dot(y, r))
            r = r + ((b - a) if kind == "sign" else (a - b)) * s
        return -r

    return f


@pytest.mark.parametrize("kind", ["sign", "order", "gamma"])
def test_planted_mistakes_are_caught(monkeypatch, kind):
    monkeypatch.setattr(lbfgs, "_direction", _broken_direction(kind))
    caught = False
    for t in (test_quadratic_minimiser_is_the_linear_solve, test_rosenbrock_minimiser,
              test_two_loop_equals_explicit_inverse_hessian_update):
        try:
            t()
        except AssertionError:
            caught = True
    assert caught, kind
