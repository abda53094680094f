"""L-BFGS minimisation of the objective over the control vector alpha.

Test infrastructure only (see ``oracle/__init__.py``).  The paper optimises
G(alpha) with L-BFGS updates (Sec. III, Appendix B), citing Nocedal & Wright,
Numerical Optimization: the search direction is -H_k g_k with the inverse
Hessian approximation H_k applied by the two-loop recursion over the last m
pairs s_i = x_{i+1} - x_i, y_i = g_{i+1} - g_i (their Algorithm 7.4), with
H_k^0 = gamma_k I, gamma_k = s^T y / y^T y of the newest pair.  The paper
names no line search or first step; the reading used here (and by the
library's ``lb_optimize``):

* first direction (no pair stored yet): -g scaled so that its largest
  component is ``step0``;
* backtracking from the unit step along d, halving until the sufficient
  decrease (Armijo) condition f(x + t d) <= f(x) + c1 t g^T d holds,
  c1 = 1e-4, at most ``max_ls`` trials (then the run stops at x);
* a pair is stored only when s^T y > 1e-10 ||s|| ||y|| (keeps H_k positive
  definite); if d is not a descent direction the pairs are dropped and the
  first-direction rule is used;
* stop when ||g||_inf <= gtol or after ``max_iter`` accepted steps.

Everything is plain NumPy in FP64, with sums taken by ``numpy.dot``.
"""

from __future__ import annotations

import numpy as np

C1 = 1e-4
CURV = 1e-10


def minimize(fg, x0, *, memory: int = 10, max_iter: int = 50, gtol: float = 1e-8, step0: float = 1e-2,
             max_ls: int = 30):
    """Minimise f by L-BFGS.  ``fg(x) -> (f, g)``.  Returns (x, f, history)
    with history a list of (f, ||g||_inf) per accepted iterate, the start
    included, and the number of f evaluations in ``history.evals``."""
    x = np.array(x0, dtype=np.float64)
    f, g = fg(x)
    g = np.asarray(g, dtype=np.float64)
    hist = [(float(f), float(np.max(np.abs(g))))]
    S, Y = [], []
    evals = 1
    for _ in range(max_iter):
        gmax = float(np.max(np.abs(g)))
        if gmax <= gtol:
            break
        d = _direction(g, S, Y, step0)
        gd = float(np.dot(g, d))
        if not gd < 0.0:
            S, Y = [], []
            d = _direction(g, S, Y, step0)
            gd = float(np.dot(g, d))
        t = 1.0
        accepted = False
        for _ls in range(max_ls):
            xn = x + t * d
            fn, gn = fg(xn)
            gn = np.asarray(gn, dtype=np.float64)
            evals += 1
            if fn <= f + C1 * t * gd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        s = xn - x
        y = gn - g
        sy = float(np.dot(s, y))
        if sy > CURV * float(np.linalg.norm(s)) * float(np.linalg.norm(y)):
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, float(fn), gn
        hist.append((f, float(np.max(np.abs(g)))))
    out = History(hist)
    out.evals = evals
    return x, f, out


class History(list):
    evals = 0


def _direction(g, S, Y, step0):
    """-H g by the two-loop recursion (newest pair first, then oldest first)."""
    if not S:
        return -g * (step0 / float(np.max(np.abs(g))))
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(np.dot(y, s))
        a = rho * float(np.dot(s, q))
        q = q - a * y
        alphas.append((rho, a))
    s, y = S[-1], Y[-1]
    r = (float(np.dot(s, y)) / float(np.dot(y, y))) * q
    for (s, y), (rho, a) in zip(zip(S, Y), reversed(alphas)):
        b = rho * float(np.dot(y, r))
        r = r + (a - b) * s
    return -r
