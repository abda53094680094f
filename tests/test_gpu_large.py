"""The two large workloads against the oracle at the shapes the dense
oracle can reach (its results stored by tests/golden/make_oracle_references.py,
which calls only the oracle), on the grid-wide sweep that runs them at full
size, with checkpoint segments crossed; and their full-size gradients against
central differences of the GPU objective.

Tolerances (the method's accuracy targets): states and objective 1e-10
relative, gradient 1e-9 relative to the oracle's adjoint gradient, 1e-6 to
central differences."""

import importlib.util
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("oracle_refs", os.path.join(HERE, "golden", "make_oracle_references.py"))
refs = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(refs)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10310_gb300 import _lib as L

    L.load(build_if_missing=True)


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run(p, **kw):
    from paper_2110_10310_gb300.system import LindbladSystem

    s = LindbladSystem(p, **kw)
    G, rhoT = s.forward(want_states=True)
    Gg, g = s.gradient()
    return s, G, Gg, g, rhoT.cpu().numpy()


def _check(name, p, **kw):
    Go, go, rho_o = refs.load(name)
    s, G, Gg, g, rhoT = _run(p, **kw)
    st = s.stats()
    assert st["sweep"] == "grid"
    assert abs(G - Go) <= 1e-10 * abs(Go), (G, Go)
    assert abs(Gg - Go) <= 1e-10 * abs(Go), (Gg, Go)
    assert _rel(rhoT, rho_o) < 1e-10
    assert _rel(g, go) < 1e-9, _rel(g, go)
    return s, st


@pytest.mark.slow
def test_qudits_4x2_full_horizon_matches_oracle():
    """The four-qudit workload's structure at 2 levels per qudit (vec 256):
    all 40000 steps of its 500 ns horizon with checkpoints every 100 steps
    (400 segments recomputed), states, objective and gradient against the
    oracle's dense LU steps."""
    from paper_2110_10310_gb300 import _lib as L

    p = refs.qudits_4x2_full()
    assert p.ckpt_every == 100 and p.system.n_steps == 40000
    _, st = _check("qudits_4x2_full", p, sweep=L.LB_SWEEP_GRID)
    assert st["ckpt_every"] == 100
    assert st["phase_steps"] == [3 * 40000] * 3


def test_qudits_4x3_prefix_matches_oracle():
    """The four-qudit workload's structure at 3 levels per qudit (vec 6561,
    the grid sweep by size) over its first 24 steps, checkpoints every 10:
    two segment boundaries crossed by the recompute."""
    p = refs.qudits_4x3_prefix()
    _, st = _check("qudits_4x3_prefix", p, ckpt_every=10)
    assert st["ckpt_every"] == 10


def test_qutrits_6x2_prefix_matches_oracle():
    """The six-qutrit workload's structure at 2 levels per subsystem (vec 4096,
    4 states: the grid sweep) over its first 24 steps, checkpoints every 10."""
    p = refs.qutrits_6x2_prefix()
    _, st = _check("qutrits_6x2_prefix", p, ckpt_every=10)
    assert st["ckpt_every"] == 10


@pytest.mark.slow
def test_qudits_4x4_gradient_against_gpu_central_differences():
    """4 x 4-level qudits at full size (vec 65536, 3 states) over the first 400
    steps at the workload's dt, checkpoints every 100: the adjoint gradient
    against central differences of the GPU objective on 16 coefficients
    spread over every subsystem, carrier, spline and real/imaginary part."""
    from paper_2110_10310_gb300.system import LindbladSystem

    p = W.prefix(W.config4(), 400)
    s = LindbladSystem(p)
    G, g = s.gradient()
    a0 = p.controls.alpha.copy()
    eps = 1e-5
    scale = np.max(np.abs(g))
    idx = np.linspace(0, len(a0) - 1, 16).round().astype(int)
    assert len(set(idx.tolist())) == 16
    for k in idx:
        a = a0.copy()
        a[k] += eps
        s.set_alpha(a)
        gp = s.forward()
        a[k] -= 2 * eps
        s.set_alpha(a)
        gm = s.forward()
        assert abs((gp - gm) / (2 * eps) - g[k]) <= 1e-6 * scale, (k, (gp - gm) / (2 * eps), g[k])
    s.set_alpha(a0)


@pytest.mark.slow
def test_qutrits_6x3_full_size_gradient_against_gpu_central_differences():
    """6 qutrits at full size (vec 531441, 2 states) over the first 20 steps,
    checkpoints every 10: the adjoint gradient against central differences of
    the GPU objective on 6 coefficients, one per subsystem."""
    from paper_2110_10310_gb300.system import LindbladSystem

    p = W.prefix(W.config5(n_states=2), 20)
    p.ckpt_every = 10
    s = LindbladSystem(p)
    G, g = s.gradient()
    assert s.stats()["sweep"] == "grid"
    a0 = p.controls.alpha.copy()
    eps = 1e-5
    scale = np.max(np.abs(g))
    per = len(a0) // 6
    for k in [q * per + 3 for q in range(6)]:
        a = a0.copy()
        a[k] += eps
        s.set_alpha(a)
        gp = s.forward()
        a[k] -= 2 * eps
        s.set_alpha(a)
        gm = s.forward()
        assert abs((gp - gm) / (2 * eps) - g[k]) <= 1e-6 * scale, (k, (gp - gm) / (2 * eps), g[k])
    s.set_alpha(a0)
