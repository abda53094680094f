"""Seeded generators for the workloads of the Lindblad implicit-midpoint path.

Everything here is input data: numbers drawn from ``numpy.random.Generator``
(PCG64, seed = workload number unless stated) and arranged into arrays.  The
physics conventions the numbers are read under (units, signs, ordering) are
stated once, here, and both consumers follow them:

* frequencies are ``value / 2pi`` in GHz, times in ns, T1/T2 in microseconds;
* ``selfkerr_ghz[q]`` is xi_q/2pi of the term -xi_q/2 a^dag a^dag a a (Sec. II,
  H_sys); a transmon anharmonicity of -0.2 GHz is ``selfkerr_ghz = +0.2``;
* ``crosskerr_ghz[p, q]`` for p < q is xi_pq/2pi of the term -xi_pq n_p n_q;
* ``t1_us`` / ``t2_us`` equal to ``inf`` switch the collapse operator off;
* subsystem 0 is the most significant digit of a basis index;
* control coefficients ``alpha`` are laid out [q][f][s][re, im] (GHz);
* density matrices are (M, N, N) complex128 arrays, rho[i][k, l] = <k|rho_i|l>.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

INF = float("inf")

# Gate matrices on the essential subspace (computational basis, subsystem 0
# most significant).  CNOT: control = subsystem 0, target = subsystem 1.
XGATE = np.array([[0, 1], [1, 0]], dtype=np.complex128)
CNOT = np.array(
    [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128
)


@dataclass
class SystemSpec:
    levels: tuple
    detuning_ghz: np.ndarray
    selfkerr_ghz: np.ndarray
    crosskerr_ghz: np.ndarray  # (Q, Q); entries p < q used
    t1_us: np.ndarray
    t2_us: np.ndarray
    T_ns: float
    n_steps: int
    essential: Optional[tuple] = None
    jc_ghz: Optional[np.ndarray] = None  # (Q, Q) Jaynes-Cummings couplings g_pq/2pi; entries p < q used
    rot_ghz: Optional[np.ndarray] = None  # (Q,) rotating-frame frequencies omega_q^rot/2pi (for the JC phases)

    @property
    def Q(self) -> int:
        return len(self.levels)

    @property
    def N(self) -> int:
        return int(np.prod(self.levels))


@dataclass
class ControlSpec:
    n_splines: int
    carriers_ghz: list  # list of 1-D float arrays, one per subsystem
    alpha: np.ndarray  # float64, layout [q][f][s][re, im]
    # the B-splines span [0, horizon_ns] (None: the system's final time T); a
    # run over the first steps of a longer horizon keeps that horizon here, so
    # that its controls are the longer problem's
    horizon_ns: float | None = None

    @property
    def n_params(self) -> int:
        return 2 * self.n_splines * sum(len(c) for c in self.carriers_ghz)


@dataclass
class Problem:
    name: str
    system: SystemSpec
    controls: ControlSpec
    rho0: np.ndarray  # (M, N, N) complex128
    objective: str = "frob"  # "frob" | "trace"
    targets: Optional[np.ndarray] = None  # (M, N, N) complex128
    gate: Optional[np.ndarray] = None  # (Ne, Ne) complex128
    weights: Optional[np.ndarray] = None  # (M,) float64, None = all ones
    gamma2: float = 0.0
    ckpt_every: int = -1  # -1: automatic (full stage tape when it fits, else every 100 steps)
    gamma1: float = 0.0  # weight of the running penalty (Sec. III, eq. optimproblem)
    penalty_a: float = 1.0  # width a (ns) of beta(t) = exp(-((t - T)/a)^2)/a
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.rho0.shape[0])


# ----------------------------------------------------------------------------
# small building blocks (index bookkeeping and random draws only)


def _digits(index: int, radices) -> list:
    out = []
    for r in reversed(radices):
        out.append(index % r)
        index //= r
    return out[::-1]


def _index(digits, radices) -> int:
    idx = 0
    for d, r in zip(digits, radices):
        idx = idx * r + d
    return idx


def essential_to_full(i: int, levels, essential) -> int:
    """Full-space basis index of essential-subspace basis index ``i``."""
    ess = essential if essential is not None else levels
    return _index(_digits(i, ess), levels)


def basis_outer(levels, essential, i: int, j: int) -> np.ndarray:
    """|i><j| for essential-basis indices i, j, embedded in the full space."""
    N = int(np.prod(levels))
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[essential_to_full(i, levels, essential), essential_to_full(j, levels, essential)] = 1.0
    return rho


def random_pure_state(rng: np.random.Generator, N: int) -> np.ndarray:
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return g / np.linalg.norm(g)


def pure_density(psi: np.ndarray) -> np.ndarray:
    return np.outer(psi, psi.conj())


def _alpha(rng, Q, n_splines, n_carriers, amp):
    n = 2 * n_splines * sum(n_carriers)
    return rng.uniform(-amp, amp, size=n)


def _all_ij_states(levels, essential):
    ess = essential if essential is not None else levels
    Ne = int(np.prod(ess))
    return np.stack([basis_outer(levels, essential, i, j) for i in range(Ne) for j in range(Ne)])


# ----------------------------------------------------------------------------
# the five workloads


def config1(seed: int = 1, n_steps: int = 1000) -> Problem:
    """1 qubit, T1 = 100 us, T2 = 50 us, T = 100 ns, 10 splines, X gate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sysm = SystemSpec(
        levels=(2,),
        detuning_ghz=np.array([0.0]),
        selfkerr_ghz=np.array([0.0]),
        crosskerr_ghz=np.zeros((1, 1)),
        t1_us=np.array([100.0]),
        t2_us=np.array([50.0]),
        T_ns=100.0,
        n_steps=n_steps,
    )
    ctrl = ControlSpec(10, [np.array([0.0])], _alpha(rng, 1, 10, [1], 0.01))
    return Problem("qubit_x_gate", sysm, ctrl, _all_ij_states((2,), None), "frob", gate=XGATE.copy())


def config2(seed: int = 2, n_steps: int = 10000, levels=(3, 3)) -> Problem:
    """2 transmons x 3 levels, CNOT on the 2-level essential subspace."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xi12 = 0.01
    ck = np.zeros((2, 2))
    ck[0, 1] = xi12
    sysm = SystemSpec(
        levels=tuple(levels),
        detuning_ghz=np.array([0.0, -0.1]),
        selfkerr_ghz=np.array([0.2, 0.2]),
        crosskerr_ghz=ck,
        t1_us=np.array([56.0, 56.0]),
        t2_us=np.array([28.0, 28.0]),
        T_ns=200.0,
        n_steps=n_steps,
        essential=(2, 2),
    )
    carriers = [np.array([0.0, -xi12]), np.array([0.0, -xi12])]
    ctrl = ControlSpec(20, carriers, _alpha(rng, 2, 20, [2, 2], 0.01))
    rho0 = _all_ij_states(sysm.levels, sysm.essential)
    return Problem("cnot_2x3", sysm, ctrl, rho0, "frob", gate=CNOT.copy())


def basis_matrices(N: int) -> np.ndarray:
    """The N^2 pure basis states B^{kj} of Sec. III-B: 1/2 (|k><k| + |j><j|)
    plus 1/2 (|k><j| + |j><k|) for k < j, or i/2 (|j><k| - |k><j|) for k > j
    (the printed k > j case is garbled; read as the pure state
    (|k> + i|j>)/sqrt 2)."""
    B = np.zeros((N, N, N, N), dtype=np.complex128)
    for k in range(N):
        for j in range(N):
            B[k, j, k, k] += 0.5
            B[k, j, j, j] += 0.5
            if k < j:
                B[k, j, k, j] += 0.5
                B[k, j, j, k] += 0.5
            elif k > j:
                B[k, j, j, k] += 0.5j
                B[k, j, k, j] -= 0.5j
    return B


def ensemble_state(N: int) -> np.ndarray:
    """rho_s = 1/N^2 sum_kj B^{kj} (Sec. III-B), one state spanning all
    initial states for a linear merit functional."""
    return basis_matrices(N).sum(axis=(0, 1)) / (N * N)


def reset_ensemble(levels=(2, 2, 20), n_steps: int = 100000, T_ns: float = 5000.0, seed: int = 7,
                   n_splines: int = 100, amp: float = 0.01) -> Problem:
    """Ground-state reset of two qubits and a readout cavity from the ensemble
    state, J_N0 (Sec. III-B and its footnote: rotating frames at the qubit
    and cavity frequencies, anharmonicities 230.56, 251.0, 0 MHz, cross-Kerr
    0.001, 1.176, 1.2 MHz for the pairs (1,2), (1,3), (2,3), T1 = 80, 90,
    0.3892 us, T2 = 26, 30 us and none for the cavity, 100 splines, carriers
    0, T = 5 us).  The step count is not printed; dt = 0.05 ns is the
    reading.  Controls start uniform in [-amp, amp] GHz."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = len(levels)
    ck = np.zeros((Q, Q))
    for (a, c), v in {(0, 1): 1e-6, (0, 2): 1.176e-3, (1, 2): 1.2e-3}.items():
        if c < Q:
            ck[a, c] = v
    sysm = SystemSpec(
        levels=tuple(levels),
        detuning_ghz=np.zeros(Q),
        selfkerr_ghz=np.array([0.23056, 0.251, 0.0])[:Q],
        crosskerr_ghz=ck,
        t1_us=np.array([80.0, 90.0, 0.3892])[:Q],
        t2_us=np.array([26.0, 30.0, 0.0])[:Q],
        T_ns=T_ns,
        n_steps=n_steps,
    )
    ctrl = ControlSpec(n_splines, [np.array([0.0]) for _ in range(Q)], _alpha(rng, Q, n_splines, [1] * Q, amp))
    N = int(np.prod(levels))
    rho0 = ensemble_state(N)[None].copy()
    return Problem("reset_ensemble", sysm, ctrl, rho0, "nm", meta={"m": 0})


def three_gate_states(levels, essential=None) -> np.ndarray:
    """The three initial states that distinguish any two unitaries on the
    essential subspace (Sec. III-C), embedded in the full space:
    rho_1 = sum_j lambda_j |j><j| with distinct lambda_j = 2 (Ne - j) / (Ne (Ne + 1)),
    rho_2 = |psi><psi| with psi the uniform superposition, rho_3 = I / Ne."""
    ess = essential if essential is not None else levels
    Ne = int(np.prod(ess))
    N = int(np.prod(levels))
    idx = [essential_to_full(i, levels, essential) for i in range(Ne)]
    rho = np.zeros((3, N, N), dtype=np.complex128)
    for j, k in enumerate(idx):
        rho[0, k, k] = 2.0 * (Ne - j) / (Ne * (Ne + 1))
        rho[2, k, k] = 1.0 / Ne
    for a in idx:
        for c in idx:
            rho[1, a, c] = 1.0 / Ne
    return rho


def cnot_three_states(n_steps: int = 10000, objective: str = "frob") -> Problem:
    """The CNOT workload of ``config2`` with the three-state gate objective
    (Sec. III-C): the states of ``three_gate_states``, weights
    beta = (20, 1, 1), and for J_Tr each weight scaled by the purity
    Tr(rho_i(0)^2) of its state."""
    p = config2(n_steps=n_steps)
    p.name = "cnot_three_states"
    p.rho0 = three_gate_states(p.system.levels, p.system.essential)
    w = np.array([20.0, 1.0, 1.0])
    if objective == "trace":
        w = w * np.array([np.real(np.trace(r @ r)) for r in p.rho0])
    p.weights = w
    p.objective = objective
    return p


def _random_problem_config3(rng, idx, n_steps):
    Q = int(rng.integers(1, 4))
    levels = tuple(int(x) for x in rng.integers(2, 5, size=Q))
    N = int(np.prod(levels))
    ck = np.zeros((Q, Q))
    for p in range(Q):
        for q in range(p + 1, Q):
            ck[p, q] = rng.uniform(0.0, 0.01)
    t1 = rng.uniform(20.0, 100.0, size=Q)
    sysm = SystemSpec(
        levels=levels,
        detuning_ghz=rng.uniform(-0.2, 0.2, size=Q),
        selfkerr_ghz=-rng.uniform(-0.25, -0.15, size=Q),
        crosskerr_ghz=ck,
        t1_us=t1,
        t2_us=t1 / 2.0,
        T_ns=100.0,
        n_steps=n_steps,
    )
    ctrl = ControlSpec(10, [np.array([0.0]) for _ in range(Q)], _alpha(rng, Q, 10, [1] * Q, 0.01))
    rho0 = np.stack([pure_density(random_pure_state(rng, N)) for _ in range(3)])
    tar = pure_density(random_pure_state(rng, N))
    targets = np.stack([tar] * 3)
    return Problem(f"batch_{idx:03d}", sysm, ctrl, rho0, "frob", targets=targets)


def config3(seed: int = 3, n_problems: int = 256, n_steps: int = 5000) -> list:
    """256 independent problems of uneven size (Q in {1,2,3}, levels in {2,3,4})."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [_random_problem_config3(rng, i, n_steps) for i in range(n_problems)]


def config4(seed: int = 4, n_steps: int = 40000, levels=(4, 4, 4, 4), n_states: int = 3) -> Problem:
    """4 qudits x 4 levels, chain cross-Kerr 0.005 GHz, state preparation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = len(levels)
    N = int(np.prod(levels))
    ck = np.zeros((Q, Q))
    for q in range(Q - 1):
        ck[q, q + 1] = 0.005
    sysm = SystemSpec(
        levels=tuple(levels),
        detuning_ghz=rng.uniform(-0.2, 0.2, size=Q),
        selfkerr_ghz=np.full(Q, 0.2),
        crosskerr_ghz=ck,
        t1_us=np.full(Q, 80.0),
        t2_us=np.full(Q, 40.0),
        T_ns=500.0,
        n_steps=n_steps,
    )
    carriers = [np.array([0.0, -0.005]) for _ in range(Q)]
    ctrl = ControlSpec(30, carriers, _alpha(rng, Q, 30, [2] * Q, 0.01))
    rho0 = np.stack([pure_density(random_pure_state(rng, N)) for _ in range(n_states)])
    tar = pure_density(random_pure_state(rng, N))
    return Problem("qudits_4x4", sysm, ctrl, rho0, "frob", targets=np.stack([tar] * n_states), ckpt_every=100)


def config5(seed: int = 5, n_steps: int = 20000, levels=(3, 3, 3, 3, 3, 3), n_states: int = 64) -> Problem:
    """6 qutrits, ring cross-Kerr 0.003 GHz, 64 random pure initial states."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = len(levels)
    N = int(np.prod(levels))
    ck = np.zeros((Q, Q))
    for q in range(Q):
        p, r = sorted((q, (q + 1) % Q))
        if p != r:
            ck[p, r] = 0.003
    t1 = rng.uniform(40.0, 80.0, size=Q)
    sysm = SystemSpec(
        levels=tuple(levels),
        detuning_ghz=rng.uniform(-0.2, 0.2, size=Q),
        selfkerr_ghz=np.full(Q, 0.2),
        crosskerr_ghz=ck,
        t1_us=t1,
        t2_us=t1 / 2.0,
        T_ns=300.0,
        n_steps=n_steps,
    )
    carriers = [np.array([0.0, -0.003]) for _ in range(Q)]
    ctrl = ControlSpec(40, carriers, _alpha(rng, Q, 40, [2] * Q, 0.01))
    rho0 = np.stack([pure_density(random_pure_state(rng, N)) for _ in range(n_states)])
    tar = pure_density(random_pure_state(rng, N))
    return Problem("qutrits_6x3", sysm, ctrl, rho0, "frob", targets=np.stack([tar] * n_states), ckpt_every=100)


def prefix(prob: Problem, n_steps: int) -> Problem:
    """The first n_steps steps of ``prob`` at its step size: the final time
    becomes n_steps dt and the controls keep their horizon (in place; returns
    ``prob``)."""
    if not prob.controls.horizon_ns:
        prob.controls.horizon_ns = prob.system.T_ns
    prob.system.T_ns = prob.system.T_ns * n_steps / prob.system.n_steps
    prob.system.n_steps = n_steps
    return prob


def config(n: int, **kw):
    return {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}[n](**kw)


# ----------------------------------------------------------------------------
# random small problems for tests


def fock_superposition(seed: int = 6, n_steps: int = 10000, T_ns: float = 200.0, amp: float = 0.01) -> Problem:
    """One 4-level qudit driven from |0><0| towards the Fock superposition
    (|0> + |3>)/sqrt(2): the paper's state-to-state example (Sec. III-A, its
    footnote parameters: rotating frame, anharmonicity 0.23 GHz, T1 = 93.79 us,
    T2 = 102.52 us, 10 splines, carriers {0, -0.23} GHz).  The horizon is read
    as 0.2 us = 200 ns; controls start uniform in [-amp, amp] GHz."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sysm = SystemSpec(
        levels=(4,),
        detuning_ghz=np.array([0.0]),
        selfkerr_ghz=np.array([0.23]),
        crosskerr_ghz=np.zeros((1, 1)),
        t1_us=np.array([93.79]),
        t2_us=np.array([102.52]),
        T_ns=T_ns,
        n_steps=n_steps,
    )
    ctrl = ControlSpec(10, [np.array([0.0, -0.23])], _alpha(rng, 1, 10, [2], amp))
    psi = np.zeros(4, dtype=np.complex128)
    psi[0] = psi[3] = 1.0 / np.sqrt(2.0)
    rho0 = np.zeros((1, 4, 4), dtype=np.complex128)
    rho0[0, 0, 0] = 1.0
    return Problem("fock_superposition", sysm, ctrl, rho0, "frob", targets=pure_density(psi)[None].copy())


def random_problem(
    seed: int,
    levels=(2, 3),
    n_states: int = 2,
    n_steps: int = 20,
    T_ns: float = 4.0,
    n_splines: int = 5,
    n_carriers: int = 2,
    amp: float = 0.3,
    objective: str = "frob",
    hermitian: bool = True,
    dissipation: bool = True,
    gamma2: float = 0.0,
    ckpt_every: int = -1,
    jc: float = 0.0,
) -> Problem:
    """A small driven, dissipative problem with every term of the model active.

    Drive amplitudes are much larger than in the benchmark workloads so that
    the control terms, and their gradients, are far from negligible.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = len(levels)
    N = int(np.prod(levels))
    ck = np.zeros((Q, Q))
    for p in range(Q):
        for q in range(p + 1, Q):
            ck[p, q] = rng.uniform(0.0, 0.05)
    if dissipation:
        t1 = rng.uniform(0.02, 0.2, size=Q)  # strong decay so the terms matter over a few ns
        t2 = rng.uniform(0.02, 0.2, size=Q)
    else:
        t1 = np.full(Q, INF)
        t2 = np.full(Q, INF)
    sysm = SystemSpec(
        levels=tuple(levels),
        detuning_ghz=rng.uniform(-0.3, 0.3, size=Q),
        selfkerr_ghz=rng.uniform(0.1, 0.3, size=Q),
        crosskerr_ghz=ck,
        t1_us=t1,
        t2_us=t2,
        T_ns=T_ns,
        n_steps=n_steps,
    )
    if jc > 0.0:
        # Jaynes-Cummings couplings of every pair and rotating frames (drawn
        # after the system so that jc = 0 keeps the earlier draws unchanged)
        jrng = np.random.Generator(np.random.PCG64(seed + 7919))
        sysm.jc_ghz = np.triu(jrng.uniform(0.2 * jc, jc, size=(Q, Q)), 1)
        sysm.rot_ghz = jrng.uniform(-0.2, 0.2, size=Q)
    carriers = [np.concatenate([[0.0], rng.uniform(-0.3, 0.3, size=n_carriers - 1)]) for _ in range(Q)]
    ctrl = ControlSpec(n_splines, carriers, _alpha(rng, Q, n_splines, [n_carriers] * Q, amp))
    if hermitian:
        rho0 = np.stack([pure_density(random_pure_state(rng, N)) for _ in range(n_states)])
    else:
        rho0 = np.stack(
            [np.outer(random_pure_state(rng, N), random_pure_state(rng, N).conj()) for _ in range(n_states)]
        )
    targets = np.stack([pure_density(random_pure_state(rng, N)) for _ in range(n_states)])
    weights = rng.uniform(0.5, 2.0, size=n_states)
    return Problem(
        f"random_{seed}",
        sysm,
        ctrl,
        rho0,
        objective,
        targets=targets,
        weights=weights,
        gamma2=gamma2,
        ckpt_every=ckpt_every,
    )
