"""The pins catch plausible mistakes: each case plants one mistake in the
oracle (on the CPU, by monkeypatching) and requires that at least one pin of
``test_oracle_pins`` then fails."""

import math

import numpy as np
import pytest

from oracle import imr, model
import tests.test_oracle_pins as pins

PIN_TESTS = [
    pins.test_qubit_t1_decay_and_t2_dephasing_closed_form,
    pins.test_qudit_top_level_decay_and_kerr_phase,
    pins.test_cross_kerr_and_subsystem_order,
    pins.test_cayley_transform_for_constant_generator,
    pins.test_bspline_partition_of_unity_and_shape,
    pins.test_control_amplitude_single_coefficient,
    lambda: pins.test_lindbladian_structure((2, 3)),
    pins.test_lindbladian_matches_textbook_qubit_generator,
    pins.test_closed_system_is_unitary,
    pins.test_trace_and_hermiticity_preserved,
    pins.test_gate_targets_brute_force,
    pins.test_adjoint_dot_product_identity,
    lambda: pins.test_gradient_matches_central_differences("frob", False, 0.0),
    lambda: pins.test_gradient_matches_central_differences("trace", True, 0.3),
    pins.test_jnm_values_and_gradient,
    pins.test_jaynes_cummings_resonant_swap_discrete_closed_form,
    pins.test_jaynes_cummings_detuned_phases_against_schrodinger,
    pins.test_running_penalty_closed_form_and_gradient,
    pins.test_control_horizon_prefix_is_the_longer_problem_truncated,
]


def _some_pin_fails():
    for t in PIN_TESTS:
        try:
            t()
        except AssertionError:
            return True
    return False


def _ham_part_transposed(H):
    N = H.shape[0]
    I = np.eye(N, dtype=np.complex128)
    return -1j * (np.kron(I, H) - np.kron(H, I))


def _ham_part_sign(H):
    N = H.shape[0]
    I = np.eye(N, dtype=np.complex128)
    return 1j * (np.kron(I, H) - np.kron(H.T, I))


def _diss_no_anticomm(Ls, N):
    D = np.zeros((N * N, N * N), dtype=np.complex128)
    for L in Ls:
        D += np.kron(L.conj(), L)
    return D


def _diss_half_jump(Ls, N):
    I = np.eye(N, dtype=np.complex128)
    D = np.zeros((N * N, N * N), dtype=np.complex128)
    for L in Ls:
        LdL = L.conj().T @ L
        D += 0.5 * np.kron(L.conj(), L) - 0.5 * (np.kron(I, LdL) + np.kron(LdL.T, I))
    return D


def _syshamiltonian_kerr_factor(sysm):
    H = ORIG["system_hamiltonian"](sysm)
    levels = sysm.levels
    for q in range(len(levels)):
        a = model.a_op(q, levels)
        ad = a.conj().T
        H -= 2 * math.pi * sysm.selfkerr_ghz[q] / 2.0 * (ad @ ad @ a @ a)  # -xi instead of -xi/2
    return H


def _syshamiltonian_crosskerr_sign(sysm):
    H = ORIG["system_hamiltonian"](sysm)
    levels = sysm.levels
    for p in range(len(levels)):
        for q in range(p + 1, len(levels)):
            n_p = model.a_op(p, levels).conj().T @ model.a_op(p, levels)
            n_q = model.a_op(q, levels).conj().T @ model.a_op(q, levels)
            H += 2 * 2 * math.pi * sysm.crosskerr_ghz[p][q] * (n_p @ n_q)
    return H


def _embed_reversed(op, q, levels):
    out = np.ones((1, 1), dtype=np.complex128)
    for p, n in reversed(list(enumerate(levels))):
        out = np.kron(out, op if p == q else np.eye(n, dtype=np.complex128))
    return out


def _bspline_shifted(s, t, n_splines, T):
    return ORIG["bspline_basis"](s + 1, t, n_splines, T)


def _control_no_2pi(ctrl, t, T):
    return ORIG["control_amplitudes"](ctrl, t, T) / (2 * math.pi)


def _control_conj_carrier(ctrl, t, T):
    Q = len(ctrl.carriers_ghz)
    d = np.zeros(Q, dtype=np.complex128)
    for q in range(Q):
        for f, om in enumerate(ctrl.carriers_ghz[q]):
            carrier = np.exp(-1j * 2 * math.pi * om * t)
            for s in range(ctrl.n_splines):
                S = model.bspline_basis(s, t, ctrl.n_splines, T)
                i = model.alpha_index(ctrl, q, f, s)
                d[q] += 2 * math.pi * S * complex(ctrl.alpha[i], ctrl.alpha[i + 1]) * carrier
    return d


def _imr_step_explicit_half(mdl, j, Qm):
    h = mdl.h
    M = mdl.M(mdl.t_half(j))
    A = np.eye(M.shape[0], dtype=np.complex128) - 0.5 * h * M
    Z = np.linalg.solve(A, Qm)
    return Qm + 0.5 * h * (M @ Z), Z


def _imr_step_wrong_time(mdl, j, Qm):
    h = mdl.h
    M = mdl.M(j * h)
    A = np.eye(M.shape[0], dtype=np.complex128) - 0.5 * h * M
    Z = np.linalg.solve(A, Qm)
    return Qm + h * (M @ Z), Z


def _terminal_sign(prob, rhoT):
    return -ORIG["terminal_adjoint"](prob, rhoT)


def _horizon_ignored(ctrl, sysm):
    return float(sysm.T_ns)


def _dd_no_imag_i(ctrl, T, t):
    out = ORIG["dd_dalpha"](ctrl, T, t)
    return [(k, q, (v / 1j if k % 2 == 1 else v)) for k, q, v in out]


ORIG = {
    "system_hamiltonian": model.system_hamiltonian,
    "bspline_basis": model.bspline_basis,
    "control_amplitudes": model.control_amplitudes,
    "terminal_adjoint": imr.terminal_adjoint,
    "dd_dalpha": imr.dd_dalpha,
}

def _merit_nm_transposed_index(kind, tar, rho):
    if kind == "nm":
        # N_m read as diag(|l - m|) with l counted from the other end
        return float(np.real(np.trace(tar[::-1, ::-1] @ rho)))
    return ORIG_MERIT(kind, tar, rho)


def _terminal_nm_negated(prob, rhoT):
    out = ORIG["terminal_adjoint"](prob, rhoT)
    return -out if prob.objective == "nm" else out


ORIG_MERIT = imr.merit
ORIG_JC = model.jc_hamiltonian
ORIG_PW = imr.penalty_weights
ORIG_MG = imr.merit_gradient


def _penalty_weights_right_endpoints(prob, NT=None):
    w = ORIG_PW(prob, NT)
    h = prob.system.T_ns / prob.system.n_steps
    a = float(prob.penalty_a)
    t = (np.arange(len(w)) + 1) * h
    return h * np.exp(-(((t - prob.system.T_ns) / a) ** 2)) / a


def _penalty_source_negated(prob, tar, q):
    return -ORIG_MG(prob, tar, q)


def _jc_phase_conjugated(sysm, t):
    return ORIG_JC(sysm, -t)


def _jc_half_coupling(sysm, t):
    return 0.5 * ORIG_JC(sysm, t)

MUTATIONS = {
    "J_Nm observable reversed": [(imr, "merit", _merit_nm_transposed_index)],
    "JC phase conjugated": [(model, "jc_hamiltonian", _jc_phase_conjugated)],
    "penalty sampled at t_j+1": [(imr, "penalty_weights", _penalty_weights_right_endpoints)],
    "penalty source negated": [(imr, "merit_gradient", _penalty_source_negated)],
    "JC coupling halved": [(model, "jc_hamiltonian", _jc_half_coupling)],
    "J_Nm terminal adjoint negated": [(imr, "terminal_adjoint", _terminal_nm_negated)],
    "hamiltonian part uses H instead of H^T": [(model, "hamiltonian_part", _ham_part_transposed),
                                               (imr, "hamiltonian_part", _ham_part_transposed)],
    "hamiltonian part with +i": [(model, "hamiltonian_part", _ham_part_sign),
                                 (imr, "hamiltonian_part", _ham_part_sign)],
    "dissipator without anticommutator": [(model, "dissipator_part", _diss_no_anticomm)],
    "dissipator jump term halved": [(model, "dissipator_part", _diss_half_jump)],
    "self-Kerr -xi instead of -xi/2": [(model, "system_hamiltonian", _syshamiltonian_kerr_factor)],
    "cross-Kerr sign flipped": [(model, "system_hamiltonian", _syshamiltonian_crosskerr_sign)],
    "subsystem order reversed": [(model, "embed", _embed_reversed)],
    "B-spline centres shifted one knot": [(model, "bspline_basis", _bspline_shifted),
                                          (imr, "bspline_basis", _bspline_shifted)],
    "controls missing 2pi": [(model, "control_amplitudes", _control_no_2pi)],
    "carrier phase conjugated": [(model, "control_amplitudes", _control_conj_carrier)],
    "IMR update with dt/2": [(imr, "imr_step", _imr_step_explicit_half)],
    "controls sampled at t_j, not t_j+1/2": [(imr, "imr_step", _imr_step_wrong_time)],
    "terminal adjoint sign": [(imr, "terminal_adjoint", _terminal_sign)],
    "imaginary-part derivative missing i": [(imr, "dd_dalpha", _dd_no_imag_i)],
    "control horizon ignored": [(model, "control_horizon", _horizon_ignored),
                                (imr, "control_horizon", _horizon_ignored)],
    "gradient's spline factors on the final time, not the horizon": [(imr, "control_horizon", _horizon_ignored)],
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pins_catch_mutation(name, monkeypatch):
    for mod, attr, fn in MUTATIONS[name]:
        monkeypatch.setattr(mod, attr, fn)
    assert _some_pin_fails(), f"no pin caught: {name}"
