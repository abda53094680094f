"""Seeded synthetic inputs for the Lindblad IMR path.

This package only draws numbers and lays them out: system parameters, control
coefficients, initial density matrices, gate matrices and target states.  It
holds none of the method's arithmetic (no Hamiltonian, no Lindbladian, no
B-spline evaluation, no time stepping), so both the CUDA path and the CPU
oracle can consume the same bytes without sharing any of the method's code.
"""

from .synthetic import (  # noqa: F401
    Problem,
    SystemSpec,
    ControlSpec,
    config,
    config1,
    config2,
    config3,
    config4,
    config5,
    prefix,
    fock_superposition,
    three_gate_states,
    cnot_three_states,
    basis_matrices,
    ensemble_state,
    reset_ensemble,
    random_problem,
    basis_outer,
    random_pure_state,
    CNOT,
    XGATE,
)
