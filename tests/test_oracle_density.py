"""Pins of the density-matrix oracle (Sec. 2.4, "Density matrices and noise")
against facts that do not come from it: the state-vector oracle (an
independent C implementation) for pure states, Kronecker products, the
defining properties of channels, and the closed forms of the standard
channels on one qubit."""
import math

import numpy as np
import pytest

import oracle
from oracle import density as od
from oracle import gates as og
from paper_2009_01845_gb300 import inputs as qi


def test_embedding_equals_kronecker_products():
    n = 4
    r = qi.rng(3)
    for q in range(n):
        M = qi.random_unitary(1, r)
        want = np.ones((1, 1))
        for j in range(n):
            want = np.kron(want, M if j == q else np.eye(2))
        np.testing.assert_allclose(od.embed(n, [q], M), want, atol=1e-15)
    # a controlled gate is the identity where the control is 0
    U = od.embed(3, [2], og.gate_matrix("X"), controls=[0])
    for x in range(8):
        y = x ^ 1 if (x >> 2) & 1 else x
        assert U[y, x] == 1.0


@pytest.mark.parametrize("n", [1, 3, 5])
def test_pure_state_follows_the_state_vector_oracle(n):
    gates = qi.random_mixed_circuit(n, 30, seed=40 + n, max_controls=min(2, n - 1), max_unitary_k=min(3, n))
    psi0 = qi.random_state(n, 41 + n)
    rho = od.apply_circuit(od.from_state(psi0), n, gates)
    psi = oracle.apply_circuit(psi0.copy(), n, gates)
    np.testing.assert_allclose(rho, od.from_state(psi), atol=1e-13)
    np.testing.assert_allclose(od.probabilities(rho), oracle.probabilities(psi, n), atol=1e-14)
    terms = qi.random_pauli_terms(n, 8, seed=n) + qi.tfim_terms(n, 0.7)
    assert abs(od.expectation(rho, n, terms) - oracle.expectation(psi, n, terms)) < 1e-12


def test_pauli_operator_phases():
    # Y = i X Z, and the masks name qubits (qubit 0 = most significant factor)
    Y = og.gate_matrix("Y")
    np.testing.assert_allclose(od.pauli_operator(1, 1, 1), Y)
    np.testing.assert_allclose(od.pauli_operator(2, 0b10, 0), np.kron(np.eye(2), og.gate_matrix("X")))


@pytest.mark.parametrize("make", [lambda: od.kraus_depolarizing(0.3), lambda: od.kraus_amplitude_damping(0.4),
                                  lambda: od.kraus_phase_damping(0.25), lambda: od.kraus_pauli(0.1, 0.2, 0.05)])
def test_channels_are_trace_preserving_and_positive(make):
    kraus = make()
    np.testing.assert_allclose(sum(K.conj().T @ K for K in kraus), np.eye(2), atol=1e-15)
    n = 3
    rho = od.from_state(qi.random_state(n, 5))
    rho = 0.6 * rho + 0.4 * od.from_state(qi.random_state(n, 6))
    for q in range(n):
        out = od.apply_channel(rho, n, [q], kraus)
        assert abs(np.trace(out) - 1.0) < 1e-14
        np.testing.assert_allclose(out, out.conj().T, atol=1e-15)
        assert np.min(np.linalg.eigvalsh(out)) > -1e-13


def bloch(rho):
    return np.real([np.trace(rho @ og.gate_matrix(p)) for p in ("X", "Y", "Z")])


def test_depolarizing_shrinks_the_bloch_vector():
    rho = od.from_state(qi.random_state(1, 8))
    for p in (0.0, 0.2, 0.75):
        out = od.apply_channel(rho, 1, [0], od.kraus_depolarizing(p))
        np.testing.assert_allclose(bloch(out), (1 - 4 * p / 3) * bloch(rho), atol=1e-14)
    # p = 3/4: the maximally mixed state
    np.testing.assert_allclose(od.apply_channel(rho, 1, [0], od.kraus_depolarizing(0.75)), np.eye(2) / 2,
                               atol=1e-15)


def test_amplitude_and_phase_damping_closed_forms():
    rho = od.from_state(qi.random_state(1, 9))
    g = 0.35
    out = od.apply_channel(rho, 1, [0], od.kraus_amplitude_damping(g))
    assert abs(out[1, 1] - (1 - g) * rho[1, 1]) < 1e-15
    assert abs(out[0, 0] - (rho[0, 0] + g * rho[1, 1])) < 1e-15
    assert abs(out[0, 1] - math.sqrt(1 - g) * rho[0, 1]) < 1e-15
    lam = 0.6
    out = od.apply_channel(rho, 1, [0], od.kraus_phase_damping(lam))
    np.testing.assert_allclose(np.diag(out), np.diag(rho), atol=1e-15)
    assert abs(out[0, 1] - math.sqrt(1 - lam) * rho[0, 1]) < 1e-15


def test_channel_acts_on_its_qubit_only():
    """On a product state rho_A (x) rho_B a channel on qubit 0 (the most
    significant) gives E(rho_A) (x) rho_B."""
    ra = od.from_state(qi.random_state(1, 10))
    rb = od.from_state(qi.random_state(2, 11))
    kraus = od.kraus_amplitude_damping(0.5)
    out = od.apply_channel(np.kron(ra, rb), 3, [0], kraus)
    np.testing.assert_allclose(out, np.kron(od.apply_channel(ra, 1, [0], kraus), rb), atol=1e-15)


def test_two_qubit_channel_of_unitaries():
    """A mixture of two-qubit unitaries: the average of the conjugated states."""
    n = 3
    r = qi.rng(12)
    U1, U2 = qi.random_unitary(2, r), qi.random_unitary(2, r)
    rho = od.from_state(qi.random_state(n, 13))
    out = od.apply_channel(rho, n, [2, 0], od.kraus_unitary_mixture([0.3, 0.7], [U1, U2]))
    E1, E2 = od.embed(n, [2, 0], U1), od.embed(n, [2, 0], U2)
    np.testing.assert_allclose(out, 0.3 * E1 @ rho @ E1.conj().T + 0.7 * E2 @ rho @ E2.conj().T, atol=1e-14)
