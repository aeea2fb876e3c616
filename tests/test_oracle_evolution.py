"""Pins of the exact time-evolution oracle (Sec. 2.6 solvers) and of the
schedule gradient (Sec. 4 schedule optimisation), against closed forms,
convergence orders, the independently written Trotter step, and finite
differences."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import evolution as ev
from paper_2009_01845_gb300 import inputs as qi


def test_constant_hamiltonian_exp_solver_is_one_exponential():
    """H0 = H1 = H: H(t) = H for all t, and the product of the exp solver's
    steps is exp(-i H T) for any dt."""
    n = 3
    H = qi.random_pauli_terms(n, 6, seed=3)
    psi0 = qi.random_state(n, 4)
    want = scipy.linalg.expm(-1j * 0.7 * ev.hamiltonian_matrix(n, H)) @ psi0
    for dt in (0.7, 0.1, 0.07):
        np.testing.assert_allclose(ev.evolve_exp(psi0, n, H, H, 0.7, dt), want, atol=1e-13)


def test_single_qubit_rotation_closed_form():
    """H = w X from |0>: psi(T) = cos(w T) |0> - i sin(w T) |1>."""
    w, T = 1.3, 0.9
    H = [(w, 1, 0)]
    want = np.array([math.cos(w * T), -1j * math.sin(w * T)])
    psi0 = np.array([1.0, 0.0], dtype=np.complex128)
    np.testing.assert_allclose(ev.evolve_exp(psi0, 1, H, H, T, 0.3), want, atol=1e-14)
    np.testing.assert_allclose(ev.evolve_rk4(psi0, 1, H, H, T, 1e-3), want, atol=1e-12)
    np.testing.assert_allclose(ev.evolve_rk45(psi0, 1, H, H, T, 1e-2), want, atol=1e-12)


def test_eigenstate_only_gains_a_phase():
    n = 3
    H = qi.tfim_terms(n, 0.9)
    w, v = np.linalg.eigh(ev.hamiltonian_matrix(n, H))
    psi0 = v[:, 2].astype(np.complex128)
    for solver, dt in (("exp", 0.5), ("rk4", 1e-3), ("rk45", 1e-2)):
        got = ev.SOLVERS[solver](psi0, n, H, H, 1.0, dt)
        np.testing.assert_allclose(got, np.exp(-1j * w[2]) * psi0, atol=1e-10)


def _slope(errs, dts):
    return np.polyfit(np.log(dts), np.log(errs), 1)[0]


def test_convergence_orders():
    """Time-dependent H(s): errors against a fine-step exp reference fall as
    dt^2 (exp at the midpoint), dt^4 (rk4) and dt^5 (rk45)."""
    n, T = 3, 1.0
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(5)) + qi.random_pauli_terms(n, 3, seed=6)
    psi0 = oracle.plus_state(n)
    ref = ev.evolve_rk45(psi0, n, h0, h1, T, 1 / 512)
    for solver, order, dts in (("exp", 2, [1 / 8, 1 / 16, 1 / 32, 1 / 64]),
                               ("rk4", 4, [1 / 8, 1 / 16, 1 / 32, 1 / 64]),
                               ("rk45", 5, [1 / 4, 1 / 8, 1 / 16, 1 / 32])):
        errs = [np.linalg.norm(ev.SOLVERS[solver](psi0, n, h0, h1, T, dt) - ref) for dt in dts]
        assert abs(_slope(errs, dts) - order) < 0.35, (solver, errs)


def test_schedule_energy_follows_the_trotter_step():
    """The dense-matrix steps of the schedule code equal the oracle's Trotter
    step (diagonal phases and RX gates on the state vector)."""
    n = 4
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(7))
    svals = [0.1, 0.35, 0.5, 0.9]
    psi = oracle.plus_state(n)
    for s in svals:
        oracle.trotter_step(psi, n, h0, h1, s, 0.2)
    E = ev.schedule_energy(n, h0, h1, svals, 0.2, oracle.plus_state(n))
    assert abs(E - oracle.expectation(psi, n, h1).real) < 1e-12


def test_schedule_gradient_against_finite_differences():
    n, dt = 4, 0.15
    h0 = qi.transverse_field_terms(n) + [(0.3, 0, 0b0110)]
    h1 = qi.random_ising_terms(n, qi.rng(8))
    svals = list(np.linspace(0.05, 0.95, 7))
    psi0 = oracle.plus_state(n)
    E, g, gdt = ev.schedule_gradient(n, h0, h1, svals, dt, psi0)
    assert abs(E - ev.schedule_energy(n, h0, h1, svals, dt, psi0)) < 1e-13
    h = 1e-5
    for k in range(len(svals)):
        sp, sm = list(svals), list(svals)
        sp[k] += h
        sm[k] -= h
        fd = (ev.schedule_energy(n, h0, h1, sp, dt, psi0) - ev.schedule_energy(n, h0, h1, sm, dt, psi0)) / (2 * h)
        assert abs(fd - g[k]) < 1e-8, (k, fd, g[k])
    fd = (ev.schedule_energy(n, h0, h1, svals, dt + h, psi0) -
          ev.schedule_energy(n, h0, h1, svals, dt - h, psi0)) / (2 * h)
    assert abs(fd - gdt) < 1e-8


def test_schedule_gradient_vanishes_when_h_does_not_depend_on_s():
    n = 3
    H = qi.tfim_terms(n, 0.7)
    _, g, _ = ev.schedule_gradient(n, H, H, [0.2, 0.5, 0.8], 0.1, qi.random_state(n, 9))
    np.testing.assert_allclose(g, 0.0, atol=1e-13)
