"""Oracle: exact small-n time evolution and schedule gradients (Sec. 2.6:
the "exp" solver and the Runge-Kutta integrators of the Schroedinger equation
i d/dt psi = H(t) psi; Sec. 4, adiabatic evolution: the schedule s(t) is
optimised so that the final energy is minimal).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Nothing here is shared
with the CUDA library.

H(t) = (1 - s) H0 + s H1 with the linear schedule s = t / T (Eq. (4)); the
Hamiltonians are Pauli sums, built here as full 2^n x 2^n matrices (n small).
Readings where the paper is silent:
  * "exp" applies exp(-i dt H(t_k + dt/2)) per step (H at the step's midpoint:
    the exponential of a time-dependent H over a step is only defined up to
    such a choice; the midpoint makes the step second order, as for Trotter);
  * "rk4" is the classical fourth-order Runge-Kutta method and "rk45" the
    fifth-order solution of Dormand and Prince's embedded 5(4) pair, both with
    the fixed step dt (the paper names the integrators, not their step
    control), with H evaluated at each stage's time;
  * the schedule gradient is that of the energy E = Re <psi_K|H1|psi_K> after
    K second-order Trotter steps (the splitting of ``oracle.trotter_step``),
    with respect to each step's schedule value s_k and to the step dt shared
    by all steps; a polynomial schedule's coefficients or the total time follow
    by the chain rule.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import density as _density


def hamiltonian_matrix(n: int, terms) -> np.ndarray:
    """sum_t c_t P_t as a full matrix (qubit 0 the most significant bit)."""
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for c, xm, zm in terms:
        H += c * _density.pauli_operator(n, int(xm), int(zm))
    return H


def h_of_s(n: int, h0_terms, h1_terms, s: float) -> np.ndarray:
    return (1.0 - s) * hamiltonian_matrix(n, h0_terms) + s * hamiltonian_matrix(n, h1_terms)


def _steps(T, dt, steps):
    K = int(round(T / dt))
    return K if steps is None else min(K, steps)


def evolve_exp(psi, n, h0_terms, h1_terms, T, dt, steps=None):
    """psi <- exp(-i dt H(s_k)) psi per step, s_k = (k + 1/2) dt / T."""
    H0, H1 = hamiltonian_matrix(n, h0_terms), hamiltonian_matrix(n, h1_terms)
    psi = np.array(psi, dtype=np.complex128)
    for k in range(_steps(T, dt, steps)):
        s = (k + 0.5) * dt / T
        psi = scipy.linalg.expm(-1j * dt * ((1.0 - s) * H0 + s * H1)) @ psi
    return psi


def _rhs(H0, H1, T):
    def f(t, y):
        s = t / T
        return -1j * (((1.0 - s) * H0 + s * H1) @ y)
    return f


def evolve_rk4(psi, n, h0_terms, h1_terms, T, dt, steps=None):
    """Classical RK4 on d psi / dt = -i H(t) psi."""
    f = _rhs(hamiltonian_matrix(n, h0_terms), hamiltonian_matrix(n, h1_terms), T)
    y = np.array(psi, dtype=np.complex128)
    for k in range(_steps(T, dt, steps)):
        t = k * dt
        k1 = f(t, y)
        k2 = f(t + dt / 2, y + dt / 2 * k1)
        k3 = f(t + dt / 2, y + dt / 2 * k2)
        k4 = f(t + dt, y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


# Dormand-Prince 5(4): nodes, stage matrix, fifth-order weights
DP_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0]
DP_A = [[],
        [1 / 5],
        [3 / 40, 9 / 40],
        [44 / 45, -56 / 15, 32 / 9],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656]]
DP_B = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]


def evolve_rk45(psi, n, h0_terms, h1_terms, T, dt, steps=None):
    """The fifth-order Dormand-Prince solution with the fixed step dt."""
    f = _rhs(hamiltonian_matrix(n, h0_terms), hamiltonian_matrix(n, h1_terms), T)
    y = np.array(psi, dtype=np.complex128)
    for k in range(_steps(T, dt, steps)):
        t = k * dt
        ks = []
        for i in range(6):
            yi = y + dt * sum(a * kj for a, kj in zip(DP_A[i], ks)) if i else y
            ks.append(f(t + DP_C[i] * dt, yi))
        y = y + dt * sum(b * kj for b, kj in zip(DP_B, ks))
    return y


SOLVERS = {"exp": evolve_exp, "rk4": evolve_rk4, "rk45": evolve_rk45}


# ---------------------------------------------------------------- schedule gradient
def _split(n, terms):
    """Diagonal (Z-string) and transverse (X) parts of a Pauli sum, as matrices."""
    d = [(c, x, z) for c, x, z in terms if int(x) == 0]
    x = [(c, xm, zm) for c, xm, zm in terms if int(xm) != 0]
    return hamiltonian_matrix(n, d), hamiltonian_matrix(n, x)


def _step_factors(D0, D1, X0, X1, s, dt):
    """The second-order step exp(-i dt/2 D(s)) exp(-i dt X(s)) exp(-i dt/2 D(s))
    as its three factors (D(s) = (1-s) D0 + s D1, X(s) likewise)."""
    Dm = scipy.linalg.expm(-0.5j * dt * ((1.0 - s) * D0 + s * D1))
    Xm = scipy.linalg.expm(-1j * dt * ((1.0 - s) * X0 + s * X1))
    return Dm, Xm


def schedule_energy(n, h0_terms, h1_terms, svals, dt, psi0):
    """E = Re <psi_K|H1|psi_K> after the Trotter steps with schedule values svals."""
    D0, X0 = _split(n, h0_terms)
    D1, X1 = _split(n, h1_terms)
    psi = np.array(psi0, dtype=np.complex128)
    for s in svals:
        Dm, Xm = _step_factors(D0, D1, X0, X1, s, dt)
        psi = Dm @ (Xm @ (Dm @ psi))
    H1 = hamiltonian_matrix(n, h1_terms)
    return float(np.real(np.vdot(psi, H1 @ psi)))


def schedule_gradient(n, h0_terms, h1_terms, svals, dt, psi0):
    """(E, dE/ds_k for every step k, dE/d dt) by the product rule: step k's
    derivative is the sum over its three factors of the factor's derivative
    (-i times its generator's derivative times the factor; the generators of
    one factor commute with it), propagated through the later steps;
    dE/dx = 2 Re <psi_K|H1| d psi_K / dx>."""
    D0, X0 = _split(n, h0_terms)
    D1, X1 = _split(n, h1_terms)
    H1 = hamiltonian_matrix(n, h1_terms)
    K = len(svals)
    steps = []
    psis = [np.array(psi0, dtype=np.complex128)]
    for s in svals:
        Dm, Xm = _step_factors(D0, D1, X0, X1, s, dt)
        steps.append((Dm, Xm))
        psis.append(Dm @ (Xm @ (Dm @ psis[-1])))
    psiK = psis[-1]
    E = float(np.real(np.vdot(psiK, H1 @ psiK)))
    lam = H1 @ psiK

    def later(k, v):  # U_{K-1} .. U_{k+1} v
        for j in range(k + 1, K):
            Dm, Xm = steps[j]
            v = Dm @ (Xm @ (Dm @ v))
        return v

    def dstep(k, GD, GX, wD, wX):
        """d/dx of step k applied to psi_k, where dD/dx = -i wD GD D and
        dX/dx = -i wX GX X."""
        Dm, Xm = steps[k]
        p = psis[k]
        a = -1j * wD * (GD @ (Dm @ (Xm @ (Dm @ p))))
        b = Dm @ (-1j * wX * (GX @ (Xm @ (Dm @ p))))
        c = Dm @ (Xm @ (-1j * wD * (GD @ (Dm @ p))))
        return a + b + c

    dE_ds = np.zeros(K)
    dE_ddt = 0.0
    for k, s in enumerate(svals):
        v = later(k, dstep(k, D1 - D0, X1 - X0, dt / 2, dt))
        dE_ds[k] = 2.0 * np.real(np.vdot(lam, v))
        Ds, Xs = (1.0 - s) * D0 + s * D1, (1.0 - s) * X0 + s * X1
        v = later(k, dstep(k, Ds, Xs, 0.5, 1.0))
        dE_ddt += 2.0 * np.real(np.vdot(lam, v))
    return E, dE_ds, dE_ddt
