"""Pins of the oracle's measurement functions (Sec. 2.4, "Measurements"; Sec.
3.3) against brute force, closed forms and a chi-squared test."""
import math

import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi


def brute_marginal(psi, n, qubits):
    """out[y], y's bit (m-1-j) = value of qubits[j]; qubit q is index bit n-1-q."""
    m = len(qubits)
    out = np.zeros(1 << m)
    for x in range(1 << n):
        y = 0
        for j, q in enumerate(qubits):
            y |= ((x >> (n - 1 - q)) & 1) << (m - 1 - j)
        out[y] += abs(psi[x]) ** 2
    return out


@pytest.mark.parametrize("qubits", [[3, 0], [4], [0, 1, 2, 3, 4], [2, 4, 1], [1, 3]])
def test_marginal_brute_force(qubits):
    n = 5
    psi = qi.random_state(n, 11)
    np.testing.assert_allclose(oracle.marginal_probabilities(psi, n, qubits), brute_marginal(psi, n, qubits),
                               rtol=0, atol=1e-14)


def test_marginal_of_product_state():
    """A product state's marginal over a group is the Kronecker product of its
    qubits' single-qubit distributions, in the group's order."""
    r = qi.rng(5)
    n = 6
    singles = []
    psi = np.ones(1, dtype=np.complex128)
    for q in range(n):  # qubit 0 first: it is the most significant index bit
        v = r.normal(size=2) + 1j * r.normal(size=2)
        v /= np.linalg.norm(v)
        singles.append(np.abs(v) ** 2)
        psi = np.kron(psi, v)
    for group in ([4, 1], [0, 5, 2], [3]):
        want = np.ones(1)
        for q in group:
            want = np.kron(want, singles[q])
        np.testing.assert_allclose(oracle.marginal_probabilities(psi, n, group), want, rtol=0, atol=1e-14)


def test_marginal_of_ghz():
    n = 7
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = psi[-1] = 1 / math.sqrt(2)
    for pair in ([0, 6], [5, 2], [3, 4]):
        np.testing.assert_allclose(oracle.marginal_probabilities(psi, n, pair), [0.5, 0, 0, 0.5], atol=1e-15)


def test_sample_basis_state_and_uniform_superposition():
    n = 6
    u = np.linspace(0, 1, 50, endpoint=False)
    assert np.all(oracle.sample(oracle.basis_state(n, 37), n, u) == 37)
    # |+>^n: cdf(x) = (x + 1) / 2^n, so u -> floor(u 2^n) away from the boundaries
    uu = (np.arange(1 << n) + 0.5) / (1 << n)
    np.testing.assert_array_equal(oracle.sample(oracle.plus_state(n), n, uu), np.arange(1 << n))


def test_sample_is_monotone_and_skips_zero_probability():
    n = 5
    psi = qi.random_state(n, 2)
    psi[[0, 1, 7, 30, 31]] = 0  # outcomes that must never be drawn
    u = np.sort(qi.rng(8).uniform(size=4000))
    x = oracle.sample(psi, n, u)
    assert np.all(np.diff(x.astype(np.int64)) >= 0)
    assert not set(x.tolist()) & {0, 1, 7, 30, 31}
    assert oracle.sample(psi, n, [0.0])[0] == 2  # the first outcome with probability > 0
    # u just below 1 (the target can round to the total): the last outcome
    # with probability > 0, never the zero-probability tail
    assert oracle.sample(psi, n, [np.nextafter(1.0, 0.0)])[0] == 29


def test_sample_chi_squared():
    """40000 shots of a random 6-qubit state against its probabilities: the
    chi-squared statistic (63 degrees of freedom) stays below its 1e-6 tail."""
    n, shots = 6, 40000
    psi = qi.random_state(n, 4)
    p = oracle.probabilities(psi, n)
    x = oracle.sample(psi, n, qi.rng(9).uniform(size=shots))
    counts = np.bincount(x.astype(np.int64), minlength=1 << n)
    chi2 = float(np.sum((counts - shots * p) ** 2 / (shots * p)))
    assert chi2 < 130.0, chi2  # P(chi2_63 > 130) ~ 2e-6
