"""Seeded synthetic inputs: gate lists, angles, Hamiltonian terms and states.

This module holds only structure and random draws, none of the simulator's
arithmetic: it names gates (kind, target qubits, control qubits, angles) and
Pauli terms (coefficient, X mask, Z mask). Both the CUDA path and the CPU oracle
read what it produces; neither side's matrices, phases or reductions live here.

Every generator takes a seed and draws from ``numpy.random.Generator(PCG64)`` in
a fixed, documented order, so a workload is reproducible from its seed alone.

Qubit q is bit (n-1-q) of a basis index (qubit 0 = most significant bit); in a
Pauli mask, bit q stands for qubit q.
"""
from __future__ import annotations

import math
from typing import NamedTuple

import numpy as np


class Gate(NamedTuple):
    kind: str                 # H X Y Z S SDG T TDG RX RY RZ U1 U2 U3 CZ CU1 SWAP UNITARY
    targets: tuple
    controls: tuple = ()
    params: tuple = ()
    matrix: object = None     # complex 2^k x 2^k array for UNITARY, else None


# targets, parameters of each named kind (structure only)
KINDS = {
    "H": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0),
    "S": (1, 0), "SDG": (1, 0), "T": (1, 0), "TDG": (1, 0),
    "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1), "U1": (1, 1),
    "U2": (1, 2), "U3": (1, 3),
    "CZ": (2, 0), "CU1": (2, 1), "SWAP": (2, 0),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ QFT
def qft_circuit(n: int) -> list:
    """Textbook QFT (Sec. 3.1: H, CZPow and SWAP gates): for i = 0..n-1, H(i)
    then CU1(2 pi / 2^(j-i+1)) with control j on target i for j = i+1..n-1;
    then SWAP(i, n-1-i) for i < n/2. Gate count n + n(n-1)/2 + floor(n/2)."""
    gates = []
    for i in range(n):
        gates.append(Gate("H", (i,)))
        for j in range(i + 1, n):
            gates.append(Gate("CU1", (j, i), (), (2.0 * math.pi / (1 << (j - i + 1)),)))
    for i in range(n // 2):
        gates.append(Gate("SWAP", (i, n - 1 - i)))
    return gates


def qft_input(n: int, seed: int = 1) -> int:
    """Basis-state input x ~ U[0, 2^n) (one draw)."""
    return int(rng(seed).integers(0, 1 << n))


# ------------------------------------------------------------------ random layers
def random_layer_circuit(n: int, layers: int = 20, seed: int = 2) -> list:
    """Random-layer circuit: in layer l, U3(theta, phi, lambda) on every qubit
    (angles ~ U[0, 2 pi), drawn as one (layers, n, 3) array in (l, q, angle)
    order), then CZ(i, i+1) for i = l mod 2, l mod 2 + 2, ... with i+1 <= n-1."""
    ang = rng(seed).uniform(0.0, 2.0 * math.pi, size=(layers, n, 3))
    gates = []
    for l in range(layers):
        for q in range(n):
            gates.append(Gate("U3", (q,), (), tuple(float(a) for a in ang[l, q])))
        for i in range(l % 2, n - 1, 2):
            gates.append(Gate("CZ", (i, i + 1)))
    return gates


# ------------------------------------------------------------------ variational
def variational_params(batch: int, layers: int, n: int, seed: int = 4) -> np.ndarray:
    """Angles ~ U[0, 2 pi), shape (batch, layers, n)."""
    return rng(seed).uniform(0.0, 2.0 * math.pi, size=(batch, layers, n))


def variational_circuit(n: int, thetas: np.ndarray) -> list:
    """Hardware-efficient ansatz (Sec. 3.2): per layer RY(theta[l, q]) on every
    qubit, then CZ(i, i+1) for i = 0..n-2. ``thetas`` has shape (layers, n);
    parameter index = l * n + q."""
    thetas = np.asarray(thetas, dtype=np.float64)
    gates = []
    for l in range(thetas.shape[0]):
        for q in range(n):
            gates.append(Gate("RY", (q,), (), (float(thetas[l, q]),)))
        for i in range(n - 1):
            gates.append(Gate("CZ", (i, i + 1)))
    return gates


def tfim_terms(n: int, g: float = 1.0) -> list:
    """Open-chain transverse-field Ising H = -sum_{i<n-1} Z_i Z_{i+1} - g sum_i X_i
    as (coeff, x_mask, z_mask) terms."""
    terms = [(-1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    terms += [(-float(g), 1 << i, 0) for i in range(n)]
    return terms


# ------------------------------------------------------------------ adiabatic
def transverse_field_terms(n: int) -> list:
    """H0 = -sum_i X_i (Eq. (5))."""
    return [(-1.0, 1 << i, 0) for i in range(n)]


def random_ising_terms(n: int, r: np.random.Generator) -> list:
    """H1 = sum_{i<j} J_ij Z_i Z_j + sum_i h_i Z_i with J_ij, h_i ~ N(0, 1);
    J drawn first in (i, j) lexicographic order, then h."""
    J = r.standard_normal(n * (n - 1) // 2)
    h = r.standard_normal(n)
    terms = []
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            terms.append((float(J[k]), 0, (1 << i) | (1 << j)))
            k += 1
    terms += [(float(h[i]), 0, 1 << i) for i in range(n)]
    return terms


def adiabatic_instances(count: int = 64, n_lo: int = 16, n_hi: int = 26, seed: int = 5) -> list:
    """``count`` instances with n ~ U{n_lo..n_hi} (all widths drawn first), then
    each instance's J, h in instance order. Returns [(n, h0_terms, h1_terms)]."""
    r = rng(seed)
    ns = r.integers(n_lo, n_hi + 1, size=count)
    return [(int(m), transverse_field_terms(int(m)), random_ising_terms(int(m), r)) for m in ns]


# ------------------------------------------------------------------ closed-form circuits
def ghz_circuit(n: int) -> list:
    """H(0), then CNOT(0 -> q) for q = 1..n-1 (X with control 0)."""
    return [Gate("H", (0,))] + [Gate("X", (q,), (0,)) for q in range(1, n)]


def grover_circuit(n: int, marked, iterations: int) -> list:
    """Grover search: H on every qubit, then ``iterations`` rounds of
    oracle (phase flip of each marked basis state: X on its 0-qubits, Z on
    qubit n-1 controlled by qubits 0..n-2, X again) and diffusion
    (H^n X^n [multi-controlled Z] X^n H^n)."""
    allq = list(range(n))
    mcz = Gate("Z", (n - 1,), tuple(range(n - 1)))
    gates = [Gate("H", (q,)) for q in allq]
    for _ in range(iterations):
        for m in marked:
            zeros = [q for q in allq if not (m >> (n - 1 - q)) & 1]
            gates += [Gate("X", (q,)) for q in zeros]
            gates.append(mcz)
            gates += [Gate("X", (q,)) for q in zeros]
        gates += [Gate("H", (q,)) for q in allq]
        gates += [Gate("X", (q,)) for q in allq]
        gates.append(mcz)
        gates += [Gate("X", (q,)) for q in allq]
        gates += [Gate("H", (q,)) for q in allq]
    return gates


# ------------------------------------------------------------------ mixed random circuits
def random_unitary(k: int, r: np.random.Generator) -> np.ndarray:
    """Haar-like random 2^k x 2^k unitary: QR of a complex Gaussian matrix
    (real part drawn before the imaginary part)."""
    d = 1 << k
    a = r.standard_normal((d, d)) + 1j * r.standard_normal((d, d))
    q, rr = np.linalg.qr(a)
    ph = np.diag(rr) / np.abs(np.diag(rr))
    return q * ph


def random_mixed_circuit(n: int, count: int, seed: int, max_controls: int = 2,
                         max_unitary_k: int = 3, kinds=None) -> list:
    """A random queue mixing every gate kind, random target positions (low,
    intra-warp and high qubits alike) and up to ``max_controls`` controls.
    Draw order per gate: kind, qubits (one permutation), control count, angles,
    then the UNITARY matrix if any."""
    r = rng(seed)
    names = list(KINDS) + ["UNITARY"] if kinds is None else list(kinds)
    names = [k for k in names if k == "UNITARY" or KINDS[k][0] <= n]
    gates = []
    for _ in range(count):
        kind = names[int(r.integers(0, len(names)))]
        if kind == "UNITARY":
            k = int(r.integers(1, min(max_unitary_k, n) + 1))
            npar = 0
        else:
            k, npar = KINDS[kind]
        perm = r.permutation(n)
        nc = int(r.integers(0, min(max_controls, n - k) + 1))
        params = tuple(float(v) for v in r.uniform(0.0, 2.0 * math.pi, size=npar))
        mat = random_unitary(k, r) if kind == "UNITARY" else None
        gates.append(Gate(kind, tuple(int(q) for q in perm[:k]),
                          tuple(int(q) for q in perm[k:k + nc]), params, mat))
    return gates


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex Gaussian state (real parts drawn before imaginary)."""
    r = rng(seed)
    v = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


def random_pauli_terms(n: int, count: int, seed: int) -> list:
    """Random Pauli strings (each qubit I, X, Y or Z uniformly) with N(0,1)
    coefficients; draw order per term: coefficient, then the n letters."""
    r = rng(seed)
    terms = []
    for _ in range(count):
        c = float(r.standard_normal())
        letters = r.integers(0, 4, size=n)
        xm = zm = 0
        for q, L in enumerate(letters):
            if L in (1, 2):
                xm |= 1 << q
            if L in (2, 3):
                zm |= 1 << q
        terms.append((c, xm, zm))
    return terms
