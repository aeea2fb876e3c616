"""Oracle: density matrices and noise channels (Sec. 2.4, "Density matrices
and noise": the state of a noisy circuit is a density matrix; channels act on
it).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Nothing here is shared
with the CUDA library.

A density matrix of n qubits is a 2^n x 2^n complex128 matrix rho whose rows
and columns are indexed by basis integers, qubit 0 the most significant bit
(as for state vectors). Everything is written with full matrices, so n stays
small (n <= 8):
  * a gate G on its targets, with controls, is the 2^n x 2^n operator U that
    applies G to the target bits of every index group whose controls are all 1
    and the identity elsewhere (Eq. (1), Sec. 2.3-2.4); rho -> U rho U^dag;
  * a channel with Kraus operators K_i on its targets (sum_i K_i^dag K_i = I)
    maps rho -> sum_i K_i rho K_i^dag, each K_i embedded like a gate (the Kraus
    form of a quantum channel; the paper names its channels but prints none);
  * read-outs: the outcome probabilities are rho's diagonal; the energy of a
    Pauli sum H is Tr(rho H), with H built from its terms as full matrices.
The standard channels below are written from their textbook Kraus forms.
"""
from __future__ import annotations

import math

import numpy as np

from . import gates as _gates


def embed(n: int, targets, M: np.ndarray, controls=()) -> np.ndarray:
    """The 2^n x 2^n operator of the matrix M (2^k x 2^k, local index with the
    first target most significant) on `targets`, applied where every control
    is 1 and the identity on the other index groups."""
    k = len(targets)
    M = np.asarray(M, dtype=np.complex128)
    if M.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the targets")
    dim = 1 << n
    bit = [1 << (n - 1 - q) for q in targets]
    cmask = 0
    for q in controls:
        cmask |= 1 << (n - 1 - q)
    tmask = sum(bit)
    U = np.zeros((dim, dim), dtype=np.complex128)
    for base in range(dim):
        if base & tmask:
            continue
        if (base & cmask) != cmask:
            for l in range(1 << k):
                i = base | sum(bit[j] for j in range(k) if (l >> (k - 1 - j)) & 1)
                U[i, i] = 1.0
            continue
        idx = [base | sum(bit[j] for j in range(k) if (l >> (k - 1 - j)) & 1) for l in range(1 << k)]
        for r in range(1 << k):
            for c in range(1 << k):
                U[idx[r], idx[c]] = M[r, c]
    return U


def pauli_operator(n: int, x_mask: int, z_mask: int) -> np.ndarray:
    """The Pauli string with X on the qubits of x_mask only, Z on z_mask only
    and Y = i X Z on both (bit q of a mask is qubit q), as the Kronecker
    product of its one-qubit factors, qubit 0 first."""
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    out = np.ones((1, 1), dtype=np.complex128)
    for q in range(n):
        xq, zq = (x_mask >> q) & 1, (z_mask >> q) & 1
        f = Y if (xq and zq) else X if xq else Z if zq else np.eye(2, dtype=np.complex128)
        out = np.kron(out, f)
    return out


def from_state(psi: np.ndarray) -> np.ndarray:
    """|psi><psi|."""
    psi = np.asarray(psi, dtype=np.complex128).reshape(-1)
    return np.outer(psi, psi.conj())


def basis(n: int, x: int) -> np.ndarray:
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[x, x] = 1.0
    return rho


def apply_gate(rho: np.ndarray, n: int, gate) -> np.ndarray:
    """U rho U^dag for one gate (controls included)."""
    U = embed(n, gate.targets, _gates.gate_matrix(gate.kind, gate.params, gate.matrix), gate.controls)
    return U @ rho @ U.conj().T


def apply_circuit(rho: np.ndarray, n: int, gates) -> np.ndarray:
    for g in gates:
        rho = apply_gate(rho, n, g)
    return rho


def apply_channel(rho: np.ndarray, n: int, targets, kraus) -> np.ndarray:
    """sum_i K_i rho K_i^dag with every Kraus operator embedded on `targets`."""
    out = np.zeros_like(rho)
    for K in kraus:
        E = embed(n, targets, K)
        out += E @ rho @ E.conj().T
    return out


def probabilities(rho: np.ndarray) -> np.ndarray:
    """Outcome probabilities: the diagonal of rho."""
    return np.real(np.diag(rho)).copy()


def expectation(rho: np.ndarray, n: int, terms) -> complex:
    """Tr(rho H) for H = sum_t c_t P_t."""
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for c, xm, zm in terms:
        H += c * pauli_operator(n, int(xm), int(zm))
    return complex(np.trace(rho @ H))


# ---------------------------------------------------------------- channels
def kraus_pauli(px: float, py: float, pz: float):
    """rho -> (1 - px - py - pz) rho + px X rho X + py Y rho Y + pz Z rho Z."""
    p0 = 1.0 - px - py - pz
    I = np.eye(2, dtype=np.complex128)
    X = _gates.gate_matrix("X")
    Y = _gates.gate_matrix("Y")
    Z = _gates.gate_matrix("Z")
    return [math.sqrt(p0) * I, math.sqrt(px) * X, math.sqrt(py) * Y, math.sqrt(pz) * Z]


def kraus_depolarizing(p: float):
    """With probability p the qubit is hit by X, Y or Z, each with p / 3."""
    return kraus_pauli(p / 3.0, p / 3.0, p / 3.0)


def kraus_amplitude_damping(gamma: float):
    """Decay |1> -> |0> with probability gamma."""
    return [np.array([[1, 0], [0, math.sqrt(1.0 - gamma)]], dtype=np.complex128),
            np.array([[0, math.sqrt(gamma)], [0, 0]], dtype=np.complex128)]


def kraus_phase_damping(lam: float):
    """Loss of phase coherence without energy loss: rho_01 -> sqrt(1 - lam) rho_01."""
    return [np.array([[1, 0], [0, math.sqrt(1.0 - lam)]], dtype=np.complex128),
            np.array([[0, 0], [0, math.sqrt(lam)]], dtype=np.complex128)]


def kraus_unitary_mixture(probs, unitaries):
    """rho -> sum_i p_i U_i rho U_i^dag."""
    return [math.sqrt(p) * np.asarray(U, dtype=np.complex128) for p, U in zip(probs, unitaries)]
