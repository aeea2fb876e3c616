"""Gate matrices of the oracle, written from their definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each named gate maps to a dense complex128 matrix in the local index order of
Eq. (1) of the Qibo paper (Sec. 2.3): for targets (t_0, .., t_{k-1}) the local
row/column index is sum_j bit(t_j) * 2^(k-1-j), i.e. the first target is the
most significant local bit.

Readings of conventions the paper leaves open (stated once here):
  * R_P(theta) = exp(-i theta P / 2) for P in {X, Y, Z};
  * U1(lam) = diag(1, e^{i lam}); CU1(theta) = diag(1, 1, 1, e^{i theta})
    (the paper's QFT uses CZPow(t), which is CU1(pi t), Sec. 3.1);
  * U3 follows OpenQASM 2:
      U3(th, ph, lam) = [[cos th/2, -e^{i lam} sin th/2],
                         [e^{i ph} sin th/2, e^{i(ph+lam)} cos th/2]];
    U2(ph, lam) = U3(pi/2, ph, lam);
  * CZ = diag(1, 1, 1, -1); SWAP exchanges |01> and |10>.
Controls are not part of the matrix: a controlled gate applies its matrix only
where every control qubit is 1 (Sec. 2.4, "Controlled gates").
"""
from __future__ import annotations

import cmath
import math

import numpy as np

# number of targets and parameters of every named kind
ARITY = {
    "H": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0),
    "S": (1, 0), "SDG": (1, 0), "T": (1, 0), "TDG": (1, 0),
    "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1), "U1": (1, 1),
    "U2": (1, 2), "U3": (1, 3),
    "CZ": (2, 0), "CU1": (2, 1), "SWAP": (2, 0),
}


def _u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array(
        [[c, -cmath.exp(1j * lam) * s],
         [cmath.exp(1j * phi) * s, cmath.exp(1j * (phi + lam)) * c]],
        dtype=np.complex128)


def gate_matrix(kind: str, params=(), matrix=None) -> np.ndarray:
    """The 2^k x 2^k matrix of one gate (controls excluded)."""
    p = tuple(float(v) for v in params)
    if kind == "UNITARY":
        m = np.asarray(matrix, dtype=np.complex128)
        return m.copy()
    if kind == "H":
        return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    if kind == "X":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if kind == "Y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if kind == "Z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if kind == "S":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if kind == "SDG":
        return np.array([[1, 0], [0, -1j]], dtype=np.complex128)
    if kind == "T":
        return np.array([[1, 0], [0, cmath.exp(1j * math.pi / 4)]], dtype=np.complex128)
    if kind == "TDG":
        return np.array([[1, 0], [0, cmath.exp(-1j * math.pi / 4)]], dtype=np.complex128)
    if kind == "RX":
        c, s = math.cos(p[0] / 2.0), math.sin(p[0] / 2.0)
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if kind == "RY":
        c, s = math.cos(p[0] / 2.0), math.sin(p[0] / 2.0)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if kind == "RZ":
        return np.array([[cmath.exp(-0.5j * p[0]), 0], [0, cmath.exp(0.5j * p[0])]],
                        dtype=np.complex128)
    if kind == "U1":
        return np.array([[1, 0], [0, cmath.exp(1j * p[0])]], dtype=np.complex128)
    if kind == "U2":
        return _u3(math.pi / 2.0, p[0], p[1])
    if kind == "U3":
        return _u3(p[0], p[1], p[2])
    if kind == "CZ":
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if kind == "CU1":
        return np.diag([1, 1, 1, cmath.exp(1j * p[0])]).astype(np.complex128)
    if kind == "SWAP":
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0, 0] = m[3, 3] = 1.0
        m[1, 2] = m[2, 1] = 1.0
        return m
    raise ValueError(f"unknown gate kind {kind!r}")


def generator_derivative(kind: str, params) -> np.ndarray:
    """dG/dtheta for the single-parameter gates, from their definitions:
    d/dth exp(-i th P/2) = (-i/2) P exp(-i th P/2); d/dl U1(l) = diag(0, i e^{il});
    d/dth CU1(th) = diag(0, 0, 0, i e^{i th})."""
    th = float(params[0])
    if kind in ("RX", "RY", "RZ"):
        P = gate_matrix({"RX": "X", "RY": "Y", "RZ": "Z"}[kind])
        return (-0.5j) * P @ gate_matrix(kind, (th,))
    if kind == "U1":
        return np.diag([0, 1j * cmath.exp(1j * th)]).astype(np.complex128)
    if kind == "CU1":
        return np.diag([0, 0, 0, 1j * cmath.exp(1j * th)]).astype(np.complex128)
    raise ValueError(f"{kind} has no single-parameter derivative")
