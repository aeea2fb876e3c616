"""Oracle: a plain, slow, obviously correct CPU complex128 state-vector simulator.

TEST INFRASTRUCTURE ONLY. Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or execute anything in this
package. It shares no code with the CUDA library and imports nothing from it;
the CUDA path never imports it.

What it computes, and where the Qibo paper defines it:
  * gate application, Eq. (1) of Sec. 2.3, with controls as in Sec. 2.4
    (``statevec.c:orc_apply_matrix``);
  * outcome probabilities (Sec. 2.4, "Measurements") and the squared norm;
  * the expectation value of a Pauli-sum Hamiltonian (the Energy callback,
    Sec. 2.4), ``expectation``;
  * the second-order Trotter step of H(s) = (1-s) H0 + s H1 (Sec. 2.6, Eq. (4)),
    ``trotter_step`` and ``adiabatic_evolve``;
  * the exact gradient of an energy with respect to rotation angles, from the
    product rule (``gradient_exact``, any controls) and by the parameter-shift
    rule (``gradient_parameter_shift``, exact for uncontrolled rotations); the
    adjoint sweep must reproduce them (the paper differentiates through its
    native backends only, Sec. 2.3);
  * the fused matrix of a gate sequence on a qubit set (Sec. 2.4, "Gate
    fusion": the product of the gates' matrices), ``fused_matrix``;
  * measurements (Sec. 2.4, "Measurements", and Sec. 3.3): the outcome
    probabilities of a group of qubits traced over the others,
    ``marginal_probabilities``, and samples of the measurement of every qubit
    drawn from the state's distribution for given uniforms, ``sample``.

Readings where the paper is silent are stated next to the code that takes them
(qubit order, matrix index order and gate conventions in ``statevec.c`` and
``gates.py``; the Trotter splitting in ``trotter_step``).

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*``
against explicit Kronecker-product matrices, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import gates as _gates

gate_matrix = _gates.gate_matrix
ARITY = _gates.ARITY

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "statevec.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C core with gcc (plain -O2; OpenMP for the optional
    all-cores gate loop, single-threaded unless ``set_threads`` asks)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC,
                                   "-o", tmp, "-lm"])
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def set_threads(t: int) -> int:
    """Threads for gate application (1 = the plain single-threaded loop);
    returns the number in effect. Results do not depend on it."""
    return int(_load().orc_set_threads(int(t)))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_apply_matrix.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P]
            lib.orc_apply_matrix.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = ctypes.c_int
            lib.orc_probabilities.argtypes = [P, ctypes.c_int, P]
            lib.orc_norm2.argtypes = [P, ctypes.c_int]
            lib.orc_norm2.restype = ctypes.c_double
            lib.orc_pauli_expectation.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
            lib.orc_apply_diagonal_evolution.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P,
                                                         ctypes.c_double]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_state(psi: np.ndarray, n: int):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.shape != (1 << n,):
        raise ValueError("oracle state must be a contiguous complex128 vector of length 2^n")


# ---------------------------------------------------------------- states
def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def basis_state(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[int(x)] = 1.0
    return psi


def plus_state(n: int) -> np.ndarray:
    """|+>^n: every amplitude 2^{-n/2}."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


# ---------------------------------------------------------------- gates
def apply_matrix(psi: np.ndarray, n: int, targets, G: np.ndarray, controls=()) -> np.ndarray:
    """Eq. (1) in place for a dense matrix on ``targets`` with ``controls``."""
    _check_state(psi, n)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    c = np.ascontiguousarray(controls if len(controls) else [0], dtype=np.int32)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    k = len(t)
    if G.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the number of targets")
    if len(set(t.tolist()) | set(list(controls))) != k + len(controls):
        raise ValueError("targets and controls must be distinct")
    if any(q < 0 or q >= n for q in list(t) + list(controls)):
        raise ValueError("qubit out of range")
    rc = _load().orc_apply_matrix(_ptr(psi), n, k, _ptr(t), len(controls), _ptr(c), _ptr(G))
    if rc != 0:
        raise ValueError("orc_apply_matrix rejected its arguments")
    return psi


def apply_gate(psi: np.ndarray, n: int, gate) -> np.ndarray:
    G = gate_matrix(gate.kind, gate.params, gate.matrix)
    return apply_matrix(psi, n, gate.targets, G, gate.controls)


def apply_circuit(psi: np.ndarray, n: int, gates) -> np.ndarray:
    """Apply the gate queue in order (Sec. 2.3: the circuit is a queue of gates)."""
    for g in gates:
        apply_gate(psi, n, g)
    return psi


def run_circuit(n: int, gates, psi0: np.ndarray | None = None) -> np.ndarray:
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    return apply_circuit(psi, n, gates)


# ---------------------------------------------------------------- read-out
def probabilities(psi: np.ndarray, n: int) -> np.ndarray:
    _check_state(psi, n)
    p = np.empty(1 << n, dtype=np.float64)
    _load().orc_probabilities(_ptr(psi), n, _ptr(p))
    return p


def norm2(psi: np.ndarray, n: int) -> float:
    _check_state(psi, n)
    return float(_load().orc_norm2(_ptr(psi), n))


def _terms_arrays(terms):
    coeff = np.ascontiguousarray([float(t[0]) for t in terms] or [0.0], dtype=np.float64)
    xm = np.ascontiguousarray([int(t[1]) for t in terms] or [0], dtype=np.uint64)
    zm = np.ascontiguousarray([int(t[2]) for t in terms] or [0], dtype=np.uint64)
    return coeff, xm, zm


def expectation(psi: np.ndarray, n: int, terms) -> complex:
    """<psi|H|psi> for H = sum_t c_t P_t; ``terms`` holds (c, x_mask, z_mask)
    with bit q of a mask <-> qubit q (X: x only, Z: z only, Y: both)."""
    _check_state(psi, n)
    coeff, xm, zm = _terms_arrays(terms)
    re = ctypes.c_double()
    im = ctypes.c_double()
    _load().orc_pauli_expectation(_ptr(psi), n, len(terms), _ptr(coeff), _ptr(xm), _ptr(zm),
                                  ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def energy(n: int, gates, terms, psi0: np.ndarray | None = None) -> float:
    """E = Re <psi|H|psi> with psi the circuit's output state."""
    psi = run_circuit(n, gates, psi0)
    return expectation(psi, n, terms).real


# ---------------------------------------------------------------- Trotter
def split_hamiltonian(terms):
    """Split a Pauli sum into its diagonal part (Z strings, x_mask = 0) and its
    transverse part (single-qubit X terms). These are the two exactly
    exponentiable commuting families the Trotter step alternates between;
    any other term is rejected."""
    diag, xs = [], []
    for c, xm, zm in terms:
        xm, zm = int(xm), int(zm)
        if xm == 0:
            diag.append((float(c), 0, zm))
        elif zm == 0 and bin(xm).count("1") == 1:
            xs.append((float(c), xm, 0))
        else:
            raise ValueError("Trotter step supports Z-string and single-qubit X terms only")
    return diag, xs


def apply_diagonal_evolution(psi: np.ndarray, n: int, diag_terms, tau: float) -> np.ndarray:
    """psi <- exp(-i tau D) psi for a diagonal Pauli sum D."""
    _check_state(psi, n)
    coeff, _, zm = _terms_arrays(diag_terms)
    _load().orc_apply_diagonal_evolution(_ptr(psi), n, len(diag_terms), _ptr(coeff), _ptr(zm),
                                         float(tau))
    return psi


def trotter_step(psi: np.ndarray, n: int, h0_terms, h1_terms, s: float, dt: float) -> np.ndarray:
    """One second-order (Strang) Trotter step of H(s) = (1-s) H0 + s H1 (Eq. (4)).

    The paper maps exp(-i H dt) onto a circuit of few-qubit unitaries (Sec. 2.6);
    it does not print the splitting. Reading taken here: split H(s) = D(s) + X(s)
    into the diagonal Z-string part D and the transverse part X = sum_q a_q X_q
    (both exactly exponentiable), and apply
        exp(-i dt/2 D(s)) exp(-i dt X(s)) exp(-i dt/2 D(s)).
    exp(-i dt a_q X_q) is RX(2 dt a_q) with RX(th) = exp(-i th X / 2).
    """
    d0, x0 = split_hamiltonian(h0_terms)
    d1, x1 = split_hamiltonian(h1_terms)
    diag = [((1.0 - s) * c, 0, z) for c, _, z in d0] + [(s * c, 0, z) for c, _, z in d1]
    a = np.zeros(n)
    for c, xm, _ in x0:
        a[int(xm).bit_length() - 1] += (1.0 - s) * c
    for c, xm, _ in x1:
        a[int(xm).bit_length() - 1] += s * c
    apply_diagonal_evolution(psi, n, diag, dt / 2.0)
    for q in range(n):
        if a[q] != 0.0:
            apply_matrix(psi, n, (q,), gate_matrix("RX", (2.0 * dt * a[q],)))
    apply_diagonal_evolution(psi, n, diag, dt / 2.0)
    return psi


def adiabatic_evolve(psi: np.ndarray, n: int, h0_terms, h1_terms, T: float, dt: float,
                     steps: int | None = None) -> np.ndarray:
    """Adiabatic evolution under H(t) = (1 - s(t)) H0 + s(t) H1 with the linear
    schedule s = t/T (Sec. 2.6), K = round(T/dt) second-order Trotter steps;
    step k evaluates s at its midpoint (k + 1/2) dt / T, which keeps the
    time-dependent splitting second order. ``steps`` < K stops early."""
    K = int(round(T / dt))
    for k in range(K if steps is None else min(K, steps)):
        s = (k + 0.5) * dt / T
        trotter_step(psi, n, h0_terms, h1_terms, s, dt)
    return psi


# ---------------------------------------------------------------- gradients
PARAMETRIC = ("RX", "RY", "RZ", "U1", "CU1")


def gradient_parameter_shift(n: int, gates, terms, psi0: np.ndarray | None = None,
                             which=None) -> np.ndarray:
    """dE/dtheta_j for every single-parameter gate j (RX, RY, RZ, U1, CU1), in
    gate order, by the parameter-shift rule
        dE/dth = [E(th + pi/2) - E(th - pi/2)] / 2,
    exact for gates exp(-i th G) whose generator G has eigenvalues +-1/2 up to a
    constant shift (a global phase, which E does not see). ``which`` restricts the
    result to a subset of parameter indices (the rest are NaN)."""
    gates = list(gates)
    pidx = [i for i, g in enumerate(gates) if g.kind in PARAMETRIC]
    out = np.full(len(pidx), np.nan)
    sel = range(len(pidx)) if which is None else which
    for j in sel:
        i = pidx[j]
        g = gates[i]
        vals = []
        for sh in (+math.pi / 2, -math.pi / 2):
            gs = list(gates)
            gs[i] = g._replace(params=(g.params[0] + sh,) + tuple(g.params[1:]))
            vals.append(energy(n, gs, terms, psi0))
        out[j] = 0.5 * (vals[0] - vals[1])
    return out


def gradient_exact(n: int, gates, terms, psi0: np.ndarray | None = None) -> np.ndarray:
    """dE/dtheta_j for every single-parameter gate j (RX, RY, RZ, U1, CU1, with
    or without controls), in gate order, from the product rule:
        dE/dtheta_j = 2 Re <psi|H|d_j psi>,
        d_j psi = U_N .. U_{j+1} (dU_j/dtheta_j) U_{j-1} .. U_1 psi0,
    where dU_j/dtheta_j is the derivative of the gate matrix on the block whose
    controls are all 1 and zero elsewhere. Re <psi|H|chi> is taken by
    polarisation, (<psi+chi|H|psi+chi> - <psi-chi|H|psi-chi>) / 4, which holds
    for Hermitian H. Exact where the two-term shift rule is not (controlled
    rotations have three generator eigenvalues)."""
    gates = list(gates)
    psi = run_circuit(n, gates, psi0)
    out = []
    for j, g in enumerate(gates):
        if g.kind not in PARAMETRIC:
            continue
        phi = run_circuit(n, gates[:j], psi0)
        if g.controls:
            keep = np.ones(1 << n, dtype=bool)
            idx = np.arange(1 << n)
            for q in g.controls:
                keep &= ((idx >> (n - 1 - q)) & 1) == 1
            phi[~keep] = 0.0
        apply_matrix(phi, n, g.targets, _gates.generator_derivative(g.kind, g.params), g.controls)
        chi = apply_circuit(phi, n, gates[j + 1:])
        plus = expectation(np.ascontiguousarray(psi + chi), n, terms).real
        minus = expectation(np.ascontiguousarray(psi - chi), n, terms).real
        out.append(2.0 * (plus - minus) / 4.0)
    return np.array(out)


# ---------------------------------------------------------------- fusion
def fused_matrix(gates, qubits) -> np.ndarray:
    """Matrix of a gate sequence restricted to ``qubits`` (Sec. 2.4, "Gate
    fusion": the product U_m ... U_1 of the gates' matrices). Built column by
    column by running the gates on each basis state of the len(qubits)-qubit
    register, with qubits[0] as the most significant local bit."""
    qubits = list(qubits)
    m = len(qubits)
    pos = {q: i for i, q in enumerate(qubits)}
    local = []
    for g in gates:
        if any(q not in pos for q in tuple(g.targets) + tuple(g.controls)):
            raise ValueError("gate acts outside the fusion block")
        local.append(g._replace(targets=tuple(pos[q] for q in g.targets),
                                controls=tuple(pos[q] for q in g.controls)))
    U = np.zeros((1 << m, 1 << m), dtype=np.complex128)
    for col in range(1 << m):
        U[:, col] = run_circuit(m, local, basis_state(m, col))
    return U


# ---------------------------------------------------------------- measurements
def marginal_probabilities(psi: np.ndarray, n: int, qubits) -> np.ndarray:
    """Outcome probabilities of the qubit group ``qubits`` (Sec. 2.4,
    "Measurements": the outcome probability traced over the unmeasured
    qubits): out[y] = sum of |psi[x]|^2 over the x whose qubits[j] has the value
    of bit (m-1-j) of y (qubits[0] the most significant bit of y, as qubit 0 is
    of the basis index). The probability tensor, one axis per qubit (axis q =
    qubit q), is summed over the other axes and its remaining axes are put in
    the group's order."""
    _check_state(psi, n)
    qubits = [int(q) for q in qubits]
    if not qubits or len(set(qubits)) != len(qubits) or any(q < 0 or q >= n for q in qubits):
        raise ValueError("qubits must be distinct and in range")
    p = (np.abs(psi) ** 2).reshape((2,) * n)
    rest = tuple(q for q in range(n) if q not in qubits)
    marg = p.sum(axis=rest) if rest else p
    kept = [q for q in range(n) if q in qubits]  # axis order after the sum
    marg = np.transpose(marg, [kept.index(q) for q in qubits])
    return np.ascontiguousarray(marg).reshape(-1)


def sample(psi: np.ndarray, n: int, uniforms) -> np.ndarray:
    """Samples of the measurement of every qubit (Sec. 2.4, "Measurements";
    Sec. 3.3 samples the final state's distribution): for each u in [0, 1)
    the smallest basis index x with cdf(x) > u * cdf(2^n - 1), cdf the
    cumulative sum of |psi|^2 in index order (FP64). The uniforms are the
    caller's random numbers; the mapping from them is deterministic. For
    u < 1 the target u * total lies below the total, so such an x exists and
    has nonzero probability; where rounding puts the target at the total, the
    answer in exact arithmetic is the last outcome of nonzero probability."""
    _check_state(psi, n)
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    u = np.asarray(uniforms, dtype=np.float64)
    x = np.searchsorted(cdf, u * cdf[-1], side="right")
    nz = np.flatnonzero(p > 0)
    last = int(nz[-1]) if nz.size else (1 << n) - 1
    return np.where(x >= (1 << n), last, x).astype(np.uint64)
