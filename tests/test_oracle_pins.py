"""Pins of the oracle against things other than itself.

Each test checks the oracle against an independent construction: explicit
2^n x 2^n Kronecker-product operators, matrix exponentials (scipy), closed forms
(QFT of a basis state, GHZ, Grover amplitudes), invariants (unitarity, norm), a
hand-derived worked example, and convergence laws (Trotter infidelity ~ dt^4).
The mistakes these are chosen to catch: a wrong qubit/bit order, a transposed
or conjugated matrix, a dropped control, a wrong sign or factor in a rotation,
a wrong Y phase in a Pauli string, a wrong Trotter splitting order.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
from oracle import gates as og
from paper_2009_01845_gb300 import inputs as qi

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Yp = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def kron_all(factors):
    out = np.array([[1.0 + 0j]])
    for f in factors:                 # qubit 0 first: it is the most significant bit
        out = np.kron(out, f)
    return out


def full_operator(n, G, targets, controls):
    """Independent 2^n x 2^n construction of a (controlled) gate:
    sum_{r,c} G[r,c] (x)_q op_q with op = |r_j><c_j| on target j, |1><1| on
    controls, I elsewhere; plus (I - prod_controls |1><1|) on the rest."""
    k = len(targets)
    d = 2 ** n
    M = np.zeros((d, d), dtype=complex)
    for r in range(2 ** k):
        for c in range(2 ** k):
            if G[r, c] == 0:
                continue
            fac = []
            for q in range(n):
                if q in targets:
                    j = targets.index(q)
                    rb = (r >> (k - 1 - j)) & 1
                    cb = (c >> (k - 1 - j)) & 1
                    e = np.zeros((2, 2), dtype=complex)
                    e[rb, cb] = 1
                    fac.append(e)
                elif q in controls:
                    fac.append(P1)
                else:
                    fac.append(I2)
            M += G[r, c] * kron_all(fac)
    if controls:
        proj = kron_all([P1 if q in controls else I2 for q in range(n)])
        M += np.eye(d) - proj
    return M


def pauli_dense(n, terms):
    d = 2 ** n
    H = np.zeros((d, d), dtype=complex)
    for c, xm, zm in terms:
        fac = []
        for q in range(n):
            xb, zb = (xm >> q) & 1, (zm >> q) & 1
            fac.append(Yp if (xb and zb) else X if xb else Z if zb else I2)
        H += c * kron_all(fac)
    return H


# ------------------------------------------------------------------ gate matrices
ANGLES = [0.0, 0.3, 1.1, math.pi / 2, 2.7, 4.9, 2 * math.pi - 0.01]


@pytest.mark.parametrize("kind", list(og.ARITY))
def test_every_named_gate_is_unitary(kind):
    r = qi.rng(11)
    for _ in range(5):
        G = og.gate_matrix(kind, r.uniform(0, 2 * math.pi, size=og.ARITY[kind][1]))
        assert np.allclose(G @ G.conj().T, np.eye(G.shape[0]), atol=1e-14)


@pytest.mark.parametrize("th", ANGLES)
def test_rotations_are_matrix_exponentials(th):
    for kind, P in (("RX", X), ("RY", Yp), ("RZ", Z)):
        assert np.allclose(og.gate_matrix(kind, (th,)), scipy.linalg.expm(-0.5j * th * P),
                           atol=1e-14)


@pytest.mark.parametrize("th", ANGLES)
def test_u3_special_cases(th):
    # U3(th,0,0) = RY(th); U3(0,0,l) = U1(l); U1(l) = e^{il/2} RZ(l)
    assert np.allclose(og.gate_matrix("U3", (th, 0, 0)), og.gate_matrix("RY", (th,)), atol=1e-15)
    assert np.allclose(og.gate_matrix("U3", (0, 0, th)), og.gate_matrix("U1", (th,)), atol=1e-15)
    assert np.allclose(og.gate_matrix("U1", (th,)),
                       np.exp(0.5j * th) * scipy.linalg.expm(-0.5j * th * Z), atol=1e-14)
    # U2(ph, l) = U3(pi/2, ph, l); U3(pi/2, 0, pi) = H = (X + Z)/sqrt 2
    assert np.allclose(og.gate_matrix("U2", (th, 0.4)), og.gate_matrix("U3", (math.pi / 2, th, 0.4)))
    assert np.allclose(og.gate_matrix("U3", (math.pi / 2, 0, math.pi)), (X + Z) / math.sqrt(2),
                       atol=1e-15)


def test_discrete_gate_relations():
    g = og.gate_matrix
    assert np.allclose(g("H"), (X + Z) / math.sqrt(2))
    assert np.allclose(g("Y"), 1j * X @ Z)
    assert np.allclose(g("S") @ g("S"), Z)
    assert np.allclose(g("T") @ g("T"), g("S"))
    assert np.allclose(g("SDG"), g("S").conj().T)
    assert np.allclose(g("TDG"), g("T").conj().T)
    assert np.allclose(g("CU1", (math.pi,)), g("CZ"))
    assert np.allclose(g("CZ"), full_operator(2, Z, [1], [0]))
    # SWAP = CNOT(0->1) CNOT(1->0) CNOT(0->1)
    c01 = full_operator(2, X, [1], [0])
    c10 = full_operator(2, X, [0], [1])
    assert np.allclose(g("SWAP"), c01 @ c10 @ c01)


@pytest.mark.parametrize("kind", ["RX", "RY", "RZ", "U1", "CU1"])
def test_generator_derivative_matches_finite_difference(kind):
    th, h = 0.77, 1e-6
    fd = (og.gate_matrix(kind, (th + h,)) - og.gate_matrix(kind, (th - h,))) / (2 * h)
    assert np.allclose(og.generator_derivative(kind, (th,)), fd, atol=1e-9)


# ------------------------------------------------------------------ Eq. (1) vs Kronecker
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_apply_matches_kronecker_operator(n):
    gates = qi.random_mixed_circuit(n, 40, seed=100 + n, max_controls=min(2, n - 1),
                                    max_unitary_k=min(3, n))
    psi = qi.random_state(n, seed=7 + n)
    ref = psi.copy()
    for g in gates:
        G = og.gate_matrix(g.kind, g.params, g.matrix)
        if G.shape[0] > 2 ** n:
            continue
        ref = full_operator(n, G, list(g.targets), list(g.controls)) @ ref
        oracle.apply_gate(psi, n, g)
        assert np.allclose(psi, ref, atol=1e-13), g


def test_apply_five_target_unitary_with_controls_matches_kronecker():
    n = 8
    r = qi.rng(3)
    U = qi.random_unitary(5, r)
    targets, controls = [6, 1, 4, 0, 7], [3, 5]
    psi = qi.random_state(n, 9)
    ref = full_operator(n, U, targets, controls) @ psi
    oracle.apply_matrix(psi, n, targets, U, controls)
    assert np.allclose(psi, ref, atol=1e-13)


def test_qubit_zero_is_most_significant_bit():
    n = 5
    psi = oracle.run_circuit(n, [qi.Gate("X", (0,))])
    p = oracle.probabilities(psi, n)
    assert p[1 << (n - 1)] == 1.0 and p.sum() == 1.0
    psi = oracle.run_circuit(n, [qi.Gate("X", (n - 1,))])
    assert oracle.probabilities(psi, n)[1] == 1.0


def test_oracle_rejects_bad_arguments():
    psi = oracle.zero_state(3)
    with pytest.raises(ValueError):
        oracle.apply_matrix(psi, 3, [0, 0], np.eye(4))
    with pytest.raises(ValueError):
        oracle.apply_matrix(psi, 3, [3], np.eye(2))
    with pytest.raises(ValueError):
        oracle.apply_matrix(psi, 3, [1], np.eye(2), controls=[1])


# ------------------------------------------------------------------ worked example and closed forms
def test_paper_sec2_3_example_golden():
    """The three-qubit example circuit printed in Sec. 2.3 (H(0), X(1),
    RX(0, pi/6) on |000>), against the hand-derived amplitudes stored in
    tests/golden/sec2_3_example.txt."""
    path = os.path.join(os.path.dirname(__file__), "golden", "sec2_3_example.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    expect = np.zeros(8, dtype=complex)
    for idx, re, im in rows:
        expect[int(idx)] = float(re) + 1j * float(im)
    gates = [qi.Gate("H", (0,)), qi.Gate("X", (1,)), qi.Gate("RX", (0,), (), (math.pi / 6,))]
    psi = oracle.run_circuit(3, gates)
    assert np.allclose(psi, expect, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_qft_closed_form_every_input(n):
    N = 2 ** n
    k = np.arange(N)
    for x in range(N):
        psi = oracle.run_circuit(n, qi.qft_circuit(n), oracle.basis_state(n, x))
        want = np.exp(2j * np.pi * x * k / N) / math.sqrt(N)
        assert np.max(np.abs(psi - want)) < 1e-13


def test_qft_closed_form_seeded_input_n14():
    n = 14
    x = qi.qft_input(n, seed=1)
    psi = oracle.run_circuit(n, qi.qft_circuit(n), oracle.basis_state(n, x))
    k = np.arange(2 ** n)
    want = np.exp(2j * np.pi * ((x * k) % 2 ** n) / 2 ** n) / 2 ** (n / 2)
    assert np.max(np.abs(psi - want)) < 1e-12
    assert len(qi.qft_circuit(18)) == 180


@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz(n):
    psi = oracle.run_circuit(n, qi.ghz_circuit(n))
    want = np.zeros(2 ** n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15


@pytest.mark.parametrize("n,marked,iters", [(5, [19], 2), (6, [3, 40], 3), (7, [0, 77, 100], 4)])
def test_grover_amplitudes(n, marked, iters):
    """Each marked amplitude is (-1)^k sin((2k+1) th)/sqrt(M) with sin th =
    sqrt(M/N); the (-1)^k comes from the diffusion built as
    H X [MCZ] X H = I - 2|s><s| (the negative of the textbook reflection)."""
    N, M = 2 ** n, len(marked)
    th = math.asin(math.sqrt(M / N))
    psi = oracle.run_circuit(n, qi.grover_circuit(n, marked, iters))
    want_m = (-1) ** iters * math.sin((2 * iters + 1) * th) / math.sqrt(M)
    want_u = (-1) ** iters * math.cos((2 * iters + 1) * th) / math.sqrt(N - M)
    for x in range(N):
        w = want_m if x in marked else want_u
        assert abs(psi[x] - w) < 1e-12


def test_norm_preserved_random_layer():
    n = 12
    psi = oracle.run_circuit(n, qi.random_layer_circuit(n, layers=6, seed=2))
    assert abs(1.0 - oracle.norm2(psi, n)) < 1e-13
    assert abs(oracle.probabilities(psi, n).sum() - 1.0) < 1e-13


def test_random_layer_gate_counts():
    assert len(qi.random_layer_circuit(32, 20)) == 640 + 310
    assert len(qi.random_layer_circuit(33, 20)) == 660 + 320


# ------------------------------------------------------------------ expectation values
@pytest.mark.parametrize("n", [1, 3, 6])
def test_pauli_expectation_matches_dense(n):
    terms = qi.random_pauli_terms(n, 12, seed=50 + n)
    psi = qi.random_state(n, 60 + n)
    H = pauli_dense(n, terms)
    want = psi.conj() @ H @ psi
    got = oracle.expectation(psi, n, terms)
    assert abs(got - want) < 1e-13
    assert abs(got.imag) < 1e-13         # H is Hermitian


def test_pauli_expectation_closed_forms():
    n = 6
    plus = oracle.plus_state(n)
    for q in range(n):
        assert abs(oracle.expectation(plus, n, [(1.0, 1 << q, 0)]) - 1) < 1e-14
        assert abs(oracle.expectation(plus, n, [(1.0, 0, 1 << q)])) < 1e-14
    zero = oracle.zero_state(n)
    assert abs(oracle.expectation(zero, n, [(1.0, 0, 1 << 2)]) - 1) < 1e-15
    one = oracle.basis_state(n, 1 << (n - 1 - 2))          # qubit 2 set
    assert abs(oracle.expectation(one, n, [(1.0, 0, 1 << 2)]) + 1) < 1e-15
    ghz = oracle.run_circuit(n, qi.ghz_circuit(n))
    assert abs(oracle.expectation(ghz, n, [(1.0, 0, (1 << 1) | (1 << 4))]) - 1) < 1e-14
    assert abs(oracle.expectation(ghz, n, [(1.0, (1 << n) - 1, 0)]) - 1) < 1e-14
    # <+i| Y |+i> = 1 with |+i> = S H |0>
    yi = oracle.run_circuit(1, [qi.Gate("H", (0,)), qi.Gate("S", (0,))])
    assert abs(oracle.expectation(yi, 1, [(1.0, 1, 1)]) - 1) < 1e-15


def test_tfim_terms_dense():
    n = 5
    H = pauli_dense(n, qi.tfim_terms(n, 1.0))
    want = np.zeros_like(H)
    for i in range(n - 1):
        want -= kron_all([Z if q in (i, i + 1) else I2 for q in range(n)])
    for i in range(n):
        want -= kron_all([X if q == i else I2 for q in range(n)])
    assert np.allclose(H, want)


# ------------------------------------------------------------------ Trotter
def _h_dense(n, terms):
    return pauli_dense(n, terms)


def test_trotter_step_no_field_is_exact_rx_product():
    n = 5
    h0 = qi.transverse_field_terms(n)
    psi = qi.random_state(n, 1)
    s, dt = 0.0, 0.37
    want = scipy.linalg.expm(-1j * dt * _h_dense(n, h0)) @ psi
    got = oracle.trotter_step(psi.copy(), n, h0, [], s, dt)
    assert np.max(np.abs(got - want)) < 1e-13


def test_trotter_step_diagonal_only_is_exact_phase():
    n = 5
    h1 = qi.random_ising_terms(n, qi.rng(4))
    psi = qi.random_state(n, 2)
    s, dt = 1.0, 0.41
    want = scipy.linalg.expm(-1j * dt * _h_dense(n, h1)) @ psi
    got = oracle.trotter_step(psi.copy(), n, qi.transverse_field_terms(n), h1, s, dt)
    assert np.max(np.abs(got - want)) < 1e-13


def test_trotter_step_is_strang_product_of_dense_exponentials():
    n = 5
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(5)) + [(0.6, 1 << 2, 0)]   # H1 with a field term too
    psi = qi.random_state(n, 3)
    s, dt = 0.3, 0.2
    H0, H1 = _h_dense(n, h0), _h_dense(n, h1)
    D = (1 - s) * 0 + s * _h_dense(n, h1[:-1])
    Xp = (1 - s) * H0 + s * _h_dense(n, h1[-1:])
    half = scipy.linalg.expm(-0.5j * dt * D)
    want = half @ scipy.linalg.expm(-1j * dt * Xp) @ half @ psi
    got = oracle.trotter_step(psi.copy(), n, h0, h1, s, dt)
    assert np.max(np.abs(got - want)) < 1e-13
    # and one step is close to the exact exp(-i dt H(s)) to O(dt^3)
    exact = scipy.linalg.expm(-1j * dt * ((1 - s) * H0 + s * H1)) @ psi
    assert np.max(np.abs(got - exact)) < 5 * dt ** 3


def _exact_adiabatic(n, h0, h1, T, psi0):
    H0, H1 = _h_dense(n, h0), _h_dense(n, h1)

    def rhs(t, y):
        s = t / T
        return -1j * (((1 - s) * H0 + s * H1) @ y)

    sol = scipy.integrate.solve_ivp(rhs, (0, T), psi0.astype(complex), method="DOP853",
                                    rtol=1e-12, atol=1e-13)
    return sol.y[:, -1]


def test_trotter_infidelity_scales_as_dt4():
    """Sec. 3.5: the overlap with the exact evolution approaches 1 as dt^4
    (TFIM, linear schedule, T = 1). Here n = 6 and the exact evolution is a
    high-order adaptive ODE solve of the Schroedinger equation."""
    n, T = 6, 1.0
    h0 = qi.transverse_field_terms(n)
    h1 = qi.tfim_terms(n, 1.0)
    psi0 = oracle.plus_state(n)
    exact = _exact_adiabatic(n, h0, h1, T, psi0)
    dts = [0.1, 0.05, 0.025, 0.0125]
    inf = []
    for dt in dts:
        psi = oracle.adiabatic_evolve(psi0.copy(), n, h0, h1, T, dt)
        inf.append(1 - abs(np.vdot(exact, psi)) ** 2)
    slope = np.polyfit(np.log(dts), np.log(inf), 1)[0]
    assert 3.7 < slope < 4.3, (inf, slope)


# ------------------------------------------------------------------ gradients
def test_parameter_shift_single_qubit_closed_form():
    # E(th) = <Z> after RY(th)|0> = cos th, dE/dth = -sin th
    for th in ANGLES:
        g = oracle.gradient_parameter_shift(1, [qi.Gate("RY", (0,), (), (th,))], [(1.0, 0, 1)])
        assert abs(g[0] + math.sin(th)) < 1e-14


def test_parameter_shift_matches_finite_differences():
    n = 5
    r = qi.rng(8)
    gates = []
    for l in range(3):
        for q in range(n):
            kind = ["RX", "RY", "RZ", "U1"][int(r.integers(0, 4))]
            gates.append(qi.Gate(kind, (q,), (), (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("CU1", (l % n, (l + 2) % n), (), (float(r.uniform(0, 6.28)),)))
        gates += [qi.Gate("H", (q,)) for q in range(0, n, 2)]
        gates += [qi.Gate("CZ", (i, i + 1)) for i in range(n - 1)]
    terms = qi.tfim_terms(n, 0.7) + qi.random_pauli_terms(n, 3, 9)
    g = oracle.gradient_parameter_shift(n, gates, terms)
    pidx = [i for i, gt in enumerate(gates) if gt.kind in oracle.PARAMETRIC]
    h = 1e-4
    for j, i in enumerate(pidx):
        gp = list(gates)
        gm = list(gates)
        gp[i] = gates[i]._replace(params=(gates[i].params[0] + h,))
        gm[i] = gates[i]._replace(params=(gates[i].params[0] - h,))
        fd = (oracle.energy(n, gp, terms) - oracle.energy(n, gm, terms)) / (2 * h)
        assert abs(fd - g[j]) < 1e-7


def test_exact_gradient_matches_shift_rule_and_finite_differences():
    """gradient_exact equals the parameter-shift rule on uncontrolled rotations
    and central finite differences everywhere, including controlled rotations
    (where the two-term shift rule is not exact)."""
    n = 5
    r = qi.rng(21)
    gates = []
    for l in range(3):
        for q in range(n):
            kind = ["RX", "RY", "RZ", "U1"][int(r.integers(0, 4))]
            ctrl = (int((q + 2) % n),) if l == 1 else ()
            gates.append(qi.Gate(kind, (q,), ctrl, (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("CU1", (l, l + 2), ((l + 4) % n,) if l == 2 else (), (float(r.uniform(0, 6.28)),)))
        gates += [qi.Gate("H", (q,)) for q in range(0, n, 2)] + [qi.Gate("CZ", (i, i + 1)) for i in range(n - 1)]
    terms = qi.tfim_terms(n, 0.8) + qi.random_pauli_terms(n, 3, 5)
    g = oracle.gradient_exact(n, gates, terms)
    ps = oracle.gradient_parameter_shift(n, gates, terms)
    pidx = [i for i, gt in enumerate(gates) if gt.kind in oracle.PARAMETRIC]
    h = 1e-4
    for j, i in enumerate(pidx):
        gp, gm = list(gates), list(gates)
        gp[i] = gates[i]._replace(params=(gates[i].params[0] + h,))
        gm[i] = gates[i]._replace(params=(gates[i].params[0] - h,))
        fd = (oracle.energy(n, gp, terms) - oracle.energy(n, gm, terms)) / (2 * h)
        assert abs(g[j] - fd) < 1e-7
        if not gates[i].controls:
            assert abs(g[j] - ps[j]) < 1e-12
    assert any(abs(g[j] - ps[j]) > 1e-3 for j, i in enumerate(pidx) if gates[i].controls)


# ------------------------------------------------------------------ fusion
def test_fused_matrix_is_product_of_kronecker_operators():
    r = qi.rng(12)
    qubits = [4, 1, 7, 2, 5]                   # any order: qubits[0] is the local MSB
    gates = []
    for _ in range(25):
        kind = ["U3", "CZ", "RY", "CU1", "H", "SWAP"][int(r.integers(0, 6))]
        k, npar = qi.KINDS[kind]
        qs = [qubits[i] for i in r.permutation(5)[:k]]
        gates.append(qi.Gate(kind, tuple(qs), (), tuple(r.uniform(0, 6.28, size=npar))))
    U = oracle.fused_matrix(gates, qubits)
    want = np.eye(32, dtype=complex)
    for g in gates:
        G = og.gate_matrix(g.kind, g.params)
        want = full_operator(5, G, [qubits.index(q) for q in g.targets], []) @ want
    assert np.allclose(U, want, atol=1e-13)
    # applying the fused block equals applying the gates one by one
    n = 9
    psi = qi.random_state(n, 4)
    a = oracle.apply_circuit(psi.copy(), n, gates)
    b = oracle.apply_matrix(psi.copy(), n, qubits, U)
    assert np.max(np.abs(a - b)) < 1e-13


def test_gate_loop_threads_do_not_change_the_result():
    """The CPU baseline's all-cores run splits the gate loop over index groups
    across threads; every group is one thread's, so the state is bit-identical
    to the single-threaded loop."""
    n = 12
    gates = qi.random_mixed_circuit(n, 40, seed=71, max_controls=2, max_unitary_k=3)
    psi0 = qi.random_state(n, 72)
    one = oracle.apply_circuit(psi0.copy(), n, gates)
    used = oracle.set_threads(4)
    try:
        many = oracle.apply_circuit(psi0.copy(), n, gates)
    finally:
        oracle.set_threads(1)
    assert used >= 1
    assert np.array_equal(one, many)
