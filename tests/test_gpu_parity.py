"""GPU parity: the CUDA path, called through the C-ABI, against the CPU oracle
on the same seeded inputs, element by element.

Tolerances (stated once): complex128 max |delta amplitude| <= 1e-12;
complex64 max |delta| <= 1e-5 and L2 <= 1e-4; indices and probabilities'
index mapping exact.
"""
import math

import numpy as np
import pytest

import circuit_utils
import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-12, 1e-11), "c64": (1e-5, 1e-4)}
MODES = ["unfused", "tiled", "auto"]


def close(got, want, dtype, scale=1.0):
    got = np.asarray(got, dtype=np.complex128).reshape(-1)
    want = np.asarray(want, dtype=np.complex128).reshape(-1)
    mx, l2 = TOL[dtype]
    err = np.max(np.abs(got - want)) if got.size else 0.0
    assert err <= mx * scale, f"max |delta| {err:.3e} > {mx * scale:.1e}"
    assert np.linalg.norm(got - want) <= l2 * scale


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


# ------------------------------------------------------------------ gate application
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14])
def test_random_mixed_circuit(qs, dtype, mode, n):
    gates = qi.random_mixed_circuit(n, 60, seed=1000 + n, max_controls=min(3, n - 1),
                                    max_unitary_k=min(5, n))
    psi0 = qi.random_state(n, 77 + n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype=dtype).set(psi0)
    st.apply(gates, mode=mode)
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", MODES)
def test_every_target_position_and_controls(qs, dtype, mode):
    """1- and 2-qubit gates on every qubit (inside a 128-bit vector, intra-warp,
    inter-warp and high bits), with and without controls."""
    n = 13
    r = qi.rng(5)
    gates = []
    for q in range(n):
        gates.append(qi.Gate("U3", (q,), (), tuple(r.uniform(0, 6.28, 3))))
        other = int((q + 5) % n)
        gates.append(qi.Gate("U3", (q,), (other,), tuple(r.uniform(0, 6.28, 3))))
        gates.append(qi.Gate("UNITARY", (q, (q + 1) % n), (), (), qi.random_unitary(2, r)))
        gates.append(qi.Gate("CU1", (q, (q + 3) % n), (), (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("RZ", (q,), (), (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("SWAP", (q, (q + 7) % n)))
    psi0 = qi.random_state(n, 3)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype=dtype).set(psi0).apply(gates, mode=mode)
    close(st.get(), want, dtype)


@pytest.mark.parametrize("mode", MODES)
def test_qft_n18_c128(qs, mode):
    """QFT on n = 18 qubits of the seeded basis state: against the oracle and the
    closed form 2^{-n/2} exp(2 pi i x k / 2^n)."""
    n = 18
    x = qi.qft_input(n, seed=1)
    gates = qi.qft_circuit(n)
    st = qs.State(n, dtype="c128").init_basis(x).apply(gates, mode=mode)
    got = st.get()
    want = oracle.run_circuit(n, gates, oracle.basis_state(n, x))
    close(got, want, "c128")
    k = np.arange(2 ** n)
    closed = np.exp(2j * np.pi * ((x * k) % 2 ** n) / 2 ** n) / 2 ** (n / 2)
    close(got, closed, "c128")
    p = st.probabilities()
    assert np.max(np.abs(p - oracle.probabilities(want, n))) < 1e-15


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_outcome_indexing_exact(qs, dtype):
    n = 9
    for q in range(n):
        st = qs.State(n, dtype=dtype).init_basis(0).apply([qi.Gate("X", (q,))])
        p = st.probabilities()
        assert p[1 << (n - 1 - q)] == 1.0 and p.sum() == 1.0
    st = qs.State(n, dtype=dtype).init_basis(0b101100111)
    assert np.argmax(st.probabilities()) == 0b101100111


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ghz_and_grover(qs, dtype):
    n = 10
    st = qs.State(n, dtype=dtype).init_basis(0).apply(qi.ghz_circuit(n))
    want = np.zeros(2 ** n, complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    close(st.get(), want, dtype)
    marked, it = [5, 700], 6
    gates = qi.grover_circuit(n, marked, it)
    st = qs.State(n, dtype=dtype).init_basis(0).apply(gates)
    close(st.get(), oracle.run_circuit(n, gates), dtype)


# ------------------------------------------------------------------ read-outs
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 4, 12, 17])
def test_probabilities_norm_expectation(qs, dtype, n):
    psi = qi.random_state(n, 200 + n)
    st = qs.State(n, dtype=dtype).set(psi)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    p = st.probabilities()
    np.testing.assert_allclose(p, oracle.probabilities(ref, n), rtol=0, atol=1e-15)
    assert abs(st.norm2()[0] - oracle.norm2(ref, n)) < 1e-13
    terms = qi.random_pauli_terms(n, 40, seed=n) + qi.tfim_terms(n, 0.9)
    got = st.expectation(terms)[0]
    want = oracle.expectation(ref, n, terms)
    tol = 1e-12 if dtype == "c128" else 2e-5
    assert abs(got - want) < tol * max(1.0, sum(abs(t[0]) for t in terms))


# ------------------------------------------------------------------ Trotter
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_trotter_step(qs, dtype):
    n = 9
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(3)) + [(0.4, 1 << 3, 0)]
    psi = qi.random_state(n, 5)
    want = oracle.trotter_step(psi.copy(), n, h0, h1, 0.37, 0.05)
    st = qs.State(n, dtype=dtype).set(psi).trotter_step(h0, h1, 0.37, 0.05)
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adiabatic_evolution(qs, dtype):
    n, T, dt = 10, 1.0, 0.05
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(8))
    want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt)
    st = qs.State(n, dtype=dtype).init_plus().adiabatic_evolve(h0, h1, T, dt)
    close(st.get(), want, dtype)


def test_trotter_rejects_unsupported_terms(qs):
    st = qs.State(4, dtype="c128").init_basis(0)
    with pytest.raises(qs.QsimError) as e:
        st.trotter_step([(1.0, 0b11, 0)], [], 0.5, 0.1)
    assert e.value.status == 4


# ------------------------------------------------------------------ batches
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batched_parameters(qs, dtype):
    import torch
    n, L, B = 7, 3, 5
    th = qi.variational_params(B, L, n, seed=4)
    tmpl = qi.variational_circuit(n, th[0])
    pidx = []
    c = 0
    for g in tmpl:
        pidx.append(c if g.kind == "RY" else -1)
        c += g.kind == "RY"
    params = torch.tensor(th.reshape(B, -1), dtype=torch.float64, device="cuda")
    st = qs.State(n, batch=B, dtype=dtype).init_basis(0).apply_batched(tmpl, pidx, params)
    got = st.get()
    for b in range(B):
        want = oracle.run_circuit(n, qi.variational_circuit(n, th[b]))
        close(got[b], want, dtype)
    e = st.expectation(qi.tfim_terms(n))
    for b in range(B):
        want = oracle.energy(n, qi.variational_circuit(n, th[b]), qi.tfim_terms(n))
        assert abs(e[b].real - want) < (1e-12 if dtype == "c128" else 1e-5)


def test_batch_members_equal_solo_runs_bit_exact(qs):
    n, B = 9, 4
    gates = qi.random_mixed_circuit(n, 40, seed=9, max_controls=2)
    psis = np.stack([qi.random_state(n, 300 + b) for b in range(B)])
    st = qs.State(n, batch=B, dtype="c64").set(psis).apply(gates)
    got = st.get()
    for b in range(B):
        solo = qs.State(n, dtype="c64").set(psis[b]).apply(gates).get()
        assert np.array_equal(got[b], solo)


# ------------------------------------------------------------------ errors
def test_invalid_gates_leave_state_unchanged(qs):
    n = 6
    psi = qi.random_state(n, 1)
    st = qs.State(n, dtype="c128").set(psi)
    bad = [
        [qi.Gate("H", (6,))],                       # out of range
        [qi.Gate("CZ", (2, 2))],                    # repeated target
        [qi.Gate("X", (1,), (1,))],                 # control == target
        [qi.Gate("H", (0,)), qi.Gate("RY", (-1,), (), (0.3,))],
        [qi.Gate("UNITARY", (0, 1, 2, 3, 4, 5), (), (), np.eye(64))],
    ]
    for g in bad:
        with pytest.raises(qs.QsimError) as e:
            st.apply(g)
        assert e.value.status == 1
    assert np.array_equal(st.get(), psi)


def test_empty_gate_list_and_tiny_states(qs):
    for n in (1, 2):
        psi = qi.random_state(n, n)
        st = qs.State(n, dtype="c128").set(psi).apply([])
        assert np.array_equal(st.get(), psi)
        gates = qi.random_mixed_circuit(n, 20, seed=n, max_controls=n - 1, max_unitary_k=n)
        st.apply(gates, mode="auto")
        close(st.get(), oracle.apply_circuit(psi.copy(), n, gates), "c128")


# ------------------------------------------------------------------ tiled passes
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [12, 13, 14, 16, 19])
def test_tiled_random_layer_matches_oracle(qs, dtype, n):
    gates = qi.random_layer_circuit(n, layers=8, seed=20 + n)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype=dtype).init_basis(0).apply(gates, mode="tiled")
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [13, 15, 18])
def test_tiled_mixed_gates_with_controls_matches_oracle(qs, dtype, n):
    """Every gate kind, controls on lane/register/warp/outside bits, diagonal
    gates on bits inside and outside the tile, 2-qubit dense gates and SWAPs."""
    gates = qi.random_mixed_circuit(n, 150, seed=500 + n, max_controls=3, max_unitary_k=2)
    psi0 = qi.random_state(n, 40 + n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype=dtype).set(psi0).apply(gates, mode="tiled")
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [13, 16])
def test_tiled_near_swap_rotations_matches_oracle(qs, dtype, n):
    """Rotations closer to a swap than to the identity, whose swap the tiled
    pass keeps in a register frame, followed in the same stages by sign flips
    on two and three register bits, controlled phases and further rotations."""
    gates = circuit_utils.near_swap_circuit(n, 6, seed=n)
    psi0 = qi.random_state(n, 90 + n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype=dtype).set(psi0).apply(gates, mode="tiled")
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tiled_batch_of_states(qs, dtype):
    n, B = 14, 3
    gates = qi.random_mixed_circuit(n, 80, seed=71, max_controls=2, max_unitary_k=2)
    psis = np.stack([qi.random_state(n, 90 + b) for b in range(B)])
    st = qs.State(n, batch=B, dtype=dtype).set(psis).apply(gates, mode="tiled")
    got = st.get()
    for b in range(B):
        close(got[b], oracle.apply_circuit(psis[b].copy(), n, gates), dtype)


def test_largest_batch_read_outs(qs):
    """batch = 65535, the largest a handle accepts (the member is a grid
    dimension): norm, probabilities, expectation and group marginals of every
    member against the oracle's definitions; 65536 is rejected."""
    n, batch = 1, 65535
    r = qi.rng(23)
    psis = r.normal(size=(batch, 2)) + 1j * r.normal(size=(batch, 2))
    psis /= np.linalg.norm(psis, axis=1, keepdims=True)
    st = qs.State(n, batch=batch, dtype="c128").set(psis)
    p = np.abs(psis) ** 2
    np.testing.assert_allclose(st.norm2(), p.sum(axis=1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(st.probabilities(), p, rtol=0, atol=1e-15)
    np.testing.assert_allclose(st.marginal_probabilities([0]), p, rtol=0, atol=1e-15)
    terms = [(0.7, 1, 0), (-0.4, 0, 1), (0.25, 1, 1)]
    e = st.expectation(terms)
    for b in range(0, batch, 4099):
        assert abs(e[b] - oracle.expectation(np.ascontiguousarray(psis[b]), n, terms)) < 1e-12
    with pytest.raises(qs.QsimError) as ex:
        qs.State(n, batch=batch + 1, dtype="c128")
    assert ex.value.status == 1


def test_tile_width_option(qs):
    """The tile width is the kernels' own: 0 or that width are accepted, any
    other is QS_ERR_UNSUPPORTED and leaves the state unchanged."""
    n = 13
    gates = qi.random_layer_circuit(n, 2, seed=95)
    want = oracle.run_circuit(n, gates)
    for dtype, k in (("c128", 12), ("c64", 13)):
        st = qs.State(n, dtype=dtype).init_basis(0).apply(gates, mode="tiled", tile_qubits=k)
        assert np.max(np.abs(st.get() - want)) < (1e-12 if dtype == "c128" else 1e-5)
        st.init_basis(0)
        with pytest.raises(qs.QsimError) as e:
            st.apply(gates, mode="tiled", tile_qubits=k - 1)
        assert e.value.status == 4
        assert st.get()[0] == 1.0
