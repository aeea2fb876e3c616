"""complex128 one-gate passes in double-float arithmetic (dense 1- and 2-qubit
gates, the default) and in FP64 (opts flag), through the C-ABI, against the
oracle (Eq. 1 in FP64).

Tolerance: complex128 max |delta amplitude| <= 1e-12, L2 <= 1e-11, as for
every complex128 result. A double-float gate rounds each input to 47
significant bits and each output to about 2^-46 of the terms' magnitude: some
1e-14 per gate relative to the amplitudes' scale, so 1e-12 holds over
hundreds of gates on an amplitude."""
import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

MX, L2 = 1e-12, 1e-11


def close(got, want):
    got = np.asarray(got, dtype=np.complex128).reshape(-1)
    want = np.asarray(want, dtype=np.complex128).reshape(-1)
    err = float(np.max(np.abs(got - want))) if got.size else 0.0
    assert err <= MX, f"max |delta| {err:.3e} > {MX:.0e}"
    assert float(np.linalg.norm(got - want)) <= L2


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 6, 11, 14])
def test_mixed_circuit_unfused(qs, n, fp64):
    gates = qi.random_mixed_circuit(n, 120, seed=3000 + n, max_controls=min(3, n - 1),
                                    max_unitary_k=min(2, n))
    psi0 = qi.random_state(n, 310 + n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype="c128").set(psi0).apply(gates, mode="unfused", fp64=fp64)
    close(st.get(), want)


def test_double_float_and_fp64_take_different_paths(qs):
    """The two arithmetics round differently: on 200 dense gates their results
    agree to the tolerance but not bit for bit (the flag reaches the kernel)."""
    n = 10
    gates = qi.random_mixed_circuit(n, 200, seed=77, max_controls=1, max_unitary_k=2,
                                    kinds=["U3", "H", "RX"])
    psi0 = qi.random_state(n, 78)
    a = qs.State(n, dtype="c128").set(psi0).apply(gates, mode="unfused").get()
    b = qs.State(n, dtype="c128").set(psi0).apply(gates, mode="unfused", fp64=True).get()
    close(a, b)
    assert not np.array_equal(a, b)


def test_random_layer_full_circuit_n22(qs):
    """The whole 20-layer random-layer circuit at n = 22 (650 gates: n U3 and
    n/2 or n/2 - 1 CZ per layer) from |0>, one gate per pass in double-float
    and in tiled passes, against the oracle."""
    n = 22
    gates = qi.random_layer_circuit(n, 20, seed=2)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype="c128")
    close(st.init_basis(0).apply(gates, mode="unfused").get(), want)
    close(st.init_basis(0).apply(gates, mode="tiled").get(), want)


def test_special_values(qs):
    """Exact zeros, signed zeros, powers of two, amplitudes at the bottom of
    the double-float range (below 2^-103 only the high float is kept, below
    2^-126 they flush to zero) and values whose low bits fill the whole
    significand: every output within the tolerance of the oracle, and H on
    every qubit twice (the identity) returns the state to within 1e-13."""
    n = 8
    r = qi.rng(91)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    psi[1] = -0.5 + 0.25j
    psi[2] = -0.0 + 0.0j
    psi[3] = np.nextafter(0.75, 1.0) + 1j * np.nextafter(-0.125, -1.0)
    psi[4:12] = (1e-32 - 3e-35j) * (1 + np.arange(8))
    psi[12:20] = 1e-40 + 1e-41j
    psi[20:] = r.normal(size=(1 << n) - 20) + 1j * r.normal(size=(1 << n) - 20)
    psi /= np.linalg.norm(psi)
    H = [qi.Gate("H", (q,)) for q in range(n)]
    gates = H + [qi.Gate("UNITARY", (1, 6), (), (), qi.random_unitary(2, r))] + H
    want = oracle.apply_circuit(psi.copy(), n, gates)
    got = qs.State(n, dtype="c128").set(psi).apply(gates, mode="unfused").get()
    close(got, want)
    hh = qs.State(n, dtype="c128").set(psi).apply(H + H, mode="unfused").get()
    assert float(np.max(np.abs(hh - psi))) <= 1e-13


def test_batch_and_controls(qs):
    n, B = 12, 3
    gates = qi.random_mixed_circuit(n, 90, seed=55, max_controls=3, max_unitary_k=2,
                                    kinds=["U3", "UNITARY", "CZ", "SWAP", "H", "RY"])
    psis = np.stack([qi.random_state(n, 560 + b) for b in range(B)])
    got = qs.State(n, batch=B, dtype="c128").set(psis).apply(gates, mode="unfused").get()
    for b in range(B):
        close(got[b], oracle.apply_circuit(psis[b].copy(), n, gates))


@pytest.mark.parametrize("n", [12, 13, 16])
def test_tiled_double_float_and_fp64(qs, n):
    """Tiled complex128 passes: the default double-float kernels and the FP64
    ones both match the oracle on a mixed circuit (controls, 2-qubit dense
    gates, swaps, diagonals inside and outside the tile), and round
    differently (the flag reaches the tiled kernels)."""
    gates = qi.random_mixed_circuit(n, 150, seed=700 + n, max_controls=2, max_unitary_k=2)
    psi0 = qi.random_state(n, 710 + n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    a = qs.State(n, dtype="c128").set(psi0).apply(gates, mode="tiled").get()
    b = qs.State(n, dtype="c128").set(psi0).apply(gates, mode="tiled", fp64=True).get()
    close(a, want)
    close(b, want)
    assert not np.array_equal(a, b)


def test_tiled_special_values(qs):
    """A tiled pass over a state holding exact zeros, powers of two, values at
    the bottom of the double-float range and full-significand values: the
    oracle's result within the tolerance, and a layer of H twice returns the
    state to within 1e-13."""
    n = 13
    r = qi.rng(93)
    psi = r.normal(size=1 << n) + 1j * r.normal(size=1 << n)
    psi[:64] = 0.0
    psi[64:80] = 0.5
    psi[80:96] = -0.25j
    psi[96:104] = 1e-35
    psi[104:112] = 1e-40 - 1e-39j
    psi[112:120] = np.nextafter(0.125, 1.0)
    psi /= np.linalg.norm(psi)
    gates = qi.random_layer_circuit(n, 3, seed=94)
    want = oracle.apply_circuit(psi.copy(), n, gates)
    close(qs.State(n, dtype="c128").set(psi).apply(gates, mode="tiled").get(), want)
    H = [qi.Gate("H", (q,)) for q in range(n)]
    hh = qs.State(n, dtype="c128").set(psi).apply(H + H, mode="tiled").get()
    assert float(np.max(np.abs(hh - psi))) <= 1e-13



@pytest.mark.parametrize("fp64", [False, True])
def test_tiled_per_member_angles(qs, fp64):
    """Tiled complex128 passes whose rotations take per-member angles (RX, RY
    as per-member rotations, RZ, U1 and CU1 as per-member diagonals), read
    from a double-float table by default and an FP64 one with the flag: every
    member against the oracle with its own angles."""
    import torch
    n, B = 13, 3
    r = qi.rng(97)
    gates, pidx = [], []
    P = 0
    for layer in range(3):
        for q in range(n):
            kind = ("RX", "RY", "RZ", "U1")[(q + layer) % 4]
            gates.append(qi.Gate(kind, (q,), (), (0.0,)))
            pidx.append(P)
            P += 1
        for q in range(layer % 2, n - 1, 2):
            gates.append(qi.Gate("CZ", (q, q + 1)))
            pidx.append(-1)
        gates.append(qi.Gate("CU1", (layer, n - 1 - layer), (), (0.0,)))
        pidx.append(P)
        P += 1
        gates.append(qi.Gate("U3", ((5 * layer) % n,), (), tuple(r.uniform(0, 6.28, 3))))
        pidx.append(-1)
    th = r.uniform(0.0, 2.0 * np.pi, size=(B, P))
    params = torch.tensor(th, dtype=torch.float64, device="cuda")
    psis = np.stack([qi.random_state(n, 980 + b) for b in range(B)])
    st = qs.State(n, batch=B, dtype="c128").set(psis)
    got = st.apply_batched(gates, pidx, params, mode="tiled", fp64=fp64).get()
    for b in range(B):
        gb = [g._replace(params=(float(th[b, pi]),)) if pi >= 0 else g for g, pi in zip(gates, pidx)]
        close(got[b], oracle.apply_circuit(psis[b].copy(), n, gb))
