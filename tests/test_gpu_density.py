"""Density matrices and noise channels (Sec. 2.4, "Density matrices and noise")
on the GPU, through the C-ABI, against the density-matrix oracle: every entry of
rho within the state tolerances (complex128 max |delta| <= 1e-12, L2 <= 1e-11;
complex64 max <= 1e-5, L2 <= 1e-4), read-outs within the same bounds scaled by
the Hamiltonian's sum of |coefficients|."""
import numpy as np
import pytest

import oracle
from oracle import density as od
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-12, 1e-11), "c64": (1e-5, 1e-4)}


def close(got, want, dtype):
    got = np.asarray(got, dtype=np.complex128).reshape(-1)
    want = np.asarray(want, dtype=np.complex128).reshape(-1)
    mx, l2 = TOL[dtype]
    err = float(np.max(np.abs(got - want)))
    assert err <= mx, f"max |delta| {err:.3e} > {mx:.0e}"
    assert float(np.linalg.norm(got - want)) <= l2


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


def noisy_program(n, seed):
    """Alternating gate blocks and channels (one- and two-qubit)."""
    r = qi.rng(seed)
    prog = []
    for blk in range(3):
        prog.append(("gates", qi.random_mixed_circuit(n, 12, seed=seed * 10 + blk, max_controls=min(2, n - 1),
                                                      max_unitary_k=min(2, n))))
        q = [int(v) for v in r.permutation(n)[:2]]
        chans = [([q[0]], od.kraus_depolarizing(0.1 + 0.1 * blk)),
                 ([q[-1]], od.kraus_amplitude_damping(0.3)),
                 ([q[0]], od.kraus_phase_damping(0.2))]
        if n >= 2:
            chans.append(([q[1], q[0]], od.kraus_unitary_mixture([0.25, 0.75], [qi.random_unitary(2, r),
                                                                                 qi.random_unitary(2, r)])))
        prog.append(("channels", chans))
    return prog


def run_oracle(rho, n, prog):
    for kind, items in prog:
        if kind == "gates":
            rho = od.apply_circuit(rho, n, items)
        else:
            for targets, kraus in items:
                rho = od.apply_channel(rho, n, targets, kraus)
    return rho


def run_gpu(dm, prog, mode):
    for kind, items in prog:
        if kind == "gates":
            dm.apply(items, mode=mode)
        else:
            dm.apply_channels(items, mode=mode)
    return dm


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["unfused", "auto"])
@pytest.mark.parametrize("n", [1, 3, 7])
def test_noisy_circuit_matches_oracle(qs, dtype, mode, n):
    prog = noisy_program(n, 7 + n)
    psi0 = qi.random_state(n, 3 + n)
    want = run_oracle(od.from_state(psi0), n, prog)
    dm = run_gpu(qs.DensityMatrix(n, dtype=dtype).init_pure(psi0), prog, mode)
    close(dm.get(), want, dtype)
    # read-outs, bounded through the entries' L2 error l2 = ||delta rho||_F:
    # diagonal entries by mx; the trace by sqrt(2^n) l2; the purity by
    # 2 l2 + l2^2; |Tr(delta rho H)| <= l2 ||H||_F <= l2 sum|c| 2^(n/2)
    mx, l2 = TOL[dtype]
    np.testing.assert_allclose(dm.probabilities(), od.probabilities(want), rtol=0, atol=mx)
    assert abs(dm.trace()[0] - 1.0) <= l2 * 2 ** (n / 2) + 1e-15
    assert abs(dm.purity()[0] - np.sum(np.abs(want) ** 2)) <= 3 * l2
    terms = qi.random_pauli_terms(n, 10, seed=n) + qi.tfim_terms(n, 0.8)
    scale = sum(abs(t[0]) for t in terms)
    e = dm.expectation(terms)[0]
    assert abs(e - od.expectation(want, n, terms)) <= l2 * scale * 2 ** (n / 2)


def test_basis_plus_and_batch_members(qs):
    n = 4
    dm = qs.DensityMatrix(n, batch=2, dtype="c128")
    dm.init_basis(5)
    got = dm.get()
    for b in range(2):
        np.testing.assert_array_equal(got[b], od.basis(n, 5))
    dm.init_plus()
    np.testing.assert_allclose(dm.get()[1], np.full((16, 16), 1 / 16), atol=1e-16)
    psis = np.stack([qi.random_state(n, 60), qi.random_state(n, 61)])
    dm.init_pure(psis)
    gates = qi.random_layer_circuit(n, 3, seed=62)
    dm.apply(gates)
    dm.apply_channels([([1], od.kraus_depolarizing(0.3))])
    got = dm.get()
    for b in range(2):
        want = od.apply_channel(od.apply_circuit(od.from_state(psis[b]), n, gates), n, [1], od.kraus_depolarizing(0.3))
        close(got[b], want, "c128")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_pure_state_at_larger_n_follows_the_state_vector_path(qs, dtype):
    """n = 11 (a 22-qubit vector, tiled passes): with no channel, rho stays
    |psi><psi| for the state-vector path's psi on the same device."""
    n = 11
    gates = qi.random_layer_circuit(n, 8, seed=63)
    psi0 = qi.random_state(n, 64)
    st = qs.State(n, dtype="c128").set(psi0).apply(gates)
    psi = st.get()
    dm = qs.DensityMatrix(n, dtype=dtype).init_pure(psi0).apply(gates)
    close(dm.get(), np.outer(psi, psi.conj()), dtype)


def test_density_argument_errors(qs):
    st = qs.State(3, dtype="c64").init_basis(0)
    with pytest.raises(qs.QsimError) as e:
        qs.DensityMatrix.apply_channels(st, [([0], od.kraus_depolarizing(0.1))])
    assert e.value.status == 1
    dm = qs.DensityMatrix(3, dtype="c64").init_basis(0)
    with pytest.raises(qs.QsimError) as e:
        dm.apply_channels([([0], [np.eye(2) * 0.9])])       # not trace preserving
    assert e.value.status == 1
    with pytest.raises(qs.QsimError) as e:
        dm.apply_channels([([0, 0], od.kraus_unitary_mixture([1.0], [np.eye(4)]))])
    assert e.value.status == 1
    with pytest.raises(qs.QsimError) as e:
        dm.marginal_probabilities([0])
    assert e.value.status == 4
    with pytest.raises(qs.QsimError) as e:
        dm.apply([qi.Gate("H", (3,))])                      # qubit >= n
    assert e.value.status == 1
