"""Host-memory states (Sec. 2.5: one device reused for the pieces of a state
larger than its memory): amplitudes in pinned host memory, gates applied to
groups of chunks streamed through a small device budget, against the in-device
path (one-gate passes: the same arithmetic, so bit-identical) and the oracle
(complex128 max |delta| <= 1e-12; complex64 max <= 1e-5, L2 <= 1e-4)."""
import numpy as np
import pytest

import oracle
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


def budget(dtype, m):
    """Device bytes for two buffers of 2^m amplitudes."""
    return 2 * (1 << m) * (8 if dtype == "c64" else 16)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_unfused_matches_the_device_path_exactly(qs, dtype):
    n = 18
    gates = qi.random_mixed_circuit(n, 80, seed=300, max_controls=2, max_unitary_k=2)
    psi0 = qi.random_state(n, 301)
    hs = qs.HostState(n, dtype=dtype, device_bytes=budget(dtype, 12)).set(psi0)
    hs.apply(gates, mode="unfused")
    st = qs.State(n, dtype=dtype).set(psi0).apply(gates, mode="unfused")
    assert np.array_equal(hs.get(), st.get())


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["unfused", "auto"])
def test_against_oracle(qs, dtype, mode):
    n = 16
    gates = qi.random_layer_circuit(n, 6, seed=302) + qi.qft_circuit(n)[:40]
    psi0 = qi.random_state(n, 303)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    hs = qs.HostState(n, dtype=dtype, device_bytes=budget(dtype, 13)).set(psi0).apply(gates, mode=mode)
    close(hs.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_read_outs(qs, dtype):
    n = 20
    gates = qi.random_layer_circuit(n, 3, seed=304)
    hs = qs.HostState(n, dtype=dtype, device_bytes=budget(dtype, 14)).init_basis(0).apply(gates)
    st = qs.State(n, dtype=dtype).init_basis(0).apply(gates)
    mx = TOL[dtype][0]
    assert abs(hs.norm2()[0] - st.norm2()[0]) < 10 * mx
    np.testing.assert_allclose(hs.probabilities(), st.probabilities(), rtol=0, atol=mx)
    # Z strings anywhere, X on the low qubits (inside a device block of 2^14)
    terms = [(0.7, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)] + \
            [(0.3, 1 << q, 0) for q in range(n - 6, n)] + [(0.2, (1 << (n - 1)) | (1 << (n - 2)), 1 << 3)]
    scale = sum(abs(t[0]) for t in terms)
    assert abs(hs.expectation(terms)[0] - st.expectation(terms)[0]) < 2 * mx * scale * 10
    hs.init_plus()
    np.testing.assert_allclose(hs.probabilities(), np.full(1 << n, 2.0 ** -n), rtol=0, atol=1e-7)


def test_host_state_limits(qs):
    n = 16
    hs = qs.HostState(n, dtype="c64", device_bytes=budget("c64", 12)).init_basis(0)
    # three dense targets above the chunk bits (buffers of 2^12: 2 high bits per group)
    u = qi.random_unitary(3, qi.rng(5))
    with pytest.raises(qs.QsimError) as e:
        hs.apply([qi.Gate("UNITARY", (0, 1, 2), (), (), u)])
    assert e.value.status == 4
    with pytest.raises(qs.QsimError) as e:
        hs.expectation([(1.0, 1, 0)])                      # X on qubit 0: above the device block
    assert e.value.status == 4
    with pytest.raises(qs.QsimError) as e:
        hs.marginal_probabilities([0])
    assert e.value.status == 4
