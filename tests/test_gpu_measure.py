"""GPU parity of the measurement calls (Sec. 2.4, "Measurements"; Sec. 3.3):
marginal probabilities of qubit groups and samples for given uniforms, through
the C-ABI, against the oracle on the same amplitudes.

Tolerances: marginals max |delta| <= 1e-12 (complex128) and 1e-6 (complex64,
|psi|^2 summed in FP32 runs before FP64); samples identical, except where the
target u * total lies within 1e-9 of a cumulative-probability boundary (the
prefix sums' rounding orders differ), where the sample must still be valid
to that tolerance."""
import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

MTOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


def groups_for(n, r):
    gs = [[0], [n - 1], [n - 1, 0]]
    for m in (2, 3, 5, min(n, 8), min(n, 12)):
        gs.append([int(q) for q in r.permutation(n)[:m]])
    return [g for g in gs if len(g) <= n]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 12, 17])
def test_marginals_match_oracle(qs, dtype, n):
    st = qs.State(n, dtype=dtype).set(qi.random_state(n, 30 + n))
    psi = np.ascontiguousarray(st.get().astype(np.complex128))  # the amplitudes the device holds
    for g in groups_for(n, qi.rng(n)):
        got = st.marginal_probabilities(g)
        want = oracle.marginal_probabilities(psi, n, g)
        assert np.max(np.abs(got - want)) <= MTOL[dtype], g


def test_marginals_per_batch_member(qs):
    n, B = 14, 3
    st = qs.State(n, batch=B, dtype="c128")
    psis = [qi.random_state(n, 70 + b) for b in range(B)]
    st.set(np.stack(psis))
    got = st.marginal_probabilities([3, 13, 0])
    for b in range(B):
        np.testing.assert_allclose(got[b], oracle.marginal_probabilities(psis[b], n, [3, 13, 0]), rtol=0, atol=1e-12)


def check_samples(psi, n, u, got):
    want = oracle.sample(psi, n, u)
    bad = np.flatnonzero(got != want)
    if bad.size == 0:
        return
    cdf = np.cumsum(np.abs(psi) ** 2)
    target = u[bad] * cdf[-1]
    xg = got[bad].astype(np.int64)
    below = np.where(xg > 0, cdf[np.maximum(xg - 1, 0)], 0.0)
    assert np.all(below <= target + 1e-9) and np.all(cdf[xg] > target - 1e-9), (bad[:5], got[bad[:5]], want[bad[:5]])
    assert bad.size <= 2


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 13, 20])
def test_samples_match_oracle(qs, dtype, n):
    psi0 = qi.random_state(n, 50 + n)
    psi0[: min(4, 1 << n) // 2] = 0  # zero-probability outcomes are never drawn
    st = qs.State(n, dtype=dtype).set(psi0)
    psi = np.ascontiguousarray(st.get().astype(np.complex128))
    u = qi.rng(60 + n).uniform(size=20000)
    got = st.sample(u)
    check_samples(psi, n, u, got)
    assert not np.any(np.abs(psi[got.astype(np.int64)]) == 0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_samples_with_zero_probability_tail(qs, dtype):
    """The last blocks of 4096 amplitudes have zero probability and the
    uniforms come close to 1: every sample is an outcome of nonzero
    probability (the last one for u -> 1). Device uniforms outside [0, 1) are
    clamped (below 0 -> the first such outcome; 1, above 1 or NaN -> the last);
    host uniforms outside [0, 1) are rejected."""
    import torch
    n = 14
    psi0 = qi.random_state(n, 91)
    psi0[:5] = 0
    psi0[2 * 4096 + 123:] = 0
    psi0 /= np.linalg.norm(psi0)
    st = qs.State(n, dtype=dtype).set(psi0)
    psi = np.ascontiguousarray(st.get().astype(np.complex128))
    nz = np.flatnonzero(np.abs(psi) > 0)
    u = np.array([np.nextafter(1.0, 0.0), 1.0 - 1e-12, 1.0 - 1e-9, 0.0, 0.5])
    got = st.sample(u)
    check_samples(psi, n, u, got)
    assert np.all(np.abs(psi[got.astype(np.int64)]) > 0)
    assert int(got[0]) == nz[-1] and int(got[3]) == nz[0]
    ud = torch.tensor([-0.5, 1.0, 1.5, float("nan"), np.nextafter(1.0, 0.0)], dtype=torch.float64, device="cuda")
    dev = st.sample(ud).cpu().numpy()
    assert list(dev[:4]) == [nz[0], nz[-1], nz[-1], nz[-1]] and dev[4] == nz[-1]
    for bad in (-0.5, 1.0, float("nan")):
        with pytest.raises(qs.QsimError):
            st.sample(np.array([0.5, bad]))


def test_marginals_full_size_ghz_and_basis(qs):
    """n = 28 complex64 (long per-thread runs, capped parts): a basis state's
    group marginal is one-hot at the group's bits of x, and GHZ's is 1/2 at
    all-zeros and all-ones, for groups with index bits below and above bit 8."""
    n = 28
    groups = [[n - 1 - b for b in (0, 3, 8, 9, 20, 27)], [n - 1 - b for b in range(2, 14)], [n - 1 - 8],
              [n - 1 - b for b in (27, 7, 8)]]
    st = qs.State(n, dtype="c64")
    x = int(qi.rng(33).integers(0, 1 << n))
    st.init_basis(x)
    for g in groups:
        got = st.marginal_probabilities(g)
        y = 0
        for q in g:
            y = (y << 1) | ((x >> (n - 1 - q)) & 1)
        want = np.zeros(1 << len(g))
        want[y] = 1.0
        assert np.max(np.abs(got - want)) < 1e-6, g
    ghz = [qi.Gate("H", (0,))] + [qi.Gate("X", (q,), (q - 1,)) for q in range(1, n)]
    st.init_basis(0).apply(ghz)
    for g in groups:
        got = st.marginal_probabilities(g)
        want = np.zeros(1 << len(g))
        want[0] = want[-1] = 0.5
        assert np.max(np.abs(got - want)) < 1e-6, g


def test_samples_device_tensors_equal_host(qs):
    import torch
    n = 16
    st = qs.State(n, dtype="c64").set(qi.random_state(n, 5))
    u = qi.rng(6).uniform(size=5000)
    host = st.sample(u)
    dev = st.sample(torch.tensor(u, device="cuda"))
    np.testing.assert_array_equal(dev.cpu().numpy().astype(np.uint64), host)


def test_measurement_argument_errors(qs):
    st = qs.State(6, dtype="c64").init_basis(0)
    for bad in ([], [0, 0], [6], [-1], list(range(6)) + [0]):
        with pytest.raises(Exception):
            st.marginal_probabilities(bad)
    with pytest.raises(Exception):
        st.sample([0.5], member=1)
    assert st.sample([]).size == 0


def test_full_size_uniform_superposition(qs):
    """|+>^n at n = 32, complex64 (the Sec. 3.3 sampling benchmark: H on every
    qubit, then measure): cdf(x) = (x + 1) / 2^n, so each sample is
    floor(u 2^n) for u away from a boundary, and every group's marginal is
    uniform."""
    n = 32
    st = qs.State(n, dtype="c64").init_plus()
    k = qi.rng(12).integers(0, 1 << n, size=4096)
    u = (k + 0.5) / float(1 << n)
    np.testing.assert_array_equal(st.sample(u).astype(np.int64), k)
    for g in ([0, 31, 7], list(range(20, 32))):
        got = st.marginal_probabilities(g)
        assert np.max(np.abs(got - 1.0 / (1 << len(g)))) < 1e-6
