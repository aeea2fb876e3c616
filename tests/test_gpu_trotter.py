"""Trotterised adiabatic evolution (Sec. 2.6) on the tiled path: Ising phase
ops fused with the RX layers, against the oracle's step-by-step evolution."""
import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

# the scope's bounds for every result: complex128 max |delta amplitude| <= 1e-12
# (L2 <= 1e-11); complex64 max <= 1e-5 and L2 <= 1e-4
TOL = {"c128": (1e-12, 1e-11), "c64": (1e-5, 1e-4)}


def close(got, want, dtype):
    got = np.asarray(got, dtype=np.complex128).reshape(-1)
    want = np.asarray(want, dtype=np.complex128).reshape(-1)
    mx, l2 = TOL[dtype]
    err = float(np.max(np.abs(got - want)))
    assert err <= mx, f"max |delta| {err:.3e} > {mx:.0e}"
    l2e = float(np.linalg.norm(got - want))
    assert l2e <= l2, f"L2 {l2e:.3e} > {l2:.0e}"


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


def tile_n(dtype):
    return 13 if dtype == "c64" else 12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_trotter_step_tiled(qs, dtype):
    n = tile_n(dtype) + 1
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(3)) + [(0.4, 1 << 3, 0), (0.25, 0, 0)]
    psi = qi.random_state(n, 5)
    want = oracle.trotter_step(psi.copy(), n, h0, h1, 0.37, 0.05)
    st = qs.State(n, dtype=dtype).set(psi).trotter_step(h0, h1, 0.37, 0.05)
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adiabatic_evolution_tiled(qs, dtype):
    n, T, dt = tile_n(dtype), 1.0, 0.05
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(8))
    want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt)
    st = qs.State(n, dtype=dtype).init_plus().adiabatic_evolve(h0, h1, T, dt)
    close(st.get(), want, dtype)


def test_tfim_example_of_sec2_6(qs):
    """The paper's example: H0 = -sum X, H1 = TFIM (field terms in H1 too),
    linear schedule; tiled evolution against the oracle in both precisions."""
    n, T, dt = 12, 3.0, 0.1
    h0 = qi.transverse_field_terms(n)
    h1 = qi.tfim_terms(n, 1.0)
    want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt)
    for dtype in ("c128", "c64"):
        st = qs.State(n, dtype=dtype).init_plus().adiabatic_evolve(h0, h1, T, dt)
        close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adiabatic_batch_own_hamiltonians(qs, dtype):
    n, B, T, dt = tile_n(dtype) + 1, 3, 0.5, 0.05
    r = qi.rng(44)
    h0 = qi.transverse_field_terms(n)
    h1s = [qi.random_ising_terms(n, r) for _ in range(B)]
    st = qs.State(n, batch=B, dtype=dtype).init_plus().adiabatic_evolve_batch(h0, h1s, T, dt)
    got = st.get()
    for b in range(B):
        want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1s[b], T, dt)
        close(got[b], want, dtype)


def test_three_body_terms_use_the_general_path(qs):
    n = 13
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(2)) + [(0.3, 0, 0b1011)]
    psi = qi.random_state(n, 6)
    want = oracle.trotter_step(psi.copy(), n, h0, h1, 0.6, 0.1)
    st = qs.State(n, dtype="c128").set(psi).trotter_step(h0, h1, 0.6, 0.1)
    close(st.get(), want, "c128")
    with pytest.raises(qs.QsimError) as e:
        qs.State(n, batch=1, dtype="c128").init_plus().adiabatic_evolve_batch(h0, [h1], 1.0, 0.1)
    assert e.value.status == 4


def test_config5_smallest_instance_sampled_steps(qs):
    """The adiabatic batch workload's first n = 16 instance (seed 5), 50 of its
    1000 steps, against the oracle, in both precisions."""
    inst = [x for x in qi.adiabatic_instances(64, seed=5) if x[0] == 16]
    assert inst, "seed 5 draws at least one n = 16 instance"
    n, h0, h1 = inst[0]
    T, dt, steps = 10.0, 0.01, 50
    want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt, steps=steps)
    for dtype in ("c128", "c64"):
        st = qs.State(n, dtype=dtype).init_plus().adiabatic_evolve(h0, h1, T, dt, steps=steps)
        close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_uneven_widths_in_one_call(qs, dtype):
    """Instances of several widths (one handle per width, two members where the
    width repeats) evolved in one qs_adiabatic_run_batch call, 24 steps (three
    chunks of the round-robin enqueue), each member against the oracle."""
    widths = [12, 13, 14, 16] if dtype == "c128" else [13, 14, 16]
    T, dt = 1.2, 0.05
    r = qi.rng(91)
    states, h0s, h1s, members = [], [], [], []
    for i, n in enumerate(widths):
        B = 2 if i % 2 == 0 else 1
        st = qs.State(n, batch=B, dtype=dtype).init_plus()
        h0 = qi.transverse_field_terms(n)
        states.append(st)
        h0s.append(h0)
        for _ in range(B):
            h1 = qi.random_ising_terms(n, r)
            h1s.append(h1)
            members.append((st, n, h0, h1))
    qs.adiabatic_run_batch(states, h0s, h1s, T, dt)
    got = {id(st): st.get().reshape(st.batch, -1) for st in states}
    seen = {}
    for st, n, h0, h1 in members:
        b = seen.get(id(st), 0)
        seen[id(st)] = b + 1
        want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt)
        close(got[id(st)][b], want, dtype)


def test_uneven_widths_argument_errors(qs):
    a = qs.State(13, dtype="c64").init_plus()
    b = qs.State(14, dtype="c128").init_plus()
    with pytest.raises(qs.QsimError) as e:
        qs.adiabatic_run_batch([a, b], [qi.transverse_field_terms(13), qi.transverse_field_terms(14)],
                               [qi.random_ising_terms(13, qi.rng(1)), qi.random_ising_terms(14, qi.rng(2))],
                               1.0, 0.1)
    assert e.value.status == 1
    with pytest.raises(qs.QsimError) as e:
        qs.adiabatic_run_batch([a, a], [qi.transverse_field_terms(13)] * 2,
                               [qi.random_ising_terms(13, qi.rng(1))] * 2, 1.0, 0.1)
    assert e.value.status == 1
