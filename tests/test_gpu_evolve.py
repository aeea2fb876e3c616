"""Exact time evolution (Sec. 2.6: exp, rk4, rk45) and the schedule gradient
of the Trotterised adiabatic evolution (Sec. 4) on the GPU, through the C-ABI,
against the oracle.

Tolerances: states within the scope's bounds (complex128 max |delta| <= 1e-12,
L2 <= 1e-11; complex64 max <= 1e-5, L2 <= 1e-4). The energy and its schedule
derivatives are sums of K steps' bilinear read-outs <lambda|G|phi> with
||G|| <= sum|c|, each within 2 sum|c| times the state's L2 bound, so they are
checked at 3 K sum|c| times that bound (at least the state bound itself)."""
import numpy as np
import pytest

import oracle
from oracle import evolution as ev
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


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("solver", ["exp", "rk4", "rk45"])
@pytest.mark.parametrize("n", [1, 5, 10])
def test_solvers_match_oracle(qs, dtype, solver, n):
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(20 + n)) + qi.random_pauli_terms(n, 4, seed=n)
    T, dt = 0.6, 0.05
    psi0 = qi.random_state(n, 30 + n)
    want = ev.SOLVERS[solver](psi0, n, h0, h1, T, dt)
    st = qs.State(n, dtype=dtype).set(psi0).evolve(h0, h1, T, dt, solver=solver)
    close(st.get(), want, dtype)


def test_batch_members_and_partial_steps(qs):
    n, B = 6, 3
    h0 = qi.transverse_field_terms(n)
    h1 = qi.tfim_terms(n, 0.8)
    psis = np.stack([qi.random_state(n, 40 + b) for b in range(B)])
    st = qs.State(n, batch=B, dtype="c128").set(psis).evolve(h0, h1, 1.0, 0.1, solver="rk4", steps=4)
    got = st.get()
    for b in range(B):
        close(got[b], ev.evolve_rk4(psis[b], n, h0, h1, 1.0, 0.1, steps=4), "c128")


def test_solvers_agree_at_larger_n(qs):
    """n = 16 (beyond the dense oracle): a constant H evolved by the exp solver
    in one step and in ten agree, and the rk45 solution with 300 steps
    matches them; the norm stays 1."""
    n, T = 16, 0.3
    H = qi.tfim_terms(n, 1.1) + qi.random_pauli_terms(n, 6, seed=3)
    psi0 = qi.random_state(n, 50)
    a = qs.State(n, dtype="c128").set(psi0).evolve(H, H, T, T, solver="exp").get()
    b = qs.State(n, dtype="c128").set(psi0).evolve(H, H, T, T / 10, solver="exp").get()
    c = qs.State(n, dtype="c128").set(psi0).evolve(H, H, T, T / 300, solver="rk45").get()
    assert np.linalg.norm(a - b) < 1e-11
    assert np.linalg.norm(a - c) < 1e-10
    assert abs(np.linalg.norm(a) - 1.0) < 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_schedule_gradient_matches_oracle(qs, dtype):
    n, dt = 6, 0.12
    h0 = qi.transverse_field_terms(n) + [(0.4, 0, 0b000110)]
    h1 = qi.random_ising_terms(n, qi.rng(60))
    svals = list(np.linspace(0.05, 0.95, 8))
    psis = np.stack([oracle.plus_state(n), qi.random_state(n, 61)])
    st = qs.State(n, batch=2, dtype=dtype).set(psis)
    E, g, gdt = st.schedule_gradient(h0, h1, svals, dt)
    mx, l2 = TOL[dtype]
    scale = sum(abs(t[0]) for t in h0 + h1)
    tol = max(mx, 3 * len(svals) * scale * l2)
    final = st.get()
    for b in range(2):
        Ew, gw, gdtw = ev.schedule_gradient(n, h0, h1, svals, dt, psis[b])
        assert abs(E[b] - Ew) < tol
        assert np.max(np.abs(g[b] - gw)) < tol, np.max(np.abs(g[b] - gw))
        assert abs(gdt[b] - gdtw) < tol
        psi = psis[b].copy()
        for s in svals:
            oracle.trotter_step(psi, n, h0, h1, s, dt)
        close(final[b], psi, dtype)


def test_schedule_gradient_at_a_tiled_width(qs):
    """n = 14 (the X layers run as tiled passes): the gradient of one step's
    schedule value against central differences of the GPU energy."""
    n, dt = 14, 0.1
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(62))
    svals = [0.2, 0.45, 0.7, 0.9]
    psi0 = oracle.plus_state(n)
    E, g, gdt = qs.State(n, dtype="c128").set(psi0).schedule_gradient(h0, h1, svals, dt)
    h = 1e-5
    for k in (0, 2):
        sp, sm = list(svals), list(svals)
        sp[k] += h
        sm[k] -= h
        ep = qs.State(n, dtype="c128").set(psi0).schedule_gradient(h0, h1, sp, dt)[0][0]
        em = qs.State(n, dtype="c128").set(psi0).schedule_gradient(h0, h1, sm, dt)[0][0]
        assert abs((ep - em) / (2 * h) - g[0, k]) < 1e-6


def test_evolution_argument_errors(qs):
    st = qs.State(4, dtype="c64").init_plus()
    a1, n1 = qs.marshal_terms([(1.0, 0, 1)])
    assert qs.load().qs_evolve(st.handle, None, 0, a1, n1, 1.0, 0.1, -1, 7) == 1   # unknown solver
    assert qs.load().qs_evolve(st.handle, None, 0, a1, n1, -1.0, 0.1, -1, 0) == 1  # T <= 0
    with pytest.raises(qs.QsimError) as e:
        st.schedule_gradient(qi.transverse_field_terms(4), [(1.0, 0b11, 0b11)], [0.5], 0.1)
    assert e.value.status == 4                                                      # not a Trotter term
