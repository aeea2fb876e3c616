"""Tiled passes on kernels specialised for them (compiled at run time with
NVRTC): the same circuits as the generic-kernel parity tests, against the
oracle at the same tolerances (complex128 max |delta| <= 1e-12; complex64 max
<= 1e-5, L2 <= 1e-4), with the launch counters showing that the specialised
kernels ran and no compile failed."""
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
    qsim.jit_set_policy("sync")
    yield qsim
    qsim.jit_wait()
    qsim.jit_set_policy("tiered")


def specialised(qs, fn):
    """Run fn; return how many tiled launches used specialised kernels."""
    before = qs.jit_stats()
    fn()
    after = qs.jit_stats()
    assert after["failed"] == before["failed"], "a specialisation failed to compile or load"
    return after["specialised_launches"] - before["specialised_launches"]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [13, 16])
def test_random_layer_circuit(qs, dtype, n):
    gates = qi.random_layer_circuit(n, 6, seed=2)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype=dtype)
    assert specialised(qs, lambda: st.init_basis(0).apply(gates, mode="tiled")) > 0
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_mixed_gates_with_controls(qs, dtype):
    n = 14
    gates = qi.random_mixed_circuit(n, 60, seed=1014, max_controls=3, max_unitary_k=2)
    psi0 = qi.random_state(n, 91)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype=dtype).set(psi0)
    assert specialised(qs, lambda: st.apply(gates, mode="tiled")) > 0
    close(st.get(), want, dtype)


@pytest.mark.parametrize("dtype,n,batch", [("c64", 13, 3), ("c64", 14, 1), ("c128", 12, 3), ("c128", 13, 1)])
def test_tile_counts_odd_and_even(qs, dtype, n, batch):
    """Specialised kernels over odd and even numbers of tiles (one tile per
    member with three members, or two tiles of one member), with per-member
    states: every member against the oracle."""
    gates = qi.random_layer_circuit(n, 6, seed=40 + n)
    psis = np.stack([qi.random_state(n, 420 + b) for b in range(batch)])
    st = qs.State(n, batch=batch, dtype=dtype).set(psis if batch > 1 else psis[0])
    assert specialised(qs, lambda: st.apply(gates, mode="tiled")) > 0
    got = np.asarray(st.get()).reshape(batch, -1)
    for b in range(batch):
        close(got[b], oracle.apply_circuit(psis[b].copy(), n, gates), dtype)


def test_qft_closed_form(qs):
    n = 15
    x = 12345
    st = qs.State(n, dtype="c128")
    assert specialised(qs, lambda: st.init_basis(x).apply(qi.qft_circuit(n), mode="tiled")) > 0
    k = np.arange(1 << n)
    close(st.get(), np.exp(2j * np.pi * x * k / (1 << n)) / np.sqrt(1 << n), "c128")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_adjoint_gradient(qs, dtype):
    """The adjoint sweep's passes (gradient ops, per-member rotations) on
    specialised kernels, against the oracle's exact gradient."""
    import torch
    n, B = 12, 2
    th = qi.variational_params(B, 3, n, seed=5)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 1.0)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype=dtype)
    out = {}

    def run():
        out["e"], out["g"] = eng.run(torch.tensor(th.reshape(B, -1), device="cuda"))

    assert specialised(qs, run) > 0
    scale = sum(abs(t[0]) for t in terms)
    tol = 2e-11 * scale if dtype == "c128" else 2e-5 * scale
    g = out["g"].cpu().numpy()
    for b in range(B):
        want = oracle.gradient_exact(n, qi.variational_circuit(n, th[b]), terms)
        assert np.max(np.abs(g[b] - want)) < tol


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_trotter_steps(qs, dtype):
    n, T, dt, steps = 13, 1.0, 0.1, 3
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(8))
    want = oracle.adiabatic_evolve(oracle.plus_state(n), n, h0, h1, T, dt, steps=steps)
    st = qs.State(n, dtype=dtype)
    assert specialised(qs, lambda: st.init_plus().adiabatic_evolve(h0, h1, T, dt, steps=steps)) > 0
    close(st.get(), want, dtype)


def test_tiered_policy_switches_after_the_second_launch(qs):
    """Under the default policy a pass launched a second time is compiled in
    the background; after the compile, its launches are specialised and give
    the generic kernel's result within rounding."""
    n = 15
    gates = qi.random_layer_circuit(n, 4, seed=77)
    st = qs.State(n, dtype="c64")
    qs.jit_set_policy("tiered")
    try:
        assert specialised(qs, lambda: st.init_basis(0).apply(gates, mode="tiled")) == 0
        generic = st.get().copy()
        st.init_basis(0).apply(gates, mode="tiled")   # second launch: queued
        qs.jit_wait()
        assert specialised(qs, lambda: st.init_basis(0).apply(gates, mode="tiled")) > 0
        assert np.max(np.abs(st.get() - generic)) < 1e-6
    finally:
        qs.jit_set_policy("sync")


def test_values_compiled_in_for_a_repeated_pass(qs):
    """With QS_JIT_FOLD a pass launched twice with the same values gets a
    second kernel with its values compiled in; the third run uses it, and its
    result matches the oracle."""
    n = 14
    gates = qi.random_layer_circuit(n, 5, seed=81)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype="c64")
    qs.jit_set_policy("sync", fold=True)
    try:
        st.init_basis(0).apply(gates, mode="tiled")
        before = qs.jit_stats()["compiled"]
        st.init_basis(0).apply(gates, mode="tiled")   # second launch: folded kernels queued
        qs.jit_wait()
        assert qs.jit_stats()["compiled"] > before
        assert specialised(qs, lambda: st.init_basis(0).apply(gates, mode="tiled")) > 0
        close(st.get(), want, "c64")
    finally:
        qs.jit_set_policy("sync")
