"""Adjoint gradients (qs_energy_gradient) against the oracle's parameter-shift
gradients, finite differences, and themselves across modes and checkpoints."""
import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


def mixed_param_circuit(n, layers, seed):
    """Rotations of every parametrised kind (some controlled) between fixed
    gates; angles are placeholders (the batch's table supplies them)."""
    r = qi.rng(seed)
    gates = []
    for l in range(layers):
        for q in range(n):
            kind = ["RX", "RY", "RZ", "U1"][int(r.integers(0, 4))]
            ctrl = (int((q + 3) % n),) if r.uniform() < 0.2 else ()
            gates.append(qi.Gate(kind, (q,), ctrl, (0.0,)))
        gates.append(qi.Gate("CU1", (l % n, (l + 2) % n), (), (0.0,)))
        gates += [qi.Gate("H", (q,)) for q in range(0, n, 3)]
        gates += [qi.Gate("CZ", (i, i + 1)) for i in range(l % 2, n - 1, 2)]
        gates.append(qi.Gate("U3", ((l + 1) % n,), (), tuple(r.uniform(0, 6.28, 3))))
        a = n - 1 - l % 3
        gates.append(qi.Gate("SWAP", (a, (a + 2) % n)))
    return gates


def with_angles(gates, pidx, theta):
    return [g._replace(params=(float(theta[p]),)) if p >= 0 else g for g, p in zip(gates, pidx)]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [5, 12, 13])
def test_adjoint_matches_parameter_shift(qs, dtype, n):
    import torch
    B = 3
    gates = mixed_param_circuit(n, 3, seed=n)
    pidx, P = qs.param_indices(gates)
    theta = qi.rng(100 + n).uniform(0, 2 * np.pi, size=(B, P))
    terms = qi.tfim_terms(n, 0.7) + qi.random_pauli_terms(n, 4, seed=n)
    eng = qs.EnergyGradient(n, B, gates, pidx, terms, dtype=dtype)
    e, g = eng.run(torch.tensor(theta, device="cuda"))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    # energies and gradients are bilinear in the state: with ||H|| <= sum |c|
    # and the amplitude bounds (L2 <= 1e-11 complex128, <= 1e-4 complex64) their
    # error is at most 2 ||H|| ||delta psi||: 2e-11 sum|c| (complex128); the
    # complex64 check is tighter than its bound (2e-5 against 2e-4)
    scale = sum(abs(t[0]) for t in terms)
    tol = 2e-11 * scale if dtype == "c128" else 2e-5 * scale
    for b in range(B):
        circ = with_angles(gates, pidx, theta[b])
        assert abs(e[b] - oracle.energy(n, circ, terms)) < tol
        want = oracle.gradient_exact(n, circ, terms)
        assert np.max(np.abs(g[b] - want)) < tol, np.max(np.abs(g[b] - want))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_variational_n10_parameter_shift_and_finite_differences(qs, dtype):
    """The variational ansatz of Sec. 3.2 with the TFIM energy (n = 10, 10
    layers, 100 angles): adjoint gradient against the exact parameter-shift
    rule and central finite differences (step 1e-3) of the GPU energies."""
    import torch
    n, L, B = 10, 10, 4
    th = qi.variational_params(B, L, n, seed=4)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 1.0)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype=dtype)
    params = torch.tensor(th.reshape(B, -1), device="cuda")
    e, g = eng.run(params)
    g = g.cpu().numpy()
    tol_ps = 1e-10 if dtype == "c128" else 2e-4
    for b in (0, B - 1):
        want = oracle.gradient_parameter_shift(n, qi.variational_circuit(n, th[b]), terms)
        assert np.max(np.abs(g[b] - want)) < tol_ps
    h = 1e-3
    cols = [0, 17, 55, 99]
    for c in cols:
        dp = torch.zeros_like(params)
        dp[:, c] = h
        ep, _ = eng.run(params + dp, mode="forward")
        em, _ = eng.run(params - dp, mode="forward")
        fd = ((ep - em) / (2 * h)).cpu().numpy()
        assert np.max(np.abs(fd - g[:, c])) < (1e-6 if dtype == "c128" else 2e-3)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_forward_then_sweep_equals_full_and_checkpoints(qs, dtype):
    import torch
    n, B = 12, 2
    gates = mixed_param_circuit(n, 4, seed=3)
    pidx, P = qs.param_indices(gates)
    params = torch.tensor(qi.rng(9).uniform(0, 6.28, size=(B, P)), device="cuda")
    terms = qi.tfim_terms(n, 1.3)
    eng = qs.EnergyGradient(n, B, gates, pidx, terms, dtype=dtype)
    e_full, g_full = eng.run(params)
    e_fw, _ = eng.run(params, mode="forward")
    _, g_sw = eng.run(params, mode="sweep")
    assert torch.equal(e_full, e_fw)
    assert torch.equal(g_full, g_sw)
    e_ck, g_ck = eng.run(params, ckpt_every=17)
    tol = 1e-11 if dtype == "c128" else 1e-4
    assert float((e_ck - e_full).abs().max()) < tol
    assert float((g_ck - g_full).abs().max()) < tol


def test_autograd_function(qs):
    import torch
    n, B = 12, 2
    th = qi.variational_params(B, 3, n, seed=5)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 1.0)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype="c128")
    params = torch.tensor(th.reshape(B, -1), device="cuda", requires_grad=True)
    E = qs.energy_function().apply(params, eng)
    (E * torch.tensor([1.0, -2.0], device="cuda", dtype=torch.float64)).sum().backward()
    _, g = eng.run(params.detach())
    assert torch.allclose(params.grad[0], g[0], atol=1e-12)
    assert torch.allclose(params.grad[1], -2.0 * g[1], atol=1e-12)


def test_autograd_two_forwards_before_backward(qs):
    """(f(p1) + f(p2)).backward() on one engine: the second forward overwrote
    the work buffer, so the first backward must not sweep it as its own."""
    import torch
    n, B = 12, 2
    th = qi.variational_params(2 * B, 3, n, seed=6)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 1.0)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype="c128")
    p1 = torch.tensor(th[:B].reshape(B, -1), device="cuda", requires_grad=True)
    p2 = torch.tensor(th[B:].reshape(B, -1), device="cuda", requires_grad=True)
    f = qs.energy_function()
    (f.apply(p1, eng).sum() + 3.0 * f.apply(p2, eng).sum()).backward()
    for par, w, rows in ((p1, 1.0, th[:B]), (p2, 3.0, th[B:])):
        for b in range(B):
            want = oracle.gradient_exact(n, qi.variational_circuit(n, rows[b]), terms)
            assert np.max(np.abs(par.grad[b].cpu().numpy() - w * want)) < 1e-10


def test_autograd_retain_graph_second_backward(qs):
    """A second backward of the same graph (retain_graph) gives the same
    gradient again although the first one swept the work buffer."""
    import torch
    n, B = 12, 2
    th = qi.variational_params(B, 3, n, seed=7)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 0.6)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype="c128")
    params = torch.tensor(th.reshape(B, -1), device="cuda", requires_grad=True)
    E = qs.energy_function().apply(params, eng).sum()
    E.backward(retain_graph=True)
    g1 = params.grad.clone()
    params.grad = None
    E.backward()
    assert torch.equal(params.grad, g1)
    want = oracle.gradient_exact(n, qi.variational_circuit(n, th[1]), terms)
    assert np.max(np.abs(g1[1].cpu().numpy() - want)) < 1e-10


def test_variational_batch_n20_sampled(qs):
    """The full-size variational batch (n = 20, 10 layers, 256 parameter sets,
    complex64): energies and sampled gradient entries against the oracle."""
    import torch
    n, L, B = 20, 10, 256
    th = qi.variational_params(B, L, n, seed=4)
    tmpl = qi.variational_circuit(n, th[0])
    pidx, P = qs.param_indices(tmpl)
    terms = qi.tfim_terms(n, 1.0)
    eng = qs.EnergyGradient(n, B, tmpl, pidx, terms, dtype="c64")
    e, g = eng.run(torch.tensor(th.reshape(B, -1), device="cuda"))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    b = 137
    circ = qi.variational_circuit(n, th[b])
    assert abs(e[b] - oracle.energy(n, circ, terms)) < 2e-4
    want = oracle.gradient_parameter_shift(n, circ, terms, which=[3, 150])
    for j in (3, 150):
        assert abs(g[b, j] - want[j]) < 5e-4
