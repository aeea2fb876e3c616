"""Fused 5-qubit blocks on tensor cores (3xTF32, FP32 accumulation) against the
FP64 oracle and the GPU complex128 path. Every test reports its error."""
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


def err(got, want):
    d = np.asarray(got, np.complex128).reshape(-1) - np.asarray(want, np.complex128).reshape(-1)
    return float(np.max(np.abs(d))), float(np.linalg.norm(d))


@pytest.mark.parametrize("n", [11, 14, 16])
def test_fused_random_layer_matches_oracle(qs, n):
    gates = qi.random_layer_circuit(n, layers=8, seed=3)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="fused")
    mx, l2 = err(st.get(), want)
    print(f"fused n={n}: max {mx:.2e} L2 {l2:.2e}")
    assert mx <= 1e-5 and l2 <= 1e-4


@pytest.mark.parametrize("n", [12, 15])
@pytest.mark.parametrize("width", [2, 3, 5])
def test_fused_mixed_gates_matches_oracle(qs, n, width):
    gates = qi.random_mixed_circuit(n, 120, seed=70 + n, max_controls=2, max_unitary_k=3)
    psi0 = qi.random_state(n, n)
    want = oracle.apply_circuit(psi0.copy(), n, gates)
    st = qs.State(n, dtype="c64").set(psi0).apply(gates, mode="fused", fuse_qubits=width)
    mx, l2 = err(st.get(), want)
    assert mx <= 1e-5 and l2 <= 1e-4


def test_fused_batch_and_complex128_fallback(qs):
    n, B = 13, 3
    gates = qi.random_layer_circuit(n, layers=5, seed=4)
    psis = np.stack([qi.random_state(n, 10 + b) for b in range(B)])
    st = qs.State(n, batch=B, dtype="c64").set(psis).apply(gates, mode="fused")
    got = st.get()
    for b in range(B):
        mx, l2 = err(got[b], oracle.apply_circuit(psis[b].copy(), n, gates))
        assert mx <= 1e-5 and l2 <= 1e-4
    st = qs.State(n, dtype="c128").set(psis[0]).apply(gates, mode="fused")   # tiled fallback
    assert err(st.get(), oracle.apply_circuit(psis[0].copy(), n, gates))[0] < 1e-12


def test_fused_n22_against_fp64_oracle(qs):
    """The fused workload's accuracy check at n = 22: the random-layer circuit
    (20 layers, seed 3) in complex64 with tensor-core blocks vs the FP64 oracle."""
    n = 22
    gates = qi.random_layer_circuit(n, layers=20, seed=3)
    want = oracle.run_circuit(n, gates)
    st = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="fused")
    mx, l2 = err(st.get(), want)
    print(f"fused n=22 vs FP64 oracle: max {mx:.2e} L2 {l2:.2e}")
    assert mx <= 1e-5 and l2 <= 1e-4


def test_fused_n30_against_gpu_complex128(qs):
    """n = 30: fused complex64 against the tiled complex128 path on the same GPU
    (6 layers of the seed-3 circuit to bound the FP64 run)."""
    import torch
    n = 30
    if torch.cuda.mem_get_info()[0] < (1 << n) * 24 * 1.2:
        pytest.skip("not enough device memory")
    gates = qi.random_layer_circuit(n, layers=6, seed=3)
    a = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="fused")
    b = qs.State(n, dtype="c128").init_basis(0).apply(gates, mode="tiled")
    d = a.tensor.to(torch.complex128) - b.tensor
    mx = float(d.abs().max())
    l2 = float(torch.linalg.vector_norm(d))
    print(f"fused n=30 vs GPU complex128: max {mx:.2e} L2 {l2:.2e}")
    assert mx <= 1e-5 and l2 <= 1e-4
