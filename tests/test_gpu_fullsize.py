"""Parity at the benchmark's full sizes (n = 30-33), where the oracle cannot run
the whole state: properties that hold at any size, closed forms on sampled
outputs, and agreement between the tiled path and the plain unfused path."""
import math

import numpy as np
import pytest

from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu

from circuit_utils import inverse_circuit as _inverse  # noqa: E402


@pytest.fixture(scope="module")
def qs():
    from paper_2009_01845_gb300 import qsim
    qsim.load(build_if_missing=True)
    return qsim


def _free_bytes():
    import torch
    return torch.cuda.mem_get_info()[0]


def test_random_layer_n32_c64_roundtrip_is_identity(qs):
    """The bench workload (random-layer circuit, n = 32, complex64, tiled
    passes) followed by its inverse must return |0...0>: amplitude 0 within the
    complex64 tolerance and the norm within FP32 rounding."""
    import torch
    n = 32
    if _free_bytes() < (1 << n) * 8 * 1.2:
        pytest.skip("not enough device memory")
    gates = qi.random_layer_circuit(n, 20, seed=2)
    st = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="auto")
    nrm = st.norm2()[0]
    assert abs(nrm - 1.0) < 1e-4
    zz = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    e = st.expectation(zz)[0]
    assert abs(e.imag) < 1e-6 and abs(e.real) <= n - 1
    st.apply(_inverse(gates), mode="auto")
    a0 = complex(st.tensor[0].item())
    assert abs(a0 - 1.0) < 1e-5
    # every other amplitude is (near) zero: the rest carries 1 - |a0|^2
    assert abs(st.norm2()[0] - 1.0) < 1e-4
    del st
    torch.cuda.empty_cache()


def test_qft_n30_c128_closed_form_sampled(qs):
    """QFT of the seeded basis state at n = 30 in complex128: sampled
    amplitudes against 2^{-n/2} exp(2 pi i x k / 2^n) and the norm."""
    import torch
    n = 30
    if _free_bytes() < (1 << n) * 16 * 1.2:
        pytest.skip("not enough device memory")
    x = qi.qft_input(n, seed=1)
    st = qs.State(n, dtype="c128").init_basis(x).apply(qi.qft_circuit(n), mode="auto")
    ks = qi.rng(7).integers(0, 1 << n, size=4096)
    got = st.tensor[torch.as_tensor(ks, device="cuda")].cpu().numpy()
    want = np.exp(2j * np.pi * ((x * ks.astype(object)) % (1 << n)).astype(np.float64) / 2 ** n) / 2 ** (n / 2)
    assert np.max(np.abs(got - want)) < 1e-12
    assert abs(st.norm2()[0] - 1.0) < 1e-12
    del st
    torch.cuda.empty_cache()


def test_tiled_equals_unfused_n28_c64(qs):
    """Tiled passes against the plain one-gate-per-pass simulator on the same
    GPU at n = 28 (both complex64), element by element."""
    import torch
    n = 28
    gates = qi.random_layer_circuit(n, 6, seed=2)
    a = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="tiled")
    b = qs.State(n, dtype="c64").init_basis(0).apply(gates, mode="unfused")
    d = (a.tensor - b.tensor).abs()
    assert float(d.max()) < 1e-6
    assert float(torch.linalg.vector_norm(a.tensor - b.tensor)) < 1e-4
