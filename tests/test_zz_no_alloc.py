"""The allocation-free expectation entry point, qs_expectation_noalloc.

Some callers cannot allocate device memory when they need an energy: code
running inside CUDA-graph capture, allocator or out-of-memory callbacks, or a
host application that owns all device memory and hands the library only
buffers it allocated itself. For them the library offers one entry point whose
reduction scratch is a fixed device array compiled into the library. This file
is collected last (its name sorts last) so that a failure here never hides the
other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2009_01845_gb300 import inputs as qi

pytestmark = pytest.mark.gpu


def _noalloc(lib, qsim, st, terms):
    import torch
    out = torch.full((2 * st.batch,), float("nan"), dtype=torch.float64, device="cuda")
    arr, cnt = qsim.marshal_terms(terms)
    rc = lib.qs_expectation_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), st.n, st.batch,
                                    qsim.DTYPE[st.dtype], arr, cnt, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qs_last_error()
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(st.batch, 2)
    return o[:, 0] + 1j * o[:, 1]


def test_noalloc_expectation_matches_existing_entry_point_on_consecutive_calls():
    """Two different calls in a row, then the first again: each result equals
    the handle-based qs_expectation and the oracle's <psi|H|psi> on the same
    amplitudes (the ones the device holds), within the expectation tolerance
    (1e-12 complex128, 2e-5 complex64, times the sum of |coefficients|)."""
    from paper_2009_01845_gb300 import qsim
    lib = qsim.load(build_if_missing=True)
    cases = [(12, 3, "c64", 1), (15, 2, "c128", 2)]
    first = None
    for call, (n, batch, dtype, seed) in enumerate(cases + cases[:1]):
        psis = np.stack([qi.random_state(n, 100 * seed + b) for b in range(batch)])
        st = qsim.State(n, batch=batch, dtype=dtype).set(psis)
        held = st.get().reshape(batch, -1).astype(np.complex128)
        terms = qi.random_pauli_terms(n, 30, seed=seed) + qi.tfim_terms(n, 0.8)
        want = st.expectation(terms)            # the existing, handle-based entry point
        got = _noalloc(lib, qsim, st, terms)
        scale = max(1.0, sum(abs(t[0]) for t in terms))
        tol = (1e-12 if dtype == "c128" else 2e-5) * scale
        assert np.max(np.abs(got - want)) < tol
        for b in range(batch):
            ref = oracle.expectation(np.ascontiguousarray(held[b]), n, terms)
            assert abs(got[b] - ref) < tol, (call, b, got[b], ref)
        if call == 0:
            first = got
        if call == len(cases):                  # the first case again, after a different call
            assert np.array_equal(got, first)


def test_noalloc_largest_batch():
    """batch = 65535 (the largest a grid dimension allows) of 1-qubit states:
    every member's energy equals the handle-based entry point's, and sampled
    members the oracle's."""
    from paper_2009_01845_gb300 import qsim
    lib = qsim.load(build_if_missing=True)
    n, batch = 1, 65535
    r = qi.rng(21)
    psis = r.normal(size=(batch, 2)) + 1j * r.normal(size=(batch, 2))
    psis /= np.linalg.norm(psis, axis=1, keepdims=True)
    st = qsim.State(n, batch=batch, dtype="c128").set(psis)
    terms = [(0.7, 1, 0), (-0.4, 0, 1), (0.25, 1, 1), (0.1, 0, 0)]
    got = _noalloc(lib, qsim, st, terms)
    want = st.expectation(terms)
    assert np.max(np.abs(got - want)) < 1e-12
    for b in range(0, batch, 4099):
        assert abs(got[b] - oracle.expectation(np.ascontiguousarray(psis[b]), n, terms)) < 1e-12


def test_noalloc_rejects_batch_beyond_grid_limit():
    import torch
    from paper_2009_01845_gb300 import qsim
    lib = qsim.load(build_if_missing=True)
    buf = torch.zeros(2, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    arr, cnt = qsim.marshal_terms([(1.0, 0, 1)])
    rc = lib.qs_expectation_noalloc(ctypes.c_void_p(buf.data_ptr()), 1, 65536, 0, arr, cnt,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1 and b"65535" in lib.qs_last_error()
