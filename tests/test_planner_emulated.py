"""The tiled planner checked on the CPU: its pass descriptors are interpreted
by a host emulator (tests/tile_emulator.cpp, the kernel's op semantics on tile
local indices) linked with the library's own planner and gate lowering, and
whole circuits, including the adjoint sweep's gradient ops, are compared with
the oracle. No GPU is involved; this pins planner logic (pass selection,
stages, diagonal-factor placement and commutation, flips, sign factors)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import circuit_utils
import oracle
from paper_2009_01845_gb300 import inputs as qi
from paper_2009_01845_gb300 import qsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2009_01845_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("emu") / "libtile_emu.so")
    cmd = [cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-I", inc, "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, os.path.join(CSRC, "plan_tiled.cpp"), os.path.join(CSRC, "gates_host.cpp"),
           os.path.join(ROOT, "tests", "tile_emulator.cpp"), "-Wl,-Bsymbolic", "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    lib = ctypes.CDLL(out)
    lib.emu_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.emu_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p]
    lib.emu_trotter.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    lib.emu_apply_flags.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_int]
    lib.emu_apply_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.emu_last_error.restype = ctypes.c_char_p
    return lib


def run_emulated(emu, n, gates, dtype, psi0=None):
    psi = np.zeros(1 << n, dtype=np.complex128) if psi0 is None else np.array(psi0, dtype=np.complex128)
    if psi0 is None:
        psi[0] = 1.0
    arr, keep = qsim.marshal_gates(gates)
    st = emu.emu_apply(n, dtype, arr, len(gates), psi.ctypes.data)
    assert st == 0, emu.emu_last_error().decode()
    return psi


# complex64 descriptors hold float constants: tolerance of a few float roundings per gate
TOL = {0: 2e-5, 1: 1e-10}


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [13, 14])
def test_random_layer_circuit(emu, dtype, n):
    gates = qi.random_layer_circuit(n, 6, seed=2)
    got = run_emulated(emu, n, gates, dtype)
    want = oracle.run_circuit(n, gates)
    assert np.max(np.abs(got - want)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_random_layer_window_passes(emu, dtype):
    """n = 18 > 13 tile bits: passes whose high tile bits are a window of
    consecutive index bits (the light cone of a nearest-neighbour circuit)
    next to greedily chosen ones, with frames, flips and blocks across them."""
    n = 18
    gates = qi.random_layer_circuit(n, 12, seed=3)
    got = run_emulated(emu, n, gates, dtype)
    want = oracle.run_circuit(n, gates)
    assert np.max(np.abs(got - want)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_pass_schedules(emu, dtype):
    """Every pass schedule the autotuner times (most gates of greedy and
    window choices, greedy only, windows only, at most 32 gates per pass)
    gives the oracle's state; the cap needs at least gates / 32 passes and the
    default no more passes than greedy alone on this nearest-neighbour
    circuit."""
    n = 18
    gates = qi.random_layer_circuit(n, 12, seed=4)
    want = oracle.run_circuit(n, gates)
    arr, keep = qsim.marshal_gates(gates)
    passes = {}
    for sched in ((0, 0), (1, 0), (2, 0), (0, 32)):
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
        npass = ctypes.c_int()
        st = emu.emu_apply_schedule(n, dtype, arr, len(gates), psi.ctypes.data, sched[0], sched[1],
                                    ctypes.byref(npass))
        assert st == 0, emu.emu_last_error().decode()
        assert np.max(np.abs(psi - want)) < TOL[dtype]
        passes[sched] = npass.value
    assert passes[(0, 32)] >= -(-len(gates) // 32)
    assert passes[(0, 0)] <= passes[(1, 0)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,seed", [(13, 1), (14, 2), (15, 3)])
def test_random_mixed_circuit(emu, dtype, n, seed):
    gates = qi.random_mixed_circuit(n, 160, seed=seed, max_controls=2)
    psi0 = qi.random_state(n, seed)
    got = run_emulated(emu, n, gates, dtype, psi0)
    want = oracle.run_circuit(n, gates, psi0)
    assert np.max(np.abs(got - want)) < TOL[dtype] * 3


def test_qft_closed_form(emu):
    n = 14
    x = 0x2b7d
    got = run_emulated(emu, n, qi.qft_circuit(n), 1, oracle.basis_state(n, x))
    k = np.arange(1 << n)
    want = np.exp(2j * np.pi * x * k / (1 << n)) / np.sqrt(1 << n)
    assert np.max(np.abs(got - want)) < 1e-11


def _apply_hamiltonian(n, terms, psi):
    """H psi for H = sum_t c_t P_t, P|x> = i^{#Y} (-1)^{popcount(x & z)} |x ^ xm>
    (qubit q = index bit n-1-q)."""
    x = np.arange(1 << n)
    out = np.zeros_like(psi)
    for c, xm, zm in terms:
        xb = sum(1 << (n - 1 - q) for q in range(n) if (xm >> q) & 1)
        zb = sum(1 << (n - 1 - q) for q in range(n) if (zm >> q) & 1)
        ny = bin(xm & zm).count("1")
        par = np.array([bin(v).count("1") & 1 for v in (x & zb)])
        out[x ^ xb] += c * (1j ** ny) * np.where(par == 1, -1.0, 1.0) * psi
    return out


def mixed_param_circuit(n, layers, seed):
    r = qi.rng(seed)
    gates = []
    for l in range(layers):
        for q in range(n):
            kind = ["RX", "RY", "RZ", "U1"][int(r.integers(0, 4))]
            ctrl = (int((q + 3) % n),) if r.uniform() < 0.2 else ()
            gates.append(qi.Gate(kind, (q,), ctrl, (float(r.uniform(0, 6.28)),)))
        gates.append(qi.Gate("CU1", (l % n, (l + 2) % n), (), (float(r.uniform(0, 6.28)),)))
        gates += [qi.Gate("H", (q,)) for q in range(0, n, 3)]
        gates += [qi.Gate("CZ", (i, i + 1)) for i in range(l % 2, n - 1, 2)]
        gates.append(qi.Gate("U3", ((l + 1) % n,), (), tuple(r.uniform(0, 6.28, 3))))
        a = n - 1 - l % 3
        gates.append(qi.Gate("SWAP", (a, (a + 2) % n)))
    return gates


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [12, 13])
def test_adjoint_sweep_gradients(emu, dtype, n):
    """The reverse sweep (gradient op before each inverse parametrised gate,
    over the (phi, lambda) buffer with the phi/lambda bit forced into every
    stage) against the oracle's exact gradients."""
    gates = mixed_param_circuit(n, 3, seed=n)
    terms = qi.tfim_terms(n, 0.7) + qi.random_pauli_terms(n, 4, seed=n)
    phi = run_emulated(emu, n, gates, dtype)
    lam = _apply_hamiltonian(n, terms, phi)
    buf = np.ascontiguousarray(np.concatenate([phi, lam]))
    pidx = [0 if g.kind in ("RX", "RY", "RZ", "U1", "CU1") else -1 for g in gates]
    arr, keep = qsim.marshal_gates(gates, pidx)
    grad = np.zeros(len(gates))
    st = emu.emu_sweep(n, dtype, arr, len(gates), buf.ctypes.data, grad.ctypes.data)
    assert st == 0, emu.emu_last_error().decode()
    got = grad[[i for i, p in enumerate(pidx) if p >= 0]]
    want = oracle.gradient_exact(n, gates, terms)
    scale = sum(abs(t[0]) for t in terms)
    assert np.max(np.abs(got - want)) < (1e-9 if dtype == 1 else 1e-4) * scale


@pytest.mark.parametrize("dtype", [0, 1])
def test_tiled_trotter_steps(emu, dtype):
    """The tiled Trotter queue (Ising phases merged across steps, RX layers)
    against the oracle's step-by-step second-order splitting (Sec. 2.6)."""
    n, T, dt, steps = 13, 1.0, 0.05, 6
    h0 = qi.transverse_field_terms(n)
    h1 = qi.random_ising_terms(n, qi.rng(11))
    a0 = np.zeros(n)
    for c, xm, zm in h0:
        a0[xm.bit_length() - 1] += c
    a1 = np.zeros(n)
    table = np.zeros(n * n + n + 1)
    for c, xm, zm in h1:
        bits = [n - 1 - q for q in range(n) if (zm >> q) & 1]
        if len(bits) == 1:
            table[n * n + bits[0]] += c
        elif len(bits) == 2:
            table[bits[0] * n + bits[1]] += c
            table[bits[1] * n + bits[0]] += c
        else:
            table[n * n + n] += c
    psi = oracle.plus_state(n)
    want = oracle.adiabatic_evolve(psi.copy(), n, h0, h1, T, dt, steps)
    got = psi.copy()
    st = emu.emu_trotter(n, dtype, a0.ctypes.data, a1.ctypes.data, table.ctypes.data, T, dt, steps, got.ctypes.data)
    assert st == 0, emu.emu_last_error().decode()
    assert np.max(np.abs(got - want)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,seed", [(13, 5), (14, 6)])
def test_register_frame(emu, dtype, n, seed):
    gates = circuit_utils.near_swap_circuit(n, 6, seed)
    psi0 = qi.random_state(n, seed)
    got = run_emulated(emu, n, gates, dtype, psi0)
    want = oracle.run_circuit(n, gates, psi0)
    assert np.max(np.abs(got - want)) < TOL[dtype] * 3


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [13, 14])
def test_three_shear_rotations(emu, dtype, n):
    """Real rotations marked for three in-place shears (as the Trotter layers
    are): runs of RY on several qubits, the same qubit rotated twice in a row
    (the deferred third shear must go out first), small and near-pi angles,
    with CZ and RZ between some runs."""
    r = qi.rng(n)
    gates = []
    for l in range(8):
        qs = r.permutation(n)[:7]
        for q in qs:
            gates.append(qi.Gate("RY", (int(q),), (), (float(r.uniform(0.01, 3.1)),)))
            if r.uniform() < 0.4:
                gates.append(qi.Gate("RY", (int(q),), (), (float(r.uniform(0.01, 3.1)),)))
        if l % 3 == 2:
            gates.append(qi.Gate("CZ", (l % n, (l + 1) % n)))
            gates.append(qi.Gate("RZ", ((l + 5) % n,), (), (float(r.uniform(0, 6.28)),)))
    psi0 = qi.random_state(n, n + 3)
    psi = np.array(psi0, dtype=np.complex128)
    arr, keep = qsim.marshal_gates(gates)
    st = emu.emu_apply_flags(n, dtype, arr, len(gates), psi.ctypes.data, 1)
    assert st == 0, emu.emu_last_error().decode()
    want = oracle.run_circuit(n, gates, psi0)
    assert np.max(np.abs(psi - want)) < TOL[dtype] * 3
