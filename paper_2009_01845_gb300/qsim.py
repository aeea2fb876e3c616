"""Thin ctypes binding over the qsim C-ABI (``include/qsim.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library ``libqsim_gb300.so``. PyTorch provides device memory (the state is a
torch tensor wrapped by the library, which never frees it) and the stream the
calls are ordered on. There is no CPU fallback: if the library is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
from typing import Iterable, Sequence

import numpy as np

from . import build as _build
from .inputs import Gate

_lock = threading.Lock()
_lib = None

KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7, "RX": 8, "RY": 9,
        "RZ": 10, "U1": 11, "U2": 12, "U3": 13, "CZ": 14, "CU1": 15, "SWAP": 16, "UNITARY": 17}
MODE = {"auto": 0, "unfused": 1, "tiled": 2, "fused": 3}
SOLVER = {"exp": 0, "rk4": 1, "rk45": 2}
DTYPE = {"c64": 0, "c128": 1}
STATUS = {0: "QS_OK", 1: "QS_ERR_ARG", 2: "QS_ERR_OOM", 3: "QS_ERR_CUDA", 4: "QS_ERR_UNSUPPORTED",
          5: "QS_ERR_TIMEOUT"}


class QsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_targets", ctypes.c_int32),
                ("targets", ctypes.c_int32 * 5), ("param_index", ctypes.c_int32),
                ("control_mask", ctypes.c_uint64), ("params", ctypes.c_double * 3),
                ("matrix", ctypes.c_void_p)]


class CTerm(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64)]


class CChannel(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int32), ("targets", ctypes.c_int32 * 2), ("n_kraus", ctypes.c_int32),
                ("kraus", ctypes.c_void_p)]


class COpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("fuse_qubits", ctypes.c_int32), ("flags", ctypes.c_int32)]


# (name, argtypes) of every exported entry point; restype is qs_status unless noted
P = ctypes.c_void_p
_SIGS = {
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_version": ([], ctypes.c_char_p),
    "qs_state_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int32, P, P], None),
    "qs_state_wrap": ([ctypes.c_int, ctypes.c_int, ctypes.c_int32, P, P, P], None),
    "qs_state_destroy": ([P], None),
    "qs_state_create_host": ([ctypes.c_int, ctypes.c_int32, ctypes.c_size_t, P, P], None),
    "qs_state_data": ([P, P], None),
    "qs_state_set_stream": ([P, P], None),
    "qs_state_init_basis": ([P, ctypes.c_uint64], None),
    "qs_state_init_plus": ([P], None),
    "qs_state_set": ([P, P, ctypes.c_int], None),
    "qs_state_get": ([P, P, ctypes.c_int], None),
    "qs_apply_gates": ([P, P, ctypes.c_size_t, P], None),
    "qs_apply_gates_batched": ([P, P, ctypes.c_size_t, P, ctypes.c_int, P], None),
    "qs_probabilities": ([P, P, ctypes.c_int], None),
    "qs_norm2": ([P, P], None),
    "qs_marginal_probabilities": ([P, P, ctypes.c_int, P, ctypes.c_int], None),
    "qs_sample": ([P, ctypes.c_int, P, ctypes.c_size_t, P, ctypes.c_int], None),
    "qs_expectation": ([P, P, ctypes.c_size_t, P, P], None),
    "qs_expectation_noalloc": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int32, P, ctypes.c_size_t, P, P],
                               None),
    "qs_energy_gradient": ([P, P, ctypes.c_size_t, P, ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int, P, P,
                            ctypes.c_int, ctypes.c_int], None),
    "qs_trotter_step": ([P, P, ctypes.c_size_t, P, ctypes.c_size_t, ctypes.c_double,
                         ctypes.c_double], None),
    "qs_adiabatic_evolve": ([P, P, ctypes.c_size_t, P, ctypes.c_size_t, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int], None),
    "qs_adiabatic_evolve_batch": ([P, P, ctypes.c_size_t, P, P, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int], None),
    "qs_plan_create": ([P, P, ctypes.c_size_t, P, ctypes.c_int, P, ctypes.c_int, P], None),
    "qs_plan_execute": ([P], None),
    "qs_plan_info": ([P, P, P, P, P], None),
    "qs_plan_destroy": ([P], None),
    "qs_plan_schedule": ([P, P, P], None),
    "qs_evolve": ([P, P, ctypes.c_size_t, P, ctypes.c_size_t, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                   ctypes.c_int], None),
    "qs_schedule_gradient": ([P, P, ctypes.c_size_t, P, ctypes.c_size_t, P, ctypes.c_int, ctypes.c_double, P, P, P],
                             None),
    "qs_adiabatic_run_batch": ([P, ctypes.c_int, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int],
                               None),
    "qs_density_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int32, P, P], None),
    "qs_density_wrap": ([ctypes.c_int, ctypes.c_int, ctypes.c_int32, P, P, P], None),
    "qs_density_init_pure": ([P, P, ctypes.c_int], None),
    "qs_density_trace": ([P, P], None),
    "qs_apply_channels": ([P, P, ctypes.c_size_t, P], None),
    "qs_jit_set_policy": ([ctypes.c_int], None),
    "qs_jit_wait": ([], None),
    "qs_jit_cancel": ([], None),
    "qs_jit_stats": ([P, P, P, P, P], None),
    "qs_profile_enable": ([ctypes.c_int], None),
    "qs_profile_collect": ([P, P, P, P, ctypes.c_int], None),
    "qs_profile_class_name": ([ctypes.c_int], ctypes.c_char_p),
    "qs_profile_class_count": ([], ctypes.c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Open libqsim_gb300.so; raise if it is not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if build_if_missing:
                    _build.build()
                else:
                    raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res if res is not None else ctypes.c_int32
            _lib = lib
            # before the interpreter exits: drop queued pass compiles, let the
            # running ones finish
            atexit.register(lib.qs_jit_cancel)
    return _lib


def _check(status: int):
    if status != 0:
        raise QsimError(status, load().qs_last_error().decode())


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ marshalling
def marshal_gates(gates: Sequence[Gate], param_index: Sequence[int] | None = None):
    """qs_gate array for a gate list; returns (array, keep-alive list)."""
    arr = (CGate * max(1, len(gates)))()
    keep = []
    for i, g in enumerate(gates):
        c = arr[i]
        if g.kind not in KIND:
            raise QsimError(1, f"gate {i}: unknown kind {g.kind!r}")
        if not 1 <= len(g.targets) <= 5:
            raise QsimError(1, f"gate {i}: {len(g.targets)} targets (1..5 supported)")
        c.kind = KIND[g.kind]
        c.n_targets = len(g.targets)
        for j, q in enumerate(g.targets):
            c.targets[j] = int(q)
        mask = 0
        for q in g.controls:
            if not 0 <= int(q) < 64:
                raise QsimError(1, f"gate {i}: control qubit {q} out of range")
            mask |= 1 << int(q)
        c.control_mask = mask
        for j, v in enumerate(g.params[:3]):
            c.params[j] = float(v)
        c.param_index = -1 if param_index is None else int(param_index[i])
        if g.matrix is not None:
            m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
            keep.append(m)
            c.matrix = m.ctypes.data
        else:
            c.matrix = None
    return arr, keep


def marshal_terms(terms: Iterable):
    terms = list(terms)
    arr = (CTerm * max(1, len(terms)))()
    for i, (c, xm, zm) in enumerate(terms):
        arr[i].coeff = float(c)
        arr[i].x_mask = int(xm)
        arr[i].z_mask = int(zm)
    return arr, len(terms)


OPT_C128_FP64 = 1


def opts(mode: str = "auto", tile_qubits: int = 0, fuse_qubits: int = 0, fp64: bool = False) -> COpts:
    """fp64: complex128 gates of the call in FP64 (QS_OPT_C128_FP64; default:
    double-float arithmetic on the FP32 pipes)."""
    return COpts(MODE[mode], int(tile_qubits), int(fuse_qubits), OPT_C128_FP64 if fp64 else 0)


# ------------------------------------------------------------------ state
class State:
    """A batch of n-qubit states in a torch CUDA tensor, wrapped by the library.

    ``tensor`` (optional) must be a contiguous complex64/complex128 CUDA tensor
    of batch * 2^n elements; otherwise one is allocated with torch.
    """

    def __init__(self, n: int, batch: int = 1, dtype: str = "c64", tensor=None, stream=None):
        import torch
        self.lib = load()
        self.n, self.batch, self.dtype = int(n), int(batch), dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        if tensor is None:
            tensor = torch.empty(self.batch << self.n, dtype=tdt, device="cuda")
        if tensor.dtype != tdt or not tensor.is_cuda or not tensor.is_contiguous() or \
                tensor.numel() != (self.batch << self.n):
            raise ValueError("state tensor must be a contiguous CUDA tensor of batch*2^n "
                             f"{tdt} elements")
        self.tensor = tensor
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self.lib.qs_state_wrap(self.n, self.batch, DTYPE[dtype], ctypes.c_void_p(tensor.data_ptr()),
                                      ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.qs_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        _check(self.lib.qs_state_set_stream(self.handle, ctypes.c_void_p(_stream_handle(stream))))

    # -- initialisation
    def init_basis(self, x: int = 0):
        _check(self.lib.qs_state_init_basis(self.handle, int(x)))
        return self

    def init_plus(self):
        _check(self.lib.qs_state_init_plus(self.handle))
        return self

    def set(self, values):
        """Copy amplitudes in from a numpy array (host) or a CUDA tensor (device)."""
        import torch
        if isinstance(values, torch.Tensor) and values.is_cuda:
            src = values.contiguous()
            _check(self.lib.qs_state_set(self.handle, ctypes.c_void_p(src.data_ptr()), 1))
        else:
            npdt = np.complex64 if self.dtype == "c64" else np.complex128
            a = np.ascontiguousarray(np.asarray(values, dtype=npdt).reshape(-1))
            if a.size != (self.batch << self.n):
                raise ValueError("wrong number of amplitudes")
            _check(self.lib.qs_state_set(self.handle, ctypes.c_void_p(a.ctypes.data), 0))
        return self

    def get(self) -> np.ndarray:
        npdt = np.complex64 if self.dtype == "c64" else np.complex128
        out = np.empty(self.batch << self.n, dtype=npdt)
        _check(self.lib.qs_state_get(self.handle, ctypes.c_void_p(out.ctypes.data), 0))
        return out.reshape(self.batch, 1 << self.n) if self.batch > 1 else out

    # -- gates
    def apply(self, gates: Sequence[Gate], mode: str = "auto", tile_qubits: int = 0,
              fuse_qubits: int = 0, fp64: bool = False):
        arr, keep = marshal_gates(gates)
        o = opts(mode, tile_qubits, fuse_qubits, fp64)
        _check(self.lib.qs_apply_gates(self.handle, arr, len(gates), ctypes.byref(o)))
        del keep
        return self

    def apply_batched(self, gates: Sequence[Gate], param_index: Sequence[int], params, mode: str = "auto",
                      fp64: bool = False):
        """``params``: CUDA float64 tensor (batch, n_params); gate i takes its angle
        from column param_index[i] when that is >= 0."""
        import torch
        if not (isinstance(params, torch.Tensor) and params.is_cuda and params.dtype == torch.float64):
            raise ValueError("params must be a CUDA float64 tensor")
        params = params.contiguous()
        if params.dim() != 2 or params.shape[0] != self.batch:
            raise ValueError("params must have shape (batch, n_params)")
        arr, keep = marshal_gates(gates, param_index)
        o = opts(mode, fp64=fp64)
        _check(self.lib.qs_apply_gates_batched(self.handle, arr, len(gates),
                                               ctypes.c_void_p(params.data_ptr()),
                                               int(params.shape[1]), ctypes.byref(o)))
        del keep
        return self

    # -- read-out
    def probabilities(self, on_device: bool = False):
        if on_device:
            import torch
            out = torch.empty(self.batch << self.n, dtype=torch.float64, device=self.tensor.device)
            _check(self.lib.qs_probabilities(self.handle, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        out = np.empty(self.batch << self.n, dtype=np.float64)
        _check(self.lib.qs_probabilities(self.handle, ctypes.c_void_p(out.ctypes.data), 0))
        return out.reshape(self.batch, 1 << self.n) if self.batch > 1 else out

    def marginal_probabilities(self, qubits):
        """Outcome probabilities of the qubit group `qubits` (qubits[0] the most
        significant bit of the outcome), per member: shape (2^m,) or (batch, 2^m)."""
        q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
        m = int(q.size)
        out = np.empty(self.batch << m, dtype=np.float64)
        _check(self.lib.qs_marginal_probabilities(self.handle, ctypes.c_void_p(q.ctypes.data), m,
                                                  ctypes.c_void_p(out.ctypes.data), 0))
        return out.reshape(self.batch, 1 << m) if self.batch > 1 else out

    def sample(self, uniforms, member: int = 0):
        """Measurement samples (basis indices) of member `member` for the given
        uniforms in [0, 1): host arrays (numpy) or device tensors (torch, float64;
        the result is then a device int64 tensor)."""
        if hasattr(uniforms, "data_ptr"):
            import torch
            u = uniforms.contiguous()
            out = torch.empty(u.numel(), dtype=torch.int64, device=u.device)
            _check(self.lib.qs_sample(self.handle, member, ctypes.c_void_p(u.data_ptr()), u.numel(),
                                      ctypes.c_void_p(out.data_ptr()), 1))
            return out
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
        out = np.empty(u.size, dtype=np.uint64)
        _check(self.lib.qs_sample(self.handle, member, ctypes.c_void_p(u.ctypes.data), u.size,
                                  ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def norm2(self) -> np.ndarray:
        out = np.empty(self.batch, dtype=np.float64)
        _check(self.lib.qs_norm2(self.handle, ctypes.c_void_p(out.ctypes.data)))
        return out

    def expectation(self, terms) -> np.ndarray:
        arr, cnt = marshal_terms(terms)
        re = np.empty(self.batch, dtype=np.float64)
        im = np.empty(self.batch, dtype=np.float64)
        _check(self.lib.qs_expectation(self.handle, arr, cnt, ctypes.c_void_p(re.ctypes.data),
                                       ctypes.c_void_p(im.ctypes.data)))
        return re + 1j * im

    # -- Trotter (Sec. 2.6)
    def trotter_step(self, h0, h1, s: float, dt: float):
        a0, n0 = marshal_terms(h0)
        a1, n1 = marshal_terms(h1)
        _check(self.lib.qs_trotter_step(self.handle, a0, n0, a1, n1, float(s), float(dt)))
        return self

    def adiabatic_evolve(self, h0, h1, T: float, dt: float, steps: int = -1):
        a0, n0 = marshal_terms(h0)
        a1, n1 = marshal_terms(h1)
        _check(self.lib.qs_adiabatic_evolve(self.handle, a0, n0, a1, n1, float(T), float(dt), int(steps)))
        return self

    def evolve(self, h0, h1, T: float, dt: float, solver: str = "exp", steps: int = -1):
        """Exact solvers of Sec. 2.6: "exp", "rk4" or "rk45" (qs_evolve)."""
        a0, n0 = marshal_terms(h0)
        a1, n1 = marshal_terms(h1)
        _check(self.lib.qs_evolve(self.handle, a0, n0, a1, n1, float(T), float(dt), int(steps), SOLVER[solver]))
        return self

    def schedule_gradient(self, h0, h1, svals, dt: float):
        """(E, dE/ds_k, dE/d dt) per member of the Trotter evolution with
        schedule values svals (qs_schedule_gradient); the state becomes psi_K."""
        a0, n0 = marshal_terms(h0)
        a1, n1 = marshal_terms(h1)
        sv = np.ascontiguousarray(np.asarray(svals, dtype=np.float64))
        K = int(sv.size)
        e = np.empty(self.batch)
        g = np.empty(self.batch * K)
        gdt = np.empty(self.batch)
        _check(self.lib.qs_schedule_gradient(self.handle, a0, n0, a1, n1, ctypes.c_void_p(sv.ctypes.data), K,
                                             float(dt), ctypes.c_void_p(e.ctypes.data),
                                             ctypes.c_void_p(g.ctypes.data), ctypes.c_void_p(gdt.ctypes.data)))
        return e, g.reshape(self.batch, K), gdt

    def adiabatic_evolve_batch(self, h0, h1_per_member, T: float, dt: float, steps: int = -1):
        """Member b evolves under its own H1 = h1_per_member[b]."""
        if len(h1_per_member) != self.batch:
            raise ValueError("one H1 per batch member")
        a0, n0 = marshal_terms(h0)
        flat = [t for h in h1_per_member for t in h]
        a1, _ = marshal_terms(flat)
        counts = (ctypes.c_size_t * self.batch)(*[len(h) for h in h1_per_member])
        _check(self.lib.qs_adiabatic_evolve_batch(self.handle, a0, n0, a1, counts, float(T), float(dt), int(steps)))
        return self


def adiabatic_run_batch(states, h0s, h1s, T: float, dt: float, steps: int = -1):
    """Evolve handles of different widths in one call (qs_adiabatic_run_batch):
    states[i] has its H0 h0s[i]; h1s holds every member's H1, handle by handle."""
    n = len(states)
    if len(h0s) != n or len(h1s) != sum(st.batch for st in states):
        raise ValueError("one H0 per handle and one H1 per member")
    arr = (ctypes.c_void_p * n)(*[st.handle.value for st in states])
    a0, _ = marshal_terms([t for h in h0s for t in h])
    c0 = (ctypes.c_size_t * n)(*[len(h) for h in h0s])
    a1, _ = marshal_terms([t for h in h1s for t in h])
    c1 = (ctypes.c_size_t * len(h1s))(*[len(h) for h in h1s])
    _check(load().qs_adiabatic_run_batch(arr, n, a0, c0, a1, c1, float(T), float(dt), int(steps)))
    return states


class HostState(State):
    """A state in pinned host memory, larger than the device holds
    (qs_state_create_host): gates and read-outs stream it through at most
    device_bytes of device memory."""

    def __init__(self, n: int, dtype: str = "c64", device_bytes: int = 0, stream=None):
        self.lib = load()
        self.n, self.batch, self.dtype = int(n), 1, dtype
        self.tensor = None
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self.lib.qs_state_create_host(self.n, DTYPE[dtype], int(device_bytes),
                                             ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h)))
        self.handle = h


# ------------------------------------------------------------------ density matrices
class DensityMatrix(State):
    """A batch of n-qubit density matrices (Sec. 2.4, "Density matrices and
    noise") in a torch CUDA tensor of batch * 4^n amplitudes, entry (r, c) of
    member b at b 4^n + r 2^n + c; gates act as rho -> U rho U^dag, channels in
    Kraus form; probabilities() is the diagonal, expectation() Tr(rho H),
    norm2() the purity Tr(rho^2)."""

    def __init__(self, n: int, batch: int = 1, dtype: str = "c64", tensor=None, stream=None):
        import torch
        self.lib = load()
        self.n, self.batch, self.dtype = int(n), int(batch), dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        if tensor is None:
            tensor = torch.empty(self.batch << (2 * self.n), dtype=tdt, device="cuda")
        if tensor.dtype != tdt or not tensor.is_cuda or not tensor.is_contiguous() or \
                tensor.numel() != (self.batch << (2 * self.n)):
            raise ValueError("density tensor must be a contiguous CUDA tensor of batch*4^n "
                             f"{tdt} elements")
        self.tensor = tensor
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self.lib.qs_density_wrap(self.n, self.batch, DTYPE[dtype], ctypes.c_void_p(tensor.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h)))
        self.handle = h

    def init_pure(self, psi):
        """rho = |psi><psi| per member from a host array of batch * 2^n amplitudes."""
        npdt = np.complex64 if self.dtype == "c64" else np.complex128
        a = np.ascontiguousarray(np.asarray(psi, dtype=npdt).reshape(-1))
        if a.size != (self.batch << self.n):
            raise ValueError("wrong number of amplitudes")
        _check(self.lib.qs_density_init_pure(self.handle, ctypes.c_void_p(a.ctypes.data), 0))
        return self

    def set(self, values):
        npdt = np.complex64 if self.dtype == "c64" else np.complex128
        a = np.ascontiguousarray(np.asarray(values, dtype=npdt).reshape(-1))
        if a.size != (self.batch << (2 * self.n)):
            raise ValueError("wrong number of entries")
        _check(self.lib.qs_state_set(self.handle, ctypes.c_void_p(a.ctypes.data), 0))
        return self

    def get(self) -> np.ndarray:
        """The matrices: shape (2^n, 2^n), or (batch, 2^n, 2^n)."""
        npdt = np.complex64 if self.dtype == "c64" else np.complex128
        out = np.empty(self.batch << (2 * self.n), dtype=npdt)
        _check(self.lib.qs_state_get(self.handle, ctypes.c_void_p(out.ctypes.data), 0))
        d = 1 << self.n
        return out.reshape(self.batch, d, d) if self.batch > 1 else out.reshape(d, d)

    def apply_channels(self, channels, mode: str = "auto"):
        """channels: list of (targets, kraus) with kraus a list of 2^k x 2^k matrices."""
        arr = (CChannel * max(1, len(channels)))()
        keep = []
        for i, (targets, kraus) in enumerate(channels):
            k = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128))
            keep.append(k)
            arr[i].n_targets = len(targets)
            for j, q in enumerate(targets):
                arr[i].targets[j] = int(q)
            arr[i].n_kraus = int(k.shape[0])
            arr[i].kraus = k.ctypes.data
        o = opts(mode)
        _check(self.lib.qs_apply_channels(self.handle, arr, len(channels), ctypes.byref(o)))
        del keep
        return self

    def trace(self) -> np.ndarray:
        out = np.empty(self.batch, dtype=np.float64)
        _check(self.lib.qs_density_trace(self.handle, ctypes.c_void_p(out.ctypes.data)))
        return out

    def purity(self) -> np.ndarray:
        return self.norm2()

    def probabilities(self, on_device: bool = False):
        if on_device:
            import torch
            out = torch.empty(self.batch << self.n, dtype=torch.float64, device=self.tensor.device)
            _check(self.lib.qs_probabilities(self.handle, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        out = np.empty(self.batch << self.n, dtype=np.float64)
        _check(self.lib.qs_probabilities(self.handle, ctypes.c_void_p(out.ctypes.data), 0))
        return out.reshape(self.batch, 1 << self.n) if self.batch > 1 else out


# ------------------------------------------------------------------ pass specialisation
JIT_POLICY = {"off": 0, "tiered": 1, "eager": 2, "sync": 3}


JIT_FOLD = 8


def jit_set_policy(policy: str, fold: bool = False):
    """When tiled passes get kernels specialised for them (qs_jit_set_policy):
    "off", "tiered" (default), "eager" or "sync"; fold: passes repeated with
    the same values also get kernels with the values compiled in."""
    _check(load().qs_jit_set_policy(JIT_POLICY[policy] | (JIT_FOLD if fold else 0)))


def jit_wait():
    """Wait for the queued background compiles."""
    _check(load().qs_jit_wait())


def jit_stats() -> dict:
    sp, ge, co, fa = (ctypes.c_longlong() for _ in range(4))
    sec = ctypes.c_double()
    _check(load().qs_jit_stats(ctypes.byref(sp), ctypes.byref(ge), ctypes.byref(co), ctypes.byref(fa),
                               ctypes.byref(sec)))
    return {"specialised_launches": sp.value, "generic_launches": ge.value, "compiled": co.value,
            "failed": fa.value, "compile_seconds": sec.value}


# ------------------------------------------------------------------ launch accounting
def profile_enable(on: bool = True):
    _check(load().qs_profile_enable(1 if on else 0))


def profile_collect() -> dict:
    """{class name: (total ms, launches, algorithmic bytes, algorithmic flops)}
    since the last collect; resets."""
    lib = load()
    nc = lib.qs_profile_class_count()
    ms = (ctypes.c_double * nc)()
    cnt = (ctypes.c_longlong * nc)()
    by = (ctypes.c_double * nc)()
    fl = (ctypes.c_double * nc)()
    _check(lib.qs_profile_collect(ms, cnt, by, fl, nc))
    return {lib.qs_profile_class_name(c).decode(): (ms[c], cnt[c], by[c], fl[c]) for c in range(nc)}


# ------------------------------------------------------------------ adjoint gradient
GRAD_MODE = {"full": 0, "forward": 1, "sweep": 2}


def param_indices(gates, kinds=("RX", "RY", "RZ", "U1", "CU1")):
    """param_index list giving every rotation of ``gates`` its own column, in order."""
    out, c = [], 0
    for g in gates:
        if g.kind in kinds:
            out.append(c)
            c += 1
        else:
            out.append(-1)
    return out, c


class EnergyGradient:
    """E_b(theta) = Re <psi_b|H|psi_b> and dE_b/dtheta for a batch of parameter
    sets, through qs_energy_gradient. ``work`` holds (psi, lambda) per member:
    a torch tensor of batch * 2^(n+1) amplitudes allocated here."""

    def __init__(self, n: int, batch: int, gates, param_index, terms, dtype: str = "c64", stream=None):
        import torch
        self.n, self.batch, self.dtype = int(n), int(batch), dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        self.work = torch.empty(self.batch << (self.n + 1), dtype=tdt, device="cuda")
        self.state = State(self.n + 1, batch=self.batch, dtype=dtype, tensor=self.work, stream=stream)
        self.lib = self.state.lib
        self.gate_arr, self._keep = marshal_gates(gates, param_index)
        self.count = len(gates)
        self.term_arr, self.n_terms = marshal_terms(terms)
        # run counter, and the run whose forward state (psi, lambda) ``work``
        # still holds (None once a sweep or a full run has consumed it)
        self.generation = 0
        self.forward_generation = None

    def run(self, params, mode: str = "full", init_zero: bool = True, ckpt_every: int = 0, energy=None,
            grad=None):
        import torch
        if not (isinstance(params, torch.Tensor) and params.is_cuda and params.dtype == torch.float64):
            raise ValueError("params must be a CUDA float64 tensor")
        params = params.contiguous()
        npar = int(params.shape[1]) if params.dim() == 2 else 0
        if mode != "sweep" and energy is None:
            energy = torch.empty(self.batch, dtype=torch.float64, device="cuda")
        if mode != "forward" and grad is None:
            grad = torch.empty(self.batch, npar, dtype=torch.float64, device="cuda")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        if mode == "sweep" and self.forward_generation is None:
            raise RuntimeError("sweep needs a forward run whose state is still in the work buffer")
        self.generation += 1
        self.forward_generation = None
        _check(self.lib.qs_energy_gradient(self.state.handle, self.gate_arr, self.count, ptr(params), npar,
                                           self.term_arr, self.n_terms, 1 if init_zero else 0, ptr(energy),
                                           ptr(grad), int(ckpt_every), GRAD_MODE[mode]))
        if mode == "forward":
            self.forward_generation = self.generation
        return energy, grad


def energy_function():
    """torch.autograd.Function computing E(theta) per batch member; backward
    runs the adjoint reverse sweep (one sweep for all parameters).

    The sweep continues from the forward state left in the engine's work
    buffer. Each forward records the engine's run counter; a backward whose
    forward is no longer the engine's last run (another forward on the same
    engine came in between, or an earlier backward already swept it, as with
    retain_graph) runs the forward again from its saved parameters first, so
    every backward sweeps the state of its own forward."""
    import torch

    class _Energy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, engine):
            energy, _ = engine.run(params, mode="forward")
            ctx.engine = engine
            ctx.generation = engine.generation
            ctx.save_for_backward(params)
            return energy

        @staticmethod
        def backward(ctx, g_energy):
            (params,) = ctx.saved_tensors
            eng = ctx.engine
            if eng.forward_generation is None or eng.forward_generation != ctx.generation:
                eng.run(params, mode="forward")
            _, grad = eng.run(params, mode="sweep")
            return g_energy[:, None] * grad, None

    return _Energy


# ------------------------------------------------------------------ plans
class Plan:
    """A gate queue captured in a CUDA graph for one state (qs_plan_*)."""

    def __init__(self, state: State, gates, mode: str = "auto", autotune: bool = True, fuse_qubits: int = 0,
                 param_index=None, params=None):
        self.state = state
        self.lib = state.lib
        arr, keep = marshal_gates(gates, param_index)
        o = opts(mode, 0, fuse_qubits)
        pp = ctypes.c_void_p(params.data_ptr()) if params is not None else None
        npar = int(params.shape[1]) if params is not None else 0
        self._params = params
        h = ctypes.c_void_p()
        _check(self.lib.qs_plan_create(state.handle, arr, len(gates), pp, npar, ctypes.byref(o),
                                       1 if autotune else 0, ctypes.byref(h)))
        del keep
        self.handle = h

    def execute(self):
        _check(self.lib.qs_plan_execute(self.handle))
        return self.state

    def info(self) -> dict:
        m, w, t, nodes = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_size_t()
        _check(self.lib.qs_plan_info(self.handle, ctypes.byref(m), ctypes.byref(w), ctypes.byref(t),
                                     ctypes.byref(nodes)))
        name = {v: k for k, v in MODE.items()}[m.value]
        sel, cap = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.qs_plan_schedule(self.handle, ctypes.byref(sel), ctypes.byref(cap)))
        return {"mode": name, "fuse_qubits": w.value, "tuned_ms": t.value, "graph_nodes": nodes.value,
                "schedule": (sel.value, cap.value)}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.qs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
