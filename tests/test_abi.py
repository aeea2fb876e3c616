"""Host-side checks of the C-ABI library: it builds, loads, exports every
symbol include/qsim.h declares, its structs match the ctypes binding, and its
argument validation rejects bad calls before touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2009_01845_gb300 import build as qbuild
from paper_2009_01845_gb300 import qsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsim.h")


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qsim.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:qs_status|const char \*|int)\s*(qs_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(qsim._SIGS)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "qsim.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(qs_gate), offsetof(qs_gate, control_mask),
         offsetof(qs_gate, params), offsetof(qs_gate, matrix), offsetof(qs_gate, param_index),
         sizeof(qs_pauli_term), sizeof(qs_opts));
  return 0;
}''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    C = qsim.CGate
    want = [ctypes.sizeof(C), C.control_mask.offset, C.params.offset, C.matrix.offset,
            C.param_index.offset, ctypes.sizeof(qsim.CTerm), ctypes.sizeof(qsim.COpts)]
    assert got == want


def test_kind_codes_match_header():
    text = open(HEADER).read()
    for name, code in qsim.KIND.items():
        m = re.search(rf"#define QS_GATE_{name}\s+(\d+)", text)
        assert m and int(m.group(1)) == code, name
    for name, code in (("QS_MODE_AUTO", 0), ("QS_MODE_UNFUSED", 1), ("QS_MODE_TILED", 2),
                       ("QS_MODE_FUSED_TC", 3), ("QS_C64", 0), ("QS_C128", 1), ("QS_MAX_BATCH", 65535),
                       ("QS_OPT_C128_FP64", qsim.OPT_C128_FP64)):
        assert int(re.search(rf"#define {name}\s+(\d+)", text).group(1)) == code
    for name, code in qsim.SOLVER.items():
        assert int(re.search(rf"#define QS_SOLVER_{name.upper()}\s+(\d+)", text).group(1)) == code


def test_version_and_validation_without_gpu(lib):
    assert b"sm_103a" in lib.qs_version()
    h = ctypes.c_void_p()
    assert lib.qs_state_create(0, 1, 0, None, ctypes.byref(h)) == 1        # n out of range
    assert b"n = 0" in lib.qs_last_error()
    assert lib.qs_state_create(41, 1, 0, None, ctypes.byref(h)) == 1
    assert lib.qs_state_create(10, 0, 0, None, ctypes.byref(h)) == 1       # batch
    assert lib.qs_state_create(10, 1, 7, None, ctypes.byref(h)) == 1       # dtype
    assert lib.qs_state_wrap(10, 1, 0, None, None, ctypes.byref(h)) == 1   # null pointer
    assert lib.qs_state_wrap(10, 1, 0, ctypes.c_void_p(8), None, ctypes.byref(h)) == 1  # misaligned
    assert lib.qs_apply_gates(None, None, 0, None) == 1
    assert lib.qs_state_destroy(None) == 0


def test_batch_limit_and_specialisation_calls_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.qs_state_create(1, 65536, 0, None, ctypes.byref(h)) == 1   # members are a grid dimension
    assert b"65535" in lib.qs_last_error()
    assert lib.qs_jit_set_policy(7) == 1
    assert lib.qs_jit_set_policy(-1) == 1
    for name in ("off", "tiered", "eager", "sync"):
        m = re.search(rf"#define QS_JIT_{name.upper()}\s+(\d+)", open(HEADER).read())
        assert m and int(m.group(1)) == qsim.JIT_POLICY[name]
    assert lib.qs_jit_set_policy(qsim.JIT_POLICY["eager"] | qsim.JIT_FOLD) == 0
    assert lib.qs_jit_set_policy(qsim.JIT_POLICY["tiered"] | 16) == 1
    assert lib.qs_jit_set_policy(qsim.JIT_POLICY["tiered"]) == 0
    assert lib.qs_jit_wait() == 0
    st = qsim.jit_stats()
    assert st["specialised_launches"] == 0 and st["failed"] == 0


def test_channel_struct_matches_binding(tmp_path):
    src = tmp_path / "probe_ch.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "qsim.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(qs_channel), offsetof(qs_channel, targets), offsetof(qs_channel, n_kraus),
         offsetof(qs_channel, kraus));
  return 0;
}''')
    exe = tmp_path / "probe_ch"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    C = qsim.CChannel
    assert got == [ctypes.sizeof(C), C.targets.offset, C.n_kraus.offset, C.kraus.offset]
