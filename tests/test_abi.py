"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares.

No compute call is made here (no GPU needed): host-only entry points are exercised
for their argument checks.
"""

import ctypes
import os
import re

import pytest

from paper_1911_12954_gb300 import build as B
from paper_1911_12954_gb300 import hotrg as HB

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "hotrg.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(hotrg_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return HB._lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(HB.SYMBOLS) == names


def test_library_is_sm103a(lib):
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(B.LIB) > 0


def test_status_strings(lib):
    assert lib.hotrg_status_string(0) == b"ok"
    assert lib.hotrg_status_string(-2).startswith(b"workspace")


def test_host_argument_checks(lib):
    ctx = ctypes.c_void_p()
    assert lib.hotrg_create(ctypes.byref(ctx), 0, 4, 0, 0) == -1          # batch 0
    assert lib.hotrg_create(ctypes.byref(ctx), 1, 17, 0, 0) == -1         # dcut_max too big
    assert lib.hotrg_create(ctypes.byref(ctx), 1, 4, 7, 0) == -1          # bad precision
    assert lib.hotrg_create(ctypes.byref(ctx), 1, 4, 0, 2) == -1          # sigma-sigma needs sigma
    assert lib.hotrg_create(ctypes.byref(ctx), 1, 4, 4, 3) == 0           # FP64OZ with impure tensors
    assert lib.hotrg_destroy(ctx) == 0
    assert lib.hotrg_create(ctypes.byref(ctx), 2, 8, 2, 3) == 0
    size = ctypes.c_size_t()
    assert lib.hotrg_workspace_size(ctx, 0, None, None, None, ctypes.byref(size)) == 0
    assert size.value > 8 ** 10 * 4 * 3                                   # A, B, C of D^10 entries
    assert lib.hotrg_step(ctx, 0, 4) == -2                                 # no workspace yet
    assert lib.hotrg_set_workspace(ctx, ctypes.c_void_p(0x1001), 1 << 20) == -1   # misaligned
    m, t = ctypes.c_double(), ctypes.c_double()
    assert lib.hotrg_step_flops(ctx, 0, 4, ctypes.byref(m), ctypes.byref(t)) == 0
    assert m.value == pytest.approx(2.0 * (4 * 4 * 4 * 2) ** 2 * (4 * 4 * 2))   # from 2x2x2x2
    assert lib.hotrg_autotune(ctx, 0, 4) == -2                            # no workspace yet
    assert lib.hotrg_set_option(ctx, 4, 2) == -1                          # autotune is 0 or 1
    assert lib.hotrg_set_option(ctx, 4, 1) == 0
    t, h = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.hotrg_tune_stats(ctx, ctypes.byref(t), ctypes.byref(h)) == 0 and (t.value, h.value) == (0, 0)
    assert lib.hotrg_tune_stats(None, None, None) == -1
    # operand scaling: 0 fixed 2^14, 1 first-pass bound, 2 exact max pass; others refused
    for v, st in ((-1, -1), (3, -1), (0, 0), (2, 0), (1, 0)):
        assert lib.hotrg_set_option(ctx, HB.OPT_MAXNORM, v) == st, v
    assert lib.hotrg_set_option(ctx, HB.OPT_GROUP, 97) == -1               # at most 96 outputs per GEMM
    assert lib.hotrg_set_option(ctx, HB.OPT_GROUP, 3) == 0
    counts = HB.SplitStats()
    assert lib.hotrg_split_stats(ctx, ctypes.byref(counts)) == -2          # no workspace yet
    assert lib.hotrg_split_stats(None, ctypes.byref(counts)) == -1
    assert lib.hotrg_destroy(ctx) == 0


def test_flops_formula_steady_state(lib):
    """All legs D: the block-spin contraction costs 2 D^15 (Sec. 2: D^(4d-1) in d = 4)."""
    import numpy as np
    ctx = ctypes.c_void_p()
    assert lib.hotrg_create(ctypes.byref(ctx), 1, 8, 0, 0) == 0
    # walk the dims to the steady state with the workspace planner, then ask for the flops
    dirs = np.array([0, 1, 2, 3], dtype=np.int32)
    dc = np.array([8, 8, 8, 8], dtype=np.int32)
    size = ctypes.c_size_t()
    assert lib.hotrg_workspace_size(ctx, 4, HB._iptr(dirs), HB._iptr(dc), None, ctypes.byref(size)) == 0
    lib.hotrg_destroy(ctx)

