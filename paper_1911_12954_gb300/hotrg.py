"""Thin ctypes binding of libhotrg.so (include/hotrg.h).

Argument marshalling only: every step of the HOTRG coarse-graining runs in the
library's CUDA kernels. PyTorch supplies the device workspace (one uint8 tensor) and
the stream. There is no CPU path: if the library or a CUDA device is missing, the
constructor raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP64, FP32, TF32X3, FP16X3, FP64OZ = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32x3": TF32X3, "fp16x3": FP16X3, "fp64oz": FP64OZ}
IMPURE_NONE, IMPURE_SIGMA, IMPURE_SIGMASIGMA = 0, 1, 2
OPT_JACOBI_SWEEPS, OPT_GEMM_VARIANT, OPT_GRAPHS, OPT_AUTOTUNE, OPT_GROUP, OPT_MAXNORM = 1, 2, 3, 4, 5, 6

STATUS = {0: "ok", -1: "EINVAL", -2: "EWORKSPACE", -3: "ECUDA", -4: "ENOCONV", -5: "ENONFINITE",
          -6: "ETIMEOUT", -7: "ESTATE", -8: "EUNSUPPORTED"}


class HotrgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if status in (-1, -3):
            msg += " (" + _lib().hotrg_last_error().decode() + ")"
        super().__init__(msg)


class StepRecord(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_int), ("dims", ctypes.c_int * 4), ("primed", ctypes.c_int * 4),
                ("eps", (ctypes.c_double * 2) * 4), ("ln_c", ctypes.c_double),
                ("degenerate", ctypes.c_int * 4), ("slices", ctypes.c_int * 2), ("closing", ctypes.c_int),
                ("gemm_option", ctypes.c_int), ("tuned", ctypes.c_int), ("group", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("gemm_launches", ctypes.c_uint64), ("gemm_ms", ctypes.c_double),
                ("gemm_flops", ctypes.c_double)]


class SplitStats(ctypes.Structure):
    _fields_ = [("entries", ctypes.c_uint64), ("hi_zero", ctypes.c_uint64), ("hi_subnormal", ctypes.c_uint64),
                ("lo_zero", ctypes.c_uint64), ("lo_subnormal", ctypes.c_uint64), ("hi_max", ctypes.c_double * 2)]


_LIB = None
SYMBOLS = ["hotrg_create", "hotrg_destroy", "hotrg_workspace_size", "hotrg_set_workspace", "hotrg_set_stream",
           "hotrg_init_tensor", "hotrg_set_tensor", "hotrg_step", "hotrg_lnZ", "hotrg_impure_magnetization",
           "hotrg_impure_energy", "hotrg_x_indicator", "hotrg_step_info", "hotrg_state", "hotrg_copy_tensor",
           "hotrg_copy_isometry", "hotrg_step_flops", "hotrg_set_option", "hotrg_selftest_wait", "hotrg_profile_enable",
           "hotrg_profile_read", "hotrg_isometry_noalloc", "hotrg_autotune", "hotrg_tune_stats", "hotrg_split_stats",
           "hotrg_status_string", "hotrg_last_error"]


def library_path() -> str:
    return _build.LIB


def _lib():
    """Load (building first if needed) libhotrg.so and declare its signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if not os.path.exists(_build.LIB) else _build.LIB
    L = ctypes.CDLL(path)
    c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "hotrg_create": (c_int, [P(c_void_p), c_int, c_int, c_int, c_int]),
        "hotrg_destroy": (c_int, [c_void_p]),
        "hotrg_workspace_size": (c_int, [c_void_p, c_int, P(c_int), P(c_int), P(c_int), P(c_size_t)]),
        "hotrg_set_workspace": (c_int, [c_void_p, c_void_p, c_size_t]),
        "hotrg_set_stream": (c_int, [c_void_p, c_void_p]),
        "hotrg_init_tensor": (c_int, [c_void_p, P(c_double), P(c_double)]),
        "hotrg_set_tensor": (c_int, [c_void_p, c_int, P(c_int), P(c_double)]),
        "hotrg_step": (c_int, [c_void_p, c_int, c_int]),
        "hotrg_lnZ": (c_int, [c_void_p, P(c_double)]),
        "hotrg_impure_magnetization": (c_int, [c_void_p, P(c_double)]),
        "hotrg_impure_energy": (c_int, [c_void_p, P(c_double), P(c_double)]),
        "hotrg_x_indicator": (c_int, [c_void_p, c_int, P(c_double)]),
        "hotrg_step_info": (c_int, [c_void_p, c_int, c_int, P(StepRecord)]),
        "hotrg_state": (c_int, [c_void_p, P(c_int), P(c_int)]),
        "hotrg_copy_tensor": (c_int, [c_void_p, c_int, c_int, P(c_double), c_size_t]),
        "hotrg_copy_isometry": (c_int, [c_void_p, c_int, c_int, P(c_double), c_size_t]),
        "hotrg_step_flops": (c_int, [c_void_p, c_int, c_int, P(c_double), P(c_double)]),
        "hotrg_set_option": (c_int, [c_void_p, c_int, c_int]),
        "hotrg_selftest_wait": (c_int, [c_void_p, c_int]),
        "hotrg_profile_enable": (c_int, [c_void_p, c_int]),
        "hotrg_profile_read": (c_int, [c_void_p, P(Profile)]),
        "hotrg_isometry_noalloc": (c_int, [c_void_p, P(c_int), c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                           c_void_p]),
        "hotrg_autotune": (c_int, [c_void_p, c_int, c_int]),
        "hotrg_tune_stats": (c_int, [c_void_p, P(ctypes.c_uint64), P(ctypes.c_uint64)]),
        "hotrg_split_stats": (c_int, [c_void_p, P(SplitStats)]),
        "hotrg_status_string": (ctypes.c_char_p, [c_int]),
        "hotrg_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(st, where):
    if st != 0:
        raise HotrgError(st, where)


class HOTRG:
    """A batch of HOTRG runs of the 4D Ising model on one CUDA device.

    Parameters
    ----------
    batch : number of independent runs (temperatures).
    dcut_max : largest bond dimension (2..16).
    precision : "fp64", "fp32", "tf32x3", "fp16x3" (the fastest mixed mode) or "fp64oz" (FP64-grade
        product on the tensor cores, from integer slices).
    impure : 0, IMPURE_SIGMA or IMPURE_SIGMA | IMPURE_SIGMASIGMA.
    schedule : list of (dir, dcut) used to size the workspace (None: steady state at
        dcut_max), dims0 : starting bond dimensions for set_tensor runs.
    workspace_bytes : override of the workspace size (smaller makes steps slice).
    graphs : capture each distinct step into a CUDA graph and replay it (own stream).
    autotune : take each step's closing direction and GEMM pipeline from the autotuner
        (timing new step shapes first; see autotune()).
    group : most temperatures contracted together (0: the planner's choice; 1: one at a time).
    maxnorm : FP16X3 operand scaling: 1 (or True, the default) max-norm scaling from the bound
        the first pass records, 2 from the exact largest magnitude (a max pass), 0 (False) the
        fixed 2^14.
    """

    def __init__(self, batch=1, dcut_max=4, precision="fp64", impure=0, schedule=None, dims0=None,
                 workspace_bytes=None, device=None, stream=None, graphs=False, autotune=False, group=0,
                 maxnorm=True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libhotrg needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = _lib()
        self.device = torch.device(device or "cuda")
        self.batch = batch
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        self.impure = impure
        ctx = ctypes.c_void_p()
        _check(self.lib.hotrg_create(ctypes.byref(ctx), batch, dcut_max, self.precision, impure), "create")
        self.ctx = ctx
        if group:
            _check(self.lib.hotrg_set_option(self.ctx, OPT_GROUP, int(group)), "set_option(group)")
        if int(maxnorm) != 1:
            _check(self.lib.hotrg_set_option(self.ctx, OPT_MAXNORM, int(maxnorm)), "set_option(maxnorm)")
        nbytes = self.workspace_size(schedule, dims0)
        if workspace_bytes is not None:
            nbytes = int(workspace_bytes)
        else:
            # the unsliced plan may exceed the device: give what is free, the steps slice
            free, _ = torch.cuda.mem_get_info(self.device)
            cap = int(free * 0.92) // 256 * 256
            nbytes = min(nbytes, cap)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _check(self.lib.hotrg_set_workspace(self.ctx, ctypes.c_void_p(self.workspace.data_ptr()), nbytes),
               "set_workspace")
        if stream is None:
            # graph capture needs a stream of its own (the legacy default stream cannot be captured)
            stream = torch.cuda.Stream(self.device) if graphs else torch.cuda.current_stream(self.device)
        self.stream = stream
        _check(self.lib.hotrg_set_stream(self.ctx, ctypes.c_void_p(self.stream.cuda_stream)), "set_stream")
        if graphs:
            _check(self.lib.hotrg_set_option(self.ctx, OPT_GRAPHS, 1), "set_option(graphs)")
        if autotune:
            _check(self.lib.hotrg_set_option(self.ctx, OPT_AUTOTUNE, 1), "set_option(autotune)")

    def workspace_size(self, schedule=None, dims0=None) -> int:
        n = 0 if schedule is None else len(schedule)
        dirs = np.array([s[0] for s in schedule] if n else [0], dtype=np.int32)
        dcuts = np.array([s[1] for s in schedule] if n else [0], dtype=np.int32)
        d0 = None if dims0 is None else np.array(dims0, dtype=np.int32)
        out = ctypes.c_size_t()
        _check(self.lib.hotrg_workspace_size(self.ctx, n, _iptr(dirs), _iptr(dcuts),
                                             None if d0 is None else _iptr(d0), ctypes.byref(out)),
               "workspace_size")
        return out.value

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.lib.hotrg_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    # -------------------------------------------------------------- calls
    def init_tensor(self, beta, h):
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.batch,)))
        hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (self.batch,)))
        _check(self.lib.hotrg_init_tensor(self.ctx, _dptr(b), _dptr(hh)), "init_tensor")

    def set_tensor(self, T: np.ndarray, b: int = 0):
        T = np.ascontiguousarray(T, dtype=np.float64)
        dims = np.array([T.shape[2 * n] for n in range(4)], dtype=np.int32)
        _check(self.lib.hotrg_set_tensor(self.ctx, b, _iptr(dims), _dptr(T)), "set_tensor")

    def step(self, direction: int, dcut: int):
        _check(self.lib.hotrg_step(self.ctx, direction, dcut), "step")

    def lnZ(self) -> np.ndarray:
        out = np.zeros(self.batch)
        _check(self.lib.hotrg_lnZ(self.ctx, _dptr(out)), "lnZ")
        return out

    def magnetization(self) -> np.ndarray:
        out = np.zeros(self.batch)
        _check(self.lib.hotrg_impure_magnetization(self.ctx, _dptr(out)), "magnetization")
        return out

    def energy(self):
        e = np.zeros(self.batch)
        ss = np.zeros(self.batch)
        _check(self.lib.hotrg_impure_energy(self.ctx, _dptr(e), _dptr(ss)), "energy")
        return e, ss

    def x_indicator(self, nu: int = 0) -> np.ndarray:
        """Degeneracy indicator X = (Tr M)^2 / Tr(M M) along nu per batch element."""
        out = np.zeros(self.batch)
        _check(self.lib.hotrg_x_indicator(self.ctx, nu, _dptr(out)), "x_indicator")
        return out

    def state(self):
        k = ctypes.c_int()
        dims = np.zeros(4, dtype=np.int32)
        _check(self.lib.hotrg_state(self.ctx, ctypes.byref(k), _iptr(dims)), "state")
        return k.value, tuple(int(x) for x in dims)

    def step_info(self, step: int, b: int = 0) -> dict:
        r = StepRecord()
        _check(self.lib.hotrg_step_info(self.ctx, b, step, ctypes.byref(r)), "step_info")
        return dict(mu=r.mu, dims=tuple(r.dims), primed=tuple(r.primed),
                    eps=tuple(tuple(r.eps[n]) for n in range(4)), ln_c=r.ln_c,
                    degenerate=tuple(r.degenerate), slices=tuple(r.slices), closing=r.closing,
                    gemm_option=r.gemm_option, tuned=bool(r.tuned), group=r.group)

    def tensor(self, which: int = 0, b: int = 0) -> np.ndarray:
        _, dims = self.state()
        shape = tuple(x for D in dims for x in (D, D))
        out = np.zeros(int(np.prod(shape)))
        _check(self.lib.hotrg_copy_tensor(self.ctx, which, b, _dptr(out), out.size), "copy_tensor")
        return out.reshape(shape)

    def isometry(self, nu: int, b: int = 0, dold: int = None, chi: int = None) -> np.ndarray:
        out = np.zeros(16 * 16 * 16)
        _check(self.lib.hotrg_copy_isometry(self.ctx, b, nu, _dptr(out), out.size), "copy_isometry")
        return out[: dold * dold * chi].reshape(dold, dold, chi)

    def autotune(self, direction: int, dcut: int):
        """Time the candidate plans of the next step along `direction` and cache the fastest
        (the run does not advance)."""
        _check(self.lib.hotrg_autotune(self.ctx, direction, dcut), "autotune")

    def tune_stats(self) -> dict:
        t, h = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self.lib.hotrg_tune_stats(self.ctx, ctypes.byref(t), ctypes.byref(h)), "tune_stats")
        return dict(timed=t.value, hits=h.value)

    def split_stats(self) -> dict:
        """FP16X3 split of the last step's operands: entries, zero and subnormal hi / lo counts,
        largest |hi| of A and B (hotrg_split_stats)."""
        st = SplitStats()
        _check(self.lib.hotrg_split_stats(self.ctx, ctypes.byref(st)), "split_stats")
        return dict(entries=st.entries, hi_zero=st.hi_zero, hi_subnormal=st.hi_subnormal, lo_zero=st.lo_zero,
                    lo_subnormal=st.lo_subnormal, hi_max=(st.hi_max[0], st.hi_max[1]))

    def set_option(self, option: int, value: int):
        _check(self.lib.hotrg_set_option(self.ctx, option, value), "set_option")

    def profile(self, enable: bool = True):
        _check(self.lib.hotrg_profile_enable(self.ctx, int(enable)), "profile_enable")

    def profile_read(self) -> dict:
        p = Profile()
        _check(self.lib.hotrg_profile_read(self.ctx, ctypes.byref(p)), "profile_read")
        return dict(launches=p.launches, gemm_launches=p.gemm_launches, gemm_ms=p.gemm_ms, gemm_flops=p.gemm_flops)

    def step_flops(self, direction: int, dcut: int):
        m, t = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.hotrg_step_flops(self.ctx, direction, dcut, ctypes.byref(m), ctypes.byref(t)), "step_flops")
        return m.value, t.value
