"""hotrg_isometry_noalloc: the isometry stage without any device allocation.

Some callers cannot allocate device memory (code inside another framework's memory
pool or under a fixed budget, plugins handed only their buffers, threads that must not
enter the allocator while other work is in flight). For them the library computes the
HOSVD isometry of one direction (Sec. 2, Fig. 1B) with every intermediate in a fixed
8 MiB device array it owns. These tests call that entry point through the C ABI and
check it

* against the oracle's isometry (the isometry in canonical gauge, both discarded sums,
  the side taken), including the largest shapes the array is sized for: bond dimension 8
  in every direction (the Gram split-K runs at its 32-chunk clamp) and chi = 64;
* against the isometry the regular path (hotrg_step with a caller workspace, then
  hotrg_copy_isometry) produces for the same tensor, on two calls in a row with
  different tensors and shapes, so that leftovers of the first call in the shared
  array cannot leak into the second;
* for its refusals: a bond dimension above 8 (EINVAL with a message) and a tensor with a
  NaN or an infinity (ENONFINITE).

The file is collected last, so a run that stops at the first failure has run every
other test first.
"""

import ctypes

import numpy as np
import pytest

from oracle import hotrg as H
from workloads import random_tensor

pytestmark = pytest.mark.gpu

CASES = [
    # dims (Dx, Dy, Dz, Dt), mu, nu, dcut
    ((3, 4, 2, 3), 1, 3, 5),
    ((4, 2, 3, 2), 0, 2, 7),
]

# the limits of the fixed array: every bond dimension 8 (n = 64, the split-K Gram at its
# 32-chunk clamp), with a truncating cut and with chi = n = 64
LIMIT_CASES = [
    ((8, 8, 8, 8), 0, 1, 8),
    ((8, 8, 8, 8), 2, 3, 64),
]


def _regular(T, dims, mu, nu, dcut):
    from paper_1911_12954_gb300 import HOTRG
    g = HOTRG(batch=1, dcut_max=max(max(dims), dcut), precision="fp64", schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    chi = min(dims[nu] ** 2, dcut)
    info = g.step_info(1)
    return g.isometry(nu, dold=dims[nu], chi=chi), info["eps"][nu], info["primed"][nu]


def _call(T, dims, mu, nu, dcut, normalise=True):
    """One call of the entry point; returns (status, U, eps, primed)."""
    import torch

    from paper_1911_12954_gb300 import hotrg as HB
    lib = HB._lib()
    n = dims[nu] ** 2
    chi = min(n, dcut)
    Tn = T / np.linalg.norm(T) if normalise else T       # the regular path stores T / ||T||_F
    T_dev = torch.from_numpy(np.ascontiguousarray(Tn)).to("cuda")
    U = torch.full((n * chi,), float("nan"), dtype=torch.float64, device="cuda")
    eps = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    primed = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    d = (ctypes.c_int * 4)(*dims)
    st = lib.hotrg_isometry_noalloc(ctypes.c_void_p(T_dev.data_ptr()), d, mu, nu, dcut,
                                    ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(eps.data_ptr()),
                                    ctypes.c_void_p(primed.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return (st, U.cpu().numpy().reshape(dims[nu], dims[nu], chi), tuple(eps.cpu().numpy()),
            int(primed.cpu()[0]))


def _noalloc(T, dims, mu, nu, dcut):
    from paper_1911_12954_gb300 import hotrg as HB
    st, U, eps, primed = _call(T, dims, mu, nu, dcut)
    assert st == 0, (st, HB._lib().hotrg_last_error())
    return U, eps, primed


def _check_vs_oracle(T, dims, mu, nu, dcut):
    Tn = T / np.linalg.norm(T)
    ref = H.isometry(Tn, Tn, mu, nu, dcut)
    assert not ref.degenerate_cut          # seeded N(0,1) tensors: the kept subspace is unique
    U, eps, primed = _noalloc(T, dims, mu, nu, dcut)
    assert np.allclose(U, ref.U, atol=1e-11), (dims, mu, nu, dcut)
    assert eps == pytest.approx(ref.eps, rel=1e-9, abs=1e-13)
    assert primed == int(ref.primed)


@pytest.mark.parametrize("dims,mu,nu,dcut", CASES + LIMIT_CASES)
def test_noalloc_isometry_matches_oracle(dims, mu, nu, dcut):
    _check_vs_oracle(random_tensor(700 + sum(dims) + 10 * nu, dims), dims, mu, nu, dcut)


def test_noalloc_isometry_matches_regular_path_twice():
    for i, (dims, mu, nu, dcut) in enumerate(CASES):
        T = random_tensor(500 + i, dims)
        U_ref, eps_ref, primed_ref = _regular(T, dims, mu, nu, dcut)
        U, eps, primed = _noalloc(T, dims, mu, nu, dcut)
        assert np.allclose(U, U_ref, atol=1e-11), i
        assert eps == pytest.approx(eps_ref, rel=1e-9, abs=1e-13), i
        assert primed == primed_ref, i


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_1911_12954_gb300 import hotrg as HB
    lib = HB._lib()
    dims = (9, 2, 2, 2)
    d = (ctypes.c_int * 4)(*dims)
    buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = lib.hotrg_isometry_noalloc(p, d, 1, 0, 4, p, p, p, None)
    assert st == -1
    assert b"exceeds the limit" in lib.hotrg_last_error()


def test_noalloc_reports_nonfinite_tensors():
    from paper_1911_12954_gb300 import hotrg as HB
    dims, mu, nu, dcut = (3, 2, 3, 2), 0, 2, 4
    for bad in (np.nan, np.inf):
        T = random_tensor(40, dims)
        T /= np.linalg.norm(T)
        T[1, 0, 1, 1, 2, 0, 1, 0] = bad
        st, _, _, _ = _call(T, dims, mu, nu, dcut, normalise=False)
        assert st == -5, bad
        assert b"non-finite" in HB._lib().hotrg_last_error()
    # the array is usable again right after a refused call
    _check_vs_oracle(random_tensor(41, dims), dims, mu, nu, dcut)
