"""Error budget of the FP64-grade product (HOTRG_FP64OZ), emulated on the CPU.

The GPU kernel splits each operand, scaled by a power of two to |x| < 1, into five planes of
8-bit integer slices (x = sum_i v_i 2^-8(i+1)) and forms the 15 slice products with
i + j <= 4 in FP32 chunk sums of 256 k. These tests restate that arithmetic with exact
integer matrix products (int64) on seeded operands whose products cancel, and check the
claims the design relies on:

* the chunk sums of slice groups 0 and 1 stay below 2^24 (exact in FP32) for any operand;
* the error of the 15-product sum against the exact product is bounded by the slices'
  resolution, per product term ~2^-40 of max|A| max|B| growing like sqrt(K) over the sum;
* the ten dropped products (i + j >= 5) are its largest part: adding group 5 removes most
  of it, while the operand slices alone are several times below;
* scaling to |x| < 1/2 (so that group 2's chunk sums are exact as well) makes the dropped
  products larger, which is why the kernel scales to |x| < 1.

Test infrastructure only: no CUDA, no library call.
"""

import numpy as np
import pytest

NSL, BITS, CHUNK = 5, 8, 256


def _slices(X, top):
    """Integer slices of X scaled by 2^e with max|X| 2^e in [2^(top-1), 2^top)."""
    m = float(np.abs(X).max())
    e = top - int(np.frexp(m)[1])
    r = X * 2.0 ** e
    v = []
    for _ in range(NSL):
        r = r * 2.0 ** BITS
        vi = np.rint(r)
        v.append(vi.astype(np.int64))
        r = r - vi
    return v, e


def _operands(seed, M=24, K=8192):
    """Rows with a decaying spectrum of scales and mixed signs: the products cancel."""
    rng = np.random.default_rng(seed)
    scale = np.exp(-rng.uniform(0, 6, size=K))
    A = rng.standard_normal((M, K)) * scale
    B = rng.standard_normal((M, K)) * scale
    return A, B


def _product(va, vb, ea, eb, gmax):
    """sum_{i+j <= gmax} v_i w_j 2^-8(i+j+2), exact (integer products, long double sum)."""
    acc = np.zeros((va[0].shape[0], vb[0].shape[0]), dtype=np.longdouble)
    for i in range(NSL):
        for j in range(NSL):
            if i + j <= gmax:
                s = (va[i] @ vb[j].T).astype(np.longdouble)     # exact: |sum| < 2^63
                acc += s * np.longdouble(2.0) ** (-BITS * (i + j + 2))
    return np.float64(acc * np.longdouble(2.0) ** (-ea - eb))


def _exact(A, B):
    return np.float64(A.astype(np.longdouble) @ B.T.astype(np.longdouble))


@pytest.mark.parametrize("seed", [1, 2])
def test_leading_chunk_sums_are_exact_in_fp32(seed):
    A, B = _operands(seed)
    va, _ = _slices(A, 0)
    vb, _ = _slices(B, 0)
    assert max(np.abs(v).max() for v in va[1:]) <= 128 and np.abs(va[0]).max() <= 256
    K = A.shape[1]
    for c0 in range(0, K, CHUNK):
        sl = slice(c0, c0 + CHUNK)
        g0 = va[0][:, sl] @ vb[0][:, sl].T
        g1 = va[0][:, sl] @ vb[1][:, sl].T + va[1][:, sl] @ vb[0][:, sl].T
        assert np.abs(g0).max() <= 2 ** 24 and np.abs(g1).max() <= 2 ** 24


@pytest.mark.parametrize("seed", [1, 2])
def test_dropped_products_dominate_and_stay_within_the_slice_bound(seed):
    A, B = _operands(seed)
    K = A.shape[1]
    exact = _exact(A, B)
    va, ea = _slices(A, 0)
    vb, eb = _slices(B, 0)
    bound = np.sqrt(K) * 2.0 ** -40 * np.abs(A).max() * np.abs(B).max()
    err15 = np.abs(_product(va, vb, ea, eb, 4) - exact).max()
    err19 = np.abs(_product(va, vb, ea, eb, 5) - exact).max()
    err_slices = np.abs(_product(va, vb, ea, eb, 8) - exact).max()
    assert err15 <= 8 * bound
    assert err19 < 0.5 * err15             # group 5 removes most of the error
    assert err_slices < 0.5 * err15        # the operand slices alone are below it


@pytest.mark.parametrize("seed", [1, 2])
def test_half_scale_makes_the_dropped_products_larger(seed):
    A, B = _operands(seed)
    exact = _exact(A, B)
    errs = []
    for top in (0, -1):
        va, ea = _slices(A, top)
        vb, eb = _slices(B, top)
        errs.append(np.abs(_product(va, vb, ea, eb, 4) - exact).max())
    assert errs[1] > 1.5 * errs[0]
