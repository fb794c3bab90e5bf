"""Pins of the ATRG oracle (``oracle/atrg.py``, Sec. 2 / Fig. 2 and Sec. 3.2 of the paper).

Independent of the oracle's own code: exact enumeration of small periodic lattices (with
nothing truncated ATRG is exact), Onsager's 2D free energy (with truncation ATRG converges to
it as D_cut grows, more slowly than HOTRG: it adds the SVD of each local tensor), the exact
truncated SVD for the randomized one of the swap (with the paper's p = 4 D_cut, q = 2 D_cut
and N(0, 1) trial matrices).
"""

import numpy as np
import pytest

from oracle import atrg as A
from oracle import exact as E
from oracle import hotrg as H

NO_CUT = 10 ** 6


@pytest.mark.parametrize("d,beta,h", [(2, 0.37, 0.0), (3, 0.21, 0.3), (4, 1 / 6.65, 0.0), (4, 0.2, -0.4)])
def test_one_untruncated_step_is_exact(d, beta, h):
    st = A.run(d, beta, h, NO_CUT, 1)
    ref = E.enumerate_lattice([2] + [1] * (d - 1), beta, h)["lnZ_over_V"]
    assert st.lnZ() == pytest.approx(ref, abs=1e-13)


def test_untruncated_2d_4x4_and_3d_2x2x1():
    st = A.run(2, 0.41, 0.1, NO_CUT, 4)
    assert st.lnZ() == pytest.approx(E.enumerate_lattice([4, 4], 0.41, 0.1)["lnZ_over_V"], abs=1e-13)
    st = A.run(3, 0.3, 0.0, NO_CUT, 2)
    assert st.lnZ() == pytest.approx(E.enumerate_lattice([2, 2, 1], 0.3, 0.0)["lnZ_over_V"], abs=1e-13)


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_2d_converges_to_onsager_behind_hotrg(beta):
    """40 steps (2^40 sites) at D_cut = 8 and 16: the error against Onsager shrinks with
    D_cut, stays below 5e-5 / 5e-7, and is never below HOTRG's at the same D_cut."""
    ons = E.onsager_lnz(beta)
    errs = []
    for D in (8, 16):
        a = abs(A.run(2, beta, 0.0, D, 40).lnZ() - ons)
        h = abs(H.run(2, beta, 0.0, D, 40).lnZ() - ons)
        assert a >= h
        errs.append(a)
    assert errs[1] < errs[0]
    assert errs[0] < 5e-5 and errs[1] < 5e-7


def test_rsvd_reproduces_the_truncated_svd():
    rng = np.random.default_rng(5)
    m, n, r = 300, 200, 12
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (U * 0.5 ** np.arange(n)) @ V.T
    Ue, se, _ = A.truncated_svd(M, r)
    Ur, sr, _ = A.rsvd(M, r, rng.standard_normal((n, r + 4 * r)), 2 * r)
    assert np.allclose(sr, se, rtol=0, atol=1e-12 * se[0])
    assert np.allclose(Ur @ Ur.T, Ue @ Ue.T, atol=1e-12)          # same rank-r subspace


class _RSVDSwap:
    """The swap of each step by RSVD with p = 4 D_cut, q = 2 D_cut, N(0, 1) trial matrices
    drawn from a seeded generator (the method's random numbers, passed in)."""

    def __init__(self, seed, dcut):
        self.rng = np.random.default_rng(seed)
        self.dcut = dcut

    def __call__(self, M, r):
        omega = self.rng.standard_normal((M.shape[1], r + 4 * self.dcut))
        return A.rsvd(M, r, omega, 2 * self.dcut)


@pytest.mark.parametrize("d,dcut,steps", [(2, 8, 16), (4, 4, 8)])
def test_rsvd_swap_run_equals_exact_swap_run(d, dcut, steps):
    beta = 0.44 if d == 2 else 1 / 6.65
    a = A.run(d, beta, 0.0, dcut, steps)
    b = A.run(d, beta, 0.0, dcut, steps, swap=_RSVDSwap(1, dcut))
    assert b.lnZ() == pytest.approx(a.lnZ(), abs=1e-12)


def test_4d_atrg_tracks_hotrg():
    """4D at T = 6.65, D_cut = 4, 8 steps: ATRG's ln Z/V within 3e-3 of HOTRG's (ATRG's
    extra SVD costs accuracy at equal D_cut, Sec. 3.2)."""
    a = A.run(4, 1 / 6.65, 0.0, 4, 8)
    h = H.run(4, 1 / 6.65, 0.0, 4, 8)
    assert abs(a.lnZ() - h.lnZ()) < 3e-3
