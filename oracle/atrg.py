"""Plain FP64 ATRG for the d-dimensional Ising model (test infrastructure only).

The anisotropic tensor renormalization group (ATRG) is the second coarse-graining scheme
of arXiv:1911.12954 (Sec. 2, Fig. 2; its 4D runs in Sec. 3.2). The paper gives its outline:
an SVD of each local tensor (the extra approximation against HOTRG), a partial SVD that swaps
tensor indices, an HOSVD of the two adjacent decomposed tensors, and a contraction of
O(D^(2d+1)); the partial SVD is a randomized SVD with oversampling p and q power iterations
and N(0, 1) trial matrices (p = 4 D_cut, q = 2 D_cut in its runs). The steps below restate the
published ATRG in that order; the readings this project takes where the paper defers to its
references are listed in the design notes.

Conventions are those of ``oracle.hotrg``: legs ``[x, x', y, y', ...]``, unprimed towards
-nu, primed towards +nu; one step along mu joins T1 (site n) and T2 (site n + mu): T1's mu'
leg with T2's mu leg; new mu legs (T1.mu, T2.mu'); the new nu leg fuses (T1.nu, T2.nu), the
new nu' leg (T1.nu', T2.nu'), both through the same isometry of shape (D_nu, D_nu, chi_nu).

One step along mu (D = D_cut):
  1. SVD of T with rows = its d unprimed legs, columns = its d primed legs, truncated to D:
     T ~ A B, A[(unprimed legs), i] = U sqrt(s), B[i, (primed legs)] = sqrt(s) V^T.
  2. Lower site T1 = A1 B1, upper site T2 = A2 B2; B1's mu' leg is summed with A2's mu leg:
     C[i, (T1's primed transverse legs), (T2's unprimed transverse legs), j].
  3. Swap: truncated SVD of C with rows (i, T2's unprimed transverse legs) and columns
     (T1's primed transverse legs, j): C ~ X Y, X = U sqrt(s), Y = sqrt(s) V^T, rank D
     (exact SVD, or ``rsvd`` with given trial matrices).
  4. G = A1 X (sum over i): legs (T1.nu for nu != mu, T1.mu, T2.nu for nu != mu, m);
     H = Y B2 (sum over j): legs (m, T1.nu', T2.nu' for nu != mu, T2.mu').
  5. For each transverse nu: the Gram matrices of the pair G H on the fused unprimed leg
     (T1.nu, T2.nu) and on the fused primed leg (T1.nu', T2.nu'), computed through the
     m-environments H H^T and G^T G; the side with the smaller discarded sum gives U^nu
     (ties to the unprimed side), canonical eigenvector gauge as in ``oracle.hotrg``.
  6. T'[new legs] = sum_m (G with U^nu on every fused unprimed pair)
                         (H with U^nu on every fused primed pair).
  7. c = ||T'||_F, ln c / 2^k accumulated; ln Z / V as in ``oracle.hotrg``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import hotrg as H

SIDE_TOL_REL = H.SIDE_TOL_REL
SIDE_TOL_ABS = H.SIDE_TOL_ABS


# --------------------------------------------------------------------------- SVDs
def truncated_svd(M: np.ndarray, r: int):
    """The r leading singular triplets of M (descending), as (U, s, Vt)."""
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    r = min(r, s.shape[0])
    return U[:, :r], s[:r], Vt[:r, :]


def rsvd(M: np.ndarray, r: int, omega: np.ndarray, q: int):
    """Randomized truncated SVD of M (Halko, Martinsson, Tropp): the range of M Omega
    (Omega: n x (r + p) trial matrix, its columns the r + p probes) refined by q power
    iterations with re-orthonormalisation after every product, then the exact SVD of the
    small matrix Q^T M. Returns the r leading triplets (U, s, Vt)."""
    Q, _ = np.linalg.qr(M @ omega)
    for _ in range(q):
        Z, _ = np.linalg.qr(M.T @ Q)
        Q, _ = np.linalg.qr(M @ Z)
    Ub, s, Vt = np.linalg.svd(Q.T @ M, full_matrices=False)
    r = min(r, s.shape[0])
    return (Q @ Ub)[:, :r], s[:r], Vt[:r, :]


# --------------------------------------------------------------------------- one step
def _split(T: np.ndarray, dcut: int):
    """Step 1: T ~ A B over the unprimed | primed legs."""
    d = T.ndim // 2
    dims = H.leg_dims(T)
    Tm = np.transpose(T, [2 * n for n in range(d)] + [2 * n + 1 for n in range(d)])
    rows = int(np.prod(dims))
    U, s, Vt = truncated_svd(Tm.reshape(rows, rows), dcut)
    r = np.sqrt(s)
    A = (U * r).reshape(tuple(dims) + (s.shape[0],))          # [x, y, ..., i]
    B = (r[:, None] * Vt).reshape((s.shape[0],) + tuple(dims))  # [i, x', y', ...]
    return A, B


@dataclass
class ATRGStep:
    T: np.ndarray            # new tensor, normalised
    ln_c: float
    isometries: dict         # nu -> hotrg.Isometry-like record (U, eps, primed)
    singular_split: np.ndarray   # singular values kept in step 1
    singular_swap: np.ndarray    # singular values kept in step 3


def step(T: np.ndarray, mu: int, dcut: int, swap=None) -> ATRGStep:
    """One ATRG coarse-graining step along mu. ``swap(M, r)`` computes the truncated SVD of
    the swap (default: exact; ``lambda M, r: rsvd(M, r, omega, q)`` for the randomized one)."""
    d = T.ndim // 2
    dims = H.leg_dims(T)
    trans = [n for n in range(d) if n != mu]
    # 1. split both sites (the same tensor: translation invariance)
    A, B = _split(T, dcut)
    rs = B.shape[0]
    s_split = np.linalg.svd(
        np.transpose(T, [2 * n for n in range(d)] + [2 * n + 1 for n in range(d)]).reshape(
            int(np.prod(dims)), -1), compute_uv=False)[:rs]
    # 2. C = B1 (mu' leg) A2 (mu leg); B: [i, primed legs in direction order], A: [unprimed legs, j]
    B1 = np.moveaxis(B, 1 + mu, -1)              # [i, T1.nu' (trans order), k]
    A2 = np.moveaxis(A, mu, 0)                   # [k, T2.nu (trans order), j]
    nt = len(trans)
    C = np.tensordot(B1, A2, axes=([1 + nt], [0]))   # [i, T1.nu'..., T2.nu..., j]
    # 3. swap: rows (i, T2.nu...), columns (T1.nu'..., j)
    order = [0] + list(range(1 + nt, 1 + 2 * nt)) + list(range(1, 1 + nt)) + [1 + 2 * nt]
    Cm = np.transpose(C, order)
    tdims = [dims[n] for n in trans]
    nrow = rs * int(np.prod(tdims))
    Ms = Cm.reshape(nrow, -1)
    svd = swap if swap is not None else truncated_svd
    U, s, Vt = svd(Ms, dcut)
    r = np.sqrt(s)
    rm = s.shape[0]
    X = (U * r).reshape((rs,) + tuple(tdims) + (rm,))        # [i, T2.nu..., m]
    Y = (r[:, None] * Vt).reshape((rm,) + tuple(tdims) + (rs,))  # [m, T1.nu'..., j]
    # 4. G = A1 X over i: A1 [T1 unprimed legs in direction order, i]
    G = np.tensordot(A, X, axes=([d], [0]))    # [T1.x, T1.y, ... (all d), T2.nu (trans), m]
    # move T1.mu to just before the T2 legs: G [T1.nu (trans), T1.mu, T2.nu (trans), m]
    G = np.moveaxis(G, mu, nt)
    Hh = np.tensordot(Y, B, axes=([1 + nt], [0]))   # [m, T1.nu' (trans), T2.x', ... (all d)]
    # H [m, T1.nu' (trans), T2.nu' (trans), T2.mu']
    Hh = np.moveaxis(Hh, 1 + nt + mu, -1)
    # 5. isometries per transverse direction from the Gram matrices of G H
    EH = np.tensordot(Hh, Hh, axes=(list(range(1, Hh.ndim)), list(range(1, Hh.ndim))))   # [m, m']
    EG = np.tensordot(G, G, axes=(list(range(G.ndim - 1)), list(range(G.ndim - 1))))     # [m, m']
    isos = {}
    for t, n in enumerate(trans):
        Dn = dims[n]
        chi = min(Dn * Dn, dcut)
        # unprimed side: legs (T1.nu = axis t, T2.nu = axis nt + 1 + t) of G
        GE = np.tensordot(G, EH, axes=([G.ndim - 1], [0]))      # G with its m leg through E_H
        keep = [t, nt + 1 + t]
        rest = [a for a in range(G.ndim) if a not in keep]
        Wu = np.tensordot(G, GE, axes=(rest, rest)).reshape(Dn * Dn, Dn * Dn)
        # primed side: legs (T1.nu' = axis 1 + t, T2.nu' = axis 1 + nt + t) of H
        HE = np.tensordot(EG, Hh, axes=([1], [0]))
        keep = [1 + t, 1 + nt + t]
        rest = [a for a in range(Hh.ndim) if a not in keep]
        Wp = np.tensordot(Hh, HE, axes=(rest, rest)).reshape(Dn * Dn, Dn * Dn)
        res = []
        for W in (Wu, Wp):
            lam, V = H.eig_desc(0.5 * (W + W.T), chi)
            res.append((float(lam[chi:].sum()), lam, V))
        e0, e1 = res[0][0], res[1][0]
        primed = e0 - e1 > SIDE_TOL_REL * (abs(e0) + abs(e1)) + SIDE_TOL_ABS * abs(res[0][1][0])
        _, lam, V = res[1 if primed else 0]
        isos[n] = H.Isometry(V[:, :chi].reshape(Dn, Dn, chi), chi, bool(primed), (e0, e1), lam,
                             any(a < chi < b for a, b in H.clusters(lam)))
    # 6. fuse the transverse pairs of G and of H with U^nu, then sum over m
    Gp, Hp = G, Hh
    for t, n in enumerate(trans):
        Un = isos[n].U
        # each fusion removes the two legs and appends the new one last, so at iteration t
        # G is [T1.nu_t.. (nt - t legs), T1.mu, T2.nu_t.. (nt - t legs), m, X_0..X_(t-1)]
        # and H is [m, T1.nu'_t.., T2.nu'_t.., T2.mu', X'_0..X'_(t-1)]
        Gp = _fuse(Gp, (0, nt - t + 1), Un)
        Hp = _fuse(Hp, (1, 1 + nt - t), Un)
    # Gp: [T1.mu, m, X_nu (trans order)]; Hp: [m, T2.mu', X'_nu (trans order)]
    Tn = np.tensordot(Gp, Hp, axes=([1], [0]))    # [T1.mu, X..., T2.mu', X'...]
    new = [None] * (2 * d)
    new[2 * mu], new[2 * mu + 1] = 0, 1 + nt
    for t, n in enumerate(trans):
        new[2 * n], new[2 * n + 1] = 1 + t, 2 + nt + t
    Tn = np.transpose(Tn, new)
    c = float(np.linalg.norm(Tn))
    return ATRGStep(Tn / c, math.log(c), isos, s_split, s)


def _fuse(X: np.ndarray, axes, U: np.ndarray) -> np.ndarray:
    """Contract axes (a1, a2) of X with U[a1, a2, new] and append the new leg last."""
    out = np.tensordot(X, U, axes=(list(axes), [0, 1]))
    return out


# --------------------------------------------------------------------------- driver
@dataclass
class ATRG:
    """State of one ATRG run: the normalised tensor and the ln c accumulator."""

    d: int
    T: np.ndarray
    lnz_acc: float
    k: int = 0
    history: list = field(default_factory=list)

    @classmethod
    def start(cls, d: int, beta: float, h: float = 0.0):
        T, _ = H.ising_tensors(d, beta, h)
        c0 = float(np.linalg.norm(T))
        return cls(d, T / c0, math.log(c0))

    def lnZ(self) -> float:
        tr = H.trace(self.T)
        if not tr > 0:
            raise FloatingPointError(f"Tr T = {tr} is not positive")
        return self.lnz_acc + math.log(tr) / 2.0 ** self.k

    def step(self, mu: int, dcut: int, swap=None) -> ATRGStep:
        st = step(self.T, mu, dcut, swap)
        self.T = st.T
        self.k += 1
        self.lnz_acc += st.ln_c / 2.0 ** self.k
        self.history.append(st)
        return st


def run(d: int, beta: float, h: float, dcut: int, nsteps: int, swap=None) -> ATRG:
    """nsteps ATRG steps with the directions cycled x, y, z, t, x, ..."""
    st = ATRG.start(d, beta, h)
    for i in range(nsteps):
        st.step(i % d, dcut, swap)
    return st
