"""Plain FP64 HOTRG for the d-dimensional Ising model (test infrastructure only).

This is the oracle the CUDA path is compared with. It is written for a reader who
checks it against the method by eye: each function does one step of the
higher-order tensor renormalisation group (HOTRG) as arXiv:1911.12954 describes it
(Sec. 2 and Fig. 1: local tensors, HOSVD of two adjacent tensors, contraction that
halves the volume; cost D^(4d-1), memory D^(2d)) and as its impure-tensor
observables are used in Sec. 3.1. Library primitives (``numpy.einsum`` on two
operands, ``numpy.linalg.eigh``, ``numpy.argsort``) serve as single steps.

Conventions (the paper prints none of them; these are the readings this project
takes, listed with their reasons in the design notes):

* A site tensor of a d-dimensional lattice has 2d legs, stored in the order
  ``[x, x', y, y', z, z', t, t']`` (d=4). The unprimed leg of direction nu points to
  -nu, the primed leg to +nu. Bond dimension of direction nu: ``D[nu]``.
* Site tensor (Fig. 1A): ``T[i_1..i_2d] = sum_s w_s prod_j W[s, i_j]`` with
  ``W = [[sqrt(cosh b), sqrt(sinh b)], [sqrt(cosh b), -sqrt(sinh b)]]``,
  ``w_s = exp(b h sigma_s)``, ``sigma = (+1, -1)``. Then
  ``sum_i W[s,i] W[s',i] = exp(b sigma_s sigma_s')``: each bond carries one
  Boltzmann factor. The sigma-impure tensor ``S`` has ``sigma_s w_s`` instead.
* One step along mu merges T1 (site n) and T2 (site n+mu). T1's mu' leg is summed
  with T2's mu leg. The new mu legs are (T1.mu, T2.mu'). For each transverse nu the
  new nu leg fuses (T1.nu, T2.nu) and the new nu' leg fuses (T1.nu', T2.nu'), both
  through the same isometry ``U[nu]`` of shape ``(D_nu, D_nu, chi_nu)``,
  ``chi_nu = min(D_nu**2, D_cut)`` (Fig. 1B/1C).
* The isometry comes from the HOSVD of the pair: the Gram matrix of the pair tensor
  on the fused (nu) leg and on the fused (nu') leg; keep the ``chi`` leading
  eigenvectors of the side whose discarded eigenvalue sum is smaller (tie: nu).
* Normalisation: ``c_i = ||T_i||_F``; ``ln Z / V = sum_i ln(c_i) / 2**i +
  ln(Tr T_k) / 2**k`` after k steps (V = 2**k sites; Tr joins each leg to its own
  primed partner, i.e. periodic boundaries).
* Impure tensors: ``S' = (C(S,T) + C(T,S)) / (2 c)``; the nearest-neighbour pair
  ``M_1 = C(S,S) / c_1`` at the first step (the pair lies along the first step's
  direction), then ``M' = (C(M,T) + C(T,M)) / (2 c)``. Isometries and c come from
  the pure tensor. ``<sigma> = Tr S_k / Tr T_k``, ``<sigma sigma> = Tr M_k / Tr T_k``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SIGN_TIE_REL = 1e-8   # |v_i| >= (1 - SIGN_TIE_REL) max|v| is a tie in the gauge rule
CLUSTER_TAU = 1e-10   # eigenvalues closer than CLUSTER_TAU * lambda_max share a cluster
SIDE_TOL_REL = 1e-9   # the primed side wins only if its discarded sum is smaller by more
SIDE_TOL_ABS = 1e-13  # than SIDE_TOL_REL (eps + eps') + SIDE_TOL_ABS lambda_max


# --------------------------------------------------------------------------- site tensor
def ising_tensors(d: int, beta: float, h: float = 0.0):
    """Site tensor T and sigma-impure tensor S of the d-dim Ising model (Fig. 1A).

    Returns two arrays of shape (2,)*2d in FP64. ``T = sum_s w_s W[s]^(x 2d)``.
    """
    if beta < 0:
        raise ValueError("beta must be >= 0 (sqrt(sinh beta) is real)")
    W = np.array([[math.sqrt(math.cosh(beta)), math.sqrt(math.sinh(beta))],
                  [math.sqrt(math.cosh(beta)), -math.sqrt(math.sinh(beta))]])
    sigma = (1.0, -1.0)
    T = np.zeros((2,) * (2 * d))
    S = np.zeros((2,) * (2 * d))
    for s in range(2):
        prod = W[s]
        for _ in range(2 * d - 1):
            prod = np.multiply.outer(prod, W[s])
        ws = math.exp(beta * h * sigma[s])
        T += ws * prod
        S += sigma[s] * ws * prod
    return T, S


def trace(T: np.ndarray) -> float:
    """Tr T: every leg nu summed with its own partner nu' (one site, periodic)."""
    d = T.ndim // 2
    letters = "abcdefghijklmnop"
    sub = "".join(letters[n] * 2 for n in range(d))
    return float(np.einsum(sub + "->", T))


def transfer_matrix(T: np.ndarray, nu: int) -> np.ndarray:
    """M[i, j] = T with leg nu = i, leg nu' = j and every other direction traced (leg
    joined to its own primed partner): the transfer matrix along nu of the one-site
    periodic network, so that Tr M = Tr T and Tr(M M) is the two-site network along nu."""
    d = T.ndim // 2
    letters = "abcdefghijklmnop"
    sub = []
    for n in range(d):
        sub += ["y", "z"] if n == nu else [letters[n], letters[n]]
    return np.einsum("".join(sub) + "->yz", T)


def x_indicator(T: np.ndarray, nu: int = 0) -> float:
    """Degeneracy indicator X of the coarse tensor, used in Sec. 3.1 to locate T_c. The
    paper cites its definition (Gu and Wen) and describes it as counting the degeneracy of
    the largest components of the local tensor; restated here: X = (Tr M)^2 / Tr(M M) with M
    the transfer matrix along nu (``transfer_matrix``). For eigenvalues m_i of M,
    X = (sum m_i)^2 / sum m_i^2: 1 when one dominates (symmetric phase), 2 for two equal
    ones (the two Z2-broken vacua)."""
    M = transfer_matrix(T, nu)
    return float(np.trace(M) ** 2 / np.trace(M @ M))


def leg_dims(T: np.ndarray):
    """Bond dimension of each direction (leg 2nu and 2nu+1 share it)."""
    d = T.ndim // 2
    dims = tuple(T.shape[2 * n] for n in range(d))
    for n in range(d):
        if T.shape[2 * n + 1] != dims[n]:
            raise ValueError("primed and unprimed legs of one direction differ")
    return dims


# --------------------------------------------------------------------------- HOSVD
def gram_half(T: np.ndarray, leg: int, kleg: int) -> np.ndarray:
    """A[a, k, b, k'] = sum over the other 2d-2 legs of T[.., a@leg, k@kleg, ..] T[.., b, k', ..].

    This is the Gram matrix of T unfolded with rows (leg, kleg).
    """
    X = np.moveaxis(T, (leg, kleg), (0, 1))
    Dl, Dk = X.shape[0], X.shape[1]
    X = X.reshape(Dl * Dk, -1)
    return (X @ X.T).reshape(Dl, Dk, Dl, Dk)


def gram(T1: np.ndarray, T2: np.ndarray, mu: int, nu: int, primed: bool) -> np.ndarray:
    """Gram matrix of the pair tensor M = T1 -mu- T2 on the fused leg (T1.l, T2.l).

    l is leg nu (primed=False) or nu' (primed=True). With M unfolded as
    M[(l1 l2), rest], G = M M^T; summing T1's and T2's own legs first gives
    G[(a1 a2), (b1 b2)] = sum_{k,k'} A1[a1,k,b1,k'] A2[a2,k,b2,k'] where k runs over
    the joined bond (T1.mu' = T2.mu). Returned as a (D_nu^2, D_nu^2) matrix whose
    row index is a1*D_nu + a2.
    """
    leg = 2 * nu + (1 if primed else 0)
    A1 = gram_half(T1, leg, 2 * mu + 1)   # T1: k is its mu' leg
    A2 = gram_half(T2, leg, 2 * mu)       # T2: k is its mu leg
    G = np.einsum("akbl,ckdl->acbd", A1, A2, optimize=True)
    D = G.shape[0]
    return G.reshape(D * D, D * D)


def canonical_basis(lam: np.ndarray, V: np.ndarray, nkeep: int | None = None,
                    tau: float = CLUSTER_TAU) -> np.ndarray:
    """Eigenvector gauge that does not depend on the eigensolver.

    ``lam`` is sorted descending and ``V`` holds matching orthonormal eigenvectors.
    Consecutive eigenvalues closer than ``tau * |lam[0]|`` form one cluster (one
    eigenspace up to rounding). Inside a cluster the basis is rebuilt one vector at
    a time: with P the projector onto the cluster's eigenspace minus the vectors
    already chosen, take the unit vector e_i with the longest projection P e_i (the
    lowest i among those within a relative SIGN_TIE_REL of the longest, comparing
    squared lengths) and use P e_i / |P e_i|. For a simple eigenvalue this is
    "largest component positive". The result depends only on the eigenspaces.
    Only the first ``nkeep`` columns are rebuilt (the rest are returned as given).
    """
    n = lam.shape[0]
    nkeep = n if nkeep is None else nkeep
    out = V.copy()
    for j, e in clusters(lam, tau):
        if j >= nkeep:
            break
        W = V[:, j:e]
        base = (W * W).sum(axis=1)          # |P_cluster e_i|^2
        chosen = []
        for t in range(min(e, nkeep) - j):
            norms = base - sum(g * g for g in chosen) if chosen else base
            i = int(np.argmax(norms >= (1.0 - SIGN_TIE_REL) * norms.max()))
            g = W @ W[i, :]                 # P_cluster e_i
            for q in chosen:
                g = g - q * q[i]            # minus the part already covered
            g = g / math.sqrt(norms[i])
            chosen.append(g)
            out[:, j + t] = g
    return out


def clusters(lam: np.ndarray, tau: float = CLUSTER_TAU):
    """[start, end) index ranges of the eigenvalue clusters used by canonical_basis."""
    n = lam.shape[0]
    res, j = [], 0
    while j < n:
        e = j + 1
        while e < n and lam[e - 1] - lam[e] <= tau * abs(lam[0]):
            e += 1
        res.append((j, e))
        j = e
    return res


def eig_desc(G: np.ndarray, nkeep: int | None = None):
    """Eigenvalues in descending order and the matching eigenvectors, the first
    ``nkeep`` of them in canonical gauge."""
    lam, V = np.linalg.eigh(G)
    order = np.argsort(-lam, kind="stable")
    lam, V = lam[order], V[:, order]
    return lam, canonical_basis(lam, V, nkeep)


@dataclass
class Isometry:
    U: np.ndarray            # (D, D, chi)
    chi: int
    primed: bool             # which side of the HOSVD was taken
    eps: tuple               # (discarded sum for nu, discarded sum for nu')
    spectrum: np.ndarray     # eigenvalues of the chosen side, descending
    degenerate_cut: bool     # the cut at chi falls inside an eigenvalue cluster


def isometry(T1, T2, mu: int, nu: int, dcut: int) -> Isometry:
    """HOSVD truncation on direction nu (Fig. 1B): keep the chi leading eigenvectors.

    Both sides are computed; the side with the smaller discarded eigenvalue sum wins.
    Sums equal up to rounding (the Ising tensor's reflection symmetry makes them
    equal in exact arithmetic) count as a tie, and a tie goes to the unprimed side.
    """
    D = T1.shape[2 * nu]
    chi = min(D * D, dcut)
    res = []
    for primed in (False, True):
        lam, V = eig_desc(gram(T1, T2, mu, nu, primed), chi)
        res.append((float(lam[chi:].sum()), lam, V))
    e0, e1 = res[0][0], res[1][0]
    primed = e0 - e1 > SIDE_TOL_REL * (abs(e0) + abs(e1)) + SIDE_TOL_ABS * abs(res[0][1][0])
    _, lam, V = res[1 if primed else 0]
    degenerate = any(a < chi < b for a, b in clusters(lam))
    U = V[:, :chi].reshape(D, D, chi)
    return Isometry(U, chi, primed, (res[0][0], res[1][0]), lam, degenerate)


# --------------------------------------------------------------------------- contraction
_LETTERS = "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz"


def _ein2(a, la, b, lb, lout):
    """Two-operand contraction; einsum on two operands reduces to one BLAS call."""
    return np.einsum(f"{''.join(la)},{''.join(lb)}->{''.join(lout)}", a, b, optimize=True)


def coarse_grain(T1: np.ndarray, T2: np.ndarray, U: dict, mu: int) -> np.ndarray:
    """T' = sum over the pair network of U^nu U^nu T1 T2 for every transverse nu (Fig. 1C).

    ``U[nu]`` has shape (D_nu, D_nu, chi_nu): first index belongs to T1, second to T2,
    third is the new leg. The new nu leg joins (T1.nu, T2.nu); the new nu' leg joins
    (T1.nu', T2.nu'). The new mu legs are (T1.mu, T2.mu'). Evaluated as: T1 with all
    but the last transverse nu-leg isometries, T2 with all but the last nu'-leg
    isometries, the product of the two over every shared index (the D^(4d-1) step),
    then the two isometries of the last transverse direction.
    """
    d = T1.ndim // 2
    trans = [n for n in range(d) if n != mu]
    L = iter(_LETTERS)
    lab = {}
    for n in range(d):
        for key in ("a1", "b1", "a2", "b2", "X", "Y"):
            lab[(key, n)] = next(L)
    m1, m2, k = next(L), next(L), next(L)

    def t_labels(which):
        out = []
        for n in range(d):
            if n == mu:
                out += [m1, k] if which == 1 else [k, m2]
            else:
                out += [lab[("a" + str(which), n)], lab[("b" + str(which), n)]]
        return out

    R, lR = T1, t_labels(1)
    for n in trans[:-1]:            # T1's nu legs: a1 -> (a2, X)
        lU = [lab[("a1", n)], lab[("a2", n)], lab[("X", n)]]
        out = [x for x in lR if x != lab[("a1", n)]] + [lab[("a2", n)], lab[("X", n)]]
        R, lR = _ein2(R, lR, U[n], lU, out), out
    Q, lQ = T2, t_labels(2)
    for n in trans[:-1]:            # T2's nu' legs: b2 -> (b1, Y)
        lU = [lab[("b1", n)], lab[("b2", n)], lab[("Y", n)]]
        out = [x for x in lQ if x != lab[("b2", n)]] + [lab[("b1", n)], lab[("Y", n)]]
        Q, lQ = _ein2(Q, lQ, U[n], lU, out), out
    shared = set(lR) & set(lQ)
    lC = [x for x in lR if x not in shared] + [x for x in lQ if x not in shared]
    C = _ein2(R, lR, Q, lQ, lC)     # the D^(4d-1) contraction
    c = trans[-1]
    lU = [lab[("a1", c)], lab[("a2", c)], lab[("X", c)]]
    out = [x for x in lC if x not in lU[:2]] + [lab[("X", c)]]
    C, lC = _ein2(C, lC, U[c], lU, out), out
    lU = [lab[("b1", c)], lab[("b2", c)], lab[("Y", c)]]
    out = [x for x in lC if x not in lU[:2]] + [lab[("Y", c)]]
    C, lC = _ein2(C, lC, U[c], lU, out), out
    final = []
    for n in range(d):
        final += [m1, m2] if n == mu else [lab[("X", n)], lab[("Y", n)]]
    return np.einsum(f"{''.join(lC)}->{''.join(final)}", C)


# --------------------------------------------------------------------------- driver
@dataclass
class StepRecord:
    mu: int
    dims_in: tuple
    dims_out: tuple
    chi: tuple               # per direction (mu keeps its dim)
    eps: dict                # nu -> (eps_nu, eps_nu')
    primed: dict             # nu -> side taken
    ln_c: float
    degenerate_cut: bool
    lnZ: float               # ln Z / V after this step (V = 2**k); nan if Tr T <= 0


@dataclass
class HOTRG:
    """State of one HOTRG run: the normalised tensors and the ln c accumulator."""

    d: int
    beta: float
    h: float
    T: np.ndarray
    S: np.ndarray | None
    M: np.ndarray | None
    lnz_acc: float           # sum_i ln(c_i) / 2**i over the steps done
    k: int = 0
    history: list = field(default_factory=list)
    impure: bool = False

    @classmethod
    def start(cls, d: int, beta: float, h: float = 0.0, impure: bool = False):
        T, S = ising_tensors(d, beta, h)
        c0 = float(np.linalg.norm(T))
        return cls(d, beta, h, T / c0, S / c0 if impure else None, None,
                   math.log(c0), 0, [], impure)

    @classmethod
    def from_tensor(cls, T: np.ndarray):
        """A run that starts from an arbitrary (already normalised or not) tensor."""
        d = T.ndim // 2
        c0 = float(np.linalg.norm(T))
        return cls(d, float("nan"), 0.0, T / c0, None, None, math.log(c0))

    # ln Z / V, <sigma>, <sigma sigma> for the 2**k-site periodic lattice
    def lnZ(self) -> float:
        tr = trace(self.T)
        if not tr > 0:
            raise FloatingPointError(f"Tr T = {tr} is not positive")
        return self.lnz_acc + math.log(tr) / 2.0 ** self.k

    def magnetization(self) -> float:
        return trace(self.S) / trace(self.T)

    def sigma_sigma(self) -> float:
        return trace(self.M) / trace(self.T)

    def energy(self) -> float:
        """E/V = -d <sigma_n sigma_(n+x)> - h <sigma> (J = 1, all d bonds per site)."""
        return -self.d * self.sigma_sigma() - self.h * self.magnetization()

    def step(self, mu: int, dcut: int, U: dict | None = None) -> StepRecord:
        """One coarse-graining step along mu. ``U`` overrides the HOSVD isometries."""
        T = self.T
        d = self.d
        dims_in = leg_dims(T)
        trans = [n for n in range(d) if n != mu]
        isos = {}
        if U is None:
            isos = {n: isometry(T, T, mu, n, dcut) for n in trans}
            U = {n: isos[n].U for n in trans}
        Tn = coarse_grain(T, T, U, mu)
        Sn = Mn = None
        if self.impure:
            Sn = 0.5 * (coarse_grain(self.S, T, U, mu) + coarse_grain(T, self.S, U, mu))
            if self.k == 0:
                Mn = coarse_grain(self.S, self.S, U, mu)
            else:
                Mn = 0.5 * (coarse_grain(self.M, T, U, mu) + coarse_grain(T, self.M, U, mu))
        c = float(np.linalg.norm(Tn))
        self.T = Tn / c
        if self.impure:
            self.S, self.M = Sn / c, Mn / c
        self.k += 1
        self.lnz_acc += math.log(c) / 2.0 ** self.k
        rec = StepRecord(
            mu=mu, dims_in=dims_in, dims_out=leg_dims(self.T),
            chi=tuple(self.T.shape[2 * n] for n in range(d)),
            eps={n: isos[n].eps for n in isos}, primed={n: isos[n].primed for n in isos},
            ln_c=math.log(c), degenerate_cut=any(i.degenerate_cut for i in isos.values()),
            lnZ=self.lnZ() if trace(self.T) > 0 else float("nan"))
        self.history.append(rec)
        return rec


def run(d: int, beta: float, h: float, dcut: int, nsteps: int, impure: bool = False,
        order=None) -> HOTRG:
    """nsteps HOTRG steps with the directions cycled x, y, z, t, x, ... (or ``order``)."""
    st = HOTRG.start(d, beta, h, impure)
    for i in range(nsteps):
        mu = (order[i % len(order)] if order is not None else i % d)
        st.step(mu, dcut)
    return st


def contract_periodic(T: np.ndarray, extents) -> float:
    """Exact value of the periodic network of prod(extents) copies of T.

    Site n's nu' leg meets site (n + e_nu mod L_nu)'s nu leg; extent 1 is a trace.
    Used to finish a lattice whose coarse network is a few tensors.
    """
    d = T.ndim // 2
    sites = list(np.ndindex(*extents))
    bond = {}
    L = iter(_LETTERS)
    for s in sites:
        for n in range(d):
            bond[(s, n)] = next(L)
    subs = []
    for s in sites:
        lbl = []
        for n in range(d):
            prev = list(s)
            prev[n] = (prev[n] - 1) % extents[n]
            lbl += [bond[(tuple(prev), n)], bond[(s, n)]]
        subs.append("".join(lbl))
    return float(np.einsum(",".join(subs) + "->", *([T] * len(sites)), optimize="greedy"))
