"""Pins of the FP64 oracle against results that do not come from the oracle itself.

Each test names what fixes the expected value: exact enumeration of all spin
states, a textbook closed form (1D transfer matrix, Onsager, Yang, the 2D exact
energy, the high-temperature series), brute-force evaluation of a definition on
tiny inputs, or a symmetry of the model. A plausible slip in the oracle (a dropped
factor, a wrong leg, a transposed operand, a wrong 2**-k weight, the wrong side of
the HOSVD, a wrong isometry direction) fails at least one of them.
"""

import math

import numpy as np
import pytest

from oracle import exact as E
from oracle import hotrg as H

BETA_C4D = 1 / 6.65     # T = 6.65, just above T_c(D_cut=13) = 6.650365 (Sec. 3.1)


# ---------------------------------------------------------------- site tensor (Fig. 1A)
@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.7, 0.2), (0.05, -0.4)])
@pytest.mark.parametrize("L", [1, 2, 5])
def test_site_tensor_1d_transfer_matrix(beta, h, L):
    """1D ring of L sites: Z = lam+^L + lam-^L (textbook transfer matrix)."""
    T, _ = H.ising_tensors(1, beta, h)
    Z = np.trace(np.linalg.matrix_power(T, L))
    eb = math.exp(beta)
    root = math.sqrt(eb ** 2 * math.sinh(beta * h) ** 2 + math.exp(-2 * beta))
    lp, lm = eb * math.cosh(beta * h) + root, eb * math.cosh(beta * h) - root
    assert Z == pytest.approx(lp ** L + lm ** L, rel=1e-13)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_single_site_trace(d):
    """k = 0: one site with every bond closing on itself, Z = 2 e^(d b) cosh(b h)."""
    beta, h = 0.41, 0.13
    st = H.HOTRG.start(d, beta, h, impure=True)
    assert st.lnZ() == pytest.approx(math.log(E.ising_trace_single_site(d, beta, h)), abs=1e-14)
    assert st.magnetization() == pytest.approx(math.tanh(beta * h), abs=1e-14)


# ---------------------------------------------------------------- exact enumeration
@pytest.mark.parametrize("beta,h", [(BETA_C4D, 0.0), (BETA_C4D, 0.1), (0.6, 0.03)])
def test_4d_untruncated_vs_enumeration(beta, h):
    """ln Z/V, <s> and <s s> after 1 and 2 untruncated steps = 2- and 4-site lattices."""
    st = H.HOTRG.start(4, beta, h, impure=True)
    for k, ext in ((1, (2, 1, 1, 1)), (2, (2, 2, 1, 1))):
        st.step(k - 1, 10 ** 6)
        ex = E.enumerate_lattice(ext, beta, h)
        assert st.lnZ() == pytest.approx(ex["lnZ_over_V"], abs=1e-13)
        assert st.magnetization() == pytest.approx(ex["sigma"], abs=1e-13)
        assert st.sigma_sigma() == pytest.approx(ex["sigma_sigma_x"], abs=1e-13)
    assert st.history[-1].dims_out == (4, 4, 16, 16)


@pytest.mark.parametrize("h", [0.0, 0.1])
def test_4d_2222_lattice_vs_enumeration(h):
    """The 2^4 periodic lattice (2^16 states): two untruncated steps, then the
    remaining 1x1x2x2 network of coarse tensors contracted exactly."""
    beta = BETA_C4D
    st = H.HOTRG.start(4, beta, h)
    st.step(0, 10 ** 6)
    st.step(1, 10 ** 6)
    lnz = st.lnz_acc + math.log(H.contract_periodic(st.T, (1, 1, 2, 2))) / 16
    assert lnz == pytest.approx(E.enumerate_lattice((2, 2, 2, 2), beta, h)["lnZ_over_V"], abs=1e-13)


def test_2d_4x4_vs_enumeration():
    beta, h = 0.4, 0.05
    st = H.HOTRG.start(2, beta, h, impure=True)
    for i in range(4):
        st.step(i % 2, 10 ** 6)
    ex = E.enumerate_lattice((4, 4), beta, h)
    assert st.lnZ() == pytest.approx(ex["lnZ_over_V"], abs=1e-13)
    assert st.magnetization() == pytest.approx(ex["sigma"], abs=1e-12)
    assert st.sigma_sigma() == pytest.approx(ex["sigma_sigma_x"], abs=1e-12)


def test_3d_2x2x2_vs_enumeration():
    beta, h = 0.25, 0.07
    st = H.HOTRG.start(3, beta, h, impure=True)
    for i in range(3):
        st.step(i, 10 ** 6)
    ex = E.enumerate_lattice((2, 2, 2), beta, h)
    assert st.lnZ() == pytest.approx(ex["lnZ_over_V"], abs=1e-13)
    assert st.magnetization() == pytest.approx(ex["sigma"], abs=1e-12)
    assert st.sigma_sigma() == pytest.approx(ex["sigma_sigma_x"], abs=1e-12)


def test_direction_order_invariance_untruncated():
    """Without truncation the 2x2x1x1 lattice does not care which step comes first."""
    beta, h = 0.3, 0.05
    a = H.run(4, beta, h, 10 ** 6, 2, order=[0, 1])
    b = H.run(4, beta, h, 10 ** 6, 2, order=[1, 0])
    assert a.lnZ() == pytest.approx(b.lnZ(), abs=1e-13)


# ---------------------------------------------------------------- closed forms
def test_onsager_two_forms_agree():
    for beta in (0.2, 0.44, 0.7):
        assert E.onsager_lnz(beta) == pytest.approx(E.onsager_lnz(beta, "double"), abs=1e-11)


def test_onsager_energy_is_derivative():
    """u = -d(ln Z/N)/d beta, by a central difference of the closed form."""
    for beta in (0.3, 0.6):
        dh = 1e-5
        num = -(E.onsager_lnz(beta + dh) - E.onsager_lnz(beta - dh)) / (2 * dh)
        assert E.onsager_energy_2d(beta) == pytest.approx(num, abs=1e-8)


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_2d_hotrg_vs_onsager(beta):
    """2D HOTRG, D_cut = 16, 2^15 x 2^15 sites, away from beta_c: error < 1e-8.
    (In the ordered phase the finite lattice adds ln 2 / V; V = 2^30 makes it 6e-10.)"""
    st = H.run(2, beta, 0.0, 16, 30)
    assert st.lnZ() == pytest.approx(E.onsager_lnz(beta), abs=1e-8)


@pytest.mark.slow
def test_2d_impure_energy_and_magnetization():
    """sigma-sigma impure tensor -> exact 2D energy; sigma impure -> Yang's m (h -> 0+:
    beta h V = 0.6e-6 * 2^30 >> 1 selects one ordered state)."""
    beta = 0.6
    st = H.run(2, beta, 1e-6, 12, 30, impure=True)
    assert -2 * st.sigma_sigma() == pytest.approx(E.onsager_energy_2d(beta), abs=2e-4)
    assert st.magnetization() == pytest.approx(E.yang_magnetization(beta), abs=2e-4)
    hot = H.run(2, 0.3, 0.0, 12, 24, impure=True)
    assert -2 * hot.sigma_sigma() == pytest.approx(E.onsager_energy_2d(0.3), abs=2e-4)


def test_high_temperature_series_2d():
    """2D: ln 2 + 2 ln cosh b + t^4 + 2 t^6 + O(t^8), exact to 1e-12 at b = 0.02."""
    assert E.high_temperature_coeffs(2) == (1, 2)
    assert E.high_temperature_coeffs(3) == (3, 22)
    st = H.run(2, 0.02, 0.0, 8, 10)
    assert st.lnZ() == pytest.approx(E.high_temperature_lnz(2, 0.02), abs=1e-12)


def test_high_temperature_series_4d_bounds():
    """4D, 16^4, D_cut = 5: HOTRG keeps the single-excitation bond states only, so it
    recovers a fraction of the plaquette term 6 t^4; it may not overshoot it, and the
    ln 2 + 4 ln cosh b part is exact."""
    beta = 0.02
    st = H.run(4, beta, 0.0, 5, 16)
    base = E.high_temperature_lnz(4, beta, 0)
    t4 = 6 * math.tanh(beta) ** 4
    assert 0.4 * t4 < st.lnZ() - base < 1.05 * t4


def test_z2_symmetry():
    """h = 0: <sigma> = 0 exactly, in the disordered phase near T_c and at T = 8."""
    for T in (6.65, 8.0):
        st = H.run(4, 1 / T, 0.0, 4, 8, impure=True)
        assert abs(st.magnetization()) < 1e-12


# ---------------------------------------------------------------- brute force on tiny inputs
def _pair_tensor(T1, T2, mu):
    """M with legs [T1.mu, T2.mu', then for each nu != mu: (T1.nu,T2.nu), (T1.nu',T2.nu')]."""
    d = T1.ndim // 2
    L = "abcdefghijklmnopqrstuvwxyz"
    l1 = list(L[: 2 * d])
    l2 = list(L[2 * d: 4 * d])
    k = "Z"
    l1[2 * mu + 1] = k
    l2[2 * mu] = k
    out = [l1[2 * mu], l2[2 * mu + 1]]
    for n in range(d):
        if n != mu:
            out += [l1[2 * n], l2[2 * n], l1[2 * n + 1], l2[2 * n + 1]]
    M = np.einsum(f"{''.join(l1)},{''.join(l2)}->{''.join(out)}", T1, T2)
    shape = [T1.shape[2 * mu], T2.shape[2 * mu + 1]]
    for n in range(d):
        if n != mu:
            D = T1.shape[2 * n]
            shape += [D * D, D * D]
    return M.reshape(shape)


def _random_tensor(rng, dims):
    return rng.standard_normal(tuple(x for D in dims for x in (D, D)))


@pytest.mark.parametrize("dims,mu", [((2, 3, 2, 2), 0), ((3, 2, 2, 3), 2), ((2, 3), 1), ((2, 2, 3), 0)])
def test_gram_vs_explicit_pair_tensor(dims, mu):
    rng = np.random.default_rng(7)
    T1 = _random_tensor(rng, dims)
    T2 = _random_tensor(rng, dims)
    M = _pair_tensor(T1, T2, mu)
    d = len(dims)
    pos = 2
    for n in range(d):
        if n == mu:
            continue
        for primed in (False, True):
            Mp = np.moveaxis(M, pos + (1 if primed else 0), 0).reshape(M.shape[pos], -1)
            assert np.allclose(H.gram(T1, T2, mu, n, primed), Mp @ Mp.T, rtol=1e-12, atol=1e-12)
        pos += 2


@pytest.mark.parametrize("dims,mu", [((2, 3, 2, 2), 1), ((2, 2, 3, 2), 3), ((3, 2), 0), ((2, 3, 2), 2)])
def test_coarse_grain_vs_full_network(dims, mu):
    """T' from the oracle's contraction order = one einsum of the whole network,
    with truncating (chi < D^2), direction-specific random isometries."""
    rng = np.random.default_rng(11)
    d = len(dims)
    T1 = _random_tensor(rng, dims)
    T2 = _random_tensor(rng, dims)
    U = {}
    for n in range(d):
        if n != mu:
            D = dims[n]
            chi = max(1, D * D - 2 - n)
            U[n] = np.linalg.qr(rng.standard_normal((D * D, chi)))[0].reshape(D, D, chi)
    got = H.coarse_grain(T1, T2, U, mu)
    M = _pair_tensor(T1, T2, mu)
    # apply the isometries to the fused legs of M explicitly
    out = M
    pos = 2
    for n in range(d):
        if n == mu:
            continue
        Um = U[n].reshape(-1, U[n].shape[2])
        out = np.moveaxis(np.tensordot(out, Um, axes=([pos], [0])), -1, pos)
        out = np.moveaxis(np.tensordot(out, Um, axes=([pos + 1], [0])), -1, pos + 1)
        pos += 2
    # out legs: [mu, mu', (X_n, Y_n) for n != mu]  -> oracle order [.., n, n', ..]
    perm = []
    pos = 2
    for n in range(d):
        if n == mu:
            perm += [0, 1]
        else:
            perm += [pos, pos + 1]
            pos += 2
    assert np.allclose(got, np.transpose(out, perm), rtol=1e-12, atol=1e-12)


def test_isometry_is_best_side_and_eps_is_projection_loss():
    """eps = ||M||^2 - ||U^T M||^2 on each side (explicit projection); the side taken
    is the one with the smaller eps; U = leading eigenvectors of M M^T."""
    rng = np.random.default_rng(5)
    dims, mu = (2, 3, 2, 2), 0
    T = _random_tensor(rng, dims)
    T = T + 0.3 * np.swapaxes(T, 2, 3)        # unequal nu / nu' sides
    M = _pair_tensor(T, T, mu)
    for n, pos in ((1, 2), (2, 4), (3, 6)):
        D = dims[n]
        chi = D * D - 2
        iso = H.isometry(T, T, mu, n, chi)
        losses = []
        for primed in (False, True):
            Mp = np.moveaxis(M, pos + (1 if primed else 0), 0).reshape(D * D, -1)
            lam, V = np.linalg.eigh(Mp @ Mp.T)
            Uside = V[:, np.argsort(-lam)[:chi]]
            losses.append(np.sum(Mp ** 2) - np.sum((Uside.T @ Mp) ** 2))
        assert iso.eps == pytest.approx(tuple(losses), rel=1e-9, abs=1e-12)
        assert iso.primed == (losses[1] < losses[0])
        Mp = np.moveaxis(M, pos + (1 if iso.primed else 0), 0).reshape(D * D, -1)
        P = iso.U.reshape(D * D, chi)
        assert np.allclose(P.T @ P, np.eye(chi), atol=1e-13)
        assert np.sum((P.T @ Mp) ** 2) == pytest.approx(np.sum(Mp ** 2) - min(losses), rel=1e-10)


def test_canonical_basis_depends_only_on_eigenspaces():
    rng = np.random.default_rng(3)
    n = 9
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    lam = np.array([5.0, 3.0, 3.0, 3.0, 2.0, 1.0, 1.0, 0.5, 0.1])
    G = (Q * lam) @ Q.T
    l1, V1 = H.eig_desc(G)
    # another orthonormal eigenbasis: rotate inside each degenerate block
    V2 = Q.copy()
    R = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    V2[:, 1:4] = V2[:, 1:4] @ R
    R = np.linalg.qr(rng.standard_normal((2, 2)))[0]
    V2[:, 5:7] = V2[:, 5:7] @ R
    V2 = V2 * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    C2 = H.canonical_basis(lam, V2)
    assert np.allclose(V1, C2, atol=1e-12)
    assert np.allclose(V1.T @ V1, np.eye(n), atol=1e-13)
    assert np.allclose(G @ V1, V1 * l1, atol=1e-12)
    for j in range(n):          # simple eigenvalue or not: first largest entry positive
        a = np.abs(V1[:, j])
        i = int(np.argmax(a >= (1 - 1e-8) * a.max()))
        assert V1[i, j] > 0 or j in (2, 3, 6)


def test_gauge_rotation_leaves_lnz_unchanged():
    """A random orthogonal rotation of a full (untruncated) isometry is a gauge change."""
    rng = np.random.default_rng(2)
    beta = 0.35
    st = H.HOTRG.start(4, beta, 0.0)
    st.step(0, 10 ** 6)
    T = st.T
    U = {n: H.isometry(T, T, 1, n, 10 ** 6).U for n in (0, 2, 3)}
    U2 = {}
    for n, u in U.items():
        D, chi = u.shape[0], u.shape[2]
        O = np.linalg.qr(rng.standard_normal((chi, chi)))[0]
        U2[n] = (u.reshape(-1, chi) @ O).reshape(D, D, chi)
    a = H.HOTRG(4, beta, 0.0, T.copy(), None, None, st.lnz_acc, 1)
    b = H.HOTRG(4, beta, 0.0, T.copy(), None, None, st.lnz_acc, 1)
    a.step(1, 10 ** 6, U)
    b.step(1, 10 ** 6, U2)
    assert a.lnZ() == pytest.approx(b.lnZ(), abs=1e-13)
    assert a.lnZ() == pytest.approx(E.enumerate_lattice((2, 2, 1, 1), beta, 0.0)["lnZ_over_V"], abs=1e-13)


def test_lnz_accumulator_weights():
    """ln Z/V does not depend on the normalisation constants (Z = prod c_i^(V/2^i) Tr T_k):
    scaling T_k by any factor a and adding -ln(a)/2^k leaves it unchanged, while the
    accumulated sum of ln c_i / 2^i is what ties the steps to the volume 2^k."""
    st = H.run(4, BETA_C4D, 0.0, 4, 3)
    ref = st.lnZ()
    st.T = st.T * 7.0
    st.lnz_acc -= math.log(7.0) / 2 ** st.k
    assert st.lnZ() == pytest.approx(ref, abs=1e-14)
    manual = sum(r.ln_c / 2 ** (i + 1) for i, r in enumerate(st.history))
    c0 = np.linalg.norm(H.ising_tensors(4, BETA_C4D, 0.0)[0])
    assert st.lnz_acc + math.log(7.0) / 2 ** st.k == pytest.approx(math.log(c0) + manual, abs=1e-14)


# ---------------------------------------------------------------- X indicator (Sec. 3.1)
@pytest.mark.parametrize("dims", [(3, 2), (2, 3, 2, 2)])
def test_x_indicator_vs_two_site_network(dims):
    """Brute force: Tr(M M) is the periodic two-site network along nu (each other leg
    closing on itself), contracted as one einsum; Tr M is the one-site trace."""
    rng = np.random.default_rng(31)
    d = len(dims)
    shape = sum(([n, n] for n in dims), [])
    T = rng.standard_normal(shape)
    for nu in range(d):
        ext = [1] * d
        ext[nu] = 2
        want = H.trace(T) ** 2 / H.contract_periodic(T, ext)
        assert H.x_indicator(T, nu) == pytest.approx(want, rel=1e-12)


def test_x_indicator_counts_degenerate_leading_states():
    """X = (sum m)^2 / sum m^2 for the eigenvalues m of the transfer matrix: a tensor whose
    transfer matrix is diag(1, 1, 0) gives 2, diag(1, 0, 0) gives 1 (all other legs of
    dimension 1)."""
    for diag, want in (((1.0, 1.0, 0.0), 2.0), ((1.0, 0.0, 0.0), 1.0), ((1.0, 1.0, 1.0), 3.0)):
        T = np.diag(diag).reshape(3, 3, 1, 1)
        assert H.x_indicator(T, 0) == pytest.approx(want, rel=1e-14)


def test_x_indicator_brackets_onsager_tc_2d():
    """2D Ising: bisection on X = 1.5 after 24 steps (a 4096^2 lattice) at D_cut = 12 lands
    on Onsager's T_c = 2 / ln(1 + sqrt 2) to 5e-4: X is 2 below it and 1 above it."""
    tc = 2 / math.log(1 + math.sqrt(2))
    lo, hi = 2.2, 2.35
    assert H.x_indicator(H.run(2, 1 / lo, 0.0, 12, 24).T) > 1.9
    assert H.x_indicator(H.run(2, 1 / hi, 0.0, 12, 24).T) < 1.1
    for _ in range(8):
        mid = 0.5 * (lo + hi)
        if H.x_indicator(H.run(2, 1 / mid, 0.0, 12, 24).T) > 1.5:
            lo = mid
        else:
            hi = mid
    assert abs(0.5 * (lo + hi) - tc) / tc < 5e-4


def test_x_indicator_4d_phases():
    """4D, D_cut = 4, 16 steps (16^4): X near 2 deep in the ordered phase (T = 5), near 1
    in the symmetric phase (T = 9), in every direction."""
    lo = H.run(4, 1 / 5.0, 0.0, 4, 16).T
    hi = H.run(4, 1 / 9.0, 0.0, 4, 16).T
    for nu in range(4):
        assert abs(H.x_indicator(lo, nu) - 2.0) < 0.01
        assert abs(H.x_indicator(hi, nu) - 1.0) < 0.05
