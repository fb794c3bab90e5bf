"""Independent exact results that pin the HOTRG oracle (test infrastructure only).

Nothing here uses tensors: these are the textbook results the tensor network must
reproduce.

* ``enumerate_lattice``: brute force over all 2**V spin states of a periodic
  hypercubic lattice with bonds (n, n + e_nu mod L_nu) for every site and
  direction (an extent-1 direction gives a self bond, an extent-2 direction two
  bonds between the same pair, exactly as the tensor network of Fig. 1A counts them).
* ``onsager_lnz``: the free energy of the 2D Ising model on the infinite square
  lattice (Onsager 1944), in two forms (double integral and the one-dimensional
  elliptic form) that the tests compare with each other.
* ``onsager_energy_2d``: the exact 2D internal energy per site.
* ``yang_magnetization``: the exact 2D spontaneous magnetisation (Yang 1952).
* ``high_temperature_lnz``: the hypercubic-lattice high-temperature series
  ln Z/V = ln 2 + d ln cosh b + c4 t^4 + c6 t^6 + O(t^8), t = tanh b, with
  c4 = d(d-1)/2 (plaquettes per site) and c6 = d(d-1) + 16 C(d,3) (1x2
  rectangles plus the non-planar six-cycles of each unit cube).
"""

from __future__ import annotations

import math
from itertools import product

import numpy as np
from scipy import integrate, special


def enumerate_lattice(extents, beta: float, h: float = 0.0):
    """Exact ln Z / V, <sigma_0> and <sigma_0 sigma_(0+x)> by summing all 2**V states.

    H = -sum_bonds s s' - h sum_n s_n; weight exp(-beta H).
    """
    d = len(extents)
    sites = list(product(*[range(L) for L in extents]))
    V = len(sites)
    if V > 22:
        raise ValueError("too many sites to enumerate")
    index = {s: i for i, s in enumerate(sites)}
    bonds = []
    for s in sites:
        for n in range(d):
            t = list(s)
            t[n] = (t[n] + 1) % extents[n]
            bonds.append((index[s], index[tuple(t)]))
    states = ((np.arange(2 ** V)[:, None] >> np.arange(V)[None, :]) & 1)
    spins = 1.0 - 2.0 * states                       # bit 0 -> +1, bit 1 -> -1
    a = np.array([b[0] for b in bonds])
    b = np.array([b[1] for b in bonds])
    E = (spins[:, a] * spins[:, b]).sum(axis=1)
    M = spins.sum(axis=1)
    logw = beta * E + beta * h * M
    shift = logw.max()
    w = np.exp(logw - shift)
    Z = w.sum()
    x1 = index[tuple(1 % L if n == 0 else 0 for n, L in enumerate(extents))]
    return {
        "lnZ_over_V": (math.log(Z) + shift) / V,
        "sigma": float((w * spins[:, 0]).sum() / Z),
        "sigma_sigma_x": float((w * spins[:, 0] * spins[:, x1]).sum() / Z),
        "V": V,
    }


def onsager_lnz(beta: float, form: str = "elliptic") -> float:
    """ln Z / N of the infinite 2D Ising model, J = 1, h = 0."""
    if form == "double":
        c2 = math.cosh(2 * beta) ** 2
        s2 = math.sinh(2 * beta)
        f = lambda t1, t2: math.log(c2 - s2 * (math.cos(t1) + math.cos(t2)))
        val, _ = integrate.dblquad(f, 0, 2 * math.pi, 0, 2 * math.pi, epsabs=1e-13, epsrel=1e-13)
        return math.log(2.0) + val / (8 * math.pi ** 2)
    kappa = 2 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    f = lambda p: math.log(0.5 * (1 + math.sqrt(max(0.0, 1 - (kappa * math.sin(p)) ** 2))))
    val, _ = integrate.quad(f, 0, math.pi / 2, epsabs=1e-14, epsrel=1e-14, limit=200)
    return math.log(2 * math.cosh(2 * beta)) + val / math.pi


def onsager_energy_2d(beta: float) -> float:
    """Internal energy per site u = -d ln Z/N / d beta of the infinite 2D Ising model."""
    kappa = 2 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    K = special.ellipk(kappa ** 2)          # scipy takes the parameter m = k^2
    return -(1 / math.tanh(2 * beta)) * (1 + (2 / math.pi) * (2 * math.tanh(2 * beta) ** 2 - 1) * K)


def yang_magnetization(beta: float) -> float:
    """Spontaneous magnetisation of the 2D Ising model; 0 above T_c."""
    beta_c = 0.5 * math.log(1 + math.sqrt(2))
    if beta <= beta_c:
        return 0.0
    return (1 - math.sinh(2 * beta) ** -4) ** 0.125


def high_temperature_coeffs(d: int):
    """(c4, c6) of ln Z/V on the infinite d-dim hypercubic lattice."""
    c4 = d * (d - 1) // 2
    c6 = d * (d - 1) + 16 * math.comb(d, 3)
    return c4, c6


def high_temperature_lnz(d: int, beta: float, order: int = 6) -> float:
    t = math.tanh(beta)
    c4, c6 = high_temperature_coeffs(d)
    val = math.log(2.0) + d * math.log(math.cosh(beta))
    if order >= 4:
        val += c4 * t ** 4
    if order >= 6:
        val += c6 * t ** 6
    return val


def ising_trace_single_site(d: int, beta: float, h: float) -> float:
    """Z of one site whose d bonds all close on itself: 2 e^(d beta) cosh(beta h)."""
    return 2.0 * math.exp(d * beta) * math.cosh(beta * h)
