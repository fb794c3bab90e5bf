"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: only the parameters of the
workloads (temperatures, fields, bond-dimension cuts, lattice sizes) and seeded
random tensors for kernel-level parity cases. The Ising site tensor itself is
built separately by the oracle (FP64 NumPy) and by the CUDA path (device kernel).

Workloads (4D Ising, J = 1, periodic lattice of 2^steps sites, directions cycled
x, y, z, t):

* ``ising16``    : T = 6.65, h = 0, D_cut = 4, 16 steps (16^4 sites).
* ``ising1024``  : T = 6.65, h = 0, D_cut = 8, 40 steps (1024^4 sites).
* ``mixed1024``  : T = 6.65, h = 0, D_cut in {10, 11, 12}, 40 steps.
* ``sweep32``    : 32 temperatures evenly spaced in [6.60, 6.72], D_cut = 8,
                   pure + sigma-impure (h = 1e-5) + sigma-sigma-impure tensors.
* ``sweep8``     : 8 temperatures in [6.66, 6.70], D_cut = 13.
"""

from __future__ import annotations

import numpy as np

T_NEAR_TC = 6.65          # just above T_c(D_cut = 13) = 6.650365 (Sec. 3.1 of the paper)

WORKLOADS = {
    "ising16": dict(temps=[T_NEAR_TC], h=0.0, dcut=4, steps=16),
    "ising1024": dict(temps=[T_NEAR_TC], h=0.0, dcut=8, steps=40),
    "mixed1024": dict(temps=[T_NEAR_TC], h=0.0, dcut=(10, 11, 12), steps=40),
    "sweep32": dict(temps=list(np.linspace(6.60, 6.72, 32)), h=1e-5, dcut=8, steps=40),
    "sweep8": dict(temps=list(np.linspace(6.66, 6.70, 8)), h=1e-5, dcut=13, steps=40),
}


def betas(temps):
    """Inverse temperatures for a list of temperatures."""
    return [1.0 / float(T) for T in temps]


def direction(step_index: int, d: int = 4) -> int:
    """Direction of coarse-graining step ``step_index`` (0-based): x, y, z, t, x, ..."""
    return step_index % d


def random_tensor(seed: int, dims, scale: float = 1.0) -> np.ndarray:
    """N(0, scale^2) FP64 tensor with legs (D0, D0, D1, D1, ...) from a seeded generator."""
    rng = np.random.default_rng(seed)
    shape = tuple(x for D in dims for x in (D, D))
    return scale * rng.standard_normal(shape)


def decaying_tensor(seed: int, dims, rate: float = 0.6) -> np.ndarray:
    """Seeded tensor whose entries fall off with the leg indices like a coarse-grained
    Ising tensor (entry ~ N(0,1) * rate^(sum of indices)), for dynamic-range tests."""
    t = random_tensor(seed, dims)
    idx = np.indices(t.shape).sum(axis=0)
    return t * rate ** idx
