"""Locating T_c from the degeneracy indicator X, and temperature scans of the internal
energy and the magnetisation (Sec. 3.1 of arXiv:1911.12954).

After the full schedule of coarse-graining steps X is close to 2 below T_c, where Z2 is
broken, and close to 1 above it (``hotrg_x_indicator``). ``bracket_tc`` narrows a
temperature interval around the crossing of X = 1.5: each round evaluates X at ``batch``
temperatures spread evenly over the current interval, in one batched run (each temperature
is one batch element of the same ``hotrg_step`` calls), and keeps the sub-interval in which X
crosses. Every round divides the interval by ``batch - 1``. ``observable_scan`` runs the
pure and impure tensors of many temperatures together and records E/V and <sigma> per volume;
``largest_jump`` reads the discontinuity off a scan. Host logic only: the tensors, steps, X,
E and m are computed by the CUDA library.
"""

from __future__ import annotations

import numpy as np

LEVEL = 1.5   # X crosses from ~2 (ordered) to ~1 (symmetric)


def crossing(temps, X, level: float = LEVEL):
    """Index i of the first adjacent pair (temperatures increasing) with X[i] > level >= X[i+1],
    or None when X does not cross the level on this grid."""
    temps = np.asarray(temps, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    if temps.ndim != 1 or temps.shape != X.shape or len(temps) < 2:
        raise ValueError("temps and X must be equal-length 1D arrays of at least two values")
    if np.any(np.diff(temps) <= 0):
        raise ValueError("temps must increase")
    for i in range(len(temps) - 1):
        if X[i] > level >= X[i + 1]:
            return i
    return None


def x_sweep(temps, dcut: int, nsteps: int = 40, precision: str = "fp16x3", h: float = 0.0, nu: int = 0,
            device=None, graphs: bool = False):
    """X after ``nsteps`` steps (directions x, y, z, t cycled, every cut ``dcut``) at each
    temperature of ``temps``, all in one batched run."""
    from .hotrg import HOTRG

    temps = np.asarray(temps, dtype=np.float64)
    sched = [(i % 4, dcut) for i in range(nsteps)]
    run = HOTRG(batch=len(temps), dcut_max=dcut, precision=precision, schedule=sched, device=device, graphs=graphs)
    run.init_tensor(1.0 / temps, h)
    for mu, dc in sched:
        run.step(mu, dc)
    return run.x_indicator(nu)


def bracket_tc(dcut: int, lo: float, hi: float, nsteps: int = 40, batch: int = 8, rounds: int = 3,
               precision: str = "fp16x3", h: float = 0.0, nu: int = 0, device=None):
    """Interval (T_lo, T_hi) with X(T_lo) > 1.5 >= X(T_hi) after ``rounds`` rounds of
    ``batch`` temperatures each, and the (temps, X) of every round."""
    if not (hi > lo) or batch < 2:
        raise ValueError("need hi > lo and batch >= 2")
    history = []
    for _ in range(rounds):
        temps = np.linspace(lo, hi, batch)
        X = x_sweep(temps, dcut, nsteps, precision, h, nu, device)
        history.append((temps, X))
        i = crossing(temps, X)
        if i is None:
            raise ValueError(f"X does not cross {LEVEL} in [{lo}, {hi}]: {X}")
        lo, hi = float(temps[i]), float(temps[i + 1])
    return lo, hi, history


def observable_scan(temps, dcut: int, nsteps: int = 40, h: float = 1e-5, precision: str = "fp16x3",
                    record_from: int = 24, device=None):
    """Internal energy and magnetisation against temperature for growing volumes (the scans of
    Sec. 3.1, Figs. 5 and 6): one batched run of the pure tensor with the sigma- and
    sigma-sigma-impure tensors at every temperature of ``temps`` (field h, which picks one of
    the two vacua below T_c), directions x, y, z, t cycled. After every step k >= record_from
    (volume 2^k) it records E/V, <sigma> and ln Z/V per temperature; returns a list of
    {"k", "E", "m", "lnZ"} with one value per temperature in each."""
    from .hotrg import HOTRG, IMPURE_SIGMA, IMPURE_SIGMASIGMA

    temps = np.asarray(temps, dtype=np.float64)
    sched = [(i % 4, dcut) for i in range(nsteps)]
    run = HOTRG(batch=len(temps), dcut_max=dcut, precision=precision, impure=IMPURE_SIGMA | IMPURE_SIGMASIGMA,
                schedule=sched, device=device)
    run.init_tensor(1.0 / temps, h)
    rows = []
    for k, (mu, dc) in enumerate(sched, 1):
        run.step(mu, dc)
        if k >= record_from:
            e, _ = run.energy()
            rows.append({"k": k, "E": e.copy(), "m": run.magnetization().copy(), "lnZ": run.lnZ().copy()})
    return rows


def largest_jump(temps, values):
    """(i, jump): the adjacent pair (temps[i], temps[i+1]) across which ``values`` changes
    most, and that change values[i+1] - values[i]. On a fine grid across a first-order
    transition this is the discontinuity (latent heat for E, the magnetisation jump for m)
    up to the grid's resolution."""
    temps = np.asarray(temps, dtype=np.float64)
    v = np.asarray(values, dtype=np.float64)
    if temps.ndim != 1 or temps.shape != v.shape or len(temps) < 2:
        raise ValueError("temps and values must be equal-length 1D arrays of at least two values")
    if np.any(np.diff(temps) <= 0):
        raise ValueError("temps must increase")
    d = np.diff(v)
    i = int(np.argmax(np.abs(d)))
    return i, float(d[i])
