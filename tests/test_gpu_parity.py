"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 mode must agree with the oracle to rounding (1e-10 relative on ln Z / V, the bar
for the FP64 path); FP32 and TF32x3 modes within the error their arithmetic allows,
stated per test. Inputs are the Ising site tensors (any T, h) and seeded random
tensors from ``workloads`` with non-uniform and odd bond dimensions; single steps are
compared element by element (tensors and isometries in the canonical gauge), runs on
gauge-invariant quantities (ln Z / V, <sigma>, <sigma sigma>, discarded sums).
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import hotrg as H
from workloads import decaying_tensor, random_tensor

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gpu(**kw):
    from paper_1911_12954_gb300 import HOTRG
    return HOTRG(**kw)


def _golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


# ------------------------------------------------------------------ site tensor, k = 0
def test_init_tensor_lnz_and_magnetization():
    betas = np.array([0.0, 0.1, 1 / 6.65, 0.7])
    hs = np.array([0.0, 0.3, 1e-5, -0.2])
    g = _gpu(batch=4, dcut_max=4, precision="fp64", impure=3, schedule=[(0, 4)])
    g.init_tensor(betas, hs)
    lnz = g.lnZ()
    m = g.magnetization()
    for i in range(4):
        st = H.HOTRG.start(4, betas[i], hs[i], impure=True)
        assert lnz[i] == pytest.approx(st.lnZ(), abs=1e-14)
        assert m[i] == pytest.approx(st.magnetization(), abs=1e-14)
        assert g.tensor(0, i) == pytest.approx(st.T, abs=1e-15)


# ------------------------------------------------------------------ single steps on random tensors
CASES = [
    # dims (Dx, Dy, Dz, Dt), mu, dcut
    ((2, 3, 2, 3), 1, 5),
    ((3, 2, 2, 2), 0, 4),
    ((2, 2, 3, 2), 3, 9),       # no truncation: chi = D^2 everywhere
    ((4, 3, 2, 3), 2, 7),
    ((3, 3, 3, 3), 3, 1),       # chi = 1
    ((2, 4, 3, 2), 1, 6),
]


@pytest.mark.parametrize("dims,mu,dcut", CASES)
def test_single_step_random_tensor_fp64(dims, mu, dcut):
    T = random_tensor(1000 + sum(dims) * 7 + mu, dims)
    ref = H.HOTRG.from_tensor(T)
    trans = [n for n in range(4) if n != mu]
    isos = {n: H.isometry(ref.T, ref.T, mu, n, dcut) for n in trans}
    ref.step(mu, dcut)
    g = _gpu(batch=1, dcut_max=max(max(dims), dcut, 2), precision="fp64", schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    k, newdims = g.state()
    assert k == 1 and newdims == ref.history[0].dims_out
    Tg = g.tensor()
    scale = np.abs(ref.T).max()
    assert np.allclose(Tg, ref.T, rtol=0, atol=1e-12 * scale)
    info = g.step_info(1)
    assert info["ln_c"] == pytest.approx(ref.history[0].ln_c, abs=1e-12)
    for n in trans:
        Ug = g.isometry(n, dold=dims[n], chi=isos[n].chi)
        assert np.allclose(Ug, isos[n].U, atol=1e-11), n
        assert info["primed"][n] == int(isos[n].primed)
        assert info["eps"][n] == pytest.approx(isos[n].eps, rel=1e-9, abs=1e-13)


def _z2_tensor(seed, dims):
    """A random tensor with the Z2 structure of the h = 0 Ising tensors: index i of a leg has
    charge i mod 2 and every entry of odd total charge is exactly zero."""
    T = random_tensor(seed, dims)
    shape = T.shape
    parity = np.zeros(shape, dtype=np.int64)
    for leg, n in enumerate(shape):
        idx = (np.arange(n) % 2).reshape([n if l == leg else 1 for l in range(len(shape))])
        parity = parity + idx
    T[parity % 2 == 1] = 0.0
    return T


@pytest.mark.parametrize("dims,sched", [((4, 2, 3, 2), [(0, 6), (3, 6)]), ((3, 2, 4, 2), [(2, 5), (0, 5)])])
def test_z2_structured_steps_fp64(dims, sched):
    """Two steps from a Z2-structured random tensor (the Gram matrices split into charge
    blocks, so the eigensolver runs one tournament per block): tensors, isometries, records
    and ln c equal the oracle's, and the entries the oracle's tensor has at rounding level
    (below 1e-11 of its largest; its eigh mixes the charge sectors at ~1e-14 here, the
    structural entries are above 1e-7) are exact zeros on the GPU."""
    T = _z2_tensor(77 + sum(dims), dims)
    ref = H.HOTRG.from_tensor(T)
    g = _gpu(batch=1, dcut_max=max(max(dims), 6), precision="fp64", schedule=sched, dims0=dims)
    g.set_tensor(T)
    for k, (mu, dcut) in enumerate(sched, 1):
        trans = [n for n in range(4) if n != mu]
        dims_k = ref.history[-1].dims_out if ref.history else dims
        isos = {n: H.isometry(ref.T, ref.T, mu, n, dcut) for n in trans}
        ref.step(mu, dcut)
        g.step(mu, dcut)
        Tg = g.tensor()
        scale = np.abs(ref.T).max()
        assert np.allclose(Tg, ref.T, rtol=0, atol=1e-12 * scale), k
        assert np.all(Tg[np.abs(ref.T) < 1e-11 * scale] == 0.0), k
        info = g.step_info(k)
        assert info["ln_c"] == pytest.approx(ref.history[-1].ln_c, abs=1e-12)
        for n in trans:
            Ug = g.isometry(n, dold=dims_k[n], chi=isos[n].chi)
            assert np.allclose(Ug, isos[n].U, atol=1e-11), (k, n)
            assert info["eps"][n] == pytest.approx(isos[n].eps, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-5), ("tf32x3", 3e-5), ("fp16x3", 3e-5)])
@pytest.mark.parametrize("dims,mu,dcut", [CASES[0], CASES[3], CASES[5]])
def test_single_step_random_tensor_mixed(prec, tol, dims, mu, dcut):
    T = random_tensor(2000 + sum(dims) * 7 + mu, dims)
    ref = H.HOTRG.from_tensor(T)
    ref.step(mu, dcut)
    g = _gpu(batch=1, dcut_max=max(max(dims), dcut, 2), precision=prec, schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    Tg = g.tensor()
    scale = np.abs(ref.T).max()
    err = np.abs(Tg - ref.T).max() / scale
    assert err < tol, err
    assert g.step_info(1)["ln_c"] == pytest.approx(ref.history[0].ln_c, abs=tol)


def test_sliced_contraction_matches_unsliced():
    """A workspace too small for the unsliced contraction makes the step slice the new
    a-leg; the result is the same to rounding."""
    dims, mu, dcut = (3, 3, 3, 3), 0, 6
    T = random_tensor(77, dims)
    full = _gpu(batch=1, dcut_max=6, precision="fp64", schedule=[(mu, dcut)], dims0=dims)
    full.set_tensor(T)
    full.step(mu, dcut)
    need = full.workspace_size([(mu, dcut)], dims)
    small = _gpu(batch=1, dcut_max=6, precision="fp64", schedule=[(mu, dcut)], dims0=dims,
                 workspace_bytes=int(need * 0.55))
    small.set_tensor(T)
    small.step(mu, dcut)
    assert np.allclose(small.tensor(), full.tensor(), atol=1e-14)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("tf32x3", 1e-6), ("fp16x3", 1e-6)])
def test_two_dimensional_slicing_matches_unsliced(prec, tol):
    """Workspaces between the smallest that works and the unsliced plan make the step
    slice the new X (rows of A) and then also the new X' (rows of B, columns of C); every
    slicing gives the unsliced tensor, and a workspace below the smallest is refused."""
    from paper_1911_12954_gb300 import HotrgError
    dims, mu, dcut = (4, 2, 4, 2), 2, 9
    T = random_tensor(78, dims)

    def run(nbytes):
        g = _gpu(batch=1, dcut_max=9, precision=prec, schedule=[(mu, dcut)], dims0=dims, workspace_bytes=nbytes)
        g.set_tensor(T)
        g.step(mu, dcut)
        return g.tensor(), g.step_info(1)["slices"]

    full = _gpu(batch=1, dcut_max=9, precision=prec, schedule=[(mu, dcut)], dims0=dims)
    need = full.workspace_size([(mu, dcut)], dims)
    ref, sl = run(need)
    assert sl == (1, 1)
    lo, hi = 0, need                      # smallest workspace that runs, by bisection
    while hi - lo > 4096:
        mid = (lo + hi) // 2 // 256 * 256
        try:
            run(mid)
            hi = mid
        except HotrgError as e:
            assert "EWORKSPACE" in str(e)
            lo = mid
    seen = set()
    for frac in (0.0, 0.1, 0.25, 0.5, 0.75):
        nbytes = (hi + int((need - hi) * frac)) // 256 * 256 + 256
        Tn, sl = run(nbytes)
        seen.add(sl)
        assert np.allclose(Tn, ref, atol=tol * np.abs(ref).max()), (frac, sl)
    assert any(a > 1 and b > 1 for a, b in seen), seen
    with pytest.raises(HotrgError, match="EWORKSPACE"):
        run(lo // 256 * 256)


# ------------------------------------------------------------------ Ising runs
def test_untruncated_two_steps_impure_vs_oracle():
    """Two untruncated steps (dims 4,4,16,16) = the exactly enumerable 2x2x1x1 lattice."""
    betas, hs = [1 / 6.65, 0.6], [0.1, 0.03]
    g = _gpu(batch=2, dcut_max=16, precision="fp64", impure=3, schedule=[(0, 16), (1, 16)])
    g.init_tensor(betas, hs)
    g.step(0, 16)
    g.step(1, 16)
    lnz, m = g.lnZ(), g.magnetization()
    e, ss = g.energy()
    for i in range(2):
        st = H.run(4, betas[i], hs[i], 10 ** 6, 2, impure=True)
        assert lnz[i] == pytest.approx(st.lnZ(), abs=1e-12)
        assert m[i] == pytest.approx(st.magnetization(), abs=1e-12)
        assert ss[i] == pytest.approx(st.sigma_sigma(), abs=1e-12)
        assert e[i] == pytest.approx(-4 * st.sigma_sigma() - hs[i] * st.magnetization(), abs=1e-12)


@pytest.mark.parametrize("name", ["ising4d_T6.65_h0_dcut4_16steps", "ising4d_T6.65_h0_dcut5_8steps"])
def test_fp64_run_vs_golden(name):
    gd = _golden(name)
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]]
    g = _gpu(batch=1, dcut_max=cfg["dcut"], precision="fp64", schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        got = g.lnZ()[0]
        assert got == pytest.approx(ref["lnZ"], rel=1e-10), (i + 1, got, ref["lnZ"])
        info = g.step_info(i + 1)
        assert list(info["dims"]) == ref["dims"]
        for n, (e0, e1) in ref["eps"].items():
            assert info["eps"][int(n)] == pytest.approx((e0, e1), rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp64oz"])
def test_fp64_impure_run_vs_golden(prec):
    """ln Z/V, <sigma>, <sigma sigma> and E/V of the impure-tensor run against the oracle's
    golden run (12 steps, D_cut = 4, h = 1e-5): the FP64 mode and the FP64-grade tensor-core
    mode (every product of T, S and M from integer slices) at the FP64 bars, but for <sigma>
    in the FP64-grade mode: at h = 1e-5 it is 2e-6 to 1e-5, the trace of an S whose entries
    cancel to ~1e-6 of their size, so the products' normwise ~1e-12 error becomes ~2e-6 of
    <sigma> (measured 8e-7 to 2.3e-6): bar 1e-5 relative."""
    gd = _golden("ising4d_T6.65_h1e-5_dcut4_impure_12steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]]
    g = _gpu(batch=1, dcut_max=cfg["dcut"], precision=prec, impure=3, schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        assert g.lnZ()[0] == pytest.approx(ref["lnZ"], rel=1e-10)
        if prec == "fp64oz":
            assert g.magnetization()[0] == pytest.approx(ref["m"], rel=1e-5)
        else:
            assert g.magnetization()[0] == pytest.approx(ref["m"], rel=1e-8, abs=1e-12)
        e, ss = g.energy()
        assert ss[0] == pytest.approx(ref["sigma_sigma"], rel=1e-9)
        assert e[0] == pytest.approx(ref["energy"], rel=1e-9)


def test_batch_of_temperatures_matches_single_runs():
    temps = [6.60, 6.65, 6.72]
    g = _gpu(batch=3, dcut_max=4, precision="fp64", schedule=[(i % 4, 4) for i in range(6)])
    g.init_tensor([1 / T for T in temps], 0.0)
    for i in range(6):
        g.step(i % 4, 4)
    lnz = g.lnZ()
    for j, T in enumerate(temps):
        assert lnz[j] == pytest.approx(H.run(4, 1 / T, 0.0, 4, 6).lnZ(), rel=1e-10)


@pytest.mark.parametrize("prec", ["fp16x3", "fp64"])
def test_grouped_contraction_matches_one_at_a_time(prec):
    """Temperatures contracted together (every tensor pass over the whole group, one grouped
    GEMM for all (temperature, tensor) outputs) give bit-identical tensors and observables to
    one temperature at a time (HOTRG_OPT_GROUP = 1): each element's arithmetic is the same.
    Pure and impure tensors, 6 steps at D_cut = 4 for 3 temperatures."""
    temps = [6.60, 6.65, 6.72]
    sched = [(i % 4, 4) for i in range(6)]
    out = []
    for group in (0, 1):
        g = _gpu(batch=3, dcut_max=4, precision=prec, impure=3, schedule=sched, group=group)
        g.init_tensor([1 / T for T in temps], 1e-5)
        for mu, dc in sched:
            g.step(mu, dc)
        e, ss = g.energy()
        out.append((tuple(g.lnZ()), tuple(g.magnetization()), tuple(ss), g.tensor(0, 2).tobytes(),
                    g.tensor(2, 1).tobytes(), g.step_info(6)["group"]))
    assert out[0][5] == 3 and out[1][5] == 1
    assert out[0][:5] == out[1][:5]


@pytest.mark.parametrize("prec", ["fp16x3", "fp64"])
def test_results_do_not_depend_on_workspace_contents(prec):
    """A workspace filled with NaN bit patterns before the run gives bit-identical results to a
    zeroed one: no step reads scratch it has not written (the first step's M operands, never
    used, are not built, so their slot's leftovers cannot reach a max-norm scale). Impure
    tensors, 3 temperatures contracted together, 5 steps at D_cut = 4."""
    temps = [6.60, 6.65, 6.72]
    sched = [(i % 4, 4) for i in range(5)]
    out = []
    for fill in (0x00, 0xFF):
        g = _gpu(batch=3, dcut_max=4, precision=prec, impure=3, schedule=sched)
        g.workspace.fill_(fill)
        g.init_tensor([1 / T for T in temps], 1e-5)
        for mu, dc in sched:
            g.step(mu, dc)
        e, ss = g.energy()
        out.append((tuple(g.lnZ()), tuple(g.magnetization()), tuple(ss)))
        assert np.all(np.isfinite(out[-1][0]))
    assert out[0] == out[1]


def test_maxnorm_modes_agree_and_keep_the_planes_in_range():
    """FP16X3 operand scaling from the first pass's bound (default), from the exact largest
    magnitude (max pass) and the fixed 2^14: the same ln Z/V to within 1e-8 (the scales are
    powers of two; only entries near fp16's range limits round differently), each within
    2e-6 of the FP64 oracle's golden run. The split statistics of the last step's operands:
    nothing at or above 2^15, the exact scale puts the largest |hi| in [2^14, 2^15), the
    bound's scale is never larger than the exact one and loses no more lo bits to fp16's
    subnormal range."""
    gd = _golden("ising4d_T6.65_h0_dcut4_16steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]][:8]
    ref = np.array([s["lnZ"] for s in gd["steps"][:8]])
    res, stats = {}, {}
    for mode in (1, 2, 0):
        g = _gpu(batch=1, dcut_max=cfg["dcut"], precision="fp16x3", schedule=sched, maxnorm=mode)
        g.init_tensor(gd["beta"], cfg["h"])
        lnz = []
        for mu, dc in sched:
            g.step(mu, dc)
            lnz.append(g.lnZ()[0])
        res[mode] = np.array(lnz)
        stats[mode] = g.split_stats()
        assert np.max(np.abs(res[mode] - ref)) < 2e-6, mode
    assert np.max(np.abs(res[1] - res[2])) < 1e-8 and np.max(np.abs(res[1] - res[0])) < 1e-8
    assert stats[0]["entries"] == stats[1]["entries"] == stats[2]["entries"] > 0
    for st in stats.values():
        assert max(st["hi_max"]) < 2.0 ** 15
        assert st["hi_zero"] + st["hi_subnormal"] <= st["entries"]
    assert min(stats[2]["hi_max"]) >= 2.0 ** 14
    for side in (0, 1):
        assert stats[1]["hi_max"][side] <= stats[2]["hi_max"][side]
    assert stats[2]["lo_subnormal"] <= stats[1]["lo_subnormal"]


def test_launches_per_step_do_not_grow_with_the_batch():
    """With every temperature's operands in one group, a step issues the same kernels for 2
    and for 8 temperatures (D_cut = 4, impure tensors: the isometry stage, the group's tensor
    passes and grouped GEMM, and the normalisation are each launched once per step)."""
    counts = []
    for batch in (2, 8):
        sched = [(i % 4, 4) for i in range(6)]
        g = _gpu(batch=batch, dcut_max=4, precision="fp16x3", impure=3, schedule=sched)
        g.init_tensor([1 / 6.65] * batch, 1e-5)
        for mu, dc in sched[:4]:
            g.step(mu, dc)
        g.profile(True)
        g.step(*sched[4])
        counts.append(g.profile_read()["launches"])
        g.profile(False)
        assert g.step_info(5)["group"] == batch
    assert counts[0] == counts[1]


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("tf32x3", 2e-6), ("fp16x3", 2e-6)])
def test_mixed_run_vs_golden(prec, tol):
    """|Delta ln Z/V| of the FP32-storage modes against the FP64 oracle, D_cut = 4, 16^4."""
    gd = _golden("ising4d_T6.65_h0_dcut4_16steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]]
    g = _gpu(batch=1, dcut_max=cfg["dcut"], precision=prec, schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    worst = 0.0
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        worst = max(worst, abs(g.lnZ()[0] - gd["steps"][i]["lnZ"]))
    assert worst < tol, worst


# ------------------------------------------------------------------ error handling
def test_errors_are_reported_not_raised_on_device():
    from paper_1911_12954_gb300 import HotrgError
    g = _gpu(batch=1, dcut_max=4, precision="fp64", schedule=[(0, 4)])
    with pytest.raises(HotrgError, match="ESTATE"):
        g.step(0, 4)                      # before init
    g.init_tensor(0.2, 0.0)
    with pytest.raises(HotrgError, match="EINVAL"):
        g.step(4, 4)                      # bad direction
    with pytest.raises(HotrgError, match="EINVAL"):
        g.step(0, 5)                      # dcut > dcut_max
    with pytest.raises(HotrgError, match="EINVAL"):
        g.init_tensor(-1.0, 0.0)          # beta < 0
    g.step(0, 4)
    assert math.isfinite(g.lnZ()[0])


# ------------------------------------------------------------------ D_cut = 8, the 1024^4 workload
@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_dcut8_mixed_first_8_steps_vs_golden(prec):
    """The benchmark's workload (T = 6.65, h = 0, D_cut = 8, towards 1024^4) in the launch
    configuration bench.py times: |Delta ln Z/V| <= 1e-6 against the FP64 oracle over the
    first 8 steps (step 2 cuts through a degenerate eigenvalue cluster)."""
    gd = _golden("ising4d_T6.65_h0_dcut8_8steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]]
    g = _gpu(batch=1, dcut_max=8, precision=prec, schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        assert abs(g.lnZ()[0] - ref["lnZ"]) <= 1e-6, (i + 1, g.lnZ()[0], ref["lnZ"])
        assert list(g.step_info(i + 1)["dims"]) == ref["dims"]


def test_dcut8_fp64_first_8_steps_vs_golden():
    """FP64 GPU path on the D_cut = 8 workload (T = 6.65, h = 0, towards 1024^4) over the
    first 8 steps, the oracle's stored values: ln Z/V and ln c to 1e-10 relative after
    every step, the discarded sums of both sides of every transverse direction to 1e-7.
    Steps 4..8 each run a 7e13-flop FP64 contraction (about a minute each)."""
    gd = _golden("ising4d_T6.65_h0_dcut8_8steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"][:8]]
    assert len(sched) == 8
    g = _gpu(batch=1, dcut_max=8, precision="fp64", schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        assert g.lnZ()[0] == pytest.approx(ref["lnZ"], rel=1e-10), (i + 1, g.lnZ()[0], ref["lnZ"])
        info = g.step_info(i + 1)
        assert info["ln_c"] == pytest.approx(ref["ln_c"], rel=1e-10)
        for n, (e0, e1) in ref["eps"].items():
            assert info["eps"][int(n)] == pytest.approx((e0, e1), rel=1e-7, abs=1e-12)


def test_fp16x3_step_legs8_elementwise_vs_oracle():
    """One FP16x3 step on a seeded decaying tensor with bond dimensions (8, 8, 7, 8), cut 4,
    element by element against the oracle's coarse_grain with the oracle's isometries:
    |T'_gpu - T'_oracle| <= 3e-5 max|T'_oracle|. The block-spin product is the benchmarked
    kernel at scale: M = N = 6272 rows (49 M tiles of 128, so the last CTA pair has one
    tile past the end and its partner a ragged 256-row tile), K = 32768 in 8 panels of
    4096, 625 pair tiles over the 76 CTA pairs (more than eight waves)."""
    dims, mu, dcut = (8, 8, 7, 8), 0, 4
    T = decaying_tensor(31, dims)
    T = T / np.linalg.norm(T)
    g = _gpu(batch=1, dcut_max=8, precision="fp16x3", schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    main, _ = g.step_flops(mu, dcut)
    assert main == pytest.approx(2.0 * 6272 ** 2 * 32768, rel=1e-12)
    g.step(mu, dcut)
    got = g.tensor()
    isos = {n: H.isometry(T, T, mu, n, dcut) for n in (1, 2, 3)}
    for iso in isos.values():
        lam = iso.spectrum
        # the kept subspace is unique well above the FP32 noise of the mixed-mode Gram
        assert not iso.degenerate_cut and lam[iso.chi - 1] - lam[iso.chi] > 1e-4 * lam[0]
    ref = H.coarse_grain(T, T, {n: iso.U for n, iso in isos.items()}, mu)
    ref = ref / np.linalg.norm(ref)
    assert got.shape == ref.shape
    err = np.abs(got - ref).max()
    assert err <= 3e-5 * np.abs(ref).max(), err


# ------------------------------------------------------------------ FP64-grade tensor-core mode
@pytest.mark.parametrize("dims,mu,dcut", [((3, 4, 2, 3), 1, 5), ((8, 8, 7, 8), 0, 4)])
def test_fp64oz_step_elementwise_vs_oracle(dims, mu, dcut):
    """HOTRG_FP64OZ (integer-slice products on the fp16 tensor cores, FP64 tensors): one step
    element by element against the oracle (coarse_grain with the oracle's isometries). The
    slices are fixed-point relative to each operand's largest entry, so the error bound is
    normwise: per product term up to 2^-40 of max|A| max|B| from the dropped slice products
    (i + j >= 5) and the FP32 rounding of the small groups' chunk sums, growing like sqrt(K)
    over the k sum. Bar: 1e-10 of the result's Frobenius norm (1 after the normalisation),
    the FP64 modes' bar on ln Z/V; measured 3.5e-13 (first case, a short k sum) and
    1.5e-11 (second case). The second case runs the product at scale: 6272 rows and columns
    (66 x 66 tiles of 128 x 96), K = 32768 in 8 panels of 4096."""
    T = (random_tensor(77, dims) if max(dims) < 8 else decaying_tensor(31, dims))
    T = T / np.linalg.norm(T)
    g = _gpu(batch=1, dcut_max=8, precision="fp64oz", schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    got = g.tensor()
    trans = [n for n in range(4) if n != mu]
    isos = {n: H.isometry(T, T, mu, n, dcut) for n in trans}
    assert not any(i.degenerate_cut for i in isos.values())
    ref = H.coarse_grain(T, T, {n: i.U for n, i in isos.items()}, mu)
    ref = ref / np.linalg.norm(ref)
    err = np.abs(got - ref).max()
    assert err <= 1e-10 * np.linalg.norm(ref), err


def test_fp64oz_dcut8_first_8_steps_vs_golden():
    """HOTRG_FP64OZ on the D_cut = 8 workload (T = 6.65, h = 0, towards 1024^4): ln Z/V within
    1e-10 relative of the oracle after each of the first 8 steps (the FP64 modes' bar), in
    about a second per steady-state step instead of a minute. ln c of each step within 1e-9:
    the product's error is normwise ~1e-10 of the result at K = 32768 (the dropped slice
    products), and ln c is the log of that norm; ln Z/V takes ln c with weight 2^-k."""
    gd = _golden("ising4d_T6.65_h0_dcut8_8steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"][:8]]
    g = _gpu(batch=1, dcut_max=8, precision="fp64oz", schedule=sched)
    g.init_tensor(gd["beta"], cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        assert g.lnZ()[0] == pytest.approx(ref["lnZ"], rel=1e-10), (i + 1, g.lnZ()[0], ref["lnZ"])
        assert g.step_info(i + 1)["ln_c"] == pytest.approx(ref["ln_c"], rel=1e-9)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("tf32x3", 3e-5), ("fp16x3", 3e-5)])
def test_long_closing_contraction(prec, tol):
    """Uniform bond dimension 9: the closing passes contract D_c^2 = 81 > 64 values per
    output (the register-accumulator fibre kernel); chi = 2 keeps the GEMM small. A
    decaying tensor keeps the kept eigenvalues apart (a random one has a flat Gram
    spectrum, whose top eigenvectors are ill-conditioned)."""
    dims, mu, dcut = (9, 9, 9, 9), 0, 2
    T = decaying_tensor(99, dims, 0.7)
    ref = H.HOTRG.from_tensor(T)
    ref.step(mu, dcut)
    g = _gpu(batch=1, dcut_max=9, precision=prec, schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    Tg = g.tensor()
    assert np.abs(Tg - ref.T).max() <= tol * np.abs(ref.T).max()
    # ln c sums 1.7e8 squares in a different order on each side: 1e-10 absolute
    assert g.step_info(1)["ln_c"] == pytest.approx(ref.history[0].ln_c, abs=max(tol, 1e-10))


@pytest.mark.parametrize("dims", [(11, 2, 2, 2), (16, 2, 2, 2)])
def test_large_gram_matrices_fp64(dims):
    """Transverse bond dimension 11 and 16: Gram matrices of side 121 and 256 (the largest the
    library takes), beyond what the eigensolver keeps in shared memory, so A and V live in
    its global workspace. One truncating step (D_cut = 6) in FP64 against the oracle: the
    tensor, the isometries, the discarded sums and the sides taken."""
    mu, dcut = 1, 6
    T = decaying_tensor(123, dims, 0.7)
    ref = H.HOTRG.from_tensor(T)
    trans = [n for n in range(4) if n != mu]
    isos = {n: H.isometry(ref.T, ref.T, mu, n, dcut) for n in trans}
    ref.step(mu, dcut)
    g = _gpu(batch=1, dcut_max=16, precision="fp64", schedule=[(mu, dcut)], dims0=dims)
    g.set_tensor(T)
    g.step(mu, dcut)
    Tg = g.tensor()
    assert np.allclose(Tg, ref.T, rtol=0, atol=1e-12 * np.abs(ref.T).max())
    info = g.step_info(1)
    for n in trans:
        Ug = g.isometry(n, dold=dims[n], chi=isos[n].chi)
        assert np.allclose(Ug, isos[n].U, atol=1e-11), n
        assert info["primed"][n] == int(isos[n].primed)
        assert info["eps"][n] == pytest.approx(isos[n].eps, rel=1e-9, abs=1e-13)


# ------------------------------------------------------------------ impure tensors in mixed precision
@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_mixed_impure_run_vs_golden(prec):
    """sigma and sigma-sigma impure tensors through the tensor-core paths, D_cut = 4,
    h = 1e-5, 12 steps: <sigma>, <sigma sigma> and E/V against the FP64 oracle."""
    gd = _golden("ising4d_T6.65_h1e-5_dcut4_impure_12steps")
    cfg = gd["config"]
    sched = [(s["mu"], cfg["dcut"]) for s in gd["steps"]]
    g = _gpu(batch=2, dcut_max=cfg["dcut"], precision=prec, impure=3, schedule=sched)
    g.init_tensor([gd["beta"]] * 2, cfg["h"])
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        ref = gd["steps"][i]
        lnz, m = g.lnZ(), g.magnetization()
        e, ss = g.energy()
        for b in range(2):                    # both batch elements see the same run
            assert abs(lnz[b] - ref["lnZ"]) < 2e-6
            assert abs(m[b] - ref["m"]) < 2e-6
            assert abs(ss[b] - ref["sigma_sigma"]) < 2e-6
            assert abs(e[b] - ref["energy"]) < 1e-5


def test_dcut8_impure_z2_and_bounds():
    """D_cut = 8, h = 0, TF32x3 with impure tensors, 6 steps: Z2 symmetry makes <sigma>
    vanish (to the arithmetic's noise); 0 < <sigma sigma> < 1; E/V = -4 <sigma sigma>;
    ln Z/V equals the pure run's to 1e-6 (the impure tensors do not feed back)."""
    sched = [(i % 4, 8) for i in range(6)]
    g = _gpu(batch=1, dcut_max=8, precision="tf32x3", impure=3, schedule=sched)
    g.init_tensor(1 / 6.65, 0.0)
    gd = _golden("ising4d_T6.65_h0_dcut8_8steps")
    for i, (mu, dc) in enumerate(sched):
        g.step(mu, dc)
        assert abs(g.lnZ()[0] - gd["steps"][i]["lnZ"]) <= 1e-6
        assert abs(g.magnetization()[0]) < 1e-6
        e, ss = g.energy()
        assert 0.0 < ss[0] < 1.0 and e[0] == pytest.approx(-4 * ss[0], rel=1e-12)


# ------------------------------------------------------------------ failure detection (no GPU fault)
def test_bounded_wait_times_out_and_context_recovers():
    """A device-side wait on a barrier nothing signals gives up after 20 ms and reports
    ETIMEOUT; the context is sticky until re-initialised and then steps normally."""
    from paper_1911_12954_gb300 import HotrgError
    g = _gpu(batch=1, dcut_max=4, precision="tf32x3", schedule=[(0, 4), (1, 4)])
    assert g.lib.hotrg_selftest_wait(g.ctx, 20) == -6          # HOTRG_ETIMEOUT
    with pytest.raises(HotrgError, match="ESTATE"):
        g.step(0, 4)                                        # sticky after the device error
    g.init_tensor(1 / 6.65, 0.0)
    g.step(0, 4)
    g.step(1, 4)
    assert g.lnZ()[0] == pytest.approx(H.run(4, 1 / 6.65, 0.0, 4, 2).lnZ(), abs=2e-6)


def test_jacobi_sweep_limit_reports_enoconv():
    from paper_1911_12954_gb300 import OPT_JACOBI_SWEEPS, HotrgError
    g = _gpu(batch=1, dcut_max=4, precision="fp64", schedule=[(i % 4, 4) for i in range(3)])
    g.set_option(OPT_JACOBI_SWEEPS, 1)
    g.init_tensor(1 / 6.65, 0.0)
    g.step(0, 4)
    g.step(1, 4)                      # 16 x 16 Gram matrices need more than one sweep
    with pytest.raises(HotrgError, match="ENOCONV"):
        g.lnZ()
    g.set_option(OPT_JACOBI_SWEEPS, 60)
    g.init_tensor(1 / 6.65, 0.0)
    for i in range(3):
        g.step(i % 4, 4)
    assert g.lnZ()[0] == pytest.approx(H.run(4, 1 / 6.65, 0.0, 4, 3).lnZ(), rel=1e-10)


def test_nonfinite_input_is_rejected_on_the_host():
    from paper_1911_12954_gb300 import HotrgError
    dims = (2, 2, 2, 2)
    T = random_tensor(3, dims)
    T[0, 1, 0, 1, 1, 0, 0, 1] = np.nan
    g = _gpu(batch=1, dcut_max=4, precision="fp64", schedule=[(0, 4)], dims0=dims)
    with pytest.raises(HotrgError, match="EINVAL"):
        g.set_tensor(T)
    T[0, 1, 0, 1, 1, 0, 0, 1] = np.inf
    with pytest.raises(HotrgError, match="EINVAL"):
        g.set_tensor(T)


@pytest.mark.parametrize("precision,variants", [("tf32x3", (0, 1)), ("fp16x3", (0, 1, 2, 3))])
def test_gemm_pipeline_variants_agree(precision, variants):
    """The tensor-core pipelines of a mode give the same step: for tf32x3 4 x 16-wide and
    2 x 32-wide k-blocks; for fp16x3 CTA pairs (cta_group::2, 256 x 256 tiles) and single
    CTAs promoting every 64, 256 and 128 k. The pair pipeline and the single-CTA one with the
    same chunk issue the same products in the same k order into the same 128-row accumulator
    per SM: bit-identical."""
    from paper_1911_12954_gb300 import OPT_GEMM_VARIANT
    dims, mu, dcut = (3, 3, 2, 3), 2, 6
    T = random_tensor(12, dims)
    out = []
    for v in variants:
        g = _gpu(batch=1, dcut_max=9, precision=precision, schedule=[(mu, dcut)], dims0=dims)
        g.set_option(OPT_GEMM_VARIANT, v)
        g.set_tensor(T)
        g.step(mu, dcut)
        out.append(g.tensor())
    for o in out[1:]:
        assert np.allclose(out[0], o, atol=1e-6 * np.abs(out[0]).max())
    if precision == "fp16x3":
        assert np.array_equal(out[0], out[3])


def test_x_indicator_matches_oracle_fp64():
    """X along every direction after 0, 1 and 16 steps (D_cut = 4, 16^4 lattice) at
    temperatures in both phases and near T_c, FP64 mode against the oracle's X."""
    temps = [5.0, 6.65, 9.0]
    sched = [(i % 4, 4) for i in range(16)]
    g = _gpu(batch=len(temps), dcut_max=4, precision="fp64", schedule=sched)
    g.init_tensor([1 / t for t in temps], 0.0)
    ref = [H.HOTRG.start(4, 1 / t, 0.0) for t in temps]
    for k, (mu, dc) in enumerate(sched):
        if k in (0, 1, 16):
            for nu in range(4):
                got = g.x_indicator(nu)
                for b, st in enumerate(ref):
                    assert got[b] == pytest.approx(H.x_indicator(st.T, nu), rel=1e-9), (k, nu, b)
        g.step(mu, dc)
        for st in ref:
            st.step(mu, dc)
    for nu in range(4):
        got = g.x_indicator(nu)
        for b, st in enumerate(ref):
            assert got[b] == pytest.approx(H.x_indicator(st.T, nu), rel=1e-9), ("end", nu, b)


def test_x_indicator_mixed_precision_phases():
    """FP16x3 at D_cut = 6 after 16 steps: X within 1e-4 of the FP64 GPU value deep in each
    phase (T = 5: ~2, T = 9: ~1)."""
    temps = [5.0, 9.0]
    sched = [(i % 4, 6) for i in range(16)]
    out = {}
    for prec in ("fp64", "fp16x3"):
        g = _gpu(batch=2, dcut_max=6, precision=prec, schedule=sched)
        g.init_tensor([1 / t for t in temps], 0.0)
        for mu, dc in sched:
            g.step(mu, dc)
        out[prec] = g.x_indicator(0)
    assert abs(out["fp64"][0] - 2.0) < 0.01 and abs(out["fp64"][1] - 1.0) < 0.05
    assert np.allclose(out["fp16x3"], out["fp64"], atol=1e-4)


def test_tc_bracket_agrees_with_oracle():
    """bracket_tc (batched GPU runs, FP64 mode, D_cut = 4, 16 steps) returns an interval whose
    ends the oracle puts on the two sides of X = 1.5."""
    from paper_1911_12954_gb300.tc import bracket_tc
    lo, hi, hist = bracket_tc(4, 6.0, 7.5, nsteps=16, batch=4, rounds=2, precision="fp64")
    assert 6.0 <= lo < hi <= 7.5 and hi - lo == pytest.approx(1.5 / 9, rel=1e-12)
    assert H.x_indicator(H.run(4, 1 / lo, 0.0, 4, 16).T) > 1.5
    assert H.x_indicator(H.run(4, 1 / hi, 0.0, 4, 16).T) <= 1.5


def test_observable_scan_matches_oracle():
    """observable_scan (one batched impure run, FP64 mode, D_cut = 4, h = 1e-5): E/V, <sigma>
    and ln Z/V recorded after steps 10..12 equal the oracle's at each temperature."""
    from paper_1911_12954_gb300.tc import observable_scan
    temps = [6.0, 7.0]
    rows = observable_scan(temps, 4, nsteps=12, h=1e-5, precision="fp64", record_from=10)
    assert [r["k"] for r in rows] == [10, 11, 12]
    for b, t in enumerate(temps):
        st = H.HOTRG.start(4, 1 / t, 1e-5, impure=True)
        for k in range(12):
            st.step(k % 4, 4)
            if k + 1 >= 10:
                r = rows[k + 1 - 10]
                assert r["E"][b] == pytest.approx(st.energy(), rel=1e-9, abs=1e-12)
                assert r["m"][b] == pytest.approx(st.magnetization(), rel=1e-9, abs=1e-12)
                assert r["lnZ"][b] == pytest.approx(st.lnZ(), rel=1e-12)


@pytest.mark.parametrize("precision", ["tf32x3", "fp16x3"])
def test_cuda_graph_steps_match_eager_steps(precision):
    """Captured-and-replayed steps (one graph launch per step, every batch element and
    impure tensor inside; for fp16x3 the GEMM is a CTA-pair cluster launch) give bit-identical
    results to eager launches: 16 steps, so the four steady-state graphs are each replayed
    several times."""
    sched = [(i % 4, 4) for i in range(16)]
    out = []
    for graphs in (False, True):
        g = _gpu(batch=2, dcut_max=4, precision=precision, impure=3, schedule=sched, graphs=graphs)
        g.init_tensor([1 / 6.65, 1 / 6.70], 1e-5)
        rows = []
        for mu, dc in sched:
            g.step(mu, dc)
        e, ss = g.energy()
        rows = (tuple(g.lnZ()), tuple(g.magnetization()), tuple(ss),
                tuple(g.step_info(k)["ln_c"] for k in range(1, 17)), g.tensor(0, 1).tobytes())
        out.append(rows)
        g.init_tensor([1 / 6.65, 1 / 6.70], 1e-5)        # graphs are reused after a re-init
        for mu, dc in sched[:5]:
            g.step(mu, dc)
        out.append(tuple(g.lnZ()))
    assert out[0] == out[2]
    assert out[1] == out[3]
