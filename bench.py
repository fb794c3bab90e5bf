#!/usr/bin/env python
"""Throughput of the 4D Ising HOTRG coarse-graining step on GB300.

Workload (synthetic, deterministic): the 4D Ising site tensor at T = 6.65, h = 0,
D_cut = 8, directions cycled x, y, z, t towards the 1024^4 lattice (40 steps). A
benchmark "step" is one HOTRG coarse-graining step: Gram matrices on both sides of the
three transverse bond pairs, FP64 Jacobi eigensolves and isometries, the block-spin
contraction (2 D^15 flops on tcgen05 tensor cores: each FP32 operand split into an fp16
hi + lo pair, three products, FP32 accumulation), normalisation and ln Z accumulation. The
W warm-up steps are steps 1..W of the run (bond dimensions reach 8 at step 3), the K
timed steps are the steady-state steps W+1..W+K.

Printed (rank 0, one JSON line): algorithmic TFLOP/s of the timed steps (value), the
block-spin GEMM against its tensor-core roofline, the FP64 GPU path on one
steady-state step, |Delta ln Z/V| of the mixed path against FP64, the FP64 NumPy oracle
timed on a bounded sample (cpu_baseline), and an end-to-end figure for the whole
40-step job through the public API with host inputs and outputs.

--impl reference times the FP64 NumPy oracle itself (the reference arm) on the host.
Multi-GPU: replicas only (each rank runs its own temperature); value = all ranks' flops
/ the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4D HOTRG step TFLOP/s (% peak), mixed vs FP64, D_cut 8–13, |Δ lnZ/V|≤1e-6"
T_WORK = 6.65
H_WORK = 0.0
LATTICE_STEPS = 40
GOLDEN_D8 = os.path.join(ROOT, "tests", "golden", "ising4d_T6.65_h0_dcut8_8steps.json")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=4)
    p.add_argument("--dcut", type=int, default=8)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--fp64", type=int, default=1, help="time one FP64 GPU step for the mixed-vs-FP64 ratio")
    p.add_argument("--e2e", type=int, default=1, help="time the whole 40-step job through the public API")
    p.add_argument("--cpu", type=int, default=1, help="time the FP64 oracle on a bounded sample (rank 0, N=1)")
    p.add_argument("--ref-steps", type=int, default=-1,
                   help="steps of the FP64-grade tensor-core reference run (HOTRG_FP64OZ) the mixed run is "
                        "compared with, step by step (-1: 8 at D_cut <= 8, 6 up to 11, 5 at 12, 4 at 13; 0: none)")
    p.add_argument("--batch", type=int, default=1, help="temperatures per GPU (evenly spaced in [6.60, 6.72])")
    p.add_argument("--impure", type=int, default=0, help="propagate the sigma and sigma-sigma impure tensors")
    p.add_argument("--graphs", type=int, default=0, help="replay each distinct step as a captured CUDA graph")
    p.add_argument("--tc", type=int, default=0,
                   help="instead of the step line: bracket T_c(D_cut) from the X indicator after 40 steps "
                        "(batched temperatures, --tc rounds) and print that as its own line")
    p.add_argument("--scan", type=int, default=0,
                   help="instead of the step line: E/V and <sigma> against T at this many temperatures in "
                        "[--scan-lo, --scan-hi] (impure tensors, h = 1e-5, 40 steps), printed as its own line")
    p.add_argument("--scan-lo", type=float, default=6.670)
    p.add_argument("--scan-hi", type=float, default=6.690)
    p.add_argument("--scan-h", type=float, default=1e-5, help="field of the scan")
    p.add_argument("--autotune", type=int, default=1,
                   help="take each step's closing direction and GEMM pipeline from the autotuner (the "
                        "steady-state shapes are tuned after the warm-up steps, outside the timed region)")
    p.add_argument("--maxnorm", type=int, default=1, choices=[0, 1, 2],
                   help="FP16X3 operand scaling: 1 bound from the first pass, 2 exact max pass, 0 fixed 2^14")
    p.add_argument("--group", type=int, default=0,
                   help="most temperatures contracted together (HOTRG_OPT_GROUP; 0: the planner's choice)")
    p.add_argument("--gemm-variant", type=int, default=0,
                   help="tensor-core GEMM pipeline option (HOTRG_OPT_GEMM_VARIANT) for every mixed run")
    p.add_argument("--precision", choices=["tf32x3", "fp16x3"], default="fp16x3",
                   help="tensor-core split of the block-spin contraction (default: fp16 hi/lo on kind::f16)")
    return p.parse_args()


# DRAM bytes (read + write) per launch of the block-spin GEMM, from one ncu capture of the
# kernel as built now (dram__bytes_read.sum + dram__bytes_write.sum, one pass, the steady
# D_cut = 8 launch: 134.78 GB + 4.71 GB), keyed by (precision, GEMM option, D_cut,
# temperatures, impure). Workloads without a capture report null.
GEMM_TRAFFIC = {("fp16x3", 0, 8, 1, False): 139.49e9}


# --------------------------------------------------------------------------- helpers
def tensor_peak(precision: str, sustained: bool = True):
    """Dense tensor peak of the GEMM's operand type. fp16 runs at the BF16 rate (the
    measured BF16 figure applies as is); TF32 = that figure x the nominal TF32/BF16 ratio
    1.1 / 2.25. The GEMM is timed inside seconds of back-to-back steps, so the sustained
    figure applies; the burst one is reported beside it. Falls back to the profiling
    recipe's 1.9 / 1.7 PFLOP/s when no measurement exists."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    r, rname = (1.0, "fp16 = bf16 rate") if precision == "fp16x3" else (1.1 / 2.25, "x nominal tf32/bf16 1.1/2.25")
    try:
        with open(path) as f:
            mp = json.load(f)
        b = mp["bf16_tflops_sustained"] if sustained else mp["bf16_tflops"]
        return b * r, ("measured bf16 sustained" if sustained else "measured bf16 burst") + " " + rname
    except Exception:
        b = 1700.0 if sustained else 1900.0
        return b * r, f"fallback bf16 {b / 1000:.1f} PF " + rname


def kernel_name(precision: str, option: int) -> str:
    """The block-spin GEMM kernel a HOTRG_OPT_GEMM_VARIANT value runs."""
    if precision == "fp16x3":
        return {0: "gemm_pair_kernel<CfgF16P> (CTA pairs, tcgen05.mma.cta_group::2)",
                1: "gemm_tf32x3_kernel<CfgF16S>", 2: "gemm_tf32x3_kernel<CfgF16L>",
                3: "gemm_tf32x3_kernel<CfgF16>"}[option]
    return {0: "gemm_tf32x3_kernel<CfgTF32>", 1: "gemm_tf32x3_kernel<CfgTF32W>"}.get(option, "gemm_simt_kernel")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()

    def summary(self):
        try:
            with open(self.tmp.name) as f:
                rows = [r.strip().split(", ") for r in f if r.strip()]
            os.unlink(self.tmp.name)
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm, smax, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                pw.append(float(r[3]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "sm_mhz_min": min(sm) if sm else None, "power_w_median": statistics.median(pw) if pw else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- replicas
def replica_temperatures(batch: int, rank: int, world: int):
    """Temperatures of one rank. Replicas share no data: with batch == 1 every rank runs
    T = 6.65 + 0.001 rank; otherwise the batch * world temperatures evenly spaced in
    [6.60, 6.72] are dealt out in contiguous blocks of `batch`."""
    import numpy as np

    if batch == 1:
        return [T_WORK + 0.001 * rank]
    allt = np.linspace(6.60, 6.72, batch * world)
    return [float(t) for t in allt[rank * batch:(rank + 1) * batch]]


class RankSync:
    """Timing plumbing across ranks: barrier, max and sum of one scalar. No data of the
    method crosses ranks. `dist` is torch.distributed (or None for one rank); `device`
    is where the reduction tensor lives (cuda for NCCL, cpu for gloo)."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)

    def throughput(self, flops_local: float, ms_local: float):
        """Whole-job TFLOP/s: every rank's flops over the slowest rank's time."""
        ms = self.max(ms_local)
        return self.sum(flops_local) / (ms * 1e-3) / 1e12, ms


# --------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(dcut: int, seed: int = 8, nx: int = 1):
    """One steady-state step of the FP64 oracle on a seeded tensor of the steady-state
    shape: the HOSVD of all three transverse directions (both sides) and the block-spin
    contraction restricted to the new x legs X, X' < nx (isometry U^x cut to its first nx
    columns), i.e. nx^2/D_cut^2 of the D^15 product. Returns (flops, seconds)."""
    import numpy as np

    from oracle import hotrg as H
    from workloads import random_tensor

    D = dcut
    mu = 0
    T = random_tensor(seed, (D, D, D, D))
    T = T / np.linalg.norm(T)
    t0 = time.perf_counter()
    isos = {n: H.isometry(T, T, mu, n, dcut) for n in (1, 2, 3)}
    U = {n: isos[n].U for n in (1, 2, 3)}
    U[1] = U[1][:, :, :nx].copy()
    H.coarse_grain(T, T, U, mu)
    dt = time.perf_counter() - t0
    # flops of what ran (2 per multiply-add): 12 half-Grams + the restricted contraction
    E = float(D) ** 8
    R = D * D
    gram = 3 * 4 * 2.0 * R * E
    rows = nx * D * D * D * D         # X (nx) * Y (chi) * c1 c1' (D^2) * mu1 (D)
    K = float(D) ** 5
    main = 2.0 * rows * rows * K
    builds = 2 * (2.0 * D * nx * E) + 2 * (2.0 * D * rows * K)    # T x U^x (nx cols), x U^y, both sides
    close = 2.0 * D * rows * rows + 2.0 * D * D * rows * rows / (D * D) * D
    return gram + main + builds + close, dt


def workload_config(args, world):
    """The workload part of a bench line's config, identical for the GPU and reference arms."""
    D = args.dcut
    nsteps = args.warmup + args.steps
    hfield = 1e-5 if args.impure else H_WORK
    workload = ((f"4D Ising HOTRG, T={T_WORK}, h={H_WORK}" if args.batch == 1 else
                 f"4D Ising HOTRG, {args.batch * world} temperatures in [6.60, 6.72], h={hfield}")
                + (", pure + sigma + sigma-sigma impure tensors" if args.impure else "")
                + f", D_cut={D}, 1024^4 lattice schedule (x,y,z,t cycled); timed steps "
                f"{args.warmup + 1}..{nsteps} (steady state)")
    return {"workload": workload, "dcut": D, "temperatures_per_gpu": args.batch, "impure": bool(args.impure),
            "lattice": "1024^4"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_sample(args.dcut)
    fl, secs = 0.0, 0.0
    for i in range(args.steps):
        f, s = oracle_sample(args.dcut, seed=100 + i)
        fl += f
        secs += s
    value = fl / secs / 1e12
    sample = (f"per step: one steady-state D_cut={args.dcut} HOTRG step of the FP64 NumPy oracle on a seeded "
              f"N(0,1) tensor of shape ({args.dcut},)*8: full HOSVD of the 3 transverse directions + the "
              f"block-spin contraction restricted to X = X' = 0 (1/{args.dcut ** 2} of the D^15 product)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def run_tc(args, local):
    """T_c(D_cut) bracket from the X indicator (Sec. 3.1): rounds of 8 temperatures each, one
    batched 40-step run (1024^4) per round, starting from [6.0, 7.5]; reports the interval,
    every round's (T, X) and the wall time, with the clocks seen."""
    import torch

    from paper_1911_12954_gb300.tc import bracket_tc

    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        lo, hi, hist = bracket_tc(args.dcut, 6.0, 7.5, nsteps=40, batch=8, rounds=args.tc, precision=args.precision)
        secs = time.perf_counter() - t0
    line = {"metric": f"T_c(D_cut={args.dcut}) bracket from the X indicator, 1024^4 lattice", "value": secs,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"4D Ising HOTRG, h=0, D_cut={args.dcut}, 40 steps (x,y,z,t cycled), "
                                   f"{args.tc} rounds x 8 temperatures from [6.0, 7.5]"},
            "tc_bracket": [lo, hi], "tc_mid": 0.5 * (lo + hi),
            "rounds": [{"T": [float(t) for t in T], "X": [float(x) for x in X]} for T, X in hist],
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_scan(args, local):
    """Internal energy and magnetisation against temperature (Sec. 3.1, Figs. 5 and 6) for the
    volumes 2^28 .. 2^40: one batched run of T, S and M at --scan temperatures (field
    --scan-h); reports the
    values at volumes 2^28, 2^32, 2^36, 2^40, the largest jumps between adjacent temperatures
    at 2^40 and the wall time, with the clocks seen."""
    import numpy as np
    import torch

    from paper_1911_12954_gb300.tc import largest_jump, observable_scan

    torch.cuda.set_device(local)
    temps = np.linspace(args.scan_lo, args.scan_hi, args.scan)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        rows = observable_scan(temps, args.dcut, nsteps=40, h=args.scan_h, precision=args.precision, record_from=28)
        secs = time.perf_counter() - t0
    last = rows[-1]
    ie, de = largest_jump(temps, last["E"])
    im, dm = largest_jump(temps, last["m"])
    line = {"metric": f"E/V and <sigma> scan against T, D_cut={args.dcut}, volumes 2^28..2^40", "value": secs,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"4D Ising HOTRG, h={args.scan_h}, D_cut={args.dcut}, 40 steps (x,y,z,t cycled), "
                                   f"{args.scan} temperatures in [{args.scan_lo}, {args.scan_hi}], pure + sigma + "
                                   f"sigma-sigma impure tensors in one batch"},
            "T": [float(t) for t in temps],
            "volumes": {f"2^{r['k']}": {"E": [float(x) for x in r["E"]], "m": [float(x) for x in r["m"]]}
                        for r in rows if r["k"] in (28, 32, 36, 40)},
            "energy_jump_2^40": {"between": [float(temps[ie]), float(temps[ie + 1])], "dE": de},
            "magnetization_jump_2^40": {"between": [float(temps[im]), float(temps[im + 1])], "dm": dm},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.tc:
        return run_tc(args, local) if rank == 0 else 0
    if args.scan:
        return run_scan(args, local) if rank == 0 else 0

    import numpy as np
    import torch

    from paper_1911_12954_gb300 import HOTRG, OPT_GEMM_VARIANT

    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    sync = RankSync(dist, device=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        sync.barrier()
        torch.cuda.synchronize()

    allmax, allsum = sync.max, sync.sum

    D = args.dcut
    temps = replica_temperatures(args.batch, rank, world)
    betas = [1.0 / t for t in temps]
    beta = betas[0]
    hfield = 1e-5 if args.impure else H_WORK
    impure = 3 if args.impure else 0
    nsteps = args.warmup + args.steps
    sched = [(i % 4, D) for i in range(max(nsteps, 8))]

    def step_flops(run, mu, dc, kdone):
        """Algorithmic flops of one step for the whole batch: per temperature the Gram and
        isometry work once, the contraction once per tensor product (5 with impure
        tensors: TT, ST, TS, MT, TM; 4 at the first step: TT, ST, TS, SS)."""
        main, total = run.step_flops(mu, dc)
        if not impure:
            return args.batch * total
        nprod = 4 if kdone == 0 else 5
        return args.batch * (nprod * main + 3 * (total - main))

    # ---------------------------------------------------------------- mixed precision, timed
    run = HOTRG(batch=args.batch, dcut_max=D, precision=args.precision, impure=impure, schedule=sched,
                graphs=bool(args.graphs), autotune=bool(args.autotune), group=args.group, maxnorm=args.maxnorm)
    run.set_option(OPT_GEMM_VARIANT, args.gemm_variant)
    run.init_tensor(betas, hfield)
    for i in range(args.warmup):
        run.step(*sched[i])
    if args.autotune:
        # the timed steps' shapes (steady state after the warm-up) are timed and cached here
        for d in sorted({mu for mu, _ in sched[args.warmup:nsteps]}):
            run.autotune(d, D)
    barrier()
    flops = 0.0
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        run.profile(True)
        start.record(run.stream)
        for i in range(args.warmup, nsteps):
            flops += step_flops(run, *sched[i], i)
            run.step(*sched[i])
        stop.record(run.stream)
        barrier()
    prof = run.profile_read()
    run.profile(False)
    plans = [{"step": k, **{f: run.step_info(k)[f] for f in ("mu", "closing", "gemm_option", "tuned", "group")}}
             for k in range(args.warmup + 1, nsteps + 1)]
    tune = run.tune_stats()
    # --steps 0: the warm-up steps and the accuracy runs only (no timed region, no throughput)
    value, ms_max = sync.throughput(flops, start.elapsed_time(stop)) if args.steps > 0 else (None, None)
    lnz_run = [float(x) for x in run.lnZ()]
    obs = {}
    if impure:
        e, ss = run.energy()
        obs = {"magnetization": [float(x) for x in run.magnetization()], "energy": [float(x) for x in e]}
    del run
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- accuracy vs FP64
    accuracy = {}
    nref = args.ref_steps if args.ref_steps >= 0 else (8 if D <= 8 else (6 if D <= 11 else (5 if D == 12 else 4)))
    nver = max(8 if D <= 8 else 3, nref)
    def verify(maxnorm):
        """The first temperature of this rank's workload, with its field and impure tensors:
        ln Z/V (and E, m) after each of the first nver steps, and the fp16 split statistics of
        the last step's operands."""
        ver = HOTRG(batch=1, dcut_max=D, precision=args.precision, impure=impure, schedule=sched[:nver],
                    maxnorm=maxnorm)
        ver.set_option(OPT_GEMM_VARIANT, args.gemm_variant)
        ver.init_tensor(beta, hfield)
        lnz, ob = [], []
        for i in range(nver):
            ver.step(*sched[i])
            lnz.append(float(ver.lnZ()[0]))
            if impure:
                e, _ = ver.energy()
                ob.append((float(e[0]), float(ver.magnetization()[0])))
        st = ver.split_stats() if args.precision == "fp16x3" else None
        del ver
        torch.cuda.empty_cache()
        return lnz, ob, st

    mixed_lnz, mixed_obs, split_default = verify(args.maxnorm)
    # the other operand scalings of the fp16 planes, on the same steps (split statistics and
    # ln Z/V; compared with the FP64 references below)
    split_runs = {}
    if args.precision == "fp16x3" and rank == 0 and D <= 8:     # two more verification runs: cheap at D <= 8
        for mode in (1, 2, 0):
            lz, _, st = (mixed_lnz, None, split_default) if mode == args.maxnorm else verify(mode)
            split_runs[mode] = (lz, st)
    if rank == 0 and D == 8 and args.batch == 1 and not impure and os.path.exists(GOLDEN_D8):
        with open(GOLDEN_D8) as f:
            gd = json.load(f)
        diffs = [abs(mixed_lnz[i] - s["lnZ"]) for i, s in enumerate(gd["steps"][:8])]
        accuracy["max_abs_dlnZ_vs_fp64_oracle_steps1to8"] = max(diffs)
        accuracy["dlnZ_per_step"] = diffs
        split_ref = [s["lnZ"] for s in gd["steps"][:8]]
    else:
        split_ref = None

    # ---------------------------------------------------------------- FP64 GPU path
    # steps 1..3 (the DFMA product; skipped where the FP64-grade reference below covers them,
    # D_cut > 8); step 4, the first steady-state step, timed when D <= 8
    fp64 = None
    ntimed64 = 1 if (args.fp64 and D <= 8) else 0
    # (impure runs: always, because ⟨σ⟩ at h = 1e-5 is a 1e-6 effect in Tr S, below the FP64-grade
    # reference's own resolution)
    n64 = 3 if (D <= 8 or nref == 0 or impure) else 0
    r64 = HOTRG(batch=1, dcut_max=D, precision="fp64", impure=impure, schedule=sched[:max(1, n64 + ntimed64)])
    r64.init_tensor(beta, hfield)
    d64, dE, dm = [], [], []
    for i in range(n64):
        r64.step(*sched[i])
        d64.append(abs(mixed_lnz[i] - float(r64.lnZ()[0])))
        if impure:
            e, _ = r64.energy()
            dE.append(abs(mixed_obs[i][0] - float(e[0])))
            dm.append(abs(mixed_obs[i][1] - float(r64.magnetization()[0])))
    if n64:
        accuracy["abs_dlnZ_mixed_vs_fp64_gpu_steps1to3"] = d64
    if dE:
        accuracy["abs_dE_per_site_mixed_vs_fp64_gpu_steps1to3"] = dE
        accuracy["abs_dmagnetization_mixed_vs_fp64_gpu_steps1to3"] = dm
    if ntimed64:
        barrier()
        f64 = r64.step_flops(*sched[3])[1]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(r64.stream)
        r64.step(*sched[3])
        e1.record(r64.stream)
        barrier()
        ms64 = allmax(e0.elapsed_time(e1))
        lnz64 = float(r64.lnZ()[0])
        fp64 = {"value": allsum(f64) / (ms64 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms64,
                "steps": 1, "warmup": 3, "timed_step": 4,
                "speedup_mixed_vs_fp64": (ms64 / (ms_max / args.steps) * args.batch * (5 if impure else 1)
                                          if ms_max else None)}
        accuracy["abs_dlnZ_mixed_vs_fp64_gpu_step4"] = abs(mixed_lnz[3] - lnz64)
    del r64
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- FP64-grade reference
    # HOTRG_FP64OZ: FP64 tensors, the block-spin product from exact integer slices on the fp16
    # tensor cores (error below 2^-40 of the operands): the steady-state reference at large
    # D_cut, where the DFMA product takes minutes to hours per step; its last step is timed.
    fp64oz = None
    oz_vals = []
    if nref > 0:
        oz = HOTRG(batch=1, dcut_max=D, precision="fp64oz", impure=impure, schedule=sched[:nref])
        oz.init_tensor(beta, hfield)
        doz, oz_vals, dEoz, dmoz = [], [], [], []
        ms_oz, fl_last = None, 0.0
        for i in range(nref):
            if i == nref - 1:
                fl_last = step_flops(oz, *sched[i], i) / args.batch   # the step about to run, one temperature
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(oz.stream)
            oz.step(*sched[i])
            if i == nref - 1:
                e1.record(oz.stream)
                barrier()
                ms_oz = allmax(e0.elapsed_time(e1))
            oz_vals.append(float(oz.lnZ()[0]))
            doz.append(abs(mixed_lnz[i] - oz_vals[-1]))
            if impure:
                e, _ = oz.energy()
                dEoz.append(abs(mixed_obs[i][0] - float(e[0])))
                dmoz.append(abs(mixed_obs[i][1] - float(oz.magnetization()[0])))
        accuracy[f"abs_dlnZ_mixed_vs_fp64oz_steps1to{nref}"] = doz
        accuracy["max_abs_dlnZ_mixed_vs_fp64oz"] = max(doz)
        if impure:
            accuracy[f"abs_dE_per_site_mixed_vs_fp64oz_steps1to{nref}"] = dEoz
            accuracy[f"abs_dmagnetization_mixed_vs_fp64oz_steps1to{nref}"] = dmoz
        fp64oz = {"value": allsum(fl_last) / (ms_oz * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms_oz,
                  "timed_step": nref, "steps_compared": nref,
                  "what": "FP64 tensors; block-spin product as 15 exact integer-slice products on the fp16 "
                          "tensor cores (FP64-grade); the step timed is the last one compared"
                          + ("; T, S and M propagated (5 products per step)" if impure else "")}
        del oz
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- fp16 split, per scaling
    # fractions of the last verification step's operand entries whose hi or lo plane value is
    # zero or in fp16's subnormal range, the largest |hi| (log2; the planes hold < 2^15), and
    # each scaling's ln Z/V error against the FP64 reference of those steps
    split = None
    if split_runs:
        ref, ref_name = (split_ref, "fp64_oracle") if split_ref else (oz_vals, "fp64oz")
        names = {1: "bound: 2^e from sqrt(D_b) x the first pass's largest |output|",
                 2: "exact: 2^e from the operand's largest |entry| (max pass)", 0: "fixed 2^14"}
        split = {"default": args.maxnorm, "step": nver, "modes": {}}
        for mode, (lz, st) in split_runs.items():
            n = max(1, st["entries"])
            d = {"scale": names[mode], "entries": st["entries"], "hi_zero_frac": st["hi_zero"] / n,
                 "hi_subnormal_frac": st["hi_subnormal"] / n, "lo_zero_frac": st["lo_zero"] / n,
                 "lo_subnormal_frac": st["lo_subnormal"] / n,
                 "hi_max_log2_A_B": [math.log2(x) if x > 0 else None for x in st["hi_max"]],
                 "max_abs_dlnZ_vs_default": max(abs(a - b) for a, b in zip(lz, split_runs[args.maxnorm][0]))}
            m = min(len(ref or []), len(lz))
            if m:
                d[f"max_abs_dlnZ_vs_{ref_name}_steps1to{m}"] = max(abs(lz[i] - ref[i]) for i in range(m))
            split["modes"][str(mode)] = d

    # ---------------------------------------------------------------- end to end, public API
    e2e = None
    if args.e2e and args.batch == 1 and not impure:
        full = [(i % 4, D) for i in range(LATTICE_STEPS)]
        job = HOTRG(batch=1, dcut_max=D, precision=args.precision, schedule=full, autotune=bool(args.autotune),
                    maxnorm=args.maxnorm)
        job.set_option(OPT_GEMM_VARIANT, args.gemm_variant)
        bh = torch.tensor([beta], dtype=torch.float64).pin_memory()
        hh = torch.tensor([H_WORK], dtype=torch.float64).pin_memory()
        job.init_tensor(bh.numpy(), hh.numpy())           # one untimed job: kernels and tuned plans warm
        for s in full:
            job.step(*s)
        job.lnZ()
        barrier()
        t0 = time.perf_counter()
        job.init_tensor(bh.numpy(), hh.numpy())
        fl = 0.0
        for s in full:
            fl += job.step_flops(*s)[1]
            job.step(*s)
        lnz40 = float(job.lnZ()[0])
        t1 = time.perf_counter()
        barrier()
        secs = allmax(t1 - t0)
        e2e = {"value": allsum(fl) / secs / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 16,
               "d2h_bytes_per_step": 32, "step": f"whole {LATTICE_STEPS}-step job (1024^4 sites): init from host "
               "beta, h (pinned) -> 40 steps -> ln Z/V read back, after one untimed job"
               + (" (autotuner cache filled)" if args.autotune else ""), "seconds": secs, "lnZ_over_V": lnz40}
        del job
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- CPU oracle baseline
    cpu = None
    if args.cpu and rank == 0 and world == 1:
        nx = 3 if D >= 8 else 1            # about 15-25 s of host work at D_cut = 8
        f, s = oracle_sample(D, nx=nx)
        cpu = {"value": f / s / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one steady-state D_cut={D} step of the FP64 NumPy oracle on a seeded N(0,1) tensor of "
                         f"shape ({D},)*8: full HOSVD + the block-spin contraction restricted to X, X' < {nx} "
                         f"({nx * nx}/{D * D} of the D^15 product); {s:.1f} s"}

    peak, peak_src = tensor_peak(args.precision, True)
    peak_burst, _ = tensor_peak(args.precision, False)
    achieved = prof["gemm_flops"] / (prof["gemm_ms"] * 1e-3) / 1e12 if prof["gemm_ms"] > 0 else None
    traffic = GEMM_TRAFFIC.get((args.precision, args.gemm_variant, D, args.batch, bool(impure)))
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps if ms_max else None, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": workload_config(args, world),
        "run_config": {"precision": f"{args.precision} (fp32 storage)", "cuda_graphs": bool(args.graphs),
                       "gemm_variant": args.gemm_variant, "autotune": bool(args.autotune),
                       "maxnorm": args.maxnorm,
                       "l2": f"operands larger than L2 (GEMM A and B: 2 x "
                             f"{(4 if args.precision == 'fp16x3' else 8) * D ** 10 / 1e9:.1f} GB per step, hi + lo)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "algorithmic_bytes": (2 * (4 if args.precision == "fp16x3" else 8) + 4) * float(D) ** 10,
                     "kernel": " + ".join(sorted({kernel_name(args.precision, pl["gemm_option"]) for pl in plans}))
                               + " (block-spin contraction, 2 M N K algorithmic flops per launch)",
                     "peak_source": peak_src, "launches": prof["gemm_launches"],
                     "avg_launch_ms": prof["gemm_ms"] / max(1, prof["gemm_launches"]),
                     "tensor_pipe_flops_frac": (3 * achieved / peak) if achieved else None,
                     "peak_burst": peak_burst, "frac_of_burst": (achieved / peak_burst) if achieved else None},
        "gpu_launches": prof["launches"],
        "plans": plans, "autotuner": tune,
        "clocks": clk.summary(),
        "fp64": fp64, "fp64oz": fp64oz, "accuracy": accuracy, "fp16_split": split, "lnZ_over_V_after_timed_steps": lnz_run, "observables": obs,
        "cpu_baseline": cpu, "e2e": e2e,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
