#!/usr/bin/env python
"""Benchmark of the B300 Spectral Ewald far-field grand mobility.

Workload (the large-scale configuration): N = 200000 monodisperse spheres (a = 1)
at volume fraction 0.45 in a cubic periodic box (seeded FCC-lattice subset, jitter,
hard-sphere MC sweeps), all 12 multipole components [F, T, S, S_tr] i.i.d. N(0, 1),
support P = 24, grid and Ewald parameters chosen for <= 1e-6 relative error against
the FP64 direct-Ewald oracle.  One step = one product y = M_inf . x (cell order ->
real space || spread -> 3D FFT + k-space scaling -> gather -> combine), inputs
resident on the device; the grids (>= 1 GB) exceed the 126 MB L2, so every step
streams them from HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); the product of one box does not shard,
so every rank runs an independent replica (weak scaling, no collective on the data
path); rank 0 prints one JSON line with the job-wide throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M∞·F products/s and GMRES solves/s at N=2e5, err≤1e-6 vs FP64; learned vs plain"
WORKLOAD = "mono_n200000_phi0.45_ncomp12_P24"

# Parameters for the workload (box side L = 123.02): error model of
# paper_1506_08481_b300.params with its prefactor calibrated on the oracle rows.
from paper_1506_08481_b300.params import LARGE_MONO as PARAMS  # noqa: E402

# arithmetic of the ALU-bound kernels (FP32 flop, FMA = 2): 13 FMAs per support point
# (the z-moment / column-coefficient form) plus the per-column work amortised over the
# P points of a column (spread: 13 column coefficients; gather: moment-to-output
# conversion and the compensated column sums)
FLOPS_PER_POINT = {"spread": 26.0, "gather": 26.0}
FLOPS_PER_COLUMN = {"spread": 75.0, "gather": 72.0}
# bytes of one stored real-space pair in FP32 (index 4 + separation 12 + 19 coefficients)
PAIR_BYTES = 92
# a monodisperse configuration's table stores 13 of the 19 coefficients (the others follow
# from a_i = a_j): 68 bytes per pair
PAIR_BYTES_MONO = 68

# DRAM bytes (read + write) per launch from one ncu capture of this workload (one product's launches,
# the command in profiles/dram_mono_n200000_P24.md); the spread stage is spread16w_kernel plus
# sum_parts_kernel.  Other sizes scale them by grid points (M^3), stored pairs or particles.  A kernel
# changed since that capture has no entry (its traffic is reported as null).
NCU_CAPTURE = {"N": 200000, "M": 144, "npairs": 88237670}
NCU_DRAM_BYTES = {"permute": 13.0e6, "real": 6438.9e6, "spread": 374.6e6, "fft_x_fwd": 50.6e6,
                  "fft_y_fwd": 48.5e6, "fft_z_scale": 54.0e6, "fft_y_inv": 48.5e6, "fft_x_inv": 49.4e6,
                  "gather": 149.5e6, "gather_real": 7028.7e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-solve", action="store_true", help="skip the GMRES solves (and the batch measurement)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU product and solve")
    ap.add_argument("--solve-maxit", type=int, default=800)
    ap.add_argument("--restart", type=int, default=100, help="GMRES restart length of the solves")
    ap.add_argument("--no-tuned", action="store_true", help="skip the error-model-tuned product")
    ap.add_argument("--gather", type=int, default=0, choices=[0, 1, 2],
                    help="gather kernel: by support size (0), warp per particle (1), staged bins (2)")
    ap.add_argument("--overlap", type=int, default=3, choices=[0, 1, 2, 3],
                    help="real-space sum beside the spread (0), beside the FFT chain (1), in line (2), "
                         "inside the gather kernel (3)")
    ap.add_argument("--fp64-solve-maxit", type=int, default=100,
                    help="iterations of the plain FP64 solve that are timed (it runs ~20x slower)")
    ap.add_argument("--workload", choices=["mono_n200k", "batch64", "brownian"], default="mono_n200k")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="batch64: the error model's parameters instead of timing candidates per box")
    ap.add_argument("--streams", type=int, default=8, help="batch64: streams of the captured graph")
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: skip the 64-box batch measurement carried in its line (--no-solve "
                         "skips it too: both are the line's secondary measurements)")
    ap.add_argument("--n", type=int, default=200000,
                    help="spheres (N-sweep of the large-scale configuration at the same phi and grid density)")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_time_ms(ms_local: float, world: int, device=None) -> float:
    """The job's time: the maximum over ranks of a locally measured time (the ranks
    run independent replicas; this reduction of one number is the only collective)."""
    if world <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_job: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / (ms_job * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def stage_algorithmic(stage: str, N: int, M: int, P: int, CO: int, npairs: int = 0, mono: bool = True):
    """(bound, units per launch, unit) of one launch of a stage (FP32 grids)."""
    Mh = M // 2 + 1
    if stage in ("spread", "gather"):
        return "alu", N * P ** 3 * FLOPS_PER_POINT[stage] + N * P ** 2 * FLOPS_PER_COLUMN[stage], "flop"
    if stage == "real":
        # the stored pair table streamed once, moments read and results written once
        return "hbm", npairs * (PAIR_BYTES_MONO if mono else PAIR_BYTES) + N * 12 * 4 * 2, "byte"
    if stage == "permute":
        return "hbm", N * 12 * 4 * 2, "byte"
    # FFT passes: one read and one write of the arrays they stream (bytes)
    real_f, spec_f, spec_o, real_o = 4 * M ** 3 * 4, 4 * M * M * Mh * 8, CO * M * M * Mh * 8, CO * M ** 3 * 4
    return "hbm", {"fft_x_fwd": real_f + spec_f, "fft_y_fwd": 2 * spec_f, "fft_z_scale": spec_f + spec_o,
                   "fft_y_inv": 2 * spec_o, "fft_x_inv": spec_o + real_o}.get(stage, 0), "byte"


def count_pairs(cfg, rc):
    """Ordered pairs i != j closer than rc (periodic), the rows of the real-space table."""
    from scipy.spatial import cKDTree
    pos = np.mod(cfg.pos, cfg.L)
    t = cKDTree(pos, boxsize=cfg.L)
    return int(t.count_neighbors(t, rc)) - cfg.N


def ncu_traffic(stage, M, npairs, N):
    """Scaled DRAM bytes per launch from the ncu capture, or None."""
    b = NCU_DRAM_BYTES.get(stage)
    if b is None:
        return None
    if stage in ("real", "gather_real"):      # the fused kernel's bytes are the pair table's, to 98%
        return b * npairs / NCU_CAPTURE["npairs"]
    if stage == "permute":
        return b * N / NCU_CAPTURE["N"]
    return b * (M / NCU_CAPTURE["M"]) ** 3


def roofline_entry(stage, ms, N, M, P, CO, npairs, peaks, peak_kind):
    bound, units, unit = stage_algorithmic(stage, N, M, P, CO, npairs)
    t = ms * 1e-3
    if bound == "alu":
        # measured in this run by the library's FP32 FMA probe (se_fp32_fma_probe)
        peak = peaks["fp32_fma_tflops"]
        achieved = units / t / 1e12
        return {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "ms": ms, "traffic": ncu_traffic(stage, M, npairs, N),
                "peak_source": (f"measured: FP32 FMA probe on {peaks['sms']} SMs (8 independent FMA chains per "
                                f"thread, 8 CTAs of 256 threads per SM, best of 5 launches, CUDA events)")}
    peak = peaks.get("hbm_gbs", 6400.0)
    achieved = units / t / 1e9
    return {"bound": "hbm", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "ms": ms, "traffic": ncu_traffic(stage, M, npairs, N),
            "algorithmic_bytes": units, "peak_source": f"hbm_gbs ({peak_kind})"}


def fused_entry(ms, N, M, P, CO, npairs, peaks, peak_kind):
    """Roofline of the gather kernel with the real-space sum fused in: its FMAs (the gather's)
    against the FP32 FMA peak and its table stream (the real-space sum's bytes) against HBM;
    the lower bound of its time is the larger of the two, and frac is that bound over the time."""
    g = roofline_entry("gather", ms, N, M, P, CO, npairs, peaks, peak_kind)
    r = roofline_entry("real", ms, N, M, P, CO, npairs, peaks, peak_kind)
    e = dict(g if g["frac"] >= r["frac"] else r)
    e["kernel"] = "gather_real"
    e["traffic"] = ncu_traffic("gather_real", M, npairs, N)
    e["alu_frac"], e["hbm_frac"] = g["frac"], r["frac"]
    e["algorithmic_flops"] = g["achieved"] * 1e12 * ms * 1e-3
    e["algorithmic_bytes"] = r["algorithmic_bytes"]
    e["note"] = ("gather + real-space sum in one kernel, timed in the product; bound: the larger of its FMA "
                 "and its HBM lower bounds")
    return e


def cpu_baseline(cfg, x, nrows_small=4, nrows_large=20):
    """The oracle timed on host cores on two row samples; a full product's time is the
    linear extrapolation in the number of target rows."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(7)
    times = []
    for nr in (nrows_small, nrows_large):
        rows = rng.choice(cfg.N, nr, replace=False)
        t = time.perf_counter()
        oracle.mobility(cfg.pos, cfg.rad, cfg.L, x, rows=rows, tol=1e-10)
        times.append(time.perf_counter() - t)
    per_row = max((times[1] - times[0]) / (nrows_large - nrows_small), 1e-9)
    t_full = times[0] + per_row * (cfg.N - nrows_small)
    return {"value": 1.0 / t_full, "unit": "products/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 direct Ewald on {nrows_small} and {nrows_large} target rows of the N=200000 "
                      f"workload ({times[0]:.1f} s, {times[1]:.1f} s); full product extrapolated linearly "
                      f"in rows ({t_full:.0f} s)"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_1506_08481_b300 import inputs
    import oracle
    oracle.build()
    cfg = inputs.mono_dense(seed=0, n=200000, phi=0.45)
    x = inputs.moments(cfg.N, np.random.default_rng(1), 12)
    # One oracle call per step, alternating between a small and a large set of target rows.
    # A call costs a fixed part (its k-space sums run over all N sources) plus a part
    # linear in the rows, so a full product's time is the least-squares line through the
    # (rows, seconds) samples taken at N rows.
    row_counts = (4, 20)
    rng = np.random.default_rng(11)
    samples, walls = [], []
    for step in range(args.warmup + args.steps):
        nr = row_counts[step % 2]
        rows = rng.choice(cfg.N, nr, replace=False)
        t = time.perf_counter()
        oracle.mobility(cfg.pos, cfg.rad, cfg.L, x, rows=rows, tol=1e-10)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            samples.append((nr, dt))
            walls.append(dt)
    if len({nr for nr, _ in samples}) < 2:   # fewer than two timed steps: fit the warm-up calls too
        rng = np.random.default_rng(11)
        for nr in row_counts:
            if nr in {n for n, _ in samples}:
                continue
            rows = rng.choice(cfg.N, nr, replace=False)
            t = time.perf_counter()
            oracle.mobility(cfg.pos, cfg.rad, cfg.L, x, rows=rows, tol=1e-10)
            samples.append((nr, time.perf_counter() - t))
    r = np.array([nr for nr, _ in samples], dtype=float)
    ts = np.array([dt for _, dt in samples])
    per_row, fixed = np.polyfit(r, ts, 1)
    per_row = max(per_row, 1e-9)
    t_full = max(fixed, 0.0) + per_row * cfg.N
    value = 1.0 / t_full
    sample = (f"one FP64 direct-Ewald oracle call per step on {row_counts[0]} or {row_counts[1]} random "
              f"target rows (alternating); a full product's time is the line through the (rows, s) "
              f"samples at N rows: {max(fixed, 0.0):.2f} s + {per_row * 1e3:.1f} ms/row x {cfg.N} = {t_full:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "ms_per_product_extrapolated": 1e3 * t_full, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{row_counts[0]} or {row_counts[1]} target rows of the product per step"},
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_1506_08481_b300 import api, inputs

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cfg = inputs.mono_dense(seed=0, n=args.n, phi=0.45)
    x_host = inputs.moments(cfg.N, np.random.default_rng(1), 12)
    P_ = dict(PARAMS)
    if args.n != 200000:
        from paper_1506_08481_b300 import params as prm
        need = P_["M"] * cfg.L / 123.018      # same grid spacing (same accuracy)
        P_["M"] = min(v for v in prm.fft_sizes() if v >= need)
    ctx = api.Context(local)
    ctx.set_params(P_["xi"], P_["M"], P_["P"], P_["rc"])
    ctx.set_option(api.SE_OPT_SHAPE_M, P_["m"])
    ctx.set_option(api.SE_OPT_SIZE_MODE, P_["size_mode"])
    ctx.set_option(api.SE_OPT_PRECISION, 0)
    ctx.set_option(api.SE_OPT_OVERLAP, args.overlap)
    ctx.set_option(api.SE_OPT_GATHER, args.gather)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    x = torch.tensor(x_host, device=dev, dtype=torch.float32)
    y = torch.empty_like(x)

    # accuracy against the stored oracle rows (computed by tests/golden/make_golden.py)
    acc, acc_blocks = None, None
    gpath = os.path.join(ROOT, "tests", "golden", "mono_n200k_rows.npz")
    if os.path.exists(gpath) and args.n == 200000:
        g = np.load(gpath)
        ctx.apply(x, y)
        yg = y.double().cpu().numpy()[g["rows"]]
        acc = float(np.linalg.norm(yg - g["y"]) / np.linalg.norm(g["y"]))
        acc_blocks = {}
        for name, sl in (("U", slice(0, 3)), ("Omega", slice(3, 6)), ("E", slice(6, 11)), ("E_tr", slice(11, 12))):
            d, r = yg[:, sl] - g["y"][:, sl], g["y"][:, sl]
            acc_blocks[name] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(r)),
                                "e_inf_r": float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(r, axis=1)))}

    for _ in range(args.warmup):
        ctx.apply(x, y)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.set_option(api.SE_OPT_TIMING, 1)
    launches0 = ctx.kernel_launches()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.apply(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    nprod, stage_ms = ctx.stage_times()
    ctx.set_option(api.SE_OPT_TIMING, 0)
    clk = clocks.stop()
    ms = job_time_ms(ms, world, dev)
    ms_step = ms / args.steps
    value = job_rate(args.steps, ms, world)

    # end to end through the host-buffer entry point (copies in the timed region)
    x64 = np.ascontiguousarray(x_host)
    y64 = np.empty_like(x64)
    try:
        xp = torch.from_numpy(x64).pin_memory().numpy()
        yp = torch.from_numpy(y64).pin_memory().numpy()
    except RuntimeError:
        xp, yp = x64, y64
    ctx.set_option(api.SE_OPT_PRECISION, 0)
    ctx.apply_host(xp, yp)
    ne2e = max(5, args.steps // 4)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t = time.perf_counter()
    for _ in range(ne2e):
        ctx.apply_host(xp, yp)
    e2e = job_rate(ne2e, job_time_ms(1e3 * (time.perf_counter() - t), world, dev), world)

    # configuration setup (what a dynamic simulation pays once per time step): wrap and
    # cell sort, spreading bins, neighbour lists and the FP32 pair table, timed as
    # set_config + one product minus the product's own time
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    ctx.apply(x, y)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t) - ms_step

    # the plain FP64 GPU path on the same workload: products/s and accuracy
    fp64 = None
    if not args.no_fp64:
        ctx.set_option(api.SE_OPT_PRECISION, 1)
        xd = x.double()
        yd = torch.empty_like(xd)
        for _ in range(3):
            ctx.apply(xd, yd)
        n64 = max(3, args.steps // 4)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n64):
            ctx.apply(xd, yd)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        ctx.set_option(api.SE_OPT_TIMING, 1)
        ctx.stage_times()
        ctx.apply(xd, yd)
        n1, st64 = ctx.stage_times()
        ctx.set_option(api.SE_OPT_TIMING, 0)
        acc64 = None
        if acc is not None:
            acc64 = float(np.linalg.norm(yd.cpu().numpy()[g["rows"]] - g["y"]) / np.linalg.norm(g["y"]))
        fp64 = {"value": world * 1e3 / ms64, "unit": "products/s", "ms_per_product": ms64,
                "rel_l2_vs_fp64_oracle": acc64, "fp32_speedup": ms64 / ms_step,
                "stage_ms_per_product": {k: v / max(n1, 1) for k, v in st64.items()}}
        # the FP64-equivalent mode: spread and gather in double-float, the rest in FP64
        ctx.set_option(api.SE_OPT_PRECISION, 2)
        yf = torch.empty_like(xd)
        for _ in range(2):
            ctx.apply(xd, yf)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n64):
            ctx.apply(xd, yf)
        e1.record(stream)
        torch.cuda.synchronize()
        msff = e0.elapsed_time(e1) / n64
        ctx.set_option(api.SE_OPT_TIMING, 1)
        ctx.stage_times()
        ctx.apply(xd, yf)
        nf, stff = ctx.stage_times()
        ctx.set_option(api.SE_OPT_TIMING, 0)
        accff = None
        if acc is not None:
            accff = float(np.linalg.norm(yf.cpu().numpy()[g["rows"]] - g["y"]) / np.linalg.norm(g["y"]))
        fp64["double_float_mode"] = {
            "value": world * 1e3 / msff, "unit": "products/s", "ms_per_product": msff,
            "rel_l2_vs_fp64_oracle": accff,
            "rel_diff_vs_fp64_mode": float(torch.linalg.norm(yf - yd) / torch.linalg.norm(yd)),
            "stage_ms_per_product": {k: v / max(nf, 1) for k, v in stff.items()}}
        del yf
        del xd, yd
        ctx.set_option(api.SE_OPT_PRECISION, 0)

    # the same product at the parameters the error model picks for this box at 5e-7 in
    # FP32 (method error plus FP32 rounding floor), so the product still meets 1e-6; the
    # support P is then the model's choice instead of the configuration's P = 24
    tuned, ct = None, None
    if not args.no_tuned and args.n == 200000:
        from paper_1506_08481_b300 import params as prm
        sp = prm.choose(cfg.L, cfg.N, 5e-7, M_max=384, precision=0)
        ct = api.Context(local)
        ct.set_params(sp.xi, sp.M, sp.P, sp.rc)
        ct.set_option(api.SE_OPT_SHAPE_M, sp.m)
        ct.set_option(api.SE_OPT_SIZE_MODE, 1)
        ct.set_option(api.SE_OPT_PRECISION, 0)
        ct.set_option(api.SE_OPT_GATHER, args.gather)
        ct.set_config(cfg.pos, cfg.rad, cfg.L)
        yt = torch.empty_like(x)
        for _ in range(3):
            ct.apply(x, yt)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ct.apply(x, yt)
        e1.record(stream)
        torch.cuda.synchronize()
        mst = e0.elapsed_time(e1) / args.steps
        acct = None
        if acc is not None:
            acct = float(np.linalg.norm(yt.double().cpu().numpy()[g["rows"]] - g["y"]) / np.linalg.norm(g["y"]))
        tuned = {"value": world * 1e3 / mst, "unit": "products/s", "ms_per_product": mst,
                 "rel_l2_vs_fp64_oracle": acct,
                 "params": {"xi": sp.xi, "M": sp.M, "P": sp.P, "rc": sp.rc, "m": sp.m, "model_tol": 5e-7}}
        del yt

    # GMRES solves of M x = b (F, T, S; b = the first 11 input components) to 1e-6:
    # FP32 products + FP64 true residual and refinement, with the plain block-diagonal,
    # the learned and the spectral preconditioner, and the plain FP64 GPU path with the
    # block one; then the block and spectral solves again at the error model's parameters
    solve = None
    if not args.no_solve:
        b = torch.tensor(x_host[:, :11], device=dev, dtype=torch.float64)
        xs = torch.zeros_like(b)
        wpath = os.path.join(ROOT, "paper_1506_08481_b300", "learned_pc_weights.npy")

        def solves(c, runs):
            out = {}
            c.set_option(api.SE_OPT_RESTART, args.restart)
            if os.path.exists(wpath):
                c.set_learned_weights(np.load(wpath))
            for name, prec, pc, maxit in runs:
                c.set_option(api.SE_OPT_PRECISION, prec)
                c.solve(b, xs, rtol=1e-6, maxit=2, precond=pc, allow_not_converged=True)   # setup
                xs.zero_()
                torch.cuda.synchronize()
                if world > 1:
                    torch.distributed.barrier()
                t = time.perf_counter()
                _, iters, relres = c.solve(b, xs, rtol=1e-6, maxit=maxit, precond=pc, allow_not_converged=True)
                torch.cuda.synchronize()
                ts = job_time_ms(1e3 * (time.perf_counter() - t), world, dev) / 1e3
                out[name] = {"solves_per_s": world / ts, "seconds": ts, "iterations": iters,
                             "relres_fp64": relres, "converged": bool(relres <= 1e-6)}
            c.set_option(api.SE_OPT_PRECISION, 0)
            return out

        runs = [("fp32_block", 0, api.SE_PRECOND_BLOCK, args.solve_maxit),
                ("fp32_learned", 0, api.SE_PRECOND_LEARNED, args.solve_maxit),
                ("fp32_spectral", 0, api.SE_PRECOND_SPECTRAL, args.solve_maxit)]
        if not args.no_fp64:
            runs.append(("fp64_block", 1, api.SE_PRECOND_BLOCK, args.fp64_solve_maxit))
        solve = {"ncomp": 11, "rtol": 1e-6, "restart": args.restart, "maxit": args.solve_maxit,
                 "learned_weights": os.path.exists(wpath),
                 "params": {k: P_[k] for k in ("xi", "M", "P", "rc")}}
        solve.update(solves(ctx, runs))
        if "fp64_block" in solve and not solve["fp64_block"]["converged"]:
            # the FP64 path timed over its first maxit iterations; the time of a whole solve
            # is projected at the iteration count of the FP32 block-preconditioned solve
            r = solve["fp64_block"]
            r["seconds_per_iteration"] = r["seconds"] / max(r["iterations"], 1)
            r["projected_seconds"] = r["seconds_per_iteration"] * solve["fp32_block"]["iterations"]
            r["solves_per_s"] = world / r["projected_seconds"]
            r["note"] = (f"timed over {r['iterations']} iterations; solves/s projected at the FP32 "
                         f"solve's {solve['fp32_block']['iterations']} iterations")
        # headline: the learned preconditioner (the block preconditioner with the
        # long-wavelength correction whose damping and cutoff the network sets); the plain
        # block and the correction with its fixed defaults beside it
        solve["solves_per_s"] = solve["fp32_learned"]["solves_per_s"]
        solve["headline"] = "fp32_learned"
        solve["spectral_vs_block"] = solve["fp32_spectral"]["solves_per_s"] / solve["fp32_block"]["solves_per_s"]
        solve["learned_vs_block"] = solve["fp32_learned"]["solves_per_s"] / solve["fp32_block"]["solves_per_s"]
        solve["learned_vs_spectral"] = solve["fp32_learned"]["solves_per_s"] / solve["fp32_spectral"]["solves_per_s"]
        if ct is not None:
            tuned_solves = solves(ct, [("fp32_block", 0, api.SE_PRECOND_BLOCK, args.solve_maxit),
                                       ("fp32_spectral", 0, api.SE_PRECOND_SPECTRAL, args.solve_maxit),
                                       ("fp32_learned", 0, api.SE_PRECOND_LEARNED, args.solve_maxit)])
            tuned_solves["params"] = tuned["params"]
            solve["tuned_params"] = tuned_solves
    if ct is not None:
        ct.close()

    # every stage as a kernel of its own (overlap 2: the real-space sum in line), so that the
    # per-kernel table times the gather without the real-space sum fused into it
    ctx.set_option(api.SE_OPT_OVERLAP, 2)
    ctx.apply(x, y)
    ctx.set_option(api.SE_OPT_TIMING, 1)
    for _ in range(5):
        ctx.apply(x, y)
    nsep, stsep = ctx.stage_times()      # the events since the last call: these 5 products
    ctx.set_option(api.SE_OPT_TIMING, 0)
    ctx.set_option(api.SE_OPT_OVERLAP, args.overlap)
    sep = {k: v / max(nsep, 1) for k, v in stsep.items()}

    # the real-space kernel alone
    ctx.set_option(api.SE_OPT_PARTS, 1)
    ctx.set_option(api.SE_OPT_TIMING, 0)
    ctx.apply(x, y)
    ctx.set_option(api.SE_OPT_TIMING, 1)
    nprod0, st0 = ctx.stage_times()
    for _ in range(5):
        ctx.apply(x, y)
    nprod1, st1 = ctx.stage_times()
    ctx.set_option(api.SE_OPT_TIMING, 0)
    ctx.set_option(api.SE_OPT_PARTS, 7)
    real_alone_ms = (st1["real"] - st0["real"]) / max(nprod1 - nprod0, 1)

    # roofline of every kernel; the dominant one is the serial stage with the largest time
    peaks, peak_kind = measured_peaks()
    peaks = dict(peaks)
    peaks["fp32_fma_tflops"], peaks["sms"] = api.fp32_fma_peak(local)
    CO = 8 if P_["size_mode"] == 0 else 4
    npairs = count_pairs(cfg, P_["rc"])
    per_prod = {k: v / max(nprod, 1) for k, v in stage_ms.items()}
    # overlap 3 runs the real-space sum inside the gather kernel: its "real" stage is empty
    # and its "gather" stage is the fused kernel
    fused = args.overlap == 3 and per_prod.get("real", 0.0) < 0.05 * sep.get("real", 1.0)
    kernels = {}
    for k, v in sep.items():
        kernels[k] = roofline_entry(k, real_alone_ms if k == "real" else v, cfg.N, P_["M"], P_["P"], CO, npairs,
                                    peaks, peak_kind)
    kernels["real"]["note"] = "timed alone (real-space part only)"
    for k in kernels:
        if k != "real":
            kernels[k]["note"] = "timed as a kernel of its own (real-space sum in line)"
    if fused:
        kernels["gather_real"] = fused_entry(per_prod["gather"], cfg.N, P_["M"], P_["P"], CO, npairs, peaks,
                                             peak_kind)
    timed = {("gather_real" if (k == "gather" and fused) else k): v for k, v in per_prod.items()}
    dom = max((k for k in timed if k not in ("real", "permute")), key=lambda k: timed[k])
    roof = dict(kernels[dom])
    roof["traffic_source"] = ("ncu DRAM bytes per launch of this workload's capture (scaled by grid points, "
                              "pairs or particles at other sizes)"
                              if roof["traffic"] is not None else "kernel changed since the last capture")

    # the 64-box batch (graph, persistent launch, per-box loop), as --workload batch64 measures it
    batch = None
    if not (args.no_batch or args.no_solve):
        bl = measure_batch(args, rank, world, local, dev)
        if rank == 0:
            batch = {k: bl[k] for k in ("metric", "value", "unit", "ms_per_step", "graph_of_per_box_launches",
                                        "persistent_launch", "per_box_launch_loop")}
            batch["boxes"], batch["N_total"] = 64, bl["config"]["N_total"]
            batch["launch"] = bl["config"]["launch"]

    workload = WORKLOAD if args.n == 200000 else WORKLOAD.replace("n200000", f"n{args.n}")
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(cfg, x_host)
        line = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload, "N": cfg.N, "L": round(cfg.L, 4), "phi": 0.45, "ncomp": 12,
                           "xi": P_["xi"], "M": P_["M"], "P": P_["P"], "rc": P_["rc"], "m": P_["m"],
                           "size_mode": "real-space" if P_["size_mode"] else "hybrid",
                           "real_space_overlap": ["beside spread", "beside FFT", "in line",
                                                  "inside the gather kernel" if fused else "in line"][args.overlap],
                           "parallelism": f"replicas x{world}",
                           "l2": "grids and spectra (>1 GB per product) exceed L2; inputs resident"},
                "accuracy": {"rel_l2_vs_fp64_oracle": acc, "rows": 1000, "per_block": acc_blocks,
                             "note": "FP32 product against the stored FP64 direct-Ewald oracle rows; "
                                     "e_inf_r = max over rows of the per-particle relative error (Eq. err-E)"},
                "roofline": roof,
                "stage_ms_per_product": per_prod, "stage_ms_per_product_separate_kernels": sep,
                "kernels": kernels, "npairs_real_space": npairs,
                "config_setup_ms": setup_ms,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e, "unit": "products/s", "h2d_bytes_per_step": int(x64.nbytes),
                        "d2h_bytes_per_step": int(y64.nbytes)},
                "gpu_launches": int(launches), "clocks": clk, "fp64_product": fp64, "tuned_product": tuned, "solve": solve,
                "batch64": batch}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args, rank, world, local):
    """64 independent boxes (N ~ U[500, 8000], radii 1 and 1.5, phi ~ U[0.1, 0.45]),
    forces only, FP32, per-box parameters for 1e-6; one step = one product of every box.
    The captured graph (boxes concurrent on 8 streams) against a per-box launch loop."""
    import torch

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    line = measure_batch(args, rank, world, local, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_batch(args, rank, world, local, dev):
    """The 64-box measurement of run_batch; returns its JSON line (a dict)."""
    import torch
    from paper_1506_08481_b300 import api, inputs, params

    boxes = inputs.batch_boxes(seed=0)
    rng = np.random.default_rng(1)
    ctxs, xs, ys, chosen = [], [], [], []
    tune_s = time.perf_counter()
    for cfg in boxes:
        # <= 1e-6 against the oracle on every box: the error model's method tolerance 2.5e-7
        # (it underestimates the method error of the small supports by about 2x) and the
        # FP32 rounding floor 1e-6 (measured: worst box 6.0e-7 over the 64 boxes)
        if args.autotune:
            sp, mode, _, opts = params.autotune(cfg, 2.5e-7, ncomp=3, fp32_tol=1e-6)
        else:
            sp = params.choose(cfg.L, cfg.N, 2.5e-7, M_max=128, a_eff=params.effective_radius(cfg.rad),
                               precision=0, fp32_tol=1e-6)
            mode, opts = 1, {"spread": 0}
        c = api.Context(local)
        c.set_params(sp.xi, sp.M, sp.P, sp.rc)
        c.set_option(api.SE_OPT_SHAPE_M, sp.m)
        c.set_option(api.SE_OPT_SIZE_MODE, mode)
        c.set_option(api.SE_OPT_SPREAD, opts["spread"])
        c.set_config(cfg.pos, cfg.rad, cfg.L)
        xs.append(torch.tensor(rng.standard_normal((cfg.N, 3)), device=f"cuda:{local}", dtype=torch.float32))
        ys.append(torch.empty_like(xs[-1]))
        ctxs.append(c)
        chosen.append((sp.M, sp.P, mode, opts["spread"]))
    tune_s = time.perf_counter() - tune_s
    stream = torch.cuda.current_stream()

    def timed(batch, use_graph):
        for _ in range(args.warmup):
            batch.apply(xs, ys, use_graph=use_graph)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            batch.apply(xs, ys, use_graph=use_graph)
        e1.record(stream)
        torch.cuda.synchronize()
        return job_time_ms(e0.elapsed_time(e1), world, dev) / args.steps

    launches0 = sum(c.kernel_launches() for c in ctxs)
    b = api.Batch(ctxs, nstreams=1)
    ms_loop = timed(b, False)
    b.close()
    clocks = ClockSampler(local)
    clocks.start()
    # (a) one CUDA graph of every box's kernels on a pool of streams
    b = api.Batch(ctxs, nstreams=args.streams)
    ms_graph = timed(b, True)
    # kernels in one replay of the graph = those of one eager pass over the boxes
    l0 = sum(c.kernel_launches() for c in ctxs)
    b.apply(xs, ys, use_graph=False)
    torch.cuda.synchronize()
    graph_kernels = sum(c.kernel_launches() for c in ctxs) - l0
    b.close()
    # (b) one persistent cooperative launch for all 64 boxes
    b = api.Batch(ctxs, nstreams=args.streams)
    ms_pers = timed(b, api.Batch.PERSISTENT)
    b.status()
    b.close()
    clk = clocks.stop()
    ntot = sum(c.N for c in boxes)
    best = "graph" if ms_graph <= ms_pers else "persistent"
    ms_best = min(ms_graph, ms_pers)
    line = None
    if rank == 0:
        line = {"metric": "aggregate box products/s, 64 uneven boxes (forces only)", "value": job_rate(64, ms_best, world),
                "unit": "box products/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_best, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch64", "boxes": 64, "N_total": ntot, "ncomp": 3,
                           "params": ("autotuned (grid, support, size mode, spreading tiles; timed)" if args.autotune
                                      else "error-model choice for 1e-6"),
                           "setup_seconds": tune_s,
                           "M_P_mode_spread_per_box": chosen, "streams": args.streams,
                           "launch": {"graph": "one CUDA graph of the boxes' kernels on a stream pool",
                                      "persistent": "one persistent cooperative launch for all boxes"}[best]},
                "gpu_launches": graph_kernels if best == "graph" else 1,
                "graph_of_per_box_launches": {"value": job_rate(64, ms_graph, world), "ms_per_step": ms_graph,
                                              "kernels_per_step": graph_kernels},
                "persistent_launch": {"value": job_rate(64, ms_pers, world), "ms_per_step": ms_pers,
                                      "kernels_per_step": 1},
                "per_box_launch_loop": {"value": job_rate(64, ms_loop, world), "ms_per_step": ms_loop},
                "graph_speedup": ms_loop / ms_graph,
                "persistent_speedup": ms_loop / ms_pers,
                "gpu_launches_setup_and_eager": sum(c.kernel_launches() for c in ctxs) - launches0,
                "clocks": clk}
    for c in ctxs:
        c.close()
    return line


def run_brownian(args, rank, world, local):
    """Far-field Brownian source M^{-1/2} Psi (F, T, S; Sec. 4.3) by the Swan-Brady IVP,
    dtau = 0.1, on the log-normal suspension (N = 20000, phi = 0.4), FP32 products with
    FP64 refinement, each of the 20 GMRES solves to 1e-6.  One step = one IVP."""
    import torch
    from paper_1506_08481_b300 import api, inputs, params

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cfg = inputs.lognormal(seed=3, n=20000, phi=0.4)
    sp = params.choose(cfg.L, cfg.N, 5e-7, M_max=128, a_eff=params.effective_radius(cfg.rad), precision=0)
    ctx = api.Context(local)
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_SIZE_MODE, 1)
    ctx.set_option(api.SE_OPT_RESTART, 100)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    psi = torch.tensor(np.random.default_rng(7).standard_normal((cfg.N, 11)), device=dev, dtype=torch.float64)
    x10, prods = ctx.brownian_ivp(psi, nsteps=10, rtol=1e-6, maxit=2000)          # warm-up (preconditioner)
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        x10, prods = ctx.brownian_ivp(psi, nsteps=10, rtol=1e-6, maxit=2000)
    ms = job_time_ms(1e3 * (time.perf_counter() - t), world, dev) / steps
    x20, prods20 = ctx.brownian_ivp(psi, nsteps=20, rtol=1e-6, maxit=2000)
    disc = float(torch.linalg.norm(x10 - x20) / torch.linalg.norm(x20))
    # far-field self-diffusivities (Sec. 6.1): 4 random force-torque samples, rigid spheres
    fr = torch.tensor(np.random.default_rng(8).standard_normal((4, cfg.N, 6)), device=dev, dtype=torch.float64)
    torch.cuda.synchronize()
    t = time.perf_counter()
    dvals, dprods = ctx.far_field_diffusivity(fr, rtol=1e-6, maxit=2000)
    dsec = time.perf_counter() - t
    a = torch.tensor(cfg.rad, device=dev, dtype=torch.float64)
    dt = float((dvals[:, 0] * 6 * math.pi * a).mean())          # d_s^t / d_0 averaged over particles
    dr = float((dvals[:, 1] * 8 * math.pi * a ** 3).mean())     # d_s^r / d_0
    # Eq. dst-corr with the far-field high-frequency viscosity: 1.76 (eta / eta_s) (phi/N)^(1/3)
    # times kT / (6 pi eta <a^3>^(1/3)), in units of each particle's d_0
    t = time.perf_counter()
    eta_s, vprods = ctx.high_frequency_viscosity(rtol=1e-6, maxit=2000)
    vsec = time.perf_counter() - t
    a3 = float(np.mean(cfg.rad ** 3)) ** (1 / 3)
    corr = float((1.76 * (a / a3) / eta_s * (0.4 / cfg.N) ** (1 / 3)).mean())
    if rank == 0:
        line = {"metric": "far-field Brownian IVPs M^-1/2 Psi per second (N=20000 log-normal, F,T,S)",
                "value": job_rate(1, ms, world), "unit": "IVPs/s", "n_gpus": world, "steps": steps, "warmup": 1,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "brownian_lognormal_n20000_phi0.4", "N": cfg.N, "ncomp": 11, "dtau": 0.1,
                           "solve_rtol": 1e-6, "params": {"xi": sp.xi, "M": sp.M, "P": sp.P, "rc": sp.rc}},
                "products_per_ivp": prods, "products_per_ivp_dtau_0.05": prods20,
                "rel_diff_dtau_0.1_vs_0.05": disc,
                "far_field_diffusivity": {"samples": 4, "seconds": dsec, "products": dprods,
                                          "dt_over_d0_mean": dt, "dr_over_d0_mean": dr,
                                          "dt_over_d0_mean_size_corrected": dt + corr,
                                          "high_frequency_viscosity_ratio": eta_s,
                                          "viscosity_seconds": vsec, "viscosity_products": vprods}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch64":
        run_batch(args, rank, world, local)
    elif args.workload == "brownian":
        run_brownian(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
