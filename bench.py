#!/usr/bin/env python
"""Benchmark: ground-state solves per second of the cascadic-multigrid PCG
solver on a GB300, plus p50/p99 solve latency.

Workload (one step = one full solve, all steps of the method): 2D, 512x512 on
[-16,16]^2, cascadic multigrid 128 -> 256 -> 512 by spectral zero padding,
harmonic trap, Omega = 0.9, gamma = 1, beta0 = 1000, beta1 = -5, seeded
vortex-phase initial guess, stop when the accepted step changes the energy by
less than 1e-12.  FP64 arithmetic (`--precision fp64`, the default) or FP32
transforms with FP64 reductions and FP64 polishing (`--precision mixed`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own seeded problem on its own GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on this machine's host cores on
a bounded sample of the same workload (see `cpu_sample`).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import seeded_inputs as si  # noqa: E402

METRIC = "ground-state solves/s & p50/p99 latency vs plain FP64 PCG, same energy tol"
N_FINE = (512, 512)
L_BOX = (16.0, 16.0)
LEVELS = 3
PAR = (0.9, 1.0, 1000.0, -5.0)
TOL = 1e-12
RES_TOL = 1e-8
WORKLOAD = ("2D CM-PCG 128->256->512, 512x512 on [-16,16]^2, harmonic trap, Omega=0.9, gamma=1, "
            "beta0=1000, beta1=-5, seeded vortex-phase guess, stop |dE|<1e-12 and max|r|<1e-8 on every level")
# Per-level iteration counts (128^2, 256^2, 512^2) of one plain FP64 solve of this workload, as the
# FP64 arm of the main run reports them in `fp64_plain.level_iters` (the GPU path follows the
# oracle's iterations step by step); the reference arm scales its timed oracle sample by them.
REF_LEVEL_ITERS = (38561, 29677, 17)
L2_BYTES = 256 << 20


def coarse_shape():
    return tuple(k >> (LEVELS - 1) for k in N_FINE)


def initial_guess(rank: int) -> np.ndarray:
    return si.gaussian_guess(coarse_shape(), L_BOX, si.seed_for(2, rank), vortex=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline bookkeeping
def fft_flops(n: int) -> float:
    """Standard operation count of a length-n complex radix-2 FFT: 5 n log2 n."""
    return 5.0 * n * math.log2(n)


# 1-D transforms per launch (of every line of one component) and 3-component arrays
# moved per launch (each array read or written once: the algorithmic minimum)
KERNEL_WORK = {
    "row_fwd_upd": (1, "row", 4), "row_fwd": (1, "row", 2), "coly_ymid_h": (3, "col", 3),
    "row_inv_h": (2, "row", 4), "row_fwd_pre": (1, "row", 4), "coly_mid_pre": (2, "col", 2),
    "row_inv_pre": (1, "row", 6), "row_fwd_proj": (1, "row", 5),
    "row_inv_p": (2, "row", 5),
}
# Hybrid iteration (FP64 state, FP32 directions): algorithmic bytes per grid point and
# component of each pass (FP64 complex 16 B, FP32 complex 8 B; every array read or
# written once).  hy_upd: R Phi, H_lin Phi (FP64), P, H_lin P (FP32); W Phi, H_lin Phi,
# H(Phi) (FP64), FP32 Phi.  row_fwd_pre_hy: R Phi, H(Phi); W r, F_x(P_V^1/2 r).
# row_inv_pre: R spectrum, FP32 Phi, r, r_prev, P_prev; W z.  coly_ymid_h in the hybrid P
# chain also reads and writes the spectra of Phi and P.  row_inv_p_hy: R T', G, P, FP32
# Phi, r, FP64 Phi; W H_lin P.
HYBRID_BYTES = {"hy_upd": 104, "row_fwd_pre_hy": 48, "coly_mid_pre": 16, "row_inv_pre": 48,
                "row_fwd_proj": 40, "coly_ymid_h": 56, "row_inv_p_hy": 64}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) measured with ncu
# on the kernel inside this workload: (kernel, grid points per axis, 1 = FP32 / 0 = FP64).
# At 128^2 the arrays stay in L2 (0 bytes written back during the launch).
NCU_DRAM_BYTES = {("coly_ymid_h", 128, 0): 869888.0,
                  # ncu --set full, one launch of the 256^2 kernel case (inputs L2-resident: reads only)
                  ("row_inv_p_hy", 256, 2): 11141632.0}


def launch_bytes(name: str, n, prec: int) -> float:
    """Algorithmic bytes of one launch on one solve in the given precision mode."""
    if prec == 2:
        return HYBRID_BYTES.get(name, 0) * 3.0 * n[0] * n[1]
    return kernel_bytes(name, n, 8 if prec == 1 else 16)


def kernel_flops(name: str, n) -> float:
    """Algorithmic flops of one launch of a 2D pass on one solve (3 components):
    the 1-D FFTs it performs, 5 n log2 n each; pointwise work is not counted."""
    nx, ny = n
    k, kind, _ = KERNEL_WORK.get(name, (0, "row", 0))
    per = fft_flops(nx) * ny if kind == "row" else fft_flops(ny) * nx
    return 3.0 * k * per


def kernel_bytes(name: str, n, elem: int) -> float:
    """Algorithmic DRAM bytes of one launch on one solve: 3-component arrays of
    n^2 complex values (elem bytes each), each read or written once."""
    return KERNEL_WORK.get(name, (0, "row", 0))[2] * 3.0 * n[0] * n[1] * elem


# ------------------------------------------------------------------ oracle (CPU) sample
def cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, or lscpu on Arm)."""
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_worker(iters_per_level):
    import os as _os
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[v] = "1"
    return oracle_sample(iters_per_level)[0]


def oracle_baseline(iters_per_level):
    """The oracle timed on one host core and on all of them: the single-core solve time
    (per-level sample x iteration counts) and the throughput of independent solves, one
    per core, all cores busy at once (spawned worker processes)."""
    import multiprocessing as mp
    t1, desc = oracle_sample(iters_per_level)
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        times = pool.map(_oracle_worker, [tuple(iters_per_level)] * cores)
    rate_all = sum(1.0 / t for t in times)
    return {"value": rate_all, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "single_core_value": 1.0 / t1, "cpu_model": cpu_model(), "nproc": cores,
            "sample": desc + f"; all {cores} cores: one independent oracle sample per core at once, "
                             "throughput = sum of their rates (extrapolated solves, not whole solves)"}


def oracle_sample(iters_per_level, budget_s: float = 20.0):
    """Time the FP64 CPU oracle's PCG iterations on each level of the workload and
    scale by the iteration counts of a full solve.  Returns (seconds per solve,
    description of the sample)."""
    from oracle.model import Grid, Model, Trap
    from oracle.pcg import Options, pcg
    psi = initial_guess(0)
    per_iter = []
    desc = []
    for lev, its in enumerate(iters_per_level):
        n = tuple(k >> (LEVELS - 1 - lev) for k in N_FINE)
        m = Model(Grid(n, L_BOX), Trap(), Omega=PAR[0], gamma=PAR[1], c0=PAR[2], c1=PAR[3])
        if lev > 0:
            psi = np.stack([np.kron(psi[c], np.ones((2, 2))) for c in range(3)])  # any state of the right size
        k = {0: 8, 1: 3, 2: 2}[lev]
        t0 = time.perf_counter()
        pcg(m, psi, Options(tol=1e-300, max_iter=k))
        dt = (time.perf_counter() - t0) / (k + 1)       # k iterations plus the final H evaluation
        per_iter.append(dt)
        desc.append(f"{n[0]}^2: {k} its, {dt * 1e3:.0f} ms/it")
    total = sum(t * i for t, i in zip(per_iter, iters_per_level))
    return total, ("oracle PCG iterations timed per level (" + "; ".join(desc) + ") x the per-level iteration "
                   f"counts of one solve {list(iters_per_level)}")


# ------------------------------------------------------------------ multi-rank bookkeeping
def reduce_max(value: float) -> float:
    """Maximum of `value` over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return value
    dev = "cpu" if tdist.get_backend() == "gloo" else torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, max_total_ms: float, solves_per_step: int = 1) -> float:
    """Solves per second of the whole job: every rank solves `solves_per_step`
    independent problems per step; the job takes the slowest rank's time."""
    return world * solves_per_step * steps * 1000.0 / max_total_ms


# ------------------------------------------------------------------ our arm
def timed_solves(prob, opts, d_psi0, flush, stream, warmup, steps, torch):
    """W untimed + K timed solves from the device-resident guess; CUDA events on
    the solver's stream around each solve, L2 flushed between solves."""
    def step():
        prob.set_initial_device(d_psi0.data_ptr(), level=LEVELS - 1)
        return prob.solve(**opts)[0]
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    lat, results = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step()
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
        results.append(r)
    return lat, results


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    from paper_2602_17950_gb300.gpsoc import probe_peaks

    build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    prec = {"fp64": 0, "mixed": 1, "hybrid": 2}[args.precision]
    psi0 = initial_guess(rank)
    d_psi0 = torch.from_numpy(psi0[None].copy()).to(dev)
    flush = torch.empty(L2_BYTES // 4, dtype=torch.float32, device=dev)
    # tiles of every level's passes, FP32 and FP64 kernels, tuned before anything is timed
    # (the table is process-wide: both arms and every level of the solve use it)
    tiles, t_tune = {}, time.perf_counter()
    if not args.no_tune:
        for lev in range(LEVELS):
            n = tuple(k >> (LEVELS - 1 - lev) for k in N_FINE)
            with Problem(n, L_BOX, [PAR]) as pt:
                for pr, key in ((2, "fp32"), (0, "fp64")):
                    pt.set_initial(si.gaussian_guess(n, L_BOX, si.seed_for(2, rank), vortex=True)[None])
                    tiles.setdefault(f"{n[0]}^2", {})[key] = pt.autotune(iters=6, precision=pr, tol=TOL)
    t_tune = time.perf_counter() - t_tune
    prob = Problem(N_FINE, L_BOX, [PAR])
    opts = dict(precision=prec, tol=TOL, res_tol=RES_TOL, cm_levels=LEVELS, check_every=64)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    launches0 = prob.kernel_launches()
    with ClockSampler(local_rank) as clk:
        lat, results = timed_solves(prob, opts, d_psi0, flush, stream, args.warmup, args.steps, torch)
    launches = prob.kernel_launches() - launches0
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    max_total_ms = reduce_max(sum(lat))
    ok = all(r["status"] == "OK" for r in results)
    # warm-up launches are included in the counter: keep only the timed solves' share
    launches_timed = int(round(launches * args.steps / (args.steps + args.warmup)))

    # the plain FP64 PCG on the same workload and tolerance (the comparison of the metric)
    fp64 = None
    if prec != 0 and not args.no_fp64:
        lat64, res64 = timed_solves(prob, dict(opts, precision=0), d_psi0, flush, stream, 1, args.fp64_steps, torch)
        fp64 = {"value": world * 1000.0 / statistics.mean(lat64), "unit": "solves/s",
                "ms_per_solve": statistics.mean(lat64), "p50_ms": float(np.percentile(lat64, 50)),
                "p99_ms": float(np.percentile(lat64, 99)), "samples": len(lat64),
                "status_ok": all(r["status"] == "OK" for r in res64),
                "energy": res64[-1]["energy"], "mu": res64[-1]["mu"], "res_inf": res64[-1]["res_inf"],
                "iters_total": res64[-1]["total_iters"], "level_iters": res64[-1]["level_iters"]}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    h_in = torch.empty(psi0[None].shape, dtype=torch.complex128, pin_memory=True)
    h_in.numpy()[...] = psi0[None]
    h_out = torch.empty((1, 3) + tuple(N_FINE[::-1]), dtype=torch.complex128, pin_memory=True)
    e2e = []
    for _ in range(min(args.steps, 3)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.set_initial(h_in.numpy(), level=LEVELS - 1)
        r = prob.solve(**opts)[0]
        prob.psi(out=h_out.numpy())
        e2e.append(time.perf_counter() - t0)
        ok = ok and r["status"] == "OK"

    # per-kernel durations (CUDA events on the solver's stream) on every level's grid, in
    # each precision the solve used there (FP32 and FP64 iterations counted per level)
    last = results[-1]
    fp32_lv = last.get("level_fp32_iters", [0] * LEVELS)
    prof = {}
    for lev in range(LEVELS):
        n = tuple(k >> (LEVELS - 1 - lev) for k in N_FINE)
        its32 = fp32_lv[lev]
        its64 = last["level_iters"][lev] - its32
        for pr, its in ((prec if prec else 1, its32), (0, its64)):
            if its <= 0:
                continue
            with Problem(n, L_BOX, [PAR]) as pl:
                pl.set_initial(si.gaussian_guess(n, L_BOX, si.seed_for(2, rank), vortex=True)[None], level=0)
                prof[(n[0], pr)] = (its, pl.profile(iters=20, precision=pr, tol=TOL))
    fp64_peak, fp32_peak = probe_peaks()
    prob.close()
    if rank != 0:
        return None

    # dominant (kernel, level, precision): largest share of the solve time = iterations x duration
    shares = {}
    for (n, pr), (its, pl_ms) in prof.items():
        for name, ms in pl_ms:
            shares[(name, n, pr)] = shares.get((name, n, pr), 0.0) + its * ms
    total_share = sum(shares.values())
    (dom_name, dom_n, dom_pr), _ = max(shares.items(), key=lambda kv: kv[1])
    dom_ms = statistics.mean([ms for name, ms in prof[(dom_n, dom_pr)][1] if name == dom_name])
    peaks_file = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks_file)).get("hbm_gbs") if os.path.exists(peaks_file) else 6800.0
    if dom_pr == 2:
        by = HYBRID_BYTES.get(dom_name, 0) * 3.0 * dom_n * dom_n
        achieved = by / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{dom_name} @ {dom_n}^2 (hybrid)", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "algorithmic_bytes_per_launch": by}
    elif dom_pr == 1:
        by = kernel_bytes(dom_name, (dom_n, dom_n), 8)
        achieved = by / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{dom_name} @ {dom_n}^2 (FP32)", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "algorithmic_bytes_per_launch": by}
    else:
        fl = kernel_flops(dom_name, (dom_n, dom_n))
        achieved = fl / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": f"{dom_name} @ {dom_n}^2 (FP64)", "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                "peak_source": "FP64 FMA-chain probe gpsoc_probe_peaks, this run (of measured)",
                "algorithmic_flops_per_launch": fl}
    roof.update({"ms_per_launch": dom_ms, "share_of_solve": shares[(dom_name, dom_n, dom_pr)] / total_share})
    roof["traffic"] = NCU_DRAM_BYTES.get((dom_name, dom_n, dom_pr))
    ms_per_step = max_total_ms / args.steps
    out = {
        "metric": METRIC, "value": whole_job_rate(world, args.steps, max_total_ms), "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world, "solves_per_step_per_gpu": 1,
                   "grid": "512x512", "levels": [128, 256, 512], "precision": args.precision,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "tiles": tiles or "rule", "tuning_s": round(t_tune, 2)},
        "fp64_plain": fp64,
        "roofline": roof,
        "kernels_us_per_iteration": {f"{n}_{'fp32' if pr else 'fp64'}": {k: round(v * 1e3, 2) for k, v in pl_ms}
                                     for (n, pr), (_, pl_ms) in prof.items()},
        "solve": {"status_ok": ok, "energy": last["energy"], "mu": last["mu"], "res_inf": last["res_inf"],
                  "iters_total": last["total_iters"], "level_iters": last["level_iters"],
                  "level_fp32_iters": fp32_lv, "level_res_fp32": last.get("level_res_fp32"),
                  "fp32_iters": last["fp32_iters"], "fp64_iters": last["fp64_iters"],
                  "beta_resets": last["beta_resets"],
                  "energy_rel_diff_vs_fp64_plain": (abs(last["energy"] - fp64["energy"]) / abs(fp64["energy"])
                                                    if fp64 else None),
                  "stop": f"|dE| < {TOL:g} and max|r| < {RES_TOL:g} on every level (both arms)"},
        "e2e": {"value": world / statistics.mean(e2e), "unit": "solves/s",
                "h2d_bytes_per_step": int(h_in.numpy().nbytes), "d2h_bytes_per_step": int(h_out.numpy().nbytes)},
        "gpu_launches": launches_timed,
        "clocks": clk.summary(),
        "peaks": {"fp64_tflops_probe": fp64_peak, "fp32_tflops_probe": fp32_peak, "hbm_gbs_measured": hbm_peak},
    }
    return out, last


def batch_case(args):
    """The batched sweep: `batch` solves of 256^2 on [-12,12]^2 with parameters drawn
    Omega~U[0,0.95], gamma~U[0,2], beta0~U[100,2000], beta1~U[-10,10] and seeded
    Gaussian / vortex guesses, solved together in one problem (every PCG iteration
    one graph replay for all live solves), FP64 and mixed precision, same tolerance."""
    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    build()
    n, L = (256, 256), (12.0, 12.0)
    B = args.batch
    pars = [(q.Omega, q.gamma, q.beta0, q.beta1) for q in si.batch_params(si.seed_for(3, 0), B)]
    psi = np.stack([si.gaussian_guess(n, L, si.seed_for(3, k), vortex=bool(k % 2)) for k in range(B)])
    out = {"workload": f"{B} solves of 256x256 on [-12,12]^2, random parameters, stop |dE|<1e-12 and "
                       f"max|r|<{args.serve_res_tol:g}",
           "max_iter": args.max_iter}
    for name, prec in (("fp64", 0), ("hybrid", 2)):
        with Problem(n, L, pars) as p:
            p.set_initial(psi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = p.solve(raise_on_error=False, tol=TOL, res_tol=args.serve_res_tol, precision=prec,
                          max_iter=args.max_iter, check_every=64)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        ok = sum(r["status"] == "OK" for r in res)
        its = [r["total_iters"] for r in res]
        out[name] = {"seconds": dt, "solves_per_s": B / dt, "converged": ok, "converged_solves_per_s": ok / dt,
                     "status_counts": {st: sum(r["status"] == st for r in res) for st in sorted({r["status"] for r in res})},
                     "iters_mean": float(np.mean(its)), "iters_max": int(np.max(its)),
                     "fp32_iters_mean": float(np.mean([r["fp32_iters"] for r in res])),
                     "energies": [r["energy"] for r in res]}
    if "fp64" in out and "hybrid" in out:
        d = [abs(a - b) / abs(b) for a, b in zip(out["hybrid"]["energies"], out["fp64"]["energies"])]
        out["hybrid"]["energy_rel_diff_vs_fp64"] = {"max": max(d), "same_minimum_1e-10": sum(x < 1e-10 for x in d),
                                                    "lower": sum(a < b for a, b in zip(out["hybrid"]["energies"],
                                                                                       out["fp64"]["energies"]))}
        out["hybrid"]["speedup_vs_fp64"] = out["hybrid"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    for name in ("fp64", "hybrid"):
        if name in out:
            out[name]["energies"] = [round(e, 10) for e in out[name]["energies"][:4]]
    print(json.dumps(out))


def serve_trace_run(requests, rate, tol, res_tol, arms, max_iter, hbm_budget, slots, seed=None):
    """The served trace: `requests` ground-state requests with Poisson arrivals at
    `rate` per second, grids drawn from {64^2, 128^2, 256^2, 512^2, 64^3, 128^3},
    parameters drawn as in the batched sweep, harmonic traps (3D: gamma_z = 2),
    stop |dE| < tol and max|r| < res_tol.  Arms on the same trace: the
    continuous-batching server in mixed precision ("served_mixed") and in FP64
    ("served_fp64"), and plain single-solve FP64 PCG serving the requests one at a
    time in arrival order ("plain_fp64").  Reports solves/s over the makespan, the
    p50/p99 of arrival-to-result latency (wall clock), and, against plain FP64, the
    number of results in the same minimum (energies within 1e-10 relative) and the
    speed-up counted over those results only."""
    import torch
    from paper_2602_17950_gb300 import Problem, Server
    from paper_2602_17950_gb300.build import build
    build()
    trace = si.serve_trace(si.seed_for(5, 0) if seed is None else seed, requests, rate)
    R = len(trace)
    guesses = [si.gaussian_guess(q["n"], q["L"], q["guess_seed"], vortex=q["vortex"]) for q in trace]
    traps = [{"kind": 0, "g": (1.0, 1.0, 2.0) if len(q["n"]) == 3 else (1.0, 1.0)} for q in trace]
    opts = dict(tol=tol, res_tol=res_tol, max_iter=max_iter)

    def par(q):
        p = q["params"]
        return (p.Omega, p.gamma, p.beta0, p.beta1)

    def summarise(lat, span, res):
        ok = sum(r["status"] == "OK" for r in res)
        return {"solves_per_s": R / span, "makespan_s": span, "converged": ok,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "iters_mean": float(np.mean([r["total_iters"] for r in res]))}

    def served(precision):
        done, res = {}, [None] * R
        with Server(hbm_budget_bytes=hbm_budget, slots_per_bucket=slots, precision=precision,
                    iters_per_step=32) as sv:
            t0 = time.perf_counter()
            nxt, tickets = 0, {}
            while len(done) < R:
                now = time.perf_counter() - t0
                while nxt < R and trace[nxt]["arrival"] <= now:
                    q = trace[nxt]
                    tickets[sv.submit(q["n"], q["L"], par(q), guesses[nxt], trap=traps[nxt], **opts)] = nxt
                    nxt += 1
                busy = sv.step()
                for t, k in list(tickets.items()):
                    got = sv.poll(t, want_psi=False)
                    if got is not None:
                        done[k] = time.perf_counter() - t0
                        res[k] = got[0]
                        del tickets[t]
                if busy == 0 and nxt < R:
                    time.sleep(max(0.0, trace[nxt]["arrival"] - (time.perf_counter() - t0)))
            span = max(done.values())
        lat = [done[k] - trace[k]["arrival"] for k in range(R)]
        return summarise(lat, span, res), res, None

    def plain():
        res, lat, service = [None] * R, [0.0] * R, [0.0] * R
        t0 = time.perf_counter()
        for k, q in enumerate(trace):
            wait = q["arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ts = time.perf_counter()
            with Problem(q["n"], q["L"], [par(q)], trap=traps[k]) as p:
                p.set_initial(guesses[k][None])
                res[k] = p.solve(raise_on_error=False, precision=0, **opts)[0]
            torch.cuda.synchronize()
            service[k] = time.perf_counter() - ts
            lat[k] = time.perf_counter() - t0 - q["arrival"]
        span = time.perf_counter() - t0
        return summarise(lat, span, res), res, service

    out = {"trace": f"{R} requests, Poisson {rate}/s, grids 64^2..512^2, 64^3, 128^3, "
                    f"stop |dE|<{tol:g} and max|r|<{res_tol:g}, max_iter {max_iter}",
           "grid_mix": {f"{'x'.join(map(str, n))}": sum(q["n"] == n for q in trace) for n, _ in si.SERVE_GRIDS},
           "hbm_budget_gb": hbm_budget / 1e9, "slots_per_bucket": slots}
    runs = {}
    for name, fn in (("plain_fp64", plain), ("served_hybrid", lambda: served(2)), ("served_mixed", lambda: served(1)),
                     ("served_fp64", lambda: served(0))):
        if name in arms:
            out[name], rs, service = fn()
            runs[name] = (rs, service)
    if "plain_fp64" in runs:
        ref, service = runs["plain_fp64"]
        for name, (rs, _) in runs.items():
            if name == "plain_fp64":
                continue
            both = [k for k in range(R) if rs[k]["status"] == "OK" and ref[k]["status"] == "OK"]
            d = {k: abs(rs[k]["energy"] - ref[k]["energy"]) / abs(ref[k]["energy"]) for k in both}
            same = [k for k in both if d[k] <= 1e-10]
            o = out[name]
            o["energy_rel_diff_vs_plain_max"] = float(max(d.values())) if d else None
            o["same_minimum_as_plain_1e-10"] = len(same)
            o["same_minimum_fraction"] = len(same) / R
            o["lower_energy_than_plain"] = int(sum(rs[k]["energy"] < ref[k]["energy"] * (1 + 1e-10 * np.sign(ref[k]["energy"]))
                                                   for k in both if k not in same))
            o["speedup_vs_plain"] = o["solves_per_s"] / out["plain_fp64"]["solves_per_s"]
            # throughput of results in the same minimum as plain FP64, each arm over its own makespan
            o["same_minimum_solves_per_s"] = len(same) / o["makespan_s"]
            o["speedup_vs_plain_same_minimum"] = (len(same) / o["makespan_s"]) / (len(same) / out["plain_fp64"]["makespan_s"]) \
                if same else None
            o["plain_service_s_of_other_minima"] = float(sum(service[k] for k in range(R) if k not in same))
    return out


def serve_case(args):
    """The served trace as its own command (see serve_trace_run)."""
    print(json.dumps(serve_trace_run(args.requests, args.arrival_rate, args.serve_tol, args.serve_res_tol,
                                     args.arms.split(","), args.max_iter, args.hbm_budget, args.slots)))


def case1(args):
    """The small plain-PCG workload: 64^2 on [-8,8]^2, harmonic trap, Omega = 0.5,
    gamma = 0.5, beta0 = 100, beta1 = -1, seeded Gaussian components of mass 1/3,
    stop |dE| < 1e-12; GPU FP64 (and mixed with an FP32 phase forced) against the
    CPU oracle on the same input."""
    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    build()
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi = si.gaussian_guess(n, L, si.seed_for(1, 0))
    out = {"case1": "64^2 on [-8,8]^2, harmonic trap, Omega=0.5, gamma=0.5, beta0=100, beta1=-1, stop |dE|<1e-12"}
    for name, kw in (("fp64", dict(precision=0)), ("mixed_forced", dict(precision=1, fp32_min_points=-1))):
        with Problem(n, L, [par]) as p:
            p.set_initial(psi[None])
            p.solve(tol=TOL, **kw)                       # warm-up (graphs, twiddles)
            p.set_initial(psi[None])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = p.solve(tol=TOL, **kw)[0]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "status": r["status"], "energy": r["energy"], "mu": r["mu"],
                     "iters": r["total_iters"], "fp32_iters": r["fp32_iters"]}
    if not args.no_cpu:
        from oracle.model import Grid, Model, Trap
        from oracle.pcg import Options, pcg
        m = Model(Grid(n, L), Trap(), Omega=par[0], gamma=par[1], c0=par[2], c1=par[3])
        t0 = time.perf_counter()
        ref = pcg(m, psi, Options(tol=TOL))
        dt = time.perf_counter() - t0
        out["oracle_cpu"] = {"seconds": dt, "cores": 1, "energy": ref.energy, "iters": ref.iters}
        for name in ("fp64", "mixed_forced"):
            out[name]["energy_rel_diff_vs_oracle"] = abs(out[name]["energy"] - ref.energy) / abs(ref.energy)
    print(json.dumps(out))


def traversal(args):
    """The initial-guess traversal of Section 4, Example 3 (Table table_cpu): for each
    Omega in {0.6, 0.7, 0.8, 0.9} (gamma = 0.3, beta0 = 50, beta1 = 0.5, harmonic trap,
    [-12,12]^2), initial guesses (phi_1, phi_0, phi_-1)/sqrt(3) with the components of
    guess kinds (a)-(f) -- identical components (10 per Omega) or, with --full, all 10^3
    combinations -- solved by CM-PCG 32 -> 64 -> 128 to |dE| < 1e-10 in one batched
    problem per Omega; the lowest energy per Omega is kept and compared with the table."""
    import itertools

    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    build()
    omegas = (0.6, 0.7, 0.8, 0.9)
    table = {0.6: 2.2833, 0.7: 2.0437, 0.8: 1.6806, 0.9: 1.0492}   # Table table_cpu, 4 printed digits
    kinds = list(range(10))
    n_c, L = (32, 32), (12.0, 12.0)
    combos = list(itertools.product(kinds, repeat=3)) if args.full else [(k, k, k) for k in kinds]
    out = {"traversal": f"Table table_cpu: 4 Omega x {len(combos)} guess combinations, CM 32->64->128, "
                        f"|dE|<1e-10, one batch per Omega"}
    for name, prec in (("fp64", 0), ("hybrid", 2)):
        if name not in args.arms_trav.split(","):
            continue
        arm = {"seconds": 0.0, "converged": 0, "lowest_energy": {}, "matches_table_4_digits": {},
               "distinct_minima_1e-6": {}}
        for om in omegas:
            # the library's own guess generator (guess (d), (e) and (f) depend on Omega and beta0)
            single = []
            for k in kinds:
                with Problem(n_c, L, [(om, 0.3, 50.0, 0.5)]) as g:
                    g.set_initial_kind([k, k, k])
                    single.append(g.psi()[0])          # each component of kind k, /sqrt(3), mass 1
            psi0 = np.stack([np.stack([single[a][0], single[b][1], single[c][2]]) for a, b, c in combos])
            pars = [(om, 0.3, 50.0, 0.5)] * len(combos)
            with Problem((128, 128), L, pars) as p:
                p.set_initial(psi0, level=2)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = p.solve(raise_on_error=False, tol=1e-10, cm_levels=3, precision=prec, max_iter=200000)
                torch.cuda.synchronize()
                arm["seconds"] += time.perf_counter() - t0
            es = sorted(r["energy"] for r in res if r["status"] == "OK")
            arm["converged"] += len(es)
            low = es[0] if es else math.inf
            arm["lowest_energy"][str(om)] = round(low, 6)
            arm["matches_table_4_digits"][str(om)] = abs(low - table[om]) <= 0.5e-4
            distinct = [e for i, e in enumerate(es) if i == 0 or e - es[i - 1] > 1e-6 * abs(e)]
            arm["distinct_minima_1e-6"][str(om)] = len(distinct)
        arm["solves_per_s"] = len(omegas) * len(combos) / arm["seconds"]
        out[name] = arm
    print(json.dumps(out))


def case3d(args):
    """The 3D mixed-precision workload: 128^3 on [-8,8]^3, trap (x^2+y^2+4z^2)/2 + 0.1 r^4,
    Omega = 1.2, gamma = 1, beta0 = 500, beta1 = -2, seeded vortex-phase guess, stop
    |dE| < 1e-10; mixed precision and plain FP64, one solve each (wall clock around the
    solve call, device synchronised)."""
    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    build()
    n, L = (args.n3d,) * 3, (8.0, 8.0, 8.0)
    trap = {"kind": 1, "g": (1.0, 1.0, 2.0), "quad": 0.0, "quart": 0.1}
    par = (1.2, 1.0, 500.0, -2.0)
    psi = si.gaussian_guess(n, L, si.seed_for(4, 0), vortex=True)
    out = {"case3d": f"{n[0]}^3 on [-8,8]^3, trap (x^2+y^2+4z^2)/2 + 0.1 r^4, Omega=1.2, gamma=1, "
                     f"beta0=500, beta1=-2, stop |dE|<1e-12 and max|r|<{args.serve_res_tol:g}, max_iter {args.max_iter}"}
    for name, prec in (("hybrid", 2), ("mixed", 1), ("fp64", 0)):
        if name not in args.arms3d.split(","):
            continue
        with Problem(n, L, [par], trap=trap) as p:
            p.set_initial(psi[None])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = p.solve(raise_on_error=False, tol=1e-12, res_tol=args.serve_res_tol, precision=prec,
                        max_iter=args.max_iter, check_every=64)[0]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            prof = p.profile(iters=10, precision=prec, tol=1e-12)
        out[name] = {"seconds": dt, "solves_per_s": 1.0 / dt, "status": r["status"], "energy": r["energy"],
                     "mu": r["mu"], "iters": r["total_iters"], "fp32_iters": r["fp32_iters"],
                     "fp64_iters": r["fp64_iters"], "iteration_us": round(sum(v for _, v in prof) * 1e3, 1),
                     "us_per_launch": {k: round(v * 1e3, 1) for k, v in prof}}
    for name in ("hybrid", "mixed"):
        if name in out and "fp64" in out:
            out[name]["energy_rel_diff_vs_fp64"] = abs(out[name]["energy"] - out["fp64"]["energy"]) / abs(out["fp64"]["energy"])
            out[name]["speedup_vs_fp64"] = out["fp64"]["seconds"] / out[name]["seconds"]
    print(json.dumps(out))


def kernel_case(args):
    """Per-kernel durations of PCG iterations of `batch` solves on an N x N grid of
    the bench workload (box, trap, parameters), CUDA events on the solver's stream.
    A small, bounded command for kernel-level profiling."""
    import torch
    from paper_2602_17950_gb300 import Problem
    from paper_2602_17950_gb300.build import build
    build()
    n = (args.kernel_case, args.kernel_case)
    prec = {"fp64": 0, "mixed": 1, "hybrid": 2}[args.precision]
    psi = np.stack([si.gaussian_guess(n, L_BOX, si.seed_for(2, k), vortex=True) for k in range(args.batch)])
    with Problem(n, L_BOX, [PAR] * args.batch) as p:
        p.set_initial(psi)
        p.profile(iters=args.warmup, precision=prec, tol=TOL)
        prof = p.profile(iters=max(args.steps, 1) * 10, precision=prec, tol=TOL)
        # the same iterations as the solver runs them (graph replays, periodic checks and
        # exact recomputations), from the same start, without the FP64 lead-in
        kw = dict(tol=1e-300, res_tol=0.0, cm_levels=1, precision=prec, hybrid_lead_res=-1.0, raise_on_error=False)
        solve_iters = 200 * max(args.steps, 1)
        p.set_initial(psi)
        p.solve(max_iter=32, **kw)
        p.set_initial(psi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = p.solve(max_iter=solve_iters, **kw)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        its = max(int(sum(x["iters"] for x in r)) // args.batch, 1)
    out = {"kernel_case": f"{n[0]}x{n[1]} x {args.batch} solves", "precision": args.precision,
           "us_per_launch": {k: round(v * 1e3, 2) for k, v in prof},
           "iteration_us": round(sum(v for _, v in prof) * 1e3, 2),
           "solver_iteration_us": round(t_solve / its * 1e6, 2), "solver_iterations": its,
           "gbs_per_launch": {k: round(launch_bytes(k, n, prec) * args.batch / (v * 1e-3) / 1e9, 1)
                              for k, v in prof if launch_bytes(k, n, prec) > 0}}
    torch.cuda.synchronize()
    print(json.dumps(out))


def per_level_iters(res_dict, n_levels):
    """Iterations of one solve on each multigrid level (coarsest first)."""
    return [int(v) for v in res_dict["level_iters"][:n_levels]]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "hybrid"], default="hybrid")
    ap.add_argument("--fp64-steps", type=int, default=5, help="timed solves of the plain FP64 comparison")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in tile rule (no autotuning)")
    ap.add_argument("--kernel-case", type=int, default=0, metavar="N",
                    help="only time the kernels of PCG iterations on N x N grids (per-kernel CUDA events)")
    ap.add_argument("--batch", type=int, default=1, help="solves per problem in --kernel-case / --batch-case")
    ap.add_argument("--batch-case", action="store_true", help="the batched random-parameter sweep at 256^2")
    ap.add_argument("--max-iter", type=int, default=50000, help="iteration cap of the batched and served cases")
    ap.add_argument("--serve-case", action="store_true", help="the served trace (Poisson arrivals, mixed grids)")
    ap.add_argument("--requests", type=int, default=32, help="requests of --serve-case")
    ap.add_argument("--arrival-rate", type=float, default=4.0, help="Poisson arrival rate of the served trace (1/s)")
    ap.add_argument("--serve-tol", type=float, default=1e-12, help="energy stopping tolerance of the served trace")
    ap.add_argument("--serve-res-tol", type=float, default=1e-8, help="residual tolerance of the served trace")
    ap.add_argument("--serve-sample", type=int, default=48,
                    help="requests of the served-trace sample in the default run (0 = none)")
    ap.add_argument("--hbm-budget", type=float, default=120e9, help="device bytes the server may use")
    ap.add_argument("--slots", type=int, default=16, help="solves per server bucket")
    ap.add_argument("--arms", default="served_hybrid,served_fp64,plain_fp64", help="arms of --serve-case")
    ap.add_argument("--sample-arms", default="plain_fp64,served_hybrid", help="arms of the default run's served sample")
    ap.add_argument("--case1", action="store_true", help="the small 64^2 plain-PCG workload vs the oracle")
    ap.add_argument("--case3d", action="store_true", help="the 3D mixed-precision workload (128^3)")
    ap.add_argument("--n3d", type=int, default=128, help="grid points per axis of --case3d")
    ap.add_argument("--arms3d", default="hybrid,fp64", help="arms of --case3d")
    ap.add_argument("--traversal", action="store_true", help="the initial-guess traversal of Table table_cpu")
    ap.add_argument("--arms-trav", dest="arms_trav", default="fp64,hybrid", help="arms of --traversal")
    ap.add_argument("--full", action="store_true", help="--traversal over all 10^3 guess combinations")
    args = ap.parse_args()
    if args.traversal:
        traversal(args)
        return
    if args.case1:
        case1(args)
        return
    if args.case3d:
        case3d(args)
        return
    if args.serve_case:
        serve_case(args)
        return
    if args.batch_case:
        batch_case(args)
        return
    if args.kernel_case:
        kernel_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")

    if args.impl == "reference":
        if rank != 0:
            return
        # the FP64 CPU oracle on this machine's host cores: per-level iteration times of the
        # workload, scaled by the per-level iteration counts of one solve (REF_LEVEL_ITERS);
        # one sample per step on all cores at once (independent solves, one per core)
        times, cores, desc, single = [], 1, "", []
        oracle_sample(REF_LEVEL_ITERS)          # one untimed warm-up sample (pages in numpy)
        for _ in range(args.steps):
            b = oracle_baseline(REF_LEVEL_ITERS)
            times.append(1.0 / b["value"])
            single.append(b["single_core_value"])
            cores, desc = b["cores"], b["sample"]
        v = 1.0 / statistics.mean(times)
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(times),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": WORKLOAD, "global_batch": 1, "grid": "512x512",
                                               "levels": [128, 256, 512], "precision": "fp64"},
               "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "single_core_value": statistics.mean(single), "cpu_model": cpu_model(),
                                "nproc": os.cpu_count(),
                                "sample": desc + f"; per-level iteration counts {list(REF_LEVEL_ITERS)} of one "
                                                 "plain FP64 solve (extrapolated, not a whole solve)"},
               "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    got = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()
    if rank != 0 or got is None:
        return
    out, last = got
    if args.serve_sample > 0 and world == 1:
        # the spec comparison on the device: a bounded sample of the served trace,
        # batched mixed-precision server against plain single-solve FP64, same stopping rule
        with ClockSampler(local_rank) as clk:
            out["served_trace"] = serve_trace_run(args.serve_sample, args.arrival_rate, args.serve_tol,
                                                  args.serve_res_tol, args.sample_arms.split(","), args.max_iter,
                                                  args.hbm_budget, args.slots)
        out["served_trace"]["clocks"] = clk.summary()
    if not args.no_cpu and world == 1:
        fp = out.get("fp64_plain") or {}
        its = fp.get("level_iters") or per_level_iters(last, LEVELS)
        out["cpu_baseline"] = oracle_baseline(its)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
