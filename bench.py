#!/usr/bin/env python3
"""Benchmark: LML + gradient evaluations per second of the sparse-kernel exact GP (gp2Scale hot path)
on GB300, through the C ABI of libgp2s.so.

Default workload (one step = one full gp2s_lml_grad call: Morton sort + cell list + count/scan/fill
assembly of the CSR, FP32 multi-RHS CG with FP64 refinement of a = A^{-1} y, SLQ log-determinant with
64 Rademacher probes x 100 Lanczos steps, and the 42-parameter adjoint gradient):
  clusters_3d: N = 1,000,000 points in 50 clipped Gaussian clusters in [0,1]^3, L = 8 bumps,
               r tuned for ~100 stored entries per row, sigma^2 = 4e-4 (synthetic, seed 0).

JSON line (rank 0): metric/value/unit, ms_per_step, roofline of the dominant kernel (the SpMM of the
Krylov solves, HBM-bound), cpu_baseline (the FP64 oracle on a bounded sample on the host cores),
e2e (host buffers, copies inside the timed region), clocks, gpu_launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload clusters_3d|sphere_4d|small_2d]
  python bench.py --impl reference    # the FP64 CPU oracle on the same metric (bounded sample)
Multi-GPU (torchrun): each rank evaluates its own independent problem (replicas); value = total
evaluations of all ranks / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LML+grad evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

THROTTLE_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
                 0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(workload: str, n: int):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of k_spmm_rb from the
    committed ncu summary of this workload, if there is one: (bytes, file) or (None, None)."""
    path = os.path.join(ROOT, "profiles", f"k_spmm_rb_{workload}_n{n // 1_000_000}m.md")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("| traffic per launch (read + write) |"):
                    v = line.split("|")[2].strip().split()
                    return float(v[0]) * {"GB": 1e9, "MB": 1e6}[v[1]], os.path.relpath(path, ROOT)
    except OSError:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--id={self.index}", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 3:
                    try:
                        self.samples.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                    except ValueError:
                        pass

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [s[0] for s in self.samples]
        mask = 0
        for s in self.samples:
            mask |= s[2]
        reasons = [name for bit, name in THROTTLE_BITS.items() if mask & bit and name != "gpu_idle"]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": reasons, "samples": len(self.samples)}


def make_workload(name: str, seed: int, n: int | None = None):
    """The named workload at its full size, or at n points with the same generator and the same
    mean entries per row (a small case of the same kernels, for profiling captures)."""
    from paper_2512_06143_gb300 import workloads as W
    kw = {} if n is None else {"n": n}
    if name == "clusters_3d":
        return W.clusters_3d(seed, **kw), dict(probes=64, lanczos_steps=100)
    if name == "sphere_4d":
        return W.sphere_4d(seed, **kw), dict(probes=32, lanczos_steps=100)
    if name == "small_2d":
        return W.small_2d(seed, **kw), dict(probes=64, lanczos_steps=100)
    raise ValueError(name)


FP32_INSTR_PEAK = 152 * 128 * 2.07e9   # FP32 lanes x SMs x maximum SM clock (instructions/s)
# GB300's nominal FP64 rate (1.25 TFLOP/s), in FP64 instructions per second (a fused multiply-add
# is two flops and one instruction)
FP64_INSTR_PEAK = 1.25e12 / 2


def assembly_roofline(n: int, d: int, L: int, nnz: int, ms: float, hbm_gbs: float, mixed: bool = True) -> dict:
    """Whole assembly (sort, cell list, count, scan, fill, FP64 values) against its algorithmic
    roofline, the slowest of three legs over the (nnz + n) / 2 unique pairs:
      memory: the CSR written once, int32 columns + FP64 values (+ FP32 values in mixed
              precision) per stored entry + 4 B per row pointer;
      FP32:   one support test per unique pair, 2d instructions, at 152 SMs x 128 lanes x 2.07 GHz;
      FP64:   one value per unique pair, 2d (differences, squares) + 1 (square root) + 7 (taper
              polynomial) + L (bump products) + 3 (w0, the Jacobi scales) instructions, at the
              nominal FP64 rate.  The values must be FP64: the refinement residual is formed with
              them, against the FP64 matrix to 1e-8."""
    mem = (16.0 if mixed else 12.0) * nnz + 4.0 * (n + 1)
    pairs = 0.5 * (nnz + n)
    instr32 = pairs * 2 * d
    instr64 = pairs * (2 * d + 1 + 7 + L + 3)
    t_mem, t_32, t_64 = mem / (hbm_gbs * 1e9), instr32 / FP32_INSTR_PEAK, instr64 / FP64_INSTR_PEAK
    legs = {"hbm": t_mem, "alu_fp32": t_32, "alu_fp64": t_64}
    bound = max(legs, key=legs.get)
    roof_ms = 1000.0 * legs[bound]
    return {"ms": ms, "gnnz_per_s": nnz / (ms * 1e6) if ms > 0 else None,
            "roofline": {"bound": bound, "roof_ms": roof_ms, "frac": roof_ms / ms if ms > 0 else None,
                         "legs_ms": {k: 1000.0 * v for k, v in legs.items()}, "bytes": mem,
                         "fp32_instr": instr32, "fp64_instr": instr64,
                         "alu_peak_instr_per_s": FP32_INSTR_PEAK, "fp64_peak_instr_per_s": FP64_INSTR_PEAK,
                         "fp64_peak_source": "nominal GB300 FP64 rate, 1.25 TFLOP/s"}}


def replica_throughput(ws: int, steps: int, total_ms: float, e2e_ms: float, device: str):
    """Whole-job throughput of ws independent replicas: every rank evaluated `steps` problems; the
    job's time is the slowest rank's (MAX all-reduce of the device-timed and end-to-end totals).
    Returns (evals/s, e2e evals/s, max total ms, max e2e ms)."""
    if ws > 1:
        import torch
        t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms, e2e_ms = float(t[0]), float(t[1])
    return ws * steps / (total_ms / 1000.0), ws * steps / (e2e_ms / 1000.0), total_ms, e2e_ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample of the workload
# ----------------------------------------------------------------------------------------------
def oracle_sample(workload: str, budget_s: float = 20.0):
    """Time the oracle's full LML + gradient pipeline on a scaled-down instance of the same
    generator (same density per row, same probes and Lanczos steps) and scale by N to the full
    workload: evaluations/s at full N ~= (N_sample / N_full) / t_sample (the work is linear in N at
    a fixed number of entries per row and iterations)."""
    import oracle
    from paper_2512_06143_gb300 import workloads as W
    oracle.build()
    if workload == "clusters_3d":
        full_n, target, m = 1_000_000, 100.0, 64
        ns = 12000
        gen = lambda n: W.clusters_3d(0, n=n, target_nnz=target)  # noqa: E731
    elif workload == "sphere_4d":
        full_n, target, m = 10_000_000, 60.0, 32
        ns = 150000
        gen = lambda n: W.sphere_4d(0, n=n, target_nnz=target)  # noqa: E731
    else:
        full_n, m = 4096, 64
        ns = 4096
        gen = lambda n: W.small_2d(0)  # noqa: E731
    w = gen(ns)
    h = oracle.Hyper(**w["hyper"])
    t0 = time.perf_counter()
    if workload == "small_2d":
        oracle.lml_exact(w["X"], w["y"], h)
        oracle.grad_exact(w["X"], w["y"], h)
    else:
        oracle.lml_slq(w["X"], w["y"], h, m=m, k=100, seed=0, tol=1e-8)
    t = time.perf_counter() - t0
    evals = (ns / full_n) / t
    asm = "brute-force assembly" if ns <= 20000 else "k-d tree candidates + exact FP64 test"
    sample = (f"oracle LML+grad ({asm}, FP64 CG to 1e-8, SLQ {m}x100, Hutchinson gradient) "
              f"on N={ns} points of the same generator, {t:.2f} s, scaled by N/{full_n}")
    return evals, oracle.num_threads(), sample, t


# ----------------------------------------------------------------------------------------------
def reference_config(workload: str) -> dict:
    """The GPU arm's workload description (same generator, sizes, probes and steps)."""
    full = {"clusters_3d": dict(n=1_000_000, d=3, L=8, probes=64, lanczos_steps=100),
            "sphere_4d": dict(n=10_000_000, d=4, L=8, probes=32, lanczos_steps=100),
            "small_2d": dict(n=4096, d=2, L=4, probes=64, lanczos_steps=100)}.get(workload, {})
    return {"workload": workload, **full, "precision": "fp64 oracle", "parallelism": "host cores"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    workload = args.workload
    vals = []
    cores = None
    sample = ""
    for _ in range(args.warmup):
        oracle_sample(workload)
    for _ in range(args.steps):
        v, cores, sample, _ = oracle_sample(workload)
        vals.append(v)
    value = float(statistics.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value if value > 0 else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": reference_config(workload),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "extrapolated": workload != "small_2d"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": ("value and ms_per_step are extrapolated from the timed sample by N (the oracle never runs "
                     "the full workload here), so ms_per_step exceeds the run's own wall time"
                     if workload != "small_2d" else "the full workload, timed")}
    print(json.dumps(line), flush=True)
    return 0


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
SAMPLE_CASES = {"clusters_3d": ("clusters_3d_150k_t0", 100.0), "sphere_4d": ("sphere_4d_150k", 60.0)}
# the oracle's run over a whole workload, stored where it could be afforded (5.2 hours on 8 cores)
FULL_CASES = {("sphere_4d", 10_000_000): "sphere_4d_10m"}


def timed_evals(ctx, X, y, hyper, opts, steps, warmup, flush, stream, barrier):
    """warmup untimed evaluations, then `steps` evaluations bracketed by CUDA events on the
    launching stream (L2 flushed before each).  Returns (per-step ms, infos)."""
    for _ in range(warmup):
        ctx.lml_grad(X, y, hyper, opts)
    import torch
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    for k in range(steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        _, _, info = ctx.lml_grad(X, y, hyper, opts)
        ev[k][1].record(stream)
        infos.append(info)
    barrier()
    return [a.elapsed_time(b) for a, b in ev], infos


def e2e_evals(ctx, Xh, yh, hyper, opts, steps, flush):
    """The same evaluation from pinned HOST buffers: the call copies X and y to the device and
    returns the LML and gradient to the host; wall clock around each call."""
    import torch
    out = []
    for k in range(steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.lml_grad(Xh, yh, hyper, opts)
        torch.cuda.synchronize()
        out.append(1000.0 * (time.perf_counter() - t0))
    return out


def spmm_roofline(gp, ctx, X, y, hyper, wopts, precision, flush, workload, n, peak, peak_src):
    """One extra evaluation with opts.profile = 1 after the timed region: CUDA events around every
    multi-RHS SpMM launch on the context's stream (graphs off for this pass only).  Gives the
    dominant kernel's per-launch time, its algorithmic bytes and its share of the evaluation."""
    flush.fill_(7)
    _, _, info = ctx.lml_grad(X, y, hyper, gp.default_opts(precision=precision, profile=1, **wopts))
    launches = max(int(info["spmm_launches"]), 1)
    ms = info["ms_spmm"] / launches
    nbytes = info["spmm_bytes"] / launches
    achieved = nbytes / (ms / 1000.0) / 1e9 if ms > 0 else None
    traffic, traffic_src = profile_traffic(workload, int(n))
    return {"kernel": "k_spmm_rb (multi-RHS RB8 SpMM of the Krylov solves)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "traffic_source": traffic_src, "peak_source": f"{peak_src} hbm_gbs",
            "launches_per_step": int(info["spmm_launches"]), "bytes_per_launch": nbytes, "ms_per_launch": ms,
            "share_of_step": info["ms_spmm"] / info["ms_total"] if info["ms_total"] > 0 else None,
            "timing": "CUDA events around each SpMM launch in one profiled evaluation after the timed region",
            "bytes_definition": "8 B per stored entry (FP32 value + int32 column) + 4 B per row pointer + 4 B per "
                                "input and per output vector element"}


def pattern_cached_evals(gp, ctx, X, y, hyper, wopts, precision, steps, flush, stream) -> dict:
    """The pattern-cached figure: evaluations where theta changes (bump amplitudes and centers, as
    an MCMC block that leaves r alone would) but X and r do not, so the assembly reuses the
    pattern.  One untimed evaluation sets the pattern, then `steps` timed ones."""
    import torch
    opts = gp.default_opts(precision=precision, **wopts)
    th0 = hyper.theta()
    L, d = hyper.L, hyper.d

    def theta(k):
        th = th0.copy()
        th[:L * d] += 0.002 * (k + 1)
        th[L * d + L:L * d + 2 * L] *= 1.0 + 0.01 * (k + 1)
        return hyper.with_theta(th)

    ctx.lml_grad(X, y, theta(-1), opts)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    reused = 0
    for k in range(steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        _, _, info = ctx.lml_grad(X, y, theta(k), opts)
        ev[k][1].record(stream)
        reused += int(info["pattern_reused"])
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"value": steps / (sum(ms) / 1000.0), "unit": "evals/s", "ms_per_step": sum(ms) / steps,
            "steps_with_pattern_reused": reused, "steps": steps, "ms_assemble": info["ms_assemble"],
            "note": "bump centers and amplitudes change every step; X and r fixed"}


def measure_workload(gp, ctx, workload, seed, n, steps, warmup, flush, stream, barrier, peak, peak_src,
                     sampler=None):
    """Device-timed evaluations (production options), the end-to-end form from host buffers, and
    the dominant kernel's roofline, for one workload."""
    import torch
    w, wopts = make_workload(workload, seed=seed, n=n)
    hyper = gp.Hyper(**w["hyper"])
    nn = w["X"].shape[0]
    precision = gp.PREC_MIXED if workload != "small_2d" else gp.PREC_FP64
    # every timed step rebuilds the pattern (the full evaluation); the pattern-cached figure below
    # changes theta every step and lets the assembly reuse the pattern
    opts = gp.default_opts(precision=precision, pattern_cache=1, **wopts)
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
    Xh = torch.tensor(w["X"], dtype=torch.float64).pin_memory()
    yh = torch.tensor(w["y"], dtype=torch.float64).pin_memory()
    for _ in range(warmup):
        ctx.lml_grad(X, y, hyper, opts)
    if sampler is not None:
        sampler.start()
    step_ms, infos = timed_evals(ctx, X, y, hyper, opts, steps, 0, flush, stream, barrier)
    clocks = sampler.stop() if sampler is not None else None
    e2e_ms = e2e_evals(ctx, Xh, yh, hyper, opts, steps, flush)
    roof = spmm_roofline(gp, ctx, X, y, hyper, wopts, precision, flush, workload, nn, peak, peak_src)
    cached = pattern_cached_evals(gp, ctx, X, y, hyper, wopts, precision, steps, flush, stream)
    i0 = infos[-1]
    return dict(w=w, hyper=hyper, opts=opts, wopts=wopts, precision=precision, X=X, y=y, n=int(nn),
                step_ms=step_ms, infos=infos, e2e_ms=e2e_ms, roofline=roof, clocks=clocks, pattern_cached=cached,
                h2d=int(Xh.numel() * 8 + yh.numel() * 8), d2h=int(8 + 8 * hyper.nparams),
                config={"workload": workload, "n": int(nn), "d": int(hyper.d), "L": hyper.L, "nnz": int(i0["nnz"]),
                        "probes": int(opts.probes), "lanczos_steps": int(opts.lanczos_steps),
                        "precision": "mixed" if precision == gp.PREC_MIXED else "fp64",
                        "l2": "flushed (256 MB write) between steps"},
                detail={"ms_assemble": i0["ms_assemble"], "ms_solve": i0["ms_solve"], "ms_logdet": i0["ms_logdet"],
                        "ms_grad": i0["ms_grad"], "iters_y": i0["iters_y"], "iters_probes": i0["iters_probes"],
                        "outer": i0["outer"], "relres": i0["relres"], "lml": i0["lml"],
                        "logdet_stderr": i0["logdet_stderr"], "bj_block": i0["bj_block"],
                        "spmm_seg_tiles": i0["spmm_seg_tiles"], "step_ms": step_ms})


def oracle_errors(gp, ctx, m: dict) -> dict:
    """Part of the oracle leg (after every timed region): each result's error against the FP64
    oracle.  (1) The full-size y solve: |y_i - A_i a| on sampled rows, the rows of A from the
    oracle's brute force over all points, against |y|.  (2) Where the oracle's run over the whole
    workload is stored (the 10M-point 4-D workload), the log-determinant, quadratic term, LML and
    gradient of the bench's own evaluation against it.  (3) The same on a 150,000-point sample of
    the generator.  Stored results live in tests/golden (written by
    tests/golden/make_oracle_large.py, which calls only the oracle); identical probes."""
    import oracle
    from paper_2512_06143_gb300 import workloads as W
    out = {}
    w, hyper = m["w"], m["hyper"]
    ctx.assemble(m["X"], hyper, m["opts"])
    a, sinfo = ctx.solve(m["y"])
    a = a.cpu().numpy()
    rows = np.random.default_rng(3).choice(m["n"], 16, replace=False)
    ynorm = float(np.linalg.norm(w["y"]))
    worst = 0.0
    for r, (oc, ov) in zip(rows, oracle.rows_brute(w["X"], oracle.Hyper(**w["hyper"]), rows)):
        worst = max(worst, abs(w["y"][r] - float(ov @ a[oc])) / ynorm)
    out["y_residual"] = {"relres_fp64": sinfo["relres"], "max_sampled_row_residual_over_ynorm": worst,
                         "rows": len(rows), "bound": 1e-8}
    # the workload itself, where the oracle's run over all of its points is stored
    full = FULL_CASES.get((m["config"]["workload"], int(m["n"])))
    fpath = os.path.join(GOLDEN_DIR, f"oracle_{full}.json") if full else None
    if fpath and os.path.exists(fpath):
        with open(fpath) as f:
            ref = json.load(f)
        if np.allclose(W.checksums(w["X"], w["y"]), ref["checksums"], rtol=1e-10, atol=0.0):
            lml, g, info = ctx.lml_grad(m["X"], m["y"], hyper, m["opts"])
            gref = np.asarray(ref["grad"])
            out["full_size"] = {"case": ref["case"], "n": ref["n"], "nnz": int(info["nnz"]), "oracle_nnz": ref["nnz"],
                                "logdet_rel_err": abs(info["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
                                "quad_rel_err": abs(info["quad"] - ref["quad"]) / abs(ref["quad"]),
                                "lml_abs_err": abs(lml - ref["lml"]),
                                "lml_bar": 0.5e-3 * abs(ref["logdet"]) + 0.5e-7 * abs(ref["quad"]),
                                "grad_max_err_over_max_abs": float(np.abs(g - gref).max() / np.abs(gref).max()),
                                "bars": {"logdet": 1e-3, "quad": 1e-7, "grad": 1e-4},
                                "oracle": f"FP64 CG to {ref['cg_tol']} over all {ref['n']} points, identical probes"}
    case = SAMPLE_CASES.get(m["config"]["workload"])
    if case is None:
        return out
    path = os.path.join(GOLDEN_DIR, f"oracle_{case[0]}.json")
    try:
        with open(path) as f:
            ref = json.load(f)
    except OSError:
        out["sample"] = {"skipped": f"{os.path.relpath(path, ROOT)} missing"}
        return out
    gen = {"clusters_3d": W.clusters_3d, "sphere_4d": W.sphere_4d}[ref["workload"]]
    ws = gen(0, n=ref["n"], target_nnz=ref["target"])
    if not np.allclose(W.checksums(ws["X"], ws["y"]), ref["checksums"], rtol=1e-10, atol=0.0):
        out["sample"] = {"skipped": "this machine's generator gave other inputs than the stored case"}
        return out
    hs = gp.Hyper(**ref["hyper"])
    opts = gp.default_opts(precision=gp.PREC_MIXED, probes=ref["probes"], lanczos_steps=ref["steps"],
                           seed=ref["seed"])
    lml, g, info = ctx.lml_grad(ws["X"], ws["y"], hs, opts)
    gref = np.asarray(ref["grad"])
    out["sample"] = {"case": ref["case"], "n": ref["n"], "nnz": int(info["nnz"]), "oracle_nnz": ref["nnz"],
                     "logdet_rel_err": abs(info["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
                     "quad_rel_err": abs(info["quad"] - ref["quad"]) / abs(ref["quad"]),
                     "lml_abs_err": abs(lml - ref["lml"]),
                     "lml_bar": 0.5e-3 * abs(ref["logdet"]) + 0.5e-7 * abs(ref["quad"]),
                     "grad_max_err_over_max_abs": float(np.abs(g - gref).max() / np.abs(gref).max()),
                     "bj_block": info["bj_block"], "spmm_seg_tiles": info["spmm_seg_tiles"],
                     "bars": {"logdet": 1e-3, "quad": 1e-7, "grad": 1e-4},
                     "probes": "identical Rademacher probes on both sides"}
    return out


def run_gpu(args):
    import torch

    import paper_2512_06143_gb300 as gp
    from paper_2512_06143_gb300 import build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    gp.load()
    stream = torch.cuda.current_stream()
    ctx = gp.Context(local, stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # 256 MB > 129 MB L2
    peak, peak_src = load_peaks()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    main_m = measure_workload(gp, ctx, args.workload, rank, args.n, args.steps, args.warmup, flush, stream, barrier,
                              peak, peak_src, sampler=ClockSampler(local))
    total_ms = sum(main_m["step_ms"])
    e2e_total = sum(main_m["e2e_ms"])
    value, e2e_value, total_ms, e2e_total = replica_throughput(ws, args.steps, total_ms, e2e_total, "cuda")
    infos = main_m["infos"]
    launches = int(sum(i["launches"] for i in infos))
    secondary = {}
    if ws == 1 and args.workload == "clusters_3d" and args.n is None and not args.no_secondary:
        # the metric's second size (N = 10M, d = 4) and the batched form, each measured the same way
        ctx2 = gp.Context(local, stream.cuda_stream)
        m2 = measure_workload(gp, ctx2, "sphere_4d", 0, None, 2, 1, flush, stream, barrier, peak, peak_src,
                              sampler=ClockSampler(local))
        t2 = sum(m2["step_ms"])
        secondary["sphere_4d"] = {
            "metric": METRIC, "value": 2 / (t2 / 1000.0), "unit": "evals/s", "steps": 2, "warmup": 1,
            "ms_per_step": t2 / 2, "config": m2["config"], "roofline": m2["roofline"], "clocks": m2["clocks"],
            "e2e": {"value": 2 / (sum(m2["e2e_ms"]) / 1000.0), "unit": "evals/s", "h2d_bytes_per_step": m2["h2d"],
                    "d2h_bytes_per_step": m2["d2h"]},
            "assembly": assembly_roofline(m2["n"], int(m2["hyper"].d), int(m2["hyper"].L),
                                          int(m2["infos"][-1]["nnz"]), m2["infos"][-1]["ms_assemble"], peak),
            "pattern_cached": m2["pattern_cached"],
            "gpu_launches": int(sum(i["launches"] for i in m2["infos"])), "detail": m2["detail"]}
        secondary["batch"] = batch_record(gp, torch, local, steps=1, warmup=1)
    if rank == 0:
        i0 = infos[-1]
        errors = None
        if not args.no_cpu_baseline:
            cpu_v, cores, sample, _ = oracle_sample(args.workload)
            errors = {args.workload: oracle_errors(gp, ctx, main_m)}
            if "sphere_4d" in secondary:
                m2["config"]["workload"] = "sphere_4d"
                errors["sphere_4d"] = oracle_errors(gp, ctx2, m2)
        else:
            cpu_v, cores, sample = None, None, "skipped"
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if main_m["precision"] == gp.PREC_MIXED else "f64", "data": "synthetic",
            "config": {**main_m["config"], "parallelism": f"replicas x{ws}",
                       "options": "production defaults (CUDA graphs on, no per-launch events)"},
            "roofline": main_m["roofline"],
            "assembly": assembly_roofline(main_m["n"], int(main_m["hyper"].d), int(main_m["hyper"].L),
                                          int(i0["nnz"]), i0["ms_assemble"], peak),
            "cpu_baseline": {"value": cpu_v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "extrapolated": True},
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": main_m["h2d"],
                    "d2h_bytes_per_step": main_m["d2h"]},
            "pattern_cached": main_m["pattern_cached"],
            "clocks": main_m["clocks"], "gpu_launches": launches,
            "errors": errors,
            "secondary": secondary or None,
            "detail": main_m["detail"],
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gp2s", choices=["gp2s", "reference"])
    ap.add_argument("--workload", default="clusters_3d", choices=["clusters_3d", "sphere_4d", "small_2d", "batch"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the N = 10M sphere_4d and batched records of the default run")
    ap.add_argument("--n", type=int, default=None,
                    help="points per problem (default: the workload's full size); smaller n = profiling case")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_gpu(args)


def batch_record(gp, torch, local, steps=1, warmup=1, seed=0) -> dict:
    """256 independent problems (N log-uniform in [2048, 65536], d in {1,2,3}, 10-200 entries per
    row), one gp2s_lml_batched call per step (SLQ, 16 probes x 100 steps, so 17 right-hand sides
    per problem with y): the mixed-precision form
    timed with inputs on the device and from host buffers, and the plain FP64 GPU form timed once
    beside it, with the accuracy of the two against each other."""
    from paper_2512_06143_gb300 import workloads as W
    ws_ = W.batch(seed)
    probs = [(torch.tensor(w["X"], device="cuda"), torch.tensor(w["y"], device="cuda"), gp.Hyper(**w["hyper"]))
             for w in ws_]
    host = [(w["X"], w["y"], gp.Hyper(**w["hyper"])) for w in ws_]
    ctx = gp.Context(local, torch.cuda.current_stream().cuda_stream)
    mixed = gp.default_opts(precision=gp.PREC_MIXED, logdet=gp.LOGDET_SLQ, probes=16, lanczos_steps=100)
    fp64 = gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_SLQ, probes=16, lanczos_steps=100, precond=1)
    for _ in range(warmup):
        ctx.lml_batched(probs, mixed)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lm, infos = ctx.lml_batched(probs, mixed)
    e1.record(stream)
    torch.cuda.synchronize()
    t_mixed = e0.elapsed_time(e1) / 1000.0 / steps
    t0 = time.perf_counter()
    ctx.lml_batched(host, mixed)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    ctx.lml_batched(probs, fp64)
    torch.cuda.synchronize()
    e0.record(stream)
    l64, i64 = ctx.lml_batched(probs, fp64)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fp64 = e0.elapsed_time(e1) / 1000.0
    lm, l64 = np.asarray(lm), np.asarray(l64)
    ld_m = np.array([i["logdet"] for i in infos])
    ld_64 = np.array([i["logdet"] for i in i64])
    q_m = np.array([i["quad"] for i in infos])
    q_64 = np.array([i["quad"] for i in i64])
    se = np.array([i["logdet_stderr"] for i in i64])
    return {"metric": "batched LML evals/s", "value": len(probs) / t_mixed, "unit": "evals/s", "steps": steps,
            "warmup": warmup, "ms_per_step": 1000.0 * t_mixed, "higher_is_better": True,
            "config": {"workload": "batch", "problems": len(probs),
                       "n_total": int(sum(p[0].shape[0] for p in probs)), "probes": 16, "lanczos_steps": 100,
                       "rhs_per_problem": 17},
            "autotuner": {"configs_used": {str(k): int(sum(1 for i in infos if i["batch_config"] == k))
                                           for k in (0, 1, 2, 3)},
                          "configs": ["bj 64, eager", "bj 128, eager", "bj 64, graphs", "bj 128, graphs"]},
            "e2e": {"value": len(probs) / t_e2e, "unit": "evals/s",
                    "h2d_bytes_per_step": int(sum(w["X"].nbytes + w["y"].nbytes for w in ws_)),
                    "d2h_bytes_per_step": 8 * len(probs)},
            "fp64_form": {"evals_per_s": len(probs) / t_fp64, "s_per_batch": t_fp64,
                          "speedup_mixed_vs_fp64": t_fp64 / t_mixed,
                          "max_rel_lml_diff_mixed_vs_fp64": float(np.max(np.abs(lm - l64) / np.abs(l64))),
                          "max_rel_logdet_diff_mixed_vs_fp64": float(np.max(np.abs(ld_m - ld_64) / np.abs(ld_64))),
                          "max_rel_quad_diff_mixed_vs_fp64": float(np.max(np.abs(q_m - q_64) / np.abs(q_64))),
                          "max_logdet_diff_in_fp64_stderr": float(np.max(np.abs(ld_m - ld_64) / se)),
                          "median_rel_logdet_stderr": float(np.median(se / np.abs(ld_64)))},
            "timing": "CUDA events on the calling stream around the batched calls (each call ends with its "
                      "stream synchronisation); e2e: host wall clock, inputs in host memory"}


def run_batch(args):
    import torch

    import paper_2512_06143_gb300 as gp
    from paper_2512_06143_gb300 import build

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    gp.load()
    rec = batch_record(gp, torch, local, steps=args.steps, warmup=args.warmup, seed=rank)
    line = {**rec, "n_gpus": 1, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
