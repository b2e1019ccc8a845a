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


def assembly_roofline(n: int, d: int, L: int, nnz: int, ms: float, hbm_gbs: float) -> dict:
    """Whole assembly (sort, cell list, count, scan, fill, FP64 values) against its algorithmic
    roofline: memory leg = the CSR written once (8 B per stored entry + 4 B per row pointer);
    compute leg = one support test (2d FP32 instructions) and one value (2d + 8 + L instructions,
    a fused multiply-add counted once) per unique pair, (nnz + n) / 2 pairs, at the FP32 issue
    rate of 152 SMs x 128 lanes x 2.07 GHz."""
    mem = 8.0 * nnz + 4.0 * (n + 1)
    instr = 0.5 * (nnz + n) * (2 * d + 2 * d + 8 + L)
    t_mem, t_alu = mem / (hbm_gbs * 1e9), instr / FP32_INSTR_PEAK
    roof_ms = 1000.0 * max(t_mem, t_alu)
    return {"ms": ms, "gnnz_per_s": nnz / (ms * 1e6) if ms > 0 else None,
            "roofline": {"bound": "hbm" if t_mem >= t_alu else "alu", "bytes": mem, "fp32_instr": instr,
                         "roof_ms": roof_ms, "frac": roof_ms / ms if ms > 0 else None,
                         "alu_peak_instr_per_s": FP32_INSTR_PEAK}}


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
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    w, wopts = make_workload(args.workload, seed=rank, n=args.n)
    hyper = gp.Hyper(**w["hyper"])
    n = w["X"].shape[0]
    precision = gp.PREC_MIXED if args.workload != "small_2d" else gp.PREC_FP64
    opts = gp.default_opts(precision=precision, **wopts)
    X = torch.tensor(w["X"], dtype=torch.float64, device="cuda")
    y = torch.tensor(w["y"], dtype=torch.float64, device="cuda")
    Xh = torch.tensor(w["X"], dtype=torch.float64).pin_memory()
    yh = torch.tensor(w["y"], dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    ctx = gp.Context(local, stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # 256 MB > 129 MB L2

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.lml_grad(X, y, hyper, opts)
    # --- timed region: device-resident inputs -------------------------------------------------
    prof_opts = gp.default_opts(precision=precision, profile=1, **wopts)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        lml, g, info = ctx.lml_grad(X, y, hyper, prof_opts)
        ev[k][1].record(stream)
        infos.append(info)
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # --- e2e: host buffers, H2D of X and y and D2H of the LML and gradient inside the call ------
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.lml_grad(Xh, yh, hyper, opts)
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_total = sum(e2e_ms)
    value, e2e_value, total_ms, e2e_total = replica_throughput(ws, args.steps, total_ms, e2e_total, "cuda")
    # roofline of the dominant kernel (SpMM of the Krylov solves)
    spmm_ms = sum(i["ms_spmm"] for i in infos)
    spmm_launches = sum(i["spmm_launches"] for i in infos)
    spmm_bytes = sum(i["spmm_bytes"] for i in infos)
    peak, peak_src = load_peaks()
    achieved = (spmm_bytes / spmm_launches) / ((spmm_ms / spmm_launches) / 1000.0) / 1e9 if spmm_ms > 0 else None
    launches = int(sum(i["launches"] for i in infos))
    traffic, traffic_src = profile_traffic(args.workload, int(n))
    if rank == 0:
        cpu_v, cores, sample, _ = oracle_sample(args.workload) if not args.no_cpu_baseline else (None, None, "skipped", 0)
        i0 = infos[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if precision == gp.PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": int(n), "d": int(hyper.d), "L": hyper.L,
                       "nnz": int(i0["nnz"]), "probes": int(opts.probes), "lanczos_steps": int(opts.lanczos_steps),
                       "precision": "mixed" if precision == gp.PREC_MIXED else "fp64", "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"kernel": "k_spmm_rb (multi-RHS RB8 SpMM of the Krylov solves)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "traffic_source": traffic_src,
                         "peak_source": f"{peak_src} hbm_gbs",
                         "launches_per_step": spmm_launches / args.steps,
                         "bytes_per_launch": spmm_bytes / max(spmm_launches, 1),
                         "ms_per_launch": spmm_ms / max(spmm_launches, 1),
                         "share_of_step": spmm_ms / total_ms if total_ms > 0 else None,
                         "bytes_definition": "8 B per stored entry (FP32 value + int32 column) + 4 B per row "
                                             "pointer + 4 B per input and per output vector element"},
            "assembly": assembly_roofline(int(n), int(hyper.d), int(hyper.L), int(i0["nnz"]), i0["ms_assemble"], peak),
            "cpu_baseline": {"value": cpu_v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": int(Xh.numel() * 8 + yh.numel() * 8),
                    "d2h_bytes_per_step": int(8 + 8 * hyper.nparams)},
            "clocks": clocks, "gpu_launches": launches,
            "detail": {"ms_assemble": i0["ms_assemble"], "ms_solve": i0["ms_solve"], "ms_logdet": i0["ms_logdet"],
                       "ms_grad": i0["ms_grad"], "iters_y": i0["iters_y"], "iters_probes": i0["iters_probes"],
                       "outer": i0["outer"], "relres": i0["relres"], "lml": i0["lml"],
                       "logdet_stderr": i0["logdet_stderr"], "step_ms": step_ms},
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
    ap.add_argument("--n", type=int, default=None,
                    help="points per problem (default: the workload's full size); smaller n = profiling case")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_gpu(args)


def run_batch(args):
    """256 independent problems (N log-uniform in [2048, 65536], d in {1,2,3}, 10-200 entries per
    row), one gp2s_lml_batched call per step (SLQ, 32 probes x 100 steps): mixed precision timed,
    and the plain FP64 GPU form timed once beside it with the accuracy of both against each other."""
    import torch

    import paper_2512_06143_gb300 as gp
    from paper_2512_06143_gb300 import build
    from paper_2512_06143_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    gp.load()
    probs = []
    for w in W.batch(rank):
        probs.append((torch.tensor(w["X"], device="cuda"), torch.tensor(w["y"], device="cuda"),
                      gp.Hyper(**w["hyper"])))
    ctx = gp.Context(local, torch.cuda.current_stream().cuda_stream)
    mixed = gp.default_opts(precision=gp.PREC_MIXED, logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=100)
    fp64 = gp.default_opts(precision=gp.PREC_FP64, logdet=gp.LOGDET_SLQ, probes=32, lanczos_steps=100, precond=1)
    for _ in range(args.warmup):
        ctx.lml_batched(probs, mixed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lm, infos = ctx.lml_batched(probs, mixed)
    torch.cuda.synchronize()
    t_mixed = (time.perf_counter() - t0) / args.steps
    ctx.lml_batched(probs, fp64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l64, i64 = ctx.lml_batched(probs, fp64)
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    lm, l64 = np.asarray(lm), np.asarray(l64)
    rel = float(np.max(np.abs(lm - l64) / np.abs(l64)))
    ld_m = np.array([i["logdet"] for i in infos])
    ld_64 = np.array([i["logdet"] for i in i64])
    q_m = np.array([i["quad"] for i in infos])
    q_64 = np.array([i["quad"] for i in i64])
    se = np.array([i["logdet_stderr"] for i in i64])
    ld_se = float(np.median(se / np.abs(ld_64)))
    line = {"metric": "batched LML evals/s", "value": len(probs) / t_mixed, "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_mixed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch", "problems": len(probs), "n_total": int(sum(p[0].shape[0] for p in probs)),
                       "probes": 32, "lanczos_steps": 100},
            "fp64_form": {"evals_per_s": len(probs) / t_fp64, "s_per_batch": t_fp64,
                          "speedup_mixed_vs_fp64": t_fp64 / t_mixed,
                          "max_rel_lml_diff_mixed_vs_fp64": rel,
                          "max_rel_logdet_diff_mixed_vs_fp64": float(np.max(np.abs(ld_m - ld_64) / np.abs(ld_64))),
                          "max_rel_quad_diff_mixed_vs_fp64": float(np.max(np.abs(q_m - q_64) / np.abs(q_64))),
                          "max_logdet_diff_in_fp64_stderr": float(np.max(np.abs(ld_m - ld_64) / se)),
                          "median_rel_logdet_stderr": ld_se},
            "timing": "host wall clock around each batched call (includes its stream synchronisation)"}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
