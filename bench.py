#!/usr/bin/env python3
"""Benchmark of the low-sync block Arnoldi solver on one GB300.

A step is one restart cycle of BGMRES(m) with the BCGSI+LS skeleton on the 2D
5-point Laplacian 512x512 (n = 262144) with an n x 8 N(0,1) right-hand side:
CholQR of B, m+1 lagged Arnoldi iterations (SpMM, one-pass Gram, small
Cholesky/least-squares kernel, two-output basis update), the cycle end
(X += V Xi C, U = V [M; -H]) and the true residual ||B - A X||_F.  One step is
one lsba_solve call with max_restarts = 0, so every step does the same work.

value = algorithmic bytes of a step / device time of a step (GB/s, the
"Arnoldi HBM GB/s" of the headline metric); the per-kernel roofline, the
end-to-end number through host buffers, the oracle timed on the host cores,
and BGMRES time-to-1e-10 on the tridiagonal workload are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2208_09899_gb300 import workloads as W  # noqa: E402

METRIC = "BGMRES time-to-1e-10 relres & Arnoldi HBM GB/s vs FP64 plain; serve p50/p99"
WORKLOAD = "lapl512_s8"
M = 20
SKELETON = "bcgsi_ls"
# The headline runs at the paper's precision: FP64 storage, with the Gram and
# update passes as exact 8-bit digit products on the tensor cores (FP64-grade
# results) and the SpMM and small kernels in native FP64.
HEADLINE_PRECISION = "fp64"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def hbm_peak():
    try:
        return float(json.load(open(PEAKS_FILE))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_cost(n, nnz, s, m, skeleton=SKELETON):
    """Algorithmic bytes and FP64 flops of one step (one lagged-skeleton cycle
    of m relations + its true residual), and of its Gram launches alone."""
    blk = 8.0 * n * s
    a_bytes = 12.0 * nnz + 4.0 * (n + 1)
    spmm_flops = 2.0 * nnz * s
    by = {"spmm": 0.0, "gram": 0.0, "update": 0.0}
    fl = {"spmm": 0.0, "gram": 0.0, "update": 0.0}
    # CholQR of B: Gram (1 blk, n s^2 FMA) + scale (read 1, write 1; n s^2 FMA incl. solve)
    by["gram"] += blk
    fl["gram"] += 2.0 * n * s * s
    by["update"] += 2 * blk + blk  # + zeroing X
    fl["update"] += 2.0 * n * s * s
    assert skeleton in ("bcgsi_ls", "bmgs_icwy", "bmgs_cwy")
    for k in range(1, m + 2):
        by["spmm"] += a_bytes + 2 * blk
        fl["spmm"] += spmm_flops
        if k == 1:
            by["gram"] += 2 * blk                       # V_1, W
            fl["gram"] += 2.0 * n * s * s               # s x s outputs
            by["update"] += 3 * blk                     # read V_1, W; write U
            fl["update"] += 2.0 * n * s * s             # U = W - V_1 H_11
        else:
            by["gram"] += (k + 1) * blk                 # V_1..V_{k-1}, U, W once
            fl["gram"] += 2.0 * n * (k * s) * (2 * s)   # ks x 2s outputs
            by["update"] += (k + 3) * blk               # read k+1, write V_k and U
            # V_k = (U - V Y) R^-1 and U' = (W - V Z - V_k P) R^-1: (2k+2) s^2 FMA per row
            fl["update"] += 2.0 * n * s * s * (2 * k + 2)
    # cycle end: read V_1..V_{m+1}, X; write X, U
    by["update"] += (m + 4) * blk
    fl["update"] += 2.0 * n * s * s * (2 * m + 1)   # V_{1:m} Xi C and V_{1:m+1} [M; -H]
    # true residual: SpMM, B - AX, Gram of the residual
    by["spmm"] += a_bytes + 2 * blk
    fl["spmm"] += spmm_flops
    by["update"] += 3 * blk
    by["gram"] += blk
    fl["gram"] += 2.0 * n * s * s
    return by, fl


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


def captured_traffic(kernel_key, bytes_per_launch):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture (profiles/roofline_traffic.json), scaled from the captured launch to
    the average launch by algorithmic bytes; None if absent or if the kernel's
    source file changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(TRAFFIC_FILE))[kernel_key]
        src = open(os.path.join(ROOT, "paper_2208_09899_gb300", "csrc", rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes"] * bytes_per_launch / rec["algorithmic_bytes"]
    except Exception:
        return None


def sample_clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
            stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def sample_clocks_stop(proc, f, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_cycle_seconds(A, B, m):
    """The CPU oracle, as it stands, on one restart cycle of the same workload."""
    from oracle import lsba_oracle as O
    t = time.perf_counter()
    O.solve(A, B, m, 1e-30, SKELETON, modification="gmres", max_restarts=0,
            verify_true_residual=False)
    return time.perf_counter() - t


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def _timed(torch, stream, fn, reps):
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def mixed_precision(torch, lsba, dev, stream):
    """FP32 inner solver inside FP64 iterative refinement vs the FP64-accurate
    paths on the same GPU.
      * per restart cycle on the 2D Laplacian 2048x2048 (n = 4194304), B n x 16,
        BGMRES(16), BCGSI+LS: one FP32 inner cycle (plus the two FP64 residuals
        of its refinement step) vs one double-float and one FP64 cycle;
      * time to relative residual 1e-10 on the 2D Laplacian 128x128, B n x 16,
        BGMRES(16), BCGSI+LS, in the three precisions."""
    out = {}
    A, B = W.workload("lapl2048_s16", 0)
    n, s = B.shape
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    dB = torch.from_numpy(B).to(f"cuda:{dev}")
    dX = torch.empty_like(dB)
    cyc = {}
    for prec, reps in (("fp32_ir", 3), ("df", 2), ("fp64", 1)):
        extra = {"ir_max_outer": 1} if prec == "fp32_ir" else {}
        sv = lsba.Solver(dev, modification="gmres", max_restarts=0, verify_true_residual=0,
                         precision=prec, **extra)
        sv.solve(dA, dB, dX, 16, 1e-30, SKELETON)
        cyc[prec] = _timed(torch, stream, lambda: sv.solve(dA, dB, dX, 16, 1e-30, SKELETON), reps)
        sv.close()
    by, _ = algorithmic_cost(n, A.nnz, s, 16)
    out["cycle"] = {"workload": "lapl2048_s16: 2D Laplacian 2048x2048 (n=4194304), B n x 16 N(0,1),"
                                " BGMRES(16), BCGSI+LS, one restart cycle",
                    "ms": cyc, "speedup_fp32_ir_vs_df": cyc["df"] / cyc["fp32_ir"],
                    "speedup_fp32_ir_vs_fp64": cyc["fp64"] / cyc["fp32_ir"],
                    "fp32_inner_gbs_algorithmic": 0.5 * sum(by.values()) / (cyc["fp32_ir"] * 1e-3) / 1e9}
    del dA, dB, dX
    A = W.laplacian_2d(128)
    B = W.gaussian_block(A.n, 16, 0)
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    dB = torch.from_numpy(B).to(f"cuda:{dev}")
    dX = torch.empty_like(dB)
    tt = {}
    for prec in ("fp32_ir", "df", "fp64"):
        sv = lsba.Solver(dev, modification="gmres", max_restarts=5000, precision=prec)
        ms = _timed(torch, stream, lambda: sv.solve(dA, dB, dX, 16, 1e-10, SKELETON), 1)
        st = sv.stats()
        tt[prec] = {"ms": ms, "cycles": st["cycles"], "relres_true": st["relres_true"],
                    "status": st["status"], "ir_outer": st["ir_outer"]}
        sv.close()
    out["time_to_1e-10"] = {"workload": "lapl128_s16: 2D Laplacian 128x128 (n=16384), B n x 16 "
                                        "N(0,1), BGMRES(16), BCGSI+LS, tol 1e-10",
                            "results": tt,
                            "speedup_fp32_ir_vs_df": tt["df"]["ms"] / tt["fp32_ir"]["ms"],
                            "speedup_fp32_ir_vs_fp64": tt["fp64"]["ms"] / tt["fp32_ir"]["ms"]}
    return out


def rgg_cycles(torch, lsba, dev, stream):
    """The ill-conditioned graph workload: random geometric graph Laplacian,
    n = 2^20, B n x 16, BGMRES(16); BCGS-PIP vs BCGSI+LS, three restart cycles
    each (per-cycle time and the restart log)."""
    A, B = W.workload("rgg1M_s16", 0)
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    dB = torch.from_numpy(B).to(f"cuda:{dev}")
    dX = torch.empty_like(dB)
    out = {"workload": "rgg1M_s16: random geometric graph Laplacian n=2^20 (mean degree "
                       f"{(A.nnz - A.n) / A.n:.2f}), weights 10^U(-3,3), shift 1e-6 max diag; "
                       "B n x 16 N(0,1); BGMRES(16), 3 cycles", "nnz": A.nnz, "skeletons": {}}
    for sk in ("bcgs_pip", "bcgsi_ls"):
        sv = lsba.Solver(dev, modification="gmres", max_restarts=2, verify_true_residual=0,
                         record_history=1)
        sv.solve(dA, dB, dX, 16, 1e-8, sk)
        ms = _timed(torch, stream, lambda: sv.solve(dA, dB, dX, 16, 1e-8, sk), 1)
        st = sv.stats()
        h = sv.history()
        out["skeletons"][sk] = {"ms_per_cycle": ms / max(st["cycles"], 1), "cycles": st["cycles"],
                                "cycle_m": h["cycle_m"], "cycle_flag": h["cycle_flag"],
                                "relres_true": st["relres_true"], "precision": st["precision"]}
        sv.close()
    return out


def skeleton_table(torch, lsba, dev, stream):
    """The 512x512 Laplacian configuration skeleton by skeleton: BGMRES(20) and
    BFOM(20) with BCGS, BCGS-PIP, BCGSI+LS and BMGS-ICWY under precision auto
    (adaptive restart on, tol 1e-8), three restart cycles each: time per cycle,
    sync points and A-calls per cycle, the precision taken and the estimate
    reached."""
    A, B = W.workload(WORKLOAD, 0)
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    dB = torch.from_numpy(B).to(f"cuda:{dev}")
    dX = torch.empty_like(dB)
    out = {"workload": f"{WORKLOAD}, m = 20, tol 1e-8, precision auto, 3 cycles per run", "runs": {}}
    for mod in ("gmres", "fom"):
        for sk in ("bcgs", "bcgs_pip", "bcgsi_ls", "bmgs_icwy"):
            sv = lsba.Solver(dev, modification=mod, max_restarts=2, verify_true_residual=0)
            sv.solve(dA, dB, dX, M, 1e-8, sk)
            ms = _timed(torch, stream, lambda: sv.solve(dA, dB, dX, M, 1e-8, sk), 1)
            st = sv.stats()
            cyc = max(st["cycles"], 1)
            out["runs"][f"{sk}/{mod}"] = {
                "ms_per_cycle": ms / cyc, "cycles": st["cycles"], "syncs_per_cycle": st["syncs"] / cyc,
                "a_calls_per_cycle": st["a_calls"] / cyc, "precision": st["precision"],
                "tensor_cores": st["tensor_cores"], "relres_est": st["relres_est"]}
            sv.close()
    return out


def autotune_table(torch, lsba, dev, stream):
    """The autotuner on the 2D Laplacian 512x512 in double-float, BGMRES(16),
    BCGSI+LS, for s = 4, 8, 16 (B n x s N(0,1)): the chosen Gram and update
    shape of every iteration k, and one restart cycle timed with the fixed
    rules and with the tuned shapes."""
    A = W.laplacian_2d(512)
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    m = 16
    out = {"workload": "lapl512: 2D Laplacian 512x512, B n x s N(0,1), BGMRES(16), BCGSI+LS, "
                       "double-float, one restart cycle", "by_s": {}}
    for s in (4, 8, 16):
        dB = torch.from_numpy(W.gaussian_block(A.n, s, 0)).to(f"cuda:{dev}")
        dX = torch.empty_like(dB)
        cyc = {}
        for tuned in (False, True):
            sv = lsba.Solver(dev, modification="gmres", max_restarts=0, verify_true_residual=0,
                             precision="df")
            if tuned:
                sv.autotune(A.n, s, m)
                table = sv.tune_table()
            sv.solve(dA, dB, dX, m, 1e-30, "bcgsi_ls")
            cyc["tuned" if tuned else "rules"] = _timed(
                torch, stream, lambda: sv.solve(dA, dB, dX, m, 1e-30, "bcgsi_ls"), 3)
            sv.close()
        out["by_s"][str(s)] = {
            "ms_per_cycle": cyc,
            "shapes": [{"k": e["k"], "gram": [e["gram_kernel"], e["gram_ctas_per_sm"], e["gram_rows"]],
                        "gram_us": round(e["gram_us"], 1), "gram_rule_us": round(e["gram_default_us"], 1),
                        "update": [e["update_kernel"], e["update_ctas_per_sm"]],
                        "update_us": round(e["update_us"], 1),
                        "update_rule_us": round(e["update_default_us"], 1)} for e in table]}
    return out


def gram_kernels(torch, lsba, dev, n=262144, s=8, b=2, reps=5):
    """Double-float Gram kernels alone (CUDA events around each launch):
    the tensor-core digit kernel vs the FP32-pipe kernel, L = a blocks and
    R = b blocks of n x s N(0,1) values, device time per launch."""
    rng = np.random.default_rng(0)
    amax = 30
    dL = torch.from_numpy(rng.standard_normal((amax, n, s))).to(f"cuda:{dev}")
    dR = torch.from_numpy(rng.standard_normal((b, n, s))).to(f"cuda:{dev}")
    sv = lsba.Solver(dev, profile=1)
    out = {"workload": f"G = L^T R, L: a blocks, R: {b} blocks of n={n} x s={s} N(0,1); "
                       "us per Gram launch (digit kernel with its reduction; FP32-pipe kernel "
                       "with its reduction)", "a": {}}
    for a in (4, 8, 12, 16, 21, 25, 30):
        L = dL[:a].contiguous()
        dG = torch.empty((a * s, b * s), dtype=torch.float64, device=f"cuda:{dev}")
        row = {}
        for tc in (True, False):
            sv.gram_df(L, dR, dG, tensor_cores=tc)
            sv.reset_profile()
            for _ in range(reps):
                sv.gram_df(L, dR, dG, tensor_cores=tc)
            ms, cnt = sv.profile()["gram"]
            row["tensor_core_us" if tc else "fp32_pipe_us"] = ms / max(cnt, 1) * 1e3
        row["speedup"] = row["fp32_pipe_us"] / row["tensor_core_us"]
        out["a"][str(a)] = row
    sv.close()
    return out


def serving(torch, lsba, dev, count, seed=5, slots=16, cap_gb=150.0):
    """Continuous batching: a seeded mix of block solves (3D 7-point Laplacian
    + delta I, delta ~ U[0,0.1], side N ~ U{22..100}, s ~ U{1,4,8,16,32},
    m ~ U{8..32}, tol 1e-8, BGMRES with BCGSI+LS) served by SolveServer with
    an HBM admission cap.  Capacity = solves/s with every request queued at
    t = 0 (also with one slot, i.e. one solve at a time); then Poisson arrivals
    at 0.8 x capacity give p50/p99 latency.  Host copies of A and B and the
    read-back of X are inside each request's latency."""
    from paper_2208_09899_gb300 import serve
    out = {"workload": f"{count} requests: 3D 7-point Laplacian + delta I, delta~U[0,0.1], "
                       "N~U{22..100} (n=N^3), s~U{1,4,8,16,32}, m~U{8..32}, B~N(0,1), tol 1e-8, "
                       "BGMRES, BCGSI+LS, max 500 restarts",
           "slots": slots, "hbm_cap_gb": cap_gb, "precisions": {}}
    warm = serve.serving_requests(slots, seed=99, side_range=(8, 12), m_range=(4, 8))
    t0 = time.perf_counter()
    base = serve.serving_requests(count, seed=seed)
    out["request_build_s"] = time.perf_counter() - t0
    for prec in ("auto", "fp32_ir"):
        for r in base:
            r.precision, r.arrival = prec, 0.0
        for r in warm:
            r.precision = prec
        res = {}
        if prec == "auto":
            one = serve.SolveServer(slots=1, hbm_cap_bytes=cap_gb * 1e9, device=dev)
            one.run(warm[:1], keep_x=False)
            res["capacity_one_slot"] = serve.summarize(one.run(base, keep_x=False))
            one.close()
        srv = serve.SolveServer(slots=slots, hbm_cap_bytes=cap_gb * 1e9, device=dev)
        srv.run(warm, keep_x=False)
        cap = serve.summarize(srv.run(base, keep_x=False))
        res["capacity"] = cap
        rate = 0.8 * cap["solves_per_s"]
        for r, a in zip(base, serve.poisson_arrivals(count, rate, seed=seed + 1)):
            r.arrival = float(a)
        load = srv.run(base, keep_x=False)
        res["load_0.8"] = dict(serve.summarize(load, t_first=0.0), rate_per_s=rate)
        res["peak_admitted_gb"] = srv.peak_bytes / 1e9
        res["status_counts"] = {str(k): sum(1 for r in load if r.stats.get("status") == k)
                                for k in sorted({r.stats.get("status") for r in load}, key=str)}
        res["mean_cycles"] = float(np.mean([r.stats.get("cycles", 0) for r in load]))
        srv.close()
        out["precisions"][prec] = res
    return out


def max_over_ranks(x, pg, device="cpu"):
    """The largest of the ranks' values: replicas run independently, and the
    job takes as long as its slowest rank."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, step_bytes, ms_step):
    """Whole-job GB/s: every rank processes one step of the workload per step
    time (weak scaling), so the job moves world x step_bytes."""
    return world * step_bytes / (ms_step * 1e-3) / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle (numpy FP64) on the same workload/metric."""
    if rank != 0:
        return 0
    A, B = W.workload(WORKLOAD, 0)
    n, s = B.shape
    by, fl = algorithmic_cost(n, A.nnz, s, M)
    step_bytes = sum(by.values())
    for _ in range(args.warmup):
        oracle_cycle_seconds(A, B, M)
    ts = [oracle_cycle_seconds(A, B, M) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    value = step_bytes / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: 2D 5-point Laplacian 512x512 (n=262144), B n x 8 "
                               f"N(0,1), BGMRES(m={M}), BCGSI+LS, one restart cycle per step",
                   "n": n, "s": s, "m": M, "skeleton": SKELETON},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": blas_threads(), "kind": "oracle",
                         "sample": f"one BGMRES({M}) restart cycle per step (numpy FP64 oracle)"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def profile_cycle(precision):
    """One restart cycle of the headline workload (the launch sequence an ncu
    capture selects its kernels from): lapl512_s8, BGMRES(20), BCGSI+LS."""
    import torch
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    lsba.load()
    A, B = W.workload(WORKLOAD, 0)
    dA = lsba.DeviceCSR.from_host(A, "cuda:0")
    dB = torch.from_numpy(B).to("cuda:0")
    dX = torch.empty_like(dB)
    extra = {"tensor_cores": 0} if precision == "fp64-plain" else {}
    prec = "fp64" if precision == "fp64-plain" else precision
    sv = lsba.Solver(0, modification="gmres", max_restarts=0, verify_true_residual=0,
                     precision=prec, cuda_graphs=0, **extra)
    sv.solve(dA, dB, dX, M, 1e-30, SKELETON)
    torch.cuda.synchronize()
    st = sv.stats()
    print(json.dumps({"profile_cycle": precision, "cycles": st["cycles"], "steps": st["steps"],
                      "tensor_cores": st["tensor_cores"]}))
    sv.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-rgg", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-gram-kernels", action="store_true")
    ap.add_argument("--no-skeletons", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--profile-cycle", default=None,
                    help="run one restart cycle of the workload in this precision (fp64, df, "
                         "fp64-plain) and exit: the launch list that ncu captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.profile_cycle:
        return profile_cycle(args.profile_cycle)

    import torch
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    lsba.load()
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    A, B = W.workload(WORKLOAD, 0)
    n, s = B.shape
    dA = lsba.DeviceCSR.from_host(A, f"cuda:{dev}")
    dB = torch.from_numpy(B).to(f"cuda:{dev}")
    dX = torch.empty_like(dB)
    sv = lsba.Solver(dev, modification="gmres", max_restarts=0, verify_true_residual=0,
                     profile=1, precision=HEADLINE_PRECISION)
    stream = torch.cuda.current_stream(dev)

    def step():
        sv.solve(dA, dB, dX, M, 1e-30, SKELETON)

    clk_path = os.path.join(tempfile.gettempdir(), f"lsba_clocks_{os.getpid()}.csv")
    proc, fh = sample_clocks_start(clk_path)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st0 = sv.stats()
    assert st0["cycles"] == 1 and st0["steps"] == M, st0
    sv.reset_profile()

    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks = sample_clocks_stop(proc, fh, clk_path, dev)
    ms_total = max_over_ranks(e0.elapsed_time(e1), pg, device=f"cuda:{dev}")
    ms_step = ms_total / args.steps
    prof = sv.profile()

    by, fl = algorithmic_cost(n, A.nnz, s, M)
    step_bytes = sum(by.values())
    value = replica_value(world, step_bytes, ms_step)
    hbm, hbm_src = hbm_peak()

    # Roofline of the dominant kernel class (by device time).
    dom = max(("gram", "update", "spmm"), key=lambda k: prof[k][0])
    dom_ms_per_step = prof[dom][0] / args.steps
    dom_launches = prof[dom][1] / args.steps
    achieved_tflops = fl[dom] / (dom_ms_per_step * 1e-3) / 1e12
    achieved_gbs = by[dom] / (dom_ms_per_step * 1e-3) / 1e9
    is_df = st0["precision"] == 1
    is_ftc = st0["precision"] == 0 and st0["tensor_cores"] == 1
    kernel_names = {
        "gram": ("k_gram_df_tcs (stored digits, tensor cores, iterations k >= 2) + k_gram_df_tma "
                 "(start block, k <= 4) + k_gram_reduce_df" if is_df else
                 "k_gram_f64tc (FP64 digit products on tcgen05) + k_gram_reduce" if is_ftc else
                 "k_gram + k_gram_reduce"),
        "update": ("k_coef_fold + k_update_df_tcs (tensor cores, iterations k >= 2 and the cycle "
                   "end; also writes the new block's digit planes) + k_coef_df + k_update_df_row "
                   "(start block, k = 1) + k_split_digits (start block)" if is_df else
                   "k_coef_fold64 + k_update_f64tc (FP64 digit products on tcgen05, every update "
                   "of the cycle and its end)" if is_ftc else "k_update"),
        "spmm": ("k_spmm_df8" if is_df else
                 "k_spmm_digits (FP64 SpMM writing W with its tile exponents and digit planes)" if is_ftc else "k_spmm"),
    }
    traffic_key = dom + ("_df" if is_df else "_f64tc" if is_ftc else "")
    roofline = {
        "kernel": kernel_names[dom],
        "bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
        "frac": achieved_gbs / hbm, "peak_source": f"{hbm_src} (copy bandwidth)",
        "traffic": captured_traffic(traffic_key, by[dom] / max(dom_launches, 1)),
        "launches_per_step": dom_launches,
        "algorithmic_bytes_per_launch": by[dom] / max(dom_launches, 1),
        "algorithmic_flops_per_launch": fl[dom] / max(dom_launches, 1),
        "fp64_equivalent_tflops": achieved_tflops,
        "dominant_by_device_time": max(prof, key=lambda k: prof[k][0]),
    }
    kernels = {k: {"ms_per_step": prof[k][0] / args.steps, "launches_per_step": prof[k][1] / args.steps,
                   "share": prof[k][0] / max(sum(v[0] for v in prof.values()), 1e-12)}
               for k in prof}
    gpu_launches = int(sum(v[1] for v in prof.values()))

    # The same steps with native FP64 (DFMA) Gram/update/SpMM kernels.
    sv64 = lsba.Solver(dev, modification="gmres", max_restarts=0, verify_true_residual=0,
                       precision="fp64", tensor_cores=0)
    for _ in range(2):
        sv64.solve(dA, dB, dX, M, 1e-30, SKELETON)
    k64 = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(k64):
        sv64.solve(dA, dB, dX, M, 1e-30, SKELETON)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    ms64 = f0.elapsed_time(f1) / k64
    fp64_plain = {"value": step_bytes / (ms64 * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms64,
                  "speedup_of_value": ms64 / ms_step,
                  "note": "native FP64 (DFMA) SpMM, Gram and update kernels (tensor_cores = 0)"}
    sv64.close()
    # The same steps in double-float (hi + lo FP32 pairs, 48-bit significand).
    svdf = lsba.Solver(dev, modification="gmres", max_restarts=0, verify_true_residual=0,
                       precision="df")
    for _ in range(2):
        svdf.solve(dA, dB, dX, M, 1e-30, SKELETON)
    torch.cuda.synchronize(dev)
    f0.record(stream)
    for _ in range(k64):
        svdf.solve(dA, dB, dX, M, 1e-30, SKELETON)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    msdf = f0.elapsed_time(f1) / k64
    df48 = {"value": step_bytes / (msdf * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": msdf,
            "note": "double-float (48-bit significand, FP32 exponent range; narrower than FP64)"}
    svdf.close()

    # End to end through the C ABI with host buffers (copies inside the timed region).
    # Inputs and the result live in pinned host memory.
    e2e_steps = min(args.steps, 3)
    hA = lsba.PinnedCSR(A)
    hB = torch.from_numpy(np.ascontiguousarray(B)).pin_memory()
    hX = torch.empty_like(hB).pin_memory()
    sv.solve_host(hA, hB, M, 1e-30, SKELETON, X=hX)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sv.solve_host(hA, hB, M, 1e-30, SKELETON, X=hX)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, pg, device=f"cuda:{dev}")
    h2d = A.nnz * 12 + (A.n + 1) * 4 + B.nbytes
    d2h = B.nbytes
    e2e = {"value": replica_value(world, step_bytes, e2e_s * 1e3), "unit": "GB/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": e2e_s * 1e3}

    # BGMRES time to 1e-10 on the tridiagonal workload (configuration 1).
    A1, B1 = W.workload("tridiag2000_s4", 0)
    dA1 = lsba.DeviceCSR.from_host(A1, f"cuda:{dev}")
    dB1 = torch.from_numpy(B1).to(f"cuda:{dev}")
    dX1 = torch.empty_like(dB1)
    sv1 = lsba.Solver(dev, modification="gmres", max_restarts=50, precision=HEADLINE_PRECISION)
    for _ in range(3):
        sv1.solve(dA1, dB1, dX1, 10, 1e-10, SKELETON)
    tts = []
    for _ in range(10):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sv1.solve(dA1, dB1, dX1, 10, 1e-10, SKELETON)
        b.record(stream)
        torch.cuda.synchronize(dev)
        tts.append(a.elapsed_time(b))
    st1 = sv1.stats()
    sv0 = lsba.Solver(dev, modification="gmres", max_restarts=50, cuda_graphs=0,
                      precision=HEADLINE_PRECISION)
    for _ in range(3):
        sv0.solve(dA1, dB1, dX1, 10, 1e-10, SKELETON)
    tts0 = []
    for _ in range(10):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sv0.solve(dA1, dB1, dX1, 10, 1e-10, SKELETON)
        b.record(stream)
        torch.cuda.synchronize(dev)
        tts0.append(a.elapsed_time(b))
    sv0.close()
    time_to_tol = {"workload": "tridiag2000_s4: tridiag(-1,4,-1) n=2000, B 2000x4 N(0,1), "
                               "BGMRES(10), BCGSI+LS, tol 1e-10, max 50 restarts",
                   "ms": statistics.median(tts), "ms_direct_launches": statistics.median(tts0),
                   "cycles": st1["cycles"], "steps": st1["steps"],
                   "relres_true": st1["relres_true"], "status": st1["status"],
                   "note": "ms: restart cycles replayed from CUDA graphs (default); "
                           "ms_direct_launches: cuda_graphs=0"}

    mixed = None if args.no_mixed else mixed_precision(torch, lsba, dev, stream)
    rgg = None if args.no_rgg else rgg_cycles(torch, lsba, dev, stream)
    served = None if args.no_serving else serving(torch, lsba, dev, args.serve_requests)
    gk = None if args.no_gram_kernels else gram_kernels(torch, lsba, dev)
    skt = None if args.no_skeletons else skeleton_table(torch, lsba, dev, stream)
    tun = None if args.no_autotune else autotune_table(torch, lsba, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_or = oracle_cycle_seconds(A, B, M)
        from oracle import lsba_oracle as O
        t1 = time.perf_counter()
        O.solve(A1, B1, 10, 1e-10, SKELETON, modification="gmres", max_restarts=50)
        t_or1 = time.perf_counter() - t1
        cpu = {"value": step_bytes / t_or / 1e9, "unit": "GB/s", "cores": blas_threads(),
               "kind": "oracle", "sample": f"one BGMRES({M}) restart cycle of {WORKLOAD} "
                                           f"({t_or:.1f} s)",
               "time_to_tol_ms": t_or1 * 1e3}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("df48 (double-float: hi+lo FP32 pairs, 48-bit significand, FP32 exponent "
                      "range; narrower than FP64)" if is_df else
                      "f64 (FP64 storage; Gram and update as exact products of 8-bit digits "
                      "carrying 53 bits, on the tcgen05 tensor cores, FP64 accumulation; SpMM "
                      "and small kernels native FP64)" if is_ftc else "f64"),
            "data": "synthetic (seeded numpy inputs shaped like the paper's lapl_2d)",
            "config": {"workload": f"{WORKLOAD}: 2D 5-point Laplacian 512x512 (n=262144), B n x 8 "
                                   f"N(0,1), BGMRES(m={M}), BCGSI+LS, one restart cycle per step",
                       "n": n, "s": s, "m": M, "nnz": A.nnz, "skeleton": SKELETON,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "no flush: a step streams a 0.39 GB working set (> 129 MB L2)",
                       "algorithmic_bytes_per_step": step_bytes},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clocks, "time_to_tol": time_to_tol,
            "fp64_plain": fp64_plain, "df48": df48, "mixed_precision": mixed,
            "graph_workload": rgg,
            "serving": served, "gram_kernels": gk, "skeletons": skt, "autotune": tun,
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
