#!/usr/bin/env python
"""Benchmark of the randomized SVD on one (or N independent) GB300.

Workload: dense FP32 A, 100000 x 20000 (8 GB), A = U diag(s) V^T with
s_i = |1/i + 1e-4 g_i|, rank k = 100, oversampling p = 20, q = 2 power
iterations, 4096 x 4096 block-cyclic tiles.  One step = one full randomized
SVD (Gaussian test matrix, 2q+2 A-passes, CholeskyQR2 after each, small SVD,
lift) with A already resident in HBM.  A (8 GB) is larger than L2 (129 MB),
so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  Options:
  --gpus N --steps K --warmup W    replicas on N GPUs (torchrun), K timed steps
  --impl reference                 time the FP64 CPU oracle on a bounded sample
  --prec bf16|fp32|bf16x3          precision of the headline path
  --mode apass|ooc|csr             A-passes alone; the out-of-core workload;
                                   the sparse (CSR) workload
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "dense_fp32_100000x20000"
METRIC = "rsvd_throughput_dense_fp32_100000x20000_k100_p20_q2"
UNIT = "rSVD/s"
ORACLE_SAMPLE_ROWS = 10000


DATA_NOTE = "synthetic: A = U diag(s) V^T, U and V from QR of seeded Gaussians, s_i = |1/i + 1e-4 g_i|"


def _config(w, prec, ws):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q, "tile": w.tile,
            "prec": prec, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (A is 8 GB)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop x SM clock.  The clock is the
# median SM clock sampled under load in the same run (max 2070 MHz).
def _fp32_peak_tflops(sm_mhz: float) -> float:
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms during a region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm.append(float(parts[2]))
                mx = float(parts[3])
            except ValueError:
                continue
            for nm, val in zip(names, parts[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_time_and_value(elapsed_ms: float, steps: int, device=None):
    """Whole-job timing over replicas: the slowest rank's time (max over ranks)
    and the aggregate throughput, world_size * steps / that time.  Without an
    initialised process group this is the single-GPU case."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if ws > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, ws * steps / (elapsed_ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _spectrum(n, noise_seed):
    from synth import spectrum_harmonic_noisy
    return spectrum_harmonic_noisy(n, 1e-4, noise_seed)


def _build_A(device):
    import torch
    from synth import WORKLOADS, prescribed_dense_torch
    w = WORKLOADS[WORKLOAD]
    s = _spectrum(w.n, w.noise_seed)
    A = prescribed_dense_torch(w.m, w.n, s, w.data_seed, device=device)
    torch.cuda.synchronize()
    return w, A


# sources that define each profiled kernel (its code and everything it includes)
KERNEL_SOURCES = {
    "tc_apass_kernel": ["gemm_tc.cu", "tc_ptx.cuh", "common.cuh", "kernels.cuh"],
    "tc_apass_kernel_bf16_run": ["gemm_tc.cu", "tc_ptx.cuh", "common.cuh", "kernels.cuh"],
    "simt_gemm_kernel": ["gemm_simt.cu", "common.cuh", "kernels.cuh"],
}


def kernel_digest(kernel_key: str) -> str:
    """SHA-256 over the names and contents of the kernel's sources, the public
    header and the compiler flags (independent of where the tree lives)."""
    import hashlib
    from paper_1907_06470_gb300 import build as b
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel_key]:
        h.update(name.encode())
        with open(os.path.join(b.CSRC, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(b.INCLUDE, "rsvd.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(b.NVCC_FLAGS).encode())
    return h.hexdigest()


def _traffic_for(kernel_key: str, elements: float):
    """DRAM bytes (read + write) per launch from the committed ncu summary
    (profiles/traffic.json), taken on a smaller launch and scaled by the entries
    of A this launch streams (`elements`) over the captured launch's -- the
    traffic of an A-pass grows in proportion -- if the kernel's sources are the
    ones the counters were taken on; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except OSError:
        return None
    ent = data.get(kernel_key)
    if not ent or ent.get("source_digest") != kernel_digest(kernel_key):
        return None
    return ent["dram_bytes_per_launch"] * elements / ent["captured_elements"]


def oracle_sample_seconds(A_rows_f32: np.ndarray, w) -> float:
    """Wall time of the FP64 CPU oracle on the first rows of A (same n, k, p, q, seed)."""
    from oracle import rsvd as OR
    t0 = time.perf_counter()
    OR.rsvd(A_rows_f32, w.k, w.p, w.q, w.seed, "f32")
    return time.perf_counter() - t0


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import torch
    device = torch.device("cuda", local) if torch.cuda.is_available() else None
    if device is None:
        print(json.dumps({"impl": "reference", "unavailable": "no CUDA device to build the synthetic matrix"}))
        return 0
    w, A = _build_A(device)
    sample = A[:ORACLE_SAMPLE_ROWS].cpu().numpy()
    del A
    torch.cuda.empty_cache()
    scale = w.m / ORACLE_SAMPLE_ROWS
    for _ in range(args.warmup):
        oracle_sample_seconds(sample, w)
    times = [oracle_sample_seconds(sample, w) for _ in range(args.steps)]
    t_sample = sum(times) / len(times)
    t_step = t_sample * scale
    value = 1.0 / t_step
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        # the timed region: K steps, each one oracle rSVD of the bounded sample
        "ms_per_step": t_sample * 1e3,
        "ms_per_full_rsvd_extrapolated": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA_NOTE,
        "config": _config(w, args.prec, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: the oracle rSVD of the first {ORACLE_SAMPLE_ROWS} of {w.m} rows "
                                   f"(full n, k, p, q); value = 1 / (sample time x m/{ORACLE_SAMPLE_ROWS} = "
                                   f"{scale:g})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# Bars of the FP32 path against the FP64 oracle: singular values within 1e-5
# relative, largest principal angle of U_k and of V_k within 1e-4.
SIGMA_BAR, ANGLE_BAR = 1e-5, 1e-4


def accuracy_vs_oracle(w, A, results):
    """Errors of each path's U, S, V against the FP64 oracle run on the same A
    (the whole workload: one oracle rSVD with the FP32-rounded test matrix for
    the FP32 path, one with the BF16-rounded test matrix for the tensor-core
    paths), and the fastest path that meets the FP32 bars with its speedup
    over the FP32 path."""
    from oracle import rsvd as OR
    from tests.metrics import cluster_safe_angles, sigma_rel_err
    A_host = A.cpu().numpy()
    refs, oracle_s = {}, {}
    out = {}
    for pr, (ms, U, S, V) in results.items():
        od = "f32" if pr == "fp32" else "bf16"
        if od not in refs:
            t0 = time.perf_counter()
            refs[od] = OR.rsvd(A_host, w.k, w.p, w.q, w.seed, od)
            oracle_s[od] = time.perf_counter() - t0
        Uo, So, Vo = refs[od]
        es = sigma_rel_err(S, So)
        eu = cluster_safe_angles(U, Uo, So, w.k)
        ev = cluster_safe_angles(V, Vo, So, w.k)
        out[pr] = {"sigma_rel_err": es, "angle_U": eu, "angle_V": ev,
                   "meets_fp32_bars": bool(es <= SIGMA_BAR and eu <= ANGLE_BAR and ev <= ANGLE_BAR),
                   "oracle_test_matrix": od}
    out["bars"] = {"sigma_rel": SIGMA_BAR, "angle": ANGLE_BAR,
                   "oracle": "FP64 oracle (oracle/rsvd.py) on the same A, whole workload",
                   "oracle_seconds": oracle_s, "cores": os.cpu_count()}
    ok = [pr for pr in results if out[pr]["meets_fp32_bars"]]
    matched = None
    if ok and "fp32" in results:
        best = min(ok, key=lambda pr: results[pr][0])
        matched = {"path": best, "ms_per_step": results[best][0], "rsvd_per_s": 1e3 / results[best][0],
                   "speedup_vs_fp32": results["fp32"][0] / results[best][0],
                   "fp32_ms_per_step": results["fp32"][0]}
    return out, matched


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_1907_06470_gb300 as g
    g.load()

    w, A = _build_A(device)
    m, n, k, p, q = w.m, w.n, w.k, w.p, w.q
    prec = args.prec

    plan = g.Plan(m, n, k, p, q, w.seed, prec=prec, mb=w.tile, nb=w.tile)
    plan.set_profiling(True)
    U = torch.empty(m, k, device=device)
    S = torch.empty(k, device=device)
    V = torch.empty(n, k, device=device)
    for _ in range(args.warmup):
        plan.run(A, U, S, V)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    stage_sum = {}
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = g.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run(A, U, S, V)
        for key, val in plan.stage_ms().items():
            stage_sum[key] = stage_sum.get(key, 0.0) + val
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = g.kernel_launches() - launches0
    clocks = sampler.stop()
    elapsed_ms, value = job_time_and_value(elapsed_ms, args.steps, device)
    ms_per_step = elapsed_ms / args.steps
    S_head = S.double().cpu().numpy()
    plan_info = plan.info()

    # --- roofline of the dominant kernel: the A-pass ---------------------------
    peaks, peak_kind = _peaks()
    apass_calls = stage_sum.get("apass_calls", 0)
    apass_ms = stage_sum.get("apass_fwd", 0.0) + stage_sum.get("apass_trans", 0.0)
    avg_apass_s = apass_ms / max(apass_calls, 1) / 1e3
    bytes_per_pass = m * n * 4 + (m + n) * (k + p) * 4
    flops_per_pass = 2.0 * m * n * (k + p)
    if prec == "bf16" and plan_info.get("bf16_copy"):
        # the first forward pass reads FP32 A and writes its BF16 copy, the next
        # 2q passes read the copy, the split-BF16 B^T pass reads FP32 A: the
        # average algorithmic bytes of the run's passes
        passes = 2 * q + 2
        panels = (m + n) * (k + p) * 4
        bytes_per_pass = ((m * n * 6 + panels) + 2 * q * (m * n * 2 + panels) + (m * n * 4 + panels)) / passes
    if prec == "fp8":
        # 2q+1 passes read the E4M3 codes (1 byte per entry); the split-BF16
        # refinement of B^T reads the FP32 A: the average over the run's passes
        passes = 2 * q + 2
        bytes_per_pass = ((passes - 1) * (m * n + (m + n) * (k + p) * 4) + (m * n * 4 + (m + n) * (k + p) * 4)) / passes
    if prec == "fp32":
        achieved = flops_per_pass / avg_apass_s / 1e12
        peak = _fp32_peak_tflops(clocks["sm_mhz"] or 2070.0)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock under load",
                "traffic": _traffic_for("simt_gemm_kernel", m * n), "kernel": "simt_gemm_kernel (A-pass)"}
    else:
        achieved = bytes_per_pass / avg_apass_s / 1e9
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs ({peak_kind})",
                "traffic": _traffic_for("tc_apass_kernel", m * n) if prec == "bf16" else None,
                "kernel": "tc_apass_kernel (A-pass)",
                "tflops": flops_per_pass / avg_apass_s / 1e12}
    roof["algorithmic_bytes_per_launch"] = bytes_per_pass
    roof["avg_launch_ms"] = avg_apass_s * 1e3
    if prec == "bf16" and plan_info.get("bf16_copy"):
        roof["passes"] = ("1 forward pass over FP32 A writing its BF16 copy, 2q passes over the copy, "
                          "1 split-BF16 pass over FP32 A; bytes and time averaged over the run's passes")
        roof["traffic"] = _traffic_for("tc_apass_kernel_bf16_run", m * n)

    # --- end to end through the public API with host buffers ----------------------
    e2e = None
    if not args.no_e2e:
        A_host = torch.empty(m, n, dtype=torch.float32, pin_memory=True)
        A_host.copy_(A)
        Uh = torch.empty(m, k, pin_memory=True)
        Sh = torch.empty(k, pin_memory=True)
        Vh = torch.empty(n, k, pin_memory=True)
        plan_h = g.Plan(m, n, k, p, q, w.seed, prec=prec, mb=w.tile, nb=w.tile)
        Ud, Sd, Vd = plan_h.run(A_host)
        # the same warm-up count as the device-resident loop: the first host reads
        # of a freshly pinned 8 GB buffer run slower than the steady state
        for _ in range(max(0, args.warmup - 1)):
            plan_h.run(A_host, Ud, Sd, Vd)
        torch.cuda.synchronize()
        steps_e2e = max(1, args.steps)  # the K steps of the device loop (about 45 ms each)
        host_split = []
        # no collector pauses inside the timed host loop
        import gc
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            ta = time.perf_counter()
            plan_h.run(A_host, Ud, Sd, Vd)
            tb = time.perf_counter()
            Uh.copy_(Ud, non_blocking=True)
            Sh.copy_(Sd, non_blocking=True)
            Vh.copy_(Vd, non_blocking=True)
            torch.cuda.synchronize()
            host_split.append([round((tb - ta) * 1e3, 2), round((time.perf_counter() - tb) * 1e3, 2)])
        t_e2e = (time.perf_counter() - t0) / steps_e2e
        # the same K steps with the inputs pipelined (Plan.prefetch): each step's
        # 8 GB copy is issued before the previous step runs, so the link works
        # while the previous matrix is factored; every step still copies its A
        # (the first copy inside the timed region too) and reads back U, S, V
        host_pipe = []
        t0 = time.perf_counter()
        plan_h.prefetch(A_host)
        for i in range(steps_e2e):
            ta = time.perf_counter()
            if i + 1 < steps_e2e:
                plan_h.prefetch(A_host)
            plan_h.run(A_host, Ud, Sd, Vd)
            tb = time.perf_counter()
            Uh.copy_(Ud, non_blocking=True)
            Sh.copy_(Sd, non_blocking=True)
            Vh.copy_(Vd, non_blocking=True)
            torch.cuda.synchronize()
            host_pipe.append([round((tb - ta) * 1e3, 2), round((time.perf_counter() - tb) * 1e3, 2)])
        t_pipe = (time.perf_counter() - t0) / steps_e2e
        gc.enable()
        plan_h.set_profiling(True)  # one more call with stage events, outside the timed loops
        plan_h.run(A_host, Ud, Sd, Vd)
        torch.cuda.synchronize()
        e2e = {"value": ws / t_pipe, "unit": UNIT, "h2d_bytes_per_step": m * n * 4,
               "d2h_bytes_per_step": (m * k + k + n * k) * 4, "ms_per_step": t_pipe * 1e3,
               "pipelined": "Plan.prefetch(A) of step i+1 issued before Plan.run of step i "
                            "(rsvd_plan_prefetch); one H2D copy of A and one read-back of U, S, V per step",
               "median_step_ms": statistics.median(a + b for a, b in host_pipe),
               "host_ms_run_and_readback": host_pipe,
               "serial": {"value": ws / t_e2e, "ms_per_step": t_e2e * 1e3,
                          "median_step_ms": statistics.median(a + b for a, b in host_split),
                          "host_ms_run_and_readback": host_split,
                          "note": "each step's copy issued by its own Plan.run"},
               "stages_ms_untimed_call": {kk: round(vv, 3) for kk, vv in plan_h.stage_ms().items()
                                          if kk in ("h2d", "total")}}
        plan_h.close()
        del A_host

    # --- other precisions of the same workload for comparison (not timed above) ----
    extra = {}
    results = {prec: (ms_per_step, U.double().cpu().numpy(), S_head, V.double().cpu().numpy())}
    if not args.no_compare:
        def timed_path(pr):
            pl = g.Plan(m, n, k, p, q, w.seed, prec=pr, mb=w.tile, nb=w.tile)
            U2, S2, V2 = pl.run(A)
            for _ in range(2):
                pl.run(A, U2, S2, V2)
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(5):
                pl.run(A, U2, S2, V2)
            f1.record(stream)
            torch.cuda.synchronize()
            ms_p = f0.elapsed_time(f1) / 5
            out = (ms_p, U2.double().cpu().numpy(), S2.double().cpu().numpy(), V2.double().cpu().numpy())
            pl.close()
            return out
        for pr in ("fp32", "bf16x3", "bf16", "fp8"):
            if pr not in results:
                results[pr] = timed_path(pr)
        ms32, S32 = results["fp32"][0], results["fp32"][2]
        extra["paths"] = {
            pr: {"ms_per_step": res[0], "rsvd_per_s": 1e3 / res[0], "speedup_vs_fp32": ms32 / res[0],
                 "sigma_rel_diff_vs_fp32_path": float(np.max(np.abs(res[2] - S32) / S32))}
            for pr, res in results.items()}
        extra["paths"]["fp8"]["note"] = "E4M3 copy of A with per-4096^2-tile scales, BF16 panel, split-BF16 B^T"
        extra["paths"]["bf16x3"]["note"] = "every A-pass in split BF16 (A = hi + lo, X = hi + lo, three products)"

    # --- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) -----------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        sample = A[:ORACLE_SAMPLE_ROWS].cpu().numpy()
        t = oracle_sample_seconds(sample, w) * (m / ORACLE_SAMPLE_ROWS)
        cpu = {"value": 1.0 / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {ORACLE_SAMPLE_ROWS} of {m} rows, full n={n}, k, p, q; time x {m / ORACLE_SAMPLE_ROWS:g}"}

    # --- accuracy of every timed path against the FP64 oracle on the same A -----------
    if rank == 0 and ws == 1 and not args.no_accuracy and not args.no_compare:
        extra["accuracy_vs_oracle"], extra["matched_accuracy"] = accuracy_vs_oracle(w, A, results)

    if rank == 0:
        stages = {kk: vv / args.steps for kk, vv in stage_sum.items() if kk != "apass_calls"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"bf16": "bf16", "bf16x3": "bf16x3",
                                                                  "fp32": "f32", "fp8": "fp8e4m3"}[prec],
            "data": DATA_NOTE,
            "config": _config(w, prec, ws),
            "roofline": roof, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
            "cpu_baseline": cpu, "stages_ms_per_step": stages,
            "apass_calls_per_step": apass_calls / args.steps,
        }
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_rsvd_rows(args):
    """The dense workload's recipe and BF16 plan at --m x --n (default
    25000 x 20000): a small whole-rSVD target for kernel profiling."""
    import torch
    import paper_1907_06470_gb300 as g
    from synth import WORKLOADS, prescribed_dense_torch
    g.load()
    w = WORKLOADS[WORKLOAD]
    m, n = args.m, args.n
    A = prescribed_dense_torch(m, n, _spectrum(n, w.noise_seed), w.data_seed, device="cuda")
    plan = g.Plan(m, n, w.k, w.p, w.q, w.seed, prec=args.prec, mb=w.tile, nb=w.tile)
    U, S, V = plan.run(A)
    for _ in range(max(0, args.warmup - 1)):
        plan.run(A, U, S, V)
    torch.cuda.synchronize()
    plan.set_profiling(True)
    stages = {}
    for _ in range(args.steps):
        plan.run(A, U, S, V)
        for key, val in plan.stage_ms().items():
            stages[key] = stages.get(key, 0.0) + val / args.steps
    torch.cuda.synchronize()
    print(json.dumps({"mode": "rsvd_rows", "m": m, "n": n, "k": w.k, "p": w.p, "q": w.q, "prec": args.prec,
                      "steps": args.steps, "stages_ms_per_rsvd": stages, "info": plan.info()}))
    return 0


def run_backward(args):
    """The differentiable workload (FP32 A 20000 x 10000, s_i = 10 * 0.95^(i-1),
    k=64, p=16, q=2): forward rSVD and the adjoint pass dA (rsvd_backward) for
    seeded cotangents of the workload's loss sum_i w_i s_i + ||U_k^T X||_F^2."""
    import torch
    import paper_1907_06470_gb300 as g
    from synth import WORKLOADS, prescribed_dense_torch
    g.load()
    w = WORKLOADS["dense_fp32_20000x10000_diff"]
    m, n, k = w.m, w.n, w.k
    s = 10.0 * 0.95 ** np.arange(n)
    A = prescribed_dense_torch(m, n, s, w.data_seed, device="cuda")
    plan = g.Plan(m, n, k, w.p, w.q, w.seed, prec="fp32", mb=w.tile, nb=w.tile)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.noise_seed)
    X = torch.randn(m, 32, generator=gen, device="cuda")
    wv = torch.rand(k, generator=gen, device="cuda")
    U, S, V = plan.run(A)

    def cotangents(U):
        # d/dU ||U^T X||_F^2 = 2 X X^T U; d/dS sum w_i s_i = w
        return 2.0 * X @ (X.T @ U), wv, None

    for _ in range(args.warmup):
        plan.run(A, U, S, V)
        dU, dS, dV = cotangents(U)
        plan.backward(U, S, V, dU, dS, dV)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd_ms = bwd_ms = 0.0
    for _ in range(args.steps):
        e[0].record()
        plan.run(A, U, S, V)
        dU, dS, dV = cotangents(U)
        e[1].record()
        dA = plan.backward(U, S, V, dU, dS, dV)
        e[2].record()
        torch.cuda.synchronize()
        fwd_ms += e[0].elapsed_time(e[1]) / args.steps
        bwd_ms += e[1].elapsed_time(e[2]) / args.steps
    peaks, peak_kind = _peaks()
    # dA = L R^T with L = [U M + (I - U U^T) dU S^-1, U S^-1] (m x 2k) and
    # R = [V, (I - V V^T) dV] (n x 2k): a product of 2 m n 2k flop, on the
    # tensor cores in split BF16 (three products), which dominates; dA is
    # written once (4 m n bytes): the pass is bound by that write
    bwd_flops = 2.0 * m * n * 2 * k
    bwd_bytes = 4 * m * n + 4 * (2 * m + n) * 2 * k
    achieved = bwd_bytes / (bwd_ms / 1e3) / 1e9
    print(json.dumps({
        "mode": "backward", "workload": w.name, "m": m, "n": n, "k": k, "p": w.p, "q": w.q, "prec": "fp32",
        "steps": args.steps, "forward_ms": fwd_ms, "backward_ms": bwd_ms,
        "backward_roofline": {"bound": "hbm", "bytes": bwd_bytes, "achieved": achieved,
                              "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                              "frac": achieved / float(peaks["hbm_gbs"]),
                              "peak_source": f"hbm_gbs ({peak_kind})",
                              "tensor_TFLOPs_split_bf16": 3 * bwd_flops / (bwd_ms / 1e3) / 1e12,
                              "note": "the whole rsvd_backward call (the k x k algebra, the two panels and the "
                                      "rank-2k product) against the dA write"},
        "dA_fro": float(torch.linalg.norm(dA)), "data": "synthetic"}))
    return 0


def run_apass_only(args):
    """Forward and transposed A-passes alone on a random FP32 matrix (a small,
    quick target for kernel profiling and tuning)."""
    import torch
    import paper_1907_06470_gb300 as g
    g.load()
    m, n, r = args.m, args.n, args.r
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    A = torch.randn(m, n, generator=gen, device="cuda")
    X = torch.randn(n, r, generator=gen, device="cuda")
    Yt = torch.randn(m, r, generator=gen, device="cuda")
    Y = torch.empty(m, r, device="cuda")
    Z = torch.empty(n, r, device="cuda")
    for _ in range(args.warmup):
        g.apass(A, X, False, args.prec, out=Y)
        g.apass(A, Yt, True, args.prec, out=Z)
    torch.cuda.synchronize()
    out = {}
    for name, (src, dst, tr) in {"forward": (X, Y, False), "transposed": (Yt, Z, True)}.items():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.apass(A, src, tr, args.prec, out=dst)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nbytes = m * n * 4 + (m + n) * r * 4
        out[name] = {"ms": ms, "GB/s": nbytes / ms / 1e6, "TFLOP/s": 2.0 * m * n * r / ms / 1e9}
    print(json.dumps({"mode": "apass", "m": m, "n": n, "r": r, "prec": args.prec, "steps": args.steps,
                      "note": "each call includes the panel conversion and a stream sync", **out}))
    return 0


def run_out_of_core(args):
    """The out-of-core workload's recipe (exp(-i/50) spectrum + 1e-3 floor,
    k=200, p=40, q=2, 8192^2 tiles), with m scaled to --ooc-rows so that A fits
    the host's pinned memory, streamed under a device cap of --ooc-cap-gb."""
    import torch
    import paper_1907_06470_gb300 as g
    from synth import WORKLOADS, LowRankPlusNoise
    g.load()
    w = WORKLOADS["dense_fp32_600000x100000_ooc"]
    m, n = args.ooc_rows, w.n
    gen = LowRankPlusNoise(m, n, 2000, 50.0, 1e-3, w.data_seed, w.noise_seed)
    A_host = torch.empty(m, n, dtype=torch.float32, pin_memory=True)
    blk = 8192
    for r0 in range(0, m, blk):
        A_host[r0:r0 + blk].copy_(gen.rows(r0, min(blk, m - r0)))
    del gen
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    cap = int(args.ooc_cap_gb * (1 << 30))
    tile = args.ooc_tile
    plan = g.Plan(m, n, w.k, w.p, w.q, w.seed, mem_cap=cap, prec=args.prec, mb=tile, nb=tile, fused=args.fused)
    plan.set_profiling(True)
    U, S, V = plan.run(A_host)
    torch.cuda.synchronize()
    times, stages = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        plan.run(A_host, U, S, V)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        stages.append(plan.stage_ms())
    st = plan.stream_stats()
    apass_ms = stages[-1]["apass_fwd"] + stages[-1]["apass_trans"] + stages[-1].get("sweep", 0.0)
    link = st["h2d_bytes"] / (apass_ms / 1e3) / 1e9
    print(json.dumps({
        "mode": "out_of_core", "workload": w.name, "m": m, "n": n, "k": w.k, "p": w.p, "q": w.q,
        "tile": tile if tile else "full-width row panels (planner default)", "prec": args.prec,
        "fused_sweeps": bool(args.fused),
        "passes_over_A": (w.q + 2) if args.fused else (2 * w.q + 2),
        "host_bytes": m * n * 4, "device_cap_bytes": cap,
        "ms_per_rsvd": 1e3 * sum(times) / len(times), "stream": st,
        "h2d_bytes_per_rsvd": st["h2d_bytes"], "apass_ms_per_rsvd": apass_ms,
        "link_GBps_during_apasses": link, "stages_ms": stages[-1],
        "note": "link GB/s = bytes copied host-to-device / time of the A-pass stages (copies overlap "
                "the tile products); compare with the pinned cudaMemcpyAsync rate of the same box",
    }))
    return 0


def run_sparse(args):
    """The sparse workload's recipe (rank-size row lengths, Zipf(1.0) columns,
    k=300, p=50, q=3) with A and the CSR of A^T resident in HBM; sizes scaled by
    --csr-m/--csr-n/--csr-nnz (default: the full 5e6 x 1e6 matrix, 5e8 entries).
    The transpose is built once by the library's host transpose (untimed)."""
    import torch
    import paper_1907_06470_gb300 as g
    from synth import WORKLOADS, zipf_csr_torch
    g.load()
    w = WORKLOADS["csr_fp32_5000000x1000000"]
    m, n, nnz = args.csr_m, args.csr_n, args.csr_nnz
    k, p, q = w.k, w.p, w.q
    t0 = time.perf_counter()
    rp, ci, v = zipf_csr_torch(m, n, nnz, w.data_seed, device="cuda")
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    nnz = int(rp[-1].item())
    streamed = args.csr_cap_gb > 0 or args.csr_resident_gb >= 0
    pin = (lambda t: t.pin_memory()) if streamed else (lambda t: t)
    A_host = torch.sparse_csr_tensor(pin(rp.cpu()), pin(ci.cpu()), pin(v.cpu()), size=(m, n))
    t0 = time.perf_counter()
    At_host = g.csr_transpose(A_host)
    t_tr = time.perf_counter() - t0
    if streamed:
        # out of core: the CSR of A and of A^T stay in pinned host memory and
        # their row blocks are streamed under the device cap
        A = A_host
        At = torch.sparse_csr_tensor(*(x.pin_memory() for x in (At_host.crow_indices(), At_host.col_indices(),
                                                                  At_host.values())), size=(n, m))
        del rp, ci, v
    else:
        A = torch.sparse_csr_tensor(rp, ci, v, size=(m, n))
        At = At_host.to("cuda")
        del A_host
    torch.cuda.empty_cache()
    cap = int(args.csr_cap_gb * (1 << 30))
    if args.csr_resident_gb >= 0:
        # the plan's own workspace plus this many GB for CSR blocks
        import ctypes as C
        from paper_1907_06470_gb300 import _lib
        o = _lib.RsvdOpts(prec=_lib.PREC[args.csr_prec], refine=1, mb=0, nb=0, n_slots=2,
                          dtype=_lib.DTYPE["f32"], kind=_lib.CSR)
        out = C.c_size_t()
        _lib.check(g.load().rsvd_plan_min_cap(m, n, k, p, C.byref(o), C.byref(out)))
        cap = out.value + int(args.csr_resident_gb * (1 << 30))
    plan = g.Plan(m, n, k, p, q, w.seed, prec=args.csr_prec, kind="csr", mem_cap=cap)
    plan.set_profiling(True)
    U, S, V = plan.run(A, At=At)
    torch.cuda.synchronize()
    for _ in range(max(0, args.warmup - 1)):
        plan.run(A, U, S, V, At=At)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    stage_sum = {}
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = g.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run(A, U, S, V, At=At)
        for key, val in plan.stage_ms().items():
            stage_sum[key] = stage_sum.get(key, 0.0) + val
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = g.kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    r = k + p
    calls = stage_sum.get("apass_calls", 0) / args.steps
    fwd_calls, tr_calls = q + 1, q + 1
    fwd_ms = stage_sum.get("apass_fwd", 0.0) / args.steps / fwd_calls
    tr_ms = stage_sum.get("apass_trans", 0.0) / args.steps / tr_calls
    ldr = (r + 3) // 4 * 4

    def algo_bytes(M, K):
        # entries (column index + value), row offsets, the panel read once, the output written once
        return nnz * 8 + (M + 1) * 4 + K * ldr * 4 + M * ldr * 4

    peaks, peak_kind = _peaks()
    # bytes per gathered panel value of the forward passes (all range-finder
    # passes: compact for BF16 / BF16X3 plans)
    bpv = {"fp32": 4, "bf16x3": 3, "bf16": 2}[args.csr_prec]
    fb = algo_bytes(m, n)
    tb = algo_bytes(n, m)
    roof = {"bound": "hbm", "kernel": "spmm_csr_vec_kernel (forward A-pass)",
            "achieved": fb / (fwd_ms / 1e3) / 1e9, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "peak_source": f"hbm_gbs ({peak_kind})", "algorithmic_bytes_per_launch": fb,
            # the gathers hit L2 at a rate that depends on the size: a smaller
            # capture does not scale, so no traffic figure for this kernel
            "avg_launch_ms": fwd_ms, "traffic": None,
            "gathered_panel_bytes_per_launch": nnz * ldr * bpv,
            "gather_GBps": nnz * ldr * bpv / (fwd_ms / 1e3) / 1e9}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # The pass is bound by the gathers of panel rows (one ldr-float row per
    # entry), not by A's bytes: measure what the same kernel gathers per second
    # when the panel is L2-resident and when every gather misses, on synthetic
    # CSRs with uniform columns (1e8 entries, rows of 128), and rate the
    # workload's gather rate against the L2-resident one.
    ceil = {}
    for name, ncols in (("l2_resident", 40000), ("dram", n)):
        Lr = 128
        mr = 100_000_000 // Lr
        gg = torch.Generator(device="cuda")
        gg.manual_seed(77)
        cci = torch.randint(0, ncols, (mr * Lr,), generator=gg, device="cuda", dtype=torch.int32)
        crp = torch.arange(0, mr * Lr + 1, Lr, device="cuda", dtype=torch.int32)
        Asyn = torch.sparse_csr_tensor(crp, cci, torch.ones(mr * Lr, device="cuda"), size=(mr, ncols))
        Xs = torch.randn(ncols, ldr, generator=gg, device="cuda")[:, :r]
        Ys = torch.empty(mr, ldr, device="cuda")[:, :r]
        g.apass(Asyn, Xs, out=Ys)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(3):
            g.apass(Asyn, Xs, out=Ys)
        c1.record()
        torch.cuda.synchronize()
        ceil[name] = mr * Lr * ldr * 4 / (c0.elapsed_time(c1) / 3 / 1e3) / 1e12
        del Asyn, Xs, Ys, cci, crp
        torch.cuda.empty_cache()
    roof["gather_roofline"] = {
        "achieved_TBps": roof["gather_GBps"] / 1e3, "l2_resident_TBps": ceil["l2_resident"],
        "all_miss_TBps": ceil["dram"], "frac_of_l2_resident": roof["gather_GBps"] / 1e3 / ceil["l2_resident"],
        "how": "the same SpMM kernel on synthetic CSRs, 1e8 entries, rows of 128, uniform columns over 40000 "
               "(panel in L2) or over n (panel far larger than L2)"}
    # the other panel precisions on the same matrix (in core): time per rSVD
    # and per pass, and the top-k singular values against the FP32 plan's
    paths = {}
    if not args.no_compare and not streamed:
        ref_S = None
        for pp in ("fp32", "bf16x3", "bf16"):
            if pp == args.csr_prec:
                Sp, ms_p, f_p, t_p = S, ms, fwd_ms, tr_ms
            else:
                pl = g.Plan(m, n, k, p, q, w.seed, prec=pp, kind="csr")
                pl.set_profiling(True)
                Up, Sp, Vp = pl.run(A, At=At)
                torch.cuda.synchronize()
                q0 = torch.cuda.Event(enable_timing=True)
                q1 = torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                pl.run(A, Up, Sp, Vp, At=At)
                q1.record(stream)
                torch.cuda.synchronize()
                sm = pl.stage_ms()
                ms_p = q0.elapsed_time(q1)
                f_p, t_p = sm["apass_fwd"] / fwd_calls, sm["apass_trans"] / tr_calls
                pl.close()
                del Up, Vp
                torch.cuda.empty_cache()
            Sv = Sp[:k].double().cpu()
            if pp == "fp32":
                ref_S = Sv
            paths[pp] = {"ms_per_rsvd": ms_p, "forward_pass_ms": f_p, "transposed_pass_ms_mean": t_p,
                         "panel_bytes_per_value": {"fp32": 4, "bf16x3": 3, "bf16": 2}[pp],
                         "sigma_rel_diff_vs_fp32_plan": None if ref_S is None else
                         float(((Sv - ref_S).abs() / ref_S).max())}
        paths["note"] = ("range-finder passes gather the panel at 4 / 3 / 2 bytes per value; the final "
                         "B^T = A^T Q gathers FP32 in every plan; the BF16X3 plan meets the FP32 bars against "
                         "the FP64 oracle at the scaled size (tests/test_gpu_sparse.py)")
    link = None
    if streamed:
        st = plan.stream_stats()
        ap_ms = stage_sum.get("apass_fwd", 0.0) / args.steps + stage_sum.get("apass_trans", 0.0) / args.steps
        link = {"h2d_bytes_per_rsvd": st["h2d_bytes"], "tiles_streamed_per_pass_pair": st["tiles_streamed_per_pass"],
                "tiles_resident": st["tiles_resident"], "device_cap_bytes": cap,
                "link_GBps_during_apasses": st["h2d_bytes"] / (ap_ms / 1e3) / 1e9,
                "note": "bytes copied host-to-device per rSVD over the time of the A-pass stages (copies overlap "
                        "the products); compare with the pinned copy rate of the box (211.7 GB/s measured)"}
    print(json.dumps({
        "mode": "csr", "workload": w.name if (m, n) == (w.m, w.n) else f"{w.name} scaled to {m}x{n}",
        "out_of_core": link,
        "m": m, "n": n, "nnz": nnz, "k": k, "p": p, "q": q, "prec": args.csr_prec, "steps": args.steps,
        "ms_per_rsvd": ms, "rsvd_per_s": 1e3 / ms, "apass_calls_per_rsvd": calls,
        "forward_pass_ms": fwd_ms, "transposed_pass_ms": tr_ms,
        "transposed_GBps_algorithmic": tb / (tr_ms / 1e3) / 1e9,
        "stages_ms_per_rsvd": {kk: vv / args.steps for kk, vv in stage_sum.items() if kk != "apass_calls"},
        "roofline": roof, "clocks": clocks, "gpu_launches": launches, "paths": paths or None,
        "setup_s": {"generate_on_gpu": t_gen, "host_transpose": t_tr},
        "S_head": [float(x) for x in S[:4].cpu()],
    }))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32", "bf16x3", "fp8"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the full-size oracle comparison")
    ap.add_argument("--mode", default="rsvd", choices=["rsvd", "apass", "ooc", "csr", "rsvd_rows", "backward"])
    ap.add_argument("--csr-m", type=int, default=5_000_000)
    ap.add_argument("--csr-n", type=int, default=1_000_000)
    ap.add_argument("--csr-nnz", type=int, default=500_000_000)
    ap.add_argument("--csr-cap-gb", type=float, default=0.0,
                    help="device cap for the sparse workload: > 0 streams the host CSR out of core")
    ap.add_argument("--csr-prec", default="fp32", choices=["fp32", "bf16x3", "bf16"],
                    help="sparse workload: panel precision of the range-finder passes")
    ap.add_argument("--csr-resident-gb", type=float, default=-1.0,
                    help=">= 0: stream the host CSR under a cap of the plan's minimum plus this many GB")
    ap.add_argument("--ooc-rows", type=int, default=150000)
    ap.add_argument("--ooc-cap-gb", type=float, default=16.0)
    ap.add_argument("--ooc-tile", type=int, default=0, help="square tile edge (0: planner default)")
    ap.add_argument("--fused", action="store_true", help="out-of-core mode: fused power sweeps (q + 2 passes)")
    ap.add_argument("--m", type=int, default=25000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--r", type=int, default=120)
    args = ap.parse_args()
    if args.mode == "rsvd_rows":
        return run_rsvd_rows(args)
    if args.mode == "backward":
        return run_backward(args)
    if args.mode == "apass":
        return run_apass_only(args)
    if args.mode == "ooc":
        return run_out_of_core(args)
    if args.mode == "csr":
        return run_sparse(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
