"""Benchmark of the sparse Tucker hot path on GB300 (one JSON line on rank 0).

Workload (default): a 1000 x 1000 x 1000 sparse tensor with 1e7 nonzeros at distinct uniform
coordinates, values U(0,1), core 50 x 50 x 50; one step = CSF build + HO-SVD + 10 passes each of
HOOI, SP and MP in FP64 (the stop test disabled so every step does the same work).  The metric
is passes ("sweeps") per second: 31 per step (HO-SVD counts as one pass).

  value       device-resident: the COO tensor is in HBM before the timed region
  e2e         through the public C ABI with host buffers: pinned-host COO in, factors/core out
  roofline    dominant kernel, achieved = algorithmic FLOPs / its event-timed device time
  cpu_baseline  the FP64 oracle on this host's cores, on a bounded sample of the workload

--impl reference times the oracle itself (CPU) on the same workload and metric.
Multi-GPU (torchrun): each rank runs its own independent tensor (weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Tucker sweeps/s & TTMc HBM GB/s on 1 GB300, mixed vs FP64 at |Δfit|≤1e-4"
DIMS, NNZ, CORE, SWEEPS = (1000, 1000, 1000), 10_000_000, (50, 50, 50), 10
WORKLOAD = ("1000x1000x1000 sparse, 1e7 nnz (1% density, distinct uniform coords), "
            "values U(0,1), core 50x50x50; CSF build + HO-SVD + HOOI/SP/MP x 10 sweeps, FP64")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 SIMT peak of GB300: 1.25 TFLOP/s (nominal FP64 rate of the part; no measured figure).
FP64_PEAK_TFLOPS = 1.25


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = f"/tmp/tucker_clocks_{os.getpid()}.csv"
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(rank):
    from paper_0711_2023_gb300 import synth
    X = synth.random_sparse_tensor(DIMS, NNZ, synth.config_seed(1 + 1000 * rank))
    C_raw = synth.uniform_matrix(DIMS[2], CORE[2], synth.config_seed(2 + 1000 * rank))
    return X, C_raw


def run_job(tk, make_tensor, C_raw, out):
    """One step: CSF build + HO-SVD + HOOI/SP/MP x SWEEPS.  Returns (fits, sweeps)."""
    T = make_tensor()
    fits = {}
    fits["hosvd"] = tk.tucker_hosvd(T, CORE, out=out)["fit"]
    fits["hooi"] = tk.tucker_hooi(T, CORE, tol=-np.inf, max_iter=SWEEPS, out=out)["fit"]
    fits["sp"] = tk.tucker_sp(T, CORE, C_raw, tol=-np.inf, max_iter=SWEEPS, out=out)["fit"]
    fits["mp"] = tk.tucker_mp(T, CORE, tol=-np.inf, max_iter=SWEEPS, out=out)["fit"]
    T.close()
    return fits, 1 + 3 * SWEEPS


def cpu_sample(X, C_raw, repeats=1):
    """The oracle on a bounded sample of the workload: HO-SVD plus one pass each of HOOI
    (from HO-SVD's B, C), SP and MP.  Returns (seconds, passes)."""
    from oracle import tucker_oracle as O
    t0 = time.perf_counter()
    passes = 0
    for _ in range(repeats):
        h = O.hosvd(X.dims, X.idx, X.val, CORE)
        O.hooi(X.dims, X.idx, X.val, CORE, -np.inf, 1, init=[None, h["U"][1], h["U"][2]])
        O.sp(X.dims, X.idx, X.val, CORE, C_raw, -np.inf, 1)
        O.mp(X.dims, X.idx, X.val, CORE, -np.inf, 1)
        passes += 4
    return time.perf_counter() - t0, passes


def run_reference(args, world, rank):
    if rank != 0:
        return
    X, C_raw = make_inputs(0)
    for _ in range(args.warmup):
        cpu_sample(X, C_raw)
    tot, passes = 0.0, 0
    for _ in range(args.steps):
        dt, p = cpu_sample(X, C_raw)
        tot += dt
        passes += p
    value = passes / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "per step: HO-SVD + 1 pass each of HOOI, "
                       "SP, MP (4 passes)"},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "HO-SVD + 1 pass each of HOOI, SP, MP"},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_0711_2023_gb300 import build, tucker as tk
    build.build()
    tk._lib()
    peaks, peak_src = load_peaks()

    X, C_raw = make_inputs(rank)
    d_idx = torch.from_numpy(X.idx).cuda()
    d_val = torch.from_numpy(X.val).cuda()
    h_idx = torch.from_numpy(X.idx).pin_memory()
    h_val = torch.from_numpy(X.val).pin_memory()
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    dev_tensor = lambda: tk.tucker_tensor_create(d_idx, d_val, X.dims)  # noqa: E731
    host_tensor = lambda: tk.tucker_tensor_create(h_idx, h_val, X.dims)  # noqa: E731

    for _ in range(args.warmup):
        run_job(tk, dev_tensor, C_raw, "device")
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------------------------
    clocks = ClockSampler(local)
    tk.tucker_profile_enable(True)
    launches0 = tk.tucker_launch_count()
    stream = torch.cuda.current_stream()
    total_ms, passes, fits = 0.0, 0, None
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush_l2(l2buf)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fits, p = run_job(tk, dev_tensor, C_raw, "device")
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        passes += p
    torch.cuda.synchronize()
    barrier(world)
    launches = tk.tucker_launch_count() - launches0
    clk = clocks.stop()
    prof = {}
    for name in ("syrk_f64", "ttmc_f64", "slice_proj_f64", "unfold_gram_f64", "gemm_nn_f64",
                 "jacobi_f64", "csf_build"):
        n, ms, fl, by = tk.tucker_profile_query(name)
        prof[name] = {"launches": n, "ms": ms, "flops": fl, "bytes": by}
    tk.tucker_profile_enable(False)

    t_max = max_over_ranks(total_ms, world)
    value = passes * world / (t_max / 1e3)

    # ---- end to end through the C ABI with host buffers -------------------------------------
    e2e_ms, e2e_passes = 0.0, 0
    barrier(world)
    for _ in range(max(1, args.steps)):
        flush_l2(l2buf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, p = run_job(tk, host_tensor, C_raw, "host")
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_passes += p
    e2e_max = max_over_ranks(e2e_ms, world)
    e2e_value = e2e_passes * world / (e2e_max / 1e3)
    h2d = X.nnz * (3 * 4 + 8)
    d2h = 4 * (8 * (CORE[0] * CORE[1] * CORE[2] + sum(DIMS[a] * CORE[a] for a in range(3))))

    if rank != 0:
        return

    # ---- roofline of the dominant kernel ----------------------------------------------------
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    flops_per_launch = d["flops"] / max(d["launches"], 1)
    achieved_tflops = flops_per_launch / (per_launch_ms * 1e-3) / 1e12 if per_launch_ms else 0.0
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved_tflops,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "nominal GB300 FP64 rate (no measured FP64 figure)",
                "share_of_step": d["ms"] / total_ms}
    tt = prof["ttmc_f64"]
    ttmc_gbs = tt["bytes"] / (tt["ms"] * 1e-3) / 1e9 if tt["ms"] else None

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        secs, p = cpu_sample(X, C_raw)
        cpu = {"value": p / secs, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "HO-SVD + 1 pass each of HOOI (from HO-SVD B, C), SP, MP on the same "
                         f"tensor: {p} passes in {secs:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "passes_per_step": 1 + 3 * SWEEPS,
                   "l2": "flushed between steps (256 MB write); tensor 200 MB > L2",
                   "parallelism": f"replicas x{world}"},
        "fits": fits,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                        "share": round(v["ms"] / total_ms, 4)} for k, v in prof.items()},
        "ttmc_f64_gbs": ttmc_gbs,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs"),
                  "bf16_tflops": peaks.get("bf16_tflops")},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
