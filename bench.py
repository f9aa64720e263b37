"""Benchmark of the sparse Tucker hot path on GB300 (one JSON line on rank 0).

Workload (default): a 1000 x 1000 x 1000 sparse tensor with 1e7 nonzeros at distinct uniform
coordinates, values U(0,1), core 50 x 50 x 50; one step = CSF build + HO-SVD + 10 passes each of
HOOI, SP and MP in FP64 (the stop test disabled so every step does the same work).  The metric
is passes ("sweeps") per second: 31 per step (HO-SVD counts as one pass).

  value       device-resident: the COO tensor is in HBM before the timed region
  e2e         through the public C ABI with host buffers: pinned-host COO in, factors/core out
  mixed       the same step in the mixed form (FP32 projections, tensor-core Gram), its speedup
              and largest fit difference against the FP64 form
  roofline    dominant kernel, achieved = algorithmic FLOPs / its event-timed device time
  cpu_baseline  the FP64 oracle on this host's cores, on a bounded sample of the workload

--impl reference times the oracle itself (CPU) on the same workload and metric.
--batched-leg (256 small tensors), --precision-leg (2000^3, core 100^3, FP64 vs mixed) and
--profile-leg fp64|mixed (one form only, for profiler captures) print their own lines.
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
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # nominal: SMs x FP32 lanes x 2 x max clock


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
        with open(self.path) as f:
            return parse_clocks(f)


def parse_clocks(lines):
    """Summary of nvidia-smi samples (ClockSampler.QUERY, csv, no header, no units): median SM
    clock under load, the maximum SM clock, and the throttle reasons seen active."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
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
        # NCCL between the GPUs of a node; gloo without a GPU or when BENCH_DIST_BACKEND says
        # so (the CPU tests of the multi-rank path).  Ranks only meet in barriers and the max
        # of their timings.
        backend = os.environ.get("BENCH_DIST_BACKEND") or (
            "nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(rank):
    from paper_0711_2023_gb300 import synth
    X = synth.random_sparse_tensor(DIMS, NNZ, synth.config_seed(1 + 1000 * rank))
    C_raw = synth.uniform_matrix(DIMS[2], CORE[2], synth.config_seed(2 + 1000 * rank))
    return X, C_raw


def run_job(tk, make_tensor, C_raw, out, precision="fp64"):
    """One step: CSF build + HO-SVD + HOOI/SP/MP x SWEEPS.  Returns (fits, sweeps)."""
    T = make_tensor()
    fits = {}
    pr = precision
    fits["hosvd"] = tk.tucker_hosvd(T, CORE, precision=pr, out=out)["fit"]
    fits["hooi"] = tk.tucker_hooi(T, CORE, tol=-np.inf, max_iter=SWEEPS, precision=pr,
                                  out=out)["fit"]
    fits["sp"] = tk.tucker_sp(T, CORE, C_raw, tol=-np.inf, max_iter=SWEEPS, precision=pr,
                              out=out)["fit"]
    fits["mp"] = tk.tucker_mp(T, CORE, tol=-np.inf, max_iter=SWEEPS, precision=pr,
                              out=out)["fit"]
    T.close()
    return fits, 1 + 3 * SWEEPS


def timed_region(tk, torch, world, local, steps, make_tensor, C_raw, l2buf, precision,
                 profile=False):
    """Device-timed steps.  With profile=True the library also records CUDA events around its
    kernels (which costs host time per launch, so the headline numbers come from unprofiled
    steps).  Returns (total_ms, passes, fits, launches, clocks, per-kernel profile)."""
    clocks = ClockSampler(local)
    tk.tucker_profile_enable(profile)
    launches0 = tk.tucker_launch_count()
    stream = torch.cuda.current_stream()
    total_ms, passes, fits = 0.0, 0, None
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(steps):
        flush_l2(l2buf)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fits, p = run_job(tk, make_tensor, C_raw, "device", precision)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        passes += p
    torch.cuda.synchronize()
    barrier(world)
    launches = tk.tucker_launch_count() - launches0
    clk = clocks.stop()
    prof = {}
    for name in (KERNELS + STAGES if profile else ()):
        n, ms, fl, by = tk.tucker_profile_query(name)
        if n:
            prof[name] = {"launches": n, "ms": ms, "flops": fl, "bytes": by}
    counters = {}
    for name in (COUNTERS if profile else ()):
        n, _, total, _ = tk.tucker_profile_query(name)
        counters[name] = {"count": n, "sum": total}
    prof["counters"] = counters
    tk.tucker_profile_enable(False)
    return total_ms, passes, fits, launches, clk, prof


def kernels_only(prof):
    return {k: v for k, v in prof.items() if k not in STAGES and k != "counters"}


KERNELS = ("syrk_f64", "gram_bf16x3", "ttmc_f64", "ttmc_mixed", "slice_proj_f64",
           "slice_proj_mixed", "unfold_gram_f64", "gemm_nn_f64", "gemm_nn_f32", "gemm_tn_f64",
           "chol_f64", "jacobi_f64", "csf_build")
STAGES = ("eig_topk", "syev_refined", "syev_jacobi32")   # spans that contain many of the kernels above
COUNTERS = ("eig_outer", "syev_steps", "syev_fp32_sweeps", "syev_fallback")   # iteration counts of the eigensolver


# DRAM traffic over algorithmic bytes per launch, from one ncu capture of each kernel on the
# 500^3 workload (dram__bytes_read.sum + dram__bytes_write.sum; profiles/syrk_f64_500cube_hooi.md
# and profiles/gram_bf16x3_500cube.md).  The traffic of a bench launch is this ratio times its
# algorithmic bytes: the traffic of both kernels grows with the rows x K of the projection read.
NCU_TRAFFIC_RATIO = {
    "syrk_f64": 10.034e6 / (8.0 * 500 * 2500 + 8.0 * 500 * 500),
    "gram_bf16x3": 105.01e6 / (4.0 * 500 * 50000 + 8.0 * 500 * 500),
}


def roofline_of(prof, name, total_ms, bound, peak, unit, peak_source, per="flops"):
    d = prof.get(name)
    if not d:
        return None
    per_launch_ms = d["ms"] / d["launches"]
    work = (d["flops"] if per == "flops" else d["bytes"]) / d["launches"]
    scale = 1e12 if unit == "TFLOP/s" else 1e9
    achieved = work / (per_launch_ms * 1e-3) / scale if per_launch_ms else 0.0
    ratio = NCU_TRAFFIC_RATIO.get(name)
    traffic = ratio * d["bytes"] / d["launches"] if ratio else None
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic,
            "traffic_note": ("bytes per launch: ncu DRAM bytes / algorithmic bytes of a 500^3 "
                             "capture x this launch's algorithmic bytes") if ratio else None,
            "algorithmic_bytes": d["bytes"] / d["launches"], "peak_source": peak_source,
            "share_of_step": d["ms"] / total_ms, "launches": d["launches"]}


def ttmc_rates(pr, name, flop_peak, hbm_gbs):
    """Algorithmic GB/s and TFLOP/s of one TTMc form from a profile, with their fractions."""
    d = pr.get(name)
    if not d or not d["ms"]:
        return None
    secs = d["ms"] * 1e-3
    gbs, tfs = d["bytes"] / secs / 1e9, d["flops"] / secs / 1e12
    return {"kernel": name, "launches": d["launches"], "ms_per_launch": d["ms"] / d["launches"],
            "algorithmic_gbs": gbs, "frac_hbm": gbs / hbm_gbs if hbm_gbs else None,
            "tflops": tfs, "frac_alu": tfs / flop_peak,
            "note": "HOOI projection; at core 50 it does J_m J_o FMAs per fiber against 12 "
                    "bytes of index data, so it is bound by arithmetic and row gathers, not HBM"}


CPU_SAMPLE = "one HOOI pass (3 projections, Grams, eigensolves, core, fit) from the HO-SVD B, C"


def cpu_setup(X):
    """Untimed: the HO-SVD start of HOOI that the CPU sample continues from."""
    from oracle import tucker_oracle as O
    return [None] + [O.leading_eigvecs(O.unfolding_gram(X.dims, X.idx, X.val, n), CORE[n])[0]
                     for n in (1, 2)]


def cpu_sample(X, init):
    """The oracle on a bounded sample of the workload (one HOOI pass).  Returns (s, passes)."""
    from oracle import tucker_oracle as O
    t0 = time.perf_counter()
    O.hooi(X.dims, X.idx, X.val, CORE, -np.inf, 1, init=init)
    return time.perf_counter() - t0, 1


def run_reference(args, world, rank):
    if rank != 0:
        return
    X, _ = make_inputs(0)
    init = cpu_setup(X)
    for _ in range(args.warmup):
        cpu_sample(X, init)
    tot, passes = 0.0, 0
    for _ in range(args.steps):
        dt, p = cpu_sample(X, init)
        tot += dt
        passes += p
    value = passes / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "per step: " + CPU_SAMPLE},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": CPU_SAMPLE},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


def batched_leg(args):
    """The batched workload: 256 independent tensors (dims uniform in [30, 300], density
    log-uniform in [1%, 20%], core dims uniform in [4, 32]); one step = HOOI and MP, 10 passes
    each, mixed form, through tucker_hooi_batched / tucker_mp_batched.  Prints tensor-passes/s."""
    import torch
    from paper_0711_2023_gb300 import build, synth, tucker as tk
    build.build()
    cfgs = synth.batched_configs(args.batch_count, synth.config_seed(5))
    Ts, Js, nnz_total = [], [], 0
    for t, (dims, nnz, core) in enumerate(cfgs):
        X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(100 + t))
        nnz_total += X.nnz
        Ts.append(tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(),
                                          torch.from_numpy(X.val).cuda(), X.dims))
        Js.append(core)

    def step():
        tk.tucker_hooi_batched(Ts, Js, tol=-np.inf, max_iter=SWEEPS, precision="mixed")
        tk.tucker_mp_batched(Ts, Js, tol=-np.inf, max_iter=SWEEPS, precision="mixed")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    b.record(stream)
    b.synchronize()
    wall = time.perf_counter() - t0
    passes = args.steps * len(Ts) * 2 * SWEEPS
    # The plain FP64 path on the same tensors, one call at a time (a bounded sample: the first
    # 32 tensors), for the comparison in the same units.
    ns = min(32, len(Ts))
    t0 = time.perf_counter()
    for t in range(ns):
        tk.tucker_hooi(Ts[t], Js[t], tol=-np.inf, max_iter=SWEEPS, precision="fp64")
        tk.tucker_mp(Ts[t], Js[t], tol=-np.inf, max_iter=SWEEPS, precision="fp64")
    torch.cuda.synchronize()
    single = time.perf_counter() - t0
    print(json.dumps({"leg": "batched", "tensors": len(Ts), "nnz_total": nnz_total,
                      "value": passes / wall, "unit": "tensor-sweeps/s",
                      "ms_per_step": 1e3 * wall / args.steps, "steps": args.steps,
                      "warmup": args.warmup, "precision": "mixed",
                      "autotune": [tk.tucker_autotune_decision(i)
                                   for i in range(tk.tucker_autotune_count())],
                      "fp64_one_at_a_time": {"value": ns * 2 * SWEEPS / single,
                                             "unit": "tensor-sweeps/s",
                                             "sample": f"first {ns} tensors, HOOI + MP"},
                      "note": "wall clock around the batched calls (they synchronise)"}),
          flush=True)


def precision_leg(args):
    """The precision form's workload: 2000^3 with 4e7 uniform nonzeros, core 100^3; HOOI and MP
    for `--precision-passes` passes each, FP64 and mixed, on the same tensor (its orderings built
    once, outside the timing).  Prints sweeps/s of both forms and the largest fit difference."""
    import torch
    from paper_0711_2023_gb300 import build, synth, tucker as tk
    build.build()
    dims, nnz, core = (2000, 2000, 2000), 40_000_000, (100, 100, 100)
    X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(3))
    T = tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(), torch.from_numpy(X.val).cuda(),
                                X.dims)
    passes = args.precision_passes
    # untimed warm-up: builds the orderings and the mixed form's FP32 copies, tunes the kernels
    tk.tucker_hooi(T, core, tol=-np.inf, max_iter=1, precision="mixed")
    tk.tucker_mp(T, core, tol=-np.inf, max_iter=1, precision="mixed")
    res = {}
    for prec in ("fp64", "mixed"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = tk.tucker_hooi(T, core, tol=-np.inf, max_iter=passes, precision=prec)
        m = tk.tucker_mp(T, core, tol=-np.inf, max_iter=passes, precision=prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[prec] = {"sweeps_per_s": 2 * passes / dt, "seconds": dt,
                     "fit_hooi": h["fit_history"], "fit_mp": m["fit_history"]}
    dfit = max(abs(a - b) for k in ("fit_hooi", "fit_mp")
               for a, b in zip(res["fp64"][k], res["mixed"][k]))
    print(json.dumps({"leg": "precision", "workload": "2000^3, 4e7 uniform nonzeros, core 100^3, "
                      f"HOOI + MP {passes} passes each", "fp64": res["fp64"],
                      "mixed": res["mixed"],
                      "speedup": res["mixed"]["sweeps_per_s"] / res["fp64"]["sweeps_per_s"],
                      "max_abs_dfit": dfit, "unit": "sweeps/s",
                      "note": "wall clock around the calls (they synchronise)"}), flush=True)


def profile_leg(args):
    """One precision leg only (warm-up + timed steps), for profiler captures.  --profile-small
    uses a 500^3 tensor with 2.5e6 nonzeros and the same core (a few hundred MB on the device)."""
    import torch
    from paper_0711_2023_gb300 import build, tucker as tk
    global DIMS, NNZ
    if args.profile_small:
        DIMS, NNZ = (500, 500, 500), 2_500_000
    build.build()
    X, C_raw = make_inputs(0)
    d_idx = torch.from_numpy(X.idx).cuda()
    d_val = torch.from_numpy(X.val).cuda()
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    dev_tensor = lambda: tk.tucker_tensor_create(d_idx, d_val, X.dims)  # noqa: E731
    for _ in range(args.warmup):
        run_job(tk, dev_tensor, C_raw, "device", args.profile_leg)
    ms_plain, passes_plain, _, _, _, _ = timed_region(
        tk, torch, 1, 0, args.steps, dev_tensor, C_raw, l2buf, args.profile_leg)
    ms, passes, fits, launches, clk, prof = timed_region(
        tk, torch, 1, 0, args.steps, dev_tensor, C_raw, l2buf, args.profile_leg, profile=True)
    print(json.dumps({"leg": args.profile_leg, "value": passes_plain / (ms_plain / 1e3),
                      "unit": "sweeps/s", "ms_per_step": ms_plain / args.steps,
                      "ms_per_step_profiled": ms / args.steps, "gpu_launches": launches,
                      "fits": fits,
                      "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                      "share": round(v["ms"] / ms, 4)}
                                  for k, v in prof.items() if k != "counters"},
                      "eig_counters": prof["counters"]}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-leg", choices=["fp64", "mixed"], default=None,
                    help="run only warm-up + timed steps of one precision leg (for ncu captures) "
                         "and print a short summary line")
    ap.add_argument("--profile-small", action="store_true",
                    help="with --profile-leg: 500^3, 2.5e6 nonzeros instead of 1000^3, 1e7")
    ap.add_argument("--batched-leg", action="store_true",
                    help="time the batched workload (256 small tensors) instead")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--precision-leg", action="store_true",
                    help="time HOOI and MP in FP64 and mixed on 2000^3 / 4e7 / core 100^3")
    ap.add_argument("--precision-passes", type=int, default=2)
    args = ap.parse_args()

    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.profile_leg:
        profile_leg(args)
        return
    if args.batched_leg:
        batched_leg(args)
        return
    if args.precision_leg:
        precision_leg(args)
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

    # ---- device-resident timed region (FP64: the workload as configured) --------------------
    total_ms, passes, fits, launches, clk, _ = timed_region(
        tk, torch, world, local, args.steps, dev_tensor, C_raw, l2buf, "fp64")
    t_max = max_over_ranks(total_ms, world)
    value = passes * world / (t_max / 1e3)
    # one more step with the in-library kernel events on: the per-kernel breakdown and rooflines
    prof_ms, _, _, _, _, prof = timed_region(
        tk, torch, world, local, 1, dev_tensor, C_raw, l2buf, "fp64", profile=True)

    # ---- the same workload in the mixed-precision form -------------------------------------
    for _ in range(min(args.warmup, 1)):
        run_job(tk, dev_tensor, C_raw, "device", "mixed")
    mx_ms, mx_passes, mx_fits, mx_launches, mx_clk, _ = timed_region(
        tk, torch, world, local, args.steps, dev_tensor, C_raw, l2buf, "mixed")
    mx_value = mx_passes * world / (max_over_ranks(mx_ms, world) / 1e3)
    mx_prof_ms, _, _, _, _, mx_prof = timed_region(
        tk, torch, world, local, 1, dev_tensor, C_raw, l2buf, "mixed", profile=True)

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

    # ---- rooflines ---------------------------------------------------------------------------
    fp64_src = "nominal GB300 FP64 rate 1.25 TFLOP/s (no measured FP64 figure)"
    kp = kernels_only(prof)
    dom = max(kp, key=lambda k: kp[k]["ms"])
    roofline = roofline_of(prof, dom, prof_ms, "alu", FP64_PEAK_TFLOPS, "TFLOP/s", fp64_src)
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    mx_gram = roofline_of(mx_prof, "gram_bf16x3", mx_prof_ms, "tensor", bf16, "TFLOP/s",
                          f"{peak_src} bf16 sustained (cuBLAS), algorithmic FP32-equivalent "
                          "Gram FLOPs (the BF16x3 kernel issues 3x as many)")

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        secs, p = cpu_sample(X, cpu_setup(X))
        cpu = {"value": p / secs, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{CPU_SAMPLE}, same tensor: {p} pass in {secs:.1f} s"}

    def kern_table(pr, tot):
        return {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                    "share": round(v["ms"] / tot, 4)} for k, v in pr.items() if k != "counters"}

    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "passes_per_step": 1 + 3 * SWEEPS,
                   "l2": "flushed between steps (256 MB write); tensor 200 MB > L2",
                   "parallelism": f"replicas x{world}"},
        "fits": fits,
        "kernels": kern_table(prof, prof_ms),
        "profiled_step_ms": prof_ms,
        "eig_counters": prof["counters"],
        "ttmc": {"fp64": ttmc_rates(prof, "ttmc_f64", FP64_PEAK_TFLOPS, peaks.get("hbm_gbs")),
                 "mixed": ttmc_rates(mx_prof, "ttmc_mixed", FP32_PEAK_TFLOPS,
                                     peaks.get("hbm_gbs"))},
        "roofline": roofline,
        "mixed": {"value": mx_value, "unit": "sweeps/s", "ms_per_step": mx_ms / args.steps,
                  "speedup_vs_fp64": mx_value / value,
                  "max_abs_dfit_vs_fp64": max(abs(mx_fits[k] - fits[k]) for k in fits),
                  "fits": mx_fits, "kernels": kern_table(mx_prof, mx_prof_ms),
                  "profiled_step_ms": mx_prof_ms,
                  "eig_counters": mx_prof["counters"],
                  "roofline_gram": mx_gram, "gpu_launches": mx_launches, "clocks": mx_clk},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs"),
                  "bf16_tflops": peaks.get("bf16_tflops"),
                  "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained")},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
