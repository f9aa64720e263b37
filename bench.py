"""Benchmark of the sparse Tucker hot path on GB300 (one JSON line on rank 0).

Workload (default): a 2000 x 2000 x 2000 sparse tensor with 4e7 nonzeros at distinct uniform
coordinates, values U(0,1), core 100 x 100 x 100.  Untimed set-up: the tensor is created in
device memory, its six mode orderings are built (reported as csf_build_ms) and the HO-SVD start
of B and C is computed once.  One step = one HOOI pass and one MP pass, each from that start
(2 sweeps; a sweep is the three factor updates, the core and the fit).

  value         FP64 sweeps/s, the tensor resident in HBM before the timed region
  mixed         the same step in the mixed form (FP32 projections, tensor-core Gram, FP64
                eigensolver/core/fit): sweeps/s, speed-up, largest |dfit| against the FP64 path
                and, for HOOI, against the oracle's own pass
  e2e           FP64, through the public C ABI from pinned host buffers: the COO tensor and the
                start factors copied in, the tensor and its orderings built, both passes run,
                cores and factors copied out, all inside the timed region
  batched       256 independent small tensors (dims 30..300, density 1..20 %, cores 4..32),
                HOOI + MP, 10 passes each, mixed, through the batched entry points
  streamed      MP with the tensor's orderings in pinned host memory, streamed to the GPU in
                chunks (the out-of-core form), one pass from the same start
  roofline      the FP64 step's dominant kernel, achieved = algorithmic FLOPs / its event-timed
                device time; roofline_gram in `mixed` does the same for the tensor-core Gram
  cpu_baseline  the FP64 oracle on this host's cores, on a bounded sample of the same step

--impl reference times the oracle itself on the same step, one piece of it per bench step (see
REFERENCE_UNITS).  --c2-leg (1000^3, all four methods), --batched-leg and --profile-leg print
their own lines.  Multi-GPU (torchrun): each rank runs its own independent tensor (weak
scaling, no collective on the data path).
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
DIMS, NNZ, CORE = (2000, 2000, 2000), 40_000_000, (100, 100, 100)
SWEEPS_PER_STEP = 2
WORKLOAD = ("2000x2000x2000 sparse, 4e7 nnz (0.5% density, distinct uniform coords), values "
            "U(0,1), core 100x100x100; step = one HOOI pass + one MP pass from the HO-SVD "
            "start of B, C (orderings built once, outside the step)")


def bench_config(world):
    """The `config` object; identical in both arms so that they name the same workload."""
    return {"workload": WORKLOAD, "sweeps_per_step": SWEEPS_PER_STEP,
            "l2": "inputs larger than L2 (one ordering ~0.5 GB) and L2 flushed between steps",
            "parallelism": f"replicas x{world}"}


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
    """The workload's tensor for this rank (ranks draw independent tensors)."""
    from paper_0711_2023_gb300 import synth
    return synth.random_sparse_tensor(DIMS, NNZ, synth.config_seed(2 + 1000 * rank))


def flush_l2(buf):
    buf.add_(1.0)


# ---- the GPU step -------------------------------------------------------------------------------

def run_step(tk, T, start, precision, out="device"):
    """One step: one HOOI pass and one MP pass from the start (B, C).  Returns the fits."""
    h = tk.tucker_hooi(T, CORE, tol=-np.inf, max_iter=1, precision=precision, init=start, out=out)
    m = tk.tucker_mp(T, CORE, tol=-np.inf, max_iter=1, precision=precision, init=start, out=out)
    return {"hooi": h["fit"], "mp": m["fit"]}


KERNELS = ("gram_ozaki", "gemm_ozaki", "eig_mv_ozaki", "eig_mv_ozaki3", "eig_tn_ozaki",
           "ttmc_ozaki", "ozaki_split", "syrk_f64", "gram_bf16x3", "gram_fused", "ttmc_f64",
           "ttmc_mixed", "slice_proj_f64", "slice_proj_mixed", "unfold_gram_f64", "gemm_nn_f64",
           "gemm_nn_f32", "gemm_tn_f64", "chol_f64", "jacobi_f64", "csf_build")
# DRAM bytes / algorithmic bytes of the 128 x 128 two-pass gram_ozaki kernel on the 500^3 MP Gram
# (one ncu capture): the second pass reads slices 0-3 again from DRAM
GRAM_OZAKI_DRAM_RATIO = (522.44e6 + 33.47e6) / (2 * 6 * 512 * 50048 + 16 * 128 * 128 * 140)
# FP64 products on the BF16 tensor cores (their FLOPs are the BF16 FLOPs issued)
OZAKI_KERNELS = ("gram_ozaki", "gemm_ozaki", "eig_mv_ozaki", "eig_mv_ozaki3", "eig_tn_ozaki",
                 "ttmc_ozaki")
# spans that contain several of the kernels above
STAGES = ("gram_f64_tc", "ttmc_f64_tc", "eig_topk", "eig_power", "eig_rr", "eig_lock",
          "eig_filter", "eig_orth", "syev_refined", "syev_jacobi32")
# eigensolver counters: iterations, and per solve its kernel launches and host synchronisations
COUNTERS = ("eig_outer", "syev_steps", "syev_fp32_sweeps", "syev_cluster_rotations",
            "syev_rotation_unconverged", "syev_fallback", "eig_launches", "eig_host_syncs")


def timed_region(tk, torch, world, local, steps, T, start, l2buf, precision, profile=False):
    """Device-timed steps (CUDA events on the launching stream; the library's calls return
    only when their results are written).  With profile=True the library also records CUDA
    events around its kernels (host work per launch, so the headline comes from unprofiled
    steps).  Returns (total_ms, fits, launches, clocks, per-kernel profile)."""
    clocks = ClockSampler(local)
    tk.tucker_profile_enable(profile)
    launches0 = tk.tucker_launch_count()
    stream = torch.cuda.current_stream()
    total_ms, fits = 0.0, None
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(steps):
        flush_l2(l2buf)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fits = run_step(tk, T, start, precision)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
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
    return total_ms, fits, launches, clk, prof


def kernels_only(prof):
    return {k: v for k, v in prof.items() if k not in STAGES and k != "counters"}


def kern_table(pr, tot):
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "share": round(v["ms"] / tot, 4)} for k, v in pr.items() if k != "counters"}


def roofline_of(prof, name, total_ms, bound, peak, unit, peak_source, traffic=None,
                traffic_note=None):
    d = prof.get(name)
    if not d:
        return None
    per_launch_ms = d["ms"] / d["launches"]
    work = d["flops"] / d["launches"]
    scale = 1e12 if unit == "TFLOP/s" else 1e9
    achieved = work / (per_launch_ms * 1e-3) / scale if per_launch_ms else 0.0
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
            "algorithmic_bytes": d["bytes"] / d["launches"], "peak_source": peak_source,
            "share_of_step": d["ms"] / total_ms, "launches": d["launches"]}


def ttmc_rates(pr, name, flop_peak, hbm_gbs, note):
    """Algorithmic GB/s and TFLOP/s of one projection kernel from a profile, with fractions."""
    d = pr.get(name)
    if not d or not d["ms"]:
        return None
    secs = d["ms"] * 1e-3
    gbs, tfs = d["bytes"] / secs / 1e9, d["flops"] / secs / 1e12
    return {"kernel": name, "launches": d["launches"], "ms_per_launch": d["ms"] / d["launches"],
            "algorithmic_gbs": gbs, "frac_hbm": gbs / hbm_gbs if hbm_gbs else None,
            "tflops": tfs, "frac_alu": tfs / flop_peak, "note": note}


# ---- the oracle on the same step ----------------------------------------------------------------
#
# One step of the workload (a HOOI pass and an MP pass from the start) takes the oracle about
# a minute on 8-16 host cores, so the CPU legs time it in units: the ten pieces below, in the
# order the two passes run them, each feeding its results to the next.  The time of a step is
# estimated as the sum over the ten unit types of their mean measured time.

REFERENCE_UNITS = (
    ("hooi", 0), ("hooi", 1), ("hooi", 2),            # HOOI factor updates (the last adds G, fit)
    ("mp_term", 0, 1), ("mp_term", 0, 2),             # MP slice sums of mode 0 (then its eig)
    ("mp_term", 1, 0), ("mp_term", 1, 2),
    ("mp_term", 2, 1), ("mp_term", 2, 0),
    ("mp_core",),                                     # MP core and fit
)
UNIT_KIND = {"hooi": "projection", "mp_term": "projection", "mp_core": "projection"}


class OracleStep:
    """State of the oracle's HOOI and MP passes run unit by unit (REFERENCE_UNITS)."""

    def __init__(self, X, start):
        from oracle import tucker_oracle as O
        self.O, self.X, self.start = O, X, start
        self.nX2 = O.norm2(X.val)
        self.fits = {}
        self.reset()

    def reset(self):
        self.Uh = [None, self.start[1], self.start[2]]
        self.Um = [None, self.start[1], self.start[2]]
        self.Mpart = None

    def run(self, unit):
        O, X = self.O, self.X
        if unit[0] == "hooi":
            n = unit[1]
            self.Uh[n], W = O.hooi_update(X.dims, X.idx, X.val, n, self.Uh, CORE[n])
            if n == 2:
                G = O.nmode_product_dense(W, 2, self.Uh[2].T)
                self.fits["hooi"] = O.fit_from_core(self.nX2, G)
        elif unit[0] == "mp_term":
            n, m = unit[1], unit[2]
            M = O.mp_term(X.dims, X.idx, X.val, n, m, self.Um[m])
            if self.Mpart is None:
                self.Mpart = M
            else:
                self.Um[n] = O.leading_eigvecs(self.Mpart + M, CORE[n])[0]
                self.Mpart = None
        else:
            G = O.core(X.dims, X.idx, X.val, self.Um)
            self.fits["mp"] = O.fit_from_core(self.nX2, G)
            self.reset()


def estimate_step_seconds(times):
    """Sum over the ten unit types of their mean time; a type not measured takes the mean of
    the measured units (every unit at this size is dominated by one sparse projection)."""
    means = {u: sum(t) / len(t) for u, t in times.items() if t}
    fill = sum(means.values()) / len(means)
    return sum(means.get(u, fill) for u in REFERENCE_UNITS), sorted(
        "/".join(str(x) for x in u) for u in REFERENCE_UNITS if u not in means)


def oracle_start(X, T, tk):
    """The HO-SVD start of B and C that both arms use (computed on the GPU when a library handle
    is given, else by the oracle)."""
    if T is not None:
        g = tk.tucker_hosvd(T, CORE)
        return [None, g["U"][1].cpu().numpy(), g["U"][2].cpu().numpy()]
    from oracle import tucker_oracle as O
    return [None] + [O.leading_eigvecs(O.unfolding_gram(X.dims, X.idx, X.val, n), CORE[n])[0]
                     for n in (1, 2)]


def run_reference(args, world, rank):
    """The oracle, as it stands, on the same step: each bench step runs the next unit of
    REFERENCE_UNITS (warm-up steps from the start of the cycle, then the timed steps from the
    start again), value = sweeps per step / the estimated seconds of a whole step."""
    if rank != 0:
        return
    X = make_inputs(0)
    start = oracle_start(X, None, None)
    st = OracleStep(X, start)
    for i in range(args.warmup):
        st.run(REFERENCE_UNITS[i % len(REFERENCE_UNITS)])
    st.reset()
    times = {u: [] for u in REFERENCE_UNITS}
    tot = 0.0
    for i in range(args.steps):
        u = REFERENCE_UNITS[i % len(REFERENCE_UNITS)]
        t0 = time.perf_counter()
        st.run(u)
        dt = time.perf_counter() - t0
        times[u].append(dt)
        tot += dt
    step_s, missing = estimate_step_seconds(times)
    value = SWEEPS_PER_STEP / step_s
    sample = ("per bench step one unit of the oracle's HOOI + MP pass pair (10 units: the 3 HOOI "
              "factor updates, the 6 MP slice sums with their eigensolves, the MP core and fit); "
              "value = 2 sweeps / sum over the unit types of their mean time"
              + (f"; not measured (filled with the mean unit): {missing}" if missing else ""))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(world),
            "estimated_s_per_oracle_step": step_s,
            "oracle_fits": st.fits,
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(X, start):
    """The oracle on a bounded sample of the step: its whole HOOI pass (3 units, which also
    gives the oracle's HOOI fit) and the first MP slice sum; the other units are estimated."""
    st = OracleStep(X, start)
    times = {u: [] for u in REFERENCE_UNITS}
    for u in REFERENCE_UNITS[:4]:
        t0 = time.perf_counter()
        st.run(u)
        times[u].append(time.perf_counter() - t0)
    step_s, missing = estimate_step_seconds(times)
    measured = sum(sum(t) for t in times.values())
    return {"value": SWEEPS_PER_STEP / step_s, "unit": "sweeps/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": (f"the oracle's HOOI pass from the same start and its first MP slice sum "
                       f"({measured:.1f} s); the other MP units estimated by the mean measured "
                       f"unit; value = 2 sweeps / estimated step ({step_s:.1f} s)")}, st.fits


# ---- legs ---------------------------------------------------------------------------------------

def batched_run(steps, warmup, count=256, sweeps=10):
    """The batched workload: `count` independent tensors (dims uniform in [30, 300], density
    log-uniform in [1%, 20%], core dims uniform in [4, 32]); one step = HOOI and MP, `sweeps`
    passes each, mixed form, through tucker_hooi_batched / tucker_mp_batched."""
    import torch
    from paper_0711_2023_gb300 import synth, tucker as tk
    cfgs = synth.batched_configs(count, synth.config_seed(5))
    Ts, Js, nnz_total = [], [], 0
    for t, (dims, nnz, core) in enumerate(cfgs):
        X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(100 + t))
        nnz_total += X.nnz
        Ts.append(tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(),
                                          torch.from_numpy(X.val).cuda(), X.dims))
        Js.append(core)

    def step():
        tk.tucker_hooi_batched(Ts, Js, tol=-np.inf, max_iter=sweeps, precision="mixed")
        tk.tucker_mp_batched(Ts, Js, tol=-np.inf, max_iter=sweeps, precision="mixed")
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    passes = steps * len(Ts) * 2 * sweeps
    # The plain FP64 path on the same tensors, one call at a time (a bounded sample: the first
    # 32 tensors), in the same unit.
    ns = min(32, len(Ts))
    torch.cuda.synchronize()
    a.record(stream)
    for t in range(ns):
        tk.tucker_hooi(Ts[t], Js[t], tol=-np.inf, max_iter=sweeps, precision="fp64")
        tk.tucker_mp(Ts[t], Js[t], tol=-np.inf, max_iter=sweeps, precision="fp64")
    b.record(stream)
    b.synchronize()
    single_ms = a.elapsed_time(b)
    for T in Ts:
        T.close()
    return {"tensors": len(Ts), "nnz_total": nnz_total, "value": passes / (ms / 1e3),
            "unit": "tensor-sweeps/s", "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "precision": "mixed",
            "fp64_one_at_a_time": {"value": ns * 2 * sweeps / (single_ms / 1e3),
                                   "unit": "tensor-sweeps/s",
                                   "sample": f"first {ns} tensors, HOOI + MP"}}


def streamed_run(X, start, budget=2 << 30, passes=1):
    """MP on the workload's tensor with its orderings in pinned host memory, streamed to the
    device in chunks of at most `budget` device bytes (the out-of-core form of SP/MP): build
    time, one pass from the start, and the host-to-device rate achieved while streaming."""
    import torch
    from paper_0711_2023_gb300 import tucker as tk
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = tk.tucker_stream_create(X.idx, X.val, X.dims, budget)
    build_s = time.perf_counter() - t0
    _, _, chunks = tk.tucker_stream_info(S)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = tk.tucker_mp_streamed(S, CORE, tol=-np.inf, max_iter=passes, init=start)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    S.close()
    return {"value": passes / dt, "unit": "sweeps/s", "method": "MP", "passes": passes,
            "device_budget_bytes": budget, "chunks": chunks, "build_s": build_s,
            "h2d_gbs_while_streaming": r["bytes_streamed"] / dt / 1e9, "fit": r["fit"],
            "note": "orderings in pinned host memory, chunks copied over NVLink-C2C while the "
                    "previous chunk's projection and Gram run"}


def batched_leg(args):
    from paper_0711_2023_gb300 import build, tucker as tk
    build.build()
    r = batched_run(args.steps, args.warmup, args.batch_count)
    r["autotune"] = [tk.tucker_autotune_decision(i) for i in range(tk.tucker_autotune_count())]
    print(json.dumps({"leg": "batched", **r}), flush=True)


def c2_leg(args):
    """The 1000^3 workload (1e7 nonzeros, core 50^3): HO-SVD and 10 passes each of HOOI, SP and
    MP (31 passes per step), FP64 and mixed, orderings built once.  Prints sweeps/s of both."""
    import torch
    from paper_0711_2023_gb300 import build, synth, tucker as tk
    build.build()
    dims, nnz, core = (1000, 1000, 1000), 10_000_000, (50, 50, 50)
    X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(1))
    C_raw = synth.uniform_matrix(dims[2], core[2], synth.config_seed(2))
    T = tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(), torch.from_numpy(X.val).cuda(),
                                X.dims)

    def step(pr):
        f = {"hosvd": tk.tucker_hosvd(T, core, precision=pr)["fit"]}
        for name, fn in (("hooi", tk.tucker_hooi), ("mp", tk.tucker_mp)):
            f[name] = fn(T, core, tol=-np.inf, max_iter=10, precision=pr)["fit"]
        f["sp"] = tk.tucker_sp(T, core, C_raw, tol=-np.inf, max_iter=10, precision=pr)["fit"]
        return f
    res = {}
    for pr in ("fp64", "mixed"):
        for _ in range(max(1, args.warmup)):
            step(pr)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fits = step(pr)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[pr] = {"sweeps_per_s": 31 * args.steps / dt, "fits": fits}
    print(json.dumps({"leg": "1000^3/1e7/J50, HO-SVD + HOOI/SP/MP x 10", **res,
                      "speedup": res["mixed"]["sweeps_per_s"] / res["fp64"]["sweeps_per_s"],
                      "max_abs_dfit": max(abs(res["fp64"]["fits"][k] - res["mixed"]["fits"][k])
                                          for k in res["fp64"]["fits"])}), flush=True)


def profile_leg(args):
    """One precision form only (warm-up + timed steps of the default step), for profiler
    captures.  --profile-small uses 500^3 with 2.5e6 nonzeros and core 50^3."""
    import torch
    from paper_0711_2023_gb300 import build, synth, tucker as tk
    global DIMS, NNZ, CORE
    if args.profile_small:
        DIMS, NNZ, CORE = (500, 500, 500), 2_500_000, (50, 50, 50)
    build.build()
    X = make_inputs(0)
    T = tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(), torch.from_numpy(X.val).cuda(),
                                X.dims)
    start = oracle_start(X, T, tk)
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        run_step(tk, T, start, args.profile_leg)
    ms_plain, _, _, _, _ = timed_region(tk, torch, 1, 0, args.steps, T, start, l2buf,
                                        args.profile_leg)
    ms, fits, launches, clk, prof = timed_region(tk, torch, 1, 0, args.steps, T, start, l2buf,
                                                 args.profile_leg, profile=True)
    print(json.dumps({"leg": args.profile_leg, "dims": DIMS, "nnz": NNZ, "core": CORE,
                      "value": SWEEPS_PER_STEP * args.steps / (ms_plain / 1e3),
                      "unit": "sweeps/s", "ms_per_step": ms_plain / args.steps,
                      "ms_per_step_profiled": ms / args.steps, "gpu_launches": launches,
                      "fits": fits, "kernels": kern_table(prof, ms),
                      "eig_counters": prof["counters"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="leave the batched workload out of the default line")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-streamed", action="store_true",
                    help="leave the host-streamed (out-of-core) MP out of the default line")
    ap.add_argument("--profile-leg", choices=["fp64", "mixed"], default=None,
                    help="run only warm-up + timed steps of one precision form (for ncu "
                         "captures) and print a short summary line")
    ap.add_argument("--profile-small", action="store_true",
                    help="with --profile-leg: 500^3, 2.5e6 nonzeros, core 50^3")
    ap.add_argument("--batched-leg", action="store_true",
                    help="time the batched workload (256 small tensors) alone")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--c2-leg", action="store_true",
                    help="time HO-SVD + HOOI/SP/MP x 10 on 1000^3 / 1e7 / core 50^3")
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
    if args.c2_leg:
        c2_leg(args)
        return

    import torch
    from paper_0711_2023_gb300 import build, tucker as tk
    build.build()
    tk._lib()
    peaks, peak_src = load_peaks()

    X = make_inputs(rank)
    d_idx = torch.from_numpy(X.idx).cuda()
    d_val = torch.from_numpy(X.val).cuda()
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    # ---- untimed set-up: tensor, orderings (timed on their own), HO-SVD start ----------------
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T = tk.tucker_tensor_create(d_idx, d_val, X.dims)
    tk.tucker_profile_enable(True)
    for n, m, o in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        tk.tucker_ordering(T, n, m, o, copy=False)
    csf_launches, csf_ms, _, _ = tk.tucker_profile_query("csf_build")
    tk.tucker_profile_enable(False)
    start = oracle_start(X, T, tk)
    setup_s = time.perf_counter() - t0

    for _ in range(args.warmup):
        run_step(tk, T, start, "fp64")
    torch.cuda.synchronize()

    # ---- FP64, device-resident ---------------------------------------------------------------
    total_ms, fits, launches, clk, _ = timed_region(tk, torch, world, local, args.steps, T, start,
                                                    l2buf, "fp64")
    t_max = max_over_ranks(total_ms, world)
    value = SWEEPS_PER_STEP * args.steps * world / (t_max / 1e3)
    # one more step with the in-library kernel events on: per-kernel breakdown and rooflines
    prof_ms, _, _, _, prof = timed_region(tk, torch, world, local, 1, T, start, l2buf, "fp64",
                                          profile=True)

    # ---- the mixed form of the same step -----------------------------------------------------
    for _ in range(max(1, min(args.warmup, 2))):
        run_step(tk, T, start, "mixed")
    mx_ms, mx_fits, mx_launches, mx_clk, _ = timed_region(tk, torch, world, local, args.steps, T,
                                                          start, l2buf, "mixed")
    mx_value = SWEEPS_PER_STEP * args.steps * world / (max_over_ranks(mx_ms, world) / 1e3)
    mx_prof_ms, _, _, _, mx_prof = timed_region(tk, torch, world, local, 1, T, start, l2buf,
                                                "mixed", profile=True)
    T.close()

    # ---- end to end through the C ABI from pinned host buffers ------------------------------
    h_idx = torch.from_numpy(X.idx).pin_memory()
    h_val = torch.from_numpy(X.val).pin_memory()
    h_start = [None] + [torch.from_numpy(np.ascontiguousarray(u)).pin_memory() for u in start[1:]]
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    e2e_ms = 0.0
    barrier(world)
    for _ in range(e2e_steps):
        flush_l2(l2buf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Th = tk.tucker_tensor_create(h_idx, h_val, X.dims)
        st_dev = [None] + [u.cuda(non_blocking=True) for u in h_start[1:]]
        run_step(tk, Th, st_dev, "fp64", out="host")
        Th.close()
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
    e2e_max = max_over_ranks(e2e_ms, world)
    e2e_value = SWEEPS_PER_STEP * e2e_steps * world / (e2e_max / 1e3)
    h2d = X.nnz * (3 * 4 + 8) + 8 * sum(DIMS[a] * CORE[a] for a in (1, 2))
    d2h = 2 * 8 * (CORE[0] * CORE[1] * CORE[2] + sum(DIMS[a] * CORE[a] for a in range(3)))

    batched = None
    if not args.no_batched:
        batched = batched_run(steps=2, warmup=1)
    streamed = None
    if not args.no_streamed:
        streamed = streamed_run(X, start)
        streamed["dfit_vs_in_memory"] = abs(streamed["fit"] - fits["mp"])

    if rank != 0:
        return

    # ---- rooflines ---------------------------------------------------------------------------
    fp64_src = "nominal GB300 FP64 rate 1.25 TFLOP/s (no measured FP64 figure)"
    kp = kernels_only(prof)
    dom = max(kp, key=lambda k: kp[k]["ms"])
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    bf16_src = (f"{peak_src} bf16 sustained (cuBLAS); algorithmic FP32-equivalent Gram FLOPs "
                "(the BF16x3 kernel issues 3x as many)")
    if dom == "gram_bf16x3":
        roofline = roofline_of(prof, dom, prof_ms, "tensor", bf16, "TFLOP/s", bf16_src)
    elif dom in OZAKI_KERNELS:
        roofline = roofline_of(prof, dom, prof_ms, "tensor", bf16, "TFLOP/s",
                               f"{peak_src} bf16 sustained (cuBLAS); BF16 FLOPs the tensor cores "
                               "issue (22 or 28 slice products per FP64 product)")
        if roofline and dom == "gram_ozaki":
            # DRAM bytes of one ncu capture of this kernel on the 500^3 MP Gram (rows 500,
            # K = 5e4): 1.62 x its algorithmic bytes (the slices once, plus slices 0-3 again in
            # the second pass, plus the int64 partials).  The slice bytes grow with rows x K, so
            # the ratio scales to the bench launches; the capture of the full-size launch is above
            # the size ncu may take.
            roofline["traffic"] = GRAM_OZAKI_DRAM_RATIO * roofline["algorithmic_bytes"]
            roofline["traffic_note"] = ("per launch, scaled from an ncu capture of the 500^3 "
                                        "MP Gram (DRAM bytes 1.62 x algorithmic: the second "
                                        "pass re-reads slices 0-3)")
    else:
        roofline = roofline_of(prof, dom, prof_ms, "alu", FP64_PEAK_TFLOPS, "TFLOP/s", fp64_src)
    mx_gram = roofline_of(mx_prof, "gram_bf16x3", mx_prof_ms, "tensor", bf16, "TFLOP/s", bf16_src)

    cpu, oracle_fits = None, {}
    if world == 1 and not args.no_cpu_baseline:
        cpu, oracle_fits = cpu_baseline_leg(X, start)

    dfit_mx = max(abs(mx_fits[k] - fits[k]) for k in fits)
    vs_oracle = None
    if "hooi" in oracle_fits:
        vs_oracle = {"hooi_fp64": abs(fits["hooi"] - oracle_fits["hooi"]),
                     "hooi_mixed": abs(mx_fits["hooi"] - oracle_fits["hooi"])}
    proj_note = ("algorithmic bytes = what the projection must read and write; HOOI's TTMc at "
                 "core 100 does J_m J_o FMAs per fiber, so it is bound by arithmetic, not HBM")
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(world),
        "fits": fits,
        "csf_build_ms": csf_ms, "csf_build_launches": csf_launches, "setup_s": setup_s,
        "kernels": kern_table(prof, prof_ms),
        "profiled_step_ms": prof_ms,
        "eig_counters": prof["counters"],
        "ttmc": {
            "fp64": ttmc_rates(prof, "ttmc_f64", FP64_PEAK_TFLOPS, peaks.get("hbm_gbs"), proj_note),
            "mixed": ttmc_rates(mx_prof, "ttmc_mixed", FP32_PEAK_TFLOPS, peaks.get("hbm_gbs"),
                                proj_note),
            "slice_proj_mixed": ttmc_rates(mx_prof, "slice_proj_mixed", FP32_PEAK_TFLOPS,
                                           peaks.get("hbm_gbs"), "MP slice projection, HBM-bound "
                                           "form (writes the split projection)")},
        "roofline": roofline,
        "mixed": {"value": mx_value, "unit": "sweeps/s", "ms_per_step": mx_ms / args.steps,
                  "speedup_vs_fp64": mx_value / value,
                  "max_abs_dfit_vs_fp64": dfit_mx, "abs_dfit_vs_oracle": vs_oracle,
                  "fits": mx_fits, "kernels": kern_table(mx_prof, mx_prof_ms),
                  "profiled_step_ms": mx_prof_ms, "eig_counters": mx_prof["counters"],
                  "roofline_gram": mx_gram, "gpu_launches": mx_launches, "clocks": mx_clk},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "batched": batched,
        "streamed": streamed,
        "gpu_launches": launches,
        "clocks": clk,
        "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs"),
                  "bf16_tflops": peaks.get("bf16_tflops"),
                  "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained")},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
