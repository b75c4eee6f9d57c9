"""Benchmark of the dense LU solve (the LINPACK hot path) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One step = one whole solve of the workload: lu_factor (the blocked
right-looking LU with partial pivoting) + lu_solve (+ lu_refine for the mixed
workloads), on a synthetic seeded HPL-shaped matrix already resident in HBM.
The metric is TFLOP/s with the HPL count (2/3 n^3 + 2 n^2 nrhs) / time.

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank solves its own
independent system on its own GPU (replicas: the single-system LU is not
sharded); value = all ranks' FLOPs / max-over-ranks time.

--impl reference times the CPU oracle (plain C FP64 GEPP) on the host cores,
each step a bounded sample of the same workload: the first block iterations of
the blocked factorization.
"""
from __future__ import annotations

import argparse
import json
import math
import os

# The served companion runs many requests' streams at once: with CUDA's
# default of 8 hardware work queues they share queues and wait behind one
# another.  Set before any CUDA context exists in this process.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the FP64 configuration: n = 16384, nb = 256, A and b uniform[-0.5, 0.5]
    "hpl_f64_n16384_nb256": dict(n=16384, nb=256, prec="f64", nrhs=1, seed=2, shift=0.0),
    # the small FP64 configuration (n = 1024, nb = 64)
    "hpl_f64_n1024_nb64": dict(n=1024, nb=64, prec="f64", nrhs=1, seed=1, shift=0.0),
    # the mixed configuration: A + (n/4) I, BF16 / FP16 tensor-core factor + FP64 refinement
    "hpl_mixed_bf16_n32768": dict(n=32768, nb=0, prec="bf16", nrhs=1, seed=3, shift=0.25),
    "hpl_mixed_fp16_n32768": dict(n=32768, nb=0, prec="fp16", nrhs=1, seed=3, shift=0.25),
    "hpl_mixed_bf16_n32768_rhs32": dict(n=32768, nb=0, prec="bf16", nrhs=32, seed=3, shift=0.25),
    # the paper's own variant (HPL-AI rules: no pivoting on a diagonally dominant
    # A): BF16 tensor-core factor + FP64 refinement, and FP32 without refinement
    "hpl_nopiv_bf16_n32768": dict(n=32768, nb=0, prec="bf16", nrhs=1, seed=3, shift=0.25, nopiv=True),
    "hpl_nopiv_f32_n32768": dict(n=32768, nb=256, prec="f32", nrhs=1, seed=3, shift=0.25, nopiv=True,
                                 norefine=True),
    # the FP64 configuration with the trailing update on the BF16 tensor cores by
    # error-free splitting (FP64-accurate products, 8 slices of 7 bits)
    "hpl_f64ozaki_n16384_nb256": dict(n=16384, nb=256, prec="f64", nrhs=1, seed=2, shift=0.0, ozaki=True),
    # smaller cases of the same shapes (profiling captures)
    "hpl_f64_n4096_nb256": dict(n=4096, nb=256, prec="f64", nrhs=1, seed=2, shift=0.0),
    "hpl_f64ozaki_n4096_nb256": dict(n=4096, nb=256, prec="f64", nrhs=1, seed=2, shift=0.0, ozaki=True),
    "hpl_mixed_bf16_n8192": dict(n=8192, nb=0, prec="bf16", nrhs=1, seed=3, shift=0.25),
    "hpl_nopiv_bf16_n8192": dict(n=8192, nb=0, prec="bf16", nrhs=1, seed=3, shift=0.25, nopiv=True),
    # the batched configuration: 4096 systems, n ~ U{32..512}, 1-8 right-hand
    # sides, A + n I, FP32 factor + FP64 refinement, one persistent launch
    "batched_4096": dict(count=4096, nmin=32, nmax=512, kmax=8, seed=5, prec="f32"),
    # a small case of the same kernel for profiling captures
    "batched_512": dict(count=512, nmin=32, nmax=512, kmax=8, seed=5, prec="f32"),
    # the served configuration: Poisson arrivals, n log-uniform 64..8192, 1-16
    # right-hand sides, 30% repeat-RHS on resident factors, FP16 factor + FP64
    # refinement, admission by a 120 GB HBM budget
    "served_2000": dict(rate=2000.0, seconds=60.0, nmin=64, nmax=8192, kmax=16, repeat=0.3, seed=6, prec="fp16",
                        budget_gb=120, slots=24, pool=48),
}
DEFAULT = "hpl_f64_n16384_nb256"
METRIC = "LU solve TFLOP/s (HPL count 2/3 n^3 + 2 n^2 nrhs) at scaled residual < 16"


def hpl_flops(n: int, nrhs: int) -> float:
    return 2.0 / 3.0 * n ** 3 + 2.0 * n ** 2 * nrhs


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_source": "fallback"}


# nominal dense rates per GB300 (TFLOP/s): used as ratios to the measured BF16 peak
NOMINAL = {"bf16": 2250.0, "fp16": 2250.0, "f64": 1.25, "f32_simt": 75.0}
FP64_CLOCK_GHZ = 2.07  # maximum SM clock (the FP64 update runs at it: clocks in the line)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend: str = "nccl"):
    """One process per GPU (torchrun): rank, world size, local rank.  The
    replicas share no data; the group only carries the barrier and the
    max-over-ranks time (gloo serves the CPU tests of this logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        lr = int(os.environ.get("LOCAL_RANK", "0"))
        if backend == "nccl":
            torch.cuda.set_device(lr)
        dist.init_process_group(backend)
        return dist.get_rank(), ws, lr
    return 0, 1, 0


def replica_seed(seed: int, rank: int) -> int:
    """Seed of rank's own system: independent replicas, no data exchanged."""
    return seed + 1000 * rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def default_nb(n: int, prec: str, ozaki: bool = False) -> int:
    """The block width the library picks for nb = 0 (its tuning table)."""
    from paper_2202_13995_gb300 import lu
    return lu.default_nb(n, prec, ozaki)


def gemm_roofline(prof: dict, n: int, nb: int, prec: str, steps: int, peaks: dict, wname: str,
                  ozaki: bool = False) -> dict:
    """Roofline of the dominant kernel, the trailing update, from its summed
    CUDA-event launch durations in the timed region.

    FP64 (DFMA, CUDA cores): bound by the FP64 pipes; algorithmic FLOPs per
    launch = 2 m'^2 nb.  BF16/FP16 (tcgen05): at nb = 256 the update's FP32
    C read-modify-write makes it HBM-bound (64 FLOP per byte, below the
    tensor ridge); algorithmic bytes per launch = 8 m' n' (C read + write)
    + 2 (m' + n') kpad (the 16-bit operands).  FP64 by error-free splitting
    (tcgen05, BF16 slices): bound by the tensor pipe; algorithmic FLOPs per
    launch = 36 slice pairs x 2 m' n' kpad."""
    gemm_ms, gemm_n = prof["gemm"]
    nbx = nb or default_nb(n, prec, ozaki)
    kpad = -(-nbx // 64) * 64
    flops = bytes_ = 0.0
    dram_alg = 0.0  # algorithmic DRAM bytes of the kernel's own data type, all launches of one step
    nlaunch = 0
    for k in range(0, n, nbx):
        w = min(nbx, n - k)
        rest = n - k - w
        if rest > 0:
            flops += 2.0 * rest * rest * w
            bytes_ += 8.0 * rest * rest + 2.0 * (2 * rest) * kpad
            if ozaki:  # FP64 C read + write, 8 BF16 slices of both operands
                dram_alg += 16.0 * rest * rest + 16.0 * (2 * rest) * kpad
            elif prec == "f64":  # FP64 C read + write, FP64 operands
                dram_alg += 16.0 * rest * rest + 8.0 * (2 * rest) * w
            else:
                dram_alg += 8.0 * rest * rest + 2.0 * (2 * rest) * kpad
            nlaunch += 1
    flops *= steps
    bytes_ *= steps
    sec = gemm_ms * 1e-3
    kernel = "oz_gemm_kernel" if ozaki else ("gemm_simt_kernel<double>" if prec == "f64" else "tc_gemm_kernel")
    # traffic per launch: the ratio of ncu DRAM bytes to algorithmic bytes of
    # launches captured on a small case of the same kernel (profiles/traffic.json,
    # one entry per kernel; counters beyond the launch time are collected only
    # on small cases), times this step's mean algorithmic bytes per update
    traffic = traffic_ratio = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath) and nlaunch:
        try:
            ent = json.load(open(tpath)).get(kernel)
            if ent:
                traffic_ratio = float(ent["ratio"])
                traffic = traffic_ratio * dram_alg / nlaunch
        except Exception:
            traffic = traffic_ratio = None
    base = {"launches": gemm_n, "kernel_ms_per_step": gemm_ms / steps, "traffic": traffic,
            "traffic_over_algorithmic": traffic_ratio,
            "tflops": flops / sec / 1e12 if sec > 0 else None}
    if ozaki:
        tflops_bf16 = 36.0 * flops / nbx * kpad / sec / 1e12 if sec > 0 else None
        peak = peaks.get("bf16_tflops_sustained", 1701.1)
        return dict(base, bound="tensor", kernel="oz_gemm_kernel", achieved=tflops_bf16, peak=peak,
                    unit="TFLOP/s", frac=(tflops_bf16 / peak) if tflops_bf16 else None,
                    peak_source=f"bf16_tflops_sustained of {peaks['_source']}",
                    fp64_equiv_tflops=base["tflops"])
    if prec == "f64":
        # FP64 pipe: the nominal 1.25 TFLOP/s is 2 FP64 FMAs per clock per SM
        # (1.25e12 / (2 x 152 x 2.07e9) = 1.99); at the 2070 MHz the kernel runs
        # at, 2 x 2 x 152 x 2.07e9 = 1.259 TFLOP/s.  ncu agrees: the kernel
        # keeps the FP64 pipe 99 % busy while doing 1.24 TFLOP/s.
        sms = int(peaks.get("sm_count", 152))
        ghz = float(peaks.get("sm_max_mhz", 1000.0 * FP64_CLOCK_GHZ)) / 1000.0
        peak = 2.0 * 2.0 * sms * ghz * 1e9 / 1e12
        ach = flops / sec / 1e12 if sec > 0 else None
        return dict(base, bound="alu", kernel="gemm_simt_kernel<double>", achieved=ach, peak=peak, unit="TFLOP/s",
                    frac=(ach / peak) if ach else None,
                    peak_source=f"derived: 2 FP64 FMA/clock/SM x {sms} SMs x {ghz} GHz max SM clock "
                                f"(the nominal 1.25 TFLOP/s)")
    peak = peaks.get("hbm_gbs", 6800.0)
    ach = bytes_ / sec / 1e9 if sec > 0 else None
    return dict(base, bound="hbm", kernel="tc_gemm_kernel", achieved=ach, peak=peak, unit="GB/s",
                frac=(ach / peak) if ach else None, peak_source=f"hbm_gbs of {peaks['_source']}",
                tensor_frac_of_sustained=(flops / sec / 1e12 / peaks.get("bf16_tflops_sustained", 1701.1))
                if sec > 0 else None)


def _block_step_flops(n: int, nb: int, s: int) -> float:
    """Operation count of block iteration s (panel, top solve, inner update)."""
    m = n - s * nb
    w = min(nb, m)
    panel = sum((m - j - 1) * (1 + 2 * (w - j - 1)) for j in range(w))
    trsm = float(w * (w - 1)) * (m - w)
    update = 2.0 * (m - w) * (m - w) * w
    return panel + trsm + update


def oracle_sample(cfg: dict, max_seconds: float = 20.0, A=None, one_core: bool = False) -> dict:
    """Time the oracle on the host cores on a bounded sample of the same
    workload: the first block iterations of the blocked factorization."""
    import numpy as np
    import oracle as O
    from paper_2202_13995_gb300 import inputs as I
    n = cfg["n"]
    nb = cfg["nb"] or 256
    if A is None:
        A = I.hpl_matrix(n, cfg["seed"], diag_shift=cfg["shift"] * n)
    O.set_threads(os.cpu_count() or 1)
    cores = O.num_threads()
    nsteps = math.ceil(n / nb)
    _, _, _, t1 = O.getrf(A, nb, ksteps=1, timed=True)
    ks = max(1, min(nsteps, int(max_seconds / max(t1, 1e-6))))
    t = t1
    if ks > 1:
        _, _, _, t = O.getrf(A, nb, ksteps=ks, timed=True)
    flops = sum(_block_step_flops(n, nb, s) for s in range(ks))
    out = {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
           "seconds": round(t, 3),
           "sample": f"first {ks} of {nsteps} block iterations (panel, interchanges, top solve, inner update) "
                     f"of the n={n}, nb={nb} FP64 blocked LU; operation count of those iterations / wall time"}
    if one_core:
        # the same code on one core, on a bounded sub-sample (a few seconds)
        n1 = min(n, 4096)
        A1 = np.ascontiguousarray(A[:n1, :n1])
        O.set_threads(1)
        _, _, _, t1c = O.getrf(A1, nb, ksteps=1, timed=True)
        O.set_threads(os.cpu_count() or 1)
        out["one_core"] = {"value": _block_step_flops(n1, nb, 0) / t1c / 1e12, "unit": "TFLOP/s", "cores": 1,
                           "seconds": round(t1c, 3),
                           "sample": f"first block iteration of the leading {n1} x {n1} block, nb={nb}"}
    return out


def run_reference(args, cfg, wname):
    # rank 0 alone times the oracle; other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    from paper_2202_13995_gb300 import inputs as I
    A = I.hpl_matrix(cfg["n"], cfg["seed"], diag_shift=cfg["shift"] * cfg["n"])
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(cfg, max_seconds=args.ref_seconds, A=A)
        if i >= args.warmup:
            vals.append(r)
    best = max(vals, key=lambda r: r["value"])
    v = statistics.median([r["value"] for r in vals])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median([r["seconds"] for r in vals]) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": cfg["n"], "nb": cfg["nb"] or 256, "nrhs": cfg["nrhs"]},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": best["cores"], "kind": "oracle",
                         "sample": best["sample"]},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_solves(ctx, stream, cfg: dict, nb, steps: int, warmup: int, rank: int, ws: int, sampler=None) -> dict:
    """Warm up, then time `steps` whole solves on the device (CUDA events on
    the library's stream, a barrier and a synchronize on both sides)."""
    import torch
    from paper_2202_13995_gb300 import inputs as I
    from paper_2202_13995_gb300 import lu
    n, prec, nrhs = cfg["n"], cfg["prec"], cfg["nrhs"]
    shift = cfg["shift"] * n
    mixed = prec != "f64"
    # the seeded inputs, generated on the device (lu_generate: the same bits
    # as inputs.hpl_matrix / hpl_rhs)
    A = lu.generate(lu.colmajor_empty(n, n), replica_seed(cfg["seed"], rank), 0, shift)
    B = lu.generate(lu.colmajor_empty(n, nrhs), replica_seed(cfg["seed"], rank), 1)
    X = lu.colmajor_empty(n, nrhs)
    torch.cuda.synchronize()
    iters = []

    nopiv = bool(cfg.get("nopiv", False))
    ozaki = bool(cfg.get("ozaki", False))
    refine = mixed and not cfg.get("norefine", False)

    def step():
        f = ctx.factor(A, prec, nb, sync=False, nopiv=nopiv, ozaki=ozaki)
        if refine:
            iters.append(f.refine(A, B, X, 16.0, 50)[0])
        else:
            X.copy_(B)
            f.solve_(X)
        f.free()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    # the timed region carries one CUDA event pair per trailing-update launch
    # (the roofline's kernel) and no other events
    ctx.profile_select(["gemm"])
    ctx.profile(True)
    l0 = ctx.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    barrier(ws)
    ck = sampler.stop() if sampler else None
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, ws)
    # the phase split from a separate pass with an event pair around every launch
    psteps = max(1, min(steps, 3))
    ctx.profile_select(None)
    ctx.profile(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(psteps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    phases = ctx.profile_read()
    ctx.profile(False)
    phases_ms = {k: round(v[0] / psteps, 3) for k, v in phases.items()}
    profiled_ms = p0.elapsed_time(p1) / psteps
    norms = ctx.residual_norms(A, X, B)
    res = float(ctx.scaled_residual(A, X, B).max())
    # the paper's own shape of the check, ||r|| / (n ||b|| eps), eps = 2^-53
    res_paper = float(max(r[0] / (n * r[3] * 2.0 ** -53) if r[3] > 0 else math.inf for r in norms))
    return {"A": A, "B": B, "X": X, "ms": ms, "prof": prof, "launches": launches, "res": res, "clocks": ck,
            "res_paper": res_paper, "phases_ms": phases_ms, "profiled_ms": profiled_ms,
            "refine_iters": iters[-1] if iters else None}


def batched_measure(ctx, stream, cfg: dict, steps: int, warmup: int, tune: bool = True) -> dict:
    """Time `steps` runs of one planned batch (each run = one graph launch)."""
    import torch
    from paper_2202_13995_gb300 import inputs as I
    from paper_2202_13995_gb300 import lu
    ns, ks = I.batch_shapes(cfg["count"], cfg["seed"], cfg["nmin"], cfg["nmax"], cfg["kmax"])
    As, Bs = I.hpl_batch_torch(ns, ks, cfg["seed"])
    xbuf = torch.empty(int(sum(int(n) * int(k) for n, k in zip(ns, ks))), dtype=torch.float64, device="cuda")
    Xs, o = [], 0
    for n, k in zip(ns, ks):
        Xs.append(xbuf[o:o + int(n) * int(k)].view(int(k), int(n)).t())
        o += int(n) * int(k)
    bt = lu.Batch(ctx, As, Bs, Xs, tune=tune)
    cnt = len(As)
    info = torch.zeros(cnt, dtype=torch.int32, device="cuda")
    iters = torch.zeros(cnt, dtype=torch.int32, device="cuda")
    resid = torch.zeros(cnt, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        bt.run(info, iters, resid)
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        bt.run(info, iters, resid)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    flops = float(sum(2.0 / 3.0 * float(n) ** 3 + 2.0 * float(n) ** 2 * float(k) for n, k in zip(ns, ks)))
    shape = bt.shape()
    out = {"workload": f"batched_{cnt}", "systems": cnt, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
           "ms_per_step": ms, "solves_per_s": cnt / (ms * 1e-3), "all_converged": bool((info == 0).all().item()),
           "max_scaled_residual": float(resid.max().item()), "max_refine_iters": int(iters.max().item()),
           "launch_shape": {"threads": shape[0], "ctas_per_sm": shape[1]}, "launches": ctx.launch_count() - l0,
           "bytes_a_fp64": int(sum(int(n) * int(n) for n in ns)) * 8}
    bt.free()
    return out


def served_measure(cfg: dict, rate: float = None, seconds: float = None) -> dict:
    """Replay a seeded Poisson request stream against lu_server and report
    throughput and latency (t_done - t_submit, queueing included)."""
    import time as _t
    import numpy as np
    import torch
    from paper_2202_13995_gb300 import inputs as I
    from paper_2202_13995_gb300 import lu
    rate = rate or cfg["rate"]
    seconds = seconds or cfg["seconds"]
    rng = np.random.default_rng(cfg["seed"])
    # a pool of distinct systems (A + (n/4) I) the requests draw from
    pool_n = np.exp(rng.uniform(np.log(cfg["nmin"]), np.log(cfg["nmax"]), cfg["pool"])).astype(int)
    pool_A = [I.hpl_matrix_torch(int(n), 600000 + i, diag_shift=n / 4.0, device="cuda") for i, n in enumerate(pool_n)]
    pool_B = [I.hpl_rhs_torch(int(n), cfg["kmax"], 600000 + i, device="cuda").contiguous().t().contiguous().t()
              for i, n in enumerate(pool_n)]
    torch.cuda.synchronize()
    nreq = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    picks = rng.integers(0, cfg["pool"], nreq)
    ks = rng.integers(1, cfg["kmax"] + 1, nreq)
    rep = rng.uniform(0, 1, nreq) < cfg["repeat"]
    srv = lu.Server(int(cfg["budget_gb"]) << 30, cfg["prec"], max_slots=cfg["slots"])
    kept = set()
    tickets, flops = [], 0.0
    t0 = _t.perf_counter()
    for i in range(nreq):
        while _t.perf_counter() - t0 < arrivals[i]:
            _t.sleep(min(2e-4, max(0.0, arrivals[i] - (_t.perf_counter() - t0))))
        p = int(picks[i])
        n, k = int(pool_n[p]), int(ks[i])
        X = lu.colmajor_empty(n, k)
        B = pool_B[p][:, :k]
        repeat = bool(rep[i]) and p in kept
        if repeat:
            t = srv.submit(pool_A[p], B, X, factor_key=p + 1, use_resident=True)
        else:
            t = srv.submit(pool_A[p], B, X, factor_key=p + 1, keep_factor=True)
            kept.add(p)
        tickets.append((t, n, k, repeat))
    res = [srv.wait(t) for t, _, _, _ in tickets]
    t_end = _t.perf_counter()
    stats = srv.stats()
    srv.close()
    lat = np.array([(r.t_done_ns - r.t_submit_ns) * 1e-6 for r in res])
    svc = np.array([(r.t_done_ns - r.t_start_ns) * 1e-6 for r in res])
    span = (max(r.t_done_ns for r in res) - min(r.t_submit_ns for r in res)) * 1e-9
    for r, (_, n, k, _) in zip(res, tickets):
        flops += (0.0 if r.reused_factor else 2.0 / 3.0 * n ** 3) + 2.0 * n * n * k * (1 + r.iters)
    ok = sum(1 for r in res if r.status == 0)
    # service time (start to done) by size bucket: where the capacity goes
    buckets = {}
    for r, (_, n, k, rp) in zip(res, tickets):
        key = "repeat" if r.reused_factor else ("n<=512" if n <= 512 else ("n<=2048" if n <= 2048 else "n>2048"))
        buckets.setdefault(key, []).append((r.t_done_ns - r.t_start_ns) * 1e-6)
    by_size = {kk: {"count": len(v), "service_p50_ms": float(np.percentile(v, 50)),
                    "service_p99_ms": float(np.percentile(v, 99))} for kk, v in sorted(buckets.items())}
    status_hist = {}
    for r in res:
        status_hist[str(r.status)] = status_hist.get(str(r.status), 0) + 1
    return {"workload": "served", "offered_rate_per_s": rate, "seconds_of_arrivals": seconds, "requests": nreq,
            "completed_ok": ok, "status_counts": status_hist, "solves_per_s": nreq / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "service_p50_ms": float(np.percentile(svc, 50)),
            "reused_factor": int(sum(r.reused_factor for r in res)),
            "refactored": int(sum(r.refactored for r in res)), "evictions": int(stats["evictions"]),
            "max_scaled_residual": float(max(r.scaled_resid for r in res)), "tflops": flops / span / 1e12,
            "service_by_size": by_size,
            "slots": cfg["slots"], "budget_gb": cfg["budget_gb"], "prec": cfg["prec"],
            "wall_s": t_end - t0}


def mixed_companion(ctx, stream, mname, args, rank, ws, peaks, f64_flops=None, f64_ms=None) -> dict:
    """One mixed-precision companion line (BF16/FP16 tensor-core factor + FP64
    refinement), timed by the same rules as the headline."""
    import torch
    mc = WORKLOADS[mname]
    mr = timed_solves(ctx, stream, mc, mc["nb"], args.steps, args.warmup, rank, ws)
    mv = hpl_flops(mc["n"], mc["nrhs"]) * ws / (mr["ms"] * 1e-3) / 1e12
    line = {"workload": mname, "value": mv, "unit": "TFLOP/s", "ms_per_step": mr["ms"], "nrhs": mc["nrhs"],
            "scaled_residual": mr["res"], "refine_iters": mr["refine_iters"],
            "roofline": gemm_roofline(mr["prof"], mc["n"], mc["nb"], mc["prec"], args.steps, peaks, mname),
            "phases_ms_per_step": mr["phases_ms"], "profiled_ms_per_step": mr["profiled_ms"],
            "_launches": mr["launches"]}
    if f64_flops:
        line["speedup_vs_f64"] = mv / (f64_flops * ws / (f64_ms * 1e-3) / 1e12)
    del mr
    torch.cuda.empty_cache()
    return line


def run_ours(args, cfg, wname):
    import torch
    from paper_2202_13995_gb300 import lu

    rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    peaks = load_peaks()
    n, nb, prec, nrhs = cfg["n"], cfg["nb"], cfg["prec"], cfg["nrhs"]
    if args.nb is not None:
        nb = args.nb
    shift = cfg["shift"] * n
    mixed = prec != "f64"
    flops = hpl_flops(n, nrhs)

    stream = torch.cuda.current_stream()
    ctx = lu.Context(stream)
    r = timed_solves(ctx, stream, cfg, nb, args.steps, args.warmup, rank, ws, ClockSampler(local))
    A, B = r["A"], r["B"]
    ms, prof, launches = r["ms"], r["prof"], r["launches"]
    res, ck, res_paper = r["res"], r["clocks"], r["res_paper"]
    phases_ms, profiled_ms = r["phases_ms"], r["profiled_ms"]
    ozaki = bool(cfg.get("ozaki", False))
    roofline = gemm_roofline(prof, n, nb, prec, args.steps, peaks, wname, ozaki)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # column-major host and device buffers held as contiguous (k, n)
        # storages, so that every transfer is one plain copy of the bytes
        Ah = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A.t())
        Bh = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True)
        Bh.copy_(B.t())
        Xh = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True)
        Ad = lu.colmajor_empty(n, n)
        Bd = lu.colmajor_empty(n, nrhs)
        Xd = lu.colmajor_empty(n, nrhs)
        assert Ad.t().is_contiguous() and Bd.t().is_contiguous() and Xd.t().is_contiguous()

        seg = []  # per step: events at start, after the H2D copies, after the solve, after the D2H copy

        def e2e_step(record=False):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
            if record:
                ev[0].record(stream)
            Ad.t().copy_(Ah, non_blocking=True)
            Bd.t().copy_(Bh, non_blocking=True)
            if record:
                ev[1].record(stream)
            f = ctx.factor(Ad, prec, nb, sync=False, nopiv=bool(cfg.get("nopiv", False)), ozaki=ozaki)
            if mixed and not cfg.get("norefine", False):
                f.refine(Ad, Bd, Xd, 16.0, 50)
            else:
                Xd.copy_(Bd)
                f.solve_(Xd)
            if record:
                ev[2].record(stream)
            Xh.copy_(Xd.t(), non_blocking=True)
            if record:
                ev[3].record(stream)
                seg.append(ev)
            f.free()

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ke = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(ke):
            e2e_step(record=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, ws)
        h2d_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in seg)
        solve_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in seg)
        d2h_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in seg)
        h2d_bytes = int(A.numel() * 8 + n * nrhs * 8)
        e2e = {"value": flops * ws / (ems * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ems,
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": int(n * nrhs * 8),
               "segments_ms_per_step": {"h2d": h2d_ms, "solve": solve_ms, "d2h": d2h_ms},
               "h2d_gbs": h2d_bytes / (h2d_ms * 1e-3) / 1e9 if h2d_ms > 0 else None}
        del Ah, Bh, Xh, Ad, Bd, Xd
    del r, A, B
    torch.cuda.empty_cache()

    # ---- the mixed-precision companion: BF16 tensor-core factor + FP64
    #      refinement on A + (n/4) I, n = 32768 (same timing rules)
    mixed_line = None
    nopiv_line = None
    if not mixed and not args.no_mixed and wname == DEFAULT:
        # the paper's own variant on the mixed configuration's matrix
        pname = "hpl_nopiv_bf16_n32768"
        pc = WORKLOADS[pname]
        pr = timed_solves(ctx, stream, pc, pc["nb"], args.steps, args.warmup, rank, ws)
        pv = hpl_flops(pc["n"], pc["nrhs"]) * ws / (pr["ms"] * 1e-3) / 1e12
        nopiv_line = {"workload": pname, "value": pv, "unit": "TFLOP/s", "ms_per_step": pr["ms"],
                      "lu_only_tflops": 2.0 / 3.0 * pc["n"] ** 3 * ws / (pr["ms"] * 1e-3) / 1e12,
                      "scaled_residual": pr["res"], "refine_iters": pr["refine_iters"],
                      "phases_ms_per_step": pr["phases_ms"], "profiled_ms_per_step": pr["profiled_ms"]}
        launches += pr["launches"]
        del pr
        torch.cuda.empty_cache()
        mixed_line = mixed_companion(ctx, stream, "hpl_mixed_bf16_n32768", args, rank, ws, peaks, flops, ms)
        launches += mixed_line.pop("_launches")
        # the same configuration with FP16 operands, and with 32 right-hand sides
        for key, nm in (("fp16", "hpl_mixed_fp16_n32768"), ("rhs32", "hpl_mixed_bf16_n32768_rhs32")):
            ln = mixed_companion(ctx, stream, nm, args, rank, ws, peaks, None, None)
            launches += ln.pop("_launches")
            mixed_line[key] = ln

    ozaki_line = None
    if not mixed and not args.no_mixed and wname == DEFAULT:
        # the same FP64 configuration with the update by error-free splitting
        oname = "hpl_f64ozaki_n16384_nb256"
        oc = WORKLOADS[oname]
        orr = timed_solves(ctx, stream, oc, oc["nb"], args.steps, args.warmup, rank, ws)
        ov = hpl_flops(oc["n"], oc["nrhs"]) * ws / (orr["ms"] * 1e-3) / 1e12
        ozaki_line = {"workload": oname, "value": ov, "unit": "TFLOP/s", "ms_per_step": orr["ms"],
                      "speedup_vs_f64": ov / (flops * ws / (ms * 1e-3) / 1e12), "scaled_residual": orr["res"],
                      "roofline": gemm_roofline(orr["prof"], oc["n"], oc["nb"], oc["prec"], args.steps, peaks, oname,
                                                True),
                      "phases_ms_per_step": orr["phases_ms"], "profiled_ms_per_step": orr["profiled_ms"]}
        launches += orr["launches"]
        del orr
        torch.cuda.empty_cache()

    # arithmetic-rate probes of this GPU (the denominators of the CUDA-core
    # kernels: the FP32 batched factor; the FP64 update keeps the rate derived
    # from unit counts and clock, which it reaches, above the probe's)
    rates = None
    if not args.no_mixed and wname == DEFAULT:
        rates = {"fp64_fma_tflops": lu.peak_probe(0), "fp64_mma_tflops": lu.peak_probe(1),
                 "fp32_fma_tflops": lu.peak_probe(2),
                 "how": "lu_peak_probe: register-only kernels on every SM, best of 3 timed launches of ~150 ms"}

    batched_line = None
    if not mixed and not args.no_mixed and wname == DEFAULT:
        batched_line = batched_measure(ctx, stream, WORKLOADS["batched_4096"], args.steps, args.warmup)
        launches += batched_line["launches"]
        # the batched kernel: FP32 factor on the CUDA cores (plus FP64
        # refinement); bound = the FP32 FMA pipe, measured by the probe above
        fpk = rates["fp32_fma_tflops"]
        batched_line["roofline"] = {"bound": "alu", "kernel": "batched_kernel", "achieved": batched_line["value"],
                                    "peak": fpk, "unit": "TFLOP/s", "frac": batched_line["value"] / fpk,
                                    "peak_source": "fp32_fma_tflops of lu_peak_probe (measured in this run)",
                                    "traffic": None}
        torch.cuda.empty_cache()

    # the served configuration: Poisson arrivals at 2000/s for 60 s, and the
    # same mix at a rate the server sustains (latencies that stay bounded)
    served_line = None
    if not mixed and not args.no_mixed and not args.no_served and wname == DEFAULT and ws == 1:
        sc = WORKLOADS["served_2000"]
        served_line = served_measure(sc, sc["rate"], args.served_seconds)
        served_line["sustainable"] = served_measure(sc, args.served_low_rate, 20.0)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_sample(dict(cfg, nb=nb or 256), max_seconds=args.cpu_seconds, one_core=True)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": flops * ws / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ("f64 (bf16-split products)" if ozaki else "f64") if not mixed else f"{prec}+f32acc+f64refine", "data": "synthetic",
            "config": {"workload": wname, "n": n, "nb": nb or "auto", "nrhs": nrhs, "precision": prec,
                       "matrix": "uniform[-0.5,0.5]" + (f" + {cfg['shift']}*n*I" if shift else ""),
                       "l2": (f"inputs larger than L2 (A = {n * n * 8 / 2 ** 30:.1f} GiB FP64)" if n * n * 8 > 129e6
                              else f"inputs smaller than L2 (A = {n * n * 8 / 2 ** 20:.0f} MiB FP64), not flushed"),
                       "parallelism": "replicas" if ws > 1 else "1 gpu"},
            "scaled_residual": res,
            "paper_residual": res_paper,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "phases_ms_per_step": phases_ms,
            "profiled_ms_per_step": profiled_ms,
            "clocks": ck,
            "mixed": mixed_line,
            "paper_nopiv": nopiv_line,
            "f64_ozaki": ozaki_line,
            "batched": batched_line,
            "served": served_line,
            "measured_rates": rates,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--nb", type=int, default=None, help="block width override (0 = library default)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision companion measurement")
    ap.add_argument("--rate", type=float, default=None, help="served: offered requests per second")
    ap.add_argument("--seconds", type=float, default=None, help="served: seconds of arrivals")
    ap.add_argument("--slots", type=int, default=None, help="served: worker slots of the server")
    ap.add_argument("--no-served", action="store_true", help="skip the served companion of the default run")
    ap.add_argument("--served-seconds", type=float, default=60.0, help="served companion: seconds of arrivals")
    ap.add_argument("--served-low-rate", type=float, default=1500.0,
                    help="served companion: the lower offered rate reported beside 2000/s")
    args = ap.parse_args()
    cfg = WORKLOADS[args.workload]
    if args.workload.startswith("served"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the served workload has no CPU reference arm"}))
            return 0
        import torch
        torch.cuda.set_device(0)
        r = served_measure(dict(cfg, slots=args.slots) if args.slots else cfg, args.rate, args.seconds)
        line = {"metric": "served solves/s, p50/p99 latency ms", "value": r["solves_per_s"], "unit": "solves/s",
                "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": r["wall_s"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "fp16+f32acc+f64refine", "data": "synthetic",
                "config": {"workload": args.workload}, "served": r}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload.startswith("batched_"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU reference arm; "
                              "the oracle solves each system in tests/test_gpu_batched.py"}))
            return 0
        import torch
        from paper_2202_13995_gb300 import lu
        torch.cuda.set_device(0)
        stream = torch.cuda.current_stream()
        ctx = lu.Context(stream)
        r = batched_measure(ctx, stream, cfg, args.steps, args.warmup)
        ctx.close()
        line = {"metric": METRIC, "value": r["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64refine", "data": "synthetic",
                "config": {"workload": args.workload, "systems": cfg["count"]}, "batched": r,
                "gpu_launches": r["launches"]}
        print(json.dumps(line), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, cfg, args.workload)
    return run_ours(args, cfg, args.workload)


if __name__ == "__main__":
    sys.exit(main())
