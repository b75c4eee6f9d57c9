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
    # smaller cases of the same shapes (profiling captures)
    "hpl_f64_n4096_nb256": dict(n=4096, nb=256, prec="f64", nrhs=1, seed=2, shift=0.0),
    "hpl_mixed_bf16_n8192": dict(n=8192, nb=0, prec="bf16", nrhs=1, seed=3, shift=0.25),
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


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        lr = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(lr)
        dist.init_process_group("nccl")
        return dist.get_rank(), ws, lr
    return 0, 1, 0


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _block_step_flops(n: int, nb: int, s: int) -> float:
    """Operation count of block iteration s (panel, top solve, inner update)."""
    m = n - s * nb
    w = min(nb, m)
    panel = sum((m - j - 1) * (1 + 2 * (w - j - 1)) for j in range(w))
    trsm = float(w * (w - 1)) * (m - w)
    update = 2.0 * (m - w) * (m - w) * w
    return panel + trsm + update


def oracle_sample(cfg: dict, max_seconds: float = 20.0, A=None) -> dict:
    """Time the oracle on the host cores on a bounded sample of the same
    workload: the first block iterations of the blocked factorization."""
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
    return {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "seconds": round(t, 3),
            "sample": f"first {ks} of {nsteps} block iterations (panel, interchanges, top solve, inner update) "
                      f"of the n={n}, nb={nb} FP64 blocked LU; operation count of those iterations / wall time"}


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


def run_ours(args, cfg, wname):
    import torch
    from paper_2202_13995_gb300 import inputs as I
    from paper_2202_13995_gb300 import lu

    rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    peaks = load_peaks()
    n, nb, prec, nrhs = cfg["n"], cfg["nb"], cfg["prec"], cfg["nrhs"]
    shift = cfg["shift"] * n
    mixed = prec != "f64"
    flops = hpl_flops(n, nrhs)

    stream = torch.cuda.current_stream()
    ctx = lu.Context(stream)
    A = I.hpl_matrix_torch(n, cfg["seed"] + 1000 * rank, diag_shift=shift, device="cuda")
    B = I.hpl_rhs_torch(n, nrhs, cfg["seed"] + 1000 * rank, device="cuda")
    X = lu.colmajor_empty(n, nrhs)
    torch.cuda.synchronize()

    def step():
        f = ctx.factor(A, prec, nb, sync=False)
        if mixed:
            f.refine(A, B, X, 16.0, 50)
        else:
            X.copy_(B)
            f.solve_(X)
        f.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the library's stream)
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    l0 = ctx.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    barrier(ws)
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms, ws)

    # residual of the last solve (FP64, on the device)
    res = float(ctx.scaled_residual(A, X, B).max())

    # ---- roofline of the dominant kernel: the trailing update (GEMM)
    gemm_ms, gemm_n = prof["gemm"]
    gemm_flops = 0.0
    step_nb = nb or (256 if n >= 2048 else 64)
    for k in range(0, n, step_nb):
        rest = n - k - min(step_nb, n - k)
        if rest > 0:
            gemm_flops += 2.0 * rest * rest * min(step_nb, n - k)
    gemm_flops *= args.steps
    achieved = gemm_flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    if mixed:
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        peak_note = f"bf16_tflops_sustained of {peaks['_source']}" + (" (fp16 at the same nominal rate)" if prec == "fp16" else "")
        bound = "tensor"
    else:
        peak = peaks.get("bf16_tflops", 1876.8) * NOMINAL["f64"] / NOMINAL["bf16"]
        peak_note = f"bf16_tflops of {peaks['_source']} x nominal FP64/BF16 ratio 1.25/2250"
        bound = "alu"
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            traffic = json.load(open(tpath)).get(wname)
        except Exception:
            traffic = None
    roofline = {"bound": bound, "kernel": "gemm_tc_kernel" if mixed else "gemm_simt_kernel<double>",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if (achieved and peak) else None, "traffic": traffic,
                "peak_source": peak_note, "launches": gemm_n, "kernel_ms": gemm_ms / args.steps}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        Ah.copy_(A)
        Bh = torch.empty((nrhs, n), dtype=torch.float64).pin_memory().t()
        Bh.copy_(B)
        Xh = torch.empty((nrhs, n), dtype=torch.float64).pin_memory().t()
        Ad = lu.colmajor_empty(n, n)
        Bd = lu.colmajor_empty(n, nrhs)
        Xd = lu.colmajor_empty(n, nrhs)

        def e2e_step():
            Ad.copy_(Ah, non_blocking=True)
            Bd.copy_(Bh, non_blocking=True)
            f = ctx.factor(Ad, prec, nb, sync=False)
            if mixed:
                f.refine(Ad, Bd, Xd, 16.0, 50)
            else:
                Xd.copy_(Bd)
                f.solve_(Xd)
            Xh.copy_(Xd, non_blocking=True)
            f.free()

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ke = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, ws)
        e2e = {"value": flops * ws / (ems * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(A.numel() * 8 + n * nrhs * 8), "d2h_bytes_per_step": int(n * nrhs * 8)}
        del Ah, Bh, Xh, Ad, Bd, Xd

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_sample(dict(cfg, nb=nb or 256), max_seconds=args.cpu_seconds)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": flops * ws / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if not mixed else f"{prec}+f32acc+f64refine", "data": "synthetic",
            "config": {"workload": wname, "n": n, "nb": nb or "auto", "nrhs": nrhs, "precision": prec,
                       "matrix": f"uniform[-0.5,0.5]" + (f" + {cfg['shift']}*n*I" if shift else ""),
                       "l2": f"inputs larger than L2 (A = {n * n * 8 / 2 ** 30:.1f} GiB FP64)",
                       "parallelism": "replicas" if ws > 1 else "1 gpu"},
            "scaled_residual": res,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "phases_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in prof.items()},
            "clocks": ck,
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
    args = ap.parse_args()
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg, args.workload)
    return run_ours(args, cfg, args.workload)


if __name__ == "__main__":
    sys.exit(main())
