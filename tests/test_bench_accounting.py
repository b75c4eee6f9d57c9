"""bench.py's accounting, checked on the CPU: the operation counts behind the
reported TFLOP/s, the roofline's algorithmic FLOPs and bytes, the derived FP64
pipe peak and the traffic scaling."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_hpl_flop_count():
    # (2/3) n^3 + 2 n^2 nrhs: 2.932e12 at n = 16384, one right-hand side
    assert math.isclose(bench.hpl_flops(16384, 1), 2.0 / 3.0 * 16384 ** 3 + 2.0 * 16384 ** 2, rel_tol=0)
    assert math.isclose(bench.hpl_flops(16384, 1), 2.932e12, rel_tol=1e-3)


def test_block_steps_sum_to_the_lu_count():
    """The per-step counts (panel, top solve, inner update) add up to the
    LU's 2/3 n^3 - n^2/2 - n/6 exactly (elimination of an n x n matrix)."""
    for n, nb in [(64, 64), (100, 32), (257, 64), (1024, 64)]:
        steps = sum(bench._block_step_flops(n, nb, s) for s in range(math.ceil(n / nb)))
        exact = 2.0 * n ** 3 / 3.0 - n ** 2 / 2.0 - n / 6.0
        assert math.isclose(steps, exact, rel_tol=1e-12), (n, nb, steps, exact)


def _prof(ms, launches):
    return {"gemm": (ms, launches)}


def test_fp64_roofline_flops_and_peak():
    """FP64 update: 2 m'^2 nb per launch (2.864e12 of the 2.932e12 at n = 16384,
    nb = 256, 97.7 %); the peak is 2 FP64 FMAs per clock per SM x 152 x 2.07 GHz."""
    n, nb = 16384, 256
    peaks = {"sm_max_mhz": 2070.0, "_source": "measured", "bf16_tflops": 1876.8}
    r = bench.gemm_roofline(_prof(1000.0, 63), n, nb, "f64", 1, peaks, "hpl_f64_n16384_nb256")
    flops = sum(2.0 * (n - k - nb) ** 2 * nb for k in range(0, n, nb) if n - k - nb > 0)
    assert math.isclose(flops, 2.864e12, rel_tol=1e-3)
    assert math.isclose(flops / bench.hpl_flops(n, 1), 0.977, abs_tol=1e-3)
    assert math.isclose(r["achieved"], flops / 1.0 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["peak"], 2 * 2 * 152 * 2.07e9 / 1e12, rel_tol=1e-12)
    assert r["bound"] == "alu"


def test_tensor_core_roofline_bytes():
    """BF16 update: 8 m' n' bytes of FP32 C read + write plus the 16-bit
    operands, against the measured copy bandwidth."""
    n, nb = 4096, 256
    peaks = {"hbm_gbs": 6674.2, "bf16_tflops_sustained": 1701.1, "_source": "measured"}
    r = bench.gemm_roofline(_prof(10.0, 15), n, nb, "bf16", 1, peaks, "x")
    b = sum(8.0 * (n - k - nb) ** 2 + 2.0 * 2 * (n - k - nb) * 256 for k in range(0, n, nb) if n - k - nb > 0)
    assert math.isclose(r["achieved"], b / 0.010 / 1e9, rel_tol=1e-12)
    assert r["bound"] == "hbm" and r["peak"] == 6674.2


def test_split_update_roofline_counts_36_products():
    n, nb = 2048, 256
    peaks = {"bf16_tflops_sustained": 1701.1, "_source": "measured"}
    r = bench.gemm_roofline(_prof(5.0, 7), n, nb, "f64", 1, peaks, "x", ozaki=True)
    flops = sum(2.0 * (n - k - nb) ** 2 * nb for k in range(0, n, nb) if n - k - nb > 0)
    assert math.isclose(r["achieved"], 36.0 * flops / 0.005 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["fp64_equiv_tflops"], flops / 0.005 / 1e12, rel_tol=1e-12)
    assert r["bound"] == "tensor"


def test_traffic_scales_the_measured_ratio():
    """traffic per launch = measured DRAM bytes / algorithmic bytes of the
    captured launches x this step's mean algorithmic bytes per update."""
    import json
    ratios = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    n, nb = 16384, 256
    r = bench.gemm_roofline(_prof(1000.0, 63), n, nb, "f64", 1, {"_source": "measured"}, "x")
    alg = [16.0 * (n - k - nb) ** 2 + 8.0 * 2 * (n - k - nb) * nb for k in range(0, n, nb) if n - k - nb > 0]
    want = ratios["gemm_simt_kernel<double>"]["ratio"] * sum(alg) / len(alg)
    assert math.isclose(r["traffic"], want, rel_tol=1e-12)
    assert r["traffic_over_algorithmic"] == ratios["gemm_simt_kernel<double>"]["ratio"]
    for k in ("gemm_simt_kernel<double>", "tc_gemm_kernel", "oz_gemm_kernel"):
        assert 0.5 < ratios[k]["ratio"] < 3.0 and "command" in ratios[k]


def test_reference_arm_line_has_the_contract_keys():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys of the bench contract."""
    import json
    import subprocess
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--ref-seconds", "0.5", "--workload", "hpl_f64_n1024_nb64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "hpl_f64_n1024_nb64" and d["metric"] == bench.METRIC
