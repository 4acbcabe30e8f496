"""The benchmark's host-side contract, checked on the CPU.

* `bench.py --impl reference` (the FP64 oracle on the host cores) prints exactly one JSON line
  with the metric, unit and config of the GPU arm, an `e2e` object with zero copy bytes and a
  `cpu_baseline` object describing the run;
* under a multi-rank launch only rank 0 prints it, the other ranks exit 0 without work;
* the kernel-family grouping and the algorithmic work counts that the roofline divides by.
"""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == "band H-applies/s" and line["unit"] == "band-applies/s"
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"].startswith("C2 (fp64)")
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert cb["sample"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"],
             env_extra={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_kernel_families():
    assert bench.family("local_pass_b<f64>") == "local_pass_b"
    assert bench.family("gemm_cn_partial<f32>:gram") == "gemm_cn_partial:gram"
    assert bench.family("tc_gemm_bf16x3:cprj") == "tc_gemm_bf16x3:cprj"
    assert bench.family("residual_norms") == "residual_norms"


def test_fft_path_hbm_figure():
    # 1000 band-applies of 1000 plane waves in FP64 (2 x 1000 x 16 B per band) over 1.0 s of the
    # three pass families: 32 MB/s; other families do not count
    fam = {"local_pass_a": (10, 100.0), "local_pass_b": (10, 800.0), "local_pass_c": (10, 100.0),
           "dense_hegv_grid": (1, 500.0)}
    h = bench.fft_path_hbm(fam, 1000, 1000, 16, 6682.0)
    assert h["algorithmic_bytes_per_band"] == 32000
    assert h["achieved_gbs"] == pytest.approx(0.032)
    assert h["frac"] == pytest.approx(0.032 / 6682.0)
    assert h["kernels"] == "local_pass_a+local_pass_b+local_pass_c"
    assert bench.fft_path_hbm({"dense_hegv_grid": (1, 5.0)}, 10, 10, 8, 6682.0) is None


def test_algorithmic_work_counts():
    class S:
        nproj = 256
    npw, nb, box, applies, rr = 34181, 564, (96, 96, 96), 10, 2
    w = bench.algorithmic_work(S(), npw, nb, 10, box, applies, rr)
    axis = 5.0 * 96 ** 3 * math.log2(96)
    assert w["local_pass_a"] == pytest.approx(applies * axis)
    assert w["local_pass_b"] == pytest.approx(4 * applies * axis)
    assert w["local_pass_c"] == pytest.approx(applies * axis)
    # the three passes together: one forward and one inverse dense 3D transform per band-apply,
    # 2 x 5 N^3 log2(N^3)
    total = w["local_pass_a"] + w["local_pass_b"] + w["local_pass_c"]
    assert total == pytest.approx(applies * 2 * 5.0 * 96 ** 3 * math.log2(96 ** 3))
    assert w["gemm_cn_partial:cprj"] == pytest.approx(applies * 8.0 * 256 * npw)
    assert w["gemm_nn:nonlocal"] == pytest.approx(applies * 8.0 * 256 * npw)
    assert w["gemm_cn_partial:gram"] == pytest.approx(rr * 2 * 8.0 * nb * nb * npw)


def test_bf16_peak_reads_the_measured_file_or_falls_back():
    pk, note = bench.bf16_peak()
    assert pk > 0 and ("measured" in note or "fallback" in note)
