#!/usr/bin/env python
"""Benchmark of the Chebyshev-filtered plane-wave eigensolver hot path on one or more GB300s.

Workload (default, FP64): cubic cell a = 20 bohr, Ecut = 20 Ha (34181 plane waves per k), FFT box
96^3, 64 seeded atoms (min separation 2 bohr) with the Gaussian V_loc and s+p projectors (256),
512 bands + 52 buffer bands, 4 shifted k-points, complex128.  One step = one Chebyshev-filtered
subspace iteration (degree-10 filter, H on the filtered block, FP64 Rayleigh-Ritz, residuals) on
every k-point.  Metric: band H-applications per second (one band-apply = H on one column).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed] [--impl ours|reference]

With --gpus N > 1 it must be launched by torchrun (one rank per GPU); every rank runs its own
independent copy of the workload (weak scaling, no collective on the data path; the process
group only carries the timing barrier and the max over ranks).  Rank 0 prints one JSON line.
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

FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; 152 SMs x 2 FMA per clock x 2 x 2070 MHz = 1.26)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz


def bf16_peak():
    """Dense BF16 tensor peak for a kernel timed inside a long step: the measured sustained cuBLAS
    figure of this machine pool when the measured-peaks file is present, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured (sustained cuBLAS BF16)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (sustained BF16)"


def hbm_peak():
    """HBM copy bandwidth of this machine pool (GB/s): the measured figure when the measured-peaks
    file is present, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--degree", type=int, default=None,
                    help="Chebyshev filter degree (default 10 for the c2 form, the paper's setting; "
                         "20 for the c3/c4/c5 full solves, where fewer Rayleigh-Ritz steps pay)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--nk", type=int, default=0, help="use only the first nk k-points (profiling)")
    ap.add_argument("--workload", choices=["c2", "c2s", "c3", "c4", "c5", "density", "lobpcg", "gemm", "dense",
                                           "apply"],
                    default="c2",
                    help="c2: default FP64 ChebFi iterations; c3/c4/c5: mixed-precision full solves, "
                         "batched and served forms; gemm: the path's complex products at the C2 "
                         "shapes; dense: the Rayleigh-Ritz eigensolve; apply: H on a large band "
                         "block of the config-1 cell (auxiliary lines)")
    ap.add_argument("--bands", type=int, default=16384, help="apply: bands in the block")
    ap.add_argument("--pin-schedule", default=None, metavar="AxB@T",
                    help="c2: pin the middle pass's schedule for the 96^3 box (split A x B at T threads) "
                         "instead of tuning it (profiling runs that must see the production schedule)")
    ap.add_argument("--no-graph", action="store_true",
                    help="c4/c5: issue the batch filter's launches directly instead of replaying a CUDA "
                         "graph, so that the kernel table times every launch (profiling)")
    ap.add_argument("--requests", type=int, default=60, help="c5: number of requests")
    ap.add_argument("--systems", type=int, default=48, help="c4: systems in the batch (48: config 4; "
                                                                "fewer: a small case for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2 line without the full-solve, config-3 and served measurements")
    args = ap.parse_args()
    if args.degree is None:
        args.degree = 10 if args.workload in ("c2", "c2s", "lobpcg") else 20
    if args.workload == "c2s":
        args.no_cpu_baseline = True  # the oracle applies S^-1 by a dense solve: infeasible at npw 34181
    return args


# ------------------------------------------------------------------------------------------------
# workload description (shared by both arms)

def workload(name: str = "c2"):
    import workloads as W
    return W.config2s(nk=4) if name == "c2s" else W.config2()


def workload_name(s, nb, form):
    if s.Q is not None:
        return (f"C2S ({form}): the C2 cell (a=20 bohr, Ecut=20 Ha, FFT 96^3, npw=34181/k, "
                f"{s.nproj} projectors, {s.nband} bands + {nb - s.nband} buffer, {len(s.kpts)} "
                f"shifted k-points) with the nonlocal overlap S = 1 + sum |beta> q <beta|, "
                f"q ~ U[0,0.5]; step = one generalised ChebFi iteration (degree-10 filter in "
                f"S^-1 H + H on the filtered block + FP64 Rayleigh-Ritz with metric Y^H S Y + "
                f"residuals |Hx - lambda Sx|) on every k-point; a band-apply is one column of "
                f"S^-1 H psi (filter) or H psi")
    return (f"C2 ({form}): cubic a=20 bohr, Ecut=20 Ha, FFT 96^3, npw=34181/k, 64 atoms x (s,p) = "
            f"{s.nproj} projectors, {s.nband} bands (+{nb - s.nband} buffer), "
            f"{len(s.kpts)} shifted k-points; step = one ChebFi iteration (degree-10 filter + "
            f"H on filtered block + FP64 Rayleigh-Ritz + residuals) on every k-point")


# ------------------------------------------------------------------------------------------------
# clocks sampler

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)

def oracle_setup(s, ik=0):
    import oracle as O
    box = tuple(s.fft_box)
    return O.build_problem(s, ik, box=box, V=O.vloc_for(s, box))


def oracle_rate(problem, seconds: float, batch: int = 4, max_bands: int = 10 ** 9):
    """Band H-applications per second of the oracle's naive-DFT apply, over a bounded sample."""
    import workloads as W
    t0 = time.perf_counter()
    n = 0
    while True:
        c = W.random_block(problem.basis.npw, batch, seed=100 + n)
        problem.apply(c)
        n += batch
        el = time.perf_counter() - t0
        if el >= seconds or n >= max_bands:
            return n / el, n, el


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args, rank: int):
    """Reference arm: the FP64 oracle on the host cores, same metric / config / unit."""
    if rank != 0:
        return
    s = workload()
    p = oracle_setup(s)
    for _ in range(args.warmup):
        oracle_rate(p, 0.0, batch=2, max_bands=2)
    rates = []
    t_all = 0.0
    bands = 0
    for _ in range(args.steps):
        r, n, el = oracle_rate(p, 0.0, batch=4, max_bands=4)
        rates.append(r)
        t_all += el
        bands += n
    value = bands / t_all
    nb = s.nband + max(4, math.ceil(s.nband / 10))
    sample = f"{bands} bands of k-point 0 in {args.steps} steps of 4 (naive-DFT H-apply, dense projector products)"
    line = {
        "impl": "reference", "metric": "band H-applies/s", "value": value, "unit": "band-applies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(s, nb, "fp64"),
                   "reference": "FP64 CPU oracle (the paper prints no code); host cores only"},
        "cpu_baseline": {"value": value, "unit": "band-applies/s", "cores": cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "band-applies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU arm

# DRAM bytes per band of the middle FFT pass on the C2 workload, from one ncu capture of two
# production launches each (dram__bytes_read.sum + dram__bytes_write.sum, mean of the two):
# pass_bw<double, 8, 12, 384> moved 73.53 + 7.28 MB per 27-band launch, pass_bw<float, 12, 8, 384>
# 69.94 + 6.15 MB per 54-band launch.  Valid for that kernel and schedule only (the bench reports
# null traffic when the autotuner picked another).
# ncu DRAM bytes per band of the middle pass (production schedule 12 x 8 at 384 threads, pruned
# stages) with the L2 state the step leaves (--cache-control none; a full-chunk production launch:
# profiles/c2_pass_b_dram_traffic.md)
PASS_B_DRAM_PER_BAND = {"fp64": (19.000832e6 + 47.424256e6) / 27, "mixed": (9.314304e6 + 41.612032e6) / 54}
PASS_B_SCHEDULE = {"fp64": "12x8 @384", "mixed": "12x8 @384"}
# FP instructions the middle pass executes per band (ncu counts: 2 per FMA, 1 per add / multiply)
# over the dense-transform count 4 x 5 N^3 log2 N, for the production schedule (12 x 8 at 384
# threads with the pruned strided stages, CW = 3)
PASS_B_EXECUTED_PER_ALGORITHMIC = {"fp64": (2 * 349526016 + 685449216 + 207194112) / 27 / (4 * 5 * 96 ** 3 * math.log2(96)),
                                   "mixed": (2 * 707014656 + 1399762944 + 439271424) / 54 / (4 * 5 * 96 ** 3 * math.log2(96))}


def algorithmic_work(s, npw, nb, degree, box, applies, rr_calls):
    """Algorithmic FLOPs per kernel family over the timed region (conventional counts:
    5 N log2 N per complex 1D FFT of length N, 8 flops per complex multiply-add)."""
    N = box[0]
    fft_axis = 5.0 * N ** 3 * math.log2(N)        # one axis of one 3D transform, one band
    nl = 8.0 * s.nproj * npw                        # one projector GEMM, one band
    gram = 8.0 * nb * nb * npw                      # one Gram-class GEMM
    return {
        "local_pass_a": applies * fft_axis,
        "local_pass_b": applies * 4 * fft_axis,
        "local_pass_c": applies * fft_axis,
        "gemm_cn_partial:cprj": applies * nl,
        "gemm_nn:nonlocal": applies * nl,
        "gemm_cn_partial:gram": rr_calls * 2 * gram,
        "gemm_nn:rotate": rr_calls * 2 * gram,
        "tc_gemm_oz7:cprj": applies * nl,
        "tc_gemm_oz7:nonlocal": applies * nl,
        "tc_gemm_oz7:gram": rr_calls * 2 * gram,
        "tc_gemm_oz7:rotate": rr_calls * 2 * gram,
    }


def fft_path_hbm(fam, applies, npw, word_bytes, hbm_gbs):
    """HBM view of the local part (passes A, B and C together): its algorithmic bytes, psi in and
    H psi out once per band-apply (2 npw complex words), over the summed event time of the three
    pass families, against the measured copy bandwidth.  The passes keep the box in shared
    memory and the slab in L2, so the figure shows how far below the HBM bound they run."""
    fams = [f for f in ("local_pass_a", "local_pass_b", "local_pass_c") if f in fam]
    ms = sum(fam[f][1] for f in fams)
    if not fams or ms <= 0:
        return None
    gbs = applies * 2.0 * npw * word_bytes / (ms / 1000.0) / 1e9
    return {"kernels": "+".join(fams), "algorithmic_bytes_per_band": 2 * npw * word_bytes,
            "achieved_gbs": gbs, "peak_gbs": hbm_gbs, "frac": gbs / hbm_gbs,
            "note": "ALU-bound, not HBM-bound: the transforms stay in shared memory and L2"}


# The FP64 products run on the BF16 tensor cores as 28 exact digit products (7 BF16 digits per
# FP64 value, the digit pairs p + q <= 8) of a real GEMM with twice the rows and twice the K of
# the complex one: 28 * 2 (2M) N (2K) = 224 M N K executed BF16 flops, 28 times the conventional
# 8 M N K count of the complex FP64 product.
OZ_EXECUTED_PER_CONVENTIONAL = 28.0


def family(name: str) -> str:
    """Kernel family of a profile entry: the name without template arguments, with its tag
    ("gemm_cn_partial<f64>:cprj" -> "gemm_cn_partial:cprj", "local_pass_b<f32>" -> "local_pass_b")."""
    base = name.split("<")[0].split(":")[0]
    tag = name.split(":", 1)[1] if ":" in name else ""
    return base + (":" + tag if tag else "")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_values(name: str):
    """Stored oracle eigenvalues (written by tests/golden/make_golden*.py from the FP64 oracle's
    dense LAPACK eigensolve), or None when the file is absent."""
    import numpy as np
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return np.array([float(l) for l in f if l.strip() and not l.startswith("#")])


def timed_solve(K, torch, sysh, ik, nband, opts, ref=None, evecs=None):
    """One full kss_chebfi_solve timed with CUDA events on the context stream; eigenvalue error
    against stored oracle eigenvalues when given."""
    import numpy as np
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ev, rs, st, code = K.kss_chebfi_solve(sysh, ik, nband, opts, evecs=evecs, allow_noconv=True)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0
    out = {"solves_per_s": 1.0 / sec, "s_per_solve": sec, "iterations": st["iters"],
           "band_applies": st["napply"], "ms_filter": st["ms_filter"], "ms_rayleigh_ritz": st["ms_rr"],
           "status": "converged" if code == K.KSS_OK else f"status {code}",
           "max_residual_Ha": float(rs.max())}
    if ref is not None:
        out["max_eig_err_vs_oracle_Ha"] = float(np.max(np.abs(np.sort(ev) - ref[: ev.size])))
    return out


def serve(K, torch, ctx, reqs, degree, clocks=None):
    """Run the request server over reqs (arrival times in seconds from the start); returns
    (seconds, server stats, per-request results)."""
    opts = K.make_opts(prec=K.KSS_PREC_MIXED, seed=5, degree=degree)
    K.kss_server_start(ctx, 150 << 30, 512, opts)
    tickets, done = {}, {}
    if clocks is not None:
        clocks.start()
    t0 = time.perf_counter()
    i = 0
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].t_arrival <= now:
            s = reqs[i].system
            tickets[i] = K.kss_server_submit(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, s.nband,
                                             fft_box=s.fft_box or (0, 0, 0))
            i += 1
        K.kss_server_pump(ctx, 5.0)
        for j, t in list(tickets.items()):
            if j in done:
                continue
            s = reqs[j].system
            r = K.kss_server_poll(ctx, t, len(s.kpts), s.nband)
            if r is not None:
                done[j] = r
        if i < len(reqs) and not tickets.keys() - done.keys():
            time.sleep(max(0.0, reqs[i].t_arrival - (time.perf_counter() - t0)))
    dt = time.perf_counter() - t0
    stats = K.kss_server_get_stats(ctx)
    K.kss_server_stop(ctx)
    return dt, stats, done


def run_extras(K, torch, ctx, degree: int = 20, nreq: int = 60):
    """The rest of the metric beside the headline rate: eigensolves/s of full solves with their
    eigenvalue error against the oracle's stored dense eigenvalues (config 2 at its first k-point
    in FP64 and in the mixed form; config 3), and the served mixed form (config 5) with p50/p99
    latency at the configured arrival rate and at a sustainable one, against the plain FP64
    per-request path."""
    import workloads as W
    out = {}
    s = W.config2()
    s.kpts = s.kpts[:1]
    sysh = K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=s.fft_box)
    ref = golden_values("c2_k0_lowest576_Ha.txt")
    out["c2_k0_fp64"] = timed_solve(K, torch, sysh, 0, s.nband,
                                    K.make_opts(degree=degree, tol=1e-8, max_iter=400, seed=5), ref)
    out["c2_k0_mixed"] = timed_solve(K, torch, sysh, 0, s.nband,
                                     K.make_opts(degree=degree, tol=3e-5, max_iter=400, seed=5,
                                                 prec=K.KSS_PREC_MIXED), ref)
    out["c2_k0_mixed"]["speedup_vs_fp64"] = out["c2_k0_mixed"]["solves_per_s"] / out["c2_k0_fp64"]["solves_per_s"]
    out["c2_what"] = ("config 2 at k = (1/4,1/4,1/4): 512 bands (+52 buffer) of 34181 plane waves, "
                      f"degree-{degree} ChebFi from a random block to residual 1e-8 (FP64) or 3e-5 "
                      "(mixed: complex64 filter, split-BF16 tensor-core projector products, FP64 "
                      "Rayleigh-Ritz and FP64 finish); oracle = the 576 lowest eigenvalues of the "
                      "dense 34181^2 H (LAPACK, tests/golden/c2_k0_lowest576_Ha.txt)")
    K.kss_sys_destroy(sysh)
    s = W.config3()
    sysh = K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=s.fft_box)
    ref3 = golden_values("c3_lowest1024_Ha.txt")
    o3 = K.make_opts(degree=degree, prec=K.KSS_PREC_MIXED, seed=11)
    K.kss_chebfi_solve(sysh, 0, s.nband, o3, allow_noconv=True)  # warm-up (autotune, workspaces)
    out["c3_mixed"] = timed_solve(K, torch, sysh, 0, s.nband, o3, ref3)
    out["c3_what"] = ("config 3: the config-1 cell (1503 plane waves, Gamma) with 1024 bands, mixed "
                      "form; oracle = the dense 1503^2 H's lowest 1024 eigenvalues (tests/golden)")
    K.kss_sys_destroy(sysh)
    reqs = W.config5(nreq=nreq)
    dt, st, done = serve(K, torch, ctx, reqs, degree)
    served = {"requests": len(reqs), "arrival_rate_per_s": 200.0, "solves_per_s": len(reqs) / dt,
              "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
              "all_ok": all(d[0] == K.KSS_OK for d in done.values()),
              "max_residual_Ha": float(max(d[2].max() for d in done.values()))}
    rate = 0.7 * served["solves_per_s"]
    reqs2 = W.config5(nreq=max(8, nreq // 3), rate=rate)
    dt2, st2, done2 = serve(K, torch, ctx, reqs2, degree)
    sustain = {"requests": len(reqs2), "arrival_rate_per_s": rate, "solves_per_s": len(reqs2) / dt2,
               "p50_ms": st2["p50_ms"], "p99_ms": st2["p99_ms"],
               "all_ok": all(d[0] == K.KSS_OK for d in done2.values())}
    sample = [r.system for r in reqs[:3]]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for sy in sample:
        h = K.kss_setup(ctx, sy.lattice, sy.ecut, sy.kpts, sy.pos, sy.D, fft_box=sy.fft_box or (0, 0, 0))
        for ik in range(len(sy.kpts)):
            K.kss_chebfi_solve(h, ik, sy.nband, K.make_opts(seed=3, degree=degree), allow_noconv=True)
        K.kss_sys_destroy(h)
    torch.cuda.synchronize()
    fp64_rate = len(sample) / (time.perf_counter() - t1)
    out["c5_served_mixed"] = served
    out["c5_served_mixed_sustainable_rate"] = sustain
    out["c5_plain_fp64_per_request"] = {"solves_per_s": fp64_rate, "requests": len(sample),
                                        "what": "the first requests solved one by one (kss_setup + "
                                                "FP64 kss_chebfi_solve per k-point)"}
    out["c5_served_vs_plain_fp64"] = served["solves_per_s"] / fp64_rate
    out["c5_what"] = ("config 5: Poisson arrivals (seed 1005), 90% config-4-distribution and 10% "
                      "config-1-size systems, 25% repeats (warm start), 150 GB admission budget; "
                      "the sustainable-rate run uses 0.7 x the measured service rate, so its "
                      "latency is service time rather than backlog")
    return out


def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_2507_08578_gb300 import multi as MR

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return MR.max_over_ranks(x, dist, "cuda")

    def sum_over_ranks(x: float) -> float:
        return MR.sum_over_ranks(x, dist, "cuda")

    # CPU baseline first (rank 0, N = 1 only), before the GPU is busy.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s0 = workload(args.workload)
        p = oracle_setup(s0)
        r, n, el = oracle_rate(p, args.cpu_seconds)
        cpu = {"value": r, "unit": "band-applies/s", "cores": cores(), "kind": "oracle",
               "sample": f"{n} bands of k-point 0 of the same workload, naive-DFT H-apply + dense "
                         f"projector products, {el:.1f} s of CPU time"}

    B.build()
    stream = torch.cuda.current_stream()
    ctx = K.kss_create(local_rank, stream.cuda_stream)
    s = workload(args.workload)
    prec = K.KSS_PREC_FP64 if args.form == "fp64" else K.KSS_PREC_MIXED
    if args.pin_schedule:
        ab, nt = args.pin_schedule.split("@")
        a_, b_ = (int(v) for v in ab.split("x"))
        K.kss_autotune_put(local_rank, prec, 96, 96, 40, a_, b_, int(nt))
    if args.nk > 0:
        s.kpts = s.kpts[: args.nk]
    sysh = K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=s.fft_box, Q=s.Q)
    nk = len(s.kpts)
    solvers = []
    for ik in range(nk):
        opts = K.make_opts(degree=args.degree, tol=1e-30, max_iter=1 << 30, prec=prec, seed=17 + ik)
        sv = K.kss_solver_create(sysh, ik, s.nband, opts)
        K.kss_solver_step(sv)  # initial Rayleigh-Ritz on the starting block (setup)
        solvers.append(sv)
    npw = K.kss_sphere(sysh, 0).shape[0]
    nb = K.kss_solver_results(solvers[0])[2]["nb"]

    def napply_total():
        return sum(K.kss_solver_results(sv)[2]["napply"] for sv in solvers)

    # The k-points are stepped together: the Rayleigh-Ritz of one (latency-bound dense FP64
    # eigensolve) runs on a helper stream beside the filter of the next.
    for _ in range(args.warmup):
        K.kss_solver_step_many(solvers)

    # ---- timed region (device time, CUDA events on the launching stream) ----
    clocks = Clocks(local_rank)
    a0 = napply_total()
    barrier()
    clocks.start()
    K.kss_profile_enable(ctx, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        K.kss_solver_step_many(solvers)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = K.profile_table(ctx)
    _, launches = K.kss_profile_count(ctx)
    K.kss_profile_enable(ctx, False)
    applies = napply_total() - a0
    ms_max = max_over_ranks(ms)
    total_applies = sum_over_ranks(applies)
    value = total_applies / (ms_max / 1000.0)
    resid = max(K.kss_solver_results(sv)[1].max() for sv in solvers)

    # ---- roofline of the dominant kernel ----
    rr_calls = args.steps * nk
    work = algorithmic_work(s, npw, nb, args.degree, tuple(s.fft_box), applies, rr_calls)
    fam = {}
    for name, (l, kms) in prof.items():
        f = family(name)
        L, M = fam.get(f, (0, 0.0))
        fam[f] = (L + l, M + kms)
    # the dominant CUDA-core (ALU-bound) family with an algorithmic count: the FFT passes (the
    # dense eigensolve has no count, and with one k-point in the mixed form it can take as long
    # as the middle pass; the tensor-core products have their own lines below)
    top = max(fam, key=lambda f: fam[f][1])
    counted = [f for f in fam if f in work and f.startswith("local_pass")]
    dom = max(counted, key=lambda f: fam[f][1]) if counted else top
    dl, dms = fam[dom]
    peak = FP64_PEAK_TFLOPS if args.form == "fp64" else FP32_PEAK_TFLOPS
    # the CUDA cores' FMA throughput measured on this device right after the timed region
    probe = K.kss_peak_probe(ctx, 0 if args.form == "fp64" else 1)
    roof = None
    if dom in work and dms > 0:
        ach = work[dom] / (dms / 1000.0) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_note": ("FP64 CUDA-core rate derived from the unit counts and clock: 152 SMs x "
                              "2 FP64 FMA per clock x 2 flops x 2070 MHz = 1.26, nominal 1.25"
                              if args.form == "fp64" else
                              "FP32 CUDA-core rate derived from 152 SMs x 128 lanes x 2 x 2070 MHz"),
                "measured_peak": probe, "frac_of_measured": ach / probe,
                "measured_note": "kss_peak_probe in this run: independent FMA chains, 8 CTAs per SM, "
                                 "best of three launches",
                "launches": dl, "avg_launch_ms": dms / dl}
        if top != dom:
            roof["longest_family"] = {"kernel": top, "ms": fam[top][1],
                                      "note": "the longest kernel family of the step is not an FFT pass"}
        roof["fft_path_hbm"] = fft_path_hbm(fam, applies, npw, 16 if args.form == "fp64" else 8, hbm_peak()[0])
        sched_now = [f"{e['A']}x{e['B']} @{e['threads']}" for e in K.kss_autotune_table() if e["N"] == 96]
        if dom == "local_pass_b" and args.workload == "c2" and sched_now and \
                all(x == PASS_B_SCHEDULE[args.form] for x in sched_now):
            # FP instructions the pruned pass executes (ncu counts of this schedule) over the
            # dense-transform count: the executed rate against the measured FMA throughput
            roof["executed_per_algorithmic"] = PASS_B_EXECUTED_PER_ALGORITHMIC[args.form]
            roof["executed_frac_of_measured"] = ach * PASS_B_EXECUTED_PER_ALGORITHMIC[args.form] / probe

    # ---- the FP64 products on the tensor cores (FP64 form) ----
    fp64_gemm = None
    oz_fams = [f for f in ("tc_gemm_oz7:cprj", "tc_gemm_oz7:nonlocal", "tc_gemm_oz7:gram", "tc_gemm_oz7:rotate")
               if f in fam and f in work]
    if args.form == "fp64" and oz_fams:
        ol = sum(fam[f][0] for f in oz_fams)
        oms = sum(fam[f][1] for f in oz_fams)
        alg = sum(work[f] for f in oz_fams)
        ach = alg / (oms / 1000.0) / 1e12
        pk, pnote = bf16_peak()
        fp64_gemm = {"kernel": "tc_gemm_oz7 (cprj + nonlocal + gram + rotate)", "bound": "tensor",
                     "achieved_fp64_equivalent": ach, "unit": "TFLOP/s",
                     "vs_fp64_peak": ach / FP64_PEAK_TFLOPS,
                     "executed_bf16": ach * OZ_EXECUTED_PER_CONVENTIONAL, "peak": pk, "peak_note": pnote,
                     "frac": ach * OZ_EXECUTED_PER_CONVENTIONAL / pk,
                     "executed_note": "7-digit error-free splitting: 28 BF16 digit products per FP64 "
                                      "product, each as many flops as the conventional complex count",
                     "launches": ol, "avg_launch_ms": oms / ol,
                     "share_of_step": oms / ms if ms > 0 else None}

    # ---- the projector products on the tensor cores (mixed form) ----
    proj = None
    tc_fams = [f for f in ("tc_gemm_bf16x3:cprj", "tc_gemm_bf16x3:nonlocal") if f in fam]
    if args.form == "mixed" and tc_fams:
        tl = sum(fam[f][0] for f in tc_fams)
        tms = sum(fam[f][1] for f in tc_fams)
        alg = len(tc_fams) * applies * 8.0 * s.nproj * npw  # conventional complex count per product
        ach = alg / (tms / 1000.0) / 1e12
        pk, pnote = bf16_peak()
        proj = {"kernel": "tc_gemm_bf16x3 (cprj + nonlocal)", "bound": "tensor", "achieved": ach,
                "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "peak_note": pnote,
                "executed_frac": 3 * ach / pk,
                "executed_note": "split BF16: three BF16 products (hi*hi, hi*lo, lo*hi) per "
                                 "complex64 product, each as many flops as the conventional count",
                "launches": tl, "avg_launch_ms": tms / tl}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
        es = 16 if prec == K.KSS_PREC_FP64 else 8
        hosts = []
        for ik, sv in enumerate(solvers):
            X = torch.empty((s.nband, npw), dtype=cdt, device="cuda")
            K.kss_solver_results(sv, X)
            hosts.append(X.cpu().pin_memory())
        dev = [torch.empty((s.nband, npw), dtype=cdt, device="cuda") for _ in range(nk)]
        h2d = d2h = 0
        napp = 0
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.e2e_steps):
            svs = []
            for ik in range(nk):
                dev[ik].copy_(hosts[ik], non_blocking=True)
                h2d += hosts[ik].numel() * es
                opts = K.make_opts(degree=args.degree, tol=1e-30, max_iter=1 << 30, prec=prec,
                                   seed=99 + ik, x0=dev[ik], x0_nb=s.nband, x0_ld=npw)
                svs.append(K.kss_solver_create(sysh, ik, s.nband, opts))
            K.kss_solver_step_many(svs)  # initial Rayleigh-Ritz on each warm start
            K.kss_solver_step_many(svs)  # one filter iteration each
            for ik, sv in enumerate(svs):
                ev, rs, st = K.kss_solver_results(sv, dev[ik])
                napp += st["napply"]
                K.kss_solver_destroy(sv)
                hosts[ik].copy_(dev[ik], non_blocking=True)
                d2h += hosts[ik].numel() * es + ev.nbytes + rs.nbytes
        t1.record(stream)
        barrier()
        ems = max_over_ranks(t0.elapsed_time(t1))
        e2e = {"value": sum_over_ranks(napp) / (ems / 1000.0), "unit": "band-applies/s",
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps,
               "what": "per k-point: pinned host block -> device, kss_solver_create (warm start); "
                       "kss_solver_step_many twice (initial Rayleigh-Ritz, one filter iteration); "
                       "results -> host"}

    for sv in solvers:
        K.kss_solver_destroy(sv)
    K.kss_sys_destroy(sysh)
    # the schedules the tuners chose for this workload (before the extra workloads add theirs)
    table = K.kss_autotune_table()
    gemm_table = K.kss_autotune_gemm_table()
    extras = None
    if rank == 0 and world == 1 and args.workload == "c2" and not args.no_extras and args.nk == 0:
        extras = run_extras(K, torch, ctx)
    K.kss_destroy(ctx)
    # pass-B schedules the autotuner picked (box, window, split, threads per CTA; 0 = per-warp form)
    sched = [f"{e['N1']}x{e['N']}^2 W3<={e['W3']}: {e['A']}x{e['B']} @{e['threads']} "
             f"({e['ncand']} timed)" for e in table]
    c2_sched = [f"{e['A']}x{e['B']} @{e['threads']}" for e in table if e["N"] == 96 and e["N1"] == 96]
    if roof is not None and roof["kernel"] == "local_pass_b" and args.workload == "c2" and c2_sched and \
            all(x == PASS_B_SCHEDULE[args.form] for x in c2_sched):
        roof["traffic"] = PASS_B_DRAM_PER_BAND[args.form] * applies / roof["launches"]
        roof["traffic_note"] = ("DRAM bytes per launch: ncu bytes per band of this kernel and schedule (L2 as "
                                "the step leaves it) x the bands per launch of this run")

    if rank == 0:
        line = {
            "metric": "band H-applies/s", "value": value, "unit": "band-applies/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "c64+f64",
            "data": "synthetic",
            "config": {"workload": workload_name(s, nb, args.form),
                       "l2": f"inputs larger than L2: {4 * nk * npw * nb * (16 if args.form == 'fp64' else 8) / 1e9:.1f} GB of band blocks per step",
                       "parallelism": "independent replica per GPU" if world > 1 else "1 GPU",
                       "band_applies_per_step": applies / args.steps,
                       "k_points": "stepped together (kss_solver_step_many): the Rayleigh-Ritz of "
                                   "one k-point on a helper stream beside the filter of the next",
                       "fft_schedule": sched,
                       "gemm_schedule": [f"kind {e['kind']} {e['Mr']}x{e['Nr']} x {e['kblocks']} k-blocks: form "
                                         f"{e['form']}, {e['splits']} split(s)" for e in gemm_table]},
            "metric_family": "band H-applies/s & eigensolves/s at <=1e-6 Ha vs FP64 oracle; p50/p99 latency",
            "gpu_launches": launches,
            "clocks": ck,
            "roofline": roof,
            "roofline_projector_gemm": proj,
            "roofline_fp64_gemm": fp64_gemm,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "max_residual_after": float(resid),
            "eigensolves_and_served": extras,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# auxiliary workloads: C3 (mixed full solve), C4 (batched), C5 (served)

def _setup(K, ctx, s):
    return K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=s.fft_box or (0, 0, 0))


def run_c3(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    s = W.config3()
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    sysh = _setup(K, ctx, s)
    opts = K.make_opts(prec=K.KSS_PREC_MIXED, seed=11, degree=args.degree)
    for _ in range(args.warmup):
        K.kss_chebfi_solve(sysh, 0, s.nband, opts)
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    napply = 0
    for i in range(args.steps):
        ev, rs, st, _ = K.kss_chebfi_solve(sysh, 0, s.nband, K.make_opts(prec=K.KSS_PREC_MIXED, seed=20 + i, degree=args.degree))
        napply += st["napply"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ck = clocks.stop()
    ref = golden_values("c3_lowest1024_Ha.txt")
    K.kss_sys_destroy(sysh)
    K.kss_destroy(ctx)
    print(json.dumps({"metric": "eigensolves/s", "value": args.steps / dt, "unit": "solves/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True,
                      "dtype": "c64+f64", "data": "synthetic",
                      "config": {"workload": "C3: a=10 bohr, Ecut=10 Ha, 24^3, 1024 bands (+103), Gamma; "
                                             "mixed: complex64 filter, tensor-core split-BF16 projector "
                                             "GEMMs, FP64 Rayleigh-Ritz, FP64 finish"},
                      "band_applies_per_s": napply / dt, "iterations": st["iters"],
                      "max_eig_err_vs_oracle_Ha": None if ref is None else float(np.max(np.abs(ev - ref))),
                      "max_residual_Ha": float(rs.max()), "degree": args.degree, "clocks": ck}), flush=True)


def run_c4(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    from paper_2507_08578_gb300 import multi as MR
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    B.build()
    systems = W.config4(48)[:max(1, min(48, args.systems))]
    # (system, k-point) units, split across ranks by a greedy longest-processing-time assignment
    all_units = [(j, ik) for j, s in enumerate(systems) for ik in range(len(s.kpts))]
    costs = [MR.unit_cost(int(MR.npw_estimate(abs(np.linalg.det(systems[j].lattice)), systems[j].ecut)),
                          systems[j].nband, args.degree) for j, _ in all_units]
    mine = MR.lpt_partition(costs, world)[rank]
    ctx = K.kss_create(local_rank, torch.cuda.current_stream().cuda_stream)
    need = sorted({all_units[u][0] for u in mine})
    handles = {j: _setup(K, ctx, systems[j]) for j in need}
    units = [(handles[all_units[u][0]], systems[all_units[u][0]], all_units[u][1]) for u in mine]
    opts = K.make_opts(prec=K.KSS_PREC_MIXED, seed=7, degree=args.degree,
                       flags=K.KSS_SOLVE_BATCH_NO_GRAPH if args.no_graph else 0)
    args_b = ([u[0] for u in units], [u[2] for u in units], [u[1].nband for u in units])
    for _ in range(args.warmup):
        K.kss_solve_batch(ctx, *args_b, opts)
    clocks = Clocks(local_rank)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    K.kss_profile_enable(ctx, True)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ev, rs, st, _ = K.kss_solve_batch(ctx, *args_b, opts)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    dt = MR.max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    ck = clocks.stop()
    prof = K.profile_table(ctx)
    _, launches = K.kss_profile_count(ctx)
    K.kss_profile_enable(ctx, False)
    napply = MR.sum_over_ranks(sum(x["napply"] for x in st), dist, "cuda")
    iters = [x["iters"] for x in st]
    max_res = MR.max_over_ranks(float(max(r.max() for r in rs)) if rs else 0.0, dist, "cuda")
    for h in handles.values():
        K.kss_sys_destroy(h)
    K.kss_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    print(json.dumps({"metric": "eigensolves/s", "value": len(systems) * args.steps / dt,
                      "unit": "systems solved/s", "n_gpus": world, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
                      "higher_is_better": True, "dtype": "c64+f64", "data": "synthetic",
                      "config": {"workload": f"C4: {len(systems)} systems, {len(all_units)} (system,k) units in one "
                                             "lockstep batch (grouped launches, " +
                                             ("filter launched directly" if args.no_graph else "CUDA-graph filter") +
                                             "), mixed precision"},
                      "units_per_s": len(all_units) * args.steps / dt, "band_applies_per_s": napply * args.steps / dt,
                      "max_residual_Ha": max_res, "scaling": "strong" if world > 1 else None,
                      "partition": "greedy longest-processing-time over (system, k) units" if world > 1 else None,
                      "max_iterations": max(iters), "gpu_launches": launches,
                      "mean_iterations": sum(iters) / len(iters), "degree": args.degree,
                      "clocks": ck,
                      "kernels": {k: {"launches": v[0], "ms": round(v[1], 2)} for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][1])[:24]}}), flush=True)


def run_density(args):
    """Density build after the solve (Eq. nandtau) on the C2 cell: every k-point's 512 bands
    (random unit-norm blocks standing in for the converged ones) accumulated into n(r) on 96^3."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    s = W.config2()
    nk = len(s.kpts) if args.nk <= 0 else args.nk
    prec = K.KSS_PREC_FP64 if args.form == "fp64" else K.KSS_PREC_MIXED
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    sysh = K.kss_setup(ctx, s.lattice, s.ecut, s.kpts[:nk], s.pos, s.D, fft_box=s.fft_box)
    blocks = []
    for ik in range(nk):
        npw = K.kss_sphere(sysh, ik).shape[0]
        g = torch.Generator(device="cuda").manual_seed(90 + ik)
        x = torch.randn((s.nband, npw), dtype=cdt, device="cuda", generator=g)
        blocks.append(x / torch.linalg.vector_norm(x, dim=1, keepdim=True))
    occ = np.full(s.nband, 2.0 / nk)
    rho = torch.zeros((96, 96, 96), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        rho.zero_()
        for ik in range(nk):
            K.kss_density_accumulate(sysh, ik, blocks[ik], occ, rho, prec)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    K.kss_profile_enable(ctx, True)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    prof = K.profile_table(ctx)
    _, launches = K.kss_profile_count(ctx)
    K.kss_profile_enable(ctx, False)
    total = float(rho.sum().item()) * (20.0 ** 3) / 96 ** 3
    bands = s.nband * nk * args.steps
    # roofline of the density pass: the y and z inverse transforms (2 of the 3 axes) per band
    name = "density_pass<f64>" if prec == K.KSS_PREC_FP64 else "density_pass<f32>"
    roof = None
    if name in prof:
        l, kms = prof[name]
        ach = bands * 2 * 5.0 * 96 ** 3 * math.log2(96) / (kms / 1000.0) / 1e12
        peak = FP64_PEAK_TFLOPS if prec == K.KSS_PREC_FP64 else FP32_PEAK_TFLOPS
        roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "launches": l, "avg_launch_ms": kms / l}
    K.kss_sys_destroy(sysh)
    K.kss_destroy(ctx)
    print(json.dumps({"metric": "band densities/s", "value": bands / (ms / 1000.0), "unit": "bands/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
                      "ms_per_step": ms / args.steps, "higher_is_better": True,
                      "dtype": "f64" if prec == K.KSS_PREC_FP64 else "c64 (FP64 accumulation)",
                      "data": "synthetic",
                      "config": {"workload": f"density n(r) = sum w |psi(r)|^2 on the C2 cell (96^3), "
                                             f"{nk} k-points x {s.nband} bands per step, inputs resident in HBM"},
                      "electrons": total, "gpu_launches": launches, "clocks": ck, "roofline": roof,
                      "kernels": {k: {"launches": v[0], "ms": round(v[1], 2)} for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][1])}}), flush=True)


def run_apply(args):
    """H applied to one large band block of the config-1 cell (a = 10 bohr, Ecut = 10 Ha, 24^3 box,
    1503 plane waves): in the mixed form the local part is the fused single kernel (box held in
    shared memory), in FP64 the three-pass pipeline.  The block (16384 bands by default: 197 MB
    in complex64) is larger than L2, so every step reads psi from HBM."""
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    s = W.config1()
    prec = K.KSS_PREC_FP64 if args.form == "fp64" else K.KSS_PREC_MIXED
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    es = 16 if prec == K.KSS_PREC_FP64 else 8
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    sysh = _setup(K, ctx, s)
    npw = K.kss_sphere(sysh, 0).shape[0]
    nb = args.bands
    g = torch.Generator(device="cuda").manual_seed(77)
    psi = torch.randn((nb, npw), dtype=cdt, device="cuda", generator=g)
    hpsi = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        K.kss_apply_H(sysh, 0, psi, hpsi, prec)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    K.kss_profile_enable(ctx, True)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        K.kss_apply_H(sysh, 0, psi, hpsi, prec)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    prof = K.profile_table(ctx)
    _, launches = K.kss_profile_count(ctx)
    K.kss_profile_enable(ctx, False)
    bands = nb * args.steps
    N = s.fft_box[0]
    flops_band = 2 * 5.0 * N ** 3 * math.log2(N ** 3)  # dense 3D transforms, forward and inverse
    fam = "local_fused<f32>" if "local_fused<f32>" in prof else (
        "local_pass_b<f64>" if prec == K.KSS_PREC_FP64 else "local_pass_b<f32>")
    roof = None
    if fam in prof:
        l, kms = prof[fam]
        per_band = bands / l
        if fam == "local_fused<f32>":
            # the whole local part: psi in and H psi out once per band (2 npw complex64 words)
            ach_gbs = per_band * 2 * npw * es / (kms / l / 1000.0) / 1e9
            ach_tf = per_band * flops_band / (kms / l / 1000.0) / 1e12
            roof = {"kernel": fam, "bound": "alu", "achieved": ach_tf, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach_tf / FP32_PEAK_TFLOPS, "traffic": None,
                    "hbm_achieved_gbs": ach_gbs, "hbm_peak_gbs": hbm_peak()[0],
                    "hbm_frac": ach_gbs / hbm_peak()[0],
                    "note": "algorithmic bytes 2 npw x 8 B per band; FFT flops 2 x 5 N^3 log2 N^3 per band; "
                            "FP32 peak derived (152 SMs x 128 lanes x 2 x 2070 MHz)",
                    "launches": l, "avg_launch_ms": kms / l}
    K.kss_sys_destroy(sysh)
    K.kss_destroy(ctx)
    print(json.dumps({"metric": "band H-applies/s", "value": bands / (ms / 1000.0), "unit": "band-applies/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
                      "ms_per_step": ms / args.steps, "higher_is_better": True,
                      "dtype": "f64" if prec == K.KSS_PREC_FP64 else "c64 (split-BF16 projector products)",
                      "data": "synthetic",
                      "config": {"workload": f"H psi on the config-1 cell (a=10 bohr, Ecut=10 Ha, 24^3, {npw} "
                                             f"plane waves, 16 projectors), one block of {nb} bands per step, "
                                             f"inputs resident in HBM",
                                 "l2": f"inputs larger than L2: {nb * npw * es / 1e6:.0f} MB block"},
                      "gpu_launches": launches, "clocks": ck, "roofline": roof,
                      "kernels": {k: {"launches": v[0], "ms": round(v[1], 2)} for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][1])}}), flush=True)


def run_lobpcg(args):
    """ChebFi against LOBPCG (the paper's two GPU eigensolvers) on one k-point of a config-4
    system (a = 11.6 bohr, Ecut = 19.3 Ha, 60 atoms, 120 bands, npw 6358, box 45^3), FP64 to
    residual 1e-8: time to solution, iterations and H-applications of each."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    s = W.config4(1)[0]
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    sysh = K.kss_setup(ctx, s.lattice, s.ecut, s.kpts[:1], s.pos, s.D)
    out = {}
    evs = {}
    for name, fn, deg in (("chebfi", K.kss_chebfi_solve, args.degree), ("lobpcg", K.kss_lobpcg_solve, 0)):
        opts = K.make_opts(degree=deg or 10, tol=1e-8, seed=11)
        for _ in range(max(1, args.warmup // 3)):
            fn(sysh, 0, s.nband, opts)
        torch.cuda.synchronize()
        K.kss_profile_enable(ctx, True)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ev, rs, st, _ = fn(sysh, 0, s.nband, opts)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        _, launches = K.kss_profile_count(ctx)
        K.kss_profile_enable(ctx, False)
        evs[name] = ev
        out[name] = {"solves_per_s": 1.0 / dt, "s_per_solve": dt, "iterations": st["iters"],
                     "band_applies": st["napply"], "max_residual": float(rs.max()),
                     "gpu_launches": launches // args.steps}
    # refinement from a loose solve (residual 1e-3): ChebFi, LOBPCG and RMM-DIIS started from it
    npw = K.kss_sphere(sysh, 0).shape[0]
    nbuf = max(4, (s.nband + 9) // 10)
    X0 = torch.zeros((s.nband + nbuf, npw), dtype=torch.complex128, device="cuda")  # whole block
    K.kss_chebfi_solve(sysh, 0, s.nband + nbuf, K.make_opts(degree=args.degree, tol=1e-3, seed=11), evecs=X0)
    refine = {}
    for name, fn in (("chebfi", K.kss_chebfi_solve), ("lobpcg", K.kss_lobpcg_solve),
                     ("rmmdiis", K.kss_rmmdiis_solve)):
        opts = K.make_opts(degree=args.degree, tol=1e-8, seed=12, nbuffer=nbuf, x0=X0, x0_nb=s.nband + nbuf,
                           x0_ld=npw)
        fn(sysh, 0, s.nband, opts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ev, rs, st, _ = fn(sysh, 0, s.nband, opts)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        refine[name] = {"s_per_refine": dt, "iterations": st["iters"], "band_applies": st["napply"],
                        "max_residual": float(rs.max()),
                        "max_eigenvalue_difference_vs_full_Ha": float(np.max(np.abs(ev - evs["chebfi"])))}
    K.kss_sys_destroy(sysh)
    K.kss_destroy(ctx)
    print(json.dumps({"metric": "eigensolves/s", "value": out["chebfi"]["solves_per_s"],
                      "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "one k-point of config-4 system 0 (a=11.6 bohr, Ecut=19.3 Ha, 60 atoms, "
                                             "240 projectors, 120 bands, npw 6358, 45^3), FP64, residual 1e-8"},
                      "chebfi": out["chebfi"], "lobpcg": out["lobpcg"],
                      "lobpcg_over_chebfi_time": out["lobpcg"]["s_per_solve"] / out["chebfi"]["s_per_solve"],
                      "refine_from_1e-3": refine,
                      "max_eigenvalue_difference_Ha": float(np.max(np.abs(evs["chebfi"] - evs["lobpcg"])))}),
          flush=True)


def run_c5(args):
    import torch
    import workloads as W
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    reqs = W.config5(nreq=args.requests)
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    clocks = Clocks(0)
    dt, stats, done = serve(K, torch, ctx, reqs, args.degree, clocks)
    ck = clocks.stop()
    # plain FP64 per-request path on a sample of the same requests, for the comparison
    sample = [r.system for r in reqs[: min(6, len(reqs))]]
    t1 = time.perf_counter()
    for s in sample:
        h = _setup(K, ctx, s)
        for ik in range(len(s.kpts)):
            K.kss_chebfi_solve(h, ik, s.nband, K.make_opts(seed=3), allow_noconv=True)
        K.kss_sys_destroy(h)
    fp64_rate = len(sample) / (time.perf_counter() - t1)
    K.kss_destroy(ctx)
    statuses = [d[0] for d in done.values()]
    print(json.dumps({"metric": "eigensolves/s", "value": len(reqs) / dt, "unit": "requests solved/s",
                      "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "n_gpus": 1,
                      "higher_is_better": True, "dtype": "c64+f64", "data": "synthetic",
                      "config": {"workload": f"C5: {len(reqs)} requests, Poisson arrivals 200/s (seed 1005), "
                                             "90% C4-distribution and 10% C1-size systems, 25% repeats "
                                             "(warm start), 150 GB admission budget, mixed precision"},
                      "server_stats": stats, "all_ok": all(s_ == K.KSS_OK for s_ in statuses),
                      "statuses": {str(k): statuses.count(k) for k in set(statuses)}, "degree": args.degree,
                      "plain_fp64_per_request_solves_per_s": fp64_rate,
                      "plain_fp64_sample": f"first {len(sample)} requests, kss_chebfi_solve FP64 one by one",
                      "clocks": ck}), flush=True)


def run_gemm(args):
    """The path's complex products at their C2 shapes, through kss_gemm, in both precisions:
    projector coefficients beta^H psi (256 x 564 x 34181), nonlocal accumulate beta C' (34181 x 564 x
    256), Gram matrix Y^H Y (564 x 564 x 34181), rotation Y Q (34181 x 564 x 564).  Per call:
    operand preparation (digit planes / BF16 splits) + product; conventional 8 M N K flops."""
    import torch
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(5)
    shapes = [("cprj", 0, 256, 564, 34181), ("nonlocal", 1, 34181, 564, 256),
              ("gram", 0, 564, 564, 34181), ("rotate", 1, 34181, 564, 564)]
    out = {}
    stream = torch.cuda.current_stream()
    K.kss_profile_enable(ctx, True)
    for prec, cdt in ((K.KSS_PREC_FP64, torch.complex128), (K.KSS_PREC_MIXED, torch.complex64)):
        for name, op, M, N, Kd in shapes:
            A = torch.randn((M, Kd) if op == 0 else (Kd, M), dtype=cdt, device="cuda", generator=g)
            Bm = torch.randn((N, Kd), dtype=cdt, device="cuda", generator=g)
            C = torch.zeros((N, M), dtype=cdt, device="cuda")
            for _ in range(args.warmup):
                K.kss_gemm(ctx, op, A, Bm, C, 1.0, 0.0, prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                K.kss_gemm(ctx, op, A, Bm, C, 1.0, 0.0, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            key = ("fp64_" if prec == K.KSS_PREC_FP64 else "mixed_") + name
            out[key] = {"M": M, "N": N, "K": Kd, "op": "A^H B" if op == 0 else "A B", "ms": ms,
                        "tflops_conventional": 8.0 * M * N * Kd / ms / 1e9}
            del A, Bm, C
    prof = K.profile_table(ctx)
    K.kss_profile_enable(ctx, False)
    K.kss_destroy(ctx)
    pk, pnote = bf16_peak()
    for k, v in out.items():
        mult = OZ_EXECUTED_PER_CONVENTIONAL if k.startswith("fp64") else 3.0
        v["executed_bf16_tflops"] = v["tflops_conventional"] * mult
        v["frac_of_bf16_peak"] = v["executed_bf16_tflops"] / pk
    print(json.dumps({"metric": "complex GEMM TFLOP/s (conventional 8MNK)", "value": out["fp64_cprj"]["tflops_conventional"],
                      "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "f64 (7-digit BF16 products) / c64 (split BF16)",
                      "data": "synthetic", "config": {"workload": "C2 shapes of the path's complex products"},
                      "peak": pk, "peak_note": pnote, "shapes": out,
                      "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in
                                  sorted(prof.items(), key=lambda kv: -kv[1][1])}}), flush=True)


def run_dense(args):
    """The Rayleigh-Ritz eigensolve (kss_dense_hegv) at the orders of the solves: one 564 x 564
    pencil (C2: 512 + 52 bands), one 1127 x 1127 pencil (C3: real symmetric at the Gamma point,
    and the same order complex for comparison) and a batch of 217 pencils of orders 20-141 (the
    C4 units); random Hermitian A and Hermitian positive definite B."""
    import numpy as np
    import torch
    import paper_2507_08578_gb300.kss as K
    from paper_2507_08578_gb300 import build as B
    B.build()
    ctx = K.kss_create(0, torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(9)

    def pencil(n, real):
        dt = torch.float64 if real else torch.complex128
        a = torch.randn((n, n), dtype=dt, device="cuda", generator=g).to(torch.complex128)
        m = torch.randn((n, n), dtype=dt, device="cuda", generator=g).to(torch.complex128)
        A = (a + a.conj().T) / 2
        Bp = m @ m.conj().T / n + torch.eye(n, dtype=torch.complex128, device="cuda")
        return A.T.contiguous(), Bp.T.contiguous()

    out = {}
    rng = np.random.default_rng(5)
    cases = [("c2_564", [564], False), ("c3_1127_real", [1127], True), ("c3_1127_complex", [1127], False),
             ("c4_batch_217", list(rng.integers(20, 142, size=217)), False),
             ("single_141", [141], False), ("single_64", [64], False)]
    for name, ns, real in cases:
        src = [pencil(int(n), real) for n in ns]
        times = []
        for it in range(args.warmup + args.steps):
            As = [a.clone() for a, _ in src]
            Bs = [b.clone() for _, b in src]
            ws = [torch.zeros(int(n), dtype=torch.float64, device="cuda") for n in ns]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = K.kss_dense_hegv(ctx, As, Bs, ws, real=real)
            times.append(time.perf_counter() - t0)
            assert not np.any(info)
        ms = 1000.0 * float(np.median(times[args.warmup:]))
        out[name] = {"pencils": len(ns), "max_order": int(max(ns)), "real": real, "ms": ms}
        if len(ns) == 1:  # device-clock phase times of the last (grid-team) solve
            out[name]["phase_ms"] = {k: round(v, 3) for k, v in K.kss_dense_hegv_phase_ms(ctx).items()}
    K.kss_destroy(ctx)
    print(json.dumps({"metric": "dense FP64 generalised eigensolve time", "value": out["c2_564"]["ms"],
                      "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "Rayleigh-Ritz pencils of the C2, C3 and C4 solves"},
                      "cases": out}), flush=True)


def main():
    args = parse()
    if args.workload not in ("c2", "c2s") and args.impl == "ours":
        {"c3": run_c3, "c4": run_c4, "c5": run_c5, "density": run_density, "apply": run_apply,
         "lobpcg": run_lobpcg, "gemm": run_gemm, "dense": run_dense}[args.workload](args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
