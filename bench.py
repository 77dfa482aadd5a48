#!/usr/bin/env python3
"""Benchmark of the rotation-voting hot path on GB300.

One step = one full solve (pair step, vote on every level, top-K, children,
fit) of the paper-scale workload: 1e6 pairs, 99% outliers, sigma 0.005,
delta 0.03, 128^3 coarse grid + 3 levels of 2x2x2 refinement of the top 16
cells (1.14e12 cell tests), in the FP16 hi/lo tensor-core form.

Prints ONE JSON line: metric / value (cell-correspondence tests per second,
whole job), rotations/s, p50/p99 solve latency, e2e through the C ABI with
pinned host buffers, the dominant kernel's roofline, clocks, and the oracle's
CPU baseline; beside them the other precision forms on the same workload and
the 1e5-pair, 64^3 + 3-level workload in the plain FP32 form.
`--impl reference` times the FP64 oracle on the host cores instead (the
reference arm).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-correspondence tests/sec and rotations/sec at 1 GB300; p50/p99 solve latency"
UNIT = "cell-correspondence tests/s"
WORKLOAD = "lowp_n1e6_128L3"
PRECISION = "fp16x2"
WORKLOAD_DESCS = {
    "lowp_n1e6_128L3": ("N=1e6 float32 unit pairs, 99% uniform outliers, inlier noise sigma=0.005, delta=0.03 rad; "
                        "128^3 coarse grid over the vector-part ball (1,136,840 cells) + 3 levels of 2x2x2 "
                        "subdivision of the top-16 cells; exact counts, EXCESS ranking, FP64 fit with 8 refits"),
    "fp32_n1e5_64L3": ("N=1e5 float32 unit pairs, 99% uniform outliers, inlier noise sigma=0.01, delta=0.03 rad; "
                       "64^3 coarse grid over the vector-part ball (146,864 cells) + 3 levels of 2x2x2 "
                       "subdivision of the top-16 cells; exact counts, EXCESS ranking, FP64 fit with 8 refits"),
    "small_n1e3_32": ("N=1e3 float32 unit pairs, 90% uniform outliers, inlier noise sigma=0.01, delta=0.03 rad; "
                      "32^3 grid, no refinement; exact counts, FP64 fit with 8 refits"),
}
FLOPS_PER_TEST = 20.0  # algorithmic: 10 multiply-adds of the (cell monomials . pair S entries) contraction
K16_FLOPS_PER_TEST = 32.0  # the contraction with K padded to 16 (one kind::f16 MMA K step)
# The tensor-core epilogue's CUDA-core bound: per 4 tests it issues 2 packed fma.rm.f32x2 sign
# counters (FMA pipe) and 2 three-input |D| minima (ALU pipe), 0.5 ALU-pipe instructions per
# test; the ALU pipe has 64 lanes per SM per clock (16 per scheduler, which also issues the
# FMA-pipe half): 152 x 64 x f_max / 0.5 tests/s.
EPI_ALU_INSTR_PER_TEST = 0.5
EPI_ALU_LANES_PER_SM = 64
# DRAM bytes (read + write) of one coarse-vote launch, from one ncu capture of the workload and
# precision named in the key.  A figure stands only while the kernel's source file hashes to the
# value it was captured with; otherwise the line reports null.
NCU_TRAFFIC = {
    ("lowp_n1e6_128L3", "fp16x2"): (5780432896 + 84005632, "k_vote_tc.cu",
                                    "ed71a6dcbfc176c6e07be02bd6c46998c7ab746d9170e3c4c18494b6bfe669fe"),
    ("fp32_n1e5_64L3", "fp16x2"): (26757376, "k_vote_tc.cu",
                                   "ed71a6dcbfc176c6e07be02bd6c46998c7ab746d9170e3c4c18494b6bfe669fe"),
    ("fp32_n1e5_64L3", "fp32"): (17170688, "k_vote_simt.cu",
                                 "7da99284336fef54f912b58e44b5284fab9b1d003d32dbeadaa929631cf286ca"),
}


def ncu_traffic(precision: str, workload: str):
    """Captured DRAM bytes per coarse-vote launch, or None (not captured, or kernel changed)."""
    import hashlib
    if (workload, precision) not in NCU_TRAFFIC:
        return None
    nbytes, src, digest = NCU_TRAFFIC[(workload, precision)]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2506_11547_gb300", "csrc", src)
    try:
        ok = hashlib.sha256(open(path, "rb").read()).hexdigest() == digest
    except OSError:
        ok = False
    return nbytes if ok else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=PRECISION)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the precision-form, batched and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--only-solve", action="store_true",
                    help="warm-up + timed solves only (a short, fixed launch sequence for profiler captures)")
    ap.add_argument("--profile-case", choices=["alg1_n1e5", "alg1_multi9", "pose_n5000"], default=None,
                    help="three calls of one Alg. 1 / peak / pose case and nothing else (for profiler captures)")
    return ap.parse_args()


def reduce_max(x: float, dist, device) -> float:
    """Maximum of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, max_elapsed_s: float) -> float:
    """Weak scaling: every rank runs `steps` steps of its own problem of the same
    shape; the job rate is all ranks' units over the slowest rank's time."""
    return units_per_step * steps * world / max_elapsed_s


def rank_problem(synth, workload: str, rank: int):
    """Rank r solves its own seeded instance (rep = r) of the workload's shape."""
    return synth.config_problem(workload, rep=rank)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 3.0  # start timing only once the sampler is producing samples
            while not self.lines and time.time() < t_end:
                time.sleep(0.01)
            self.skip = len(self.lines)  # samples taken before the timed region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "skip", 0):] or self.lines[-1:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _angle(q1, q2) -> float:
    """Angle between the rotations of two unit quaternions (for the report line)."""
    w = abs(sum(float(x) * float(y) for x, y in zip(q1, q2)))
    return 2.0 * math.atan2(math.sqrt(max(0.0, 1.0 - w * w)), w)


def percentile(xs, p):
    s = sorted(xs)
    if not s:
        return None
    k = min(len(s) - 1, max(0, int(math.ceil(p / 100.0 * len(s))) - 1))
    return s[k]


def cpu_oracle_rate(p, grid_n, seconds: float, threads: int, m_hint: int = 0):
    """Oracle (FP64 C, as it stands) vote over a bounded sample of coarse cells:
    tests/s on `threads` host threads.  m_hint > 0: the sample size a previous
    call settled on (skips the calibration)."""
    import numpy as np
    import oracle
    cells = oracle.level_cells(grid_n)
    rng = np.random.default_rng(0)
    order = rng.permutation(len(cells))
    # calibrate on a few cells, then size the sample to ~seconds; the short
    # calibration carries fixed costs, so a sample that ends well short of the
    # target is rescaled (at most twice) and timed again
    if m_hint > 0:
        m = int(min(len(cells), m_hint))
    else:
        m0 = max(threads, 8)
        t0 = time.perf_counter()
        oracle.vote_cells(p.a, p.b, float(np.float32(p.delta)), grid_n, cells[order[:m0]], nthreads=threads)
        dt0 = max(1e-3, time.perf_counter() - t0)
        m = int(min(len(cells), max(m0, m0 * seconds / dt0)))
    for attempt in range(3):
        t0 = time.perf_counter()
        oracle.vote_cells(p.a, p.b, float(np.float32(p.delta)), grid_n, cells[order[:m]], nthreads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds or m >= len(cells) or attempt == 2:
            break
        m = int(min(len(cells), m * seconds / max(dt, 1e-3)))
    return m * p.n / dt, m, dt


def bench_batched(rv, synth, torch, stream, flush, launches: int = 3):
    """4096 independent problems (N log-uniform in [50, 2e4], outliers U[0.5, 0.95],
    sigma U[0.001, 0.02], delta = 3 sigma; 32^3 + 2 levels) in one rot_vote_solve
    call: one pass of the pipeline over all of them, replayed from a CUDA graph."""
    probs = synth.batched_problems(4096)
    dev = [(torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda()) for p in probs]
    P = len(probs)
    arr = (rv.rot_vote_problem * P)()
    keep = []
    for k, p in enumerate(probs):
        arr[k], kk = rv.problem(dev[k][0], dev[k][1], p.delta)
        keep.append(kk)
    out = (rv.rot_vote_result * P)()
    res = {}
    for prec in ("fp16x2", "fp32"):
        ctx = rv.Context(grid_n=32, levels=2, precision=prec, cuda_stream=stream.cuda_stream)
        for _ in range(2):  # autotune + graph capture, then a replay
            ctx.solve_raw(arr, P, out)
        ts = []
        for _ in range(launches):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            ctx.solve_raw(arr, P, out)
            s1.record(stream)
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(s1))
        ctx.close()
        ms = sum(ts) / len(ts)
        tests = sum(int(out[k].tests) for k in range(P))
        res[prec] = {"value": tests / (ms / 1e3), "unit": "cell-correspondence tests/s",
                     "rotations_per_s": P / (ms / 1e3), "ms_per_call": ms, "problems": P,
                     "tests_per_call": tests, "status_ok": sum(int(out[k].status == 0) for k in range(P)),
                     "degenerate": sum(int(out[k].status == -6) for k in range(P))}
    res["workload"] = ("4096 problems, N log-uniform [50, 2e4] (sum N = %d), outliers U[0.5, 0.95], "
                       "sigma U[0.001, 0.02], delta = 3 sigma; 32^3 + 2 levels; one call (CUDA graph replay)"
                       % sum(p.n for p in probs))
    return res


def bench_alg1(rv, synth, torch, stream, flush, peaks, reps: int = 5):
    """Alg. 1 (Sec. 4.3.2) at the paper's default resolution (1/180: a 360^3
    accumulator) and J = 180, on 1e5 and 1e6 pairs with 99% outliers, and on 1e6
    pairs with 50% outliers, where the winning cell's count passes the 16-bit
    counters' 65536.  Device time per solve (inputs resident, L2 flushed before
    each), the end-to-end call with pinned host inputs, and each stage's time
    from a profiled run.  A context solving the wrapping problem after one
    without wraps votes twice (vote path 1, timed apart); solving it again, it
    votes once with the wrap record (path 2)."""
    res = {}
    prev = None
    for key, n, rho, sigma, seed in (("n100000", 100000, 0.99, 0.01, 2301), ("n1000000", 1000000, 0.99, 0.005, 2302),
                                     ("n1000000_outliers50", 1000000, 0.5, 0.005, 2303)):
        p = synth.make_problem(n, rho, sigma, 0.03, seed=seed)
        a_d, b_d = torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda()
        a_h, b_h = torch.from_numpy(p.a).pin_memory(), torch.from_numpy(p.b).pin_memory()
        arr = (rv.rot_vote_alg1_problem * 1)(rv.rot_vote_alg1_problem(a_d.data_ptr(), b_d.data_ptr(), n, 180, 360,
                                                                        None))
        arr_h = (rv.rot_vote_alg1_problem * 1)(rv.rot_vote_alg1_problem(a_h.data_ptr(), b_h.data_ptr(), n, 180, 360,
                                                                          None))
        out = (rv.rot_vote_alg1_result * 1)()
        ctx = rv.Context(cuda_stream=stream.cuda_stream)
        path1 = []
        if prev is not None:
            # vote path 1: the wrapping problem right after one without wraps (the previous
            # case, of the same size, so the workspace is already allocated)
            for _ in range(reps):
                ctx.alg1_raw(prev[0], 1, out)
                flush.zero_()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                ctx.alg1_raw(arr, 1, out)
                s1.record(stream)
                torch.cuda.synchronize()
                assert out[0].vote_path == 1
                path1.append(s0.elapsed_time(s1))
        for _ in range(3):
            ctx.alg1_raw(arr, 1, out)
        ts = []
        for _ in range(reps):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            ctx.alg1_raw(arr, 1, out)
            s1.record(stream)
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(s1))
        r = rv.Alg1Result.of(out[0])
        e2e = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.alg1_raw(arr_h, 1, out)
            e2e.append(time.perf_counter() - t0)
        ctx.close()
        prof = rv.Context(cuda_stream=stream.cuda_stream, keep_trace=2)
        st = {}
        for k in range(4):
            flush.zero_()
            prof.alg1_raw(arr, 1, out)
            if k:
                for kind, _, ms, _ in prof.stage_times():
                    st.setdefault(kind, []).append(ms)
        prof.close()
        st = {k: sum(v) / len(v) for k, v in st.items()}
        ms = sum(ts) / len(ts)
        cells = 360 ** 3
        acc_bytes = 4 * ((cells + 1) // 2)  # 16-bit counters, two per 32-bit word
        res[key] = {
            "ms_per_solve": ms, "samples_per_s": r.samples_cast / (ms / 1e3), "rotations_per_s": 1e3 / ms,
            "e2e_ms": 1e3 * sum(e2e) / len(e2e), "samples_cast": r.samples_cast, "rechecked": r.rechecked,
            "best_count": r.best_count, "angle_to_truth_rad": _angle(r.q, p.q_true), "status": r.status,
            "vote_path": r.vote_path, "wrapped_words": r.wrapped_words,
            "ms_per_solve_vote_path1": sum(path1) / len(path1) if path1 else None, "stage_ms": st,
            # the accumulator pass: its 2 n^3 bytes read per argmax launch, written per zeroing
            "argmax_gbs": acc_bytes / (st["alg1_argmax"] / 1e3) / 1e9 if st.get("alg1_argmax") else None,
            "zero_gbs": acc_bytes / (st["alg1_zero"] / 1e3) / 1e9 if st.get("alg1_zero") else None,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "vote_samples_per_s": r.samples_cast / (st["alg1_vote"] / 1e3) if st.get("alg1_vote") else None,
            "paper_s": 0.04 if n == 100000 else 0.5,
            "paper_note": ("RTX 4080, Python + CuPy, 1e5 pairs (Table I); context only" if n == 100000 else
                           "the paper's bound for 1e6 pairs (Sec. 1, abstract); context only"),
            "outlier_ratio": rho,
        }
        prev = (arr, a_d, b_d) if key == "n1000000" else None  # the problem before the wrapping one
    # multiple rotations (Sec. 4.4): the paper's largest multiple-rotation setting (9 motions x 3000 pairs,
    # noise 0.01, J = 540), 9 peaks by greedy suppression within 0.1 rad
    mp = synth.make_multi_problem(9, 3000, sigma=0.01, seed=2802)
    a_d, b_d = torch.from_numpy(mp.a).cuda(), torch.from_numpy(mp.b).cuda()
    pk = (rv.rot_vote_peak * 9)()
    arr = (rv.rot_vote_alg1_problem * 1)(rv.rot_vote_alg1_problem(a_d.data_ptr(), b_d.data_ptr(), mp.n, 540, 360,
                                                                    None, 9, 0, 0.1, ctypes.cast(pk, ctypes.c_void_p)))
    out = (rv.rot_vote_alg1_result * 1)()
    ctx = rv.Context(cuda_stream=stream.cuda_stream)
    for _ in range(3):
        ctx.alg1_raw(arr, 1, out)
    ts = []
    for _ in range(reps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx.alg1_raw(arr, 1, out)
        s1.record(stream)
        torch.cuda.synchronize()
        ts.append(s0.elapsed_time(s1))
    ctx.close()
    r = rv.Alg1Result.of(out[0], pk)
    errs = [min(_angle(q, qt) for _, _, q in r.peaks) for qt in mp.q_true] if r.peaks else []
    res["multi9"] = {"ms_per_solve": sum(ts) / len(ts), "peaks": len(r.peaks), "peak_threshold": r.peak_threshold,
                     "max_angle_to_truth_rad": max(errs) if errs else None, "samples_cast": r.samples_cast,
                     "workload": "9 motions x 3000 pairs, noise 0.01, J = 540, 360^3, 9 peaks within 0.1 rad"}
    res["workload"] = ("Alg. 1: J = 180 samples per circle, 360^3 accumulator over [-1,1]^3 (resolution 1/180), "
                       "99% outliers (and 50% at 1e6 pairs); one problem per call")
    return res


def tensor_pipe_fraction(rv, prec, grid_n, levels, a_d, b_d, delta, stream, flush, tests0, peaks, peak_src):
    """The tcgen05 coarse-vote launch of a precision form against the dense bf16/fp16 tensor peak:
    its duration from stage events on the launching stream (mean of 3 solves after one, L2 flushed
    before each), the algorithmic rate (20 flops per test, the 10 multiply-adds of the contraction)
    and the executed MMA rate (2 K flops per test: K = 32 for the hi/lo forms, 16 otherwise)."""
    ctx = rv.Context(grid_n=grid_n, levels=levels, precision=prec, cuda_stream=stream.cuda_stream, keep_trace=2)
    ms = []
    for k in range(4):
        flush.zero_()
        ctx.solve([(a_d, b_d, delta)])
        if k:
            ms += [t for kind, lev, t, _ in ctx.stage_times() if kind == "vote" and lev == 0]
    ctx.close()
    t = sum(ms) / len(ms) / 1e3
    k = 32 if prec.endswith("x2") else 16
    peak = peaks["bf16_tflops"]
    return {"kernel": "vote level 0", "kernel_ms": t * 1e3, "tests_per_launch": tests0,
            "algorithmic_tflops": FLOPS_PER_TEST * tests0 / t / 1e12, "mma_flops_per_test": 2 * k,
            "mma_tflops": 2 * k * tests0 / t / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac_algorithmic": FLOPS_PER_TEST * tests0 / t / 1e12 / peak, "frac_mma": 2 * k * tests0 / t / 1e12 / peak,
            "peak_source": f"dense bf16 tensor burst ({peak_src}); fp16 dense has the same nominal rate"}


def bench_pose(rv, synth, torch, stream, flush, reps: int = 5):
    """Rigid pose (Sec. 4.5) on the paper's default synthetic setting (Sec. 5.4.1): N = 5000,
    90% outliers, noise 0.01; mu_t = 0.04; rotation vote 32^3 + 2 levels, delta = 0.03; the
    paper's 400^3 translation grid over [-5, 5]^3.  Times the whole call on the device, and the
    rotation solve's stages with event pairs on a profiling context."""
    import numpy as np
    p = synth.make_pose_problem(5000, 0.9, 0.01, seed=3003)
    x, y = torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda()
    res = {}
    for prec in ("fp32", "fp16x2"):
        ctx = rv.Context(grid_n=32, levels=2, precision=prec, cuda_stream=stream.cuda_stream)
        for _ in range(2):
            ctx.pose(x, y, 0.04, 0.03)
        ts, front = [], []
        for _ in range(reps):
            flush.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            r = ctx.pose(x, y, 0.04, 0.03)
            s1.record(stream)
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(s1))
            front.append(r.ms_gpu)
        ctx.close()
        # the rotation solve's stages (event pairs around each stage; mean of 3 poses after one)
        prof = rv.Context(grid_n=32, levels=2, precision=prec, cuda_stream=stream.cuda_stream, keep_trace=2)
        st = {}
        for k in range(4):
            flush.zero_()
            prof.pose(x, y, 0.04, 0.03)
            if k:
                for kind, lev, ms, _ in prof.stage_times():
                    key = f"{kind}:{lev}"
                    st[key] = st.get(key, 0.0) + ms / 3
        prof.close()
        res[prec] = {"ms_per_pose": sum(ts) / len(ts), "ms_pairs_and_translation": sum(front) / len(front),
                     "ms_rotation_solve": r.rot.ms_gpu, "rotation_stage_ms": st,
                     "pairs_tested": r.pairs_tested, "pairs_kept": r.pairs_kept,
                     "pairs_rechecked": r.pairs_rechecked, "rotation_tests": r.rot.tests,
                     "angle_to_truth_rad": _angle(r.rot.q, p.q_true),
                     "translation_error": float(np.linalg.norm(r.t - p.t_true)), "status": r.status}
    res["workload"] = ("rigid pose: N = 5000 correspondences, 90% outliers, noise 0.01, mu_t = 0.04, "
                       "32^3 + 2 levels, delta 0.03, 400^3 translation grid over [-5, 5]^3")
    res["paper_note"] = "the paper plots its rigid-pose running time (Fig. 9) without a table; context only"
    return res


def bench_serving(rv, synth, torch, seconds: float, rate_hz: float = 2000.0, distinct: int = 512):
    """Poisson arrivals at rate_hz (N log-uniform [100, 1e5], outliers U[0.8, 0.99],
    sigma 0.01, delta 0.03; 32^3 + 2 levels, FP16 hi/lo form) through
    rot_vote_submit / rot_vote_poll while earlier requests run; `distinct`
    generated problems are cycled."""
    import numpy as np
    t_arr, probs = synth.serving_stream(distinct, rate_hz=rate_hz)
    gaps = np.diff(t_arr, prepend=0.0)
    dev = [(torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda(), p.delta) for p in probs]
    ctx = rv.Context(grid_n=32, levels=2, precision="fp16x2", max_inflight=256)
    # warm-up at the same rate for 1 s (tuning, workspace growth), then the timed stream
    due = time.perf_counter()
    warm = []
    for k in range(int(rate_hz)):
        due += gaps[k % distinct]
        while time.perf_counter() < due:
            pass
        t = ctx.submit(*dev[k % distinct])
        if t > 0:
            warm.append(t)
    for t in warm:
        while ctx.poll(t, timeout_us=10000) is None:
            pass
    total = int(seconds * rate_hz)
    lat, tests, done_t = [], [0], []
    tickets, refused = [], [0]
    lock = threading.Lock()
    finished = threading.Event()

    def poller():
        pending = []
        while True:
            with lock:
                pending.extend(tickets)
                tickets.clear()
            if not pending and finished.is_set():
                return
            keep_p = []
            for t in pending:
                r = ctx.poll(t, timeout_us=0)
                if r is None:
                    keep_p.append(t)
                else:
                    lat.append(r.latency_ms)
                    tests[0] += r.tests
                    done_t.append(time.perf_counter())
            pending = keep_p
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    due = t0
    for k in range(total):
        due += gaps[k % distinct] if k else 0.0
        while time.perf_counter() < due:
            pass
        t = ctx.submit(*dev[k % distinct])
        if t < 0:
            refused[0] += 1
        else:
            with lock:
                tickets.append(t)
    t_sub = time.perf_counter() - t0
    finished.set()
    th.join()
    spans = ctx.serve_spans()
    ctx.close()
    span = max(done_t) - t0
    return {"rotations_per_s": len(lat) / span, "offered_per_s": total / t_sub,
            "tests_per_s": tests[0] / span, "unit": "rotations/s",
            "latency_ms": {"p50": percentile(lat, 50), "p90": percentile(lat, 90), "p99": percentile(lat, 99),
                           "max": max(lat)},
            "completed": len(lat), "refused_eagain": refused[0], "overlap": span_overlap(spans),
            "workload": ("Poisson %.0f/s for %.1f s; N log-uniform [100, 1e5], outliers U[0.8, 0.99], sigma 0.01, "
                         "delta 0.03; 32^3 + 2 levels; fp16x2; %d distinct problems cycled; after a 1 s warm-up at the same "
                         "rate; latency = submit to result ready (library clock)" % (rate_hz, seconds, distinct))}


def span_overlap(spans):
    """How much the serving batches overlapped on the device, from their device-time spans
    (t_start_ms, t_end_ms, wave, problems): the mean number of batches in flight over the time
    any was, and the share of that time with two or more in flight."""
    if not spans:
        return None
    ev = sorted([(s[0], 1) for s in spans] + [(s[1], -1) for s in spans])
    busy = multi = 0.0
    depth, prev = 0, ev[0][0]
    for t, d in ev:
        if depth > 0:
            busy += t - prev
        if depth > 1:
            multi += t - prev
        depth += d
        prev = t
    total = sum(s[1] - s[0] for s in spans)
    return {"batches": len(spans), "waves_used": len({s[2] for s in spans}),
            "mean_batch_problems": sum(s[3] for s in spans) / len(spans),
            "mean_in_flight": total / busy if busy > 0 else None,
            "share_two_or_more": multi / busy if busy > 0 else None,
            "note": ("spans run from a batch's first to its last event on its wave's stream: overlapping spans "
                     "mean both batches' work was in flight together; the tcgen05 vote holds a whole SM, so "
                     "two waves' coarse votes share no SM")}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2506_11547_gb300 import synth
    p, grid_n, levels = synth.config_problem(args.workload)
    threads = os.cpu_count() or 1
    per_step = max(0.5, min(5.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_rate(p, grid_n, per_step / 4, threads)
    rates, samples, secs = [], [], []
    m = 0
    for _ in range(args.steps):  # the first step sizes the sample; the others reuse that size
        r, m, dt = cpu_oracle_rate(p, grid_n, per_step, threads, m_hint=m)
        rates.append(r)
        samples.append(m)
        secs.append(dt)
    total_tests = sum(m * p.n for m in samples)
    value = float(sum(rates) / len(rates))
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESCS.get(args.workload, args.workload)},
        "ms_per_step": 1e3 * total_tests / value / args.steps,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"per step {sum(secs) / len(secs):.1f} s: the FP64 oracle's vote of {samples[0]} "
                                   f"random coarse cells x {p.n} pairs ({threads} threads over cells)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def profile_case(case: str):
    """Three calls of one case, each after a 256 MiB L2 flush, for profiler captures."""
    import torch
    from paper_2506_11547_gb300 import rot_vote as rv
    from paper_2506_11547_gb300 import synth
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if case == "alg1_n1e5":  # 1e5 pairs, 99% outliers, J = 180, 360^3
        p = synth.make_problem(100000, 0.99, 0.01, 0.03, seed=2301)
        args = [(torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda(), 180, 360)]
        kw = {}
    elif case == "alg1_multi9":  # 9 motions x 3000 pairs, J = 540, 360^3, 9 peaks within 0.1 rad
        mp = synth.make_multi_problem(9, 3000, sigma=0.01, seed=2802)
        args = [(torch.from_numpy(mp.a).cuda(), torch.from_numpy(mp.b).cuda(), 540, 360)]
        kw = dict(peaks=9, nms_angle=0.1)
    else:  # rigid pose, N = 5000, 90% outliers, FP16X2 rotation vote 32^3 + 2 levels
        p = synth.make_pose_problem(5000, 0.9, 0.01, seed=3003)
        x, y = torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda()
    with rv.Context(grid_n=32, levels=2, precision="fp16x2") as ctx:
        for _ in range(3):
            flush.zero_()
            r = ctx.pose(x, y, 0.04, 0.03) if case == "pose_n5000" else ctx.alg1(args, **kw)[0]
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "status": r.status}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2506_11547_gb300 import rot_vote as rv
    from paper_2506_11547_gb300 import synth

    # weak scaling: each rank solves its own problem instance of the same shape
    p, grid_n, levels = rank_problem(synth, args.workload, rank)
    a_d = torch.from_numpy(p.a).to(dev)
    b_d = torch.from_numpy(p.b).to(dev)
    stream = torch.cuda.current_stream()
    ctx = rv.Context(grid_n=grid_n, levels=levels, precision=args.precision, cuda_stream=stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    arr = (rv.rot_vote_problem * 1)()
    arr[0], keep = rv.problem(a_d, b_d, p.delta)
    out = (rv.rot_vote_result * 1)()
    for _ in range(max(3, args.warmup)):
        ctx.solve_raw(arr, 1, out)
    res0 = rv.Result.of(out[0])
    tests_per_step = res0.tests
    if args.only_solve:
        for _ in range(args.steps):
            ctx.solve_raw(arr, 1, out)
        torch.cuda.synchronize()
        if rank == 0:
            r = rv.Result.of(out[0])
            print(json.dumps({"only_solve": True, "workload": args.workload, "precision": args.precision,
                              "status": r.status, "ms_gpu": r.ms_gpu, "tests": r.tests}))
        return

    # ---- device-timed steps (inputs resident in HBM; L2 flushed before each) ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.solve_raw(arr, 1, out)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    per = [s.elapsed_time(e) for s, e in evs]
    elapsed = reduce_max(sum(per), dist, dev)
    value = whole_job_rate(tests_per_step, args.steps, ws, elapsed / 1e3)
    ms_per_step = elapsed / args.steps
    clocks = clk.summary()

    # ---- e2e: public API with pinned host inputs, copies inside the timed region ----
    a_h = torch.from_numpy(p.a).pin_memory()
    b_h = torch.from_numpy(p.b).pin_memory()
    arr_h = (rv.rot_vote_problem * 1)()
    arr_h[0], keep_h = rv.problem(a_h, b_h, p.delta)
    ctx.solve_raw(arr_h, 1, out)
    e2e_t = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_raw(arr_h, 1, out)  # blocking: H2D, pipeline, D2H of the result
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = reduce_max(sum(e2e_t), dist, dev)
    e2e_value = whole_job_rate(tests_per_step, args.steps, ws, e2e_s)
    h2d = 2 * p.n * 3 * 4
    d2h = ctypes.sizeof(rv.rot_vote_result) + 4  # result struct + device error word
    ctx.close()

    # ---- roofline of the dominant kernel (profiled solves on the same stream) ----
    peaks, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stage_avg, launches, n_cells0 = stage_profile(rv, grid_n, levels, args.precision, a_d, b_d, p.delta, stream,
                                                  flush)
    roofline = roofline_of(stage_avg, n_cells0 * p.n, args.precision, args.workload, peaks, peak_src, sms)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and ws == 1:
        threads = os.cpu_count() or 1
        rate, m, dt = cpu_oracle_rate(p, grid_n, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{m} random coarse cells x {p.n} pairs of this workload's level 0 ({dt:.1f} s, "
                         f"FP64 C oracle, threads over cells)"}

    # ---- the other precision forms on the same workload (device-timed the same way) ----
    extra = None
    if not args.no_extra and ws == 1:
        extra = {}
        for prec in [x for x in ("fp16", "bf16", "bf16x2", "fp32") if x != args.precision]:
            m = measure_form(rv, torch, prec, grid_n, levels, arr, out, stream, flush, max(3, args.steps // 4))
            rr = m.pop("result")
            m["same_result"] = bool(rr.best_cell == res0.best_cell and list(rr.q) == list(res0.q) and
                                    rr.best_count == res0.best_count and rr.ambiguous == res0.ambiguous)
            if prec != "fp32":
                m["tensor_pipe"] = tensor_pipe_fraction(rv, prec, grid_n, levels, a_d, b_d, p.delta, stream, flush,
                                                        n_cells0 * p.n, peaks, peak_src)
            extra[prec] = m
        extra["note"] = ("K = 16 forms (fp16, bf16): operands rounded once to 16 bits, the contraction's A = "
                         "[m, -tau_hi, -tau_lo], band = each cell's rigorous bound; hi/lo forms (fp16x2, bf16x2): "
                         "K = 32 split operands, a far narrower rigorous band (reading C11); every form gives the "
                         "same exact counts")

    # ---- the 1e5-pair, 64^3 + 3-level workload: the plain FP32 form and the FP16 hi/lo form ----
    scale1 = None
    if not args.no_extra and ws == 1 and args.workload != "fp32_n1e5_64L3":
        scale1 = bench_scale1(rv, synth, torch, stream, flush, peaks, peak_src, sms, max(5, args.steps))

    batched = serving = alg1 = pose = None
    if not args.no_extra and ws == 1:
        batched = bench_batched(rv, synth, torch, stream, flush)
        serving = bench_serving(rv, synth, torch, args.serve_seconds)
        alg1 = bench_alg1(rv, synth, torch, stream, flush, peaks)
        pose = bench_pose(rv, synth, torch, stream, flush)

    lat = per
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESCS.get(args.workload, args.workload),
                   "precision": args.precision, "tests_per_step": tests_per_step,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"independent problem per GPU x{ws}",
                   "form": ("FP16 hi/lo split operands (K = 32) on tcgen05 with FP32 accumulation in TMEM, rigorous "
                            "per-cell re-check band, FP32 re-check, FP64 decision within 2e-6 of the threshold "
                            "(the hi/lo reading of C11)" if args.precision.endswith("x2") else args.precision)},
        "rotations_per_s": ws * args.steps / (elapsed / 1e3),
        "latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99), "mean": ms_per_step},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * e2e_s / args.steps},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "stage_ms": {f"{k[0]}:{k[1]}": v for k, v in sorted(stage_avg.items(), key=lambda x: -x[1])},
        "precision_forms": extra,
        "fp32_n1e5_64L3": scale1,
        "batched": batched,
        "serving": serving,
        "alg1": alg1,
        "pose": pose,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "result": {"status": res0.status, "angle_to_truth_rad": _angle(res0.q, p.q_true),
                   "rechecked": res0.rechecked, "resolved_fp64": res0.resolved, "ambiguous": res0.ambiguous,
                   "best_cell": res0.best_cell, "best_count": res0.best_count, "inliers": res0.inliers},
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def stage_profile(rv, grid_n, levels, prec, a_d, b_d, delta, stream, flush, n_prof: int = 5):
    """Per-stage device times (event pairs on the launching stream, mean of n_prof solves after
    one, L2 flushed before each), the kernels one solve launches, and the coarse cell count."""
    prof = rv.Context(grid_n=grid_n, levels=levels, precision=prec, cuda_stream=stream.cuda_stream, keep_trace=2)
    stage_ms = {}
    launches = 0
    for _ in range(n_prof + 1):
        flush.zero_()
        prof.solve([(a_d, b_d, delta)])
        st = prof.stage_times()
        launches = sum(k for _, _, _, k in st)
        for kind, lev, ms, _ in st:
            stage_ms.setdefault((kind, lev), []).append(ms)
    n_cells0 = len(prof.level_trace(0, 0)[0])
    prof.close()
    return {k: sum(v[1:]) / len(v[1:]) for k, v in stage_ms.items()}, launches, n_cells0


def roofline_of(stage_avg, tests0, prec, workload, peaks, peak_src, sms):
    """The dominant stage (the coarse vote) against its pipe: the FP32 FMA pipe for the plain form;
    for the tensor-core forms the dense 16-bit tensor peak (measured bf16 burst; fp16 has the same
    nominal rate), with the epilogue's CUDA-core bound beside it."""
    dom = max(stage_avg, key=stage_avg.get)
    if dom != ("vote", 0):
        return None
    t = stage_avg[dom] / 1e3
    achieved = FLOPS_PER_TEST * tests0 / t / 1e12
    f_mhz = peaks.get("sm_max_mhz", 2070.0)
    r = {"achieved": achieved, "unit": "TFLOP/s", "traffic": ncu_traffic(prec, workload),
         "traffic_unit": "B per launch", "kernel": "vote level 0", "kernel_ms": stage_avg[dom],
         "flops_per_test": FLOPS_PER_TEST, "tests_per_launch": tests0,
         "share_of_step": stage_avg[dom] / sum(stage_avg.values())}
    if prec == "fp32":
        peak = sms * 128 * 2 * f_mhz * 1e6 / 1e12
        r.update(bound="alu", peak=peak, frac=achieved / peak, executed_fma_per_test=9,
                 peak_source=f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 flops x {f_mhz} MHz")
    else:
        peak = peaks["bf16_tflops"]
        k = 32 if prec.endswith("x2") else 16
        epi = sms * EPI_ALU_LANES_PER_SM * f_mhz * 1e6 / EPI_ALU_INSTR_PER_TEST
        r.update(bound="tensor", peak=peak, frac=achieved / peak,
                 peak_source=f"dense bf16 tensor burst ({peak_src}); fp16 dense has the same nominal rate",
                 frac_k16=K16_FLOPS_PER_TEST * tests0 / t / 1e12 / peak,
                 frac_executed_mma=2 * k * tests0 / t / 1e12 / peak, mma_flops_per_test=2 * k,
                 epilogue={"bound": "alu", "tests_per_s": tests0 / t, "peak_tests_per_s": epi,
                           "frac": tests0 / t / epi,
                           "peak_source": (f"{sms} SMs x {EPI_ALU_LANES_PER_SM} ALU lanes x {f_mhz} MHz / "
                                           f"{EPI_ALU_INSTR_PER_TEST} ALU instructions per test (|D| minima; "
                                           "the sign counts run on the FMA pipe)")})
    return r


def measure_form(rv, torch, prec, grid_n, levels, arr, out, stream, flush, reps):
    """Device time per solve of one precision form (L2 flushed before each), after its autotune."""
    cx = rv.Context(grid_n=grid_n, levels=levels, precision=prec, cuda_stream=stream.cuda_stream)
    for _ in range(3):
        cx.solve_raw(arr, 1, out)
    ts = []
    for _ in range(reps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        cx.solve_raw(arr, 1, out)
        s1.record(stream)
        torch.cuda.synchronize()
        ts.append(s0.elapsed_time(s1))
    cx.close()
    rr = rv.Result.of(out[0])
    ms = sum(ts) / len(ts)
    return {"value": rr.tests / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "tests_per_step": rr.tests,
            "rechecked": rr.rechecked, "resolved_fp64": rr.resolved, "ambiguous": rr.ambiguous, "result": rr}


def bench_scale1(rv, synth, torch, stream, flush, peaks, peak_src, sms, reps):
    """The 1e5-pair, 99%-outlier, 64^3 + 3-level workload: the plain FP32 CUDA-core form (the
    baseline the precision forms must beat) and the FP16 hi/lo tensor-core form, each with its
    coarse vote against its pipe; and the same workload in the stereographic chart (FP32)."""
    p, g, L = synth.config_problem("fp32_n1e5_64L3")
    a_d, b_d = torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda()
    arr = (rv.rot_vote_problem * 1)()
    arr[0], keep = rv.problem(a_d, b_d, p.delta)
    out = (rv.rot_vote_result * 1)()
    res = {}
    for prec in ("fp32", "fp16x2"):
        m = measure_form(rv, torch, prec, g, L, arr, out, stream, flush, reps)
        rr = m.pop("result")
        st, launches, nc0 = stage_profile(rv, g, L, prec, a_d, b_d, p.delta, stream, flush)
        m.update(angle_to_truth_rad=_angle(rr.q, p.q_true), kernels_per_step=launches,
                 stage_ms={f"{k[0]}:{k[1]}": v for k, v in sorted(st.items(), key=lambda x: -x[1])},
                 roofline=roofline_of(st, nc0 * p.n, prec, "fp32_n1e5_64L3", peaks, peak_src, sms))
        res[prec] = m
    cx = rv.Context(grid_n=g, levels=L, precision="fp32", chart="stereographic", cuda_stream=stream.cuda_stream)
    for _ in range(3):
        cx.solve_raw(arr, 1, out)
    ts = []
    for _ in range(reps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        cx.solve_raw(arr, 1, out)
        s1.record(stream)
        torch.cuda.synchronize()
        ts.append(s0.elapsed_time(s1))
    rr = rv.Result.of(out[0])
    cx.close()
    res["stereographic_fp32"] = {"value": rr.tests / (sum(ts) / len(ts) / 1e3), "unit": UNIT,
                                 "ms_per_step": sum(ts) / len(ts), "tests_per_step": rr.tests,
                                 "angle_to_truth_rad": _angle(rr.q, p.q_true)}
    res["workload"] = WORKLOAD_DESCS["fp32_n1e5_64L3"]
    return res


if __name__ == "__main__":
    main()
