#!/usr/bin/env python
"""Benchmark of the GB300 SK-NR entropic-OT solver.

Metric: time to reach an L1 marginal error of 1e-6 at eps = 1e-3, SK-NR(30)
against plain log-domain Sinkhorn, on n = m = 4096 points in R^3 drawn from a
4-component Gaussian mixture (sigma 0.1, means uniform in [0,1]^3),
Dirichlet(1) weights, squared Euclidean cost normalised to max 1 and stored in
float32, eps continuation 1e-1 -> 1e-3 (factor 1/2).  One step is one full
solve through the C ABI (cost built on the device from X, Y, continuation,
modes, Newton steps, evaluation), inputs resident in HBM.  L2 is flushed
between steps (a 512 MB write outside the timed region).

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle instead (bounded sample, scaled to one solve).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = M = 4096
EPS = 1e-3
TOL = 1e-6
LEVEL_TOL = 1e-4   # intermediate continuation levels (warm starts): L1 1e-4
# Ritz residual at which a level's modes stop (started from the previous
# level's modes): measured on this workload, 1e-2 / 3e-2 / 5e-2 / 1e-1 took
# 23 / 13 / 9 / 7 subspace iterations and 14.7 / 12.7 / 12.2 / 11.7 ms with
# 69 / 67 / 69 / 68 SK-NR iterations: the Newton step needs the modes' span,
# not tight Ritz vectors.  At 1e-1 the first level's modes stop after one step
# from the random start (the absolute residual of the many tiny rho_k^2 is
# small whatever the vectors) and the float64 oracle then needs 98 iterations
# instead of 67; at 5e-2 it needs 67 (11 subspace iterations)
EIG_TOL = 5e-2
ELL = 30
METRIC = ("time-to-L1-marginal 1e-6 at eps=1e-3 (SK-NR(30), eps continuation 1e-1->1e-3, "
          "intermediate levels to 1e-4)")
WORKLOAD = "gaussian_mixture_4096x4096_d3_stored_fp32_cost"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", action="store_true",
                    help="one SK-NR solve per step, no Sinkhorn comparison (for ncu)")
    ap.add_argument("--sk-steps", type=int, default=None)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="skip the additional configurations (on-the-fly cost, batch, serving)")
    ap.add_argument("--oracle-sample", action="store_true",
                    help="time the bounded oracle sample of the CPU baseline and print it (JSON)")
    ap.add_argument("--case", default=None,
                    choices=["coop16k", "stream8k", "sknr4k", "gram", "batch", "s4_8k"],
                    help="run one small case for a profiler and exit (no timing, no JSON)")
    return ap.parse_args()


def max_over_ranks(value: float, ws: int, device: str) -> float:
    """The largest of the ranks' figures (each rank a replica on its own GPU and
    problem: the slowest one times the job).  All ranks call it; one all-reduce
    of one float64 on `device` (cuda under NCCL, cpu under gloo)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Seed of the workload a rank solves: replicas solve independent draws."""
    return rank


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def options(pkg, ell, stream=None, **kw):
    o = pkg.default_options(tol=TOL, max_iter=200000, ell=ell, eps_start=1e-1, eps_factor=0.5,
                            level_tol=LEVEL_TOL, oversample=10, eig_tol=EIG_TOL, eig_max_iter=100)
    for k, v in kw.items():
        setattr(o, k, v)
    if stream is not None:
        o.stream = stream
    return o


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(torch, buf):
    buf.zero_()


def run_ours(args):
    import torch
    import torch.distributed as dist

    import workloads
    import paper_2506_14780_gb300 as pkg

    ws, rank, local = dist_info()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    pkg.load()
    prob = workloads.gaussian_mixture(N, M, seed=replica_seed(rank), eps=EPS)
    X = torch.as_tensor(prob.X).cuda()
    Y = torch.as_tensor(prob.Y).cuda()
    a = torch.as_tensor(prob.a).cuda()
    b = torch.as_tensor(prob.b).cuda()
    f = torch.zeros(N, dtype=torch.float64, device="cuda")
    g = torch.zeros(M, dtype=torch.float64, device="cuda")
    keep = []
    p = pkg.make_problem(a, b, X=X, Y=Y, eps=EPS, normalize_cost=True, keep=keep)
    stream = torch.cuda.current_stream()
    o_nr = options(pkg, ELL, stream.cuda_stream)
    o_sk = options(pkg, 0, stream.cuda_stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def solve(o):
        st, res = pkg.eot_solve(p, o, f, g)
        if st < 0:
            raise RuntimeError(f"eot_solve failed: {pkg.last_error()}")
        return res.as_dict()

    for _ in range(max(args.warmup, 0)):
        solve(o_nr)
        if not args.profile:
            solve(o_sk)
    torch.cuda.synchronize()

    def timed(o, steps):
        times, results = [], []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush_l2(torch, flush)
            ev[k][0].record()
            results.append(solve(o))
            ev[k][1].record()
        torch.cuda.synchronize()
        times = [e0.elapsed_time(e1) for e0, e1 in ev]
        return times, results

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    nr_times, nr_res = timed(o_nr, args.steps)
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    ms_nr = max_over_ranks(statistics.median(nr_times), ws, "cuda")

    out = {"metric": METRIC, "value": round(ms_nr, 4), "unit": "ms",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms_nr, 4), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "m": M, "d": 3, "eps": EPS, "tol": TOL,
                      "ell": ELL, "eps_schedule": "1e-1 x 0.5^k -> 1e-3 (8 levels)",
                      "level_tol": LEVEL_TOL, "eig_tol": EIG_TOL, "oversample": 10,
                      "potentials": "f64 (exponents formed exactly, f32 exp/sums)",
                      "l2": "flushed between steps (512 MB write)",
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}}
    last = nr_res[-1]
    pairs = {"c2_sknr30": (f.cpu().numpy().copy(), g.cpu().numpy().copy())}
    out["sknr"] = {"p50_ms": round(statistics.median(nr_times), 4),
                   "p99_ms": round(sorted(nr_times)[min(len(nr_times) - 1,
                                                     int(0.99 * len(nr_times)))], 4),
                   "iters_last_level": last["iters"], "total_iters": last["total_iters"],
                   "eig_iters": last["eig_iters"], "nr_accepted_last": last["nr_accepted"],
                   "l1_marginal": last["l1_marginal"], "last_level_ms": round(1e3 * last["seconds_last_level"], 4),
                   "eig_ms": round(1e3 * last["seconds_eig"], 4), "status": last["status_name"]}
    out["gpu_launches"] = int(sum(r["kernel_launches"] for r in nr_res))
    out["clocks"] = clk
    if not args.profile:
        sk_steps = args.sk_steps if args.sk_steps is not None else max(1, min(args.steps, 5))
        sk_times, sk_res = timed(o_sk, sk_steps)
        pairs["c2_sinkhorn"] = (f.cpu().numpy().copy(), g.cpu().numpy().copy())
        sl = sk_res[-1]
        out["plain_sk"] = {"p50_ms": round(statistics.median(sk_times), 4),
                           "iters_last_level": sl["iters"], "total_iters": sl["total_iters"],
                           "l1_marginal": sl["l1_marginal"],
                           "last_level_ms": round(1e3 * sl["seconds_last_level"], 4),
                           "status": sl["status_name"], "steps": sk_steps}
        sk_ms = max_over_ranks(statistics.median(sk_times), ws, "cuda")
        out["plain_sk"]["max_over_ranks_ms"] = round(sk_ms, 4)
        out["speedup_sknr_vs_sk"] = round(sk_ms / ms_nr, 3)
        # the same solve with the Chebyshev-filtered mode computation (degree 2)
        o_cf = options(pkg, ELL, stream.cuda_stream, eig_degree=2)
        solve(o_cf)
        cf_times, cf_res = timed(o_cf, max(1, min(args.steps, 5)))
        cl = cf_res[-1]
        out["sknr"]["chebyshev_modes_degree2"] = {
            "p50_ms": round(statistics.median(cf_times), 4), "total_iters": cl["total_iters"],
            "eig_iters": cl["eig_iters"], "eig_ms": round(1e3 * cl["seconds_eig"], 4),
            "status": cl["status_name"],
            "note": "eig_degree = 2: fewer Rayleigh-Ritz steps, more products per step"}
        out["speedup_last_level"] = round(sl["seconds_last_level"] / max(last["seconds_last_level"], 1e-12), 3)
        # end to end through the public API with host buffers (H2D + D2H inside)
        e2e = []
        fh = np.zeros(N)
        gh = np.zeros(M)
        keep_h = []
        ph = pkg.make_problem(prob.a, prob.b, X=prob.X, Y=prob.Y, eps=EPS, normalize_cost=True,
                              keep=keep_h)
        oh = options(pkg, ELL)
        for _ in range(max(1, min(args.steps, 5))):
            flush_l2(torch, flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, _ = pkg.eot_solve(ph, oh, fh, gh)
            t1 = time.perf_counter()
            e2e.append((t1 - t0) * 1e3)
        h2d = prob.X.nbytes + prob.Y.nbytes + prob.a.nbytes + prob.b.nbytes
        out["e2e"] = {"value": round(max_over_ranks(statistics.median(e2e), ws, "cuda"), 4),
                      "unit": "ms",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * (N + M))}
        out["roofline"] = roofline(pkg, torch, p, f, g, stream)
        c3 = None
        # the additional configurations run on one GPU only (with replicas the
        # line reports the headline solve, max over ranks)
        if not args.quick and ws == 1:
            out["configs_extra"], c3 = extras(pkg, torch, stream)
    if rank == 0 and not args.no_cpu and not args.profile:
        stage("cpu baseline (oracle)")
        out["cpu_baseline"] = cpu_baseline()
        stage("oracle scores of the returned potentials")
        out["oracle_scores"] = oracle_scores(prob, pairs, c3)
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def stage(msg):
    """Progress note on stderr (the JSON line goes to stdout)."""
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def per_pass_ms(pkg, torch, p, f, g, stream, r1, r2, **kw):
    """Average time of one log-sum-exp half-step: two single-level Sinkhorn
    solves from the same potentials with a fixed number of iterations (the
    tolerance is unreachable) differ by exactly 2 (r2 - r1) half-steps; CUDA
    events on this stream, best of three."""
    fi = f.clone()
    ms = {}
    for R in (r1, r2):
        o = options(pkg, 0, stream.cuda_stream, tol=1e-300, max_iter=R, eps_start=0.0, **kw)
        p2 = type(p).from_buffer_copy(p)
        p2.f_init = fi.data_ptr()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, res = pkg.eot_solve(p2, o, f, g)
            e1.record()
            torch.cuda.synchronize()
            if st < 0:
                raise RuntimeError(pkg.last_error())
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        ms[R] = best
    return (ms[r2] - ms[r1]) / (2 * (r2 - r1))


def load_peaks():
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            return json.load(fh)
    return {}


def sknr_stage_times(pkg, torch, n, seed, eps, flush, stream, reps=7):
    """Device time of the stages of one SK-NR(30) iteration (row half-step, S4
    pass, Newton solve, trial pass) on the gaussian_mixture n x n workload,
    from CUDA events that eot_sknr_step records on its stream around each
    stage; the state is a Sinkhorn solve at eps (L1 1e-4) and 30 modes there.
    L2 is flushed before every step.  Returns the median seconds per stage."""
    import workloads
    prob = workloads.gaussian_mixture(n, n, seed=seed, eps=eps)
    X, Y = torch.as_tensor(prob.X).cuda(), torch.as_tensor(prob.Y).cuda()
    a, b = torch.as_tensor(prob.a).cuda(), torch.as_tensor(prob.b).cuda()
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    if pkg.eot_cost(n, n, 3, X, Y, True, C) != pkg.EOT_OK:
        raise RuntimeError(pkg.last_error())
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    keep = []
    pc = pkg.make_problem(a, b, C=C, eps=eps, keep=keep)
    o = options(pkg, 0, stream.cuda_stream, tol=1e-4, max_iter=20000, eps_start=0.0)
    st, _ = pkg.eot_solve(pc, o, f, g)
    if st < 0:
        raise RuntimeError(pkg.last_error())
    V = torch.zeros((n, ELL), dtype=torch.float64, device="cuda")
    st, _, _ = pkg.eot_spectral_modes(n, n, C, f, g, a, b, eps, ELL, 10, 1e-2, 30, False, V)
    if st < 0:
        raise RuntimeError(pkg.last_error())
    times = []
    for r in range(reps + 2):
        flush_l2(torch, flush)
        st, info = pkg.eot_sknr_step(n, n, ELL, C, a, b, eps, g, V, stream=stream.cuda_stream)
        if st < 0:
            raise RuntimeError(pkg.last_error())
        if r >= 2:
            times.append(info["stage_seconds"])
    del X, Y, C, V
    return [statistics.median(t[k] for t in times) for k in range(4)]


def roofline(pkg, torch, p, f, g, stream):
    """Roofline of the SK-NR solve's dominant kernel, the S4 pass
    (mma_tma_kernel<32, 0>: column log-sum-exp, h = f_k^{C,eps}, the L1 test
    and W = pi(f_k, h)^T V on the tensor cores): it reads the n x m float32
    cost once, 4 n m algorithmic bytes per launch (the tensor-core work, 3xTF32
    products of an n x m by m x 32 block, is 6 n m 32 flops, far below the
    tensor peak at this byte count).  Timed live with CUDA events on the
    launching stream (eot_sknr_step) on an HBM-resident 16384^2 cost and on
    the benchmark's 4096^2 cost (67 MB, L2-resident during a solve).  Beside
    it: the whole SK-NR iteration (three passes, 12 n m bytes) and the plain
    Sinkhorn half-step of the cooperative loop (sk_coop_kernel)."""
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stage("roofline: SK-NR stages 16384^2")
    nl = 16384
    big = sknr_stage_times(pkg, torch, nl, 1, 1e-2, flush, stream)
    stage("roofline: SK-NR stages 4096^2")
    small = sknr_stage_times(pkg, torch, N, 0, 1e-2, flush, stream)
    b_big, b_small = 4.0 * nl * nl, 4.0 * N * M
    s4 = big[1]
    achieved = b_big / s4 / 1e9
    it_big, it_small = sum(big), sum(small)
    stage("roofline: plain Sinkhorn half-step 16384^2")
    coop = coop_half_step(pkg, torch, stream)
    return {"kernel": "mma_tma_kernel<32, 0> (S4 pass: column log-sum-exp, h, L1 test, "
                      "W = pi^T V on tcgen05; largest share of the SK-NR solve)",
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 3), "traffic": s4_traffic(),
            "per_launch_us": round(s4 * 1e6, 2),
            "workload": f"{nl}x{nl} cost (1.07 GB, HBM-resident), l = {ELL}",
            "algorithmic_bytes_per_launch": int(b_big),
            "tensor_flops_per_launch": int(6 * nl * nl * 32),
            "l2_resident_4096": {"per_launch_us": round(small[1] * 1e6, 2),
                                 "achieved_gbs": round(b_small / small[1] / 1e9, 1)},
            "sknr_iteration": {
                "stages": "row half-step, S4, Newton (reduce + LDL^T + f'), trial pass",
                "16384_us": [round(x * 1e6, 2) for x in big],
                "16384_achieved_gbs": round(3 * b_big / it_big / 1e9, 1),
                "16384_frac": round(3 * b_big / it_big / 1e9 / hbm, 3),
                "4096_us": [round(x * 1e6, 2) for x in small],
                "4096_achieved_gbs": round(3 * b_small / it_small / 1e9, 1)},
            "plain_sk_half_step": coop,
            "note": "CUDA events on the launching stream around each stage of one SK-NR "
                    "iteration (eot_sknr_step), median of 7 after 2 warm-up steps, L2 "
                    "flushed before each; peak of measured (MEASURED_PEAKS.json hbm_gbs)"}


def coop_half_step(pkg, torch, stream):
    """The plain Sinkhorn half-step (sk_coop_kernel) on the same HBM-resident
    16384^2 cost: two single-level solves with fixed iteration counts differ
    by exactly 2 (R2 - R1) half-steps."""
    import workloads
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    nl = 16384
    big = workloads.gaussian_mixture(nl, nl, seed=1, eps=EPS)
    keep = []
    Xb, Yb = torch.as_tensor(big.X).cuda(), torch.as_tensor(big.Y).cuda()
    ab, bb = torch.as_tensor(big.a).cuda(), torch.as_tensor(big.b).cuda()
    fb = torch.zeros(nl, dtype=torch.float64, device="cuda")
    gb = torch.zeros(nl, dtype=torch.float64, device="cuda")
    pb = pkg.make_problem(ab, bb, X=Xb, Y=Yb, eps=1e-2, normalize_cost=True, keep=keep)
    o = options(pkg, 0, stream.cuda_stream, tol=1e-4, max_iter=2000, eps_start=0.0)
    pkg.eot_solve(pb, o, fb, gb)
    torch.cuda.synchronize()
    large = per_pass_ms(pkg, torch, pb, fb, gb, stream, 20, 80)
    achieved = 4.0 * nl * nl / (large * 1e-3) / 1e9
    del Xb, Yb, fb, gb
    return {"kernel": "sk_coop_kernel", "per_half_step_us": round(large * 1e3, 3),
            "achieved": round(achieved, 1), "frac": round(achieved / hbm, 3),
            "traffic": coop_traffic()}


# DRAM traffic of one S4 launch (mma_tma_kernel<32, 0>) at 16384^2 with l = 30:
# dram__bytes_read.sum + dram__bytes_write.sum of the 8192^2 launch of an ncu
# capture (`bench.py --case s4_8k`; 285,006,848 B, 1.062 x its 4 n m bytes,
# profiles/mma_tma_kernel_s4_8192.md) scaled by the 4x elements of the 16384^2
# launch; valid while the kernel's sources hash to the recorded SHA-256.
S4_TRAFFIC_BYTES = 4 * 285006848
S4_TRAFFIC_SOURCES = ("mma.cu", "tc.cuh", "eot_device.cuh", "eot_internal.h")
S4_TRAFFIC_SHA256 = "b000e60774c4db88aadfb436f74dc5dc3d76e8a90db2c322e0de8f0c8ef69cf7"


def s4_traffic():
    if S4_TRAFFIC_BYTES is None:
        return None
    return S4_TRAFFIC_BYTES if _sources_sha(S4_TRAFFIC_SOURCES) == S4_TRAFFIC_SHA256 else None


def _sources_sha(files):
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2506_14780_gb300", "csrc")
    try:
        for fn in files:
            with open(os.path.join(src, fn), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return h.hexdigest()


# Pipe use of one on-the-fly-cost pass (gram_pass_kernel, 20000 x 30000 x 64)
# from an ncu capture of `bench.py --case gram` (profiles/gram_pass_kernel_20000x30000_d64.md):
# the tensor pipe's active cycles and the MUFU (xu) and FMA pipes' instruction
# rates, as % of their sustained peaks; valid while the kernel's sources hash to
# the recorded SHA-256.
GRAM_PIPES = {"tensor_pipe_active_pct": 44.37, "mufu_xu_pipe_pct": 16.01, "fma_pipe_pct": 24.35,
              "duration_us_cold": 449.9}
GRAM_PIPES_SOURCES = ('gram.cu', 'eot_device.cuh', 'eot_internal.h', 'pass_common.cuh', 'reduce.cuh', 'stream_common.cuh', 'tc.cuh')
GRAM_PIPES_SHA256 = "d5ad9d2fdbbbab3d81383a50df85249e4e3951e44616fa08aebd517399790ab8"


def gram_pipes():
    return GRAM_PIPES if _sources_sha(GRAM_PIPES_SOURCES) == GRAM_PIPES_SHA256 else None


# DRAM traffic of one sk_coop_kernel half-step at 16384^2 (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch of four half-steps, divided by four; ncu capture
# summarised in profiles/sk_coop_kernel_16384_traffic.md).  It describes the kernel
# built from the sources it was taken on, identified by their SHA-256: after any change
# to them the bench reports no traffic until the capture is taken again.
COOP_TRAFFIC_BYTES = 1082535040
COOP_TRAFFIC_SOURCES = ("stream.cu", "stream_common.cuh", "eot_device.cuh", "eot_internal.h",
                        "pass_common.cuh", "reduce.cuh", "tc.cuh")
COOP_TRAFFIC_SHA256 = "7b87389493b74b86d65b33e1e932f5301bd16ae52ada8b00f5a7a9ed1b076090"


def coop_traffic():
    return COOP_TRAFFIC_BYTES if _sources_sha(COOP_TRAFFIC_SOURCES) == COOP_TRAFFIC_SHA256 else None


def extras(pkg, torch, stream):
    """The other configurations, measured briefly: on-the-fly cost (c3), a
    batch of problems (c4) and a served stream (c5)."""
    import workloads
    out = {}
    peaks = load_peaks()
    # c3: 20000 x 30000 points in R^64 ~ N(0, I)/8, raw cost, eps = 1e-3, the
    # cost formed on the tensor cores each half-step (3xTF32)
    n3, m3 = 20000, 30000
    stage("c3: per-pass")
    c3 = workloads.gaussian_cloud(n3, m3, d=64, seed=0, eps=1e-3)
    keep = []
    X3, Y3 = torch.as_tensor(c3.X).cuda(), torch.as_tensor(c3.Y).cuda()
    a3, b3 = torch.as_tensor(c3.a).cuda(), torch.as_tensor(c3.b).cuda()
    f3 = torch.zeros(n3, dtype=torch.float64, device="cuda")
    g3 = torch.zeros(m3, dtype=torch.float64, device="cuda")
    p3 = pkg.make_problem(a3, b3, X=X3, Y=Y3, eps=1e-3, keep=keep)
    pp = per_pass_ms(pkg, torch, p3, f3, g3, stream, 10, 40, prec=pkg.EOT_PREC_SPLIT_TC)
    flops = 3 * 2.0 * n3 * m3 * 64
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
    o3 = options(pkg, 0, stream.cuda_stream, tol=TOL, max_iter=200000, eps_start=1e-1,
                 prec=pkg.EOT_PREC_SPLIT_TC)
    stage("c3: solve")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st, res = pkg.eot_solve(p3, o3, f3, g3)
    e1.record()
    torch.cuda.synchronize()
    r3 = res.as_dict()
    out["c3_on_the_fly_cost"] = {
        "workload": "gaussian_cloud_20000x30000_d64 (N(0,I)/8, raw cost), eps 1e-3, SPLIT_TC",
        "per_pass_us": round(pp * 1e3, 1),
        "tensor_tflops": round(flops / (pp * 1e-3) / 1e12, 1),
        "tensor_frac": round(flops / (pp * 1e-3) / 1e12 / tf32_peak, 3),
        "tensor_peak_note": "TF32 peak = measured bf16 x (1.1 / 2.25) nominal ratio",
        "stored_cost_equivalent_gbs": round(4.0 * n3 * m3 / (pp * 1e-3) / 1e9, 1),
        "solve_ms": round(e0.elapsed_time(e1), 1), "status": r3["status_name"],
        "total_iters": r3["total_iters"], "l1_marginal_own_cost": r3["l1_marginal"],
        "ncu_pipes": gram_pipes()}
    c3_pair = (c3.X, c3.Y, c3.a, c3.b, 1e-3, f3.cpu().numpy(), g3.cpu().numpy())
    del X3, Y3, f3, g3
    # c4: batch of problems of uneven size and eps (one call)
    stage("c4: batch")
    probs = workloads.batch_problems(512, seed=0)
    keepb = []
    ps = [pkg.make_problem(q.a, q.b, X=q.X, Y=q.Y, eps=q.eps, normalize_cost=True, keep=keepb)
          for q in probs]
    ob = pkg.default_options(tol=TOL, max_iter=200000, eps_start=1e-1)
    # the first call in a process calibrates the gang cost model (once per
    # device); the figure is the median of three calls after it
    t0 = time.perf_counter()
    pkg.eot_solve_batch(ps, ob, [np.zeros(q.n) for q in probs], [np.zeros(q.m) for q in probs])
    first = time.perf_counter() - t0
    times = []
    for _ in range(3):
        fs = [np.zeros(q.n) for q in probs]
        gs = [np.zeros(q.m) for q in probs]
        t0 = time.perf_counter()
        st, resb = pkg.eot_solve_batch(ps, ob, fs, gs)
        times.append(time.perf_counter() - t0)
    tb = statistics.median(times)
    iters = sum(r.total_iters for r in resb)
    # cost bytes of the iterations: two half-steps of 4 n m bytes each per iteration
    cost_bytes = sum(8.0 * q.n * q.m * r.total_iters for q, r in zip(probs, resb))
    ok = sum(1 for r in resb if r.status == pkg.EOT_OK)
    out["c4_batch"] = {"problems": len(probs), "converged": ok, "seconds": round(tb, 3),
                       "problems_per_s": round(len(probs) / tb, 1),
                       "first_call_seconds": round(first, 3),
                       "total_iters": int(iters),
                       "cost_gb_streamed_per_s": round(cost_bytes / tb / 1e9, 1),
                       "note": "host arrays in and out; one persistent cooperative launch "
                               "(graph-captured) runs every problem, gang sizes from a "
                               "calibrated cost model, pass tiles from the autotuner; median "
                               "of 3 calls after a first call that also calibrates the model "
                               "and tunes the tiles (first_call_seconds)"}
    stt, tun = pkg.eot_batch_tuning()
    if stt == pkg.EOT_OK:
        out["c4_batch"]["tuning"] = {
            "tiles_by_m_class": tun["tiles"].tolist(),
            "m_classes": "<=64, <=128, <=256, <=512, <=1024, <=2048, larger",
            "tile_ms": np.round(tun["tile_ms"], 3).tolist(),
            "step_ns": round(tun["step_ns"], 2), "fix_ns": round(tun["fix_ns"], 1),
            "bar_ns": round(tun["bar_ns"], 1),
            "note": "tile bit 0: 64-column blocks of the column half-step; bit 1: eight rows "
                    "a warp per row chunk; calibrated with a copy on every resident CTA"}
    # the same batch with SK-NR(30): every problem a whole solve on one of the
    # worker threads (own stream), the longest predicted first
    stage("c4: batch, SK-NR(30)")
    obn = pkg.default_options(tol=TOL, max_iter=200000, eps_start=1e-1, ell=ELL)
    t0 = time.perf_counter()
    stn, resn = pkg.eot_solve_batch(ps, obn, [np.zeros(q.n) for q in probs],
                                    [np.zeros(q.m) for q in probs])
    tn = time.perf_counter() - t0
    out["c4_batch"]["sknr30"] = {
        "seconds": round(tn, 3), "problems_per_s": round(len(probs) / tn, 1),
        "converged": sum(1 for r in resn if r.status == pkg.EOT_OK),
        "total_iters": int(sum(r.total_iters for r in resn)),
        "note": "ell = 30: whole SK-NR solves (modes, Newton steps) on 8 host worker threads "
                "with their own streams, overlapping on the device; one call"}
    # c5: served stream (Poisson arrivals, continuous batching, warm restarts):
    # at the offered 2000 requests/s (its first requests: far beyond capacity,
    # latency is queueing) and at half the rate measured there
    stage("c5: serving at 2000/s")
    os5 = pkg.default_options(tol=TOL, max_iter=200000, eps_start=1e-1, level_tol=LEVEL_TOL,
                              ell=ELL)
    reqs = workloads.served_stream(seed=1, rate_per_s=2000.0, duration_s=60.0, max_requests=200)
    hi = serve(pkg, reqs, os5)
    rate = max(1.0, 0.5 * hi["solves_per_s"])
    stage(f"c5: serving at {rate:.1f}/s")
    # the same seed: the same sequence of problems (arrival gaps scale with the
    # rate), so its first 200 requests are the ones measured above
    reqs2 = workloads.served_stream(seed=1, rate_per_s=rate, duration_s=20.0, max_requests=2000)
    lo = serve(pkg, reqs2, os5)
    out["c5_serving"] = {
        "offered_2000_per_s": dict(hi, offered_rate_per_s=2000.0,
                                   note="the first 200 requests of the 2000/s stream"),
        "sustainable": dict(lo, offered_rate_per_s=round(rate, 1),
                            note="20 s Poisson stream at 0.5 x the solves/s measured at 2000/s"),
        "note": "n, m log-uniform in [128, 16384], d in {2, 3, 64}, eps in {1e-1, 1e-2, 1e-3}, "
                "half the requests re-use an earlier cloud (warm start from its resident "
                "potentials and modes); every request SK-NR(30) on a stored float32 cost, continuation "
                "from 1e-1 (intermediate levels to 1e-4), a level stops on a stall (under 1% "
                "gain per 1000 iterations); 8 slots, 48 GB budget; admitted solves overlap on "
                "the device (own streams); converged = EOT_OK (the returned pair meets 1e-6)"}
    stage("paper Sec. 5 workloads")
    out["paper_sec5"] = paper_sec5(pkg)
    return out, c3_pair


def paper_sec5(pkg):
    """The paper's Sec. 5 experiments through the library (iteration counts and
    device times; the paper prints figures only, so these are not compared with
    numbers of its own): the 2-D Gaussian experiment of Fig. 5.1 (200 vs 400
    points, raw cost, continuation from eps = 1 halving) under the sequential
    and static-mode protocols and the l sweep at eps = 0.25 from eps' = 1, and
    the single-cell shapes of Fig. 5.2 in R^30 (synthetic N(0, I)/8 clouds stand
    in for the data set), eps from 1 halving to 1/64, l = 30."""
    import workloads
    out = {}
    p = workloads.gaussians_2d(200, seed=0)

    def run(prob, eps, **kw):
        prob.eps = eps
        f, g, r = pkg.solve(prob, tol=TOL, max_iter=200000, **kw)
        return r

    levels = (1.0, 0.5, 0.25)
    prot = {}
    for name, kw in (("sinkhorn", dict(ell=0)), ("sequential_sknr10", dict(ell=10, sequential_modes=1)),
                     ("static_sknr10", dict(ell=10, sequential_modes=0))):
        rs = [run(p, e, eps_start=1.0, eps_factor=0.5, **kw) for e in levels]
        prot[name] = {"iters_at_eps_1_0.5_0.25": [r["iters"] for r in rs],
                      "status": [r["status_name"] for r in rs],
                      "ms_to_0.25": round(rs[-1]["seconds"] * 1e3, 2)}
    sweep = {}
    for ell in (0, 2, 5, 10, 20):
        r = run(p, 0.25, eps_start=1.0, eps_factor=0.25, ell=ell)
        sweep[str(ell)] = {"iters_at_0.25": r["iters"], "ms": round(r["seconds"] * 1e3, 2),
                           "status": r["status_name"]}
    out["two_gaussians_200x400"] = {"protocols": prot, "modes_sweep_from_eps1": sweep}
    cells = {}
    for n, m in ((6507, 3815), (3815, 2982)):
        q = workloads.gaussian_cloud(n, m, d=30, seed=n, eps=1.0 / 64)
        q.normalize_cost = True
        rr = {}
        for ell in (0, 30):
            f, g, r = pkg.solve(q, tol=TOL, max_iter=200000, eps_start=1.0, eps_factor=0.5, ell=ell)
            rr["sinkhorn" if ell == 0 else "sknr30"] = {
                "total_iters": r["total_iters"], "ms": round(r["seconds"] * 1e3, 2),
                "status": r["status_name"]}
        cells[f"{n}x{m}"] = rr
    out["single_cell_shapes_R30"] = cells
    out["note"] = ("L1 target 1e-6 at every level; iteration counts per level (iters) or over "
                   "the continuation (total_iters); device time of the whole solve")
    return out


# The float64 oracle's own iteration counts on the benchmark workload (SK-NR(30)
# and plain Sinkhorn over the eps continuation, subspace iterations of the
# modes), written by tests/golden/make_c2_oracle_counts.py, which calls only
# the oracle.  The timed CPU baseline scales a bounded sample by these counts.
ORACLE_COUNTS = os.path.join(ROOT, "tests", "golden", "c2_oracle_counts.json")


def oracle_sample(seed=0):
    """Bounded sample of the float64 oracle on the benchmark workload: one
    plain Sinkhorn iteration, one SK-NR(30) iteration (row and column
    transforms, L1 test, Newton step with its trial transform), and the mode
    computation's set-up (the coupling) and per-iteration cost (one and two
    subspace iterations), at eps = 1e-3.  Returns the seconds of each."""
    import workloads
    import oracle as O
    prob = workloads.gaussian_mixture(N, M, seed=seed, eps=EPS)
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32).astype(np.float64)
    a, b = prob.a, prob.b
    f0 = O.c_transform_g(np.zeros(M), C, b, EPS)
    g0 = O.c_transform_f(f0, C, a, EPS)
    V = O.splitmix64_uniform(7, N * ELL).reshape(N, ELL)
    V = V - np.ones((N, 1)) * (a @ V)[None, :]
    V = O.eot_oracle._alpha_orthonormalize(V, a)

    def t(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    out = {"sk_iter_s": t(lambda: O.sknr(C, a, b, EPS, None, tol=1e-300, max_iter=1, f0=f0)),
           "sknr_iter_s": t(lambda: O.sknr(C, a, b, EPS, V, tol=1e-300, max_iter=1, f0=f0,
                                           hessian="diag_alpha"))}
    e1 = t(lambda: O.spectral_modes_subspace(f0, g0, C, a, b, EPS, ELL, oversample=10,
                                             tol=0.0, max_iter=1))
    e2 = t(lambda: O.spectral_modes_subspace(f0, g0, C, a, b, EPS, ELL, oversample=10,
                                             tol=0.0, max_iter=2))
    out["eig_iter_s"] = max(e2 - e1, 0.0)
    out["eig_setup_s"] = max(e1 - out["eig_iter_s"], 0.0)
    return out


def oracle_estimate(sample, counts):
    """Seconds of one oracle SK-NR(30) solve and one plain Sinkhorn solve of
    the benchmark workload: the sampled per-iteration times times the oracle's
    own counts (the first continuation level of SK-NR runs plain Sinkhorn)."""
    nr = counts["sknr30"]["per_level"]
    t_nr = 0.0
    for k, lv in enumerate(nr):
        t_nr += lv["iters"] * (sample["sk_iter_s"] if k == 0 else sample["sknr_iter_s"])
        if lv["eig_iters"]:
            t_nr += sample["eig_setup_s"] + lv["eig_iters"] * sample["eig_iter_s"]
    t_sk = (counts["sinkhorn"]["total_iters"] * sample["sk_iter_s"]
            if "sinkhorn" in counts else None)
    return t_nr, t_sk


def _sample_in_child(threads):
    """Run oracle_sample in a fresh Python with the BLAS thread count fixed
    (NumPy's elementwise work is single-threaded either way)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def serve(pkg, reqs, opts, slots=8, budget=48 << 30):
    """Play a request stream into a server in real time; latencies are
    submit -> completion.  Samples the queue depth and admitted bytes."""
    srv = pkg.Server(opts, hbm_budget_bytes=budget, max_slots=slots)
    qmax, hbm_max = 0, 0
    try:
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            while time.perf_counter() - t0 < r["t"]:
                time.sleep(0.0002)
            tickets.append(srv.submit(r["problem"], cloud_id=r["cloud_id"]))
            s5 = srv.status()
            qmax = max(qmax, s5["queued"])
            hbm_max = max(hbm_max, s5["hbm_in_use"])
        done = conv = 0
        for t in tickets:
            while True:
                st5, _, _, _ = srv.poll(t)
                if st5 != pkg.EOT_PENDING:
                    break
                s5 = srv.status()
                qmax = max(qmax, s5["queued"])
                hbm_max = max(hbm_max, s5["hbm_in_use"])
                time.sleep(0.001)
            done += st5 in (pkg.EOT_OK, pkg.EOT_NOT_CONVERGED)
            conv += st5 == pkg.EOT_OK
        t1 = time.perf_counter()
        p50, p99, sps = srv.stats()
    finally:
        srv.close()
    return {"requests": len(reqs), "completed": int(done), "converged": int(conv),
            "p50_ms": round(p50 * 1e3, 2),
            "p99_ms": round(p99 * 1e3, 2), "solves_per_s": round(sps, 1),
            "wall_s": round(t1 - t0, 3), "max_queue_depth": qmax,
            "max_hbm_admitted_gb": round(hbm_max / 2 ** 30, 2)}


def cpu_baseline():
    """The float64 oracle timed on this machine's host cores (bounded sample,
    scaled to one solve by the oracle's own iteration counts), with all cores
    and with one, and the small FP64 configuration (256^2 points, eps 1e-2,
    L1 1e-9) solved in full."""
    import workloads
    import oracle as O
    with open(ORACLE_COUNTS) as fh:
        counts = json.load(fh)
    cores = os.cpu_count() or 1
    s_all = _sample_in_child(cores)
    s_one = _sample_in_child(1)
    nr_all, sk_all = oracle_estimate(s_all, counts)
    nr_one, sk_one = oracle_estimate(s_one, counts)
    c1 = workloads.uniform_square(256, 256, seed=0, eps=1e-2)
    C1 = O.sq_euclidean_cost(c1.X, c1.Y, normalize=True)
    t0 = time.perf_counter()
    r_sk = O.sinkhorn(C1, c1.a, c1.b, 1e-2, tol=1e-9, max_iter=100000)
    t1 = time.perf_counter()
    sk1 = O.sinkhorn(C1, c1.a, c1.b, 1e-1, tol=1e-9, max_iter=100000)
    V1, _ = O.spectral_modes_dense(sk1.f, sk1.g, C1, c1.a, c1.b, 1e-1, ELL)
    r_nr = O.sknr(C1, c1.a, c1.b, 1e-2, V1, tol=1e-9, max_iter=100000)
    t2 = time.perf_counter()
    return {"value": round(nr_all * 1e3, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": (f"float64 NumPy oracle on the {N}x{M} workload: one Sinkhorn iteration "
                       f"({s_all['sk_iter_s']:.2f} s), one SK-NR(30) iteration "
                       f"({s_all['sknr_iter_s']:.2f} s), the modes' set-up "
                       f"({s_all['eig_setup_s']:.2f} s) and one subspace iteration "
                       f"({s_all['eig_iter_s']:.2f} s), scaled by the oracle's own counts for "
                       f"the continuation 1e-1 -> 1e-3 ({counts['sknr30']['total_iters']} SK-NR "
                       f"iterations, {counts['sknr30']['eig_iters']} subspace iterations); BLAS "
                       f"on {cores} threads, elementwise work single-threaded"),
            "plain_sk_ms": None if sk_all is None else round(sk_all * 1e3, 1),
            "plain_sk_iters": counts.get("sinkhorn", {}).get("total_iters"),
            "single_core": {"value": round(nr_one * 1e3, 1),
                            "plain_sk_ms": None if sk_one is None else round(sk_one * 1e3, 1),
                            "cores": 1},
            "c1_fp64_256": {"sinkhorn_s": round(t1 - t0, 3), "sinkhorn_iters": r_sk.iters,
                            "sknr30_static_s": round(t2 - t1, 3), "sknr30_iters": r_nr.iters,
                            "note": "full solves to L1 1e-9 at eps 1e-2 (SK-NR modes from the "
                                    "eps' = 1e-1 solution, included in its time)"}}


def oracle_scores(prob, pairs, c3=None):
    """The float64 oracle's evaluation of pairs the GPU returned: L1 marginal
    error of the benchmark workload's SK-NR and Sinkhorn potentials on the
    same float32 cost, and of the on-the-fly-cost potentials (20000 x 30000,
    d = 64) against the exact float64 cost, in row blocks."""
    import oracle as O
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32).astype(np.float64)
    out = {}
    for name, (f, g) in pairs.items():
        ev = O.evaluate(f, g, C, prob.a, prob.b, EPS)
        out[name] = {"l1": ev["l1"], "row_l1": ev["row_l1"], "col_l1": ev["col_l1"],
                     "gap": ev["gap"]}
    del C
    if c3 is not None:
        X, Y, a, b, eps, f, g = c3
        r = np.zeros(X.shape[0])
        c = np.zeros(Y.shape[0])
        step = 1000
        for i0 in range(0, X.shape[0], step):
            i1 = min(X.shape[0], i0 + step)
            Cb = O.sq_euclidean_cost_gram(X[i0:i1], Y)
            P = O.plan(f[i0:i1], g, Cb, a[i0:i1], b, eps)
            r[i0:i1] = P.sum(axis=1)
            c += P.sum(axis=0)
        out["c3_on_the_fly_exact_cost"] = {
            "l1": float(np.abs(r - a).sum() + np.abs(c - b).sum()),
            "row_l1": float(np.abs(r - a).sum()), "col_l1": float(np.abs(c - b).sum()),
            "note": "potentials from the on-the-fly-cost solve, scored against the exact "
                    "float64 cost (the kernel meets 1e-6 against its own cost)"}
    return out


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    with open(ORACLE_COUNTS) as fh:
        counts = json.load(fh)
    for _ in range(max(0, args.warmup)):
        oracle_sample()
    vals, samples = [], []
    for _ in range(max(1, args.steps)):
        smp = oracle_sample()
        samples.append(smp)
        vals.append(oracle_estimate(smp, counts)[0] * 1e3)
    v = round(statistics.median(vals), 1)
    smp = samples[len(samples) // 2]
    cores = os.cpu_count() or 1
    cb = {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
          "sample": (f"per step: one Sinkhorn iteration, one SK-NR(30) iteration, the modes' "
                     f"set-up and one subspace iteration of the float64 NumPy oracle on the "
                     f"{N}x{M} workload (median: {smp['sk_iter_s']:.2f}, {smp['sknr_iter_s']:.2f}, "
                     f"{smp['eig_setup_s']:.2f}, {smp['eig_iter_s']:.2f} s), scaled by the "
                     f"oracle's own counts ({counts['sknr30']['total_iters']} SK-NR iterations, "
                     f"{counts['sknr30']['eig_iters']} subspace iterations over the "
                     f"continuation); BLAS on up to {cores} threads")}
    out = {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "m": M, "d": 3, "eps": EPS, "tol": TOL,
                      "ell": ELL, "level_tol": LEVEL_TOL, "eig_tol": EIG_TOL,
                      "oversample": 10}, "impl": "reference",
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def profile_case(name):
    """Small cases for ncu captures: one plain Sinkhorn launch of two iterations
    on a 16384 x 16384 cost (coop16k); column and row transforms on an 8192 x
    8192 cost (stream8k); one SK-NR(30) solve of the 4096 x 4096 workload
    (sknr4k, two solves); ten on-the-fly-cost iterations on 20000 x 30000 points in R^64
    (gram); the batch of 512 problems (batch)."""
    import torch
    import workloads
    import paper_2506_14780_gb300 as pkg
    pkg.load()
    if name == "coop16k":
        prob = workloads.gaussian_mixture(16384, 16384, seed=1, eps=1e-2)
        _, _, res = pkg.solve(prob, tol=1e-300, ell=0, eps_start=0.0, max_iter=2)
    elif name == "stream8k":
        n = 8192
        prob = workloads.gaussian_mixture(n, n, seed=2, eps=1e-2)
        X = torch.as_tensor(prob.X).double().cuda()
        Y = torch.as_tensor(prob.Y).double().cuda()
        C = torch.cdist(X, Y) ** 2
        C = (C / C.max()).float().contiguous()
        a = torch.as_tensor(prob.a).cuda()
        b = torch.as_tensor(prob.b).cuda()
        f = torch.zeros(n, dtype=torch.float64, device="cuda")
        og = torch.zeros(n, dtype=torch.float64, device="cuda")
        of = torch.zeros(n, dtype=torch.float64, device="cuda")
        for _ in range(2):
            if pkg.eot_ctransform(pkg.EOT_SIDE_COL, n, n, C, f, a, None, 1e-2, og, None) != 0:
                raise RuntimeError(pkg.last_error())
            if pkg.eot_ctransform(pkg.EOT_SIDE_ROW, n, n, C, og, b, of, 1e-2, of, None) != 0:
                raise RuntimeError(pkg.last_error())
        res = {"status_name": "EOT_OK"}
    elif name == "s4_8k":
        # three single SK-NR iterations (eot_sknr_step) on the 8192^2 mixture
        # (268 MB cost, beyond L2) from a Sinkhorn state with 30 modes
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        st4 = sknr_stage_times(pkg, torch, 8192, 2, 1e-2, flush, torch.cuda.current_stream(),
                               reps=1)
        res = {"status_name": f"stage us {[round(x * 1e6, 1) for x in st4]}"}
    elif name == "sknr4k":
        # two solves (the first also builds the solver) under the benchmark's protocol
        prob = workloads.gaussian_mixture(N, M, seed=0, eps=EPS)
        for _ in range(2):
            _, _, res = pkg.solve(prob, tol=TOL, ell=ELL, eps_start=1e-1, max_iter=200000,
                                  level_tol=LEVEL_TOL, oversample=10, eig_tol=EIG_TOL,
                                  eig_max_iter=100)
    elif name == "batch":
        probs = workloads.batch_problems(512, seed=0)
        keepb = []
        ps = [pkg.make_problem(q.a, q.b, X=q.X, Y=q.Y, eps=q.eps, normalize_cost=True, keep=keepb)
              for q in probs]
        ob = pkg.default_options(tol=TOL, max_iter=200000, eps_start=1e-1)
        st, _ = pkg.eot_solve_batch(ps, ob, [np.zeros(q.n) for q in probs],
                                    [np.zeros(q.m) for q in probs])
        res = {"status_name": "EOT_OK" if st == pkg.EOT_OK else str(st)}
    else:
        prob = workloads.gaussian_cloud(20000, 30000, d=64, seed=0, eps=1e-3)
        _, _, res = pkg.solve(prob, tol=1e-300, ell=0, eps_start=0.0, max_iter=10,
                              prec=pkg.EOT_PREC_SPLIT_TC)
    torch.cuda.synchronize()
    stage(f"case {name}: {res.get('status_name')}")


def main():
    args = parse()
    if args.oracle_sample:
        print(json.dumps(oracle_sample()), flush=True)
        return
    if args.case:
        profile_case(args.case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
