#!/usr/bin/env python
"""Benchmark of the 1D NMGM on GB300: steady solves/s and p99 latency at
residual <= 1e-10 (FP64 Newton multigrid, nested Algorithm 3).

Workload (one step = one batch of independent solves, inputs resident in HBM):
1D irregular channel, N = 4096 cells on [0, 25], width
B(x) = 1 + 0.2 sin(2 pi k x / 25), k ~ U{1..4}, Gaussian hump A ~ U[0.05, 0.2],
xc ~ U[8, 12], w ~ U[1, 2], upstream discharge 4.42, downstream depth 2.0,
WENO3 + HLL, simplified Jacobian J3, 8-level multigrid, seeded instances.

Arms
  default            CUDA library through its C ABI (device-timed value; e2e
                     through the same API from pinned host buffers).
  --impl reference   the CPU oracle on the host cores (the slow baseline).

Multi-GPU: independent replicas (each rank solves its own instances; no
collective on the data path), reported as weak scaling.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "steady solves/s and p99 latency at residual <=1e-10 vs plain FP64 Newton-MG"
UNIT = "solves/s"
TOL = 1e-10  # the metric's residual threshold: the default FP64 line stops at res < TOL
# Lines that compare precisions or execution forms at equal solution accuracy stop at res < TOL_SOLUTION
# and are checked against the oracle's converged discrete solution (res < TOL_CONVERGED). Damped Newton
# (tau = 0.6) leaves a solve stopped at res < 1e-10 a few 1e-9 from that solution whatever the precision
# of its steps. On the oracle, res < 3e-13 puts the 4096-cell channels within 1.6e-11 of it (48 seeds)
# and the serving requests within 4.9e-11 (the first 24; res < 1e-12 left one at 1.3e-10).
TOL_SOLUTION = 3e-13
TOL_CONVERGED = 3e-14
MIXED_BOUND = 1e-10  # relative distance to the converged FP64 discrete solution
# Derived FMA peaks (reported beside the measured ones of measure_fma_peaks, which the rooflines use)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070  # SMs x FP64 FMA/clk/SM x 2 flop x max SM GHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070  # SMs x FP32 lanes x 2 flop x max SM GHz
# The latency form of the 1D solve timed beside the block form: cluster sizes and the smallest
# multigrid level (cells) run on every CTA of the cluster.
CLUSTER_CTAS = (8, 16)
CLUSTER_TEAM_CELLS = 1024
# Light-load serving latency: the first LIGHT_REQUESTS serving requests arriving at LIGHT_RATE per second,
# through the server in the block form and with its cluster form (LIGHT_CTAS CTAs per problem while at most
# LIGHT_MAX_IN_FLIGHT solves are in flight: 16 x 9 = 144 of the 152 SMs).
LIGHT_REQUESTS, LIGHT_RATE, LIGHT_CTAS, LIGHT_MAX_IN_FLIGHT = 128, 25.0, 16, 9
# DRAM bytes (read + write) of one colour pass of k2_sor_split<double, J9> at 512 x 256 with colour-major J9,
# from one ncu capture of `bench.py --workload wedge2d --phases-only` (None: not captured for this kernel).
SOR_PASS_TRAFFIC_512 = 34.606336e6 + 0.020480e6
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_solve launch of the 608-channel J3 step
# per (precision, launch shape, stopping tolerance), each from a one-pass ncu capture of
# `bench.py --steps 1 --warmup 3 --no-cpu --no-serving --shape S [--precision mixed]`; no entry: not captured
# (the bytes grow with the Newton steps, so a capture stands only for its own tolerance).
TRAFFIC_608 = {("fp64", "128x4", 1e-10): 209567876096 + 103480428800,
               ("mixed", "256x4", 3e-13): 153810537216 + 96052265472,
               ("mixed", "192x4", 3e-13): 144785353728 + 91365382400}


# The 1D workloads of the default line: the irregular channel (N = 4096, the metric's configuration)
# and the small smooth channel (N = 200): cells, levels, nested start (cells), description, seeds.
CONFIG1D = {"irregular": (4096, 8, 256, "1D irregular channel, N=4096, 8-level MG", "numpy default_rng(2000 + k)"),
            "small": (200, 4, 25, "1D smooth subcritical channel, N=200, 4-level MG, omega 1.2",
                      "numpy default_rng(1000 + k)")}


def workload_config(batch, nb, precision="fp64", tol=TOL, kind="irregular"):
    prec = "FP64" if precision == "fp64" else "mixed FP64 residual/update + FP32 Jacobian/MG"
    N, levels, start, desc, seeds = CONFIG1D[kind]
    return {"workload": "%s, J%d, %s, subcritical" % (desc, nb, prec),
            "precision": precision,
            "N": N, "levels": levels, "nest_start_cells": start, "instances_per_step_per_gpu": batch,
            "jacobian": "J3 (simplified)" if nb == 3 else "J5 (full)", "tol": tol,
            "l2": ("inputs + workspace per step (%.0f MB) exceed the 129 MB L2" % (batch * N * 0.95e-3)
                   if batch * N * 0.95e3 >= 2 * 129e6 else
                   "inputs + workspace per step (%.0f MB) fit in L2: 256 MB written between timed steps, each "
                   "step timed on its own" % (batch * N * 0.95e-3)),
            "seeds": seeds}


def make_instances(first, count, nb, tol=TOL, kind="irregular"):
    from paper_2505_10857_gb300 import inputs as I
    make = I.channel_irregular if kind == "irregular" else I.channel_small
    inps = [make(k) for k in range(first, first + count)]
    prms = [I.Params1D.for_problem(p, tol=tol, n_max=800, nb=nb) for p in inps]
    return inps, prms


# ------------------------------------------------------------------------------------------------
# Algorithmic FP64 flop count of one solve (add/sub/mul = 1, fused multiply-add = 2, division = 1,
# square root = 1), following the steps the kernels execute; per cell unless noted.
F_WENO = 38          # one component of one cell: smoothness, candidates, one reciprocal, two weights
F_STATE = 10         # HLL quantities of one interface state (1/H, u, h, c, physical flux)
F_STATE_Q = 3        # the same for a state that differs from a computed one only in Q (u, flux)
F_HLL = 20           # HLL combination of two states
F_SOURCE = 36        # two-point Gauss source of one cell (Eq. 9)
F_UPDATE = 4         # damped Newton update of H and Q
F_DINV = 9           # 2x2 inverse
F_INTERP = 8         # App. A per fine cell


def f_res():
    """Residual alone per cell (Eq. 10): WENO of both components of the
    cells j-1, j, j+1, two faces of 1 reciprocal + 2 states + HLL, the
    source and the differences."""
    return 6 * F_WENO + 2 * (1 + 2 * F_STATE + F_HLL) + F_SOURCE + 4


def f_res_jac(nb):
    """Residual + FD Jacobian per cell: 8 WENO variants (+6 perturbations);
    per face 8 full interface states (the two base states and the six with H
    perturbed), 6 states with only Q perturbed (u and the flux from the base
    state's 1/H and pressure term: F_STATE_Q) and 9 HLL combinations; per cell
    the base source and one source per block (an H perturbation; a Q
    perturbation leaves the source), and per block the differences and
    scaling (+6 for the diagonal)."""
    pass_a = 8 * F_WENO + 6
    pass_b = 8 * F_STATE + 6 * F_STATE_Q + 9 * F_HLL
    pass_c = (nb + 1) * F_SOURCE + 18 * nb + 6
    return pass_a + pass_b + pass_c


def f_smooth(N, nb, steps):
    """Fused multicolour SOR: per pass the neighbour sum and D^-1 product
    once (8(nb-1)+6) and the relaxation per repeat (6), cells of one colour."""
    C = (nb - 1) // 2 + 1
    seq = [c for _ in range(steps) for c in list(range(C)) + list(range(C - 1, -1, -1))]
    tot, i = 0, 0
    while i < len(seq):
        j = i
        while j < len(seq) and seq[j] == seq[i]:
            j += 1
        ncell = len(range(seq[i], N, C))
        tot += ncell * (8 * (nb - 1) + 6 + 6 * (j - i))
        i = j
    return tot


def f_restrict(nb):  # per coarse cell
    return 16 * nb + 2


def lu_flops(n, kl):
    return n * (kl + 1 + 4 * kl * kl), n * (6 * kl + 1)  # factor, solve


def solve_flops(N, levels, start, iters, nb, nu1, nu2, nu3, mixed=False):
    """(FP64 flops, FP32 flops) of one nested solve. FP64 path: R and J
    together at each state. Mixed path: the FP64 residual at each state, the
    FP32 Jacobian (which also forms R) and linear solve at each step."""
    L = levels - 1
    f64 = f32 = 0.0
    for l in range(start, -1, -1):
        Nl = N >> l
        if l < start:
            f64 += F_INTERP * Nl
        lin = 0.0
        nbl = [nb if k == l else 3 for k in range(L + 1)]
        for k in range(l + 1, L + 1):
            lin += 8 * nbl[k - 1] * (N >> k)
        for k in range(l, L):
            lin += F_DINV * (N >> k)
        hw = (nbl[L] - 1) // 2
        fac, sol = lu_flops(2 * (N >> L), 2 * hw + 1)
        lin += fac
        if l == L:
            lin += sol
        else:
            vc = sol
            for k in range(l, L):
                Nk = N >> k
                vc += f_smooth(Nk, nbl[k], nu1) + f_smooth(Nk, nbl[k], nu2) + (N >> (k + 1)) * f_restrict(nbl[k]) \
                    + 2 * Nk
            lin += nu3 * vc
        if mixed:
            f64 += f_res() * Nl + iters[l] * Nl * (f_res() + F_UPDATE)
            f32 += iters[l] * (Nl * (f_res_jac(nb) + 1) + lin)
        else:
            f64 += f_res_jac(nb) * Nl + iters[l] * (Nl * (f_res_jac(nb) + F_UPDATE) + lin)
    return f64, f32


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json
    at the repository root), else the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


# ------------------------------------------------------------------------------------------------
def measure_fma_peaks(device=0, reps=3):
    """FP64 and FP32 FMA throughput of this GPU (TFLOP/s, best of `reps`
    launches after one untimed), from the library's probe kernel: 8 resident
    blocks of 256 threads per SM, 8 independent FMA chains per thread."""
    import torch

    from paper_2505_10857_gb300 import nswe
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, threads = 8 * sms, 256
    stream = torch.cuda.current_stream(device)
    out = {"sms": sms, "blocks": blocks, "threads": threads}
    for name, prec, dt, iters in (("fp64", nswe.PREC_FP64, torch.float64, 16384),
                                  ("fp32", nswe.PREC_MIXED, torch.float32, 262144)):
        sink = torch.zeros(blocks * threads, dtype=dt, device=f"cuda:{device}")
        best = None
        for r in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = nswe.nswe_probe_fma(stream.cuda_stream, prec, blocks, threads, iters, sink)
            b.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                t = fl / (a.elapsed_time(b) / 1000.0) / 1e12
                best = t if best is None else max(best, t)
        out[name + "_tflops"] = best
        out[name + "_finite"] = bool(torch.isfinite(sink).all())
    out["what"] = "nswe_probe_fma: best of %d timed launches (CUDA events) after one untimed" % reps
    return out


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------------------------------------
def _oracle_worker(args):
    first, count, nb, tol, kind = args
    import oracle
    inps, prms = make_instances(first, count, nb, tol, kind)
    out = []
    for p, q in zip(inps, prms):
        U, info = oracle.solve_problem(p, q)
        out.append((U, info["status"]))
    return out


def oracle_sample(first, count, nb, workers, tol=TOL, kind="irregular"):
    """Solves `count` instances with the CPU oracle on `workers` processes
    (spawn); returns (wall seconds, results)."""
    import oracle
    oracle.build()
    chunks = [(first + i, 1, nb, tol, kind) for i in range(count)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_worker, [(first, 1, nb, tol, kind)] * workers)  # warm the workers
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, chunks)
        wall = time.perf_counter() - t0
    return wall, [r[0][0] for r in res]


def oracle_build_info():
    import oracle
    return oracle.compiler_info()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = host_cores()
    sample = cores
    times = []
    for s in range(args.warmup + args.steps):
        wall, _ = oracle_sample((s * sample) % args.batch, sample, args.nb, cores, TOL, args.config1d)
        if s >= args.warmup:
            times.append(wall)
    ms = 1000.0 * sum(times) / len(times)
    value = sample / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.batch, args.nb, kind=args.config1d),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} of the step's {args.batch} instances per timed step (seeds rotate), "
                                       f"one solve per process (spawn pool)", **oracle_build_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# Replicas across ranks (one process per GPU): each rank solves its own instances, no collective on
# the data path; only the timing is reduced.

def replica_instances(rank, world, per_rank):
    """Instance indices of `rank`: a disjoint block of per_rank seeds per rank."""
    assert 0 <= rank < world and per_rank > 0
    return rank * per_rank, per_rank


def max_over_ranks(x, world, device=None):
    """Max of a float over all ranks (identity for one process)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, per_rank, ms_max):
    """Solves per second of the whole job: all ranks' instances over the slowest rank's time."""
    return world * per_rank / (ms_max / 1000.0)


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2505_10857_gb300 import nswe

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B, nb = args.batch, args.nb
    mixed = args.precision == "mixed"
    tol = args.tol if args.tol is not None else (TOL_SOLUTION if mixed else TOL)
    first, _ = replica_instances(rank, world, B)
    kind = args.config1d
    inps, prms = make_instances(first, B, nb, tol, kind)
    # about 0.95 KB of arena per finest cell: flush L2 between timed steps when a step's data fits in it
    l2_flush = B * inps[0].N * 0.95e3 < 2 * 129e6
    prm = nswe.params_from(prms[0])
    prm.precision = nswe.PREC_MIXED if mixed else nswe.PREC_FP64
    for q in prms[1:]:
        assert list(q.eps) == list(prms[0].eps) and q.omega == prms[0].omega

    ctx = nswe.Context(local_rank)
    stream = torch.cuda.current_stream(dev)
    probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps]
    # every problem's guess and result as a 256-byte-aligned view of one device
    # buffer each, so that the end-to-end step moves them in one copy each way
    u0_off = np.cumsum([0] + [-(-p.U0_start.size // 32) * 32 for p in inps])
    u_off = np.cumsum([0] + [-(-2 * p.N // 32) * 32 for p in inps])
    U0_all = torch.zeros(int(u0_off[-1]), dtype=torch.float64, device=dev)
    U_all = torch.zeros(int(u_off[-1]), dtype=torch.float64, device=dev)
    U0s = [U0_all[int(u0_off[k]):int(u0_off[k]) + p.U0_start.size].view(2, -1) for k, p in enumerate(inps)]
    Us = [U_all[int(u_off[k]):int(u_off[k]) + 2 * p.N].view(2, -1) for k, p in enumerate(inps)]
    for k, p in enumerate(inps):
        U0s[k].copy_(torch.from_numpy(p.U0_start))

    def step(want_info=False):
        return nswe.nswe_newton_solve_batch(ctx, probs, U0s, Us, prm, want_info=want_info)

    # Steady throughput: consecutive steps alternate between two independent copies of the batch,
    # each with its own context and stream, so that one step's launch starts on the SMs that the
    # previous step's slowest problems leave idle. Every step still solves all B problems.
    pipelined = not l2_flush and not args.sequential_steps
    if pipelined:
        stream_b = torch.cuda.Stream(dev)
        ctx_b = nswe.Context(local_rank, stream=stream_b.cuda_stream)
        probs_b = [nswe.Problem1D.from_inputs(ctx_b, p) for p in inps]
        U0_all_b, U_all_b = torch.zeros_like(U0_all), torch.zeros_like(U_all)
        U0s_b = [U0_all_b[int(u0_off[k]):int(u0_off[k]) + p.U0_start.size].view(2, -1) for k, p in enumerate(inps)]
        Us_b = [U_all_b[int(u_off[k]):int(u_off[k]) + 2 * p.N].view(2, -1) for k, p in enumerate(inps)]
        U0_all_b.copy_(U0_all)
        torch.cuda.synchronize()

        def step_b():
            nswe.nswe_newton_solve_batch(ctx_b, probs_b, U0s_b, Us_b, prm, want_info=False)

    # Launch-shape autotuning on this batch (before the warm-up; not timed).
    tune = None
    shape = 0
    if args.shape is not None:
        shape = args.shape
        nswe.nswe_ctx_set_solve_shape(ctx, prm.precision, shape)
    elif not args.no_autotune:
        ms_shapes, best = nswe.nswe_autotune_solve_batch(ctx, probs, U0s, Us, prm, reps=1)
        tune = {"shapes": ["%dx%d" % tb for tb in nswe.solve_shapes()], "ms_per_batch": ms_shapes,
                "chosen": "%dx%d" % nswe.solve_shapes()[best],
                "what": "threads per block x resident blocks per SM of k_solve, one timed batch each"}
        shape = best
    shape_name = "%dx%d" % nswe.solve_shapes()[shape]
    if pipelined:
        nswe.nswe_ctx_set_solve_shape(ctx_b, prm.precision, shape)

    def barrier():
        if world > 1:
            dist.barrier()

    for w in range(args.warmup):
        step_b() if (pipelined and w % 2) else step()
    torch.cuda.synchronize()

    # ---- device-timed throughput (inputs resident in HBM)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    if l2_flush:
        # the step's data fits in L2: each step timed on its own, a 256 MB write between steps
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
        ea = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for s in range(args.steps):
            flush.fill_(float(s))
            ea[s].record(stream)
            step()
            eb[s].record(stream)
        torch.cuda.synchronize()
        per_launch = [ea[s].elapsed_time(eb[s]) for s in range(args.steps)]
        ms = sum(per_launch) / args.steps
        del flush
    else:
        # one step at a time on one stream (reported beside the steady figure, and the roofline's
        # per-launch duration)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for s in range(args.steps):
            step()
            ev[s + 1].record(stream)
        torch.cuda.synchronize()
        per_launch = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
        ms = ev[0].elapsed_time(ev[-1]) / args.steps
        ms_sequential = ms
        if pipelined:
            # steady throughput: the same K steps alternating between the two streams
            barrier()
            torch.cuda.synchronize()
            e0, e1, eb_end = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            stream_b.wait_event(e0)
            for s in range(args.steps):
                step_b() if s % 2 else step()
            eb_end.record(stream_b)
            stream.wait_event(eb_end)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
    barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, dev)
    value = whole_job_rate(world, B, ms_max)

    # ---- one more step with per-solve records (status, iterations, device timestamps)
    infos = step(want_info=True)
    torch.cuda.synchronize()
    status = [i["status"] for i in infos]
    res0 = [i["res"][0] for i in infos]
    t0 = min(i["t_start_ns"] for i in infos)
    lat = sorted((i["t_end_ns"] - t0) / 1e6 for i in infos)
    dur = sorted((i["t_end_ns"] - i["t_start_ns"]) / 1e6 for i in infos)

    def pct(a, p):
        return a[min(len(a) - 1, int(math.ceil(p / 100.0 * len(a))) - 1)]

    fl = [solve_flops(inps[k].N, inps[k].levels, inps[k].start_level, infos[k]["iters"], nb, prm.nu1, prm.nu2,
                      prm.nu3, mixed)
          for k in range(B)]
    f64, f32 = sum(a for a, _ in fl), sum(b for _, b in fl)
    launch_ms = statistics.mean(per_launch)
    # the roofline of the steady form: each launch's flops over the timed region per launch
    launch_ms_steady = ms if pipelined else launch_ms
    peaks = measure_fma_peaks(local_rank)
    p64, p32 = peaks["fp64_tflops"], peaks["fp32_tflops"]
    # FP64-equivalent rate: FP32 flops weighted by the FP64:FP32 peak ratio, so
    # that achieved / FP64 peak is the fraction of the time at both peaks.
    flops = f64 + f32 * p64 / p32
    achieved = flops / (launch_ms_steady / 1000.0) / 1e12
    achieved_one = flops / (launch_ms / 1000.0) / 1e12

    # ---- single-solve latency (one instance alone on the GPU)
    single = []
    for s in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nswe.nswe_newton_solve(ctx, probs[s], U0s[s], Us[s], prm, want_info=False)
        e1.record(stream)
        torch.cuda.synchronize()
        single.append(e0.elapsed_time(e1))
    # the latency form: the same solves, each alone on a thread-block cluster
    single_cluster = {}
    for ctas in CLUSTER_CTAS:
        try:
            nswe.nswe_ctx_set_solve_cluster(ctx, ctas, CLUSTER_TEAM_CELLS)
            t = []
            for s in range(3):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nswe.nswe_newton_solve(ctx, probs[s], U0s[s], Us[s], prm, want_info=False)
                e1.record(stream)
                torch.cuda.synchronize()
                t.append(e0.elapsed_time(e1))
            single_cluster[str(ctas)] = statistics.median(t)
        except nswe.NsweError as e:
            single_cluster[str(ctas)] = f"unavailable: {e}"
        finally:
            nswe.nswe_ctx_set_solve_cluster(ctx, 1, CLUSTER_TEAM_CELLS)

    # ---- end to end through the C ABI from pinned host buffers: every step
    # uploads all problems' geometry (one batched call) and guesses, solves,
    # and reads the results back
    pin_sf = [torch.from_numpy(p.sig_face).pin_memory().numpy() for p in inps]
    pin_gq = [torch.from_numpy(p.gq_all()).pin_memory().numpy() for p in inps]
    pin_u0 = U0_all.cpu().pin_memory()
    pin_u = torch.empty_like(U_all, device="cpu").pin_memory()
    bcl, bcr = [p.bcl for p in inps], [p.bcr for p in inps]
    h2d = sum(a.nbytes for a in pin_sf + pin_gq) + pin_u0.numel() * 8  # the bytes copied, padding included
    if pipelined:
        # steady form: the steps alternate between the two batches and streams; each step uploads its
        # geometry and guesses, solves and copies its results back, asynchronously on its own stream,
        # so one step's uploads overlap the other's solve; every step's copies lie in the timed region
        pin_u_b = torch.empty_like(U_all_b, device="cpu").pin_memory()
        d2h = pin_u.numel() * 8
        sets = [(ctx, probs, U0_all, U0s, U_all, Us, pin_u, stream),
                (ctx_b, probs_b, U0_all_b, U0s_b, U_all_b, Us_b, pin_u_b, stream_b)]

        def e2e_step(s):
            c_ctx, c_probs, c_u0_all, c_u0s, c_u_all, c_us, c_pin_u, c_stream = sets[s % 2]
            nswe.nswe_prob_set_geometry_batch_1d(c_ctx, c_probs, pin_sf, pin_gq, bcl, bcr)
            with torch.cuda.stream(c_stream):
                c_u0_all.copy_(pin_u0, non_blocking=True)
            nswe.nswe_newton_solve_batch(c_ctx, c_probs, c_u0s, c_us, prm, want_info=False)
            with torch.cuda.stream(c_stream):
                c_pin_u.copy_(c_u_all, non_blocking=True)

        for s in range(args.warmup):
            e2e_step(s)
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for s in range(args.steps):
            e2e_step(s)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(1000.0 * (time.perf_counter() - w0) / args.steps, world, dev)
        assert np.array_equal(pin_u.numpy(), U_all.cpu().numpy())  # the results copied back are the solves'
    else:
        d2h = pin_u.numel() * 8 + B * ctypes.sizeof(nswe.Info)
        e2e_times = []
        for s in range(args.warmup + args.steps):
            barrier()
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            nswe.nswe_prob_set_geometry_batch_1d(ctx, probs, pin_sf, pin_gq, bcl, bcr)
            U0_all.copy_(pin_u0, non_blocking=True)
            infos_e = step(want_info=True)  # synchronous: includes the D2H of the per-solve records
            pin_u.copy_(U_all, non_blocking=True)
            torch.cuda.synchronize()
            if s >= args.warmup:
                e2e_times.append(time.perf_counter() - w0)
            assert all(i["status"] == 0 for i in infos_e)
        e2e_ms = max_over_ranks(1000.0 * statistics.mean(e2e_times), world, dev)
    e2e_value = whole_job_rate(world, B, e2e_ms)

    out = None
    if rank == 0:
        cpu = None
        parity = None
        if world == 1 and not args.no_cpu:
            cores = host_cores()
            n = B  # the whole step: about 10-15 s of CPU work on 16 cores
            wall, refs = oracle_sample(first, n, nb, cores, tol, kind)
            n1 = 4  # per-solve latency on one core: a few solves one after another in one process
            wall1, _ = oracle_sample(first, n1, nb, 1, tol, kind)
            cpu = {"value": n / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"all {n} instances of the step, one solve per process (spawn pool), "
                             f"{wall:.1f} s wall",
                   "latency_1core_ms": 1000.0 * wall1 / n1,
                   "latency_1core_sample": f"the step's first {n1} instances solved one after another on one core",
                   **oracle_build_info()}
            what = "the oracle's solve with the same stopping test"
            if tol < TOL:  # equal-accuracy lines: against the converged discrete solution
                _, refs = oracle_sample(first, n, nb, cores, TOL_CONVERGED, kind)
                what = f"the oracle's converged discrete solution (res < {TOL_CONVERGED:g})"
            errs = [float(np.abs(Us[k].cpu().numpy() - refs[k]).max() / np.abs(refs[k]).max()) for k in range(n)]
            parity = {"max_rel_err_vs_oracle": max(errs), "instances": n, "reference": what,
                      "bound": MIXED_BOUND if tol < TOL else 1e-10}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
            "config": workload_config(B, nb, args.precision, tol, kind),
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99),
                           "what": "per-solve completion time from the start of its batch (device timer)",
                           "solve_p50": pct(dur, 50), "solve_p99": pct(dur, 99),
                           "single_solve_alone": statistics.median(single),
                           "single_solve_cluster": single_cluster,
                           "single_solve_cluster_what": "the same solve alone on a thread-block cluster of that "
                                                        "many CTAs (nswe_ctx_set_solve_cluster; multigrid levels "
                                                        f"of >= {CLUSTER_TEAM_CELLS} cells on every CTA)"},
            "converged": {"all_status_ok": all(s == 0 for s in status), "max_res": max(res0),
                          "mean_newton_iters": statistics.mean(i["total_iters"] for i in infos)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms,
                    "form": ("steps alternating between two batches and streams, copies and solves asynchronous"
                             if pipelined else "one step at a time, synchronous")},
            "steps_form": ({"form": "steady: consecutive steps alternate between two independent copies of the "
                                    "batch, each with its own context and stream, so that a step's launch starts "
                                    "on the SMs the previous step's slowest problems leave idle; every step "
                                    "solves all instances; ms_per_step = timed region / steps",
                            "one_step_at_a_time": {"ms_per_step": ms_sequential,
                                                   "value": whole_job_rate(world, B, ms_sequential)}}
                           if pipelined else {"form": "one step at a time on one stream"}),
            "gpu_launches": args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": p64,
                         "unit": "TFLOP/s", "frac": achieved / p64,
                         "traffic": (TRAFFIC_608.get((args.precision, shape_name, tol))
                                     if (B == 608 and nb == 3 and kind == "irregular") else None),
                         "traffic_note": "DRAM bytes per launch from one ncu capture of this workload; "
                                         "8-16 % of the HBM copy rate over the launch, far from bound",
                         "kernel": f"k_solve (persistent nested NMGM, one block per instance, shape {shape_name})",
                         "flops_per_launch": flops, "fp64_flops": f64, "fp32_flops": f32,
                         "launch_ms": launch_ms_steady,
                         "launch_ms_note": ("timed region per launch, two launches in flight (steady form); one "
                                            f"launch alone takes {launch_ms:.1f} ms, frac "
                                            f"{achieved_one / p64:.3f} of the peak" if pipelined
                                            else "mean launch duration (CUDA events on the launching stream)"),
                         "peak_note": "FP64 FMA peak measured in this run (nswe_probe_fma); derived "
                                      "152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz = %.3f TFLOP/s" % (FP64_PEAK_GFLOPS / 1e3)
                                      + ("; FP32 flops counted at the measured FP64/FP32 peak ratio" if mixed else ""),
                         "peaks_measured": peaks},
            "clocks": clk,
        }
        if tune:
            out["autotune"] = tune
        if cpu:
            out["cpu_baseline"] = cpu
            out["parity"] = parity
        if world == 1 and not args.no_serving:
            out.update(serving_comparison(args, ctx))
        print(json.dumps(out), flush=True)
    return out


def run_wedge2d(args):
    """2D measurement (not the default line): a nested solve of the seeded
    wedge channel at the size given by --nx/--ny, plus the time of each
    phase of one Newton step at 512 x 256 (Section 4 kernels, FP64)."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    ctx = nswe.Context(0)
    stream = torch.cuda.current_stream()

    def timed(f, reps):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            f()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    big = I.wedge_channel(0)
    pb = nswe.Problem2D.from_inputs(ctx, big)
    n = big.Nx * big.Ny
    X, _ = big.centres(0)
    s0 = big.bc_state[0]
    U = torch.tensor(np.stack([s0[0] * (1 + 0.01 * np.sin(X.ravel())), np.full(n, s0[1]), np.full(n, s0[2])]),
                     dtype=torch.float64, device="cuda")
    R, res = torch.zeros_like(U), torch.zeros(1, dtype=torch.float64, device="cuda")
    J9 = torch.zeros((9, 9, n), dtype=torch.float64, device="cuda")
    J21 = torch.zeros((21, 9, n), dtype=torch.float64, device="cuda")
    dU = torch.zeros_like(U)
    prm = nswe.params(96, big.levels, omega=args.omega2d, nu1=20, nu2=20, nu3=3)
    # The dominant kernel of the 2D solve: the multicolour block-SOR pass (Eq. 22) of the finest level,
    # with J9 colour-major as the solve stores levels of 512 x 256 cells and more. Per-launch duration from
    # two smoothing runs of different lengths (CUDA events on the launching stream): their difference holds
    # colour passes only.
    nswe.nswe_jacobian_simplified(ctx, pb, 0, U, 1e-6, 3.0, R, J9, res)
    w3 = (big.Nx + 2) // 3
    ii, jj = np.meshgrid(np.arange(big.Nx), np.arange(big.Ny))
    pos = torch.from_numpy(((((ii + jj) % 3) * big.Ny + jj) * w3 + ii // 3).ravel()).cuda()
    J9cm = torch.zeros((9, 9, 3 * big.Ny * w3), dtype=torch.float64, device="cuda")
    J9cm[:, :, pos] = J9
    sweeps = {}
    for nu in (10, 30):
        q = nswe.params(96, big.levels, omega=args.omega2d, nu1=nu, nu2=nu, nu3=3)
        nl = nswe.nswe_mg_smooth(ctx, pb, 0, 9, J9cm, R, dU, q, colour_major=True)
        sweeps[nu] = (timed(lambda: nswe.nswe_mg_smooth(ctx, pb, 0, 9, J9cm, R, dU, q, colour_major=True), 3), nl)
    pass_ms = (sweeps[30][0] - sweeps[10][0]) / (sweeps[30][1] - sweeps[10][1])
    # Per cell of the pass (n/3 cells): 8 off-diagonal 3x3 blocks times the neighbours' dU (8 x 9 FMA),
    # D^-1 times the sum (9 FMA), the relaxation of 3 components (2 flops each): 168 flops. Bytes: J9 648 B,
    # D^-1 72 B, R 24 B, own dU read and written 48 B per cell, the other colours' dU (2n/3 x 24 B) once.
    pass_flops = n / 3.0 * (8 * 18 + 18 + 6)
    pass_bytes = n / 3.0 * (648 + 72 + 24 + 48) + 2.0 * n / 3.0 * 24
    pk = measure_fma_peaks(0)
    hbm, hbm_src = hbm_peak_gbs()
    achieved = pass_flops / (pass_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["fp64_tflops"], "traffic": SOR_PASS_TRAFFIC_512,
            "peak_note": "FP64 FMA peak measured in this run (nswe_probe_fma)",
            "kernel": "k2_sor_split<double, J9>: one colour pass of the 512x256 level, colour-major J9",
            "flops_per_launch": pass_flops, "bytes_per_launch": pass_bytes, "launch_us": 1000.0 * pass_ms,
            "hbm": {"achieved_gbs": pass_bytes / (pass_ms / 1000.0) / 1e9, "peak_gbs": hbm, "peak_note": hbm_src},
            "what": "algorithmic flops (and bytes) per pass / per-pass time from nswe_mg_smooth with nu = 30 minus "
                    "nu = 10 (%d vs %d colour passes); ncu: FP64 pipe 73 %% busy, DRAM 26 %% of peak, so the pass "
                    "is bound by FP64 issue" % (sweeps[30][1], sweeps[10][1])}
    kern = {"residual_ms": timed(lambda: nswe.nswe_residual(ctx, pb, 0, U, R, res), 10),
            "jacobian_j9_ms": timed(lambda: nswe.nswe_jacobian_simplified(ctx, pb, 0, U, 1e-6, 3.0, R, J9, res), 3),
            "jacobian_j21_ms": timed(lambda: nswe.nswe_jacobian_full(ctx, pb, 0, U, 1e-6, 3.0, R, J21, res), 2),
            "jacobian_j9_frozen_ms": timed(lambda: nswe.nswe_jacobian_frozen(ctx, pb, 0, 9, U, 1e-6, 3.0, R, J9, res),
                                           3),
            "vcycle_j9_nu20_ms": timed(lambda: nswe.nswe_mg_vcycle(ctx, pb, 0, 9, J9, R, dU, prm), 2),
            "grid": "512x256, 7 levels"}
    # mixed precision: FP64-evaluated J9 stored in FP32, FP32 V-cycle
    J32 = torch.zeros((9, 9, n), dtype=torch.float32, device="cuda")
    R32, dU32 = torch.zeros((3, n), dtype=torch.float32, device="cuda"), torch.zeros((3, n), dtype=torch.float32,
                                                                                        device="cuda")
    kern["jacobian_j9_f32_ms"] = timed(lambda: nswe.nswe_jacobian_f32(ctx, pb, 0, 9, U, 1e-6, 3.0, R, J32, res), 3)
    R32.copy_(R.float())
    kern["vcycle_j9_nu20_f32_ms"] = timed(lambda: nswe.nswe_mg_vcycle_f32(ctx, pb, 0, 9, J32, R32, dU32, prm), 2)
    kern["sor_pass_colour_major_us"] = 1000.0 * pass_ms
    if args.phases_only:
        print(json.dumps({"metric": "2D phase times at 512x256 (ms)", "kernels_512x256": kern, "roofline": roof}),
              flush=True)
        return
    # nested from the 16 x 8 grid as in Section 5.2.2 (the V-cycles reach 8 x 4)
    frozen = args.jacobian2d == "frozen"
    w = I.wedge(args.nx, args.ny, args.levels2d, x1=40.0, y1=30.0, x_wall=8.0, theta_deg=big.meta["theta_deg"],
                start_level=args.levels2d - 2)
    pw = nswe.Problem2D.from_inputs(ctx, w)
    p2 = nswe.params2d_from(I.Params2D(levels=args.levels2d, nu1=[20], nu2=[20], omega=args.omega2d, tol=TOL,
                                       n_max=3000, nest_start=args.levels2d - 2, frozen=frozen))
    mixed = args.precision == "mixed"
    p2.precision = nswe.PREC_MIXED if mixed else nswe.PREC_FP64
    U0 = torch.from_numpy(w.U0_start).cuda()
    Uo = torch.zeros((3, args.nx * args.ny), dtype=torch.float64, device="cuda")
    times, info = [], None
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = nswe.nswe_newton_solve(ctx, pw, U0, Uo, p2)
        torch.cuda.synchronize()
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * statistics.mean(times)
    cpu = None if args.no_cpu else wedge2d_oracle_estimate(w, args, info["iters"], frozen)
    line = {
        "metric": METRIC, "value": 1000.0 / ms, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"2D wedge channel {args.nx}x{args.ny} on [0,40]x[0,30], J9"
                               + (" (frozen linearisation)" if frozen else "") + f", {args.levels2d} levels, "
                               f"nested from 16x8, omega {args.omega2d}, nu 20, nu3 3, eps 1e-6, "
                               + ("mixed FP64/FP32" if mixed else "FP64"),
                   "theta_deg": big.meta["theta_deg"], "launch_overlap": not args.no_launch_overlap},
        "converged": {"status": info["status"], "iters": info["iters"][:args.levels2d], "res": info["res"][0]},
        "kernels_512x256": kern, "roofline": roof}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def _wedge2d_step_worker(args):
    """One oracle Newton step (Eq. 12-14 with the V-cycles of Algorithm 2) of
    the wedge at nx x ny from its inflow guess; returns seconds."""
    nx, ny, lev, theta, omega, frozen = args
    import oracle
    from paper_2505_10857_gb300 import inputs as I
    w = I.wedge(nx, ny, lev, x1=40.0, y1=30.0, x_wall=8.0, theta_deg=theta, start_level=0)
    prm = I.Params2D(levels=lev, nu1=[20], nu2=[20], omega=omega, tol=1e-30, n_max=1, nest_start=0, frozen=frozen)
    t0 = time.perf_counter()
    oracle.newton2d(oracle.problem_levels2d(w)[0], w.U0_start, lev, prm)
    return time.perf_counter() - t0


def wedge2d_oracle_estimate(w, args, iters, frozen):
    """The oracle's time for the nested wedge solve, estimated: one Newton
    step timed per nested level up to 256 x 128 cells (a process each, run
    side by side), finer levels extrapolated in proportion to their cells
    from the 256 x 128 step, times the GPU solve's Newton steps per level.
    The oracle is single-threaded; one solve uses one core."""
    import oracle
    oracle.build()
    s0 = args.levels2d - 2
    levels = [l for l in range(s0, -1, -1)]
    jobs, timed_l = [], []
    for l in levels:
        nx, ny = args.nx >> l, args.ny >> l
        if nx * ny <= 256 * 128:
            jobs.append((nx, ny, args.levels2d - l, w.meta["theta_deg"], args.omega2d, frozen))
            timed_l.append(l)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        secs = pool.map(_wedge2d_step_worker, jobs)
    t = dict(zip(timed_l, secs))
    lmin = min(timed_l)
    ref_cells = (args.nx >> lmin) * (args.ny >> lmin)
    for l in levels:
        if l not in t:
            t[l] = t[lmin] * (args.nx >> l) * (args.ny >> l) / ref_cells
    total = sum(iters[l] * t[l] for l in levels)
    return {"value": 1.0 / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one Newton step per nested level up to 256x128 timed (one process each), the finer levels "
                      "extrapolated in proportion to cells from the 256x128 step, times the GPU solve's Newton "
                      "steps per level; one solve is single-threaded",
            "step_s_per_level": {f"{args.nx >> l}x{args.ny >> l}": t[l] for l in levels},
            "extrapolated_levels": [f"{args.nx >> l}x{args.ny >> l}" for l in levels if l not in timed_l],
            "estimated_solve_s": total, **oracle_build_info()}


def _serve_oracle_worker(args):
    """Oracle solves of serving request k: at the line's stopping residual
    (timed, the CPU baseline) and converged (the parity reference)."""
    k, tol = args
    import oracle
    from paper_2505_10857_gb300 import inputs as I
    inp = I.serving_instance(k)
    t0 = time.perf_counter()
    U, info = oracle.solve_problem(inp, I.Params1D.for_problem(inp, tol=tol, n_max=800))
    dt = time.perf_counter() - t0
    Uc, ic = oracle.solve_problem(inp, I.Params1D.for_problem(inp, tol=TOL_CONVERGED, n_max=800))
    return U, info["status"], dt, Uc, ic["status"]


def serving_requests(M, tol, mixed):
    """The serving workload: M seeded 1D requests (N log-uniform in [256,
    16384], q ~ U[1, 6]) and their parameters."""
    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe
    inps = [I.serving_instance(k) for k in range(M)]
    prms = []
    for p in inps:
        q = nswe.params_from(I.Params1D.for_problem(p, tol=tol, n_max=800))
        q.precision = nswe.PREC_MIXED if mixed else nswe.PREC_FP64
        prms.append(q)
    return inps, prms


def serve1d_measure(inps, prms, rate, streams, max_batch, mem_gb, warm, seed=4999, cluster=None):
    """One pass of the requests through a fresh continuous-batching server:
    `warm` requests first (discarded), then all of them arriving as a seeded
    Poisson process at `rate` per second (rate = inf: all at once). cluster:
    None, or (ctas, max_in_flight) for the server's light-load cluster form.
    Returns the results per request, the per-request host timestamps and the
    server's launch count."""
    import numpy as np
    from paper_2505_10857_gb300 import nswe
    M = len(inps)
    sv = nswe.Server(0, device_bytes=mem_gb << 30, host_bytes=1 << 30, streams=streams, max_batch=max_batch)
    if cluster:
        sv.set_cluster(cluster[0], cluster[1], CLUSTER_TEAM_CELLS)
    results = {}

    def drain(block_until=None):
        while True:
            for t in sv.poll():
                results[t] = sv.take(t)
            if block_until is None or len(results) >= block_until:
                return
            sv.wait(1, 1.0)

    warm = min(M, warm)
    for k in range(warm):
        sv.submit(inps[k], prms[k])
    drain(warm)
    results.clear()
    st0 = sv.stats()
    if math.isinf(rate):
        arrive = np.zeros(M)
    else:
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(1.0 / rate, size=M)
        arrive = np.cumsum(gaps) - gaps[0]
    tickets = []
    t0 = time.perf_counter()
    for k in range(M):
        while True:
            dt = t0 + arrive[k] - time.perf_counter()
            if dt <= 0:
                break
            if dt > 0.002:
                for t in sv.poll():
                    results[t] = sv.take(t)
            time.sleep(min(dt, 0.001))
        tickets.append(sv.submit(inps[k], prms[k]))
    drain(M)
    st1 = sv.stats()
    sv.close()
    tim = [results[t][2] for t in tickets]
    out = {"U": [results[t][0] for t in tickets], "info": [results[t][1] for t in tickets],
           "lat_ms": sorted((x["t_done_ns"] - x["t_submit_ns"]) / 1e6 for x in tim),
           "queue_ms": sorted((x["t_launch_ns"] - x["t_submit_ns"]) / 1e6 for x in tim),
           "span_s": (max(x["t_done_ns"] for x in tim) - min(x["t_submit_ns"] for x in tim)) / 1e9,
           "launches": st1["launches"] - st0["launches"], "device_bytes_peak": st1["device_bytes_peak"]}
    out["ok"] = [k for k in range(M) if out["info"][k]["status"] == 0]
    out["value"] = len(out["ok"]) / out["span_s"]  # solves that reached res < tol
    return out


def pct(a, q):
    return a[min(len(a) - 1, int(math.ceil(q / 100.0 * len(a))) - 1)]


def serving_oracle(n, tol):
    """The oracle on the host cores for the first n serving requests: timing
    at the line's stopping residual, and the converged references."""
    cores = host_cores()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_serve_oracle_worker, [(0, tol)] * cores)  # warm the workers
        t0 = time.perf_counter()
        refs = pool.map(_serve_oracle_worker, [(k, tol) for k in range(n)])
        wall = time.perf_counter() - t0
    cpu_seconds = sum(r[2] for r in refs)
    return refs, {"value": n / cpu_seconds * cores, "unit": UNIT, "cores": cores, "kind": "oracle",
                  "sample": f"the first {n} requests, one solve per process (spawn pool): their summed one-core "
                            f"solve times at res < {tol:g}, scaled to {cores} cores ({cpu_seconds:.1f} core-s)",
                  "latency_1core_ms_mean": 1000.0 * cpu_seconds / n, **oracle_build_info()}


def _parity(Us, infos, refs, idx):
    import numpy as np
    errs = [float(np.abs(Us[k] - refs[k][3]).max() / np.abs(refs[k][3]).max())
            for k in idx if infos[k]["status"] == 0 and refs[k][4] == 0]
    return {"max_rel_err_vs_oracle": max(errs) if errs else None, "instances": len(errs),
            "reference": f"the oracle's converged discrete solution (res < {TOL_CONVERGED:g})", "bound": MIXED_BOUND}


def run_latency1d(args):
    """Single-solve latency of the 1D channel workload (N = 4096, 8 levels, J3)
    in the block form and in the cluster form over cluster sizes and the
    smallest multigrid level run on every CTA (team_cells): each of the first
    three instances solved alone, the median of the three (CUDA events). FP64
    at res < TOL and mixed precision at res < TOL_SOLUTION. Prints one JSON
    line."""
    import statistics

    import torch

    from paper_2505_10857_gb300 import nswe
    inps, _ = make_instances(0, 3, 3)
    ctx = nswe.Context(0)
    probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps]
    U0s = [torch.from_numpy(p.U0_start).cuda() for p in inps]
    Us = [torch.zeros(2, p.N, dtype=torch.float64, device="cuda") for p in inps]
    stream = torch.cuda.current_stream()
    rows = []
    for prec, tol in ((nswe.PREC_FP64, TOL), (nswe.PREC_MIXED, TOL_SOLUTION)):
        from paper_2505_10857_gb300 import inputs as I
        prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=tol, n_max=800))
        prm.precision = prec
        nswe.nswe_ctx_set_solve_shape(ctx, prec, 3)  # 128 x 4: no spills, the best single-block shape
        configs = [(1, CLUSTER_TEAM_CELLS)] + [(c, t) for c in (2, 4, 8, 16)
                                               for t in (256, 512, 1024, 2048, 4096, 1 << 30)]
        for ctas, cells in configs:
            nswe.nswe_ctx_set_solve_cluster(ctx, ctas, cells)
            ms, its = [], []
            for k in range(3):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = nswe.nswe_newton_solve(ctx, probs[k], U0s[k], Us[k], prm)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                its.append(info["total_iters"])
            rows.append({"precision": "mixed" if prec == nswe.PREC_MIXED else "fp64", "ctas": ctas,
                         "team_cells": cells, "ms_median": statistics.median(ms), "newton_steps": its})
        nswe.nswe_ctx_set_solve_cluster(ctx, 1, CLUSTER_TEAM_CELLS)
    print(json.dumps({"metric": "single-solve latency (ms), 1D irregular channel N=4096, 8-level MG, J3",
                      "config": {"workload": "1D irregular channel, N=4096, 8-level MG, J3, seeds 2000-2002",
                                 "what": "each instance alone, CUDA events, median of three; ctas 1: one block "
                                         "of 128 threads"},
                      "rows": rows}), flush=True)


def serving_comparison(args, ctx):
    """The metric's comparison, measured beside the default line: the batched
    mixed-precision serving form (the 1D serving workload through the
    continuous-batching server) against the plain FP64 path solving one
    instance at a time, both stopped at res < TOL_SOLUTION so that both land
    within MIXED_BOUND of the converged FP64 discrete solution (checked on a
    sample against the oracle)."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import nswe
    M = args.requests
    inps, prm_mixed = serving_requests(M, TOL_SOLUTION, True)
    _, prm_fp64 = serving_requests(M, TOL_SOLUTION, False)
    cfg = {"workload": f"1D serving: {M} requests, N log-uniform [256,16384] (mean "
                       f"{np.mean([p.N for p in inps]):.0f} cells), q~U[1,6], sinusoidal width, Gaussian hump",
           "tol": TOL_SOLUTION, "accuracy": f"res < {TOL_SOLUTION:g}: within {MIXED_BOUND:g} (relative) of the "
                                            f"converged FP64 discrete solution", "seeds": "numpy default_rng(4000 + k)"}
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    sat = serve1d_measure(inps, prm_mixed, math.inf, args.streams, args.max_batch, args.serve_mem_gb, 64)
    paced = serve1d_measure(inps, prm_mixed, args.rate, args.streams, args.max_batch, args.serve_mem_gb, 64)
    sat64 = serve1d_measure(inps, prm_fp64, math.inf, args.streams, args.max_batch, args.serve_mem_gb, 64)
    # light load, where a request's latency is its own solve time: block form against the cluster form
    nl = min(M, LIGHT_REQUESTS)
    light = {}
    for form, cl in (("block_form", None), ("cluster_form", (LIGHT_CTAS, LIGHT_MAX_IN_FLIGHT))):
        r = serve1d_measure(inps[:nl], prm_mixed[:nl], LIGHT_RATE, args.streams, args.max_batch, args.serve_mem_gb, 8,
                            cluster=cl)
        light[form] = {"p50": pct(r["lat_ms"], 50), "p99": pct(r["lat_ms"], 99), "max": r["lat_ms"][-1],
                       "converged": len(r["ok"]), "of": nl}
    light["cluster_form"].update({"ctas": LIGHT_CTAS, "max_in_flight": LIGHT_MAX_IN_FLIGHT})
    light.update({"offered_rate": LIGHT_RATE, "requests": nl,
                  "what": "completion minus submission per request (host clock), seeded Poisson arrivals, mixed "
                          "precision; the cluster form runs a launch's problems on thread-block clusters while "
                          "at most max_in_flight 1D solves are in flight"})
    # the plain FP64 single-instance path: one request at a time, one solve per launch
    K = args.single_requests
    stream = torch.cuda.current_stream()
    t_single, U_single, inf_single = [], [], []
    for k in range(K):
        pr = nswe.Problem1D.from_inputs(ctx, inps[k])
        U0 = torch.from_numpy(inps[k].U0_start).cuda()
        U = torch.zeros((2, inps[k].N), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = nswe.nswe_newton_solve(ctx, pr, U0, U, prm_fp64[k])
        e1.record(stream)
        torch.cuda.synchronize()
        t_single.append(e0.elapsed_time(e1))
        U_single.append(U.cpu().numpy())
        inf_single.append(info)
        del pr
    clk = clocks.stop()
    ok_single = [k for k in range(K) if inf_single[k]["status"] == 0]
    single_value = len(ok_single) / (sum(t_single) / 1000.0)
    out = {
        "serving": {"value": sat["value"], "unit": UNIT, "precision": "mixed FP64 residual/update + FP32 "
                    "Jacobian/MG", "form": "continuous-batching server, all requests submitted at once",
                    "config": dict(cfg, streams=args.streams, max_batch=args.max_batch),
                    "converged": len(sat["ok"]), "of": M,
                    "not_converged_seeds": [4000 + k for k in range(M) if sat["info"][k]["status"] != 0],
                    "max_res": max(sat["info"][k]["res"][0] for k in sat["ok"]),
                    "gpu_launches": sat["launches"], "span_s": sat["span_s"],
                    "latency_ms_at_offered_rate": {"offered_rate": args.rate, "p50": pct(paced["lat_ms"], 50),
                                                   "p99": pct(paced["lat_ms"], 99), "max": paced["lat_ms"][-1],
                                                   "completed_per_s_over_run": paced["value"],
                                                   "what": "completion minus submission per request (host clock), "
                                                           "seeded Poisson arrivals"},
                    "latency_ms_light_load": light},
        "serving_fp64": {"value": sat64["value"], "unit": UNIT, "precision": "FP64",
                         "form": "the same server and requests in FP64", "converged": len(sat64["ok"]), "of": M},
        "plain_fp64_single": {"value": single_value, "unit": UNIT, "precision": "FP64",
                              "form": "one request at a time through nswe_newton_solve (one solve per launch), "
                                      "device-timed",
                              "sample": f"the first {K} requests of the serving workload",
                              "converged": len(ok_single), "of": K,
                              "latency_ms_p50": pct(sorted(t_single), 50)},
        "serving_over_plain_fp64_single": sat["value"] / single_value,
        "serving_clocks": clk,
    }
    if not args.no_cpu:
        n = min(K, 2 * host_cores())
        refs, cpu = serving_oracle(n, TOL_SOLUTION)
        out["serving"]["parity"] = _parity(sat["U"], sat["info"], refs, range(n))
        out["serving"]["cpu_baseline"] = cpu
        out["plain_fp64_single"]["parity"] = _parity(U_single, inf_single, refs, range(min(n, K)))
    return out


def run_serve1d(args):
    """Serving measurement (not the default line): `--requests` seeded 1D
    requests (N log-uniform in [256, 16384], q ~ U[1, 6]) arriving as a
    seeded Poisson process at `--rate` per second into the continuous-batching
    server, mixed precision by default, stopped at res < TOL_SOLUTION (or
    --tol). Throughput counts the solves that reached res < tol over the span
    from the first submission to the last completion; latency is completion
    minus submission, host clock, per request."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import nswe

    mixed = args.precision != "fp64"
    tol = args.tol if args.tol is not None else TOL_SOLUTION
    M = args.requests
    inps, prms = serving_requests(M, tol, mixed)
    foot = [nswe.Server.footprint(p.N, p.levels, p.start_level) for p in inps]
    torch.cuda.init()
    clocks = ClockSampler(0)
    clocks.start()
    cluster = (args.cluster_ctas, LIGHT_MAX_IN_FLIGHT) if args.cluster_ctas > 1 else None
    r = serve1d_measure(inps, prms, args.rate, args.streams, args.max_batch, args.serve_mem_gb,
                        64 * max(1, args.warmup), cluster=cluster)
    clk = clocks.stop()
    lat, queue, ok, infos = r["lat_ms"], r["queue_ms"], r["ok"], r["info"]
    line_parity, cpu = None, None
    if not args.no_cpu:
        n = min(M, 2 * host_cores())
        refs, cpu = serving_oracle(n, tol)
        line_parity = _parity(r["U"], infos, refs, range(n))
    h2d = sum(p.sig_face.nbytes + p.gq_all().nbytes + p.U0_start.nbytes for p in inps) / M
    d2h = sum(2 * p.N * 8 for p in inps) / M + ctypes.sizeof(nswe.Info)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1000.0 * r["span_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"1D serving: {M} requests, N log-uniform [256,16384] (mean {np.mean([p.N for p in inps]):.0f}"
                               f" cells), q~U[1,6], Poisson arrivals at {args.rate}/s, "
                               + ("mixed FP64/FP32" if mixed else "FP64"),
                   "offered_rate": args.rate, "streams": args.streams, "max_batch": args.max_batch, "tol": tol,
                   "device_arena_gb": args.serve_mem_gb, "seeds": "numpy default_rng(4000 + k); arrivals 4999",
                   "cluster_form": ({"ctas": args.cluster_ctas, "max_in_flight": LIGHT_MAX_IN_FLIGHT}
                                    if cluster else None),
                   "l2": "resident workspace of the requests in flight exceeds the 129 MB L2"},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": lat[-1],
                       "what": "completion minus submission per request (host clock)",
                       "queue_p50": pct(queue, 50), "queue_p99": pct(queue, 99)},
        "converged": {"all_status_ok": len(ok) == M, "converged": len(ok), "of": M,
                      "not_converged_seeds": [4000 + k for k in range(M) if infos[k]["status"] != 0],
                      "max_res": max(infos[k]["res"][0] for k in ok),
                      "mean_newton_iters": statistics.mean(infos[k]["total_iters"] for k in ok)},
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": h2d * M, "d2h_bytes_per_step": d2h * M,
                "what": "the serving throughput is end to end: host arrays in, host results out"},
        "gpu_launches": r["launches"],
        "serving": {"device_bytes_peak": r["device_bytes_peak"], "mean_footprint_mb": float(np.mean(foot)) / 2**20,
                    "launches": r["launches"]},
        "clocks": clk,
    }
    if line_parity:
        line["parity"] = line_parity
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


CONFIG5_SIZES = [(128, 64, 5), (256, 128, 6), (512, 256, 7), (1024, 512, 8)]


def config5_instances(B):
    """The batched 2D serving workload at its stated sizes: B seeded channels,
    grids 128 x 64 to 1024 x 512 (the four sizes in equal numbers, in the
    order k mod 4), even k supercritical wedges (Froude 2-4, deflection 5-15
    degrees, frozen linearisation, nested from 16 x 8), odd k subcritical
    channels over a Gaussian bottom bump (Eq. 12, nested from 8 x 4); J9,
    omega 0.1, nu1 = nu2 = 20, nu3 = 3, eps 1e-6."""
    from paper_2505_10857_gb300 import inputs as I
    inps, prms = [], []
    for k in range(B):
        Nx, Ny, lev = CONFIG5_SIZES[(k // 2) % 4]
        if k % 2 == 0:
            inps.append(I.wedge_serving_2d(k, Nx, Ny, lev))
            prms.append(I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=TOL, n_max=400, nest_start=lev - 2,
                                   omega=0.1, frozen=True))
        else:
            inps.append(I.gauss_bump_channel_2d(k, Nx, Ny, lev))
            prms.append(I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=TOL, n_max=400))
    return inps, prms


def batch2d_instances(B, family):
    """The batched 2D workload: instance k is a wedge (even k, or all with
    family "wedge") or a bump channel (odd k, or all with family "bump"), on
    128 x 64 (5 levels) or 256 x 128 (6 levels) alternating in pairs. Wedges:
    `wedge_serving_2d` under the frozen linearisation, omega 0.1, nested from
    16 x 8; bumps: `bump_channel_2d` with Eq. 12, nested from 8 x 4 (Eq. 30);
    both J9, nu1 = nu2 = 20, nu3 = 3, eps 1e-6."""
    from paper_2505_10857_gb300 import inputs as I
    inps, prms = [], []
    for k in range(B):
        fam = family if family != "mix" else ("wedge" if k % 2 == 0 else "bump")
        Nx, Ny, lev = (256, 128, 6) if (k // 2) % 2 == 1 else (128, 64, 5)
        if fam == "wedge":
            inps.append(I.wedge_serving_2d(k, Nx, Ny, lev))
            prms.append(I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=TOL, n_max=400, nest_start=lev - 2,
                                   omega=0.1, frozen=True))
        else:
            inps.append(I.bump_channel_2d(k, Nx, Ny, lev))
            prms.append(I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=TOL, n_max=400))
    return inps, prms


def run_batch2d(args):
    """Batched 2D measurement (not the default line), shaped like the batched
    2D serving configuration: `--batch2d` seeded supercritical wedge channels
    (Froude 2-4, deflection 5-15 degrees) and subcritical parabolic-bump
    channels (around Section 5.2.1) on 128 x 64 and 256 x 128 grids, each with
    its own parameters, solved by one batched call whose solves run
    concurrently, against the same solves one after another. Host-timed (the
    solves run on several streams); the value counts the solves that reached
    res < tol; latencies are per solve from the start of the batch."""
    import torch

    from paper_2505_10857_gb300 import nswe

    mixed = args.precision != "fp64"
    B = args.batch2d
    inps, prms_in = config5_instances(B) if args.sizes2d == "config5" else batch2d_instances(B, args.family2d)
    ctx = nswe.Context(0)
    lockstep = args.batch2d_mode == "lockstep"
    nswe.nswe_ctx_set_batch_2d(ctx, nswe.BATCH2D_LOCKSTEP if lockstep else nswe.BATCH2D_CONCURRENT)
    probs = [nswe.Problem2D.from_inputs(ctx, p) for p in inps]
    U0s = [torch.from_numpy(p.U0_start).cuda() for p in inps]
    Us = [torch.zeros((3, p.Nx * p.Ny), dtype=torch.float64, device="cuda") for p in inps]
    prms = []
    for q in prms_in:
        c = nswe.params2d_from(q)
        c.precision = nswe.PREC_MIXED if mixed else nswe.PREC_FP64
        prms.append(c)

    def batched():
        return nswe.nswe_newton_solve_batch_each(ctx, probs, U0s, Us, prms)

    def one_by_one():
        return [nswe.nswe_newton_solve(ctx, probs[k], U0s[k], Us[k], prms[k]) for k in range(B)]

    for _ in range(args.warmup):  # --warmup 0 for the multi-minute serving sizes: one timed batch includes capture
        batched()
    times = []
    infos = None
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = batched()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    seq, t_seq = None, None
    if not args.no_one_by_one:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq = one_by_one()
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
    ms = 1000.0 * statistics.mean(times)
    ok = [k for k in range(B) if infos[k]["status"] == 0]
    # per-solve latency from the batch start, from the device timestamps of each solve
    t0s = min(i["t_start_ns"] for i in infos)
    lat = sorted((i["t_end_ns"] - t0s) / 1e6 for i in infos)
    pick = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
    kinds = {}
    for k, p in enumerate(inps):
        key = f"{'wedge' if 'froude' in p.meta else p.meta.get('case', 'bump')} {p.Nx}x{p.Ny}"
        kinds.setdefault(key, [0, 0])
        kinds[key][0] += 1
        kinds[key][1] += int(infos[k]["status"] == 0)
    print(json.dumps({
        "metric": METRIC, "value": len(ok) / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": (f"2D batched serving sizes: {B} seeded channels (wedges Froude 2-4, 5-15 deg, "
                                "frozen linearisation; Gaussian-bump channels, Eq. 12), 128x64, 256x128, 512x256 "
                                "and 1024x512 in equal numbers, J9, nu 20, "
                                if args.sizes2d == "config5" else
                                f"2D batched: {B} seeded channels ({args.family2d}: wedges Froude 2-4, 5-15 deg, "
                                "frozen linearisation; parabolic bumps, Eq. 12), 128x64 and 256x128, J9, nu 20, ")
                               + ("mixed FP64/FP32" if mixed else "FP64"),
                   "batch_mode": args.batch2d_mode, "launch_overlap": not args.no_launch_overlap,
                   "seeds": "wedges default_rng(7000 + k), bumps default_rng(%d + k)"
                            % (6000 if args.sizes2d == "config5" else 5000)},
        "latency_ms": {"p50": pick(0.5), "p99": pick(0.99), "what": "per-solve completion from the batch start"},
        "converged": {"all_status_ok": len(ok) == B, "converged": len(ok), "of": B,
                      "by_kind": {k: {"n": v[0], "converged": v[1]} for k, v in kinds.items()},
                      "failed": [(inps[k].meta.get("seed"), infos[k]["status"], infos[k]["iters"][:inps[k].levels])
                                 for k in range(B) if infos[k]["status"] != 0][:8],
                      "max_res": max((infos[k]["res"][0] for k in ok), default=None),
                      "one_by_one_equal_iters": (all(seq[k]["iters"] == infos[k]["iters"] for k in range(B))
                                                 if seq else None)},
        "one_by_one": ({"solves_per_s": sum(1 for i in seq if i["status"] == 0) / t_seq, "ms": 1000.0 * t_seq}
                       if seq else None),
        "what": "host-timed: " + ("one launch per phase and colour pass over all problems (lockstep)" if lockstep
                                  else "the batched call runs the solves concurrently on worker streams")}),
          flush=True)


def run_serve2d(args):
    """2D serving measurement (not the default line): the `--batch2d` seeded
    channels of the batched 2D workload (`batch2d_instances`) arriving as a
    seeded Poisson process at `--rate2d` per second into the server's 2D
    worker pool (`--streams` workers, a 2D device budget of `--serve-mem-gb`
    GB). Throughput counts the solves that reached res < tol over the span
    from the first submission to the last completion; latency is completion
    minus submission per request (host clock)."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import nswe

    mixed = args.precision != "fp64"
    B = args.batch2d
    c5 = args.sizes2d == "config5"
    inps, prms_in = config5_instances(B) if c5 else batch2d_instances(B, args.family2d)
    prms = []
    for q in prms_in:
        c = nswe.params2d_from(q)
        c.precision = nswe.PREC_MIXED if mixed else nswe.PREC_FP64
        prms.append(c)
    torch.cuda.init()
    sv = nswe.Server(0, device_bytes=64 << 20, host_bytes=64 << 20, streams=args.streams, max_batch=4,
                     device_bytes_2d=args.serve_mem_gb << 30)
    results = {}

    def drain(block_until):
        while len(results) < block_until:
            for t in sv.poll():
                results[t] = sv.take(t)
            if len(results) < block_until:
                sv.wait(1, 1.0)

    warm = min(B, max(1, args.warmup))  # first requests once, discarded
    for k in range(warm):
        sv.submit2d(inps[k], prms[k])
    drain(warm)
    results.clear()
    clocks = ClockSampler(0)
    clocks.start()
    rng = np.random.default_rng(6999)
    gaps = rng.exponential(1.0 / args.rate2d, size=B)
    arrive = np.cumsum(gaps) - gaps[0]
    tickets = []
    t0 = time.perf_counter()
    for k in range(B):
        while True:
            dt = t0 + arrive[k] - time.perf_counter()
            if dt <= 0:
                break
            for t in sv.poll():
                results[t] = sv.take(t)
            time.sleep(min(dt, 0.005))
        tickets.append(sv.submit2d(inps[k], prms[k]))
    drain(B)
    clk = clocks.stop()
    st = sv.stats()
    sv.close()
    tim = [results[t][2] for t in tickets]
    infos = [results[t][1] for t in tickets]
    lat = sorted((x["t_done_ns"] - x["t_submit_ns"]) / 1e6 for x in tim)
    queue = sorted((x["t_launch_ns"] - x["t_submit_ns"]) / 1e6 for x in tim)
    span = (max(x["t_done_ns"] for x in tim) - min(x["t_submit_ns"] for x in tim)) / 1e9
    ok = [k for k in range(B) if infos[k]["status"] == 0]

    def pct(a, q):
        return a[min(len(a) - 1, int(math.ceil(q / 100.0 * len(a))) - 1)]

    print(json.dumps({
        "metric": METRIC, "value": len(ok) / span, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1000.0 * span, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": (f"2D serving: {B} requests (wedges Froude 2-4, 5-15 deg, frozen linearisation; "
                                "Gaussian-bump channels, Eq. 12), 128x64, 256x128, 512x256 and 1024x512 in equal "
                                "numbers, J9, nu 20, " if c5 else
                                f"2D serving: {B} requests ({args.family2d}: wedges Froude 2-4, 5-15 deg, frozen "
                                "linearisation; parabolic bumps, Eq. 12), 128x64 and 256x128, J9, nu 20, ")
                               + f"Poisson arrivals at {args.rate2d}/s, " + ("mixed FP64/FP32" if mixed else "FP64"),
                   "offered_rate": args.rate2d, "workers": args.streams, "device_budget_2d_gb": args.serve_mem_gb,
                   "seeds": "wedges default_rng(7000 + k), bumps default_rng(%d + k); arrivals 6999"
                            % (6000 if c5 else 5000)},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "queue_p50": pct(queue, 50),
                       "queue_p99": pct(queue, 99), "what": "completion minus submission per request (host clock)"},
        "converged": {"converged": len(ok), "of": B, "max_res": max((infos[k]["res"][0] for k in ok), default=None)},
        "server": {"completed": st["completed"], "submitted": st["submitted"]},
        "clocks": clk}), flush=True)


def run_autotune2d(args):
    """The 2D autotuner's log (not the default line): for seeded wedge
    channels of 64 x 32 to 512 x 256 cells in FP64 and mixed precision, the
    time of one V-cycle (nu 20) for every smoothing schedule (0: the stencil
    colouring; K: the directional schedule) and tail threshold, and the
    choice nswe_autotune_2d records."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    ctx = nswe.Context(0)
    schedules, tails = [0, 3, 5, 7], [64, 256, 1024, 4096, 16384]
    rows = []
    for Nx, Ny, lev in ((64, 32, 4), (128, 64, 5), (256, 128, 6), (512, 256, 7)):
        inp = I.wedge_serving_2d(0, Nx, Ny, lev)
        prob = nswe.Problem2D.from_inputs(ctx, inp)
        X, _ = inp.centres(0)
        s0 = inp.bc_state[0]
        U = torch.tensor(np.stack([s0[0] * (1 + 0.02 * np.sin(X.ravel())), np.full(X.size, s0[1]),
                                   np.full(X.size, s0[2])]), dtype=torch.float64, device="cuda")
        for prec in ("fp64", "mixed"):
            q = nswe.params2d_from(I.Params2D(levels=lev, nu1=[20], nu2=[20], omega=0.1, frozen=True))
            q.precision = nswe.PREC_MIXED if prec == "mixed" else nswe.PREC_FP64
            ms, bs, bt = nswe.nswe_autotune_2d(ctx, prob, U, q, schedules, tails, reps=2)
            rows.append({"grid": f"{Nx}x{Ny}", "precision": prec, "ms_per_vcycle": ms, "chosen_schedule": bs,
                         "chosen_tail": bt, "default_ms": ms[0][tails.index(256 if prec == "fp64" else 4096)]})
        del prob
    print(json.dumps({"metric": "2D V-cycle time per schedule and tail threshold (ms), the autotuner's choices",
                      "schedules": schedules, "tails": tails, "rows": rows}), flush=True)


def run_jac1d(args):
    """1D Jacobian cost (not the default line): the residual and the FD
    Jacobians J3 and J5 (Eq. 12-13) of one seeded channel of 2^20 cells,
    CUDA events on the launching stream, FP64 and FP32 storage. Section 3.3
    expects J3 to cost about 40 % less than J5."""
    import numpy as np
    import torch

    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    N, levels = 1 << 20, 14  # coarsest level 128 cells
    inp = I.channel_small(0, N=N, levels=levels)
    ctx = nswe.Context(0)
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    xc = (np.arange(N) + 0.5) * 25.0 / N
    U = torch.tensor(np.stack([2.0 - 0.1 * np.exp(-((xc - 10.0) / 1.5) ** 2) + 1e-3 * rng.standard_normal(N),
                               np.full(N, 4.42)]), dtype=torch.float64, device="cuda")
    R, res = torch.zeros_like(U), torch.zeros(1, dtype=torch.float64, device="cuda")
    J5 = torch.zeros((5, 4, N), dtype=torch.float64, device="cuda")
    J5f = torch.zeros((5, 4, N), dtype=torch.float32, device="cuda")
    eps = 0.05

    def timed(f, reps=20):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            f()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t = {"residual_ms": timed(lambda: nswe.nswe_residual(ctx, prob, 0, U, R, res)),
         "jacobian_j3_ms": timed(lambda: nswe.nswe_jacobian_simplified(ctx, prob, 0, U, eps, 3.0, R, J5[:3], res)),
         "jacobian_j5_ms": timed(lambda: nswe.nswe_jacobian_full(ctx, prob, 0, U, eps, 3.0, R, J5, res)),
         "jacobian_j3_f32_ms": timed(lambda: nswe.nswe_jacobian_f32(ctx, prob, 0, 3, U, eps, 3.0, R, J5f[:3], res)),
         "jacobian_j5_f32_ms": timed(lambda: nswe.nswe_jacobian_f32(ctx, prob, 0, 5, U, eps, 3.0, R, J5f, res))}
    t["j3_saving_vs_j5"] = 1.0 - t["jacobian_j3_ms"] / t["jacobian_j5_ms"]
    # one V-cycle (Algorithm 2) on J3 of the same level, 14 levels down to 128 cells
    nswe.nswe_jacobian_simplified(ctx, prob, 0, U, eps, 3.0, R, J5[:3], res)
    dU = torch.zeros_like(U)
    prm = nswe.params(N, levels, omega=inp.omega, nu1=2, nu2=2, nu3=1)
    t["vcycle_j3_ms"] = timed(lambda: nswe.nswe_mg_vcycle(ctx, prob, 0, 3, J5[:3], R, dU, prm), 5)
    print(json.dumps({"metric": "1D residual, Jacobian and V-cycle times at 2^20 cells (ms)", "cells": N,
                      "phases": t}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--batch", type=int, default=608, help="instances per GPU per step")
    ap.add_argument("--config1d", choices=["irregular", "small"], default="irregular",
                    help="the 1D workload: the irregular channel N=4096 (default) or the smooth channel N=200")
    ap.add_argument("--nb", type=int, default=3, choices=[3, 5], help="3: simplified J3, 5: full J5")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape of k_solve")
    ap.add_argument("--shape", type=int, default=None, help="launch shape index of k_solve (no autotuning)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: every step in FP64; mixed: FP32 Jacobian and multigrid, FP64 residual and update")
    ap.add_argument("--workload", default="channel1d",
                    choices=["channel1d", "wedge2d", "serve1d", "batch2d", "serve2d", "jac1d", "peaks",
                             "autotune2d", "latency1d"])
    ap.add_argument("--batch2d", type=int, default=16, help="batch2d: 2D problems per batch")
    ap.add_argument("--batch2d-mode", choices=["lockstep", "concurrent"], default="lockstep",
                    help="batch2d: shared launches over all problems, or concurrent per-problem streams")
    ap.add_argument("--sizes2d", choices=["small", "config5"], default="small",
                    help="batch2d: 128x64/256x128, or the serving sizes 128x64 to 1024x512")
    ap.add_argument("--no-one-by-one", action="store_true", help="batch2d: skip the one-by-one comparison")
    ap.add_argument("--no-launch-overlap", action="store_true",
                    help="2D workloads: launch the 2D kernels without programmatic dependent launch")
    ap.add_argument("--rate2d", type=float, default=1.0, help="serve2d: Poisson arrival rate (requests/s)")
    ap.add_argument("--family2d", choices=["mix", "wedge", "bump"], default="mix",
                    help="batch2d: wedge and bump channels, or one family")
    ap.add_argument("--requests", type=int, default=1024, help="serve1d: requests in the arrival schedule")
    ap.add_argument("--rate", type=float, default=1500.0, help="serve1d: Poisson arrival rate (requests/s)")
    ap.add_argument("--streams", type=int, default=8, help="serve1d: concurrent launches")
    ap.add_argument("--max-batch", type=int, default=512, help="serve1d: solves per launch")
    ap.add_argument("--serve-mem-gb", type=int, default=16, help="serve1d: device arena (GB)")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=64)
    ap.add_argument("--levels2d", type=int, default=5)
    ap.add_argument("--jacobian2d", choices=["frozen", "eq12"], default="frozen",
                    help="wedge2d: the 2D Jacobian of the nested solve (Eq. 12 as printed, or frozen weights)")
    ap.add_argument("--omega2d", type=float, default=0.1)
    ap.add_argument("--phases-only", action="store_true", help="wedge2d: only the 512x256 phase times")
    ap.add_argument("--tol", type=float, default=None,
                    help="stopping residual (default: 1e-10 for the FP64 line, 3e-13 for mixed and serving lines)")
    ap.add_argument("--cluster-ctas", type=int, default=1,
                    help="serve1d: the server's light-load cluster form with that many CTAs per request (1: off)")
    ap.add_argument("--sequential-steps", action="store_true",
                    help="time the 1D steps one at a time on one stream only (no steady two-stream form)")
    ap.add_argument("--no-serving", action="store_true",
                    help="default line: skip the serving / plain FP64 single-instance comparison")
    ap.add_argument("--single-requests", type=int, default=24,
                    help="default line: requests solved one at a time for the plain FP64 single-instance rate")
    args = ap.parse_args()
    if args.no_launch_overlap:
        from paper_2505_10857_gb300 import build
        build.build()
        from paper_2505_10857_gb300 import nswe
        nswe.nswe_set_launch_overlap_2d(0)
    if args.config1d == "small" and "--batch" not in sys.argv:
        args.batch = 256  # the 256 seeded instances of the N = 200 configuration
    if args.workload == "wedge2d":
        from paper_2505_10857_gb300 import build
        build.build()
        run_wedge2d(args)
        return
    if args.workload == "batch2d":
        from paper_2505_10857_gb300 import build
        build.build()
        run_batch2d(args)
        return
    if args.workload == "peaks":
        from paper_2505_10857_gb300 import build
        build.build()
        pk = measure_fma_peaks(0, reps=5)
        pk.update({"derived_fp64_tflops": FP64_PEAK_GFLOPS / 1e3, "derived_fp32_tflops": FP32_PEAK_GFLOPS / 1e3})
        print(json.dumps({"metric": "FP64 and FP32 FMA throughput (TFLOP/s)", "peaks": pk}), flush=True)
        return
    if args.workload == "autotune2d":
        from paper_2505_10857_gb300 import build
        build.build()
        run_autotune2d(args)
        return
    if args.workload == "jac1d":
        from paper_2505_10857_gb300 import build
        build.build()
        run_jac1d(args)
        return
    if args.workload == "latency1d":
        from paper_2505_10857_gb300 import build
        build.build()
        run_latency1d(args)
        return
    if args.workload == "serve2d":
        from paper_2505_10857_gb300 import build
        build.build()
        if args.precision == "fp64" and "--precision" not in sys.argv:
            args.precision = "mixed"  # the batched 2D serving workload is specified in mixed precision
        run_serve2d(args)
        return
    if args.workload == "serve1d":
        from paper_2505_10857_gb300 import build
        build.build()
        if args.precision == "fp64" and "--precision" not in sys.argv:
            args.precision = "mixed"  # the serving workload is specified in mixed precision
        run_serve1d(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2505_10857_gb300 import build
    build.build()
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
