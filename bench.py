"""Benchmark: seconds per spectral projector (hQDWH in HODLR format) on GB300.

Step = one full projector of the workload: HODLR ingest of the shifted band,
parameter estimation, the QR-based first QDWH step, the Cholesky-based steps,
P = (I - S)/2 and its trace (the whole hot path), through the library's C ABI.

Default workload: tridiagonal n = 100000, off-diagonal -1, diagonal i.i.d.
U[-0.5, 0.5], nu = n/2 (mu between lambda_nu and lambda_nu+1), leaf 256,
tol 1e-10, binary64.  `--workload band4`: b = 4 with N(0,1) entries.

Multi-GPU: one process per GPU (torchrun).  A single projector does not
shard, so every rank computes an independent replica (its own seed) and the
job's value is the max step time over ranks divided by the number of ranks.
`--workload batched` partitions the instances across ranks (longest first,
greedy by estimated cost), with no collective on the data path; the value is
all instances over the max wall time over ranks.

--impl reference: the CPU oracle (dense eigensolver projector) timed on the
host on a bounded sample of the same workload, scaled to the metric's unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sp_inputs  # noqa: E402

METRIC = "s/projector at n=1e5 & batched projectors/s; mixed vs FP64 GPU at ‖ΔΠ‖≤1e-8"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 binary64 rate (1.203 measured by a DFMA loop on this machine)


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="tridiag", choices=["tridiag", "band4", "band16", "batched"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed-ns"])
    p.add_argument("--polish", type=int, default=1)
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--nstreams", type=int, default=16)
    p.add_argument("--n", type=int, default=None,
                   help="order of the band (default: 32768 for band16, 100000 otherwise)")
    p.add_argument("--leaf", type=int, default=256)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--tsqr-chunk", type=int, default=0,
                   help="rows of a TSQR chunk in the recompression (0: the library default, 256)")
    p.add_argument("--autotune", action="store_true",
                   help="before timing, tune the TSQR chunk and GEMM tiling on the workload's leading block "
                        "(sp_autotune) and use them; the leaf stays the workload's")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-sample-n", type=int, default=1536)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mixed-steps", type=int, default=2,
                   help="timed steps of the mixed-precision (Newton-Schulz tail) form measured beside the binary64 "
                        "run, with ||P_mixed - P_fp64||_2 by power iteration (0: skip)")
    args = p.parse_args(argv)
    if args.n is None:
        args.n = 32768 if args.workload == "band16" else 100000
    return args


def workload_band(args, rank):
    """The workload's band for this rank (rank r > 0: same recipe, seed + r)."""
    if args.workload == "band16":
        seed = sp_inputs.workload_seed(2, rank)
        return "normal_band16", sp_inputs.normal_band(args.n, 16, seed, 0.25), args.n // 2
    variant = "band4" if args.workload == "band4" else "main"
    if rank == 0:
        (name, ab, nu), = sp_inputs.workload(4, variant=variant, n=args.n)
        return name, ab, nu
    seed = sp_inputs.workload_seed(4, rank)
    if args.workload == "band4":
        return "normal_band4", sp_inputs.normal_band(args.n, 4, seed + 1), args.n // 2
    return "anderson_wide", sp_inputs.anderson(args.n, seed, 0.5), args.n // 2


def config_dict(args, name, ab, nu):
    return {"workload": f"{name} n={args.n} b={ab.shape[1] - 1} nu={nu} leaf={args.leaf} tol={args.tol:g} "
                        f"{args.precision}" + (f" polish={args.polish}" if args.precision != "fp64" else ""),
            "n": args.n, "b": ab.shape[1] - 1, "nu": nu, "leaf": args.leaf, "tol": args.tol,
            "l2": "flushed between steps (256 MiB write); working set (GBs) exceeds L2"}


# ------------------------------------------------------------ multi-rank ----

def rank_env():
    """(world, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device="cpu"):
    """Max of a per-rank scalar over all ranks (identity at world 1)."""
    if world <= 1 or x is None:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_instances(costs, world):
    """Partition instance indices over ranks: longest first, each to the rank
    with the least estimated cost so far (ties to the lowest rank).  Every
    rank computes the same partition from the same costs."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return parts


def instance_cost(n, b):
    """Relative cost estimate of one projector: HODLR work ~ n (b + log n)^2."""
    return n * (b + np.log2(max(n, 2))) ** 2


# ------------------------------------------------------------ CPU oracle ----

def oracle_sample_band(args, ab_full):
    """The leading n_s x n_s principal block of the workload's band."""
    n_s = min(args.cpu_sample_n, args.n)
    ab = np.ascontiguousarray(ab_full[:n_s]).copy()
    for d in range(1, ab.shape[1]):
        ab[n_s - d:, d] = 0.0
    return n_s, ab


def _oracle_core_worker(ab, mu, barrier, queue):
    import oracle
    barrier.wait()
    t0 = time.perf_counter()
    oracle.projector(ab, mu)
    queue.put(time.perf_counter() - t0)


def cpu_oracle_all_cores(args, ab_full):
    """The same oracle sample on every host core at once (one spawned process
    per core, released together by a barrier): seconds per projector at full
    occupancy = slowest process / cores, scaled by (n/n_s)^3."""
    import multiprocessing as mp
    import oracle
    n_s, ab = oracle_sample_band(args, ab_full)
    mu = oracle.locate_mu(ab, n_s // 2).mu
    cores = max(1, min(os.cpu_count() or 1, 64))
    mpc = mp.get_context("spawn")
    bar, q = mpc.Barrier(cores), mpc.Queue()
    procs = [mpc.Process(target=_oracle_core_worker, args=(ab, mu, bar, q)) for _ in range(cores)]
    for pr in procs:
        pr.start()
    ts = [q.get(timeout=900) for _ in range(cores)]
    for pr in procs:
        pr.join()
    wall = max(ts)
    return cores, wall, n_s, wall / cores * (args.n / n_s) ** 3


def cpu_oracle_sample(args, ab_full, nu_full, reps=1):
    """Dense oracle projector on the leading n_s x n_s principal block of the
    workload (same recipe), seconds per projector scaled by (n/n_s)^3 (the
    dense eigensolver is O(n^3))."""
    import oracle
    n_s, ab = oracle_sample_band(args, ab_full)
    sh = oracle.locate_mu(ab, n_s // 2)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.projector(ab, sh.mu)
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    return t, n_s, t * (args.n / n_s) ** 3


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return 0
    name, ab, nu = workload_band(args, 0)
    for _ in range(args.warmup):
        cpu_oracle_sample(args, ab, nu)
    vals = []
    samples = []
    for _ in range(args.steps):
        t, n_s, scaled = cpu_oracle_sample(args, ab, nu)
        vals.append(scaled)
        samples.append(t)
    v = float(np.mean(vals))
    line = {"metric": METRIC, "value": v, "unit": "s/projector", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(samples)), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, name, ab, nu), "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "s/projector", "cores": 1, "kind": "oracle",
                             "sample": f"dense oracle projector (Householder + implicit QR eigensolver) of the "
                                       f"leading {n_s}x{n_s} block, scaled by (n/{n_s})^3"},
            "e2e": {"value": v, "unit": "s/projector", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------ accuracy, roofline --

def diff_norm2(sp, ctx, P1, P2, n, steps=30, s=4, seed=99):
    """||P1 - P2||_2 by block power iteration on the symmetric difference
    through sp_apply (device operands); a lower bound converging to the norm."""
    import torch
    X = torch.from_numpy(sp_inputs.normal(seed, n * s).reshape(s, n)).cuda()  # rows = columns of n x s
    Y1 = torch.empty_like(X)
    Y2 = torch.empty_like(X)
    est = 0.0
    for _ in range(steps):
        q, _ = torch.linalg.qr(X.T)
        X = q.T.contiguous()
        sp.sp_apply(ctx, P1, s, X, n, Y1, n)
        sp.sp_apply(ctx, P2, s, X, n, Y2, n)
        X = Y1 - Y2
        est = max(est, float(torch.linalg.norm(X, dim=1).max()))
    return est


def kernel_table(prof, givens_rotations):
    """Per kernel family: launches, ms, share of device time, counted GFLOP and
    the fraction of the binary64 rate; latency-bound chains report their
    critical path per unit instead."""
    fam = {}
    for k, (la, ms_k, fl) in prof.items():
        if k == "host_wait" or la == 0:
            continue
        base = k.split("[")[0] if k.startswith("k_gemm") and "fp32" not in k else k
        a = fam.setdefault(base, [0, 0.0, 0.0])
        a[0] += la
        a[1] += ms_k
        a[2] += fl
    total = max(sum(v[1] for v in fam.values()), 1e-9)
    out = {}
    for k, (la, ms_k, fl) in sorted(fam.items(), key=lambda kv: -kv[1][1]):
        e = {"launches": la, "ms": round(ms_k, 3), "share": round(ms_k / total, 4), "gflop": round(fl / 1e9, 3)}
        if fl > 0 and ms_k > 0:
            tf = fl / (ms_k * 1e-3) / 1e12
            e["tflops"] = round(tf, 4)
            e["frac_fp64"] = round(tf / FP64_PEAK_TFLOPS, 4)
        if k == "k_givens" and givens_rotations:
            e["ns_per_rotation"] = round(ms_k * 1e6 / givens_rotations, 1)
            e["bound"] = "latency: one dependent chain of rotations (critical path = ms)"
        out[k] = e
    return out


# ---------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- our arm -----

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1608_01164_gb300 as sp

    world, rank, local = rank_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    sp.load()
    stream = torch.cuda.current_stream().cuda_stream
    ctx = sp.sp_ctx_create(stream)
    name, ab, nu = workload_band(args, rank)
    mu, _, _ = sp.sp_locate_shift(ctx, ab, nu)
    ab_dev = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tuning = None
    if args.autotune:
        r = sp.sp_autotune(ctx, np.ascontiguousarray(ab), mu, args.tol, 0 if args.precision == "fp64" else 1)
        sp.sp_ctx_set_tuning(ctx, r.tsqr_chunk, bool(r.small_tiles))
        tuning = {"tsqr_chunk": r.tsqr_chunk, "small_tiles": int(r.small_tiles), "tuned_leaf": r.leaf,
                  "trials": r.trials, "n_tuned": r.n_tuned}
    elif args.tsqr_chunk > 0:
        sp.sp_ctx_set_tuning(ctx, args.tsqr_chunk, True)
        tuning = {"tsqr_chunk": args.tsqr_chunk, "small_tiles": 1}

    opts = sp.sp_qdwh_opts_default()
    if args.precision != "fp64":
        opts.precision = sp.SP_MIXED_FP32 if args.precision == "mixed" else sp.SP_MIXED_NS
        opts.polish_steps = args.polish

    def step(band):
        A = sp.sp_hodlr_from_band(ctx, band, mu, args.leaf, args.tol)
        S, info = sp.sp_qdwh_sign(ctx, A, opts)
        P = sp.sp_projector(ctx, S)
        tr = sp.sp_trace(ctx, P)
        for h in (A, S, P):
            sp.sp_hodlr_destroy(h)
        return tr, info

    for _ in range(args.warmup):
        tr, info = step(ab_dev)
    assert round(tr) == nu, (tr, nu)

    sampler = ClockSampler(local)
    l0 = sp.sp_launch_count()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    traces = []
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record()
        tr, info = step(ab_dev)
        ev[k][1].record()
        traces.append(tr)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    launches = sp.sp_launch_count() - l0
    ms = [a.elapsed_time(b) for a, b in ev]
    step_ms = max_over_ranks(float(np.mean(ms)), world, "cuda")
    # one more step with the library's per-launch CUDA-event profiler on (not
    # part of the timed steps): kernel breakdown, roofline, per-level times
    sp.sp_ctx_set_profiling(ctx, True)
    flush.fill_(-1.0)
    prof_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    prof_ev[0].record()
    step(ab_dev)
    prof_ev[1].record()
    torch.cuda.synchronize()
    prof_step_ms = prof_ev[0].elapsed_time(prof_ev[1])
    prof = sp.sp_ctx_profile(ctx)
    chol_levels = [round(float(v), 2) for v in sp.sp_ctx_profile_levels(ctx, 24)]
    while chol_levels and chol_levels[-1] == 0.0:
        chol_levels.pop()
    sp.sp_ctx_set_profiling(ctx, False)
    # end to end through the C ABI: host band in, trace out
    ab_host = np.ascontiguousarray(ab)
    e2e = []
    for _ in range(args.e2e_steps):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr, _ = step(ab_host)
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(e2e)) if e2e else None, world, "cuda")
    # dominant kernel by device time; the k_gemm call-site buckets are one kernel
    b = ab.shape[1] - 1
    n_rot = (2 * b + 1) * args.n - b * b - b
    table = kernel_table(prof, n_rot)
    kname, kt = next(iter(table.items()))
    kl, kms, kfl = kt["launches"], kt["ms"], kt["gflop"] * 1e9
    achieved = (kfl / (kms * 1e-3)) / 1e12 if kms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "launches": kl, "ms_total": kms, "share": kt["share"],
                "peak_source": "nominal binary64 rate (recipe table); a DFMA loop measured 1.203 TFLOP/s",
                "flops": "counted in-kernel from the actual (device-resident) sizes of every launch",
                "measured": "CUDA events around every launch of one extra, profiled step after the timed ones"}
    # the mixed-precision form beside it: time per projector and its distance
    # to the binary64 projector (power iteration on the difference)
    mixed = None
    if args.precision == "fp64" and args.mixed_steps > 0 and world == 1:
        mopts = sp.sp_qdwh_opts_default()
        mopts.precision = sp.SP_MIXED_NS
        mopts.polish_steps = args.polish

        def mstep(band, keep=False):
            A = sp.sp_hodlr_from_band(ctx, band, mu, args.leaf, args.tol)
            S, minfo = sp.sp_qdwh_sign(ctx, A, mopts)
            P = sp.sp_projector(ctx, S)
            sp.sp_hodlr_destroy(A)
            sp.sp_hodlr_destroy(S)
            if keep:
                return P, minfo
            sp.sp_hodlr_destroy(P)
            return None, minfo

        mstep(ab_dev)
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.mixed_steps)]
        for k in range(args.mixed_steps):
            flush.fill_(float(k))
            mev[k][0].record()
            mstep(ab_dev)
            mev[k][1].record()
        torch.cuda.synchronize()
        m_ms = float(np.mean([a.elapsed_time(b_) for a, b_ in mev]))
        Pm, minfo = mstep(ab_dev, keep=True)
        A = sp.sp_hodlr_from_band(ctx, ab_dev, mu, args.leaf, args.tol)
        S, _ = sp.sp_qdwh_sign(ctx, A, opts)
        P64 = sp.sp_projector(ctx, S)
        dn = diff_norm2(sp, ctx, Pm, P64, args.n)
        for h in (A, S, P64, Pm):
            sp.sp_hodlr_destroy(h)
        mixed = {"precision": "SP_MIXED_NS (binary32 Newton-Schulz tail) + binary64 polish", "steps": args.mixed_steps,
                 "s_per_projector": m_ms / 1e3, "speedup_vs_fp64": (step_ms / m_ms) if m_ms > 0 else None,
                 "diff_norm2_vs_fp64": dn, "diff_norm_method": "30 steps of block power iteration (4 vectors) "
                                                               "on P_mixed - P_fp64 through sp_apply",
                 "iters": minfo.iters, "kinds": list(minfo.kind[:minfo.iters])}
    if rank != 0:
        sp.sp_ctx_destroy(ctx)
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        t, n_s, scaled = cpu_oracle_sample(args, ab, nu)
        cpu = {"value": scaled, "unit": "s/projector", "cores": 1, "kind": "oracle",
               "sample": f"dense oracle projector of the leading {n_s}x{n_s} block of the workload "
                         f"({t:.2f} s measured), scaled by (n/{n_s})^3"}
        try:
            cores, wall, n_s2, scaled_all = cpu_oracle_all_cores(args, ab)
            cpu["all_cores"] = {"value": scaled_all, "unit": "s/projector", "cores": cores,
                                "sample": f"{cores} concurrent oracle projectors of the same {n_s2}x{n_s2} block "
                                          f"(slowest {wall:.2f} s), per-projector time / cores, scaled by "
                                          f"(n/{n_s2})^3"}
        except Exception as e:  # the one-core figure stands on its own
            cpu["all_cores"] = {"unavailable": str(e)[:200]}
    value = step_ms / 1e3 / world
    line = {"metric": METRIC, "value": value, "unit": "s/projector", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic", "config": dict(config_dict(args, name, ab, nu), **({"tuning": tuning} if tuning else {})),
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_s / world if e2e_s else None, "unit": "s/projector", "steps": len(e2e),
                    "h2d_bytes_per_step": int(ab_host.nbytes), "d2h_bytes_per_step": 8},
            "gpu_launches": int(launches), "clocks": clocks,
            "detail": {"iters": info.iters, "kinds": list(info.kind[:info.iters]), "max_rank": info.max_rank,
                       "alpha": info.alpha, "l0": info.l0, "ms_polish": info.ms_polish,
                       "ms_param": info.ms_param, "ms_qr": info.ms_qr, "ms_chol": info.ms_chol,
                       "ms_chol_phases": {"square": info.ms_mult, "factor": info.ms_factor, "solve": info.ms_solve,
                                          "combine": info.ms_combine},
                       "trace_minus_nu": traces[-1] - nu, "wall_s": t_wall,
                       "chol_self_ms_per_level": chol_levels, "profiled_step_ms": prof_step_ms,
                       "levels": info.levels, "max_rank_level": list(info.max_rank_level[:info.levels]),
                       "mean_rank_level": [round(x, 2) for x in info.mean_rank_level[:info.levels]],
                       "nominal_bytes": info.nominal_bytes, "allocated_bytes": info.bytes,
                       "mixed": mixed,
                       "kernel_families": table,
                       "kernels": {k: {"launches": v[0], "ms": round(v[1], 3), "gflop": round(v[2] / 1e9, 3)}
                                   for k, v in prof.items() if v[0]}}}
    print(json.dumps(line), flush=True)
    sp.sp_ctx_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Workload 3: independent instances (n log-uniform in [512, 8192], b in
    {1,2,4,8}, U[-1,1], nu in {n/3, n/2}); metric projectors/s.  Under
    torchrun each rank takes its share of the instances.  A step is one
    sp_batched_projector call over this rank's instances plus the traces."""
    import torch
    import torch.distributed as dist

    import paper_1608_01164_gb300 as sp

    world, rank, local = rank_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    sp.load()
    stream = torch.cuda.current_stream().cuda_stream
    ctx = sp.sp_ctx_create(stream)
    everything = sp_inputs.workload(3, n=args.batch)
    mine = shard_instances([instance_cost(ab.shape[0], ab.shape[1] - 1) for _, ab, _ in everything], world)[rank]
    inst = [everything[i] for i in mine]
    mus = [sp.sp_locate_shift(ctx, ab, nu)[0] for _, ab, nu in inst]
    bands = [torch.from_numpy(np.ascontiguousarray(ab)).cuda() for _, ab, _ in inst]
    hosts = [np.ascontiguousarray(ab) for _, ab, _ in inst]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(bs):
        Ps, infos = sp.sp_batched_projector(ctx, bs, mus, leaf=0, tol=args.tol, nstreams=args.nstreams)
        trs = [sp.sp_trace(ctx, P) for P in Ps]
        for P in Ps:
            sp.sp_hodlr_destroy(P)
        return trs, infos

    for _ in range(args.warmup):
        trs, infos = step(bands)
    bad = sum(1 for (_, _, nu), t in zip(inst, trs) if round(t) != nu)
    l0 = sp.sp_launch_count()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record()
        trs, infos = step(bands)
        ev[k][1].record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = sp.sp_launch_count() - l0
    dt = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])) / 1e3, world, "cuda")
    bad = int(max_over_ranks(bad, world, "cuda") if world > 1 else bad)
    # one profiled step (not timed): kernel families and the dominant one
    sp.sp_ctx_set_profiling(ctx, True)
    step(bands)
    torch.cuda.synchronize()
    prof = sp.sp_ctx_profile(ctx)
    sp.sp_ctx_set_profiling(ctx, False)
    table = kernel_table(prof, 0)
    if not table:
        raise RuntimeError("the profiled batch reported no kernel launches")
    kname, kt = next(iter(table.items()))
    achieved = kt.get("tflops", 0.0)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "launches": kt["launches"],
                "ms_total": kt["ms"], "share": kt["share"],
                "peak_source": "nominal binary64 rate (recipe table); a DFMA loop measured 1.203 TFLOP/s",
                "flops": "counted in-kernel from the actual (device-resident) sizes of every launch",
                "measured": "CUDA events around every launch of one extra, profiled step after the timed ones "
                            "(kernels of concurrent instances overlap, so shares are of summed kernel time)"}
    # end to end: host bands in, traces out
    e2e = []
    for _ in range(max(1, args.e2e_steps)):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(hosts)
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(e2e)), world, "cuda")
    sp.sp_ctx_destroy(ctx)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            import oracle
            # the oracle on the smallest instances, whole projectors, until ~10 s of CPU work
            order = sorted(range(len(everything)), key=lambda i: everything[i][1].shape[0])
            t_cpu, done, n_sum = 0.0, 0, 0
            for i in order:
                _, ab, nu = everything[i]
                sh = oracle.locate_mu(ab, nu)
                t0 = time.perf_counter()
                oracle.projector(ab, sh.mu)
                t_cpu += time.perf_counter() - t0
                done += 1
                n_sum += ab.shape[0]
                if t_cpu > 10.0:
                    break
            # scale by sum n^3 of all instances over sum n^3 of the sample
            w_all = sum(ab.shape[0] ** 3 for _, ab, _ in everything)
            w_s = sum(everything[i][1].shape[0] ** 3 for i in order[:done])
            cpu = {"value": len(everything) / (t_cpu * w_all / w_s), "unit": "projectors/s", "cores": 1,
                   "kind": "oracle",
                   "sample": f"dense oracle projectors of the {done} smallest instances ({t_cpu:.1f} s), "
                             f"scaled to all {len(everything)} instances by sum n^3"}
        h2d = int(sum(h.nbytes for h in hosts))
        line = {"metric": METRIC, "value": len(everything) / dt, "unit": "projectors/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt, "higher_is_better": True,
                "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": f"batched: {len(everything)} instances, n log-uniform [512, 8192], "
                                       f"b in {{1,2,4,8}}, U[-1,1], nu in {{n/3, n/2}}, leaf auto, tol {args.tol:g}, "
                                       f"{args.nstreams} streams per GPU",
                           "l2": "flushed between steps (256 MiB write)"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": len(everything) / e2e_s, "unit": "projectors/s", "steps": len(e2e),
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * len(inst)},
                "gpu_launches": int(launches), "clocks": clocks, "trace_mismatches": bad,
                "timing": "CUDA events on the calling stream around each batch call (the call synchronises its "
                          "worker streams), max over ranks",
                "detail": {"kernel_families": table}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
