#!/usr/bin/env python
"""Benchmark of the Schur-complement PCG solve path on GB300.

Workload: the latency sweep's largest single instance -- seeded Kuka-shaped
LQ data, nx = 14, nu = 7, N = 512 knot points, float32 storage with
extended-precision dot products, PCG warm-started from the previous solution
perturbed by 1% relative N(0, 1) noise, exit at relative residual 1e-6.
One step = one whole pass of the path: form_schur and form_precon (one fused
launch), pcg_solve, recover_step.  L2 is flushed (a 256 MiB write) between timed steps; steps
are timed on the device with CUDA events on the launching stream.

Also measured in the same run and reported in the same JSON line:
  e2e        the same solve through the public API with host buffers: the
             step's inputs copied from pinned host memory (one copy) and the
             results read back (one copy) inside the timed region;
  batched    256 ragged instances (N_i ~ U{32..512}), 20 warm solves per
             instance captured in one CUDA graph, against the single-instance
             path looped over the same solves on the same GPU;
  roofline   the PCG kernel's algorithmic bytes per launch over its
             event-timed duration, against the measured HBM copy bandwidth;
  cpu_baseline  the FP64 oracle (banded LU of the full KKT system, one core)
             on a bounded sample of the same instance.

`--impl reference` times the oracle alone on the host cores (the CPU
comparison arm) and prints the same metric.
Multi-GPU (torchrun): the single-instance solve does not shard, so each
rank runs independent replicas; value is aggregated over all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workload import gen  # noqa: E402

NX, NU, NKNOT = 14, 7, 512
SEED = gen.CONFIG_SWEEP["seed_base"] + NKNOT
METRIC = "Schur-PCG us/solve at N=512 (nx=14, nu=7, warm start, rel. residual 1e-6)"
UNIT = "us/solve"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--batched-solves", type=int, default=gen.CONFIG_BATCH["solves"])
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--sweep-reps", type=int, default=gen.CONFIG_SWEEP.get("reps", 1000))
    p.add_argument("--no-large", action="store_true")
    p.add_argument("--large-solves", type=int, default=gen.CONFIG_LARGE["solves"])
    p.add_argument("--large-refine-tol", type=float, default=1e-2,
                   help="exit tolerance of the large-state refinement's correction solves")
    p.add_argument("--large-batch", type=int, default=gen.CONFIG_LARGE["B"],
                   help="instances of the large-state batch (a smaller batch for profiling)")
    return p.parse_args()


def workload_config(world: int = 1) -> dict:
    """The `config` of both arms' JSON lines (the same workload)."""
    return {"workload": f"single instance N={NKNOT} nx={NX} nu={NU}, warm-started "
                        f"(lambda* x (1 + 0.01 xi)), tol 1e-6 relative residual",
            "seed": SEED, "l2": "flushed between steps (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "dot_accumulation": "double-float (f32 pair)"}


def workload_lq():
    c = gen.CONFIG_SWEEP
    return gen.kuka_lq(NX, NU, NKNOT, SEED, dt=c["dt"], qd=c["qd"]).astype(np.float32)


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- helpers
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cluster_kernel_sha() -> str:
    """sha256[:16] over the sources the cluster PCG kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("pcg.cu", "pcg_rows.cuh", "common.cuh", "launch.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2309_08079_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def pcg_traffic_from_profile():
    """DRAM bytes per PCG launch from the committed ncu summary, if it was
    captured from the current kernel source (else None)."""
    prof = os.path.join(ROOT, "profiles", "pcg_cluster_kernel_N512.md")
    try:
        sha = cluster_kernel_sha()
        txt = open(prof).read()
        m_sha = re.search(r"cluster kernel sources sha256\[:16\]:\s*([0-9a-f]+)", txt)
        m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        if m_sha and m_tr and m_sha.group(1) == sha:
            return float(m_tr.group(1))
    except Exception:
        pass
    return None


def pcg_bytes_per_knot_iter(nx: int, esize: int = 4) -> int:
    """Algorithmic bytes one PCG iteration moves per knot: both symmetric
    block-tridiagonal matrices once (T = nx(nx+1)/2 + nx^2 words each) and
    seven vectors."""
    T = nx * (nx + 1) // 2 + nx * nx
    return (2 * T + 7 * nx) * esize


def latency_roofline(s, lt, sch, opts, iters_mean: float, launch_us: float, rounds: int = 2000) -> dict:
    """The single-instance PCG kernel against its synchronisation floor: each
    iteration of Algorithm 1 takes two cluster reductions, each at least the
    time mpcg_bench_exchange measures for the launch shape the solve uses
    (the same exchange code with no arithmetic), so the floor is
    2 x exchange per iteration.  achieved / peak in PCG iterations per second."""
    sh = s.pcg_shape(lt, sch, opts)
    if sh["form"] != "cluster":
        return {"bound": "n/a", "note": f"kernel form {sh['form']}"}
    x = s.bench_exchange(sh["C"], sh["threads"] // 32, rounds=rounds)
    floor_ns = 2.0 * x["ns"]
    t_it_ns = launch_us * 1e3 / max(iters_mean, 1.0)
    return {"bound": "sync_latency", "achieved": 1e9 / t_it_ns, "peak": 1e9 / floor_ns,
            "unit": "PCG iterations/s", "frac": floor_ns / t_it_ns,
            "peak_source": f"measured: mpcg_bench_exchange on the solve's launch shape "
                           f"(C={sh['C']} CTAs x {sh['threads'] // 32} warps), 2 exchanges per iteration",
            "exchange_ns": x["ns"], "exchange_cycles": x["cycles"], "ns_per_iteration": t_it_ns,
            "floor_ns_per_iteration": floor_ns, "shape": sh}


def profile_onchip():
    """SMEM-pipe share and barrier-stall share of the cluster kernel from the
    committed ncu summary, when it was taken from the current sources."""
    prof = os.path.join(ROOT, "profiles", "pcg_cluster_kernel_N512.md")
    try:
        txt = open(prof).read()
        m_sha = re.search(r"cluster kernel sources sha256\[:16\]:\s*([0-9a-f]+)", txt)
        if not m_sha or m_sha.group(1) != cluster_kernel_sha():
            return None
        out = {}
        for key, pat in (("smem_pipe_frac_active_sms", r"smem_pipe_frac_active_sms:\s*([0-9.eE+-]+)"),
                         ("barrier_stall_share", r"barrier_stall_share:\s*([0-9.eE+-]+)")):
            m = re.search(pat, txt)
            if m:
                out[key] = float(m.group(1))
        return out or None
    except Exception:
        return None


def hbm_peak():
    hbm = measured_peaks().get("hbm_gbs")
    return (hbm, "of measured") if hbm is not None else (6800.0, "of fallback")


def pct(x):
    x = np.asarray(x, dtype=np.float64)
    return {"p10": float(np.percentile(x, 10)), "p50": float(np.median(x)),
            "p90": float(np.percentile(x, 90)), "max": float(np.max(x))}


def _oracle_worker(lq64):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.kkt_solve(lq64)
    return time.perf_counter() - t0


def oracle_batched_baseline(items, seconds: float):
    """FP64 oracle over all host cores, one instance per worker process
    (a spawned pool: nothing forked after CUDA is initialised), on the first
    instances of the batch until about `seconds` of wall time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [items[0].astype(np.float64)] * cores)  # warm the workers
        n, t0 = 0, time.perf_counter()
        while n < len(items):
            chunk = [it.astype(np.float64) for it in items[n:n + cores]]
            pool.map(_oracle_worker, chunk)
            n += len(chunk)
            if time.perf_counter() - t0 >= seconds:
                break
        el = time.perf_counter() - t0
    return n / el, n, cores


def oracle_baseline(lq, seconds: float):
    """FP64 oracle on one host core, repeated on the workload instance."""
    import oracle
    oracle.build()
    lq64 = lq.astype(np.float64)
    oracle.kkt_solve(lq64)
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.kkt_solve(lq64)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 10000:
            break
    return el / n * 1e6, n


def max_over_ranks(x: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the job's
    time is its slowest rank's); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    lq = workload_lq()
    import oracle
    oracle.build()
    lq64 = lq.astype(np.float64)
    for _ in range(max(args.warmup, 0)):
        oracle.kkt_solve(lq64)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.kkt_solve(lq64)
    el = time.perf_counter() - t0
    us = el / args.steps * 1e6
    sample = (f"{args.steps} FP64 banded-LU KKT solves of the N={NKNOT}, nx={NX}, nu={NU} "
              f"instance (seed {SEED}), one thread")
    line = {"impl": "reference", "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": us / 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(1),
            "cpu_baseline": {"value": us, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": us, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2309_08079_gb300 import build as libbuild
    from paper_2309_08079_gb300.solver import LQTensors, Solver, make_opts, read_stats

    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    lq = workload_lq()
    s = Solver(dev)
    lt = LQTensors.from_numpy(lq, device=dev)
    opts = make_opts(tol=1e-6)
    sch = s.alloc_schur(lt)

    # cold solve gives lambda*; warm starts are lambda* perturbed per step
    lam_star, _, _, st0, _ = s.solve(lt, opts=opts, schur=sch)
    torch.cuda.synchronize()
    cold = read_stats(st0)[0]
    lam_star_np = lam_star.cpu().double().numpy()
    nsteps = args.warmup + args.steps
    lam0 = [torch.as_tensor(gen.warm_start(lam_star_np, SEED, i), dtype=torch.float32, device=dev)
            for i in range(nsteps)]
    lam_bufs = [t.clone() for t in lam0]
    stats = s.alloc_stats(nsteps, dev)
    dx = torch.empty(NKNOT, NX, device=dev)
    du = torch.empty(NKNOT - 1, NU, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nsteps)]

    def step(i):
        e = ev[i]
        e[0].record(stream)
        s.form(lt, sch)
        e[1].record(stream)
        s.pcg_solve(lt, sch, lam_bufs[i], opts, stats[i * 24:(i + 1) * 24])
        e[2].record(stream)
        s.recover_step(lt, lam_bufs[i], dx, du)
        e[3].record(stream)

    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    torch.cuda.synchronize()
    for i in range(args.warmup, nsteps):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    timed = range(args.warmup, nsteps)
    step_ms = [ev[i][0].elapsed_time(ev[i][3]) for i in timed]
    pcg_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in timed]
    form_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in timed]
    tot_ms = max_over_ranks(float(np.sum(step_ms)), dev)
    st = read_stats(stats)[args.warmup:]
    converged = bool(np.all(st["status"] == 0))
    iters = st["iters"].astype(np.float64)

    # parity spot check of the last timed step against the oracle
    import oracle
    lo, xo, uo = oracle.kkt_solve(lq.astype(np.float64))
    err_lam = oracle.relerr(lam_bufs[nsteps - 1].cpu().double().numpy(), lo)
    err_dz = oracle.relerr(np.concatenate([dx.cpu().double().numpy().ravel(),
                                           du.cpu().double().numpy().ravel()]),
                           np.concatenate([xo.ravel(), uo.ravel()]))

    # ---- end to end through the public API with host buffers ---------------
    e2e = run_e2e(s, lq, lam0, opts, dev, flush, min(args.steps, 50), args.warmup)

    # ---- roofline of the PCG kernel -----------------------------------------
    T = NX * (NX + 1) // 2 + NX * NX
    bytes_per_knot_iter = (2 * T + 7 * NX) * 4
    alg_bytes = float(np.mean(iters)) * NKNOT * bytes_per_knot_iter
    pcg_s = float(np.mean(pcg_ms)) / 1e3
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_note = "of measured"
    if hbm is None:
        hbm, peak_note = 6800.0, "of fallback"
    achieved = alg_bytes / pcg_s / 1e9
    # the kernel's operators stay on chip (registers): what bounds it is the
    # latency of its two cluster reductions per iteration, measured by the
    # exchange microbenchmark on the same launch shape; HBM is secondary
    roofline = latency_roofline(s, lt, sch, opts, float(np.mean(iters)), pcg_s * 1e6)
    roofline.update({"traffic": pcg_traffic_from_profile(), "kernel": "pcg_cluster_kernel",
                     "launch_us": pcg_s * 1e6, "onchip_ncu": profile_onchip(),
                     "hbm": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_source": peak_note,
                             "alg_bytes_per_launch": alg_bytes}})

    batched = backward = sweep = exit_sweep = precon_compare = dense_cost = nmpc = large = None
    dot64 = run_dot64(s, dev, lq, lam0, flush, min(args.steps, 50), us_default=float(np.mean(pcg_ms)) * 1e3,
                      iters_default=float(np.mean(iters)))
    if not args.no_sweep:
        sweep = run_sweep(s, dev, args.sweep_reps, flush)
        exit_sweep = run_exit_sweep(s, dev, min(args.sweep_reps, 200))
        precon_compare = run_precon_compare(s, dev, min(args.sweep_reps, 100))
        dense_cost = run_dense_cost(s, dev, min(args.sweep_reps, 50))
        nmpc = run_nmpc(s, dev, 20)
    if not args.no_batched:
        batched = run_batched(s, dev, args.batched_solves)
        backward = run_backward(s, dev)
    if not args.no_large:
        large = run_large(s, dev, args.large_solves, args.large_batch, args.large_refine_tol)
    if batched is not None and rank == 0 and world == 1 and not args.no_cpu:
        c = gen.CONFIG_BATCH
        Ns_b = gen.batch_horizons(c["B"], c["N_lo"], c["N_hi"], c["n_seed"])
        items = [gen.kuka_lq(c["nx"], c["nu"], int(n), c["seed_base"] + i, dt=c["dt"], qd=c["qd"]).astype(np.float32)
                 for i, n in enumerate(Ns_b)]
        rate, n_done, cores = oracle_batched_baseline(items, args.cpu_seconds)
        batched["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                   "sample": f"{n_done} FP64 banded-LU KKT solves of the batch's first instances, "
                                             f"one per process"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        us, n = oracle_baseline(lq, args.cpu_seconds)
        cpu = {"value": us, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} FP64 banded-LU KKT solves of the same N={NKNOT} instance, one thread"}

    value = tot_ms * 1e3 / (args.steps * world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(world),
        "step_us": pct(np.array(step_ms) * 1e3),
        "step_breakdown_us": {"form": float(np.mean(form_ms)) * 1e3, "pcg": float(np.mean(pcg_ms)) * 1e3,
                              "recover": float(np.mean(step_ms) - np.mean(form_ms) - np.mean(pcg_ms)) * 1e3},
        "pcg_iters": {"mean": float(np.mean(iters)), "min": int(iters.min()), "max": int(iters.max()),
                      "cold": int(cold["iters"])},
        "converged": converged,
        "parity": {"err_lambda": err_lam, "err_dz": err_dz, "tol": 1e-4},
        "clocks": clk, "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roofline,
        "cpu_baseline": cpu, "batched": batched, "backward": backward, "sweep": sweep,
        "exit_sweep": exit_sweep, "precon_compare": precon_compare, "dense_cost": dense_cost,
        "nmpc": nmpc,
        "large_state": large,
        "dot_fp64": dot64,
    }
    line["summary"] = summarize(line)
    if rank == 0:
        print(json.dumps(line), flush=True)


def summarize(line):
    """The secondary figures in a few keys, last in the line (a reader of its
    tail sees them)."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    out = {"us_per_solve_N512": line["value"], "e2e_us": g(line, "e2e", "value"),
           "pcg_us": g(line, "step_breakdown_us", "pcg"), "iters": g(line, "pcg_iters", "mean"),
           "sync_latency_frac": g(line, "roofline", "frac"), "hbm_frac": g(line, "roofline", "hbm", "frac"),
           "parity_lambda": g(line, "parity", "err_lambda"), "parity_dz": g(line, "parity", "err_dz"),
           "dot_fp64_us": g(line, "dot_fp64", "pcg_us"), "dot_fp64_err_lambda": g(line, "dot_fp64", "err_lambda"),
           "batched_solves_per_s": g(line, "batched", "solves_per_s"),
           "batched_loop_solves_per_s": g(line, "batched", "loop_solves_per_s"),
           "batched_speedup_vs_loop": g(line, "batched", "speedup_vs_loop"),
           "batched_roofline": {k: g(line, "batched", "per_kernel", "autotuned", "pcg_roofline", k)
                                for k in ("bound", "frac")},
           "backward_fwd_ms": g(line, "backward", "fwd_ms"), "backward_bwd_ms": g(line, "backward", "bwd_ms"),
           "backward_grad_err": g(line, "backward", "grad_relerr_vs_oracle"),
           "large_fwd_ms": g(line, "large_state", "fwd_ms"), "large_bwd_ms": g(line, "large_state", "bwd_ms"),
           "large_err_lambda": g(line, "large_state", "err_lambda_vs_oracle", "max"),
           "large_grad_err": g(line, "large_state", "grad_err_vs_oracle", "max"),
           "large_pcg_hbm_frac": g(line, "large_state", "pcg_roofline", "frac"),
           "large_pcg_streamed_frac": g(line, "large_state", "pcg_roofline", "streamed_frac"),
           "large_pcg_ms": g(line, "large_state", "pcg_roofline", "pcg_ms"),
           "large_pcg_dot_fp64_ms": g(line, "large_state", "dot_fp64", "pcg_ms")}
    sw = g(line, "sweep", "per_N") or {}
    out["sweep_p50_us"] = {k: g(v, "us_per_solve", "p50") for k, v in sw.items()}
    return out


def run_dot64(s, dev, lq, lam0, flush, steps, us_default, iters_default):
    """The measured workload with the PCG dot products accumulated in FP64
    instructions (opts.dot = 1) instead of float pairs: µs per PCG solve,
    iterations and parity, beside the default."""
    import torch
    import oracle
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    lt = LQTensors.from_numpy(lq, device=dev)
    sch = s.alloc_schur(lt)
    s.form(lt, sch)
    o = make_opts(tol=1e-6, dot=1)
    stream = torch.cuda.current_stream(dev)
    lams = [t.clone() for t in lam0[:steps + 3]]
    stats = s.alloc_stats(len(lams), dev)
    for i in range(3):
        s.pcg_solve(lt, sch, lams[i], o, stats[i * 24:(i + 1) * 24])
    torch.cuda.synchronize()
    tim = _step_timer(s, stream)
    for i in range(3, len(lams)):
        flush.zero_()
        tim(lambda: s.pcg_solve(lt, sch, lams[i], o, stats[i * 24:(i + 1) * 24]))
    torch.cuda.synchronize()
    st = read_stats(stats)[3:]
    us = np.array(tim.ms()) * 1e3
    lo, _, _ = oracle.kkt_solve(lq.astype(np.float64))
    err = oracle.relerr(lams[-1].cpu().double().numpy(), lo)
    return {"workload": f"the N={lq.N} warm-started solve, PCG only, {len(us)} solves",
            "pcg_us": float(np.median(us)), "us_pct": pct(us), "iters_mean": float(np.mean(st["iters"])),
            "converged": bool(np.all(st["status"] == 0)), "err_lambda": err,
            "default_pcg_us": us_default, "default_iters_mean": iters_default,
            "slowdown_vs_default": float(np.median(us)) / us_default}


def run_e2e(s, lq, lam0, opts, dev, flush, steps, warmup):
    """Same solve through the public API with host buffers: the step's inputs
    (A..c and lambda0) staged in one pinned buffer and copied in with one
    H2D copy, the three launches, and lambda, dx, du and the stats copied
    back with one D2H copy (paper_2309_08079_gb300.staging.HostStaging)."""
    import torch
    from paper_2309_08079_gb300.staging import HostStaging
    stream = torch.cuda.current_stream()
    stg = HostStaging(s, lq.nx, lq.nu, lq.N, device=dev)
    stg.load(lq)
    lam_h = [t.cpu().numpy() for t in lam0[:warmup + steps]]
    times = []
    for i in range(warmup + steps):
        flush.zero_()
        stg.host["lam"][:] = lam_h[i]  # the controller's own host memory, before the timed region
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        stg.step(opts, stream)
        b.record(stream)
        b.synchronize()
        if i >= warmup:
            times.append(a.elapsed_time(b))
    st = stg.read_stats()[0]
    return {"value": float(np.mean(times)) * 1e3, "unit": UNIT, "h2d_bytes_per_step": int(stg.h2d_bytes),
            "d2h_bytes_per_step": int(stg.d2h_bytes), "steps": steps, "copies_per_step": 2,
            "last_status": int(st["status"])}


def run_batched(s, dev, solves):
    """256 ragged instances, `solves` warm solves each: one CUDA graph of
    batched calls vs the single-instance path looped on the same GPU."""
    import torch
    from paper_2309_08079_gb300.autotune import Autotuner, PlanRunner
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_BATCH
    Ns = gen.batch_horizons(c["B"], c["N_lo"], c["N_hi"], c["n_seed"])
    batch = gen.kuka_batch(c["nx"], c["nu"], Ns, c["seed_base"], dt=c["dt"], qd=c["qd"]).astype(np.float32)
    lt = LQTensors.from_batch(batch, device=dev)
    opts = make_opts(tol=1e-6)
    sch = s.alloc_schur(lt)
    ws = s.alloc_workspace(lt)
    lam_star, _, _, st0, _ = s.solve(lt, opts=opts, schur=sch, workspace=ws)
    torch.cuda.synchronize()
    ls = lam_star.cpu().double().numpy()
    ko = batch.knot_off
    master = []
    for rep in range(solves):
        parts = [gen.warm_start(ls[ko[b]:ko[b + 1]], c["seed_base"] + b, rep) for b in range(batch.B)]
        master.append(torch.as_tensor(np.concatenate(parts), dtype=torch.float32, device=dev))
    work = [m.clone() for m in master]
    stats = [s.alloc_stats(batch.B, dev) for _ in range(solves)]
    dx = torch.empty(lt.total, lt.nx, device=dev)
    du = torch.empty(lt.total - lt.nb, lt.nu, device=dev)

    def restore():
        for w, m in zip(work, master):
            w.copy_(m)

    def body(opts_m):
        for r in range(solves):
            s.form(lt, sch)
            if isinstance(opts_m, PlanRunner):
                opts_m.pcg_solve(sch, work[r], stats[r])
            else:
                s.pcg_solve(lt, sch, work[r], opts_m, stats[r], ws)
            s.recover_step(lt, work[r], dx, du)

    # the autotuner times its candidate launch plans on the first warm start,
    # each captured in a CUDA graph as below (a fresh cache, so every run
    # tunes), and the chosen plan is graphed too
    with tempfile.TemporaryDirectory() as td:
        tuner = Autotuner(s, cache_path=os.path.join(td, "tune.json"), reps=3, graph=True)
        tuned = tuner.tune(lt, sch, master[0], opts)
        runner = tuner.runner(lt, sch, master[0], opts)

    # Sync-latency floor of the cluster launches: the clusters keep each
    # instance's operators on chip, so an instance solved on C CTAs holds C
    # SMs for at least iterations x 2 exchanges at the latency
    # mpcg_bench_exchange measures on its launch shape; the floor is that
    # SM-time summed over the graph's solves and spread over every SM.
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    xcache = {}

    def cluster_floor_ms(groups, iters):
        """(floor over the cluster groups, their shapes, the instances of
        the other groups, which stream their operators from HBM)."""
        sm_ns, shapes, other = 0.0, [], []
        for o_g, N_g, idx in groups:
            sh = s.pcg_shape(lt, sch, o_g, N=N_g)
            if sh["form"] != "cluster":
                other.extend(int(i) for i in idx)
                continue
            key = (sh["C"], sh["threads"] // 32)
            if key not in xcache:
                xcache[key] = s.bench_exchange(*key, rounds=1000)["ns"]
            sm_ns += float(np.sum(iters[idx])) * 2.0 * xcache[key] * sh["C"]
            shapes.append({"C": sh["C"], "threads": sh["threads"], "instances": int(len(idx))})
        if not shapes:
            return None, None, other
        return sm_ns / n_sms * 1e-6, shapes, other

    # capture the repeated solves in one graph, once per PCG kernel form
    per_mode = {}
    for mode, name in ((1, "cluster"), (2, "cta_l2"), (3, "cta_tma"), (runner, "autotuned")):
        om = make_opts(tol=1e-6, mode=mode) if isinstance(mode, int) else mode
        restore()
        body(om)  # warm-up outside capture (chooses the launch shape)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                body(om)
        torch.cuda.current_stream().wait_stream(side)
        times = []
        for _ in range(3):
            restore()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        stb = np.concatenate([read_stats(x) for x in stats])
        # PCG algorithmic bytes of all the graph's solves over the whole graph
        # time (formation and recovery included in the time)
        alg = float(np.sum(stb["iters"].astype(np.float64) * np.tile(Ns, solves))) * \
            pcg_bytes_per_knot_iter(c["nx"])
        hbm, note = hbm_peak()
        gms = float(np.median(times))
        hbm_frac = alg / (gms / 1e3) / 1e9 / hbm
        if name in ("cluster", "autotuned"):
            it_b = stb["iters"].astype(np.float64).reshape(solves, batch.B).sum(axis=0)
            groups = ([(om, int(np.max(Ns)), np.arange(batch.B))] if name == "cluster" else
                      [(l.opts, l.N, l.inst.cpu().numpy()) for l in om.launches])
            floor, shapes, other = cluster_floor_ms(groups, it_b)
        else:
            floor, shapes, other = None, None, []
        if floor is not None:
            roof = {"bound": "sync_latency", "frac": floor / gms, "floor_ms": floor, "shapes": shapes,
                    "note": "SM-time of every cluster-launched instance at 2 measured exchanges "
                            "(mpcg_bench_exchange, its launch shape) per PCG iteration, spread over all "
                            "SMs, over the graph time (formation and recovery included); operators stay "
                            "on chip",
                    "hbm_equivalent_frac": hbm_frac, "peak_source": note}
            if other:
                # a mixed plan: the tiled (or L2) groups stream their operators
                ot = np.asarray(other)
                alg_o = float(np.sum(it_b[ot] * Ns[ot])) * pcg_bytes_per_knot_iter(c["nx"])
                roof["other_groups"] = {"instances": int(len(ot)), "bound": "hbm",
                                        "frac": alg_o / (gms / 1e3) / 1e9 / hbm,
                                        "note": "their PCG algorithmic bytes over the same graph time"}
        else:
            roof = {"bound": "hbm", "frac": hbm_frac, "peak_source": note,
                    "note": "PCG algorithmic bytes of all solves over the graph time (operators streamed "
                            "from L2/HBM every iteration)"}
        per_mode[name] = {"graph_ms": gms,
                          "converged": bool(np.all(stb["status"] == 0)),
                          "mean_iters": float(np.mean(stb["iters"])),
                          "pcg_roofline": roof}
        del g
    best = min(per_mode, key=lambda k: per_mode[k]["graph_ms"])
    t_graph = per_mode[best]["graph_ms"] / 1e3
    ok_b = all(v["converged"] for v in per_mode.values())
    iters_b = per_mode[best]["mean_iters"]

    # plain loop: the single-instance path over the same solves
    items = [LQTensors.from_numpy(it, device=dev) for it in batch.items]
    schs = [s.alloc_schur(it) for it in items]
    st1 = s.alloc_stats(1, dev)
    restore()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for r in range(solves):
        for bi, it in enumerate(items):
            lam_i = work[r][ko[bi]:ko[bi + 1]]
            s.form(it, schs[bi])
            s.pcg_solve(it, schs[bi], lam_i, opts, st1)
            s.recover_step(it, lam_i)
    b.record()
    b.synchronize()
    t_loop = a.elapsed_time(b) / 1e3
    n = batch.B * solves
    return {"workload": f"{batch.B} instances, N_i ~ U{{{c['N_lo']}..{c['N_hi']}}} "
                        f"(sum {int(ko[-1])} knots), {solves} warm solves each",
            "solves_per_s": n / t_graph, "loop_solves_per_s": n / t_loop,
            "speedup_vs_loop": t_loop / t_graph, "graph_ms": t_graph * 1e3, "kernel": best,
            "per_kernel": {k: {"solves_per_s": n / (v["graph_ms"] / 1e3), **v} for k, v in per_mode.items()},
            "autotune": {"plan": tuned["plan"], "groups": len(runner.launches),
                         "one_solve_ms": {k: round(v, 3) for k, v in tuner.last_timings.items()}},
            "mean_iters": iters_b, "converged": ok_b, "cold_iters_mean": float(np.mean(read_stats(st0)["iters"]))}


def run_backward(s, dev, reps=5):
    """Forward + backward of the gradient workload (64 instances, N = 128,
    loss sum ||dz||^2 + w^T lambda): batched calls vs the single-instance
    path looped over the same instances."""
    import torch
    import oracle
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_GRAD
    batch = gen.kuka_batch(c["nx"], c["nu"], [c["N"]] * c["B"], c["seed_base"], dt=c["dt"],
                           qd=c["qd"]).astype(np.float32)
    lt = LQTensors.from_batch(batch, device=dev)
    K = lt.total
    w = torch.as_tensor(gen.loss_weights(K * c["nx"], c["w_seed"]).reshape(K, c["nx"]),
                        dtype=torch.float32, device=dev)
    opts = make_opts(tol=1e-6)
    sch = s.alloc_schur(lt)
    ws = s.alloc_workspace(lt)
    st = s.alloc_stats(lt.nb, dev)
    lam = torch.zeros(K, c["nx"], device=dev)

    def fwd():
        lam.zero_()
        return s.solve(lt, lam, opts=opts, schur=sch, stats=st, workspace=ws)

    def bwd(lam_, dx, du):
        return s.backward(lt, sch, lam_, dx, du, w, 2 * dx, 2 * du, opts=opts, workspace=ws)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b), out

    fwd_ms, bwd_ms = [], []
    for i in range(reps + 1):
        tf, (lam_o, dx, du, _, _) = timed(fwd)
        tb, (g, bst) = timed(lambda: bwd(lam_o, dx, du))
        if i:
            fwd_ms.append(tf)
            bwd_ms.append(tb)
    ok = bool(np.all(read_stats(bst)["status"] == 0))
    hbm, note = hbm_peak()
    it_f = read_stats(st)["iters"].astype(np.float64)
    it_b = read_stats(bst)["iters"].astype(np.float64)
    alg = float(np.sum(it_f + it_b)) * c["N"] * pcg_bytes_per_knot_iter(c["nx"])
    # the batch's clusters keep their operators on chip: the floor is the
    # reductions' latency, 2 exchanges per iteration on each cluster, the
    # instances spread over the co-resident clusters
    sh = s.pcg_shape(lt, sch, opts)
    lat = None
    if sh["form"] == "cluster":
        x = s.bench_exchange(sh["C"], sh["threads"] // 32, rounds=1000)
        lat = float(np.sum(it_f + it_b)) * 2.0 * x["ns"] * 1e-6 / max(1, min(sh["clusters"], c["B"]))
    # gradient of instance 0 against the oracle's analytic gradient
    it0 = batch.items[0].astype(np.float64)
    l0, x0, u0 = oracle.kkt_solve(it0)
    w0 = w[:c["N"]].double().cpu().numpy()
    go = oracle.grad(it0, l0, x0, u0, w0, 2 * x0, 2 * u0)
    gerr = max(oracle.relerr(g["A"][:c["N"] - 1].double().cpu().numpy(), go["A"]),
               oracle.relerr(g["Qd"][:c["N"]].double().cpu().numpy(), go["Qd"]),
               oracle.relerr(g["c"][:c["N"]].double().cpu().numpy(), go["c"]))
    # looped single-instance forward + backward
    items = [LQTensors.from_numpy(it, device=dev) for it in batch.items]
    schs = [s.alloc_schur(it) for it in items]
    wss = [s.alloc_workspace(it) for it in items]
    ko = batch.knot_off

    def loop():
        for bi, it in enumerate(items):
            lam_i = torch.zeros(it.total, it.nx, device=dev)
            l_, dx_, du_, _, _ = s.solve(it, lam_i, opts=opts, schur=schs[bi])
            s.backward(it, schs[bi], l_, dx_, du_, w[ko[bi]:ko[bi + 1]], 2 * dx_, 2 * du_, opts=opts,
                       workspace=wss[bi])

    timed(loop)
    t_loop = float(np.median([timed(loop)[0] for _ in range(3)]))
    f, bw = float(np.median(fwd_ms)), float(np.median(bwd_ms))
    return {"workload": f"{c['B']} instances x N={c['N']} (nx={c['nx']}, nu={c['nu']}), loss sum ||dz||^2 + w^T lambda",
            "fwd_ms": f, "bwd_ms": bw, "bwd_over_fwd": bw / f, "loop_fwd_bwd_ms": t_loop,
            "speedup_vs_loop": t_loop / (f + bw), "converged": ok, "grad_relerr_vs_oracle": gerr,
            "pcg_roofline": {"bound": "sync_latency", "frac": (lat / (f + bw)) if lat else None,
                             "floor_ms": lat, "shape": sh,
                             "note": "forward + adjoint PCG iterations x 2 measured exchanges, spread over the "
                                     "co-resident clusters, over fwd + bwd time",
                             "hbm_equivalent_frac": alg / ((f + bw) / 1e3) / 1e9 / hbm, "peak_source": note}}


def _step_timer(s, stream):
    import torch

    class T:
        def __init__(self):
            self.ev = []

        def __call__(self, fn):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            self.ev.append((a, b))

        def ms(self):
            return [a.elapsed_time(b) for a, b in self.ev]
    return T()


def run_sweep(s, dev, reps, flush):
    """Latency sweep: single instances at N in {64, 128, 256, 512}, each
    solved `reps` times warm-started from its converged lambda perturbed
    (seed 2 + N, repetition r); one solve = the fused form_schur +
    form_precon, pcg_solve, recover_step, L2 flushed before each."""
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_SWEEP
    hbm, note = hbm_peak()
    stream = torch.cuda.current_stream(dev)
    out = {}
    for N in c["Ns"]:
        lq = gen.kuka_lq(c["nx"], c["nu"], N, c["seed_base"] + N, dt=c["dt"], qd=c["qd"]).astype(np.float32)
        lt = LQTensors.from_numpy(lq, device=dev)
        opts = make_opts(tol=1e-6)
        sch = s.alloc_schur(lt)
        lam_star, _, _, _, _ = s.solve(lt, opts=opts, schur=sch)
        ls = lam_star.cpu().double().numpy()
        lams = torch.as_tensor(np.stack([gen.warm_start(ls, c["seed_base"] + N, r) for r in range(reps)]),
                               dtype=torch.float32, device=dev)
        stats = s.alloc_stats(reps, dev)
        dx = torch.empty(N, c["nx"], device=dev)
        du = torch.empty(max(N - 1, 1), c["nu"], device=dev)
        tim, pcg = _step_timer(s, stream), _step_timer(s, stream)

        def one(r):
            s.form(lt, sch)
            pcg(lambda: s.pcg_solve(lt, sch, lams[r], opts, stats[r * 24:(r + 1) * 24]))
            s.recover_step(lt, lams[r], dx, du)

        for r in range(min(3, reps)):  # warm-up on copies
            w = lams[r].clone()
            s.form(lt, sch)
            s.pcg_solve(lt, sch, w, opts)
        torch.cuda.synchronize()
        for r in range(reps):
            flush.zero_()
            tim(lambda: one(r))
        torch.cuda.synchronize()
        st = read_stats(stats)
        us = np.array(tim.ms()) * 1e3
        pus = np.array(pcg.ms()) * 1e3
        it = st["iters"].astype(np.float64)
        ach = float(np.mean(it)) * N * pcg_bytes_per_knot_iter(c["nx"]) / (np.mean(pus) * 1e-6) / 1e9
        rl = latency_roofline(s, lt, sch, opts, float(np.mean(it)), float(np.median(pus)), rounds=1000)
        rl["hbm"] = {"achieved_gbs": ach, "frac": ach / hbm, "peak_source": note}
        out[str(N)] = {"us_per_solve": pct(us), "pcg_us": float(np.median(pus)),
                       "iters": pct(it), "converged": bool(np.all(st["status"] == 0)), "roofline": rl}
    return {"workload": f"single instances N in {list(c['Ns'])}, nx={c['nx']}, nu={c['nu']}, "
                        f"{reps} warm solves each (L2 flushed before each)", "per_N": out}


def run_exit_sweep(s, dev, reps):
    """The paper's exit test (absolute eta' = r^T Phi^-1 r < eps, Alg. 1) at
    eps in {1e-4, 5e-5, 1e-5}, beside the relative-residual default, at
    N = 128 on warm-started repeat solves: iteration and time
    distributions and the error each eps leaves against the oracle."""
    import torch
    import oracle
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_SWEEP
    N = 128
    lq = gen.kuka_lq(c["nx"], c["nu"], N, c["seed_base"] + N, dt=c["dt"], qd=c["qd"]).astype(np.float32)
    lo, _, _ = oracle.kkt_solve(lq.astype(np.float64))
    lt = LQTensors.from_numpy(lq, device=dev)
    sch = s.alloc_schur(lt)
    lam_star, _, _, _, _ = s.solve(lt, opts=make_opts(), schur=sch)
    ls = lam_star.cpu().double().numpy()
    lams0 = torch.as_tensor(np.stack([gen.warm_start(ls, c["seed_base"] + N, r) for r in range(reps)]),
                            dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, o in (("rel_1e-6", make_opts(tol=1e-6)),
                    ("abs_1e-4", make_opts(tol=1e-4, tol_mode=1)),
                    ("abs_5e-5", make_opts(tol=5e-5, tol_mode=1)),
                    ("abs_1e-5", make_opts(tol=1e-5, tol_mode=1))):
        lams = lams0.clone()
        stats = s.alloc_stats(reps, dev)
        s.pcg_solve(lt, sch, lams0[0].clone(), o)       # launch shape chosen outside timing
        torch.cuda.synchronize()
        tim = _step_timer(s, stream)
        for r in range(reps):
            tim(lambda: s.pcg_solve(lt, sch, lams[r], o, stats[r * 24:(r + 1) * 24]))
        torch.cuda.synchronize()
        st = read_stats(stats)
        errs = [oracle.relerr(lams[r].cpu().double().numpy(), lo) for r in range(0, reps, max(1, reps // 20))]
        out[name] = {"pcg_us": pct(np.array(tim.ms()) * 1e3), "iters": pct(st["iters"]),
                     "converged": bool(np.all(st["status"] == 0)),
                     "err_lambda_vs_oracle": pct(errs)}
    return {"workload": f"single instance N={N}, nx={c['nx']}, {reps} warm-started PCG solves per exit test",
            "per_exit": out}


def run_precon_compare(s, dev, reps):
    """The symmetric stair preconditioner of Sec. IV-A against block Jacobi
    (Phi^-1 = D^-1) on the sweep instances N = 128 and 512: warm-started PCG
    iterations and time, and the error each leaves against the oracle; and
    the non-symmetric stair preconditioner (one capped cold solve: PCG has
    no convergence guarantee with it)."""
    import torch
    import oracle
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_SWEEP
    stream = torch.cuda.current_stream(dev)
    out = {}
    for N in (128, 512):
        lq = gen.kuka_lq(c["nx"], c["nu"], N, c["seed_base"] + N, dt=c["dt"], qd=c["qd"]).astype(np.float32)
        lo, _, _ = oracle.kkt_solve(lq.astype(np.float64))
        lt = LQTensors.from_numpy(lq, device=dev)
        sch = s.alloc_schur(lt)
        lam_star, _, _, _, _ = s.solve(lt, opts=make_opts(), schur=sch)
        ls = lam_star.cpu().double().numpy()
        lams0 = torch.as_tensor(np.stack([gen.warm_start(ls, c["seed_base"] + N, r) for r in range(reps)]),
                                dtype=torch.float32, device=dev)
        for name, pc in (("symmetric_stair", 0), ("block_jacobi", 1)):
            o = make_opts(tol=1e-6, precon=pc)
            cold = s.alloc_stats(1, dev)
            s.pcg_solve(lt, sch, torch.zeros_like(lams0[0]), o, cold)
            lams = lams0.clone()
            stats = s.alloc_stats(reps, dev)
            s.pcg_solve(lt, sch, lams0[0].clone(), o)
            torch.cuda.synchronize()
            tim = _step_timer(s, stream)
            for r in range(reps):
                tim(lambda: s.pcg_solve(lt, sch, lams[r], o, stats[r * 24:(r + 1) * 24]))
            torch.cuda.synchronize()
            st = read_stats(stats)
            out[f"N{N}_{name}"] = {"pcg_us": pct(np.array(tim.ms()) * 1e3), "iters": pct(st["iters"]),
                                   "cold_iters": int(read_stats(cold)["iters"][0]),
                                   "converged": bool(np.all(st["status"] == 0)),
                                   "err_lambda_vs_oracle": oracle.relerr(lams[reps - 1].cpu().double().numpy(), lo)}
        # the non-symmetric stair preconditioner: one cold solve, capped
        cap = 5000
        lam = torch.zeros_like(lams0[0])
        st = read_stats(s.pcg_solve(lt, sch, lam, make_opts(tol=1e-6, precon=2, max_iter=cap)))
        out[f"N{N}_nonsymmetric_stair"] = {"cold_iters": int(st["iters"][0]), "max_iter": cap,
                                           "converged": bool(st["status"][0] == 0),
                                           "relres_at_exit": float(st["relres"][0]),
                                           "err_lambda_vs_oracle": oracle.relerr(lam.cpu().double().numpy(), lo)}
    return {"workload": f"single instances N in (128, 512), nx={c['nx']}, {reps} warm-started PCG solves "
                        f"per preconditioner, rel. residual 1e-6; the non-symmetric stair preconditioner "
                        f"one cold solve capped at 5000 iterations", "per_case": out}


def run_dense_cost(s, dev, reps):
    """General SPD cost blocks Q_k, R_k (dense) against the diagonal costs of
    the same instances, N = 128 and 512: µs per whole solve, the formation
    share, iterations, error against the oracle."""
    import torch
    import oracle
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_SWEEP
    stream = torch.cuda.current_stream(dev)
    out = {}
    for N in (128, 512):
        for name, dense in (("diagonal", False), ("dense", True)):
            lq = gen.kuka_lq(c["nx"], c["nu"], N, c["seed_base"] + N, dt=c["dt"], qd=c["qd"],
                             dense=dense).astype(np.float32)
            lo, xo, uo = oracle.kkt_solve(lq.astype(np.float64))
            lt = LQTensors.from_numpy(lq, device=dev)
            sch = s.alloc_schur(lt)
            o = make_opts(tol=1e-6)
            lam = torch.zeros(N, c["nx"], device=dev)
            dx = torch.empty(N, c["nx"], device=dev)
            du = torch.empty(max(N - 1, 1), c["nu"], device=dev)
            st = s.alloc_stats(1, dev)
            s.solve(lt, lam.clone(), opts=o, schur=sch)
            torch.cuda.synchronize()
            tim, frm = _step_timer(s, stream), _step_timer(s, stream)

            def one():
                lam.zero_()
                frm(lambda: s.form(lt, sch))
                s.pcg_solve(lt, sch, lam, o, st)
                s.recover_step(lt, lam, dx, du)

            for _ in range(reps):
                tim(one)
            torch.cuda.synchronize()
            e_lam = oracle.relerr(lam.cpu().double().numpy(), lo)
            e_dz = oracle.relerr(np.concatenate([dx.cpu().double().numpy().ravel(),
                                                 du[:N - 1].cpu().double().numpy().ravel()]),
                                 np.concatenate([xo.ravel(), uo.ravel()]))
            out[f"N{N}_{name}"] = {"us_per_solve": pct(np.array(tim.ms()) * 1e3),
                                   "form_us": float(np.median(frm.ms())) * 1e3,
                                   "iters": int(read_stats(st)["iters"][0]),
                                   "converged": bool(read_stats(st)["status"][0] == 0),
                                   "err_lambda": e_lam, "err_dz": e_dz}
    return {"workload": f"single instances N in (128, 512), nx={c['nx']}, cold solves, "
                        f"diagonal vs dense SPD cost blocks (same A, B, q, r, c)", "per_case": out}


def run_nmpc(s, dev, reps):
    """SQP outer loop on the device (Sec. II-A Steps 1-3, Sec. IV-C) on the
    synthetic Kuka-shaped model: one replay = reset to the straight-line
    initial guess, then 8 SQP iterations (linearise, form, precondition,
    warm-started PCG, recover, 9-step parallel line search) captured in one
    CUDA graph.  N = 128 and 512; PCG exit at relative residual 1e-6 and at
    the paper's absolute eta' < 1e-4 (Alg. 1)."""
    import torch
    import oracle
    from oracle import nmpc as onmpc
    from paper_2309_08079_gb300.nmpc import SQP
    from paper_2309_08079_gb300.solver import make_opts, read_stats
    c = gen.CONFIG_NMPC
    m = gen.nmpc_model(c["nx"], c["nu"], c["model_seed"], dt=c["dt"]).astype(np.float32)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for (N, exit_name, o) in [(N, e, o) for N in c["Ns"] for e, o in
                              (("rel_1e-6", make_opts(tol=1e-6)),
                               ("paper_abs_1e-4", make_opts(tol=1e-4, tol_mode=1)))]:
        t = gen.nmpc_tracking(m, N, c["seed_base"] + N).astype(np.float32)
        q = SQP(s, m, t, device=dev, opts=o, n_alpha=c["n_alpha"])
        X0, U0 = q.X.clone(), q.U.clone()

        def reset():
            q.X.copy_(X0)
            q.U.copy_(U0)
            q.lam.zero_()

        q.step()  # launch shapes chosen outside the capture
        reset()
        g = q.graph(c["sqp_iters"])
        tim = _step_timer(s, stream)
        for _ in range(reps + 1):
            reset()
            tim(g.replay)
        torch.cuda.synchronize()
        ms = tim.ms()[1:]
        hist = onmpc.sqp(m, t, c["sqp_iters"])
        X = q.X.cpu().double().numpy()
        per_it = float(np.median(ms)) * 1e3 / c["sqp_iters"]
        out[f"N{N}_{exit_name}"] = {"us_per_sqp_iteration": per_it, "sqp_iterations_per_s": 1e6 / per_it,
                        "replay_ms": pct(ms), "err_X_vs_oracle_sqp": oracle.relerr(X, hist[-1]["X"]),
                        "final_defect_max": float(np.abs(onmpc.defects(m, t, X, q.U.cpu().double().numpy())).max()),
                        "last_pcg_iters": int(read_stats(q.stats)["iters"][0])}
    return {"workload": f"synthetic Kuka-shaped model nx={c['nx']}, nu={c['nu']}, {c['sqp_iters']} SQP "
                        f"iterations per replay from the initial guess, {c['n_alpha']} step sizes",
            "per_N": out,
            "paper_context": "MPCGPU on an RTX 4090 with the Kuka dynamics: 4 kHz per iteration at N=128, "
                             "1 kHz control at N=512 (not this model)"}


def run_large(s, dev, solves, B=None, refine_tol=1e-2):
    """Large-state batch: nx = 36, nu = 12, 1024 instances with
    N_i ~ U{64..256}, dt = 0.005, Qd ~ U[0.1, 100].  One step = `solves`
    warm-started forward solves (each with one refinement step) through the
    autograd Function and the backward of loss sum ||dz||^2 + w^T lambda over
    all of them (each adjoint solve with one refinement step too).  The PCG launch plan comes from the autotuner (single-launch
    plans, so the same launch serves refinement and the adjoint solve)."""
    import torch
    import oracle
    from paper_2309_08079_gb300.autograd import MPCGSolve
    from paper_2309_08079_gb300.autotune import Autotuner, PlanRunner
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    c = gen.CONFIG_LARGE
    Ns = gen.batch_horizons(c["B"], c["N_lo"], c["N_hi"], c["n_seed"])[:B or c["B"]]
    batch = gen.kuka_batch(c["nx"], c["nu"], Ns, c["seed_base"], dt=c["dt"], qd=c["qd"]).astype(np.float32)
    lt = LQTensors.from_batch(batch, device=dev)
    base = make_opts(tol=1e-6)
    sch = s.alloc_schur(lt)
    ws = s.alloc_workspace(lt)
    s.form(lt, sch)
    zero = torch.zeros(lt.total, lt.nx, device=dev)
    with tempfile.TemporaryDirectory() as td:
        tuner = Autotuner(s, cache_path=os.path.join(td, "tune.json"), reps=1)
        best = tuner.tune(lt, sch, zero, base, only=("single_auto", "single_cta_l2", "single_cta_tma"))
    runner = PlanRunner(s, lt, best["groups"], base)  # owns the instance list opts points at
    opts = runner.launches[0].opts
    # refinement's correction solves stop at relative residual refine_tol
    # (1e-2): the correction only shrinks an error already at the float32
    # floor of S+ (~1e-3 here); measured on this batch, lambda and gradient
    # errors 1.6e-5 / 4.8e-5 at 1e-2 against 1.1e-5 / 2.7e-5 at 1e-3, for
    # 17 % less time per step (3e-2 reaches 4.7e-5 / 9.1e-5: too close to
    # the 1e-4 bar)
    opts.refine_tol = refine_tol
    t0 = time.perf_counter()
    lam_star, _, _, st0, _ = s.solve(lt, zero.clone(), opts=opts, schur=sch, workspace=ws, refine=1)
    ls = lam_star.cpu().double().numpy()
    ko = batch.knot_off
    lam0 = [torch.as_tensor(np.concatenate([gen.warm_start(ls[ko[b]:ko[b + 1]], c["seed_base"] + b, r)
                                            for b in range(batch.B)]), dtype=torch.float32, device=dev)
            for r in range(solves)]
    K = lt.total
    w = torch.as_tensor(gen.loss_weights(K * c["nx"], c["seed_base"]).reshape(K, c["nx"]),
                        dtype=torch.float32, device=dev)
    leaves = {f: getattr(lt, f).clone().requires_grad_(True) for f in LQTensors.FIELDS}
    cfg = dict(solver=s, nx=lt.nx, nu=lt.nu, N=lt.N, knot_off=lt.knot_off, nb=lt.nb, total=K,
               opts=opts, workspace=ws, refine=1)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    outs, loss = [], 0.0
    for r in range(solves):
        lam, dx, du, st = MPCGSolve.apply(*(leaves[f] for f in LQTensors.FIELDS), lam0[r], cfg)
        outs.append((lam, dx, du, st))
        loss = loss + (dx * dx).sum() + (du * du).sum() + (w * lam).sum()
    ev[1].record(stream)
    loss.backward()
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    sts = np.concatenate([read_stats(o[3]) for o in outs])
    # per-instance error of the last solve against the FP64 oracle, on a sample
    lam_l = outs[-1][0].detach().cpu().double().numpy()
    picks = sorted({int(np.argmin(Ns)), int(np.argmax(Ns))} | set(range(0, batch.B, 128)))
    errs = {int(b): oracle.relerr(lam_l[ko[b]:ko[b + 1]], oracle.kkt_solve(batch.items[b].astype(np.float64))[0])
            for b in picks}
    # gradient of the summed loss w.r.t. each sampled instance's inputs against
    # the oracle's analytic gradient (field by field, max over fields); the
    # loss terms of the `solves` solves add, and every solve reaches the same
    # (lambda, dz) up to the solve's error, so the oracle gradient is
    # `solves` times the one-solve gradient
    co = batch.ctrl_off()
    gerrs = {}
    for b in picks[:4]:
        it64 = batch.items[b].astype(np.float64)
        lo_, xo_, uo_ = oracle.kkt_solve(it64)
        go = oracle.grad(it64, lo_, xo_, uo_, w[ko[b]:ko[b + 1]].double().cpu().numpy(), 2 * xo_, 2 * uo_)
        e = 0.0
        for f in LQTensors.FIELDS:
            sl = slice(co[b], co[b + 1]) if f in ("A", "B", "Rd", "r") else slice(ko[b], ko[b + 1])
            gf = leaves[f].grad[sl].double().cpu().numpy()
            e = max(e, oracle.relerr(gf, solves * go[f]))
        gerrs[int(b)] = e
    n = batch.B * solves
    hbm, note = hbm_peak()
    it = sts["iters"].astype(np.float64)
    Nrep = np.tile(Ns, solves)
    alg = float(np.sum(it * Nrep)) * pcg_bytes_per_knot_iter(c["nx"])
    # the PCG kernel alone: one warm-started solve of the batch timed by
    # itself, against the algorithmic bytes (symmetric diagonal blocks) and
    # against the bytes the tiled kernel streams (full diagonal and
    # off-diagonal tiles, two passes per iteration)
    lam1 = lam0[0].clone()
    st1 = s.alloc_stats(batch.B, dev)
    s.pcg_solve(lt, sch, lam0[0].clone(), opts, st1, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.pcg_solve(lt, sch, lam1, opts, st1, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    pcg_ms = e0.elapsed_time(e1)
    it1 = read_stats(st1)["iters"].astype(np.float64)
    # the same solve with the dot products accumulated in float64
    # (mpcg_opts.dot = 1), the precision the workload names
    from paper_2309_08079_gb300 import _lib as L
    o64 = L.mpcg_opts.from_buffer_copy(opts)
    o64.dot = 1
    st64 = s.alloc_stats(batch.B, dev)
    s.pcg_solve(lt, sch, lam0[0].clone(), o64, st64, ws)
    torch.cuda.synchronize()
    lam64 = lam0[0].clone()
    e0.record(stream)
    s.pcg_solve(lt, sch, lam64, o64, st64, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    pcg64_ms = e0.elapsed_time(e1)
    it64 = read_stats(st64)["iters"].astype(np.float64)
    ok64 = bool(np.all(read_stats(st64)["status"] == 0))
    ki = float(np.sum(it1 * Ns))
    alg1 = ki * pcg_bytes_per_knot_iter(c["nx"])
    # bytes the tiled kernel copies per knot and pass: the diagonal block
    # (packed upper triangle when the launch streams it) and O_k
    sh1 = s.pcg_shape(lt, sch, opts)
    nx_ = c["nx"]
    dwords = ((nx_ * (nx_ + 1) // 2 + 3) // 4 * 4) if sh1.get("packed") else nx_ * nx_
    streamed1 = ki * 2 * (dwords + nx_ * nx_) * 4
    pcg_alone = {"bound": "hbm", "pcg_ms": pcg_ms, "plan": best["plan"],
                 "achieved": alg1 / (pcg_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                 "frac": alg1 / (pcg_ms / 1e3) / 1e9 / hbm, "peak_source": note,
                 "streamed_gbs": streamed1 / (pcg_ms / 1e3) / 1e9,
                 "streamed_frac": streamed1 / (pcg_ms / 1e3) / 1e9 / hbm,
                 "shape": sh1,
                 "note": "one warm-started PCG solve of the whole batch timed alone; achieved = algorithmic "
                         "bytes (symmetric diagonal blocks, (2T + 7 nx) x 4 B per knot-iteration); streamed = "
                         "the tiles the kernel copies (diagonal block, packed when shape.packed, and "
                         "off-diagonal block per knot and pass)"}
    return {"workload": f"{batch.B} instances, nx={c['nx']}, nu={c['nu']}, N_i ~ U{{{c['N_lo']}..{c['N_hi']}}} "
                        f"(sum {int(ko[-1])} knots), {solves} warm solves per step + backward, one refinement "
                        f"step after the forward and after the adjoint solve (corrections to {refine_tol:g})",
            "plan": best["plan"], "tune_ms": {k: round(v, 2) for k, v in tuner.last_timings.items()},
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "solves_per_s_fwd": n / (fwd_ms / 1e3),
            "solves_per_s_fwd_bwd": n / ((fwd_ms + bwd_ms) / 1e3),
            "iters_first_pcg": pct(it), "converged": bool(np.all(sts["status"] == 0)),
            "err_lambda_vs_oracle": {"max": max(errs.values()), "instances": len(errs)},
            "grad_err_vs_oracle": {"max": max(gerrs.values()), "per_instance": gerrs,
                                   "note": "every gradient field against the oracle's analytic gradient "
                                           "(normwise per field, max over fields); forward and adjoint "
                                           "solves each with one refinement step"},
            "pcg_roofline": pcg_alone,
            "dot_fp64": {"pcg_ms": pcg64_ms, "default_pcg_ms": pcg_ms, "iters_mean": float(np.mean(it64)),
                         "default_iters_mean": float(np.mean(it1)), "converged": ok64,
                         "note": "the same warm-started batch PCG solve with float64-accumulated dot products "
                                 "(mpcg_opts.dot = 1) in the tiled kernel"},
            "pcg_roofline_fwd": {"bound": "hbm", "note": "first PCG of each solve only, over the whole forward "
                                                         "time (formation, both PCG solves of the refinement, "
                                                         "recovery)",
                                 "achieved_gbs": alg / (fwd_ms / 1e3) / 1e9,
                                 "frac": alg / (fwd_ms / 1e3) / 1e9 / hbm, "peak_source": note},
            "wall_s": time.perf_counter() - t0}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
