"""Launch-plan autotuner for the batched PCG solve.

A ragged batch can be solved in several ways that reach the same answer to
the solver tolerance but take different times:

* one persistent launch of the cluster kernel, with the cluster size the
  LONGEST horizon needs, so every instance occupies that many SMs;
* one persistent launch of a CTA-per-instance kernel (blocks read from L2,
  or TMA-staged through shared memory), with no cross-SM exchange;
* one launch per horizon class, each sized for its own class (a short
  instance gets a small cluster, or a single CTA), the launches running at
  once on their own streams.

Every plan orders each launch's instance queue by decreasing horizon, so the
longest solves start first and the tail of a persistent launch is short.

The tuner times each candidate plan on the caller's batch with CUDA events,
keeps the fastest one whose solves all reach the status of the reference
plan, and stores the choice in a JSON file keyed by the device, the element
type, nx, the batch size and the histogram of horizons over power-of-two
classes, so a later process with a batch of the same shape reuses it.  The
choice only changes launch geometry: each instance's arithmetic is the same
algorithm under every plan.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np
import torch

from . import _lib as L
from .solver import LQTensors, SchurTensors, Solver, make_opts

INF = 1 << 30
# workspace bytes one batched PCG launch uses (its instance queue)
QUEUE_BYTES = 256


def horizon_classes(Ns: np.ndarray) -> List[int]:
    """Upper edges of the power-of-two horizon classes the batch occupies:
    class e holds horizons in (e/2, e] (the first one (0, e])."""
    edges = sorted({1 << max(0, math.ceil(math.log2(int(n)))) for n in Ns})
    return edges


def histogram_key(Ns: np.ndarray) -> str:
    """Counts of instances per power-of-two horizon class, e.g. '32:5,64:12'."""
    e = np.array([1 << max(0, math.ceil(math.log2(int(n)))) for n in Ns])
    vals, cnt = np.unique(e, return_counts=True)
    return ",".join(f"{v}:{c}" for v, c in zip(vals.tolist(), cnt.tolist()))


def candidate_plans(Ns: np.ndarray) -> Dict[str, List[dict]]:
    """Plans to time.  A plan is a list of groups {lo, hi, mode, cluster}:
    the instances with lo < N_b <= hi, launched with opts.mode / opts.cluster
    (mode 0 = the library's automatic choice, cluster 0 = the size the
    group's longest horizon needs)."""
    edges = horizon_classes(Ns)
    one = lambda mode: [{"lo": 0, "hi": INF, "mode": mode, "cluster": 0}]
    plans = {"single_auto": one(0), "single_cta_l2": one(2), "single_cta_tma": one(3),
             "single_wide": one(4)}
    if len(edges) > 1:
        lo = [0] + edges[:-1]
        plans["classes_auto"] = [{"lo": a, "hi": b, "mode": 0, "cluster": 0}
                                 for a, b in zip(lo, edges)]
        # the shortest classes (a quarter of the longest horizon or less) on
        # the CTA-per-instance kernel, the rest on clusters
        cut = edges[-1] // 4
        short = [{"lo": 0, "hi": cut, "mode": 2, "cluster": 0}] if edges[0] <= cut else []
        plans["classes_cta_short"] = short + [
            {"lo": max(a, cut) if short else a, "hi": b, "mode": 0, "cluster": 0}
            for a, b in zip(lo, edges) if b > cut]
        if short:
            plans["classes_tile_short"] = [dict(short[0], mode=3)] + plans["classes_cta_short"][1:]
        # per-class launches of the CTA-per-instance kernels (each class's
        # shared vectors sized for its own longest horizon)
        plans["classes_cta_l2"] = [{"lo": a, "hi": b, "mode": 2, "cluster": 0}
                                   for a, b in zip(lo, edges)]
        plans["classes_tile"] = [{"lo": a, "hi": b, "mode": 3, "cluster": 0}
                                 for a, b in zip(lo, edges)]
        plans["classes_wide"] = [{"lo": a, "hi": b, "mode": 4, "cluster": 0}
                                 for a, b in zip(lo, edges)]
        # finer knots-per-CTA tiling: clusters of ceil(hi / kpc) CTAs holding
        # kpc knots each, so a smaller CTA shares its SM with another
        # instance's CTA (classes whose cluster would exceed 16 keep the
        # library's choice)
        for kpc in (16, 8):
            plans[f"classes_kpc{kpc}"] = [
                {"lo": a, "hi": b, "mode": 0,
                 "cluster": -(-b // kpc) if -(-b // kpc) <= 16 else 0}
                for a, b in zip(lo, edges)]
        # groups of equal cluster size: horizons in 32- (64-) knot steps, so
        # each instance gets the ceil(N / 32) CTAs it needs instead of its
        # power-of-two class's (an N = 260 instance takes 9 CTAs, not 16);
        # mixed cluster sizes on concurrent streams also fill the GPCs that
        # 16-CTA clusters leave partly idle
        for step in (32, 64, 96, 128, 192):
            top = -(-int(np.max(Ns)) // step) * step
            bounds = list(range(step, top + 1, step))
            plans[f"steps{step}_auto"] = [{"lo": b - step, "hi": b, "mode": 0, "cluster": 0}
                                          for b in bounds]
        # the same, the short horizons (a quarter of the longest class or
        # less) on the tiled CTA-per-instance kernel
        if edges[-1] >= 256:
            cut = edges[-1] // 4
            for step in (32, 64):
                top = max(cut, -(-int(np.max(Ns)) // step) * step)
                plans[f"steps{step}_tile_short"] = [{"lo": 0, "hi": cut, "mode": 3, "cluster": 0}] + [
                    {"lo": b - step, "hi": b, "mode": 0, "cluster": 0}
                    for b in range(cut + step, top + 1, step)]
        # two halves of the horizon range
        mid = edges[-1] // 2
        if edges[0] <= mid:
            plans["halves_auto"] = [{"lo": 0, "hi": mid, "mode": 0, "cluster": 0},
                                    {"lo": mid, "hi": INF, "mode": 0, "cluster": 0}]
    return plans


def group_instances(Ns: np.ndarray, plan: List[dict]):
    """[(group, indices)] for the plan's non-empty groups, each group's
    instances ordered longest first; raises unless every instance falls in
    exactly one group."""
    Ns = np.asarray(Ns)
    out, seen = [], np.zeros(len(Ns), dtype=np.int64)
    for g in plan:
        idx = np.nonzero((Ns > g["lo"]) & (Ns <= g["hi"]))[0]
        seen[idx] += 1
        if len(idx):
            out.append((g, idx[np.argsort(-Ns[idx], kind="stable")]))
    if not np.all(seen == 1):
        raise ValueError("plan groups do not cover every instance exactly once")
    return out


@dataclass
class _Launch:
    opts: object          # mpcg_opts (holds the instance list's pointer)
    N: int                # longest horizon in the group
    inst: torch.Tensor    # int32 instance indices, longest first
    ws: torch.Tensor      # this launch's 256-byte queue


class PlanRunner:
    """Executes one plan on one batch: fixed instance lists, streams and
    queues, so its launches can be captured in a CUDA graph."""

    def __init__(self, solver: Solver, lq: LQTensors, plan: List[dict], base_opts=None):
        if not lq.batched or lq.Ns is None:
            raise ValueError("a plan needs a batched LQTensors with host horizons")
        self.solver, self.lq, self.plan = solver, lq, plan
        b = base_opts if base_opts is not None else make_opts()
        Ns = np.asarray(lq.Ns)
        # launch the groups longest horizon first: the long solves start at
        # once and the short groups fill the SMs behind them (measured on the
        # 256-instance batch: 30.1 vs 32.1 ms per solve for 64-knot steps)
        groups = sorted(group_instances(Ns, plan), key=lambda gi: -int(Ns[gi[1]].max()))
        self.ws = torch.zeros(QUEUE_BYTES * len(groups), dtype=torch.uint8, device=lq.device)
        self.launches: List[_Launch] = []
        for j, (g, idx) in enumerate(groups):
            inst = torch.as_tensor(idx.astype(np.int32), device=lq.device)
            o = make_opts(tol=b.tol, tol_mode=b.tol_mode, max_iter=b.max_iter,
                          cluster=g["cluster"], mode=g["mode"], instances=inst, precon=b.precon)
            self.launches.append(_Launch(o, int(Ns[idx].max()), inst,
                                         self.ws[QUEUE_BYTES * j:QUEUE_BYTES * (j + 1)]))
        self.streams = [torch.cuda.Stream(lq.device) for _ in self.launches[1:]]

    def pcg_solve(self, schur: SchurTensors, lam: torch.Tensor, stats: torch.Tensor,
                  stream: Optional[torch.cuda.Stream] = None):
        """Solve every instance in place (lam holds the warm starts); the
        launches fork from and join back into `stream` (default: current)."""
        main = stream if stream is not None else torch.cuda.current_stream(self.lq.device)
        for s in self.streams:          # fork every side stream before any launch
            s.wait_stream(main)
        for j, l in enumerate(self.launches):
            st = main if j == 0 else self.streams[j - 1]
            self.solver.pcg_solve(self.lq, schur, lam, l.opts, stats, l.ws, stream=st, N=l.N)
        for s in self.streams:
            main.wait_stream(s)
        return stats


def _default_cache() -> str:
    return os.environ.get("MPCG_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mpcg_gb300",
                                       "autotune.json"))


class Autotuner:
    """Chooses, times and caches the launch plan of batched PCG solves."""

    def __init__(self, solver: Solver, cache_path: Optional[str] = None, reps: int = 5,
                 graph: bool = False):
        """graph=True times each plan captured in a CUDA graph (for callers
        that replay graphs: concurrent branches of a graph have no launch
        order, so a plan's longest-first start is not kept there)."""
        self.solver = solver
        self.graph = bool(graph)
        self.cache_path = cache_path if cache_path is not None else _default_cache()
        self.reps = max(1, int(reps))
        self.last_timings: Dict[str, float] = {}

    # ---------------------------------------------------------------- cache
    def key(self, lq: LQTensors) -> str:
        p = torch.cuda.get_device_properties(lq.device)
        dt = {torch.float32: "f32", torch.float64: "f64"}[lq.dtype]
        return (f"{p.name}|sm{p.multi_processor_count}|{dt}|nx{lq.nx}|nu{lq.nu}|B{lq.nb}|"
                f"{histogram_key(lq.Ns)}" + ("|graph" if self.graph else ""))

    def _load(self) -> dict:
        try:
            with open(self.cache_path) as f:
                d = json.load(f)
            return d if isinstance(d, dict) else {}
        except (OSError, ValueError):
            return {}

    def _store(self, key: str, entry: dict) -> None:
        d = self._load()
        d[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(self.cache_path)))
        with os.fdopen(fd, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def cached_plan(self, lq: LQTensors) -> Optional[dict]:
        return self._load().get(self.key(lq))

    # ---------------------------------------------------------------- tuning
    def _time(self, runner: PlanRunner, schur, lam0, lam, stats) -> float:
        if self.graph:
            return self._time_graph(runner, schur, lam0, lam, stats)
        times = []
        for r in range(self.reps + 1):
            lam.copy_(lam0)
            torch.cuda.synchronize(lam.device)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            runner.pcg_solve(schur, lam, stats)
            b.record()
            b.synchronize()
            if r:  # the first run chooses launch shapes
                times.append(a.elapsed_time(b))
        return float(np.median(times))

    def _time_graph(self, runner: PlanRunner, schur, lam0, lam, stats) -> float:
        dev = lam.device
        lam.copy_(lam0)
        runner.pcg_solve(schur, lam, stats)  # chooses launch shapes outside the capture
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                lam.copy_(lam0)
                runner.pcg_solve(schur, lam, stats)
        torch.cuda.current_stream(dev).wait_stream(side)
        times = []
        for r in range(self.reps + 1):
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            b.synchronize()
            if r:
                times.append(a.elapsed_time(b))
        del g
        return float(np.median(times))

    def tune(self, lq: LQTensors, schur: SchurTensors, lam0: torch.Tensor, opts=None,
             store: bool = True, only=None) -> dict:
        """Times every candidate plan (or those named in `only`) on this batch
        (schur formed, lam0 the warm starts; neither is changed) and returns
        the fastest entry {"plan": name, "groups": [...], "ms": t}."""
        from .solver import read_stats
        lam = torch.empty_like(lam0)
        stats = self.solver.alloc_stats(lq.nb, lq.device)
        ref_status = None
        best = None
        self.last_timings = {}
        for name, groups in candidate_plans(lq.Ns).items():
            if only is not None and name not in only:
                continue
            try:
                runner = PlanRunner(self.solver, lq, groups, opts)
                t = self._time(runner, schur, lam0, lam, stats)
            except L.MPCGError as e:  # a shape this plan cannot launch
                if e.code != L.MPCG_EUNSUPPORTED:
                    raise
                continue
            st = read_stats(stats)["status"].copy()
            if ref_status is None:
                ref_status = st
            elif not np.array_equal(st, ref_status):
                continue
            self.last_timings[name] = t
            if best is None or t < best["ms"]:
                best = {"plan": name, "groups": groups, "ms": t}
        if best is None:
            raise RuntimeError("no launch plan could solve this batch")
        if store:
            self._store(self.key(lq), best)
        return best

    def runner(self, lq: LQTensors, schur: SchurTensors, lam0: torch.Tensor, opts=None,
               retune: bool = False) -> PlanRunner:
        """The PlanRunner of the cached plan for this batch's shape, tuning
        (and caching) first when there is none."""
        entry = None if retune else self.cached_plan(lq)
        if entry is None:
            entry = self.tune(lq, schur, lam0, opts)
        return PlanRunner(self.solver, lq, entry["groups"], opts)
