"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the byte
counts per knot-iteration, the summary at the end of the JSON line and the
config object both arms share."""
import numpy as np
import pytest

import bench


class _FakeSolver:
    """Stands in for Solver: a fixed launch shape and exchange time."""

    def __init__(self, form="cluster", C=16, threads=256, ns=650.0):
        self.shape = {"form": form, "C": C, "clusters": 1, "threads": threads}
        self.ns = ns
        self.calls = []

    def pcg_shape(self, lt, sch, opts=None):
        return dict(self.shape)

    def bench_exchange(self, C, W, rounds=2000):
        self.calls.append((C, W, rounds))
        return {"ns": self.ns, "cycles": self.ns * 2.07, "C": C, "W": W, "rounds": rounds}


def test_latency_roofline_is_two_exchanges_per_iteration():
    s = _FakeSolver(ns=650.0)
    r = bench.latency_roofline(s, None, None, None, iters_mean=700.0, launch_us=1624.0)
    t_it = 1624.0 * 1e3 / 700.0
    assert r["bound"] == "sync_latency" and r["unit"] == "PCG iterations/s"
    assert r["floor_ns_per_iteration"] == pytest.approx(1300.0)
    assert r["frac"] == pytest.approx(1300.0 / t_it)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    # measured on the solve's own launch shape: 16 CTAs x 256 threads = 8 warps
    assert s.calls == [(16, 8, 2000)]


def test_latency_roofline_only_for_the_cluster_kernel():
    r = bench.latency_roofline(_FakeSolver(form="cta_tma"), None, None, None, 100.0, 1000.0)
    assert r["bound"] == "n/a"


def test_bytes_per_knot_iteration():
    # both symmetric block-tridiagonal matrices once (T words each) and 7 vectors
    assert bench.pcg_bytes_per_knot_iter(14) == (2 * (14 * 15 // 2 + 196) + 7 * 14) * 4 == 2800
    assert bench.pcg_bytes_per_knot_iter(36, 8) == (2 * (36 * 37 // 2 + 1296) + 7 * 36) * 8


def test_both_arms_share_the_config():
    a, b = bench.workload_config(1), bench.workload_config(1)
    assert a == b and "N=512" in a["workload"] and a["seed"] == bench.SEED
    assert "flushed" in a["l2"]
    assert bench.workload_config(4)["parallelism"] == "replicas"


def test_summary_collects_the_secondary_figures_last():
    line = {"value": 1650.0, "e2e": {"value": 1665.0}, "step_breakdown_us": {"pcg": 1624.0},
            "pcg_iters": {"mean": 728.0}, "roofline": {"frac": 0.59, "hbm": {"frac": 0.096}},
            "parity": {"err_lambda": 4e-5, "err_dz": 3e-5},
            "batched": {"solves_per_s": 8500.0, "loop_solves_per_s": 850.0, "speedup_vs_loop": 10.0},
            "backward": None, "large_state": {"pcg_roofline": {"frac": 0.64, "streamed_frac": 0.8}},
            "sweep": {"per_N": {"64": {"us_per_solve": {"p50": 410.0}}}}, "dot_fp64": {"pcg_us": 3770.0}}
    s = bench.summarize(line)
    assert s["us_per_solve_N512"] == 1650.0 and s["sync_latency_frac"] == 0.59
    assert s["hbm_frac"] == 0.096 and s["batched_solves_per_s"] == 8500.0
    assert s["backward_fwd_ms"] is None  # missing sections read as None
    assert s["large_pcg_streamed_frac"] == 0.8 and s["sweep_p50_us"] == {"64": 410.0}
    line["summary"] = s
    assert list(line)[-1] == "summary"


def test_percentiles():
    p = bench.pct(np.arange(1, 11, dtype=float))
    assert p["p50"] == pytest.approx(5.5) and p["max"] == 10.0 and p["p10"] < p["p90"]
