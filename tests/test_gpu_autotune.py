"""Instance lists in batched PCG, the launch plans built on them, and the
autotuner that picks among the plans: every plan solves every instance to
the parity bar against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, TOL_KNOT_F32, knot_err, solver
from workload import gen

pytestmark = pytest.mark.gpu

NS = [3, 17, 40, 64, 100, 200, 300, 512, 33, 1]


def _setup(Ns, seed, lam0=None):
    import torch
    from paper_2309_08079_gb300.solver import LQTensors
    s = solver()
    batch = gen.kuka_batch(14, 7, Ns, seed).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    sch = s.alloc_schur(lt)
    s.form_schur(lt, sch)
    s.form_precon(lt, sch)
    lam = (torch.zeros(lt.total, lt.nx, device="cuda") if lam0 is None
           else torch.as_tensor(lam0, dtype=torch.float32, device="cuda").clone())
    return s, batch, lt, sch, lam


def _oracle_lams(batch):
    return [oracle.kkt_solve(it.astype(np.float64))[0] for it in batch.items]


def _check_lam(batch, lam, st, los, which=None):
    ko = batch.knot_off
    for b in (range(batch.B) if which is None else which):
        assert st["status"][b] == 0, (b, st[b])
        e = oracle.relerr(lam[ko[b]:ko[b + 1]], los[b])
        assert e < TOL_F32, (b, batch.items[b].N, e)
        ek = knot_err(lam[ko[b]:ko[b + 1]], los[b])
        assert ek < TOL_KNOT_F32, (b, batch.items[b].N, ek)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_instance_list_solves_only_the_listed_instances(mode):
    import torch
    from paper_2309_08079_gb300.solver import make_opts, read_stats
    s, batch, lt, sch, lam = _setup(NS, 4100)
    los = _oracle_lams(batch)
    pick = [7, 2, 5, 9]
    inst = torch.tensor(pick, dtype=torch.int32, device="cuda")
    stats = s.alloc_stats(batch.B)
    stats.fill_(0xFF)                              # status -1 marks "not written"
    lam.fill_(7.0)
    for b in pick:                                 # cold start for the listed ones
        lam[batch.knot_off[b]:batch.knot_off[b + 1]] = 0.0
    N = max(NS[b] for b in pick)
    s.pcg_solve(lt, sch, lam, make_opts(mode=mode, instances=inst), stats, N=N)
    torch.cuda.synchronize()
    st = read_stats(stats)
    out = lam.cpu().double().numpy()
    _check_lam(batch, out, st, los, pick)
    ko = batch.knot_off
    for b in set(range(batch.B)) - set(pick):
        assert st["status"][b] == -1 and np.all(out[ko[b]:ko[b + 1]] == 7.0), b


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_horizon_beyond_the_launch_is_refused_per_instance(mode):
    """dims.N sized for 64 knots: the listed 100- and 512-knot instances get
    MPCG_BADINPUT, the others are solved."""
    import torch
    from paper_2309_08079_gb300.solver import make_opts, read_stats
    s, batch, lt, sch, lam = _setup(NS, 4200)
    los = _oracle_lams(batch)
    pick = [0, 1, 2, 3, 4, 7]                      # N = 3, 17, 40, 64, 100, 512
    inst = torch.tensor(pick, dtype=torch.int32, device="cuda")
    stats = s.alloc_stats(batch.B)
    s.pcg_solve(lt, sch, lam, make_opts(mode=mode, instances=inst), stats, N=64)
    torch.cuda.synchronize()
    st = read_stats(stats)
    assert st["status"][4] == 4 and st["status"][7] == 4
    _check_lam(batch, lam.cpu().double().numpy(), st, los, [0, 1, 2, 3])


def test_every_candidate_plan_matches_the_oracle():
    import torch
    from paper_2309_08079_gb300.autotune import PlanRunner, candidate_plans
    from paper_2309_08079_gb300.solver import read_stats
    s, batch, lt, sch, lam = _setup(NS, 4300)
    los = _oracle_lams(batch)
    plans = candidate_plans(lt.Ns)
    assert len(plans) >= 5
    results = {}
    for name, plan in plans.items():
        r = PlanRunner(s, lt, plan)
        lam.zero_()
        stats = s.alloc_stats(batch.B)
        r.pcg_solve(sch, lam, stats)
        torch.cuda.synchronize()
        results[name] = lam.cpu().double().numpy()
        _check_lam(batch, results[name], read_stats(stats), los)
    # the CTA-per-instance kernel is deterministic whatever the queue order
    lone = PlanRunner(s, lt, [{"lo": 0, "hi": 1 << 30, "mode": 2, "cluster": 0}])
    np.testing.assert_array_equal(results["single_cta_l2"], _run(s, lt, sch, lone))


def _run(s, lt, sch, runner):
    import torch
    lam = torch.zeros(lt.total, lt.nx, device="cuda")
    runner.pcg_solve(sch, lam, s.alloc_stats(lt.nb))
    torch.cuda.synchronize()
    return lam.cpu().double().numpy()


def test_autotuner_tunes_caches_and_reuses(tmp_path):
    import torch
    from paper_2309_08079_gb300.autotune import Autotuner
    from paper_2309_08079_gb300.solver import read_stats
    Ns = gen.batch_horizons(48, 32, 512, 11)
    s, batch, lt, sch, lam0 = _setup(Ns, 4400)
    los = _oracle_lams(batch)
    tuner = Autotuner(s, cache_path=str(tmp_path / "tune.json"), reps=2)
    assert tuner.cached_plan(lt) is None
    best = tuner.tune(lt, sch, lam0)
    assert best["plan"] in tuner.last_timings and len(tuner.last_timings) >= 3
    assert best["ms"] == min(tuner.last_timings.values())
    assert tuner.cached_plan(lt)["plan"] == best["plan"]
    runner = tuner.runner(lt, sch, lam0)           # from the cache: no tuning
    assert runner.plan == best["groups"]
    lam = lam0.clone()
    stats = s.alloc_stats(batch.B)
    runner.pcg_solve(sch, lam, stats)
    torch.cuda.synchronize()
    _check_lam(batch, lam.cpu().double().numpy(), read_stats(stats), los)


def test_graph_mode_tuning_has_its_own_cache_entry(tmp_path):
    """Autotuner(graph=True) times each plan captured in a CUDA graph; its
    choice is cached under its own key (the eager entry is separate), and
    the runner it returns solves the batch."""
    import torch
    from paper_2309_08079_gb300.autotune import Autotuner
    from paper_2309_08079_gb300.solver import read_stats
    Ns = gen.batch_horizons(24, 32, 300, 12)
    s, batch, lt, sch, lam0 = _setup(Ns, 4500)
    los = _oracle_lams(batch)
    path = str(tmp_path / "tune.json")
    g = Autotuner(s, cache_path=path, reps=1, graph=True)
    best = g.tune(lt, sch, lam0, only=("single_auto", "classes_auto", "steps64_auto"))
    assert best["plan"] in g.last_timings and all(t > 0 for t in g.last_timings.values())
    assert g.key(lt).endswith("|graph")
    assert g.cached_plan(lt)["plan"] == best["plan"]
    assert Autotuner(s, cache_path=path, reps=1).cached_plan(lt) is None
    lam = lam0.clone()
    stats = s.alloc_stats(batch.B)
    g.runner(lt, sch, lam0).pcg_solve(sch, lam, stats)
    torch.cuda.synchronize()
    _check_lam(batch, lam.cpu().double().numpy(), read_stats(stats), los)


def test_plan_runner_in_a_cuda_graph():
    """A multi-stream plan captured in a CUDA graph gives the eager result."""
    import torch
    from paper_2309_08079_gb300.autotune import PlanRunner, candidate_plans
    from paper_2309_08079_gb300.solver import read_stats
    s, batch, lt, sch, lam = _setup(NS, 4500)
    runner = PlanRunner(s, lt, candidate_plans(lt.Ns)["classes_auto"])
    assert len(runner.launches) > 1
    eager = _run(s, lt, sch, runner)
    stats = s.alloc_stats(batch.B)
    lam.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            runner.pcg_solve(sch, lam, stats)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        lam.zero_()
        g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lam.cpu().double().numpy(), eager)
    assert np.all(read_stats(stats)["status"] == 0)
