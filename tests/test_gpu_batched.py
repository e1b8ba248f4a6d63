"""Batched (ragged-horizon) solves against the oracle, instance by instance."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, TOL_F64, TOL_KNOT_F32, TOL_KNOT_F64, assert_knots, solver
from workload import gen

pytestmark = pytest.mark.gpu


def _run_batch(batch, dtype="float32", lam0=None, opts=None):
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, read_stats
    tdt = torch.float32 if dtype == "float32" else torch.float64
    s = solver()
    lt = LQTensors.from_batch(batch, dtype=tdt)
    lam = None if lam0 is None else torch.as_tensor(lam0, dtype=tdt, device="cuda").clone()
    lam, dx, du, stats, _ = s.solve(lt, lam, opts=opts)
    torch.cuda.synchronize()
    return (lam.cpu().double().numpy(), dx.cpu().double().numpy(), du.cpu().double().numpy(),
            read_stats(stats))


def _check(batch, lam, dx, du, st, tol):
    ko = batch.knot_off
    co = batch.ctrl_off()
    for b, it in enumerate(batch.items):
        lo, xo, uo = oracle.kkt_solve(it.astype(np.float64))
        assert st["status"][b] == 0, (b, st[b])
        e_lam = oracle.relerr(lam[ko[b]:ko[b + 1]], lo)
        z = np.concatenate([dx[ko[b]:ko[b + 1]].ravel(), du[co[b]:co[b + 1]].ravel()])
        e_dz = oracle.relerr(z, np.concatenate([xo.ravel(), uo.ravel()]))
        assert e_lam < tol and e_dz < tol, (b, it.N, e_lam, e_dz)
        assert_knots(lam[ko[b]:ko[b + 1]], dx[ko[b]:ko[b + 1]], du[co[b]:co[b + 1]], lo, xo, uo,
                     TOL_KNOT_F32 if tol >= TOL_F32 else TOL_KNOT_F64, (b, it.N))


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
@pytest.mark.parametrize("Ns", [[1, 5, 32, 33, 100, 64], [512, 3, 257], [2] * 7])
def test_batched_ragged_parity(Ns, mode):
    from paper_2309_08079_gb300.solver import make_opts
    batch = gen.kuka_batch(14, 7, Ns, 1000).astype(np.float32)
    lam, dx, du, st = _run_batch(batch, opts=make_opts(mode=mode))
    _check(batch, lam, dx, du, st, TOL_F32)


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_batched_queue_more_instances_than_clusters(mode):
    """300 instances: more than the co-resident clusters or CTAs, so the
    persistent grid drains the instance queue."""
    from paper_2309_08079_gb300.solver import make_opts
    Ns = gen.batch_horizons(300, 8, 64, 3)
    batch = gen.kuka_batch(14, 7, Ns, 2000).astype(np.float32)
    lam, dx, du, st = _run_batch(batch, opts=make_opts(mode=mode))
    _check(batch, lam, dx, du, st, TOL_F32)


def test_batched_modes_agree():
    """The cluster and the CTA-per-instance kernels solve the same batch to
    the same tolerance; the CTA kernel is deterministic across batch shapes."""
    from paper_2309_08079_gb300.solver import make_opts
    from gpu_util import run_gpu
    Ns = [40, 7, 129, 300]
    batch = gen.kuka_batch(14, 7, Ns, 56).astype(np.float32)
    l1, _, _, s1 = _run_batch(batch, opts=make_opts(mode=1))
    l2, _, _, s2 = _run_batch(batch, opts=make_opts(mode=2))
    l3, _, _, s3 = _run_batch(batch, opts=make_opts(mode=3))
    assert oracle.relerr(l1, l2) < 2 * TOL_F32 and oracle.relerr(l2, l3) < 2 * TOL_F32
    ko = batch.knot_off
    for b, it in enumerate(batch.items):
        lone, _, _, st, _ = run_gpu(it, opts=make_opts(mode=2))
        np.testing.assert_array_equal(l2[ko[b]:ko[b + 1]], lone)
        assert st["iters"][0] == s2["iters"][b]


def test_batched_other_shapes_and_f64():
    from paper_2309_08079_gb300.solver import make_opts
    batch = gen.kuka_batch(4, 2, [3, 17, 40], 77)
    lam, dx, du, st = _run_batch(batch, "float64", opts=make_opts(tol=1e-13))
    _check(batch, lam, dx, du, st, TOL_F64)
    batch36 = gen.kuka_batch(36, 12, [4, 16, 9], 78).astype(np.float32)
    lam, dx, du, st = _run_batch(batch36)
    _check(batch36, lam, dx, du, st, TOL_F32)


def test_batched_matches_single_solves():
    """A batch gives each instance what a single-instance call gives it."""
    from gpu_util import run_gpu
    Ns = [40, 7, 129]
    batch = gen.kuka_batch(14, 7, Ns, 55).astype(np.float32)
    lam, dx, du, st = _run_batch(batch)
    ko = batch.knot_off
    for b, it in enumerate(batch.items):
        l1, _, _, s1, _ = run_gpu(it)
        np.testing.assert_array_equal(lam[ko[b]:ko[b + 1]], l1)
        assert s1["iters"][0] == st["iters"][b]


def test_batched_poisoned_instance_isolated():
    Ns = [20, 30, 25]
    items = [gen.kuka_lq(14, 7, n, 900 + i) for i, n in enumerate(Ns)]
    items[1].Rd[3, 0] = 0.0
    batch = gen.concat_batch(items).astype(np.float32)
    lam, dx, du, st = _run_batch(batch)
    assert st["status"][1] == 4
    for b in (0, 2):
        assert st["status"][b] == 0
        lo, _, _ = oracle.kkt_solve(batch.items[b].astype(np.float64))
        assert oracle.relerr(lam[batch.knot_off[b]:batch.knot_off[b + 1]], lo) < TOL_F32


def test_batched_warm_start():
    Ns = [64, 200, 33]
    batch = gen.kuka_batch(14, 7, Ns, 1500).astype(np.float32)
    los = [oracle.kkt_solve(it.astype(np.float64))[0] for it in batch.items]
    lam0 = np.concatenate([gen.warm_start(l, 1500 + i, 0) for i, l in enumerate(los)])
    lam, dx, du, st = _run_batch(batch, lam0=lam0)
    _check(batch, lam, dx, du, st, TOL_F32)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_out_of_range_instance_entry_is_skipped(mode):
    """An instance-list entry outside [0, B) reads and writes nothing: the
    listed in-range instances are solved, the others' lambda and stats stay
    as they were."""
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    s = solver()
    Ns = [30, 12, 45]
    batch = gen.kuka_batch(14, 7, Ns, 3100).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    sch = s.alloc_schur(lt)
    s.form(lt, sch)
    inst = torch.tensor([0, 7, 2], dtype=torch.int32, device="cuda")
    lam = torch.full((lt.total, 14), 0.25, device="cuda")
    stats = s.alloc_stats(lt.nb)
    stats.fill_(0xFF)
    s.pcg_solve(lt, sch, lam, make_opts(mode=mode, instances=inst), stats, s.alloc_workspace(lt), N=45)
    torch.cuda.synchronize()
    st = read_stats(stats)
    lam = lam.cpu().double().numpy()
    ko = batch.knot_off
    assert st["iters"][1] == -1 and st["status"][1] == -1, st
    assert np.all(lam[ko[1]:ko[2]] == 0.25)
    for b in (0, 2):
        assert st["status"][b] == 0, (b, st[b])
        lo, _, _ = oracle.kkt_solve(batch.items[b].astype(np.float64))
        assert oracle.relerr(lam[ko[b]:ko[b + 1]], lo) < TOL_F32, b


@pytest.mark.parametrize("nx,nu,lo_bound,hi_bound", [(36, 12, 400, 500), (14, 7, 1200, 1342)])
def test_tiled_kernel_at_its_largest_horizon(nx, nu, lo_bound, hi_bound):
    """At the largest horizon the tiled form accepts, the three
    shared vectors leave room for one knot stream (one warp walking every
    knot of each pass; two 16-lane streams at nx = 14), and the solve meets
    the oracle (one refinement step, as at the large-state shape).  One knot
    more fits no kernel form (clusters end at 16 CTAs x 16 knots at nx = 36
    and 512 knots at nx = 14, the L2 CTA kernel's five vectors at ~320 and
    ~724 knots): mode 3 and the automatic choice both refuse it with
    MPCG_EUNSUPPORTED, before any launch."""
    import torch
    from paper_2309_08079_gb300._lib import MPCG_EUNSUPPORTED, MPCGError
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    s = solver()
    probe = LQTensors.from_batch(gen.kuka_batch(nx, nu, [4, 3], 1).astype(np.float32))
    psch = s.alloc_schur(probe)
    o3 = make_opts(mode=3, refine_tol=1e-2)

    def tiled(N):
        try:
            return s.pcg_shape(probe, psch, o3, N=N)["form"] == "cta_tma"
        except MPCGError:
            return False
    lo, hi = 64, 4096  # tiled(lo), not tiled(hi)
    assert tiled(lo) and not tiled(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if tiled(mid) else (lo, mid)
    Nmax = lo
    assert lo_bound <= Nmax <= hi_bound, Nmax
    batch = gen.kuka_batch(nx, nu, [Nmax, 9], 3200 + Nmax).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    lam, dx, du, st, sch = s.solve(lt, opts=o3, workspace=s.alloc_workspace(lt), refine=1)
    sh = s.pcg_shape(lt, sch, o3)
    assert sh["form"] == "cta_tma" and sh["threads"] == 32, sh  # one warp
    torch.cuda.synchronize()
    lam, dx, du = (t.cpu().double().numpy() for t in (lam, dx, du))
    _check(batch, lam, dx, du, read_stats(st), TOL_F32)
    for o in (o3, make_opts()):
        with pytest.raises(MPCGError) as ei:
            s.pcg_shape(probe, psch, o, N=Nmax + 1)
        assert ei.value.code == MPCG_EUNSUPPORTED
