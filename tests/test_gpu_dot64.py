"""float32 storage with float64-accumulated dot products (mpcg_opts.dot = 1)
in the cluster PCG kernel and the tiled kernel's compile-time shapes
(nx = 14, 36): parity against the oracle, and the same iteration counts as
the default double-float accumulation to within a few."""
import numpy as np
import pytest

from gpu_util import TOL_F32, parity, run_gpu
from workload import gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,nu,N", [(14, 7, 32), (14, 7, 128), (14, 7, 512), (14, 7, 300),
                                     (36, 12, 64), (4, 2, 33)])
def test_fp64_accumulation_parity(nx, nu, N):
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(nx, nu, N, 2 + N + nx)
    e_lam, e_dz, st = parity(lq, opts=make_opts(dot=1))
    assert st["status"][0] == 0, st
    assert e_lam < TOL_F32 and e_dz < TOL_F32, (e_lam, e_dz)
    _, _, st0 = parity(lq, opts=make_opts(dot=0))
    it1, it0 = int(st["iters"][0]), int(st0["iters"][0])
    assert abs(it1 - it0) <= max(3, 0.03 * it0), (it1, it0)


def test_fp64_accumulation_warm_start_n512():
    """The measured configuration: N = 512 warm-started from lambda* with 1%
    relative noise."""
    from paper_2309_08079_gb300.solver import make_opts
    import oracle
    c = gen.CONFIG_SWEEP
    lq = gen.kuka_lq(14, 7, 512, c["seed_base"] + 512, dt=c["dt"], qd=c["qd"])
    lo, _, _ = oracle.kkt_solve(lq.astype(np.float32).astype(np.float64))
    e_lam, e_dz, st = parity(lq, lam0=gen.warm_start(lo, c["seed_base"] + 512, 0),
                             opts=make_opts(dot=1))
    assert st["status"][0] == 0 and e_lam < TOL_F32 and e_dz < TOL_F32, (e_lam, e_dz)


def test_fp64_accumulation_batched():
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    from gpu_util import solver
    import oracle
    s = solver()
    batch = gen.kuka_batch(14, 7, [40, 7, 129, 300], 57).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    lam, _, _, st, _ = s.solve(lt, opts=make_opts(dot=1), workspace=s.alloc_workspace(lt))
    torch.cuda.synchronize()
    st = read_stats(st)
    lam = lam.cpu().double().numpy()
    ko = batch.knot_off
    for b, it in enumerate(batch.items):
        assert st["status"][b] == 0
        lo, _, _ = oracle.kkt_solve(it.astype(np.float64))
        assert oracle.relerr(lam[ko[b]:ko[b + 1]], lo) < TOL_F32


@pytest.mark.parametrize("nx,nu,Ns,large", [(14, 7, [1, 40, 7, 129, 300], False),
                                            (36, 12, [2, 64, 17, 200], True)])
def test_fp64_accumulation_tiled_kernel(nx, nu, Ns, large):
    """The tiled kernel (mode 3) with float64 dot products: every instance
    against the oracle (large-state shape with one refinement step, as the
    large-state workload runs), iterations within a few of double-float."""
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    from gpu_util import TOL_KNOT_F32, assert_knots, solver
    import oracle
    s = solver()
    c = gen.CONFIG_LARGE
    kw = dict(dt=c["dt"], qd=c["qd"]) if large else {}
    batch = gen.kuka_batch(nx, nu, Ns, 61 + nx, **kw).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    out = {}
    for dot in (0, 1):
        o = make_opts(dot=dot, mode=3, refine_tol=1e-2)
        lam, dx, du, st, sch = s.solve(lt, opts=o, workspace=s.alloc_workspace(lt), refine=1 if large else 0)
        assert s.pcg_shape(lt, sch, o)["form"] == "cta_tma"
        torch.cuda.synchronize()
        out[dot] = (lam.cpu().double().numpy(), dx.cpu().double().numpy(), du.cpu().double().numpy(),
                    read_stats(st))
    lam, dx, du, st = out[1]
    ko, co = batch.knot_off, batch.ctrl_off()
    for b, it in enumerate(batch.items):
        assert st["status"][b] == 0, (b, st[b])
        lo, xo, uo = oracle.kkt_solve(it.astype(np.float64))
        assert oracle.relerr(lam[ko[b]:ko[b + 1]], lo) < TOL_F32, (b, it.N)
        assert_knots(lam[ko[b]:ko[b + 1]], dx[ko[b]:ko[b + 1]], du[co[b]:co[b + 1]], lo, xo, uo,
                     TOL_KNOT_F32, (b, it.N))
        it1, it0 = int(st["iters"][b]), int(out[0][3]["iters"][b])
        assert abs(it1 - it0) <= max(3, 0.03 * it0), (b, it1, it0)


def test_fp64_accumulation_kernel_forms():
    """Supported in the cluster kernel and in the tiled kernel's nx = 14 and
    36 forms; refused by the L2 CTA kernel and by tiled shapes compiled
    without it."""
    from paper_2309_08079_gb300._lib import MPCG_EINVAL, MPCG_EUNSUPPORTED, MPCGError
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(14, 7, 16, 1).astype(np.float32)
    with pytest.raises(MPCGError) as ei:
        run_gpu(lq, opts=make_opts(dot=1, mode=2))
    assert ei.value.code == MPCG_EUNSUPPORTED
    _, _, _, st, _ = run_gpu(lq, opts=make_opts(dot=1, mode=3))
    assert st["status"][0] == 0
    with pytest.raises(MPCGError) as ei:
        run_gpu(gen.kuka_lq(4, 2, 16, 1).astype(np.float32), opts=make_opts(dot=1, mode=3))
    assert ei.value.code == MPCG_EUNSUPPORTED
    for bad in (-1, 2):
        with pytest.raises(MPCGError) as ei:
            run_gpu(lq, opts=make_opts(dot=bad))
        assert ei.value.code == MPCG_EINVAL
    # float64 storage ignores the switch (it always accumulates in float64)
    _, _, _, st, _ = run_gpu(lq.astype(np.float64), "float64", opts=make_opts(dot=1, tol=1e-12))
    assert st["status"][0] == 0
