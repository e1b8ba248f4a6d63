"""float32 storage with float64-accumulated dot products (mpcg_opts.dot = 1)
in the cluster PCG kernel: parity against the oracle, and the same iteration
counts as the default double-float accumulation to within a few."""
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


def test_fp64_accumulation_only_in_the_cluster_kernel():
    from paper_2309_08079_gb300._lib import MPCG_EINVAL, MPCG_EUNSUPPORTED, MPCGError
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(14, 7, 16, 1).astype(np.float32)
    for mode in (2, 3):
        with pytest.raises(MPCGError) as ei:
            run_gpu(lq, opts=make_opts(dot=1, mode=mode))
        assert ei.value.code == MPCG_EUNSUPPORTED
    for bad in (-1, 2):
        with pytest.raises(MPCGError) as ei:
            run_gpu(lq, opts=make_opts(dot=bad))
        assert ei.value.code == MPCG_EINVAL
    # float64 storage ignores the switch (it always accumulates in float64)
    _, _, _, st, _ = run_gpu(lq.astype(np.float64), "float64", opts=make_opts(dot=1, tol=1e-12))
    assert st["status"][0] == 0
