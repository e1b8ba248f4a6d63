"""General SPD cost blocks Q_k, R_k (Sec. II-A's QP with full matrices):
form_schur and recover_step with dense blocks against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, TOL_F64, TOL_KNOT_F32, assert_knots, parity, run_gpu, solver
from workload import gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,nu,N,dtype", [(14, 7, 1, "float32"), (14, 7, 2, "float32"),
                                           (14, 7, 17, "float32"), (14, 7, 128, "float32"),
                                           (14, 7, 512, "float32"), (36, 12, 64, "float32"),
                                           (4, 2, 33, "float32"), (14, 7, 100, "float64"),
                                           (36, 12, 40, "float64")])
def test_dense_cost_parity(nx, nu, N, dtype):
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(nx, nu, N, 800 + N + nx, dense=True)
    f32 = dtype == "float32"
    e_lam, e_dz, st = parity(lq, dtype=dtype, opts=make_opts(tol=1e-6 if f32 else 1e-13))
    assert st["status"][0] == 0, st
    bar = TOL_F32 if f32 else TOL_F64
    assert e_lam < bar and e_dz < bar, (e_lam, e_dz)


def test_dense_blocks_with_diagonal_values_match_the_diagonal_path():
    """Q_k = diag(Qd_k), R_k = diag(Rd_k) as dense blocks: S+, gamma agree with
    the diagonal path to float32 rounding, and both solves meet the bar."""
    import torch
    from paper_2309_08079_gb300.solver import LQTensors
    lq = gen.kuka_lq(14, 7, 64, 811).astype(np.float32)
    dq = lq.copy()
    dq.Q = np.stack([np.diag(v) for v in lq.Qd]).astype(np.float32)
    dq.R = np.stack([np.diag(v) for v in lq.Rd]).astype(np.float32)
    s = solver()
    out = []
    for x in (lq, dq):
        lt = LQTensors.from_numpy(x)
        sch = s.alloc_schur(lt)
        s.form_schur(lt, sch)
        torch.cuda.synchronize()
        out.append([t.cpu().double().numpy() for t in (sch.Sd, sch.So, sch.gamma)])
    for a, b in zip(*out):
        assert oracle.relerr(b, a) < 1e-6
    lo, _, _ = oracle.kkt_solve(lq.astype(np.float64))
    for x in (lq, dq):
        lam, _, _, st, _ = run_gpu(x)
        assert st["status"][0] == 0 and oracle.relerr(lam, lo) < TOL_F32


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_dense_cost_batched(mode):
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    s = solver()
    batch = gen.kuka_batch(14, 7, [40, 3, 129, 64], 820, dense=True).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    lam, dx, du, st, _ = s.solve(lt, opts=make_opts(mode=mode), workspace=s.alloc_workspace(lt))
    torch.cuda.synchronize()
    st = read_stats(st)
    lam, dx, du = (t.cpu().double().numpy() for t in (lam, dx, du))
    ko, co = batch.knot_off, batch.ctrl_off()
    for b, it in enumerate(batch.items):
        lo, xo, uo = oracle.kkt_solve(it.astype(np.float64))
        assert st["status"][b] == 0
        assert oracle.relerr(lam[ko[b]:ko[b + 1]], lo) < TOL_F32
        z = np.concatenate([dx[ko[b]:ko[b + 1]].ravel(), du[co[b]:co[b + 1]].ravel()])
        assert oracle.relerr(z, np.concatenate([xo.ravel(), uo.ravel()])) < TOL_F32
        assert_knots(lam[ko[b]:ko[b + 1]], dx[ko[b]:ko[b + 1]], du[co[b]:co[b + 1]], lo, xo, uo,
                     TOL_KNOT_F32, b)


def test_dense_block_not_spd_is_bad_input():
    lq = gen.kuka_lq(14, 7, 30, 830, dense=True)
    lq.Q[7] = -lq.Q[7]
    lam, _, _, st, _ = run_gpu(lq.astype(np.float32), lam0=np.full((30, 14), 3.0))
    assert st["status"][0] == 4 and np.all(lam == 3.0)


def test_dense_refine_and_backward_are_refused():
    import torch
    from paper_2309_08079_gb300._lib import MPCG_EUNSUPPORTED, MPCGError
    from paper_2309_08079_gb300.solver import LQTensors, make_opts
    s = solver()
    lt = LQTensors.from_numpy(gen.kuka_lq(14, 7, 20, 840, dense=True).astype(np.float32))
    with pytest.raises(MPCGError) as e:
        s.solve(lt, opts=make_opts(), refine=1)
    assert e.value.code == MPCG_EUNSUPPORTED
    lam, dx, du, _, sch = s.solve(lt, opts=make_opts())
    with pytest.raises(MPCGError) as e:
        s.backward(lt, sch, lam, dx, du, torch.zeros_like(lam), dx, du)
    assert e.value.code == MPCG_EUNSUPPORTED
