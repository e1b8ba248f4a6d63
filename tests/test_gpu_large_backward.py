"""Backward pass at the large-state shape (nx = 36, nu = 12, dt = 0.005,
Qd ~ U[0.1, 100]) against the oracle's analytic gradient, field by field.

Rounding S+ to float32 costs up to ~1e-3 in lambda here, so the forward
solve and the adjoint solve both take one step of iterative refinement
(MPCGSolve's cfg["refine"], which sets mpcg_opts.refine for the adjoint)."""
import numpy as np
import pytest

import oracle
from gpu_util import solver
from workload import gen

pytestmark = pytest.mark.gpu

FIELDS = ("A", "B", "Qd", "Rd", "q", "r", "c")
LARGE = gen.CONFIG_LARGE
GRAD_BAR = 1e-4


def _grads(lt, w, refine, workspace=None, refine_tol=0.0):
    import torch
    from paper_2309_08079_gb300.autograd import MPCGSolve
    from paper_2309_08079_gb300.solver import make_opts
    s = solver()
    leaves = {f: getattr(lt, f).clone().requires_grad_(True) for f in FIELDS}
    cfg = dict(solver=s, nx=lt.nx, nu=lt.nu, N=lt.N, knot_off=lt.knot_off, nb=lt.nb,
               total=lt.total, opts=make_opts(refine_tol=refine_tol), refine=refine,
               workspace=workspace if workspace is not None else s.alloc_workspace(lt))
    lam, dx, du, _ = MPCGSolve.apply(*(leaves[f] for f in FIELDS), None, cfg)
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    ((dx * dx).sum() + (du * du).sum() + (wt * lam).sum()).backward()
    torch.cuda.synchronize()
    return {f: leaves[f].grad.cpu().double().numpy() for f in FIELDS}


def _oracle_grad(it, w):
    it64 = it.astype(np.float64)
    lo, xo, uo = oracle.kkt_solve(it64)
    return oracle.grad(it64, lo, xo, uo, w, 2 * xo, 2 * uo)


def _field_errs(g, go, sl_k=slice(None), sl_c=slice(None)):
    return {f: oracle.relerr(g[f][sl_c if f in ("A", "B", "Rd", "r") else sl_k], go[f]) for f in FIELDS}


@pytest.mark.parametrize("N", [64, 256])
def test_large_state_backward_meets_the_oracle(N):
    from paper_2309_08079_gb300.solver import LQTensors
    lq = gen.kuka_lq(36, 12, N, LARGE["seed_base"] + N, dt=LARGE["dt"], qd=LARGE["qd"]).astype(np.float32)
    w = gen.loss_weights(N * 36, LARGE["seed_base"] + N).reshape(N, 36)
    go = _oracle_grad(lq, w)
    lt = LQTensors.from_numpy(lq)
    e0 = _field_errs(_grads(lt, w, refine=0), go)
    e1 = _field_errs(_grads(lt, w, refine=1), go)
    print(f"N={N} unrefined {max(e0.values()):.2e} refined {max(e1.values()):.2e}", e1)
    assert max(e1.values()) < GRAD_BAR, (e0, e1)
    assert max(e1.values()) < max(e0.values()), (e0, e1)


@pytest.mark.parametrize("refine_tol", [0.0, 1e-2])
def test_large_state_backward_batched(refine_tol):
    """A ragged batch of large-state instances through the batched backward
    with refinement: every instance's gradient, field by field.  Also with
    the refinement's correction solves stopped at relative residual 1e-2
    (the large-state workload's setting), for the forward and the adjoint."""
    from paper_2309_08079_gb300.solver import LQTensors
    Ns = [64, 150, 256, 97]
    batch = gen.kuka_batch(36, 12, Ns, LARGE["seed_base"], dt=LARGE["dt"], qd=LARGE["qd"]).astype(np.float32)
    K = int(batch.knot_off[-1])
    w = gen.loss_weights(K * 36, LARGE["seed_base"]).reshape(K, 36)
    lt = LQTensors.from_batch(batch)
    g = _grads(lt, w, refine=1, refine_tol=refine_tol)
    ko, co = batch.knot_off, batch.ctrl_off()
    for b, it in enumerate(batch.items):
        e = _field_errs(g, _oracle_grad(it, w[ko[b]:ko[b + 1]]), slice(ko[b], ko[b + 1]),
                        slice(co[b], co[b + 1]))
        assert max(e.values()) < GRAD_BAR, (b, Ns[b], e)


def test_adjoint_refinement_argument_is_checked():
    import torch
    from paper_2309_08079_gb300._lib import MPCGError
    from paper_2309_08079_gb300.solver import LQTensors, make_opts
    s = solver()
    lq = gen.kuka_lq(14, 7, 8, 3).astype(np.float32)
    lt = LQTensors.from_numpy(lq)
    lam, dx, du, _, sch = s.solve(lt)
    z = torch.zeros_like
    with pytest.raises(MPCGError):
        s.backward(lt, sch, lam, dx, du, z(lam), z(dx), z(du), opts=make_opts(refine=-1))
