"""Backward pass against the oracle's analytic gradient (KKT adjoint) and
against FP64 central differences of the oracle's loss."""
import numpy as np
import pytest

import oracle
from gpu_util import solver
from workload import gen

pytestmark = pytest.mark.gpu

FIELDS = ("A", "B", "Qd", "Rd", "q", "r", "c")


def _gpu_grads(lq, w, dtype="float32", opts=None, batch=None):
    import torch
    from paper_2309_08079_gb300.autograd import MPCGSolve
    from paper_2309_08079_gb300.solver import LQTensors
    tdt = torch.float32 if dtype == "float32" else torch.float64
    s = solver()
    lt = LQTensors.from_batch(batch, dtype=tdt) if batch is not None else LQTensors.from_numpy(lq, dtype=tdt)
    leaves = {f: getattr(lt, f).clone().requires_grad_(True) for f in FIELDS}
    cfg = dict(solver=s, nx=lt.nx, nu=lt.nu, N=lt.N, knot_off=lt.knot_off, nb=lt.nb,
               total=lt.total, opts=opts)
    if batch is not None:
        cfg["workspace"] = s.alloc_workspace(lt)
    lam, dx, du, _ = MPCGSolve.apply(*(leaves[f] for f in FIELDS), None, cfg)
    wt = torch.as_tensor(w, dtype=tdt, device="cuda")
    Lval = (dx * dx).sum() + (du * du).sum() + (wt * lam).sum()
    Lval.backward()
    torch.cuda.synchronize()
    return {f: leaves[f].grad.cpu().double().numpy() for f in FIELDS}, lam.detach().cpu().double().numpy()


def _oracle_grads(lq64, w):
    lam, dx, du = oracle.kkt_solve(lq64)
    return oracle.grad(lq64, lam, dx, du, w, 2 * dx, 2 * du)


@pytest.mark.parametrize("N", [2, 16, 128])
def test_backward_vs_oracle_f32(N):
    lq = gen.kuka_lq(14, 7, N, 4000 + N).astype(np.float32)
    w = gen.loss_weights(N * 14, 4).reshape(N, 14)
    g, _ = _gpu_grads(lq, w)
    go = _oracle_grads(lq.astype(np.float64), w)
    for f in FIELDS:
        e = oracle.relerr(g[f], go[f])
        assert e < 1e-3, (f, e)


def test_backward_f64_vs_oracle_and_central_differences():
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(6, 3, 8, 41)
    w = gen.loss_weights(8 * 6, 4).reshape(8, 6)
    g, _ = _gpu_grads(lq, w, "float64", opts=make_opts(tol=1e-13))
    go = _oracle_grads(lq, w)
    for f in FIELDS:
        assert oracle.relerr(g[f], go[f]) < 1e-8, f

    def L(l):
        lam, dx, du = oracle.kkt_solve(l)
        return oracle.loss(lam, dx, du, w)

    h = 1e-6
    round_err = 50 * np.finfo(np.float64).eps * abs(L(lq)) / h
    rng = np.random.default_rng(4)
    for f in FIELDS:
        arr = getattr(lq, f)
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            p, m = lq.copy(), lq.copy()
            getattr(p, f)[idx] += h
            getattr(m, f)[idx] -= h
            fd = (L(p) - L(m)) / (2 * h)
            assert abs(g[f][idx] - fd) <= 1e-7 * max(1, abs(fd)) + round_err, (f, idx)


def test_backward_batched():
    Ns = [16, 40, 9]
    batch = gen.kuka_batch(14, 7, Ns, 4100).astype(np.float32)
    K = int(batch.knot_off[-1])
    w = gen.loss_weights(K * 14, 4).reshape(K, 14)
    g, _ = _gpu_grads(None, w, batch=batch)
    ko, co = batch.knot_off, batch.ctrl_off()
    for b, it in enumerate(batch.items):
        go = _oracle_grads(it.astype(np.float64), w[ko[b]:ko[b + 1]])
        for f in FIELDS:
            if f in ("A", "B", "Rd", "r"):
                sl = slice(co[b], co[b + 1])
            else:
                sl = slice(ko[b], ko[b + 1])
            e = oracle.relerr(g[f][sl], go[f])
            assert e < 1e-3, (b, f, e)
