"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the
same seeded inputs."""
import numpy as np

import oracle
from workload import gen

# Parity bars (normwise relative error on lambda and dz against the FP64
# oracle run on the same rounded inputs).
TOL_F32 = 1e-4
TOL_F64 = 1e-9


def solver():
    from paper_2309_08079_gb300.solver import Solver
    global _S
    try:
        return _S
    except NameError:
        _S = Solver()
        return _S


def oracle_solution(lq):
    """Oracle (lambda, dx, du) on the inputs as the GPU sees them."""
    return oracle.kkt_solve(lq.astype(np.float64))


def run_gpu(lq, dtype="float32", lam0=None, opts=None):
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, read_stats
    tdt = torch.float32 if dtype == "float32" else torch.float64
    s = solver()
    lt = LQTensors.from_numpy(lq, dtype=tdt)
    lam = None if lam0 is None else torch.as_tensor(lam0, dtype=tdt, device="cuda").clone()
    lam, dx, du, stats, schur = s.solve(lt, lam, opts=opts)
    torch.cuda.synchronize()
    return (lam.cpu().double().numpy(), dx.cpu().double().numpy(), du.cpu().double().numpy(),
            read_stats(stats), schur)


def parity(lq, dtype="float32", lam0=None, opts=None):
    """Returns (err_lam, err_dz, stats) for one instance."""
    np_dt = np.float32 if dtype == "float32" else np.float64
    lq_in = lq.astype(np_dt)
    lam, dx, du, st, _ = run_gpu(lq_in, dtype, lam0, opts)
    lo, xo, uo = oracle_solution(lq_in)
    e_lam = oracle.relerr(lam, lo)
    e_dz = oracle.relerr(np.concatenate([dx.ravel(), du[:max(lq.N - 1, 0)].ravel()]),
                         np.concatenate([xo.ravel(), uo.ravel()]))
    return e_lam, e_dz, st
