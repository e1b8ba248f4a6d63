"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the
same seeded inputs."""
import numpy as np

import oracle
from workload import gen

# Parity bars against the FP64 oracle run on the same rounded inputs.
# Normwise: relative error over the whole lambda and over the whole dz.
TOL_F32 = 1e-4
TOL_F64 = 1e-9
# Per knot: max over k of ||x_k - x*_k|| / ||x*_k|| for lambda_k, dx_k and
# du_k separately.  lambda_k is the PCG's own output: the exact solve of S+
# rounded to float32 is up to 9.4e-5 from the oracle per knot at N = 512,
# seed 514, and a wrong row of one knot (a halo copy, a CTA boundary) shows
# up here long before it moves the normwise error.  dz is recovered per knot
# from lambda through dx_k = (lambda_k - A_k^T lambda_{k+1} - q_k) / Qd_k,
# which cancels where A_k ~ I: storing even the exact lambda in float32
# leaves up to 7e-4 in dx_k at the worst knot (nx = 36, dt = 0.005), so
# dx_k and du_k have their own bar.
TOL_KNOT_F32 = 1e-3
TOL_KNOT_DZ_F32 = 5e-3
TOL_KNOT_F64 = 1e-8


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


def knot_err(x, ref) -> float:
    """max over knots k of ||x_k - ref_k||_2 / ||ref_k||_2 (rows = knots)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    x = x.reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.linalg.norm(x - ref, axis=1) / den))


def knot_errs(lam, dx, du, lo, xo, uo):
    """Per-knot errors (lambda_k, dx_k, du_k) as a tuple."""
    n_u = uo.shape[0] if np.ndim(uo) > 1 else 0
    return (knot_err(lam, lo), knot_err(dx, xo),
            knot_err(np.asarray(du)[:n_u], uo) if n_u else 0.0)


def assert_knots(lam, dx, du, lo, xo, uo, bar=TOL_KNOT_F32, what=""):
    """Per-knot bars: `bar` on lambda_k; on dx_k and du_k the float32 dz bar
    (5x) when `bar` is the float32 lambda bar, else `bar` itself."""
    e = knot_errs(lam, dx, du, lo, xo, uo)
    bar_dz = TOL_KNOT_DZ_F32 if bar == TOL_KNOT_F32 else bar
    assert e[0] < bar and max(e[1:]) < bar_dz, ("per-knot error (lambda, dx, du)", what, e)
    return e


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
    """Returns (err_lam, err_dz, stats) for one instance (normwise errors).

    When the solve converged it also asserts the per-knot bar
    (TOL_KNOT_F32 / TOL_KNOT_F64) on lambda_k, dx_k and du_k."""
    np_dt = np.float32 if dtype == "float32" else np.float64
    lq_in = lq.astype(np_dt)
    lam, dx, du, st, _ = run_gpu(lq_in, dtype, lam0, opts)
    lo, xo, uo = oracle_solution(lq_in)
    e_lam = oracle.relerr(lam, lo)
    e_dz = oracle.relerr(np.concatenate([dx.ravel(), du[:max(lq.N - 1, 0)].ravel()]),
                         np.concatenate([xo.ravel(), uo.ravel()]))
    if st["status"][0] == 0:
        assert_knots(lam, dx, du[:max(lq.N - 1, 0)], lo, xo, uo,
                     TOL_KNOT_F32 if dtype == "float32" else TOL_KNOT_F64, f"N={lq.N}")
    return e_lam, e_dz, st
