"""The paper's exit test (Alg. 1: stop once eta' = r^T Phi^-1 r < eps,
tol_mode = 1) against the oracle's Algorithm 1 with the same test, at the
eps values of Sec. V-B / Fig. 5, cold and warm-started, N = 128."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, TOL_KNOT_F32, assert_knots, oracle_solution, run_gpu
from workload import gen

pytestmark = pytest.mark.gpu

N = 128
C = gen.CONFIG_SWEEP
SEED = C["seed_base"] + N


@pytest.mark.parametrize("eps", [1e-4, 5e-5, 1e-5])
@pytest.mark.parametrize("start", ["cold", "warm"])
def test_paper_exit_test_matches_the_oracle(eps, start):
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(C["nx"], C["nu"], N, SEED, dt=C["dt"], qd=C["qd"]).astype(np.float32)
    lo, xo, uo = oracle_solution(lq)
    lam0 = None
    if start == "warm":
        lam0 = gen.warm_start(lo, SEED, 0).astype(np.float32)
    lam, dx, du, st, _ = run_gpu(lq, lam0=lam0, opts=make_opts(tol=eps, tol_mode=1))
    assert st["status"][0] == 0 and st["eta"][0] < eps, st
    # the oracle's Algorithm 1 on S+, Phi^-1 and b formed in FP64 from the
    # same float32 inputs, from the same float32 start
    Sd, So, g = oracle.schur_blocks(lq.astype(np.float64))
    Pd, Po = oracle.precon_blocks(Sd, So)
    lam_o, it_o, ok = oracle.pcg(Sd, So, Pd, Po, -g, lam0=lam0, tol=eps, tol_mode=1)
    assert ok
    it_g = int(st["iters"][0])
    assert abs(it_g - it_o) <= max(3, 0.1 * it_o), (it_g, it_o)
    # both stop within the parity bar of the exact KKT solution
    assert oracle.relerr(lam, lo) < TOL_F32 and oracle.relerr(lam_o, lo.ravel()) < TOL_F32
    z = np.concatenate([dx.ravel(), du.ravel()])
    assert oracle.relerr(z, np.concatenate([xo.ravel(), uo.ravel()])) < TOL_F32
    assert_knots(lam, dx, du, lo, xo, uo, TOL_KNOT_F32, (eps, start))


def test_paper_exit_test_is_looser_than_the_relative_one():
    """At N = 128 eps = 1e-4 stops well before ||r|| <= 1e-6 ||b|| (the
    oracle takes the same order of iterations for both tests)."""
    from paper_2309_08079_gb300.solver import make_opts
    lq = gen.kuka_lq(C["nx"], C["nu"], N, SEED, dt=C["dt"], qd=C["qd"]).astype(np.float32)
    _, _, _, st1, _ = run_gpu(lq, opts=make_opts(tol=1e-4, tol_mode=1))
    _, _, _, st0, _ = run_gpu(lq, opts=make_opts(tol=1e-6))
    Sd, So, g = oracle.schur_blocks(lq.astype(np.float64))
    Pd, Po = oracle.precon_blocks(Sd, So)
    _, it1, _ = oracle.pcg(Sd, So, Pd, Po, -g, tol=1e-4, tol_mode=1)
    _, it0, _ = oracle.pcg(Sd, So, Pd, Po, -g, tol=1e-6)
    assert st1["iters"][0] < st0["iters"][0] and it1 < it0
