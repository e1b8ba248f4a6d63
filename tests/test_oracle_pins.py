"""Pins for the FP64 oracle: each test checks the oracle against something
other than itself (brute force, exact rational arithmetic, an independent
Riccati solver, the paper's closed forms, invariants, finite differences).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from pins import dense_kkt, riccati
from workload import gen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            vals[k.strip()] = np.array([float(t) for t in v.split()])
    return vals


def _golden_lq():
    g = _read_golden("scalar_two_knot.txt")
    lq = gen.LQ(1, 1, 2, g["A"].reshape(1, 1, 1), g["B"].reshape(1, 1, 1),
                g["Qd"].reshape(2, 1), g["Rd"].reshape(1, 1), g["q"].reshape(2, 1),
                g["r"].reshape(1, 1), g["c"].reshape(2, 1))
    return lq, g


# ---------------------------------------------------------------- worked example
def test_golden_scalar_two_knot_solution():
    lq, g = _golden_lq()
    lam, dx, du = oracle.kkt_solve(lq)
    np.testing.assert_allclose(lam.ravel(), g["lam"], atol=1e-15)
    np.testing.assert_allclose(dx.ravel(), g["dx"], atol=1e-15)
    np.testing.assert_allclose(du.ravel(), g["du"], atol=1e-15)


def test_golden_scalar_two_knot_blocks():
    lq, g = _golden_lq()
    Sd, So, gamma = oracle.schur_blocks(lq)
    np.testing.assert_allclose(Sd.ravel(), g["Sd"], atol=1e-15)
    np.testing.assert_allclose(So.ravel(), g["So"], atol=1e-15)
    np.testing.assert_allclose(gamma.ravel(), g["gamma"], atol=1e-15)
    Pd, Po = oracle.precon_blocks(Sd, So)
    np.testing.assert_allclose(Pd.ravel(), g["Pd"], atol=1e-15)
    np.testing.assert_allclose(Po.ravel(), g["Po"], atol=1e-15)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("nx,nu,N,seed", [(2, 1, 1, 0), (2, 1, 2, 1), (4, 2, 5, 2),
                                          (14, 7, 8, 3), (36, 12, 3, 4), (6, 3, 8, 5)])
def test_kkt_vs_dense_solve(nx, nu, N, seed, dense):
    lq = gen.kuka_lq(nx, nu, N, seed, dense=dense)
    K, h, _ = dense_kkt(lq)
    y = np.linalg.solve(K, h)
    nz = N * nx + (N - 1) * nu
    lam, dx, du = oracle.kkt_solve(lq)
    np.testing.assert_allclose(lam.ravel(), y[nz:], rtol=0, atol=1e-10 * np.abs(y).max())
    np.testing.assert_allclose(oracle.natural_z(dx, du), -y[:nz], rtol=0,
                               atol=1e-10 * np.abs(y).max())


def test_kkt_exact_rational():
    """Exact rational solve of a small KKT system (no rounding anywhere)."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(11)
    nx, nu, N = 2, 1, 3

    def rat(lo, hi, shape):
        return rng.integers(lo, hi, size=shape).astype(np.float64) / 4.0

    lq = gen.LQ(nx, nu, N, rat(-4, 5, (N - 1, nx, nx)), rat(-4, 5, (N - 1, nx, nu)),
                rat(1, 9, (N, nx)), rat(1, 9, (N - 1, nu)), rat(-8, 9, (N, nx)),
                rat(-8, 9, (N - 1, nu)), rat(-8, 9, (N, nx)))
    K, h, _ = dense_kkt(lq)
    Ks = sympy.Matrix([[Fraction(v).limit_denominator() for v in row] for row in K])
    hs = sympy.Matrix([Fraction(v).limit_denominator() for v in h])
    y = np.array([float(v) for v in Ks.LUsolve(hs)])
    nz = N * nx + (N - 1) * nu
    lam, dx, du = oracle.kkt_solve(lq)
    np.testing.assert_allclose(lam.ravel(), y[nz:], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.natural_z(dx, du), -y[:nz], rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- Riccati
@pytest.mark.parametrize("nx,nu,N,seed,kw", [
    (14, 7, 32, 1, {}),
    (14, 7, 128, 130, {}),
    (14, 7, 512, 514, {}),
    (36, 12, 64, 5000, dict(dt=0.005, qd=(0.1, 100.0))),
    (14, 7, 128, 131, dict(dense=True)),
    (36, 12, 48, 5001, dict(dt=0.005, qd=(0.1, 100.0), dense=True)),
])
def test_kkt_vs_riccati(nx, nu, N, seed, kw):
    lq = gen.kuka_lq(nx, nu, N, seed, **kw)
    lam, dx, du = oracle.kkt_solve(lq)
    lr, xr, ur = riccati(lq)
    assert oracle.relerr(lam, lr) < 1e-9
    assert oracle.relerr(dx, xr) < 1e-9
    assert oracle.relerr(du, ur) < 1e-9


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("N,seed", [(32, 1), (128, 7)])
def test_kkt_invariants(N, seed):
    lq = gen.kuka_lq(14, 7, N, seed)
    lam, dx, du = oracle.kkt_solve(lq)
    # linearised dynamics C dz + c = 0
    scale = max(1.0, np.abs(lq.c).max(), np.abs(dx).max() * (1 + np.abs(lq.A).max()))
    res0 = dx[0] + lq.c[0]
    resk = dx[1:] - np.einsum("kij,kj->ki", lq.A, dx[:-1]) - np.einsum("kij,kj->ki", lq.B, du) + lq.c[1:]
    assert max(np.abs(res0).max(), np.abs(resk).max()) <= 1e-12 * scale * 10
    # stationarity G dz + g - C^T lam = 0
    sx = lq.Qd * dx + lq.q - lam
    sx[:-1] += np.einsum("kji,kj->ki", lq.A, lam[1:])
    su = lq.Rd * du + lq.r + np.einsum("kji,kj->ki", lq.B, lam[1:])
    sc = max(1.0, np.abs(lam).max() * 10)
    assert np.abs(sx).max() < 1e-11 * sc and np.abs(su).max() < 1e-11 * sc


def test_schur_spd_and_precon_spd():
    lq = gen.kuka_lq(14, 7, 24, 3)
    Sd, So, _ = oracle.schur_blocks(lq)
    S = oracle.block_tridiag_sparse(Sd, So).toarray()
    np.linalg.cholesky(S)
    Pd, Po = oracle.precon_blocks(Sd, So)
    P = oracle.block_tridiag_sparse(Pd, Po).toarray()
    assert np.abs(P - P.T).max() < 1e-12 * np.abs(P).max()
    assert np.linalg.eigvalsh(P).min() > 0


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("nx,nu,N,seed", [(14, 7, 9, 21), (4, 2, 6, 22), (36, 12, 4, 23)])
def test_schur_closed_forms(nx, nu, N, seed, dense):
    """schur_blocks (sparse C G^-1 C^T) against Eq. trajoptSchur_1/2; dense
    cost blocks are inverted here through a Cholesky factorisation."""
    import scipy.linalg as sla
    lq = gen.kuka_lq(nx, nu, N, seed, dense=dense)
    Sd, So, gamma = oracle.schur_blocks(lq)
    if dense:
        inv = lambda M: sla.cho_solve(sla.cho_factor(M), np.eye(M.shape[0]))
        Qi = [inv(lq.Q[k]) for k in range(N)]
        Ri = [inv(lq.R[k]) for k in range(N - 1)]
    else:
        Qi = [np.diag(1.0 / lq.Qd[k]) for k in range(N)]
        Ri = [np.diag(1.0 / lq.Rd[k]) for k in range(N - 1)]
    np.testing.assert_allclose(Sd[0], Qi[0], atol=1e-14)
    np.testing.assert_allclose(gamma[0], lq.c[0] - Qi[0] @ lq.q[0], atol=1e-13)
    for k in range(N - 1):
        A, B = lq.A[k], lq.B[k]
        theta = A @ Qi[k] @ A.T + B @ Ri[k] @ B.T + Qi[k + 1]
        phi = -A @ Qi[k]
        zeta = -A @ Qi[k] @ lq.q[k] - B @ Ri[k] @ lq.r[k] + Qi[k + 1] @ lq.q[k + 1]
        np.testing.assert_allclose(Sd[k + 1], theta, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(So[k], phi, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(gamma[k + 1], lq.c[k + 1] - zeta, rtol=1e-12, atol=1e-12)


def test_precon_matches_dense_formula_and_printed_blocks():
    """Phi^-1 blocks against D^-1 - D^-1 O D^-1 (dense) and against the
    blocks printed in Sec. IV-A for the first block rows."""
    lq = gen.kuka_lq(6, 3, 7, 31)
    Sd, So, _ = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    P = oracle.block_tridiag_sparse(Pd, Po).toarray()
    Pdense = oracle.dense_Phi_inv(Sd, So)
    np.testing.assert_allclose(P, Pdense, rtol=1e-12, atol=1e-12)
    nx = 6
    Q0 = np.diag(lq.Qd[0])
    th0 = Sd[1]
    th1 = Sd[2]
    ph0, ph1 = So[0], So[1]
    inv = np.linalg.inv
    np.testing.assert_allclose(P[:nx, :nx], Q0, atol=1e-12)
    np.testing.assert_allclose(P[:nx, nx:2 * nx], -Q0 @ ph0.T @ inv(th0), atol=1e-12)
    np.testing.assert_allclose(P[nx:2 * nx, :nx], -inv(th0) @ ph0 @ Q0, atol=1e-12)
    np.testing.assert_allclose(P[nx:2 * nx, nx:2 * nx], inv(th0), atol=1e-12)
    np.testing.assert_allclose(P[nx:2 * nx, 2 * nx:3 * nx], -inv(th0) @ ph1.T @ inv(th1), atol=1e-12)
    np.testing.assert_allclose(P[2 * nx:3 * nx, nx:2 * nx], -inv(th1) @ ph1 @ inv(th0), atol=1e-12)


def test_schur_route_reaches_kkt_solution():
    """Solving S+ lambda = -gamma then dz = -G^-1 (g - C^T lambda) gives the
    KKT solution: pins schur_blocks, the sign reading and recover."""
    lq = gen.kuka_lq(14, 7, 20, 41)
    Sd, So, gamma = oracle.schur_blocks(lq)
    S = oracle.block_tridiag_sparse(Sd, So).toarray()
    lam_s = np.linalg.solve(S, -gamma.ravel())
    lam, dx, du = oracle.kkt_solve(lq)
    assert oracle.relerr(lam_s, lam) < 1e-12
    dx2, du2 = oracle.recover(lq, lam)
    assert oracle.relerr(dx2, dx) < 1e-12 and oracle.relerr(du2, du) < 1e-12


# ---------------------------------------------------------------- PCG special cases
def test_pcg_reaches_kkt_solution():
    lq = gen.kuka_lq(14, 7, 32, 1)
    Sd, So, gamma = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    lam_p, it, ok = oracle.pcg(Sd, So, Pd, Po, -gamma, tol=1e-12)
    lam, _, _ = oracle.kkt_solve(lq)
    assert ok and oracle.relerr(lam_p, lam) < 1e-9 and it > 10


def test_pcg_decoupled_converges_in_one_iteration():
    """A_k = B_k = 0: S+ is block diagonal and Phi^-1 = S+^-1 exactly."""
    lq = gen.kuka_lq(14, 7, 16, 5)
    lq.A[:] = 0.0
    lq.B[:] = 0.0
    Sd, So, gamma = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    assert np.abs(Po).max() == 0.0
    lam_p, it, ok = oracle.pcg(Sd, So, Pd, Po, -gamma, tol=1e-12)
    assert ok and it == 1
    lam, _, _ = oracle.kkt_solve(lq)
    assert oracle.relerr(lam_p, lam) < 1e-13


def test_pcg_identity_precon_is_textbook_cg():
    """Phi = I reduces Algorithm 1 to plain CG: compare against scipy's CG."""
    import scipy.sparse.linalg as spla
    lq = gen.kuka_lq(4, 2, 10, 9)
    Sd, So, gamma = oracle.schur_blocks(lq)
    I = np.broadcast_to(np.eye(4), Sd.shape).copy()
    Z = np.zeros_like(So)
    lam_p, it, ok = oracle.pcg(Sd, So, I, Z, -gamma, tol=1e-11)
    S = oracle.block_tridiag_sparse(Sd, So)
    x, info = spla.cg(S, -gamma.ravel(), rtol=1e-13, maxiter=10000)
    assert ok and info == 0 and oracle.relerr(lam_p, x) < 1e-8


def test_pcg_finite_termination():
    """In exact arithmetic CG ends within n = N nx steps; in FP64 on a tiny
    well-conditioned system it reaches 1e-12 by then."""
    lq = gen.kuka_lq(2, 1, 4, 3)
    Sd, So, gamma = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    _, it, ok = oracle.pcg(Sd, So, Pd, Po, -gamma, tol=1e-12)
    assert ok and it <= 8


def test_pcg_warm_start_exact_takes_zero_iterations():
    lq = gen.kuka_lq(4, 2, 6, 2)
    Sd, So, gamma = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    lam, _, _ = oracle.kkt_solve(lq)
    _, it, ok = oracle.pcg(Sd, So, Pd, Po, -gamma, lam0=lam, tol=1e-8)
    assert ok and it == 0


# ---------------------------------------------------------------- gradient
def test_grad_vs_central_differences():
    """Analytic gradient (KKT adjoint) vs FP64 central differences, h = 1e-6,
    on random coordinates of every parameter array."""
    lq = gen.kuka_lq(6, 3, 6, 77)
    w = gen.loss_weights(6 * 6, 4).reshape(6, 6)

    def L(lq_):
        lam, dx, du = oracle.kkt_solve(lq_)
        return oracle.loss(lam, dx, du, w)

    lam, dx, du = oracle.kkt_solve(lq)
    g = oracle.grad(lq, lam, dx, du, w, 2 * dx, 2 * du)
    rng = np.random.default_rng(4)
    h = 1e-6
    # central differences carry a rounding error of about eps |L| / h
    round_err = 50 * np.finfo(np.float64).eps * abs(L(lq)) / h
    for name in ("A", "B", "Qd", "Rd", "q", "r", "c"):
        arr = getattr(lq, name)
        for _ in range(8):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            p = lq.copy()
            m = lq.copy()
            getattr(p, name)[idx] += h
            getattr(m, name)[idx] -= h
            fd = (L(p) - L(m)) / (2 * h)
            an = g[name][idx]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + round_err, (name, idx, fd, an)


# ---------------------------------------------------------------- block-Jacobi comparison preconditioner
def test_jacobi_blocks_invert_the_block_diagonal():
    lq = gen.kuka_lq(14, 7, 20, 31)
    Sd, So, _ = oracle.schur_blocks(lq)
    Jd, Jo = oracle.jacobi_blocks(Sd, So)
    assert np.all(Jo == 0.0)
    eye = np.broadcast_to(np.eye(14), Sd.shape)
    assert np.abs(np.einsum("kij,kjl->kil", Jd, Sd) - eye).max() < 1e-10


def test_jacobi_pcg_matches_scipy_preconditioned_cg():
    """Algorithm 1 with Phi^-1 = D^-1 against scipy's CG given the same
    preconditioner as a LinearOperator (an independent PCG)."""
    import scipy.sparse.linalg as spla
    lq = gen.kuka_lq(4, 2, 12, 19)
    Sd, So, gamma = oracle.schur_blocks(lq)
    Jd, Jo = oracle.jacobi_blocks(Sd, So)
    lam_p, it, ok = oracle.pcg(Sd, So, Jd, Jo, -gamma, tol=1e-11)
    S = oracle.block_tridiag_sparse(Sd, So)
    Dinv = np.linalg.inv(Sd)
    M = spla.LinearOperator(S.shape, matvec=lambda v: np.einsum("kij,kj->ki", Dinv, v.reshape(Sd.shape[:2])).ravel())
    x, info = spla.cg(S, -gamma.ravel(), M=M, rtol=1e-13, maxiter=10000)
    assert ok and info == 0 and oracle.relerr(lam_p, x) < 1e-8


def test_jacobi_decoupled_converges_in_one_iteration():
    lq = gen.kuka_lq(6, 3, 10, 23)
    lq.A[:] = 0.0
    lq.B[:] = 0.0
    Sd, So, gamma = oracle.schur_blocks(lq)
    Jd, Jo = oracle.jacobi_blocks(Sd, So)
    lam_p, it, ok = oracle.pcg(Sd, So, Jd, Jo, -gamma, tol=1e-12)
    lam, _, _ = oracle.kkt_solve(lq)
    assert ok and it == 1 and oracle.relerr(lam_p, lam) < 1e-13


def test_symmetric_stair_needs_fewer_iterations_than_block_jacobi():
    """The reason Sec. IV-A adds the off-diagonal blocks: on the Kuka-shaped
    workload the symmetric stair preconditioner roughly halves the PCG
    iterations of block Jacobi."""
    lq = gen.kuka_lq(14, 7, 128, 130)
    Sd, So, gamma = oracle.schur_blocks(lq)
    _, it_s, ok_s = oracle.pcg(Sd, So, *oracle.precon_blocks(Sd, So), -gamma, tol=1e-6)
    _, it_j, ok_j = oracle.pcg(Sd, So, *oracle.jacobi_blocks(Sd, So), -gamma, tol=1e-6)
    assert ok_s and ok_j and it_s < 0.7 * it_j, (it_s, it_j)



# ---------------------------------------------------------------- stair (non-symmetric) comparison preconditioner
@pytest.mark.parametrize("N", [1, 2, 7, 12])
@pytest.mark.parametrize("odd", [True, False])
def test_stair_inverse_inverts_the_stair_matrix(N, odd):
    """The closed-form stair inverse against the stair matrix built from the
    blocks of S+ directly (dense product = identity), and its pattern: rows
    without neighbours hold D_k^-1 alone."""
    lq = gen.kuka_lq(6, 3, N, 40 + N)
    Sd, So, _ = oracle.schur_blocks(lq)
    P = oracle.stair_matrix(Sd, So, odd).toarray()
    Pi = oracle.stair_inverse(Sd, So, odd).toarray()
    assert np.abs(Pi @ P - np.eye(P.shape[0])).max() < 1e-10
    nx = 6
    for k in range(N):
        if (k % 2 == 1) != odd:
            row = Pi[k * nx:(k + 1) * nx]
            off = np.delete(row, np.s_[k * nx:(k + 1) * nx], axis=1)
            assert np.all(off == 0.0)


def test_symmetric_stair_is_the_sum_of_the_two_stair_inverses():
    """Phi^-1 of Sec. IV-A = P_odd^-1 + P_even^-1 - D^-1 with each stair
    matrix inverted densely (np.linalg.inv, not the closed form): pins
    precon_blocks through the construction of the cited work."""
    lq = gen.kuka_lq(14, 7, 9, 77)
    Sd, So, _ = oracle.schur_blocks(lq)
    Pd, Po = oracle.precon_blocks(Sd, So)
    Phi = oracle.block_tridiag_sparse(Pd, Po).toarray()
    Lo = np.linalg.inv(oracle.stair_matrix(Sd, So, True).toarray())
    Le = np.linalg.inv(oracle.stair_matrix(Sd, So, False).toarray())
    Dinv = np.linalg.inv(oracle.block_tridiag_sparse(Sd, np.zeros_like(So)).toarray())
    assert np.abs(Lo + Le - Dinv - Phi).max() <= 1e-10 * np.abs(Phi).max()


def test_stair_pcg_converges_on_a_short_horizon_and_not_on_a_long_one():
    """The reason for the symmetric form: with the non-symmetric stair
    preconditioner Algorithm 1 loses its guarantees.  On the Kuka-shaped
    workload it still reaches the KKT solution at N = 8 but stalls at
    N = 32 (10 N nx iterations), where the symmetric stair converges."""
    for N, expect in ((8, True), (32, False)):
        lq = gen.kuka_lq(14, 7, N, 2 + N)
        Sd, So, g = oracle.schur_blocks(lq)
        S = oracle.block_tridiag_sparse(Sd, So)
        lam, it, ok = oracle.pcg_op(S, oracle.stair_inverse(Sd, So), -g, tol=1e-8)
        assert ok == expect, (N, it)
        if ok:
            lo, _, _ = oracle.kkt_solve(lq)
            assert oracle.relerr(lam, lo) < 1e-6
    _, _, ok = oracle.pcg(Sd, So, *oracle.precon_blocks(Sd, So), -g, tol=1e-8)
    assert ok


# ---------------------------------------------------------------- dense SPD cost blocks
def test_dense_blocks_with_diagonal_values_match_the_diagonal_problem():
    """Q_k = diag(Qd_k), R_k = diag(Rd_k) given as dense blocks: the same
    solution as the diagonal statement of the problem."""
    lq = gen.kuka_lq(14, 7, 40, 41)
    dq = lq.copy()
    dq.Q = np.stack([np.diag(v) for v in lq.Qd])
    dq.R = np.stack([np.diag(v) for v in lq.Rd])
    a, b = oracle.kkt_solve(lq), oracle.kkt_solve(dq)
    for x, y in zip(a, b):
        assert oracle.relerr(y, x) < 1e-13


def test_dense_invariants():
    """Linearised dynamics and stationarity G dz + g - C^T lambda = 0 with
    dense cost blocks."""
    lq = gen.kuka_lq(14, 7, 64, 43, dense=True)
    lam, dx, du = oracle.kkt_solve(lq)
    res = dx[1:] - np.einsum("kij,kj->ki", lq.A, dx[:-1]) - np.einsum("kij,kj->ki", lq.B, du) + lq.c[1:]
    assert np.abs(res).max() < 1e-11 and np.abs(dx[0] + lq.c[0]).max() < 1e-12
    sx = np.einsum("kij,kj->ki", lq.Q, dx) + lq.q - lam
    sx[:-1] += np.einsum("kji,kj->ki", lq.A, lam[1:])
    su = np.einsum("kij,kj->ki", lq.R, du) + lq.r + np.einsum("kji,kj->ki", lq.B, lam[1:])
    sc = max(1.0, np.abs(lam).max() * 10)
    assert np.abs(sx).max() < 1e-11 * sc and np.abs(su).max() < 1e-11 * sc


def test_dense_schur_route_reaches_kkt_solution():
    lq = gen.kuka_lq(14, 7, 48, 47, dense=True)
    Sd, So, gamma = oracle.schur_blocks(lq)
    S = oracle.block_tridiag_sparse(Sd, So).toarray()
    np.linalg.cholesky(S)
    lam_s = np.linalg.solve(S, -gamma.ravel()).reshape(lq.N, lq.nx)
    lam, dx, du = oracle.kkt_solve(lq)
    assert oracle.relerr(lam_s, lam) < 1e-11
    dx2, du2 = oracle.recover(lq, lam)
    assert oracle.relerr(dx2, dx) < 1e-12 and oracle.relerr(du2, du) < 1e-12
