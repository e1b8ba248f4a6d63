"""ORACLE -- test infrastructure, not part of the product.

Plain FP64 numpy statement of the outer loop around the solve path for the
synthetic model of ``workload.gen.Model``: the dynamics and their exact
Jacobians, Step 1 of Sec. II-A (the LQ subproblem of the QP at the current
trajectory), Step 3 with the parallel line search of Sec. IV-C (every step
size of a halving set evaluated, the smallest L1 merit kept), and the SQP
iteration that strings them together with the oracle's KKT solve.
"""
from __future__ import annotations

import numpy as np

from workload.gen import LQ
from .oracle import kkt_solve


def _split(model, x):
    h = model.nx // 2
    return x[..., :h], x[..., h:]


def dynamics(model, x, u):
    """x+ = f(x, u): v+ = v + dt (P u - damp v - stiff sin p), p+ = p + dt v+."""
    p, v = _split(model, np.asarray(x, np.float64))
    vn = v + model.dt * (np.asarray(u, np.float64) @ np.asarray(model.P, np.float64).T
                         - model.damp * v - model.stiff * np.sin(p))
    pn = p + model.dt * vn
    return np.concatenate([pn, vn], axis=-1)


def jacobians(model, x, u):
    """A = df/dx, B = df/du at one (x, u)."""
    h, dt = model.nx // 2, model.dt
    p, _ = _split(model, np.asarray(x, np.float64))
    dvdp = -dt * np.diag(model.stiff * np.cos(p))
    dvdv = np.eye(h) - dt * np.diag(model.damp)
    dvdu = dt * np.asarray(model.P, np.float64)
    A = np.block([[np.eye(h) + dt * dvdp, dt * dvdv], [dvdp, dvdv]])
    B = np.vstack([dt * dvdu, dvdu])
    return A, B


def cost(model, trk, X, U):
    """J = sum_k l(x_k, u_k) + l_f(x_{N-1})."""
    X, U = np.asarray(X, np.float64), np.asarray(U, np.float64)
    e = X - trk.xref
    J = 0.5 * np.sum(model.wq * e[:-1] ** 2) + 0.5 * np.sum(model.wr * U ** 2)
    return J + 0.5 * np.sum(model.wf * e[-1] ** 2)


def defects(model, trk, X, U):
    """c of Eq. KKT: (x_0 - x_s, x_{k+1} - f(x_k, u_k))."""
    X, U = np.asarray(X, np.float64), np.asarray(U, np.float64)
    c = np.empty_like(X)
    c[0] = X[0] - trk.xs
    if trk.N > 1:
        c[1:] = X[1:] - dynamics(model, X[:-1], U)
    return c


def linearize(model, trk, X, U) -> LQ:
    """Step 1 of Sec. II-A at (X, U): A_k, B_k, diagonal Q_k, R_k, gradients
    q_k, r_k and defects c_k of the QP for the step (dX, dU)."""
    nx, nu, N = model.nx, model.nu, trk.N
    X, U = np.asarray(X, np.float64), np.asarray(U, np.float64)
    A = np.empty((N - 1, nx, nx))
    B = np.empty((N - 1, nx, nu))
    for k in range(N - 1):
        A[k], B[k] = jacobians(model, X[k], U[k])
    Qd = np.tile(np.asarray(model.wq, np.float64), (N, 1))
    Qd[-1] = model.wf
    Rd = np.tile(np.asarray(model.wr, np.float64), (N - 1, 1))
    q = Qd * (X - trk.xref)
    r = Rd * U
    return LQ(nx, nu, N, A, B, Qd, Rd, q, r, defects(model, trk, X, U))


def merit(model, trk, X, U, mu):
    """L1 merit: J + mu * ||c||_1."""
    return cost(model, trk, X, U) + mu * np.abs(defects(model, trk, X, U)).sum()


def penalty(lam):
    """mu = 1.1 max(1, ||lambda||_inf): above the multipliers' magnitude, the
    condition under which the L1 merit is exact."""
    return 1.1 * max(1.0, float(np.abs(lam).max()))


def line_search(model, trk, X, U, dX, dU, mu, n_alpha=9):
    """Sec. IV-C: merits of (X, U) + a (dX, dU) for a in {1, 1/2, ...,
    2^-(n_alpha-1)}; the smallest merit wins, merits within a relative 1e-11
    of it (below the rounding of their FP64 sums) count as ties, and the
    longest tied step is taken.  Returns (X', U', index, merits)."""
    X, U, dX, dU = (np.asarray(a) for a in (X, U, dX, dU))
    t = X.dtype.type  # candidates are formed in the trajectory's own precision
    alphas = [t(0.5 ** a) for a in range(n_alpha)]
    m = np.array([merit(model, trk, X + a * dX, U + a * dU, mu) for a in alphas])
    best = np.nanmin(m)
    i = int(np.nonzero(m <= best + 1e-11 * abs(best))[0][0])
    return X + alphas[i] * dX, U + alphas[i] * dU, i, m


def sqp(model, trk, iters, n_alpha=9):
    """SQP iterations from the tracking problem's initial guess: linearise,
    solve the KKT system, line-search.  Returns the trajectory after each
    iteration with the chosen step index and merit."""
    X, U = np.asarray(trk.X, np.float64).copy(), np.asarray(trk.U, np.float64).copy()
    hist = []
    for _ in range(iters):
        lq = linearize(model, trk, X, U)
        lam, dX, dU = kkt_solve(lq)
        mu = penalty(lam)
        X, U, i, m = line_search(model, trk, X, U, dX, dU, mu, n_alpha)
        hist.append(dict(X=X.copy(), U=U.copy(), idx=i, merits=m, mu=mu, lam=lam))
    return hist
