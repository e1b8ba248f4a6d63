"""Independent statements used to pin the oracle (test-side only).

Nothing here is imported by the oracle or by the product.  Each routine
reaches the same quantity by a different route than the oracle does.
"""
import numpy as np


def dense_kkt(lq):
    """Dense KKT matrix [G C^T; C 0] and rhs [g; c] in the paper's natural
    ordering (Sec. II-A, Step 2), assembled entry by entry."""
    nx, nu, N = lq.nx, lq.nu, lq.N
    nz = N * nx + (N - 1) * nu
    n = nz + N * nx
    K = np.zeros((n, n))
    h = np.zeros(n)

    def xi(k):
        return k * (nx + nu)

    def ui(k):
        return k * (nx + nu) + nx

    dense = getattr(lq, "Q", None) is not None
    for k in range(N):
        for i in range(nx):
            if dense:
                for j in range(nx):
                    K[xi(k) + i, xi(k) + j] = lq.Q[k][i][j]
            else:
                K[xi(k) + i, xi(k) + i] = lq.Qd[k][i]
            h[xi(k) + i] = lq.q[k][i]
        if k < N - 1:
            for i in range(nu):
                if dense:
                    for j in range(nu):
                        K[ui(k) + i, ui(k) + j] = lq.R[k][i][j]
                else:
                    K[ui(k) + i, ui(k) + i] = lq.Rd[k][i]
                h[ui(k) + i] = lq.r[k][i]
    C = np.zeros((N * nx, nz))
    C[0:nx, xi(0):xi(0) + nx] = np.eye(nx)
    for k in range(N - 1):
        rr = (k + 1) * nx
        C[rr:rr + nx, xi(k):xi(k) + nx] = -lq.A[k]
        C[rr:rr + nx, ui(k):ui(k) + nu] = -lq.B[k]
        C[rr:rr + nx, xi(k + 1):xi(k + 1) + nx] = np.eye(nx)
    K[nz:, :nz] = C
    K[:nz, nz:] = C.T
    h[nz:] = np.asarray(lq.c, dtype=np.float64).ravel()
    return K, h, C


def riccati(lq):
    """Affine discrete-time LQR by the backward Riccati recursion.

    Problem: min sum 1/2 dx'Q dx + q'dx + 1/2 du'R du + r'du subject to
    dx_0 = -c_0 and dx_{k+1} = A_k dx_k + B_k du_k - c_{k+1}, which is the
    constraint block C dz + c = 0 of Eq. KKT.  Multipliers follow from the
    value-function gradient lam_k = P_k dx_k + p_k.
    """
    nx, nu, N = lq.nx, lq.nu, lq.N
    A = np.asarray(lq.A, np.float64)
    B = np.asarray(lq.B, np.float64)
    if getattr(lq, "Q", None) is not None:
        Q = [np.asarray(lq.Q[k], np.float64) for k in range(N)]
        R = [np.asarray(lq.R[k], np.float64) for k in range(N - 1)]
    else:
        Q = [np.diag(np.asarray(lq.Qd[k], np.float64)) for k in range(N)]
        R = [np.diag(np.asarray(lq.Rd[k], np.float64)) for k in range(N - 1)]
    q = np.asarray(lq.q, np.float64)
    r = np.asarray(lq.r, np.float64)
    c = np.asarray(lq.c, np.float64)
    P = [None] * N
    p = [None] * N
    K = [None] * (N - 1)
    kff = [None] * (N - 1)
    P[N - 1] = Q[N - 1].copy()
    p[N - 1] = q[N - 1].copy()
    for k in range(N - 2, -1, -1):
        d = -c[k + 1]
        Pn, pn = P[k + 1], p[k + 1]
        Qxx = Q[k] + A[k].T @ Pn @ A[k]
        Quu = R[k] + B[k].T @ Pn @ B[k]
        Qux = B[k].T @ Pn @ A[k]
        Qx = q[k] + A[k].T @ (Pn @ d + pn)
        Qu = r[k] + B[k].T @ (Pn @ d + pn)
        K[k] = -np.linalg.solve(Quu, Qux)
        kff[k] = -np.linalg.solve(Quu, Qu)
        P[k] = Qxx + Qux.T @ K[k]
        P[k] = 0.5 * (P[k] + P[k].T)
        p[k] = Qx + Qux.T @ kff[k]
    dx = np.zeros((N, nx))
    du = np.zeros((N - 1, nu))
    dx[0] = -c[0]
    for k in range(N - 1):
        du[k] = K[k] @ dx[k] + kff[k]
        dx[k + 1] = A[k] @ dx[k] + B[k] @ du[k] - c[k + 1]
    lam = np.stack([P[k] @ dx[k] + p[k] for k in range(N)])
    return lam, dx, du
