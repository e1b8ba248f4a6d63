"""ORACLE -- test infrastructure, not part of the product.

Plain FP64 statements of each step of the linear-solve path, written from
the paper's definitions.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may use this module.

Functions and the passage each follows:

  kkt_solve      exact (lambda, dz) of the KKT system, Sec. II-A Step 2
                 (Eq. KKT); banded LU with partial pivoting in kkt_band.c.
  schur_blocks   S+ = C G^-1 C^T and gamma = c - C G^-1 g by their
                 definition, Sec. II-B (Eq. schur), as sparse products.
  precon_blocks  symmetric stair preconditioner Phi^-1, Sec. IV-A: diagonal
                 blocks D_k^-1, off-diagonal blocks -D_{k+1}^-1 phi_k D_k^-1.
  stair_matrix,  the non-symmetric stair matrix of S+ (odd block rows keep
  stair_inverse  their neighbours) and its closed-form inverse: the
                 comparison preconditioner of the work Sec. IV-A cites.
  jacobi_blocks  block Jacobi Phi^-1 = D^-1 (comparison preconditioner).
  pcg, pcg_op    Algorithm 1 (PCG) with the exit tests described below
                 (pcg_op: operators as matrices, Phi^-1 may be non-symmetric).
  recover        dz = -G^-1 (g - C^T lambda), Sec. II-B (Eq. schur).
  grad           gradient of a scalar loss of (lambda, dz) through the exact
                 KKT solution (implicit-function theorem on Eq. KKT).

Sign reading (Sec. II-B): the paper writes S = -C G^-1 C^T and S lambda =
gamma; with G positive definite that S is negative definite, so the
positive definite form S+ = C G^-1 C^T with right-hand side b = -gamma is
used.  Both give the same lambda.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kkt_band.c")
_LIB = os.path.join(_HERE, "_kkt_band.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile kkt_band.c with the host gcc (plain -O2, no BLAS)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", _SRC,
                               "-o", _LIB, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_kkt_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         dp, dp, dp, dp, dp, dp]
        lib.oracle_kkt_solve.restype = ctypes.c_int
        lib.oracle_kkt_solve_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           dp, dp, dp, dp, dp, dp, dp, dp]
        lib.oracle_kkt_solve_g.restype = ctypes.c_int
        lib.oracle_kkt_dim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_kkt_dim.restype = ctypes.c_long
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def kkt_dim(nx: int, nu: int, N: int) -> int:
    return 2 * N * nx + (N - 1) * nu


def natural_z(dx: np.ndarray, du: np.ndarray) -> np.ndarray:
    """Interleave (x_0, u_0, x_1, u_1, ..., x_{N-1}) into one vector."""
    N, nx = dx.shape
    nu = du.shape[1] if du.size else 0
    z = np.empty(N * nx + (N - 1) * nu)
    for k in range(N):
        z[k * (nx + nu): k * (nx + nu) + nx] = dx[k]
        if k < N - 1:
            z[k * (nx + nu) + nx: (k + 1) * (nx + nu)] = du[k]
    return z


def split_z(z: np.ndarray, nx: int, nu: int, N: int) -> Tuple[np.ndarray, np.ndarray]:
    dx = np.empty((N, nx))
    du = np.empty((max(N - 1, 0), nu))
    for k in range(N):
        dx[k] = z[k * (nx + nu): k * (nx + nu) + nx]
        if k < N - 1:
            du[k] = z[k * (nx + nu) + nx: (k + 1) * (nx + nu)]
    return dx, du


def kkt_solve_rhs(lq, h: np.ndarray) -> np.ndarray:
    """Solve K y = h for the KKT matrix K of `lq` (natural ordering)."""
    lib = _load()
    A, B, Qd, Rd = (_f64(getattr(lq, f)) for f in ("A", "B", "Qd", "Rd"))
    h = _f64(h).copy()
    y = np.empty_like(h)
    if _dense(lq):
        Q, R = _f64(lq.Q), _f64(lq.R)
        st = lib.oracle_kkt_solve_g(lq.nx, lq.nu, lq.N, _dp(A), _dp(B), _dp(Qd), _dp(Rd),
                                    _dp(Q), _dp(R), _dp(h), _dp(y))
    else:
        st = lib.oracle_kkt_solve(lq.nx, lq.nu, lq.N, _dp(A), _dp(B), _dp(Qd), _dp(Rd),
                                  _dp(h), _dp(y))
    if st != 0:
        raise RuntimeError(f"oracle KKT solve failed with status {st}")
    return y


def kkt_solve(lq):
    """Exact (lambda, dx, du) of Eq. KKT: [G C^T; C 0][-dz; lambda] = [g; c]."""
    nx, nu, N = lq.nx, lq.nu, lq.N
    g = natural_z(_f64(lq.q), _f64(lq.r))
    h = np.concatenate([g, _f64(lq.c).ravel()])
    y = kkt_solve_rhs(lq, h)
    nz = N * nx + (N - 1) * nu
    dx, du = split_z(-y[:nz], nx, nu, N)
    lam = y[nz:].reshape(N, nx)
    return lam, dx, du


def solve_batch(batch):
    """kkt_solve for every instance of an LQBatch; concatenated outputs."""
    outs = [kkt_solve(it) for it in batch.items]
    return (np.concatenate([o[0] for o in outs]), np.concatenate([o[1] for o in outs]),
            np.concatenate([o[2] for o in outs]))


# --------------------------------------------------------------------------
# Sparse statements of G, C, g (Sec. II-A, Step 2) for the definitions below.
# --------------------------------------------------------------------------
def _C_sparse(lq) -> sp.csr_matrix:
    nx, nu, N = lq.nx, lq.nu, lq.N
    A, B = _f64(lq.A), _f64(lq.B)
    rows, cols, vals = [], [], []

    def put(r0, c0, M):
        rr, cc = np.nonzero(np.ones_like(M, dtype=bool))
        rows.extend((r0 + rr).tolist())
        cols.extend((c0 + cc).tolist())
        vals.extend(M[rr, cc].tolist())

    put(0, 0, np.eye(nx))
    for k in range(N - 1):
        r0 = (k + 1) * nx
        put(r0, k * (nx + nu), -A[k])
        put(r0, k * (nx + nu) + nx, -B[k])
        put(r0, (k + 1) * (nx + nu), np.eye(nx))
    nz = N * nx + (N - 1) * nu
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * nx, nz))


def _dense(lq) -> bool:
    return getattr(lq, "Q", None) is not None


def _G_diag(lq) -> np.ndarray:
    return natural_z(_f64(lq.Qd), _f64(lq.Rd))


def _Ginv_sparse(lq) -> sp.csr_matrix:
    """G^-1 = blockdiag(Q_0^-1, R_0^-1, ..., Q_{N-1}^-1): reciprocals of the
    diagonals, or inverses of the dense SPD cost blocks."""
    if not _dense(lq):
        return sp.diags(1.0 / _G_diag(lq)).tocsr()
    Q, R = _f64(lq.Q), _f64(lq.R)
    rows, cols, vals = [], [], []
    o = 0
    for k in range(lq.N):
        for M in ([Q[k], R[k]] if k < lq.N - 1 else [Q[k]]):
            n = M.shape[0]
            ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            rows.append((o + ii).ravel())
            cols.append((o + jj).ravel())
            vals.append(np.linalg.inv(M).ravel())
            o += n
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(o, o))


def _g_vec(lq) -> np.ndarray:
    return natural_z(_f64(lq.q), _f64(lq.r))


def schur_blocks(lq):
    """S+ = C G^-1 C^T and gamma = c - C G^-1 g (Eq. schur), by definition.

    Returns the block-tridiagonal S+ as Sd[N][nx][nx] (diagonal blocks) and
    So[N-1][nx][nx] (So[k] = block (k+1, k)), plus gamma[N][nx].
    """
    nx, N = lq.nx, lq.N
    C = _C_sparse(lq)
    Ginv = _Ginv_sparse(lq)
    S = (C @ Ginv @ C.T).toarray() if N * nx <= 4096 else (C @ Ginv @ C.T).tocsr()
    gamma = _f64(lq.c).ravel() - C @ (Ginv @ _g_vec(lq))
    Sd = np.empty((N, nx, nx))
    So = np.empty((max(N - 1, 0), nx, nx))
    for k in range(N):
        blk = S[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx]
        Sd[k] = blk.toarray() if sp.issparse(blk) else blk
        if k < N - 1:
            blk = S[(k + 1) * nx:(k + 2) * nx, k * nx:(k + 1) * nx]
            So[k] = blk.toarray() if sp.issparse(blk) else blk
    return Sd, So, gamma.reshape(N, nx)


def precon_blocks(Sd: np.ndarray, So: np.ndarray):
    """Symmetric stair preconditioner Phi^-1 (Sec. IV-A).

    Diagonal blocks are the inverses of S+'s diagonal blocks (Q_0 for knot 0,
    theta_{k-1}^-1 after it); the block below the diagonal in block column k
    is -D_{k+1}^-1 phi_k D_k^-1, and the block above is its transpose, which
    reproduces every block printed in Sec. IV-A.
    """
    Pd = np.linalg.inv(Sd)
    Po = np.empty_like(So)
    for k in range(So.shape[0]):
        Po[k] = -Pd[k + 1] @ So[k] @ Pd[k]
    return Pd, Po


def jacobi_blocks(Sd: np.ndarray, So: np.ndarray):
    """Block-Jacobi preconditioner Phi^-1 = D^-1 (the block diagonal of S+
    inverted; no off-diagonal blocks): the comparison baseline for the
    symmetric stair preconditioner of Sec. IV-A."""
    return np.linalg.inv(Sd), np.zeros_like(So)


def stair_matrix(Sd: np.ndarray, So: np.ndarray, odd: bool = True) -> sp.csr_matrix:
    """The (non-symmetric) stair matrix of S+: every block row keeps its
    diagonal block; the odd block rows (even ones if odd=False) also keep
    their two off-diagonal blocks of S+.  The preconditioner the symmetric
    stair preconditioner of Sec. IV-A (and its cited work) is built from."""
    N = Sd.shape[0]
    blocks = [[None] * N for _ in range(N)]
    for k in range(N):
        blocks[k][k] = sp.csr_matrix(Sd[k])
        if (k % 2 == 1) == odd:
            if k >= 1:
                blocks[k][k - 1] = sp.csr_matrix(So[k - 1])
            if k + 1 < N:
                blocks[k][k + 1] = sp.csr_matrix(So[k].T)
    return sp.bmat(blocks, format="csr")


def stair_inverse(Sd: np.ndarray, So: np.ndarray, odd: bool = True) -> sp.csr_matrix:
    """Inverse of stair_matrix(Sd, So, odd), in closed form: block row k is
    D_k^-1 alone in the rows without neighbours; in the others it is
    (-D_k^-1 O_{k,k-1} D_{k-1}^-1, D_k^-1, -D_k^-1 O_{k,k+1} D_{k+1}^-1),
    because the neighbouring rows of such a row are diagonal.  These are the
    rows of the symmetric stair Phi^-1 with the other rows' off-diagonal
    blocks dropped."""
    N = Sd.shape[0]
    Pd = np.linalg.inv(Sd)
    blocks = [[None] * N for _ in range(N)]
    for k in range(N):
        blocks[k][k] = sp.csr_matrix(Pd[k])
        if (k % 2 == 1) == odd:
            if k >= 1:
                blocks[k][k - 1] = sp.csr_matrix(-Pd[k] @ So[k - 1] @ Pd[k - 1])
            if k + 1 < N:
                blocks[k][k + 1] = sp.csr_matrix(-Pd[k] @ So[k].T @ Pd[k + 1])
    return sp.bmat(blocks, format="csr")


def block_tridiag_sparse(Dd: np.ndarray, Do: np.ndarray) -> sp.csr_matrix:
    """Assemble a symmetric block-tridiagonal matrix from Dd and Do (below)."""
    N, nx, _ = Dd.shape
    blocks = [[None] * N for _ in range(N)]
    for k in range(N):
        blocks[k][k] = sp.csr_matrix(Dd[k])
        if k < N - 1:
            blocks[k + 1][k] = sp.csr_matrix(Do[k])
            blocks[k][k + 1] = sp.csr_matrix(Do[k].T)
    return sp.bmat(blocks, format="csr")


def dense_S(lq) -> np.ndarray:
    """Dense S+ = C G^-1 C^T (small problems only)."""
    C = _C_sparse(lq).toarray()
    return C @ _Ginv_sparse(lq).toarray() @ C.T


def dense_Phi_inv(Sd: np.ndarray, So: np.ndarray) -> np.ndarray:
    """Dense D^-1 - D^-1 O D^-1 restricted to the block-tridiagonal pattern.

    D is the block diagonal of S+ and O its off-diagonal part; because O has
    zero diagonal blocks the product D^-1 O D^-1 is itself block-tridiagonal.
    """
    N, nx, _ = Sd.shape
    S = block_tridiag_sparse(Sd, So).toarray()
    D = np.zeros_like(S)
    for k in range(N):
        D[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx] = Sd[k]
    O = S - D
    Dinv = np.linalg.inv(D)
    return Dinv - Dinv @ O @ Dinv


def pcg(Sd, So, Pd, Po, b, lam0=None, tol=1e-6, tol_mode=0, max_iter=None):
    """Algorithm 1 (PCG) on S+ lambda = b with preconditioner Phi^-1.

    Exit tests: tol_mode 0 stops when ||r||_2 <= tol ||b||_2 (r the
    recurrence residual); tol_mode 1 is the paper's eta' = r^T Phi^-1 r < tol.
    A starting point that already passes the test returns with 0 iterations.
    Returns (lambda, iterations, converged).
    """
    return pcg_op(block_tridiag_sparse(Sd, So), block_tridiag_sparse(Pd, Po), b, lam0, tol,
                  tol_mode, max_iter)


def pcg_op(S, P, b, lam0=None, tol=1e-6, tol_mode=0, max_iter=None):
    """Algorithm 1 with S+ and Phi^-1 given as (sparse) matrices; Phi^-1 may
    be non-symmetric (the stair preconditioner).  Same exits and returns as
    pcg()."""
    b = _f64(b).ravel()
    n = b.size
    lam = np.zeros(n) if lam0 is None else _f64(lam0).ravel().copy()
    if max_iter is None:
        max_iter = 10 * n
    bnorm = np.linalg.norm(b)

    def done(r, eta):
        return (np.linalg.norm(r) <= tol * bnorm) if tol_mode == 0 else (eta < tol)

    r = b - S @ lam
    rt = P @ r
    p = rt.copy()
    eta = r @ rt
    if done(r, eta):
        return lam, 0, True
    for it in range(1, max_iter + 1):
        Sp = S @ p
        alpha = eta / (p @ Sp)
        r = r - alpha * Sp
        lam = lam + alpha * p
        rt = P @ r
        eta_new = r @ rt
        if done(r, eta_new):
            return lam, it, True
        beta = eta_new / eta
        p = rt + beta * p
        eta = eta_new
    return lam, max_iter, False


def recover(lq, lam: np.ndarray):
    """dz = -G^-1 (g - C^T lambda) (Eq. schur), by definition."""
    C = _C_sparse(lq)
    z = -(_Ginv_sparse(lq) @ (_g_vec(lq) - C.T @ _f64(lam).ravel()))
    return split_z(z, lq.nx, lq.nu, lq.N)


def loss(lam, dx, du, w):
    """Scalar loss sum ||dz||^2 + w^T lambda."""
    return float(np.sum(dx * dx) + np.sum(du * du) + np.dot(w.ravel(), np.ravel(lam)))


def grad(lq, lam, dx, du, l_lam, l_dx, l_du):
    """Gradient of a scalar loss L(lambda, dz) through the exact KKT solution.

    With K y = h, y = (-dz, lambda), h = (g, c): the adjoint a solves
    K a = dL/dy (K is symmetric), then dL/dh = a and dL/dK = -a y^T.
    Reading K's entries back to the parameters:
      Qd_k, Rd_k  : diagonal of G            -> -a_z * y_z
      q_k, r_k    : g                        ->  a_z
      c_k         : c                        ->  a_lam
      A_k, B_k    : C holds -A_k, -B_k in block row k+1 (and C^T in the
                    transposed position)     ->  a_lam,k+1 y_z^T + lam_{k+1} a_z^T
    Returns a dict with the layouts of the inputs.
    """
    if _dense(lq):
        raise NotImplementedError("the gradient is stated for diagonal cost blocks")
    nx, nu, N = lq.nx, lq.nu, lq.N
    nz = N * nx + (N - 1) * nu
    yz = -natural_z(_f64(dx), _f64(du))
    ybar = np.concatenate([-natural_z(_f64(l_dx), _f64(l_du)), _f64(l_lam).ravel()])
    a = kkt_solve_rhs(lq, ybar)
    az, al = a[:nz], a[nz:].reshape(N, nx)
    gG = -az * yz
    gQd, gRd = split_z(gG, nx, nu, N)
    gq, gr = split_z(az, nx, nu, N)
    yx, yu = split_z(yz, nx, nu, N)
    azx, azu = gq, gr
    lam = _f64(lam).reshape(N, nx)
    gA = np.empty((N - 1, nx, nx))
    gB = np.empty((N - 1, nx, nu))
    for k in range(N - 1):
        gA[k] = np.outer(al[k + 1], yx[k]) + np.outer(lam[k + 1], azx[k])
        gB[k] = np.outer(al[k + 1], yu[k]) + np.outer(lam[k + 1], azu[k])
    return dict(A=gA, B=gB, Qd=gQd, Rd=gRd, q=gq, r=gr, c=al.copy())


def relerr(x, ref) -> float:
    """Normwise relative error ||x - ref||_2 / ||ref||_2."""
    x = np.asarray(x, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))
