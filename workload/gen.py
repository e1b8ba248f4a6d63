"""Seeded, synthetic, Kuka-shaped LQ subproblems (Sec. II-A, Step 1 output).

The paper's measurements use the LQ subproblems produced inside 100 NMPC
trials of a simulated Kuka IIWA-14 (Sec. V-A).  Those traces are not
available, so every input here is drawn from a seeded generator with the
same shapes (nx = 14 states = 7 joint positions + 7 velocities, nu = 7
torques, 32..512 knot points) and a semi-implicit-Euler structure for the
dynamics Jacobians:

    A_k = [[I, dt I], [dt M_k, I + dt D_k]]       M_k, D_k ~ N(0, 0.5^2)
    B_k = [[0], [dt (L_k L_k^T + 0.1 I)[:, :nu]]] L_k ~ N(0, 1), (nx/2)x(nx/2)
    Qd_k ~ U[1, 10]   (diagonal of Q_k)      Rd_k ~ U[0.01, 0.1] (diag of R_k)
    q_k, r_k, c_k ~ N(0, 1)

Index convention: N is the number of knot points, i.e. the number of state
blocks x_0..x_{N-1} and of block rows of the Schur complement; controls are
u_0..u_{N-2}.  Array layouts (row-major, float64 master copies):

    A[N-1][nx][nx]  B[N-1][nx][nu]  Qd[N][nx]  Rd[N-1][nu]
    q[N][nx]        r[N-1][nu]      c[N][nx]
    Q[N][nx][nx]    R[N-1][nu][nu]  (optional dense SPD cost blocks)

Draw order per instance (numpy default_rng(seed)): M, Dm, L, Qd, Rd, q, r, c.
No solver arithmetic lives here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# Workload definitions (shapes, seeds, distributions) of the five measured
# configurations.  Each is plain data.
CONFIG_SMALL = dict(name="single-N32", nx=14, nu=7, N=32, seed=1, dt=0.01,
                    qd=(1.0, 10.0))
CONFIG_SWEEP = dict(name="sweep", nx=14, nu=7, Ns=(64, 128, 256, 512),
                    seed_base=2, dt=0.01, qd=(1.0, 10.0), noise=0.01, reps=1000)
CONFIG_BATCH = dict(name="batch256", nx=14, nu=7, B=256, N_lo=32, N_hi=512,
                    n_seed=3, seed_base=1000, dt=0.01, qd=(1.0, 10.0),
                    noise=0.01, solves=20)
CONFIG_GRAD = dict(name="grad64", nx=14, nu=7, B=64, N=128, seed_base=4000,
                   w_seed=4, dt=0.01, qd=(1.0, 10.0), fd_coords=50, fd_h=1e-6)
CONFIG_LARGE = dict(name="large1024", nx=36, nu=12, B=1024, N_lo=64, N_hi=256,
                    n_seed=5, seed_base=5000, dt=0.005, qd=(0.1, 100.0),
                    noise=0.01, solves=10)


@dataclass
class LQ:
    """One LQ subproblem; arrays in the layouts given in the module docstring."""
    nx: int
    nu: int
    N: int
    A: np.ndarray
    B: np.ndarray
    Qd: np.ndarray
    Rd: np.ndarray
    q: np.ndarray
    r: np.ndarray
    c: np.ndarray
    # optional dense SPD cost blocks Q[N][nx][nx], R[N-1][nu][nu] (the
    # general Q_k, R_k of Sec. II-A); when present, Qd and Rd hold their
    # diagonals and the dense blocks define the problem
    Q: Optional[np.ndarray] = None
    R: Optional[np.ndarray] = None

    FIELDS = ("A", "B", "Qd", "Rd", "q", "r", "c")
    DENSE = ("Q", "R")

    @property
    def dtype(self):
        return self.A.dtype

    @property
    def dense(self) -> bool:
        return self.Q is not None

    def astype(self, dt) -> "LQ":
        kw = {f: np.ascontiguousarray(getattr(self, f), dtype=dt) for f in self.FIELDS}
        for f in self.DENSE:
            v = getattr(self, f)
            kw[f] = None if v is None else np.ascontiguousarray(v, dtype=dt)
        return LQ(self.nx, self.nu, self.N, **kw)

    def copy(self) -> "LQ":
        kw = {f: np.array(getattr(self, f), copy=True) for f in self.FIELDS}
        for f in self.DENSE:
            v = getattr(self, f)
            kw[f] = None if v is None else np.array(v, copy=True)
        return LQ(self.nx, self.nu, self.N, **kw)


def to_f32(lq: LQ) -> LQ:
    """Round every array to float32 (the precision the GPU path stores)."""
    return lq.astype(np.float32)


def kuka_lq(nx: int, nu: int, N: int, seed: int, dt: float = 0.01,
            qd=(1.0, 10.0), rd=(0.01, 0.1), dense: bool = False) -> LQ:
    """Draw one Kuka-shaped LQ subproblem (float64).  dense=True adds general
    SPD cost blocks Q_k = diag(Qd_k) + (0.5/nx) W W^T and R_k = diag(Rd_k) +
    (0.01/nu) V V^T with W, V ~ N(0, 1)."""
    if nx % 2 or not (1 <= nu <= nx // 2) or N < 1:
        raise ValueError("need even nx, 1 <= nu <= nx/2 and N >= 1")
    h = nx // 2
    K = max(N - 1, 0)
    rng = np.random.default_rng(seed)
    M = rng.normal(0.0, 0.5, size=(K, h, h))
    Dm = rng.normal(0.0, 0.5, size=(K, h, h))
    L = rng.normal(0.0, 1.0, size=(K, h, h))
    Qd = rng.uniform(qd[0], qd[1], size=(N, nx))
    Rd = rng.uniform(rd[0], rd[1], size=(K, nu))
    q = rng.normal(0.0, 1.0, size=(N, nx))
    r = rng.normal(0.0, 1.0, size=(K, nu))
    c = rng.normal(0.0, 1.0, size=(N, nx))
    eye = np.eye(h)
    A = np.zeros((K, nx, nx))
    A[:, :h, :h] = eye
    A[:, :h, h:] = dt * eye
    A[:, h:, :h] = dt * M
    A[:, h:, h:] = eye + dt * Dm
    Minv = np.einsum("kij,klj->kil", L, L) + 0.1 * eye
    B = np.zeros((K, nx, nu))
    B[:, h:, :] = dt * Minv[:, :, :nu]
    lq = LQ(nx, nu, N, A, B, Qd, Rd, q, r, c)
    if dense:
        # general SPD cost blocks: the drawn diagonals plus a random
        # positive semidefinite coupling (drawn after everything above, so
        # A, B, q, r, c match the diagonal instance of the same seed)
        Wq = rng.normal(0.0, 1.0, size=(N, nx, nx))
        Wr = rng.normal(0.0, 1.0, size=(K, nu, nu))
        Q = np.einsum("kij,klj->kil", Wq, Wq) * (0.5 / nx)
        R = np.einsum("kij,klj->kil", Wr, Wr) * (0.01 / nu)
        Q[:, np.arange(nx), np.arange(nx)] += Qd
        R[:, np.arange(nu), np.arange(nu)] += Rd
        lq.Q, lq.R = Q, R
        lq.Qd = np.ascontiguousarray(Q[:, np.arange(nx), np.arange(nx)])
        lq.Rd = np.ascontiguousarray(R[:, np.arange(nu), np.arange(nu)])
    return lq


@dataclass
class LQBatch:
    """Many independent LQ subproblems with ragged horizons, concatenated.

    knot_off[b] is the first knot of instance b in every per-knot array
    (Qd, q, c and the per-knot outputs); the per-control arrays (A, B, Rd, r
    and the off-diagonal outputs) of instance b start at knot_off[b] - b.
    """
    nx: int
    nu: int
    Ns: np.ndarray
    knot_off: np.ndarray
    lq: LQ                       # concatenated arrays; lq.N = total knots
    items: List[LQ] = field(default_factory=list)

    @property
    def B(self) -> int:
        return len(self.Ns)

    def ctrl_off(self) -> np.ndarray:
        return self.knot_off - np.arange(len(self.knot_off))

    def astype(self, dt) -> "LQBatch":
        return LQBatch(self.nx, self.nu, self.Ns.copy(), self.knot_off.copy(),
                       self.lq.astype(dt), [it.astype(dt) for it in self.items])


def concat_batch(items: Sequence[LQ]) -> LQBatch:
    nx, nu = items[0].nx, items[0].nu
    Ns = np.array([it.N for it in items], dtype=np.int64)
    knot_off = np.zeros(len(items) + 1, dtype=np.int64)
    knot_off[1:] = np.cumsum(Ns)
    cat = {f: np.ascontiguousarray(np.concatenate([getattr(it, f) for it in items], axis=0))
           for f in LQ.FIELDS}
    if all(it.dense for it in items):
        for f in LQ.DENSE:
            cat[f] = np.ascontiguousarray(np.concatenate([getattr(it, f) for it in items], axis=0))
    elif any(it.dense for it in items):
        raise ValueError("a batch mixes dense and diagonal cost blocks")
    lq = LQ(nx, nu, int(knot_off[-1]), **cat)
    return LQBatch(nx, nu, Ns, knot_off, lq, list(items))


def batch_horizons(B: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Ragged horizons N_i ~ U{lo..hi} (inclusive)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=B)


def kuka_batch(nx: int, nu: int, Ns: Sequence[int], seed_base: int, dt: float = 0.01,
               qd=(1.0, 10.0), dense: bool = False) -> LQBatch:
    items = [kuka_lq(nx, nu, int(n), seed_base + i, dt=dt, qd=qd, dense=dense)
             for i, n in enumerate(Ns)]
    return concat_batch(items)


def warm_noise(seed: int, rep: int, shape) -> np.ndarray:
    """Standard-normal draws for repetition `rep` of instance `seed`."""
    return np.random.default_rng([seed, rep]).normal(0.0, 1.0, size=shape)


def warm_start(lam_star: np.ndarray, seed: int, rep: int, rel: float = 0.01) -> np.ndarray:
    """Perturbed warm start lam0 = lam_star * (1 + rel * xi), xi ~ N(0, 1).

    Mimics the previous SQP iteration's multipliers (Sec. IV-B, last
    sentences): a nearby but not converged starting point.
    """
    xi = warm_noise(seed, rep, lam_star.shape)
    return (lam_star * (1.0 + rel * xi)).astype(lam_star.dtype)


def loss_weights(n_lam: int, seed: int) -> np.ndarray:
    """w ~ N(0, 1) for the scalar loss sum ||dz||^2 + w^T lambda."""
    return np.random.default_rng(seed).normal(0.0, 1.0, size=n_lam)


# ---------------------------------------------------------------------------
# Synthetic nonlinear model for the SQP outer loop and the parallel line
# search (Sec. II-A Step 3, Sec. IV-C).  The paper's experiments linearise
# the Kuka rigid-body dynamics; that model is not available, so a
# Kuka-shaped stand-in with the same state layout is used: h = nx/2 joints,
# x = (joint positions p, joint velocities v), nu actuated joints,
#     v+ = v + dt (P u - damp * v - stiff * sin(p)),   p+ = p + dt v+
# (semi-implicit Euler), and a tracking cost
#     l(x, u) = 1/2 sum wq (x - xref_k)^2 + 1/2 sum wr u^2,
#     l_f(x)  = 1/2 sum wf (x - xref_{N-1})^2.
# Only parameters and initial data are drawn here; the dynamics, their
# Jacobians and the merit function live in the oracle and in the kernels.
# ---------------------------------------------------------------------------
@dataclass
class Model:
    nx: int
    nu: int
    dt: float
    P: np.ndarray       # [h][nu] input matrix
    damp: np.ndarray    # [h]
    stiff: np.ndarray   # [h]
    wq: np.ndarray      # [nx] stage state weights
    wr: np.ndarray      # [nu] control weights
    wf: np.ndarray      # [nx] terminal state weights

    def astype(self, dt) -> "Model":
        f = lambda a: np.ascontiguousarray(a, dtype=dt)
        return Model(self.nx, self.nu, self.dt, f(self.P), f(self.damp), f(self.stiff),
                     f(self.wq), f(self.wr), f(self.wf))


@dataclass
class Tracking:
    """One tracking problem for the model: start state, reference, initial guess."""
    N: int
    xs: np.ndarray      # [nx]
    xref: np.ndarray    # [N][nx]
    X: np.ndarray       # [N][nx] initial state trajectory
    U: np.ndarray       # [N-1][nu] initial controls

    def astype(self, dt) -> "Tracking":
        f = lambda a: np.ascontiguousarray(a, dtype=dt)
        return Tracking(self.N, f(self.xs), f(self.xref), f(self.X), f(self.U))


CONFIG_NMPC = dict(name="nmpc", nx=14, nu=7, Ns=(128, 512), model_seed=6, seed_base=6000,
                   dt=0.01, n_alpha=9, sqp_iters=8)


def nmpc_model(nx: int, nu: int, seed: int, dt: float = 0.01) -> Model:
    if nx % 2 or not (1 <= nu <= nx // 2):
        raise ValueError("need even nx and 1 <= nu <= nx/2")
    h = nx // 2
    rng = np.random.default_rng(seed)
    L = rng.normal(0.0, 1.0, size=(h, h))
    P = (L @ L.T + 0.1 * np.eye(h))[:, :nu]
    damp = rng.uniform(0.1, 1.0, size=h)
    stiff = rng.uniform(1.0, 10.0, size=h)
    wq = rng.uniform(1.0, 10.0, size=nx)
    wr = rng.uniform(0.01, 0.1, size=nu)
    return Model(nx, nu, dt, P, damp, stiff, wq, wr, 10.0 * wq)


def nmpc_tracking(model: Model, N: int, seed: int) -> Tracking:
    """Start state ~ N(0, 0.5^2); joint-position targets a sin(w t + phi) with
    matching velocity targets; initial guess = straight line from the start
    to the final reference state, zero controls (not dynamically feasible)."""
    nx, nu, h = model.nx, model.nu, model.nx // 2
    rng = np.random.default_rng(seed)
    xs = rng.normal(0.0, 0.5, size=nx)
    amp = rng.uniform(0.2, 1.0, size=h)
    w = rng.uniform(0.5, 3.0, size=h)
    ph = rng.uniform(0.0, 2 * np.pi, size=h)
    t = np.arange(N)[:, None] * model.dt
    xref = np.concatenate([amp * np.sin(w * t + ph), amp * w * np.cos(w * t + ph)], axis=1)
    s = np.linspace(0.0, 1.0, N)[:, None]
    X = xs[None, :] + s * (xref[-1] - xs)[None, :]
    U = np.zeros((max(N - 1, 0), nu))
    return Tracking(N, xs, xref, X, U)
