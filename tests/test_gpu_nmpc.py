"""The outer loop on the device (linearisation, parallel line search, SQP
iterations) against the oracle's FP64 statement of the same steps."""
import numpy as np
import pytest

import oracle
from oracle import nmpc as onmpc
from gpu_util import solver
from workload import gen

pytestmark = pytest.mark.gpu


def _problem(N, seed=6100, dtype=np.float32):
    m = gen.nmpc_model(14, 7, 6)
    t = gen.nmpc_tracking(m, N, seed)
    return m.astype(dtype), t.astype(dtype)


def _sqp(m, t, dtype="float32", **kw):
    import torch
    from paper_2309_08079_gb300.nmpc import SQP
    from paper_2309_08079_gb300.solver import make_opts
    tdt = torch.float32 if dtype == "float32" else torch.float64
    opts = make_opts(tol=1e-6 if dtype == "float32" else 1e-13)
    return SQP(solver(), m, t, dtype=tdt, opts=opts, **kw)


@pytest.mark.parametrize("dtype,tol", [("float32", 2e-6), ("float64", 1e-13)])
def test_linearize_matches_oracle(dtype, tol):
    import torch
    npdt = np.float32 if dtype == "float32" else np.float64
    m, t = _problem(40, dtype=npdt)
    q = _sqp(m, t, dtype)
    q.linearize()
    torch.cuda.synchronize()
    ref = onmpc.linearize(m, t, t.X, t.U)
    for f in ("A", "B", "Qd", "Rd", "q", "r", "c"):
        got = getattr(q.lq, f).cpu().double().numpy()
        want = getattr(ref, f)
        assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max()), f


def test_line_search_matches_oracle_on_an_overlong_direction():
    """Direction from the oracle (8x its SQP step, so the search must back
    off); merits at the float32 candidates against the oracle's FP64 merits
    at the same candidates, the same choice, the same update."""
    import torch
    m, t = _problem(64)
    lq = onmpc.linearize(m, t, t.X, t.U)
    lam, dX, dU = oracle.kkt_solve(lq)
    dX32, dU32 = (8 * dX).astype(np.float32), (8 * dU).astype(np.float32)
    lam32 = lam.astype(np.float32)
    q = _sqp(m, t)
    q.dx.copy_(torch.as_tensor(dX32))
    q.du.copy_(torch.as_tensor(dU32))
    q.lam.copy_(torch.as_tensor(lam32))
    q.line_search()
    torch.cuda.synchronize()
    mu = onmpc.penalty(lam32.astype(np.float64))
    X2, U2, i, mer = onmpc.line_search(m, t, t.X, t.U, dX32, dU32, mu)
    got = q.merit.cpu().numpy()[0]
    assert np.abs(got - mer).max() <= 1e-10 * np.abs(mer).max(), (got, mer)
    assert int(q.alpha_index.cpu()[0]) == i and i >= 2
    np.testing.assert_array_equal(q.X.cpu().numpy(), X2)
    np.testing.assert_array_equal(q.U.cpu().numpy(), U2)


def test_sqp_iterations_track_the_oracle():
    import torch
    m, t = _problem(128)
    q = _sqp(m, t)
    hist = onmpc.sqp(m, t, 6)
    idx, mer = [], []
    for it in range(6):
        q.step()
        idx.append(int(q.alpha_index.cpu()[0]))
        mer.append(q.merit.cpu().numpy()[0].copy())
    torch.cuda.synchronize()
    X, U = q.X.cpu().double().numpy(), q.U.cpu().double().numpy()
    # the first steps are clear-cut full steps on both sides; later, near the
    # solution, the merits of several step sizes differ by less than the
    # float32 solve's noise, so only the consistency of the choice is checked
    assert idx[:2] == [h["idx"] for h in hist[:2]] == [0, 0]
    for i, m_ in zip(idx, mer):
        assert m_[i] <= m_.min() * (1 + 1e-11) and np.all(m_[:i] > m_.min() * (1 + 1e-11))
    # the float32 solves (<= 1e-4 normwise each) leave the float32 outer loop
    # within about 1e-3 of the FP64 iterates
    assert oracle.relerr(X, hist[-1]["X"]) < 1e-3 and oracle.relerr(U, hist[-1]["U"]) < 1e-3
    d = onmpc.defects(m, t, X, U)
    assert np.abs(d).max() < 1e-4 * max(1.0, np.abs(X).max())


def test_sqp_float64_tracks_the_oracle_closely():
    import torch
    """Both sides converged (8 iterations): the same first-order point."""
    m, t = _problem(48, dtype=np.float64)
    q = _sqp(m, t, "float64")
    q.run(8)
    torch.cuda.synchronize()
    hist = onmpc.sqp(m, t, 8)
    assert oracle.relerr(q.X.cpu().numpy(), hist[-1]["X"]) < 1e-10
    assert oracle.relerr(q.U.cpu().numpy(), hist[-1]["U"]) < 1e-9


def test_sqp_in_a_cuda_graph_equals_eager():
    import torch
    m, t = _problem(64)
    a = _sqp(m, t)
    a.run(3)
    b = _sqp(m, t)
    b.step()  # choose launch shapes outside the capture
    b2 = _sqp(m, t)
    g = b2.graph(3)
    b2.X.copy_(torch.as_tensor(t.X))
    b2.U.copy_(torch.as_tensor(t.U))
    b2.lam.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.X.cpu().numpy(), b2.X.cpu().numpy())
    np.testing.assert_array_equal(a.U.cpu().numpy(), b2.U.cpu().numpy())


def test_batched_sqp_matches_the_oracle_per_instance():
    import torch
    m = gen.nmpc_model(14, 7, 6).astype(np.float32)
    trks = [gen.nmpc_tracking(m, N, 6200 + i).astype(np.float32) for i, N in enumerate([40, 17, 96])]
    q = _sqp(m, trks)
    q.run(5)
    torch.cuda.synchronize()
    X, U = q.X.cpu().double().numpy(), q.U.cpu().double().numpy()
    ko = np.concatenate([[0], np.cumsum([t.N for t in trks])])
    for b, t in enumerate(trks):
        h = onmpc.sqp(m, t, 5)[-1]
        assert oracle.relerr(X[ko[b]:ko[b + 1]], h["X"]) < 1e-4
        assert oracle.relerr(U[ko[b] - b:ko[b + 1] - b - 1], h["U"]) < 1e-3
