"""Pins of the oracle's outer loop (Sec. II-A Steps 1 and 3, Sec. IV-C) on
the synthetic model: Jacobians against finite differences, the QP special
case, the line search's choice, SQP convergence."""
import numpy as np
import pytest

import oracle
from oracle import nmpc
from workload import gen


@pytest.fixture(scope="module")
def prob():
    m = gen.nmpc_model(14, 7, 6)
    return m, gen.nmpc_tracking(m, 48, 6001)


def test_jacobians_match_central_differences(prob):
    m, t = prob
    rng = np.random.default_rng(0)
    x, u = rng.normal(size=14) * 2, rng.normal(size=7)
    A, B = nmpc.jacobians(m, x, u)
    h = 1e-6
    Af = np.stack([(nmpc.dynamics(m, x + h * e, u) - nmpc.dynamics(m, x - h * e, u)) / (2 * h)
                   for e in np.eye(14)], axis=1)
    Bf = np.stack([(nmpc.dynamics(m, x, u + h * e) - nmpc.dynamics(m, x, u - h * e)) / (2 * h)
                   for e in np.eye(7)], axis=1)
    assert np.abs(A - Af).max() < 1e-8 and np.abs(B - Bf).max() < 1e-8


def test_linearization_fields(prob):
    m, t = prob
    lq = nmpc.linearize(m, t, t.X, t.U)
    assert np.allclose(lq.c[0], t.X[0] - t.xs)
    assert np.allclose(lq.c[5], t.X[5] - nmpc.dynamics(m, t.X[4], t.U[4]))
    assert np.allclose(lq.q[3], m.wq * (t.X[3] - t.xref[3]))
    assert np.allclose(lq.Qd[-1], m.wf) and np.allclose(lq.Rd[0], m.wr)
    # the merit at the current point is J + mu ||c||_1 by its pieces
    mu = 7.0
    assert np.isclose(nmpc.merit(m, t, t.X, t.U, mu),
                      nmpc.cost(m, t, t.X, t.U) + mu * np.abs(lq.c).sum())


def test_linear_model_converges_in_one_full_step(prob):
    """With stiff = 0 the dynamics are linear and the problem is the QP
    itself: one full SQP step lands on its optimum (next step ~ 0, no
    defects)."""
    m, t = prob
    lin = gen.Model(m.nx, m.nu, m.dt, m.P, m.damp, np.zeros_like(m.stiff), m.wq, m.wr, m.wf)
    hist = nmpc.sqp(lin, t, 2)
    assert hist[0]["idx"] == 0
    lam, dX, dU = oracle.kkt_solve(nmpc.linearize(lin, t, hist[0]["X"], hist[0]["U"]))
    assert np.abs(dX).max() < 1e-9 * max(1.0, np.abs(hist[0]["X"]).max())
    assert np.abs(nmpc.defects(lin, t, hist[0]["X"], hist[0]["U"])).max() < 1e-12


def test_line_search_picks_the_smallest_merit(prob):
    """An overlong direction (8x the SQP step): the search must back off, and
    its choice is the argmin of merits computed by definition."""
    m, t = prob
    lq = nmpc.linearize(m, t, t.X, t.U)
    lam, dX, dU = oracle.kkt_solve(lq)
    mu = nmpc.penalty(lam)
    X2, U2, i, mer = nmpc.line_search(m, t, t.X, t.U, 8 * dX, 8 * dU, mu)
    ref = [nmpc.merit(m, t, t.X + a * 8 * dX, t.U + a * 8 * dU, mu) for a in 0.5 ** np.arange(9)]
    assert np.allclose(mer, ref, rtol=1e-15) and i == int(np.argmin(ref)) and i >= 2
    # near-equal merits (within 1e-11 relative) resolve to the longest step
    Xt, Ut, it, _ = nmpc.line_search(m, t, t.X, t.U, 0 * dX, 0 * dU, mu)
    assert it == 0
    assert np.allclose(X2, t.X + 0.5 ** i * 8 * dX)


def test_sqp_converges_to_a_first_order_point(prob):
    m, t = prob
    hist = nmpc.sqp(m, t, 8)
    assert all(h["idx"] == 0 for h in hist[:3])
    merits = [h["merits"][h["idx"]] for h in hist]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(merits, merits[1:]))
    X, U = hist[-1]["X"], hist[-1]["U"]
    lam, dX, dU = oracle.kkt_solve(nmpc.linearize(m, t, X, U))
    assert np.abs(nmpc.defects(m, t, X, U)).max() < 1e-10
    assert np.abs(dX).max() < 1e-8 * max(1.0, np.abs(X).max())
    assert np.abs(dU).max() < 1e-8 * max(1.0, np.abs(U).max())
