"""Packed diagonal blocks in the tiled CTA kernel (mode 3, nx = 36).

The tiled kernel streams only the upper triangle of each symmetric diagonal
block of S+ and Phi^-1 (symmetric by Eq. 5 and Sec. IV-A), stored column by
column, and reads it in place, when the smaller slots fit more knot streams.
Checks: the packed layout formation writes; when the launch takes the packed
blocks; the packed solve meets the oracle; the cluster and L2 kernels ignore
the packed copies.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, TOL_KNOT_F32, assert_knots, solver
from workload import gen

pytestmark = pytest.mark.gpu


def _setup(Ns, seed, large=False):
    import torch
    from paper_2309_08079_gb300.solver import LQTensors
    c = gen.CONFIG_LARGE
    kw = dict(dt=c["dt"], qd=c["qd"]) if large else {}
    batch = gen.kuka_batch(36, 12, Ns, seed, **kw).astype(np.float32)
    return batch, solver(), LQTensors.from_batch(batch, dtype=torch.float32)


def _pcg(s, lt, sch, mode=3, max_iter=0):
    import torch
    from paper_2309_08079_gb300.solver import make_opts, read_stats
    lam = torch.zeros(lt.total, lt.nx, dtype=torch.float32, device="cuda")
    stats = s.alloc_stats(lt.nb)
    o = make_opts(mode=mode, max_iter=max_iter, tol=1e-6 if max_iter == 0 else 1e-30)
    s.pcg_solve(lt, sch, lam, opts=o, stats=stats)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), read_stats(stats)


def test_packed_layout():
    import torch
    from paper_2309_08079_gb300.solver import packed_len
    batch, s, lt = _setup([3, 1, 17], 4136)
    sch = s.alloc_schur(lt, packed=True)
    s.form(lt, sch)
    torch.cuda.synchronize()
    nx = 36
    rows, cols = [], []
    for j in range(nx):          # column by column, rows 0..j
        for i in range(j + 1):
            rows.append(i)
            cols.append(j)
    n = len(rows)
    for full, pk in ((sch.Sd, sch.Sdp), (sch.Pd, sch.Pdp)):
        F = full.cpu().numpy()
        Pk = pk.cpu().numpy()
        assert Pk.shape == (lt.total, packed_len(nx))
        np.testing.assert_array_equal(Pk[:, :n], F[:, rows, cols])
        np.testing.assert_array_equal(Pk[:, n:], 0.0)


def test_packed_blocks_taken_when_they_fit_more_streams():
    """The launch streams the packed blocks only when their smaller slots fit
    more knot streams than full tiles (long horizons); otherwise the shape,
    and the kernel, are those of an unpacked allocation."""
    from paper_2309_08079_gb300.solver import make_opts
    batch, s, lt = _setup([256, 40], 4236)
    o = make_opts(mode=3)
    sp, sf = s.alloc_schur(lt, packed=True), s.alloc_schur(lt, packed=False)
    long_p, long_f = s.pcg_shape(lt, sp, o, N=256), s.pcg_shape(lt, sf, o, N=256)
    assert long_p["threads"] > long_f["threads"], (long_p, long_f)
    assert long_p["packed"] and not long_f["packed"]
    short_p, short_f = s.pcg_shape(lt, sp, o, N=16), s.pcg_shape(lt, sf, o, N=16)
    assert short_p == short_f and not short_p["packed"], (short_p, short_f)


def test_packed_solve_meets_oracle():
    """Large-state shape, ragged horizons 1 .. 256, one refinement step (the
    workload's setting): every instance against the oracle, per knot too."""
    import torch
    from paper_2309_08079_gb300.solver import make_opts
    batch, s, lt = _setup([256, 1, 77, 200, 2, 130], 4336, large=True)
    sch = s.alloc_schur(lt)  # packed by default for float32 nx = 36 batches
    assert sch.Sdp is not None
    o = make_opts(mode=3, refine_tol=1e-2)
    lam, dx, du, st, sch = s.solve(lt, opts=o, schur=sch, workspace=s.alloc_workspace(lt), refine=1)
    torch.cuda.synchronize()
    from paper_2309_08079_gb300.solver import read_stats
    st = read_stats(st)
    lam, dx, du = (t.cpu().double().numpy() for t in (lam, dx, du))
    ko, co = batch.knot_off, batch.ctrl_off()
    for b, it in enumerate(batch.items):
        lo, xo, uo = oracle.kkt_solve(it.astype(np.float64))
        assert st["status"][b] == 0, (b, st[b])
        assert oracle.relerr(lam[ko[b]:ko[b + 1]], lo) < TOL_F32, (b, it.N)
        assert_knots(lam[ko[b]:ko[b + 1]], dx[ko[b]:ko[b + 1]], du[co[b]:co[b + 1]], lo, xo, uo,
                     TOL_KNOT_F32, (b, it.N))


def test_packed_ignored_by_other_kernels():
    """The cluster and L2 CTA kernels read the full blocks: a packed
    allocation changes nothing there."""
    batch, s, lt = _setup([40, 7, 129], 4436)
    sp = s.alloc_schur(lt, packed=True)
    s.form(lt, sp)
    sf = s.alloc_schur(lt, packed=False)
    s.form(lt, sf)
    for mode in (1, 2):
        lp, _ = _pcg(s, lt, sp, mode)
        lf, _ = _pcg(s, lt, sf, mode)
        np.testing.assert_array_equal(lp, lf)


def test_packed_blocks_with_the_comparison_preconditioners():
    """The packed path under opts.precon 1 (block Jacobi: Pd alone in the
    Phi^-1 passes) and 2 (the non-symmetric stair: Pd alone at even knots):
    after a fixed number of iterations lambda equals the oracle's Algorithm 1
    iterate with the same preconditioner, instance by instance, on a batch
    long enough that the launch takes the packed blocks."""
    import torch
    from paper_2309_08079_gb300.solver import make_opts, read_stats
    m = 10
    batch, s, lt = _setup([256, 33, 190], 4536)
    sch = s.alloc_schur(lt)
    s.form(lt, sch)
    ko = batch.knot_off
    for precon in (1, 2):
        o = make_opts(mode=3, precon=precon, tol=1e-30, max_iter=m)
        assert s.pcg_shape(lt, sch, o)["packed"]
        lam = torch.zeros(lt.total, 36, device="cuda")
        st = s.alloc_stats(lt.nb)
        s.pcg_solve(lt, sch, lam, o, st)
        torch.cuda.synchronize()
        st = read_stats(st)
        lam = lam.cpu().double().numpy()
        for b, it in enumerate(batch.items):
            Sd, So, g = oracle.schur_blocks(it.astype(np.float64))
            S = oracle.block_tridiag_sparse(Sd, So)
            if precon == 1:
                Pd, _ = oracle.precon_blocks(Sd, So)
                Pm = oracle.block_tridiag_sparse(Pd, np.zeros_like(So))
            else:
                Pm = oracle.stair_inverse(Sd, So)
            lo, its, _ = oracle.pcg_op(S, Pm, -g, tol=1e-30, max_iter=m)
            assert its == m and st["status"][b] == 1 and st["iters"][b] == m, (precon, b, st[b])
            e = oracle.relerr(lam[ko[b]:ko[b + 1]], lo.reshape(-1, 36))
            assert e < 1e-3, (precon, b, e)
