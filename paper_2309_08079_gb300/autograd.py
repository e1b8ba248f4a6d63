"""torch.autograd.Function around the solve path (no counterpart in the paper).

Forward runs the fused form_schur + form_precon, pcg_solve and recover_step; it saves
only S+, Phi^-1 (Sd, So, Pd, Po) and the solution (lambda, dx, du) besides
the inputs.  Backward runs the library's adjoint: a second PCG solve on the
same S+ with the same preconditioner, then per-knot outer products (see
mpcg_backward in include/mpcg.h).  cfg["refine"] refinement steps follow
the forward solve and, through opts.refine, the adjoint solve.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .solver import LQTensors, SchurTensors, make_opts


class MPCGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, Qd, Rd, q, r, c, lam0, cfg):
        """cfg: dict(solver, nx, nu, N, knot_off, nb, total, opts, workspace,
        refine, refine_tol) -- refine = steps of iterative refinement after the
        forward and after the adjoint PCG solve; refine_tol = exit tolerance of
        their correction solves (default: the solve's own)."""
        s = cfg["solver"]
        lq = LQTensors(cfg["nx"], cfg["nu"], cfg["N"], A.contiguous(), B.contiguous(),
                       Qd.contiguous(), Rd.contiguous(), q.contiguous(), r.contiguous(),
                       c.contiguous(), knot_off=cfg.get("knot_off"), nb=cfg.get("nb", 1),
                       total=cfg.get("total", cfg["N"]))
        opts = cfg.get("opts") or make_opts()
        if cfg.get("refine_tol"):
            opts = L.mpcg_opts.from_buffer_copy(opts)
            opts.refine_tol = float(cfg["refine_tol"])
        lam = lam0.detach().clone() if lam0 is not None else torch.zeros(
            lq.total, lq.nx, dtype=lq.dtype, device=lq.device)
        lam, dx, du, stats, schur = s.solve(lq, lam, opts=opts, workspace=cfg.get("workspace"),
                                            refine=int(cfg.get("refine", 0)))
        ctx.lq_meta = (lq.nx, lq.nu, lq.N, lq.knot_off, lq.nb, lq.total)
        ctx.solver = s
        bopts = L.mpcg_opts.from_buffer_copy(opts)
        bopts.refine = int(cfg.get("refine", 0))
        ctx.opts = bopts
        ctx.workspace = cfg.get("workspace")
        ctx.save_for_backward(lq.A, lq.B, lq.Qd, lq.Rd, lq.q, lq.r, lq.c, schur.Sd, schur.So,
                              schur.Pd, schur.Po, schur.gamma, schur.info, lam, dx, du, schur.Sdp,
                              schur.Pdp)
        ctx.fwd_stats = stats
        ctx.mark_non_differentiable(stats)
        return lam, dx, du, stats

    @staticmethod
    def backward(ctx, g_lam, g_dx, g_du, _g_stats):
        (A, B, Qd, Rd, q, r, c, Sd, So, Pd, Po, gamma, info, lam, dx, du, Sdp, Pdp) = ctx.saved_tensors
        nx, nu, N, knot_off, nb, total = ctx.lq_meta
        lq = LQTensors(nx, nu, N, A, B, Qd, Rd, q, r, c, knot_off=knot_off, nb=nb, total=total)
        schur = SchurTensors(Sd, So, Pd, Po, gamma, info, Sdp, Pdp)
        z = lambda t, like: (t.contiguous() if t is not None else torch.zeros_like(like))
        g, stats = ctx.solver.backward(lq, schur, lam, dx, du, z(g_lam, lam), z(g_dx, dx),
                                       z(g_du, du), opts=ctx.opts, workspace=ctx.workspace)
        ctx.bwd_stats = stats
        return g["A"], g["B"], g["Qd"], g["Rd"], g["q"], g["r"], g["c"], None, None
