"""SQP outer loop on the device around the solve path (Sec. II-A Steps 1-3,
Sec. IV-C), on the library's synthetic model (mpcg_model in include/mpcg.h).

One SQP iteration is five stream-ordered library calls with no host
synchronisation: linearise at the current trajectory, form S+, gamma and the
stair preconditioner (one fused launch), PCG (warm-started from the previous iteration's
multipliers, as the paper does), recover the step, and the parallel line
search that evaluates every step size of a halving set and applies the one
with the smallest L1 merit.  `SQP.graph()` captures iterations in a CUDA
graph.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Union

import numpy as np
import torch

from . import _lib as L
from .solver import LQTensors, Solver, _ptr, _stream, make_opts

_DT = {torch.float32: 0, torch.float64: 1}


class ModelTensors:
    """The model's parameters on the device (layouts of mpcg_model)."""

    FIELDS = ("P", "damp", "stiff", "wq", "wr", "wf")

    def __init__(self, model, device="cuda", dtype=torch.float32):
        self.nx, self.nu, self.dt = model.nx, model.nu, float(model.dt)
        for f in self.FIELDS:
            setattr(self, f, torch.as_tensor(np.ascontiguousarray(getattr(model, f)), dtype=dtype,
                                             device=device))

    def struct(self) -> L.mpcg_model:
        return L.mpcg_model(self.nx, self.nu, self.dt, *(getattr(self, f).data_ptr() for f in self.FIELDS))


class SQP:
    """Device-resident SQP iterations for one tracking problem or a ragged
    batch of them (a list of `workload.gen.Tracking`)."""

    def __init__(self, solver: Solver, model, tracking: Union[object, Sequence[object]],
                 device="cuda", dtype=torch.float32, opts=None, n_alpha: int = 9, mu: float = 0.0):
        self.s = solver
        self.dev = torch.device(device)
        trks = list(tracking) if isinstance(tracking, (list, tuple)) else [tracking]
        self.batched = isinstance(tracking, (list, tuple))
        self.model = ModelTensors(model, self.dev, dtype)
        nx, nu = model.nx, model.nu
        Ns = np.array([t.N for t in trks], dtype=np.int64)
        ko = np.zeros(len(trks) + 1, dtype=np.int64)
        ko[1:] = np.cumsum(Ns)
        K, B = int(ko[-1]), len(trks)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=self.dev)
        cat = lambda f: np.concatenate([getattr(x, f) for x in trks], axis=0)
        self.X, self.U = t(cat("X")), t(cat("U")) if K - B > 0 else torch.zeros(1, nu, dtype=dtype, device=self.dev)
        self.xref = t(cat("xref"))
        self.xs = t(np.stack([x.xs for x in trks]))
        e = lambda *shape: torch.zeros(*shape, dtype=dtype, device=self.dev)
        Kc = max(K - B, 1)
        self.lq = LQTensors(nx, nu, int(Ns.max()), e(Kc, nx, nx), e(Kc, nx, nu), e(K, nx), e(Kc, nu),
                            e(K, nx), e(Kc, nu), e(K, nx),
                            knot_off=torch.as_tensor(ko.astype(np.int32), device=self.dev) if self.batched else None,
                            nb=B, total=K, Ns=Ns if self.batched else None)
        self.schur = solver.alloc_schur(self.lq)
        self.ws = solver.alloc_workspace(self.lq) if self.batched else None
        self.lam = e(K, nx)
        self.dx, self.du = e(K, nx), e(Kc, nu)
        self.stats = solver.alloc_stats(B, self.dev)
        self.merit = torch.zeros(B, n_alpha, dtype=torch.float64, device=self.dev)
        self.alpha_index = torch.zeros(B, dtype=torch.int32, device=self.dev)
        self.opts = opts if opts is not None else make_opts()
        self.n_alpha, self.mu = int(n_alpha), float(mu)
        self.B = B

    def _dims(self) -> L.mpcg_dims:
        return self.lq.dims()

    def linearize(self, stream=None):
        lq = self.lq
        out = L.mpcg_lq_out(*(getattr(lq, f).data_ptr() for f in LQTensors.FIELDS))
        m = self.model.struct()
        if self.batched:
            rc = self.s.lib.mpcg_linearize_batched(self.s.h, self._dims(), self.B, _ptr(lq.knot_off),
                                                   C.byref(m), _ptr(self.X), _ptr(self.U),
                                                   _ptr(self.xref), _ptr(self.xs), C.byref(out),
                                                   _stream(stream))
        else:
            rc = self.s.lib.mpcg_linearize(self.s.h, self._dims(), C.byref(m), _ptr(self.X),
                                           _ptr(self.U), _ptr(self.xref), _ptr(self.xs),
                                           C.byref(out), _stream(stream))
        L.check("mpcg_linearize", rc)

    def line_search(self, stream=None):
        m = self.model.struct()
        args = (C.byref(m), _ptr(self.X), _ptr(self.U), _ptr(self.dx), _ptr(self.du), _ptr(self.xref),
                _ptr(self.xs), _ptr(self.lam), C.c_double(self.mu), self.n_alpha, _ptr(self.merit),
                _ptr(self.alpha_index), _stream(stream))
        if self.batched:
            rc = self.s.lib.mpcg_line_search_batched(self.s.h, self._dims(), self.B,
                                                     _ptr(self.lq.knot_off), *args)
        else:
            rc = self.s.lib.mpcg_line_search(self.s.h, self._dims(), *args)
        L.check("mpcg_line_search", rc)

    def step(self, stream=None):
        """One SQP iteration (no host synchronisation)."""
        s, lq = self.s, self.lq
        self.linearize(stream)
        s.form(lq, self.schur, stream)
        s.pcg_solve(lq, self.schur, self.lam, self.opts, self.stats, self.ws, stream)
        s.recover_step(lq, self.lam, self.dx, self.du, stream)
        self.line_search(stream)

    def run(self, iters: int, stream=None):
        for _ in range(iters):
            self.step(stream)

    def graph(self, iters: int = 1) -> torch.cuda.CUDAGraph:
        """A CUDA graph of `iters` SQP iterations (run one eager iteration
        first so launch shapes are chosen outside the capture)."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self.run(iters)
        torch.cuda.current_stream(self.dev).wait_stream(side)
        return g
