"""PyTorch-facing binding of libmpcg.so.

PyTorch supplies device memory and the current stream; every step of the
solve path runs in the library's CUDA kernels.  Functions keep the C names
of the entry points they call (form_schur, form_precon, pcg_solve,
recover_step, backward) and only marshal tensor pointers.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib as L

_DT = {torch.float32: 0, torch.float64: 1}
STATS_DTYPE = np.dtype([("iters", "<i4"), ("status", "<i4"), ("eta", "<f8"), ("relres", "<f8")])


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class LQTensors:
    """LQ data on the device (layouts of include/mpcg.h).

    For a ragged batch, knot_off is an int32 device tensor of B+1 offsets and
    N is the largest horizon; for a single instance knot_off is None.
    """
    nx: int
    nu: int
    N: int
    A: torch.Tensor
    B: torch.Tensor
    Qd: torch.Tensor
    Rd: torch.Tensor
    q: torch.Tensor
    r: torch.Tensor
    c: torch.Tensor
    knot_off: Optional[torch.Tensor] = None
    nb: int = 1            # number of instances
    total: int = 0         # total knots
    Ns: Optional[np.ndarray] = None  # host copy of the horizons (batched)
    Q: Optional[torch.Tensor] = None  # dense SPD cost blocks [N][nx][nx] (None: diagonal Qd)
    R: Optional[torch.Tensor] = None  # dense SPD cost blocks [N-1][nu][nu]

    FIELDS = ("A", "B", "Qd", "Rd", "q", "r", "c")

    @property
    def dtype(self):
        return self.A.dtype

    @property
    def device(self):
        return self.A.device

    @property
    def batched(self) -> bool:
        return self.knot_off is not None

    def dims(self) -> L.mpcg_dims:
        return L.mpcg_dims(self.nx, self.nu, self.N, _DT[self.dtype])

    def lq_struct(self) -> L.mpcg_lq:
        dense = [None if t is None else t.data_ptr() for t in (self.Q, self.R)]
        return L.mpcg_lq(*(t.data_ptr() for t in (self.A, self.B, self.Qd, self.Rd, self.q,
                                                   self.r, self.c)), *dense)

    @staticmethod
    def _dense(src, device, dtype):
        if getattr(src, "Q", None) is None:
            return {}
        return {f: torch.as_tensor(np.ascontiguousarray(getattr(src, f)), dtype=dtype, device=device)
                for f in ("Q", "R")}

    @staticmethod
    def from_numpy(lq, device="cuda", dtype=torch.float32) -> "LQTensors":
        t = {f: torch.as_tensor(np.ascontiguousarray(getattr(lq, f)), dtype=dtype, device=device)
             for f in LQTensors.FIELDS}
        return LQTensors(lq.nx, lq.nu, lq.N, **t, knot_off=None, nb=1, total=lq.N,
                         **LQTensors._dense(lq, device, dtype))

    @staticmethod
    def from_batch(batch, device="cuda", dtype=torch.float32) -> "LQTensors":
        t = {f: torch.as_tensor(np.ascontiguousarray(getattr(batch.lq, f)), dtype=dtype,
                                device=device) for f in LQTensors.FIELDS}
        ko = torch.as_tensor(batch.knot_off.astype(np.int32), device=device)
        return LQTensors(batch.nx, batch.nu, int(batch.Ns.max()), **t, knot_off=ko,
                         nb=batch.B, total=int(batch.knot_off[-1]),
                         Ns=np.asarray(batch.Ns, dtype=np.int64).copy(),
                         **LQTensors._dense(batch.lq, device, dtype))


def packed_len(nx: int) -> int:
    """Entries per packed diagonal block: nx(nx+1)/2 rounded up to 4."""
    return (nx * (nx + 1) // 2 + 3) // 4 * 4


@dataclass
class SchurTensors:
    Sd: torch.Tensor
    So: torch.Tensor
    Pd: torch.Tensor
    Po: torch.Tensor
    gamma: torch.Tensor
    info: torch.Tensor
    Sdp: Optional[torch.Tensor] = None  # packed upper triangles of Sd, Pd ([K][packed_len(nx)])
    Pdp: Optional[torch.Tensor] = None

    def struct(self) -> L.mpcg_schur:
        pk = [None if t is None else t.data_ptr() for t in (self.Sdp, self.Pdp)]
        return L.mpcg_schur(*(t.data_ptr() for t in (self.Sd, self.So, self.Pd, self.Po,
                                                      self.gamma, self.info)), *pk)


def make_opts(tol=1e-6, tol_mode=0, max_iter=0, cluster=0, mode=0, instances=None,
              precon=0, refine=0, dot=0, refine_tol=0.0) -> L.mpcg_opts:
    """mode: 0 automatic, 1 cluster per instance, 2 one CTA per instance
    reading blocks from L2, 3 one CTA per instance streaming TMA tiles (as 2
    when blocks are not 16-byte multiples), 4 cluster per instance with
    shared-memory operators and up to 64 knots per CTA (nx <= 16).  precon:
    0 symmetric stair
    (Sec. IV-A), 1 block Jacobi, 2 the non-symmetric stair preconditioner
    (comparison only: no convergence guarantee).  refine: refinement steps
    of the adjoint solve in the backward calls.  dot: float32 dot-product
    accumulation, 0 float pairs (default), 1 float64.  refine_tol: exit
    tolerance of refinement's correction solves (<= 0: tol)."""
    o = L.mpcg_opts(float(tol), int(tol_mode), int(max_iter), int(cluster), int(mode), None, 0,
                    int(precon), int(refine), int(dot), float(refine_tol))
    if instances is not None:  # a device int32 tensor of instance indices
        o.instances = instances.data_ptr()
        o.n_instances = int(instances.numel())
    return o


def read_stats(stats: torch.Tensor) -> np.ndarray:
    """Device stats buffer -> numpy structured array (iters, status, eta, relres)."""
    return stats.cpu().numpy().view(STATS_DTYPE)


class Solver:
    """Owns one library handle bound to a CUDA device."""

    def __init__(self, device=None):
        self.lib = L.load()
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            h = C.c_void_p()
            L.check("mpcg_create", self.lib.mpcg_create(C.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                self.lib.mpcg_destroy(self.h)
                self.h = C.c_void_p()
        except Exception:
            pass

    # ---------------------------------------------------------------- buffers
    def alloc_schur(self, lq: LQTensors, packed: Optional[bool] = None) -> SchurTensors:
        """S+, Phi^-1 and gamma buffers.  packed (default: float32 batches at
        nx = 36, where the tiled kernel is bound by HBM bandwidth) adds the
        packed diagonal blocks the tiled kernel streams instead of Sd, Pd."""
        nx, K, dt, dev = lq.nx, lq.total, lq.dtype, lq.device
        Kc = K - lq.nb
        e = lambda *s: torch.empty(*s, dtype=dt, device=dev)
        if packed is None:
            packed = lq.batched and dt == torch.float32 and nx == 36
        pk = (e(K, packed_len(nx)), e(K, packed_len(nx))) if packed else (None, None)
        return SchurTensors(e(K, nx, nx), e(max(Kc, 1), nx, nx), e(K, nx, nx),
                            e(max(Kc, 1), nx, nx), e(K, nx),
                            torch.zeros(lq.nb, dtype=torch.int32, device=dev), *pk)

    def alloc_stats(self, nb: int = 1, device=None) -> torch.Tensor:
        return torch.zeros(nb * L.STATS_BYTES, dtype=torch.uint8,
                           device=device if device is not None else self.device)

    def workspace_bytes(self, lq: LQTensors) -> int:
        return int(self.lib.mpcg_workspace_bytes(lq.dims(), lq.nb))

    def alloc_workspace(self, lq: LQTensors) -> torch.Tensor:
        return torch.zeros(self.workspace_bytes(lq), dtype=torch.uint8, device=lq.device)

    # ---------------------------------------------------------------- introspection
    def pcg_shape(self, lq: LQTensors, schur: SchurTensors, opts=None, N: Optional[int] = None) -> dict:
        """The launch shape pcg_solve uses for these arguments (nothing is
        launched): kernel form, CTAs per cluster, clusters in the grid,
        threads per CTA."""
        ss = schur.struct()
        o = opts if opts is not None else make_opts()
        dims = lq.dims()
        if N is not None:
            dims.N = int(N)
        shape = (C.c_int * 6)()
        L.check("mpcg_pcg_shape", self.lib.mpcg_pcg_shape(self.h, dims, lq.nb, C.byref(ss), C.byref(o), shape))
        return {"form": ("cluster", "cta_l2", "cta_tma")[shape[0]], "C": shape[1], "clusters": shape[2],
                "threads": shape[3], "depth": shape[4], "packed": bool(shape[5])}

    def bench_exchange(self, C_: int, W: int, rounds: int = 2000, stream=None) -> dict:
        """Latency of one cluster reduction of the PCG kernels (both of
        Algorithm 1's per-iteration reductions take one) on a C_ x W launch
        shape, from mpcg_bench_exchange: cycles and nanoseconds per
        exchange."""
        out = torch.zeros(3, dtype=torch.int64, device=self.device)
        st = torch.full((C_,), -1, dtype=torch.int32, device=self.device)
        L.check("mpcg_bench_exchange", self.lib.mpcg_bench_exchange(self.h, int(C_), int(W), int(rounds),
                                                                  _ptr(out), _ptr(st), _stream(stream)))
        torch.cuda.synchronize(self.device)
        if not bool((st == 0).all()):
            raise RuntimeError(f"mpcg_bench_exchange: a wait gave up ({st.tolist()})")
        o = out.cpu().tolist()
        return {"cycles": o[0] / (2.0 * rounds), "ns": o[1] / (2.0 * rounds), "C": int(C_), "W": int(W),
                "rounds": int(rounds)}

    # ---------------------------------------------------------------- the path
    def form_schur(self, lq: LQTensors, schur: SchurTensors, stream=None) -> SchurTensors:
        ls, ss = lq.lq_struct(), schur.struct()
        if lq.batched:
            rc = self.lib.mpcg_form_schur_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off),
                                                  C.byref(ls), C.byref(ss), _stream(stream))
        else:
            rc = self.lib.mpcg_form_schur(self.h, lq.dims(), C.byref(ls), C.byref(ss),
                                          _stream(stream))
        L.check("mpcg_form_schur", rc)
        return schur

    def form_precon(self, lq: LQTensors, schur: SchurTensors, stream=None) -> SchurTensors:
        ss = schur.struct()
        if lq.batched:
            rc = self.lib.mpcg_form_precon_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off),
                                                   C.byref(ss), _stream(stream))
        else:
            rc = self.lib.mpcg_form_precon(self.h, lq.dims(), C.byref(ss), _stream(stream))
        L.check("mpcg_form_precon", rc)
        return schur

    def form(self, lq: LQTensors, schur: SchurTensors, stream=None) -> SchurTensors:
        """form_schur and form_precon in one launch (mpcg_form_schur_precon)."""
        ls, ss = lq.lq_struct(), schur.struct()
        if lq.batched:
            rc = self.lib.mpcg_form_schur_precon_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off),
                                                         C.byref(ls), C.byref(ss), _stream(stream))
        else:
            rc = self.lib.mpcg_form_schur_precon(self.h, lq.dims(), C.byref(ls), C.byref(ss),
                                                 _stream(stream))
        L.check("mpcg_form_schur_precon", rc)
        return schur

    def pcg_solve(self, lq: LQTensors, schur: SchurTensors, lam: torch.Tensor, opts=None,
                  stats: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                  stream=None, N: Optional[int] = None) -> torch.Tensor:
        """Solve S+ lam = -gamma in place (lam holds the warm start).

        N (batched calls with an instance list in opts) is the largest
        horizon among the listed instances; it sizes the launch.
        """
        ss = schur.struct()
        o = opts if opts is not None else make_opts()
        if stats is None:
            stats = self.alloc_stats(lq.nb, lq.device)
        if lq.batched:
            if workspace is None:
                workspace = self.alloc_workspace(lq)
            dims = lq.dims()
            if N is not None:
                dims.N = int(N)
            rc = self.lib.mpcg_pcg_solve_batched(self.h, dims, lq.nb, _ptr(lq.knot_off),
                                                 C.byref(ss), _ptr(lam), C.byref(o), _ptr(stats),
                                                 _ptr(workspace), _stream(stream))
        else:
            rc = self.lib.mpcg_pcg_solve(self.h, lq.dims(), C.byref(ss), _ptr(lam), C.byref(o),
                                         _ptr(stats), _stream(stream))
        L.check("mpcg_pcg_solve", rc)
        return stats

    def recover_step(self, lq: LQTensors, lam: torch.Tensor, dx=None, du=None, stream=None):
        if dx is None:
            dx = torch.empty(lq.total, lq.nx, dtype=lq.dtype, device=lq.device)
        if du is None:
            du = torch.empty(max(lq.total - lq.nb, 1), lq.nu, dtype=lq.dtype, device=lq.device)
        ls = lq.lq_struct()
        if lq.batched:
            rc = self.lib.mpcg_recover_step_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off),
                                                    C.byref(ls), _ptr(lam), _ptr(dx), _ptr(du),
                                                    _stream(stream))
        else:
            rc = self.lib.mpcg_recover_step(self.h, lq.dims(), C.byref(ls), _ptr(lam), _ptr(dx),
                                            _ptr(du), _stream(stream))
        L.check("mpcg_recover_step", rc)
        return dx, du

    def refine_step(self, lq: LQTensors, schur: SchurTensors, lam: torch.Tensor, opts=None,
                    stats: Optional[torch.Tensor] = None, workspace=None, stream=None):
        """One step of iterative refinement of lam (in place) with the exact residual."""
        ss, ls = schur.struct(), lq.lq_struct()
        o = opts if opts is not None else make_opts()
        if stats is None:
            stats = self.alloc_stats(lq.nb, lq.device)
        if workspace is None:
            workspace = self.alloc_workspace(lq)
        if lq.batched:
            rc = self.lib.mpcg_refine_step_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off),
                                                   C.byref(ls), C.byref(ss), _ptr(lam), C.byref(o),
                                                   _ptr(stats), _ptr(workspace), _stream(stream))
        else:
            rc = self.lib.mpcg_refine_step(self.h, lq.dims(), C.byref(ls), C.byref(ss), _ptr(lam),
                                           C.byref(o), _ptr(stats), _ptr(workspace), _stream(stream))
        L.check("mpcg_refine_step", rc)
        return stats

    def solve(self, lq: LQTensors, lam0: Optional[torch.Tensor] = None, opts=None,
              schur: Optional[SchurTensors] = None, stats=None, workspace=None, stream=None,
              refine: int = 0):
        """The whole path: form_schur and form_precon (one fused launch),
        pcg_solve, `refine` steps of iterative refinement, recover_step.

        Returns (lam, dx, du, stats, schur); lam0 (if given) is overwritten.
        stats are those of the first PCG solve.
        """
        if schur is None:
            schur = self.alloc_schur(lq)
        lam = lam0 if lam0 is not None else torch.zeros(lq.total, lq.nx, dtype=lq.dtype,
                                                        device=lq.device)
        self.form(lq, schur, stream)
        stats = self.pcg_solve(lq, schur, lam, opts, stats, workspace, stream)
        if refine > 0:
            if workspace is None:
                workspace = self.alloc_workspace(lq)
            rstats = self.alloc_stats(lq.nb, lq.device)
            for _ in range(refine):
                self.refine_step(lq, schur, lam, opts, rstats, workspace, stream)
        dx, du = self.recover_step(lq, lam, stream=stream)
        return lam, dx, du, stats, schur

    def backward(self, lq: LQTensors, schur: SchurTensors, lam, dx, du, lam_bar, dx_bar, du_bar,
                 opts=None, stats=None, workspace=None, stream=None):
        """Gradients of a loss of (lam, dx, du) w.r.t. (A, B, Qd, Rd, q, r, c)."""
        g = {f: torch.empty_like(getattr(lq, f)) for f in LQTensors.FIELDS}
        gs = L.mpcg_grads(*(g[f].data_ptr() for f in LQTensors.FIELDS))
        o = opts if opts is not None else make_opts()
        if stats is None:
            stats = self.alloc_stats(lq.nb, lq.device)
        if workspace is None:
            workspace = self.alloc_workspace(lq)
        ls, ss = lq.lq_struct(), schur.struct()
        args = (C.byref(ls), C.byref(ss), _ptr(lam), _ptr(dx), _ptr(du), _ptr(lam_bar),
                _ptr(dx_bar), _ptr(du_bar), C.byref(gs), C.byref(o), _ptr(stats),
                _ptr(workspace), _stream(stream))
        if lq.batched:
            rc = self.lib.mpcg_backward_batched(self.h, lq.dims(), lq.nb, _ptr(lq.knot_off), *args)
        else:
            rc = self.lib.mpcg_backward(self.h, lq.dims(), *args)
        L.check("mpcg_backward", rc)
        return g, stats
