"""Host-driven solves with one copy each way (plumbing, no arithmetic).

A controller that owns its LQ data on the host pays a fixed latency per
cudaMemcpyAsync, so a step built from one copy per array (A, B, Qd, Rd, q, r,
c, lambda0 in; lambda, dx, du, stats out) spends more time in copy overheads
than in the transfers themselves.  `HostStaging` lays every array of one
solve out in one device buffer, in that order, with the matching pinned host
buffer: the inputs and lambda0 form one contiguous prefix (one H2D copy), and
lambda, dx, du and the stats records one contiguous suffix (one D2H copy).
lambda sits where both meet: it is the warm start on the way in and the
result on the way out, since pcg_solve overwrites it in place.  Each array
starts on a 256-byte boundary.
"""
from __future__ import annotations

from typing import Dict

import numpy as np
import torch

from . import _lib as L
from .solver import STATS_DTYPE, LQTensors, SchurTensors, Solver

_ALIGN = 256
_ORDER = ("A", "B", "Qd", "Rd", "q", "r", "c", "lam", "dx", "du", "stats")


def layout(nx: int, nu: int, N: int, esz: int):
    """Element offsets of one solve's arrays in the shared buffer.

    Returns (shapes, offsets, total, in_end, out_begin, out_end): shapes and
    offsets by name (order A, B, Qd, Rd, q, r, c, lam, dx, du, stats; each
    offset a multiple of 256 bytes), the buffer length, the end of the input
    prefix [0, in_end) and the output suffix [out_begin, out_end)."""
    Kc = max(N - 1, 1)
    shapes = {"A": (Kc, nx, nx), "B": (Kc, nx, nu), "Qd": (N, nx), "Rd": (Kc, nu),
              "q": (N, nx), "r": (Kc, nu), "c": (N, nx), "lam": (N, nx), "dx": (N, nx),
              "du": (Kc, nu), "stats": (L.STATS_BYTES // esz,)}
    step = _ALIGN // esz
    off, o = {}, 0
    for name in _ORDER:
        off[name] = o
        o += -(-int(np.prod(shapes[name])) // step) * step
    return (shapes, off, o, off["lam"] + N * nx, off["lam"],
            off["stats"] + L.STATS_BYTES // esz)


class HostStaging:
    """Pinned host and device buffers for one solve of a fixed shape.

    Write the inputs through `host[name]` (numpy views; names A, B, Qd, Rd,
    q, r, c, lam), then `step()` copies them in, runs the solve path
    (fused formation, PCG, recovery) on the stream and copies the results
    back into `host["lam"]`, `host["dx"]`, `host["du"]`, `host["stats"]`
    (complete once the stream has reached that point).  Single instances
    only (knot_off None)."""

    def __init__(self, solver: Solver, nx: int, nu: int, N: int, dtype=torch.float32,
                 device="cuda"):
        self.s = solver
        esz = torch.empty((), dtype=dtype).element_size()
        shapes, off, o, self.in_end, self.out_begin, self.out_end = layout(nx, nu, N, esz)
        self.numel = o
        self.dev = torch.zeros(o, dtype=dtype, device=device)
        self.host_t = torch.zeros(o, dtype=dtype).pin_memory()
        d: Dict[str, torch.Tensor] = {}
        self.host: Dict[str, np.ndarray] = {}
        hnp = self.host_t.numpy()
        for name in _ORDER:
            shp = shapes[name]
            n = int(np.prod(shp))
            d[name] = self.dev[off[name]:off[name] + n].view(*shp)
            self.host[name] = hnp[off[name]:off[name] + n].reshape(shp)
        self.lq = LQTensors(nx, nu, N, *(d[f] for f in LQTensors.FIELDS), knot_off=None, nb=1,
                            total=N)
        self.lam, self.dx, self.du = d["lam"], d["dx"], d["du"]
        self.stats = d["stats"].view(torch.uint8)
        self.schur: SchurTensors = solver.alloc_schur(self.lq)

    @property
    def h2d_bytes(self) -> int:
        return self.in_end * self.dev.element_size()

    @property
    def d2h_bytes(self) -> int:
        return (self.out_end - self.out_begin) * self.dev.element_size()

    def load(self, lq) -> None:
        """Copy a host LQ problem (numpy fields, see workload) into the pinned
        input views (host memory only)."""
        for f in LQTensors.FIELDS:
            src = np.asarray(getattr(lq, f))
            self.host[f][:src.shape[0]] = src

    def step(self, opts=None, stream=None) -> None:
        """One host-driven solve: 1 H2D copy, 3 kernel launches, 1 D2H copy,
        all stream-ordered (no synchronisation)."""
        st = stream if stream is not None else torch.cuda.current_stream(self.dev.device)
        with torch.cuda.stream(st):
            self.dev[:self.in_end].copy_(self.host_t[:self.in_end], non_blocking=True)
            self.s.form(self.lq, self.schur, st)
            self.s.pcg_solve(self.lq, self.schur, self.lam, opts, self.stats, None, st)
            self.s.recover_step(self.lq, self.lam, self.dx, self.du, st)
            self.host_t[self.out_begin:self.out_end].copy_(self.dev[self.out_begin:self.out_end],
                                                          non_blocking=True)

    def read_stats(self) -> np.ndarray:
        """The stats records of the last completed step (host copy)."""
        return self.host["stats"].view(np.uint8).view(STATS_DTYPE)
