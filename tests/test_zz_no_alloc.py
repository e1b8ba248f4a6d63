"""The backward entry point that allocates nothing (mpcg_backward_batched_noalloc).

It serves callers that cannot allocate device memory when they
differentiate (a controller with memory fixed at start-up, a host framework
that owns every allocation): its scratch is a fixed device array inside the
library instead of a caller workspace.  These tests call it through the C
ABI and compare it with mpcg_backward_batched, which takes a workspace, on
two calls in a row -- the second call must not see the first one's scratch.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32, solver
from workload import gen

pytestmark = pytest.mark.gpu

FIELDS = ("A", "B", "Qd", "Rd", "q", "r", "c")


def _noalloc_outputs(s, lt):
    import torch
    g = {f: torch.full_like(getattr(lt, f), float("nan")) for f in FIELDS}
    return g, s.alloc_stats(lt.nb)


def _noalloc_backward(s, lt, sch, lam, dx, du, lam_bar, dx_bar, du_bar, opts, outputs=None):
    import torch
    from paper_2309_08079_gb300 import _lib as L
    g, stats = outputs if outputs is not None else _noalloc_outputs(s, lt)
    gs = L.mpcg_grads(*(g[f].data_ptr() for f in FIELDS))
    ls, ss = lt.lq_struct(), sch.struct()
    ptr = lambda t: C.c_void_p(t.data_ptr())
    ko = None if lt.knot_off is None else ptr(lt.knot_off)
    rc = s.lib.mpcg_backward_batched_noalloc(
        s.h, lt.dims(), lt.nb, ko, C.byref(ls), C.byref(ss), ptr(lam), ptr(dx), ptr(du),
        ptr(lam_bar), ptr(dx_bar), ptr(du_bar), C.byref(gs), C.byref(opts), ptr(stats),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    L.check("mpcg_backward_batched_noalloc", rc)
    return g, stats


def test_noalloc_backward_matches_workspace_backward_on_two_calls():
    import torch
    from paper_2309_08079_gb300.solver import LQTensors, make_opts, read_stats
    s = solver()
    batch = gen.kuka_batch(14, 7, [16, 40, 9, 33], 4200).astype(np.float32)
    lt = LQTensors.from_batch(batch)
    opts = make_opts()
    lam, dx, du, st, sch = s.solve(lt, opts=opts, workspace=s.alloc_workspace(lt))
    K = lt.total
    seeds = [(gen.loss_weights(K * 14, 40), 2.0, 2.0), (-gen.loss_weights(K * 14, 41), 1.0, 3.0)]
    keep = []  # every call's tensors stay alive, so the allocator's count moves only by new allocations
    for call, (w, ax, au) in enumerate(seeds):
        lam_bar = torch.as_tensor(w.reshape(K, 14), dtype=torch.float32, device="cuda")
        dx_bar = (ax * dx).contiguous()
        du_bar = (au * du).contiguous()
        ref, st_ref = s.backward(lt, sch, lam, dx, du, lam_bar, dx_bar, du_bar, opts=opts)
        outs = _noalloc_outputs(s, lt)
        torch.cuda.synchronize()
        free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        new, st_new = _noalloc_backward(s, lt, sch, lam, dx, du, lam_bar, dx_bar, du_bar, opts, outs)
        torch.cuda.synchronize()
        if call == 1:
            # the second call allocates nothing: neither device memory at the
            # driver level nor through the caller's allocator
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == used0
        keep.append((lam_bar, dx_bar, du_bar, ref, st_ref, outs, new, st_new))
        assert np.all(read_stats(st_new)["status"] == 0), (call, read_stats(st_new))
        assert np.array_equal(read_stats(st_new)["iters"], read_stats(st_ref)["iters"])
        for f in FIELDS:
            a = new[f].double().cpu().numpy()
            b = ref[f].double().cpu().numpy()
            assert np.all(np.isfinite(a)), (call, f)
            assert oracle.relerr(a, b) <= TOL_F32, (call, f, oracle.relerr(a, b))


def test_noalloc_backward_refuses_problems_beyond_its_scratch():
    import torch
    from paper_2309_08079_gb300 import _lib as L
    from paper_2309_08079_gb300.solver import LQTensors, make_opts
    s = solver()
    lq = gen.kuka_lq(14, 7, 8, 4300).astype(np.float32)
    lt = LQTensors.from_numpy(lq)
    lam, dx, du, st, sch = s.solve(lt)
    # claim 1000 instances of 512 knots: far more scratch than the array holds
    lt_big = LQTensors(14, 7, 512, lt.A, lt.B, lt.Qd, lt.Rd, lt.q, lt.r, lt.c,
                       knot_off=torch.zeros(1001, dtype=torch.int32, device="cuda"), nb=1000,
                       total=lt.total)
    assert s.lib.mpcg_workspace_bytes(lt_big.dims(), 1000) > 8 << 20
    with pytest.raises(L.MPCGError) as ei:
        _noalloc_backward(s, lt_big, sch, lam, dx, du, lam, dx, du, make_opts())
    assert ei.value.code == L.MPCG_ETOOLARGE
    # nothing was launched and the next call works
    g, st2 = _noalloc_backward(s, lt, sch, lam, dx, du, lam, dx, du, make_opts())
    torch.cuda.synchronize()
    assert all(np.all(np.isfinite(g[f].cpu().numpy())) for f in FIELDS)
