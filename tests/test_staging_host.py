"""Host-side layout of staging.HostStaging (no GPU): one buffer per solve,
inputs and lambda0 a contiguous prefix, results a contiguous suffix."""
import numpy as np
import pytest

from paper_2309_08079_gb300 import staging


@pytest.mark.parametrize("nx,nu,N,esz", [(14, 7, 512, 4), (14, 7, 1, 4), (36, 12, 77, 8), (2, 1, 3, 4)])
def test_layout_prefix_suffix_and_alignment(nx, nu, N, esz):
    shapes, off, total, in_end, out_begin, out_end = staging.layout(nx, nu, N, esz)
    order = staging._ORDER
    ends = {k: off[k] + int(np.prod(shapes[k])) for k in order}
    for a, b in zip(order, order[1:]):
        assert ends[a] <= off[b]                      # no overlap, in order
    for k in order:
        assert (off[k] * esz) % 256 == 0              # 256-byte aligned
    assert in_end == ends["lam"] and out_begin == off["lam"] and out_end == ends["stats"]
    assert out_end <= total
    # the prefix holds every input and lambda0, the suffix every result
    assert all(ends[k] <= in_end for k in ("A", "B", "Qd", "Rd", "q", "r", "c", "lam"))
    assert all(off[k] >= out_begin for k in ("lam", "dx", "du", "stats"))
    assert int(np.prod(shapes["stats"])) * esz == 24
    assert shapes["A"][0] == max(N - 1, 1) and shapes["lam"] == (N, nx)
