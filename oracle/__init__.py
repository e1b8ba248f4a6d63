"""ORACLE -- test infrastructure, not part of the product.

A plain, slow, obviously correct FP64 CPU statement of what the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it.  It shares no code with the CUDA path; both
take their inputs from ``workload``.
"""
from .oracle import (  # noqa: F401
    build, kkt_solve, kkt_solve_rhs, kkt_dim, schur_blocks, precon_blocks, jacobi_blocks,
    dense_S, dense_Phi_inv, block_tridiag_sparse, stair_matrix, stair_inverse, pcg, pcg_op,
    recover, grad, loss,
    solve_batch, natural_z, split_z, relerr,
)
from . import nmpc  # noqa: F401
