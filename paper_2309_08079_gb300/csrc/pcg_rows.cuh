// Row products shared by the PCG kernels: one row of a block row of a
// symmetric block-tridiagonal matrix times the halo'd vector.
#pragma once

#include "launch.cuh"

namespace mpcg {

constexpr uint64_t WAIT_LIMIT_NS = 4000000000ull;  // 4 s: never reached in a healthy run
constexpr uint64_t DRAIN_LIMIT_NS = 100000000ull;  // 0.1 s for the peers to stop after a give-up
constexpr uint64_t DRAIN_GRACE_NS = 20000ull;      // pushes already in flight land within this

// Row i of one block row times the halo'd vector (PTR mode).  D: diagonal
// block (symmetric: column i == row i); L: block (k, k-1) read by rows;
// U: So-type block (k+1, k) read by columns (= row i of its transpose).
template <typename T>
__device__ __forceinline__ T rowdot_ptr(int nx, int i, const T *D, const T *L, const T *U,
                                        const T *vprev, const T *vself, const T *vnext) {
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int j = 0; j < nx; ++j) a0 = fma_rn(D[j * nx + i], vself[j], a0);
    if (L)
        for (int j = 0; j < nx; ++j) a1 = fma_rn(L[i * nx + j], vprev[j], a1);
    if (U)
        for (int j = 0; j < nx; ++j) a2 = fma_rn(U[j * nx + i], vnext[j], a2);
    return (a0 + a1) + a2;
}

// Row i of one block row times the halo'd vector, all loads issued before
// the arithmetic (nx <= NXM): keeps 3*NXM independent global loads in flight
// per thread when the blocks stream from L2.
template <typename T, int NXM>
__device__ __forceinline__ T rowdot_wide(int nx, int i, const T *D, const T *L, const T *U,
                                         const T *vprev, const T *vself, const T *vnext) {
    T d[NXM], l[NXM], u[NXM];
#pragma unroll
    for (int j = 0; j < NXM; ++j) {
        const bool in = j < nx;
        d[j] = in ? __ldg(D + j * nx + i) : T(0);
        l[j] = (in && L) ? __ldg(L + i * nx + j) : T(0);
        u[j] = (in && U) ? __ldg(U + j * nx + i) : T(0);
    }
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
    for (int j = 0; j < NXM; ++j) {
        a0 = fma_rn(d[j], vself[j], a0);
        a1 = fma_rn(l[j], vprev[j], a1);
        a2 = fma_rn(u[j], vnext[j], a2);
    }
    return (a0 + a1) + a2;
}

// Initial residual b_i - (row i) . v with exact products and an extended
// sum.  A warm start lambda_0 makes b - S lambda_0 a difference of nearly
// equal vectors; rounding it to working precision would leave an error
// close to the exit tolerance in r_0 that the recurrence r -= alpha S p
// never removes.
template <typename T>
__device__ __forceinline__ T resid_ptr(int nx, int i, T b, const T *D, const T *L, const T *U,
                                       const T *vprev, const T *vself, const T *vnext) {
    using AT = Acc<T>;
    typename AT::type a = AT::prod(b, T(1));
    for (int j = 0; j < nx; ++j) a = AT::add(a, AT::prod(-D[j * nx + i], vself[j]));
    if (L)
        for (int j = 0; j < nx; ++j) a = AT::add(a, AT::prod(-L[i * nx + j], vprev[j]));
    if (U)
        for (int j = 0; j < nx; ++j) a = AT::add(a, AT::prod(-U[j * nx + i], vnext[j]));
    return AT::to_T(a);
}

}  // namespace mpcg
