// Diagnostic of the bounded waits (no counterpart in the paper).  Every
// exchange of the PCG kernels completes on an mbarrier that a peer CTA's
// st.async pushes fill, and the receiving thread waits for it with a
// %globaltimer deadline (mbar_wait_bounded) instead of forever, so a push
// that never comes ends the solve with MPCG_TIMEOUT and leaves the context
// usable.  This kernel runs that exact pattern in a two-CTA cluster: each
// CTA expects 4 bytes on its own mbarrier, each pushes 4 bytes to the other
// only when asked to, and each waits with the given deadline.
#include <cstdint>

#include "common.cuh"

namespace mpcg {
namespace {

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32)
wait_selftest_kernel(int push, uint64_t limit_ns, int *status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ float slot;
    const uint32_t rank = cluster_rank();
    if (threadIdx.x == 0) {
        slot = 0.0f;
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    cluster_sync_all();  // both barriers initialised before any push
    if (threadIdx.x == 0) {
        mbar_arrive_expect(smem_u32(&bar), (uint32_t)sizeof(float));
        if (push) {
            const uint32_t peer = rank ^ 1u;
            st_async(map_rank(smem_u32(&slot), peer), 1.0f, map_rank(smem_u32(&bar), peer));
        }
        const bool ok = mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns);
        status[rank] = ok && slot == 1.0f ? MPCG_CONVERGED : MPCG_TIMEOUT;
    }
    cluster_sync_all();  // no CTA leaves while a peer may still write to it
}

}  // namespace
}  // namespace mpcg

using namespace mpcg;

extern "C" int mpcg_selftest_wait(mpcg_handle *h, int push, double limit_s, int *status,
                                  void *stream) {
    if (!h || !status || !(limit_s >= 1e-6 && limit_s <= 1.0)) return MPCG_EINVAL;
    wait_selftest_kernel<<<2, 32, 0, (cudaStream_t)stream>>>(push ? 1 : 0,
                                                            (uint64_t)(limit_s * 1e9), status);
    return cudaGetLastError() == cudaSuccess ? MPCG_OK : MPCG_ECUDA;
}
