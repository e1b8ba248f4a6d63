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

// The give-up path of the PCG kernels in a four-CTA cluster: every CTA
// expects one 4-byte push from each of the other three.  mode 0: all push,
// every wait completes.  mode 1: CTA 0 withholds its pushes and gives up at
// once; the others cannot complete, and must be released by the abort flag
// that CTA 0's drain sets (long before their wait limit), then drain too.
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(32)
drain_selftest_kernel(int mode, uint64_t limit_ns, int *status, unsigned long long *elapsed) {
    __shared__ __align__(8) uint64_t bar[2];  // [0] the exchange, [1] peers stopped
    __shared__ float slot[4];
    __shared__ int abort_flag;
    const uint32_t rank = cluster_rank(), C = cluster_size();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) slot[i] = 0.0f;
        abort_flag = 0;
        mbar_init(smem_u32(&bar[0]), 1);
        mbar_init(smem_u32(&bar[1]), C - 1);
        fence_mbar_init();
    }
    cluster_sync_all();  // every barrier and flag initialised before any push
    int gave_up = 0;
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_ns();
        const uint32_t mb = smem_u32(&bar[0]);
        mbar_arrive_expect(mb, (C - 1) * (uint32_t)sizeof(float));
        if (mode == 1 && rank == 0) {
            gave_up = 1;
        } else {
            for (uint32_t q = 0; q < C; ++q)
                if (q != rank) st_async(map_rank(smem_u32(&slot[rank]), q), 1.0f, map_rank(mb, q));
            gave_up = !mbar_wait_bounded_abort(mb, 0u, limit_ns, &abort_flag);
        }
        if (gave_up) {
            const bool all = cluster_drain(rank, C, smem_u32(&abort_flag), smem_u32(&bar[1]), limit_ns, 20000ull);
            status[rank] = all ? MPCG_TIMEOUT : -MPCG_TIMEOUT;
        } else {
            status[rank] = MPCG_CONVERGED;
        }
        elapsed[rank] = global_ns() - t0;
    }
    gave_up = __shfl_sync(0xffffffffu, gave_up, 0);
    if (!gave_up) cluster_sync_all();  // no CTA leaves while a peer may still write to it
}

}  // namespace
}  // namespace mpcg

using namespace mpcg;

extern "C" int mpcg_selftest_drain(mpcg_handle *h, int mode, double limit_s, int *status,
                                   unsigned long long *elapsed_ns, void *stream) {
    if (!h || !status || !elapsed_ns || (mode != 0 && mode != 1) || !(limit_s >= 1e-3 && limit_s <= 1.0))
        return MPCG_EINVAL;
    drain_selftest_kernel<<<4, 32, 0, (cudaStream_t)stream>>>(mode, (uint64_t)(limit_s * 1e9), status,
                                                             elapsed_ns);
    return cudaGetLastError() == cudaSuccess ? MPCG_OK : MPCG_ECUDA;
}

extern "C" int mpcg_selftest_wait(mpcg_handle *h, int push, double limit_s, int *status,
                                  void *stream) {
    if (!h || !status || !(limit_s >= 1e-6 && limit_s <= 1.0)) return MPCG_EINVAL;
    wait_selftest_kernel<<<2, 32, 0, (cudaStream_t)stream>>>(push ? 1 : 0,
                                                            (uint64_t)(limit_s * 1e9), status);
    return cudaGetLastError() == cudaSuccess ? MPCG_OK : MPCG_ECUDA;
}
