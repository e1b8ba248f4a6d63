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

// The cluster all-reduce of the PCG kernels with nothing else around it: the
// latency floor of one reduction of Algorithm 1 on a given launch shape.
// Per exchange, as the float32 kernels do it: boundary warps push a 64-byte
// halo slot to each neighbour, every warp sums its lanes (shuffle
// butterfly of float pairs), warp 0 sums the warp partials (named barrier)
// and pushes the CTA partial into every CTA, one thread waits (bounded) for
// the C partials and the halos, a CTA barrier, every warp sums the C slots.
// Exchanges A and B alternate on their own buffers, as in the kernels.
constexpr int XB_CMAX = 16, XB_WMAX = 16;
struct XbenchSmem {
    dfloat slot[2][XB_CMAX];
    dfloat wpart[2][XB_WMAX];
    float halo[2][32];
    uint64_t mb[3];  // exchange A, exchange B, peers stopped
    int abort_flag;
};

__device__ __forceinline__ dfloat xb_butterfly(dfloat v, int width) {
    for (int m = width >> 1; m >= 1; m >>= 1) v = df_add_lazy(v, Acc<float>::shfl_xor(v, m));
    return v;
}

__global__ void __launch_bounds__(512, 1)
exchange_bench_kernel(int rounds, uint64_t limit_ns, int *status, unsigned long long *out) {
    __shared__ __align__(16) XbenchSmem S;
    const uint32_t C = cluster_size(), rank = cluster_rank();
    const int tid = threadIdx.x, nthreads = blockDim.x, W = nthreads / 32;
    const uint32_t warp = tid / 32, lane = tid % 32;
    int wpow = 1, cpow = 1;
    while (wpow < W) wpow <<= 1;
    while (cpow < (int)C) cpow <<= 1;
    const bool has_left = rank > 0, has_right = rank + 1 < C;
    if (tid == 0) {
        mbar_init(smem_u32(&S.mb[0]), 1);
        mbar_init(smem_u32(&S.mb[1]), 1);
        mbar_init(smem_u32(&S.mb[2]), C > 1 ? C - 1 : 1);
        S.abort_flag = 0;
        fence_mbar_init();
    }
    cluster_sync_all();
    const uint32_t peer = lane < C ? lane : 0;
    const uint32_t halo_bytes = 64u * ((has_left ? 1u : 0u) + (has_right ? 1u : 0u));
    uint32_t ph[2] = {0u, 0u};
    int fail = 0;
    dfloat v{1e-3f * (float)(tid + 1), 0.f};
    const unsigned long long c0 = clock64();
    const uint64_t g0 = global_ns();
    for (int r = 0; r < rounds && !fail; ++r) {
        for (int x = 0; x < 2 && !fail; ++x) {
            const uint32_t mb = smem_u32(&S.mb[x]);
            // halo slots: the first warp to the left neighbour, the last to the right
            if (lane < 4) {
                if (has_left && warp == 0)
                    st_async_v4(map_rank(smem_u32(&S.halo[x][16 + 4 * lane]), rank - 1), v.hi, v.lo, 0.f, 0.f,
                                map_rank(mb, rank - 1));
                if (has_right && (int)warp == W - 1)
                    st_async_v4(map_rank(smem_u32(&S.halo[x][4 * lane]), rank + 1), v.hi, v.lo, 0.f, 0.f,
                                map_rank(mb, rank + 1));
            }
            const dfloat w = xb_butterfly(v, 32);
            if (lane == 0) S.wpart[x][warp] = w;
            if (warp == 0) {
                named_bar_sync(1, nthreads);
                const int q = (int)lane & (wpow - 1);
                const dfloat y = xb_butterfly(q < W ? S.wpart[x][q] : dfloat{0.f, 0.f}, wpow);
                if (lane < C) st_async(map_rank(smem_u32(&S.slot[x][rank]), peer), y, map_rank(mb, peer));
            } else {
                named_bar_arrive(1, nthreads);
            }
            int f = 0;
            if (tid == 0) {
                mbar_arrive_expect(mb, C * (uint32_t)sizeof(dfloat) + halo_bytes);
                f = !mbar_wait_bounded_abort(mb, ph[x], limit_ns, &S.abort_flag);
            }
            ph[x] ^= 1u;
            if (__syncthreads_or(f)) fail = 1;
            const int q = (int)lane & (cpow - 1);
            const dfloat t = xb_butterfly(q < (int)C ? S.slot[x][q] : dfloat{0.f, 0.f}, cpow);
            v.lo = __fmaf_rn(t.hi, 1e-12f, v.lo);
        }
    }
    const unsigned long long c1 = clock64();
    const uint64_t g1 = global_ns();
    if (tid == 0) {
        status[rank] = fail ? MPCG_TIMEOUT : MPCG_CONVERGED;
        if (rank == 0) {
            out[0] = c1 - c0;
            out[1] = g1 - g0;
            out[2] = (unsigned long long)__float_as_uint(v.hi);  // keeps the arithmetic live
        }
    }
    if (fail) {
        if (tid == 0)
            cluster_drain(rank, C, smem_u32(&S.abort_flag), smem_u32(&S.mb[2]), limit_ns, 20000ull);
        __syncthreads();
        return;
    }
    cluster_sync_all();  // no CTA leaves while a peer may still write to it
}

}  // namespace
}  // namespace mpcg

using namespace mpcg;

extern "C" int mpcg_bench_exchange(mpcg_handle *h, int C, int W, int rounds, unsigned long long *out,
                                   int *status, void *stream) {
    if (!h || !out || !status || C < 1 || C > XB_CMAX || W < 1 || W > XB_WMAX || rounds < 1 ||
        rounds > 1000000)
        return MPCG_EINVAL;
    if (cudaFuncSetAttribute(exchange_bench_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
        cudaGetLastError();
        return MPCG_ECUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(32 * W, 1, 1);
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, exchange_bench_kernel, rounds, (uint64_t)1000000000ull,
                                             status, out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPCG_ECUDA;
    }
    return MPCG_OK;
}

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
