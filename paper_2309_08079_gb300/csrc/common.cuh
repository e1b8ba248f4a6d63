// Device utilities shared by the mpcg kernels: extended-precision
// accumulators, thread-block-cluster primitives (inline PTX, sm_90+ ISA,
// compiled for sm_103a) and instance bookkeeping for ragged batches.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/mpcg.h"

namespace mpcg {

// ---------------------------------------------------------------------------
// Accumulators.  GB300's FP64 pipe runs at a small fraction of its FP32 rate,
// so float32 dot products are accumulated as unevaluated float pairs
// (hi + lo, "double-float"): the product of two floats is split exactly with
// one FMA, and pairs are added with Knuth's TwoSum.  Both operations are
// exact transformations, commutative in their operands, and give about 44
// significant bits.  The float64 path accumulates in plain double.
// ---------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return dfloat{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    float s = __fadd_rn(x.hi, y.hi);
    float bb = __fsub_rn(s, x.hi);
    float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    float hi = __fadd_rn(s, e);
    return dfloat{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

// Tree form of the pair addition: the high parts are added with TwoSum and
// the rounding error is carried into the low part without renormalising.
// Exact in the high part, commutative, and about 35% shorter on the
// dependency chain than df_add; used for shuffle and slot reductions.
__device__ __forceinline__ dfloat df_add_lazy(dfloat a, dfloat b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return dfloat{s, __fadd_rn(__fadd_rn(a.lo, b.lo), e)};
}

// float-pair times a float, renormalised
__device__ __forceinline__ dfloat df_mul_f(dfloat x, float b) {
    float p = __fmul_rn(x.hi, b);
    float e = __fmaf_rn(x.hi, b, -p);
    e = __fmaf_rn(x.lo, b, e);
    float hi = __fadd_rn(p, e);
    return dfloat{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

// float-pair divided by a float (one correction step)
__device__ __forceinline__ dfloat df_div_f(dfloat x, float b) {
    float q1 = __fdiv_rn(x.hi, b);
    dfloat p = df_prod(q1, b);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    float q2 = __fdiv_rn(r, b);
    float hi = __fadd_rn(q1, q2);
    return dfloat{hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}

template <typename T>
struct Acc;

template <>
struct Acc<float> {
    using type = dfloat;
    __device__ static __forceinline__ dfloat zero() { return dfloat{0.f, 0.f}; }
    __device__ static __forceinline__ dfloat prod(float a, float b) { return df_prod(a, b); }
    __device__ static __forceinline__ dfloat add(dfloat a, dfloat b) { return df_add(a, b); }
    __device__ static __forceinline__ dfloat add_tree(dfloat a, dfloat b) { return df_add_lazy(a, b); }
    __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    __device__ static __forceinline__ dfloat shfl_xor(dfloat a, int m) {
        return dfloat{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
    }
    __device__ static __forceinline__ dfloat bcast0(dfloat a) {
        return dfloat{__shfl_sync(0xffffffffu, a.hi, 0), __shfl_sync(0xffffffffu, a.lo, 0)};
    }
    __device__ static __forceinline__ double to_double(dfloat a) {
        return (double)a.hi + (double)a.lo;
    }
    __device__ static __forceinline__ float to_T(dfloat a) { return __fadd_rn(a.hi, a.lo); }
    __device__ static __forceinline__ dfloat from(float a) { return dfloat{a, 0.f}; }
    __device__ static __forceinline__ dfloat neg(dfloat a) { return dfloat{-a.hi, -a.lo}; }
    // acc + a * x for a float a and an extended x
    __device__ static __forceinline__ dfloat fma_x(float a, dfloat x, dfloat acc) {
        return df_add(acc, df_mul_f(x, a));
    }
    __device__ static __forceinline__ dfloat div_x(dfloat x, float b) { return df_div_f(x, b); }
};

template <>
struct Acc<double> {
    using type = double;
    __device__ static __forceinline__ double zero() { return 0.0; }
    __device__ static __forceinline__ double prod(double a, double b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ double add_tree(double a, double b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ double div(double a, double b) { return a / b; }
    __device__ static __forceinline__ double shfl_xor(double a, int m) {
        return __shfl_xor_sync(0xffffffffu, a, m);
    }
    __device__ static __forceinline__ double bcast0(double a) { return __shfl_sync(0xffffffffu, a, 0); }
    __device__ static __forceinline__ double to_double(double a) { return a; }
    __device__ static __forceinline__ double to_T(double a) { return a; }
    __device__ static __forceinline__ double from(double a) { return a; }
    __device__ static __forceinline__ double neg(double a) { return -a; }
    __device__ static __forceinline__ double fma_x(double a, double x, double acc) { return __fma_rn(a, x, acc); }
    __device__ static __forceinline__ double div_x(double x, double b) { return x / b; }
};

// float32 storage with float64 accumulation (mpcg_opts.dot = 1): products of
// two floats are exact in double, partial sums are rounded FP64 additions;
// the iteration's scalars are still taken in float.
struct AccF64 {
    using type = double;
    __device__ static __forceinline__ double zero() { return 0.0; }
    __device__ static __forceinline__ double prod(float a, float b) {
        return __dmul_rn((double)a, (double)b);
    }
    __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ double add_tree(double a, double b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    __device__ static __forceinline__ double shfl_xor(double a, int m) {
        return __shfl_xor_sync(0xffffffffu, a, m);
    }
    __device__ static __forceinline__ double to_double(double a) { return a; }
    __device__ static __forceinline__ float to_T(double a) { return __double2float_rn(a); }
};

template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) {
    return __fma_rn(a, b, c);
}

// ---------------------------------------------------------------------------
// Thread-block cluster primitives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t num_clusters_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// Full cluster barrier: release orders this thread's earlier shared and
// distributed-shared stores before the arrival, acquire makes the peers'
// stores visible after the wait.  Every thread of every CTA takes part.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Named CTA barrier `id` (1..15) over `n` threads: producers arrive without
// waiting, the consumer waits for all n; the producers' earlier shared-memory
// stores are visible to the consumer after its bar.sync.
__device__ __forceinline__ void named_bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Address of the same shared-memory variable in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, dfloat v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.hi), "f"(v.lo)
                 : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// mbarrier-completed distributed-shared-memory pushes.  st.async writes a
// value into a peer CTA's shared memory and completes `bytes` of
// transaction count on the peer's mbarrier; the receiver waits for the
// phase, so no cluster-wide barrier or sender-side fence is needed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One local arrival that also raises the phase's expected transaction bytes.
// Relaxed: the arrival publishes no data of its own (the payload completes
// through st.async transaction bytes), so it orders nothing before it.
__device__ __forceinline__ void mbar_arrive_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Non-blocking probe of the phase of `parity` (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` with a deadline; false if it gave up.  The
// first microseconds spin on test_wait (a suspended try_wait can wake late
// on the critical path); after that try_wait lets the thread sleep.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, uint64_t limit_ns) {
    for (int i = 0; i < 4096; ++i)
        if (mbar_test_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// As mbar_wait_bounded without the spin: try_wait from the start, so a
// waiting warp leaves its issue slots to the SM's other warps (for kernels
// whose warps stream independently rather than wait on one critical path).
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint32_t mbar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// As mbar_wait_bounded, and also gives up once the word at shared address
// `abort_flag` (this CTA's shared memory) is non-zero: a peer that has given
// up sets it.  The flag is read only after the fast spin, so a healthy
// exchange never pays for it.
__device__ __forceinline__ bool mbar_wait_bounded_abort(uint32_t mbar, uint32_t parity, uint64_t limit_ns,
                                                        const volatile int *abort_flag) {
    for (int i = 0; i < 4096; ++i)
        if (mbar_test_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// One arrival on the mbarrier at shared::cluster address `mbar` (a peer's),
// ordered after this thread's earlier memory operations (release, cluster).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t mbar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_cluster() {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
}

// Bounded busy wait of about `ns` nanoseconds.
__device__ __forceinline__ void spin_ns(uint64_t ns) {
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < ns) {
    }
}

// Leaving a cluster after a wait gave up (called by one thread of the CTA).
// A CTA must not leave while peers may still push into its shared memory:
// it tells every peer to stop (their bounded waits poll `abort_flag`),
// reports to every peer that it has stopped pushing (one arrival on each
// peer's `stopped` mbarrier, initialised with C - 1 arrivals), waits up to
// `limit_ns` until every peer has reported the same, and lets pushes
// already in flight land (`grace_ns`).  Best effort: a peer that is stuck
// for good never reports, and the wait gives up.  Returns true if every
// peer reported.
__device__ __forceinline__ bool cluster_drain(uint32_t rank, uint32_t C, uint32_t abort_flag, uint32_t stopped,
                                              uint64_t limit_ns, uint64_t grace_ns) {
    if (C < 2) return true;
    for (uint32_t q = 0; q < C; ++q)
        if (q != rank) st_cluster(map_rank(abort_flag, q), 1);
    fence_acq_rel_cluster();
    for (uint32_t q = 0; q < C; ++q)
        if (q != rank) mbar_arrive_remote(map_rank(stopped, q));
    const bool all = mbar_wait_bounded(stopped, 0u, limit_ns);
    spin_ns(grace_ns);
    return all;
}

__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"(__double_as_longlong(v)), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, dfloat v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(
                     addr),
                 "r"(__float_as_uint(v.hi)), "r"(__float_as_uint(v.lo)), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void st_async_v4(uint32_t addr, float a, float b, float c, float d,
                                            uint32_t mbar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
        "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
        "r"(mbar)
        : "memory");
}

// Bulk (TMA, 1-D) copy of `bytes` from global to this CTA's shared memory,
// completing on `mbar`.  Both addresses 16-byte aligned, bytes % 16 == 0.
// Orders this thread's (and, after a warp or CTA barrier, its peers')
// generic-proxy accesses to shared memory before later async-proxy (TMA)
// writes to the same locations.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_smem),
        "l"(__cvta_generic_to_global(src_gmem)), "r"(bytes), "r"(mbar)
        : "memory");
}

// ---------------------------------------------------------------------------
// Ragged batches: instance b owns knots [knot_off[b], knot_off[b+1]) and
// controls [knot_off[b] - b, knot_off[b+1] - b - 1).  A single instance is
// described by knot_off == nullptr and N1.
// ---------------------------------------------------------------------------
struct BatchView {
    const int *knot_off;
    int B;
    int N1;
    // b outside [0, B) (a bad instance-list entry) reads nothing and is an
    // empty instance
    __device__ __forceinline__ void range(int b, int &k0, int &n) const {
        if (b < 0 || b >= B) {
            k0 = 0;
            n = 0;
        } else if (knot_off) {
            k0 = knot_off[b];
            n = knot_off[b + 1] - k0;
        } else {
            k0 = 0;
            n = N1;
        }
    }
    // total knots of the batch
    __device__ __forceinline__ int total() const { return knot_off ? knot_off[B] : N1; }
    // instance that owns global knot kg (binary search over knot_off)
    __device__ __forceinline__ int owner(int kg) const {
        if (!knot_off) return 0;
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (knot_off[mid] <= kg) lo = mid; else hi = mid - 1;
        }
        return lo;
    }
};

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// An NVTX range over a host call (visible to Nsight and other NVTX tools; a
// no-op when none is attached).  The C ABI's entry points open one each.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define MPCG_NVTX(name) ::mpcg::NvtxRange mpcg_nvtx_range_(name)


}  // namespace mpcg
