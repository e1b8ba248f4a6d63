// Persistent, thread-block-cluster PCG for block-tridiagonal S+ (Algorithm 1,
// organised per block row as in Algorithm 2 of the paper).
//
// Launch shape: a grid of clusters of C CTAs (C <= 16).  A cluster solves
// one instance at a time and takes instances from a queue until the batch
// is exhausted.  CTA r of the cluster owns knots [r*KPC, (r+1)*KPC) of the
// instance (KPC = ceil(N/C)); inside the CTA, LPK consecutive threads own
// the rows of one knot, RPT rows per thread (rows li, li+LPK, ...).
//
// Data placement (GB300: 256 KB registers + 227 KB shared memory per SM):
//  * REG mode (float32, nx = 14): each thread keeps its two rows of S+ and
//    of Phi^-1 (row i of the diagonal block and of both neighbour blocks:
//    168 floats) in registers for the whole solve; the matrices are read
//    from global memory once per solve.
//  * PTR mode (any dtype / nx): the instance's blocks are staged once into
//    shared memory when they fit, else read from global memory (L2) each
//    iteration.
//  * p and r, with one halo knot on each side, live in shared memory; each
//    thread's rows of lambda, r, p stay in registers.
//
// Communication: two exchanges per iteration, one per reduction of
// Algorithm 1 (A: p^T S p; B: r^T r~ and ||r||^2).  Each warp reduces its
// lanes; the warps hand their partials to warp 0 through shared memory (a
// named barrier that only warp 0 waits on), and warp 0 pushes the CTA's
// partial with st.async into every CTA of the cluster (its own included).
// The pushes complete transaction bytes on the receiver's mbarrier, so a
// CTA waits only for the data it needs and no cluster-wide barrier or fence
// sits on the critical path.  One push per source CTA matters: a receiver
// takes in the pushes of an exchange one after another (measured on GB300:
// ~6.6 cycles each), and one push per warp (C*W = 128 at N = 512) made the
// exchange ~1.5x longer.  The same exchanges carry the halo rows the next
// phase needs (S p of the boundary knots with A, Phi^-1 r with B; in REG
// mode four 16-byte pushes per side), so Algorithm 2's separate neighbour
// loads of p and r cost nothing extra: a CTA updates its halo copies of r
// and p with the same fused multiply-adds the owner uses (bit-identical).
// Every CTA adds the C partials in the same butterfly order (the pair
// additions are commutative), so all CTAs take identical scalar decisions
// (alpha, beta, exit).
//
// Dot products: exact float products accumulated as float pairs (see
// common.cuh), or in float64 (mpcg_opts.dot = 1, the AccF64 policy); ||r||^2,
// used only by the exit test, is a sum of squares and is accumulated in
// plain working precision (in float64 with float64 accumulators).
#include <type_traits>

#include "pcg_rows.cuh"

namespace mpcg {

constexpr int CMAX = 16;
constexpr int WMAX = 16;  // warps per CTA (512 threads)

template <typename A>
struct PayB;  // payload of exchange B: (r^T r~, ||r||^2), by accumulator type
template <>
struct PayB<dfloat> {
    dfloat eta;
    float rr, pad;
};
template <>
struct PayB<double> {
    double eta, rr;
};

// ||r||^2 += r_i^2 in the payload's precision
__device__ __forceinline__ float rr_acc(float r, float acc) { return __fmaf_rn(r, r, acc); }
__device__ __forceinline__ double rr_acc(float r, double acc) { return __fma_rn((double)r, (double)r, acc); }
__device__ __forceinline__ double rr_acc(double r, double acc) { return __fma_rn(r, r, acc); }

// Shared-memory carve-up (dynamic).  Slot arrays hold one partial per
// source CTA, the wpart arrays one per warp of this CTA.  Offsets in bytes,
// computed identically on the host (pcg_smem_bytes) and the device.
// A: accumulator type.
template <typename T, typename A>
struct SmemLayout {
    size_t vecP, vecR, haloA, haloB, slotA, slotB, wpartA, wpartB, mbar, misc, mats, total;
    __host__ __device__ SmemLayout(int kpc_max, int vs, int W, int nx, int stage) {
        size_t o = 0;
        auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
        vecP = o; o = al(o + sizeof(T) * (kpc_max + 2) * vs);
        vecR = o; o = al(o + sizeof(T) * (kpc_max + 2) * vs);
        haloA = o; o = al(o + sizeof(T) * 2 * vs);
        haloB = o; o = al(o + sizeof(T) * 2 * vs);
        slotA = o; o = al(o + sizeof(A) * CMAX);
        slotB = o; o = al(o + sizeof(PayB<A>) * CMAX);
        wpartA = o; o = al(o + sizeof(A) * WMAX);
        wpartB = o; o = al(o + sizeof(PayB<A>) * WMAX);
        (void)W;
        mbar = o; o = al(o + 3 * sizeof(uint64_t));  // exchange A, exchange B, peers stopped
        misc = o; o = al(o + 16);
        mats = o;
        if (stage) o = al(o + sizeof(T) * (size_t)(4 * kpc_max + 2) * nx * nx);
        total = o;
    }
};

constexpr int NXR = 14;  // REG-mode block size

// Two rows of one block row times the halo'd vector (REG mode): the knot's
// three 16-float vector slots are read once for both rows.
__device__ __forceinline__ void rowdot_reg2(const float (&d)[2][NXR], const float (&l)[2][NXR],
                                            const float (&u)[2][NXR], const float *vprev,
                                            const float *vself, const float *vnext, float &y0,
                                            float &y1) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
    const float4 *s4 = reinterpret_cast<const float4 *>(vself);
    const float4 *p4 = reinterpret_cast<const float4 *>(vprev);
    const float4 *n4 = reinterpret_cast<const float4 *>(vnext);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 xs = s4[q], xp = p4[q], xn = n4[q];
        const float vs_[4] = {xs.x, xs.y, xs.z, xs.w};
        const float vp_[4] = {xp.x, xp.y, xp.z, xp.w};
        const float vn_[4] = {xn.x, xn.y, xn.z, xn.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * q + t;
            if (j < NXR) {
                a0 = __fmaf_rn(d[0][j], vs_[t], a0);
                b0 = __fmaf_rn(d[1][j], vs_[t], b0);
                a1 = __fmaf_rn(l[0][j], vp_[t], a1);
                b1 = __fmaf_rn(l[1][j], vp_[t], b1);
                a2 = __fmaf_rn(u[0][j], vn_[t], a2);
                b2 = __fmaf_rn(u[1][j], vn_[t], b2);
            }
        }
    }
    y0 = (a0 + a1) + a2;
    y1 = (b0 + b1) + b2;
}

__device__ __forceinline__ float resid_reg(float b, const float (&d)[NXR], const float (&l)[NXR],
                                           const float (&u)[NXR], const float *vprev,
                                           const float *vself, const float *vnext) {
    dfloat a{b, 0.f};
#pragma unroll
    for (int j = 0; j < NXR; ++j) {
        a = df_add(a, df_prod(-d[j], vself[j]));
        a = df_add(a, df_prod(-l[j], vprev[j]));
        a = df_add(a, df_prod(-u[j], vnext[j]));
    }
    return __fadd_rn(a.hi, a.lo);
}

__device__ __forceinline__ dfloat acc_add_tree(dfloat a, dfloat b) { return df_add_lazy(a, b); }
__device__ __forceinline__ double acc_add_tree(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ dfloat acc_shfl(dfloat a, int m) {
    return dfloat{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ double acc_shfl(double a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }

template <typename A>
__device__ __forceinline__ PayB<A> payb_add(const PayB<A> &x, const PayB<A> &y) {
    PayB<A> r;
    r.eta = acc_add_tree(x.eta, y.eta);
    r.rr = x.rr + y.rr;
    if constexpr (std::is_same<A, dfloat>::value) r.pad = 0.f;
    return r;
}
template <typename A>
__device__ __forceinline__ PayB<A> payb_shfl(const PayB<A> &x, int m) {
    PayB<A> r;
    r.eta = acc_shfl(x.eta, m);
    r.rr = __shfl_xor_sync(0xffffffffu, x.rr, m);
    if constexpr (std::is_same<A, dfloat>::value) r.pad = 0.f;
    return r;
}
template <typename A>
__device__ __forceinline__ PayB<A> payb_zero() {
    PayB<A> r;
    r.eta = A{};
    r.rr = 0;
    if constexpr (std::is_same<A, dfloat>::value) r.pad = 0.f;
    return r;
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const dfloat &v, uint32_t mbar) {
    st_async(addr, v, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const double &v, uint32_t mbar) {
    st_async(addr, v, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const PayB<dfloat> &v, uint32_t mbar) {
    st_async_v4(addr, v.eta.hi, v.eta.lo, v.rr, 0.f, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const PayB<double> &v, uint32_t mbar) {
    st_async(addr, v.eta, mbar);
    st_async(addr + 8, v.rr, mbar);
}

// REG mode keeps 168 matrix floats per thread: at most 256 threads per CTA.
template <int MODE>
constexpr int pcg_max_threads() { return MODE == MODE_REG ? 256 : 512; }

template <typename T, typename AT, int MODE, int LPK, int RPT>
__global__ void __launch_bounds__(pcg_max_threads<MODE>(), 1) pcg_cluster_kernel(const PcgParams<T> P) {
    using A = typename AT::type;
    using PB = PayB<A>;
    extern __shared__ __align__(16) unsigned char smem[];

    const uint32_t C = cluster_size();
    const uint32_t rank = cluster_rank();
    const int nthreads = blockDim.x;
    const int W = nthreads / 32;
    const int tid = threadIdx.x;
    const uint32_t warp = tid / 32, lane = tid % 32;
    const int kl = tid / LPK;  // local knot slot
    const int li = tid % LPK;  // lane within the knot
    const int nx = P.nx;
    const int vs = P.vs;

    SmemLayout<T, A> L(P.kpc_max, vs, W, nx, P.stage_smem);
    T *vecP = reinterpret_cast<T *>(smem + L.vecP);
    T *vecR = reinterpret_cast<T *>(smem + L.vecR);
    T *haloA = reinterpret_cast<T *>(smem + L.haloA);  // [0, vs): left nbr's last knot; [vs, 2vs): right nbr's first
    T *haloB = reinterpret_cast<T *>(smem + L.haloB);
    A *slotA = reinterpret_cast<A *>(smem + L.slotA);
    PB *slotB = reinterpret_cast<PB *>(smem + L.slotB);
    A *wpartA = reinterpret_cast<A *>(smem + L.wpartA);
    PB *wpartB = reinterpret_cast<PB *>(smem + L.wpartB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    int *s_inst = reinterpret_cast<int *>(smem + L.misc);
    int *s_abort = s_inst + 1;  // set by a peer that gave up waiting
    T *mats = reinterpret_cast<T *>(smem + L.mats);

    const bool has_left = rank > 0, has_right = rank + 1 < C;
    const uint32_t rl = has_left ? rank - 1 : rank, rr_ = has_right ? rank + 1 : rank;
    const uint32_t mbA = smem_u32(&mbar[0]), mbB = smem_u32(&mbar[1]);
    // peer addresses used by the exchanges
    const uint32_t mbA_l = map_rank(mbA, rl), mbA_r = map_rank(mbA, rr_);
    const uint32_t mbB_l = map_rank(mbB, rl), mbB_r = map_rank(mbB, rr_);
    const uint32_t hA_l = map_rank(smem_u32(haloA + vs), rl), hA_r = map_rank(smem_u32(haloA), rr_);
    const uint32_t hB_l = map_rank(smem_u32(haloB + vs), rl), hB_r = map_rank(smem_u32(haloB), rr_);
    // lane q < C of warp 0 pushes the CTA's partial to slot [rank] of CTA q
    const uint32_t peer = lane < C ? lane : 0;
    const uint32_t slotA_peer = map_rank(smem_u32(slotA + rank), peer);
    const uint32_t slotB_peer = map_rank(smem_u32(slotB + rank), peer);
    const uint32_t mbA_peer = map_rank(mbA, peer), mbB_peer = map_rank(mbB, peer);
    const uint32_t bytesA_slots = C * (uint32_t)sizeof(A), bytesB_slots = C * (uint32_t)sizeof(PB);
    // butterfly widths: warps per CTA and CTAs per cluster, rounded up to powers of two (<= 16)
    int wpow = 1, cpow = 1;
    while (wpow < W) wpow <<= 1;
    while (cpow < (int)C) cpow <<= 1;
    // REG mode sends a boundary knot's 16-float slot (14 rows and 2 zeros) as
    // four 16-byte pushes; PTR mode one push per row
    const uint32_t side_bytes = MODE == MODE_REG ? 16u * (uint32_t)sizeof(float) : (uint32_t)(nx * sizeof(T));
    const uint32_t halo_bytes = side_bytes * ((has_left ? 1u : 0u) + (has_right ? 1u : 0u));

    const uint32_t mbS = smem_u32(&mbar[2]);  // one arrival per peer that has stopped pushing
    if (tid == 0) {
        mbar_init(mbA, 1);
        mbar_init(mbB, 1);
        mbar_init(mbS, C > 1 ? C - 1 : 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    cluster_sync_all();  // peers may push only after every mbarrier is initialised
    uint32_t phA = 0, phB = 0;
    bool timed_out = false;

    int served = 0;
    for (;;) {
        // ---- take the next instance ---------------------------------------
        if (rank == 0 && tid == 0) {
            int b;
            if (P.queue) b = atomicAdd(P.queue, 1);
            else b = (int)(cluster_id_x() + (uint32_t)served * num_clusters_x());
            b = b >= P.n_tickets ? -1 : (P.inst_list ? P.inst_list[b] : b);
            for (uint32_t q = 0; q < C; ++q) st_cluster(map_rank(smem_u32(s_inst), q), b);
        }
        cluster_sync_all();
        const int b = *s_inst;
        ++served;
        if (b < 0) break;

        int k0, Nb;
        P.bv.range(b, k0, Nb);
        const int c0 = k0 - b;  // first control/off-diagonal index
        const int KPC = ceil_div(Nb, (int)C);
        const int kfirst = (int)rank * KPC;  // instance-local index of slot 0
        const int k = kfirst + kl;            // this thread's knot
        const bool active_knot = kl < KPC && k < Nb;
        // an instance longer than the launch was sized for is refused
        const bool bad = Nb < 1 || (P.info && P.info[b] != 0u) || KPC > P.kpc_max;
        const int max_iter = P.max_iter > 0 ? P.max_iter : 10 * Nb * nx;
        const bool send_left = kl == 0 && has_left;
        const bool send_right = kl == KPC - 1 && has_right;

        // ---- rows owned by this thread ------------------------------------
        int rows[RPT];
        bool rv[RPT], rx[RPT];
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            rows[m] = li + m * LPK;
            rx[m] = kl < KPC && rows[m] < nx;  // row slot exists (may lie past the horizon)
            rv[m] = active_knot && rows[m] < nx;
        }

        // REG mode: the thread's rows of S+ and Phi^-1 in registers.
        float sd[2][NXR], sl[2][NXR], su[2][NXR], qd[2][NXR], ql[2][NXR], qu[2][NXR];
        // PTR mode: block pointers (shared or global).
        const T *pSd = nullptr, *pSl = nullptr, *pSu = nullptr;
        const T *pPd = nullptr, *pPl = nullptr, *pPu = nullptr;
        const int nx2 = nx * nx;

        // Phi^-1 rows without off-diagonal blocks: every row for block Jacobi
        // (precon 1), the even knots' rows for the stair preconditioner (2)
        const bool jac = P.precon == 1 || (P.precon == 2 && (k & 1) == 0);
        if (!bad) {
            if constexpr (MODE == MODE_REG) {
                const bool hl = active_knot && k >= 1, hu = active_knot && k + 1 < Nb;
                const float *Sd = reinterpret_cast<const float *>(P.Sd) + (size_t)(k0 + k) * nx2;
                const float *Pd = reinterpret_cast<const float *>(P.Pd) + (size_t)(k0 + k) * nx2;
                const float *SoL = reinterpret_cast<const float *>(P.So) + (size_t)(c0 + k - 1) * nx2;
                const float *PoL = reinterpret_cast<const float *>(P.Po) + (size_t)(c0 + k - 1) * nx2;
                const float *SoU = reinterpret_cast<const float *>(P.So) + (size_t)(c0 + k) * nx2;
                const float *PoU = reinterpret_cast<const float *>(P.Po) + (size_t)(c0 + k) * nx2;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int i = rows[m];
                    const bool v = rv[m];
#pragma unroll
                    for (int j = 0; j < NXR; ++j) {
                        sd[m][j] = v ? __ldg(Sd + j * NXR + i) : 0.f;
                        qd[m][j] = v ? __ldg(Pd + j * NXR + i) : 0.f;
                        sl[m][j] = (v && hl) ? __ldg(SoL + i * NXR + j) : 0.f;
                        ql[m][j] = (v && hl && !jac) ? __ldg(PoL + i * NXR + j) : 0.f;
                        su[m][j] = (v && hu) ? __ldg(SoU + j * NXR + i) : 0.f;
                        qu[m][j] = (v && hu && !jac) ? __ldg(PoU + j * NXR + i) : 0.f;
                    }
                }
            } else {
                if (P.stage_smem) {
                    // own diagonal blocks and the KPC+1 neighbouring off-diagonal blocks
                    T *mSd = mats;
                    T *mPd = mSd + (size_t)P.kpc_max * nx2;
                    T *mSo = mPd + (size_t)P.kpc_max * nx2;
                    T *mPo = mSo + (size_t)(P.kpc_max + 1) * nx2;
                    const int nd = max(0, min(KPC, Nb - kfirst));
                    const size_t dn = (size_t)nd * nx2;
                    const T *gSd = P.Sd + (size_t)(k0 + kfirst) * nx2;
                    const T *gPd = P.Pd + (size_t)(k0 + kfirst) * nx2;
                    for (size_t e = tid; e < dn; e += nthreads) {
                        mSd[e] = gSd[e];
                        mPd[e] = gPd[e];
                    }
                    // off-diagonal slot m <-> So[kfirst + m - 1], valid for 1 <= kfirst+m <= Nb-1
                    const int m_lo = max(0, 1 - kfirst), m_hi = min(KPC, Nb - 1 - kfirst);
                    if (m_hi >= m_lo) {
                        const size_t on = (size_t)(m_hi - m_lo + 1) * nx2;
                        const T *gSo = P.So + (size_t)(c0 + kfirst + m_lo - 1) * nx2;
                        const T *gPo = P.Po + (size_t)(c0 + kfirst + m_lo - 1) * nx2;
                        T *dSo = mSo + (size_t)m_lo * nx2;
                        T *dPo = mPo + (size_t)m_lo * nx2;
                        for (size_t e = tid; e < on; e += nthreads) {
                            dSo[e] = gSo[e];
                            dPo[e] = gPo[e];
                        }
                    }
                    if (active_knot) {
                        pSd = mSd + (size_t)kl * nx2;
                        pPd = mPd + (size_t)kl * nx2;
                        if (k >= 1) { pSl = mSo + (size_t)kl * nx2; pPl = mPo + (size_t)kl * nx2; }
                        if (k + 1 < Nb) { pSu = mSo + (size_t)(kl + 1) * nx2; pPu = mPo + (size_t)(kl + 1) * nx2; }
                    }
                } else if (active_knot) {
                    pSd = P.Sd + (size_t)(k0 + k) * nx2;
                    pPd = P.Pd + (size_t)(k0 + k) * nx2;
                    if (k >= 1) { pSl = P.So + (size_t)(c0 + k - 1) * nx2; pPl = P.Po + (size_t)(c0 + k - 1) * nx2; }
                    if (k + 1 < Nb) { pSu = P.So + (size_t)(c0 + k) * nx2; pPu = P.Po + (size_t)(c0 + k) * nx2; }
                }
                if (jac) pPl = pPu = nullptr;
            }
        }

        // y[m] = (row rows[m] of S+ or Phi^-1) . vec (halo'd)
        auto matvec = [&](bool precon, const T *vec, T (&y)[RPT]) {
            const T *vp = vec + kl * vs, *vsf = vec + (kl + 1) * vs, *vn = vec + (kl + 2) * vs;
            if constexpr (MODE == MODE_REG) {
                float y0 = 0.f, y1 = 0.f;
                if (active_knot) {
                    if (precon) rowdot_reg2(qd, ql, qu, vp, vsf, vn, y0, y1);
                    else rowdot_reg2(sd, sl, su, vp, vsf, vn, y0, y1);
                }
                y[0] = y0;
                y[1] = y1;
            } else {
#pragma unroll
                for (int m = 0; m < RPT; ++m)
                    y[m] = rv[m] ? (precon ? rowdot_ptr<T>(nx, rows[m], pPd, pPl, pPu, vp, vsf, vn)
                                           : rowdot_ptr<T>(nx, rows[m], pSd, pSl, pSu, vp, vsf, vn))
                                 : T(0);
            }
        };

        // the warps holding the first and last knot slot (warp-uniform)
        const bool warp_left = has_left && warp == 0;
        const bool warp_right = has_right && (int)warp == ((KPC - 1) * LPK) / 32;
        // Push this knot's boundary rows into the neighbours' halo slots.
        auto push_halo = [&](uint32_t h_l, uint32_t m_l, uint32_t h_r, uint32_t m_r, const T (&val)[RPT]) {
            if constexpr (MODE == MODE_REG) {
                // Rows 4j..4j+3 gathered into lane j (< 4) of the knot's group:
                // row i sits in lane i % 8 as val[i / 8]; rows 14, 15 are zero.
                if (!(warp_left || warp_right)) return;
                const int base = (int)lane & ~(LPK - 1), j = (int)lane & (LPK - 1);
                const int src0 = base + (j & 1) * 4;
                float x[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float a = __shfl_sync(0xffffffffu, val[0], src0 + t);
                    const float b = __shfl_sync(0xffffffffu, val[1], src0 + t);
                    x[t] = (j & 2) ? b : a;
                }
                if (j < 4) {
                    const uint32_t off = 16u * (uint32_t)j;
                    if (send_left) st_async_v4(h_l + off, x[0], x[1], x[2], x[3], m_l);
                    if (send_right) st_async_v4(h_r + off, x[0], x[1], x[2], x[3], m_r);
                }
            } else {
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!rx[m]) continue;
                    const uint32_t off = rows[m] * (uint32_t)sizeof(T);
                    if (send_left) st_async(h_l + off, val[m], m_l);
                    if (send_right) st_async(h_r + off, val[m], m_r);
                }
            }
        };

        // Exchange A: cluster sum of one accumulator per thread.  Each warp
        // reduces its lanes; lane 0 stores the warp partial, the other warps
        // arrive on named barrier 1 and go on to the exchange's CTA barrier,
        // warp 0 waits there, adds the W partials and its lanes q < C push
        // the CTA partial into slot [rank] of CTA q.  After the wait every
        // warp adds the C slots (butterfly over lanes mod cpow).
        auto exchangeA = [&](A v) -> A {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) v = AT::add_tree(v, AT::shfl_xor(v, m));
            if (lane == 0) wpartA[warp] = v;
            if (warp == 0) {
                named_bar_sync(1, nthreads);
                // every group of wpow lanes loads the W partials, so every
                // lane (in particular lanes q < C) ends with the CTA total
                const int wq = (int)lane & (wpow - 1);
                A y = wq < W ? wpartA[wq] : AT::zero();
                for (int m = wpow >> 1; m >= 1; m >>= 1) y = AT::add_tree(y, AT::shfl_xor(y, m));
                if (lane < C) st_async_pay(slotA_peer, y, mbA_peer);
            } else {
                named_bar_arrive(1, nthreads);
            }
            int fail = 0;
            if (tid == 0) {
                mbar_arrive_expect(mbA, bytesA_slots + halo_bytes);
                fail = !mbar_wait_bounded_abort(mbA, phA, WAIT_LIMIT_NS, s_abort);
            }
            phA ^= 1u;
            if (__syncthreads_or(fail)) timed_out = true;
            const int q = (int)lane & (cpow - 1);
            A t = q < (int)C ? slotA[q] : AT::zero();
            for (int m = cpow >> 1; m >= 1; m >>= 1) t = AT::add_tree(t, AT::shfl_xor(t, m));
            return t;
        };
        // Exchange B: cluster sums of (r^T r~, ||r||^2), same pattern.
        auto exchangeB = [&](PB v) -> PB {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) v = payb_add<A>(v, payb_shfl<A>(v, m));
            if (lane == 0) wpartB[warp] = v;
            if (warp == 0) {
                named_bar_sync(1, nthreads);
                const int wq = (int)lane & (wpow - 1);
                PB y = wq < W ? wpartB[wq] : payb_zero<A>();
                for (int m = wpow >> 1; m >= 1; m >>= 1) y = payb_add<A>(y, payb_shfl<A>(y, m));
                if (lane < C) st_async_pay(slotB_peer, y, mbB_peer);
            } else {
                named_bar_arrive(1, nthreads);
            }
            int fail = 0;
            if (tid == 0) {
                mbar_arrive_expect(mbB, bytesB_slots + halo_bytes);
                fail = !mbar_wait_bounded_abort(mbB, phB, WAIT_LIMIT_NS, s_abort);
            }
            phB ^= 1u;
            if (__syncthreads_or(fail)) timed_out = true;
            const int q = (int)lane & (cpow - 1);
            PB t = q < (int)C ? slotB[q] : payb_zero<A>();
            for (int m = cpow >> 1; m >= 1; m >>= 1) t = payb_add<A>(t, payb_shfl<A>(t, m));
            return t;
        };

        T lam_r[RPT], r_r[RPT], p_r[RPT];
        int iters = 0, status = MPCG_CONVERGED;
        A eta = AT::zero(), bb = AT::zero();
        T rr_t = T(0);

        if (bad) {
            status = MPCG_BADINPUT;
        } else {
            // ---- initialisation: r = b - S lambda0; p = r~ = Phi^-1 r ------
            for (int e = tid; e < (P.kpc_max + 2) * vs; e += nthreads) {
                vecP[e] = T(0);
                vecR[e] = T(0);
            }
            __syncthreads();
            T bv[RPT];
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                lam_r[m] = T(0);
                bv[m] = T(0);
                if (rv[m]) {
                    lam_r[m] = P.lam[(size_t)(k0 + k) * nx + rows[m]];
                    bv[m] = P.rhs_sign * P.rhs[(size_t)(k0 + k) * nx + rows[m]];
                    vecP[(kl + 1) * vs + rows[m]] = lam_r[m];
                }
            }
            // lambda0 halo straight from global memory
            if (kl == 0 && kfirst >= 1 && kfirst - 1 < Nb)
                for (int m = 0; m < RPT; ++m)
                    if (rows[m] < nx) vecP[rows[m]] = P.lam[(size_t)(k0 + kfirst - 1) * nx + rows[m]];
            if (kl == KPC - 1 && kfirst + KPC < Nb)
                for (int m = 0; m < RPT; ++m)
                    if (rows[m] < nx)
                        vecP[(KPC + 1) * vs + rows[m]] = P.lam[(size_t)(k0 + kfirst + KPC) * nx + rows[m]];
            __syncthreads();
            A sb = AT::zero();
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                r_r[m] = T(0);
                if (rv[m]) {
                    const T *vp = vecP + kl * vs, *vsf = vecP + (kl + 1) * vs, *vn = vecP + (kl + 2) * vs;
                    if constexpr (MODE == MODE_REG)
                        r_r[m] = resid_reg(bv[m], sd[m], sl[m], su[m], vp, vsf, vn);
                    else
                        r_r[m] = resid_ptr<T>(nx, rows[m], bv[m], pSd, pSl, pSu, vp, vsf, vn);
                }
                sb = AT::add(sb, AT::prod(bv[m], bv[m]));
                if (rx[m]) vecR[(kl + 1) * vs + rows[m]] = r_r[m];
            }
            push_halo(hA_l, mbA_l, hA_r, mbA_r, r_r);
            bb = exchangeA(sb);
            if (!timed_out) {
                if (kl == 0 && has_left)
                    for (int m = 0; m < RPT; ++m)
                        if (rows[m] < nx) vecR[rows[m]] = haloA[rows[m]];
                if (kl == KPC - 1 && has_right)
                    for (int m = 0; m < RPT; ++m)
                        if (rows[m] < nx) vecR[(KPC + 1) * vs + rows[m]] = haloA[vs + rows[m]];
                __syncthreads();
                T rt[RPT];
                matvec(true, vecR, rt);
                PB s2 = payb_zero<A>();
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    s2.eta = AT::add(s2.eta, AT::prod(r_r[m], rt[m]));
                    s2.rr = rr_acc(r_r[m], s2.rr);
                    p_r[m] = rt[m];
                    if (rx[m]) vecP[(kl + 1) * vs + rows[m]] = rt[m];
                }
                push_halo(hB_l, mbB_l, hB_r, mbB_r, rt);
                s2 = exchangeB(s2);
                eta = s2.eta;
                rr_t = (T)s2.rr;
            }
            if (!timed_out) {
                if (kl == 0 && has_left)
                    for (int m = 0; m < RPT; ++m)
                        if (rows[m] < nx) vecP[rows[m]] = haloB[rows[m]];
                if (kl == KPC - 1 && has_right)
                    for (int m = 0; m < RPT; ++m)
                        if (rows[m] < nx) vecP[(KPC + 1) * vs + rows[m]] = haloB[vs + rows[m]];
                __syncthreads();
            }

            // Scalars of the iteration (alpha, beta, exit tests) are taken in the
            // working precision T from the extended accumulators: the float path
            // issues no FP64 instruction inside the loop.
            const double tol = P.tol > 0 ? P.tol : 1e-6;
            const T tol_eta = (T)tol;
            const T tol_rr = (T)(tol * tol * AT::to_double(bb));
            auto converged = [&](T rr_, T eta_) -> bool {
                if (P.tol_mode == 1) return eta_ < tol_eta;
                return rr_ <= tol_rr;
            };
            T eta_t = AT::to_T(eta);

            if (timed_out) {
                status = MPCG_TIMEOUT;
            } else if (!(isfinite(eta_t) && isfinite(rr_t))) {
                status = MPCG_NONFINITE;
            } else if (!converged(rr_t, eta_t)) {
                status = MPCG_NOT_CONVERGED;
                for (int it = 1; it <= max_iter; ++it) {
                    // ---- Upsilon = S p, upsilon = p^T S p ---------------------------
                    T up[RPT];
                    matvec(false, vecP, up);
                    A s1 = AT::zero();
#pragma unroll
                    for (int m = 0; m < RPT; ++m) s1 = AT::add(s1, AT::prod(p_r[m], up[m]));
                    push_halo(hA_l, mbA_l, hA_r, mbA_r, up);
                    s1 = exchangeA(s1);
                    iters = it;
                    // the boundary slots' halo operands do not depend on alpha:
                    // load them before it is formed (one side per thread; a
                    // thread owning both, when a CTA has one knot slot, loads
                    // its right side late)
                    T hh[RPT], hv[RPT];
                    const bool hleft = kl == 0 && has_left, hright = kl == KPC - 1 && has_right;
                    const int hbase = hleft ? 0 : (KPC + 1) * vs, hoff = hleft ? 0 : vs;
                    const bool hboth = hleft && hright;
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        hh[m] = hv[m] = T(0);
                        if ((hleft || hright) && rows[m] < nx) {
                            hh[m] = haloA[hoff + rows[m]];
                            hv[m] = vecR[hbase + rows[m]];
                        }
                    }
                    if (timed_out) {
                        status = MPCG_TIMEOUT;
                        break;
                    }
                    const T ups = AT::to_T(s1);
                    if (!(ups > T(0)) || !isfinite(ups)) {
                        status = MPCG_BREAKDOWN;
                        break;
                    }
                    const T alpha = AT::div(eta_t, ups);
                    // ---- lambda += alpha p; r -= alpha Upsilon (own + halo) ---------
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        lam_r[m] = fma_rn(alpha, p_r[m], lam_r[m]);
                        r_r[m] = fma_rn(-alpha, up[m], r_r[m]);
                        if (rx[m]) vecR[(kl + 1) * vs + rows[m]] = r_r[m];
                    }
                    if (hleft || hright)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) vecR[hbase + rows[m]] = fma_rn(-alpha, hh[m], hv[m]);
                    if (hboth)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) {
                                T *x = &vecR[(KPC + 1) * vs + rows[m]];
                                *x = fma_rn(-alpha, haloA[vs + rows[m]], *x);
                            }
                    __syncthreads();
                    // ---- r~ = Phi^-1 r; eta' = r^T r~, ||r||^2 ----------------------
                    T rt[RPT];
                    matvec(true, vecR, rt);
                    PB s2 = payb_zero<A>();
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        s2.eta = AT::add(s2.eta, AT::prod(r_r[m], rt[m]));
                        s2.rr = rr_acc(r_r[m], s2.rr);
                    }
                    push_halo(hB_l, mbB_l, hB_r, mbB_r, rt);
                    s2 = exchangeB(s2);
                    if (timed_out) {
                        status = MPCG_TIMEOUT;
                        break;
                    }
                    // halo operands of the p update, loaded before beta is formed
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        hh[m] = hv[m] = T(0);
                        if ((hleft || hright) && rows[m] < nx) {
                            hh[m] = haloB[hoff + rows[m]];
                            hv[m] = vecP[hbase + rows[m]];
                        }
                    }
                    const T etan = AT::to_T(s2.eta);
                    rr_t = (T)s2.rr;
                    eta = s2.eta;
                    if (!isfinite(etan) || !isfinite(rr_t)) {
                        status = MPCG_NONFINITE;
                        break;
                    }
                    if (converged(rr_t, etan)) {
                        status = MPCG_CONVERGED;
                        break;
                    }
                    // ---- p = r~ + beta p (own + halo) -------------------------------
                    const T beta = AT::div(etan, eta_t);
                    eta_t = etan;
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        p_r[m] = fma_rn(beta, p_r[m], rt[m]);
                        if (rx[m]) vecP[(kl + 1) * vs + rows[m]] = p_r[m];
                    }
                    if (hleft || hright)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) vecP[hbase + rows[m]] = fma_rn(beta, hv[m], hh[m]);
                    if (hboth)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) {
                                T *x = &vecP[(KPC + 1) * vs + rows[m]];
                                *x = fma_rn(beta, *x, haloB[vs + rows[m]]);
                            }
                    __syncthreads();
                }
            }
            // ---- write back ----------------------------------------------------
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (rv[m]) P.lam[(size_t)(k0 + k) * nx + rows[m]] = lam_r[m];
        }
        if (rank == 0 && tid == 0 && P.stats && b < P.bv.B) {
            mpcg_stats st;
            st.iters = iters;
            st.status = status;
            st.eta = AT::to_double(eta);
            const double bbd = AT::to_double(bb), rrd = (double)rr_t;
            st.relres = bbd > 0.0 ? sqrt(rrd / bbd) : sqrt(rrd);
            P.stats[b] = st;
        }
        // A CTA whose wait gave up (or that a peer told to stop) must not
        // enter another cluster-wide barrier, which a stuck peer would never
        // reach, nor leave while peers may still push into its shared
        // memory: it drains the cluster (cluster_drain) and leaves.
        if (timed_out) {
            if (tid == 0) cluster_drain(rank, C, smem_u32(s_abort), mbS, DRAIN_LIMIT_NS, DRAIN_GRACE_NS);
            __syncthreads();
            return;
        }
        // every CTA is done with this instance's shared data before the next
        // instance id is pushed
        cluster_sync_all();
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from api.cu).
// ---------------------------------------------------------------------------
template <typename T>
size_t pcg_smem_bytes(int kpc_max, int vs, int C, int W, int nx, int stage, int dot) {
    (void)C;
    if (sizeof(T) == 4 && !dot) return SmemLayout<T, dfloat>(kpc_max, vs, W, nx, stage).total;
    return SmemLayout<T, double>(kpc_max, vs, W, nx, stage).total;
}

template <typename T, typename AT>
static void (*pcg_fn_acc(const PcgLaunch &L))(const PcgParams<T>) {
    if constexpr (sizeof(T) == 4) {
        if (L.mode == MODE_REG) return pcg_cluster_kernel<float, AT, MODE_REG, 8, 2>;
    }
    if (L.lpk == 8) return pcg_cluster_kernel<T, AT, MODE_PTR, 8, 2>;
    if (L.lpk == 16) return pcg_cluster_kernel<T, AT, MODE_PTR, 16, 1>;
    if (L.rpt == 1) return pcg_cluster_kernel<T, AT, MODE_PTR, 32, 1>;
    return pcg_cluster_kernel<T, AT, MODE_PTR, 32, 2>;
}

template <typename T>
static void (*pcg_fn(const PcgLaunch &L))(const PcgParams<T>) {
    if constexpr (sizeof(T) == 4) {
        if (L.dot) return pcg_fn_acc<float, AccF64>(L);
    }
    return pcg_fn_acc<T, Acc<T>>(L);
}

template <typename T>
cudaError_t pcg_launch(const PcgLaunch &L, const PcgParams<T> &P0, cudaStream_t s) {
    PcgParams<T> P = P0;
    P.kpc_max = L.kpc_max;
    P.stage_smem = L.stage;
    P.vs = L.vs;
    void (*fn)(const PcgParams<T>) = pcg_fn<T>(L);
    // the function attributes were set once per device (pcg_prepare)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.C * L.clusters, 1, 1);
    cfg.blockDim = dim3(L.threads, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = L.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, P);
}

// Function attributes of every PCG instantiation, set once per device:
// the dynamic shared-memory ceiling is raised to the device's opt-in
// maximum (it is a ceiling, so one value serves every launch shape) and
// 16-CTA clusters are allowed.
template <typename T>
static cudaError_t prepare_one(void (*fn)(const PcgParams<T>), int smem_optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename T, typename AT>
static cudaError_t prepare_acc(int smem_optin) {
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        if ((e = prepare_one<T>(pcg_cluster_kernel<T, AT, MODE_REG, 8, 2>, smem_optin))) return e;
    }
    if ((e = prepare_one<T>(pcg_cluster_kernel<T, AT, MODE_PTR, 8, 2>, smem_optin))) return e;
    if ((e = prepare_one<T>(pcg_cluster_kernel<T, AT, MODE_PTR, 16, 1>, smem_optin))) return e;
    if ((e = prepare_one<T>(pcg_cluster_kernel<T, AT, MODE_PTR, 32, 1>, smem_optin))) return e;
    return prepare_one<T>(pcg_cluster_kernel<T, AT, MODE_PTR, 32, 2>, smem_optin);
}

cudaError_t pcg_prepare(int smem_optin) {
    cudaError_t e;
    if ((e = prepare_acc<float, Acc<float>>(smem_optin))) return e;
    if ((e = prepare_acc<float, AccF64>(smem_optin))) return e;
    return prepare_acc<double, Acc<double>>(smem_optin);
}

// Largest number of co-resident clusters of this shape (0 if it cannot run).
template <typename T>
int pcg_max_clusters(const PcgLaunch &L) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.C, 1, 1);
    cfg.blockDim = dim3(L.threads, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = L.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, pcg_fn<T>(L), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template cudaError_t pcg_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_max_clusters<float>(const PcgLaunch &);
template int pcg_max_clusters<double>(const PcgLaunch &);
template size_t pcg_smem_bytes<float>(int, int, int, int, int, int, int);
template size_t pcg_smem_bytes<double>(int, int, int, int, int, int, int);

}  // namespace mpcg
