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
// Algorithm 1 (A: p^T S p; B: r^T r~ and ||r||^2).  Each CTA reduces its
// partial sum, then pushes it with st.async into every CTA of the cluster
// (its own included); the pushes complete transaction bytes on the
// receiver's mbarrier, so a CTA waits only for the data it needs and no
// cluster-wide barrier or fence sits on the critical path.  The same
// exchanges carry the halo rows the next phase needs (S p of the boundary
// knots with A, Phi^-1 r with B), so Algorithm 2's separate neighbour loads
// of p and r cost nothing extra: a CTA updates its halo copies of r and p
// with the same fused multiply-adds the owner uses (bit-identical).
// Every CTA adds the C partials in rank order, so all CTAs take identical
// scalar decisions (alpha, beta, exit).
//
// Dot products: exact float products accumulated as float pairs (see
// common.cuh); ||r||^2, used only by the exit test, is a sum of squares and
// is accumulated in plain working precision.
#include <type_traits>

#include "launch.cuh"

namespace mpcg {

constexpr int CMAX = 16;
constexpr uint64_t WAIT_LIMIT_NS = 4000000000ull;  // 4 s: never reached in a healthy run

template <typename T>
struct PayB;  // payload of exchange B: (r^T r~, ||r||^2)
template <>
struct PayB<float> {
    dfloat eta;
    float rr, pad;
};
template <>
struct PayB<double> {
    double eta, rr;
};

// Shared-memory carve-up (dynamic).  Slot arrays hold one partial per
// (source CTA, source warp).  Offsets in bytes, computed identically
// on the host (pcg_smem_bytes) and the device.
template <typename T>
struct SmemLayout {
    size_t vecP, vecR, haloA, haloB, slotA, slotB, mbar, misc, mats, total;
    __host__ __device__ SmemLayout(int kpc_max, int vs, int W, int nx, int stage) {
        using A = typename std::conditional<sizeof(T) == 4, dfloat, double>::type;
        size_t o = 0;
        auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
        vecP = o; o = al(o + sizeof(T) * (kpc_max + 2) * vs);
        vecR = o; o = al(o + sizeof(T) * (kpc_max + 2) * vs);
        haloA = o; o = al(o + sizeof(T) * 2 * vs);
        haloB = o; o = al(o + sizeof(T) * 2 * vs);
        slotA = o; o = al(o + sizeof(A) * CMAX * W);
        slotB = o; o = al(o + sizeof(PayB<T>) * CMAX * W);
        mbar = o; o = al(o + 2 * sizeof(uint64_t));
        misc = o; o = al(o + 16);
        mats = o;
        if (stage) o = al(o + sizeof(T) * (size_t)(4 * kpc_max + 2) * nx * nx);
        total = o;
    }
};

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

template <typename T>
__device__ __forceinline__ PayB<T> payb_add(const PayB<T> &x, const PayB<T> &y) {
    PayB<T> r;
    r.eta = Acc<T>::add_tree(x.eta, y.eta);
    r.rr = x.rr + y.rr;
    if constexpr (sizeof(T) == 4) r.pad = 0.f;
    return r;
}
template <typename T>
__device__ __forceinline__ PayB<T> payb_shfl(const PayB<T> &x, int m) {
    PayB<T> r;
    r.eta = Acc<T>::shfl_xor(x.eta, m);
    r.rr = __shfl_xor_sync(0xffffffffu, x.rr, m);
    if constexpr (sizeof(T) == 4) r.pad = 0.f;
    return r;
}
template <typename T>
__device__ __forceinline__ PayB<T> payb_zero() {
    PayB<T> r;
    r.eta = Acc<T>::zero();
    r.rr = T(0);
    if constexpr (sizeof(T) == 4) r.pad = 0.f;
    return r;
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const dfloat &v, uint32_t mbar) {
    st_async(addr, v, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const double &v, uint32_t mbar) {
    st_async(addr, v, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const PayB<float> &v, uint32_t mbar) {
    st_async_v4(addr, v.eta.hi, v.eta.lo, v.rr, 0.f, mbar);
}
__device__ __forceinline__ void st_async_pay(uint32_t addr, const PayB<double> &v, uint32_t mbar) {
    st_async(addr, v.eta, mbar);
    st_async(addr + 8, v.rr, mbar);
}

// REG mode keeps 168 matrix floats per thread: at most 256 threads per CTA.
template <int MODE>
constexpr int pcg_max_threads() { return MODE == MODE_REG ? 256 : 512; }

template <typename T, int MODE, int LPK, int RPT>
__global__ void __launch_bounds__(pcg_max_threads<MODE>(), 1) pcg_cluster_kernel(const PcgParams<T> P) {
    using AT = Acc<T>;
    using A = typename AT::type;
    using PB = PayB<T>;
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

    SmemLayout<T> L(P.kpc_max, vs, W, nx, P.stage_smem);
    T *vecP = reinterpret_cast<T *>(smem + L.vecP);
    T *vecR = reinterpret_cast<T *>(smem + L.vecR);
    T *haloA = reinterpret_cast<T *>(smem + L.haloA);  // [0, vs): left nbr's last knot; [vs, 2vs): right nbr's first
    T *haloB = reinterpret_cast<T *>(smem + L.haloB);
    A *slotA = reinterpret_cast<A *>(smem + L.slotA);
    PB *slotB = reinterpret_cast<PB *>(smem + L.slotB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    int *s_inst = reinterpret_cast<int *>(smem + L.misc);
    T *mats = reinterpret_cast<T *>(smem + L.mats);

    const bool has_left = rank > 0, has_right = rank + 1 < C;
    const uint32_t rl = has_left ? rank - 1 : rank, rr_ = has_right ? rank + 1 : rank;
    const uint32_t mbA = smem_u32(&mbar[0]), mbB = smem_u32(&mbar[1]);
    // peer addresses used by the exchanges
    const uint32_t mbA_l = map_rank(mbA, rl), mbA_r = map_rank(mbA, rr_);
    const uint32_t mbB_l = map_rank(mbB, rl), mbB_r = map_rank(mbB, rr_);
    const uint32_t hA_l = map_rank(smem_u32(haloA + vs), rl), hA_r = map_rank(smem_u32(haloA), rr_);
    const uint32_t hB_l = map_rank(smem_u32(haloB + vs), rl), hB_r = map_rank(smem_u32(haloB), rr_);
    // lane q < C of every warp pushes the warp's partial to slot [rank][warp] of CTA q
    const uint32_t peer = lane < C ? lane : 0;
    const uint32_t slotA_peer = map_rank(smem_u32(slotA + rank * W + warp), peer);
    const uint32_t slotB_peer = map_rank(smem_u32(slotB + rank * W + warp), peer);
    const uint32_t mbA_peer = map_rank(mbA, peer), mbB_peer = map_rank(mbB, peer);
    const uint32_t bytesA_slots = C * W * (uint32_t)sizeof(A), bytesB_slots = C * W * (uint32_t)sizeof(PB);
    const int nslots = (int)C * W;
    const uint32_t halo_bytes = (uint32_t)(nx * sizeof(T)) * ((has_left ? 1u : 0u) + (has_right ? 1u : 0u));

    if (tid == 0) {
        mbar_init(mbA, 1);
        mbar_init(mbB, 1);
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
        const bool bad = (P.info && P.info[b] != 0u) || Nb < 1 || KPC > P.kpc_max;
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
                        ql[m][j] = (v && hl) ? __ldg(PoL + i * NXR + j) : 0.f;
                        su[m][j] = (v && hu) ? __ldg(SoU + j * NXR + i) : 0.f;
                        qu[m][j] = (v && hu) ? __ldg(PoU + j * NXR + i) : 0.f;
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

        // Push this knot's boundary rows into the neighbours' halo slots.
        auto push_halo = [&](uint32_t h_l, uint32_t m_l, uint32_t h_r, uint32_t m_r, const T (&val)[RPT]) {
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!rx[m]) continue;
                const uint32_t off = rows[m] * (uint32_t)sizeof(T);
                if (send_left) st_async(h_l + off, val[m], m_l);
                if (send_right) st_async(h_r + off, val[m], m_r);
            }
        };

        // Exchange A: cluster sum of one accumulator per thread.  Each warp
        // reduces its lanes and pushes the warp partial into slot
        // [rank][warp] of every CTA; after the wait every warp adds the C*W
        // slots in one fixed order (lane-strided, then a shuffle tree).
        auto exchangeA = [&](A v) -> A {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) v = AT::add_tree(v, AT::shfl_xor(v, m));
            if (lane < C) st_async_pay(slotA_peer, v, mbA_peer);
            int fail = 0;
            if (tid == 0) {
                mbar_arrive_expect(mbA, bytesA_slots + halo_bytes);
                fail = !mbar_wait_bounded(mbA, phA, WAIT_LIMIT_NS);
            }
            phA ^= 1u;
            if (__syncthreads_or(fail)) timed_out = true;
            A t = AT::zero();
            for (int q = lane; q < nslots; q += 32) t = AT::add_tree(t, slotA[q]);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t = AT::add_tree(t, AT::shfl_xor(t, m));
            return t;
        };
        // Exchange B: cluster sums of (r^T r~, ||r||^2), same pattern.
        auto exchangeB = [&](PB v) -> PB {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) v = payb_add<T>(v, payb_shfl<T>(v, m));
            if (lane < C) st_async_pay(slotB_peer, v, mbB_peer);
            int fail = 0;
            if (tid == 0) {
                mbar_arrive_expect(mbB, bytesB_slots + halo_bytes);
                fail = !mbar_wait_bounded(mbB, phB, WAIT_LIMIT_NS);
            }
            phB ^= 1u;
            if (__syncthreads_or(fail)) timed_out = true;
            PB t = payb_zero<T>();
            for (int q = lane; q < nslots; q += 32) t = payb_add<T>(t, slotB[q]);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t = payb_add<T>(t, payb_shfl<T>(t, m));
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
                PB s2 = payb_zero<T>();
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    s2.eta = AT::add(s2.eta, AT::prod(r_r[m], rt[m]));
                    s2.rr = fma_rn(r_r[m], r_r[m], s2.rr);
                    p_r[m] = rt[m];
                    if (rx[m]) vecP[(kl + 1) * vs + rows[m]] = rt[m];
                }
                push_halo(hB_l, mbB_l, hB_r, mbB_r, rt);
                s2 = exchangeB(s2);
                eta = s2.eta;
                rr_t = s2.rr;
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
                    if (kl == 0 && has_left)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) vecR[rows[m]] = fma_rn(-alpha, haloA[rows[m]], vecR[rows[m]]);
                    if (kl == KPC - 1 && has_right)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) {
                                T *x = &vecR[(KPC + 1) * vs + rows[m]];
                                *x = fma_rn(-alpha, haloA[vs + rows[m]], *x);
                            }
                    __syncthreads();
                    // ---- r~ = Phi^-1 r; eta' = r^T r~, ||r||^2 ----------------------
                    T rt[RPT];
                    matvec(true, vecR, rt);
                    PB s2 = payb_zero<T>();
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        s2.eta = AT::add(s2.eta, AT::prod(r_r[m], rt[m]));
                        s2.rr = fma_rn(r_r[m], r_r[m], s2.rr);
                    }
                    push_halo(hB_l, mbB_l, hB_r, mbB_r, rt);
                    s2 = exchangeB(s2);
                    if (timed_out) {
                        status = MPCG_TIMEOUT;
                        break;
                    }
                    const T etan = AT::to_T(s2.eta);
                    rr_t = s2.rr;
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
                    if (kl == 0 && has_left)
                        for (int m = 0; m < RPT; ++m)
                            if (rows[m] < nx) vecP[rows[m]] = fma_rn(beta, vecP[rows[m]], haloB[rows[m]]);
                    if (kl == KPC - 1 && has_right)
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
        if (rank == 0 && tid == 0 && P.stats) {
            mpcg_stats st;
            st.iters = iters;
            st.status = status;
            st.eta = AT::to_double(eta);
            const double bbd = AT::to_double(bb), rrd = (double)rr_t;
            st.relres = bbd > 0.0 ? sqrt(rrd / bbd) : sqrt(rrd);
            P.stats[b] = st;
        }
        // a CTA whose wait gave up leaves at once: it must not enter another
        // cluster-wide barrier that a stuck peer would never reach
        if (timed_out) return;
        // every CTA is done with this instance's shared data before the next
        // instance id is pushed
        cluster_sync_all();
    }
}

// ---------------------------------------------------------------------------
// CTA-per-instance PCG (batched throughput form).  One CTA owns a whole
// instance: p, r, r~, S p and lambda live in shared memory for every knot,
// the rows of S+ and Phi^-1 are streamed from global memory (L2) in chunks
// of (threads / LPK) knots each iteration, and both reductions are CTA-wide
// (warp shuffle trees plus one barrier), so no cross-SM exchange sits on the
// critical path.  A persistent grid of such CTAs drains the instance queue:
// many instances progress at once instead of one per 16-SM cluster.
// ---------------------------------------------------------------------------
template <typename T>
struct CtaLayout {
    size_t lam, r, p, rt, up, wpart, misc, total;
    __host__ __device__ CtaLayout(int nmax, int vs, int W) {
        using A = typename std::conditional<sizeof(T) == 4, dfloat, double>::type;
        size_t o = 0;
        auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
        const size_t v = sizeof(T) * (size_t)(nmax + 2) * vs;
        lam = o; o = al(o + v);
        r = o; o = al(o + v);
        p = o; o = al(o + v);
        rt = o; o = al(o + v);
        up = o; o = al(o + v);
        wpart = o; o = al(o + 2 * sizeof(A) * W);
        misc = o; o = al(o + 16);
        total = o;
    }
};

template <typename T, int LPK, int RPT>
__global__ void __launch_bounds__(512, 1) pcg_cta_kernel(const PcgParams<T> P) {
    using AT = Acc<T>;
    using A = typename AT::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int W = nthreads / 32;
    const int warp = tid / 32, lane = tid % 32;
    const int kl = tid / LPK, li = tid % LPK;
    const int chunk = nthreads / LPK;  // knots per pass
    const int nx = P.nx, vs = P.vs;
    CtaLayout<T> L(P.kpc_max, vs, W);
    T *vlam = reinterpret_cast<T *>(smem + L.lam);
    T *vr = reinterpret_cast<T *>(smem + L.r);
    T *vp = reinterpret_cast<T *>(smem + L.p);
    T *vrt = reinterpret_cast<T *>(smem + L.rt);
    T *vup = reinterpret_cast<T *>(smem + L.up);
    A *wpart = reinterpret_cast<A *>(smem + L.wpart);
    int *s_inst = reinterpret_cast<int *>(smem + L.misc);
    const int nx2 = nx * nx;

    // CTA-wide sum of two accumulators (identical result in every thread)
    auto reduce2 = [&](A &x, A &y) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            x = AT::add_tree(x, AT::shfl_xor(x, m));
            y = AT::add_tree(y, AT::shfl_xor(y, m));
        }
        if (lane == 0) {
            wpart[2 * warp] = x;
            wpart[2 * warp + 1] = y;
        }
        __syncthreads();
        x = lane < W ? wpart[2 * lane] : AT::zero();
        y = lane < W ? wpart[2 * lane + 1] : AT::zero();
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            x = AT::add_tree(x, AT::shfl_xor(x, m));
            y = AT::add_tree(y, AT::shfl_xor(y, m));
        }
    };

    int served = 0;
    for (;;) {
        if (tid == 0) {
            int t = P.queue ? atomicAdd(P.queue, 1) : (int)(blockIdx.x + served * gridDim.x);
            *s_inst = t >= P.n_tickets ? -1 : (P.inst_list ? P.inst_list[t] : t);
        }
        __syncthreads();
        const int b = *s_inst;
        ++served;
        if (b < 0) break;
        int k0, Nb;
        P.bv.range(b, k0, Nb);
        const int c0 = k0 - b;
        const bool bad = (P.info && P.info[b] != 0u) || Nb < 1 || Nb > P.kpc_max;
        const int max_iter = P.max_iter > 0 ? P.max_iter : 10 * Nb * nx;
        int iters = 0, status = MPCG_CONVERGED;
        A eta = AT::zero(), bb = AT::zero();
        T rr_t = T(0);

        // rows of knot k (instance-local), PTR-style block pointers
        auto blocks = [&](int k, bool precon, const T *&D, const T *&Lo, const T *&U) {
            const T *Md = precon ? P.Pd : P.Sd;
            const T *Mo = precon ? P.Po : P.So;
            D = Md + (size_t)(k0 + k) * nx2;
            Lo = k >= 1 ? Mo + (size_t)(c0 + k - 1) * nx2 : nullptr;
            U = k + 1 < Nb ? Mo + (size_t)(c0 + k) * nx2 : nullptr;
        };
        // y = M v over all knots into out; returns the thread's partial dots
        // (v . y, v . v) accumulated in extended precision / plain T.
        auto apply = [&](bool precon, const T *v, T *out, A &dot, T &sq) {
            for (int kb = 0; kb < Nb; kb += chunk) {
                const int k = kb + kl;
                if (kl < chunk && k < Nb) {
                    const T *D, *Lo, *U;
                    blocks(k, precon, D, Lo, U);
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int i = li + m * LPK;
                        if (i < nx) {
                            T y;
                            if constexpr (LPK == 16)  // vs == 16: padded vector slots are zero
                                y = rowdot_wide<T, 16>(nx, i, D, Lo, U, v + k * vs, v + (k + 1) * vs, v + (k + 2) * vs);
                            else
                                y = rowdot_ptr<T>(nx, i, D, Lo, U, v + k * vs, v + (k + 1) * vs, v + (k + 2) * vs);
                            out[(k + 1) * vs + i] = y;
                            const T vi = v[(k + 1) * vs + i];
                            dot = AT::add(dot, AT::prod(vi, y));
                            sq = fma_rn(vi, vi, sq);
                        }
                    }
                }
            }
        };

        if (bad) {
            status = MPCG_BADINPUT;
        } else {
            const int nv = (Nb + 2) * vs;
            for (int e = tid; e < nv; e += nthreads) {
                vlam[e] = T(0); vr[e] = T(0); vp[e] = T(0); vrt[e] = T(0); vup[e] = T(0);
            }
            __syncthreads();
            for (int e = tid; e < Nb * nx; e += nthreads) {
                const int k = e / nx, i = e % nx;
                vlam[(k + 1) * vs + i] = P.lam[(size_t)(k0 + k) * nx + i];
            }
            __syncthreads();
            // r = b - S lambda0 (extended precision), ||b||^2
            A sbb = AT::zero(), dummy = AT::zero();
            for (int kb = 0; kb < Nb; kb += chunk) {
                const int k = kb + kl;
                if (kl < chunk && k < Nb) {
                    const T *D, *Lo, *U;
                    blocks(k, false, D, Lo, U);
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int i = li + m * LPK;
                        if (i < nx) {
                            const T bi = P.rhs_sign * P.rhs[(size_t)(k0 + k) * nx + i];
                            vr[(k + 1) * vs + i] = resid_ptr<T>(nx, i, bi, D, Lo, U, vlam + k * vs,
                                                                vlam + (k + 1) * vs, vlam + (k + 2) * vs);
                            sbb = AT::add(sbb, AT::prod(bi, bi));
                        }
                    }
                }
            }
            reduce2(sbb, dummy);
            bb = sbb;
            __syncthreads();  // r complete (and wpart read) before it is used
            A s_eta = AT::zero(), s_rr = AT::zero();
            T sq = T(0);
            apply(true, vr, vrt, s_eta, sq);
            s_rr = AT::prod(sq, T(1));
            reduce2(s_eta, s_rr);
            eta = s_eta;
            rr_t = AT::to_T(s_rr);
            __syncthreads();
            for (int e = tid; e < nv; e += nthreads) vp[e] = vrt[e];
            __syncthreads();

            const double tol = P.tol > 0 ? P.tol : 1e-6;
            const T tol_eta = (T)tol;
            const T tol_rr = (T)(tol * tol * AT::to_double(bb));
            auto converged = [&](T rr_, T eta_) -> bool {
                if (P.tol_mode == 1) return eta_ < tol_eta;
                return rr_ <= tol_rr;
            };
            T eta_t = AT::to_T(eta);
            if (!(isfinite(eta_t) && isfinite(rr_t))) {
                status = MPCG_NONFINITE;
            } else if (!converged(rr_t, eta_t)) {
                status = MPCG_NOT_CONVERGED;
                for (int it = 1; it <= max_iter; ++it) {
                    A s1 = AT::zero(), s1b = AT::zero();
                    T sq1 = T(0);
                    apply(false, vp, vup, s1, sq1);  // S p and p^T S p
                    reduce2(s1, s1b);
                    iters = it;
                    const T ups = AT::to_T(s1);
                    if (!(ups > T(0)) || !isfinite(ups)) {
                        status = MPCG_BREAKDOWN;
                        break;
                    }
                    const T alpha = AT::div(eta_t, ups);
                    for (int e = tid; e < Nb * vs; e += nthreads) {
                        const int o = vs + e;
                        vlam[o] = fma_rn(alpha, vp[o], vlam[o]);
                        vr[o] = fma_rn(-alpha, vup[o], vr[o]);
                    }
                    __syncthreads();
                    A s2 = AT::zero();
                    T sq2 = T(0);
                    apply(true, vr, vrt, s2, sq2);  // r~ = Phi^-1 r, r^T r~, ||r||^2
                    A s2b = AT::prod(sq2, T(1));
                    reduce2(s2, s2b);
                    const T etan = AT::to_T(s2);
                    rr_t = AT::to_T(s2b);
                    eta = s2;
                    if (!isfinite(etan) || !isfinite(rr_t)) {
                        status = MPCG_NONFINITE;
                        break;
                    }
                    if (converged(rr_t, etan)) {
                        status = MPCG_CONVERGED;
                        break;
                    }
                    const T beta = AT::div(etan, eta_t);
                    eta_t = etan;
                    for (int e = tid; e < Nb * vs; e += nthreads) {
                        const int o = vs + e;
                        vp[o] = fma_rn(beta, vp[o], vrt[o]);
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            for (int e = tid; e < Nb * nx; e += nthreads) {
                const int k = e / nx, i = e % nx;
                P.lam[(size_t)(k0 + k) * nx + i] = vlam[(k + 1) * vs + i];
            }
        }
        if (tid == 0 && P.stats) {
            mpcg_stats st;
            st.iters = iters;
            st.status = status;
            st.eta = AT::to_double(eta);
            const double bbd = AT::to_double(bb), rrd = (double)rr_t;
            st.relres = bbd > 0.0 ? sqrt(rrd / bbd) : sqrt(rrd);
            P.stats[b] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Streaming CTA-per-instance PCG (batched throughput form).  As
// pcg_cta_kernel, one CTA owns a whole instance with p, r, r~ and S p in
// shared memory, but the blocks of S+ and Phi^-1 reach shared memory by
// TMA bulk copies: each pass over the instance (S+ for the matvec, Phi^-1
// for the preconditioner) is cut into chunks of KC knots whose diagonal and
// off-diagonal blocks are contiguous in global memory, and chunk q+2 is
// copied into the stage chunk q just released while chunk q+1 is already in
// flight.  The stream of chunks runs straight through the reductions, so
// the next pass's blocks arrive while the scalars are being formed.
// lambda stays in global memory (one read-modify-write per iteration).
// ---------------------------------------------------------------------------
template <typename T>
struct StreamLayout {
    size_t r, p, rt, up, stage, stage_bytes, mbar, wpart, misc, total;
    __host__ __device__ StreamLayout(int nmax, int vs, int W, int nx, int KC) {
        using A = typename std::conditional<sizeof(T) == 4, dfloat, double>::type;
        size_t o = 0;
        auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
        const size_t v = sizeof(T) * (size_t)(nmax + 2) * vs;
        r = o; o = al(o + v);
        p = o; o = al(o + v);
        rt = o; o = al(o + v);
        up = o; o = al(o + v);
        stage_bytes = al(sizeof(T) * (size_t)(2 * KC + 1) * nx * nx);
        stage = o; o = o + 2 * stage_bytes;
        mbar = o; o = al(o + 2 * sizeof(uint64_t));
        wpart = o; o = al(o + 2 * sizeof(A) * W);
        misc = o; o = al(o + 16);
        total = o;
    }
};

template <typename T, int LPK, int RPT>
__global__ void __launch_bounds__(256, 1) pcg_stream_kernel(const PcgParams<T> P) {
    using AT = Acc<T>;
    using A = typename AT::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int W = nthreads / 32;
    const int warp = tid / 32, lane = tid % 32;
    const int kl = tid / LPK, li = tid % LPK;
    const int KC = nthreads / LPK;  // knots per chunk
    const int nx = P.nx, vs = P.vs;
    const int nx2 = nx * nx;
    StreamLayout<T> Lo(P.kpc_max, vs, W, nx, KC);
    T *vr = reinterpret_cast<T *>(smem + Lo.r);
    T *vp = reinterpret_cast<T *>(smem + Lo.p);
    T *vrt = reinterpret_cast<T *>(smem + Lo.rt);
    T *vup = reinterpret_cast<T *>(smem + Lo.up);
    unsigned char *stage0 = smem + Lo.stage;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lo.mbar);
    A *wpart = reinterpret_cast<A *>(smem + Lo.wpart);
    int *s_misc = reinterpret_cast<int *>(smem + Lo.misc);  // [0] instance, [1] wait failure

    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t ph[2] = {0u, 0u};  // next phase to wait for, per stage (tracked by every thread)

    auto reduce2 = [&](A &x, A &y) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            x = AT::add_tree(x, AT::shfl_xor(x, m));
            y = AT::add_tree(y, AT::shfl_xor(y, m));
        }
        if (lane == 0) {
            wpart[2 * warp] = x;
            wpart[2 * warp + 1] = y;
        }
        __syncthreads();
        x = lane < W ? wpart[2 * lane] : AT::zero();
        y = lane < W ? wpart[2 * lane + 1] : AT::zero();
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            x = AT::add_tree(x, AT::shfl_xor(x, m));
            y = AT::add_tree(y, AT::shfl_xor(y, m));
        }
    };

    int served = 0;
    bool failed = false;
    for (;;) {
        if (tid == 0) {
            int t = P.queue ? atomicAdd(P.queue, 1) : (int)(blockIdx.x + served * gridDim.x);
            s_misc[0] = t >= P.n_tickets ? -1 : (P.inst_list ? P.inst_list[t] : t);
        }
        __syncthreads();
        const int b = s_misc[0];
        ++served;
        if (b < 0 || failed) break;
        int k0, Nb;
        P.bv.range(b, k0, Nb);
        const int c0 = k0 - b;
        const bool bad = (P.info && P.info[b] != 0u) || Nb < 1 || Nb > P.kpc_max;
        const int max_iter = P.max_iter > 0 ? P.max_iter : 10 * Nb * nx;
        const int nch = ceil_div(Nb, KC);
        int iters = 0, status = MPCG_CONVERGED;
        A eta = AT::zero(), bb = AT::zero();
        T rr_t = T(0);

        // ---- the chunk stream: chunk q = pass q / nch, chunk q % nch; even
        // passes read S+, odd passes Phi^-1 -------------------------------
        auto issue = [&](int q) {  // thread 0 only
            const int pass = q / nch, kb = (q % nch) * KC;
            const T *Md = (pass & 1) ? P.Pd : P.Sd;
            const T *Mo = (pass & 1) ? P.Po : P.So;
            const int st = q & 1;
            const uint32_t mb = smem_u32(&mbar[st]);
            T *sD = reinterpret_cast<T *>(stage0 + st * Lo.stage_bytes);
            T *sO = sD + (size_t)KC * nx2;
            const int nd = min(KC, Nb - kb);
            const int jlo = max(kb - 1, 0), jhi = min(kb + KC - 1, Nb - 2);
            const uint32_t bd = (uint32_t)(nd * nx2 * sizeof(T));
            const uint32_t bo = jhi >= jlo ? (uint32_t)((jhi - jlo + 1) * nx2 * sizeof(T)) : 0u;
            mbar_arrive_expect(mb, bd + bo);
            bulk_g2s(smem_u32(sD), Md + (size_t)(k0 + kb) * nx2, bd, mb);
            if (bo) bulk_g2s(smem_u32(sO + (size_t)(jlo - (kb - 1)) * nx2), Mo + (size_t)(c0 + jlo) * nx2, bo, mb);
        };
        int q = 0;  // next chunk to consume
        int issued = 0;
        auto wait_chunk = [&]() {
            const int st = q & 1;
            int fail = 0;
            if (tid == 0) fail = !mbar_wait_bounded(smem_u32(&mbar[st]), ph[st], WAIT_LIMIT_NS);
            ph[st] ^= 1u;
            if (__syncthreads_or(fail)) failed = true;
        };
        auto release_chunk = [&]() {
            __syncthreads();  // everyone is done reading stage q & 1
            if (tid == 0) issue(issued);
            ++issued;
            ++q;
        };
        // one pass: y = M v for every knot (M = S+ or Phi^-1 by the pass
        // parity); returns the thread's partial v . y (extended) and v . v
        auto pass_apply = [&](const T *v, T *out, A &dot, T &sq) {
            for (int c = 0; c < nch; ++c) {
                wait_chunk();
                if (failed) return;
                const int st = (q & 1);
                const T *sD = reinterpret_cast<const T *>(stage0 + st * Lo.stage_bytes);
                const T *sO = sD + (size_t)KC * nx2;
                const int k = c * KC + kl;
                if (kl < KC && k < Nb) {
                    const T *D = sD + (size_t)kl * nx2;
                    const T *Lb = k >= 1 ? sO + (size_t)kl * nx2 : nullptr;
                    const T *U = k + 1 < Nb ? sO + (size_t)(kl + 1) * nx2 : nullptr;
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int i = li + m * LPK;
                        if (i < nx) {
                            const T y = rowdot_ptr<T>(nx, i, D, Lb, U, v + k * vs, v + (k + 1) * vs, v + (k + 2) * vs);
                            out[(k + 1) * vs + i] = y;
                            const T vi = v[(k + 1) * vs + i];
                            dot = AT::add(dot, AT::prod(vi, y));
                            sq = fma_rn(vi, vi, sq);
                        }
                    }
                }
                release_chunk();
            }
        };
        // residual pass: r = b - S lambda0 with extended sums (lambda0 in up)
        auto pass_resid = [&](A &sbb) {
            for (int c = 0; c < nch; ++c) {
                wait_chunk();
                if (failed) return;
                const int st = (q & 1);
                const T *sD = reinterpret_cast<const T *>(stage0 + st * Lo.stage_bytes);
                const T *sO = sD + (size_t)KC * nx2;
                const int k = c * KC + kl;
                if (kl < KC && k < Nb) {
                    const T *D = sD + (size_t)kl * nx2;
                    const T *Lb = k >= 1 ? sO + (size_t)kl * nx2 : nullptr;
                    const T *U = k + 1 < Nb ? sO + (size_t)(kl + 1) * nx2 : nullptr;
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int i = li + m * LPK;
                        if (i < nx) {
                            const T bi = P.rhs_sign * P.rhs[(size_t)(k0 + k) * nx + i];
                            vr[(k + 1) * vs + i] = resid_ptr<T>(nx, i, bi, D, Lb, U, vup + k * vs,
                                                                vup + (k + 1) * vs, vup + (k + 2) * vs);
                            sbb = AT::add(sbb, AT::prod(bi, bi));
                        }
                    }
                }
                release_chunk();
            }
        };

        if (bad) {
            status = MPCG_BADINPUT;
        } else {
            const int nv = (Nb + 2) * vs;
            for (int e = tid; e < nv; e += nthreads) {
                vr[e] = T(0); vp[e] = T(0); vrt[e] = T(0); vup[e] = T(0);
            }
            __syncthreads();
            for (int e = tid; e < Nb * nx; e += nthreads) {
                const int k = e / nx, i = e % nx;
                vup[(k + 1) * vs + i] = P.lam[(size_t)(k0 + k) * nx + i];
            }
            // prime the stream with the first two chunks
            if (tid == 0) {
                issue(0);
                issue(1);
            }
            issued = 2;
            __syncthreads();
            A sbb = AT::zero(), dummy = AT::zero();
            pass_resid(sbb);
            reduce2(sbb, dummy);
            bb = sbb;
            __syncthreads();
            A s_eta = AT::zero();
            T sq = T(0);
            if (!failed) pass_apply(vr, vrt, s_eta, sq);
            A s_rr = AT::prod(sq, T(1));
            reduce2(s_eta, s_rr);
            eta = s_eta;
            rr_t = AT::to_T(s_rr);
            __syncthreads();
            for (int e = tid; e < nv; e += nthreads) vp[e] = vrt[e];
            __syncthreads();

            const double tol = P.tol > 0 ? P.tol : 1e-6;
            const T tol_eta = (T)tol;
            const T tol_rr = (T)(tol * tol * AT::to_double(bb));
            auto converged = [&](T rr_, T eta_) -> bool {
                if (P.tol_mode == 1) return eta_ < tol_eta;
                return rr_ <= tol_rr;
            };
            T eta_t = AT::to_T(eta);
            if (failed) {
                status = MPCG_TIMEOUT;
            } else if (!(isfinite(eta_t) && isfinite(rr_t))) {
                status = MPCG_NONFINITE;
            } else if (!converged(rr_t, eta_t)) {
                status = MPCG_NOT_CONVERGED;
                for (int it = 1; it <= max_iter; ++it) {
                    A s1 = AT::zero(), s1b = AT::zero();
                    T sq1 = T(0);
                    pass_apply(vp, vup, s1, sq1);  // S p and p^T S p
                    reduce2(s1, s1b);
                    iters = it;
                    if (failed) { status = MPCG_TIMEOUT; break; }
                    const T ups = AT::to_T(s1);
                    if (!(ups > T(0)) || !isfinite(ups)) {
                        status = MPCG_BREAKDOWN;
                        break;
                    }
                    const T alpha = AT::div(eta_t, ups);
                    for (int e = tid; e < Nb * nx; e += nthreads) {
                        const int k = e / nx, i = e % nx;
                        const int o = (k + 1) * vs + i;
                        T *lp = &P.lam[(size_t)(k0 + k) * nx + i];
                        *lp = fma_rn(alpha, vp[o], *lp);
                        vr[o] = fma_rn(-alpha, vup[o], vr[o]);
                    }
                    __syncthreads();
                    A s2 = AT::zero();
                    T sq2 = T(0);
                    pass_apply(vr, vrt, s2, sq2);  // r~ = Phi^-1 r, r^T r~, ||r||^2
                    A s2b = AT::prod(sq2, T(1));
                    reduce2(s2, s2b);
                    if (failed) { status = MPCG_TIMEOUT; break; }
                    const T etan = AT::to_T(s2);
                    rr_t = AT::to_T(s2b);
                    eta = s2;
                    if (!isfinite(etan) || !isfinite(rr_t)) {
                        status = MPCG_NONFINITE;
                        break;
                    }
                    if (converged(rr_t, etan)) {
                        status = MPCG_CONVERGED;
                        break;
                    }
                    const T beta = AT::div(etan, eta_t);
                    eta_t = etan;
                    for (int e = tid; e < Nb * nx; e += nthreads) {
                        const int k = e / nx, i = e % nx;
                        const int o = (k + 1) * vs + i;
                        vp[o] = fma_rn(beta, vp[o], vrt[o]);
                    }
                    __syncthreads();
                }
            }
            // drain the copies still in flight (chunks q and q+1) before the
            // stages are reused or the CTA leaves
            for (int d = 0; d < 2 && !failed; ++d) {
                wait_chunk();
                ++q;
            }
            __syncthreads();
        }
        if (tid == 0 && P.stats) {
            mpcg_stats st;
            st.iters = iters;
            st.status = status;
            st.eta = AT::to_double(eta);
            const double bbd = AT::to_double(bb), rrd = (double)rr_t;
            st.relres = bbd > 0.0 ? sqrt(rrd / bbd) : sqrt(rrd);
            P.stats[b] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from api.cu).
// ---------------------------------------------------------------------------
template <typename T>
size_t pcg_smem_bytes(int kpc_max, int vs, int C, int W, int nx, int stage) {
    (void)C;
    return SmemLayout<T>(kpc_max, vs, W, nx, stage).total;
}

template <typename T>
static void (*pcg_fn(const PcgLaunch &L))(const PcgParams<T>) {
    if constexpr (sizeof(T) == 4) {
        if (L.mode == MODE_REG) return pcg_cluster_kernel<float, MODE_REG, 8, 2>;
    }
    if (L.lpk == 16) return pcg_cluster_kernel<T, MODE_PTR, 16, 1>;
    if (L.rpt == 1) return pcg_cluster_kernel<T, MODE_PTR, 32, 1>;
    return pcg_cluster_kernel<T, MODE_PTR, 32, 2>;
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

cudaError_t pcg_prepare(int smem_optin) {
    cudaError_t e;
    if ((e = prepare_one<float>(pcg_cluster_kernel<float, MODE_REG, 8, 2>, smem_optin))) return e;
    if ((e = prepare_one<float>(pcg_cluster_kernel<float, MODE_PTR, 16, 1>, smem_optin))) return e;
    if ((e = prepare_one<float>(pcg_cluster_kernel<float, MODE_PTR, 32, 1>, smem_optin))) return e;
    if ((e = prepare_one<float>(pcg_cluster_kernel<float, MODE_PTR, 32, 2>, smem_optin))) return e;
    if ((e = prepare_one<double>(pcg_cluster_kernel<double, MODE_PTR, 16, 1>, smem_optin))) return e;
    if ((e = prepare_one<double>(pcg_cluster_kernel<double, MODE_PTR, 32, 1>, smem_optin))) return e;
    return prepare_one<double>(pcg_cluster_kernel<double, MODE_PTR, 32, 2>, smem_optin);
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

template <typename T>
static void (*pcg_cta_fn(const PcgLaunch &L))(const PcgParams<T>) {
    if (L.lpk == 16) return pcg_cta_kernel<T, 16, 1>;
    if (L.rpt == 1) return pcg_cta_kernel<T, 32, 1>;
    return pcg_cta_kernel<T, 32, 2>;
}

template <typename T>
size_t pcg_cta_smem_bytes(int nmax, int vs, int W) {
    return CtaLayout<T>(nmax, vs, W).total;
}

template <typename T>
cudaError_t pcg_cta_launch(const PcgLaunch &L, const PcgParams<T> &P0, cudaStream_t s) {
    PcgParams<T> P = P0;
    P.kpc_max = L.kpc_max;  // largest horizon: sizes the shared vectors
    P.stage_smem = 0;
    P.vs = L.vs;
    pcg_cta_fn<T>(L)<<<L.clusters, L.threads, L.smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T>
int pcg_cta_max_blocks(const PcgLaunch &L) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pcg_cta_fn<T>(L), L.threads, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t pcg_cta_prepare(int smem_optin) {
    cudaError_t e;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(pcg_cta_kernel<float, 16, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_cta_kernel<float, 32, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_cta_kernel<float, 32, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_cta_kernel<double, 16, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_cta_kernel<double, 32, 1>, a, smem_optin))) return e;
    return cudaFuncSetAttribute(pcg_cta_kernel<double, 32, 2>, a, smem_optin);
}

template <typename T>
static void (*pcg_stream_fn(const PcgLaunch &L))(const PcgParams<T>) {
    if (L.lpk == 16) return pcg_stream_kernel<T, 16, 1>;
    if (L.rpt == 1) return pcg_stream_kernel<T, 32, 1>;
    return pcg_stream_kernel<T, 32, 2>;
}

template <typename T>
size_t pcg_stream_smem_bytes(int nmax, int vs, int W, int nx, int KC) {
    return StreamLayout<T>(nmax, vs, W, nx, KC).total;
}

template <typename T>
cudaError_t pcg_stream_launch(const PcgLaunch &L, const PcgParams<T> &P0, cudaStream_t s) {
    PcgParams<T> P = P0;
    P.kpc_max = L.kpc_max;
    P.stage_smem = 0;
    P.vs = L.vs;
    pcg_stream_fn<T>(L)<<<L.clusters, L.threads, L.smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T>
int pcg_stream_max_blocks(const PcgLaunch &L) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pcg_stream_fn<T>(L), L.threads, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t pcg_stream_prepare(int smem_optin) {
    cudaError_t e;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(pcg_stream_kernel<float, 16, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_stream_kernel<float, 32, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_stream_kernel<float, 32, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_stream_kernel<double, 16, 1>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_stream_kernel<double, 32, 1>, a, smem_optin))) return e;
    return cudaFuncSetAttribute(pcg_stream_kernel<double, 32, 2>, a, smem_optin);
}

template size_t pcg_stream_smem_bytes<float>(int, int, int, int, int);
template size_t pcg_stream_smem_bytes<double>(int, int, int, int, int);
template cudaError_t pcg_stream_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_stream_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_stream_max_blocks<float>(const PcgLaunch &);
template int pcg_stream_max_blocks<double>(const PcgLaunch &);
template size_t pcg_cta_smem_bytes<float>(int, int, int);
template size_t pcg_cta_smem_bytes<double>(int, int, int);
template cudaError_t pcg_cta_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_cta_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_cta_max_blocks<float>(const PcgLaunch &);
template int pcg_cta_max_blocks<double>(const PcgLaunch &);
template cudaError_t pcg_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_max_clusters<float>(const PcgLaunch &);
template int pcg_max_clusters<double>(const PcgLaunch &);
template size_t pcg_smem_bytes<float>(int, int, int, int, int, int);
template size_t pcg_smem_bytes<double>(int, int, int, int, int, int);

}  // namespace mpcg
