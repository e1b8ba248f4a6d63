// One-CTA-per-instance PCG kernels (batched throughput forms of Algorithm 1):
// pcg_cta_kernel reads the blocks of S+ and Phi^-1 from L2 each iteration;
// pcg_tile_kernel streams them through shared memory with TMA bulk copies,
// one pipeline per knot stream.
#include <type_traits>

#include "pcg_rows.cuh"

namespace mpcg {

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
    extern __shared__ __align__(128) unsigned char smem[];
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
        const bool bad = Nb < 1 || (P.info && P.info[b] != 0u) || Nb > P.kpc_max;
        const int max_iter = P.max_iter > 0 ? P.max_iter : 10 * Nb * nx;
        int iters = 0, status = MPCG_CONVERGED;
        A eta = AT::zero(), bb = AT::zero();
        T rr_t = T(0);

        // rows of knot k (instance-local), PTR-style block pointers
        auto blocks = [&](int k, bool precon, const T *&D, const T *&Lo, const T *&U) {
            const T *Md = precon ? P.Pd : P.Sd;
            const T *Mo = precon ? P.Po : P.So;
            // Phi^-1 rows without off-diagonal blocks: all (block Jacobi,
            // precon 1) or the even knots' (stair, precon 2)
            const bool off = !(precon && (P.precon == 1 || (P.precon == 2 && (k & 1) == 0)));
            D = Md + (size_t)(k0 + k) * nx2;
            Lo = (off && k >= 1) ? Mo + (size_t)(c0 + k - 1) * nx2 : nullptr;
            U = (off && k + 1 < Nb) ? Mo + (size_t)(c0 + k) * nx2 : nullptr;
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
        if (tid == 0 && P.stats && b < P.bv.B) {
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
// Tiled CTA-per-instance PCG (batched throughput form, opts.mode = 3).
// One CTA owns an instance: r, p and a work vector w (S p, then Phi^-1 r)
// live in shared memory for every knot, lambda in global memory.  The
// CTA's lanes form knot streams of LPK lanes (two streams per warp when
// LPK = 16); stream s owns a contiguous range of knots and walks it once per
// pass (a pass is one product with S+ or with Phi^-1).  A step of a stream
// consumes the tiles of one knot k: the diagonal block D_k and the
// off-diagonal block O_k = block (k+1, k), which serves as the upper block of
// row k (read by columns) and, in the same step, as the lower block of row
// k+1 (read by rows; the products, which need only v_k, are carried in
// registers to the next step), so each block crosses HBM once per pass and
// leaves its ring slot after one step.  The tiles
// arrive by TMA bulk copies that complete on the stream's own mbarriers;
// the copies for step g+1 are issued when step g starts, across pass
// boundaries, so a stream's memory traffic keeps flowing while the CTA forms
// the scalars.  Only the first knot of a range reads its lower block from
// global memory directly (once per pass).  The diagonal blocks are exactly
// symmetric, so reading row i of D_k gives the same products, in the same
// order, as reading its column i -- and at nx = 36 the launch may stream
// only their upper triangles (packed by columns, read in place) when the
// smaller slots fit more knot streams.
// ---------------------------------------------------------------------------
// Per knot stream and pipeline depth d: a ring of d+1 diagonal-block slots
// (full or packed blocks), d+1 off-diagonal tiles and d+1 mbarriers.

template <typename T>
struct TileLayout {
    size_t r, p, w, tiles, tile_bytes, dtile_bytes, stream_bytes, mbar, wpart, misc, total;
    // npk > 0: the diagonal slots hold packed blocks of npk entries
    __host__ __device__ TileLayout(int nmax, int vs, int W, int NS, int nx, int depth, int npk) {
        using A = typename std::conditional<sizeof(T) == 4, dfloat, double>::type;
        auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
        size_t o = 0;
        const size_t v = sizeof(T) * (size_t)(nmax + 2) * vs;
        r = o; o = al(o + v);
        p = o; o = al(o + v);
        w = o; o = al(o + v);
        tile_bytes = (sizeof(T) * (size_t)nx * nx + 15) & ~size_t(15);
        dtile_bytes = npk > 0 ? (sizeof(T) * (size_t)npk + 15) & ~size_t(15) : tile_bytes;
        stream_bytes = (size_t)(depth + 1) * (dtile_bytes + tile_bytes);
        // Two 16-lane streams share a warp when nx <= 16; their rings are
        // padded to 64 bytes past a multiple of 128, so the two half-warps'
        // column reads of their upper blocks (14 consecutive words each,
        // same slot offset) fall on disjoint banks.
        if (nx <= 16) stream_bytes += (64 + 128 - stream_bytes % 128) % 128;
        tiles = o; o = al(o + (size_t)NS * stream_bytes);
        mbar = o; o = al(o + (size_t)NS * (depth + 1) * sizeof(uint64_t));
        wpart = o; o = al(o + 2 * sizeof(A) * W);
        misc = o; o = al(o + 16);
        total = o;
    }
};

template <typename T, int VW> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<double, 2> { using type = double2; };

// VW consecutive elements from 16- (or 8-) byte aligned shared memory
template <typename T, int VW>
__device__ __forceinline__ void vload(const T *p, T (&o)[VW]) {
    const typename VecT<T, VW>::type v = *reinterpret_cast<const typename VecT<T, VW>::type *>(p);
    if constexpr (VW == 4) {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        o[0] = v.x; o[1] = v.y;
    }
}

// One column group [j, j + VW) of rows li, li + LPK, ... (RPT of them; rows
// >= nx skipped) of block row k: D_k by rows times v_k and, with HU, the
// upper block O_k = block (k+1, k) by columns times v_{k+1}; with HN also
// O_k by rows times v_k -- the lower-block products of row k+1, which the
// stream's next step uses while O_k's slot is already being refilled.  Each
// block's products go to two accumulators (even and odd columns), each in
// column order.  nx % VW == 0.
// Entry (i, j) of a packed symmetric block (upper triangle by columns:
// (i, j), i <= j, at j (j + 1) / 2 + i; (j, i) is the same entry).
__host__ __device__ __forceinline__ int packed_index(int i, int j) {
    return i <= j ? j * (j + 1) / 2 + i : i * (i + 1) / 2 + j;
}

template <typename T, int VW, int RPT, int LPK, bool HU, bool HN, bool PK, int ND>
__device__ __forceinline__ void tile_cols(int nx, int j, int li, const bool (&ok)[RPT], const T *D,
                                          const T *O, const T *vself, const T *vnext, T (&a0)[RPT],
                                          T (&a2)[RPT], T (&b0)[RPT], T (&b2)[RPT], T (&c1)[RPT],
                                          T (&d1)[RPT], const int (&doff)[ND]) {
    T xs[VW], xn[VW];
    vload<T, VW>(vself + j, xs);
    if (HU) vload<T, VW>(vnext + j, xn);
#pragma unroll
    for (int m = 0; m < RPT; ++m)
        if (ok[m]) {
            const int i = li + m * LPK;
            T d[VW], l[VW];
            if constexpr (PK) {
                // row li of the packed block: consecutive words up to the
                // diagonal's column, a per-lane stride past it (offsets
                // computed once per launch)
#pragma unroll
                for (int t = 0; t < VW; ++t) d[t] = D[doff[j + t]];
            } else {
                vload<T, VW>(D + i * nx + j, d);
            }
            if (HN) vload<T, VW>(O + i * nx + j, l);
#pragma unroll
            for (int t = 0; t < VW; t += 2) {  // even columns into a / c, odd into b / d
                a0[m] = fma_rn(d[t], xs[t], a0[m]);
                if (HN) c1[m] = fma_rn(l[t], xs[t], c1[m]);
                if (HU) a2[m] = fma_rn(O[(j + t) * nx + i], xn[t], a2[m]);
                b0[m] = fma_rn(d[t + 1], xs[t + 1], b0[m]);
                if (HN) d1[m] = fma_rn(l[t + 1], xs[t + 1], d1[m]);
                if (HU) b2[m] = fma_rn(O[(j + t + 1) * nx + i], xn[t + 1], b2[m]);
            }
        }
}

// Rows li, li + LPK, ... (RPT of them; rows >= nx skipped) of block row k
// times the halo'd vector.  The lower block's products come from the
// previous step of the stream (lc: carried in cl / dl, and ts for the split
// rows), or, on a stream's first knot, from Lg (O_{k-1} straight from global
// memory, sequential columns); the diagonal and the upper block (hu) are
// swept here, and with hn the carry for row k+1 is formed from O_k (out in
// cl / dl / ts).  Sum: ((D_e + D_o) + (L_e + L_o)) + (U_e + U_o), the even
// / odd column split halving the chains (measured 1-2 % faster).  NXC > 0
// fixes nx at compile time (the column loop unrolls completely).
template <typename T, int VW, int RPT, int LPK, int NXC, bool PK, int ND>
__device__ __forceinline__ void tile_rows(int nx_rt, int li, const T *D, const T *O, bool hu, bool hn,
                                          const T *Lg, bool lc, const T *vprev, const T *vself,
                                          const T *vnext, T (&y)[RPT], T (&cl)[RPT], T (&dl)[RPT],
                                          T &ts, const int (&doff)[ND]) {
    const int nx = NXC > 0 ? NXC : nx_rt;
    // nx fixed a little above a warp (nx = 36): the 4 rows past the first 32
    // are split over the whole warp, 8 lanes per row with a strided subset
    // of the columns each and a 3-level shuffle sum, instead of a second
    // pass in which 4 of 32 lanes work.  (These rows keep their own, equally
    // valid, summation order.)
    constexpr bool SPLIT = RPT == 2 && LPK == 32 && NXC > LPK && NXC - LPK <= 4;
    T a0[RPT], a1[RPT], a2[RPT], b0[RPT], b1[RPT], b2[RPT], c1[RPT], d1[RPT];
    bool ok[RPT];
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        a0[m] = a2[m] = b0[m] = b2[m] = c1[m] = d1[m] = T(0);
        a1[m] = lc ? cl[m] : T(0);
        b1[m] = lc ? dl[m] : T(0);
        ok[m] = li + m * LPK < nx && !(SPLIT && m > 0);
    }
    auto sweep = [&](auto u_, auto n_) {
        constexpr bool HU = decltype(u_)::value, HN = decltype(n_)::value;
        if constexpr (NXC > 0) {
#pragma unroll
            for (int j = 0; j < NXC; j += VW)
                tile_cols<T, VW, RPT, LPK, HU, HN, PK, ND>(nx, j, li, ok, D, O, vself, vnext, a0, a2, b0, b2,
                                                            c1, d1, doff);
        } else {
#pragma unroll 2
            for (int j = 0; j < nx; j += VW)
                tile_cols<T, VW, RPT, LPK, HU, HN, PK, ND>(nx, j, li, ok, D, O, vself, vnext, a0, a2, b0, b2,
                                                            c1, d1, doff);
        }
    };
    using Y = std::true_type;
    using N = std::false_type;
    if (hu && hn) sweep(Y{}, Y{});
    else if (hu) sweep(Y{}, N{});
    else if (hn) sweep(N{}, Y{});
    else sweep(N{}, N{});
    if (Lg) {  // lower block of a stream's first knot, straight from global memory
#pragma unroll
        for (int m = 0; m < RPT; ++m)
            if (ok[m])
                for (int j = 0; j < nx; ++j)
                    a1[m] = fma_rn(__ldg(Lg + (li + m * LPK) * nx + j), vprev[j], a1[m]);
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        y[m] = ((a0[m] + b0[m]) + (a1[m] + b1[m])) + (a2[m] + b2[m]);
        cl[m] = c1[m];
        dl[m] = d1[m];
    }
    if constexpr (SPLIT) {
        const int row = LPK + (li >> 3), g = li & 7;
        const bool live = row < NXC;
        T t0 = T(0), t1 = lc ? ts : T(0), t2 = T(0), tn = T(0);
#pragma unroll
        for (int q = 0; q < (NXC + 7) / 8; ++q) {
            const int j = g + 8 * q;
            if (live && j < NXC) {
                t0 = fma_rn(PK ? D[packed_index(row, j)] : D[row * NXC + j], vself[j], t0);
                if (Lg) t1 = fma_rn(Lg[row * NXC + j], vprev[j], t1);
                if (hu) t2 = fma_rn(O[j * NXC + row], vnext[j], t2);
                if (hn) tn = fma_rn(O[row * NXC + j], vself[j], tn);
            }
        }
        ts = tn;
        T t = (t0 + t1) + t2;
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        y[1] = __shfl_sync(0xffffffffu, t, (li & 3) * 8);  // lanes 0..3: rows 32..35
    }
}

// b_i - (row i) . v with exact products and an extended sum (as resid_ptr)
template <typename T>
__device__ __forceinline__ T tile_resid(int nx, int i, T b, const T *D, bool packed, const T *Lg, const T *U,
                                        const T *vprev, const T *vself, const T *vnext) {
    using AT = Acc<T>;
    typename AT::type a = AT::prod(b, T(1));
    for (int j = 0; j < nx; ++j)
        a = AT::add(a, AT::prod(-(packed ? D[packed_index(i, j)] : D[i * nx + j]), vself[j]));
    if (Lg)
        for (int j = 0; j < nx; ++j) a = AT::add(a, AT::prod(-__ldg(Lg + i * nx + j), vprev[j]));
    if (U)
        for (int j = 0; j < nx; ++j) a = AT::add(a, AT::prod(-U[j * nx + i], vnext[j]));
    return AT::to_T(a);
}

// The nx = 36 form caps its CTA at 8 warps so each thread may use up to 255
// registers (its unrolled column loop keeps 2 rows x 3 accumulators plus the
// vector chunks live).
template <int NXC>
constexpr int tile_max_threads() { return NXC == 36 ? 256 : 512; }

// AT: accumulator of the dot products (Acc<T>; AccF64 for float32 with
// mpcg_opts.dot = 1, where the few FP64 operations per row and step cost
// little beside the tile products)
template <typename T, int LPK, int RPT, int VW, int NXC = 0, typename AT = Acc<T>, bool PK = false>
__global__ void __launch_bounds__(tile_max_threads<NXC>(), 1) pcg_tile_kernel(const PcgParams<T> P) {
    // PK: the diagonal blocks arrive packed (upper triangle by columns) and
    // are read in place, each lane through its row's 36 offsets
    static_assert(!PK || (NXC == 36 && LPK == 32 && RPT == 2), "packed blocks: the nx = 36 form");
    using A = typename AT::type;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SW = 32 / LPK;  // streams per warp
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int W = nthreads / 32;
    const int warp = tid / 32, lane = tid % 32;
    const int NS = W * SW;
    const int s = warp * SW + lane / LPK;  // this lane's stream
    const int li = lane % LPK;
    const bool leader = li == 0;
    const int nx = NXC > 0 ? NXC : P.nx, vs = P.vs, nx2 = nx * nx;
    // packed blocks: this lane's row li at column j is entry doff[j]
    constexpr int ND = PK ? NXC : 1;
    int doff[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) doff[j] = packed_index(li, j);
    const uint32_t nxb = (uint32_t)(nx2 * sizeof(T));
    const int depth = P.depth;       // steps copied ahead
    const int RD = depth + 1, RO = depth + 1, RM = depth + 1;  // ring sizes
    TileLayout<T> Lo(P.kpc_max, vs, W, NS, nx, depth, PK ? P.npk : 0);
    T *vr = reinterpret_cast<T *>(smem + Lo.r);
    T *vp = reinterpret_cast<T *>(smem + Lo.p);
    T *vw = reinterpret_cast<T *>(smem + Lo.w);
    unsigned char *tb = smem + Lo.tiles + (size_t)s * Lo.stream_bytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lo.mbar);
    A *wpart = reinterpret_cast<A *>(smem + Lo.wpart);
    int *s_misc = reinterpret_cast<int *>(smem + Lo.misc);
    const uint32_t mbs = smem_u32(&mbar[(size_t)s * RM]);  // this stream's barriers

    for (int e = tid; e < NS * RM; e += nthreads) mbar_init(smem_u32(&mbar[e]), 1);
    if (tid == 0) fence_mbar_init();
    __syncthreads();
    uint32_t ph = 0u;  // bit x: next phase parity of this stream's barrier x

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
        const bool bad = Nb < 1 || (P.info && P.info[b] != 0u) || Nb > P.kpc_max;
        const int max_iter = P.max_iter > 0 ? P.max_iter : 10 * Nb * nx;
        int iters = 0, status = MPCG_CONVERGED;
        A eta = AT::zero(), bb = AT::zero();
        T rr_t = T(0);

        // this stream's knots [ks0, ks0 + len); every stream runs Lmax steps
        // per pass so the two streams of a warp stay converged
        const int ks0 = bad ? 0 : (int)(((long long)s * Nb) / NS);
        const int len = bad ? 0 : (int)(((long long)(s + 1) * Nb) / NS) - ks0;
        const int Lmax = bad ? 0 : ceil_div(Nb, NS);
        // Pipeline state of this stream (identical in all its lanes).  Steps
        // are numbered across passes; ring positions advance by one per step
        // (no divisions in the loop).
        int outstanding = 0;       // steps issued but not yet consumed
        int i_t = 0, i_ps = 0;     // next step to issue: knot offset, pass
        int i_d = 0, i_o = 0, i_m = 0;  // its D slot, O slot, barrier
        int c_d = 0, c_o = 0, c_m = 0;  // next step to consume: D slot, O slot, barrier
        auto wrap = [](int x, int n) { return x + 1 == n ? 0 : x + 1; };
        auto dslot = [&](int slot) { return reinterpret_cast<T *>(tb + (size_t)slot * Lo.dtile_bytes); };
        auto oslot = [&](int slot) {
            return reinterpret_cast<T *>(tb + (size_t)RD * Lo.dtile_bytes + (size_t)slot * Lo.tile_bytes);
        };
        // the copies of the next step to issue (leader lane; len > 0): even
        // passes read S+, odd passes Phi^-1
        auto issue_next = [&]() {
            const int k = ks0 + i_t;
            const T *Md = (i_ps & 1) ? P.Pd : P.Sd;
            const T *Mo = (i_ps & 1) ? P.Po : P.So;
            const uint32_t bar = mbs + (uint32_t)(i_m * sizeof(uint64_t));
            // block Jacobi passes (odd, Phi^-1) use no off-diagonal blocks; a
            // stair pass needs O_k in row k (k odd) or in row k + 1 (k even)
            const bool hasU = k + 1 < Nb && !((i_ps & 1) && P.precon == 1);
            const uint32_t db = PK ? (uint32_t)(P.npk * sizeof(T)) : nxb;
            mbar_arrive_expect(bar, hasU ? db + nxb : db);
            if constexpr (PK) {
                const T *Mp = (i_ps & 1) ? P.Pdp : P.Sdp;
                bulk_g2s(smem_u32(dslot(i_d)), Mp + (size_t)(k0 + k) * P.npk, db, bar);
            } else {
                bulk_g2s(smem_u32(dslot(i_d)), Md + (size_t)(k0 + k) * nx2, nxb, bar);
            }
            if (hasU) bulk_g2s(smem_u32(oslot(i_o)), Mo + (size_t)(c0 + k) * nx2, nxb, bar);
        };
        auto advance_issue = [&]() {
            if (++i_t == len) {
                i_t = 0;
                ++i_ps;
            }
            i_d = wrap(i_d, RD);
            i_o = wrap(i_o, RO);
            i_m = wrap(i_m, RM);
            ++outstanding;
        };
        // wait for the next step's tiles (leader polls; warp-uniform result)
        auto wait_next = [&](bool act) -> bool {
            int f = 0;
            if (act && leader) {
                // 16-lane streams (nx <= 16, up to 16 warps): a waiting warp
                // sleeps and leaves its issue slots to the SM's other warps
                // (measured 2 % faster); 32-lane streams (at most 2 warps
                // per SMSP) spin, which wakes sooner (5 % faster at nx = 36)
                const uint32_t bar = mbs + (uint32_t)(c_m * sizeof(uint64_t)), par = (ph >> c_m) & 1u;
                f = LPK == 16 ? !mbar_wait_bounded_sleep(bar, par, WAIT_LIMIT_NS)
                              : !mbar_wait_bounded(bar, par, WAIT_LIMIT_NS);
            }
            if (act) ph ^= 1u << c_m;
            return __any_sync(0xffffffffu, f) != 0;
        };
        auto advance_use = [&]() {
            c_d = wrap(c_d, RD);
            c_o = wrap(c_o, RO);
            c_m = wrap(c_m, RM);
            --outstanding;
        };
        // one pass: kind 0 = residual out = b - S v (dot += b^2); kind 1 =
        // product out = M v with partial dots (v . out, v . v).  lam_alpha
        // != 0: each step also applies lambda += lam_alpha p to its knot's
        // rows (p is not written during a pass), with the global loads issued
        // before the step's tile wait, so their latency hides behind it.
        auto run_pass = [&](int kind, int ps, const T *v, T *out, A &dot, T &sq, T lam_alpha = T(0)) {
            const T *Mo = (ps & 1) ? P.Po : P.So;
            const bool lam_upd = lam_alpha != T(0);
            // row k uses its off-diagonal blocks (all but the block Jacobi
            // rows of a Phi^-1 pass, and the even rows of the stair's)
            auto offd = [&](int k) { return !((ps & 1) && (P.precon == 1 || (P.precon == 2 && (k & 1) == 0))); };
            T cl[RPT], dl[RPT], ts = T(0);  // lower-block products carried to the next step
#pragma unroll
            for (int m = 0; m < RPT; ++m) cl[m] = dl[m] = T(0);
            for (int t = 0; t < Lmax; ++t) {
                const bool act = t < len;
                T lv[RPT];
                T *lrow = nullptr;
                if (lam_upd && act) {
                    lrow = P.lam + (size_t)(k0 + ks0 + t) * nx;
#pragma unroll
                    for (int m = 0; m < RPT; ++m) {
                        const int i = li + m * LPK;
                        lv[m] = i < nx ? lrow[i] : T(0);
                    }
                }
                __syncwarp();
                if (act) {
                    if (leader) {
                        fence_proxy_async();  // generic reads of the slots precede the refill
                        issue_next();
                    }
                    advance_issue();
                }
                if (wait_next(act)) {
                    failed = true;
                    break;
                }
                if (act) {
                    const int k = ks0 + t;
                    const bool off = offd(k);
                    const T *D = dslot(c_d);
                    // O_k was copied when some row uses it (as in issue_next)
                    const T *O = (k + 1 < Nb && !((ps & 1) && P.precon == 1)) ? oslot(c_o) : nullptr;
                    const bool hu = off && k + 1 < Nb;
                    advance_use();
                    if (kind == 0) {
                        // the residual pass (once per solve) reads every
                        // lower block from global memory
                        const T *Lg = (off && k >= 1) ? Mo + (size_t)(c0 + k - 1) * nx2 : nullptr;
#pragma unroll
                        for (int m = 0; m < RPT; ++m) {
                            const int i = li + m * LPK;
                            if (i < nx) {
                                const T bi = P.rhs_sign * P.rhs[(size_t)(k0 + k) * nx + i];
                                out[(k + 1) * vs + i] = tile_resid<T>(nx, i, bi, D, PK, Lg, hu ? O : nullptr, v + k * vs,
                                                                      v + (k + 1) * vs, v + (k + 2) * vs);
                                dot = AT::add(dot, AT::prod(bi, bi));
                            }
                        }
                    } else {
                        // row k's lower products: carried from step t - 1, or
                        // O_{k-1} from global memory on the range's first knot
                        const bool lc = off && t >= 1;
                        const T *Lg = (off && k >= 1 && t == 0) ? Mo + (size_t)(c0 + k - 1) * nx2 : nullptr;
                        // row k+1's, for this stream's next step
                        const bool hn = t + 1 < len && k + 1 < Nb && offd(k + 1);
                        T y[RPT];
                        tile_rows<T, VW, RPT, LPK, NXC, PK, ND>(nx, li, D, O, hu, hn, Lg, lc, v + k * vs,
                                                                v + (k + 1) * vs, v + (k + 2) * vs, y, cl, dl,
                                                                ts, doff);
#pragma unroll
                        for (int m = 0; m < RPT; ++m) {
                            const int i = li + m * LPK;
                            if (i < nx) {
                                const int o = (k + 1) * vs + i;
                                out[o] = y[m];
                                const T vi = v[o];
                                dot = AT::add(dot, AT::prod(vi, y[m]));
                                sq = fma_rn(vi, vi, sq);
                                if (lam_upd) lrow[i] = fma_rn(lam_alpha, vp[o], lv[m]);
                            }
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
                vr[e] = T(0); vp[e] = T(0); vw[e] = T(0);
            }
            __syncthreads();
            for (int e = tid; e < Nb * nx; e += nthreads) {  // lambda0 into w (halo'd)
                const int k = e / nx, i = e % nx;
                vw[(k + 1) * vs + i] = P.lam[(size_t)(k0 + k) * nx + i];
            }
            // prime each stream's pipeline with its first `depth` steps
            if (len > 0)
                for (int g = 0; g < depth; ++g) {
                    if (leader) issue_next();
                    advance_issue();
                }
            __syncthreads();
            // pass 0: r = b - S lambda0 (extended), ||b||^2; pass 1: r~ = Phi^-1 r
            A sbb = AT::zero(), dummy = AT::zero();
            T sq0 = T(0);
            run_pass(0, 0, vw, vr, sbb, sq0);
            reduce2(sbb, dummy);
            bb = sbb;
            if (__syncthreads_or(failed)) failed = true;  // r complete, wpart read
            A s_eta = AT::zero();
            T sq = T(0);
            if (!failed) run_pass(1, 1, vr, vw, s_eta, sq);
            A s_rr = AT::prod(sq, T(1));
            reduce2(s_eta, s_rr);
            eta = s_eta;
            rr_t = AT::to_T(s_rr);
            if (__syncthreads_or(failed)) failed = true;
            for (int e = tid; e < nv; e += nthreads) vp[e] = vw[e];
            __syncthreads();

            const double tol = P.tol > 0 ? P.tol : 1e-6;
            const T tol_eta = (T)tol;
            const T tol_rr = (T)(tol * tol * AT::to_double(bb));
            auto converged = [&](T rr_, T eta_) -> bool {
                if (P.tol_mode == 1) return eta_ < tol_eta;
                return rr_ <= tol_rr;
            };
            T eta_t = AT::to_T(eta);
            int ps = 2;
            if (failed) {
                status = MPCG_TIMEOUT;
            } else if (!(isfinite(eta_t) && isfinite(rr_t))) {
                status = MPCG_NONFINITE;
            } else if (!converged(rr_t, eta_t)) {
                status = MPCG_NOT_CONVERGED;
                for (int it = 1; it <= max_iter; ++it) {
                    A s1 = AT::zero(), s1b = AT::zero();
                    T sq1 = T(0);
                    run_pass(1, ps++, vp, vw, s1, sq1);  // S p and p^T S p
                    reduce2(s1, s1b);
                    iters = it;
                    if (__syncthreads_or(failed)) {
                        failed = true;
                        status = MPCG_TIMEOUT;
                        break;
                    }
                    const T ups = AT::to_T(s1);
                    if (!(ups > T(0)) || !isfinite(ups)) {
                        status = MPCG_BREAKDOWN;
                        break;
                    }
                    const T alpha = AT::div(eta_t, ups);
                    // r -= alpha S p (shared memory); lambda += alpha p rides
                    // on the next pass, step by step
                    for (int e = tid; e < Nb * nx; e += nthreads) {
                        const int o = (e / nx + 1) * vs + e % nx;
                        vr[o] = fma_rn(-alpha, vw[o], vr[o]);
                    }
                    __syncthreads();
                    A s2 = AT::zero();
                    T sq2 = T(0);
                    // r~ = Phi^-1 r, r^T r~, ||r||^2; lambda += alpha p
                    run_pass(1, ps++, vr, vw, s2, sq2, alpha);
                    A s2b = AT::prod(sq2, T(1));
                    reduce2(s2, s2b);
                    if (__syncthreads_or(failed)) {
                        failed = true;
                        status = MPCG_TIMEOUT;
                        break;
                    }
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
                        vp[o] = fma_rn(beta, vp[o], vw[o]);
                    }
                    __syncthreads();
                }
            }
            // drain this stream's copies still in flight (issued, not
            // consumed) before the slots are reused or the CTA leaves; after
            // a timed-out wait both barriers may still be pending
            // (at most depth + 1; a warp-uniform trip count keeps both
            // streams of a warp together)
            for (int d = 0; d <= depth; ++d) {
                const bool act = len > 0 && outstanding > 0;
                if (wait_next(act)) failed = true;
                if (act) advance_use();
            }
            if (__syncthreads_or(failed)) failed = true;
        }
        if (tid == 0 && P.stats && b < P.bv.B) {
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
static void (*pcg_tile_fn(const PcgLaunch &L))(const PcgParams<T>) {
    if constexpr (sizeof(T) == 4) {
        // the measured shapes with nx fixed at compile time
        if (L.nxc == 36 && L.pk)
            return L.dot ? pcg_tile_kernel<T, 32, 2, 4, 36, AccF64, true>
                         : pcg_tile_kernel<T, 32, 2, 4, 36, Acc<T>, true>;
        if (L.dot) {
            if (L.nxc == 14) return pcg_tile_kernel<T, 16, 1, 2, 14, AccF64>;
            return pcg_tile_kernel<T, 32, 2, 4, 36, AccF64>;  // nxc 36 (the only other)
        }
        if (L.nxc == 14) return pcg_tile_kernel<T, 16, 1, 2, 14>;
        if (L.nxc == 36) return pcg_tile_kernel<T, 32, 2, 4, 36>;
        if (L.vw == 4) {
            if (L.lpk == 16) return pcg_tile_kernel<T, 16, 1, 4>;
            if (L.rpt == 1) return pcg_tile_kernel<T, 32, 1, 4>;
            return pcg_tile_kernel<T, 32, 2, 4>;
        }
    }
    if (L.lpk == 16) return pcg_tile_kernel<T, 16, 1, 2>;
    if (L.rpt == 1) return pcg_tile_kernel<T, 32, 1, 2>;
    return pcg_tile_kernel<T, 32, 2, 2>;
}

template <typename T>
size_t pcg_tile_smem_bytes(int nmax, int vs, int W, int NS, int nx, int depth, int npk) {
    return TileLayout<T>(nmax, vs, W, NS, nx, depth, npk).total;
}

template <typename T>
cudaError_t pcg_tile_launch(const PcgLaunch &L, const PcgParams<T> &P0, cudaStream_t s) {
    PcgParams<T> P = P0;
    P.kpc_max = L.kpc_max;  // largest horizon: sizes the shared vectors
    P.stage_smem = 0;
    P.vs = L.vs;
    P.depth = L.depth;
    pcg_tile_fn<T>(L)<<<L.clusters, L.threads, L.smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T>
int pcg_tile_max_blocks(const PcgLaunch &L) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pcg_tile_fn<T>(L), L.threads, L.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t pcg_tile_prepare(int smem_optin) {
    cudaError_t e;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 16, 1, 2, 14>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 4, 36>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 16, 1, 2, 14, AccF64>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 4, 36, AccF64>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 4, 36, Acc<float>, true>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 4, 36, AccF64, true>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 16, 1, 4>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 1, 4>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 4>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 16, 1, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 1, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<float, 32, 2, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<double, 16, 1, 2>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(pcg_tile_kernel<double, 32, 1, 2>, a, smem_optin))) return e;
    return cudaFuncSetAttribute(pcg_tile_kernel<double, 32, 2, 2>, a, smem_optin);
}

template size_t pcg_tile_smem_bytes<float>(int, int, int, int, int, int, int);
template size_t pcg_tile_smem_bytes<double>(int, int, int, int, int, int, int);
template cudaError_t pcg_tile_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_tile_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_tile_max_blocks<float>(const PcgLaunch &);
template int pcg_tile_max_blocks<double>(const PcgLaunch &);
template size_t pcg_cta_smem_bytes<float>(int, int, int);
template size_t pcg_cta_smem_bytes<double>(int, int, int);
template cudaError_t pcg_cta_launch<float>(const PcgLaunch &, const PcgParams<float> &, cudaStream_t);
template cudaError_t pcg_cta_launch<double>(const PcgLaunch &, const PcgParams<double> &, cudaStream_t);
template int pcg_cta_max_blocks<float>(const PcgLaunch &);
template int pcg_cta_max_blocks<double>(const PcgLaunch &);

}  // namespace mpcg
