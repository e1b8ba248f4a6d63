// One-CTA-per-instance PCG kernels (batched throughput forms of Algorithm 1):
// pcg_cta_kernel reads the blocks of S+ and Phi^-1 from L2 each iteration;
// pcg_stream_kernel stages them into shared memory with TMA bulk copies.
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

}  // namespace mpcg
