// C ABI of the solve path (include/mpcg.h): argument checks, launch-shape
// selection and stream-ordered launches.  No call allocates memory.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "launch.cuh"

namespace mpcg {
// fused formation (csrc/form.cu): S+, gamma, Pd, Po in one launch
template <typename T> cudaError_t launch_form_fused(const SchurArgs<T> &, T *Pd, T *Po, int sms,
                                                    cudaStream_t);
template <typename T> size_t form_fused_smem_bytes(int nx, int nu, int Kgrid, int sms);
}  // namespace mpcg

using namespace mpcg;

struct mpcg_handle {
    int device = 0;
    int sms = 0;
    int smem_optin = 0;
    std::mutex mu;
    // launch shapes already chosen: (dtype, nx, N, B, requested cluster) -> shape
    std::map<std::tuple<int, int, int, int, int>, PcgLaunch> shapes;
};

namespace {

constexpr int kMaxThreads = 512;

// Options of refinement's correction solves: the caller's, with the exit
// test on the correction's own relative residual at refine_tol (if set).
mpcg_opts correction_opts(const mpcg_opts *o) {
    mpcg_opts c{};
    if (o) c = *o;
    else c.tol = 1e-6;
    if (o && o->refine_tol > 0) {
        c.tol = o->refine_tol;
        c.tol_mode = 0;
    }
    return c;
}
constexpr int kMaxCluster = 16;

inline int err_cuda(cudaError_t e) {
    if (e == cudaSuccess) return MPCG_OK;
    std::fprintf(stderr, "mpcg: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
    cudaGetLastError();  // a launch error is not sticky: do not leave it for the caller's next call
    return MPCG_ECUDA;
}

inline bool dims_ok(const mpcg_dims &d) {
    return d.nx >= 1 && d.nu >= 1 && d.N >= 1 && (d.dtype == 0 || d.dtype == 1);
}

inline size_t esize(const mpcg_dims &d) { return d.dtype == 1 ? 8 : 4; }
inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

BatchView make_bv(const int *knot_off, int B, int N) {
    BatchView bv;
    bv.knot_off = knot_off;
    bv.B = B;
    bv.N1 = N;
    return bv;
}

// Launch shape of the one-CTA-per-instance PCG kernel (throughput form).
template <typename T>
int choose_pcg_cta(mpcg_handle *h, const mpcg_dims &d, int B, PcgLaunch &L) {
    const int nx = d.nx;
    if (nx <= 16) { L.lpk = 16; L.rpt = 1; }
    else if (nx <= 32) { L.lpk = 32; L.rpt = 1; }
    else if (nx <= 64) { L.lpk = 32; L.rpt = 2; }
    else return MPCG_EUNSUPPORTED;
    L.cta_mode = 1;
    L.C = 1;
    L.mode = MODE_PTR;
    L.stage = 0;
    L.threads = kMaxThreads;
    L.vs = nx <= 16 ? 16 : ceil_div(nx, 4) * 4;
    L.kpc_max = d.N;
    L.smem = pcg_cta_smem_bytes<T>(d.N, L.vs, L.threads / 32);
    if (L.smem > (size_t)h->smem_optin) return MPCG_EUNSUPPORTED;
    const int per_sm = pcg_cta_max_blocks<T>(L);
    if (per_sm < 1) return MPCG_EUNSUPPORTED;
    L.clusters = std::max(1, std::min(B, per_sm * h->sms));
    return MPCG_OK;
}

// Launch shape of the tiled CTA-per-instance kernel; MPCG_EUNSUPPORTED when
// its TMA tiles cannot be used (odd nx: a block is not a 16-byte multiple;
// a block array not 16-byte aligned; nx > 64) or nothing fits in shared
// memory.  Each knot stream's steps are bound by their own instruction
// latency more than by the copies (measured: time falls with the stream
// count, hardly with the depth), so the launch takes as many streams as fit
// (at most one per four knots of the longest horizon, at most 16 warps) and
// then the deepest pipeline (up to 2 steps ahead) that still fits.
template <typename T>
int choose_pcg_tile(mpcg_handle *h, const mpcg_dims &d, int B, const mpcg_schur *s, PcgLaunch &L) {
    const int nx = d.nx;
    if (nx > 64 || nx % 2 != 0) return MPCG_EUNSUPPORTED;
    if ((sizeof(T) * (size_t)nx * nx) % 16 != 0) return MPCG_EUNSUPPORTED;
    for (const void *ptr : {s->Sd, s->So, s->Pd, s->Po})
        if (ptr && ((uintptr_t)ptr % 16) != 0) return MPCG_EUNSUPPORTED;
    L.cta_mode = 2;
    L.C = 1;
    L.mode = MODE_PTR;
    L.stage = 0;
    L.lpk = nx <= 16 ? 16 : 32;
    L.rpt = nx <= 32 ? 1 : 2;
    L.vw = (sizeof(T) == 4 && nx % 4 == 0) ? 4 : 2;
    L.nxc = (sizeof(T) == 4 && (nx == 14 || nx == 36)) ? nx : 0;
    // vector slots padded only to the load width (nx = 14: 14, not 16;
    // measured 3 % faster on 64-knot batches)
    L.vs = ceil_div(nx, L.vw) * L.vw;
    L.kpc_max = d.N;
    const int SW = 32 / L.lpk;
    const int ns_want = std::max(1, std::min(32, ceil_div(d.N, 4)));
    const int wmax = L.nxc == 36 ? 8 : 16;  // the nx = 36 form is compiled for <= 256 threads
    // the most streams (then the deepest ring) that fit, with diagonal slots
    // of npk entries (0: full tiles)
    auto fit = [&](int npk_, int &W_, int &D_) {
        W_ = D_ = 0;
        for (int W = std::min(wmax, ceil_div(ns_want, SW)); W >= 1 && !W_; --W)
            for (int dep = 2; dep >= 1; --dep)
                if (pcg_tile_smem_bytes<T>(d.N, L.vs, W, W * SW, nx, dep, npk_) <= (size_t)h->smem_optin) {
                    W_ = W;
                    D_ = dep;
                    break;
                }
    };
    int bestW = 0, bestD = 0;
    fit(0, bestW, bestD);
    // Packed diagonal blocks (nx = 36, when the caller formed them) cut the
    // bytes per step by a quarter but add a scalar load per entry: taken
    // only when their smaller slots fit more knot streams (long horizons,
    // where the kernel is bound by bytes in flight; measured 1.16-1.21x at
    // N = 160-256, 5 % slower at N = 64 where the streams are capped anyway).
    L.pk = 0;
    int npk = 0;
    if (L.nxc == 36 && s->Sdp && s->Pdp && (((uintptr_t)s->Sdp | (uintptr_t)s->Pdp) % 16) == 0) {
        int pW = 0, pD = 0;
        fit(packed_len(nx), pW, pD);
        if (pW > bestW) {
            L.pk = 1;
            npk = packed_len(nx);
            bestW = pW;
            bestD = pD;
        }
    }
    if (!bestW) return MPCG_EUNSUPPORTED;
    L.depth = bestD;
    L.smem = pcg_tile_smem_bytes<T>(d.N, L.vs, bestW, bestW * SW, nx, bestD, npk);
    L.threads = 32 * bestW;
    const int per_sm = pcg_tile_max_blocks<T>(L);
    if (per_sm < 1) return MPCG_EUNSUPPORTED;
    L.clusters = std::max(1, std::min(B, per_sm * h->sms));
    return MPCG_OK;
}

// Launch shape of the cluster PCG kernel for horizons up to Nmax.  `wide`
// (opts.mode = 4, nx <= 16): operators staged in shared memory, 8 lanes x 2
// rows per knot, up to 64 knots per CTA -- half the SMs per instance of the
// register-resident form, for throughput.
template <typename T>
int choose_pcg_cluster(mpcg_handle *h, const mpcg_dims &d, int B, const mpcg_opts *o, PcgLaunch &L,
                       bool wide = false) {
    L.cta_mode = 0;
    L.dot = (std::is_same<T, float>::value && o && o->dot == 1) ? 1 : 0;
    const int nx = d.nx;
    if (wide && nx > 16) return MPCG_EUNSUPPORTED;
    const bool reg = !wide && std::is_same<T, float>::value && nx == 14;
    int max_threads = kMaxThreads;
    if (reg) { L.lpk = 8; L.rpt = 2; max_threads = 256; }  // 2 register-resident rows per thread
    else if (wide) { L.lpk = 8; L.rpt = 2; }
    else if (nx <= 16) { L.lpk = 16; L.rpt = 1; }
    else if (nx <= 32) { L.lpk = 32; L.rpt = 1; }
    else if (nx <= 64) { L.lpk = 32; L.rpt = 2; }
    else return MPCG_EUNSUPPORTED;
    const int kpc_cap = max_threads / L.lpk;  // knot slots per CTA
    // A single instance runs fastest spread over more CTAs than it fills:
    // register form (float32, nx = 14) at about 8 knots per CTA (fewer warps
    // per CTA barrier and reduction tree; measured on GB300, N = 64 / 128:
    // 402 / 697 us against 447 / 765 us with full 32-knot CTAs), the shared-
    // memory form at the largest cluster (each lane's rows per iteration grow
    // with the knots per CTA: FP64 N = 128 4.9 ms at 16 CTAs against 13.0 ms
    // at 4; nx = 36 N = 64 2.0 against 4.3 ms).  Batches fill the CTAs (the
    // autotuner tries the other packings).
    const int kpc_pref = B > 1 ? kpc_cap : (reg ? std::min(kpc_cap, 8) : 1);
    int C = (o && o->cluster > 0) ? o->cluster : std::min(kMaxCluster, ceil_div(d.N, kpc_pref));
    if (!(o && o->cluster > 0)) C = std::max(C, ceil_div(d.N, kpc_cap));
    if (C > kMaxCluster) return MPCG_EUNSUPPORTED;
    C = std::max(1, std::min(C, d.N));
    for (;;) {
        L.C = C;
        L.kpc_max = ceil_div(d.N, C);
        if (L.kpc_max > kpc_cap) return MPCG_EUNSUPPORTED;
        L.threads = std::max(32, ceil_div(L.kpc_max * L.lpk, 32) * 32);
        L.mode = reg ? MODE_REG : MODE_PTR;
        L.vs = nx <= 16 ? 16 : ceil_div(nx, 4) * 4;
        const int W = L.threads / 32;
        L.stage = 0;
        if (L.mode == MODE_PTR) {
            size_t with = pcg_smem_bytes<T>(L.kpc_max, L.vs, C, W, nx, 1, L.dot);
            if (with <= (size_t)h->smem_optin) L.stage = 1;
        }
        L.smem = pcg_smem_bytes<T>(L.kpc_max, L.vs, C, W, nx, L.stage, L.dot);
        const int active = pcg_max_clusters<T>(L);
        if (active >= 1) {
            L.clusters = std::max(1, std::min(B, active));
            return MPCG_OK;
        }
        // this cluster size cannot be co-scheduled: try a smaller one
        if (o && o->cluster > 0) return MPCG_EUNSUPPORTED;
        if (C <= 1 || ceil_div(d.N, C / 2) > kpc_cap) return MPCG_EUNSUPPORTED;
        C = C / 2;
    }
}

// Kernel choice (mode 0): a cluster per instance whenever the horizon fits
// one (fastest for single solves; for float32 nx = 14 batches the
// register-resident clusters match the tiled kernel), the tiled kernel for
// larger batches of other shapes, one CTA per instance reading L2 for
// horizons beyond both.
template <typename T>
int choose_pcg(mpcg_handle *h, const mpcg_dims &d, int B, const mpcg_opts *o, const mpcg_schur *s,
               PcgLaunch &L) {
    const int mode = o ? o->mode : 0;
    // float64 accumulation of float32 dot products exists in the cluster
    // kernel and in the tiled kernel's compile-time shapes (nx = 14, 36);
    // the L2 CTA kernel has none
    const int dot = (std::is_same<T, float>::value && o && o->dot == 1) ? 1 : 0;
    auto tile = [&](PcgLaunch &Lt) -> int {
        const int r = choose_pcg_tile<T>(h, d, B, s, Lt);
        if (r != MPCG_OK || !dot) return r;
        if (Lt.nxc == 0) return MPCG_EUNSUPPORTED;
        Lt.dot = 1;
        return MPCG_OK;
    };
    if (mode == 2) return dot ? MPCG_EUNSUPPORTED : choose_pcg_cta<T>(h, d, B, L);
    if (mode == 3) {
        if (tile(L) == MPCG_OK) return MPCG_OK;
        return dot ? MPCG_EUNSUPPORTED : choose_pcg_cta<T>(h, d, B, L);
    }
    if (mode == 1) return choose_pcg_cluster<T>(h, d, B, o, L);
    if (mode == 4) return choose_pcg_cluster<T>(h, d, B, o, L, true);
    int rc = choose_pcg_cluster<T>(h, d, B, o, L);
    // A batch that needs more than one wave of clusters, with operators the
    // cluster kernel cannot keep in registers (anything but float32 nx = 14),
    // goes to the tiled kernel: measured 1.25 s vs 3.16 s per solve of the
    // 1024-instance nx = 36 batch.
    const bool reg = std::is_same<T, float>::value && d.nx == 14;
    if (!reg && !(o && o->cluster > 0) && (rc != MPCG_OK || (long)B * L.C > h->sms)) {
        PcgLaunch Lt{};
        if (tile(Lt) == MPCG_OK) {
            L = Lt;
            return MPCG_OK;
        }
    }
    if (rc == MPCG_EUNSUPPORTED && !(o && o->cluster > 0) && !dot) return choose_pcg_cta<T>(h, d, B, L);
    return rc;
}

template <typename T>
int form_schur_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
                 mpcg_schur *s, cudaStream_t st) {
    (void)h;  // formation needs no handle state (the signature matches the other calls)
    SchurArgs<T> a;
    a.nx = d.nx;
    a.nu = d.nu;
    a.bv = make_bv(knot_off, B, d.N);
    a.Kgrid = knot_off ? B * d.N : d.N;
    a.A = (const T *)lq->A; a.B = (const T *)lq->B; a.Qd = (const T *)lq->Qd;
    a.Rd = (const T *)lq->Rd; a.q = (const T *)lq->q; a.r = (const T *)lq->r;
    a.c = (const T *)lq->c;
    a.Qf = (const T *)lq->Q;
    a.Rf = (const T *)lq->R;
    a.Sd = (T *)s->Sd; a.So = (T *)s->So; a.gamma = (T *)s->gamma;
    a.info = s->info;
    if (s->info) {
        int e = err_cuda(cudaMemsetAsync(s->info, 0, sizeof(unsigned) * B, st));
        if (e) return e;
    }
    return err_cuda(launch_form_schur<T>(a, st));
}

// The launch shape of a PCG call (chosen once per shape key, then cached).
template <typename T>
int pcg_shape_t(mpcg_handle *h, const mpcg_dims &d, int B, const mpcg_opts *o, const mpcg_schur *s,
                PcgLaunch &L) {
    if (o && (o->refine < 0 || o->dot < 0 || o->dot > 1)) return MPCG_EINVAL;
    std::lock_guard<std::mutex> g(h->mu);
    // the tiled kernel's eligibility depends on pointer alignment
    const int aligned = (((uintptr_t)s->Sd | (uintptr_t)s->So | (uintptr_t)s->Pd | (uintptr_t)s->Po) % 16) == 0;
    // packed diagonal blocks change the tiled kernel's shared-memory layout
    const int packed = (s->Sdp && s->Pdp && (((uintptr_t)s->Sdp | (uintptr_t)s->Pdp) % 16) == 0) ? 1 : 0;
    const int tickets = (o && o->instances && o->n_instances > 0) ? o->n_instances : B;
    auto key = std::make_tuple(d.dtype, d.nx, d.N, tickets,
                               (o ? o->cluster : 0) | ((o ? o->mode : 0) << 8) | (aligned << 16) |
                                   ((o ? o->dot : 0) << 17) | (packed << 18));
    auto it = h->shapes.find(key);
    if (it != h->shapes.end()) {
        L = it->second;
        return MPCG_OK;
    }
    const int rc = choose_pcg<T>(h, d, tickets, o, s, L);
    if (rc == MPCG_OK) h->shapes.emplace(key, L);
    return rc;
}

template <typename T>
int pcg_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_schur *s,
          const T *rhs, T sign, T *lam, const mpcg_opts *o, mpcg_stats *stats, void *ws,
          cudaStream_t st) {
    PcgLaunch L{};
    int rc = pcg_shape_t<T>(h, d, B, o, s, L);
    if (rc) return rc;
    PcgParams<T> P;
    P.nx = d.nx;
    P.bv = make_bv(knot_off, B, d.N);
    P.Sd = (const T *)s->Sd; P.So = (const T *)s->So;
    P.Pd = (const T *)s->Pd; P.Po = (const T *)s->Po;
    P.rhs = rhs;
    P.rhs_sign = sign;
    P.lam = lam;
    P.info = s->info;
    P.stats = stats;
    P.queue = nullptr;
    P.tol = o ? o->tol : 1e-6;
    P.tol_mode = o ? o->tol_mode : 0;
    P.max_iter = o ? o->max_iter : 0;
    P.precon = o ? o->precon : 0;
    if (P.precon < 0 || P.precon > 2) return MPCG_EINVAL;
    P.inst_list = (o && o->instances && o->n_instances > 0) ? o->instances : nullptr;
    P.n_tickets = P.inst_list ? o->n_instances : B;
    P.Sdp = (L.cta_mode == 2 && L.pk) ? (const T *)s->Sdp : nullptr;
    P.Pdp = (L.cta_mode == 2 && L.pk) ? (const T *)s->Pdp : nullptr;
    P.npk = packed_len(d.nx);
    if (P.inst_list && !knot_off) return MPCG_EINVAL;
    if (P.n_tickets > 1 && L.clusters < P.n_tickets) {
        if (!ws) return MPCG_EINVAL;
        P.queue = (int *)ws;
        rc = err_cuda(cudaMemsetAsync(ws, 0, sizeof(int), st));
        if (rc) return rc;
    }
    if (L.cta_mode == 2) return err_cuda(pcg_tile_launch<T>(L, P, st));
    if (L.cta_mode == 1) return err_cuda(pcg_cta_launch<T>(L, P, st));
    return err_cuda(pcg_launch<T>(L, P, st));
}

template <typename T>
int backward_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
               const mpcg_schur *s, const T *lam, const T *dx, const T *du, const T *lam_bar,
               const T *dx_bar, const T *du_bar, const mpcg_grads *g, const mpcg_opts *o,
               mpcg_stats *stats, void *ws, cudaStream_t st) {
    BatchView bv = make_bv(knot_off, B, d.N);
    const int Kgrid = knot_off ? B * d.N : d.N;
    const size_t vec = al256((size_t)Kgrid * d.nx * sizeof(T));
    char *w = (char *)ws;
    T *lbar = (T *)(w + 256);
    T *mu = (T *)(w + 256 + vec);
    const T *A = (const T *)lq->A, *Bm = (const T *)lq->B, *Qd = (const T *)lq->Qd,
            *Rd = (const T *)lq->Rd;
    int rc = err_cuda(launch_cgh<T>(d.nx, d.nu, bv, Kgrid, A, Bm, Qd, Rd, dx_bar, du_bar, lam_bar,
                                    lbar, st));
    if (rc) return rc;
    rc = err_cuda(cudaMemsetAsync(mu, 0, (size_t)Kgrid * d.nx * sizeof(T), st));
    if (rc) return rc;
    rc = pcg_t<T>(h, d, B, knot_off, s, lbar, T(1), mu, o, stats, ws, st);
    if (rc) return rc;
    // Refinement of the adjoint solve: res = lambda_bar' - S+ mu formed from
    // the inputs (resid_kernel with g = 0 and the seed as -c), a correction
    // solve S+ delta = res from delta = 0, mu += delta.  g->c and g->q (both
    // [K][nx]) hold res and delta until their gradients overwrite them.
    const int nref = o ? o->refine : 0;
    for (int i = 0; i < nref; ++i) {
        T *res = (T *)g->c, *delta = (T *)g->q;
        rc = err_cuda(launch_resid<T>(d.nx, d.nu, bv, Kgrid, A, Bm, Qd, Rd, nullptr, nullptr, lbar,
                                      T(-1), mu, res, st));
        if (rc) return rc;
        // delta is the caller's [K][nx] array: zero the batch's own K knots
        // (a memset of the launch's Kgrid = B * N knots would overrun it)
        rc = err_cuda(launch_zero<T>(d.nx, bv, Kgrid, delta, st));
        if (rc) return rc;
        const mpcg_opts oc = correction_opts(o);
        rc = pcg_t<T>(h, d, B, knot_off, s, res, T(1), delta, &oc, nullptr, ws, st);
        if (rc) return rc;
        rc = err_cuda(launch_axpy<T>(d.nx, bv, Kgrid, delta, mu, st));
        if (rc) return rc;
    }
    rc = err_cuda(launch_recover<T>(d.nx, d.nu, bv, Kgrid, A, Bm, Qd, Rd, dx_bar, du_bar, mu,
                                    (T *)g->q, (T *)g->r, st));
    if (rc) return rc;
    return err_cuda(launch_grad<T>(d.nx, d.nu, bv, Kgrid, lam, mu, dx, du, (const T *)g->q,
                                   (const T *)g->r, (T *)g->A, (T *)g->B, (T *)g->Qd, (T *)g->Rd,
                                   (T *)g->c, st));
}

// Formation of S+, gamma and Phi^-1 in one launch (diagonal costs); dense
// cost blocks take the two-call route.
template <typename T>
int form_all_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
               mpcg_schur *s, cudaStream_t st);

// The packed diagonal blocks, when the caller provides them (after Sd and Pd
// are final).
template <typename T>
int pack_t(const mpcg_dims &d, int B, const int *knot_off, mpcg_schur *s, cudaStream_t st) {
    if (!s->Sdp || !s->Pdp) return MPCG_OK;
    if ((((uintptr_t)s->Sdp | (uintptr_t)s->Pdp) % 16) != 0) return MPCG_EINVAL;
    const BatchView bv = make_bv(knot_off, B, d.N);
    const int Kgrid = knot_off ? B * d.N : d.N, npk = packed_len(d.nx);
    int rc = err_cuda(launch_pack_diag<T>(d.nx, npk, bv, Kgrid, (const T *)s->Sd, (T *)s->Sdp, st));
    if (rc) return rc;
    return err_cuda(launch_pack_diag<T>(d.nx, npk, bv, Kgrid, (const T *)s->Pd, (T *)s->Pdp, st));
}

template <typename T>
int precon_t(const mpcg_dims &d, int B, const int *knot_off, mpcg_schur *s, cudaStream_t st) {
    const int rc = err_cuda(launch_form_precon<T>(d.nx, make_bv(knot_off, B, d.N), knot_off ? B * d.N : d.N,
                                                  (const T *)s->Sd, (const T *)s->So, (T *)s->Pd,
                                                  (T *)s->Po, st));
    return rc ? rc : pack_t<T>(d, B, knot_off, s, st);
}

template <typename T>
int form_all_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
               mpcg_schur *s, cudaStream_t st) {
    // Dense costs, and nx > 16 (one CTA per knot, where repeating D_{k+1}'s
    // formation and inversion in every CTA costs more than the two launches
    // it saves): the two separate launches.
    const int Kgrid = knot_off ? B * d.N : d.N;
    if (lq->Q || d.nx > 16 || form_fused_smem_bytes<T>(d.nx, d.nu, Kgrid, h->sms) > (size_t)h->smem_optin) {
        int rc = form_schur_t<T>(h, d, B, knot_off, lq, s, st);
        return rc ? rc : precon_t<T>(d, B, knot_off, s, st);
    }
    SchurArgs<T> a;
    a.nx = d.nx;
    a.nu = d.nu;
    a.bv = make_bv(knot_off, B, d.N);
    a.Kgrid = Kgrid;
    a.A = (const T *)lq->A; a.B = (const T *)lq->B; a.Qd = (const T *)lq->Qd;
    a.Rd = (const T *)lq->Rd; a.q = (const T *)lq->q; a.r = (const T *)lq->r;
    a.c = (const T *)lq->c;
    a.Qf = nullptr;
    a.Rf = nullptr;
    a.Sd = (T *)s->Sd; a.So = (T *)s->So; a.gamma = (T *)s->gamma;
    a.info = s->info;
    if (s->info) {
        int e = err_cuda(cudaMemsetAsync(s->info, 0, sizeof(unsigned) * B, st));
        if (e) return e;
    }
    const int rc = err_cuda(launch_form_fused<T>(a, (T *)s->Pd, (T *)s->Po, h->sms, st));
    return rc ? rc : pack_t<T>(d, B, knot_off, s, st);
}

template <typename T>
int solve_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off,
                   const mpcg_schur *s, void *lam, const mpcg_opts *o, mpcg_stats *stats, void *ws,
                   cudaStream_t st) {
    return pcg_t<T>(h, d, B, knot_off, s, (const T *)s->gamma, T(-1), (T *)lam, o, stats, ws, st);
}

template <typename T>
int recover_t(const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
                     const void *lam, void *dx, void *du, cudaStream_t st) {
    if (lq->Q)
        return err_cuda(launch_recover_dense<T>(d.nx, d.nu, make_bv(knot_off, B, d.N),
                                                knot_off ? B * d.N : d.N, (const T *)lq->A,
                                                (const T *)lq->B, (const T *)lq->Q,
                                                (const T *)lq->R, (const T *)lq->q,
                                                (const T *)lq->r, (const T *)lam, (T *)dx,
                                                (T *)du, st));
    return err_cuda(launch_recover<T>(d.nx, d.nu, make_bv(knot_off, B, d.N),
                                      knot_off ? B * d.N : d.N, (const T *)lq->A,
                                      (const T *)lq->B, (const T *)lq->Qd, (const T *)lq->Rd,
                                      (const T *)lq->q, (const T *)lq->r, (const T *)lam, (T *)dx,
                                      (T *)du, st));
}

template <typename T>
int refine_t(mpcg_handle *h, const mpcg_dims &d, int B, const int *knot_off, const mpcg_lq *lq,
             const mpcg_schur *s, T *lam, const mpcg_opts *o, mpcg_stats *stats, void *ws,
             cudaStream_t st) {
    BatchView bv = make_bv(knot_off, B, d.N);
    const int Kgrid = knot_off ? B * d.N : d.N;
    const size_t vec = al256((size_t)Kgrid * d.nx * sizeof(T));
    char *w = (char *)ws;
    T *res = (T *)(w + 256);
    T *delta = (T *)(w + 256 + vec);
    int rc = err_cuda(launch_resid<T>(d.nx, d.nu, bv, Kgrid, (const T *)lq->A, (const T *)lq->B,
                                      (const T *)lq->Qd, (const T *)lq->Rd, (const T *)lq->q,
                                      (const T *)lq->r, (const T *)lq->c, T(1), lam, res, st));
    if (rc) return rc;
    rc = err_cuda(cudaMemsetAsync(delta, 0, (size_t)Kgrid * d.nx * sizeof(T), st));
    if (rc) return rc;
    const mpcg_opts oc = correction_opts(o);
    rc = pcg_t<T>(h, d, B, knot_off, s, res, T(1), delta, &oc, stats, ws, st);
    if (rc) return rc;
    return err_cuda(launch_axpy<T>(d.nx, bv, Kgrid, delta, lam, st));
}

// Per-control arrays (A, B, Rd, r) are empty, and may be NULL, when every
// horizon is 1 (dims.N == 1).
bool lq_ok(const mpcg_lq *lq, const mpcg_dims &d) {
    if (!lq || !lq->q || !lq->c) return false;
    if (lq->Q) return d.N == 1 || (lq->A && lq->B && lq->R && lq->r);
    if (!lq->Qd) return false;
    return d.N == 1 || (lq->A && lq->B && lq->Rd && lq->r);
}

// below: resolves the no-allocation scratch on the handle's device
int noalloc_setup(mpcg_handle *h);

}  // namespace

extern "C" {

const char *mpcg_version(void) { return "0.1.0"; }

const char *mpcg_strerror(int code) {
    switch (code) {
        case MPCG_OK: return "ok (converged)";
        case MPCG_EINVAL: return "invalid argument";
        case MPCG_ECUDA: return "CUDA runtime or launch error";
        case MPCG_EUNSUPPORTED: return "shape not supported by the kernels";
        case MPCG_ETOOLARGE: return "problem needs more scratch than the no-allocation entry point holds";
        case MPCG_NOT_CONVERGED: return "not converged within max_iter";
        case MPCG_BREAKDOWN: return "breakdown: p^T S p <= 0 or not finite";
        case MPCG_NONFINITE: return "residual not finite";
        case MPCG_BADINPUT: return "bad input: a cost block not positive definite (or Qd, Rd not positive and finite)";
        case MPCG_TIMEOUT: return "bounded device wait gave up";
        default: return "unknown code";
    }
}

int mpcg_create(mpcg_handle **out) {
    if (!out) return MPCG_EINVAL;
    *out = nullptr;
    mpcg_handle *h = new mpcg_handle();
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MPCG_ECUDA;
    }
    if (pcg_prepare(h->smem_optin) != cudaSuccess || pcg_cta_prepare(h->smem_optin) != cudaSuccess ||
        pcg_tile_prepare(h->smem_optin) != cudaSuccess ||
        form_prepare(h->smem_optin) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MPCG_ECUDA;
    }
    // the no-allocation backward's scratch array is committed here, not on
    // that entry point's first call (under lazy module loading the array's
    // module loads, and its memory is reserved, when its address is first
    // looked up)
    if (int rc = noalloc_setup(h)) {
        delete h;
        return rc;
    }
    *out = h;
    return MPCG_OK;
}

void mpcg_destroy(mpcg_handle *h) { delete h; }

size_t mpcg_workspace_bytes(mpcg_dims d, int B) {
    if (!dims_ok(d) || B < 1) return 0;
    const size_t vec = al256((size_t)B * d.N * d.nx * esize(d));
    return 256 + 2 * vec;
}

#define DISPATCH(d, F, ...) ((d).dtype == 1 ? F<double>(__VA_ARGS__) : F<float>(__VA_ARGS__))

int mpcg_form_schur_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                            const mpcg_lq *lq, mpcg_schur *s, void *stream) {
    MPCG_NVTX("mpcg_form_schur_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !s || !s->Sd ||
        (!s->So && d.N > 1) || !s->gamma)
        return MPCG_EINVAL;
    return DISPATCH(d, form_schur_t, h, d, B, knot_off, lq, s, (cudaStream_t)stream);
}

int mpcg_form_schur(mpcg_handle *h, mpcg_dims d, const mpcg_lq *lq, mpcg_schur *s, void *stream) {
    return mpcg_form_schur_batched(h, d, 1, nullptr, lq, s, stream);
}

int mpcg_form_schur_precon_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                                   const mpcg_lq *lq, mpcg_schur *s, void *stream) {
    MPCG_NVTX("mpcg_form_schur_precon_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !s || !s->Sd ||
        !s->Pd || !s->gamma || (d.N > 1 && (!s->So || !s->Po)))
        return MPCG_EINVAL;
    return DISPATCH(d, form_all_t, h, d, B, knot_off, lq, s, (cudaStream_t)stream);
}

int mpcg_form_schur_precon(mpcg_handle *h, mpcg_dims d, const mpcg_lq *lq, mpcg_schur *s,
                           void *stream) {
    return mpcg_form_schur_precon_batched(h, d, 1, nullptr, lq, s, stream);
}

int mpcg_form_precon_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off, mpcg_schur *s,
                             void *stream) {
    MPCG_NVTX("mpcg_form_precon_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !s || !s->Sd || !s->Pd ||
        (d.N > 1 && (!s->So || !s->Po)))
        return MPCG_EINVAL;
    return DISPATCH(d, precon_t, d, B, knot_off, s, (cudaStream_t)stream);
}

int mpcg_form_precon(mpcg_handle *h, mpcg_dims d, mpcg_schur *s, void *stream) {
    return mpcg_form_precon_batched(h, d, 1, nullptr, s, stream);
}

int mpcg_pcg_solve_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                           const mpcg_schur *s, void *lambda, const mpcg_opts *opts,
                           mpcg_stats *stats, void *workspace, void *stream) {
    MPCG_NVTX("mpcg_pcg_solve_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !s || !s->Sd || !s->Pd ||
        (d.N > 1 && (!s->So || !s->Po)) || !s->gamma || !lambda)
        return MPCG_EINVAL;
    return DISPATCH(d, solve_t, h, d, B, knot_off, s, lambda, opts, stats, workspace,
                    (cudaStream_t)stream);
}

int mpcg_pcg_shape(mpcg_handle *h, mpcg_dims d, int B, const mpcg_schur *s, const mpcg_opts *opts,
                   int *shape) {
    if (!h || !dims_ok(d) || B < 1 || !s || !shape) return MPCG_EINVAL;
    PcgLaunch L{};
    const int rc = DISPATCH(d, pcg_shape_t, h, d, B, opts, s, L);
    if (rc) return rc;
    shape[0] = L.cta_mode;
    shape[1] = L.C;
    shape[2] = L.clusters;
    shape[3] = L.threads;
    shape[4] = L.cta_mode == 2 ? L.depth : 0;
    shape[5] = L.cta_mode == 2 ? L.pk : 0;
    return MPCG_OK;
}

int mpcg_pcg_solve(mpcg_handle *h, mpcg_dims d, const mpcg_schur *s, void *lambda,
                   const mpcg_opts *opts, mpcg_stats *stats, void *stream) {
    return mpcg_pcg_solve_batched(h, d, 1, nullptr, s, lambda, opts, stats, nullptr, stream);
}

int mpcg_recover_step_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                              const mpcg_lq *lq, const void *lambda, void *dx, void *du,
                              void *stream) {
    MPCG_NVTX("mpcg_recover_step_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !lambda || !dx ||
        (!du && d.N > 1))
        return MPCG_EINVAL;
    return DISPATCH(d, recover_t, d, B, knot_off, lq, lambda, dx, du, (cudaStream_t)stream);
}

int mpcg_recover_step(mpcg_handle *h, mpcg_dims d, const mpcg_lq *lq, const void *lambda, void *dx,
                      void *du, void *stream) {
    return mpcg_recover_step_batched(h, d, 1, nullptr, lq, lambda, dx, du, stream);
}

int mpcg_refine_step_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                             const mpcg_lq *lq, const mpcg_schur *s, void *lambda,
                             const mpcg_opts *opts, mpcg_stats *stats, void *workspace,
                             void *stream) {
    MPCG_NVTX("mpcg_refine_step_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !s || !s->Sd ||
        !s->Pd || (d.N > 1 && (!s->So || !s->Po)) || !lambda || !workspace)
        return MPCG_EINVAL;
    if (lq->Q) return MPCG_EUNSUPPORTED;  // the exact residual is stated for diagonal costs
    if (d.dtype == 1)
        return refine_t<double>(h, d, B, knot_off, lq, s, (double *)lambda, opts, stats, workspace,
                                (cudaStream_t)stream);
    return refine_t<float>(h, d, B, knot_off, lq, s, (float *)lambda, opts, stats, workspace,
                           (cudaStream_t)stream);
}

int mpcg_refine_step(mpcg_handle *h, mpcg_dims d, const mpcg_lq *lq, const mpcg_schur *s,
                     void *lambda, const mpcg_opts *opts, mpcg_stats *stats, void *workspace,
                     void *stream) {
    return mpcg_refine_step_batched(h, d, 1, nullptr, lq, s, lambda, opts, stats, workspace, stream);
}

int mpcg_backward_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                          const mpcg_lq *lq, const mpcg_schur *s, const void *lambda,
                          const void *dx, const void *du, const void *lam_bar, const void *dx_bar,
                          const void *du_bar, const mpcg_grads *g, const mpcg_opts *opts,
                          mpcg_stats *stats, void *workspace, void *stream) {
    MPCG_NVTX("mpcg_backward_batched");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !s || !lambda || !dx ||
        !lam_bar || !dx_bar || !g || !g->A || !g->B || !g->Qd || !g->Rd || !g->q || !g->r ||
        !g->c || !workspace || (d.N > 1 && (!du || !du_bar)) || (opts && opts->refine < 0))
        return MPCG_EINVAL;
    if (lq->Q) return MPCG_EUNSUPPORTED;  // gradients are stated for diagonal costs
    if (d.dtype == 1)
        return backward_t<double>(h, d, B, knot_off, lq, s, (const double *)lambda,
                                  (const double *)dx, (const double *)du, (const double *)lam_bar,
                                  (const double *)dx_bar, (const double *)du_bar, g, opts, stats,
                                  workspace, (cudaStream_t)stream);
    return backward_t<float>(h, d, B, knot_off, lq, s, (const float *)lambda, (const float *)dx,
                             (const float *)du, (const float *)lam_bar, (const float *)dx_bar,
                             (const float *)du_bar, g, opts, stats, workspace,
                             (cudaStream_t)stream);
}

int mpcg_backward(mpcg_handle *h, mpcg_dims d, const mpcg_lq *lq, const mpcg_schur *s,
                  const void *lambda, const void *dx, const void *du, const void *lam_bar,
                  const void *dx_bar, const void *du_bar, const mpcg_grads *g,
                  const mpcg_opts *opts, mpcg_stats *stats, void *workspace, void *stream) {
    return mpcg_backward_batched(h, d, 1, nullptr, lq, s, lambda, dx, du, lam_bar, dx_bar, du_bar,
                                 g, opts, stats, workspace, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward pass without a workspace, for callers that cannot allocate device
// memory when they differentiate (see mpcg_backward_batched_noalloc in
// include/mpcg.h).  Its scratch is this one file-scope array.  Host code
// cannot use the array's name as a device address, so mpcg_create looks the
// address up once per device with cudaGetSymbolAddress while that device is
// current (which also loads the array's module and reserves its memory).
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[MPCG_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch(mpcg_handle *h, void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPCG_ECUDA;
    }
    if (dev != h->device) return MPCG_EINVAL;  // the handle belongs to another device
    if (dev < 0 || dev >= kMaxDevices) return MPCG_EUNSUPPORTED;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return err_cuda(e);
        if (!p) return MPCG_ECUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return MPCG_OK;
}

int noalloc_setup(mpcg_handle *h) {
    void *p = nullptr;
    return noalloc_scratch(h, &p);
}
}  // namespace

extern "C" int mpcg_backward_batched_noalloc(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                                             const mpcg_lq *lq, const mpcg_schur *s,
                                             const void *lambda, const void *dx, const void *du,
                                             const void *lam_bar, const void *dx_bar,
                                             const void *du_bar, const mpcg_grads *g,
                                             const mpcg_opts *opts, mpcg_stats *stats,
                                             void *stream) {
    MPCG_NVTX("mpcg_backward_batched_noalloc");
    if (!h || !dims_ok(d) || B < 1 || (B > 1 && !knot_off) || !lq_ok(lq, d) || !s || !lambda || !dx ||
        !lam_bar || !dx_bar || !g || !g->A || !g->B || !g->Qd || !g->Rd || !g->q || !g->r ||
        !g->c || (d.N > 1 && (!du || !du_bar)) || (opts && opts->refine < 0))
        return MPCG_EINVAL;
    if (lq->Q) return MPCG_EUNSUPPORTED;  // gradients are stated for diagonal costs
    const size_t need = mpcg_workspace_bytes(d, B);
    if (need == 0) return MPCG_EINVAL;
    if (need > MPCG_NOALLOC_SCRATCH_BYTES) {
        std::fprintf(stderr,
                     "mpcg_backward_batched_noalloc: needs %zu bytes of scratch, holds %zu; "
                     "use mpcg_backward_batched with a workspace\n",
                     need, (size_t)MPCG_NOALLOC_SCRATCH_BYTES);
        return MPCG_ETOOLARGE;
    }
    void *ws = nullptr;
    int rc = noalloc_scratch(h, &ws);
    if (rc) return rc;
    if (d.dtype == 1)
        return backward_t<double>(h, d, B, knot_off, lq, s, (const double *)lambda,
                                  (const double *)dx, (const double *)du, (const double *)lam_bar,
                                  (const double *)dx_bar, (const double *)du_bar, g, opts, stats,
                                  ws, (cudaStream_t)stream);
    return backward_t<float>(h, d, B, knot_off, lq, s, (const float *)lambda, (const float *)dx,
                             (const float *)du, (const float *)lam_bar, (const float *)dx_bar,
                             (const float *)du_bar, g, opts, stats, ws, (cudaStream_t)stream);
}
