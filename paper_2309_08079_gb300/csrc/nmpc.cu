// The outer loop around the solve path on the library's synthetic model
// (include/mpcg.h, mpcg_model): Step 1 of Sec. II-A (the LQ subproblem of the
// QP at the current trajectory) and Step 3 with the parallel line search of
// Sec. IV-C (every step size of a halving set evaluated at once, the
// smallest L1 merit kept and applied).  All three kernels are stream-ordered
// and allocate nothing, so a whole SQP iteration can be captured in a graph.
//
// Model: h = nx/2 joints, x = (p, v), nu actuated inputs,
//     v+ = v + dt (P u - damp * v - stiff * sin p),   p+ = p + dt v+,
// cost l(x, u) = 1/2 sum wq (x - xref)^2 + 1/2 sum wr u^2, terminal weights wf.
#include <cmath>
#include <cstdio>

#include "common.cuh"

namespace mpcg {
namespace {

constexpr int LIN_THREADS = 128;  // 4 knots per block, one warp each
constexpr int MERIT_THREADS = 64;   // one (knot, joint) pair per thread
constexpr int MAX_ALPHA = 32;

template <typename T>
struct ModelView {
    int nx, nu, h;
    double dt;  // kept exact; rounded to the working type where that type computes
    const T *P, *damp, *stiff, *wq, *wr, *wf;
};

template <typename T>
__device__ __forceinline__ T sin_t(T x) {
    if constexpr (sizeof(T) == 4) return sinf(x);
    else return sin(x);
}

template <typename T>
__device__ __forceinline__ T cos_t(T x) {
    if constexpr (sizeof(T) == 4) return cosf(x);
    else return cos(x);
}

// Velocity update of joint i: v_i + dt (P_i u - damp_i v_i - stiff_i sin p_i),
// evaluated in Acc (the merit takes it in FP64 from working-type points).
template <typename T, typename Acc>
__device__ __forceinline__ Acc vnext(const ModelView<T> &m, int i, const T *x, const T *u) {
    Acc f = Acc(0);
    for (int j = 0; j < m.nu; ++j) f += Acc(m.P[i * m.nu + j]) * Acc(u[j]);
    f += -Acc(m.damp[i]) * Acc(x[m.h + i]) - Acc(m.stiff[i]) * sin_t<Acc>(Acc(x[i]));
    return Acc(x[m.h + i]) + Acc(m.dt) * f;
}

// Row i of f(x, u) (positions then velocities).
template <typename T, typename Acc>
__device__ __forceinline__ Acc fdyn(const ModelView<T> &m, int i, const T *x, const T *u) {
    if (i >= m.h) return vnext<T, Acc>(m, i - m.h, x, u);
    return Acc(x[i]) + Acc(m.dt) * vnext<T, Acc>(m, i, x, u);
}

// ---------------------------------------------------------------------------
// linearize: one warp per knot k (instance b, control index j = kg - b):
//   Qd_k = wq (wf at the last knot), Rd_k = wr, q_k = Qd_k (x_k - xref_k),
//   r_k = wr u_k, c_0 = x_0 - x_s, c_k = x_k - f(x_{k-1}, u_{k-1}),
//   A_k = df/dx, B_k = df/du at (x_k, u_k):
//     dv/dp = -dt diag(stiff cos p), dv/dv = I - dt diag(damp), dv/du = dt P,
//     A = [[I + dt dv/dp, dt dv/dv], [dv/dp, dv/dv]], B = [[dt dv/du], [dv/du]].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS)
linearize_kernel(ModelView<T> m, BatchView bv, const T *__restrict__ X, const T *__restrict__ U,
                 const T *__restrict__ xref, const T *__restrict__ xs, T *A, T *B, T *Qd, T *Rd,
                 T *q, T *r, T *c) {
    const int lane = threadIdx.x % 32;
    const int kg = blockIdx.x * (LIN_THREADS / 32) + threadIdx.x / 32;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const int k = kg - k0;
    const bool last = k + 1 >= Nb;
    const int nx = m.nx, nu = m.nu, h = m.h;
    const T *x = X + (size_t)kg * nx;
    for (int i = lane; i < nx; i += 32) {
        const T w = last ? m.wf[i] : m.wq[i];
        Qd[(size_t)kg * nx + i] = w;
        q[(size_t)kg * nx + i] = w * (x[i] - xref[(size_t)kg * nx + i]);
        T ci;
        if (k == 0) {
            ci = x[i] - xs[(size_t)b * nx + i];
        } else {
            const int jp = kg - b - 1;  // control index of (x_{k-1}, u_{k-1})
            ci = x[i] - fdyn<T, T>(m, i, X + (size_t)(kg - 1) * nx, U + (size_t)jp * nu);
        }
        c[(size_t)kg * nx + i] = ci;
    }
    if (last) return;
    const int j = kg - b;
    const T *u = U + (size_t)j * nu;
    for (int i = lane; i < nu; i += 32) {
        Rd[(size_t)j * nu + i] = m.wr[i];
        r[(size_t)j * nu + i] = m.wr[i] * u[i];
    }
    const T dt = (T)m.dt;
    T *Aj = A + (size_t)j * nx * nx;
    for (int e = lane; e < nx * nx; e += 32) {
        const int i = e / nx, l = e % nx;
        const int ii = i % h, ll = l % h;
        const bool rowp = i < h, colp = l < h;
        // velocity-row entries of dv/dx
        T dv = T(0);
        if (ii == ll) dv = colp ? -dt * m.stiff[ii] * cos_t<T>(x[ii]) : T(1) - dt * m.damp[ii];
        T a;
        if (rowp) a = (colp && i == l ? T(1) : T(0)) + dt * dv;  // p+ = p + dt v+
        else a = dv;
        Aj[e] = a;
    }
    T *Bj = B + (size_t)j * nx * nu;
    for (int e = lane; e < nx * nu; e += 32) {
        const int i = e / nu, l = e % nu;
        const T dvdu = dt * m.P[(i % h) * nu + l];
        Bj[e] = i < h ? dt * dvdu : dvdu;
    }
}

// ---------------------------------------------------------------------------
// merit: the L1 merit of (X, U) + alpha_a (dX, dU), alpha_a = 2^-a, in FP64:
// J + mu_b (||x'_0 - x_s||_1 + sum ||x'_{k+1} - f(x'_k, u'_k)||_1).  The
// candidate point is rounded to the working type first, as the applied step
// will be.  mu_b = mu when mu > 0, else 1.1 max(1, max |lambda_b|).  Block
// (b, a, chunk) takes 64 (knot, joint) pairs of instance b, one per thread:
// thread (k, i) adds the cost of state rows i and h + i of knot k (and of
// input i, nu <= h), and the defects of those two rows, which need joint i's
// velocity update alone.  Its share goes to merit[b][a] (zeroed before the
// launch) with an FP64 atomic: the FP64 work (one sine per pair) spreads
// over h times more threads than one knot per thread would, and the
// summation order only moves the merits by rounding, far below the tie
// tolerance of the choice.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32, W = blockDim.x / 32;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < W ? red[lane] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ double block_max(double v, double *red) {
    for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32, W = blockDim.x / 32;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < W ? red[lane] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__global__ void __launch_bounds__(MERIT_THREADS)
merit_kernel(ModelView<T> m, BatchView bv, int n_alpha, const T *__restrict__ X,
             const T *__restrict__ U, const T *__restrict__ dX, const T *__restrict__ dU,
             const T *__restrict__ xref, const T *__restrict__ xs, const T *__restrict__ lam,
             double mu, double *merit) {
    __shared__ double red[MERIT_THREADS / 32];
    const int b = blockIdx.x / n_alpha, a = blockIdx.x % n_alpha;
    if (b >= bv.B) return;
    int k0, Nb;
    bv.range(b, k0, Nb);
    const int nx = m.nx, nu = m.nu, h = m.h;
    const int ebase = blockIdx.y * MERIT_THREADS;
    if (ebase >= Nb * h) return;  // whole block: this instance is shorter
    const int c0 = k0 - b;
    const T alpha = T(ldexp(1.0, -a));
    double mub = mu;
    if (!(mu > 0.0)) {
        // max |lambda_b|: eight independent loads per thread in flight
        const T *lb = lam + (size_t)k0 * nx;
        const int n = Nb * nx, step = blockDim.x;
        T mx = T(0);
        for (int e0 = threadIdx.x; e0 < n; e0 += 8 * step) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e0 + u * step < n ? lb[e0 + u * step] : T(0);
#pragma unroll
            for (int u = 0; u < 8; ++u) mx = fmax(mx, fabs(v[u]));
        }
        mub = 1.1 * fmax(1.0, block_max<T>((double)mx, red));
    }
    double J = 0.0, viol = 0.0;
    const int e = ebase + threadIdx.x;
    if (e < Nb * h) {
        const int k = e / h, i = e % h;
        const size_t o = (size_t)(k0 + k) * nx;
        const bool last = k + 1 >= Nb;
        // candidate position and velocity of joint i at knot k
        const T pk = X[o + i] + alpha * dX[o + i];
        const T vk = X[o + h + i] + alpha * dX[o + h + i];
        const T *w = last ? m.wf : m.wq;
        const double ep = (double)pk - (double)xref[o + i];
        const double ev = (double)vk - (double)xref[o + h + i];
        J += 0.5 * (double)w[i] * ep * ep;
        J += 0.5 * (double)w[h + i] * ev * ev;
        if (!last && i < nu) {
            const size_t ou = (size_t)(c0 + k) * nu + i;
            const T ui = U[ou] + alpha * dU[ou];
            J += 0.5 * (double)m.wr[i] * (double)ui * (double)ui;
        }
        if (k == 0) {
            viol += fabs((double)pk - (double)xs[(size_t)b * nx + i]);
            viol += fabs((double)vk - (double)xs[(size_t)b * nx + h + i]);
        } else {
            // joint i's velocity update from the candidate (x'_{k-1}, u'_{k-1})
            const size_t op = o - nx, ou = (size_t)(c0 + k - 1) * nu;
            const T pp = X[op + i] + alpha * dX[op + i];
            const T vp = X[op + h + i] + alpha * dX[op + h + i];
            double f = 0.0;
            for (int j = 0; j < nu; ++j) {
                const T uj = U[ou + j] + alpha * dU[ou + j];
                f += (double)m.P[i * nu + j] * (double)uj;
            }
            f += -(double)m.damp[i] * (double)vp - (double)m.stiff[i] * sin((double)pp);
            const double vn = (double)vp + m.dt * f;
            viol += fabs((double)pk - ((double)pp + m.dt * vn));
            viol += fabs((double)vk - vn);
        }
    }
    const double part = block_sum<T>(J + mub * viol, red);
    if (threadIdx.x == 0) atomicAdd(&merit[(size_t)b * n_alpha + a], part);
}

// ---------------------------------------------------------------------------
// apply: every knot's warp picks its instance's smallest merit and adds that
// step.  Merits within a relative 1e-11 of the smallest (below the rounding
// of their FP64 sums) count as ties, and the longest tied step wins; a NaN
// merit never wins.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS)
apply_kernel(int nx, int nu, BatchView bv, int n_alpha, const double *__restrict__ merit, T *X,
             T *U, const T *__restrict__ dX, const T *__restrict__ dU, int *alpha_index) {
    const int lane = threadIdx.x % 32;
    const int kg = blockIdx.x * (LIN_THREADS / 32) + threadIdx.x / 32;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    double bm = merit[(size_t)b * n_alpha];
    for (int a = 1; a < n_alpha; ++a) {
        const double v = merit[(size_t)b * n_alpha + a];
        if (v < bm || (bm != bm && v == v)) bm = v;
    }
    int best = 0;
    for (int a = 0; a < n_alpha; ++a)
        if (merit[(size_t)b * n_alpha + a] <= bm + 1e-11 * fabs(bm)) {
            best = a;
            break;
        }
    const T alpha = T(ldexp(1.0, -best));
    if (kg == k0 && lane == 0 && alpha_index) alpha_index[b] = best;
    for (int i = lane; i < nx; i += 32) X[(size_t)kg * nx + i] += alpha * dX[(size_t)kg * nx + i];
    if (kg - k0 + 1 < Nb) {
        const int j = kg - b;
        for (int i = lane; i < nu; i += 32) U[(size_t)j * nu + i] += alpha * dU[(size_t)j * nu + i];
    }
}

template <typename T>
ModelView<T> view(const mpcg_model *m) {
    ModelView<T> v;
    v.nx = m->nx;
    v.nu = m->nu;
    v.h = m->nx / 2;
    v.dt = m->dt;
    v.P = (const T *)m->P;
    v.damp = (const T *)m->damp;
    v.stiff = (const T *)m->stiff;
    v.wq = (const T *)m->wq;
    v.wr = (const T *)m->wr;
    v.wf = (const T *)m->wf;
    return v;
}

int err(cudaError_t e) {
    if (e == cudaSuccess) return MPCG_OK;
    std::fprintf(stderr, "mpcg: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
    cudaGetLastError();
    return MPCG_ECUDA;
}

bool model_ok(const mpcg_model *m, const mpcg_dims &d) {
    return m && m->nx == d.nx && m->nu == d.nu && d.nx % 2 == 0 && d.nx <= 64 && d.nu <= 32 &&
           m->nu <= m->nx / 2 && m->dt > 0.0 && m->P && m->damp && m->stiff && m->wq && m->wr &&
           m->wf && d.N >= 1 && (d.dtype == 0 || d.dtype == 1);
}

BatchView bview(const int *knot_off, int B, int N) {
    BatchView bv;
    bv.knot_off = knot_off;
    bv.B = B;
    bv.N1 = N;
    return bv;
}

template <typename T>
int linearize_t(const mpcg_dims &d, int B, const int *knot_off, const mpcg_model *m, const void *X,
                const void *U, const void *xref, const void *xs, const mpcg_lq_out *o,
                cudaStream_t st) {
    const int K = knot_off ? B * d.N : d.N;  // upper bound on the total knots
    const int per = LIN_THREADS / 32;
    linearize_kernel<T><<<(K + per - 1) / per, LIN_THREADS, 0, st>>>(
        view<T>(m), bview(knot_off, B, d.N), (const T *)X, (const T *)U, (const T *)xref,
        (const T *)xs, (T *)o->A, (T *)o->B, (T *)o->Qd, (T *)o->Rd, (T *)o->q, (T *)o->r,
        (T *)o->c);
    return err(cudaGetLastError());
}

template <typename T>
int line_search_t(const mpcg_dims &d, int B, const int *knot_off, const mpcg_model *m, void *X,
                  void *U, const void *dX, const void *dU, const void *xref, const void *xs,
                  const void *lam, double mu, int n_alpha, double *merit, int *alpha_index,
                  cudaStream_t st) {
    const BatchView bv = bview(knot_off, B, d.N);
    int rc = err(cudaMemsetAsync(merit, 0, sizeof(double) * (size_t)B * n_alpha, st));
    if (rc) return rc;
    const dim3 grid(B * n_alpha, (d.N * (d.nx / 2) + MERIT_THREADS - 1) / MERIT_THREADS);
    merit_kernel<T><<<grid, MERIT_THREADS, 0, st>>>(
        view<T>(m), bv, n_alpha, (const T *)X, (const T *)U, (const T *)dX, (const T *)dU,
        (const T *)xref, (const T *)xs, (const T *)lam, mu, merit);
    rc = err(cudaGetLastError());
    if (rc) return rc;
    const int K = knot_off ? B * d.N : d.N;
    const int per = LIN_THREADS / 32;
    apply_kernel<T><<<(K + per - 1) / per, LIN_THREADS, 0, st>>>(
        d.nx, d.nu, bv, n_alpha, merit, (T *)X, (T *)U, (const T *)dX, (const T *)dU, alpha_index);
    return err(cudaGetLastError());
}

}  // namespace
}  // namespace mpcg

using namespace mpcg;

extern "C" {

int mpcg_linearize_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                           const mpcg_model *model, const void *X, const void *U,
                           const void *xref, const void *xs, const mpcg_lq_out *out,
                           void *stream) {
    MPCG_NVTX("mpcg_linearize_batched");
    if (!h || B < 1 || (B > 1 && !knot_off) || !model_ok(model, d) || !X || !xref || !xs || !out ||
        !out->Qd || !out->q || !out->c ||
        (d.N > 1 && (!U || !out->A || !out->B || !out->Rd || !out->r)))
        return MPCG_EINVAL;
    if (d.dtype == 1)
        return linearize_t<double>(d, B, knot_off, model, X, U, xref, xs, out, (cudaStream_t)stream);
    return linearize_t<float>(d, B, knot_off, model, X, U, xref, xs, out, (cudaStream_t)stream);
}

int mpcg_linearize(mpcg_handle *h, mpcg_dims d, const mpcg_model *model, const void *X,
                   const void *U, const void *xref, const void *xs, const mpcg_lq_out *out,
                   void *stream) {
    return mpcg_linearize_batched(h, d, 1, nullptr, model, X, U, xref, xs, out, stream);
}

int mpcg_line_search_batched(mpcg_handle *h, mpcg_dims d, int B, const int *knot_off,
                             const mpcg_model *model, void *X, void *U, const void *dX,
                             const void *dU, const void *xref, const void *xs,
                             const void *lambda, double mu, int n_alpha, double *merit,
                             int *alpha_index, void *stream) {
    MPCG_NVTX("mpcg_line_search_batched");
    if (!h || B < 1 || (B > 1 && !knot_off) || !model_ok(model, d) || !X || !dX || !xref || !xs ||
        !merit || n_alpha < 1 || n_alpha > MAX_ALPHA || (d.N > 1 && (!U || !dU)) ||
        (!(mu > 0.0) && !lambda))
        return MPCG_EINVAL;
    if (d.dtype == 1)
        return line_search_t<double>(d, B, knot_off, model, X, U, dX, dU, xref, xs, lambda, mu,
                                     n_alpha, merit, alpha_index, (cudaStream_t)stream);
    return line_search_t<float>(d, B, knot_off, model, X, U, dX, dU, xref, xs, lambda, mu, n_alpha,
                                merit, alpha_index, (cudaStream_t)stream);
}

int mpcg_line_search(mpcg_handle *h, mpcg_dims d, const mpcg_model *model, void *X, void *U,
                     const void *dX, const void *dU, const void *xref, const void *xs,
                     const void *lambda, double mu, int n_alpha, double *merit, int *alpha_index,
                     void *stream) {
    return mpcg_line_search_batched(h, d, 1, nullptr, model, X, U, dX, dU, xref, xs, lambda, mu,
                                    n_alpha, merit, alpha_index, stream);
}

}  // extern "C"
