// Per-knot kernels of the solve path: Schur complement and gamma
// (Sec. II-B, Eq. trajoptSchur_1/2), the symmetric stair preconditioner
// (Sec. IV-A), primal step recovery (Eq. schur), and the element-wise parts
// of the backward pass.
//
// Every kernel assigns one group of G threads to one block row (knot) and
// stages that knot's small blocks in shared memory; G = 32 (one warp) for
// nx <= 16 and 128 otherwise.  Knots of a ragged batch are numbered
// globally; a group finds its instance by binary search over knot_off.
#include <algorithm>
#include <type_traits>

#include "launch.cuh"

namespace mpcg {

constexpr int FORM_THREADS = 128;

__host__ __device__ __forceinline__ int group_size(int nx) { return nx <= 16 ? 32 : 128; }

// Synchronise the threads of one group (a warp, or the whole CTA).
__device__ __forceinline__ void group_sync(int G) {
    if (G == 32) __syncwarp();
    else __syncthreads();
}

template <typename T>
__device__ __forceinline__ bool good_weight(T v) {
    return v > T(0) && isfinite((double)v);
}

// ---------------------------------------------------------------------------
// form_schur: block row k of S+ and gamma_k.
//   k = 0: D_0 = Qd_0^-1, gamma_0 = c_0 - Qd_0^-1 q_0
//   k > 0: D_k = theta_{k-1}, So[k-1] = phi_{k-1}, gamma_k = c_k - zeta_{k-1}
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS) form_schur_kernel(const SchurArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, nu = a.nu;
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    // per-group scratch
    const size_t per = (size_t)2 * nx * nx + 2 * nx * nu + 4 * nx + 2 * nu;
    T *S = reinterpret_cast<T *>(smem_raw) + per * g;
    T *Am = S, *As = Am + nx * nx, *Bm = As + nx * nx, *Bs = Bm + nx * nu;
    T *iq0 = Bs + nx * nu, *iq1 = iq0 + nx, *qs = iq1 + nx, *q1 = qs + nx, *ir = q1 + nx,
      *rs = ir + nu;
    if (kg >= a.bv.total()) return;  // whole group leaves together
    const int b = a.bv.owner(kg);
    int k0, Nb;
    a.bv.range(b, k0, Nb);
    const int k = kg - k0;
    bool bad = false;
    const T *Qk = a.Qd + (size_t)kg * nx;
    for (int i = t; i < nx; i += G) {
        T v = Qk[i];
        bad |= !good_weight(v);
        iq1[i] = T(1) / v;
        q1[i] = a.q[(size_t)kg * nx + i];
    }
    if (k == 0) {
        group_sync(G);
        T *Sd = a.Sd + (size_t)kg * nx * nx;
        for (int e = t; e < nx * nx; e += G) {
            int i = e / nx, j = e % nx;
            Sd[e] = i == j ? iq1[i] : T(0);
        }
        for (int i = t; i < nx; i += G)
            a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - q1[i] * iq1[i];
    } else {
        const int j = kg - b - 1;  // control index of (A, B, Rd, r, So) for this row
        const T *Ak = a.A + (size_t)j * nx * nx;
        const T *Bk = a.B + (size_t)j * nx * nu;
        for (int i = t; i < nx; i += G) {
            T v = a.Qd[(size_t)(kg - 1) * nx + i];
            bad |= !good_weight(v);
            iq0[i] = T(1) / v;
            qs[i] = a.q[(size_t)(kg - 1) * nx + i] / v;
        }
        for (int i = t; i < nu; i += G) {
            T v = a.Rd[(size_t)j * nu + i];
            bad |= !good_weight(v);
            ir[i] = T(1) / v;
            rs[i] = a.r[(size_t)j * nu + i] / v;
        }
        group_sync(G);
        for (int e = t; e < nx * nx; e += G) {
            T v = Ak[e];
            Am[e] = v;
            As[e] = v * iq0[e % nx];
        }
        for (int e = t; e < nx * nu; e += G) {
            T v = Bk[e];
            Bm[e] = v;
            Bs[e] = v * ir[e % nu];
        }
        group_sync(G);
        T *Sd = a.Sd + (size_t)kg * nx * nx;
        T *So = a.So + (size_t)j * nx * nx;
        // theta (upper triangle computed once, mirrored: exactly symmetric)
        for (int e = t; e < nx * nx; e += G) {
            const int i = e / nx, jj = e % nx;
            So[e] = -As[e];
            if (i > jj) continue;
            T s = T(0);
            for (int m = 0; m < nx; ++m) s += As[i * nx + m] * Am[jj * nx + m];
            for (int m = 0; m < nu; ++m) s += Bs[i * nu + m] * Bm[jj * nu + m];
            if (i == jj) s += iq1[i];
            Sd[i * nx + jj] = s;
            Sd[jj * nx + i] = s;
        }
        // zeta and gamma
        for (int i = t; i < nx; i += G) {
            T z = q1[i] * iq1[i];
            for (int m = 0; m < nx; ++m) z -= Am[i * nx + m] * qs[m];
            for (int m = 0; m < nu; ++m) z -= Bm[i * nu + m] * rs[m];
            a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - z;
        }
    }
    if (a.info && __any_sync(0xffffffffu, bad) && (t % 32) == 0) atomicOr(&a.info[b], MPCG_INFO_BADINPUT);
}

// ---------------------------------------------------------------------------
// form_precon, part 1: Pd[k] = Sd[k]^-1 by Gauss-Jordan elimination without
// pivoting (Sd[k] is symmetric positive definite), symmetrised on output.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
precon_inv_kernel(int nx, BatchView bv, const T *__restrict__ Sd, T *__restrict__ Pd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    T *M = reinterpret_cast<T *>(smem_raw) + (size_t)g * nx * nx;
    if (kg >= bv.total()) return;
    const T *src = Sd + (size_t)kg * nx * nx;
    for (int e = t; e < nx * nx; e += G) M[e] = src[e];
    group_sync(G);
    for (int j = 0; j < nx; ++j) {
        const T d = T(1) / M[j * nx + j];
        for (int c = t; c < nx; c += G)
            if (c != j) M[j * nx + c] *= d;
        group_sync(G);
        const int n1 = nx - 1;
        for (int e = t; e < n1 * n1; e += G) {
            int i = e / n1, c = e % n1;
            i += (i >= j);
            c += (c >= j);
            M[i * nx + c] -= M[i * nx + j] * M[j * nx + c];
        }
        group_sync(G);
        for (int i = t; i < nx; i += G) {
            if (i != j) M[i * nx + j] = -M[i * nx + j] * d;
            else M[j * nx + j] = d;
        }
        group_sync(G);
    }
    T *dst = Pd + (size_t)kg * nx * nx;
    for (int e = t; e < nx * nx; e += G) {
        int i = e / nx, c = e % nx;
        dst[e] = T(0.5) * (M[i * nx + c] + M[c * nx + i]);
    }
}

// ---------------------------------------------------------------------------
// form_precon, part 2: Po[j] = -Pd[k+1] So[j] Pd[k] for every knot k that has
// a successor in its instance (j = its control index).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
precon_off_kernel(int nx, BatchView bv, const T *__restrict__ Pd,
                  const T *__restrict__ So, T *__restrict__ Po) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    const int n2 = nx * nx;
    T *X = reinterpret_cast<T *>(smem_raw) + (size_t)g * 4 * n2;
    T *S = X + n2, *Y = S + n2, *T1 = Y + n2;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    if (kg - k0 + 1 >= Nb) return;  // last knot of its instance
    const int j = kg - b;
    for (int e = t; e < n2; e += G) {
        X[e] = Pd[(size_t)kg * n2 + e];
        Y[e] = Pd[(size_t)(kg + 1) * n2 + e];
        S[e] = So[(size_t)j * n2 + e];
    }
    group_sync(G);
    for (int e = t; e < n2; e += G) {
        int i = e / nx, c = e % nx;
        T s = T(0);
        for (int m = 0; m < nx; ++m) s += S[i * nx + m] * X[m * nx + c];
        T1[e] = s;
    }
    group_sync(G);
    for (int e = t; e < n2; e += G) {
        int i = e / nx, c = e % nx;
        T s = T(0);
        for (int m = 0; m < nx; ++m) s += Y[i * nx + m] * T1[m * nx + c];
        Po[(size_t)j * n2 + e] = -s;
    }
}

// ---------------------------------------------------------------------------
// recover: z = G^-1 (C^T v - h) for a multiplier-shaped v and h = (hx, hu):
//   zx_k = (v_k - A_k^T v_{k+1} - hx_k) / Qd_k   (last knot: no A term)
//   zu_k = (-B_k^T v_{k+1} - hu_k) / Rd_k
// With (v, h) = (lambda, g) this is dz (Eq. schur); with (mu, dL/ddz) it is
// the adjoint's g_bar.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
recover_kernel(int nx, int nu, BatchView bv, const T *__restrict__ A,
               const T *__restrict__ B, const T *__restrict__ Qd, const T *__restrict__ Rd,
               const T *__restrict__ hx, const T *__restrict__ hu, const T *__restrict__ v,
               T *__restrict__ zx, T *__restrict__ zu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    T *vn = reinterpret_cast<T *>(smem_raw) + (size_t)g * nx;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const bool last = kg - k0 + 1 >= Nb;
    const int j = kg - b;
    for (int i = t; i < nx; i += G) vn[i] = last ? T(0) : v[(size_t)(kg + 1) * nx + i];
    group_sync(G);
    // v_k - A_k^T v_{k+1} - hx_k cancels heavily when v is large against z:
    // accumulate with exact products and an extended sum, round once.
    using AT = Acc<T>;
    for (int i = t; i < nx + nu; i += G) {
        if (i < nx) {
            auto s = AT::add(AT::from(v[(size_t)kg * nx + i]), AT::from(-hx[(size_t)kg * nx + i]));
            if (!last) {
                const T *Ak = A + (size_t)j * nx * nx;
                for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Ak[m * nx + i], vn[m]));
            }
            zx[(size_t)kg * nx + i] = AT::to_T(AT::div_x(s, Qd[(size_t)kg * nx + i]));
        } else if (!last) {
            const int u = i - nx;
            const T *Bk = B + (size_t)j * nx * nu;
            auto s = AT::from(-hu[(size_t)j * nu + u]);
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Bk[m * nu + u], vn[m]));
            zu[(size_t)j * nu + u] = AT::to_T(AT::div_x(s, Rd[(size_t)j * nu + u]));
        }
    }
}

// ---------------------------------------------------------------------------
// Backward seed: out = w + C G^-1 (hx, hu), block row k:
//   k = 0: w_0 + hx_0 / Qd_0
//   k > 0: w_k - A_{k-1} (hx_{k-1}/Qd_{k-1}) - B_{k-1} (hu_{k-1}/Rd_{k-1}) + hx_k/Qd_k
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
cgh_kernel(int nx, int nu, BatchView bv, const T *__restrict__ A,
           const T *__restrict__ B, const T *__restrict__ Qd, const T *__restrict__ Rd,
           const T *__restrict__ hx, const T *__restrict__ hu, const T *__restrict__ w,
           T *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    T *xs = reinterpret_cast<T *>(smem_raw) + (size_t)g * (nx + nu);
    T *us = xs + nx;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const int k = kg - k0;
    const int j = kg - b - 1;
    if (k > 0) {
        for (int i = t; i < nx; i += G) xs[i] = hx[(size_t)(kg - 1) * nx + i] / Qd[(size_t)(kg - 1) * nx + i];
        for (int i = t; i < nu; i += G) us[i] = hu[(size_t)j * nu + i] / Rd[(size_t)j * nu + i];
    }
    group_sync(G);
    for (int i = t; i < nx; i += G) {
        T s = w[(size_t)kg * nx + i] + hx[(size_t)kg * nx + i] / Qd[(size_t)kg * nx + i];
        if (k > 0) {
            const T *Ak = A + (size_t)j * nx * nx;
            const T *Bk = B + (size_t)j * nx * nu;
            for (int m = 0; m < nx; ++m) s -= Ak[i * nx + m] * xs[m];
            for (int m = 0; m < nu; ++m) s -= Bk[i * nu + m] * us[m];
        }
        out[(size_t)kg * nx + i] = s;
    }
}

// ---------------------------------------------------------------------------
// Backward outer products (gq = g_bar_x and gr = g_bar_u already written):
//   Qd_bar = g_bar_x * dx, Rd_bar = g_bar_u * du, c_bar = -mu,
//   A_bar_k = mu_{k+1} dx_k^T + lam_{k+1} g_bar_x_k^T,
//   B_bar_k = mu_{k+1} du_k^T + lam_{k+1} g_bar_u_k^T.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
grad_kernel(int nx, int nu, BatchView bv, const T *__restrict__ lam,
            const T *__restrict__ mu, const T *__restrict__ dx, const T *__restrict__ du,
            const T *__restrict__ gq, const T *__restrict__ gr, T *__restrict__ gA,
            T *__restrict__ gB, T *__restrict__ gQd, T *__restrict__ gRd, T *__restrict__ gc) {
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const bool last = kg - k0 + 1 >= Nb;
    const int j = kg - b;
    for (int i = t; i < nx; i += G) {
        const size_t o = (size_t)kg * nx + i;
        gQd[o] = gq[o] * dx[o];
        gc[o] = -mu[o];
    }
    if (last) return;
    for (int i = t; i < nu; i += G) {
        const size_t o = (size_t)j * nu + i;
        gRd[o] = gr[o] * du[o];
    }
    const T *mun = mu + (size_t)(kg + 1) * nx, *lamn = lam + (size_t)(kg + 1) * nx;
    for (int e = t; e < nx * nx; e += G) {
        int i = e / nx, m = e % nx;
        gA[(size_t)j * nx * nx + e] = mun[i] * dx[(size_t)kg * nx + m] + lamn[i] * gq[(size_t)kg * nx + m];
    }
    for (int e = t; e < nx * nu; e += G) {
        int i = e / nu, m = e % nu;
        gB[(size_t)j * nx * nu + e] = mun[i] * du[(size_t)j * nu + m] + lamn[i] * gr[(size_t)j * nu + m];
    }
}

// ---------------------------------------------------------------------------
// Exact-operator residual for iterative refinement.  For S+ = C G^-1 C^T and
// b = -gamma = C G^-1 g - c, the residual of a multiplier estimate is
//     b - S+ lambda = -(C dz(lambda) + c),   dz(lambda) = G^-1 (C^T lambda - g),
// i.e. the defect of the linearised dynamics at the recovered step.  It is
// formed per knot in extended precision straight from the inputs, so it
// carries neither the rounding of S+ to working precision nor the drift of
// the PCG recurrences.  Block row k:
//   k = 0: -(dx_0 + c_0)
//   k > 0: A_{k-1} dx_{k-1} + B_{k-1} du_{k-1} - dx_k - c_k
// With q = r = nullptr (g = 0) and c scaled by csign = -1 the same kernel
// forms v - S+ mu = v - C G^-1 C^T mu for any right-hand side v (passed as
// c): the residual of the adjoint solve of the backward pass.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
resid_kernel(int nx, int nu, BatchView bv, const T *__restrict__ A, const T *__restrict__ B,
             const T *__restrict__ Qd, const T *__restrict__ Rd, const T *__restrict__ q,
             const T *__restrict__ r, const T *__restrict__ c, T csign, const T *__restrict__ lam,
             T *__restrict__ out) {
    using AT = Acc<T>;
    using X = typename AT::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    X *xs = reinterpret_cast<X *>(smem_raw) + (size_t)g * (2 * nx + nu);
    X *dx_cur = xs, *dx_prev = xs + nx, *du_prev = xs + 2 * nx;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const int k = kg - k0;
    const bool last = k + 1 >= Nb;
    // dz entries of this knot (dx_k) and of the previous one (dx_{k-1}, du_{k-1})
    for (int i = t; i < nx; i += G) {
        X s = AT::from(lam[(size_t)kg * nx + i]);
        if (q) s = AT::add(s, AT::from(-q[(size_t)kg * nx + i]));
        if (!last) {
            const T *Ak = A + (size_t)(kg - b) * nx * nx;
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Ak[m * nx + i], lam[(size_t)(kg + 1) * nx + m]));
        }
        dx_cur[i] = AT::div_x(s, Qd[(size_t)kg * nx + i]);
    }
    if (k > 0) {
        const int j = kg - b - 1;
        const T *Ap = A + (size_t)j * nx * nx;
        const T *Bp = B + (size_t)j * nx * nu;
        for (int i = t; i < nx; i += G) {
            X s = AT::from(lam[(size_t)(kg - 1) * nx + i]);
            if (q) s = AT::add(s, AT::from(-q[(size_t)(kg - 1) * nx + i]));
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Ap[m * nx + i], lam[(size_t)kg * nx + m]));
            dx_prev[i] = AT::div_x(s, Qd[(size_t)(kg - 1) * nx + i]);
        }
        for (int i = t; i < nu; i += G) {
            X s = AT::from(r ? -r[(size_t)j * nu + i] : T(0));
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Bp[m * nu + i], lam[(size_t)kg * nx + m]));
            du_prev[i] = AT::div_x(s, Rd[(size_t)j * nu + i]);
        }
    }
    group_sync(G);
    for (int i = t; i < nx; i += G) {
        X s = AT::add(AT::neg(dx_cur[i]), AT::from(-csign * c[(size_t)kg * nx + i]));
        if (k > 0) {
            const int j = kg - b - 1;
            const T *Ap = A + (size_t)j * nx * nx;
            const T *Bp = B + (size_t)j * nx * nu;
            for (int m = 0; m < nx; ++m) s = AT::fma_x(Ap[i * nx + m], dx_prev[m], s);
            for (int m = 0; m < nu; ++m) s = AT::fma_x(Bp[i * nu + m], du_prev[m], s);
        }
        out[(size_t)kg * nx + i] = AT::to_T(s);
    }
}

// lam[i] += d[i] over every knot of the batch
template <typename T>
__global__ void axpy_kernel(int nx, BatchView bv, const T *__restrict__ d, T *__restrict__ lam) {
    const size_t n = (size_t)bv.total() * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        lam[i] += d[i];
}

// v[i] = 0 over every knot of the batch (a caller's [K][nx] array, K = the
// batch's own knot count, which only the device knows for a ragged batch)
template <typename T>
__global__ void zero_kernel(int nx, BatchView bv, T *__restrict__ v) {
    const size_t n = (size_t)bv.total() * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[i] = T(0);
}

// ---------------------------------------------------------------------------
// Fused formation (diagonal costs): block row k of S+ and gamma_k (Sec.
// II-B, Eq. schur and Eq. trajoptSchur_1/2, as form_schur_kernel), Pd[k] =
// D_k^-1 (Sec. IV-A, as precon_inv_kernel) and, when k has a successor,
// Po[k] = -Pd[k+1] phi_k Pd[k] (Sec. IV-A, as precon_off_kernel) in one
// launch, with no round trip through memory for the intermediate blocks.
// The operations and their order are those of the three kernels; the values
// agree with theirs to rounding (compile-time loop shapes let the compiler
// contract other multiply-adds).
// ---------------------------------------------------------------------------
// NXC, NUC: compile-time nx, nu (0: taken from the arguments at run time).
template <typename T, int NXC, int NUC>
__device__ __forceinline__ void row_blocks(const SchurArgs<T> &a, int t, int kgrow, int j,
                                           T *Am, T *As, T *Bm, T *Bs, T *iq0, T *iq1, T *qs,
                                           T *ir, T *rs, T *q1, T *D, bool &bad) {
    // theta for row kgrow (> instance start): D = A Q^-1 A^T + B R^-1 B^T + Q+^-1,
    // As = A Q^-1 (so phi = -As); qs = Q^-1 q, rs = R^-1 r, q1 = q+
    constexpr int G = 32;
    const int nx = NXC ? NXC : a.nx, nu = NUC ? NUC : a.nu;
    for (int i = t; i < nx; i += G) {
        T v = a.Qd[(size_t)kgrow * nx + i];
        bad |= !good_weight(v);
        iq1[i] = T(1) / v;
        q1[i] = a.q[(size_t)kgrow * nx + i];
        v = a.Qd[(size_t)(kgrow - 1) * nx + i];
        bad |= !good_weight(v);
        iq0[i] = T(1) / v;
        qs[i] = a.q[(size_t)(kgrow - 1) * nx + i] / v;
    }
    for (int i = t; i < nu; i += G) {
        T v = a.Rd[(size_t)j * nu + i];
        bad |= !good_weight(v);
        ir[i] = T(1) / v;
        rs[i] = a.r[(size_t)j * nu + i] / v;
    }
    group_sync(G);
    const T *Ak = a.A + (size_t)j * nx * nx;
    const T *Bk = a.B + (size_t)j * nx * nu;
    for (int e = t; e < nx * nx; e += G) {
        T v = Ak[e];
        Am[e] = v;
        As[e] = v * iq0[e % nx];
    }
    for (int e = t; e < nx * nu; e += G) {
        T v = Bk[e];
        Bm[e] = v;
        Bs[e] = v * ir[e % nu];
    }
    group_sync(G);
    for (int e = t; e < nx * nx; e += G) {
        const int i = e / nx, jj = e % nx;
        if (i > jj) continue;
        T s = T(0);
        for (int m = 0; m < nx; ++m) s += As[i * nx + m] * Am[jj * nx + m];
        for (int m = 0; m < nu; ++m) s += Bs[i * nu + m] * Bm[jj * nu + m];
        if (i == jj) s += iq1[i];
        D[i * nx + jj] = s;
        D[jj * nx + i] = s;
    }
    group_sync(G);
}

// Gauss-Jordan inverse of the SPD block M in place, then M <- (M + M^T)/2 into
// out (the operations of precon_inv_kernel).
template <typename T, int NXC>
__device__ __forceinline__ void gj_inverse_sym(T *M, T *out, int nx_rt, int t) {
    constexpr int G = 32;
    const int nx = NXC ? NXC : nx_rt;
    for (int j = 0; j < nx; ++j) {
        const T d = T(1) / M[j * nx + j];
        for (int c = t; c < nx; c += G)
            if (c != j) M[j * nx + c] *= d;
        group_sync(G);
        const int n1 = nx - 1;
        for (int e = t; e < n1 * n1; e += G) {
            int i = e / n1, c = e % n1;
            i += (i >= j);
            c += (c >= j);
            M[i * nx + c] -= M[i * nx + j] * M[j * nx + c];
        }
        group_sync(G);
        for (int i = t; i < nx; i += G) {
            if (i != j) M[i * nx + j] = -M[i * nx + j] * d;
            else M[j * nx + j] = d;
        }
        group_sync(G);
    }
    for (int e = t; e < nx * nx; e += G) {
        int i = e / nx, c = e % nx;
        out[e] = T(0.5) * (M[i * nx + c] + M[c * nx + i]);
    }
    group_sync(G);
}

// The same inversion with compile-time NX <= 32, one row per lane in
// registers: pivot j's scaled row is broadcast by shuffles, every other lane
// updates its own row, then its column entry.  The element operations and
// their order are those above (scale row j, M_ic -= M_ij M_jc, M_ij = -M_ij
// d, M_jj = d); only the indexing, the shared-memory round trips and the
// warp barriers of the loops are gone.  M is read and the symmetrised
// inverse written through shared memory (both nx x nx, row-major).
template <typename T, int NX>
__device__ __forceinline__ void gj_inverse_sym_reg(T *M, T *out, int t) {
    static_assert(NX >= 1 && NX <= 32, "one row per lane");
    T row[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) row[c] = t < NX ? M[t * NX + c] : T(0);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const T d = T(1) / __shfl_sync(0xffffffffu, row[j], j);
        if (t == j) {
#pragma unroll
            for (int c = 0; c < NX; ++c)
                if (c != j) row[c] *= d;
        }
        T rj[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) rj[c] = __shfl_sync(0xffffffffu, row[c], j);
        if (t != j) {
            const T mij = row[j];
#pragma unroll
            for (int c = 0; c < NX; ++c)
                if (c != j) row[c] -= mij * rj[c];
            row[j] = -row[j] * d;
        } else {
            row[j] = d;
        }
    }
    __syncwarp();  // every lane has read M
    if (t < NX) {
#pragma unroll
        for (int c = 0; c < NX; ++c) M[t * NX + c] = row[c];
    }
    __syncwarp();
    if (t < NX) {
#pragma unroll
        for (int c = 0; c < NX; ++c) out[t * NX + c] = T(0.5) * (M[t * NX + c] + M[c * NX + t]);
    }
    __syncwarp();
}

// Warp form of the fused formation (nx <= 16: one warp per knot).  A CTA
// takes `kpb` consecutive knots plus one extra warp for the successor of its
// last knot; after a CTA barrier, warp w forms Po[k] from its own Pd[k] and
// the phi_k (= -As) and Pd[k+1] that warp w + 1 left in shared memory.  Only
// the extra warp repeats work (one knot in kpb), and each warp's dependent
// chain is one formation, one inversion and the two products -- the chain of
// the three separate kernels.  The host picks kpb
// so that the grid covers the SMs (small problems are latency-bound) and
// raises it to FUSED_KPB_MAX for large batches (less repeated work).
constexpr int FUSED_KPB_MAX = 16;

template <typename T>
__host__ __device__ inline size_t fused_warp_words(int nx, int nu) {
    return (size_t)4 * nx * nx + (size_t)2 * nx * nu + 4 * nx + 2 * nu;
}

template <typename T, int NXC, int NUC>
__global__ void __launch_bounds__(32 * (FUSED_KPB_MAX + 1))
form_fused_warp_kernel(const SchurArgs<T> a, T *Pd, T *Po, int kpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = NXC ? NXC : a.nx, nu = NUC ? NUC : a.nu, n2 = nx * nx;
    const int w = threadIdx.x / 32, t = threadIdx.x % 32;
    const size_t words = fused_warp_words<T>(nx, nu);
    T *Am = reinterpret_cast<T *>(smem_raw) + words * w;
    T *As = Am + n2, *D = As + n2, *P = D + n2, *Bm = P + n2, *Bs = Bm + nx * nu,
      *iq0 = Bs + nx * nu, *iq1 = iq0 + nx, *qs = iq1 + nx, *q1 = qs + nx, *ir = q1 + nx,
      *rs = ir + nu;
    T *T1 = D;  // D is dead once P = D^-1 is formed
    const int kg = blockIdx.x * kpb + w;
    const bool extra = w == kpb;  // formed and inverted, never written
    int b = 0, k = 0, Nb = 0;
    bool active = kg < a.bv.total();    // warp-uniform
    if (active) {
        int k0;
        b = a.bv.owner(kg);
        a.bv.range(b, k0, Nb);
        k = kg - k0;
        if (extra && k == 0) active = false;  // starts an instance: no predecessor needs it
    }
    bool bad = false;
    if (active) {
        if (k == 0) {
            for (int i = t; i < nx; i += 32) {
                T v = a.Qd[(size_t)kg * nx + i];
                bad |= !good_weight(v);
                iq1[i] = T(1) / v;
                q1[i] = a.q[(size_t)kg * nx + i];
            }
            __syncwarp();
            for (int e = t; e < n2; e += 32) {
                int i = e / nx, j = e % nx;
                D[e] = i == j ? iq1[i] : T(0);
            }
            for (int i = t; i < nx; i += 32)
                a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - q1[i] * iq1[i];
            __syncwarp();
        } else {
            const int j = kg - b - 1;
            row_blocks<T, NXC, NUC>(a, t, kg, j, Am, As, Bm, Bs, iq0, iq1, qs, ir, rs, q1, D, bad);
            if (!extra) {
                T *So = a.So + (size_t)j * n2;
                for (int e = t; e < n2; e += 32) So[e] = -As[e];
                for (int i = t; i < nx; i += 32) {
                    T z = q1[i] * iq1[i];
                    for (int m = 0; m < nx; ++m) z -= Am[i * nx + m] * qs[m];
                    for (int m = 0; m < nu; ++m) z -= Bm[i * nu + m] * rs[m];
                    a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - z;
                }
            }
            __syncwarp();
        }
        if (!extra) {
            T *Sd = a.Sd + (size_t)kg * n2;
            for (int e = t; e < n2; e += 32) Sd[e] = D[e];
        }
        __syncwarp();
        // float32: one row per lane (FP32 pipes are wide; measured 21 -> 16
        // us at N = 512).  float64 keeps the 32-lane loops: each lane's row
        // doubles the warp's FP64 instructions, and GB300's FP64 rate makes
        // that the cost (measured 43 -> 51 us).
        if constexpr (NXC > 0 && sizeof(T) == 4) gj_inverse_sym_reg<T, NXC>(D, P, t);
        else gj_inverse_sym<T, NXC>(D, P, nx, t);
        if (!extra)
            for (int e = t; e < n2; e += 32) Pd[(size_t)kg * n2 + e] = P[e];
    }
    __syncthreads();
    if (!active || extra) return;
    if (k + 1 < Nb) {
        // knot kg + 1 is warp w + 1's (the extra warp's for the last knot)
        const T *Asn = As + words, *Pn = P + words;
        const int j = kg - b;
        for (int e = t; e < n2; e += 32) {
            int i = e / nx, c = e % nx;
            T s = T(0);
            for (int m = 0; m < nx; ++m) s += (-Asn[i * nx + m]) * P[m * nx + c];
            T1[e] = s;
        }
        __syncwarp();
        for (int e = t; e < n2; e += 32) {
            int i = e / nx, c = e % nx;
            T s = T(0);
            for (int m = 0; m < nx; ++m) s += Pn[i * nx + m] * T1[m * nx + c];
            Po[(size_t)j * n2 + e] = -s;
        }
    }
    if (a.info && __any_sync(0xffffffffu, bad) && t == 0) atomicOr(&a.info[b], MPCG_INFO_BADINPUT);
}

// ---------------------------------------------------------------------------
// General SPD cost blocks (the Q_k, R_k of Sec. II-A's QP as full matrices).
// A group inverts its blocks in shared memory by Gauss-Jordan elimination
// without pivoting (positive pivots are exactly the SPD condition), then
// forms Eq. trajoptSchur_1/2 with the inverses:
//   theta_k = A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T + Q_{k+1}^-1,
//   phi_k = -A_k Q_k^-1,
//   zeta_k = -A_k Q_k^-1 q_k - B_k R_k^-1 r_k + Q_{k+1}^-1 q_{k+1}.
// ---------------------------------------------------------------------------

// In-place inverse of the n x n SPD block M (group of G threads; all of them
// call it).  Returns true (in every thread) when a pivot is not positive and
// finite, i.e. M is not SPD.  The result is symmetrised.
template <typename T>
__device__ bool gj_inverse_spd(T *M, int n, int G, int t) {
    bool bad = false;
    for (int j = 0; j < n; ++j) {
        const T piv = M[j * n + j];
        bad |= !(piv > T(0) && isfinite((double)piv));
        const T d = T(1) / piv;
        for (int c = t; c < n; c += G)
            if (c != j) M[j * n + c] *= d;
        group_sync(G);
        const int n1 = n - 1;
        for (int e = t; e < n1 * n1; e += G) {
            int i = e / n1, c = e % n1;
            i += (i >= j);
            c += (c >= j);
            M[i * n + c] -= M[i * n + j] * M[j * n + c];
        }
        group_sync(G);
        for (int i = t; i < n; i += G) {
            if (i != j) M[i * n + j] = -M[i * n + j] * d;
            else M[j * n + j] = d;
        }
        group_sync(G);
    }
    for (int e = t; e < n * n; e += G) {
        const int i = e / n, c = e % n;
        if (i < c) {
            const T v = T(0.5) * (M[i * n + c] + M[c * n + i]);
            M[i * n + c] = v;
            M[c * n + i] = v;
        }
    }
    group_sync(G);
    return bad;
}

template <typename T>
__host__ __device__ inline size_t dense_form_words(int nx, int nu) {
    return (size_t)4 * nx * nx + (size_t)nu * nu + (size_t)2 * nx * nu + 2 * nx + nu;
}

template <typename T>
__global__ void __launch_bounds__(FORM_THREADS) form_schur_dense_kernel(const SchurArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, nu = a.nu;
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    const int n2 = nx * nx;
    T *Qi0 = reinterpret_cast<T *>(smem_raw) + dense_form_words<T>(nx, nu) * g;
    T *Qi1 = Qi0 + n2, *Am = Qi1 + n2, *As = Am + n2, *Ri = As + n2, *Bm = Ri + nu * nu,
      *Bs = Bm + nx * nu, *q0 = Bs + nx * nu, *q1 = q0 + nx, *rr = q1 + nx;
    if (kg >= a.bv.total()) return;  // whole group leaves together
    const int b = a.bv.owner(kg);
    int k0, Nb;
    a.bv.range(b, k0, Nb);
    const int k = kg - k0;
    const int j = kg - b - 1;  // control index of (A, B, R, r, So) for this row (k > 0)
    for (int e = t; e < n2; e += G) Qi1[e] = a.Qf[(size_t)kg * n2 + e];
    for (int i = t; i < nx; i += G) q1[i] = a.q[(size_t)kg * nx + i];
    if (k > 0) {
        for (int e = t; e < n2; e += G) {
            Qi0[e] = a.Qf[(size_t)(kg - 1) * n2 + e];
            Am[e] = a.A[(size_t)j * n2 + e];
        }
        for (int e = t; e < nu * nu; e += G) Ri[e] = a.Rf[(size_t)j * nu * nu + e];
        for (int e = t; e < nx * nu; e += G) Bm[e] = a.B[(size_t)j * nx * nu + e];
        for (int i = t; i < nx; i += G) q0[i] = a.q[(size_t)(kg - 1) * nx + i];
        for (int i = t; i < nu; i += G) rr[i] = a.r[(size_t)j * nu + i];
    }
    group_sync(G);
    bool bad = gj_inverse_spd(Qi1, nx, G, t);
    if (k == 0) {
        T *Sd = a.Sd + (size_t)kg * n2;
        for (int e = t; e < n2; e += G) Sd[e] = Qi1[e];
        for (int i = t; i < nx; i += G) {
            T z = T(0);
            for (int m = 0; m < nx; ++m) z += Qi1[i * nx + m] * q1[m];
            a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - z;
        }
    } else {
        bad |= gj_inverse_spd(Qi0, nx, G, t);
        bad |= gj_inverse_spd(Ri, nu, G, t);
        for (int e = t; e < n2; e += G) {  // As = A Q_{k-1}^-1
            const int i = e / nx, c = e % nx;
            T s = T(0);
            for (int m = 0; m < nx; ++m) s += Am[i * nx + m] * Qi0[m * nx + c];
            As[e] = s;
        }
        for (int e = t; e < nx * nu; e += G) {  // Bs = B R^-1
            const int i = e / nu, c = e % nu;
            T s = T(0);
            for (int m = 0; m < nu; ++m) s += Bm[i * nu + m] * Ri[m * nu + c];
            Bs[e] = s;
        }
        group_sync(G);
        T *Sd = a.Sd + (size_t)kg * n2;
        T *So = a.So + (size_t)j * n2;
        // theta (upper triangle computed once, mirrored: exactly symmetric)
        for (int e = t; e < n2; e += G) {
            const int i = e / nx, jj = e % nx;
            So[e] = -As[e];
            if (i > jj) continue;
            T s = Qi1[i * nx + jj];
            for (int m = 0; m < nx; ++m) s += As[i * nx + m] * Am[jj * nx + m];
            for (int m = 0; m < nu; ++m) s += Bs[i * nu + m] * Bm[jj * nu + m];
            Sd[i * nx + jj] = s;
            Sd[jj * nx + i] = s;
        }
        for (int i = t; i < nx; i += G) {
            T z = T(0);
            for (int m = 0; m < nx; ++m) z += Qi1[i * nx + m] * q1[m] - As[i * nx + m] * q0[m];
            for (int m = 0; m < nu; ++m) z -= Bs[i * nu + m] * rr[m];
            a.gamma[(size_t)kg * nx + i] = a.c[(size_t)kg * nx + i] - z;
        }
    }
    if (a.info && bad && t == 0) atomicOr(&a.info[b], MPCG_INFO_BADINPUT);
}

// recover with dense cost blocks: zx_k = Q_k^-1 (v_k - A_k^T v_{k+1} - hx_k),
// zu_k = R_k^-1 (-B_k^T v_{k+1} - hu_k); the right-hand sides are summed with
// exact products in extended precision (they cancel when v is large against
// z), the products with the inverses likewise, each rounded once.
template <typename T>
__global__ void __launch_bounds__(FORM_THREADS)
recover_dense_kernel(int nx, int nu, BatchView bv, const T *__restrict__ A,
                     const T *__restrict__ B, const T *__restrict__ Qf, const T *__restrict__ Rf,
                     const T *__restrict__ hx, const T *__restrict__ hu, const T *__restrict__ v,
                     T *__restrict__ zx, T *__restrict__ zu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = group_size(nx);
    const int groups = FORM_THREADS / G;
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int kg = blockIdx.x * groups + g;
    const int n2 = nx * nx;
    T *Qi = reinterpret_cast<T *>(smem_raw) + ((size_t)n2 + nu * nu + 2 * nx + nu) * g;
    T *Ri = Qi + n2, *vn = Ri + nu * nu, *sx = vn + nx, *su = sx + nx;
    if (kg >= bv.total()) return;
    const int b = bv.owner(kg);
    int k0, Nb;
    bv.range(b, k0, Nb);
    const bool last = kg - k0 + 1 >= Nb;
    const int j = kg - b;
    for (int e = t; e < n2; e += G) Qi[e] = Qf[(size_t)kg * n2 + e];
    if (!last)
        for (int e = t; e < nu * nu; e += G) Ri[e] = Rf[(size_t)j * nu * nu + e];
    for (int i = t; i < nx; i += G) vn[i] = last ? T(0) : v[(size_t)(kg + 1) * nx + i];
    group_sync(G);
    gj_inverse_spd(Qi, nx, G, t);
    if (!last) gj_inverse_spd(Ri, nu, G, t);
    using AT = Acc<T>;
    for (int i = t; i < nx + nu; i += G) {
        if (i < nx) {
            auto s = AT::add(AT::from(v[(size_t)kg * nx + i]), AT::from(-hx[(size_t)kg * nx + i]));
            if (!last) {
                const T *Ak = A + (size_t)j * n2;
                for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Ak[m * nx + i], vn[m]));
            }
            sx[i] = AT::to_T(s);
        } else if (!last) {
            const int u = i - nx;
            const T *Bk = B + (size_t)j * nx * nu;
            auto s = AT::from(-hu[(size_t)j * nu + u]);
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(-Bk[m * nu + u], vn[m]));
            su[u] = AT::to_T(s);
        }
    }
    group_sync(G);
    for (int i = t; i < nx + nu; i += G) {
        if (i < nx) {
            auto s = AT::zero();
            for (int m = 0; m < nx; ++m) s = AT::add(s, AT::prod(Qi[i * nx + m], sx[m]));
            zx[(size_t)kg * nx + i] = AT::to_T(s);
        } else if (!last) {
            const int u = i - nx;
            auto s = AT::zero();
            for (int m = 0; m < nu; ++m) s = AT::add(s, AT::prod(Ri[u * nu + m], su[m]));
            zu[(size_t)j * nu + u] = AT::to_T(s);
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline int form_grid(int nx, int Ktot) {
    const int groups = FORM_THREADS / group_size(nx);
    return ceil_div(Ktot, groups);
}

template <typename T>
cudaError_t launch_form_schur(const SchurArgs<T> &a, cudaStream_t s) {
    const int G = group_size(a.nx);
    if (a.Qf) {
        const size_t smem = dense_form_words<T>(a.nx, a.nu) * sizeof(T) * (FORM_THREADS / G);
        form_schur_dense_kernel<T><<<form_grid(a.nx, a.Kgrid), FORM_THREADS, smem, s>>>(a);
        return cudaGetLastError();
    }
    const size_t per = (size_t)2 * a.nx * a.nx + 2 * a.nx * a.nu + 4 * a.nx + 2 * a.nu;
    const size_t smem = per * sizeof(T) * (FORM_THREADS / G);
    form_schur_kernel<T><<<form_grid(a.nx, a.Kgrid), FORM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// Knots per CTA of the warp form for Kgrid knots on `sms` SMs.
static inline int fused_kpb(int Kgrid, int sms) {
    const int k = ceil_div(Kgrid, sms > 0 ? sms : 1);
    return k < 2 ? 2 : (k > FUSED_KPB_MAX ? FUSED_KPB_MAX : k);
}

template <typename T>
size_t form_fused_smem_bytes(int nx, int nu, int Kgrid, int sms) {
    return fused_warp_words<T>(nx, nu) * sizeof(T) * (fused_kpb(Kgrid, sms) + 1);
}

// nx <= 16 only (one warp per knot); larger states take the separate launches.
template <typename T>
cudaError_t launch_form_fused(const SchurArgs<T> &a, T *Pd, T *Po, int sms, cudaStream_t s) {
    if (group_size(a.nx) != 32) return cudaErrorInvalidValue;
    const size_t smem = form_fused_smem_bytes<T>(a.nx, a.nu, a.Kgrid, sms);
    const int kpb = fused_kpb(a.Kgrid, sms);
    const dim3 grid(ceil_div(a.Kgrid, kpb)), block(32 * (kpb + 1));
    if (a.nx == 14 && a.nu == 7)  // the Kuka arm's shape, specialised
        form_fused_warp_kernel<T, 14, 7><<<grid, block, smem, s>>>(a, Pd, Po, kpb);
    else
        form_fused_warp_kernel<T, 0, 0><<<grid, block, smem, s>>>(a, Pd, Po, kpb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_form_precon(int nx, BatchView bv, int Kgrid, const T *Sd, const T *So, T *Pd,
                               T *Po, cudaStream_t s) {
    const int groups = FORM_THREADS / group_size(nx);
    size_t smem1 = sizeof(T) * (size_t)nx * nx * groups;
    size_t smem2 = sizeof(T) * (size_t)4 * nx * nx * groups;
    cudaError_t e;
    precon_inv_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, smem1, s>>>(nx, bv, Sd, Pd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    precon_off_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, smem2, s>>>(nx, bv, Pd, So, Po);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recover(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                           const T *Qd, const T *Rd, const T *hx, const T *hu, const T *v, T *zx,
                           T *zu, cudaStream_t s) {
    const int groups = FORM_THREADS / group_size(nx);
    recover_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, sizeof(T) * nx * groups, s>>>(
        nx, nu, bv, A, B, Qd, Rd, hx, hu, v, zx, zu);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recover_dense(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                                 const T *Qf, const T *Rf, const T *hx, const T *hu, const T *v,
                                 T *zx, T *zu, cudaStream_t s) {
    const int groups = FORM_THREADS / group_size(nx);
    const size_t smem = sizeof(T) * ((size_t)nx * nx + nu * nu + 2 * nx + nu) * groups;
    recover_dense_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, smem, s>>>(
        nx, nu, bv, A, B, Qf, Rf, hx, hu, v, zx, zu);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cgh(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                       const T *Qd, const T *Rd, const T *hx, const T *hu, const T *w, T *out,
                       cudaStream_t s) {
    const int groups = FORM_THREADS / group_size(nx);
    cgh_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, sizeof(T) * (nx + nu) * groups, s>>>(
        nx, nu, bv, A, B, Qd, Rd, hx, hu, w, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad(int nx, int nu, BatchView bv, int Kgrid, const T *lam, const T *mu,
                        const T *dx, const T *du, const T *gq, const T *gr, T *gA, T *gB, T *gQd,
                        T *gRd, T *gc, cudaStream_t s) {
    grad_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, 0, s>>>(nx, nu, bv, lam, mu, dx, du,
                                                                  gq, gr, gA, gB, gQd, gRd, gc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B, const T *Qd,
                         const T *Rd, const T *q, const T *r, const T *c, T csign, const T *lam,
                         T *out, cudaStream_t s) {
    using X = typename Acc<T>::type;
    const int groups = FORM_THREADS / group_size(nx);
    resid_kernel<T><<<form_grid(nx, Kgrid), FORM_THREADS, sizeof(X) * (2 * nx + nu) * groups, s>>>(
        nx, nu, bv, A, B, Qd, Rd, q, r, c, csign, lam, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy(int nx, BatchView bv, int Kgrid, const T *d, T *lam, cudaStream_t s) {
    const int threads = 256;
    const int blocks = std::max(1, std::min(1024, ceil_div(Kgrid * nx, threads)));
    axpy_kernel<T><<<blocks, threads, 0, s>>>(nx, bv, d, lam);
    return cudaGetLastError();
}

// Packed copy of the symmetric diagonal blocks: Dp[k] holds the upper
// triangle of D[k] column by column (entry (i, j), i <= j, at j (j + 1) / 2
// + i) and zeros up to npk.  One thread per packed entry of one knot.
template <typename T>
__global__ void pack_diag_kernel(int nx, int npk, BatchView bv, const T *__restrict__ D, T *__restrict__ Dp) {
    const size_t n = (size_t)bv.total() * npk;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t k = e / npk;
        const int p = (int)(e % npk);
        T v = T(0);
        if (p < nx * (nx + 1) / 2) {
            int j = 0;  // column j holds entries [j (j + 1) / 2, (j + 1) (j + 2) / 2)
            while ((j + 1) * (j + 2) / 2 <= p) ++j;
            const int i = p - j * (j + 1) / 2;
            v = D[k * nx * nx + (size_t)i * nx + j];
        }
        Dp[e] = v;
    }
}

template <typename T>
cudaError_t launch_pack_diag(int nx, int npk, BatchView bv, int Kgrid, const T *D, T *Dp, cudaStream_t s) {
    const int threads = 256;
    const int blocks = std::max(1, std::min(4096, ceil_div(Kgrid * npk, threads)));
    pack_diag_kernel<T><<<blocks, threads, 0, s>>>(nx, npk, bv, D, Dp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(int nx, BatchView bv, int Kgrid, T *v, cudaStream_t s) {
    const int threads = 256;
    const int blocks = std::max(1, std::min(1024, ceil_div(Kgrid * nx, threads)));
    zero_kernel<T><<<blocks, threads, 0, s>>>(nx, bv, v);
    return cudaGetLastError();
}

// Raise every per-knot kernel's dynamic shared-memory ceiling once per device
// (large nx needs more than the 48 KB default).
template <typename T>
static cudaError_t form_prepare_t(int smem_optin) {
    cudaError_t e;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(form_schur_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(precon_inv_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(precon_off_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(recover_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(resid_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(form_schur_dense_kernel<T>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(form_fused_warp_kernel<T, 14, 7>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(form_fused_warp_kernel<T, 0, 0>, a, smem_optin))) return e;
    if ((e = cudaFuncSetAttribute(recover_dense_kernel<T>, a, smem_optin))) return e;
    return cudaFuncSetAttribute(cgh_kernel<T>, a, smem_optin);
}

cudaError_t form_prepare(int smem_optin) {
    cudaError_t e = form_prepare_t<float>(smem_optin);
    return e != cudaSuccess ? e : form_prepare_t<double>(smem_optin);
}

#define MPCG_INST(T)                                                                              \
    template cudaError_t launch_form_schur<T>(const SchurArgs<T> &, cudaStream_t);                \
    template cudaError_t launch_form_precon<T>(int, BatchView, int, const T *, const T *, T *,    \
                                               T *, cudaStream_t);                                \
    template cudaError_t launch_recover<T>(int, int, BatchView, int, const T *, const T *,        \
                                           const T *, const T *, const T *, const T *, const T *, \
                                           T *, T *, cudaStream_t);                               \
    template cudaError_t launch_cgh<T>(int, int, BatchView, int, const T *, const T *, const T *, \
                                       const T *, const T *, const T *, const T *, T *,           \
                                       cudaStream_t);                                             \
    template cudaError_t launch_grad<T>(int, int, BatchView, int, const T *, const T *,           \
                                        const T *, const T *, const T *, const T *, T *, T *,     \
                                        T *, T *, T *, cudaStream_t);                             \
    template cudaError_t launch_resid<T>(int, int, BatchView, int, const T *, const T *,          \
                                         const T *, const T *, const T *, const T *, const T *,   \
                                         T, const T *, T *, cudaStream_t);                        \
    template cudaError_t launch_axpy<T>(int, BatchView, int, const T *, T *, cudaStream_t);     \
    template cudaError_t launch_zero<T>(int, BatchView, int, T *, cudaStream_t);                 \
    template cudaError_t launch_pack_diag<T>(int, int, BatchView, int, const T *, T *, cudaStream_t); \
    template cudaError_t launch_form_fused<T>(const SchurArgs<T> &, T *, T *, int, cudaStream_t); \
    template size_t form_fused_smem_bytes<T>(int, int, int, int);                                \
    template cudaError_t launch_recover_dense<T>(int, int, BatchView, int, const T *, const T *, \
                                                 const T *, const T *, const T *, const T *,     \
                                                 const T *, T *, T *, cudaStream_t);
MPCG_INST(float)
MPCG_INST(double)
#undef MPCG_INST

}  // namespace mpcg
