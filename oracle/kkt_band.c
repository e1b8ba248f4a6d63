/*
 * ORACLE -- test infrastructure only.  Plain FP64 C, no BLAS, no blocking.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * What it computes: the exact solution of the trajectory-optimisation KKT
 * system (Sec. II-A, Step 2, Eq. KKT)
 *
 *      [ G  C^T ] [ y_z ]   [ h_z ]
 *      [ C   0  ] [ y_l ] = [ h_l ]
 *
 * with G = diag(Q_0, R_0, Q_1, R_1, ..., Q_{N-1}) (diagonal Q_k, R_k, or
 * dense SPD blocks when given) and C
 * the dynamics Jacobian: block row 0 is [I 0 ...]; block row k+1 holds
 * -A_k, -B_k, I on the columns of x_k, u_k, x_{k+1}.  For the forward solve
 * the right-hand side is (g, c) and the unknown is (-dz, lambda); the same
 * routine serves the adjoint solve because K is symmetric.
 *
 * Vectors use the paper's natural ordering: the z-part is
 * (x_0, u_0, x_1, u_1, ..., x_{N-1}) and the lambda-part is
 * (lambda_0, ..., lambda_{N-1}).
 *
 * How: the rows and columns are permuted symmetrically into a per-knot
 * interleaved order (lambda_k, x_k, u_k), which makes K banded with equal
 * lower and upper half-bandwidth kb = 2 nx + nu - 1.  K is indefinite (zero
 * (2,2) block), so the band is factorised by Gaussian elimination with
 * partial (row) pivoting, the band-storage scheme of a general banded LU
 * (the upper band grows to 2 kb through row interchanges).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Position of variable blocks in the interleaved order. */
static long knot_base(long k, int nx, int nu) { return k * (2L * nx + nu); }

/* Natural-order index of x_k[i], u_k[i] inside the z-part. */
static long nat_x(long k, int i, int nx, int nu) { return k * (nx + nu) + i; }
static long nat_u(long k, int i, int nx, int nu) { return k * (nx + nu) + nx + i; }

typedef struct {
    long n;      /* matrix order */
    int kb;      /* half-bandwidth of K */
    int w;       /* stored row width: columns i-kb .. i+2kb */
    double *ab;  /* row-major band rows */
} band_t;

static double *band_at(band_t *m, long i, long j) {
    return &m->ab[i * (long)m->w + (j - i + m->kb)];
}

static void band_set(band_t *m, long i, long j, double v) { *band_at(m, i, j) = v; }

/*
 * Assemble K in interleaved order.  Row/column blocks per knot k:
 *   lam_k (nx) | x_k (nx) | u_k (nu, only for k < N-1)
 * Rows for lam_k hold the constraint block row k of C; rows for x_k and u_k
 * hold the stationarity rows [G C^T].
 */
static void assemble(band_t *m, int nx, int nu, int N, const double *A, const double *B,
                     const double *Qd, const double *Rd, const double *Q, const double *R) {
    for (int k = 0; k < N; ++k) {
        long bl = knot_base(k, nx, nu), bx = bl + nx, bu = bl + 2 * nx;
        /* constraint row k: I on x_k, and -A_{k-1}, -B_{k-1} on x_{k-1}, u_{k-1} */
        for (int i = 0; i < nx; ++i) {
            band_set(m, bl + i, bx + i, 1.0);
            if (k > 0) {
                long pb = knot_base(k - 1, nx, nu);
                const double *Ak = A + (long)(k - 1) * nx * nx;
                const double *Bk = B + (long)(k - 1) * nx * nu;
                for (int j = 0; j < nx; ++j) band_set(m, bl + i, pb + nx + j, -Ak[i * nx + j]);
                for (int j = 0; j < nu; ++j) band_set(m, bl + i, pb + 2 * nx + j, -Bk[i * nu + j]);
            }
        }
        /* stationarity of x_k: Q_k on x_k, I on lam_k, -A_k^T on lam_{k+1} */
        for (int i = 0; i < nx; ++i) {
            if (Q)
                for (int j = 0; j < nx; ++j) band_set(m, bx + i, bx + j, Q[((long)k * nx + i) * nx + j]);
            else
                band_set(m, bx + i, bx + i, Qd[(long)k * nx + i]);
            band_set(m, bx + i, bl + i, 1.0);
            if (k < N - 1) {
                long nb = knot_base(k + 1, nx, nu);
                const double *Ak = A + (long)k * nx * nx;
                for (int j = 0; j < nx; ++j) band_set(m, bx + i, nb + j, -Ak[j * nx + i]);
            }
        }
        /* stationarity of u_k: R_k on u_k, -B_k^T on lam_{k+1} */
        if (k < N - 1) {
            long nb = knot_base(k + 1, nx, nu);
            const double *Bk = B + (long)k * nx * nu;
            for (int i = 0; i < nu; ++i) {
                if (R)
                    for (int j = 0; j < nu; ++j) band_set(m, bu + i, bu + j, R[((long)k * nu + i) * nu + j]);
                else
                    band_set(m, bu + i, bu + i, Rd[(long)k * nu + i]);
                for (int j = 0; j < nx; ++j) band_set(m, bu + i, nb + j, -Bk[j * nu + i]);
            }
        }
    }
}

/* Gaussian elimination with partial pivoting on the band, then back
 * substitution.  Returns 0, or 1 on an exactly singular pivot. */
static int band_solve(band_t *m, double *b) {
    long n = m->n;
    int kb = m->kb;
    for (long j = 0; j < n; ++j) {
        long last = j + kb < n - 1 ? j + kb : n - 1;
        long p = j;
        double best = fabs(*band_at(m, j, j));
        for (long i = j + 1; i <= last; ++i) {
            double v = fabs(*band_at(m, i, j));
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return 1;
        long cend = j + 2L * kb < n - 1 ? j + 2L * kb : n - 1;
        if (p != j) {
            for (long c = j; c <= cend; ++c) {
                double t = *band_at(m, j, c);
                *band_at(m, j, c) = *band_at(m, p, c);
                *band_at(m, p, c) = t;
            }
            double t = b[j]; b[j] = b[p]; b[p] = t;
        }
        double piv = *band_at(m, j, j);
        for (long i = j + 1; i <= last; ++i) {
            double l = *band_at(m, i, j) / piv;
            if (l == 0.0) continue;
            *band_at(m, i, j) = 0.0;
            for (long c = j + 1; c <= cend; ++c) *band_at(m, i, c) -= l * *band_at(m, j, c);
            b[i] -= l * b[j];
        }
    }
    for (long i = n - 1; i >= 0; --i) {
        long cend = i + 2L * kb < n - 1 ? i + 2L * kb : n - 1;
        double s = b[i];
        for (long c = i + 1; c <= cend; ++c) s -= *band_at(m, i, c) * b[c];
        b[i] = s / *band_at(m, i, i);
    }
    return 0;
}

long oracle_kkt_dim(int nx, int nu, int N) {
    return 2L * N * nx + (long)(N - 1) * nu;
}

/*
 * Solve K y = h.  h and y are in natural order: z-part (N nx + (N-1) nu
 * entries) followed by the lambda-part (N nx).  y may alias h.  Q and R,
 * when not NULL, are dense cost blocks Q[N][nx][nx], R[N-1][nu][nu] used
 * instead of the diagonals Qd, Rd.
 * Returns 0 on success, 1 if singular, 2 on bad arguments, 3 on allocation
 * failure.
 */
int oracle_kkt_solve_g(int nx, int nu, int N, const double *A, const double *B,
                       const double *Qd, const double *Rd, const double *Q, const double *R,
                       const double *h, double *y) {
    if (nx <= 0 || nu <= 0 || N <= 0) return 2;
    long n = oracle_kkt_dim(nx, nu, N);
    long nz = (long)N * nx + (long)(N - 1) * nu;
    band_t m;
    m.n = n;
    m.kb = 2 * nx + nu - 1;
    m.w = 3 * m.kb + 1;
    m.ab = (double *)calloc((size_t)n * m.w, sizeof(double));
    double *b = (double *)malloc((size_t)n * sizeof(double));
    if (!m.ab || !b) { free(m.ab); free(b); return 3; }
    assemble(&m, nx, nu, N, A, B, Qd, Rd, Q, R);
    /* natural -> interleaved */
    for (int k = 0; k < N; ++k) {
        long bl = knot_base(k, nx, nu);
        for (int i = 0; i < nx; ++i) {
            b[bl + i] = h[nz + (long)k * nx + i];
            b[bl + nx + i] = h[nat_x(k, i, nx, nu)];
        }
        if (k < N - 1)
            for (int i = 0; i < nu; ++i) b[bl + 2 * nx + i] = h[nat_u(k, i, nx, nu)];
    }
    int st = band_solve(&m, b);
    if (st == 0) {
        for (int k = 0; k < N; ++k) {
            long bl = knot_base(k, nx, nu);
            for (int i = 0; i < nx; ++i) {
                y[nz + (long)k * nx + i] = b[bl + i];
                y[nat_x(k, i, nx, nu)] = b[bl + nx + i];
            }
            if (k < N - 1)
                for (int i = 0; i < nu; ++i) y[nat_u(k, i, nx, nu)] = b[bl + 2 * nx + i];
        }
    }
    free(m.ab);
    free(b);
    return st;
}

/* The diagonal-cost form. */
int oracle_kkt_solve(int nx, int nu, int N, const double *A, const double *B,
                     const double *Qd, const double *Rd, const double *h, double *y) {
    return oracle_kkt_solve_g(nx, nu, N, A, B, Qd, Rd, NULL, NULL, h, y);
}
