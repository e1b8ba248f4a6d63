/*
 * mpcg.h -- C ABI of the GB300 (sm_103a) Schur-complement PCG solve path
 * for the KKT systems of direct trajectory optimisation (MPCGPU, arXiv
 * 2309.08079).
 *
 * The path (Sec. IV of the paper):
 *   mpcg_form_schur    S+ = C G^-1 C^T and gamma          (Sec. II-B, Eq. schur,
 *                                                          Eq. trajoptSchur_1/2)
 *   mpcg_form_precon   symmetric stair preconditioner     (Sec. IV-A)
 *   mpcg_pcg_solve     PCG on S+ lambda = -gamma          (Algorithm 1; the
 *                                                          per-block form of
 *                                                          Algorithm 2)
 *   mpcg_recover_step  dz = -G^-1 (g - C^T lambda)        (Eq. schur)
 *   mpcg_form_schur_precon  the first two in one launch
 * plus additions with no counterpart in the paper: batched (ragged horizon)
 * forms of every call, a backward (adjoint) pass, iterative refinement,
 * comparison preconditioners (mpcg_opts.precon), and a diagnostic of the
 * bounded device waits (mpcg_selftest_wait).  The outer loop's device
 * pieces on a synthetic model follow at the end: linearisation (Sec. II-A
 * Step 1) and the parallel line search (Sec. IV-C).
 *
 * Problem statement (Sec. II-A, Step 2).  N knot points, states
 * x_0..x_{N-1} (nx each), controls u_0..u_{N-2} (nu each).  G is diagonal:
 * G = diag(Qd_0, Rd_0, Qd_1, ..., Qd_{N-1}).  C has I in block row 0 and
 * [-A_k  -B_k  I] on (x_k, u_k, x_{k+1}) in block row k+1.
 *
 * Sign convention.  The paper writes S = -C G^-1 C^T, S lambda = gamma.
 * This library stores the positive definite S+ = C G^-1 C^T and solves
 * S+ lambda = -gamma, which has the same solution lambda.
 *
 * Conventions for every call:
 *  - All array arguments are DEVICE pointers owned by the caller, dense,
 *    row-major, of the element type named by dims.dtype (0 = float32,
 *    1 = float64).  Layouts (per instance):
 *        A[N-1][nx][nx]   B[N-1][nx][nu]   Qd[N][nx]   Rd[N-1][nu]
 *        q[N][nx]         r[N-1][nu]       c[N][nx]
 *        Sd[N][nx][nx]    diagonal blocks of S+ (D_0 = Qd_0^-1, D_{k+1} = theta_k)
 *        So[N-1][nx][nx]  So[k] = block (k+1, k) of S+ = phi_k = -A_k Q_k^-1
 *        Pd[N][nx][nx]    diagonal blocks of Phi^-1 (D_k^-1)
 *        Po[N-1][nx][nx]  Po[k] = block (k+1, k) of Phi^-1 = -Pd[k+1] So[k] Pd[k]
 *        gamma[N][nx]     gamma = c - C G^-1 g
 *        lambda[N][nx]    dx[N][nx]   du[N-1][nu]
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  They allocate no memory.  Calls made on one
 *    handle from several host threads at once must use different handles.
 *  - The return value reports argument and launch errors synchronously
 *    (MPCG_OK, MPCG_EINVAL, MPCG_ECUDA, MPCG_EUNSUPPORTED).  Numerical
 *    outcomes are written to device memory (mpcg_stats.status, info words).
 *  - Batched calls take `knot_off`, a DEVICE int array of B+1 entries:
 *    instance b owns knots knot_off[b] .. knot_off[b+1]-1 of every per-knot
 *    array and entries knot_off[b]-b .. knot_off[b+1]-b-2 of every
 *    per-control array (A, B, Rd, r, So, Po, du).  dims.N is then the LARGEST
 *    horizon in the batch (used to size launches) and every N_b >= 1.
 */
#ifndef MPCG_H
#define MPCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes (negative: never equal to a status code) */
#define MPCG_OK 0
#define MPCG_EINVAL (-1)       /* bad argument (null pointer, size, dtype) */
#define MPCG_ECUDA (-2)        /* a CUDA runtime call or launch failed */
#define MPCG_EUNSUPPORTED (-3) /* shape outside what the kernels support (float32: horizons
                                  up to ~1,340 knots at nx = 14, ~500 at nx = 36; every
                                  form keeps an instance's vectors on chip) */
#define MPCG_ETOOLARGE (-4)    /* needs more scratch than MPCG_NOALLOC_SCRATCH_BYTES */

/* numerical status written to mpcg_stats.status */
#define MPCG_CONVERGED 0
#define MPCG_NOT_CONVERGED 1 /* max_iter reached; lambda holds the last iterate */
#define MPCG_BREAKDOWN 2     /* p^T S+ p <= 0 or not finite */
#define MPCG_NONFINITE 3     /* a residual or preconditioned residual is not finite */
#define MPCG_BADINPUT 4      /* form_schur found Qd or Rd <= 0 or not finite */
#define MPCG_TIMEOUT 5       /* a bounded device wait gave up (never expected); lambda is then unspecified */

/* info bits written by mpcg_form_schur into mpcg_schur.info[b] */
#define MPCG_INFO_BADINPUT 1u

typedef struct {
    int nx, nu, N; /* N: horizon (batched calls: largest horizon) */
    int dtype;     /* 0 = float32, 1 = float64 */
} mpcg_dims;

typedef struct {
    const void *A, *B, *Qd, *Rd, *q, *r, *c;
    /* Optional general cost blocks (the Q_k, R_k of Sec. II-A's QP as full
       matrices): Q[N][nx][nx], R[N-1][nu][nu], symmetric positive definite,
       row-major.  When Q is not NULL, form_schur and recover_step use Q and
       R (R required when N > 1) and ignore Qd and Rd (which may be NULL); a
       block that is not SPD marks its instance MPCG_INFO_BADINPUT.
       refine_step and backward support diagonal costs only and return
       MPCG_EUNSUPPORTED for dense blocks.  NULL: diagonal Qd, Rd. */
    const void *Q, *R;
} mpcg_lq;

typedef struct {
    void *Sd, *So, *Pd, *Po, *gamma;
    unsigned int *info; /* device, one word per instance, or NULL */
    /* Optional packed copies of the symmetric diagonal blocks for the tiled
       PCG kernel at nx = 36 (float32): Sdp[K][npk], Pdp[K][npk] hold the
       upper triangles of Sd[k] and Pd[k] column by column (entry (i, j),
       i <= j, at j (j + 1) / 2 + i), npk = nx (nx + 1) / 2 rounded up to a
       multiple of 4, zero-padded; 16-byte aligned, caller-owned.  When both
       are non-NULL, mpcg_form_precon[_batched] and
       mpcg_form_schur_precon[_batched] write them after Pd, and the tiled
       kernel streams them instead of Sd and Pd (666 of 1,296 words per
       block); entry (j, i) is read as (i, j).  A caller that changes Sd or Pd
       after formation must form again or pass NULL.  NULL: unused. */
    void *Sdp, *Pdp;
} mpcg_schur;

typedef struct {
    double tol;    /* exit tolerance (<= 0: 1e-6) */
    int tol_mode;  /* 0: ||r||_2 <= tol ||b||_2 (recurrence residual);
                      1: paper's eta' = r^T Phi^-1 r < tol (Algorithm 1) */
    int max_iter;  /* <= 0: 10 N nx */
    int cluster;   /* CTAs per instance (1..16); 0 = automatic */
    int mode;      /* PCG kernel: 0 automatic; 1 a thread-block cluster per instance
                      (matrices held on chip, in registers for float32 nx = 14;
                      the automatic choice whenever the horizon fits); 2 one CTA
                      per instance reading the blocks from L2 (many instances at
                      once, any horizon that fits shared memory; the automatic
                      choice beyond a cluster); 3 one CTA per instance streaming
                      each knot's blocks through shared memory as TMA tiles
                      (even nx and 16-byte-aligned block arrays, else as 2);
                      4 a cluster per instance with the matrices staged in
                      shared memory, 8 lanes x 2 rows per knot and up to 64
                      knots per CTA (nx <= 16): half the SMs per instance of
                      mode 1, for throughput */
    /* Batched PCG only: solve just the instances listed (a DEVICE int
       array of n_instances distinct indices into the batch); NULL solves
       all B.  With a list, dims.N may be the largest horizon among the
       listed instances, which sizes the launch.  An entry >= B is skipped
       (nothing read or written for it, no stats); a negative entry ends
       the list for the CTA or cluster that draws it. */
    const int *instances;
    int n_instances;
    /* Preconditioner applied by the PCG: 0 the symmetric stair Phi^-1 of
       Sec. IV-A (Pd and Po, the default); for comparison, 1 block Jacobi,
       Phi^-1 = D^-1 (Pd only; Po is not read), and 2 the non-symmetric
       stair preconditioner of the work Sec. IV-A cites: the inverse of the
       stair matrix whose odd block rows (instance-local knot k odd) keep
       their off-diagonal blocks of S+, i.e. the rows of Phi^-1 at odd k and
       only Pd[k] at even k (same Pd, Po arrays).  It is not symmetric, so
       PCG has no convergence guarantee with it (on the Kuka-shaped workload
       it stalls from N = 32 on; it exists to show why the paper symmetrises
       it).  Other values: MPCG_EINVAL. */
    int precon;
    /* Backward calls only (mpcg_backward*): steps of iterative refinement of
       the adjoint solve S+ mu = lambda_bar' (as mpcg_refine_step does for
       the forward solve: the residual lambda_bar' - S+ mu formed in extended
       precision from the inputs, not from the stored S+, a correction PCG
       with the same S+ and Phi^-1, mu += correction).  0: none.  While they
       run, grads->q and grads->c serve as the correction's scratch; both
       receive their gradients afterwards.  Ignored by the other calls;
       negative: MPCG_EINVAL. */
    int refine;
    /* Accumulation of the PCG dot products for float32 (dtype 0):
       0 float pairs ("double-float": exact products by FMA, TwoSum
       additions, ~44 significant bits; the default), 1 float64 (products
       and every partial sum in FP64 instructions; slower on GB300, whose
       FP64 pipe is a small fraction of its FP32 rate).  1 runs in the
       cluster kernel and in the tiled kernel for nx = 14 and 36; the L2
       CTA kernel (mode 2) and other tiled shapes return
       MPCG_EUNSUPPORTED.  float64 always accumulates in float64.  Other
       values: MPCG_EINVAL. */
    int dot;
    /* Exit tolerance (relative residual, the correction's own right-hand
       side) of the correction solves of iterative refinement
       (mpcg_refine_step*, and the backward's opts.refine steps).  <= 0: tol.
       The correction only has to shrink an error already at the float32
       floor of S+, so a loose test (1e-3) reaches the same result in about
       half the iterations of 1e-6. */
    double refine_tol;
} mpcg_opts;

typedef struct {
    int iters;     /* PCG iterations performed */
    int status;    /* MPCG_CONVERGED, ... */
    double eta;    /* final r^T Phi^-1 r */
    double relres; /* final ||r||_2 / ||b||_2 (recurrence residual) */
} mpcg_stats;

typedef struct {
    void *A, *B, *Qd, *Rd, *q, *r, *c; /* gradients, input layouts */
} mpcg_grads;

typedef struct mpcg_handle mpcg_handle;

/* Library version as "major.minor.patch". */
const char *mpcg_version(void);

/* Message for a return code (< 0 or MPCG_OK) or a status code (>= 0); never NULL. */
const char *mpcg_strerror(int code);

/*
 * Create a handle bound to the CUDA device current on the calling thread.
 * Queries the device (SM count, cluster limits) and sets the kernels'
 * launch attributes once.  Returns MPCG_ECUDA if no device is usable.
 */
int mpcg_create(mpcg_handle **out);
void mpcg_destroy(mpcg_handle *h);

/*
 * Bytes of device workspace the batched and backward calls need for a
 * batch of B instances with the given dims (single-instance calls need
 * none and accept NULL).  The workspace is caller-owned and may be reused
 * across calls that do not overlap on the GPU.
 */
size_t mpcg_workspace_bytes(mpcg_dims dims, int B);

/*
 * S+ and gamma, one block row per knot (Sec. II-B, Eq. trajoptSchur_1/2):
 *   theta_k = A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T + Q_{k+1}^-1
 *   phi_k   = -A_k Q_k^-1
 *   zeta_k  = -A_k Q_k^-1 q_k - B_k R_k^-1 r_k + Q_{k+1}^-1 q_{k+1}
 * Writes Sd, So, gamma.  If schur->info is not NULL it is cleared and
 * MPCG_INFO_BADINPUT is set when any Qd or Rd entry is <= 0 or not finite.
 */
int mpcg_form_schur(mpcg_handle *h, mpcg_dims dims, const mpcg_lq *lq, mpcg_schur *schur,
                    void *stream);

/*
 * Symmetric stair preconditioner (Sec. IV-A): Pd[k] = Sd[k]^-1 (Gauss-Jordan,
 * symmetrised) and Po[k] = -Pd[k+1] So[k] Pd[k].  Reads Sd, So; writes Pd, Po.
 */
int mpcg_form_precon(mpcg_handle *h, mpcg_dims dims, mpcg_schur *schur, void *stream);

/*
 * mpcg_form_schur followed by mpcg_form_precon in one launch (nx <= 16): one
 * warp per knot k forms block row k of S+, gamma_k and Pd[k]; a CTA takes
 * consecutive knots and one extra warp that forms D_{k+1} and phi_k of the
 * knot after its last, so that Po[k] = -Pd[k+1] phi_k Pd[k] is formed from
 * shared memory.  The outputs are those of the two calls up to rounding
 * (the same formulas in the same order; ~1 ulp per entry where the compiler
 * contracts other multiply-adds).
 * Dense cost blocks (lq->Q) and nx > 16 take the two calls' route.  Same
 * arguments and errors as mpcg_form_schur; schur->Pd and schur->Po are
 * required.
 */
int mpcg_form_schur_precon(mpcg_handle *h, mpcg_dims dims, const mpcg_lq *lq, mpcg_schur *schur,
                           void *stream);

/*
 * PCG (Algorithm 1) on S+ lambda = -gamma with preconditioner Phi^-1, in one
 * persistent launch.  `lambda` is read as the warm start lambda_0 and
 * overwritten with the result.  `stats` is a DEVICE pointer (one entry)
 * written at exit.  `opts` is a HOST pointer (NULL: defaults).  Dot
 * products are accumulated beyond the storage precision (float32 pairs for
 * dtype 0, float64 for dtype 1).  If schur->info flags bad input, lambda is
 * left unchanged and stats->status = MPCG_BADINPUT.
 */
int mpcg_pcg_solve(mpcg_handle *h, mpcg_dims dims, const mpcg_schur *schur, void *lambda,
                   const mpcg_opts *opts, mpcg_stats *stats, void *stream);

/*
 * The launch shape mpcg_pcg_solve[_batched] uses for these arguments (the
 * same choice, made once and cached on the handle; nothing is launched):
 * shape[0] = kernel form (0 a thread-block cluster per instance, 1 one CTA
 * per instance reading the blocks from L2, 2 the tiled kernel streaming
 * TMA tiles), shape[1] = CTAs per cluster, shape[2] = clusters (or CTAs) in
 * the grid, shape[3] = threads per CTA, shape[4] = tiled kernel: steps each
 * knot stream copies ahead (else 0), shape[5] = tiled kernel: 1 if it
 * streams the packed diagonal blocks (schur->Sdp, Pdp), else 0.  `shape` is
 * a HOST int[6]; the schur pointers matter only through their alignment
 * (the tiled kernel needs 16-byte-aligned blocks) and whether the packed
 * copies are given.  B = 1 for a single instance.
 */
int mpcg_pcg_shape(mpcg_handle *h, mpcg_dims dims, int B, const mpcg_schur *schur,
                   const mpcg_opts *opts, int *shape);

/*
 * Primal step (Eq. schur): dz = -G^-1 (g - C^T lambda), i.e.
 *   dx_k = (lambda_k - A_k^T lambda_{k+1} - q_k) / Qd_k   (k < N-1)
 *   dx_{N-1} = (lambda_{N-1} - q_{N-1}) / Qd_{N-1}
 *   du_k = (-B_k^T lambda_{k+1} - r_k) / Rd_k
 */
int mpcg_recover_step(mpcg_handle *h, mpcg_dims dims, const mpcg_lq *lq, const void *lambda,
                      void *dx, void *du, void *stream);

/*
 * One step of mixed-precision iterative refinement of lambda (no
 * counterpart in the paper; it lifts the accuracy floor that rounding S+ to
 * working precision sets).  The exact residual
 *     b - S+ lambda = -(C dz(lambda) + c),   dz(lambda) = G^-1 (C^T lambda - g),
 * is formed per knot in extended precision from the inputs `lq` (not from
 * the stored S+), the correction S+ d = residual is solved by PCG with the
 * same S+ and Phi^-1 from d = 0 (exit test: relative residual
 * opts->refine_tol, else opts->tol), and lambda += d.  `workspace` needs
 * mpcg_workspace_bytes(dims, B) bytes; `stats` (device) receives the
 * correction solve's stats (relres is relative to the residual).
 */
int mpcg_refine_step(mpcg_handle *h, mpcg_dims dims, const mpcg_lq *lq, const mpcg_schur *schur,
                     void *lambda, const mpcg_opts *opts, mpcg_stats *stats, void *workspace,
                     void *stream);
int mpcg_refine_step_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                             const mpcg_lq *lq, const mpcg_schur *schur, void *lambda,
                             const mpcg_opts *opts, mpcg_stats *stats, void *workspace,
                             void *stream);

/* Batched forms: B independent instances in one launch each (see knot_off
 * above).  Stats has B entries; pcg_solve_batched takes a workspace of
 * mpcg_workspace_bytes(dims, B) bytes, of which it uses only the first 256
 * (its instance queue), so calls that run at once on different streams
 * (e.g. one per horizon class, each with an instance list in opts) need
 * 256-byte workspaces of their own.  An instance whose horizon exceeds what
 * dims.N sized the launch for gets status MPCG_BADINPUT and is not solved. */
int mpcg_form_schur_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                            const mpcg_lq *lq, mpcg_schur *schur, void *stream);
int mpcg_form_precon_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                             mpcg_schur *schur, void *stream);
int mpcg_form_schur_precon_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                                   const mpcg_lq *lq, mpcg_schur *schur, void *stream);
int mpcg_pcg_solve_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                           const mpcg_schur *schur, void *lambda, const mpcg_opts *opts,
                           mpcg_stats *stats, void *workspace, void *stream);
int mpcg_recover_step_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                              const mpcg_lq *lq, const void *lambda, void *dx, void *du,
                              void *stream);

/*
 * Backward pass (no counterpart in the paper).  Given the forward inputs,
 * the S+ / Phi^-1 built by the forward, its solution (lambda, dx, du) and
 * the loss gradients lam_bar = dL/dlambda, dx_bar = dL/ddx, du_bar =
 * dL/ddu, computes dL/d(A, B, Qd, Rd, q, r, c) into `grads`:
 *   seed      lambda_bar' = lam_bar + C G^-1 (dx_bar, du_bar)
 *   adjoint   S+ mu = lambda_bar'  (PCG with the same Phi^-1)
 *   g_bar     = G^-1 (C^T mu - (dx_bar, du_bar))
 *   Qd_bar = g_bar_x * dx, Rd_bar = g_bar_u * du, q_bar = g_bar_x,
 *   r_bar = g_bar_u, c_bar = -mu,
 *   A_bar_k = mu_{k+1} dx_k^T + lambda_{k+1} g_bar_x_k^T,
 *   B_bar_k = mu_{k+1} du_k^T + lambda_{k+1} g_bar_u_k^T.
 * `workspace` needs mpcg_workspace_bytes(dims, B) bytes (holds lambda_bar'
 * and mu).  `stats` (device, B entries) receives the adjoint solve's stats.
 * The _batched form takes knot_off as above; the plain form is B = 1 with
 * knot_off = NULL.
 */
int mpcg_backward_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                          const mpcg_lq *lq, const mpcg_schur *schur, const void *lambda,
                          const void *dx, const void *du, const void *lam_bar,
                          const void *dx_bar, const void *du_bar, const mpcg_grads *grads,
                          const mpcg_opts *opts, mpcg_stats *stats, void *workspace,
                          void *stream);
int mpcg_backward(mpcg_handle *h, mpcg_dims dims, const mpcg_lq *lq, const mpcg_schur *schur,
                  const void *lambda, const void *dx, const void *du, const void *lam_bar,
                  const void *dx_bar, const void *du_bar, const mpcg_grads *grads,
                  const mpcg_opts *opts, mpcg_stats *stats, void *workspace, void *stream);

/*
 * Backward pass that allocates nothing and takes no workspace (the paper
 * has no counterpart).
 *
 * Who needs it: callers that cannot allocate device memory when they
 * differentiate -- a controller whose memory is fixed at start-up and
 * whose control loop must not enter the allocator (an allocation can take
 * locks and has no bounded latency), or a host framework that owns every
 * allocation and hands this library only the problem's tensors.  For them
 * the scratch that mpcg_backward_batched takes as `workspace` (the adjoint
 * right-hand side, the adjoint solution and the instance queue:
 * mpcg_workspace_bytes(dims, B) bytes) comes instead from one fixed array
 * of MPCG_NOALLOC_SCRATCH_BYTES bytes of device memory.  mpcg_create
 * reserves it on the handle's device (looking up its address there, which
 * under CUDA's lazy module loading is what commits it), so a device that
 * has not that much memory free fails at mpcg_create, not inside this call;
 * every GPU that gets a handle keeps the array until the process exits.
 *
 * Arguments, layouts and results are those of mpcg_backward_batched
 * (knot_off may be NULL when B == 1).  Behaviour specific to this call:
 *  - the handle must belong to the current device (else MPCG_EINVAL);
 *  - a problem whose scratch exceeds MPCG_NOALLOC_SCRATCH_BYTES is refused
 *    with MPCG_ETOOLARGE before anything is launched;
 *  - it calls no cudaMalloc, cudaFree or allocating library routine;
 *  - all calls share the one array, which keeps the last call's contents:
 *    each call clears what must start at zero, and calls that overlap on
 *    the GPU (other streams, other host threads) race -- serialise them.
 */
#define MPCG_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
int mpcg_backward_batched_noalloc(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                                  const mpcg_lq *lq, const mpcg_schur *schur, const void *lambda,
                                  const void *dx, const void *du, const void *lam_bar,
                                  const void *dx_bar, const void *du_bar, const mpcg_grads *grads,
                                  const mpcg_opts *opts, mpcg_stats *stats, void *stream);

/* ---------------------------------------------------------------------
 * The outer loop around the solve (Sec. II-A Steps 1 and 3, Sec. IV-C) on
 * the library's synthetic model.  The paper linearises robot dynamics that
 * are not part of this library; these calls use a Kuka-shaped stand-in so
 * that a whole SQP iteration (linearise, form, precondition, solve,
 * recover, line-search) runs on the device:
 *   h = nx/2 joints, x = (p, v), u in R^nu (nu <= h),
 *   v+ = v + dt (P u - damp * v - stiff * sin p),   p+ = p + dt v+,
 *   l(x, u) = 1/2 sum wq (x - xref_k)^2 + 1/2 sum wr u^2 (stage),
 *   l_f(x)  = 1/2 sum wf (x - xref_{N-1})^2 (terminal).
 * Trajectories use the solve path's layouts: X[N][nx], U[N-1][nu],
 * xref[N][nx]; batched calls add knot_off (as above) and xs[B][nx].
 * nx <= 64, nu <= 32.
 * --------------------------------------------------------------------- */
typedef struct {
    int nx, nu;
    double dt;
    const void *P;           /* [h][nu] input matrix */
    const void *damp, *stiff; /* [h] */
    const void *wq, *wr, *wf; /* [nx], [nu], [nx] diagonal cost weights */
} mpcg_model;

/* Writable LQ arrays (layouts of mpcg_lq). */
typedef struct {
    void *A, *B, *Qd, *Rd, *q, *r, *c;
} mpcg_lq_out;

/* Step 1 of Sec. II-A at the trajectory (X, U): A_k = df/dx, B_k = df/du,
 * Qd_k = wq (wf at the last knot), Rd_k = wr, q_k = Qd_k (x_k - xref_k),
 * r_k = wr u_k, c_0 = x_0 - x_s, c_{k+1} = x_{k+1} - f(x_k, u_k) (the c of
 * Eq. KKT).  The outputs feed mpcg_form_schur as an mpcg_lq. */
int mpcg_linearize(mpcg_handle *h, mpcg_dims dims, const mpcg_model *model, const void *X,
                   const void *U, const void *xref, const void *xs, const mpcg_lq_out *out,
                   void *stream);
int mpcg_linearize_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                           const mpcg_model *model, const void *X, const void *U,
                           const void *xref, const void *xs, const mpcg_lq_out *out,
                           void *stream);

/* Parallel line search (Sec. IV-C): for a = 0 .. n_alpha-1 (n_alpha <= 32)
 * the L1 merit  J(X', U') + mu (||x'_0 - x_s||_1 + sum_k ||x'_{k+1} -
 * f(x'_k, u'_k)||_1)  of (X', U') = (X, U) + 2^-a (dX, dU), evaluated in
 * FP64 at the working-precision candidate points, is written to merit[b][a]
 * (DEVICE double array, B x n_alpha); then every instance takes its
 * smallest merit (merits within a relative 1e-11 of it count as ties; the
 * longest tied step wins) and X, U are updated in
 * place; alpha_index[b] (DEVICE int array, or NULL) receives the chosen a.
 * mu > 0 is used as given; mu <= 0 takes mu_b = 1.1 max(1, ||lambda_b||_inf)
 * from lambda (the multipliers of the solve that produced dX, dU). */
int mpcg_line_search(mpcg_handle *h, mpcg_dims dims, const mpcg_model *model, void *X, void *U,
                     const void *dX, const void *dU, const void *xref, const void *xs,
                     const void *lambda, double mu, int n_alpha, double *merit, int *alpha_index,
                     void *stream);
int mpcg_line_search_batched(mpcg_handle *h, mpcg_dims dims, int B, const int *knot_off,
                             const mpcg_model *model, void *X, void *U, const void *dX,
                             const void *dU, const void *xref, const void *xs,
                             const void *lambda, double mu, int n_alpha, double *merit,
                             int *alpha_index, void *stream);

/* Diagnostic of the bounded device waits (not in the paper).  Every PCG
 * exchange completes on an mbarrier filled by peer CTAs' st.async pushes and
 * is awaited with a %globaltimer deadline, so a missing push ends the solve
 * with MPCG_TIMEOUT instead of hanging.  This call runs that pattern in one
 * two-CTA cluster: each CTA expects 4 bytes on its own mbarrier, pushes 4
 * bytes to the other only if `push` is non-zero, and waits at most limit_s
 * seconds (1e-6 <= limit_s <= 1, else MPCG_EINVAL).  `status` is a DEVICE
 * int[2] that receives, per CTA, MPCG_CONVERGED if its wait completed with
 * the pushed value and MPCG_TIMEOUT if it gave up.  With push = 0 both waits
 * run out by construction; the context stays usable. */
int mpcg_selftest_wait(mpcg_handle *h, int push, double limit_s, int *status, void *stream);

/* Diagnostic of the give-up path (not in the paper).  A cluster CTA whose
 * bounded wait gave up must not leave while peers may still push into its
 * shared memory, nor leave its peers waiting out their own limits: the PCG
 * kernels then drain the cluster -- set an abort flag in every peer (their
 * waits poll it), arrive once on every peer's "stopped" mbarrier, wait
 * (bounded) for every peer's arrival, let pushes in flight land, leave.
 * This call runs that path in one four-CTA cluster where every CTA expects a
 * 4-byte push from each of the other three.  mode 0: every CTA pushes and
 * every wait completes.  mode 1: CTA 0 withholds its pushes and gives up at
 * once; the other three cannot complete and are released by the abort flag.
 * Waits are bounded by limit_s seconds (1e-3 <= limit_s <= 1, else
 * MPCG_EINVAL).  DEVICE outputs, one entry per CTA: status[4] =
 * MPCG_CONVERGED (wait completed), MPCG_TIMEOUT (gave up or was told to
 * stop, and every peer reported stopping) or -MPCG_TIMEOUT (a peer never
 * reported within the limit); elapsed_ns[4] = nanoseconds from the start of
 * its wait to its exit (well below limit_s when the flag released it). */
int mpcg_selftest_drain(mpcg_handle *h, int mode, double limit_s, int *status,
                        unsigned long long *elapsed_ns, void *stream);

/* Microbenchmark of the PCG kernels' cluster reduction (not in the paper;
 * the latency floor that the single-instance solve is measured against).
 * One cluster of C CTAs x W warps (1 <= C, W <= 16; else MPCG_EINVAL) runs
 * `rounds` (1..10^6) rounds of the two exchanges of a PCG iteration
 * (Algorithm 1's two reductions) exactly as the float32 cluster kernel
 * performs them -- halo pushes from the boundary warps, a shuffle sum per
 * warp, warp 0 combining the warp sums and pushing the CTA sum into every
 * CTA with st.async, a bounded mbarrier wait, a CTA barrier and the sum of
 * the C partials -- with no other arithmetic.  DEVICE outputs: out[0] =
 * SM clock cycles and out[1] = nanoseconds over all rounds (CTA 0), so one
 * exchange takes out / (2 rounds); status[C] = MPCG_CONVERGED per CTA, or
 * MPCG_TIMEOUT if a wait gave up (after 1 s). */
int mpcg_bench_exchange(mpcg_handle *h, int C, int W, int rounds, unsigned long long *out,
                        int *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MPCG_H */
