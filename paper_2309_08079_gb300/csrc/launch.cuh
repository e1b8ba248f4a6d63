// Internal launch interface shared by api.cu, form.cu and pcg.cu.
#pragma once

#include "common.cuh"

namespace mpcg {

template <typename T>
struct SchurArgs {
    int nx, nu;
    BatchView bv;
    int Kgrid;  // host-side upper bound on the total knots (grid size only)
    const T *A, *B, *Qd, *Rd, *q, *r, *c;
    const T *Qf, *Rf;  // dense SPD cost blocks (nullptr: diagonal Qd, Rd)
    T *Sd, *So, *gamma;
    unsigned *info;
};

enum { MODE_REG = 0, MODE_PTR = 1 };

template <typename T>
struct PcgParams {
    int nx;
    BatchView bv;
    const T *Sd, *So, *Pd, *Po;
    const T *rhs;  // b = rhs_sign * rhs
    T rhs_sign;
    T *lam;
    const unsigned *info;
    mpcg_stats *stats;
    int *queue;       // instance counter (nullptr: static round robin)
    const int *inst_list;  // tickets -> instances (nullptr: ticket t is instance t)
    int n_tickets;         // instances to solve (B, or the list's length)
    double tol;
    int tol_mode;
    int max_iter;     // <= 0: 10 N nx
    int precon;       // 0: symmetric stair Phi^-1 (Pd, Po); 1: block Jacobi (Pd only)
    int kpc_max;      // knot slots per CTA (blockDim.x / LPK)
    int stage_smem;   // PTR mode: stage blocks in shared memory
    int vs;           // shared vector stride (elements per knot)
    int depth;        // pcg_tile_kernel: steps each knot stream copies ahead
    const T *Sdp, *Pdp;  // pcg_tile_kernel: packed diagonal blocks (nullptr: full Sd, Pd)
    int npk;             // entries per packed diagonal block
};

struct PcgLaunch {
    int cta_mode;  // 0: cluster per instance; 1: one CTA per instance, blocks from L2
                   // (pcg_cta_kernel); 2: one CTA per instance, blocks streamed as
                   // TMA tiles (pcg_tile_kernel)
    int C;         // CTAs per cluster
    int clusters;  // clusters in the grid
    int threads;   // threads per CTA
    int lpk, rpt, mode, stage, vs, kpc_max;
    int vw;        // pcg_tile_kernel: elements per shared-memory row load (2 or 4)
    int depth;     // pcg_tile_kernel: steps each knot stream copies ahead (1..4)
    int nxc;       // pcg_tile_kernel: nx fixed at compile time (14, 36), else 0
    int pk;        // pcg_tile_kernel: streams the packed diagonal blocks (nx = 36)
    int dot;       // float32 only: 1 accumulates the dot products in float64 (AccF64)
    size_t smem;
};

template <typename T> cudaError_t launch_form_schur(const SchurArgs<T> &, cudaStream_t);
template <typename T>
cudaError_t launch_form_precon(int nx, BatchView bv, int Kgrid, const T *Sd, const T *So, T *Pd,
                               T *Po, cudaStream_t s);
template <typename T>
cudaError_t launch_recover(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                           const T *Qd, const T *Rd, const T *hx, const T *hu, const T *v, T *zx,
                           T *zu, cudaStream_t s);
template <typename T>
cudaError_t launch_recover_dense(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                                 const T *Qf, const T *Rf, const T *hx, const T *hu, const T *v,
                                 T *zx, T *zu, cudaStream_t s);
template <typename T>
cudaError_t launch_cgh(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B,
                       const T *Qd, const T *Rd, const T *hx, const T *hu, const T *w, T *out,
                       cudaStream_t s);
template <typename T>
cudaError_t launch_grad(int nx, int nu, BatchView bv, int Kgrid, const T *lam, const T *mu,
                        const T *dx, const T *du, const T *gq, const T *gr, T *gA, T *gB, T *gQd,
                        T *gRd, T *gc, cudaStream_t s);
template <typename T>
cudaError_t launch_resid(int nx, int nu, BatchView bv, int Kgrid, const T *A, const T *B, const T *Qd,
                         const T *Rd, const T *q, const T *r, const T *c, T csign, const T *lam,
                         T *out, cudaStream_t s);
template <typename T>
cudaError_t launch_axpy(int nx, BatchView bv, int Kgrid, const T *d, T *lam, cudaStream_t s);
template <typename T>
cudaError_t launch_zero(int nx, BatchView bv, int Kgrid, T *v, cudaStream_t s);
template <typename T>
cudaError_t launch_pack_diag(int nx, int npk, BatchView bv, int Kgrid, const T *D, T *Dp, cudaStream_t s);
// entries per packed diagonal block: nx(nx+1)/2 rounded up to 4 (16 bytes)
__host__ __device__ __forceinline__ int packed_len(int nx) { return (nx * (nx + 1) / 2 + 3) / 4 * 4; }
template <typename T> cudaError_t pcg_launch(const PcgLaunch &, const PcgParams<T> &, cudaStream_t);
template <typename T> int pcg_max_clusters(const PcgLaunch &);
cudaError_t pcg_prepare(int smem_optin);
cudaError_t pcg_cta_prepare(int smem_optin);
cudaError_t pcg_tile_prepare(int smem_optin);
template <typename T>
size_t pcg_tile_smem_bytes(int nmax, int vs, int W, int NS, int nx, int depth, int npk);
template <typename T> cudaError_t pcg_tile_launch(const PcgLaunch &, const PcgParams<T> &, cudaStream_t);
template <typename T> int pcg_tile_max_blocks(const PcgLaunch &);
template <typename T> size_t pcg_cta_smem_bytes(int nmax, int vs, int W);
template <typename T> cudaError_t pcg_cta_launch(const PcgLaunch &, const PcgParams<T> &, cudaStream_t);
template <typename T> int pcg_cta_max_blocks(const PcgLaunch &);
cudaError_t form_prepare(int smem_optin);
template <typename T> size_t pcg_smem_bytes(int kpc_max, int vs, int C, int W, int nx, int stage, int dot);

}  // namespace mpcg
