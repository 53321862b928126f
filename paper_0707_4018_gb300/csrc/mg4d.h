// Two-level adaptive multigrid for the 4d SU(3) Wilson operator (paper: the
// adaptive setup, Eq. P1, Eq. Galerkin and the V-cycle, applied to the
// four-dimensional case of its outlook). Internal interface between the C ABI
// (mg.cu) and the 4d engine (mg4d.cu, mg4d_kernels.cu).
#pragma once

#include <vector>

#include "kernels.h"

namespace mg {

// blocking of the fine 4d lattice: blocks of B[0] x .. x B[3] sites, coarse
// lattice nb[mu] = L[mu] / B[mu]; Nv near-null vectors, each split by
// chirality, so N = 2 Nv coarse dofs per site. Column c < N of a block's
// prolongator is the chirality half chi = c / Nv of vector k = c % Nv: it lives
// on the 6 dofs 6 chi .. 6 chi + 5 of each site (spins 2 chi, 2 chi + 1).
struct Block4 {
  int L[4], B[4], nb[4];
  int bvol;     // sites per block
  int nblocks;  // coarse sites
  int Nv;       // vectors per chirality
};

struct Coarse4 {
  int nb[4];
  int N;
  long long nsites;
};

// ---- kernels (mg4d_kernels.cu); V: [b][c][s][6] (block-major, Nh = bvol * 6 per column),
// Y: [j][dir][col][row] with dir 0 = self, 1 + 2 mu = +mu (source j + mu), 2 + 2 mu = -mu ----
template <typename R>
void launch_restrict4(const Cx<R> *V, const Cx<R> *fine, Cx<R> *coarse, const Block4 &g, cudaStream_t s,
                      int nvec = 1);
// fine += P coarse
template <typename R>
void launch_prolong4(const Cx<R> *V, const Cx<R> *coarse, Cx<R> *fine, const Block4 &g, cudaStream_t s,
                     int nvec = 1);
// V[b][chi Nv + k] = chirality half chi of vector k (vectors [k][x][12], stride vstride)
void launch_gather_split4(const Cx<double> *vecs, long long vstride, Cx<double> *V, const Block4 &g, cudaStream_t s);
// modified Gram-Schmidt, twice, of the Nv columns of each (block, chirality), in place
void launch_block_gs4(Cx<double> *V, const Block4 &g, cudaStream_t s);
// Y = P^dagger D P (written in FP64) for the fine Wilson operator with diagonal `diag`; CT the
// links', prolongator's and arithmetic's type (float: FP32 products for mixed hierarchies)
template <typename CT>
void launch_galerkin4(const Cx<CT> *U, double diag, const Cx<CT> *V, Cx<double> *Y, const Block4 &g, cudaStream_t s);
// out = a (A + shift_v) in + c b on the coarse lattice (nvec vectors, stride nsites * N);
// the operator's precision RY may be below the vectors' RV (float / double: FP32 sums)
template <typename RY, typename RV>
void launch_coarse4_apply(const Cx<RY> *Y, const Cx<RV> *in, Cx<RV> *out, const Coarse4 &g, const Cx<RV> *b,
                          double a, double c, cudaStream_t s, int nvec = 1, const double *shift = nullptr);
// Minv[j] = inverse of the self block Y[j][0] (FP64 Gauss-Jordan, partial pivoting); *info
// set to 1 if a block is singular
void launch_block_invert4(const Cx<double> *Y, Cx<double> *Minv, const Coarse4 &g, int *info, cudaStream_t s);
// z_j = Minv_j r_j for nvec vectors (FP64, stride nsites N; Minv in R)
template <typename R>
void launch_block_apply4(const Cx<R> *Minv, const Cx<double> *r, Cx<double> *z, const Coarse4 &g, cudaStream_t s,
                         int nvec = 1);
// GCR step with device-side coefficients formed from the reduction of launch_gcr_dots:
// projection, normalisation and the x, r update; state[0] = |r|^2 - |alpha|^2
void launch_gcr_update_dev(const Cx<double> *W, Cx<double> *Wk, const Cx<double> *Z, Cx<double> *Zk, int k,
                           const double *dots, double *state, Cx<double> *x, Cx<double> *r, long long n,
                           cudaStream_t s);
// FP32 vectors (coefficients formed in FP64), and the block-Jacobi apply on FP32 vectors
void launch_gcr_update_dev(const Cx<float> *W, Cx<float> *Wk, const Cx<float> *Z, Cx<float> *Zk, int k,
                           const double *dots, double *state, Cx<float> *x, Cx<float> *r, long long n,
                           cudaStream_t s);
// coarse apply with the operator in FP16 (32-bit words, real part in the low half, laid out as
// Y) and FP32 vectors and sums: out = a A in + c b (one vector); the FP16 copy of an FP64 stencil
void launch_coarse4_apply_h(const unsigned int *Yh, const Cx<float> *in, Cx<float> *out, const Coarse4 &g,
                            const Cx<float> *b, double a, double c, cudaStream_t s);
void launch_pack_half2(const Cx<double> *in, unsigned int *out, long long n, cudaStream_t s);
// graph-replayed coarse GCR on FP32 vectors: the step with k = ctl[1], w = wt and z = r (W_k, Z_k
// written at W + k n, Z + k n); the kernel that starts a restart cycle (k = 0) and sets the WHILE
// condition; the kernel that ends an iteration and decides whether the loop goes on (state:
// st[0] residual estimate, st[1] |b|^2, st[3] iterations)
void launch_gcr_update_loop(Cx<float> *W, Cx<float> *Z, const Cx<float> *wt, const int *ctl, const double *dots,
                            double *state, Cx<float> *x, Cx<float> *r, long long n, cudaStream_t s);
void launch_coarse4_cycle_start(int *ctl, const double *st, int max_iter, cudaGraphConditionalHandle h,
                                cudaStream_t s);
void launch_coarse4_control(int *ctl, double *st, double tol2_rel, int restart, int max_iter,
                            cudaGraphConditionalHandle h, cudaStream_t s);
// its batched form (nb <= 32 vectors): estimates, thresholds and active flags from |b_v|^2, and
// the kernel that starts a restart cycle (the iterations use the batched device-k kernels of
// kernels.h)
void launch_coarse4_batch_init(const double *bn2, double tol2_rel, int nb, double *stv, int *act, cudaStream_t s);
void launch_coarse4_batch_cycle_start(int *ctl, const int *act, int nb, int max_iter, cudaGraphConditionalHandle h,
                                      cudaStream_t s);
void launch_block_apply4_32(const Cx<float> *Minv, const Cx<float> *r, Cx<float> *z, const Coarse4 &g,
                            cudaStream_t s, int nvec = 1);
// Yt[j][dir] = Y[j][dir] Minv[src(j, dir)]: the block-Jacobi right-preconditioned stencil A M
void launch_precondition4(const Cx<double> *Y, const Cx<double> *Minv, Cx<double> *Yt, const Coarse4 &g,
                          cudaStream_t s);
// batched MR: out[3 v .. 3 v + 2] = (<a_v, b_v>, |a_v|^2) summed in R (partials: nvec x
// max_blocks x 3 doubles, tickets: nvec zeroed counters), then x_v += alpha_v r_v,
// r_v -= alpha_v Ar_v with alpha_v = omega <Ar_v, r_v> / |Ar_v|^2 from those sums
template <typename R>
void launch_dot_norm_batch(const Cx<R> *a, const Cx<R> *b, long long n, int nvec, double *out, double *partials,
                           unsigned int *tickets, int max_blocks, cudaStream_t s);
template <typename R>
void launch_mr_update_batch(const double *sc, double omega, Cx<R> *x, Cx<R> *r, const Cx<R> *Ar, long long n,
                            int nvec, cudaStream_t s);
// tensor-core coarse apply (coarse_tc.cu), N = 48: BF16 A-fragments of Re Y and Im Y
// (nsites x 9 x 2 x 9 x 32 uint4) from the FP64 stencil (lo: of what the BF16 rounding
// leaves), then out_n = A_c in_n for nvec complex64 vectors [n][site][48]; split 0: BF16
// operands, 1: vectors as BF16 hi + lo, 2: the operator too (needs Ypklo)
void launch_pack_coarse4_bf16(const Cx<double> *Y, uint4 *Ypk, long long nsites, cudaStream_t s, bool lo = false);
void launch_coarse4_apply_tc(const uint4 *Ypk, const Cx<float> *in, Cx<float> *out, const int nb[4], int nvec,
                             cudaStream_t s, int split = 0, const uint4 *Ypklo = nullptr);
// exports: Y in [j][dir][row][col]; P as N fine vectors [c][x][12]
void launch_coarse4_to_canonical(const Cx<double> *Yi, Cx<double> *Yc, const Coarse4 &g, cudaStream_t s);
void launch_prolongator4_to_canonical(const Cx<double> *V, Cx<double> *out, const Block4 &g, cudaStream_t s);

// ---- engine (mg4d.cu) ----
struct Engine4;
struct Solve4 {
  int iters = 0;
  bool converged = false;
  double rel = 0.0;
  long long apps[MG_MAX_LEVELS] = {0, 0, 0, 0};
  long long coarsest_iters = 0;
  float ms = 0.f;
};

void validate4(const mg_geom *g, const mg_params *p);
// allocates the hierarchy and copies U (device complex128 [x][4][3][3]) on stream s, then runs
// the full adaptive setup (run_setup; otherwise the caller builds the level from saved vectors
// with engine4_build_level before any solve)
Engine4 *engine4_create(const mg_geom *g, const void *U, double m, const mg_params *p, cudaStream_t s,
                        bool run_setup = true);
void engine4_destroy(Engine4 *e);
Solve4 engine4_solve(Engine4 &e, const void *chi, void *psi, double tol);
void engine4_update_mass(Engine4 &e, double m);
void engine4_level_size(const Engine4 &e, int level, long long *n_sites, int *n_int);
void engine4_level_apply(Engine4 &e, int level, const void *in, void *out);
void engine4_restrict(Engine4 &e, const void *fine, void *coarse);
void engine4_prolong(Engine4 &e, const void *coarse, void *fine);
void engine4_vcycle(Engine4 &e, const void *b, void *x);
void engine4_smooth(Engine4 &e, const void *b, void *x, int nu);
void engine4_build_level(Engine4 &e, const void *vectors);
long long engine4_null_vector_count(const Engine4 &e);  // complex128 elements of the Nv fine vectors
const void *engine4_links(const Engine4 &e);            // the engine's FP64 copy of U (device)
void engine4_get_null_vectors(Engine4 &e, void *out);
void engine4_get_prolongator(Engine4 &e, void *out);
void engine4_get_coarse_op(Engine4 &e, void *out);
long long engine4_coarsest_solve(Engine4 &e, const void *b, void *x, float *ms);
// nrhs systems D psi_v = chi_v (at the context mass) in lockstep through one hierarchy
// (FP64 flexible GCR over the batch, batched V-cycles whose coarse solve applies the
// coarse operator to all vectors on tensor cores); nrhs <= max_rhs
std::vector<Solve4> engine4_solve_batch(Engine4 &e, int nrhs, const void *chi, void *psi, double tol);
// out_n = A_c in_n for nrhs complex64 coarse vectors: tensor cores (BF16 operands, FP32 sums)
// or, with tensor_cores = 0, CUDA cores in FP32 (the comparison path)
void engine4_coarse_apply_mrhs(Engine4 &e, int nrhs, const void *in, void *out, int tensor_cores);

}  // namespace mg
