// Host-side launchers of the multigrid kernels (one launch each, asynchronous
// on the given stream). R is double or float; complex fields are Cx<R>.
#pragma once

#include <functional>
#include <string>

#include "common.cuh"

namespace mg {

// message returned by mg_last_error() on this thread
void set_last_error(const std::string &msg);

// one level's operator: the fine Wilson D (wilson) or a coarse stencil Y with N x N blocks
template <typename R>
struct OpDesc {
  bool wilson;
  const Cx<R> *U;
  const Cx<R> *Y;
  Geo2 geo;
  int N;
  double diag;
  const double *shift = nullptr;  // per batched vector: diagonal + shift[v] (null: none)
};

// ---- fused MR smoothing (one launch per iteration) ----
// step = false: Ar_new = A r_old; the launch's block partials of (<Ar_new, r_old>, |Ar_new|^2)
// go to part_out. step = true: alpha = omega <Ar_old, r_old>/|Ar_old|^2 from part_in (the
// previous launch's partials); x (+)= alpha r_old (x_init: x = alpha r_old);
// r_new = r_old - alpha Ar_old; Ar_new = A r_new; partials to part_out. r_new / Ar_new /
// part_out must differ from r_old / Ar_old / part_in. Batched over nvec vectors stored with
// stride n (the level's dofs); part_capacity: entries of type R in each partials buffer.
template <typename R>
int mr_grid(const OpDesc<R> &op);  // blocks of one MR launch per vector
template <typename R>
void launch_mr_iteration(const OpDesc<R> &op, bool step, const Cx<R> *r_old, const Cx<R> *Ar_old, const R *part_in,
                         double omega, Cx<R> *x, bool x_init, Cx<R> *r_new, Cx<R> *Ar_new, R *part_out,
                         long long part_capacity, cudaStream_t s, int nvec = 1);
// x (+)= alpha r_old with alpha from part_in (the last MR launch on `op`); with r_out, also
// the final residual r_out = r_old - alpha Ar_old (r_out may equal r_old)
template <typename R>
void launch_mr_last(const OpDesc<R> &op, const Cx<R> *r_old, const Cx<R> *Ar_old, const R *part_in, double omega,
                    Cx<R> *x, bool x_init, Cx<R> *r_out, long long n, cudaStream_t s, int nvec = 1);

// ---- fine Wilson operator (2d, U(1), gamma_1 = sigma_1, gamma_2 = sigma_2) ----
// out = a * D in + c * b   (b may be null when c == 0); D has diagonal `diag` = d + m,
// plus shift[v] for batched vector v when `shift` (device, nvec doubles) is given
template <typename R>
void launch_dslash(const Cx<R> *U, const Cx<R> *in, Cx<R> *out, Geo2 g, double diag, const Cx<R> *b, double a,
                   double c, cudaStream_t s, int nvec = 1, const double *shift = nullptr);

// ---- fine Wilson operator (4d, SU(3), DeGrand-Rossi gammas) ----
// out = a * D in + c * b on psi[x][4][3], U[x][4][3][3]; diagonal `diag` = 4 + m (+ shift[v])
template <typename R>
void launch_dslash4(const Cx<R> *U, const Cx<R> *in, Cx<R> *out, Geo4 g, double diag, const Cx<R> *b, double a,
                    double c, cudaStream_t s, int nvec = 1, const double *shift = nullptr);
// Ar = D r (FP32, nvec vectors) with each vector's MR sums (Re <Ar, r>, Im <Ar, r>, |Ar|^2) in
// sums[3 v], from the tiled kernel's epilogue (partials: nvec x nsites / 64 x 3 doubles, tickets:
// nvec counters at zero); returns false, launching nothing, where that kernel does not apply
bool launch_dslash4_mr(const Cx<float> *U, const Cx<float> *r, Cx<float> *Ar, Geo4 g, double diag, int nvec,
                       double *sums, double *partials, long long partials_cap, unsigned int *tickets,
                       cudaStream_t s);

// ---- coarse stencil operator, N x N blocks, internal layout Y[j][dir][col][row] ----
// out = a * A in + c * b; with `shift`, vector v sees A + shift[v] * identity
template <typename R>
void launch_coarse_apply(const Cx<R> *Y, const Cx<R> *in, Cx<R> *out, Geo2 g, int N, const Cx<R> *b, double a,
                         double c, cudaStream_t s, int nvec = 1, const double *shift = nullptr);

// ---- coarse stencil apply on tensor cores (N = 8, many vectors, BF16 operands, FP32 sums) ----
// Ypk: nsites * 5 * 32 words packed from the FP32 internal stencil Y (A-fragment order)
void launch_pack_coarse_bf16(const Cx<float> *Y, uint2 *Ypk, long long nsites, cudaStream_t s);
// out_n = a (A + shift_n) in_n + c b_n for nvec vectors stored with stride nsites * 8
// (b and shift may be null)
void launch_coarse_apply_tc(const uint2 *Ypk, const Cx<float> *in, Cx<float> *out, Geo2 g, int nvec,
                            const Cx<float> *b, double a, double c, const double *shift, cudaStream_t s);

// ---- half-precision storage with per-site norms (wilson_half.cu) ----
void launch_dslash_half(const void *U, const void *in, void *out, Geo2 g, double diag, cudaStream_t s);
// fine level of FP32 V-cycles with half storage (MG_FP16 contexts; wilson_half.cu): the fused MR
// iteration and its last step on half r / A r fields (12 V bytes per field of a batch), the
// residual apply on FP32 vectors with half links
int mr_half_grid(Geo2 g);
void launch_mr_iteration_half(const void *U16, Geo2 g, double diag, const double *shift, bool step,
                              const Cx<float> *b, void *r_old, void *Ar_old, const float *part_in, double omega,
                              Cx<float> *x, bool x_init, void *r_new, void *Ar_new, float *part_out,
                              long long part_capacity, cudaStream_t s, int nvec);
void launch_mr_last_half(void *r_old, void *Ar_old, const float *part_in, double omega, Cx<float> *x, bool x_init,
                         Cx<float> *r_out, Geo2 g, cudaStream_t s, int nvec);
void launch_dslash_hl(const void *U16, const Cx<float> *in, Cx<float> *out, Geo2 g, double diag, const Cx<float> *b,
                      double a, double c, cudaStream_t s, int nvec, const double *shift);
void launch_half_convert(int what, int precision, const void *in, void *out, long long nsites, cudaStream_t s);

// ---- outer GCR driven on the device (blas.cu): ctl = {iterations, k, stop reason}, st = {|r|^2
// estimate, tol^2 |b|^2, new estimate, breakdown flag}; the control kernel sets the condition
// of the WHILE graph node that replays one iteration ----
void launch_gcr_dots_devk(const Cx<double> *W, const Cx<double> *w, const Cx<double> *r, const int *ctl, int restart,
                          long long n, double *out, const ReduceWs &ws, cudaStream_t s);
void launch_gcr_update_devk(Cx<double> *W, Cx<double> *Z, const Cx<double> *w, const Cx<double> *z, const int *ctl,
                            const double *dots, double *st, Cx<double> *x, Cx<double> *r, long long n,
                            cudaStream_t s);
void launch_gcr_control(int *ctl, double *st, int restart, int max_iter, cudaGraphConditionalHandle handle,
                        cudaStream_t s);

// batched (nb vectors in lockstep): act[v] iterating flags, stv[2 v] |r_v|^2 estimate and
// stv[2 v + 1] tol^2 |b_v|^2, coef[4 v ..] (inv, alpha, mode); dots stride 2 (restart + 3) per vector
// (VT double or float: the vectors' type; reductions and coefficients in FP64)
template <typename VT>
void launch_copy_active(const Cx<VT> *x, Cx<VT> *y, long long n, int nb, const int *act, cudaStream_t s);
template <typename VT>
void launch_gcr_dots_batch_devk(const Cx<VT> *W, const Cx<VT> *w, const Cx<VT> *r, const int *ctl, int nb,
                                int restart, long long n, double *out, const ReduceWs &ws, cudaStream_t s);
void launch_gcr_coef_batch(const double *dots, const int *ctl, int nb, int restart, int *act, double *stv,
                           double *coef, cudaStream_t s);
template <typename VT>
void launch_gcr_update_batch_devk(Cx<VT> *W, Cx<VT> *Z, const Cx<VT> *w, const Cx<VT> *z, const int *ctl, int nb,
                                  int restart, const double *dots, const double *coef, Cx<VT> *x, Cx<VT> *r,
                                  long long n, cudaStream_t s);
void launch_gcr_control_batch(int *ctl, const int *act, int nb, int restart, int max_iter,
                              cudaGraphConditionalHandle handle, cudaStream_t s);

// ---- autotuner of launch shapes (autotune.cu) ----
// Index of the fastest of `count` launch variants of one kernel for one problem shape, by
// timing each on stream s (one untimed launch, then three timed with CUDA events); cached
// under `key` for the process. Every variant must compute the same result: only the launch
// shape may differ. While s is being captured into a graph an unknown key is not timed and
// variant 0 is returned (uncached).
int autotune_choose(const std::string &key, int count, const std::function<void(int)> &launch, cudaStream_t s);
// "key=variant;..." for every cached choice
std::string autotune_report();

// ---- BLAS-1 ----
template <typename R>
void launch_zero(Cx<R> *x, long long n, cudaStream_t s);
template <typename R>
void launch_copy(const Cx<R> *x, Cx<R> *y, long long n, cudaStream_t s);
template <typename To, typename From>
void launch_convert(const Cx<From> *x, Cx<To> *y, long long n, cudaStream_t s);
// y = x - y (in place on y)
template <typename R>
void launch_xmy(const Cx<R> *x, Cx<R> *y, long long n, cudaStream_t s);

// ---- reductions (deterministic, results in FP64 on the device) ----
// out[0..1] = <a, b> (complex), out[2] = |a|^2
template <typename R>
void launch_dot_norm(const Cx<R> *a, const Cx<R> *b, long long n, double *out, const ReduceWs &ws, cudaStream_t s);
// out[0] = |a|^2
template <typename R>
void launch_norm2(const Cx<R> *a, long long n, double *out, const ReduceWs &ws, cudaStream_t s);
// MR step: alpha = omega <Ar, r>/|Ar|^2 (sc[0..2]); x += alpha r; r -= alpha Ar
template <typename R>
void launch_mr_update(const double *sc, double omega, Cx<R> *x, Cx<R> *r, const Cx<R> *Ar, long long n,
                      cudaStream_t s);

// outer GCR, FP64: out[2j..2j+1] = <W_j, w> (j < k), out[2k] = |w|^2, out[2k+2..2k+3] = <w, r>,
// out[2k+4] = |r|^2
void launch_gcr_dots(const Cx<double> *W, const Cx<double> *w, const Cx<double> *r, int k, long long n, double *out,
                     const ReduceWs &ws, cudaStream_t s);
// the same reductions on FP32 vectors (products and sums in FP64)
void launch_gcr_dots(const Cx<float> *W, const Cx<float> *w, const Cx<float> *r, int k, long long n, double *out,
                     const ReduceWs &ws, cudaStream_t s);
// the same with k = *kdev read by the kernel (a graph-replayed loop; kmax bounds k)
template <typename VT>
void launch_gcr_dots_kdev(const Cx<VT> *W, const Cx<VT> *w, const Cx<VT> *r, const int *kdev, int kmax, long long n,
                          double *out, const ReduceWs &ws, cudaStream_t s);
// w = (w - sum beta_j W_j) inv and z likewise (written to Wk / Zk); then, if update_xr,
// x += alpha z and r -= alpha w. beta_dev: 2k doubles on the device.
void launch_gcr_project_update(const Cx<double> *W, Cx<double> *Wk, const Cx<double> *Z, Cx<double> *Zk, int k,
                               const double *beta_dev, double inv, double are, double aim, Cx<double> *x,
                               Cx<double> *r, long long n, bool update_xr, cudaStream_t s);

// batched outer GCR over nb systems (vector v at v * n; bases W[j][v][n], Z[j][v][n]):
// y_v = mask bit v ? x_v : 0
template <typename VT>
void launch_copy_masked(const Cx<VT> *x, Cx<VT> *y, long long n, int nb, unsigned int mask, cudaStream_t s);
// out[v] = |a_v|^2
template <typename VT>
void launch_norm2_batch(const Cx<VT> *a, long long n, int nb, double *out, const ReduceWs &ws, cudaStream_t s);
// out[v * 2 (k + 3) + 2 j] = <W_j,v, W_k,v> (j < k), then |W_k,v|^2, <W_k,v, r_v> and |r_v|^2
template <typename VT>
void launch_gcr_dots_batch(const Cx<VT> *W, const Cx<VT> *r, int k, int nb, long long n, double *out,
                           const ReduceWs &ws, cudaStream_t s);
// per vector, coef[4 v .. 4 v + 3] = (inv, alpha, mode): mode 0 skip, 2 project W_k / Z_k
// with the betas in dots, 1 project, scale by inv, x += alpha Z_k, r -= alpha W_k
template <typename VT>
void launch_gcr_update_batch(Cx<VT> *W, Cx<VT> *Z, int k, int nb, const double *dots, const double *coef,
                             Cx<VT> *x, Cx<VT> *r, long long n, cudaStream_t s);

// ---- transfer between levels ----
// coarse[b][k] = sum_i conj(V[b][k][i]) fine[site(b,s)][a]
template <typename R>
void launch_restrict(const Cx<R> *V, const Cx<R> *fine, Cx<R> *coarse, BlockGeo bg, int Nv, cudaStream_t s,
                     int nvec = 1);
// fine[site(b,s)][a] += sum_k V[b][k][i] coarse[b][k]
template <typename R>
void launch_prolong_add(const Cx<R> *V, const Cx<R> *coarse, Cx<R> *fine, BlockGeo bg, int Nv, cudaStream_t s,
                        int nvec = 1);
// block Gram-Schmidt (modified, twice, k order) of Nv level vectors into V[b][k][i]; FP64
void launch_block_mgs(const Cx<double> *vecs, long long vec_stride, Cx<double> *V, BlockGeo bg, int Nv,
                      double *min_norm_dev, cudaStream_t s);
// Galerkin coarse operator Yc[b][dir][col][row] (internal layout) of P^dagger A P; FP64 inputs and
// output, arithmetic in FP64 or (fp32_arith, the hierarchies of mixed-precision cycles) FP32
void launch_galerkin_wilson(const Cx<double> *U, double diag, const Cx<double> *V, Cx<double> *Yc, BlockGeo bg,
                            int Nv, cudaStream_t s, bool fp32_arith = false);
void launch_galerkin_stencil(const Cx<double> *Y, const Cx<double> *V, Cx<double> *Yc, BlockGeo bg, int Nv,
                             cudaStream_t s, bool fp32_arith = false);

// ---- layout conversions at the boundary ----
// internal Y[j][dir][col][row] <-> canonical Y[j][dir][row][col]
void launch_coarse_to_canonical(const Cx<double> *Yi, Cx<double> *Yc, long long nsites, int N, cudaStream_t s);
// P columns: internal V[b][k][i] -> canonical v[k][site][a]
void launch_prolongator_to_canonical(const Cx<double> *V, Cx<double> *out, BlockGeo bg, int Nv, cudaStream_t s);

// ---- random vectors: Philox4x32-10 + Box-Muller, counter (i lo, i hi, k, level) ----
void launch_gaussian(Cx<double> *out, long long n, unsigned long long seed, int k, int level, cudaStream_t s);

// ---- coarsest level: dense LU with partial pivoting, column-major ----
// dense matrix of the stencil plus shift * identity
void launch_dense_from_stencil(const Cx<double> *Y, Cx<double> *A, Geo2 g, int N, cudaStream_t s, double shift = 0.0);
// factor in place; ipiv[k] = pivot row of step k; info_dev[0] = 1 + first zero pivot (0 if none)
void lu_factor(Cx<double> *A, int n, int *ipiv, int *info_dev, cudaStream_t s);
// x = A^{-1} b with the factors; work: n entries, must alias neither b nor x (b may equal work)
void lu_solve_ws(const Cx<double> *LU, const int *ipiv, int n, const Cx<double> *b, Cx<double> *x, Cx<double> *work,
                 cudaStream_t s);

// ---- coarsest level: restarted GCR as one persistent cooperative kernel (FP64) ----
// Preparation for A = Y + shift * identity: Minv[j] = (X_j + shift)^{-1} (self blocks) and,
// unless Yt is null, Yt = stencil of A M, M = blockdiag(Minv); work: nsites * 2 N^2 entries;
// info_dev[0] = 1 if a self block is singular.
void prepare_coarsest_gcr(const Cx<double> *Y, Geo2 g, int N, Cx<double> *Minv, Cx<double> *Yt, Cx<double> *work,
                          int *info_dev, cudaStream_t s, double shift = 0.0);
// x = A^{-1} b to relative true residual tol (GCR on A M y = b, x = M y); y, r: n entries;
// Z/W: restart * n each (restart <= 32); partials: grid * kCoarsestSlots doubles; bar: 2 uints;
// out[0] += iterations, out[1] = 1 on a barrier timeout, out[2] += 1 if the tolerance was missed.
void launch_coarsest_gcr(const Cx<double> *Yt, const Cx<double> *Minv, Geo2 g, int N, const Cx<double> *b,
                         Cx<double> *x, Cx<double> *y, Cx<double> *r, Cx<double> *Z, Cx<double> *W, double *partials,
                         unsigned int *bar, double tol, int restart, int max_iter, int *out, double *out_rel, int grid,
                         cudaStream_t s);
int coarsest_gcr_grid(int device);
// bounded-barrier self-test (2 CTAs, `expected` arrivals); returns 1 if a wait gave up
// cooperative launches and graphs holding them: serialised per device (see coarsest.cu)
void coop_launch(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t s);
bool coop_captured_take();  // a cooperative kernel was captured on this thread since the last call
void coop_graph_launch(cudaGraphExec_t g, cudaStream_t s);
int barrier_selftest(unsigned int expected, long long spin_limit, cudaStream_t s);
constexpr int kCoarsestSlots = 68;
// Same solve with each CTA's rows, vectors and Krylov basis resident in shared memory
// (N = 8, restart <= 16, at most 64 dofs per CTA when spread over `sms` CTAs): rpub, ypub
// are n-entry publication buffers for the neighbours' reads; 2 grid barriers per iteration.
// With Yt32 (an FP32 copy of A M) the stencil is stored and applied in FP32 while the Krylov
// vectors, Gram-Schmidt, residuals and updates stay FP64.
// FP32 variant of launch_coarsest_gcr (stencil A M and Krylov vectors in FP32, every reduction
// summed in FP64) for mixed-precision cycles with a loose coarsest tolerance
void launch_coarsest_gcr32(const Cx<float> *Yt, const Cx<double> *Minv, Geo2 g, int N, const Cx<double> *b,
                           Cx<double> *x, Cx<float> *y, Cx<float> *r, Cx<float> *Z, Cx<float> *W, double *partials,
                           unsigned int *bar, double tol, int restart, int max_iter, int *out, double *out_rel,
                           int grid, cudaStream_t s);
bool coarsest_smem_fits(Geo2 g, int N, int restart, int sms);
void launch_coarsest_gcr_smem(const Cx<double> *Yt, const Cx<float> *Yt32, const Cx<double> *Minv, Geo2 g,
                              const Cx<double> *b, Cx<double> *x, Cx<double> *rpub, Cx<double> *ypub,
                              double *partials, unsigned int *bar, double tol, int restart, int max_iter, int *out,
                              double *out_rel, int sms, cudaStream_t s);

// One-cluster variant (coarsest_cluster.cu) for mixed-precision cycles with a loose tolerance:
// FP32 GCR on A M (Yt32, row-major blocks) with FP64 cross-warp / cross-CTA sums, 16 CTAs of one thread-block
// cluster per vector (nvec clusters in one launch, vector v at offset v n of b, x and of the
// FP32 publication buffers rpub, ypub of nvec n entries each); N = 8, at most 8192 dofs.
bool coarsest_cluster_fits(Geo2 g, int N, int restart);
// the cluster kernel reads A M as row-major 8 x 8 blocks: [j][dir][col][row] -> [j][dir][row][col]
void launch_transpose_blocks8(const Cx<float> *in, Cx<float> *out, long long nblocks, cudaStream_t s);
void launch_coarsest_gcr_cluster(const Cx<float> *Yt32, const Cx<double> *Minv, Geo2 g, int nvec,
                                 const Cx<double> *b, Cx<double> *x, Cx<float> *rpub, Cx<float> *ypub, double tol,
                                 int restart, int max_iter, int *out, double *out_rel, cudaStream_t s);

// Batched variant: nb <= 4 right-hand sides in one launch, vector v solving
// (Y + shift[v]) x_v = b_v (shift: device, null for none) with M_v = Minv + v * minv_stride
// (minv_stride 0: one preconditioner for all); Y is the raw stencil. b, x, upub, xpub hold
// nb vectors of n; partials: kBatchPartials(grid) doubles; out / out_rel as above (out[0]
// adds the iterations of every vector, out_rel[0] the largest relative residual).
bool coarsest_batch_fits(Geo2 g, int N, int restart, int sms);
constexpr int kCoarsestBatchVecs = 4;
inline long long coarsest_batch_partials(int grid) { return 4LL * (2 * 16 + 4) * grid; }
void launch_coarsest_gcr_batch(const Cx<double> *Y, const Cx<double> *Minv, long long minv_stride,
                               const double *shift, Geo2 g, int nb, const Cx<double> *b, Cx<double> *x,
                               Cx<double> *upub, Cx<double> *xpub, double *partials, unsigned int *bar, double tol,
                               int restart, int max_iter, int *out, double *out_rel, int sms, cudaStream_t s);

}  // namespace mg
