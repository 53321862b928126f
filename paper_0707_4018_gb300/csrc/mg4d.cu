// Engine of the 4d SU(3) two-level adaptive multigrid (paper: the adaptive
// setup with Eq. relax and Eq. P1, Eq. Galerkin, the five V-cycle steps with
// an exact coarse solve; the four-dimensional case of its outlook).
//
//   setup: Nv Gaussian vectors (Philox, keyed by seed, vector, dof) relaxed by
//          nu_setup MR iterations on D v = 0; split by chirality
//          ((1 +- gamma_5) / 2, 2 Nv coarse dofs); block Gram-Schmidt (FP64);
//          Galerkin P^dagger D P (FP64); passes 2..n_pass: v <- v - V(D v).
//   V-cycle (FP64, or FP32 for MG_FP32): MR pre-smoothing from 0, residual,
//          restriction, coarse solve (FP64 GCR to coarsest_tol, right-
//          preconditioned by the inverses of the coarse self blocks; the
//          operator applied in FP32 for MG_FP32), prolongation and correction,
//          residual, MR post-smoothing. MG_FP32 also relaxes the setup vectors
//          in FP32.
//   solve: FP64 flexible GCR with the V-cycle as right preconditioner and the
//          true residual at every restart.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include <cstdlib>

#include "mg4d.h"

namespace mg {

struct Engine4 {
  mg_geom geom{};
  mg_params p{};
  double m = 0.0;
  cudaStream_t s = nullptr;
  bool f32 = false;
  Geo4 fg{};
  Block4 bg{};
  Coarse4 cg{};
  long long nf = 0, nc = 0;  // fine / coarse dofs
  int N = 0;
  DevBuf<Cx<double>> U64, nullv, V64, Y64, Minv64, Yt64;  // Yt: A M, the preconditioned stencil
  DevBuf<Cx<float>> U32, V32, Yt32, Minv32;
  // A M in FP16 for the single-vector coarse GCR when its tolerance is loose (>= 0.05)
  DevBuf<unsigned int> Yth;
  DevBuf<int> info;  // set by the block inversion when a self block is singular
  // multi-vector coarse apply (made on first use after each Galerkin build): BF16 tensor-core
  // fragments and an FP32 copy of Y
  DevBuf<uint4> Ypk4, Ypk4lo;  // Ypk4lo: the low BF16 part, for the split-operator apply
  DevBuf<Cx<float>> Y32;
  bool mrhs_ready = false;
  // V-cycle work
  DevBuf<Cx<double>> vr64, vAr64, vx64, vb64;
  DevBuf<Cx<float>> vr32, vAr32, vx32, vb32;
  DevBuf<Cx<double>> cb, cx, cy;  // coarse right-hand side / solution / preconditioned solution (FP64)
  DevBuf<Cx<float>> cb32, cx32;
  DevBuf<Cx<double>> cZ, cW, cr;  // coarse GCR
  DevBuf<Cx<float>> cZ32, cW32, cr32, cy32;  // coarse GCR on FP32 vectors (MG_FP32, loose coarsest_tol)
  // the same GCR replayed by a graph (a WHILE node over iterations, one launch per restart
  // cycle): its counters, the operator output and the instantiated graph with the buffers
  // it was captured on
  DevBuf<int> cctl;
  DevBuf<Cx<float>> cwt32;
  cudaGraphExec_t cloop = nullptr;
  std::vector<const void *> cloop_key;
  DevBuf<Cx<double>> oZ, oW, orr, t64;  // outer GCR, setup scratch
  DevBuf<double> partials, scal;
  DevBuf<unsigned int> tickets;
  // batched MR reductions (setup relaxation of the Nv vectors, V-cycle MR): per-vector
  // partials, tickets and (<Ar, r>, |Ar|^2) sums
  DevBuf<double> bpart, bsc;
  DevBuf<unsigned int> btickets;
  DevBuf<Cx<float>> sx32, sr32, sAr32;  // setup relaxation batch (MG_FP32)
  DevBuf<Cx<double>> sr64, sAr64;       // setup relaxation batch (MG_FP64; x is the vector set itself)
  ReduceWs ws{};
  ReduceWs wsc{};  // the same workspace with fewer blocks per reduction (coarse vectors are short)
  double *host = nullptr;  // pinned: [0, 256) outer, [256, 512) coarse
  long long apps[MG_MAX_LEVELS] = {0, 0, 0, 0};
  long long coarsest_iters = 0;
  // batched solves (made on the first batched call, for max_rhs vectors): outer Krylov bases
  // [k][v][nf] and residuals, V-cycle vectors [v][nf], coarse GCR vectors [v][nc] and bases
  // [k][v][nc], FP32 operands of the tensor-core coarse apply, reductions and coefficients
  struct Batch {
    int cap = 0;
    DevBuf<Cx<double>> Z, W, r, rin, z64;
    DevBuf<Cx<float>> r32, Ar32, x32, b32;
    DevBuf<Cx<double>> r64, Ar64, x64, b64;
    DevBuf<Cx<double>> cb, cx, cr, crin, cZ, cW;
    DevBuf<Cx<float>> cin32, cout32;
    DevBuf<Cx<float>> cb32, cx32, cr32, crin32, cZ32, cW32;  // coarse GCR on FP32 vectors
    // its iterations replayed by a graph: preconditioned and operator outputs, counters, active
    // flags, estimates, |b|^2 and |r|^2 per vector, the graph and what it was captured for
    DevBuf<Cx<float>> czt32, cwt32;
    DevBuf<int> cctl, cact;
    DevBuf<double> cstv, cnorm;
    cudaGraphExec_t loop = nullptr;
    std::vector<const void *> loop_key;
    DevBuf<double> dots, coef, cdots, ccoef, part;
    DevBuf<unsigned int> tickets;
    ReduceWs ws{};
    ReduceWs wsc{};  // the same workspace with few blocks per reduction, for the short coarse vectors
    double *host = nullptr, *chost = nullptr;  // pinned: dots, then coefficients (outer / coarse)
  } bt;
  ~Engine4() {
    if (s) cudaStreamSynchronize(s);
    if (cloop) cudaGraphExecDestroy(cloop);
    if (bt.loop) cudaGraphExecDestroy(bt.loop);
    if (host) cudaFreeHost(host);
    if (bt.host) cudaFreeHost(bt.host);
    if (bt.chost) cudaFreeHost(bt.chost);
  }
};

namespace {

constexpr int kScalOuter = 0, kScalCoarse = 256, kScalMr = 512, kScalCount = 640;

double diag4(const Engine4 &e) { return 4.0 + e.m; }

template <typename R>
const Cx<R> *U_of(const Engine4 &e);
template <>
const Cx<double> *U_of<double>(const Engine4 &e) { return e.U64.p; }
template <>
const Cx<float> *U_of<float>(const Engine4 &e) { return e.U32.p; }
template <typename R>
const Cx<R> *V_of(const Engine4 &e);
template <>
const Cx<double> *V_of<double>(const Engine4 &e) { return e.V64.p; }
template <>
const Cx<float> *V_of<float>(const Engine4 &e) { return e.V32.p; }

// out = a D in + c b on the fine lattice
template <typename R>
void fine_apply(Engine4 &e, const Cx<R> *in, Cx<R> *out, const Cx<R> *b = nullptr, double a = 1.0, double c = 0.0) {
  launch_dslash4<R>(U_of<R>(e), in, out, e.fg, diag4(e), b, a, c, e.s);
  ++e.apps[0];
}

// out = a A_c in + c b on FP64 vectors
void coarse_apply64(Engine4 &e, const Cx<double> *in, Cx<double> *out, const Cx<double> *b = nullptr, double a = 1.0,
                    double c = 0.0) {
  launch_coarse4_apply<double, double>(e.Y64.p, in, out, e.cg, b, a, c, e.s);
  ++e.apps[1];
}

struct Gcr {
  int iters = 0;
  bool converged = false;
  double rel = 0.0;
};

// Flexible GCR (FP64) for A x = b with right preconditioner z = M r; x starts at 0.
// Classical Gram-Schmidt coefficients from one fused reduction, a second projection
// when |w - W beta|^2 shows cancellation, the residual norm |r|^2 - |alpha|^2 from a
// fresh |r|^2, and the true residual b - A x at every restart.
template <typename ApplyF, typename PrecF>
Gcr fgcr(Engine4 &e, ApplyF &&apply, PrecF &&prec, const Cx<double> *b, Cx<double> *x, long long n, double tol,
         int restart, int max_iter, Cx<double> *Z, Cx<double> *W, Cx<double> *r, int slot) {
  double *dots = e.scal.p + slot;
  double *h = e.host + slot;
  Gcr out;
  auto fetch = [&](int count) {
    MG_CUDA(cudaMemcpyAsync(h, dots, count * sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    for (int i = 0; i < count; ++i)
      if (std::isnan(h[i])) fail(MG_ERR_NAN, "GCR: NaN in a reduction");
  };
  launch_zero<double>(x, n, e.s);
  launch_copy<double>(b, r, n, e.s);
  launch_norm2<double>(b, n, dots, e.ws, e.s);
  fetch(1);
  const double bn2 = h[0];
  if (!(bn2 > 0.0)) {
    out.converged = true;
    return out;
  }
  double rel = 1.0;
  while (out.iters < max_iter) {
    int k = 0;
    for (; k < restart && out.iters < max_iter; ++k) {
      Cx<double> *z = Z + (long long)k * n, *w = W + (long long)k * n;
      prec(r, z);
      apply(z, w);
      launch_gcr_dots(W, w, r, k, n, dots, e.ws, e.s);
      fetch(2 * (k + 3));
      const double rr = h[2 * k + 4];
      double nw0 = h[2 * k], nw2 = nw0;
      for (int j = 0; j < k; ++j) nw2 -= h[2 * j] * h[2 * j] + h[2 * j + 1] * h[2 * j + 1];
      double wr = h[2 * k + 2], wi = h[2 * k + 3];
      if (k > 0 && !(nw2 > 0.5 * nw0)) {
        launch_gcr_project_update(W, w, Z, z, k, dots, 1.0, 0.0, 0.0, x, r, n, false, e.s);
        launch_gcr_dots(W, w, r, k, n, dots, e.ws, e.s);
        fetch(2 * (k + 3));
        nw0 = h[2 * k];
        nw2 = nw0;
        for (int j = 0; j < k; ++j) nw2 -= h[2 * j] * h[2 * j] + h[2 * j + 1] * h[2 * j + 1];
        wr = h[2 * k + 2];
        wi = h[2 * k + 3];
      }
      if (!(nw2 > 1e-28 * nw0)) break;
      const double inv = 1.0 / std::sqrt(nw2);
      const double are = wr * inv, aim = wi * inv;
      launch_gcr_project_update(W, w, Z, z, k, dots, inv, are, aim, x, r, n, true, e.s);
      ++out.iters;
      rel = std::sqrt(std::max(rr - (are * are + aim * aim), 0.0) / bn2);
      if (rel <= tol) {
        ++k;
        break;
      }
    }
    apply(x, r, b);  // r = b - A x
    launch_norm2<double>(r, n, dots, e.ws, e.s);
    fetch(1);
    rel = std::sqrt(h[0] / bn2);
    if (rel <= tol) {
      out.converged = true;
      break;
    }
    if (k == 0) break;
  }
  out.rel = rel;
  return out;
}

// coarse solve: cx = A_c^{-1} cb by GCR to coarsest_tol on A M y = b, x = M y, with M the
// inverses of the coarse self blocks (block Jacobi) folded into the stencil A M. The
// Gram-Schmidt coefficients are formed on the device, so the host reads the residual
// estimate only every 4 iterations. With MG_FP32 and a tolerance FP32 arithmetic can reach
// (>= 1e-5), the stencil and M are applied from their FP32 copies; the Krylov vectors
// and reductions stay FP64.
// coarse solve on FP32 vectors: cx32 = A_c^{-1} cb32 by the GCR below with the FP32 stencil A M,
// FP32 Krylov vectors and updates, and every reduction in FP64 (MG_FP32 with a coarsest
// tolerance FP32 arithmetic can reach, >= 1e-5: the FP64 Gram-Schmidt over up to 64 basis
// vectors, at 1/74 of the FP32 rate, was most of an iteration's time)
// out = A M in (rhs: out = rhs - A M in) on FP32 vectors, with the FP16 operator when there is one
static void apply_coarse32(Engine4 &e, const Cx<float> *in, Cx<float> *out, const Cx<float> *rhs) {
  if (e.Yth.p != nullptr)
    launch_coarse4_apply_h(e.Yth.p, in, out, e.cg, rhs, rhs ? -1.0 : 1.0, rhs ? 1.0 : 0.0, e.s);
  else
    launch_coarse4_apply<float, float>(e.Yt32.p, in, out, e.cg, rhs, rhs ? -1.0 : 1.0, rhs ? 1.0 : 0.0, e.s);
}

// The coarse GCR of coarse_solve32 with its iterations on the device: one graph per engine, a
// cycle-start kernel and a WHILE node whose body is one iteration (operator, reduction, step,
// control), captured once and launched once per restart cycle. The estimate is checked after
// every iteration (the host-driven loop reads it every kCheck iterations).
constexpr int kCoarseLoopMaxRestart = 99;  // 2 (restart + 3) dots and the state fit the coarse slots

static bool coarse_loop_enabled(const Engine4 &e) {
  return e.cwt32.p != nullptr && e.p.coarsest_restart <= kCoarseLoopMaxRestart &&
         std::getenv("MG_COARSE4_HOST_LOOP") == nullptr;
}

static cudaGraphExec_t coarse_loop_graph(Engine4 &e) {
  double *dots = e.scal.p + kScalCoarse, *st = dots + 204;
  const std::vector<const void *> key = {e.Yt32.p, e.Yth.p, e.cr32.p, e.cy32.p, e.cZ32.p, e.cW32.p, e.cwt32.p, e.cctl.p,
                                         dots, e.wsc.partials, e.wsc.ticket,
                                         reinterpret_cast<const void *>((long long)e.p.coarsest_restart),
                                         reinterpret_cast<const void *>((long long)e.p.coarsest_max_iter)};
  if (e.cloop != nullptr && key == e.cloop_key) return e.cloop;
  if (e.cloop != nullptr) {
    MG_CUDA(cudaGraphExecDestroy(e.cloop));
    e.cloop = nullptr;
  }
  const long long n = e.nc;
  const int restart = e.p.coarsest_restart, max_iter = e.p.coarsest_max_iter;
  const double tol2_rel = e.p.coarsest_tol * e.p.coarsest_tol;
  cudaGraph_t top = nullptr;
  MG_CUDA(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle h;
    MG_CUDA(cudaGraphConditionalHandleCreate(&h, top, 0, cudaGraphCondAssignDefault));
    MG_CUDA(cudaStreamBeginCaptureToGraph(e.s, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_coarse4_cycle_start(e.cctl.p, st, max_iter, h, e.s);
    MG_CUDA(cudaStreamEndCapture(e.s, &top));
    size_t count = 1;
    cudaGraphNode_t start;
    MG_CUDA(cudaGraphGetNodes(top, &start, &count));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MG_CUDA(cudaGraphAddNode(&node, top, &start, nullptr, 1, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    MG_CUDA(cudaStreamBeginCaptureToGraph(e.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    apply_coarse32(e, e.cr32.p, e.cwt32.p, nullptr);
    launch_gcr_dots_kdev<float>(e.cW32.p, e.cwt32.p, e.cr32.p, e.cctl.p + 1, restart - 1, n, dots, e.wsc, e.s);
    launch_gcr_update_loop(e.cW32.p, e.cZ32.p, e.cwt32.p, e.cctl.p, dots, st, e.cy32.p, e.cr32.p, n, e.s);
    launch_coarse4_control(e.cctl.p, st, tol2_rel, restart, max_iter, h, e.s);
    MG_CUDA(cudaStreamEndCapture(e.s, &body));
    MG_CUDA(cudaGraphInstantiate(&e.cloop, top, 0));
  } catch (...) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t partial = nullptr;
    if (cudaStreamIsCapturing(e.s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(e.s, &partial);  // a graph owned by top (or top itself)
    cudaGetLastError();
    cudaGraphDestroy(top);
    throw;
  }
  cudaGraphDestroy(top);
  e.cloop_key = key;
  return e.cloop;
}

static long long coarse_solve32_loop(Engine4 &e) {
  const long long n = e.nc;
  Cx<float> *x = e.cy32.p, *r = e.cr32.p;
  const Cx<float> *b = e.cb32.p;
  double *st = e.scal.p + kScalCoarse + 204, *h = e.host + kScalCoarse + 204;
  cudaGraphExec_t g = coarse_loop_graph(e);
  launch_zero<float>(x, n, e.s);
  launch_copy<float>(b, r, n, e.s);
  launch_norm2<float>(b, n, st + 1, e.wsc, e.s);
  MG_CUDA(cudaMemsetAsync(e.cctl.p, 0, 2 * sizeof(int), e.s));
  MG_CUDA(cudaMemsetAsync(st + 3, 0, sizeof(double), e.s));
  const double tol2_rel = e.p.coarsest_tol * e.p.coarsest_tol;
  long long iters = 0;
  for (;;) {
    MG_CUDA(cudaGraphLaunch(g, e.s));
    apply_coarse32(e, x, r, b);  // true residual
    launch_norm2<float>(r, n, st + 2, e.wsc, e.s);
    MG_CUDA(cudaMemcpyAsync(h + 1, st + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    if (std::isnan(h[1]) || std::isnan(h[2])) fail(MG_ERR_NAN, "coarse GCR: NaN in a reduction");
    const long long it = (long long)h[3];
    e.apps[1] += it - iters + 1;
    iters = it;
    if (!(h[1] > 0.0) || h[2] <= tol2_rel * h[1] || iters >= e.p.coarsest_max_iter) break;
  }
  launch_block_apply4_32(e.Minv32.p, x, e.cx32.p, e.cg, e.s);  // x = M y
  e.coarsest_iters += iters;
  return iters;
}

long long coarse_solve32(Engine4 &e) {
  if (coarse_loop_enabled(e)) return coarse_solve32_loop(e);
  const long long n = e.nc;
  Cx<float> *x = e.cy32.p, *r = e.cr32.p, *Z = e.cZ32.p, *W = e.cW32.p;
  const Cx<float> *b = e.cb32.p;
  auto apply = [&](const Cx<float> *in, Cx<float> *out, const Cx<float> *rhs = nullptr) {
    apply_coarse32(e, in, out, rhs);
    ++e.apps[1];
  };
  double *dots = e.scal.p + kScalCoarse, *state = dots + 204;
  double *h = e.host + kScalCoarse;
  auto fetch = [&](const double *src) {
    MG_CUDA(cudaMemcpyAsync(h, src, sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    if (std::isnan(h[0])) fail(MG_ERR_NAN, "coarse GCR: NaN in a reduction");
    return h[0];
  };
  launch_zero<float>(x, n, e.s);
  launch_copy<float>(b, r, n, e.s);
  launch_norm2<float>(b, n, dots, e.wsc, e.s);
  const double bn2 = fetch(dots);
  long long iters = 0;
  if (bn2 > 0.0) {
    const double tol2 = e.p.coarsest_tol * e.p.coarsest_tol * bn2;
    const int restart = e.p.coarsest_restart, max_iter = e.p.coarsest_max_iter;
    constexpr int kCheck = 4;
    while (iters < max_iter) {
      int k = 0;
      for (; k < restart && iters < max_iter; ++k) {
        Cx<float> *z = Z + (long long)k * n, *w = W + (long long)k * n;
        launch_copy<float>(r, z, n, e.s);
        apply(z, w);
        launch_gcr_dots(W, w, r, k, n, dots, e.wsc, e.s);
        launch_gcr_update_dev(W, w, Z, z, k, dots, state, x, r, n, e.s);
        ++iters;
        if ((k + 1) % kCheck == 0 && fetch(state) <= tol2) {
          ++k;
          break;
        }
      }
      apply(x, r, b);  // true residual
      launch_norm2<float>(r, n, dots, e.wsc, e.s);
      if (fetch(dots) <= tol2) break;
    }
  }
  launch_block_apply4_32(e.Minv32.p, x, e.cx32.p, e.cg, e.s);  // x = M y
  e.coarsest_iters += iters;
  return iters;
}

long long coarse_solve(Engine4 &e) {
  const bool fast = e.f32 && e.p.coarsest_tol >= 1e-5;
  if (fast && std::getenv("MG_COARSE4_FP64_VECTORS") == nullptr) {  // FP64 in, FP64 out, FP32 inside
    launch_convert<float, double>(e.cb.p, e.cb32.p, e.nc, e.s);
    const long long it = coarse_solve32(e);
    launch_convert<double, float>(e.cx32.p, e.cx.p, e.nc, e.s);
    return it;
  }
  auto apply = [&](const Cx<double> *in, Cx<double> *out, const Cx<double> *b = nullptr) {
    if (fast)
      launch_coarse4_apply<float, double>(e.Yt32.p, in, out, e.cg, b, b ? -1.0 : 1.0, b ? 1.0 : 0.0, e.s);
    else
      launch_coarse4_apply<double, double>(e.Yt64.p, in, out, e.cg, b, b ? -1.0 : 1.0, b ? 1.0 : 0.0, e.s);
    ++e.apps[1];
  };
  const long long n = e.nc;
  Cx<double> *x = e.cy.p, *r = e.cr.p, *Z = e.cZ.p, *W = e.cW.p;
  const Cx<double> *b = e.cb.p;
  double *dots = e.scal.p + kScalCoarse, *state = dots + 204;
  double *h = e.host + kScalCoarse;
  auto fetch = [&](const double *src) {
    MG_CUDA(cudaMemcpyAsync(h, src, sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    if (std::isnan(h[0])) fail(MG_ERR_NAN, "coarse GCR: NaN in a reduction");
    return h[0];
  };
  launch_zero<double>(x, n, e.s);
  launch_copy<double>(b, r, n, e.s);
  launch_norm2<double>(b, n, dots, e.wsc, e.s);
  const double bn2 = fetch(dots);
  long long iters = 0;
  if (bn2 > 0.0) {
    const double tol2 = e.p.coarsest_tol * e.p.coarsest_tol * bn2;
    const int restart = e.p.coarsest_restart, max_iter = e.p.coarsest_max_iter;
    constexpr int kCheck = 4;  // iterations between host reads of the residual estimate
    while (iters < max_iter) {
      int k = 0;
      for (; k < restart && iters < max_iter; ++k) {
        Cx<double> *z = Z + (long long)k * n, *w = W + (long long)k * n;
        launch_copy<double>(r, z, n, e.s);
        apply(z, w);
        launch_gcr_dots(W, w, r, k, n, dots, e.wsc, e.s);
        launch_gcr_update_dev(W, w, Z, z, k, dots, state, x, r, n, e.s);
        ++iters;
        if ((k + 1) % kCheck == 0 && fetch(state) <= tol2) {
          ++k;
          break;
        }
      }
      apply(x, r, b);  // true residual
      launch_norm2<double>(r, n, dots, e.wsc, e.s);
      if (fetch(dots) <= tol2) break;
    }
  }
  // x = M y
  if (fast)
    launch_block_apply4<float>(e.Minv32.p, x, e.cx.p, e.cg, e.s);
  else
    launch_block_apply4<double>(e.Minv64.p, x, e.cx.p, e.cg, e.s);
  e.coarsest_iters += iters;
  return iters;
}

// Flexible GCR over nb systems in lockstep (FP64, vectors [v][n], bases [k][v][n]): one
// batched preconditioner, one batched operator apply and one batched reduction per
// iteration; the host forms every vector's coefficients from one fetch, with a second
// projection where |w - W beta|^2 <= reproject |w|^2 shows cancellation (reproject 0: only
// where nothing is left, as the one-pass single-vector coarse GCR). A vector whose tracked residual meets
// tol (or whose basis breaks down) rests until the next restart, where the true residuals
// decide which vectors go on; a resting vector's preconditioner input is zero.
struct GcrB {
  int iters = 0;
  bool converged = false;
  double rel = 0.0;
};

// VT: the vectors' precision (FP64; FP32 for the inexact coarse solves of mixed-precision
// cycles, with every reduction and coefficient in FP64)
template <typename VT, typename ApplyF, typename PrecF>
void fgcr_batch(Engine4 &e, int nb, ApplyF &&apply, PrecF &&prec, const Cx<VT> *b, Cx<VT> *x, long long n,
                double tol, int restart, int max_iter, Cx<VT> *Z, Cx<VT> *W, Cx<VT> *r, Cx<VT> *rin, double *dots,
                double *coef, double *h, const ReduceWs &ws, std::vector<GcrB> &out, double reproject = 0.5) {
  double *hcoef = h + (size_t)nb * 2 * (restart + 3);
  out.assign(nb, GcrB{});
  auto fetch = [&](int count) {
    MG_CUDA(cudaMemcpyAsync(h, dots, count * sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    for (int i = 0; i < count; ++i)
      if (std::isnan(h[i])) fail(MG_ERR_NAN, "GCR (batched): NaN in a reduction");
  };
  launch_zero<VT>(x, n * nb, e.s);
  launch_copy<VT>(b, r, n * nb, e.s);
  launch_norm2_batch(b, n, nb, dots, ws, e.s);
  fetch(nb);
  std::vector<double> bn2(h, h + nb), rn2(bn2), nw0(nb), nw2(nb), wr(nb), wi(nb), rr(nb);
  const unsigned int all = nb == 32 ? 0xffffffffu : (1u << nb) - 1u;
  unsigned int done = 0u;
  for (int v = 0; v < nb; ++v)
    if (!(bn2[v] > 0.0)) {
      done |= 1u << v;
      out[v].converged = true;
    }
  int iters = 0;
  while (done != all && iters < max_iter) {
    unsigned int act = all & ~done;
    int k = 0;
    for (; k < restart && iters < max_iter && act != 0u; ++k) {
      Cx<VT> *Zk = Z + (long long)k * nb * n, *Wk = W + (long long)k * nb * n;
      launch_copy_masked(r, rin, n, nb, act, e.s);
      prec(rin, Zk);
      apply(Zk, Wk, nullptr);
      launch_gcr_dots_batch(W, r, k, nb, n, dots, ws, e.s);
      const int stride = 2 * (k + 3);
      fetch(nb * stride);
      unsigned int cancel = 0u;
      for (int v = 0; v < nb; ++v) {
        const double *hv = h + v * stride;
        rr[v] = hv[2 * k + 4];
        nw0[v] = nw2[v] = hv[2 * k];
        for (int j = 0; j < k; ++j) nw2[v] -= hv[2 * j] * hv[2 * j] + hv[2 * j + 1] * hv[2 * j + 1];
        wr[v] = hv[2 * k + 2];
        wi[v] = hv[2 * k + 3];
        if (((act >> v) & 1u) && k > 0 && !(nw2[v] > reproject * nw0[v])) cancel |= 1u << v;
      }
      if (cancel != 0u) {  // project those vectors once, then take fresh coefficients for them
        for (int v = 0; v < nb; ++v) {
          hcoef[4 * v] = 1.0;
          hcoef[4 * v + 1] = hcoef[4 * v + 2] = 0.0;
          hcoef[4 * v + 3] = ((cancel >> v) & 1u) ? 2.0 : 0.0;
        }
        MG_CUDA(cudaMemcpyAsync(coef, hcoef, 4 * nb * sizeof(double), cudaMemcpyHostToDevice, e.s));
        launch_gcr_update_batch(W, Z, k, nb, dots, coef, x, r, n, e.s);
        launch_gcr_dots_batch(W, r, k, nb, n, dots, ws, e.s);
        fetch(nb * stride);
        for (int v = 0; v < nb; ++v) {
          if (!((cancel >> v) & 1u)) continue;
          const double *hv = h + v * stride;
          nw0[v] = nw2[v] = hv[2 * k];
          for (int j = 0; j < k; ++j) nw2[v] -= hv[2 * j] * hv[2 * j] + hv[2 * j + 1] * hv[2 * j + 1];
        }
      }
      for (int v = 0; v < nb; ++v) {
        hcoef[4 * v + 3] = 0.0;
        if (!((act >> v) & 1u)) continue;
        if (!(nw2[v] > 1e-28 * nw0[v])) {
          act &= ~(1u << v);  // breakdown: this vector waits for the restart
          continue;
        }
        const double inv = 1.0 / std::sqrt(nw2[v]);
        const double are = wr[v] * inv, aim = wi[v] * inv;
        hcoef[4 * v] = inv;
        hcoef[4 * v + 1] = are;
        hcoef[4 * v + 2] = aim;
        hcoef[4 * v + 3] = 1.0;
        rn2[v] = std::max(rr[v] - (are * are + aim * aim), 0.0);
        ++out[v].iters;
        if (std::sqrt(rn2[v] / bn2[v]) <= tol) act &= ~(1u << v);
      }
      MG_CUDA(cudaMemcpyAsync(coef, hcoef, 4 * nb * sizeof(double), cudaMemcpyHostToDevice, e.s));
      launch_gcr_update_batch(W, Z, k, nb, dots, coef, x, r, n, e.s);
      ++iters;
    }
    apply(x, r, b);  // true residuals r = b - A x
    launch_norm2_batch(r, n, nb, dots, ws, e.s);
    fetch(nb);
    for (int v = 0; v < nb; ++v) {
      if ((done >> v) & 1u) continue;
      out[v].rel = std::sqrt(h[v] / bn2[v]);
      if (out[v].rel <= tol) {
        done |= 1u << v;
        out[v].converged = true;
      }
    }
    if (k == 0) break;
  }
}

constexpr int kMrBlocks = 152 * 4;  // grid cap of the batched MR reductions

// x (+)= nu MR iterations on D e = r for nvec vectors (stride nf; r updated to the
// recurrence residual); the reductions are summed in the vectors' precision
template <typename R>
void mr_fine(Engine4 &e, Cx<R> *x, Cx<R> *r, Cx<R> *Ar, int nu, int nvec = 1) {
  for (int it = 0; it < nu; ++it) {
    e.apps[0] += nvec;
    if constexpr (sizeof(R) == 4) {
      // the tiled FP32 apply forms the MR sums in its epilogue (no second pass over r and A r)
      if (launch_dslash4_mr(U_of<R>(e), r, Ar, e.fg, diag4(e), nvec, e.bsc.p, e.bpart.p, e.bpart.n, e.btickets.p,
                            e.s)) {
        launch_mr_update_batch<R>(e.bsc.p, e.p.omega, x, r, Ar, e.nf, nvec, e.s);
        continue;
      }
    }
    launch_dslash4<R>(U_of<R>(e), r, Ar, e.fg, diag4(e), nullptr, 1.0, 0.0, e.s, nvec);
    launch_dot_norm_batch<R>(Ar, r, e.nf, nvec, e.bsc.p, e.bpart.p, e.btickets.p, kMrBlocks, e.s);
    launch_mr_update_batch<R>(e.bsc.p, e.p.omega, x, r, Ar, e.nf, nvec, e.s);
  }
}

template <typename R>
struct VWork;
template <>
struct VWork<double> {
  static Cx<double> *r(Engine4 &e) { return e.vr64.p; }
  static Cx<double> *Ar(Engine4 &e) { return e.vAr64.p; }
  static Cx<double> *x(Engine4 &e) { return e.vx64.p; }
  static Cx<double> *b(Engine4 &e) { return e.vb64.p; }
};
template <>
struct VWork<float> {
  static Cx<float> *r(Engine4 &e) { return e.vr32.p; }
  static Cx<float> *Ar(Engine4 &e) { return e.vAr32.p; }
  static Cx<float> *x(Engine4 &e) { return e.vx32.p; }
  static Cx<float> *b(Engine4 &e) { return e.vb32.p; }
};

// FP64 <-> cycle precision
template <typename R>
void from64(Engine4 &e, const Cx<double> *src, Cx<R> *dst, long long n);
template <>
void from64<double>(Engine4 &e, const Cx<double> *src, Cx<double> *dst, long long n) {
  launch_copy<double>(src, dst, n, e.s);
}
template <>
void from64<float>(Engine4 &e, const Cx<double> *src, Cx<float> *dst, long long n) {
  launch_convert<float, double>(src, dst, n, e.s);
}
template <typename R>
void to64(Engine4 &e, const Cx<R> *src, Cx<double> *dst, long long n);
template <>
void to64<double>(Engine4 &e, const Cx<double> *src, Cx<double> *dst, long long n) {
  launch_copy<double>(src, dst, n, e.s);
}
template <>
void to64<float>(Engine4 &e, const Cx<float> *src, Cx<double> *dst, long long n) {
  launch_convert<double, float>(src, dst, n, e.s);
}

// x = V b (b, x FP64; the cycle runs in R)
template <typename R>
void vcycle(Engine4 &e, const Cx<double> *b64, Cx<double> *x64) {
  Cx<R> *r = VWork<R>::r(e), *Ar = VWork<R>::Ar(e), *x = VWork<R>::x(e), *b = VWork<R>::b(e);
  from64<R>(e, b64, b, e.nf);
  // 1. pre-smoothing from x = 0
  launch_zero<R>(x, e.nf, e.s);
  launch_copy<R>(b, r, e.nf, e.s);
  mr_fine<R>(e, x, r, Ar, e.p.nu_pre);
  // 2. residual and restriction
  fine_apply<R>(e, x, r, b, -1.0, 1.0);
  Cx<R> *rc = sizeof(R) == 8 ? reinterpret_cast<Cx<R> *>(e.cb.p) : reinterpret_cast<Cx<R> *>(e.cb32.p);
  launch_restrict4<R>(V_of<R>(e), r, rc, e.bg, e.s);
  // 3. coarse solve (FP32 vectors throughout when the coarse GCR runs on them)
  const bool c32 = sizeof(R) == 4 && e.cy32.p != nullptr && std::getenv("MG_COARSE4_FP64_VECTORS") == nullptr;
  if (c32) {
    coarse_solve32(e);
  } else {
    if (sizeof(R) == 4) to64<R>(e, rc, e.cb.p, e.nc);
    coarse_solve(e);
  }
  // 4. prolongation and correction
  Cx<R> *ec = sizeof(R) == 8 ? reinterpret_cast<Cx<R> *>(e.cx.p) : reinterpret_cast<Cx<R> *>(e.cx32.p);
  if (sizeof(R) == 4 && !c32) from64<R>(e, e.cx.p, ec, e.nc);
  launch_prolong4<R>(V_of<R>(e), ec, x, e.bg, e.s);
  // 5. post-smoothing on the new residual
  fine_apply<R>(e, x, r, b, -1.0, 1.0);
  mr_fine<R>(e, x, r, Ar, e.p.nu_post);
  to64<R>(e, x, x64, e.nf);
}

void precondition(Engine4 &e, const Cx<double> *r, Cx<double> *z) {
  if (e.f32)
    vcycle<float>(e, r, z);
  else
    vcycle<double>(e, r, z);
}

// MG_ERR_NAN if the last block inversion met a singular (or NaN) coarse self block
void check_info(Engine4 &e) {
  int info = 0;
  MG_CUDA(cudaMemcpyAsync(&info, e.info.p, sizeof(int), cudaMemcpyDeviceToHost, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
  if (info != 0) {
    MG_CUDA(cudaMemsetAsync(e.info.p, 0, sizeof(int), e.s));
    fail(MG_ERR_NAN, "coarse level: a self block is singular or not finite");
  }
}

// block-Jacobi inverses of the coarse self blocks and the preconditioned stencil A M, then
// the FP32 copies (MG_FP32)
void prepare_coarse(Engine4 &e) {
  e.mrhs_ready = false;
  launch_block_invert4(e.Y64.p, e.Minv64.p, e.cg, e.info.p, e.s);
  launch_precondition4(e.Y64.p, e.Minv64.p, e.Yt64.p, e.cg, e.s);
  if (!e.f32) return;
  launch_convert<float, double>(e.V64.p, e.V32.p, e.V64.n, e.s);
  launch_convert<float, double>(e.Yt64.p, e.Yt32.p, e.Yt64.n, e.s);
  launch_convert<float, double>(e.Minv64.p, e.Minv32.p, e.Minv64.n, e.s);
  if (e.Yth.p != nullptr) launch_pack_half2(e.Yt64.p, e.Yth.p, e.Yt64.n, e.s);
}

// Galerkin products in FP32 arithmetic (from the FP32 links and prolongator) for mixed-precision
// hierarchies whose coarse solve is inexact anyway (coarsest_tol >= 1e-5): the operator then
// differs from the FP64 one by FP32 rounding, far below what that solve leaves;
// MG_FP64_GALERKIN keeps FP64
static bool galerkin4_f32(const Engine4 &e) {
  return e.f32 && e.p.coarsest_tol >= 1e-5 && std::getenv("MG_FP64_GALERKIN") == nullptr;
}

static void galerkin4(Engine4 &e) {
  if (galerkin4_f32(e)) {
    launch_convert<float, double>(e.V64.p, e.V32.p, e.V64.n, e.s);
    launch_galerkin4<float>(e.U32.p, diag4(e), e.V32.p, e.Y64.p, e.bg, e.s);
  } else {
    launch_galerkin4<double>(e.U64.p, diag4(e), e.V64.p, e.Y64.p, e.bg, e.s);
  }
}

// chirality split, block Gram-Schmidt and Galerkin operator from the current vectors
void build(Engine4 &e) {
  launch_gather_split4(e.nullv.p, e.nf, e.V64.p, e.bg, e.s);
  launch_block_gs4(e.V64.p, e.bg, e.s);
  galerkin4(e);
  prepare_coarse(e);
}

void setup(Engine4 &e) {
  const int Nv = e.bg.Nv;
  for (int k = 0; k < Nv; ++k) launch_gaussian(e.nullv.p + (long long)k * e.nf, e.nf, e.p.seed, k, 0, e.s);
  // relaxation of all Nv vectors as one batch: MR on D x = 0 from x = v (r = -D v); in FP32
  // on FP32 copies in mixed mode
  const long long nall = (long long)Nv * e.nf;
  if (e.f32) {
    launch_convert<float, double>(e.nullv.p, e.sx32.p, nall, e.s);
    launch_dslash4<float>(e.U32.p, e.sx32.p, e.sr32.p, e.fg, diag4(e), nullptr, -1.0, 0.0, e.s, Nv);
    mr_fine<float>(e, e.sx32.p, e.sr32.p, e.sAr32.p, e.p.nu_setup, Nv);
    launch_convert<double, float>(e.sx32.p, e.nullv.p, nall, e.s);
  } else {
    launch_dslash4<double>(e.U64.p, e.nullv.p, e.sr64.p, e.fg, diag4(e), nullptr, -1.0, 0.0, e.s, Nv);
    mr_fine<double>(e, e.nullv.p, e.sr64.p, e.sAr64.p, e.p.nu_setup, Nv);
  }
  build(e);
  for (int pass = 2; pass <= e.p.n_pass; ++pass) {
    for (int k = 0; k < Nv; ++k) {
      Cx<double> *v = e.nullv.p + (long long)k * e.nf;
      fine_apply<double>(e, v, e.t64.p);
      precondition(e, e.t64.p, e.orr.p);        // orr = V (D v)
      launch_xmy<double>(v, e.orr.p, e.nf, e.s);  // orr = v - V (D v)
      launch_copy<double>(e.orr.p, v, e.nf, e.s);
    }
    build(e);
  }
}

}  // namespace

void validate4(const mg_geom *g, const mg_params *p) {
  if (!g || !p) fail(MG_ERR_INVALID_ARG, "null geometry or parameters");
  if (g->Nc != 3) fail(MG_ERR_UNSUPPORTED, "d = 4 needs Nc = 3 (SU(3))");
  long long vol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (g->dims[mu] < 2) fail(MG_ERR_INVALID_ARG, "lattice extents must be >= 2");
    vol *= g->dims[mu];
  }
  if (vol * 12 >= (1LL << 31)) fail(MG_ERR_UNSUPPORTED, "4d lattices are limited to fewer than 2^31 / 12 sites");
  if (p->levels != 2) fail(MG_ERR_UNSUPPORTED, "the 4d hierarchy is built with 2 levels");
  if (p->chiral_split != 1) fail(MG_ERR_UNSUPPORTED, "the 4d hierarchy needs chiral_split = 1");
  if (p->precision != MG_FP64 && p->precision != MG_FP32) fail(MG_ERR_INVALID_ARG, "unknown precision");
  if (p->n_pass < 1 || p->nu_pre < 0 || p->nu_post < 0 || p->nu_setup < 0) fail(MG_ERR_INVALID_ARG, "bad counts");
  if (p->gcr_restart < 1 || p->gcr_restart > 128) fail(MG_ERR_INVALID_ARG, "gcr_restart must be in [1, 128]");
  if (p->coarsest_restart < 1 || p->coarsest_restart > 64)
    fail(MG_ERR_INVALID_ARG, "coarsest_restart must be in [1, 64] for d = 4");
  if (p->max_iter < 1 || p->coarsest_max_iter < 1) fail(MG_ERR_INVALID_ARG, "iteration limits must be >= 1");
  if (p->max_rhs < 1 || p->max_rhs > 32) fail(MG_ERR_INVALID_ARG, "max_rhs must be in [1, 32]");
  int bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int B = p->block[0][mu];
    if (B < 1 || g->dims[mu] % B) fail(MG_ERR_INVALID_ARG, "level 0: extents not divisible by the block");
    bvol *= B;
  }
  if (bvol > 512) fail(MG_ERR_UNSUPPORTED, "4d blocks are limited to 512 sites");
  if (p->Nv[0] < 1 || p->Nv[0] > 32 || p->Nv[0] > 6 * bvol)
    fail(MG_ERR_INVALID_ARG, "level 0: Nv must be in [1, min(6 x block sites, 32)]");
}

Engine4 *engine4_create(const mg_geom *g, const void *U, double m, const mg_params *p, cudaStream_t s,
                        bool run_setup) {
  validate4(g, p);
  auto e = std::make_unique<Engine4>();
  e->geom = *g;
  e->p = *p;
  e->m = m;
  e->s = s;
  e->f32 = p->precision == MG_FP32;
  long long vol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    e->fg.L[mu] = g->dims[mu];
    e->bg.L[mu] = g->dims[mu];
    e->bg.B[mu] = p->block[0][mu];
    e->bg.nb[mu] = g->dims[mu] / p->block[0][mu];
    e->cg.nb[mu] = e->bg.nb[mu];
    vol *= g->dims[mu];
  }
  e->fg.nsites = vol;
  e->bg.bvol = p->block[0][0] * p->block[0][1] * p->block[0][2] * p->block[0][3];
  e->bg.nblocks = (int)(vol / e->bg.bvol);
  e->bg.Nv = p->Nv[0];
  e->N = 2 * p->Nv[0];
  e->cg.N = e->N;
  e->cg.nsites = e->bg.nblocks;
  e->nf = vol * 12;
  e->nc = (long long)e->bg.nblocks * e->N;
  MG_CUDA(cudaMallocHost(&e->host, kScalCount * sizeof(double)));
  e->U64.alloc((size_t)vol * 36);
  e->nullv.alloc((size_t)e->bg.Nv * e->nf);
  e->V64.alloc((size_t)e->bg.nblocks * e->N * e->bg.bvol * 6);
  e->Y64.alloc((size_t)e->bg.nblocks * 9 * e->N * e->N);
  e->Minv64.alloc((size_t)e->bg.nblocks * e->N * e->N);
  e->Yt64.alloc(e->Y64.n);
  e->info.alloc(1);
  e->vr64.alloc(e->nf);
  e->vAr64.alloc(e->nf);
  e->vx64.alloc(e->nf);
  e->vb64.alloc(e->nf);
  if (e->f32) {
    e->U32.alloc(e->U64.n);
    e->V32.alloc(e->V64.n);
    e->Yt32.alloc(e->Y64.n);
    e->Minv32.alloc(e->Minv64.n);
    e->vr32.alloc(e->nf);
    e->vAr32.alloc(e->nf);
    e->vx32.alloc(e->nf);
    e->vb32.alloc(e->nf);
    e->cb32.alloc(e->nc);
    e->cx32.alloc(e->nc);
    if (p->coarsest_tol >= 1e-5) {
      e->cZ32.alloc((size_t)p->coarsest_restart * e->nc);
      e->cW32.alloc((size_t)p->coarsest_restart * e->nc);
      e->cr32.alloc(e->nc);
      e->cy32.alloc(e->nc);
      e->cwt32.alloc(e->nc);
      e->cctl.alloc(2);
      // the FP16 operator: its rounding (2^-11 of each entry) is far below a loose coarse tolerance
      if (p->coarsest_tol >= 0.05 && std::getenv("MG_COARSE4_FP32_OPERATOR") == nullptr) e->Yth.alloc(e->Yt64.n);
    }
  }
  e->cb.alloc(e->nc);
  e->cx.alloc(e->nc);
  e->cy.alloc(e->nc);
  e->cZ.alloc((size_t)p->coarsest_restart * e->nc);
  e->cW.alloc((size_t)p->coarsest_restart * e->nc);
  e->cr.alloc(e->nc);
  e->oZ.alloc((size_t)p->gcr_restart * e->nf);
  e->oW.alloc((size_t)p->gcr_restart * e->nf);
  e->orr.alloc(e->nf);
  e->t64.alloc(e->nf);
  e->ws.max_blocks = 152 * 8;
  const long long cap = std::max<long long>((long long)e->ws.max_blocks * 4, 2LL * (std::max(p->gcr_restart, p->coarsest_restart) + 3) * 64);
  e->partials.alloc((size_t)cap + 16);
  e->ws.capacity = cap;
  e->ws.tickets = 160;
  e->tickets.alloc((size_t)e->ws.tickets);
  e->scal.alloc(kScalCount);
  const int nbat = std::max(e->bg.Nv, std::max(1, p->max_rhs));  // vectors of a batched MR
  // per-block partials of the batched MR sums: the reduction kernel's grid, or the tiled Wilson
  // apply's tiles when it forms the sums itself (64 sites per tile)
  e->bpart.alloc((size_t)nbat * std::max<long long>(kMrBlocks, e->fg.nsites / 64) * 3 + 16);
  e->bsc.alloc((size_t)nbat * 3);
  e->btickets.alloc((size_t)nbat);
  if (e->f32) {
    e->sx32.alloc((size_t)e->bg.Nv * e->nf);
    e->sr32.alloc((size_t)e->bg.Nv * e->nf);
    e->sAr32.alloc((size_t)e->bg.Nv * e->nf);
  } else {
    e->sr64.alloc((size_t)e->bg.Nv * e->nf);
    e->sAr64.alloc((size_t)e->bg.Nv * e->nf);
  }
  pool_ready();
  MG_CUDA(cudaMemsetAsync(e->btickets.p, 0, e->btickets.n * sizeof(unsigned int), s));
  MG_CUDA(cudaMemsetAsync(e->tickets.p, 0, e->ws.tickets * sizeof(unsigned int), s));
  MG_CUDA(cudaMemsetAsync(e->scal.p, 0, kScalCount * sizeof(double), s));
  MG_CUDA(cudaMemsetAsync(e->info.p, 0, sizeof(int), s));
  e->ws.partials = e->partials.p;
  e->ws.ticket = e->tickets.p;
  e->wsc = e->ws;
  e->wsc.max_blocks = 8;
  MG_CUDA(cudaMemcpyAsync(e->U64.p, U, e->U64.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, s));
  if (e->f32) launch_convert<float, double>(e->U64.p, e->U32.p, e->U64.n, s);
  if (run_setup) {
    setup(*e);
    check_info(*e);
  }
  return e.release();
}

void engine4_destroy(Engine4 *e) { delete e; }

Solve4 engine4_solve(Engine4 &e, const void *chi, void *psi, double tol) {
  for (long long &a : e.apps) a = 0;
  e.coarsest_iters = 0;
  EventPair ev;
  ev.start(e.s);
  auto apply = [&](const Cx<double> *in, Cx<double> *out, const Cx<double> *b = nullptr) {
    if (b != nullptr)
      fine_apply<double>(e, in, out, b, -1.0, 1.0);
    else
      fine_apply<double>(e, in, out);
  };
  auto prec = [&](const Cx<double> *r, Cx<double> *z) { precondition(e, r, z); };
  Gcr g = fgcr(e, apply, prec, static_cast<const Cx<double> *>(chi), static_cast<Cx<double> *>(psi), e.nf, tol,
               e.p.gcr_restart, e.p.max_iter, e.oZ.p, e.oW.p, e.orr.p, kScalOuter);
  Solve4 out;
  out.ms = ev.stop(e.s);
  out.iters = g.iters;
  out.converged = g.converged;
  out.rel = g.rel;
  for (int l = 0; l < MG_MAX_LEVELS; ++l) out.apps[l] = e.apps[l];
  out.coarsest_iters = e.coarsest_iters;
  return out;
}

void engine4_update_mass(Engine4 &e, double m) {
  e.m = m;
  galerkin4(e);
  prepare_coarse(e);
  check_info(e);
}

void engine4_level_size(const Engine4 &e, int level, long long *n_sites, int *n_int) {
  if (n_sites) *n_sites = level == 0 ? e.fg.nsites : e.cg.nsites;
  if (n_int) *n_int = level == 0 ? 12 : e.N;
}

void engine4_level_apply(Engine4 &e, int level, const void *in, void *out) {
  if (level == 0)
    fine_apply<double>(e, static_cast<const Cx<double> *>(in), static_cast<Cx<double> *>(out));
  else
    coarse_apply64(e, static_cast<const Cx<double> *>(in), static_cast<Cx<double> *>(out));
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_restrict(Engine4 &e, const void *fine, void *coarse) {
  launch_restrict4<double>(e.V64.p, static_cast<const Cx<double> *>(fine), static_cast<Cx<double> *>(coarse), e.bg,
                           e.s);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_prolong(Engine4 &e, const void *coarse, void *fine) {
  launch_zero<double>(static_cast<Cx<double> *>(fine), e.nf, e.s);
  launch_prolong4<double>(e.V64.p, static_cast<const Cx<double> *>(coarse), static_cast<Cx<double> *>(fine), e.bg,
                          e.s);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_vcycle(Engine4 &e, const void *b, void *x) {
  precondition(e, static_cast<const Cx<double> *>(b), static_cast<Cx<double> *>(x));
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_smooth(Engine4 &e, const void *b, void *x, int nu) {
  Cx<double> *xx = static_cast<Cx<double> *>(x);
  launch_zero<double>(xx, e.nf, e.s);
  launch_copy<double>(static_cast<const Cx<double> *>(b), e.vr64.p, e.nf, e.s);
  mr_fine<double>(e, xx, e.vr64.p, e.vAr64.p, nu);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_build_level(Engine4 &e, const void *vectors) {
  MG_CUDA(cudaMemcpyAsync(e.nullv.p, vectors, e.nullv.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e.s));
  build(e);
  check_info(e);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

long long engine4_null_vector_count(const Engine4 &e) { return (long long)e.nullv.n; }

const void *engine4_links(const Engine4 &e) { return e.U64.p; }

void engine4_get_null_vectors(Engine4 &e, void *out) {
  MG_CUDA(cudaMemcpyAsync(out, e.nullv.p, e.nullv.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_get_prolongator(Engine4 &e, void *out) {
  launch_prolongator4_to_canonical(e.V64.p, static_cast<Cx<double> *>(out), e.bg, e.s);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

void engine4_get_coarse_op(Engine4 &e, void *out) {
  launch_coarse4_to_canonical(e.Y64.p, static_cast<Cx<double> *>(out), e.cg, e.s);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

namespace {

// buffers of batched solves, for max_rhs vectors
void alloc_batch(Engine4 &e) {
  auto &b = e.bt;
  const int nb = std::max(1, e.p.max_rhs), ro = e.p.gcr_restart, rc = e.p.coarsest_restart;
  b.cap = nb;
  b.Z.alloc((size_t)ro * nb * e.nf);
  b.W.alloc((size_t)ro * nb * e.nf);
  b.r.alloc((size_t)nb * e.nf);
  b.rin.alloc((size_t)nb * e.nf);
  b.z64.alloc((size_t)nb * e.nf);
  if (e.f32) {
    b.r32.alloc((size_t)nb * e.nf);
    b.Ar32.alloc((size_t)nb * e.nf);
    b.x32.alloc((size_t)nb * e.nf);
    b.b32.alloc((size_t)nb * e.nf);
  } else {
    b.r64.alloc((size_t)nb * e.nf);
    b.Ar64.alloc((size_t)nb * e.nf);
    b.x64.alloc((size_t)nb * e.nf);
    b.b64.alloc((size_t)nb * e.nf);
  }
  b.cb.alloc((size_t)nb * e.nc);
  b.cx.alloc((size_t)nb * e.nc);
  b.cr.alloc((size_t)nb * e.nc);
  b.crin.alloc((size_t)nb * e.nc);
  b.cZ.alloc((size_t)rc * nb * e.nc);
  b.cW.alloc((size_t)rc * nb * e.nc);
  b.cin32.alloc((size_t)nb * e.nc);
  b.cout32.alloc((size_t)nb * e.nc);
  if (e.f32 && e.p.coarsest_tol >= 1e-5 && e.N == 48) {
    b.cb32.alloc((size_t)nb * e.nc);
    b.cx32.alloc((size_t)nb * e.nc);
    b.cr32.alloc((size_t)nb * e.nc);
    b.crin32.alloc((size_t)nb * e.nc);
    b.cZ32.alloc((size_t)rc * nb * e.nc);
    b.cW32.alloc((size_t)rc * nb * e.nc);
    b.czt32.alloc((size_t)nb * e.nc);
    b.cwt32.alloc((size_t)nb * e.nc);
    b.cctl.alloc(3);
    b.cact.alloc((size_t)nb);
    b.cstv.alloc((size_t)2 * nb);
    b.cnorm.alloc((size_t)2 * nb);
  }
  const int rows = std::max(ro, rc) + 3;
  b.dots.alloc((size_t)nb * 2 * (ro + 3));
  b.coef.alloc((size_t)nb * 4);
  b.cdots.alloc((size_t)nb * 2 * (rc + 3));
  b.ccoef.alloc((size_t)nb * 4);
  b.ws.max_blocks = 64;
  b.ws.tickets = (long long)rows * nb;
  b.ws.capacity = 2LL * rows * nb * 64;
  b.part.alloc((size_t)b.ws.capacity + 16);
  b.tickets.alloc((size_t)b.ws.tickets);
  MG_CUDA(cudaMallocHost(&b.host, ((size_t)nb * 2 * (ro + 3) + nb * 4) * sizeof(double)));
  MG_CUDA(cudaMallocHost(&b.chost, ((size_t)nb * 2 * (rc + 3) + nb * 4) * sizeof(double)));
  pool_ready();
  MG_CUDA(cudaMemsetAsync(b.tickets.p, 0, b.ws.tickets * sizeof(unsigned int), e.s));
  b.ws.partials = b.part.p;
  b.ws.ticket = b.tickets.p;
  // 64 blocks per reduction suit the fine vectors; on 512 x 48 coarse dofs they made 12 x (k + 3)
  // x 64 blocks of 1.5 elements per thread, and the batched dots took 164 us per launch
  b.wsc = b.ws;
  b.wsc.max_blocks = 8;
}

// operand precision of the batched tensor-core coarse apply (launch_coarse4_apply_tc's split):
// MG_COARSE4_TC_SPLIT = 0, 1 or 2, else 2
static int tc_split() {
  const char *v = std::getenv("MG_COARSE4_TC_SPLIT");
  if (v == nullptr) return 2;
  const int s = std::atoi(v);
  return s < 0 || s > 2 ? 2 : s;
}

// the multi-vector coarse operands after a Galerkin build: BF16 fragments (hi, and lo when
// a split-operator apply wants them) and an FP32 copy of Y
static void ensure_mrhs(Engine4 &e, bool lo) {
  if (e.Ypk4.p == nullptr) {
    e.Ypk4.alloc((size_t)e.cg.nsites * 9 * 2 * 9 * 32);
    e.Y32.alloc(e.Y64.n);
    pool_ready();
  }
  if (lo && e.Ypk4lo.p == nullptr) {
    e.Ypk4lo.alloc((size_t)e.cg.nsites * 9 * 2 * 9 * 32);
    pool_ready();
    e.mrhs_ready = false;
  }
  if (e.mrhs_ready) return;
  launch_pack_coarse4_bf16(e.Y64.p, e.Ypk4.p, e.cg.nsites, e.s);
  if (e.Ypk4lo.p != nullptr) launch_pack_coarse4_bf16(e.Y64.p, e.Ypk4lo.p, e.cg.nsites, e.s, true);
  launch_convert<float, double>(e.Y64.p, e.Y32.p, e.Y64.n, e.s);
  e.mrhs_ready = true;
}

// batched coarse solve of nb vectors: cx_v = A_c^{-1} cb_v by lockstep GCR to coarsest_tol,
// right-preconditioned by block Jacobi; the operator applied to all vectors at once on
// tensor cores (N = 48; BF16 operands split as tc_split says, FP32 sums) or, otherwise, in FP64
// The batched coarse GCR on FP32 vectors with its iterations on the device: a cycle-start kernel
// and a WHILE node whose body is one lockstep iteration (masked copy of r, block-Jacobi
// preconditioner, tensor-core operator, reduction with k read from device memory, per-vector
// coefficients, update, control), captured once per batch size and launched once per restart
// cycle; the host reads the true residuals after each launch. Classical Gram-Schmidt in one
// pass, as the single-vector coarse GCR.
static cudaGraphExec_t coarse_batch_loop_graph(Engine4 &e, int nb, int split) {
  auto &b = e.bt;
  const std::vector<const void *> key = {reinterpret_cast<const void *>((long long)nb),
                                         reinterpret_cast<const void *>((long long)split), e.Ypk4.p, e.Ypk4lo.p,
                                         e.Minv32.p, b.cZ32.p, b.cW32.p, b.cdots.p, b.ccoef.p, b.wsc.partials};
  if (b.loop != nullptr && key == b.loop_key) return b.loop;
  if (b.loop != nullptr) {
    MG_CUDA(cudaGraphExecDestroy(b.loop));
    b.loop = nullptr;
  }
  const long long n = e.nc;
  const int restart = e.p.coarsest_restart, max_iter = e.p.coarsest_max_iter;
  cudaGraph_t top = nullptr;
  MG_CUDA(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle h;
    MG_CUDA(cudaGraphConditionalHandleCreate(&h, top, 0, cudaGraphCondAssignDefault));
    MG_CUDA(cudaStreamBeginCaptureToGraph(e.s, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_coarse4_batch_cycle_start(b.cctl.p, b.cact.p, nb, max_iter, h, e.s);
    MG_CUDA(cudaStreamEndCapture(e.s, &top));
    size_t count = 1;
    cudaGraphNode_t start;
    MG_CUDA(cudaGraphGetNodes(top, &start, &count));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MG_CUDA(cudaGraphAddNode(&node, top, &start, nullptr, 1, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    MG_CUDA(cudaStreamBeginCaptureToGraph(e.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_copy_active<float>(b.cr32.p, b.crin32.p, n, nb, b.cact.p, e.s);
    launch_block_apply4_32(e.Minv32.p, b.crin32.p, b.czt32.p, e.cg, e.s, nb);
    launch_coarse4_apply_tc(e.Ypk4.p, b.czt32.p, b.cwt32.p, e.cg.nb, nb, e.s, split, e.Ypk4lo.p);
    launch_gcr_dots_batch_devk<float>(b.cW32.p, b.cwt32.p, b.cr32.p, b.cctl.p, nb, restart, n, b.cdots.p, b.wsc, e.s);
    launch_gcr_coef_batch(b.cdots.p, b.cctl.p, nb, restart, b.cact.p, b.cstv.p, b.ccoef.p, e.s);
    launch_gcr_update_batch_devk<float>(b.cW32.p, b.cZ32.p, b.cwt32.p, b.czt32.p, b.cctl.p, nb, restart, b.cdots.p,
                                        b.ccoef.p, b.cx32.p, b.cr32.p, n, e.s);
    launch_gcr_control_batch(b.cctl.p, b.cact.p, nb, restart, max_iter, h, e.s);
    MG_CUDA(cudaStreamEndCapture(e.s, &body));
    MG_CUDA(cudaGraphInstantiate(&b.loop, top, 0));
  } catch (...) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t partial = nullptr;
    if (cudaStreamIsCapturing(e.s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(e.s, &partial);  // a graph owned by top (or top itself)
    cudaGetLastError();
    cudaGraphDestroy(top);
    throw;
  }
  cudaGraphDestroy(top);
  b.loop_key = key;
  return b.loop;
}

// cb (FP64, nb vectors) -> cx by the graph-replayed lockstep GCR; returns the lockstep iterations
static long long coarse_solve_batch32_loop(Engine4 &e, int nb, int split) {
  auto &b = e.bt;
  const long long n = e.nc, nn = (long long)nb * n;
  cudaGraphExec_t g = coarse_batch_loop_graph(e, nb, split);
  launch_convert<float, double>(b.cb.p, b.cb32.p, nn, e.s);
  launch_zero<float>(b.cx32.p, nn, e.s);
  launch_copy<float>(b.cb32.p, b.cr32.p, nn, e.s);
  double *bn2 = b.cnorm.p, *rn2 = b.cnorm.p + nb;
  launch_norm2_batch(static_cast<const Cx<float> *>(b.cb32.p), n, nb, bn2, b.wsc, e.s);
  const double tol = e.p.coarsest_tol;
  launch_coarse4_batch_init(bn2, tol * tol, nb, b.cstv.p, b.cact.p, e.s);
  MG_CUDA(cudaMemsetAsync(b.cctl.p, 0, 3 * sizeof(int), e.s));
  std::vector<double> hn(2 * nb);
  std::vector<int> act(nb);
  int ctl[3] = {0, 0, 0};
  for (;;) {
    MG_CUDA(cudaGraphLaunch(g, e.s));
    // true residuals r_v = b_v - A x_v
    launch_coarse4_apply_tc(e.Ypk4.p, b.cx32.p, b.cr32.p, e.cg.nb, nb, e.s, split, e.Ypk4lo.p);
    launch_xmy<float>(b.cb32.p, b.cr32.p, nn, e.s);
    launch_norm2_batch(static_cast<const Cx<float> *>(b.cr32.p), n, nb, rn2, b.wsc, e.s);
    MG_CUDA(cudaMemcpyAsync(hn.data(), b.cnorm.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaMemcpyAsync(ctl, b.cctl.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
    e.apps[1] += (long long)nb;
    int left = 0;
    for (int v = 0; v < nb; ++v) {
      if (std::isnan(hn[v]) || std::isnan(hn[nb + v])) fail(MG_ERR_NAN, "GCR (batched): NaN in a reduction");
      act[v] = hn[v] > 0.0 && hn[nb + v] > tol * tol * hn[v] ? 1 : 0;
      left += act[v];
    }
    if (left == 0 || ctl[0] >= e.p.coarsest_max_iter) break;
    MG_CUDA(cudaMemcpyAsync(b.cact.p, act.data(), nb * sizeof(int), cudaMemcpyHostToDevice, e.s));
  }
  e.apps[1] += (long long)ctl[0] * nb;
  launch_convert<double, float>(b.cx32.p, b.cx.p, nn, e.s);
  return ctl[0];
}

void coarse_solve_batch(Engine4 &e, int nb) {
  auto &b = e.bt;
  const bool tc = e.N == 48;
  const int split = tc_split();
  if (tc) ensure_mrhs(e, split == 2);
  if (tc && b.czt32.p != nullptr && nb <= 32 && e.p.coarsest_restart <= kCoarseLoopMaxRestart &&
      std::getenv("MG_COARSE4_FP64_VECTORS") == nullptr && std::getenv("MG_COARSE4_HOST_LOOP") == nullptr) {
    e.coarsest_iters += coarse_solve_batch32_loop(e, nb, split);
    return;
  }
  auto apply = [&](const Cx<double> *in, Cx<double> *out, const Cx<double> *rhs) {
    if (tc) {
      launch_convert<float, double>(in, b.cin32.p, (long long)nb * e.nc, e.s);
      launch_coarse4_apply_tc(e.Ypk4.p, b.cin32.p, b.cout32.p, e.cg.nb, nb, e.s, split, e.Ypk4lo.p);
      launch_convert<double, float>(b.cout32.p, out, (long long)nb * e.nc, e.s);
      if (rhs != nullptr) launch_xmy<double>(rhs, out, (long long)nb * e.nc, e.s);  // out = rhs - A in
    } else {
      launch_coarse4_apply<double, double>(e.Y64.p, in, out, e.cg, rhs, rhs ? -1.0 : 1.0, rhs ? 1.0 : 0.0, e.s,
                                           nb);
    }
    e.apps[1] += nb;
  };
  auto prec = [&](const Cx<double> *r, Cx<double> *z) {
    if (e.f32)
      launch_block_apply4<float>(e.Minv32.p, r, z, e.cg, e.s, nb);
    else
      launch_block_apply4<double>(e.Minv64.p, r, z, e.cg, e.s, nb);
  };
  std::vector<GcrB> out;
  if (tc && b.cZ32.p != nullptr && std::getenv("MG_COARSE4_FP64_VECTORS") == nullptr) {
    // FP32 Krylov vectors (FP64 reductions and coefficients): the FP64 Gram-Schmidt of 12 vectors
    // over up to 64 basis vectors was most of a batched coarse iteration
    auto apply32 = [&](const Cx<float> *in, Cx<float> *o, const Cx<float> *rhs) {
      launch_coarse4_apply_tc(e.Ypk4.p, in, o, e.cg.nb, nb, e.s, split, e.Ypk4lo.p);
      if (rhs != nullptr) launch_xmy<float>(rhs, o, (long long)nb * e.nc, e.s);  // o = rhs - A in
      e.apps[1] += nb;
    };
    auto prec32 = [&](const Cx<float> *r, Cx<float> *z) { launch_block_apply4_32(e.Minv32.p, r, z, e.cg, e.s, nb); };
    launch_convert<float, double>(b.cb.p, b.cb32.p, (long long)nb * e.nc, e.s);
    fgcr_batch(e, nb, apply32, prec32, static_cast<const Cx<float> *>(b.cb32.p), b.cx32.p, e.nc, e.p.coarsest_tol,
               e.p.coarsest_restart, e.p.coarsest_max_iter, b.cZ32.p, b.cW32.p, b.cr32.p, b.crin32.p, b.cdots.p,
               b.ccoef.p, b.chost, b.wsc, out, 0.0);
    launch_convert<double, float>(b.cx32.p, b.cx.p, (long long)nb * e.nc, e.s);
  } else {
    fgcr_batch(e, nb, apply, prec, static_cast<const Cx<double> *>(b.cb.p), b.cx.p, e.nc, e.p.coarsest_tol,
               e.p.coarsest_restart, e.p.coarsest_max_iter, b.cZ.p, b.cW.p, b.cr.p, b.crin.p, b.cdots.p, b.ccoef.p,
               b.chost, b.wsc, out);
  }
  int mx = 0;
  for (const auto &o : out) mx = std::max(mx, o.iters);
  e.coarsest_iters += mx;
}

// batched V-cycle x_v = V b_v (FP64 in and out, the cycle in R)
template <typename R>
struct BWork;
template <>
struct BWork<double> {
  static Cx<double> *r(Engine4 &e) { return e.bt.r64.p; }
  static Cx<double> *Ar(Engine4 &e) { return e.bt.Ar64.p; }
  static Cx<double> *x(Engine4 &e) { return e.bt.x64.p; }
  static Cx<double> *b(Engine4 &e) { return e.bt.b64.p; }
};
template <>
struct BWork<float> {
  static Cx<float> *r(Engine4 &e) { return e.bt.r32.p; }
  static Cx<float> *Ar(Engine4 &e) { return e.bt.Ar32.p; }
  static Cx<float> *x(Engine4 &e) { return e.bt.x32.p; }
  static Cx<float> *b(Engine4 &e) { return e.bt.b32.p; }
};

template <typename R>
void vcycle_batch(Engine4 &e, int nb, const Cx<double> *b64, Cx<double> *x64) {
  Cx<R> *r = BWork<R>::r(e), *Ar = BWork<R>::Ar(e), *x = BWork<R>::x(e), *b = BWork<R>::b(e);
  const long long nall = (long long)nb * e.nf;
  from64<R>(e, b64, b, nall);
  launch_zero<R>(x, nall, e.s);
  launch_copy<R>(b, r, nall, e.s);
  mr_fine<R>(e, x, r, Ar, e.p.nu_pre, nb);
  launch_dslash4<R>(U_of<R>(e), x, r, e.fg, diag4(e), b, -1.0, 1.0, e.s, nb);
  e.apps[0] += nb;
  // restriction in R, coarse solve in FP64
  Cx<R> *rc = sizeof(R) == 8 ? reinterpret_cast<Cx<R> *>(e.bt.cb.p) : reinterpret_cast<Cx<R> *>(e.bt.cin32.p);
  launch_restrict4<R>(V_of<R>(e), r, rc, e.bg, e.s, nb);
  if (sizeof(R) == 4) to64<R>(e, rc, e.bt.cb.p, (long long)nb * e.nc);
  coarse_solve_batch(e, nb);
  Cx<R> *ec = sizeof(R) == 8 ? reinterpret_cast<Cx<R> *>(e.bt.cx.p) : reinterpret_cast<Cx<R> *>(e.bt.cin32.p);
  if (sizeof(R) == 4) from64<R>(e, e.bt.cx.p, ec, (long long)nb * e.nc);
  launch_prolong4<R>(V_of<R>(e), ec, x, e.bg, e.s, nb);
  launch_dslash4<R>(U_of<R>(e), x, r, e.fg, diag4(e), b, -1.0, 1.0, e.s, nb);
  e.apps[0] += nb;
  mr_fine<R>(e, x, r, Ar, e.p.nu_post, nb);
  to64<R>(e, x, x64, nall);
}

}  // namespace

std::vector<Solve4> engine4_solve_batch(Engine4 &e, int nrhs, const void *chi, void *psi, double tol) {
  if (e.bt.cap == 0) alloc_batch(e);
  if (nrhs < 1 || nrhs > e.bt.cap) fail(MG_ERR_INVALID_ARG, "nrhs must be in [1, max_rhs]");
  for (long long &a : e.apps) a = 0;
  e.coarsest_iters = 0;
  EventPair ev;
  ev.start(e.s);
  auto apply = [&](const Cx<double> *in, Cx<double> *out, const Cx<double> *rhs) {
    launch_dslash4<double>(e.U64.p, in, out, e.fg, diag4(e), rhs, rhs ? -1.0 : 1.0, rhs ? 1.0 : 0.0, e.s, nrhs);
    e.apps[0] += nrhs;
  };
  auto prec = [&](const Cx<double> *r, Cx<double> *z) {
    if (e.f32)
      vcycle_batch<float>(e, nrhs, r, z);
    else
      vcycle_batch<double>(e, nrhs, r, z);
  };
  std::vector<GcrB> g;
  fgcr_batch(e, nrhs, apply, prec, static_cast<const Cx<double> *>(chi), static_cast<Cx<double> *>(psi), e.nf, tol,
             e.p.gcr_restart, e.p.max_iter, e.bt.Z.p, e.bt.W.p, e.bt.r.p, e.bt.rin.p, e.bt.dots.p, e.bt.coef.p,
             e.bt.host, e.bt.ws, g);
  const float ms = ev.stop(e.s);
  std::vector<Solve4> out(nrhs);
  for (int v = 0; v < nrhs; ++v) {
    out[v].iters = g[v].iters;
    out[v].converged = g[v].converged;
    out[v].rel = g[v].rel;
    for (int l = 0; l < MG_MAX_LEVELS; ++l) out[v].apps[l] = e.apps[l];
    out[v].coarsest_iters = e.coarsest_iters;
    out[v].ms = ms;
  }
  return out;
}

void engine4_coarse_apply_mrhs(Engine4 &e, int nrhs, const void *in, void *out, int tensor_cores) {
  if (e.N != 48) fail(MG_ERR_UNSUPPORTED, "the 4d multi-vector coarse apply is built for N = 48 (Nv = 24)");
  if (tensor_cores < 0 || tensor_cores > 3) fail(MG_ERR_INVALID_ARG, "tensor_cores must be 0, 1, 2 or 3");
  ensure_mrhs(e, tensor_cores == 3);
  const Cx<float> *x = static_cast<const Cx<float> *>(in);
  Cx<float> *y = static_cast<Cx<float> *>(out);
  if (tensor_cores != 0)
    launch_coarse4_apply_tc(e.Ypk4.p, x, y, e.cg.nb, nrhs, e.s, tensor_cores - 1, e.Ypk4lo.p);
  else
    launch_coarse4_apply<float, float>(e.Y32.p, x, y, e.cg, nullptr, 1.0, 0.0, e.s, nrhs);
  MG_CUDA(cudaStreamSynchronize(e.s));
}

long long engine4_coarsest_solve(Engine4 &e, const void *b, void *x, float *ms) {
  EventPair ev;
  MG_CUDA(cudaMemcpyAsync(e.cb.p, b, e.nc * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e.s));
  ev.start(e.s);
  const long long it = coarse_solve(e);
  const float t = ev.stop(e.s);
  MG_CUDA(cudaMemcpyAsync(x, e.cx.p, e.nc * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
  if (ms) *ms = t;
  return it;
}

}  // namespace mg
