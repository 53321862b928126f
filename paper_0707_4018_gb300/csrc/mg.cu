// Host orchestration of the adaptive multigrid solver and the C ABI (mg.h).
//
// Paper structure followed here:
//   * adaptive setup (Eq. relax, Eq. P1, the adaptive passes, recursion to
//     further levels) with the Galerkin operator P^dagger A P (Eq. Galerkin);
//   * V-cycle in five steps (pre-relaxation, restriction of the residual,
//     coarse cycle or exact coarsest solve, coarse-grid correction,
//     post-relaxation), 2 nu + 2 operator applications per level;
//   * outer Krylov loop preconditioned with one V-cycle per iteration
//     (flexible GCR on D, FP64, true residual at every restart).
// Every arithmetic step runs in the kernels of this library on the context's
// stream; the host only sequences launches and reads convergence scalars.
#include <cmath>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.h"
#include "mg4d.h"
#include "nullnet.h"

namespace mg {

std::atomic<long long> g_launches{0};

void pool_init() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long keep = ~0ULL;  // never hand freed memory back to the driver
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

void pool_ready() { MG_CUDA(cudaStreamSynchronize(cudaStreamPerThread)); }

static thread_local std::string t_last_error;

void set_last_error(const std::string &msg) { t_last_error = msg; }

template <typename R>
struct Work {
  DevBuf<Cx<R>> b, x, r, Ar, r2, Ar2;  // r / r2 and Ar / Ar2 alternate inside the MR smoother
};

struct Level {
  Geo2 geo{};
  int nint = 0;
  long long n = 0;  // complex dofs
  // coarse operator of this level (level >= 1), internal layout
  DevBuf<Cx<double>> Y64;
  DevBuf<Cx<float>> Y32;
  DevBuf<uint2> Ypk;  // BF16 A fragments of Y32 for the tensor-core apply (N = 8, FP32 mode)
  // transfer to the next level
  BlockGeo bg{};
  int Nv = 0;
  DevBuf<Cx<double>> nullv;  // Nv level vectors
  DevBuf<Cx<double>> V64;    // prolongator [b][k][i]
  DevBuf<Cx<float>> V32;
  DevBuf<double> mgs_min;    // per-block smallest Gram-Schmidt norm
  Work<double> w64;
  Work<float> w32;
  DevBuf<Cx<double>> tA, tB;  // setup temporaries
  DevBuf<Cx<float>> sv, sA, sB;  // FP32 setup copies of the near-null vectors and temporaries
  bool stale = false;
};

// scalar slots on the device (FP64)
enum : int {
  kSlotOuter = 0,   // outer GCR reductions: 2 (restart + 3) doubles
  kSlotCount = 512
};
constexpr int kMaxBatch = 32;  // vectors per batched V-cycle (the setup batches the Nv near-null vectors)

// an instantiated graph of one V-cycle with the launches and operator
// applications it replays
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  long long apps[MG_MAX_LEVELS] = {0, 0, 0, 0};
  bool coop = false;  // holds a cooperative kernel: launched through the cooperative lane
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
};

}  // namespace mg

struct mg_ctx {
  mg_geom geom{};
  mg_params p{};
  double m = 0.0;
  cudaStream_t s = nullptr;      // the context's own stream (all library work)
  cudaStream_t user = nullptr;   // the caller's stream given to mg_setup
  cudaEvent_t ev = nullptr;      // orders the context stream after the caller's stream
  std::vector<mg::Level> lv;
  mg::DevBuf<mg::Cx<double>> U64;
  mg::DevBuf<mg::Cx<float>> U32;
  // MG_FP16: the fine level of the solve's FP32 cycles keeps its links and the smoother's r and
  // A r in half with per-site norms (12 V bytes per field); half_now while such a cycle is built
  bool half_fine = false, half_now = false;
  mg::DevBuf<float> U16;             // 2 V floats: V x (U^0, U^1) half2 pairs
  mg::DevBuf<float> hr[2], hA[2];    // 3 V floats per field, max_rhs fields
  // coarsest
  bool use_lu = false;
  int nc = 0;
  mg::DevBuf<mg::Cx<double>> LU, lu_work;
  mg::DevBuf<int> ipiv, info;
  mg::DevBuf<mg::Cx<double>> cZ, cW, cr, cb, cx;
  mg::DevBuf<double> cg_partials, cg_rel;
  mg::DevBuf<mg::Cx<double>> cg_Minv, cg_Yt, cg_work, cg_y;
  mg::DevBuf<mg::Cx<float>> cg_Yt32;  // FP32 copy of A M for mixed-precision cycles (shared-memory kernel)
  bool cg_cluster = false;            // one-cluster FP32 coarsest GCR (mixed precision, loose tolerance)
  bool cg_large32 = false;            // whole-chip FP32 coarsest GCR for large coarsest levels (same regime)
  mg::DevBuf<mg::Cx<float>> cZ32, cW32, cr32, cy32;
  mg::DevBuf<mg::Cx<float>> cl_rpub, cl_ypub;  // its publication buffers (nbatch vectors)
  mg::DevBuf<mg::Cx<float>> cl_Yr;             // A M in FP32 as row-major blocks
  mg::DevBuf<int> dl_ctl;                      // device-driven outer loop: counters, residual state, w
  mg::DevBuf<double> dl_st;
  mg::DevBuf<mg::Cx<double>> dl_w;
  bool tc_batch = false;                       // coarse residual applies of batched cycles on tensor cores
  mg::DevBuf<mg::Cx<double>> dl_wb;            // batched device loop: w, flags, state, coefficients
  mg::DevBuf<int> dl_act;
  mg::DevBuf<double> dl_stv, dl_coef;
  mg::DevBuf<int> cg_info;
  mg::DevBuf<unsigned int> cg_bar;
  mg::DevBuf<int> cg_out;  // [0] iterations, [1] timeout flag, [2] solves above tolerance
  int cg_grid = 0;
  bool cg_smem = false;  // shared-memory-resident coarsest solver
  int nbatch = 1;        // vectors the level work buffers hold (max of Nv and max_rhs)
  // batched solves: vector v of a batch sees every level's operator shifted by shift[v]
  // (mass_v - m; exact on the coarse levels because P^dagger P = 1) and uses coarsest slot v
  const double *cur_shift = nullptr;  // set while a batched solve records or runs its V-cycles
  mg::DevBuf<double> shift_dev;
  std::vector<double> slot_shift;     // shift each slot was prepared for (NaN: not prepared)
  mg::DevBuf<mg::Cx<double>> bMinv, bYt;               // per slot (iterative coarsest)
  std::vector<mg::DevBuf<mg::Cx<double>>> bLU;         // per slot (dense coarsest)
  std::vector<mg::DevBuf<int>> bipiv;
  bool cg_batch = false;  // batched shared-memory coarsest kernel usable
  mg::DevBuf<mg::Cx<double>> cgb_u, cgb_x;
  mg::DevBuf<double> cgb_partials;
  // batched outer GCR
  mg::DevBuf<mg::Cx<double>> bZ, bW, br, brin, bz64;
  mg::DevBuf<mg::Cx<float>> bz32;
  mg::DevBuf<double> bdots, bcoef;
  double *bhost = nullptr;  // pinned: dots, then coefficients
  std::vector<mg::GraphCache> preb[2];  // batched preconditioner graphs, per precision and batch size
  // outer
  mg::DevBuf<mg::Cx<double>> oZ, oW, orr;
  mg::DevBuf<mg::Cx<float>> z32;
  // reductions and scalars
  mg::DevBuf<double> partials, scal;
  mg::DevBuf<double> mrpart[2];  // MR block partials (alternating), reused as float in FP32 cycles
  mg::DevBuf<unsigned int> tickets;
  mg::ReduceWs ws{};
  double *host = nullptr;  // pinned scalars
  long long apps[MG_MAX_LEVELS] = {0, 0, 0, 0};
  long long coarsest_iters = 0;
  // CUDA graphs of the V-cycle: preconditioner (per precision) and setup cycles (per level)
  mg::GraphCache pre[2];
  mg::GraphCache setup_vc[MG_MAX_LEVELS];
  bool graphs_ok = true;
  mg::DevBuf<mg::Cx<double>> z64;
  mg::Engine4 *e4 = nullptr;  // the 4d SU(3) hierarchy (d = 4); the members above stay empty
  double setup_s = 0.0;       // seconds of the setup, load or clone that made this context
  ~mg_ctx() {
    if (s) cudaStreamSynchronize(s);  // no work may still use the buffers released below
    if (e4) mg::engine4_destroy(e4);
    for (auto &g : pre) g.reset();
    for (auto &v : preb)
      for (auto &g : v) g.reset();
    if (bhost) cudaFreeHost(bhost);
    for (auto &g : setup_vc) g.reset();
    if (s) cudaStreamDestroy(s);
    if (ev) cudaEventDestroy(ev);
    if (host) cudaFreeHost(host);
  }
};

namespace mg {

// Galerkin products in FP32 arithmetic for the hierarchies of mixed-precision cycles whose
// coarsest solve is itself inexact (iterative, tolerance >= 1e-5): their coarse operators are
// applied in FP32 and a 1e-7 relative change of them is far below what the cycle resolves.
// FP64 contexts and exact coarsest solves keep FP64 products.
static bool galerkin_f32(const mg_ctx &c) {
  return c.p.precision == MG_FP32 && !c.use_lu && c.p.coarsest_tol >= 1e-5 &&
         std::getenv("MG_FP64_GALERKIN") == nullptr;
}

static double diag_of(const mg_ctx &c) { return c.geom.d + c.m; }

template <typename R>
static Work<R> &work(Level &L);
template <>
Work<double> &work<double>(Level &L) { return L.w64; }
template <>
Work<float> &work<float>(Level &L) { return L.w32; }

template <typename R>
static const Cx<R> *Uof(const mg_ctx &c);
template <>
const Cx<double> *Uof<double>(const mg_ctx &c) { return c.U64.p; }
template <>
const Cx<float> *Uof<float>(const mg_ctx &c) { return c.U32.p; }

template <typename R>
static const Cx<R> *Yof(const Level &L);
template <>
const Cx<double> *Yof<double>(const Level &L) { return L.Y64.p; }
template <>
const Cx<float> *Yof<float>(const Level &L) { return L.Y32.p; }

template <typename R>
static const Cx<R> *Vof(const Level &L);
template <>
const Cx<double> *Vof<double>(const Level &L) { return L.V64.p; }
template <>
const Cx<float> *Vof<float>(const Level &L) { return L.V32.p; }

// FP32 copy of a coarse level's operator (and its packed BF16 form where it exists)
static void refresh_y32(mg_ctx &c, int l) {
  Level &L = c.lv[l];
  launch_convert<float, double>(L.Y64.p, L.Y32.p, L.Y64.n, c.s);
  if (L.Ypk.p != nullptr) launch_pack_coarse_bf16(L.Y32.p, L.Ypk.p, L.geo.nsites, c.s);
}

// out = a * A_l in + c * b
template <typename R>
static void apply_op(mg_ctx &c, int l, const Cx<R> *in, Cx<R> *out, const Cx<R> *b = nullptr, double a = 1.0,
                     double cc = 0.0, int nvec = 1) {
  Level &L = c.lv[l];
  if (l == 0 && sizeof(R) == 4 && c.half_now)  // FP16 fine level: half links, FP32 vectors
    launch_dslash_hl(c.U16.p, reinterpret_cast<const Cx<float> *>(in), reinterpret_cast<Cx<float> *>(out), L.geo,
                     diag_of(c), reinterpret_cast<const Cx<float> *>(b), a, cc, c.s, nvec, c.cur_shift);
  else if (l == 0)
    launch_dslash<R>(Uof<R>(c), in, out, L.geo, diag_of(c), b, a, cc, c.s, nvec, c.cur_shift);
  else if (sizeof(R) == 4 && c.tc_batch && nvec >= 8 && L.Ypk.p != nullptr)
    // batched solves: the coarse operator on tensor cores for all vectors at once (BF16
    // operands, FP32 sums; an N-tile of the MMA is 8 vectors)
    launch_coarse_apply_tc(L.Ypk.p, reinterpret_cast<const Cx<float> *>(in), reinterpret_cast<Cx<float> *>(out),
                           L.geo, nvec, reinterpret_cast<const Cx<float> *>(b), a, cc, c.cur_shift, c.s);
  else
    launch_coarse_apply<R>(Yof<R>(L), in, out, L.geo, L.nint, b, a, cc, c.s, nvec, c.cur_shift);
  c.apps[l] += nvec;
}

template <typename R>
static OpDesc<R> op_of(mg_ctx &c, int l) {
  Level &L = c.lv[l];
  OpDesc<R> o;
  o.wilson = (l == 0);
  o.U = Uof<R>(c);
  o.Y = l > 0 ? Yof<R>(L) : nullptr;
  o.geo = L.geo;
  o.N = L.nint;
  o.diag = diag_of(c);
  o.shift = c.cur_shift;
  return o;
}

// x (+)= nu MR iterations for A_l x = b from zero (accumulate: added to x), with the
// fused kernels: nu + 1 launches for a batch of nvec vectors (stride n). b may be the
// level's r buffer (consumed then). With r_out (not accumulating), the last launch also
// leaves the smoothed residual b - A x there (the MR recurrence r <- r - alpha A r;
// r_out may be the level's r buffer).
template <typename R>
static void smooth(mg_ctx &c, int l, const Cx<R> *b, Cx<R> *x, int nu, bool accumulate, int nvec = 1,
                   Cx<R> *r_out = nullptr) {
  Level &L = c.lv[l];
  Work<R> &w = work<R>(L);
  if (nu <= 0) {
    if (!accumulate) launch_zero<R>(x, L.n * nvec, c.s);
    if (r_out != nullptr && r_out != b) launch_copy<R>(b, r_out, L.n * nvec, c.s);
    return;
  }
  if (l == 0 && sizeof(R) == 4 && c.half_now) {
    // FP16 fine level: r and A r alternate between two half fields; x, b and r_out stay FP32
    if (nvec > c.p.max_rhs) fail(MG_ERR_STATE, "half-storage smoother: batch larger than max_rhs");
    float *hp[2] = {reinterpret_cast<float *>(c.mrpart[0].p), reinterpret_cast<float *>(c.mrpart[1].p)};
    const long long hcap = (long long)(c.mrpart[0].n * sizeof(double) / sizeof(float));
    Cx<float> *xf = reinterpret_cast<Cx<float> *>(x);
    launch_mr_iteration_half(c.U16.p, L.geo, diag_of(c), c.cur_shift, false, reinterpret_cast<const Cx<float> *>(b),
                             nullptr, nullptr, nullptr, c.p.omega, nullptr, false, c.hr[0].p, c.hA[0].p, hp[0], hcap,
                             c.s, nvec);
    c.apps[l] += nvec;
    int cur = 0;
    for (int i = 1; i < nu; ++i) {
      launch_mr_iteration_half(c.U16.p, L.geo, diag_of(c), c.cur_shift, true, nullptr, c.hr[cur].p, c.hA[cur].p,
                               hp[cur], c.p.omega, xf, i == 1 && !accumulate, c.hr[cur ^ 1].p, c.hA[cur ^ 1].p,
                               hp[cur ^ 1], hcap, c.s, nvec);
      c.apps[l] += nvec;
      cur ^= 1;
    }
    launch_mr_last_half(c.hr[cur].p, c.hA[cur].p, hp[cur], c.p.omega, xf, nu == 1 && !accumulate,
                        reinterpret_cast<Cx<float> *>(r_out), L.geo, c.s, nvec);
    return;
  }
  // two alternating partials buffers in the vectors' precision
  R *part[2] = {reinterpret_cast<R *>(c.mrpart[0].p), reinterpret_cast<R *>(c.mrpart[1].p)};
  const long long cap = (long long)(c.mrpart[0].n * sizeof(double) / sizeof(R));
  const OpDesc<R> op = op_of<R>(c, l);
  Cx<R> *rbuf[2] = {w.r.p, w.r2.p};
  Cx<R> *Arbuf[2] = {w.Ar.p, w.Ar2.p};
  launch_mr_iteration<R>(op, false, b, nullptr, nullptr, c.p.omega, nullptr, false, nullptr, Arbuf[0], part[0], cap,
                         c.s, nvec);
  c.apps[l] += nvec;
  const Cx<R> *r_old = b;
  int rsel = (b == rbuf[0]) ? 1 : 0, asel = 1, psel = 1;
  for (int i = 1; i < nu; ++i) {
    launch_mr_iteration<R>(op, true, r_old, Arbuf[asel ^ 1], part[psel ^ 1], c.p.omega, x, i == 1 && !accumulate,
                           rbuf[rsel], Arbuf[asel], part[psel], cap, c.s, nvec);
    c.apps[l] += nvec;
    r_old = rbuf[rsel];
    rsel ^= 1;
    asel ^= 1;
    psel ^= 1;
  }
  launch_mr_last<R>(op, r_old, Arbuf[asel ^ 1], part[psel ^ 1], c.p.omega, x, nu == 1 && !accumulate, r_out, L.n,
                    c.s, nvec);
}

static void precondition(mg_ctx &c, const Cx<double> *r, Cx<double> *z);

struct GcrOut {
  int iters = 0;
  bool converged = false;
  double rel = 0.0;
};

// Outer flexible GCR on D (FP64) with the V-cycle as right preconditioner.
// Per iteration: z = V r, w = D z, one fused reduction of <W_j, w>, |w|^2, <w, r>, |r|^2;
// the host forms the classical Gram-Schmidt coefficients, the Pythagorean norm
// |w - W beta|^2 = |w|^2 - |beta|^2 and alpha = <w_hat, r>, and runs a second
// projection only when that norm shows cancellation (< half of |w|^2); then one
// fused kernel projects, normalises and updates x and r. The new residual norm is
// |r|^2 - |alpha|^2 with |r|^2 freshly reduced (a running |b|^2 - sum |alpha|^2
// cannot resolve residuals below about sqrt(eps) |b| = 1e-8 |b|), and the true
// residual b - D x is recomputed at every restart (defect correction).
static GcrOut outer_fgcr(mg_ctx &c, const Cx<double> *b, Cx<double> *x, double tol, int restart, int max_iter) {
  Level &F = c.lv[0];
  const long long n = F.n;
  Cx<double> *Z = c.oZ.p, *W = c.oW.p, *r = c.orr.p;
  double *dots = c.scal.p + kSlotOuter;  // 2 (k + 3) doubles
  double *h = c.host;
  GcrOut out;
  auto fetch = [&](int count) {
    MG_CUDA(cudaMemcpyAsync(h, dots, count * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    MG_CUDA(cudaStreamSynchronize(c.s));
    for (int i = 0; i < count; ++i)
      if (std::isnan(h[i])) fail(MG_ERR_NAN, "outer GCR: NaN in a reduction");
  };
  launch_zero<double>(x, n, c.s);
  launch_copy<double>(b, r, n, c.s);
  launch_norm2<double>(b, n, dots, c.ws, c.s);
  fetch(1);
  const double bn2 = h[0];
  if (!(bn2 > 0.0)) {
    out.converged = true;
    return out;
  }
  double rn2 = bn2, rel = 1.0;
  while (out.iters < max_iter) {
    int k = 0;
    for (; k < restart && out.iters < max_iter; ++k) {
      Cx<double> *z = Z + (long long)k * n, *w = W + (long long)k * n;
      precondition(c, r, z);
      apply_op<double>(c, 0, z, w);
      launch_gcr_dots(W, w, r, k, n, dots, c.ws, c.s);
      fetch(2 * (k + 3));
      const double rr = h[2 * k + 4];  // |r|^2 before this update
      double nw0 = h[2 * k], nw2 = nw0;
      for (int j = 0; j < k; ++j) nw2 -= h[2 * j] * h[2 * j] + h[2 * j + 1] * h[2 * j + 1];
      double wr = h[2 * k + 2], wi = h[2 * k + 3];
      if (k > 0 && !(nw2 > 0.5 * nw0)) {
        // cancellation: project once, then take fresh coefficients for a second projection
        launch_gcr_project_update(W, w, Z, z, k, dots, 1.0, 0.0, 0.0, x, r, n, false, c.s);
        launch_gcr_dots(W, w, r, k, n, dots, c.ws, c.s);
        fetch(2 * (k + 3));
        nw0 = h[2 * k];
        nw2 = nw0;
        for (int j = 0; j < k; ++j) nw2 -= h[2 * j] * h[2 * j] + h[2 * j + 1] * h[2 * j + 1];
        wr = h[2 * k + 2];
        wi = h[2 * k + 3];
      }
      if (!(nw2 > 1e-28 * nw0)) break;  // breakdown: restart from the true residual
      const double inv = 1.0 / std::sqrt(nw2);
      const double are = wr * inv, aim = wi * inv;
      launch_gcr_project_update(W, w, Z, z, k, dots, inv, are, aim, x, r, n, true, c.s);
      rn2 = std::max(rr - (are * are + aim * aim), 0.0);
      ++out.iters;
      rel = std::sqrt(rn2 / bn2);
      if (rel <= tol) {
        ++k;
        break;
      }
    }
    apply_op<double>(c, 0, x, r, b, -1.0, 1.0);  // true residual r = b - D x
    launch_norm2<double>(r, n, dots, c.ws, c.s);
    fetch(1);
    rn2 = h[0];
    rel = std::sqrt(rn2 / bn2);
    if (rel <= tol) {
      out.converged = true;
      break;
    }
    if (k == 0) break;  // no progress possible
  }
  out.rel = rel;
  return out;
}

// exact solve on the coarsest level (FP64): dense LU or GCR to coarsest_tol. Slot 0 holds
// the factors / preconditioner at the context mass, slot 1 + v those of batched vector v.
static void coarsest_solve64(mg_ctx &c, const Cx<double> *b, Cx<double> *x, int slot = 0) {
  const int l = c.p.levels - 1;
  const Level &L = c.lv[l];
  if (c.use_lu) {
    const Cx<double> *LU = slot == 0 ? c.LU.p : c.bLU[slot - 1].p;
    const int *piv = slot == 0 ? c.ipiv.p : c.bipiv[slot - 1].p;
    lu_solve_ws(LU, piv, c.nc, b, x, c.lu_work.p, c.s);
    c.apps[l]++;
    return;
  }
  const long long m2 = L.geo.nsites * (long long)L.nint * L.nint;
  const Cx<double> *Minv = slot == 0 ? c.cg_Minv.p : c.bMinv.p + (slot - 1) * m2;
  const Cx<double> *Yt = slot == 0 ? c.cg_Yt.p : c.bYt.p + (slot - 1) * 5 * m2;
  if (c.cg_cluster && slot == 0)
    launch_coarsest_gcr_cluster(c.cl_Yr.p, Minv, L.geo, 1, b, x, c.cl_rpub.p, c.cl_ypub.p, c.p.coarsest_tol,
                                c.p.coarsest_restart, c.p.coarsest_max_iter, c.cg_out.p, c.cg_rel.p, c.s);
  else if (c.cg_smem)
    launch_coarsest_gcr_smem(Yt, slot == 0 ? c.cg_Yt32.p : nullptr, Minv, L.geo, b, x, c.cr.p, c.cg_y.p,
                             c.cg_partials.p, c.cg_bar.p,
                             c.p.coarsest_tol, c.p.coarsest_restart, c.p.coarsest_max_iter, c.cg_out.p, c.cg_rel.p,
                             c.cg_grid, c.s);
  else if (c.cg_large32 && slot == 0)
    // a quarter of the SMs: the FP32 solve is latency-bound (grid barriers over fewer CTAs are
    // cheaper), and the other SMs stay free for the non-cooperative work of concurrent streams
    launch_coarsest_gcr32(c.cg_Yt32.p, Minv, L.geo, L.nint, b, x, c.cy32.p, c.cr32.p, c.cZ32.p, c.cW32.p,
                          c.cg_partials.p, c.cg_bar.p, c.p.coarsest_tol, c.p.coarsest_restart, c.p.coarsest_max_iter,
                          c.cg_out.p, c.cg_rel.p, std::max(1, c.cg_grid / 4), c.s);
  else
    launch_coarsest_gcr(Yt, Minv, L.geo, L.nint, b, x, c.cg_y.p, c.cr.p, c.cZ.p, c.cW.p,
                        c.cg_partials.p, c.cg_bar.p, c.p.coarsest_tol, c.p.coarsest_restart, c.p.coarsest_max_iter,
                        c.cg_out.p, c.cg_rel.p, c.cg_grid, c.s);
}

// coarsest solves of nvec vectors (stride n). In a batched solve (cur_shift set) vector v
// uses slot 1 + v; otherwise every vector uses slot 0. Several vectors at once go through
// the batched shared-memory kernel (up to 4 per launch) when it applies.
static void coarsest_vectors64(mg_ctx &c, const Cx<double> *b, Cx<double> *x, int nvec) {
  const int l = c.p.levels - 1;
  const Level &L = c.lv[l];
  const long long n = L.n;
  const bool batch = c.cur_shift != nullptr;
  if (c.cg_cluster && nvec > 1 && !batch) {
    // every vector at the context mass: one cluster per vector, all in one launch
    launch_coarsest_gcr_cluster(c.cl_Yr.p, c.cg_Minv.p, L.geo, nvec, b, x, c.cl_rpub.p, c.cl_ypub.p,
                                c.p.coarsest_tol, c.p.coarsest_restart, c.p.coarsest_max_iter, c.cg_out.p, c.cg_rel.p,
                                c.s);
    return;
  }
  if (c.cg_batch && (nvec > 1 || batch)) {
    const long long m2 = L.geo.nsites * 64LL;
    for (int v0 = 0; v0 < nvec; v0 += kCoarsestBatchVecs) {
      const int nb = std::min(kCoarsestBatchVecs, nvec - v0);
      launch_coarsest_gcr_batch(L.Y64.p, batch ? c.bMinv.p + v0 * m2 : c.cg_Minv.p, batch ? m2 : 0,
                                batch ? c.cur_shift + v0 : nullptr, L.geo, nb, b + v0 * n, x + v0 * n, c.cgb_u.p,
                                c.cgb_x.p, c.cgb_partials.p, c.cg_bar.p, c.p.coarsest_tol, c.p.coarsest_restart,
                                c.p.coarsest_max_iter, c.cg_out.p, c.cg_rel.p, c.cg_grid, c.s);
    }
    return;
  }
  for (int v = 0; v < nvec; ++v) coarsest_solve64(c, b + v * n, x + v * n, batch ? 1 + v : 0);
}

// iterations of the persistent coarsest solves since the last reset; fails on a barrier timeout
static long long collect_coarsest(mg_ctx &c) {
  if (c.use_lu) return 0;
  int out[3] = {0, 0, 0};
  MG_CUDA(cudaMemcpyAsync(out, c.cg_out.p, sizeof(out), cudaMemcpyDeviceToHost, c.s));
  MG_CUDA(cudaStreamSynchronize(c.s));
  MG_CUDA(cudaMemsetAsync(c.cg_out.p, 0, 3 * sizeof(int), c.s));
  if (out[1] != 0) fail(MG_ERR_TIMEOUT, "coarsest solve: a grid barrier wait ran out (kernel returned early)");
  return out[0];
}

template <typename R>
static void coarsest_solve(mg_ctx &c, const Cx<R> *b, Cx<R> *x, int nvec);
template <>
void coarsest_solve<double>(mg_ctx &c, const Cx<double> *b, Cx<double> *x, int nvec) {
  coarsest_vectors64(c, b, x, nvec);
}
template <>
void coarsest_solve<float>(mg_ctx &c, const Cx<float> *b, Cx<float> *x, int nvec) {
  const long long n = c.lv.back().n * nvec;
  launch_convert<double, float>(b, c.cb.p, n, c.s);
  coarsest_vectors64(c, c.cb.p, c.cx.p, nvec);
  launch_convert<float, double>(c.cx.p, x, n, c.s);
}

static void check_fresh(const mg_ctx &c) {
  for (const Level &L : c.lv)
    if (L.stale) fail(MG_ERR_STATE, "hierarchy has a level whose prolongator predates its operator; rebuild it");
}

// x = V^(l) b (the five steps) for a batch of nvec vectors (stride: the level's dofs);
// b must not alias the level's work vectors or x
template <typename R>
static void vcycle(mg_ctx &c, int l, const Cx<R> *b, Cx<R> *x, int nvec = 1) {
  if (l == c.p.levels - 1) {
    coarsest_solve<R>(c, b, x, nvec);
    return;
  }
  Level &L = c.lv[l];
  Level &C = c.lv[l + 1];
  Work<R> &w = work<R>(L);
  Work<R> &wc = work<R>(C);
  // 1. pre-relaxation from zero, leaving the residual b - A x in w.r
  smooth<R>(c, l, b, x, c.p.nu_pre, false, nvec, w.r.p);
  // 2. restrict the residual
  launch_restrict<R>(Vof<R>(L), w.r.p, wc.b.p, L.bg, L.Nv, c.s, nvec);
  // 3. coarse V-cycle (or exact coarsest solve)
  vcycle<R>(c, l + 1, wc.b.p, wc.x.p, nvec);
  // 4. coarse-grid correction
  launch_prolong_add<R>(Vof<R>(L), wc.x.p, x, L.bg, L.Nv, c.s, nvec);
  // 5. post-relaxation on the final residual
  apply_op<R>(c, l, x, w.r.p, b, -1.0, 1.0, nvec);
  smooth<R>(c, l, w.r.p, x, c.p.nu_post, true, nvec);
}

// Runs `body` (a fixed sequence of launches on the context stream) through a
// CUDA graph captured on first use; later calls replay it. When capture is not
// possible the body runs as ordinary launches.
template <typename F>
static void graph_run(mg_ctx &c, GraphCache &g, F &&body) {
  if (c.graphs_ok && g.exec == nullptr) {
    const long long l0 = g_launches.load();
    long long a0[MG_MAX_LEVELS];
    for (int l = 0; l < MG_MAX_LEVELS; ++l) a0[l] = c.apps[l];
    bool ok = cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      (void)coop_captured_take();
      try {
        body();
      } catch (const Error &) {
        ok = false;
      }
      g.coop = coop_captured_take();
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c.s, &graph);
      ok = ok && e == cudaSuccess && graph != nullptr;
      if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
      if (ok) {
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(graph, nodes.data(), &nn);
        long long k = 0;
        for (auto nd : nodes) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
        }
        g.kernels = k;
        for (int l = 0; l < MG_MAX_LEVELS; ++l) g.apps[l] = c.apps[l] - a0[l];
      }
      if (graph) cudaGraphDestroy(graph);
    }
    (void)cudaGetLastError();
    g_launches.store(l0);
    for (int l = 0; l < MG_MAX_LEVELS; ++l) c.apps[l] = a0[l];
    if (!ok) {
      g.reset();
      c.graphs_ok = false;
    }
  }
  if (g.exec != nullptr) {
    if (g.coop)
      coop_graph_launch(g.exec, c.s);
    else
      MG_CUDA(cudaGraphLaunch(g.exec, c.s));
    g_launches.fetch_add(g.kernels);
    for (int l = 0; l < MG_MAX_LEVELS; ++l) c.apps[l] += g.apps[l];
  } else {
    body();
  }
}

// z = V r on the finest level in the context precision (r, z FP64). The cycle
// reads r from the fixed buffer `rfix` (the outer residual) and leaves its result
// in a fixed buffer, so one captured graph serves every call.
// the solve's cycles of an MG_FP16 context run their fine level in half storage
struct HalfCycles {
  mg_ctx &c;
  bool old;
  explicit HalfCycles(mg_ctx &cc) : c(cc), old(cc.half_now) { c.half_now = c.half_fine; }
  ~HalfCycles() { c.half_now = old; }
};

static void precondition(mg_ctx &c, const Cx<double> *r, Cx<double> *z) {
  Level &F = c.lv[0];
  const Cx<double> *rfix = c.orr.p;
  if (r != rfix) launch_copy<double>(r, c.orr.p, F.n, c.s);
  HalfCycles hc(c);
  if (c.p.precision == MG_FP32) {
    graph_run(c, c.pre[1], [&] {
      launch_convert<float, double>(rfix, F.w32.b.p, F.n, c.s);
      vcycle<float>(c, 0, F.w32.b.p, c.z32.p);
    });
    launch_convert<double, float>(c.z32.p, z, F.n, c.s);
  } else {
    graph_run(c, c.pre[0], [&] { vcycle<double>(c, 0, rfix, c.z64.p); });
    launch_copy<double>(c.z64.p, z, F.n, c.s);
  }
}

// ---------------------------------------------------------------------------
// batched solves: nb systems (D + shift_v) psi_v = chi_v sharing one hierarchy
// ---------------------------------------------------------------------------

// coarsest slots 1..nb for the shifts (prepared again only when a shift changed)
static void prepare_slots(mg_ctx &c, int nb, const double *shift) {
  Level &L = c.lv.back();
  const long long m2 = L.geo.nsites * (long long)L.nint * L.nint;
  for (int v = 0; v < nb; ++v) {
    if (c.slot_shift[v] == shift[v]) continue;
    if (c.use_lu) {
      if (c.bLU[v].p == nullptr) {
        c.bLU[v].alloc((size_t)c.nc * c.nc);
        c.bipiv[v].alloc(c.nc);
        pool_ready();
      }
      launch_dense_from_stencil(L.Y64.p, c.bLU[v].p, L.geo, L.nint, c.s, shift[v]);
      lu_factor(c.bLU[v].p, c.nc, c.bipiv[v].p, c.info.p, c.s);
      int info = 0;
      MG_CUDA(cudaMemcpyAsync(&info, c.info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
      MG_CUDA(cudaStreamSynchronize(c.s));
      if (info != 0) fail(MG_ERR_NAN, "coarsest LU (batched mass): zero pivot at column " + std::to_string(info - 1));
    } else {
      prepare_coarsest_gcr(L.Y64.p, L.geo, L.nint, c.bMinv.p + v * m2, c.cg_batch ? nullptr : c.bYt.p + v * 5 * m2,
                           c.cg_work.p, c.cg_info.p, c.s, shift[v]);
      int info = 0;
      MG_CUDA(cudaMemcpyAsync(&info, c.cg_info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
      MG_CUDA(cudaStreamSynchronize(c.s));
      if (info != 0) fail(MG_ERR_NAN, "coarsest level (batched mass): a self block is singular");
    }
    c.slot_shift[v] = shift[v];
  }
}

// z_v = V r_v for the vectors in mask (0 for the others), all nb in one batched V-cycle
// in the context precision; the cycle reads the fixed buffer brin, so one captured graph
// per batch size serves every call
static void precondition_batch(mg_ctx &c, int nb, const Cx<double> *r, unsigned int mask, Cx<double> *z) {
  Level &F = c.lv[0];
  const long long n = F.n;
  launch_copy_masked(r, c.brin.p, n, nb, mask, c.s);
  HalfCycles hc(c);
  if (c.p.precision == MG_FP32) {
    graph_run(c, c.preb[1][nb], [&] {
      launch_convert<float, double>(c.brin.p, F.w32.b.p, n * nb, c.s);
      vcycle<float>(c, 0, F.w32.b.p, c.bz32.p, nb);
    });
    launch_convert<double, float>(c.bz32.p, z, n * nb, c.s);
  } else {
    graph_run(c, c.preb[0][nb], [&] { vcycle<double>(c, 0, c.brin.p, c.bz64.p, nb); });
    launch_copy<double>(c.bz64.p, z, n * nb, c.s);
  }
}

// Outer flexible GCR over nb systems in lockstep (the single-system loop above, per
// vector): one batched V-cycle, one batched D apply and one batched reduction per
// iteration; the host forms each vector's coefficients from one fetch. A vector whose
// tracked residual meets tol (or whose basis breaks down) stops until the next restart,
// where the true residuals b - D x decide which vectors continue.
static void outer_fgcr_batch(mg_ctx &c, int nb, const Cx<double> *b, Cx<double> *x, double tol,
                             std::vector<GcrOut> &out) {
  Level &F = c.lv[0];
  const long long n = F.n;
  const int restart = c.p.gcr_restart;
  Cx<double> *Z = c.bZ.p, *W = c.bW.p, *r = c.br.p;
  double *h = c.bhost;
  double *hcoef = c.bhost + (size_t)c.p.max_rhs * 2 * (restart + 3);
  out.assign(nb, GcrOut{});
  auto fetch = [&](const double *dev, int count) {
    MG_CUDA(cudaMemcpyAsync(h, dev, count * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    MG_CUDA(cudaStreamSynchronize(c.s));
    for (int i = 0; i < count; ++i)
      if (std::isnan(h[i])) fail(MG_ERR_NAN, "outer GCR (batched): NaN in a reduction");
  };
  launch_zero<double>(x, n * nb, c.s);
  launch_copy<double>(b, r, n * nb, c.s);
  launch_norm2_batch(b, n, nb, c.bdots.p, c.ws, c.s);
  fetch(c.bdots.p, nb);
  std::vector<double> bn2(h, h + nb), rn2(bn2);
  unsigned int done = 0u;
  for (int v = 0; v < nb; ++v) {
    if (!(bn2[v] > 0.0)) {
      done |= 1u << v;
      out[v].converged = true;
    }
  }
  const unsigned int all = nb == 32 ? 0xffffffffu : (1u << nb) - 1u;
  int iters = 0;
  std::vector<double> nw0(nb), nw2(nb), wr(nb), wi(nb), rr(nb);
  while (done != all && iters < c.p.max_iter) {
    unsigned int act = all & ~done;
    int k = 0;
    for (; k < restart && iters < c.p.max_iter && act != 0u; ++k) {
      Cx<double> *Zk = Z + (long long)k * nb * n, *Wk = W + (long long)k * nb * n;
      precondition_batch(c, nb, r, act, Zk);
      apply_op<double>(c, 0, Zk, Wk, nullptr, 1.0, 0.0, nb);
      launch_gcr_dots_batch(W, r, k, nb, n, c.bdots.p, c.ws, c.s);
      const int stride = 2 * (k + 3);
      fetch(c.bdots.p, nb * stride);
      unsigned int cancel = 0u;
      for (int v = 0; v < nb; ++v) {
        const double *hv = h + v * stride;
        rr[v] = hv[2 * k + 4];  // |r_v|^2 before this update
        nw0[v] = hv[2 * k];
        nw2[v] = nw0[v];
        for (int j = 0; j < k; ++j) nw2[v] -= hv[2 * j] * hv[2 * j] + hv[2 * j + 1] * hv[2 * j + 1];
        wr[v] = hv[2 * k + 2];
        wi[v] = hv[2 * k + 3];
        if (((act >> v) & 1u) && k > 0 && !(nw2[v] > 0.5 * nw0[v])) cancel |= 1u << v;
      }
      if (cancel != 0u) {
        // cancellation: project those vectors once, then take fresh coefficients for them
        for (int v = 0; v < nb; ++v) {
          hcoef[4 * v] = 1.0;
          hcoef[4 * v + 1] = hcoef[4 * v + 2] = 0.0;
          hcoef[4 * v + 3] = ((cancel >> v) & 1u) ? 2.0 : 0.0;
        }
        MG_CUDA(cudaMemcpyAsync(c.bcoef.p, hcoef, 4 * nb * sizeof(double), cudaMemcpyHostToDevice, c.s));
        launch_gcr_update_batch(W, Z, k, nb, c.bdots.p, c.bcoef.p, x, r, n, c.s);
        launch_gcr_dots_batch(W, r, k, nb, n, c.bdots.p, c.ws, c.s);
        fetch(c.bdots.p, nb * stride);
        for (int v = 0; v < nb; ++v) {
          if (!((cancel >> v) & 1u)) continue;
          const double *hv = h + v * stride;
          nw0[v] = hv[2 * k];
          nw2[v] = nw0[v];
          for (int j = 0; j < k; ++j) nw2[v] -= hv[2 * j] * hv[2 * j] + hv[2 * j + 1] * hv[2 * j + 1];
        }
        // vectors without cancellation keep their first coefficients: their w is unchanged,
        // so the fresh reduction reproduced them
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
      // mode 1 projects with the betas now in bdots: fresh ones for the vectors that were
      // projected once already, the original ones (the same reduction again) for the others
      MG_CUDA(cudaMemcpyAsync(c.bcoef.p, hcoef, 4 * nb * sizeof(double), cudaMemcpyHostToDevice, c.s));
      launch_gcr_update_batch(W, Z, k, nb, c.bdots.p, c.bcoef.p, x, r, n, c.s);
      ++iters;
    }
    // true residuals r = b - D x of every unfinished vector (defect correction)
    apply_op<double>(c, 0, x, r, b, -1.0, 1.0, nb);
    launch_norm2_batch(r, n, nb, c.bdots.p, c.ws, c.s);
    fetch(c.bdots.p, nb);
    for (int v = 0; v < nb; ++v) {
      if ((done >> v) & 1u) continue;
      rn2[v] = h[v];
      out[v].rel = std::sqrt(rn2[v] / bn2[v]);
      if (out[v].rel <= tol) {
        done |= 1u << v;
        out[v].converged = true;
      }
    }
    if (k == 0) break;  // no progress possible
  }
}

// ---------------------------------------------------------------------------
// Outer flexible GCR driven on the device: one iteration (V-cycle, D apply, Gram-Schmidt
// reduction, update, control) is captured into the body of a conditional WHILE graph node,
// which the GPU replays until the control kernel clears the condition; the loops of several
// contexts sit side by side in one graph, so one launch runs all their solves with no host
// round trip per iteration. Gram-Schmidt is classical, one pass (the host-driven loop adds a
// second pass on cancellation); a restart starts a new basis from the recurrence residual,
// and the true residual b - D x is recomputed after the launch (relaunching if it misses tol).
// ---------------------------------------------------------------------------
struct DevSolve {
  mg_ctx *c = nullptr;
  const Cx<double> *b = nullptr;
  Cx<double> *x = nullptr;
  int nb = 1;                 // right-hand sides of this context (lockstep batch when > 1)
  std::vector<double> bn2;    // |b_v|^2
  std::vector<GcrOut> out;    // per vector
  int iters = 0;              // outer iterations of the context's loop
  long long kernels_per_it = 0, apps_per_it[MG_MAX_LEVELS] = {0, 0, 0, 0};
  bool coop = false;          // the loop body holds a cooperative kernel
};

static void alloc_batch(mg_ctx &c);

static void devloop_buffers(mg_ctx &c, int nb) {
  if (c.dl_ctl.p == nullptr) {
    c.dl_ctl.alloc(4);
    c.dl_st.alloc(4);
    c.dl_w.alloc(c.lv[0].n);
  }
  if (nb > 1 && (long long)c.dl_wb.n < nb * c.lv[0].n) {
    if (c.bZ.p == nullptr) alloc_batch(c);
    c.dl_wb.alloc((size_t)c.p.max_rhs * c.lv[0].n);
    c.dl_act.alloc((size_t)c.p.max_rhs);
    c.dl_stv.alloc((size_t)2 * c.p.max_rhs);
    c.dl_coef.alloc((size_t)4 * c.p.max_rhs);
  }
  pool_ready();
}

// batch: per-vector flags and residual state for a (re)start from the residuals now in c.br
static void devloop_arm_batch(mg_ctx &c, int nb, const std::vector<int> &act, const std::vector<double> &rn2,
                              const std::vector<double> &tol2, int iters_done) {
  const int ctl[4] = {iters_done, 0, 0, 0};
  std::vector<double> stv(2 * nb);
  for (int v = 0; v < nb; ++v) {
    stv[2 * v] = rn2[v];
    stv[2 * v + 1] = tol2[v];
  }
  MG_CUDA(cudaMemcpyAsync(c.dl_ctl.p, ctl, sizeof(ctl), cudaMemcpyHostToDevice, c.s));
  MG_CUDA(cudaMemcpyAsync(c.dl_act.p, act.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c.s));
  MG_CUDA(cudaMemcpyAsync(c.dl_stv.p, stv.data(), 2 * nb * sizeof(double), cudaMemcpyHostToDevice, c.s));
  MG_CUDA(cudaStreamSynchronize(c.s));
}

// counters and residual state for a (re)start from the residual now in c.orr (|r|^2 = rn2)
static void devloop_arm(mg_ctx &c, double rn2, double tol2, int iters_done) {
  const int ctl[4] = {iters_done, 0, 0, 0};
  const double st[4] = {rn2, tol2, rn2, 0.0};
  MG_CUDA(cudaMemcpyAsync(c.dl_ctl.p, ctl, sizeof(ctl), cudaMemcpyHostToDevice, c.s));
  MG_CUDA(cudaMemcpyAsync(c.dl_st.p, st, sizeof(st), cudaMemcpyHostToDevice, c.s));
  MG_CUDA(cudaStreamSynchronize(c.s));  // the host arrays are stack memory
}

// |v|^2 of a fine FP64 vector, read back
static double fine_norm2(mg_ctx &c, const Cx<double> *v) {
  double *dots = c.scal.p + kSlotOuter;
  launch_norm2<double>(v, c.lv[0].n, dots, c.ws, c.s);
  MG_CUDA(cudaMemcpyAsync(c.host, dots, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  MG_CUDA(cudaStreamSynchronize(c.s));
  return c.host[0];
}

static void devloop_capture(DevSolve &d, cudaGraph_t body, cudaGraphConditionalHandle h) {
  mg_ctx &c = *d.c;
  Level &F = c.lv[0];
  const long long n = F.n;
  const long long l0 = g_launches.load();
  long long a0[MG_MAX_LEVELS];
  for (int l = 0; l < MG_MAX_LEVELS; ++l) a0[l] = c.apps[l];
  MG_CUDA(cudaStreamBeginCaptureToGraph(c.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  (void)coop_captured_take();
  HalfCycles hc(c);
  bool ok = true;
  if (d.nb > 1) {
    // one lockstep iteration of the batch: z_v = V r_v for the iterating vectors (0 for the
    // others), w_v = D z_v, the reductions, the per-vector coefficients, the update, the control
    const int nb = d.nb, R = c.p.gcr_restart;
    c.tc_batch = c.p.precision == MG_FP32 && nb >= 8 && std::getenv("MG_NO_TC_BATCH") == nullptr;
    try {  // every vector at the context mass (no shift)
      launch_copy_active(c.br.p, c.brin.p, n, nb, c.dl_act.p, c.s);
      Cx<double> *z = c.bz64.p;
      if (c.p.precision == MG_FP32) {
        launch_convert<float, double>(c.brin.p, F.w32.b.p, n * nb, c.s);
        vcycle<float>(c, 0, F.w32.b.p, c.bz32.p, nb);
        launch_convert<double, float>(c.bz32.p, c.brin.p, n * nb, c.s);  // z in brin (r was copied already)
        z = c.brin.p;
      } else {
        vcycle<double>(c, 0, c.brin.p, c.bz64.p, nb);
      }
      apply_op<double>(c, 0, z, c.dl_wb.p, nullptr, 1.0, 0.0, nb);
      double *dots = c.bdots.p;
      launch_gcr_dots_batch_devk(c.bW.p, c.dl_wb.p, c.br.p, c.dl_ctl.p, nb, R, n, dots, c.ws, c.s);
      launch_gcr_coef_batch(dots, c.dl_ctl.p, nb, R, c.dl_act.p, c.dl_stv.p, c.dl_coef.p, c.s);
      launch_gcr_update_batch_devk(c.bW.p, c.bZ.p, c.dl_wb.p, z, c.dl_ctl.p, nb, R, dots, c.dl_coef.p, d.x, c.br.p, n,
                                   c.s);
      launch_gcr_control_batch(c.dl_ctl.p, c.dl_act.p, nb, R, c.p.max_iter, h, c.s);
    } catch (const Error &) {
      ok = false;
    }
    c.tc_batch = false;
  } else try {
    if (c.p.precision == MG_FP32) {
      launch_convert<float, double>(c.orr.p, F.w32.b.p, n, c.s);
      vcycle<float>(c, 0, F.w32.b.p, c.z32.p);
      launch_convert<double, float>(c.z32.p, c.z64.p, n, c.s);
    } else {
      vcycle<double>(c, 0, c.orr.p, c.z64.p);
    }
    apply_op<double>(c, 0, c.z64.p, c.dl_w.p);
    double *dots = c.scal.p + kSlotOuter;
    launch_gcr_dots_devk(c.oW.p, c.dl_w.p, c.orr.p, c.dl_ctl.p, c.p.gcr_restart, n, dots, c.ws, c.s);
    launch_gcr_update_devk(c.oW.p, c.oZ.p, c.dl_w.p, c.z64.p, c.dl_ctl.p, dots, c.dl_st.p, d.x, c.orr.p, n, c.s);
    launch_gcr_control(c.dl_ctl.p, c.dl_st.p, c.p.gcr_restart, c.p.max_iter, h, c.s);
  } catch (const Error &) {
    ok = false;
  }
  d.coop = coop_captured_take();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.s, &g);
  d.kernels_per_it = g_launches.load() - l0;
  g_launches.store(l0);
  for (int l = 0; l < MG_MAX_LEVELS; ++l) {
    d.apps_per_it[l] = c.apps[l] - a0[l];
    c.apps[l] = a0[l];
  }
  if (!ok || e != cudaSuccess) {
    (void)cudaGetLastError();
    fail(MG_ERR_CUDA, std::string("capture of the device-driven GCR iteration failed: ") + cudaGetErrorString(e));
  }
}

// one graph with a WHILE loop per unfinished solve, launched once on stream ls
static void devloop_launch(std::vector<DevSolve *> &act, cudaStream_t ls) {
  cudaGraph_t top = nullptr;
  MG_CUDA(cudaGraphCreate(&top, 0));
  cudaGraphExec_t exec = nullptr;
  try {
    for (DevSolve *d : act) {
      // tensor-core coarse applies of batched cycles: tune their launch shape outside the capture
      mg_ctx &c = *d->c;
      if (c.p.precision == MG_FP32 && d->nb >= 8 && std::getenv("MG_NO_TC_BATCH") == nullptr)
        for (int l = 1; l < c.p.levels; ++l)
          if (c.lv[l].Ypk.p != nullptr)
            launch_coarse_apply_tc(c.lv[l].Ypk.p, c.lv[l].w32.r.p, c.lv[l].w32.Ar.p, c.lv[l].geo, d->nb, nullptr, 1.0,
                                   0.0, nullptr, c.s);
    }
    // loops that hold cooperative kernels run one after another (their grid barriers need the
    // whole GPU); the others run beside them
    cudaGraphNode_t last_coop = nullptr;
    bool any_coop = false;
    for (DevSolve *d : act) {
      cudaGraphConditionalHandle h;
      MG_CUDA(cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      MG_CUDA(cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &np));
      devloop_capture(*d, np.conditional.phGraph_out[0], h);
      if (d->coop) {
        if (last_coop != nullptr) MG_CUDA(cudaGraphAddDependencies(top, &last_coop, &node, nullptr, 1));
        last_coop = node;
        any_coop = true;
      }
    }
    MG_CUDA(cudaGraphInstantiate(&exec, top, 0));
    for (DevSolve *d : act) {  // the launch stream waits for every context's queued work
      MG_CUDA(cudaEventRecord(d->c->ev, d->c->s));
      MG_CUDA(cudaStreamWaitEvent(ls, d->c->ev, 0));
    }
    if (any_coop)
      coop_graph_launch(exec, ls);
    else
      MG_CUDA(cudaGraphLaunch(exec, ls));
    MG_CUDA(cudaStreamSynchronize(ls));
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(top);
    throw;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(top);
}

static void devloop_solve(std::vector<DevSolve> &v, double tol) {
  const double tol2 = tol * tol;
  for (DevSolve &d : v) {
    mg_ctx &c = *d.c;
    check_fresh(c);
    devloop_buffers(c, d.nb);
    for (long long &a : c.apps) a = 0;
    collect_coarsest(c);
    const long long n = c.lv[0].n;
    d.out.assign(d.nb, GcrOut{});
    d.bn2.assign(d.nb, 0.0);
    d.iters = 0;
    launch_zero<double>(d.x, n * d.nb, c.s);
    if (d.nb == 1) {
      launch_copy<double>(d.b, c.orr.p, n, c.s);
      d.bn2[0] = fine_norm2(c, d.b);
      if (!(d.bn2[0] > 0.0)) {
        d.out[0].converged = true;
        continue;
      }
      devloop_arm(c, d.bn2[0], tol2 * d.bn2[0], 0);
    } else {
      launch_copy<double>(d.b, c.br.p, n * d.nb, c.s);
      launch_norm2_batch(d.b, n, d.nb, c.bdots.p, c.ws, c.s);
      MG_CUDA(cudaMemcpyAsync(d.bn2.data(), c.bdots.p, d.nb * sizeof(double), cudaMemcpyDeviceToHost, c.s));
      MG_CUDA(cudaStreamSynchronize(c.s));
      std::vector<int> act(d.nb);
      std::vector<double> t2(d.nb);
      for (int q = 0; q < d.nb; ++q) {
        act[q] = d.bn2[q] > 0.0 ? 1 : 0;
        d.out[q].converged = !act[q];
        t2[q] = tol2 * d.bn2[q];
      }
      devloop_arm_batch(c, d.nb, act, d.bn2, t2, 0);
    }
  }
  auto open = [](const DevSolve &d) {
    for (const GcrOut &o : d.out)
      if (!o.converged) return d.iters < d.c->p.max_iter;
    return false;
  };
  for (int round = 0; round < 8; ++round) {
    std::vector<DevSolve *> act;
    for (DevSolve &d : v)
      if (open(d)) act.push_back(&d);
    if (act.empty()) break;
    devloop_launch(act, act[0]->c->s);
    MG_CUDA(cudaEventRecord(act[0]->c->ev, act[0]->c->s));
    for (DevSolve *d : act) {
      mg_ctx &c = *d->c;
      const long long n = c.lv[0].n;
      MG_CUDA(cudaStreamWaitEvent(c.s, act[0]->c->ev, 0));
      int ctl[4];
      MG_CUDA(cudaMemcpyAsync(ctl, c.dl_ctl.p, sizeof(ctl), cudaMemcpyDeviceToHost, c.s));
      MG_CUDA(cudaStreamSynchronize(c.s));
      const long long done = ctl[0] - d->iters;
      d->iters = ctl[0];
      g_launches.fetch_add(done * d->kernels_per_it);
      for (int l = 0; l < MG_MAX_LEVELS; ++l) c.apps[l] += done * d->apps_per_it[l];
      // true residuals (defect correction)
      if (d->nb == 1) {
        GcrOut &o = d->out[0];
        o.iters = d->iters;
        apply_op<double>(c, 0, d->x, c.orr.p, d->b, -1.0, 1.0);
        const double rn2 = fine_norm2(c, c.orr.p);
        if (!std::isfinite(rn2)) fail(MG_ERR_NAN, "outer GCR (device loop): NaN in the true residual");
        o.rel = std::sqrt(rn2 / d->bn2[0]);
        o.converged = o.rel <= tol;
        if (!o.converged) {
          if (ctl[2] == 3 && done <= 1) d->iters = c.p.max_iter;  // no progress possible: give up
          else devloop_arm(c, rn2, tol2 * d->bn2[0], ctl[0]);
        }
      } else {
        apply_op<double>(c, 0, d->x, c.br.p, d->b, -1.0, 1.0, d->nb);
        launch_norm2_batch(c.br.p, n, d->nb, c.bdots.p, c.ws, c.s);
        std::vector<double> rn2(d->nb), t2(d->nb);
        MG_CUDA(cudaMemcpyAsync(rn2.data(), c.bdots.p, d->nb * sizeof(double), cudaMemcpyDeviceToHost, c.s));
        MG_CUDA(cudaStreamSynchronize(c.s));
        std::vector<int> more(d->nb, 0);
        bool any = false;
        for (int q = 0; q < d->nb; ++q) {
          GcrOut &o = d->out[q];
          t2[q] = tol2 * d->bn2[q];
          if (o.converged && d->bn2[q] == 0.0) continue;
          if (!std::isfinite(rn2[q])) fail(MG_ERR_NAN, "outer GCR (device loop, batch): NaN in a true residual");
          o.iters = d->iters;
          o.rel = std::sqrt(rn2[q] / d->bn2[q]);
          o.converged = o.rel <= tol;
          more[q] = o.converged ? 0 : 1;
          any = any || more[q];
        }
        if (any) {
          if (done <= 0) d->iters = c.p.max_iter;  // no progress possible: give up
          else devloop_arm_batch(c, d->nb, more, rn2, t2, ctl[0]);
        }
      }
    }
  }
  for (DevSolve &d : v) {
    mg_ctx &c = *d.c;
    c.coarsest_iters = collect_coarsest(c);
    if (!c.use_lu) c.apps[c.p.levels - 1] += c.coarsest_iters;
  }
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static void prepare_coarsest(mg_ctx &c) {
  Level &L = c.lv.back();
  std::fill(c.slot_shift.begin(), c.slot_shift.end(), std::nan(""));  // batched slots are stale
  if (!c.use_lu) {
    prepare_coarsest_gcr(L.Y64.p, L.geo, L.nint, c.cg_Minv.p, c.cg_Yt.p, c.cg_work.p, c.cg_info.p, c.s);
    if (c.cg_Yt32.p != nullptr) launch_convert<float, double>(c.cg_Yt.p, c.cg_Yt32.p, c.cg_Yt.n, c.s);
    if (c.cl_Yr.p != nullptr) launch_transpose_blocks8(c.cg_Yt32.p, c.cl_Yr.p, (long long)c.cg_Yt.n / 64, c.s);
    int info = 0;
    MG_CUDA(cudaMemcpyAsync(&info, c.cg_info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    MG_CUDA(cudaStreamSynchronize(c.s));
    if (info != 0) fail(MG_ERR_NAN, "coarsest level: a self block is singular");
    return;
  }
  launch_dense_from_stencil(L.Y64.p, c.LU.p, L.geo, L.nint, c.s);
  lu_factor(c.LU.p, c.nc, c.ipiv.p, c.info.p, c.s);
  int info = 0;
  MG_CUDA(cudaMemcpyAsync(&info, c.info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  MG_CUDA(cudaStreamSynchronize(c.s));
  if (info != 0) fail(MG_ERR_NAN, "coarsest LU: zero pivot at column " + std::to_string(info - 1));
}

// block Gram-Schmidt of the level's vectors and the Galerkin operator of l+1
static void build_level(mg_ctx &c, int l) {
  Level &L = c.lv[l];
  Level &C = c.lv[l + 1];
  launch_block_mgs(L.nullv.p, L.n, L.V64.p, L.bg, L.Nv, L.mgs_min.p, c.s);
  if (l == 0)
    launch_galerkin_wilson(c.U64.p, diag_of(c), L.V64.p, C.Y64.p, L.bg, L.Nv, c.s, galerkin_f32(c));
  else
    launch_galerkin_stencil(L.Y64.p, L.V64.p, C.Y64.p, L.bg, L.Nv, c.s, galerkin_f32(c));
}

// One adaptive-setup level in the context precision. In FP32 mode the relaxation
// and the adaptive V-cycles run in FP32 on an FP32 copy of the vectors, which are
// kept in FP64 for the block Gram-Schmidt and the Galerkin build.
template <typename R>
static void relax_and_adapt(mg_ctx &c, int l, int pass);

template <>
void relax_and_adapt<double>(mg_ctx &c, int l, int pass) {
  Level &L = c.lv[l];
  const long long n = L.n;
  const int nv = L.Nv;
  Cx<double> *V = L.nullv.p;
  if (pass == 1) {
    apply_op<double>(c, l, V, L.tA.p, nullptr, -1.0, 0.0, nv);  // r = -A v
    smooth<double>(c, l, L.tA.p, V, c.p.nu_setup, true, nv);
  } else {
    apply_op<double>(c, l, V, L.tA.p, nullptr, 1.0, 0.0, nv);
    graph_run(c, c.setup_vc[l], [&] { vcycle<double>(c, l, L.tA.p, L.tB.p, nv); });
    launch_xmy<double>(V, L.tB.p, n * nv, c.s);  // tB = v - V(A v)
    launch_copy<double>(L.tB.p, V, n * nv, c.s);
  }
}

template <>
void relax_and_adapt<float>(mg_ctx &c, int l, int pass) {
  Level &L = c.lv[l];
  const long long n = L.n;
  const int nv = L.Nv;
  launch_convert<float, double>(L.nullv.p, L.sv.p, n * nv, c.s);
  if (pass == 1) {
    apply_op<float>(c, l, L.sv.p, L.sA.p, nullptr, -1.0, 0.0, nv);
    smooth<float>(c, l, L.sA.p, L.sv.p, c.p.nu_setup, true, nv);
  } else {
    apply_op<float>(c, l, L.sv.p, L.sA.p, nullptr, 1.0, 0.0, nv);
    graph_run(c, c.setup_vc[l], [&] { vcycle<float>(c, l, L.sA.p, L.sB.p, nv); });
    launch_xmy<float>(L.sv.p, L.sB.p, n * nv, c.s);
    launch_copy<float>(L.sB.p, L.sv.p, n * nv, c.s);
  }
  launch_convert<double, float>(L.sv.p, L.nullv.p, n * nv, c.s);
}

static void setup_level(mg_ctx &c, int l, bool full) {
  Level &L = c.lv[l];
  const long long n = L.n;
  // pass 1: random vectors relaxed on A x = 0 (nu_setup MR iterations from x = v: the
  // corrections solve A d = -A v from d = 0); later passes v <- v - V(A v), one V-cycle
  // on the homogeneous problem. All Nv vectors form one batch.
  Cx<double> *V = L.nullv.p;
  const int nv = L.Nv;
  const bool f32 = c.p.precision == MG_FP32;
  for (int k = 0; k < nv; ++k) launch_gaussian(V + (long long)k * n, n, c.p.seed, k, l, c.s);
  if (f32)
    relax_and_adapt<float>(c, l, 1);
  else
    relax_and_adapt<double>(c, l, 1);
  const int n_pass = full ? c.p.n_pass : 1;
  for (int pass = 1; pass <= n_pass; ++pass) {
    if (pass > 1) {
      if (f32)
        relax_and_adapt<float>(c, l, pass);
      else
        relax_and_adapt<double>(c, l, pass);
    }
    build_level(c, l);
    if (f32) {
      launch_convert<float, double>(L.V64.p, L.V32.p, L.V64.n, c.s);
      Level &C = c.lv[l + 1];
      refresh_y32(c, l + 1);
    }
    if (l + 1 == c.p.levels - 1)
      prepare_coarsest(c);
    else
      setup_level(c, l + 1, full && pass == n_pass);
  }
  L.stale = false;
}

static void make_fp32_copies(mg_ctx &c) {
  if (c.p.precision != MG_FP32) return;
  launch_convert<float, double>(c.U64.p, c.U32.p, c.lv[0].geo.nsites * 2, c.s);
  for (size_t l = 0; l < c.lv.size(); ++l) {
    Level &L = c.lv[l];
    if (l + 1 < c.lv.size()) launch_convert<float, double>(L.V64.p, L.V32.p, L.V64.n, c.s);
    if (l > 0) refresh_y32(c, (int)l);
  }
}

static void validate(const mg_geom *g, const mg_params *p) {
  if (!g || !p) fail(MG_ERR_INVALID_ARG, "null geometry or parameters");
  if (g->d != 2) fail(MG_ERR_UNSUPPORTED, "only d = 2 is built");
  if (g->Nc != 1) fail(MG_ERR_UNSUPPORTED, "only Nc = 1 (U(1)) is built");
  if (g->dims[0] < 2 || g->dims[1] < 2) fail(MG_ERR_INVALID_ARG, "lattice extents must be >= 2");
  if ((long long)g->dims[0] * g->dims[1] * 8 >= (1LL << 31))
    fail(MG_ERR_UNSUPPORTED, "lattices are limited to fewer than 2^28 sites (32-bit dof indexing)");
  if (p->levels < 2 || p->levels > MG_MAX_LEVELS) fail(MG_ERR_INVALID_ARG, "levels must be in [2, 4]");
  if (p->precision != MG_FP64 && p->precision != MG_FP32 && p->precision != MG_FP16)
    fail(MG_ERR_INVALID_ARG, "unknown precision");
  if (p->n_pass < 1 || p->nu_pre < 0 || p->nu_post < 0 || p->nu_setup < 0) fail(MG_ERR_INVALID_ARG, "bad counts");
  if (p->gcr_restart < 1 || p->gcr_restart > 128) fail(MG_ERR_INVALID_ARG, "gcr_restart must be in [1, 128]");
  if (p->coarsest_restart < 1 || p->coarsest_restart > 32)
    fail(MG_ERR_INVALID_ARG, "coarsest_restart must be in [1, 32]");
  if (p->max_iter < 1 || p->coarsest_max_iter < 1) fail(MG_ERR_INVALID_ARG, "iteration limits must be >= 1");
  if (p->max_rhs < 1 || p->max_rhs > kMaxBatch) fail(MG_ERR_INVALID_ARG, "max_rhs must be in [1, 32]");
  int L0 = g->dims[0], L1 = g->dims[1], nint = 2;
  for (int l = 0; l + 1 < p->levels; ++l) {
    const int B0 = p->block[l][0], B1 = p->block[l][1];
    if (B0 < 1 || B1 < 1 || L0 % B0 || L1 % B1)
      fail(MG_ERR_INVALID_ARG, "level " + std::to_string(l) + ": extents not divisible by the block");
    const int Nb = B0 * B1 * nint;
    if (p->Nv[l] < 1 || p->Nv[l] > Nb || p->Nv[l] > 32)
      fail(MG_ERR_INVALID_ARG, "level " + std::to_string(l) + ": Nv must be in [1, min(block dofs, 32)]");
    L0 /= B0;
    L1 /= B1;
    nint = p->Nv[l];
  }
}

// order the context stream after the caller's stream (work the caller queued
// before this call, e.g. writing the inputs, completes first)
static void enter(mg_ctx &c) {
  MG_CUDA(cudaEventRecord(c.ev, c.user));
  MG_CUDA(cudaStreamWaitEvent(c.s, c.ev, 0));
}

// buffers of batched solves (allocated at setup when max_rhs > 1, else on the first
// mg_solve_batch call, before any batched graph is captured)
static void alloc_batch(mg_ctx &c) {
  const Level &F = c.lv[0];
  const Level &Cst = c.lv.back();
  const bool f32 = c.p.precision == MG_FP32;
  const size_t nr = (size_t)c.p.max_rhs;
  const size_t m2 = (size_t)Cst.geo.nsites * Cst.nint * Cst.nint;
  if (c.use_lu) {
    c.bLU.resize(nr);
    c.bipiv.resize(nr);
  } else {
    c.bMinv.alloc(nr * m2);
    if (!c.cg_batch) c.bYt.alloc(nr * 5 * m2);
  }
  c.bZ.alloc((size_t)c.p.gcr_restart * nr * F.n);
  c.bW.alloc((size_t)c.p.gcr_restart * nr * F.n);
  c.br.alloc(nr * F.n);
  c.brin.alloc(nr * F.n);
  if (f32)
    c.bz32.alloc(nr * F.n);
  else
    c.bz64.alloc(nr * F.n);
  c.bdots.alloc(nr * 2 * (c.p.gcr_restart + 3));
  c.bcoef.alloc(nr * 4);
  MG_CUDA(cudaMallocHost(&c.bhost, (nr * 2 * (c.p.gcr_restart + 3) + nr * 4) * sizeof(double)));
  pool_ready();
}

// the parameters as the caller gave them (an MG_FP16 context runs as FP32 internally)
static mg_params user_params(const mg_ctx &c) {
  mg_params p = c.p;
  if (c.half_fine) p.precision = MG_FP16;
  return p;
}

// FP32 and half copies of the fine links for the cycles
static void make_link_copies(mg_ctx &c) {
  if (c.p.precision == MG_FP32) launch_convert<float, double>(c.U64.p, c.U32.p, c.U64.n, c.s);
  if (c.half_fine) launch_half_convert(2, MG_FP64, c.U64.p, c.U16.p, c.lv[0].geo.nsites, c.s);
}

static std::unique_ptr<mg_ctx> create(const mg_geom *g, double m, const mg_params *p, void *stream) {
  validate(g, p);
  auto c = std::make_unique<mg_ctx>();
  c->geom = *g;
  c->p = *p;
  // MG_FP16 is an FP32 context whose solve cycles keep the fine level in half storage
  c->half_fine = p->precision == MG_FP16;
  if (c->half_fine) c->p.precision = MG_FP32;
  c->m = m;
  c->user = static_cast<cudaStream_t>(stream);
  MG_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
  MG_CUDA(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
  enter(*c);
  c->graphs_ok = std::getenv("MG_NO_GRAPHS") == nullptr;
  MG_CUDA(cudaMallocHost(&c->host, 512 * sizeof(double)));
  c->lv.resize(p->levels);
  c->nbatch = 1;
  for (int l = 0; l + 1 < p->levels; ++l) c->nbatch = std::max(c->nbatch, p->Nv[l]);
  c->nbatch = std::max(c->nbatch, p->max_rhs);
  int L0 = g->dims[0], L1 = g->dims[1], nint = 2;
  const bool f32 = c->p.precision == MG_FP32;
  for (int l = 0; l < p->levels; ++l) {
    Level &L = c->lv[l];
    L.geo = Geo2{L0, L1, (long long)L0 * L1};
    L.nint = nint;
    L.n = L.geo.nsites * nint;
    if (l > 0) {
      L.Y64.alloc(L.geo.nsites * 5 * (size_t)nint * nint);
      if (f32) L.Y32.alloc(L.Y64.n);
      if (f32 && nint == 8) L.Ypk.alloc(L.geo.nsites * 5 * 32);
    }
    const size_t nb = (size_t)c->nbatch;
    L.w64.b.alloc(L.n * nb);
    L.w64.x.alloc(L.n * nb);
    L.w64.r.alloc(L.n * nb);
    L.w64.Ar.alloc(L.n * nb);
    if (f32) {
      L.w32.b.alloc(L.n * nb);
      L.w32.x.alloc(L.n * nb);
      L.w32.r.alloc(L.n * nb);
      L.w32.Ar.alloc(L.n * nb);
    }
    if (l + 1 < p->levels) {
      const int B0 = p->block[l][0], B1 = p->block[l][1];
      L.Nv = p->Nv[l];
      L.bg = BlockGeo{L0, L1, B0, B1, L0 / B0, L1 / B1, B0 * B1, nint, B0 * B1 * nint,
                      (long long)(L0 / B0) * (L1 / B1)};
      L.nullv.alloc((size_t)L.Nv * L.n);
      L.V64.alloc((size_t)L.Nv * L.n);
      if (f32) L.V32.alloc(L.V64.n);
      L.mgs_min.alloc(L.bg.nblocks);
      L.tA.alloc(L.n * (size_t)L.Nv);
      L.tB.alloc(L.n * (size_t)L.Nv);
      if (f32) {
        L.sv.alloc(L.n * (size_t)L.Nv);
        L.sA.alloc(L.n * (size_t)L.Nv);
        L.sB.alloc(L.n * (size_t)L.Nv);
      }
      L0 /= B0;
      L1 /= B1;
      nint = L.Nv;
    }
  }
  const Level &F = c->lv[0];
  for (int l = 0; l < p->levels; ++l) {
    Level &L = c->lv[l];
    L.w64.r2.alloc(L.n * (size_t)c->nbatch);
    L.w64.Ar2.alloc(L.n * (size_t)c->nbatch);
    if (f32) {
      L.w32.r2.alloc(L.n * (size_t)c->nbatch);
      L.w32.Ar2.alloc(L.n * (size_t)c->nbatch);
    }
  }
  c->U64.alloc(F.geo.nsites * 2);
  if (f32) c->U32.alloc(F.geo.nsites * 2);
  if (c->half_fine) {
    c->U16.alloc(F.geo.nsites * 2);
    for (int i = 0; i < 2; ++i) {
      c->hr[i].alloc(F.geo.nsites * 3 * (size_t)p->max_rhs);
      c->hA[i].alloc(F.geo.nsites * 3 * (size_t)p->max_rhs);
    }
  }
  // coarsest
  const Level &Cst = c->lv.back();
  c->nc = (int)Cst.n;
  c->use_lu = Cst.n <= p->coarsest_lu_max;
  if (c->use_lu) {
    c->LU.alloc((size_t)Cst.n * Cst.n);
    c->lu_work.alloc(Cst.n);
    c->ipiv.alloc(Cst.n);
    c->info.alloc(1);
  } else {
    c->cZ.alloc((size_t)p->coarsest_restart * Cst.n);
    c->cW.alloc((size_t)p->coarsest_restart * Cst.n);
    c->cr.alloc(Cst.n);
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    c->cg_grid = coarsest_gcr_grid(dev);
    c->cg_smem = coarsest_smem_fits(Cst.geo, Cst.nint, p->coarsest_restart, c->cg_grid) &&
                 std::getenv("MG_NO_SMEM_COARSEST") == nullptr;
    c->cg_partials.alloc((size_t)c->cg_grid * kCoarsestSlots);
    c->cg_bar.alloc(2);
    c->cg_out.alloc(3);
    c->cg_rel.alloc(1);
    c->cg_Minv.alloc((size_t)Cst.geo.nsites * Cst.nint * Cst.nint);
    c->cg_Yt.alloc((size_t)Cst.geo.nsites * 5 * Cst.nint * Cst.nint);
    // mixed precision: store and apply A M in FP32 when the requested coarsest accuracy is far
    // above FP32 rounding (the Krylov vectors and reductions stay FP64)
    c->cg_cluster = f32 && p->coarsest_tol >= 1e-5 && std::getenv("MG_NO_CLUSTER_COARSEST") == nullptr &&
                    coarsest_cluster_fits(Cst.geo, Cst.nint, p->coarsest_restart);
    c->cg_large32 = f32 && !c->cg_smem && !c->cg_cluster && p->coarsest_tol >= 1e-5 &&
                    std::getenv("MG_FP64_COARSEST_STENCIL") == nullptr;
    if ((f32 && c->cg_smem && p->coarsest_tol >= 1e-5 && std::getenv("MG_FP64_COARSEST_STENCIL") == nullptr) ||
        c->cg_cluster || c->cg_large32)
      c->cg_Yt32.alloc(c->cg_Yt.n);
    if (c->cg_large32) {
      c->cZ32.alloc((size_t)p->coarsest_restart * Cst.n);
      c->cW32.alloc((size_t)p->coarsest_restart * Cst.n);
      c->cr32.alloc(Cst.n);
      c->cy32.alloc(Cst.n);
    }
    if (c->cg_cluster) {
      c->cl_Yr.alloc(c->cg_Yt.n);
      c->cl_rpub.alloc((size_t)c->nbatch * Cst.n);
      c->cl_ypub.alloc((size_t)c->nbatch * Cst.n);
    }
    c->cg_work.alloc((size_t)Cst.geo.nsites * 2 * Cst.nint * Cst.nint);
    c->cg_y.alloc(Cst.n);
    c->cg_info.alloc(1);
    c->cg_batch = c->cg_smem && coarsest_batch_fits(Cst.geo, Cst.nint, p->coarsest_restart, c->cg_grid) &&
                  std::getenv("MG_NO_BATCH_COARSEST") == nullptr;
    if (c->cg_batch) {
      c->cgb_u.alloc((size_t)kCoarsestBatchVecs * Cst.n);
      c->cgb_x.alloc((size_t)kCoarsestBatchVecs * Cst.n);
      c->cgb_partials.alloc((size_t)coarsest_batch_partials(c->cg_grid));
    }
  }
  if (f32) {
    c->cb.alloc(Cst.n * (size_t)c->nbatch);
    c->cx.alloc(Cst.n * (size_t)c->nbatch);
    c->z32.alloc(F.n);
  }
  // batched solves
  c->shift_dev.alloc(std::max(p->max_rhs, 1));
  c->slot_shift.assign(p->max_rhs, std::nan(""));
  c->preb[0].resize(p->max_rhs + 1);
  c->preb[1].resize(p->max_rhs + 1);
  if (p->max_rhs > 1) alloc_batch(*c);

  // outer
  c->z64.alloc(F.n);
  c->oZ.alloc((size_t)p->gcr_restart * F.n);
  c->oW.alloc((size_t)p->gcr_restart * F.n);
  c->orr.alloc(F.n);
  // reductions
  c->ws.max_blocks = 152 * 8;
  // the fused MR kernels reduce over one block per 256 sites (fine) or dofs (coarse)
  long long cap = (long long)c->ws.max_blocks * 4;
  for (int l = 0; l < p->levels; ++l) {
    // fine: a thread per site; coarse N = 8: four threads per dof; other N: a thread per dof
    const long long units = l == 0 ? c->lv[l].geo.nsites : (c->lv[l].nint == 8 ? 4 : 1) * c->lv[l].n;
    cap = std::max(cap, 3 * ((units + 255) / 256) * c->nbatch);
  }
  cap = std::max(cap, 2LL * (p->gcr_restart + 3) * p->max_rhs * 64);
  c->partials.alloc((size_t)cap + 16);
  c->ws.capacity = cap;
  c->mrpart[0].alloc((size_t)cap);
  c->mrpart[1].alloc((size_t)cap);
  c->ws.tickets = std::max(160, (p->gcr_restart + 3) * p->max_rhs);
  c->tickets.alloc((size_t)c->ws.tickets);
  pool_ready();  // every buffer above is usable on the context stream from here
  if (!c->use_lu) MG_CUDA(cudaMemsetAsync(c->cg_out.p, 0, 3 * sizeof(int), c->s));
  MG_CUDA(cudaMemsetAsync(c->tickets.p, 0, c->ws.tickets * sizeof(unsigned int), c->s));
  c->scal.alloc(kSlotCount);
  MG_CUDA(cudaMemsetAsync(c->scal.p, 0, kSlotCount * sizeof(double), c->s));
  c->ws.partials = c->partials.p;
  c->ws.ticket = c->tickets.p;
  return c;
}

}  // namespace mg

// ===========================================================================
// C ABI
// ===========================================================================
using namespace mg;

template <typename F>
static int guarded(F &&f) {
  try {
    f();
    t_last_error.clear();
    return MG_OK;
  } catch (const Error &e) {
    t_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    t_last_error = "host allocation failed";
    return MG_ERR_OOM;
  } catch (...) {
    t_last_error = "unexpected exception";
    return MG_ERR_CUDA;
  }
}

// every call on a context first orders the context stream after the caller's stream
static void need_ctx(mg_ctx *c) {
  if (!c) fail(MG_ERR_INVALID_ARG, "null context");
  enter(*c);
}
static void need_level(mg_ctx *c, int l, bool needs_next) {
  need_ctx(c);
  if (l < 0 || l >= c->p.levels || (needs_next && l + 1 >= c->p.levels))
    fail(MG_ERR_INVALID_ARG, "level out of range");
}
static void need_ptr(const void *p) {
  if (!p) fail(MG_ERR_INVALID_ARG, "null pointer");
}

static double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Asymptotic convergence factor of the stationary multigrid iteration on the homogeneous
// problem, e <- e - V(D e) (the error propagator the adaptive passes apply): from a Philox
// Gaussian e_0, (|e_steps| / |e_1|)^(1 / (steps - 1)). Uses the level-0 setup temporaries.
static double convergence_rate(mg_ctx &c, int steps, uint64_t seed) {
  Level &F = c.lv[0];
  const long long n = F.n;
  if ((long long)F.tA.n < 2 * n) fail(MG_ERR_STATE, "rate measurement needs Nv >= 2 on level 0");
  Cx<double> *e = F.tA.p, *t = F.tB.p, *z = F.tA.p + n;
  double *dots = c.scal.p + kSlotOuter;
  auto norm = [&](const Cx<double> *v) {
    launch_norm2<double>(v, n, dots, c.ws, c.s);
    MG_CUDA(cudaMemcpyAsync(c.host, dots, sizeof(double), cudaMemcpyDeviceToHost, c.s));
    MG_CUDA(cudaStreamSynchronize(c.s));
    return std::sqrt(c.host[0]);
  };
  launch_gaussian(e, n, seed, 0, 0x5241, c.s);
  double n1 = 0.0, nl = 0.0;
  for (int i = 1; i <= steps; ++i) {
    apply_op<double>(c, 0, e, t);
    precondition(c, t, z);
    launch_xmy<double>(e, z, n, c.s);  // z = e - V(D e)
    launch_copy<double>(z, e, n, c.s);
    if (i == 1) n1 = norm(e);
    if (i == steps) nl = norm(e);
  }
  if (!(n1 > 0.0) || !std::isfinite(nl)) fail(MG_ERR_NAN, "rate measurement: degenerate error vector");
  return std::pow(nl / n1, 1.0 / (steps - 1));
}

// A context at mass m on links U: the full adaptive setup, or, with saved vectors
// (`vectors[l]`: the host copy of level l's near-null vectors), the rebuild of every
// level from them (block Gram-Schmidt, Galerkin operators, coarsest preparation) with no
// relaxation or adaptive pass.
static std::unique_ptr<mg_ctx> make_context(const mg_geom *g, const void *U, double m, const mg_params *p,
                                            void *stream, const std::vector<std::vector<Cx<double>>> *vectors) {
  const auto t0 = std::chrono::steady_clock::now();
  if (g != nullptr && g->d == 4) {
    validate4(g, p);
    auto c = std::make_unique<mg_ctx>();
    c->geom = *g;
    c->p = *p;
    c->m = m;
    c->user = static_cast<cudaStream_t>(stream);
    MG_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
    MG_CUDA(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
    enter(*c);
    c->e4 = engine4_create(g, U, m, p, c->s, vectors == nullptr);
    if (vectors != nullptr) {
      const std::vector<Cx<double>> &v = (*vectors)[0];
      if ((long long)v.size() != engine4_null_vector_count(*c->e4))
        fail(MG_ERR_INVALID_ARG, "saved setup: vector count does not match the hierarchy");
      DevBuf<Cx<double>> tmp;
      tmp.alloc(v.size());
      pool_ready();
      MG_CUDA(cudaMemcpyAsync(tmp.p, v.data(), v.size() * sizeof(Cx<double>), cudaMemcpyHostToDevice, c->s));
      engine4_build_level(*c->e4, tmp.p);
    }
    MG_CUDA(cudaStreamSynchronize(c->s));
    c->setup_s = seconds_since(t0);
    return c;
  }
  auto c = create(g, m, p, stream);
  MG_CUDA(cudaMemcpyAsync(c->U64.p, U, c->U64.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
  make_link_copies(*c);
  if (vectors == nullptr) {
    setup_level(*c, 0, true);
  } else {
    for (int l = 0; l + 1 < c->p.levels; ++l) {
      Level &L = c->lv[l];
      const std::vector<Cx<double>> &v = (*vectors)[l];
      if (v.size() != L.nullv.n) fail(MG_ERR_INVALID_ARG, "saved setup: vector count does not match the hierarchy");
      MG_CUDA(cudaMemcpyAsync(L.nullv.p, v.data(), v.size() * sizeof(Cx<double>), cudaMemcpyHostToDevice, c->s));
      build_level(*c, l);
      if (l + 2 == c->p.levels) prepare_coarsest(*c);
    }
  }
  make_fp32_copies(*c);
  collect_coarsest(*c);
  MG_CUDA(cudaStreamSynchronize(c->s));
  c->setup_s = seconds_since(t0);
  return c;
}

// ---- saved setups: header, then the near-null vectors of every level ----
struct SetupFileHeader {
  char magic[8];
  uint32_t version, levels_saved;
  mg_geom g;
  mg_params p;
  double m;
  uint64_t links_digest, payload_digest;
  uint64_t count[MG_MAX_LEVELS];  // complex128 elements of each level's vectors
};
static const char kSetupMagic[8] = {'M', 'G', 'S', 'E', 'T', 'U', 'P', '1'};

// 64-bit FNV-1a (Fowler, Noll, Vo) over bytes
static uint64_t fnv1a(const void *data, size_t n, uint64_t h = 14695981039346656037ULL) {
  const unsigned char *q = static_cast<const unsigned char *>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= q[i];
    h *= 1099511628211ULL;
  }
  return h;
}

static size_t link_bytes(const mg_geom &g) {
  long long vol = 1;
  for (int mu = 0; mu < g.d; ++mu) vol *= g.dims[mu];
  return (size_t)vol * g.d * g.Nc * g.Nc * sizeof(Cx<double>);
}

static uint64_t device_digest(const void *dev, size_t bytes, cudaStream_t s) {
  std::vector<unsigned char> h(bytes);
  MG_CUDA(cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return fnv1a(h.data(), bytes);
}

extern "C" {

void mg_default_params(mg_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->levels = 2;
  for (int l = 0; l < MG_MAX_LEVELS - 1; ++l) {
    p->block[l][0] = 4;
    p->block[l][1] = 4;
    p->block[l][2] = 1;
    p->block[l][3] = 1;
    p->Nv[l] = 8;
  }
  p->nu_pre = 4;
  p->nu_post = 4;
  p->omega = 0.8;
  p->n_pass = 5;
  p->nu_setup = 8;
  p->gcr_restart = 16;
  p->max_iter = 500;
  p->coarsest_lu_max = 2048;
  p->coarsest_tol = 1e-12;
  p->coarsest_restart = 16;
  p->coarsest_max_iter = 20000;
  p->precision = MG_FP64;
  p->seed = 20070704ULL;
  p->max_rhs = 1;
}

const char *mg_last_error(void) { return t_last_error.c_str(); }

long long mg_kernel_launches(void) { return g_launches.load(); }

int mg_setup(mg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, void *stream) {
  return guarded([&] {
    if (!ctx) fail(MG_ERR_INVALID_ARG, "null context out-pointer");
    *ctx = nullptr;
    need_ptr(U);
    *ctx = make_context(g, U, m, p, stream, nullptr).release();
  });
}

int mg_setup_batch(int count, mg_ctx **ctx, const mg_geom *g, const void *const *U, const double *m,
                   const mg_params *p, void *stream) {
  return guarded([&] {
    if (count < 1) fail(MG_ERR_INVALID_ARG, "count must be >= 1");
    if (!ctx || !g || !U || !m || !p) fail(MG_ERR_INVALID_ARG, "null array");
    for (int i = 0; i < count; ++i) ctx[i] = nullptr;
    for (int i = 0; i < count; ++i) need_ptr(U[i]);
    std::vector<std::unique_ptr<mg_ctx>> made(count);
    std::vector<Error> errs(count, Error{MG_OK, ""});
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));  // the workers set up on the caller's device
    // one host thread per configuration (at most 16 at a time); each setup runs on its
    // own context stream, so the GPU overlaps them
    const int width = std::min(count, 16);
    for (int i0 = 0; i0 < count; i0 += width) {
      std::vector<std::thread> th;
      for (int i = i0; i < std::min(count, i0 + width); ++i)
        th.emplace_back([&, i] {
          try {
            MG_CUDA(cudaSetDevice(dev));
            made[i] = make_context(&g[i], U[i], m[i], &p[i], stream, nullptr);
          } catch (const Error &e) {
            errs[i] = e;
          } catch (const std::bad_alloc &) {
            errs[i] = Error{MG_ERR_OOM, "host allocation failed"};
          } catch (...) {
            errs[i] = Error{MG_ERR_CUDA, "unexpected exception"};
          }
        });
      for (auto &t : th) t.join();
    }
    for (int i = 0; i < count; ++i)
      if (errs[i].code != MG_OK) throw Error{errs[i].code, "configuration " + std::to_string(i) + ": " + errs[i].msg};
    for (int i = 0; i < count; ++i) ctx[i] = made[i].release();
  });
}

int mg_solve(mg_ctx *c, const void *chi, void *psi, int nrhs, double tol, mg_stats *st) {
  if (nrhs != 1) {
    if (nrhs < 1) {
      t_last_error = "nrhs must be >= 1";
      return MG_ERR_INVALID_ARG;
    }
    return mg_solve_batch(c, nrhs, chi, psi, nullptr, tol, st);
  }
  int status = MG_OK;
  int rc = guarded([&] {
    need_ctx(c);
    need_ptr(chi);
    need_ptr(psi);
    if (c->e4) {
      const Solve4 o = engine4_solve(*c->e4, chi, psi, tol);
      if (st) {
        st->iters = o.iters;
        st->converged = o.converged ? 1 : 0;
        st->true_rel_residual = o.rel;
        for (int l = 0; l < MG_MAX_LEVELS; ++l) st->level_apps[l] = o.apps[l];
        st->coarsest_iters = o.coarsest_iters;
        st->ms = o.ms;
        st->graphs = 0;
        st->setup_s = c->setup_s;
        st->solve_s = o.ms * 1e-3;
        st->fine_D_apps = o.apps[0];
      }
      if (!o.converged) status = MG_ERR_NOT_CONVERGED;
      return;
    }
    check_fresh(*c);
    for (long long &a : c->apps) a = 0;
    collect_coarsest(*c);
    c->coarsest_iters = 0;
    EventPair ev;
    ev.start(c->s);
    GcrOut o = outer_fgcr(*c, static_cast<const Cx<double> *>(chi), static_cast<Cx<double> *>(psi), tol,
                          c->p.gcr_restart, c->p.max_iter);
    const float ms = ev.stop(c->s);
    c->coarsest_iters = collect_coarsest(*c);
    if (!c->use_lu) c->apps[c->p.levels - 1] += c->coarsest_iters;
    if (st) {
      st->iters = o.iters;
      st->converged = o.converged ? 1 : 0;
      st->true_rel_residual = o.rel;
      for (int l = 0; l < MG_MAX_LEVELS; ++l) st->level_apps[l] = c->apps[l];
      st->coarsest_iters = c->coarsest_iters;
      st->ms = ms;
      st->graphs = (c->graphs_ok && c->pre[c->p.precision == MG_FP32 ? 1 : 0].exec != nullptr) ? 1 : 0;
      st->setup_s = c->setup_s;
      st->solve_s = ms * 1e-3;
      st->fine_D_apps = c->apps[0];
    }
    if (!o.converged) status = MG_ERR_NOT_CONVERGED;
  });
  if (rc == MG_OK && status != MG_OK) {
    t_last_error = "not converged within max_iter";
    return status;
  }
  return rc;
}

int mg_solve_batch(mg_ctx *c, int nrhs, const void *chi, void *psi, const double *mass, double tol, mg_stats *st) {
  int status = MG_OK;
  int rc = guarded([&] {
    need_ctx(c);
    need_ptr(chi);
    need_ptr(psi);
    if (c->e4) {
      if (mass != nullptr)
        for (int v = 0; v < nrhs; ++v)
          if (mass[v] != c->m) fail(MG_ERR_UNSUPPORTED, "4d batched solves take the context mass (mass = NULL)");
      const std::vector<Solve4> o = engine4_solve_batch(*c->e4, nrhs, chi, psi, tol);
      for (int v = 0; v < nrhs; ++v) {
        if (!o[v].converged) status = MG_ERR_NOT_CONVERGED;
        if (!st) continue;
        st[v].iters = o[v].iters;
        st[v].converged = o[v].converged ? 1 : 0;
        st[v].true_rel_residual = o[v].rel;
        for (int l = 0; l < MG_MAX_LEVELS; ++l) st[v].level_apps[l] = o[v].apps[l];
        st[v].coarsest_iters = o[v].coarsest_iters;
        st[v].ms = o[v].ms;
        st[v].graphs = 0;
        st[v].setup_s = c->setup_s;
        st[v].solve_s = o[v].ms * 1e-3;
        st[v].fine_D_apps = o[v].apps[0];
      }
      return;
    }
    if (nrhs < 1 || nrhs > c->p.max_rhs) fail(MG_ERR_INVALID_ARG, "nrhs must be in [1, max_rhs]");
    check_fresh(*c);
    if (c->bZ.p == nullptr) alloc_batch(*c);
    std::vector<double> sh(nrhs, 0.0);
    for (int v = 0; v < nrhs; ++v) {
      if (mass != nullptr) sh[v] = mass[v] - c->m;
      if (!std::isfinite(sh[v])) fail(MG_ERR_INVALID_ARG, "mass must be finite");
    }
    prepare_slots(*c, nrhs, sh.data());
    MG_CUDA(cudaMemcpyAsync(c->shift_dev.p, sh.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->s));
    for (long long &a : c->apps) a = 0;
    collect_coarsest(*c);
    c->coarsest_iters = 0;
    EventPair ev;
    ev.start(c->s);
    std::vector<GcrOut> o;
    c->cur_shift = c->shift_dev.p;
    try {
      outer_fgcr_batch(*c, nrhs, static_cast<const Cx<double> *>(chi), static_cast<Cx<double> *>(psi), tol, o);
    } catch (...) {
      c->cur_shift = nullptr;
      throw;
    }
    c->cur_shift = nullptr;
    const float ms = ev.stop(c->s);
    c->coarsest_iters = collect_coarsest(*c);
    if (!c->use_lu) c->apps[c->p.levels - 1] += c->coarsest_iters;
    for (int v = 0; v < nrhs; ++v) {
      if (!o[v].converged) status = MG_ERR_NOT_CONVERGED;
      if (!st) continue;
      st[v].iters = o[v].iters;
      st[v].converged = o[v].converged ? 1 : 0;
      st[v].true_rel_residual = o[v].rel;
      for (int l = 0; l < MG_MAX_LEVELS; ++l) st[v].level_apps[l] = c->apps[l];
      st[v].coarsest_iters = c->coarsest_iters;
      st[v].ms = ms;
      st[v].graphs = (c->graphs_ok && c->preb[c->p.precision == MG_FP32 ? 1 : 0][nrhs].exec != nullptr) ? 1 : 0;
      st[v].setup_s = c->setup_s;
      st[v].solve_s = ms * 1e-3;
      st[v].fine_D_apps = c->apps[0];
    }
  });
  if (rc == MG_OK && status != MG_OK) {
    t_last_error = "a right-hand side did not converge within max_iter";
    return status;
  }
  return rc;
}

// Captured V-cycles hold the fine diagonal d + m as a kernel argument: a new mass
// needs new graphs (every buffer they touch is unchanged, the coarse operators are
// rebuilt in place).
static void drop_graphs(mg_ctx &c) {
  for (auto &g : c.pre) g.reset();
  for (auto &g : c.setup_vc) g.reset();
  for (auto &v : c.preb)
    for (auto &g : v) g.reset();
}

int mg_update_mass(mg_ctx *c, double m) {
  return guarded([&] {
    need_ctx(c);
    if (c->e4) {
      c->m = m;
      engine4_update_mass(*c->e4, m);
      return;
    }
    check_fresh(*c);
    c->m = m;
    MG_CUDA(cudaStreamSynchronize(c->s));  // no replay of the old graphs is still in flight
    drop_graphs(*c);
    for (int l = 0; l + 1 < c->p.levels; ++l) {
      Level &L = c->lv[l];
      if (l == 0)
        launch_galerkin_wilson(c->U64.p, diag_of(*c), L.V64.p, c->lv[1].Y64.p, L.bg, L.Nv, c->s, galerkin_f32(*c));
      else
        launch_galerkin_stencil(L.Y64.p, L.V64.p, c->lv[l + 1].Y64.p, L.bg, L.Nv, c->s, galerkin_f32(*c));
    }
    prepare_coarsest(*c);
    make_fp32_copies(*c);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_clone(mg_ctx *src, double m, void *stream, mg_ctx **out) {
  return guarded([&] {
    if (!out) fail(MG_ERR_INVALID_ARG, "null context out-pointer");
    *out = nullptr;
    need_ctx(src);
    const auto t0 = std::chrono::steady_clock::now();
    if (src->e4) fail(MG_ERR_UNSUPPORTED, "clones are built for d = 2");
    check_fresh(*src);
    MG_CUDA(cudaStreamSynchronize(src->s));  // the source's buffers are final
    const mg_params sp = user_params(*src);
    auto c = create(&src->geom, m, &sp, stream);
    MG_CUDA(cudaMemcpyAsync(c->U64.p, src->U64.p, c->U64.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
    make_link_copies(*c);
    for (int l = 0; l + 1 < c->p.levels; ++l) {
      Level &L = c->lv[l];
      const Level &S = src->lv[l];
      MG_CUDA(cudaMemcpyAsync(L.nullv.p, S.nullv.p, L.nullv.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
      MG_CUDA(cudaMemcpyAsync(L.V64.p, S.V64.p, L.V64.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
      // Galerkin operators at the clone's mass, level by level (level l + 1 needs Y of level l)
      if (l == 0)
        launch_galerkin_wilson(c->U64.p, diag_of(*c), L.V64.p, c->lv[1].Y64.p, L.bg, L.Nv, c->s, galerkin_f32(*c));
      else
        launch_galerkin_stencil(L.Y64.p, L.V64.p, c->lv[l + 1].Y64.p, L.bg, L.Nv, c->s, galerkin_f32(*c));
    }
    prepare_coarsest(*c);
    make_fp32_copies(*c);
    collect_coarsest(*c);
    MG_CUDA(cudaStreamSynchronize(c->s));
    c->setup_s = seconds_since(t0);
    *out = c.release();
  });
}

int mg_save_setup(mg_ctx *c, const char *path) {
  return guarded([&] {
    need_ctx(c);
    need_ptr(path);
    SetupFileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kSetupMagic, 8);
    h.version = 1;
    h.g = c->geom;
    h.p = user_params(*c);
    h.m = c->m;
    std::vector<std::vector<Cx<double>>> vecs;
    if (c->e4) {
      h.levels_saved = 1;
      vecs.emplace_back((size_t)engine4_null_vector_count(*c->e4));
      DevBuf<Cx<double>> tmp;
      tmp.alloc(vecs[0].size());
      pool_ready();
      engine4_get_null_vectors(*c->e4, tmp.p);
      MG_CUDA(cudaMemcpy(vecs[0].data(), tmp.p, vecs[0].size() * sizeof(Cx<double>), cudaMemcpyDeviceToHost));
      h.links_digest = device_digest(engine4_links(*c->e4), link_bytes(c->geom), c->s);
    } else {
      check_fresh(*c);
      h.levels_saved = (uint32_t)(c->p.levels - 1);
      for (int l = 0; l + 1 < c->p.levels; ++l) {
        const Level &L = c->lv[l];
        vecs.emplace_back(L.nullv.n);
        MG_CUDA(cudaMemcpyAsync(vecs.back().data(), L.nullv.p, L.nullv.n * sizeof(Cx<double>),
                                cudaMemcpyDeviceToHost, c->s));
      }
      MG_CUDA(cudaStreamSynchronize(c->s));
      h.links_digest = device_digest(c->U64.p, link_bytes(c->geom), c->s);
    }
    uint64_t pd = 14695981039346656037ULL;
    for (size_t l = 0; l < vecs.size(); ++l) {
      h.count[l] = vecs[l].size();
      pd = fnv1a(vecs[l].data(), vecs[l].size() * sizeof(Cx<double>), pd);
    }
    h.payload_digest = pd;
    FILE *f = std::fopen(path, "wb");
    if (!f) fail(MG_ERR_UNSUPPORTED, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    for (const auto &v : vecs) ok = ok && std::fwrite(v.data(), sizeof(Cx<double>), v.size(), f) == v.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) fail(MG_ERR_UNSUPPORTED, std::string("writing ") + path + " failed");
  });
}

int mg_solve_multi(int count, mg_ctx *const *ctx, const int *nrhs, const void *const *chi, void *const *psi,
                   double tol, mg_stats *st) {
  int status = MG_OK;
  int rc = guarded([&] {
    if (count < 1 || !ctx || !chi || !psi) fail(MG_ERR_INVALID_ARG, "need count >= 1 and non-null arrays");
    int dev0 = -1;
    std::vector<DevSolve> v(count);
    for (int i = 0; i < count; ++i) {
      need_ctx(ctx[i]);
      need_ptr(chi[i]);
      need_ptr(psi[i]);
      if (ctx[i]->e4) fail(MG_ERR_UNSUPPORTED, "the device-driven multi-solve is built for d = 2");
      for (int j = 0; j < i; ++j)
        if (ctx[j] == ctx[i]) fail(MG_ERR_INVALID_ARG, "a context appears twice (its buffers would be shared)");
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, psi[i]) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        (void)cudaGetLastError();
        fail(MG_ERR_INVALID_ARG, "psi must be device memory");
      }
      if (dev0 < 0) dev0 = pa.device;
      if (pa.device != dev0) fail(MG_ERR_INVALID_ARG, "all contexts must be on one device");
      v[i].c = ctx[i];
      v[i].b = static_cast<const Cx<double> *>(chi[i]);
      v[i].x = static_cast<Cx<double> *>(psi[i]);
      v[i].nb = nrhs ? nrhs[i] : 1;
      if (v[i].nb < 1 || v[i].nb > ctx[i]->p.max_rhs)
        fail(MG_ERR_INVALID_ARG, "nrhs[i] must be in [1, max_rhs of context i]");
    }
    EventPair ev;
    ev.start(v[0].c->s);
    devloop_solve(v, tol);
    const float ms = ev.stop(v[0].c->s);
    int e = 0;
    for (int i = 0; i < count; ++i) {
      mg_ctx &c = *v[i].c;
      for (int q = 0; q < v[i].nb; ++q, ++e) {
        const GcrOut &o = v[i].out[q];
        if (!o.converged) status = MG_ERR_NOT_CONVERGED;
        if (!st) continue;
        st[e].iters = o.iters;
        st[e].converged = o.converged ? 1 : 0;
        st[e].true_rel_residual = o.rel;
        for (int l = 0; l < MG_MAX_LEVELS; ++l) st[e].level_apps[l] = c.apps[l];
        st[e].coarsest_iters = c.coarsest_iters;
        st[e].ms = ms;
        st[e].graphs = 1;
        st[e].setup_s = c.setup_s;
        st[e].solve_s = ms * 1e-3;
        st[e].fine_D_apps = c.apps[0];
      }
    }
  });
  if (rc == MG_OK && status != MG_OK) {
    t_last_error = "a system did not converge within max_iter";
    return status;
  }
  return rc;
}

int mg_convergence_rate(mg_ctx *c, int steps, uint64_t seed, double *rate) {
  return guarded([&] {
    need_ctx(c);
    if (c->e4) fail(MG_ERR_UNSUPPORTED, "the convergence-rate measurement is built for d = 2");
    if (steps < 2) fail(MG_ERR_INVALID_ARG, "steps must be >= 2");
    check_fresh(*c);
    const double r = convergence_rate(*c, steps, seed);
    if (rate) *rate = r;
  });
}

int mg_setup_learned(mg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, mg_nullnet *net,
                     uint64_t noise_seed, int nu_refine, double max_rate, int rate_steps, int *used_learned,
                     double *rate, void *stream) {
  return guarded([&] {
    if (!ctx) fail(MG_ERR_INVALID_ARG, "null context out-pointer");
    *ctx = nullptr;
    need_ptr(U);
    need_ptr(net);
    if (!g || g->d != 2) fail(MG_ERR_UNSUPPORTED, "the learned setup is built for d = 2");
    if (!p) fail(MG_ERR_INVALID_ARG, "null parameters");
    if (nullnet_nv(*net) != p->Nv[0]) fail(MG_ERR_INVALID_ARG, "the network predicts nv != Nv[0] vectors");
    if (nu_refine < 0 || rate_steps < 2) fail(MG_ERR_INVALID_ARG, "need nu_refine >= 0 and rate_steps >= 2");
    const auto t0 = std::chrono::steady_clock::now();
    auto c = create(g, m, p, stream);
    MG_CUDA(cudaMemcpyAsync(c->U64.p, U, c->U64.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
    const bool f32 = c->p.precision == MG_FP32;
    make_link_copies(*c);
    Level &F = c->lv[0];
    nullnet_predict(*net, *g, c->U64.p, noise_seed, F.nullv.p, c->s);
    if (nu_refine > 0) {
      // the predicted vectors start the relaxation of Eq. relax in place of random ones
      const int keep = c->p.nu_setup;
      c->p.nu_setup = nu_refine;
      if (f32)
        relax_and_adapt<float>(*c, 0, 1);
      else
        relax_and_adapt<double>(*c, 0, 1);
      c->p.nu_setup = keep;
    }
    // the adaptive passes 2..n_pass follow as in the plain setup, from the learned start
    for (int pass = 1; pass <= c->p.n_pass; ++pass) {
      if (pass > 1) {
        if (f32)
          relax_and_adapt<float>(*c, 0, pass);
        else
          relax_and_adapt<double>(*c, 0, pass);
      }
      build_level(*c, 0);
      if (f32) {
        launch_convert<float, double>(F.V64.p, F.V32.p, F.V64.n, c->s);
        refresh_y32(*c, 1);
      }
      if (c->p.levels > 2)
        setup_level(*c, 1, pass == c->p.n_pass);
      else
        prepare_coarsest(*c);
    }
    F.stale = false;
    make_fp32_copies(*c);
    collect_coarsest(*c);
    double r = convergence_rate(*c, rate_steps, noise_seed ^ 0x5241544552ULL);
    int used = 1;
    if (!(r <= max_rate)) {
      // the judge rejects the learned vectors: the plain adaptive setup takes over
      MG_CUDA(cudaStreamSynchronize(c->s));
      drop_graphs(*c);
      setup_level(*c, 0, true);
      make_fp32_copies(*c);
      collect_coarsest(*c);
      r = convergence_rate(*c, rate_steps, noise_seed ^ 0x5241544552ULL);
      used = 0;
    }
    MG_CUDA(cudaStreamSynchronize(c->s));
    c->setup_s = seconds_since(t0);
    if (used_learned) *used_learned = used;
    if (rate) *rate = r;
    *ctx = c.release();
  });
}

int mg_context_info(const mg_ctx *c, mg_geom *g, mg_params *p, double *m) {
  return guarded([&] {
    if (!c) fail(MG_ERR_INVALID_ARG, "null context");
    if (g) *g = c->geom;
    if (p) *p = c->e4 ? c->p : user_params(*c);
    if (m) *m = c->m;
  });
}

int mg_load_setup(mg_ctx **ctx, const char *path, const void *U, void *stream) {
  return guarded([&] {
    if (!ctx) fail(MG_ERR_INVALID_ARG, "null context out-pointer");
    *ctx = nullptr;
    need_ptr(path);
    need_ptr(U);
    FILE *f = std::fopen(path, "rb");
    if (!f) fail(MG_ERR_INVALID_ARG, std::string("cannot open ") + path);
    SetupFileHeader h;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kSetupMagic, 8) == 0 && h.version == 1 &&
              h.levels_saved >= 1 && h.levels_saved < MG_MAX_LEVELS;
    std::vector<std::vector<Cx<double>>> vecs;
    uint64_t pd = 14695981039346656037ULL;
    for (uint32_t l = 0; ok && l < h.levels_saved; ++l) {
      if (h.count[l] == 0 || h.count[l] > (1ULL << 34)) {
        ok = false;
        break;
      }
      vecs.emplace_back((size_t)h.count[l]);
      ok = std::fread(vecs.back().data(), sizeof(Cx<double>), vecs.back().size(), f) == vecs.back().size();
      if (ok) pd = fnv1a(vecs.back().data(), vecs.back().size() * sizeof(Cx<double>), pd);
    }
    std::fclose(f);
    if (!ok) fail(MG_ERR_INVALID_ARG, std::string(path) + " is not a complete saved setup of this version");
    if (pd != h.payload_digest) fail(MG_ERR_INVALID_ARG, std::string(path) + ": payload digest mismatch (corrupt)");
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    const size_t lb = link_bytes(h.g);
    if (h.g.d != 2 && h.g.d != 4) fail(MG_ERR_INVALID_ARG, "saved setup: bad geometry");
    if (device_digest(U, lb, static_cast<cudaStream_t>(stream)) != h.links_digest)
      fail(MG_ERR_INVALID_ARG, "saved setup was made on other links (digest mismatch)");
    if (h.g.d == 2 && (int)h.levels_saved != h.p.levels - 1)
      fail(MG_ERR_INVALID_ARG, "saved setup: level count does not match its parameters");
    *ctx = make_context(&h.g, U, h.m, &h.p, stream, &vecs).release();
  });
}

void mg_destroy(mg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  delete c;
}


int mg_dslash(const mg_geom *g, const void *U, double m, const void *in, void *out, int precision, void *stream) {
  return guarded([&] {
    if (!g) fail(MG_ERR_INVALID_ARG, "null geometry");
    if (!((g->d == 2 && g->Nc == 1) || (g->d == 4 && g->Nc == 3)))
      fail(MG_ERR_UNSUPPORTED, "built: d = 2 with Nc = 1, d = 4 with Nc = 3");
    long long vol = 1;
    for (int mu = 0; mu < g->d; ++mu) {
      if (g->dims[mu] < 2) fail(MG_ERR_INVALID_ARG, "lattice extents must be >= 2");
      vol *= g->dims[mu];
    }
    if (vol >= (1LL << 31)) fail(MG_ERR_INVALID_ARG, "lattice volume must be below 2^31 sites");
    need_ptr(U);
    need_ptr(in);
    need_ptr(out);
    if (in == out) fail(MG_ERR_INVALID_ARG, "in and out must not alias");
    if (g->d == 4) {
      Geo4 g4{{g->dims[0], g->dims[1], g->dims[2], g->dims[3]}, vol};
      cudaStream_t s4 = static_cast<cudaStream_t>(stream);
      if (precision == MG_FP64)
        launch_dslash4<double>(static_cast<const Cx<double> *>(U), static_cast<const Cx<double> *>(in),
                               static_cast<Cx<double> *>(out), g4, 4.0 + m, nullptr, 1.0, 0.0, s4);
      else if (precision == MG_FP32)
        launch_dslash4<float>(static_cast<const Cx<float> *>(U), static_cast<const Cx<float> *>(in),
                              static_cast<Cx<float> *>(out), g4, 4.0 + m, nullptr, 1.0, 0.0, s4);
      else
        fail(MG_ERR_INVALID_ARG, "unknown precision");
      return;
    }
    Geo2 geo{g->dims[0], g->dims[1], (long long)g->dims[0] * g->dims[1]};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == MG_FP64)
      launch_dslash<double>(static_cast<const Cx<double> *>(U), static_cast<const Cx<double> *>(in),
                            static_cast<Cx<double> *>(out), geo, 2.0 + m, nullptr, 1.0, 0.0, s);
    else if (precision == MG_FP32)
      launch_dslash<float>(static_cast<const Cx<float> *>(U), static_cast<const Cx<float> *>(in),
                           static_cast<Cx<float> *>(out), geo, 2.0 + m, nullptr, 1.0, 0.0, s);
    else if (precision == MG_FP16)
      launch_dslash_half(U, in, out, geo, 2.0 + m, s);
    else
      fail(MG_ERR_INVALID_ARG, "unknown precision");
  });
}

int mg_half_convert(int what, int precision, const void *in, void *out, long long nsites, void *stream) {
  return guarded([&] {
    need_ptr(in);
    need_ptr(out);
    if (in == out) fail(MG_ERR_INVALID_ARG, "in and out must not alias");
    if (what < 0 || what > 2) fail(MG_ERR_INVALID_ARG, "what must be 0, 1 or 2");
    if (precision != MG_FP64 && precision != MG_FP32) fail(MG_ERR_INVALID_ARG, "precision must be MG_FP64 or MG_FP32");
    if (nsites < 1 || nsites >= (1LL << 31)) fail(MG_ERR_INVALID_ARG, "nsites out of range");
    launch_half_convert(what, precision, in, out, nsites, static_cast<cudaStream_t>(stream));
  });
}

int mg_level_apply(mg_ctx *c, int level, const void *in, void *out) {
  return guarded([&] {
    need_level(c, level, false);
    need_ptr(in);
    need_ptr(out);
    if (c->e4) {
      engine4_level_apply(*c->e4, level, in, out);
      return;
    }
    apply_op<double>(*c, level, static_cast<const Cx<double> *>(in), static_cast<Cx<double> *>(out));
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_restrict(mg_ctx *c, int level, const void *fine, void *coarse) {
  return guarded([&] {
    need_level(c, level, true);
    need_ptr(fine);
    need_ptr(coarse);
    if (c->e4) {
      engine4_restrict(*c->e4, fine, coarse);
      return;
    }
    Level &L = c->lv[level];
    launch_restrict<double>(L.V64.p, static_cast<const Cx<double> *>(fine), static_cast<Cx<double> *>(coarse), L.bg,
                            L.Nv, c->s);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_prolong(mg_ctx *c, int level, const void *coarse, void *fine) {
  return guarded([&] {
    need_level(c, level, true);
    need_ptr(fine);
    need_ptr(coarse);
    if (c->e4) {
      engine4_prolong(*c->e4, coarse, fine);
      return;
    }
    Level &L = c->lv[level];
    launch_zero<double>(static_cast<Cx<double> *>(fine), L.n, c->s);
    launch_prolong_add<double>(L.V64.p, static_cast<const Cx<double> *>(coarse), static_cast<Cx<double> *>(fine),
                               L.bg, L.Nv, c->s);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_vcycle(mg_ctx *c, const void *b, void *x) {
  return guarded([&] {
    need_ctx(c);
    need_ptr(b);
    need_ptr(x);
    if (c->e4) {
      engine4_vcycle(*c->e4, b, x);
      return;
    }
    check_fresh(*c);
    precondition(*c, static_cast<const Cx<double> *>(b), static_cast<Cx<double> *>(x));
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_coarse_apply_mrhs(mg_ctx *c, int level, int nrhs, const void *in, void *out, int tensor_cores) {
  return guarded([&] {
    need_level(c, level, false);
    need_ptr(in);
    need_ptr(out);
    if (nrhs >= 1 && level >= 1) {
      // the stencil reads neighbours of `in` while it writes `out`: the ranges must be disjoint
      long long ns = 0;
      int ni = 0;
      if (c->e4)
        engine4_level_size(*c->e4, level, &ns, &ni);
      else {
        ns = c->lv[level].geo.nsites;
        ni = c->lv[level].nint;
      }
      const unsigned long long bytes = (unsigned long long)nrhs * ns * ni * sizeof(Cx<float>);
      const unsigned long long a0 = reinterpret_cast<uintptr_t>(in), b0 = reinterpret_cast<uintptr_t>(out);
      if (a0 < b0 + bytes && b0 < a0 + bytes) fail(MG_ERR_INVALID_ARG, "in and out must not overlap");
    }
    if (c->e4) {
      if (level != 1) fail(MG_ERR_INVALID_ARG, "the 4d hierarchy has one coarse level (level 1)");
      if (nrhs < 1) fail(MG_ERR_INVALID_ARG, "nrhs must be >= 1");
      engine4_coarse_apply_mrhs(*c->e4, nrhs, in, out, tensor_cores);
      return;
    }
    if (tensor_cores < 0 || tensor_cores > 3) fail(MG_ERR_INVALID_ARG, "tensor_cores must be 0, 1, 2 or 3");
    if (tensor_cores > 1) fail(MG_ERR_UNSUPPORTED, "the split-operand tensor-core apply is built for the 4d level");
    if (level < 1) fail(MG_ERR_INVALID_ARG, "the tensor-core apply is for coarse levels (level >= 1)");
    if (nrhs < 1) fail(MG_ERR_INVALID_ARG, "nrhs must be >= 1");
    check_fresh(*c);
    Level &L = c->lv[level];
    if (L.Ypk.p == nullptr) fail(MG_ERR_UNSUPPORTED, "needs an MG_FP32 context and N = 8 on that level");
    if (tensor_cores)
      launch_coarse_apply_tc(L.Ypk.p, static_cast<const Cx<float> *>(in), static_cast<Cx<float> *>(out), L.geo,
                             nrhs, nullptr, 1.0, 0.0, nullptr, c->s);
    else
      launch_coarse_apply<float>(L.Y32.p, static_cast<const Cx<float> *>(in), static_cast<Cx<float> *>(out), L.geo,
                                 L.nint, nullptr, 1.0, 0.0, c->s, nrhs);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

size_t mg_autotune_report(char *buf, size_t len) {
  const std::string r = autotune_report();
  if (buf != nullptr && len > 0) {
    const size_t m = std::min(len - 1, r.size());
    std::memcpy(buf, r.data(), m);
    buf[m] = '\0';
  }
  return r.size();
}

int mg_selftest_barrier(int missing_arrivals, void *stream) {
  return guarded([&] {
    if (missing_arrivals < 0 || missing_arrivals > 1) fail(MG_ERR_INVALID_ARG, "missing_arrivals must be 0 or 1");
    // about 2^16 polls of >= 64 ns: the wait gives up within a few milliseconds
    const int timed_out = barrier_selftest(2u + (unsigned)missing_arrivals, 1LL << 16, static_cast<cudaStream_t>(stream));
    if (timed_out) fail(MG_ERR_TIMEOUT, "grid barrier self-test: the wait ran out (as arranged when an arrival is missing)");
  });
}

int mg_coarsest_solve(mg_ctx *c, const void *b, void *x, long long *iters, double *ms) {
  return guarded([&] {
    need_ctx(c);
    need_ptr(b);
    need_ptr(x);
    if (c->e4) {
      float t = 0.f;
      const long long it = engine4_coarsest_solve(*c->e4, b, x, &t);
      if (iters) *iters = it;
      if (ms) *ms = t;
      return;
    }
    check_fresh(*c);
    collect_coarsest(*c);
    EventPair ev;
    ev.start(c->s);
    coarsest_solve64(*c, static_cast<const Cx<double> *>(b), static_cast<Cx<double> *>(x));
    const float t = ev.stop(c->s);
    const long long it = collect_coarsest(*c);
    if (iters) *iters = it;
    if (ms) *ms = t;
  });
}

int mg_smooth(mg_ctx *c, int level, const void *b, void *x, int nu) {
  return guarded([&] {
    need_level(c, level, false);
    need_ptr(b);
    need_ptr(x);
    if (nu < 0) fail(MG_ERR_INVALID_ARG, "nu must be >= 0");
    if (c->e4) {
      if (level != 0) fail(MG_ERR_UNSUPPORTED, "the 4d hierarchy smooths on level 0 only");
      engine4_smooth(*c->e4, b, x, nu);
      return;
    }
    Level &L = c->lv[level];
    (void)L;
    smooth<double>(*c, level, static_cast<const Cx<double> *>(b), static_cast<Cx<double> *>(x), nu, false);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_build_level(mg_ctx *c, int level, const void *vectors) {
  return guarded([&] {
    need_level(c, level, true);
    need_ptr(vectors);
    if (c->e4) {
      engine4_build_level(*c->e4, vectors);
      return;
    }
    Level &L = c->lv[level];
    MG_CUDA(cudaMemcpyAsync(L.nullv.p, vectors, L.nullv.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
    build_level(*c, level);
    if (level + 1 == c->p.levels - 1)
      prepare_coarsest(*c);
    else
      c->lv[level + 1].stale = true;
    L.stale = false;
    make_fp32_copies(*c);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_get_null_vectors(mg_ctx *c, int level, void *out) {
  return guarded([&] {
    need_level(c, level, true);
    need_ptr(out);
    if (c->e4) {
      engine4_get_null_vectors(*c->e4, out);
      return;
    }
    Level &L = c->lv[level];
    MG_CUDA(cudaMemcpyAsync(out, L.nullv.p, L.nullv.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, c->s));
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_get_prolongator(mg_ctx *c, int level, void *out) {
  return guarded([&] {
    need_level(c, level, true);
    need_ptr(out);
    if (c->e4) {
      engine4_get_prolongator(*c->e4, out);
      return;
    }
    Level &L = c->lv[level];
    launch_prolongator_to_canonical(L.V64.p, static_cast<Cx<double> *>(out), L.bg, L.Nv, c->s);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_get_coarse_op(mg_ctx *c, int level, void *out) {
  return guarded([&] {
    need_level(c, level, false);
    if (level < 1) fail(MG_ERR_INVALID_ARG, "level 0 has no stencil blocks");
    need_ptr(out);
    if (c->e4) {
      engine4_get_coarse_op(*c->e4, out);
      return;
    }
    Level &L = c->lv[level];
    launch_coarse_to_canonical(L.Y64.p, static_cast<Cx<double> *>(out), L.geo.nsites, L.nint, c->s);
    MG_CUDA(cudaStreamSynchronize(c->s));
  });
}

int mg_level_size(mg_ctx *c, int level, long long *n_sites, int *n_int) {
  return guarded([&] {
    need_level(c, level, false);
    if (c->e4) {
      engine4_level_size(*c->e4, level, n_sites, n_int);
      return;
    }
    if (n_sites) *n_sites = c->lv[level].geo.nsites;
    if (n_int) *n_int = c->lv[level].nint;
  });
}

}  // extern "C"
