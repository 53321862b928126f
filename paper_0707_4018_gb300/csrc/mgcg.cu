// MG-preconditioned conjugate gradients on the normal equations: the paper's own experiment
// (numerical-results section). The operator is A = D^dagger D (hermitian positive definite), the
// hierarchy is built by the adaptive procedure on A with 4 x 4 blocks and M = 8 vectors, the
// relaxation is the degree-2 MR polynomial with frozen coefficients (so R = R^dagger), the
// V-cycle of Eq. vcycle preconditions CG, and the coarsest level is solved exactly.
//
// The Galerkin operator P^dagger A P couples a coarse site to its 8 neighbours, diagonal ones
// included (D^dagger D reaches x +- 2 mu-hat and x +- mu-hat +- nu-hat), so the coarse levels are
// 9-point stencils y_j = sum_o Y[j][o] x_{j+o}, o in {-1, 0, 1}^2 (index 3 (o1 + 1) + (o0 + 1)),
// with N x N complex blocks stored row-major ([j][o][row][col]). They are built by probing: the
// coarse sites are coloured by (j0 mod p0, j1 mod p1) with periods >= 3 that divide the coarse
// extents, so the 9 neighbours of a site have distinct colours; A applied to the prolongation of
// the unit vectors (all sites of colour c, dof k), restricted, holds column k of Y[j][o] at every
// site j whose neighbour j + o has colour c. Everything is FP64: this mode reproduces the paper's
// iteration counts, the solver path of the bench is the FGCR one.
#include <chrono>
#include <cmath>
#include <memory>
#include <vector>

#include "kernels.h"

namespace mg {

namespace {

constexpr int kOffsets = 9;
constexpr int kSmootherVector = 0x2C;  // Philox vector index of the smoother coefficients' source

__device__ __forceinline__ int colour_of(int j0, int j1, int p0, int p1) { return (j0 % p0) + p0 * (j1 % p1); }

// the site j + o of a coarse lattice (periodic)
__device__ __forceinline__ int shifted(int j0, int j1, int o, int L0, int L1) {
  const int o0 = o % 3 - 1, o1 = o / 3 - 1;
  const int s0 = (j0 + o0 + L0) % L0, s1 = (j1 + o1 + L1) % L1;
  return s0 + L0 * s1;
}

// gamma_5 = sigma_3 on 2d spinors: the second component changes sign
__global__ void gamma5_kernel(Cx<double> *x, long long V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < V) x[2 * i + 1] = mk(-x[2 * i + 1].re, -x[2 * i + 1].im);
}

// out_j = sum_o Y[j][o] in_{j+o}: one thread per (site, row)
__global__ void stencil9_kernel(const Cx<double> *__restrict__ Y, const Cx<double> *__restrict__ in,
                                Cx<double> *__restrict__ out, int L0, int L1, int N) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long V = (long long)L0 * L1;
  if (t >= V * N) return;
  const int j = (int)(t / N), row = (int)(t - (long long)j * N);
  const int j1 = j / L0, j0 = j - j1 * L0;
  Cx<double> acc = mk(0.0, 0.0);
  for (int o = 0; o < kOffsets; ++o) {
    const long long src = shifted(j0, j1, o, L0, L1);
    const Cx<double> *Yr = Y + (((long long)j * kOffsets + o) * N + row) * N;
    const Cx<double> *x = in + src * N;
    for (int c = 0; c < N; ++c) cmac(acc, Yr[c], x[c]);
  }
  out[t] = acc;
}

// e[b][a] = 1 where a = k and b has colour `colour`, else 0
__global__ void probe_vector_kernel(Cx<double> *e, int L0, int L1, int N, int p0, int p1, int colour, int k) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)L0 * L1 * N) return;
  const int b = (int)(t / N), a = (int)(t - (long long)b * N);
  const int b1 = b / L0, b0 = b - b1 * L0;
  e[t] = mk(a == k && colour_of(b0, b1, p0, p1) == colour ? 1.0 : 0.0, 0.0);
}

// Y[j][o][a][k] = y[j][a] for the offsets o whose neighbour j + o has colour `colour`
__global__ void probe_scatter_kernel(const Cx<double> *__restrict__ y, Cx<double> *__restrict__ Y, int L0, int L1,
                                     int N, int p0, int p1, int colour, int k) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)L0 * L1 * kOffsets * N) return;
  const int a = (int)(t % N);
  const long long jo = t / N;
  const int o = (int)(jo % kOffsets), j = (int)(jo / kOffsets);
  const int j1 = j / L0, j0 = j - j1 * L0;
  const int src = shifted(j0, j1, o, L0, L1);
  const int s1 = src / L0, s0 = src - s1 * L0;
  if (colour_of(s0, s1, p0, p1) == colour) Y[(((long long)j * kOffsets + o) * N + a) * N + k] = y[(long long)j * N + a];
}

// the 9-point operator as a dense column-major matrix (coarsest level)
__global__ void dense_from_stencil9_kernel(const Cx<double> *__restrict__ Y, Cx<double> *__restrict__ A, int L0,
                                           int L1, int N) {
  const long long n = (long long)L0 * L1 * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const long long col = t / n, row = t - col * n;
  const int j = (int)(row / N), sc = (int)(col / N);
  const int ar = (int)(row - (long long)j * N), ac = (int)(col - (long long)sc * N);
  const int j1 = j / L0, j0 = j - j1 * L0;
  Cx<double> v = mk(0.0, 0.0);
  for (int o = 0; o < kOffsets; ++o)
    if (shifted(j0, j1, o, L0, L1) == sc) v = v + Y[(((long long)j * kOffsets + o) * N + ar) * N + ac];
  A[t] = v;
}

// x += a r; r -= a w
__global__ void step_kernel(Cx<double> *__restrict__ x, Cx<double> *__restrict__ r, const Cx<double> *__restrict__ w,
                            double are, double aim, long long n) {
  const Cx<double> a = mk(are, aim), ma = mk(-are, -aim);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cmac(x[i], a, r[i]);
    Cx<double> ri = r[i];
    cmac(ri, ma, w[i]);
    r[i] = ri;
  }
}

// the CG step x += alpha p, r -= alpha q
__global__ void cg_update_kernel(Cx<double> *__restrict__ x, Cx<double> *__restrict__ r,
                                 const Cx<double> *__restrict__ p, const Cx<double> *__restrict__ q, double alpha,
                                 long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = mk(x[i].re + alpha * p[i].re, x[i].im + alpha * p[i].im);
    r[i] = mk(r[i].re - alpha * q[i].re, r[i].im - alpha * q[i].im);
  }
}

// x += t; and the CG direction p = z + beta p
__global__ void add_kernel(Cx<double> *__restrict__ x, const Cx<double> *__restrict__ t, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = x[i] + t[i];
}

__global__ void direction_kernel(Cx<double> *__restrict__ p, const Cx<double> *__restrict__ z, double beta,
                                 long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = mk(z[i].re + beta * p[i].re, z[i].im + beta * p[i].im);
}

unsigned int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned int)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// the engine
// ---------------------------------------------------------------------------
struct CgLevel {
  Geo2 geo{};
  int nint = 0;
  long long n = 0;
  BlockGeo bg{};              // transfer to the next level
  int Nv = 0;
  int p0 = 0, p1 = 0;         // probe colour periods of the next level
  DevBuf<Cx<double>> V;       // prolongator [b][k][i]
  DevBuf<Cx<double>> Y;       // this level's 9-point stencil (level >= 1)
  DevBuf<Cx<double>> vecs;    // Nv near-null vectors of this level, [k][n]
  DevBuf<Cx<double>> b, x, r, w, t, r2;
  double alpha[2] = {0.0, 0.0};
};

struct CgEngine {
  mg_geom geom{};
  mg_params p{};
  double m = 0.0;
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev = nullptr;
  DevBuf<Cx<double>> U, tmp;  // links; fine scratch of the D^dagger D apply
  std::vector<CgLevel> lv;
  DevBuf<Cx<double>> LU, lu_work;
  DevBuf<int> ipiv, info;
  DevBuf<double> partials, mgs_min, dots;
  DevBuf<unsigned int> tickets;
  ReduceWs ws{};
  DevBuf<Cx<double>> rhs, cx, cr, cp, cq, cz;  // CG vectors
  double *host = nullptr;
  long long fine_apps = 0;
  ~CgEngine() {
    if (host) cudaFreeHost(host);
    if (ev) cudaEventDestroy(ev);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

static int colour_period(int n) {
  if (n < 3) fail(MG_ERR_INVALID_ARG, "MG-CG: every coarse extent must be at least 3 (9-point Galerkin probe)");
  for (int q = 3; q <= n; ++q)
    if (n % q == 0) return q;
  return n;
}

// A x on level l: D^dagger D x = gamma5 D gamma5 D x on the fine level, the 9-point stencil below
static void cg_apply(CgEngine &e, int l, const Cx<double> *in, Cx<double> *out) {
  CgLevel &L = e.lv[l];
  if (l == 0) {
    const double diag = 2.0 + e.m;
    launch_dslash<double>(e.U.p, in, e.tmp.p, L.geo, diag, nullptr, 1.0, 0.0, e.s, 1, nullptr);
    gamma5_kernel<<<grid_for(L.geo.nsites, 256), 256, 0, e.s>>>(e.tmp.p, L.geo.nsites);
    MG_LAUNCHED();
    launch_dslash<double>(e.U.p, e.tmp.p, out, L.geo, diag, nullptr, 1.0, 0.0, e.s, 1, nullptr);
    gamma5_kernel<<<grid_for(L.geo.nsites, 256), 256, 0, e.s>>>(out, L.geo.nsites);
    MG_LAUNCHED();
    ++e.fine_apps;
  } else {
    stencil9_kernel<<<grid_for(L.n, 256), 256, 0, e.s>>>(L.Y.p, in, out, L.geo.L0, L.geo.L1, L.nint);
    MG_LAUNCHED();
  }
}

// <a, b> (conjugate-linear in a) and |a|^2
static void cg_dot(CgEngine &e, const Cx<double> *a, const Cx<double> *b, long long n, double out[3]) {
  launch_dot_norm<double>(a, b, n, e.dots.p, e.ws, e.s);
  MG_CUDA(cudaMemcpyAsync(e.host, e.dots.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
  for (int i = 0; i < 3; ++i) {
    if (std::isnan(e.host[i])) fail(MG_ERR_NAN, "MG-CG: NaN in a reduction");
    out[i] = e.host[i];
  }
}

// x = R b with the frozen two-step MR polynomial; r = b - A x
static void frozen_smooth(CgEngine &e, int l, const Cx<double> *b, Cx<double> *x, Cx<double> *r) {
  CgLevel &L = e.lv[l];
  launch_zero<double>(x, L.n, e.s);
  launch_copy<double>(b, r, L.n, e.s);
  for (int i = 0; i < 2; ++i) {
    cg_apply(e, l, r, L.w.p);
    step_kernel<<<blocks_for(L.n), 256, 0, e.s>>>(x, r, L.w.p, L.alpha[i], 0.0, L.n);
    MG_LAUNCHED();
  }
}

// x = V_l b (Eq. vcycle, R = R^dagger); b must not be a buffer of level l
static void cg_vcycle(CgEngine &e, int l, const Cx<double> *b, Cx<double> *x) {
  CgLevel &L = e.lv[l];
  if (l + 1 == (int)e.lv.size()) {
    lu_solve_ws(e.LU.p, e.ipiv.p, (int)L.n, b, x, e.lu_work.p, e.s);
    return;
  }
  CgLevel &C = e.lv[l + 1];
  frozen_smooth(e, l, b, x, L.r.p);
  launch_restrict<double>(L.V.p, L.r.p, C.b.p, L.bg, L.Nv, e.s);
  cg_vcycle(e, l + 1, C.b.p, C.x.p);
  launch_prolong_add<double>(L.V.p, C.x.p, x, L.bg, L.Nv, e.s);
  cg_apply(e, l, x, L.w.p);
  launch_copy<double>(L.w.p, L.r.p, L.n, e.s);
  launch_xmy<double>(b, L.r.p, L.n, e.s);  // r = b - A x
  frozen_smooth(e, l, L.r.p, L.t.p, L.r2.p);
  add_kernel<<<blocks_for(L.n), 256, 0, e.s>>>(x, L.t.p, L.n);
  MG_LAUNCHED();
}

// the Nv vectors of level l: Philox draws relaxed by nu_setup MR iterations on A x = 0
static void cg_relax(CgEngine &e, int l) {
  CgLevel &L = e.lv[l];
  for (int k = 0; k < L.Nv; ++k) {
    Cx<double> *v = L.vecs.p + (long long)k * L.n;
    launch_gaussian(v, L.n, e.p.seed, k, l, e.s);
    cg_apply(e, l, v, L.w.p);
    launch_zero<double>(L.r.p, L.n, e.s);
    launch_xmy<double>(L.r.p, L.w.p, L.n, e.s);  // w = 0 - A v
    launch_copy<double>(L.w.p, L.r.p, L.n, e.s);
    for (int it = 0; it < e.p.nu_setup; ++it) {
      cg_apply(e, l, L.r.p, L.w.p);
      double d[3];
      cg_dot(e, L.w.p, L.r.p, L.n, d);
      if (d[2] == 0.0) break;
      step_kernel<<<blocks_for(L.n), 256, 0, e.s>>>(v, L.r.p, L.w.p, e.p.omega * d[0] / d[2], e.p.omega * d[1] / d[2],
                                                      L.n);
      MG_LAUNCHED();
    }
  }
}

// block Gram-Schmidt of level l's vectors and the 9-point Galerkin operator of level l + 1
static void cg_build(CgEngine &e, int l) {
  CgLevel &L = e.lv[l];
  CgLevel &C = e.lv[l + 1];
  launch_block_mgs(L.vecs.p, L.n, L.V.p, L.bg, L.Nv, e.mgs_min.p, e.s);
  MG_CUDA(cudaMemsetAsync(C.Y.p, 0, C.Y.n * sizeof(Cx<double>), e.s));
  for (int colour = 0; colour < L.p0 * L.p1; ++colour)
    for (int k = 0; k < L.Nv; ++k) {
      probe_vector_kernel<<<grid_for(C.n, 256), 256, 0, e.s>>>(C.t.p, C.geo.L0, C.geo.L1, C.nint, L.p0, L.p1, colour,
                                                               k);
      MG_LAUNCHED();
      launch_zero<double>(L.t.p, L.n, e.s);
      launch_prolong_add<double>(L.V.p, C.t.p, L.t.p, L.bg, L.Nv, e.s);
      cg_apply(e, l, L.t.p, L.r2.p);
      launch_restrict<double>(L.V.p, L.r2.p, C.r2.p, L.bg, L.Nv, e.s);
      probe_scatter_kernel<<<grid_for(C.geo.nsites * kOffsets * C.nint, 256), 256, 0, e.s>>>(
          C.r2.p, C.Y.p, C.geo.L0, C.geo.L1, C.nint, L.p0, L.p1, colour, k);
      MG_LAUNCHED();
    }
}

// frozen smoother coefficients of every non-coarsest level (two MR steps on A x = b_l from 0,
// b_l Philox vector 0x2C of level l) and the LU factors of the coarsest level
static void cg_prepare(CgEngine &e) {
  for (int l = 0; l + 1 < (int)e.lv.size(); ++l) {
    CgLevel &L = e.lv[l];
    launch_gaussian(L.r.p, L.n, e.p.seed, kSmootherVector, l, e.s);
    for (int i = 0; i < 2; ++i) {
      cg_apply(e, l, L.r.p, L.w.p);
      double d[3];
      cg_dot(e, L.w.p, L.r.p, L.n, d);
      if (d[2] <= 0.0) fail(MG_ERR_NAN, "MG-CG: zero operator image in the smoother setup");
      L.alpha[i] = e.p.omega * d[0] / d[2];  // real for hermitian A
      step_kernel<<<blocks_for(L.n), 256, 0, e.s>>>(L.t.p, L.r.p, L.w.p, L.alpha[i], 0.0, L.n);
      MG_LAUNCHED();
    }
  }
  CgLevel &C = e.lv.back();
  const int n = (int)C.n;
  dense_from_stencil9_kernel<<<grid_for((long long)n * n, 256), 256, 0, e.s>>>(C.Y.p, e.LU.p, C.geo.L0, C.geo.L1,
                                                                              C.nint);
  MG_LAUNCHED();
  lu_factor(e.LU.p, n, e.ipiv.p, e.info.p, e.s);
  int info = 0;
  MG_CUDA(cudaMemcpyAsync(&info, e.info.p, sizeof(int), cudaMemcpyDeviceToHost, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
  if (info != 0) fail(MG_ERR_NAN, "MG-CG: coarsest LU hit a zero pivot");
}


static std::unique_ptr<CgEngine> cg_create(const mg_geom *g, const void *U, double m, const mg_params *p,
                                           void *stream) {
  if (!g || !p || !U) fail(MG_ERR_INVALID_ARG, "null geometry, links or parameters");
  if (g->d != 2 || g->Nc != 1) fail(MG_ERR_UNSUPPORTED, "MG-CG is built for d = 2, Nc = 1");
  if (p->levels < 2 || p->levels > MG_MAX_LEVELS) fail(MG_ERR_INVALID_ARG, "levels must be in [2, 4]");
  if (p->n_pass < 1 || p->nu_setup < 0) fail(MG_ERR_INVALID_ARG, "bad setup counts");
  if ((long long)g->dims[0] * g->dims[1] * 8 >= (1LL << 31)) fail(MG_ERR_UNSUPPORTED, "lattice too large");
  auto e = std::make_unique<CgEngine>();
  e->geom = *g;
  e->p = *p;
  e->m = m;
  e->user = static_cast<cudaStream_t>(stream);
  MG_CUDA(cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking));
  MG_CUDA(cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming));
  MG_CUDA(cudaEventRecord(e->ev, e->user));
  MG_CUDA(cudaStreamWaitEvent(e->s, e->ev, 0));
  MG_CUDA(cudaMallocHost(&e->host, 8 * sizeof(double)));
  e->lv.resize(p->levels);
  int L0 = g->dims[0], L1 = g->dims[1], nint = 2;
  for (int l = 0; l < p->levels; ++l) {
    CgLevel &L = e->lv[l];
    L.geo = Geo2{L0, L1, (long long)L0 * L1};
    L.nint = nint;
    L.n = L.geo.nsites * nint;
    for (DevBuf<Cx<double>> *b : {&L.b, &L.x, &L.r, &L.w, &L.t, &L.r2}) b->alloc((size_t)L.n);
    if (l > 0) L.Y.alloc((size_t)L.geo.nsites * kOffsets * nint * nint);
    if (l + 1 < p->levels) {
      const int B0 = p->block[l][0], B1 = p->block[l][1];
      if (B0 < 2 || B1 < 2 || L0 % B0 || L1 % B1)
        fail(MG_ERR_INVALID_ARG, "MG-CG: blocks must be at least 2 x 2 and divide the extents");
      L.Nv = p->Nv[l];
      if (L.Nv < 1 || L.Nv > B0 * B1 * nint || L.Nv > 32) fail(MG_ERR_INVALID_ARG, "MG-CG: bad Nv");
      L.bg = BlockGeo{L0, L1, B0, B1, L0 / B0, L1 / B1, B0 * B1, nint, B0 * B1 * nint,
                      (long long)(L0 / B0) * (L1 / B1)};
      L.p0 = colour_period(L0 / B0);
      L.p1 = colour_period(L1 / B1);
      L.V.alloc((size_t)L.Nv * L.n);
      L.vecs.alloc((size_t)L.Nv * L.n);
      L0 /= B0;
      L1 /= B1;
      nint = L.Nv;
    }
  }
  const long long nc = e->lv.back().n;
  if (nc > 4096) fail(MG_ERR_UNSUPPORTED, "MG-CG: the coarsest level is solved by dense LU (at most 4096 dofs)");
  e->LU.alloc((size_t)(nc * nc));
  e->lu_work.alloc((size_t)nc);
  e->ipiv.alloc((size_t)nc);
  e->info.alloc(1);
  const long long nf = e->lv[0].n;
  e->U.alloc((size_t)e->lv[0].geo.nsites * 2);
  e->tmp.alloc((size_t)nf);
  for (DevBuf<Cx<double>> *b : {&e->rhs, &e->cx, &e->cr, &e->cp, &e->cq, &e->cz}) b->alloc((size_t)nf);
  long long maxb = 1;
  for (auto &L : e->lv) maxb = std::max(maxb, L.bg.nblocks);
  e->mgs_min.alloc((size_t)maxb);
  e->ws.max_blocks = 152 * 8;
  e->ws.capacity = (long long)e->ws.max_blocks * 4;
  e->ws.tickets = 16;
  e->partials.alloc((size_t)e->ws.capacity);
  e->ws.partials = e->partials.p;
  e->dots.alloc(4);
  e->tickets.alloc((size_t)e->ws.tickets);
  e->ws.ticket = e->tickets.p;
  pool_ready();
  MG_CUDA(cudaMemsetAsync(e->tickets.p, 0, e->ws.tickets * sizeof(unsigned int), e->s));
  MG_CUDA(cudaMemcpyAsync(e->U.p, U, e->U.n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e->s));
  return e;
}

// the adaptive setup on A: pass 1 relaxes and builds every level in turn; passes 2..n_pass
// replace each vector v of level l by v - V_l(A v) and rebuild levels l, l + 1, ...
static void cg_setup(CgEngine &e) {
  const int nl = (int)e.lv.size();
  for (int l = 0; l + 1 < nl; ++l) {
    cg_relax(e, l);
    cg_build(e, l);
  }
  cg_prepare(e);
  for (int pass = 1; pass < e.p.n_pass; ++pass) {
    for (int l = 0; l + 1 < nl; ++l) {
      CgLevel &L = e.lv[l];
      for (int k = 0; k < L.Nv; ++k) {
        Cx<double> *v = L.vecs.p + (long long)k * L.n;
        cg_apply(e, l, v, L.b.p);
        cg_vcycle(e, l, L.b.p, L.x.p);
        launch_xmy<double>(v, L.x.p, L.n, e.s);  // x = v - V(A v)
        launch_copy<double>(L.x.p, v, L.n, e.s);
      }
      for (int q = l; q + 1 < nl; ++q) cg_build(e, q);
      cg_prepare(e);
    }
  }
  MG_CUDA(cudaStreamSynchronize(e.s));
}

// (preconditioned) CG on A psi = D^dagger chi from psi = 0 until |r| <= tol |D^dagger chi|
static void cg_solve(CgEngine &e, const Cx<double> *chi, Cx<double> *psi, double tol, int max_iter, bool precond,
                     mg_cg_stats *st) {
  const auto t0 = std::chrono::steady_clock::now();
  CgLevel &F = e.lv[0];
  const long long n = F.n;
  e.fine_apps = 0;
  // rhs = D^dagger chi = gamma5 D gamma5 chi
  launch_copy<double>(chi, e.cr.p, n, e.s);
  gamma5_kernel<<<grid_for(F.geo.nsites, 256), 256, 0, e.s>>>(e.cr.p, F.geo.nsites);
  MG_LAUNCHED();
  launch_dslash<double>(e.U.p, e.cr.p, e.rhs.p, F.geo, 2.0 + e.m, nullptr, 1.0, 0.0, e.s, 1, nullptr);
  gamma5_kernel<<<grid_for(F.geo.nsites, 256), 256, 0, e.s>>>(e.rhs.p, F.geo.nsites);
  MG_LAUNCHED();
  double d[3];
  cg_dot(e, e.rhs.p, e.rhs.p, n, d);
  const double bn2 = d[2];
  launch_zero<double>(e.cx.p, n, e.s);
  launch_copy<double>(e.rhs.p, e.cr.p, n, e.s);
  int it = 0;
  bool met = bn2 == 0.0;
  if (bn2 > 0.0) {
    if (precond)
      cg_vcycle(e, 0, e.cr.p, e.cz.p);
    else
      launch_copy<double>(e.cr.p, e.cz.p, n, e.s);
    launch_copy<double>(e.cz.p, e.cp.p, n, e.s);
    cg_dot(e, e.cr.p, e.cz.p, n, d);
    double rz = d[0], rn2 = bn2;
    const double tol2 = tol * tol * bn2;
    while (it < max_iter && rn2 > tol2) {
      cg_apply(e, 0, e.cp.p, e.cq.p);
      cg_dot(e, e.cp.p, e.cq.p, n, d);
      if (d[0] <= 0.0) fail(MG_ERR_NAN, "MG-CG: non-positive curvature <p, A p>");
      const double alpha = rz / d[0];
      cg_update_kernel<<<blocks_for(n), 256, 0, e.s>>>(e.cx.p, e.cr.p, e.cp.p, e.cq.p, alpha, n);
      MG_LAUNCHED();
      ++it;
      cg_dot(e, e.cr.p, e.cr.p, n, d);
      rn2 = d[2];
      if (precond)
        cg_vcycle(e, 0, e.cr.p, e.cz.p);
      else
        launch_copy<double>(e.cr.p, e.cz.p, n, e.s);
      cg_dot(e, e.cr.p, e.cz.p, n, d);
      const double beta = d[0] / rz;
      rz = d[0];
      direction_kernel<<<blocks_for(n), 256, 0, e.s>>>(e.cp.p, e.cz.p, beta, n);
      MG_LAUNCHED();
    }
    met = rn2 <= tol2;
  }
  const long long apps = e.fine_apps;
  // true residual of the normal equations
  cg_apply(e, 0, e.cx.p, e.cq.p);
  launch_xmy<double>(e.rhs.p, e.cq.p, n, e.s);
  cg_dot(e, e.cq.p, e.cq.p, n, d);
  MG_CUDA(cudaMemcpyAsync(psi, e.cx.p, n * sizeof(Cx<double>), cudaMemcpyDeviceToDevice, e.s));
  MG_CUDA(cudaStreamSynchronize(e.s));
  const double rel = bn2 > 0.0 ? std::sqrt(d[2] / bn2) : 0.0;
  if (st) {
    st->iters = it;
    st->converged = met ? 1 : 0;  // the CG criterion: the recursive residual met the tolerance
    st->rel_residual = rel;
    st->fine_apps = apps;
    st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
}

}  // namespace mg

// ===========================================================================
// C ABI
// ===========================================================================
struct mg_cg_ctx {
  std::unique_ptr<mg::CgEngine> e;
};

namespace {
template <typename F>
int cg_guarded(F &&f) {
  try {
    f();
    mg::set_last_error("");
    return MG_OK;
  } catch (const mg::Error &e) {
    mg::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    mg::set_last_error("host allocation failed");
    return MG_ERR_OOM;
  } catch (...) {
    mg::set_last_error("unexpected exception");
    return MG_ERR_CUDA;
  }
}
void cg_enter(mg_cg_ctx *c) {
  if (!c || !c->e) mg::fail(MG_ERR_INVALID_ARG, "null MG-CG context");
  MG_CUDA(cudaEventRecord(c->e->ev, c->e->user));
  MG_CUDA(cudaStreamWaitEvent(c->e->s, c->e->ev, 0));
}
}  // namespace

extern "C" {

int mg_cg_setup(mg_cg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, void *stream) {
  return cg_guarded([&] {
    if (!ctx) mg::fail(MG_ERR_INVALID_ARG, "null context out-pointer");
    *ctx = nullptr;
    auto c = std::make_unique<mg_cg_ctx>();
    c->e = mg::cg_create(g, U, m, p, stream);
    mg::cg_setup(*c->e);
    *ctx = c.release();
  });
}

int mg_cg_solve(mg_cg_ctx *ctx, const void *chi, void *psi, double tol, int max_iter, int precondition,
                mg_cg_stats *st) {
  return cg_guarded([&] {
    cg_enter(ctx);
    if (!chi || !psi) mg::fail(MG_ERR_INVALID_ARG, "null pointer");
    if (!(tol > 0.0) || max_iter < 1) mg::fail(MG_ERR_INVALID_ARG, "need tol > 0 and max_iter >= 1");
    mg_cg_stats local{};
    mg::cg_solve(*ctx->e, static_cast<const mg::Cx<double> *>(chi), static_cast<mg::Cx<double> *>(psi), tol, max_iter,
                 precondition != 0, &local);
    if (st) *st = local;
    if (!local.converged) mg::fail(MG_ERR_NOT_CONVERGED, "MG-CG: not converged within max_iter");
  });
}

int mg_cg_get_coarse_op(mg_cg_ctx *ctx, int level, void *out) {
  return cg_guarded([&] {
    cg_enter(ctx);
    if (!out) mg::fail(MG_ERR_INVALID_ARG, "null pointer");
    mg::CgEngine &e = *ctx->e;
    if (level < 1 || level >= (int)e.lv.size()) mg::fail(MG_ERR_INVALID_ARG, "level out of range");
    const mg::CgLevel &L = e.lv[level];
    MG_CUDA(cudaMemcpyAsync(out, L.Y.p, L.Y.n * sizeof(mg::Cx<double>), cudaMemcpyDeviceToDevice, e.s));
    MG_CUDA(cudaStreamSynchronize(e.s));
  });
}

int mg_cg_destroy(mg_cg_ctx *ctx) {
  return cg_guarded([&] { delete ctx; });
}

}  // extern "C"
