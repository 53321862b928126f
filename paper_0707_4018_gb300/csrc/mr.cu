// Fused minimum-residual (MR) smoothing kernels (paper: the relaxation steps
// of the V-cycle; MR with under-relaxation omega as the relaxation method).
//
// One MR iteration is  alpha = omega <A r, r> / |A r|^2,  x += alpha r,
// r -= alpha A r. Unfused, that is three kernels (apply, reduce, update). Here
// an iteration is one kernel: it reads the previous r and A r, forms
// r_new = r - alpha A r on the fly at the neighbours it needs, updates x and r
// at its own site, applies A to r_new and reduces <A r_new, r_new> and
// |A r_new|^2 (last-block reduction, fixed order; within a block the sums are
// in the vectors' precision, across blocks in FP64). r and A r alternate between
// two buffers, so no thread overwrites a value another thread still reads.
// nu MR iterations therefore cost nu + 1 launches.
#include "kernels.h"
#include "wilson.cuh"

namespace mg {

// alpha = omega <A r, r> / |A r|^2 from the FP64 sums, formed once per block by thread 0
// and broadcast through shared memory (an FP64 division per thread would cost GB300's
// slow FP64 unit more than the rest of these kernels); every thread must call it
template <typename R>
__device__ __forceinline__ Cx<R> mr_alpha(const double *sc, double omega) {
  __shared__ R s_alpha[2];
  if (threadIdx.x == 0) {
    const double den = sc[2];
    s_alpha[0] = (R)(den > 0.0 ? omega * sc[0] / den : 0.0);
    s_alpha[1] = (R)(den > 0.0 ? omega * sc[1] / den : 0.0);
  }
  __syncthreads();
  return mk(s_alpha[0], s_alpha[1]);
}

// value of the MR residual at a site: r (first iteration) or r - alpha A r
template <typename R, bool STEP>
struct MrSrc {
  const Cx<R> *r, *Ar;
  Cx<R> malpha;
  __device__ __forceinline__ Cx<R> at(long long i) const {
    Cx<R> v = r[i];
    if (STEP) cmac(v, malpha, Ar[i]);
    return v;
  }
};

// ---- fine Wilson level: one thread per site ----
template <typename R, bool STEP>
__global__ void __launch_bounds__(256) mr_wilson_kernel(const Cx<R> *__restrict__ U, const Cx<R> *r_old,
                                                        const Cx<R> *Ar_old, const double *sc_old, double omega,
                                                        Cx<R> *x, int x_init, Cx<R> *r_new, Cx<R> *Ar_new, int L0,
                                                        int L1, R diag, double *partials, double *sc_new,
                                                        unsigned int *ticket, const double *shift) {
  __shared__ R sh[32 * 3];
  if (shift != nullptr) diag += (R)shift[blockIdx.y];
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long V = (long long)L0 * L1;
  {  // vector blockIdx.y of the batch (stride 2 V); scalars, partials and ticket per vector
    const long long off = blockIdx.y * 2 * V;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      sc_old += 4 * blockIdx.y;
      x += off;
      r_new += off;
    }
    Ar_new += off;
    sc_new += 4 * blockIdx.y;
    partials += 3LL * gridDim.x * blockIdx.y;
    ticket += blockIdx.y;
  }
  R v[3] = {(R)0, (R)0, (R)0};
  Cx<R> alpha = mk((R)0, (R)0);
  if (STEP) alpha = mr_alpha<R>(sc_old, omega);  // all threads of the block
  if (s < V) {
    MrSrc<R, STEP> src;
    src.r = r_old;
    src.Ar = Ar_old;
    if (STEP) src.malpha = mk(-alpha.re, -alpha.im);
    const int x1 = (int)(s / L0), x0 = (int)(s - (long long)x1 * L0);
    const long long row = (long long)x1 * L0;
    const long long xp0 = row + (x0 + 1 == L0 ? 0 : x0 + 1);
    const long long xm0 = row + (x0 == 0 ? L0 - 1 : x0 - 1);
    const long long xp1 = (x1 + 1 == L1 ? 0 : row + L0) + x0;
    const long long xm1 = (x1 == 0 ? (long long)(L1 - 1) * L0 : row - L0) + x0;
    const Cx<R> s0 = src.at(2 * s), s1 = src.at(2 * s + 1);
    if (STEP) {
      const Cx<R> o0 = r_old[2 * s], o1 = r_old[2 * s + 1];
      Cx<R> xa = x_init ? mk((R)0, (R)0) : x[2 * s], xb = x_init ? mk((R)0, (R)0) : x[2 * s + 1];
      cmac(xa, alpha, o0);
      cmac(xb, alpha, o1);
      x[2 * s] = xa;
      x[2 * s + 1] = xb;
      r_new[2 * s] = s0;
      r_new[2 * s + 1] = s1;
    }
    const Pair<R> ux = reinterpret_cast<const Pair<R> *>(U)[s];
    const Cx<R> ub0 = U[2 * xm0 + 0], ub1 = U[2 * xm1 + 1];
    const Cx<R> f0a = src.at(2 * xp0), f0b = src.at(2 * xp0 + 1);
    const Cx<R> f1a = src.at(2 * xp1), f1b = src.at(2 * xp1 + 1);
    const Cx<R> g0a = src.at(2 * xm0), g0b = src.at(2 * xm0 + 1);
    const Cx<R> g1a = src.at(2 * xm1), g1b = src.at(2 * xm1 + 1);
    const Cx<R> t1 = ux.a * (f0a - f0b);
    const Cx<R> t2 = cmul_conj(ub0, g0a + g0b);
    const Cx<R> t3 = ux.b * (f1a + times_i(f1b));
    const Cx<R> t4 = cmul_conj(ub1, g1a - times_i(g1b));
    const Cx<R> hu = mk(t1.re + t2.re + t3.re + t4.re, t1.im + t2.im + t3.im + t4.im);
    const Cx<R> hl = mk(-t1.re + t2.re + t3.im - t4.im, -t1.im + t2.im - t3.re + t4.re);
    const R h = (R)0.5;
    const Cx<R> a0 = mk(diag * s0.re - h * hu.re, diag * s0.im - h * hu.im);
    const Cx<R> a1 = mk(diag * s1.re - h * hl.re, diag * s1.im - h * hl.im);
    Ar_new[2 * s] = a0;
    Ar_new[2 * s + 1] = a1;
    v[0] = a0.re * s0.re + a0.im * s0.im + a1.re * s1.re + a1.im * s1.im;
    v[1] = a0.re * s0.im - a0.im * s0.re + a1.re * s1.im - a1.im * s1.re;
    v[2] = a0.re * a0.re + a0.im * a0.im + a1.re * a1.re + a1.im * a1.im;
  }
  grid_finish_t<3, R>(v, partials, sc_new, ticket, sh);
}

// ---- coarse stencil level: one thread per (site, row) ----
template <typename R, bool STEP, int NT>
__global__ void __launch_bounds__(256) mr_stencil_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *r_old,
                                                         const Cx<R> *Ar_old, const double *sc_old, double omega,
                                                         Cx<R> *x, int x_init, Cx<R> *r_new, Cx<R> *Ar_new, int L0,
                                                         int L1, int Nrt, double *partials, double *sc_new,
                                                         unsigned int *ticket, const double *shift) {
  __shared__ R sh[32 * 3];
  const int N = NT > 0 ? NT : Nrt;
  {
    const long long off = blockIdx.y * (long long)L0 * L1 * N;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      sc_old += 4 * blockIdx.y;
      x += off;
      r_new += off;
    }
    Ar_new += off;
    sc_new += 4 * blockIdx.y;
    partials += 3LL * gridDim.x * blockIdx.y;
    ticket += blockIdx.y;
  }
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long j = t / N;
  const int row = (int)(t - j * N);
  R v[3] = {(R)0, (R)0, (R)0};
  Cx<R> alpha = mk((R)0, (R)0);
  if (STEP) alpha = mr_alpha<R>(sc_old, omega);  // all threads of the block
  if (j < (long long)L0 * L1) {
    MrSrc<R, STEP> src;
    src.r = r_old;
    src.Ar = Ar_old;
    if (STEP) src.malpha = mk(-alpha.re, -alpha.im);
    const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
    const long long rowo = (long long)x1 * L0;
    long long nb[5];
    nb[0] = j;
    nb[1] = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
    nb[2] = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
    nb[3] = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
    nb[4] = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
    const Cx<R> self = src.at(t);
    if (STEP) {
      Cx<R> xv = x_init ? mk((R)0, (R)0) : x[t];
      cmac(xv, alpha, r_old[t]);
      x[t] = xv;
      r_new[t] = self;
    }
    Cx<R> acc = mk((R)0, (R)0);
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const Cx<R> *Yd = Y + (j * 5 + dir) * (long long)N * N + row;
      const long long base = nb[dir] * N;
#pragma unroll(NT > 0 ? NT : 1)
      for (int col = 0; col < N; ++col) cmac(acc, Yd[(long long)col * N], src.at(base + col));
    }
    if (shift != nullptr) {  // self block + shift * identity for this vector
      const R sv = (R)shift[blockIdx.y];
      acc.re = fma(sv, self.re, acc.re);
      acc.im = fma(sv, self.im, acc.im);
    }
    Ar_new[t] = acc;
    v[0] = acc.re * self.re + acc.im * self.im;
    v[1] = acc.re * self.im - acc.im * self.re;
    v[2] = acc.re * acc.re + acc.im * acc.im;
  }
  grid_finish_t<3, R>(v, partials, sc_new, ticket, sh);
}

// ---- coarse stencil level with N = 8: four threads per (site, row), a warp per site ----
// Thread q of a row takes 10 of the 40 (direction, column) terms; the four partial rows
// are combined by shuffles. Four times the threads of the one-thread-per-row form and
// short FMA chains: these levels are small and latency-bound.
template <typename R>
__device__ __forceinline__ long long nbr_of(int dir, long long j, long long xp0, long long xm0, long long xp1,
                                            long long xm1) {
  return dir == 0 ? j : dir == 1 ? xp0 : dir == 2 ? xm0 : dir == 3 ? xp1 : xm1;
}

template <typename R, bool STEP>
__global__ void __launch_bounds__(256) mr_stencil8_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *r_old,
                                                          const Cx<R> *Ar_old, const double *sc_old, double omega,
                                                          Cx<R> *x, int x_init, Cx<R> *r_new, Cx<R> *Ar_new, int L0,
                                                          int L1, double *partials, double *sc_new,
                                                          unsigned int *ticket, const double *shift) {
  __shared__ R sh[32 * 3];
  {
    const long long off = blockIdx.y * (long long)L0 * L1 * 8;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      sc_old += 4 * blockIdx.y;
      x += off;
      r_new += off;
    }
    Ar_new += off;
    sc_new += 4 * blockIdx.y;
    partials += 3LL * gridDim.x * blockIdx.y;
    ticket += blockIdx.y;
  }
  const long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int row = (threadIdx.x >> 2) & 7, q = threadIdx.x & 3;
  R v[3] = {(R)0, (R)0, (R)0};
  Cx<R> alpha = mk((R)0, (R)0);
  if (STEP) alpha = mr_alpha<R>(sc_old, omega);  // all threads of the block
  if (j < (long long)L0 * L1) {  // uniform over the warp
    MrSrc<R, STEP> src;
    src.r = r_old;
    src.Ar = Ar_old;
    if (STEP) src.malpha = mk(-alpha.re, -alpha.im);
    const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
    const long long rowo = (long long)x1 * L0;
    const long long xp0 = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
    const long long xm0 = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
    const long long xp1 = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
    const long long xm1 = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
    Cx<R> acc = mk((R)0, (R)0);
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int term = q * 10 + u, dir = term >> 3, col = term & 7;
      const long long nbj = nbr_of<R>(dir, j, xp0, xm0, xp1, xm1);
      cmac(acc, Y[(j * 5 + dir) * 64 + col * 8 + row], src.at(nbj * 8 + col));
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (q == 0) {
      const long long i = j * 8 + row;
      const Cx<R> self = src.at(i);
      if (STEP) {
        Cx<R> xv = x_init ? mk((R)0, (R)0) : x[i];
        cmac(xv, alpha, r_old[i]);
        x[i] = xv;
        r_new[i] = self;
      }
      if (shift != nullptr) {
        const R sv = (R)shift[blockIdx.y];
        acc.re = fma(sv, self.re, acc.re);
        acc.im = fma(sv, self.im, acc.im);
      }
      Ar_new[i] = acc;
      v[0] = acc.re * self.re + acc.im * self.im;
      v[1] = acc.re * self.im - acc.im * self.re;
      v[2] = acc.re * acc.re + acc.im * acc.im;
    }
  }
  grid_finish_t<3, R>(v, partials, sc_new, ticket, sh);
}

// x (+)= alpha r for the last MR iteration; with r_out, also the final residual
// r_out = r_old - alpha A r_old (= b - A x; r_out may be r_old)
template <typename R>
__global__ void mr_last_kernel(const Cx<R> *r_old, const Cx<R> *__restrict__ Ar_old, const double *__restrict__ sc_old,
                               double omega, Cx<R> *__restrict__ x, int x_init, Cx<R> *r_out, long long n) {
  r_old += blockIdx.y * n;
  x += blockIdx.y * n;
  const Cx<R> alpha = mr_alpha<R>(sc_old + 4 * blockIdx.y, omega);
  const Cx<R> malpha = mk(-alpha.re, -alpha.im);
  if (r_out != nullptr) {
    Ar_old += blockIdx.y * n;
    r_out += blockIdx.y * n;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> ri = r_old[i];
    Cx<R> xv = x_init ? mk((R)0, (R)0) : x[i];
    cmac(xv, alpha, ri);
    x[i] = xv;
    if (r_out != nullptr) {
      Cx<R> rn = ri;
      cmac(rn, malpha, Ar_old[i]);
      r_out[i] = rn;
    }
  }
}

// ---------------------------------------------------------------------------
template <typename R>
void launch_mr_iteration(const OpDesc<R> &op, bool step, const Cx<R> *r_old, const Cx<R> *Ar_old, const double *sc_old,
                         double omega, Cx<R> *x, bool x_init, Cx<R> *r_new, Cx<R> *Ar_new, double *sc_new,
                         const ReduceWs &ws, cudaStream_t s, int nvec) {
  const int threads = 256;
  if (nvec > 128) fail(MG_ERR_UNSUPPORTED, "MR batch larger than 128 vectors");
  if (op.wilson) {
    const dim3 grid(grid_for(op.geo.nsites, threads), nvec);
    if ((long long)grid.x * 3 * nvec > ws.capacity) fail(MG_ERR_STATE, "MR reduction workspace too small");
    if (step)
      mr_wilson_kernel<R, true><<<grid, threads, 0, s>>>(op.U, r_old, Ar_old, sc_old, omega, x, x_init ? 1 : 0, r_new,
                                                         Ar_new, op.geo.L0, op.geo.L1, (R)op.diag, ws.partials,
                                                         sc_new, ws.ticket, op.shift);
    else
      mr_wilson_kernel<R, false><<<grid, threads, 0, s>>>(op.U, r_old, Ar_old, sc_old, omega, x, 0, r_new, Ar_new,
                                                          op.geo.L0, op.geo.L1, (R)op.diag, ws.partials, sc_new,
                                                          ws.ticket, op.shift);
  } else if (op.N == 8) {
    const dim3 grid(grid_for(op.geo.nsites * 32, threads), nvec);
    if ((long long)grid.x * 3 * nvec > ws.capacity) fail(MG_ERR_STATE, "MR reduction workspace too small");
    if (step)
      mr_stencil8_kernel<R, true><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, sc_old, omega, x, x_init ? 1 : 0,
                                                           r_new, Ar_new, op.geo.L0, op.geo.L1, ws.partials, sc_new,
                                                           ws.ticket, op.shift);
    else
      mr_stencil8_kernel<R, false><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, sc_old, omega, x, 0, r_new, Ar_new,
                                                            op.geo.L0, op.geo.L1, ws.partials, sc_new, ws.ticket,
                                                            op.shift);
  } else {
    const dim3 grid(grid_for(op.geo.nsites * op.N, threads), nvec);
    if ((long long)grid.x * 3 * nvec > ws.capacity) fail(MG_ERR_STATE, "MR reduction workspace too small");
#define MG_MR_STENCIL(STEPV, NTV)                                                                                    \
  mr_stencil_kernel<R, STEPV, NTV><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, sc_old, omega, x, x_init ? 1 : 0,   \
                                                            r_new, Ar_new, op.geo.L0, op.geo.L1, op.N, ws.partials, \
                                                            sc_new, ws.ticket, op.shift)
    if (step) MG_MR_STENCIL(true, 0); else MG_MR_STENCIL(false, 0);
#undef MG_MR_STENCIL
  }
  MG_LAUNCHED();
}

template <typename R>
void launch_mr_last(const Cx<R> *r_old, const double *sc_old, double omega, Cx<R> *x, bool x_init, long long n,
                    cudaStream_t s, int nvec, const Cx<R> *Ar_old, Cx<R> *r_out) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  mr_last_kernel<R><<<dim3((unsigned int)(b < 1 ? 1 : b), nvec), 256, 0, s>>>(r_old, Ar_old, sc_old, omega, x,
                                                                              x_init ? 1 : 0, r_out, n);
  MG_LAUNCHED();
}

template void launch_mr_iteration<double>(const OpDesc<double> &, bool, const Cx<double> *, const Cx<double> *,
                                          const double *, double, Cx<double> *, bool, Cx<double> *, Cx<double> *,
                                          double *, const ReduceWs &, cudaStream_t, int);
template void launch_mr_iteration<float>(const OpDesc<float> &, bool, const Cx<float> *, const Cx<float> *,
                                         const double *, double, Cx<float> *, bool, Cx<float> *, Cx<float> *,
                                         double *, const ReduceWs &, cudaStream_t, int);
template void launch_mr_last<double>(const Cx<double> *, const double *, double, Cx<double> *, bool, long long,
                                     cudaStream_t, int, const Cx<double> *, Cx<double> *);
template void launch_mr_last<float>(const Cx<float> *, const double *, double, Cx<float> *, bool, long long,
                                    cudaStream_t, int, const Cx<float> *, Cx<float> *);

}  // namespace mg
