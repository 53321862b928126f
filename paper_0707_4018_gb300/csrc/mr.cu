// Fused minimum-residual (MR) smoothing kernels (paper: the relaxation steps
// of the V-cycle; MR with under-relaxation omega as the relaxation method).
//
// One MR iteration is  alpha = omega <A r, r> / |A r|^2,  x += alpha r,
// r -= alpha A r. Unfused, that is three kernels (apply, reduce, update). Here
// an iteration is one kernel: it reads the previous r and A r, forms
// r_new = r - alpha A r on the fly at the neighbours it needs, updates x and r
// at its own site, applies A to r_new and publishes its block's sums of
// <A r_new, r_new> and |A r_new|^2. nu MR iterations cost nu + 1 launches.
//
// Reductions are finished by the consumer: every block of the next launch sums
// the previous launch's block partials itself, in one fixed order (so every
// block, and every run, forms the same alpha), while its own loads of r, A r
// and the operator are already in flight. The producer has no tail (no fence,
// ticket or last block), which matters because these small levels are latency-
// bound. Partials alternate between two buffers; r and A r alternate between
// two buffers too, so no thread overwrites a value another thread still reads.
// Sums are in the vectors' precision.
#include "kernels.h"
#include "mr.cuh"
#include "wilson.cuh"

namespace mg {

// ---- fine Wilson level: one thread per site ----
template <typename R, bool STEP>
__global__ void __launch_bounds__(256) mr_wilson_kernel(const Cx<R> *__restrict__ U, const Cx<R> *r_old,
                                                        const Cx<R> *Ar_old, const R *part_in, int nb_in,
                                                        double omega, Cx<R> *x, int x_init, Cx<R> *r_new,
                                                        Cx<R> *Ar_new, int L0, int L1, R diag, R *part_out,
                                                        const double *shift) {
  __shared__ R sh[32 * 3];
  if (shift != nullptr) diag += (R)shift[blockIdx.y];
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long V = (long long)L0 * L1;
  {  // vector blockIdx.y of the batch (stride 2 V); partials per vector
    const long long off = blockIdx.y * 2 * V;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      x += off;
      r_new += off;
      part_in += 3LL * nb_in * blockIdx.y;
    }
    Ar_new += off;
    part_out += 3LL * gridDim.x * blockIdx.y;
  }
  // issue every load of the site first; alpha (a reduction) overlaps with them
  const bool live = s < V;
  const Cx<R> z = mk((R)0, (R)0);
  Cx<R> rv[10], av[10];  // self, +0, +1, -0, -1 (two spin components each)
  Cx<R> xa = z, xb = z, ux0 = z, ux1 = z, ub0 = z, ub1 = z;
#pragma unroll
  for (int k = 0; k < 10; ++k) rv[k] = av[k] = z;
  if (live) {
    const int x1 = (int)(s / L0), x0 = (int)(s - (long long)x1 * L0);
    const long long row = (long long)x1 * L0;
    const long long nbr[5] = {s, row + (x0 + 1 == L0 ? 0 : x0 + 1), (x1 + 1 == L1 ? 0 : row + L0) + x0,
                              row + (x0 == 0 ? L0 - 1 : x0 - 1),
                              (x1 == 0 ? (long long)(L1 - 1) * L0 : row - L0) + x0};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      rv[2 * k] = r_old[2 * nbr[k]];
      rv[2 * k + 1] = r_old[2 * nbr[k] + 1];
      if (STEP) {
        av[2 * k] = Ar_old[2 * nbr[k]];
        av[2 * k + 1] = Ar_old[2 * nbr[k] + 1];
      }
    }
    if (STEP && !x_init) {
      xa = x[2 * s];
      xb = x[2 * s + 1];
    }
    const Pair<R> ux = reinterpret_cast<const Pair<R> *>(U)[s];
    ux0 = ux.a;
    ux1 = ux.b;
    ub0 = U[2 * nbr[3] + 0];
    ub1 = U[2 * nbr[4] + 1];
  }
  Cx<R> alpha = z;
  if (STEP) alpha = mr_alpha<R>(part_in, nb_in, omega, sh);  // all threads of the block
  R v[3] = {(R)0, (R)0, (R)0};
  if (live) {
    const Cx<R> ma = mk(-alpha.re, -alpha.im);
    Cx<R> w[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) w[k] = STEP ? mr_step(rv[k], av[k], ma) : rv[k];
    if (STEP) {
      cmac(xa, alpha, rv[0]);
      cmac(xb, alpha, rv[1]);
      x[2 * s] = xa;
      x[2 * s + 1] = xb;
      r_new[2 * s] = w[0];
      r_new[2 * s + 1] = w[1];
    }
    const Cx<R> s0 = w[0], s1 = w[1];
    const Cx<R> t1 = ux0 * (w[2] - w[3]);                    // +0: (1 - s1) U psi(x+0)
    const Cx<R> t2 = cmul_conj(ub0, w[6] + w[7]);            // -0: (1 + s1) U^* psi(x-0)
    const Cx<R> t3 = ux1 * (w[4] + times_i(w[5]));           // +1: (1 - s2) U psi(x+1)
    const Cx<R> t4 = cmul_conj(ub1, w[8] - times_i(w[9]));   // -1: (1 + s2) U^* psi(x-1)
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
  mr_publish<R>(v, part_out, sh);
}

// ---- coarse stencil level, N = 8: four threads per (site, row), a warp per site ----
// Thread q of a row takes 10 of the 40 (direction, column) terms; the four partial rows
// are combined by shuffles. The stencil is linear, so before alpha is known the thread
// accumulates Y r and Y (A r) separately and forms Y (r - alpha A r) = Y r - alpha Y A r
// afterwards: the loads overlap the reduction without holding them in registers.
template <typename R, bool STEP>
__global__ void __launch_bounds__(256) mr_stencil8_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *r_old,
                                                          const Cx<R> *Ar_old, const R *part_in, int nb_in,
                                                          double omega, Cx<R> *x, int x_init, Cx<R> *r_new,
                                                          Cx<R> *Ar_new, int L0, int L1, R *part_out,
                                                          const double *shift) {
  __shared__ R sh[32 * 3];
  {
    const long long off = blockIdx.y * (long long)L0 * L1 * 8;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      x += off;
      r_new += off;
      part_in += 3LL * nb_in * blockIdx.y;
    }
    Ar_new += off;
    part_out += 3LL * gridDim.x * blockIdx.y;
  }
  const long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int row = (threadIdx.x >> 2) & 7, q = threadIdx.x & 3;
  const bool live = j < (long long)L0 * L1;  // uniform over the warp
  const long long i = j * 8 + row;
  const Cx<R> z = mk((R)0, (R)0);
  Cx<R> acc_r = z, acc_a = z;  // Y r and Y (A r) over this thread's terms
  Cx<R> rself = z, aself = z, xself = z;
  if (live) {
    const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
    const long long rowo = (long long)x1 * L0;
    const long long xp0 = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
    const long long xm0 = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
    const long long xp1 = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
    const long long xm1 = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
    if (q == 0) {
      rself = r_old[i];
      if (STEP) {
        aself = Ar_old[i];
        if (!x_init) xself = x[i];
      }
    }
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int term = q * 10 + u, dir = term >> 3, col = term & 7;
      const long long nbj = dir == 0 ? j : dir == 1 ? xp0 : dir == 2 ? xm0 : dir == 3 ? xp1 : xm1;
      const Cx<R> yv = Y[(j * 5 + dir) * 64 + col * 8 + row];
      cmac(acc_r, yv, r_old[nbj * 8 + col]);
      if (STEP) cmac(acc_a, yv, Ar_old[nbj * 8 + col]);
    }
  }
  Cx<R> alpha = z;
  if (STEP) alpha = mr_alpha<R>(part_in, nb_in, omega, sh);  // all threads of the block
  R v[3] = {(R)0, (R)0, (R)0};
  if (live) {
    const Cx<R> ma = mk(-alpha.re, -alpha.im);
    Cx<R> acc = STEP ? mr_step(acc_r, acc_a, ma) : acc_r;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (q == 0) {
      const Cx<R> self = STEP ? mr_step(rself, aself, ma) : rself;
      if (STEP) {
        cmac(xself, alpha, rself);
        x[i] = xself;
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
  mr_publish<R>(v, part_out, sh);
}

// ---- coarse stencil level, any N: one thread per (site, row) ----
template <typename R, bool STEP>
__global__ void __launch_bounds__(256) mr_stencil_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *r_old,
                                                         const Cx<R> *Ar_old, const R *part_in, int nb_in,
                                                         double omega, Cx<R> *x, int x_init, Cx<R> *r_new,
                                                         Cx<R> *Ar_new, int L0, int L1, int N, R *part_out,
                                                         const double *shift) {
  __shared__ R sh[32 * 3];
  {
    const long long off = blockIdx.y * (long long)L0 * L1 * N;
    r_old += off;
    if (STEP) {
      Ar_old += off;
      x += off;
      r_new += off;
      part_in += 3LL * nb_in * blockIdx.y;
    }
    Ar_new += off;
    part_out += 3LL * gridDim.x * blockIdx.y;
  }
  Cx<R> alpha = mk((R)0, (R)0);
  if (STEP) alpha = mr_alpha<R>(part_in, nb_in, omega, sh);  // all threads of the block
  const Cx<R> ma = mk(-alpha.re, -alpha.im);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long j = t / N;
  const int row = (int)(t - j * N);
  R v[3] = {(R)0, (R)0, (R)0};
  if (j < (long long)L0 * L1) {
    auto src = [&](long long k) { return STEP ? mr_step(r_old[k], Ar_old[k], ma) : r_old[k]; };
    const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
    const long long rowo = (long long)x1 * L0;
    long long nb[5];
    nb[0] = j;
    nb[1] = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
    nb[2] = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
    nb[3] = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
    nb[4] = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
    const Cx<R> self = src(t);
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
      for (int col = 0; col < N; ++col) cmac(acc, Yd[(long long)col * N], src(base + col));
    }
    if (shift != nullptr) {
      const R sv = (R)shift[blockIdx.y];
      acc.re = fma(sv, self.re, acc.re);
      acc.im = fma(sv, self.im, acc.im);
    }
    Ar_new[t] = acc;
    v[0] = acc.re * self.re + acc.im * self.im;
    v[1] = acc.re * self.im - acc.im * self.re;
    v[2] = acc.re * acc.re + acc.im * acc.im;
  }
  mr_publish<R>(v, part_out, sh);
}

// x (+)= alpha r for the last MR iteration; with r_out, also the final residual
// r_out = r_old - alpha A r_old (= b - A x; r_out may be r_old)
template <typename R>
__global__ void mr_last_kernel(const Cx<R> *r_old, const Cx<R> *Ar_old, const R *part_in, int nb_in, double omega,
                               Cx<R> *__restrict__ x, int x_init, Cx<R> *r_out, long long n) {
  __shared__ R sh[32 * 3];
  r_old += blockIdx.y * n;
  x += blockIdx.y * n;
  Ar_old += blockIdx.y * n;
  if (r_out != nullptr) r_out += blockIdx.y * n;
  const Cx<R> alpha = mr_alpha<R>(part_in + 3LL * nb_in * blockIdx.y, nb_in, omega, sh);
  const Cx<R> malpha = mk(-alpha.re, -alpha.im);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> ri = r_old[i];
    Cx<R> xv = x_init ? mk((R)0, (R)0) : x[i];
    cmac(xv, alpha, ri);
    x[i] = xv;
    if (r_out != nullptr) r_out[i] = mr_step(ri, Ar_old[i], malpha);
  }
}

// ---------------------------------------------------------------------------
template <typename R>
int mr_grid(const OpDesc<R> &op) {
  const int threads = 256;
  if (op.wilson) return (int)grid_for(op.geo.nsites, threads);
  if (op.N == 8) return (int)grid_for(op.geo.nsites * 32, threads);
  return (int)grid_for(op.geo.nsites * op.N, threads);
}

template <typename R>
void launch_mr_iteration(const OpDesc<R> &op, bool step, const Cx<R> *r_old, const Cx<R> *Ar_old, const R *part_in,
                         double omega, Cx<R> *x, bool x_init, Cx<R> *r_new, Cx<R> *Ar_new, R *part_out,
                         long long part_capacity, cudaStream_t s, int nvec) {
  const int threads = 256;
  if (nvec > 128) fail(MG_ERR_UNSUPPORTED, "MR batch larger than 128 vectors");
  const int nb = mr_grid(op);
  if (3LL * nb * nvec > part_capacity) fail(MG_ERR_STATE, "MR reduction workspace too small");
  const dim3 grid(nb, nvec);
  const int xi = x_init ? 1 : 0;
  if (op.wilson) {
    if (step)
      mr_wilson_kernel<R, true><<<grid, threads, 0, s>>>(op.U, r_old, Ar_old, part_in, nb, omega, x, xi, r_new,
                                                         Ar_new, op.geo.L0, op.geo.L1, (R)op.diag, part_out, op.shift);
    else
      mr_wilson_kernel<R, false><<<grid, threads, 0, s>>>(op.U, r_old, Ar_old, part_in, nb, omega, x, 0, r_new, Ar_new,
                                                          op.geo.L0, op.geo.L1, (R)op.diag, part_out, op.shift);
  } else if (op.N == 8) {
    if (step)
      mr_stencil8_kernel<R, true><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, part_in, nb, omega, x, xi, r_new,
                                                           Ar_new, op.geo.L0, op.geo.L1, part_out, op.shift);
    else
      mr_stencil8_kernel<R, false><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, part_in, nb, omega, x, 0, r_new,
                                                            Ar_new, op.geo.L0, op.geo.L1, part_out, op.shift);
  } else {
    if (step)
      mr_stencil_kernel<R, true><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, part_in, nb, omega, x, xi, r_new,
                                                          Ar_new, op.geo.L0, op.geo.L1, op.N, part_out, op.shift);
    else
      mr_stencil_kernel<R, false><<<grid, threads, 0, s>>>(op.Y, r_old, Ar_old, part_in, nb, omega, x, 0, r_new,
                                                           Ar_new, op.geo.L0, op.geo.L1, op.N, part_out, op.shift);
  }
  MG_LAUNCHED();
}

template <typename R>
void launch_mr_last(const OpDesc<R> &op, const Cx<R> *r_old, const Cx<R> *Ar_old, const R *part_in, double omega,
                    Cx<R> *x, bool x_init, Cx<R> *r_out, long long n, cudaStream_t s, int nvec) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  mr_last_kernel<R><<<dim3((unsigned int)(b < 1 ? 1 : b), nvec), 256, 0, s>>>(
      r_old, Ar_old, part_in, mr_grid(op), omega, x, x_init ? 1 : 0, r_out, n);
  MG_LAUNCHED();
}

#define MG_INST_MR(R)                                                                                              \
  template int mr_grid<R>(const OpDesc<R> &);                                                                      \
  template void launch_mr_iteration<R>(const OpDesc<R> &, bool, const Cx<R> *, const Cx<R> *, const R *, double,  \
                                       Cx<R> *, bool, Cx<R> *, Cx<R> *, R *, long long, cudaStream_t, int);        \
  template void launch_mr_last<R>(const OpDesc<R> &, const Cx<R> *, const Cx<R> *, const R *, double, Cx<R> *,     \
                                  bool, Cx<R> *, long long, cudaStream_t, int);
MG_INST_MR(double)
MG_INST_MR(float)
#undef MG_INST_MR

}  // namespace mg
