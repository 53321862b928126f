// Fine Wilson operator on the 2d U(1) lattice (paper, definition of D
// following Eq. 1; diagonal d + m, periodic boundaries).
//
// One thread per site, site-major fields: psi[x] = (psi0, psi1) (one 16-byte
// load in FP32, two in FP64), U[x] = (U_x^0, U_x^1). Neighbour rows are reused
// through L1/L2, so each field streams from HBM about once per apply: 6
// complex numbers per site (psi in, U, psi out) = 48 B (FP32) / 96 B (FP64).
// The fused epilogue out = a * D in + c * b forms residuals b - D x in the
// same pass.
#include "kernels.h"
#include "wilson.cuh"

namespace mg {

// FP32: at most 32 registers, so that 8 blocks of 256 threads fit an SM (this kernel is
// HBM-bound and needs the memory parallelism of full occupancy)
template <typename R, bool SHIFT>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 8 : 4) dslash_kernel(const Cx<R> *__restrict__ U, const Cx<R> *__restrict__ in,
                                                     Cx<R> *__restrict__ out, int L0, int L1, R diag,
                                                     const Cx<R> *__restrict__ b, R a, R c, long long ldv,
                                                     const double *__restrict__ shift) {
  // vector blockIdx.y of a batch stored with stride ldv (the links are shared); its
  // diagonal is diag + shift[blockIdx.y] when a shift array is given
  if (SHIFT) diag += (R)shift[blockIdx.y];
  in += blockIdx.y * ldv;
  out += blockIdx.y * ldv;
  if (b != nullptr) b += blockIdx.y * ldv;
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long V = (long long)L0 * L1;
  if (x >= V) return;
  const int x1 = (int)(x / L0), x0 = (int)(x - (long long)x1 * L0);
  const long long row = (long long)x1 * L0;
  const long long xp0 = row + (x0 + 1 == L0 ? 0 : x0 + 1);
  const long long xm0 = row + (x0 == 0 ? L0 - 1 : x0 - 1);
  const long long xp1 = (x1 + 1 == L1 ? 0 : row + L0) + x0;
  const long long xm1 = (x1 == 0 ? (long long)(L1 - 1) * L0 : row - L0) + x0;

  const Pair<R> *P = reinterpret_cast<const Pair<R> *>(in);
  const Pair<R> *UL = reinterpret_cast<const Pair<R> *>(U);
  const Pair<R> self = P[x];
  const Pair<R> ux = UL[x];
  const Pair<R> f0 = P[xp0], f1 = P[xp1], g0 = P[xm0], g1 = P[xm1];
  const Cx<R> ub0 = U[2 * xm0 + 0], ub1 = U[2 * xm1 + 1];

  const Cx<R> t1 = ux.a * (f0.a - f0.b);                 // +0: (1 - s1) U psi(x+0)
  const Cx<R> t2 = cmul_conj(ub0, g0.a + g0.b);          // -0: (1 + s1) U^* psi(x-0)
  const Cx<R> t3 = ux.b * (f1.a + times_i(f1.b));        // +1: (1 - s2) U psi(x+1)
  const Cx<R> t4 = cmul_conj(ub1, g1.a - times_i(g1.b)); // -1: (1 + s2) U^* psi(x-1)

  // upper: t1 + t2 + t3 + t4; lower: -t1 + t2 - i t3 + i t4
  Cx<R> hu = mk(t1.re + t2.re + t3.re + t4.re, t1.im + t2.im + t3.im + t4.im);
  Cx<R> hl = mk(-t1.re + t2.re + t3.im - t4.im, -t1.im + t2.im - t3.re + t4.re);
  const R h = (R)0.5;
  Cx<R> o0 = mk(diag * self.a.re - h * hu.re, diag * self.a.im - h * hu.im);
  Cx<R> o1 = mk(diag * self.b.re - h * hl.re, diag * self.b.im - h * hl.im);
  Pair<R> res;
  if (b != nullptr) {
    const Pair<R> bb = reinterpret_cast<const Pair<R> *>(b)[x];
    res.a = mk(a * o0.re + c * bb.a.re, a * o0.im + c * bb.a.im);
    res.b = mk(a * o1.re + c * bb.b.re, a * o1.im + c * bb.b.im);
  } else {
    res.a = mk(a * o0.re, a * o0.im);
    res.b = mk(a * o1.re, a * o1.im);
  }
  reinterpret_cast<Pair<R> *>(out)[x] = res;
}

template <typename R>
void launch_dslash(const Cx<R> *U, const Cx<R> *in, Cx<R> *out, Geo2 g, double diag, const Cx<R> *b, double a,
                   double c, cudaStream_t s, int nvec, const double *shift) {
  const int threads = 256;
  const dim3 grid(grid_for(g.nsites, threads), nvec);
  if (shift != nullptr)
    dslash_kernel<R, true><<<grid, threads, 0, s>>>(U, in, out, g.L0, g.L1, (R)diag, b, (R)a, (R)c, 2 * g.nsites, shift);
  else
    dslash_kernel<R, false><<<grid, threads, 0, s>>>(U, in, out, g.L0, g.L1, (R)diag, b, (R)a, (R)c, 2 * g.nsites,
                                                     nullptr);
  MG_LAUNCHED();
}

template void launch_dslash<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, Geo2, double,
                                    const Cx<double> *, double, double, cudaStream_t, int,
                                    const double *);
template void launch_dslash<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, Geo2, double,
                                   const Cx<float> *, double, double, cudaStream_t, int,
                                   const double *);

}  // namespace mg
