// Coarse levels: the Galerkin stencil operator y_j = sum_dir Y[j][dir] x_{j+dir}
// (paper, Eq. Galerkin with A = D) and the exact coarsest solve by dense LU
// with partial pivoting.
//
// Coarse apply: one thread per (coarse site, row); Y is stored column-major per
// block (Y[j][dir][col][row]) so the N threads of a site read each column of a
// block with unit stride, and the N input values of a neighbour are broadcast.
// Bytes per coarse site: 5 N^2 complex of Y plus 2 N of x, y (N = 8: 5.4 KB in
// FP64, 2.7 KB in FP32).
#include "kernels.h"

namespace mg {

template <typename R, int NT>
__global__ void __launch_bounds__(256) coarse_apply_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *__restrict__ in,
                                                           Cx<R> *__restrict__ out, int L0, int L1, int Nrt,
                                                           const Cx<R> *__restrict__ b, R a, R c, long long ldv,
                                                           const double *__restrict__ shift) {
  in += blockIdx.y * ldv;
  out += blockIdx.y * ldv;
  if (b != nullptr) b += blockIdx.y * ldv;
  const int N = NT > 0 ? NT : Nrt;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long j = t / N;
  const int row = (int)(t - j * N);
  if (j >= (long long)L0 * L1) return;
  const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
  const long long rowo = (long long)x1 * L0;
  long long src[5];
  src[0] = j;
  src[1] = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
  src[2] = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
  src[3] = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
  src[4] = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
  Cx<R> acc = mk((R)0, (R)0);
#pragma unroll
  for (int dir = 0; dir < 5; ++dir) {
    const Cx<R> *Yd = Y + (j * 5 + dir) * (long long)N * N + row;
    const Cx<R> *xs = in + src[dir] * N;
#pragma unroll(NT > 0 ? NT : 1)
    for (int col = 0; col < N; ++col) cmac(acc, Yd[(long long)col * N], xs[col]);
  }
  if (shift != nullptr) {  // vector blockIdx.y: self block + shift * identity
    const R sv = (R)shift[blockIdx.y];
    const Cx<R> xt = in[t];
    acc.re = fma(sv, xt.re, acc.re);
    acc.im = fma(sv, xt.im, acc.im);
  }
  Cx<R> o = mk(a * acc.re, a * acc.im);
  if (b != nullptr) {
    const Cx<R> bb = b[t];
    o = mk(o.re + c * bb.re, o.im + c * bb.im);
  }
  out[t] = o;
}

// N = 8: four threads per (site, row), a warp per site (10 of the 40 terms each,
// combined by shuffles)
template <typename R>
__global__ void __launch_bounds__(256) coarse_apply8_kernel(const Cx<R> *__restrict__ Y, const Cx<R> *__restrict__ in,
                                                            Cx<R> *__restrict__ out, int L0, int L1,
                                                            const Cx<R> *__restrict__ b, R a, R c, long long ldv,
                                                            const double *__restrict__ shift) {
  in += blockIdx.y * ldv;
  out += blockIdx.y * ldv;
  if (b != nullptr) b += blockIdx.y * ldv;
  const long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int row = (threadIdx.x >> 2) & 7, q = threadIdx.x & 3;
  if (j >= (long long)L0 * L1) return;  // whole warps
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
    const long long nbj = dir == 0 ? j : dir == 1 ? xp0 : dir == 2 ? xm0 : dir == 3 ? xp1 : xm1;
    cmac(acc, Y[(j * 5 + dir) * 64 + col * 8 + row], in[nbj * 8 + col]);
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  if (q != 0) return;
  const long long t = j * 8 + row;
  if (shift != nullptr) {
    const R sv = (R)shift[blockIdx.y];
    const Cx<R> xt = in[t];
    acc.re = fma(sv, xt.re, acc.re);
    acc.im = fma(sv, xt.im, acc.im);
  }
  Cx<R> o = mk(a * acc.re, a * acc.im);
  if (b != nullptr) {
    const Cx<R> bb = b[t];
    o = mk(o.re + c * bb.re, o.im + c * bb.im);
  }
  out[t] = o;
}

template <typename R>
void launch_coarse_apply(const Cx<R> *Y, const Cx<R> *in, Cx<R> *out, Geo2 g, int N, const Cx<R> *b, double a,
                         double c, cudaStream_t s, int nvec, const double *shift) {
  const int threads = 256;
  const dim3 grid(grid_for(g.nsites * N, threads), nvec);
  const long long ldv = g.nsites * N;
  if (N == 8)
    coarse_apply8_kernel<R><<<dim3(grid_for(g.nsites * 32, threads), nvec), threads, 0, s>>>(Y, in, out, g.L0, g.L1, b,
                                                                                            (R)a, (R)c, ldv, shift);
  else
    coarse_apply_kernel<R, 0><<<grid, threads, 0, s>>>(Y, in, out, g.L0, g.L1, N, b, (R)a, (R)c, ldv, shift);
  MG_LAUNCHED();
}

template void launch_coarse_apply<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, Geo2, int,
                                          const Cx<double> *, double, double, cudaStream_t, int, const double *);
template void launch_coarse_apply<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, Geo2, int,
                                         const Cx<float> *, double, double, cudaStream_t, int, const double *);

// ---------------------------------------------------------------------------
// dense matrix of the coarsest stencil, column-major A[col * n + row]
// ---------------------------------------------------------------------------
__global__ void dense_from_stencil_kernel(const Cx<double> *__restrict__ Y, Cx<double> *__restrict__ A, int L0, int L1,
                                          int N, double shift) {
  const long long n = (long long)L0 * L1 * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const long long col = t / n, row = t - col * n;
  const long long j = row / N, sc = col / N;
  const int ar = (int)(row - j * N), ac = (int)(col - sc * N);
  const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
  const long long rowo = (long long)x1 * L0;
  long long src[5];
  src[0] = j;
  src[1] = rowo + (x0 + 1 == L0 ? 0 : x0 + 1);
  src[2] = rowo + (x0 == 0 ? L0 - 1 : x0 - 1);
  src[3] = (x1 + 1 == L1 ? 0 : rowo + L0) + x0;
  src[4] = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0;
  Cx<double> v = mk(0.0, 0.0);
  for (int dir = 0; dir < 5; ++dir)
    if (src[dir] == sc) v = v + Y[(j * 5 + dir) * (long long)N * N + (long long)ac * N + ar];
  if (row == col) v.re += shift;
  A[t] = v;
}

void launch_dense_from_stencil(const Cx<double> *Y, Cx<double> *A, Geo2 g, int N, cudaStream_t s, double shift) {
  const long long n = g.nsites * N;
  dense_from_stencil_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(Y, A, g.L0, g.L1, N, shift);
  MG_LAUNCHED();
}

// ---------------------------------------------------------------------------
// LU with partial pivoting (right-looking, one column per step)
// ---------------------------------------------------------------------------
constexpr int kPivThreads = 1024;

__global__ void __launch_bounds__(kPivThreads) lu_pivot_kernel(Cx<double> *A, int n, int k, int *ipiv, int *info) {
  __shared__ double sv[kPivThreads / 32];
  __shared__ int si[kPivThreads / 32];
  __shared__ int piv_row;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // argmax |A(i,k)|^2 over i >= k, ties to the smallest i
  double best = -1.0;
  int bi = n;
  for (int i = k + tid; i < n; i += blockDim.x) {
    const double v = norm2(A[(long long)k * n + i]);
    if (v > best) { best = v; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { sv[wid] = best; si[wid] = bi; }
  __syncthreads();
  if (wid == 0) {
    best = (lane < (int)(blockDim.x >> 5)) ? sv[lane] : -1.0;
    bi = (lane < (int)(blockDim.x >> 5)) ? si[lane] : n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      piv_row = bi;
      ipiv[k] = bi;
      if (!(best > 0.0) && *info == 0) *info = k + 1;
    }
  }
  __syncthreads();
  const int p = piv_row;
  if (p != k && p < n) {
    for (int j = tid; j < n; j += blockDim.x) {
      const Cx<double> t = A[(long long)j * n + k];
      A[(long long)j * n + k] = A[(long long)j * n + p];
      A[(long long)j * n + p] = t;
    }
  }
  __syncthreads();
  const Cx<double> pv = A[(long long)k * n + k];
  const double d = norm2(pv);
  if (d > 0.0) {
    const Cx<double> inv = mk(pv.re / d, -pv.im / d);
    for (int i = k + 1 + tid; i < n; i += blockDim.x) A[(long long)k * n + i] = A[(long long)k * n + i] * inv;
  }
}

// trailing update A(i, j) -= A(i, k) A(k, j), i, j > k
__global__ void lu_update_kernel(Cx<double> *A, int n, int k) {
  const int m = n - k - 1;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * m) return;
  const int jj = (int)(t / m), ii = (int)(t - (long long)jj * m);
  const int i = k + 1 + ii, j = k + 1 + jj;
  const Cx<double> l = A[(long long)k * n + i], u = A[(long long)j * n + k];
  Cx<double> a = A[(long long)j * n + i];
  cmac(a, mk(-l.re, -l.im), u);
  A[(long long)j * n + i] = a;
}

void lu_factor(Cx<double> *A, int n, int *ipiv, int *info_dev, cudaStream_t s) {
  MG_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
  for (int k = 0; k < n; ++k) {
    lu_pivot_kernel<<<1, kPivThreads, 0, s>>>(A, n, k, ipiv, info_dev);
    MG_LAUNCHED();
    const long long m = n - k - 1;
    if (m > 0) {
      lu_update_kernel<<<grid_for(m * m, 256), 256, 0, s>>>(A, n, k);
      MG_LAUNCHED();
    }
  }
}

// ---------------------------------------------------------------------------
// triangular solves, one tile of kTile columns per step: a single block solves
// the tile's triangle and writes it to `out`; a grid then removes the tile's
// columns from the remaining rows of `x` (one warp per row)
// ---------------------------------------------------------------------------
constexpr int kTile = 64;

__global__ void permute_kernel(const int *ipiv, int n, Cx<double> *x) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = ipiv[k];
      if (p != k && p < n) {
        const Cx<double> t = x[k];
        x[k] = x[p];
        x[p] = t;
      }
    }
  }
}

template <bool LOWER>
__global__ void tri_tile_kernel(const Cx<double> *__restrict__ LU, int n, int t0, int t1, const Cx<double> *x,
                                Cx<double> *out) {
  __shared__ Cx<double> xt[kTile];
  const int r = threadIdx.x, T = t1 - t0;
  if (r < T) xt[r] = x[t0 + r];
  __syncthreads();
  if (LOWER) {
    for (int c = 0; c < T; ++c) {
      if (r > c && r < T) cmac(xt[r], mk(-LU[(long long)(t0 + c) * n + t0 + r].re, -LU[(long long)(t0 + c) * n + t0 + r].im), xt[c]);
      __syncthreads();
    }
  } else {
    for (int c = T - 1; c >= 0; --c) {
      if (r == c) {
        const Cx<double> d = LU[(long long)(t0 + c) * n + t0 + c];
        const double dn = norm2(d);
        xt[c] = xt[c] * mk(d.re / dn, -d.im / dn);
      }
      __syncthreads();
      if (r < c) cmac(xt[r], mk(-LU[(long long)(t0 + c) * n + t0 + r].re, -LU[(long long)(t0 + c) * n + t0 + r].im), xt[c]);
      __syncthreads();
    }
  }
  if (r < T) out[t0 + r] = xt[r];
}

// rows [r0, r1) of x -= LU(rows, t0..t1) * sol(t0..t1)
__global__ void tri_update_kernel(const Cx<double> *__restrict__ LU, int n, int t0, int t1, const Cx<double> *sol,
                                  Cx<double> *x, int r0, int r1) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int i = r0 + warp;
  if (i >= r1) return;
  Cx<double> acc = mk(0.0, 0.0);
  for (int c = t0 + lane; c < t1; c += 32) cmac(acc, LU[(long long)c * n + i], sol[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  if (lane == 0) x[i] = x[i] - acc;
}

// x = A^{-1} b using the factors; `work` holds n entries (may not alias b or x)
void lu_solve_ws(const Cx<double> *LU, const int *ipiv, int n, const Cx<double> *b, Cx<double> *x, Cx<double> *work,
                 cudaStream_t s) {
  // work = P b
  if (work != b) launch_copy<double>(b, work, n, s);
  permute_kernel<<<1, 32, 0, s>>>(ipiv, n, work);
  MG_LAUNCHED();
  // forward: L y = P b; y goes to x, work holds the running right-hand side
  for (int t0 = 0; t0 < n; t0 += kTile) {
    const int t1 = t0 + kTile < n ? t0 + kTile : n;
    tri_tile_kernel<true><<<1, kTile, 0, s>>>(LU, n, t0, t1, work, x);
    MG_LAUNCHED();
    if (t1 < n) {
      tri_update_kernel<<<grid_for((long long)(n - t1) * 32, 256), 256, 0, s>>>(LU, n, t0, t1, x, work, t1, n);
      MG_LAUNCHED();
    }
  }
  // backward: U z = y; copy y into work as the running right-hand side, solution to x
  launch_copy<double>(x, work, n, s);
  for (int t1 = n; t1 > 0; t1 -= kTile) {
    const int t0 = t1 - kTile > 0 ? t1 - kTile : 0;
    tri_tile_kernel<false><<<1, kTile, 0, s>>>(LU, n, t0, t1, work, x);
    MG_LAUNCHED();
    if (t0 > 0) {
      tri_update_kernel<<<grid_for((long long)t0 * 32, 256), 256, 0, s>>>(LU, n, t0, t1, x, work, 0, t0);
      MG_LAUNCHED();
    }
  }
}

}  // namespace mg
