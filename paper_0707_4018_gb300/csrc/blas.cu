// Vector kernels of the smoother and the Krylov loops: fused updates and
// deterministic reductions (fixed element -> thread map, fixed warp/block
// trees, partials summed in block order by the last block). Products are
// accumulated in FP64 whatever the storage precision.
#include "kernels.h"

namespace mg {

template <typename R>
__global__ void zero_kernel(Cx<R> *x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = mk((R)0, (R)0);
}

template <typename R>
__global__ void copy_kernel(const Cx<R> *__restrict__ x, Cx<R> *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

template <typename To, typename From>
__global__ void convert_kernel(const Cx<From> *__restrict__ x, Cx<To> *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = cvt<To>(x[i]);
}

template <typename R>
__global__ void axpy_dev_kernel(const double *__restrict__ alpha, double sign, const Cx<R> *__restrict__ x,
                                Cx<R> *__restrict__ y, long long n) {
  const Cx<R> a = mk((R)(sign * alpha[0]), (R)(sign * alpha[1]));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cmac(y[i], a, x[i]);
}

template <typename R>
__global__ void xmy_kernel(const Cx<R> *__restrict__ x, Cx<R> *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] - y[i];
}

template <typename R>
__global__ void __launch_bounds__(kReduceThreads) dot_norm_kernel(const Cx<R> *__restrict__ a,
                                                                  const Cx<R> *__restrict__ b, long long n,
                                                                  double *partials, double *out,
                                                                  unsigned int *ticket) {
  __shared__ double sh[32 * 3];
  double v[3] = {0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<double> x = cvt<double>(a[i]), y = cvt<double>(b[i]);
    v[0] += x.re * y.re + x.im * y.im;
    v[1] += x.re * y.im - x.im * y.re;
    v[2] += x.re * x.re + x.im * x.im;
  }
  grid_finish<3>(v, partials, out, ticket, sh);
}

template <typename R>
__global__ void __launch_bounds__(kReduceThreads) norm2_kernel(const Cx<R> *__restrict__ a, long long n,
                                                               double *partials, double *out, unsigned int *ticket) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<double> x = cvt<double>(a[i]);
    v[0] += x.re * x.re + x.im * x.im;
  }
  grid_finish<1>(v, partials, out, ticket, sh);
}

// blockIdx.y = j: <W_j, w>; partials/ticket are per j
template <typename R>
__global__ void __launch_bounds__(kReduceThreads) multi_dot_kernel(const Cx<R> *__restrict__ W,
                                                                   const Cx<R> *__restrict__ w, long long n,
                                                                   double *partials, double *out,
                                                                   unsigned int *ticket, int pstride) {
  __shared__ double sh[32 * 2];
  const int j = blockIdx.y;
  const Cx<R> *Wj = W + (long long)j * n;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<double> x = cvt<double>(Wj[i]), y = cvt<double>(w[i]);
    v[0] += x.re * y.re + x.im * y.im;
    v[1] += x.re * y.im - x.im * y.re;
  }
  grid_finish<2>(v, partials + (long long)j * pstride, out + 2 * j, ticket + j, sh);
}

template <typename R>
__global__ void multi_axpy_kernel(const double *__restrict__ beta, int k, const Cx<R> *__restrict__ W,
                                  Cx<R> *__restrict__ w, const Cx<R> *__restrict__ Z, Cx<R> *__restrict__ z,
                                  long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<R> acc = w[i];
    Cx<R> accz = z ? z[i] : mk((R)0, (R)0);
    for (int j = 0; j < k; ++j) {
      const Cx<R> bj = mk((R)-beta[2 * j], (R)-beta[2 * j + 1]);
      cmac(acc, bj, W[(long long)j * n + i]);
      if (z) cmac(accz, bj, Z[(long long)j * n + i]);
    }
    w[i] = acc;
    if (z) z[i] = accz;
  }
}

template <typename R>
__global__ void normalize_kernel(const double *__restrict__ nrm2, Cx<R> *__restrict__ w, Cx<R> *__restrict__ z,
                                 long long n) {
  const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
  const R sr = (R)s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    w[i] = sr * w[i];
    if (z) z[i] = sr * z[i];
  }
}

template <typename R>
__global__ void mr_update_kernel(const double *__restrict__ sc, double omega, Cx<R> *__restrict__ x,
                                 Cx<R> *__restrict__ r, const Cx<R> *__restrict__ Ar, long long n) {
  // alpha = omega <Ar, r> / <Ar, Ar>  (zero when Ar vanishes)
  const double den = sc[2];
  const double ar = den > 0.0 ? omega * sc[0] / den : 0.0;
  const double ai = den > 0.0 ? omega * sc[1] / den : 0.0;
  const Cx<R> alpha = mk((R)ar, (R)ai), malpha = mk((R)-ar, (R)-ai);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> ri = r[i];
    cmac(x[i], alpha, ri);
    Cx<R> rn = ri;
    cmac(rn, malpha, Ar[i]);
    r[i] = rn;
  }
}

template <typename R>
__global__ void __launch_bounds__(kReduceThreads) gcr_update_kernel(const double *__restrict__ sc, Cx<R> *__restrict__ x,
                                                                    const Cx<R> *__restrict__ z, Cx<R> *__restrict__ r,
                                                                    const Cx<R> *__restrict__ w, long long n,
                                                                    double *partials, double *out,
                                                                    unsigned int *ticket) {
  __shared__ double sh[32];
  const Cx<R> alpha = mk((R)sc[0], (R)sc[1]), malpha = mk((R)-sc[0], (R)-sc[1]);
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cmac(x[i], alpha, z[i]);
    Cx<R> rn = r[i];
    cmac(rn, malpha, w[i]);
    r[i] = rn;
    const Cx<double> rd = cvt<double>(rn);
    v[0] += rd.re * rd.re + rd.im * rd.im;
  }
  grid_finish<1>(v, partials, out, ticket, sh);
}

// ---------------------------------------------------------------------------
static unsigned int stream_grid(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned int)b;
}

template <typename R>
void launch_zero(Cx<R> *x, long long n, cudaStream_t s) {
  zero_kernel<R><<<stream_grid(n), 256, 0, s>>>(x, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_copy(const Cx<R> *x, Cx<R> *y, long long n, cudaStream_t s) {
  copy_kernel<R><<<stream_grid(n), 256, 0, s>>>(x, y, n);
  MG_LAUNCHED();
}
template <typename To, typename From>
void launch_convert(const Cx<From> *x, Cx<To> *y, long long n, cudaStream_t s) {
  convert_kernel<To, From><<<stream_grid(n), 256, 0, s>>>(x, y, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_axpy_dev(const double *alpha_dev, double sign, const Cx<R> *x, Cx<R> *y, long long n, cudaStream_t s) {
  axpy_dev_kernel<R><<<stream_grid(n), 256, 0, s>>>(alpha_dev, sign, x, y, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_xmy(const Cx<R> *x, Cx<R> *y, long long n, cudaStream_t s) {
  xmy_kernel<R><<<stream_grid(n), 256, 0, s>>>(x, y, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_dot_norm(const Cx<R> *a, const Cx<R> *b, long long n, double *out, const ReduceWs &ws, cudaStream_t s) {
  dot_norm_kernel<R><<<reduce_blocks(n, ws.max_blocks), kReduceThreads, 0, s>>>(a, b, n, ws.partials, out, ws.ticket);
  MG_LAUNCHED();
}
template <typename R>
void launch_norm2(const Cx<R> *a, long long n, double *out, const ReduceWs &ws, cudaStream_t s) {
  norm2_kernel<R><<<reduce_blocks(n, ws.max_blocks), kReduceThreads, 0, s>>>(a, n, ws.partials, out, ws.ticket);
  MG_LAUNCHED();
}
template <typename R>
void launch_multi_dot(const Cx<R> *W, int k, const Cx<R> *w, long long n, double *out, const ReduceWs &ws,
                      cudaStream_t s) {
  if (k <= 0) return;
  // the workspace holds max_blocks * 4 partials and 128 tickets: split the blocks across the k rows
  int per = ws.max_blocks * 4 / (2 * k);
  if (per < 1) per = 1;
  if (k > 128) fail(MG_ERR_UNSUPPORTED, "multi_dot: more than 128 vectors");
  dim3 grid(reduce_blocks(n, per), k);
  multi_dot_kernel<R><<<grid, kReduceThreads, 0, s>>>(W, w, n, ws.partials, out, ws.ticket, 2 * (int)grid.x);
  MG_LAUNCHED();
}
template <typename R>
void launch_multi_axpy(const double *beta, int k, const Cx<R> *W, Cx<R> *w, const Cx<R> *Z, Cx<R> *z, long long n,
                       cudaStream_t s) {
  if (k <= 0) return;
  multi_axpy_kernel<R><<<stream_grid(n), 256, 0, s>>>(beta, k, W, w, Z, z, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_normalize(const double *nrm2_dev, Cx<R> *w, Cx<R> *z, long long n, cudaStream_t s) {
  normalize_kernel<R><<<stream_grid(n), 256, 0, s>>>(nrm2_dev, w, z, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_mr_update(const double *sc, double omega, Cx<R> *x, Cx<R> *r, const Cx<R> *Ar, long long n,
                      cudaStream_t s) {
  mr_update_kernel<R><<<stream_grid(n), 256, 0, s>>>(sc, omega, x, r, Ar, n);
  MG_LAUNCHED();
}
template <typename R>
void launch_gcr_update(const double *sc, Cx<R> *x, const Cx<R> *z, Cx<R> *r, const Cx<R> *w, long long n,
                       double *out_nrm, const ReduceWs &ws, cudaStream_t s) {
  gcr_update_kernel<R><<<reduce_blocks(n, ws.max_blocks), kReduceThreads, 0, s>>>(sc, x, z, r, w, n, ws.partials,
                                                                                  out_nrm, ws.ticket);
  MG_LAUNCHED();
}

#define MG_INST_BLAS(R)                                                                                          \
  template void launch_zero<R>(Cx<R> *, long long, cudaStream_t);                                                \
  template void launch_copy<R>(const Cx<R> *, Cx<R> *, long long, cudaStream_t);                                 \
  template void launch_axpy_dev<R>(const double *, double, const Cx<R> *, Cx<R> *, long long, cudaStream_t);     \
  template void launch_xmy<R>(const Cx<R> *, Cx<R> *, long long, cudaStream_t);                                  \
  template void launch_dot_norm<R>(const Cx<R> *, const Cx<R> *, long long, double *, const ReduceWs &, cudaStream_t); \
  template void launch_norm2<R>(const Cx<R> *, long long, double *, const ReduceWs &, cudaStream_t);             \
  template void launch_multi_dot<R>(const Cx<R> *, int, const Cx<R> *, long long, double *, const ReduceWs &,    \
                                    cudaStream_t);                                                               \
  template void launch_multi_axpy<R>(const double *, int, const Cx<R> *, Cx<R> *, const Cx<R> *, Cx<R> *,        \
                                     long long, cudaStream_t);                                                   \
  template void launch_normalize<R>(const double *, Cx<R> *, Cx<R> *, long long, cudaStream_t);                  \
  template void launch_mr_update<R>(const double *, double, Cx<R> *, Cx<R> *, const Cx<R> *, long long,          \
                                    cudaStream_t);                                                               \
  template void launch_gcr_update<R>(const double *, Cx<R> *, const Cx<R> *, Cx<R> *, const Cx<R> *, long long,  \
                                     double *, const ReduceWs &, cudaStream_t);

MG_INST_BLAS(double)
MG_INST_BLAS(float)
template void launch_convert<float, double>(const Cx<double> *, Cx<float> *, long long, cudaStream_t);
template void launch_convert<double, float>(const Cx<float> *, Cx<double> *, long long, cudaStream_t);

}  // namespace mg
