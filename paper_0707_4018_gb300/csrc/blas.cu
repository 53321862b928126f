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

template <typename R>
__global__ void mr_update_kernel(const double *__restrict__ sc, double omega, Cx<R> *__restrict__ x,
                                 Cx<R> *__restrict__ r, const Cx<R> *__restrict__ Ar, long long n) {
  // alpha = omega <Ar, r> / <Ar, Ar>  (zero when Ar vanishes), once per block
  __shared__ double s_a[2];
  if (threadIdx.x == 0) {
    const double den = sc[2];
    s_a[0] = den > 0.0 ? omega * sc[0] / den : 0.0;
    s_a[1] = den > 0.0 ? omega * sc[1] / den : 0.0;
  }
  __syncthreads();
  const Cx<R> alpha = mk((R)s_a[0], (R)s_a[1]), malpha = mk((R)-s_a[0], (R)-s_a[1]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> ri = r[i];
    cmac(x[i], alpha, ri);
    Cx<R> rn = ri;
    cmac(rn, malpha, Ar[i]);
    r[i] = rn;
  }
}

// rows j < k: <W_j, w>; row k: <w, w>; row k + 1: <w, r>; row k + 2: <r, r>  (blockIdx.y = row)
// (VT = float: FP32 vectors; each thread sums its few products in FP32, the block and grid
// trees sum in FP64)
// (kdev: k read from device memory, for loops replayed by a graph; the grid then has rows
// for the longest basis, and the rows above k + 2 return at once, all blocks of a row alike)
template <typename VT>
__global__ void __launch_bounds__(kReduceThreads) gcr_dots_kernel(const Cx<VT> *__restrict__ W,
                                                                  const Cx<VT> *__restrict__ w,
                                                                  const Cx<VT> *__restrict__ r, int k_host,
                                                                  const int *__restrict__ kdev, long long n,
                                                                  double *partials, double *out,
                                                                  unsigned int *ticket, int pstride) {
  __shared__ double sh[32 * 2];
  const int row = blockIdx.y, k = kdev != nullptr ? *kdev : k_host;
  if (row > k + 2) return;
  const Cx<VT> *a = row < k ? W + (long long)row * n : (row == k + 2 ? r : w);
  const Cx<VT> *b = row > k ? r : w;
  VT t0 = (VT)0, t1 = (VT)0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<VT> x = a[i], y = b[i];
    t0 += x.re * y.re + x.im * y.im;
    t1 += x.re * y.im - x.im * y.re;
  }
  double v[2] = {(double)t0, (double)t1};
  grid_finish<2>(v, partials + (long long)row * pstride, out + 2 * row, ticket + row, sh);
}

// w <- (w - sum_j beta_j W_j) * inv, z likewise; W_k = w, Z_k = z; x += alpha z; r -= alpha w
__global__ void gcr_project_update_kernel(const Cx<double> *__restrict__ W, Cx<double> *__restrict__ Wk,
                                          const Cx<double> *__restrict__ Z, Cx<double> *__restrict__ Zk, int k,
                                          const double *__restrict__ beta, double inv, double are, double aim,
                                          Cx<double> *__restrict__ x, Cx<double> *__restrict__ r, long long n,
                                          int update_xr) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<double> w = Wk[i], z = Zk[i];
    for (int j = 0; j < k; ++j) {
      const Cx<double> bj = mk(-beta[2 * j], -beta[2 * j + 1]);
      cmac(w, bj, W[(long long)j * n + i]);
      cmac(z, bj, Z[(long long)j * n + i]);
    }
    w = inv * w;
    z = inv * z;
    Wk[i] = w;
    Zk[i] = z;
    if (update_xr) {
      cmac(x[i], mk(are, aim), z);
      Cx<double> ri = r[i];
      cmac(ri, mk(-are, -aim), w);
      r[i] = ri;
    }
  }
}

template <typename VT>
static void gcr_dots_any(const Cx<VT> *W, const Cx<VT> *w, const Cx<VT> *r, int k, long long n, double *out,
                         const ReduceWs &ws, cudaStream_t s) {
  const int rows = k + 3;
  if (rows > 128) fail(MG_ERR_UNSUPPORTED, "gcr_dots: too many basis vectors");
  int per = (int)(ws.capacity / (2 * rows));
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) per = 1;
  dim3 grid(reduce_blocks(n, per), rows);
  gcr_dots_kernel<VT><<<grid, kReduceThreads, 0, s>>>(W, w, r, k, nullptr, n, ws.partials, out, ws.ticket,
                                                      2 * (int)grid.x);
  MG_LAUNCHED();
}

// the same reduction with k = *kdev (grid rows for k up to kmax)
template <typename VT>
void launch_gcr_dots_kdev(const Cx<VT> *W, const Cx<VT> *w, const Cx<VT> *r, const int *kdev, int kmax, long long n,
                          double *out, const ReduceWs &ws, cudaStream_t s) {
  const int rows = kmax + 3;
  if (rows > 128) fail(MG_ERR_UNSUPPORTED, "gcr_dots: too many basis vectors");
  int per = (int)(ws.capacity / (2 * rows));
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) per = 1;
  dim3 grid(reduce_blocks(n, per), rows);
  gcr_dots_kernel<VT><<<grid, kReduceThreads, 0, s>>>(W, w, r, 0, kdev, n, ws.partials, out, ws.ticket,
                                                      2 * (int)grid.x);
  MG_LAUNCHED();
}
template void launch_gcr_dots_kdev<float>(const Cx<float> *, const Cx<float> *, const Cx<float> *, const int *, int,
                                          long long, double *, const ReduceWs &, cudaStream_t);

void launch_gcr_dots(const Cx<double> *W, const Cx<double> *w, const Cx<double> *r, int k, long long n, double *out,
                     const ReduceWs &ws, cudaStream_t s) {
  gcr_dots_any<double>(W, w, r, k, n, out, ws, s);
}

void launch_gcr_dots(const Cx<float> *W, const Cx<float> *w, const Cx<float> *r, int k, long long n, double *out,
                     const ReduceWs &ws, cudaStream_t s) {
  gcr_dots_any<float>(W, w, r, k, n, out, ws, s);
}

void launch_gcr_project_update(const Cx<double> *W, Cx<double> *Wk, const Cx<double> *Z, Cx<double> *Zk, int k,
                               const double *beta_dev, double inv, double are, double aim, Cx<double> *x,
                               Cx<double> *r, long long n, bool update_xr, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  gcr_project_update_kernel<<<(unsigned int)(b < 1 ? 1 : b), 256, 0, s>>>(W, Wk, Z, Zk, k, beta_dev, inv, are, aim, x,
                                                                          r, n, update_xr ? 1 : 0);
  MG_LAUNCHED();
}


// ---------------------------------------------------------------------------
// batched outer GCR (FP64): nb systems in lockstep, vector v of a batch at v * n;
// Krylov bases W[j][v][n], Z[j][v][n]
// ---------------------------------------------------------------------------

// y_v = x_v for the vectors with mask bit v, else 0
template <typename VT>
__global__ void copy_masked_kernel(const Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ y, long long n,
                                   unsigned int mask) {
  const long long off = blockIdx.y * n;
  const bool on = (mask >> blockIdx.y) & 1u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[off + i] = on ? x[off + i] : mk((VT)0, (VT)0);
}

// out[v] = |a_v|^2 (blockIdx.y = v)
template <typename VT>
__global__ void __launch_bounds__(kReduceThreads) norm2_batch_kernel(const Cx<VT> *__restrict__ a, long long n,
                                                                     double *partials, double *out,
                                                                     unsigned int *ticket) {
  __shared__ double sh[32];
  const Cx<VT> *av = a + blockIdx.y * n;
  VT t = (VT)0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    t += norm2(av[i]);
  double v[1] = {(double)t};
  grid_finish<1>(v, partials + (long long)blockIdx.y * gridDim.x, out + blockIdx.y, ticket + blockIdx.y, sh);
}

// vector v = blockIdx.z, row = blockIdx.y: rows j < k <W_j, w>, row k |w|^2, row k + 1 <w, r>,
// row k + 2 |r|^2; results at out[v * 2 (k + 3) + 2 row]
// (VT = float: FP32 vectors, each thread's products summed in FP32, the trees in FP64)
template <typename VT>
__global__ void __launch_bounds__(kReduceThreads) gcr_dots_batch_kernel(const Cx<VT> *__restrict__ W,
                                                                        const Cx<VT> *__restrict__ r, int k,
                                                                        int nb, long long n, double *partials,
                                                                        double *out, unsigned int *ticket) {
  __shared__ double sh[32 * 2];
  const int row = blockIdx.y, v = blockIdx.z, rows = k + 3;
  const Cx<VT> *w = W + ((long long)k * nb + v) * n;
  const Cx<VT> *rv = r + (long long)v * n;
  const Cx<VT> *a = row < k ? W + ((long long)row * nb + v) * n : (row == k + 2 ? rv : w);
  const Cx<VT> *b = row > k ? rv : w;
  VT t0 = (VT)0, t1 = (VT)0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<VT> x = a[i], y = b[i];
    t0 += x.re * y.re + x.im * y.im;
    t1 += x.re * y.im - x.im * y.re;
  }
  double acc[2] = {(double)t0, (double)t1};
  const long long slot = (long long)v * rows + row;
  grid_finish<2>(acc, partials + slot * 2 * gridDim.x, out + 2 * slot, ticket + slot, sh);
}

// per vector v (blockIdx.y), coef[4 v .. 4 v + 3] = (inv, alpha re, alpha im, mode):
// mode 0 leaves the vector alone; mode 2 projects w_k, z_k against the basis with beta_j =
// dots[v * 2 (k + 3) + 2 j]; mode 1 projects, scales both by inv and updates x += alpha z_k,
// r -= alpha w_k
template <typename VT>
__global__ void gcr_update_batch_kernel(Cx<VT> *__restrict__ W, Cx<VT> *__restrict__ Z, int k, int nb,
                                        const double *__restrict__ dots, const double *__restrict__ coef,
                                        Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ r, long long n) {
  const int v = blockIdx.y;
  const int mode = (int)coef[4 * v + 3];
  if (mode == 0) return;
  const double *beta = dots + (long long)v * 2 * (k + 3);
  const VT inv = (VT)(mode == 1 ? coef[4 * v] : 1.0);
  const Cx<VT> alpha = mk((VT)coef[4 * v + 1], (VT)coef[4 * v + 2]);
  Cx<VT> *Wk = W + ((long long)k * nb + v) * n, *Zk = Z + ((long long)k * nb + v) * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<VT> w = Wk[i], z = Zk[i];
    for (int j = 0; j < k; ++j) {
      const Cx<VT> bj = mk((VT)-beta[2 * j], (VT)-beta[2 * j + 1]);
      const long long o = ((long long)j * nb + v) * n + i;
      cmac(w, bj, W[o]);
      cmac(z, bj, Z[o]);
    }
    w = inv * w;
    z = inv * z;
    Wk[i] = w;
    Zk[i] = z;
    if (mode == 1) {
      cmac(x[(long long)v * n + i], alpha, z);
      Cx<VT> ri = r[(long long)v * n + i];
      cmac(ri, mk(-alpha.re, -alpha.im), w);
      r[(long long)v * n + i] = ri;
    }
  }
}

// the same step with kLanes consecutive lanes per element, each summing the basis vectors
// j = lane, lane + kLanes, ... (short coarse vectors: one thread per element left most SMs idle
// while each thread walked the whole basis); the loop is steered by the warp's first element
// so that every lane takes part in every shuffle
constexpr int kLanes = 4;

template <typename VT>
__global__ void gcr_update_batch_split_kernel(Cx<VT> *__restrict__ W, Cx<VT> *__restrict__ Z, int k, int nb,
                                              const double *__restrict__ dots, const double *__restrict__ coef,
                                              Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ r, long long n) {
  const int v = blockIdx.y;
  const int mode = (int)coef[4 * v + 3];
  if (mode == 0) return;
  const double *beta = dots + (long long)v * 2 * (k + 3);
  const VT inv = (VT)(mode == 1 ? coef[4 * v] : 1.0);
  const Cx<VT> alpha = mk((VT)coef[4 * v + 1], (VT)coef[4 * v + 2]);
  Cx<VT> *Wk = W + ((long long)k * nb + v) * n, *Zk = Z + ((long long)k * nb + v) * n;
  const int sub = threadIdx.x % kLanes, lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * (blockDim.x / kLanes);
  long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / kLanes;
  for (long long i0 = i - lane / kLanes; i0 < n; i0 += stride, i += stride) {
    const bool valid = i < n;
    Cx<VT> pw = mk((VT)0, (VT)0), pz = mk((VT)0, (VT)0);
    for (int j = sub; valid && j < k; j += kLanes) {
      const Cx<VT> bj = mk((VT)-beta[2 * j], (VT)-beta[2 * j + 1]);
      const long long o = ((long long)j * nb + v) * n + i;
      cmac(pw, bj, W[o]);
      cmac(pz, bj, Z[o]);
    }
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) {
      pw.re += __shfl_xor_sync(0xffffffffu, pw.re, o);
      pw.im += __shfl_xor_sync(0xffffffffu, pw.im, o);
      pz.re += __shfl_xor_sync(0xffffffffu, pz.re, o);
      pz.im += __shfl_xor_sync(0xffffffffu, pz.im, o);
    }
    if (valid && sub == 0) {
      const Cx<VT> w = inv * (Wk[i] + pw), z = inv * (Zk[i] + pz);
      Wk[i] = w;
      Zk[i] = z;
      if (mode == 1) {
        cmac(x[(long long)v * n + i], alpha, z);
        Cx<VT> ri = r[(long long)v * n + i];
        cmac(ri, mk(-alpha.re, -alpha.im), w);
        r[(long long)v * n + i] = ri;
      }
    }
  }
}

static unsigned int stream_grid(long long n);

template <typename VT>
void launch_copy_masked(const Cx<VT> *x, Cx<VT> *y, long long n, int nb, unsigned int mask, cudaStream_t s) {
  copy_masked_kernel<VT><<<dim3(stream_grid(n), nb), 256, 0, s>>>(x, y, n, mask);
  MG_LAUNCHED();
}

template <typename VT>
void launch_norm2_batch(const Cx<VT> *a, long long n, int nb, double *out, const ReduceWs &ws, cudaStream_t s) {
  int per = (int)(ws.capacity / nb);
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) per = 1;
  norm2_batch_kernel<VT><<<dim3(reduce_blocks(n, per), nb), kReduceThreads, 0, s>>>(a, n, ws.partials, out,
                                                                                    ws.ticket);
  MG_LAUNCHED();
}

template <typename VT>
void launch_gcr_dots_batch(const Cx<VT> *W, const Cx<VT> *r, int k, int nb, long long n, double *out,
                           const ReduceWs &ws, cudaStream_t s) {
  const int rows = k + 3;
  if ((long long)rows * nb > ws.tickets) fail(MG_ERR_UNSUPPORTED, "gcr_dots_batch: too many reductions");
  int per = (int)(ws.capacity / (2LL * rows * nb));
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) fail(MG_ERR_STATE, "gcr_dots_batch: reduction workspace too small");
  gcr_dots_batch_kernel<VT><<<dim3(reduce_blocks(n, per), rows, nb), kReduceThreads, 0, s>>>(W, r, k, nb, n,
                                                                                             ws.partials, out,
                                                                                             ws.ticket);
  MG_LAUNCHED();
}

template <typename VT>
void launch_gcr_update_batch(Cx<VT> *W, Cx<VT> *Z, int k, int nb, const double *dots, const double *coef, Cx<VT> *x,
                             Cx<VT> *r, long long n, cudaStream_t s) {
  if (n < (1LL << 18)) {  // short (coarse) vectors: kLanes lanes per element
    gcr_update_batch_split_kernel<VT><<<dim3(stream_grid(n * kLanes), nb), 256, 0, s>>>(W, Z, k, nb, dots, coef, x,
                                                                                        r, n);
    MG_LAUNCHED();
    return;
  }
  gcr_update_batch_kernel<VT><<<dim3(stream_grid(n), nb), 256, 0, s>>>(W, Z, k, nb, dots, coef, x, r, n);
  MG_LAUNCHED();
}

#define MG_INST_BATCH(VT)                                                                                          \
  template void launch_copy_masked<VT>(const Cx<VT> *, Cx<VT> *, long long, int, unsigned int, cudaStream_t);     \
  template void launch_norm2_batch<VT>(const Cx<VT> *, long long, int, double *, const ReduceWs &, cudaStream_t); \
  template void launch_gcr_dots_batch<VT>(const Cx<VT> *, const Cx<VT> *, int, int, long long, double *,          \
                                          const ReduceWs &, cudaStream_t);                                         \
  template void launch_gcr_update_batch<VT>(Cx<VT> *, Cx<VT> *, int, int, const double *, const double *,          \
                                            Cx<VT> *, Cx<VT> *, long long, cudaStream_t);
MG_INST_BATCH(double)
MG_INST_BATCH(float)
#undef MG_INST_BATCH

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
void launch_mr_update(const double *sc, double omega, Cx<R> *x, Cx<R> *r, const Cx<R> *Ar, long long n,
                      cudaStream_t s) {
  mr_update_kernel<R><<<stream_grid(n), 256, 0, s>>>(sc, omega, x, r, Ar, n);
  MG_LAUNCHED();
}
#define MG_INST_BLAS(R)                                                                                          \
  template void launch_zero<R>(Cx<R> *, long long, cudaStream_t);                                                \
  template void launch_copy<R>(const Cx<R> *, Cx<R> *, long long, cudaStream_t);                                 \
  template void launch_xmy<R>(const Cx<R> *, Cx<R> *, long long, cudaStream_t);                                  \
  template void launch_dot_norm<R>(const Cx<R> *, const Cx<R> *, long long, double *, const ReduceWs &, cudaStream_t); \
  template void launch_norm2<R>(const Cx<R> *, long long, double *, const ReduceWs &, cudaStream_t);             \
  template void launch_mr_update<R>(const double *, double, Cx<R> *, Cx<R> *, const Cx<R> *, long long,          \
                                    cudaStream_t);                                                               \


MG_INST_BLAS(double)
MG_INST_BLAS(float)
template void launch_convert<float, double>(const Cx<double> *, Cx<float> *, long long, cudaStream_t);
template void launch_convert<double, float>(const Cx<float> *, Cx<double> *, long long, cudaStream_t);

}  // namespace mg

// ---------------------------------------------------------------------------
// Outer flexible GCR with the loop on the device (a conditional WHILE node of a CUDA graph
// replays one iteration until the control kernel clears the condition). The basis index k
// and the counters live in device memory: ctl[0] iterations, ctl[1] k, ctl[2] stop reason
// (1 converged by the estimate, 2 iteration limit, 3 breakdown); st[0] the running |r|^2
// estimate, st[1] tol^2 |b|^2. Gram-Schmidt is classical with one pass.
// ---------------------------------------------------------------------------
namespace mg {

// rows j < k: <W_j, w>; row k: |w|^2; row k + 1: <w, r>; row k + 2: |r|^2, with k = ctl[1];
// the grid has restart + 3 rows, the rows above k + 2 only finish their (empty) reduction
__global__ void __launch_bounds__(kReduceThreads) gcr_dots_devk_kernel(const Cx<double> *__restrict__ W,
                                                                       const Cx<double> *__restrict__ w,
                                                                       const Cx<double> *__restrict__ r,
                                                                       const int *__restrict__ ctl, long long n,
                                                                       double *partials, double *out,
                                                                       unsigned int *ticket, int pstride) {
  __shared__ double sh[32 * 2];
  const int row = blockIdx.y, k = ctl[1];
  double v[2] = {0.0, 0.0};
  if (row <= k + 2) {
    const Cx<double> *a = row < k ? W + (long long)row * n : (row == k + 2 ? r : w);
    const Cx<double> *b = row > k ? r : w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const Cx<double> x = a[i], y = b[i];
      v[0] += x.re * y.re + x.im * y.im;
      v[1] += x.re * y.im - x.im * y.re;
    }
  }
  grid_finish<2>(v, partials + (long long)row * pstride, out + 2 * row, ticket + row, sh);
}

// W_k = (w - sum_j beta_j W_j) / |.|, Z_k likewise from z; x += alpha Z_k; r -= alpha W_k;
// st[2] = |r|^2 - |alpha|^2 (the new residual estimate), st[3] = 1 on breakdown
__global__ void gcr_update_devk_kernel(Cx<double> *__restrict__ W, Cx<double> *__restrict__ Z,
                                       const Cx<double> *__restrict__ w, const Cx<double> *__restrict__ z,
                                       const int *__restrict__ ctl, const double *__restrict__ dots,
                                       double *__restrict__ st, Cx<double> *__restrict__ x,
                                       Cx<double> *__restrict__ r, long long n) {
  __shared__ double coef[3];
  const int k = ctl[1];
  if (threadIdx.x == 0) {
    const double nw0 = dots[2 * k];
    double nw2 = nw0;
    for (int j = 0; j < k; ++j) nw2 -= dots[2 * j] * dots[2 * j] + dots[2 * j + 1] * dots[2 * j + 1];
    double inv = 0.0, are = 0.0, aim = 0.0;
    const bool ok = nw2 > 1e-28 * nw0;
    if (ok) {
      inv = 1.0 / sqrt(nw2);
      are = dots[2 * k + 2] * inv;
      aim = dots[2 * k + 3] * inv;
    }
    coef[0] = inv;
    coef[1] = are;
    coef[2] = aim;
    if (blockIdx.x == 0) {
      st[2] = fmax(dots[2 * k + 4] - (are * are + aim * aim), 0.0);
      st[3] = ok ? 0.0 : 1.0;
    }
  }
  __syncthreads();
  const double inv = coef[0];
  const Cx<double> alpha = mk(coef[1], coef[2]), malpha = mk(-coef[1], -coef[2]);
  Cx<double> *Wk = W + (long long)k * n, *Zk = Z + (long long)k * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<double> wi = w[i], zi = z[i];
    for (int j = 0; j < k; ++j) {
      const Cx<double> bj = mk(-dots[2 * j], -dots[2 * j + 1]);
      cmac(wi, bj, W[(long long)j * n + i]);
      cmac(zi, bj, Z[(long long)j * n + i]);
    }
    wi = inv * wi;
    zi = inv * zi;
    Wk[i] = wi;
    Zk[i] = zi;
    cmac(x[i], alpha, zi);
    Cx<double> ri = r[i];
    cmac(ri, malpha, wi);
    r[i] = ri;
  }
}

// one thread: counts the iteration, advances k (a restart starts a new basis from the
// recurrence residual), decides whether the loop goes on, and sets the WHILE condition
__global__ void gcr_control_kernel(int *ctl, double *st, int restart, int max_iter,
                                   cudaGraphConditionalHandle handle) {
  const int it = ctl[0] + 1;
  int k = ctl[1] + 1;
  if (k == restart) k = 0;
  ctl[0] = it;
  ctl[1] = k;
  st[0] = st[2];
  int reason = 0;
  if (!(st[0] > st[1])) reason = 1;
  else if (it >= max_iter) reason = 2;
  else if (st[3] != 0.0) reason = 3;
  ctl[2] = reason;
  cudaGraphSetConditional(handle, reason == 0 ? 1u : 0u);
}

void launch_gcr_dots_devk(const Cx<double> *W, const Cx<double> *w, const Cx<double> *r, const int *ctl, int restart,
                          long long n, double *out, const ReduceWs &ws, cudaStream_t s) {
  const int rows = restart + 3;
  int per = (int)(ws.capacity / (2 * rows));
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) per = 1;
  dim3 grid(reduce_blocks(n, per), rows);
  gcr_dots_devk_kernel<<<grid, kReduceThreads, 0, s>>>(W, w, r, ctl, n, ws.partials, out, ws.ticket, 2 * (int)grid.x);
  MG_LAUNCHED();
}

void launch_gcr_update_devk(Cx<double> *W, Cx<double> *Z, const Cx<double> *w, const Cx<double> *z, const int *ctl,
                            const double *dots, double *st, Cx<double> *x, Cx<double> *r, long long n,
                            cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  gcr_update_devk_kernel<<<(unsigned int)(b < 1 ? 1 : b), 256, 0, s>>>(W, Z, w, z, ctl, dots, st, x, r, n);
  MG_LAUNCHED();
}

void launch_gcr_control(int *ctl, double *st, int restart, int max_iter, cudaGraphConditionalHandle handle,
                        cudaStream_t s) {
  gcr_control_kernel<<<1, 1, 0, s>>>(ctl, st, restart, max_iter, handle);
  MG_LAUNCHED();
}

}  // namespace mg

// ---------------------------------------------------------------------------
// Device-driven outer GCR over a batch of nb vectors in lockstep (one WHILE loop per context):
// act[v] says whether vector v still iterates (it stops on its residual estimate or on a
// breakdown); stv[2 v] its |r|^2 estimate, stv[2 v + 1] its tol^2 |b_v|^2; coef[4 v ..] the
// update coefficients (inv, alpha re, alpha im, mode: 1 update, 0 leave alone). Dots are laid out
// per vector with stride 2 (restart + 3), as the host-driven batched loop's.
// ---------------------------------------------------------------------------
namespace mg {

// (VT: the vectors' type; FP32 vectors keep each thread's products in FP32, the trees in FP64)
template <typename VT>
__global__ void copy_active_kernel(const Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ y, long long n,
                                   const int *__restrict__ act) {
  const long long off = blockIdx.y * n;
  const bool on = act[blockIdx.y] != 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[off + i] = on ? x[off + i] : mk((VT)0, (VT)0);
}

// vector v = blockIdx.z, row = blockIdx.y < restart + 3, k = ctl[1]; the rows above k + 2
// return at once (all blocks of such a row alike, so their tickets stay untouched)
template <typename VT>
__global__ void __launch_bounds__(kReduceThreads) gcr_dots_batch_devk_kernel(
    const Cx<VT> *__restrict__ W, const Cx<VT> *__restrict__ w, const Cx<VT> *__restrict__ r,
    const int *__restrict__ ctl, int nb, int restart, long long n, double *partials, double *out,
    unsigned int *ticket) {
  __shared__ double sh[32 * 2];
  const int row = blockIdx.y, v = blockIdx.z, rows = restart + 3, k = ctl[1];
  if (row > k + 2) return;
  const Cx<VT> *wv = w + (long long)v * n;
  const Cx<VT> *rv = r + (long long)v * n;
  const Cx<VT> *a = row < k ? W + ((long long)row * nb + v) * n : (row == k + 2 ? rv : wv);
  const Cx<VT> *b = row > k ? rv : wv;
  VT t0 = (VT)0, t1 = (VT)0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<VT> x = a[i], y = b[i];
    t0 += x.re * y.re + x.im * y.im;
    t1 += x.re * y.im - x.im * y.re;
  }
  double acc[2] = {(double)t0, (double)t1};
  const long long slot = (long long)v * rows + row;
  grid_finish<2>(acc, partials + slot * 2 * gridDim.x, out + 2 * slot, ticket + slot, sh);
}

// one thread per vector: classical Gram-Schmidt coefficients, breakdown and convergence
__global__ void gcr_coef_batch_kernel(const double *__restrict__ dots, const int *__restrict__ ctl, int nb,
                                      int restart, int *__restrict__ act, double *__restrict__ stv,
                                      double *__restrict__ coef) {
  const int v = threadIdx.x;
  if (v >= nb) return;
  const int k = ctl[1];
  const double *d = dots + (long long)v * 2 * (restart + 3);
  double inv = 0.0, are = 0.0, aim = 0.0, mode = 0.0;
  if (act[v]) {
    const double nw0 = d[2 * k];
    double nw2 = nw0;
    for (int j = 0; j < k; ++j) nw2 -= d[2 * j] * d[2 * j] + d[2 * j + 1] * d[2 * j + 1];
    if (nw2 > 1e-28 * nw0) {
      inv = 1.0 / sqrt(nw2);
      are = d[2 * k + 2] * inv;
      aim = d[2 * k + 3] * inv;
      mode = 1.0;
      const double rn2 = fmax(d[2 * k + 4] - (are * are + aim * aim), 0.0);
      stv[2 * v] = rn2;
      if (rn2 <= stv[2 * v + 1]) act[v] = 0;
    } else {
      act[v] = 0;  // breakdown: this vector waits for the true residual after the launch
    }
  }
  coef[4 * v] = inv;
  coef[4 * v + 1] = are;
  coef[4 * v + 2] = aim;
  coef[4 * v + 3] = mode;
}

// W_{k,v} = (w_v - sum_j beta_j W_{j,v}) inv, Z likewise from z_v; x_v += alpha Z_{k,v}; r_v -= alpha W_{k,v}
template <typename VT>
__global__ void gcr_update_batch_devk_kernel(Cx<VT> *__restrict__ W, Cx<VT> *__restrict__ Z,
                                             const Cx<VT> *__restrict__ w, const Cx<VT> *__restrict__ z,
                                             const int *__restrict__ ctl, int nb, int restart,
                                             const double *__restrict__ dots, const double *__restrict__ coef,
                                             Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ r, long long n) {
  const int v = blockIdx.y, k = ctl[1];
  if (coef[4 * v + 3] == 0.0) return;
  const double *beta = dots + (long long)v * 2 * (restart + 3);
  const VT inv = (VT)coef[4 * v];
  const Cx<VT> alpha = mk((VT)coef[4 * v + 1], (VT)coef[4 * v + 2]);
  Cx<VT> *Wk = W + ((long long)k * nb + v) * n, *Zk = Z + ((long long)k * nb + v) * n;
  const Cx<VT> *wv = w + (long long)v * n, *zv = z + (long long)v * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<VT> wi = wv[i], zi = zv[i];
    for (int j = 0; j < k; ++j) {
      const Cx<VT> bj = mk((VT)-beta[2 * j], (VT)-beta[2 * j + 1]);
      const long long o = ((long long)j * nb + v) * n + i;
      cmac(wi, bj, W[o]);
      cmac(zi, bj, Z[o]);
    }
    wi = inv * wi;
    zi = inv * zi;
    Wk[i] = wi;
    Zk[i] = zi;
    cmac(x[(long long)v * n + i], alpha, zi);
    Cx<VT> ri = r[(long long)v * n + i];
    cmac(ri, mk(-alpha.re, -alpha.im), wi);
    r[(long long)v * n + i] = ri;
  }
}

__global__ void gcr_control_batch_kernel(int *ctl, const int *act, int nb, int restart, int max_iter,
                                         cudaGraphConditionalHandle handle) {
  const int it = ctl[0] + 1;
  int k = ctl[1] + 1;
  if (k == restart) k = 0;
  ctl[0] = it;
  ctl[1] = k;
  int any = 0;
  for (int v = 0; v < nb; ++v) any |= act[v];
  const int reason = !any ? 1 : (it >= max_iter ? 2 : 0);
  ctl[2] = reason;
  cudaGraphSetConditional(handle, reason == 0 ? 1u : 0u);
}

template <typename VT>
void launch_copy_active(const Cx<VT> *x, Cx<VT> *y, long long n, int nb, const int *act, cudaStream_t s) {
  copy_active_kernel<VT><<<dim3(stream_grid(n), nb), 256, 0, s>>>(x, y, n, act);
  MG_LAUNCHED();
}

template <typename VT>
void launch_gcr_dots_batch_devk(const Cx<VT> *W, const Cx<VT> *w, const Cx<VT> *r, const int *ctl, int nb,
                                int restart, long long n, double *out, const ReduceWs &ws, cudaStream_t s) {
  const int rows = restart + 3;
  int per = (int)(ws.capacity / (2LL * rows * nb));
  if (per > ws.max_blocks) per = ws.max_blocks;
  if (per < 1) per = 1;
  if ((long long)rows * nb > ws.tickets) fail(MG_ERR_UNSUPPORTED, "gcr_dots_batch: too many reduction slots");
  gcr_dots_batch_devk_kernel<VT><<<dim3(reduce_blocks(n, per), rows, nb), kReduceThreads, 0, s>>>(
      W, w, r, ctl, nb, restart, n, ws.partials, out, ws.ticket);
  MG_LAUNCHED();
}

void launch_gcr_coef_batch(const double *dots, const int *ctl, int nb, int restart, int *act, double *stv,
                           double *coef, cudaStream_t s) {
  gcr_coef_batch_kernel<<<1, 32, 0, s>>>(dots, ctl, nb, restart, act, stv, coef);
  MG_LAUNCHED();
}

template <typename VT>
void launch_gcr_update_batch_devk(Cx<VT> *W, Cx<VT> *Z, const Cx<VT> *w, const Cx<VT> *z, const int *ctl, int nb,
                                  int restart, const double *dots, const double *coef, Cx<VT> *x, Cx<VT> *r,
                                  long long n, cudaStream_t s) {
  gcr_update_batch_devk_kernel<VT><<<dim3(stream_grid(n), nb), 256, 0, s>>>(W, Z, w, z, ctl, nb, restart, dots, coef,
                                                                              x, r, n);
  MG_LAUNCHED();
}

#define MG_INST_DEVK(VT)                                                                                           \
  template void launch_copy_active<VT>(const Cx<VT> *, Cx<VT> *, long long, int, const int *, cudaStream_t);     \
  template void launch_gcr_dots_batch_devk<VT>(const Cx<VT> *, const Cx<VT> *, const Cx<VT> *, const int *, int,   \
                                               int, long long, double *, const ReduceWs &, cudaStream_t);        \
  template void launch_gcr_update_batch_devk<VT>(Cx<VT> *, Cx<VT> *, const Cx<VT> *, const Cx<VT> *, const int *, \
                                                 int, int, const double *, const double *, Cx<VT> *, Cx<VT> *,    \
                                                 long long, cudaStream_t);
MG_INST_DEVK(double)
MG_INST_DEVK(float)
#undef MG_INST_DEVK

void launch_gcr_control_batch(int *ctl, const int *act, int nb, int restart, int max_iter,
                              cudaGraphConditionalHandle handle, cudaStream_t s) {
  gcr_control_batch_kernel<<<1, 1, 0, s>>>(ctl, act, nb, restart, max_iter, handle);
  MG_LAUNCHED();
}

}  // namespace mg
