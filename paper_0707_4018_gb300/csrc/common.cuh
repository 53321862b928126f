// Internal definitions shared by the CUDA translation units of the multigrid
// library: complex arithmetic on interleaved (re, im) pairs, error handling,
// device buffers, lattice geometry and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>

#include "../../include/mg.h"

namespace mg {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string &msg) { throw Error{code, msg}; }

#define MG_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) ::mg::fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern std::atomic<long long> g_launches;

// Checks a kernel launch and counts it.
#define MG_LAUNCHED()                                                                           \
  do {                                                                                          \
    ::mg::g_launches.fetch_add(1, std::memory_order_relaxed);                                   \
    cudaError_t e_ = cudaGetLastError();                                                        \
    if (e_ != cudaSuccess) ::mg::fail(MG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// complex numbers (interleaved, same layout as complex128 / complex64)
// ---------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) Cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ Cx<R> mk(R re, R im) {
  Cx<R> c;
  c.re = re;
  c.im = im;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return mk(s * a.re, s * a.im); }
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ Cx<R> cmul_conj(Cx<R> a, Cx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// i * a
template <typename R>
__host__ __device__ __forceinline__ Cx<R> times_i(Cx<R> a) { return mk(-a.im, a.re); }
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cmac(Cx<R> &acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cmac_conj(Cx<R> &acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(Cx<R> a) { return a.re * a.re + a.im * a.im; }

template <typename To, typename From>
__host__ __device__ __forceinline__ Cx<To> cvt(Cx<From> a) { return mk((To)a.re, (To)a.im); }

// ---------------------------------------------------------------------------
// device buffers: stream-ordered allocations from the device's default memory
// pool, ordered on the calling thread's per-thread stream. Contexts are made and
// dropped often (one per configuration); the pool keeps freed memory, so that
// costs neither driver allocations nor device-wide synchronisation (a plain
// cudaFree synchronises the whole device, stalling every other context).
// The owner must have finished all work on a buffer before it is released, and
// must order its first use after the allocation (pool_ready below).
// ---------------------------------------------------------------------------
void pool_init();   // once per process and device: keep freed memory in the pool
void pool_ready();  // allocations made by this thread so far are usable on any stream

template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    pool_init();
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, count * sizeof(T), cudaStreamPerThread);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      fail(MG_ERR_OOM, "cudaMallocAsync of " + std::to_string(count * sizeof(T)) + " bytes: " + cudaGetErrorString(e));
    }
    p = static_cast<T *>(q);
    n = count;
  }
  void release() {
    if (p) cudaFreeAsync(p, cudaStreamPerThread);
    p = nullptr;
    n = 0;
  }
};

// two timing events recorded around a region of a stream; destroyed on every exit path
// (a solve that throws must not leak them)
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventPair() {
    MG_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      fail(MG_ERR_CUDA, "cudaEventCreate failed");
    }
  }
  EventPair(const EventPair &) = delete;
  EventPair &operator=(const EventPair &) = delete;
  ~EventPair() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  void start(cudaStream_t s) { MG_CUDA(cudaEventRecord(e0, s)); }
  // records the end, waits for it and returns the milliseconds between the two events
  float stop(cudaStream_t s) {
    MG_CUDA(cudaEventRecord(e1, s));
    MG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  }
};

// ---------------------------------------------------------------------------
// geometry of one 2d level and of a blocking between two levels
// ---------------------------------------------------------------------------
struct Geo2 {
  int L0, L1;
  long long nsites;
};

// periodic 4d lattice, x = x0 + L0 (x1 + L1 (x2 + L2 x3)); fewer than 2^31 sites
struct Geo4 {
  int L[4];
  long long nsites;
};

// fine level (extents L0 x L1, nint dofs per site) blocked by B0 x B1 into a
// coarse level of extents nb0 x nb1; a block holds bvol = B0*B1 sites and
// Nb = bvol * nint dofs ordered (in-block site s, internal dof a) -> s*nint + a.
struct BlockGeo {
  int L0, L1, B0, B1, nb0, nb1, bvol, nint, Nb;
  long long nblocks;
};

// 32-bit index arithmetic (a 64-bit division costs about a hundred instructions; lattices
// are limited to fewer than 2^31 sites at setup)
__host__ __device__ __forceinline__ long long fine_site_of(const BlockGeo &g, long long b, int s) {
  const int bi = (int)b;
  const int cb1 = bi / g.nb0, cb0 = bi - cb1 * g.nb0;
  const int sy = s / g.B0, sx = s - sy * g.B0;
  return (long long)(cb0 * g.B0 + sx) + (long long)g.L0 * (cb1 * g.B1 + sy);
}

// ---------------------------------------------------------------------------
// deterministic reductions: fixed thread->element map and fixed trees
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of NOUT doubles over a block of blockDim.x (multiple of 32, <= 1024)
// threads; the result is valid in thread 0. Uses `sh` (>= 32*NOUT doubles).
template <int NOUT>
__device__ __forceinline__ void block_sum(double (&v)[NOUT], double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NOUT; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) sh[wid * NOUT + k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) v[k] = (lane < nw) ? sh[lane * NOUT + k] : 0.0;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) v[k] = warp_sum(v[k]);
  }
  __syncthreads();
}

// Grid reduction epilogue: every block writes its NOUT partials; the last
// block to finish sums all partials in block order and stores them in out[].
// `ticket` must be zero before the launch; the last block resets it.
template <int NOUT>
__device__ __forceinline__ void grid_finish(double (&v)[NOUT], double *partials, double *out, unsigned int *ticket,
                                            double *sh) {
  block_sum<NOUT>(v, sh);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) partials[blockIdx.x * NOUT + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w[NOUT];
#pragma unroll
  for (int k = 0; k < NOUT; ++k) w[k] = 0.0;
  // fixed order: thread t sums partials t, t + blockDim, ...; then the block tree
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) w[k] += ((volatile double *)partials)[b * NOUT + k];
  }
  block_sum<NOUT>(w, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) out[k] = w[k];
    *ticket = 0u;
  }
}

// Same epilogue with the per-thread values and the block tree in type T (float
// for FP32 vectors: GB300's FP64 unit is far slower) and FP64 partials / final sum.
template <int NOUT, typename T>
__device__ __forceinline__ void grid_finish_t(T (&v)[NOUT], double *partials, double *out, unsigned int *ticket,
                                              T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NOUT; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) sh[wid * NOUT + k] = v[k];
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      T t = (T)0;
      for (int w = 0; w < nw; ++w) t += sh[w * NOUT + k];
      partials[blockIdx.x * NOUT + k] = (double)t;
    }
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w[NOUT];
#pragma unroll
  for (int k = 0; k < NOUT; ++k) w[k] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) w[k] += ((volatile double *)partials)[b * NOUT + k];
  }
  __shared__ double shd[32 * NOUT];
  block_sum<NOUT>(w, shd);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) out[k] = w[k];
    *ticket = 0u;
  }
}

// Workspace for grid reductions (partials + ticket) owned by a context.
struct ReduceWs {
  double *partials;
  unsigned int *ticket;
  int max_blocks;         // grid cap of the grid-stride reductions
  long long capacity = 0; // doubles available in partials
  long long tickets = 0;  // counters available in ticket
};

constexpr int kReduceThreads = 256;
inline int reduce_blocks(long long n, int max_blocks) {
  long long b = (n + kReduceThreads - 1) / kReduceThreads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

inline unsigned int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned int)b;
}

}  // namespace mg
