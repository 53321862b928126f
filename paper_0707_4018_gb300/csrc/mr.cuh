// Reduction helpers of the fused MR smoothing kernels (paper: MR with under-relaxation
// omega as the relaxation method): block trees of the partial sums, and the step length
// alpha = omega <A r, r> / |A r|^2 formed by every block of the consuming launch from the
// producing launch's block partials, in one fixed order.
#pragma once

#include "common.cuh"

namespace mg {

// block-wide sum of NOUT values of type T; the result is valid in thread 0 (sh: 32 NOUT)
template <int NOUT, typename T>
__device__ __forceinline__ void block_reduce(T (&v)[NOUT], T *sh) {
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
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      T t = (T)0;
      for (int w = 0; w < nw; ++w) t += sh[w * NOUT + k];
      v[k] = t;
    }
  }
}

// this block's (<A r, r> re, im, |A r|^2) into part_out[3 blockIdx.x ..]
template <typename R>
__device__ __forceinline__ void mr_publish(R (&v)[3], R *part_out, R *sh) {
  block_reduce<3, R>(v, sh);
  if (threadIdx.x == 0) {
    part_out[3 * blockIdx.x] = v[0];
    part_out[3 * blockIdx.x + 1] = v[1];
    part_out[3 * blockIdx.x + 2] = v[2];
  }
}

// alpha = omega <A r, r> / |A r|^2 from the `nb` block partials of the previous launch:
// thread t adds blocks t, t + blockDim, ..., then the block tree; thread 0 divides and
// broadcasts. Every thread of the block must call it.
template <typename R>
__device__ __forceinline__ Cx<R> mr_alpha(const R *part_in, int nb, double omega, R *sh) {
  R v[3] = {(R)0, (R)0, (R)0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v[0] += __ldcg(part_in + 3 * b);
    v[1] += __ldcg(part_in + 3 * b + 1);
    v[2] += __ldcg(part_in + 3 * b + 2);
  }
  block_reduce<3, R>(v, sh);
  __shared__ R s_alpha[2];
  if (threadIdx.x == 0) {
    const R den = v[2];
    s_alpha[0] = den > (R)0 ? (R)omega * v[0] / den : (R)0;
    s_alpha[1] = den > (R)0 ? (R)omega * v[1] / den : (R)0;
  }
  __syncthreads();
  return mk(s_alpha[0], s_alpha[1]);
}

template <typename R>
__device__ __forceinline__ Cx<R> mr_step(Cx<R> r, Cx<R> Ar, Cx<R> malpha) {
  cmac(r, malpha, Ar);
  return r;
}

}  // namespace mg
