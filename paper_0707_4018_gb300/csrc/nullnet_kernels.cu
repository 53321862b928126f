// Kernels of the learned near-null setup: a gauge-covariant parallel-transport network
// that maps random spinor fields to Nv near-null vector candidates (replacing most of the
// null-space relaxation of Eq. relax and the adaptive passes), its training by
// backpropagation of a rotation-invariant block loss, and Adam.
//
// Network (per site x, channel-spin index l = 2 c + s, directions self, +0, -0, +1, -1):
//   a_x = sum_dir W_dir T_dir(h)_x,  T_self h_x = h_x, T_{+mu} h_x = U_x^mu h_{x+mu},
//   T_{-mu} h_x = conj(U_{x-mu}^mu) h_{x-mu};   hidden layers h = a / sqrt(1 + |a_c|^2)
// per channel c (both spin components), last layer linear. The weights act on channel and
// spin only, so every layer commutes with U(1) gauge transformations.
//
// Layouts: activations h[f][x][2 C] as bfloat16 pairs (re, im); pre-activations and
// gradients float2 [f][x][2 C]; links float2 [f][x][2]; weights float2 [5][2 co][2 ci].
// One warp owns one site; lane l holds channel-spin entry l (2 C <= 32).
#include <cuda_bf16.h>

#include "nullnet.h"

namespace mg {

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cmacf(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cmacf_conj(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 bf2f(__nv_bfloat162 v) {
  return make_float2(__bfloat162float(v.x), __bfloat162float(v.y));
}
__device__ __forceinline__ __nv_bfloat162 f2bf(float2 v) {
  __nv_bfloat162 r;
  r.x = __float2bfloat16_rn(v.x);
  r.y = __float2bfloat16_rn(v.y);
  return r;
}

// neighbour site and transport phase of direction dir for the forward operator at x:
// T_dir h_x = phase * h_{nb}
__device__ __forceinline__ void fwd_hop(int dir, int x0, int x1, int L0, int L1, const float2 *Uf, long long &nb,
                                        float2 &ph) {
  const long long x = x0 + (long long)L0 * x1;
  switch (dir) {
    case 0: nb = x; ph = make_float2(1.f, 0.f); break;
    case 1: nb = (x0 + 1 == L0 ? 0 : x0 + 1) + (long long)L0 * x1; ph = Uf[2 * x]; break;
    case 2: {
      nb = (x0 == 0 ? L0 - 1 : x0 - 1) + (long long)L0 * x1;
      ph = conjf2(Uf[2 * nb]);
      break;
    }
    case 3: nb = x0 + (long long)L0 * (x1 + 1 == L1 ? 0 : x1 + 1); ph = Uf[2 * x + 1]; break;
    default: {
      nb = x0 + (long long)L0 * (x1 == 0 ? L1 - 1 : x1 - 1);
      ph = conjf2(Uf[2 * nb + 1]);
      break;
    }
  }
}

// adjoint: the contribution of direction dir to dL/dh^*_z comes from site src with phase
// (T_{+mu}: src = z - mu, conj(U_{z-mu}^mu); T_{-mu}: src = z + mu, U_z^mu)
__device__ __forceinline__ void adj_hop(int dir, int z0, int z1, int L0, int L1, const float2 *Uf, long long &src,
                                        float2 &ph) {
  const long long z = z0 + (long long)L0 * z1;
  switch (dir) {
    case 0: src = z; ph = make_float2(1.f, 0.f); break;
    case 1: {
      src = (z0 == 0 ? L0 - 1 : z0 - 1) + (long long)L0 * z1;
      ph = conjf2(Uf[2 * src]);
      break;
    }
    case 2: src = (z0 + 1 == L0 ? 0 : z0 + 1) + (long long)L0 * z1; ph = Uf[2 * z]; break;
    case 3: {
      src = z0 + (long long)L0 * (z1 == 0 ? L1 - 1 : z1 - 1);
      ph = conjf2(Uf[2 * src + 1]);
      break;
    }
    default: src = z0 + (long long)L0 * (z1 + 1 == L1 ? 0 : z1 + 1); ph = Uf[2 * z + 1]; break;
  }
}

constexpr int kWarps = 8;

// One layer forward. h_in: [f][x][ci2] bf16 pairs; out: pre-activation a (float2, may be null),
// gated bf16 h_out (hidden layers) or float2 y (last layer, LAST).
template <bool LAST>
__global__ void __launch_bounds__(256) ptconv_fwd_kernel(const __nv_bfloat162 *__restrict__ h_in,
                                                         const float2 *__restrict__ U, const int *__restrict__ fmap,
                                                         const float2 *__restrict__ W, int ci2, int co2, int L0,
                                                         int L1, float2 *__restrict__ a_out,
                                                         __nv_bfloat162 *__restrict__ h_out) {
  __shared__ float2 Ws[5 * 32 * 32];
  for (int q = threadIdx.x; q < 5 * co2 * ci2; q += blockDim.x) {
    const int dir = q / (co2 * ci2), r = q - dir * co2 * ci2, lo = r / ci2, li = r - lo * ci2;
    Ws[(dir * 32 + lo) * 32 + li] = W[q];
  }
  __syncthreads();
  const int f = blockIdx.y;
  const long long V = (long long)L0 * L1;
  const float2 *Uf = U + (size_t)(fmap ? fmap[f] : f) * 2 * V;
  const __nv_bfloat162 *hin = h_in + (size_t)f * V * ci2;
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)gridDim.x * kWarps;
  for (long long x = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); x < V; x += wstride) {
    const int x1 = (int)(x / L0), x0 = (int)(x - (long long)x1 * L0);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      long long nb;
      float2 ph;
      fwd_hop(dir, x0, x1, L0, L1, Uf, nb, ph);
      float2 v = lane < ci2 ? bf2f(hin[nb * ci2 + lane]) : make_float2(0.f, 0.f);
      v = cmulf(ph, v);
      const float2 *wrow = Ws + (dir * 32 + (lane < co2 ? lane : 0)) * 32;
      for (int li = 0; li < ci2; ++li) cmacf(acc, wrow[li], shfl2(v, li));
    }
    const size_t o = (size_t)f * V * co2 + (size_t)x * co2 + lane;
    if (LAST) {
      if (lane < co2) a_out[o] = acc;
    } else {
      if (a_out != nullptr && lane < co2) a_out[o] = acc;
      float s = acc.x * acc.x + acc.y * acc.y;
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      const float g = rsqrtf(1.f + s);
      if (lane < co2) h_out[o] = f2bf(make_float2(acc.x * g, acc.y * g));
    }
  }
}

// dL/dh^* of a layer's input from dL/da^* of its output, then (GATE_PREV) through the gate of
// the previous layer: ga_prev = g gh + 2 g'(s) Re(a^dagger gh)_c a
template <bool GATE_PREV>
__global__ void __launch_bounds__(256) ptconv_bwd_data_kernel(const float2 *__restrict__ ga,
                                                              const float2 *__restrict__ U,
                                                              const int *__restrict__ fmap,
                                                              const float2 *__restrict__ W, int ci2, int co2, int L0,
                                                              int L1, const float2 *__restrict__ a_prev,
                                                              float2 *__restrict__ ga_prev) {
  __shared__ float2 Ws[5 * 32 * 32];
  for (int q = threadIdx.x; q < 5 * co2 * ci2; q += blockDim.x) {
    const int dir = q / (co2 * ci2), r = q - dir * co2 * ci2, lo = r / ci2, li = r - lo * ci2;
    Ws[(dir * 32 + li) * 32 + lo] = W[q];  // transposed: row li holds W[dir][.][li]
  }
  __syncthreads();
  const int f = blockIdx.y;
  const long long V = (long long)L0 * L1;
  const float2 *Uf = U + (size_t)(fmap ? fmap[f] : f) * 2 * V;
  const float2 *gaf = ga + (size_t)f * V * co2;
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)gridDim.x * kWarps;
  for (long long z = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); z < V; z += wstride) {
    const int z1 = (int)(z / L0), z0 = (int)(z - (long long)z1 * L0);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      long long src;
      float2 ph;
      adj_hop(dir, z0, z1, L0, L1, Uf, src, ph);
      const float2 g = lane < co2 ? gaf[src * co2 + lane] : make_float2(0.f, 0.f);
      const float2 *wcol = Ws + (dir * 32 + (lane < ci2 ? lane : 0)) * 32;
      float2 t = make_float2(0.f, 0.f);
      for (int lo = 0; lo < co2; ++lo) cmacf_conj(t, wcol[lo], shfl2(g, lo));
      cmacf(acc, ph, t);
    }
    const size_t o = (size_t)f * V * ci2 + (size_t)z * ci2 + lane;
    if (GATE_PREV) {
      const float2 a = lane < ci2 ? a_prev[o] : make_float2(0.f, 0.f);
      float s = a.x * a.x + a.y * a.y;
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      float re = a.x * acc.x + a.y * acc.y;
      re += __shfl_xor_sync(0xffffffffu, re, 1);
      const float g = rsqrtf(1.f + s);
      const float dg2 = -g * g * g * re;  // 2 g'(s) Re(a^dagger gh), g' = -g^3 / 2
      if (lane < ci2) ga_prev[o] = make_float2(g * acc.x + dg2 * a.x, g * acc.y + dg2 * a.y);
    } else if (lane < ci2) {
      ga_prev[o] = acc;
    }
  }
}

// Per-CTA partial sums of dL/dW^*[dir][lo][li] = sum_x ga_x[lo] conj(T_dir h_x[li]) over a
// contiguous range of (field, site) pairs; partials[cta][entry] (entry = (dir co2 + lo) ci2 + li)
constexpr int kWG = 8;  // sites staged per group
__global__ void __launch_bounds__(256) ptconv_bwd_weight_kernel(const float2 *__restrict__ ga,
                                                                const __nv_bfloat162 *__restrict__ h_in,
                                                                const float2 *__restrict__ U,
                                                                const int *__restrict__ fmap, int nf, int ci2,
                                                                int co2, int L0, int L1,
                                                                float2 *__restrict__ partials) {
  __shared__ float2 gs[kWG][32];
  __shared__ float2 Ts[kWG][5][32];
  const long long V = (long long)L0 * L1, total = V * nf;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long p0 = (long long)blockIdx.x * per, p1 = p0 + per < total ? p0 + per : total;
  const int ne = 5 * co2 * ci2;
  constexpr int kEnt = 20;  // 5 * 32 * 32 / 256
  float2 acc[kEnt];
#pragma unroll
  for (int e = 0; e < kEnt; ++e) acc[e] = make_float2(0.f, 0.f);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long g0 = p0; g0 < p1; g0 += kWG) {
    __syncthreads();
    // warp w stages site g0 + w: its gradient row and its five transported inputs
    const long long p = g0 + wid;
    if (wid < kWG) {
      float2 gv = make_float2(0.f, 0.f);
      float2 tv[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) tv[d] = make_float2(0.f, 0.f);
      if (p < p1) {
        const int f = (int)(p / V);
        const long long x = p - (long long)f * V;
        const int x1 = (int)(x / L0), x0 = (int)(x - (long long)x1 * L0);
        const float2 *Uf = U + (size_t)(fmap ? fmap[f] : f) * 2 * V;
        if (lane < co2) gv = ga[(size_t)p * co2 + lane];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          long long nb;
          float2 ph;
          fwd_hop(d, x0, x1, L0, L1, Uf, nb, ph);
          if (lane < ci2) tv[d] = cmulf(ph, bf2f(h_in[((size_t)f * V + nb) * ci2 + lane]));
        }
      }
      gs[wid][lane] = gv;
#pragma unroll
      for (int d = 0; d < 5; ++d) Ts[wid][d][lane] = tv[d];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kEnt; ++e) {
      const int q = threadIdx.x + 256 * e;
      if (q < ne) {
        const int dir = q / (co2 * ci2), r = q - dir * co2 * ci2, lo = r / ci2, li = r - lo * ci2;
#pragma unroll
        for (int s = 0; s < kWG; ++s) cmacf_conj(acc[e], Ts[s][dir][li], gs[s][lo]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < kEnt; ++e) {
    const int q = threadIdx.x + 256 * e;
    if (q < ne) partials[(size_t)blockIdx.x * ne + q] = acc[e];
  }
}

// gW[q] = sum over CTAs of partials[cta][q] (fixed order, FP64 sums)
__global__ void sum_partials_kernel(const float2 *__restrict__ partials, int nparts, int ne,
                                    float2 *__restrict__ gW) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ne) return;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < nparts; ++c) {
    const float2 v = partials[(size_t)c * ne + q];
    re += v.x;
    im += v.y;
  }
  gW[q] = make_float2((float)re, (float)im);
}

// Rotation-invariant block loss and dL/dy^*: one warp per (field, block), lane r = 2 i + s
// (site i of the block, spin s). G = W^dagger W and C = W^dagger V in FP32 warp sums, then the
// small dense algebra in FP64: G = L L^dagger (a relative ridge of 1e-7 tr G / nv keeps FP32
// round-off from breaking it), A = G^{-1} C, L_b = nv - Re tr(C^dagger A); grad = -(V - W A) A^dagger.
constexpr int kMaxNv = 8;
__global__ void __launch_bounds__(128) nullnet_loss_kernel(const float2 *__restrict__ y,
                                                           const float2 *__restrict__ target,
                                                           const int *__restrict__ fmap, int nv, BlockGeo bg,
                                                           float scale, float2 *__restrict__ gy,
                                                           double *__restrict__ lossb) {
  __shared__ double Gs[4][kMaxNv * kMaxNv * 2];
  __shared__ double Cs[4][kMaxNv * kMaxNv * 2];
  __shared__ double As[4][kMaxNv * kMaxNv * 2];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nb = bg.nblocks;
  const long long wglob = (long long)blockIdx.x * 4 + wid;
  const int f = blockIdx.y;
  const long long V = (long long)bg.L0 * bg.L1;
  if (wglob >= nb) return;  // whole warps leave together
  const long long b = wglob;
  const int rows = bg.bvol * 2;
  const bool act = lane < rows;
  long long site = 0;
  int sp = 0;
  if (act) {
    site = fine_site_of(bg, b, lane >> 1);
    sp = lane & 1;
  }
  const float2 *yf = y + (size_t)f * V * 2 * nv;
  const float2 *tf = target + (size_t)(fmap ? fmap[f] : f) * nv * V * 2;
  float2 w[kMaxNv], v[kMaxNv];
#pragma unroll
  for (int k = 0; k < kMaxNv; ++k) {
    w[k] = (act && k < nv) ? yf[(size_t)site * 2 * nv + 2 * k + sp] : make_float2(0.f, 0.f);
    v[k] = (act && k < nv) ? tf[((size_t)k * V + site) * 2 + sp] : make_float2(0.f, 0.f);
  }
  double *G = Gs[wid], *C = Cs[wid], *A = As[wid];
  for (int k = 0; k < nv; ++k) {
    for (int j = 0; j < nv; ++j) {
      float2 g = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
      cmacf_conj(g, w[k], w[j]);
      cmacf_conj(c, w[k], v[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
        c.x += __shfl_xor_sync(0xffffffffu, c.x, o);
        c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
      }
      if (lane == 0) {
        G[(k * nv + j) * 2] = g.x;
        G[(k * nv + j) * 2 + 1] = g.y;
        C[(k * nv + j) * 2] = c.x;
        C[(k * nv + j) * 2 + 1] = c.y;
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    // Cholesky G = L L^dagger in place (lower triangle), with the ridge
    double tr = 0.0;
    for (int k = 0; k < nv; ++k) tr += G[(k * nv + k) * 2];
    const double ridge = 1e-7 * tr / nv + 1e-30;
    for (int k = 0; k < nv; ++k) G[(k * nv + k) * 2] += ridge;
    for (int j = 0; j < nv; ++j) {
      double d = G[(j * nv + j) * 2];
      for (int k = 0; k < j; ++k) d -= G[(j * nv + k) * 2] * G[(j * nv + k) * 2] + G[(j * nv + k) * 2 + 1] * G[(j * nv + k) * 2 + 1];
      d = sqrt(fmax(d, 1e-300));
      G[(j * nv + j) * 2] = d;
      G[(j * nv + j) * 2 + 1] = 0.0;
      for (int i = j + 1; i < nv; ++i) {
        // L_ij = (G_ij - sum_k L_ik conj(L_jk)) / L_jj, G_ij = conj(G_ji) read from the upper part
        double re = G[(j * nv + i) * 2], im = -G[(j * nv + i) * 2 + 1];
        for (int k = 0; k < j; ++k) {
          const double ar = G[(i * nv + k) * 2], ai = G[(i * nv + k) * 2 + 1];
          const double br = G[(j * nv + k) * 2], bi = G[(j * nv + k) * 2 + 1];
          re -= ar * br + ai * bi;
          im -= ai * br - ar * bi;
        }
        G[(i * nv + j) * 2] = re / d;
        G[(i * nv + j) * 2 + 1] = im / d;
      }
    }
  }
  __syncwarp();
  // column j of A = G^{-1} C by lane j: L u = c_j, then L^dagger a = u
  if (lane < nv) {
    const int j = lane;
    double ur[kMaxNv], ui[kMaxNv];
    for (int i = 0; i < nv; ++i) {
      double re = C[(i * nv + j) * 2], im = C[(i * nv + j) * 2 + 1];
      for (int k = 0; k < i; ++k) {
        const double lr = G[(i * nv + k) * 2], li = G[(i * nv + k) * 2 + 1];
        re -= lr * ur[k] - li * ui[k];
        im -= lr * ui[k] + li * ur[k];
      }
      const double d = G[(i * nv + i) * 2];
      ur[i] = re / d;
      ui[i] = im / d;
    }
    for (int i = nv - 1; i >= 0; --i) {
      double re = ur[i], im = ui[i];
      for (int k = i + 1; k < nv; ++k) {
        // (L^dagger)_ik = conj(L_ki)
        const double lr = G[(k * nv + i) * 2], li = -G[(k * nv + i) * 2 + 1];
        re -= lr * A[(k * nv + j) * 2] - li * A[(k * nv + j) * 2 + 1];
        im -= lr * A[(k * nv + j) * 2 + 1] + li * A[(k * nv + j) * 2];
      }
      const double d = G[(i * nv + i) * 2];
      A[(i * nv + j) * 2] = re / d;
      A[(i * nv + j) * 2 + 1] = im / d;
    }
  }
  __syncwarp();
  if (lane == 0) {
    double tr = 0.0;  // Re tr(C^dagger A) = sum_ij Re(conj(C_ij) A_ij)
    for (int q = 0; q < nv * nv; ++q) tr += C[2 * q] * A[2 * q] + C[2 * q + 1] * A[2 * q + 1];
    lossb[(size_t)f * nb + b] = (double)nv - tr;
  }
  if (!act) return;
  // R = V - W A, grad_k' = -sum_k R_k conj(A_k'k)
  float2 r[kMaxNv];
#pragma unroll
  for (int k = 0; k < kMaxNv; ++k) {
    if (k >= nv) break;
    float2 t = v[k];
    for (int q = 0; q < nv; ++q) {
      const float2 a = make_float2((float)A[(q * nv + k) * 2], (float)A[(q * nv + k) * 2 + 1]);
      cmacf(t, make_float2(-w[q].x, -w[q].y), a);
    }
    r[k] = t;
  }
  float2 *gf = gy + (size_t)f * V * 2 * nv;
  for (int kp = 0; kp < nv; ++kp) {
    float2 t = make_float2(0.f, 0.f);
    for (int k = 0; k < nv; ++k) {
      const float2 a = make_float2((float)A[(kp * nv + k) * 2], (float)A[(kp * nv + k) * 2 + 1]);
      cmacf(t, r[k], conjf2(a));
    }
    gf[(size_t)site * 2 * nv + 2 * kp + sp] = make_float2(-scale * t.x, -scale * t.y);
  }
}

// Adam on the real and imaginary parts (the real-parameter gradient is 2 (Re, Im) of dL/dW^*)
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, long long n, float lr, float b1, float b2, float c1, float c2,
                            float eps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = 2.f * g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// noise [c][f][x][2] complex128 (Philox Gaussians) -> bf16 [f][x][2 c + s]
__global__ void pack_noise_kernel(const Cx<double> *__restrict__ z, int cin, long long V, int nf,
                                  __nv_bfloat162 *__restrict__ h) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)nf * V * 2 * cin;
  if (i >= n) return;
  const int l = (int)(i % (2 * cin));
  const long long fx = i / (2 * cin);
  const int c = l >> 1, s = l & 1;
  const Cx<double> v = z[((size_t)c * nf * V + fx) * 2 + s];
  h[i] = f2bf(make_float2((float)v.re, (float)v.im));
}

// predicted vectors y[x][2 nv] (float2) -> v[k][x][2] complex128 (the layout of the setup's vectors)
__global__ void unpack_vectors_kernel(const float2 *__restrict__ y, int nv, long long V,
                                      Cx<double> *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nv * V * 2) return;
  const int s = (int)(i & 1);
  const long long kx = i >> 1;
  const int k = (int)(kx / V);
  const long long x = kx - (long long)k * V;
  const float2 v = y[(size_t)x * 2 * nv + 2 * k + s];
  out[i] = mk((double)v.x, (double)v.y);
}

// complex128 -> float2 (links, targets)
__global__ void to_float2_kernel(const Cx<double> *__restrict__ a, long long n, float2 *__restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].re, (float)a[i].im);
}

int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

int site_grid(long long V) {
  const long long want = (V + kWarps - 1) / kWarps;
  return (int)(want < 152 * 16 ? want : 152 * 16);
}

}  // namespace

void launch_ptconv_fwd(const void *h_in, const float2 *U, const int *fmap, const float2 *W, int ci2, int co2,
                       int L0, int L1, int nf, bool last, float2 *a_out, void *h_out, cudaStream_t s) {
  const dim3 grid(site_grid((long long)L0 * L1), nf);
  const auto *hi = static_cast<const __nv_bfloat162 *>(h_in);
  if (last)
    ptconv_fwd_kernel<true><<<grid, 256, 0, s>>>(hi, U, fmap, W, ci2, co2, L0, L1, a_out, nullptr);
  else
    ptconv_fwd_kernel<false><<<grid, 256, 0, s>>>(hi, U, fmap, W, ci2, co2, L0, L1, a_out,
                                                   static_cast<__nv_bfloat162 *>(h_out));
  MG_LAUNCHED();
}

void launch_ptconv_bwd_data(const float2 *ga, const float2 *U, const int *fmap, const float2 *W, int ci2, int co2,
                            int L0, int L1, int nf, const float2 *a_prev, float2 *ga_prev, cudaStream_t s) {
  const dim3 grid(site_grid((long long)L0 * L1), nf);
  if (a_prev != nullptr)
    ptconv_bwd_data_kernel<true><<<grid, 256, 0, s>>>(ga, U, fmap, W, ci2, co2, L0, L1, a_prev, ga_prev);
  else
    ptconv_bwd_data_kernel<false><<<grid, 256, 0, s>>>(ga, U, fmap, W, ci2, co2, L0, L1, nullptr, ga_prev);
  MG_LAUNCHED();
}

void launch_ptconv_bwd_weight(const float2 *ga, const void *h_in, const float2 *U, const int *fmap, int nf, int ci2,
                              int co2, int L0, int L1, float2 *partials, int nparts, float2 *gW, cudaStream_t s) {
  ptconv_bwd_weight_kernel<<<nparts, 256, 0, s>>>(ga, static_cast<const __nv_bfloat162 *>(h_in), U, fmap, nf, ci2,
                                                  co2, L0, L1, partials);
  MG_LAUNCHED();
  const int ne = 5 * co2 * ci2;
  sum_partials_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(partials, nparts, ne, gW);
  MG_LAUNCHED();
}

void launch_nullnet_loss(const float2 *y, const float2 *target, const int *fmap, int nv, const BlockGeo &bg, int nf,
                         float scale, float2 *gy, double *lossb, cudaStream_t s) {
  const dim3 grid(blocks_for(bg.nblocks, 4), nf);
  nullnet_loss_kernel<<<grid, 128, 0, s>>>(y, target, fmap, nv, bg, scale, gy, lossb);
  MG_LAUNCHED();
}

void launch_adam(float *w, const float *g, float *m1, float *m2, long long n, float lr, long long t,
                 cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(w, g, m1, m2, n, lr, b1, b2, c1, c2, 1e-8f);
  MG_LAUNCHED();
}

void launch_pack_noise(const Cx<double> *z, int cin, long long V, int nf, void *h, cudaStream_t s) {
  const long long n = (long long)nf * V * 2 * cin;
  pack_noise_kernel<<<blocks_for(n, 256), 256, 0, s>>>(z, cin, V, nf, static_cast<__nv_bfloat162 *>(h));
  MG_LAUNCHED();
}

void launch_unpack_vectors(const float2 *y, int nv, long long V, Cx<double> *out, cudaStream_t s) {
  unpack_vectors_kernel<<<blocks_for((long long)nv * V * 2, 256), 256, 0, s>>>(y, nv, V, out);
  MG_LAUNCHED();
}

void launch_to_float2(const Cx<double> *a, long long n, float2 *b, cudaStream_t s) {
  to_float2_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, n, b);
  MG_LAUNCHED();
}

}  // namespace mg
