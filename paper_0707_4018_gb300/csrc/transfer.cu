// Block-local transfer between levels (paper, Eq. P1 and the adaptive step):
// restriction P^dagger, prolongation P, block Gram-Schmidt of the near-null
// vectors, the Galerkin coarse operator P^dagger A P (Eq. Galerkin) and the
// Philox draws of the setup's random vectors.
//
// Mapping: one warp per block S_j; lane l owns the block dofs i = l + 32 p
// (i = s * n_int + a: in-block site s, internal dof a). Block vectors live in
// the prolongator array V[b][k][i] (block-major, FP64 or FP32), so a warp
// reads its block's Nv columns with unit stride.
#include "kernels.h"
#include "wilson.cuh"

namespace mg {

constexpr int kMaxNv = 32;

template <typename R>
__device__ __forceinline__ R shfl_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// restriction: coarse[b][k] = sum_i conj(V[b][k][i]) fine[site(b, s)][a]
// ---------------------------------------------------------------------------
template <typename R, int NVM>
__global__ void __launch_bounds__(128) restrict_kernel(const Cx<R> *__restrict__ V, const Cx<R> *__restrict__ fine,
                                                       Cx<R> *__restrict__ coarse, BlockGeo g, int Nv) {
  // vector blockIdx.y of a batch: fine stride nblocks * Nb, coarse stride nblocks * Nv
  fine += blockIdx.y * (g.nblocks * (long long)g.Nb);
  coarse += blockIdx.y * (g.nblocks * (long long)Nv);
  const long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= g.nblocks) return;
  Cx<R> acc[NVM];
#pragma unroll
  for (int k = 0; k < NVM; ++k) acc[k] = mk((R)0, (R)0);
  const Cx<R> *Vb = V + b * (long long)Nv * g.Nb;
  for (int i = lane; i < g.Nb; i += 32) {
    const int s = i / g.nint, a = i - s * g.nint;
    const Cx<R> r = fine[fine_site_of(g, b, s) * g.nint + a];
#pragma unroll
    for (int k = 0; k < NVM; ++k)
      if (k < Nv) cmac_conj(acc[k], Vb[(long long)k * g.Nb + i], r);
  }
  Cx<R> mine = mk((R)0, (R)0);
#pragma unroll
  for (int k = 0; k < NVM; ++k) {
    if (k < Nv) {
      const R re = shfl_sum(acc[k].re), im = shfl_sum(acc[k].im);
      if (lane == k) mine = mk(re, im);
    }
  }
  if (lane < Nv) coarse[b * Nv + lane] = mine;
}

// Streaming restriction for Nv = 8 (the hot levels): a CTA of 256 threads takes BPC
// consecutive blocks, whose prolongator rows V[b][k][0..Nb) form one contiguous tile
// (16 KB in FP32), and reads it with 16-byte loads in order (four per thread): every
// load instruction of a warp covers 512 contiguous bytes. A 16-byte vector holds CPV
// complex numbers (2 in FP32, 1 in FP64) of one (block, k) row and of one site (n_int is
// a multiple of CPV), so the matching residual entries are one 16-byte vector too; the CTA
// stages its blocks' residual entries in shared memory once, and the eight rows k of a block
// read them there (loading them once per k from L1/L2 held the kernel at 0.54 of HBM). The Nb / CPV vectors of a row belong to consecutive
// lanes and are summed by a shuffle tree within that lane group.
template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int cpv = 2;
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int cpv = 1;
};

template <typename R>
__device__ __forceinline__ void cmac_conj_vec(Cx<R> &acc, typename Vec16<R>::T v, typename Vec16<R>::T r);
template <>
__device__ __forceinline__ void cmac_conj_vec<float>(Cx<float> &acc, float4 v, float4 r) {
  cmac_conj(acc, mk(v.x, v.y), mk(r.x, r.y));
  cmac_conj(acc, mk(v.z, v.w), mk(r.z, r.w));
}
template <>
__device__ __forceinline__ void cmac_conj_vec<double>(Cx<double> &acc, double2 v, double2 r) {
  cmac_conj(acc, mk(v.x, v.y), mk(r.x, r.y));
}

template <typename R, int BPC, int PER_ROW>
__global__ void __launch_bounds__(256) restrict8_stream_kernel(const Cx<R> *__restrict__ V,
                                                               const Cx<R> *__restrict__ fine,
                                                               Cx<R> *__restrict__ coarse, BlockGeo g) {
  using T = typename Vec16<R>::T;
  constexpr int CPV = Vec16<R>::cpv;
  constexpr int NV = 8;
  constexpr int ITERS = BPC * NV * PER_ROW / 256;  // vectors per thread
  static_assert(ITERS * 256 == BPC * NV * PER_ROW && PER_ROW <= 32 && (PER_ROW & (PER_ROW - 1)) == 0, "tile");
  fine += blockIdx.y * (g.nblocks * (long long)g.Nb);
  coarse += blockIdx.y * (g.nblocks * (long long)NV);
  const long long b0 = (long long)blockIdx.x * BPC;
  const T *tile = reinterpret_cast<const T *>(V + b0 * NV * g.Nb);
  const int lane = threadIdx.x & 31;
  // coarse coordinates of the CTA's first block, once (32-bit: index arithmetic, not
  // bandwidth, bounded the first version of this kernel)
  const int b0i = (int)b0;
  const int c1_0 = b0i / g.nb0, c0_0 = b0i - c1_0 * g.nb0;
  // the residual entries of the CTA's blocks, one 16-byte vector per (block, j)
  __shared__ T rs[BPC * PER_ROW];
  for (int q = threadIdx.x; q < BPC * PER_ROW; q += 256) {
    const int bl = q / PER_ROW, j = q - bl * PER_ROW;
    T val = T{};
    if (b0i + bl < g.nblocks) {
      int c0 = c0_0 + bl, c1 = c1_0;
      while (c0 >= g.nb0) {  // the CTA's blocks are consecutive in x, wrapping into the next row
        c0 -= g.nb0;
        ++c1;
      }
      const int i = j * CPV, st = i / g.nint, a = i - st * g.nint;
      const int sy = st / g.B0, sx = st - sy * g.B0;
      const long long site = (long long)(c0 * g.B0 + sx) + (long long)g.L0 * (c1 * g.B1 + sy);
      val = *reinterpret_cast<const T *>(fine + site * g.nint + a);
    }
    rs[q] = val;
  }
  // all tile loads first: ITERS tile vectors in flight together
  T vv[ITERS];
#pragma unroll
  for (int u = 0; u < ITERS; ++u) {
    const int f = threadIdx.x + 256 * u;
    const int bl = f / PER_ROW / NV;
    vv[u] = b0i + bl < g.nblocks ? tile[f] : T{};
  }
  __syncthreads();
  T rr[ITERS];
#pragma unroll
  for (int u = 0; u < ITERS; ++u) {
    const int f = threadIdx.x + 256 * u;
    const int row = f / PER_ROW, j = f - row * PER_ROW;
    rr[u] = rs[(row / NV) * PER_ROW + j];
  }
#pragma unroll
  for (int u = 0; u < ITERS; ++u) {
    const int f = threadIdx.x + 256 * u;
    const int row = f / PER_ROW;
    const long long b = b0 + row / NV;
    Cx<R> acc = mk((R)0, (R)0);
    cmac_conj_vec<R>(acc, vv[u], rr[u]);
#pragma unroll
    for (int o = PER_ROW >> 1; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if ((lane & (PER_ROW - 1)) == 0 && b < g.nblocks) coarse[b * NV + (row - (row / NV) * NV)] = acc;
  }
}

// ---------------------------------------------------------------------------
// prolongation: fine[site(b, s)][a] += sum_k V[b][k][i] coarse[b][k]
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) prolong_add_kernel(const Cx<R> *__restrict__ V, const Cx<R> *__restrict__ coarse,
                                                          Cx<R> *__restrict__ fine, BlockGeo g, int Nv) {
  fine += blockIdx.y * (g.nblocks * (long long)g.Nb);
  coarse += blockIdx.y * (g.nblocks * (long long)Nv);
  const long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= g.nblocks) return;
  const Cx<R> *Vb = V + b * (long long)Nv * g.Nb;
  const Cx<R> *e = coarse + b * Nv;
  const int c1 = (int)(b / g.nb0), c0 = (int)(b - (long long)c1 * g.nb0);
  for (int i = lane; i < g.Nb; i += 32) {
    const int s = i / g.nint, a = i - s * g.nint;
    const int sy = s / g.B0, sx = s - sy * g.B0;
    const long long f = ((long long)(c0 * g.B0 + sx) + (long long)g.L0 * (c1 * g.B1 + sy)) * g.nint + a;
    Cx<R> acc = fine[f];
    for (int k = 0; k < Nv; ++k) cmac(acc, Vb[(long long)k * g.Nb + i], e[k]);
    fine[f] = acc;
  }
}

// ---------------------------------------------------------------------------
// block Gram-Schmidt: modified GS in k order, two passes, FP64; each lane only
// touches its own dofs (kept in shared memory), sums go through shuffles
// ---------------------------------------------------------------------------
__global__ void block_mgs_kernel(const Cx<double> *__restrict__ vecs, long long vstride, Cx<double> *__restrict__ V,
                                 BlockGeo g, int Nv, double *__restrict__ min_norm) {
  extern __shared__ Cx<double> smem_mgs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long b = blockIdx.x * (long long)(blockDim.x >> 5) + warp;
  if (b >= g.nblocks) return;
  Cx<double> *v = smem_mgs + (long long)warp * Nv * g.Nb;  // v[k * Nb + i]
  for (int k = 0; k < Nv; ++k)
    for (int i = lane; i < g.Nb; i += 32) {
      const int s = i / g.nint, a = i - s * g.nint;
      v[k * g.Nb + i] = vecs[k * vstride + fine_site_of(g, b, s) * g.nint + a];
    }
  double mn = 1e300;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < Nv; ++k) {
      Cx<double> *vk = v + k * g.Nb;
      for (int j = 0; j < k; ++j) {
        const Cx<double> *vj = v + j * g.Nb;
        Cx<double> d = mk(0.0, 0.0);
        for (int i = lane; i < g.Nb; i += 32) cmac_conj(d, vj[i], vk[i]);
        d.re = shfl_sum(d.re);
        d.im = shfl_sum(d.im);
        const Cx<double> md = mk(-d.re, -d.im);
        for (int i = lane; i < g.Nb; i += 32) cmac(vk[i], md, vj[i]);
      }
      double n2 = 0.0;
      for (int i = lane; i < g.Nb; i += 32) n2 += norm2(vk[i]);
      n2 = shfl_sum(n2);
      const double nrm = sqrt(n2);
      mn = fmin(mn, nrm);
      const double inv = 1.0 / nrm;
      for (int i = lane; i < g.Nb; i += 32) vk[i] = inv * vk[i];
    }
  }
  Cx<double> *Vb = V + b * (long long)Nv * g.Nb;
  for (int k = 0; k < Nv; ++k)
    for (int i = lane; i < g.Nb; i += 32) Vb[(long long)k * g.Nb + i] = v[k * g.Nb + i];
  if (lane == 0 && min_norm) min_norm[b] = mn;
}

// ---------------------------------------------------------------------------
// Galerkin coarse operator. For every block b and vector k, the five parts of
// A W_k at the block's dofs are formed (W_k = column k of P in every block):
// dir 0 collects the site-local term and the hops that stay inside the block,
// dir d collects the hops from direction d that cross the block face. Then
// Yc[b][dir](k', k) = sum_i conj(V[b][k'][i]) part[dir][k][i].
// ---------------------------------------------------------------------------
struct NbrInfo {
  long long src_b;
  int src_s;
  long long site;
  bool face;
};

__device__ __forceinline__ NbrInfo neighbour_in_blocks(const BlockGeo &g, int x0, int x1, int dir) {
  int y0 = x0, y1 = x1;
  bool face;
  switch (dir) {
    case 1: y0 = (x0 + 1 == g.L0) ? 0 : x0 + 1; face = (x0 % g.B0) == g.B0 - 1; break;
    case 2: y0 = (x0 == 0) ? g.L0 - 1 : x0 - 1; face = (x0 % g.B0) == 0; break;
    case 3: y1 = (x1 + 1 == g.L1) ? 0 : x1 + 1; face = (x1 % g.B1) == g.B1 - 1; break;
    default: y1 = (x1 == 0) ? g.L1 - 1 : x1 - 1; face = (x1 % g.B1) == 0; break;
  }
  NbrInfo n;
  n.src_b = (long long)(y0 / g.B0) + (long long)g.nb0 * (y1 / g.B1);
  n.src_s = (y0 % g.B0) + g.B0 * (y1 % g.B1);
  n.site = (long long)y0 + (long long)g.L0 * y1;
  n.face = face;
  return n;
}

// parts for the fine Wilson level (n_int = 2); arithmetic in CT (FP64, or FP32 for the
// setup of mixed-precision hierarchies), inputs and output FP64
template <typename CT>
__device__ void galerkin_parts_wilson(const Cx<double> *__restrict__ U, double diag, const Cx<double> *__restrict__ V,
                                      const BlockGeo &g, int Nv, long long b, int lane, Cx<CT> *parts) {
  const long long pstride = (long long)Nv * g.Nb;  // parts[dir][k][i]
  for (int i = lane; i < g.Nb; i += 32) {
    const int s = i >> 1, spin = i & 1;
    const long long x = fine_site_of(g, b, s);
    const int x0 = (int)(x % g.L0), x1 = (int)(x / g.L0);
    NbrInfo nb[5];
    Cx<CT> link[5];
    for (int dir = 1; dir <= 4; ++dir) {
      nb[dir] = neighbour_in_blocks(g, x0, x1, dir);
      // +mu: U_x^mu; -mu: U_{x-mu}^mu (conjugated inside hop_scalar)
      link[dir] = cvt<CT, double>((dir == 1)   ? U[2 * x]
                                  : (dir == 2) ? U[2 * nb[2].site]
                                  : (dir == 3) ? U[2 * x + 1]
                                               : U[2 * nb[4].site + 1]);
    }
    for (int k = 0; k < Nv; ++k) {
      Cx<CT> self = (CT)diag * cvt<CT, double>(V[(b * Nv + k) * (long long)g.Nb + i]);
      for (int dir = 1; dir <= 4; ++dir) {
        const Cx<double> *Vs = V + (nb[dir].src_b * Nv + k) * (long long)g.Nb + 2 * nb[dir].src_s;
        const Cx<CT> t = hop_scalar<CT>(dir, link[dir], cvt<CT, double>(Vs[0]), cvt<CT, double>(Vs[1]));
        Cx<CT> comp = spin == 0 ? t : hop_lower<CT>(dir, t);
        comp = (CT)-0.5 * comp;
        if (nb[dir].face) {
          parts[dir * pstride + (long long)k * g.Nb + i] = comp;
        } else {
          self = self + comp;
          parts[dir * pstride + (long long)k * g.Nb + i] = mk((CT)0, (CT)0);
        }
      }
      parts[(long long)k * g.Nb + i] = self;
    }
  }
}

// parts for a coarse stencil level (n_int = N, Y internal [j][dir][col][row]); arithmetic in CT
template <typename CT>
__device__ void galerkin_parts_stencil(const Cx<double> *__restrict__ Y, const Cx<double> *__restrict__ V,
                                       const BlockGeo &g, int Nv, long long b, int lane, Cx<CT> *parts) {
  const int N = g.nint;
  const long long pstride = (long long)Nv * g.Nb;
  for (int i = lane; i < g.Nb; i += 32) {
    const int s = i / N, arow = i - s * N;
    const long long x = fine_site_of(g, b, s);
    const int x0 = (int)(x % g.L0), x1 = (int)(x / g.L0);
    for (int k = 0; k < Nv; ++k) {
      // self term: X(arow, c) W_k(x, c)
      Cx<CT> self = mk((CT)0, (CT)0);
      {
        const Cx<double> *Yd = Y + (x * 5 + 0) * (long long)N * N;
        const Cx<double> *Ws = V + (b * Nv + k) * (long long)g.Nb + (long long)s * N;
        for (int c = 0; c < N; ++c) cmac(self, cvt<CT, double>(Yd[(long long)c * N + arow]), cvt<CT, double>(Ws[c]));
      }
      for (int dir = 1; dir <= 4; ++dir) {
        const NbrInfo nb = neighbour_in_blocks(g, x0, x1, dir);
        const Cx<double> *Yd = Y + (x * 5 + dir) * (long long)N * N;
        const Cx<double> *Ws = V + (nb.src_b * Nv + k) * (long long)g.Nb + (long long)nb.src_s * N;
        Cx<CT> comp = mk((CT)0, (CT)0);
        for (int c = 0; c < N; ++c) cmac(comp, cvt<CT, double>(Yd[(long long)c * N + arow]), cvt<CT, double>(Ws[c]));
        if (nb.face) {
          parts[dir * pstride + (long long)k * g.Nb + i] = comp;
        } else {
          self = self + comp;
          parts[dir * pstride + (long long)k * g.Nb + i] = mk((CT)0, (CT)0);
        }
      }
      parts[(long long)k * g.Nb + i] = self;
    }
  }
}

template <bool WILSON, typename CT>
__global__ void galerkin_kernel(const Cx<double> *__restrict__ U_or_Y, double diag, const Cx<double> *__restrict__ V,
                                Cx<double> *__restrict__ Yc, BlockGeo g, int Nv) {
  extern __shared__ __align__(16) unsigned char smem_gal_raw[];
  Cx<CT> *smem_gal = reinterpret_cast<Cx<CT> *>(smem_gal_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long b = blockIdx.x * (long long)(blockDim.x >> 5) + warp;
  if (b >= g.nblocks) return;
  Cx<CT> *parts = smem_gal + (long long)warp * 5 * Nv * g.Nb;
  if (WILSON)
    galerkin_parts_wilson<CT>(U_or_Y, diag, V, g, Nv, b, lane, parts);
  else
    galerkin_parts_stencil<CT>(U_or_Y, V, g, Nv, b, lane, parts);
  __syncwarp();
  const long long pstride = (long long)Nv * g.Nb;
  const Cx<double> *Vb = V + b * (long long)Nv * g.Nb;
  for (int o = lane; o < 5 * Nv * Nv; o += 32) {
    const int dir = o / (Nv * Nv), rem = o - dir * Nv * Nv, k = rem / Nv, kp = rem - k * Nv;
    Cx<CT> acc = mk((CT)0, (CT)0);
    const Cx<CT> *p = parts + dir * pstride + (long long)k * g.Nb;
    const Cx<double> *vk = Vb + (long long)kp * g.Nb;
    for (int i = 0; i < g.Nb; ++i) cmac_conj(acc, cvt<CT, double>(vk[i]), p[i]);
    // internal layout [b][dir][col = k][row = kp]
    Yc[((b * 5 + dir) * Nv + k) * (long long)Nv + kp] = cvt<double, CT>(acc);
  }
}

__global__ void coarse_to_canonical_kernel(const Cx<double> *__restrict__ Yi, Cx<double> *__restrict__ Yc,
                                           long long nsites, int N) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = 5LL * N * N;
  if (t >= nsites * per) return;
  const long long jd = t / ((long long)N * N);
  const int rem = (int)(t - jd * N * N), row = rem / N, col = rem - row * N;
  Yc[t] = Yi[jd * N * N + (long long)col * N + row];
}

__global__ void prolongator_to_canonical_kernel(const Cx<double> *__restrict__ V, Cx<double> *__restrict__ out,
                                                BlockGeo g, int Nv) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nfine = g.nblocks * (long long)g.Nb;
  if (t >= nfine * Nv) return;
  const long long b = t / ((long long)Nv * g.Nb);
  const long long rem = t - b * Nv * (long long)g.Nb;
  const int k = (int)(rem / g.Nb), i = (int)(rem - (long long)k * g.Nb);
  const int s = i / g.nint, a = i - s * g.nint;
  out[(long long)k * nfine + fine_site_of(g, b, s) * g.nint + a] = V[t];
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies
// (0xD2511F53, 0xCD9E8D57) with a Weyl key schedule (0x9E3779B9, 0xBB67AE85),
// then Box-Muller on two 53-bit uniforms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__global__ void gaussian_kernel(Cx<double> *out, long long n, unsigned long long seed, int k, int level) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c[4] = {(uint32_t)(unsigned long long)i, (uint32_t)((unsigned long long)i >> 32), (uint32_t)k,
                   (uint32_t)level};
  philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const unsigned long long a = ((((unsigned long long)c[1]) << 32) | c[0]) >> 11;
  const unsigned long long bb = ((((unsigned long long)c[3]) << 32) | c[2]) >> 11;
  const double u1 = (double)(a + 1) * 0x1.0p-53, u2 = (double)bb * 0x1.0p-53;
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586476925286766559 * u2;
  out[i] = mk(rad * cos(ang), rad * sin(ang));
}

// ---------------------------------------------------------------------------
template <typename R>
void launch_restrict(const Cx<R> *V, const Cx<R> *fine, Cx<R> *coarse, BlockGeo bg, int Nv, cudaStream_t s,
                     int nvec) {
  constexpr int CPV = Vec16<R>::cpv;
  if (Nv == 8 && bg.nint % CPV == 0 && bg.Nb / CPV == 32 / CPV) {
    // streaming form: 32 dofs per block (4 x 4 sites x 2 spins, or 2 x 2 sites x 8)
    constexpr int BPC = 4 * CPV;  // 16 KB tiles in FP32, 32 KB in FP64
    const dim3 grid((unsigned int)((bg.nblocks + BPC - 1) / BPC), nvec);
    restrict8_stream_kernel<R, BPC, 32 / CPV><<<grid, 256, 0, s>>>(V, fine, coarse, bg);
    MG_LAUNCHED();
    return;
  }
  const int threads = 128;
  const dim3 grid(grid_for(bg.nblocks * 32, threads), nvec);
  if (Nv <= 8)
    restrict_kernel<R, 8><<<grid, threads, 0, s>>>(V, fine, coarse, bg, Nv);
  else if (Nv <= 16)
    restrict_kernel<R, 16><<<grid, threads, 0, s>>>(V, fine, coarse, bg, Nv);
  else if (Nv <= kMaxNv)
    restrict_kernel<R, kMaxNv><<<grid, threads, 0, s>>>(V, fine, coarse, bg, Nv);
  else
    fail(MG_ERR_UNSUPPORTED, "restrict: Nv > 32");
  MG_LAUNCHED();
}

template <typename R>
void launch_prolong_add(const Cx<R> *V, const Cx<R> *coarse, Cx<R> *fine, BlockGeo bg, int Nv, cudaStream_t s,
                        int nvec) {
  const int threads = 128;
  prolong_add_kernel<R><<<dim3(grid_for(bg.nblocks * 32, threads), nvec), threads, 0, s>>>(V, coarse, fine, bg, Nv);
  MG_LAUNCHED();
}

static int warps_for_smem(size_t per_warp, size_t limit) {
  int w = (int)(limit / per_warp);
  if (w > 4) w = 4;
  return w;
}

void launch_block_mgs(const Cx<double> *vecs, long long vec_stride, Cx<double> *V, BlockGeo bg, int Nv,
                      double *min_norm_dev, cudaStream_t s) {
  const size_t per_warp = (size_t)Nv * bg.Nb * sizeof(Cx<double>);
  const size_t limit = 200 * 1024;
  const int warps = warps_for_smem(per_warp, limit);
  if (warps < 1) fail(MG_ERR_UNSUPPORTED, "block Gram-Schmidt: block too large for shared memory");
  const size_t smem = per_warp * warps;
  MG_CUDA(cudaFuncSetAttribute(block_mgs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned int grid = (unsigned int)((bg.nblocks + warps - 1) / warps);
  block_mgs_kernel<<<grid, 32 * warps, smem, s>>>(vecs, vec_stride, V, bg, Nv, min_norm_dev);
  MG_LAUNCHED();
}

template <bool WILSON, typename CT>
static void launch_galerkin_impl(const Cx<double> *UY, double diag, const Cx<double> *V, Cx<double> *Yc, BlockGeo bg,
                                 int Nv, cudaStream_t s) {
  const size_t per_warp = (size_t)5 * Nv * bg.Nb * sizeof(Cx<CT>);
  const int warps = warps_for_smem(per_warp, 200 * 1024);
  if (warps < 1) fail(MG_ERR_UNSUPPORTED, "Galerkin build: block too large for shared memory");
  const size_t smem = per_warp * warps;
  MG_CUDA(cudaFuncSetAttribute(galerkin_kernel<WILSON, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned int grid = (unsigned int)((bg.nblocks + warps - 1) / warps);
  galerkin_kernel<WILSON, CT><<<grid, 32 * warps, smem, s>>>(UY, diag, V, Yc, bg, Nv);
  MG_LAUNCHED();
}

void launch_galerkin_wilson(const Cx<double> *U, double diag, const Cx<double> *V, Cx<double> *Yc, BlockGeo bg,
                            int Nv, cudaStream_t s, bool fp32_arith) {
  if (bg.nint != 2) fail(MG_ERR_INVALID_ARG, "Galerkin (Wilson): n_int must be 2");
  if (fp32_arith)
    launch_galerkin_impl<true, float>(U, diag, V, Yc, bg, Nv, s);
  else
    launch_galerkin_impl<true, double>(U, diag, V, Yc, bg, Nv, s);
}

void launch_galerkin_stencil(const Cx<double> *Y, const Cx<double> *V, Cx<double> *Yc, BlockGeo bg, int Nv,
                             cudaStream_t s, bool fp32_arith) {
  if (fp32_arith)
    launch_galerkin_impl<false, float>(Y, 0.0, V, Yc, bg, Nv, s);
  else
    launch_galerkin_impl<false, double>(Y, 0.0, V, Yc, bg, Nv, s);
}

void launch_coarse_to_canonical(const Cx<double> *Yi, Cx<double> *Yc, long long nsites, int N, cudaStream_t s) {
  coarse_to_canonical_kernel<<<grid_for(nsites * 5LL * N * N, 256), 256, 0, s>>>(Yi, Yc, nsites, N);
  MG_LAUNCHED();
}

void launch_prolongator_to_canonical(const Cx<double> *V, Cx<double> *out, BlockGeo bg, int Nv, cudaStream_t s) {
  prolongator_to_canonical_kernel<<<grid_for(bg.nblocks * (long long)bg.Nb * Nv, 256), 256, 0, s>>>(V, out, bg, Nv);
  MG_LAUNCHED();
}

void launch_gaussian(Cx<double> *out, long long n, unsigned long long seed, int k, int level, cudaStream_t s) {
  gaussian_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, seed, k, level);
  MG_LAUNCHED();
}

template void launch_restrict<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, BlockGeo, int,
                                      cudaStream_t, int);
template void launch_restrict<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, BlockGeo, int, cudaStream_t,
                                     int);
template void launch_prolong_add<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, BlockGeo, int,
                                         cudaStream_t, int);
template void launch_prolong_add<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, BlockGeo, int,
                                        cudaStream_t, int);

}  // namespace mg
