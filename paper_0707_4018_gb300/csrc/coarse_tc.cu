// Coarse stencil apply on tensor cores for many right-hand sides (N = 8 coarse
// levels; paper: the coarse operator P^dagger D P of Eq. Galerkin applied to a block
// of vectors, as in the setup's many-vector passes and multi-RHS solves).
//
// Per coarse site and direction, the 8 x 8 complex block Y acting on R complex
// vectors is a real product: [y_re; y_im] = [[Y_re, -Y_im], [Y_im, Y_re]] [x_re; x_im],
// a 16 x 16 real matrix times a 16 x R real matrix. One warp takes one site and 8
// right-hand sides: the 5 directions are 5 mma.sync.m16n8k16 (BF16 operands, FP32
// accumulation) into one 16 x 8 accumulator. tcgen05 does not fit: its smallest tile
// is M = 64 rows, and every site has its own A and its own B (the neighbours'
// vectors), so sites cannot be stacked into one larger product. BF16 rather than FP16:
// it keeps FP32's exponent range, so the small residuals late in a solve need no
// rescaling.
//
// Operator layout (packed once per level): for site j, direction d and lane l
// (g = l / 4, t = l % 4) one 8-byte word holds Y[g][2t], Y[g][2t+1] as (re, re) and
// (im, im) BF16 pairs: exactly the lane's A fragment registers 0 and 1; registers 2 and
// 3 are the sign-flipped register 1 and a copy of register 0. 256 bytes per (site,
// direction), the size of the complex block in 16-bit storage.
#include <cuda_bf16.h>

#include <string>

#include "kernels.h"

namespace mg {

__device__ __forceinline__ unsigned int pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low 16 bits), .y = hi
  return *reinterpret_cast<const unsigned int *>(&v);
}

// Ypk[(j * 5 + d) * 32 + l] from the internal FP32 stencil Y[j][d][col][row]
__global__ void pack_coarse_bf16_kernel(const Cx<float> *__restrict__ Y, uint2 *__restrict__ Ypk, long long nsites) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // (j, d, l)
  if (q >= nsites * 5 * 32) return;
  const int l = (int)(q & 31);
  const long long jd = q >> 5;
  const int g = l >> 2, t = l & 3;
  const Cx<float> y0 = Y[jd * 64 + (2 * t) * 8 + g], y1 = Y[jd * 64 + (2 * t + 1) * 8 + g];
  Ypk[q] = make_uint2(pack_bf16x2(y0.re, y1.re), pack_bf16x2(y0.im, y1.im));
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], unsigned int a0, unsigned int a1, unsigned int a2,
                                               unsigned int a3, unsigned int b0, unsigned int b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// out_n = a (A + shift_n) in_n + c b_n for the nvec vectors (stride ldv), item w = (site j,
// group of 8 vectors), j = w / tiles
__device__ __forceinline__ void tc_item(long long w, int lane, const uint2 *__restrict__ Ypk,
                                        const Cx<float> *__restrict__ in, Cx<float> *__restrict__ out, int L0, int L1,
                                        long long ldv, int nvec, int tiles, const Cx<float> *b, float a, float c,
                                        const double *shift) {
  const int g = lane >> 2, t = lane & 3;
  const long long j = w / tiles;
  const int n0 = (int)(w - j * tiles) * 8;
  const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
  const long long rowo = (long long)x1 * L0;
  const long long nbr[5] = {j, rowo + (x0 + 1 == L0 ? 0 : x0 + 1), rowo + (x0 == 0 ? L0 - 1 : x0 - 1),
                            (x1 + 1 == L1 ? 0 : rowo + L0) + x0,
                            (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0};
  // B fragment: this lane's vector n = n0 + g, dofs 2t and 2t + 1 of the neighbour site
  const int nb = n0 + g;
  const bool bcol = nb < nvec;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const uint2 ya = Ypk[(j * 5 + d) * 32 + lane];
    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (bcol) xv = *reinterpret_cast<const float4 *>(in + nb * ldv + nbr[d] * 8 + 2 * t);
    const unsigned int b0 = pack_bf16x2(xv.x, xv.z), b1 = pack_bf16x2(xv.y, xv.w);
    mma_bf16_16816(acc, ya.x, ya.y, ya.y ^ 0x80008000u, ya.x, b0, b1);
  }
  // C fragment: y[n0 + 2t][g] = (acc0, acc2), y[n0 + 2t + 1][g] = (acc1, acc3)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int n = n0 + 2 * t + h;
    if (n >= nvec) continue;
    const long long e = n * ldv + j * 8 + g;
    float re = h ? acc[1] : acc[0], im = h ? acc[3] : acc[2];
    if (shift != nullptr) {
      const float sv = (float)shift[n];
      const Cx<float> xs = in[e];
      re = fmaf(sv, xs.re, re);
      im = fmaf(sv, xs.im, im);
    }
    Cx<float> o = mk(a * re, a * im);
    if (b != nullptr) {
      const Cx<float> bb = b[e];
      o = mk(o.re + c * bb.re, o.im + c * bb.im);
    }
    out[e] = o;
  }
}

// one warp per SPW consecutive items; the launch shape (warps per CTA, SPW) changes
// neither the arithmetic nor its order
template <int SPW>
__global__ void __launch_bounds__(256) coarse_apply_tc_kernel(const uint2 *__restrict__ Ypk,
                                                              const Cx<float> *__restrict__ in,
                                                              Cx<float> *__restrict__ out, int L0, int L1,
                                                              long long ldv, int nvec, const Cx<float> *b,
                                                              float a, float c, const double *shift) {
  const long long w0 = ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5) * SPW;
  const int lane = threadIdx.x & 31;
  const int tiles = (nvec + 7) >> 3;
  const long long items = (long long)L0 * L1 * tiles;
#pragma unroll
  for (int q = 0; q < SPW; ++q)
    if (w0 + q < items) tc_item(w0 + q, lane, Ypk, in, out, L0, L1, ldv, nvec, tiles, b, a, c, shift);
}

void launch_pack_coarse_bf16(const Cx<float> *Y, uint2 *Ypk, long long nsites, cudaStream_t s) {
  pack_coarse_bf16_kernel<<<grid_for(nsites * 5 * 32, 256), 256, 0, s>>>(Y, Ypk, nsites);
  MG_LAUNCHED();
}

// launch shapes: (warps per CTA, items per warp)
static const int kTcShapes[6][2] = {{8, 1}, {4, 1}, {2, 1}, {8, 2}, {4, 2}, {2, 2}};

static void tc_launch(int shape, const uint2 *Ypk, const Cx<float> *in, Cx<float> *out, Geo2 g, int nvec,
                      const Cx<float> *b, double a, double c, const double *shift, cudaStream_t s) {
  const int wpc = kTcShapes[shape][0], spw = kTcShapes[shape][1];
  const long long items = g.nsites * ((nvec + 7) / 8);
  const long long warps = (items + spw - 1) / spw;
  const unsigned int grid = grid_for(warps, wpc);
  if (spw == 1)
    coarse_apply_tc_kernel<1><<<grid, 32 * wpc, 0, s>>>(Ypk, in, out, g.L0, g.L1, g.nsites * 8, nvec, b, (float)a,
                                                        (float)c, shift);
  else
    coarse_apply_tc_kernel<2><<<grid, 32 * wpc, 0, s>>>(Ypk, in, out, g.L0, g.L1, g.nsites * 8, nvec, b, (float)a,
                                                        (float)c, shift);
  MG_LAUNCHED();
}

void launch_coarse_apply_tc(const uint2 *Ypk, const Cx<float> *in, Cx<float> *out, Geo2 g, int nvec,
                            const Cx<float> *b, double a, double c, const double *shift, cudaStream_t s) {
  if (nvec < 1) return;
  // the launch shape is picked once per problem shape by timing all six (the result does not
  // depend on it)
  const std::string key = "coarse_apply_tc/" + std::to_string(g.L0) + "x" + std::to_string(g.L1) + "/nvec" +
                          std::to_string(nvec);
  const int shape = autotune_choose(key, 6, [&](int v) { tc_launch(v, Ypk, in, out, g, nvec, b, a, c, shift, s); }, s);
  tc_launch(shape, Ypk, in, out, g, nvec, b, a, c, shift, s);
}

// ===========================================================================
// 4d coarse level (N = 48, 9 directions). The complex block Y = A + i B (48 x 48)
// acts on x = xr + i xi as the real product [[A, -B], [B, A]] [xr; xi]; with 16 x 16
// tiles (48 = 3 x 16) every tile of that real matrix is a tile of A, of B or of -B.
// Only the A and B tiles are packed (BF16, A-fragment order, 512 B per tile); -B is
// B with the sign bits flipped. A warp takes one site, 16 complex output rows (row
// tile tm) and 8 vectors: for every direction and column tile tk it loads the A and
// B fragments once and issues 4 mma.sync.m16n8k16 (A xr, -B xi into the real rows;
// B xr, A xi into the imaginary rows): 108 per warp, FP32 accumulation.
// ===========================================================================

// Ypk4[((j * 9 + dir) * 2 + q) * 9 + tm * 3 + tk][lane] (uint4), q = 0: A = Re Y, 1: B = Im Y,
// from the FP64 internal stencil Y[j][dir][col][row]; LO: the BF16 rounding of what the BF16
// value leaves (y - bf16(y)), so that hi + lo carries about 16 significant bits
template <bool LO>
__global__ void pack_coarse4_bf16_kernel(const Cx<double> *__restrict__ Y, uint4 *__restrict__ Ypk, long long nsites) {
  const long long qi = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // (j, dir, q, tile, lane)
  if (qi >= nsites * 9 * 2 * 9 * 32) return;
  const int lane = (int)(qi & 31);
  long long r = qi >> 5;
  const int tile = (int)(r % 9);
  r /= 9;
  const int q = (int)(r & 1);
  const long long jd = r >> 1;  // j * 9 + dir
  const int tm = tile / 3, tk = tile - tm * 3, g = lane >> 2, t = lane & 3;
  const Cx<double> *Yb = Y + jd * 48 * 48;
  auto el = [&](int row, int col) {  // element (row, col) of A or B
    const Cx<double> y = Yb[(long long)(16 * tk + col) * 48 + 16 * tm + row];
    const double v = q == 0 ? y.re : y.im;
    const float f = (float)v;  // the hi part is the BF16 rounding of this float, as in the kernel above
    return LO ? (float)(v - (double)__bfloat162float(__float2bfloat16_rn(f))) : f;
  };
  uint4 out;
  out.x = pack_bf16x2(el(g, 2 * t), el(g, 2 * t + 1));
  out.y = pack_bf16x2(el(g + 8, 2 * t), el(g + 8, 2 * t + 1));
  out.z = pack_bf16x2(el(g, 2 * t + 8), el(g, 2 * t + 9));
  out.w = pack_bf16x2(el(g + 8, 2 * t + 8), el(g + 8, 2 * t + 9));
  Ypk[qi] = out;
}

// x = hi + lo for a pair of floats: hi their BF16 rounding, lo the BF16 rounding of the rest
__device__ __forceinline__ void split_bf16x2(float a, float b, unsigned int &hi, unsigned int &lo) {
  hi = pack_bf16x2(a, b);
  lo = pack_bf16x2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}

// out_n = A_c in_n with one warp per (site, row tile, group of 8 vectors): the form taken for
// SPLIT 0 and 1, where it beats the per-site form below (more CTAs in flight; 19.6 against
// 25.9 us for SPLIT 0 at 512 sites x 12 vectors). The operands as in the per-site form.
template <int SPLIT>
__global__ void __launch_bounds__(256) coarse4_apply_tc_warp_kernel(const uint4 *__restrict__ Ypk,
                                                               const uint4 *__restrict__ Ypklo,
                                                               const Cx<float> *__restrict__ in,
                                                               Cx<float> *__restrict__ out, int nb0, int nb1, int nb2,
                                                               int nb3, long long ldv, int nvec) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long nsites = (long long)nb0 * nb1 * nb2 * nb3;
  const int tiles = (nvec + 7) >> 3;
  if (w >= nsites * 3 * tiles) return;  // whole warps
  const long long j = w / (3 * tiles);
  const int rem = (int)(w - j * 3 * tiles), tm = rem / tiles, n0 = (rem - tm * tiles) * 8;
  const int nb[4] = {nb0, nb1, nb2, nb3};
  int jc[4];
  {
    long long q = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = (int)(q % nb[mu]);
      q /= nb[mu];
    }
  }
  const int nv = n0 + g;  // this lane's vector in the B fragments
  const bool bcol = nv < nvec;
  float cre[4] = {0.f, 0.f, 0.f, 0.f}, cim[4] = {0.f, 0.f, 0.f, 0.f};
  for (int dir = 0; dir < 9; ++dir) {
    long long src = j;
    if (dir != 0) {
      const int mu = (dir - 1) >> 1;
      int cc[4] = {jc[0], jc[1], jc[2], jc[3]};
      cc[mu] = ((dir - 1) & 1) == 0 ? (cc[mu] + 1) % nb[mu] : (cc[mu] + nb[mu] - 1) % nb[mu];
      src = cc[0] + (long long)nb[0] * (cc[1] + (long long)nb[1] * (cc[2] + (long long)nb[2] * cc[3]));
    }
    const Cx<float> *xs = in + nv * ldv + src * 48;
    const uint4 *Yd = Ypk + (j * 9 + dir) * 2 * 9 * 32;
#pragma unroll
    for (int tk = 0; tk < 3; ++tk) {
      float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;  // x[16 tk + 2t .. +1], x[16 tk + 2t + 8 .. +9]
      if (bcol) {
        lo = *reinterpret_cast<const float4 *>(xs + 16 * tk + 2 * t);
        hi = *reinterpret_cast<const float4 *>(xs + 16 * tk + 2 * t + 8);
      }
      unsigned int r0, r1, i0, i1, r0l = 0u, r1l = 0u, i0l = 0u, i1l = 0u;  // xr, xi fragments (hi, lo)
      if (SPLIT == 0) {
        r0 = pack_bf16x2(lo.x, lo.z);
        r1 = pack_bf16x2(hi.x, hi.z);
        i0 = pack_bf16x2(lo.y, lo.w);
        i1 = pack_bf16x2(hi.y, hi.w);
      } else {
        split_bf16x2(lo.x, lo.z, r0, r0l);
        split_bf16x2(hi.x, hi.z, r1, r1l);
        split_bf16x2(lo.y, lo.w, i0, i0l);
        split_bf16x2(hi.y, hi.w, i1, i1l);
      }
      const int fi = (tm * 3 + tk) * 32 + lane;
      const uint4 fa = Yd[fi], fb = Yd[9 * 32 + fi];
      const unsigned int s = 0x80008000u;
      mma_bf16_16816(cre, fa.x, fa.y, fa.z, fa.w, r0, r1);                  // + A xr
      mma_bf16_16816(cre, fb.x ^ s, fb.y ^ s, fb.z ^ s, fb.w ^ s, i0, i1);  // - B xi
      mma_bf16_16816(cim, fb.x, fb.y, fb.z, fb.w, r0, r1);                  // + B xr
      mma_bf16_16816(cim, fa.x, fa.y, fa.z, fa.w, i0, i1);                  // + A xi
      if (SPLIT >= 1) {
        mma_bf16_16816(cre, fa.x, fa.y, fa.z, fa.w, r0l, r1l);
        mma_bf16_16816(cre, fb.x ^ s, fb.y ^ s, fb.z ^ s, fb.w ^ s, i0l, i1l);
        mma_bf16_16816(cim, fb.x, fb.y, fb.z, fb.w, r0l, r1l);
        mma_bf16_16816(cim, fa.x, fa.y, fa.z, fa.w, i0l, i1l);
      }
      if (SPLIT == 2) {
        const uint4 *Yl = Ypklo + (j * 9 + dir) * 2 * 9 * 32;
        const uint4 ga = Yl[fi], gb = Yl[9 * 32 + fi];
        mma_bf16_16816(cre, ga.x, ga.y, ga.z, ga.w, r0, r1);
        mma_bf16_16816(cre, gb.x ^ s, gb.y ^ s, gb.z ^ s, gb.w ^ s, i0, i1);
        mma_bf16_16816(cim, gb.x, gb.y, gb.z, gb.w, r0, r1);
        mma_bf16_16816(cim, ga.x, ga.y, ga.z, ga.w, i0, i1);
      }
    }
  }
  // C fragment: rows g, g + 8 of the tile (complex rows 16 tm + g, + 8), vectors n0 + 2t, + 1
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int n = n0 + 2 * t + h;
    if (n >= nvec) continue;
    Cx<float> *o = out + n * ldv + j * 48 + 16 * tm;
    o[g] = mk(cre[h], cim[h]);
    o[g + 8] = mk(cre[2 + h], cim[2 + h]);
  }
}

// out_n = A_c in_n for nvec vectors (stride ldv = nsites * 48). A CTA takes one site and up to
// 16 vectors (two 8-vector groups, blockIdx.y selects the pair); its 9 warps are (row tile tm,
// direction group dg): warp (tm, dg) applies the directions 3 dg .. 3 dg + 2 of row tile tm to
// both vector groups, so every operator fragment is loaded once per 16 vectors, and the three
// direction groups' partial sums meet in shared memory. SPLIT = 0: operator and vectors in
// BF16 (4 MMAs per tile pair and group); 1: vectors as BF16 hi + lo (8 MMAs); 2: operator split
// as well (Ypklo), the product hi hi + hi lo + lo hi (12 MMAs): about 2^-16 of sum |Y| |x|
// instead of 2^-8
constexpr int kTcWarps = 9;

template <int SPLIT>
__global__ void __launch_bounds__(32 * kTcWarps) coarse4_apply_tc_kernel(const uint4 *__restrict__ Ypk,
                                                                        const uint4 *__restrict__ Ypklo,
                                                                        const Cx<float> *__restrict__ in,
                                                                        Cx<float> *__restrict__ out, int nb0,
                                                                        int nb1, int nb2, int nb3, long long ldv,
                                                                        int nvec) {
  __shared__ float part[2][3][32][16];  // partial sums of direction groups 1 and 2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int tm = warp % 3, dg = warp / 3;
  const long long j = blockIdx.x;
  const int nbase = blockIdx.y * 16;
  const int nb[4] = {nb0, nb1, nb2, nb3};
  int jc[4];
  {
    long long q = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = (int)(q % nb[mu]);
      q /= nb[mu];
    }
  }
  const bool grp1 = nbase + 8 < nvec;  // the second vector group exists
  float acc[2][8];                       // [group][cre 0..3, cim 0..3]
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[q][i] = 0.f;
  const unsigned int s = 0x80008000u;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    const int dir = 3 * dg + dd;
    long long src = j;
    if (dir != 0) {
      const int mu = (dir - 1) >> 1;
      int cc[4] = {jc[0], jc[1], jc[2], jc[3]};
      cc[mu] = ((dir - 1) & 1) == 0 ? (cc[mu] + 1) % nb[mu] : (cc[mu] + nb[mu] - 1) % nb[mu];
      src = cc[0] + (long long)nb[0] * (cc[1] + (long long)nb[1] * (cc[2] + (long long)nb[2] * cc[3]));
    }
    const uint4 *Yd = Ypk + (j * 9 + dir) * 2 * 9 * 32;
    const uint4 *Yl = SPLIT == 2 ? Ypklo + (j * 9 + dir) * 2 * 9 * 32 : nullptr;
#pragma unroll
    for (int tk = 0; tk < 3; ++tk) {
      const int fi = (tm * 3 + tk) * 32 + lane;
      const uint4 fa = Yd[fi], fb = Yd[9 * 32 + fi];
      uint4 ga = make_uint4(0u, 0u, 0u, 0u), gb = ga;
      if (SPLIT == 2) {
        ga = Yl[fi];
        gb = Yl[9 * 32 + fi];
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !grp1) break;
        const int nv = nbase + 8 * q + g;  // this lane's vector in the B fragments
        float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;  // x[16 tk + 2t .. +1], x[16 tk + 2t + 8 .. +9]
        if (nv < nvec) {
          const Cx<float> *xs = in + nv * ldv + src * 48;
          lo = *reinterpret_cast<const float4 *>(xs + 16 * tk + 2 * t);
          hi = *reinterpret_cast<const float4 *>(xs + 16 * tk + 2 * t + 8);
        }
        unsigned int r0, r1, i0, i1, r0l = 0u, r1l = 0u, i0l = 0u, i1l = 0u;  // xr, xi fragments (hi, lo)
        if (SPLIT == 0) {
          r0 = pack_bf16x2(lo.x, lo.z);
          r1 = pack_bf16x2(hi.x, hi.z);
          i0 = pack_bf16x2(lo.y, lo.w);
          i1 = pack_bf16x2(hi.y, hi.w);
        } else {
          split_bf16x2(lo.x, lo.z, r0, r0l);
          split_bf16x2(hi.x, hi.z, r1, r1l);
          split_bf16x2(lo.y, lo.w, i0, i0l);
          split_bf16x2(hi.y, hi.w, i1, i1l);
        }
        float(&cre)[4] = *reinterpret_cast<float(*)[4]>(&acc[q][0]);
        float(&cim)[4] = *reinterpret_cast<float(*)[4]>(&acc[q][4]);
        mma_bf16_16816(cre, fa.x, fa.y, fa.z, fa.w, r0, r1);                  // + A xr
        mma_bf16_16816(cre, fb.x ^ s, fb.y ^ s, fb.z ^ s, fb.w ^ s, i0, i1);  // - B xi
        mma_bf16_16816(cim, fb.x, fb.y, fb.z, fb.w, r0, r1);                  // + B xr
        mma_bf16_16816(cim, fa.x, fa.y, fa.z, fa.w, i0, i1);                  // + A xi
        if (SPLIT >= 1) {
          mma_bf16_16816(cre, fa.x, fa.y, fa.z, fa.w, r0l, r1l);
          mma_bf16_16816(cre, fb.x ^ s, fb.y ^ s, fb.z ^ s, fb.w ^ s, i0l, i1l);
          mma_bf16_16816(cim, fb.x, fb.y, fb.z, fb.w, r0l, r1l);
          mma_bf16_16816(cim, fa.x, fa.y, fa.z, fa.w, i0l, i1l);
        }
        if (SPLIT == 2) {
          mma_bf16_16816(cre, ga.x, ga.y, ga.z, ga.w, r0, r1);
          mma_bf16_16816(cre, gb.x ^ s, gb.y ^ s, gb.z ^ s, gb.w ^ s, i0, i1);
          mma_bf16_16816(cim, gb.x, gb.y, gb.z, gb.w, r0, r1);
          mma_bf16_16816(cim, ga.x, ga.y, ga.z, ga.w, i0, i1);
        }
      }
    }
  }
  if (dg > 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < 8; ++i) part[dg - 1][tm][lane][8 * q + i] = acc[q][i];
  }
  __syncthreads();
  if (dg != 0) return;
  // C fragment: rows g, g + 8 of the tile (complex rows 16 tm + g, + 8), vectors n0 + 2t, + 1
#pragma unroll
  for (int q = 0; q < 2; ++q) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[q][i] += part[0][tm][lane][8 * q + i] + part[1][tm][lane][8 * q + i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = nbase + 8 * q + 2 * t + h;
      if (n >= nvec) continue;
      Cx<float> *o = out + n * ldv + j * 48 + 16 * tm;
      o[g] = mk(acc[q][h], acc[q][4 + h]);
      o[g + 8] = mk(acc[q][2 + h], acc[q][4 + 2 + h]);
    }
  }
}

void launch_pack_coarse4_bf16(const Cx<double> *Y, uint4 *Ypk, long long nsites, cudaStream_t s, bool lo) {
  if (lo)
    pack_coarse4_bf16_kernel<true><<<grid_for(nsites * 9 * 2 * 9 * 32, 256), 256, 0, s>>>(Y, Ypk, nsites);
  else
    pack_coarse4_bf16_kernel<false><<<grid_for(nsites * 9 * 2 * 9 * 32, 256), 256, 0, s>>>(Y, Ypk, nsites);
  MG_LAUNCHED();
}

void launch_coarse4_apply_tc(const uint4 *Ypk, const Cx<float> *in, Cx<float> *out, const int nb[4], int nvec,
                             cudaStream_t s, int split, const uint4 *Ypklo) {
  if (nvec < 1) return;
  if (split < 0 || split > 2 || (split == 2 && Ypklo == nullptr))
    fail(MG_ERR_INVALID_ARG, "tensor-core apply: split must be 0, 1 or 2 (2 needs the low BF16 part)");
  const long long nsites = (long long)nb[0] * nb[1] * nb[2] * nb[3];
  if (split < 2) {  // a warp per (site, row tile, 8 vectors)
    const long long warps = nsites * 3 * ((nvec + 7) / 8);
    const unsigned int grid = grid_for(warps * 32, 256);
    if (split == 0)
      coarse4_apply_tc_warp_kernel<0><<<grid, 256, 0, s>>>(Ypk, Ypklo, in, out, nb[0], nb[1], nb[2], nb[3],
                                                           nsites * 48, nvec);
    else
      coarse4_apply_tc_warp_kernel<1><<<grid, 256, 0, s>>>(Ypk, Ypklo, in, out, nb[0], nb[1], nb[2], nb[3],
                                                           nsites * 48, nvec);
  } else {  // a CTA per (site, 16 vectors)
    const dim3 grid((unsigned int)nsites, (unsigned int)((nvec + 15) / 16));
    coarse4_apply_tc_kernel<2><<<grid, 32 * kTcWarps, 0, s>>>(Ypk, Ypklo, in, out, nb[0], nb[1], nb[2], nb[3],
                                                              nsites * 48, nvec);
  }
  MG_LAUNCHED();
}

}  // namespace mg
