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

}  // namespace mg
