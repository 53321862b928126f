// Fine Wilson operator on a 4d SU(3) lattice (paper, definition of D following
// Eq. 1, with four spins, three colours and the DeGrand-Rossi gamma basis;
// diagonal d + m = 4 + m, periodic boundaries).
//
// DeGrand-Rossi: every gamma_mu = [[0, A_mu], [A_mu^dagger, 0]] in 2 x 2 spin
// blocks with A_mu unitary, so (1 -+ gamma_mu) has rank two and is fixed by its
// upper half:
//   (1 - gamma_mu) psi = (h, -A_mu^dagger h),  h = psi_up - A_mu psi_dn
//   (1 + gamma_mu) psi = (h,  A_mu^dagger h),  h = psi_up + A_mu psi_dn
// with psi_up = (psi_0, psi_1), psi_dn = (psi_2, psi_3). A hop therefore
// projects the neighbour's spinor to the half spinor h (2 spins x 3 colours),
// applies the colour link to it (18 complex multiply-adds instead of 36) and
// rebuilds the lower spins from the upper ones. The A_mu are
//   mu = 0: [[0, i], [i, 0]]    mu = 1: [[0, -1], [1, 0]]
//   mu = 2: [[i, 0], [0, -i]]   mu = 3: [[1, 0], [0, 1]].
//
// Layouts (site-major, the library's boundary layout): psi[x][s][c] (12 complex,
// 96 B in FP32), U[x][mu][a][b] (4 x 9 complex; U_x^mu links x to x + mu-hat).
// A warp computes 32 consecutive sites, one per lane, hop after hop; the
// neighbours' spinors and the hop's links are gathered by the whole warp in
// contiguous pieces through shared memory. The backward links are the
// neighbours' forward links, so an apply streams psi, U and out from HBM about
// once: 60 complex per site = 480 B (FP32) / 960 B (FP64). The neighbour
// spinors (8 per site) and links (2 reads each) come from L2, which makes the
// on-chip traffic about 3x the HBM traffic.
#include "kernels.h"
#include "wilson4d.cuh"

namespace mg {

namespace {

// ---------------------------------------------------------------------------
// Warp-cooperative staging. A warp owns 32 consecutive sites. The 96-B spinors
// and 72-B links of its 32 neighbours in one direction are gathered by the
// whole warp in 16-B (spinor) and 8-B (link) pieces, consecutive lanes taking
// consecutive pieces, so every load instruction reads contiguous memory
// wherever the 32 neighbours are consecutive sites (everywhere except at the
// periodic wrap of direction mu). Each thread then reads its own record from
// shared memory. Strides: a staged FP32 spinor takes 7 float4 (112 B), a staged
// FP64 spinor 13 double2 (208 B) and a link 9 complex: conflict-free reads.
// ---------------------------------------------------------------------------
template <typename R>
struct Stage;
template <>
struct Stage<float> {
  using V = float4;                 // one gathered spinor piece (2 complex)
  static constexpr int PIECES = 6;  // pieces per spinor
  static constexpr int STRIDE = 7;  // staged spinor stride in pieces
};
template <>
struct Stage<double> {
  using V = double2;  // one complex
  static constexpr int PIECES = 12;
  static constexpr int STRIDE = 13;
};

// sp[lane] <- spinor of site `site` of lane `lane` (all 32 lanes take part)
template <typename R>
__device__ __forceinline__ void gather_spinors(const Cx<R> *__restrict__ f, int site, int lane,
                                               typename Stage<R>::V *sp) {
  using S = Stage<R>;
  const typename S::V *src = reinterpret_cast<const typename S::V *>(f);
#pragma unroll
  for (int k = 0; k < S::PIECES; ++k) {
    const int c = lane + 32 * k, i = c / S::PIECES, j = c - i * S::PIECES;
    const int si = __shfl_sync(0xffffffffu, site, i);
    sp[i * S::STRIDE + j] = __ldg(src + (long long)si * S::PIECES + j);
  }
}

// lk[lane] <- link mu of site `site` of lane `lane`
template <typename R>
__device__ __forceinline__ void gather_links(const Cx<R> *__restrict__ U, int site, int mu, int lane, Cx<R> *lk) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int c = lane + 32 * k, i = c / 9, j = c - i * 9;
    const int si = __shfl_sync(0xffffffffu, site, i);
    lk[i * 9 + j] = U[((long long)si * 4 + mu) * 9 + j];
  }
}

template <typename R>
__device__ __forceinline__ void read_spinor(const typename Stage<R>::V *sp, int lane, Cx<R> (&p)[12]) {
  using S = Stage<R>;
  const typename S::V *q = sp + lane * S::STRIDE;
  if (sizeof(R) == 4) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 w = *reinterpret_cast<const float4 *>(q + i);
      p[2 * i] = mk((R)w.x, (R)w.y);
      p[2 * i + 1] = mk((R)w.z, (R)w.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const double2 w = *reinterpret_cast<const double2 *>(q + i);
      p[i] = mk((R)w.x, (R)w.y);
    }
  }
}

}  // namespace

constexpr int DSLASH4_WARPS = 4;

// out = a (D in) + c b for vector blockIdx.y of a batch (stride ldv complex); with
// SHIFT the diagonal of that vector is diag + shift[blockIdx.y]
template <typename R, bool SHIFT>
__global__ void __launch_bounds__(32 * DSLASH4_WARPS, sizeof(R) == 4 ? 5 : 2) dslash4_kernel(const Cx<R> *__restrict__ U,
                                                                   const Cx<R> *__restrict__ in,
                                                                   Cx<R> *__restrict__ out, Geo4 g, R diag,
                                                                   const Cx<R> *__restrict__ b, R a, R c,
                                                                   long long ldv,
                                                                   const double *__restrict__ shift) {
  using S = Stage<R>;
  __shared__ typename S::V sp_all[DSLASH4_WARPS][32 * S::STRIDE];
  __shared__ Cx<R> lk_all[DSLASH4_WARPS][32 * 9];
  if (SHIFT) diag += (R)shift[blockIdx.y];
  in += blockIdx.y * ldv;
  out += blockIdx.y * ldv;
  if (b != nullptr) b += blockIdx.y * ldv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int V = (int)g.nsites;
  const int warp_first = (blockIdx.x * DSLASH4_WARPS + w) * 32;
  if (warp_first >= V) return;  // whole warps leave together
  const int xr = warp_first + lane;
  const bool valid = xr < V;
  const int x = valid ? xr : V - 1;  // tail lanes shadow the last site (no store)
  typename S::V *sp = sp_all[w];
  Cx<R> *lk = lk_all[w];
  // coordinates and strides of this lane's site
  int cc[4], st[4];
  {
    int r = x, stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cc[mu] = mu < 3 ? r % g.L[mu] : r;
      r = mu < 3 ? r / g.L[mu] : 0;
      st[mu] = stride;
      stride *= g.L[mu];
    }
  }
  Cx<R> acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = mk((R)0, (R)0);
  // the 8 hops one after another (not unrolled: one hop's loads are not hoisted into
  // another's registers)
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1;
    int cm = cc[0], sm = st[0], Lm = g.L[0];
    if (mu == 1) { cm = cc[1]; sm = st[1]; Lm = g.L[1]; }
    if (mu == 2) { cm = cc[2]; sm = st[2]; Lm = g.L[2]; }
    if (mu == 3) { cm = cc[3]; sm = st[3]; Lm = g.L[3]; }
    const bool fwd = (hop & 1) == 0;
    const int nb = fwd ? (cm + 1 == Lm ? x - cm * sm : x + sm) : (cm == 0 ? x + (Lm - 1) * sm : x - sm);
    __syncwarp();
    gather_spinors<R>(in, nb, lane, sp);
    gather_links<R>(U, fwd ? x : nb, mu, lane, lk);
    __syncwarp();
    Cx<R> p[12];
    read_spinor<R>(sp, lane, p);
    hop_dispatch<R>(hop, p, lk + lane * 9, acc);
  }
  // own spinor for the diagonal, then (optionally) b for the epilogue
  Cx<R> o[12];
  __syncwarp();
  gather_spinors<R>(in, x, lane, sp);
  __syncwarp();
  read_spinor<R>(sp, lane, o);
  const R h = (R)0.5;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const Cx<R> v = mk(diag * o[i].re - h * acc[i].re, diag * o[i].im - h * acc[i].im);
    o[i] = mk(a * v.re, a * v.im);
  }
  if (b != nullptr) {
    Cx<R> bb[12];
    __syncwarp();
    gather_spinors<R>(b, x, lane, sp);
    __syncwarp();
    read_spinor<R>(sp, lane, bb);
#pragma unroll
    for (int i = 0; i < 12; ++i) o[i] = mk(o[i].re + c * bb[i].re, o[i].im + c * bb[i].im);
  }
  // coalesced store through the staging buffer: consecutive lanes write consecutive pieces
  __syncwarp();
  {
    typename S::V *q = sp + lane * S::STRIDE;
    if (sizeof(R) == 4) {
#pragma unroll
      for (int i = 0; i < 6; ++i)
        reinterpret_cast<float4 *>(q)[i] =
            make_float4((float)o[2 * i].re, (float)o[2 * i].im, (float)o[2 * i + 1].re, (float)o[2 * i + 1].im);
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) reinterpret_cast<double2 *>(q)[i] = make_double2((double)o[i].re, (double)o[i].im);
    }
  }
  __syncwarp();
  typename S::V *dst = reinterpret_cast<typename S::V *>(out);
#pragma unroll
  for (int k = 0; k < S::PIECES; ++k) {
    const int cidx = lane + 32 * k, i = cidx / S::PIECES, j = cidx - i * S::PIECES;
    if (warp_first + i < V) dst[(long long)(warp_first + i) * S::PIECES + j] = sp[i * S::STRIDE + j];
  }
}

template <typename R>
void launch_dslash4(const Cx<R> *U, const Cx<R> *in, Cx<R> *out, Geo4 g, double diag, const Cx<R> *b, double a,
                    double c, cudaStream_t s, int nvec, const double *shift) {
  const int threads = 32 * DSLASH4_WARPS;
  const dim3 grid(grid_for(g.nsites, threads), nvec);
  if (shift != nullptr)
    dslash4_kernel<R, true><<<grid, threads, 0, s>>>(U, in, out, g, (R)diag, b, (R)a, (R)c, 12 * g.nsites, shift);
  else
    dslash4_kernel<R, false><<<grid, threads, 0, s>>>(U, in, out, g, (R)diag, b, (R)a, (R)c, 12 * g.nsites,
                                                      nullptr);
  MG_LAUNCHED();
}

template void launch_dslash4<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, Geo4, double,
                                     const Cx<double> *, double, double, cudaStream_t, int, const double *);
template void launch_dslash4<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, Geo4, double,
                                    const Cx<float> *, double, double, cudaStream_t, int, const double *);

}  // namespace mg
