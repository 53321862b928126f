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
#include <cstdlib>

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

// ---------------------------------------------------------------------------
// Tiled FP32 apply, for extents divisible by the tile: one CTA per tile of the lattice, one site
// per thread. Each site reads its spinor and its four forward links once and uses every link
// twice: U_x^mu for its own forward hop (applied to the projected spinor of x + mu) and
// U_x^mu^dagger for the backward hop of x + mu (applied to its own projected spinor here and
// handed over). Per direction the tile exchanges these two half spinors (2 spins x 3 colours)
// through shared memory; a site on a face of the tile forms the missing one itself from the
// outside neighbour (its spinor, and for a backward hop its link, read through L2). On-chip
// traffic per site: the 480 algorithmic bytes plus the faces' share, instead of 8 neighbour
// spinors and 8 links per site.
// ---------------------------------------------------------------------------

// tile extents (powers of two) and the thread-id step of one hop in each direction
template <int A0, int A1, int A2, int A3>
struct Tile4 {
  static constexpr int sites = A0 * A1 * A2 * A3;
  template <int MU>
  __host__ __device__ static constexpr int n() {
    return MU == 0 ? A0 : MU == 1 ? A1 : MU == 2 ? A2 : A3;
  }
  template <int MU>
  __host__ __device__ static constexpr int d() {
    return MU == 0 ? 1 : MU == 1 ? A0 : MU == 2 ? A0 * A1 : A0 * A1 * A2;
  }
};

__device__ __forceinline__ void load_spinor32(const Cx<float> *__restrict__ f, int x, Cx<float> (&p)[12]) {
  const float4 *q = reinterpret_cast<const float4 *>(f) + (long long)x * 6;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float4 w = __ldg(q + i);
    p[2 * i] = mk(w.x, w.y);
    p[2 * i + 1] = mk(w.z, w.w);
  }
}

__device__ __forceinline__ void load_link32(const Cx<float> *__restrict__ U, int x, int mu, Cx<float> (&u)[9]) {
  const float2 *q = reinterpret_cast<const float2 *>(U) + ((long long)x * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 w = __ldg(q + i);
    u[i] = mk(w.x, w.y);
  }
}

// h = psi_up - A_mu psi_dn (MINUS, the forward hop's (1 - gamma_mu)) or psi_up + A_mu psi_dn
template <int MU, bool MINUS>
__device__ __forceinline__ void project4(const Cx<float> (&p)[12], Cx<float> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<float> a0, a1;
    a_times<float, MU>(p[6 + c], p[9 + c], a0, a1);
    h[c] = MINUS ? p[c] - a0 : p[c] + a0;
    h[3 + c] = MINUS ? p[3 + c] - a1 : p[3 + c] + a1;
  }
}

// t = U h (DAG false) or U^dagger h, for both spin rows of h
template <bool DAG>
__device__ __forceinline__ void link_times4(const Cx<float> (&u)[9], const Cx<float> (&h)[6], Cx<float> (&t)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<float> t0 = mk(0.f, 0.f), t1 = mk(0.f, 0.f);
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      if (DAG) {
        cmac_conj(t0, u[bb * 3 + a], h[bb]);
        cmac_conj(t1, u[bb * 3 + a], h[3 + bb]);
      } else {
        cmac(t0, u[a * 3 + bb], h[bb]);
        cmac(t1, u[a * 3 + bb], h[3 + bb]);
      }
    }
    t[a] = t0;
    t[3 + a] = t1;
  }
}

// acc_up += t, acc_dn -= A_mu^dagger t (forward hop) or += (backward hop)
template <int MU, bool FWD>
__device__ __forceinline__ void reconstruct4(const Cx<float> (&t)[6], Cx<float> (&acc)[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<float> l0, l1;
    adag_times<float, MU>(t[c], t[3 + c], l0, l1);
    acc[c] = acc[c] + t[c];
    acc[3 + c] = acc[3 + c] + t[3 + c];
    if (FWD) {
      acc[6 + c] = acc[6 + c] - l0;
      acc[9 + c] = acc[9 + c] - l1;
    } else {
      acc[6 + c] = acc[6 + c] + l0;
      acc[9 + c] = acc[9 + c] + l1;
    }
  }
}

// the two hops of direction MU for the site of thread t (tile coordinate lm, lattice coordinate
// cm, extent Lm, site stride sm); sF / sM: [6][sites] half spinors in flight
template <class T, int MU>
__device__ __forceinline__ void tile_hops(const Cx<float> *__restrict__ U, const Cx<float> *__restrict__ in,
                                          const Cx<float> (&p)[12], int x, int t, int lm, int cm, int Lm, int sm,
                                          float2 (*sF)[T::sites], float2 (*sM)[T::sites], Cx<float> (&acc)[12]) {
  constexpr int n = T::template n<MU>(), d = T::template d<MU>();
  Cx<float> u[9];
  load_link32(U, x, MU, u);
  Cx<float> h[6], m[6];
  if (lm > 0) {  // the forward hop of x - mu needs (1 - gamma_mu) psi_x
    project4<MU, true>(p, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) sF[k][t - d] = make_float2(h[k].re, h[k].im);
  }
  if (lm < n - 1) {  // the backward hop of x + mu needs U_x^mu^dagger (1 + gamma_mu) psi_x
    project4<MU, false>(p, h);
    link_times4<true>(u, h, m);
#pragma unroll
    for (int k = 0; k < 6; ++k) sM[k][t + d] = make_float2(m[k].re, m[k].im);
  }
  __syncthreads();
  if (lm < n - 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float2 w = sF[k][t];
      h[k] = mk(w.x, w.y);
    }
  } else {
    Cx<float> q[12];
    load_spinor32(in, cm + 1 == Lm ? x - cm * sm : x + sm, q);
    project4<MU, true>(q, h);
  }
  link_times4<false>(u, h, m);
  reconstruct4<MU, true>(m, acc);
  if (lm > 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float2 w = sM[k][t];
      m[k] = mk(w.x, w.y);
    }
  } else {
    const int y = cm == 0 ? x + (Lm - 1) * sm : x - sm;
    Cx<float> q[12];
    load_spinor32(in, y, q);
    load_link32(U, y, MU, u);
    project4<MU, false>(q, h);
    link_times4<true>(u, h, m);
  }
  reconstruct4<MU, false>(m, acc);
  __syncthreads();
}

// DOTS: also the sums of an MR step on each vector (blockIdx.y), (<out, in>, |out|^2) as
// (re, im, norm), formed from the values the kernel holds anyway (its input and output at the
// site): per-thread and per-block in FP32, FP64 partials and final sum, into mr.out[3 v]
struct MrSums {
  double *partials;  // [vector][tile][3]
  double *out;       // [vector][3]
  unsigned int *tickets;
};

template <class T, int MINB, bool SHIFT, bool DOTS = false>
__global__ void __launch_bounds__(T::sites, MINB) dslash4_tile_kernel(const Cx<float> *__restrict__ U,
                                                                      const Cx<float> *__restrict__ in,
                                                                      Cx<float> *__restrict__ out, Geo4 g,
                                                                      float diag, const Cx<float> *__restrict__ b,
                                                                      float a, float c, long long ldv,
                                                                      const double *__restrict__ shift,
                                                                      MrSums mr = MrSums{}) {
  constexpr int A0 = T::template n<0>(), A1 = T::template n<1>(), A2 = T::template n<2>();
  __shared__ float2 sF[6][T::sites], sM[6][T::sites];
  if (SHIFT) diag += (float)shift[blockIdx.y];
  in += blockIdx.y * ldv;
  out += blockIdx.y * ldv;
  if (b != nullptr) b += blockIdx.y * ldv;
  const int t = threadIdx.x;
  const int l0 = t % A0, l1 = (t / A0) % A1, l2 = (t / (A0 * A1)) % A2, l3 = t / (A0 * A1 * A2);
  const int n0 = g.L[0] / A0, n1 = g.L[1] / A1, n2 = g.L[2] / A2;
  int tb = blockIdx.x;
  const int b0 = tb % n0;
  tb /= n0;
  const int b1 = tb % n1;
  tb /= n1;
  const int b2 = tb % n2;
  const int b3 = tb / n2;
  const int c0 = b0 * A0 + l0, c1 = b1 * A1 + l1, c2 = b2 * A2 + l2, c3 = b3 * T::template n<3>() + l3;
  const int s1 = g.L[0], s2 = g.L[0] * g.L[1], s3 = s2 * g.L[2];
  const int x = c0 + c1 * s1 + c2 * s2 + c3 * s3;
  Cx<float> p[12], acc[12];
  load_spinor32(in, x, p);
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = mk(0.f, 0.f);
  tile_hops<T, 0>(U, in, p, x, t, l0, c0, g.L[0], 1, sF, sM, acc);
  tile_hops<T, 1>(U, in, p, x, t, l1, c1, g.L[1], s1, sF, sM, acc);
  tile_hops<T, 2>(U, in, p, x, t, l2, c2, g.L[2], s2, sF, sM, acc);
  tile_hops<T, 3>(U, in, p, x, t, l3, c3, g.L[3], s3, sF, sM, acc);
  float sums[3] = {0.f, 0.f, 0.f};  // <out, in> and |out|^2 at this site (DOTS)
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const Cx<float> o = mk(a * (diag * p[i].re - 0.5f * acc[i].re), a * (diag * p[i].im - 0.5f * acc[i].im));
    if (DOTS) {
      sums[0] += o.re * p[i].re + o.im * p[i].im;
      sums[1] += o.re * p[i].im - o.im * p[i].re;
      sums[2] += o.re * o.re + o.im * o.im;
    }
    p[i] = o;
  }
  if (b != nullptr) {
    Cx<float> q[12];
    load_spinor32(b, x, q);
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = mk(p[i].re + c * q[i].re, p[i].im + c * q[i].im);
  }
  float4 *o = reinterpret_cast<float4 *>(out) + (long long)x * 6;
#pragma unroll
  for (int i = 0; i < 6; ++i) o[i] = make_float4(p[2 * i].re, p[2 * i].im, p[2 * i + 1].re, p[2 * i + 1].im);
  if (DOTS) {
    __shared__ float sh[32 * 3];
    grid_finish_t<3, float>(sums, mr.partials + (long long)blockIdx.y * gridDim.x * 3, mr.out + 3 * blockIdx.y,
                            mr.tickets + blockIdx.y, sh);
  }
}

// tile shapes of the tiled kernel; MG_DSLASH4_TILE picks one (default 7, the fastest at 32^3 x 64:
// 0.365 ms against 0.373 to 0.426 for the other shapes and 0.429 for the warp-gather kernel),
// MG_DSLASH4_GATHER the warp-gather kernel
using TileA = Tile4<8, 4, 4, 4>;  // 512 threads, 1 CTA per SM
using TileB = Tile4<8, 4, 4, 2>;  // 256 threads, 2 CTAs per SM
using TileC = Tile4<4, 4, 4, 2>;  // 128 threads, 4 CTAs per SM
using TileD = Tile4<8, 4, 2, 2>;  // 128 threads, 4 CTAs per SM
using TileE = Tile4<4, 4, 2, 2>;  // 64 threads, 8 CTAs per SM
using TileF = Tile4<8, 2, 2, 2>;  // 64 threads, 8 CTAs per SM

template <class T>
static bool tile_divides(const Geo4 &g) {
  return g.L[0] % T::template n<0>() == 0 && g.L[1] % T::template n<1>() == 0 && g.L[2] % T::template n<2>() == 0 &&
         g.L[3] % T::template n<3>() == 0;
}

template <class T, int MINB>
static void launch_tile4(const Cx<float> *U, const Cx<float> *in, Cx<float> *out, Geo4 g, double diag,
                         const Cx<float> *b, double a, double c, cudaStream_t s, int nvec, const double *shift) {
  const dim3 grid((unsigned int)(g.nsites / T::sites), nvec);
  if (shift != nullptr)
    dslash4_tile_kernel<T, MINB, true><<<grid, T::sites, 0, s>>>(U, in, out, g, (float)diag, b, (float)a, (float)c,
                                                                  12 * g.nsites, shift);
  else
    dslash4_tile_kernel<T, MINB, false><<<grid, T::sites, 0, s>>>(U, in, out, g, (float)diag, b, (float)a,
                                                                   (float)c, 12 * g.nsites, nullptr);
  MG_LAUNCHED();
}

// true when a tiled kernel took the apply
static bool try_tile4(const Cx<float> *U, const Cx<float> *in, Cx<float> *out, Geo4 g, double diag,
                      const Cx<float> *b, double a, double c, cudaStream_t s, int nvec, const double *shift) {
  if (std::getenv("MG_DSLASH4_GATHER") != nullptr) return false;
  const char *v = std::getenv("MG_DSLASH4_TILE");
  const int which = v != nullptr ? std::atoi(v) : 7;
  if (which == 0 && tile_divides<TileA>(g)) {
    launch_tile4<TileA, 1>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 2 && tile_divides<TileC>(g)) {
    launch_tile4<TileC, 4>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 6 && tile_divides<TileE>(g)) {
    launch_tile4<TileE, 8>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 7 && tile_divides<TileF>(g)) {
    launch_tile4<TileF, 8>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 3 && tile_divides<TileD>(g)) {
    launch_tile4<TileD, 4>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 4 && tile_divides<TileB>(g)) {  // 3 CTAs per SM: at most 85 registers
    launch_tile4<TileB, 3>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 5 && tile_divides<TileC>(g)) {  // 6 CTAs per SM
    launch_tile4<TileC, 6>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (which == 1 && tile_divides<TileB>(g)) {
    launch_tile4<TileB, 2>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (tile_divides<TileF>(g)) {
    launch_tile4<TileF, 8>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  if (tile_divides<TileB>(g)) {
    launch_tile4<TileB, 2>(U, in, out, g, diag, b, a, c, s, nvec, shift);
    return true;
  }
  return false;
}

// Ar = D r for nvec FP32 vectors together with the MR sums (<Ar, r>, |Ar|^2) of each, by the
// default tiled kernel; false (nothing launched) when that kernel does not take this lattice
// or another variant is selected
bool launch_dslash4_mr(const Cx<float> *U, const Cx<float> *r, Cx<float> *Ar, Geo4 g, double diag, int nvec,
                       double *sums, double *partials, long long partials_cap, unsigned int *tickets,
                       cudaStream_t s) {
  if (std::getenv("MG_DSLASH4_GATHER") != nullptr || std::getenv("MG_DSLASH4_TILE") != nullptr) return false;
  if (!tile_divides<TileF>(g)) return false;
  const long long tiles = g.nsites / TileF::sites;
  if (tiles * 3 * nvec > partials_cap) return false;
  const dim3 grid((unsigned int)tiles, nvec);
  dslash4_tile_kernel<TileF, 8, false, true><<<grid, TileF::sites, 0, s>>>(U, r, Ar, g, (float)diag, nullptr, 1.f,
                                                                           0.f, 12 * g.nsites, nullptr,
                                                                           MrSums{partials, sums, tickets});
  MG_LAUNCHED();
  return true;
}

template <typename R>
void launch_dslash4(const Cx<R> *U, const Cx<R> *in, Cx<R> *out, Geo4 g, double diag, const Cx<R> *b, double a,
                    double c, cudaStream_t s, int nvec, const double *shift) {
  if constexpr (sizeof(R) == 4) {
    if (try_tile4(U, in, out, g, diag, b, a, c, s, nvec, shift)) return;
  }
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
