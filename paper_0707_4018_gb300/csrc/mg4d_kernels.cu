// Transfer, Gram-Schmidt, Galerkin and coarse-operator kernels of the 4d SU(3)
// two-level multigrid (paper: Eq. P1 and the adaptive step for the block-local
// prolongator, Eq. Galerkin for P^dagger D P, the V-cycle's restriction and
// prolongation).
//
// The prolongator keeps only the nonzero chirality half of each column:
// V[b][c][s][d6], c < N = 2 Nv, s < bvol, d6 < 6, is dof 6 chi + d6 (chi = c / Nv)
// of site s of block b; per column Nh = 6 bvol complex, contiguous, so the block
// reductions and the prolongation read V with unit stride.
#include <cuda_fp16.h>
#include <algorithm>

#include <cstdlib>

#include "mg4d.h"
#include "wilson4d.cuh"

namespace mg {

namespace {

__device__ __forceinline__ int fine_site4(const Block4 &g, int b, int s) {
  int x = 0, stride = 1;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int bc = b % g.nb[mu];
    b /= g.nb[mu];
    const int sc = s % g.B[mu];
    s /= g.B[mu];
    x += (bc * g.B[mu] + sc) * stride;
    stride *= g.L[mu];
  }
  return x;
}

template <typename R>
__device__ __forceinline__ void warp_sum2(R &a, R &b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// sum of (a, b) over the CTA, returned to every thread (fixed order: deterministic)
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*red)[32]) {
  warp_sum2(a, b);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][w] = a;
    red[1][w] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < nw; ++i) {
    a += red[0][i];
    b += red[1][i];
  }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// restriction r_c[b][c] = sum_{s, d6} conj(V[b][c][s][d6]) r[x(b, s)][6 chi + d6]:
// the block's fine values are staged in shared memory, a warp reduces one column
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) restrict4_kernel(const Cx<R> *__restrict__ V, const Cx<R> *__restrict__ fine,
                                                        Cx<R> *__restrict__ coarse, Block4 g, long long fine_ld,
                                                        long long coarse_ld) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Cx<R> *sm = reinterpret_cast<Cx<R> *>(sm_raw);
  const int b = blockIdx.x;
  fine += blockIdx.y * fine_ld;
  coarse += blockIdx.y * coarse_ld;
  const int N = 2 * g.Nv, Nh = g.bvol * 6;
  for (int e = threadIdx.x; e < g.bvol * 12; e += blockDim.x) {
    const int s = e / 12, d = e - s * 12;
    sm[e] = fine[(long long)fine_site4(g, b, s) * 12 + d];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < N; c += nw) {
    const int chi = c / g.Nv;
    const Cx<R> *Vc = V + ((long long)b * N + c) * Nh;
    R re = 0, im = 0;
    for (int e = lane; e < Nh; e += 32) {
      const int s = e / 6, d6 = e - s * 6;
      const Cx<R> v = Vc[e], f = sm[s * 12 + 6 * chi + d6];
      re += v.re * f.re + v.im * f.im;
      im += v.re * f.im - v.im * f.re;
    }
    warp_sum2(re, im);
    if (lane == 0) coarse[(long long)b * N + c] = mk(re, im);
  }
}

// prolongation fine[x(b, s)][6 chi + d6] += sum_k V[b][chi Nv + k][s][d6] e[b][chi Nv + k]
template <typename R>
__global__ void __launch_bounds__(256) prolong4_kernel(const Cx<R> *__restrict__ V, const Cx<R> *__restrict__ coarse,
                                                       Cx<R> *__restrict__ fine, Block4 g, long long fine_ld,
                                                       long long coarse_ld) {
  __shared__ Cx<R> es[128];
  const int b = blockIdx.x;
  fine += blockIdx.y * fine_ld;
  coarse += blockIdx.y * coarse_ld;
  const int N = 2 * g.Nv, Nh = g.bvol * 6;
  for (int c = threadIdx.x; c < N; c += blockDim.x) es[c] = coarse[(long long)b * N + c];
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * Nh; e += blockDim.x) {
    const int chi = e / Nh, r = e - chi * Nh, s = r / 6, d6 = r - s * 6;
    const Cx<R> *Vb = V + ((long long)b * N + chi * g.Nv) * Nh + r;
    Cx<R> acc = mk((R)0, (R)0);
    for (int k = 0; k < g.Nv; ++k) cmac(acc, Vb[(long long)k * Nh], es[chi * g.Nv + k]);
    Cx<R> *f = fine + (long long)fine_site4(g, b, s) * 12 + 6 * chi + d6;
    *f = *f + acc;
  }
}

// V[b][chi Nv + k][s][d6] = vecs[k][x(b, s)][6 chi + d6]
__global__ void gather_split4_kernel(const Cx<double> *__restrict__ vecs, long long vstride,
                                     Cx<double> *__restrict__ V, Block4 g) {
  const int N = 2 * g.Nv, Nh = g.bvol * 6;
  const long long total = (long long)g.nblocks * N * Nh;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % Nh);
    const long long bc = e / Nh;
    const int c = (int)(bc % N), b = (int)(bc / N);
    const int chi = c / g.Nv, k = c - chi * g.Nv, s = r / 6, d6 = r - s * 6;
    V[e] = vecs[k * vstride + (long long)fine_site4(g, b, s) * 12 + 6 * chi + d6];
  }
}

// modified Gram-Schmidt in k order, run twice, on the Nv columns of one (block, chirality)
__global__ void __launch_bounds__(256) block_gs4_kernel(Cx<double> *__restrict__ V, Block4 g) {
  __shared__ double red[2][32];
  const int b = blockIdx.x, chi = blockIdx.y, N = 2 * g.Nv, Nh = g.bvol * 6;
  Cx<double> *base = V + ((long long)b * N + chi * g.Nv) * Nh;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < g.Nv; ++k) {
      Cx<double> *vk = base + (long long)k * Nh;
      for (int j = 0; j < k; ++j) {
        const Cx<double> *vj = base + (long long)j * Nh;
        double re = 0.0, im = 0.0;  // <v_j, v_k>
        for (int e = threadIdx.x; e < Nh; e += blockDim.x) {
          const Cx<double> a = vj[e], c = vk[e];
          re += a.re * c.re + a.im * c.im;
          im += a.re * c.im - a.im * c.re;
        }
        block_sum2(re, im, red);
        for (int e = threadIdx.x; e < Nh; e += blockDim.x) {
          const Cx<double> a = vj[e];
          Cx<double> c = vk[e];
          c.re -= re * a.re - im * a.im;
          c.im -= re * a.im + im * a.re;
          vk[e] = c;
        }
      }
      double n2 = 0.0, zero = 0.0;
      for (int e = threadIdx.x; e < Nh; e += blockDim.x) n2 += norm2(vk[e]);
      block_sum2(n2, zero, red);
      const double inv = 1.0 / sqrt(n2);
      for (int e = threadIdx.x; e < Nh; e += blockDim.x) vk[e] = inv * vk[e];
    }
  }
}

// ---------------------------------------------------------------------------
// Galerkin operator: CTA (coarse site j, direction dir). For every fine site x of
// block j that dir involves (all sites for dir 0; the forward / backward face in mu
// for +mu / -mu) the N columns are moved through the part of D that dir denotes
// (diagonal plus in-block hops; the hop from the neighbouring block), and the
// rows of block j at x are contracted with them:
//   Y[j][dir][col][row] += sum_d conj(V_row(x)_d) (D_dir V_col)(x)_d
// ---------------------------------------------------------------------------
constexpr int kGalPairs = 16;  // (row, col) pairs per thread: N <= 64

// CT: the arithmetic (and the links' and prolongator's storage) type; Y is written in FP64.
// FP32 for mixed-precision hierarchies with an inexact coarse solve: the kernel is FP64-ALU
// bound on this part (73 ms at 16^3 x 32 with Nv = 24).
template <typename CT>
__global__ void __launch_bounds__(256) galerkin4_kernel(const Cx<CT> *__restrict__ U, double diag,
                                                        const Cx<CT> *__restrict__ V, Cx<double> *__restrict__ Y,
                                                        Block4 g) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int N = 2 * g.Nv, Nh = g.bvol * 6;
  Cx<CT> *Hs = reinterpret_cast<Cx<CT> *>(sm_raw);  // [N][12]
  Cx<CT> *Vs = Hs + N * 12;                          // [N][6]
  const int j = blockIdx.x, dir = blockIdx.y, tid = threadIdx.x;
  int jc[4];
  {
    int r = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = r % g.nb[mu];
      r /= g.nb[mu];
    }
  }
  const int mu = dir == 0 ? 0 : (dir - 1) >> 1;
  const bool fwd = dir != 0 && ((dir - 1) & 1) == 0;
  int jsrc = j;
  if (dir != 0) {
    int cc[4] = {jc[0], jc[1], jc[2], jc[3]};
    cc[mu] = fwd ? (cc[mu] + 1) % g.nb[mu] : (cc[mu] + g.nb[mu] - 1) % g.nb[mu];
    jsrc = cc[0] + g.nb[0] * (cc[1] + g.nb[1] * (cc[2] + g.nb[2] * cc[3]));
  }
  int bst[4], fst[4];  // in-block and fine strides
  bst[0] = 1;
  fst[0] = 1;
  for (int m2 = 1; m2 < 4; ++m2) {
    bst[m2] = bst[m2 - 1] * g.B[m2 - 1];
    fst[m2] = fst[m2 - 1] * g.L[m2 - 1];
  }
  const int npairs = N * N;
  Cx<CT> acc[kGalPairs];
#pragma unroll
  for (int i = 0; i < kGalPairs; ++i) acc[i] = mk((CT)0, (CT)0);
  const int nvisit = dir == 0 ? g.bvol : g.bvol / g.B[mu];
  for (int q = 0; q < nvisit; ++q) {
    // in-block position s of the q-th site (for a face: coordinate mu fixed)
    int sc[4];
    if (dir == 0) {
      int r = q;
      for (int m2 = 0; m2 < 4; ++m2) {
        sc[m2] = r % g.B[m2];
        r /= g.B[m2];
      }
    } else {
      int r = q;
      for (int m2 = 0; m2 < 4; ++m2) {
        if (m2 == mu) {
          sc[m2] = fwd ? g.B[mu] - 1 : 0;
        } else {
          sc[m2] = r % g.B[m2];
          r /= g.B[m2];
        }
      }
    }
    const int s = sc[0] + bst[1] * sc[1] + bst[2] * sc[2] + bst[3] * sc[3];
    const int x = fine_site4(g, j, s);
    __syncthreads();  // the previous site's shared data is consumed
    for (int e = tid; e < N * 6; e += blockDim.x) {
      const int r = e / 6, d6 = e - r * 6;
      Vs[e] = V[((long long)j * N + r) * Nh + s * 6 + d6];
    }
    if (tid < N) {
      const int c = tid, chi = c / g.Nv;
      Cx<CT> hacc[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) hacc[i] = mk((CT)0, (CT)0);
      Cx<CT> p[12];
      auto load_col = [&](int blk, int spos) {
#pragma unroll
        for (int i = 0; i < 12; ++i) p[i] = mk((CT)0, (CT)0);
        const Cx<CT> *src = V + ((long long)blk * N + c) * Nh + spos * 6;
#pragma unroll
        for (int d6 = 0; d6 < 6; ++d6) p[6 * chi + d6] = src[d6];
      };
      Cx<CT> h[12];
      if (dir == 0) {
        load_col(j, s);
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] = (CT)diag * p[i];
        for (int m2 = 0; m2 < 4; ++m2) {
          if (sc[m2] + 1 < g.B[m2]) {  // x + m2 inside the block
            load_col(j, s + bst[m2]);
            hop_dispatch<CT>(2 * m2, p, U + ((long long)x * 4 + m2) * 9, hacc);
          }
          if (sc[m2] > 0) {  // x - m2 inside the block
            load_col(j, s - bst[m2]);
            hop_dispatch<CT>(2 * m2 + 1, p, U + ((long long)(x - fst[m2]) * 4 + m2) * 9, hacc);
          }
        }
      } else {
        int sn = s + (fwd ? -(g.B[mu] - 1) : (g.B[mu] - 1)) * bst[mu];  // mirror position in the source block
        load_col(jsrc, sn);
        const int xn = fine_site4(g, jsrc, sn);
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] = mk((CT)0, (CT)0);
        hop_dispatch<CT>(fwd ? 2 * mu : 2 * mu + 1, p, U + ((long long)(fwd ? x : xn) * 4 + mu) * 9, hacc);
      }
#pragma unroll
      for (int i = 0; i < 12; ++i)
        Hs[c * 12 + i] = mk(h[i].re - (CT)0.5 * hacc[i].re, h[i].im - (CT)0.5 * hacc[i].im);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kGalPairs; ++i) {
      const int pr = tid + 256 * i;
      if (pr < npairs) {
        const int col = pr / N, row = pr - col * N, chr = row / g.Nv;
        Cx<CT> a = acc[i];
#pragma unroll
        for (int d6 = 0; d6 < 6; ++d6) cmac_conj(a, Vs[row * 6 + d6], Hs[col * 12 + 6 * chr + d6]);
        acc[i] = a;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kGalPairs; ++i) {
    const int pr = tid + 256 * i;
    if (pr < npairs) Y[((long long)j * 9 + dir) * npairs + pr] = mk((double)acc[i].re, (double)acc[i].im);
  }
}

// ---------------------------------------------------------------------------
// coarse apply: CTA (site j, vector v), QP N threads (QP = min(8, 512 / N) partial sums
// per row): the 9 N source values in shared memory, thread (q, row) sums the (dir, col)
// pairs p = q, q + QP, ... of its row.
// The operator may be stored in lower precision than the vectors (RY = float with
// RV = double: the sums run in FP32, inputs rounded once, the result widened).
// ---------------------------------------------------------------------------
template <typename RY, typename RV>
__global__ void coarse4_apply_kernel(const Cx<RY> *__restrict__ Y, const Cx<RV> *__restrict__ in,
                                     Cx<RV> *__restrict__ out, Coarse4 g, const Cx<RV> *__restrict__ b, RV a, RV c,
                                     long long ldv, const double *__restrict__ shift) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int N = g.N;
  const int QP = blockDim.x / N;                     // partial sums per row
  Cx<RY> *xs = reinterpret_cast<Cx<RY> *>(sm_raw);  // [9][N]
  Cx<RY> *red = xs + 9 * N;                          // [QP][N]
  const int j = blockIdx.x, v = blockIdx.y;
  in += v * ldv;
  out += v * ldv;
  if (b != nullptr) b += v * ldv;
  int jc[4];
  {
    int r = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = r % g.nb[mu];
      r /= g.nb[mu];
    }
  }
  for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
    const int dir = e / N, col = e - dir * N;
    int src = j;
    if (dir != 0) {
      const int mu = (dir - 1) >> 1;
      int cc[4] = {jc[0], jc[1], jc[2], jc[3]};
      cc[mu] = ((dir - 1) & 1) == 0 ? (cc[mu] + 1) % g.nb[mu] : (cc[mu] + g.nb[mu] - 1) % g.nb[mu];
      src = cc[0] + g.nb[0] * (cc[1] + g.nb[1] * (cc[2] + g.nb[2] * cc[3]));
    }
    xs[e] = cvt<RY, RV>(in[(long long)src * N + col]);
  }
  __syncthreads();
  const int row = threadIdx.x % N, q = threadIdx.x / N;
  const Cx<RY> *Yj = Y + (long long)j * 9 * N * N;
  RY re = 0, im = 0;
#pragma unroll 4
  for (int p = q; p < 9 * N; p += QP) {  // independent loads: unrolled for memory parallelism
    const Cx<RY> y = Yj[(long long)p * N + row], xv = xs[p];
    re += y.re * xv.re - y.im * xv.im;
    im += y.re * xv.im + y.im * xv.re;
  }
  red[q * N + row] = mk(re, im);
  __syncthreads();
  if (q == 0) {
    RV sre = 0, sim = 0;
    for (int i = 0; i < QP; ++i) {
      sre += (RV)red[i * N + row].re;
      sim += (RV)red[i * N + row].im;
    }
    if (shift != nullptr) {
      const Cx<RV> xv = in[(long long)j * N + row];
      sre += (RV)shift[v] * xv.re;
      sim += (RV)shift[v] * xv.im;
    }
    Cx<RV> o = mk(a * sre, a * sim);
    if (b != nullptr) {
      const Cx<RV> bb = b[(long long)j * N + row];
      o = mk(o.re + c * bb.re, o.im + c * bb.im);
    }
    out[(long long)j * N + row] = o;
  }
}

// ---------------------------------------------------------------------------
// block-Jacobi preconditioner of the coarse solve: Minv[j] = X_j^{-1}, X_j the self
// block Y[j][0], by Gauss-Jordan elimination with partial pivoting (FP64, one CTA per
// site, the N x 2N tableau in shared memory); stored column-major like Y
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) block_invert4_kernel(const Cx<double> *__restrict__ Y,
                                                            Cx<double> *__restrict__ Minv, int N, int *info) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Cx<double> *T = reinterpret_cast<Cx<double> *>(sm_raw);  // T[row][0..2N)
  __shared__ int piv;
  __shared__ double pscale[2];
  const int j = blockIdx.x, W = 2 * N;
  const Cx<double> *X = Y + (long long)j * 9 * N * N;  // dir 0, [col][row]
  for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
    const int r = e / W, cc = e - r * W;
    T[e] = cc < N ? X[(long long)cc * N + r] : mk(cc - N == r ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x < 32) {  // pivot: largest |T[i][k]| for i >= k, lowest index on ties
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < N; i += 32) {
        const double v = norm2(T[i * W + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > 0.0)) atomicExch(info, 1);
      }
    }
    __syncthreads();
    if (piv != k)
      for (int cc = threadIdx.x; cc < W; cc += blockDim.x) {
        const Cx<double> t = T[k * W + cc];
        T[k * W + cc] = T[piv * W + cc];
        T[piv * W + cc] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) {  // 1 / pivot
      const Cx<double> p = T[k * W + k];
      const double d = norm2(p);
      pscale[0] = p.re / d;
      pscale[1] = -p.im / d;
    }
    __syncthreads();
    const Cx<double> ip = mk(pscale[0], pscale[1]);
    for (int cc = threadIdx.x; cc < W; cc += blockDim.x) T[k * W + cc] = T[k * W + cc] * ip;
    __syncthreads();
    for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
      const int r = e / W, cc = e - r * W;
      if (r == k || cc == k) continue;
      const Cx<double> f = T[r * W + k];
      T[e] = T[e] - f * T[k * W + cc];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x)
      if (r != k) T[r * W + k] = mk(0.0, 0.0);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int cc = e / N, r = e - cc * N;
    Minv[(long long)j * N * N + e] = T[r * W + N + cc];
  }
}

// z_j = Minv_j r_j (one CTA per site and vector blockIdx.y, one thread per row; vectors at
// stride ld)
template <typename R, typename VT>
__global__ void block_apply4_kernel(const Cx<R> *__restrict__ Minv, const Cx<VT> *__restrict__ r,
                                    Cx<VT> *__restrict__ z, int N, long long ld) {
  __shared__ Cx<R> rs[64];
  r += blockIdx.y * ld;
  z += blockIdx.y * ld;
  const int j = blockIdx.x, row = threadIdx.x;
  if (row < N) rs[row] = cvt<R, VT>(r[(long long)j * N + row]);
  __syncthreads();
  if (row >= N) return;
  const Cx<R> *M = Minv + (long long)j * N * N;
  Cx<R> acc = mk((R)0, (R)0);
#pragma unroll 8
  for (int cc = 0; cc < N; ++cc) cmac(acc, M[(long long)cc * N + row], rs[cc]);
  z[(long long)j * N + row] = cvt<VT, R>(acc);
}

// ---------------------------------------------------------------------------
// GCR step with the coefficients formed on the device (no host round trip per
// iteration): from the fused reduction dots = (<W_j, w>_j<k, |w|^2, <w, r>, |r|^2) each
// CTA forms the classical Gram-Schmidt norm |w - W beta|^2 = |w|^2 - |beta|^2,
// inv = 1 / that norm and alpha = <w, r> inv (a breakdown gives inv = alpha = 0: the
// step changes nothing); CTA 0 also stores the residual estimate |r|^2 - |alpha|^2 in
// state[0]. Then w <- (w - sum_j beta_j W_j) inv, z likewise; W_k = w, Z_k = z;
// x += alpha z; r -= alpha w.
// ---------------------------------------------------------------------------
// (VT = float: FP32 vectors; the coefficients are formed in FP64 and applied in FP32)
template <typename VT>
__global__ void gcr_update_dev_kernel(const Cx<VT> *__restrict__ W, Cx<VT> *__restrict__ Wk,
                                      const Cx<VT> *__restrict__ Z, Cx<VT> *__restrict__ Zk, int k,
                                      const double *__restrict__ dots, double *__restrict__ state,
                                      Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ r, long long n) {
  __shared__ double coef[3];
  if (threadIdx.x == 0) {
    const double nw0 = dots[2 * k];
    double nw2 = nw0;
    for (int j = 0; j < k; ++j) nw2 -= dots[2 * j] * dots[2 * j] + dots[2 * j + 1] * dots[2 * j + 1];
    double inv = 0.0, are = 0.0, aim = 0.0;
    if (nw2 > 1e-28 * nw0) {
      inv = 1.0 / sqrt(nw2);
      are = dots[2 * k + 2] * inv;
      aim = dots[2 * k + 3] * inv;
    }
    coef[0] = inv;
    coef[1] = are;
    coef[2] = aim;
    if (blockIdx.x == 0) state[0] = fmax(dots[2 * k + 4] - (are * are + aim * aim), 0.0);
  }
  __syncthreads();
  const VT inv = (VT)coef[0];
  const Cx<VT> alpha = mk((VT)coef[1], (VT)coef[2]), malpha = mk((VT)-coef[1], (VT)-coef[2]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Cx<VT> w = Wk[i], z = Zk[i];
    for (int j = 0; j < k; ++j) {
      const Cx<VT> bj = mk((VT)-dots[2 * j], (VT)-dots[2 * j + 1]);
      cmac(w, bj, W[(long long)j * n + i]);
      cmac(z, bj, Z[(long long)j * n + i]);
    }
    w = inv * w;
    z = inv * z;
    Wk[i] = w;
    Zk[i] = z;
    cmac(x[i], alpha, z);
    Cx<VT> ri = r[i];
    cmac(ri, malpha, w);
    r[i] = ri;
  }
}

// Yt[j][dir] = Y[j][dir] Minv[src(j, dir)] (column-major blocks): the block-Jacobi
// right-preconditioned stencil A M, one thread per entry
__global__ void precondition4_kernel(const Cx<double> *__restrict__ Y, const Cx<double> *__restrict__ Minv,
                                     Cx<double> *__restrict__ Yt, Coarse4 g) {
  const int N = g.N;
  const long long per = 9LL * N * N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.nsites * per) return;
  const long long j = t / per;
  const int rem = (int)(t - j * per), dir = rem / (N * N), cr = rem - dir * N * N, col = cr / N, row = cr - col * N;
  long long src = j;
  if (dir != 0) {
    int jc[4];
    long long q = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = (int)(q % g.nb[mu]);
      q /= g.nb[mu];
    }
    const int mu = (dir - 1) >> 1;
    jc[mu] = ((dir - 1) & 1) == 0 ? (jc[mu] + 1) % g.nb[mu] : (jc[mu] + g.nb[mu] - 1) % g.nb[mu];
    src = jc[0] + (long long)g.nb[0] * (jc[1] + (long long)g.nb[1] * (jc[2] + (long long)g.nb[2] * jc[3]));
  }
  const Cx<double> *Yd = Y + (j * 9 + dir) * (long long)N * N;
  const Cx<double> *Ms = Minv + src * (long long)N * N;
  Cx<double> acc = mk(0.0, 0.0);
  for (int q = 0; q < N; ++q) cmac(acc, Yd[(long long)q * N + row], Ms[(long long)col * N + q]);
  Yt[t] = acc;
}

// ---------------------------------------------------------------------------
// batched MR pieces for nvec vectors of n complex each (vector v = blockIdx.y):
// sc[3 v .. 3 v + 2] = (<Ar_v, r_v>, |Ar_v|^2), summed per thread and per block in R
// (FP32 for FP32 vectors: GB300's FP64 unit is far slower), partials and the final
// sum in FP64; then x_v += alpha_v r_v, r_v -= alpha_v Ar_v with
// alpha_v = omega <Ar_v, r_v> / |Ar_v|^2
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kReduceThreads) dot_norm_batch_kernel(const Cx<R> *__restrict__ a,
                                                                        const Cx<R> *__restrict__ b, long long n,
                                                                        double *partials, double *out,
                                                                        unsigned int *ticket) {
  __shared__ R sh[32 * 3];
  const long long off = blockIdx.y * n;
  R v[3] = {(R)0, (R)0, (R)0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> x = a[off + i], y = b[off + i];
    v[0] += x.re * y.re + x.im * y.im;
    v[1] += x.re * y.im - x.im * y.re;
    v[2] += x.re * x.re + x.im * x.im;
  }
  grid_finish_t<3, R>(v, partials + (long long)blockIdx.y * gridDim.x * 3, out + 3 * blockIdx.y,
                      ticket + blockIdx.y, sh);
}

template <typename R>
__global__ void mr_update_batch_kernel(const double *__restrict__ sc, double omega, Cx<R> *__restrict__ x,
                                       Cx<R> *__restrict__ r, const Cx<R> *__restrict__ Ar, long long n) {
  const int v = blockIdx.y;
  const double den = sc[3 * v + 2];
  const R are = den > 0.0 ? (R)(omega * sc[3 * v] / den) : (R)0, aim = den > 0.0 ? (R)(omega * sc[3 * v + 1] / den) : (R)0;
  const long long off = v * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Cx<R> ri = r[off + i], ai = Ar[off + i];
    Cx<R> xi = x[off + i];
    xi.re += are * ri.re - aim * ri.im;
    xi.im += are * ri.im + aim * ri.re;
    x[off + i] = xi;
    r[off + i] = mk(ri.re - (are * ai.re - aim * ai.im), ri.im - (are * ai.im + aim * ai.re));
  }
}

__global__ void coarse4_to_canonical_kernel(const Cx<double> *__restrict__ Yi, Cx<double> *__restrict__ Yc,
                                            long long total, int N) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // canonical [j][dir][row][col]
  if (e >= total) return;
  const int col = (int)(e % N);
  const long long t = e / N;
  const int row = (int)(t % N);
  const long long jd = t / N;
  Yc[e] = Yi[(jd * N + col) * N + row];
}

__global__ void prolongator4_to_canonical_kernel(const Cx<double> *__restrict__ V, Cx<double> *__restrict__ out,
                                                 Block4 g, long long nsites) {
  const int N = 2 * g.Nv, Nh = g.bvol * 6;
  const long long total = (long long)N * nsites * 12;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // [c][x][12]
  if (e >= total) return;
  const int dof = (int)(e % 12);
  const long long cx = e / 12;
  const int x = (int)(cx % nsites), c = (int)(cx / nsites);
  const int chi = c / g.Nv;
  Cx<double> v = mk(0.0, 0.0);
  if (dof / 6 == chi) {
    int b = 0, s = 0, bstr = 1, sstr = 1, r = x;
    for (int mu = 0; mu < 4; ++mu) {
      const int xc = r % g.L[mu];
      r /= g.L[mu];
      b += (xc / g.B[mu]) * bstr;
      s += (xc % g.B[mu]) * sstr;
      bstr *= g.nb[mu];
      sstr *= g.B[mu];
    }
    v = V[((long long)b * N + c) * Nh + s * 6 + (dof - 6 * chi)];
  }
  out[e] = v;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename R>
void launch_restrict4(const Cx<R> *V, const Cx<R> *fine, Cx<R> *coarse, const Block4 &g, cudaStream_t s, int nvec) {
  const size_t smem = (size_t)g.bvol * 12 * sizeof(Cx<R>);
  static bool attr = false;  // one opt-in per process for more than 48 KB
  if (!attr) {
    MG_CUDA(cudaFuncSetAttribute(restrict4_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr = true;
  }
  const long long nf = (long long)g.nblocks * g.bvol * 12;
  restrict4_kernel<R><<<dim3(g.nblocks, nvec), 256, smem, s>>>(V, fine, coarse, g, nf, (long long)g.nblocks * 2 * g.Nv);
  MG_LAUNCHED();
}

template <typename R>
void launch_prolong4(const Cx<R> *V, const Cx<R> *coarse, Cx<R> *fine, const Block4 &g, cudaStream_t s, int nvec) {
  const long long nf = (long long)g.nblocks * g.bvol * 12;
  prolong4_kernel<R><<<dim3(g.nblocks, nvec), 256, 0, s>>>(V, coarse, fine, g, nf, (long long)g.nblocks * 2 * g.Nv);
  MG_LAUNCHED();
}

void launch_gather_split4(const Cx<double> *vecs, long long vstride, Cx<double> *V, const Block4 &g, cudaStream_t s) {
  const long long total = (long long)g.nblocks * 2 * g.Nv * g.bvol * 6;
  const unsigned int grid = (unsigned int)std::min<long long>((total + 255) / 256, 152LL * 16);
  gather_split4_kernel<<<grid, 256, 0, s>>>(vecs, vstride, V, g);
  MG_LAUNCHED();
}

void launch_block_gs4(Cx<double> *V, const Block4 &g, cudaStream_t s) {
  block_gs4_kernel<<<dim3(g.nblocks, 2), 256, 0, s>>>(V, g);
  MG_LAUNCHED();
}

template <typename CT>
void launch_galerkin4(const Cx<CT> *U, double diag, const Cx<CT> *V, Cx<double> *Y, const Block4 &g, cudaStream_t s) {
  const int N = 2 * g.Nv;
  const size_t smem = (size_t)N * 18 * sizeof(Cx<CT>);
  galerkin4_kernel<CT><<<dim3(g.nblocks, 9), 256, smem, s>>>(U, diag, V, Y, g);
  MG_LAUNCHED();
}
template void launch_galerkin4<double>(const Cx<double> *, double, const Cx<double> *, Cx<double> *, const Block4 &,
                                       cudaStream_t);
template void launch_galerkin4<float>(const Cx<float> *, double, const Cx<float> *, Cx<double> *, const Block4 &,
                                      cudaStream_t);

template <typename RY, typename RV>
void launch_coarse4_apply(const Cx<RY> *Y, const Cx<RV> *in, Cx<RV> *out, const Coarse4 &g, const Cx<RV> *b,
                          double a, double c, cudaStream_t s, int nvec, const double *shift) {
  const int qp = std::max(1, std::min(8, 512 / g.N));
  const size_t smem = (size_t)(9 + qp) * g.N * sizeof(Cx<RY>);
  coarse4_apply_kernel<RY, RV><<<dim3((unsigned int)g.nsites, nvec), qp * g.N, smem, s>>>(
      Y, in, out, g, b, (RV)a, (RV)c, g.nsites * g.N, shift);
  MG_LAUNCHED();
}

// The same apply with the operator stored in FP16 (one 32-bit word per complex entry, the real
// part in the low half; [j][dir][col][row] as Y) and the vectors and sums in FP32: half the
// bytes of the FP32 operator, for coarse solves whose tolerance is far looser than the FP16
// rounding (2^-11 of each entry)
__global__ void coarse4_apply_h_kernel(const unsigned int *__restrict__ Yh, const Cx<float> *__restrict__ in,
                                       Cx<float> *__restrict__ out, Coarse4 g, const Cx<float> *__restrict__ b,
                                       float a, float c) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int N = g.N;
  const int QP = blockDim.x / N;
  Cx<float> *xs = reinterpret_cast<Cx<float> *>(sm_raw);  // [9][N]
  Cx<float> *red = xs + 9 * N;                             // [QP][N]
  const int j = blockIdx.x;
  int jc[4];
  {
    int r = j;
    for (int mu = 0; mu < 4; ++mu) {
      jc[mu] = r % g.nb[mu];
      r /= g.nb[mu];
    }
  }
  for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
    const int dir = e / N, col = e - dir * N;
    int src = j;
    if (dir != 0) {
      const int mu = (dir - 1) >> 1;
      int cc[4] = {jc[0], jc[1], jc[2], jc[3]};
      cc[mu] = ((dir - 1) & 1) == 0 ? (cc[mu] + 1) % g.nb[mu] : (cc[mu] + g.nb[mu] - 1) % g.nb[mu];
      src = cc[0] + g.nb[0] * (cc[1] + g.nb[1] * (cc[2] + g.nb[2] * cc[3]));
    }
    xs[e] = in[(long long)src * N + col];
  }
  __syncthreads();
  const int row = threadIdx.x % N, q = threadIdx.x / N;
  const unsigned int *Yj = Yh + (long long)j * 9 * N * N;
  float re = 0.f, im = 0.f;
#pragma unroll 4
  for (int p = q; p < 9 * N; p += QP) {
    const unsigned int w = Yj[(long long)p * N + row];
    const float2 y = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    const Cx<float> xv = xs[p];
    re += y.x * xv.re - y.y * xv.im;
    im += y.x * xv.im + y.y * xv.re;
  }
  red[q * N + row] = mk(re, im);
  __syncthreads();
  if (q == 0) {
    float sre = 0.f, sim = 0.f;
    for (int i = 0; i < QP; ++i) {
      sre += red[i * N + row].re;
      sim += red[i * N + row].im;
    }
    Cx<float> o = mk(a * sre, a * sim);
    if (b != nullptr) {
      const Cx<float> bb = b[(long long)j * N + row];
      o = mk(o.re + c * bb.re, o.im + c * bb.im);
    }
    out[(long long)j * N + row] = o;
  }
}

__global__ void pack_half2_kernel(const Cx<double> *__restrict__ in, unsigned int *__restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const __half2 h = __floats2half2_rn((float)in[i].re, (float)in[i].im);
  out[i] = *reinterpret_cast<const unsigned int *>(&h);
}

void launch_pack_half2(const Cx<double> *in, unsigned int *out, long long n, cudaStream_t s) {
  pack_half2_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  MG_LAUNCHED();
}

void launch_coarse4_apply_h(const unsigned int *Yh, const Cx<float> *in, Cx<float> *out, const Coarse4 &g,
                            const Cx<float> *b, double a, double c, cudaStream_t s) {
  const int qp = std::max(1, std::min(8, 512 / g.N));
  const size_t smem = (size_t)(9 + qp) * g.N * sizeof(Cx<float>);
  coarse4_apply_h_kernel<<<(unsigned int)g.nsites, qp * g.N, smem, s>>>(Yh, in, out, g, b, (float)a, (float)c);
  MG_LAUNCHED();
}

void launch_block_invert4(const Cx<double> *Y, Cx<double> *Minv, const Coarse4 &g, int *info, cudaStream_t s) {
  const size_t smem = (size_t)g.N * 2 * g.N * sizeof(Cx<double>);
  static bool attr = false;
  if (!attr) {
    MG_CUDA(cudaFuncSetAttribute(block_invert4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  block_invert4_kernel<<<(unsigned int)g.nsites, 256, smem, s>>>(Y, Minv, g.N, info);
  MG_LAUNCHED();
}

template <typename R>
void launch_block_apply4(const Cx<R> *Minv, const Cx<double> *r, Cx<double> *z, const Coarse4 &g, cudaStream_t s,
                         int nvec) {
  block_apply4_kernel<R, double><<<dim3((unsigned int)g.nsites, nvec), 64, 0, s>>>(Minv, r, z, g.N, g.nsites * g.N);
  MG_LAUNCHED();
}

void launch_block_apply4_32(const Cx<float> *Minv, const Cx<float> *r, Cx<float> *z, const Coarse4 &g,
                            cudaStream_t s, int nvec) {
  block_apply4_kernel<float, float><<<dim3((unsigned int)g.nsites, nvec), 64, 0, s>>>(Minv, r, z, g.N,
                                                                                     g.nsites * g.N);
  MG_LAUNCHED();
}

// the same step with kSplit consecutive lanes per element, each summing the basis vectors
// j = lane, lane + kSplit, ... (the coarse vectors are short: one thread per element left most
// SMs without work while every thread walked the whole basis)
constexpr int kSplit = 4;

//
// LOOP: the step of a graph-replayed loop: k = ctl[1], W_k = Wb + k n and Z_k = Zb + k n, the new
// direction's inputs are w = wt and z = r (the unpreconditioned residual itself, so no copy)
template <typename VT, bool LOOP>
__global__ void gcr_update_split_kernel(const Cx<VT> *__restrict__ W, Cx<VT> *__restrict__ Wk_,
                                        const Cx<VT> *__restrict__ Z, Cx<VT> *__restrict__ Zk_, int k_host,
                                        const int *__restrict__ ctl, const Cx<VT> *__restrict__ wt,
                                        const double *__restrict__ dots, double *__restrict__ state,
                                        Cx<VT> *__restrict__ x, Cx<VT> *__restrict__ r, long long n) {
  __shared__ double coef[3];
  const int k = LOOP ? ctl[1] : k_host;
  Cx<VT> *Wk = LOOP ? Wk_ + (long long)k * n : Wk_, *Zk = LOOP ? Zk_ + (long long)k * n : Zk_;
  if (threadIdx.x == 0) {
    const double nw0 = dots[2 * k];
    double nw2 = nw0;
    for (int j = 0; j < k; ++j) nw2 -= dots[2 * j] * dots[2 * j] + dots[2 * j + 1] * dots[2 * j + 1];
    double inv = 0.0, are = 0.0, aim = 0.0;
    if (nw2 > 1e-28 * nw0) {
      inv = 1.0 / sqrt(nw2);
      are = dots[2 * k + 2] * inv;
      aim = dots[2 * k + 3] * inv;
    }
    coef[0] = inv;
    coef[1] = are;
    coef[2] = aim;
    if (blockIdx.x == 0) state[0] = fmax(dots[2 * k + 4] - (are * are + aim * aim), 0.0);
  }
  __syncthreads();
  const VT inv = (VT)coef[0];
  const Cx<VT> alpha = mk((VT)coef[1], (VT)coef[2]), malpha = mk((VT)-coef[1], (VT)-coef[2]);
  const int sub = threadIdx.x % kSplit, lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * (blockDim.x / kSplit);
  long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / kSplit;
  // i0, the warp's first element, steers the loop: every lane of the warp takes part in every
  // shuffle, and lanes past the end only contribute zeros
  for (long long i0 = i - lane / kSplit; i0 < n; i0 += stride, i += stride) {
    const bool valid = i < n;
    Cx<VT> pw = mk((VT)0, (VT)0), pz = mk((VT)0, (VT)0);
    for (int j = sub; valid && j < k; j += kSplit) {
      const Cx<VT> bj = mk((VT)-dots[2 * j], (VT)-dots[2 * j + 1]);
      cmac(pw, bj, W[(long long)j * n + i]);
      cmac(pz, bj, Z[(long long)j * n + i]);
    }
#pragma unroll
    for (int o = kSplit / 2; o > 0; o >>= 1) {
      pw.re += __shfl_xor_sync(0xffffffffu, pw.re, o);
      pw.im += __shfl_xor_sync(0xffffffffu, pw.im, o);
      pz.re += __shfl_xor_sync(0xffffffffu, pz.re, o);
      pz.im += __shfl_xor_sync(0xffffffffu, pz.im, o);
    }
    if (valid && sub == 0) {
      Cx<VT> ri = r[i];
      const Cx<VT> w = inv * ((LOOP ? wt[i] : Wk[i]) + pw), z = inv * ((LOOP ? ri : Zk[i]) + pz);
      Wk[i] = w;
      Zk[i] = z;
      cmac(x[i], alpha, z);
      cmac(ri, malpha, w);
      r[i] = ri;
    }
  }
}

template <typename VT>
static void gcr_update_dev_any(const Cx<VT> *W, Cx<VT> *Wk, const Cx<VT> *Z, Cx<VT> *Zk, int k, const double *dots,
                               double *state, Cx<VT> *x, Cx<VT> *r, long long n, cudaStream_t s) {
  if (sizeof(VT) == 4 && std::getenv("MG_COARSE4_UPDATE_ONE") == nullptr) {
    // kSplit threads per element in blocks of 256
    long long b = (n * kSplit + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    gcr_update_split_kernel<VT, false><<<(unsigned int)(b < 1 ? 1 : b), 256, 0, s>>>(W, Wk, Z, Zk, k, nullptr, nullptr,
                                                                                     dots, state, x, r, n);
    MG_LAUNCHED();
    return;
  }
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  gcr_update_dev_kernel<VT><<<(unsigned int)(b < 1 ? 1 : b), 256, 0, s>>>(W, Wk, Z, Zk, k, dots, state, x, r, n);
  MG_LAUNCHED();
}

void launch_gcr_update_dev(const Cx<double> *W, Cx<double> *Wk, const Cx<double> *Z, Cx<double> *Zk, int k,
                           const double *dots, double *state, Cx<double> *x, Cx<double> *r, long long n,
                           cudaStream_t s) {
  gcr_update_dev_any<double>(W, Wk, Z, Zk, k, dots, state, x, r, n, s);
}

void launch_gcr_update_dev(const Cx<float> *W, Cx<float> *Wk, const Cx<float> *Z, Cx<float> *Zk, int k,
                           const double *dots, double *state, Cx<float> *x, Cx<float> *r, long long n,
                           cudaStream_t s) {
  gcr_update_dev_any<float>(W, Wk, Z, Zk, k, dots, state, x, r, n, s);
}

void launch_gcr_update_loop(Cx<float> *W, Cx<float> *Z, const Cx<float> *wt, const int *ctl, const double *dots,
                            double *state, Cx<float> *x, Cx<float> *r, long long n, cudaStream_t s) {
  long long b = (n * kSplit + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  gcr_update_split_kernel<float, true><<<(unsigned int)(b < 1 ? 1 : b), 256, 0, s>>>(W, W, Z, Z, 0, ctl, wt, dots,
                                                                                    state, x, r, n);
  MG_LAUNCHED();
}

// Control of the graph-replayed coarse GCR (ctl[0] iterations so far, ctl[1] the basis index
// k; st[0] the residual estimate, st[1] |b|^2, st[3] the iteration count as a double for the
// host's one read per restart cycle). The cycle-start kernel runs before the WHILE node and
// sets its condition; the control kernel ends every iteration.
__global__ void coarse4_cycle_start_kernel(int *ctl, const double *st, int max_iter,
                                           cudaGraphConditionalHandle handle) {
  ctl[1] = 0;
  cudaGraphSetConditional(handle, (st[1] > 0.0 && ctl[0] < max_iter) ? 1u : 0u);
}

__global__ void coarse4_control_kernel(int *ctl, double *st, double tol2_rel, int restart, int max_iter,
                                       cudaGraphConditionalHandle handle) {
  const int it = ctl[0] + 1, k = ctl[1] + 1;
  ctl[0] = it;
  ctl[1] = k;
  st[3] = (double)it;
  // a NaN estimate ends the loop; the host finds it in the true residual
  const bool go = st[0] > tol2_rel * st[1] && k < restart && it < max_iter;
  cudaGraphSetConditional(handle, go ? 1u : 0u);
}

// batched form: stv[2 v] = |b_v|^2 (the first estimate), stv[2 v + 1] = tol^2 |b_v|^2, act[v] = b_v != 0
__global__ void coarse4_batch_init_kernel(const double *bn2, double tol2_rel, int nb, double *stv, int *act) {
  const int v = threadIdx.x;
  if (v >= nb) return;
  stv[2 * v] = bn2[v];
  stv[2 * v + 1] = tol2_rel * bn2[v];
  act[v] = bn2[v] > 0.0 ? 1 : 0;
}

// starts a restart cycle of the batched loop (k = 0); it runs while a vector is active and the
// iteration limit is not reached
__global__ void coarse4_batch_cycle_start_kernel(int *ctl, const int *act, int nb, int max_iter,
                                                 cudaGraphConditionalHandle handle) {
  ctl[1] = 0;
  int any = 0;
  for (int v = 0; v < nb; ++v) any |= act[v];
  cudaGraphSetConditional(handle, (any && ctl[0] < max_iter) ? 1u : 0u);
}

void launch_coarse4_batch_init(const double *bn2, double tol2_rel, int nb, double *stv, int *act, cudaStream_t s) {
  coarse4_batch_init_kernel<<<1, 32, 0, s>>>(bn2, tol2_rel, nb, stv, act);
  MG_LAUNCHED();
}

void launch_coarse4_batch_cycle_start(int *ctl, const int *act, int nb, int max_iter, cudaGraphConditionalHandle h,
                                      cudaStream_t s) {
  coarse4_batch_cycle_start_kernel<<<1, 1, 0, s>>>(ctl, act, nb, max_iter, h);
  MG_LAUNCHED();
}

void launch_coarse4_cycle_start(int *ctl, const double *st, int max_iter, cudaGraphConditionalHandle h,
                                cudaStream_t s) {
  coarse4_cycle_start_kernel<<<1, 1, 0, s>>>(ctl, st, max_iter, h);
  MG_LAUNCHED();
}

void launch_coarse4_control(int *ctl, double *st, double tol2_rel, int restart, int max_iter,
                            cudaGraphConditionalHandle h, cudaStream_t s) {
  coarse4_control_kernel<<<1, 1, 0, s>>>(ctl, st, tol2_rel, restart, max_iter, h);
  MG_LAUNCHED();
}

void launch_precondition4(const Cx<double> *Y, const Cx<double> *Minv, Cx<double> *Yt, const Coarse4 &g,
                          cudaStream_t s) {
  const long long total = g.nsites * 9LL * g.N * g.N;
  precondition4_kernel<<<grid_for(total, 256), 256, 0, s>>>(Y, Minv, Yt, g);
  MG_LAUNCHED();
}

template <typename R>
void launch_dot_norm_batch(const Cx<R> *a, const Cx<R> *b, long long n, int nvec, double *out, double *partials,
                           unsigned int *tickets, int max_blocks, cudaStream_t s) {
  dot_norm_batch_kernel<R><<<dim3(reduce_blocks(n, max_blocks), nvec), kReduceThreads, 0, s>>>(a, b, n, partials, out,
                                                                                                tickets);
  MG_LAUNCHED();
}

template <typename R>
void launch_mr_update_batch(const double *sc, double omega, Cx<R> *x, Cx<R> *r, const Cx<R> *Ar, long long n,
                            int nvec, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 8) b = 152LL * 8;
  mr_update_batch_kernel<R><<<dim3((unsigned int)b, nvec), 256, 0, s>>>(sc, omega, x, r, Ar, n);
  MG_LAUNCHED();
}

void launch_coarse4_to_canonical(const Cx<double> *Yi, Cx<double> *Yc, const Coarse4 &g, cudaStream_t s) {
  const long long total = g.nsites * 9 * g.N * g.N;
  coarse4_to_canonical_kernel<<<grid_for(total, 256), 256, 0, s>>>(Yi, Yc, total, g.N);
  MG_LAUNCHED();
}

void launch_prolongator4_to_canonical(const Cx<double> *V, Cx<double> *out, const Block4 &g, cudaStream_t s) {
  const long long nsites = (long long)g.nblocks * g.bvol;
  prolongator4_to_canonical_kernel<<<grid_for(2LL * g.Nv * nsites * 12, 256), 256, 0, s>>>(V, out, g, nsites);
  MG_LAUNCHED();
}

template void launch_restrict4<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, const Block4 &,
                                       cudaStream_t, int);
template void launch_restrict4<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, const Block4 &, cudaStream_t,
                                      int);
template void launch_prolong4<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, const Block4 &,
                                      cudaStream_t, int);
template void launch_prolong4<float>(const Cx<float> *, const Cx<float> *, Cx<float> *, const Block4 &, cudaStream_t,
                                     int);
template void launch_coarse4_apply<double, double>(const Cx<double> *, const Cx<double> *, Cx<double> *,
                                                   const Coarse4 &, const Cx<double> *, double, double, cudaStream_t,
                                                   int, const double *);
template void launch_coarse4_apply<float, float>(const Cx<float> *, const Cx<float> *, Cx<float> *, const Coarse4 &,
                                                 const Cx<float> *, double, double, cudaStream_t, int, const double *);
template void launch_coarse4_apply<float, double>(const Cx<float> *, const Cx<double> *, Cx<double> *,
                                                  const Coarse4 &, const Cx<double> *, double, double, cudaStream_t,
                                                  int, const double *);
template void launch_dot_norm_batch<float>(const Cx<float> *, const Cx<float> *, long long, int, double *, double *,
                                           unsigned int *, int, cudaStream_t);
template void launch_dot_norm_batch<double>(const Cx<double> *, const Cx<double> *, long long, int, double *,
                                            double *, unsigned int *, int, cudaStream_t);
template void launch_mr_update_batch<float>(const double *, double, Cx<float> *, Cx<float> *, const Cx<float> *,
                                            long long, int, cudaStream_t);
template void launch_mr_update_batch<double>(const double *, double, Cx<double> *, Cx<double> *, const Cx<double> *,
                                             long long, int, cudaStream_t);
template void launch_block_apply4<double>(const Cx<double> *, const Cx<double> *, Cx<double> *, const Coarse4 &,
                                          cudaStream_t, int);
template void launch_block_apply4<float>(const Cx<float> *, const Cx<double> *, Cx<double> *, const Coarse4 &,
                                         cudaStream_t, int);

}  // namespace mg
