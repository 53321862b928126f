// Fine Wilson operator on 2d U(1) with half-precision storage (paper, definition of D following
// Eq. 1; diagonal d + m, periodic), the FP16 storage of the mixed-precision scheme:
//
//   spinor field: per site the two spin components as IEEE half pairs (re, im), scaled by a
//   per-site FP32 norm nu_x = max(|Re psi_0|, |Im psi_0|, |Re psi_1|, |Im psi_1|):
//       psi_x = nu_x * (h_x0, h_x1),  |h| <= 1,
//   stored as [V][2] half2 followed by [V] float (12 bytes per site);
//   links: U_x^mu = (cos, sin) as half pairs, [V][2] half2 (8 bytes per site; |U| = 1 needs no norm).
//
// Arithmetic is FP32: every load is scaled back to FP32, the stencil is the FP32 one, and the
// output site is rescaled by its own max component before it is rounded to half. One apply
// moves 12 + 8 + 12 = 32 bytes per site (48 in FP32).
//
// The same storage serves the fine level of FP32 V-cycles in MG_FP16 contexts: the MR
// smoother's vectors r and A r (read at five sites per iteration) and the links are half,
// the smoother's iterate x, the cycle's input and the residual handed to the restriction stay
// FP32, every sum is FP32. A batch of half fields is stored field after field, 12 V bytes each.
#include <cuda_fp16.h>

#include "kernels.h"
#include "mr.cuh"
#include "wilson.cuh"

namespace mg {

namespace {

__device__ __forceinline__ Cx<float> h2c(__half2 h, float nu) {
  const float2 f = __half22float2(h);
  return mk(f.x * nu, f.y * nu);
}

__device__ __forceinline__ Pair<float> load_site(const __half2 *d, const float *nrm, long long x) {
  const float nu = nrm[x];
  const uint2 raw = reinterpret_cast<const uint2 *>(d)[x];  // both spin components in one 8-byte load
  __half2 a, b;
  memcpy(&a, &raw.x, 4);
  memcpy(&b, &raw.y, 4);
  Pair<float> p;
  p.a = h2c(a, nu);
  p.b = h2c(b, nu);
  return p;
}

__device__ __forceinline__ void store_site(__half2 *d, float *nrm, long long x, Cx<float> o0, Cx<float> o1) {
  const float nu = fmaxf(fmaxf(fabsf(o0.re), fabsf(o0.im)), fmaxf(fabsf(o1.re), fabsf(o1.im)));
  // sites below 1e-30 (far under any FP32 field's scale here) are stored as zero: no infinite scale
  const float inv = nu > 1e-30f ? __frcp_rn(nu) : 0.f;
  const __half2 a = __floats2half2_rn(o0.re * inv, o0.im * inv);
  const __half2 b = __floats2half2_rn(o1.re * inv, o1.im * inv);
  uint2 raw;
  memcpy(&raw.x, &a, 4);
  memcpy(&raw.y, &b, 4);
  reinterpret_cast<uint2 *>(d)[x] = raw;
  nrm[x] = inv > 0.f ? nu : 0.f;
}

struct Nbr {
  long long p0, p1, m0, m1;  // x+0, x+1, x-0, x-1 (periodic)
};

// 32-bit index arithmetic: lattices hold fewer than 2^28 sites
__device__ __forceinline__ Nbr neighbours(long long x, int L0, int L1) {
  const unsigned int xs = (unsigned int)x, l0 = (unsigned int)L0;
  const unsigned int x1 = xs / l0, x0 = xs - x1 * l0;
  const unsigned int row = x1 * l0;
  Nbr n;
  n.p0 = row + (x0 + 1 == l0 ? 0u : x0 + 1);
  n.m0 = row + (x0 == 0 ? l0 - 1 : x0 - 1);
  n.p1 = (x1 + 1 == (unsigned int)L1 ? 0u : row + l0) + x0;
  n.m1 = (x1 == 0 ? ((unsigned int)L1 - 1) * l0 : row - l0) + x0;
  return n;
}

// D psi at one site in FP32 from the site's own components (s), those of x+0 (f0), x+1 (f1),
// x-0 (g0), x-1 (g1), the forward links U_x^0, U_x^1 and the backward ones U_{x-0}^0, U_{x-1}^1
__device__ __forceinline__ Pair<float> wilson_at(Pair<float> s, Pair<float> f0, Pair<float> f1, Pair<float> g0,
                                                 Pair<float> g1, Cx<float> ux0, Cx<float> ux1, Cx<float> ub0,
                                                 Cx<float> ub1, float diag) {
  const Cx<float> t1 = ux0 * (f0.a - f0.b);                // +0: (1 - s1) U psi(x+0)
  const Cx<float> t2 = cmul_conj(ub0, g0.a + g0.b);        // -0: (1 + s1) U^* psi(x-0)
  const Cx<float> t3 = ux1 * (f1.a + times_i(f1.b));       // +1: (1 - s2) U psi(x+1)
  const Cx<float> t4 = cmul_conj(ub1, g1.a - times_i(g1.b));  // -1: (1 + s2) U^* psi(x-1)
  const Cx<float> hu = mk(t1.re + t2.re + t3.re + t4.re, t1.im + t2.im + t3.im + t4.im);
  const Cx<float> hl = mk(-t1.re + t2.re + t3.im - t4.im, -t1.im + t2.im - t3.re + t4.re);
  Pair<float> o;
  o.a = mk(diag * s.a.re - 0.5f * hu.re, diag * s.a.im - 0.5f * hu.im);
  o.b = mk(diag * s.b.re - 0.5f * hl.re, diag * s.b.im - 0.5f * hl.im);
  return o;
}

__global__ void __launch_bounds__(256, 8) dslash_half_kernel(const __half2 *__restrict__ U,
                                                             const __half2 *__restrict__ in,
                                                             const float *__restrict__ in_nrm,
                                                             __half2 *__restrict__ out, float *__restrict__ out_nrm,
                                                             int L0, int L1, float diag) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long V = (long long)L0 * L1;
  if (x >= V) return;
  const Nbr n = neighbours(x, L0, L1);
  const Pair<float> self = load_site(in, in_nrm, x);
  const Pair<float> f0 = load_site(in, in_nrm, n.p0), f1 = load_site(in, in_nrm, n.p1);
  const Pair<float> g0 = load_site(in, in_nrm, n.m0), g1 = load_site(in, in_nrm, n.m1);
  const Cx<float> ux0 = h2c(U[2 * x], 1.f), ux1 = h2c(U[2 * x + 1], 1.f);
  const Cx<float> ub0 = h2c(U[2 * n.m0], 1.f), ub1 = h2c(U[2 * n.m1 + 1], 1.f);
  const Pair<float> o = wilson_at(self, f0, f1, g0, g1, ux0, ux1, ub0, ub1, diag);
  store_site(out, out_nrm, x, o.a, o.b);
}

// two sites (x0, x0 + 1) of a row per thread, L0 even: the pair's own values, its neighbours in
// rows x1 +- 1 and its forward links are one 16-byte load each (8-byte norm pairs), the two
// sites are each other's x0 neighbours, and only x0 - 1 and x0 + 2 are single loads; the
// per-thread instruction count, which bounds the one-site kernel, is about halved
__device__ __forceinline__ void load_pair2(const __half2 *d, const float *nrm, long long x, Pair<float> &p,
                                           Pair<float> &q) {
  const uint4 raw = reinterpret_cast<const uint4 *>(d)[x >> 1];  // sites x, x + 1 (x even)
  const float2 nu = reinterpret_cast<const float2 *>(nrm)[x >> 1];
  __half2 h[4];
  memcpy(&h[0], &raw.x, 4);
  memcpy(&h[1], &raw.y, 4);
  memcpy(&h[2], &raw.z, 4);
  memcpy(&h[3], &raw.w, 4);
  p.a = h2c(h[0], nu.x);
  p.b = h2c(h[1], nu.x);
  q.a = h2c(h[2], nu.y);
  q.b = h2c(h[3], nu.y);
}

__device__ __forceinline__ void store_pair2(__half2 *d, float *nrm, long long x, const Pair<float> &p,
                                            const Pair<float> &q) {
  const float np = fmaxf(fmaxf(fabsf(p.a.re), fabsf(p.a.im)), fmaxf(fabsf(p.b.re), fabsf(p.b.im)));
  const float nq = fmaxf(fmaxf(fabsf(q.a.re), fabsf(q.a.im)), fmaxf(fabsf(q.b.re), fabsf(q.b.im)));
  const float ip = np > 1e-30f ? __frcp_rn(np) : 0.f, iq = nq > 1e-30f ? __frcp_rn(nq) : 0.f;
  const __half2 h0 = __floats2half2_rn(p.a.re * ip, p.a.im * ip), h1 = __floats2half2_rn(p.b.re * ip, p.b.im * ip);
  const __half2 h2 = __floats2half2_rn(q.a.re * iq, q.a.im * iq), h3 = __floats2half2_rn(q.b.re * iq, q.b.im * iq);
  uint4 raw;
  memcpy(&raw.x, &h0, 4);
  memcpy(&raw.y, &h1, 4);
  memcpy(&raw.z, &h2, 4);
  memcpy(&raw.w, &h3, 4);
  reinterpret_cast<uint4 *>(d)[x >> 1] = raw;
  reinterpret_cast<float2 *>(nrm)[x >> 1] = make_float2(ip > 0.f ? np : 0.f, iq > 0.f ? nq : 0.f);
}

__global__ void __launch_bounds__(256, 6) dslash_half2_kernel(const __half2 *__restrict__ U,
                                                              const __half2 *__restrict__ in,
                                                              const float *__restrict__ in_nrm,
                                                              __half2 *__restrict__ out, float *__restrict__ out_nrm,
                                                              int L0, int L1, float diag) {
  const unsigned int pr = blockIdx.x * blockDim.x + threadIdx.x;  // pair index
  const unsigned int h0 = (unsigned int)L0 >> 1;
  if (pr >= h0 * (unsigned int)L1) return;
  const unsigned int x1 = pr / h0, x0 = 2 * (pr - x1 * h0);
  const unsigned int row = x1 * (unsigned int)L0;
  const long long xa = row + x0;  // even: sites xa (a) and xa + 1 (b)
  const long long up = (x1 + 1 == (unsigned int)L1 ? 0u : row + L0) + x0;
  const long long dn = (x1 == 0 ? ((unsigned int)L1 - 1) * L0 : row - L0) + x0;
  const long long am = row + (x0 == 0 ? L0 - 1 : x0 - 1);                 // a - 0
  const long long bp = row + (x0 + 2 == (unsigned int)L0 ? 0u : x0 + 2);  // b + 0
  Pair<float> sa, sb, ua, ub, da, db;
  load_pair2(in, in_nrm, xa, sa, sb);
  load_pair2(in, in_nrm, up, ua, ub);
  load_pair2(in, in_nrm, dn, da, db);
  const Pair<float> am_v = load_site(in, in_nrm, am), bp_v = load_site(in, in_nrm, bp);
  // links: forward of a and b (one 16-byte load), U^1 of dn and dn + 1 (one 16-byte load), U^0 of a - 0
  const uint4 lf = reinterpret_cast<const uint4 *>(U)[xa >> 1];
  const uint4 ld = reinterpret_cast<const uint4 *>(U)[dn >> 1];
  __half2 f[4], g1, g3;
  memcpy(&f[0], &lf.x, 4);
  memcpy(&f[1], &lf.y, 4);
  memcpy(&f[2], &lf.z, 4);
  memcpy(&f[3], &lf.w, 4);
  memcpy(&g1, &ld.y, 4);
  memcpy(&g3, &ld.w, 4);
  const Cx<float> ua0 = h2c(f[0], 1.f), ua1 = h2c(f[1], 1.f), ub0 = h2c(f[2], 1.f), ub1 = h2c(f[3], 1.f);
  const Cx<float> dna1 = h2c(g1, 1.f), dnb1 = h2c(g3, 1.f);
  const Cx<float> am0 = h2c(U[2 * am], 1.f);
  // a: +0 = b, +1 = ua, -0 = am, -1 = da; backward links U_{a-0}^0 = am0, U_{a-1}^1 = dna1
  const Pair<float> oa = wilson_at(sa, sb, ua, am_v, da, ua0, ua1, am0, dna1, diag);
  // b: +0 = bp, +1 = ub, -0 = a, -1 = db; backward links U_{b-0}^0 = U_a^0, U_{b-1}^1 = dnb1
  const Pair<float> ob = wilson_at(sb, bp_v, ub, sa, db, ub0, ub1, ua0, dnb1, diag);
  store_pair2(out, out_nrm, xa, oa, ob);
}

// complex (FP64 / FP32) spinor field -> half storage with per-site norms, and back
template <typename R>
__global__ void spinor_to_half_kernel(const Cx<R> *__restrict__ in, __half2 *__restrict__ out,
                                      float *__restrict__ nrm, long long V) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= V) return;
  const Cx<float> a = cvt<float, R>(in[2 * x]), b = cvt<float, R>(in[2 * x + 1]);
  store_site(out, nrm, x, a, b);
}

template <typename R>
__global__ void spinor_from_half_kernel(const __half2 *__restrict__ in, const float *__restrict__ nrm,
                                        Cx<R> *__restrict__ out, long long V) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= V) return;
  const Pair<float> p = load_site(in, nrm, x);
  out[2 * x] = cvt<R, float>(p.a);
  out[2 * x + 1] = cvt<R, float>(p.b);
}

template <typename R>
__global__ void links_to_half_kernel(const Cx<R> *__restrict__ in, __half2 *__restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = __floats2half2_rn((float)in[i].re, (float)in[i].im);
}

// ---- the fine level of FP32 V-cycles with half storage ----
struct HalfField {
  __half2 *h;
  float *n;
};

// field v of a batch at base (12 V bytes per field: V half2 pairs, then V norms)
__device__ __forceinline__ HalfField half_field(void *base, long long V, int v) {
  char *p = static_cast<char *>(base) + (long long)v * 12 * V;
  return {reinterpret_cast<__half2 *>(p), reinterpret_cast<float *>(p + 8 * V)};
}

__device__ __forceinline__ Pair<float> load_pair(const Cx<float> *f, long long x) {
  return reinterpret_cast<const Pair<float> *>(f)[x];
}

// One fused MR iteration on the fine Wilson level (the FP32 kernel's scheme with half r and A r).
// STEP = false: r_new = b (rounded to half) and Ar_new = A b, partials of (<A b, b>, |A b|^2).
// STEP = true: alpha from part_in, x (+)= alpha r_old at the site, r_new = r_old - alpha Ar_old
// (formed at the five sites the stencil needs), Ar_new = A r_new, partials to part_out.
template <bool STEP>
__global__ void __launch_bounds__(256) mr_wilson_half_kernel(const __half2 *__restrict__ U,
                                                             const Cx<float> *__restrict__ b, void *r_old,
                                                             void *Ar_old, const float *part_in, int nb_in,
                                                             double omega, Cx<float> *x, int x_init, void *r_new,
                                                             void *Ar_new, int L0, int L1, float diag,
                                                             float *part_out, const double *shift) {
  __shared__ float sh[32 * 3];
  const int v = blockIdx.y;
  if (shift != nullptr) diag += (float)shift[v];
  const long long V = (long long)L0 * L1;
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = s < V;
  const Cx<float> z = mk(0.f, 0.f);
  Pair<float> w[5], a[5];  // self, +0, +1, -0, -1
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k].a = w[k].b = a[k].a = a[k].b = z;
  Pair<float> xs;
  xs.a = xs.b = z;
  Cx<float> ux0 = z, ux1 = z, ub0 = z, ub1 = z;
  if (live) {
    const Nbr n = neighbours(s, L0, L1);
    const long long nb[5] = {s, n.p0, n.p1, n.m0, n.m1};
    if (STEP) {
      const HalfField ro = half_field(r_old, V, v), ao = half_field(Ar_old, V, v);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        w[k] = load_site(ro.h, ro.n, nb[k]);
        a[k] = load_site(ao.h, ao.n, nb[k]);
      }
      if (!x_init) xs = load_pair(x + 2 * V * v, s);
    } else {
      const Cx<float> *bv = b + 2 * V * v;
#pragma unroll
      for (int k = 0; k < 5; ++k) w[k] = load_pair(bv, nb[k]);
    }
    ux0 = h2c(U[2 * s], 1.f);
    ux1 = h2c(U[2 * s + 1], 1.f);
    ub0 = h2c(U[2 * n.m0], 1.f);
    ub1 = h2c(U[2 * n.m1 + 1], 1.f);
  }
  Cx<float> alpha = z;
  if (STEP) alpha = mr_alpha<float>(part_in + 3LL * nb_in * v, nb_in, omega, sh);  // all threads of the block
  float acc[3] = {0.f, 0.f, 0.f};
  if (live) {
    if (STEP) {
      cmac(xs.a, alpha, w[0].a);
      cmac(xs.b, alpha, w[0].b);
      reinterpret_cast<Pair<float> *>(x + 2 * V * v)[s] = xs;
      const Cx<float> ma = mk(-alpha.re, -alpha.im);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        w[k].a = mr_step(w[k].a, a[k].a, ma);
        w[k].b = mr_step(w[k].b, a[k].b, ma);
      }
    }
    const HalfField rn = half_field(r_new, V, v), an = half_field(Ar_new, V, v);
    store_site(rn.h, rn.n, s, w[0].a, w[0].b);
    const Pair<float> o = wilson_at(w[0], w[1], w[2], w[3], w[4], ux0, ux1, ub0, ub1, diag);
    store_site(an.h, an.n, s, o.a, o.b);
    const Cx<float> s0 = w[0].a, s1 = w[0].b, a0 = o.a, a1 = o.b;
    acc[0] = a0.re * s0.re + a0.im * s0.im + a1.re * s1.re + a1.im * s1.im;
    acc[1] = a0.re * s0.im - a0.im * s0.re + a1.re * s1.im - a1.im * s1.re;
    acc[2] = a0.re * a0.re + a0.im * a0.im + a1.re * a1.re + a1.im * a1.im;
  }
  mr_publish<float>(acc, part_out + 3LL * gridDim.x * v, sh);
}

// last MR step: x (+)= alpha r_old, and r_out = r_old - alpha Ar_old in FP32 when requested
__global__ void mr_last_half_kernel(void *r_old, void *Ar_old, const float *part_in, int nb_in, double omega,
                                    Cx<float> *__restrict__ x, int x_init, Cx<float> *r_out, long long V) {
  __shared__ float sh[32 * 3];
  const int v = blockIdx.y;
  const Cx<float> alpha = mr_alpha<float>(part_in + 3LL * nb_in * v, nb_in, omega, sh);
  const Cx<float> ma = mk(-alpha.re, -alpha.im);
  const HalfField ro = half_field(r_old, V, v), ao = half_field(Ar_old, V, v);
  Pair<float> *xv = reinterpret_cast<Pair<float> *>(x + 2 * V * v);
  Pair<float> *rv = r_out != nullptr ? reinterpret_cast<Pair<float> *>(r_out + 2 * V * v) : nullptr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const Pair<float> ri = load_site(ro.h, ro.n, i);
    Pair<float> xs;
    if (x_init) {
      xs.a = xs.b = mk(0.f, 0.f);
    } else {
      xs = xv[i];
    }
    cmac(xs.a, alpha, ri.a);
    cmac(xs.b, alpha, ri.b);
    xv[i] = xs;
    if (rv != nullptr) {
      const Pair<float> ai = load_site(ao.h, ao.n, i);
      Pair<float> ro2;
      ro2.a = mr_step(ri.a, ai.a, ma);
      ro2.b = mr_step(ri.b, ai.b, ma);
      rv[i] = ro2;
    }
  }
}

// out = a D in + c b on FP32 vectors with half links (the cycle's residual), batched with
// stride 2 V complex; diagonal + shift[v] when a shift array is given
__global__ void __launch_bounds__(256, 8) dslash_hl_kernel(const __half2 *__restrict__ U,
                                                           const Cx<float> *__restrict__ in,
                                                           Cx<float> *__restrict__ out, int L0, int L1, float diag,
                                                           const Cx<float> *__restrict__ b, float a, float c,
                                                           const double *__restrict__ shift) {
  const int v = blockIdx.y;
  if (shift != nullptr) diag += (float)shift[v];
  const long long V = (long long)L0 * L1;
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= V) return;
  in += 2 * V * v;
  out += 2 * V * v;
  const Nbr n = neighbours(x, L0, L1);
  const Pair<float> o = wilson_at(load_pair(in, x), load_pair(in, n.p0), load_pair(in, n.p1), load_pair(in, n.m0),
                                  load_pair(in, n.m1), h2c(U[2 * x], 1.f), h2c(U[2 * x + 1], 1.f),
                                  h2c(U[2 * n.m0], 1.f), h2c(U[2 * n.m1 + 1], 1.f), diag);
  Pair<float> res;
  if (b != nullptr) {
    const Pair<float> bb = load_pair(b + 2 * V * v, x);
    res.a = mk(a * o.a.re + c * bb.a.re, a * o.a.im + c * bb.a.im);
    res.b = mk(a * o.b.re + c * bb.b.re, a * o.b.im + c * bb.b.im);
  } else {
    res.a = mk(a * o.a.re, a * o.a.im);
    res.b = mk(a * o.b.re, a * o.b.im);
  }
  reinterpret_cast<Pair<float> *>(out)[x] = res;
}

}  // namespace

void launch_dslash_half(const void *U, const void *in, void *out, Geo2 g, double diag, cudaStream_t s) {
  const long long V = g.nsites;
  const __half2 *ih = static_cast<const __half2 *>(in);
  __half2 *oh = static_cast<__half2 *>(out);
  if ((g.L0 & 1) == 0) {
    dslash_half2_kernel<<<grid_for(V / 2, 256), 256, 0, s>>>(static_cast<const __half2 *>(U), ih,
                                                             reinterpret_cast<const float *>(ih + 2 * V), oh,
                                                             reinterpret_cast<float *>(oh + 2 * V), g.L0, g.L1,
                                                             (float)diag);
    MG_LAUNCHED();
    return;
  }
  dslash_half_kernel<<<grid_for(V, 256), 256, 0, s>>>(static_cast<const __half2 *>(U), ih,
                                                      reinterpret_cast<const float *>(ih + 2 * V), oh,
                                                      reinterpret_cast<float *>(oh + 2 * V), g.L0, g.L1, (float)diag);
  MG_LAUNCHED();
}

// what: 0 spinor to half, 1 spinor from half, 2 links to half; precision of the complex side
void launch_half_convert(int what, int precision, const void *in, void *out, long long nsites, cudaStream_t s) {
  const unsigned int grid = grid_for(what == 2 ? 2 * nsites : nsites, 256);
  if (what == 0) {
    __half2 *o = static_cast<__half2 *>(out);
    float *nrm = reinterpret_cast<float *>(o + 2 * nsites);
    if (precision == MG_FP64)
      spinor_to_half_kernel<double><<<grid, 256, 0, s>>>(static_cast<const Cx<double> *>(in), o, nrm, nsites);
    else
      spinor_to_half_kernel<float><<<grid, 256, 0, s>>>(static_cast<const Cx<float> *>(in), o, nrm, nsites);
  } else if (what == 1) {
    const __half2 *i = static_cast<const __half2 *>(in);
    const float *nrm = reinterpret_cast<const float *>(i + 2 * nsites);
    if (precision == MG_FP64)
      spinor_from_half_kernel<double><<<grid, 256, 0, s>>>(i, nrm, static_cast<Cx<double> *>(out), nsites);
    else
      spinor_from_half_kernel<float><<<grid, 256, 0, s>>>(i, nrm, static_cast<Cx<float> *>(out), nsites);
  } else {
    if (precision == MG_FP64)
      links_to_half_kernel<double><<<grid, 256, 0, s>>>(static_cast<const Cx<double> *>(in),
                                                        static_cast<__half2 *>(out), 2 * nsites);
    else
      links_to_half_kernel<float><<<grid, 256, 0, s>>>(static_cast<const Cx<float> *>(in),
                                                       static_cast<__half2 *>(out), 2 * nsites);
  }
  MG_LAUNCHED();
}

int mr_half_grid(Geo2 g) { return (int)grid_for(g.nsites, 256); }

void launch_mr_iteration_half(const void *U16, Geo2 g, double diag, const double *shift, bool step,
                              const Cx<float> *b, void *r_old, void *Ar_old, const float *part_in, double omega,
                              Cx<float> *x, bool x_init, void *r_new, void *Ar_new, float *part_out,
                              long long part_capacity, cudaStream_t s, int nvec) {
  if (nvec > 128) fail(MG_ERR_UNSUPPORTED, "MR batch larger than 128 vectors");
  const int nb = mr_half_grid(g);
  if (3LL * nb * nvec > part_capacity) fail(MG_ERR_STATE, "MR reduction workspace too small");
  const dim3 grid(nb, nvec);
  const __half2 *U = static_cast<const __half2 *>(U16);
  if (step)
    mr_wilson_half_kernel<true><<<grid, 256, 0, s>>>(U, nullptr, r_old, Ar_old, part_in, nb, omega, x, x_init ? 1 : 0,
                                                     r_new, Ar_new, g.L0, g.L1, (float)diag, part_out, shift);
  else
    mr_wilson_half_kernel<false><<<grid, 256, 0, s>>>(U, b, nullptr, nullptr, nullptr, nb, omega, nullptr, 0, r_new,
                                                      Ar_new, g.L0, g.L1, (float)diag, part_out, shift);
  MG_LAUNCHED();
}

void launch_mr_last_half(void *r_old, void *Ar_old, const float *part_in, double omega, Cx<float> *x, bool x_init,
                         Cx<float> *r_out, Geo2 g, cudaStream_t s, int nvec) {
  long long blocks = (g.nsites + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  mr_last_half_kernel<<<dim3((unsigned int)(blocks < 1 ? 1 : blocks), nvec), 256, 0, s>>>(
      r_old, Ar_old, part_in, mr_half_grid(g), omega, x, x_init ? 1 : 0, r_out, g.nsites);
  MG_LAUNCHED();
}

void launch_dslash_hl(const void *U16, const Cx<float> *in, Cx<float> *out, Geo2 g, double diag, const Cx<float> *b,
                      double a, double c, cudaStream_t s, int nvec, const double *shift) {
  dslash_hl_kernel<<<dim3(grid_for(g.nsites, 256), nvec), 256, 0, s>>>(static_cast<const __half2 *>(U16), in, out,
                                                                      g.L0, g.L1, (float)diag, b, (float)a, (float)c,
                                                                      shift);
  MG_LAUNCHED();
}

}  // namespace mg
