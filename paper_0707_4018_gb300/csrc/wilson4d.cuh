// Hopping terms of the 4d Wilson operator in the DeGrand-Rossi basis (paper,
// definition of D following Eq. 1, four spins and SU(3) colour). Every
// gamma_mu = [[0, A_mu], [A_mu^dagger, 0]] in 2 x 2 spin blocks, A_mu unitary:
//   (1 - gamma_mu) psi = (h, -A_mu^dagger h),  h = psi_up - A_mu psi_dn
//   (1 + gamma_mu) psi = (h,  A_mu^dagger h),  h = psi_up + A_mu psi_dn
//   mu = 0: A = [[0, i], [i, 0]]    mu = 1: A = [[0, -1], [1, 0]]
//   mu = 2: A = [[i, 0], [0, -i]]   mu = 3: A = [[1, 0], [0, 1]]
// A spinor is 12 complex, index 3 * spin + colour; a link is 9 complex, row-major.
#pragma once

#include "common.cuh"

namespace mg {

// A_mu psi_dn for the two lower spins (d0, d1) = (psi_2, psi_3) of one colour
template <typename R, int MU>
__device__ __forceinline__ void a_times(Cx<R> d0, Cx<R> d1, Cx<R> &o0, Cx<R> &o1) {
  if (MU == 0) { o0 = times_i(d1); o1 = times_i(d0); }
  if (MU == 1) { o0 = mk(-d1.re, -d1.im); o1 = d0; }
  if (MU == 2) { o0 = times_i(d0); o1 = mk(d1.im, -d1.re); }
  if (MU == 3) { o0 = d0; o1 = d1; }
}

// A_mu^dagger t for the two upper-spin components (t0, t1) of one colour
template <typename R, int MU>
__device__ __forceinline__ void adag_times(Cx<R> t0, Cx<R> t1, Cx<R> &o0, Cx<R> &o1) {
  if (MU == 0) { o0 = mk(t1.im, -t1.re); o1 = mk(t0.im, -t0.re); }  // (-i t1, -i t0)
  if (MU == 1) { o0 = t1; o1 = mk(-t0.re, -t0.im); }                // (t1, -t0)
  if (MU == 2) { o0 = mk(t0.im, -t0.re); o1 = times_i(t1); }        // (-i t0, i t1)
  if (MU == 3) { o0 = t0; o1 = t1; }
}

// One hop into the accumulators: FWD: (1 - gamma_mu) U psi_nbr; else
// (1 + gamma_mu) U^dagger psi_nbr (the -1/2 is applied at the end).
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void hop4(const Cx<R> (&p)[12], const Cx<R> *link, Cx<R> (&acc)[12]) {
  Cx<R> h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> a0, a1;
    a_times<R, MU>(p[6 + c], p[9 + c], a0, a1);
    h[0][c] = FWD ? p[c] - a0 : p[c] + a0;
    h[1][c] = FWD ? p[3 + c] - a1 : p[3 + c] + a1;
  }
  Cx<R> t[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    t[0][a] = mk((R)0, (R)0);
    t[1][a] = mk((R)0, (R)0);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (FWD) {
        const Cx<R> u = link[a * 3 + b];  // U_ab
        cmac(t[0][a], u, h[0][b]);
        cmac(t[1][a], u, h[1][b]);
      } else {
        const Cx<R> u = link[b * 3 + a];  // (U^dagger)_ab = conj(U_ba)
        cmac_conj(t[0][a], u, h[0][b]);
        cmac_conj(t[1][a], u, h[1][b]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> l0, l1;
    adag_times<R, MU>(t[0][c], t[1][c], l0, l1);
    acc[c] = acc[c] + t[0][c];
    acc[3 + c] = acc[3 + c] + t[1][c];
    if (FWD) {
      acc[6 + c] = acc[6 + c] - l0;
      acc[9 + c] = acc[9 + c] - l1;
    } else {
      acc[6 + c] = acc[6 + c] + l0;
      acc[9 + c] = acc[9 + c] + l1;
    }
  }
}

// apply hop number `hop` (mu = hop / 2, forward for even hop) to the staged spinor
template <typename R>
__device__ __forceinline__ void hop_dispatch(int hop, const Cx<R> (&p)[12], const Cx<R> *link, Cx<R> (&acc)[12]) {
  switch (hop) {
    case 0: hop4<R, 0, true>(p, link, acc); break;
    case 1: hop4<R, 0, false>(p, link, acc); break;
    case 2: hop4<R, 1, true>(p, link, acc); break;
    case 3: hop4<R, 1, false>(p, link, acc); break;
    case 4: hop4<R, 2, true>(p, link, acc); break;
    case 5: hop4<R, 2, false>(p, link, acc); break;
    case 6: hop4<R, 3, true>(p, link, acc); break;
    default: hop4<R, 3, false>(p, link, acc); break;
  }
}

}  // namespace mg
