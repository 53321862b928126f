// The four hopping terms of the 2d Wilson operator with gamma_1 = sigma_1,
// gamma_2 = sigma_2 (paper, definition of D following Eq. 1). In 2d every
// projector (1 -+ gamma_mu) has rank one, so a hop is one complex multiply:
//   (1 - s1) psi = (psi0 - psi1)   (1, -1)      (1 + s1) psi = (psi0 + psi1)   (1, 1)
//   (1 - s2) psi = (psi0 + i psi1) (1, -i)      (1 + s2) psi = (psi0 - i psi1) (1, i)
// The forward hop from x + mu multiplies by U_x^mu, the backward hop from
// x - mu by conj(U_{x-mu}^mu); the -1/2 is applied by the caller.
#pragma once

#include "common.cuh"

namespace mg {

template <typename R>
struct alignas(4 * sizeof(R)) Pair {
  Cx<R> a, b;
};

// dir 1: +0, 2: -0, 3: +1, 4: -1. Returns the projected, transported scalar t;
// the spin components of the hop are (t, t * spin1_factor(dir)).
template <typename R>
__device__ __forceinline__ Cx<R> hop_scalar(int dir, Cx<R> u, Cx<R> p0, Cx<R> p1) {
  switch (dir) {
    case 1: return u * (p0 - p1);                     // U (psi0 - psi1)
    case 2: return cmul_conj(u, p0 + p1);             // U^* (psi0 + psi1)
    case 3: return u * (p0 + times_i(p1));            // U (psi0 + i psi1)
    default: return cmul_conj(u, p0 - times_i(p1));   // U^* (psi0 - i psi1)
  }
}

// second spin component of the hop: dir 1: -t, 2: t, 3: -i t, 4: i t
template <typename R>
__device__ __forceinline__ Cx<R> hop_lower(int dir, Cx<R> t) {
  switch (dir) {
    case 1: return mk(-t.re, -t.im);
    case 2: return t;
    case 3: return mk(t.im, -t.re);
    default: return mk(-t.im, t.re);
  }
}

}  // namespace mg
