/*
 * GPU twin of the quenched U(1) Metropolis generator in gen.c (input generation only;
 * none of the multigrid method's arithmetic lives here).
 *
 * It runs the same Markov chain as metropolis_u1_2d in gen.c, step for step: the same
 * four checkerboard sub-sweeps (mu = 0 on rows of x1 parity 0 and 1, then mu = 1 on
 * columns of x0 parity 0 and 1; links of one sub-sweep share no plaquette), the same
 * Philox4x32-10 counter (x, sweep, mu + 2 hit, 0x4D45) under key = seed, the same
 * proposal theta' = theta + step (2 u_b - 1) and the same acceptance test
 * dS >= 0 or u_a <= exp(dS). Every rounding step that decides the chain is written with
 * explicit round-to-nearest intrinsics (no fused multiply-add), matching gen.c's
 * -ffp-contract=off build. The chains can therefore differ only where the two hosts'
 * cos / sin / exp round differently AND that difference flips an accept decision
 * (about 1e-16 per hit); callers compare the digest of the angles with the CPU
 * generator's stored digest.
 *
 * Several fields of equal size run in one launch per sub-sweep (blockIdx.y = field).
 * Layout: theta[f][x][mu], x = x0 + L0 x1.
 *
 * Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -shared -Xcompiler -fPIC.
 */
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__global__ void metropolis_sub_kernel(int L0, int L1, int mu, int parity, int sweep, int hits, double step,
                                      const double *__restrict__ beta, const uint64_t *__restrict__ seed,
                                      double *__restrict__ theta, unsigned long long *__restrict__ accepted) {
  const int f = blockIdx.y;
  const long long V = (long long)L0 * L1;
  double *th = theta + (size_t)f * 2 * V;
  const int n_other = (mu == 0) ? L1 / 2 : L0 / 2;
  const int n_along = (mu == 0) ? L0 : L1;
  const long long nwork = (long long)n_other * n_along;
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int acc = 0;
  if (w < nwork) {
    const int along = (int)(w % n_along), other = 2 * (int)(w / n_along) + parity;
    const int x0 = (mu == 0) ? along : other, x1 = (mu == 0) ? other : along;
    const int x0p = (x0 + 1) % L0, x0m = (x0 + L0 - 1) % L0;
    const int x1p = (x1 + 1) % L1, x1m = (x1 + L1 - 1) % L1;
    const long long x = x0 + (long long)L0 * x1;
    double a, b;
    if (mu == 0) {
      a = __dsub_rn(__dsub_rn(th[2 * (x0p + (long long)L0 * x1) + 1], th[2 * (x0 + (long long)L0 * x1p) + 0]),
                    th[2 * x + 1]);
      const long long y = x0 + (long long)L0 * x1m;
      b = __dsub_rn(__dadd_rn(th[2 * y + 0], th[2 * (x0p + (long long)L0 * x1m) + 1]), th[2 * y + 1]);
    } else {
      const long long y = x0m + (long long)L0 * x1;
      a = __dsub_rn(__dsub_rn(th[2 * y + 0], th[2 * (x0m + (long long)L0 * x1p) + 0]), th[2 * y + 1]);
      b = __dsub_rn(__dadd_rn(th[2 * x + 0], th[2 * (x0p + (long long)L0 * x1) + 1]),
                    th[2 * (x0 + (long long)L0 * x1p) + 0]);
    }
    const double Sr = __dadd_rn(cos(a), cos(b)), Si = __dsub_rn(sin(a), sin(b));
    double t = th[2 * x + mu];
    double local = __dsub_rn(__dmul_rn(cos(t), Sr), __dmul_rn(sin(t), Si));
    const double bt = beta[f];
    const uint64_t sd = seed[f];
    const uint32_t k0 = (uint32_t)sd, k1 = (uint32_t)(sd >> 32);
    const double two53 = 1.0 / 9007199254740992.0;
    for (int h = 0; h < hits; ++h) {
      uint32_t c[4] = {(uint32_t)x, (uint32_t)sweep, (uint32_t)(mu + 2 * h), 0x4D45u};
      philox(c, k0, k1);
      const uint64_t ia = ((((uint64_t)c[1] << 32) | c[0]) >> 11) + 1;
      const uint64_t ib = (((uint64_t)c[3] << 32) | c[2]) >> 11;
      const double ua = __dmul_rn((double)ia, two53), ub = __dmul_rn((double)ib, two53);
      const double tn = __dadd_rn(t, __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, ub), 1.0)));
      double sn, cn;
      sincos(tn, &sn, &cn);
      const double local_n = __dsub_rn(__dmul_rn(cn, Sr), __dmul_rn(sn, Si));
      const double dS = __dmul_rn(bt, __dsub_rn(local_n, local));
      if (dS >= 0.0 || ua <= exp(dS)) {
        t = tn;
        local = local_n;
        ++acc;
      }
    }
    const double two_pi = 6.283185307179586476925286766559;
    t = remainder(t, two_pi);
    if (t <= -3.14159265358979323846) t = __dadd_rn(t, two_pi);
    th[2 * x + mu] = t;
  }
  // one atomic per warp
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0) atomicAdd(accepted + f, (unsigned long long)acc);
}

}  // namespace

extern "C" {

/*
 * nfields independent chains on L0 x L1 (even extents) from the angles already in theta
 * (device, nfields x L0 L1 x 2; zeros = a cold start), `sweeps` sweeps of `hits` hits
 * each with proposals uniform in [-step, step]; beta, seed: device arrays of nfields;
 * accepted: device array of nfields counters (added to). Asynchronous on `stream`.
 * Returns 0, or a cudaError_t code of the first failing launch.
 */
int gen_metropolis_u1_2d_gpu(int L0, int L1, int nfields, int sweeps, int hits, double step, const double *beta,
                             const uint64_t *seed, double *theta, unsigned long long *accepted, void *stream) {
  if (L0 < 2 || L1 < 2 || (L0 & 1) || (L1 & 1) || nfields < 1 || nfields > 65535) return (int)cudaErrorInvalidValue;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int threads = 128;
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int sub = 0; sub < 4; ++sub) {
      const int mu = sub >> 1, parity = sub & 1;
      const long long nwork = (long long)((mu == 0) ? L1 / 2 : L0 / 2) * ((mu == 0) ? L0 : L1);
      dim3 grid((unsigned)((nwork + threads - 1) / threads), (unsigned)nfields);
      metropolis_sub_kernel<<<grid, threads, 0, s>>>(L0, L1, mu, parity, sweep, hits, step, beta, seed, theta,
                                                     accepted);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return (int)e;
    }
  }
  return 0;
}

}  // extern "C"
