// Coarsest-level solve on one thread-block cluster (paper: the coarsest level of the V-cycle
// is an exact solve; here to the relative residual coarsest_tol inside the FP64 outer defect
// correction). Used in mixed-precision cycles when the coarsest tolerance is loose (>= 1e-5)
// and the coarsest level is small (N = 8, at most 8192 dofs): GCR on A M y = b (right block
// Jacobi folded into the stencil, x = M y) in FP32, with every reduction's cross-warp and
// cross-CTA sums in FP64.
//
// Design for GB300: the whole-chip cooperative solver pays two grid-wide barriers per
// iteration over ~150 CTAs and keeps every SM busy for the whole solve. Here one cluster of
// 16 CTAs (one per SM, 1024 threads each) owns the system: barriers are the hardware cluster
// barrier (barrier.cluster arrive.release / wait.acquire), the per-CTA partial sums are read
// across the cluster from distributed shared memory, and the Krylov basis Z, W of each CTA's
// rows stays in its shared memory for the whole solve. Only r (and y at restarts) goes to
// global memory for the neighbours' stencil reads (through L2). The other ~136 SMs stay free
// for the concurrent work of other solves.
//
// Each CTA owns dpc = n / 16 consecutive dofs (whole coarse sites). All decisions (restart,
// convergence, second Gram-Schmidt pass) come from sums that are identical in every CTA, so
// every CTA takes the same path through every barrier.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace mg {

namespace {

constexpr int kClCtas = 16;
constexpr int kClThreads = 1024;
constexpr int kClMaxDofs = 512;  // dofs per CTA
constexpr int kClMaxRestart = 16;
constexpr int kClSlots = 2 * kClMaxRestart + 4;

struct ClArgs {
  const Cx<float> *Yt;       // A M in FP32, internal layout [j][dir][col][row], N = 8
  const Cx<double> *Minv;    // [j][col][row]
  int L0, L1;
  long long nsites;
  int dpc;                   // dofs per CTA
  const Cx<double> *b;
  Cx<double> *x;
  Cx<float> *rpub, *ypub;    // published r and y (n entries each)
  double tol;
  int restart, max_iter;
  int *out;
  double *out_rel;
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums nv per-thread values val(s) over the cluster: FP32 warp trees, then FP64 over the warps of
// the CTA (in warp order) and over the CTAs (in rank order, read from distributed shared
// memory). part: this CTA's double-buffered slots [2][kClSlots]; wsum: [32][kClSlots].
template <typename F>
__device__ __forceinline__ void cluster_sum(cg::cluster_group &cl, F &&val, int nv, float *wsum, double *part,
                                            int &parity, double *res) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nv; ++s) {
    const float t = warp_sumf(val(s));
    if (lane == 0) wsum[wid * kClSlots + s] = t;
  }
  __syncthreads();
  double *mine = part + parity * kClSlots;
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int w = 0; w < kClThreads / 32; ++w) t += (double)wsum[w * kClSlots + threadIdx.x];
    mine[threadIdx.x] = t;
  }
  cluster_barrier();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int q = 0; q < kClCtas; ++q) t += cl.map_shared_rank(mine, q)[threadIdx.x];
    res[threadIdx.x] = t;
  }
  parity ^= 1;
  __syncthreads();
}

// A M v on the CTA's rows: two threads per row, 20 of the 40 (dir, col) terms each
__device__ __forceinline__ void stencil(const ClArgs &a, const Cx<float> *v, long long dof0, Cx<float> *outs) {
  const int h = threadIdx.x & 1;
  for (int lr = threadIdx.x >> 1; lr < kClMaxDofs; lr += kClThreads / 2) {
    Cx<float> acc = mk(0.f, 0.f);
    const bool act = lr < a.dpc;
    if (act) {
      const long long d = dof0 + lr, j = d >> 3;
      const int row = (int)(d & 7);
      const int x1 = (int)(j / a.L0), x0 = (int)(j - (long long)x1 * a.L0);
      const long long rowo = (long long)x1 * a.L0;
      long long src[5];
      src[0] = j;
      src[1] = rowo + (x0 + 1 == a.L0 ? 0 : x0 + 1);
      src[2] = rowo + (x0 == 0 ? a.L0 - 1 : x0 - 1);
      src[3] = (x1 + 1 == a.L1 ? 0 : rowo + a.L0) + x0;
      src[4] = (x1 == 0 ? (long long)(a.L1 - 1) * a.L0 : rowo - a.L0) + x0;
#pragma unroll
      for (int u = 0; u < 20; ++u) {
        const int term = h * 20 + u, dir = term >> 3, col = term & 7;
        const float2 vv = __ldcg(reinterpret_cast<const float2 *>(v + src[dir] * 8 + col));
        const Cx<float> y = a.Yt[(j * 5 + dir) * 64 + col * 8 + row];
        cmac(acc, y, mk(vv.x, vv.y));
      }
    }
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, 1);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, 1);
    if (act && h == 0) outs[lr] = acc;
  }
}

__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(kClThreads, 1)
    coarsest_gcr_cluster_kernel(ClArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smc[];
  double *part = smc;                                   // [2][kClSlots]
  double *res = part + 2 * kClSlots;                    // [kClSlots]
  float *wsum = reinterpret_cast<float *>(res + kClSlots);  // [32][kClSlots]
  Cx<float> *Zs = reinterpret_cast<Cx<float> *>(wsum + 32 * kClSlots);  // [restart][kClMaxDofs]
  Cx<float> *Ws = Zs + kClMaxRestart * kClMaxDofs;
  Cx<float> *rs = Ws + kClMaxRestart * kClMaxDofs;
  Cx<float> *ys = rs + kClMaxDofs;
  Cx<float> *bs = ys + kClMaxDofs;
  const int tid = threadIdx.x;
  const int rank = (int)cl.block_rank();
  // cluster v solves vector v of the batch: its b, x and publication buffers are offset by v n
  const long long n = a.nsites * 8, voff = (long long)(blockIdx.x / kClCtas) * n;
  a.b += voff;
  a.x += voff;
  a.rpub += voff;
  a.ypub += voff;
  const long long dof0 = (long long)rank * a.dpc;
  const bool own = tid < a.dpc;  // thread tid owns local dof tid for the vector work
  int parity = 0;

  if (own) {
    const Cx<double> bd = a.b[dof0 + tid];
    const Cx<float> bf = mk((float)bd.re, (float)bd.im);
    bs[tid] = bf;
    rs[tid] = bf;
    ys[tid] = mk(0.f, 0.f);
    a.rpub[dof0 + tid] = bf;
  }
  __syncthreads();
  cluster_sum(cl, [&](int) { return own ? norm2(bs[tid]) : 0.f; }, 1, wsum, part, parity, res);  // also publishes r
  const double bn2 = res[0];
  const double tol2 = a.tol * a.tol * bn2;
  int it = 0;
  bool converged = !(bn2 > 0.0);
  double rn2 = bn2;
  while (!converged && it < a.max_iter) {
    int k = 0;
    bool breakdown = false;
    for (; k < a.restart && it < a.max_iter; ++k) {
      Cx<float> *Wk = Ws + k * kClMaxDofs, *Zk = Zs + k * kClMaxDofs;
      stencil(a, a.rpub, dof0, Wk);  // w_k = (A M) r with the published r
      if (own) Zk[tid] = rs[tid];
      __syncthreads();
      // |w|^2, <w, r>, <W_j, w>
      const int nv = 3 + 2 * k;
      const Cx<float> w0 = own ? Wk[tid] : mk(0.f, 0.f), r0 = own ? rs[tid] : mk(0.f, 0.f);
      auto dots = [&](int sl) -> float {
        if (!own) return 0.f;
        if (sl == 0) return norm2(w0);
        if (sl == 1) return w0.re * r0.re + w0.im * r0.im;
        if (sl == 2) return w0.re * r0.im - w0.im * r0.re;
        const Cx<float> u = Ws[((sl - 3) >> 1) * kClMaxDofs + tid];
        return (sl & 1) ? u.re * w0.re + u.im * w0.im : u.re * w0.im - u.im * w0.re;
      };
      cluster_sum(cl, dots, nv, wsum, part, parity, res);
      double nw0 = res[0], nw2 = nw0;
      for (int j = 0; j < k; ++j) nw2 -= res[3 + 2 * j] * res[3 + 2 * j] + res[4 + 2 * j] * res[4 + 2 * j];
      const double wr = res[1], wi = res[2];
      for (int pass = 0; pass < 2; ++pass) {
        if (own) {
          Cx<float> w = Wk[tid], z = Zk[tid];
          for (int j = 0; j < k; ++j) {
            const Cx<float> bj = mk((float)-res[3 + 2 * j], (float)-res[4 + 2 * j]);
            cmac(w, bj, Ws[j * kClMaxDofs + tid]);
            cmac(z, bj, Zs[j * kClMaxDofs + tid]);
          }
          Wk[tid] = w;
          Zk[tid] = z;
        }
        __syncthreads();
        if (pass == 1 || k == 0 || nw2 > 0.5 * nw0) break;
        // cancellation: fresh coefficients for a second projection (same branch in every CTA)
        const Cx<float> w1 = own ? Wk[tid] : mk(0.f, 0.f);
        auto dots2 = [&](int sl) -> float {
          if (!own || sl == 1 || sl == 2) return 0.f;
          if (sl == 0) return norm2(w1);
          const Cx<float> u = Ws[((sl - 3) >> 1) * kClMaxDofs + tid];
          return (sl & 1) ? u.re * w1.re + u.im * w1.im : u.re * w1.im - u.im * w1.re;
        };
        cluster_sum(cl, dots2, nv, wsum, part, parity, res);
        nw2 = res[0];
        for (int j = 0; j < k; ++j) nw2 -= res[3 + 2 * j] * res[3 + 2 * j] + res[4 + 2 * j] * res[4 + 2 * j];
      }
      breakdown = !(nw2 > 1e-12 * nw0);
      const double inv = breakdown ? 0.0 : 1.0 / sqrt(nw2);
      // <w', r> = <w, r>: r is orthogonal to every earlier W_j
      const float ar = (float)(wr * inv), ai = (float)(wi * inv), fi = (float)inv;
      if (own) {
        const Cx<float> w = fi * Wk[tid], z = fi * Zk[tid];
        Wk[tid] = w;
        Zk[tid] = z;
        cmac(ys[tid], mk(ar, ai), z);
        Cx<float> rd = rs[tid];
        cmac(rd, mk(-ar, -ai), w);
        rs[tid] = rd;
        a.rpub[dof0 + tid] = rd;
      }
      rn2 = fmax(rn2 - ((double)ar * ar + (double)ai * ai), 0.0);
      ++it;
      cluster_barrier();  // the new r is visible to every CTA's stencil
      if (rn2 <= tol2 || breakdown) {
        ++k;
        break;
      }
    }
    // true residual r = b - (A M) y with the published y
    if (own) a.ypub[dof0 + tid] = ys[tid];
    cluster_barrier();
    stencil(a, a.ypub, dof0, rs);
    __syncthreads();
    if (own) {
      const Cx<float> rd = bs[tid] - rs[tid];
      rs[tid] = rd;
      a.rpub[dof0 + tid] = rd;
    }
    cluster_sum(cl, [&](int) { return own ? norm2(rs[tid]) : 0.f; }, 1, wsum, part, parity, res);
    rn2 = res[0];
    converged = rn2 <= tol2;
    if (!(rn2 == rn2) || (breakdown && k <= 1)) break;
  }
  // x = M y on the CTA's sites (site-local)
  __syncthreads();
  if (own) {
    const long long d = dof0 + tid, j = d >> 3;
    const int row = (int)(d & 7), sl = tid >> 3;
    Cx<double> acc = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) cmac(acc, a.Minv[j * 64 + c * 8 + row], cvt<double, float>(ys[sl * 8 + c]));
    a.x[d] = acc;
  }
  if (rank == 0 && tid == 0) {
    if (voff == 0) atomicAdd(a.out, it);
    if (!converged) atomicAdd(a.out + 2, 1);
    a.out_rel[0] = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
  }
  cluster_barrier();  // no CTA leaves while others may still read its shared memory
}

size_t cluster_smem_bytes() {
  return (size_t)3 * kClSlots * sizeof(double) + (size_t)32 * kClSlots * sizeof(float) +
         (size_t)(2 * kClMaxRestart + 3) * kClMaxDofs * sizeof(Cx<float>);
}

}  // namespace

bool coarsest_cluster_fits(Geo2 g, int N, int restart) {
  if (N != 8 || restart > kClMaxRestart || g.nsites % kClCtas != 0) return false;
  const long long dpc = g.nsites * 8 / kClCtas;
  if (dpc > kClMaxDofs || dpc > kClThreads) return false;
  const void *fn = (const void *)coarsest_gcr_cluster_kernel;
  const size_t smem = cluster_smem_bytes();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClCtas);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

void launch_coarsest_gcr_cluster(const Cx<float> *Yt32, const Cx<double> *Minv, Geo2 g, int nvec,
                                 const Cx<double> *b, Cx<double> *x, Cx<float> *rpub, Cx<float> *ypub, double tol,
                                 int restart, int max_iter, int *out, double *out_rel, cudaStream_t s) {
  ClArgs a;
  a.Yt = Yt32;
  a.Minv = Minv;
  a.L0 = g.L0;
  a.L1 = g.L1;
  a.nsites = g.nsites;
  a.dpc = (int)(g.nsites * 8 / kClCtas);
  a.b = b;
  a.x = x;
  a.rpub = rpub;
  a.ypub = ypub;
  a.tol = tol;
  a.restart = restart;
  a.max_iter = max_iter;
  a.out = out;
  a.out_rel = out_rel;
  if (restart > kClMaxRestart || a.dpc > kClMaxDofs || g.nsites % kClCtas != 0)
    fail(MG_ERR_UNSUPPORTED, "cluster coarsest solve: level too large or restart above 16");
  const size_t smem = cluster_smem_bytes();
  const void *fn = (const void *)coarsest_gcr_cluster_kernel;
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  coarsest_gcr_cluster_kernel<<<kClCtas * nvec, kClThreads, smem, s>>>(a);
  MG_LAUNCHED();
}

}  // namespace mg
