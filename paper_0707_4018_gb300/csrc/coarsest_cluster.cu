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
constexpr int kClThreads = 512;
constexpr int kClMaxDofs = 512;  // dofs per CTA
constexpr int kClMaxRestart = 16;
constexpr int kClSlots = 2 * kClMaxRestart + 4;

struct ClArgs {
  const Cx<float> *Yt;       // A M in FP32, row-major blocks [j][dir][row][col], N = 8
  const Cx<double> *Minv;    // [j][col][row]
  int L0, L1;
  long long nsites;
  int dpc;                   // dofs per CTA
  int spc;                   // sites per CTA
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

// Sums nv per-thread values val(s) over the cluster: FP32 warp trees, a second FP32 warp tree
// over the CTA's 16 warps (warp w reduces slots w, w + 16, ...), then FP64 over the 16 CTAs in rank order, read
// from distributed shared memory. part: this CTA's double-buffered slots [2][kClSlots] (float);
// wsum: [32][kClSlots]. Every CTA ends with the same sums in res.
template <typename F>
__device__ __forceinline__ void cluster_sum(cg::cluster_group &cl, F &&val, int nv, float *wsum, float *part,
                                            int &parity, double *res) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nv; ++s) {
    const float t = warp_sumf(val(s));
    if (lane == 0) wsum[wid * kClSlots + s] = t;
  }
  __syncthreads();
  float *mine = part + parity * kClSlots;
  for (int sl = wid; sl < nv; sl += kClThreads / 32) {
    const float t = warp_sumf(lane < kClThreads / 32 ? wsum[lane * kClSlots + sl] : 0.f);
    if (lane == 0) mine[sl] = t;
  }
  cluster_barrier();
  if (threadIdx.x < nv) {
    float v[kClCtas];
#pragma unroll
    for (int q = 0; q < kClCtas; ++q) v[q] = cl.map_shared_rank(mine, q)[threadIdx.x];
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kClCtas; ++q) t += (double)v[q];
    res[threadIdx.x] = t;
  }
  parity ^= 1;
  __syncthreads();
}

// A M v on the CTA's rows. The CTA's sites and their neighbours form the contiguous (periodic)
// range [site0 - L0, site0 + spc + L0): its values of v are staged in shared memory with one
// coalesced pass, then one thread per row reads that row's 5 x 8 coefficients as float4 pairs
// (layout [j][dir][row][col]) and the neighbour values from shared memory.
constexpr int kClMaxStage = 256;  // staged sites
__device__ __forceinline__ void stencil(const ClArgs &a, const Cx<float> *v, long long dof0, Cx<float> *vs,
                                        Cx<float> *outs) {
  const long long site0 = dof0 >> 3, nst = a.spc + 2LL * a.L0;
  const long long base = site0 - a.L0 + a.nsites;  // + nsites keeps the modulo non-negative
  __syncthreads();  // earlier readers of vs are done
  for (int q = threadIdx.x; q < nst * 4; q += kClThreads) {
    const long long st = q >> 2;
    const long long g = (base + st) % a.nsites;
    reinterpret_cast<float4 *>(vs)[q] = __ldcg(reinterpret_cast<const float4 *>(v + g * 8) + (q & 3));
  }
  __syncthreads();
  const int lr = threadIdx.x;
  if (lr < a.dpc) {
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
    Cx<float> acc = mk(0.f, 0.f);
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const int sidx = (int)((src[dir] - base + 2 * a.nsites) % a.nsites);
      const float4 *yp = reinterpret_cast<const float4 *>(a.Yt + ((j * 5 + dir) * 8 + row) * 8);
      const Cx<float> *vv = vs + sidx * 8;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 y = __ldcg(yp + q);
        cmac(acc, mk(y.x, y.y), vv[2 * q]);
        cmac(acc, mk(y.z, y.w), vv[2 * q + 1]);
      }
    }
    outs[lr] = acc;
  }
}

__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(kClThreads, 1)
    coarsest_gcr_cluster_kernel(ClArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smc[];
  double *res = smc;                                    // [kClSlots]
  float *part = reinterpret_cast<float *>(res + kClSlots);  // [2][kClSlots]
  float *wsum = part + 2 * kClSlots;                    // [32][kClSlots]
  Cx<float> *Zs = reinterpret_cast<Cx<float> *>(wsum + 32 * kClSlots);  // [restart][kClMaxDofs]
  Cx<float> *Ws = Zs + kClMaxRestart * kClMaxDofs;
  Cx<float> *rs = Ws + kClMaxRestart * kClMaxDofs;
  Cx<float> *ys = rs + kClMaxDofs;
  Cx<float> *bs = ys + kClMaxDofs;
  Cx<float> *vst = bs + kClMaxDofs;  // staged stencil input [kClMaxStage][8]
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
  // the scalar work of every iteration (coefficients, norms, decisions) is done once, by thread
  // 0, and shared as floats / flags: GB300's FP64 rate is far too low for 1024 threads to repeat it
  __shared__ float s_beta[2 * kClMaxRestart];
  __shared__ float s_coef[3];    // 1 / |w'|, Re alpha, Im alpha
  __shared__ int s_flag[3];      // second projection, leave the inner loop, breakdown
  __shared__ double s_sc[3];     // |w|^2, |w'|^2, running |r|^2 estimate
  __shared__ int s_conv;
  if (tid == 0) {
    s_sc[2] = bn2;
    s_conv = converged ? 1 : 0;
  }
  __syncthreads();
  auto betas = [&](int k) {  // thread 0: Gram-Schmidt coefficients and |w'|^2 from res
    double nw2 = res[0];
    for (int j = 0; j < k; ++j) {
      nw2 -= res[3 + 2 * j] * res[3 + 2 * j] + res[4 + 2 * j] * res[4 + 2 * j];
      s_beta[2 * j] = (float)-res[3 + 2 * j];
      s_beta[2 * j + 1] = (float)-res[4 + 2 * j];
    }
    s_sc[1] = nw2;
  };
  auto project = [&](int k, Cx<float> *Wk, Cx<float> *Zk) {
    if (own) {
      Cx<float> w = Wk[tid], z = Zk[tid];
      for (int j = 0; j < k; ++j) {
        const Cx<float> bj = mk(s_beta[2 * j], s_beta[2 * j + 1]);
        cmac(w, bj, Ws[j * kClMaxDofs + tid]);
        cmac(z, bj, Zs[j * kClMaxDofs + tid]);
      }
      Wk[tid] = w;
      Zk[tid] = z;
    }
    __syncthreads();
  };
  while (!s_conv && it < a.max_iter) {
    int k = 0;
    bool breakdown = false;
    for (; k < a.restart && it < a.max_iter; ++k) {
      Cx<float> *Wk = Ws + k * kClMaxDofs, *Zk = Zs + k * kClMaxDofs;
      stencil(a, a.rpub, dof0, vst, Wk);  // w_k = (A M) r with the published r
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
      double wr = 0.0, wi = 0.0;
      if (tid == 0) {
        wr = res[1];
        wi = res[2];
        s_sc[0] = res[0];
        betas(k);
        s_flag[0] = (k > 0 && !(s_sc[1] > 0.5 * s_sc[0])) ? 1 : 0;
      }
      __syncthreads();
      project(k, Wk, Zk);
      if (s_flag[0]) {
        // cancellation: fresh coefficients for a second projection (same branch in every CTA)
        const Cx<float> w1 = own ? Wk[tid] : mk(0.f, 0.f);
        auto dots2 = [&](int sl) -> float {
          if (!own || sl == 1 || sl == 2) return 0.f;
          if (sl == 0) return norm2(w1);
          const Cx<float> u = Ws[((sl - 3) >> 1) * kClMaxDofs + tid];
          return (sl & 1) ? u.re * w1.re + u.im * w1.im : u.re * w1.im - u.im * w1.re;
        };
        cluster_sum(cl, dots2, nv, wsum, part, parity, res);
        if (tid == 0) betas(k);
        __syncthreads();
        project(k, Wk, Zk);
      }
      if (tid == 0) {
        const float nw0 = (float)s_sc[0], nw2 = (float)s_sc[1];
        const bool bd = !(nw2 > 1e-12f * nw0);
        const float inv = bd ? 0.f : rsqrtf(nw2);
        // <w', r> = <w, r>: r is orthogonal to every earlier W_j
        const float ar = (float)wr * inv, ai = (float)wi * inv;
        s_coef[0] = inv;
        s_coef[1] = ar;
        s_coef[2] = ai;
        s_sc[2] = fmax(s_sc[2] - ((double)ar * ar + (double)ai * ai), 0.0);
        s_flag[1] = (s_sc[2] <= tol2 || bd) ? 1 : 0;
        s_flag[2] = bd ? 1 : 0;
      }
      __syncthreads();
      const float fi = s_coef[0], ar = s_coef[1], ai = s_coef[2];
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
      ++it;
      breakdown = s_flag[2] != 0;
      const bool leave = s_flag[1] != 0;
      cluster_barrier();  // the new r is visible to every CTA's stencil
      if (leave) {
        ++k;
        break;
      }
    }
    // true residual r = b - (A M) y with the published y
    if (own) a.ypub[dof0 + tid] = ys[tid];
    cluster_barrier();
    stencil(a, a.ypub, dof0, vst, rs);
    __syncthreads();
    if (own) {
      const Cx<float> rd = bs[tid] - rs[tid];
      rs[tid] = rd;
      a.rpub[dof0 + tid] = rd;
    }
    cluster_sum(cl, [&](int) { return own ? norm2(rs[tid]) : 0.f; }, 1, wsum, part, parity, res);
    if (tid == 0) {
      s_sc[2] = res[0];
      s_conv = s_sc[2] <= tol2 ? 1 : 0;
      if (!(s_sc[2] == s_sc[2]) || (breakdown && k <= 1)) s_conv = 2;  // stop: NaN or no progress
    }
    __syncthreads();
    if (s_conv == 2) break;
  }
  converged = s_conv == 1;
  rn2 = s_sc[2];
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
  return (size_t)kClSlots * sizeof(double) + (size_t)34 * kClSlots * sizeof(float) +
         (size_t)(2 * kClMaxRestart + 3) * kClMaxDofs * sizeof(Cx<float>) +
         (size_t)kClMaxStage * 8 * sizeof(Cx<float>);
}

// [j][dir][col][row] -> [j][dir][row][col] for 8 x 8 complex blocks
__global__ void transpose8_kernel(const Cx<float> *__restrict__ in, Cx<float> *__restrict__ out, long long nblk) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nblk * 64) return;
  const long long blk = i >> 6;
  const int rc = (int)(i & 63), col = rc >> 3, row = rc & 7;
  out[blk * 64 + row * 8 + col] = in[i];
}

}  // namespace

void launch_transpose_blocks8(const Cx<float> *in, Cx<float> *out, long long nblocks, cudaStream_t s) {
  const long long n = nblocks * 64;
  transpose8_kernel<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(in, out, nblocks);
  MG_LAUNCHED();
}

bool coarsest_cluster_fits(Geo2 g, int N, int restart) {
  if (N != 8 || restart > kClMaxRestart || g.nsites % kClCtas != 0) return false;
  const long long dpc = g.nsites * 8 / kClCtas;
  if (dpc > kClMaxDofs || dpc > kClThreads) return false;
  if (g.nsites / kClCtas + 2LL * g.L0 > kClMaxStage || 2LL * g.L0 > g.nsites) return false;
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
  a.spc = (int)(g.nsites / kClCtas);
  a.b = b;
  a.x = x;
  a.rpub = rpub;
  a.ypub = ypub;
  a.tol = tol;
  a.restart = restart;
  a.max_iter = max_iter;
  a.out = out;
  a.out_rel = out_rel;
  if (restart > kClMaxRestart || a.dpc > kClMaxDofs || g.nsites % kClCtas != 0 ||
      a.spc + 2LL * g.L0 > kClMaxStage || 2LL * g.L0 > g.nsites)
    fail(MG_ERR_UNSUPPORTED, "cluster coarsest solve: level too large or restart above 16");
  const size_t smem = cluster_smem_bytes();
  const void *fn = (const void *)coarsest_gcr_cluster_kernel;
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  coarsest_gcr_cluster_kernel<<<kClCtas * nvec, kClThreads, smem, s>>>(a);
  MG_LAUNCHED();
}

}  // namespace mg
