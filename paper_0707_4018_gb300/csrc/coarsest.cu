// Coarsest-level solve as one persistent kernel (paper: the coarsest level of
// the V-cycle is an exact solve). The coarsest system of the three-level
// hierarchy is far too large for a dense factorisation at every setup pass, so
// it is iterated to a relative residual `tol` with restarted GCR, entirely on
// the device:
//
//  * right block-Jacobi preconditioning folded into the stencil: with
//    M = blockdiag(X_j^{-1}) (X_j the coarse self blocks), GCR runs on
//    A M y = b, whose blocks are Y_{j,dir} X_{src}^{-1} (same sparsity, self
//    blocks = I); its residual is the true residual b - A x with x = M y;
//  * one cooperative launch of G CTAs (all co-resident); each thread owns the
//    dofs i = gid, gid + G*T, ... for the whole solve;
//  * grid-wide barriers are a counter + generation flag with a bounded spin:
//    after `spin_limit` polls a CTA records timeout status and returns, so the
//    kernel always terminates;
//  * deterministic reductions: fixed warp/block trees, per-CTA partials staged
//    into shared memory by every CTA and summed in CTA order (identical in
//    every CTA);
//  * classical Gram-Schmidt applied twice; the second pass shares its grid
//    reduction with |w|^2 and <w, r> (|w - W b|^2 = |w|^2 - |b|^2 for the
//    orthonormal W), so an iteration costs 3 grid synchronisations.
// Arithmetic: FP64 throughout (the coarsest solve stays in FP64 in every mode).
#include <mutex>

#include "kernels.h"

namespace mg {

// Cooperative kernels wait on one another's CTAs at grid barriers, so all their CTAs must be
// resident at once. Two of them in flight on different streams (concurrent setups, solves
// from several host threads, parallel branches of one graph) can each hold part of the GPU
// and wait for the rest. Every cooperative launch outside a capture therefore passes through
// one lane per device: it waits on the lane's event (the previous cooperative launch, from
// any stream) and records the event after itself. A launch captured into a graph marks the
// capturing thread instead; the graph's launch then takes the lane as a whole.
namespace {
struct CoopLane {
  std::mutex mu;
  cudaEvent_t ev = nullptr;
};
constexpr int kMaxLaneDevices = 64;
CoopLane g_lanes[kMaxLaneDevices];
thread_local bool t_coop_captured = false;

template <typename F>
void through_lane(cudaStream_t s, F &&launch) {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxLaneDevices) fail(MG_ERR_UNSUPPORTED, "device ordinal beyond the cooperative lanes");
  CoopLane &L = g_lanes[dev];
  std::lock_guard<std::mutex> lk(L.mu);
  if (L.ev == nullptr) MG_CUDA(cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming));
  MG_CUDA(cudaStreamWaitEvent(s, L.ev, 0));
  launch();
  MG_CUDA(cudaEventRecord(L.ev, s));
}
}  // namespace

void coop_launch(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MG_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    t_coop_captured = true;
    MG_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s));
    return;
  }
  through_lane(s, [&] { MG_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s)); });
}

bool coop_captured_take() {
  const bool v = t_coop_captured;
  t_coop_captured = false;
  return v;
}

void coop_graph_launch(cudaGraphExec_t g, cudaStream_t s) {
  through_lane(s, [&] { MG_CUDA(cudaGraphLaunch(g, s)); });
}

constexpr int kMaxRestart = 32;
constexpr int kSlots = 2 * kMaxRestart + 4;
static_assert(kSlots == kCoarsestSlots, "slot count shared with the host");

// VT: precision of the stencil A M and of the Krylov vectors (double; float in mixed-precision
// cycles with a loose coarsest tolerance, where every reduction still sums in FP64)
template <typename VT>
struct CgArgs {
  const Cx<VT> *Y;         // preconditioned stencil A M, internal layout
  const Cx<double> *Minv;  // X_j^{-1}, [j][col][row]
  int L0, L1, N;
  long long n;
  const Cx<double> *b;
  Cx<double> *x;
  Cx<VT> *y, *r, *Z, *W;
  double *partials;   // [G][kSlots]
  unsigned int *bar;  // [0] count, [1] generation
  double tol;
  int restart, max_iter;
  long long spin_limit;
  int *out;         // [0] iterations (accumulated), [1] sticky status (1 = barrier timeout),
                    // [2] solves that missed the tolerance (accumulated)
  double *out_rel;  // relative true residual of the last solve
};

// bounded grid barrier; clears `ok` (and sets the status) when the wait gave up
template <typename A>
__device__ __forceinline__ void grid_sync(const A &a, bool &ok) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = a.bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(a.bar, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (++polls > a.spin_limit) {
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!good) atomicExch(a.out + 1, 1);
    s_ok = good;
  }
  __syncthreads();
  ok = ok && s_ok;
}

// warp tree of one per-thread value; lane 0 stores it as slot s of its warp
__device__ __forceinline__ void warp_put(double t, int s, double *swarp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) swarp[(threadIdx.x >> 5) * kSlots + s] = t;
}

// Sum slots [0, nv) of every warp across the grid. Block tree -> per-CTA
// partials -> barrier -> every CTA stages all partials in shared memory with
// independent loads -> one warp per slot sums them in CTA order.
template <typename A>
__device__ __forceinline__ void grid_sum(const A &a, int nv, double *swarp, double *stage, double *sres,
                                         bool &ok) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int s = threadIdx.x; s < nv; s += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += swarp[w * kSlots + s];
    a.partials[(long long)blockIdx.x * kSlots + s] = t;
  }
  __threadfence();
  grid_sync(a, ok);
  const int total = (int)gridDim.x * nv;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int c = q / nv, s = q - c * nv;
    stage[q] = __ldcg(a.partials + (long long)c * kSlots + s);
  }
  __syncthreads();
  for (int s = wid; s < nv; s += nw) {
    double t = 0.0;
    for (unsigned int c = lane; c < gridDim.x; c += 32) t += stage[c * nv + s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sres[s] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ Cx<double> ldcg2(const Cx<double> *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ Cx<float> ldcg2(const Cx<float> *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return mk(v.x, v.y);
}

template <int NT, typename VT>
__device__ __forceinline__ Cx<VT> apply_row(const CgArgs<VT> &a, long long i, const Cx<VT> *v) {
  const int N = NT > 0 ? NT : a.N;
  const long long j = i / N;
  const int row = (int)(i - j * N);
  const int x1 = (int)(j / a.L0), x0 = (int)(j - (long long)x1 * a.L0);
  const long long rowo = (long long)x1 * a.L0;
  long long src[5];
  src[0] = j;
  src[1] = rowo + (x0 + 1 == a.L0 ? 0 : x0 + 1);
  src[2] = rowo + (x0 == 0 ? a.L0 - 1 : x0 - 1);
  src[3] = (x1 + 1 == a.L1 ? 0 : rowo + a.L0) + x0;
  src[4] = (x1 == 0 ? (long long)(a.L1 - 1) * a.L0 : rowo - a.L0) + x0;
  Cx<VT> acc = mk<VT>(0, 0);
#pragma unroll
  for (int dir = 0; dir < 5; ++dir) {
    const Cx<VT> *Yd = a.Y + (j * 5 + dir) * (long long)N * N + row;
    const Cx<VT> *xs = v + src[dir] * N;
#pragma unroll(NT > 0 ? NT : 1)
    for (int c = 0; c < N; ++c) {
      // neighbour values were written by other CTAs: read through L2 (no stale L1 lines)
      cmac(acc, Yd[(long long)c * N], ldcg2(xs + c));
    }
  }
  return acc;
}

// sum over own dofs of conj(W_j) * Wk for j < k, into warp slots off + 2j, off + 2j + 1
template <typename VT>
__device__ __forceinline__ void gs_dots(const CgArgs<VT> &a, int k, const Cx<VT> *Wk, long long gid, long long gs,
                                        double *swarp, int off) {
  for (int j = 0; j < k; ++j) {
    double re = 0.0, im = 0.0;
    for (long long i = gid; i < a.n; i += gs) {
      const Cx<VT> wj = a.W[(long long)j * a.n + i], w = Wk[i];
      re += (double)(wj.re * w.re + wj.im * w.im);
      im += (double)(wj.re * w.im - wj.im * w.re);
    }
    warp_put(re, off + 2 * j, swarp);
    warp_put(im, off + 2 * j + 1, swarp);
  }
}

template <int NT, typename VT>
__global__ void __launch_bounds__(256) coarsest_gcr_kernel(CgArgs<VT> a) {
  extern __shared__ double sdyn[];
  double *swarp = sdyn;               // 8 warps x kSlots
  double *sres = sdyn + 8 * kSlots;   // kSlots
  double *stage = sdyn + 9 * kSlots;  // G x kSlots
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const long long n = a.n;
  const int N = NT > 0 ? NT : a.N;
  bool ok = true;

  // y = 0, r = b, |b|^2
  double t0 = 0.0;
  for (long long i = gid; i < n; i += gs) {
    const Cx<double> bi = a.b[i];
    a.y[i] = mk<VT>(0, 0);
    a.r[i] = cvt<VT, double>(bi);
    t0 += norm2(bi);
  }
  warp_put(t0, 0, swarp);
  grid_sum(a, 1, swarp, stage, sres, ok);
  if (!ok) return;
  const double bn2 = sres[0];
  const double tol2 = a.tol * a.tol * bn2;
  int it = 0;
  bool converged = !(bn2 > 0.0);
  double rn2 = bn2;
  while (!converged && it < a.max_iter) {
    for (int k = 0; k < a.restart && it < a.max_iter; ++k) {
      Cx<VT> *Zk = a.Z + (long long)k * n, *Wk = a.W + (long long)k * n;
      // z_k = r, w_k = (A M) r
      for (long long i = gid; i < n; i += gs) {
        Wk[i] = apply_row<NT, VT>(a, i, a.r);
        Zk[i] = a.r[i];
      }
      if (k > 0) {
        // first classical Gram-Schmidt pass
        gs_dots(a, k, Wk, gid, gs, swarp, 0);
        grid_sum(a, 2 * k, swarp, stage, sres, ok);
        if (!ok) return;
        for (long long i = gid; i < n; i += gs) {
          Cx<VT> w = Wk[i], z = Zk[i];
          for (int j = 0; j < k; ++j) {
            const Cx<VT> bj = mk((VT)-sres[2 * j], (VT)-sres[2 * j + 1]);
            cmac(w, bj, a.W[(long long)j * n + i]);
            cmac(z, bj, a.Z[(long long)j * n + i]);
          }
          Wk[i] = w;
          Zk[i] = z;
        }
        // second pass dots (slots 3 + 2j) share the reduction with the norms below
        gs_dots(a, k, Wk, gid, gs, swarp, 3);
      }
      double nn = 0.0, wr = 0.0, wi = 0.0;
      for (long long i = gid; i < n; i += gs) {
        const Cx<VT> w = Wk[i], ri = a.r[i];
        nn += (double)norm2(w);
        wr += (double)(w.re * ri.re + w.im * ri.im);
        wi += (double)(w.re * ri.im - w.im * ri.re);
      }
      warp_put(nn, 0, swarp);
      warp_put(wr, 1, swarp);
      warp_put(wi, 2, swarp);
      grid_sum(a, 3 + 2 * k, swarp, stage, sres, ok);
      if (!ok) return;
      // second pass: w -= W beta2; |w|^2 -= |beta2|^2; <w, r> unchanged to O(eps^2)
      double nw2 = sres[0];
      for (int j = 0; j < k; ++j) nw2 -= sres[3 + 2 * j] * sres[3 + 2 * j] + sres[4 + 2 * j] * sres[4 + 2 * j];
      const bool breakdown = !(nw2 > 1e-28 * sres[0]);
      const double inv = breakdown ? 0.0 : 1.0 / sqrt(nw2);
      const double ar = sres[1] * inv, ai = sres[2] * inv;  // <w_hat, r>
      const Cx<VT> alpha = mk((VT)ar, (VT)ai);
      const VT vinv = (VT)inv;
      for (long long i = gid; i < n; i += gs) {
        Cx<VT> w = Wk[i], z = Zk[i];
        for (int j = 0; j < k; ++j) {
          const Cx<VT> bj = mk((VT)-sres[3 + 2 * j], (VT)-sres[4 + 2 * j]);
          cmac(w, bj, a.W[(long long)j * n + i]);
          cmac(z, bj, a.Z[(long long)j * n + i]);
        }
        w = vinv * w;
        z = vinv * z;
        Wk[i] = w;
        Zk[i] = z;
        cmac(a.y[i], alpha, z);
        Cx<VT> ri = a.r[i];
        cmac(ri, mk(-alpha.re, -alpha.im), w);
        a.r[i] = ri;
      }
      rn2 = fmax(rn2 - (ar * ar + ai * ai), 0.0);
      ++it;
      grid_sync(a, ok);
      if (!ok) return;
      if (rn2 <= tol2 || breakdown) break;
    }
    // true residual r = b - (A M) y
    double tr = 0.0;
    for (long long i = gid; i < n; i += gs) {
      const Cx<VT> ri = cvt<VT, double>(a.b[i]) - apply_row<NT, VT>(a, i, a.y);
      a.r[i] = ri;
      tr += (double)norm2(ri);
    }
    warp_put(tr, 0, swarp);
    grid_sum(a, 1, swarp, stage, sres, ok);
    if (!ok) return;
    rn2 = sres[0];
    converged = rn2 <= tol2;
    if (!(rn2 == rn2)) break;  // NaN: stop; reported through out_rel
  }
  // x = M y (site-local; y is complete after the last grid reduction)
  for (long long i = gid; i < n; i += gs) {
    const long long j = i / N;
    const int row = (int)(i - j * N);
    const Cx<double> *Mj = a.Minv + j * (long long)N * N + row;
    Cx<double> acc = mk(0.0, 0.0);
    for (int c = 0; c < N; ++c) cmac(acc, Mj[(long long)c * N], cvt<double, VT>(ldcg2(a.y + j * N + c)));
    a.x[i] = acc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(a.out, it);
    if (!converged) atomicAdd(a.out + 2, 1);
    a.out_rel[0] = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// block-Jacobi preparation: Minv_j = X_j^{-1} (Gauss-Jordan with partial
// pivoting, one thread per coarse site) and the stencil A M
// ---------------------------------------------------------------------------
__global__ void self_block_inverse_kernel(const Cx<double> *__restrict__ Y, Cx<double> *__restrict__ Minv,
                                          Cx<double> *__restrict__ work, long long nsites, int N, int *info,
                                          double shift) {
  // one warp per coarse site; the augmented matrix [X | I] lives in `work` (2 N^2 entries per
  // site, column-major); lane r < N owns row r and lane N + r its copy of the identity part
  const long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= nsites) return;
  Cx<double> *Aw = work + j * 2LL * N * N;
  Cx<double> *Iw = Aw + (long long)N * N;
  const Cx<double> *X = Y + (j * 5) * (long long)N * N;  // [col][row]
  for (int q = lane; q < N * N; q += 32) {
    const bool dg = (q % N) == (q / N);
    Aw[q] = dg ? mk(X[q].re + shift, X[q].im) : X[q];
    Iw[q] = mk(dg ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  for (int c = 0; c < N; ++c) {
    // pivot: largest |A(r, c)|, r >= c, ties to the smallest r (same answer in every lane)
    int p = c;
    double best = norm2(Aw[c * N + c]);
    for (int rr = c + 1; rr < N; ++rr) {
      const double v = norm2(Aw[c * N + rr]);
      if (v > best) {
        best = v;
        p = rr;
      }
    }
    if (!(best > 0.0)) {
      if (lane == 0) atomicExch(info, 1);
      return;
    }
    __syncwarp();
    if (p != c) {
      for (int cc = lane; cc < 2 * N; cc += 32) {
        Cx<double> *M = cc < N ? Aw : Iw;
        const int col = cc < N ? cc : cc - N;
        const Cx<double> t = M[col * N + c];
        M[col * N + c] = M[col * N + p];
        M[col * N + p] = t;
      }
    }
    __syncwarp();
    const Cx<double> pv = Aw[c * N + c];
    const double d = norm2(pv);
    const Cx<double> inv = mk(pv.re / d, -pv.im / d);
    __syncwarp();
    for (int cc = lane; cc < 2 * N; cc += 32) {
      Cx<double> *M = cc < N ? Aw : Iw;
      const int col = cc < N ? cc : cc - N;
      M[col * N + c] = M[col * N + c] * inv;
    }
    __syncwarp();
    // eliminate column c from every other row: element (rr, col) of [A | I]. The
    // multipliers A(rr, c) are taken first (lane rr) and broadcast, because the
    // update overwrites column c itself.
    const Cx<double> fl = lane < N ? Aw[c * N + lane] : mk(0.0, 0.0);
    __syncwarp();
    for (int base = 0; base < 2 * N * N; base += 32) {
      const int q = base + lane;
      const int cc = q / N, rr = q - cc * N;
      const double fre = __shfl_sync(0xffffffffu, fl.re, rr & 31);
      const double fim = __shfl_sync(0xffffffffu, fl.im, rr & 31);
      if (q < 2 * N * N && rr != c) {
        Cx<double> *M = cc < N ? Aw : Iw;
        const int col = cc < N ? cc : cc - N;
        cmac(M[col * N + rr], mk(-fre, -fim), M[col * N + c]);
      }
    }
    __syncwarp();
  }
  Cx<double> *Mj = Minv + j * (long long)N * N;
  for (int q = lane; q < N * N; q += 32) Mj[q] = Iw[q];
}

// Yt[j][dir] = Y[j][dir] * Minv[src(j, dir)]  (column-major blocks); thread per (j, dir, col, row)
__global__ void precondition_stencil_kernel(const Cx<double> *__restrict__ Y, const Cx<double> *__restrict__ Minv,
                                            Cx<double> *__restrict__ Yt, int L0, int L1, int N, double shift) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nsites = (long long)L0 * L1;
  const long long per = 5LL * N * N;
  if (t >= nsites * per) return;
  const long long j = t / per;
  const int rem = (int)(t - j * per), dir = rem / (N * N), cr = rem - dir * N * N, col = cr / N, row = cr - col * N;
  const int x1 = (int)(j / L0), x0 = (int)(j - (long long)x1 * L0);
  const long long rowo = (long long)x1 * L0;
  long long src;
  switch (dir) {
    case 0: src = j; break;
    case 1: src = rowo + (x0 + 1 == L0 ? 0 : x0 + 1); break;
    case 2: src = rowo + (x0 == 0 ? L0 - 1 : x0 - 1); break;
    case 3: src = (x1 + 1 == L1 ? 0 : rowo + L0) + x0; break;
    default: src = (x1 == 0 ? (long long)(L1 - 1) * L0 : rowo - L0) + x0; break;
  }
  const Cx<double> *Yd = Y + (j * 5 + dir) * (long long)N * N;
  const Cx<double> *Ms = Minv + src * (long long)N * N;
  Cx<double> acc = mk(0.0, 0.0);
  for (int q = 0; q < N; ++q) cmac(acc, Yd[(long long)q * N + row], Ms[(long long)col * N + q]);
  if (dir == 0) acc = acc + shift * Ms[(long long)col * N + row];  // (X + shift) Minv
  Yt[t] = acc;
}

void prepare_coarsest_gcr(const Cx<double> *Y, Geo2 g, int N, Cx<double> *Minv, Cx<double> *Yt, Cx<double> *work,
                          int *info_dev, cudaStream_t s, double shift) {
  MG_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
  self_block_inverse_kernel<<<grid_for(g.nsites * 32, 128), 128, 0, s>>>(Y, Minv, work, g.nsites, N, info_dev,
                                                                         shift);
  MG_LAUNCHED();
  if (Yt == nullptr) return;
  precondition_stencil_kernel<<<grid_for(g.nsites * 5LL * N * N, 256), 256, 0, s>>>(Y, Minv, Yt, g.L0, g.L1, N,
                                                                                    shift);
  MG_LAUNCHED();
}

int coarsest_gcr_grid(int device) {
  int sms = 0;
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  return sms;
}

template <typename VT>
static void coarsest_gcr_go(const Cx<VT> *Yt, const Cx<double> *Minv, Geo2 g, int N, const Cx<double> *b,
                            Cx<double> *x, Cx<VT> *y, Cx<VT> *r, Cx<VT> *Z, Cx<VT> *W, double *partials,
                            unsigned int *bar, double tol, int restart, int max_iter, int *out, double *out_rel,
                            int grid, cudaStream_t s) {
  if (restart > kMaxRestart) fail(MG_ERR_INVALID_ARG, "coarsest restart exceeds 32");
  CgArgs<VT> a;
  a.Y = Yt;
  a.Minv = Minv;
  a.L0 = g.L0;
  a.L1 = g.L1;
  a.N = N;
  a.n = g.nsites * N;
  a.b = b;
  a.x = x;
  a.y = y;
  a.r = r;
  a.Z = Z;
  a.W = W;
  a.partials = partials;
  a.bar = bar;
  a.tol = tol;
  a.restart = restart;
  a.max_iter = max_iter;
  a.spin_limit = 1LL << 24;  // about a second of polling
  a.out = out;
  a.out_rel = out_rel;
  long long per = (a.n + grid - 1) / grid;
  int threads = (int)((per + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > 256) threads = 256;
  const size_t smem = (size_t)(9 + grid) * kSlots * sizeof(double);
  const void *fn = (N == 8) ? (const void *)coarsest_gcr_kernel<8, VT> : (const void *)coarsest_gcr_kernel<0, VT>;
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&per_sm, fn, threads, smem, 0));
  if (per_sm < 1) fail(MG_ERR_CUDA, "coarsest solve kernel cannot be resident");
  MG_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
  void *args[] = {&a};
  coop_launch(fn, dim3(grid), dim3(threads), args, smem, s);
  MG_LAUNCHED();
}

void launch_coarsest_gcr(const Cx<double> *Yt, const Cx<double> *Minv, Geo2 g, int N, const Cx<double> *b,
                         Cx<double> *x, Cx<double> *y, Cx<double> *r, Cx<double> *Z, Cx<double> *W, double *partials,
                         unsigned int *bar, double tol, int restart, int max_iter, int *out, double *out_rel, int grid,
                         cudaStream_t s) {
  coarsest_gcr_go<double>(Yt, Minv, g, N, b, x, y, r, Z, W, partials, bar, tol, restart, max_iter, out, out_rel, grid,
                          s);
}

void launch_coarsest_gcr32(const Cx<float> *Yt, const Cx<double> *Minv, Geo2 g, int N, const Cx<double> *b,
                           Cx<double> *x, Cx<float> *y, Cx<float> *r, Cx<float> *Z, Cx<float> *W, double *partials,
                           unsigned int *bar, double tol, int restart, int max_iter, int *out, double *out_rel,
                           int grid, cudaStream_t s) {
  coarsest_gcr_go<float>(Yt, Minv, g, N, b, x, y, r, Z, W, partials, bar, tol, restart, max_iter, out, out_rel, grid,
                         s);
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// Shared-memory-resident variant for small coarsest systems (N = 8, at most
// 8 coarse sites = 64 dofs per CTA, restart <= 16). Each CTA owns whole coarse
// sites and keeps, for the whole solve, its rows of A M, its blocks of M, its
// chunks of b, r, y and of the Krylov basis Z, W in shared memory; only r (and
// y at restarts) is published to global memory for the neighbours' stencil
// reads. Gram-Schmidt is classical with the Pythagorean norm; a second pass
// runs only when |w'|^2 < |w|^2 / 2 (the decision is made from the same grid
// sums in every CTA, so all CTAs take the same branch). A typical iteration
// costs 2 grid barriers: after the stencil + dot products, after the update.
// ---------------------------------------------------------------------------
constexpr int kSmMaxDofs = 64;
constexpr int kSmMaxRestart = 16;
constexpr int kSmSlots = 2 * kSmMaxRestart + 4;  // |w|^2, <w, r>, then 2 per basis vector

// RS: precision in which A M is stored and applied (double; float in mixed-precision cycles,
// where the Krylov vectors, Gram-Schmidt and updates stay FP64); rpub / ypub, the copies of r
// and y that neighbouring CTAs read for the stencil, are kept in RS too.
template <typename RS>
struct Cg3Args {
  const Cx<RS> *Yt;        // A M, internal layout [j][dir][col][row], N = 8
  const Cx<double> *Minv;  // [j][col][row]
  int L0, L1;
  long long nsites;
  int spc;  // sites per CTA
  const Cx<double> *b;
  Cx<double> *x;
  Cx<RS> *rpub, *ypub;
  double *partials;
  unsigned int *bar;
  double tol;
  int restart, max_iter;
  long long spin_limit;
  int *out;
  double *out_rel;
};

template <typename A>
__device__ __forceinline__ void grid_sync3(const A &a, bool &ok) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = a.bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(a.bar, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (++polls > a.spin_limit) {
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!good) atomicExch(a.out + 1, 1);
    s_ok = good;
  }
  __syncthreads();
  ok = ok && s_ok;
}

// cpart[0..nv) holds this CTA's sums; publish them slot-major (partials[s * G + cta]),
// barrier, and sum each slot over the CTAs into sres: a warp takes four slots at a time,
// each lane loads all its partials of them at once (lane l adds CTAs l, l + 32, ... in
// that order, then the shuffle tree: a fixed order in every CTA)
constexpr int kMaxGrid3 = 256;
template <typename A>
__device__ __forceinline__ void grid_sum3(const A &a, int nv, const double *cpart, double *sres, bool &ok) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = (int)gridDim.x;
  __syncthreads();
  for (int q = threadIdx.x; q < nv; q += blockDim.x) a.partials[(long long)q * G + blockIdx.x] = cpart[q];
  __threadfence();
  grid_sync3(a, ok);
  for (int q0 = wid * 4; q0 < nv; q0 += nw * 4) {
    double vals[4][kMaxGrid3 / 32];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double *src = a.partials + (long long)(q0 + u) * G;
#pragma unroll
      for (int i = 0; i < kMaxGrid3 / 32; ++i) {
        const int c = lane + 32 * i;
        vals[u][i] = (q0 + u < nv && c < G) ? __ldcg(src + c) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double t = 0.0;
#pragma unroll
      for (int i = 0; i < kMaxGrid3 / 32; ++i) t += vals[u][i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0 && q0 + u < nv) sres[q0 + u] = t;
    }
  }
  __syncthreads();
}

// out[d] = (A M v)_d for the CTA's rows, v read from global (published) memory;
// 4 threads per row, 10 of the 40 (dir, col) terms each, combined by shuffles
__device__ __forceinline__ Cx<double> ldcg_cx(const Cx<double> *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ Cx<float> ldcg_cx(const Cx<float> *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return mk(v.x, v.y);
}

template <typename RS>
__device__ __forceinline__ void stencil_rows(const Cg3Args<RS> &a, const Cx<RS> *Ys, const Cx<RS> *v,
                                             long long site0, int nd, Cx<double> *outs) {
  const int t = threadIdx.x, d = t >> 2, q = t & 3;
  Cx<RS> acc = mk<RS>(0, 0);
  if (d < nd) {
    const long long j = site0 + (d >> 3);
    const int x1 = (int)(j / a.L0), x0 = (int)(j - (long long)x1 * a.L0);
    const long long rowo = (long long)x1 * a.L0;
    long long src[5];
    src[0] = j;
    src[1] = rowo + (x0 + 1 == a.L0 ? 0 : x0 + 1);
    src[2] = rowo + (x0 == 0 ? a.L0 - 1 : x0 - 1);
    src[3] = (x1 + 1 == a.L1 ? 0 : rowo + a.L0) + x0;
    src[4] = (x1 == 0 ? (long long)(a.L1 - 1) * a.L0 : rowo - a.L0) + x0;
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int term = q * 10 + u, dir = term >> 3, col = term & 7;
      cmac(acc, Ys[(d * 5 + dir) * 8 + col], ldcg_cx(v + src[dir] * 8 + col));
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  if (d < nd && q == 0) outs[d] = cvt<double, RS>(acc);
}

// CTA-local sums: slot 0 |w|^2, slots 1, 2 <w, r>, slots 3 + 2j, 4 + 2j <W_j, w> (j < k);
// one warp per dot product, lanes over the CTA's dofs
__device__ __forceinline__ void cta_dots(int k, int nd, const Cx<double> *Ws, const Cx<double> *w,
                                         const Cx<double> *rs, double *cpart) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = wid; t < k + 2; t += nw) {
    double re = 0.0, im = 0.0;
    for (int d = lane; d < nd; d += 32) {
      const Cx<double> wd = w[d];
      if (t == 0) {
        re += norm2(wd);
      } else {
        const Cx<double> u = (t == 1) ? wd : Ws[(t - 2) * kSmMaxDofs + d];
        const Cx<double> v = (t == 1) ? rs[d] : wd;
        re += u.re * v.re + u.im * v.im;
        im += u.re * v.im - u.im * v.re;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      if (t == 0) {
        cpart[0] = re;
      } else if (t == 1) {
        cpart[1] = re;
        cpart[2] = im;
      } else {
        cpart[3 + 2 * (t - 2)] = re;
        cpart[4 + 2 * (t - 2)] = im;
      }
    }
  }
}

// two CTAs per SM (at most 128 registers, about 86 KB of shared memory each), so that the
// coarsest solves of two contexts running on different streams can share the GPU
template <typename RS>
__global__ void __launch_bounds__(256, 2) coarsest_gcr_smem_kernel(Cg3Args<RS> a) {
  extern __shared__ double sm3[];
  Cx<RS> *Ys = reinterpret_cast<Cx<RS> *>(sm3);                         // [64 rows][5][8]
  Cx<double> *Ms = reinterpret_cast<Cx<double> *>(Ys + kSmMaxDofs * 40);  // [8 sites][64]
  Cx<double> *bs = Ms + 8 * 64;
  Cx<double> *rs = bs + kSmMaxDofs;
  Cx<double> *ys = rs + kSmMaxDofs;
  Cx<double> *Zs = ys + kSmMaxDofs;                       // [16][64]
  Cx<double> *Ws = Zs + kSmMaxRestart * kSmMaxDofs;       // [16][64]
  double *cpart = reinterpret_cast<double *>(Ws + kSmMaxRestart * kSmMaxDofs);  // [kSmSlots]
  double *sres = cpart + kSmSlots;
  const int tid = threadIdx.x;
  const long long site0 = blockIdx.x * (long long)a.spc;
  long long ns = a.nsites - site0;
  if (ns > a.spc) ns = a.spc;
  if (ns < 0) ns = 0;
  const int nd = (int)ns * 8;
  const long long dof0 = site0 * 8;
  bool ok = true;

  for (int q = tid; q < nd * 40; q += blockDim.x) {
    const int d = q / 40, rem = q - d * 40, dir = rem >> 3, col = rem & 7;
    const long long j = site0 + (d >> 3);
    Ys[q] = a.Yt[(j * 5 + dir) * 64 + col * 8 + (d & 7)];
  }
  for (int q = tid; q < (int)ns * 64; q += blockDim.x) Ms[q] = a.Minv[site0 * 64 + q];
  for (int d = tid; d < nd; d += blockDim.x) {
    const Cx<double> bd = a.b[dof0 + d];
    bs[d] = bd;
    rs[d] = bd;
    ys[d] = mk(0.0, 0.0);
    a.rpub[dof0 + d] = cvt<RS, double>(bd);
  }
  __syncthreads();
  // |b|^2
  if (tid < 32) {
    double t = 0.0;
    for (int d = tid; d < nd; d += 32) t += norm2(bs[d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) cpart[0] = t;
  }
  grid_sum3(a, 1, cpart, sres, ok);
  if (!ok) return;
  const double bn2 = sres[0];
  const double tol2 = a.tol * a.tol * bn2;
  int it = 0;
  bool converged = !(bn2 > 0.0);
  double rn2 = bn2;
  while (!converged && it < a.max_iter) {
    for (int k = 0; k < a.restart && it < a.max_iter; ++k) {
      Cx<double> *Wk = Ws + k * kSmMaxDofs, *Zk = Zs + k * kSmMaxDofs;
      // w_k = (A M) r (neighbours from the published r), z_k = r
      stencil_rows(a, Ys, a.rpub, site0, nd, Wk);
      for (int d = tid; d < nd; d += blockDim.x) Zk[d] = rs[d];
      __syncthreads();
      cta_dots(k, nd, Ws, Wk, rs, cpart);
      grid_sum3(a, 3 + 2 * k, cpart, sres, ok);
      if (!ok) return;
      double nw0 = sres[0];
      double nw2 = nw0;
      for (int j = 0; j < k; ++j) nw2 -= sres[3 + 2 * j] * sres[3 + 2 * j] + sres[4 + 2 * j] * sres[4 + 2 * j];
      const double wr = sres[1], wi = sres[2];
      // first projection
      for (int d = tid; d < nd; d += blockDim.x) {
        Cx<double> w = Wk[d], z = Zk[d];
        for (int j = 0; j < k; ++j) {
          const Cx<double> bj = mk(-sres[3 + 2 * j], -sres[4 + 2 * j]);
          cmac(w, bj, Ws[j * kSmMaxDofs + d]);
          cmac(z, bj, Zs[j * kSmMaxDofs + d]);
        }
        Wk[d] = w;
        Zk[d] = z;
      }
      if (k > 0 && !(nw2 > 0.5 * nw0)) {
        // cancellation: project once more against the basis (same branch in every CTA)
        __syncthreads();
        cta_dots(k, nd, Ws, Wk, rs, cpart);
        grid_sum3(a, 3 + 2 * k, cpart, sres, ok);
        if (!ok) return;
        nw2 = sres[0];
        for (int j = 0; j < k; ++j) nw2 -= sres[3 + 2 * j] * sres[3 + 2 * j] + sres[4 + 2 * j] * sres[4 + 2 * j];
        for (int d = tid; d < nd; d += blockDim.x) {
          Cx<double> w = Wk[d], z = Zk[d];
          for (int j = 0; j < k; ++j) {
            const Cx<double> bj = mk(-sres[3 + 2 * j], -sres[4 + 2 * j]);
            cmac(w, bj, Ws[j * kSmMaxDofs + d]);
            cmac(z, bj, Zs[j * kSmMaxDofs + d]);
          }
          Wk[d] = w;
          Zk[d] = z;
        }
      }
      const bool breakdown = !(nw2 > 1e-28 * nw0);
      const double inv = breakdown ? 0.0 : 1.0 / sqrt(nw2);
      // <w', r> = <w, r> - sum conj(beta_j) <W_j, r>, and <W_j, r> vanishes (r is orthogonal to W_j)
      const Cx<double> alpha = mk(wr * inv, wi * inv);
      for (int d = tid; d < nd; d += blockDim.x) {
        const Cx<double> w = inv * Wk[d], z = inv * Zk[d];
        Wk[d] = w;
        Zk[d] = z;
        cmac(ys[d], alpha, z);
        Cx<double> rd = rs[d];
        cmac(rd, mk(-alpha.re, -alpha.im), w);
        rs[d] = rd;
        a.rpub[dof0 + d] = cvt<RS, double>(rd);
      }
      rn2 = fmax(rn2 - norm2(alpha), 0.0);
      ++it;
      __threadfence();
      grid_sync3(a, ok);
      if (!ok) return;
      if (rn2 <= tol2 || breakdown) break;
    }
    // true residual r = b - (A M) y with the published y
    for (int d = tid; d < nd; d += blockDim.x) a.ypub[dof0 + d] = cvt<RS, double>(ys[d]);
    __threadfence();
    grid_sync3(a, ok);
    if (!ok) return;
    stencil_rows(a, Ys, a.ypub, site0, nd, rs);
    __syncthreads();
    for (int d = tid; d < nd; d += blockDim.x) {
      const Cx<double> rd = bs[d] - rs[d];
      rs[d] = rd;
      a.rpub[dof0 + d] = cvt<RS, double>(rd);
    }
    __syncthreads();
    if (tid < 32) {
      double t = 0.0;
      for (int d = tid; d < nd; d += 32) t += norm2(rs[d]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (tid == 0) cpart[0] = t;
    }
    __threadfence();
    grid_sum3(a, 1, cpart, sres, ok);
    if (!ok) return;
    rn2 = sres[0];
    converged = rn2 <= tol2;
    if (!(rn2 == rn2)) break;
  }
  // x = M y on the CTA's sites (site-local)
  for (int d = tid; d < nd; d += blockDim.x) {
    const int sl = d >> 3, row = d & 7;
    Cx<double> acc = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) cmac(acc, Ms[sl * 64 + c * 8 + row], ys[sl * 8 + c]);
    a.x[dof0 + d] = acc;
  }
  if (blockIdx.x == 0 && tid == 0) {
    atomicAdd(a.out, it);
    if (!converged) atomicAdd(a.out + 2, 1);
    a.out_rel[0] = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
  }
}

bool coarsest_smem_fits(Geo2 g, int N, int restart, int sms) {
  if (N != 8 || restart > kSmMaxRestart) return false;
  const long long spc = (g.nsites + sms - 1) / sms;
  return spc * 8 <= kSmMaxDofs;
}

template <typename RS>
static void coarsest_smem_go(const Cx<RS> *Yt, const Cx<double> *Minv, Geo2 g, const Cx<double> *b, Cx<double> *x,
                             Cx<double> *rpub, Cx<double> *ypub, double *partials, unsigned int *bar, double tol,
                             int restart, int max_iter, int *out, double *out_rel, int sms, cudaStream_t s) {
  Cg3Args<RS> a;
  a.Yt = Yt;
  a.Minv = Minv;
  a.L0 = g.L0;
  a.L1 = g.L1;
  a.nsites = g.nsites;
  a.spc = (int)((g.nsites + sms - 1) / sms);
  const int grid = (int)((g.nsites + a.spc - 1) / a.spc);
  a.b = b;
  a.x = x;
  // the published copies fit in the FP64 buffers whatever RS is
  a.rpub = reinterpret_cast<Cx<RS> *>(rpub);
  a.ypub = reinterpret_cast<Cx<RS> *>(ypub);
  a.partials = partials;
  a.bar = bar;
  a.tol = tol;
  a.restart = restart;
  a.max_iter = max_iter;
  a.spin_limit = 1LL << 24;
  a.out = out;
  a.out_rel = out_rel;
  if (grid > kMaxGrid3) fail(MG_ERR_UNSUPPORTED, "coarsest solve: more than 256 CTAs");
  const size_t smem = (size_t)kSmMaxDofs * 40 * sizeof(Cx<RS>) +
                      (size_t)(8 * 64 + 3 * kSmMaxDofs + 2 * kSmMaxRestart * kSmMaxDofs) * sizeof(Cx<double>) +
                      (size_t)2 * kSmSlots * sizeof(double);
  const void *fn = (const void *)coarsest_gcr_smem_kernel<RS>;
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&per_sm, fn, 256, smem, 0));
  if (per_sm < 1) fail(MG_ERR_CUDA, "coarsest solve kernel (shared-memory variant) cannot be resident");
  MG_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
  void *args[] = {&a};
  coop_launch(fn, dim3(grid), dim3(256), args, smem, s);
  MG_LAUNCHED();
}

void launch_coarsest_gcr_smem(const Cx<double> *Yt, const Cx<float> *Yt32, const Cx<double> *Minv, Geo2 g,
                              const Cx<double> *b, Cx<double> *x, Cx<double> *rpub, Cx<double> *ypub,
                              double *partials, unsigned int *bar, double tol, int restart, int max_iter, int *out,
                              double *out_rel, int sms, cudaStream_t s) {
  if (Yt32 != nullptr)
    coarsest_smem_go<float>(Yt32, Minv, g, b, x, rpub, ypub, partials, bar, tol, restart, max_iter, out, out_rel, sms,
                            s);
  else
    coarsest_smem_go<double>(Yt, Minv, g, b, x, rpub, ypub, partials, bar, tol, restart, max_iter, out, out_rel, sms,
                             s);
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// Self-test of the bounded grid barrier: a 2-CTA cooperative kernel waits at a
// barrier that expects `expected` arrivals. With expected = 3 the generation
// flag never advances (nothing sets it), every wait gives up after
// `spin_limit` polls, status[0] records the timeout and the kernel returns.
// ---------------------------------------------------------------------------
__global__ void barrier_selftest_kernel(unsigned int *bar, unsigned int expected, long long spin_limit, int *status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    int good = 1;
    if (arrived == expected - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (++polls > spin_limit) {
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!good) atomicExch(status, 1);
    s_ok = good;
  }
  __syncthreads();
  if (!s_ok) return;
}

int barrier_selftest(unsigned int expected, long long spin_limit, cudaStream_t s) {
  DevBuf<unsigned int> bar;
  DevBuf<int> status;
  bar.alloc(2);
  status.alloc(1);
  pool_ready();
  MG_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned int), s));
  MG_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  void *args[] = {&bar.p, &expected, &spin_limit, &status.p};
  coop_launch((const void *)barrier_selftest_kernel, dim3(2), dim3(32), args, 0, s);
  MG_LAUNCHED();
  int h = 0;
  MG_CUDA(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// Batched shared-memory coarsest GCR: up to kBatchMaxVecs right-hand sides in
// lockstep in one persistent cooperative launch, so that all of them share
// the grid barriers (2 per iteration). Vector v solves (Y + shift_v) x_v = b_v
// with right block-Jacobi preconditioning M_v = blockdiag((X_j + shift_v)^-1)
// (the raw stencil Y is kept once in shared memory, the blocks of M_v per
// vector). The Krylov directions are kept in x-space: z_k = M_v r, w_k = A_v z_k,
// x += alpha z_k, so no final M multiply is needed. Each CTA owns whole coarse
// sites; z = M r is formed on the CTA's own sites right after the update and
// published for the neighbours' stencil reads. A vector whose tracked residual
// meets the tolerance, or whose basis breaks down, stops for the rest of the
// cycle; every restart recomputes the true residuals and reactivates the
// vectors that missed it. Grid sums are in fixed order (partials stored slot-
// major, each warp summing whole slots over the CTAs in CTA order).
// ---------------------------------------------------------------------------
constexpr int kBatchMaxVecs = 4;

struct CgBArgs {
  const Cx<double> *Y;     // stencil at the context mass, [j][dir][col][row], N = 8
  const Cx<double> *Minv;  // vector v: Minv + v * minv_stride, [j][col][row]
  long long minv_stride;
  const double *shift;     // vector v: diagonal shift (device) or null
  int L0, L1;
  long long nsites;
  int spc;  // sites per CTA
  int nb;   // vectors (<= kBatchMaxVecs)
  const Cx<double> *b;
  Cx<double> *x, *upub, *xpub;  // vector stride n
  double *partials;             // [slot][cta]
  unsigned int *bar;
  double tol;
  int restart, max_iter;
  long long spin_limit;
  int *out;
  double *out_rel;
};

__device__ __forceinline__ void grid_sync_b(const CgBArgs &a, bool &ok) {
  __shared__ int s_okb;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = a.bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(a.bar, 1u);
    int good = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (++polls > a.spin_limit) {
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!good) atomicExch(a.out + 1, 1);
    s_okb = good;
  }
  __syncthreads();
  ok = ok && s_okb;
}

// cpart[v * kSmSlots + s] (s < ns) holds this CTA's sums; the grid totals land in sres.
// Each warp takes four slots at a time and each lane loads all its partials of them at
// once (at most kMaxGridB CTAs), so a sum costs one L2 round trip per four slots. Lane l
// adds CTAs l, l + 32, ... in that order, then the shuffle tree: a fixed order.
constexpr int kMaxGridB = 256;
__device__ __forceinline__ void grid_sum_b(const CgBArgs &a, int ns, const double *cpart, double *sres, bool &ok) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = (int)gridDim.x;
  const int S = a.nb * ns;
  __syncthreads();
  for (int q = threadIdx.x; q < S; q += blockDim.x) {
    const int v = q / ns, sl = q - v * ns;
    a.partials[(long long)(v * kSmSlots + sl) * G + blockIdx.x] = cpart[v * kSmSlots + sl];
  }
  __threadfence();
  grid_sync_b(a, ok);
  for (int q0 = wid * 4; q0 < S; q0 += nw * 4) {
    double vals[4][kMaxGridB / 32];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u;
      const int v = q / ns, sl = q - v * ns;
      const double *src = a.partials + (long long)(v * kSmSlots + sl) * G;
#pragma unroll
      for (int i = 0; i < kMaxGridB / 32; ++i) {
        const int c = lane + 32 * i;
        vals[u][i] = (q < S && c < G) ? __ldcg(src + c) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double t = 0.0;
#pragma unroll
      for (int i = 0; i < kMaxGridB / 32; ++i) t += vals[u][i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int q = q0 + u;
      if (lane == 0 && q < S) {
        const int v = q / ns, sl = q - v * ns;
        sres[v * kSmSlots + sl] = t;
      }
    }
  }
  __syncthreads();
}

// per-vector shared-memory block: M blocks, then b, r, x, z (= M r) chunks, then Z, W
struct BVec {
  Cx<double> *Ms, *bs, *rs, *xs, *us, *Zs, *Ws;
};

__device__ __forceinline__ BVec bvec_at(Cx<double> *base, int v, int restart) {
  const int per = 8 * 64 + 4 * kSmMaxDofs + 2 * restart * kSmMaxDofs;
  Cx<double> *p = base + (long long)v * per;
  BVec r;
  r.Ms = p;
  r.bs = p + 8 * 64;
  r.rs = r.bs + kSmMaxDofs;
  r.xs = r.rs + kSmMaxDofs;
  r.us = r.xs + kSmMaxDofs;
  r.Zs = r.us + kSmMaxDofs;
  r.Ws = r.Zs + restart * kSmMaxDofs;
  return r;
}

// out_v[d] = ((Y + shift_v) pub_v)_d on the CTA's rows for the vectors with mask bit v;
// pub_v in global memory (neighbours), the self shift from the CTA's own copy self_v
// (us or xs, selected by `self_x`); 4 threads per row, 10 of the 40 terms each
__device__ __forceinline__ void stencil_rows_b(const CgBArgs &a, const Cx<double> *Ys, const Cx<double> *pub,
                                               Cx<double> *vbase, int restart, unsigned mask, bool self_x,
                                               long long site0, int nd, int kout) {
  const int t = threadIdx.x, d = t >> 2, q = t & 3;
  const long long n = a.nsites * 8;
  Cx<double> acc[kBatchMaxVecs];
#pragma unroll
  for (int v = 0; v < kBatchMaxVecs; ++v) acc[v] = mk(0.0, 0.0);
  if (d < nd) {
    const long long j = site0 + (d >> 3);
    const int x1 = (int)(j / a.L0), x0 = (int)(j - (long long)x1 * a.L0);
    const long long rowo = (long long)x1 * a.L0;
    long long src[5];
    src[0] = j;
    src[1] = rowo + (x0 + 1 == a.L0 ? 0 : x0 + 1);
    src[2] = rowo + (x0 == 0 ? a.L0 - 1 : x0 - 1);
    src[3] = (x1 + 1 == a.L1 ? 0 : rowo + a.L0) + x0;
    src[4] = (x1 == 0 ? (long long)(a.L1 - 1) * a.L0 : rowo - a.L0) + x0;
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int term = q * 10 + u, dir = term >> 3, col = term & 7;
      const Cx<double> yv = Ys[(d * 5 + dir) * 8 + col];
      const long long off = src[dir] * 8 + col;
#pragma unroll
      for (int v = 0; v < kBatchMaxVecs; ++v) {
        if (v < a.nb && ((mask >> v) & 1u)) {
          const double2 vv = __ldcg(reinterpret_cast<const double2 *>(pub + v * n + off));
          cmac(acc[v], yv, mk(vv.x, vv.y));
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < kBatchMaxVecs; ++v) {
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      acc[v].re += __shfl_xor_sync(0xffffffffu, acc[v].re, o);
      acc[v].im += __shfl_xor_sync(0xffffffffu, acc[v].im, o);
    }
  }
  if (d < nd && q == 0) {
#pragma unroll
    for (int v = 0; v < kBatchMaxVecs; ++v) {
      if (v < a.nb && ((mask >> v) & 1u)) {
        BVec B = bvec_at(vbase, v, restart);
        Cx<double> w = acc[v];
        if (a.shift != nullptr) {
          const double sv = a.shift[v];
          const Cx<double> own = self_x ? B.xs[d] : B.us[d];
          w.re = fma(sv, own.re, w.re);
          w.im = fma(sv, own.im, w.im);
        }
        if (kout < 0)
          B.rs[d] = B.bs[d] - w;  // residual form (restart): r = b - A x
        else
          B.Ws[kout * kSmMaxDofs + d] = w;
      }
    }
  }
}

// z = M_v r on the CTA's sites for the vectors in `mask`; stored in us and published
__device__ __forceinline__ void apply_m_b(const CgBArgs &a, Cx<double> *vbase, int restart, unsigned mask, int nd,
                                          long long dof0) {
  const long long n = a.nsites * 8;
  for (int q = threadIdx.x; q < a.nb * nd; q += blockDim.x) {
    const int v = q / nd, d = q - v * nd;
    if (!((mask >> v) & 1u)) continue;
    BVec B = bvec_at(vbase, v, restart);
    const int sl = d >> 3, row = d & 7;
    Cx<double> acc = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) cmac(acc, B.Ms[sl * 64 + c * 8 + row], B.rs[sl * 8 + c]);
    B.us[d] = acc;
    a.upub[v * n + dof0 + d] = acc;
  }
}

// CTA sums for the vectors in mask: slot 0 |w_k|^2, 1-2 <w_k, r>, 3 + 2j, 4 + 2j <W_j, w_k>
__device__ __forceinline__ void cta_dots_b(const CgBArgs &a, Cx<double> *vbase, int restart, unsigned mask, int k,
                                           int nd, double *cpart) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = k + 2;
  for (int task = wid; task < a.nb * per; task += nw) {
    const int v = task / per, t = task - v * per;
    double re = 0.0, im = 0.0;
    if ((mask >> v) & 1u) {
      BVec B = bvec_at(vbase, v, restart);
      const Cx<double> *w = B.Ws + k * kSmMaxDofs;
      for (int d = lane; d < nd; d += 32) {
        const Cx<double> wd = w[d];
        if (t == 0) {
          re += norm2(wd);
        } else {
          const Cx<double> u = (t == 1) ? wd : B.Ws[(t - 2) * kSmMaxDofs + d];
          const Cx<double> vv = (t == 1) ? B.rs[d] : wd;
          re += u.re * vv.re + u.im * vv.im;
          im += u.re * vv.im - u.im * vv.re;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      double *cp = cpart + v * kSmSlots;
      if (t == 0) {
        cp[0] = re;
      } else if (t == 1) {
        cp[1] = re;
        cp[2] = im;
      } else {
        cp[3 + 2 * (t - 2)] = re;
        cp[4 + 2 * (t - 2)] = im;
      }
    }
  }
}

// w_k -= sum_j beta_j W_j, z_k likewise, for the vectors in mask (beta from sres)
__device__ __forceinline__ void project_b(const CgBArgs &a, Cx<double> *vbase, int restart, unsigned mask, int k,
                                          int nd, const double *sres) {
  for (int q = threadIdx.x; q < a.nb * nd; q += blockDim.x) {
    const int v = q / nd, d = q - v * nd;
    if (!((mask >> v) & 1u)) continue;
    BVec B = bvec_at(vbase, v, restart);
    const double *sr = sres + v * kSmSlots;
    Cx<double> w = B.Ws[k * kSmMaxDofs + d], z = B.Zs[k * kSmMaxDofs + d];
    for (int j = 0; j < k; ++j) {
      const Cx<double> bj = mk(-sr[3 + 2 * j], -sr[4 + 2 * j]);
      cmac(w, bj, B.Ws[j * kSmMaxDofs + d]);
      cmac(z, bj, B.Zs[j * kSmMaxDofs + d]);
    }
    B.Ws[k * kSmMaxDofs + d] = w;
    B.Zs[k * kSmMaxDofs + d] = z;
  }
}

__device__ __forceinline__ double pyth_norm(const double *sr, int k) {
  double nw2 = sr[0];
  for (int j = 0; j < k; ++j) nw2 -= sr[3 + 2 * j] * sr[3 + 2 * j] + sr[4 + 2 * j] * sr[4 + 2 * j];
  return nw2;
}

__global__ void __launch_bounds__(256, 1) coarsest_gcr_batch_kernel(CgBArgs a) {
  extern __shared__ double smb[];
  Cx<double> *Ys = reinterpret_cast<Cx<double> *>(smb);  // [64 rows][5][8]
  Cx<double> *vbase = Ys + kSmMaxDofs * 40;
  const int restart = a.restart;
  const int per = 8 * 64 + 4 * kSmMaxDofs + 2 * restart * kSmMaxDofs;
  double *cpart = reinterpret_cast<double *>(vbase + (long long)kBatchMaxVecs * per);  // [v][kSmSlots]
  double *sres = cpart + kBatchMaxVecs * kSmSlots;
  __shared__ double s_bn2[kBatchMaxVecs], s_rn2[kBatchMaxVecs], s_nw0[kBatchMaxVecs], s_nw2[kBatchMaxVecs],
      s_wr[kBatchMaxVecs], s_wi[kBatchMaxVecs];
  __shared__ int s_it[kBatchMaxVecs];
  const int tid = threadIdx.x;
  const int nb = a.nb;
  const long long n = a.nsites * 8;
  const long long site0 = blockIdx.x * (long long)a.spc;
  long long ns = a.nsites - site0;
  if (ns > a.spc) ns = a.spc;
  if (ns < 0) ns = 0;
  const int nd = (int)ns * 8;
  const long long dof0 = site0 * 8;
  bool ok = true;
  const unsigned all = (1u << nb) - 1u;

  for (int q = tid; q < nd * 40; q += blockDim.x) {
    const int d = q / 40, rem = q - d * 40, dir = rem >> 3, col = rem & 7;
    const long long j = site0 + (d >> 3);
    Ys[q] = a.Y[(j * 5 + dir) * 64 + col * 8 + (d & 7)];
  }
  for (int q = tid; q < nb * (int)ns * 64; q += blockDim.x) {
    const int v = q / ((int)ns * 64), e = q - v * (int)ns * 64;
    bvec_at(vbase, v, restart).Ms[e] = a.Minv[v * a.minv_stride + site0 * 64 + e];
  }
  for (int q = tid; q < nb * nd; q += blockDim.x) {
    const int v = q / nd, d = q - v * nd;
    BVec B = bvec_at(vbase, v, restart);
    const Cx<double> bd = a.b[v * n + dof0 + d];
    B.bs[d] = bd;
    B.rs[d] = bd;
    B.xs[d] = mk(0.0, 0.0);
  }
  __syncthreads();
  apply_m_b(a, vbase, restart, all, nd, dof0);
  // |b_v|^2
  for (int v = tid >> 5; v < nb; v += blockDim.x >> 5) {
    const int lane = tid & 31;
    BVec B = bvec_at(vbase, v, restart);
    double t = 0.0;
    for (int d = lane; d < nd; d += 32) t += norm2(B.bs[d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) cpart[v * kSmSlots] = t;
  }
  __threadfence();
  grid_sum_b(a, 1, cpart, sres, ok);
  if (!ok) return;
  unsigned done = 0u;  // vectors whose true residual met the tolerance
  if (tid < nb) {
    s_bn2[tid] = sres[tid * kSmSlots];
    s_rn2[tid] = s_bn2[tid];
    s_it[tid] = 0;
  }
  __syncthreads();
  for (int v = 0; v < nb; ++v)
    if (!(s_bn2[v] > 0.0)) done |= 1u << v;
  const double tol2f = a.tol * a.tol;
  int iter = 0;
  while (done != all && iter < a.max_iter) {
    unsigned act = all & ~done;
    int k = 0;
    for (; k < restart && iter < a.max_iter && act != 0u; ++k) {
      // w_k = A_v z with z = M_v r published; z_k = z
      stencil_rows_b(a, Ys, a.upub, vbase, restart, act, false, site0, nd, k);
      for (int q = tid; q < nb * nd; q += blockDim.x) {
        const int v = q / nd, d = q - v * nd;
        if ((act >> v) & 1u) {
          BVec B = bvec_at(vbase, v, restart);
          B.Zs[k * kSmMaxDofs + d] = B.us[d];
        }
      }
      __syncthreads();
      cta_dots_b(a, vbase, restart, act, k, nd, cpart);
      grid_sum_b(a, 3 + 2 * k, cpart, sres, ok);
      if (!ok) return;
      unsigned cancel = 0u;
      for (int v = 0; v < nb; ++v) {
        if (!((act >> v) & 1u)) continue;
        const double *sr = sres + v * kSmSlots;
        const double nw2 = pyth_norm(sr, k);
        if (k > 0 && !(nw2 > 0.5 * sr[0])) cancel |= 1u << v;
      }
      __syncthreads();
      if (tid < nb && ((act >> tid) & 1u)) {
        const double *sr = sres + tid * kSmSlots;
        s_nw0[tid] = sr[0];
        s_nw2[tid] = pyth_norm(sr, k);
        s_wr[tid] = sr[1];
        s_wi[tid] = sr[2];
      }
      project_b(a, vbase, restart, act, k, nd, sres);
      if (cancel != 0u) {
        // second projection for the vectors that lost precision (same branch in every CTA)
        __syncthreads();
        cta_dots_b(a, vbase, restart, cancel, k, nd, cpart);
        grid_sum_b(a, 3 + 2 * k, cpart, sres, ok);
        if (!ok) return;
        if (tid < nb && ((cancel >> tid) & 1u)) s_nw2[tid] = pyth_norm(sres + tid * kSmSlots, k);
        project_b(a, vbase, restart, cancel, k, nd, sres);
        __syncthreads();
      }
      __syncthreads();
      // normalise and update; vectors that break down or meet the tolerance stop for this cycle
      unsigned upd = 0u;
      for (int v = 0; v < nb; ++v) {
        if (!((act >> v) & 1u)) continue;
        if (s_nw2[v] > 1e-28 * s_nw0[v]) upd |= 1u << v;
      }
      for (int q = tid; q < nb * nd; q += blockDim.x) {
        const int v = q / nd, d = q - v * nd;
        if (!((upd >> v) & 1u)) continue;
        BVec B = bvec_at(vbase, v, restart);
        const double inv = 1.0 / sqrt(s_nw2[v]);
        const Cx<double> alpha = mk(s_wr[v] * inv, s_wi[v] * inv);
        const Cx<double> w = inv * B.Ws[k * kSmMaxDofs + d], z = inv * B.Zs[k * kSmMaxDofs + d];
        B.Ws[k * kSmMaxDofs + d] = w;
        B.Zs[k * kSmMaxDofs + d] = z;
        cmac(B.xs[d], alpha, z);
        Cx<double> rd = B.rs[d];
        cmac(rd, mk(-alpha.re, -alpha.im), w);
        B.rs[d] = rd;
      }
      __syncthreads();
      apply_m_b(a, vbase, restart, upd, nd, dof0);
      for (int v = 0; v < nb; ++v) {
        if (!((act >> v) & 1u)) continue;
        if (!((upd >> v) & 1u)) {
          act &= ~(1u << v);  // breakdown: wait for the restart
          continue;
        }
        const double inv2 = 1.0 / s_nw2[v];
        const double rn2 = fmax(s_rn2[v] - (s_wr[v] * s_wr[v] + s_wi[v] * s_wi[v]) * inv2, 0.0);
        __syncthreads();
        if (tid == 0) {
          s_rn2[v] = rn2;
          s_it[v] += 1;
        }
        __syncthreads();
        if (rn2 <= tol2f * s_bn2[v]) act &= ~(1u << v);
      }
      ++iter;
      __threadfence();
      grid_sync_b(a, ok);
      if (!ok) return;
    }
    // true residuals r = b - A x of the unfinished vectors from the published x
    const unsigned live = all & ~done;
    for (int q = tid; q < nb * nd; q += blockDim.x) {
      const int v = q / nd, d = q - v * nd;
      if ((live >> v) & 1u) a.xpub[v * n + dof0 + d] = bvec_at(vbase, v, restart).xs[d];
    }
    __threadfence();
    grid_sync_b(a, ok);
    if (!ok) return;
    stencil_rows_b(a, Ys, a.xpub, vbase, restart, live, true, site0, nd, -1);
    __syncthreads();
    apply_m_b(a, vbase, restart, live, nd, dof0);
    for (int v = tid >> 5; v < nb; v += blockDim.x >> 5) {
      const int lane = tid & 31;
      double t = 0.0;
      if ((live >> v) & 1u) {
        BVec B = bvec_at(vbase, v, restart);
        for (int d = lane; d < nd; d += 32) t += norm2(B.rs[d]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) cpart[v * kSmSlots] = t;
    }
    __threadfence();
    grid_sum_b(a, 1, cpart, sres, ok);
    if (!ok) return;
    bool bad = false;
    for (int v = 0; v < nb; ++v) {
      if (!((live >> v) & 1u)) continue;
      const double rn2 = sres[v * kSmSlots];
      if (!(rn2 == rn2)) bad = true;
      if (rn2 <= tol2f * s_bn2[v]) done |= 1u << v;
    }
    __syncthreads();
    if (tid < nb && ((live >> tid) & 1u)) s_rn2[tid] = sres[tid * kSmSlots];
    __syncthreads();
    if (bad || k == 0) break;
  }
  for (int q = tid; q < nb * nd; q += blockDim.x) {
    const int v = q / nd, d = q - v * nd;
    a.x[v * n + dof0 + d] = bvec_at(vbase, v, restart).xs[d];
  }
  if (blockIdx.x == 0 && tid == 0) {
    int its = 0, missed = 0;
    double worst = 0.0;
    for (int v = 0; v < nb; ++v) {
      its += s_it[v];
      if (!((done >> v) & 1u)) ++missed;
      if (s_bn2[v] > 0.0) worst = fmax(worst, sqrt(s_rn2[v] / s_bn2[v]));
    }
    atomicAdd(a.out, its);
    if (missed) atomicAdd(a.out + 2, missed);
    a.out_rel[0] = worst;
  }
}

static size_t batch_smem_bytes(int restart) {
  const size_t per = 8 * 64 + 4 * kSmMaxDofs + 2 * (size_t)restart * kSmMaxDofs;
  return ((size_t)kSmMaxDofs * 40 + kBatchMaxVecs * per) * sizeof(Cx<double>) +
         2 * (size_t)kBatchMaxVecs * kSmSlots * sizeof(double);
}

bool coarsest_batch_fits(Geo2 g, int N, int restart, int sms) {
  if (!coarsest_smem_fits(g, N, restart, sms)) return false;
  return batch_smem_bytes(restart) <= 227 * 1024;
}

void launch_coarsest_gcr_batch(const Cx<double> *Y, const Cx<double> *Minv, long long minv_stride,
                               const double *shift, Geo2 g, int nb, const Cx<double> *b, Cx<double> *x,
                               Cx<double> *upub, Cx<double> *xpub, double *partials, unsigned int *bar, double tol,
                               int restart, int max_iter, int *out, double *out_rel, int sms, cudaStream_t s) {
  if (nb < 1 || nb > kBatchMaxVecs) fail(MG_ERR_INVALID_ARG, "batched coarsest solve: 1..4 vectors per launch");
  CgBArgs a;
  a.Y = Y;
  a.Minv = Minv;
  a.minv_stride = minv_stride;
  a.shift = shift;
  a.L0 = g.L0;
  a.L1 = g.L1;
  a.nsites = g.nsites;
  a.spc = (int)((g.nsites + sms - 1) / sms);
  a.nb = nb;
  const int grid = (int)((g.nsites + a.spc - 1) / a.spc);
  if (grid > kMaxGridB) fail(MG_ERR_UNSUPPORTED, "batched coarsest solve: more than 256 CTAs");
  a.b = b;
  a.x = x;
  a.upub = upub;
  a.xpub = xpub;
  a.partials = partials;
  a.bar = bar;
  a.tol = tol;
  a.restart = restart;
  a.max_iter = max_iter;
  a.spin_limit = 1LL << 24;
  a.out = out;
  a.out_rel = out_rel;
  const size_t smem = batch_smem_bytes(restart);
  const void *fn = (const void *)coarsest_gcr_batch_kernel;
  MG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&per_sm, fn, 256, smem, 0));
  if (per_sm < 1) fail(MG_ERR_CUDA, "batched coarsest solve kernel cannot be resident");
  MG_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
  void *args[] = {&a};
  coop_launch(fn, dim3(grid), dim3(256), args, smem, s);
  MG_LAUNCHED();
}

}  // namespace mg
