// Host side and C ABI of the learned near-null setup (mg_nullnet_*): the network's weights
// and Adam state, its forward pass over batches of gauge fields, the gradient of the
// rotation-invariant block loss against the plain setup's prolongator columns, and the
// training loop. Every arithmetic step runs in nullnet_kernels.cu; the host only sequences
// launches, picks the batches and reads the loss.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "nullnet.h"

struct mg_nullnet {
  int cin = 0, ch = 0, nv = 0;
  int ci[4] = {0, 0, 0, 0}, co[4] = {0, 0, 0, 0};
  long long off[5] = {0, 0, 0, 0, 0};  // complex offset of each layer's weights in the packed buffer
  mg::DevBuf<float2> W, gW, m1, m2;     // packed [l][5][2 co][2 ci]
  long long t = 0;                      // Adam steps taken
  // workspace for nf fields of V sites (grown on demand)
  long long cap = 0;                    // nf * V it was sized for
  mg::DevBuf<__nv_bfloat162> h[4];       // input of layer l ([f][x][2 ci])
  mg::DevBuf<float2> a[4];               // pre-activation of layer l ([f][x][2 co]); a[3] is the output
  mg::DevBuf<float2> g0, g1;             // gradient ping-pong ([f][x][32])
  mg::DevBuf<mg::Cx<double>> z64;        // noise draws
  mg::DevBuf<float2> U32, tgt32, parts;
  mg::DevBuf<double> lossb;
  mg::DevBuf<int> fmap;
  long long U32cap = 0, tgtcap = 0;
};

namespace mg {
namespace {

constexpr int kWeightParts = 152 * 2;  // CTAs of partial weight-gradient sums

void nn_ensure(mg_nullnet &n, long long nfV, int nf, long long nblocks) {
  if (nfV > n.cap) {
    for (int l = 0; l < 4; ++l) {
      n.h[l].alloc((size_t)nfV * 2 * n.ci[l]);
      n.a[l].alloc((size_t)nfV * 2 * n.co[l]);
    }
    n.g0.alloc((size_t)nfV * 32);
    n.g1.alloc((size_t)nfV * 32);
    n.z64.alloc((size_t)nfV * 2 * n.cin);
    n.cap = nfV;
  }
  if ((long long)n.lossb.n < (long long)nf * nblocks) n.lossb.alloc((size_t)nf * nblocks);
  if (n.parts.p == nullptr) n.parts.alloc((size_t)kWeightParts * 5 * 32 * 32);
  if ((long long)n.fmap.n < nf) n.fmap.alloc((size_t)nf);
  pool_ready();
}

void nn_validate_geom(const mg_geom *g) {
  if (!g) fail(MG_ERR_INVALID_ARG, "null geometry");
  if (g->d != 2 || g->Nc != 1) fail(MG_ERR_UNSUPPORTED, "the learned setup is built for d = 2, Nc = 1");
  if (g->dims[0] < 2 || g->dims[1] < 2) fail(MG_ERR_INVALID_ARG, "lattice extents must be >= 2");
}

// noise of nf fields (seed per field) into h[0]
void nn_noise(mg_nullnet &n, long long V, int nf, const uint64_t *seeds, cudaStream_t s) {
  for (int f = 0; f < nf; ++f)
    for (int c = 0; c < n.cin; ++c)
      launch_gaussian(n.z64.p + ((size_t)c * nf + f) * V * 2, V * 2, seeds[f], c, kNullnetNoiseTag, s);
  launch_pack_noise(n.z64.p, n.cin, V, nf, n.h[0].p, s);
}

// the four layers on nf fields whose float2 links are U32 (through fmap when given)
void nn_forward(mg_nullnet &n, const mg_geom &g, int nf, const float2 *U32, const int *fmap, bool keep,
                cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    const bool last = l == 3;
    launch_ptconv_fwd(n.h[l].p, U32, fmap, n.W.p + n.off[l], 2 * n.ci[l], 2 * n.co[l], g.dims[0], g.dims[1], nf,
                      last, (keep || last) ? n.a[l].p : nullptr, last ? nullptr : n.h[l + 1].p, s);
  }
}

BlockGeo nn_blocks(const mg_geom &g, const int *block) {
  const int L0 = g.dims[0], L1 = g.dims[1], B0 = block[0], B1 = block[1];
  if (B0 < 1 || B1 < 1 || L0 % B0 || L1 % B1) fail(MG_ERR_INVALID_ARG, "extents not divisible by the block");
  if (B0 * B1 * 2 > 32) fail(MG_ERR_UNSUPPORTED, "the loss kernel takes blocks of at most 16 sites");
  return BlockGeo{L0, L1, B0, B1, L0 / B0, L1 / B1, B0 * B1, 2, B0 * B1 * 2, (long long)(L0 / B0) * (L1 / B1)};
}

// loss of the forward pass just run (a[3]) against float2 targets, and the weight gradient in gW
double nn_backward(mg_nullnet &n, const mg_geom &g, int nf, const float2 *U32, const int *fmap,
                   const float2 *tgt, const BlockGeo &bg, cudaStream_t s) {
  const float scale = (float)(1.0 / ((double)bg.nblocks * n.nv * nf));
  launch_nullnet_loss(n.a[3].p, tgt, fmap, n.nv, bg, nf, scale, n.g0.p, n.lossb.p, s);
  float2 *ga = n.g0.p, *gn = n.g1.p;
  for (int l = 3; l >= 0; --l) {
    launch_ptconv_bwd_weight(ga, n.h[l].p, U32, fmap, nf, 2 * n.ci[l], 2 * n.co[l], g.dims[0], g.dims[1], n.parts.p,
                             kWeightParts, n.gW.p + n.off[l], s);
    if (l > 0) {
      launch_ptconv_bwd_data(ga, U32, fmap, n.W.p + n.off[l], 2 * n.ci[l], 2 * n.co[l], g.dims[0], g.dims[1], nf,
                             n.a[l - 1].p, gn, s);
      std::swap(ga, gn);
    }
  }
  std::vector<double> lb((size_t)nf * bg.nblocks);
  MG_CUDA(cudaMemcpyAsync(lb.data(), n.lossb.p, lb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  double tot = 0.0;
  for (double v : lb) tot += v;
  if (!std::isfinite(tot)) fail(MG_ERR_NAN, "learned setup: the loss is not finite");
  return tot / ((double)bg.nblocks * n.nv * nf);
}

// deterministic host generator for the initial weights (splitmix64 + Box-Muller)
double init_gauss(uint64_t &st) {
  auto next = [&st]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  const double u1 = ((next() >> 11) + 1) * (1.0 / 9007199254740992.0);
  const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

template <typename F>
int nn_guarded(F &&f) {
  try {
    f();
    set_last_error("");
    return MG_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return MG_ERR_OOM;
  } catch (...) {
    set_last_error("unexpected exception");
    return MG_ERR_CUDA;
  }
}

}  // namespace

// predicted near-null vectors (complex128 [k][x][2]) for one field: used by mg_setup_learned
void nullnet_predict(mg_nullnet &n, const mg_geom &g, const void *U, uint64_t seed, Cx<double> *out,
                     cudaStream_t s) {
  nn_validate_geom(&g);
  const long long V = (long long)g.dims[0] * g.dims[1];
  nn_ensure(n, V, 1, 1);
  if ((long long)n.U32.n < V * 2) {
    n.U32.alloc((size_t)V * 2);
    pool_ready();
  }
  launch_to_float2(static_cast<const Cx<double> *>(U), V * 2, n.U32.p, s);
  nn_noise(n, V, 1, &seed, s);
  nn_forward(n, g, 1, n.U32.p, nullptr, false, s);
  launch_unpack_vectors(n.a[3].p, n.nv, V, out, s);
}

int nullnet_nv(const mg_nullnet &n) { return n.nv; }

}  // namespace mg

using namespace mg;

extern "C" {

int mg_nullnet_create(mg_nullnet **net, int cin, int channels, int nv, uint64_t seed) {
  return nn_guarded([&] {
    if (!net) fail(MG_ERR_INVALID_ARG, "null out-pointer");
    *net = nullptr;
    if (cin < 1 || cin > 16 || channels < 1 || channels > 16 || nv < 1 || nv > 8)
      fail(MG_ERR_INVALID_ARG, "cin and channels must be in [1, 16], nv in [1, 8]");
    auto n = std::make_unique<mg_nullnet>();
    n->cin = cin;
    n->ch = channels;
    n->nv = nv;
    const int dims[5] = {cin, channels, channels, channels, nv};
    for (int l = 0; l < 4; ++l) {
      n->ci[l] = dims[l];
      n->co[l] = dims[l + 1];
      n->off[l + 1] = n->off[l] + 5LL * 2 * n->co[l] * 2 * n->ci[l];
    }
    const long long nw = n->off[4];
    std::vector<float2> w((size_t)nw);
    uint64_t st = seed;
    for (int l = 0; l < 4; ++l) {
      const double sd = std::sqrt(0.5 / (5.0 * 2 * n->ci[l]));  // keeps the per-component variance
      for (long long q = n->off[l]; q < n->off[l + 1]; ++q)
        w[(size_t)q] = make_float2((float)(sd * init_gauss(st)), (float)(sd * init_gauss(st)));
    }
    n->W.alloc((size_t)nw);
    n->gW.alloc((size_t)nw);
    n->m1.alloc((size_t)nw);
    n->m2.alloc((size_t)nw);
    pool_ready();
    MG_CUDA(cudaMemcpy(n->W.p, w.data(), nw * sizeof(float2), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemset(n->m1.p, 0, nw * sizeof(float2)));
    MG_CUDA(cudaMemset(n->m2.p, 0, nw * sizeof(float2)));
    MG_CUDA(cudaMemset(n->gW.p, 0, nw * sizeof(float2)));
    *net = n.release();
  });
}

void mg_nullnet_destroy(mg_nullnet *net) { delete net; }

long long mg_nullnet_weight_count(const mg_nullnet *net) { return net ? net->off[4] : 0; }

int mg_nullnet_get_weights(mg_nullnet *net, void *out) {
  return nn_guarded([&] {
    if (!net || !out) fail(MG_ERR_INVALID_ARG, "null pointer");
    MG_CUDA(cudaMemcpy(out, net->W.p, net->off[4] * sizeof(float2), cudaMemcpyDeviceToHost));
  });
}

int mg_nullnet_set_weights(mg_nullnet *net, const void *in) {
  return nn_guarded([&] {
    if (!net || !in) fail(MG_ERR_INVALID_ARG, "null pointer");
    MG_CUDA(cudaMemcpy(net->W.p, in, net->off[4] * sizeof(float2), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemset(net->m1.p, 0, net->off[4] * sizeof(float2)));
    MG_CUDA(cudaMemset(net->m2.p, 0, net->off[4] * sizeof(float2)));
    net->t = 0;
  });
}

int mg_nullnet_forward(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const uint64_t *noise_seeds,
                       void *out, void *stream) {
  return nn_guarded([&] {
    if (!net || !U || !noise_seeds || !out) fail(MG_ERR_INVALID_ARG, "null pointer");
    nn_validate_geom(g);
    if (nfields < 1 || nfields > 65535) fail(MG_ERR_INVALID_ARG, "nfields must be in [1, 65535]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long V = (long long)g->dims[0] * g->dims[1];
    nn_ensure(*net, V * nfields, nfields, 1);
    if ((long long)net->U32.n < V * 2 * nfields) {
      net->U32.alloc((size_t)V * 2 * nfields);
      pool_ready();
    }
    launch_to_float2(static_cast<const Cx<double> *>(U), V * 2 * nfields, net->U32.p, s);
    nn_noise(*net, V, nfields, noise_seeds, s);
    nn_forward(*net, *g, nfields, net->U32.p, nullptr, false, s);
    MG_CUDA(cudaMemcpyAsync(out, net->a[3].p, (size_t)nfields * V * 2 * net->nv * sizeof(float2),
                            cudaMemcpyDeviceToDevice, s));
    MG_CUDA(cudaStreamSynchronize(s));
  });
}

int mg_nullnet_gradient(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const uint64_t *noise_seeds,
                        const void *target, const int *block, double *loss, void *grad, void *stream) {
  return nn_guarded([&] {
    if (!net || !U || !noise_seeds || !target || !block) fail(MG_ERR_INVALID_ARG, "null pointer");
    nn_validate_geom(g);
    if (nfields < 1 || nfields > 65535) fail(MG_ERR_INVALID_ARG, "nfields must be in [1, 65535]");
    const BlockGeo bg = nn_blocks(*g, block);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long V = (long long)g->dims[0] * g->dims[1];
    nn_ensure(*net, V * nfields, nfields, bg.nblocks);
    if ((long long)net->U32.n < V * 2 * nfields) net->U32.alloc((size_t)V * 2 * nfields);
    if ((long long)net->tgt32.n < V * 2 * net->nv * nfields) net->tgt32.alloc((size_t)V * 2 * net->nv * nfields);
    pool_ready();
    launch_to_float2(static_cast<const Cx<double> *>(U), V * 2 * nfields, net->U32.p, s);
    launch_to_float2(static_cast<const Cx<double> *>(target), V * 2 * net->nv * nfields, net->tgt32.p, s);
    nn_noise(*net, V, nfields, noise_seeds, s);
    nn_forward(*net, *g, nfields, net->U32.p, nullptr, true, s);
    const double l = nn_backward(*net, *g, nfields, net->U32.p, nullptr, net->tgt32.p, bg, s);
    if (loss) *loss = l;
    if (grad) MG_CUDA(cudaMemcpy(grad, net->gW.p, net->off[4] * sizeof(float2), cudaMemcpyDeviceToHost));
  });
}

int mg_nullnet_train(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const void *target,
                     const int *block, int steps, int batch, double lr, uint64_t seed, double *losses,
                     void *stream) {
  return nn_guarded([&] {
    if (!net || !U || !target || !block) fail(MG_ERR_INVALID_ARG, "null pointer");
    nn_validate_geom(g);
    if (nfields < 1 || batch < 1 || batch > nfields || steps < 0 || !(lr > 0.0))
      fail(MG_ERR_INVALID_ARG, "need 1 <= batch <= nfields, steps >= 0 and lr > 0");
    const BlockGeo bg = nn_blocks(*g, block);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long V = (long long)g->dims[0] * g->dims[1];
    nn_ensure(*net, V * batch, batch, bg.nblocks);
    // links and targets of every field in float2, once
    net->U32.alloc((size_t)V * 2 * nfields);
    net->tgt32.alloc((size_t)V * 2 * net->nv * nfields);
    pool_ready();
    launch_to_float2(static_cast<const Cx<double> *>(U), V * 2 * nfields, net->U32.p, s);
    launch_to_float2(static_cast<const Cx<double> *>(target), V * 2 * net->nv * nfields, net->tgt32.p, s);
    std::vector<int> fm(batch);
    std::vector<uint64_t> seeds(batch);
    for (int step = 0; step < steps; ++step) {
      // batch: a cyclic walk through the fields (every field once per epoch), fresh noise per draw
      for (int j = 0; j < batch; ++j) {
        const long long draw = (long long)step * batch + j;
        fm[j] = (int)(draw % nfields);
        seeds[j] = seed + ((uint64_t)draw << 20);
      }
      MG_CUDA(cudaMemcpyAsync(net->fmap.p, fm.data(), batch * sizeof(int), cudaMemcpyHostToDevice, s));
      nn_noise(*net, V, batch, seeds.data(), s);
      nn_forward(*net, *g, batch, net->U32.p, net->fmap.p, true, s);
      const double l = nn_backward(*net, *g, batch, net->U32.p, net->fmap.p, net->tgt32.p, bg, s);
      if (losses) losses[step] = l;
      ++net->t;
      launch_adam(reinterpret_cast<float *>(net->W.p), reinterpret_cast<const float *>(net->gW.p),
                  reinterpret_cast<float *>(net->m1.p), reinterpret_cast<float *>(net->m2.p), 2 * net->off[4],
                  (float)lr, net->t, s);
    }
    MG_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
