// Internal interface of the learned near-null setup (kernels in nullnet_kernels.cu, host
// code and C ABI in nullnet.cu). Layouts are described in nullnet_kernels.cu.
#pragma once

#include "kernels.h"

namespace mg {

constexpr int kNullnetNoiseTag = 0x4E4E;  // level field of the Philox draws of the noise input

// one layer: a = sum_dir W_dir T_dir(h_in); hidden layers also write the gated bf16 h_out
void launch_ptconv_fwd(const void *h_in, const float2 *U, const int *fmap, const float2 *W, int ci2, int co2,
                       int L0, int L1, int nf, bool last, float2 *a_out, void *h_out, cudaStream_t s);
// dL/dh^* of the layer input (through the previous gate when a_prev is given)
void launch_ptconv_bwd_data(const float2 *ga, const float2 *U, const int *fmap, const float2 *W, int ci2, int co2,
                            int L0, int L1, int nf, const float2 *a_prev, float2 *ga_prev, cudaStream_t s);
// dL/dW^* of a layer (nparts CTAs of partial sums, then a fixed-order sum)
void launch_ptconv_bwd_weight(const float2 *ga, const void *h_in, const float2 *U, const int *fmap, int nf, int ci2,
                              int co2, int L0, int L1, float2 *partials, int nparts, float2 *gW, cudaStream_t s);
// block loss L_b per (field, block) into lossb and scale * dL/dy^* into gy
void launch_nullnet_loss(const float2 *y, const float2 *target, const int *fmap, int nv, const BlockGeo &bg, int nf,
                         float scale, float2 *gy, double *lossb, cudaStream_t s);
void launch_adam(float *w, const float *g, float *m1, float *m2, long long n, float lr, long long t, cudaStream_t s);
void launch_pack_noise(const Cx<double> *z, int cin, long long V, int nf, void *h, cudaStream_t s);
void launch_unpack_vectors(const float2 *y, int nv, long long V, Cx<double> *out, cudaStream_t s);
void launch_to_float2(const Cx<double> *a, long long n, float2 *b, cudaStream_t s);

// the network's Nv predicted vectors (complex128 [k][x][2]) for one field U (complex128 [x][2])
void nullnet_predict(mg_nullnet &n, const mg_geom &g, const void *U, uint64_t seed, Cx<double> *out, cudaStream_t s);
int nullnet_nv(const mg_nullnet &n);

}  // namespace mg
