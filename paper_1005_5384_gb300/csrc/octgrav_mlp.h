// octgrav_mlp.h -- learned opening criterion: the feature definition shared by
// the walk kernel and the sample/label kernels, and the layout of the
// criterion record. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace og {

constexpr int MLP_NF = 12;  // inputs
constexpr int MLP_NH = 64;  // hidden units per layer
// Parameter vector: W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3.
constexpr int MLP_NPARAM = MLP_NH * MLP_NF + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1;  // 5057
// Criterion record (floats): mu[12], sigma[12], xmin[12], xmax[12], params[5057].
constexpr int MLP_RECORD = 4 * MLP_NF + MLP_NPARAM;  // 5105

// Device-side criterion in the layout the walk kernel copies to shared
// memory: tensor-core B fragments of W1^T and W2^T in bf16 (one uint2 per lane
// per 16x8 tile), FP32 biases, output weights and the input scaling.
struct MlpDevice {
  uint2 w1f[8][32];     // layer 1: 8 n-tiles (K = 16: 12 inputs + 4 zeros)
  uint2 w2f[4][8][32];  // layer 2: 4 k-steps x 8 n-tiles
  float b1[MLP_NH], b2[MLP_NH], w3[MLP_NH];
  float mu[16], isig[16], xmin[16], xmax[16];
  float b3, tau, pad0, pad1;
};

// Inputs of the learned criterion for a group and a candidate cell, in FP32
// (the definition the CPU oracle restates in FP64):
//   0 log2 l, 1 log2 d, 2 log2 |com - C_g|, 3 l/d, 4 log2 M, 5 |S|_F / (M l^2),
//   6 log2 count, 7..9 group half extents / l, 10 group count / N_group,
//   11 log2 |C_g - com_root|
// l = 2h (boundary cube side), d = distance between the group box and the cube,
// S the second moments about the centre of mass. Logarithms of values below
// 1e-30 are taken at 1e-30.
//   geo = (cube centre, h); q0 = (com_hi, M); q1 = (com_lo, count);
//   q2 = (3Sxx, 3Syy, 3Szz, 3Sxy); q3 = (3Sxz, 3Syz, ...)
__device__ __forceinline__ float mlp_lg2(float x) { return __log2f(fmaxf(x, 1e-30f)); }

__device__ __forceinline__ void mlp_features(float4 geo, float4 q0, float4 q1, float4 q2, float4 q3, float3 gmin,
                                             float3 gmax, float3 chi, float3 clo, float f10, float f11,
                                             float* f) {
  const float h = geo.w, l = 2.f * h;
  const float bx = fmaxf(0.f, fmaxf(gmin.x - (geo.x + h), (geo.x - h) - gmax.x));
  const float by = fmaxf(0.f, fmaxf(gmin.y - (geo.y + h), (geo.y - h) - gmax.y));
  const float bz = fmaxf(0.f, fmaxf(gmin.z - (geo.z + h), (geo.z - h) - gmax.z));
  const float d = sqrtf(bx * bx + by * by + bz * bz);
  const float rx = (q0.x - chi.x) + (q1.x - clo.x);
  const float ry = (q0.y - chi.y) + (q1.y - clo.y);
  const float rz = (q0.z - chi.z) + (q1.z - clo.z);
  const float sf = sqrtf(q2.x * q2.x + q2.y * q2.y + q2.z * q2.z +
                         2.f * (q2.w * q2.w + q3.x * q3.x + q3.y * q3.y)) * (1.f / 3.f);
  const float M = q0.w;
  f[0] = mlp_lg2(l);
  f[1] = mlp_lg2(d);
  f[2] = mlp_lg2(sqrtf(rx * rx + ry * ry + rz * rz));
  f[3] = l / d;
  f[4] = mlp_lg2(M);
  f[5] = M > 0.f ? sf / (M * l * l) : 0.f;
  f[6] = mlp_lg2(q1.w);
  f[7] = 0.5f * (gmax.x - gmin.x) / l;
  f[8] = 0.5f * (gmax.y - gmin.y) / l;
  f[9] = 0.5f * (gmax.z - gmin.z) / l;
  f[10] = f10;
  f[11] = f11;
}

}  // namespace og
