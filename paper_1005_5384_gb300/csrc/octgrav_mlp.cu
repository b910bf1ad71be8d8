// octgrav_mlp.cu -- learned opening criterion: training samples (features and
// FP64 error labels) and training (FP32 forward/backward of the 12-64-64-1
// network, Adam), all on the GPU.
//
// A label is the error of accepting cell c for group g: the largest, over the
// group's particles i, of |a_multipole(c, i) - a_direct(members of c, i)| /
// |a_ref(i)|, with a_ref a tight reference of the particle's total
// acceleration. The network learns log10 of it from the inputs defined in
// octgrav_mlp.h; the walk then accepts a cell when the prediction is below a
// threshold.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "octgrav_internal.h"
#include "octgrav_mlp.h"

namespace og {
namespace {

// ---------------------------------------------------------------- samples

__global__ void feature_kernel(MlpSampleArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const int item = a.item[s], c = a.cell[s];
  const int4 it = a.items[item];
  const float4 b0 = a.ibox[4 * item], b1 = a.ibox[4 * item + 1], b2 = a.ibox[4 * item + 2];
  const float4 b3 = a.ibox[4 * item + 3];
  const float3 gmin = make_float3(b0.x, b0.y, b0.z), gmax = make_float3(b1.x, b1.y, b1.z);
  const float3 chi = make_float3(b0.w, b1.w, b2.w), clo = make_float3(b2.x, b2.y, b2.z);
  const float4 r0 = a.mp[4 * it.x], r1 = a.mp[4 * it.x + 1];  // root centre of mass (hi, lo)
  const float ox = (chi.x - r0.x) + (clo.x - r1.x), oy = (chi.y - r0.y) + (clo.y - r1.y),
              oz = (chi.z - r0.z) + (clo.z - r1.z);
  const float f10 = static_cast<float>(__float_as_int(b3.y)) / static_cast<float>(a.n_group);
  const float f11 = mlp_lg2(sqrtf(ox * ox + oy * oy + oz * oz));
  float f[MLP_NF];
  mlp_features(a.geo[c], a.mp[4 * c], a.mp[4 * c + 1], a.mp[4 * c + 2], a.mp[4 * c + 3], gmin, gmax, chi, clo, f10,
               f11, f);
  for (int k = 0; k < MLP_NF; ++k) a.feat[MLP_NF * s + k] = f[k];
}

// One warp per (sample, chunk of 32 group particles): lane = particle.
__global__ void label_kernel(MlpSampleArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int s = warp / a.chunks, chunk = warp % a.chunks;
  if (s >= a.n) return;
  const int item = a.item[s], c = a.cell[s];
  const float4 b3 = a.ibox[4 * item + 3];
  const int gfirst = __float_as_int(b3.x), gcount = __float_as_int(b3.y);
  const int k = chunk * 32 + lane;
  double e = 0.0;
  if (k < gcount) {
    const int i = gfirst + k;
    const float4 hi = a.parts[2 * i], lo = a.parts[2 * i + 1];
    const double xi = (double)hi.x + lo.x, yi = (double)hi.y + lo.y, zi = (double)hi.z + lo.z;
    // multipole (monopole + quadrupole, FP64 moments)
    const double* cm = a.com64 + 3 * c;
    const double* S = a.S64 + 6 * c;
    const double M = a.M64[c];
    const double y0 = xi - cm[0], y1 = yi - cm[1], y2 = zi - cm[2];
    const double r2 = y0 * y0 + y1 * y1 + y2 * y2 + a.eps2;
    const double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
    const double s0 = S[0] * y0 + S[3] * y1 + S[4] * y2;
    const double s1 = S[3] * y0 + S[1] * y1 + S[5] * y2;
    const double s2 = S[4] * y0 + S[5] * y1 + S[2] * y2;
    const double ySy = y0 * s0 + y1 * s1 + y2 * s2, tr = S[0] + S[1] + S[2];
    const double cy = -M / r3 - 7.5 * ySy / r7 + 1.5 * tr / r5;
    const double am0 = cy * y0 + 3.0 * s0 / r5, am1 = cy * y1 + 3.0 * s1 / r5, am2 = cy * y2 + 3.0 * s2 / r5;
    // direct sum over the cell's members
    const int2 lk = a.link_first_count[c];
    double ad0 = 0, ad1 = 0, ad2 = 0;
    for (int j = lk.x; j < lk.x + lk.y; ++j) {
      const float4 hj = a.parts[2 * j], lj = a.parts[2 * j + 1];
      const double dx = ((double)hj.x + lj.x) - xi, dy = ((double)hj.y + lj.y) - yi,
                   dz = ((double)hj.z + lj.z) - zi;
      const double rinv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz + a.eps2);
      const double mr3 = (double)hj.w * rinv * rinv * rinv;
      ad0 += mr3 * dx;
      ad1 += mr3 * dy;
      ad2 += mr3 * dz;
    }
    const float4 ar = a.aref[i];
    const double na = sqrt((double)ar.x * ar.x + (double)ar.y * ar.y + (double)ar.z * ar.z);
    const double ea = sqrt((am0 - ad0) * (am0 - ad0) + (am1 - ad1) * (am1 - ad1) + (am2 - ad2) * (am2 - ad2));
    e = na > 0 ? ea / na : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(a.label64 + s), __double_as_longlong(e));
}

// ---------------------------------------------------------------- training

// Counter-based uniform index in [0, n): splitmix64 of (seed, step, b).
__device__ __forceinline__ int sample_index(uint64_t seed, int step, int b, int n) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (static_cast<uint64_t>(step) * 1000003ull + b + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<int>(z % static_cast<uint64_t>(n));
}

constexpr int TB = 32;  // samples per block in the gradient kernel

// Gradient of L = sum_b (y_b - t_b)^2 / (2B) for the samples of one block,
// added to grad; L added to loss. Dense layer algebra written out per sample
// row and hidden unit, everything in shared memory.
__global__ void __launch_bounds__(256) grad_kernel(const float* __restrict__ w, const float* __restrict__ X,
                                                    const float* __restrict__ t, int n_total, int B, int step,
                                                    uint64_t seed, int use_all, float* grad, float* loss) {
  __shared__ float W[MLP_NPARAM];
  __shared__ float xs[TB][MLP_NF + 1];
  __shared__ float ts[TB];
  __shared__ float h1[TB][MLP_NH + 1];  // relu(z1); sign of z1 kept as h1 > 0
  __shared__ float z2[TB][MLP_NH + 1];  // becomes dz2
  __shared__ float d1[TB][MLP_NH + 1];  // dz1
  __shared__ float dy[TB];
  const int tid = threadIdx.x;
  const float* W1 = W;
  const float* b1 = W1 + MLP_NH * MLP_NF;
  const float* W2 = b1 + MLP_NH;
  const float* b2 = W2 + MLP_NH * MLP_NH;
  const float* w3 = b2 + MLP_NH;
  for (int k = tid; k < MLP_NPARAM; k += blockDim.x) W[k] = w[k];
  const int base = blockIdx.x * TB;
  const int nb = min(TB, B - base);
  for (int k = tid; k < TB * MLP_NF; k += blockDim.x) {
    const int r = k / MLP_NF, f = k % MLP_NF;
    float v = 0.f;
    if (r < nb) {
      const int sidx = use_all ? base + r : sample_index(seed, step, base + r, n_total);
      v = X[static_cast<size_t>(sidx) * MLP_NF + f];
      if (f == 0) ts[r] = t[sidx];
    }
    xs[r][f] = v;
  }
  __syncthreads();
  const float b3 = w3[MLP_NH];
  const float invB = 1.f / static_cast<float>(B);
  // layer 1
  for (int k = tid; k < TB * MLP_NH; k += blockDim.x) {
    const int r = k / MLP_NH, j = k % MLP_NH;
    float z = b1[j];
    for (int i = 0; i < MLP_NF; ++i) z = fmaf(W1[j * MLP_NF + i], xs[r][i], z);
    h1[r][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  // layer 2
  for (int k = tid; k < TB * MLP_NH; k += blockDim.x) {
    const int r = k / MLP_NH, j = k % MLP_NH;
    float z = b2[j];
    for (int i = 0; i < MLP_NH; ++i) z = fmaf(W2[j * MLP_NH + i], h1[r][i], z);
    z2[r][j] = z;
  }
  __syncthreads();
  // output, residual, loss
  if (tid < TB) {
    float y = b3;
    for (int j = 0; j < MLP_NH; ++j) y = fmaf(w3[j], fmaxf(z2[tid][j], 0.f), y);
    const float res = tid < nb ? y - ts[tid] : 0.f;
    dy[tid] = res * invB;
    atomicAdd(loss, 0.5f * res * res * invB);
  }
  __syncthreads();
  // output layer gradients
  float* gW1 = grad;
  float* gb1 = gW1 + MLP_NH * MLP_NF;
  float* gW2 = gb1 + MLP_NH;
  float* gb2 = gW2 + MLP_NH * MLP_NH;
  float* gw3 = gb2 + MLP_NH;
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g = fmaf(dy[r], fmaxf(z2[r][tid], 0.f), g);
    atomicAdd(gw3 + tid, g);
  }
  if (tid == MLP_NH) {
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g += dy[r];
    atomicAdd(gw3 + MLP_NH, g);
  }
  __syncthreads();
  // dz2 = dy w3 [z2 > 0]
  for (int k = tid; k < TB * MLP_NH; k += blockDim.x) {
    const int r = k / MLP_NH, j = k % MLP_NH;
    z2[r][j] = z2[r][j] > 0.f ? dy[r] * w3[j] : 0.f;
  }
  __syncthreads();
  // gW2[j][i] = sum_r dz2[r][j] h1[r][i]; gb2[j] = sum_r dz2[r][j]
  for (int k = tid; k < MLP_NH * MLP_NH; k += blockDim.x) {
    const int j = k / MLP_NH, i = k % MLP_NH;
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g = fmaf(z2[r][j], h1[r][i], g);
    atomicAdd(gW2 + k, g);
  }
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g += z2[r][tid];
    atomicAdd(gb2 + tid, g);
  }
  // dz1[r][i] = (sum_j dz2[r][j] W2[j][i]) [h1 > 0]
  for (int k = tid; k < TB * MLP_NH; k += blockDim.x) {
    const int r = k / MLP_NH, i = k % MLP_NH;
    float g = 0.f;
    for (int j = 0; j < MLP_NH; ++j) g = fmaf(z2[r][j], W2[j * MLP_NH + i], g);
    d1[r][i] = h1[r][i] > 0.f ? g : 0.f;
  }
  __syncthreads();
  for (int k = tid; k < MLP_NH * MLP_NF; k += blockDim.x) {
    const int j = k / MLP_NF, i = k % MLP_NF;
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g = fmaf(d1[r][j], xs[r][i], g);
    atomicAdd(gW1 + k, g);
  }
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int r = 0; r < TB; ++r) g += d1[r][tid];
    atomicAdd(gb1 + tid, g);
  }
}

__global__ void adam_kernel(float* w, float* m, float* v, const float* g, float lr, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= MLP_NPARAM) return;
  const float gk = g[k];
  const float mk = 0.9f * m[k] + 0.1f * gk;
  const float vk = 0.999f * v[k] + 0.001f * gk * gk;
  m[k] = mk;
  v[k] = vk;
  w[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + 1e-8f);
}

}  // namespace

cudaError_t mlp_sample_features(const MlpSampleArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  feature_kernel<<<(a.n + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t mlp_sample_labels(const MlpSampleArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const long long warps = static_cast<long long>(a.n) * a.chunks;
  label_kernel<<<static_cast<unsigned>((warps * 32 + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* w, const float* X, const float* t, int n_total, int B, int step, uint64_t seed,
                     bool use_all, float* grad, float* loss, cudaStream_t st) {
  grad_kernel<<<(B + TB - 1) / TB, 256, 0, st>>>(w, X, t, n_total, B, step, seed, use_all ? 1 : 0, grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* w, float* m, float* v, const float* g, float lr, int step, cudaStream_t st) {
  const float c1 = 1.f / (1.f - powf(0.9f, static_cast<float>(step)));
  const float c2 = 1.f / (1.f - powf(0.999f, static_cast<float>(step)));
  adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(w, m, v, g, lr, c1, c2);
  return cudaGetLastError();
}

}  // namespace og
