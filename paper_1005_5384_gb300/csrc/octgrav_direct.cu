// octgrav_direct.cu -- direct Plummer-softened summation in FP64 on the GPU for
// a set of target particles: the exact reference of the error measurements
// Delta a / a = |a_tree - a_direct| / |a_direct| (Sec. 3.1, where the direct
// sums also ran on the GPU). O(n * targets) work; every source tile is staged
// in shared memory and reused by a block of 256 targets; the sources are cut
// into fixed chunks whose partial sums are added in chunk order, so results
// do not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "octgrav_internal.h"

namespace og {
namespace {

constexpr int TB = 256;

__global__ void __launch_bounds__(TB) k_direct(const double* __restrict__ pos, const double* __restrict__ mass,
                                               int64_t n, const int64_t* __restrict__ targets, int64_t nt,
                                               double eps2, int64_t chunk, double* __restrict__ part) {
  __shared__ double sx[TB], sy[TB], sz[TB], sm[TB];
  const int64_t t = blockIdx.x * static_cast<int64_t>(TB) + threadIdx.x;
  const bool live = t < nt;
  const int64_t ti = live ? (targets ? targets[t] : t) : -1;
  const double xi = live ? pos[3 * ti] : 0, yi = live ? pos[3 * ti + 1] : 0, zi = live ? pos[3 * ti + 2] : 0;
  double ax = 0, ay = 0, az = 0, ph = 0;
  const int64_t j0 = blockIdx.y * chunk, j1 = min(n, j0 + chunk);
  for (int64_t base = j0; base < j1; base += TB) {
    const int64_t j = base + threadIdx.x;
    __syncthreads();
    if (j < j1) {
      sx[threadIdx.x] = pos[3 * j];
      sy[threadIdx.x] = pos[3 * j + 1];
      sz[threadIdx.x] = pos[3 * j + 2];
      sm[threadIdx.x] = mass[j];
    }
    __syncthreads();
    const int m = static_cast<int>(min(static_cast<int64_t>(TB), j1 - base));
    for (int k = 0; k < m; ++k) {
      if (base + k == ti) continue;  // self term excluded
      const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
      const double r2 = ((dx * dx + dy * dy) + dz * dz) + eps2;
      const double ri = rsqrt(r2);
      const double mr = sm[k] * ri;
      const double mr3 = mr * ri * ri;
      ax += mr3 * dx;
      ay += mr3 * dy;
      az += mr3 * dz;
      ph -= mr;
    }
  }
  if (live) {
    double* p = &part[4 * (blockIdx.y * nt + t)];
    p[0] = ax;
    p[1] = ay;
    p[2] = az;
    p[3] = ph;
  }
}

__global__ void k_direct_sum(const double* __restrict__ part, int64_t nt, int nchunks, double G,
                             double* __restrict__ acc, double* __restrict__ pot) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= nt) return;
  double s[4] = {0, 0, 0, 0};
  for (int c = 0; c < nchunks; ++c)
    for (int k = 0; k < 4; ++k) s[k] += part[4 * (c * nt + t) + k];
  acc[3 * t] = G * s[0];
  acc[3 * t + 1] = G * s[1];
  acc[3 * t + 2] = G * s[2];
  pot[t] = G * s[3];
}

}  // namespace

int64_t direct_chunks(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>(64, (n + 16383) / 16384)); }

cudaError_t direct_sum(const double* pos, const double* mass, int64_t n, const int64_t* targets, int64_t nt,
                       double eps, double G, double* part, double* acc, double* pot, cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  const int64_t nch = direct_chunks(n);
  const int64_t chunk = (n + nch - 1) / nch;
  dim3 grid(static_cast<unsigned>((nt + TB - 1) / TB), static_cast<unsigned>(nch));
  k_direct<<<grid, TB, 0, st>>>(pos, mass, n, targets, nt, eps * eps, chunk, part);
  k_direct_sum<<<static_cast<unsigned>((nt + 255) / 256), 256, 0, st>>>(part, nt, static_cast<int>(nch), G, acc, pot);
  return cudaGetLastError();
}

}  // namespace og
