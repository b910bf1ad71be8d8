// octgrav_sim.cu -- device side of the time integration: the kick and drift
// updates of a kick-drift-kick leapfrog on FP64 state arrays, and FP64
// energy partial sums. The forces between the kicks come from the tree build
// and the walk kernel. Compiled with -fmad=false so that every update is the
// plain rounded product then sum (the oracle integrator's arithmetic).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "octgrav_internal.h"

namespace og {
namespace {

constexpr int TB = 256;

int grid(int64_t n) { return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + TB - 1) / TB, 152 * 16))); }

// v += a h (h = dt / 2), then, when dt != 0, x += v dt.
__global__ void k_kick_drift(double* __restrict__ x, double* __restrict__ v, const double* __restrict__ a, int64_t n3,
                             double h, double dt, int drift) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n3;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double vi = v[i] + a[i] * h;
    v[i] = vi;
    if (drift) x[i] = x[i] + vi * dt;
  }
}

// Per block: (sum m |v|^2 / 2, sum m phi / 2) over a grid-stride slice, in a
// fixed order (the grid is fixed), so repeated calls give the same bits.
__global__ void __launch_bounds__(TB) k_energy(const double* __restrict__ v, const double* __restrict__ m,
                                               const double* __restrict__ pot, int64_t n,
                                               double* __restrict__ part) {
  double kin = 0, pe = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(TB) + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * TB) {
    const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
    kin += 0.5 * m[i] * ((vx * vx + vy * vy) + vz * vz);
    pe += 0.5 * m[i] * pot[i];
  }
  __shared__ double sk[TB], sp[TB];
  sk[threadIdx.x] = kin;
  sp[threadIdx.x] = pe;
  __syncthreads();
  for (int s = TB / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      sk[threadIdx.x] += sk[threadIdx.x + s];
      sp[threadIdx.x] += sp[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sk[0];
    part[2 * blockIdx.x + 1] = sp[0];
  }
}

}  // namespace

cudaError_t sim_kick_drift(double* x, double* v, const double* a, int64_t n, double h, double dt, bool drift,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_kick_drift<<<grid(3 * n), TB, 0, st>>>(x, v, a, 3 * n, h, dt, drift ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t sim_energy_partials(const double* v, const double* m, const double* pot, int64_t n, double* part,
                                cudaStream_t st) {
  k_energy<<<SIM_EBLOCKS, TB, 0, st>>>(v, m, pot, n, part);
  return cudaGetLastError();
}

}  // namespace og
