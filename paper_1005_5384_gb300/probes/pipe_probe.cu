// pipe_probe.cu -- throughput of the arithmetic pipes the library leans on,
// measured on the current GPU: FP32 FMA (scalar and packed FFMA2, with the
// operand patterns of the evaluation kernel), MUFU rsqrt, and FP64 (the tree
// build). Prints one JSON line per case: lane operations per clock per SM at
// the device's maximum SM clock. Built and run by `bench.py --leg pipes`.
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int ITERS = 2048;

__device__ __forceinline__ float rsq(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// FP32 cases; every loop iteration does OPS lane operations per thread.
template <int MODE>
__global__ void k32(float* out, float a, float b) {
  float2 x[8], y[8], acc[8];
  for (int i = 0; i < 8; i++) {
    x[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
    y[i] = make_float2(1.0f - i * 1e-3f, 0.999f + i * 1e-4f);
    acc[i] = make_float2(0.f, 0.f);
  }
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int it = 0; it < ITERS; ++it) {
    if (MODE == 0) {  // scalar FFMA, operands repeat
      float* s = reinterpret_cast<float*>(x);
#pragma unroll
      for (int i = 0; i < 16; i++) s[i] = fmaf(s[i], a, b);
#pragma unroll
      for (int i = 0; i < 16; i++) s[i] = fmaf(s[i], a, b);
    } else if (MODE == 1) {  // FFMA2, one operand repeats
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = __ffma2_rn(x[i], A, acc[i]);
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ffma2_rn(acc[i], A, x[i]);
    } else if (MODE == 2) {  // FFMA2, three distinct register pairs
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = __ffma2_rn(x[i], y[i], acc[i]);
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ffma2_rn(y[i], acc[i], x[i]);
    } else if (MODE == 3) {  // scalar FFMA, three distinct registers
      float* xs = reinterpret_cast<float*>(x);
      float* ys = reinterpret_cast<float*>(y);
      float* as = reinterpret_cast<float*>(acc);
#pragma unroll
      for (int i = 0; i < 16; i++) as[i] = fmaf(xs[i], ys[i], as[i]);
#pragma unroll
      for (int i = 0; i < 16; i++) xs[i] = fmaf(ys[i], as[i], xs[i]);
    } else if (MODE == 4) {  // MUFU rsqrt
      float* s = reinterpret_cast<float*>(x);
#pragma unroll
      for (int i = 0; i < 16; i++) s[i] = rsq(s[i]);
#pragma unroll
      for (int i = 0; i < 16; i++) s[i] = rsq(s[i]);
    } else if (MODE == 5) {  // FFMA2 (operand repeats) with one MUFU per 16 FFMA2
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = __ffma2_rn(x[i], A, acc[i]);
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ffma2_rn(acc[i], A, x[i]);
      y[0].x = rsq(y[0].x + B.x);
    } else if (MODE == 6) {  // FFMA2 whose repeated operand is a register pair that changes
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = __ffma2_rn(x[i], y[0], acc[i]);
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ffma2_rn(acc[i], y[1], x[i]);
      y[0] = __ffma2_rn(y[0], y[2], y[3]);
      y[1] = __ffma2_rn(y[1], y[2], y[3]);
    } else if (MODE == 7) {  // FFMA2 with one operand a 32-bit register in both halves
      float* ys = reinterpret_cast<float*>(y);
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = __ffma2_rn(x[i], make_float2(ys[i], ys[i]), acc[i]);
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ffma2_rn(acc[i], make_float2(ys[i + 8], ys[i + 8]), x[i]);
#pragma unroll
      for (int i = 0; i < 16; i++) ys[i] = fmaf(ys[i], a, b);
    }
  }
  float t = 0;
  for (int i = 0; i < 8; i++) t += acc[i].x + acc[i].y + x[i].x + x[i].y + y[i].x;
  if (t == 1234.5f) out[threadIdx.x] = t;
}

template <int MODE>
__global__ void k64(double* out, double a, double b) {
  double s[8];
  for (int i = 0; i < 8; i++) s[i] = threadIdx.x * 1e-3 + i + 1.0;
  for (int it = 0; it < ITERS / 8; ++it) {
    if (MODE == 0) {
#pragma unroll
      for (int i = 0; i < 8; i++) s[i] = fma(s[i], a, b);
    } else if (MODE == 1) {
#pragma unroll
      for (int i = 0; i < 8; i++) s[i] = (i & 1) ? s[i] * a : s[i] + b;
    } else if (MODE == 2) {
#pragma unroll
      for (int i = 0; i < 8; i++) s[i] = b / s[i] + 1.0;
    }
  }
  double t = 0;
  for (int i = 0; i < 8; i++) t += s[i];
  if (t == 1234.5) out[threadIdx.x] = t;
}

template <class K>
void run(const char* name, K kern, bool fp64, double lane_ops_per_iter, double iters, int warps_per_sm) {
  void* o = nullptr;
  cudaMalloc(&o, 8192);
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  const int threads = 256;
  dim3 g(sms * warps_per_sm / 8);
  auto launch = [&]() {
    if (fp64) reinterpret_cast<void (*)(double*, double, double)>(kern)<<<g, threads>>>(static_cast<double*>(o), 0.999, 1e-3);
    else reinterpret_cast<void (*)(float*, float, float)>(kern)<<<g, threads>>>(static_cast<float*>(o), 0.999f, 1e-3f);
  };
  for (int w = 0; w < 2; ++w) launch();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  for (int r = 0; r < 5; r++) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  const double ops = 5.0 * g.x * threads * iters * lane_ops_per_iter;
  printf("{\"case\": \"%s\", \"warps_per_sm\": %d, \"lane_ops_per_clk_per_sm\": %.2f, \"at_mhz\": %d, \"error\": \"%s\"}\n",
         name, warps_per_sm, ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000, cudaGetErrorString(cudaGetLastError()));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(o);
}

}  // namespace

int main() {
  for (int w : {16, 32}) {
    run("fp32 FFMA, operands repeat", reinterpret_cast<void*>(k32<0>), false, 32, ITERS, w);
    run("fp32 FFMA2, one operand repeats", reinterpret_cast<void*>(k32<1>), false, 32, ITERS, w);
    run("fp32 FFMA2, three distinct operand pairs", reinterpret_cast<void*>(k32<2>), false, 32, ITERS, w);
    run("fp32 FFMA, three distinct operands", reinterpret_cast<void*>(k32<3>), false, 32, ITERS, w);
    run("MUFU rsqrt", reinterpret_cast<void*>(k32<4>), false, 32, ITERS, w);
    run("fp32 FFMA2 + 1 MUFU per 16 (FMA lane-ops)", reinterpret_cast<void*>(k32<5>), false, 32, ITERS, w);
    run("fp32 FFMA2, one operand a changing register pair", reinterpret_cast<void*>(k32<6>), false, 36, ITERS, w);
    run("fp32 FFMA2, one operand one register in both halves (+16 FFMA)", reinterpret_cast<void*>(k32<7>), false, 48,
        ITERS, w);
    run("fp64 DFMA", reinterpret_cast<void*>(k64<0>), true, 8, ITERS / 8, w);
    run("fp64 DADD/DMUL", reinterpret_cast<void*>(k64<1>), true, 8, ITERS / 8, w);
    run("fp64 division (+ add)", reinterpret_cast<void*>(k64<2>), true, 8, ITERS / 8, w);
  }
  return 0;
}
