// Microbenchmarks of the FP32 min/max issue rate, the roofline of the median
// selection networks, and of the FP32 add issue rate. Each thread runs kChains independent clamp chains
// x = max(min(x, hi), lo); the values come from memory, so nothing folds.
#pragma once

#include <cuda_runtime.h>

namespace crb {

constexpr int kPeakChains = 16;

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

template <bool kThree>
__global__ void __launch_bounds__(256) alu_peak_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                       int iters) {
  float x[kPeakChains], lo[kPeakChains], hi[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) {
    x[i] = in[(threadIdx.x + i) & 63];
    lo[i] = in[64 + ((threadIdx.x + 3 * i) & 63)];
    hi[i] = in[128 + ((threadIdx.x + 5 * i) & 63)];
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) {
      if (kThree) {
        x[i] = max3f(min3f(x[i], hi[i], hi[(i + 1) % kPeakChains]), lo[i], lo[(i + 1) % kPeakChains]);
      } else {
        x[i] = fmaxf(fminf(x[i], hi[i]), lo[i]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}

// FP32 add issue rate: kPeakChains independent chains x = x + y per thread.
__global__ void __launch_bounds__(256) fadd_peak_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                        int iters) {
  float x[kPeakChains], y[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) {
    x[i] = in[(threadIdx.x + i) & 63];
    y[i] = in[64 + ((threadIdx.x + 3 * i) & 63)];
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = __fadd_rn(x[i], y[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace crb
