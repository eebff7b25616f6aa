// The POISSON work function (declarations and contract in include/crb.h).
//
// CRBLASTER measures the cost of its own framework by swapping L.A.Cosmic for
// a work function with an equal, known load per pixel and no overlap regions
// (Sec. 6.3.2): each output pixel is a Poisson deviate whose mean is the input
// pixel, drawn with Knuth's multiplicative method (Algorithm Q, Seminumerical
// Algorithms Sec. 3.4.1): uniforms are multiplied until the product falls
// below e^-mu, and the number of factors taken before that is the deviate.
// Its cost grows linearly with mu.
//
// One thread per pixel over all frames of a call. The uniforms come from
// SplitMix64 (Steele, Lea and Flood 2014) used as a counter-based generator,
// so a pixel's draws depend only on its frame's seed, its index and the draw
// number: value(s, j) = mix13(s + (j + 1) * gamma); pixel p draws from the
// stream keyed by value(seed, p), its j-th uniform being the top 53 bits of
// value(key, j) times 2^-53. e^-mu is formed by fixed IEEE double steps
// (Cody-Waite reduction -mu = n ln2 + r, the Taylor polynomial of e^r to
// degree 13 by Horner's rule, scaling by 2^n), with the rounded operations
// spelled out so that no multiply-add is fused; the comparisons q >= e^-mu are
// therefore those of any implementation that takes the same steps. mu <= 0 or
// NaN gives 0, mu above 700 is taken as 700, and at most 4096 factors are
// drawn, which bounds every thread's loop.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>

#include "crb.h"

void crb_detail_set_error(const char* msg);  // crb.cu

namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;
constexpr double kMuMax = 700.0;
constexpr int kQMax = 4096;
constexpr int kFramesPerLaunch = 256;  // the frame table travels in the launch parameters

struct PFrame {
  const float* in;
  float* out;
  long long pix0;  // first pixel of the frame in the launch's pixel index
  uint64_t seed;
};

struct PLaunch {
  PFrame f[kFramesPerLaunch];
  int n;
  long long total;
  double c[14];  // 1/i!
  double ln2_hi, ln2_lo, inv_ln2;
};

__device__ __forceinline__ uint64_t mix13(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t stream_value(uint64_t s, uint64_t j) { return mix13(s + (j + 1) * kGamma); }

// (v >> 11) * 2^-53, built from its bits with integer operations (the value
// is exact either way): the FP64 pipe is left to the product.
__device__ __forceinline__ double uniform53(uint64_t v) {
  const uint64_t m = v >> 11;
  if (m == 0) return 0.0;
  const int e = 63 - __clzll((long long)m);  // top bit of m, 0 .. 52
  const uint64_t frac = (m << (52 - e)) & ((uint64_t(1) << 52) - 1);
  return __longlong_as_double((long long)((uint64_t(e - 53 + 1023) << 52) | frac));
}

__device__ __forceinline__ double exp_neg(double mu, const PLaunch& P) {
  const double x = -mu;
  const double n = rint(__dmul_rn(x, P.inv_ln2));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(n, P.ln2_hi)), __dmul_rn(n, P.ln2_lo));
  double p = P.c[13];
#pragma unroll
  for (int i = 12; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, r), P.c[i]);
  return ldexp(p, int(n));
}

__global__ void __launch_bounds__(256) poisson_kernel(const __grid_constant__ PLaunch P) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < P.total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = P.n - 1;  // frame of pixel t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.f[mid].pix0 <= t) lo = mid; else hi = mid - 1;
    }
    const PFrame& f = P.f[lo];
    const long long p = t - f.pix0;
    double mu = double(__ldg(f.in + p));
    int k = 0;
    if (mu > 0.0) {
      mu = fmin(mu, kMuMax);
      // q and e^-mu are non-negative doubles, which order as their bit patterns
      const long long L = __double_as_longlong(exp_neg(mu, P));
      const uint64_t key = stream_value(f.seed, uint64_t(p));
      uint64_t ctr = key + kGamma;  // key + (j + 1) * gamma for draw j
      double q = uniform53(mix13(ctr));
      while (__double_as_longlong(q) >= L && k < kQMax) {
        ++k;
        ctr += kGamma;
        q = __dmul_rn(q, uniform53(mix13(ctr)));
      }
    }
    f.out[p] = float(k);
  }
}

int fail(int code, const std::string& msg) {
  crb_detail_set_error(msg.c_str());
  return code;
}

// The constants of exp_neg, by the same steps on the host: ln2 rounded to
// double, its high part with the low 20 significand bits cleared (n * ln2_hi is
// exact for |n| < 2^20), the remainder, and 1/i! by repeated division.
void fill_constants(PLaunch& P) {
  const double ln2 = 0.693147180559945309417232121458;
  uint64_t bits;
  std::memcpy(&bits, &ln2, 8);
  bits &= ~((uint64_t(1) << 20) - 1);
  std::memcpy(&P.ln2_hi, &bits, 8);
  P.ln2_lo = ln2 - P.ln2_hi;
  P.inv_ln2 = 1.0 / ln2;
  P.c[0] = 1.0;
  for (int i = 1; i < 14; ++i) P.c[i] = P.c[i - 1] / double(i);
}

int launch(PLaunch& P, cudaStream_t stream) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return fail(CRB_ECUDA, "crb_poisson: no CUDA device");
  }
  const long long blocks = std::min<long long>((P.total + 255) / 256, (long long)sms * 8);
  poisson_kernel<<<int(std::max<long long>(blocks, 1)), 256, 0, stream>>>(P);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CRB_ECUDA, std::string("crb_poisson launch: ") + cudaGetErrorString(e));
  return CRB_OK;
}

}  // namespace

extern "C" int crb_poisson_batch(int n, const float* const* imgs, const int* ws, const int* hs, const uint64_t* seeds,
                                 float* const* outs, cudaStream_t stream) {
  if (n < 0 || (n > 0 && (!imgs || !ws || !hs || !seeds || !outs)))
    return fail(CRB_EINVAL, "crb_poisson_batch: invalid batch arrays");
  for (int i = 0; i < n; ++i) {
    if (ws[i] < 1 || hs[i] < 1 || (long long)ws[i] * hs[i] >= (1LL << 31))
      return fail(CRB_EINVAL, "crb_poisson_batch: frame " + std::to_string(i) + ": sizes");
    if (!imgs[i] || !outs[i]) return fail(CRB_EINVAL, "crb_poisson_batch: frame " + std::to_string(i) + ": null");
  }
  PLaunch P;  // about 8 KB, passed by value in the launch parameters
  for (int a = 0; a < n; a += kFramesPerLaunch) {
    const int m = std::min(kFramesPerLaunch, n - a);
    fill_constants(P);
    P.n = m;
    P.total = 0;
    for (int i = 0; i < m; ++i) {
      const long long px = (long long)ws[a + i] * hs[a + i];
      P.f[i] = PFrame{imgs[a + i], outs[a + i], P.total, seeds[a + i]};
      P.total += px;
    }
    const int rc = launch(P, stream);
    if (rc) return rc;
  }
  return CRB_OK;
}

extern "C" int crb_poisson(const float* img, int w, int h, uint64_t seed, float* out, cudaStream_t stream) {
  if (!img || !out) return fail(CRB_EINVAL, "crb_poisson: null image or output pointer");
  const float* const imgs[1] = {img};
  float* const outs[1] = {out};
  return crb_poisson_batch(1, imgs, &w, &h, &seed, outs, stream);
}
