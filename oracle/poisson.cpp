// ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// The POISSON work function of CRBLASTER (Mighell, PASP 2010, Sec. 6.3.2): each
// output pixel is a Poisson deviate whose mean is the input pixel, drawn with
// Knuth's multiplicative method (Algorithm Q; Knuth, Seminumerical
// Algorithms, Sec. 3.4.1): multiply uniform deviates until the product falls
// below e^-mu; the number of factors before that is the deviate. A plain,
// slow, pixel-by-pixel restatement. Only the test suite and the benchmark's
// CPU legs may load it; the CUDA library never does, and the two share no code.
//
// Readings (the paper prints its generator only as a figure that is not
// available):
//   - the uniforms come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014;
//     golden gamma 0x9e3779b97f4a7c15 and Stafford's Mix13 finaliser), used as
//     a counter-based generator: value(s, j) = mix(s + (j + 1) * gamma). Pixel
//     p (row-major index in its frame) of a frame with seed s draws from the
//     stream keyed by value(s, p); its j-th uniform is the top 53 bits of
//     value(key, j) times 2^-53, in [0, 1);
//   - mu <= 0 (and NaN) give 0; mu above 700 is taken as 700, where e^-mu is
//     still a normal double; at most 4096 factors are drawn (Poisson(700)
//     never comes near that);
//   - e^-mu is computed by the one procedure below in IEEE double (no fused
//     operations): Cody and Waite's reduction -mu = n ln2 + r, then the Taylor
//     polynomial of e^r to degree 13 by Horner's rule, then scaling by 2^n.
//     Any kernel that follows the same steps takes every decision q >= e^-mu
//     identically.
// Parity status: the uniform stream against published SplitMix64 outputs, the
// generator's statistics (mean, variance, the distribution against the Poisson
// pmf) and Algorithm Q on given uniforms are pinned by the tests; that the
// paper's own generator drew the same uniforms is not (parity unpinned against
// the paper for the choice of uniform generator).

#include <cmath>
#include <cstdint>
#include <cstring>

namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;
constexpr double kMuMax = 700.0;
constexpr int kQMax = 4096;

uint64_t mix13(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// The j-th value of the counter-based stream with key s.
uint64_t stream_value(uint64_t s, uint64_t j) { return mix13(s + (j + 1) * kGamma); }

double uniform53(uint64_t v) { return double(v >> 11) * 0x1.0p-53; }

// e^-mu for 0 <= mu <= 700, by fixed IEEE double steps.
double exp_neg(double mu) {
  const double ln2 = 0.693147180559945309417232121458;  // rounded to double
  // high part of ln2 with its low 20 significand bits cleared: n * ln2_hi is
  // exact for |n| < 2^20
  uint64_t bits;
  double ln2_hi;
  static_assert(sizeof(bits) == sizeof(ln2_hi), "double is 64-bit");
  std::memcpy(&bits, &ln2, 8);
  bits &= ~((uint64_t(1) << 20) - 1);
  std::memcpy(&ln2_hi, &bits, 8);
  const double ln2_lo = ln2 - ln2_hi;
  const double inv_ln2 = 1.0 / ln2;
  const double x = -mu;
  const double n = std::nearbyint(x * inv_ln2);
  const double r = (x - n * ln2_hi) - n * ln2_lo;
  double c[14];
  c[0] = 1.0;
  for (int i = 1; i < 14; ++i) c[i] = c[i - 1] / double(i);
  double p = c[13];
  for (int i = 12; i >= 0; --i) p = p * r + c[i];
  return std::ldexp(p, int(n));
}

// Algorithm Q on the uniforms u(0), u(1), ...: the number of factors the
// product takes while it stays >= e^-mu.
template <typename U>
int algorithm_q(double mu, U&& u) {
  if (!(mu > 0.0)) return 0;
  if (mu > kMuMax) mu = kMuMax;
  const double L = exp_neg(mu);
  double q = u(0);
  int k = 0;
  while (q >= L && k < kQMax) {
    ++k;
    q = q * u(k);
  }
  return k;
}

}  // namespace

extern "C" {

double oracle_exp_neg(double mu) { return exp_neg(mu); }

uint64_t oracle_stream_value(uint64_t s, uint64_t j) { return stream_value(s, j); }

// Algorithm Q on n given uniforms (u[j] for the j-th factor); -1 if it needs more.
int oracle_algorithm_q(double mu, const double* u, int n) {
  bool over = false;
  const int k = algorithm_q(mu, [&](int j) {
    if (j >= n) {
      over = true;
      return 0.0;
    }
    return u[j];
  });
  return over ? -1 : k;
}

// The POISSON work function on one frame: out[p] = deviate of mean in[p].
int oracle_poisson(const float* in, int w, int h, uint64_t seed, float* out) {
  if (!in || !out || w < 1 || h < 1) return 1;
  const long long n = (long long)w * h;
#pragma omp parallel for schedule(static)
  for (long long p = 0; p < n; ++p) {
    const uint64_t key = stream_value(seed, uint64_t(p));
    out[p] = float(algorithm_q(double(in[p]), [&](int j) { return uniform53(stream_value(key, uint64_t(j))); }));
  }
  return 0;
}

}  // extern "C"
