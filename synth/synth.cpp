// Seeded synthetic CCD frames for the cosmic-ray cleaner.
//
// This module only makes inputs. It holds none of the cleaning arithmetic and
// is shared by the CUDA path's tests/bench and by the CPU oracle's tests, so
// that both read identical bytes.
//
// Generative model (electrons, then divided by the gain to give DN):
//   pixel = Poisson(sky + sum of stars) + cosmic-ray deposits + Normal(0, rn)
// * Stars: pixel-integrated circular Gaussians (differences of erf), FWHM
//   uniform in [1.5, 2.5] px, total flux log-uniform in [1e3, 1e6] e-, centres
//   continuous-uniform over the frame.
// * Cosmic rays: start uniform over the frame, angle uniform in [0, pi); 20 %
//   hit one pixel, the rest are straight tracks of length uniform in [1, 10] px
//   sampled every 0.25 px; every touched pixel receives the track amplitude
//   once; amplitude log-uniform in [1e2, 1e4] e- per pixel. The pixels touched
//   are returned as a truth mask (for recall/precision only).
//
// Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
// splitmix64; one independent stream per (seed, frame, purpose, index).
// Gaussians by Box-Muller; Poisson deviates by inversion for mean < 10 and by
// Hoermann's PTRS transformed rejection (Hoermann 1993) for mean >= 10.
// Rows of the Poisson/noise pass use their own streams, so the result does not
// depend on the number of threads.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

inline uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

struct Rng {
  uint64_t s[4];

  Rng(uint64_t seed, uint64_t frame, uint64_t purpose, uint64_t index) {
    uint64_t x = seed;
    uint64_t k = splitmix64(x) ^ (frame * 0xd1b54a32d192ed03ULL);
    x = k;
    k = splitmix64(x) ^ (purpose * 0x8cb92ba72f3d8dd7ULL);
    x = k;
    k = splitmix64(x) ^ (index * 0xaef17502108ef2d9ULL);
    x = k;
    for (auto& w : s) w = splitmix64(x);
  }

  uint64_t next() {  // xoshiro256**
    const uint64_t r = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
  }

  // uniform in [0, 1) with 53 random bits
  double uniform() { return double(next() >> 11) * 0x1.0p-53; }

  double gauss() {  // Box-Muller, one deviate per call
    const double u1 = 1.0 - uniform();  // (0, 1]
    const double u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }

  long poisson(double mu) {
    if (!(mu > 0.0)) return 0;
    if (mu < 10.0) {  // inversion by sequential search
      double p = std::exp(-mu), cdf = p;
      const double u = uniform();
      long k = 0;
      while (u > cdf && k < 1000) {
        ++k;
        p *= mu / double(k);
        cdf += p;
      }
      return k;
    }
    // PTRS (Hoermann 1993), transformed rejection with squeeze
    const double smu = std::sqrt(mu), lmu = std::log(mu);
    const double b = 0.931 + 2.53 * smu;
    const double a = -0.059 + 0.02483 * b;
    const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    const double v_r = 0.9277 - 3.6224 / (b - 2.0);
    for (;;) {
      const double u = uniform() - 0.5;
      const double v = uniform();
      const double us = 0.5 - std::fabs(u);
      const double k = std::floor((2.0 * a / us + b) * u + mu + 0.43);
      if (us >= 0.07 && v <= v_r) return long(k);
      if (k < 0.0 || (us < 0.013 && v > us)) continue;
      if (std::log(v) + std::log(inv_alpha) - std::log(a / (us * us) + b) <=
          -mu + k * lmu - std::lgamma(k + 1.0))
        return long(k);
    }
  }
};

enum : uint64_t { kStars = 1, kRows = 2, kCosmics = 3 };

}  // namespace

extern "C" {

// Fills out_dn[h*w] (row-major, DN) and, if out_truth is not null, the
// cosmic-ray truth mask out_truth[h*w] (1 where a track deposited charge).
// Returns 0, or -1 on invalid sizes.
int synth_frame(int w, int h, uint64_t seed, int frame, double sky_e, double gain,
                double readnoise, int nstars, int ncr, float* out_dn, uint8_t* out_truth) {
  if (w <= 0 || h <= 0 || !(gain > 0.0) || out_dn == nullptr) return -1;
  const size_t npix = size_t(w) * size_t(h);

  // 1. expected electrons: flat sky plus pixel-integrated Gaussian stars
  std::vector<float> lam(npix, float(sky_e));
  {
    Rng rng(seed, uint64_t(frame), kStars, 0);
    std::vector<double> fx, fy;
    for (int i = 0; i < nstars; ++i) {
      const double xc = rng.uniform() * w;
      const double yc = rng.uniform() * h;
      const double fwhm = 1.5 + rng.uniform();
      const double flux = std::pow(10.0, 3.0 + 3.0 * rng.uniform());
      const double sigma = fwhm / 2.3548200450309493;
      const double k = 1.0 / (std::sqrt(2.0) * sigma);
      const int rad = int(std::ceil(6.0 * sigma)) + 1;
      const int x0 = std::max(0, int(std::floor(xc)) - rad), x1 = std::min(w - 1, int(std::floor(xc)) + rad);
      const int y0 = std::max(0, int(std::floor(yc)) - rad), y1 = std::min(h - 1, int(std::floor(yc)) + rad);
      if (x0 > x1 || y0 > y1) continue;
      fx.assign(size_t(x1 - x0 + 1), 0.0);
      fy.assign(size_t(y1 - y0 + 1), 0.0);
      for (int x = x0; x <= x1; ++x)  // pixel x spans [x, x+1)
        fx[size_t(x - x0)] = 0.5 * (std::erf((x + 1 - xc) * k) - std::erf((x - xc) * k));
      for (int y = y0; y <= y1; ++y)
        fy[size_t(y - y0)] = 0.5 * (std::erf((y + 1 - yc) * k) - std::erf((y - yc) * k));
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x)
          lam[size_t(y) * w + x] += float(flux * fy[size_t(y - y0)] * fx[size_t(x - x0)]);
    }
  }

  // 2. Poisson photon noise plus Gaussian read noise, one stream per row
  std::vector<float> e(npix);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < h; ++y) {
    Rng rng(seed, uint64_t(frame), kRows, uint64_t(y));
    for (int x = 0; x < w; ++x) {
      const size_t i = size_t(y) * w + x;
      e[i] = float(double(rng.poisson(double(lam[i]))) + readnoise * rng.gauss());
    }
  }
  std::vector<float>().swap(lam);

  // 3. cosmic-ray tracks, deposited without photon noise
  if (out_truth) std::memset(out_truth, 0, npix);
  {
    Rng rng(seed, uint64_t(frame), kCosmics, 0);
    std::vector<std::pair<int, int>> hit;
    for (int i = 0; i < ncr; ++i) {
      const double xs = rng.uniform() * w;
      const double ys = rng.uniform() * h;
      const double theta = rng.uniform() * 3.141592653589793;
      const bool single = rng.uniform() < 0.2;
      const double len = 1.0 + 9.0 * rng.uniform();
      const double amp = std::pow(10.0, 2.0 + 2.0 * rng.uniform());
      hit.clear();
      const int nsamp = single ? 1 : int(std::floor(len / 0.25)) + 1;
      const double c = std::cos(theta), s = std::sin(theta);
      for (int t = 0; t < nsamp; ++t) {
        const int px = int(std::floor(xs + 0.25 * t * c));
        const int py = int(std::floor(ys + 0.25 * t * s));
        if (px < 0 || px >= w || py < 0 || py >= h) continue;
        const std::pair<int, int> q(px, py);
        if (std::find(hit.begin(), hit.end(), q) == hit.end()) hit.push_back(q);
      }
      for (const auto& q : hit) {
        const size_t j = size_t(q.second) * w + q.first;
        e[j] += float(amp);
        if (out_truth) out_truth[j] = 1;
      }
    }
  }

  // 4. electrons -> DN
  const double inv_gain = 1.0 / gain;
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < (long long)npix; ++i) out_dn[i] = float(double(e[size_t(i)]) * inv_gain);
  return 0;
}

}  // extern "C"
