// ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow CPU implementation of one L.A.Cosmic iteration (van Dokkum
// 2001), the work function that CRBLASTER runs on every sub-image (Mighell,
// PASP 2010, Sec. 5 and Sec. 7), repeated niter times. It is written from the
// method's definition, stage by stage, on whole-frame maps, with no tiling,
// fusion or reordering. Only the test suite, the package's smoke check and the
// benchmark's CPU-baseline leg may load it; the CUDA library never does, and
// the two share no code.
//
// Every map is filtered with its own coordinates clamped into the frame
// (replicate edge). The paper leaves the outer pixels undefined (Sec. 6.1), so
// clamping at every stage is this implementation's stated reading.
//
// The arithmetic is templated on the scalar type T:
//   T = double : the reference (the paper's C code works in double, Sec. 6.2);
//   T = float  : the same steps in single precision, in the same order, so
//                that threshold decisions can be compared with an FP32 kernel
//                exactly. Compile with -ffp-contract=off.
// Inputs J are float; every median is an exact selection, so maps that are
// medians of J are exact in either type.
//
// Parity status: medians, L+, the replacement rule, the dependency radius and
// the fragile map are pinned by the tests (brute force, closed forms,
// invariants). The objlim statistic form, the cumulative-mask rule and the tie
// and edge rules are readings of a paper that does not restate the algorithm:
// parity unpinned against the paper for those readings.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
  double gain;       // e- per DN
  double readnoise;  // e-
  double sigclip;    // detection limit for cosmic rays (in sigma)
  double sigfrac;    // fractional detection limit for neighbouring pixels
  double objlim;     // contrast limit between cosmic rays and objects
  int objlim_form;   // 0: script form S'/max(F/N, 0.01); 1: article form 2S/max(F/N, 0.01)
} oracle_params;
}

namespace {

enum MapId { M5 = 0, LPLUS, NOISE, S, SPRIME, M3, F, R, CAND, G1, G2, NMAPS };

template <typename T>
struct Map {
  int w = 0, h = 0;
  std::vector<T> v;
  Map(int w_, int h_) : w(w_), h(h_), v(size_t(w_) * size_t(h_), T(0)) {}
  T& at(int x, int y) { return v[size_t(y) * w + x]; }
  // value with the coordinates clamped into the frame (replicate edge)
  T clamped(int x, int y) const {
    x = std::min(std::max(x, 0), w - 1);
    y = std::min(std::max(y, 0), h - 1);
    return v[size_t(y) * w + x];
  }
};

// Median of the (2r+1)x(2r+1) window around every pixel, coordinates clamped.
// The count is odd, so the median is the unique middle element.
template <typename T>
Map<T> median_filter(const Map<T>& in, int r) {
  Map<T> out(in.w, in.h);
  const int n = (2 * r + 1) * (2 * r + 1);
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < in.h; ++y) {
    std::vector<T> win(static_cast<size_t>(n));
    for (int x = 0; x < in.w; ++x) {
      int k = 0;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) win[size_t(k++)] = in.clamped(x + dx, y + dy);
      std::nth_element(win.begin(), win.begin() + n / 2, win.end());
      out.v[size_t(y) * in.w + x] = win[size_t(n / 2)];
    }
  }
  return out;
}

// Stage (a): L+ = Laplacian of the 2x block-replicated image with negatives set
// to zero, averaged back over each 2x2 block. On the original grid the four
// sub-pixels of p give
//   L+(p) = 1/4 [max(0,dN+dW) + max(0,dN+dE) + max(0,dS+dW) + max(0,dS+dE)],
// dX = J(p) - J(neighbour X) with the neighbour clamped into the frame.
template <typename T>
Map<T> lplus(const Map<T>& J) {
  Map<T> out(J.w, J.h);
  const T zero = T(0), quarter = T(0.25);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < J.h; ++y)
    for (int x = 0; x < J.w; ++x) {
      const T c = J.clamped(x, y);
      const T dn = c - J.clamped(x, y - 1);
      const T ds = c - J.clamped(x, y + 1);
      const T dw = c - J.clamped(x - 1, y);
      const T de = c - J.clamped(x + 1, y);
      T acc = std::max(zero, dn + dw);
      acc = acc + std::max(zero, dn + de);
      acc = acc + std::max(zero, ds + dw);
      acc = acc + std::max(zero, ds + de);
      out.v[size_t(y) * J.w + x] = quarter * acc;
    }
  return out;
}

// 3x3 dilation of a 0/1 map (out-of-frame neighbours add nothing; clamping
// them would only repeat pixels already in the window).
Map<uint8_t> dilate3(const Map<uint8_t>& in) {
  Map<uint8_t> out(in.w, in.h);
  for (int y = 0; y < in.h; ++y)
    for (int x = 0; x < in.w; ++x) {
      uint8_t any = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) any |= in.clamped(x + dx, y + dy);
      out.v[size_t(y) * in.w + x] = any ? 1 : 0;
    }
  return out;
}

// Stage (e): every flagged pixel takes the lower median (sorted element
// ceil(n/2)-1) of the n values J(q), q in its clamped 5x5 window, q unflagged;
// clamped duplicates count. With n = 0 it takes m5(p). Unflagged pixels keep J.
template <typename T>
long long replace(const Map<T>& J, const Map<uint8_t>& Mk, const Map<T>& m5, Map<T>& out) {
  long long none_left = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : none_left)
  for (int y = 0; y < J.h; ++y) {
    std::vector<T> vals;
    vals.reserve(25);
    for (int x = 0; x < J.w; ++x) {
      const size_t i = size_t(y) * J.w + x;
      if (!Mk.v[i]) {
        out.v[i] = J.v[i];
        continue;
      }
      vals.clear();
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx)
          if (!Mk.clamped(x + dx, y + dy)) vals.push_back(J.clamped(x + dx, y + dy));
      const size_t n = vals.size();
      if (n == 0) {
        out.v[i] = m5.v[i];
        ++none_left;
        continue;
      }
      const size_t k = (n + 1) / 2 - 1;
      std::nth_element(vals.begin(), vals.begin() + long(k), vals.end());
      out.v[i] = vals[k];
    }
  }
  return none_left;
}

template <typename T>
struct IterOut {
  std::vector<float> Ik;
  std::vector<uint8_t> Mk;
  std::vector<Map<T>> maps;
  std::vector<uint8_t> fragile;
  long long n_new = 0, n_none_left = 0;
};

// One L.A.Cosmic iteration on J = I_{k-1} with cumulative flags M_{k-1}.
template <typename T>
void iterate(const float* Jf, const uint8_t* Mprev, int w, int h, const oracle_params& p,
             IterOut<T>& o, bool keep_maps, bool want_fragile) {
  const T gain = T(p.gain), rn = T(p.readnoise), sigclip = T(p.sigclip);
  const T sigfrac = T(p.sigfrac), objlim = T(p.objlim);
  Map<T> J(w, h);
  for (size_t i = 0; i < J.v.size(); ++i) J.v[i] = T(Jf[i]);

  // Stage (b): noise model from the 5x5 median, floored before the square root.
  Map<T> m5 = median_filter(J, 2);
  for (auto& v : m5.v)
    if (v <= T(0)) v = T(0.0001);
  Map<T> noise(w, h);
  const T rn2 = rn * rn;
  for (size_t i = 0; i < noise.v.size(); ++i) noise.v[i] = std::sqrt(gain * m5.v[i] + rn2) / gain;

  // Stage (a) and the significance S = L+ / (2N), S' = S - med5(S).
  Map<T> lp = lplus(J);
  Map<T> s(w, h);
  for (size_t i = 0; i < s.v.size(); ++i) s.v[i] = lp.v[i] / (T(2) * noise.v[i]);
  Map<T> s_med = median_filter(s, 2);
  Map<T> sp(w, h);
  for (size_t i = 0; i < sp.v.size(); ++i) sp.v[i] = s.v[i] - s_med.v[i];

  // Stage (c): fine structure F = med3(J) - med7(med3(J)), and the objlim
  // statistic with the normalised fine structure floored at 0.01.
  Map<T> m3 = median_filter(J, 1);
  Map<T> m37 = median_filter(m3, 3);
  Map<T> f(w, h), r(w, h);
  for (size_t i = 0; i < f.v.size(); ++i) {
    f.v[i] = m3.v[i] - m37.v[i];
    const T fn = std::max(f.v[i] / noise.v[i], T(0.01));
    r.v[i] = (p.objlim_form == 1) ? (T(2) * s.v[i]) / fn : sp.v[i] / fn;
  }

  // Stage (d): candidates, then two 3x3 growth steps at sigclip and at
  // sigfrac*sigclip; all comparisons strict.
  const T sigcliplow = sigfrac * sigclip;
  Map<uint8_t> cand(w, h);
  for (size_t i = 0; i < cand.v.size(); ++i) cand.v[i] = (sp.v[i] > sigclip && r.v[i] > objlim) ? 1 : 0;
  Map<uint8_t> g1 = dilate3(cand);
  for (size_t i = 0; i < g1.v.size(); ++i) g1.v[i] = (g1.v[i] && sp.v[i] > sigclip) ? 1 : 0;
  Map<uint8_t> g2 = dilate3(g1);
  for (size_t i = 0; i < g2.v.size(); ++i) g2.v[i] = (g2.v[i] && sp.v[i] > sigcliplow) ? 1 : 0;

  // Cumulative flags M_k = M_{k-1} | g2.
  Map<uint8_t> Mk(w, h);
  o.n_new = 0;
  for (size_t i = 0; i < Mk.v.size(); ++i) {
    const uint8_t prev = Mprev ? (Mprev[i] ? 1 : 0) : 0;
    Mk.v[i] = prev | g2.v[i];
    o.n_new += (g2.v[i] && !prev) ? 1 : 0;
  }

  // Stage (e): replacement with the cumulative flags.
  Map<T> Ik(w, h);
  o.n_none_left = replace(J, Mk, m5, Ik);
  o.Ik.resize(Ik.v.size());
  for (size_t i = 0; i < Ik.v.size(); ++i) o.Ik[i] = float(Ik.v[i]);
  o.Mk = Mk.v;

  if (want_fragile) {
    // A statistic within 1e-4 (relative) of the threshold it is compared with
    // marks the 5x5 growth cone around it as fragile.
    const double tol = 1e-4;
    const double c = double(sigclip), c2 = double(sigcliplow), ol = double(objlim);
    Map<uint8_t> near(w, h);
    for (size_t i = 0; i < near.v.size(); ++i) {
      const double spv = double(sp.v[i]), rv = double(r.v[i]);
      const bool a = std::fabs(spv - c) <= tol * c;
      const bool b = std::fabs(spv - c2) <= tol * c2;
      const bool d = spv > c * (1.0 - tol) && std::fabs(rv - ol) <= tol * ol;
      near.v[i] = (a || b || d) ? 1 : 0;
    }
    o.fragile.assign(near.v.size(), 0);
    for (int y = 0; y < h; ++y)
      for (int x = 0; x < w; ++x) {
        uint8_t any = 0;
        for (int dy = -2; dy <= 2; ++dy)
          for (int dx = -2; dx <= 2; ++dx) any |= near.clamped(x + dx, y + dy);
        o.fragile[size_t(y) * w + x] = any;
      }
  }

  if (keep_maps) {
    o.maps.clear();
    o.maps.reserve(NMAPS);
    o.maps.push_back(m5);
    o.maps.push_back(lp);
    o.maps.push_back(noise);
    o.maps.push_back(s);
    o.maps.push_back(sp);
    o.maps.push_back(m3);
    o.maps.push_back(f);
    o.maps.push_back(r);
    Map<T> mc(w, h), m1(w, h), m2(w, h);
    for (size_t i = 0; i < mc.v.size(); ++i) {
      mc.v[i] = T(cand.v[i]);
      m1.v[i] = T(g1.v[i]);
      m2.v[i] = T(g2.v[i]);
    }
    o.maps.push_back(mc);
    o.maps.push_back(m1);
    o.maps.push_back(m2);
  }
}

bool valid(int w, int h, const oracle_params* p) {
  return w > 0 && h > 0 && p && p->gain > 0 && p->readnoise >= 0 && p->sigclip > 0 &&
         p->sigfrac > 0 && p->objlim > 0;
}

template <typename T>
int iter_entry(const float* J, const uint8_t* Mprev, int w, int h, const oracle_params* p, float* Ik,
               uint8_t* Mk, T* maps, uint8_t* fragile, long long* counts) {
  if (!valid(w, h, p) || !J || !Ik || !Mk) return -1;
  IterOut<T> o;
  iterate<T>(J, Mprev, w, h, *p, o, maps != nullptr, fragile != nullptr);
  const size_t n = size_t(w) * size_t(h);
  std::memcpy(Ik, o.Ik.data(), n * sizeof(float));
  std::memcpy(Mk, o.Mk.data(), n);
  if (maps)
    for (int m = 0; m < NMAPS; ++m) std::memcpy(maps + size_t(m) * n, o.maps[size_t(m)].v.data(), n * sizeof(T));
  if (fragile) std::memcpy(fragile, o.fragile.data(), n);
  if (counts) {
    counts[0] = o.n_new;
    counts[1] = o.n_none_left;
  }
  return 0;
}

template <typename T>
int clean_entry(const float* I0, int w, int h, const oracle_params* p, int niter, float* out_clean,
                uint8_t* out_mask, long long* counts, uint8_t* fragile_any) {
  if (!valid(w, h, p) || niter < 0 || !I0 || !out_clean || !out_mask) return -1;
  const size_t n = size_t(w) * size_t(h);
  std::vector<float> J(I0, I0 + n);
  std::vector<uint8_t> M(n, 0);
  if (fragile_any) std::memset(fragile_any, 0, n);
  for (int k = 0; k < niter; ++k) {
    IterOut<T> o;
    iterate<T>(J.data(), M.data(), w, h, *p, o, false, fragile_any != nullptr);
    J.swap(o.Ik);
    M.swap(o.Mk);
    if (counts) {
      counts[2 * k] = o.n_new;
      counts[2 * k + 1] = o.n_none_left;
    }
    if (fragile_any)
      for (size_t i = 0; i < n; ++i) fragile_any[i] |= o.fragile[i];
  }
  std::memcpy(out_clean, J.data(), n * sizeof(float));
  std::memcpy(out_mask, M.data(), n);
  return 0;
}

template <typename T>
int replace_entry(const float* Jf, const uint8_t* Mk, int w, int h, float* out, long long* none_left) {
  if (w <= 0 || h <= 0 || !Jf || !Mk || !out) return -1;
  Map<T> J(w, h);
  for (size_t i = 0; i < J.v.size(); ++i) J.v[i] = T(Jf[i]);
  Map<T> m5 = median_filter(J, 2);
  for (auto& v : m5.v)
    if (v <= T(0)) v = T(0.0001);
  Map<uint8_t> M(w, h);
  for (size_t i = 0; i < M.v.size(); ++i) M.v[i] = Mk[i] ? 1 : 0;
  Map<T> o(w, h);
  const long long c = replace(J, M, m5, o);
  for (size_t i = 0; i < o.v.size(); ++i) out[i] = float(o.v[i]);
  if (none_left) *none_left = c;
  return 0;
}

}  // namespace

extern "C" {

int oracle_num_maps(void) { return NMAPS; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Median filter of radius r (window (2r+1)^2), clamped coordinates.
int oracle_median_filter_f64(const double* in, int w, int h, int r, double* out) {
  if (w <= 0 || h <= 0 || r < 0 || !in || !out) return -1;
  Map<double> m(w, h);
  std::memcpy(m.v.data(), in, m.v.size() * sizeof(double));
  Map<double> o = median_filter(m, r);
  std::memcpy(out, o.v.data(), o.v.size() * sizeof(double));
  return 0;
}

// L+ on the original grid (stage (a)).
int oracle_lplus_f64(const double* in, int w, int h, double* out) {
  if (w <= 0 || h <= 0 || !in || !out) return -1;
  Map<double> m(w, h);
  std::memcpy(m.v.data(), in, m.v.size() * sizeof(double));
  Map<double> o = lplus(m);
  std::memcpy(out, o.v.data(), o.v.size() * sizeof(double));
  return 0;
}

// Stage (e) alone: replacement of flagged pixels of J under flags Mk.
int oracle_replace_f64(const float* J, const uint8_t* Mk, int w, int h, float* out, long long* none_left) {
  return replace_entry<double>(J, Mk, w, h, out, none_left);
}
int oracle_replace_f32(const float* J, const uint8_t* Mk, int w, int h, float* out, long long* none_left) {
  return replace_entry<float>(J, Mk, w, h, out, none_left);
}

// One iteration. maps (nullable) receives NMAPS whole-frame maps in the order
// m5, L+, N, S, S', m3, F, R, cand, g1, g2; fragile (nullable) the fragile map;
// counts (nullable) {new flags, flagged pixels with no unflagged neighbour}.
int oracle_iter_f64(const float* J, const uint8_t* Mprev, int w, int h, const oracle_params* p, float* Ik,
                    uint8_t* Mk, double* maps, uint8_t* fragile, long long* counts) {
  return iter_entry<double>(J, Mprev, w, h, p, Ik, Mk, maps, fragile, counts);
}
int oracle_iter_f32(const float* J, const uint8_t* Mprev, int w, int h, const oracle_params* p, float* Ik,
                    uint8_t* Mk, float* maps, uint8_t* fragile, long long* counts) {
  return iter_entry<float>(J, Mprev, w, h, p, Ik, Mk, maps, fragile, counts);
}

// niter iterations from I0 with no flags. counts (nullable) gets 2*niter
// values, {new flags, no-unflagged-neighbour pixels} per iteration;
// fragile_any (nullable) the OR of the per-iteration fragile maps.
int oracle_clean_f64(const float* I0, int w, int h, const oracle_params* p, int niter, float* out_clean,
                     uint8_t* out_mask, long long* counts, uint8_t* fragile_any) {
  return clean_entry<double>(I0, w, h, p, niter, out_clean, out_mask, counts, fragile_any);
}
int oracle_clean_f32(const float* I0, int w, int h, const oracle_params* p, int niter, float* out_clean,
                     uint8_t* out_mask, long long* counts, uint8_t* fragile_any) {
  return clean_entry<float>(I0, w, h, p, niter, out_clean, out_mask, counts, fragile_any);
}

}  // extern "C"
