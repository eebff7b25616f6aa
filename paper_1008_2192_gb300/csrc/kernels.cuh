// CUDA kernels of one L.A.Cosmic iteration (van Dokkum 2001; the work
// function of CRBLASTER, Mighell 2010, Sec. 5) for sm_103a.
//
// detect  : stages (a)-(d) on an output tile plus a 6-pixel halo staged in
//           shared memory. 6 is the dependency radius of the new flags on the
//           input (S' and F need 4, the two growths add 2), the same as the
//           overlap CRBLASTER gives its sub-images (BORDER = 6, Sec. 6.2).
// replace : stage (e) on a tile plus a 2-pixel halo.
//
// Edge rule: every map is filtered with its own coordinates clamped into the
// frame. Each stage computes its map on the in-frame part of its region and
// then replicates the frame-edge values into the out-of-frame part, so the
// next stage reads clamped values without per-read clamping.
//
// Arithmetic: IEEE float32 with explicit round-to-nearest intrinsics (no FMA
// contraction), in the order the stages define: medians are exact selections
// (min/max networks), so every map is the float32 evaluation of its formula.

#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "networks.cuh"

namespace crb {

constexpr int kThreads = 256;
constexpr int kNumMaps = 11;  // m5, L+, N, S, S', m3, F, R, cand, g1, g2

// One frame of a launch. The image buffers alternate between iterations so
// that iteration niter writes out_clean: I_k goes to out_clean when
// (niter - k) is even and to ws otherwise; iteration 1 reads img.
struct Frame {
  const float* img;       // I_0 (input, read-only)
  float* out_clean;       // caller's output
  float* ws;              // workspace image of the same size
  uint32_t* bits;         // cumulative flags: bit x&31 of word [y*wpr + x/32]
  uint8_t* out_mask;      // caller's 0/1 mask, written by the last replacement
  float* maps;            // kNumMaps debug maps (crb_iterate) or nullptr
  unsigned long long* counters;  // 2 per iteration: new flags, no-unflagged-neighbour pixels
  int w, h, wpr;
  float gain, rn;
  int tiles_x, rtiles_x;  // detect / replace tiles per row of tiles
  long long tile0, rtile0;  // first tile index of this frame in the launch
};

struct Params {
  float sigclip, sigfrac, objlim;
  int objlim_form;
};

__device__ __forceinline__ const float* iter_src(const Frame& f, int k, int niter) {
  if (k == 1) return f.img;
  return ((niter - (k - 1)) % 2 == 0) ? f.out_clean : f.ws;
}
__device__ __forceinline__ float* iter_dst(const Frame& f, int k, int niter) {
  return ((niter - k) % 2 == 0) ? f.out_clean : f.ws;
}

// Finds the frame of global tile t (frames sorted by first tile index).
template <bool kReplace>
__device__ __forceinline__ int frame_of(const Frame* frames, int nframes, long long t) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long base = kReplace ? frames[mid].rtile0 : frames[mid].tile0;
    if (base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// --------------------------------------------------------------------------------------------
// Stage formulas, float32, no contraction.

// (a) L+ from the pixel c and its four edge neighbours.
__device__ __forceinline__ float lplus(float c, float up, float down, float left, float right) {
  const float dn = __fsub_rn(c, up), ds = __fsub_rn(c, down);
  const float dw = __fsub_rn(c, left), de = __fsub_rn(c, right);
  float acc = fmaxf(0.f, __fadd_rn(dn, dw));
  acc = __fadd_rn(acc, fmaxf(0.f, __fadd_rn(dn, de)));
  acc = __fadd_rn(acc, fmaxf(0.f, __fadd_rn(ds, dw)));
  acc = __fadd_rn(acc, fmaxf(0.f, __fadd_rn(ds, de)));
  return __fmul_rn(0.25f, acc);
}

// (b) floored 5x5 median -> noise N.
__device__ __forceinline__ float floor_m5(float m5) { return m5 <= 0.f ? 1e-4f : m5; }
__device__ __forceinline__ float noise_of(float m5f, float gain, float rn2) {
  return __fdiv_rn(__fsqrt_rn(__fadd_rn(__fmul_rn(gain, m5f), rn2)), gain);
}

// --------------------------------------------------------------------------------------------
// detect: stages (a)-(d) for one output tile of TW x TH pixels.
//
// Shared-memory regions, each centred on the tile, "Rk" = tile grown by k:
//   sJ  (R6): J, clamped at load (replicate edge);
//   sS  (R4): S = L+/(2N);        sM3 (R5): med3(J);
//   sN  (R2): N (for F/N);        sSp (R2): S' (-inf outside the frame);
//   sC  (R2): candidate flags;    sG1 (R1): first-growth flags.
template <int TW, int TH>
struct DetectLayout {
  static constexpr int JW = TW + 12, JH = TH + 12;
  static constexpr int W4 = TW + 8, H4 = TH + 8;
  static constexpr int W5 = TW + 10, H5 = TH + 10;
  static constexpr int W2 = TW + 4, H2 = TH + 4;
  static constexpr int W1 = TW + 2, H1 = TH + 2;
  static constexpr int oJ = 0;
  static constexpr int oS = oJ + JW * JH;
  static constexpr int oM3 = oS + W4 * H4;
  static constexpr int oN = oM3 + W5 * H5;
  static constexpr int oSp = oN + W2 * H2;
  static constexpr int nFloats = oSp + W2 * H2;
  static constexpr int oC = nFloats * 4;          // bytes
  static constexpr int oG1 = oC + W2 * H2;
  static constexpr size_t bytes = size_t(oG1 + W1 * H1 + 15) / 16 * 16;
};

template <int TW, int TH, bool kMaps>
__device__ void detect_tile(const Frame& f, const Params& p, int k, int niter, long long tile,
                            char* smem) {
  using L = DetectLayout<TW, TH>;
  float* sJ = reinterpret_cast<float*>(smem) + L::oJ;
  float* sS = reinterpret_cast<float*>(smem) + L::oS;
  float* sM3 = reinterpret_cast<float*>(smem) + L::oM3;
  float* sN = reinterpret_cast<float*>(smem) + L::oN;
  float* sSp = reinterpret_cast<float*>(smem) + L::oSp;
  uint8_t* sC = reinterpret_cast<uint8_t*>(smem) + L::oC;
  uint8_t* sG1 = reinterpret_cast<uint8_t*>(smem) + L::oG1;

  const int w = f.w, h = f.h;
  const int ty = int(tile / f.tiles_x), tx = int(tile - (long long)ty * f.tiles_x);
  const int x0 = tx * TW, y0 = ty * TH;
  const float* __restrict__ J = iter_src(f, k, niter);
  const float gain = f.gain, rn2 = __fmul_rn(f.rn, f.rn);
  const float sigclip = p.sigclip, siglow = __fmul_rn(p.sigfrac, p.sigclip), objlim = p.objlim;
  const bool edge = (x0 - 6 < 0) || (y0 - 6 < 0) || (x0 + TW + 6 > w) || (y0 + TH + 6 > h);
  const size_t npix = size_t(w) * size_t(h);

  // 1. J over R6, replicate edge
  for (int i = threadIdx.x; i < L::JW * L::JH; i += kThreads) {
    const int iy = i / L::JW, ix = i - iy * L::JW;
    const int gx = clampi(x0 - 6 + ix, 0, w - 1), gy = clampi(y0 - 6 + iy, 0, h - 1);
    sJ[i] = __ldg(J + size_t(gy) * w + gx);
  }
  __syncthreads();

  // 2. (a)+(b) over R4: m5, N, L+, S; med3 over R5
  for (int i = threadIdx.x; i < L::W4 * L::H4; i += kThreads) {
    const int iy = i / L::W4, ix = i - iy * L::W4;
    const int gx = x0 - 4 + ix, gy = y0 - 4 + iy;
    if (gx < 0 || gx >= w || gy < 0 || gy >= h) continue;
    const int cx = ix + 2, cy = iy + 2;  // centre in sJ
    float v[25];
#pragma unroll
    for (int dy = 0; dy < 5; ++dy)
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = sJ[(cy - 2 + dy) * L::JW + cx - 2 + dx];
    const float m5f = floor_m5(sel_med25(v));
    const float n = noise_of(m5f, gain, rn2);
    const float* c = sJ + cy * L::JW + cx;
    const float lp = lplus(c[0], c[-L::JW], c[L::JW], c[-1], c[1]);
    const float s = __fdiv_rn(lp, __fmul_rn(2.f, n));
    sS[i] = s;
    if (ix >= 2 && ix < L::W4 - 2 && iy >= 2 && iy < L::H4 - 2) sN[(iy - 2) * L::W2 + ix - 2] = n;
    if (kMaps && ix >= 4 && ix < 4 + TW && iy >= 4 && iy < 4 + TH) {
      const size_t o = size_t(gy) * w + gx;
      f.maps[0 * npix + o] = m5f;
      f.maps[1 * npix + o] = lp;
      f.maps[2 * npix + o] = n;
      f.maps[3 * npix + o] = s;
    }
  }
  for (int i = threadIdx.x; i < L::W5 * L::H5; i += kThreads) {
    const int iy = i / L::W5, ix = i - iy * L::W5;
    const int gx = x0 - 5 + ix, gy = y0 - 5 + iy;
    if (gx < 0 || gx >= w || gy < 0 || gy >= h) continue;
    const int cx = ix + 1, cy = iy + 1;
    float v[9];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = sJ[(cy - 1 + dy) * L::JW + cx - 1 + dx];
    const float m3 = sel_med9(v);
    sM3[i] = m3;
    if (kMaps && ix >= 5 && ix < 5 + TW && iy >= 5 && iy < 5 + TH) f.maps[5 * npix + size_t(gy) * w + gx] = m3;
  }
  __syncthreads();
  if (edge) {  // replicate frame-edge values of S and m3 into their out-of-frame entries
    for (int i = threadIdx.x; i < L::W4 * L::H4; i += kThreads) {
      const int iy = i / L::W4, ix = i - iy * L::W4;
      const int gx = x0 - 4 + ix, gy = y0 - 4 + iy;
      if (gx >= 0 && gx < w && gy >= 0 && gy < h) continue;
      const int sx = clampi(gx, 0, w - 1) - (x0 - 4), sy = clampi(gy, 0, h - 1) - (y0 - 4);
      sS[i] = sS[sy * L::W4 + sx];
    }
    for (int i = threadIdx.x; i < L::W5 * L::H5; i += kThreads) {
      const int iy = i / L::W5, ix = i - iy * L::W5;
      const int gx = x0 - 5 + ix, gy = y0 - 5 + iy;
      if (gx >= 0 && gx < w && gy >= 0 && gy < h) continue;
      const int sx = clampi(gx, 0, w - 1) - (x0 - 5), sy = clampi(gy, 0, h - 1) - (y0 - 5);
      sM3[i] = sM3[sy * L::W5 + sx];
    }
    __syncthreads();
  }

  // 3. (b)+(c)+(d) over R2: S' = S - med5(S); candidates with the lazy fine structure
  for (int i = threadIdx.x; i < L::W2 * L::H2; i += kThreads) {
    const int iy = i / L::W2, ix = i - iy * L::W2;
    const int gx = x0 - 2 + ix, gy = y0 - 2 + iy;
    float sp = -INFINITY;
    uint8_t cand = 0;
    if (gx >= 0 && gx < w && gy >= 0 && gy < h) {
      const int cx = ix + 2, cy = iy + 2;  // centre in sS
      float v[25];
#pragma unroll
      for (int dy = 0; dy < 5; ++dy)
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = sS[(cy - 2 + dy) * L::W4 + cx - 2 + dx];
      const float s = sS[cy * L::W4 + cx];
      sp = __fsub_rn(s, sel_med25(v));
      float fval = NAN, rval = NAN;
      if (sp > sigclip) {
        const int mx = ix + 3, my = iy + 3;  // centre in sM3
        float u[49];
#pragma unroll
        for (int dy = 0; dy < 7; ++dy)
#pragma unroll
          for (int dx = 0; dx < 7; ++dx) u[dy * 7 + dx] = sM3[(my - 3 + dy) * L::W5 + mx - 3 + dx];
        fval = __fsub_rn(sM3[my * L::W5 + mx], sel_med49(u));
        const float fn = fmaxf(__fdiv_rn(fval, sN[i]), 0.01f);
        rval = (p.objlim_form == 1) ? __fdiv_rn(__fmul_rn(2.f, s), fn) : __fdiv_rn(sp, fn);
        cand = rval > objlim ? 1 : 0;
      }
      if (kMaps && ix >= 2 && ix < 2 + TW && iy >= 2 && iy < 2 + TH) {
        const size_t o = size_t(gy) * w + gx;
        f.maps[4 * npix + o] = sp;
        f.maps[6 * npix + o] = fval;
        f.maps[7 * npix + o] = rval;
        f.maps[8 * npix + o] = float(cand);
      }
    }
    sSp[i] = sp;
    sC[i] = cand;
  }
  __syncthreads();

  // 4. first growth over R1: 3x3 dilation of the candidates, S' > sigclip
  for (int i = threadIdx.x; i < L::W1 * L::H1; i += kThreads) {
    const int iy = i / L::W1, ix = i - iy * L::W1;
    const int cx = ix + 1, cy = iy + 1;  // centre in R2
    uint8_t any = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) any |= sC[(cy + dy) * L::W2 + cx + dx];
    const uint8_t g1 = (any && sSp[cy * L::W2 + cx] > sigclip) ? 1 : 0;
    sG1[i] = g1;
    if (kMaps && ix >= 1 && ix < 1 + TW && iy >= 1 && iy < 1 + TH) {
      const int gx = x0 - 1 + ix, gy = y0 - 1 + iy;
      if (gx < w && gy < h) f.maps[9 * npix + size_t(gy) * w + gx] = float(g1);
    }
  }
  __syncthreads();

  // 5. second growth on the tile, one 32-pixel mask word per warp step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWordsPerRow = TW / 32;
  unsigned int new_flags = 0;
  for (int wi = warp; wi < kWordsPerRow * TH; wi += kThreads / 32) {
    const int r = wi / kWordsPerRow, wc = wi - r * kWordsPerRow;
    const int lx = wc * 32 + lane, gx = x0 + lx, gy = y0 + r;
    bool g2 = false;
    if (gx < w && gy < h) {
      const int cx = lx + 1, cy = r + 1;  // centre in R1
      uint8_t any = 0;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) any |= sG1[(cy + dy) * L::W1 + cx + dx];
      g2 = any && sSp[(r + 2) * L::W2 + lx + 2] > siglow;
      if (kMaps) f.maps[10 * npix + size_t(gy) * w + gx] = g2 ? 1.f : 0.f;
    }
    const unsigned int word = __ballot_sync(0xffffffffu, g2);
    if (lane == 0 && gy < h && (x0 >> 5) + wc < f.wpr) {
      uint32_t* wp = f.bits + size_t(gy) * f.wpr + (x0 >> 5) + wc;
      const uint32_t prev = *wp;
      *wp = prev | word;
      new_flags += __popc(word & ~prev);
    }
  }
  if (lane == 0 && new_flags) atomicAdd(f.counters + 2 * (k - 1), (unsigned long long)new_flags);
}

template <int TW, int TH, bool kMaps>
__global__ void __launch_bounds__(kThreads) detect_kernel(const Frame* __restrict__ frames, int nframes,
                                                          long long ntiles, Params p, int k, int niter) {
  extern __shared__ __align__(16) char smem[];
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int fi = frame_of<false>(frames, nframes, t);
    const Frame f = frames[fi];
    detect_tile<TW, TH, kMaps>(f, p, k, niter, t - f.tile0, smem);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------------------------
// replace: stage (e) for one tile of RW x RH pixels.
//
// For a flagged pixel with n unflagged window entries, 1 <= n <= 25, the lower
// median (sorted element ceil(n/2)-1 of the unflagged values) equals the
// plain 25-median of the window after a = 13 - ceil(n/2) of its flagged
// entries are set to -inf and the other 12 - floor(n/2) to +inf: the median
// (element 12) is then element 12 - a = ceil(n/2) - 1 of the unflagged values.
// n = 0 falls back to the floored 5x5 median of the window.
template <int RW, int RH>
struct ReplaceLayout {
  static constexpr int W = RW + 4, H = RH + 4;
  static constexpr size_t bytes = size_t(W * H) * 4 + size_t(W * H);
};

__device__ __forceinline__ bool flag_at(const Frame& f, int x, int y) {
  return (f.bits[size_t(y) * f.wpr + (x >> 5)] >> (x & 31)) & 1u;
}

template <int RW, int RH>
__device__ void replace_tile(const Frame& f, int k, int niter, int dense, long long tile, char* smem) {
  using L = ReplaceLayout<RW, RH>;
  float* sJ = reinterpret_cast<float*>(smem);
  uint8_t* sF = reinterpret_cast<uint8_t*>(smem) + L::W * L::H * 4;
  const int w = f.w, h = f.h;
  const int ty = int(tile / f.rtiles_x), tx = int(tile - (long long)ty * f.rtiles_x);
  const int x0 = tx * RW, y0 = ty * RH;
  const float* __restrict__ J = iter_src(f, k, niter);
  float* __restrict__ D = iter_dst(f, k, niter);
  const bool last = (k == niter);

  for (int i = threadIdx.x; i < L::W * L::H; i += kThreads) {
    const int iy = i / L::W, ix = i - iy * L::W;
    const int gx = clampi(x0 - 2 + ix, 0, w - 1), gy = clampi(y0 - 2 + iy, 0, h - 1);
    sJ[i] = __ldg(J + size_t(gy) * w + gx);
    sF[i] = flag_at(f, gx, gy) ? 1 : 0;
  }
  __syncthreads();

  unsigned int none_left = 0;
  for (int i = threadIdx.x; i < RW * RH; i += kThreads) {
    const int ly = i / RW, lx = i - ly * RW;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= w || gy >= h) continue;
    const int c = (ly + 2) * L::W + lx + 2;
    const bool flagged = sF[c];
    const size_t o = size_t(gy) * w + gx;
    float out = sJ[c];
    if (flagged) {
      int n = 0;
#pragma unroll
      for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) n += sF[c + dy * L::W + dx] ? 0 : 1;
      float v[25];
      if (n > 0) {
        const int a = 13 - (n + 1) / 2;  // flagged entries sent to -inf
        int seen = 0;
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
          for (int dx = -2; dx <= 2; ++dx) {
            const int q = c + dy * L::W + dx;
            float val = sJ[q];
            if (sF[q]) {
              val = (seen < a) ? -INFINITY : INFINITY;
              ++seen;
            }
            v[(dy + 2) * 5 + dx + 2] = val;
          }
        out = sel_med25(v);
      } else {
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
          for (int dx = -2; dx <= 2; ++dx) v[(dy + 2) * 5 + dx + 2] = sJ[c + dy * L::W + dx];
        out = floor_m5(sel_med25(v));
        ++none_left;
      }
      D[o] = out;
    } else if (dense) {
      D[o] = out;
    }
    if (last && f.out_mask) f.out_mask[o] = flagged ? 1 : 0;
  }
  // warp-reduce the count of flagged pixels with no unflagged neighbour
  for (int off = 16; off; off >>= 1) none_left += __shfl_xor_sync(0xffffffffu, none_left, off);
  if ((threadIdx.x & 31) == 0 && none_left)
    atomicAdd(f.counters + 2 * (k - 1) + 1, (unsigned long long)none_left);
}

template <int RW, int RH>
__global__ void __launch_bounds__(kThreads) replace_kernel(const Frame* __restrict__ frames, int nframes,
                                                           long long ntiles, int k, int niter, int dense) {
  extern __shared__ __align__(16) char smem[];
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int fi = frame_of<true>(frames, nframes, t);
    const Frame f = frames[fi];
    replace_tile<RW, RH>(f, k, niter, dense, t - f.rtile0, smem);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------------------------
// Helpers: u8 mask <-> flag bits, one warp per 32-pixel word.
static __global__ void bytes_to_bits_kernel(const uint8_t* __restrict__ m, uint32_t* __restrict__ bits, int w, int h,
                                     int wpr) {
  const long long nwords = (long long)wpr * h;
  const int lane = threadIdx.x & 31;
  for (long long wd = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wd < nwords;
       wd += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int y = int(wd / wpr), xw = int(wd - (long long)y * wpr);
    const int x = xw * 32 + lane;
    const bool b = (x < w) && m && m[size_t(y) * w + x];
    const unsigned int word = __ballot_sync(0xffffffffu, b);
    if (lane == 0) bits[wd] = word;
  }
}

}  // namespace crb
