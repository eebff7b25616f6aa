// Queue pipeline: small kernels connected by global work queues, so that every
// sparse step runs with full warps and no block barriers.
//
// Detection (stages a-d) of iteration k:
//   bound          L+ and the upper bound S+ of every pixel -> bit planes hot
//                  (S+ > sigclip), act (S+ > min(sigclip, sigfrac*sigclip))
//                  and lpz (L+ = 0, where S = 0 exactly); in iteration 1 (the
//                  dense pass) also med3 of every pixel -> map M3;
//   need           nsp = needS' = dilate5(hot) & act, needS = dilate5(nsp)
//                  -> queues QS (S to compute) and QSP (S' to compute);
//   s              at QS: m5, N, L+, S -> maps N, S;
//   sp             at QSP: S' = S - med5(S) -> map S'; S' > sigclip -> bit
//                  plane test;
//   m3need         QT = the test bits to (re)test, needM3 = dilate3(QT) ->
//                  queues QT and QM3 (iteration 1: QT only, M3 is whole);
//   m3             at QM3: med3 -> map M3 (iterations >= 2);
//   cand_test      at QT: the objlim test from bounds of med7(m3) (smallest
//                  and largest column median), decided exactly where they
//                  suffice -> candidates; otherwise -> open tests;
//   cand_full      at the open tests: F = m3 - med7(m3) and the test ->
//                  candidates;
//   grow           at the candidates: the two growths, ORed into the flags M.
// Replacement (stage e): the flagged pixels whose value can change are queued,
// their values computed into a side array (rep_compute) and then written in
// place into the one image buffer (rep_write), which the first bound pass
// starts as a copy of I0.
//
// Incremental iterations. Every stage value at a pixel depends on J only within
// a fixed radius (hot/act 2, S 2, nsp 4, S' 4, M3 1, F and the candidate test 4,
// a candidate's growth 6). Iteration k >= 2 therefore recomputes each map only
// where J changed within its radius since iteration k-1, and tests only the
// candidates within 6 px of a change: a candidate farther away grows exactly
// what it grew before, which M already holds. The changed pixels are those that
// the replacement gave a new value: it sets their bits in a changed-pixel plane
// and marks, per cell of one word x kCH rows, the smallest radius class (2, 4
// or 6 px) that reaches into the cell. The bound pass re-tests exactly the
// pixels within 2 px of a changed one (d2, bound_sparse). Validity planes sval
// and m3val record where mapS/mapN and mapM3 hold current values; S' is
// current on all of nsp (nsp and S' change only within 4 px). Iteration 1
// treats every cell as changed; from iteration kSegFrom on, the bit-plane
// kernels walk only the listed segments that hold work.
//
// Replacement is exact in place: a flagged pixel with an unflagged window pixel
// takes the lower median of its unflagged window pixels, which are I0 values
// that are never written; only pixels whose whole window is flagged read
// replaced values, and all values are computed before any is written. Its value
// changes only when its window gains a flag, or, for a fully flagged window,
// when J changes in it; iteration k >= 2 queues the flagged pixels within 2 px
// of a new flag, and every pixel known to have a fully flagged window.
//
// The sets, and the argument that pruning leaves the flags unchanged, are those
// of detect_tile (kernels.cuh). Positions in queues are global pixel indices
// over all frames of the call (frame base + y*w + x); cells are global cell
// indices. Every window read clamps its coordinates into the frame, which
// equals the per-map replicate-edge rule.

#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace crb {

namespace cg = cooperative_groups;

constexpr int kCH = 8;         // rows per cell
// rows per strip of the column-sliding kernels (32 words wide); strips of 32
// rows measured 0.7 % slower per batch step (half the blocks per SM)
constexpr int kSH = 16;
constexpr int kTabShift = 16;  // pixels per entry of the frame table: 2^kTabShift

// queue counters (Queues::n)
enum : int {
  kNS = 0,      // QS (word entries)
  kNSP = 1,     // QSP (word entries)
  kNM3 = 2,     // QM3 (word entries)
  kNT = 3,      // QT (word entries)
  kNRep = 4,    // replacement queue
  kNFresh = 5,  // new flags of this iteration
  kNFb = 6,     // pixels with a fully flagged window (kept over the iterations)
  kNReserved = 7,  // (not used)
  kNPass = 8,   // candidates (passed the objlim test)
  kNAmb = 9,    // tests the column-median bounds leave open
  kNSpx = 10,   // positions in QS, QSP, QM3, QT (work counters)
  kNSPpx = 11,
  kNM3px = 12,
  kNTpx = 13,
  kNB = 14,     // pixels to re-test in the bound pass (word entries)
  kNBpx = 15,
  kNSeg = 16,   // segments (1 word x kSH rows) listed for m3need_seg_kernel,
  kNSegN = 17,  // for need_seg_kernel,
  kNSegD = 18,  // for d2_seg_kernel (the three in Queues::seg order)
  kNCount = 19
};

// QS, QSP, QM3 and QT hold word entries: (global word index, mask of the
// word's pixels), one per word with a set bit, so that the bit-plane kernels
// write one entry per word; the kernels that use them expand the masks into
// one pixel (or group of pixels) per thread (expand_words).
struct Queues {
  uint32_t* q0;     // QS, then QM3, then the candidates, then the replacement values (as float)
  uint32_t* q1;     // QSP, then the open tests, then the replacement queue
  uint32_t* q2;     // the bound pass's pixels (iterations >= 2), then QT
  uint32_t* fresh;  // new flags
  uint32_t* fbl;    // fully flagged windows
  unsigned int* n;  // kNCount counters
  const uint32_t* ftab;  // frame of global pixel t << kTabShift
  uint32_t* seg[3];      // segments listed for m3need, need, d2 (iterations >= kSegFrom): 32 * strip + word
};

// the image J of iteration k (I0, then the in-place buffer)
__device__ __forceinline__ const float* qsrc(const Frame& f, int k) { return k == 1 ? f.img : f.out_clean; }

// frame of word block b (frames sorted by first block)
__device__ __forceinline__ int frame_of_block(const Frame* frames, int nframes, long long b) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].blk0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// frame of strip u (frames sorted by first strip)
__device__ __forceinline__ int frame_of_unit(const Frame* frames, int nframes, long long u) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].u0 <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kBW = 8;   // words (32 px each) per block row: one warp per word column
constexpr int kBH = 32;  // rows per block

// Appends g to queue q from divergent code: one atomic per group of lanes that
// arrive together.
__device__ __forceinline__ void group_append(uint32_t g, uint32_t* q, unsigned int* n) {
  cg::coalesced_group grp = cg::coalesced_threads();
  unsigned int base = 0;
  if (grp.thread_rank() == 0) base = atomicAdd(n, grp.size());
  base = grp.shfl(base, 0);
  q[base + grp.thread_rank()] = g;
}

// ---------------------------------------------------------------------------------------------
// bound: per pixel L+ and the lower bound of m5 (smallest of the five column
// medians) -> bits of S+ > sigclip and S+ > min(sigclip, sigfrac*sigclip) (see detect_tile
// for the bound and its margin). In iteration 1 a warp walks down a strip of
// four word columns, two rows per step, keeping the rows of its columns (and of
// the halo columns, held by lanes 0-3) in registers.
//
// Sliding column medians: the windows of rows y and y+1 share the four values
// of rows y-1..y+2. With c1 <= c2 the two middle values of those four, the
// median of the four and one more value e is min(max(e, c1), c2).

__device__ __forceinline__ float clamp_med(float e, float c1, float c2) { return fminf(fmaxf(e, c1), c2); }

// Thresholds of the bound test of a frame: S+ = L+ / (2 N-) with N- from the
// floored lower bound mlow of m5, so S+ > t is L+^2 > 4 t^2 / gain^2 * (gain *
// max(mlow, 0) + rn^2). kh uses t = sigclip (hot), kl t = min(sigclip,
// sigfrac*sigclip) (act); the factor 0.9999 keeps the test conservative
// against the roundings of both sides. Computed once per frame on the host,
// so the dense pass and the re-test compare against the same values.
__host__ __device__ inline void bound_thresholds(const Params& p, float gain, float& kl, float& kh) {
  const float sigclip = p.sigclip, tlow = fminf(p.sigfrac * p.sigclip, sigclip), g2 = gain * gain;
  kh = 4.f * sigclip * sigclip * 0.9999f / g2;
  kl = 4.f * tlow * tlow * 0.9999f / g2;
}

// The two bound tests of one pixel from its L+ and the smallest of its five
// column medians, with every rounding spelled out: the dense pass and the
// re-test share it, so a pixel re-tested with an unchanged window keeps its
// bits exactly.
__device__ __forceinline__ void bound_test(float lp, float mlow, float gain, float rn2, float kl, float kh, bool& act,
                                           bool& hot) {
  const float den = __fmaf_rn(gain, mlow > 0.f ? mlow : 0.f, rn2);
  const float lhs = __fmul_rn(lp, lp);
  act = lhs > __fmul_rn(kl, den);
  hot = lhs > __fmul_rn(kh, den);
}

// Sliding column-median state of one column: rows r-2 .. r+1 of the current step.
struct Col4 {
  float a, b, c, d;
};

// Advances a column by the two rows (e, g) below it: the medians of the five
// rows around the first and the second row of the step.
__device__ __forceinline__ void col_step(Col4& s, float e, float g, float& m0, float& m1) {
  const float l1 = fminf(s.b, s.c), h1 = fmaxf(s.b, s.c), l2 = fminf(s.d, e), h2 = fmaxf(s.d, e);
  const float u = fmaxf(l1, l2), v = fminf(h1, h2);
  const float c1 = fminf(u, v), c2 = fmaxf(u, v);
  m0 = clamp_med(s.a, c1, c2);
  m1 = clamp_med(g, c1, c2);
}

// The three values sorted: lo <= mi <= hi.
__device__ __forceinline__ void sort3(float a, float b, float c, float& lo, float& mi, float& hi) {
  const float s0 = fminf(a, b), s1 = fmaxf(a, b);
  hi = fmaxf(s1, c);
  const float t = fminf(s1, c);
  lo = fminf(s0, t);
  mi = fmaxf(s0, t);
}
__device__ __forceinline__ float med3f(float a, float b, float c) { return fmaxf(fminf(a, b), fminf(fmaxf(a, b), c)); }

// hot/act/lpz bits of the NP word columns wc .. wc+NP-1 (wc a multiple of NP),
// rows [y0, y1), of frame f (whole warp), NP pixels per lane (NP = 4 or 8):
// lane l holds x0+NP*l .. x0+NP*l+NP-1 (16-byte loads per row when the row
// pitch and the base allow), so a shuffle brings two neighbours of NP pixels;
// lanes 0-3 also hold the halo columns x0-2, x0-1, x0+32NP, x0+32NP+1. Each
// group of 32/NP lanes forms one word of every plane by OR-ing its lanes'
// NP-bit fields in log2(32/NP) shuffles. The re-test (bound_sparse_kernel)
// forms the same values with the same roundings (bound_test), so a re-tested
// pixel whose window did not change keeps its bits.
template <int NP>
__device__ __forceinline__ void bound_span(const Frame& f, const float* __restrict__ J, int wc, int y0, int y1,
                                           float* __restrict__ copy, float* __restrict__ m3out) {
  static_assert(NP == 4 || NP == 8, "whole 16-byte vectors, whole words per lane group");
  constexpr int kLanesPerWord = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int w = f.w, h = f.h;
  const float gain = f.gain, rn2 = __fmul_rn(f.rn, f.rn), kl = f.bkl, kh = f.bkh;
  const int x0 = wc * 32, xp = x0 + NP * lane;
  int cx[NP];
  uint32_t valid = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    cx[i] = min(xp + i, w - 1);
    valid |= (xp + i < w ? 1u : 0u) << i;
  }
  const int hx = lane < 2 ? x0 - 2 + lane : x0 + 32 * NP - 2 + lane;  // halo columns (lanes 0-3)
  const int hc = clampi(hx, 0, w - 1);
  const bool vec = ((reinterpret_cast<uintptr_t>(J) & 15u) == 0) && ((w & 3) == 0) && (xp + NP - 1 < w);
  const bool vcopy = vec && ((reinterpret_cast<uintptr_t>(copy) & 15u) == 0);
  const bool vm3 = vec && ((reinterpret_cast<uintptr_t>(m3out) & 15u) == 0);
  const int src_h0 = lane == 0 ? 0 : 2, src_h1 = lane == 0 ? 1 : 3, src_hl = lane == 0 ? 1 : 2;
  auto ld = [&](int yy, float (&v)[NP], float& vh) {
    const float* r = J + size_t(clampi(yy, 0, h - 1)) * size_t(w);
    if (vec) {
#pragma unroll
      for (int q = 0; q < NP / 4; ++q) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(r + xp) + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = __ldg(r + cx[i]);
    }
    vh = __ldg(r + hc);
  };
  Col4 A[NP], H;
  {
    float v[NP];
    ld(y0 - 2, v, H.a);
#pragma unroll
    for (int i = 0; i < NP; ++i) A[i].a = v[i];
    ld(y0 - 1, v, H.b);
#pragma unroll
    for (int i = 0; i < NP; ++i) A[i].b = v[i];
    ld(y0, v, H.c);
#pragma unroll
    for (int i = 0; i < NP; ++i) A[i].c = v[i];
    ld(y0 + 1, v, H.d);
#pragma unroll
    for (int i = 0; i < NP; ++i) A[i].d = v[i];
  }
  const int sh = NP * (lane % kLanesPerWord);
  for (int y = y0; y < y1; y += 2) {
    float e[NP], g[NP], eh, gh;
    ld(y + 2, e, eh);
    ld(y + 3, g, gh);
    float m[NP][2], mh[2];
#pragma unroll
    for (int i = 0; i < NP; ++i) col_step(A[i], e[i], g[i], m[i][0], m[i][1]);
    col_step(H, eh, gh, mh[0], mh[1]);
    // vertical differences: the first row's c - down is minus the second row's c - up
    float vd[NP];  // rows y+1 - y
#pragma unroll
    for (int i = 0; i < NP; ++i) vd[i] = __fsub_rn(A[i].d, A[i].c);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int yy = y + s;
      if (yy >= y1) break;
      // column medians x-2, x-1 (lane-1) and x+NP, x+NP+1 (lane+1) of the lane's NP; halo at the ends
      float c[NP + 4];
#pragma unroll
      for (int i = 0; i < NP; ++i) c[i + 2] = m[i][s];
      c[0] = __shfl_up_sync(0xffffffffu, m[NP - 2][s], 1);
      c[1] = __shfl_up_sync(0xffffffffu, m[NP - 1][s], 1);
      c[NP + 2] = __shfl_down_sync(0xffffffffu, m[0][s], 1);
      c[NP + 3] = __shfl_down_sync(0xffffffffu, m[1][s], 1);
      const float hX = __shfl_sync(0xffffffffu, mh[s], src_h0), hY = __shfl_sync(0xffffffffu, mh[s], src_h1);
      if (lane == 0) {
        c[0] = hX;
        c[1] = hY;
      }
      if (lane == 31) {
        c[NP + 2] = hX;
        c[NP + 3] = hY;
      }
      // the row of the step and its differences to the rows above and below
      float cc[NP], du[NP], dd[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        cc[i] = s ? A[i].d : A[i].c;
        du[i] = s ? vd[i] : __fsub_rn(A[i].c, A[i].b);
        dd[i] = s ? __fsub_rn(A[i].d, e[i]) : -vd[i];
      }
      const float hcc = s ? H.d : H.c;
      const float hL = __shfl_sync(0xffffffffu, hcc, src_hl);
      float lft = __shfl_up_sync(0xffffffffu, cc[NP - 1], 1), rgt = __shfl_down_sync(0xffffffffu, cc[0], 1);
      if (lane == 0) lft = hL;
      if (lane == 31) rgt = hL;
      if (copy) {
        float* o = copy + size_t(yy) * w;
        if (vcopy) {
#pragma unroll
          for (int q = 0; q < NP / 4; ++q)
            reinterpret_cast<float4*>(o + xp)[q] = make_float4(cc[4 * q], cc[4 * q + 1], cc[4 * q + 2], cc[4 * q + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < NP; ++i)
            if (xp + i < w) o[xp + i] = cc[i];
        }
      }
      if (m3out) {
        // med3 of the row (as m3_kernel): each column's three rows sorted, then the median of the
        // largest column minimum, the median of the column medians and the smallest column maximum;
        // columns x-1 and x+NP from the neighbour lanes, x0-1 and x0+32*NP from the halo lanes 1, 2
        float lo[NP + 2], mi[NP + 2], hi[NP + 2];
#pragma unroll
        for (int i = 0; i < NP; ++i) sort3(s ? A[i].c : A[i].b, cc[i], s ? e[i] : A[i].d, lo[i + 1], mi[i + 1], hi[i + 1]);
        float tl, tm, th;
        sort3(s ? H.c : H.b, s ? H.d : H.c, s ? eh : H.d, tl, tm, th);
        tl = __shfl_sync(0xffffffffu, tl, src_hl);
        tm = __shfl_sync(0xffffffffu, tm, src_hl);
        th = __shfl_sync(0xffffffffu, th, src_hl);
        lo[0] = __shfl_up_sync(0xffffffffu, lo[NP], 1);
        mi[0] = __shfl_up_sync(0xffffffffu, mi[NP], 1);
        hi[0] = __shfl_up_sync(0xffffffffu, hi[NP], 1);
        lo[NP + 1] = __shfl_down_sync(0xffffffffu, lo[1], 1);
        mi[NP + 1] = __shfl_down_sync(0xffffffffu, mi[1], 1);
        hi[NP + 1] = __shfl_down_sync(0xffffffffu, hi[1], 1);
        if (lane == 0) lo[0] = tl, mi[0] = tm, hi[0] = th;
        if (lane == 31) lo[NP + 1] = tl, mi[NP + 1] = tm, hi[NP + 1] = th;
        float m3v[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const float pl = max3f(lo[i], lo[i + 1], lo[i + 2]);
          const float pm = med3f(mi[i], mi[i + 1], mi[i + 2]);
          const float ph = min3f(hi[i], hi[i + 1], hi[i + 2]);
          m3v[i] = med3f(pl, pm, ph);
        }
        float* o = m3out + size_t(yy) * w;
        if (vm3) {
#pragma unroll
          for (int q = 0; q < NP / 4; ++q)
            reinterpret_cast<float4*>(o + xp)[q] = make_float4(m3v[4 * q], m3v[4 * q + 1], m3v[4 * q + 2], m3v[4 * q + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < NP; ++i)
            if (xp + i < w) o[xp + i] = m3v[i];
        }
      }
      // horizontal differences: pixel i's c - left is dh[i], its c - right is -dh[i + 1]
      float dh[NP + 1];
      dh[0] = __fsub_rn(cc[0], lft);
#pragma unroll
      for (int i = 1; i < NP; ++i) dh[i] = __fsub_rn(cc[i], cc[i - 1]);
      dh[NP] = __fsub_rn(rgt, cc[NP - 1]);
      uint32_t va = 0, vh = 0, vz = 0;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const float mlow = min3f(min3f(c[i], c[i + 1], c[i + 2]), c[i + 3], c[i + 4]);
        const float lp = lplus_d(du[i], dd[i], dh[i], -dh[i + 1]);
        bool act, hot;
        bound_test(lp, mlow, gain, rn2, kl, kh, act, hot);
        va |= uint32_t(act) << i;
        vh |= uint32_t(hot) << i;
        vz |= uint32_t(lp == 0.f) << i;
      }
      va = (va & valid) << sh;
      vh = (vh & valid) << sh;
      vz = (vz & valid) << sh;
#pragma unroll
      for (int o = 1; o < kLanesPerWord; o <<= 1) {
        va |= __shfl_xor_sync(0xffffffffu, va, o);
        vh |= __shfl_xor_sync(0xffffffffu, vh, o);
        vz |= __shfl_xor_sync(0xffffffffu, vz, o);
      }
      const int wo = wc + lane / kLanesPerWord;
      if (lane % kLanesPerWord == 0 && wo < f.wpr) {
        const size_t o = size_t(yy) * f.wpr + wo;
        f.act[o] = va;
        f.hot[o] = vh;
        f.lpz[o] = vz;
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) A[i] = Col4{A[i].c, A[i].d, e[i], g[i]};
    H = Col4{H.c, H.d, eh, gh};
  }
}

// bound_dense_kernel (iteration 1): the dense bound pass, blocks of kBW words
// x kBH rows, warps of kBoundNP words (kBoundNP pixels per lane). Eight pixels
// per lane (126 registers, sixteen one-warp blocks per SM) measured 10 % faster
// than four (80 registers, twelve two-warp blocks); spans of 64 or 128 rows per
// warp measured slower than 32.
constexpr int kBoundNP = 8;
constexpr int kBoundThreads = 32 * kBW / kBoundNP;

__global__ void __launch_bounds__(kBoundThreads, kBoundNP == 4 ? 12 : 16)
    bound_dense_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks, Params p) {
  const int warp = threadIdx.x >> 5;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int wc = bxs * kBW + kBoundNP * warp;
    if (wc >= f.wpr) continue;  // whole warp
    const int y0 = bys * kBH;
    bound_span<kBoundNP>(f, f.img, wc, y0, min(y0 + kBH, f.h), f.out_clean, f.mapM3);
  }
}

// ---------------------------------------------------------------------------------------------
// Block-level helpers for the bit-plane kernels: a block covers kBW words x kBH
// rows of one frame; 256 threads = one thread per word.

// horizontal dilation by R of word v with its neighbours l (left), r (right)
template <int R>
__device__ __forceinline__ uint32_t hdil(uint32_t l, uint32_t v, uint32_t r) {
  uint32_t o = v;
#pragma unroll
  for (int d = 1; d <= R; ++d) o |= (v << d) | (l >> (32 - d)) | (v >> d) | (r << (32 - d));
  return o;
}

// in-frame bits of word wc (bits beyond the frame width are 0)
__device__ __forceinline__ uint32_t frame_word(int wc, int w) {
  const int lim = w - 32 * wc;
  return lim >= 32 ? 0xffffffffu : (lim <= 0 ? 0u : ((1u << lim) - 1u));
}

// Appends g to each list j with put[j] (NL <= 3 lists, counters n[0..NL-1]),
// in thread order; one atomic per block and list. Every thread of the block
// calls it; ws holds kThreads/32 + 1 ints, sbase NL.
template <int NL>
__device__ __forceinline__ void block_append(const bool (&put)[NL], uint32_t g, uint32_t* const (&q)[NL],
                                             unsigned int* n, int* ws, unsigned int* sbase) {
  int packed = 0;  // 10 bits per list (at most kThreads entries each)
#pragma unroll
  for (int j = 0; j < NL; ++j) packed |= (put[j] ? 1 : 0) << (10 * j);
  int total = 0;
  const int off = block_excl_scan(packed, ws, total);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const unsigned int t = unsigned(total >> (10 * j)) & 1023u;
      sbase[j] = t ? atomicAdd(n + j, t) : 0u;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NL; ++j)
    if (put[j]) q[j][sbase[j] + (unsigned(off >> (10 * j)) & 1023u)] = g;
  __syncthreads();
}

// cell class of word (wc, y) of frame f; 4 (everything changed) without classes
__device__ __forceinline__ uint32_t cell_class(const uint32_t* __restrict__ cls, const Frame& f, int wc, int y) {
  return cls ? cls[f.cell0 + (long long)(y / kCH) * f.wpr + wc] : 4u;
}

// The column kernels (need, m3need): one warp per strip of 32 words x kSH rows,
// lane = word. The lane walks down the strip keeping the last rows of its word
// in registers, so a vertical dilation is an OR of registers and a horizontal
// one an OR across lanes; lanes 0 and 31 also carry the words left and right of
// the strip, of which only the bits next to the strip are used. The strip's
// queue words wait in shared memory until the warp has counted them: one
// atomic per warp and queue, then one coalesced entry per nonzero word.
constexpr int kColWarps = 4;
// rows per load chunk of the strip kernels: a chunk's loads are issued together
constexpr int kColChunk = 4;

struct ColWords {
  uint32_t w[kColWarps][kSH][2][32];  // per warp, row, queue: the word of each lane
};

// Counts a row's words of queue j (entries: words with a bit; positions: bits).
__device__ __forceinline__ void col_count(uint32_t v, unsigned int& ents, unsigned int& pix) {
  ents += __popc(__ballot_sync(0xffffffffu, v != 0u));
  pix += __reduce_add_sync(0xffffffffu, unsigned(__popc(v)));
}

// Writes the warp's entries of queue j: row rr of the lane's column is the
// global word gw0 + rr * wpr (both per lane).
__device__ __forceinline__ void col_write(const ColWords& sw, int warp, int j, uint32_t gw0, int wpr,
                                          unsigned int base, uint2* q) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int rr = 0; rr < kSH; ++rr) {
    const uint32_t v = sw.w[warp][rr][j][lane];
    const unsigned bal = __ballot_sync(0xffffffffu, v != 0u);
    if (v) q[base + __popc(bal & ((1u << lane) - 1u))] = make_uint2(gw0 + uint32_t(rr) * uint32_t(wpr), v);
    base += __popc(bal);
  }
}

// Reserves the strip's entries and positions of two queues (counters ne[0..1],
// np[0..1]); returns the entry bases to every lane.
__device__ __forceinline__ void col_reserve(const unsigned int (&ents)[2], const unsigned int (&pix)[2],
                                            unsigned int* ne0, unsigned int* ne1, unsigned int* np0,
                                            unsigned int* np1, unsigned int (&base)[2]) {
  const int lane = threadIdx.x & 31;
  unsigned int b0 = 0, b1 = 0;
  if (lane == 0) {
    if (ents[0]) b0 = atomicAdd(ne0, ents[0]);
    if (ents[1]) b1 = atomicAdd(ne1, ents[1]);
    if (pix[0]) atomicAdd(np0, pix[0]);
    if (pix[1]) atomicAdd(np1, pix[1]);
  }
  base[0] = __shfl_sync(0xffffffffu, b0, 0);
  base[1] = __shfl_sync(0xffffffffu, b1, 0);
}

// Whether this lane's word (and halo word) has a cell of class >= 2 among the
// strip's cell rows, widened by `margin` cell rows: a strip where no lane has
// one has nothing to compute (iterations >= 2).
__device__ __forceinline__ bool strip_has_class2(const uint32_t* __restrict__ cls, const Frame& f, int wc, bool inw,
                                                 int hw, bool hin, int y0, int margin) {
  const int cy0 = y0 / kCH - margin, cy1 = min((y0 + kSH) / kCH + margin, f.ncy);
  bool any = false;
  for (int cy = max(cy0, 0); cy < cy1; ++cy) {
    const uint32_t* row = cls + f.cell0 + (long long)cy * f.wpr;
    if ((inw && row[wc] >= 2u) || (hin && row[hw] >= 2u)) any = true;
  }
  return any;
}

// need_kernel: nsp = dilate5(hot) & act, needS = dilate5(nsp) within the frame,
// per word by cell class (iteration 1: class 4 everywhere): within 4 px of a
// change (class >= 3) nsp is written, test cleared (sp sets it again) and all of
// nsp queued for S'; within 6 px (class >= 2), S is queued where needS holds
// and S is not current (sval; cleared within 2 px). Column kernel: rows
// y0-4 .. y0+kSH+3 feed the five-row windows of hot and nsp.
__global__ void __launch_bounds__(kColWarps * 32) need_kernel(const Frame* __restrict__ frames, int nframes,
                                                              long long nunits, Queues Q,
                                                              const uint32_t* __restrict__ cls) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long u = (long long)blockIdx.x * kColWarps + warp; u < nunits; u += (long long)gridDim.x * kColWarps) {
    const Frame& f = frames[frame_of_unit(frames, nframes, u)];
    const long long lu = u - f.u0;
    const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
    const int wc0 = ux * 32, y0 = uy * kSH, wc = wc0 + lane;
    const bool inw = wc < f.wpr;
    const int hw = lane == 0 ? wc0 - 1 : wc0 + 32;  // halo word (lanes 0 and 31)
    const bool hin = (lane == 0 || lane == 31) && hw >= 0 && hw < f.wpr;
    const uint32_t fmask = inw ? frame_word(wc, f.w) : 0u;
    if (cls && !__any_sync(0xffffffffu, strip_has_class2(cls, f, wc, inw, -1, false, y0, 0))) continue;
    uint32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0, h4 = 0;  // own hot, rows r-4 .. r
    uint32_t g0 = 0, g1 = 0, g2 = 0, g3 = 0, g4 = 0;  // halo hot
    uint32_t a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;  // act, rows r-2 .. r (own, halo)
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0, n4 = 0;  // own nsp, rows r-6 .. r-2
    uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0;  // halo nsp
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    // rows y0-4 .. y0+kSH+3 in chunks of kColChunk: the chunk's loads are issued together
    static_assert((kSH + 8) % kColChunk == 0, "whole chunks");
    for (int rc = y0 - 4; rc < y0 + kSH + 4; rc += kColChunk) {
      uint32_t Lh[kColChunk], La[kColChunk], Lgh[kColChunk], Lga[kColChunk], Lc[kColChunk], Ls[kColChunk],
          Lz[kColChunk];
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        const int r = rc + i, yo = r - 4;
        const bool rin = r >= 0 && r < f.h;
        const size_t ro = size_t(rin ? r : 0) * f.wpr;
        Lh[i] = (rin && inw) ? f.hot[ro + wc] : 0u;
        La[i] = (rin && inw) ? f.act[ro + wc] : 0u;
        Lgh[i] = (rin && hin) ? f.hot[ro + hw] : 0u;
        Lga[i] = (rin && hin) ? f.act[ro + hw] : 0u;
        const bool out = yo >= y0 && yo < f.h && inw;
        // the sval and lpz loads do not wait for the class: it masks them afterwards
        Lc[i] = out ? cell_class(cls, f, wc, yo) : 0u;
        Ls[i] = (out && cls) ? f.sval[size_t(yo) * f.wpr + wc] : 0u;
        Lz[i] = out ? f.lpz[size_t(yo) * f.wpr + wc] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        h0 = h1; h1 = h2; h2 = h3; h3 = h4; h4 = Lh[i];
        g0 = g1; g1 = g2; g2 = g3; g3 = g4; g4 = Lgh[i];
        a0 = a1; a1 = a2; a2 = La[i];
        b0 = b1; b1 = b2; b2 = Lga[i];
        // nsp of row r-2
        const uint32_t vh = h0 | h1 | h2 | h3 | h4, gvh = g0 | g1 | g2 | g3 | g4;
        uint32_t left = __shfl_up_sync(0xffffffffu, vh, 1), right = __shfl_down_sync(0xffffffffu, vh, 1);
        const uint32_t gl = __shfl_sync(0xffffffffu, gvh, 0), gr = __shfl_sync(0xffffffffu, gvh, 31);
        if (lane == 0) left = gl;
        if (lane == 31) right = gr;
        const uint32_t nsp = hdil<2>(left, vh, right) & a0;
        const uint32_t gn = (lane == 0 ? hdil<2>(0u, gvh, vh) : hdil<2>(vh, gvh, 0u)) & b0;
        n0 = n1; n1 = n2; n2 = n3; n3 = n4; n4 = nsp;
        m0 = m1; m1 = m2; m2 = m3; m3 = m4; m4 = gn;
        // needS of row r-4
        const int yo = rc + i - 4;
        if (yo < y0) continue;  // whole warp
        const uint32_t vn = n0 | n1 | n2 | n3 | n4, gvn = m0 | m1 | m2 | m3 | m4;
        uint32_t nl = __shfl_up_sync(0xffffffffu, vn, 1), nr = __shfl_down_sync(0xffffffffu, vn, 1);
        const uint32_t gnl = __shfl_sync(0xffffffffu, gvn, 0), gnr = __shfl_sync(0xffffffffu, gvn, 31);
        if (lane == 0) nl = gnl;
        if (lane == 31) nr = gnr;
        uint32_t qs = 0, qsp = 0;
        const uint32_t cl = Lc[i];  // 0 outside the frame
        if (cl >= 2u) {
          const uint32_t needS = hdil<2>(nl, vn, nr) & fmask;
          const size_t o = size_t(yo) * f.wpr + wc;
          if (cl >= 3u) {
            qsp = n2;  // nsp of row yo
            f.nsp[o] = qsp;
            f.test[o] = 0u;
          }
          const uint32_t sv = cl >= 4u ? 0u : Ls[i];  // nothing is current in cells of class 4
          qs = needS & ~sv & ~Lz[i];                  // S = 0 exactly where L+ = 0: no median needed
          if ((sv | needS) != sv || cl >= 4u) f.sval[o] = sv | needS;
        }
        sw.w[warp][yo - y0][0][lane] = qs;
        sw.w[warp][yo - y0][1][lane] = qsp;
        col_count(qs, ents[0], pix[0]);
        col_count(qsp, ents[1], pix[1]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNS, Q.n + kNSP, Q.n + kNSpx, Q.n + kNSPpx, base);
    __syncwarp();
    col_write(sw, warp, 0, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[0], reinterpret_cast<uint2*>(Q.q0));
    col_write(sw, warp, 1, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[1], reinterpret_cast<uint2*>(Q.q1));
    __syncwarp();  // the shared words are refilled for the next strip
  }
}

// m3need_kernel: QT = the test bits of cells of class >= 2, needM3 = dilate3(QT)
// within the frame -> queue QT, and queue QM3 where M3 is not current (m3val;
// cleared in cells of class 4); bit plane m3val. Column kernel: rows y0-3 ..
// y0+kSH+2 feed the seven-row window of QT. kAll (iteration 1): every cell
// counts as changed and cls is not read; the dense bound pass has written M3
// on the whole frame, so QM3 is empty and m3val full.
template <bool kAll>
__global__ void __launch_bounds__(kColWarps * 32) m3need_kernel(const Frame* __restrict__ frames, int nframes,
                                                                long long nunits, Queues Q,
                                                                const uint32_t* __restrict__ cls_in) {
  const uint32_t* __restrict__ cls = kAll ? nullptr : cls_in;
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long u = (long long)blockIdx.x * kColWarps + warp; u < nunits; u += (long long)gridDim.x * kColWarps) {
    const Frame& f = frames[frame_of_unit(frames, nframes, u)];
    const long long lu = u - f.u0;
    const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
    const int wc0 = ux * 32, y0 = uy * kSH, wc = wc0 + lane;
    const bool inw = wc < f.wpr;
    const int hw = lane == 0 ? wc0 - 1 : wc0 + 32;
    const bool hin = (lane == 0 || lane == 31) && hw >= 0 && hw < f.wpr;
    const uint32_t fmask = inw ? frame_word(wc, f.w) : 0u;
    if (cls && !__any_sync(0xffffffffu, strip_has_class2(cls, f, wc, inw, hw, hin, y0, 1))) continue;
    if constexpr (kAll) {
      // iteration 1: the dense bound pass wrote M3 everywhere, so M3 is current on the whole frame and
      // nothing is queued for m3; QT = the test words
      unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
      uint32_t tq[kSH];
#pragma unroll
      for (int t = 0; t < kSH; ++t) tq[t] = (inw && y0 + t < f.h) ? f.test[size_t(y0 + t) * f.wpr + wc] : 0u;
#pragma unroll
      for (int t = 0; t < kSH; ++t) {
        if (inw && y0 + t < f.h) f.m3val[size_t(y0 + t) * f.wpr + wc] = fmask;
        sw.w[warp][t][0][lane] = 0u;
        sw.w[warp][t][1][lane] = tq[t];
        col_count(tq[t], ents[1], pix[1]);
      }
      unsigned int base[2];
      col_reserve(ents, pix, Q.n + kNM3, Q.n + kNT, Q.n + kNM3px, Q.n + kNTpx, base);
      __syncwarp();
      col_write(sw, warp, 1, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[1],
                reinterpret_cast<uint2*>(Q.q2));
      __syncwarp();
      continue;
    }
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0;  // own QT words, rows r-6 .. r
    uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0;  // halo QT words
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    // rows y0-3 .. y0+kSH+2 in chunks of kColChunk (the last chunk runs past the end)
    for (int rc = y0 - 3; rc < y0 + kSH + 3; rc += kColChunk) {
      uint32_t Lq[kColChunk], Lg[kColChunk], Lm[kColChunk], Lc4[kColChunk];
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        const int r = rc + i, yo = r - 3;
        const bool rin = r >= 0 && r < f.h && r < y0 + kSH + 3;
        const size_t ro = size_t(rin ? r : 0) * f.wpr;
        Lq[i] = (rin && inw && cell_class(cls, f, wc, r) >= 2u) ? f.test[ro + wc] : 0u;
        Lg[i] = (rin && hin && cell_class(cls, f, hw, r) >= 2u) ? f.test[ro + hw] : 0u;
        const bool out = yo >= y0 && yo < y0 + kSH && yo < f.h && inw;
        Lc4[i] = out ? uint32_t(cell_class(cls, f, wc, yo) >= 4u) : 0u;
        Lm[i] = (out && !Lc4[i]) ? f.m3val[size_t(yo) * f.wpr + wc] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = Lq[i];
        s0 = s1; s1 = s2; s2 = s3; s3 = s4; s4 = s5; s5 = s6; s6 = Lg[i];
        const int yo = rc + i - 3;
        if (yo < y0 || yo >= y0 + kSH) continue;  // whole warp
        const uint32_t v = t0 | t1 | t2 | t3 | t4 | t5 | t6, gv = s0 | s1 | s2 | s3 | s4 | s5 | s6;
        uint32_t left = __shfl_up_sync(0xffffffffu, v, 1), right = __shfl_down_sync(0xffffffffu, v, 1);
        const uint32_t gl = __shfl_sync(0xffffffffu, gv, 0), gr = __shfl_sync(0xffffffffu, gv, 31);
        if (lane == 0) left = gl;
        if (lane == 31) right = gr;
        uint32_t qm = 0, qto = 0;
        if (yo < f.h && inw) {
          const uint32_t need = hdil<3>(left, v, right) & fmask;
          const bool c4 = Lc4[i] != 0u;
          if (need || c4) {
            const uint32_t old = Lm[i];  // 0 in cells of class 4
            qm = need & ~old;
            if (c4 || qm) f.m3val[size_t(yo) * f.wpr + wc] = old | need;
          }
          qto = t3;  // QT word of row yo
        }
        sw.w[warp][yo - y0][0][lane] = qm;
        sw.w[warp][yo - y0][1][lane] = qto;
        col_count(qm, ents[0], pix[0]);
        col_count(qto, ents[1], pix[1]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNM3, Q.n + kNT, Q.n + kNM3px, Q.n + kNTpx, base);
    __syncwarp();
    col_write(sw, warp, 0, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[0], reinterpret_cast<uint2*>(Q.q0));
    col_write(sw, warp, 1, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[1], reinterpret_cast<uint2*>(Q.q2));
    __syncwarp();
  }
}

// d2_kernel (iteration >= 2): the pixels within 2 px of a change (the
// changed-pixel plane of this iteration, dilated by 5 x 5 within the frame) ->
// word entries of the pixels the bound pass re-tests (q2). Column kernel: rows
// y0-2 .. y0+kSH+1 feed the five-row window.
__global__ void __launch_bounds__(kColWarps * 32) d2_kernel(const Frame* __restrict__ frames, int nframes,
                                                            long long nunits, Queues Q, int k) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long u = (long long)blockIdx.x * kColWarps + warp; u < nunits; u += (long long)gridDim.x * kColWarps) {
    const Frame& f = frames[frame_of_unit(frames, nframes, u)];
    const uint32_t* __restrict__ chg = f.chg[k & 1];
    const long long lu = u - f.u0;
    const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
    const int wc0 = ux * 32, y0 = uy * kSH, wc = wc0 + lane;
    const bool inw = wc < f.wpr;
    const int hw = lane == 0 ? wc0 - 1 : wc0 + 32;
    const bool hin = (lane == 0 || lane == 31) && hw >= 0 && hw < f.wpr;
    const uint32_t fmask = inw ? frame_word(wc, f.w) : 0u;
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0, e4 = 0;
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    for (int rc = y0 - 2; rc < y0 + kSH + 2; rc += kColChunk) {  // the last chunk may run past the end
      uint32_t L[kColChunk], G[kColChunk];
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        const int r = rc + i;
        const bool rin = r >= 0 && r < f.h && r < y0 + kSH + 2;
        const size_t ro = size_t(rin ? r : 0) * f.wpr;
        L[i] = (rin && inw) ? chg[ro + wc] : 0u;
        G[i] = (rin && hin) ? chg[ro + hw] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kColChunk; ++i) {
        c0 = c1; c1 = c2; c2 = c3; c3 = c4; c4 = L[i];
        e0 = e1; e1 = e2; e2 = e3; e3 = e4; e4 = G[i];
        const int yo = rc + i - 2;
        if (yo < y0 || yo >= y0 + kSH) continue;  // whole warp
        const uint32_t v = c0 | c1 | c2 | c3 | c4, gv = e0 | e1 | e2 | e3 | e4;
        uint32_t left = __shfl_up_sync(0xffffffffu, v, 1), right = __shfl_down_sync(0xffffffffu, v, 1);
        const uint32_t gl = __shfl_sync(0xffffffffu, gv, 0), gr = __shfl_sync(0xffffffffu, gv, 31);
        if (lane == 0) left = gl;
        if (lane == 31) right = gr;
        const uint32_t d2 = (yo < f.h) ? (hdil<2>(left, v, right) & fmask) : 0u;
        sw.w[warp][yo - y0][0][lane] = d2;
        col_count(d2, ents[0], pix[0]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNB, Q.n + kNB, Q.n + kNBpx, Q.n + kNBpx, base);
    __syncwarp();
    col_write(sw, warp, 0, uint32_t(f.word0 + (long long)y0 * f.wpr + wc), f.wpr, base[0], reinterpret_cast<uint2*>(Q.q2));
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Segment kernels (iterations >= kSegFrom). A segment is one word column of a
// strip (32 px x kSH rows). From the third iteration on, the cells near a
// change are a small part of each frame, though they still touch most strips;
// so the segments with work are listed first, and the lanes of a warp each walk
// one listed segment down its rows, loading the words left and right of it
// themselves (the strip kernels above share them across lanes instead). The
// outputs are those of the strip kernels: a segment left out of the list has
// none, because every output of need, m3need and d2 lies within 3 px of a cell
// of class >= 2.
constexpr int kSegFrom = 3;

// seg_list_kernel: lists the segments each segment kernel walks. d2: a cell
// of class 4 among the segment's own cells (a pixel within 2 px of a change
// lies in one); need: a cell of class >= 2 among them; m3need: a cell of class
// >= 2 in the segment's word column or the ones left and right of it, among
// the segment's cell rows widened by one each way (QT of those cells reaches 3
// px into the segment). 8 strips per block (warp = strip, lane = word); one
// atomic per block and list.
__global__ void __launch_bounds__(kThreads) seg_list_kernel(const Frame* __restrict__ frames, int nframes,
                                                            long long nunits, Queues Q,
                                                            const uint32_t* __restrict__ cls) {
  __shared__ int ws[kThreads / 32 + 1];
  __shared__ unsigned int sbase[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kThreads / 32, kCells = kSH / kCH;
  for (long long ub = (long long)blockIdx.x * kWarps; ub < nunits; ub += (long long)gridDim.x * kWarps) {
    const long long u = ub + warp;
    bool put[3] = {false, false, false};
    if (u < nunits) {  // whole warp
      const Frame& f = frames[frame_of_unit(frames, nframes, u)];
      const long long lu = u - f.u0;
      const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
      const int wc0 = ux * 32, wc = wc0 + lane;
      const bool inw = wc < f.wpr;
      const int hw = lane == 0 ? wc0 - 1 : wc0 + 32;
      const bool hin = (lane == 0 || lane == 31) && hw >= 0 && hw < f.wpr;
      bool own2 = false, own4 = false, near2 = false, halo2 = false;
      for (int cy = max(uy * kCells - 1, 0); cy < min((uy + 1) * kCells + 1, f.ncy); ++cy) {
        const uint32_t* row = cls + f.cell0 + (long long)cy * f.wpr;
        const uint32_t c = inw ? row[wc] : 0u;
        const bool mine = cy >= uy * kCells && cy < (uy + 1) * kCells;
        near2 |= c >= 2u;
        own2 |= mine && c >= 2u;
        own4 |= mine && c >= 4u;
        if (hin && row[hw] >= 2u) halo2 = true;
      }
      const bool l = __shfl_up_sync(0xffffffffu, near2, 1), r = __shfl_down_sync(0xffffffffu, near2, 1);
      put[0] = inw && (near2 || (lane == 0 ? halo2 : l) || (lane == 31 ? halo2 : r));
      put[1] = own2;
      put[2] = own4;
    }
    uint32_t* const qq[3] = {Q.seg[0], Q.seg[1], Q.seg[2]};
    block_append<3>(put, uint32_t(u * 32 + lane), qq, Q.n + kNSeg, ws, sbase);
  }
}

// A lane's listed segment: frame, word column wc, first row y0; ok = false for
// the lanes past the end of the list (their loads and outputs are masked off).
struct SegLane {
  const Frame* f;
  int wc, y0, wpr, h;
  bool ok, inl, inr;  // inl, inr: the words left and right of wc are in the frame
  uint32_t fmask;     // in-frame bits of word wc
  uint32_t gw0;       // global word of (wc, y0)
};

__device__ __forceinline__ SegLane seg_lane(const Frame* __restrict__ frames, int nframes, const uint32_t* seg,
                                            unsigned int b, unsigned int nseg) {
  const int lane = threadIdx.x & 31;
  SegLane L;
  L.ok = b + lane < nseg;
  const uint32_t s = seg[L.ok ? b + lane : b];
  const long long u = s >> 5;
  L.f = frames + frame_of_unit(frames, nframes, u);
  const Frame& f = *L.f;
  const long long lu = u - f.u0;
  const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
  L.wc = ux * 32 + int(s & 31u);
  L.y0 = uy * kSH;
  L.wpr = f.wpr;
  L.h = f.h;
  L.inl = L.ok && L.wc > 0;
  L.inr = L.ok && L.wc + 1 < f.wpr;
  L.fmask = L.ok ? frame_word(L.wc, f.w) : 0u;
  L.gw0 = uint32_t(f.word0 + (long long)L.y0 * f.wpr + L.wc);
  return L;
}

// d2_seg_kernel: d2_kernel over the listed segments.
__global__ void __launch_bounds__(kColWarps * 32) d2_seg_kernel(const Frame* __restrict__ frames, int nframes,
                                                                Queues Q, int k) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int nseg = Q.n[kNSegD];
  for (unsigned int b = (blockIdx.x * kColWarps + warp) * 32u; b < nseg; b += gridDim.x * kColWarps * 32u) {
    const SegLane S = seg_lane(frames, nframes, Q.seg[2], b, nseg);
    const Frame& f = *S.f;
    const int wc = S.wc, y0 = S.y0, wpr = S.wpr, h = S.h;
    const bool ok = S.ok, inl = S.inl, inr = S.inr;
    const uint32_t* __restrict__ chg = f.chg[k & 1];
    uint32_t cl0 = 0, cl1 = 0, cl2 = 0, cl3 = 0, cl4 = 0;  // rows r-4 .. r: left, own, right words
    uint32_t cc0 = 0, cc1 = 0, cc2 = 0, cc3 = 0, cc4 = 0;
    uint32_t cr0 = 0, cr1 = 0, cr2 = 0, cr3 = 0, cr4 = 0;
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    for (int tc = -2; tc < kSH + 2; tc += 8) {  // rows y0-2 .. y0+kSH+1 (the last chunk runs past them)
      uint32_t L[8], C[8], R[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = y0 + tc + i;
        const bool rin = ok && r >= 0 && r < h && tc + i < kSH + 2;
        const size_t ro = size_t(rin ? r : 0) * wpr + wc;
        C[i] = rin ? chg[ro] : 0u;
        L[i] = (rin && inl) ? chg[ro - 1] : 0u;
        R[i] = (rin && inr) ? chg[ro + 1] : 0u;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        cl0 = cl1; cl1 = cl2; cl2 = cl3; cl3 = cl4; cl4 = L[i];
        cc0 = cc1; cc1 = cc2; cc2 = cc3; cc3 = cc4; cc4 = C[i];
        cr0 = cr1; cr1 = cr2; cr2 = cr3; cr3 = cr4; cr4 = R[i];
        const int t = tc + i - 2;
        if (t < 0 || t >= kSH) continue;  // whole warp
        const uint32_t v = cc0 | cc1 | cc2 | cc3 | cc4;
        const uint32_t d2 = (y0 + t < h) ? (hdil<2>(cl0 | cl1 | cl2 | cl3 | cl4, v, cr0 | cr1 | cr2 | cr3 | cr4) & S.fmask) : 0u;
        sw.w[warp][t][0][lane] = d2;
        col_count(d2, ents[0], pix[0]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNB, Q.n + kNB, Q.n + kNBpx, Q.n + kNBpx, base);
    __syncwarp();
    col_write(sw, warp, 0, S.gw0, wpr, base[0], reinterpret_cast<uint2*>(Q.q2));
    __syncwarp();
  }
}

// need_seg_kernel: need_kernel over the listed segments.
__global__ void __launch_bounds__(kColWarps * 32) need_seg_kernel(const Frame* __restrict__ frames, int nframes,
                                                                  Queues Q, const uint32_t* __restrict__ cls) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int nseg = Q.n[kNSegN];
  for (unsigned int b = (blockIdx.x * kColWarps + warp) * 32u; b < nseg; b += gridDim.x * kColWarps * 32u) {
    const SegLane S = seg_lane(frames, nframes, Q.seg[1], b, nseg);
    const Frame& f = *S.f;
    const int wc = S.wc, y0 = S.y0, wpr = S.wpr, h = S.h;
    const bool ok = S.ok, inl = S.inl, inr = S.inr;
    const uint32_t* __restrict__ hot = f.hot;
    const uint32_t* __restrict__ act = f.act;
    const long long cb = f.cell0 + wc;  // cell (wc, y / kCH) at cb + (y / kCH) * wpr
    uint32_t hl[5] = {}, hc[5] = {}, hr[5] = {};  // hot, rows r-4 .. r: left, own, right words
    uint32_t al[3] = {}, ac[3] = {}, ar[3] = {};  // act, rows r-2 .. r
    uint32_t nl[5] = {}, nc[5] = {}, nr[5] = {};  // nsp, rows r-6 .. r-2
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    constexpr int kC = 4;  // rows per chunk of loads
    for (int tc = -4; tc < kSH + 4; tc += kC) {  // rows y0-4 .. y0+kSH+3
      uint32_t Hl[kC], Hc[kC], Hr[kC], Al[kC], Ac[kC], Ar[kC], Cl[kC], Sv[kC], Lz[kC];
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int r = y0 + tc + i, yo = r - 4;
        const bool rin = ok && r >= 0 && r < h;
        const size_t ro = size_t(rin ? r : 0) * wpr + wc;
        Hc[i] = rin ? hot[ro] : 0u;
        Ac[i] = rin ? act[ro] : 0u;
        Hl[i] = (rin && inl) ? hot[ro - 1] : 0u;
        Al[i] = (rin && inl) ? act[ro - 1] : 0u;
        Hr[i] = (rin && inr) ? hot[ro + 1] : 0u;
        Ar[i] = (rin && inr) ? act[ro + 1] : 0u;
        const bool out = ok && tc + i >= 4 && yo < h;
        const size_t oo = size_t(out ? yo : 0) * wpr + wc;
        // the loads do not wait for the class (the few listed segments make the extra bytes cheap)
        Cl[i] = out ? cls[cb + (long long)(yo / kCH) * wpr] : 0u;
        Sv[i] = out ? f.sval[oo] : 0u;
        Lz[i] = out ? f.lpz[oo] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kC; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) { hl[j] = hl[j + 1]; hc[j] = hc[j + 1]; hr[j] = hr[j + 1]; }
        hl[4] = Hl[i]; hc[4] = Hc[i]; hr[4] = Hr[i];
#pragma unroll
        for (int j = 0; j < 2; ++j) { al[j] = al[j + 1]; ac[j] = ac[j + 1]; ar[j] = ar[j + 1]; }
        al[2] = Al[i]; ac[2] = Ac[i]; ar[2] = Ar[i];
        // nsp of row r-2: exact in the own word, and in the two bits of each side word next to it
        const uint32_t vl = hl[0] | hl[1] | hl[2] | hl[3] | hl[4];
        const uint32_t vc = hc[0] | hc[1] | hc[2] | hc[3] | hc[4];
        const uint32_t vr = hr[0] | hr[1] | hr[2] | hr[3] | hr[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) { nl[j] = nl[j + 1]; nc[j] = nc[j + 1]; nr[j] = nr[j + 1]; }
        nl[4] = hdil<2>(0u, vl, vc) & al[0];
        nc[4] = hdil<2>(vl, vc, vr) & ac[0];
        nr[4] = hdil<2>(vc, vr, 0u) & ar[0];
        // needS of row r-4
        const int t = tc + i - 4;
        if (t < 0) continue;  // whole warp
        uint32_t qs = 0, qsp = 0;
        const uint32_t cl = Cl[i];  // 0 outside the frame
        if (cl >= 2u) {
          const uint32_t needS = hdil<2>(nl[0] | nl[1] | nl[2] | nl[3] | nl[4], nc[0] | nc[1] | nc[2] | nc[3] | nc[4],
                                         nr[0] | nr[1] | nr[2] | nr[3] | nr[4]) &
                                 S.fmask;
          const size_t o = size_t(y0 + t) * wpr + wc;
          if (cl >= 3u) {
            qsp = nc[2];  // nsp of row y0+t
            f.nsp[o] = qsp;
            f.test[o] = 0u;
          }
          const uint32_t sv = cl < 4u ? Sv[i] : 0u;  // S is not current anywhere in cells of class 4
          qs = needS & ~sv & ~Lz[i];
          if ((sv | needS) != sv || cl >= 4u) f.sval[o] = sv | needS;
        }
        sw.w[warp][t][0][lane] = qs;
        sw.w[warp][t][1][lane] = qsp;
        col_count(qs, ents[0], pix[0]);
        col_count(qsp, ents[1], pix[1]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNS, Q.n + kNSP, Q.n + kNSpx, Q.n + kNSPpx, base);
    __syncwarp();
    col_write(sw, warp, 0, S.gw0, wpr, base[0], reinterpret_cast<uint2*>(Q.q0));
    col_write(sw, warp, 1, S.gw0, wpr, base[1], reinterpret_cast<uint2*>(Q.q1));
    __syncwarp();
  }
}

// m3need_seg_kernel: m3need_kernel over the listed segments.
__global__ void __launch_bounds__(kColWarps * 32) m3need_seg_kernel(const Frame* __restrict__ frames, int nframes,
                                                                    Queues Q, const uint32_t* __restrict__ cls) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int nseg = Q.n[kNSeg];
  for (unsigned int b = (blockIdx.x * kColWarps + warp) * 32u; b < nseg; b += gridDim.x * kColWarps * 32u) {
    const SegLane S = seg_lane(frames, nframes, Q.seg[0], b, nseg);
    const Frame& f = *S.f;
    const int wc = S.wc, y0 = S.y0, wpr = S.wpr, h = S.h;
    const bool ok = S.ok, inl = S.inl, inr = S.inr;
    const uint32_t* __restrict__ test = f.test;
    const long long cb = f.cell0 + wc;
    uint32_t ql[7] = {}, qc[7] = {}, qr[7] = {};  // QT, rows r-6 .. r: left, own, right words
    unsigned int ents[2] = {0u, 0u}, pix[2] = {0u, 0u};
    for (int tc = -3; tc < kSH + 3; tc += 8) {  // rows y0-3 .. y0+kSH+2 (the last chunk runs past them)
      uint32_t Ql[8], Qc[8], Qr[8], Lm[8], Lc4[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = y0 + tc + i, t = tc + i - 3;
        const bool rin = ok && r >= 0 && r < h && tc + i < kSH + 3;
        const size_t ro = size_t(rin ? r : 0) * wpr + wc;
        const long long cr = cb + (long long)((rin ? r : 0) / kCH) * wpr;
        // the loads do not wait for the classes: test is masked by them afterwards
        Qc[i] = rin ? test[ro] & (cls[cr] >= 2u ? ~0u : 0u) : 0u;
        Ql[i] = (rin && inl) ? test[ro - 1] & (cls[cr - 1] >= 2u ? ~0u : 0u) : 0u;
        Qr[i] = (rin && inr) ? test[ro + 1] & (cls[cr + 1] >= 2u ? ~0u : 0u) : 0u;
        const bool out = ok && t >= 0 && t < kSH && y0 + t < h;
        Lc4[i] = out ? uint32_t(cls[cb + (long long)((y0 + t) / kCH) * wpr] >= 4u) : 0u;
        Lm[i] = out ? f.m3val[size_t(y0 + t) * wpr + wc] : 0u;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 6; ++j) { ql[j] = ql[j + 1]; qc[j] = qc[j + 1]; qr[j] = qr[j + 1]; }
        ql[6] = Ql[i]; qc[6] = Qc[i]; qr[6] = Qr[i];
        const int t = tc + i - 3;
        if (t < 0 || t >= kSH) continue;  // whole warp
        uint32_t qm = 0, qto = 0;
        if (ok && y0 + t < h) {
          const uint32_t need = hdil<3>(ql[0] | ql[1] | ql[2] | ql[3] | ql[4] | ql[5] | ql[6],
                                        qc[0] | qc[1] | qc[2] | qc[3] | qc[4] | qc[5] | qc[6],
                                        qr[0] | qr[1] | qr[2] | qr[3] | qr[4] | qr[5] | qr[6]) &
                                S.fmask;
          const bool c4 = Lc4[i] != 0u;
          if (need || c4) {
            const uint32_t old = c4 ? 0u : Lm[i];  // M3 is not current anywhere in cells of class 4
            qm = need & ~old;
            if (c4 || qm) f.m3val[size_t(y0 + t) * wpr + wc] = old | need;
          }
          qto = qc[3];  // QT word of row y0+t
        }
        sw.w[warp][t][0][lane] = qm;
        sw.w[warp][t][1][lane] = qto;
        col_count(qm, ents[0], pix[0]);
        col_count(qto, ents[1], pix[1]);
      }
    }
    unsigned int base[2];
    col_reserve(ents, pix, Q.n + kNM3, Q.n + kNT, Q.n + kNM3px, Q.n + kNTpx, base);
    __syncwarp();
    col_write(sw, warp, 0, S.gw0, wpr, base[0], reinterpret_cast<uint2*>(Q.q0));
    col_write(sw, warp, 1, S.gw0, wpr, base[1], reinterpret_cast<uint2*>(Q.q2));
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Queue kernels: one thread per entry, grid-stride over the queue length.

struct Pix {
  int fi, x, y;
};

// Frame and coordinates of global pixel index g: the table gives the frame of
// the first pixel of g's 2^kTabShift block, later frames in the block follow.
__device__ __forceinline__ Pix decode(const Frame* frames, int nframes, const Queues& Q, uint32_t g) {
  Pix p;
  int fi = int(__ldg(Q.ftab + (g >> kTabShift)));
  while (fi + 1 < nframes && frames[fi + 1].pix0 <= (long long)g) ++fi;
  p.fi = fi;
  const uint32_t o = g - uint32_t(frames[fi].pix0);
  const int w = frames[fi].w;
  p.y = int(o / uint32_t(w));
  p.x = int(o - uint32_t(p.y) * uint32_t(w));
  return p;
}

// The (2R+1)^2 window of map a around (x, y), row-major, coordinates clamped
// into the w x h frame; away from the frame edge the loads take immediate
// offsets from one row pointer.
template <int R>
__device__ __forceinline__ void load_window(const float* __restrict__ a, int x, int y, int w, int h,
                                            float (&v)[(2 * R + 1) * (2 * R + 1)]) {
  constexpr int D = 2 * R + 1;
  if (x >= R && x < w - R && y >= R && y < h - R) {
    const float* __restrict__ p = a + size_t(y - R) * w + (x - R);
#pragma unroll
    for (int dy = 0; dy < D; ++dy)
#pragma unroll
      for (int dx = 0; dx < D; ++dx) v[dy * D + dx] = __ldg(p + size_t(dy) * w + dx);
  } else {
    int xs[D];
    size_t ro[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      xs[d] = clampi(x - R + d, 0, w - 1);
      ro[d] = size_t(clampi(y - R + d, 0, h - 1)) * w;
    }
#pragma unroll
    for (int dy = 0; dy < D; ++dy)
#pragma unroll
      for (int dx = 0; dx < D; ++dx) v[dy * D + dx] = __ldg(a + ro[dy] + xs[dx]);
  }
}

// Bits of columns xs .. xs+4 of row qy of a bit plane (bit dx = column
// xs + dx); columns outside [0, w) read as 0.
__device__ __forceinline__ uint32_t plane_bits5(const uint32_t* __restrict__ plane, int wpr, int w, int xs, int qy) {
  const int wl = max(xs, 0) >> 5, wr = min(xs + 4, w - 1) >> 5;
  const uint64_t pair = uint64_t(plane[size_t(qy) * wpr + wl]) | (uint64_t(plane[size_t(qy) * wpr + wr]) << 32);
  const int sh = xs - 32 * wl;  // in [-2, 31]
  uint32_t b = uint32_t(sh >= 0 ? (pair >> sh) : (pair << -sh)) & 31u;
#pragma unroll
  for (int dx = 0; dx < 5; ++dx)
    if (xs + dx < 0 || xs + dx >= w) b &= ~(1u << dx);
  return b;
}

// Frame, row and first column of global word gw (frames sorted by first word).
__device__ __forceinline__ void decode_word(const Frame* frames, int nframes, uint32_t gw, int& fi, int& y, int& x0) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].word0 <= (long long)gw) lo = mid; else hi = mid - 1;
  }
  fi = lo;
  const uint32_t lw = gw - uint32_t(frames[lo].word0), wpr = uint32_t(frames[lo].wpr);
  y = int(lw / wpr);
  x0 = 32 * int(lw - uint32_t(y) * wpr);
}

// Rows y-R .. y+R and columns x0-R .. x0+3+R of a (clamped at the frame's
// edges, as load_window) for a group of four pixels, x0 a multiple of 4: away
// from the edges, three aligned 16-byte loads per row (x0-4 .. x0+7).
template <int R>
__device__ __forceinline__ void load_span(const float* __restrict__ a, int x0, int y, int w, int h,
                                          float (&v)[2 * R + 1][4 + 2 * R]) {
  static_assert(R >= 1 && R <= 4, "the 16-byte loads cover 4 columns either side");
  const bool vec = x0 >= 4 && x0 + 8 <= w && (w & 3) == 0 && (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
#pragma unroll
  for (int dy = 0; dy <= 2 * R; ++dy) {
    const float* __restrict__ r = a + size_t(clampi(y - R + dy, 0, h - 1)) * size_t(w);
    if (vec) {
      const float4 A = __ldg(reinterpret_cast<const float4*>(r + x0 - 4));
      const float4 M = __ldg(reinterpret_cast<const float4*>(r + x0));
      const float4 C = __ldg(reinterpret_cast<const float4*>(r + x0 + 4));
      const float s12[12] = {A.x, A.y, A.z, A.w, M.x, M.y, M.z, M.w, C.x, C.y, C.z, C.w};
#pragma unroll
      for (int c = 0; c < 4 + 2 * R; ++c) v[dy][c] = s12[4 - R + c];
    } else {
#pragma unroll
      for (int c = 0; c < 4 + 2 * R; ++c) v[dy][c] = __ldg(r + clampi(x0 - R + c, 0, w - 1));
    }
  }
}

// The mask of the kGran-pixel groups of word mask m that hold a set bit (bit i:
// pixels kGran*i .. kGran*i + kGran-1).
template <int kGran>
__device__ __forceinline__ uint32_t group_mask(uint32_t m) {
  if (kGran == 1) return m;
  uint32_t g = 0;
#pragma unroll
  for (int i = 0; i < 32 / kGran; ++i) g |= uint32_t(((m >> (kGran * i)) & ((1u << kGran) - 1u)) != 0u) << i;
  return g;
}

// Expands a queue of n word entries into items of kGran pixels (1: pixels; 4:
// the groups of four with a listed pixel), one warp at a time: the warp takes
// 32 entries, each lane writes the items of its entry (entry lane, group
// index) to the warp's list in shared memory at its exclusive prefix, and the
// warp then hands one item per lane per round from that list. There is no
// block barrier, so a warp waiting on its loads holds back no other. Every
// lane of the warp runs every round and calls body(valid, frame, x, y) with x
// the item's first pixel (grouped: body(valid, frame, x, y, bits), bits = the
// listed pixels of the group, bit i for pixel x + i), so body may hold
// warp-wide steps. kRev takes the entries from the end of the queue first: a
// kernel that reads what the previous one wrote last (still in L2) then starts
// with it. Blocks of kThreads threads.
template <int kGran = 1, bool kRev = false, typename F>
__device__ __forceinline__ void expand_words(const Frame* __restrict__ frames, int nframes, const uint2* __restrict__ q,
                                             unsigned int n, F&& body) {
  constexpr int kPer = 32 / kGran;  // items per entry at most
  __shared__ uint16_t items[kThreads / 32][32 * kPer];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int wpb = blockDim.x >> 5;
  for (unsigned int c0 = (blockIdx.x * wpb + warp) * 32u; c0 < n; c0 += gridDim.x * wpb * 32u) {
    uint32_t m = 0, pm = 0;
    int fi = 0, y = 0, x0 = 0;
    if (c0 + lane < n) {
      const uint2 e = q[kRev ? n - 1u - (c0 + lane) : c0 + lane];
      pm = e.y;
      m = group_mask<kGran>(e.y);
      decode_word(frames, nframes, e.x, fi, y, x0);
    }
    const int cnt = __popc(m);
    int incl = cnt;  // inclusive prefix of the item counts over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    {
      int pos = incl - cnt;
      uint32_t mm = m;
      while (mm) {
        const int b = __ffs(mm) - 1;
        mm &= mm - 1u;
        items[warp][pos++] = uint16_t((lane << 5) | b);
      }
    }
    __syncwarp();
    for (int r0 = 0; r0 < total; r0 += 32) {
      const int j = r0 + lane;
      const bool valid = j < total;
      const int code = valid ? int(items[warp][j]) : 0;
      const int k = code >> 5, bit = code & 31;
      const int fk = __shfl_sync(0xffffffffu, fi, k), yk = __shfl_sync(0xffffffffu, y, k);
      const int xk = __shfl_sync(0xffffffffu, x0, k);
      if constexpr (kGran == 1) {
        body(valid, fk, xk + bit, yk);
      } else {
        const uint32_t pk = __shfl_sync(0xffffffffu, pm, k);
        const uint32_t bits = valid ? (pk >> (kGran * bit)) & ((1u << kGran) - 1u) : 0u;
        body(valid, fk, xk + kGran * bit, yk, bits);
      }
    }
    __syncwarp();  // the list is refilled for the next entries
  }
}

// Per-warp staging of NL lists in shared memory: a warp adds its lanes' entries
// without an atomic, and moves a list to global memory with one atomic when it
// would overflow and at the end (flush). Warp-wide calls; no block barrier.
template <int NL, int CAP>
struct WarpLists {
  uint32_t v[kThreads / 32][NL][CAP];
  unsigned int n[kThreads / 32][NL];

  __device__ __forceinline__ void init() {
    if ((threadIdx.x & 31) < NL) n[threadIdx.x >> 5][threadIdx.x & 31] = 0u;
    __syncwarp();
  }

  __device__ __forceinline__ void flush_list(int j, uint32_t* q, unsigned int* cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int m = n[warp][j];
    unsigned int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, m);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (unsigned int i = lane; i < m; i += 32) q[base + i] = v[warp][j][i];
    __syncwarp();
    if (lane == 0) n[warp][j] = 0u;
    __syncwarp();
  }

  // adds g to list j (global list q[j], counter cnt[j]) on the lanes with put[j]
  __device__ __forceinline__ void put(const bool (&p)[NL], uint32_t g, uint32_t* const (&q)[NL], unsigned int* cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const unsigned bal = __ballot_sync(0xffffffffu, p[j]);
      if (!bal) continue;
      if (n[warp][j] + unsigned(__popc(bal)) > unsigned(CAP)) flush_list(j, q[j], cnt + j);
      const unsigned int n0 = n[warp][j];
      if (p[j]) v[warp][j][n0 + __popc(bal & ((1u << lane) - 1u))] = g;
      __syncwarp();
      if (lane == 0) n[warp][j] = n0 + unsigned(__popc(bal));
      __syncwarp();
    }
  }

  __device__ __forceinline__ void flush(uint32_t* const (&q)[NL], unsigned int* cnt) {
#pragma unroll
    for (int j = 0; j < NL; ++j) flush_list(j, q[j], cnt + j);
  }
};

// Rows y-2 .. y+2 and columns x0-2 .. x0+3 of a (clamped at the frame's
// edges, as load_window) for a pair of pixels, x0 even: away from the edges,
// three aligned 8-byte loads per row.
__device__ __forceinline__ void load_pair_span(const float* __restrict__ a, int x0, int y, int w, int h,
                                               float (&v)[5][6]) {
  const bool vec = x0 >= 2 && x0 + 4 <= w && (w & 1) == 0 && (reinterpret_cast<uintptr_t>(a) & 7u) == 0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const float* __restrict__ r = a + size_t(clampi(y - 2 + dy, 0, h - 1)) * size_t(w);
    if (vec) {
      const float2 A = __ldg(reinterpret_cast<const float2*>(r + x0 - 2));
      const float2 M = __ldg(reinterpret_cast<const float2*>(r + x0));
      const float2 C = __ldg(reinterpret_cast<const float2*>(r + x0 + 2));
      v[dy][0] = A.x, v[dy][1] = A.y, v[dy][2] = M.x, v[dy][3] = M.y, v[dy][4] = C.x, v[dy][5] = C.y;
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) v[dy][c] = __ldg(r + clampi(x0 - 2 + c, 0, w - 1));
    }
  }
}

// s_kernel: at QS, m5 (floored), N, L+ and S of J, by aligned pairs of pixels
// x0, x0+1 that hold a listed one: both 5x5 medians come from one network over
// the pair's six sorted columns x0-2 .. x0+3 (med25_row2), which loads and
// sorts each column once instead of five times. A pair's unlisted pixel is
// computed but not written. (QS is mostly small isolated 5x5 blobs: aligned
// groups of four would hold 1.9 listed pixels on average, and measured slower
// than single medians; a run of five listed pixels fills three pairs.)
__global__ void __launch_bounds__(256, 4) s_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, int k) {
  expand_words<2, true>(frames, nframes, reinterpret_cast<const uint2*>(Q.q0), Q.n[kNS],
                  [&](bool valid, int fi, int x0, int y, uint32_t bits) {
                    if (!valid) return;
                    const Frame& f = frames[fi];
                    float v[5][6], m5[2];
                    load_pair_span(qsrc(f, k), x0, y, f.w, f.h, v);
                    med25_row2(v, m5);
                    const float rn2 = __fmul_rn(f.rn, f.rn);
                    const size_t o = size_t(y) * f.w + x0;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                      if (!((bits >> i) & 1u)) continue;
                      const float lp = lplus(v[2][i + 2], v[1][i + 2], v[3][i + 2], v[2][i + 1], v[2][i + 3]);
                      const float nn = noise_of(floor_m5(m5[i]), f.gain, rn2);
                      f.mapS[o + i] = __fdiv_rn(lp, __fmul_rn(2.f, nn));
                      f.mapN[o + i] = nn;
                    }
                  });
}

// Bits of columns xs .. xs+7 of row qy of a bit plane (bit c = column xs + c),
// for 0 <= xs and xs + 7 < w: at most two words.
__device__ __forceinline__ uint32_t plane_bits8(const uint32_t* __restrict__ plane, int wpr, int xs, int qy) {
  const size_t ro = size_t(qy) * wpr + (xs >> 5);
  const int sh = xs & 31;
  uint64_t pair = plane[ro];
  if (sh > 24) pair |= uint64_t(plane[ro + 1]) << 32;
  return uint32_t(pair >> sh) & 0xffu;
}

// sp_kernel: at QSP, S' = S - med5(S); S' > sigclip -> test bit (in iteration
// 1 also S' > sigfrac*sigclip -> low bit, for grow_first_kernel). By aligned
// pairs as s_kernel (S is exactly 0 where L+ = 0, the lpz plane, where mapS is
// not written); the pair's bits go out with one atomic OR per plane. Three blocks
// per SM (80 registers, 20 B of spills) measured 4 % faster than two (103).
__global__ void __launch_bounds__(256, 3) sp_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, Params p,
                                                    int k) {
  const float siglow = __fmul_rn(p.sigfrac, p.sigclip);
  expand_words<2, true>(frames, nframes, reinterpret_cast<const uint2*>(Q.q1), Q.n[kNSP],
                  [&](bool valid, int fi, int x0, int y, uint32_t bits) {
                    if (!valid) return;
                    const Frame& f = frames[fi];
                    float v[5][6], med[2];
                    load_pair_span(f.mapS, x0, y, f.w, f.h, v);
                    if (x0 >= 2 && x0 + 5 < f.w) {
#pragma unroll
                      for (int dy = 0; dy < 5; ++dy) {
                        const uint32_t z = plane_bits8(f.lpz, f.wpr, x0 - 2, clampi(y - 2 + dy, 0, f.h - 1));
#pragma unroll
                        for (int c = 0; c < 6; ++c)
                          if ((z >> c) & 1u) v[dy][c] = 0.f;
                      }
                    } else {
#pragma unroll
                      for (int dy = 0; dy < 5; ++dy) {
                        const size_t ro = size_t(clampi(y - 2 + dy, 0, f.h - 1)) * f.wpr;
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                          const int xx = clampi(x0 - 2 + c, 0, f.w - 1);
                          if ((f.lpz[ro + (xx >> 5)] >> (xx & 31)) & 1u) v[dy][c] = 0.f;
                        }
                      }
                    }
                    med25_row2(v, med);
                    float* __restrict__ out = f.mapSp + size_t(y) * f.w + x0;
                    uint32_t tb = 0, lb = 0;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                      if (!((bits >> i) & 1u)) continue;
                      const float sp = __fsub_rn(v[2][i + 2], med[i]);
                      out[i] = sp;
                      tb |= uint32_t(sp > p.sigclip) << i;
                      lb |= uint32_t(sp > siglow) << i;
                    }
                    if (tb) atomicOr(&f.test[size_t(y) * f.wpr + (x0 >> 5)], tb << (x0 & 31));
                    if (k == 1 && lb) atomicOr(&f.low[size_t(y) * f.wpr + (x0 >> 5)], lb << (x0 & 31));
                  });
}

// m3_kernel: at QM3, med3 of J, by groups of four pixels x0 .. x0+3 that hold
// a listed one. The six columns x0-1 .. x0+4 of the rows y-1 .. y+1 are sorted
// once; the median of a 3x3 window is then the median of three values: the
// largest of its column minima, the median of its column medians and the
// smallest of its column maxima (an exact selection of the fifth of nine).
__global__ void __launch_bounds__(256) m3_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, int k) {
  expand_words<4, true>(frames, nframes, reinterpret_cast<const uint2*>(Q.q0), Q.n[kNM3],
                  [&](bool valid, int fi, int x0, int y, uint32_t bits) {
                    if (!valid) return;
                    const Frame& f = frames[fi];
                    float v[3][6];
                    load_span<1>(qsrc(f, k), x0, y, f.w, f.h, v);
                    float lo[6], mi[6], hi[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {  // sort the column: lo <= mi <= hi
                      const float s0 = fminf(v[0][c], v[1][c]), s1 = fmaxf(v[0][c], v[1][c]);
                      hi[c] = fmaxf(s1, v[2][c]);
                      const float t = fminf(s1, v[2][c]);
                      lo[c] = fminf(s0, t);
                      mi[c] = fmaxf(s0, t);
                    }
                    float* __restrict__ out = f.mapM3 + size_t(y) * f.w + x0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                      if (!((bits >> i) & 1u)) continue;
                      const float a = max3f(lo[i], lo[i + 1], lo[i + 2]);
                      const float b = fmaxf(fminf(mi[i], mi[i + 1]), fminf(fmaxf(mi[i], mi[i + 1]), mi[i + 2]));
                      const float c = min3f(hi[i], hi[i + 1], hi[i + 2]);
                      out[i] = fmaxf(fminf(a, b), fminf(fmaxf(a, b), c));
                    }
                  });
}

// bound_sparse_kernel (iteration >= 2): the bound test of the pixels listed in
// q2 (within 2 px of a change), by groups of four pixels x .. x+3 that hold a
// listed one: one thread forms the column medians of the eight columns x-2 ..
// x+5 (rows and columns clamped at the frame's edges, as in the dense pass),
// then per pixel the minimum of five of them and L+: the dense pass's
// values. The whole group is rewritten (an unlisted pixel gets the value it
// holds, its window being unchanged). A group's bits belong to it alone during
// the kernel, so the thread reads the plane words and XORs in only the bits
// that changed, with no atomic where none did (most re-tests change nothing);
// XORs of disjoint bits by other groups of the word commute with it.
__global__ void __launch_bounds__(256, 4) bound_sparse_kernel(const Frame* __restrict__ frames, int nframes, Queues Q,
                                                           Params p) {
  expand_words<4, true>(frames, nframes, reinterpret_cast<const uint2*>(Q.q2), Q.n[kNB],
                  [&](bool valid, int fi, int x0, int y, uint32_t) {
                    if (!valid) return;
                    const Frame& f = frames[fi];
                    const int w = f.w, h = f.h;
                    float v[5][8];  // rows y-2 .. y+2, columns x0-2 .. x0+5
                    load_span<2>(f.out_clean, x0, y, w, h, v);
                    float cm[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                      const float col[5] = {v[0][c], v[1][c], v[2][c], v[3][c], v[4][c]};
                      cm[c] = sel_med5(col);
                    }
                    const float gain = f.gain, rn2 = __fmul_rn(f.rn, f.rn), kl = f.bkl, kh = f.bkh;
                    uint32_t hb = 0, ab = 0, zb = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                      const float mlow = min3f(min3f(cm[i], cm[i + 1], cm[i + 2]), cm[i + 3], cm[i + 4]);
                      const float lp = lplus(v[2][i + 2], v[1][i + 2], v[3][i + 2], v[2][i + 1], v[2][i + 3]);
                      bool act, hot;
                      bound_test(lp, mlow, gain, rn2, kl, kh, act, hot);
                      ab |= uint32_t(act) << i;
                      hb |= uint32_t(hot) << i;
                      zb |= uint32_t(lp == 0.f) << i;
                    }
                    const int sh = x0 & 31;
                    const uint32_t gm = (15u << sh) & frame_word(x0 >> 5, w);
                    const size_t wo = size_t(y) * f.wpr + (x0 >> 5);
                    const uint32_t dh = (f.hot[wo] ^ (hb << sh)) & gm, da = (f.act[wo] ^ (ab << sh)) & gm,
                                   dz = (f.lpz[wo] ^ (zb << sh)) & gm;
                    if (dh) atomicXor(f.hot + wo, dh);
                    if (da) atomicXor(f.act + wo, da);
                    if (dz) atomicXor(f.lpz + wo, dz);
                  });
}

// The objlim test of candidate c: S'(c) / max(F/N, 0.01) > objlim (article
// form: 2S(c) / max(F/N, 0.01)), F = m3(c) - med7(m3)(c). Every operation is
// monotone (IEEE rounding is monotone; N > 0, and S, S' > 0 at a test
// position), so a lower bound of med7 gives an upper bound of F and a lower
// bound of the statistic, and vice versa.
__device__ __forceinline__ float objlim_stat(const Params& p, float fval, float nn, float s, float sp) {
  const float fn = fmaxf(__fdiv_rn(fval, nn), 0.01f);
  return (p.objlim_form == 1) ? __fdiv_rn(__fmul_rn(2.f, s), fn) : __fdiv_rn(sp, fn);
}

// Rows y-3 .. y+3 and columns x0-3 .. x0+4 of a (clamped at the frame's
// edges, as load_window) for a pair of pixels, x0 even: away from the edges,
// three aligned 8-byte loads and two 4-byte loads per row.
__device__ __forceinline__ void load_pair_span7(const float* __restrict__ a, int x0, int y, int w, int h,
                                                float (&v)[7][8]) {
  const bool vec = x0 >= 4 && x0 + 5 <= w && (w & 1) == 0 && (reinterpret_cast<uintptr_t>(a) & 7u) == 0;
#pragma unroll
  for (int dy = 0; dy < 7; ++dy) {
    const float* __restrict__ r = a + size_t(clampi(y - 3 + dy, 0, h - 1)) * size_t(w);
    if (vec) {
      const float2 B = __ldg(reinterpret_cast<const float2*>(r + x0 - 2));
      const float2 C = __ldg(reinterpret_cast<const float2*>(r + x0));
      const float2 D = __ldg(reinterpret_cast<const float2*>(r + x0 + 2));
      v[dy][0] = __ldg(r + x0 - 3);
      v[dy][1] = B.x, v[dy][2] = B.y, v[dy][3] = C.x, v[dy][4] = C.y, v[dy][5] = D.x, v[dy][6] = D.y;
      v[dy][7] = __ldg(r + x0 + 4);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) v[dy][c] = __ldg(r + clampi(x0 - 3 + c, 0, w - 1));
    }
  }
}

// cand_test_kernel: at QT, the 7 column medians of the 7x7 window of m3; at
// most 3 values of a column lie below (above) its median, so at most 21 of 49
// lie below the smallest (above the largest) column median, which bound
// med7(m3) from below (above). Tests the bounds decide go to the candidates
// (pass; in iteration 1 the candidate plane) or are dropped; the rest to the
// open tests. By aligned pairs x0, x0+1 holding a listed test: the pair's
// windows share six of their eight columns, each loaded and sorted once.
// Three blocks per SM (80 registers, 68 B of spills) measured 2 % faster than
// two (102 registers).
__global__ void __launch_bounds__(256, 3) cand_test_kernel(const Frame* __restrict__ frames, int nframes, Queues Q,
                                                           Params p, int k) {
  __shared__ WarpLists<2, 128> wl;
  wl.init();
  uint32_t* const lists[2] = {Q.q0, Q.q1};
  expand_words<2, true>(frames, nframes, reinterpret_cast<const uint2*>(Q.q2), Q.n[kNT],
                  [&](bool valid, int fi, int x0, int y, uint32_t bits) {
                    bool pass[2] = {false, false}, open[2] = {false, false};
                    uint32_t g = 0;
                    if (valid) {
                      const Frame& f = frames[fi];
                      const size_t o = size_t(y) * f.w + x0;
                      g = uint32_t(f.pix0 + (long long)o);
                      // only the statistic's numerator is loaded: 2S (article form) or S'
                      const bool form1 = p.objlim_form == 1;
                      float nn[2], sv[2], spv[2];
#pragma unroll
                      for (int i = 0; i < 2; ++i) {
                        const bool on = (bits >> i) & 1u;
                        nn[i] = on ? f.mapN[o + i] : 1.f;
                        sv[i] = (on && form1) ? f.mapS[o + i] : 0.f;
                        spv[i] = (on && !form1) ? f.mapSp[o + i] : 0.f;
                      }
                      float v[7][8], cm[8];
                      load_pair_span7(f.mapM3, x0, y, f.w, f.h, v);
#pragma unroll
                      for (int c = 0; c < 8; ++c) {
                        float col[7];
#pragma unroll
                        for (int dy = 0; dy < 7; ++dy) col[dy] = v[dy][c];
                        cm[c] = sel_med7(col);
                      }
                      float lo = cm[1], hi = cm[1];  // the shared columns 1 .. 6
#pragma unroll
                      for (int c = 2; c < 7; ++c) lo = fminf(lo, cm[c]), hi = fmaxf(hi, cm[c]);
                      const float los[2] = {fminf(lo, cm[0]), fminf(lo, cm[7])};
                      const float his[2] = {fmaxf(hi, cm[0]), fmaxf(hi, cm[7])};
                      uint32_t cb = 0;
#pragma unroll
                      for (int i = 0; i < 2; ++i) {
                        if (!((bits >> i) & 1u)) continue;
                        const float mc = v[3][3 + i];
                        // F at its largest, then at its smallest
                        const float rlow = objlim_stat(p, __fsub_rn(mc, los[i]), nn[i], sv[i], spv[i]);
                        const float rhigh = objlim_stat(p, __fsub_rn(mc, his[i]), nn[i], sv[i], spv[i]);
                        pass[i] = rlow > p.objlim;
                        open[i] = !pass[i] && rhigh > p.objlim;
                        cb |= uint32_t(pass[i]) << i;
                      }
                      if (k == 1 && cb) atomicOr(&f.cand[size_t(y) * f.wpr + (x0 >> 5)], cb << (x0 & 31));
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                      const bool put[2] = {pass[i] && k != 1, open[i]};  // iteration 1: candidates as bits
                      wl.put(put, g + uint32_t(i), lists, Q.n + kNPass);
                    }
                  });
  wl.flush(lists, Q.n + kNPass);
}

// cand_full_kernel: at the open tests, the exact F = m3 - med7(m3) and the
// objlim test -> candidates.
__global__ void __launch_bounds__(256) cand_full_kernel(const Frame* __restrict__ frames, int nframes, Queues Q,
                                                        Params p, int k) {
  __shared__ WarpLists<1, 128> wl;
  wl.init();
  uint32_t* const lists[1] = {Q.q0};
  const unsigned int n = Q.n[kNAmb];
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // whole warps iterate together
    const unsigned int i = i0 + threadIdx.x;
    bool pass = false;
    uint32_t g = 0;
    if (i < n) {
      g = Q.q1[i];
      const Pix P = decode(frames, nframes, Q, g);
      const Frame& f = frames[P.fi];
      float u[49];
      load_window<3>(f.mapM3, P.x, P.y, f.w, f.h, u);
      const size_t o = size_t(g - uint32_t(f.pix0));
      const float fval = __fsub_rn(u[24], sel_med49(u));
      const bool form1 = p.objlim_form == 1;  // only the numerator is loaded: 2S, else S'
      pass = objlim_stat(p, fval, f.mapN[o], form1 ? f.mapS[o] : 0.f, form1 ? 0.f : f.mapSp[o]) > p.objlim;
      if (k == 1 && pass) atomicOr(&f.cand[size_t(P.y) * f.wpr + (P.x >> 5)], 1u << (P.x & 31));
    }
    const bool put[1] = {pass && k != 1};  // iteration 1: candidates as bits
    wl.put(put, g, lists, Q.n + kNPass);
  }
  wl.flush(lists, Q.n + kNPass);
}

// grow_first_kernel (iteration 1): both growths as bit-plane algebra,
// M_1 = dilate3(dilate3(cand) & T) & L, where T (the test plane) holds
// S' > sigclip and L (low) S' > sigfrac*sigclip, both set by sp_kernel at the
// nsp pixels (the only pixels whose S' can pass either threshold), and cand
// the candidates. This is the union of every candidate's growth (the 3x3 of
// T around it, then the 3x3 of L around those). One warp per strip (lane =
// word) walks rows y0-2 .. y0+kSH+1; lanes 0 and 31 also form the words beyond
// the strip. Writes M_1 (no flag exists before: the queue pipeline takes no
// explicit previous mask), counts it per frame, and queues its pixels for the
// replacement, all of them being new.
__global__ void __launch_bounds__(kColWarps * 32) grow_first_kernel(const Frame* __restrict__ frames, int nframes,
                                                                    long long nunits, Queues Q) {
  __shared__ ColWords sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long u = (long long)blockIdx.x * kColWarps + warp; u < nunits; u += (long long)gridDim.x * kColWarps) {
    const Frame& f = frames[frame_of_unit(frames, nframes, u)];
    const long long lu = u - f.u0;
    const int uy = int(lu / f.ugx), ux = int(lu - (long long)uy * f.ugx);
    const int wc0 = ux * 32, y0 = uy * kSH, wc = wc0 + lane;
    const bool inw = wc < f.wpr;
    const int hw = lane == 0 ? wc0 - 1 : wc0 + 32;  // the word beyond the strip (lanes 0 and 31)
    const bool hin = (lane == 0 || lane == 31) && hw >= 0 && hw < f.wpr;
    const uint32_t fmask = inw ? frame_word(wc, f.w) : 0u;
    uint32_t c0 = 0, c1 = 0, c2 = 0, e0 = 0, e1 = 0, e2 = 0;  // cand, rows r-2 .. r (own, beyond)
    uint32_t tp = 0, etp = 0;                                  // T of row r-1 (own, beyond)
    uint32_t a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;  // g1, rows r-3 .. r-1 (own, beyond)
    uint32_t l0 = 0, l1 = 0, l2 = 0;                           // L, rows r-2 .. r (own)
    unsigned int cnt = 0;
    for (int r = y0 - 2; r < y0 + kSH + 2; ++r) {
      const bool rin = r >= 0 && r < f.h;
      const size_t ro = size_t(rin ? r : 0) * f.wpr;
      const uint32_t cr = (rin && inw) ? f.cand[ro + wc] : 0u, er = (rin && hin) ? f.cand[ro + hw] : 0u;
      const uint32_t tr = (rin && inw) ? f.test[ro + wc] : 0u, etr = (rin && hin) ? f.test[ro + hw] : 0u;
      const uint32_t lr = (rin && inw) ? f.low[ro + wc] : 0u;
      c0 = c1; c1 = c2; c2 = cr;
      e0 = e1; e1 = e2; e2 = er;
      l0 = l1; l1 = l2; l2 = lr;
      // g1 of row r-1
      const uint32_t vc = c0 | c1 | c2, evc = e0 | e1 | e2;
      uint32_t left = __shfl_up_sync(0xffffffffu, vc, 1), right = __shfl_down_sync(0xffffffffu, vc, 1);
      if (lane == 0) left = evc;
      if (lane == 31) right = evc;
      const uint32_t g1 = hdil<1>(left, vc, right) & tp;
      const uint32_t eg1 = (lane == 0 ? hdil<1>(0u, evc, vc) : hdil<1>(vc, evc, 0u)) & etp;
      tp = tr;
      etp = etr;
      a0 = a1; a1 = a2; a2 = g1;
      b0 = b1; b1 = b2; b2 = eg1;
      // M_1 of row r-2
      const int yo = r - 2;
      if (yo < y0) continue;  // whole warp
      const uint32_t vg = a0 | a1 | a2, evg = b0 | b1 | b2;
      uint32_t gl = __shfl_up_sync(0xffffffffu, vg, 1), gr = __shfl_down_sync(0xffffffffu, vg, 1);
      if (lane == 0) gl = evg;
      if (lane == 31) gr = evg;
      const uint32_t m = (yo < f.h) ? (hdil<1>(gl, vg, gr) & l0 & fmask) : 0u;
      if (yo < f.h && inw) f.bits_a[size_t(yo) * f.wpr + wc] = m;
      sw.w[warp][yo - y0][0][lane] = m;
      cnt += unsigned(__popc(m));
    }
    // the strip's flags: one count per frame, then the replacement queue, one atomic per warp
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0;
    if (lane == 0 && total) {
      base = atomicAdd(Q.n + kNRep, total);
      atomicAdd(f.counters + 0, (unsigned long long)total);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    unsigned int o = base + incl - cnt;
    if (inw) {
      for (int rr = 0; rr < kSH; ++rr) {
        uint32_t v = sw.w[warp][rr][0][lane];
        const uint32_t row = uint32_t(f.pix0 + (long long)(y0 + rr) * f.w + 32 * wc);
        while (v) {
          const int bb = __ffs(v) - 1;
          v &= v - 1u;
          Q.q1[o++] = row + bb;
        }
      }
    }
    __syncwarp();  // the shared words are refilled for the next strip
  }
}

// grow_kernel (iterations 2 on): for each candidate c, the first growth g1
// (S' > sigclip in the 3x3 around c) and the second (S' > sigfrac*sigclip in
// the 3x3 around g1), as bit masks over the 5x5 around c, ORed into the flag
// bits of M_k; counts the new flags of each frame and lists them. S' is read
// only where the bit plane nsp says it is current; elsewhere it cannot pass
// either threshold.
__global__ void __launch_bounds__(256, 4) grow_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, Params p,
                                                   int k) {
  const unsigned int n = Q.n[kNPass];
  const float sigclip = p.sigclip, siglow = __fmul_rn(p.sigfrac, p.sigclip);
  const unsigned int stride = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (unsigned int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // whole warps iterate together
    const unsigned int i = i0 + threadIdx.x;
    uint32_t fm = 0;  // new flags, bit (dy+2)*5 + (dx+2)
    uint32_t g = 0;
    int w = 1;
    if (i < n) {
      g = Q.q0[i];
      const Pix P = decode(frames, nframes, Q, g);
      const Frame& f = frames[P.fi];
      w = f.w;
      const int h = f.h;
      // the 5x5 around c: nsp bits and S' values, loaded without dependencies
      // (clamped; out-of-frame positions are masked)
      const int xs = P.x - 2;                      // first column of the 5x5
      const int wl = max(xs, 0) >> 5, wr = min(P.x + 2, w - 1) >> 5;
      int cx[5];
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) cx[dx] = clampi(xs + dx, 0, w - 1);
      uint32_t nb[5];
      float sv[5][5];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const size_t qy = size_t(clampi(P.y + r - 2, 0, h - 1));
        const uint64_t pair = uint64_t(f.nsp[qy * f.wpr + wl]) | (uint64_t(f.nsp[qy * f.wpr + wr]) << 32);
        // bit dx = nsp at column xs + dx (columns left of the frame read as 0 below)
        const int sh = xs - 32 * wl;  // in [-2, 31]
        nb[r] = uint32_t(sh >= 0 ? (pair >> sh) : (pair << -sh)) & 31u;
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) sv[r][dx] = f.mapSp[qy * w + cx[dx]];
      }
      uint32_t inx = 0;  // columns inside the frame
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) inx |= (xs + dx >= 0 && xs + dx < w) ? (1u << dx) : 0u;
      uint32_t A = 0, B = 0;  // S' > sigclip (3x3), S' > sigfrac*sigclip (5x5)
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const bool rowin = P.y + r - 2 >= 0 && P.y + r - 2 < h;
        const uint32_t ok = rowin ? (nb[r] & inx) : 0u;
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) {
          const bool valid = (ok >> dx) & 1u;
          const int bb = r * 5 + dx;
          if (valid && sv[r][dx] > siglow) B |= 1u << bb;
          if (valid && r >= 1 && r <= 3 && dx >= 1 && dx <= 3 && sv[r][dx] > sigclip) A |= 1u << bb;
        }
      }
      // 3x3 dilation of A (inside the inner 3x3, so no shift leaves the 5x5)
      const uint32_t dA = A | (A << 1) | (A >> 1) | (A << 5) | (A >> 5) | (A << 4) | (A >> 4) | (A << 6) | (A >> 6);
      const uint32_t g2 = dA & B;
      // OR each row's flags into its (at most two) flag words: the row's 5 bits
      // shifted to the word of its lowest flag (sh in [-4, 31])
      uint32_t* wp[5];
      uint64_t mm[5];
      int sh[5];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const uint32_t m = (g2 >> (5 * r)) & 31u;
        const int w0 = m ? (xs + __ffs(m) - 1) >> 5 : 0;
        sh[r] = xs - 32 * w0;
        mm[r] = sh[r] >= 0 ? (uint64_t(m) << sh[r]) : (uint64_t(m) >> -sh[r]);
        wp[r] = f.bits_a + size_t(clampi(P.y + r - 2, 0, h - 1)) * f.wpr + w0;
      }
      {
        uint32_t old[5][2];
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint32_t part = uint32_t(mm[r] >> (32 * j));
            old[r][j] = part ? atomicOr(wp[r] + j, part) : 0u;
          }
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          const uint64_t fresh = mm[r] & ~(uint64_t(old[r][0]) | (uint64_t(old[r][1]) << 32));
          fm |= (uint32_t(sh[r] >= 0 ? (fresh >> sh[r]) : (fresh << -sh[r])) & 31u) << (5 * r);
        }
        if (fm) atomicAdd(f.counters + 2 * (k - 1), (unsigned long long)__popc(fm));
      }
    }
    {  // list the new flags: one atomic per warp
      const int c = __popc(fm);
      int x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      const int total = __shfl_sync(0xffffffffu, x, 31);
      if (total) {
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(Q.n + kNFresh, (unsigned int)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        unsigned int out = base + unsigned(x - c);
        while (fm) {
          const int bb = __ffs(fm) - 1;
          fm &= fm - 1u;
          // g + (dy * w + dx), with the new flag inside the frame
          Q.fresh[out++] = uint32_t(int64_t(g) + (long long)(bb / 5 - 2) * w + (bb % 5 - 2));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Replacement (stage e).

// ORs a 5x5 mask (bit r*5 + dx = column xs + dx of row y0 + r; only in-frame
// positions set) into a bit plane, one atomic per row and word, and returns the
// bits that were clear before.
__device__ __forceinline__ uint32_t or_window(uint32_t* plane, int wpr, int h, int xs, int y0, uint32_t m25) {
  uint32_t* wp[5];
  uint64_t mm[5];
  int sh[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const uint32_t m = (m25 >> (5 * r)) & 31u;
    const int w0 = m ? (xs + __ffs(m) - 1) >> 5 : 0;  // word of the row's first bit
    sh[r] = xs - 32 * w0;                            // in [-4, 31]
    mm[r] = sh[r] >= 0 ? (uint64_t(m) << sh[r]) : (uint64_t(m) >> -sh[r]);
    wp[r] = plane + size_t(clampi(y0 + r, 0, h - 1)) * wpr + w0;
  }
  uint32_t old[5][2];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t part = uint32_t(mm[r] >> (32 * j));
      old[r][j] = part ? atomicOr(wp[r] + j, part) : 0u;
    }
  uint32_t res = 0;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const uint64_t fresh = mm[r] & ~(uint64_t(old[r][0]) | (uint64_t(old[r][1]) << 32));
    res |= (uint32_t(sh[r] >= 0 ? (fresh >> sh[r]) : (fresh << -sh[r])) & 31u) << (5 * r);
  }
  return res;
}

// rq_kernel (iteration >= 2): the flagged pixels within 2 px of a new flag
// (their windows gained a flag) and every pixel with a fully flagged window (J
// may have changed in it) -> the replacement queue, each once (bit plane rq;
// one append atomic per block).
__global__ void __launch_bounds__(256) rq_kernel(const Frame* __restrict__ frames, int nframes, Queues Q) {
  __shared__ int ws[kThreads / 32 + 1];
  __shared__ unsigned int sbase;
  const unsigned int nf = Q.n[kNFresh], n = nf + Q.n[kNFb];
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // whole blocks iterate together
    const unsigned int i = i0 + threadIdx.x;
    uint32_t nq = 0;  // newly queued, bit (dy+2)*5 + (dx+2) around the entry
    uint32_t g = 0;
    int w = 1;
    if (i < n) {
      const bool is_fresh = i < nf;
      g = is_fresh ? Q.fresh[i] : Q.fbl[i - nf];
      const Pix P = decode(frames, nframes, Q, g);
      const Frame& f = frames[P.fi];
      w = f.w;
      uint32_t want = 1u << 12;  // the pixel itself (fully flagged window)
      if (is_fresh) {           // the flagged pixels of the 5x5
        want = 0;
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          const int qy = P.y + r - 2;
          if (qy >= 0 && qy < f.h) want |= plane_bits5(f.bits_a, f.wpr, f.w, P.x - 2, qy) << (5 * r);
        }
      }
      nq = or_window(f.rq, f.wpr, f.h, P.x - 2, P.y - 2, want);
    }
    int total = 0;
    const int off = block_excl_scan(__popc(nq), ws, total);
    if (threadIdx.x == 0) sbase = total ? atomicAdd(Q.n + kNRep, (unsigned int)total) : 0u;
    __syncthreads();
    unsigned int out = sbase + unsigned(off);
    while (nq) {
      const int bb = __ffs(nq) - 1;
      nq &= nq - 1u;
      Q.q1[out++] = uint32_t(int64_t(g) + (long long)(bb / 5 - 2) * w + (bb % 5 - 2));
    }
    __syncthreads();
  }
}

// Marks a change at (x, y) for iteration knext: its bit in the changed-pixel
// plane, and in the cell classes `cls` the cells it reaches: class 4 within
// 2 px, 3 within 4 px, 2 within 6 px (distance to the cell's rectangle,
// Chebyshev).
__device__ __forceinline__ void mark_change(const Frame& f, int x, int y, uint32_t* cls, int knext) {
  atomicOr(f.chg[knext & 1] + size_t(y) * f.wpr + (x >> 5), 1u << (x & 31));
  const int cx0 = max(x - 6, 0) >> 5, cx1 = min(x + 6, f.w - 1) >> 5;
  const int cy0 = max(y - 6, 0) / kCH, cy1 = min(y + 6, f.h - 1) / kCH;
  for (int cy = cy0; cy <= cy1; ++cy)
    for (int cx = cx0; cx <= cx1; ++cx) {
      const int dx = max(0, max(32 * cx - x, x - (32 * cx + 31)));
      const int dy = max(0, max(kCH * cy - y, y - (kCH * cy + kCH - 1)));
      const int d = max(dx, dy);
      const uint32_t cl = d <= 2 ? 4u : d <= 4 ? 3u : d <= 6 ? 2u : 0u;
      if (!cl) continue;
      uint32_t* p = cls + f.cell0 + (long long)cy * f.wpr + cx;
      if (*p < cl) atomicMax(p, cl);
    }
}

// rep_compute_kernel: I_k at the queued pixels, from J = I_{k-1} and M_k, into
// the side array q0 (nothing is written to the image yet). A pixel whose
// window is fully flagged is counted and, the first time, listed. In
// iteration 1, J = I0 is not the image buffer, so the values go to the buffer
// directly (`cls_next`: cell classes to mark, or nullptr).
__global__ void __launch_bounds__(256) rep_compute_kernel(const Frame* __restrict__ frames, int nframes, Queues Q,
                                                          int k, uint32_t* cls_next) {
  const unsigned int n = Q.n[kNRep];
  float* __restrict__ vals = reinterpret_cast<float*>(Q.q0);
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q1[i];
    const Pix P = decode(frames, nframes, Q, g);
    const Frame& f = frames[P.fi];
    const float* __restrict__ J = qsrc(f, k);
    float v[25];
    load_window<2>(J, P.x, P.y, f.w, f.h, v);
    uint32_t win = 0;  // 25 window flags, row-major, of the clamped window
    if (P.x >= 2 && P.x < f.w - 2) {
#pragma unroll
      for (int dy = 0; dy < 5; ++dy)
        win |= plane_bits5(f.bits_a, f.wpr, f.w, P.x - 2, clampi(P.y - 2 + dy, 0, f.h - 1)) << (5 * dy);
    } else {
#pragma unroll
      for (int dy = 0; dy < 5; ++dy) {
        const size_t ro = size_t(clampi(P.y - 2 + dy, 0, f.h - 1)) * f.wpr;
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) {
          const int xx = clampi(P.x - 2 + dx, 0, f.w - 1);
          win |= ((f.bits_a[ro + (xx >> 5)] >> (xx & 31)) & 1u) << (dy * 5 + dx);
        }
      }
    }
    const int nu = 25 - __popc(win);
    float out;
    if (nu > 0) {
      const int a = 13 - (nu + 1) / 2;  // flagged entries sent to -inf
      int seen = 0;
#pragma unroll
      for (int q = 0; q < 25; ++q)
        if ((win >> q) & 1u) {
          v[q] = (seen < a) ? -INFINITY : INFINITY;
          ++seen;
        }
      out = sel_med25(v);
    } else {
      out = floor_m5(sel_med25(v));
      atomicAdd(f.counters + 2 * (k - 1) + 1, 1ull);
      const size_t wo = size_t(P.y) * f.wpr + (P.x >> 5);
      const uint32_t bit = 1u << (P.x & 31);
      if (!(f.fb[wo] & bit) && !(atomicOr(&f.fb[wo], bit) & bit)) group_append(g, Q.fbl, Q.n + kNFb);
    }
    if (k == 1) {
      const size_t o = size_t(g - uint32_t(f.pix0));
      f.out_clean[o] = out;
      if (cls_next && __float_as_uint(out) != __float_as_uint(J[o])) mark_change(f, P.x, P.y, cls_next, k + 1);
    } else {
      vals[i] = out;
    }
  }
}

// rep_write_kernel: writes the computed values in place; a changed value marks
// the cells of the next iteration (cls_next, or nothing after the last one).
// Clears the queued bits.
__global__ void __launch_bounds__(256) rep_write_kernel(const Frame* __restrict__ frames, int nframes, Queues Q,
                                                        uint32_t* cls_next, int knext, int clear_rq) {
  const unsigned int n = Q.n[kNRep];
  const float* __restrict__ vals = reinterpret_cast<const float*>(Q.q0);
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q1[i];
    const Pix P = decode(frames, nframes, Q, g);
    const Frame& f = frames[P.fi];
    const size_t o = size_t(g - uint32_t(f.pix0));
    const float v = vals[i];
    if (__float_as_uint(f.out_clean[o]) != __float_as_uint(v)) {
      f.out_clean[o] = v;
      if (cls_next) mark_change(f, P.x, P.y, cls_next, knext);
    }
    if (clear_rq) atomicAnd(&f.rq[size_t(P.y) * f.wpr + (P.x >> 5)], ~(1u << (P.x & 31)));
  }
}

// mask_kernel: the u8 mask of every frame from its flag bits (one word per
// thread; two 16-byte stores when the 32 bytes are aligned).
__device__ __forceinline__ uint32_t nibble_bytes(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

__global__ void __launch_bounds__(256) mask_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks) {
  const int t = threadIdx.x;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int y = bys * kBH + t / kBW, wc = bxs * kBW + t % kBW;
    if (y >= f.h || wc >= f.wpr || !f.out_mask) continue;
    const uint32_t v = f.bits_a[size_t(y) * f.wpr + wc];
    uint8_t* o = f.out_mask + size_t(y) * f.w + 32 * wc;
    const int nb = min(32, f.w - 32 * wc);
    if (nb == 32 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
      uint4 q0, q1;
      q0.x = nibble_bytes(v & 15u);
      q0.y = nibble_bytes((v >> 4) & 15u);
      q0.z = nibble_bytes((v >> 8) & 15u);
      q0.w = nibble_bytes((v >> 12) & 15u);
      q1.x = nibble_bytes((v >> 16) & 15u);
      q1.y = nibble_bytes((v >> 20) & 15u);
      q1.z = nibble_bytes((v >> 24) & 15u);
      q1.w = nibble_bytes(v >> 28);
      reinterpret_cast<uint4*>(o)[0] = q0;
      reinterpret_cast<uint4*>(o)[1] = q1;
    } else {
      for (int bb = 0; bb < nb; ++bb) o[bb] = uint8_t((v >> bb) & 1u);
    }
  }
}

// Adds the queue lengths of iteration k to the work counters of frame 0 (the
// totals of the call) and clears the per-iteration counters. Bound tests:
// `dense` positions in iteration 1, the re-tested pixels after it.
__global__ void queue_work_kernel(const Frame* __restrict__ frames, Queues Q, int k, long long dense) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long* wk = frames[0].work + kWork * (k - 1);
    wk[0] += Q.n[kNSpx];
    wk[1] += Q.n[kNSPpx];
    wk[2] += Q.n[kNM3px];
    wk[3] += Q.n[kNTpx];
    wk[4] += Q.n[kNAmb];
    wk[5] += (k == 1) ? (unsigned long long)dense : (unsigned long long)Q.n[kNBpx];
    for (int i = 0; i < kNCount; ++i)
      if (i != kNFb) Q.n[i] = 0u;
  }
}

}  // namespace crb
