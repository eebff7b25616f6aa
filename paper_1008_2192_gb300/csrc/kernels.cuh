// CUDA kernels of one L.A.Cosmic iteration (van Dokkum 2001; the work
// function of CRBLASTER, Mighell 2010, Sec. 5) for sm_103a.
//
// detect  : stages (a)-(d) on an output tile plus a 6-pixel halo staged in
//           shared memory. 6 is the dependency radius of the new flags on the
//           input (S' and F need 4, the two growths add 2), the same as the
//           overlap CRBLASTER gives its sub-images (BORDER = 6, Sec. 6.2).
//           The staged region is the tile plus 8 pixels (the fused form needs
//           them for the replacement in front): one TMA box for a tile inside
//           the frame, clamped 4-byte copies at the frame's edges.
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
#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>

#include "networks.cuh"

namespace crb {

constexpr int kThreads = 256;
constexpr int kNumMaps = 11;  // m5, L+, N, S, S', m3, F, R, cand, g1, g2
// work counters per iteration: positions given S, S', med3, a candidate test,
// the full 7x7 median of that test, and the bound test
constexpr int kWork = 6;

// One frame of a launch. In the tile pipeline the image buffers alternate
// between iterations so that iteration niter writes out_clean: I_k goes to
// out_clean when (niter - k) is even and to ws otherwise; iteration 1 reads
// img. The queue pipeline (pipeline.cuh) replaces in place in out_clean.
struct Frame {
  const float* img;       // I_0 (input, read-only)
  float* out_clean;       // caller's output
  float* ws;              // workspace image of the same size
  uint32_t* bits_a;       // cumulative flags M_k, bit x&31 of word [y*wpr + x/32]: in bits_a
  uint32_t* bits_b;       // for odd k, in bits_b for even k (M_0 = bits_b); equal pointers
                          // update the flags in place (detection and replacement as two launches)
  uint8_t* out_mask;      // caller's 0/1 mask, written by the last replacement
  float* maps;            // kNumMaps debug maps (crb_iterate) or nullptr
  unsigned long long* counters;  // 2 per iteration: new flags, no-unflagged-neighbour pixels
  unsigned long long* work;      // nullable; kWork per iteration (see kWork)
  int w, h, wpr;
  float gain, rn;
  int tiles_x, rtiles_x;  // detect / replace tiles per row of tiles
  long long tile0, rtile0;  // first tile index of this frame in the launch
  // tile pipeline: tensor maps of img, out_clean and ws (one box of the image
  // region of a detection tile each) for TMA loads of interior tiles, or
  // nullptr (every tile then loads element by element)
  const CUtensorMap* tmap;
  unsigned int* status;   // device status word of the call (nonzero: a bounded wait gave up)
  // tile pipeline: the replacements of iterations up to dense_upto write their
  // whole tile (the first write into each image buffer must), later ones only
  // the flagged pixels; from iteration flip_from on, the flag planes of odd and
  // even iterations swap (after a launch that fused two iterations)
  int dense_upto, flip_from;
  // queue pipeline (pipeline.cuh): bit planes (flag-word layout) and float maps
  uint32_t *hot, *act, *nsp, *test;
  uint32_t *sval, *m3val;  // positions whose mapS/mapN, mapM3 hold the current iteration's values
  uint32_t* lpz;           // L+ == 0 (then S == 0 exactly, and no median is needed)
  uint32_t *cand, *low;    // iteration 1: candidates; S' > sigfrac*sigclip (at the nsp pixels)
  float bkl, bkh;          // bound test thresholds over gain^2 (bound_thresholds)
  uint32_t *rq, *fb;       // queued for replacement; known to have a fully flagged window
  uint32_t* chg[2];        // pixels the replacement changed, for even / odd next iterations
  float *mapS, *mapN, *mapSp, *mapM3;
  long long pix0;  // first global pixel index of this frame
  long long blk0;  // first word block (kBW words x kBH rows) of this frame
  long long cell0; // first cell (one word x kCH rows) of this frame
  int bx;          // word blocks per row of blocks
  int ncy;         // rows of cells
  long long u0;    // first strip (32 words x kSH rows) of this frame
  long long word0; // first word (32 px of a row) of this frame
  int ugx;         // strips per row of strips
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

__device__ __forceinline__ uint32_t* mask_bits(const Frame& f, int k) {
  return ((k & 1) != (k >= f.flip_from ? 1 : 0)) ? f.bits_a : f.bits_b;
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
// The clip max(0, t) is taken as t + |t| = 2 max(0, t), exact for finite t
// below FLT_MAX/2 (an add with an operand modifier instead of a min/max
// instruction); the doubled partial sums round exactly as the plain ones, so
// 1/8 of their sum equals 1/4 of the sum of the clips in every bit.
// L+ from the four differences dn = c - up, ds = c - down, dw = c - left,
// de = c - right. A difference that is the negation of another (c(i) - c(i+1)
// = -(c(i+1) - c(i)) exactly) may differ from it only in the sign of a zero,
// which the clipping t + |t| removes, so callers may share differences
// between neighbours and get the same value.
__device__ __forceinline__ float lplus_d(float dn, float ds, float dw, float de) {
  const float t0 = __fadd_rn(dn, dw), t1 = __fadd_rn(dn, de), t2 = __fadd_rn(ds, dw), t3 = __fadd_rn(ds, de);
  float acc = __fadd_rn(t0, fabsf(t0));
  acc = __fadd_rn(acc, __fadd_rn(t1, fabsf(t1)));
  acc = __fadd_rn(acc, __fadd_rn(t2, fabsf(t2)));
  acc = __fadd_rn(acc, __fadd_rn(t3, fabsf(t3)));
  return __fmul_rn(0.125f, acc);
}
__device__ __forceinline__ float lplus(float c, float up, float down, float left, float right) {
  return lplus_d(__fsub_rn(c, up), __fsub_rn(c, down), __fsub_rn(c, left), __fsub_rn(c, right));
}

// (b) floored 5x5 median -> noise N.
__device__ __forceinline__ float floor_m5(float m5) { return m5 <= 0.f ? 1e-4f : m5; }
__device__ __forceinline__ float noise_of(float m5f, float gain, float rn2) {
  return __fdiv_rn(__fsqrt_rn(__fadd_rn(__fmul_rn(gain, m5f), rn2)), gain);
}

// --------------------------------------------------------------------------------------------
// Appends idx to a shared-memory list when pred holds (warp-aggregated). Every
// lane of the warp must call it: loops that use it are padded to whole blocks.
__device__ __forceinline__ void push_if(bool pred, int idx, uint16_t* list, int* count) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = uint16_t(idx);
}

__host__ __device__ constexpr int round16(int b) { return (b + 15) / 16 * 16; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

// --------------------------------------------------------------------------------------------
// Bit-row maps: one bit per pixel, word j of a row covers x0 - 32 + 32j ... + 31,
// rows are the rows of R6 (y0 - 6 ...). x0 is a multiple of 32.

// bits [lo, hi) of a word, clipped to [0, 32)
__device__ __forceinline__ uint32_t bits_between(int lo, int hi) {
  lo = max(lo, 0);
  hi = min(hi, 32);
  if (lo >= hi) return 0u;
  const uint32_t m = (hi == 32) ? 0xffffffffu : ((1u << hi) - 1u);
  return m & ~((1u << lo) - 1u);
}

// Exclusive prefix sum over the block (one value per thread); ws holds kThreads/32 + 1 ints.
__device__ __forceinline__ int block_excl_scan(int v, int* ws, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kThreads / 32;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int s = lane < kWarps ? ws[lane] : 0;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < kWarps) ws[lane] = inc - s;
    if (lane == kWarps - 1) ws[kWarps] = inc;
  }
  __syncthreads();
  total = ws[kWarps];
  const int r = ws[warp] + x - v;
  __syncthreads();
  return r;
}

// 4-byte asynchronous global -> shared copy (completion: cp_async_wait_all + barrier)
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// TMA (cp.async.bulk.tensor) with an mbarrier: a box of a tensor map into
// shared memory, its completion counted in bytes on the barrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Makes a tensor map written through the generic proxy (by an earlier kernel)
// visible to this thread's TMA instructions.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* bar,
                                            unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)), "l"(m), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
// Waits for phase `parity` of the barrier to complete, giving up after
// `limit` polls; returns whether it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i) {
    unsigned done = 0;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Polls of a TMA wait before it gives up (each poll suspends the thread for a
// while in hardware; a box lands in microseconds).
constexpr unsigned kTmaWaitPolls = 1u << 22;
// Value of Frame::status after a wait gave up.
constexpr unsigned kStatusTimeout = 1u;

// --------------------------------------------------------------------------------------------
// detect: stages (a)-(d) for one output tile of TW x TH pixels, computed only
// where they can change a flag.
//
// Exact pruning. S >= 0 and med5(S) >= 0, so S' <= S (also after float
// rounding). A flag needs a candidate within 2 px, a candidate needs
// S' > sigclip, and a growth flag needs S' > sigclip (first growth) or
// S' > sigfrac*sigclip (second). With an upper bound S+ >= S and
// tlow = min(sigclip, sigfrac*sigclip), the only positions whose S' can matter are
//   needS' = dilate5({S+ > sigclip}) and S+ > tlow,
// the exact S is needed on dilate5(needS'), and med3 on the 7x7
// neighbourhoods of the positions with S' > sigclip. S' elsewhere is replaced
// by -inf, which passes no threshold: the flags are unchanged.
// S+ comes from a lower bound of the 5x5 median: at most two values of each
// column lie below that column's median, so at most 10 of the 25 lie below the
// smallest column median, which is therefore <= the median. The threshold test
// S+ > t is evaluated as L+^2 gain^2 > 4 t^2 (1 - 1e-4) (gain m + rn^2): the
// 1e-4 margin exceeds the few float roundings of either side, so the test
// never rejects a position whose exact float32 S exceeds t.
// The sets are bit-row maps; dilations are word shifts and ORs, and the work
// lists are read off the set bits with block-wide prefix sums.
//
// The fused variant first performs the replacement of iteration k-1 (stage
// e) on R6 from I_{k-2} and M_{k-1} over R8, writes the tile's I_{k-1}, and
// then detects on the result.
//
// A persistent CTA walks its tiles; in detect_kernel the image region (and,
// fused, the flag words) of the next tile is loaded into the second of two
// buffers while the current tile is processed; detect1_kernel keeps one buffer
// and loads the next region after the tile.
//
// Shared memory, regions centred on the tile ("Rk" = tile grown by k px):
//   two image buffers, one in detect1_kernel (R8 of J, or fused of I_{k-2});
//   sCM (R2 rows x R4 columns) column medians, aliased by sS (R4) S; sM3 (R5)
//   med3; sN, sSp (R2) N and S' (-inf unless computed); fused: a flag buffer
//   (R8 rows) per image buffer; 9 bit maps; three position lists and small
//   counters.
template <int TW, int TH, bool kFused = false, bool kDouble = true>
struct DetectLayout {
  static constexpr int JW = TW + 12, JH = TH + 12;  // R6
  // The loaded image region is R8 (rows y0-8 .., columns x0-8 ..) in both
  // forms, so that the first column (x0 - 8, x0 a multiple of 32) lies on a
  // 16-byte boundary, as a TMA box must.
  static constexpr int JP = TW + 16, JR = TH + 16;
  static constexpr int JOFF = 2 * JP + 2;  // R6 origin inside an image buffer
  static constexpr int HALO = 8;           // halo of the loaded image region
  static constexpr int W5 = TW + 10, H5 = TH + 10;
  static constexpr int W4 = TW + 8, H4 = TH + 8;
  static constexpr int W2 = TW + 4, H2 = TH + 4;
  static constexpr int W1 = TW + 2, H1 = TH + 2;
  static constexpr int NW = TW / 32 + 2;           // words per bit-map row
  static constexpr int MW = NW * JH;               // words per bit map (R6 rows)
  static constexpr int MWF = kFused ? NW * (TH + 16) : 0;  // flag words of M_{k-1} (R8 rows)
  static_assert(TW % 32 == 0 && 32 * NW <= 256 && JH <= 255, "list entries pack (row << 8 | bit column)");
  static_assert(MW % 4 == 0, "bit maps are cleared as 16-byte vectors");
  static constexpr int oB0 = 0;  // floats
  static constexpr int oB1 = kDouble ? oB0 + JP * JR : oB0;  // kDouble = false: one image buffer
  static constexpr int oS = oB1 + JP * JR;
  static constexpr int oM3 = oS + imax(W4 * H4, H2 * W4);
  static constexpr int oN = oM3 + W5 * H5;
  static constexpr int oSp = oN + W2 * H2;
  static constexpr int nF = oSp + W2 * H2;
  static_assert(imax(W4 * H4, H2 * W4) + W5 * H5 >= JW * JH, "replacement values fit in the S/med3 area");
  static constexpr int kMaps = 9;  // hot, act, tmp, needS', needS, test, needM3, g1, g2
  static constexpr int oF0 = round16(nF * 4);  // bytes
  static constexpr int oF1 = kDouble ? oF0 + round16(MWF * 4) : oF0;
  static constexpr int oBits = oF1 + round16(MWF * 4);
  static constexpr int oL0 = round16(oBits + kMaps * MW * 4);
  static constexpr int oL1 = oL0 + round16(imax(W5 * H5, JW * JH) * 2);
  static constexpr int oL2 = oL1 + round16(W2 * H2 * 2);
  static constexpr int oCnt = oL2 + round16(W2 * H2 * 2);  // 16 ints: counters + scan scratch
  static constexpr int oBar = oCnt + 16 * 4;  // two mbarriers (one per image buffer), then the load flag
  static constexpr size_t bytes = size_t(oBar + 32);
  static_assert((JP * JR * 4) % 128 == 0, "both image buffers start on the 128-byte boundary a TMA box needs");
};

// bits of word j of bit-map row `row` (an R6 row) that lie in Rk and in the frame
template <int TW, int TH>
__device__ __forceinline__ uint32_t region_word(int kreg, int row, int j, int x0, int y0, int w, int h) {
  const int y = y0 - 6 + row;
  if (y < imax(0, y0 - kreg) || y >= min(h, y0 + TH + kreg)) return 0u;
  const int xw = x0 - 32 + 32 * j;
  return bits_between(imax(0, x0 - kreg) - xw, min(w, x0 + TW + kreg) - xw);
}

// out = in dilated by a (2R+1)^2 box, within Rk and the frame (and and_map if
// given); one pass, one barrier.
template <int TW, int TH, int R>
__device__ __forceinline__ void dilate_map(const uint32_t* in, uint32_t* out, const uint32_t* and_map, int kreg,
                                           int x0, int y0, int w, int h) {
  using L = DetectLayout<TW, TH>;
  for (int t = threadIdx.x; t < L::MW; t += kThreads) {
    const int row = t / L::NW, j = t - row * L::NW;
    uint32_t a = 0, l = 0, r = 0;  // vertical ORs of words j, j-1, j+1
#pragma unroll
    for (int d = -R; d <= R; ++d) {
      const int rr = row + d;
      if (rr < 0 || rr >= L::JH) continue;
      const uint32_t* p = in + rr * L::NW + j;
      a |= p[0];
      if (j > 0) l |= p[-1];
      if (j < L::NW - 1) r |= p[1];
    }
    uint32_t o = a;
#pragma unroll
    for (int d = 1; d <= R; ++d) o |= (a << d) | (l >> (32 - d)) | (a >> d) | (r << (32 - d));
    out[t] = o & region_word<TW, TH>(kreg, row, j, x0, y0, w, h) & (and_map ? and_map[t] : 0xffffffffu);
  }
  __syncthreads();
}

// region & frame mask of Rk as a bit map (dense mode)
template <int TW, int TH>
__device__ __forceinline__ void region_map(uint32_t* out, int kreg, int x0, int y0, int w, int h) {
  using L = DetectLayout<TW, TH>;
  for (int t = threadIdx.x; t < L::MW; t += kThreads) {
    const int row = t / L::NW, j = t - row * L::NW;
    out[t] = region_word<TW, TH>(kreg, row, j, x0, y0, w, h);
  }
}

// Positions of the set bits of up to two bit maps (words given by wordA(t),
// wordB(t)) -> list entries (row << 8 | bit column), with one block-wide scan.
template <int NW, int MW, typename FA, typename FB>
__device__ __forceinline__ void bits_to_lists(FA wordA, uint16_t* listA, int& nA, FB wordB, uint16_t* listB,
                                              int& nB, int* ws) {
  constexpr int kPer = (MW + kThreads - 1) / kThreads;
  const int t0 = threadIdx.x * kPer;
  uint32_t va[kPer], vb[kPer];
  int c = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    va[q] = (t0 + q < MW) ? wordA(t0 + q) : 0u;
    vb[q] = (t0 + q < MW) ? wordB(t0 + q) : 0u;
    c += __popc(va[q]) | (__popc(vb[q]) << 16);
  }
  int total = 0;
  const int off = block_excl_scan(c, ws, total);
  nA = total & 0xffff;
  nB = total >> 16;
  int oa = off & 0xffff, ob = off >> 16;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int t = t0 + q;
    const int row = t / NW, j = t - row * NW;
    uint32_t v = va[q];
    while (v) {
      const int b = __ffs(v) - 1;
      v &= v - 1u;
      listA[oa++] = uint16_t((row << 8) | (32 * j + b));
    }
    v = vb[q];
    while (v) {
      const int b = __ffs(v) - 1;
      v &= v - 1u;
      listB[ob++] = uint16_t((row << 8) | (32 * j + b));
    }
  }
}

// Whether tile (x0, y0) of frame f loads its image region by TMA: the frame
// has tensor maps and the whole region lies in the frame (no clamped reads).
template <int TW, int TH>
__device__ __forceinline__ bool tile_by_tma(const Frame& f, int x0, int y0) {
  return f.tmap != nullptr && x0 - 8 >= 0 && x0 + TW + 8 <= f.w && y0 - 8 >= 0 && y0 + TH + 8 <= f.h;
}

// Issues the asynchronous load of tile t's image region (and, fused, the flag
// words of an inner tile) into buffer b: one TMA box for a tile inside the
// frame (thread 0, completion on the buffer's mbarrier), else 4-byte copies of
// clamped positions by every thread. Returns whether the box was used.
// `acquired`: the tensor map thread 0 last made visible to its TMA loads.
template <int TW, int TH, bool kFused, bool kDouble = true>
__device__ __forceinline__ bool issue_tile_load(const Frame* __restrict__ frames, int nframes, long long t, int k,
                                                int niter, char* smem, int b, const CUtensorMap*& acquired) {
  using L = DetectLayout<TW, TH, kFused, kDouble>;
  const int fi = frame_of<false>(frames, nframes, t);
  const Frame& f = frames[fi];
  const long long tile = t - f.tile0;
  const int ty = int(tile / f.tiles_x), tx = int(tile - (long long)ty * f.tiles_x);
  const int x0 = tx * TW, y0 = ty * TH, w = f.w, h = f.h;
  const int ks = kFused ? k - 1 : k;
  const float* src = iter_src(f, ks, niter);
  float* buf = reinterpret_cast<float*>(smem) + (b ? L::oB1 : L::oB0);
  const bool tma = tile_by_tma<TW, TH>(f, x0, y0);
  if (tma) {
    if (threadIdx.x == 0) {
      // the source's map: img in iteration 1, then out_clean or ws as iter_src alternates them
      const CUtensorMap* m = f.tmap + (ks == 1 ? 0 : (src == f.out_clean ? 1 : 2));
      if (m != acquired) {  // once per map and block
        tensormap_acquire(m);
        acquired = m;
      }
      fence_proxy_async_smem();  // the block's earlier reads and writes of this buffer come first
      tma_load_2d(buf, m, x0 - 8, y0 - 8, reinterpret_cast<uint64_t*>(smem + L::oBar) + b,
                  unsigned(L::JP * L::JR * 4));
    }
  } else {
    for (int i = threadIdx.x; i < L::JP * L::JR; i += kThreads) {
      const int iy = i / L::JP, ix = i - iy * L::JP;
      const int gx = clampi(x0 - L::HALO + ix, 0, w - 1), gy = clampi(y0 - L::HALO + iy, 0, h - 1);
      cp_async4(buf + i, src + size_t(gy) * w + gx);
    }
  }
  if (kFused && x0 - 8 >= 0 && x0 + TW + 8 <= w && y0 - 8 >= 0 && y0 + TH + 8 <= h) {
    const uint32_t* Mb = mask_bits(f, k - 1);
    uint32_t* fl = reinterpret_cast<uint32_t*>(smem + (b ? L::oF1 : L::oF0));
    for (int i = threadIdx.x; i < L::MWF; i += kThreads) {
      const int row = i / L::NW, j = i - row * L::NW;
      cp_async4(fl + i, Mb + size_t(y0 - 8 + row) * f.wpr + (x0 >> 5) - 1 + j);
    }
  }
  cp_async_commit();
  return tma;
}

// Passes of detect_tile: a tile of the launch (0); the super tile of a
// two-step fused tile (1: iteration k over the tile widened to cover R8 of the
// inner tile; its flags M_k go to mOut, its replaced image stays in shared
// memory); the inner tile's second step (2: iteration k+1, whose replacement
// input -- I_k's predecessor and M_k over R8 -- is already in shared memory).
// New flags and pixels with no unflagged neighbour are counted only in the
// region (cy0, cx0, cth, ctw) of the tile (rows and columns from its origin).
enum { kPassTile = 0, kPassSuper = 1, kPassSecond = 2 };

template <int TW, int TH, bool kMaps, bool kFused, int kPass = kPassTile, bool kDouble = true>
__device__ void detect_tile(const Frame& f, const Params& p, int k, int niter, int x0, int y0, char* smem, int b,
                            uint32_t* mOut = nullptr, int cy0 = 0, int cx0 = 0, int cth = TH, int ctw = TW) {
  using L = DetectLayout<TW, TH, kFused, kDouble>;
  float* sBuf = reinterpret_cast<float*>(smem) + (b ? L::oB1 : L::oB0);
  float* sJ = sBuf + L::JOFF;  // R6 of J, row pitch L::JP
  float* sS = reinterpret_cast<float*>(smem) + L::oS;
  float* sCM = sS;  // column medians; dead before S is written
  float* sM3 = reinterpret_cast<float*>(smem) + L::oM3;
  float* sN = reinterpret_cast<float*>(smem) + L::oN;
  float* sSp = reinterpret_cast<float*>(smem) + L::oSp;
  uint32_t* mFl = reinterpret_cast<uint32_t*>(smem + (b ? L::oF1 : L::oF0));  // fused: M_{k-1} over R8 rows
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + L::oBits);
  uint32_t* mHot = bits + 0 * L::MW;
  uint32_t* mAct = bits + 1 * L::MW;
  uint32_t* mNeedSp = bits + 3 * L::MW;
  uint32_t* mNeedS = bits + 4 * L::MW;
  uint32_t* mTest = bits + 5 * L::MW;
  uint32_t* mNeedM3 = bits + 6 * L::MW;
  uint32_t* mG1 = bits + 7 * L::MW;
  uint32_t* mG2 = bits + 8 * L::MW;
  uint16_t* L0 = reinterpret_cast<uint16_t*>(smem + L::oL0);
  uint16_t* L1 = reinterpret_cast<uint16_t*>(smem + L::oL1);
  uint16_t* L2 = reinterpret_cast<uint16_t*>(smem + L::oL2);
  int* cnt = reinterpret_cast<int*>(smem + L::oCnt);  // [0] cand tests; [4..] scan scratch

  const int w = f.w, h = f.h;
  const float gain = f.gain, rn2 = __fmul_rn(f.rn, f.rn), g2 = __fmul_rn(f.gain, f.gain);
  const float sigclip = p.sigclip, siglow = __fmul_rn(p.sigfrac, p.sigclip), objlim = p.objlim;
  const float tlow = fminf(siglow, sigclip);
  const float chot = 4.f * sigclip * sigclip * 0.9999f, clow = 4.f * tlow * tlow * 0.9999f;
  const bool edge = (x0 - 6 < 0) || (y0 - 6 < 0) || (x0 + TW + 6 > w) || (y0 + TH + 6 > h);
  const bool inner = x0 - 8 >= 0 && x0 + TW + 8 <= w && y0 - 8 >= 0 && y0 + TH + 8 <= h;
  const size_t npix = size_t(w) * size_t(h);
  const int tid = threadIdx.x;

  // P0: clear bit maps and counters, S' = -inf (the image region is already in sBuf)
  for (int i = tid; i < L::kMaps * L::MW / 4; i += kThreads)
    reinterpret_cast<uint4*>(bits)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid < 4) cnt[tid] = 0;
  for (int i = tid; i < L::W2 * L::H2; i += kThreads) sSp[i] = -INFINITY;
  if (kFused && !inner && kPass != kPassSecond)
    for (int i = tid; i < L::MWF; i += kThreads) mFl[i] = 0u;
  __syncthreads();

  if (kFused) {
    // Iteration k-1's replacement on R6 from I_{k-2} (sBuf, R8) and M_{k-1} (mFl, R8 rows).
    const int kr = k - 1;
    if (!inner && kPass != kPassSecond) {  // clamped flag of every R8 position (replicate edge)
      const uint32_t* __restrict__ Mb = mask_bits(f, kr);
      for (int i = tid; i < L::JP * L::JR; i += kThreads) {
        const int iy = i / L::JP, ix = i - iy * L::JP;
        const int gx = clampi(x0 - 8 + ix, 0, w - 1), gy = clampi(y0 - 8 + iy, 0, h - 1);
        if ((__ldg(Mb + size_t(gy) * f.wpr + (gx >> 5)) >> (gx & 31)) & 1u)
          atomicOr(&mFl[iy * L::NW + ((ix + 24) >> 5)], 1u << ((ix + 24) & 31));
      }
      __syncthreads();
    }
    int nR = 0, nDummy = 0;
    bits_to_lists<L::NW, L::MW>(
        [&](int t) {  // flagged in-frame R6 positions
          const int row = t / L::NW, j = t - row * L::NW;
          return mFl[(row + 2) * L::NW + j] & region_word<TW, TH>(6, row, j, x0, y0, w, h);
        },
        L0, nR, [](int) { return 0u; }, L1, nDummy, cnt + 4);
    __syncthreads();
    float* val = sS;  // scratch for the replacement values (the S / med3 area is free here)
    unsigned int none_left = 0;
    for (int j = tid; j < nR; j += kThreads) {
      const int e = L0[j];
      const int r6 = e >> 8, xb = e & 255;
      const int cy = r6 + 2, cx = xb - 24;  // R8 coordinates
      uint32_t win = 0;                     // 25 window flags, row-major
#pragma unroll
      for (int dy = 0; dy < 5; ++dy) {
        const int wj = (xb - 2) >> 5, sh = (xb - 2) & 31;
        const uint32_t* rowp = mFl + (cy - 2 + dy) * L::NW;
        const uint32_t lo = rowp[wj], hi = (wj + 1 < L::NW) ? rowp[wj + 1] : 0u;
        win |= (__funnelshift_r(lo, hi, sh) & 31u) << (5 * dy);
      }
      const int n = 25 - __popc(win);
      float v[25];
      float out;
      if (n > 0) {
        const int a = 13 - (n + 1) / 2;  // flagged entries sent to -inf
        int seen = 0;
#pragma unroll
        for (int q = 0; q < 25; ++q) {
          float x = sBuf[(cy - 2 + q / 5) * L::JP + cx - 2 + q % 5];
          if ((win >> q) & 1u) {
            x = (seen < a) ? -INFINITY : INFINITY;
            ++seen;
          }
          v[q] = x;
        }
        out = sel_med25(v);
      } else {
#pragma unroll
        for (int q = 0; q < 25; ++q) v[q] = sBuf[(cy - 2 + q / 5) * L::JP + cx - 2 + q % 5];
        out = floor_m5(sel_med25(v));
        if (r6 >= 6 + cy0 && r6 < 6 + cy0 + cth && xb >= 32 + cx0 && xb < 32 + cx0 + ctw) ++none_left;
      }
      val[j] = out;
    }
    for (int off = 16; off; off >>= 1) none_left += __shfl_xor_sync(0xffffffffu, none_left, off);
    if ((tid & 31) == 0 && none_left) atomicAdd(f.counters + 2 * (kr - 1) + 1, (unsigned long long)none_left);
    __syncthreads();
    float* __restrict__ Dprev = iter_dst(f, kr, niter);
    for (int j = tid; j < nR; j += kThreads) {
      const int e = L0[j];
      const int r6 = e >> 8, xb = e & 255;
      sBuf[(r6 + 2) * L::JP + xb - 24] = val[j];
      if (kPass != kPassSuper && r6 >= 6 && r6 < 6 + TH && xb >= 32 && xb < 32 + TW)
        Dprev[size_t(y0 - 6 + r6) * w + (x0 - 32 + xb)] = val[j];
    }
    if (kPass != kPassSuper && kr <= f.dense_upto) {  // a buffer's first write is dense
      for (int i = tid; i < TW * TH; i += kThreads) {
        const int ly = i / TW, lx = i - ly * TW;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= w || gy >= h) continue;
        if ((mFl[(ly + 8) * L::NW + ((lx + 32) >> 5)] >> (lx & 31)) & 1u) continue;
        Dprev[size_t(gy) * w + gx] = sBuf[(ly + 8) * L::JP + lx + 8];
      }
    }
    __syncthreads();
    if (edge) {  // replicate the replaced frame edge into the out-of-frame part of R6
      for (int i = tid; i < L::JW * L::JH; i += kThreads) {
        const int iy = i / L::JW, ix = i - iy * L::JW;
        const int gx = x0 - 6 + ix, gy = y0 - 6 + iy;
        if (gx >= 0 && gx < w && gy >= 0 && gy < h) continue;
        const int sx = clampi(gx, 0, w - 1) - (x0 - 6), sy = clampi(gy, 0, h - 1) - (y0 - 6);
        sJ[iy * L::JP + ix] = sJ[sy * L::JP + sx];
      }
      __syncthreads();
    }
  }

  if (kMaps) {
    region_map<TW, TH>(mAct, 2, x0, y0, w, h);
    region_map<TW, TH>(mNeedSp, 2, x0, y0, w, h);
    region_map<TW, TH>(mNeedS, 4, x0, y0, w, h);
    __syncthreads();
  } else {
    // P1: medians of the 5 vertical values of every column of R4, rows of R2
    for (int i = tid; i < L::H2 * L::W4; i += kThreads) {
      const int iy = i / L::W4, ix = i - iy * L::W4;
      float v[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) v[d] = sJ[(iy + 2 + d) * L::JP + ix + 2];
      sCM[i] = sel_med5(v);
    }
    __syncthreads();

    // P2: L+ and the bound S+ on R2 -> bits of S+ > sigclip (hot) and S+ > tlow (act)
    for (int i = tid; i < L::W2 * L::H2; i += kThreads) {
      const int iy = i / L::W2, ix = i - iy * L::W2;
      const int gx = x0 - 2 + ix, gy = y0 - 2 + iy;
      if (gx < 0 || gx >= w || gy < 0 || gy >= h) continue;
      const float* c = sJ + (iy + 4) * L::JP + ix + 4;
      const float lp = lplus(c[0], c[-L::JP], c[L::JP], c[-1], c[1]);
      const float* cm = sCM + iy * L::W4 + ix;
      const float mlow = min3f(min3f(cm[0], cm[1], cm[2]), cm[3], cm[4]);
      const float den = gain * (mlow > 0.f ? mlow : 0.f) + rn2;
      const float lhs = lp * lp * g2;
      if (lhs > clow * den) {
        const int xb = ix + 30, wd = (iy + 4) * L::NW + (xb >> 5);
        const uint32_t bit = 1u << (xb & 31);
        atomicOr(&mAct[wd], bit);
        if (lhs > chot * den) atomicOr(&mHot[wd], bit);
      }
    }
    __syncthreads();

    // needS' = dilate5(hot) & act;  needS = dilate5(needS') within R4 and the frame
    dilate_map<TW, TH, 2>(mHot, mNeedSp, mAct, 2, x0, y0, w, h);
    dilate_map<TW, TH, 2>(mNeedSp, mNeedS, nullptr, 4, x0, y0, w, h);
  }

  // lists: L0 <- needS (R4), L2 <- needS' (R2)
  int nS = 0, nSp = 0;
  bits_to_lists<L::NW, L::MW>([&](int t) { return mNeedS[t]; }, L0, nS, [&](int t) { return mNeedSp[t]; }, L2,
                              nSp, cnt + 4);
  __syncthreads();
  if (tid == 0 && f.work) {
    unsigned long long* wk = f.work + kWork * (k - 1);
    const long long dense = (long long)(min(x0 + TW + 2, w) - imax(x0 - 2, 0)) * (min(y0 + TH + 2, h) - imax(y0 - 2, 0));
    atomicAdd(wk + 0, (unsigned long long)nS);
    atomicAdd(wk + 1, (unsigned long long)nSp);
    atomicAdd(wk + 5, (unsigned long long)dense);
  }

  // P6: (a)+(b) at the listed positions: m5, N, L+, S
  for (int j = tid; j < nS; j += kThreads) {
    const int e = L0[j];
    const int iy = (e >> 8) - 2, ix = (e & 255) - 28;  // R4 coordinates
    const int i = iy * L::W4 + ix;
    const int cx = ix + 2, cy = iy + 2;  // centre in sJ
    float v[25];
#pragma unroll
    for (int dy = 0; dy < 5; ++dy)
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = sJ[(cy - 2 + dy) * L::JP + cx - 2 + dx];
    const float m5f = floor_m5(sel_med25(v));
    const float n = noise_of(m5f, gain, rn2);
    const float* c = sJ + cy * L::JP + cx;
    const float lp = lplus(c[0], c[-L::JP], c[L::JP], c[-1], c[1]);
    const float s = __fdiv_rn(lp, __fmul_rn(2.f, n));
    sS[i] = s;
    if (ix >= 2 && ix < L::W4 - 2 && iy >= 2 && iy < L::H4 - 2) sN[(iy - 2) * L::W2 + ix - 2] = n;
    if (kMaps && ix >= 4 && ix < 4 + TW && iy >= 4 && iy < 4 + TH) {
      const size_t o = size_t(y0 - 4 + iy) * w + (x0 - 4 + ix);
      f.maps[0 * npix + o] = m5f;
      f.maps[1 * npix + o] = lp;
      f.maps[2 * npix + o] = n;
      f.maps[3 * npix + o] = s;
    }
  }
  __syncthreads();
  if (edge) {  // replicate the frame-edge S into out-of-frame entries
    for (int i = tid; i < L::W4 * L::H4; i += kThreads) {
      const int iy = i / L::W4, ix = i - iy * L::W4;
      const int gx = x0 - 4 + ix, gy = y0 - 4 + iy;
      if (gx >= 0 && gx < w && gy >= 0 && gy < h) continue;
      const int sx = clampi(gx, 0, w - 1) - (x0 - 4), sy = clampi(gy, 0, h - 1) - (y0 - 4);
      sS[i] = sS[sy * L::W4 + sx];
    }
    __syncthreads();
  }

  // P7: S' = S - med5(S) at the listed R2 positions; list the candidate tests (S' > sigclip)
  for (int j0 = 0; j0 < nSp; j0 += kThreads) {
    const int j = j0 + tid;
    bool test = false;
    int i = 0;
    if (j < nSp) {
      const int e = L2[j];
      const int iy = (e >> 8) - 4, ix = (e & 255) - 30;  // R2 coordinates
      i = iy * L::W2 + ix;
      const int cx = ix + 2, cy = iy + 2;  // centre in sS
      float v[25];
#pragma unroll
      for (int dy = 0; dy < 5; ++dy)
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = sS[(cy - 2 + dy) * L::W4 + cx - 2 + dx];
      const float sp = __fsub_rn(sS[cy * L::W4 + cx], sel_med25(v));
      sSp[i] = sp;
      test = sp > sigclip;
      if (test) atomicOr(&mTest[(e >> 8) * L::NW + ((e & 255) >> 5)], 1u << (e & 31));
      if (kMaps && ix >= 2 && ix < 2 + TW && iy >= 2 && iy < 2 + TH) {
        const size_t o = size_t(y0 - 2 + iy) * w + (x0 - 2 + ix);
        f.maps[4 * npix + o] = sp;
        f.maps[8 * npix + o] = 0.f;  // overwritten below where the candidate test runs
      }
    }
    push_if(test, i, L1, &cnt[0]);
  }
  __syncthreads();

  // needM3 = dilate7(test) within R5 and the frame; list it
  if (kMaps) {
    region_map<TW, TH>(mNeedM3, 5, x0, y0, w, h);
    __syncthreads();
  } else {
    dilate_map<TW, TH, 3>(mTest, mNeedM3, nullptr, 5, x0, y0, w, h);
  }
  int nM3 = 0, nDummy = 0;
  bits_to_lists<L::NW, L::MW>([&](int t) { return mNeedM3[t]; }, L0, nM3, [](int) { return 0u; }, L2, nDummy,
                              cnt + 4);
  __syncthreads();
  if (tid == 0 && f.work) {
    atomicAdd(f.work + kWork * (k - 1) + 2, (unsigned long long)nM3);
    atomicAdd(f.work + kWork * (k - 1) + 3, (unsigned long long)cnt[0]);  // every test takes the full median
    atomicAdd(f.work + kWork * (k - 1) + 4, (unsigned long long)cnt[0]);
  }

  // P9: med3 at the listed positions
  for (int j = tid; j < nM3; j += kThreads) {
    const int e = L0[j];
    const int iy = (e >> 8) - 1, ix = (e & 255) - 27;  // R5 coordinates
    const int cx = ix + 1, cy = iy + 1;                 // centre in sJ
    float v[9];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = sJ[(cy - 1 + dy) * L::JP + cx - 1 + dx];
    const float m3 = sel_med9(v);
    sM3[iy * L::W5 + ix] = m3;
    if (kMaps && ix >= 5 && ix < 5 + TW && iy >= 5 && iy < 5 + TH)
      f.maps[5 * npix + size_t(y0 - 5 + iy) * w + (x0 - 5 + ix)] = m3;
  }
  __syncthreads();
  if (edge) {
    for (int i = tid; i < L::W5 * L::H5; i += kThreads) {
      const int iy = i / L::W5, ix = i - iy * L::W5;
      const int gx = x0 - 5 + ix, gy = y0 - 5 + iy;
      if (gx >= 0 && gx < w && gy >= 0 && gy < h) continue;
      const int sx = clampi(gx, 0, w - 1) - (x0 - 5), sy = clampi(gy, 0, h - 1) - (y0 - 5);
      sM3[i] = sM3[sy * L::W5 + sx];
    }
    __syncthreads();
  }

  // P10: (c)+(d) at the candidate tests: F, the objlim statistic, and for each
  // candidate the two growths it causes inside the tile (bits of g2)
  const int nT = cnt[0];
  for (int j = tid; j < nT; j += kThreads) {
    const int i = L1[j];
    const int iy = i / L::W2, ix = i - iy * L::W2;
    const int mx = ix + 3, my = iy + 3;  // centre in sM3
    float u[49];
#pragma unroll
    for (int dy = 0; dy < 7; ++dy)
#pragma unroll
      for (int dx = 0; dx < 7; ++dx) u[dy * 7 + dx] = sM3[(my - 3 + dy) * L::W5 + mx - 3 + dx];
    const float fval = __fsub_rn(sM3[my * L::W5 + mx], sel_med49(u));
    const float fn = fmaxf(__fdiv_rn(fval, sN[i]), 0.01f);
    const float sp = sSp[i];
    const float rval = (p.objlim_form == 1) ? __fdiv_rn(__fmul_rn(2.f, sS[(iy + 2) * L::W4 + ix + 2]), fn)
                                            : __fdiv_rn(sp, fn);
    const bool cand = rval > objlim;
    if (kMaps && ix >= 2 && ix < 2 + TW && iy >= 2 && iy < 2 + TH) {
      const size_t o = size_t(y0 - 2 + iy) * w + (x0 - 2 + ix);
      f.maps[6 * npix + o] = fval;
      f.maps[7 * npix + o] = rval;
      f.maps[8 * npix + o] = cand ? 1.f : 0.f;
    }
    if (!cand) continue;
    for (int ey = -1; ey <= 1; ++ey) {
      const int qy = iy + ey;  // first-growth position (R2 coordinates)
      if (qy < 1 || qy > L::H2 - 2) continue;
      for (int ex = -1; ex <= 1; ++ex) {
        const int qx = ix + ex;
        if (qx < 1 || qx > L::W2 - 2) continue;
        if (!(sSp[qy * L::W2 + qx] > sigclip)) continue;
        if (kMaps) atomicOr(&mG1[(qy + 4) * L::NW + ((qx + 30) >> 5)], 1u << ((qx + 30) & 31));
        for (int ry = qy - 1; ry <= qy + 1; ++ry) {
          if (ry < 2 || ry >= 2 + TH) continue;
          for (int rx = qx - 1; rx <= qx + 1; ++rx) {
            if (rx < 2 || rx >= 2 + TW) continue;
            if (sSp[ry * L::W2 + rx] > siglow)
              atomicOr(&mG2[(ry + 4) * L::NW + ((rx + 30) >> 5)], 1u << ((rx + 30) & 31));
          }
        }
      }
    }
  }
  __syncthreads();

  // P11: the tile's flag words, M_k = M_{k-1} | g2
  constexpr int kWordsPerRow = TW / 32;
  unsigned int new_flags = 0;
  for (int wi = tid; wi < kWordsPerRow * TH; wi += kThreads) {
    const int r = wi / kWordsPerRow, wc = wi - r * kWordsPerRow;
    const int gy = y0 + r, gwc = (x0 >> 5) + wc;
    if (gy < 0 || gy >= h || gwc < 0 || gwc >= f.wpr) continue;
    const uint32_t g2w = mG2[(r + 6) * L::NW + 1 + wc];  // x0 + 32 wc is word 1 + wc of the row
    const size_t wo = size_t(gy) * f.wpr + gwc;
    // M_{k-1}: in shared memory for the second step of a fused pair (R8 rows, word 1 = x0)
    const uint32_t prev = (kPass == kPassSecond) ? mFl[(r + 8) * L::NW + 1 + wc] : mask_bits(f, k - 1)[wo];
    if (kPass == kPassSuper)
      mOut[r * kWordsPerRow + wc] = prev | g2w;
    else
      mask_bits(f, k)[wo] = prev | g2w;
    if (r >= cy0 && r < cy0 + cth && 32 * wc >= cx0 && 32 * wc < cx0 + ctw) new_flags += __popc(g2w & ~prev);
    if (kMaps) {
      const uint32_t g1w = mG1[(r + 6) * L::NW + 1 + wc];
      for (int bb = 0; bb < 32; ++bb) {
        const int gx = x0 + 32 * wc + bb;
        if (gx >= w) break;
        const size_t o = size_t(gy) * w + gx;
        f.maps[9 * npix + o] = ((g1w >> bb) & 1u) ? 1.f : 0.f;
        f.maps[10 * npix + o] = ((g2w >> bb) & 1u) ? 1.f : 0.f;
      }
    }
  }
  for (int off = 16; off; off >>= 1) new_flags += __shfl_xor_sync(0xffffffffu, new_flags, off);
  if ((tid & 31) == 0 && new_flags) atomicAdd(f.counters + 2 * (k - 1), (unsigned long long)new_flags);
}

// The tiles of a detection launch, block-strided. kDouble: two image
// buffers, the next tile's region loading while this tile is computed; else
// one buffer, loaded after the tile (for launches in which a block has about
// one tile, at three resident blocks per SM: detect1_kernel).
template <int TW, int TH, bool kMaps, bool kFused, bool kDouble>
__device__ __forceinline__ void detect_tiles(const Frame* __restrict__ frames, int nframes, long long ntiles,
                                             Params p, int k, int niter) {
  extern __shared__ __align__(128) char smem[];
  using L = DetectLayout<TW, TH, kFused, kDouble>;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::oBar);
  int* ok = reinterpret_cast<int*>(smem + L::oBar + 16);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  unsigned phase = 0;  // thread 0: parity of the next completion of each buffer's barrier (bit b)
  const CUtensorMap* acquired = nullptr;
  long long t = blockIdx.x;
  bool tma = t < ntiles && issue_tile_load<TW, TH, kFused, kDouble>(frames, nframes, t, k, niter, smem, 0, acquired);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int b = kDouble ? (it & 1) : 0;
    cp_async_wait_all();
    if (threadIdx.x == 0) {
      bool landed = true;
      if (tma) {
        landed = mbar_wait(bar + b, (phase >> b) & 1u, kTmaWaitPolls);
        phase ^= 1u << b;
        if (!landed) {
          if (frames[0].status) atomicOr(frames[0].status, kStatusTimeout);
          mbar_wait(bar + b, ((phase >> b) & 1u) ^ 1u, kTmaWaitPolls);  // the box still in flight, bounded
        }
      }
      *ok = landed ? 1 : 0;
    }
    __syncthreads();  // tile t's image region has landed in buffer b
    if (!*ok) return;  // every thread of the block leaves together; the status reports it
    const long long tn = t + gridDim.x;
    bool tma_next = false;
    if (kDouble)
      tma_next = tn < ntiles && issue_tile_load<TW, TH, kFused, kDouble>(frames, nframes, tn, k, niter, smem, b ^ 1,
                                                                         acquired);
    const int fi = frame_of<false>(frames, nframes, t);
    const Frame f = frames[fi];
    const long long tile = t - f.tile0;
    const int ty = int(tile / f.tiles_x), tx = int(tile - (long long)ty * f.tiles_x);
    detect_tile<TW, TH, kMaps, kFused, kPassTile, kDouble>(f, p, k, niter, tx * TW, ty * TH, smem, b);
    __syncthreads();  // the block is done with buffer b
    if (!kDouble)
      tma_next = tn < ntiles && issue_tile_load<TW, TH, kFused, kDouble>(frames, nframes, tn, k, niter, smem, 0,
                                                                         acquired);
    tma = tma_next;
  }
}

template <int TW, int TH, bool kMaps, bool kFused = false>
__global__ void __launch_bounds__(kThreads) detect_kernel(const Frame* __restrict__ frames, int nframes,
                                                          long long ntiles, Params p, int k, int niter) {
  detect_tiles<TW, TH, kMaps, kFused, true>(frames, nframes, ntiles, p, k, niter);
}

// One image buffer, at most 80 registers: three blocks per SM where the
// shared memory of a block is at most 75 KB (64 x 28 tiles).
template <int TW, int TH, bool kMaps, bool kFused = false>
__global__ void __launch_bounds__(kThreads, 3) detect1_kernel(const Frame* __restrict__ frames, int nframes,
                                                              long long ntiles, Params p, int k, int niter) {
  detect_tiles<TW, TH, kMaps, kFused, false>(frames, nframes, ntiles, p, k, niter);
}

// --------------------------------------------------------------------------------------------
// detect2: iterations k and k+1 of a TW x TH tile in one launch (temporal
// fusion with halo recompute). Iteration k+1's detection on the tile needs I_k
// on R6 of the tile, whose replacement needs M_k on R8; so the block first
// runs the fused iteration k (replacement of k-1, then detection) over the
// super tile -- the tile widened by 32 columns (whole flag words) and 8 rows
// each way -- from I_{k-2} and M_{k-1}, keeping its replaced image and its
// flags in shared memory, then the fused iteration k+1 on the tile itself
// from those. Each block recomputes the ring its neighbours also compute, and
// no block reads what another writes in the launch: I_{k-1} and M_k never
// leave shared memory, I_k and M_{k+1} go to buffers nobody reads here.
template <int TW, int TH>
struct Detect2Layout {
  using LS = DetectLayout<TW + 64, TH + 16, true, false>;  // super tile, one image buffer
  using LT = DetectLayout<TW, TH, true, false>;
  static constexpr int oT = (int(LS::bytes) + 127) / 128 * 128;
  static constexpr int oOut = oT + (int(LT::bytes) + 127) / 128 * 128;  // M_k of the super tile
  static constexpr int kOutWords = (TH + 16) * (TW / 32 + 2);
  static constexpr size_t bytes = size_t(oOut + kOutWords * 4);
  static_assert(bytes <= 227 * 1024, "fits the shared memory of one block");
};

template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) detect2_kernel(const Frame* __restrict__ frames, int nframes,
                                                           long long ntiles, Params p, int k, int niter) {
  using D = Detect2Layout<TW, TH>;
  using LS = typename D::LS;
  using LT = typename D::LT;
  constexpr int SW = TW + 64, SH = TH + 16, NWT = LT::NW;
  extern __shared__ __align__(128) char smem[];
  char* smemT = smem + D::oT;
  uint32_t* mOut = reinterpret_cast<uint32_t*>(smem + D::oOut);
  const int tid = threadIdx.x;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int fi = frame_of<false>(frames, nframes, t);
    const Frame f = frames[fi];
    const long long tile = t - f.tile0;
    const int ty = int(tile / f.tiles_x), tx = int(tile - (long long)ty * f.tiles_x);
    const int x0 = tx * TW, y0 = ty * TH, w = f.w, h = f.h;
    const int xs = x0 - 32, ys = y0 - 8;  // the super tile
    // I_{k-2} over R8 of the super tile (clamped), M_{k-1} flag words of an inner super tile
    {
      const float* src = iter_src(f, k - 1, niter);
      float* buf = reinterpret_cast<float*>(smem) + LS::oB0;
      for (int i = tid; i < LS::JP * LS::JR; i += kThreads) {
        const int iy = i / LS::JP, ix = i - iy * LS::JP;
        const int gx = clampi(xs - 8 + ix, 0, w - 1), gy = clampi(ys - 8 + iy, 0, h - 1);
        cp_async4(buf + i, src + size_t(gy) * w + gx);
      }
      if (xs - 8 >= 0 && xs + SW + 8 <= w && ys - 8 >= 0 && ys + SH + 8 <= h) {
        const uint32_t* Mb = mask_bits(f, k - 1);
        uint32_t* fl = reinterpret_cast<uint32_t*>(smem + LS::oF0);
        for (int i = tid; i < LS::MWF; i += kThreads) {
          const int row = i / LS::NW, j = i - row * LS::NW;
          cp_async4(fl + i, Mb + size_t(ys - 8 + row) * f.wpr + (xs >> 5) - 1 + j);
        }
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
    }
    // iteration k over the super tile; new flags and pixels with no unflagged neighbour counted on the tile
    Frame fs = f;
    fs.work = nullptr;
    detect_tile<SW, SH, false, true, kPassSuper, false>(fs, p, k, niter, xs, ys, smem, 0, mOut, 8, 32, TH, TW);
    __syncthreads();
    // the tile's replacement input: I_{k-1} and M_k over its R8, clamped at the frame's edges
    {
      const float* sImg = reinterpret_cast<const float*>(smem) + LS::oB0;  // R8 of the super tile
      float* tImg = reinterpret_cast<float*>(smemT) + LT::oB0;
      uint32_t* tFl = reinterpret_cast<uint32_t*>(smemT + LT::oF0);
      for (int i = tid; i < LT::JP * LT::JR; i += kThreads) {  // R8 of the tile lies in R6 of the super tile
        const int iy = i / LT::JP, ix = i - iy * LT::JP;
        tImg[i] = sImg[(iy + 8) * LS::JP + ix + 32];
      }
      const bool inner = x0 - 8 >= 0 && x0 + TW + 8 <= w && y0 - 8 >= 0 && y0 + TH + 8 <= h;
      constexpr int kSWords = SW / 32;  // words per row of mOut; word j of a row covers xs + 32 j
      if (inner) {  // the tile's flag word j of R8 row r (covering x0 - 32 + 32 j) is mOut's word j of row r
        for (int i = tid; i < LT::MWF; i += kThreads) {
          const int r = i / NWT, j = i - r * NWT;
          tFl[i] = mOut[r * kSWords + j];
        }
      } else {  // the flag of the clamped position (replicate edge), bit ix + 24 of the row's words
        for (int i = tid; i < LT::MWF; i += kThreads) tFl[i] = 0u;
        __syncthreads();
        for (int i = tid; i < LT::JP * LT::JR; i += kThreads) {
          const int iy = i / LT::JP, ix = i - iy * LT::JP;
          const int gx = clampi(x0 - 8 + ix, 0, w - 1), gy = clampi(y0 - 8 + iy, 0, h - 1);
          const int sx = gx - xs, sy = gy - ys;  // inside the super tile
          if ((mOut[sy * kSWords + (sx >> 5)] >> (sx & 31)) & 1u)
            atomicOr(&tFl[iy * NWT + ((ix + 24) >> 5)], 1u << ((ix + 24) & 31));
        }
      }
      __syncthreads();
    }
    // iteration k+1 on the tile: the replacement of iteration k, then detection -> I_k, M_{k+1}
    detect_tile<TW, TH, false, true, kPassSecond, false>(f, p, k + 1, niter, x0, y0, smemT, 0);
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
// A tile without flagged pixels only copies (dense iterations) or is skipped.
template <int RW, int RH>
struct ReplaceLayout {
  static constexpr int W = RW + 4, H = RH + 4;
  static constexpr int FW = RW / 32 + 2;  // flag words per row: (x0 >> 5) - 1 ... (x0 >> 5) + RW / 32
  static constexpr int oF = round16(W * H * 4);
  static constexpr int oL = oF + round16(W * H);
  static constexpr int oWd = oL + round16(RW * RH * 2);
  static constexpr int oCnt = oWd + round16(H * FW * 4);
  static constexpr size_t bytes = size_t(oCnt + 16);
};

template <int RW, int RH>
__device__ void replace_tile(const Frame& f, int k, int niter, int dense, long long tile, char* smem) {
  using L = ReplaceLayout<RW, RH>;
  static_assert(RW % 32 == 0, "tile width must be whole flag words");
  float* sJ = reinterpret_cast<float*>(smem);
  uint8_t* sF = reinterpret_cast<uint8_t*>(smem + L::oF);
  uint16_t* list = reinterpret_cast<uint16_t*>(smem + L::oL);
  int* cnt = reinterpret_cast<int*>(smem + L::oCnt);
  const int w = f.w, h = f.h;
  const int ty = int(tile / f.rtiles_x), tx = int(tile - (long long)ty * f.rtiles_x);
  const int x0 = tx * RW, y0 = ty * RH;
  const float* __restrict__ J = iter_src(f, k, niter);
  float* __restrict__ D = iter_dst(f, k, niter);
  const bool last = (k == niter);
  const int tid = threadIdx.x;
  const uint32_t* __restrict__ M = mask_bits(f, k);

  // any flagged pixel in the tile?
  constexpr int kWords = RW / 32;
  bool any = false;
  for (int wi = tid; wi < kWords * RH; wi += kThreads) {
    const int r = wi / kWords, wc = wi - r * kWords;
    const int gy = y0 + r, wx = (x0 >> 5) + wc;
    if (gy < h && wx < f.wpr) any |= M[size_t(gy) * f.wpr + wx] != 0u;
  }
  if (tid == 0) cnt[0] = 0;
  any = __syncthreads_or(any);
  if (!any) {
    if (dense || (last && f.out_mask)) {
      for (int i = tid; i < RW * RH; i += kThreads) {
        const int ly = i / RW, lx = i - ly * RW;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= w || gy >= h) continue;
        const size_t o = size_t(gy) * w + gx;
        if (dense) D[o] = __ldg(J + o);
        if (last && f.out_mask) f.out_mask[o] = 0;
      }
    }
    return;
  }

  uint32_t* sWd = reinterpret_cast<uint32_t*>(smem + L::oWd);  // flag words of the rows (clamped)
  for (int i = tid; i < L::H * L::FW; i += kThreads) {
    const int iy = i / L::FW, j = i - iy * L::FW;
    const int gy = clampi(y0 - 2 + iy, 0, h - 1), wx = (x0 >> 5) - 1 + j;
    sWd[i] = (wx >= 0 && wx < f.wpr) ? __ldg(M + size_t(gy) * f.wpr + wx) : 0u;
  }
  for (int i = tid; i < L::W * L::H; i += kThreads) {
    const int iy = i / L::W, ix = i - iy * L::W;
    const int gx = clampi(x0 - 2 + ix, 0, w - 1), gy = clampi(y0 - 2 + iy, 0, h - 1);
    sJ[i] = __ldg(J + size_t(gy) * w + gx);
  }
  __syncthreads();
  for (int i = tid; i < L::W * L::H; i += kThreads) {
    const int iy = i / L::W, ix = i - iy * L::W;
    const int bit = clampi(x0 - 2 + ix, 0, w - 1) - (x0 - 32);  // bit index in the row's words
    sF[i] = uint8_t((sWd[iy * L::FW + (bit >> 5)] >> (bit & 31)) & 1u);
  }
  __syncthreads();

  for (int i0 = 0; i0 < RW * RH; i0 += kThreads) {
    const int i = i0 + tid;
    bool flagged = false;
    if (i < RW * RH) {
      const int ly = i / RW, lx = i - ly * RW;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx < w && gy < h) {
        const int c = (ly + 2) * L::W + lx + 2;
        flagged = sF[c] != 0;
        const size_t o = size_t(gy) * w + gx;
        if (dense && !flagged) D[o] = sJ[c];
        if (last && f.out_mask) f.out_mask[o] = flagged ? 1 : 0;
      }
    }
    push_if(flagged, i, list, cnt);
  }
  __syncthreads();

  unsigned int none_left = 0;
  for (int j = tid; j < cnt[0]; j += kThreads) {
    const int i = list[j];
    const int ly = i / RW, lx = i - ly * RW;
    const int c = (ly + 2) * L::W + lx + 2;
    int n = 0;
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
      for (int dx = -2; dx <= 2; ++dx) n += sF[c + dy * L::W + dx] ? 0 : 1;
    float v[25];
    float out;
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
    D[size_t(y0 + ly) * w + x0 + lx] = out;
  }
  for (int off = 16; off; off >>= 1) none_left += __shfl_xor_sync(0xffffffffu, none_left, off);
  if ((tid & 31) == 0 && none_left) atomicAdd(f.counters + 2 * (k - 1) + 1, (unsigned long long)none_left);
}

template <int RW, int RH>
__global__ void __launch_bounds__(kThreads) replace_kernel(const Frame* __restrict__ frames, int nframes,
                                                           long long ntiles, int k, int niter, int dense) {
  extern __shared__ __align__(128) char smem[];
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
