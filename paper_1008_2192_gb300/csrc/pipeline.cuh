// Queue pipeline of one detection (stages a-d): small kernels connected by
// global work queues, so that every sparse step runs with full warps and no
// block barriers.
//
//   bound_kernel   dense: L+ and the upper bound S+ of every pixel -> bit
//                  planes hot (S+ > sigclip) and act (S+ > sigfrac*sigclip);
//   need_kernel    needS' = dilate5(hot) & act and needS = dilate5(needS')
//                  -> queues QS (needS) and QSP (needS'), bit plane nsp;
//   s_kernel       at QS: m5, N, L+, S -> maps N, S;
//   sp_kernel      at QSP: S' = S - med5(S) -> map S'; S' > sigclip -> queue QT
//                  and bit plane test;
//   m3need_kernel  needM3 = dilate7(test) -> queue QM3;
//   m3_kernel      at QM3: med3 -> map M3;
//   cand_kernel    at QT: F = m3 - med7(m3), the objlim statistic, and for each
//                  candidate the two growths, ORed into the flag bits.
//
// The sets, and the argument that the flags equal those of the full
// computation, are those of detect_tile (kernels.cuh). Positions in queues are
// global pixel indices over all frames of the call (frame base + y*w + x).
// Every window read clamps its coordinates into the frame, which equals the
// per-map replicate-edge rule.

#pragma once

#include "kernels.cuh"

namespace crb {

struct Queues {
  uint32_t* q0;   // QS, then QM3
  uint32_t* q1;   // QSP
  uint32_t* q2;   // QT
  unsigned int* n;  // [0] QS, [1] QSP, [2] QM3, [3] QT, [4] flagged pixels
};

// frame of global pixel index g (frames sorted by first pixel)
__device__ __forceinline__ int frame_of_pixel(const Frame* frames, int nframes, long long g) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].pix0 <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// frame of word block b (frames sorted by first block)
__device__ __forceinline__ int frame_of_block(const Frame* frames, int nframes, long long b) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].blk0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kBW = 8;   // words (32 px each) per block row: one warp per word column
constexpr int kBH = 32;  // rows per block

// ---------------------------------------------------------------------------------------------
// bound_kernel: per pixel L+ and the lower bound of m5 (smallest of the five
// column medians) -> bits of S+ > sigclip and S+ > sigfrac*sigclip (see
// detect_tile for the bound and its margin). One warp walks down one 32-pixel
// word column of kBH rows, two rows per step, keeping the rows of its column
// (and of the two halo columns on each side, held by lanes 0-3) in registers.
//
// Sliding column medians: the windows of rows y and y+1 share the four values
// of rows y-1..y+2. With c1 <= c2 the two middle values of those four, the
// median of the four and one more value e is min(max(e, c1), c2); the pair
// (min, max) of rows y+1, y+2 is shared with the next step.
struct ColPair {  // running state of one column
  float lo, hi;   // min / max of the last row pair
};

__device__ __forceinline__ float clamp_med(float e, float c1, float c2) { return fminf(fmaxf(e, c1), c2); }

__global__ void __launch_bounds__(256) bound_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks,
                                                    Params p, int k, int niter) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float sigclip = p.sigclip, siglow = __fmul_rn(p.sigfrac, p.sigclip);
  const float chot = 4.f * sigclip * sigclip * 0.9999f, clow = 4.f * siglow * siglow * 0.9999f;
  // halo routing: src lane of the column median at x-2 (lanes 0,1) or x+2 (30,31); at x-1 (0) or x+1 (31)
  const int srcA = lane == 0 ? 0 : lane == 1 ? 1 : lane == 30 ? 2 : 3;
  const int srcB = lane == 0 ? 1 : 2;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int wc = bxs * kBW + warp;
    if (wc >= f.wpr) continue;  // whole warp
    const int w = f.w, h = f.h;
    const float* __restrict__ J = iter_src(f, k, niter);
    const float gain = f.gain, rn2 = __fmul_rn(f.rn, f.rn), g2 = __fmul_rn(f.gain, f.gain);
    const int x0 = wc * 32, x = x0 + lane;
    const int col = min(x, w - 1);
    const int hx = lane < 2 ? x0 - 2 + lane : x0 + 30 + lane;  // halo columns (lanes 0-3)
    const int hcol = clampi(hx, 0, w - 1);
    const int y0 = bys * kBH, y1 = min(y0 + kBH, h);
    const float* __restrict__ Jc = J + col;
    const float* __restrict__ Jh = J + hcol;
    auto rowp = [&](int yy) { return size_t(clampi(yy, 0, h - 1)) * size_t(w); };
    // rows y0-2 .. y0+1 of the column (a..d) and of the halo column
    float a = __ldg(Jc + rowp(y0 - 2)), bq = __ldg(Jc + rowp(y0 - 1));
    float cq = __ldg(Jc + rowp(y0)), d = __ldg(Jc + rowp(y0 + 1));
    float ha = __ldg(Jh + rowp(y0 - 2)), hb = __ldg(Jh + rowp(y0 - 1));
    float hc = __ldg(Jh + rowp(y0)), hd = __ldg(Jh + rowp(y0 + 1));
    for (int y = y0; y < y1; y += 2) {
      // next two rows y+2, y+3
      const float e = __ldg(Jc + rowp(y + 2)), g = __ldg(Jc + rowp(y + 3));
      const float he = __ldg(Jh + rowp(y + 2)), hg = __ldg(Jh + rowp(y + 3));
      // core rows y-1..y+2 = (bq, cq) and (d, e): middle two values
      float cm0, cm1, hcm0, hcm1;
      {
        const float l1 = fminf(bq, cq), h1 = fmaxf(bq, cq), l2 = fminf(d, e), h2 = fmaxf(d, e);
        const float u = fmaxf(l1, l2), v = fminf(h1, h2);
        const float c1 = fminf(u, v), c2 = fmaxf(u, v);
        cm0 = clamp_med(a, c1, c2);   // rows y-2..y+2
        cm1 = clamp_med(g, c1, c2);   // rows y-1..y+3
        const float hl1 = fminf(hb, hc), hh1 = fmaxf(hb, hc), hl2 = fminf(hd, he), hh2 = fmaxf(hd, he);
        const float hu = fmaxf(hl1, hl2), hv = fminf(hh1, hh2);
        const float hc1 = fminf(hu, hv), hc2 = fmaxf(hu, hv);
        hcm0 = clamp_med(ha, hc1, hc2);
        hcm1 = clamp_med(hg, hc1, hc2);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int yy = y + s;
        if (yy >= y1) break;
        const float cm = s ? cm1 : cm0, hcm = s ? hcm1 : hcm0;
        float m2 = __shfl_up_sync(0xffffffffu, cm, 2), m1 = __shfl_up_sync(0xffffffffu, cm, 1);
        float p1 = __shfl_down_sync(0xffffffffu, cm, 1), p2 = __shfl_down_sync(0xffffffffu, cm, 2);
        const float hA = __shfl_sync(0xffffffffu, hcm, srcA), hB = __shfl_sync(0xffffffffu, hcm, srcB);
        if (lane < 2) m2 = hA;
        if (lane == 0) m1 = hB;
        if (lane >= 30) p2 = hA;
        if (lane == 31) p1 = hB;
        const float mlow = min3f(min3f(m2, m1, cm), p1, p2);
        // L+: the pixel, its column neighbours and its row neighbours (lanes, halo at the ends)
        const float cc = s ? d : cq, up = s ? cq : bq, dn = s ? e : d;
        const float hcc = s ? hd : hc;
        const float hL = __shfl_sync(0xffffffffu, hcc, lane == 0 ? 1 : 2);
        float left = __shfl_up_sync(0xffffffffu, cc, 1), right = __shfl_down_sync(0xffffffffu, cc, 1);
        if (lane == 0) left = hL;
        if (lane == 31) right = hL;
        const float lp = lplus(cc, up, dn, left, right);
        const float den = gain * (mlow > 0.f ? mlow : 0.f) + rn2;
        const float lhs = lp * lp * g2;
        const bool ok = x < w;
        const unsigned act = __ballot_sync(0xffffffffu, ok && lhs > clow * den);
        const unsigned hot = __ballot_sync(0xffffffffu, ok && lhs > chot * den);
        if (lane == 0) {
          const size_t o = size_t(yy) * f.wpr + wc;
          f.act[o] = act;
          f.hot[o] = hot;
          f.test[o] = 0u;
        }
      }
      a = cq; bq = d; cq = e; d = g;
      ha = hc; hb = hd; hc = he; hd = hg;
    }
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

// Appends, for each thread's word `v` at (wc, y) of frame f, the set bits as
// global pixel indices to queue q (counter *n); one atomic per block.
__device__ __forceinline__ void emit_word(uint32_t v, const Frame& f, int wc, int y, uint32_t* q, unsigned int* n,
                                          int* ws) {
  int total = 0;
  const int off = block_excl_scan(__popc(v), ws, total);
  __shared__ unsigned int base;
  if (threadIdx.x == 0) base = total ? atomicAdd(n, (unsigned int)total) : 0u;
  __syncthreads();
  unsigned int o = base + off;
  const uint32_t row = uint32_t(f.pix0 + (long long)y * f.w + 32 * wc);
  while (v) {
    const int bb = __ffs(v) - 1;
    v &= v - 1u;
    q[o++] = row + bb;
  }
  __syncthreads();
}

// need_kernel: needS' = dilate5(hot) & act, needS = dilate5(needS') within the
// frame -> queues QS, QSP and the bit plane nsp.
__global__ void __launch_bounds__(256) need_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks,
                                                   Queues Q) {
  // rows y0-4 .. y0+kBH+3 (kBH + 8), words wc0-1 .. wc0+kBW (kBW + 2)
  constexpr int RW = kBW + 2, RR = kBH + 8;
  __shared__ uint32_t sHot[RR][RW], sAct[RR][RW], sNsp[RR][RW];
  __shared__ int ws[kThreads / 32 + 1];
  const int t = threadIdx.x;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int wc0 = bxs * kBW, y0 = bys * kBH;
    for (int i = t; i < RR * RW; i += kThreads) {
      const int rr = i / RW, cc = i - rr * RW;
      const int y = y0 - 4 + rr, wc = wc0 - 1 + cc;
      const bool in = y >= 0 && y < f.h && wc >= 0 && wc < f.wpr;
      sHot[rr][cc] = in ? f.hot[size_t(y) * f.wpr + wc] : 0u;
      sAct[rr][cc] = in ? f.act[size_t(y) * f.wpr + wc] : 0u;
    }
    __syncthreads();
    // needS' on rows y0-2 .. y0+kBH+1 (kBH + 4), all RW words
    for (int i = t; i < (kBH + 4) * RW; i += kThreads) {
      const int rr = i / RW + 2, cc = i - (i / RW) * RW;
      uint32_t a = 0, l = 0, r = 0;
#pragma unroll
      for (int d = -2; d <= 2; ++d) {
        a |= sHot[rr + d][cc];
        if (cc > 0) l |= sHot[rr + d][cc - 1];
        if (cc < RW - 1) r |= sHot[rr + d][cc + 1];
      }
      sNsp[rr][cc] = hdil<2>(l, a, r) & sAct[rr][cc];
    }
    __syncthreads();
    // the block's own words: needS = dilate5(needS') in the frame; emit both queues
    const int rr = t / kBW + 4, cc = t % kBW + 1;
    const int y = y0 + t / kBW, wc = wc0 + t % kBW;
    const bool mine = y < f.h && wc < f.wpr;
    uint32_t a = 0, l = 0, r = 0;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
      a |= sNsp[rr + d][cc];
      l |= sNsp[rr + d][cc - 1];
      r |= sNsp[rr + d][cc + 1];
    }
    const uint32_t needS = mine ? (hdil<2>(l, a, r) & frame_word(wc, f.w)) : 0u;
    const uint32_t needSp = mine ? sNsp[rr][cc] : 0u;
    if (mine) f.nsp[size_t(y) * f.wpr + wc] = needSp;
    emit_word(needS, f, wc, y, Q.q0, Q.n + 0, ws);
    emit_word(needSp, f, wc, y, Q.q1, Q.n + 1, ws);
  }
}

// m3need_kernel: needM3 = dilate7(test) within the frame -> queue QM3.
__global__ void __launch_bounds__(256) m3need_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks,
                                                     Queues Q) {
  constexpr int RW = kBW + 2, RR = kBH + 6;
  __shared__ uint32_t sT[RR][RW];
  __shared__ int ws[kThreads / 32 + 1];
  const int t = threadIdx.x;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int wc0 = bxs * kBW, y0 = bys * kBH;
    for (int i = t; i < RR * RW; i += kThreads) {
      const int rr = i / RW, cc = i - rr * RW;
      const int y = y0 - 3 + rr, wc = wc0 - 1 + cc;
      sT[rr][cc] = (y >= 0 && y < f.h && wc >= 0 && wc < f.wpr) ? f.test[size_t(y) * f.wpr + wc] : 0u;
    }
    __syncthreads();
    const int rr = t / kBW + 3, cc = t % kBW + 1;
    const int y = y0 + t / kBW, wc = wc0 + t % kBW;
    uint32_t a = 0, l = 0, r = 0;
#pragma unroll
    for (int d = -3; d <= 3; ++d) {
      a |= sT[rr + d][cc];
      l |= sT[rr + d][cc - 1];
      r |= sT[rr + d][cc + 1];
    }
    const uint32_t need = (y < f.h && wc < f.wpr) ? (hdil<3>(l, a, r) & frame_word(wc, f.w)) : 0u;
    emit_word(need, f, wc, y, Q.q0, Q.n + 2, ws);
  }
}

// ---------------------------------------------------------------------------------------------
// Queue kernels: one thread per entry, grid-stride over the queue length.

struct Pix {
  int fi, x, y;
};

__device__ __forceinline__ Pix decode(const Frame* frames, int nframes, uint32_t g) {
  Pix p;
  p.fi = frame_of_pixel(frames, nframes, (long long)g);
  const uint32_t o = g - uint32_t(frames[p.fi].pix0);
  const int w = frames[p.fi].w;
  p.y = int(o / uint32_t(w));
  p.x = int(o - uint32_t(p.y) * uint32_t(w));
  return p;
}

// s_kernel: at QS, m5 (floored), N, L+ and S of J.
__global__ void __launch_bounds__(256) s_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, int k,
                                                int niter) {
  const unsigned int n = Q.n[0];
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q0[i];
    const Pix P = decode(frames, nframes, g);
    const Frame& f = frames[P.fi];
    const float* __restrict__ J = iter_src(f, k, niter);
    int xs[5];
    size_t ro[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      xs[d] = clampi(P.x - 2 + d, 0, f.w - 1);
      ro[d] = size_t(clampi(P.y - 2 + d, 0, f.h - 1)) * f.w;
    }
    float v[25];
#pragma unroll
    for (int dy = 0; dy < 5; ++dy)
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = __ldg(J + ro[dy] + xs[dx]);
    const float lp = lplus(v[12], v[7], v[17], v[11], v[13]);
    const float m5f = floor_m5(sel_med25(v));
    const float nn = noise_of(m5f, f.gain, __fmul_rn(f.rn, f.rn));
    const size_t o = size_t(g - uint32_t(f.pix0));
    f.mapS[o] = __fdiv_rn(lp, __fmul_rn(2.f, nn));
    f.mapN[o] = nn;
  }
}

// sp_kernel: at QSP, S' = S - med5(S); S' > sigclip -> test bit and queue QT.
__global__ void __launch_bounds__(256) sp_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, Params p) {
  const unsigned int n = Q.n[1];
  const unsigned int stride = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (unsigned int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // whole warps iterate together
    const unsigned int i = i0 + threadIdx.x;
    bool test = false;
    uint32_t g = 0;
    if (i < n) {
      g = Q.q1[i];
      const Pix P = decode(frames, nframes, g);
      const Frame& f = frames[P.fi];
      int xs[5];
      size_t ro[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        xs[d] = clampi(P.x - 2 + d, 0, f.w - 1);
        ro[d] = size_t(clampi(P.y - 2 + d, 0, f.h - 1)) * f.w;
      }
      float v[25];
#pragma unroll
      for (int dy = 0; dy < 5; ++dy)
#pragma unroll
        for (int dx = 0; dx < 5; ++dx) v[dy * 5 + dx] = f.mapS[ro[dy] + xs[dx]];
      const float sp = __fsub_rn(v[12], sel_med25(v));
      const size_t o = size_t(g - uint32_t(f.pix0));
      f.mapSp[o] = sp;
      test = sp > p.sigclip;
      if (test) atomicOr(&f.test[size_t(P.y) * f.wpr + (P.x >> 5)], 1u << (P.x & 31));
    }
    const unsigned m = __ballot_sync(0xffffffffu, test);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned int base = 0;
      if (lane == leader) base = atomicAdd(Q.n + 3, (unsigned int)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (test) Q.q2[base + __popc(m & ((1u << lane) - 1u))] = g;
    }
  }
}

// m3_kernel: at QM3, med3 of J.
__global__ void __launch_bounds__(256) m3_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, int k,
                                                 int niter) {
  const unsigned int n = Q.n[2];
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q0[i];
    const Pix P = decode(frames, nframes, g);
    const Frame& f = frames[P.fi];
    const float* __restrict__ J = iter_src(f, k, niter);
    int xs[3];
    size_t ro[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xs[d] = clampi(P.x - 1 + d, 0, f.w - 1);
      ro[d] = size_t(clampi(P.y - 1 + d, 0, f.h - 1)) * f.w;
    }
    float v[9];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = __ldg(J + ro[dy] + xs[dx]);
    f.mapM3[size_t(g - uint32_t(f.pix0))] = sel_med9(v);
  }
}

// cand_kernel: at QT, F = m3 - med7(m3), the objlim statistic, and for each
// candidate the first growth (S' > sigclip) and the second (S' > sigfrac*sigclip)
// ORed into the flag bits of M_k; counts the new flags of each frame.
// S' is read only where the bit plane nsp says it was computed; elsewhere it
// cannot pass a threshold.
__global__ void __launch_bounds__(256) cand_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, Params p,
                                                   int k) {
  const unsigned int n = Q.n[3];
  const float sigclip = p.sigclip, siglow = __fmul_rn(p.sigfrac, p.sigclip);
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q2[i];
    const Pix P = decode(frames, nframes, g);
    const Frame& f = frames[P.fi];
    const int w = f.w, h = f.h;
    int xs[7];
    size_t ro[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      xs[d] = clampi(P.x - 3 + d, 0, w - 1);
      ro[d] = size_t(clampi(P.y - 3 + d, 0, h - 1)) * w;
    }
    float u[49];
#pragma unroll
    for (int dy = 0; dy < 7; ++dy)
#pragma unroll
      for (int dx = 0; dx < 7; ++dx) u[dy * 7 + dx] = f.mapM3[ro[dy] + xs[dx]];
    const size_t o = size_t(g - uint32_t(f.pix0));
    const float fval = __fsub_rn(u[24], sel_med49(u));
    const float fn = fmaxf(__fdiv_rn(fval, f.mapN[o]), 0.01f);
    const float rval = (p.objlim_form == 1) ? __fdiv_rn(__fmul_rn(2.f, f.mapS[o]), fn) : __fdiv_rn(f.mapSp[o], fn);
    if (!(rval > p.objlim)) continue;
    unsigned int fresh = 0;
    for (int qy = max(P.y - 1, 0); qy <= min(P.y + 1, h - 1); ++qy)
      for (int qx = max(P.x - 1, 0); qx <= min(P.x + 1, w - 1); ++qx) {
        if (!((f.nsp[size_t(qy) * f.wpr + (qx >> 5)] >> (qx & 31)) & 1u)) continue;
        if (!(f.mapSp[size_t(qy) * w + qx] > sigclip)) continue;  // first growth
        for (int ry = max(qy - 1, 0); ry <= min(qy + 1, h - 1); ++ry)
          for (int rx = max(qx - 1, 0); rx <= min(qx + 1, w - 1); ++rx) {
            const size_t wo = size_t(ry) * f.wpr + (rx >> 5);
            const uint32_t bit = 1u << (rx & 31);
            if (!(f.nsp[wo] & bit)) continue;
            if (!(f.mapSp[size_t(ry) * w + rx] > siglow)) continue;  // second growth
            if (f.bits_a[wo] & bit) continue;                        // already flagged
            const uint32_t old = atomicOr(&f.bits_a[wo], bit);
            fresh += (old & bit) ? 0u : 1u;
          }
      }
    if (fresh) atomicAdd(f.counters + 2 * (k - 1), (unsigned long long)fresh);
  }
}

// ---------------------------------------------------------------------------------------------
// Replacement (stage e) over a queue of the flagged pixels. Both image buffers
// start as copies of I0, so unflagged pixels are never written and every
// iteration only writes its flagged pixels (see replace_tile for the
// +/-inf form of the lower median).

// init_images_kernel: I0 into both image buffers of every frame (out_clean and,
// for niter >= 2, ws). Pointers come from the descriptors, so a captured graph
// replays correctly for new frames.
__global__ void __launch_bounds__(256) init_images_kernel(const Frame* __restrict__ frames, int nframes) {
  const size_t t0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x, stride = size_t(gridDim.x) * blockDim.x;
  for (int fi = 0; fi < nframes; ++fi) {
    const float* __restrict__ src = frames[fi].img;
    float* __restrict__ a = frames[fi].out_clean;
    float* __restrict__ b = frames[fi].ws;
    const size_t n = size_t(frames[fi].w) * size_t(frames[fi].h);
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(a) |
                       reinterpret_cast<uintptr_t>(b)) & 15u) == 0;
    size_t done = 0;
    if (vec) {
      const size_t n4 = n / 4;
      for (size_t i = t0; i < n4; i += stride) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(src) + i);
        reinterpret_cast<float4*>(a)[i] = v;
        if (b) reinterpret_cast<float4*>(b)[i] = v;
      }
      done = n4 * 4;
    }
    for (size_t i = done + t0; i < n; i += stride) {
      const float v = __ldg(src + i);
      a[i] = v;
      if (b) b[i] = v;
    }
  }
}

// flagq_kernel: the flagged pixels of M_k -> queue q1 (counter n[4]).
__global__ void __launch_bounds__(256) flagq_kernel(const Frame* __restrict__ frames, int nframes, long long nblocks,
                                                    Queues Q) {
  __shared__ int ws[kThreads / 32 + 1];
  const int t = threadIdx.x;
  for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int fi = frame_of_block(frames, nframes, b);
    const Frame& f = frames[fi];
    const long long lb = b - f.blk0;
    const int bys = int(lb / f.bx), bxs = int(lb - (long long)bys * f.bx);
    const int y = bys * kBH + t / kBW, wc = bxs * kBW + t % kBW;
    const uint32_t v = (y < f.h && wc < f.wpr) ? (f.bits_a[size_t(y) * f.wpr + wc] & frame_word(wc, f.w)) : 0u;
    emit_word(v, f, wc, y, Q.q1, Q.n + 4, ws);
  }
}

// rep_kernel: I_k at the queued flagged pixels, from J = I_{k-1} and M_k.
__global__ void __launch_bounds__(256) rep_kernel(const Frame* __restrict__ frames, int nframes, Queues Q, int k,
                                                  int niter) {
  const unsigned int n = Q.n[4];
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = Q.q1[i];
    const Pix P = decode(frames, nframes, g);
    const Frame& f = frames[P.fi];
    const float* __restrict__ J = iter_src(f, k, niter);
    const uint32_t* __restrict__ M = f.bits_a;
    int xs[5], ys[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      xs[d] = clampi(P.x - 2 + d, 0, f.w - 1);
      ys[d] = clampi(P.y - 2 + d, 0, f.h - 1);
    }
    uint32_t win = 0;  // 25 window flags, row-major
    float v[25];
#pragma unroll
    for (int dy = 0; dy < 5; ++dy)
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) {
        const int q = dy * 5 + dx;
        v[q] = __ldg(J + size_t(ys[dy]) * f.w + xs[dx]);
        win |= ((__ldg(M + size_t(ys[dy]) * f.wpr + (xs[dx] >> 5)) >> (xs[dx] & 31)) & 1u) << q;
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
    }
    iter_dst(f, k, niter)[size_t(g - uint32_t(f.pix0))] = out;
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

// Adds the queue lengths of this iteration to the work counters of frame 0
// (the totals of the call) and clears them for the next iteration.
__global__ void queue_work_kernel(const Frame* __restrict__ frames, Queues Q, int k, long long dense) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long* wk = frames[0].work + 5 * (k - 1);
    wk[0] += Q.n[0];
    wk[1] += Q.n[1];
    wk[2] += Q.n[2];
    wk[3] += Q.n[3];
    wk[4] += (unsigned long long)dense;
    for (int i = 0; i < 5; ++i) Q.n[i] = 0u;
  }
}

}  // namespace crb
