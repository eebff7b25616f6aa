// C ABI of the cleaner (declarations and contracts in include/crb.h).
//
// A call validates its arguments, sizes the context's workspace, writes one
// descriptor per frame and enqueues, per iteration, one detection launch and
// one replacement launch over the tiles of all its frames. Calls on one
// context are ordered (each waits for the previous one's completion event),
// so descriptors and workspace can be reused.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "alu_peak.cuh"
#include "crb.h"
#include "kernels.cuh"
#include "pipeline.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? CRB_ENOMEM : CRB_ECUDA;
}

#define CRB_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

using DetectFn = void (*)(const crb::Frame*, int, long long, crb::Params, int, int);
using ReplaceFn = void (*)(const crb::Frame*, int, long long, int, int, int);

struct DetectShape {
  int tw, th;
  DetectFn fn, fn_maps, fn_fused;
  size_t smem, smem_fused;
};

template <int TW, int TH>
DetectShape make_detect() {
  return DetectShape{TW, TH, crb::detect_kernel<TW, TH, false, false>, crb::detect_kernel<TW, TH, true, false>,
                     crb::detect_kernel<TW, TH, false, true>, crb::DetectLayout<TW, TH, false>::bytes,
                     crb::DetectLayout<TW, TH, true>::bytes};
}

// One image buffer and three resident blocks per SM (at most 80 registers and
// 75 KB of shared memory each): for calls whose tiles all fit in one round.
template <int TW, int TH>
DetectShape make_detect_single() {
  return DetectShape{TW, TH, crb::detect1_kernel<TW, TH, false, false>, crb::detect1_kernel<TW, TH, true, false>,
                     crb::detect1_kernel<TW, TH, false, true>,
                     crb::DetectLayout<TW, TH, false, false>::bytes, crb::DetectLayout<TW, TH, true, false>::bytes};
}

const std::vector<DetectShape>& detect_shapes() {
  static const std::vector<DetectShape> v = {make_detect<64, 32>(), make_detect<32, 32>(),
                                             make_detect<64, 16>(), make_detect<128, 32>(),
                                             make_detect<64, 64>(), make_detect_single<64, 28>()};
  return v;
}

// tile_shape 0 takes 64 x 32 tiles, or the single-buffered 64 x 28 tiles when
// all of those fit in one round of resident blocks and the 64 x 32 tiles do
// not. A tile's detection is a chain of block-wide phases whose latency, not
// an issue or memory rate, bounds the launch, so a second round of a few tiles
// costs nearly a whole tile latency (one 800 x 800 frame: 325 tiles of 64 x 32
// on 152 SMs x 2 blocks; 377 tiles of 64 x 28 on 152 x 3).
constexpr int kOneRoundShape = 5;

constexpr int kRW = 64, kRH = 16;  // replacement tile
const ReplaceFn kReplace = crb::replace_kernel<kRW, kRH>;
constexpr size_t kReplaceSmem = crb::ReplaceLayout<kRW, kRH>::bytes;

// Two iterations in one launch (crb_options.fuse2): 64 x 16 tiles, the tile
// shape of index kFuse2Shape, for the other launches of such a call too.
constexpr int kFuse2Shape = 2;
const DetectFn kDetect2 = crb::detect2_kernel<64, 16>;
constexpr size_t kDetect2Smem = crb::Detect2Layout<64, 16>::bytes;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// profiling kinds (crb_profile_kernels order); kinds below kProfReplace0 are detection
enum ProfKind {
  kPBound, kPNeed, kPS, kPSp, kPM3need, kPM3, kPCand, kPGrow, kPReserved, kPTileDetect,  // detection
  kPRep, kPMask, kPTileReplace,                                                      // replacement
  kPWork,                                                                             // work counters
  kProfKinds
};
constexpr int kProfReplace0 = kPRep;

// crb_clean_batch_host: staging slots and chunks per call
constexpr int kStageSlots = 4, kStageChunks = 8;
// descriptor buffers per context
constexpr int kDescSlots = 4;

// queue pipeline kernels, for the occupancy table
enum QK {
  kQBound, kQNeed, kQS, kQSp, kQM3need, kQM3, kQCand, kQRepCompute, kQBoundSparse, kQRq, kQRepWrite, kQD2,
  kQCandFull, kQGrow, kQMask, kQSegList, kQD2Seg, kQNeedSeg, kQM3needSeg, kQM3needAll, kQGrowFirst, kQKernels
};

struct GraphKey {
  int n, niter, shape;
  bool fuse, fuse2, queue;
  int seg_from;
  long long occ_sig;  // the queue kernels' blocks per SM, packed
  long long tiles, rtiles, nblocks, ncells, npix;
  size_t bits_total;
  int ncounters, dgrid, fgrid, rgrid;
  void* ws;
  void* counters;
  void* frames;
  void* tab;
  bool operator==(const GraphKey& o) const {
    return n == o.n && niter == o.niter && shape == o.shape && fuse == o.fuse && fuse2 == o.fuse2 && queue == o.queue &&
           seg_from == o.seg_from && occ_sig == o.occ_sig &&
           tiles == o.tiles && nblocks == o.nblocks && ncells == o.ncells && npix == o.npix &&
           rtiles == o.rtiles && bits_total == o.bits_total && ncounters == o.ncounters && dgrid == o.dgrid &&
           fgrid == o.fgrid && rgrid == o.rgrid && ws == o.ws && counters == o.counters && frames == o.frames &&
           tab == o.tab;
  }
};

struct FrameSpec {
  const float* img;
  float* out_clean;
  uint8_t* out_mask;
  float* maps;
  const uint8_t* mprev;  // crb_iterate only
  int w, h;
  float gain, rn;
};

}  // namespace

// Lets the library's other translation units report a message through crb_last_error().
void crb_detail_set_error(const char* msg) { g_err = msg ? msg : ""; }

struct crb_ctx {
  crb::Params p{};
  float gain = 0, rn = 0;
  int niter = 0;
  crb_options opt{};
  int device = 0, num_sms = 0;
  std::vector<int> occ_detect, occ_detect_maps, occ_fused;
  int occ_q[kQKernels] = {};  // queue pipeline kernels (QK order)
  int occ_replace = 0;
  int occ_detect2 = 0;

  void* ws = nullptr;
  size_t ws_bytes = 0;
  // Descriptors (and the queue pipeline's frame table: frame of each
  // 2^kTabShift pixels) are staged in a ring of kDescSlots page-locked host
  // buffers, so that a call waits only for the upload of the call kDescSlots
  // back before refilling one, and uploaded into one device buffer of the
  // context: calls on a context are ordered (each starts after the previous
  // one's completion event), so no kernel still reads the device copy when the
  // next upload overwrites it, and a captured graph always finds its
  // descriptors at the same address. The fields below view the slot of the
  // current call.
  struct DescSlot {
    crb::Frame* h_frames = nullptr;
    uint32_t* h_tab = nullptr;
    CUtensorMap* h_maps = nullptr;  // tile pipeline: 3 per frame (capacity 3 * frames_cap)
    int frames_cap = 0;
    size_t tab_cap = 0;
    cudaEvent_t upload_ev = nullptr;
  } slot[kDescSlots];
  int cur = 0;
  crb::Frame* d_frames = nullptr;  // device descriptors (capacity d_frames_cap)
  crb::Frame* h_frames = nullptr;  // pinned staging of the current slot
  CUtensorMap* d_maps = nullptr;   // device tensor maps (capacity 3 * d_frames_cap)
  CUtensorMap* h_maps = nullptr;   // pinned staging of the current slot
  size_t maps_n = 0;               // tensor maps the current call uploads
  unsigned int* d_status = nullptr;  // device status word: a kernel's bounded wait gave up
  uint32_t* d_tab = nullptr;       // device frame table (capacity d_tab_cap)
  uint32_t* h_tab = nullptr;
  int d_frames_cap = 0;
  size_t d_tab_cap = 0;
  size_t tab_n = 0;  // entries
  unsigned long long* d_counters = nullptr;
  int counters_cap = 0;  // in unsigned long longs
  int last_niter = 0;
  int last_launches = 0;  // kernels the work of the last call launches
  int mprev_frames = 0;   // crb_iterate: frames given an explicit M_{k-1}
  int last_nframes = 0;
  cudaEvent_t upload_ev = nullptr, done_ev = nullptr;  // upload_ev: the current slot's
  bool any_call = false;
  int latched = CRB_OK;

  // graphs of the work of a call, by launch signature; autotuned tile shape by frame sizes
  std::vector<std::pair<GraphKey, cudaGraphExec_t>> graphs;
  cudaStream_t cap_stream = nullptr;

  // crb_clean_batch_host: copy-in, clean and copy-out streams, kStageSlots device
  // staging slots; chunks alternate between this context and a twin (own
  // workspace, own clean stream), so that consecutive chunks' cleans overlap
  crb_ctx* twin = nullptr;
  cudaStream_t hs_in = nullptr, hs_cmp = nullptr, hs_cmp2 = nullptr, hs_out = nullptr;
  cudaEvent_t h_entry = nullptr, h_in[kStageSlots] = {}, h_cmp[kStageSlots] = {}, h_free[kStageSlots] = {};
  char* d_stage[kStageSlots] = {};
  size_t stage_cap = 0;
  // crb_clean_rects: the crops (input, cleaned, mask) of the rectangles of a call
  char* d_rects = nullptr;
  size_t rects_cap = 0;
  std::vector<std::pair<std::vector<long long>, int>> tuned;

  // queue-pipeline autotuner (crb_options.autotune): the chosen launch
  // configuration of each call signature, and the per-launch events of a trial
  struct QTune {
    std::vector<long long> sig;
    int occ[kQKernels];
    int seg_from;
    bool tile;  // the tile pipeline measured faster for this signature
  };
  std::vector<QTune> qtuned;
  bool tuning = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> tune_ev;
  int last_occ[kQKernels] = {};
  int last_seg_from = 0, last_pipeline = 0;
  // profiling: event pairs around launches, by kernel kind (0 detect, 1 replace)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[kProfKinds];
  double prof_ms[kProfKinds] = {};
  int prof_n[kProfKinds] = {};
};

// Lets the server turn graph replay on for the calls whose signature repeats (single-frame waves).
void crb_detail_set_graphs(crb_ctx* c, int on) {
  if (c) c->opt.use_graphs = on;
}

namespace {

int init_ctx(crb_ctx* c) {
  CRB_CUDA(cudaGetDevice(&c->device));
  CRB_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  for (const auto& s : detect_shapes()) {
    int occ = 0, occm = 0, occf = 0;
    CRB_CUDA(cudaFuncSetAttribute(s.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem)));
    CRB_CUDA(cudaFuncSetAttribute(s.fn_maps, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem)));
    CRB_CUDA(cudaFuncSetAttribute(s.fn_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem_fused)));
    CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, s.fn, crb::kThreads, s.smem));
    CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occm, s.fn_maps, crb::kThreads, s.smem));
    CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occf, s.fn_fused, crb::kThreads, s.smem_fused));
    if (&s == &detect_shapes()[kOneRoundShape])  // three blocks need the largest shared-memory carveout
      for (DetectFn fn : {s.fn, s.fn_maps, s.fn_fused})
        CRB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      int(cudaSharedmemCarveoutMaxShared)));
    c->occ_detect.push_back(occ > 0 ? occ : 1);
    c->occ_detect_maps.push_back(occm > 0 ? occm : 1);
    c->occ_fused.push_back(occf > 0 ? occf : 1);
  }
  {
    const void* fns[kQKernels] = {
        reinterpret_cast<const void*>(crb::bound_dense_kernel),      reinterpret_cast<const void*>(crb::need_kernel),
        reinterpret_cast<const void*>(crb::s_kernel),           reinterpret_cast<const void*>(crb::sp_kernel),
        reinterpret_cast<const void*>(crb::m3need_kernel<false>), reinterpret_cast<const void*>(crb::m3_kernel),
        reinterpret_cast<const void*>(crb::cand_test_kernel),   reinterpret_cast<const void*>(crb::rep_compute_kernel),
        reinterpret_cast<const void*>(crb::bound_sparse_kernel),   reinterpret_cast<const void*>(crb::rq_kernel),
        reinterpret_cast<const void*>(crb::rep_write_kernel),   reinterpret_cast<const void*>(crb::d2_kernel),
        reinterpret_cast<const void*>(crb::cand_full_kernel),   reinterpret_cast<const void*>(crb::grow_kernel),
        reinterpret_cast<const void*>(crb::mask_kernel),        reinterpret_cast<const void*>(crb::seg_list_kernel),
        reinterpret_cast<const void*>(crb::d2_seg_kernel),      reinterpret_cast<const void*>(crb::need_seg_kernel),
        reinterpret_cast<const void*>(crb::m3need_seg_kernel),  reinterpret_cast<const void*>(crb::m3need_kernel<true>),
        reinterpret_cast<const void*>(crb::grow_first_kernel)};
    for (int i = 0; i < kQKernels; ++i) {
      int o = 0;
      const bool col = i == kQNeed || i == kQM3need || i == kQD2 || i == kQD2Seg || i == kQNeedSeg ||
                       i == kQM3needSeg || i == kQM3needAll || i == kQGrowFirst;
      const int threads = i == kQBound ? crb::kBoundThreads : col ? crb::kColWarps * 32 : 256;
      CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fns[i], threads, 0));
      c->occ_q[i] = o > 0 ? o : 1;
    }
  }
  CRB_CUDA(cudaFuncSetAttribute(kDetect2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDetect2Smem)));
  CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_detect2, kDetect2, crb::kThreads, kDetect2Smem));
  if (c->occ_detect2 < 1) c->occ_detect2 = 1;
  CRB_CUDA(cudaFuncSetAttribute(kReplace, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kReplaceSmem)));
  CRB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->occ_replace, kReplace, crb::kThreads, kReplaceSmem));
  if (c->occ_replace < 1) c->occ_replace = 1;
  for (auto& sl : c->slot) CRB_CUDA(cudaEventCreateWithFlags(&sl.upload_ev, cudaEventDisableTiming));
  c->upload_ev = c->slot[0].upload_ev;
  CRB_CUDA(cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming));
  CRB_CUDA(cudaMalloc(&c->d_status, 256));
  CRB_CUDA(cudaMemset(c->d_status, 0, 256));
  return CRB_OK;
}

cudaEvent_t take_event(crb_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch bracketed by events when profiling (kind 0 detect, 1 replace).
template <typename F>
void timed(crb_ctx* c, int kind, cudaStream_t stream, F&& launch) {
  if (!c->opt.profile) {
    launch();
    return;
  }
  cudaEvent_t a = take_event(c), b = take_event(c);
  cudaEventRecord(a, stream);
  launch();
  cudaEventRecord(b, stream);
  c->pending[kind].emplace_back(a, b);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

// Moves to the next descriptor slot, with room for n frames and tab_entries
// table entries, once the slot's previous upload has run; sets the views and
// grows the device copies if needed.
int next_desc_slot(crb_ctx* c, int n, size_t tab_entries) {
  c->cur = (c->cur + 1) % kDescSlots;
  crb_ctx::DescSlot& S = c->slot[c->cur];
  // generous first capacities, so that growing (which synchronises the device) is rare
  n = std::max(n, 64);
  tab_entries = std::max<size_t>(tab_entries, 8192);
  if (n > S.frames_cap || tab_entries > S.tab_cap || n > c->d_frames_cap || tab_entries > c->d_tab_cap) {
    CRB_CUDA(cudaDeviceSynchronize());
    if (n > S.frames_cap) {
      cudaFreeHost(S.h_frames);
      cudaFreeHost(S.h_maps);
      S.h_frames = nullptr;
      S.h_maps = nullptr;
      S.frames_cap = 0;
      CRB_CUDA(cudaMallocHost(&S.h_frames, sizeof(crb::Frame) * size_t(n)));
      CRB_CUDA(cudaMallocHost(&S.h_maps, sizeof(CUtensorMap) * 3 * size_t(n)));
      S.frames_cap = n;
    }
    if (tab_entries > S.tab_cap) {
      cudaFreeHost(S.h_tab);
      S.h_tab = nullptr;
      S.tab_cap = 0;
      CRB_CUDA(cudaMallocHost(&S.h_tab, sizeof(uint32_t) * tab_entries));
      S.tab_cap = tab_entries;
    }
    if (n > c->d_frames_cap) {
      cudaFree(c->d_frames);
      cudaFree(c->d_maps);
      c->d_frames = nullptr;
      c->d_maps = nullptr;
      c->d_frames_cap = 0;
      CRB_CUDA(cudaMalloc(&c->d_frames, sizeof(crb::Frame) * size_t(n)));
      CRB_CUDA(cudaMalloc(&c->d_maps, sizeof(CUtensorMap) * 3 * size_t(n)));  // 256-byte aligned
      c->d_frames_cap = n;
    }
    if (tab_entries > c->d_tab_cap) {
      cudaFree(c->d_tab);
      c->d_tab = nullptr;
      c->d_tab_cap = 0;
      CRB_CUDA(cudaMalloc(&c->d_tab, sizeof(uint32_t) * tab_entries));
      c->d_tab_cap = tab_entries;
    }
  }
  CRB_CUDA(cudaEventSynchronize(S.upload_ev));  // the staging buffers are free again
  c->h_frames = S.h_frames;
  c->h_maps = S.h_maps;
  c->maps_n = 0;
  c->h_tab = S.h_tab;
  c->upload_ev = S.upload_ev;
  return CRB_OK;
}

int ensure_ws(crb_ctx* c, size_t bytes, int ncounters) {
  if (bytes > c->ws_bytes) {
    CRB_CUDA(cudaDeviceSynchronize());
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&c->ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(CRB_ENOMEM, "workspace of " + std::to_string(bytes) + " bytes could not be allocated");
    }
    c->ws_bytes = bytes;
  }
  if (ncounters > c->counters_cap) {
    CRB_CUDA(cudaDeviceSynchronize());
    cudaFree(c->d_counters);
    c->d_counters = nullptr;
    CRB_CUDA(cudaMalloc(&c->d_counters, sizeof(unsigned long long) * size_t(ncounters)));
    c->counters_cap = ncounters;
  }
  return CRB_OK;
}

// Work of one call after the descriptors are in device memory: the memsets
// and kernel launches. Issued on `stream` directly, or into a CUDA graph.
struct Plan {
  int n = 0, niter = 0, shape = 0;
  bool maps = false, fuse = false, queue = false;
  bool fuse2 = false;  // tile pipeline: iterations 2 and 3 in one launch
  long long tiles = 0, rtiles = 0;
  size_t bits_total = 0;  // bytes from the start of the workspace that start at zero
  int ncounters = 0;
  int dgrid = 0, fgrid = 0, rgrid = 0;
  long long nblocks = 0, npix = 0;  // queue pipeline: word blocks, pixels
  long long ncells = 0;             // queue pipeline: cells (one word x kCH rows)
  long long nunits = 0;             // queue pipeline: strips of 32 words x kSH rows
  uint32_t* cells[2] = {nullptr, nullptr};  // cell classes for even / odd iterations
  char* chg[2] = {nullptr, nullptr};         // changed-pixel planes (all frames) for even / odd iterations
  size_t chg_bytes = 0;
  crb::Queues Q{};
  int occ[kQKernels] = {};       // queue pipeline: blocks per SM of each kernel (QK order)
  int seg_from = crb::kSegFrom;  // queue pipeline: first iteration of the segment-list forms
};

int enqueue_work(crb_ctx* c, const Plan& P, const std::vector<FrameSpec>& specs, cudaStream_t stream) {
  const DetectShape& ds = detect_shapes()[size_t(P.shape)];
  CRB_CUDA(cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * size_t(P.ncounters), stream));
  if (P.niter == 0) {
    for (const auto& s : specs) {
      CRB_CUDA(cudaMemcpyAsync(s.out_clean, s.img, size_t(s.w) * s.h * 4, cudaMemcpyDeviceToDevice, stream));
      CRB_CUDA(cudaMemsetAsync(s.out_mask, 0, size_t(s.w) * s.h, stream));
    }
    return CRB_OK;
  }
  CRB_CUDA(cudaMemsetAsync(c->ws, 0, P.bits_total, stream));
  if (P.queue) {
    // the image buffer starts as I0 (copied by the first bound pass): every
    // replacement then writes only its flagged pixels
    auto grid = [&](int kind, long long units) {
      return int(std::max<long long>(1, std::min<long long>(units, (long long)c->num_sms * P.occ[kind])));
    };
    const int gq = c->num_sms;  // queue and list kernels: grid-stride over lengths known on the device
    // while tuning, every launch is bracketed by events keyed by its kernel (QK order)
    auto tq = [&](int kernel, auto&& launch) {
      if (!c->tuning) {
        launch();
        return;
      }
      cudaEvent_t a = take_event(c), b = take_event(c);
      cudaEventRecord(a, stream);
      launch();
      cudaEventRecord(b, stream);
      c->tune_ev.push_back({kernel, {a, b}});
    };
    const size_t cells_bytes = size_t(P.ncells) * 4;
    for (int k = 1; k <= P.niter; ++k) {
      uint32_t* cls = P.cells[k & 1];
      uint32_t* cls_next = (k < P.niter) ? P.cells[(k + 1) & 1] : nullptr;
      const uint32_t* kcls = (k == 1) ? nullptr : cls;
      const long long ucol = (P.nunits + crb::kColWarps - 1) / crb::kColWarps;
      const int gcol = grid(kQNeed, ucol);
      const int gcolm = grid(kQM3need, ucol), gcol1m = grid(kQM3needAll, ucol);
      const bool seg = k >= P.seg_from;  // the column kernels walk the listed segments only
      const int tcol = crb::kColWarps * 32;
      timed(c, kPBound, stream, [&] {
        if (k == 1) {
          tq(kQBound, [&] {
            crb::bound_dense_kernel<<<grid(kQBound, P.nblocks), crb::kBoundThreads, 0, stream>>>(c->d_frames, P.n,
                                                                                         P.nblocks, c->p);
          });
        } else {  // the pixels within 2 px of a change, re-tested one by one
          if (seg) {
            tq(kQSegList, [&] {
              crb::seg_list_kernel<<<grid(kQSegList, (P.nunits + 7) / 8), crb::kThreads, 0, stream>>>(
                  c->d_frames, P.n, P.nunits, P.Q, cls);
            });
            tq(kQD2Seg, [&] {
              crb::d2_seg_kernel<<<gq * P.occ[kQD2Seg], tcol, 0, stream>>>(c->d_frames, P.n, P.Q, k);
            });
          } else {
            tq(kQD2, [&] {
              crb::d2_kernel<<<grid(kQD2, ucol), tcol, 0, stream>>>(c->d_frames, P.n, P.nunits, P.Q, k);
            });
          }
          tq(kQBoundSparse, [&] {
            crb::bound_sparse_kernel<<<gq * P.occ[kQBoundSparse], 256, 0, stream>>>(c->d_frames, P.n, P.Q, c->p);
          });
        }
      });
      timed(c, kPNeed, stream, [&] {
        if (seg)
          tq(kQNeedSeg, [&] {
            crb::need_seg_kernel<<<gq * P.occ[kQNeedSeg], tcol, 0, stream>>>(c->d_frames, P.n, P.Q, cls);
          });
        else
          tq(kQNeed, [&] {
            crb::need_kernel<<<gcol, tcol, 0, stream>>>(c->d_frames, P.n, P.nunits, P.Q, kcls);
          });
      });
      timed(c, kPS, stream, [&] {
        tq(kQS, [&] { crb::s_kernel<<<gq * P.occ[kQS], 256, 0, stream>>>(c->d_frames, P.n, P.Q, k); });
      });
      timed(c, kPSp, stream, [&] {
        tq(kQSp, [&] { crb::sp_kernel<<<gq * P.occ[kQSp], 256, 0, stream>>>(c->d_frames, P.n, P.Q, c->p, k); });
      });
      timed(c, kPM3need, stream, [&] {
        if (seg)
          tq(kQM3needSeg, [&] {
            crb::m3need_seg_kernel<<<gq * P.occ[kQM3needSeg], tcol, 0, stream>>>(c->d_frames, P.n, P.Q, cls);
          });
        else if (k == 1)
          tq(kQM3needAll, [&] {
            crb::m3need_kernel<true><<<gcol1m, tcol, 0, stream>>>(c->d_frames, P.n, P.nunits, P.Q, nullptr);
          });
        else
          tq(kQM3need, [&] {
            crb::m3need_kernel<false><<<gcolm, tcol, 0, stream>>>(c->d_frames, P.n, P.nunits, P.Q, kcls);
          });
      });
      timed(c, kPM3, stream, [&] {
        tq(kQM3, [&] { crb::m3_kernel<<<gq * P.occ[kQM3], 256, 0, stream>>>(c->d_frames, P.n, P.Q, k); });
      });
      timed(c, kPCand, stream, [&] {
        tq(kQCand, [&] {
          crb::cand_test_kernel<<<gq * P.occ[kQCand], 256, 0, stream>>>(c->d_frames, P.n, P.Q, c->p, k);
        });
        tq(kQCandFull, [&] {
          crb::cand_full_kernel<<<gq * P.occ[kQCandFull], 256, 0, stream>>>(c->d_frames, P.n, P.Q, c->p, k);
        });
      });
      timed(c, kPGrow, stream, [&] {
        if (k == 1)  // both growths from the bit planes; flags counted and queued for the replacement
          tq(kQGrowFirst, [&] {
            crb::grow_first_kernel<<<grid(kQGrowFirst, ucol), tcol, 0, stream>>>(c->d_frames, P.n, P.nunits, P.Q);
          });
        else
          tq(kQGrow, [&] {
            crb::grow_kernel<<<gq * P.occ[kQGrow], 256, 0, stream>>>(c->d_frames, P.n, P.Q, c->p, k);
          });
      });
      // the classes and changed pixels of iteration k+1 start at zero (those of iteration k-1 were read by now)
      if (k >= 3 && cls_next) {
        CRB_CUDA(cudaMemsetAsync(cls_next, 0, cells_bytes, stream));
        CRB_CUDA(cudaMemsetAsync(P.chg[(k + 1) & 1], 0, P.chg_bytes, stream));
      }
      timed(c, kPRep, stream, [&] {
        if (k >= 2)
          tq(kQRq, [&] { crb::rq_kernel<<<gq * P.occ[kQRq], 256, 0, stream>>>(c->d_frames, P.n, P.Q); });
        tq(kQRepCompute, [&] {
          crb::rep_compute_kernel<<<gq * P.occ[kQRepCompute], 256, 0, stream>>>(c->d_frames, P.n, P.Q, k,
                                                                                cls_next);
        });
        if (k >= 2)
          tq(kQRepWrite, [&] {
            crb::rep_write_kernel<<<gq * P.occ[kQRepWrite], 256, 0, stream>>>(c->d_frames, P.n, P.Q, cls_next,
                                                                              k + 1, 1);
          });
      });
      if (k == P.niter)
        timed(c, kPMask, stream, [&] {
          crb::mask_kernel<<<grid(kQMask, P.nblocks), 256, 0, stream>>>(c->d_frames, P.n, P.nblocks);
        });
      timed(c, kPWork, stream, [&] { crb::queue_work_kernel<<<1, 32, 0, stream>>>(c->d_frames, P.Q, k, P.npix); });
    }
    CRB_CUDA(cudaGetLastError());
    return CRB_OK;
  }
  for (int i = 0; i < P.n; ++i) {
    const auto& s = specs[size_t(i)];
    if (s.mprev) {
      const crb::Frame& f = c->h_frames[i];
      const long long nwords = (long long)f.wpr * f.h;
      const int blocks = int((nwords * 32 + 255) / 256 < 65535 ? (nwords * 32 + 255) / 256 : 65535);
      crb::bytes_to_bits_kernel<<<blocks, 256, 0, stream>>>(s.mprev, f.bits_b, f.w, f.h, f.wpr);  // M_0
    }
  }
  for (int k = 1; k <= P.niter; ++k) {
    if (P.fuse2 && k == 2) {  // iterations 2 and 3 in one launch (the replacements of 1 and 2 fused in)
      timed(c, kPTileDetect, stream, [&] {
        const int g = int(std::min<long long>(P.tiles, (long long)c->num_sms * c->occ_detect2));
        kDetect2<<<g, crb::kThreads, kDetect2Smem, stream>>>(c->d_frames, P.n, P.tiles, c->p, k, P.niter);
      });
    } else if (P.fuse2 && k == 3) {
      // done with iteration 2
    } else if (P.fuse && k >= 2) {  // replacement of iteration k-1 fused in front of detection k
      timed(c, kPTileDetect, stream, [&] {
        ds.fn_fused<<<P.fgrid, crb::kThreads, ds.smem_fused, stream>>>(c->d_frames, P.n, P.tiles, c->p, k, P.niter);
      });
    } else {
      timed(c, kPTileDetect, stream, [&] {
        (P.maps ? ds.fn_maps : ds.fn)<<<P.dgrid, crb::kThreads, ds.smem, stream>>>(c->d_frames, P.n, P.tiles, c->p, k,
                                                                                     P.niter);
      });
    }
    if (!P.fuse || k == P.niter) {
      // a buffer's first write is dense: iterations 1 and 2, and 3 after a fused pair (I_1 is never stored)
      const int dense = (k <= 2 || (P.fuse2 && k == 3)) ? 1 : 0;
      timed(c, kPTileReplace, stream, [&] {
        kReplace<<<P.rgrid, crb::kThreads, kReplaceSmem, stream>>>(c->d_frames, P.n, P.rtiles, k, P.niter, dense);
      });
    }
  }
  CRB_CUDA(cudaGetLastError());
  return CRB_OK;
}

// Queue pipeline: workspace = [queue counters | per frame: bit planes M, rq, fb |
// cell classes x 2 | changed-pixel planes x 2] (zeroed at the start of a call)
// then [per frame: bit planes hot, act, nsp, test, sval, m3val, lpz; maps S, N, S',
// M3] then [queues q0, q1, q2 (a pixel index per pixel or a word entry per
// word), fresh, fbl (a pixel index per pixel)].
int prepare_queue(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, Plan& P) {
  const int n = int(specs.size());
  long long npix = 0, nblocks = 0, ncells = 0, nwords = 0, nsegs = 0;
  for (const auto& s : specs) {
    npix += (long long)s.w * s.h;
    nsegs += 32LL * (((s.w + 31) / 32 + 31) / 32) * ((s.h + crb::kSH - 1) / crb::kSH);  // 32 per strip
    nwords += (long long)((s.w + 31) / 32) * s.h;
    ncells += (long long)((s.w + 31) / 32) * ((s.h + crb::kCH - 1) / crb::kCH);
  }
  size_t total = 256;  // queue counters
  std::vector<size_t> off_zero(static_cast<size_t>(n)), off_bits(static_cast<size_t>(n)),
      off_maps(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    off_zero[size_t(i)] = total;
    total += 5 * align256(size_t(s.w + 31) / 32 * size_t(s.h) * 4);
  }
  const size_t off_cells = total;
  total += 2 * align256(size_t(ncells) * 4);
  // changed-pixel planes, one region per parity (all frames), zeroed with one memset each
  std::vector<size_t> off_chg(static_cast<size_t>(n));
  size_t chg_bytes = 0;
  for (int i = 0; i < n; ++i) {
    off_chg[size_t(i)] = chg_bytes;
    chg_bytes += align256(size_t(specs[size_t(i)].w + 31) / 32 * size_t(specs[size_t(i)].h) * 4);
  }
  const size_t off_chg0 = total;
  total += 2 * chg_bytes;
  const size_t zero_bytes = total;
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    off_bits[size_t(i)] = total;
    total += 7 * align256(size_t(s.w + 31) / 32 * size_t(s.h) * 4);
    off_maps[size_t(i)] = total;
    total += 4 * align256(size_t(s.w) * size_t(s.h) * 4);
  }
  // q0..q2 hold a pixel index per pixel or a word entry (8 bytes) per word
  const size_t qbytes = align256(std::max(size_t(npix) * 4, size_t(nwords) * 8));
  const size_t fbytes = align256(size_t(npix) * 4);
  const size_t off_q = total;
  total += 3 * qbytes + 2 * fbytes;
  const size_t off_seg = total;  // three segment lists, one entry per segment at most
  const size_t segbytes = align256(size_t(nsegs) * 4);
  total += 3 * segbytes;
  const int nit = niter > 0 ? niter : 1;
  const int ncounters = (2 + crb::kWork) * nit * n;
  const size_t tab_n = size_t(npix >> crb::kTabShift) + 1;
  int rc = ensure_ws(c, total, ncounters);
  if (rc) return rc;
  rc = next_desc_slot(c, n, tab_n);
  if (rc) return rc;
  char* ws = static_cast<char*>(c->ws);
  long long pix0 = 0, rtiles = 0, cell0 = 0, nunits = 0, word0 = 0;
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    crb::Frame& f = c->h_frames[i];
    f = crb::Frame{};
    const size_t plane = align256(size_t(s.w + 31) / 32 * size_t(s.h) * 4);
    const size_t fmap = align256(size_t(s.w) * size_t(s.h) * 4);
    char* pz = ws + off_zero[size_t(i)];
    char* pb = ws + off_bits[size_t(i)];
    char* pm = ws + off_maps[size_t(i)];
    f.img = s.img;
    f.out_clean = s.out_clean;
    f.ws = nullptr;  // replacement is in place
    f.bits_a = f.bits_b = reinterpret_cast<uint32_t*>(pz);  // one plane, updated in place
    f.rq = reinterpret_cast<uint32_t*>(pz + plane);
    f.fb = reinterpret_cast<uint32_t*>(pz + 2 * plane);
    f.cand = reinterpret_cast<uint32_t*>(pz + 3 * plane);
    f.low = reinterpret_cast<uint32_t*>(pz + 4 * plane);
    f.chg[0] = reinterpret_cast<uint32_t*>(ws + off_chg0 + off_chg[size_t(i)]);
    f.chg[1] = reinterpret_cast<uint32_t*>(ws + off_chg0 + chg_bytes + off_chg[size_t(i)]);
    f.hot = reinterpret_cast<uint32_t*>(pb);
    f.act = reinterpret_cast<uint32_t*>(pb + plane);
    f.nsp = reinterpret_cast<uint32_t*>(pb + 2 * plane);
    f.test = reinterpret_cast<uint32_t*>(pb + 3 * plane);
    f.sval = reinterpret_cast<uint32_t*>(pb + 4 * plane);
    f.m3val = reinterpret_cast<uint32_t*>(pb + 5 * plane);
    f.lpz = reinterpret_cast<uint32_t*>(pb + 6 * plane);
    f.mapS = reinterpret_cast<float*>(pm);
    f.mapN = reinterpret_cast<float*>(pm + fmap);
    f.mapSp = reinterpret_cast<float*>(pm + 2 * fmap);
    f.mapM3 = reinterpret_cast<float*>(pm + 3 * fmap);
    f.out_mask = s.out_mask;
    f.maps = nullptr;
    f.counters = c->d_counters + size_t(2 + crb::kWork) * nit * i;
    f.work = f.counters + size_t(2) * nit;
    f.status = c->d_status;
    f.flip_from = 1 << 30;
    f.w = s.w;
    f.h = s.h;
    f.wpr = (s.w + 31) / 32;
    f.gain = s.gain;
    f.rn = s.rn;
    crb::bound_thresholds(c->p, s.gain, f.bkl, f.bkh);
    f.rtiles_x = (s.w + kRW - 1) / kRW;
    f.rtile0 = rtiles;
    rtiles += (long long)f.rtiles_x * ((s.h + kRH - 1) / kRH);
    f.pix0 = pix0;
    pix0 += (long long)s.w * s.h;
    f.bx = (f.wpr + crb::kBW - 1) / crb::kBW;
    f.blk0 = nblocks;
    nblocks += (long long)f.bx * ((s.h + crb::kBH - 1) / crb::kBH);
    f.ncy = (s.h + crb::kCH - 1) / crb::kCH;
    f.cell0 = cell0;
    cell0 += (long long)f.wpr * f.ncy;
    f.word0 = word0;
    word0 += (long long)f.wpr * s.h;
    f.ugx = (f.wpr + 31) / 32;
    f.u0 = nunits;
    nunits += (long long)f.ugx * ((s.h + crb::kSH - 1) / crb::kSH);
  }
  // frame of the first pixel of each 2^kTabShift pixels (frames are consecutive ranges)
  c->tab_n = tab_n;
  for (size_t t = 0, fi = 0; t < tab_n; ++t) {
    const long long g = (long long)t << crb::kTabShift;
    while (fi + 1 < size_t(n) && c->h_frames[fi + 1].pix0 <= g) ++fi;
    c->h_tab[t] = uint32_t(fi);
  }
  P.n = n;
  P.niter = niter;
  P.shape = 0;
  P.maps = false;
  P.fuse = false;
  P.queue = true;
  P.rtiles = rtiles;
  P.bits_total = zero_bytes;
  P.ncounters = ncounters;
  P.rgrid = int(std::min<long long>(rtiles, (long long)c->num_sms * c->occ_replace));
  std::copy(c->occ_q, c->occ_q + kQKernels, P.occ);
  P.seg_from = crb::kSegFrom;
  P.nblocks = nblocks;
  P.npix = npix;
  P.ncells = ncells;
  P.nunits = nunits;
  P.cells[0] = reinterpret_cast<uint32_t*>(ws + off_cells);
  P.cells[1] = reinterpret_cast<uint32_t*>(ws + off_cells + align256(size_t(ncells) * 4));
  P.Q.n = reinterpret_cast<unsigned int*>(ws);
  P.Q.ftab = c->d_tab;
  P.Q.q0 = reinterpret_cast<uint32_t*>(ws + off_q);
  P.Q.q1 = reinterpret_cast<uint32_t*>(ws + off_q + qbytes);
  P.Q.q2 = reinterpret_cast<uint32_t*>(ws + off_q + 2 * qbytes);
  P.Q.fresh = reinterpret_cast<uint32_t*>(ws + off_q + 3 * qbytes);
  P.Q.fbl = reinterpret_cast<uint32_t*>(ws + off_q + 3 * qbytes + fbytes);
  for (int j = 0; j < 3; ++j) P.Q.seg[j] = reinterpret_cast<uint32_t*>(ws + off_seg + size_t(j) * segbytes);
  P.chg[0] = ws + off_chg0;
  P.chg[1] = ws + off_chg0 + chg_bytes;
  P.chg_bytes = chg_bytes;
  return CRB_OK;
}

// The tile pipeline loads the image region of a detection tile inside the
// frame with one TMA box (crb::issue_tile_load).
constexpr bool kTileTma = true;

// cuTensorMapEncodeTiled from the driver (no link against libcuda), or nullptr.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return PFN_cuTensorMapEncodeTiled_v12000(nullptr);
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Writes the tensor maps of frame f's three image buffers (img, out_clean,
// ws) into host[0..2], each a 2-D float map of the frame with one box of the
// detection tile's image region (ds.tw + 16) x (ds.th + 16); returns the
// device address they are uploaded to, or nullptr when the frame does not
// qualify (row pitch or a buffer off the 16-byte boundary TMA needs, frame
// smaller than a box, or no encoder): its tiles then load element by element.
const CUtensorMap* encode_tile_maps(const crb::Frame& f, const DetectShape& ds, CUtensorMap* host,
                                    const CUtensorMap* dev) {
  const auto enc = tensor_map_encoder();
  const int bw = ds.tw + 16, bh = ds.th + 16;
  if (!enc || f.w % 4 != 0 || f.w < bw || f.h < bh) return nullptr;
  const void* bufs[3] = {f.img, f.out_clean, f.ws};
  for (int j = 0; j < 3; ++j) {
    if (!bufs[j]) {  // ws when niter < 2: never a source
      std::memset(&host[j], 0, sizeof(CUtensorMap));
      continue;
    }
    if ((reinterpret_cast<uintptr_t>(bufs[j]) & 15u) != 0) return nullptr;
    const cuuint64_t dims[2] = {cuuint64_t(f.w), cuuint64_t(f.h)};
    const cuuint64_t strides[1] = {cuuint64_t(f.w) * 4};
    const cuuint32_t box[2] = {cuuint32_t(bw), cuuint32_t(bh)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&host[j], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(bufs[j]), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return nullptr;
  }
  return dev;
}

// Lays out the workspace and writes the descriptors (host), for tile shape `shape`.
int prepare(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, bool maps, int shape, Plan& P) {
  const int n = int(specs.size());
  // two iterations per launch: needs the fused form, iterations 2 and 3, and its own tile shape
  const bool fuse2 = c->opt.fuse2 && !maps && !c->opt.no_fusion && niter >= 3 && shape == kFuse2Shape;
  const DetectShape& ds = detect_shapes()[size_t(shape)];
  std::vector<size_t> off_bits(static_cast<size_t>(n)), off_img(static_cast<size_t>(n));
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    const size_t wpr = size_t(s.w + 31) / 32;
    off_bits[size_t(i)] = total;
    total += 2 * align256(wpr * size_t(s.h) * 4);  // M for odd and for even iterations
  }
  const size_t bits_total = total;
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    off_img[size_t(i)] = total;
    if (niter >= 2) total += align256(size_t(s.w) * size_t(s.h) * 4);
  }
  const int nit = niter > 0 ? niter : 1;
  const int ncounters = (2 + crb::kWork) * nit * n;  // per frame: 2 per iteration, then kWork per iteration
  int rc = ensure_ws(c, total > 0 ? total : 256, ncounters);
  if (rc) return rc;
  rc = next_desc_slot(c, n, 0);
  if (rc) return rc;

  long long tiles = 0, rtiles = 0;
  for (int i = 0; i < n; ++i) {
    const auto& s = specs[size_t(i)];
    crb::Frame& f = c->h_frames[i];
    f.img = s.img;
    f.out_clean = s.out_clean;
    f.ws = (niter >= 2) ? reinterpret_cast<float*>(static_cast<char*>(c->ws) + off_img[size_t(i)]) : nullptr;
    f.bits_a = reinterpret_cast<uint32_t*>(static_cast<char*>(c->ws) + off_bits[size_t(i)]);
    f.bits_b = reinterpret_cast<uint32_t*>(static_cast<char*>(c->ws) + off_bits[size_t(i)] +
                                           align256(size_t(s.w + 31) / 32 * size_t(s.h) * 4));
    f.out_mask = s.out_mask;
    f.maps = s.maps;
    f.counters = c->d_counters + size_t(2 + crb::kWork) * nit * i;
    f.work = f.counters + size_t(2) * nit;
    f.w = s.w;
    f.h = s.h;
    f.wpr = (s.w + 31) / 32;
    f.gain = s.gain;
    f.rn = s.rn;
    f.status = c->d_status;
    f.dense_upto = fuse2 ? 3 : 2;
    f.flip_from = fuse2 ? 3 : (1 << 30);
    f.tmap = (!maps && kTileTma) ? encode_tile_maps(f, ds, c->h_maps + 3 * size_t(i), c->d_maps + 3 * size_t(i))
                                 : nullptr;
    if (f.tmap) c->maps_n = 3 * size_t(i + 1);
    f.tiles_x = (s.w + ds.tw - 1) / ds.tw;
    f.rtiles_x = (s.w + kRW - 1) / kRW;
    f.tile0 = tiles;
    f.rtile0 = rtiles;
    tiles += (long long)f.tiles_x * ((s.h + ds.th - 1) / ds.th);
    rtiles += (long long)f.rtiles_x * ((s.h + kRH - 1) / kRH);
  }
  P.n = n;
  P.niter = niter;
  P.shape = shape;
  P.maps = maps;
  P.fuse = !maps && !c->opt.no_fusion;
  P.fuse2 = fuse2;
  P.tiles = tiles;
  P.rtiles = rtiles;
  P.bits_total = bits_total;
  P.ncounters = ncounters;
  P.dgrid = int(std::min<long long>(tiles, (long long)c->num_sms *
                                               (maps ? c->occ_detect_maps : c->occ_detect)[size_t(shape)]));
  P.fgrid = int(std::min<long long>(tiles, (long long)c->num_sms * c->occ_fused[size_t(shape)]));
  P.rgrid = int(std::min<long long>(rtiles, (long long)c->num_sms * c->occ_replace));
  return CRB_OK;
}

// Copies n0 4-byte words src0 -> dst0 and n1 words src1 -> dst1 from
// page-locked host memory, read directly by the kernel: the descriptors reach
// the device without a copy engine, so they do not queue behind large
// transfers of other streams (crb_clean_batch_host), and one launch carries
// them all.
__global__ void upload_kernel(uint32_t* __restrict__ dst0, const uint32_t* __restrict__ src0, size_t n0,
                              uint32_t* __restrict__ dst1, const uint32_t* __restrict__ src1, size_t n1) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n0 + n1; i += size_t(gridDim.x) * blockDim.x)
    if (i < n0)
      dst0[i] = src0[i];
    else
      dst1[i - n0] = src1[i - n0];
  // tensor maps among the words are read by TMA (the tensormap proxy) in later kernels
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

int upload(crb_ctx* c, const Plan& P, cudaStream_t stream) {
  static_assert(sizeof(crb::Frame) % 4 == 0 && sizeof(CUtensorMap) % 4 == 0, "whole words");
  const size_t nf = sizeof(crb::Frame) * size_t(P.n) / 4;
  // the second segment: the frame table of the queue pipeline, or the tile pipeline's tensor maps
  uint32_t* d1 = P.queue ? c->d_tab : reinterpret_cast<uint32_t*>(c->d_maps);
  const uint32_t* h1 = P.queue ? c->h_tab : reinterpret_cast<const uint32_t*>(c->h_maps);
  const size_t n1 = P.queue ? c->tab_n : sizeof(CUtensorMap) * c->maps_n / 4;
  upload_kernel<<<int(std::min<size_t>((nf + n1 + 255) / 256, 64)), 256, 0, stream>>>(
      reinterpret_cast<uint32_t*>(c->d_frames), reinterpret_cast<const uint32_t*>(c->h_frames), nf, d1, h1, n1);
  CRB_CUDA(cudaGetLastError());
  CRB_CUDA(cudaEventRecord(c->upload_ev, stream));
  c->last_niter = P.niter;
  c->last_nframes = P.n;
  // the launches of this upload and of enqueue_work for this plan (memsets and copies not counted)
  if (P.niter == 0)
    c->last_launches = 1;
  else if (P.queue)  // the upload; iteration 1: 11 kernels, later ones 14 (15 with the segment list), the mask
    c->last_launches = 1 + 11 + 14 * (P.niter - 1) + std::max(0, P.niter - (P.seg_from - 1)) + 1;
  else
    c->last_launches = 1 + (P.fuse ? P.niter + 1 : 2 * P.niter) - (P.fuse2 ? 1 : 0) + c->mprev_frames;
  return CRB_OK;
}

// Replays (or captures once) the work of plan P as a CUDA graph on `stream`.
int launch_graph(crb_ctx* c, const Plan& P, const std::vector<FrameSpec>& specs, cudaStream_t stream) {
  long long occ_sig = 0;
  for (int i = 0; i < kQKernels; ++i) occ_sig = occ_sig * 31 + P.occ[i];
  GraphKey key{P.n,      P.niter,      P.shape,      P.fuse,  P.fuse2, P.queue, P.seg_from,  occ_sig,      P.tiles,
               P.rtiles, P.nblocks,    P.ncells,     P.npix,  P.bits_total, P.ncounters, P.dgrid, P.fgrid,
               P.rgrid,  c->ws,        c->d_counters, c->d_frames, P.queue ? c->d_tab : nullptr};
  for (auto& g : c->graphs)
    if (g.first == key) {
      CRB_CUDA(cudaGraphLaunch(g.second, stream));
      return CRB_OK;
    }
  if (!c->cap_stream) CRB_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  CRB_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_work(c, P, specs, c->cap_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (rc != CRB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
  if (c->graphs.size() >= 16) {  // keep the cache small
    cudaGraphExecDestroy(c->graphs.front().second);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.emplace_back(key, exec);
  CRB_CUDA(cudaGraphLaunch(exec, stream));
  return CRB_OK;
}

// crb_options.pipeline
enum { kPipeAuto = 0, kPipeTile = 1, kPipeQueue = 2 };
// Automatic choice: the queue pipeline from this many pixels per call on. Its
// ~60 dependent launches cost about 0.5 ms per call whatever the size, while
// the tile pipeline's 5 cost little but each pixel about 4.5 times more:
// single 800x800 and 1024x1024 frames clean in 0.17-0.18 ms on tiles and
// 0.54-0.67 ms on queues, 2048x4096 in 0.99 ms against 0.72-0.85 ms.
constexpr long long kAutoQueuePixels = 6000000;

// ---- Autotuner of the queue pipeline (crb_options.autotune) --------------------------------------
// The launch configuration does not change any result: every queue-pipeline
// kernel walks its work with a grid-stride loop, so any grid size gives the
// same outputs; the segment-list forms and the strip forms of the column
// kernels give the same queues; both pipelines give the same clean. The tuner
// therefore times trial cleans of the call's own frames and keeps the fastest
// configuration for the call signature (frame sizes and niter).

// Times one queue-pipeline clean of specs with blocks per SM occ[] and segment
// lists from iteration seg_from, synchronising `stream`; per_kernel (if not
// NULL) receives the device time of each kernel summed over its launches.
int trial_queue(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, const int* occ, int seg_from,
                cudaStream_t stream, float* ms, double* per_kernel) {
  Plan P;
  int rc = prepare_queue(c, specs, niter, P);
  if (rc) return rc;
  std::copy(occ, occ + kQKernels, P.occ);
  P.seg_from = seg_from;
  rc = upload(c, P, stream);
  if (rc) return rc;
  cudaEvent_t a = take_event(c), b = take_event(c);
  CRB_CUDA(cudaEventRecord(a, stream));
  c->tuning = per_kernel != nullptr;
  rc = enqueue_work(c, P, specs, stream);
  c->tuning = false;
  if (rc) return rc;
  CRB_CUDA(cudaEventRecord(b, stream));
  CRB_CUDA(cudaEventSynchronize(b));
  CRB_CUDA(cudaEventElapsedTime(ms, a, b));
  c->ev_pool.push_back(a);
  c->ev_pool.push_back(b);
  if (per_kernel) {
    std::fill(per_kernel, per_kernel + kQKernels, 0.0);
    for (auto& e : c->tune_ev) {
      float t = 0.f;
      CRB_CUDA(cudaEventElapsedTime(&t, e.second.first, e.second.second));
      per_kernel[e.first] += t;
      c->ev_pool.push_back(e.second.first);
      c->ev_pool.push_back(e.second.second);
    }
    c->tune_ev.clear();
  }
  return CRB_OK;
}

// The tile shape that tile_shape 0 takes for a call (see kOneRoundShape).
int default_shape(const crb_ctx* c, const std::vector<FrameSpec>& specs) {
  const auto& v = detect_shapes();
  auto tiles = [&](const DetectShape& d) {
    long long t = 0;
    for (const auto& s : specs) t += (long long)((s.w + d.tw - 1) / d.tw) * ((s.h + d.th - 1) / d.th);
    return t;
  };
  auto slots = [&](int i) {
    return (long long)c->num_sms * std::min(c->occ_detect[size_t(i)], c->occ_fused[size_t(i)]);
  };
  return (tiles(v[kOneRoundShape]) <= slots(kOneRoundShape) && tiles(v[0]) > slots(0)) ? kOneRoundShape : 0;
}

// Times one tile-pipeline clean (with the shape tile_shape 0 takes when that is
// the option, else 64 x 32), synchronising `stream`.
int trial_tile(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, cudaStream_t stream, float* ms) {
  Plan P;
  int rc = prepare(c, specs, niter, false, c->opt.tile_shape == 0 ? default_shape(c, specs) : 0, P);
  if (rc == CRB_OK) rc = upload(c, P, stream);
  if (rc) return rc;
  cudaEvent_t a = take_event(c), b = take_event(c);
  CRB_CUDA(cudaEventRecord(a, stream));
  rc = enqueue_work(c, P, specs, stream);
  if (rc) return rc;
  CRB_CUDA(cudaEventRecord(b, stream));
  CRB_CUDA(cudaEventSynchronize(b));
  CRB_CUDA(cudaEventElapsedTime(ms, a, b));
  c->ev_pool.push_back(a);
  c->ev_pool.push_back(b);
  return CRB_OK;
}

// Calls below this many pixels also try the tile pipeline.
constexpr long long kTuneTilePixels = 1LL << 25;

// Tunes the queue pipeline for specs: (1) four occupancy levels (all, 3/4, 1/2,
// 1/4 of each kernel's largest blocks per SM), each kernel keeping the level at
// which its own launches took least device time (the kernels run one after
// another, so their times add up independently), a lower level only if it wins
// by 2 %; (2) the first iteration of the segment-list forms (2, 3, 4 or none),
// by the time of the whole clean (best of two), another than the default only
// if it wins by 1 %; (3) below kTuneTilePixels, the tile pipeline against the
// result. The margins keep timing noise from deciding.
int tune_queue(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, long long npix, bool may_tile,
               cudaStream_t stream, crb_ctx::QTune& t) {
  const int saved_profile = c->opt.profile;
  c->opt.profile = 0;  // trials are not profiled
  std::copy(c->occ_q, c->occ_q + kQKernels, t.occ);
  t.seg_from = crb::kSegFrom;
  t.tile = false;
  float ms = 0.f;
  int rc = trial_queue(c, specs, niter, t.occ, t.seg_from, stream, &ms, nullptr);  // workspace and caches
  double best[kQKernels], pk[kQKernels];
  std::fill(best, best + kQKernels, 1e30);
  for (int lv = 4; lv >= 1 && rc == CRB_OK; --lv) {
    int occ[kQKernels];
    for (int i = 0; i < kQKernels; ++i) occ[i] = std::max(1, (c->occ_q[i] * lv + 3) / 4);
    rc = trial_queue(c, specs, niter, occ, t.seg_from, stream, &ms, pk);
    for (int i = 0; i < kQKernels && rc == CRB_OK; ++i)
      // a lower level must win by 2 % (a kernel that never runs keeps the first level)
      if (lv == 4 ? pk[i] < best[i] : pk[i] < 0.98 * best[i]) {
        best[i] = pk[i];
        t.occ[i] = occ[i];
      }
  }
  // the default start first; another must win by 1 % of the whole clean
  const int def_sf = std::min(crb::kSegFrom, niter + 1);
  float best_ms = 1e30f;
  for (int j = 0; j <= niter && rc == CRB_OK; ++j) {
    const int sf = j == 0 ? def_sf : j + 1;
    if (j > 0 && sf == def_sf) continue;
    float m = 1e30f;
    for (int rep = 0; rep < 2 && rc == CRB_OK; ++rep) {
      rc = trial_queue(c, specs, niter, t.occ, sf, stream, &ms, nullptr);
      m = std::min(m, ms);
    }
    if (j == 0 ? true : m < 0.99f * best_ms) {
      best_ms = m;
      t.seg_from = sf;
    }
  }
  if (rc == CRB_OK && may_tile && npix < kTuneTilePixels) {
    float m = 1e30f;
    for (int rep = 0; rep < 2 && rc == CRB_OK; ++rep) {
      rc = trial_tile(c, specs, niter, stream, &ms);
      m = std::min(m, ms);
    }
    t.tile = m < best_ms;
  }
  c->opt.profile = saved_profile;
  return rc;
}

// Enqueues the whole clean of `specs` (niter iterations) on `stream`.
int run(crb_ctx* c, const std::vector<FrameSpec>& specs, int niter, bool maps, cudaStream_t stream) {
  const int nshapes = int(detect_shapes().size());
  if (c->any_call) CRB_CUDA(cudaStreamWaitEvent(stream, c->done_ev, 0));
  long long npix = 0;
  for (const auto& s : specs) npix += (long long)s.w * s.h;
  const bool queue_ok = !maps && niter > 0 && npix < (1LL << 32) &&
                        std::all_of(specs.begin(), specs.end(), [](const FrameSpec& s) { return s.mprev == nullptr; });
  bool queue = queue_ok && (c->opt.pipeline == kPipeQueue ||
                            (c->opt.pipeline == kPipeAuto && npix >= kAutoQueuePixels));
  const crb_ctx::QTune* tuned = nullptr;
  if (c->opt.autotune && queue_ok && c->opt.pipeline != kPipeTile) {
    std::vector<long long> sig{niter};
    for (const auto& s : specs) {
      sig.push_back(s.w);
      sig.push_back(s.h);
    }
    for (const auto& t : c->qtuned)
      if (t.sig == sig) tuned = &t;
    if (!tuned) {
      crb_ctx::QTune t;
      t.sig = sig;
      const int rc = tune_queue(c, specs, niter, npix, c->opt.pipeline == kPipeAuto, stream, t);
      if (rc) return rc;
      c->qtuned.push_back(t);
      tuned = &c->qtuned.back();
    }
    queue = !tuned->tile;
  }
  int shape = c->opt.tile_shape;
  if (shape >= nshapes) shape = 0;
  if (c->opt.fuse2) shape = kFuse2Shape;
  if (shape < 0 && !maps && !queue) {
    // autotuning: the first call of a signature (frame sizes, niter) times every tile shape
    std::vector<long long> sig{niter};
    for (const auto& s : specs) {
      sig.push_back(s.w);
      sig.push_back(s.h);
    }
    shape = -1;
    for (const auto& t : c->tuned)
      if (t.first == sig) shape = t.second;
    if (shape < 0) {
      float best = 0.f;
      int best_shape = 0;
      cudaEvent_t a = nullptr, b = nullptr;
      CRB_CUDA(cudaEventCreate(&a));
      CRB_CUDA(cudaEventCreate(&b));
      for (int sh = 0; sh < nshapes; ++sh) {
        Plan P;
        int rc = prepare(c, specs, niter, maps, sh, P);
        if (rc == CRB_OK) rc = upload(c, P, stream);
        if (rc == CRB_OK && cudaEventRecord(a, stream) != cudaSuccess) rc = CRB_ECUDA;
        if (rc == CRB_OK) rc = enqueue_work(c, P, specs, stream);
        float ms = 0.f;
        if (rc == CRB_OK && (cudaEventRecord(b, stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
          rc = CRB_ECUDA;
        if (rc != CRB_OK) {
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return rc;
        }
        if (sh == 0 || ms < best) {
          best = ms;
          best_shape = sh;
        }
      }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      c->tuned.emplace_back(sig, best_shape);
      // every trial produced the same outputs; the last one stays
      CRB_CUDA(cudaEventRecord(c->done_ev, stream));
      c->any_call = true;
      return CRB_OK;
    }
  }
  if (shape < 0) shape = 0;
  if (shape == 0 && c->opt.tile_shape == 0 && !maps && !queue) shape = default_shape(c, specs);
  Plan P;
  int rc = queue ? prepare_queue(c, specs, niter, P) : prepare(c, specs, niter, maps, shape, P);
  if (rc) return rc;
  if (queue && tuned) {
    std::copy(tuned->occ, tuned->occ + kQKernels, P.occ);
    P.seg_from = tuned->seg_from;
  }
  std::copy(P.occ, P.occ + kQKernels, c->last_occ);
  c->last_seg_from = P.seg_from;
  c->last_pipeline = queue ? kPipeQueue : kPipeTile;
  c->mprev_frames = int(std::count_if(specs.begin(), specs.end(), [](const FrameSpec& s) { return s.mprev; }));
  rc = upload(c, P, stream);
  if (rc) return rc;
  // graphs replay only work whose pointers all come from the descriptors
  const bool graphable = niter > 0 && !maps && !c->opt.profile &&
                         std::all_of(specs.begin(), specs.end(), [](const FrameSpec& s) { return !s.mprev; });
  if (c->opt.use_graphs && graphable)
    rc = launch_graph(c, P, specs, stream);
  else
    rc = enqueue_work(c, P, specs, stream);
  if (rc) return rc;
  CRB_CUDA(cudaEventRecord(c->done_ev, stream));
  c->any_call = true;
  return CRB_OK;
}

bool valid_params(float gain, float rn, float sigclip, float sigfrac, float objlim, int niter) {
  return gain > 0.f && rn >= 0.f && sigclip > 0.f && sigfrac > 0.f && objlim > 0.f && niter >= 0 &&
         gain < 1e30f && rn < 1e30f && sigclip < 1e30f && sigfrac < 1e30f && objlim < 1e30f;
}

int check_frame(const void* img, int w, int h, const void* out_clean, const void* out_mask) {
  if (w < 1 || h < 1) return fail(CRB_EINVAL, "frame sizes must be >= 1");
  if ((long long)w * h >= (1LL << 31)) return fail(CRB_EINVAL, "w*h must be < 2^31");
  if (!img || !out_clean || !out_mask) return fail(CRB_EINVAL, "null image or output pointer");
  const size_t n = size_t(w) * size_t(h);
  if (overlaps(img, n * 4, out_clean, n * 4) || overlaps(img, n * 4, out_mask, n) ||
      overlaps(out_clean, n * 4, out_mask, n))
    return fail(CRB_EALIAS, "outputs must not overlap the input or each other");
  return CRB_OK;
}

}  // namespace

extern "C" {

crb_ctx* crb_create_ex(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter,
                       const crb_options* opts) {
  if (!valid_params(gain, readnoise, sigclip, sigfrac, objlim, niter)) {
    g_err = "invalid parameters: need gain > 0, readnoise >= 0, sigclip > 0, sigfrac > 0, objlim > 0, niter >= 0";
    return nullptr;
  }
  if (opts && (opts->objlim_form < 0 || opts->objlim_form > 1)) {
    g_err = "objlim_form must be 0 or 1";
    return nullptr;
  }
  auto* c = new crb_ctx();
  if (opts) c->opt = *opts;
  c->gain = gain;
  c->rn = readnoise;
  c->niter = niter;
  c->p = crb::Params{sigclip, sigfrac, objlim, c->opt.objlim_form};
  if (init_ctx(c) != CRB_OK) {
    crb_destroy(c);
    return nullptr;
  }
  g_err.clear();
  return c;
}

crb_ctx* crb_create(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter) {
  return crb_create_ex(gain, readnoise, sigclip, sigfrac, objlim, niter, nullptr);
}

void crb_destroy(crb_ctx* c) {
  if (!c) return;
  if (c->any_call) cudaEventSynchronize(c->done_ev);
  for (auto& v : c->pending)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->hs_out) cudaStreamSynchronize(c->hs_out);
  if (c->twin) crb_destroy(c->twin);
  for (cudaStream_t st : {c->hs_in, c->hs_cmp, c->hs_cmp2, c->hs_out})
    if (st) cudaStreamDestroy(st);
  if (c->h_entry) cudaEventDestroy(c->h_entry);
  for (int i = 0; i < kStageSlots; ++i) {
    for (cudaEvent_t e : {c->h_in[i], c->h_cmp[i], c->h_free[i]})
      if (e) cudaEventDestroy(e);
    cudaFree(c->d_stage[i]);
  }
  cudaFree(c->ws);
  cudaFree(c->d_rects);
  cudaFree(c->d_frames);
  cudaFree(c->d_maps);
  cudaFree(c->d_status);
  cudaFree(c->d_tab);
  for (auto& sl : c->slot) {
    if (sl.h_frames) cudaFreeHost(sl.h_frames);
    if (sl.h_maps) cudaFreeHost(sl.h_maps);
    if (sl.h_tab) cudaFreeHost(sl.h_tab);
    if (sl.upload_ev) cudaEventDestroy(sl.upload_ev);
  }
  cudaFree(c->d_counters);
  if (c->done_ev) cudaEventDestroy(c->done_ev);
  delete c;
}

int crb_clean(crb_ctx* c, const float* img, int w, int h, float* out_clean, uint8_t* out_mask,
              cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  int rc = check_frame(img, w, h, out_clean, out_mask);
  if (rc) return rc;
  std::vector<FrameSpec> specs{FrameSpec{img, out_clean, out_mask, nullptr, nullptr, w, h, c->gain, c->rn}};
  return run(c, specs, c->niter, false, stream);
}

int crb_clean_batch(crb_ctx* c, int n, const float* const* imgs, const int* ws, const int* hs,
                    const float* gains, const float* readnoises, float* const* out_cleans,
                    uint8_t* const* out_masks, cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  if (n < 0 || (n > 0 && (!imgs || !ws || !hs || !out_cleans || !out_masks)))
    return fail(CRB_EINVAL, "invalid batch arrays");
  if (n == 0) return CRB_OK;
  std::vector<FrameSpec> specs;
  specs.reserve(size_t(n));
  for (int i = 0; i < n; ++i) {
    int rc = check_frame(imgs[i], ws[i], hs[i], out_cleans[i], out_masks[i]);
    if (rc) return fail(rc, "frame " + std::to_string(i) + ": " + g_err);
    const float g = gains ? gains[i] : c->gain;
    const float r = readnoises ? readnoises[i] : c->rn;
    if (!(g > 0.f) || !(r >= 0.f)) return fail(CRB_EINVAL, "frame " + std::to_string(i) + ": gain/readnoise");
    specs.push_back(FrameSpec{imgs[i], out_cleans[i], out_masks[i], nullptr, nullptr, ws[i], hs[i], g, r});
  }
  return run(c, specs, c->niter, false, stream);
}

int crb_clean_batch_host(crb_ctx* c, int n, const float* const* imgs, const int* ws, const int* hs,
                         const float* gains, const float* readnoises, float* const* out_cleans,
                         uint8_t* const* out_masks, cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  if (n < 0 || (n > 0 && (!imgs || !ws || !hs || !out_cleans || !out_masks)))
    return fail(CRB_EINVAL, "invalid batch arrays");
  if (n == 0) return CRB_OK;
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    if (ws[i] < 1 || hs[i] < 1 || (long long)ws[i] * hs[i] >= (1LL << 31))
      return fail(CRB_EINVAL, "frame " + std::to_string(i) + ": sizes");
    if (!imgs[i] || !out_cleans[i] || !out_masks[i]) return fail(CRB_EINVAL, "frame " + std::to_string(i) + ": null");
    const long long px = (long long)ws[i] * hs[i];
    total += px;
  }
  // chunks of consecutive frames of about total/kStageChunks pixels, ramped at
  // both ends (total/32, total/16): the first copy-in and the last copy-out
  // overlap no other work, so they are kept short
  const long long mid = (total + kStageChunks - 1) / kStageChunks;
  auto px_of = [&](int i) { return (long long)ws[i] * hs[i]; };
  // the tail: the last chunk up to total/32, the one before up to total/16 (a frame at least each)
  std::vector<int> tail_first;  // first frames of the tail chunks, last chunk first
  int end = n;
  for (const long long t : {total / 32, total / 16}) {
    int i = end - 1;
    for (long long acc = px_of(i); i > 0 && acc + px_of(i - 1) <= t; --i) acc += px_of(i - 1);
    if (i <= 0) break;
    tail_first.push_back(i);
    end = i;
  }
  std::vector<int> first{0};
  long long target = total / 32;  // then total/16, then total/kStageChunks
  for (long long acc = 0, i = 0; i < end; ++i) {
    const long long px = px_of(int(i));
    if (acc > 0 && acc + px > target) {
      first.push_back(int(i));
      acc = 0;
      target = std::min(2 * target, mid);
    }
    acc += px;
  }
  for (auto it = tail_first.rbegin(); it != tail_first.rend(); ++it) first.push_back(*it);
  first.push_back(n);
  auto frame_bytes = [&](int i) { return align256(size_t(ws[i]) * hs[i] * 4) * 2 + align256(size_t(ws[i]) * hs[i]); };
  size_t need = 0;
  for (size_t k = 0; k + 1 < first.size(); ++k) {
    size_t b = 0;
    for (int i = first[k]; i < first[k + 1]; ++i) b += frame_bytes(i);
    need = std::max(need, b);
  }
  if (!c->twin) {
    crb_options o = c->opt;
    o.profile = 0;
    c->twin = crb_create_ex(c->gain, c->rn, c->p.sigclip, c->p.sigfrac, c->p.objlim,
                            c->niter, &o);
    if (!c->twin) return fail(CRB_ENOMEM, "crb_clean_batch_host: second context: " + g_err);
    c->twin->p = c->p;
  }
  if (!c->hs_in) {
    for (cudaStream_t* st : {&c->hs_in, &c->hs_cmp, &c->hs_cmp2, &c->hs_out})
      CRB_CUDA(cudaStreamCreateWithFlags(st, cudaStreamNonBlocking));
    CRB_CUDA(cudaEventCreateWithFlags(&c->h_entry, cudaEventDisableTiming));
    for (int i = 0; i < kStageSlots; ++i)
      for (cudaEvent_t* e : {&c->h_in[i], &c->h_cmp[i], &c->h_free[i]})
        CRB_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (need > c->stage_cap) {
    CRB_CUDA(cudaDeviceSynchronize());
    for (int s = 0; s < kStageSlots; ++s) {
      cudaFree(c->d_stage[s]);
      c->d_stage[s] = nullptr;
    }
    c->stage_cap = 0;
    for (int s = 0; s < kStageSlots; ++s) {
      const cudaError_t e = cudaMalloc(&c->d_stage[s], need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CRB_ENOMEM, "staging buffers of " + std::to_string(kStageSlots) + " x " + std::to_string(need) +
                                    " bytes could not be allocated");
      }
    }
    c->stage_cap = need;
  }
  // the pipeline starts after the work already on `stream`
  CRB_CUDA(cudaEventRecord(c->h_entry, stream));
  CRB_CUDA(cudaStreamWaitEvent(c->hs_in, c->h_entry, 0));
  for (size_t k = 0; k + 1 < first.size(); ++k) {
    const int slot = int(k % kStageSlots), a = first[k], b = first[k + 1], m = b - a;
    std::vector<const float*> d_img(static_cast<size_t>(m));
    std::vector<float*> d_out(static_cast<size_t>(m));
    std::vector<uint8_t*> d_msk(static_cast<size_t>(m));
    char* p = c->d_stage[slot];
    for (int i = a; i < b; ++i) {
      const size_t px = size_t(ws[i]) * hs[i];
      d_img[size_t(i - a)] = reinterpret_cast<const float*>(p);
      d_out[size_t(i - a)] = reinterpret_cast<float*>(p + align256(px * 4));
      d_msk[size_t(i - a)] = reinterpret_cast<uint8_t*>(p + 2 * align256(px * 4));
      p += frame_bytes(i);
    }
    // copy in once the slot's previous copy-out is done
    CRB_CUDA(cudaStreamWaitEvent(c->hs_in, c->h_free[slot], 0));
    for (int i = a; i < b; ++i)
      CRB_CUDA(cudaMemcpyAsync(const_cast<float*>(d_img[size_t(i - a)]), imgs[i], size_t(ws[i]) * hs[i] * 4,
                               cudaMemcpyHostToDevice, c->hs_in));
    CRB_CUDA(cudaEventRecord(c->h_in[slot], c->hs_in));
    // clean, on this context or its twin
    crb_ctx* cc = (k & 1) ? c->twin : c;
    cudaStream_t cs = (k & 1) ? c->hs_cmp2 : c->hs_cmp;
    CRB_CUDA(cudaStreamWaitEvent(cs, c->h_in[slot], 0));
    const int rc = crb_clean_batch(cc, m, d_img.data(), ws + a, hs + a, gains ? gains + a : nullptr,
                                   readnoises ? readnoises + a : nullptr, d_out.data(), d_msk.data(), cs);
    if (rc != CRB_OK) return rc;
    CRB_CUDA(cudaEventRecord(c->h_cmp[slot], cs));
    // copy out
    CRB_CUDA(cudaStreamWaitEvent(c->hs_out, c->h_cmp[slot], 0));
    for (int i = a; i < b; ++i) {
      const size_t px = size_t(ws[i]) * hs[i];
      CRB_CUDA(cudaMemcpyAsync(out_cleans[i], d_out[size_t(i - a)], px * 4, cudaMemcpyDeviceToHost, c->hs_out));
      CRB_CUDA(cudaMemcpyAsync(out_masks[i], d_msk[size_t(i - a)], px, cudaMemcpyDeviceToHost, c->hs_out));
    }
    CRB_CUDA(cudaEventRecord(c->h_free[slot], c->hs_out));
  }
  // `stream` continues after the last copy-out
  CRB_CUDA(cudaEventRecord(c->h_entry, c->hs_out));
  CRB_CUDA(cudaStreamWaitEvent(stream, c->h_entry, 0));
  return CRB_OK;
}

int crb_clean_rects(crb_ctx* c, const float* img, int w, int h, int n, const crb_rect* rects, float* out_clean,
                    uint8_t* out_mask, cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  int rc = check_frame(img, w, h, out_clean, out_mask);
  if (rc) return rc;
  if (n < 0 || (n > 0 && !rects)) return fail(CRB_EINVAL, "crb_clean_rects: invalid rectangle array");
  if (n == 0) return CRB_OK;
  auto crop_bytes = [](const crb_rect& r) {
    const size_t px = size_t(r.cw) * size_t(r.ch);
    return 2 * align256(px * 4) + align256(px);
  };
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    const crb_rect& r = rects[i];
    using ll = long long;  // sums of caller-given ints: no overflow can pass the checks
    const bool ok = r.w >= 1 && r.h >= 1 && r.cx0 >= 0 && r.cy0 >= 0 && r.cx0 <= r.x0 && r.cy0 <= r.y0 &&
                    ll(r.x0) + r.w <= ll(r.cx0) + r.cw && ll(r.y0) + r.h <= ll(r.cy0) + r.ch &&
                    ll(r.cx0) + r.cw <= w && ll(r.cy0) + r.ch <= h;
    if (!ok)
      return fail(CRB_EINVAL, "crb_clean_rects: rectangle " + std::to_string(i) +
                                  ": the context region must contain the interior and lie in the frame");
    need += crop_bytes(r);
  }
  if (need > c->rects_cap) {
    CRB_CUDA(cudaDeviceSynchronize());
    cudaFree(c->d_rects);
    c->d_rects = nullptr;
    c->rects_cap = 0;
    const cudaError_t e = cudaMalloc(&c->d_rects, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(CRB_ENOMEM, "crb_clean_rects: crops of " + std::to_string(need) + " bytes could not be allocated");
    }
    c->rects_cap = need;
  }
  // the crops are reused: copy into them after the context's previous call is done
  if (c->any_call) CRB_CUDA(cudaStreamWaitEvent(stream, c->done_ev, 0));
  std::vector<const float*> in(static_cast<size_t>(n));
  std::vector<float*> out(static_cast<size_t>(n));
  std::vector<uint8_t*> msk(static_cast<size_t>(n));
  std::vector<int> cws(static_cast<size_t>(n)), chs(static_cast<size_t>(n));
  char* p = c->d_rects;
  for (int i = 0; i < n; ++i) {
    const crb_rect& r = rects[i];
    const size_t px = size_t(r.cw) * size_t(r.ch);
    float* ci = reinterpret_cast<float*>(p);
    in[size_t(i)] = ci;
    out[size_t(i)] = reinterpret_cast<float*>(p + align256(px * 4));
    msk[size_t(i)] = reinterpret_cast<uint8_t*>(p + 2 * align256(px * 4));
    cws[size_t(i)] = r.cw;
    chs[size_t(i)] = r.ch;
    p += crop_bytes(r);
    CRB_CUDA(cudaMemcpy2DAsync(ci, size_t(r.cw) * 4, img + size_t(r.cy0) * w + r.cx0, size_t(w) * 4,
                               size_t(r.cw) * 4, size_t(r.ch), cudaMemcpyDeviceToDevice, stream));
  }
  rc = crb_clean_batch(c, n, in.data(), cws.data(), chs.data(), nullptr, nullptr, out.data(), msk.data(), stream);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {  // the interiors into the frame (the director's assembly)
    const crb_rect& r = rects[i];
    const size_t o = size_t(r.y0 - r.cy0) * r.cw + size_t(r.x0 - r.cx0);
    CRB_CUDA(cudaMemcpy2DAsync(out_clean + size_t(r.y0) * w + r.x0, size_t(w) * 4, out[size_t(i)] + o,
                               size_t(r.cw) * 4, size_t(r.w) * 4, size_t(r.h), cudaMemcpyDeviceToDevice, stream));
    CRB_CUDA(cudaMemcpy2DAsync(out_mask + size_t(r.y0) * w + r.x0, size_t(w), msk[size_t(i)] + o, size_t(r.cw),
                               size_t(r.w), size_t(r.h), cudaMemcpyDeviceToDevice, stream));
  }
  CRB_CUDA(cudaEventRecord(c->done_ev, stream));  // the next call waits for these reads of the crops
  return CRB_OK;
}

int crb_iterate(crb_ctx* c, const float* J, const uint8_t* Mprev, int w, int h, float* out_J, uint8_t* out_M,
                float* maps, cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  int rc = check_frame(J, w, h, out_J, out_M);
  if (rc) return rc;
  std::vector<FrameSpec> specs{FrameSpec{J, out_J, out_M, maps, Mprev, w, h, c->gain, c->rn}};
  if (maps) {
    CRB_CUDA(cudaMemsetAsync(maps, 0xff, sizeof(float) * crb::kNumMaps * size_t(w) * h, stream));  // NaN
  }
  return run(c, specs, 1, maps != nullptr, stream);
}

int crb_sync_status(crb_ctx* c, cudaStream_t stream) {
  if (!c) return fail(CRB_EINVAL, "null context");
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "device execution");
  unsigned int st = 0;
  CRB_CUDA(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st != 0) {
    CRB_CUDA(cudaMemset(c->d_status, 0, sizeof st));
    c->latched = CRB_ETIMEOUT;
    g_err = "a bounded device-side wait gave up (a tile's TMA load did not land)";
  }
  const int s = c->latched;
  c->latched = CRB_OK;
  return s;
}

namespace {
// Sums, over the frames of the last call, `width` counters per iteration
// stored at offset `base` (per iteration) of each frame's block.
int read_counters(crb_ctx* c, long long* out, int max_iter, int base, int width) {
  if (!c || !out || max_iter < 0) return -1;
  const int k = std::min(c->last_niter, max_iter);
  if (k == 0 || c->last_nframes == 0) return 0;
  const int nit = c->last_niter;
  std::vector<unsigned long long> tmp(size_t(2 + crb::kWork) * nit * c->last_nframes);
  if (cudaMemcpy(tmp.data(), c->d_counters, sizeof(unsigned long long) * tmp.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return -1;
  for (int it = 0; it < k; ++it)
    for (int j = 0; j < width; ++j) {
      long long s = 0;
      for (int fr = 0; fr < c->last_nframes; ++fr)
        s += (long long)tmp[size_t(2 + crb::kWork) * nit * fr + size_t(base) * nit + size_t(width) * it + j];
      out[width * it + j] = s;
    }
  return k;
}
}  // namespace

int crb_last_counts(crb_ctx* c, long long* out, int max_iter) { return read_counters(c, out, max_iter, 0, 2); }

int crb_last_launches(const crb_ctx* c) { return c ? c->last_launches : -1; }

int crb_last_work(crb_ctx* c, long long* out, int max_iter) {
  return read_counters(c, out, max_iter, 2, crb::kWork);
}

namespace {
// Folds the finished event pairs of every kind into the totals.
int profile_collect(crb_ctx* c) {
  for (int kind = 0; kind < kProfKinds; ++kind) {
    for (auto& pr : c->pending[kind]) {
      float ms = 0.f;
      CRB_CUDA(cudaEventSynchronize(pr.second));
      CRB_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
      c->prof_ms[kind] += ms;
      c->prof_n[kind] += 1;
      c->ev_pool.push_back(pr.first);
      c->ev_pool.push_back(pr.second);
    }
    c->pending[kind].clear();
  }
  return CRB_OK;
}
}  // namespace

int crb_profile_read(crb_ctx* c, double* detect_ms, int* detect_launches, double* replace_ms,
                     int* replace_launches, int reset) {
  if (!c || !c->opt.profile) return fail(CRB_EINVAL, "profiling is off for this context");
  const int rc = profile_collect(c);
  if (rc) return rc;
  double dm = 0, rm = 0;
  int dn = 0, rn = 0;
  for (int kind = 0; kind < kPWork; ++kind) {
    if (kind < kProfReplace0) {
      dm += c->prof_ms[kind];
      dn += c->prof_n[kind];
    } else {
      rm += c->prof_ms[kind];
      rn += c->prof_n[kind];
    }
  }
  if (detect_ms) *detect_ms = dm;
  if (detect_launches) *detect_launches = dn;
  if (replace_ms) *replace_ms = rm;
  if (replace_launches) *replace_launches = rn;
  if (reset)
    for (int kind = 0; kind < kProfKinds; ++kind) {
      c->prof_ms[kind] = 0;
      c->prof_n[kind] = 0;
    }
  return CRB_OK;
}

int crb_profile_kernels(crb_ctx* c, double* ms, int* brackets, int max, int reset) {
  if (!c || !c->opt.profile || max < 0 || (max > 0 && !ms)) return fail(CRB_EINVAL, "profiling off / bad arguments");
  const int rc = profile_collect(c);
  if (rc) return rc;
  const int k = std::min(max, int(kProfKinds));
  for (int i = 0; i < k; ++i) {
    ms[i] = c->prof_ms[i];
    if (brackets) brackets[i] = c->prof_n[i];
  }
  if (reset)
    for (int kind = 0; kind < kProfKinds; ++kind) {
      c->prof_ms[kind] = 0;
      c->prof_n[kind] = 0;
    }
  return k;
}

int crb_fadd_peak(double* ops_per_s, cudaStream_t stream) {
  int dev = 0, sms = 0;
  CRB_CUDA(cudaGetDevice(&dev));
  CRB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* buf = nullptr;
  CRB_CUDA(cudaMalloc(&buf, sizeof(float) * (192 + size_t(sms) * 8 * 256)));
  std::vector<float> init(192);
  for (int i = 0; i < 192; ++i) init[size_t(i)] = 1e-3f * float(i + 1);
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = CRB_OK;
  const int blocks = sms * 8, iters = 4096;
  double best = 0;
  if (cudaMemcpy(buf, init.data(), sizeof(float) * 192, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    rc = cuda_fail(cudaGetLastError(), "crb_fadd_peak setup");
  for (int rep = 0; rep < 4 && rc == CRB_OK; ++rep) {
    cudaEventRecord(a, stream);
    crb::fadd_peak_kernel<<<blocks, 256, 0, stream>>>(buf, buf + 192, iters);
    cudaEventRecord(b, stream);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "crb_fadd_peak");
      break;
    }
    const double ops = double(blocks) * 256 * iters * crb::kPeakChains;
    if (rep > 0) best = std::max(best, ops / (ms * 1e-3));
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  if (rc == CRB_OK && ops_per_s) *ops_per_s = best;
  return rc;
}

int crb_alu_peak(double* ops2_per_s, double* ops3_per_s, cudaStream_t stream) {
  int dev = 0, sms = 0;
  CRB_CUDA(cudaGetDevice(&dev));
  CRB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* buf = nullptr;
  CRB_CUDA(cudaMalloc(&buf, sizeof(float) * (192 + size_t(sms) * 8 * 256)));
  std::vector<float> init(192);
  for (int i = 0; i < 192; ++i) init[size_t(i)] = (i < 64) ? float(i) : (i < 128 ? -1000.f + i : 1000.f + i);
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = CRB_OK;
  const int blocks = sms * 8, iters = 4096;
  double best[2] = {0, 0};
  if (cudaMemcpy(buf, init.data(), sizeof(float) * 192, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "crb_alu_peak setup");
  }
  for (int form = 0; form < 2 && rc == CRB_OK; ++form) {
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(a, stream);
      if (form == 0)
        crb::alu_peak_kernel<false><<<blocks, 256, 0, stream>>>(buf, buf + 192, iters);
      else
        crb::alu_peak_kernel<true><<<blocks, 256, 0, stream>>>(buf, buf + 192, iters);
      cudaEventRecord(b, stream);
      cudaError_t e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "crb_alu_peak");
        break;
      }
      const double ops = double(blocks) * 256 * iters * crb::kPeakChains * 2;
      if (rep > 0) best[form] = std::max(best[form], ops / (ms * 1e-3));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  if (rc == CRB_OK) {
    if (ops2_per_s) *ops2_per_s = best[0];
    if (ops3_per_s) *ops3_per_s = best[1];
  }
  return rc;
}

namespace {
// Waits on an mbarrier that nothing arms, with the given poll limit, the way
// the tile kernels wait for a TMA box; records the timeout in *status.
__global__ void wait_selftest_kernel(unsigned polls, unsigned int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    crb::mbar_init(&bar, 1);
    if (!crb::mbar_wait(&bar, 0, polls)) atomicOr(status, crb::kStatusTimeout);
  }
}
}  // namespace

int crb_selftest_wait_timeout(crb_ctx* c, unsigned polls, cudaStream_t stream) {
  if (!c || polls == 0 || polls > (1u << 22)) return fail(CRB_EINVAL, "crb_selftest_wait_timeout: 1 <= polls <= 2^22");
  if (c->any_call) CRB_CUDA(cudaStreamWaitEvent(stream, c->done_ev, 0));
  wait_selftest_kernel<<<1, 32, 0, stream>>>(polls, c->d_status);
  CRB_CUDA(cudaGetLastError());
  CRB_CUDA(cudaEventRecord(c->done_ev, stream));
  c->any_call = true;
  return CRB_OK;
}

int crb_tuned_config(const crb_ctx* c, int* blocks_per_sm, int max, int* seg_from, int* pipeline) {
  if (!c || max < 0 || (max > 0 && !blocks_per_sm)) return fail(CRB_EINVAL, "crb_tuned_config: bad arguments");
  const int k = std::min(max, int(kQKernels));
  for (int i = 0; i < k; ++i) blocks_per_sm[i] = c->last_occ[i];
  if (seg_from) *seg_from = c->last_seg_from;
  if (pipeline) *pipeline = c->last_pipeline;
  return k;
}

int crb_num_tile_shapes(void) { return int(detect_shapes().size()); }

int crb_tile_shape(int index, int* tile_w, int* tile_h) {
  if (index < 0 || index >= int(detect_shapes().size())) return CRB_EINVAL;
  if (tile_w) *tile_w = detect_shapes()[size_t(index)].tw;
  if (tile_h) *tile_h = detect_shapes()[size_t(index)].th;
  return CRB_OK;
}

const char* crb_last_error(void) { return g_err.c_str(); }

const char* crb_strerror(int s) {
  switch (s) {
    case CRB_OK: return "ok";
    case CRB_EINVAL: return "invalid argument";
    case CRB_ENOMEM: return "out of device memory";
    case CRB_ECUDA: return "CUDA error";
    case CRB_ETIMEOUT: return "device wait timed out";
    case CRB_EBUSY: return "busy: admission refused";
    case CRB_EALIAS: return "output overlaps input";
    case CRB_EDEVICE: return "device-side check failed";
    default: return "unknown status";
  }
}

}  // extern "C"
