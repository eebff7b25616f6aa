// crb_clean_noalloc: the clean of one frame with no device allocation at call
// time (declaration and contract in include/crb.h).
//
// Some callers cannot allocate device memory while they run: onboard or
// embedded pipelines that fix their memory plan at start-up, latency-bound
// loops in which cudaMalloc/cudaFree would synchronise the device, and host
// processes whose device memory is owned by another allocator. For them the
// scratch of the clean (the second image buffer, the flag bits, the counters
// and the frame descriptor) lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process
// exits. The caller still passes the input and both outputs.

#include <mutex>
#include <string>
#include <vector>

#include "crb.h"
#include "kernels.cuh"

void crb_detail_set_error(const char* msg);  // crb.cu

namespace {

constexpr long long kMaxPixels = 1LL << 22;  // 4,194,304 pixels, e.g. 2048 x 2048
constexpr int kMaxSide = 16384;
constexpr int kMaxIter = 64;
constexpr int kTW = 64, kTH = 32;  // detection tile
constexpr int kRW = 64, kRH = 16;  // replacement tile

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffCount = up256(sizeof(crb::Frame));
constexpr size_t kOffBits = kOffCount + up256(sizeof(unsigned long long) * 2 * kMaxIter);
// ceil(w/32) * h <= w*h/32 + h words
constexpr size_t kOffImg = kOffBits + up256(sizeof(uint32_t) * (size_t(kMaxPixels) / 32 + kMaxSide));
constexpr size_t kScratchBytes = kOffImg + up256(sizeof(float) * size_t(kMaxPixels));

// The scratch shared by every call on a device (about 17 MB). Host code must
// not take its address directly: the host-side symbol is only a stand-in.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;  // device address of g_scratch
  int sms = 0, occ_detect = 1, occ_replace = 1;
};

std::mutex g_mu;
std::vector<DeviceSetup> g_setup;  // by device; read and written under g_mu only

using Detect = void (*)(const crb::Frame*, int, long long, crb::Params, int, int);
using Replace = void (*)(const crb::Frame*, int, long long, int, int, int);
const Detect kDetect = crb::detect_kernel<kTW, kTH, false>;
const Replace kReplace = crb::replace_kernel<kRW, kRH>;
constexpr size_t kDetectSmem = crb::DetectLayout<kTW, kTH>::bytes;
constexpr size_t kReplaceSmem = crb::ReplaceLayout<kRW, kRH>::bytes;

// Writes the descriptor and clears the counters.
__global__ void noalloc_prepare(crb::Frame f, crb::Frame* desc, unsigned long long* counters, int ncounters) {
  if (threadIdx.x == 0) *desc = f;
  for (int i = threadIdx.x; i < ncounters; i += blockDim.x) counters[i] = 0;
}

int err(int code, const std::string& msg) {
  crb_detail_set_error(msg.c_str());
  return code;
}

int cuda_err(cudaError_t e, const char* what) {
  return err(CRB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Once per device, with that device current: the device address of the
// scratch array and the kernels' launch attributes. The caller gets a copy, so
// a first call on another device (which may grow g_setup) from another host
// thread cannot move the entry under it.
int setup_current_device(DeviceSetup* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  if (int(g_setup.size()) <= dev) g_setup.resize(size_t(dev) + 1);
  DeviceSetup& s = g_setup[size_t(dev)];
  if (!s.done) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
    if ((e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(kDetect, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDetectSmem))) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(kReplace, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kReplaceSmem))) !=
            cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.occ_detect, kDetect, crb::kThreads, kDetectSmem)) !=
            cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.occ_replace, kReplace, crb::kThreads,
                                                           kReplaceSmem)) != cudaSuccess)
      return cuda_err(e, "crb_clean_noalloc set-up");
    if (s.occ_detect < 1) s.occ_detect = 1;
    if (s.occ_replace < 1) s.occ_replace = 1;
    s.scratch = static_cast<unsigned char*>(p);
    s.done = true;
  }
  *out = s;
  return CRB_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int crb_clean_noalloc(float gain, float readnoise, float sigclip, float sigfrac, float objlim,
                                 int niter, const float* img, int w, int h, float* out_clean, uint8_t* out_mask,
                                 cudaStream_t stream) {
  if (!(gain > 0.f) || !(readnoise >= 0.f) || !(sigclip > 0.f) || !(sigfrac > 0.f) || !(objlim > 0.f))
    return err(CRB_EINVAL, "crb_clean_noalloc: need gain > 0, readnoise >= 0, sigclip > 0, sigfrac > 0, objlim > 0");
  if (niter < 0 || niter > kMaxIter)
    return err(CRB_EINVAL, "crb_clean_noalloc: niter must be in [0, " + std::to_string(kMaxIter) + "]");
  if (w < 1 || h < 1 || w > kMaxSide || h > kMaxSide || (long long)w * h > kMaxPixels)
    return err(CRB_EINVAL, "crb_clean_noalloc: frame " + std::to_string(w) + "x" + std::to_string(h) +
                               " exceeds the fixed scratch (at most " + std::to_string(kMaxPixels) +
                               " pixels and " + std::to_string(kMaxSide) + " per side); use crb_clean");
  if (!img || !out_clean || !out_mask) return err(CRB_EINVAL, "crb_clean_noalloc: null image or output pointer");
  const size_t n = size_t(w) * size_t(h);
  if (overlap(img, n * 4, out_clean, n * 4) || overlap(img, n * 4, out_mask, n) || overlap(out_clean, n * 4, out_mask, n))
    return err(CRB_EALIAS, "crb_clean_noalloc: outputs must not overlap the input or each other");

  DeviceSetup setup;
  int rc = setup_current_device(&setup);
  if (rc != CRB_OK) return rc;
  const DeviceSetup* s = &setup;

  cudaError_t e;
  if (niter == 0) {
    if ((e = cudaMemcpyAsync(out_clean, img, n * 4, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(out_mask, 0, n, stream)) != cudaSuccess)
      return cuda_err(e, "crb_clean_noalloc");
    return CRB_OK;
  }

  crb::Frame f{};
  f.img = img;
  f.out_clean = out_clean;
  f.ws = reinterpret_cast<float*>(s->scratch + kOffImg);
  f.bits_a = reinterpret_cast<uint32_t*>(s->scratch + kOffBits);  // one buffer: flags updated in place
  f.bits_b = f.bits_a;
  f.out_mask = out_mask;
  f.maps = nullptr;
  f.counters = reinterpret_cast<unsigned long long*>(s->scratch + kOffCount);
  f.w = w;
  f.h = h;
  f.wpr = (w + 31) / 32;
  f.gain = gain;
  f.rn = readnoise;
  f.tiles_x = (w + kTW - 1) / kTW;
  f.rtiles_x = (w + kRW - 1) / kRW;
  f.tile0 = 0;
  f.rtile0 = 0;
  const long long tiles = (long long)f.tiles_x * ((h + kTH - 1) / kTH);
  const long long rtiles = (long long)f.rtiles_x * ((h + kRH - 1) / kRH);
  auto* desc = reinterpret_cast<crb::Frame*>(s->scratch + kOffDesc);
  const crb::Params p{sigclip, sigfrac, objlim, 0};

  noalloc_prepare<<<1, 128, 0, stream>>>(f, desc, f.counters, 2 * niter);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "crb_clean_noalloc: descriptor upload");
  if ((e = cudaMemsetAsync(f.bits_a, 0, sizeof(uint32_t) * size_t(f.wpr) * size_t(h), stream)) != cudaSuccess)
    return cuda_err(e, "crb_clean_noalloc: clearing flag bits");
  const int dgrid = int(std::min<long long>(tiles, (long long)s->sms * s->occ_detect));
  const int rgrid = int(std::min<long long>(rtiles, (long long)s->sms * s->occ_replace));
  for (int k = 1; k <= niter; ++k) {
    kDetect<<<dgrid, crb::kThreads, kDetectSmem, stream>>>(desc, 1, tiles, p, k, niter);
    kReplace<<<rgrid, crb::kThreads, kReplaceSmem, stream>>>(desc, 1, rtiles, k, niter, k <= 2 ? 1 : 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "crb_clean_noalloc launch");
  return CRB_OK;
}
