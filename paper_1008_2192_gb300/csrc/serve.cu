// Serving loop of the cleaner (declarations and contracts in include/crb.h).
//
// Continuous batching: submitted frames wait in a queue; a worker thread packs
// everything that is queued into the next "wave" (one crb_clean_batch call)
// as soon as one of max_inflight wave slots is free. Each slot has its own
// stream and context, so waves overlap on the GPU. A CUDA event marks the end
// of each wave; the worker polls the events and moves finished frames to the
// done queue, releasing their share of the memory budget.
//
// This is the GPU counterpart of CRBLASTER's director, which receives results
// from whichever actor is ready (MPI_Iprobe round robin, no barrier; Mighell
// 2010, Sec. 6.2 and 6.3.3); here whichever wave is done is collected.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "crb.h"

void crb_detail_set_error(const char* msg);  // crb.cu
void crb_detail_set_graphs(crb_ctx* c, int on);  // crb.cu

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Request {
  const float* img;
  float* out_clean;
  uint8_t* out_mask;
  int w, h;
  float gain, rn;
  uint64_t tag;
  size_t bytes;
  double t_submit;
};

struct Wave {
  std::vector<Request> reqs;
  cudaEvent_t done = nullptr;
  int slot = -1;
  double t_launch = 0;
};

struct Done {
  uint64_t tag;
  double t_submit, t_done;
  int status;
};

}  // namespace

struct crb_server {
  int device = 0;
  size_t budget = 0, resident = 0;
  int max_inflight = 2, max_batch = 64;
  float gain, rn, sigclip, sigfrac, objlim;
  int niter;
  crb_options opt{};

  std::vector<crb_ctx*> ctx;        // one per slot
  std::vector<cudaStream_t> stream;  // one per slot
  std::vector<bool> busy;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  std::vector<Wave> inflight;
  std::deque<Done> done;
  std::thread worker;
  std::atomic<bool> stop{false};
  int error = CRB_OK;
  // statistics
  long long n_submitted = 0, n_done = 0, n_waves = 0, n_rejected = 0, max_wave = 0;
  size_t peak_resident = 0;
  double max_enqueue_s = 0;      // longest enqueue of a wave (host time in crb_clean_batch and its event)
  double max_submit_wait_s = 0;  // longest time a submission waited for the server lock
};

namespace {

size_t frame_bytes(int w, int h) {
  // the caller's input, cleaned output and mask (resident while queued), and the
  // workspace of the queue pipeline: 4 float maps, 5 queue entries per pixel,
  // 14 bit planes (2 of them changed-pixel planes), 2 words per cell of one
  // word x 8 rows (the class arrays) and 3 words per segment of one word x 16
  // rows (the segment lists)
  const size_t n = size_t(w) * size_t(h);
  const size_t wpr = size_t(w + 31) / 32;
  const size_t plane = wpr * size_t(h) * 4;
  const size_t cells = wpr * ((size_t(h) + 7) / 8);
  const size_t segs = 32 * ((wpr + 31) / 32) * ((size_t(h) + 15) / 16);
  return n * (4 + 4 + 1) + n * 4 * 4 + n * 5 * 4 + 14 * plane + 2 * 4 * cells + 3 * 4 * segs;
}

// Enqueues one wave on slot `slot`. Called by the worker with the server lock
// held in `lk`; the lock is released while the wave is enqueued (which can take
// milliseconds: a first call of a signature grows the slot's workspace or
// captures a graph), so that submissions and polls are not held up, and taken
// again to publish the wave. Only the worker uses the slot's context and stream.
void launch_wave(crb_server* s, int slot, std::vector<Request>&& reqs, std::unique_lock<std::mutex>& lk) {
  Wave wv;
  wv.reqs = std::move(reqs);
  wv.slot = slot;
  s->busy[size_t(slot)] = true;
  lk.unlock();
  wv.t_launch = now_s();
  const int n = int(wv.reqs.size());
  std::vector<const float*> imgs(size_t(n), nullptr);
  std::vector<float*> outs(size_t(n), nullptr);
  std::vector<uint8_t*> masks(size_t(n), nullptr);
  std::vector<int> ws(static_cast<size_t>(n)), hs(static_cast<size_t>(n));
  std::vector<float> gs(static_cast<size_t>(n)), rs(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const Request& r = wv.reqs[size_t(i)];
    imgs[size_t(i)] = r.img;
    outs[size_t(i)] = r.out_clean;
    masks[size_t(i)] = r.out_mask;
    ws[size_t(i)] = r.w;
    hs[size_t(i)] = r.h;
    gs[size_t(i)] = r.gain;
    rs[size_t(i)] = r.rn;
  }
  // a single frame's launch signature repeats across waves (a handful of frame sizes), so its
  // work is captured once per size and replayed; a mixed wave's signature rarely repeats
  crb_detail_set_graphs(s->ctx[size_t(slot)], n == 1);
  int rc = crb_clean_batch(s->ctx[size_t(slot)], n, imgs.data(), ws.data(), hs.data(), gs.data(), rs.data(),
                           outs.data(), masks.data(), s->stream[size_t(slot)]);
  if (rc == CRB_OK && cudaEventCreateWithFlags(&wv.done, cudaEventDisableTiming) != cudaSuccess) rc = CRB_ECUDA;
  if (rc == CRB_OK && cudaEventRecord(wv.done, s->stream[size_t(slot)]) != cudaSuccess) rc = CRB_ECUDA;
  const double t_enq = now_s() - wv.t_launch;
  lk.lock();
  s->max_enqueue_s = std::max(s->max_enqueue_s, t_enq);
  if (rc != CRB_OK) {  // report every frame of the wave as failed
    for (const Request& r : wv.reqs) {
      s->done.push_back(Done{r.tag, r.t_submit, now_s(), rc});
      s->resident -= r.bytes;
    }
    if (wv.done) cudaEventDestroy(wv.done);
    s->busy[size_t(slot)] = false;
    s->error = rc;
    s->cv_done.notify_all();
    return;
  }
  s->n_waves += 1;
  s->max_wave = std::max<long long>(s->max_wave, n);
  s->inflight.push_back(std::move(wv));
}

void worker_main(crb_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop.load()) {
    // collect finished waves
    bool progressed = false;
    for (size_t i = 0; i < s->inflight.size();) {
      Wave& wv = s->inflight[i];
      const cudaError_t q = cudaEventQuery(wv.done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const double t = now_s();
      const int st = (q == cudaSuccess) ? crb_sync_status(s->ctx[size_t(wv.slot)], s->stream[size_t(wv.slot)])
                                        : CRB_ECUDA;
      for (const Request& r : wv.reqs) {
        s->done.push_back(Done{r.tag, r.t_submit, t, st});
        s->resident -= r.bytes;
        s->n_done += 1;
      }
      cudaEventDestroy(wv.done);
      s->busy[size_t(wv.slot)] = false;
      s->inflight.erase(s->inflight.begin() + long(i));
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // launch the next wave from everything queued, if a slot is free
    if (!s->pending.empty()) {
      int slot = -1;
      for (int i = 0; i < s->max_inflight; ++i)
        if (!s->busy[size_t(i)]) {
          slot = i;
          break;
        }
      if (slot >= 0) {
        std::vector<Request> reqs;
        while (!s->pending.empty() && int(reqs.size()) < s->max_batch) {
          reqs.push_back(s->pending.front());
          s->pending.pop_front();
        }
        launch_wave(s, slot, std::move(reqs), lk);
        continue;
      }
    }
    // wait for a submission, or poll the in-flight events again shortly
    if (s->inflight.empty() && s->pending.empty())
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      lk.lock();
    }
  }
}

}  // namespace

extern "C" {

crb_server* crb_server_create(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter,
                              const crb_options* opts, size_t budget_bytes, int max_inflight, int max_batch) {
  if (max_inflight < 1 || max_inflight > 16 || max_batch < 1 || budget_bytes == 0) {
    crb_detail_set_error("crb_server_create: need 1 <= max_inflight <= 16, max_batch >= 1, budget_bytes > 0");
    return nullptr;
  }
  auto* s = new crb_server();
  s->budget = budget_bytes;
  s->max_inflight = max_inflight;
  s->max_batch = max_batch;
  s->gain = gain;
  s->rn = readnoise;
  s->sigclip = sigclip;
  s->sigfrac = sigfrac;
  s->objlim = objlim;
  s->niter = niter;
  if (opts) s->opt = *opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    crb_detail_set_error("crb_server_create: no CUDA device");
    delete s;
    return nullptr;
  }
  for (int i = 0; i < max_inflight; ++i) {
    crb_ctx* c = crb_create_ex(gain, readnoise, sigclip, sigfrac, objlim, niter, opts);
    cudaStream_t st = nullptr;
    if (!c || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      if (c) crb_destroy(c);
      for (auto* x : s->ctx) crb_destroy(x);
      for (auto y : s->stream) cudaStreamDestroy(y);
      delete s;
      return nullptr;
    }
    s->ctx.push_back(c);
    s->stream.push_back(st);
    s->busy.push_back(false);
  }
  s->worker = std::thread(worker_main, s);
  return s;
}

int crb_server_submit(crb_server* s, const float* img, int w, int h, float gain, float readnoise, float* out_clean,
                      uint8_t* out_mask, uint64_t tag) {
  if (!s) return CRB_EINVAL;
  if (w < 1 || h < 1 || (long long)w * h >= (1LL << 31) || !img || !out_clean || !out_mask || !(gain > 0.f) ||
      !(readnoise >= 0.f)) {
    crb_detail_set_error("crb_server_submit: invalid frame");
    return CRB_EINVAL;
  }
  const size_t need = frame_bytes(w, h);
  if (need > s->budget) {  // could never be admitted: refusing it as busy would have the caller retry forever
    crb_detail_set_error(("crb_server_submit: a " + std::to_string(w) + "x" + std::to_string(h) + " frame counts " +
                          std::to_string(need) + " bytes, more than the whole budget of " + std::to_string(s->budget))
                             .c_str());
    return CRB_EINVAL;
  }
  const double t0 = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_submit_wait_s = std::max(s->max_submit_wait_s, now_s() - t0);
  if (s->error != CRB_OK) return s->error;
  if (need > s->budget - std::min(s->budget, s->resident)) {
    s->n_rejected += 1;
    crb_detail_set_error("crb_server_submit: memory budget exhausted; poll and resubmit");
    return CRB_EBUSY;
  }
  s->resident += need;
  s->peak_resident = std::max(s->peak_resident, s->resident);
  s->pending.push_back(Request{img, out_clean, out_mask, w, h, gain, readnoise, tag, need, now_s()});
  s->n_submitted += 1;
  s->cv_work.notify_one();
  return CRB_OK;
}

int crb_server_poll(crb_server* s, uint64_t* done_tags, double* latency_s, int* status, int max, int block_ms) {
  if (!s || max < 0 || (max > 0 && !done_tags)) return -1;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && block_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(block_ms), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < max && !s->done.empty()) {
    const Done d = s->done.front();
    s->done.pop_front();
    done_tags[n] = d.tag;
    if (latency_s) latency_s[n] = d.t_done - d.t_submit;
    if (status) status[n] = d.status;
    ++n;
  }
  return n;
}

size_t crb_server_frame_bytes(int w, int h) { return (w < 1 || h < 1) ? 0 : frame_bytes(w, h); }

int crb_server_stats(crb_server* s, long long* out, int max) {
  if (!s || !out || max < 0) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  const long long v[10] = {s->n_submitted,       s->n_done,
                           s->n_waves,           s->max_wave,
                           s->n_rejected,        (long long)s->resident,
                           (long long)s->peak_resident, (long long)s->pending.size(),
                           (long long)(s->max_enqueue_s * 1e6), (long long)(s->max_submit_wait_s * 1e6)};
  const int k = std::min(max, 10);
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return k;
}

void crb_server_destroy(crb_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& wv : s->inflight) {
    cudaEventSynchronize(wv.done);
    cudaEventDestroy(wv.done);
  }
  for (auto* c : s->ctx) crb_destroy(c);
  for (auto st : s->stream) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
