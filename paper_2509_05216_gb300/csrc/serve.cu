// Render server: continuous batching of camera requests against a resident
// Gaussian set (gs_serve_* in include/gs.h).
//
// The paper's goal is interactive visualisation of the trained splats
// (Sections I and V); serving renders arbitrary orbit cameras of a trained,
// resident model.  A worker thread forms batches from the pending requests as
// slots free up and launches each batch (projection, binning and forward
// compositing, the same kernels as training) on its own slot, i.e. its own
// context and CUDA stream, so batches overlap on the device.
//
// Nothing on the launch path waits for the device or allocates: every slot
// context is created once with a fixed instance capacity and workspaces
// reserved for the largest admissible batch (max_batch_views views of
// max_view_pixels), sized from the memory budget.  A batch's sort is bounded
// by an instance estimate (per resolution, the most instances a view of that
// size has needed so far, plus a margin); its status word and per-view
// instance counts are copied back asynchronously and read when the batch
// retires.  A batch that overflowed its estimate is put back at the front of
// the queue (the estimates have learnt the true counts by then); a bounded
// device wait that ran out fails the batch's requests with GS_ETIMEOUT.
// Completion is signalled by a host callback on the slot's stream;
// gs_serve_poll waits for it.  Outputs go either to a caller buffer or to a
// region of the server's output pool (first-fit).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx_internal.h"
#include "gs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kTimelineCap = 4096;  // batches kept for gs_serve_timeline
constexpr int kMaxRetries = 4;      // capacity retries of one request
constexpr int32_t kDefaultViewPixels = 3840 * 2160;
// reservation per slot (documented with gs_serve_cfg): per view 72 bytes per
// Gaussian (records, tile rect, tile count), 20 bytes per pixel (T_final,
// n_last, batch image) and 8 per tile (ranges); 26 bytes per tile instance
// (keys and values double-buffered, sort look-back)
constexpr int64_t kGaussBytes = 72, kPixelBytes = 20, kTileBytes = 8, kInstanceBytes = 26;
constexpr int64_t kSlackBytes = 1 << 20;
constexpr int64_t kMaxInstances = ((int64_t)1 << 30) - 2;
constexpr int64_t kMinInstances = 1 << 16;

int64_t max_view_tiles(const gs_serve_cfg& c) { return (int64_t)c.max_view_pixels / 128 + 64; }

int64_t slot_fixed_bytes(const gs_serve_cfg& c, int64_t stride) {
  const int64_t B = c.max_batch_views;
  return B * (kGaussBytes * stride + kPixelBytes * (int64_t)c.max_view_pixels + kTileBytes * max_view_tiles(c)) +
         kSlackBytes;
}

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct Request {
  gs_camera cam;
  float* out = nullptr;      // destination (caller's or pool)
  int64_t pool_off = -1;     // offset in the output pool, -1 if caller-owned
  size_t out_bytes = 0;
  int retries = 0;           // capacity overflows so far
  int state = kPending;
  gs_status result = GS_OK;
};

struct Slot {
  gs_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  float* batch = nullptr;    // batch image buffer, reserved at creation
  std::vector<uint64_t> tickets;
  std::vector<int64_t> pixels;   // W * H of each view of the running batch
  int64_t capacity = 0;      // instance capacity of the slot context
  int64_t estimate = 0;      // instance capacity given to the running batch
  int* status_h = nullptr;   // page-locked: the batch's status word
  uint64_t* totals_h = nullptr;  // page-locked: its per-view instance counts
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  bool busy = false;
  bool finished = false;     // set by the stream callback
  struct gs_server* srv = nullptr;
};

// First-fit allocator over the output pool (offsets in bytes, 256-aligned).
class Pool {
 public:
  void init(size_t size) { free_[0] = size; }
  int64_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        return (int64_t)off;
      }
    }
    return -1;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

}  // namespace

struct gs_server {
  int device = 0;
  gs_params resident{};
  gs_serve_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  char* pool_base = nullptr;
  Pool pool;
  int64_t batches = 0, rendered = 0, retried = 0;
  // most instances one view of a given pixel count has needed so far
  std::map<int64_t, uint64_t> view_instances;
  cudaEvent_t ev_origin = nullptr;     // start of the device timeline
  std::vector<double> timeline;        // (start, end) ms of retired batches
};

namespace {

// Instance estimate of one view (caller holds the lock): 1.25 x the most a
// view of the same pixel count has needed, or, for a size not seen yet, two
// instances per resident Gaussian plus four per pixel.
int64_t view_estimate(const gs_server* s, const gs_camera& c) {
  const int64_t px = (int64_t)c.width * c.height;
  auto it = s->view_instances.find(px);
  if (it == s->view_instances.end()) return 2 * s->resident.n + 4 * px;
  return (int64_t)(it->second + it->second / 4) + 4096;
}

void CUDART_CB on_batch_done(void* user) {
  Slot* sl = static_cast<Slot*>(user);
  gs_server* s = sl->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    sl->finished = true;
  }
  s->cv_work.notify_all();
}

// Retire finished slots (caller holds the lock): learn the per-view instance
// counts, then complete the requests, or put them back at the front of the
// queue after a capacity overflow.
void retire(gs_server* s) {
  for (auto& sl : s->slots) {
    if (!sl.busy || !sl.finished) continue;
    const int st = *sl.status_h;
    for (size_t v = 0; v < sl.pixels.size(); v++) {
      uint64_t& m = s->view_instances[sl.pixels[v]];
      m = std::max(m, sl.totals_h[v]);
    }
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, s->ev_origin, sl.ev_start) == cudaSuccess &&
        cudaEventElapsedTime(&t1, s->ev_origin, sl.ev_end) == cudaSuccess) {
      if (s->timeline.size() >= 2 * (size_t)kTimelineCap) s->timeline.erase(s->timeline.begin(), s->timeline.begin() + 2);
      s->timeline.push_back(t0);
      s->timeline.push_back(t1);
    } else {
      (void)cudaGetLastError();
    }
    const bool overflow = (st & gs::kStatusCapacity) != 0, timeout = (st & gs::kStatusTimeout) != 0;
    // requeue in the original order at the front (a request that overflowed
    // the whole slot capacity alone, or too often, fails instead)
    for (auto t = sl.tickets.rbegin(); t != sl.tickets.rend(); ++t) {
      auto it = s->reqs.find(*t);
      if (it == s->reqs.end()) continue;
      Request& r = it->second;
      if (timeout) {
        r.state = kDone;
        r.result = GS_ETIMEOUT;
      } else if (overflow) {
        const bool hopeless = (sl.tickets.size() == 1 && sl.estimate >= sl.capacity) || r.retries >= kMaxRetries;
        if (hopeless) {
          r.state = kDone;
          r.result = GS_ECAPACITY;
        } else {
          r.retries++;
          r.state = kPending;
          s->pending.push_front(*t);
        }
      } else {
        r.state = kDone;
        r.result = GS_OK;
        s->rendered++;
      }
    }
    if (overflow && !timeout) s->retried++;
    sl.tickets.clear();
    sl.pixels.clear();
    sl.busy = sl.finished = false;
    s->cv_done.notify_all();
  }
}

// Launch one batch on a slot; nothing here waits for the device or
// allocates (every workspace was reserved when the slot was created).
gs_status launch_batch(gs_server* s, Slot& sl, std::vector<gs_camera>& cams, std::vector<Request*>& rq) {
  cudaSetDevice(s->device);
  gs::ctx_set_batch_capacity(sl.ctx, sl.estimate);
  if (cudaEventRecord(sl.ev_start, sl.stream) != cudaSuccess) return GS_ECUDA;
  gs_status st = gs_project(sl.ctx, &s->resident, cams.data(), (int32_t)cams.size());
  if (st == GS_OK) st = gs_bin_sort(sl.ctx);
  if (st == GS_OK) st = gs_raster_fwd(sl.ctx, sl.batch);
  if (st != GS_OK) return st;
  size_t off = 0;
  for (size_t i = 0; i < rq.size(); i++) {
    const size_t bytes = (size_t)3 * cams[i].width * cams[i].height * sizeof(float);
    if (cudaMemcpyAsync(rq[i]->out, sl.batch + off, bytes, cudaMemcpyDeviceToDevice, sl.stream) != cudaSuccess)
      return GS_ECUDA;
    off += bytes / sizeof(float);
  }
  st = gs::ctx_read_status_async(sl.ctx, sl.status_h, sl.totals_h, (int)cams.size());
  if (st != GS_OK) return st;
  if (cudaEventRecord(sl.ev_end, sl.stream) != cudaSuccess) return GS_ECUDA;
  if (cudaLaunchHostFunc(sl.stream, on_batch_done, &sl) != cudaSuccess) return GS_ECUDA;
  return GS_OK;
}

void worker_main(gs_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    retire(s);
    Slot* free_slot = nullptr;
    for (auto& sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot || s->pending.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // form a batch from the oldest pending requests whose instance
    // estimates fit the slot's reserved capacity (at least one request)
    Slot& sl = *free_slot;
    std::vector<gs_camera> cams;
    std::vector<Request*> rq;
    std::vector<uint64_t> tickets;
    std::vector<int64_t> pixels;
    int64_t est = 65536;
    while (!s->pending.empty() && (int)cams.size() < s->cfg.max_batch_views) {
      const uint64_t t = s->pending.front();
      Request& r = s->reqs[t];
      const int64_t e = view_estimate(s, r.cam);
      if (!cams.empty() && est + e > sl.capacity) break;
      s->pending.pop_front();
      est += e;
      r.state = kRunning;
      cams.push_back(r.cam);
      rq.push_back(&r);
      tickets.push_back(t);
      pixels.push_back((int64_t)r.cam.width * r.cam.height);
    }
    sl.busy = true;
    sl.finished = false;
    sl.tickets = tickets;
    sl.pixels = pixels;
    sl.estimate = std::min(est, sl.capacity);
    s->batches++;
    lk.unlock();
    const gs_status st = launch_batch(s, sl, cams, rq);
    lk.lock();
    if (st != GS_OK) {
      for (uint64_t t : tickets) {
        auto it = s->reqs.find(t);
        if (it != s->reqs.end()) {
          it->second.state = kDone;
          it->second.result = st;
        }
      }
      sl.tickets.clear();
      sl.pixels.clear();
      sl.busy = false;
      s->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

gs_status gs_serve_create(gs_server** out, int device, const gs_params* resident, const gs_serve_cfg* cfg) {
  if (!out || !resident || !resident->data || resident->n <= 0 || resident->stride < resident->n ||
      resident->stride % 4 != 0 || resident->sh_degree < 0 || resident->sh_degree > 3)
    return GS_EINVAL;
  *out = nullptr;
  gs_serve_cfg c{};
  if (cfg) c = *cfg;
  if (c.slots <= 0) c.slots = 2;
  if (c.slots > 16) return GS_EINVAL;
  if (c.max_batch_views <= 0) c.max_batch_views = 16;
  if (c.max_batch_views > 64) return GS_EINVAL;
  if (c.max_queue <= 0) c.max_queue = 4096;
  if (c.max_view_pixels <= 0) c.max_view_pixels = kDefaultViewPixels;
  if (c.memory_budget_bytes <= 0) c.memory_budget_bytes = (int64_t)16 << 30;
  if (c.output_pool_bytes < 0) return GS_EINVAL;
  // per slot: fixed workspaces of the largest batch, then tile instances
  const int64_t fixed = slot_fixed_bytes(c, resident->stride);
  const int64_t share = c.memory_budget_bytes / c.slots;
  const int64_t capacity = std::min<int64_t>((share - fixed) / kInstanceBytes, kMaxInstances);
  if (capacity < kMinInstances) return GS_EINVAL;  // budget too small for the slots' reservations
  gs_server* s = new gs_server();
  s->device = device;
  s->resident = *resident;
  s->cfg = c;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete s;
    return GS_ECUDA;
  }
  if (c.output_pool_bytes > 0) {
    if (cudaMalloc(&s->pool_base, (size_t)c.output_pool_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      delete s;
      return GS_ENOMEM;
    }
    s->pool.init((size_t)c.output_pool_bytes);
  }
  s->slots.resize(c.slots);
  const int64_t B = c.max_batch_views, px = c.max_view_pixels;
  for (auto& sl : s->slots) {
    sl.srv = s;
    sl.capacity = capacity;
    gs_config gc{};
    gc.max_views = c.max_batch_views;
    gc.instance_capacity = capacity;
    if (gs_create(&sl.ctx, device, &gc) != GS_OK ||
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.ev_start) != cudaSuccess || cudaEventCreate(&sl.ev_end) != cudaSuccess ||
        cudaMallocHost(&sl.status_h, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&sl.totals_h, sizeof(uint64_t) * gs::kMaxViews) != cudaSuccess) {
      (void)cudaGetLastError();
      gs_serve_destroy(s);
      return GS_ECUDA;
    }
    gs_set_stream(sl.ctx, sl.stream);
    gs::ctx_set_forward_only(sl.ctx, true);
    // every workspace of the largest admissible batch, once
    const gs_status rs = gs::ctx_reserve(sl.ctx, resident->stride, (int)B, B * max_view_tiles(c), B * px,
                                         max_view_tiles(c));
    if (rs != GS_OK || cudaMalloc(&sl.batch, sizeof(float) * 3 * B * px) != cudaSuccess) {
      (void)cudaGetLastError();
      sl.batch = nullptr;
      gs_serve_destroy(s);
      return GS_ENOMEM;
    }
  }
  if (cudaEventCreate(&s->ev_origin) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
      cudaEventRecord(s->ev_origin, s->slots[0].stream) != cudaSuccess) {
    (void)cudaGetLastError();
    gs_serve_destroy(s);
    return GS_ECUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return GS_OK;
}

void gs_serve_destroy(gs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.batch) cudaFree(sl.batch);
    if (sl.ctx) gs_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.ev_end) cudaEventDestroy(sl.ev_end);
    if (sl.status_h) cudaFreeHost(sl.status_h);
    if (sl.totals_h) cudaFreeHost(sl.totals_h);
  }
  if (s->ev_origin) cudaEventDestroy(s->ev_origin);
  if (s->pool_base) cudaFree(s->pool_base);
  delete s;
}

gs_status gs_serve_submit(gs_server* s, const gs_camera* cam, float* out_device, uint64_t* ticket) {
  if (!s || !cam || !ticket) return GS_EINVAL;
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 65536 || cam->height > 65536 || !(cam->fx > 0.f) ||
      !(cam->fy > 0.f))
    return GS_EINVAL;
  const int64_t tiles = (int64_t)((cam->width + gs::kTile - 1) / gs::kTile) * ((cam->height + gs::kTile - 1) / gs::kTile);
  if ((int64_t)cam->width * cam->height > s->cfg.max_view_pixels || tiles > max_view_tiles(s->cfg)) return GS_EINVAL;
  Request r;
  r.cam = *cam;
  r.out_bytes = (size_t)3 * cam->width * cam->height * sizeof(float);
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->pending.size() >= s->cfg.max_queue) return GS_EBUSY;
  if (out_device) {
    r.out = out_device;
  } else {
    if (!s->pool_base) return GS_EINVAL;
    const int64_t off = s->pool.alloc(r.out_bytes);
    if (off < 0) return GS_EBUSY;  // output pool full: poll and release earlier results
    r.pool_off = off;
    r.out = reinterpret_cast<float*>(s->pool_base + off);
  }
  const uint64_t t = s->next_ticket++;
  s->reqs.emplace(t, r);
  s->pending.push_back(t);
  *ticket = t;
  s->cv_work.notify_all();
  return GS_OK;
}

gs_status gs_serve_poll(gs_server* s, uint64_t ticket, int64_t timeout_us, const float** image, gs_status* result) {
  if (!s) return GS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GS_EINVAL;
  // negative or huge timeouts wait (practically) forever; cap to keep the
  // deadline arithmetic in range
  const int64_t cap_us = (int64_t)1 << 40;  // about 12 days
  const int64_t wait_us = (timeout_us < 0 || timeout_us > cap_us) ? cap_us : timeout_us;
  const auto deadline = Clock::now() + std::chrono::microseconds(wait_us);
  while (it->second.state != kDone) {
    if (timeout_us == 0) return GS_EAGAIN;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state != kDone)
      return GS_EAGAIN;
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GS_EINVAL;
  }
  if (image) *image = it->second.out;
  if (result) *result = it->second.result;
  return GS_OK;
}

gs_status gs_serve_release(gs_server* s, uint64_t ticket) {
  if (!s) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GS_EINVAL;
  if (it->second.state != kDone) return GS_EBUSY;
  if (it->second.pool_off >= 0) s->pool.release((size_t)it->second.pool_off, it->second.out_bytes);
  s->reqs.erase(it);
  return GS_OK;
}

gs_status gs_serve_timeline(gs_server* s, double* start_end_ms, int32_t cap, int32_t* count, int64_t* retried) {
  if (!s || !count || cap < 0 || (cap > 0 && !start_end_ms)) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const int32_t have = (int32_t)(s->timeline.size() / 2);
  const int32_t k = std::min(have, cap);
  for (int32_t i = 0; i < k; i++) {
    start_end_ms[2 * i] = s->timeline[2 * (size_t)(have - k + i)];
    start_end_ms[2 * i + 1] = s->timeline[2 * (size_t)(have - k + i) + 1];
  }
  *count = k;
  if (retried) *retried = s->retried;
  return GS_OK;
}

gs_status gs_serve_stats(gs_server* s, int64_t* batches, int64_t* rendered, int64_t* pending) {
  if (!s) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (rendered) *rendered = s->rendered;
  if (pending) *pending = (int64_t)s->pending.size();
  return GS_OK;
}

}  // extern "C"
