// Render server: continuous batching of camera requests against a resident
// Gaussian set (gs_serve_* in include/gs.h).
//
// The paper's goal is interactive visualisation of the trained splats
// (Sections I and V); serving renders arbitrary orbit cameras of a trained,
// resident model.  A worker thread forms batches from the pending requests as
// slots and memory free up and launches each batch (projection, binning and
// forward compositing, the same kernels as training) on its own slot, i.e. its
// own context and CUDA stream, so batches overlap on the device.  Completion
// is signalled by a host callback on the slot's stream; gs_serve_poll waits
// for it.  Outputs go either to a caller buffer or to a region of the server's
// output pool (first-fit), and a request is admitted only when its output
// region and its workspace estimate fit the memory budget.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct Request {
  gs_camera cam;
  float* out = nullptr;      // destination (caller's or pool)
  int64_t pool_off = -1;     // offset in the output pool, -1 if caller-owned
  size_t out_bytes = 0;
  size_t work_bytes = 0;     // workspace estimate charged while running
  int state = kPending;
  gs_status result = GS_OK;
};

struct Slot {
  gs_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  float* batch = nullptr;    // batch image buffer
  size_t batch_cap = 0;
  std::vector<uint64_t> tickets;
  size_t charged = 0;
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
  size_t mem_in_use = 0;     // workspace estimates of running batches
  char* pool_base = nullptr;
  Pool pool;
  int64_t batches = 0, rendered = 0;
};

namespace {

size_t workspace_estimate(const gs_server* s, const gs_camera& c) {
  // per view: projected records and tile counts of every Gaussian, about three
  // tile instances per visible Gaussian (keys and values, double-buffered),
  // per-pixel state and the batch image
  const size_t n = (size_t)s->resident.stride;
  const size_t px = (size_t)c.width * (size_t)c.height;
  return n * (52 + 3 * 24) + px * (8 + 12);
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

// Retire finished slots (caller holds the lock).
void retire(gs_server* s) {
  for (auto& sl : s->slots) {
    if (!sl.busy || !sl.finished) continue;
    for (uint64_t t : sl.tickets) {
      auto it = s->reqs.find(t);
      if (it != s->reqs.end()) it->second.state = kDone;
    }
    s->mem_in_use -= sl.charged;
    sl.charged = 0;
    sl.tickets.clear();
    sl.busy = sl.finished = false;
    s->cv_done.notify_all();
  }
}

gs_status launch_batch(gs_server* s, Slot& sl, std::vector<gs_camera>& cams, std::vector<Request*>& rq) {
  cudaSetDevice(s->device);
  size_t total = 0;
  for (auto& c : cams) total += (size_t)3 * c.width * c.height;
  if (sl.batch_cap < total) {
    if (sl.batch) {
      cudaStreamSynchronize(sl.stream);
      cudaFree(sl.batch);
    }
    sl.batch = nullptr;
    sl.batch_cap = 0;
    if (cudaMalloc(&sl.batch, total * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      return GS_ENOMEM;
    }
    sl.batch_cap = total;
  }
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
    // form a batch from the oldest pending requests that fit
    std::vector<gs_camera> cams;
    std::vector<Request*> rq;
    std::vector<uint64_t> tickets;
    size_t charge = 0;
    const size_t budget = (size_t)s->cfg.memory_budget_bytes;
    while (!s->pending.empty() && (int)cams.size() < s->cfg.max_batch_views) {
      const uint64_t t = s->pending.front();
      Request& r = s->reqs[t];
      if (s->mem_in_use + charge + r.work_bytes > budget && !cams.empty()) break;
      if (s->mem_in_use + charge + r.work_bytes > budget && s->mem_in_use > 0) break;  // wait for memory
      s->pending.pop_front();
      charge += r.work_bytes;
      r.state = kRunning;
      cams.push_back(r.cam);
      rq.push_back(&r);
      tickets.push_back(t);
    }
    if (cams.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    Slot& sl = *free_slot;
    sl.busy = true;
    sl.finished = false;
    sl.tickets = tickets;
    sl.charged = charge;
    s->mem_in_use += charge;
    s->batches++;
    s->rendered += (int64_t)cams.size();
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
      s->mem_in_use -= sl.charged;
      sl.charged = 0;
      sl.tickets.clear();
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
  if (c.memory_budget_bytes <= 0) c.memory_budget_bytes = (int64_t)16 << 30;
  if (c.output_pool_bytes < 0) return GS_EINVAL;
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
  for (auto& sl : s->slots) {
    sl.srv = s;
    gs_config gc{};
    gc.max_views = c.max_batch_views;
    if (gs_create(&sl.ctx, device, &gc) != GS_OK ||
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      gs_serve_destroy(s);
      return GS_ECUDA;
    }
    gs_set_stream(sl.ctx, sl.stream);
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
  }
  if (s->pool_base) cudaFree(s->pool_base);
  delete s;
}

gs_status gs_serve_submit(gs_server* s, const gs_camera* cam, float* out_device, uint64_t* ticket) {
  if (!s || !cam || !ticket) return GS_EINVAL;
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 65536 || cam->height > 65536 || !(cam->fx > 0.f) ||
      !(cam->fy > 0.f))
    return GS_EINVAL;
  Request r;
  r.cam = *cam;
  r.out_bytes = (size_t)3 * cam->width * cam->height * sizeof(float);
  r.work_bytes = workspace_estimate(s, *cam) + r.out_bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->pending.size() >= s->cfg.max_queue) return GS_EBUSY;
  if (r.work_bytes > (size_t)s->cfg.memory_budget_bytes) return GS_EBUSY;
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

gs_status gs_serve_stats(gs_server* s, int64_t* batches, int64_t* rendered, int64_t* pending) {
  if (!s) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (rendered) *rendered = s->rendered;
  if (pending) *pending = (int64_t)s->pending.size();
  return GS_OK;
}

}  // extern "C"
