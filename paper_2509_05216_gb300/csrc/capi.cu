// Host side of the C ABI declared in include/gs.h: context, workspaces,
// argument checks and the launch sequence of each step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx_internal.h"
#include "gs_internal.cuh"
#include "launch.h"

using namespace gs;

namespace {

constexpr size_t kViewStagingBytes = sizeof(ViewRec) * kMaxViews;
constexpr size_t kAdamStagingOff = kViewStagingBytes;
constexpr size_t kTargetStagingOff = kViewStagingBytes + 72 * sizeof(float);  // 8-byte aligned
constexpr size_t kStagingBytes = kTargetStagingOff + sizeof(void*);

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct gs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  gs_config cfg{};
  std::string err;
  int* status_d = nullptr;
  int* status_h = nullptr;     // pinned
  uint64_t* pinned = nullptr;  // pinned scratch for small read-backs (16 KB)
  // pinned staging of the per-step constants (cameras, Adam constants) read by
  // the copies of a captured training graph
  unsigned char* staging = nullptr;
  bool capturing = false;
  cudaStream_t graph_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t staged_ev = nullptr;  // the graph's staging copies have run
  // a captured step clears the 2D-gradient records on a side branch that
  // runs beside the forward compositing (fork and join events)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool g2d_cleared = false;  // the next gs_raster_bwd finds the records zeroed
  int graph_B = 0;
  std::vector<int> graph_res;        // W, H per view of the captured batch
  gs_adam_hp graph_hp{};
  int64_t graph_kernels = 0;         // kernels per replay
  int graph_planes = 0;
  float* graph_loss = nullptr;       // device loss the graph writes
  int64_t graph_count = 0;           // image elements per step
  // host-target replays: targets uploaded on a copy stream into two device
  // buffers, so the upload of step k + 1 overlaps step k
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t tgt_copied[2] = {nullptr, nullptr};
  cudaEvent_t tgt_free[2] = {nullptr, nullptr};
  int64_t host_launches = 0;
  int raster_fwd = 2;  // compositing variants (pixels per thread; 8 = one warp per tile)
  int raster_bwd = 2;
  int bwd_direct = 2;  // per-lane gradient atomics when at most this many lanes contribute
  int sort_passes = 0;  // LSD passes of the last tile sort
  int sort_items = 16;  // keys per thread of a sort partition
  int sort_wait = 1 << 20;  // look-back rounds before a sort gives up
  int tile_order_mode = 0;  // 0: composite tiles in bin order; 1: longest lists first
  float* dens_grad = nullptr;   // densification statistic accumulated by gs_raster_bwd (caller-owned)
  float* dens_count = nullptr;
  bool tile_order_ready = false;
  int64_t batch_cap = 0;    // instance capacity of the next sorts (0: cfg.instance_capacity)
  bool forward_only = false;  // no contribution cells: gs_raster_bwd unavailable (render server)
  bool cells_ready = false;   // the last forward recorded contribution cells

  // last batch
  int B = 0, deg = 0;
  int64_t n = 0, stride = 0, bins = 0, pixels = 0, instances = 0, nblocks = 0;
  bool projected = false, sorted = false, rastered = false;
  std::vector<ViewRec> views_h;

  DevBuf views, rec, rec3, tiles, block_sums, block_offsets, total, keys0, keys1, vals0, vals1,
      hist, hist_scan, lookback, counters, ranges, tfinal, nlast, g2d, l1_partial, sorted_slots, adam_consts,
      target_slot, host_tgt0, host_tgt1, pair_stats, cells, vismask, ssim_table, ssim_partials, ssim_sums,
      init_pts, init_scales, knn_part, knn_table, ord_keys0, ord_keys1, ord_vals0, ord_vals1, ord_total, ord_hist,
      ord_hist_scan, ord_lookback, ord_counters, ord_views, tile_order, vis_sums, vis_offsets, dtotal, dkeys0,
      dkeys1, dvals0, dvals1, dhist, dhist_scan, dlookback, elookback, dorder, torder;

  // launch accounting and optional per-kernel event timing
  struct KStat {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
  };
  std::vector<KStat> kstats;
  struct Pending {
    int kernel;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  bool profiling = false;
};

namespace {

gs_status fail(gs_ctx* c, gs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

#define GS_CUDA(ctx, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      (void)cudaGetLastError(); /* do not leave it for the next launch check */             \
      return fail(ctx, GS_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                \
    }                                                                                       \
  } while (0)

#define GS_CHECK_LAUNCH(ctx)                                                                    \
  do {                                                                                          \
    cudaError_t e_ = cudaGetLastError();                                                        \
    if (e_ != cudaSuccess)                                                                      \
      return fail(ctx, GS_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                    \
  } while (0)

gs_status ensure(gs_ctx* c, DevBuf& b, size_t bytes, bool exact = false) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return GS_OK;
  size_t want = exact ? bytes : bytes + bytes / 8;
  if (b.p) {
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    GS_CUDA(c, cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    b.p = nullptr;
    return fail(c, GS_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", want, cudaGetErrorString(e));
  }
  b.cap = want;
  return GS_OK;
}

#define GS_TRY(expr)                  \
  do {                                \
    gs_status s_ = (expr);            \
    if (s_ != GS_OK) return s_;       \
  } while (0)

template <class T>
T* P(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

gs_status check_params(gs_ctx* c, const gs_params* p, const char* what) {
  if (!p) return fail(c, GS_EINVAL, "%s is NULL", what);
  if (!p->data) return fail(c, GS_EINVAL, "%s->data is NULL", what);
  if (p->n <= 0) return fail(c, GS_EINVAL, "%s->n must be > 0", what);
  if (p->n >= (int64_t)1 << 31) return fail(c, GS_EINVAL, "%s->n too large", what);
  if (p->stride < p->n || p->stride % 4 != 0)
    return fail(c, GS_EINVAL, "%s->stride must be >= n and a multiple of 4", what);
  if (p->sh_degree < 0 || p->sh_degree > 3) return fail(c, GS_EINVAL, "%s->sh_degree must be 0..3", what);
  if (reinterpret_cast<uintptr_t>(p->data) % 16 != 0) return fail(c, GS_EINVAL, "%s->data not 16-byte aligned", what);
  return GS_OK;
}

int kernel_index(gs_ctx* c, const char* name) {
  for (size_t i = 0; i < c->kstats.size(); i++)
    if (c->kstats[i].name == name) return (int)i;
  c->kstats.push_back(gs_ctx::KStat{name, 0, 0.0});
  return (int)c->kstats.size() - 1;
}

cudaEvent_t take_event(gs_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one library launch (of `kernels` kernels) for the accounting.
struct LaunchScope {
  gs_ctx* c;
  int k;
  cudaEvent_t a = nullptr;
  LaunchScope(gs_ctx* ctx, const char* name, int kernels = 1) : c(ctx), k(kernel_index(ctx, name)) {
    if (c->capturing) {  // counted per replay instead
      c->graph_kernels += kernels;
      return;
    }
    c->kstats[k].launches += kernels;
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~LaunchScope() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->pending.push_back(gs_ctx::Pending{k, a, b});
    }
  }
};

void set_device(gs_ctx* c) { cudaSetDevice(c->device); }

// Per-view records of a batch (host side), with each view's first tile bin
// and first pixel.
gs_status build_views(gs_ctx* c, const gs_camera* cams, int B, int64_t* tiles_out, int64_t* pixels_out) {
  c->views_h.assign(B, ViewRec{});
  int64_t tile_off = 0, pix_off = 0;
  for (int v = 0; v < B; v++) {
    const gs_camera& k = cams[v];
    if (k.width <= 0 || k.height <= 0 || k.width > 65536 || k.height > 65536)
      return fail(c, GS_EINVAL, "camera %d: bad size %dx%d", v, k.width, k.height);
    if (!(k.fx > 0.f) || !(k.fy > 0.f)) return fail(c, GS_EINVAL, "camera %d: focal must be > 0", v);
    ViewRec& r = c->views_h[v];
    for (int i = 0; i < 3; i++) {
      for (int j = 0; j < 3; j++) r.R[3 * i + j] = k.viewmat[4 * i + j];
      r.t[i] = k.viewmat[4 * i + 3];
    }
    r.fx = k.fx; r.fy = k.fy; r.cx = k.cx; r.cy = k.cy;
    r.znear = k.znear;
    r.limx = (float)(1.3 * (double)k.width / (2.0 * (double)k.fx));
    r.limy = (float)(1.3 * (double)k.height / (2.0 * (double)k.fy));
    for (int j = 0; j < 3; j++) {
      double s = 0.0;
      for (int i = 0; i < 3; i++) s -= (double)k.viewmat[4 * i + j] * (double)k.viewmat[4 * i + 3];
      r.campos[j] = (float)s;
      r.bg[j] = k.bg[j];
    }
    r.W = k.width; r.H = k.height;
    r.gw = (k.width + kTile - 1) / kTile;
    r.gh = (k.height + kTile - 1) / kTile;
    r.tile_offset = (int)tile_off;
    r.pix_offset = pix_off;
    tile_off += (int64_t)r.gw * r.gh;
    pix_off += (int64_t)k.width * k.height;
  }
  *tiles_out = tile_off;
  *pixels_out = pix_off;
  return GS_OK;
}

// Per-plane learning rate divided by the first-moment bias correction, and
// 1 / sqrt(second-moment bias correction) in slot 64.
void adam_constants(const gs_adam_hp* hp, int planes, int64_t step, int B, float* out) {
  const double bc1 = 1.0 - std::pow((double)hp->beta1, (double)step);
  const double bc2 = 1.0 - std::pow((double)hp->beta2, (double)step);
  const double lr_mul = (hp->flags & GS_ADAM_SQRT_BATCH_LR) ? std::sqrt((double)(B > 0 ? B : 1)) : 1.0;
  for (int pl = 0; pl < 64; pl++) {
    double lr = 0.0;
    if (pl < planes) {
      if (pl < 3) lr = hp->lr_mean;
      else if (pl < 6) lr = hp->lr_scale;
      else if (pl < 10) lr = hp->lr_quat;
      else if (pl < 11) lr = hp->lr_opacity;
      else if (pl < 14) lr = hp->lr_sh_dc;
      else lr = hp->lr_sh_rest;
    }
    out[pl] = (float)(lr * lr_mul / bc1);
  }
  out[64] = (float)(1.0 / std::sqrt(bc2));
}

}  // namespace

// Device words of one sort: total (u64) | view totals (u64 x 64) | seg (u32 x 65)
// | part_off (u32 x 65) | ctrl (u32 x 16) | single-digit flags (u32 x 64 x 8).
struct SortWords {
  uint64_t* total;
  uint64_t* view_total;
  uint32_t* seg;
  uint32_t* part_off;
  uint32_t* ctrl;
  uint32_t* single;
};

static size_t sort_words_bytes() {
  return sizeof(uint64_t) * (1 + kMaxViews) + sizeof(uint32_t) * (2 * (kMaxViews + 1) + 16 + 8 * kMaxViews);
}

static SortWords sort_words(DevBuf& b) {
  SortWords w;
  w.total = P<uint64_t>(b);
  w.view_total = w.total + 1;
  w.seg = reinterpret_cast<uint32_t*>(w.view_total + kMaxViews);
  w.part_off = w.seg + kMaxViews + 1;
  w.ctrl = w.part_off + kMaxViews + 1;
  w.single = w.ctrl + 16;
  return w;
}

constexpr int kDepthPasses = 4;  // 32 depth bits
constexpr int kSortCounters = 24;  // tickets: [0, 8) tile sort, [8, 16) depth sort, [16] emission

// LSD passes of the tile sort: the bits of the largest tile index inside a view.
static int tile_passes(int64_t view_tiles) {
  int bits = 0;
  while (((int64_t)1 << bits) < view_tiles) bits++;
  return std::max(1, (bits + 7) / 8);
}

namespace gs {

gs_status ctx_reserve(gs_ctx* c, int64_t stride, int B, int64_t bins, int64_t pixels, int64_t view_tiles) {
  if (!c || stride <= 0 || B < 1 || B > kMaxViews || bins < 1 || pixels < 1 || view_tiles < 1)
    return GS_EINVAL;
  if (c->cfg.instance_capacity <= 0) return fail(c, GS_EINVAL, "ctx_reserve needs a fixed instance capacity");
  set_device(c);
  auto ensure_exact = [](gs_ctx* cc, DevBuf& b, size_t bytes) { return ensure(cc, b, bytes, true); };
  const int64_t cap = c->cfg.instance_capacity;
  const int64_t nb = (stride + project_fwd_block() - 1) / project_fwd_block();
  const int tpass = tile_passes(view_tiles);
  const int64_t pc = (int64_t)B * stride;  // visible pairs at most
  GS_TRY(ensure_exact(c, c->views, sizeof(ViewRec) * B));
  GS_TRY(ensure_exact(c, c->rec, sizeof(float4) * kRecStride * B * stride));
  GS_TRY(ensure_exact(c, c->rec3, sizeof(int4) * B * stride));
  GS_TRY(ensure_exact(c, c->tiles, sizeof(uint2) * B * stride));
  GS_TRY(ensure_exact(c, c->block_sums, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure_exact(c, c->vis_sums, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure_exact(c, c->vismask, sizeof(uint64_t) * stride));
  GS_TRY(ensure_exact(c, c->block_offsets, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure_exact(c, c->vis_offsets, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure_exact(c, c->total, sort_words_bytes()));
  GS_TRY(ensure_exact(c, c->dtotal, sort_words_bytes()));
  GS_TRY(ensure_exact(c, c->keys0, sizeof(uint32_t) * cap));
  GS_TRY(ensure_exact(c, c->keys1, sizeof(uint32_t) * cap));
  GS_TRY(ensure_exact(c, c->vals0, sizeof(uint32_t) * cap));
  GS_TRY(ensure_exact(c, c->vals1, sizeof(uint32_t) * cap));
  GS_TRY(ensure_exact(c, c->dkeys0, sizeof(uint32_t) * pc));
  GS_TRY(ensure_exact(c, c->dkeys1, sizeof(uint32_t) * pc));
  GS_TRY(ensure_exact(c, c->dvals0, sizeof(uint32_t) * pc));
  GS_TRY(ensure_exact(c, c->dvals1, sizeof(uint32_t) * pc));
  GS_TRY(ensure_exact(c, c->ranges, sizeof(uint2) * bins));
  GS_TRY(ensure_exact(c, c->hist, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure_exact(c, c->hist_scan, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure_exact(c, c->dhist, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure_exact(c, c->dhist_scan, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure_exact(c, c->lookback, sort_lookback_bytes(cap, c->sort_items, B) * tpass));
  GS_TRY(ensure_exact(c, c->dlookback, sort_lookback_bytes(pc, c->sort_items, B) * kDepthPasses));
  GS_TRY(ensure_exact(c, c->elookback, emit_lookback_bytes(pc, B)));
  GS_TRY(ensure_exact(c, c->torder, sizeof(uint32_t) * sort_partitions(cap, c->sort_items, B)));
  GS_TRY(ensure_exact(c, c->dorder, sizeof(uint32_t) * sort_partitions(pc, c->sort_items, B)));
  GS_TRY(ensure_exact(c, c->counters, sizeof(uint32_t) * kSortCounters));
  GS_TRY(ensure_exact(c, c->sorted_slots, 2 * sizeof(void*)));
  GS_TRY(ensure_exact(c, c->tfinal, sizeof(float) * pixels));
  GS_TRY(ensure_exact(c, c->nlast, sizeof(uint32_t) * pixels));
  return GS_OK;
}

void ctx_set_batch_capacity(gs_ctx* c, int64_t cap) {
  if (c) c->batch_cap = cap > 0 ? cap : 0;
}

void ctx_set_forward_only(gs_ctx* c, bool on) {
  if (c) c->forward_only = on;
}

gs_status ctx_read_status_async(gs_ctx* c, int* status_host, uint64_t* view_totals_host, int B) {
  if (!c || !status_host || !view_totals_host || B < 1 || B > kMaxViews) return GS_EINVAL;
  if (!c->sorted) return fail(c, GS_ESTATE, "no sort to read");
  set_device(c);
  GS_CUDA(c, cudaMemcpyAsync(status_host, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream));
  GS_CUDA(c, cudaMemcpyAsync(view_totals_host, P<uint64_t>(c->total) + 1, sizeof(uint64_t) * B,
                             cudaMemcpyDeviceToHost, c->stream));
  return GS_OK;
}

}  // namespace gs

extern "C" {

gs_status gs_create(gs_ctx** out, int device, const gs_config* cfg) {
  if (!out) return GS_EINVAL;
  *out = nullptr;
  gs_config conf{};
  if (cfg) conf = *cfg;
  if (conf.max_views == 0) conf.max_views = kMaxViews;
  if (conf.max_views < 0 || conf.max_views > kMaxViews) return GS_EINVAL;
  if (conf.max_gaussians < 0 || conf.instance_capacity < 0) return GS_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return GS_ECUDA;
  }
  gs_ctx* c = new gs_ctx();
  c->device = device;
  c->cfg = conf;
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&c->status_d, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->status_d, 0, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->status_h, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->pinned, 16384) != cudaSuccess ||
      cudaMallocHost(&c->staging, kStagingBytes) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->staged_ev, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    gs_destroy(c);
    return GS_ECUDA;
  }
  *out = c;
  return GS_OK;
}

void gs_destroy(gs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->views, &c->rec, &c->rec3, &c->tiles, &c->block_sums, &c->block_offsets,
                    &c->total, &c->keys0, &c->keys1, &c->vals0, &c->vals1, &c->hist, &c->hist_scan,
                    &c->lookback, &c->counters, &c->ranges, &c->tfinal, &c->nlast, &c->g2d, &c->l1_partial,
                    &c->sorted_slots, &c->adam_consts, &c->target_slot, &c->host_tgt0, &c->host_tgt1,
                    &c->pair_stats, &c->cells, &c->vismask, &c->ssim_table, &c->ssim_partials, &c->ssim_sums,
                    &c->init_pts, &c->init_scales, &c->knn_part, &c->knn_table, &c->ord_keys0, &c->ord_keys1,
                    &c->ord_vals0, &c->ord_vals1, &c->ord_total, &c->ord_hist, &c->ord_hist_scan, &c->ord_lookback,
                    &c->ord_counters, &c->ord_views, &c->tile_order, &c->vis_sums, &c->vis_offsets, &c->dtotal,
                    &c->dkeys0, &c->dkeys1, &c->dvals0, &c->dvals1, &c->dhist, &c->dhist_scan, &c->dlookback,
                    &c->elookback, &c->dorder, &c->torder};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  for (const auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->status_d) cudaFree(c->status_d);
  if (c->status_h) cudaFreeHost(c->status_h);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->staging) cudaFreeHost(c->staging);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
  if (c->staged_ev) cudaEventDestroy(c->staged_ev);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (int i = 0; i < 2; i++) {
    if (c->tgt_copied[i]) cudaEventDestroy(c->tgt_copied[i]);
    if (c->tgt_free[i]) cudaEventDestroy(c->tgt_free[i]);
  }
  delete c;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->err.c_str() : "null context"; }

gs_status gs_set_stream(gs_ctx* c, void* stream) {
  if (!c) return GS_EINVAL;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return GS_OK;
}

gs_status gs_sync(gs_ctx* c) {
  if (!c) return GS_EINVAL;
  set_device(c);
  GS_CUDA(c, cudaMemcpyAsync(c->status_h, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  const int st = *c->status_h;
  if (st & kStatusTimeout) return fail(c, GS_ETIMEOUT, "a bounded device-side wait ran out");
  if (st & kStatusCapacity) return fail(c, GS_ECAPACITY, "instance capacity exceeded");
  return GS_OK;
}

gs_status gs_project(gs_ctx* c, const gs_params* params, const gs_camera* cams, int32_t B) {
  if (!c) return GS_EINVAL;
  GS_TRY(check_params(c, params, "params"));
  if (!cams) return fail(c, GS_EINVAL, "cams is NULL");
  if (B < 1 || B > c->cfg.max_views) return fail(c, GS_EINVAL, "B must be in 1..%d", c->cfg.max_views);
  set_device(c);
  c->projected = c->sorted = c->rastered = c->cells_ready = false;
  int64_t tile_off = 0, pix_off = 0;
  GS_TRY(build_views(c, cams, B, &tile_off, &pix_off));
  if (tile_off >= ((int64_t)1 << 31)) return fail(c, GS_EINVAL, "too many tiles in the batch");
  const int64_t n = params->n, stride = params->stride;
  const int64_t nb = (n + project_fwd_block() - 1) / project_fwd_block();
  GS_TRY(ensure(c, c->views, sizeof(ViewRec) * B));
  GS_TRY(ensure(c, c->rec, sizeof(float4) * kRecStride * B * stride));
  GS_TRY(ensure(c, c->rec3, sizeof(int4) * B * stride));
  GS_TRY(ensure(c, c->tiles, sizeof(uint2) * B * stride));
  GS_TRY(ensure(c, c->block_sums, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure(c, c->vis_sums, sizeof(uint32_t) * B * nb));
  GS_TRY(ensure(c, c->vismask, sizeof(uint64_t) * stride));
  GS_CUDA(c, cudaMemsetAsync(c->vismask.p, 0, sizeof(uint64_t) * stride, c->stream));
  if (c->capturing) {
    // a captured step copies the cameras from the pinned staging area at its start
  } else {
    GS_CUDA(c, cudaMemcpyAsync(c->views.p, c->views_h.data(), sizeof(ViewRec) * B, cudaMemcpyHostToDevice,
                               c->stream));
  }
  ProjectArgs a{};
  a.params = params->data;
  a.n = n;
  a.stride = stride;
  a.views = P<ViewRec>(c->views);
  a.B = B;
  a.rec0 = P<float4>(c->rec);
  a.rec1 = P<float4>(c->rec) + 1;
  a.rec2 = P<float4>(c->rec) + 2;
  a.rec3 = P<int4>(c->rec3);
  a.tiles = P<uint2>(c->tiles);
  a.block_sums = P<uint32_t>(c->block_sums);
  a.vis_sums = P<uint32_t>(c->vis_sums);
  a.vismask = P<uint64_t>(c->vismask);
  {
    LaunchScope ls(c, "project_fwd");
    launch_project_fwd(a, params->sh_degree, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->B = B;
  c->n = n;
  c->stride = stride;
  c->deg = params->sh_degree;
  c->bins = tile_off;
  c->pixels = pix_off;
  c->nblocks = nb;
  c->projected = true;
  return GS_OK;
}

static gs_status sort_tiles_longest_first(gs_ctx* c);

gs_status gs_bin_sort(gs_ctx* c) {
  if (!c) return GS_EINVAL;
  if (!c->projected) return fail(c, GS_ESTATE, "gs_bin_sort needs gs_project first");
  set_device(c);
  c->sorted = c->rastered = c->cells_ready = false;
  const int B = c->B;
  GS_TRY(ensure(c, c->block_offsets, sizeof(uint32_t) * B * c->nblocks));
  GS_TRY(ensure(c, c->vis_offsets, sizeof(uint32_t) * B * c->nblocks));
  GS_TRY(ensure(c, c->total, sort_words_bytes()));
  GS_TRY(ensure(c, c->dtotal, sort_words_bytes()));
  const SortWords iw = sort_words(c->total);   // instances (tile sort)
  const SortWords dw = sort_words(c->dtotal);  // visible pairs (depth sort)
  {
    LaunchScope ls(c, "scan_block_sums", 4);
    launch_scan_block_sums(P<uint32_t>(c->block_sums), c->nblocks, B, P<uint32_t>(c->block_offsets),
                           iw.view_total, iw.seg, iw.total, c->stream);
    launch_scan_block_sums(P<uint32_t>(c->vis_sums), c->nblocks, B, P<uint32_t>(c->vis_offsets), dw.view_total,
                           dw.seg, dw.total, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  // capacity: the exact count (grow-on-demand contexts read it, one stream
  // synchronisation) or the context's fixed capacity (no host read, so the
  // sequence can be captured in a CUDA graph; overflow -> GS_ECAPACITY)
  int64_t cap;
  if (c->cfg.instance_capacity > 0) {
    cap = c->batch_cap > 0 ? std::min(c->batch_cap, c->cfg.instance_capacity) : c->cfg.instance_capacity;
    c->instances = -1;
  } else {
    GS_CUDA(c, cudaMemcpyAsync(c->pinned, c->total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    cap = (int64_t)c->pinned[0];
    c->instances = cap;
  }
  if (cap >= ((int64_t)1 << 30) - 1) return fail(c, GS_ECAPACITY, "%lld instances exceed 2^30", (long long)cap);
  const int64_t pc = (int64_t)B * c->n;  // visible pairs at most
  if (pc >= ((int64_t)1 << 32) - 1) return fail(c, GS_ECAPACITY, "%lld (view, Gaussian) pairs exceed 2^32", (long long)pc);
  GS_TRY(ensure(c, c->keys0, sizeof(uint32_t) * cap));
  GS_TRY(ensure(c, c->keys1, sizeof(uint32_t) * cap));
  GS_TRY(ensure(c, c->vals0, sizeof(uint32_t) * cap));
  GS_TRY(ensure(c, c->vals1, sizeof(uint32_t) * cap));
  GS_TRY(ensure(c, c->dkeys0, sizeof(uint32_t) * pc));
  GS_TRY(ensure(c, c->dkeys1, sizeof(uint32_t) * pc));
  GS_TRY(ensure(c, c->dvals0, sizeof(uint32_t) * pc));
  GS_TRY(ensure(c, c->dvals1, sizeof(uint32_t) * pc));
  GS_TRY(ensure(c, c->ranges, sizeof(uint2) * c->bins));
  // each view is sorted on its own: the tile sort on the bits of the
  // largest tile index inside a view
  int64_t most_tiles = 1;
  for (int v = 0; v < B; v++) most_tiles = std::max<int64_t>(most_tiles, (int64_t)c->views_h[v].gw * c->views_h[v].gh);
  const int tpass = tile_passes(most_tiles);
  c->sort_passes = tpass;
  const size_t lb = sort_lookback_bytes(cap, c->sort_items, B);
  const size_t dlb = sort_lookback_bytes(pc, c->sort_items, B);
  const size_t elb = emit_lookback_bytes(pc, B);
  GS_TRY(ensure(c, c->hist, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure(c, c->hist_scan, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure(c, c->dhist, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure(c, c->dhist_scan, sizeof(uint32_t) * (size_t)B * 8 * 256));
  GS_TRY(ensure(c, c->lookback, lb * tpass));
  GS_TRY(ensure(c, c->dlookback, dlb * kDepthPasses));
  GS_TRY(ensure(c, c->elookback, elb));
  GS_TRY(ensure(c, c->torder, sizeof(uint32_t) * sort_partitions(cap, c->sort_items, B)));
  GS_TRY(ensure(c, c->dorder, sizeof(uint32_t) * sort_partitions(pc, c->sort_items, B)));
  GS_TRY(ensure(c, c->counters, sizeof(uint32_t) * kSortCounters));
  GS_TRY(ensure(c, c->sorted_slots, 2 * sizeof(void*)));
  // contribution masks: every tile's region padded to whole batches of 32
  if (!c->forward_only) GS_TRY(ensure(c, c->cells, sizeof(uint32_t) * (cap + 32 * c->bins)));
  uint32_t* counters = P<uint32_t>(c->counters);
  GS_CUDA(c, cudaMemsetAsync(c->counters.p, 0, sizeof(uint32_t) * kSortCounters, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->dhist.p, 0, sizeof(uint32_t) * (size_t)B * kDepthPasses * 256, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->hist.p, 0, sizeof(uint32_t) * (size_t)B * tpass * 256, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->dlookback.p, 0, dlb * kDepthPasses, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->elookback.p, 0, elb, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->lookback.p, 0, lb * tpass, c->stream));

  // 1. visible pairs -> (depth bits, Gaussian), view by view in Gaussian order
  CompactArgs ca{};
  ca.n = c->n;
  ca.stride = c->stride;
  ca.B = B;
  ca.tiles = P<uint2>(c->tiles);
  ca.vis_offsets = P<uint32_t>(c->vis_offsets);
  ca.vseg = dw.seg;
  ca.dkeys = P<uint32_t>(c->dkeys0);
  ca.dvals = P<uint32_t>(c->dvals0);
  {
    LaunchScope ls(c, "compact");
    launch_compact(ca, c->stream);
  }
  GS_CHECK_LAUNCH(c);

  // 2. stable sort of each view's pairs by depth
  SortArgs ds{};
  ds.keys[0] = c->dkeys0.p;
  ds.keys[1] = c->dkeys1.p;
  ds.vals[0] = P<uint32_t>(c->dvals0);
  ds.vals[1] = P<uint32_t>(c->dvals1);
  ds.key_bytes = 4;
  ds.view_shift = 0;
  ds.views = nullptr;
  ds.count = dw.total;
  ds.capacity = pc;
  ds.bins = 0;
  ds.B = B;
  ds.seg = dw.seg;
  ds.part_off = dw.part_off;
  ds.part_order = P<uint32_t>(c->dorder);
  ds.hist = P<uint32_t>(c->dhist);
  ds.hist_scan = P<uint32_t>(c->dhist_scan);
  ds.ctrl = dw.ctrl;
  ds.single = dw.single;
  ds.lookback = P<uint32_t>(c->dlookback);
  ds.lookback_stride = dlb / sizeof(uint32_t);
  ds.counters = counters + 8;
  ds.npass = kDepthPasses;
  ds.wait_rounds = c->sort_wait;
  ds.status = c->status_d;
  {
    LaunchScope ls(c, "depth_histogram", 4);
    launch_digit_histogram(ds, pc, c->sort_items, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  for (int p = 0; p < kDepthPasses; p++) {
    LaunchScope ls(c, "depth_pass");
    launch_onesweep_pass(ds, p, c->sort_items, c->stream);
  }
  GS_CHECK_LAUNCH(c);

  // 3. one instance per touched tile, in depth order; tile digit counts
  EmitArgs ea{};
  ea.B = B;
  ea.n = c->n;
  ea.stride = c->stride;
  ea.views = P<ViewRec>(c->views);
  ea.rec3 = P<int4>(c->rec3);
  ea.dvals[0] = P<uint32_t>(c->dvals0);
  ea.dvals[1] = P<uint32_t>(c->dvals1);
  ea.dctrl = dw.ctrl;
  ea.dpass = kDepthPasses;
  ea.vseg = dw.seg;
  ea.seg = iw.seg;
  ea.keys = P<uint32_t>(c->keys0);
  ea.vals = P<uint32_t>(c->vals0);
  ea.capacity = cap;
  ea.lookback = P<uint64_t>(c->elookback);
  ea.counter = counters + 16;
  ea.hist = P<uint32_t>(c->hist);
  ea.tpass = tpass;
  ea.wait_rounds = c->sort_wait;
  ea.status = c->status_d;
  {
    LaunchScope ls(c, "emit");
    launch_emit(ea, pc, c->stream);
  }
  GS_CHECK_LAUNCH(c);

  // 4. stable sort of each view's instances by tile
  SortArgs sa{};
  sa.keys[0] = c->keys0.p;
  sa.keys[1] = c->keys1.p;
  sa.vals[0] = P<uint32_t>(c->vals0);
  sa.vals[1] = P<uint32_t>(c->vals1);
  sa.key_bytes = 4;
  sa.view_shift = 0;
  sa.views = P<ViewRec>(c->views);
  sa.count = iw.total;
  sa.capacity = cap;
  sa.bins = c->bins;
  sa.B = B;
  sa.seg = iw.seg;
  sa.part_off = iw.part_off;
  sa.part_order = P<uint32_t>(c->torder);
  sa.hist = P<uint32_t>(c->hist);
  sa.hist_scan = P<uint32_t>(c->hist_scan);
  sa.ctrl = iw.ctrl;
  sa.single = iw.single;
  sa.lookback = P<uint32_t>(c->lookback);
  sa.lookback_stride = lb / sizeof(uint32_t);
  sa.counters = counters;
  sa.npass = tpass;
  sa.wait_rounds = c->sort_wait;
  sa.status = c->status_d;
  sa.sorted_keys = reinterpret_cast<const void**>(c->sorted_slots.p);
  sa.sorted_vals = reinterpret_cast<const uint32_t**>(P<unsigned char>(c->sorted_slots) + sizeof(void*));
  {
    LaunchScope ls(c, "tile_scan", 3);
    launch_digit_scan(sa, c->sort_items, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  for (int p = 0; p < tpass; p++) {
    LaunchScope ls(c, "tile_pass");
    launch_onesweep_pass(sa, p, c->sort_items, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  // 5. per-tile ranges
  GS_CUDA(c, cudaMemsetAsync(c->ranges.p, 0, sizeof(uint2) * c->bins, c->stream));
  {
    LaunchScope ls(c, "tile_ranges");
    launch_tile_ranges(sa, cap, P<uint2>(c->ranges), c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->tile_order_ready = false;
  if (c->tile_order_mode == 1) GS_TRY(sort_tiles_longest_first(c));
  c->sorted = true;
  return GS_OK;
}

// Longest-list-first order of the batch's tiles (bins bucketed by
// floor(log2(length + 1)), a one-pass stable sort, bin order inside a
// bucket) into c->tile_order; every step on the device, so a captured step
// replays it.
static gs_status sort_tiles_longest_first(gs_ctx* c) {
  const int64_t bins = c->bins;
  const int items = 16;
  const size_t lb = sort_lookback_bytes(bins, items, 1);
  GS_TRY(ensure(c, c->ord_keys0, sizeof(uint64_t) * bins));
  GS_TRY(ensure(c, c->ord_keys1, sizeof(uint64_t) * bins));
  GS_TRY(ensure(c, c->ord_vals0, sizeof(uint32_t) * bins));
  GS_TRY(ensure(c, c->ord_vals1, sizeof(uint32_t) * bins));
  GS_TRY(ensure(c, c->ord_total, sizeof(uint64_t) + sizeof(uint32_t) * (2 + 2 + 16 + 8)));
  GS_TRY(ensure(c, c->ord_hist, sizeof(uint32_t) * 256));
  GS_TRY(ensure(c, c->ord_hist_scan, sizeof(uint32_t) * 256));
  GS_TRY(ensure(c, c->ord_lookback, lb));
  GS_TRY(ensure(c, c->ord_counters, sizeof(uint32_t) * 8));
  GS_TRY(ensure(c, c->ord_views, sizeof(ViewRec)));
  GS_TRY(ensure(c, c->tile_order, sizeof(uint32_t) * bins));
  uint64_t* count = P<uint64_t>(c->ord_total);
  uint32_t* seg = reinterpret_cast<uint32_t*>(count + 1);
  uint32_t* part_off = seg + 2;
  uint32_t* ctrl = part_off + 2;
  SortArgs sa{};
  sa.keys[0] = c->ord_keys0.p;
  sa.keys[1] = c->ord_keys1.p;
  sa.key_bytes = 8;
  sa.view_shift = 32;
  sa.vals[0] = P<uint32_t>(c->ord_vals0);
  sa.vals[1] = P<uint32_t>(c->ord_vals1);
  sa.count = count;
  sa.capacity = bins;
  sa.bins = bins;
  sa.B = 1;
  sa.views = P<ViewRec>(c->ord_views);
  sa.seg = seg;
  sa.part_off = part_off;
  sa.hist = P<uint32_t>(c->ord_hist);
  sa.hist_scan = P<uint32_t>(c->ord_hist_scan);
  sa.ctrl = ctrl;
  sa.single = ctrl + 16;
  sa.lookback = P<uint32_t>(c->ord_lookback);
  sa.lookback_stride = lb / sizeof(uint32_t);
  sa.counters = P<uint32_t>(c->ord_counters);
  sa.npass = 1;
  sa.wait_rounds = c->sort_wait;
  sa.status = c->status_d;
  GS_CUDA(c, cudaMemsetAsync(c->ord_views.p, 0, sizeof(ViewRec), c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->ord_hist.p, 0, sizeof(uint32_t) * 256, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->ord_counters.p, 0, sizeof(uint32_t) * 8, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->ord_lookback.p, 0, lb, c->stream));
  {
    LaunchScope ls(c, "tile_order", 6);
    launch_tile_order_keys(P<uint2>(c->ranges), bins, P<uint64_t>(c->ord_keys0), sa.vals[0], count, seg, c->stream);
    launch_digit_histogram(sa, bins, items, c->stream);
    launch_onesweep_pass(sa, 0, items, c->stream);
    launch_tile_order_finish(ctrl, 1, sa.vals[0], sa.vals[1], bins, P<uint32_t>(c->tile_order), c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->tile_order_ready = true;
  return GS_OK;
}

static RasterArgs raster_args(gs_ctx* c) {
  RasterArgs r{};
  r.views = P<ViewRec>(c->views);
  r.B = c->B;
  r.n = c->n;
  r.stride = c->stride;
  r.ranges = P<uint2>(c->ranges);
  r.vals = reinterpret_cast<const uint32_t* const*>(P<unsigned char>(c->sorted_slots) + sizeof(void*));
  r.rec0 = P<float4>(c->rec);
  r.rec1 = P<float4>(c->rec) + 1;
  r.rec2 = P<float4>(c->rec) + 2;
  r.tfinal = P<float>(c->tfinal);
  r.nlast = P<uint32_t>(c->nlast);
  r.cells = c->forward_only ? nullptr : P<uint32_t>(c->cells);
  r.tile_order = c->tile_order_ready ? P<uint32_t>(c->tile_order) : nullptr;
  return r;
}

gs_status gs_raster_fwd(gs_ctx* c, float* images) {
  if (!c) return GS_EINVAL;
  if (!c->sorted) return fail(c, GS_ESTATE, "gs_raster_fwd needs gs_bin_sort first");
  if (!images) return fail(c, GS_EINVAL, "images is NULL");
  set_device(c);
  GS_TRY(ensure(c, c->tfinal, sizeof(float) * c->pixels));
  GS_TRY(ensure(c, c->nlast, sizeof(uint32_t) * c->pixels));
  RasterArgs r = raster_args(c);
  r.image = images;
  {
    LaunchScope ls(c, "raster_fwd");
    launch_raster_fwd(r, c->bins, c->raster_fwd, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->rastered = true;
  c->cells_ready = !c->forward_only;
  return GS_OK;
}

gs_status gs_raster_fwd_l1(gs_ctx* c, float* images, const float* targets, float* loss, float* dL_dimages) {
  if (!c) return GS_EINVAL;
  if (!c->sorted) return fail(c, GS_ESTATE, "gs_raster_fwd_l1 needs gs_bin_sort first");
  if (!targets || !loss || !dL_dimages) return fail(c, GS_EINVAL, "targets, loss and dL_dimages must not be NULL");
  set_device(c);
  GS_TRY(ensure(c, c->tfinal, sizeof(float) * c->pixels));
  GS_TRY(ensure(c, c->nlast, sizeof(uint32_t) * c->pixels));
  const int64_t nparts = raster_fwd_warps(c->bins, c->raster_fwd);
  // per-warp partial sums, then the 256 block sums of the finishing reduction
  const size_t part_bytes = (sizeof(float) * std::max<int64_t>(nparts, 1) + 255) / 256 * 256;
  GS_TRY(ensure(c, c->l1_partial, part_bytes + l1_finish_scratch_bytes()));
  const int64_t count = 3 * c->pixels;
  RasterArgs r = raster_args(c);
  r.image = images;
  r.target = targets;
  // inside a captured step the targets are read through the device slot
  r.target_slot = c->capturing ? reinterpret_cast<const float* const*>(c->target_slot.p) : nullptr;
  r.l1_grad = dL_dimages;
  r.l1_partial = P<float>(c->l1_partial);
  r.inv_count = (float)(1.0 / (double)count);
  {
    LaunchScope ls(c, "raster_fwd");
    launch_raster_fwd(r, c->bins, c->raster_fwd, c->stream);
  }
  {
    LaunchScope ls(c, "l1_loss", 2);
    launch_l1_finish(P<float>(c->l1_partial), nparts,
                     reinterpret_cast<double*>(P<unsigned char>(c->l1_partial) + part_bytes), 1.0 / (double)count,
                     loss, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->rastered = true;
  c->cells_ready = !c->forward_only;
  return GS_OK;
}

gs_status gs_raster_bwd(gs_ctx* c, const gs_params* params, const float* dL_dimages, gs_params* grads) {
  if (!c) return GS_EINVAL;
  if (!c->rastered) return fail(c, GS_ESTATE, "gs_raster_bwd needs gs_raster_fwd first");
  if (!c->cells_ready) return fail(c, GS_ESTATE, "the last forward pass of this context is forward-only");
  GS_TRY(check_params(c, params, "params"));
  GS_TRY(check_params(c, grads, "grads"));
  if (!dL_dimages) return fail(c, GS_EINVAL, "dL_dimages is NULL");
  if (params->n != c->n || params->stride != c->stride || params->sh_degree != c->deg)
    return fail(c, GS_EINVAL, "params differ from the projected set");
  if (grads->n != c->n || grads->stride != c->stride || grads->sh_degree != c->deg)
    return fail(c, GS_EINVAL, "grads must match params in n, stride and sh_degree");
  set_device(c);
  const size_t g2d_bytes = sizeof(float) * (kG2dGeo + kG2dCol) * c->B * c->stride;
  GS_TRY(ensure(c, c->g2d, g2d_bytes));
  if (!c->g2d_cleared) GS_CUDA(c, cudaMemsetAsync(c->g2d.p, 0, g2d_bytes, c->stream));
  c->g2d_cleared = false;
  RasterArgs r = raster_args(c);
  r.dimage = dL_dimages;
  r.g2d = P<float>(c->g2d);
  r.direct_max = c->bwd_direct;
  {
    LaunchScope ls(c, "raster_bwd");
    launch_raster_bwd(r, c->bins, c->raster_bwd, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  ProjectBwdArgs b{};
  b.params = params->data;
  b.n = c->n;
  b.stride = c->stride;
  b.views = P<ViewRec>(c->views);
  b.B = c->B;
  b.g2d = P<float>(c->g2d);
  b.grads = grads->data;
  b.vismask = P<uint64_t>(c->vismask);
  b.dens_grad = c->dens_grad;
  b.dens_count = c->dens_count;
  if (grads->stride > grads->n) {
    // padding columns are not written by the kernel; keep them zero
    GS_CUDA(c, cudaMemsetAsync(grads->data, 0, sizeof(float) * n_planes(c->deg) * grads->stride, c->stream));
  }
  {
    LaunchScope ls(c, "project_bwd", 2);
    launch_project_bwd(b, c->deg, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

gs_status gs_l1_loss(gs_ctx* c, const float* x, const float* y, int64_t count, float* loss, float* dL_dx) {
  if (!c) return GS_EINVAL;
  if (!x || !y) return fail(c, GS_EINVAL, "x and y must not be NULL");
  if (count <= 0) return fail(c, GS_EINVAL, "count must be > 0");
  set_device(c);
  const int parts = l1_parts(count);
  GS_TRY(ensure(c, c->l1_partial, sizeof(float) * parts));
  {
    LaunchScope ls(c, "l1_loss", loss ? 2 : 1);
    // inside a captured step the targets are read through the device slot
    const float* const* slot = c->capturing ? reinterpret_cast<const float* const*>(c->target_slot.p) : nullptr;
    launch_l1(x, y, slot, count, P<float>(c->l1_partial), parts, loss, dL_dx, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

gs_status gs_adam(gs_ctx* c, gs_params* p, const gs_params* g, gs_params* m, gs_params* v,
                  const gs_adam_hp* hp, int64_t step) {
  if (!c) return GS_EINVAL;
  GS_TRY(check_params(c, p, "p"));
  GS_TRY(check_params(c, g, "g"));
  GS_TRY(check_params(c, m, "m"));
  GS_TRY(check_params(c, v, "v"));
  if (!hp) return fail(c, GS_EINVAL, "hp is NULL");
  if (step < 1) return fail(c, GS_EINVAL, "step must be >= 1");
  const gs_params* all[3] = {g, m, v};
  for (const gs_params* q : all)
    if (q->n != p->n || q->stride != p->stride || q->sh_degree != p->sh_degree)
      return fail(c, GS_EINVAL, "p, g, m, v must share n, stride and sh_degree");
  set_device(c);
  AdamArgs a{};
  a.p = p->data;
  a.g = g->data;
  a.m = m->data;
  a.v = v->data;
  a.stride = p->stride;
  a.planes = n_planes(p->sh_degree);
  float consts[65];
  adam_constants(hp, a.planes, step, c->B, consts);
  GS_TRY(ensure(c, c->adam_consts, sizeof(consts)));
  if (c->capturing) {
    // a captured step copies the constants from the pinned staging area at its start
  } else {
    GS_CUDA(c, cudaMemcpyAsync(c->adam_consts.p, consts, sizeof(consts), cudaMemcpyHostToDevice, c->stream));
  }
  a.consts = P<float>(c->adam_consts);
  a.beta1 = hp->beta1;
  a.beta2 = hp->beta2;
  a.eps = hp->eps;
  if (hp->flags & GS_ADAM_VISIBLE_ONLY) {
    // the visibility of the context's last projected batch
    if (!c->vismask.p || c->n != p->n || c->stride != p->stride)
      return fail(c, GS_ESTATE, "visible-only Adam needs gs_project of the same set first");
    a.vismask = P<uint64_t>(c->vismask);
  }
  {
    LaunchScope ls(c, "adam");
    launch_adam(a, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

gs_status gs_get_buffer(gs_ctx* c, int32_t which, void** ptr, int64_t* count) {
  if (!c || !ptr || !count) return GS_EINVAL;
  const int64_t bn = (int64_t)c->B * c->stride;
  switch (which) {
    case GS_BUF_REC0:
    case GS_BUF_REC1:
    case GS_BUF_REC2:
      if (!c->projected) return GS_ESTATE;
      *ptr = P<float4>(c->rec) + (which - GS_BUF_REC0);  // stride kRecStride float4
      *count = bn;
      break;
    case GS_BUF_REC3: if (!c->projected) return GS_ESTATE; *ptr = c->rec3.p; *count = bn; break;
    case GS_BUF_KEYS:
    case GS_BUF_VALS: {
      if (!c->sorted) return GS_ESTATE;
      void* slots[2] = {nullptr, nullptr};
      uint64_t cnt = 0;
      GS_CUDA(c, cudaMemcpyAsync(slots, c->sorted_slots.p, sizeof(slots), cudaMemcpyDeviceToHost, c->stream));
      GS_CUDA(c, cudaMemcpyAsync(&cnt, c->total.p, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
      GS_CUDA(c, cudaStreamSynchronize(c->stream));
      *ptr = slots[which == GS_BUF_KEYS ? 0 : 1];
      *count = (int64_t)cnt;
      break;
    }
    case GS_BUF_RANGES: if (!c->sorted) return GS_ESTATE; *ptr = c->ranges.p; *count = c->bins; break;
    case GS_BUF_TFINAL: if (!c->rastered) return GS_ESTATE; *ptr = c->tfinal.p; *count = c->pixels; break;
    case GS_BUF_NLAST: if (!c->rastered) return GS_ESTATE; *ptr = c->nlast.p; *count = c->pixels; break;
    case GS_BUF_G2D: if (!c->g2d.p) return GS_ESTATE; *ptr = c->g2d.p; *count = (kG2dGeo + kG2dCol) * bn; break;
    case GS_BUF_VISMASK: if (!c->projected) return GS_ESTATE; *ptr = c->vismask.p; *count = c->n; break;
    case GS_BUF_SORT_CTRL:
      if (!c->sorted) return GS_ESTATE;
      *ptr = sort_words(c->total).ctrl;
      *count = c->sort_passes + 1;
      break;
    case GS_BUF_DEPTH_CTRL:
      if (!c->sorted) return GS_ESTATE;
      *ptr = sort_words(c->dtotal).ctrl;
      *count = kDepthPasses + 1;
      break;
    default: return fail(c, GS_EINVAL, "unknown buffer %d", which);
  }
  return GS_OK;
}

gs_status gs_get_counts(gs_ctx* c, int64_t* instances, int64_t* bins, int64_t* pixels) {
  if (!c) return GS_EINVAL;
  if (!c->projected) return fail(c, GS_ESTATE, "no batch projected");
  set_device(c);
  uint64_t cnt = 0;
  if (c->sorted) GS_CUDA(c, cudaMemcpyAsync(&cnt, c->total.p, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  if (instances) *instances = c->sorted ? (int64_t)cnt : -1;
  if (bins) *bins = c->bins;
  if (pixels) *pixels = c->pixels;
  return GS_OK;
}

// SSIM forward (and backward) over the last projected batch's views.
static gs_status run_ssim(gs_ctx* c, const float* images, const float* targets, float lambda, float* loss,
                          float* dL_dimages) {
  if (!c->projected) return fail(c, GS_ESTATE, "SSIM needs a projected batch (view sizes)");
  if (!images || !targets) return fail(c, GS_EINVAL, "images and targets must not be NULL");
  if (!(lambda >= 0.f && lambda <= 1.f)) return fail(c, GS_EINVAL, "lambda must be in [0, 1]");
  set_device(c);
  const int B = c->B;
  std::vector<int> first(B + 1, 0);
  for (int v = 0; v < B; v++) first[v + 1] = first[v] + ssim_blocks_of_view(c->views_h[v].W, c->views_h[v].H);
  const int blocks = first[B];
  const int64_t count = 3 * c->pixels;
  GS_TRY(ensure(c, c->ssim_table, sizeof(int) * (B + 1)));
  GS_TRY(ensure(c, c->ssim_partials, sizeof(float) * 3 * count));
  GS_TRY(ensure(c, c->ssim_sums, sizeof(double) * (3 * (size_t)blocks + 3 * kMaxViews)));
  GS_CUDA(c, cudaMemcpyAsync(c->ssim_table.p, first.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, c->stream));
  SsimArgs a{};
  a.views = P<ViewRec>(c->views);
  a.B = B;
  a.first_block = P<int>(c->ssim_table);
  a.x = images;
  a.y = targets;
  a.count = count;
  a.partials = P<float>(c->ssim_partials);
  a.block_sums = P<double>(c->ssim_sums);
  a.grad = dL_dimages;
  ssim_window(a.win);
  a.w_l1 = 1.f - lambda;
  a.w_ssim = lambda;
  a.inv_count = (float)(1.0 / (double)count);
  a.w_l1_d = 1.0 - (double)lambda;
  a.w_ssim_d = (double)lambda;
  {
    LaunchScope ls(c, "ssim", 2 + (loss ? 1 : 0) + (dL_dimages ? 1 : 0));
    launch_ssim(a, blocks, dL_dimages != nullptr, P<double>(c->ssim_sums) + 3 * (size_t)blocks, loss, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

gs_status gs_ssim_loss(gs_ctx* c, const float* images, const float* targets, float lambda, float* loss,
                       float* dL_dimages) {
  if (!c) return GS_EINVAL;
  if (!loss && !dL_dimages) return fail(c, GS_EINVAL, "loss and dL_dimages are both NULL");
  return run_ssim(c, images, targets, lambda, loss, dL_dimages);
}

gs_status gs_image_metrics(gs_ctx* c, const float* images, const float* targets, double* ssim, double* psnr) {
  if (!c) return GS_EINVAL;
  if (!ssim && !psnr) return fail(c, GS_EINVAL, "ssim and psnr are both NULL");
  GS_TRY(run_ssim(c, images, targets, 0.f, nullptr, nullptr));
  std::vector<double> sums(3 * (size_t)c->B);
  int blocks = 0;
  for (int v = 0; v < c->B; v++) blocks += ssim_blocks_of_view(c->views_h[v].W, c->views_h[v].H);
  GS_CUDA(c, cudaMemcpyAsync(sums.data(), P<double>(c->ssim_sums) + 3 * (size_t)blocks,
                             sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int v = 0; v < c->B; v++) {
    const double cnt = 3.0 * c->views_h[v].W * c->views_h[v].H;
    if (ssim) ssim[v] = sums[3 * v] / cnt;
    if (psnr) psnr[v] = 10.0 * std::log10(cnt / sums[3 * v + 2]);
  }
  return GS_OK;
}

// ---------------------------------------------------------------- initialisation

// Stable LSD sort of n (key, value) pairs on the low `bits` key bits with the
// binning's onesweep (one segment), in the context's instance buffers;
// *which = the buffer (0 / 1) holding the result.  Synchronises the stream.
static gs_status sort_pairs(gs_ctx* c, int64_t n, int bits, int* which) {
  const int npass = std::max(1, (bits + 7) / 8);
  GS_TRY(ensure(c, c->views, sizeof(ViewRec)));
  GS_TRY(ensure(c, c->total, sort_words_bytes()));
  const size_t lb = sort_lookback_bytes(n, c->sort_items, 1);
  GS_TRY(ensure(c, c->hist, sizeof(uint32_t) * 8 * 256));
  GS_TRY(ensure(c, c->hist_scan, sizeof(uint32_t) * 8 * 256));
  GS_TRY(ensure(c, c->lookback, lb * npass));
  GS_TRY(ensure(c, c->counters, sizeof(uint32_t) * 8));
  uint64_t* total = P<uint64_t>(c->total);
  uint32_t* seg = reinterpret_cast<uint32_t*>(total + 1 + kMaxViews);
  uint32_t* part_off = seg + kMaxViews + 1;
  uint32_t* ctrl = part_off + kMaxViews + 1;
  const uint64_t cnt = (uint64_t)n;
  const uint32_t segs[2] = {0u, (uint32_t)n};
  GS_CUDA(c, cudaMemsetAsync(c->views.p, 0, sizeof(ViewRec), c->stream));
  GS_CUDA(c, cudaMemcpyAsync(total, &cnt, sizeof(cnt), cudaMemcpyHostToDevice, c->stream));
  GS_CUDA(c, cudaMemcpyAsync(seg, segs, sizeof(segs), cudaMemcpyHostToDevice, c->stream));
  SortArgs sa{};
  sa.keys[0] = c->keys0.p;
  sa.keys[1] = c->keys1.p;
  sa.key_bytes = 8;
  sa.view_shift = 32;
  sa.vals[0] = P<uint32_t>(c->vals0);
  sa.vals[1] = P<uint32_t>(c->vals1);
  sa.count = total;
  sa.capacity = n;
  sa.bins = 1;
  sa.B = 1;
  sa.views = P<ViewRec>(c->views);
  sa.seg = seg;
  sa.part_off = part_off;
  sa.hist = P<uint32_t>(c->hist);
  sa.hist_scan = P<uint32_t>(c->hist_scan);
  sa.ctrl = ctrl;
  sa.single = ctrl + 16;
  sa.lookback = P<uint32_t>(c->lookback);
  sa.lookback_stride = lb / sizeof(uint32_t);
  sa.counters = P<uint32_t>(c->counters);
  sa.npass = npass;
  sa.wait_rounds = c->sort_wait;
  sa.status = c->status_d;
  GS_CUDA(c, cudaMemsetAsync(c->hist.p, 0, sizeof(uint32_t) * npass * 256, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->counters.p, 0, sizeof(uint32_t) * 8, c->stream));
  GS_CUDA(c, cudaMemsetAsync(c->lookback.p, 0, lb * npass, c->stream));
  {
    LaunchScope ls(c, "digit_histogram", 3);
    launch_digit_histogram(sa, n, c->sort_items, c->stream);
  }
  for (int p = 0; p < npass; p++) {
    LaunchScope ls(c, "onesweep_pass");
    launch_onesweep_pass(sa, p, c->sort_items, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  uint32_t par = 0;
  GS_CUDA(c, cudaMemcpyAsync(&par, ctrl + npass, sizeof(par), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  *which = (int)(par & 1u);
  return GS_OK;
}

gs_status gs_iso_crossings(gs_ctx* c, const float* volume, int32_t nx, int32_t ny, int32_t nz, float iso,
                           const float* origin, const float* spacing, float* points, float* normals, int64_t capacity,
                           int64_t* count) {
  if (!c) return GS_EINVAL;
  if (!volume || !origin || !spacing || !count) return fail(c, GS_EINVAL, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1) return fail(c, GS_EINVAL, "volume dimensions must be >= 1");
  if ((points == nullptr) != (normals == nullptr)) return fail(c, GS_EINVAL, "points and normals go together");
  set_device(c);
  c->projected = c->sorted = c->rastered = c->cells_ready = false;
  IsoArgs a{};
  a.vol = volume;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nverts = (int64_t)nx * ny * nz;
  a.iso = iso;
  for (int d = 0; d < 3; d++) {
    a.origin[d] = origin[d];
    a.h[d] = spacing[d];
  }
  const int64_t nb = (a.nverts + 255) / 256;
  GS_TRY(ensure(c, c->block_sums, sizeof(uint32_t) * nb));
  GS_TRY(ensure(c, c->block_offsets, sizeof(uint32_t) * nb));
  GS_TRY(ensure(c, c->total, sizeof(uint64_t) * (1 + kMaxViews) +
                                 sizeof(uint32_t) * (2 * (kMaxViews + 1) + 16 + 8 * kMaxViews)));
  a.block_counts = P<uint32_t>(c->block_sums);
  a.block_offsets = P<uint32_t>(c->block_offsets);
  a.status = c->status_d;
  uint64_t* total = P<uint64_t>(c->total);
  {
    LaunchScope ls(c, "iso_crossings");
    launch_iso(a, false, c->stream);
  }
  {
    LaunchScope ls(c, "scan_block_sums", 2);
    launch_scan_block_sums(P<uint32_t>(c->block_sums), nb, 1, P<uint32_t>(c->block_offsets), total + 1,
                           reinterpret_cast<uint32_t*>(total + 1 + kMaxViews), total, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  uint64_t m = 0;
  GS_CUDA(c, cudaMemcpyAsync(&m, total, sizeof(m), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  *count = (int64_t)m;
  if (!points) return GS_OK;
  if ((int64_t)m > capacity) return fail(c, GS_ECAPACITY, "%llu crossings exceed the capacity", (unsigned long long)m);
  a.points = points;
  a.normals = normals;
  a.capacity = capacity;
  {
    LaunchScope ls(c, "iso_crossings");
    launch_iso(a, true, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

gs_status gs_init_gaussians(gs_ctx* c, const float* points, const float* normals, int64_t m, const int64_t* select,
                            int64_t n, float flatten, float opacity_logit, gs_params* out) {
  if (!c) return GS_EINVAL;
  if (!points || !normals) return fail(c, GS_EINVAL, "points and normals must not be NULL");
  GS_TRY(check_params(c, out, "out"));
  if (out->n != n || n < 4 || m < n || (!select && m != n))
    return fail(c, GS_EINVAL, "need n = out->n >= 4 and m >= n (m = n without select)");
  if (!(flatten > 0.f) || n >= ((int64_t)1 << 31)) return fail(c, GS_EINVAL, "bad flatten or n");
  set_device(c);
  c->projected = c->sorted = c->rastered = c->cells_ready = false;
  // the selected points, contiguous
  const float* pts = points;
  if (select) {
    GS_TRY(ensure(c, c->init_pts, sizeof(float) * 3 * n));
    launch_init_gather(points, select, n, P<float>(c->init_pts), c->stream);
    GS_CHECK_LAUNCH(c);
    pts = P<float>(c->init_pts);
  }
  // bounds -> grid of about one point per cell volume
  const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8));
  GS_TRY(ensure(c, c->knn_part, sizeof(float) * 6 * (nparts + 1)));
  float* bounds_d = P<float>(c->knn_part) + 6 * nparts;
  launch_knn_bounds(pts, n, P<float>(c->knn_part), nparts, bounds_d, c->stream);
  GS_CHECK_LAUNCH(c);
  float bounds[6];
  GS_CUDA(c, cudaMemcpyAsync(bounds, bounds_d, sizeof(bounds), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  KnnArgs k{};
  k.pts = pts;
  k.n = n;
  k.k = 3;
  double ext[3], vol = 1.0, emax = 0.0;
  for (int d = 0; d < 3; d++) {
    ext[d] = (double)bounds[3 + d] - (double)bounds[d];
    emax = std::max(emax, ext[d]);
  }
  if (!(emax > 0.0) || !std::isfinite(emax)) return fail(c, GS_EINVAL, "points must span a finite, nonzero box");
  for (int d = 0; d < 3; d++) vol *= std::max(ext[d], emax * 1e-3);
  double cell = std::cbrt(vol / (double)n);
  int64_t cells = 1;
  for (int d = 0; d < 3; d++) {
    int64_t dim = (int64_t)(ext[d] / cell) + 1;
    while (dim > (1 << 20)) {  // keep every axis within 2^20 cells
      cell *= 2.0;
      dim = (int64_t)(ext[d] / cell) + 1;
    }
    k.dims[d] = (int)dim;
  }
  for (int d = 0; d < 3; d++) {
    k.dims[d] = (int)((int64_t)(ext[d] / cell) + 1);
    cells *= k.dims[d];
    k.lo[d] = bounds[d];
  }
  k.cell = (float)cell;
  k.inv_cell = (float)(1.0 / cell);
  int bits = 1;
  while (((int64_t)1 << bits) < cells) bits++;
  int tbits = 10;
  while (((int64_t)1 << tbits) < 2 * n) tbits++;
  k.table_bits = tbits;
  GS_TRY(ensure(c, c->keys0, sizeof(uint64_t) * n));
  GS_TRY(ensure(c, c->keys1, sizeof(uint64_t) * n));
  GS_TRY(ensure(c, c->vals0, sizeof(uint32_t) * n));
  GS_TRY(ensure(c, c->vals1, sizeof(uint32_t) * n));
  GS_TRY(ensure(c, c->knn_table, (sizeof(uint64_t) + sizeof(uint32_t)) << tbits));
  GS_TRY(ensure(c, c->init_scales, sizeof(float) * n));
  {
    LaunchScope ls(c, "knn_cells");
    launch_knn_keys(k, P<uint64_t>(c->keys0), P<uint32_t>(c->vals0), c->stream);
  }
  GS_CHECK_LAUNCH(c);
  int which = 0;
  GS_TRY(sort_pairs(c, n, bits, &which));
  k.skeys = which ? P<uint64_t>(c->keys1) : P<uint64_t>(c->keys0);
  k.svals = which ? P<uint32_t>(c->vals1) : P<uint32_t>(c->vals0);
  k.table_keys = P<uint64_t>(c->knn_table);
  k.table_start = reinterpret_cast<uint32_t*>(P<uint64_t>(c->knn_table) + ((size_t)1 << tbits));
  k.out = P<float>(c->init_scales);
  GS_CUDA(c, cudaMemsetAsync(k.table_keys, 0xff, sizeof(uint64_t) << tbits, c->stream));
  {
    LaunchScope ls(c, "knn_query", 2);
    launch_knn_query(k, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  InitArgs a{};
  a.points = points;
  a.normals = normals;
  a.sel = select;
  a.n = n;
  a.log_scales = P<float>(c->init_scales);
  a.log_flatten = std::log(flatten);
  a.opacity_logit = opacity_logit;
  a.params = out->data;
  a.stride = out->stride;
  a.planes = n_planes(out->sh_degree);
  {
    LaunchScope ls(c, "init_params");
    launch_init_params(a, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  return GS_OK;
}

// ---------------------------------------------------------------- densification

gs_status gs_set_densify_stats(gs_ctx* c, float* grad_accum, float* count) {
  if (!c) return GS_EINVAL;
  if ((grad_accum == nullptr) != (count == nullptr)) return fail(c, GS_EINVAL, "both arrays or neither");
  if (c->capturing || c->gexec) return fail(c, GS_ESTATE, "the statistic arrays are fixed once a graph is captured");
  c->dens_grad = grad_accum;
  c->dens_count = count;
  return GS_OK;
}

static gs_status check_out_set(gs_ctx* c, const gs_params* o, int deg, const char* what) {
  if (!o || !o->data) return fail(c, GS_EINVAL, "%s is NULL", what);
  if (o->stride < 4 || o->stride % 4 != 0 || reinterpret_cast<uintptr_t>(o->data) % 16 != 0)
    return fail(c, GS_EINVAL, "%s: stride must be a positive multiple of 4, data 16-byte aligned", what);
  if (o->sh_degree != deg) return fail(c, GS_EINVAL, "%s: SH degree differs from the input set", what);
  return GS_OK;
}

gs_status gs_densify(gs_ctx* c, const gs_params* p, const gs_params* m, const gs_params* v, const float* grad_accum,
                     const float* count, const float* noise, const gs_densify_hp* hp, gs_params* p_out,
                     gs_params* m_out, gs_params* v_out, int64_t* n_out) {
  if (!c) return GS_EINVAL;
  GS_TRY(check_params(c, p, "p"));
  GS_TRY(check_params(c, m, "m"));
  GS_TRY(check_params(c, v, "v"));
  if (m->n != p->n || v->n != p->n || m->stride != p->stride || v->stride != p->stride ||
      m->sh_degree != p->sh_degree || v->sh_degree != p->sh_degree)
    return fail(c, GS_EINVAL, "p, m, v must share n, stride and sh_degree");
  if (!grad_accum || !count || !noise || !hp || !n_out) return fail(c, GS_EINVAL, "NULL argument");
  if (hp->split_n < 1 || hp->split_n > 4) return fail(c, GS_EINVAL, "split_n must be 1..4");
  GS_TRY(check_out_set(c, p_out, p->sh_degree, "p_out"));
  GS_TRY(check_out_set(c, m_out, p->sh_degree, "m_out"));
  GS_TRY(check_out_set(c, v_out, p->sh_degree, "v_out"));
  if (m_out->stride != p_out->stride || v_out->stride != p_out->stride)
    return fail(c, GS_EINVAL, "p_out, m_out, v_out must share the stride");
  set_device(c);
  const int64_t nb = (p->n + 255) / 256;
  GS_TRY(ensure(c, c->block_sums, sizeof(uint32_t) * nb));
  GS_TRY(ensure(c, c->block_offsets, sizeof(uint32_t) * nb));
  GS_TRY(ensure(c, c->total, sizeof(uint64_t) * (1 + kMaxViews) +
                                 sizeof(uint32_t) * (2 * (kMaxViews + 1) + 16 + 8 * kMaxViews)));
  DensifyArgs a{};
  a.p = p->data;
  a.m = m->data;
  a.v = v->data;
  a.n = p->n;
  a.stride = p->stride;
  a.planes = n_planes(p->sh_degree);
  a.grad = grad_accum;
  a.count = count;
  a.noise = noise;
  a.tau = hp->grad_threshold;
  a.dense_extent = hp->percent_dense * hp->scene_extent;
  a.min_opacity = hp->min_opacity;
  a.split_n = hp->split_n;
  a.log_shrink = (float)std::log(0.8 * hp->split_n);
  a.block_counts = P<uint32_t>(c->block_sums);
  a.block_offsets = P<uint32_t>(c->block_offsets);
  uint64_t* total = P<uint64_t>(c->total);
  {
    LaunchScope ls(c, "densify");
    launch_densify(a, false, c->stream);
  }
  {
    LaunchScope ls(c, "scan_block_sums", 2);
    launch_scan_block_sums(P<uint32_t>(c->block_sums), nb, 1, P<uint32_t>(c->block_offsets), total + 1,
                           reinterpret_cast<uint32_t*>(total + 1 + kMaxViews), total, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  uint64_t cnt = 0;
  GS_CUDA(c, cudaMemcpyAsync(&cnt, total, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  *n_out = (int64_t)cnt;
  if ((int64_t)cnt > p_out->stride)
    return fail(c, GS_ECAPACITY, "%llu Gaussians after densification exceed the output stride",
                (unsigned long long)cnt);
  a.po = p_out->data;
  a.mo = m_out->data;
  a.vo = v_out->data;
  a.out_stride = p_out->stride;
  {
    LaunchScope ls(c, "densify");
    launch_densify(a, true, c->stream);
  }
  GS_CHECK_LAUNCH(c);
  c->projected = c->sorted = c->rastered = c->cells_ready = false;
  return GS_OK;
}

gs_status gs_pair_stats(gs_ctx* c, int64_t* entries, int64_t* contributing) {
  if (!c || !entries || !contributing) return GS_EINVAL;
  if (!c->rastered) return fail(c, GS_ESTATE, "gs_pair_stats needs gs_raster_fwd first");
  if (c->capturing) return fail(c, GS_ESTATE, "gs_pair_stats cannot be captured");
  set_device(c);
  GS_TRY(ensure(c, c->pair_stats, 2 * sizeof(unsigned long long)));
  GS_CUDA(c, cudaMemsetAsync(c->pair_stats.p, 0, 2 * sizeof(unsigned long long), c->stream));
  {
    LaunchScope ls(c, "pair_stats");
    launch_pair_stats(raster_args(c), c->bins, P<unsigned long long>(c->pair_stats), c->stream);
  }
  GS_CHECK_LAUNCH(c);
  GS_CUDA(c, cudaMemcpyAsync(c->pinned, c->pair_stats.p, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
  GS_CUDA(c, cudaStreamSynchronize(c->stream));
  *entries = (int64_t)c->pinned[0];
  *contributing = (int64_t)c->pinned[1];
  return GS_OK;
}

gs_status gs_set_option(gs_ctx* c, int32_t option, int64_t value) {
  if (!c) return GS_EINVAL;
  switch (option) {
    case GS_OPT_RASTER_FWD:
    case GS_OPT_RASTER_BWD:
      if (value != 1 && value != 2 && value != 4 && value != 8)
        return fail(c, GS_EINVAL, "raster variant must be 1, 2, 4 or 8");
      (option == GS_OPT_RASTER_FWD ? c->raster_fwd : c->raster_bwd) = (int)value;
      return GS_OK;
    case GS_OPT_BWD_DIRECT:
      if (value < 0 || value > 32) return fail(c, GS_EINVAL, "direct-atomic lane limit must be 0..32");
      c->bwd_direct = (int)value;
      return GS_OK;
    case GS_OPT_SORT_ITEMS:
      if (value != 12 && value != 16 && value != 20 && value != 24)
        return fail(c, GS_EINVAL, "sort items per thread must be 12, 16, 20 or 24");
      if (c->capturing || c->gexec) return fail(c, GS_ESTATE, "sort partition size is fixed once a graph is captured");
      c->sort_items = (int)value;
      return GS_OK;
    case GS_OPT_TILE_ORDER:
      if (value != 0 && value != 1) return fail(c, GS_EINVAL, "tile order must be 0 or 1");
      if (c->capturing || c->gexec) return fail(c, GS_ESTATE, "tile order is fixed once a graph is captured");
      c->tile_order_mode = (int)value;
      return GS_OK;
    case GS_OPT_SORT_WAIT:
      if (value < 0 || value > (1 << 20)) return fail(c, GS_EINVAL, "sort wait rounds must be 0..1048576");
      if (c->capturing || c->gexec) return fail(c, GS_ESTATE, "sort wait is fixed once a graph is captured");
      c->sort_wait = (int)value;
      return GS_OK;
    default:
      return fail(c, GS_EINVAL, "unknown option %d", option);
  }
}

gs_status gs_get_option(gs_ctx* c, int32_t option, int64_t* value) {
  if (!c || !value) return GS_EINVAL;
  switch (option) {
    case GS_OPT_RASTER_FWD: *value = c->raster_fwd; return GS_OK;
    case GS_OPT_RASTER_BWD: *value = c->raster_bwd; return GS_OK;
    case GS_OPT_BWD_DIRECT: *value = c->bwd_direct; return GS_OK;
    case GS_OPT_SORT_ITEMS: *value = c->sort_items; return GS_OK;
    case GS_OPT_SORT_WAIT: *value = c->sort_wait; return GS_OK;
    case GS_OPT_TILE_ORDER: *value = c->tile_order_mode; return GS_OK;
    default: return fail(c, GS_EINVAL, "unknown option %d", option);
  }
}

gs_status gs_train_graph_capture(gs_ctx* c, gs_params* p, gs_params* g, gs_params* m, gs_params* v,
                                 const gs_adam_hp* hp, const gs_camera* cams, int32_t B, const float* targets,
                                 float* images, float* dL_dimages, float* loss) {
  if (!c) return GS_EINVAL;
  if (c->cfg.instance_capacity <= 0)
    return fail(c, GS_EINVAL, "graph capture needs a context with a fixed instance capacity");
  if (!hp || !cams || !targets || !images || !dL_dimages || !loss)
    return fail(c, GS_EINVAL, "NULL argument");
  set_device(c);
  // 1. one uncaptured pass (no parameter update) sizes every workspace
  GS_TRY(gs_project(c, p, cams, B));
  GS_TRY(gs_bin_sort(c));
  GS_TRY(ensure(c, c->target_slot, sizeof(void*)));
  GS_TRY(gs_raster_fwd_l1(c, images, targets, loss, dL_dimages));
  GS_TRY(gs_raster_bwd(c, p, dL_dimages, g));
  GS_TRY(ensure(c, c->adam_consts, 65 * sizeof(float)));
  GS_TRY(gs_sync(c));
  // 2. capture on a private stream
  if (!c->graph_stream) GS_CUDA(c, cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
  if (!c->side_stream) GS_CUDA(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
  if (!c->fork_ev) GS_CUDA(c, cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
  if (!c->join_ev) GS_CUDA(c, cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
  const size_t g2d_bytes = sizeof(float) * (kG2dGeo + kG2dCol) * (size_t)B * c->stride;
  if (c->g2d.cap < g2d_bytes) return fail(c, GS_ESTATE, "2D-gradient records not sized by the warm-up pass");
  if (c->gexec) {
    GS_CUDA(c, cudaGraphExecDestroy(c->gexec));
    c->gexec = nullptr;
  }
  cudaStream_t user = c->stream;
  c->stream = c->graph_stream;
  c->capturing = true;
  c->graph_kernels = 0;
  gs_status st = GS_OK;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->graph_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    // per-step constants: staging area -> device, then the step
    e = cudaMemcpyAsync(c->views.p, c->staging, sizeof(ViewRec) * B, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->adam_consts.p, c->staging + kAdamStagingOff, 65 * sizeof(float),
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->target_slot.p, c->staging + kTargetStagingOff, sizeof(void*), cudaMemcpyHostToDevice,
                          c->stream);
    // an external record: the event is recorded at every replay, so the host
    // can wait on it before rewriting the staging area
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->staged_ev, c->stream, cudaEventRecordExternal);
    if (e == cudaSuccess) st = gs_project(c, p, cams, B);
    if (e == cudaSuccess && st == GS_OK) st = gs_bin_sort(c);
    // the 2D-gradient records are cleared on a side branch beside the
    // forward compositing (compute-bound, little DRAM traffic), joined
    // before the backward adds into them
    if (e == cudaSuccess && st == GS_OK) e = cudaEventRecord(c->fork_ev, c->stream);
    if (e == cudaSuccess && st == GS_OK) e = cudaStreamWaitEvent(c->side_stream, c->fork_ev, 0);
    if (e == cudaSuccess && st == GS_OK) e = cudaMemsetAsync(c->g2d.p, 0, g2d_bytes, c->side_stream);
    if (e == cudaSuccess && st == GS_OK) e = cudaEventRecord(c->join_ev, c->side_stream);
    if (e == cudaSuccess && st == GS_OK) st = gs_raster_fwd_l1(c, images, targets, loss, dL_dimages);
    if (e == cudaSuccess && st == GS_OK) e = cudaStreamWaitEvent(c->stream, c->join_ev, 0);
    if (e == cudaSuccess && st == GS_OK) c->g2d_cleared = true;
    if (e == cudaSuccess && st == GS_OK) st = gs_raster_bwd(c, p, dL_dimages, g);
    c->g2d_cleared = false;
    if (e == cudaSuccess && st == GS_OK) st = gs_adam(c, p, g, m, v, hp, 1);
    const cudaError_t e2 = cudaStreamEndCapture(c->graph_stream, &graph);
    if (e == cudaSuccess) e = e2;
  }
  c->capturing = false;
  c->stream = user;
  if (e == cudaSuccess && st == GS_OK) e = cudaGraphInstantiate(&c->gexec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != GS_OK) return st;
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    c->gexec = nullptr;
    return fail(c, GS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  c->graph_B = B;
  c->graph_res.clear();
  for (int i = 0; i < B; i++) {
    c->graph_res.push_back(cams[i].width);
    c->graph_res.push_back(cams[i].height);
  }
  c->graph_hp = *hp;
  c->graph_planes = n_planes(p->sh_degree);
  c->graph_loss = loss;
  c->graph_count = 3 * c->pixels;
  return GS_OK;
}

gs_status gs_train_graph_launch(gs_ctx* c, const gs_camera* cams, int32_t B, const float* targets, int64_t step) {
  if (!c) return GS_EINVAL;
  if (!c->gexec) return fail(c, GS_ESTATE, "no captured training graph");
  if (!cams || !targets || B != c->graph_B || step < 1)
    return fail(c, GS_EINVAL, "cameras must match the captured batch; targets must not be NULL");
  for (int i = 0; i < B; i++)
    if (cams[i].width != c->graph_res[2 * i] || cams[i].height != c->graph_res[2 * i + 1])
      return fail(c, GS_EINVAL, "camera %d: resolution differs from the captured batch", i);
  set_device(c);
  int64_t tiles = 0, pixels = 0;
  GS_TRY(build_views(c, cams, B, &tiles, &pixels));
  // the previous replay must have read the staging area before it is rewritten
  GS_CUDA(c, cudaEventSynchronize(c->staged_ev));
  memcpy(c->staging, c->views_h.data(), sizeof(ViewRec) * B);
  adam_constants(&c->graph_hp, c->graph_planes, step, c->graph_B,
                 reinterpret_cast<float*>(c->staging + kAdamStagingOff));
  memcpy(c->staging + kTargetStagingOff, &targets, sizeof(void*));
  {
    LaunchScope ls(c, "train_graph", (int)c->graph_kernels);
    GS_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
  }
  c->projected = c->sorted = c->rastered = true;
  c->cells_ready = !c->forward_only;
  return GS_OK;
}

gs_status gs_train_graph_launch_host(gs_ctx* c, const gs_camera* cams, int32_t B, const float* host_targets,
                                     int64_t step, float* host_loss) {
  if (!c) return GS_EINVAL;
  if (!c->gexec) return fail(c, GS_ESTATE, "no captured training graph");
  if (!host_targets) return fail(c, GS_EINVAL, "targets must not be NULL");
  set_device(c);
  if (!c->copy_stream) {
    GS_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++) {
      GS_CUDA(c, cudaEventCreateWithFlags(&c->tgt_copied[i], cudaEventDisableTiming));
      GS_CUDA(c, cudaEventCreateWithFlags(&c->tgt_free[i], cudaEventDisableTiming));
    }
  }
  const int slot = (int)(c->host_launches & 1);
  DevBuf& buf = slot ? c->host_tgt1 : c->host_tgt0;
  const size_t bytes = sizeof(float) * (size_t)c->graph_count;
  GS_TRY(ensure(c, buf, bytes));
  // the upload is issued once the previous replay has started (has copied
  // its staging area): issued earlier, it occupied the copy engine ahead of
  // that replay's own small staging copy and delayed the replay by the
  // length of the upload
  GS_CUDA(c, cudaEventSynchronize(c->staged_ev));
  // the buffer is rewritten once the replay that read it (two calls ago) is done
  GS_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->tgt_free[slot], 0));
  GS_CUDA(c, cudaMemcpyAsync(buf.p, host_targets, bytes, cudaMemcpyHostToDevice, c->copy_stream));
  GS_CUDA(c, cudaEventRecord(c->tgt_copied[slot], c->copy_stream));
  GS_CUDA(c, cudaStreamWaitEvent(c->stream, c->tgt_copied[slot], 0));
  GS_TRY(gs_train_graph_launch(c, cams, B, P<float>(buf), step));
  GS_CUDA(c, cudaEventRecord(c->tgt_free[slot], c->stream));
  if (host_loss)
    GS_CUDA(c, cudaMemcpyAsync(host_loss, c->graph_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  c->host_launches++;
  return GS_OK;
}

gs_status gs_profile_enable(gs_ctx* c, int32_t enable) {
  if (!c) return GS_EINVAL;
  c->profiling = enable != 0;
  return GS_OK;
}

gs_status gs_profile_read(gs_ctx* c, gs_kernel_stat* out, int32_t cap, int32_t* count) {
  if (!c || !count || (cap > 0 && !out)) return GS_EINVAL;
  set_device(c);
  if (!c->pending.empty()) {
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    for (const auto& p : c->pending) {
      float ms = 0.f;
      GS_CUDA(c, cudaEventElapsedTime(&ms, p.a, p.b));
      c->kstats[p.kernel].ms += ms;
      c->event_pool.push_back(p.a);
      c->event_pool.push_back(p.b);
    }
    c->pending.clear();
  }
  const int32_t nk = (int32_t)c->kstats.size();
  for (int32_t i = 0; i < nk && i < cap; i++) {
    memset(&out[i], 0, sizeof(gs_kernel_stat));
    strncpy(out[i].name, c->kstats[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = c->kstats[i].launches;
    out[i].total_ms = c->kstats[i].ms;
  }
  *count = nk;
  return GS_OK;
}

gs_status gs_profile_reset(gs_ctx* c) {
  if (!c) return GS_EINVAL;
  set_device(c);
  if (!c->pending.empty()) {
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    for (const auto& p : c->pending) {
      c->event_pool.push_back(p.a);
      c->event_pool.push_back(p.b);
    }
    c->pending.clear();
  }
  for (auto& k : c->kstats) {
    k.launches = 0;
    k.ms = 0.0;
  }
  return GS_OK;
}

}  // extern "C"

