// Kernel argument blocks and launchers (host side of the CUDA kernels).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

struct ProjectArgs {
  const float* params;
  int64_t n, stride;
  const ViewRec* views;
  int B;
  float4* rec0;  // records 0, 1, 2 of entry o at rec0[3 o], rec1[3 o], rec2[3 o]
  float4* rec1;  // (one interleaved array: rec1 = rec0 + 1, rec2 = rec0 + 2)
  float4* rec2;
  int4* rec3;            // (radius, tiles, x0 | x1 << 16, y0 | y1 << 16) per (view, Gaussian)
  uint2* tiles;          // [B][stride]: (tiles touched, bits of the depth)
  uint32_t* block_sums;  // [B][ceil(n / block)] instance counts per view and block
  uint32_t* vis_sums;    // [B][ceil(n / block)] visible (tiles > 0) Gaussians per view and block
  uint64_t* vismask;     // [stride]: bit v = the Gaussian touches a tile of view v
};

struct ProjectBwdArgs {
  const float* params;
  int64_t n, stride;
  const ViewRec* views;
  int B;
  const float* g2d;   // [B][stride] geometry records (kG2dGeo floats), then [B][stride] colour records (kG2dCol)
  float* grads;       // [P][stride]
  const uint64_t* vismask;  // [stride] views where the Gaussian touches a tile (others: zero 2D gradient)
  float* dens_grad;   // densification statistic (NULL: not accumulated): += sum of NDC mean-gradient norms
  float* dens_count;  //   and += the number of views where the Gaussian touches a tile
};

// Visible (view, Gaussian) pairs -> (depth bits, Gaussian), view by view.
struct CompactArgs {
  int64_t n, stride;
  int B;
  const uint2* tiles;             // [B][stride] (tiles touched, bits of the depth)
  const uint32_t* vis_offsets;    // [B][blocks] exclusive scan of each view's visible counts per block
  const uint32_t* vseg;           // [B + 1] first pair of each view's segment
  uint32_t* dkeys;                // depth bits
  uint32_t* dvals;                // Gaussian index
};

// Depth-sorted visible pairs -> one (bin, Gaussian) instance per touched tile.
struct EmitArgs {
  int B;
  int64_t n, stride;
  const ViewRec* views;
  const int4* rec3;               // [B][stride] (radius, tiles, x0 | x1 << 16, y0 | y1 << 16)
  const uint32_t* dvals[2];       // the depth sort's buffers; dctrl[dpass] bit 0 says which is sorted
  const uint32_t* dctrl;
  int dpass;
  const uint32_t* vseg;           // [B + 1] visible pairs: first of each view
  const uint32_t* seg;            // [B + 1] instances: first of each view
  uint32_t* keys;                 // [capacity] bins
  uint32_t* vals;                 // [capacity] Gaussians
  int64_t capacity;
  uint64_t* lookback;             // [emit_partitions] status words, zeroed before the launch
  uint32_t* counter;              // partition ticket, zeroed before the launch
  uint32_t* hist;                 // [B][tpass][256] tile digit counts (added to; zeroed before)
  int tpass;
  int wait_rounds;
  int* status;
};

struct RasterArgs {
  const ViewRec* views;
  int B;
  int64_t stride;       // view stride of the records
  int64_t n;            // Gaussians (indices at or above are ignored)
  const uint2* ranges;  // [bins]
  const uint32_t* const* vals;  // device slot holding the sorted Gaussian indices
  const float4* rec0;
  const float4* rec1;
  const float4* rec2;
  float* image;         // [B][3][H][W] concatenated (forward: may be NULL when fused with the L1 loss)
  float* tfinal;        // [pixels]
  uint32_t* nlast;      // [pixels]
  // contribution masks: per tile, per batch of 32 list entries and per cell
  // of 2 x 4 pixels, the entries that contributed to a pixel of the cell
  // (instances + 32 bins words; written by the forward, NULL: not recorded;
  // read by the backward, which walks only those entries)
  uint32_t* cells;
  // tile order of the compositing kernels: block slot k composites bin
  // tile_order[k] (NULL: bin order)
  const uint32_t* tile_order;
  const float* dimage;  // backward only
  float* g2d;           // backward only: [B][stride] geometry records, then [B][stride] colour records
  int direct_max;       // backward only: at most this many contributing lanes -> per-lane atomics
  // forward fused with the L1 loss (target non-NULL or read from target_slot):
  // writes dL/dimage = sign(image - target) * inv_count and one partial sum
  // of |image - target| per block
  const float* target;
  const float* const* target_slot;
  float* l1_grad;
  float* l1_partial;
  float inv_count;
};

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

int project_fwd_block();
void launch_project_fwd(const ProjectArgs& a, int deg, cudaStream_t s);
void launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t s);

void launch_scan_block_sums(const uint32_t* sums, int64_t nb, int B, uint32_t* offsets, uint64_t* view_total,
                            uint32_t* seg, uint64_t* total, cudaStream_t s);
void launch_compact(const CompactArgs& a, cudaStream_t s);
// pair_capacity: visible pairs the grid covers (B x stride)
void launch_emit(const EmitArgs& a, int64_t pair_capacity, cudaStream_t s);
int64_t emit_partitions(int64_t pairs, int segments);
size_t emit_lookback_bytes(int64_t pair_capacity, int segments);

// LSD radix sort of (key, value) pairs on key bits [0, 8 npass), ping-pong
// between keys[0]/vals[0] (input) and keys[1]/vals[1].  Everything that
// depends on the data (instance count, skipped passes, which buffer ends up
// sorted) is decided on the device, so the sequence can be captured in a
// CUDA graph.
struct SortArgs {
  void* keys[2];             // uint32 or uint64 keys (key_bytes)
  uint32_t* vals[2];
  int key_bytes;             // 4 or 8
  int view_shift;            // a segment's key base: views[v].tile_offset << view_shift
  const uint64_t* count;     // device: number of pairs (clamped to capacity)
  int64_t capacity;          // pairs the buffers hold
  int64_t bins;              // valid bin ids are [0, bins)
  int B;                     // views: one segment each
  const ViewRec* views;      // NULL: key base 0 for every segment
  const uint32_t* seg;       // [B + 1] segment offsets
  uint32_t* part_off;        // [B + 1] first partition of each segment
  uint32_t* part_order;      // [partitions] status slot of the partition each ticket takes
                             // (views interleaved; NULL: ticket order)
  uint32_t* single;          // [B][8] 1 if the view's keys share one digit in the pass
  uint32_t* hist;            // [B][npass][256] digit counts
  uint32_t* hist_scan;       // [B][npass][256] exclusive digit offsets within the segment
  uint32_t* ctrl;            // [npass + 1] pass control: source buffer, skipped
  uint32_t* lookback;        // [npass][lookback_stride]
  size_t lookback_stride;    // uint32 per pass (sort_lookback_bytes / 4)
  uint32_t* counters;        // [8] partition tickets
  int npass;
  int wait_rounds;  // look-back rounds before giving up (0: give up at once)
  int* status;
  const void** sorted_keys;  // device slots: where the sorted list ends up (tile_ranges)
  const uint32_t** sorted_vals;
};

// Longest-list-first tile order: key = 31 - floor(log2(list length + 1)),
// value = bin, for a one-segment stable sort of the bins; the count and the
// segment bounds of that sort; the sorted values copied into `order`.
void launch_tile_order_keys(const uint2* ranges, int64_t bins, uint64_t* keys, uint32_t* vals, uint64_t* count,
                            uint32_t* seg, cudaStream_t s);
void launch_tile_order_finish(const uint32_t* ctrl, int npass, const uint32_t* v0, const uint32_t* v1, int64_t bins,
                              uint32_t* order, cudaStream_t s);

size_t sort_lookback_bytes(int64_t count, int items, int segments);
int64_t sort_partitions(int64_t count, int items, int segments);
// digit counts (into a.hist, zeroed before), their scans and the pass control words
void launch_digit_histogram(const SortArgs& a, int64_t grid_hint, int items, cudaStream_t s);
// the scans, control words and partition order only (a.hist counted elsewhere)
void launch_digit_scan(const SortArgs& a, int items, cudaStream_t s);
// items: keys per thread (12, 16, 20 or 24); the grid covers a.capacity
void launch_onesweep_pass(const SortArgs& a, int pass, int items, cudaStream_t s);
void launch_tile_ranges(const SortArgs& a, int64_t grid_hint, uint2* ranges, cudaStream_t s);

void launch_raster_fwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s);
// warps of a forward launch (one L1 partial sum each when fused)
int64_t raster_fwd_warps(int64_t bins, int ppt);
int64_t l1_finish_scratch_bytes();
void launch_l1_finish(const float* partial, int64_t nparts, double* scratch, double inv_count, float* loss,
                      cudaStream_t s);
void launch_raster_bwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s);
// out[0] += list entries up to each pixel's last contributor, out[1] += contributing pairs
void launch_pair_stats(const RasterArgs& a, int64_t bins, unsigned long long* out, cudaStream_t s);

void launch_l1(const float* x, const float* y, const float* const* y_slot, int64_t count, float* partial,
               int nparts, float* loss, float* grad, cudaStream_t s);
int l1_parts(int64_t count);

// SSIM / D-SSIM over a batch of views (ssim.cu).
struct SsimArgs {
  const ViewRec* views;
  int B;
  const int* first_block;  // [B + 1] first block of each view (3 channels x 32 x 16 tiles)
  const float* x;          // images (batch layout)
  const float* y;          // targets
  int64_t count;           // 3 x pixels of the batch
  float* partials;         // [3][count]: dSSIM/d(mx), dSSIM/dE[x^2], dSSIM/dE[xy] per pixel
  double* block_sums;      // [blocks][3]: sums of the SSIM map, |x - y|, (x - y)^2
  float* grad;             // dL/dx (backward)
  float win[11];           // normalised Gaussian window (sigma 1.5)
  float w_l1, w_ssim, inv_count;
  double w_l1_d, w_ssim_d;
};
int ssim_blocks_of_view(int W, int H);
void ssim_window(float* w);
// forward (+ per-view sums into out_view[3 B] and the loss) and, if
// backward, the gradient
void launch_ssim(const SsimArgs& a, int blocks, bool backward, double* out_view, float* loss, cudaStream_t s);

// Point-cloud initialisation (init.cu).
struct IsoArgs {
  const float* vol;  // [nz][ny][nx]
  int nx, ny, nz;
  int64_t nverts;
  float iso;
  float origin[3], h[3];
  uint32_t* block_counts;         // count pass: crossings per block of 256 vertices
  const uint32_t* block_offsets;  // emit pass: exclusive scan of block_counts
  float* points;                  // [capacity][3]
  float* normals;                 // [capacity][3]
  int64_t capacity;
  int* status;
};
void launch_iso(const IsoArgs& a, bool emit, cudaStream_t s);

struct KnnArgs {
  const float* pts;  // [n][3]
  int64_t n;
  int k;             // 1..8 neighbours
  float lo[3], cell, inv_cell;
  int dims[3];
  const uint64_t* skeys;  // cell ids, sorted
  const uint32_t* svals;  // point of each sorted position
  uint64_t* table_keys;   // [2^table_bits] cell id (all ones: empty)
  uint32_t* table_start;  // first sorted position of the cell
  int table_bits;
  float* out;        // [n] log-scales
};
void launch_knn_bounds(const float* pts, int64_t n, float* part, int nparts, float* out, cudaStream_t s);
void launch_knn_keys(const KnnArgs& a, uint64_t* keys, uint32_t* vals, cudaStream_t s);
void launch_knn_query(const KnnArgs& a, cudaStream_t s);

struct InitArgs {
  const float* points;   // [m][3]
  const float* normals;  // [m][3]
  const int64_t* sel;    // [n] indices into the points (NULL: the first n)
  int64_t n;
  const float* log_scales;  // [n]
  float log_flatten, opacity_logit;
  float* params;
  int64_t stride;
  int planes;
};
void launch_init_params(const InitArgs& a, cudaStream_t s);
void launch_init_gather(const float* pts, const int64_t* sel, int64_t n, float* out, cudaStream_t s);

// Adaptive density control (densify.cu).
struct DensifyArgs {
  const float* p;
  const float* m;
  const float* v;
  int64_t n, stride;
  int planes;
  const float* grad;   // [n] summed statistic
  const float* count;  // [n] views counted
  const float* noise;  // [n][split_n][3] standard normals
  float tau, dense_extent, min_opacity, log_shrink;
  int split_n;
  uint32_t* block_counts;
  const uint32_t* block_offsets;
  float* po;
  float* mo;
  float* vo;
  int64_t out_stride;
};
void launch_densify(const DensifyArgs& a, bool emit, cudaStream_t s);

struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t stride;
  int planes;
  const float* consts;  // device: [64] per-plane lr / (1 - beta1^t), [64] = 1 / sqrt(1 - beta2^t)
  float beta1, beta2, eps;
  const uint64_t* vismask;  // visible-only update: Gaussians with mask 0 keep p, m, v (NULL: dense)
};
void launch_adam(const AdamArgs& a, cudaStream_t s);

}  // namespace gs
