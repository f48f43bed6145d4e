// Binning: scan of tile counts, duplication into (tile, depth) keyed
// instances, an LSD onesweep radix sort and per-tile ranges.
//
// 3D-GS renders tile by tile from a list sorted by (tile, depth) (Section I);
// each Gaussian is emitted once per 16x16 tile its rect touches with the key
// (bin << 32) | bits(depth).  Depths are positive FP32 values, so their bit
// patterns order like the values.  The sort is stable, so equal keys keep the
// emission order, which is increasing Gaussian index within a bin.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

// ---------------------------------------------------------------- scan

// Exclusive scan of the per-block instance counts of the projection, one
// block of 1024 threads looping over chunks; writes the total too.
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(const uint32_t* __restrict__ sums,
                                                                int64_t nb, uint32_t* __restrict__ offsets,
                                                                uint64_t* __restrict__ total) {
  __shared__ uint64_t warp_tot[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + threadIdx.x;
    uint64_t x = i < nb ? sums[i] : 0;
    uint64_t inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = warp_tot[lane];
      uint64_t winc = w;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, winc, off);
        if (lane >= off) winc += y;
      }
      warp_tot[lane] = winc - w;  // exclusive over warps
    }
    __syncthreads();
    const uint64_t excl = carry + warp_tot[wid] + inc - x;
    if (i < nb) offsets[i] = (uint32_t)excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

void launch_scan_block_sums(const uint32_t* sums, int64_t nb, uint32_t* offsets, uint64_t* total,
                            cudaStream_t s) {
  scan_block_sums_kernel<<<1, 1024, 0, s>>>(sums, nb, offsets, total);
}

// ---------------------------------------------------------------- duplicate

// Same block partition as the projection (256 Gaussians per block, all views).
// Each warp emits the instances of its 32 Gaussians view by view: the
// warp's (Gaussian, view) items are expanded cooperatively, lane j writing
// output position base + 32 i + j of the chunk i, so every store of keys and
// values is coalesced.  Within a view the order is (Gaussian, ty, tx), so in
// every bin the instances appear in increasing Gaussian index, which the
// stable sort preserves for equal keys.
__global__ void __launch_bounds__(256) duplicate_kernel(DuplicateArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = g < a.n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t mine = 0;
  if (live)
    for (int v = 0; v < a.B; v++) mine += a.tiles[(int64_t)v * a.stride + g];
  // per-warp totals -> block exclusive scan over warps
  __shared__ uint32_t wsum[32];
  const uint32_t wtot = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) wsum[wid] = wtot;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? wsum[lane] : 0u;
    uint32_t winc = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, winc, off);
      if (lane >= off) winc += y;
    }
    wsum[lane] = winc - w;
  }
  __syncthreads();
  int64_t base = (int64_t)a.block_offsets[blockIdx.x] + wsum[wid];
  if (wtot == 0) return;
  if (base + wtot > a.capacity) {
    if (lane == 0) atomicOr(a.status, kStatusCapacity);
    return;
  }
  const unsigned lt = (1u << lane) - 1u;
  for (int v = 0; v < a.B; v++) {
    const int64_t o = (int64_t)v * a.stride + g;
    const uint32_t cnt = live ? a.tiles[o] : 0u;
    // exclusive offsets of the warp's items in this view
    uint32_t inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    const uint32_t excl = inc - cnt;
    const uint32_t vtot = __shfl_sync(0xffffffffu, inc, 31);
    if (vtot == 0) continue;
    const ViewRec& V = a.views[v];
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    uint32_t dbits = 0;
    if (cnt) {
      const float4 r0 = a.rec0[kRecStride * o];
      tile_rect(V, r0.x, r0.y, a.rec3[o].x, x0, x1, y0, y1);
      dbits = __float_as_uint(a.rec2[kRecStride * o].w);
    }
    const int rw = x1 - x0;
    for (uint32_t q0 = 0; q0 < vtot; q0 += 32) {
      const uint32_t q = q0 + lane;
      // owner: the last lane whose exclusive offset is <= q
      int own = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cand = own + step;
        const uint32_t ec = __shfl_sync(0xffffffffu, excl, cand & 31);
        if (cand < 32 && ec <= q) own = cand;
      }
      const uint32_t e_own = __shfl_sync(0xffffffffu, excl, own);
      const int ox0 = __shfl_sync(0xffffffffu, x0, own);
      const int oy0 = __shfl_sync(0xffffffffu, y0, own);
      const int orw = __shfl_sync(0xffffffffu, rw, own);
      const uint32_t od = __shfl_sync(0xffffffffu, dbits, own);
      const uint32_t oc = __shfl_sync(0xffffffffu, cnt, own);
      if (q < vtot && q - e_own < oc && orw > 0) {
        const uint32_t local = q - e_own;
        const int tx = ox0 + (int)(local % (uint32_t)orw);
        const int ty = oy0 + (int)(local / (uint32_t)orw);
        const uint64_t bin = (uint64_t)(V.tile_offset + ty * V.gw + tx);
        a.keys[base + q] = (bin << 32) | (uint64_t)od;
        a.vals[base + q] = (uint32_t)(g - lane + own);
      }
    }
    base += vtot;
  }
  (void)lt;
}

void launch_duplicate(const DuplicateArgs& a, cudaStream_t s) {
  const int threads = project_fwd_block();
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  duplicate_kernel<<<blocks, threads, 0, s>>>(a);
}

// ---------------------------------------------------------------- onesweep radix sort

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
// keys per thread (12, 16, 20 or 24; a context option, autotuned): a
// partition holds 256 x items keys
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 20;  // look-back rounds before giving up (about a second)
constexpr int kLookWindow = 16;       // statuses read per look-back round

int64_t sort_partitions(int64_t count, int items) {
  const int64_t tile = (int64_t)kSortThreads * items;
  return (count + tile - 1) / tile;
}

size_t sort_lookback_bytes(int64_t count, int items) {
  const int64_t parts = sort_partitions(count, items);
  return (size_t)(parts > 0 ? parts : 1) * kRadix * sizeof(uint32_t);
}

// Digit counts of every pass in one read of the keys.  hist: [npass][256].
__global__ void __launch_bounds__(256) digit_histogram_kernel(const uint64_t* __restrict__ keys,
                                                               const uint64_t* __restrict__ count_ptr,
                                                               int64_t capacity, int npass,
                                                               uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[8][kRadix];
  for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  const int64_t count = min((int64_t)*count_ptr, capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (int p = 0; p < npass; p++) atomicAdd(&sh[p][(k >> (kRadixBits * p)) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x) {
    const uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// Passes whose digit histogram is a single bucket leave the order unchanged
// and are skipped.  ctrl[p] (written once per sort by digit_scan_kernel):
// bit 0 = which ping-pong buffer holds the keys before pass p (p == npass:
// the sorted result), bit 1 = pass p is skipped.
constexpr uint32_t kCtrlParity = 1u, kCtrlTrivial = 2u;

// One LSD pass: rank keys of the partition by digit (stable), find the
// partition's offset for each digit by decoupled look-back over the earlier
// partitions (bounded waits), then scatter through shared memory so that the
// global writes are coalesced.  Keys are loaded up front (all loads in
// flight before ranking); keys and then values go through one shared buffer,
// which keeps the block at 46 KB of shared memory and 64 registers per thread
// (four blocks per SM).  hist_pass: exclusive digit offsets of this pass.
template <int ITEMS>
struct SortSmem {
  static constexpr int kTile = kSortThreads * ITEMS;
  uint32_t warp_hist[kSortWarps][kRadix];  // per-warp digit counts -> offsets
  uint32_t digit_start[kRadix];            // exclusive scan of the tile's digit counts
  uint32_t global_base[kRadix];            // global destination of the digit's first key
  uint32_t part;
  int timed_out;
  uint64_t buf[kTile];                     // keys, then values, in tile-sorted order
  uint8_t dig[kTile];                      // digit of each tile-sorted position
};

template <int ITEMS, int MIN_BLOCKS>
__global__ void __launch_bounds__(kSortThreads, MIN_BLOCKS) onesweep_pass_kernel(SortArgs a, int pass) {
  constexpr int kSortItems = ITEMS;
  constexpr int kSortTile = kSortThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<ITEMS>& sm = *reinterpret_cast<SortSmem<ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t count = min((int64_t)*a.count, a.capacity);
  const uint32_t ctrl = a.ctrl[pass];
  if (ctrl & kCtrlTrivial) return;  // whole block: this digit is the same for every key
  const int par = (int)(ctrl & kCtrlParity);
  // selects, not a dynamically indexed parameter array (which would be
  // copied to local memory)
  const uint64_t* __restrict__ kin = par ? a.keys[1] : a.keys[0];
  const uint32_t* __restrict__ vin = par ? a.vals[1] : a.vals[0];
  uint64_t* __restrict__ kout = par ? a.keys[0] : a.keys[1];
  uint32_t* __restrict__ vout = par ? a.vals[0] : a.vals[1];
  const int shift = kRadixBits * pass;
  const uint32_t* __restrict__ hist_pass = a.hist_scan + pass * kRadix;
  uint32_t* lookback = a.lookback + (size_t)pass * a.lookback_stride;
  int* status = a.status;
  if (tid == 0) {
    sm.part = atomicAdd(a.counters + pass, 1u);
    sm.timed_out = 0;
  }
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&sm.warp_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t part = sm.part;
  const int64_t nparts = (count + kSortTile - 1) / kSortTile;
  if ((int64_t)part >= nparts) return;
  const int64_t base = (int64_t)part * kSortTile;
  const int64_t wbase = base + (int64_t)wid * kSortItems * 32 + lane;  // item i at wbase + 32 i

  uint64_t key[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int64_t p = wbase + 32 * i;
    key[i] = p < count ? kin[p] : ~0ull;
  }
  // stable rank inside the warp (warp-striped order), 16-bit per item
  uint32_t rk[kSortItems / 2];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const bool ok = wbase + 32 * i < count;
    const uint32_t d = ok ? (uint32_t)(key[i] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t r = 0, before = 0;
    if (ok) {
      before = sm.warp_hist[wid][d];
      r = before + __popc(peers & lt);
    }
    __syncwarp();
    if (ok && (peers & lt) == 0) sm.warp_hist[wid][d] = before + __popc(peers);
    __syncwarp();
    if (i & 1) rk[i >> 1] |= r << 16; else rk[i >> 1] = r;
  }
  __syncthreads();

  // per digit: counts over warps -> warp offsets; publish the tile count
  const uint32_t d = tid;  // kSortThreads == kRadix
  uint32_t tile_count = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; w++) {
    const uint32_t c = sm.warp_hist[w][d];
    sm.warp_hist[w][d] = tile_count;
    tile_count += c;
  }
  volatile uint32_t* lb = lookback;
  lb[(int64_t)part * kRadix + d] = (part == 0 ? kFlagPrefix : kFlagAggregate) | tile_count;
  // digit starts inside the tile (block exclusive scan over the 256 digits)
  {
    uint32_t inc = tile_count;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    __shared__ uint32_t wtot[kSortWarps];
    if (lane == 31) wtot[wid] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; w++) wpre += wtot[w];
    sm.digit_start[d] = wpre + inc - tile_count;
  }
  __syncthreads();
  const int n_here = (int)((count - base) < kSortTile ? (count - base) : kSortTile);
  // keys -> tile-sorted positions in shared memory (frees the key registers
  // before the look-back); remember the positions for the values
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const bool ok = wbase + 32 * i < count;
    const uint32_t r = (rk[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
    uint32_t lp = 0xffffu;
    if (ok) {
      const uint32_t dd = (uint32_t)(key[i] >> shift) & (kRadix - 1);
      lp = sm.digit_start[dd] + sm.warp_hist[wid][dd] + r;
      sm.buf[lp] = key[i];
      sm.dig[lp] = (uint8_t)dd;
    }
    if (i & 1) rk[i >> 1] = (rk[i >> 1] & 0xffffu) | (lp << 16); else rk[i >> 1] = (rk[i >> 1] & 0xffff0000u) | lp;
  }
  // decoupled look-back over the earlier partitions, kLookWindow statuses
  // per round trip; a status that is not ready yet is re-read (bounded)
  uint32_t excl = 0;
  if (part > 0) {
    int64_t j = (int64_t)part - 1;
    int rounds = 0;
    bool found = false;
    while (!found) {
      uint32_t w[kLookWindow];
#pragma unroll
      for (int t = 0; t < kLookWindow; t++)
        w[t] = (j - t >= 0) ? (uint32_t)lb[(j - t) * kRadix + d] : (uint32_t)kFlagPrefix;
      int used = 0;
      bool stalled = false;
#pragma unroll
      for (int t = 0; t < kLookWindow; t++) {
        if (found || stalled) continue;
        const uint32_t flag = w[t] & ~kValueMask;
        if (flag == 0) {
          stalled = true;
          continue;
        }
        excl += w[t] & kValueMask;
        used++;
        if (flag == kFlagPrefix) found = true;
      }
      j -= used;
      if (!found && (++rounds > kSpinLimit || j < 0)) {
        sm.timed_out = 1;
        break;
      }
    }
    lb[(int64_t)part * kRadix + d] = kFlagPrefix | ((excl + tile_count) & kValueMask);
  }
  sm.global_base[d] = hist_pass[d] + excl;
  __syncthreads();
  if (sm.timed_out) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    return;
  }
  for (int lp = tid; lp < n_here; lp += kSortThreads) {
    const uint32_t dd = sm.dig[lp];
    const uint32_t dst = sm.global_base[dd] + (lp - sm.digit_start[dd]);
    if (dst < (uint64_t)count) kout[dst] = sm.buf[lp];
  }
  __syncthreads();
  // values through the same buffer
  uint32_t* vb = reinterpret_cast<uint32_t*>(sm.buf);
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int64_t p = wbase + 32 * i;
    const uint32_t lp = (rk[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
    if (p < count) vb[lp] = vin[p];
  }
  __syncthreads();
  for (int lp = tid; lp < n_here; lp += kSortThreads) {
    const uint32_t dd = sm.dig[lp];
    const uint32_t dst = sm.global_base[dd] + (lp - sm.digit_start[dd]);
    if (dst < (uint64_t)count) vout[dst] = vb[lp];
  }
}

template <int ITEMS, int MIN_BLOCKS>
static void launch_pass(const SortArgs& a, int pass, int64_t grid, cudaStream_t s) {
  const size_t smem = sizeof(SortSmem<ITEMS>);
  // once per device (the attribute is per device; not repeated inside a graph capture)
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaFuncSetAttribute(onesweep_pass_kernel<ITEMS, MIN_BLOCKS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  onesweep_pass_kernel<ITEMS, MIN_BLOCKS><<<(unsigned)grid, kSortThreads, smem, s>>>(a, pass);
}

void launch_onesweep_pass(const SortArgs& a, int pass, int items, cudaStream_t s) {
  const int64_t grid = sort_partitions(a.capacity, items);
  if (grid <= 0) return;
  switch (items) {
    case 12: launch_pass<12, 4>(a, pass, grid, s); break;
    case 20: launch_pass<20, 3>(a, pass, grid, s); break;
    case 24: launch_pass<24, 2>(a, pass, grid, s); break;
    default: launch_pass<16, 4>(a, pass, grid, s); break;
  }
}

// Exclusive scan of each pass's 256 digit counts, and the pass control
// words (one block of 256 threads, passes in order).
__global__ void __launch_bounds__(kRadix) digit_scan_kernel(const uint32_t* __restrict__ hist,
                                                             const uint64_t* __restrict__ count_ptr,
                                                             int64_t capacity, int npass,
                                                             uint32_t* __restrict__ scanned,
                                                             uint32_t* __restrict__ ctrl) {
  __shared__ uint32_t wsum[kRadix / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t count = (uint32_t)min((int64_t)*count_ptr, capacity);
  uint32_t parity = 0;
  for (int p = 0; p < npass; p++) {
    const uint32_t c = hist[p * kRadix + tid];
    const bool trivial = __syncthreads_or(c == count) != 0;
    uint32_t inc = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < wid; w++) pre += wsum[w];
    scanned[p * kRadix + tid] = pre + inc - c;
    if (tid == 0) ctrl[p] = parity | (trivial ? kCtrlTrivial : 0u);
    if (!trivial) parity ^= 1u;
    __syncthreads();
  }
  if (tid == 0) ctrl[npass] = parity;
}

void launch_digit_histogram(const SortArgs& a, int64_t grid_hint, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (grid_hint + 4095) / 4096;
  const unsigned blocks = (unsigned)(want < 1 ? 1 : (want > (int64_t)sms * 8 ? (int64_t)sms * 8 : want));
  digit_histogram_kernel<<<blocks, 256, 0, s>>>(a.keys[0], a.count, a.capacity, a.npass, a.hist);
  digit_scan_kernel<<<1, kRadix, 0, s>>>(a.hist, a.count, a.capacity, a.npass, a.hist_scan, a.ctrl);
}

// ---------------------------------------------------------------- tile ranges

// ranges[bin] = [first, last + 1) of the bin in the sorted keys; block 0
// also records which buffers hold the sorted list.
__global__ void __launch_bounds__(256) tile_ranges_kernel(SortArgs a, uint2* __restrict__ ranges) {
  const int64_t count = min((int64_t)*a.count, a.capacity);
  const int par = (int)(a.ctrl[a.npass] & kCtrlParity);
  const uint64_t* __restrict__ keys = par ? a.keys[1] : a.keys[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.sorted_keys = keys;
    *a.sorted_vals = par ? a.vals[1] : a.vals[0];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t bin = (uint32_t)(keys[i] >> 32);
    if ((int64_t)bin >= a.bins) continue;  // only after a capacity overflow (reported by the status)
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != bin) ranges[bin].x = (uint32_t)i;
    if (i == count - 1 || (uint32_t)(keys[i + 1] >> 32) != bin) ranges[bin].y = (uint32_t)(i + 1);
  }
}

void launch_tile_ranges(const SortArgs& a, int64_t grid_hint, uint2* ranges, cudaStream_t s) {
  int64_t blocks = (grid_hint + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  tile_ranges_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, ranges);
}

}  // namespace gs
