// Binning: scan of tile counts, a per-view depth sort of the visible
// Gaussians, emission of one instance per touched tile in depth order, a
// stable LSD onesweep radix sort of the instances by tile and per-tile
// ranges.
//
// 3D-GS renders tile by tile from a list sorted by (tile, depth) (Section I).
// Sorting (bin << 32 | depth bits) keys of every instance takes the 32 depth
// bits through every instance, although they are the same for all instances
// of one (view, Gaussian) pair.  Here the depth order is settled once per
// visible pair instead: each view's visible Gaussians (in Gaussian order)
// are sorted by depth bits, the instances are emitted in that order, and a
// stable sort by tile only (2 passes of 8 bits for up to 65,536 tiles per
// view) leaves each tile's list in (depth, Gaussian index) order -- the
// same list as the stable sort of the 64-bit keys.  Depths of visible
// Gaussians are positive FP32 values, so their bit patterns order like the
// values.
//
// Both sorts order each view's segment on its own (the tile sort on bin -
// view's first bin), so the view part of a bin needs no radix pass.
#include <algorithm>

#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

// ---------------------------------------------------------------- scan

// Exclusive scan of the projection's per-(view, block) instance counts: block
// v of the grid scans view v's nb counts (1024 threads looping over chunks)
// and writes the view's total.
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(const uint32_t* __restrict__ sums,
                                                                int64_t nb, uint32_t* __restrict__ offsets,
                                                                uint64_t* __restrict__ view_total) {
  __shared__ uint64_t warp_tot[32];
  __shared__ uint64_t carry;
  const int v = blockIdx.x;
  sums += (int64_t)v * nb;
  offsets += (int64_t)v * nb;
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
  if (threadIdx.x == 0) view_total[v] = carry;
}

// Segment offsets: seg[v] = first instance of view v, seg[B] = *total.
__global__ void segment_offsets_kernel(const uint64_t* __restrict__ view_total, int B, uint32_t* __restrict__ seg,
                                       uint64_t* __restrict__ total) {
  if (threadIdx.x != 0) return;
  uint64_t run = 0;
  for (int v = 0; v < B; v++) {
    seg[v] = (uint32_t)min(run, (uint64_t)0xffffffffu);
    run += view_total[v];
  }
  seg[B] = (uint32_t)min(run, (uint64_t)0xffffffffu);
  *total = run;
}

void launch_scan_block_sums(const uint32_t* sums, int64_t nb, int B, uint32_t* offsets, uint64_t* view_total,
                            uint32_t* seg, uint64_t* total, cudaStream_t s) {
  scan_block_sums_kernel<<<B, 1024, 0, s>>>(sums, nb, offsets, view_total);
  segment_offsets_kernel<<<1, 32, 0, s>>>(view_total, B, seg, total);
}

// ---------------------------------------------------------------- compaction

// Same block partition as the projection (256 Gaussians per block).  Each
// view's visible (view, Gaussian) pairs -- tiles touched > 0 -- are written
// in Gaussian order as (depth bits, Gaussian) into the view's segment of the
// depth sort's input: offset = the view's first pair + the block's scanned
// count + the earlier warps of the block + the lane's rank in the warp.
// Phase 1 takes each warp's ballot per view, phase 2 re-reads the depth bits
// of the visible lanes (the block's own lines, still in cache) and writes.
__global__ void __launch_bounds__(256) compact_kernel(CompactArgs a) {
  __shared__ uint32_t s_mask[kMaxViews][8];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = g < a.n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nb = gridDim.x;
  for (int v = 0; v < a.B; v++) {
    const uint32_t c = live ? a.tiles[(int64_t)v * a.stride + g].x : 0u;
    const unsigned m = __ballot_sync(0xffffffffu, c != 0u);
    if (lane == 0) s_mask[v][wid] = m;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int v = 0; v < a.B; v++) {
    const unsigned m = s_mask[v][wid];
    if (!((m >> lane) & 1u)) continue;
    uint32_t wpre = 0;
    for (int w = 0; w < wid; w++) wpre += __popc(s_mask[v][w]);
    const int64_t pos = (int64_t)a.vseg[v] + a.vis_offsets[(int64_t)v * nb + blockIdx.x] + wpre + __popc(m & lt);
    a.dkeys[pos] = a.tiles[(int64_t)v * a.stride + g].y;
    a.dvals[pos] = (uint32_t)g;
  }
}

void launch_compact(const CompactArgs& a, cudaStream_t s) {
  const int threads = project_fwd_block();
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  compact_kernel<<<blocks, threads, 0, s>>>(a);
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
// a partition that gave up its look-back publishes this instead of a prefix,
// so that the partitions after it give up too instead of scattering with a
// wrong offset
constexpr uint32_t kFlagFailed = 3u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kLookWindow = 16;       // statuses read per look-back round

// Partitions never straddle a view's segment: at most one partial
// partition per segment.
int64_t sort_partitions(int64_t count, int items, int segments) {
  const int64_t tile = (int64_t)kSortThreads * items;
  return (count + tile - 1) / tile + segments;
}

size_t sort_lookback_bytes(int64_t count, int items, int segments) {
  const int64_t parts = sort_partitions(count, items, segments);
  return (size_t)(parts > 0 ? parts : 1) * kRadix * sizeof(uint32_t);
}

// Largest u in [0, B) with off[u] <= i (off nondecreasing): for i below
// off[B], the non-empty segment holding i.
__device__ __forceinline__ int segment_of(const uint32_t* off, int B, uint64_t i) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((uint64_t)off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Partition order of the passes of a sort: ticket t takes partition lp of
// view v, the tickets going round the views (every view's partition 0, then
// every view's partition 1, ...; views out of partitions are passed over).
// The partitions in flight then spread over the views, so a partition's
// look-back -- which stops at its view's first partition -- meets a
// published prefix a few partitions back instead of walking past every
// partition in flight.  Within a view the partitions still take increasing
// tickets, which is all the look-back needs to make progress.
// order[t] = part_off[v] + lp, the partition's status slot.
__global__ void partition_order_kernel(const uint32_t* __restrict__ part_off, int B, uint32_t* __restrict__ order,
                                       int64_t slots) {
  const uint32_t total = part_off[B];
  uint32_t most = 0;
  for (int v = 0; v < B; v++) most = max(most, part_off[v + 1] - part_off[v]);
  for (int64_t ti = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ti < slots && ti < (int64_t)total;
       ti += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)ti;
    // the largest round lo with c(lo) <= t, c(L) = sum_v min(P_v, L) (the
    // tickets of rounds 0 .. L - 1); c(most) = total > t
    uint32_t lo = 0, hi = most;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      uint32_t cm = 0;
      for (int v = 0; v < B; v++) cm += min(part_off[v + 1] - part_off[v], mid);
      if (cm <= t) lo = mid; else hi = mid;
    }
    uint32_t r = t;
    for (int v = 0; v < B; v++) r -= min(part_off[v + 1] - part_off[v], lo);
    // the r-th view, in view order, that still has a partition in round lo
    for (int v = 0; v < B; v++) {
      if (part_off[v + 1] - part_off[v] > lo) {
        if (r == 0) {
          order[t] = part_off[v] + lo;
          break;
        }
        r--;
      }
    }
  }
}

// The key base of segment v: its keys' digits are taken from key - base.
__device__ __forceinline__ uint64_t segment_key_base(const SortArgs& a, int v) {
  return a.views ? (uint64_t)(uint32_t)a.views[v].tile_offset << a.view_shift : 0ull;
}

// Digit counts of every pass of every view in one read of the keys.  hist:
// [B][npass][256], digits of key - segment base.  Block (x, v) counts view
// v's segment with a grid stride over the x blocks of the view, in shared
// memory.  The two top digits vary slowly along the keys (the tile digits
// of instances in emission order, the exponent byte of depths), so their
// counts are first aggregated over the lanes holding the same digit; the
// others are added lane by lane.
template <typename KeyT>
__global__ void __launch_bounds__(256) digit_histogram_kernel(SortArgs a) {
  __shared__ uint32_t sh[8][kRadix];
  for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  const int v = blockIdx.y;
  const int64_t count = min((int64_t)*a.count, a.capacity);
  const int64_t lo = min((int64_t)a.seg[v], count), hi = min((int64_t)a.seg[v + 1], count);
  const KeyT kb = (KeyT)segment_key_base(a, v);
  const KeyT* __restrict__ keys = static_cast<const KeyT*>(a.keys[0]);
  const int npass = a.npass, lane = threadIdx.x & 31;
  for (int64_t i0 = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < hi;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    const bool ok = i < hi;
    const KeyT k = ok ? (KeyT)(keys[i] - kb) : (KeyT)0;
    for (int p = 0; p < npass; p++) {
      const uint32_t dg = (uint32_t)(k >> (kRadixBits * p)) & (kRadix - 1);
      if (p < npass - 2) {
        if (ok) atomicAdd(&sh[p][dg], 1u);
      } else {
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? dg : (uint32_t)kRadix);
        if (ok && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&sh[p][dg], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  uint32_t* h = a.hist + (int64_t)v * npass * kRadix;
  for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x) {
    const uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&h[i], c);
  }
}

// Passes where every view's keys share one digit leave the order unchanged
// and are skipped.  ctrl[p] (written once per sort by digit_scan_kernel):
// bit 0 = which ping-pong buffer holds the keys before pass p (p == npass:
// the sorted result), bit 1 = pass p is skipped.
constexpr uint32_t kCtrlParity = 1u, kCtrlTrivial = 2u;

// One LSD pass, each view's segment sorted on its own: a partition lies in
// one segment; rank its keys by digit of key - segment base (stable), find
// its offset for each digit by decoupled look-back over the earlier
// partitions of its segment (bounded waits), then scatter through shared
// memory so that the global writes are coalesced.  Only the 32-bit word of
// a key that holds the pass's digit is loaded up front (all loads in flight
// before ranking; for 64-bit keys, half the registers of whole keys, which
// spilled); keys and then values go through one shared buffer, and the
// scatter takes each staged key's digit from the key.
template <typename KeyT, int ITEMS>
struct SortSmem {
  static constexpr int kTile = kSortThreads * ITEMS;
  // per-warp digit counts -> position of the warp's first key of the digit
  // in the partition-sorted order
  uint32_t warp_hist[kSortWarps][kRadix];
  // global destination of the digit's first key minus its position in the
  // partition-sorted order (the scatter adds the position)
  uint32_t global_base[kRadix];
  uint32_t wtot[kSortWarps];
  uint32_t part, seg, seg_lo, seg_hi, first_part;
  uint64_t key_base;
  int timed_out;
  KeyT buf[kTile];                         // keys, then values, in tile-sorted order
};

template <typename KeyT, int ITEMS, int MIN_BLOCKS>
__global__ void __launch_bounds__(kSortThreads, MIN_BLOCKS) onesweep_pass_kernel(SortArgs a, int pass) {
  constexpr int kSortItems = ITEMS;
  constexpr int kSortTile = kSortThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<KeyT, ITEMS>& sm = *reinterpret_cast<SortSmem<KeyT, ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t ctrl = a.ctrl[pass];
  if (ctrl & kCtrlTrivial) return;  // whole block: every view has one digit here
  const int par = (int)(ctrl & kCtrlParity);
  // selects, not a dynamically indexed parameter array (which would be
  // copied to local memory)
  const KeyT* __restrict__ kin = static_cast<const KeyT*>(par ? a.keys[1] : a.keys[0]);
  const uint32_t* __restrict__ vin = par ? a.vals[1] : a.vals[0];
  KeyT* __restrict__ kout = static_cast<KeyT*>(par ? a.keys[0] : a.keys[1]);
  uint32_t* __restrict__ vout = par ? a.vals[0] : a.vals[1];
  const int shift = kRadixBits * pass;
  const uint32_t nparts = a.part_off[a.B];
  if (tid == 0) {
    const uint32_t t = atomicAdd(a.counters + pass, 1u);
    const uint32_t part = t < nparts ? (a.part_order ? a.part_order[t] : t) : nparts;  // status slot
    sm.part = part;
    sm.timed_out = 0;
    if (part < nparts) {
      const int u = segment_of(a.part_off, a.B, part);
      const uint32_t cap = (uint32_t)min(a.capacity, (int64_t)0xffffffff);
      sm.seg = (uint32_t)u;
      sm.first_part = a.part_off[u];
      sm.seg_lo = min(a.seg[u], cap);
      sm.seg_hi = min(a.seg[u + 1], cap);
      sm.key_base = segment_key_base(a, u);
    }
  }
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&sm.warp_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t part = sm.part;
  if (part >= nparts) return;
  const int v = (int)sm.seg;
  const uint32_t lp0 = part - sm.first_part;  // partition index inside the segment
  const int64_t base = (int64_t)sm.seg_lo + (int64_t)lp0 * kSortTile;
  const int n_here = (int)min((int64_t)kSortTile, (int64_t)sm.seg_hi - base);
  const KeyT kb = (KeyT)sm.key_base;
  const uint32_t* __restrict__ hist_pass = a.hist_scan + ((int64_t)v * a.npass + pass) * kRadix;
  uint32_t* lookback = a.lookback + (size_t)pass * a.lookback_stride;
  const int wl = wid * kSortItems * 32 + lane;  // item i at base + wl + 32 i

  // the 32-bit word of the key that holds the pass's digit (8-bit digits
  // never straddle the halves of a 64-bit key)
  constexpr int kWords = (int)(sizeof(KeyT) / 4);
  const int hw = kWords == 2 && shift >= 32 ? 1 : 0;
  const int wsh = shift & 31;
  const uint32_t wsub = (uint32_t)((uint64_t)kb >> (32 * hw));
  const uint32_t* __restrict__ kin32 = reinterpret_cast<const uint32_t*>(kin) + hw;
  uint32_t word[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int p = wl + 32 * i;
    word[i] = p < n_here ? kin32[kWords * (base + p)] - wsub : 0u;
  }
  // stable rank inside the warp (warp-striped order), 16-bit per item
  uint32_t rk[kSortItems / 2];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const bool ok = wl + 32 * i < n_here;
    const uint32_t d = ok ? (word[i] >> wsh) & (kRadix - 1) : (uint32_t)kRadix;
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

  // per digit: counts over warps -> warp offsets; publish the partition count
  const uint32_t d = tid;  // kSortThreads == kRadix
  uint32_t tile_count = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; w++) {
    const uint32_t c = sm.warp_hist[w][d];
    sm.warp_hist[w][d] = tile_count;
    tile_count += c;
  }
  volatile uint32_t* lb = lookback;
  lb[(int64_t)part * kRadix + d] = (lp0 == 0 ? kFlagPrefix : kFlagAggregate) | tile_count;
  // digit starts inside the partition (block exclusive scan over the 256
  // digits), folded into the warp offsets and the global bases
  {
    uint32_t inc = tile_count;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) sm.wtot[wid] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; w++) wpre += sm.wtot[w];
    const uint32_t digit_start = wpre + inc - tile_count;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) sm.warp_hist[w][d] += digit_start;
    // (thread d owns entry d; the digit's destination is added after the look-back)
    sm.global_base[d] = 0u - digit_start;
  }
  __syncthreads();
  // keys -> partition-sorted positions in shared memory (before the
  // look-back); remember the positions for the values
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const bool ok = wl + 32 * i < n_here;
    const uint32_t r = (rk[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
    uint32_t lpos = 0xffffu;
    if (ok) {
      const uint32_t dd = (word[i] >> wsh) & (kRadix - 1);
      lpos = sm.warp_hist[wid][dd] + r;
      sm.buf[lpos] = kWords == 1 ? (KeyT)(word[i] + wsub) : kin[base + wl + 32 * i];
    }
    if (i & 1) rk[i >> 1] = (rk[i >> 1] & 0xffffu) | (lpos << 16); else rk[i >> 1] = (rk[i >> 1] & 0xffff0000u) | lpos;
  }
  // decoupled look-back over the earlier partitions of this segment,
  // kLookWindow statuses per round trip; a status that is not ready yet is
  // re-read (bounded)
  uint32_t excl = 0;
  if (lp0 > 0 && a.wait_rounds <= 0) {
    sm.timed_out = 1;  // give up without looking (exercises the timeout path)
    lb[(int64_t)part * kRadix + d] = kFlagFailed;
  } else if (lp0 > 0) {
    const int64_t first = (int64_t)sm.first_part;
    int64_t j = (int64_t)part - 1;
    int rounds = 0;
    bool found = false, failed = false;
    while (!found) {
      uint32_t w[kLookWindow];
#pragma unroll
      for (int t = 0; t < kLookWindow; t++)
        w[t] = (j - t >= first) ? (uint32_t)lb[(j - t) * kRadix + d] : (uint32_t)kFlagPrefix;
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
        if (flag == kFlagFailed) {  // an earlier partition gave up: so does this one
          failed = found = true;
          continue;
        }
        excl += w[t] & kValueMask;
        used++;
        if (flag == kFlagPrefix) found = true;
      }
      j -= used;
      if (!found && ++rounds > a.wait_rounds) {
        failed = true;
        break;
      }
    }
    if (failed) sm.timed_out = 1;
    lb[(int64_t)part * kRadix + d] = failed ? kFlagFailed : (kFlagPrefix | ((excl + tile_count) & kValueMask));
  }
  sm.global_base[d] += sm.seg_lo + hist_pass[d] + excl;
  __syncthreads();
  if (sm.timed_out) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    return;
  }
  // sorted keys out, coalesced; the digit of a staged key is taken from the
  // key itself, and each thread keeps its destinations for the values
  const uint32_t hi = sm.seg_hi;
  uint32_t dst[kSortItems];
#pragma unroll
  for (int t = 0; t < kSortItems; t++) {
    const int q = tid + t * kSortThreads;
    dst[t] = 0xffffffffu;
    if (q < n_here) {
      const KeyT k = sm.buf[q];
      const uint32_t dd = (uint32_t)((KeyT)(k - kb) >> shift) & (kRadix - 1);
      dst[t] = sm.global_base[dd] + (uint32_t)q;
      if (dst[t] < hi) kout[dst[t]] = k;
    }
  }
  __syncthreads();
  // values through the same buffer
  uint32_t* vb = reinterpret_cast<uint32_t*>(sm.buf);
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int p = wl + 32 * i;
    const uint32_t lpos = (rk[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
    if (p < n_here) vb[lpos] = vin[base + p];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kSortItems; t++) {
    const int q = tid + t * kSortThreads;
    if (q < n_here && dst[t] < hi) vout[dst[t]] = vb[q];
  }
}

template <typename KeyT, int ITEMS, int MIN_BLOCKS>
static void launch_pass(const SortArgs& a, int pass, int64_t grid, cudaStream_t s) {
  const size_t smem = sizeof(SortSmem<KeyT, ITEMS>);
  // once per device (the attribute is per device; not repeated inside a graph capture)
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    cudaFuncSetAttribute(onesweep_pass_kernel<KeyT, ITEMS, MIN_BLOCKS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  onesweep_pass_kernel<KeyT, ITEMS, MIN_BLOCKS><<<(unsigned)grid, kSortThreads, smem, s>>>(a, pass);
}

template <typename KeyT>
static void launch_pass_items(const SortArgs& a, int pass, int items, int64_t grid, cudaStream_t s) {
  switch (items) {
    case 12: launch_pass<KeyT, 12, 4>(a, pass, grid, s); break;
    case 20: launch_pass<KeyT, 20, 3>(a, pass, grid, s); break;
    case 24: launch_pass<KeyT, 24, 2>(a, pass, grid, s); break;
    default: launch_pass<KeyT, 16, 4>(a, pass, grid, s); break;
  }
}

void launch_onesweep_pass(const SortArgs& a, int pass, int items, cudaStream_t s) {
  const int64_t grid = sort_partitions(a.capacity, items, a.B);
  if (grid <= 0) return;
  if (a.key_bytes == 4) launch_pass_items<uint32_t>(a, pass, items, grid, s);
  else launch_pass_items<uint64_t>(a, pass, items, grid, s);
}

// Exclusive scan of each (view, pass)'s 256 digit counts (block v of the
// grid: view v), and whether the view's keys share one digit in the pass.
__global__ void __launch_bounds__(kRadix) digit_scan_kernel(SortArgs a) {
  __shared__ uint32_t wsum[kRadix / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int v = blockIdx.x;
  const uint32_t cap = (uint32_t)min(a.capacity, (int64_t)0xffffffff);
  const uint32_t cnt = min(a.seg[v + 1], cap) - min(a.seg[v], cap);
  for (int p = 0; p < a.npass; p++) {
    const int64_t o = ((int64_t)v * a.npass + p) * kRadix + tid;
    const uint32_t c = a.hist[o];
    const bool single = __syncthreads_or(c == cnt) != 0;
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
    a.hist_scan[o] = pre + inc - c;
    if (tid == 0) a.single[v * 8 + p] = single ? 1u : 0u;
    __syncthreads();
  }
}

// Pass control words and the first partition of every view's segment (one
// thread; B <= 64 views, npass <= 8).
__global__ void sort_control_kernel(SortArgs a, int items) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t parity = 0;
  for (int p = 0; p < a.npass; p++) {
    bool trivial = true;
    for (int v = 0; v < a.B; v++) trivial &= a.single[v * 8 + p] != 0;
    a.ctrl[p] = parity | (trivial ? kCtrlTrivial : 0u);
    if (!trivial) parity ^= 1u;
  }
  a.ctrl[a.npass] = parity;
  const uint32_t cap = (uint32_t)min(a.capacity, (int64_t)0xffffffff);
  const uint32_t tile = (uint32_t)(kSortThreads * items);
  uint32_t run = 0;
  for (int v = 0; v < a.B; v++) {
    a.part_off[v] = run;
    const uint32_t cnt = min(a.seg[v + 1], cap) - min(a.seg[v], cap);
    run += (cnt + tile - 1) / tile;
  }
  a.part_off[a.B] = run;
}

void launch_digit_scan(const SortArgs& a, int items, cudaStream_t s) {
  digit_scan_kernel<<<a.B, kRadix, 0, s>>>(a);
  sort_control_kernel<<<1, 32, 0, s>>>(a, items);
  if (a.part_order) {
    const int64_t slots = sort_partitions(a.capacity, items, a.B);
    const int64_t blocks = std::min<int64_t>((slots + 255) / 256, (int64_t)sm_count() * 4);
    partition_order_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a.part_off, a.B, a.part_order,
                                                                               slots);
  }
}

void launch_digit_histogram(const SortArgs& a, int64_t grid_hint, int items, cudaStream_t s) {
  const int sms = sm_count();
  // about 8 blocks per SM over all views, at least one per view
  int64_t want = (grid_hint + 4095) / 4096;
  want = want < 1 ? 1 : (want > (int64_t)sms * 8 ? (int64_t)sms * 8 : want);
  const unsigned per_view = (unsigned)std::max<int64_t>(1, want / a.B);
  if (a.key_bytes == 4) digit_histogram_kernel<uint32_t><<<dim3(per_view, a.B), 256, 0, s>>>(a);
  else digit_histogram_kernel<uint64_t><<<dim3(per_view, a.B), 256, 0, s>>>(a);
  launch_digit_scan(a, items, s);
}

// ---------------------------------------------------------------- emission

// Emission status words (one per partition): flag in the two top bits, the
// partition's instance count (aggregate) or the instances of the segment up
// to and including it (prefix) below.
constexpr uint64_t kEmitAggregate = 1ull << 62;
constexpr uint64_t kEmitPrefix = 2ull << 62;
constexpr uint64_t kEmitFailed = 3ull << 62;
constexpr uint64_t kEmitValue = (1ull << 62) - 1;
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 16;  // visible pairs per thread
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kEmitTile = kEmitThreads * kEmitItems;
constexpr int kEmitChunkLane = kEmitWarps * kEmitItems / 32;  // chunks per lane in the block's chunk scan
static_assert(kEmitWarps * kEmitItems % 32 == 0, "the chunk scan takes whole chunks per lane");

int64_t emit_partitions(int64_t pairs, int segments) { return (pairs + kEmitTile - 1) / kEmitTile + segments; }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// One partition of kEmitTile depth-sorted visible pairs of one view per
// block (partitions taken by ticket, so every earlier partition is running
// or done).  Warp w holds chunks of 32 consecutive pairs; each pair's tile
// rect comes from its (view, Gaussian) entry.  The block scans the chunks'
// instance counts, warp 0 finds the instances of the view's earlier
// partitions by decoupled look-back (32 statuses per round, bounded waits),
// and each lane writes its pair's (tile, Gaussian) instances, tiles of a
// rect in row-major order.  The tile digits of the following sort are
// counted on the way (shared memory, one flush per block).
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(EmitArgs a) {
  __shared__ uint32_t s_part[kMaxViews + 1];
  __shared__ uint32_t s_chunk[kEmitWarps * kEmitItems];
  __shared__ uint32_t s_hist[4][kRadix];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_ticket, s_total;
  __shared__ int s_failed;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < 4 * kRadix; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
  if (wid == 0) {
    // partitions per view (B <= 64: lanes take views lane and lane + 32)
    uint32_t c[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int v = lane + 32 * h;
      c[h] = v < a.B ? (a.vseg[v + 1] - a.vseg[v] + kEmitTile - 1) / kEmitTile : 0u;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      uint32_t inc = c[h];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      const int v = lane + 32 * h;
      if (v <= a.B) s_part[v] = carry + inc - c[h];
      if (v + 1 == a.B) s_part[a.B] = carry + inc;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) s_ticket = atomicAdd(a.counter, 1u);
  }
  __syncthreads();
  const uint32_t part = s_ticket;
  if (part >= s_part[a.B]) return;
  const int v = segment_of(s_part, a.B, part);
  const uint32_t lp = part - s_part[v];
  const int64_t lo = (int64_t)a.vseg[v] + (int64_t)lp * kEmitTile;
  const int n_here = (int)min((int64_t)kEmitTile, (int64_t)a.vseg[v + 1] - lo);
  const uint32_t* __restrict__ src = (a.dctrl[a.dpass] & kCtrlParity) ? a.dvals[1] : a.dvals[0];
  const int4* __restrict__ rec3 = a.rec3 + (int64_t)v * a.stride;

  uint32_t gi[kEmitItems], rx[kEmitItems], ry[kEmitItems], cnt[kEmitItems];
#pragma unroll
  for (int r = 0; r < kEmitItems; r++) {
    const int p = (wid * kEmitItems + r) * 32 + lane;
    gi[r] = 0u;
    rx[r] = ry[r] = cnt[r] = 0u;
    if (p < n_here) gi[r] = src[lo + p];
  }
#pragma unroll
  for (int r = 0; r < kEmitItems; r++) {
    const int p = (wid * kEmitItems + r) * 32 + lane;
    // (an index at or above n only comes from a depth sort that gave up)
    if (p < n_here && (int64_t)gi[r] < a.n) {
      const int4 e = rec3[gi[r]];
      cnt[r] = (uint32_t)e.y;
      rx[r] = (uint32_t)e.z;
      ry[r] = (uint32_t)e.w;
    }
  }
#pragma unroll
  for (int r = 0; r < kEmitItems; r++) {
    const uint32_t t = __reduce_add_sync(0xffffffffu, cnt[r]);
    if (lane == 0) s_chunk[wid * kEmitItems + r] = t;
  }
  __syncthreads();
  if (wid == 0) {
    // exclusive scan of the block's chunk counts (kEmitChunkLane consecutive chunks per lane)
    uint32_t cc[kEmitChunkLane], t = 0;
#pragma unroll
    for (int i = 0; i < kEmitChunkLane; i++) {
      cc[i] = s_chunk[kEmitChunkLane * lane + i];
      t += cc[i];
    }
    uint32_t inc = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    uint32_t run = inc - t;
#pragma unroll
    for (int i = 0; i < kEmitChunkLane; i++) {
      s_chunk[kEmitChunkLane * lane + i] = run;
      run += cc[i];
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    volatile uint64_t* lb = a.lookback;
    if (lane == 0) lb[part] = (lp == 0 ? kEmitPrefix : kEmitAggregate) | (uint64_t)total;
    uint64_t excl = 0;
    bool failed = false;
    if (lp > 0 && a.wait_rounds <= 0) {
      failed = true;  // give up without looking (exercises the timeout path)
    } else if (lp > 0) {
      const int64_t first = (int64_t)s_part[v];
      int64_t j = (int64_t)part - 1;
      int rounds = 0;
      while (true) {
        const int64_t q = j - lane;
        const uint64_t w = q >= first ? (uint64_t)lb[q] : (uint64_t)kEmitPrefix;
        const uint32_t flag = (uint32_t)(w >> 62);
        const unsigned waiting = __ballot_sync(0xffffffffu, flag == 0u);
        const unsigned stops = __ballot_sync(0xffffffffu, flag >= 2u);
        const int first_wait = waiting ? __ffs(waiting) - 1 : 32;
        const int first_stop = stops ? __ffs(stops) - 1 : 32;
        if (first_stop < first_wait) {
          const bool take = lane <= first_stop;
          failed = __any_sync(0xffffffffu, take && flag == 3u) != 0;
          excl += warp_sum_u64(take ? (w & kEmitValue) : 0ull);
          break;
        }
        excl += warp_sum_u64(lane < first_wait ? (w & kEmitValue) : 0ull);
        j -= first_wait;
        if (++rounds > a.wait_rounds) {
          failed = true;
          break;
        }
      }
    }
    if (lane == 0) {
      if (lp > 0) lb[part] = failed ? kEmitFailed : (kEmitPrefix | ((excl + total) & kEmitValue));
      s_base = excl;
      s_total = total;
      s_failed = failed ? 1 : 0;
    }
  }
  __syncthreads();
  if (s_failed) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    return;
  }
  const int64_t gbase = (int64_t)a.seg[v] + (int64_t)s_base;
  if (gbase + (int64_t)s_total > a.capacity) {
    if (tid == 0) atomicOr(a.status, kStatusCapacity);
    return;
  }
  const ViewRec& V = a.views[v];
  const uint32_t gw = (uint32_t)V.gw, toff = (uint32_t)V.tile_offset;
  const int tpass = a.tpass;
#pragma unroll
  for (int r = 0; r < kEmitItems; r++) {
    const uint32_t c = cnt[r];
    uint32_t inc = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    // each lane writes its own pair's tiles, row by row, at the pair's
    // offset in the chunk (pairs average under two tiles: the lanes' short
    // runs are adjacent, so the stores of one step still fall in a few
    // sectors, and no owner search or division per instance is needed);
    // a pair of more than 32 tiles is expanded by the whole warp below
    const int64_t o0 = gbase + s_chunk[wid * kEmitItems + r] + (inc - c);
    const uint32_t x0 = rx[r] & 0xffffu, x1 = rx[r] >> 16;
    const uint32_t t0 = (ry[r] & 0xffffu) * gw + x0;
    const bool big = c > 32u;
    {
      int64_t o = o0;
      uint32_t tx = x0, t = t0;
      for (uint32_t k = 0; k < (big ? 0u : c); k++) {
        a.keys[o] = toff + t;
        a.vals[o] = gi[r];
        o++;
        atomicAdd(&s_hist[0][t & (kRadix - 1)], 1u);
        for (int p = 1; p < tpass; p++) atomicAdd(&s_hist[p][(t >> (kRadixBits * p)) & (kRadix - 1)], 1u);
        if (++tx == x1) {  // next row of the rect
          tx = x0;
          t += gw - (x1 - x0) + 1;
        } else {
          t++;
        }
      }
    }
    for (unsigned bigs = __ballot_sync(0xffffffffu, big); bigs; bigs &= bigs - 1u) {
      const int src = __ffs(bigs) - 1;
      const uint32_t bc = __shfl_sync(0xffffffffu, c, src);
      const int64_t bo = __shfl_sync(0xffffffffu, o0, src);
      const uint32_t bx0 = __shfl_sync(0xffffffffu, x0, src), bw = __shfl_sync(0xffffffffu, x1, src) - bx0;
      const uint32_t bt0 = __shfl_sync(0xffffffffu, t0, src), bg = __shfl_sync(0xffffffffu, gi[r], src);
      for (uint32_t q0 = 0; q0 < bc; q0 += 32) {
        const uint32_t q = q0 + lane;
        if (q < bc) {
          const uint32_t t = bt0 + (q / bw) * gw + q % bw;
          a.keys[bo + q] = toff + t;
          a.vals[bo + q] = bg;
          atomicAdd(&s_hist[0][t & (kRadix - 1)], 1u);
          for (int p = 1; p < tpass; p++) atomicAdd(&s_hist[p][(t >> (kRadixBits * p)) & (kRadix - 1)], 1u);
        }
      }
    }
  }
  __syncthreads();
  uint32_t* h = a.hist + (int64_t)v * tpass * kRadix;
  for (int i = tid; i < tpass * kRadix; i += kEmitThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(&h[i], c);
  }
}

void launch_emit(const EmitArgs& a, int64_t pair_capacity, cudaStream_t s) {
  const int64_t grid = emit_partitions(pair_capacity, a.B);
  if (grid <= 0) return;
  emit_kernel<<<(unsigned)grid, kEmitThreads, 0, s>>>(a);
}

size_t emit_lookback_bytes(int64_t pair_capacity, int segments) {
  return (size_t)emit_partitions(pair_capacity, segments) * sizeof(uint64_t);
}

// ---------------------------------------------------------------- tile ranges

// ranges[bin] = [first, last + 1) of the bin in the sorted instance keys
// (32-bit bins); block 0 also records which buffers hold the sorted list.
// Each key is loaded once: a lane compares its bin with its neighbours'
// through shuffles (the warp's edge lanes load one neighbour each).
__global__ void __launch_bounds__(256) tile_ranges_kernel(SortArgs a, uint2* __restrict__ ranges) {
  const int64_t count = min((int64_t)*a.count, a.capacity);
  const int par = (int)(a.ctrl[a.npass] & kCtrlParity);
  const uint32_t* __restrict__ keys = static_cast<const uint32_t*>(par ? a.keys[1] : a.keys[0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.sorted_keys = keys;
    *a.sorted_vals = par ? a.vals[1] : a.vals[0];
  }
  const int lane = threadIdx.x & 31;
  const uint32_t none = 0xffffffffu;
  // a warp takes 128 consecutive keys per round: four loads in flight per
  // lane, neighbours across the four chunks by shuffles
  constexpr int U = 4;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = warp * 32 * U; w0 < count; w0 += nwarps * 32 * U) {
    uint32_t bin[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = w0 + 32 * u + lane;
      bin[u] = i < count ? keys[i] : none;
    }
    const uint32_t before = (lane == 0 && w0 > 0) ? keys[w0 - 1] : none;
    const uint32_t after = (lane == 31 && w0 + 32 * U < count) ? keys[w0 + 32 * U] : none;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = w0 + 32 * u + lane;
      uint32_t prev = __shfl_up_sync(0xffffffffu, bin[u], 1);
      uint32_t next = __shfl_down_sync(0xffffffffu, bin[u], 1);
      const uint32_t prev_chunk = __shfl_sync(0xffffffffu, u > 0 ? bin[u > 0 ? u - 1 : 0] : none, 31);
      const uint32_t next_chunk = __shfl_sync(0xffffffffu, u < U - 1 ? bin[u < U - 1 ? u + 1 : 0] : none, 0);
      if (lane == 0) prev = u > 0 ? prev_chunk : before;
      if (lane == 31) next = u < U - 1 ? next_chunk : after;
      if (i >= count || (int64_t)bin[u] >= a.bins) continue;  // (bins only overflow after a capacity overflow)
      if (prev != bin[u]) ranges[bin[u]].x = (uint32_t)i;
      if (next != bin[u]) ranges[bin[u]].y = (uint32_t)(i + 1);
    }
  }
}

// ---------------------------------------------------------------- tile order

// Keys of the longest-list-first order: tiles bucketed by floor(log2(length
// + 1)), longest bucket first (a stable sort keeps bin order inside a bucket,
// so the order is deterministic); block 0 also writes the sort's count and
// segment bounds.
__global__ void __launch_bounds__(256) tile_order_keys_kernel(const uint2* __restrict__ ranges, int64_t bins,
                                                              uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                              uint64_t* count, uint32_t* seg) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    *count = (uint64_t)bins;
    seg[0] = 0u;
    seg[1] = (uint32_t)bins;
  }
  if (b >= bins) return;
  const uint2 r = ranges[b];
  const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
  keys[b] = (uint64_t)(31 - (31 - __clz(len + 1u)));
  vals[b] = (uint32_t)b;
}

__global__ void __launch_bounds__(256) tile_order_finish_kernel(const uint32_t* __restrict__ ctrl, int npass,
                                                                const uint32_t* __restrict__ v0,
                                                                const uint32_t* __restrict__ v1, int64_t bins,
                                                                uint32_t* __restrict__ order) {
  const uint32_t* src = (ctrl[npass] & kCtrlParity) ? v1 : v0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < bins; b += (int64_t)gridDim.x * blockDim.x)
    order[b] = src[b];
}

void launch_tile_order_keys(const uint2* ranges, int64_t bins, uint64_t* keys, uint32_t* vals, uint64_t* count,
                            uint32_t* seg, cudaStream_t s) {
  tile_order_keys_kernel<<<(unsigned)((bins + 255) / 256), 256, 0, s>>>(ranges, bins, keys, vals, count, seg);
}

void launch_tile_order_finish(const uint32_t* ctrl, int npass, const uint32_t* v0, const uint32_t* v1, int64_t bins,
                              uint32_t* order, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((bins + 255) / 256, (int64_t)sm_count() * 8);
  tile_order_finish_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(ctrl, npass, v0, v1, bins, order);
}

void launch_tile_ranges(const SortArgs& a, int64_t grid_hint, uint2* ranges, cudaStream_t s) {
  int64_t blocks = (grid_hint + 255) / 256;
  const int64_t most = (int64_t)sm_count() * 32;
  if (blocks > most) blocks = most;
  if (blocks < 1) blocks = 1;
  tile_ranges_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, ranges);
}

}  // namespace gs
