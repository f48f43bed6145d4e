// Point-cloud initialisation of the Gaussians on the GPU: isosurface edge
// crossings of a volume and k-nearest-neighbour scales.
//
// The paper starts 3D-GS from the isosurface of a scientific volume,
// extracted as a point cloud instead of SfM points (Method Overview).  The
// crossings are the contour filter's vertices: every grid edge whose end
// values lie on different sides of the level gives the linearly
// interpolated point, with the volume gradient (central differences,
// one-sided at the border) interpolated the same way as its normal, emitted
// in vertex order (x fastest, then y, then z; per vertex its +x, +y, +z
// edges).  Each Gaussian's initial scale is log sqrt of the mean squared
// distance to its k nearest other points, found exactly with a uniform grid:
// points are sorted by cell (the onesweep radix sort), cell starts go into
// an open-addressing table, and each query examines growing cubes of cells
// until the k-th distance lies inside the examined radius.
#include <cmath>

#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

// ---------------------------------------------------------------- crossings

namespace {

__device__ __forceinline__ float vol_at(const IsoArgs& a, int x, int y, int z) {
  return __ldg(a.vol + ((int64_t)z * a.ny + y) * a.nx + x);
}

// Gradient of the volume at a vertex: central differences inside, one-sided
// at the border (0 along an axis of one sample).
__device__ __forceinline__ float3 vol_grad(const IsoArgs& a, int x, int y, int z) {
  float3 g;
  const int xm = max(x - 1, 0), xp = min(x + 1, a.nx - 1);
  const int ym = max(y - 1, 0), yp = min(y + 1, a.ny - 1);
  const int zm = max(z - 1, 0), zp = min(z + 1, a.nz - 1);
  g.x = xp > xm ? (vol_at(a, xp, y, z) - vol_at(a, xm, y, z)) / ((float)(xp - xm) * a.h[0]) : 0.f;
  g.y = yp > ym ? (vol_at(a, x, yp, z) - vol_at(a, x, ym, z)) / ((float)(yp - ym) * a.h[1]) : 0.f;
  g.z = zp > zm ? (vol_at(a, x, y, zp) - vol_at(a, x, y, zm)) / ((float)(zp - zm) * a.h[2]) : 0.f;
  return g;
}

// Crossing edges of vertex v: bit d set for the +x (0), +y (1), +z (2) edge.
__device__ __forceinline__ uint32_t crossing_edges(const IsoArgs& a, int64_t v, int& x, int& y, int& z) {
  x = (int)(v % a.nx);
  y = (int)((v / a.nx) % a.ny);
  z = (int)(v / ((int64_t)a.nx * a.ny));
  const bool in = vol_at(a, x, y, z) >= a.iso;
  uint32_t e = 0;
  if (x + 1 < a.nx && (vol_at(a, x + 1, y, z) >= a.iso) != in) e |= 1u;
  if (y + 1 < a.ny && (vol_at(a, x, y + 1, z) >= a.iso) != in) e |= 2u;
  if (z + 1 < a.nz && (vol_at(a, x, y, z + 1) >= a.iso) != in) e |= 4u;
  return e;
}

// Exclusive prefix of `c` over the block (256 threads); *total = block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t c, uint32_t* warp_tot, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  uint32_t pre = 0, all = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
    pre += w < wid ? warp_tot[w] : 0u;
    all += warp_tot[w];
  }
  *total = all;
  return pre + inc - c;
}

}  // namespace

__global__ void __launch_bounds__(256) iso_count_kernel(IsoArgs a) {
  __shared__ uint32_t warp_tot[8];
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  const uint32_t c = v < a.nverts ? (uint32_t)__popc(crossing_edges(a, v, x, y, z)) : 0u;
  uint32_t tot;
  block_excl_scan(c, warp_tot, &tot);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) iso_emit_kernel(IsoArgs a) {
  __shared__ uint32_t warp_tot[8];
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int x = 0, y = 0, z = 0;
  const uint32_t e = v < a.nverts ? crossing_edges(a, v, x, y, z) : 0u;
  uint32_t tot;
  const uint32_t pre = block_excl_scan((uint32_t)__popc(e), warp_tot, &tot);
  if (!e) return;
  int64_t o = (int64_t)a.block_offsets[blockIdx.x] + pre;
  if (o + __popc(e) > a.capacity) {
    atomicOr(a.status, kStatusCapacity);
    return;
  }
  const float fa = vol_at(a, x, y, z);
  const float3 ga = vol_grad(a, x, y, z);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (!((e >> d) & 1u)) continue;
    const int x2 = x + (d == 0), y2 = y + (d == 1), z2 = z + (d == 2);
    const float fb = vol_at(a, x2, y2, z2);
    const float t = (a.iso - fa) / (fb - fa);
    const float3 gb = vol_grad(a, x2, y2, z2);
    float* p = a.points + 3 * o;
    p[0] = a.origin[0] + a.h[0] * ((float)x + (d == 0 ? t : 0.f));
    p[1] = a.origin[1] + a.h[1] * ((float)y + (d == 1 ? t : 0.f));
    p[2] = a.origin[2] + a.h[2] * ((float)z + (d == 2 ? t : 0.f));
    float nx = fmaf(t, gb.x - ga.x, ga.x), ny = fmaf(t, gb.y - ga.y, ga.y), nz = fmaf(t, gb.z - ga.z, ga.z);
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    const float inv = len > 0.f ? 1.f / len : 0.f;
    float* q = a.normals + 3 * o;
    q[0] = nx * inv;
    q[1] = ny * inv;
    q[2] = len > 0.f ? nz * inv : 1.f;
    o++;
  }
}

void launch_iso(const IsoArgs& a, bool emit, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.nverts + 255) / 256);
  if (blocks == 0) return;
  if (emit) iso_emit_kernel<<<blocks, 256, 0, s>>>(a);
  else iso_count_kernel<<<blocks, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- k nearest neighbours

// Per-block bounds of the points (6 floats: min xyz, max xyz), then one
// block combines them.
__global__ void __launch_bounds__(256) knn_bounds_kernel(const float* __restrict__ pts, int64_t n,
                                                         float* __restrict__ part) {
  __shared__ float red[6][8];
  float b[6] = {3.0e38f, 3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const float v = pts[3 * i + d];
      b[d] = fminf(b[d], v);
      b[3 + d] = fmaxf(b[3 + d], v);
    }
#pragma unroll
  for (int d = 0; d < 6; d++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float o = __shfl_down_sync(0xffffffffu, b[d], off);
      b[d] = d < 3 ? fminf(b[d], o) : fmaxf(b[d], o);
    }
    if ((threadIdx.x & 31) == 0) red[d][threadIdx.x >> 5] = b[d];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int d = threadIdx.x;
    float v = red[d][0];
    for (int w = 1; w < 8; w++) v = d < 3 ? fminf(v, red[d][w]) : fmaxf(v, red[d][w]);
    part[6 * (int64_t)blockIdx.x + d] = v;
  }
}

__global__ void knn_bounds_finish_kernel(const float* __restrict__ part, int nparts, float* __restrict__ out) {
  if (threadIdx.x >= 6) return;
  const int d = threadIdx.x;
  float v = part[d];
  for (int b = 1; b < nparts; b++) v = d < 3 ? fminf(v, part[6 * b + d]) : fmaxf(v, part[6 * b + d]);
  out[d] = v;
}

namespace {

__device__ __forceinline__ void cell_of(const KnnArgs& a, float x, float y, float z, int& cx, int& cy, int& cz) {
  cx = min(max((int)((x - a.lo[0]) * a.inv_cell), 0), a.dims[0] - 1);
  cy = min(max((int)((y - a.lo[1]) * a.inv_cell), 0), a.dims[1] - 1);
  cz = min(max((int)((z - a.lo[2]) * a.inv_cell), 0), a.dims[2] - 1);
}

__device__ __forceinline__ uint64_t cell_id(const KnnArgs& a, int cx, int cy, int cz) {
  return ((uint64_t)cz * (uint64_t)a.dims[1] + (uint64_t)cy) * (uint64_t)a.dims[0] + (uint64_t)cx;
}

__device__ __forceinline__ uint64_t slot_of(uint64_t key, int bits) {
  return (key * 0x9E3779B97F4A7C15ull) >> (64 - bits);
}

constexpr uint64_t kEmptySlot = ~0ull;

// First sorted position of a cell, or -1 when no point lies in it.
__device__ __forceinline__ int64_t cell_start(const KnnArgs& a, uint64_t key) {
  const uint64_t mask = (1ull << a.table_bits) - 1ull;
  for (uint64_t s = slot_of(key, a.table_bits), probes = 0; probes <= mask; s = (s + 1) & mask, probes++) {
    const uint64_t k = a.table_keys[s];
    if (k == key) return (int64_t)a.table_start[s];
    if (k == kEmptySlot) return -1;
  }
  return -1;
}

}  // namespace

__global__ void __launch_bounds__(256) knn_cell_keys_kernel(KnnArgs a, uint64_t* __restrict__ keys,
                                                            uint32_t* __restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_of(a, a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2], cx, cy, cz);
    keys[i] = cell_id(a, cx, cy, cz);
    vals[i] = (uint32_t)i;
  }
}

// Insert the first sorted position of every cell into the table.
__global__ void __launch_bounds__(256) knn_cell_table_kernel(KnnArgs a) {
  const uint64_t mask = (1ull << a.table_bits) - 1ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = a.skeys[i];
    if (i > 0 && a.skeys[i - 1] == key) continue;
    for (uint64_t s = slot_of(key, a.table_bits), probes = 0; probes <= mask; s = (s + 1) & mask, probes++) {
      const unsigned long long prev =
          atomicCAS(reinterpret_cast<unsigned long long*>(a.table_keys + s), (unsigned long long)kEmptySlot,
                    (unsigned long long)key);
      if (prev == kEmptySlot) {
        a.table_start[s] = (uint32_t)i;
        break;
      }
    }
  }
}

// One thread per point (in cell order): the k smallest squared distances to
// other points over cubes of (2 r + 1)^3 cells, r = 1, 2, ..., until the
// k-th lies within r cells (every point closer than r cell widths lies in
// the cube), then out[point] = 0.5 log(max(1e-14, mean)).
__global__ void __launch_bounds__(256) knn_query_kernel(KnnArgs a) {
  constexpr int KMAX = 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t me = a.svals[i];
    const float px = a.pts[3 * me], py = a.pts[3 * me + 1], pz = a.pts[3 * me + 2];
    int cx, cy, cz;
    cell_of(a, px, py, pz, cx, cy, cz);
    float best[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; k++) best[k] = 3.0e38f;
    const int maxr = max(a.dims[0], max(a.dims[1], a.dims[2]));
    for (int r = 1; r <= maxr; r++) {
      for (int dz = -r; dz <= r; dz++)
        for (int dy = -r; dy <= r; dy++)
          for (int dx = -r; dx <= r; dx++) {
            // only the shell of the cube: the inside was examined with r - 1
            if (r > 1 && max(abs(dx), max(abs(dy), abs(dz))) < r) continue;
            const int x = cx + dx, y = cy + dy, z = cz + dz;
            if (x < 0 || y < 0 || z < 0 || x >= a.dims[0] || y >= a.dims[1] || z >= a.dims[2]) continue;
            const uint64_t key = cell_id(a, x, y, z);
            const int64_t s0 = cell_start(a, key);
            if (s0 < 0) continue;
            for (int64_t j = s0; j < a.n && a.skeys[j] == key; j++) {
              const uint32_t o = a.svals[j];
              if (o == me) continue;
              const float ex = a.pts[3 * o] - px, ey = a.pts[3 * o + 1] - py, ez = a.pts[3 * o + 2] - pz;
              float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
              // insert into the sorted list of the k best
#pragma unroll
              for (int k = 0; k < KMAX; k++) {
                if (k < a.k && d2 < best[k]) {
                  const float t = best[k];
                  best[k] = d2;
                  d2 = t;
                }
              }
            }
          }
      // (with a margin for the rounding of the cell coordinates)
      const float reach = (float)r * a.cell * 0.999f;
      if (best[a.k - 1] <= reach * reach) break;
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; k++) sum += k < a.k ? best[k] : 0.f;
    a.out[me] = 0.5f * logf(fmaxf(sum / (float)a.k, 1e-14f));
  }
}

void launch_knn_bounds(const float* pts, int64_t n, float* part, int nparts, float* out, cudaStream_t s) {
  knn_bounds_kernel<<<nparts, 256, 0, s>>>(pts, n, part);
  knn_bounds_finish_kernel<<<1, 32, 0, s>>>(part, nparts, out);
}

void launch_knn_keys(const KnnArgs& a, uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((a.n + 255) / 256, (int64_t)sm_count() * 32);
  knn_cell_keys_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a, keys, vals);
}

void launch_knn_query(const KnnArgs& a, cudaStream_t s) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, (int64_t)sm_count() * 32));
  knn_cell_table_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  knn_query_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- initial parameters

// Parameter planes of the initial Gaussians: mean = point, log-scales
// (s, s, s + log flatten), rotation taking +z onto the normal, the given
// opacity logit, SH DC of the Lambertian grey under the light (1,1,1)/sqrt 3,
// higher SH 0.  sel (optional) picks the points.
__global__ void __launch_bounds__(256) init_params_kernel(InitArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const int64_t S = a.stride;
  float* P = a.params;
  const int64_t src = a.sel ? a.sel[g] : g;
  const float nx = a.normals[3 * src], ny = a.normals[3 * src + 1], nz = a.normals[3 * src + 2];
#pragma unroll
  for (int d = 0; d < 3; d++) P[d * S + g] = a.points[3 * src + d];
  const float s = a.log_scales[g];
  P[3 * S + g] = s;
  P[4 * S + g] = s;
  P[5 * S + g] = s + a.log_flatten;
  float qw = 1.f + nz, qx = -ny, qy = nx, qz = 0.f;
  if (qw < 1e-6f) {
    qw = 0.f;
    qx = 1.f;
    qy = 0.f;
  }
  const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  P[6 * S + g] = qw * inv;
  P[7 * S + g] = qx * inv;
  P[8 * S + g] = qy * inv;
  P[9 * S + g] = qz * inv;
  P[10 * S + g] = a.opacity_logit;
  const float c = 0.1f + 0.9f * fmaxf(0.f, (nx + ny + nz) * 0.57735026918962576f);
  const float dc = (c - 0.5f) * 3.5449077018110318f;  // 2 sqrt(pi)
  for (int k = 0; k < a.planes - 11; k++) P[(11 + k) * S + g] = k < 3 ? dc : 0.f;
}

// Gather the selected points (for the neighbour search, which runs on the
// selected set).
__global__ void __launch_bounds__(256) init_gather_kernel(const float* __restrict__ pts,
                                                          const int64_t* __restrict__ sel, int64_t n,
                                                          float* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int64_t s = sel[g];
#pragma unroll
  for (int d = 0; d < 3; d++) out[3 * g + d] = pts[3 * s + d];
}

void launch_init_params(const InitArgs& a, cudaStream_t s) {
  if (a.n <= 0) return;
  init_params_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
}

void launch_init_gather(const float* pts, const int64_t* sel, int64_t n, float* out, cudaStream_t s) {
  if (n <= 0) return;
  init_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, sel, n, out);
}

}  // namespace gs
