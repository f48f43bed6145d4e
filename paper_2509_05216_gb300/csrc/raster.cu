// Per-tile front-to-back alpha compositing (forward) and its reverse-order
// backward pass.
//
// 3D-GS composites each pixel over its tile's depth-sorted list (the paper
// trains that renderer, Section I/III): alpha = min(0.99, opacity *
// exp(power)), skip if power > 0 or alpha < 1/255, stop before a Gaussian
// that would bring T below 1e-4.  The backward pass walks the same list from
// each pixel's last contributor towards the front, recovering T by division
// and keeping the colour composited behind.
//
// Two launch shapes, selected per context (GS_OPT_RASTER_*):
//  * block per tile (PPT = 1, 2, 4 pixels per thread): 256 / PPT threads;
//    warp w covers an 8-pixel-wide band of 4 * PPT rows of the tile;
//  * warp per tile (PPT = 8): lane l owns column l & 15 and 8 rows.
// A staged Gaussian carries the half-extents of the ellipse on which
// alpha = 1/255 (slightly widened); a warp whose pixel rectangle misses that
// box skips the Gaussian with one uniform branch.  This removes only pairs
// that the per-pixel test would skip, so the result is unchanged.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ int view_of_bin(const ViewRec* views, int B, int bin) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_offset <= bin) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Staged Gaussian (shared memory, three float4):
//   s0 = (mu_x, mu_y, cA, cB), s1 = (cC, opacity, r, g), s2 = (b, hx, hy, -)
// with p2 = cA dx^2 + cB dx dy + cC dy^2 = power * log2(e), dx = mu_x - x.
__device__ __forceinline__ void stage_one(const RasterArgs& a, int v, uint32_t g, float4& s0, float4& s1,
                                          float4& s2) {
  const int64_t o = (int64_t)v * a.stride + g;
  const float4 r0 = a.rec0[o], r1 = a.rec1[o];
  const float blue = a.rec2[o].x;
  const float A = r0.z, B = r0.w, C = r1.x, op = r1.y;
  // alpha >= 1/255  <=>  d^T K d <= tau = 2 ln(255 opacity); the ellipse's
  // bounding box has half-extents sqrt(tau * (K^-1)_xx), sqrt(tau * (K^-1)_yy).
  const float detK = A * C - B * B;
  float hx = 3.0e38f, hy = 3.0e38f;
  const float t = 255.f * op;
  if (t <= 1.f) {
    hx = hy = -3.0e38f;  // never reaches 1/255: no box is hit
  } else if (detK > 0.f) {
    const float tau = 2.f * __logf(t) * 1.001f + 1e-3f;
    hx = sqrtf(tau * C / detK) * 1.001f + 0.01f;
    hy = sqrtf(tau * A / detK) * 1.001f + 0.01f;
  }
  s0 = make_float4(r0.x, r0.y, -0.5f * kLog2e * A, -kLog2e * B);
  s1 = make_float4(-0.5f * kLog2e * C, op, r1.z, r1.w);
  s2 = make_float4(blue, hx, hy, 0.f);
}

// Does the splat's alpha >= 1/255 box meet the pixel rectangle [x0,x1]x[y0,y1]?
__device__ __forceinline__ bool box_hits(const float4& s0, const float4& s2, float x0, float x1, float y0,
                                         float y1) {
  return s0.x + s2.y >= x0 && s0.x - s2.y <= x1 && s0.y + s2.z >= y0 && s0.y - s2.z <= y1;
}

// p2 at row offset dy = mu_y - y for a lane with column coefficients
// a0 = cA dx^2, a1 = cB dx.  Every kernel variant, forward and backward,
// evaluates it with the same instructions on the same operands for a given
// pixel, so their skip decisions agree.
__device__ __forceinline__ float splat_p2(float cC, float a1, float a0, float dy) {
  return __fmaf_rn(__fmaf_rn(cC, dy, a1), dy, a0);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float splat_alpha2(float op, float p2, float& G) {
  G = ex2_approx(p2);
  return fminf(kAlphaClamp, __fmul_rn(op, G));
}

// Sum 16 per-lane values over the warp, reduce-scatter style: afterwards
// lanes 2q and 2q+1 hold the total of value q (16 shuffles instead of 80).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int off = 16, half = 8; off >= 2; off >>= 1, half >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; i++) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Apply the warp's reduced gradient of one Gaussian: lanes 2q (q < 9) add
// the total of value q.  Accumulators hold d/d(mu_x, mu_y) of p2 and raw
// dx^2, dx dy, dy^2 sums; undo those scalings here.
__device__ __forceinline__ void push_grad(float4* g2d, int64_t rec, float (&acc)[16], int lane) {
  const float tot = warp_reduce_scatter16(acc, lane);
  const int q = lane >> 1;
  if ((lane & 1) == 0 && q < 9) {
    const float scale = q < 2 ? (1.f / kLog2e) : (q == 2 || q == 4) ? -0.5f : (q == 3 ? -1.f : 1.f);
    atomicAdd(reinterpret_cast<float*>(g2d + rec * 3) + q, tot * scale);
  }
}

// One backward (pixel, Gaussian) pair, branch-free so that the pixels of a
// thread interleave.  `live` says the pair lies before the pixel's last
// contributor.  T is the transmittance behind the Gaussian on entry and in
// front of it on exit; dCS = sum_c dL/dC_c S_c with S the colour composited
// behind.  Skipped pairs leave every value unchanged.  Returns whether the
// pair contributed.
__device__ __forceinline__ bool bwd_pair(bool live, const float4& q0, const float4& q1, const float (&rgb)[3],
                                         float a0, float a1, float dy, float dx, float dx2, float cA2dx, float cBdx,
                                         float& T, float& dCS, const float (&dC)[3], float bgd, float (&acc)[16]) {
  const float p2 = splat_p2(q1.x, a1, a0, dy);
  float G;
  const float alpha = splat_alpha2(q1.y, p2, G);
  const bool on = live && !(p2 > 0.f) && !(alpha < kAlphaSkip);
  const float ae = on ? alpha : 0.f;
  const float inv_om = __frcp_rn(1.f - ae);
  const float Ti = T * inv_om;
  const float wgt = ae * Ti;
  const float dcr = dC[0] * rgb[0] + dC[1] * rgb[1] + dC[2] * rgb[2];
  const float dLda = Ti * dcr - inv_om * (bgd + dCS);
  acc[6] = fmaf(dC[0], wgt, acc[6]);
  acc[7] = fmaf(dC[1], wgt, acc[7]);
  acc[8] = fmaf(dC[2], wgt, acc[8]);
  dCS = fmaf(wgt, dcr, dCS);
  T = Ti;
  // zero through a clamped alpha (opacity G > 0.99)
  const float dLg = (on && __fmul_rn(q1.y, G) <= kAlphaClamp) ? dLda : 0.f;
  acc[5] = fmaf(dLg, G, acc[5]);
  const float dp = dLg * alpha;  // dL/dpower
  acc[0] = fmaf(dp, fmaf(q0.w, dy, cA2dx), acc[0]);       // d p2 / d mu_x
  acc[1] = fmaf(dp, fmaf(2.f * q1.x, dy, cBdx), acc[1]);  // d p2 / d mu_y
  acc[2] = fmaf(dp, dx2, acc[2]);
  acc[3] = fmaf(dp, dx * dy, acc[3]);
  acc[4] = fmaf(dp, dy * dy, acc[4]);
  return on;
}

// One forward (pixel, Gaussian) pair, branch-free.  bit = this pixel's bit in
// `done`; idx = 1 + the pair's list position.
__device__ __forceinline__ void fwd_pair(const float4& q1, float blue, float a0, float a1, float dy, uint32_t bit,
                                         uint32_t idx, uint32_t& done, float& T, float (&C)[3], uint32_t& last) {
  const float p2 = splat_p2(q1.x, a1, a0, dy);
  float G;
  const float alpha = splat_alpha2(q1.y, p2, G);
  const bool ok = !(done & bit) && !(p2 > 0.f) && !(alpha < kAlphaSkip);
  const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
  const bool stop = ok && Tn < kTStop;
  done |= stop ? bit : 0u;
  const bool acc = ok && !stop;
  const float wgt = acc ? alpha * T : 0.f;
  C[0] = fmaf(q1.z, wgt, C[0]);
  C[1] = fmaf(q1.w, wgt, C[1]);
  C[2] = fmaf(blue, wgt, C[2]);
  T = acc ? Tn : T;
  last = acc ? idx : last;
}

// ---------------------------------------------------------------- block per tile

template <int PPT>
struct BlockShape {
  static constexpr int NT = 256 / PPT;    // threads
  static constexpr int NW = NT / 32;      // warps
  static constexpr int BAND = 4 * PPT;    // rows per warp
  // pixel of (warp, lane, k) inside the tile
  __device__ static int col(int w, int lane) { return (w & 1) * 8 + (lane & 7); }
  __device__ static int row(int w, int lane) { return (w >> 1) * BAND + (lane >> 3) * PPT; }
};

template <int PPT>
__global__ void __launch_bounds__(256 / PPT) raster_fwd_kernel(RasterArgs a) {
  using S = BlockShape<PPT>;
  constexpr int NT = S::NT;
  __shared__ float4 s0[NT], s1[NT], s2[NT];
  const int bin = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = view_of_bin(a.views, a.B, bin);
  const ViewRec& V = a.views[v];
  const int tile = bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + S::col(w, lane);
  const int py0 = ty * kTile + S::row(w, lane);
  // the warp's pixel rectangle
  const float wx0 = (float)(tx * kTile + (w & 1) * 8), wx1 = wx0 + 7.f;
  const float wy0 = (float)(ty * kTile + (w >> 1) * S::BAND), wy1 = wy0 + (float)(S::BAND - 1);
  const uint2 rg = a.ranges[bin];
  const int n = (int)(rg.y - rg.x);

  float T[PPT], C[PPT][3];
  uint32_t last[PPT];
  uint32_t done = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    T[k] = 1.f;
    C[k][0] = C[k][1] = C[k][2] = 0.f;
    last[k] = 0;
    if (!(px < V.W && py0 + k < V.H)) done |= 1u << k;
  }
  const uint32_t all_done = (1u << PPT) - 1u;
  const float fpx = (float)px, fpy = (float)py0;
  for (int b0 = 0; b0 < n; b0 += NT) {
    if (__syncthreads_count(done == all_done) == NT) break;
    const int i = b0 + (int)threadIdx.x;
    if (i < n) stage_one(a, v, a.vals[rg.x + i], s0[threadIdx.x], s1[threadIdx.x], s2[threadIdx.x]);
    __syncthreads();
    const int cnt = min(NT, n - b0);
    bool warp_done = __all_sync(0xffffffffu, done == all_done);
    for (int j = 0; j < cnt && !warp_done; j++) {
      const float4 q0 = s0[j];
      const float4 q2 = s2[j];
      if (!box_hits(q0, q2, wx0, wx1, wy0, wy1)) continue;
      const float4 q1 = s1[j];
      const float dx = __fsub_rn(q0.x, fpx);
      const float a0 = __fmul_rn(q0.z, __fmul_rn(dx, dx));
      const float a1 = __fmul_rn(q0.w, dx);
#pragma unroll
      for (int k = 0; k < PPT; k++)
        fwd_pair(q1, q2.x, a0, a1, __fsub_rn(q0.y, fpy + (float)k), 1u << k, (uint32_t)(b0 + j + 1), done, T[k],
                 C[k], last[k]);
      warp_done = __all_sync(0xffffffffu, done == all_done);
    }
    __syncthreads();
  }
  const int64_t plane = (int64_t)V.W * V.H;
  float* img = a.image + 3 * V.pix_offset;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    if (px >= V.W || py >= V.H) continue;
    const int64_t p = (int64_t)py * V.W + px;
    img[p] = fmaf(T[k], V.bg[0], C[k][0]);
    img[plane + p] = fmaf(T[k], V.bg[1], C[k][1]);
    img[2 * plane + p] = fmaf(T[k], V.bg[2], C[k][2]);
    a.tfinal[V.pix_offset + p] = T[k];
    a.nlast[V.pix_offset + p] = last[k];
  }
}

template <int PPT>
__global__ void __launch_bounds__(256 / PPT) raster_bwd_kernel(RasterArgs a) {
  using S = BlockShape<PPT>;
  constexpr int NT = S::NT;
  __shared__ float4 s0[NT], s1[NT], s2[NT];
  __shared__ uint32_t sg[NT];
  __shared__ uint32_t s_maxlast;
  const int bin = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = view_of_bin(a.views, a.B, bin);
  const ViewRec& V = a.views[v];
  const int tile = bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + S::col(w, lane);
  const int py0 = ty * kTile + S::row(w, lane);
  const float wx0 = (float)(tx * kTile + (w & 1) * 8), wx1 = wx0 + 7.f;
  const float wy0 = (float)(ty * kTile + (w >> 1) * S::BAND), wy1 = wy0 + (float)(S::BAND - 1);
  const uint2 rg = a.ranges[bin];
  if (threadIdx.x == 0) s_maxlast = 0;

  const int64_t plane = (int64_t)V.W * V.H;
  const float* dimg = a.dimage + 3 * V.pix_offset;
  float T[PPT], dC[PPT][3], dCS[PPT], bgd[PPT];
  uint32_t nl[PPT];
  uint32_t mymax = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    const bool in = px < V.W && py < V.H;
    const int64_t p = (int64_t)py * V.W + px;
    T[k] = in ? a.tfinal[V.pix_offset + p] : 1.f;
    nl[k] = in ? a.nlast[V.pix_offset + p] : 0u;
#pragma unroll
    for (int c = 0; c < 3; c++) dC[k][c] = in ? dimg[c * plane + p] : 0.f;
    dCS[k] = 0.f;
    bgd[k] = T[k] * (dC[k][0] * V.bg[0] + dC[k][1] * V.bg[1] + dC[k][2] * V.bg[2]);
    mymax = max(mymax, nl[k]);
  }
  const uint32_t warp_max = __reduce_max_sync(0xffffffffu, mymax);
  __syncthreads();
  if (lane == 0) atomicMax(&s_maxlast, warp_max);
  __syncthreads();
  const int total = (int)s_maxlast;
  const float fpx = (float)px, fpy = (float)py0;
  for (int bend = total; bend > 0; bend -= NT) {
    const int bstart = max(0, bend - NT);
    const int i = bstart + (int)threadIdx.x;
    if (i < bend) {
      const uint32_t g = a.vals[rg.x + i];
      stage_one(a, v, g, s0[threadIdx.x], s1[threadIdx.x], s2[threadIdx.x]);
      sg[threadIdx.x] = g;
    }
    __syncthreads();
    const int jmax = min(bend - bstart, (int)warp_max - bstart);  // entries this warp needs
    for (int j = jmax - 1; j >= 0; j--) {
      const float4 q0 = s0[j];
      const float4 q2 = s2[j];
      if (!box_hits(q0, q2, wx0, wx1, wy0, wy1)) continue;
      const float4 q1 = s1[j];
      const uint32_t idx = (uint32_t)(bstart + j);
      const float rgb[3] = {q1.z, q1.w, q2.x};
      const float dx = __fsub_rn(q0.x, fpx);
      const float dx2 = __fmul_rn(dx, dx);
      const float a0 = __fmul_rn(q0.z, dx2);
      const float a1 = __fmul_rn(q0.w, dx);
      const float cA2dx = 2.f * q0.z * dx;
      const float cBdx = q0.w * dx;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; q++) acc[q] = 0.f;
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; k++)
        any |= bwd_pair(idx < nl[k], q0, q1, rgb, a0, a1, __fsub_rn(q0.y, fpy + (float)k), dx, dx2, cA2dx, cBdx, T[k],
                        dCS[k], dC[k], bgd[k], acc);
      if (__any_sync(0xffffffffu, any)) push_grad(a.g2d, (int64_t)v * a.stride + sg[j], acc, lane);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- warp per tile

constexpr int kRows = 8;

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS) raster_fwd_warp_kernel(RasterArgs a, int64_t bins) {
  __shared__ float4 s0[WARPS][32], s1[WARPS][32], s2[WARPS][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t bin = (int64_t)blockIdx.x * WARPS + w;
  if (bin >= bins) return;
  const int v = view_of_bin(a.views, a.B, (int)bin);
  const ViewRec& V = a.views[v];
  const int tile = (int)bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + (lane & 15);
  const int py0 = ty * kTile + (lane >> 4) * kRows;
  const float wx0 = (float)(tx * kTile), wx1 = wx0 + 15.f, wy0 = (float)(ty * kTile), wy1 = wy0 + 15.f;
  const uint2 rg = a.ranges[bin];
  const int n = (int)(rg.y - rg.x);

  float T[kRows], C[kRows][3];
  uint32_t last[kRows];
  uint32_t done = 0;
#pragma unroll
  for (int k = 0; k < kRows; k++) {
    T[k] = 1.f;
    C[k][0] = C[k][1] = C[k][2] = 0.f;
    last[k] = 0;
    if (!(px < V.W && py0 + k < V.H)) done |= 1u << k;
  }
  const float fpx = (float)px, fpy = (float)py0;
  for (int b0 = 0; b0 < n; b0 += 32) {
    if (__all_sync(0xffffffffu, done == (1u << kRows) - 1)) break;
    const int i = b0 + lane;
    __syncwarp();
    if (i < n) stage_one(a, v, a.vals[rg.x + i], s0[w][lane], s1[w][lane], s2[w][lane]);
    __syncwarp();
    const int cnt = min(32, n - b0);
    for (int j = 0; j < cnt; j++) {
      const float4 q0 = s0[w][j];
      const float4 q2 = s2[w][j];
      if (!box_hits(q0, q2, wx0, wx1, wy0, wy1)) continue;
      const float4 q1 = s1[w][j];
      const float dx = __fsub_rn(q0.x, fpx);
      const float a0 = __fmul_rn(q0.z, __fmul_rn(dx, dx));
      const float a1 = __fmul_rn(q0.w, dx);
#pragma unroll
      for (int k = 0; k < kRows; k++)
        fwd_pair(q1, q2.x, a0, a1, __fsub_rn(q0.y, fpy + (float)k), 1u << k, (uint32_t)(b0 + j + 1), done, T[k],
                 C[k], last[k]);
    }
  }
  const int64_t plane = (int64_t)V.W * V.H;
  float* img = a.image + 3 * V.pix_offset;
#pragma unroll
  for (int k = 0; k < kRows; k++) {
    const int py = py0 + k;
    if (px >= V.W || py >= V.H) continue;
    const int64_t p = (int64_t)py * V.W + px;
    img[p] = fmaf(T[k], V.bg[0], C[k][0]);
    img[plane + p] = fmaf(T[k], V.bg[1], C[k][1]);
    img[2 * plane + p] = fmaf(T[k], V.bg[2], C[k][2]);
    a.tfinal[V.pix_offset + p] = T[k];
    a.nlast[V.pix_offset + p] = last[k];
  }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS) raster_bwd_warp_kernel(RasterArgs a, int64_t bins) {
  __shared__ float4 s0[WARPS][32], s1[WARPS][32], s2[WARPS][32];
  __shared__ uint32_t sg[WARPS][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t bin = (int64_t)blockIdx.x * WARPS + w;
  if (bin >= bins) return;
  const int v = view_of_bin(a.views, a.B, (int)bin);
  const ViewRec& V = a.views[v];
  const int tile = (int)bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + (lane & 15);
  const int py0 = ty * kTile + (lane >> 4) * kRows;
  const float wx0 = (float)(tx * kTile), wx1 = wx0 + 15.f, wy0 = (float)(ty * kTile), wy1 = wy0 + 15.f;
  const uint2 rg = a.ranges[bin];
  const int64_t plane = (int64_t)V.W * V.H;
  const float* dimg = a.dimage + 3 * V.pix_offset;

  float T[kRows], dC[kRows][3], dCS[kRows], bgd[kRows];
  uint32_t nl[kRows];
  uint32_t mymax = 0;
#pragma unroll
  for (int k = 0; k < kRows; k++) {
    const int py = py0 + k;
    const bool in = px < V.W && py < V.H;
    const int64_t p = (int64_t)py * V.W + px;
    T[k] = in ? a.tfinal[V.pix_offset + p] : 1.f;
    nl[k] = in ? a.nlast[V.pix_offset + p] : 0u;
#pragma unroll
    for (int c = 0; c < 3; c++) dC[k][c] = in ? dimg[c * plane + p] : 0.f;
    dCS[k] = 0.f;
    bgd[k] = T[k] * (dC[k][0] * V.bg[0] + dC[k][1] * V.bg[1] + dC[k][2] * V.bg[2]);
    mymax = max(mymax, nl[k]);
  }
  const int total = (int)__reduce_max_sync(0xffffffffu, mymax);
  const float fpx = (float)px, fpy = (float)py0;
  for (int bend = total; bend > 0; bend -= 32) {
    const int bstart = max(0, bend - 32);
    const int i = bstart + lane;
    __syncwarp();
    if (i < bend) {
      const uint32_t g = a.vals[rg.x + i];
      stage_one(a, v, g, s0[w][lane], s1[w][lane], s2[w][lane]);
      sg[w][lane] = g;
    }
    __syncwarp();
    for (int j = bend - bstart - 1; j >= 0; j--) {
      const float4 q0 = s0[w][j];
      const float4 q2 = s2[w][j];
      if (!box_hits(q0, q2, wx0, wx1, wy0, wy1)) continue;
      const float4 q1 = s1[w][j];
      const uint32_t idx = (uint32_t)(bstart + j);
      const float rgb[3] = {q1.z, q1.w, q2.x};
      const float dx = __fsub_rn(q0.x, fpx);
      const float dx2 = __fmul_rn(dx, dx);
      const float a0 = __fmul_rn(q0.z, dx2);
      const float a1 = __fmul_rn(q0.w, dx);
      const float cA2dx = 2.f * q0.z * dx;
      const float cBdx = q0.w * dx;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; q++) acc[q] = 0.f;
      bool any = false;
#pragma unroll
      for (int k = 0; k < kRows; k++)
        any |= bwd_pair(idx < nl[k], q0, q1, rgb, a0, a1, __fsub_rn(q0.y, fpy + (float)k), dx, dx2, cA2dx, cBdx, T[k],
                        dCS[k], dC[k], bgd[k], acc);
      if (__any_sync(0xffffffffu, any)) push_grad(a.g2d, (int64_t)v * a.stride + sg[w][j], acc, lane);
    }
  }
}

void launch_raster_fwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 8: raster_fwd_warp_kernel<4><<<(unsigned)((bins + 3) / 4), 128, 0, s>>>(a, bins); break;
    case 1: raster_fwd_kernel<1><<<(unsigned)bins, 256, 0, s>>>(a); break;
    case 4: raster_fwd_kernel<4><<<(unsigned)bins, 64, 0, s>>>(a); break;
    default: raster_fwd_kernel<2><<<(unsigned)bins, 128, 0, s>>>(a); break;
  }
}

void launch_raster_bwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 8: raster_bwd_warp_kernel<4><<<(unsigned)((bins + 3) / 4), 128, 0, s>>>(a, bins); break;
    case 1: raster_bwd_kernel<1><<<(unsigned)bins, 256, 0, s>>>(a); break;
    case 4: raster_bwd_kernel<4><<<(unsigned)bins, 64, 0, s>>>(a); break;
    default: raster_bwd_kernel<2><<<(unsigned)bins, 128, 0, s>>>(a); break;
  }
}

}  // namespace gs
