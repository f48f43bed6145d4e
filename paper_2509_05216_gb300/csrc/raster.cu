// Per-tile front-to-back alpha compositing (forward) and its reverse-order
// backward pass.
//
// 3D-GS composites each pixel over its tile's depth-sorted list (Section I of
// the paper cites it as the renderer the method trains): alpha =
// min(0.99, opacity * exp(power)), skip if power > 0 or alpha < 1/255, stop
// before a Gaussian that would bring T below 1e-4.  The backward pass walks
// the same list from each pixel's last contributor towards the front,
// recovering T by division and keeping the colour composited behind.
//
// One block per 16x16 tile; each thread owns PPT vertically adjacent pixels.
// The tile's list is staged through shared memory in batches of one record
// per thread, and a block stops as soon as every pixel has saturated.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

// alpha and the Gaussian factor G = exp(power); identical in both kernels.
__device__ __forceinline__ float splat_alpha(float opacity, float power, float& G) {
  G = __expf(power);
  return fminf(kAlphaClamp, __fmul_rn(opacity, G));
}

__device__ __forceinline__ int view_of_bin(const ViewRec* views, int B, int bin) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_offset <= bin) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int PPT>
__global__ void __launch_bounds__(256 / PPT) raster_fwd_kernel(RasterArgs a) {
  constexpr int NT = 256 / PPT;
  __shared__ float4 s0[NT], s1[NT];
  __shared__ float s2[NT];
  const int bin = blockIdx.x;
  const int v = view_of_bin(a.views, a.B, bin);
  const ViewRec& V = a.views[v];
  const int tile = bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + (threadIdx.x & 15);
  const int py0 = ty * kTile + (threadIdx.x >> 4) * PPT;
  const uint2 rg = a.ranges[bin];
  const int n = (int)(rg.y - rg.x);

  float T[PPT], C[PPT][3];
  uint32_t last[PPT];
  bool done[PPT];
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    T[k] = 1.f;
    C[k][0] = C[k][1] = C[k][2] = 0.f;
    last[k] = 0;
    done[k] = !(px < V.W && py0 + k < V.H);
  }
  const float fpx = (float)px;
  for (int b0 = 0; b0 < n; b0 += NT) {
    bool all = true;
#pragma unroll
    for (int k = 0; k < PPT; k++) all &= done[k];
    if (__syncthreads_count(all) == NT) break;
    const int i = b0 + (int)threadIdx.x;
    if (i < n) {
      const int64_t o = (int64_t)v * a.stride + a.vals[rg.x + i];
      s0[threadIdx.x] = a.rec0[o];
      s1[threadIdx.x] = a.rec1[o];
      s2[threadIdx.x] = a.rec2[o].x;
    }
    __syncthreads();
    const int cnt = min(NT, n - b0);
    for (int j = 0; j < cnt; j++) {
      const float4 r0 = s0[j], r1 = s1[j];
      const float blue = s2[j];
      const float dx = __fsub_rn(r0.x, fpx);
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        if (done[k]) continue;
        const float dy = __fsub_rn(r0.y, (float)(py0 + k));
        const float power = splat_power(r0.z, r0.w, r1.x, dx, dy);
        if (power > 0.f) continue;
        float G;
        const float alpha = splat_alpha(r1.y, power, G);
        if (alpha < kAlphaSkip) continue;
        const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
        if (Tn < kTStop) {
          done[k] = true;
          continue;
        }
        const float w = alpha * T[k];
        C[k][0] = fmaf(r1.z, w, C[k][0]);
        C[k][1] = fmaf(r1.w, w, C[k][1]);
        C[k][2] = fmaf(blue, w, C[k][2]);
        T[k] = Tn;
        last[k] = (uint32_t)(b0 + j + 1);
      }
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
  constexpr int NT = 256 / PPT;
  __shared__ float4 s0[NT], s1[NT];
  __shared__ float s2[NT];
  __shared__ uint32_t sg[NT];
  __shared__ uint32_t s_maxlast;
  const int bin = blockIdx.x;
  const int v = view_of_bin(a.views, a.B, bin);
  const ViewRec& V = a.views[v];
  const int tile = bin - V.tile_offset;
  const int tx = tile % V.gw, ty = tile / V.gw;
  const int px = tx * kTile + (threadIdx.x & 15);
  const int py0 = ty * kTile + (threadIdx.x >> 4) * PPT;
  const uint2 rg = a.ranges[bin];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_maxlast = 0;

  const int64_t plane = (int64_t)V.W * V.H;
  const float* dimg = a.dimage + 3 * V.pix_offset;
  float T[PPT], Tf[PPT], dC[PPT][3], S[PPT][3], bgdot[PPT];
  uint32_t nl[PPT];
  uint32_t mymax = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    const bool in = px < V.W && py < V.H;
    const int64_t p = (int64_t)py * V.W + px;
    Tf[k] = in ? a.tfinal[V.pix_offset + p] : 1.f;
    nl[k] = in ? a.nlast[V.pix_offset + p] : 0u;
    T[k] = Tf[k];
    for (int c = 0; c < 3; c++) {
      dC[k][c] = in ? dimg[c * plane + p] : 0.f;
      S[k][c] = 0.f;
    }
    bgdot[k] = Tf[k] * (dC[k][0] * V.bg[0] + dC[k][1] * V.bg[1] + dC[k][2] * V.bg[2]);
    mymax = max(mymax, nl[k]);
  }
  mymax = __reduce_max_sync(0xffffffffu, mymax);
  __syncthreads();
  if (lane == 0) atomicMax(&s_maxlast, mymax);
  __syncthreads();
  const int total = (int)s_maxlast;
  const float fpx = (float)px;
  float4* g2d = a.g2d;
  for (int bend = total; bend > 0; bend -= NT) {
    const int bstart = max(0, bend - NT);
    const int i = bstart + (int)threadIdx.x;
    if (i < bend) {
      const uint32_t g = a.vals[rg.x + i];
      const int64_t o = (int64_t)v * a.stride + g;
      s0[threadIdx.x] = a.rec0[o];
      s1[threadIdx.x] = a.rec1[o];
      s2[threadIdx.x] = a.rec2[o].x;
      sg[threadIdx.x] = g;
    }
    __syncthreads();
    for (int j = bend - bstart - 1; j >= 0; j--) {
      const uint32_t idx = (uint32_t)(bstart + j);
      const float4 r0 = s0[j], r1 = s1[j];
      const float rgb[3] = {r1.z, r1.w, s2[j]};
      const float dx = __fsub_rn(r0.x, fpx);
      float acc[9];
#pragma unroll
      for (int q = 0; q < 9; q++) acc[q] = 0.f;
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        if (idx >= nl[k]) continue;
        const float dy = __fsub_rn(r0.y, (float)(py0 + k));
        const float power = splat_power(r0.z, r0.w, r1.x, dx, dy);
        if (power > 0.f) continue;
        float G;
        const float alpha = splat_alpha(r1.y, power, G);
        if (alpha < kAlphaSkip) continue;
        any = true;
        const float om = 1.f - alpha;
        const float Ti = T[k] / om;  // transmittance in front of this Gaussian
        const float w = alpha * Ti;
        float dLda = -bgdot[k] / om;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          dLda += dC[k][c] * (Ti * rgb[c] - S[k][c] / om);
          acc[6 + c] += dC[k][c] * w;
          S[k][c] = fmaf(rgb[c], w, S[k][c]);
        }
        T[k] = Ti;
        if (__fmul_rn(r1.y, G) <= kAlphaClamp) {
          acc[5] += dLda * G;
          const float dp = dLda * alpha;
          acc[0] -= dp * (r0.z * dx + r0.w * dy);
          acc[1] -= dp * (r1.x * dy + r0.w * dx);
          acc[2] -= 0.5f * dp * dx * dx;
          acc[3] -= dp * dx * dy;
          acc[4] -= 0.5f * dp * dy * dy;
        }
      }
      if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int q = 0; q < 9; q++) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        }
        if (lane == 0) {
          float4* dst = g2d + ((int64_t)v * a.stride + sg[j]) * 3;
          atomicAdd(dst, make_float4(acc[0], acc[1], acc[2], acc[3]));
          atomicAdd(dst + 1, make_float4(acc[4], acc[5], acc[6], acc[7]));
          atomicAdd(&dst[2].x, acc[8]);
        }
      }
    }
    __syncthreads();
  }
}

void launch_raster_fwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 1: raster_fwd_kernel<1><<<(unsigned)bins, 256, 0, s>>>(a); break;
    case 4: raster_fwd_kernel<4><<<(unsigned)bins, 64, 0, s>>>(a); break;
    default: raster_fwd_kernel<2><<<(unsigned)bins, 128, 0, s>>>(a); break;
  }
}

void launch_raster_bwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 1: raster_bwd_kernel<1><<<(unsigned)bins, 256, 0, s>>>(a); break;
    case 4: raster_bwd_kernel<4><<<(unsigned)bins, 64, 0, s>>>(a); break;
    default: raster_bwd_kernel<2><<<(unsigned)bins, 128, 0, s>>>(a); break;
  }
}

}  // namespace gs
