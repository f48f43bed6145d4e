// Adaptive density control of 3D-GS: clone, split and prune Gaussians from
// the screen-space gradient statistic accumulated by the projection
// backward.
//
// The paper is silent on densification (N comes from the point cloud); this
// is 3D-GS's step: a Gaussian whose mean gradient, averaged over the views
// where it touches a tile, reaches the threshold is cloned when small
// (largest scale <= percent_dense x scene extent) and split into N samples
// of its own distribution (scales shrunk by 0.8 N) when large; Gaussians
// whose opacity is below the minimum are removed.  New Gaussians start with
// zero Adam moments.  The output keeps the input order, a Gaussian's outputs
// together: a counting pass (outputs per block of 256 Gaussians), the
// binning's block-sum scan, and an emitting pass that rescans inside each
// block.
#include <cmath>

#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

namespace {

enum { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

__device__ __forceinline__ int decide(const DensifyArgs& a, int64_t g) {
  const int64_t S = a.stride;
  const float o = a.p[10 * S + g];
  if (1.f / (1.f + expf(-o)) < a.min_opacity) return kPrune;
  const float c = a.count[g];
  const float avg = c > 0.f ? a.grad[g] / c : 0.f;
  if (!(avg >= a.tau)) return kKeep;
  const float smax = expf(fmaxf(a.p[3 * S + g], fmaxf(a.p[4 * S + g], a.p[5 * S + g])));
  return smax <= a.dense_extent ? kClone : kSplit;
}

__device__ __forceinline__ int outputs(int kind, int split_n) {
  return kind == kPrune ? 0 : kind == kKeep ? 1 : kind == kClone ? 2 : split_n;
}

__device__ __forceinline__ uint32_t block_prefix(uint32_t c, uint32_t* warp_tot, uint32_t* total) {
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

__global__ void __launch_bounds__(256) densify_count_kernel(DensifyArgs a) {
  __shared__ uint32_t warp_tot[8];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t c = g < a.n ? (uint32_t)outputs(decide(a, g), a.split_n) : 0u;
  uint32_t tot;
  block_prefix(c, warp_tot, &tot);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) densify_emit_kernel(DensifyArgs a) {
  __shared__ uint32_t warp_tot[8];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int kind = g < a.n ? decide(a, g) : kPrune;
  const int cnt = outputs(kind, a.split_n);
  uint32_t tot;
  const uint32_t pre = block_prefix((uint32_t)cnt, warp_tot, &tot);
  if (!cnt) return;
  const int64_t o0 = (int64_t)a.block_offsets[blockIdx.x] + pre;
  const int64_t S = a.stride, OS = a.out_stride;
  if (kind == kKeep || kind == kClone) {
    for (int pl = 0; pl < a.planes; pl++) {
      const float pv = a.p[pl * S + g];
      a.po[pl * OS + o0] = pv;
      a.mo[pl * OS + o0] = a.m[pl * S + g];
      a.vo[pl * OS + o0] = a.v[pl * S + g];
      if (kind == kClone) {  // the copy: same parameters, fresh moments
        a.po[pl * OS + o0 + 1] = pv;
        a.mo[pl * OS + o0 + 1] = 0.f;
        a.vo[pl * OS + o0 + 1] = 0.f;
      }
    }
    return;
  }
  // split: N samples of the Gaussian's own distribution, mean + R (s * z)
  const float w0 = a.p[6 * S + g], x0 = a.p[7 * S + g], y0 = a.p[8 * S + g], z0 = a.p[9 * S + g];
  const float iq = rsqrtf(w0 * w0 + x0 * x0 + y0 * y0 + z0 * z0);
  const float w = w0 * iq, x = x0 * iq, y = y0 * iq, z = z0 * iq;
  const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z),       2.f * (x * z + w * y),
                      2.f * (x * y + w * z),       1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                      2.f * (x * z - w * y),       2.f * (y * z + w * x),       1.f - 2.f * (x * x + y * y)};
  float sc[3];
#pragma unroll
  for (int d = 0; d < 3; d++) sc[d] = expf(a.p[(3 + d) * S + g]);
  for (int k = 0; k < a.split_n; k++) {
    const int64_t o = o0 + k;
    const float* zz = a.noise + 3 * ((int64_t)g * a.split_n + k);
    const float u0 = sc[0] * zz[0], u1 = sc[1] * zz[1], u2 = sc[2] * zz[2];
#pragma unroll
    for (int d = 0; d < 3; d++)
      a.po[d * OS + o] = a.p[d * S + g] + (R[3 * d] * u0 + R[3 * d + 1] * u1 + R[3 * d + 2] * u2);
#pragma unroll
    for (int d = 0; d < 3; d++) a.po[(3 + d) * OS + o] = a.p[(3 + d) * S + g] - a.log_shrink;
    for (int pl = 6; pl < a.planes; pl++) a.po[pl * OS + o] = a.p[pl * S + g];
    for (int pl = 0; pl < a.planes; pl++) {
      a.mo[pl * OS + o] = 0.f;
      a.vo[pl * OS + o] = 0.f;
    }
  }
}

void launch_densify(const DensifyArgs& a, bool emit, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.n + 255) / 256);
  if (blocks == 0) return;
  if (emit) densify_emit_kernel<<<blocks, 256, 0, s>>>(a);
  else densify_count_kernel<<<blocks, 256, 0, s>>>(a);
}

}  // namespace gs
