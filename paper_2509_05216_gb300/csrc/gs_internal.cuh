// Internal definitions shared by the CUDA kernels of libgs.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = 16;               // 16x16 screen tiles
constexpr int kMaxViews = 64;           // views per batch
constexpr float kAlphaClamp = 0.99f;    // alpha = min(0.99, opacity * G)
constexpr float kAlphaSkip = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;         // stop before T would fall below this
constexpr float kDilation = 0.3f;       // added to the 2D covariance diagonal
constexpr float kGuard = 1.3f;          // slope clamp, in half fields of view
constexpr float kLog2e = 1.4426950408889634f;

// Projected records: three float4 per (view, Gaussian), stored together
// (48 bytes), so a compositing kernel's gather of one record touches two
// 32-byte sectors instead of three.  Record k of entry o is rec[kRecStride * o + k].
constexpr int kRecStride = 3;

// 2D gradients per (view, Gaussian), two arrays of records: geometry
// (kG2dGeo floats: dL/d(mu_x, mu_y, A, B), dL/d(C, opacity), 0, 0) for all
// B x stride entries, then colour (kG2dCol floats: dL/d(r, g, b), 0).
constexpr int kG2dGeo = 8;
constexpr int kG2dCol = 4;

// Device status word bits.
constexpr int kStatusCapacity = 1;
constexpr int kStatusTimeout = 2;

// Per-view record, built on the host from gs_camera.
struct ViewRec {
  float R[9];         // world->camera rotation (row-major)
  float t[3];         // world->camera translation
  float fx, fy, cx, cy;
  float znear;
  float limx, limy;   // slope clamp limits: 1.3 * W / (2 fx), 1.3 * H / (2 fy)
  float campos[3];    // camera centre in world coordinates
  float bg[3];
  int W, H, gw, gh;
  int tile_offset;    // first bin of this view
  int pad0;
  long long pix_offset;  // first pixel of this view (per channel plane)
};

// Real orthonormal SH constants (Y_{l,m} without the Condon-Shortley phase):
// Y00 = 1/(2 sqrt(pi)), Y1m = sqrt(3/(4 pi)) (y, z, x), and for l = 2, 3 the
// normalisations of the Cartesian forms listed in evaluate_sh below.
constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // (1/2) sqrt(15/pi)
constexpr float kSH2b = 0.31539156525252005f;  // (1/4) sqrt(5/pi)
constexpr float kSH2c = 0.5462742152960396f;   // (1/4) sqrt(15/pi)
constexpr float kSH3e = 0.5900435899266435f;   // (1/4) sqrt(35/(2 pi))
constexpr float kSH3f = 2.890611442640554f;    // (1/2) sqrt(105/pi)
constexpr float kSH3g = 0.4570457994644658f;   // (1/4) sqrt(21/(2 pi))
constexpr float kSH3h = 0.3731763325901154f;   // (1/4) sqrt(7/pi)
constexpr float kSH3k = 1.445305721320277f;    // (1/4) sqrt(105/pi)

__host__ __device__ inline int n_sh(int deg) { return (deg + 1) * (deg + 1); }
__host__ __device__ inline int n_planes(int deg) { return 11 + 3 * n_sh(deg); }

// Depth used to order and cull: FP32 value of t_z evaluated as
// ((R20 mx + R21 my) + R22 mz) + t2, each operation rounded (no FMA).
__device__ __forceinline__ float depth_key(const ViewRec& v, float mx, float my, float mz) {
  float a = __fmul_rn(v.R[6], mx);
  float b = __fmul_rn(v.R[7], my);
  float c = __fmul_rn(v.R[8], mz);
  return __fadd_rn(__fadd_rn(__fadd_rn(a, b), c), v.t[2]);
}

// Alpha of a Gaussian at a pixel offset (dx, dy) = mu2D - pixel, with the
// exact same instruction sequence in the forward and backward kernels (so
// their skip decisions agree).  Returns power through *pw.
__device__ __forceinline__ float splat_power(float A, float B, float C, float dx, float dy) {
  float q = __fmaf_rn(A, __fmul_rn(dx, dx), __fmul_rn(C, __fmul_rn(dy, dy)));
  return __fmaf_rn(-0.5f, q, -__fmul_rn(B, __fmul_rn(dx, dy)));
}

// One Adam step of one scalar (torch.optim.Adam with bias correction):
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr' m / (sqrt(v) /
// sqrt(1 - b2^t) + eps) with lr' = lr / (1 - b1^t).  Every rounding is
// spelled out, so the stand-alone Adam kernel and the projection backward's
// fused update give the same bits.
struct AdamStep {
  float b1, b2, c1, c2, eps, isb2;  // c1 = 1 - b1, c2 = 1 - b2, isb2 = 1 / sqrt(1 - b2^t)
};
__device__ __forceinline__ void adam_scalar(float& p, float& m, float& v, float g, float lr, const AdamStep& s) {
  m = __fmaf_rn(s.b1, m, __fmul_rn(s.c1, g));
  v = __fmaf_rn(s.b2, v, __fmul_rn(__fmul_rn(s.c2, g), g));
  p = __fsub_rn(p, __fdiv_rn(__fmul_rn(lr, m), __fmaf_rn(__fsqrt_rn(v), s.isb2, s.eps)));
}

// Tile rect of a splat: x in [floor((mx - r)/16), floor((mx + r + 15)/16)),
// likewise y, clamped to the view's tile grid.  Shared by the projection
// (tile counts) and the duplication (instances), so both see the same rect.
__device__ __forceinline__ bool tile_rect(const ViewRec& V, float mx, float my, int radius, int& x0,
                                          int& x1, int& y0, int& y1) {
  const float fr = (float)radius, fr15 = (float)(radius + kTile - 1);
  const float gw = (float)V.gw, gh = (float)V.gh;
  const float inv = 1.0f / (float)kTile;  // exact
  x0 = (int)fminf(gw, fmaxf(0.f, floorf(__fmul_rn(__fsub_rn(mx, fr), inv))));
  x1 = (int)fminf(gw, fmaxf(0.f, floorf(__fmul_rn(__fadd_rn(mx, fr15), inv))));
  y0 = (int)fminf(gh, fmaxf(0.f, floorf(__fmul_rn(__fsub_rn(my, fr), inv))));
  y1 = (int)fminf(gh, fmaxf(0.f, floorf(__fmul_rn(__fadd_rn(my, fr15), inv))));
  return x1 > x0 && y1 > y0;
}

// Tiles of one axis that the box [m - h, m + h] reaches with a pixel:
// [t0, t1), clamped to [0, g).  Tile t spans pixels 16 t .. 16 t + 15; it is
// reached iff 16 t <= m + h and 16 t + 15 >= m - h, with m + h and m - h the
// FP32 sums the compositing kernels' box test forms, so a tile outside the
// range fails that test at every pixel of it.  h < 0 (a splat that never
// reaches alpha >= 1/255) gives an empty range.
__device__ __forceinline__ void box_tiles(float m, float h, int g, int& t0, int& t1) {
  const float lo = __fsub_rn(m, h), hi = __fadd_rn(m, h);
  const float f = floorf(__fmul_rn(lo, 0.0625f));
  const float first = lo <= __fadd_rn(__fmul_rn(16.f, f), 15.f) ? f : __fadd_rn(f, 1.f);
  const float last = __fadd_rn(floorf(__fmul_rn(hi, 0.0625f)), 1.f);
  t0 = (int)fminf((float)g, fmaxf(0.f, first));
  t1 = (int)fminf((float)g, fmaxf(0.f, last));
}

}  // namespace gs
