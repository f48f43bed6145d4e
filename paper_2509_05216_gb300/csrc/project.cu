// EWA projection of 3D Gaussians to 2D conics with view-dependent SH colour,
// forward (per view and Gaussian) and backward (chain rule to the parameters,
// summed over the views of a batch).
//
// The paper initialises 3D-GS primitives from isosurface points and fits them
// to orbit views (Section III); the projection is the EWA splatting step of
// 3D-GS (Section I): Sigma' = J W Sigma W^T J^T + 0.3 I, conic = Sigma'^-1,
// radius ceil(3 sqrt(lambda_max)), colour max(0, SH(d) + 0.5).
//
// Layout: one thread per Gaussian loads its parameters once (coalesced plane
// reads) and loops over the B views, so a batch reads the parameter set once.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

template <int DEG>
struct ShEval {
  static constexpr int K = (DEG + 1) * (DEG + 1);
  // Y[k] of the unit direction (x, y, z): the unit-sphere forms of the
  // real harmonics' Cartesian polynomials.
  __device__ __forceinline__ static void basis(float x, float y, float z, float* Y) {
    Y[0] = kSH0;
    if (DEG < 1) return;
    Y[1] = kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = kSH1 * x;
    if (DEG < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSH2a * x * y;
    Y[5] = kSH2a * y * z;
    Y[6] = kSH2b * (3.f * zz - 1.f);
    Y[7] = kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    if (DEG < 3) return;
    Y[9] = kSH3e * y * (3.f * xx - yy);
    Y[10] = kSH3f * x * y * z;
    Y[11] = kSH3g * y * (5.f * zz - 1.f);
    Y[12] = kSH3h * z * (5.f * zz - 3.f);
    Y[13] = kSH3g * x * (5.f * zz - 1.f);
    Y[14] = kSH3k * z * (xx - yy);
    Y[15] = kSH3e * x * (xx - 3.f * yy);
  }
  // g += sum_k w[k] grad Y_k(x, y, z)
  __device__ __forceinline__ static void grad(float x, float y, float z, const float* w, float& gx,
                                              float& gy, float& gz) {
    gx = gy = gz = 0.f;
    if (DEG < 1) return;
    gy += kSH1 * w[1];
    gz += kSH1 * w[2];
    gx += kSH1 * w[3];
    if (DEG < 2) return;
    gx += kSH2a * (y * w[4] + z * w[7]) + 2.f * kSH2c * x * w[8];
    gy += kSH2a * (x * w[4] + z * w[5]) - 2.f * kSH2c * y * w[8];
    gz += kSH2a * (y * w[5] + x * w[7]) + 6.f * kSH2b * z * w[6];
    if (DEG < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += kSH3e * 6.f * x * y * w[9] + kSH3f * y * z * w[10] + kSH3g * (5.f * zz - 1.f) * w[13] +
          2.f * kSH3k * x * z * w[14] + kSH3e * 3.f * (xx - yy) * w[15];
    gy += kSH3e * 3.f * (xx - yy) * w[9] + kSH3f * x * z * w[10] + kSH3g * (5.f * zz - 1.f) * w[11] -
          2.f * kSH3k * y * z * w[14] - kSH3e * 6.f * x * y * w[15];
    gz += kSH3f * x * y * w[10] + 10.f * kSH3g * y * z * w[11] + kSH3h * (15.f * zz - 3.f) * w[12] +
          10.f * kSH3g * x * z * w[13] + kSH3k * (xx - yy) * w[14];
  }
};

// The batch's view records copied into shared memory by the whole block
// (ends with a block barrier).  The view loops read a record at every step,
// and there a load that misses L1 sits on the step's dependency chain.
__device__ __forceinline__ void stage_views(const ViewRec* views, int B, ViewRec* s_views) {
  static_assert(sizeof(ViewRec) % 4 == 0, "view records are copied as 32-bit words");
  const int words = B * (int)(sizeof(ViewRec) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(views);
  uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// View-independent part of the covariance: Sigma = M M^T with
// M = R(q / |q|) diag(exp(s)), computed once per Gaussian.
struct GaussCov {
  float s[3];    // exp(log-scale)
  float qn[4];   // normalised quaternion
  float qinv;    // 1 / |q|
  float Rq[9];   // rotation of the normalised quaternion
  float Sig[6];  // Sigma: 00 01 02 11 12 22
};

__device__ __forceinline__ void gauss_cov(const float* lsc, const float* quat, GaussCov& gc) {
  for (int i = 0; i < 3; i++) gc.s[i] = expf(lsc[i]);
  float qq = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
  gc.qinv = rsqrtf(qq);
  for (int i = 0; i < 4; i++) gc.qn[i] = quat[i] * gc.qinv;
  const float w = gc.qn[0], x = gc.qn[1], y = gc.qn[2], z = gc.qn[3];
  float* Q = gc.Rq;
  Q[0] = 1.f - 2.f * (y * y + z * z);
  Q[1] = 2.f * (x * y - w * z);
  Q[2] = 2.f * (x * z + w * y);
  Q[3] = 2.f * (x * y + w * z);
  Q[4] = 1.f - 2.f * (x * x + z * z);
  Q[5] = 2.f * (y * z - w * x);
  Q[6] = 2.f * (x * z - w * y);
  Q[7] = 2.f * (y * z + w * x);
  Q[8] = 1.f - 2.f * (x * x + y * y);
  float M[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) M[3 * i + j] = Q[3 * i + j] * gc.s[j];
  gc.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  gc.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  gc.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  gc.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  gc.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  gc.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// View-dependent part of one (view, Gaussian) projection.
struct ProjState {
  float tx, ty, tz;
  float ux, uy;       // clamped slopes used in J
  bool clx, cly;      // slope clamped
  float T[6];         // J W (2x3, row-major)
  float c00, c01, c11, det;
};

// Sigma' = J W Sigma W^T J^T + 0.3 I for one view (shared by forward and
// backward).
__device__ __forceinline__ void project_cov(const ViewRec& V, const float* mean, const float* Sig, float depth,
                                            ProjState& st) {
  const float* R = V.R;
  st.tx = fmaf(R[0], mean[0], fmaf(R[1], mean[1], fmaf(R[2], mean[2], V.t[0])));
  st.ty = fmaf(R[3], mean[0], fmaf(R[4], mean[1], fmaf(R[5], mean[2], V.t[1])));
  st.tz = depth;
  float ux = st.tx / st.tz, uy = st.ty / st.tz;
  st.clx = fabsf(ux) > V.limx;
  st.cly = fabsf(uy) > V.limy;
  st.ux = fminf(fmaxf(ux, -V.limx), V.limx);
  st.uy = fminf(fmaxf(uy, -V.limy), V.limy);

  const float itz = 1.f / st.tz;
  const float J00 = V.fx * itz, J02 = -V.fx * st.ux * itz;
  const float J11 = V.fy * itz, J12 = -V.fy * st.uy * itz;
  for (int j = 0; j < 3; j++) {
    st.T[j] = J00 * R[j] + J02 * R[6 + j];
    st.T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
  }
  // Sigma' = T Sigma T^T + 0.3 I
  const float* S = Sig;
  float a[3], b[3];  // a = Sigma T0^T, b = Sigma T1^T
  a[0] = S[0] * st.T[0] + S[1] * st.T[1] + S[2] * st.T[2];
  a[1] = S[1] * st.T[0] + S[3] * st.T[1] + S[4] * st.T[2];
  a[2] = S[2] * st.T[0] + S[4] * st.T[1] + S[5] * st.T[2];
  b[0] = S[0] * st.T[3] + S[1] * st.T[4] + S[2] * st.T[5];
  b[1] = S[1] * st.T[3] + S[3] * st.T[4] + S[4] * st.T[5];
  b[2] = S[2] * st.T[3] + S[4] * st.T[4] + S[5] * st.T[5];
  st.c00 = st.T[0] * a[0] + st.T[1] * a[1] + st.T[2] * a[2] + kDilation;
  st.c01 = st.T[3] * a[0] + st.T[4] * a[1] + st.T[5] * a[2];
  st.c11 = st.T[3] * b[0] + st.T[4] * b[1] + st.T[5] * b[2] + kDilation;
  st.det = st.c00 * st.c11 - st.c01 * st.c01;
}

template <int DEG>
__global__ void __launch_bounds__(256) project_fwd_kernel(ProjectArgs a) {
  constexpr int K = ShEval<DEG>::K;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = g < a.n;
  float mean[3], lsc[3], quat[4], op = 0.f, sh[3 * K];
  if (live) {
    const float* P = a.params;
    const int64_t S = a.stride;
#pragma unroll
    for (int i = 0; i < 3; i++) mean[i] = __ldg(P + i * S + g);
#pragma unroll
    for (int i = 0; i < 3; i++) lsc[i] = __ldg(P + (3 + i) * S + g);
#pragma unroll
    for (int i = 0; i < 4; i++) quat[i] = __ldg(P + (6 + i) * S + g);
    op = __ldg(P + 10 * S + g);
#pragma unroll
    for (int i = 0; i < 3 * K; i++) sh[i] = __ldg(P + (11 + i) * S + g);
  }
  const float opacity = 1.f / (1.f + expf(-op));
  GaussCov gc;
  gauss_cov(lsc, quat, gc);  // view-independent: once per Gaussian
  __shared__ float4 s_rec[8][32 * kRecStride];  // 256 threads: 8 warps x 32 records
  __shared__ uint32_t s_bsum[kMaxViews];          // the block's instance count per view
  __shared__ uint32_t s_vsum[kMaxViews];          // and its visible Gaussians per view
  __shared__ ViewRec s_views[kMaxViews];
  for (int i = threadIdx.x; i < a.B; i += blockDim.x) s_bsum[i] = s_vsum[i] = 0;
  stage_views(a.views, a.B, s_views);
  uint64_t vis = 0;  // views where the Gaussian touches a tile
  for (int v = 0; v < a.B; v++) {
    const ViewRec& V = s_views[v];
    const int64_t o = (int64_t)v * a.stride + g;
    uint32_t tiles = 0;
    bool touched = false;  // the 3-sigma rect meets the view
    int radius = 0;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;  // tile rect (half-open)
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    float depth = 0.f, blue = 0.f;
    float2 ex = make_float2(-3.0e38f, -3.0e38f);
    if (live) {
      depth = depth_key(V, mean[0], mean[1], mean[2]);
      if (depth > V.znear) {
        ProjState st;
        project_cov(V, mean, gc.Sig, depth, st);
        if (st.det != 0.f) {
          const float idet = 1.f / st.det;
          // lambda_max = mid + sqrt(max(0.1, mid^2 - det)); mid^2 - det is
          // evaluated as ((c00 - c11)/2)^2 + c01^2, the same quantity without
          // the cancellation of the difference form.
          const float mid = 0.5f * (st.c00 + st.c11);
          const float hd = 0.5f * (st.c00 - st.c11);
          const float lam = mid + sqrtf(fmaxf(0.1f, fmaf(hd, hd, st.c01 * st.c01)));
          radius = (int)ceilf(3.f * sqrtf(lam));
          const float mx = fmaf(V.fx, st.tx / st.tz, V.cx);
          const float my = fmaf(V.fy, st.ty / st.tz, V.cy);
          if (radius > 0 && tile_rect(V, mx, my, radius, x0, x1, y0, y1)) {
            touched = true;
            // colour
            float dx = mean[0] - V.campos[0], dy = mean[1] - V.campos[1], dz = mean[2] - V.campos[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv; dy *= inv; dz *= inv;
            float Y[K];
            ShEval<DEG>::basis(dx, dy, dz, Y);
            float rgb[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
              float acc = 0.5f;
#pragma unroll
              for (int k = 0; k < K; k++) acc = fmaf(sh[3 * k + c], Y[k], acc);
              rgb[c] = fmaxf(acc, 0.f);
            }
            // compositing form of the conic: p2 = cA dx^2 + cB dx dy + cC dy^2
            // is the exponent in base 2 (power * log2 e); hx, hy bound the
            // box around the ellipse where opacity * exp(power) >= 1/255
            // (d^T conic d <= 2 ln(255 opacity), whose extents are
            // sqrt(tau Sigma'_xx), sqrt(tau Sigma'_yy)), slightly widened.
            const float A = st.c11 * idet, Bc = -st.c01 * idet, C = st.c00 * idet;
            float hx = -3.0e38f, hy = -3.0e38f;  // never reaches 1/255
            const float t255 = 255.f * opacity;
            if (t255 > 1.f) {
              const float tau = 2.f * logf(t255) * 1.001f + 1e-3f;
              hx = sqrtf(tau * st.c00) * 1.001f + 0.01f;
              hy = sqrtf(tau * st.c11) * 1.001f + 0.01f;
            }
            r0 = make_float4(mx, my, -0.5f * kLog2e * A, -kLog2e * Bc);
            r1 = make_float4(-0.5f * kLog2e * C, opacity, rgb[0], rgb[1]);
            blue = rgb[2];
            ex = make_float2(hx, hy);
            // instances only in the rect's tiles that the alpha >= 1/255 box
            // reaches: the others hold no pixel where the Gaussian passes the
            // compositing kernels' box test, so no pixel changes without them
            int bx0, bx1, by0, by1;
            box_tiles(mx, hx, V.gw, bx0, bx1);
            box_tiles(my, hy, V.gh, by0, by1);
            x0 = max(x0, bx0);
            x1 = min(x1, bx1);
            y0 = max(y0, by0);
            y1 = min(y1, by1);
            if (x1 > x0 && y1 > y0) {
              tiles = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
            } else {
              x0 = x1 = y0 = y1 = 0;
            }
          } else {
            radius = 0;
            x0 = x1 = y0 = y1 = 0;
          }
        }
      }
      a.rec3[o] = make_int4(touched ? radius : 0, (int)tiles, x0 | (x1 << 16), y0 | (y1 << 16));
      a.tiles[o] = make_uint2(tiles, __float_as_uint(depth));
      vis |= touched ? 1ull << v : 0ull;
    }
    // the warp's 32 records (48 bytes each) go out through shared memory as
    // 96 coalesced 16-byte stores instead of 3 x 32 stores at a 48-byte stride
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* stage = s_rec[wid];
    __syncwarp();
    stage[3 * lane] = r0;
    stage[3 * lane + 1] = r1;
    stage[3 * lane + 2] = make_float4(blue, ex.x, ex.y, depth);
    __syncwarp();
    const int64_t g0 = g - lane;  // the warp's first Gaussian
    float4* dst = a.rec0 + kRecStride * ((int64_t)v * a.stride + g0);
#pragma unroll
    for (int m = 0; m < kRecStride; m++) {
      const int f = lane + 32 * m;
      if (g0 + f / kRecStride < a.n) dst[f] = stage[f];
    }
    const uint32_t wt = __reduce_add_sync(0xffffffffu, tiles);
    const uint32_t wv = (uint32_t)__popc(__ballot_sync(0xffffffffu, tiles != 0u));
    if (lane == 0 && wt) {
      atomicAdd(&s_bsum[v], wt);
      atomicAdd(&s_vsum[v], wv);
    }
  }
  if (live) a.vismask[g] = vis;
  // the block's instance and visible counts per view (for the per-view scans)
  __syncthreads();
  for (int i = threadIdx.x; i < a.B; i += blockDim.x) {
    a.block_sums[(int64_t)i * gridDim.x + blockIdx.x] = s_bsum[i];
    a.vis_sums[(int64_t)i * gridDim.x + blockIdx.x] = s_vsum[i];
  }
}

// Backward, colour part: dL/drgb per (view, Gaussian) -> dL/dSH and the
// part of dL/dmean that flows through the view direction.  Writes the SH
// gradient planes and initialises the mean planes.
//
// One thread per Gaussian takes all three channels: the view direction, the
// SH basis and the basis gradient are evaluated once per (view, Gaussian)
// and shared by the channels.  The direction gradient is linear in the
// per-channel weights gc_c sh_kc, so it is evaluated once on their sum over
// the unclamped channels.  The colour record of the next visible view but
// one is loaded while a view is processed.  The thread holds 96 values of
// its own (coefficients and their gradients): capped at 128 registers (4
// blocks, 16 warps per SM) it spills a few of them to L1, which measured
// faster than 160 registers and 12 warps.
template <int DEG>
__global__ void __launch_bounds__(128, 4) project_bwd_color_kernel(ProjectBwdArgs a) {
  constexpr int K = ShEval<DEG>::K;
  // camera centres of the batch's views
  __shared__ float4 s_cam[kMaxViews];
  for (int i = threadIdx.x; i < a.B; i += blockDim.x)
    s_cam[i] = make_float4(a.views[i].campos[0], a.views[i].campos[1], a.views[i].campos[2], 0.f);
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const float* P = a.params;
  const int64_t S = a.stride;
  // only the views where the Gaussian touches a tile have a nonzero 2D
  // gradient, and only their records are read; the parameters are loaded
  // without waiting for the mask (a Gaussian invisible in every view reads
  // them for nothing, but no load of the prologue waits on another)
  uint64_t vm = a.vismask[g];
  float mean[3], sh[3][K], gsh[3][K];
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      sh[c][k] = __ldg(P + (11 + 3 * k + c) * S + g);
      gsh[c][k] = 0.f;
    }
#pragma unroll
  for (int i = 0; i < 3; i++) mean[i] = __ldg(P + i * S + g);
  float gm[3] = {0.f, 0.f, 0.f};
  // dL/d(r, g, b) of (view v, Gaussian g): the colour record's first three floats
  const float4* gcol = reinterpret_cast<const float4*>(a.g2d + kG2dGeo * (int64_t)a.B * S) + g;
  auto next_view = [&]() {
    const int v = vm ? __ffsll((long long)vm) - 1 : -1;
    vm &= vm - 1;
    return v;
  };
  int v0 = next_view(), v1 = next_view();
  float4 c0 = v0 >= 0 ? __ldg(gcol + (int64_t)v0 * S) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 c1 = v1 >= 0 ? __ldg(gcol + (int64_t)v1 * S) : make_float4(0.f, 0.f, 0.f, 0.f);
  while (v0 >= 0) {
    const int v = v0;
    const float4 gc = c0;
    v0 = v1;
    c0 = c1;
    v1 = next_view();
    if (v1 >= 0) c1 = __ldg(gcol + (int64_t)v1 * S);
    if (gc.x == 0.f && gc.y == 0.f && gc.z == 0.f) continue;
    const float4 cam = s_cam[v];
    // rgb_c = max(0, 0.5 + sum_k sh_kc Y_k(d)), d = (mu - campos) / |mu - campos|
    float dx = mean[0] - cam.x, dy = mean[1] - cam.y, dz = mean[2] - cam.z;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[K];
    ShEval<DEG>::basis(dx, dy, dz, Y);
    const float gin[3] = {gc.x, gc.y, gc.z};
    float gcc[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < K; k++) acc = fmaf(sh[c][k], Y[k], acc);
      gcc[c] = acc < 0.f ? 0.f : gin[c];  // a clamped channel has no gradient
    }
    float wk[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
      for (int c = 0; c < 3; c++) gsh[c][k] = fmaf(gcc[c], Y[k], gsh[c][k]);
      wk[k] = fmaf(gcc[2], sh[2][k], fmaf(gcc[1], sh[1][k], gcc[0] * sh[0][k]));
    }
    float gdx, gdy, gdz;
    ShEval<DEG>::grad(dx, dy, dz, wk, gdx, gdy, gdz);
    const float dd = gdx * dx + gdy * dy + gdz * dz;
    gm[0] += (gdx - dx * dd) * inv;
    gm[1] += (gdy - dy * dd) * inv;
    gm[2] += (gdz - dz * dd) * inv;
  }
  float* G = a.grads;
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) G[(11 + 3 * k + c) * S + g] = gsh[c][k];
#pragma unroll
  for (int i = 0; i < 3; i++) G[i * S + g] = gm[i];
}

// Backward, geometry part: dL/d(mu2D, conic, opacity) per (view, Gaussian)
// -> dL/d(mean, log-scale, quaternion, opacity logit); adds to the mean
// planes written by the colour part.
__global__ void __launch_bounds__(128, 5) project_bwd_geom_kernel(ProjectBwdArgs a) {
  __shared__ ViewRec s_views[kMaxViews];
  stage_views(a.views, a.B, s_views);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const float* P = a.params;
  const int64_t S = a.stride;
  uint64_t vm = a.vismask[g];
  float* G = a.grads;
  float mean[3], lsc[3], quat[4];
#pragma unroll
  for (int i = 0; i < 3; i++) mean[i] = __ldg(P + i * S + g);
#pragma unroll
  for (int i = 0; i < 3; i++) lsc[i] = __ldg(P + (3 + i) * S + g);
#pragma unroll
  for (int i = 0; i < 4; i++) quat[i] = __ldg(P + (6 + i) * S + g);
  const float op = __ldg(P + 10 * S + g);  // (loaded before the mask is known, as above)
  if (!vm) {  // no tile in any view: every gradient of this Gaussian is zero
    // (the mean planes were written by the colour part)
#pragma unroll
    for (int i = 3; i < 11; i++) G[i * S + g] = 0.f;
    return;
  }
  const float opacity = 1.f / (1.f + expf(-op));

  GaussCov gc;
  gauss_cov(lsc, quat, gc);  // view-independent: once per Gaussian
  // dL/dSigma summed over the views: the chain from Sigma to the scale and
  // rotation is linear in it, so it runs once per Gaussian after the loop
  float gm[3] = {0.f, 0.f, 0.f}, gSig[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gop = 0.f;
  // prefetch the first view's six gradient values (the geometry record's
  // first float4 and the float2 after it)
  auto load6 = [&](int v, float (&q)[6]) {
    const float* r = a.g2d + kG2dGeo * ((int64_t)v * S + g);
    const float4 x = __ldg(reinterpret_cast<const float4*>(r));
    const float2 y = __ldg(reinterpret_cast<const float2*>(r + 4));
    q[0] = x.x; q[1] = x.y; q[2] = x.z; q[3] = x.w; q[4] = y.x; q[5] = y.y;
  };
  float cur[6], nxt[6];
  int vn = __ffsll((long long)vm) - 1;
  load6(vn, cur);
  // densification statistic: the screen-space mean gradient in normalised
  // device coordinates, summed over the views where the Gaussian touches a
  // tile, and the number of those views
  float dens_g = 0.f, dens_c = 0.f;
  while (vn >= 0) {  // the views where the Gaussian touches a tile
    const int v = vn;
    vm &= vm - 1;
    vn = vm ? __ffsll((long long)vm) - 1 : -1;
    if (vn >= 0) load6(vn, nxt);
    const float gmx = cur[0], gmy = cur[1], gA = cur[2], gB = cur[3], gC = cur[4], gsig = cur[5];
#pragma unroll
    for (int q = 0; q < 6; q++) cur[q] = nxt[q];
    if (a.dens_grad) {
      const ViewRec& Vd = s_views[v];
      const float nx = gmx * 0.5f * (float)Vd.W, ny = gmy * 0.5f * (float)Vd.H;
      dens_g += sqrtf(fmaf(nx, nx, ny * ny));
      dens_c += 1.f;
    }
    if (gmx == 0.f && gmy == 0.f && gA == 0.f && gB == 0.f && gC == 0.f && gsig == 0.f) continue;
    const ViewRec& V = s_views[v];
    const float depth = depth_key(V, mean[0], mean[1], mean[2]);
    if (!(depth > V.znear)) continue;
    ProjState st;
    project_cov(V, mean, gc.Sig, depth, st);

    // conic = (c11, -c01, c00) / det  ->  Sigma'
    const float id = 1.f / st.det, id2 = id * id;
    const float c00 = st.c00, c01 = st.c01, c11 = st.c11;
    const float gc00 = gA * (-c11 * c11 * id2) + gB * (c01 * c11 * id2) + gC * (id - c00 * c11 * id2);
    const float gc11 = gA * (id - c00 * c11 * id2) + gB * (c01 * c00 * id2) + gC * (-c00 * c00 * id2);
    const float gc01 = gA * (2.f * c11 * c01 * id2) + gB * (-id - 2.f * c01 * c01 * id2) +
                       gC * (2.f * c00 * c01 * id2);
    const float gh = 0.5f * gc01;
    // Sigma' = T Sigma T^T: dL/dSigma = T^T G T, dL/dT = 2 G T Sigma
    float GT[6];
#pragma unroll
    for (int j = 0; j < 3; j++) {
      GT[j] = gc00 * st.T[j] + gh * st.T[3 + j];
      GT[3 + j] = gh * st.T[j] + gc11 * st.T[3 + j];
    }
    const float* Sg = gc.Sig;
    const float Sfull[9] = {Sg[0], Sg[1], Sg[2], Sg[1], Sg[3], Sg[4], Sg[2], Sg[4], Sg[5]};
    float gT[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int b = 0; b < 3; b++)
        gT[3 * i + b] = 2.f * (GT[3 * i] * Sfull[b] + GT[3 * i + 1] * Sfull[3 + b] + GT[3 * i + 2] * Sfull[6 + b]);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) gSig[3 * i + j] += st.T[i] * GT[j] + st.T[3 + i] * GT[3 + j];
    // T = J W
    const float* R = V.R;
    const float gJ00 = gT[0] * R[0] + gT[1] * R[1] + gT[2] * R[2];
    const float gJ02 = gT[0] * R[6] + gT[1] * R[7] + gT[2] * R[8];
    const float gJ11 = gT[3] * R[3] + gT[4] * R[4] + gT[5] * R[5];
    const float gJ12 = gT[3] * R[6] + gT[4] * R[7] + gT[5] * R[8];
    const float itz = 1.f / st.tz, itz2 = itz * itz;
    float gtx = 0.f, gty = 0.f;
    float gtz = -gJ00 * V.fx * itz2 + gJ02 * V.fx * st.ux * itz2 - gJ11 * V.fy * itz2 + gJ12 * V.fy * st.uy * itz2;
    const float gux = -gJ02 * V.fx * itz, guy = -gJ12 * V.fy * itz;
    if (!st.clx) {
      gtx += gux * itz;
      gtz -= gux * st.tx * itz2;
    }
    if (!st.cly) {
      gty += guy * itz;
      gtz -= guy * st.ty * itz2;
    }
    // mu2D = (fx tx/tz + cx, fy ty/tz + cy)
    gtx += gmx * V.fx * itz;
    gty += gmy * V.fy * itz;
    gtz -= (gmx * V.fx * st.tx + gmy * V.fy * st.ty) * itz2;
    // t = W mu + tau
#pragma unroll
    for (int j = 0; j < 3; j++) gm[j] += R[j] * gtx + R[3 + j] * gty + R[6 + j] * gtz;
    gop += gsig * opacity * (1.f - opacity);
  }
  // Sigma = M M^T, M = Rq diag(s): dL/dM = (gS + gS^T) M
  float gR[9], gls[3];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    float gsj = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      float gMij = 0.f;
#pragma unroll
      for (int k = 0; k < 3; k++) gMij += (gSig[3 * i + k] + gSig[3 * k + i]) * gc.Rq[3 * k + j] * gc.s[j];
      gsj += gMij * gc.Rq[3 * i + j];
      gR[3 * i + j] = gMij * gc.s[j];
    }
    gls[j] = gsj * gc.s[j];
  }
  // rotation of the unit quaternion (w, x, y, z)
  const float w = gc.qn[0], x = gc.qn[1], y = gc.qn[2], z = gc.qn[3];
  float gqn[4];
  gqn[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
  gqn[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                  2.f * x * gR[8]);
  gqn[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                  2.f * y * gR[8]);
  gqn[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] +
                  y * gR[7]);
  const float dq = gqn[0] * gc.qn[0] + gqn[1] * gc.qn[1] + gqn[2] * gc.qn[2] + gqn[3] * gc.qn[3];
#pragma unroll
  for (int i = 0; i < 3; i++) G[i * S + g] += gm[i];
  if (a.dens_grad) {
    a.dens_grad[g] += dens_g;
    a.dens_count[g] += dens_c;
  }
#pragma unroll
  for (int i = 0; i < 3; i++) G[(3 + i) * S + g] = gls[i];
#pragma unroll
  for (int i = 0; i < 4; i++) G[(6 + i) * S + g] = (gqn[i] - gc.qn[i] * dq) * gc.qinv;
  G[10 * S + g] = gop;
}

void launch_project_fwd(const ProjectArgs& a, int deg, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  switch (deg) {
    case 0: project_fwd_kernel<0><<<blocks, threads, 0, s>>>(a); break;
    case 1: project_fwd_kernel<1><<<blocks, threads, 0, s>>>(a); break;
    case 2: project_fwd_kernel<2><<<blocks, threads, 0, s>>>(a); break;
    default: project_fwd_kernel<3><<<blocks, threads, 0, s>>>(a); break;
  }
}

int project_fwd_block() { return 256; }

void launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  switch (deg) {
    case 0: project_bwd_color_kernel<0><<<blocks, threads, 0, s>>>(a); break;
    case 1: project_bwd_color_kernel<1><<<blocks, threads, 0, s>>>(a); break;
    case 2: project_bwd_color_kernel<2><<<blocks, threads, 0, s>>>(a); break;
    default: project_bwd_color_kernel<3><<<blocks, threads, 0, s>>>(a); break;
  }
  project_bwd_geom_kernel<<<blocks, threads, 0, s>>>(a);
}

}  // namespace gs
