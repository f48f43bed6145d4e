// SSIM and PSNR of rendered views, and the D-SSIM term of the training loss.
//
// The paper judges its renders by PSNR and SSIM (Results, Tables II-III); the
// 3D-GS training it runs adds a D-SSIM term to the L1 loss:
//   L = (1 - lambda) mean |x - y| + lambda (1 - mean SSIM).
// SSIM uses the 11 x 11 Gaussian window (sigma 1.5) over each channel with
// zero padding, C1 = 0.01^2, C2 = 0.03^2:
//   s_p = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2)).
// Its gradient: with A, B, C the partial derivatives of s_p with respect to
// mx, E[x^2] and E[xy], dS/dx_q = E[A]_q + 2 x_q E[B]_q + y_q E[C]_q (the
// blur is linear and the window symmetric).
//
// Layout: one block per 32 x 16 output tile of one channel of one view.  The
// tile and a 5-pixel halo are staged in shared memory (zero outside the
// image), blurred horizontally into per-row sums, then vertically.  The
// forward writes A, B, C (three planes shaped like the image) and one
// partial sum per block; the backward blurs A, B, C the same way and writes
// dL/dx.  Per-view sums come from the blocks of each view in a fixed order.
#include <cmath>

#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

namespace {

constexpr int kTW = 32, kTH = 16;      // output tile
constexpr int kR = 5;                  // window radius
constexpr int kSW = kTW + 2 * kR, kSH = kTH + 2 * kR;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Tile {
  int v, c, x0, y0;
  const ViewRec* V;
};

// Block b -> (view, channel, tile); first[v] = the view's first block.
__device__ __forceinline__ Tile tile_of(const SsimArgs& a, int b) {
  int lo = 0, hi = a.B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.first_block[mid] <= b) lo = mid; else hi = mid - 1;
  }
  Tile t;
  t.v = lo;
  t.V = &a.views[lo];
  const int tx = (t.V->W + kTW - 1) / kTW, ty = (t.V->H + kTH - 1) / kTH;
  const int k = b - a.first_block[lo];
  t.c = k / (tx * ty);
  const int r = k % (tx * ty);
  t.x0 = (r % tx) * kTW;
  t.y0 = (r / tx) * kTH;
  return t;
}

// Stage a (kSH x kSW) window of up to three planes (zero outside the image).
template <int NM>
__device__ __forceinline__ void stage(const Tile& t, const float* const (&src)[NM], float (*s)[kSH][kSW]) {
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  for (int i = threadIdx.x; i < kSH * kSW; i += blockDim.x) {
    const int r = i / kSW, q = i % kSW;
    const int y = t.y0 + r - kR, x = t.x0 + q - kR;
    const bool in = x >= 0 && x < V.W && y >= 0 && y < V.H;
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
#pragma unroll
    for (int m = 0; m < NM; m++) s[m][r][q] = in ? __ldg(src[m] + o) : 0.f;
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
  return t;
}

}  // namespace

// Forward: the SSIM map's partials A, B, C per pixel and, per block, the
// sums of the SSIM map, |x - y| and (x - y)^2 over its pixels.
__global__ void __launch_bounds__(256) ssim_fwd_kernel(SsimArgs a) {
  __shared__ float s_in[2][kSH][kSW];
  __shared__ float s_h[5][kSH][kTW];
  __shared__ double red[8];
  const Tile t = tile_of(a, blockIdx.x);
  const float* const src[2] = {a.x, a.y};
  stage<2>(t, src, s_in);
  __syncthreads();
  // horizontal sums of x, y, x^2, y^2, xy
  for (int i = threadIdx.x; i < kSH * kTW; i += blockDim.x) {
    const int r = i / kTW, q = i % kTW;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + 1; k++) {
      const float x = s_in[0][r][q + k], y = s_in[1][r][q + k], w = a.win[k];
      h0 = fmaf(w, x, h0);
      h1 = fmaf(w, y, h1);
      h2 = fmaf(w, x * x, h2);
      h3 = fmaf(w, y * y, h3);
      h4 = fmaf(w, x * y, h4);
    }
    s_h[0][r][q] = h0;
    s_h[1][r][q] = h1;
    s_h[2][r][q] = h2;
    s_h[3][r][q] = h3;
    s_h[4][r][q] = h4;
  }
  __syncthreads();
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  double ssum = 0.0, asum = 0.0, qsum = 0.0;
  for (int i = threadIdx.x; i < kTH * kTW; i += blockDim.x) {
    const int r = i / kTW, q = i % kTW;
    const int x = t.x0 + q, y = t.y0 + r;
    if (x >= V.W || y >= V.H) continue;
    float e[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2 * kR + 1; k++)
#pragma unroll
      for (int m = 0; m < 5; m++) e[m] = fmaf(a.win[k], s_h[m][r + k][q], e[m]);
    const float mx = e[0], my = e[1];
    const float sxx = e[2] - mx * mx, syy = e[3] - my * my, sxy = e[4] - mx * my;
    const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
    const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
    const float D = d1 * d2;
    const float s = n1 * n2 / D;
    const float A = (2.f * my * (n2 - n1) - s * 2.f * mx * (d2 - d1)) / D;
    const float Bp = -s / d2;
    const float Cp = 2.f * n1 / D;
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
    const int64_t total = a.count;
    a.partials[o] = A;
    a.partials[total + o] = Bp;
    a.partials[2 * total + o] = Cp;
    const float d = s_in[0][r + kR][q + kR] - s_in[1][r + kR][q + kR];
    ssum += s;
    asum += fabsf(d);
    qsum += (double)d * d;
  }
  const double bs = block_sum(ssum, red);
  __syncthreads();
  const double ba = block_sum(asum, red);
  __syncthreads();
  const double bq = block_sum(qsum, red);
  if (threadIdx.x == 0) {
    a.block_sums[3 * (int64_t)blockIdx.x] = bs;
    a.block_sums[3 * (int64_t)blockIdx.x + 1] = ba;
    a.block_sums[3 * (int64_t)blockIdx.x + 2] = bq;
  }
}

// Backward: dL/dx = (1 - lambda) sign(x - y) / count - lambda dS/dx / count.
__global__ void __launch_bounds__(256) ssim_bwd_kernel(SsimArgs a) {
  __shared__ float s_in[3][kSH][kSW];
  __shared__ float s_h[3][kSH][kTW];
  const Tile t = tile_of(a, blockIdx.x);
  const int64_t total = a.count;
  const float* const src[3] = {a.partials, a.partials + total, a.partials + 2 * total};
  stage<3>(t, src, s_in);
  __syncthreads();
  for (int i = threadIdx.x; i < kSH * kTW; i += blockDim.x) {
    const int r = i / kTW, q = i % kTW;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + 1; k++) {
      const float w = a.win[k];
      h0 = fmaf(w, s_in[0][r][q + k], h0);
      h1 = fmaf(w, s_in[1][r][q + k], h1);
      h2 = fmaf(w, s_in[2][r][q + k], h2);
    }
    s_h[0][r][q] = h0;
    s_h[1][r][q] = h1;
    s_h[2][r][q] = h2;
  }
  __syncthreads();
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  for (int i = threadIdx.x; i < kTH * kTW; i += blockDim.x) {
    const int r = i / kTW, q = i % kTW;
    const int x = t.x0 + q, y = t.y0 + r;
    if (x >= V.W || y >= V.H) continue;
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * kR + 1; k++) {
      const float w = a.win[k];
      e0 = fmaf(w, s_h[0][r + k][q], e0);
      e1 = fmaf(w, s_h[1][r + k][q], e1);
      e2 = fmaf(w, s_h[2][r + k][q], e2);
    }
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
    const float xv = __ldg(a.x + o), yv = __ldg(a.y + o);
    const float dS = e0 + 2.f * xv * e1 + yv * e2;
    const float d = xv - yv;
    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    a.grad[o] = (a.w_l1 * sg - a.w_ssim * dS) * a.inv_count;
  }
}

// Per-view sums of the block sums: block v of the grid adds view v's block
// sums (a strided subset per thread, then a tree: a fixed order).
// out_view[3 v + m]: view v's sums of the SSIM map (m = 0), |x - y| (1) and
// (x - y)^2 (2).
__global__ void __launch_bounds__(256) ssim_view_sums_kernel(SsimArgs a, double* out_view) {
  __shared__ double red[3][8];
  const int v = blockIdx.x;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = a.first_block[v] + (int)threadIdx.x; b < a.first_block[v + 1]; b += blockDim.x)
#pragma unroll
    for (int m = 0; m < 3; m++) s[m] += a.block_sums[3 * (int64_t)b + m];
#pragma unroll
  for (int m = 0; m < 3; m++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s[m] += __shfl_down_sync(0xffffffffu, s[m], off);
    if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = s[m];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[threadIdx.x][w];
    out_view[3 * v + threadIdx.x] = t;
  }
}

// *loss = w_l1 sum|x - y| / count + w_ssim (1 - sum s / count), views in order.
__global__ void ssim_loss_kernel(SsimArgs a, const double* out_view, float* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0, l1 = 0.0;
  for (int v = 0; v < a.B; v++) {
    s += out_view[3 * v];
    l1 += out_view[3 * v + 1];
  }
  const double cnt = (double)a.count;
  *loss = (float)(a.w_l1_d * l1 / cnt + a.w_ssim_d * (1.0 - s / cnt));
}

int ssim_blocks_of_view(int W, int H) { return 3 * ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH); }

void ssim_window(float* w) {
  double g[2 * kR + 1], sum = 0.0;
  for (int k = 0; k <= 2 * kR; k++) {
    const double d = (double)(k - kR);
    g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += g[k];
  }
  for (int k = 0; k <= 2 * kR; k++) w[k] = (float)(g[k] / sum);
}

void launch_ssim(const SsimArgs& a, int blocks, bool backward, double* out_view, float* loss, cudaStream_t s) {
  if (blocks <= 0) return;
  ssim_fwd_kernel<<<blocks, 256, 0, s>>>(a);
  ssim_view_sums_kernel<<<a.B, 256, 0, s>>>(a, out_view);
  if (loss) ssim_loss_kernel<<<1, 32, 0, s>>>(a, out_view, loss);
  if (backward) ssim_bwd_kernel<<<blocks, 256, 0, s>>>(a);
}

}  // namespace gs
