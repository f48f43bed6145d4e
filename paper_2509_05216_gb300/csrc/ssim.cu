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
// Layout: one block (256 threads) per 32 x 32 output tile of one channel of
// one view.  The tile and a 5-pixel halo are staged in shared memory (zero
// outside the image); a horizontal pass (a thread slides the 11-tap window
// over 4 adjacent columns of one row, so each input is loaded once per 4
// outputs) writes per-row sums, and a vertical pass (a thread slides down 4
// adjacent rows of one column) forms the window sums.  The forward writes
// A, B, C (three planes shaped like the image) and one partial sum per
// block; the backward blurs A, B, C the same way and writes dL/dx.  Per-view
// sums come from the blocks of each view in a fixed order.
#include <cmath>

#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

namespace {

constexpr int kT = 32;                 // output tile (kT x kT)
constexpr int kR = 5;                  // window radius
constexpr int kS = kT + 2 * kR;        // staged rows / columns
constexpr int kCols = 4, kRows = 4;    // outputs per thread in each pass
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
  const int tx = (t.V->W + kT - 1) / kT, ty = (t.V->H + kT - 1) / kT;
  const int k = b - a.first_block[lo];
  t.c = k / (tx * ty);
  const int r = k % (tx * ty);
  t.x0 = (r % tx) * kT;
  t.y0 = (r / tx) * kT;
  return t;
}

// Stage a kS x kS window of NM planes (zero outside the image).
template <int NM>
__device__ __forceinline__ void stage(const Tile& t, const float* const (&src)[NM], float (*s)[kS][kS]) {
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  for (int i = threadIdx.x; i < kS * kS; i += blockDim.x) {
    const int r = i / kS, q = i % kS;
    const int y = t.y0 + r - kR, x = t.x0 + q - kR;
    const bool in = x >= 0 && x < V.W && y >= 0 && y < V.H;
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
#pragma unroll
    for (int m = 0; m < NM; m++) s[m][r][q] = in ? __ldg(src[m] + o) : 0.f;
  }
}

// Horizontal pass: h[m][r][q] = sum_k w_k f_m(r, q + k) for the NM staged
// planes, where with PROD the five functions are x, y, x^2, y^2, xy of the
// two staged planes (forward) and otherwise the staged planes themselves.
template <int NM, int NH, bool PROD>
__device__ __forceinline__ void hpass(const float (&win)[2 * kR + 1], const float (*s)[kS][kS], float (*h)[kS][kT]) {
  for (int i = threadIdx.x; i < kS * (kT / kCols); i += blockDim.x) {
    const int r = i / (kT / kCols), q0 = (i % (kT / kCols)) * kCols;
    float acc[NH][kCols];
#pragma unroll
    for (int m = 0; m < NH; m++)
#pragma unroll
      for (int c = 0; c < kCols; c++) acc[m][c] = 0.f;
#pragma unroll
    for (int j = 0; j < 2 * kR + kCols; j++) {  // input column q0 + j
      float f[NH];
      if constexpr (PROD) {
        const float x = s[0][r][q0 + j], y = s[1][r][q0 + j];
        f[0] = x; f[1] = y; f[2] = x * x; f[3] = y * y; f[4] = x * y;
      } else {
#pragma unroll
        for (int m = 0; m < NH; m++) f[m] = s[m][r][q0 + j];
      }
#pragma unroll
      for (int c = 0; c < kCols; c++) {
        const int k = j - c;  // tap of output column q0 + c
        if (k >= 0 && k <= 2 * kR) {
#pragma unroll
          for (int m = 0; m < NH; m++) acc[m][c] = fmaf(win[k], f[m], acc[m][c]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < NH; m++)
#pragma unroll
      for (int c = 0; c < kCols; c++) h[m][r][q0 + c] = acc[m][c];
  }
}

// Vertical pass for the kRows outputs of one thread: e[m][j] = sum_k w_k
// h[m][r0 + j + k][q].
template <int NH>
__device__ __forceinline__ void vpass(const float (&win)[2 * kR + 1], const float (*h)[kS][kT], int r0, int q,
                                      float (&e)[NH][kRows]) {
#pragma unroll
  for (int m = 0; m < NH; m++)
#pragma unroll
    for (int j = 0; j < kRows; j++) e[m][j] = 0.f;
#pragma unroll
  for (int i = 0; i < 2 * kR + kRows; i++) {  // h row r0 + i
#pragma unroll
    for (int m = 0; m < NH; m++) {
      const float f = h[m][r0 + i][q];
#pragma unroll
      for (int j = 0; j < kRows; j++) {
        const int k = i - j;
        if (k >= 0 && k <= 2 * kR) e[m][j] = fmaf(win[k], f, e[m][j]);
      }
    }
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
  __shared__ float s_in[2][kS][kS];
  __shared__ float s_h[5][kS][kT];
  __shared__ double red[8];
  const Tile t = tile_of(a, blockIdx.x);
  const float* const src[2] = {a.x, a.y};
  stage<2>(t, src, s_in);
  __syncthreads();
  hpass<2, 5, true>(a.win, s_in, s_h);
  __syncthreads();
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  const int q = threadIdx.x % kT, r0 = (threadIdx.x / kT) * kRows;
  float e[5][kRows];
  vpass<5>(a.win, s_h, r0, q, e);
  float ssum = 0.f, asum = 0.f, qsum = 0.f;  // at most kRows terms each
  const int64_t total = a.count;
  const int x = t.x0 + q;
#pragma unroll
  for (int j = 0; j < kRows; j++) {
    const int y = t.y0 + r0 + j;
    if (x >= V.W || y >= V.H) continue;
    const float mx = e[0][j], my = e[1][j];
    const float sxx = e[2][j] - mx * mx, syy = e[3][j] - my * my, sxy = e[4][j] - mx * my;
    const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
    const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
    const float D = d1 * d2;
    const float s = n1 * n2 / D;
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
    a.partials[o] = (2.f * my * (n2 - n1) - s * 2.f * mx * (d2 - d1)) / D;  // dS/d(mx)
    a.partials[total + o] = -s / d2;                                       // dS/dE[x^2]
    a.partials[2 * total + o] = 2.f * n1 / D;                              // dS/dE[xy]
    const float d = s_in[0][r0 + j + kR][q + kR] - s_in[1][r0 + j + kR][q + kR];
    ssum += s;
    asum += fabsf(d);
    qsum = fmaf(d, d, qsum);
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
  __shared__ float s_in[3][kS][kS];
  __shared__ float s_h[3][kS][kT];
  const Tile t = tile_of(a, blockIdx.x);
  const int64_t total = a.count;
  const float* const src[3] = {a.partials, a.partials + total, a.partials + 2 * total};
  stage<3>(t, src, s_in);
  __syncthreads();
  hpass<3, 3, false>(a.win, s_in, s_h);
  __syncthreads();
  const ViewRec& V = *t.V;
  const int64_t plane = (int64_t)V.W * V.H;
  const int q = threadIdx.x % kT, r0 = (threadIdx.x / kT) * kRows;
  float e[3][kRows];
  vpass<3>(a.win, s_h, r0, q, e);
  const int x = t.x0 + q;
#pragma unroll
  for (int j = 0; j < kRows; j++) {
    const int y = t.y0 + r0 + j;
    if (x >= V.W || y >= V.H) continue;
    const int64_t o = 3 * V.pix_offset + t.c * plane + (int64_t)y * V.W + x;
    const float xv = __ldg(a.x + o), yv = __ldg(a.y + o);
    const float dS = e[0][j] + 2.f * xv * e[1][j] + yv * e[2][j];
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

int ssim_blocks_of_view(int W, int H) { return 3 * ((W + kT - 1) / kT) * ((H + kT - 1) / kT); }

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
