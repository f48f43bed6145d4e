// L1 photometric loss and the Adam update.
//
// The paper fits the Gaussians to the orbit views (Section III); the loss is
// the mean absolute error between rendered and target images and the
// optimiser is Adam with bias correction (torch.optim.Adam semantics), one
// learning rate per parameter group.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

constexpr int kL1Threads = 256;

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    (void)cudaGetLastError();
    sms = 1;  // only sizes grids; any positive value is correct
  }
  if (dev >= 0 && dev < 64) cached[dev] = sms;
  return sms;
}

int l1_parts(int64_t count) {
  int64_t parts = (count + kL1Threads * 16 - 1) / (kL1Threads * 16);
  if (parts < 1) parts = 1;
  const int64_t most = (int64_t)sm_count() * 8;
  if (parts > most) parts = most;
  return (int)parts;
}

__global__ void __launch_bounds__(kL1Threads) l1_kernel(const float* __restrict__ x, const float* y_arg,
                                                        const float* const* y_slot, int64_t count, float inv_count,
                                                        float* __restrict__ grad, float* __restrict__ partial) {
  // the target pointer comes from device memory when given through a slot
  // (a captured training step reads each batch's targets there)
  const float* __restrict__ y = y_slot ? *y_slot : y_arg;
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = x[i] - y[i];
    s += fabsf(d);
    if (grad) grad[i] = d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f);
  }
  __shared__ float red[kL1Threads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kL1Threads / 32; w++) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void l1_finish_kernel(const float* __restrict__ partial, int nparts, double inv_count, float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; i++) t += partial[i];
    *loss = (float)(t * inv_count);
  }
}

void launch_l1(const float* x, const float* y, const float* const* y_slot, int64_t count, float* partial,
               int nparts, float* loss, float* grad, cudaStream_t s) {
  const float inv = (float)(1.0 / (double)count);
  l1_kernel<<<nparts, kL1Threads, 0, s>>>(x, y, y_slot, count, inv, grad, partial);
  if (loss) l1_finish_kernel<<<1, 32, 0, s>>>(partial, nparts, 1.0 / (double)count, loss);
}

// Adam over [planes][stride] float planes.  A thread owns one float4 column
// (4 consecutive Gaussians) and walks the planes, so the per-plane learning
// rate is uniform across the warp and, in the visible-only variant, the
// column's visibility is read once: a column of 4 invisible Gaussians reads
// and writes nothing; otherwise invisible lanes write their values back
// unchanged.
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
  // step-dependent constants come from device memory, so the launch can be
  // captured once and replayed for any step
  __shared__ float lr_s[64];
  __shared__ float isb2_s;
  if (threadIdx.x < 64) lr_s[threadIdx.x] = a.consts[threadIdx.x];
  if (threadIdx.x == 0) isb2_s = a.consts[64];
  __syncthreads();
  AdamStep st;
  st.b1 = a.beta1;
  st.b2 = a.beta2;
  st.c1 = 1.f - a.beta1;
  st.c2 = 1.f - a.beta2;
  st.eps = a.eps;
  st.isb2 = isb2_s;
  const int64_t cols = a.stride / 4;
  float4* p4 = reinterpret_cast<float4*>(a.p);
  const float4* g4 = reinterpret_cast<const float4*>(a.g);
  float4* m4 = reinterpret_cast<float4*>(a.m);
  float4* v4 = reinterpret_cast<float4*>(a.v);
  for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
       col += (int64_t)gridDim.x * blockDim.x) {
    bool on[4] = {true, true, true, true};
    if (a.vismask) {
      const ulonglong2 q0 = reinterpret_cast<const ulonglong2*>(a.vismask)[2 * col];
      const ulonglong2 q1 = reinterpret_cast<const ulonglong2*>(a.vismask)[2 * col + 1];
      on[0] = q0.x != 0ull;
      on[1] = q0.y != 0ull;
      on[2] = q1.x != 0ull;
      on[3] = q1.y != 0ull;
      if (!(on[0] || on[1] || on[2] || on[3])) continue;
    }
    for (int pl = 0; pl < a.planes; pl++) {
      const int64_t i = pl * cols + col;
      const float lr = lr_s[pl];
      const float4 g = g4[i];
      const float4 m0 = m4[i], v0 = v4[i], p0 = p4[i];
      float4 m = m0, v = v0, p = p0;
#define ADAM_LANE(f, k)                \
  adam_scalar(p.f, m.f, v.f, g.f, lr, st); \
  if (!on[k]) { m.f = m0.f; v.f = v0.f; p.f = p0.f; }
      ADAM_LANE(x, 0) ADAM_LANE(y, 1) ADAM_LANE(z, 2) ADAM_LANE(w, 3)
#undef ADAM_LANE
      m4[i] = m;
      v4[i] = v;
      p4[i] = p;
    }
  }
}

void launch_adam(const AdamArgs& a, cudaStream_t s) {
  const int64_t cols = a.stride / 4;
  int64_t blocks = (cols + 255) / 256;
  const int64_t most = (int64_t)sm_count() * 16;
  if (blocks > most) blocks = most;
  if (blocks < 1) blocks = 1;
  adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
}

}  // namespace gs
