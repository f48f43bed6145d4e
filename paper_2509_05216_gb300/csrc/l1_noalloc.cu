// Allocation-free variant of the L1 loss (gs_l1_loss_noalloc).
//
// The regular gs_l1_loss keeps its per-block partial sums in a buffer that its
// context allocates with cudaMalloc on first use.  Some callers cannot allow
// that: a host application that hands this library a fixed slice of device
// memory and forbids any further device allocation, a real-time render or
// training loop that must not allocate (and so never synchronise the device)
// once it runs, or a plugin whose host owns every allocation.  This variant
// takes no context and allocates nothing: its partial sums live in the
// file-scope array below, which exists once per GPU that loads the library
// and stays until the process exits.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int64_t kNoAllocChunk = 65536;  // elements reduced by one block
constexpr int kNoAllocMaxParts = 4096;    // partial sums held by the scratch array
constexpr int64_t kNoAllocMaxCount = kNoAllocChunk * kNoAllocMaxParts;  // 268,435,456
constexpr int kMaxDevices = 64;

// 16 KiB of partial sums, shared by every call on the same GPU.
static __device__ __align__(256) float g_l1_partials[kNoAllocMaxParts];

// Block b reduces elements [b * chunk, (b + 1) * chunk) and writes slot b.
__global__ void __launch_bounds__(kNoAllocThreads) l1_chunk_kernel(const float* __restrict__ x,
                                                                   const float* __restrict__ y, int64_t count,
                                                                   float inv_count, float* __restrict__ grad,
                                                                   float* __restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * kNoAllocChunk;
  const int64_t end = base + kNoAllocChunk < count ? base + kNoAllocChunk : count;
  float s = 0.f;
  for (int64_t i = base + threadIdx.x; i < end; i += kNoAllocThreads) {
    const float d = x[i] - y[i];
    s += fabsf(d);
    if (grad) grad[i] = d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f);
  }
  __shared__ float red[kNoAllocThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kNoAllocThreads / 32; w++) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void l1_chunk_finish_kernel(const float* __restrict__ partials, int nparts, double inv_count,
                                       float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; i++) t += partials[i];
    *loss = (float)(t * inv_count);
  }
}

// Device address of g_l1_partials per device, looked up once per device with
// that device current (host code cannot use the array's name as a pointer).
std::mutex g_setup_lock;
float* g_partials_addr[kMaxDevices] = {};

gs_status partials_for_current_device(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return GS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_lock);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_l1_partials);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return GS_ECUDA;
    }
    g_partials_addr[dev] = static_cast<float*>(p);
  }
  *out = g_partials_addr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_l1_loss_noalloc(const float* x, const float* y, int64_t count, float* loss, float* dL_dx,
                                        void* stream) {
  if (!x || !y || count <= 0) return GS_EINVAL;
  if (count > kNoAllocMaxCount) return GS_EINVAL;
  float* partials = nullptr;
  const gs_status st = partials_for_current_device(&partials);
  if (st != GS_OK) return st;
  const int nparts = (int)((count + kNoAllocChunk - 1) / kNoAllocChunk);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  l1_chunk_kernel<<<nparts, kNoAllocThreads, 0, s>>>(x, y, count, (float)(1.0 / (double)count), dL_dx, partials);
  if (loss) l1_chunk_finish_kernel<<<1, 32, 0, s>>>(partials, nparts, 1.0 / (double)count, loss);
  if (cudaGetLastError() != cudaSuccess) return GS_ECUDA;
  return GS_OK;
}
