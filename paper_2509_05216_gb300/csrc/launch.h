// Kernel argument blocks and launchers (host side of the CUDA kernels).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

struct ProjectArgs {
  const float* params;
  int64_t n, stride;
  const ViewRec* views;
  int B;
  float4* rec0;
  float4* rec1;
  float4* rec2;
  int2* rec3;
  uint32_t* tiles;       // [B][stride]
  uint32_t* block_sums;  // [ceil(n / block)]
};

struct ProjectBwdArgs {
  const float* params;
  int64_t n, stride;
  const ViewRec* views;
  int B;
  const float* g2d;   // 9 planes of [B][stride]: dL/d(mu_x, mu_y, A, B, C, opacity, r, g, b)
  float* grads;       // [P][stride]
};

struct DuplicateArgs {
  int64_t n, stride;
  const ViewRec* views;
  int B;
  const float4* rec0;
  const float4* rec2;
  const int2* rec3;
  const uint32_t* tiles;
  const uint32_t* block_offsets;  // exclusive scan of the projection block sums
  uint64_t* keys;
  uint32_t* vals;
  int64_t capacity;
  int* status;
};

struct RasterArgs {
  const ViewRec* views;
  int B;
  int64_t stride;       // view stride of the records
  const uint2* ranges;  // [bins]
  const uint32_t* vals; // sorted Gaussian indices
  const float4* rec0;
  const float4* rec1;
  const float4* rec2;
  float* image;         // [B][3][H][W] concatenated
  float* tfinal;        // [pixels]
  uint32_t* nlast;      // [pixels]
  const float* dimage;  // backward only
  float* g2d;           // backward only: 9 planes of [B][stride]
};

int project_fwd_block();
void launch_project_fwd(const ProjectArgs& a, int deg, cudaStream_t s);
void launch_project_bwd(const ProjectBwdArgs& a, int deg, cudaStream_t s);

void launch_scan_block_sums(const uint32_t* sums, int64_t nb, uint32_t* offsets, uint64_t* total,
                            cudaStream_t s);
void launch_duplicate(const DuplicateArgs& a, cudaStream_t s);

// Radix sort of (key, value) pairs on key bits [0, 8 * npass_max) with the
// passes `pass_list` (digit positions, ascending).  Buffers ping-pong; returns
// 0 if the sorted result ends in (keys0, vals0), 1 if in (keys1, vals1).
size_t sort_lookback_bytes(int64_t count);
void launch_digit_histogram(const uint64_t* keys, int64_t count, int npass, uint32_t* hist, cudaStream_t s);
void launch_onesweep_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                          int64_t count, int digit, const uint32_t* hist_pass, uint32_t* lookback,
                          uint32_t* counter, int* status, cudaStream_t s);
void launch_tile_ranges(const uint64_t* keys, int64_t count, uint2* ranges, cudaStream_t s);

void launch_raster_fwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s);
void launch_raster_bwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s);

void launch_l1(const float* x, const float* y, int64_t count, float* partial, int nparts, float* loss,
               float* grad, cudaStream_t s);
int l1_parts(int64_t count);

struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t stride;
  int planes;
  float lr[64];  // per plane, already multiplied by 1 / (1 - beta1^t)
  float beta1, beta2, eps;
  float inv_sqrt_bc2;  // 1 / sqrt(1 - beta2^t)
};
void launch_adam(const AdamArgs& a, cudaStream_t s);

}  // namespace gs
