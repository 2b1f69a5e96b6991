// Loading of R band spectra into the plan's resident layout.
//
// The caller's rows (nrec complex values) are copied into rows padded to
// r_pad (the padding stays zero), by a kernel that reads either device
// memory or pinned host memory directly (mapped into the device address
// space), so a host load is one pass over the interconnect with no staging
// copy.  (Implementation section: the reflection data is read, transformed
// and kept for all iterations; here it stays resident in HBM.)

#include "mk_internal.h"
#include "mk_rstore.cuh"

namespace mk {
namespace {

// Rows of complex FP32 into the 16-bit storage of the tensor-core path
// (conversion rules in store_r16).  Output rows have 2 r_pad 16-bit values.
__global__ void __launch_bounds__(256) load_rows_q_kernel(const float2* __restrict__ src, SurveyDev s,
                                                         int64_t row0, int64_t rows) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nrec = s.nr;
  for (int64_t row = warp; row < rows; row += nwarps) {
    const float2* sr = src + row * nrec;
    const int64_t o = (row0 + row) * s.r_pad;  // in complex elements
    for (int i = lane; i < nrec; i += 32) store_r16(s, s.rprec, o + i, __ldg(sr + i));
  }
}

__global__ void __launch_bounds__(256) load_rows_c64_kernel(const float2* __restrict__ src, float2* __restrict__ dst,
                                                           int64_t rows, int nrec, int r_pad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < rows; row += nwarps) {
    const float2* sr = src + row * nrec;
    float2* dr = dst + row * r_pad;
#pragma unroll 4
    for (int i = lane; i < nrec; i += 32) dr[i] = __ldg(sr + i);
  }
}

}  // namespace

// The row loads run beside the contraction and the epilogue when R is loaded
// asynchronously: they ask for the shared-memory-heavy carveout those kernels
// use, so that an SM can hold both (kernels whose carveouts differ cannot
// share an SM until it drains).
cudaError_t prepare_load() {
  cudaError_t e = cudaFuncSetAttribute(load_rows_c64_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(load_rows_q_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_load_rows_q(const float2* src, const SurveyDev& s, int64_t row0, int64_t rows, cudaStream_t st,
                               int max_blocks) {
  int64_t grid = (rows + 7) / 8;
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  load_rows_q_kernel<<<(unsigned)grid, 256, 0, st>>>(src, s, row0, rows);
  return cudaGetLastError();
}

cudaError_t launch_load_rows(const float2* src, float2* dst, int64_t rows, int nrec, int r_pad, cudaStream_t st,
                             int max_blocks) {
  int64_t grid = (rows + 7) / 8;
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  load_rows_c64_kernel<<<(unsigned)grid, 256, 0, st>>>(src, dst, rows, nrec, r_pad);
  return cudaGetLastError();
}

}  // namespace mk
