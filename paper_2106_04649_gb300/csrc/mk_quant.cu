// Scaled FP16 split (MK_R_SPLIT_F16): the contraction of Eq. (1) on the
// tensor cores with both operands split into FP16 hi + lo parts, 3 products
// (hh, hl, lh).  FP16 keeps 11 significant bits per part, 22 with the lo
// part, but only within its normal range (2^-14 .. 65504); so R_m is scaled
// by a power of two per frequency and the field spectrum by a power of two
// per (frequency, focal point) that bring their largest magnitude into
// [2^14, 2^15).  Powers of two scale exactly; the contraction divides them
// out of each output (mk_umma.cu).
//
//  * r_amax_kernel / r_scale_kernel: the scale of each frequency of R from
//    the largest |Re| or |Im| of its rows, before they are converted
//    (mk_rstore.cuh, store_r16 with q = 5);
//  * quantize_kernel: at every contraction, per (frequency, focal point) row
//    of the complex FP32 field spectrum Nw written by the epilogue, its scale
//    and its 2-part FP16 embedding (rows 2f = (Nr, -Ni), 2f+1 = (Ni, Nr), the
//    B operand layout of the tensor-core contraction).

#include <cuda_fp16.h>

#include "mk_embed.cuh"
#include "mk_internal.h"

namespace mk {
namespace {

// one warp per row of nrec complex values of the caller's R; bin of global
// row g = g / ns
__global__ void __launch_bounds__(256) r_amax_kernel(const float2* __restrict__ src, SurveyDev s, int64_t row0,
                                                    int64_t rows) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < rows; row += nwarps) {
    const float2* sr = src + row * s.nr;
    float mx = 0.f;
    for (int i = lane; i < s.nr; i += 32) {
      const float2 v = __ldg(sr + i);
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // non-negative floats order like their bit patterns
    if (lane == 0) atomicMax(reinterpret_cast<unsigned*>(s.rsc) + (row0 + row) / s.ns, __float_as_uint(mx));
  }
}

__global__ void r_scale_kernel(float* rsc, int w_begin, int w_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < w_count) rsc[w_begin + i] = f16_scale(__uint_as_float(reinterpret_cast<unsigned*>(rsc)[w_begin + i]));
}

// one warp per (m, f) row of Nw (r_pad values, the padding zero)
__global__ void __launch_bounds__(256) quantize_kernel(SurveyDev s) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nrows = (int64_t)s.nw * s.F;
  uint32_t* b0 = reinterpret_cast<uint32_t*>(s.Bq0);
  uint32_t* b1 = reinterpret_cast<uint32_t*>(s.Bq1);
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const int m = (int)(row / s.F), f = (int)(row - (int64_t)m * s.F);
    const float2* src = s.Nw + (int64_t)m * s.nw_stride + (int64_t)f * s.r_pad;
    float mx = 0.f;
    for (int i = lane; i < s.r_pad; i += 32) {
      const float2 v = src[i];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float sc = f16_scale(mx);
    if (lane == 0) s.nsc[row] = sc;
    const int64_t w0 = ((int64_t)m * 2 * s.F + 2 * f) * s.r_pad;  // 32-bit word of row 2f, position 0
    for (int i = lane; i < s.r_pad; i += 32) {
      const float2 v = src[i];
      float hr, hi, lr, li;
      const uint32_t h = round_pair<false>(v.x * sc, v.y * sc, hr, hi);
      const uint32_t l = round_pair<false>(v.x * sc - hr, v.y * sc - hi, lr, li);
      b0[w0 + i] = pair_neg_hi(h);
      b0[w0 + s.r_pad + i] = pair_swap(h);
      b1[w0 + i] = pair_neg_hi(l);
      b1[w0 + s.r_pad + i] = pair_swap(l);
    }
  }
}

}  // namespace

cudaError_t launch_r_amax(const float2* src, const SurveyDev& s, int64_t row0, int64_t rows, cudaStream_t st,
                          int max_blocks) {
  int64_t grid = (rows + 7) / 8;
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  r_amax_kernel<<<(unsigned)grid, 256, 0, st>>>(src, s, row0, rows);
  return cudaGetLastError();
}

cudaError_t launch_r_scale(const SurveyDev& s, int w_begin, int w_count, cudaStream_t st) {
  r_scale_kernel<<<(w_count + 255) / 256, 256, 0, st>>>(s.rsc, w_begin, w_count);
  return cudaGetLastError();
}

cudaError_t launch_quantize_field(const SurveyDev& s, cudaStream_t st, int num_sms) {
  const int64_t rows = (int64_t)s.nw * s.F;
  int64_t grid = (rows + 7) / 8;
  if (grid > (int64_t)num_sms * 8) grid = (int64_t)num_sms * 8;
  quantize_kernel<<<(unsigned)grid, 256, 0, st>>>(s);
  return cudaGetLastError();
}

}  // namespace mk
