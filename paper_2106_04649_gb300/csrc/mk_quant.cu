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

// The 2-part FP16 embedding of two consecutive values (a, b) of one row,
// scaled by sc, as 8-byte stores into rows 2f and 2f+1 of both parts.
__device__ __forceinline__ void put_pair(uint32_t* b0, uint32_t* b1, int64_t w, int64_t rp, float4 ab, float sc) {
  float hr0, hi0, hr1, hi1, lr, li;
  const uint32_t h0 = round_pair<false>(ab.x * sc, ab.y * sc, hr0, hi0);
  const uint32_t h1 = round_pair<false>(ab.z * sc, ab.w * sc, hr1, hi1);
  const uint32_t l0 = round_pair<false>(ab.x * sc - hr0, ab.y * sc - hi0, lr, li);
  const uint32_t l1 = round_pair<false>(ab.z * sc - hr1, ab.w * sc - hi1, lr, li);
  *reinterpret_cast<uint2*>(b0 + w) = make_uint2(pair_neg_hi(h0), pair_neg_hi(h1));
  *reinterpret_cast<uint2*>(b0 + w + rp) = make_uint2(pair_swap(h0), pair_swap(h1));
  *reinterpret_cast<uint2*>(b1 + w) = make_uint2(pair_neg_hi(l0), pair_neg_hi(l1));
  *reinterpret_cast<uint2*>(b1 + w + rp) = make_uint2(pair_swap(l0), pair_swap(l1));
}

// One warp per (m, f) row of Nw (r_pad values, a multiple of 32, the padding
// zero), two values per lane and step.  PER > 0: the row is held in
// registers (r_pad <= 64 PER), one read; PER = 0: two reads.
template <int PER>
__global__ void __launch_bounds__(256) quantize_kernel(SurveyDev s) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nrows = (int64_t)s.nw * s.F;
  const int npair = s.r_pad / 2;
  uint32_t* b0 = reinterpret_cast<uint32_t*>(s.Bq0);
  uint32_t* b1 = reinterpret_cast<uint32_t*>(s.Bq1);
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const int m = (int)(row / s.F), f = (int)(row - (int64_t)m * s.F);
    const float4* src = reinterpret_cast<const float4*>(s.Nw + (int64_t)m * s.nw_stride + (int64_t)f * s.r_pad);
    const int64_t w0 = ((int64_t)m * 2 * s.F + 2 * f) * s.r_pad;  // 32-bit word of row 2f, position 0
    float mx = 0.f;
    if constexpr (PER > 0) {
      float4 v[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int i = lane + 32 * u;
        v[u] = i < npair ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float sc = f16_scale(mx);
      if (lane == 0) s.nsc[row] = sc;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int i = lane + 32 * u;
        if (i < npair) put_pair(b0, b1, w0 + 2 * i, s.r_pad, v[u], sc);
      }
    } else {
      for (int i = lane; i < npair; i += 32) {
        const float4 v = src[i];
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float sc = f16_scale(mx);
      if (lane == 0) s.nsc[row] = sc;
      for (int i = lane; i < npair; i += 32) put_pair(b0, b1, w0 + 2 * i, s.r_pad, src[i], sc);
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
  const int per = (s.r_pad + 63) / 64;  // float4 pairs per lane
  if (per <= 4) {
    quantize_kernel<4><<<(unsigned)grid, 256, 0, st>>>(s);
  } else if (per <= 10) {
    quantize_kernel<10><<<(unsigned)grid, 256, 0, st>>>(s);
  } else if (per <= 20) {
    quantize_kernel<20><<<(unsigned)grid, 256, 0, st>>>(s);
  } else {
    quantize_kernel<0><<<(unsigned)grid, 256, 0, st>>>(s);
  }
  return cudaGetLastError();
}

}  // namespace mk
