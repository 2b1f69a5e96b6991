// Conversion of one complex FP32 value of R into the 16-bit storage of the
// tensor-core contraction: BF16 or FP16 rounded to nearest even (q = 1, 2),
// BF16 hi + lo with lo = rn(x - hi) (q = 3), or BF16 hi + mid + lo with
// mid = rn(x - hi), lo = rn(x - hi - mid) (q = 4), or FP16 hi + lo of the
// value scaled by its frequency's power of two s.rsc[m] (q = 5).  idx counts complex
// elements of the [nw][ns][r_pad] layout; each part holds one 16-bit pair
// per element.  Shared by the R loads from band spectra and from time traces.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mk_internal.h"

namespace mk {

__device__ __forceinline__ void store_r16(const SurveyDev& s, int q, int64_t idx, float2 v) {
  if (q == 5) {  // FP16 hi + lo of the value scaled by the power of two of its frequency
    const float sc = s.rsc[idx / ((int64_t)s.ns * s.r_pad)];
    const float x = v.x * sc, y = v.y * sc;  // exact: a power of two
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    reinterpret_cast<__half2*>(const_cast<void*>(s.Rq0))[idx] = h;
    reinterpret_cast<__half2*>(const_cast<void*>(s.Rq1))[idx] = __floats2half2_rn(x - hf.x, y - hf.y);
    return;
  }
  if (q == 2) {
    reinterpret_cast<__half2*>(const_cast<void*>(s.Rq0))[idx] = __floats2half2_rn(v.x, v.y);
    return;
  }
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  reinterpret_cast<__nv_bfloat162*>(const_cast<void*>(s.Rq0))[idx] = h;
  if (q >= 3) {
    const float2 hf = __bfloat1622float2(h);
    const float rx = v.x - hf.x, ry = v.y - hf.y;  // exact in FP32
    const __nv_bfloat162 m2 = __floats2bfloat162_rn(rx, ry);
    reinterpret_cast<__nv_bfloat162*>(const_cast<void*>(s.Rq1))[idx] = m2;
    if (q == 4) {
      const float2 mf = __bfloat1622float2(m2);
      reinterpret_cast<__nv_bfloat162*>(const_cast<void*>(s.Rq2))[idx] = __floats2bfloat162_rn(rx - mf.x, ry - mf.y);
    }
  }
}

}  // namespace mk
