// The field spectrum as the B operand of the tensor-core contraction: the
// K-major real 2x2 embedding of each complex value N = (nr, ni), split into
// 16-bit parts (hi + lo, or hi + mid + lo for the 3-way split form):
//     row 2f: (Nr, -Ni), row 2f+1: (Ni, Nr) at columns 2k, 2k+1
// of the [nw][2F][2 r_pad] embedding.  Shared by the epilogues and the band
// kernels that write field spectra.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mk_internal.h"

namespace mk {

// (a, b) rounded to 16 bits (nearest even) as one packed pair; their values
// back in FP32 in ra, rb.
template <bool BF16>
__device__ __forceinline__ uint32_t round_pair(float a, float b, float& ra, float& rb) {
  if (BF16) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(v);
    ra = f.x;
    rb = f.y;
    return *reinterpret_cast<const uint32_t*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(a, b);
    const float2 f = __half22float2(v);
    ra = f.x;
    rb = f.y;
    return *reinterpret_cast<const uint32_t*>(&v);
  }
}
// From the packed pair (x, y): (x, -y) flips the sign bit of the upper half,
// (y, x) swaps the halves.
__device__ __forceinline__ uint32_t pair_neg_hi(uint32_t w) { return w ^ 0x80000000u; }
__device__ __forceinline__ uint32_t pair_swap(uint32_t w) { return __byte_perm(w, 0, 0x1032); }

// Band value N = (nr, ni) of trace t at bin m into the K-major real
// embedding of the tensor-core contraction, split into hi + lo 16-bit parts:
// rows 2f: (Nr, -Ni), 2f+1: (Ni, Nr) at columns 2k, 2k+1.
template <bool BF16>
__device__ __forceinline__ void store_embedding_at(const SurveyDev& s, int64_t e0, float nr, float ni);

template <bool BF16>
__device__ __forceinline__ void store_embedding(const SurveyDev& s, int m, int f, int k, float nr, float ni) {
  const int64_t kp = 2 * (int64_t)s.r_pad;
  store_embedding_at<BF16>(s, ((int64_t)m * 2 * s.F + 2 * f) * kp + 2 * k, nr, ni);
}

// The same, at element offset e0 = ((m 2F + 2f) 2 r_pad + 2k) of the embedding.
template <bool BF16>
__device__ __forceinline__ void store_embedding_at(const SurveyDev& s, int64_t e0, float nr, float ni) {
  const int64_t kp = 2 * (int64_t)s.r_pad;
  uint32_t* b0 = reinterpret_cast<uint32_t*>(s.Bq0);
  uint32_t* b1 = reinterpret_cast<uint32_t*>(s.Bq1);
  float hr, hi;
  const uint32_t h = round_pair<BF16>(nr, ni, hr, hi);
  float lr = nr - hr, li = ni - hi;  // exact in FP32
  b0[e0 >> 1] = pair_neg_hi(h);
  b0[(e0 + kp) >> 1] = pair_swap(h);
  if (s.rprec == 4) {  // 3-way split: hi, mid = rn(x - hi), lo = rn(x - hi - mid)
    float mr, mi;
    const uint32_t md = round_pair<BF16>(lr, li, mr, mi);
    b1[e0 >> 1] = pair_neg_hi(md);
    b1[(e0 + kp) >> 1] = pair_swap(md);
    lr -= mr;
    li -= mi;
    uint32_t* b2 = reinterpret_cast<uint32_t*>(s.Bq2);
    float dr, di;
    const uint32_t lo = round_pair<BF16>(lr, li, dr, di);
    b2[e0 >> 1] = pair_neg_hi(lo);
    b2[(e0 + kp) >> 1] = pair_swap(lo);
  } else {
    float dr, di;
    const uint32_t lo = round_pair<BF16>(lr, li, dr, di);
    b1[e0 >> 1] = pair_neg_hi(lo);
    b1[(e0 + kp) >> 1] = pair_swap(lo);
  }
}

}  // namespace mk
