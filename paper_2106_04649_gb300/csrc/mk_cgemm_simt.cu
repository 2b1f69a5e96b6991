// The contraction of Eq. (1) for many focal points with complex FP32 R: a
// register-tiled SIMT complex GEMM per frequency,
// S_m[k][f] = c * sum_r R_m[k][r] Nw_m[r][f], with exact FP32 products
// (the plain-precision form; the tensor-core forms are in mk_umma.cu).
// 64 x 64 output tile per CTA, 16-deep K slices double-buffered through
// shared memory with register prefetch, 4 x 4 complex accumulators per
// thread.  (Paper, Implementation section: many focal points share each
// batch of R, which is what makes the synthesis compute-dense.)

#include "mk_internal.h"

namespace mk {
namespace {

constexpr int GM = 64, GN = 64, GK = 16;

// C_m[k][f] = c * sum_r A_m[k][r] B_m[r][f]; A = R_m (rows of r_pad, zero
// padded, so K needs no predicate), B = Nw_m ([r][f], row stride F),
// C = S_m ([k][f], row stride F).  blockIdx = (k tile, f tile, m).
__global__ void __launch_bounds__(256)
cgemm_f32_kernel(const float2* __restrict__ R, const float2* __restrict__ Nw, float2* __restrict__ S, int ns, int F,
                 int r_pad, int64_t nw_stride, int64_t s_stride, float c) {
  __shared__ __align__(16) float2 As[2][GK][GM];  // transposed A tile: As[r][k]
  __shared__ __align__(16) float2 Bs[2][GK][GN];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int m = blockIdx.z;
  const int k0 = blockIdx.x * GM, f0 = blockIdx.y * GN;
  const float2* A = R + (int64_t)m * ns * r_pad;
  const float2* B = Nw + (int64_t)m * nw_stride;
  // global -> register staging: A: row ak = t/4, complex cols (t%4)*2 + {0,1} and +8
  const int ak = t >> 2, ac = (t & 3) * 2;
  const bool arow_ok = k0 + ak < ns;
  const float2* Ap = A + (int64_t)(k0 + ak) * r_pad + ac;
  // B: rows br = t/32 and br + 8, complex cols (t%32)*2 + {0,1}
  const int br = t >> 5, bc = (t & 31) * 2;
  const bool bc0 = f0 + bc < F, bc1 = f0 + bc + 1 < F;
  float4 ra0, ra1;
  float2 rb[2][2];
  auto load_tile = [&](int kb) {
    if (arow_ok) {
      ra0 = __ldg(reinterpret_cast<const float4*>(Ap + kb));
      ra1 = __ldg(reinterpret_cast<const float4*>(Ap + kb + 8));
    } else {
      ra0 = ra1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2* bp = B + (int64_t)(kb + br + 8 * h) * F + f0 + bc;
      rb[h][0] = bc0 ? __ldg(bp) : make_float2(0.f, 0.f);
      rb[h][1] = bc1 ? __ldg(bp + 1) : make_float2(0.f, 0.f);
    }
  };
  auto store_tile = [&](int buf) {
    As[buf][ac][ak] = make_float2(ra0.x, ra0.y);
    As[buf][ac + 1][ak] = make_float2(ra0.z, ra0.w);
    As[buf][ac + 8][ak] = make_float2(ra1.x, ra1.y);
    As[buf][ac + 9][ak] = make_float2(ra1.z, ra1.w);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Bs[buf][br + 8 * h][bc] = rb[h][0];
      Bs[buf][br + 8 * h][bc + 1] = rb[h][1];
    }
  };
  float accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = 0.f;

  const int nk = r_pad / GK;
  load_tile(0);
  store_tile(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) load_tile((kt + 1) * GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a01 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a23 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4 + 2]);
      const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                           make_float2(a23.z, a23.w)};
      float2 b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fmaf(a[i].x, b[j].x, accr[i][j]);
          accr[i][j] = fmaf(-a[i].y, b[j].y, accr[i][j]);
          acci[i][j] = fmaf(a[i].x, b[j].y, acci[i][j]);
          acci[i][j] = fmaf(a[i].y, b[j].x, acci[i][j]);
        }
    }
    if (kt + 1 < nk) store_tile(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + ty * 4 + i;
    if (k >= ns) continue;
    float2* crow = S + (int64_t)m * s_stride + (int64_t)k * F;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + tx + 16 * j;
      if (f < F) crow[f] = make_float2(c * accr[i][j], c * acci[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_cgemm_simt(const SurveyDev& s, cudaStream_t st) {
  const dim3 grid((s.ns + GM - 1) / GM, (s.F + GN - 1) / GN, s.nw);
  cgemm_f32_kernel<<<grid, 256, 0, st>>>(s.R, s.Nw, s.S, s.ns, s.F, s.r_pad, s.nw_stride, s.s_stride, s.c);
  return cudaGetLastError();
}

}  // namespace mk
