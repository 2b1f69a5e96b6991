// The contraction of Eq. (1) for many focal points with complex FP32 R: a
// register-tiled SIMT complex GEMM per frequency,
// S_m[k][f] = c * sum_r R_m[k][r] Nw_m[f][r], with exact FP32 products
// (the plain-precision form; the tensor-core forms are in mk_umma.cu).
// 64 x 64 output tile per CTA, 16-deep K slices double-buffered through
// shared memory with register prefetch, 4 x 4 complex accumulators per
// thread.  (Paper, Implementation section: many focal points share each
// batch of R, which is what makes the synthesis compute-dense.)

#include "mk_internal.h"

namespace mk {
namespace {

constexpr int GM = 64, GN = 64, GK = 16;

// C_m[k][f] = c * sum_r A_m[k][r] B_m[f][r]; A = R_m (rows of r_pad, zero
// padded, so K needs no predicate), B = Nw_m ([f][r_pad], K-contiguous),
// C = S_m[f * ns + k].  blockIdx = (k tile, f tile, m).  Thread (tx, ty)
// owns rows k = k0 + tx + 16 i and columns f = f0 + 4 ty + j, so that a
// half-warp stores 16 consecutive k of one f (coalesced).
__global__ void __launch_bounds__(256)
cgemm_f32_kernel(const float2* __restrict__ R, const float2* __restrict__ Nw, float2* __restrict__ S, int ns, int F,
                 int r_pad, int64_t nw_stride, int64_t s_stride, float c) {
  __shared__ __align__(16) float2 As[2][GK][GM];  // As[r][k]
  __shared__ __align__(16) float2 Bs[2][GK][GN];  // Bs[r][f]
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int m = blockIdx.z;
  const int k0 = blockIdx.x * GM, f0 = blockIdx.y * GN;
  const float2* A = R + (int64_t)m * ns * r_pad;
  const float2* B = Nw + (int64_t)m * nw_stride;
  // global -> register staging: row (t / 4) of the tile, complex cols (t % 4) * 2 + {0, 1} and + 8
  const int lr = t >> 2, lc = (t & 3) * 2;
  const bool arow_ok = k0 + lr < ns;
  const bool brow_ok = f0 + lr < F;
  const float2* Ap = A + (int64_t)(k0 + lr) * r_pad + lc;
  const float2* Bp = B + (int64_t)(f0 + lr) * r_pad + lc;
  float4 ra0, ra1, rb0, rb1;
  auto load_tile = [&](int kb) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    ra0 = arow_ok ? __ldg(reinterpret_cast<const float4*>(Ap + kb)) : z;
    ra1 = arow_ok ? __ldg(reinterpret_cast<const float4*>(Ap + kb + 8)) : z;
    rb0 = brow_ok ? __ldg(reinterpret_cast<const float4*>(Bp + kb)) : z;
    rb1 = brow_ok ? __ldg(reinterpret_cast<const float4*>(Bp + kb + 8)) : z;
  };
  auto store_tile = [&](int buf) {
    As[buf][lc][lr] = make_float2(ra0.x, ra0.y);
    As[buf][lc + 1][lr] = make_float2(ra0.z, ra0.w);
    As[buf][lc + 8][lr] = make_float2(ra1.x, ra1.y);
    As[buf][lc + 9][lr] = make_float2(ra1.z, ra1.w);
    Bs[buf][lc][lr] = make_float2(rb0.x, rb0.y);
    Bs[buf][lc + 1][lr] = make_float2(rb0.z, rb0.w);
    Bs[buf][lc + 8][lr] = make_float2(rb1.x, rb1.y);
    Bs[buf][lc + 9][lr] = make_float2(rb1.z, rb1.w);
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
      float2 a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tx + 16 * i];
      const float4 b01 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b23 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4 + 2]);
      const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                           make_float2(b23.z, b23.w)};
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
  float2* Sm = S + (int64_t)m * s_stride;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int f = f0 + ty * 4 + j;
    if (f >= F) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + tx + 16 * i;
      if (k < ns) Sm[(int64_t)f * ns + k] = make_float2(c * accr[i][j], c * acci[i][j]);
    }
  }
}

// The wide form for n_s >= 128: a 128 x 64 output tile per CTA, 8 x 4
// complex accumulators per thread (rows k0 + tx + 16 i, i < 8), 128 FMAs per
// 6 shared-memory loads per K step; two CTAs per SM (48 KB shared each).
constexpr int WM = 128;

__global__ void __launch_bounds__(256, 2)
cgemm_f32_wide_kernel(const float2* __restrict__ R, const float2* __restrict__ Nw, float2* __restrict__ S, int ns,
                      int F, int r_pad, int64_t nw_stride, int64_t s_stride, float c) {
  __shared__ __align__(16) float2 As[2][GK][WM];  // As[r][k]
  __shared__ __align__(16) float2 Bs[2][GK][GN];  // Bs[r][f]
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int m = blockIdx.z;
  const int k0 = blockIdx.x * WM, f0 = blockIdx.y * GN;
  const float2* A = R + (int64_t)m * ns * r_pad;
  const float2* B = Nw + (int64_t)m * nw_stride;
  // staging: rows lr and lr + 64 of the A tile, row lr of the B tile;
  // complex columns lc, lc + 1 and lc + 8, lc + 9 of the K slice
  const int lr = t >> 2, lc = (t & 3) * 2;
  const bool a0_ok = k0 + lr < ns, a1_ok = k0 + lr + 64 < ns;
  const bool b_ok = f0 + lr < F;
  const float2* Ap0 = A + (int64_t)(k0 + lr) * r_pad + lc;
  const float2* Ap1 = Ap0 + (int64_t)64 * r_pad;
  const float2* Bp = B + (int64_t)(f0 + lr) * r_pad + lc;
  float4 ra[4], rb[2];
  auto load_tile = [&](int kb) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    ra[0] = a0_ok ? __ldg(reinterpret_cast<const float4*>(Ap0 + kb)) : z;
    ra[1] = a0_ok ? __ldg(reinterpret_cast<const float4*>(Ap0 + kb + 8)) : z;
    ra[2] = a1_ok ? __ldg(reinterpret_cast<const float4*>(Ap1 + kb)) : z;
    ra[3] = a1_ok ? __ldg(reinterpret_cast<const float4*>(Ap1 + kb + 8)) : z;
    rb[0] = b_ok ? __ldg(reinterpret_cast<const float4*>(Bp + kb)) : z;
    rb[1] = b_ok ? __ldg(reinterpret_cast<const float4*>(Bp + kb + 8)) : z;
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = lr + 64 * h;
      As[buf][lc][row] = make_float2(ra[2 * h].x, ra[2 * h].y);
      As[buf][lc + 1][row] = make_float2(ra[2 * h].z, ra[2 * h].w);
      As[buf][lc + 8][row] = make_float2(ra[2 * h + 1].x, ra[2 * h + 1].y);
      As[buf][lc + 9][row] = make_float2(ra[2 * h + 1].z, ra[2 * h + 1].w);
    }
    Bs[buf][lc][lr] = make_float2(rb[0].x, rb[0].y);
    Bs[buf][lc + 1][lr] = make_float2(rb[0].z, rb[0].w);
    Bs[buf][lc + 8][lr] = make_float2(rb[1].x, rb[1].y);
    Bs[buf][lc + 9][lr] = make_float2(rb[1].z, rb[1].w);
  };
  float accr[8][4], acci[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
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
      float2 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[buf][kk][tx + 16 * i];
      const float4 b01 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b23 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4 + 2]);
      const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                           make_float2(b23.z, b23.w)};
#pragma unroll
      for (int i = 0; i < 8; ++i)
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
  float2* Sm = S + (int64_t)m * s_stride;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int f = f0 + ty * 4 + j;
    if (f >= F) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + tx + 16 * i;
      if (k < ns) Sm[(int64_t)f * ns + k] = make_float2(c * accr[i][j], c * acci[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_cgemm_simt(const SurveyDev& s, cudaStream_t st) {
  if (s.ns >= WM) {
    const dim3 grid((s.ns + WM - 1) / WM, (s.F + GN - 1) / GN, s.nw);
    cgemm_f32_wide_kernel<<<grid, 256, 0, st>>>(s.R, s.Nw, s.S, s.ns, s.F, s.r_pad, s.nw_stride, s.s_stride, s.c);
    return cudaGetLastError();
  }
  const dim3 grid((s.ns + GM - 1) / GM, (s.F + GN - 1) / GN, s.nw);
  cgemm_f32_kernel<<<grid, 256, 0, st>>>(s.R, s.Nw, s.S, s.ns, s.F, s.r_pad, s.nw_stride, s.s_stride, s.c);
  return cudaGetLastError();
}

}  // namespace mk
