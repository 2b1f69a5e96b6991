// The contraction of Eq. (1) per frequency: S_m(k, f) = c * sum_r R_m(k, r) Nw_m(r, f).
//
// Paper, Implementation section: the space integral over the fastest axis of
// R is a segmented dot product (pointwise product followed by a segmented
// reduction, one segment per shot).  Here the product and the reduction are
// one pass: R is read from HBM exactly once per iteration, the field
// spectrum stays on chip, and a warp-shuffle tree reduces each row.
//
//  * F = 1 (one focal point): a complex GEMV, bound by HBM bandwidth.  Each
//    warp owns a contiguous range of rows (m, k) of the frequency-major R, so
//    its slice of Nw_m (held in registers) changes at most a few times; R is
//    streamed with 128-bit non-coherent loads that do not allocate in L1.
//  * F > 1: a plain per-output kernel (correctness path for small F).

#include "mk_internal.h"

namespace mk {
namespace {

__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Rows of RQ float4 (two complex each); lane l owns float4 l, l + 32, ...
template <int PER>
__global__ void __launch_bounds__(256)
gemv_c64_kernel(const float4* __restrict__ R, const float4* __restrict__ Nw, float2* __restrict__ S,
                int ns, int rq, int64_t nw_stride4, int64_t s_stride, float c, int64_t total_rows) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t row0 = warp * total_rows / nwarps;
  const int64_t row1 = (warp + 1) * total_rows / nwarps;
  int cur_w = -1;
  float4 nv[PER];
  for (int64_t row = row0; row < row1; ++row) {
    const int w = (int)(row / ns);
    const int k = (int)(row - (int64_t)w * ns);
    if (w != cur_w) {
      const float4* nrow = Nw + (int64_t)w * nw_stride4;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int i = lane + 32 * q;
        nv[q] = i < rq ? __ldg(nrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      cur_w = w;
    }
    const float4* rrow = R + row * rq;
    float4 rv[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = lane + 32 * q;
      rv[q] = i < rq ? ld_stream(rrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      re = fmaf(rv[q].x, nv[q].x, re);
      re = fmaf(-rv[q].y, nv[q].y, re);
      re = fmaf(rv[q].z, nv[q].z, re);
      re = fmaf(-rv[q].w, nv[q].w, re);
      im = fmaf(rv[q].x, nv[q].y, im);
      im = fmaf(rv[q].y, nv[q].x, im);
      im = fmaf(rv[q].z, nv[q].w, im);
      im = fmaf(rv[q].w, nv[q].z, im);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) S[(int64_t)w * s_stride + k] = make_float2(c * re, c * im);
  }
}

// Rows longer than the register-resident form: Nw is re-read through L1.
__global__ void __launch_bounds__(256)
gemv_c64_long_kernel(const float4* __restrict__ R, const float4* __restrict__ Nw, float2* __restrict__ S,
                     int ns, int rq, int64_t nw_stride4, int64_t s_stride, float c, int64_t total_rows) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t row0 = warp * total_rows / nwarps;
  const int64_t row1 = (warp + 1) * total_rows / nwarps;
  for (int64_t row = row0; row < row1; ++row) {
    const int w = (int)(row / ns);
    const int k = (int)(row - (int64_t)w * ns);
    const float4* nrow = Nw + (int64_t)w * nw_stride4;
    const float4* rrow = R + row * rq;
    float re = 0.f, im = 0.f;
    for (int base = 0; base < rq; base += 32 * 8) {
      float4 rv[8], nv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = base + lane + 32 * q;
        rv[q] = i < rq ? ld_stream(rrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        nv[q] = i < rq ? __ldg(nrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        re = fmaf(rv[q].x, nv[q].x, re);
        re = fmaf(-rv[q].y, nv[q].y, re);
        re = fmaf(rv[q].z, nv[q].z, re);
        re = fmaf(-rv[q].w, nv[q].w, re);
        im = fmaf(rv[q].x, nv[q].y, im);
        im = fmaf(rv[q].y, nv[q].x, im);
        im = fmaf(rv[q].z, nv[q].w, im);
        im = fmaf(rv[q].w, nv[q].z, im);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) S[(int64_t)w * s_stride + k] = make_float2(c * re, c * im);
  }
}

// F > 1, one thread per output (m, k, f).
__global__ void contract_naive_kernel(const float2* __restrict__ R, const float2* __restrict__ Nw,
                                      float2* __restrict__ S, int nw, int ns, int F, int r_pad,
                                      int64_t nw_stride, int64_t s_stride, float c) {
  const int64_t total = (int64_t)nw * ns * F;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i % F);
    const int64_t mk = i / F;
    const int k = (int)(mk % ns);
    const int m = (int)(mk / ns);
    const float2* rrow = R + ((int64_t)m * ns + k) * r_pad;
    const float2* ncol = Nw + (int64_t)m * nw_stride + f;
    float re = 0.f, im = 0.f;
    for (int r = 0; r < ns; ++r) {
      const float2 a = rrow[r], b = ncol[(int64_t)r * F];
      re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
      im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
    }
    S[(int64_t)m * s_stride + (int64_t)k * F + f] = make_float2(c * re, c * im);
  }
}

template <int PER>
cudaError_t launch_gemv_per(const SurveyDev& s, cudaStream_t st, int num_sms) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gemv_c64_kernel<PER>, 256, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const int64_t total = (int64_t)s.nw * s.ns;
  int64_t grid = (int64_t)num_sms * occ;
  if (grid * 8 > total) grid = (total + 7) / 8;
  gemv_c64_kernel<PER><<<(unsigned)grid, 256, 0, st>>>(
      reinterpret_cast<const float4*>(s.R), reinterpret_cast<const float4*>(s.Nw), s.S, s.ns,
      s.r_pad / 2, s.nw_stride / 2, s.s_stride, s.c, total);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_contract(const SurveyDev& s, cudaStream_t st, int num_sms, int* nlaunch) {
  *nlaunch = 1;
  if (s.F == 1) {
    const int rq = s.r_pad / 2;
    const int per = (rq + 31) / 32;
    switch (per) {
      case 1: return launch_gemv_per<1>(s, st, num_sms);
      case 2: return launch_gemv_per<2>(s, st, num_sms);
      case 3: case 4: return launch_gemv_per<4>(s, st, num_sms);
      case 5: case 6: return launch_gemv_per<6>(s, st, num_sms);
      case 7: case 8: return launch_gemv_per<8>(s, st, num_sms);
      case 9: case 10: return launch_gemv_per<10>(s, st, num_sms);
      case 11: case 12: return launch_gemv_per<12>(s, st, num_sms);
      default: {
        const int64_t total = (int64_t)s.nw * s.ns;
        int64_t grid = (int64_t)num_sms * 8;
        if (grid * 8 > total) grid = (total + 7) / 8;
        gemv_c64_long_kernel<<<(unsigned)grid, 256, 0, st>>>(
            reinterpret_cast<const float4*>(s.R), reinterpret_cast<const float4*>(s.Nw), s.S, s.ns, rq,
            s.nw_stride / 2, s.s_stride, s.c, total);
        return cudaGetLastError();
      }
    }
  }
  const int64_t total = (int64_t)s.nw * s.ns * s.F;
  int64_t grid = (total + 255) / 256;
  if (grid > (int64_t)num_sms * 16) grid = (int64_t)num_sms * 16;
  contract_naive_kernel<<<(unsigned)grid, 256, 0, st>>>(s.R, s.Nw, s.S, s.nw, s.ns, s.F, s.r_pad,
                                                       s.nw_stride, s.s_stride, s.c);
  return cudaGetLastError();
}

}  // namespace mk
