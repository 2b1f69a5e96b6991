// The contraction of Eq. (1) for one focal point: a complex GEMV per frequency,
// S_m(k) = c * sum_r R_m(k, r) Nw_m(r), bound by HBM bandwidth; for a few
// focal points (complex FP32 R, F <= 8) the same kernel takes 2 or 4 of them
// per pass over R.
//
// Paper, Implementation section: the space integral over the fastest axis of
// R is a segmented dot product (pointwise product followed by a segmented
// reduction, one segment per shot).  Here the product and the reduction are
// one pass: R is read from HBM exactly once per iteration, the field
// spectrum stays on chip, and a warp-shuffle tree reduces each row.
//
// Main kernel (gemv_bulk_kernel): one CTA per SM streams units of up to 64
// rows (m, k) of one frequency of the frequency-major R, taken from a global
// work counter, through a ring of shared-memory stages filled by bulk
// asynchronous copies (cp.async.bulk + mbarrier), so that ~190 KB per SM are
// in flight; one producer lane issues the copies, eight consumer warps each
// reduce one row per stage with 128-bit shared loads, their slice of Nw_m
// held in registers (reloaded only when m changes), and a warp-shuffle tree.
// Every wait is bounded: on time-out the kernel drains its copies, sets an
// error word and finishes.  Rows too long for the ring use the
// register-streaming kernels.

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

// ---------------------------------------------------------------- bulk-copy ring
constexpr int kConsWarps = 8;                       // consumer warps = rows per stage
constexpr int kBulkThreads = (kConsWarps + 1) * 32;  // + one producer warp
constexpr int kMaxStages = 8;
constexpr int kRingBytes = 200 * 1024;
constexpr uint32_t kSpinLimit = 1u << 24;  // bounded mbarrier polls (seconds at worst)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

constexpr int kUnitRows = 64;  // rows per work unit, all of one frequency (8 stages of 8 rows)

// Work is handed out dynamically: after its first unit (unit blockIdx.x) the
// producer lane takes units of up to 64 rows of one frequency from a global
// counter, so SMs that stream faster take more units and all finish together.  A stage records its first row and row
// count; a stage without rows ends the stream.  The last CTA to finish
// resets the counters (queue[0]: next unit, queue[1]: finished CTAs), so
// every launch starts from zero; no thread leaves before the final barrier.
//
// FV > 1 (a few focal points): each row of R meets the spectra of nf <= FV
// focal points (Nw rows f = 0 .. nf-1 of the pass, rq float4 apart) in one
// pass, with the F = 1 arithmetic per focal point; outputs go to column
// f * ns + k of S.
template <int PER, int FV>
__global__ void __launch_bounds__(kBulkThreads, 1)
gemv_bulk_kernel(const float4* __restrict__ R, const float4* __restrict__ Nw, float2* __restrict__ S, int ns,
                 int rq, int64_t nw_stride4, int64_t s_stride, float c, int nw, int stages,
                 unsigned* __restrict__ queue, int* __restrict__ err, int nf) {
  extern __shared__ __align__(128) float4 ring[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ int64_t st_row[kMaxStages];  // first row m * ns + k of a stage; -1 ends the stream
  __shared__ int st_n[kMaxStages];        // rows in a stage
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int upf = (ns + kUnitRows - 1) / kUnitRows;  // units per frequency
  const int nunits = nw * upf;
  const int stage_f4 = kConsWarps * rq;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), kConsWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kConsWarps) {  // producer: one lane takes units and issues the bulk copies
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0;
      // the first unit is this CTA's own (its rows of R can stream before the
      // previous kernel has finished); the counter hands out the rest, after
      // the wait for the previous grid (which may be a GEMV still using it)
      for (int u = blockIdx.x;; u = (int)gridDim.x + (int)atomicAdd(queue, 1u)) {
        if (u >= nunits) break;
        const int m = u / upf;
        const int k0 = (u - m * upf) * kUnitRows;
        const int kn = ns - k0 < kUnitRows ? ns - k0 : kUnitRows;
        for (int g = 0; g < kn; g += kConsWarps, ++it) {
          const int s = (int)(it % stages);
          if (!mbar_wait_bounded(smem_u32(&empty_bar[s]), ((it / stages) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          const int nrows = kn - g < kConsWarps ? kn - g : kConsWarps;
          const int64_t row = (int64_t)m * ns + k0 + g;
          st_row[s] = row;
          st_n[s] = nrows;
          const uint32_t bytes = (uint32_t)nrows * (uint32_t)rq * 16u;
          mbar_expect_tx(smem_u32(&full_bar[s]), bytes);
          bulk_g2s(smem_u32(ring + (size_t)s * stage_f4), R + row * rq, bytes, smem_u32(&full_bar[s]));
        }
        if (!ok) break;
        if (u == (int)blockIdx.x) asm volatile("griddepcontrol.wait;" ::: "memory");
      }
      if (ok) {  // end of the stream: a stage without rows
        const int s = (int)(it % stages);
        if (mbar_wait_bounded(smem_u32(&empty_bar[s]), ((it / stages) & 1u) ^ 1u)) {
          st_row[s] = -1;
          st_n[s] = 0;
          mbar_arrive(smem_u32(&full_bar[s]));
          ++it;
        } else {
          ok = false;
        }
      }
      // no copy may still be in flight when the CTA exits
      for (uint32_t q = (it > (uint32_t)stages ? it - stages : 0); q < it; ++q) {
        if (!mbar_wait_bounded(smem_u32(&full_bar[q % stages]), (q / stages) & 1u)) ok = false;
      }
      if (!ok && err) atomicExch(err, 1);
    }
  } else {
    // consumers: warp w reduces row w of every stage.  When launched as a
    // programmatic dependent of the previous kernel (the epilogue that writes
    // Nw and reads S), wait for that grid here: the producer's copies of R
    // may already be under way.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int cur_w = -1;
    float4 nv1[PER];
    float4 nv[FV > 1 ? FV : 1][FV > 1 ? PER : 1];
    for (uint32_t it = 0;; ++it) {
      const int s = (int)(it % stages);
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(smem_u32(&full_bar[s]), (it / stages) & 1u));
      if (!ok) {
        if (lane == 0 && err) atomicExch(err, 2);
        break;
      }
      const int64_t row0 = st_row[s];
      if (row0 < 0) break;
      if (warp < st_n[s]) {
        const int64_t row = row0 + warp;
        const int w = (int)(row / ns);
        const int k = (int)(row - (int64_t)w * ns);
        if constexpr (FV == 1) {
          if (w != cur_w) {
            const float4* nrow = Nw + (int64_t)w * nw_stride4;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
              const int i = lane + 32 * q;
              nv1[q] = i < rq ? __ldg(nrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cur_w = w;
          }
          const float4* rr = ring + (size_t)s * stage_f4 + (size_t)warp * rq;
          float re = 0.f, im = 0.f;
#pragma unroll
          for (int q = 0; q < PER; ++q) {
            const int i = lane + 32 * q;
            const float4 rv = i < rq ? rr[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            re = fmaf(rv.x, nv1[q].x, re);
            re = fmaf(-rv.y, nv1[q].y, re);
            re = fmaf(rv.z, nv1[q].z, re);
            re = fmaf(-rv.w, nv1[q].w, re);
            im = fmaf(rv.x, nv1[q].y, im);
            im = fmaf(rv.y, nv1[q].x, im);
            im = fmaf(rv.z, nv1[q].w, im);
            im = fmaf(rv.w, nv1[q].z, im);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
          }
          if (lane == 0) S[(int64_t)w * s_stride + k] = make_float2(c * re, c * im);
        } else {
          if (w != cur_w) {
            const float4* nrow = Nw + (int64_t)w * nw_stride4;
#pragma unroll
            for (int f = 0; f < FV; ++f)
#pragma unroll
              for (int q = 0; q < PER; ++q) {
                const int i = lane + 32 * q;
                nv[f][q] = i < rq && f < nf ? __ldg(nrow + (int64_t)f * rq + i) : make_float4(0.f, 0.f, 0.f, 0.f);
              }
            cur_w = w;
          }
          const float4* rr = ring + (size_t)s * stage_f4 + (size_t)warp * rq;
          float re[FV], im[FV];
#pragma unroll
          for (int f = 0; f < FV; ++f) re[f] = im[f] = 0.f;
#pragma unroll
          for (int q = 0; q < PER; ++q) {
            const int i = lane + 32 * q;
            const float4 rv = i < rq ? rr[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int f = 0; f < FV; ++f) {
              re[f] = fmaf(rv.x, nv[f][q].x, re[f]);
              re[f] = fmaf(-rv.y, nv[f][q].y, re[f]);
              re[f] = fmaf(rv.z, nv[f][q].z, re[f]);
              re[f] = fmaf(-rv.w, nv[f][q].w, re[f]);
              im[f] = fmaf(rv.x, nv[f][q].y, im[f]);
              im[f] = fmaf(rv.y, nv[f][q].x, im[f]);
              im[f] = fmaf(rv.z, nv[f][q].w, im[f]);
              im[f] = fmaf(rv.w, nv[f][q].z, im[f]);
            }
          }
#pragma unroll
          for (int f = 0; f < FV; ++f)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              re[f] += __shfl_xor_sync(0xffffffffu, re[f], o);
              im[f] += __shfl_xor_sync(0xffffffffu, im[f], o);
            }
          if (lane == 0) {
#pragma unroll
            for (int f = 0; f < FV; ++f)
              if (f < nf) S[(int64_t)w * s_stride + (int64_t)f * ns + k] = make_float2(c * re[f], c * im[f]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty_bar[s]));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      atomicExch(queue, 0u);
      atomicExch(queue + 1, 0u);
    }
  }
}

int bulk_stages(int rq) {
  const int stage_bytes = kConsWarps * rq * 16;
  int st = kRingBytes / stage_bytes;
  return st > kMaxStages ? kMaxStages : st;
}

template <int PER, int FV>
cudaError_t launch_bulk_per(const SurveyDev& s, cudaStream_t st, int num_sms, int f0, int nf) {
  const int rq = s.r_pad / 2;
  const int stages = bulk_stages(rq);
  const size_t smem = (size_t)stages * kConsWarps * rq * 16;
  const int64_t units = (int64_t)s.nw * ((s.ns + kUnitRows - 1) / kUnitRows);
  const int64_t grid = units < num_sms ? units : num_sms;  // every CTA has a first unit
  // programmatic dependent launch (when the host allows it, s.pdl): the CTAs
  // may start on SMs the previous kernel has left while its last CTAs finish,
  // and stream their first unit of R before that kernel ends.  The host
  // allows it only when the preceding kernel writes no R (normally the
  // epilogue); after an R load the launch is an ordinary stream-ordered one,
  // for which griddepcontrol.wait returns at once.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBulkThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = s.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, gemv_bulk_kernel<PER, FV>, reinterpret_cast<const float4*>(s.R),
                            reinterpret_cast<const float4*>(s.Nw) + (int64_t)f0 * rq, s.S + (int64_t)f0 * s.ns,
                            s.ns, rq, s.nw_stride / 2, s.s_stride, s.c, s.nw, stages, s.counter + 1, s.err, nf);
}

template <int PER, int FV>
cudaError_t set_bulk_attr() {
  return cudaFuncSetAttribute(gemv_bulk_kernel<PER, FV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
}

// Focal points per pass of R: 1 for F = 1; else 4 where the field slices fit
// in registers (PER <= 6), else 2.
int focal_per_pass(int F, int per) { return F == 1 ? 1 : (F > 2 && per <= 6 ? 4 : 2); }

template <int PER>
cudaError_t launch_bulk(const SurveyDev& s, cudaStream_t st, int num_sms) {
  const int fv = focal_per_pass(s.F, PER);
  for (int f0 = 0; f0 < s.F; f0 += fv) {
    const int nf = s.F - f0 < fv ? s.F - f0 : fv;
    cudaError_t e;
    if (fv == 1) {
      e = launch_bulk_per<PER, 1>(s, st, num_sms, f0, nf);
    } else if constexpr (PER <= 6) {
      e = fv == 4 ? launch_bulk_per<PER, 4>(s, st, num_sms, f0, nf) : launch_bulk_per<PER, 2>(s, st, num_sms, f0, nf);
    } else if constexpr (PER <= 12) {
      e = launch_bulk_per<PER, 2>(s, st, num_sms, f0, nf);
    } else {
      e = cudaErrorNotSupported;  // gemv_takes() keeps these surveys off the multi-focal form
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

cudaError_t prepare_gemv() {
  cudaError_t e;
#define MK_BULK_ATTR(P, V) \
  if ((e = set_bulk_attr<P, V>()) != cudaSuccess) return e;
  MK_BULK_ATTR(1, 1) MK_BULK_ATTR(2, 1) MK_BULK_ATTR(4, 1) MK_BULK_ATTR(6, 1) MK_BULK_ATTR(8, 1) MK_BULK_ATTR(10, 1)
  MK_BULK_ATTR(12, 1) MK_BULK_ATTR(16, 1) MK_BULK_ATTR(20, 1)
  MK_BULK_ATTR(1, 2) MK_BULK_ATTR(2, 2) MK_BULK_ATTR(4, 2) MK_BULK_ATTR(6, 2) MK_BULK_ATTR(8, 2) MK_BULK_ATTR(10, 2)
  MK_BULK_ATTR(12, 2) MK_BULK_ATTR(1, 4) MK_BULK_ATTR(2, 4) MK_BULK_ATTR(4, 4) MK_BULK_ATTR(6, 4)
#undef MK_BULK_ATTR
  return cudaSuccess;
}

bool gemv_takes(const SurveyDev& s) {
  if (s.F == 1) return true;
  const int rq = s.r_pad / 2;
  const int per = (rq + 31) / 32;
  return s.F <= kGemvMaxFocal && per <= 12 && bulk_stages(rq) >= 2;
}

cudaError_t launch_gemv(const SurveyDev& s, cudaStream_t st, int num_sms) {
  const int rq = s.r_pad / 2;
  const int per = (rq + 31) / 32;
  if (s.F > 1 && !gemv_takes(s)) return cudaErrorNotSupported;
  if (per <= 20 && bulk_stages(rq) >= 2) {
    switch (per) {
      case 1: return launch_bulk<1>(s, st, num_sms);
      case 2: return launch_bulk<2>(s, st, num_sms);
      case 3: case 4: return launch_bulk<4>(s, st, num_sms);
      case 5: case 6: return launch_bulk<6>(s, st, num_sms);
      case 7: case 8: return launch_bulk<8>(s, st, num_sms);
      case 9: case 10: return launch_bulk<10>(s, st, num_sms);
      case 11: case 12: return launch_bulk<12>(s, st, num_sms);
      case 13: case 14: case 15: case 16: return launch_bulk<16>(s, st, num_sms);
      default: return launch_bulk<20>(s, st, num_sms);
    }
  }
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

}  // namespace mk
