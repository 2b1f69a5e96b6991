// Internal declarations shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mk {

// Device-side view of one survey: sizes, strides and workspace carvings.
// Traces are ordered focal-major: t = f * ns + k, so that neighbouring
// traces (same focal point, neighbouring positions) touch neighbouring
// addresses in every spectrum buffer.  Field offset of trace t is t * nt.
// S is frequency-major with element (m, t) at m * s_stride + t.  Nw holds
// [nw][F][r_pad]: element (m, f, r) at m * nw_stride + f * r_pad + r, the
// padding r >= ns zero.
struct SurveyDev {
  int ns;          // output positions held (all nsrc, or the rows of a shot-row shard)
  int nr;          // summed positions (nrec): the r axis of R rows and of the field spectrum
  int row0;        // position of output row 0 on the r axis (first row of a shard, else 0)
  int nt;          // samples
  int F;           // focal points
  int nw;          // kept frequency bins
  int r_pad;       // padded row length of R (multiple of 32)
  int ncols;       // ns * F
  int64_t s_stride;   // complex elements per S row (>= ncols + 1, multiple of 4)
  int64_t nw_stride;  // complex elements per Nw frequency (F * r_pad)
  double dt;       // sample interval (s)
  float c;         // synthesis scale dx * dt
  float inv_nt;    // 1 / nt
  int rprec;       // mk_rprec

  const float2* R;  // [nw][ns][r_pad] complex FP32 (MK_R_C64)
  const void* Rq0;  // 16-bit R [nw][ns][2 r_pad] (hi part of split forms)
  const void* Rq1;  // lo (2-way split) or mid (3-way split) part
  const void* Rq2;  // lo part of the 3-way split
  void* Bq0;        // 16-bit field embedding [nw][2F][2 r_pad], hi part
  void* Bq1;        // lo (mid for the 3-way split) part
  void* Bq2;        // lo part of the 3-way split
  float2* Nw;       // [nw][F][r_pad] (complex FP32 R, and the FP32 field of the scaled FP16 split)
  float* rsc;       // [nw] power-of-two scale of R_m (scaled FP16 split), else null
  float* nsc;       // [nw][F] power-of-two scale of the field spectrum (scaled FP16 split), else null
  float2* S;        // [nw][s_stride]
  float* fN;        // [F][ns][nt] last N_i
  float* f1p;
  float* f1m;
  float* f2p;
  float* pmin;
  float* scratch;   // [F][ns][nt] staging (G_d upload, G for host output)
  float* gm;        // [F][ns][nt] G^- (formed on request)
  float* gp;        // [F][ns][nt] G^+ (formed on request)
  int* L;           // [ncols] window half-lengths
  double* td;       // [F][ns] staging of t_d uploaded from the host
  double* Epart;    // [ncols + 1] per-trace energies
  unsigned* counter;  // [8]: epilogue last-CTA count; GEMV work counter and finished CTAs (1, 2);
                      // tensor-core contraction work counter and finished CTAs (4, 5)
  const float2* tw;   // [nt] FFT twiddles in the pass-by-pass layout of the shared-memory FFT
  const float2* twl;  // [nt] e^{-2 pi i j / nt}, j = 0 .. nt-1 (per-lane twiddles of the register FFT)
  int* err;           // device error word (bounded waits that ran out); may be null
  int* iter;          // device iteration index (parity and energy slot; advanced by the epilogue)
  int epi_g;          // epilogue pairs per block: 0 = chosen from shared memory and grid size, else 1, 2 or 4
  // Host-side launch choices (not read by kernels except where noted):
  int pdl;            // 1: the F = 1 contraction may start as a programmatic dependent of the
                      // preceding kernel, streaming R before that kernel ends; the host sets it
                      // only when no kernel that writes R can precede it on the stream
  float2* pacc;       // null, or [nw][s_stride] running sum of the contraction outputs S of the
                      // Neumann iterations (the band spectrum of pmin, Algorithm 1), added to by
                      // the epilogue when it reads S
};

#ifdef __CUDACC__
// bytes [a, a + n) into L2 (a 16-byte aligned, n a multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void* a, unsigned n) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"(n) : "memory");
}
#endif

// Storage precisions whose epilogue writes the complex FP32 field spectrum Nw
// (complex FP32 R, and the scaled FP16 split, which quantises Nw at each
// contraction); the other 16-bit forms write their embedding directly.
__host__ __device__ inline bool field_in_nw(const SurveyDev& s) { return s.rprec == 0 || s.rprec == 5; }

// Power-of-two scale that maps a largest magnitude amax into [2^14, 2^15):
// with it the FP16 hi part of every value and the lo part of values down to
// 2^-17 of amax stay normal.  1 for amax = 0 (or not finite).
__host__ __device__ inline float f16_scale(float amax) {
  if (!(amax > 0.f) || !(amax < 3.0e38f)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, 15 - e < 126 ? 15 - e : 126);  // finite for the smallest magnitudes
}

// Kernel launchers (return the launch status; the caller checks it).
struct UmmaMaps;  // tensor maps of the tcgen05 contraction (mk_umma.cu)
UmmaMaps* umma_create(const SurveyDev& s);
cudaError_t umma_prepare();
void umma_destroy(UmmaMaps* mp);
cudaError_t launch_umma(const SurveyDev& s, const UmmaMaps* mp, cudaStream_t st, int num_sms);
cudaError_t launch_contract(const SurveyDev& s, const UmmaMaps* mp, cudaStream_t st, int num_sms, int* nlaunch);
// R row loads (grid-stride, at most max_blocks blocks of 256 threads)
cudaError_t prepare_load();
cudaError_t launch_load_rows_q(const float2* src, const SurveyDev& s, int64_t row0, int64_t rows, cudaStream_t st,
                               int max_blocks);
// scaled FP16 split: the largest |Re|, |Im| per frequency of rows row0 .. row0 + rows
// (whole frequencies) into s.rsc as the bits of a float (atomic max; cleared first)
cudaError_t launch_r_amax(const float2* src, const SurveyDev& s, int64_t row0, int64_t rows, cudaStream_t st,
                          int max_blocks);
cudaError_t launch_r_scale(const SurveyDev& s, int w_begin, int w_count, cudaStream_t st);  // amax -> scale
// scaled FP16 split: per (frequency, focal point) the scale of Nw and its 2-part embedding
cudaError_t launch_quantize_field(const SurveyDev& s, cudaStream_t st, int num_sms);
// Energies of iteration i go to ring[(i % slots) * F + f].
cudaError_t launch_epilogue(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms);
cudaError_t launch_set_iter(const SurveyDev& s, int value, cudaStream_t st);
cudaError_t launch_twiddles(float2* tw, int nt, cudaStream_t st);  // FFT twiddle table of nt entries
cudaError_t launch_twiddles_linear(float2* tw, int nt, cudaStream_t st);  // e^{-2 pi i j / nt}, j < nt
bool epilogue_fits(int nt, int nw);  // shared memory of the epilogue within the per-CTA limit
// The epilogue with the transforms in registers, one lane group per trace (mk_epi.cu):
// nt = 64 .. 2048 with a band whose shared stage fits; launch_epilogue uses it
// whenever it supports the shape and falls back to the shared-memory kernel otherwise.
bool epilogue_warp_supports(int nt, int nw);
cudaError_t prepare_epilogue_warp();
cudaError_t launch_epilogue_warp(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms);
// whether launch_epilogue runs the register epilogue for this survey (enough traces
// to fill the GPU with blocks, a supported shape); otherwise the shared-memory one
bool epilogue_uses_warp(const SurveyDev& s, int num_sms);
int epilogue_max_pairs(const SurveyDev& s, int num_sms);  // largest block-size choice of the survey's epilogue
bool umma_set_bn(UmmaMaps* mp, const SurveyDev& s, int bn);  // N tile of the tensor-core contraction
int umma_get_bn(const UmmaMaps* mp);
cudaError_t launch_init(const SurveyDev& s, const float* Gd, cudaStream_t st, int num_sms);
cudaError_t launch_spectrum(const SurveyDev& s, const float* src, cudaStream_t st, int num_sms);  // band spectrum of a field
cudaError_t launch_inverse(const SurveyDev& s, float* dst, int mode, cudaStream_t st, int num_sms);
cudaError_t launch_f2p(const SurveyDev& s, float* diff, cudaStream_t st, int num_sms);
cudaError_t launch_load_rows(const float2* src, float2* dst, int64_t rows, int nrec, int r_pad, cudaStream_t st,
                             int max_blocks);
cudaError_t launch_windows(const SurveyDev& s, const double* td, double eps, cudaStream_t st);
cudaError_t launch_green(const SurveyDev& s, float* out, cudaStream_t st, int num_sms);
cudaError_t launch_lincomb(const SurveyDev& s, float* out, const float* A, int revA, float alpha, const float* B,
                           int revB, float beta, cudaStream_t st, int num_sms);
cudaError_t launch_image(const SurveyDev& s, const float* gm, double scale, double* out, cudaStream_t st);
cudaError_t prepare_kernels();  // one-time function attributes (large dynamic smem)
cudaError_t prepare_contract();  // called by prepare_kernels
cudaError_t prepare_gemv();
cudaError_t launch_gemv(const SurveyDev& s, cudaStream_t st, int num_sms);
// Complex FP32 R with a few focal points (F <= kGemvMaxFocal): the GEMV takes
// 2 or 4 of them per pass over R (memory-bound) where a GEMM tile of 64
// columns would compute mostly padding.
constexpr int kGemvMaxFocal = 8;
bool gemv_takes(const SurveyDev& s);
cudaError_t launch_cgemm_simt(const SurveyDev& s, cudaStream_t st);
void set_noplan_error(const char* msg);  // message returned by mk_last_error(NULL)

}  // namespace mk
