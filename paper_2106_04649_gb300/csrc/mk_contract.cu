// Dispatch of the contraction of Eq. (1): S_m(k, f) = c * sum_r R_m(k, r) Nw_m(r, f).
// Complex FP32 R: one focal point -> the HBM-bound complex GEMV (mk_gemv.cu);
// several -> a SIMT FP32 complex GEMM per frequency (mk_cgemm_simt.cu).
// 16-bit R (BF16, FP16, split BF16): the tcgen05 tensor-core GEMM
// (mk_umma.cu) for any number of focal points; the scaled FP16 split first
// quantises the field spectrum (mk_quant.cu).

#include "mk_internal.h"

namespace mk {

cudaError_t prepare_contract() {
  cudaError_t e = prepare_gemv();
  return e != cudaSuccess ? e : umma_prepare();
}

cudaError_t launch_contract(const SurveyDev& s, const UmmaMaps* mp, cudaStream_t st, int num_sms, int* nlaunch) {
  *nlaunch = 1;
  if (s.rprec == 5) {  // scaled FP16 split: quantise the FP32 field spectrum, then the tensor cores
    *nlaunch = 2;
    const cudaError_t e = launch_quantize_field(s, st, num_sms);
    return e != cudaSuccess ? e : launch_umma(s, mp, st, num_sms);
  }
  if (s.rprec != 0) return launch_umma(s, mp, st, num_sms);
  if (gemv_takes(s)) return launch_gemv(s, st, num_sms);
  return launch_cgemm_simt(s, st);
}

}  // namespace mk
