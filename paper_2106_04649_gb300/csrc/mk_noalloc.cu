// mk_run_noalloc: the whole Neumann series of one survey without any device
// allocation, for callers that cannot allocate GPU memory themselves.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed at the point of the call -- for example a host framework that owns
// all device memory through its own pool and hands out only fixed input and
// output buffers, or a process whose memory budget is fixed up front.  Such
// a caller cannot provide the plan workspace of mk_plan.  This entry point
// runs the same kernels as mk_set_Gd_window + mk_iterate, on caller-owned
// inputs and outputs, and keeps its intermediate data (mute windows, band
// spectra of N_i and of the synthesis result, per-trace energies, the
// completion counter and the FFT twiddles) in one file-scope device array of
// fixed size, MK_NOALLOC_SCRATCH_BYTES, which every GPU that loads the
// library holds until the process exits.

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/marchenko.h"
#include "mk_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// The scratch array.  Host code must not use the symbol's host-side address:
// the device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MK_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Failures are reported through mk_last_error(NULL).
mk_status set_err(mk_status st, const char* msg, const char* detail = nullptr) {
  char buf[512];
  snprintf(buf, sizeof buf, "mk_run_noalloc: %s%s%s", msg, detail ? ": " : "", detail ? detail : "");
  mk::set_noplan_error(buf);
  return st;
}

// Once per device, with that device current: the device address of the
// array, and the kernels' shared-memory attributes.
mk_status setup_device(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_err(MK_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return set_err(MK_ERR_CUDA, "cudaGetSymbolAddress failed", cudaGetErrorString(e));
    e = mk::prepare_kernels();
    if (e != cudaSuccess) return set_err(MK_ERR_CUDA, "kernel setup failed", cudaGetErrorString(e));
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return MK_OK;
}

// A device time-out of the contraction (its bounded waits) sets the error
// word; the call does not wait for the GPU, so instead of a status the
// outputs are overwritten with NaN, which no valid result contains.
__global__ void poison_kernel(const int* __restrict__ err, float* __restrict__ fields, size_t nf,
                              double* __restrict__ energy, size_t ne) {
  if (*err == 0) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) fields[i] = __int_as_float(0x7fc00000);
  if (energy)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += stride)
      energy[i] = __longlong_as_double(0x7ff8000000000000LL);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" mk_status mk_run_noalloc(const mk_desc* d, const void* R, const float* Gd, const double* td,
                                    double eps_s, int32_t niter, float* fields, double* energy,
                                    void* cuda_stream) {
  mk::set_noplan_error("");
  if (!d || !R || !Gd || !td || !fields) return set_err(MK_ERR_ARG, "null pointer argument");
  if (niter < 0 || !isfinite(eps_s)) return set_err(MK_ERR_ARG, "niter < 0 or eps not finite");
  if (d->nsrc < 1 || d->nfocal < 1 || d->nsrc != d->nrec)
    return set_err(MK_ERR_ARG, "nsrc == nrec >= 1 and nfocal >= 1 are required");
  if (d->nt < 32 || d->nt > 8192 || (d->nt & (d->nt - 1)))
    return set_err(MK_ERR_UNSUPPORTED, "nt must be a power of two in [32, 8192]");
  if (!(d->dt > 0.0) || !(d->dx > 0.0)) return set_err(MK_ERR_ARG, "dt and dx must be > 0");
  if (d->rprec != MK_R_C64) return set_err(MK_ERR_UNSUPPORTED, "only complex FP32 R (MK_R_C64)");
  if (d->row_count != 0 && !(d->row_begin == 0 && d->row_count == d->nsrc))
    return set_err(MK_ERR_UNSUPPORTED, "shot-row shards need a plan (mk_plan)");
  if ((int64_t)d->nsrc * d->nfocal > (int64_t)1 << 30) return set_err(MK_ERR_ARG, "nsrc * nfocal too large");

  // sizes, strides and the carving of the scratch array
  mk::SurveyDev v;
  memset(&v, 0, sizeof v);
  v.ns = d->nsrc;
  v.nr = d->nrec;
  v.row0 = 0;
  v.nt = d->nt;
  v.F = d->nfocal;
  if (!(d->fmax_hz > 0.0)) {
    v.nw = d->nt / 2 + 1;
  } else {
    const double q = floor(d->fmax_hz * d->nt * d->dt);
    v.nw = (q >= d->nt / 2 ? d->nt / 2 : (int)q) + 1;
  }
  if (!mk::epilogue_fits(d->nt, v.nw)) return set_err(MK_ERR_UNSUPPORTED, "nt and band exceed the epilogue's shared memory");
  v.r_pad = (d->nrec + 31) / 32 * 32;
  v.ncols = v.ns * v.F;
  v.s_stride = ((int64_t)v.ncols + 1 + 3) / 4 * 4;
  v.nw_stride = (int64_t)v.r_pad * v.F;
  v.dt = d->dt;
  v.c = (float)(d->dx * d->dt);
  v.inv_nt = 1.0f / (float)d->nt;
  v.rprec = d->rprec;
  const size_t nw_bytes = align256((size_t)v.nw * v.nw_stride * sizeof(float2));
  const size_t s_bytes = align256((size_t)v.nw * v.s_stride * sizeof(float2));
  const size_t l_bytes = align256((size_t)(v.ncols + 1) * sizeof(int));
  const size_t e_bytes = align256((size_t)(v.ncols + 1) * sizeof(double));
  const size_t c_bytes = 256;
  const size_t tw_bytes = align256((size_t)v.nt * sizeof(float2));
  const size_t slot_bytes = align256((size_t)v.F * sizeof(double));
  const size_t err_bytes = 256;
  const size_t need = nw_bytes + s_bytes + l_bytes + e_bytes + c_bytes + 2 * tw_bytes + slot_bytes + err_bytes + 256;
  if (need > MK_NOALLOC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "the survey needs %zu bytes of scratch, the static array holds %zu (MK_NOALLOC_SCRATCH_BYTES); "
             "use mk_plan with a caller-allocated workspace",
             need, (size_t)MK_NOALLOC_SCRATCH_BYTES);
    return set_err(MK_ERR_ARG, buf);
  }

  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(MK_ERR_CUDA, "cudaGetDevice failed", cudaGetErrorString(e));
  void* base_v = nullptr;
  mk_status st = setup_device(dev, &base_v);
  if (st != MK_OK) return st;
  int num_sms = 1;
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_err(MK_ERR_CUDA, "cudaDeviceGetAttribute failed", cudaGetErrorString(e));

  char* base = static_cast<char*>(base_v);
  size_t off = 0;
  v.Nw = reinterpret_cast<float2*>(base + off);
  off += nw_bytes;
  v.S = reinterpret_cast<float2*>(base + off);
  off += s_bytes;
  v.L = reinterpret_cast<int*>(base + off);
  off += l_bytes;
  v.Epart = reinterpret_cast<double*>(base + off);
  off += e_bytes;
  v.counter = reinterpret_cast<unsigned*>(base + off);
  off += c_bytes;
  v.iter = reinterpret_cast<int*>(base + off);  // starts at 0 (cleared below)
  off += 256;
  v.err = reinterpret_cast<int*>(base + off);   // error word of the bounded waits (cleared below)
  off += err_bytes;
  float2* tw = reinterpret_cast<float2*>(base + off);
  off += tw_bytes;
  float2* twl = reinterpret_cast<float2*>(base + off);
  off += tw_bytes;
  double* slot = reinterpret_cast<double*>(base + off);
  v.tw = tw;
  v.twl = twl;
  v.td = nullptr;
  v.scratch = nullptr;
  v.R = static_cast<const float2*>(R);
  const size_t field = (size_t)v.F * v.ns * v.nt;
  v.fN = fields;
  v.f1p = fields + field;
  v.f1m = fields + 2 * field;
  v.f2p = fields + 3 * field;
  v.pmin = fields + 4 * field;

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // The array keeps the previous call's contents: clear everything this call
  // reads before writing (Nw padding, S padding, completion counter).
  if ((e = cudaMemsetAsync(base, 0, off, stream)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "cudaMemsetAsync failed", cudaGetErrorString(e));
  if ((e = mk::launch_twiddles(tw, v.nt, stream)) != cudaSuccess ||
      (e = mk::launch_twiddles_linear(twl, v.nt, stream)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "twiddle launch", cudaGetErrorString(e));
  if ((e = mk::launch_windows(v, td, eps_s, stream)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "window launch", cudaGetErrorString(e));
  if ((e = mk::launch_init(v, Gd, stream, num_sms)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "init launch", cudaGetErrorString(e));
  for (int it = 0; it < niter; ++it) {
    int nl = 0;
    if ((e = mk::launch_contract(v, nullptr, stream, num_sms, &nl)) != cudaSuccess)
      return set_err(MK_ERR_CUDA, "contraction launch", cudaGetErrorString(e));
    if ((e = energy ? mk::launch_epilogue(v, energy, niter, stream, num_sms)
                    : mk::launch_epilogue(v, slot, 1, stream, num_sms)) != cudaSuccess)
      return set_err(MK_ERR_CUDA, "epilogue launch", cudaGetErrorString(e));
  }
  // The iterations accumulate f1plus and f1min; N, f2p and pmin follow from
  // them (the pmin slot of the output serves as the input of its synthesis).
  if (niter > 0 && (e = mk::launch_inverse(v, v.fN, 0, stream, num_sms)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "inverse launch", cudaGetErrorString(e));
  if ((e = mk::launch_f2p(v, v.pmin, stream, num_sms)) != cudaSuccess)
    return set_err(MK_ERR_CUDA, "f2p launch", cudaGetErrorString(e));
  if (niter == 0) {
    if ((e = cudaMemsetAsync(v.pmin, 0, field * sizeof(float), stream)) != cudaSuccess)
      return set_err(MK_ERR_CUDA, "cudaMemsetAsync failed", cudaGetErrorString(e));
  } else {
    int nl = 0;
    if ((e = mk::launch_spectrum(v, v.pmin, stream, num_sms)) != cudaSuccess ||
        (e = mk::launch_contract(v, nullptr, stream, num_sms, &nl)) != cudaSuccess ||
        (e = mk::launch_inverse(v, v.pmin, 1, stream, num_sms)) != cudaSuccess)
      return set_err(MK_ERR_CUDA, "pmin synthesis launch", cudaGetErrorString(e));
  }
  poison_kernel<<<num_sms * 4, 256, 0, stream>>>(v.err, fields, 5 * field, energy, energy ? (size_t)niter * v.F : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_err(MK_ERR_CUDA, "error check launch", cudaGetErrorString(e));
  return MK_OK;
}
