// Host side of the C ABI declared in include/marchenko.h: argument checks,
// workspace carving, call-order state, launches and error reporting.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/marchenko.h"
#include "mk_internal.h"

namespace {

constexpr int kMaxIterSlots = 256;  // energies buffered on the device per chunk of iterations
constexpr size_t kAlign = 256;

thread_local char g_noplan_err[512] = "";

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Survey {
  mk_desc d;
  mk::SurveyDev dev;
  mk::UmmaMaps* umma = nullptr;  // tensor maps (16-bit R precisions)
  double* energy = nullptr;  // [kMaxIterSlots][F] device
  std::vector<unsigned char> loaded;
  int nloaded = 0;
  bool ready = false;
  int iter = 0;
  bool n_in_field = true;   // fN holds the last N (else it follows from S)
  bool derived_valid = false;  // f2p and pmin formed since the last change
  bool gm_valid = false, gp_valid = false;  // G^- and G^+ formed since the last change
  // R was written (mk_load_R, mk_load_R_time) since the last contraction launch:
  // the next contraction must not start as a programmatic dependent
  bool r_written = true;
  float2* pacc = nullptr;   // band spectrum of pmin, accumulated by the iterations (F = 1 surveys)
  bool pacc_valid = false;  // pacc holds the spectrum of pmin of the current series
  size_t offset = 0, bytes = 0;  // carving inside the workspace
  // streaming of R from pinned host memory (MK_FLAG_STREAM_R)
  bool stream_r = false;
  int chunk_w = 0;                  // frequencies per streamed chunk
  float2* rbuf[2] = {nullptr, nullptr};  // device chunk buffers
  const float2* host_r = nullptr;   // caller's pinned R, [nw][ns][r_pad]
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ready_ev[2] = {nullptr, nullptr}, free_ev[2] = {nullptr, nullptr};
  mk_tuning_t tuning = {0, 0, 0, 0, 0.f, 0.f};
};

struct TimedPair {
  cudaEvent_t a, b;
  int kind;  // 0 contraction, 1 epilogue
};

}  // namespace

struct mk_plan_s {
  std::vector<Survey> s;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 1;
  bool timing = false;
  int timing_stride = 1;        // time the launches of every timing_stride-th iteration
  unsigned long long timing_count = 0;  // iterations launched with timing on
  char err[512] = "";
  mk_stats_t stats{};
  std::vector<TimedPair> events;  // created once, reused
  size_t next_event = 0;
  bool graph = false;                       // MK_FLAG_GRAPH on every survey
  cudaStream_t cap_stream = nullptr;        // capture stream and per-survey branches
  std::vector<cudaStream_t> side;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  cudaGraphExec_t graph_exec = nullptr;
  int* err_host = nullptr;  // page-locked copy of the device error words (one per survey)
};

namespace {

mk_status fail(mk_plan_t p, mk_status st, const char* fmt, ...) {
  char* buf = p ? p->err : g_noplan_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define MK_CUDA(p, call)                                                                    \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((p), MK_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                      \
  } while (0)

int band_bins(const mk_desc& d) {
  if (!(d.fmax_hz > 0.0)) return d.nt / 2 + 1;
  const double q = floor(d.fmax_hz * d.nt * d.dt);
  const int half = d.nt / 2;
  return (q >= half ? half : (int)q) + 1;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

mk_status check_desc(mk_plan_t p, const mk_desc& d, int i) {
  if (d.nsrc < 1 || d.nrec < 1 || d.nfocal < 1)
    return fail(p, MK_ERR_ARG, "survey %d: nsrc, nrec and nfocal must be >= 1", i);
  if (d.nsrc != d.nrec)
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: nsrc (%d) != nrec (%d); coincident positions required",
                i, d.nsrc, d.nrec);
  if (!is_pow2(d.nt) || d.nt < 32 || d.nt > 8192)
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: nt=%d must be a power of two in [32, 8192]", i, d.nt);
  if (!(d.dt > 0.0) || !(d.dx > 0.0) || !isfinite(d.dt) || !isfinite(d.dx))
    return fail(p, MK_ERR_ARG, "survey %d: dt and dx must be finite and > 0", i);
  if (!mk::epilogue_fits(d.nt, band_bins(d)))
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: nt=%d with %d kept bins exceeds the epilogue's shared memory", i,
                d.nt, band_bins(d));
  if (d.rprec < MK_R_C64 || d.rprec > MK_R_SPLIT_F16)
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: unknown R storage precision %d", i, d.rprec);
  if ((d.flags & MK_FLAG_STREAM_R) && d.rprec != MK_R_C64)
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: streaming R from the host needs complex FP32 R", i);
  if ((int64_t)d.nsrc * d.nfocal > (int64_t)1 << 30)
    return fail(p, MK_ERR_ARG, "survey %d: nsrc * nfocal too large", i);
  if (d.row_count < 0 || (d.row_count > 0 && (d.row_begin < 0 || d.row_begin % 32 != 0 ||
                                               d.row_begin + d.row_count > d.nsrc)))
    return fail(p, MK_ERR_ARG, "survey %d: rows [%d, %d) must lie in [0, %d) and start at a multiple of 32", i,
                d.row_begin, d.row_begin + d.row_count, d.nsrc);
  if (d.row_count > 0 && (d.flags & MK_FLAG_STREAM_R))
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: a shot-row shard keeps its R resident", i);
  return MK_OK;
}

bool is_shard(const mk_desc& d) { return d.row_count > 0 && d.row_count < d.nsrc; }

// Sizes and strides of one survey; carves the workspace when base != nullptr.
size_t layout(Survey& sv, char* base) {
  const mk_desc& d = sv.d;
  mk::SurveyDev& v = sv.dev;
  v.ns = is_shard(d) ? d.row_count : d.nsrc;
  v.nr = d.nrec;
  v.row0 = is_shard(d) ? d.row_begin : 0;
  v.nt = d.nt;
  v.F = d.nfocal;
  v.nw = band_bins(d);
  // rows of R padded for aligned loads: to 32 complex values for the tensor-core and
  // SIMT GEMM tiles and for the host layout of streamed R; a GEMV-only survey (complex
  // FP32, one focal point, resident R) needs 16-byte rows only, an even count
  const bool gemv_only = d.rprec == MK_R_C64 && d.nfocal == 1 && !(d.flags & MK_FLAG_STREAM_R) && !is_shard(d);
  v.r_pad = gemv_only ? (d.nrec + 1) / 2 * 2 : (d.nrec + 31) / 32 * 32;
  v.ncols = v.ns * v.F;
  v.s_stride = ((int64_t)v.ncols + 1 + 3) / 4 * 4;
  v.nw_stride = (int64_t)v.r_pad * v.F;
  v.dt = d.dt;
  v.c = (float)(d.dx * d.dt);
  v.inv_nt = 1.0f / (float)d.nt;
  v.rprec = d.rprec;
  v.epi_g = 0;
  v.pdl = 0;
  v.pacc = nullptr;
  v.rsc = v.nsc = nullptr;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off += align_up(bytes);
    return ptr;
  };
  const size_t field = (size_t)v.F * v.ns * v.nt * sizeof(float);
  if (d.rprec == MK_R_C64 && (d.flags & MK_FLAG_STREAM_R)) {
    // two chunk buffers of chunk_w frequencies: at least 4 chunks, at most 128 MB each
    const size_t row = (size_t)v.ns * v.r_pad * sizeof(float2);
    int cw = (v.nw + 3) / 4;
    const int cap = (int)((size_t)128 << 20) / (int)(row ? row : 1);
    if (cw > cap) cw = cap;
    if (cw < 1) cw = 1;
    sv.stream_r = true;
    sv.chunk_w = cw;
    sv.rbuf[0] = reinterpret_cast<float2*>(take((size_t)cw * row));
    sv.rbuf[1] = reinterpret_cast<float2*>(take((size_t)cw * row));
    v.R = nullptr;
    v.Nw = reinterpret_cast<float2*>(take((size_t)v.nw * v.nw_stride * sizeof(float2)));
    v.Rq0 = v.Rq1 = v.Rq2 = nullptr;
    v.Bq0 = v.Bq1 = v.Bq2 = nullptr;
  } else if (d.rprec == MK_R_C64) {
    v.R = reinterpret_cast<const float2*>(take((size_t)v.nw * v.ns * v.r_pad * sizeof(float2)));
    v.Nw = reinterpret_cast<float2*>(take((size_t)v.nw * v.nw_stride * sizeof(float2)));
    v.Rq0 = v.Rq1 = v.Rq2 = nullptr;
    v.Bq0 = v.Bq1 = v.Bq2 = nullptr;
  } else {
    // 16-bit interleaved complex rows of 2 r_pad values; field embedding [nw][2F][2 r_pad]
    const size_t rq = (size_t)v.nw * v.ns * 2 * v.r_pad * 2;
    const size_t bq = (size_t)v.nw * 2 * v.F * 2 * v.r_pad * 2;
    v.R = nullptr;
    v.Nw = nullptr;
    v.Rq0 = take(rq);
    v.Rq1 = d.rprec >= MK_R_SPLIT_BF16 ? take(rq) : nullptr;
    v.Rq2 = d.rprec == MK_R_SPLIT3_BF16 ? take(rq) : nullptr;
    v.Bq0 = take(bq);
    v.Bq1 = take(bq);
    v.Bq2 = d.rprec == MK_R_SPLIT3_BF16 ? take(bq) : nullptr;
    if (d.rprec == MK_R_SPLIT_F16) {
      // the epilogue writes the FP32 field spectrum; each contraction scales and
      // splits it into the embedding (powers of two per frequency and focal point)
      v.Nw = reinterpret_cast<float2*>(take((size_t)v.nw * v.nw_stride * sizeof(float2)));
      v.rsc = reinterpret_cast<float*>(take((size_t)v.nw * sizeof(float)));
      v.nsc = reinterpret_cast<float*>(take((size_t)v.nw * v.F * sizeof(float)));
    }
  }
  v.S = reinterpret_cast<float2*>(take((size_t)v.nw * v.s_stride * sizeof(float2)));
  // a survey contracted by the GEMV (complex FP32, one focal point, resident or
  // streamed R) accumulates pmin as a band spectrum during the iterations
  // (Algorithm 1 adds every synthesis result to pmin): n_w * ns complex values,
  // far less than R, and no extra contraction when pmin or G is fetched
  // A shot-row shard keeps it too: its fetch-time synthesis would need the
  // field spectrum of every shard.
  const bool gemv = d.rprec == MK_R_C64 && d.nfocal == 1;
  sv.pacc = gemv || is_shard(d) ? reinterpret_cast<float2*>(take((size_t)v.nw * v.s_stride * sizeof(float2)))
                                : nullptr;
  v.fN = reinterpret_cast<float*>(take(field));
  v.f1p = reinterpret_cast<float*>(take(field));
  v.f1m = reinterpret_cast<float*>(take(field));
  v.f2p = reinterpret_cast<float*>(take(field));
  v.pmin = reinterpret_cast<float*>(take(field));
  v.scratch = reinterpret_cast<float*>(take(field));
  v.gm = reinterpret_cast<float*>(take(field));
  v.gp = reinterpret_cast<float*>(take(field));
  v.L = reinterpret_cast<int*>(take((size_t)(v.ncols + 1) * sizeof(int)));
  v.td = reinterpret_cast<double*>(take((size_t)v.ncols * sizeof(double)));
  v.Epart = reinterpret_cast<double*>(take((size_t)(v.ncols + 1) * sizeof(double)));
  v.counter = reinterpret_cast<unsigned*>(take(8 * sizeof(unsigned)));
  v.err = reinterpret_cast<int*>(take(sizeof(int)));
  v.iter = reinterpret_cast<int*>(take(sizeof(int)));
  v.tw = reinterpret_cast<const float2*>(take((size_t)v.nt * sizeof(float2)));
  v.twl = reinterpret_cast<const float2*>(take((size_t)v.nt * sizeof(float2)));
  sv.energy = reinterpret_cast<double*>(take((size_t)kMaxIterSlots * v.F * sizeof(double)));
  return off;
}

mk_status get_survey(mk_plan_t p, int32_t survey, Survey** out) {
  if (!p) return fail(nullptr, MK_ERR_ARG, "null plan");
  if (survey < 0 || survey >= (int32_t)p->s.size())
    return fail(p, MK_ERR_ARG, "survey index %d out of range [0, %d)", survey, (int)p->s.size());
  *out = &p->s[survey];
  return MK_OK;
}

mk_status ensure_device(mk_plan_t p) {
  int dev = -1;
  MK_CUDA(p, cudaGetDevice(&dev));
  if (dev != p->device)
    return fail(p, MK_ERR_STATE, "current device %d is not the plan's device %d", dev, p->device);
  return MK_OK;
}

// Reads and clears the device error words (after a stream synchronisation).
mk_status check_device_errors(mk_plan_t p) {
  if (!p->err_host) {
    // page-locked, so the read is an ordinary stream-ordered copy
    MK_CUDA(p, cudaHostAlloc(reinterpret_cast<void**>(&p->err_host), p->s.size() * sizeof(int), cudaHostAllocDefault));
  }
  for (size_t i = 0; i < p->s.size(); ++i)
    MK_CUDA(p, cudaMemcpyAsync(p->err_host + i, p->s[i].dev.err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  MK_CUDA(p, cudaStreamSynchronize(p->stream));
  for (size_t i = 0; i < p->s.size(); ++i) {
    const int h = p->err_host[i];
    if (h != 0) {
      MK_CUDA(p, cudaMemsetAsync(p->s[i].dev.err, 0, sizeof(int), p->stream));
      return fail(p, MK_ERR_TIMEOUT, "survey %d: a bounded device wait ran out (code %d); results are invalid",
                  (int)i, h);
    }
  }
  return MK_OK;
}

TimedPair* next_pair(mk_plan_t p, int kind) {
  if (!p->timing) return nullptr;
  if (p->next_event == p->events.size()) {
    TimedPair tp;
    if (cudaEventCreate(&tp.a) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&tp.b) != cudaSuccess) {
      cudaEventDestroy(tp.a);
      return nullptr;
    }
    p->events.push_back(tp);
  }
  TimedPair* tp = &p->events[p->next_event++];
  tp->kind = kind;
  return tp;
}

// Forms the fields Algorithm 1 accumulates but the hot loop does not (N_last,
// f2p, pmin) from the accumulated ones, for a fetch:
//   N_last = -theta s_last(-t) (inverse transform of the last synthesis S),
//   f2p = f1plus - f1min(-t),  pmin = synthesis(f2p - N_last).
// The pmin synthesis reuses the contraction; the band spectrum of N_last is
// restored afterwards so the series continues unchanged.
// The contraction of one survey on stream st.  With R streamed from pinned
// host memory, R arrives in chunks of chunk_w frequencies on the survey's
// copy stream, double-buffered: the copy of chunk c + 1 overlaps the
// contraction of chunk c (each chunk is an independent set of frequencies).
mk_status contract(mk_plan_t p, Survey& sv, cudaStream_t st, int* nlaunch) {
  if (!sv.stream_r) {
    mk::SurveyDev v = sv.dev;
    // the GEMV may stream R before the preceding kernel ends only when that
    // kernel cannot have written R
    v.pdl = sv.r_written ? 0 : 1;
    sv.r_written = false;
    MK_CUDA(p, mk::launch_contract(v, sv.umma, st, p->num_sms, nlaunch));
    return MK_OK;
  }
  mk::SurveyDev v = sv.dev;
  v.pdl = 0;
  const size_t row = (size_t)v.ns * v.r_pad;  // complex elements per frequency
  *nlaunch = 0;
  int c = 0;
  for (int w0 = 0; w0 < sv.dev.nw; w0 += sv.chunk_w, ++c) {
    const int cw = sv.dev.nw - w0 < sv.chunk_w ? sv.dev.nw - w0 : sv.chunk_w;
    const int b = c & 1;
    // the buffer is free once the contraction that last read it is done
    MK_CUDA(p, cudaStreamWaitEvent(sv.copy_stream, sv.free_ev[b], 0));
    MK_CUDA(p, cudaMemcpyAsync(sv.rbuf[b], sv.host_r + (size_t)w0 * row, (size_t)cw * row * sizeof(float2),
                               cudaMemcpyHostToDevice, sv.copy_stream));
    MK_CUDA(p, cudaEventRecord(sv.ready_ev[b], sv.copy_stream));
    MK_CUDA(p, cudaStreamWaitEvent(st, sv.ready_ev[b], 0));
    v.R = sv.rbuf[b];
    v.nw = cw;
    v.Nw = sv.dev.Nw + (size_t)w0 * v.nw_stride;
    v.S = sv.dev.S + (size_t)w0 * v.s_stride;
    int nl = 0;
    MK_CUDA(p, mk::launch_contract(v, nullptr, st, p->num_sms, &nl));
    MK_CUDA(p, cudaEventRecord(sv.free_ev[b], st));
    *nlaunch += nl;
  }
  return MK_OK;
}

// Tuning (MK_FLAG_AUTOTUNE): per-process cache of the fastest kernel shapes,
// keyed by (nsrc, nt, n_w, nfocal, rprec) and the device's SM count.
struct TuneChoice {
  int bn, g;
  float contract_ms, epilogue_ms;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, TuneChoice> g_tune_cache;

// Times each candidate shape of the survey's contraction and epilogue on its
// own buffers (the fields are initialised afterwards) and keeps the fastest.
mk_status tune_survey(mk_plan_t p, Survey& sv) {
  mk::SurveyDev& v = sv.dev;
  const auto key = std::make_tuple(v.ns, v.nt, v.nw, v.F, v.rprec, p->num_sms);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      if (sv.umma && !mk::umma_set_bn(sv.umma, v, it->second.bn))
        return fail(p, MK_ERR_CUDA, "tensor map encoding for N tile %d failed", it->second.bn);
      v.epi_g = it->second.g;
      sv.tuning = {2, sv.umma ? it->second.bn : 0, it->second.g, 0, it->second.contract_ms, it->second.epilogue_ms};
      return MK_OK;
    }
  }
  cudaEvent_t e0, e1;
  MK_CUDA(p, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(p, MK_ERR_CUDA, "cudaEventCreate failed");
  }
  int candidates = 0;
  mk_status result = MK_OK;
  // best of three timed runs after one untimed run
  auto time_it = [&](auto&& launch, float* best) -> mk_status {
    *best = 1e30f;
    for (int r = 0; r < 4; ++r) {
      MK_CUDA(p, cudaEventRecord(e0, p->stream));
      int nl = 0;
      mk_status st = launch(&nl);
      if (st != MK_OK) return st;
      MK_CUDA(p, cudaEventRecord(e1, p->stream));
      MK_CUDA(p, cudaEventSynchronize(e1));
      float ms = 0.f;
      MK_CUDA(p, cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0 && ms < *best) *best = ms;
    }
    ++candidates;
    return MK_OK;
  };
  TuneChoice best = {sv.umma ? mk::umma_get_bn(sv.umma) : 0, 0, 0.f, 0.f};
  do {
    if (sv.umma) {
      int cover = 16;
      while (cover < 2 * v.F && cover < 128) cover *= 2;
      float best_ms = 1e30f;
      for (int bn = 16; bn <= cover; bn *= 2) {
        if (!mk::umma_set_bn(sv.umma, v, bn)) {
          result = fail(p, MK_ERR_CUDA, "tensor map encoding for N tile %d failed", bn);
          break;
        }
        float ms = 0.f;
        result = time_it([&](int* nl) { return contract(p, sv, p->stream, nl); }, &ms);
        if (result != MK_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          best.bn = bn;
        }
      }
      if (result != MK_OK) break;
      if (!mk::umma_set_bn(sv.umma, v, best.bn)) {
        result = fail(p, MK_ERR_CUDA, "tensor map encoding for N tile %d failed", best.bn);
        break;
      }
      best.contract_ms = best_ms;
    }
    // the epilogue advances the device iteration index: start it from 0
    MK_CUDA(p, mk::launch_set_iter(v, 0, p->stream));
    const int gmax = mk::epilogue_max_pairs(v, p->num_sms);
    float best_ms = 1e30f;
    for (int g = 1; g <= gmax; g *= 2) {
      v.epi_g = g;
      float ms = 0.f;
      result = time_it(
          [&](int* nl) -> mk_status {
            *nl = 1;
            MK_CUDA(p, mk::launch_epilogue(v, sv.energy, kMaxIterSlots, p->stream, p->num_sms));
            return MK_OK;
          },
          &ms);
      if (result != MK_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best.g = g;
      }
    }
    if (result != MK_OK) break;
    v.epi_g = best.g;
    best.epilogue_ms = best_ms;
  } while (false);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != MK_OK) return result;
  sv.tuning = {1, sv.umma ? best.bn : 0, best.g, candidates, best.contract_ms, best.epilogue_ms};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return MK_OK;
}

// One plain synthesis (Eq. 1 before the mute) of a field into dst: band
// spectrum, contraction, inverse transform.  Overwrites Nw and S.
mk_status synthesize(mk_plan_t p, Survey& sv, const float* src, float* dst) {
  mk::SurveyDev& v = sv.dev;
  int nl = 0;
  MK_CUDA(p, mk::launch_spectrum(v, src, p->stream, p->num_sms));
  mk_status st = contract(p, sv, p->stream, &nl);
  if (st != MK_OK) return st;
  MK_CUDA(p, mk::launch_inverse(v, dst, 1, p->stream, p->num_sms));
  p->stats.launches += 2 + nl;
  p->stats.other_launches += 2 + nl;
  return MK_OK;
}

// G^- = synthesis(f1plus) - f1min (Algorithm 1, after the loop) and
// G^+ = f1plus(-t) - synthesis(f1min(-t)), each one extra synthesis.
mk_status materialize_up_down(mk_plan_t p, Survey& sv, uint32_t mask) {
  mk::SurveyDev& v = sv.dev;
  mk_status st;
  bool touched = false;
  if ((mask & MK_F_GMINUS) && !sv.gm_valid) {
    if ((st = synthesize(p, sv, v.f1p, v.scratch)) != MK_OK) return st;
    MK_CUDA(p, mk::launch_lincomb(v, v.gm, v.scratch, 0, 1.f, v.f1m, 0, -1.f, p->stream, p->num_sms));
    p->stats.launches++;
    p->stats.other_launches++;
    sv.gm_valid = touched = true;
  }
  if ((mask & MK_F_GPLUS) && !sv.gp_valid) {
    MK_CUDA(p, mk::launch_lincomb(v, v.scratch, v.f1m, 1, 1.f, nullptr, 0, 0.f, p->stream, p->num_sms));
    if ((st = synthesize(p, sv, v.scratch, v.scratch)) != MK_OK) return st;
    MK_CUDA(p, mk::launch_lincomb(v, v.gp, v.f1p, 1, 1.f, v.scratch, 0, -1.f, p->stream, p->num_sms));
    p->stats.launches += 2;
    p->stats.other_launches += 2;
    sv.gp_valid = touched = true;
  }
  if (touched) {  // restore the band spectrum of N_last for the next iteration
    MK_CUDA(p, mk::launch_spectrum(v, v.fN, p->stream, p->num_sms));
    p->stats.launches++;
    p->stats.other_launches++;
  }
  return MK_OK;
}

mk_status materialize(mk_plan_t p, Survey& sv, uint32_t mask) {
  mk::SurveyDev& v = sv.dev;
  const bool need_pmin = mask & (MK_F_PMIN | MK_F_G);
  if (is_shard(sv.d)) {
    // a shard holds only its own positions of every field: what needs a
    // synthesis of a whole field needs the other shards
    if (mask & (MK_F_GMINUS | MK_F_GPLUS))
      return fail(p, MK_ERR_UNSUPPORTED, "G^- and G^+ of a shot-row shard need the fields of every shard");
    if (need_pmin && sv.iter > 0 && !sv.pacc_valid && !sv.derived_valid)
      return fail(p, MK_ERR_UNSUPPORTED, "pmin of a shot-row shard whose R changed during the series");
  }
  const bool need_f2p = need_pmin || (mask & MK_F_F2P);
  const bool need_n = need_f2p || (mask & (MK_F_N | MK_F_GMINUS | MK_F_GPLUS));
  if (need_n && !sv.n_in_field) {
    MK_CUDA(p, mk::launch_inverse(v, v.fN, 0, p->stream, p->num_sms));
    p->stats.launches++;
    p->stats.other_launches++;
    sv.n_in_field = true;
  }
  if (mask & (MK_F_GMINUS | MK_F_GPLUS)) {
    mk_status st = materialize_up_down(p, sv, mask);
    if (st != MK_OK) return st;
  }
  if (!need_f2p || sv.derived_valid) return MK_OK;
  MK_CUDA(p, mk::launch_f2p(v, v.scratch, p->stream, p->num_sms));  // f2p, and f2p - N into scratch
  p->stats.launches++;
  p->stats.other_launches++;
  const size_t field = (size_t)v.F * v.ns * v.nt * sizeof(float);
  if (sv.iter == 0) {
    MK_CUDA(p, cudaMemsetAsync(v.pmin, 0, field, p->stream));
  } else if (sv.pacc_valid) {
    // pmin = sum of the iterations' synthesis results: one inverse transform of
    // their summed band spectra
    mk::SurveyDev w = v;
    w.S = sv.pacc;
    MK_CUDA(p, mk::launch_inverse(w, v.pmin, 1, p->stream, p->num_sms));
    p->stats.launches++;
    p->stats.other_launches++;
  } else {
    int nl = 0;
    MK_CUDA(p, mk::launch_spectrum(v, v.scratch, p->stream, p->num_sms));
    mk_status st = contract(p, sv, p->stream, &nl);
    if (st != MK_OK) return st;
    MK_CUDA(p, mk::launch_inverse(v, v.pmin, 1, p->stream, p->num_sms));
    MK_CUDA(p, mk::launch_spectrum(v, v.fN, p->stream, p->num_sms));  // restore the spectrum of N_last
    p->stats.launches += 3 + nl;
    p->stats.other_launches += 3 + nl;
  }
  sv.derived_valid = true;
  return MK_OK;
}

}  // namespace

namespace mk {
void set_noplan_error(const char* msg) { snprintf(g_noplan_err, sizeof g_noplan_err, "%s", msg); }
}  // namespace mk

extern "C" {

mk_status mk_workspace_size(const mk_desc* d, int32_t ndesc, size_t* bytes) {
  g_noplan_err[0] = 0;
  if (!d || !bytes || ndesc < 1) return fail(nullptr, MK_ERR_ARG, "null pointer or ndesc < 1");
  size_t total = 0;
  for (int i = 0; i < ndesc; ++i) {
    mk_status st = check_desc(nullptr, d[i], i);
    if (st != MK_OK) return st;
    Survey sv;
    sv.d = d[i];
    total += layout(sv, nullptr);
  }
  *bytes = total;
  return MK_OK;
}

mk_status mk_plan(const mk_desc* d, int32_t ndesc, void* cuda_stream, void* workspace,
                  size_t workspace_bytes, mk_plan_t* out) {
  g_noplan_err[0] = 0;
  if (!d || !out || ndesc < 1 || !workspace) return fail(nullptr, MK_ERR_ARG, "null pointer or ndesc < 1");
  *out = nullptr;
  if (((uintptr_t)workspace) % kAlign != 0) return fail(nullptr, MK_ERR_ARG, "workspace not 256-byte aligned");
  size_t need = 0;
  mk_status st = mk_workspace_size(d, ndesc, &need);
  if (st != MK_OK) return st;
  if (workspace_bytes < need)
    return fail(nullptr, MK_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
                need);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, workspace);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(nullptr, MK_ERR_ARG, "workspace is not device memory");
  }
  mk_plan_t p = new (std::nothrow) mk_plan_s();
  if (!p) return fail(nullptr, MK_ERR_OOM, "host allocation of the plan failed");
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->device = attr.device;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != attr.device) {
    delete p;
    return fail(nullptr, MK_ERR_ARG, "workspace belongs to device %d, current device is %d", attr.device, cur);
  }
  if ((e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, cur)) != cudaSuccess ||
      (e = mk::prepare_kernels()) != cudaSuccess) {
    delete p;
    return fail(nullptr, MK_ERR_CUDA, "device setup failed: %s", cudaGetErrorString(e));
  }
  p->s.resize(ndesc);
  size_t off = 0;
  char* base = static_cast<char*>(workspace);
  bool timing = true, graph = true;
  for (int i = 0; i < ndesc; ++i) {
    Survey& sv = p->s[i];
    sv.d = d[i];
    sv.offset = off;
    sv.bytes = layout(sv, base + off);
    off += sv.bytes;
    sv.loaded.assign(sv.dev.nw, 0);
    timing = timing && (d[i].flags & MK_FLAG_TIMING);
    graph = graph && (d[i].flags & MK_FLAG_GRAPH);
  }
  p->timing = timing;
  p->graph = graph;
  // Zero the workspace (padding of R and Nw must be zero), then the twiddles.
  if ((e = cudaMemsetAsync(workspace, 0, off, p->stream)) != cudaSuccess) {
    delete p;
    return fail(nullptr, MK_ERR_CUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
  }
  for (auto& sv : p->s) {
    if (sv.d.rprec != MK_R_C64) {
      sv.umma = mk::umma_create(sv.dev);
      if (!sv.umma) {
        for (auto& o : p->s) mk::umma_destroy(o.umma);
        delete p;
        return fail(nullptr, MK_ERR_CUDA, "tensor map encoding for the tensor-core contraction failed");
      }
    }
    // the FFT twiddle table, formed on the device (the same generator serves
    // every entry point)
    e = mk::launch_twiddles(const_cast<float2*>(sv.dev.tw), sv.dev.nt, p->stream);
    if (e == cudaSuccess) e = mk::launch_twiddles_linear(const_cast<float2*>(sv.dev.twl), sv.dev.nt, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
      for (auto& o : p->s) mk::umma_destroy(o.umma);
      delete p;
      return fail(nullptr, MK_ERR_CUDA, "twiddle upload failed: %s", cudaGetErrorString(e));
    }
  }
  *out = p;
  return MK_OK;
}

mk_status mk_load_R(mk_plan_t p, int32_t survey, const void* Rw, int32_t w_begin, int32_t w_count,
                    int32_t src_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  const mk::SurveyDev& v = sv->dev;
  if (sv->stream_r) return fail(p, MK_ERR_STATE, "survey %d streams R from the host: use mk_attach_R_host", survey);
  if (!Rw) return fail(p, MK_ERR_ARG, "null R pointer");
  if (w_begin < 0 || w_count < 0 || w_begin + w_count > v.nw)
    return fail(p, MK_ERR_ARG, "bins [%d, %d) outside the band [0, %d)", w_begin, w_begin + w_count, v.nw);
  if (w_count == 0) return MK_OK;
  const int64_t rows = (int64_t)w_count * v.ns;
  const int64_t row0 = (int64_t)w_begin * v.ns;
  if (src_on_device < MK_SRC_HOST || src_on_device > MK_SRC_HOST_ASYNC)
    return fail(p, MK_ERR_ARG, "src_on_device must be MK_SRC_HOST, MK_SRC_DEVICE or MK_SRC_HOST_ASYNC");
  const float2* src = static_cast<const float2*>(Rw);
  bool direct = src_on_device == MK_SRC_DEVICE;
  bool pinned = false;
  if (!direct) {
    // pinned (page-locked) host memory is read in place (mapped) by the
    // conversion kernel or by the copy engine
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, Rw);
    if (e == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer) {
      src = static_cast<const float2*>(attr.devicePointer);
      pinned = true;
    } else {
      cudaGetLastError();
    }
    if (src_on_device == MK_SRC_HOST_ASYNC && !pinned)
      return fail(p, MK_ERR_ARG, "MK_SRC_HOST_ASYNC needs page-locked host memory");
  }
  // Page-locked host memory is read in place by the load kernel (one pass over
  // the host link).  An asynchronous load runs beside other work, so it takes
  // one block per SM, which already saturates the link, and leaves the rest
  // of each SM to the kernels it overlaps.
  const int max_blocks = src_on_device == MK_SRC_HOST_ASYNC ? p->num_sms : p->num_sms * 16;
  if (v.rprec == MK_R_C64) {
    float2* dst = const_cast<float2*>(v.R) + row0 * v.r_pad;
    if (direct || pinned) {
      MK_CUDA(p, mk::launch_load_rows(src, dst, rows, v.nr, v.r_pad, p->stream, max_blocks));
      p->stats.launches++;
      p->stats.other_launches++;
    } else {
      // pageable host memory: the CUDA driver stages the copy
      MK_CUDA(p, cudaMemcpy2DAsync(dst, (size_t)v.r_pad * sizeof(float2), Rw, (size_t)v.nr * sizeof(float2),
                                   (size_t)v.nr * sizeof(float2), (size_t)rows, cudaMemcpyHostToDevice,
                                   p->stream));
    }
  } else if (direct || pinned) {
    if (v.rprec == MK_R_SPLIT_F16) {  // the frequencies' scales first
      MK_CUDA(p, cudaMemsetAsync(v.rsc + w_begin, 0, (size_t)w_count * sizeof(float), p->stream));
      MK_CUDA(p, mk::launch_r_amax(src, v, row0, rows, p->stream, max_blocks));
      MK_CUDA(p, mk::launch_r_scale(v, w_begin, w_count, p->stream));
      p->stats.launches += 2;
      p->stats.other_launches += 2;
    }
    MK_CUDA(p, mk::launch_load_rows_q(src, v, row0, rows, p->stream, max_blocks));
    p->stats.launches++;
    p->stats.other_launches++;
  } else {
    // pageable host memory into 16-bit storage: chunks through the scratch field
    const size_t scratch_bytes = (size_t)v.F * v.ns * v.nt * sizeof(float);
    int64_t chunk = (int64_t)(scratch_bytes / ((size_t)v.nr * sizeof(float2)));
    if (chunk < 1) return fail(p, MK_ERR_UNSUPPORTED, "pageable R rows larger than the staging area");
    if (v.rprec == MK_R_SPLIT_F16) {  // the frequencies' scales: one staged pass before the conversion
      MK_CUDA(p, cudaMemsetAsync(v.rsc + w_begin, 0, (size_t)w_count * sizeof(float), p->stream));
      for (int64_t r = 0; r < rows; r += chunk) {
        const int64_t n = rows - r < chunk ? rows - r : chunk;
        MK_CUDA(p, cudaMemcpyAsync(v.scratch, static_cast<const float2*>(Rw) + r * v.nr,
                                   (size_t)n * v.nr * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
        MK_CUDA(p, mk::launch_r_amax(reinterpret_cast<const float2*>(v.scratch), v, row0 + r, n, p->stream,
                                     p->num_sms * 16));
      }
      MK_CUDA(p, mk::launch_r_scale(v, w_begin, w_count, p->stream));
    }
    for (int64_t r = 0; r < rows; r += chunk) {
      const int64_t n = rows - r < chunk ? rows - r : chunk;
      MK_CUDA(p, cudaMemcpyAsync(v.scratch, static_cast<const float2*>(Rw) + r * v.nr,
                                 (size_t)n * v.nr * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
      MK_CUDA(p, mk::launch_load_rows_q(reinterpret_cast<const float2*>(v.scratch), v, row0 + r, n, p->stream,
                                        p->num_sms * 16));
      p->stats.launches++;
      p->stats.other_launches++;
    }
  }
  sv->r_written = true;
  sv->pacc_valid = false;  // a series continued on new R: pmin follows from the current R
  sv->derived_valid = sv->gm_valid = sv->gp_valid = false;
  if (src_on_device == MK_SRC_HOST) MK_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int m = w_begin; m < w_begin + w_count; ++m) {
    if (!sv->loaded[m]) {
      sv->loaded[m] = 1;
      ++sv->nloaded;
    }
  }
  return MK_OK;
}

mk_status mk_load_R_time(mk_plan_t p, int32_t survey, const float* Rt, int32_t src_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  const mk::SurveyDev& v = sv->dev;
  if (sv->stream_r) return fail(p, MK_ERR_STATE, "survey %d streams R from the host: use mk_attach_R_host", survey);
  if (is_shard(sv->d)) return fail(p, MK_ERR_UNSUPPORTED, "survey %d is a shot-row shard: load its R rows with mk_load_R", survey);
  if (sv->d.rprec == MK_R_SPLIT_F16)
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d: the scaled FP16 split loads its band spectra with mk_load_R", survey);
  if (!Rt) return fail(p, MK_ERR_ARG, "null R pointer");
  const float* src = Rt;
  bool direct = src_on_device != 0;
  if (!direct) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, Rt);
    if (e == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer) {
      src = static_cast<const float*>(attr.devicePointer);  // pinned: read in place
      direct = true;
    } else {
      cudaGetLastError();
    }
  }
  // A view of R as a band-spectrum target: trace t = k * ns + r (source row
  // k, receiver r) lands at bin m in row k, column r of R_m.
  mk::SurveyDev t = v;
  t.nw_stride = (int64_t)v.ns * v.r_pad;
  t.rprec = v.rprec == MK_R_C64 ? 0 : 8 + v.rprec;
  const int64_t row_floats = (int64_t)v.ns * v.nt;  // one source row of traces
  // pageable host memory goes through the scratch field, F source rows at a time
  const int64_t kb = direct ? v.ns : (int64_t)v.F;
  for (int64_t k0 = 0; k0 < v.ns; k0 += kb) {
    const int64_t n = v.ns - k0 < kb ? v.ns - k0 : kb;
    const float* blk = src + k0 * row_floats;
    if (!direct) {
      MK_CUDA(p, cudaMemcpyAsync(v.scratch, Rt + k0 * row_floats, (size_t)(n * row_floats) * sizeof(float),
                                 cudaMemcpyHostToDevice, p->stream));
      blk = v.scratch;
    }
    t.F = (int)n;
    t.ncols = (int)(n * v.ns);
    const int64_t off = k0 * v.r_pad;  // complex elements
    if (v.rprec == MK_R_C64) {
      t.Nw = const_cast<float2*>(v.R) + off;
    } else {
      t.Rq0 = static_cast<const uint32_t*>(v.Rq0) + off;
      t.Rq1 = v.Rq1 ? static_cast<const uint32_t*>(v.Rq1) + off : nullptr;
      t.Rq2 = v.Rq2 ? static_cast<const uint32_t*>(v.Rq2) + off : nullptr;
    }
    MK_CUDA(p, mk::launch_spectrum(t, blk, p->stream, p->num_sms));
    p->stats.launches++;
    p->stats.other_launches++;
  }
  sv->r_written = true;
  sv->pacc_valid = false;
  sv->derived_valid = sv->gm_valid = sv->gp_valid = false;
  if (!src_on_device) MK_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int m = 0; m < v.nw; ++m) sv->loaded[m] = 1;
  sv->nloaded = v.nw;
  return MK_OK;
}

mk_status mk_attach_R_host(mk_plan_t p, int32_t survey, const void* Rpad, size_t bytes) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!sv->stream_r) return fail(p, MK_ERR_STATE, "survey %d keeps R resident: use mk_load_R", survey);
  const mk::SurveyDev& v = sv->dev;
  const size_t need = (size_t)v.nw * v.ns * v.r_pad * sizeof(float2);
  if (!Rpad || bytes != need) return fail(p, MK_ERR_ARG, "host R must be %zu bytes ([n_w][nsrc][r_pad])", need);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, Rpad);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(p, MK_ERR_ARG, "host R must be page-locked (pinned) memory");
  }
  if (!sv->copy_stream) {
    MK_CUDA(p, cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      MK_CUDA(p, cudaEventCreateWithFlags(&sv->ready_ev[b], cudaEventDisableTiming));
      MK_CUDA(p, cudaEventCreateWithFlags(&sv->free_ev[b], cudaEventDisableTiming));
      MK_CUDA(p, cudaEventRecord(sv->free_ev[b], p->stream));  // both buffers start free
    }
  }
  sv->host_r = static_cast<const float2*>(Rpad);
  sv->pacc_valid = false;  // a series continued on new R: pmin follows from the current R
  sv->derived_valid = sv->gm_valid = sv->gp_valid = false;
  for (int m = 0; m < v.nw; ++m) sv->loaded[m] = 1;
  sv->nloaded = v.nw;
  return MK_OK;
}

mk_status mk_get_tuning(mk_plan_t p, int32_t survey, mk_tuning_t* out) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  if (!out) return fail(p, MK_ERR_ARG, "null output");
  *out = sv->tuning;
  if (!out->tuned) {
    out->umma_bn = sv->umma ? mk::umma_get_bn(sv->umma) : 0;
    out->epi_pairs = sv->dev.epi_g;
  }
  return MK_OK;
}

mk_status mk_set_Gd_window(mk_plan_t p, int32_t survey, const float* Gd, const double* td, double eps_s,
                           int32_t src_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!Gd || !td) return fail(p, MK_ERR_ARG, "null G_d or t_d pointer");
  if (!isfinite(eps_s)) return fail(p, MK_ERR_ARG, "eps must be finite");
  mk::SurveyDev& v = sv->dev;
  if (sv->nloaded != v.nw)
    return fail(p, MK_ERR_STATE, "R of survey %d has %d of %d bins loaded", survey, sv->nloaded, v.nw);
  // windows from t_d, then N_{-1}, accumulators and the spectrum of N_{-1}
  const double* tsrc = td;
  const float* gsrc = Gd;
  if (!src_on_device) {
    MK_CUDA(p, cudaMemcpyAsync(v.td, td, (size_t)v.F * v.ns * sizeof(double), cudaMemcpyHostToDevice,
                               p->stream));
    MK_CUDA(p, cudaMemcpyAsync(v.scratch, Gd, (size_t)v.F * v.ns * v.nt * sizeof(float),
                               cudaMemcpyHostToDevice, p->stream));
    tsrc = v.td;
    gsrc = v.scratch;
  }
  MK_CUDA(p, mk::launch_windows(v, tsrc, eps_s, p->stream));
  if ((sv->d.flags & MK_FLAG_AUTOTUNE) && !sv->tuning.tuned) {
    // before the fields are initialised: tuning runs write them
    if ((st = tune_survey(p, *sv)) != MK_OK) return st;
    if (p->graph_exec) {  // captured launches hold the old shapes
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
  }
  MK_CUDA(p, mk::launch_init(v, gsrc, p->stream, p->num_sms));
  MK_CUDA(p, mk::launch_set_iter(v, 0, p->stream));
  if (sv->pacc)
    MK_CUDA(p, cudaMemsetAsync(sv->pacc, 0, (size_t)v.nw * v.s_stride * sizeof(float2), p->stream));
  p->stats.launches += 3;
  p->stats.other_launches += 3;
  if (!src_on_device) MK_CUDA(p, cudaStreamSynchronize(p->stream));
  sv->pacc_valid = sv->pacc != nullptr;
  sv->ready = true;
  sv->iter = 0;
  sv->n_in_field = true;
  sv->derived_valid = sv->gm_valid = sv->gp_valid = false;
  return MK_OK;
}

}  // extern "C"

namespace {

// One iteration of every survey: contraction then epilogue, survey after
// survey on one stream (timed launches), or -- when captured into a graph --
// each survey on its own branch.
mk_status launch_iteration(mk_plan_t p, bool timed, cudaStream_t main, bool branches) {
  for (size_t i = 0; i < p->s.size(); ++i) {
    Survey& sv = p->s[i];
    cudaStream_t st = main;
    if (branches) {
      st = p->side[i];
      MK_CUDA(p, cudaStreamWaitEvent(st, p->fork_ev, 0));
    }
    TimedPair* tp = timed ? next_pair(p, 0) : nullptr;
    if (tp) MK_CUDA(p, cudaEventRecord(tp->a, st));
    int nl = 0;
    mk_status cs = contract(p, sv, st, &nl);
    if (cs != MK_OK) return cs;
    if (tp) MK_CUDA(p, cudaEventRecord(tp->b, st));
    tp = timed ? next_pair(p, 1) : nullptr;
    if (tp) MK_CUDA(p, cudaEventRecord(tp->a, st));
    {
      // the iteration's epilogue adds S to the pmin spectrum where the survey keeps one
      mk::SurveyDev v = sv.dev;
      v.pacc = sv.pacc;
      MK_CUDA(p, mk::launch_epilogue(v, sv.energy, kMaxIterSlots, st, p->num_sms));
    }
    if (tp) MK_CUDA(p, cudaEventRecord(tp->b, st));
    if (branches) {
      MK_CUDA(p, cudaEventRecord(p->join_ev[i], st));
      MK_CUDA(p, cudaStreamWaitEvent(main, p->join_ev[i], 0));
    }
  }
  return MK_OK;
}

// Captures one iteration of all surveys into a graph (once per plan): the
// iteration index lives on the device, so every replay is identical.
mk_status build_graph(mk_plan_t p) {
  if (p->graph_exec) return MK_OK;
  if (!p->cap_stream) {
    MK_CUDA(p, cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    MK_CUDA(p, cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
    p->side.resize(p->s.size());
    p->join_ev.resize(p->s.size());
    for (size_t i = 0; i < p->s.size(); ++i) {
      MK_CUDA(p, cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking));
      MK_CUDA(p, cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming));
    }
  }
  MK_CUDA(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  mk_status st = MK_OK;
  cudaError_t e = cudaEventRecord(p->fork_ev, p->cap_stream);
  if (e == cudaSuccess) st = launch_iteration(p, false, p->cap_stream, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
  if (e != cudaSuccess || st != MK_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st != MK_OK) return st;
    return fail(p, MK_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&p->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->graph_exec = nullptr;
    return fail(p, MK_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  return MK_OK;
}

}  // namespace

extern "C" mk_status mk_iterate(mk_plan_t p, int32_t niter, double* energy) {
  if (!p) return fail(nullptr, MK_ERR_ARG, "null plan");
  p->err[0] = 0;
  mk_status st = ensure_device(p);
  if (st != MK_OK) return st;
  if (niter < 0) return fail(p, MK_ERR_ARG, "niter < 0");
  int Ftot = 0;
  for (size_t i = 0; i < p->s.size(); ++i) {
    if (!p->s[i].ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", (int)i);
    Ftot += p->s[i].dev.F;
  }
  bool streaming = false;
  for (auto& sv : p->s) streaming = streaming || sv.stream_r;
  const bool use_graph = p->graph && !p->timing && !streaming && niter > 0;
  if (use_graph && (st = build_graph(p)) != MK_OK) return st;
  for (int done = 0; done < niter;) {
    const int chunk = niter - done < kMaxIterSlots ? niter - done : kMaxIterSlots;
    std::vector<int> start(p->s.size());
    for (size_t i = 0; i < p->s.size(); ++i) start[i] = p->s[i].iter;
    for (int it = 0; it < chunk; ++it) {
      if (use_graph) {
        MK_CUDA(p, cudaGraphLaunch(p->graph_exec, p->stream));
      } else if ((st = launch_iteration(p, p->timing && (p->timing_count++ % (unsigned long long)p->timing_stride) == 0,
                                        p->stream, false)) != MK_OK) {
        return st;
      }
    }
    for (auto& sv : p->s) {
      p->stats.launches += 2 * chunk;
      p->stats.contract_launches += chunk;
      p->stats.epilogue_launches += chunk;
      sv.iter += chunk;
      sv.n_in_field = false;
      sv.derived_valid = sv.gm_valid = sv.gp_valid = false;
    }
    if (energy) {
      // iteration i of a survey left its energies in ring slot i % kMaxIterSlots
      int foff = 0;
      for (size_t i = 0; i < p->s.size(); ++i) {
        Survey& sv = p->s[i];
        const int s0 = start[i] % kMaxIterSlots;
        const int n1 = chunk < kMaxIterSlots - s0 ? chunk : kMaxIterSlots - s0;
        const size_t fb = (size_t)sv.dev.F * sizeof(double);
        MK_CUDA(p, cudaMemcpy2DAsync(energy + (size_t)done * Ftot + foff, (size_t)Ftot * sizeof(double),
                                     sv.energy + (size_t)s0 * sv.dev.F, fb, fb, n1, cudaMemcpyDeviceToHost, p->stream));
        if (n1 < chunk)
          MK_CUDA(p, cudaMemcpy2DAsync(energy + (size_t)(done + n1) * Ftot + foff, (size_t)Ftot * sizeof(double),
                                       sv.energy, fb, fb, chunk - n1, cudaMemcpyDeviceToHost, p->stream));
        foff += sv.dev.F;
      }
      MK_CUDA(p, cudaStreamSynchronize(p->stream));
      if ((st = check_device_errors(p)) != MK_OK) return st;
    }
    done += chunk;
  }
  return MK_OK;
}

extern "C" {

mk_status mk_fetch_fields(mk_plan_t p, int32_t survey, uint32_t mask, float* out, size_t out_bytes,
                          int32_t dst_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!out) return fail(p, MK_ERR_ARG, "null output pointer");
  if (mask == 0 || (mask & ~MK_F_ALL)) return fail(p, MK_ERR_ARG, "field mask 0x%x invalid", mask);
  if (!sv->ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", survey);
  const mk::SurveyDev& v = sv->dev;
  const size_t field = (size_t)v.F * v.ns * v.nt;
  const size_t need = (size_t)__builtin_popcount(mask) * field * sizeof(float);
  if (out_bytes < need) return fail(p, MK_ERR_ARG, "output of %zu bytes, %zu needed", out_bytes, need);
  if ((st = materialize(p, *sv, mask)) != MK_OK) return st;
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const float* src[8] = {v.fN, v.f1p, v.f1m, v.f2p, v.pmin, nullptr, v.gm, v.gp};
  float* o = out;
  for (int b = 0; b < 8; ++b) {
    if (!(mask & (1u << b))) continue;
    if (b == 5) {
      float* gdst = dst_on_device ? o : v.scratch;
      MK_CUDA(p, mk::launch_green(v, gdst, p->stream, p->num_sms));
      p->stats.launches++;
      p->stats.other_launches++;
      if (!dst_on_device)
        MK_CUDA(p, cudaMemcpyAsync(o, v.scratch, field * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    } else {
      MK_CUDA(p, cudaMemcpyAsync(o, src[b], field * sizeof(float), kind, p->stream));
    }
    o += field;
  }
  if (!dst_on_device) {
    MK_CUDA(p, cudaStreamSynchronize(p->stream));
    if ((st = check_device_errors(p)) != MK_OK) return st;
  }
  return MK_OK;
}

mk_status mk_set_fields(mk_plan_t p, int32_t survey, uint32_t mask, const float* in, size_t in_bytes,
                        int32_t iteration, int32_t src_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!in) return fail(p, MK_ERR_ARG, "null input pointer");
  const uint32_t state = MK_F_N | MK_F_F1P | MK_F_F1M;
  if ((mask & state) != state || (mask & ~(state | MK_F_F2P | MK_F_PMIN)))
    return fail(p, MK_ERR_ARG, "field mask 0x%x invalid: N, f1plus and f1min are required, G cannot be set", mask);
  if (iteration < 0) return fail(p, MK_ERR_ARG, "iteration < 0");
  if (!sv->ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", survey);
  if (is_shard(sv->d))
    return fail(p, MK_ERR_UNSUPPORTED, "survey %d is a shot-row shard: its pmin cannot be resumed from fields", survey);
  const mk::SurveyDev& v = sv->dev;
  const size_t field = (size_t)v.F * v.ns * v.nt;
  const size_t need = (size_t)__builtin_popcount(mask) * field * sizeof(float);
  if (in_bytes < need) return fail(p, MK_ERR_ARG, "input of %zu bytes, %zu needed", in_bytes, need);
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  float* dst[5] = {v.fN, v.f1p, v.f1m, nullptr, nullptr};  // f2p and pmin follow from these
  const float* q = in;
  for (int b = 0; b < 5; ++b) {
    if (!(mask & (1u << b))) continue;
    if (dst[b]) MK_CUDA(p, cudaMemcpyAsync(dst[b], q, field * sizeof(float), kind, p->stream));
    q += field;
  }
  MK_CUDA(p, mk::launch_spectrum(v, v.fN, p->stream, p->num_sms));
  MK_CUDA(p, mk::launch_set_iter(v, iteration, p->stream));
  p->stats.launches += 2;
  p->stats.other_launches += 2;
  if (!src_on_device) MK_CUDA(p, cudaStreamSynchronize(p->stream));
  sv->iter = iteration;
  sv->pacc_valid = false;  // pmin of resumed fields follows from the synthesis at fetch
  sv->n_in_field = true;
  sv->derived_valid = sv->gm_valid = sv->gp_valid = false;
  return MK_OK;
}

mk_status mk_image(mk_plan_t p, int32_t survey, double* image, int32_t dst_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!image) return fail(p, MK_ERR_ARG, "null output pointer");
  if (!sv->ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", survey);
  if ((st = materialize(p, *sv, MK_F_GMINUS)) != MK_OK) return st;
  const mk::SurveyDev& v = sv->dev;
  double* dst = image;
  if (!dst_on_device) dst = v.Epart;  // staging: the per-trace energy buffer holds >= F doubles
  MK_CUDA(p, mk::launch_image(v, v.gm, sv->d.dx * sv->d.dt, dst, p->stream));
  p->stats.launches++;
  p->stats.other_launches++;
  if (!dst_on_device) {
    MK_CUDA(p, cudaMemcpyAsync(image, dst, (size_t)v.F * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    MK_CUDA(p, cudaStreamSynchronize(p->stream));
    if ((st = check_device_errors(p)) != MK_OK) return st;
  }
  return MK_OK;
}

}  // extern "C"

namespace {

// Rows [r0, r0 + rc) of the field spectrum operand as a packed buffer: one
// strided 2-D copy per part.  Complex FP32 Nw [nw][F][r_pad]: rows of rc
// complex values; 16-bit embedding parts [nw][2F][2 r_pad]: rows of 2 rc
// 16-bit values.  Packed layout [part][nw][F or 2F][row values], part after
// part; bytes = parts * nw * F * rc * 8 in both cases.
mk_status field_spectrum_copy(mk_plan_t p, Survey& sv, void* packed, int r0, int rc, size_t bytes, int on_device,
                              bool out) {
  const mk::SurveyDev& v = sv.dev;
  const int parts = mk::field_in_nw(v) ? 1 : (v.rprec == MK_R_SPLIT3_BF16 ? 3 : 2);
  const size_t need = (size_t)parts * v.nw * v.F * rc * 8;
  if (bytes < need) return fail(p, MK_ERR_ARG, "field spectrum rows need %zu bytes, %zu given", need, bytes);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  char* pk = static_cast<char*>(packed);
  for (int q = 0; q < parts; ++q) {
    size_t pitch, width, height;
    char* op;
    if (mk::field_in_nw(v)) {
      pitch = (size_t)v.r_pad * sizeof(float2);
      width = (size_t)rc * sizeof(float2);
      height = (size_t)v.nw * v.F;
      op = reinterpret_cast<char*>(v.Nw) + (size_t)r0 * sizeof(float2);
    } else {
      void* part = q == 0 ? v.Bq0 : (q == 1 ? v.Bq1 : v.Bq2);
      pitch = (size_t)v.r_pad * 4;
      width = (size_t)rc * 4;
      height = (size_t)v.nw * 2 * v.F;
      op = static_cast<char*>(part) + (size_t)r0 * 4;
    }
    char* pq = pk + (size_t)q * width * height;
    if (out) {
      MK_CUDA(p, cudaMemcpy2DAsync(pq, width, op, pitch, width, height, kind, p->stream));
    } else {
      MK_CUDA(p, cudaMemcpy2DAsync(op, pitch, pq, width, width, height, kind, p->stream));
    }
  }
  if (!on_device) MK_CUDA(p, cudaStreamSynchronize(p->stream));
  return MK_OK;
}

}  // namespace

extern "C" {

mk_status mk_export_field_spectrum(mk_plan_t p, int32_t survey, void* dst, size_t bytes, int32_t dst_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!dst) return fail(p, MK_ERR_ARG, "null output pointer");
  if (!sv->ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", survey);
  return field_spectrum_copy(p, *sv, dst, sv->dev.row0, sv->dev.ns, bytes, dst_on_device, true);
}

mk_status mk_import_field_spectrum(mk_plan_t p, int32_t survey, const void* src, int32_t row_begin,
                                   int32_t row_count, size_t bytes, int32_t src_on_device) {
  Survey* sv = nullptr;
  mk_status st = get_survey(p, survey, &sv);
  if (st != MK_OK) return st;
  p->err[0] = 0;
  if ((st = ensure_device(p)) != MK_OK) return st;
  if (!src) return fail(p, MK_ERR_ARG, "null input pointer");
  if (!sv->ready) return fail(p, MK_ERR_STATE, "survey %d has no G_d (call mk_set_Gd_window)", survey);
  if (row_begin < 0 || row_count < 1 || row_begin + row_count > sv->dev.nr)
    return fail(p, MK_ERR_ARG, "rows [%d, %d) outside [0, %d)", row_begin, row_begin + row_count, sv->dev.nr);
  return field_spectrum_copy(p, *sv, const_cast<void*>(src), row_begin, row_count, bytes, src_on_device, false);
}

mk_status mk_set_timing(mk_plan_t p, int32_t stride, int32_t reserve_pairs) {
  if (!p) return fail(nullptr, MK_ERR_ARG, "null plan");
  p->err[0] = 0;
  if (stride < 1 || reserve_pairs < 0) return fail(p, MK_ERR_ARG, "stride must be >= 1 and reserve >= 0");
  if (!p->timing) return fail(p, MK_ERR_STATE, "the plan was made without MK_FLAG_TIMING");
  mk_status st = ensure_device(p);
  if (st != MK_OK) return st;
  p->timing_stride = stride;
  p->timing_count = 0;
  while (p->events.size() < p->next_event + (size_t)reserve_pairs) {
    TimedPair tp;
    MK_CUDA(p, cudaEventCreate(&tp.a));
    if (cudaEventCreate(&tp.b) != cudaSuccess) {
      cudaEventDestroy(tp.a);
      return fail(p, MK_ERR_CUDA, "cudaEventCreate failed");
    }
    tp.kind = 0;
    p->events.push_back(tp);
  }
  return MK_OK;
}

mk_status mk_get_stats(mk_plan_t p, mk_stats_t* out, int32_t reset) {
  if (!p || !out) return fail(p, MK_ERR_ARG, "null pointer");
  p->err[0] = 0;
  if (p->next_event) {
    MK_CUDA(p, cudaStreamSynchronize(p->stream));
    for (size_t i = 0; i < p->next_event; ++i) {
      float ms = 0.f;
      MK_CUDA(p, cudaEventElapsedTime(&ms, p->events[i].a, p->events[i].b));
      if (p->events[i].kind == 0) {
        p->stats.contract_ms += ms;
        p->stats.contract_timed++;
      } else {
        p->stats.epilogue_ms += ms;
        p->stats.epilogue_timed++;
      }
    }
    p->next_event = 0;
  }
  *out = p->stats;
  if (reset) p->stats = mk_stats_t{};
  return check_device_errors(p);
}

mk_status mk_destroy(mk_plan_t p) {
  if (!p) return MK_OK;
  cudaStreamSynchronize(p->stream);
  for (auto& tp : p->events) {
    cudaEventDestroy(tp.a);
    cudaEventDestroy(tp.b);
  }
  for (auto& sv : p->s) {
    mk::umma_destroy(sv.umma);
    if (sv.copy_stream) cudaStreamDestroy(sv.copy_stream);
    for (int b = 0; b < 2; ++b) {
      if (sv.ready_ev[b]) cudaEventDestroy(sv.ready_ev[b]);
      if (sv.free_ev[b]) cudaEventDestroy(sv.free_ev[b]);
    }
  }
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (auto st : p->side) cudaStreamDestroy(st);
  for (auto ev : p->join_ev) cudaEventDestroy(ev);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->err_host) cudaFreeHost(p->err_host);
  delete p;
  return MK_OK;
}

const char* mk_last_error(mk_plan_t p) { return p ? p->err : g_noplan_err; }

}  // extern "C"
