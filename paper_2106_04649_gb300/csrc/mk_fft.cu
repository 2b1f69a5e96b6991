// Per-trace transforms of the Neumann iteration, staged in shared memory.
//
//  * epilogue: inverse transform of the band-limited synthesis result
//    (Theory: "reverse Fourier transform"; Implementation: "padding"), time
//    reversal and sign flip, theta mute, accumulation of f1min / f1plus
//    (Algorithm 1), FP64 energy, and the forward transform of N_i
//    restricted to the band for the next contraction;
//  * init: N_{-1} = f1plus = G_d(-t), f1min = 0 and the band spectrum of
//    N_{-1} (Theory: initialisation);
//  * fetch-time fields: N_i = -theta s_i(-t) from the last synthesis result,
//    f2p = f1plus - f1min(-t), pmin = IDFT of a synthesis of f2p - N_last,
//    G(t) = f2p(-t) + pmin(t).
//
// Only f1plus / f1min are accumulated per iteration.  Algorithm 1 also
// accumulates f2p and pmin; both follow from the series exactly:
//    f2p = N_{-1} + sum_i N_i = f1plus - f1min(-t)   (odd N_i go to f1plus,
//          even N_i reversed and negated to f1min),
//    pmin = sum_{i<n} synthesis(N_{i-1}) = synthesis(f2p - N_{n-1})  (linearity),
// so they are formed when fetched, which removes two full-length
// read-modify-writes per trace and iteration from the hot loop.
//
// Two real traces share one complex transform (a + i b): the inverse
// transform of X + iY with Hermitian X, Y gives x + iy; the forward transform
// Z of a + ib gives A_m = (Z_m + conj Z_{-m})/2, B_m = (Z_m - conj Z_{-m})/(2i).
// The complex transform is a Stockham autosort FFT in shared memory with
// twiddles from an FP64 table rounded to FP32 (radix-8 passes,
// contiguous per-pass twiddle tables and a padded shared-memory index keep
// the accesses bank-conflict free).  The epilogue and the band kernel
// (initialisation, field spectra) take blocks of up to 8 consecutive traces:
// the blocks' band spectra pass through a trace-major shared stage, so that
// the loads from S and the stores to Nw or the 16-bit embedding are
// coalesced; the pairs of a block are transformed one after the other.
// Grids are sized to the SM count times the CTAs that fit per SM.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mk_embed.cuh"
#include "mk_internal.h"
#include "mk_rstore.cuh"

namespace mk {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward transform) or +i (inverse transform)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 v) {
  return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_mi<INV>(csub(v1, v3));
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  v1 = cadd(a1, a3);
  v3 = csub(a1, a3);
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int threads_for(int nt) { return nt / 8 < 32 ? 32 : (nt / 8 > 512 ? 512 : nt / 8); }

// Shared-memory index with one float2 of padding after every 16: the strided
// writes of the early passes then hit distinct banks per half-warp.
__device__ __forceinline__ int P(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded(int n) { return n + n / 16; }

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  // radix-2 split into even/odd outputs: a_n = v_n + v_{n+4} -> DFT4 gives
  // V_{2m}; b_n = (v_n - v_{n+4}) W8^{+-n} -> DFT4 gives V_{2m+1}
  const float c = 0.70710678118654752f;
  float2 a0 = cadd(v[0], v[4]), a1 = cadd(v[1], v[5]), a2 = cadd(v[2], v[6]), a3 = cadd(v[3], v[7]);
  float2 b0 = csub(v[0], v[4]), b1 = csub(v[1], v[5]), b2 = csub(v[2], v[6]), b3 = csub(v[3], v[7]);
  b1 = INV ? make_float2(c * (b1.x - b1.y), c * (b1.x + b1.y)) : make_float2(c * (b1.x + b1.y), c * (b1.y - b1.x));
  b2 = mul_mi<INV>(b2);
  b3 = INV ? make_float2(-c * (b3.x + b3.y), c * (b3.x - b3.y)) : make_float2(c * (b3.y - b3.x), -c * (b3.x + b3.y));
  dft4<INV>(a0, a1, a2, a3);
  dft4<INV>(b0, b1, b2, b3);
  v[0] = a0;
  v[2] = a1;
  v[4] = a2;
  v[6] = a3;
  v[1] = b0;
  v[3] = b1;
  v[5] = b2;
  v[7] = b3;
}

template <bool INV, int R>
__device__ __forceinline__ void dftR(float2 (&v)[R]) {
  if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
}

// One Stockham pass of radix R with current sub-length Ns: butterfly j
// (k = j mod Ns) reads x[j + r NT/R], multiplies by w^{r k NT/(Ns R)} =
// e^{-+2 pi i r k / (Ns R)}, does a length-R DFT and writes
// x[(j - k) R + k + r Ns].  The pass's twiddles are a contiguous table
// tw[toff + (r - 1) Ns + k] (consecutive k on consecutive lanes).  Reads and
// writes are separated by a barrier, so the pass works in place.
template <int NT, int THREADS, bool INV, int R>
__device__ __forceinline__ void stockham_pass(float2* x, const float2* tw, int Ns, int toff) {
  constexpr int NB = NT / R;
  constexpr int PB = (NB + THREADS - 1) / THREADS;
  float2 v[PB][R];
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int j = threadIdx.x + q * THREADS;
    if (j < NB) {
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = x[P(j + r * NB)];
      if (Ns > 1) {  // the first pass (Ns = 1) has unit twiddles
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[toff + (r - 1) * Ns + k];
          if (INV) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dftR<INV, R>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int j = threadIdx.x + q * THREADS;
    if (j < NB) {
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[P(base + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// The same pass out of place, with the sub-length NS known at compile
// time (index and twiddle offsets fold into constants): reads in, writes
// out, one barrier.  The pass before wrote in and read out before its own
// barrier, so nothing else orders the two.
template <int NT, int THREADS, bool INV, int R, int NS>
__device__ __forceinline__ void stockham_pass_pp(const float2* in, float2* out, const float2* tw) {
  constexpr int NB = NT / R;
  constexpr int PB = (NB + THREADS - 1) / THREADS;
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int j = threadIdx.x + q * THREADS;
    if (j < NB) {
      const int k = j & (NS - 1);
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in[P(j + r * NB)];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r - 1) * NS + k];
          if (INV) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dftR<INV, R>(v);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) out[P(base + r * NS)] = v[r];
    }
  }
  __syncthreads();
}

// Complex DFT of in[P(0 .. NT-1)] ping-ponging between in and out, one pass
// per level of the compile-time recursion (radix-8 passes, then one radix-2
// or radix-4 pass); returns the buffer that holds the result.  The twiddle
// table holds the passes' tables back to back.
template <int NT, int THREADS, bool INV, int PASS, int NS, int TOFF>
__device__ __forceinline__ float2* fft_pp_from(float2* in, float2* out, const float2* tw) {
  constexpr int LOG2 = ilog2(NT);
  constexpr int N8 = LOG2 / 3;
  constexpr int REM = LOG2 % 3;
  if constexpr (PASS < N8) {
    stockham_pass_pp<NT, THREADS, INV, 8, NS>(in, out, tw + TOFF);
    return fft_pp_from<NT, THREADS, INV, PASS + 1, NS * 8, TOFF + 7 * NS>(out, in, tw);
  } else if constexpr (REM == 1) {
    stockham_pass_pp<NT, THREADS, INV, 2, NS>(in, out, tw + TOFF);
    return out;
  } else if constexpr (REM == 2) {
    stockham_pass_pp<NT, THREADS, INV, 4, NS>(in, out, tw + TOFF);
    return out;
  } else {
    return in;
  }
}

template <int NT, int THREADS, bool INV>
__device__ __forceinline__ float2* fft_smem_pp(float2* a, float2* b, const float2* tw) {
  return fft_pp_from<NT, THREADS, INV, 0, 1, 0>(a, b, tw);
}

// In-place complex DFT of x[P(0 .. NT-1)] (unnormalised; sign -1 forward,
// +1 inverse): radix-8 passes, then one radix-2 or radix-4 pass when log2 NT
// is not a multiple of 3.  The twiddle table holds the passes' tables back to
// back (NT - 1 entries in all, see twiddle_kernel).
template <int NT, int THREADS, bool INV>
__device__ __forceinline__ void fft_smem(float2* x, const float2* tw) {
  constexpr int LOG2 = ilog2(NT);
  constexpr int N8 = LOG2 / 3;
  constexpr int REM = LOG2 % 3;
  int Ns = 1, toff = 0;
#pragma unroll 1
  for (int p = 0; p < N8; ++p) {
    stockham_pass<NT, THREADS, INV, 8>(x, tw, Ns, toff);
    toff += 7 * Ns;
    Ns *= 8;
  }
  if (REM == 1) stockham_pass<NT, THREADS, INV, 2>(x, tw, Ns, toff);
  if (REM == 2) stockham_pass<NT, THREADS, INV, 4>(x, tw, Ns, toff);
}

__device__ __forceinline__ int64_t field_offset(const SurveyDev& s, int t) { return (int64_t)t * s.nt; }

// Hermitian pack of the band spectra S[m][t0], S[m][t0 + 1] into
// x = X + iY (bins outside the band zero; DC and Nyquist real).  All global
// loads of a thread are issued before its shared-memory stores.
template <int NT, int THREADS>
__device__ __forceinline__ void pack_pair(const SurveyDev& s, float2* x, int t0, bool hasb) {
  constexpr int PM = (NT / 2 + THREADS) / THREADS;  // bins 0 .. NT/2 per thread
  float4 v[PM];
#pragma unroll
  for (int q = 0; q < PM; ++q) {
    const int m = threadIdx.x + q * THREADS;
    v[q] = (m <= NT / 2 && m < s.nw)
               ? __ldg(reinterpret_cast<const float4*>(s.S + (int64_t)m * s.s_stride + t0))
               : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < PM; ++q) {
    const int m = threadIdx.x + q * THREADS;
    if (m > NT / 2) continue;
    float2 X = make_float2(v[q].x, v[q].y);
    float2 Y = hasb ? make_float2(v[q].z, v[q].w) : make_float2(0.f, 0.f);
    if (m == 0 || m == NT / 2) {
      X.y = 0.f;
      Y.y = 0.f;
    }
    x[P(m)] = make_float2(X.x - Y.y, X.y + Y.x);
    if (m > 0 && m < NT / 2) x[P(NT - m)] = make_float2(X.x + Y.y, Y.x - X.y);
  }
}

// ---------------------------------------------------------------------------
// Epilogue, blocked: a CTA takes a block of up to 2G consecutive traces
// (G pairs).  Their band spectra are loaded from S into a trace-major
// shared stage with one coalesced pass (consecutive threads read consecutive
// traces of one frequency), the pairs are transformed one after the other,
// each writing its new band spectra back into its own stage rows, and one
// coalesced pass writes the block to Nw or to the 16-bit embedding.  The
// stage's leading dimension ld is odd, so both the per-frequency and the
// per-trace accesses of the stage are free of bank conflicts.

__host__ __device__ __forceinline__ int stage_ld(int nw) { return nw | 1; }

// Resident epilogue CTAs per SM the launch is built for (registers and
// shared memory are sized to fit that many, the grid holds that many per SM):
// 16 warps per SM at every length; 256 threads per CTA from nt = 2048 up.
__host__ __device__ constexpr int epi_ctas(int nt) { return nt <= 512 ? 8 : (nt <= 1024 ? 4 : (nt <= 4096 ? 2 : 1)); }
__host__ __device__ constexpr int epi_threads(int nt) { return nt == 4096 ? 256 : threads_for(nt); }
__host__ __device__ constexpr size_t epi_smem_target(int nt) {
  return (size_t)227 * 1024 / epi_ctas(nt) - 2 * 1024;
}

// The f1 window samples of a pair are prefetched into shared memory (2 NT
// floats) up to NT = 4096; above that the shared memory is needed elsewhere.
__host__ __device__ constexpr bool epi_prefetch(int nt) { return nt <= 2048; }
// Up to NT = 4096 the transforms ping-pong between two buffers (one barrier
// per pass instead of two).
__host__ __device__ constexpr bool epi_pingpong(int nt) { return nt <= 2048; }
__host__ __device__ constexpr size_t epi_base_bytes(int nt) {
  return ((epi_pingpong(nt) ? 2 : 1) * (size_t)padded(nt) + nt) * sizeof(float2) +
         (epi_prefetch(nt) ? 2 * (size_t)nt * sizeof(float) : 0);
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Dynamic shared memory the epilogue may use (below the 227 KB per-CTA limit,
// leaving room for its static shared memory).
constexpr int kEpiSmemMax = 220 * 1024;

// Hermitian pack of stage rows (a, b) into x (bins outside the band zero).
template <int NT, int THREADS>
__device__ __forceinline__ void pack_stage(const SurveyDev& s, float2* x, const float2* ra, const float2* rb,
                                           bool hasb) {
  for (int m = threadIdx.x; m <= NT / 2; m += THREADS) {
    float2 X = make_float2(0.f, 0.f), Y = make_float2(0.f, 0.f);
    if (m < s.nw) {
      X = ra[m];
      if (hasb) Y = rb[m];
    }
    if (m == 0 || m == NT / 2) {
      X.y = 0.f;
      Y.y = 0.f;
    }
    x[P(m)] = make_float2(X.x - Y.y, X.y + Y.x);
    if (m > 0 && m < NT / 2) x[P(NT - m)] = make_float2(X.x + Y.y, Y.x - X.y);
  }
}

// Band spectra of the transformed pair z (a + i b) into stage rows.
template <int NT, int THREADS>
__device__ __forceinline__ void unpack_band_stage(const SurveyDev& s, const float2* z, float2* ra, float2* rb,
                                                  bool hasb) {
  for (int m = threadIdx.x; m < s.nw; m += THREADS) {
    const float2 zm = z[P(m)];
    const float2 zc = cconj(z[P((NT - m) & (NT - 1))]);
    ra[m] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y + zc.y));
    if (hasb) rb[m] = make_float2(0.5f * (zm.y - zc.y), -0.5f * (zm.x - zc.x));
  }
}

// A block's band spectra from the trace-major stage (row c of trace tb + c)
// to Nw, to the 16-bit field embedding, or (rprec >= 8, loading R from its
// time traces) to the R layout, in one coalesced pass: thread column cc, bins
// mc, mc + mstep, ...
__device__ __forceinline__ void stage_store(const SurveyDev& s, const float2* stage, int ld, int tb, int ntr, int cc,
                                            int mc, int mstep) {
  if (cc >= ntr) return;
  const int t = tb + cc;
  const int f = t / s.ns, k = t - f * s.ns + s.row0;  // k on the field spectrum's r axis
  const float2* row = stage + cc * ld;
  if (field_in_nw(s)) {
    float2* dst = s.Nw + (int64_t)f * s.r_pad + k;
    for (int m = mc; m < s.nw; m += mstep) dst[(int64_t)m * s.nw_stride] = row[m];
  } else if (s.rprec >= 8) {
    const int64_t base = (int64_t)f * s.r_pad + k;
    for (int m = mc; m < s.nw; m += mstep) store_r16(s, s.rprec - 8, (int64_t)m * s.nw_stride + base, row[m]);
  } else if (s.rprec == 2) {
    for (int m = mc; m < s.nw; m += mstep) store_embedding<false>(s, m, f, k, row[m].x, row[m].y);
  } else {
    for (int m = mc; m < s.nw; m += mstep) store_embedding<true>(s, m, f, k, row[m].x, row[m].y);
  }
}

template <int NT>
__global__ void __launch_bounds__(epi_threads(NT), epi_ctas(NT))
epilogue_kernel(SurveyDev s, double* __restrict__ ring, int slots, int G) {
  constexpr int THREADS = epi_threads(NT);
  extern __shared__ float4 smem_raw[];
  constexpr bool kPingPong = epi_pingpong(NT);
  float2* x = reinterpret_cast<float2*>(smem_raw);  // the pair: s, then N_i, then its transform
  float2* y = x + (kPingPong ? padded(NT) : 0);     // second buffer of the ping-pong transforms
  float2* tw = y + padded(NT);
  float2* stage = tw + NT;                          // [2G][ld] band spectra of the block
  const int ld = stage_ld(s.nw);
  constexpr bool kPrefetch = epi_prefetch(NT);
  float* hbuf = reinterpret_cast<float*>(stage + 2 * G * ld);  // [2][NT] f1 window samples (2G ld is even: 16-byte aligned)
  constexpr int kWarps = THREADS / 32;
  __shared__ double ered[8 * kWarps];  // per-warp energy sums of the block's traces (at most 8)
  __shared__ int sL[8];                // window half-lengths of the block's traces
  __shared__ int s_last;

  // a kernel launched as a programmatic dependent of this one (the next
  // contraction) may be scheduled now; it waits for this grid to complete
  // before it reads what this grid writes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // the twiddle table arrives asynchronously while the first block's spectra
  // load; the wait sits before the block's first barrier
  for (int i = 2 * threadIdx.x; i < NT; i += 2 * THREADS)
    cp_async16(reinterpret_cast<float*>(tw + i), reinterpret_cast<const float*>(s.tw + i));
  cp_async_commit();

  // the iteration index lives on the device (the last CTA advances it), so
  // every iteration launches with identical arguments (graph replay)
  const int iter = *s.iter;
  const int odd = iter & 1;
  double* energy_slot = ring + (int64_t)(iter % slots) * s.F;
  const int bt = 2 * G;  // traces per block (2, 4 or 8)
  const int nblocks = (s.ncols + bt - 1) / bt;
  const int cc = threadIdx.x & (bt - 1);                 // this thread's trace column
  const int mc = threadIdx.x / bt, mstep = THREADS / bt;  // and its bins mc, mc + mstep, ...
  const float inv = s.inv_nt;
  float* __restrict__ f1 = odd ? s.f1p : s.f1m;
  for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const int tb = blk * bt;
    const int ntr = s.ncols - tb < bt ? s.ncols - tb : bt;
    // 1. the block's band spectra, one coalesced pass (bt is a power of two
    //    dividing THREADS, so each thread keeps one trace column c)
    if (cc < ntr) {
      // eight predicated loads in flight per thread, then the stage stores;
      // with a pmin band spectrum kept, pmin += S as fire-and-forget
      // reductions (one per (m, t) and launch, so the sum is the same in
      // any schedule)
      const float2* src = s.S + tb + cc;
      float2* dst = stage + cc * ld;
      float2* acc = s.pacc ? s.pacc + tb + cc : nullptr;
      for (int m0 = mc; m0 < s.nw; m0 += 8 * mstep) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int m = m0 + u * mstep;
          if (m < s.nw) v[u] = __ldg(src + (int64_t)m * s.s_stride);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int m = m0 + u * mstep;
          if (m < s.nw) {
            dst[m] = v[u];
            if (acc) atomicAdd(acc + (int64_t)m * s.s_stride, v[u]);
          }
        }
      }
    }
    if (threadIdx.x < ntr) sL[threadIdx.x] = s.L[tb + threadIdx.x];  // the block's window lengths
    cp_async_wait_all();  // the twiddle table (first block)
    __syncthreads();
    for (int q = 0; 2 * q < ntr; ++q) {
      const int t0 = tb + 2 * q;
      const bool hasb = 2 * q + 1 < ntr;
      float2* ra = stage + (2 * q) * ld;
      float2* rb = ra + ld;
      const int La = sL[2 * q];
      const int Lb = hasb ? sL[2 * q + 1] : 0;
      const int64_t ba = field_offset(s, t0);
      const int64_t bb = hasb ? field_offset(s, t0 + 1) : 0;
      if constexpr (kPrefetch) {
        // the window samples of f1 for this pair, copied asynchronously into
        // shared memory while the inverse transform runs (16-byte chunks
        // that touch the window |j| < L)
        for (int c4 = threadIdx.x; c4 < NT / 2; c4 += THREADS) {
          const int tr = c4 >= NT / 4;
          const int j = 4 * (c4 - tr * (NT / 4));
          const int L = tr ? Lb : La;
          if (j < L || NT - (j + 3) < L) cp_async16(hbuf + tr * NT + j, f1 + (tr ? bb : ba) + j);
        }
        cp_async_commit();
      }
      // 2. Hermitian pack (bins outside the band are zero), inverse transform
      pack_stage<NT, THREADS>(s, x, ra, rb, hasb);
      __syncthreads();
      float2* z = x;
      if constexpr (kPingPong) {
        z = fft_smem_pp<NT, THREADS, true>(x, y, tw);
      } else {
        fft_smem<NT, THREADS, true>(x, tw);
      }
      // 3. reverse, negate, mute; accumulate f1 (window samples only).  A
      //    thread takes the mirror positions j and NT - j together (both have
      //    |signed index| j and each one's N_i comes from the other's s), so
      //    N_i overwrites s in place.
      double ea = 0.0, eb = 0.0;
      if constexpr (kPrefetch) {
        cp_async_wait_all();
        __syncthreads();
      }
      constexpr int PH = (NT / 2 + THREADS) / THREADS;  // mirror pairs j = 0 .. NT/2 per thread
#pragma unroll
      for (int k = 0; k < PH; ++k) {
        const int j = threadIdx.x + k * THREADS;
        if (j > NT / 2) continue;
        const int jr = (NT - j) & (NT - 1);
        const float2 zj = z[P(j)];
        const float2 zr = z[P(jr)];
        const bool ina = j < La, inb = j < Lb;
        float haj = 0.f, har = 0.f, hbj = 0.f, hbr = 0.f;
        if constexpr (kPrefetch) {
          if (ina) {
            haj = hbuf[j];
            har = hbuf[jr];
          }
          if (inb) {
            hbj = hbuf[NT + j];
            hbr = hbuf[NT + jr];
          }
        } else {
          if (ina) {
            haj = f1[ba + j];
            har = f1[ba + jr];
          }
          if (inb) {
            hbj = f1[bb + j];
            hbr = f1[bb + jr];
          }
        }
        // N_i(j) = -theta s(-j) = -s(jr), N_i(jr) = -s(j) inside the window
        const float naj = ina ? -(zr.x * inv) : 0.f, nar = ina ? -(zj.x * inv) : 0.f;
        const float nbj = inb ? -(zr.y * inv) : 0.f, nbr = inb ? -(zj.y * inv) : 0.f;
        z[P(j)] = make_float2(naj, nbj);
        if (jr != j) z[P(jr)] = make_float2(nar, nbr);
        // odd: f1plus += N_i; even: f1min -= N_i(-t) = theta s(t)
        if (ina) {
          f1[ba + j] = haj + (odd ? naj : -nar);
          ea += (double)naj * (double)naj;
          if (jr != j) {
            f1[ba + jr] = har + (odd ? nar : -naj);
            ea += (double)nar * (double)nar;
          }
        }
        if (inb) {
          f1[bb + j] = hbj + (odd ? nbj : -nbr);
          eb += (double)nbj * (double)nbj;
          if (jr != j) {
            f1[bb + jr] = hbr + (odd ? nbr : -nbj);
            eb += (double)nbr * (double)nbr;
          }
        }
      }
      __syncthreads();
      // 4. forward transform of N_i, band spectra into the stage rows of this pair
      float2* w = z;
      if constexpr (kPingPong) {
        w = fft_smem_pp<NT, THREADS, false>(z, z == x ? y : x, tw);
      } else {
        fft_smem<NT, THREADS, false>(z, tw);
      }
      unpack_band_stage<NT, THREADS>(s, w, ra, rb, hasb);
      // 5. per-trace energies: warp sums here (fixed shuffle tree), the sum
      //    over warps in warp order once the block is done
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ea += __shfl_down_sync(0xffffffffu, ea, o);
        eb += __shfl_down_sync(0xffffffffu, eb, o);
      }
      if ((threadIdx.x & 31) == 0) {
        ered[(2 * q) * kWarps + (threadIdx.x >> 5)] = ea;
        ered[(2 * q + 1) * kWarps + (threadIdx.x >> 5)] = eb;
      }
      __syncthreads();
    }
    if (threadIdx.x < ntr) {
      double e = 0.0;
      for (int w = 0; w < kWarps; ++w) e += ered[threadIdx.x * kWarps + w];
      s.Epart[tb + threadIdx.x] = e;
    }
    // 6. the block's new band spectra, one coalesced pass
    stage_store(s, stage, ld, tb, ntr, cc, mc, mstep);
    __syncthreads();
  }

  // The last CTA to finish sums the per-trace energies per focal point, one
  // warp per focal point: lane l adds k = l, l + 32, ... in ascending order,
  // then a fixed shuffle tree; the order never depends on scheduling.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(s.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int f = wid; f < s.F; f += THREADS / 32) {
      const double* e = s.Epart + (int64_t)f * s.ns;
      double acc = 0.0;
      for (int k = lane; k < s.ns; k += 32) acc += __ldcg(e + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) energy_slot[f] = acc;
    }
    if (threadIdx.x == 0) {
      *s.counter = 0u;
      *s.iter = iter + 1;
    }
  }
}

// Band spectra of a field, in blocks of 2G consecutive traces: per pair a
// forward transform in shared memory, the band into the block's stage, then
// one coalesced pass out (stage_store).  MODE 0: the spectrum of a field
// src [F][ns][nt] (Nw or its embedding; R when loading R from time traces).
// MODE 1: the initialisation N_{-1} = f1plus = G_d(-t), f1min = 0 from
// src = G_d, and the spectrum of N_{-1}.
template <int NT, int MODE>
__global__ void __launch_bounds__(threads_for(NT))
band_kernel(SurveyDev s, const float* __restrict__ src, int G) {
  constexpr int THREADS = threads_for(NT);
  constexpr int PJ = NT / THREADS;
  extern __shared__ float4 smem_raw[];
  float2* x = reinterpret_cast<float2*>(smem_raw);
  float2* tw = x + padded(NT);
  float2* stage = tw + NT;  // [2G][ld]
  const int ld = stage_ld(s.nw);
  for (int i = threadIdx.x; i < NT; i += THREADS) tw[i] = s.tw[i];
  __syncthreads();
  const int bt = 2 * G;
  const int nblocks = (s.ncols + bt - 1) / bt;
  const int cc = threadIdx.x & (bt - 1);
  const int mc = threadIdx.x / bt, mstep = THREADS / bt;
  for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const int tb = blk * bt;
    const int ntr = s.ncols - tb < bt ? s.ncols - tb : bt;
    for (int q = 0; 2 * q < ntr; ++q) {
      const int t0 = tb + 2 * q;
      const bool hasb = 2 * q + 1 < ntr;
      const int64_t ba = field_offset(s, t0);
      const int64_t bb = hasb ? field_offset(s, t0 + 1) : 0;
      if constexpr (MODE == 1) {
#pragma unroll
        for (int u = 0; u < PJ; ++u) {
          const int j = threadIdx.x + u * THREADS;
          const int jr = (NT - j) & (NT - 1);
          const float na = src[ba + jr];  // G_d has the field layout [F][nrec][nt]
          const float nb = hasb ? src[bb + jr] : 0.f;
          x[P(j)] = make_float2(na, nb);
          s.fN[ba + j] = na;
          s.f1p[ba + j] = na;
          s.f1m[ba + j] = 0.f;
          if (hasb) {
            s.fN[bb + j] = nb;
            s.f1p[bb + j] = nb;
            s.f1m[bb + j] = 0.f;
          }
        }
      } else {
        for (int j = threadIdx.x; j < NT; j += THREADS)
          x[P(j)] = make_float2(src[ba + j], hasb ? src[bb + j] : 0.f);
      }
      __syncthreads();
      fft_smem<NT, THREADS, false>(x, tw);
      unpack_band_stage<NT, THREADS>(s, x, stage + (2 * q) * ld, stage + (2 * q + 1) * ld, hasb);
      __syncthreads();
    }
    stage_store(s, stage, ld, tb, ntr, cc, mc, mstep);
    __syncthreads();
  }
}

// theta window half-length per trace: the number of n >= 0 with
// n * dt < t_d - eps, evaluated in FP64 exactly as written (IEEE products and
// differences, so every device and the host take the same decisions), capped
// at nt/2 + 1 (everything kept).  Non-finite t_d gives an empty window.
__global__ void window_kernel(SurveyDev s, const double* __restrict__ td, double eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.ncols) return;
  const double T = td[t] - eps;  // t = f * ns + k, the layout of t_d [F][ns]
  int L = 0;
  if (T > 0.0 && isfinite(T)) {
    const double q = ceil(T / s.dt);
    long long Lq = q > (double)s.nt ? (long long)s.nt : (long long)q;
    if (Lq < 0) Lq = 0;
    while (Lq > 0 && (double)(Lq - 1) * s.dt >= T) --Lq;
    while (Lq <= s.nt / 2 && (double)Lq * s.dt < T) ++Lq;
    L = (int)(Lq > s.nt / 2 + 1 ? s.nt / 2 + 1 : Lq);
  }
  s.L[t] = L;
}

// Inverse transform of the band spectra in S, per trace:
//   mode 0: dst = N = -theta s(-t) (the N_i of the last synthesis),
//   mode 1: dst = s (a plain synthesis result, e.g. pmin).
template <int NT>
__global__ void __launch_bounds__(threads_for(NT))
inverse_kernel(SurveyDev s, float* __restrict__ dst, int mode) {
  constexpr int THREADS = threads_for(NT);
  extern __shared__ float4 smem_raw[];
  float2* x = reinterpret_cast<float2*>(smem_raw);
  float2* tw = x + padded(NT);
  for (int i = threadIdx.x; i < NT; i += THREADS) tw[i] = s.tw[i];
  __syncthreads();
  const int npairs = (s.ncols + 1) / 2;
  for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
    const int t0 = 2 * p;
    const bool hasb = t0 + 1 < s.ncols;
    pack_pair<NT, THREADS>(s, x, t0, hasb);
    __syncthreads();
    fft_smem<NT, THREADS, true>(x, tw);
    const int La = s.L[t0];
    const int Lb = hasb ? s.L[t0 + 1] : 0;
    const int64_t ba = field_offset(s, t0);
    const int64_t bb = hasb ? field_offset(s, t0 + 1) : 0;
    for (int j = threadIdx.x; j < NT; j += THREADS) {
      float va, vb;
      if (mode == 0) {
        const int d = j < NT - j ? j : NT - j;
        const float2 zr = x[P((NT - j) & (NT - 1))];
        va = d < La ? -(zr.x * s.inv_nt) : 0.f;
        vb = d < Lb ? -(zr.y * s.inv_nt) : 0.f;
      } else {
        const float2 z = x[P(j)];
        va = z.x * s.inv_nt;
        vb = z.y * s.inv_nt;
      }
      dst[ba + j] = va;
      if (hasb) dst[bb + j] = vb;
    }
    __syncthreads();
  }
}

// f2p = f1plus - f1min(-t); diff = f2p - N (input of the pmin synthesis).
__global__ void f2p_kernel(SurveyDev s, float* __restrict__ diff) {
  const int64_t total = (int64_t)s.F * s.ns * s.nt;
  const int mask = s.nt - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & mask);
    const int64_t base = i - j;
    const float v = s.f1p[i] - s.f1m[base + ((s.nt - j) & mask)];
    s.f2p[i] = v;
    diff[i] = v - s.fN[i];
  }
}

// out = alpha * A(+-t) + beta * B(+-t) per trace (revA / revB: read at -t).
__global__ void lincomb_kernel(SurveyDev s, float* __restrict__ out, const float* __restrict__ A, int revA,
                               float alpha, const float* __restrict__ B, int revB, float beta) {
  const int64_t total = (int64_t)s.F * s.ns * s.nt;
  const int mask = s.nt - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & mask);
    const int64_t base = i - j;
    const int jr = (s.nt - j) & mask;
    float v = alpha * A[revA ? base + jr : i];
    if (B) v += beta * B[revB ? base + jr : i];
    out[i] = v;
  }
}

// Double-focusing image per focal point: zero-time sample of the time
// convolution of G^- with f1plus, integrated over positions,
// image(f) = dx dt sum_k sum_j G^-(f, k, j) f1plus(f, k, -j); FP64
// accumulation in a fixed order (one CTA per focal point).
__global__ void image_kernel(SurveyDev s, const float* __restrict__ gm, double scale, double* __restrict__ out) {
  const int f = blockIdx.x;
  const int64_t n = (int64_t)s.ns * s.nt;
  const int mask = s.nt - 1;
  const float* g = gm + (int64_t)f * n;
  const float* p = s.f1p + (int64_t)f * n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int j = (int)(i & mask);
    acc += (double)g[i] * (double)p[i - j + ((s.nt - j) & mask)];
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[f] = scale * t;
  }
}

__global__ void green_kernel(SurveyDev s, float* __restrict__ out) {
  const int64_t total = (int64_t)s.F * s.ns * s.nt;
  const int mask = s.nt - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & mask);
    const int64_t base = i - j;
    out[i] = s.f2p[base + ((s.nt - j) & mask)] + s.pmin[i];
  }
}

template <int NT>
cudaError_t set_attrs() {
  constexpr int one = (padded(NT) + NT) * (int)sizeof(float2);
  // the epilogue's stage grows with the band: allow the per-CTA maximum
  cudaError_t e = cudaFuncSetAttribute(epilogue_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEpiSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(band_kernel<NT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEpiSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(band_kernel<NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEpiSmemMax);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(inverse_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, one);
}

template <int NT>
cudaError_t launch_inv_nt(const SurveyDev& s, float* dst, int mode, cudaStream_t st, int num_sms) {
  const int npairs = (s.ncols + 1) / 2;
  int grid = num_sms * 4;
  if (grid > npairs) grid = npairs;
  inverse_kernel<NT><<<grid, threads_for(NT), (padded(NT) + NT) * sizeof(float2), st>>>(s, dst, mode);
  return cudaGetLastError();
}

// Blocks of the band kernels: up to 4 pairs while two CTAs fit per SM, fewer
// when there are few traces, so that every SM gets work.
template <int NT, int MODE>
cudaError_t launch_band_nt(const SurveyDev& s, const float* src, cudaStream_t st, int num_sms) {
  const size_t base = ((size_t)padded(NT) + NT) * sizeof(float2);
  const size_t row = (size_t)stage_ld(s.nw) * sizeof(float2);
  int G = 4;
  while (G > 1 && (base + 2 * G * row > 113 * 1024 || (s.ncols + 2 * G - 1) / (2 * G) < 2 * num_sms)) G /= 2;
  const size_t bytes = base + 2 * (size_t)G * row;
  const int nblocks = (s.ncols + 2 * G - 1) / (2 * G);
  int grid = num_sms * 2;
  if (grid > nblocks) grid = nblocks;
  band_kernel<NT, MODE><<<grid, threads_for(NT), bytes, st>>>(s, src, G);
  return cudaGetLastError();
}

// Pairs per epilogue block: as many as keep epi_ctas CTAs per SM within
// shared memory: 4, 2 or 1.
template <int NT>
int epi_pairs(int nw, size_t* bytes) {
  const size_t base = epi_base_bytes(NT);
  const size_t ld = (size_t)(nw | 1);
  int G = 4;  // a power of two: blocks of 2, 4 or 8 traces
  while (G > 1 && base + 2 * G * ld * sizeof(float2) > epi_smem_target(NT)) G /= 2;
  *bytes = base + 2 * G * ld * sizeof(float2);
  return G;
}

template <int NT>
cudaError_t launch_epi_nt(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms) {
  size_t bytes = 0;
  int G = epi_pairs<NT>(s.nw, &bytes);
  if (s.epi_g > 0) {
    while (G > s.epi_g) G /= 2;  // a tuned choice, never above the shared-memory fit
  } else {
    // few traces: smaller blocks so that every SM gets work
    while (G > 1 && (s.ncols + 2 * G - 1) / (2 * G) < epi_ctas(NT) * num_sms) G /= 2;
  }
  bytes = epi_base_bytes(NT) + 2 * (size_t)G * (size_t)(s.nw | 1) * sizeof(float2);
  const int nblocks = (s.ncols + 2 * G - 1) / (2 * G);
  int grid = num_sms * epi_ctas(NT);
  if (grid > nblocks) grid = nblocks;
  epilogue_kernel<NT><<<grid, epi_threads(NT), bytes, st>>>(s, ring, slots, G);
  return cudaGetLastError();
}



}  // namespace

#define MK_NT_SWITCH(nt, CALL)          \
  switch (nt) {                         \
    case 32: return CALL(32);           \
    case 64: return CALL(64);           \
    case 128: return CALL(128);         \
    case 256: return CALL(256);         \
    case 512: return CALL(512);         \
    case 1024: return CALL(1024);       \
    case 2048: return CALL(2048);       \
    case 4096: return CALL(4096);       \
    case 8192: return CALL(8192);       \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t prepare_kernels() {
  cudaError_t e = prepare_contract();
  if (e != cudaSuccess) return e;
  if ((e = prepare_load()) != cudaSuccess) return e;
  if ((e = prepare_epilogue_warp()) != cudaSuccess) return e;
#define MK_ATTR(N) \
  if ((e = set_attrs<N>()) != cudaSuccess) return e;
  MK_ATTR(32) MK_ATTR(64) MK_ATTR(128) MK_ATTR(256) MK_ATTR(512) MK_ATTR(1024) MK_ATTR(2048)
  MK_ATTR(4096) MK_ATTR(8192)
#undef MK_ATTR
  return cudaSuccess;
}

int epilogue_max_pairs(const SurveyDev& s, int num_sms) {
  if (epilogue_uses_warp(s, num_sms)) return 2;  // one or two rounds of traces per block
  const int nt = s.nt, nw = s.nw;
  size_t bytes = 0;
  switch (nt) {
#define MK_FIT(N) \
  case N: return epi_pairs<N>(nw, &bytes);
    MK_FIT(32) MK_FIT(64) MK_FIT(128) MK_FIT(256) MK_FIT(512) MK_FIT(1024) MK_FIT(2048) MK_FIT(4096) MK_FIT(8192)
#undef MK_FIT
    default: return 1;
  }
}

bool epilogue_fits(int nt, int nw) {
  size_t bytes = 0;
  switch (nt) {
#define MK_FIT(N) \
  case N: epi_pairs<N>(nw, &bytes); break;
    MK_FIT(32) MK_FIT(64) MK_FIT(128) MK_FIT(256) MK_FIT(512) MK_FIT(1024) MK_FIT(2048) MK_FIT(4096) MK_FIT(8192)
#undef MK_FIT
    default: return false;
  }
  return bytes <= (size_t)kEpiSmemMax;
}

// FFT twiddles in the pass-by-pass layout the shared-memory FFT reads
// (radix-8 passes, then one radix-2 or radix-4 pass when log2 nt is not a
// multiple of 3): pass (R, Ns) at offset toff stores e^{-2 pi i r k / (Ns R)}
// at toff + (r - 1) Ns + k, r = 1 .. R-1, k < Ns; nt - 1 entries, the last slot
// zero.  Each value is formed in FP64 (sincospi of the exact rational angle)
// and rounded to FP32.
__global__ void twiddle_kernel(float2* tw, int nt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  int lg = 0;
  while ((1 << lg) < nt) ++lg;
  int Ns = 1, toff = 0;
  for (int p = 0; p < lg / 3 + (lg % 3 ? 1 : 0); ++p) {
    const int R = p < lg / 3 ? 8 : (lg % 3 == 1 ? 2 : 4);
    if (e < toff + (R - 1) * Ns) {
      const int r = (e - toff) / Ns + 1, k = (e - toff) % Ns;
      const long long q = (long long)r * k * (nt / (Ns * R));  // angle in units of 2 pi / nt
      double sv, cv;
      sincospi(-2.0 * (double)q / (double)nt, &sv, &cv);
      tw[e] = make_float2((float)cv, (float)sv);
      return;
    }
    toff += (R - 1) * Ns;
    Ns *= R;
  }
  tw[e] = make_float2(0.f, 0.f);
}

// e^{-2 pi i j / nt} for j < nt, formed in FP64 and rounded to FP32.
__global__ void twiddle_linear_kernel(float2* tw, int nt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  double sv, cv;
  sincospi(-2.0 * (double)j / (double)nt, &sv, &cv);
  tw[j] = make_float2((float)cv, (float)sv);
}

cudaError_t launch_twiddles_linear(float2* tw, int nt, cudaStream_t st) {
  twiddle_linear_kernel<<<(nt + 255) / 256, 256, 0, st>>>(tw, nt);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(float2* tw, int nt, cudaStream_t st) {
  twiddle_kernel<<<(nt + 255) / 256, 256, 0, st>>>(tw, nt);
  return cudaGetLastError();
}

__global__ void set_iter_kernel(int* it, int v) { *it = v; }

cudaError_t launch_set_iter(const SurveyDev& s, int value, cudaStream_t st) {
  set_iter_kernel<<<1, 1, 0, st>>>(s.iter, value);
  return cudaGetLastError();
}

// The register epilogue needs enough traces to give every CTA slot a block
// (one block of up to 8 traces per CTA, two CTAs per SM); with fewer each warp
// holds a single trace and the shared-memory epilogue, whose 256 threads share
// a pair of traces, finishes sooner.
// At nt = 4096 a register-epilogue block holds 4 traces (shared memory), so
// the 16-bit embedding's row segments are 16-byte halves of 32-byte sectors;
// there the shared-memory epilogue, whose blocks hold 8 traces, is faster
// (4001 positions, 128 focal points, 3-way split: 25.6 vs 30.7 ms per
// launch), while for the complex FP32 spectrum the register form wins
// (15.6 vs 10.8 ms).
bool epilogue_uses_warp(const SurveyDev& s, int num_sms) {
  if (s.nt == 4096 && !field_in_nw(s)) return false;
  return s.ncols >= 16 * num_sms && epilogue_warp_supports(s.nt, s.nw);
}

cudaError_t launch_epilogue(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms) {
  if (epilogue_uses_warp(s, num_sms)) return launch_epilogue_warp(s, ring, slots, st, num_sms);
#define MK_CALL(N) launch_epi_nt<N>(s, ring, slots, st, num_sms)
  MK_NT_SWITCH(s.nt, MK_CALL)
#undef MK_CALL
}

cudaError_t launch_init(const SurveyDev& s, const float* Gd, cudaStream_t st, int num_sms) {
#define MK_CALL(N) launch_band_nt<N, 1>(s, Gd, st, num_sms)
  MK_NT_SWITCH(s.nt, MK_CALL)
#undef MK_CALL
}

cudaError_t launch_windows(const SurveyDev& s, const double* td, double eps, cudaStream_t st) {
  window_kernel<<<(s.ncols + 255) / 256, 256, 0, st>>>(s, td, eps);
  return cudaGetLastError();
}

cudaError_t launch_spectrum(const SurveyDev& s, const float* src, cudaStream_t st, int num_sms) {
#define MK_CALL(N) launch_band_nt<N, 0>(s, src, st, num_sms)
  MK_NT_SWITCH(s.nt, MK_CALL)
#undef MK_CALL
}

cudaError_t launch_inverse(const SurveyDev& s, float* dst, int mode, cudaStream_t st, int num_sms) {
#define MK_CALL(N) launch_inv_nt<N>(s, dst, mode, st, num_sms)
  MK_NT_SWITCH(s.nt, MK_CALL)
#undef MK_CALL
}

cudaError_t launch_f2p(const SurveyDev& s, float* diff, cudaStream_t st, int num_sms) {
  f2p_kernel<<<num_sms * 8, 256, 0, st>>>(s, diff);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const SurveyDev& s, float* out, const float* A, int revA, float alpha, const float* B,
                           int revB, float beta, cudaStream_t st, int num_sms) {
  lincomb_kernel<<<num_sms * 8, 256, 0, st>>>(s, out, A, revA, alpha, B, revB, beta);
  return cudaGetLastError();
}

cudaError_t launch_image(const SurveyDev& s, const float* gm, double scale, double* out, cudaStream_t st) {
  image_kernel<<<s.F, 512, 0, st>>>(s, gm, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_green(const SurveyDev& s, float* out, cudaStream_t st, int num_sms) {
  green_kernel<<<num_sms * 8, 256, 0, st>>>(s, out);
  return cudaGetLastError();
}

}  // namespace mk
