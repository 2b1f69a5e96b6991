// Epilogue of one Neumann iteration with the transforms held in registers:
// per trace, the inverse transform of the band-limited synthesis result
// (Theory: frequency domain; Implementation: "padding"), the theta mute, the
// accumulation of f1min / f1plus and the energy (Algorithm 1), and the band
// spectrum of N_i for the next contraction.
//
// Two identities of the real transforms remove every data exchange the time
// reversal would need:
//  * N_i(j) = -theta(j) s(-j), so DFT(N_i)_k = -conj(DFT(theta s)_k): the
//    forward transform takes y = theta s as it comes out of the inverse one,
//    and the reversal becomes a conjugation of the band spectrum;
//  * f1min(j) += y(j) on even iterations and f1plus(-j) -= y(j) on odd ones,
//    so each lane updates the f1 samples of its own y (mirrored addresses on
//    odd iterations), and E_i = sum y^2 from its own registers.
//
// A real trace of nt samples is transformed as a complex sequence of
// M = nt/2 points, z_n = x(2n) + i x(2n+1), with the usual pre- and
// post-processing of the half-length complex transform.  The M-point complex
// DFT runs on a group of P = nt/64 lanes holding 32 values each (index
// n = p + P e at register e): a 32-point DFT in registers, twiddles, one
// transpose through a shared buffer private to the group, and 32/P DFTs of
// P points in registers.  The result comes back in the same index layout
// (k = q + P e'), so the inverse transform's output feeds the forward
// transform directly.  For nt = 4096 (P = 64) a trace takes two warps: the
// 64-point DFTs over the lanes split by decimation in frequency into a
// butterfly across the two warps (through the group's shared buffer, the
// warps meeting at a named barrier) and 32-point DFTs in registers.
// Constant twiddles are compile-time 64th roots of unity; per-lane twiddles
// are products of two entries of a table of e^{-2 pi i j / nt} (FP64 values
// rounded to FP32), kept in shared memory per CTA.
//
// A CTA of 8 warps takes blocks of consecutive traces (focal-major order, so
// neighbouring traces are neighbouring addresses in S and Nw): the block's
// band spectra are copied from S into a frequency-major shared stage with
// asynchronous copies, one block ahead (double-buffered when shared memory
// allows), each trace group transforms its trace and writes the new band
// spectrum into the same stage column, and one coalesced pass writes the
// block to Nw or to the 16-bit embedding of the tensor-core contraction.
// Energies: each lane sums its squares in FP32, the lanes of a trace are
// combined with error-free FP32 transformations, per trace and per focal
// point the sums are FP64, in a fixed order (deterministic).

#include <utility>

#include "mk_embed.cuh"
#include "mk_internal.h"

namespace mk {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

// cos(2 pi r / 64), r = 0 .. 16 (FP64 values rounded to FP32)
__host__ __device__ constexpr float qcos(int r) {
  return r == 0    ? 1.0f
         : r == 1  ? 0.9951847195625305f
         : r == 2  ? 0.9807852506637573f
         : r == 3  ? 0.9569403529167175f
         : r == 4  ? 0.9238795042037964f
         : r == 5  ? 0.8819212913513184f
         : r == 6  ? 0.8314695954322815f
         : r == 7  ? 0.7730104327201843f
         : r == 8  ? 0.7071067690849304f
         : r == 9  ? 0.6343932747840881f
         : r == 10 ? 0.5555702447891235f
         : r == 11 ? 0.4713967442512512f
         : r == 12 ? 0.3826834261417389f
         : r == 13 ? 0.290284663438797f
         : r == 14 ? 0.19509032368659973f
         : r == 15 ? 0.0980171412229538f
                   : 0.0f;
}
// e^{2 pi i m / 64} = (w64c(m), w64s(m)) for any integer m
__host__ __device__ constexpr float w64c(int m) {
  return ((m & 63) >> 4) == 0   ? qcos(m & 15)
         : ((m & 63) >> 4) == 1 ? -qcos(16 - (m & 15))
         : ((m & 63) >> 4) == 2 ? -qcos(m & 15)
                                : qcos(16 - (m & 15));
}
__host__ __device__ constexpr float w64s(int m) {
  return ((m & 63) >> 4) == 0   ? qcos(16 - (m & 15))
         : ((m & 63) >> 4) == 1 ? qcos(m & 15)
         : ((m & 63) >> 4) == 2 ? -qcos(16 - (m & 15))
                                : -qcos(m & 15);
}

template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
// f(std::integral_constant<int, i>) for i = 0 .. N-1, with i a constant expression
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// v * e^{-+2 pi i m / 64} (forward: minus, inverse: plus), m a constant
template <int Mi, bool INV>
__host__ __device__ __forceinline__ float2 rot64(float2 v) {
  constexpr int m = (INV ? Mi : -Mi) & 63;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 16) {
    return make_float2(-v.y, v.x);
  } else if constexpr (m == 32) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 48) {
    return make_float2(v.y, -v.x);
  } else {
    constexpr float c = w64c(m), s = w64s(m);
    return make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
  }
}

// Unnormalised DFT of N values in registers, natural order in and out
// (forward kernel e^{-2 pi i nk/N}, inverse e^{+2 pi i nk/N}); N | 64.
template <int N, bool INV>
__host__ __device__ __forceinline__ void dft(float2 (&v)[N]);

template <int N1, int N2, bool INV>
__host__ __device__ __forceinline__ void dft_split(float2 (&v)[N1 * N2]) {
  // n = n1 + N1 n2, k = k2 + N2 k1: N1 DFTs of N2 points over n2, twiddles
  // W_N^{n1 k2}, N2 DFTs of N1 points over n1
  constexpr int N = N1 * N2;
  float2 y[N1][N2];
  static_for<N1>([&](auto I1) {
    constexpr int n1 = decltype(I1)::value;
    float2 t[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) t[n2] = v[n1 + N1 * n2];
    dft<N2, INV>(t);
    static_for<N2>([&](auto I2) {
      constexpr int k2 = decltype(I2)::value;
      y[n1][k2] = rot64<(64 / N) * n1 * k2, INV>(t[k2]);
    });
  });
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    float2 t[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) t[n1] = y[n1][k2];
    dft<N1, INV>(t);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k2 + N2 * k1] = t[k1];
  }
}

template <int N, bool INV>
__host__ __device__ __forceinline__ void dft(float2 (&v)[N]) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (N == 4) {
    const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]);
    const float2 a3 = rot64<16, INV>(csub(v[1], v[3]));  // * -+i
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
  } else if constexpr (N == 8) {
    dft_split<2, 4, INV>(v);
  } else if constexpr (N == 16) {
    dft_split<4, 4, INV>(v);
  } else if constexpr (N == 32) {
    dft_split<4, 8, INV>(v);
  } else {
    static_assert(N == 64, "DFT length");
    dft_split<8, 8, INV>(v);
  }
}

// Register index of the transform's output e' (index k = q + P e') as it
// comes out of group_fft, and the inverse map.
template <int P>
__host__ __device__ constexpr int out_e(int a) { return a / P + (32 / P) * (a % P); }
template <int P>
__host__ __device__ constexpr int out_slot(int e) { return P >= 32 ? e : (e % (32 / P)) * P + e / (32 / P); }

// Shared buffer of one trace group (float2 elements): the 32 x P transpose,
// rows of P + 1; for P < 16 the groups sharing a half-warp are staggered by
// P elements so that their accesses hit disjoint banks.  One lane per trace
// (P = 1) needs no transpose.  For P = 64 (two warps per trace) the buffer
// also carries the post-processing exchange (M values) and, past them, the
// second warp's energy partial.
template <int P>
__host__ __device__ constexpr int group_buf() { return P == 1 ? 0 : 32 * (P + 1) + (P < 16 ? P : 0); }

// Per-lane twiddle W_M^{p k2} (W_M = e^{-2 pi i / M}, M = nt/2) as the product
// of two entries of the table e^{-2 pi i j / nt}: k2 = 8a + b,
// W_M^{p k2} = W_M^{8 p a} W_M^{p b} (W_M^x = entry 2x mod nt).  The ten
// factors of lane p (b = 1 .. 7, a = 1 .. 3) depend on p only: the CTA keeps
// them in shared memory, factor j of lane p at tws[j P + p].
constexpr int kLaneTw = 10;
template <int NT>
__device__ __forceinline__ float2 lane_twiddle_entry(const float2* __restrict__ twl, int j, int p) {
  return __ldg(twl + ((j < 7 ? 2 * p * (j + 1) : 16 * p * (j - 6)) & (NT - 1)));
}
template <int NT>
__device__ __forceinline__ void lane_twiddles(const float2* tws, int p, float2 (&wa)[4], float2 (&wb)[8]) {
  constexpr int P = NT / 64;
#pragma unroll
  for (int b = 1; b < 8; ++b) wb[b] = tws[(b - 1) * P + p];
#pragma unroll
  for (int a = 1; a < 4; ++a) wa[a] = tws[(6 + a) * P + p];
}

// The two warps of a P = 64 group meet at named barrier bar (1 + group).
__device__ __forceinline__ void pair_sync(int bar) { asm volatile("bar.sync %0, 64;" ::"r"(bar) : "memory"); }

// Complex DFT of M = 32 P points over the P lanes of a group (lane p holds
// n = p + P e at v[e]); afterwards lane q holds index k = q + P out_e(a) at
// v[a].  gbuf is the group's shared buffer.
//
// P = 64 (nt = 4096, two warps per trace): after the 32-point DFTs over e
// and the twiddles W_M^{p k2}, the 64-point DFTs over p run split by
// decimation in frequency, k1 = 2j + h: lane (h, k2) of warp h forms
// u_p = (x_p + (-1)^h x_{p+32}) W_64^{p h}, p < 32, from the transposed
// values and takes its 32-point DFT, so that lane q = 32h + k2 ends with
// index k = q + 64 j at v[j].  Both warps call this with the same bar.
template <int NT, bool INV>
__device__ __forceinline__ void group_fft(float2 (&v)[32], float2* gbuf, int p, const float2* tws, int bar) {
  constexpr int P = NT / 64;
  if constexpr (P == 64) {
    float2 wa[4], wb[8];
    lane_twiddles<NT>(tws, p, wa, wb);
    dft<32, INV>(v);  // over e: v[k2]
    static_for<32>([&](auto K) {
      constexpr int k2 = decltype(K)::value;
      constexpr int a = k2 >> 3, b = k2 & 7;
      if constexpr (k2 > 0) {
        float2 w;
        if constexpr (a == 0) {
          w = wb[b];
        } else if constexpr (b == 0) {
          w = wa[a];
        } else {
          w = cmul(wa[a], wb[b]);
        }
        v[k2] = INV ? cmulc(v[k2], w) : cmul(v[k2], w);
      }
    });
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) gbuf[k2 * 65 + p] = v[k2];
    pair_sync(bar);
    const float2* row = gbuf + (p & 31) * 65;  // k2 = p mod 32
    if (p >= 32) {
      static_for<32>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        v[q] = rot64<q, INV>(csub(row[q], row[q + 32]));
      });
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = cadd(row[q], row[q + 32]);
    }
    pair_sync(bar);  // the buffer is free again
    dft<32, INV>(v);
  } else if constexpr (P > 1) {
    float2 wa[4], wb[8];
    lane_twiddles<NT>(tws, p, wa, wb);
    dft<32, INV>(v);  // over e: v[k2]
    static_for<32>([&](auto K) {
      constexpr int k2 = decltype(K)::value;
      constexpr int a = k2 >> 3, b = k2 & 7;
      if constexpr (k2 > 0) {
        float2 w;
        if constexpr (a == 0) {
          w = wb[b];
        } else if constexpr (b == 0) {
          w = wa[a];
        } else {
          w = cmul(wa[a], wb[b]);
        }
        v[k2] = INV ? cmulc(v[k2], w) : cmul(v[k2], w);
      }
    });
    // transpose: row k2 of lane n1 to column k2, which lane q = k2 mod P
    // takes (columns k2 = q + P c)
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) gbuf[k2 * (P + 1) + p] = v[k2];
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 32 / P; ++c) {
      float2 t[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) t[n1] = gbuf[(p + P * c) * (P + 1) + n1];
      dft<P, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) v[c * P + k1] = t[k1];
    }
    __syncwarp();
  } else {
    dft<32, INV>(v);  // 32 points: the register DFT is the whole transform
  }
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// error-free sum of two floats: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// floor(x / d) and ceil(x / d) for d > 0 and any x
__device__ __forceinline__ int floor_div(int x, int d) { return x >= 0 ? x / d : -((d - 1 - x) / d); }
__device__ __forceinline__ int ceil_div(int x, int d) { return -floor_div(-x, d); }
__device__ __forceinline__ int clamp32(int x) { return x < 0 ? 0 : (x > 32 ? 32 : x); }

struct EpiShape {
  int rounds;  // traces per group per block (1 or 2)
  int nbuf;    // stage buffers (2: the next block loads while this one is transformed)
  int bt;      // traces per block
  size_t smem;
};

constexpr int kCtasPerSm = 2;
constexpr size_t kSmemPerCta = 110 * 1024;  // two CTAs per SM

// traces a CTA transforms at once (one per group of P = nt/64 lanes)
template <int NT>
__host__ __device__ constexpr int traces_per_cta() { return kThreads / (NT / 64); }

template <int NT>
size_t epi_smem(int nw, int rounds, int nbuf) {
  constexpr int P = NT / 64;
  const int bt = traces_per_cta<NT>() * rounds;
  return (size_t)nbuf * nw * (bt + 1) * sizeof(float2) +
         (size_t)traces_per_cta<NT>() * group_buf<P>() * sizeof(float2) +
         (size_t)kLaneTw * P * sizeof(float2) + (size_t)nbuf * bt * sizeof(int);
}

// A full block's band spectra to Nw[m][f][k0 .. k0 + bt): 16-byte stores of
// two complex values, consecutive threads on consecutive pairs.
__device__ __forceinline__ void store_block_nw(const SurveyDev& s, const float2* st, int ldm, int f, int k0, int bt,
                                               int lbt) {
  const int lq = lbt - 1;  // bt / 2 pairs per frequency
  const int total = s.nw << lq;
  float2* base = s.Nw + (int64_t)f * s.r_pad + k0;
  for (int i = threadIdx.x; i < total; i += kThreads) {
    const int m = i >> lq, q = i & ((bt >> 1) - 1);
    const float2 a = st[m * ldm + 2 * q], b = st[m * ldm + 2 * q + 1];
    *reinterpret_cast<float4*>(base + (int64_t)m * s.nw_stride + 2 * q) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// A full block's band spectra into the 16-bit embedding of the tensor-core
// contraction: NP parts (hi + lo, or hi + mid + lo), rows 2f (Nr, -Ni) and
// 2f+1 (Ni, Nr).  A task is four consecutive positions of one frequency;
// consecutive lanes take consecutive tasks, so each row segment of a part
// (bt 32-bit pairs) is written by neighbouring lanes as whole 32-byte
// sectors.  Same roundings as store_embedding.
template <bool BF16, int NP>
__device__ __forceinline__ void store_block_embedding(const SurveyDev& s, const float2* st, int ldm, int f, int k0,
                                                      int bt, int lbt) {
  const int64_t rp = s.r_pad;
  const int lq = lbt - 2;  // bt / 4 tasks per frequency
  const int total = s.nw << lq;
  uint32_t* b0 = reinterpret_cast<uint32_t*>(s.Bq0);
  uint32_t* b1 = reinterpret_cast<uint32_t*>(s.Bq1);
  uint32_t* b2 = reinterpret_cast<uint32_t*>(s.Bq2);
  for (int i = threadIdx.x; i < total; i += kThreads) {
    const int m = i >> lq, q = 4 * (i & ((1 << lq) - 1));
    const int64_t w0 = ((int64_t)m * 2 * s.F + 2 * f) * rp + k0 + q;  // 32-bit word of row 2f
    uint32_t wd[NP][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 v = st[m * ldm + q + u];
      float hr, hi, mr, mi;
      wd[0][u] = round_pair<BF16>(v.x, v.y, hr, hi);
      const float lr = v.x - hr, li = v.y - hi;  // exact in FP32
      wd[1][u] = round_pair<BF16>(lr, li, mr, mi);
      if constexpr (NP == 3) wd[2][u] = round_pair<BF16>(lr - mr, li - mi, mr, mi);
    }
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      uint32_t* b = pp == 0 ? b0 : (pp == 1 ? b1 : b2);
      *reinterpret_cast<uint4*>(b + w0) =
          make_uint4(pair_neg_hi(wd[pp][0]), pair_neg_hi(wd[pp][1]), pair_neg_hi(wd[pp][2]), pair_neg_hi(wd[pp][3]));
      *reinterpret_cast<uint4*>(b + w0 + rp) =
          make_uint4(pair_swap(wd[pp][0]), pair_swap(wd[pp][1]), pair_swap(wd[pp][2]), pair_swap(wd[pp][3]));
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
epi_warp_kernel(SurveyDev s, double* __restrict__ ring, int slots, int rounds, int nbuf) {
  constexpr int M = NT / 2;
  constexpr int P = NT / 64;
  constexpr int NG = kThreads / P;  // trace groups per CTA
  constexpr int GB = group_buf<P>();
  extern __shared__ float4 smem_raw[];
  __shared__ int s_last;

  // the next contraction may be scheduled now; it waits for this grid to
  // complete before it reads what this grid writes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  const int bt = NG * rounds;
  const int ldm = bt + 1;
  const int nw = s.nw;
  float2* stage_base = reinterpret_cast<float2*>(smem_raw);
  const size_t stage_elems = (size_t)nw * ldm;
  float2* gbufs = stage_base + nbuf * stage_elems;
  float2* tws = gbufs + NG * GB;  // the lanes' twiddle factors
  int* sL_base = reinterpret_cast<int*>(tws + kLaneTw * P);
  for (int i = threadIdx.x; i < kLaneTw * P; i += kThreads) tws[i] = lane_twiddle_entry<NT>(s.twl, i / P, i % P);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = (int)threadIdx.x / P, p = (int)threadIdx.x % P;  // trace group, lane in the group
  float2* gbuf = gbufs + slot * GB;
  float2 up;  // e^{+2 pi i p / nt}
  {
    const float2 w = __ldg(s.twl + p);
    up = make_float2(w.x, -w.y);
  }

  const int iter = *s.iter;
  const int odd = iter & 1;
  double* energy_slot = ring + (int64_t)(iter % slots) * s.F;
  float* __restrict__ f1 = odd ? s.f1p : s.f1m;
  const float inv = s.inv_nt;
  // blocks never straddle focal points: block (f, kb) holds positions
  // k0 = kb bt .. k0 + ntr - 1 of focal point f (traces t = f ns + k)
  const int nkb = (s.ns + bt - 1) / bt;
  const int nblocks = s.F * nkb;
  int lbt = 0;
  while ((1 << lbt) < bt) ++lbt;  // bt is a power of two dividing kThreads

  // each thread of the block passes keeps one trace column: c = tid mod bt,
  // frequencies m = tid / bt, tid / bt + 256 / bt, ...
  const int pc = threadIdx.x & (bt - 1);
  const int pm0 = threadIdx.x >> lbt, pms = kThreads >> lbt;

  // the band spectra of block blk into stage buffer buf, asynchronously
  auto issue_load = [&](int blk, int buf) {
    const int bf = blk / nkb;
    const int k0 = (blk - bf * nkb) * bt;
    const int tb = bf * s.ns + k0;
    const int ntr = s.ns - k0 < bt ? s.ns - k0 : bt;
    float2* st = stage_base + buf * stage_elems;
    if (pc < ntr) {
      const float2* src = s.S + (int64_t)pm0 * s.s_stride + tb + pc;
      const int64_t sstep = (int64_t)pms * s.s_stride;
      for (int m = pm0; m < nw; m += pms, src += sstep) cp_async8(st + m * ldm + pc, src);
    }
    int* sL = sL_base + buf * bt;
    for (int c = threadIdx.x; c < bt; c += kThreads) sL[c] = c < ntr ? s.L[tb + c] : 0;
    cp_async_commit();
  };

  int blk = blockIdx.x;
  if (blk < nblocks) issue_load(blk, 0);
  for (int it = 0; blk < nblocks; blk += gridDim.x, ++it) {
    const int buf = nbuf == 2 ? (it & 1) : 0;
    const int nxt = blk + (int)gridDim.x;
    if (nbuf == 2) {
      if (nxt < nblocks) {
        issue_load(nxt, buf ^ 1);
      } else {
        cp_async_commit();  // an empty group keeps the wait count uniform
      }
      cp_async_wait_1();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    float2* st = stage_base + buf * stage_elems;
    const int* sL = sL_base + buf * bt;
    const int bf = blk / nkb;
    const int k0 = (blk - bf * nkb) * bt;
    const int tb = bf * s.ns + k0;
    const int ntr = s.ns - k0 < bt ? s.ns - k0 : bt;
    if (s.pacc) {
      // pmin's band spectrum += S from the stage, as fire-and-forget
      // reductions (one per (m, t) and launch: the same sum in any schedule),
      // before the transforms overwrite the stage
      if (pc < ntr) {
        float2* acc = s.pacc + (int64_t)pm0 * s.s_stride + tb + pc;
        const int64_t astep = (int64_t)pms * s.s_stride;
        for (int m = pm0; m < nw; m += pms, acc += astep) atomicAdd(acc, st[m * ldm + pc]);
      }
      __syncthreads();
    }

    for (int r = 0; r < rounds; ++r) {
      const int c = r * NG + slot;  // stage column of this group's trace
      const bool active = c < ntr;
      const int L = active ? sL[c] : 0;
      float* __restrict__ ft = f1 + (int64_t)(tb + (active ? c : 0)) * NT;  // this trace of f1
      float2* col = st + c;
      if (active && p == 0 && L > 0) {
        // the window samples j < L and j > nt - L of f1 (both parities touch
        // only these) into L2 while the inverse transform runs: 16-byte
        // aligned ranges (the trace starts on a 16-byte boundary)
        const unsigned n0 = (unsigned)((4 * L + 15) & ~15);
        const int j2 = L > NT ? 0 : (NT - L + 1) & ~3;  // L <= nt/2 + 1 from the window kernel
        prefetch_l2(ft, n0 < 4u * NT ? n0 : 4u * NT);
        if (j2 < NT) prefetch_l2(ft + j2, 4u * (unsigned)(NT - j2));
      }
      // Bounds in register index e, once per trace (inactive groups: none):
      //  band bins k = p + P e < nw  <=>  e < ek;  M - k < nw  <=>  e >= em;
      //  window samples j0 = 2(p + P e): j0 < L <=> e < a0, j0 > nt - L <=> e >= b0;
      //  j1 = j0 + 1 likewise with a1, b1 (theta(j) = j < L or j > nt - L).
      const int ek = active ? clamp32(ceil_div(nw - p, P)) : 0;
      const int em = active ? clamp32(floor_div(M - p - nw, P) + 1) : 32;
      const int a0 = clamp32(ceil_div(L - 2 * p, 2 * P));
      const int b0 = active ? clamp32(floor_div(NT - L - 2 * p, 2 * P) + 1) : 32;
      const int a1 = clamp32(ceil_div(L - 2 * p - 1, 2 * P));
      const int b1 = active ? clamp32(floor_div(NT - L - 2 * p - 1, 2 * P) + 1) : 32;
      const float2* colp = col + p * ldm;         // bin k = p + P e at colp[e P ldm]
      const float2* colm = col + (M - p) * ldm;   // bin M - k at colm[-e P ldm]
      const int pst = P * ldm;

      // 1. the half-length complex spectrum Z_k = (X_k + conj X_{M-k}) +
      //    i (X_k - conj X_{M-k}) e^{2 pi i k / nt}, k = p + P e, from the
      //    band spectrum X of the synthesis result (bins outside the band
      //    zero; the imaginary parts of DC and Nyquist dropped)
      float2 v[32];
      static_for<32>([&](auto E) {
        constexpr int e = decltype(E)::value;
        float2 X = make_float2(0.f, 0.f), Xm = make_float2(0.f, 0.f);
        if (e < ek) X = colp[e * pst];
        if (e >= em) Xm = colm[-e * pst];
        if (e == 0 && p == 0) {
          X.y = 0.f;
          Xm.y = 0.f;  // M - k == M: the Nyquist bin
        }
        const float2 A = make_float2(X.x + Xm.x, X.y - Xm.y);
        const float2 B = make_float2(X.x - Xm.x, X.y + Xm.y);
        const float2 Bt = rot64<e, true>(cmul(B, up));
        v[e] = make_float2(A.x - Bt.y, A.y + Bt.x);
      });

      // 2. inverse transform: z_n = x(2n) + i x(2n+1) up to the factor 1/nt
      group_fft<NT, true>(v, gbuf, p, tws, 1 + slot);

      // 3. y = theta s on the window samples of this lane (the rest is zero),
      //    its energy, and f1 on the window: even iterations
      //    f1min(j) -= N_i(-j) = y(j), odd iterations f1plus(-j) += N_i(-j) = -y(j).
      //    Register e of the forward input holds n = p + P e (samples 2n and
      //    2n + 1), taken from register out_slot(e) of the inverse output.
      //    Chunks of four registers that no lane of the warp needs in f1 skip
      //    the f1 traffic; a chunk's loads are issued together.
      float2 w[32];
      static_for<8>([&](auto Ch) {
        constexpr int e0 = 4 * decltype(Ch)::value;
        bool need[4];
        bool any = false;
        static_for<4>([&](auto U) {
          constexpr int u = decltype(U)::value;
          constexpr int e = e0 + u;
          const bool in0 = e < a0 || e >= b0;
          const bool in1 = e < a1 || e >= b1;
          const float2 z = v[out_slot<P>(e)];
          const float y0 = in0 ? z.x * inv : 0.f;
          const float y1 = in1 ? z.y * inv : 0.f;
          w[e] = make_float2(y0, y1);
          need[u] = in0 || in1;
          any = any || need[u];
        });
        if (__any_sync(0xffffffffu, any)) {
          float2 old[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int n = p + P * (e0 + u);
            old[u] = make_float2(0.f, 0.f);
            if (need[u]) {
              if (odd) {
                old[u].x = ft[(NT - 2 * n) & (NT - 1)];
                old[u].y = ft[NT - 2 * n - 1];
              } else {
                old[u] = reinterpret_cast<const float2*>(ft)[n];
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int n = p + P * (e0 + u);
            if (need[u]) {
              const float2 y = w[e0 + u];
              if (odd) {
                ft[(NT - 2 * n) & (NT - 1)] = old[u].x - y.x;
                ft[NT - 2 * n - 1] = old[u].y - y.y;
              } else {
                reinterpret_cast<float2*>(ft)[n] = make_float2(old[u].x + y.x, old[u].y + y.y);
              }
            }
          }
        }
      });

      // the lane's share of the energy: four partial sums in a fixed order
      float eq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        eq[e & 3] = fmaf(w[e].x, w[e].x, eq[e & 3]);
        eq[e & 3] = fmaf(w[e].y, w[e].y, eq[e & 3]);
      }
      const float esum = (eq[0] + eq[1]) + (eq[2] + eq[3]);

      // 5. forward transform of y
      group_fft<NT, false>(w, gbuf, p, tws, 1 + slot);

      // 6. post-processing for the band bins k = q + P e' < nw: the partner
      //    Zf_{(M-k) mod M} comes from lane (P - q) mod P of the group
      //    (its register e'' = 31 - e'), or for lane 0 from its own register
      //    (32 - e') mod 32.  Y_k = E_k + e^{-2 pi i k/nt} O_k with
      //    E_k = (Zf_k + conj Zf_{M-k})/2, O_k = (Zf_k - conj Zf_{M-k})/(2i);
      //    the band spectrum of N_i is -conj(Y_k).
      //    For P = 64 the partners sit in the other warp: the group's Zf
      //    pass through its buffer, and so does the second warp's energy sum.
      // the lanes' energy sums of this warp, combined error-free
      auto warp_energy = [&](float& hi, float& lo) {
        constexpr int WD = P < 32 ? P : 32;
        hi = esum;
        lo = 0.f;
#pragma unroll
        for (int o = WD / 2; o > 0; o >>= 1) {
          const float h2 = __shfl_down_sync(0xffffffffu, hi, o, WD);
          const float l2 = __shfl_down_sync(0xffffffffu, lo, o, WD);
          float sum, err;
          two_sum(hi, h2, sum, err);
          hi = sum;
          lo = lo + l2 + err;
        }
      };
      float hi = 0.f, lo = 0.f;
      if constexpr (P == 64) {
        warp_energy(hi, lo);
#pragma unroll
        for (int e = 0; e < 32; ++e) gbuf[p + 64 * e] = w[e];
        if (p == 32) gbuf[M] = make_float2(hi, lo);
        pair_sync(1 + slot);
      }
      static_for<32>([&](auto Ee) {
        constexpr int e = decltype(Ee)::value;
        if (e * P < nw) {  // uniform: some lane of every group has k < nw
          const float2 Z = w[out_slot<P>(e)];
          float2 pz;
          if constexpr (P == 64) {
            pz = gbuf[(M - (p + 64 * e)) & (M - 1)];
          } else {
            const int src = (P - p) & (P - 1);
            const float2 offer = w[out_slot<P>(31 - e)];
            float2 got;
            got.x = __shfl_sync(0xffffffffu, offer.x, src, P);
            got.y = __shfl_sync(0xffffffffu, offer.y, src, P);
            pz = p != 0 ? got : w[out_slot<P>((32 - e) & 31)];
          }
          if (e < ek) {
            const float2 Zc = make_float2(pz.x, -pz.y);
            const float2 Ev = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
            const float2 D = csub(Z, Zc);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            const float2 T = rot64<e, false>(cmulc(O, up));
            col[(p + P * e) * ldm] = make_float2(-(Ev.x + T.x), Ev.y + T.y);
          }
        }
      });
      if (active && p == 0 && nw == M + 1) {  // Nyquist bin (full band): Y_M = Re Zf_0 - Im Zf_0
        col[M * ldm] = make_float2(-(w[0].x - w[0].y), 0.f);
      }

      // 7. the trace's energy: lanes combined error-free in FP32 (for P = 64
      //    the second warp's sum joins through the group buffer), then FP64
      if constexpr (P < 64) {
        warp_energy(hi, lo);
      } else {
        if (p == 0) {
          const float2 o2 = gbuf[M];
          float sum, err;
          two_sum(hi, o2.x, sum, err);
          hi = sum;
          lo = lo + o2.y + err;
        }
        pair_sync(1 + slot);  // the buffer is free again
      }
      if (active && p == 0) s.Epart[tb + c] = (double)hi + (double)lo;
    }
    __syncthreads();

    // 8. the block's new band spectra.  A full block writes whole row
    //    segments with 16-byte stores (its positions start at a multiple of bt,
    //    so the segments are 16-byte aligned); a ragged one element by element.
    if (ntr == bt) {
      const int kr = k0 + s.row0;  // on the field spectrum's r axis (row0 is a multiple of 32)
      if (field_in_nw(s)) {
        store_block_nw(s, st, ldm, bf, kr, bt, lbt);
      } else if (s.rprec == 2) {
        store_block_embedding<false, 2>(s, st, ldm, bf, kr, bt, lbt);
      } else if (s.rprec == 4) {
        store_block_embedding<true, 3>(s, st, ldm, bf, kr, bt, lbt);
      } else {
        store_block_embedding<true, 2>(s, st, ldm, bf, kr, bt, lbt);
      }
    } else if (pc < ntr) {
      const int k = k0 + pc + s.row0;
      if (field_in_nw(s)) {
        float2* dst = s.Nw + (int64_t)pm0 * s.nw_stride + (int64_t)bf * s.r_pad + k;
        const int64_t dstep = (int64_t)pms * s.nw_stride;
        for (int m = pm0; m < nw; m += pms, dst += dstep) *dst = st[m * ldm + pc];
      } else {
        const int64_t kp = 2 * (int64_t)s.r_pad;
        int64_t e0 = ((int64_t)pm0 * 2 * s.F + 2 * bf) * kp + 2 * k;
        const int64_t estep = (int64_t)pms * 2 * s.F * kp;
        for (int m = pm0; m < nw; m += pms, e0 += estep) {
          const float2 val = st[m * ldm + pc];
          if (s.rprec == 2) {
            store_embedding_at<false>(s, e0, val.x, val.y);
          } else {
            store_embedding_at<true>(s, e0, val.x, val.y);
          }
        }
      }
    }
    __syncthreads();
    if (nbuf == 1 && nxt < nblocks) issue_load(nxt, 0);
  }
  cp_async_wait_all();

  // The last CTA to finish sums the per-trace energies per focal point, one
  // warp per focal point: lane l adds k = l, l + 32, ... in ascending order,
  // then a fixed shuffle tree; the order never depends on scheduling.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(s.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int f = warp; f < s.F; f += kWarps) {
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

template <int NT>
bool epi_shape(const SurveyDev& s, int num_sms, EpiShape* out) {
  int rounds = 2;
  if (s.epi_g > 0) {
    rounds = s.epi_g >= 2 ? 2 : 1;
  } else {
    // few traces: one round per block, so that more SMs get blocks
    const int bt2 = traces_per_cta<NT>() * 2;
    if (s.F * ((s.ns + bt2 - 1) / bt2) < kCtasPerSm * num_sms) rounds = 1;
  }
  for (; rounds >= 1; --rounds) {
    for (int nbuf = 2; nbuf >= 1; --nbuf) {
      const size_t smem = epi_smem<NT>(s.nw, rounds, nbuf);
      if (smem <= kSmemPerCta) {
        *out = {rounds, nbuf, traces_per_cta<NT>() * rounds, smem};
        return true;
      }
    }
  }
  return false;
}

template <int NT>
cudaError_t launch_nt(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms) {
  EpiShape sh;
  if (!epi_shape<NT>(s, num_sms, &sh)) return cudaErrorNotSupported;
  const int nblocks = s.F * ((s.ns + sh.bt - 1) / sh.bt);
  const int grid = nblocks < kCtasPerSm * num_sms ? nblocks : kCtasPerSm * num_sms;
  epi_warp_kernel<NT><<<grid, kThreads, sh.smem, st>>>(s, ring, slots, sh.rounds, sh.nbuf);
  return cudaGetLastError();
}

template <int NT>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(epi_warp_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemPerCta);
}

}  // namespace

bool epilogue_warp_supports(int nt, int nw) {
  SurveyDev s{};
  s.nw = nw;
  s.ncols = 1;
  EpiShape sh;
  switch (nt) {
    case 64: return epi_shape<64>(s, 1, &sh);
    case 128: return epi_shape<128>(s, 1, &sh);
    case 256: return epi_shape<256>(s, 1, &sh);
    case 512: return epi_shape<512>(s, 1, &sh);
    case 1024: return epi_shape<1024>(s, 1, &sh);
    case 2048: return epi_shape<2048>(s, 1, &sh);
    case 4096: return epi_shape<4096>(s, 1, &sh);
    default: return false;
  }
}

cudaError_t prepare_epilogue_warp() {
  cudaError_t e;
  if ((e = set_attr<64>()) != cudaSuccess) return e;
  if ((e = set_attr<128>()) != cudaSuccess) return e;
  if ((e = set_attr<256>()) != cudaSuccess) return e;
  if ((e = set_attr<512>()) != cudaSuccess) return e;
  if ((e = set_attr<1024>()) != cudaSuccess) return e;
  if ((e = set_attr<2048>()) != cudaSuccess) return e;
  return set_attr<4096>();
}

cudaError_t launch_epilogue_warp(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms) {
  switch (s.nt) {
    case 64: return launch_nt<64>(s, ring, slots, st, num_sms);
    case 128: return launch_nt<128>(s, ring, slots, st, num_sms);
    case 256: return launch_nt<256>(s, ring, slots, st, num_sms);
    case 512: return launch_nt<512>(s, ring, slots, st, num_sms);
    case 1024: return launch_nt<1024>(s, ring, slots, st, num_sms);
    case 2048: return launch_nt<2048>(s, ring, slots, st, num_sms);
    case 4096: return launch_nt<4096>(s, ring, slots, st, num_sms);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace mk
