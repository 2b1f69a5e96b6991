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
// transform directly.  Constant twiddles are compile-time 64th roots of
// unity; per-lane twiddles are products of two values formed once per lane
// in FP64 and rounded to FP32.
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
constexpr size_t kSmemMax = 220 * 1024;

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
__host__ __device__ constexpr int out_slot(int e) { return (e % (32 / P)) * P + e / (32 / P); }

// Shared buffer of one trace group (float2 elements): 32 rows of P + 1; for
// P < 16 the groups sharing a half-warp are staggered by P elements so that
// their transposes hit disjoint banks.
template <int P>
__host__ __device__ constexpr int group_buf(int /*unused*/ = 0) { return 32 * (P + 1) + (P < 16 ? P : 0); }

// Per-lane twiddles of the M-point transform: W_M^{p k2} for k2 = 8a + b is
// wa[a] * wb[b] (wa[a] = W_M^{8 p a}, wb[b] = W_M^{p b}, W_M = e^{-2 pi i / M}).
struct LaneTw {
  float2 wa[4], wb[8];
  float2 up;  // e^{+2 pi i p / nt} (pre- and post-processing of the real transform)
};

__device__ __forceinline__ float2 tw_rounded(long long num, long long den) {  // e^{-2 pi i num / den}
  double sv, cv;
  sincospi(-2.0 * (double)(num % den) / (double)den, &sv, &cv);
  return make_float2((float)cv, (float)sv);
}

// Complex DFT of M = 32 P points over the P lanes of a group (lane p holds
// n = p + P e at v[e]); afterwards lane q holds index k = q + P out_e(a) at
// v[a].  gbuf is the group's shared buffer.
template <int P, bool INV>
__device__ __forceinline__ void group_fft(float2 (&v)[32], float2* gbuf, int p, const LaneTw& tw) {
  dft<32, INV>(v);  // over e: v[k2]
  static_for<32>([&](auto K) {
    constexpr int k2 = decltype(K)::value;
    constexpr int a = k2 >> 3, b = k2 & 7;
    if constexpr (k2 > 0 && P > 1) {
      float2 w;
      if constexpr (a == 0) {
        w = tw.wb[b];
      } else if constexpr (b == 0) {
        w = tw.wa[a];
      } else {
        w = cmul(tw.wa[a], tw.wb[b]);
      }
      v[k2] = INV ? cmulc(v[k2], w) : cmul(v[k2], w);
    }
  });
  if constexpr (P > 1) {  // (P = 1: 32 points, the register DFT is the whole transform)
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

struct EpiShape {
  int rounds;  // traces per group per block (1 or 2)
  int nbuf;    // stage buffers (2: the next block loads while this one is transformed)
  int bt;      // traces per block
  size_t smem;
};

template <int NT>
__host__ __device__ constexpr int traces_per_warp() { return 32 / (NT / 64); }

template <int NT>
size_t epi_smem(int nw, int rounds, int nbuf) {
  constexpr int P = NT / 64;
  const int bt = kWarps * traces_per_warp<NT>() * rounds;
  return (size_t)nbuf * nw * (bt + 1) * sizeof(float2) +
         (size_t)kWarps * traces_per_warp<NT>() * group_buf<P>() * sizeof(float2) + (size_t)nbuf * bt * sizeof(int);
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
epi_warp_kernel(SurveyDev s, double* __restrict__ ring, int slots, int rounds, int nbuf) {
  constexpr int M = NT / 2;
  constexpr int P = NT / 64;
  constexpr int TPW = 32 / P;
  constexpr int GB = group_buf<P>();
  extern __shared__ float4 smem_raw[];
  __shared__ int s_last;

  // the next contraction may be scheduled now; it waits for this grid to
  // complete before it reads what this grid writes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  const int bt = kWarps * TPW * rounds;
  const int ldm = bt + 1;
  const int nw = s.nw;
  float2* stage_base = reinterpret_cast<float2*>(smem_raw);
  const size_t stage_elems = (size_t)nw * ldm;
  float2* gbufs = stage_base + nbuf * stage_elems;
  int* sL_base = reinterpret_cast<int*>(gbufs + kWarps * TPW * GB);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / P, p = lane % P;
  float2* gbuf = gbufs + (warp * TPW + grp) * GB;

  LaneTw tw;
#pragma unroll
  for (int b = 0; b < 8; ++b) tw.wb[b] = tw_rounded((long long)p * b, M);
#pragma unroll
  for (int a = 0; a < 4; ++a) tw.wa[a] = tw_rounded((long long)8 * p * a, M);
  {
    const float2 w = tw_rounded(p, NT);  // e^{-2 pi i p / nt}
    tw.up = make_float2(w.x, -w.y);
  }

  const int iter = *s.iter;
  const int odd = iter & 1;
  double* energy_slot = ring + (int64_t)(iter % slots) * s.F;
  float* __restrict__ f1 = odd ? s.f1p : s.f1m;
  const float inv = s.inv_nt;
  const int nblocks = (s.ncols + bt - 1) / bt;
  int lbt = 0;
  while ((1 << lbt) < bt) ++lbt;  // bt is a power of two

  // the band spectra of block blk into stage buffer buf, asynchronously
  auto issue_load = [&](int blk, int buf) {
    const int tb = blk * bt;
    const int ntr = s.ncols - tb < bt ? s.ncols - tb : bt;
    float2* st = stage_base + buf * stage_elems;
    const int total = nw << lbt;
    for (int i = threadIdx.x; i < total; i += kThreads) {
      const int m = i >> lbt, c = i & (bt - 1);
      if (c < ntr) cp_async8(st + (size_t)m * ldm + c, s.S + (int64_t)m * s.s_stride + tb + c);
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
    const int tb = blk * bt;
    const int ntr = s.ncols - tb < bt ? s.ncols - tb : bt;

    for (int r = 0; r < rounds; ++r) {
      const int c = r * (kWarps * TPW) + warp * TPW + grp;  // stage column of this group's trace
      const bool active = c < ntr;
      const int L = active ? sL[c] : 0;
      const int64_t base = (int64_t)(tb + (active ? c : 0)) * NT;

      // 1. f1 samples of this lane's outputs (window only), loaded early:
      //    lane p ends the inverse transform with z_n at n = p + P out_e(a)
      float fa[32], fb[32];
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        const int n = p + P * out_e<P>(a);
        const int j0 = 2 * n, j1 = 2 * n + 1;
        const bool in0 = active && (j0 < NT - j0 ? j0 : NT - j0) < L;
        const bool in1 = active && (j1 < NT - j1 ? j1 : NT - j1) < L;
        fa[a] = 0.f;
        fb[a] = 0.f;
        if (odd) {
          if (in0) fa[a] = f1[base + ((NT - j0) & (NT - 1))];
          if (in1) fb[a] = f1[base + (NT - j1)];
        } else if (in0 || in1) {
          const float2 w = reinterpret_cast<const float2*>(f1 + base)[n];
          fa[a] = w.x;
          fb[a] = w.y;
        }
      }

      // 2. the half-length complex spectrum Z_k = (X_k + conj X_{M-k}) +
      //    i (X_k - conj X_{M-k}) e^{2 pi i k / nt}, k = p + P e, from the
      //    band spectrum X of the synthesis result (bins outside the band
      //    zero; the imaginary parts of DC and Nyquist dropped)
      float2 v[32];
      static_for<32>([&](auto E) {
        constexpr int e = decltype(E)::value;
        const int k = p + P * e;
        const int km = M - k;
        float2 X = make_float2(0.f, 0.f), Xm = make_float2(0.f, 0.f);
        if (active && k < nw) X = st[(size_t)k * ldm + c];
        if (active && km < nw) Xm = st[(size_t)km * ldm + c];
        if (k == 0) X.y = 0.f;
        if (km == M) Xm.y = 0.f;
        const float2 A = make_float2(X.x + Xm.x, X.y - Xm.y);
        const float2 B = make_float2(X.x - Xm.x, X.y + Xm.y);
        const float2 Bt = rot64<e, true>(cmul(B, tw.up));
        v[e] = make_float2(A.x - Bt.y, A.y + Bt.x);
      });

      // 3. inverse transform: z_n = x(2n) + i x(2n+1) up to the factor 1/nt
      group_fft<P, true>(v, gbuf, p, tw);

      // 4. y = theta s; f1 update; energy; y feeds the forward transform
      float esum = 0.f;
      float2 w[32];
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        const int n = p + P * out_e<P>(a);
        const int j0 = 2 * n, j1 = 2 * n + 1;
        const bool in0 = active && (j0 < NT - j0 ? j0 : NT - j0) < L;
        const bool in1 = active && (j1 < NT - j1 ? j1 : NT - j1) < L;
        const float y0 = in0 ? v[a].x * inv : 0.f;
        const float y1 = in1 ? v[a].y * inv : 0.f;
        esum = fmaf(y0, y0, esum);
        esum = fmaf(y1, y1, esum);
        if (odd) {  // f1plus(-j) += N_i(-j) = -theta(j) s(j)
          if (in0) f1[base + ((NT - j0) & (NT - 1))] = fa[a] - y0;
          if (in1) f1[base + (NT - j1)] = fb[a] - y1;
        } else if (in0 || in1) {  // f1min(j) -= N_i(-j) = theta(j) s(j)
          reinterpret_cast<float2*>(f1 + base)[n] = make_float2(fa[a] + y0, fb[a] + y1);
        }
        // forward input layout: register e = out_e(a) holds n = p + P e
        w[out_e<P>(a)] = make_float2(y0, y1);
      }

      // 5. forward transform of y
      group_fft<P, false>(w, gbuf, p, tw);

      // 6. post-processing: partner Zf_{(M-k) mod M} from lane (P - q) mod P
      //    (register e'' = 31 - e' there), or for lane 0 its own register
      //    (32 - e') mod 32
      float2 part[32];
      const int src = (P - p) & (P - 1);
      static_for<32>([&](auto Rr) {
        constexpr int r = decltype(Rr)::value;  // e' of the value this lane offers
        const float2 val = w[out_slot<P>(r)];
        float2 got;
        got.x = __shfl_sync(0xffffffffu, val.x, src, P);
        got.y = __shfl_sync(0xffffffffu, val.y, src, P);
        constexpr int et = 31 - r;
        constexpr int own = (r + 1) & 31;
        part[out_slot<P>(et)] = p != 0 ? got : w[out_slot<P>(own)];
      });
      // Y_k = E_k + e^{-2 pi i k/nt} O_k; the band spectrum of N_i is -conj(Y_k)
      static_for<32>([&](auto Aa) {
        constexpr int a = decltype(Aa)::value;
        constexpr int e = out_e<P>(a);
        const int k = p + P * e;
        if (active && k < nw) {
          const float2 Z = w[a];
          const float2 Zc = make_float2(part[a].x, -part[a].y);
          const float2 E = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
          const float2 D = csub(Z, Zc);
          const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
          const float2 T = rot64<e, false>(cmulc(O, tw.up));
          st[(size_t)k * ldm + c] = make_float2(-(E.x + T.x), E.y + T.y);
        }
      });
      if (active && p == 0 && nw == M + 1) {  // Nyquist bin (full band): Y_M = Re Zf_0 - Im Zf_0
        st[(size_t)M * ldm + c] = make_float2(-(w[0].x - w[0].y), 0.f);
      }

      // 7. the trace's energy: lanes combined error-free in FP32, then FP64
      float hi = esum, lo = 0.f;
#pragma unroll
      for (int o = P / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o, P);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o, P);
        float sum, err;
        two_sum(hi, h2, sum, err);
        hi = sum;
        lo = lo + l2 + err;
      }
      if (active && p == 0) s.Epart[tb + c] = (double)hi + (double)lo;
    }
    __syncthreads();

    // 8. the block's new band spectra, one coalesced pass
    const int total = nw << lbt;
    for (int i = threadIdx.x; i < total; i += kThreads) {
      const int m = i >> lbt, c = i & (bt - 1);
      if (c >= ntr) continue;
      const int t = tb + c;
      const int f = t / s.ns, k = t - f * s.ns;
      const float2 val = st[(size_t)m * ldm + c];
      if (s.rprec == 0) {
        s.Nw[(int64_t)m * s.nw_stride + (int64_t)f * s.r_pad + k] = val;
      } else if (s.rprec == 2) {
        store_embedding<false>(s, m, f, k, val.x, val.y);
      } else {
        store_embedding<true>(s, m, f, k, val.x, val.y);
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
    const int bt2 = kWarps * traces_per_warp<NT>() * 2;
    if ((s.ncols + bt2 - 1) / bt2 < num_sms) rounds = 1;
  }
  for (; rounds >= 1; --rounds) {
    for (int nbuf = 2; nbuf >= 1; --nbuf) {
      const size_t smem = epi_smem<NT>(s.nw, rounds, nbuf);
      if (smem <= kSmemMax) {
        *out = {rounds, nbuf, kWarps * traces_per_warp<NT>() * rounds, smem};
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
  const int nblocks = (s.ncols + sh.bt - 1) / sh.bt;
  const int grid = nblocks < num_sms ? nblocks : num_sms;
  epi_warp_kernel<NT><<<grid, kThreads, sh.smem, st>>>(s, ring, slots, sh.rounds, sh.nbuf);
  return cudaGetLastError();
}

template <int NT>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(epi_warp_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
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
  return set_attr<2048>();
}

cudaError_t launch_epilogue_warp(const SurveyDev& s, double* ring, int slots, cudaStream_t st, int num_sms) {
  switch (s.nt) {
    case 64: return launch_nt<64>(s, ring, slots, st, num_sms);
    case 128: return launch_nt<128>(s, ring, slots, st, num_sms);
    case 256: return launch_nt<256>(s, ring, slots, st, num_sms);
    case 512: return launch_nt<512>(s, ring, slots, st, num_sms);
    case 1024: return launch_nt<1024>(s, ring, slots, st, num_sms);
    case 2048: return launch_nt<2048>(s, ring, slots, st, num_sms);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace mk
