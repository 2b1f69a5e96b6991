// The contraction of Eq. (1) on the 5th-generation tensor cores (tcgen05),
// for R stored in 16-bit precision:
//     S_m[k][f] = c * sum_r R_m[k][r] Nw_m[r][f]      (complex)
//
// Complex products as one real GEMM per frequency, with no wasted flops:
//  * A = R_m as stored, [k][2r + {re, im}] (16-bit, K-major: the interleaved
//    complex row is a real row of length K' = 2 r_pad);
//  * B = the real 2x2 embedding of the field spectrum, K-major:
//        B[2f][2r] = Nr, B[2f][2r+1] = -Ni, B[2f+1][2r] = Ni, B[2f+1][2r+1] = Nr,
//    written directly by the forward-transform epilogue;
//  * D[k][2f] = Re S, D[k][2f+1] = Im S (FP32 accumulators in TMEM).
// Precision forms (the field is split into 16-bit parts every iteration):
//  * 16-bit R (BF16 or FP16):  D = R B_hi + R B_lo;
//  * split BF16 R (hi + lo):   D = R_hi B_hi + R_hi B_lo + R_lo B_hi
//    (about 16 significant bits per operand);
//  * 3-way split BF16 (hi + mid + lo for R and the field):
//    D = hh + hm + mh + hl + lh + mm, the six products down to 2^-16 of the
//    leading term (about 24 significant bits, FP32-like);
//  * scaled FP16 split (hi + lo, each operand scaled by a power of two into
//    FP16's normal range, mk_quant.cu): D = hh + hl + lh, about 22 significant
//    bits per operand; the epilogue divides the scales out.
//
// Kernel: persistent, one CTA per SM, warp-specialised:
//  warp 0 lane 0 : TMA producer (3-D tensor maps [K', rows, frequency],
//                  128-byte swizzle, OOB rows zero-filled) into a ring of
//                  shared-memory stages (mbarrier full/empty pairs);
//  warp 1 lane 0 : MMA issuer (tcgen05.mma kind::f16, M = 128, N = BN,
//                  K = 16 per instruction, FP32 accumulate) into one of two
//                  TMEM accumulators; tcgen05.commit frees stages and
//                  signals the epilogue;
//  warps 2..5    : epilogue, one TMEM lane (= output row) per thread:
//                  tcgen05.ld -> scale by c -> complex stores to S.
// Tiles (frequency, 128-row block, N block; N block fastest, so that
// neighbouring CTAs share an R tile through L2) come from a global work
// counter: the producer takes each tile index and passes it to the MMA lane
// and the epilogue warps through a small mbarrier-guarded queue in shared
// memory; a tile index of -1 ends the work, and the last CTA to finish
// resets the counter.
// Accuracy: the tensor core's FP32 accumulation over a long K chain carries
// a rounding bias that, on cancelling sums, dominates the operand precision
// of the split forms.  With PROMOTE the MMAs of each 64-wide K block start a
// fresh accumulator (four TMEM buffers rotate, two for N tiles above 128
// columns) and the epilogue warps add
// each block's partial sums into FP32 registers with round-to-nearest adds.
// Every mbarrier wait is bounded; on time-out the CTA records an error word,
// drains its copies and MMAs, frees TMEM and returns.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "mk_internal.h"

namespace mk {

struct UmmaMaps {
  CUtensorMap a0, a1, a2, b0, b1, b2;
  int bn;
  int na;   // 1, 2 or 3 A operands (parts of R)
  int nb;   // 2 or 3 B operands (parts of the field embedding)
  int fmt;  // 1: bf16, 0: fp16
};

namespace {

constexpr int UM = 128;          // rows per tile (MMA M)
constexpr int UKB = 64;          // K elements per stage (128 bytes of 16-bit data)
constexpr int kThreads = 192;    // 2 control warps + 4 epilogue warps
constexpr int kMaxStages = 8;
constexpr int kSmemBudget = 200 * 1024;
constexpr uint32_t kSpin = 1u << 24;

struct UmmaParams {
  float2* S;
  int ns, F, nw, kblocks, mtiles, ntiles;
  int64_t s_stride;
  float c;
  int* err;
  unsigned* queue;  // [2]: next tile, finished CTAs (the last CTA resets both)
  const float* rsc;  // scaled FP16 split: [nw] scale of R_m, else null
  const float* nsc;  // [nw][F] scale of the field spectrum (with rsc)
};

constexpr int kTQ = 4;  // tile-index slots between the producer and the MMA and epilogue warps

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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpin; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand tile, rows of 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart (tile base 1024-aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B of the same
// 16-bit format (fmt 1 = BF16, 0 = FP16), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t make_idesc(int fmt, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(UM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x 16 / 32 consecutive 32-bit TMEM columns into registers (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN, int NA, int NB, int FMT, bool PROMOTE>
__global__ void __launch_bounds__(kThreads, 1)
umma_cgemm_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                  const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
                  const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2, UmmaParams P,
                  int stages) {
  constexpr int A_BYTES = UM * UKB * 2;
  constexpr int B_BYTES = BN * UKB * 2;
  constexpr int STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;
  // TMEM accumulators: two (one per tile, alternating) without promotion; with
  // promotion one per K block, four of them where TMEM's 512 columns allow, so
  // that the MMAs run up to three K blocks ahead of the epilogue's drain
  constexpr int NACC = PROMOTE && 4 * BN <= 512 ? 4 : 2;
  constexpr int TMEM_COLS = NACC * BN < 32 ? 32 : NACC * BN;
  constexpr uint32_t IDESC = make_idesc(FMT, BN);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t tfull[4];
  __shared__ __align__(8) uint64_t tempty[4];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ __align__(8) uint64_t tq_full[kTQ];   // tile index written
  __shared__ __align__(8) uint64_t tq_empty[kTQ];  // read by the MMA lane and the 4 epilogue warps
  __shared__ int tq[kTQ];                           // tile index, -1 ends the work
  __shared__ uint32_t tmem_slot;
  __shared__ float sfac[4][64];                     // per epilogue warp: output factors of the tile's columns

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ring = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int tiles_per_m = P.mtiles * P.ntiles;
  const int total_tiles = P.nw * tiles_per_m;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(smem_u32(&tfull[a]), 1);
      mbar_init(smem_u32(&tempty[a]), 4);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    for (int q = 0; q < kTQ; ++q) {
      mbar_init(smem_u32(&tq_full[q]), 1);
      mbar_init(smem_u32(&tq_empty[q]), 5);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      bool ok = true;
      uint32_t it = 0;
      // tiles come from a work counter, so SMs that run faster take more of them
      for (uint32_t tc = 0; ok; ++tc) {
        const int q = (int)(tc % kTQ);
        if (!mbar_wait(smem_u32(&tq_empty[q]), ((tc / kTQ) & 1u) ^ 1u)) {
          ok = false;
          break;
        }
        int tile = (int)atomicAdd(P.queue, 1u);
        if (tile >= total_tiles) tile = -1;
        tq[q] = tile;
        mbar_arrive(smem_u32(&tq_full[q]));
        if (tile < 0) break;
        const int m = tile / tiles_per_m;
        const int rem = tile - m * tiles_per_m;
        const int mt = rem / P.ntiles, nt = rem - (rem / P.ntiles) * P.ntiles;
        for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)stages);
          const uint32_t ph = (it / (uint32_t)stages) & 1u;
          if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t base = ring + (uint32_t)s * STAGE_BYTES;
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(fb, STAGE_BYTES);
          tma_load_3d(base, &tmA0, kb * UKB, mt * UM, m, fb);
          if (NA >= 2) tma_load_3d(base + A_BYTES, &tmA1, kb * UKB, mt * UM, m, fb);
          if (NA >= 3) tma_load_3d(base + 2 * A_BYTES, &tmA2, kb * UKB, mt * UM, m, fb);
          tma_load_3d(base + NA * A_BYTES, &tmB0, kb * UKB, nt * BN, m, fb);
          tma_load_3d(base + NA * A_BYTES + B_BYTES, &tmB1, kb * UKB, nt * BN, m, fb);
          if (NB >= 3) tma_load_3d(base + NA * A_BYTES + 2 * B_BYTES, &tmB2, kb * UKB, nt * BN, m, fb);
        }
      }
      // no copy may be in flight when the CTA exits
      const uint32_t lo = it > (uint32_t)stages ? it - (uint32_t)stages : 0u;
      for (uint32_t q = lo; q < it; ++q)
        if (!mbar_wait(smem_u32(&full_bar[q % (uint32_t)stages]), (q / (uint32_t)stages) & 1u)) ok = false;
      if (!ok && P.err) atomicExch(P.err, 11);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      bool ok = true;
      uint32_t it = 0;
      for (uint32_t tc = 0; ok; ++tc) {
        const int q = (int)(tc % kTQ);
        if (!mbar_wait(smem_u32(&tq_full[q]), (tc / kTQ) & 1u)) {
          ok = false;
          break;
        }
        const int tile = tq[q];
        mbar_arrive(smem_u32(&tq_empty[q]));
        if (tile < 0) break;
        uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
        if (!PROMOTE) {
          if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
          if (PROMOTE) {  // one fresh accumulator per K block, buffers alternate
            acc = it % NACC;
            aph = (it / NACC) & 1u;
            if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1u)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t d = tmem_base + acc * BN;
          const int s = (int)(it % (uint32_t)stages);
          const uint32_t ph = (it / (uint32_t)stages) & 1u;
          if (!mbar_wait(smem_u32(&full_bar[s]), ph)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = ring + (uint32_t)s * STAGE_BYTES;
          const bool fresh = PROMOTE || kb == 0;
#pragma unroll
          for (int k4 = 0; k4 < UKB / 16; ++k4) {
            const uint64_t a0 = sw128_desc(base + k4 * 32);
            const uint64_t b0 = sw128_desc(base + NA * A_BYTES + k4 * 32);
            const uint64_t b1 = sw128_desc(base + NA * A_BYTES + B_BYTES + k4 * 32);
            umma(d, a0, b0, IDESC, (fresh && k4 == 0) ? 0u : 1u);  // hi * hi
            umma(d, a0, b1, IDESC, 1u);                             // hi * (lo | mid)
            if (NA >= 2) {
              const uint64_t a1 = sw128_desc(base + A_BYTES + k4 * 32);
              umma(d, a1, b0, IDESC, 1u);                           // (lo | mid) * hi
              if (NA >= 3) {
                const uint64_t a2 = sw128_desc(base + 2 * A_BYTES + k4 * 32);
                const uint64_t b2 = sw128_desc(base + NA * A_BYTES + 2 * B_BYTES + k4 * 32);
                umma(d, a0, b2, IDESC, 1u);                         // hi * lo
                umma(d, a2, b0, IDESC, 1u);                         // lo * hi
                umma(d, a1, b1, IDESC, 1u);                         // mid * mid
              }
            }
          }
          umma_commit(smem_u32(&empty_bar[s]));
          if (PROMOTE) umma_commit(smem_u32(&tfull[acc]));
        }
        if (!ok) break;
        if (!PROMOTE) umma_commit(smem_u32(&tfull[acc]));
      }
      // every MMA issued by this CTA has completed before TMEM is released
      umma_commit(smem_u32(&drain_bar));
      if (!mbar_wait(smem_u32(&drain_bar), 0u)) ok = false;
      if (!ok && P.err) atomicExch(P.err, 12);
    }
  } else {  // -------------------------------------------------------------- epilogue
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    uint32_t it = 0;
    for (uint32_t tc = 0;; ++tc) {
      const int q = (int)(tc % kTQ);
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tq_full[q]), (tc / kTQ) & 1u))) {
        if (lane == 0 && P.err) atomicExch(P.err, 14);
        break;
      }
      const int tile = tq[q];
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tq_empty[q]));
      if (tile < 0) break;
      const int m = tile / tiles_per_m;
      const int rem = tile - m * tiles_per_m;
      const int mt = rem / P.ntiles, nt = rem - (rem / P.ntiles) * P.ntiles;
      const int row = mt * UM + quad * 32 + lane;
      float2* scol = P.S + (int64_t)m * P.s_stride + row;  // S[m][f * ns + row]: lanes write consecutive rows
      if (PROMOTE) {
        float accv[BN];
#pragma unroll
        for (int i = 0; i < BN; ++i) accv[i] = 0.f;
        // scaled operands: the scales of this tile's columns are loaded now and
        // used after the K loop (their latency hides behind it)
        const int f0 = nt * BN / 2;
        float rs = 1.f, n0 = 1.f, n1 = 1.f;
        if (P.rsc) {
          rs = __ldg(P.rsc + m);
          if (lane < BN / 2 && f0 + lane < P.F) n0 = __ldg(P.nsc + (int64_t)m * P.F + f0 + lane);
          if (lane + 32 < BN / 2 && f0 + lane + 32 < P.F) n1 = __ldg(P.nsc + (int64_t)m * P.F + f0 + lane + 32);
        }
        bool ok = true;
        for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
          const uint32_t buf = it % NACC, ph = (it / NACC) & 1u;
          ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[buf]), ph));
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int ch = 0; ch < BN / 16; ++ch) {
            float v[16];
            tmem_ld16(tmem_base + lane_base + buf * BN + ch * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) accv[ch * 16 + i] += v[i];
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
        }
        if (!ok) {
          if (lane == 0 && P.err) atomicExch(P.err, 13);
          break;
        }
        if (P.rsc) {  // the operands were scaled by powers of two: c / (scale of R_m x scale of column)
          sfac[quad][lane] = P.c / (rs * n0);
          sfac[quad][lane + 32] = P.c / (rs * n1);
          __syncwarp();
        }
        if (row < P.ns) {
          if (P.rsc) {
#pragma unroll
            for (int j = 0; j < BN / 2; ++j)
              if (f0 + j < P.F) {
                const float q = sfac[quad][j];
                scol[(int64_t)(f0 + j) * P.ns] = make_float2(q * accv[2 * j], q * accv[2 * j + 1]);
              }
          } else {
#pragma unroll
            for (int j = 0; j < BN / 2; ++j)
              if (f0 + j < P.F)
                scol[(int64_t)(f0 + j) * P.ns] = make_float2(P.c * accv[2 * j], P.c * accv[2 * j + 1]);
          }
        }
        __syncwarp();  // sfac is rewritten by the next tile
        continue;
      }
      const uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), aph));
      if (!ok) {
        if (lane == 0 && P.err) atomicExch(P.err, 13);
        break;
      }
      tc_fence_after();
#pragma unroll 1
      for (int ch = 0; ch < BN / 16; ++ch) {
        float v[16];
        tmem_ld16(tmem_base + lane_base + acc * BN + ch * 16, v);
        if (row < P.ns) {
          const int f0 = (nt * BN + ch * 16) / 2;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (f0 + j < P.F) scol[(int64_t)(f0 + j) * P.ns] = make_float2(P.c * v[2 * j], P.c * v[2 * j + 1]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0) {  // the last CTA to finish resets the work counters
    __threadfence();
    if (atomicAdd(P.queue + 1, 1u) == gridDim.x - 1) {
      atomicExch(P.queue, 0u);
      atomicExch(P.queue + 1, 0u);
    }
  }
}

template <int BN, int NA, int NB>
int stages_for() {
  const int stage = NA * UM * UKB * 2 + NB * BN * UKB * 2;
  int st = (kSmemBudget - 1024) / stage;
  return st > kMaxStages ? kMaxStages : st;
}

template <int BN, int NA, int NB, int FMT, bool PROMOTE>
cudaError_t launch_bn(const SurveyDev& s, const UmmaMaps& mp, cudaStream_t st, int num_sms) {
  const int stages = stages_for<BN, NA, NB>();
  const int stage = NA * UM * UKB * 2 + NB * BN * UKB * 2;
  const size_t smem = (size_t)stages * stage + 1024;
  UmmaParams P;
  P.S = s.S;
  P.ns = s.ns;
  P.F = s.F;
  P.nw = s.nw;
  P.kblocks = (2 * s.r_pad) / UKB;
  P.mtiles = (s.ns + UM - 1) / UM;
  P.ntiles = (2 * s.F + BN - 1) / BN;
  P.s_stride = s.s_stride;
  P.c = s.c;
  P.err = s.err;
  P.queue = s.counter + 4;
  P.rsc = s.rsc;
  P.nsc = s.nsc;
  const int64_t tiles = (int64_t)P.nw * P.mtiles * P.ntiles;
  const int grid = (int)(tiles < num_sms ? tiles : num_sms);
  umma_cgemm_kernel<BN, NA, NB, FMT, PROMOTE><<<grid, kThreads, smem, st>>>(mp.a0, mp.a1, mp.a2, mp.b0, mp.b1, mp.b2, P,
                                                                    stages);
  return cudaGetLastError();
}

template <int BN, int NA, int NB, int FMT, bool PROMOTE>
cudaError_t set_attr_bn() {
  const int stage = NA * UM * UKB * 2 + NB * BN * UKB * 2;
  const size_t smem = (size_t)stages_for<BN, NA, NB>() * stage + 1024;
  return cudaFuncSetAttribute(umma_cgemm_kernel<BN, NA, NB, FMT, PROMOTE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int NA, int NB, int FMT, bool PROMOTE>
cudaError_t set_attr_na() {
  cudaError_t e;
  if ((e = set_attr_bn<16, NA, NB, FMT, PROMOTE>()) != cudaSuccess) return e;
  if ((e = set_attr_bn<32, NA, NB, FMT, PROMOTE>()) != cudaSuccess) return e;
  if ((e = set_attr_bn<64, NA, NB, FMT, PROMOTE>()) != cudaSuccess) return e;
  return set_attr_bn<128, NA, NB, FMT, PROMOTE>();
}

template <int NA, int NB, int FMT, bool PROMOTE>
cudaError_t launch_na(const SurveyDev& s, const UmmaMaps& mp, cudaStream_t st, int num_sms) {
  switch (mp.bn) {
    case 16: return launch_bn<16, NA, NB, FMT, PROMOTE>(s, mp, st, num_sms);
    case 32: return launch_bn<32, NA, NB, FMT, PROMOTE>(s, mp, st, num_sms);
    case 64: return launch_bn<64, NA, NB, FMT, PROMOTE>(s, mp, st, num_sms);
    default: return launch_bn<128, NA, NB, FMT, PROMOTE>(s, mp, st, num_sms);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D map over [K' = 2 r_pad][rows][nw] 16-bit elements, box [64][box_rows][1].
bool encode_map(CUtensorMap* tm, const void* base, int kprime, int rows, int nw, int box_rows, int fmt) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)kprime, (cuuint64_t)rows, (cuuint64_t)nw};
  const cuuint64_t strides[2] = {(cuuint64_t)kprime * 2, (cuuint64_t)kprime * 2 * rows};
  const cuuint32_t box[3] = {(cuuint32_t)UKB, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(tm, fmt ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

// Shared-memory attributes of every instantiation (once per device, before
// any launch, so that launches can be captured into graphs).
cudaError_t umma_prepare() {
  cudaError_t e;
  if ((e = set_attr_na<3, 3, 1, true>()) != cudaSuccess) return e;
  if ((e = set_attr_na<2, 2, 1, true>()) != cudaSuccess) return e;
  if ((e = set_attr_na<2, 2, 0, true>()) != cudaSuccess) return e;
  if ((e = set_attr_na<1, 2, 1, false>()) != cudaSuccess) return e;
  return set_attr_na<1, 2, 0, false>();
}

int umma_bn(int F) {
  const int n = 2 * F;
  if (n <= 16) return 16;
  if (n <= 32) return 32;
  if (n <= 64) return 64;
  return 128;
}

UmmaMaps* umma_create(const SurveyDev& s) {
  UmmaMaps* mp = new UmmaMaps();
  mp->bn = umma_bn(s.F);
  mp->na = (s.rprec == 3 || s.rprec == 5) ? 2 : (s.rprec == 4 ? 3 : 1);
  mp->nb = s.rprec == 4 ? 3 : 2;
  mp->fmt = (s.rprec == 2 || s.rprec == 5) ? 0 : 1;
  const int kp = 2 * s.r_pad;
  bool ok = encode_map(&mp->a0, s.Rq0, kp, s.ns, s.nw, UM, mp->fmt) &&
            encode_map(&mp->a1, mp->na >= 2 ? s.Rq1 : s.Rq0, kp, s.ns, s.nw, UM, mp->fmt) &&
            encode_map(&mp->a2, mp->na >= 3 ? s.Rq2 : s.Rq0, kp, s.ns, s.nw, UM, mp->fmt) &&
            encode_map(&mp->b0, s.Bq0, kp, 2 * s.F, s.nw, mp->bn, mp->fmt) &&
            encode_map(&mp->b1, s.Bq1, kp, 2 * s.F, s.nw, mp->bn, mp->fmt) &&
            encode_map(&mp->b2, mp->nb >= 3 ? s.Bq2 : s.Bq1, kp, 2 * s.F, s.nw, mp->bn, mp->fmt);
  if (!ok) {
    delete mp;
    return nullptr;
  }
  return mp;
}

void umma_destroy(UmmaMaps* mp) { delete mp; }

bool umma_set_bn(UmmaMaps* mp, const SurveyDev& s, int bn) {
  if (!mp || (bn != 16 && bn != 32 && bn != 64 && bn != 128)) return false;
  const int kp = 2 * s.r_pad;
  UmmaMaps t = *mp;
  t.bn = bn;
  const bool ok = encode_map(&t.b0, s.Bq0, kp, 2 * s.F, s.nw, bn, t.fmt) &&
                  encode_map(&t.b1, s.Bq1, kp, 2 * s.F, s.nw, bn, t.fmt) &&
                  encode_map(&t.b2, t.nb >= 3 ? s.Bq2 : s.Bq1, kp, 2 * s.F, s.nw, bn, t.fmt);
  if (ok) *mp = t;
  return ok;
}

int umma_get_bn(const UmmaMaps* mp) { return mp ? mp->bn : 0; }

cudaError_t launch_umma(const SurveyDev& s, const UmmaMaps* mp, cudaStream_t st, int num_sms) {
  if (!mp) return cudaErrorInvalidValue;
  // the split forms target FP32-level accuracy: they promote per K block
  if (mp->na == 3) return launch_na<3, 3, 1, true>(s, *mp, st, num_sms);
  if (mp->na == 2 && mp->fmt == 0) return launch_na<2, 2, 0, true>(s, *mp, st, num_sms);  // scaled FP16 split
  if (mp->na == 2) return launch_na<2, 2, 1, true>(s, *mp, st, num_sms);
  if (mp->fmt == 1) return launch_na<1, 2, 1, false>(s, *mp, st, num_sms);
  return launch_na<1, 2, 0, false>(s, *mp, st, num_sms);
}

}  // namespace mk
