// Multi-right-hand-side operator products Y = M X (M = L or R, X = nrhs complex vectors).
//
// Three engines:
//  * k_tc_gemm: tensor cores (tcgen05.mma, kind::tf32 on the FP32 operator or kind::f16 on its
//    BF16 copy) for the inner Krylov products of mixed-precision refinement. The complex
//    product is a real GEMM: row i of the complex64 operator read as 2*ld reals
//    [Re M_i0, Im M_i0, Re M_i1, ...] times the real matrix B whose column c < P is
//    (Re x_c0, -Im x_c0, Re x_c1, ...) and column P + c is (Im x_c0, Re x_c0, ...); then
//    Y[i][c] = Re (M x_c)_i and Y[i][P + c] = Im (M x_c)_i. At tens of right-hand sides this is
//    far below the tensor ridge, so the kernel is built to stream the operator at HBM speed:
//    a persistent grid (one CTA per SM) splits the (128-row tile, K block) iteration space into
//    equal contiguous ranges (stream-K), so every SM streams the same number of operator bytes
//    whatever the tile count. One thread issues TMA copies (128-byte swizzle) of the A tile and
//    of B into a ring of up to eight shared-memory stages guarded by mbarriers; one thread
//    issues the MMAs into one of two TMEM accumulators (128 lanes x N columns, FP32), switching
//    at each new row tile, so four epilogue warps drain the previous tile's accumulator
//    (tcgen05.ld) while the next one fills. Each CTA writes one partial tile per row tile it
//    touched; k_tc_reduce adds a tile's partials in K order in FP64 (a fixed order, so results
//    do not depend on timing).
//  * k_tc_gemm_x6: the products that must carry FP32 accuracy (refinement residuals, the plain
//    multi-RHS solve) with L from 8 RHS up, on tensor cores: L and X split exactly into three
//    BF16 pieces, the six piece products with i + j <= 4, the accumulator drained after every
//    K block into float-float sums.
//  * k_cgemm_sk: FP32 CUDA-core complex GEMM (persistent stream-K, up to 64 RHS per tile, FP32
//    products summed in FP32 over 128 terms, then carried as float-float pairs) for the other
//    FP32-accurate products: the right-hand side R G and products with fewer than 8 RHS.
//    k_cgemm_fp32 (fixed tiles, FP64 carries) computes the same product for operators whose
//    leading dimension is odd.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets an error flag, the kernel
// skips its remaining work, waits (bounded) for its own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <string>

#include "internal.h"

namespace natbem {

// ------------------------------------------------------------------ PTX wrappers (sm_100+)
namespace {

constexpr int kTcRows = 128;         // M of the MMA (rows of the operator per tile)
constexpr int kTcMaxStages = 8;      // shared-memory ring (as many as fit, at most this)
constexpr int kTcThreads = 192;      // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kTcMinBlocks = 4;      // K blocks per CTA at least (small products use fewer CTAs)
constexpr uint32_t kTcSmemMax = 227 * 1024 - 256;  // dynamic shared memory (static needs a little)
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: false if the phase did not complete within timeout_ns (default about two
// seconds) or kSpinLimit polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint64_t timeout_ns = 2000000000ull) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 1023u) == 1023u && globaltimer_ns() - t0 > timeout_ns) return false;
  }
  return false;
}

// The same wait, giving up early once *abort is set by another role of the block.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, const volatile int* abort,
                                                   uint64_t timeout_ns = 2000000000ull) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && (*abort || globaltimer_ns() - t0 > timeout_ns)) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B formats (TF32 = 2 for kind::tf32, BF16 = 1
// for kind::f16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t n, uint32_t m) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

template <int kKind>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if (kKind == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  // the loaded registers pass through the wait, so no use of them is scheduled before it
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// 16 columns of this warp's 32 TMEM lanes (32x32b.x16), waited for before use
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
      :
      : "memory");
}

}  // namespace

// Partial products of the stream-K partition: the iteration space is the m_tiles x nkb grid of
// (row tile, K block) pairs in row-major order, T = m_tiles * nkb, a row tile being kTiles x 128
// rows; CTA c takes the pairs [c per, min((c + 1) per, T)). Each contiguous run of one row tile
// is a segment; segment j of CTA c goes to partial slot c * msp + j (msp: most segments a CTA
// can have), stored column by column: part[slot][col][row in tile]. With kTiles = 2 one B stage
// feeds two M = 128 MMAs (two accumulators), halving B's share of the shared-memory traffic.
// A: n x Kt (tensor map ta, box BK x 128 kTiles), B: Ng x Kt
// (tensor map tb, box BK x Ng). kKind 0: TF32 (FP32 storage, BK = 32), 1: BF16, 2: FP16 (the
// row-scaled copy; BK = 64); either way a stage row is 128 bytes and one MMA covers 32 bytes
// of K, four per stage.
template <int kKind, int kTiles>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int n,
          int nkb, int per, int msp, int Ng, int stages, float* __restrict__ part,
          int* __restrict__ err, const int* __restrict__ scal) {
  constexpr int BK = kKind == 0 ? 32 : 64;
  constexpr int TM = kTcRows * kTiles;
  if (scal && scal[1]) return;  // every right-hand side has converged
  const int m_tiles = (n + TM - 1) / TM;
  const int64_t T = (int64_t)m_tiles * nkb;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = min(T, t0 + per);
  if (t0 >= T) return;
  const int mt_first = (int)(t0 / nkb);
  const int nseg = (int)((t1 - 1) / nkb) - mt_first + 1;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment of the shared-memory address itself (the 128-byte swizzle atom)
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t a_bytes = TM * 128, b_bytes = (uint32_t)Ng * 128;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + stages * stage_bytes);
  uint64_t* full = bars;                     // [stages] TMA -> MMA
  uint64_t* empty = bars + kTcMaxStages;     // [stages] MMA -> TMA
  uint64_t* tfull = bars + 2 * kTcMaxStages; // [2] MMA -> epilogue: accumulators ready
  uint64_t* tempty = tfull + 2;              // [2] epilogue -> MMA: accumulators drained
  uint64_t* fin = tempty + 2;                // every MMA of the block complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;  // TMEM columns per accumulator (a power of two >= Ng)
  while ((int)ncols < Ng) ncols <<= 1;
  const uint32_t alloc_cols = 2 * kTiles * ncols;  // two buffers of kTiles accumulators

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < stages; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);
      mbar_init(smem_u32(&tempty[q]), 4);
    }
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(alloc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA copies of A tile (mt, kb) and of B's K block kb into the ring
    int issued = 0;
    for (int64_t t = t0; t < t1 && !s_abort; ++t) {
      const int it = (int)(t - t0);
      const int q = it % stages;
      const uint32_t ph = (uint32_t)(it / stages) & 1u;
      if (!mbar_wait_or_abort(smem_u32(&empty[q]), ph ^ 1u, &s_abort)) {
        atomicOr(err, 1);
        s_abort = 1;
        break;
      }
      const uint32_t sa = smem_u32(base + q * stage_bytes);
      const uint32_t fb = smem_u32(&full[q]);
      mbar_expect_tx(fb, stage_bytes);
      const int mt = (int)(t / nkb), kb = (int)(t % nkb);
      tma_load_2d(sa, &ta, kb * BK, mt * TM, fb);
      tma_load_2d(sa + a_bytes, &tb, kb * BK, 0, fb);
      issued = it + 1;
    }
    if (s_abort) {
      // let the copies already issued land before the block exits
      for (int it = max(0, issued - stages); it < issued; ++it)
        mbar_wait(smem_u32(&full[it % stages]), (uint32_t)(it / stages) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: kTiles accumulators per segment, alternating between the two TMEM buffers
    // operand formats: TF32 = 2 (kind::tf32); BF16 = 1, F16 = 0 (kind::f16)
    const uint32_t idesc = instr_desc(kKind == 0 ? 2u : kKind == 1 ? 1u : 0u, (uint32_t)Ng, (uint32_t)kTcRows);
    int seg = -1, mt_cur = -1;
    uint32_t acc = tmem;
    bool first = true;
    for (int64_t t = t0; t < t1 && !s_abort; ++t) {
      const int it = (int)(t - t0);
      const int mt = (int)(t / nkb);
      if (mt != mt_cur) {
        if (seg >= 0) mma_commit(smem_u32(&tfull[seg & 1]));
        ++seg;
        mt_cur = mt;
        if (!mbar_wait_or_abort(smem_u32(&tempty[seg & 1]), ((uint32_t)(seg >> 1) & 1u) ^ 1u, &s_abort)) {
          atomicOr(err, 8);
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        acc = tmem + (uint32_t)(seg & 1) * kTiles * ncols;
        first = true;
      }
      const int q = it % stages;
      const uint32_t ph = (uint32_t)(it / stages) & 1u;
      if (!mbar_wait_or_abort(smem_u32(&full[q]), ph, &s_abort)) {
        atomicOr(err, 2);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + q * stage_bytes);
      const uint64_t db = smem_desc(sa + a_bytes);
#pragma unroll
      for (int u = 0; u < kTiles; ++u) {
        const uint64_t da = smem_desc(sa + u * kTcRows * 128);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)  // 32 bytes of K per MMA: +2 in the 16-byte address field
          mma<kKind>(acc + u * ncols, da + 2 * kk, db + 2 * kk, idesc, (!first || kk > 0) ? 1u : 0u);
      }
      first = false;
      mma_commit(smem_u32(&empty[q]));
    }
    if (seg >= 0) mma_commit(smem_u32(&tfull[seg & 1]));
    mma_commit(smem_u32(fin));
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of each accumulator, i.e. rows
    // u 128 + 32 (w % 4) + lane of the row tile
    const int quarter = warp & 3;
    for (int j = 0; j < nseg; ++j) {
      const int b = j & 1;
      if (!mbar_wait_or_abort(smem_u32(&tfull[b]), (uint32_t)(j >> 1) & 1u, &s_abort)) {
        if (lane == 0) atomicOr(err, 4);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* out = part + ((size_t)blockIdx.x * msp + j) * (size_t)Ng * TM;
#pragma unroll
      for (int u = 0; u < kTiles; ++u) {
        const int r = u * kTcRows + quarter * 32 + lane;
        for (int c0 = 0; c0 < Ng; c0 += 32) {  // Ng is a multiple of 32
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTiles + u) * ncols + (uint32_t)c0, v);
          if (!s_abort) {
#pragma unroll
            for (int q = 0; q < 32; ++q) out[(size_t)(c0 + q) * TM + r] = __uint_as_float(v[q]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
    }
  }
  __syncwarp();
  __syncthreads();
  if (warp == 0) {
    // every MMA of the block has completed before the accumulators are released (bounded)
    if (!mbar_wait(smem_u32(fin), 0) && lane == 0) atomicOr(err, 16);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(alloc_cols));
  }
}

// hi + lo += c, exactly up to the rounding of lo (TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float c) {
  const float s = __fadd_rn(hi, c);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(c, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// ------------------------------------------ FP32-accurate product on tensor cores (x6)
// The operator and the right-hand sides are split exactly into three BF16 pieces each:
// a1 = bf16(a), a2 = bf16(a - a1), a3 = bf16(a - a1 - a2), every difference exact in FP32, so
// a = a1 + a2 + a3 to within 2^-24 |a| or so. The product sums the six piece products with
// i + j <= 4 (the three omitted ones lie below 2^-24 of a x); a BF16 x BF16 product is exact
// in the FP32 accumulator. The accumulator is drained after every K block (64 real terms,
// 24 MMAs) into FP32 registers: the tensor core's FP32 accumulation error grows linearly with
// the run length (measured at 20480 rows, 64 RHS, per column against an FP64 product: 1.1e-7,
// 4.3e-7, 9.2e-7, 1.8e-6 for runs of 1, 2, 4, 8 K blocks, the mark of a biased, truncating
// accumulation, where round-to-nearest errors would grow as the square root). With one-block
// runs the product is more accurate than the CUDA-core GEMM (3.3e-7) for 10% more time than
// four-block runs. Each run is added to a float-float pair per (row, column) by TwoSum, so
// the register sums add no rounding of their own. Eight epilogue warps, two per TMEM lane
// quarter, each hold half of the columns.
constexpr int kX6Drain = 1;  // K blocks per accumulator run
constexpr int kX6Threads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue

__device__ __forceinline__ void split3(float a, __nv_bfloat16& p1, __nv_bfloat16& p2, __nv_bfloat16& p3) {
  p1 = __float2bfloat16_rn(a);
  const float r1 = __fsub_rn(a, __bfloat162float(p1));   // exact
  p2 = __float2bfloat16_rn(r1);
  const float r2 = __fsub_rn(r1, __bfloat162float(p2));  // exact
  p3 = __float2bfloat16_rn(r2);
}

// The three pieces of `count` floats (a multiple of 4) into planes `plane` elements apart.
__global__ void k_split3(const float4* __restrict__ a, int64_t count4, __nv_bfloat16* __restrict__ out,
                         int64_t plane) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = a[i];
    __nv_bfloat16 p[3][4];
    split3(v.x, p[0][0], p[1][0], p[2][0]);
    split3(v.y, p[0][1], p[1][1], p[2][1]);
    split3(v.z, p[0][2], p[1][2], p[2][2]);
    split3(v.w, p[0][3], p[1][3], p[2][3]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uint2 w;
      w.x = (uint32_t)__bfloat16_as_ushort(p[q][0]) | ((uint32_t)__bfloat16_as_ushort(p[q][1]) << 16);
      w.y = (uint32_t)__bfloat16_as_ushort(p[q][2]) | ((uint32_t)__bfloat16_as_ushort(p[q][3]) << 16);
      *reinterpret_cast<uint2*>(out + q * plane + 4 * i) = w;
    }
  }
}

// B of the x6 product: the layout of k_pack_b's BF16 form, one plane per piece.
__global__ void k_pack_b3(const float2* __restrict__ X, int ld, int nrhs, int P, __nv_bfloat16* __restrict__ B,
                          int64_t plane, const int* __restrict__ scal) {
  if (scal && scal[1]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over P * ld
  if (i >= (int64_t)P * ld) return;
  const int c = (int)(i / ld), j = (int)(i % ld);
  const float2 x = c < nrhs ? X[(size_t)c * ld + j] : make_float2(0.f, 0.f);
  const size_t Kt = 2 * (size_t)ld;
  const float v[4] = {x.x, -x.y, x.y, x.x};
  const size_t at[4] = {(size_t)c * Kt + 2 * j, (size_t)c * Kt + 2 * j + 1, (size_t)(P + c) * Kt + 2 * j,
                        (size_t)(P + c) * Kt + 2 * j + 1};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __nv_bfloat16 p1, p2, p3;
    split3(v[e], p1, p2, p3);
    B[at[e]] = p1;
    B[plane + at[e]] = p2;
    B[2 * plane + at[e]] = p3;
  }
}

// The stream-K partition of k_tc_gemm with one 128-row tile per stage and K blocks of 64;
// each stage holds the three A pieces then the three B pieces. The MMA thread switches TMEM
// buffer at every accumulator run (kX6Drain K blocks, or the end of a segment); the epilogue adds
// each run into float-float register sums (Ng <= 128 columns per row, half of them per warp)
// and writes the segment's partial tile (hi + lo in FP32) at its end.
__global__ void __launch_bounds__(kX6Threads, 1)
k_tc_gemm_x6(const __grid_constant__ CUtensorMap ta1, const __grid_constant__ CUtensorMap ta2,
             const __grid_constant__ CUtensorMap ta3, const __grid_constant__ CUtensorMap tb1,
             const __grid_constant__ CUtensorMap tb2, const __grid_constant__ CUtensorMap tb3, int n,
             int nkb, int per, int msp, int Ng, int stages, float* __restrict__ part,
             int* __restrict__ err, const int* __restrict__ scal) {
  constexpr int BK = 64, TM = kTcRows;
  if (scal && scal[1]) return;
  const int m_tiles = (n + TM - 1) / TM;
  const int64_t T = (int64_t)m_tiles * nkb;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = min(T, t0 + per);
  if (t0 >= T) return;
  const int mt_first = (int)(t0 / nkb);
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t a_bytes = TM * 128, b_bytes = (uint32_t)Ng * 128;
  const uint32_t stage_bytes = 3 * (a_bytes + b_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + stages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kTcMaxStages;
  uint64_t* tfull = bars + 2 * kTcMaxStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* fin = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;
  while ((int)ncols < Ng) ncols <<= 1;
  const uint32_t alloc_cols = 2 * ncols;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < stages; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);
      mbar_init(smem_u32(&tempty[q]), 8);
    }
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(alloc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: the three A pieces of tile (mt, kb) and the three B pieces of K block kb
    int issued = 0;
    for (int64_t t = t0; t < t1 && !s_abort; ++t) {
      const int it = (int)(t - t0);
      const int q = it % stages;
      const uint32_t ph = (uint32_t)(it / stages) & 1u;
      if (!mbar_wait_or_abort(smem_u32(&empty[q]), ph ^ 1u, &s_abort)) {
        atomicOr(err, 1);
        s_abort = 1;
        break;
      }
      const uint32_t sa = smem_u32(base + q * stage_bytes);
      const uint32_t fb = smem_u32(&full[q]);
      mbar_expect_tx(fb, stage_bytes);
      const int mt = (int)(t / nkb), kb = (int)(t % nkb);
      tma_load_2d(sa, &ta1, kb * BK, mt * TM, fb);
      tma_load_2d(sa + a_bytes, &ta2, kb * BK, mt * TM, fb);
      tma_load_2d(sa + 2 * a_bytes, &ta3, kb * BK, mt * TM, fb);
      tma_load_2d(sa + 3 * a_bytes, &tb1, kb * BK, 0, fb);
      tma_load_2d(sa + 3 * a_bytes + b_bytes, &tb2, kb * BK, 0, fb);
      tma_load_2d(sa + 3 * a_bytes + 2 * b_bytes, &tb3, kb * BK, 0, fb);
      issued = it + 1;
    }
    if (s_abort) {
      for (int it = max(0, issued - stages); it < issued; ++it)
        mbar_wait(smem_u32(&full[it % stages]), (uint32_t)(it / stages) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: piece pairs (A i, B j), smallest first
    const uint32_t idesc = instr_desc(1u, (uint32_t)Ng, (uint32_t)kTcRows);
    constexpr int kPa[6] = {0, 1, 2, 0, 1, 0}, kPb[6] = {2, 1, 0, 1, 0, 0};
    int chunk = -1;
    uint32_t acc = tmem;
    bool first = true;
    for (int64_t t = t0; t < t1 && !s_abort; ++t) {
      const int it = (int)(t - t0);
      const int kb = (int)(t % nkb);
      if (t == t0 || kb % kX6Drain == 0) {  // a new drain chunk (a new segment starts at kb = 0)
        if (chunk >= 0) mma_commit(smem_u32(&tfull[chunk & 1]));
        ++chunk;
        if (!mbar_wait_or_abort(smem_u32(&tempty[chunk & 1]), ((uint32_t)(chunk >> 1) & 1u) ^ 1u, &s_abort)) {
          atomicOr(err, 8);
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        acc = tmem + (uint32_t)(chunk & 1) * ncols;
        first = true;
      }
      const int q = it % stages;
      const uint32_t ph = (uint32_t)(it / stages) & 1u;
      if (!mbar_wait_or_abort(smem_u32(&full[q]), ph, &s_abort)) {
        atomicOr(err, 2);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + q * stage_bytes);
#pragma unroll
      for (int pr = 0; pr < 6; ++pr) {
        const uint64_t da = smem_desc(sa + kPa[pr] * a_bytes);
        const uint64_t db = smem_desc(sa + 3 * a_bytes + kPb[pr] * b_bytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma<1>(acc, da + 2 * kk, db + 2 * kk, idesc, (first && pr == 0 && kk == 0) ? 0u : 1u);
      }
      first = false;
      mma_commit(smem_u32(&empty[q]));
    }
    if (chunk >= 0) mma_commit(smem_u32(&tfull[chunk & 1]));
    mma_commit(smem_u32(fin));
  } else if (warp >= 2) {
    // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (rows of the tile), columns
    // 64 h .. 64 h + 63 with h = (w - 2) / 4, into float-float sums (hi, lo)
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = quarter * 32 + lane;
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) hi[c] = lo[c] = 0.f;
    int chunk = -1;
    for (int64_t t = t0; t < t1; ++t) {
      const int kb = (int)(t % nkb);
      const bool seg_end = t + 1 == t1 || kb + 1 == nkb;
      if (!seg_end && (kb + 1) % kX6Drain != 0) continue;  // not the last K block of a chunk
      ++chunk;
      const int b = chunk & 1;
      if (!mbar_wait_or_abort(smem_u32(&tfull[b]), (uint32_t)(chunk >> 1) & 1u, &s_abort)) {
        if (lane == 0) atomicOr(err, 4);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        const int col = 64 * half + c0;
        if (col < Ng) {  // Ng is a multiple of 32: whole 16-column loads
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * ncols + (uint32_t)col, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) two_sum_acc(hi[c0 + q], lo[c0 + q], __uint_as_float(v[q]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
      if (seg_end) {
        const int j = (int)(t / nkb) - mt_first;
        float* out = part + ((size_t)blockIdx.x * msp + j) * (size_t)Ng * TM;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 32) {
          const int col = 64 * half + c0;
          if (col < Ng && !s_abort) {
#pragma unroll
            for (int q = 0; q < 32; ++q) out[(size_t)(col + q) * TM + r] = __fadd_rn(hi[c0 + q], lo[c0 + q]);
          }
#pragma unroll
          for (int q = 0; q < 32; ++q) hi[c0 + q] = lo[c0 + q] = 0.f;
        }
      }
    }
  }
  __syncwarp();
  __syncthreads();
  if (warp == 0) {
    if (!mbar_wait(smem_u32(fin), 0) && lane == 0) atomicOr(err, 16);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(alloc_cols));
  }
}

// B for the tensor-core product from nrhs complex64 vectors (x_c at X + c * ld), P = nrhs
// rounded up to 16 (so the epilogue reads whole 32-column TMEM chunks): rows c < P
// (Re, -Im) pairs, rows P + c (Im, Re) pairs; rows of absent RHS are zero. TF32: FP32 storage;
// BF16 / FP16: round to nearest (the Krylov vectors have unit norm, inside FP16's range).
template <int kKind>
__global__ void k_pack_b(const float2* __restrict__ X, int ld, int nrhs, int P, void* __restrict__ B,
                         const int* __restrict__ scal) {
  if (scal && scal[1]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over P * ld
  if (i >= (int64_t)P * ld) return;
  const int c = (int)(i / ld), j = (int)(i % ld);
  const float2 x = c < nrhs ? X[(size_t)c * ld + j] : make_float2(0.f, 0.f);
  const size_t Kt = 2 * (size_t)ld;
  if (kKind == 0) {
    float* b = static_cast<float*>(B);
    b[(size_t)c * Kt + 2 * j] = x.x;
    b[(size_t)c * Kt + 2 * j + 1] = -x.y;
    b[(size_t)(P + c) * Kt + 2 * j] = x.y;
    b[(size_t)(P + c) * Kt + 2 * j + 1] = x.x;
  } else if (kKind == 1) {
    __nv_bfloat16* b = static_cast<__nv_bfloat16*>(B);
    b[(size_t)c * Kt + 2 * j] = __float2bfloat16_rn(x.x);
    b[(size_t)c * Kt + 2 * j + 1] = __float2bfloat16_rn(-x.y);
    b[(size_t)(P + c) * Kt + 2 * j] = __float2bfloat16_rn(x.y);
    b[(size_t)(P + c) * Kt + 2 * j + 1] = __float2bfloat16_rn(x.x);
  } else {
    __half* b = static_cast<__half*>(B);
    b[(size_t)c * Kt + 2 * j] = __float2half_rn(x.x);
    b[(size_t)c * Kt + 2 * j + 1] = __float2half_rn(-x.y);
    b[(size_t)(P + c) * Kt + 2 * j] = __float2half_rn(x.y);
    b[(size_t)(P + c) * Kt + 2 * j + 1] = __float2half_rn(x.x);
  }
}

// Y[c][row] (complex128, column c at Y + c * n) = the sum of the row tile's partial tiles in K
// order (the CTAs c_lo..c_hi that covered it, see k_tc_gemm; TM rows per tile), in FP64.
__global__ void k_tc_reduce(const float* __restrict__ part, int n, int TM, int Ng, int P, int nrhs,
                            int nkb, int per, int msp, double2* __restrict__ Y,
                            const int* __restrict__ done, const int* __restrict__ scal,
                            const float* __restrict__ rs) {
  if (scal && scal[1]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nrhs * n
  if (i >= (int64_t)nrhs * n) return;
  const int c = (int)(i / n), row = (int)(i % n);
  if (done && done[c]) return;
  const int mt = row / TM, r = row % TM;
  const int64_t first = (int64_t)mt * nkb, last = first + nkb - 1;
  const int c_lo = (int)(first / per), c_hi = (int)(last / per);
  double re = 0.0, im = 0.0;
  for (int cta = c_lo; cta <= c_hi; ++cta) {
    const int j = mt - (int)(((int64_t)cta * per) / nkb);  // the segment of this tile in CTA cta
    const float* p = part + ((size_t)cta * msp + j) * (size_t)Ng * TM;
    re += p[(size_t)c * TM + r];
    im += p[(size_t)(P + c) * TM + r];
  }
  const double sc = rs ? (double)rs[row] : 1.0;  // the FP16 copy's row scale (a power of two)
  Y[(size_t)c * n + row] = make_double2(re * sc, im * sc);
}

// ------------------------------------------------------------- FP32 CUDA-core complex GEMM
namespace {
constexpr int kGmRows = 64, kGmRhs = 32, kGmK = 32;  // block tile and K chunk (complex)
}

// Y[s][row] (complex128) = sum_j A[row][j] X[s][j] for s in the block's RHS tile; A is n x ld
// complex64, X holds nrhs vectors of ld complex64 (pad zero). 256 threads as 16 x 16: each
// thread 4 rows x 2 RHS. FP32 products summed in FP32 over 4 chunks (128 terms), then FP64.
__global__ void __launch_bounds__(256)
k_cgemm_fp32(const float2* __restrict__ A, int n, int ld, const float2* __restrict__ X, int nrhs,
             double2* __restrict__ Y, const int* __restrict__ done, const int* __restrict__ scal) {
  __shared__ float2 sA[kGmRows][kGmK + 1];
  if (scal && scal[1]) return;
  __shared__ float2 sX[kGmK][kGmRhs];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.x * kGmRows, s0 = blockIdx.y * kGmRhs;
  float ar[4][2], ai[4][2];
  double dr[4][2], di[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 2; ++q) ar[i][q] = ai[i][q] = 0.f, dr[i][q] = di[i][q] = 0.0;
  int chunk = 0;
  for (int k0 = 0; k0 < ld; k0 += kGmK, ++chunk) {
    // stage A (64 x 32) and X (32 x 32)
    for (int t = threadIdx.x; t < kGmRows * kGmK; t += 256) {
      const int r = t / kGmK, k = t % kGmK;
      const int row = r0 + r, col = k0 + k;
      sA[r][k] = (row < n && col < ld) ? A[(size_t)row * ld + col] : make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < kGmK * kGmRhs; t += 256) {
      const int s = t / kGmK, k = t % kGmK;
      const int rhs = s0 + s, col = k0 + k;
      sX[k][s] = (rhs < nrhs && col < ld) ? X[(size_t)rhs * ld + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGmK; ++k) {
      float2 a[4], x[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[ty * 4 + i][k];
#pragma unroll
      for (int q = 0; q < 2; ++q) x[q] = sX[k][tx * 2 + q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          ar[i][q] = fmaf(a[i].x, x[q].x, fmaf(-a[i].y, x[q].y, ar[i][q]));
          ai[i][q] = fmaf(a[i].x, x[q].y, fmaf(a[i].y, x[q].x, ai[i][q]));
        }
    }
    __syncthreads();
    if ((chunk & 3) == 3 || k0 + kGmK >= ld) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          dr[i][q] += ar[i][q];
          di[i][q] += ai[i][q];
          ar[i][q] = ai[i][q] = 0.f;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int row = r0 + ty * 4 + i, rhs = s0 + tx * 2 + q;
      if (row < n && rhs < nrhs && !(done && done[rhs]))
        Y[(size_t)rhs * n + row] = make_double2(dr[i][q], di[i][q]);
    }
}

// ------------------------------------------- FP32 CUDA-core complex GEMM, stream-K form
// The same product Y = M X with FP32 products, organised for the FP32 pipe and for GB300's
// narrow FP64 pipe:
//  * 256 threads as RG = 256 / CG row groups x CG RHS groups; thread (rg, cg) holds rows
//    rg + RG i (i < 4) and RHS cg + CG q (q < TN): a block tile of BM = 4 RG rows x BN = CG TN
//    right-hand sides. A warp spans 32 / CG row groups and CG RHS groups, so its 16-byte
//    shared loads of A and of X each touch few distinct addresses (broadcasts); CG is chosen
//    from nrhs so that few columns of a tile are padding;
//  * K blocks of BK complex terms stream through a ring of shared-memory stages by 16-byte
//    cp.async copies (rows past n and RHS past nrhs are zero-filled);
//  * the FP32 sums are folded every 128 terms into a float-float pair by TwoSum (Knuth), so no
//    FP64 instruction runs inside the loop; a partial is hi + lo in FP64;
//  * persistent stream-K: the (row tile, RHS tile, K block) space is split into equal
//    contiguous ranges, one per CTA, so every SM does the same work whatever the tile count;
//    each CTA writes one FP64 partial tile per tile it touched, and k_cgemm_sk_reduce adds a
//    tile's partials in CTA order (fixed, so results do not depend on timing).
// K blocks past the leading dimension ld are zero-filled. ld must be even and A, X 16-byte
// aligned (every operator this library builds is); otherwise k_cgemm_fp32 runs.
namespace {
constexpr int kCgTerms = 128;   // FP32 terms summed before each float-float fold
constexpr int kCgMinBlocks = 8;  // K blocks per CTA at least

__host__ __device__ constexpr int cg_stage_bytes(int CG, int TN, int BK) {
  return (4 * (256 / CG) + CG * TN) * (BK + 2) * 8;
}
// ring depth: as many stages as fit (at most 4) beside MINB - 1 other CTAs on the SM
__host__ __device__ constexpr int cg_stages(int CG, int TN, int BK, int MINB) {
  return (MINB == 2 ? 113 * 1024 : 225 * 1024) / cg_stage_bytes(CG, TN, BK) < 4
             ? (MINB == 2 ? 113 * 1024 : 225 * 1024) / cg_stage_bytes(CG, TN, BK)
             : 4;
}

__device__ __forceinline__ void cg_copy16(float2* dst, const float2* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cg_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cg_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
}  // namespace

template <int CG, int TN, int BK, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_cgemm_sk(const float2* __restrict__ A, int n, int ld, const float2* __restrict__ X, int nrhs, int ntn,
           int nkb, int per, int msp, double2* __restrict__ part, const int* __restrict__ scal) {
  constexpr int RG = 256 / CG, BM = 4 * RG, BN = CG * TN;
  constexpr int kPitch = BK + 2;  // float2 per shared row: 16-byte loads of 8 rows hit 8 bank groups
  constexpr int kFlush = kCgTerms / BK;
  constexpr int S = cg_stages(CG, TN, BK, MINB);
  constexpr int kStage = (BM + BN) * kPitch;  // float2 per stage
  static_assert(S >= 2, "shared-memory ring too shallow");
  extern __shared__ float4 cg_smem[];
  float2* sm = reinterpret_cast<float2*>(cg_smem);
  if (scal && scal[1]) return;
  const int tid = threadIdx.x, cg = tid % CG, rg = tid / CG;
  const int64_t mt = (n + BM - 1) / BM;
  const int64_t T = mt * ntn * nkb;
  const int64_t u0 = (int64_t)blockIdx.x * per, u1 = min(T, u0 + per);
  if (u0 >= u1) return;
  const int64_t tile0 = u0 / nkb;

  auto load = [&](int st, int64_t u) {
    const int64_t tile = u / nkb;
    const int kb = (int)(u - tile * nkb);
    const int row0 = (int)(tile / ntn) * BM, rhs0 = (int)(tile % ntn) * BN, k0 = kb * BK;
    float2* sA = sm + st * kStage;
    float2* sX = sA + BM * kPitch;
    constexpr int kPieces = BK / 2;  // 16-byte pieces per row
#pragma unroll
    for (int e = tid; e < BM * kPieces; e += 256) {
      const int r = e / kPieces, c = (e % kPieces) * 2;
      const bool ok = row0 + r < n && k0 + c < ld;
      cg_copy16(sA + r * kPitch + c, ok ? A + (size_t)(row0 + r) * ld + k0 + c : A, ok);
    }
#pragma unroll
    for (int e = tid; e < BN * kPieces; e += 256) {
      const int r = e / kPieces, c = (e % kPieces) * 2;
      const bool ok = rhs0 + r < nrhs && k0 + c < ld;
      cg_copy16(sX + r * kPitch + c, ok ? X + (size_t)(rhs0 + r) * ld + k0 + c : X, ok);
    }
  };

  float ar[4][TN], ai[4][TN], hr[4][TN], hi_[4][TN], lr[4][TN], li[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < TN; ++q) ar[i][q] = ai[i][q] = hr[i][q] = hi_[i][q] = lr[i][q] = li[i][q] = 0.f;

#pragma unroll
  for (int p = 0; p < S - 1; ++p) {
    if (u0 + p < u1) load(p, u0 + p);
    cg_commit();
  }
  int since = 0;  // K blocks summed in FP32 since the last fold
  for (int64_t u = u0; u < u1; ++u) {
    const int it = (int)(u - u0);
    cg_wait<S - 2>();
    __syncthreads();  // stage it is in; every thread is done with the stage the next copy overwrites
    if (u + S - 1 < u1) load((it + S - 1) % S, u + S - 1);
    cg_commit();
    const float2* sA = sm + (it % S) * kStage;
    const float2* sX = sA + BM * kPitch;
#pragma unroll
    for (int k = 0; k < BK; k += 2) {
      float4 a[4], x[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(sA + (rg + RG * i) * kPitch + k);
#pragma unroll
      for (int q = 0; q < TN; ++q) x[q] = *reinterpret_cast<const float4*>(sX + (cg + CG * q) * kPitch + k);
      // per accumulator: re -= Im a Im x, re += Re a Re x, im += Im a Re x, im += Re a Im x for
      // term k, then term k + 1; written pass by pass so dependent FMAs sit far apart
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ar[i][q] = fmaf(-a[i].y, x[q].y, ar[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ai[i][q] = fmaf(a[i].y, x[q].x, ai[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ar[i][q] = fmaf(a[i].x, x[q].x, ar[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ai[i][q] = fmaf(a[i].x, x[q].y, ai[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ar[i][q] = fmaf(-a[i].w, x[q].w, ar[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ai[i][q] = fmaf(a[i].w, x[q].z, ai[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ar[i][q] = fmaf(a[i].z, x[q].z, ar[i][q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) ai[i][q] = fmaf(a[i].z, x[q].w, ai[i][q]);
    }
    const int64_t tile = u / nkb;
    const bool seg_end = u + 1 == u1 || (u + 1) % nkb == 0;
    if (++since == kFlush || seg_end) {
      since = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
          two_sum_acc(hr[i][q], lr[i][q], ar[i][q]);
          two_sum_acc(hi_[i][q], li[i][q], ai[i][q]);
          ar[i][q] = ai[i][q] = 0.f;
        }
    }
    if (seg_end) {
      double2* p = part + ((size_t)blockIdx.x * msp + (size_t)(tile - tile0)) * BN * BM;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
          p[(size_t)(cg + CG * q) * BM + rg + RG * i] =
              make_double2((double)hr[i][q] + (double)lr[i][q], (double)hi_[i][q] + (double)li[i][q]);
          hr[i][q] = hi_[i][q] = lr[i][q] = li[i][q] = 0.f;
        }
    }
  }
  cg_wait<0>();
}

// Y[c][row] = the sum, in CTA order, of the partials of the tile holding (row, c)
__global__ void k_cgemm_sk_reduce(const double2* __restrict__ part, int n, int nrhs, int BM, int BN, int ntn,
                                  int nkb, int per, int msp, double2* __restrict__ Y,
                                  const int* __restrict__ done, const int* __restrict__ scal) {
  if (scal && scal[1]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nrhs * n
  if (i >= (int64_t)nrhs * n) return;
  const int c = (int)(i / n), row = (int)(i % n);
  if (done && done[c]) return;
  const int64_t tile = (int64_t)(row / BM) * ntn + c / BN;
  const int r = row % BM, cl = c % BN;
  const int64_t first = tile * nkb, last = first + nkb - 1;
  const int c_lo = (int)(first / per), c_hi = (int)(last / per);
  double re = 0.0, im = 0.0;
  for (int cta = c_lo; cta <= c_hi; ++cta) {
    const int64_t j = tile - ((int64_t)cta * per) / nkb;
    const double2 v = part[((size_t)cta * msp + (size_t)j) * BN * BM + (size_t)cl * BM + r];
    re += v.x;
    im += v.y;
  }
  Y[(size_t)c * n + row] = make_double2(re, im);
}

// An mbarrier that nothing completes: the bounded wait must give up (result 2) and return.
__global__ void k_selftest_wait(uint64_t timeout_ns, int* __restrict__ result) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar), 0, timeout_ns);
  if (threadIdx.x == 0) *result = ok ? 1 : 2;
}

// --------------------------------------------------------------------------- host side
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::mutex g_encode_mu;

nat_bem_status get_encode(EncodeTiledFn* fn) {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return NAT_BEM_ECUDA;
    }
    g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  *fn = g_encode;
  return NAT_BEM_OK;
}

nat_bem_status make_map(CUtensorMap* map, CUtensorMapDataType dt, const void* ptr, uint64_t inner,
                        uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn enc = nullptr;
  NB_TRY(get_encode(&enc));
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    return NAT_BEM_ECUDA;
  }
  return NAT_BEM_OK;
}

}  // namespace

namespace {
// The stream-K partition of k_tc_gemm for n rows in tiles of tm and nkb K blocks on `ctas`
// CTAs at most: the CTA count, the K blocks per CTA and the most row-tile segments one CTA can
// touch.
struct TcPlan {
  int grid, per, msp;
};
TcPlan tc_plan(int64_t n, int64_t tm, int64_t nkb, int ctas) {
  const int64_t m_tiles = (n + tm - 1) / tm;
  const int64_t T = m_tiles * nkb;
  int64_t g = std::max<int64_t>(1, std::min<int64_t>(ctas, (T + kTcMinBlocks - 1) / kTcMinBlocks));
  const int64_t per = (T + g - 1) / g;
  g = (T + per - 1) / per;
  return TcPlan{(int)g, (int)per, (int)((per + nkb - 1) / nkb + 1)};
}

// Launch shape of k_tc_gemm: row tiles per stage (1 or 2 x 128 rows), ring stages, CTAs per SM.
struct TcShape {
  int tiles, stages, cps;
};

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}

uint32_t tc_fixed_bytes() { return 1024 + 8 * (2 * kTcMaxStages + 5) + 16; }

uint32_t tc_ncols(int Ng) {
  uint32_t c = 32;
  while ((int)c < Ng) c <<= 1;
  return c;
}

// A shape with as many stages as fit beside `cps` - 1 other CTAs on the SM, or stages = 0 if the
// two TMEM buffers of every CTA on the SM do not fit in its 512 columns or the operator is
// shorter than one row tile.
TcShape tc_fit(int Ng, int64_t n, int tiles, int cps, int max_stages = kTcMaxStages) {
  TcShape sh{tiles, 0, cps};
  if (2u * tiles * tc_ncols(Ng) * cps > 512u || (tiles > 1 && n < (int64_t)tiles * kTcRows)) return sh;
  const uint32_t budget = cps == 1 ? kTcSmemMax : (228u * 1024u / 2u - 1024u - 256u);
  const uint32_t stage_bytes = (uint32_t)(kTcRows * tiles * 128 + Ng * 128);
  const int fit = (int)((budget - tc_fixed_bytes()) / stage_bytes);
  sh.stages = std::min(std::min(kTcMaxStages, max_stages), fit);
  if (sh.stages < 2) sh.stages = 0;
  return sh;
}

// Candidate shapes in order of preference: two CTAs per SM (two independent TMA / MMA streams),
// two row tiles per stage (B read once for 256 rows), one of each.
std::vector<TcShape> tc_candidates(int Ng, int64_t n) {
  std::vector<TcShape> out;
  for (auto tc : {std::make_pair(1, 2), std::make_pair(2, 1), std::make_pair(1, 1)}) {
    const TcShape sh = tc_fit(Ng, n, tc.first, tc.second);
    if (sh.stages) out.push_back(sh);
  }
  return out;
}

// Shapes the autotuner chose, per (device, operator rows rounded up to 1024, Ng, engine).
std::mutex g_tc_mu;
std::map<std::tuple<int, int64_t, int, int>, TcShape> g_tc_tuned;

// The shape for this product: NATBEM_TC_TILES / _CPS / _STAGES when set (diagnostics), else the
// tuned one, else the first candidate.
TcShape tc_shape(int dev, int64_t n, int Ng, int engine) {
  const char* et = std::getenv("NATBEM_TC_TILES");
  const char* ec = std::getenv("NATBEM_TC_CPS");
  if (et || ec) {
    TcShape sh = tc_fit(Ng, n, std::max(1, std::min(2, env_int("NATBEM_TC_TILES", 1))),
                        std::max(1, std::min(2, env_int("NATBEM_TC_CPS", 1))),
                        std::max(2, env_int("NATBEM_TC_STAGES", kTcMaxStages)));
    if (sh.stages) return sh;
  }
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    auto f = g_tc_tuned.find(std::make_tuple(dev, round_up(n, 1024), Ng, engine));
    if (f != g_tc_tuned.end()) return f->second;
  }
  return tc_candidates(Ng, n).front();
}
}  // namespace

namespace {
// Shapes of k_cgemm_sk: RHS groups, RHS per thread, K block, CTAs per SM. Picked by nrhs so that
// at most half of a tile's columns are padding; measured on GB300 at 20480 rows (FP32 operator
// 3.36 GB): 0.60 ms at 1-2 RHS (5.6 TB/s), 0.69 at 3-4, 0.98 at 5-8, 1.62 at 9-16, 2.52 at
// 17-32, 4.80 at 33-64 (45 TFLOP/s); deeper K blocks paid at every width (fewer barriers and
// longer runs of each operator row per visit).
struct CgCfg {
  int cg, tn, bk, minb;
};
constexpr CgCfg kCgCfgs[] = {{16, 4, 64, 1}, {16, 2, 32, 2}, {16, 1, 32, 2},
                             {8, 1, 64, 1},  {4, 1, 32, 1},  {2, 1, 16, 1}};
constexpr int kCgNumCfgs = (int)(sizeof(kCgCfgs) / sizeof(kCgCfgs[0]));

int cg_pick(int nrhs) { return nrhs > 32 ? 0 : nrhs > 16 ? 1 : nrhs > 8 ? 2 : nrhs > 4 ? 3 : nrhs > 2 ? 4 : 5; }

// The stream-K partition of k_cgemm_sk: its shape, tile sizes, RHS tile count, K blocks, CTAs,
// K blocks per CTA, the most tiles one CTA can touch.
struct CgPlan {
  int cfg, bm, bn, ntn, nkb, grid, per, msp;
};
CgPlan cg_plan(int64_t n, int64_t ld, int nrhs, int sms) {
  CgPlan p;
  p.cfg = cg_pick(nrhs);
  const CgCfg& c = kCgCfgs[p.cfg];
  p.bm = 4 * (256 / c.cg);
  p.bn = c.cg * c.tn;
  p.ntn = (nrhs + p.bn - 1) / p.bn;
  p.nkb = (int)((ld + c.bk - 1) / c.bk);  // the last K block may run past ld: zero-filled
  const int64_t T = (n + p.bm - 1) / p.bm * p.ntn * p.nkb;
  int64_t g = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * c.minb, (T + kCgMinBlocks - 1) / kCgMinBlocks));
  const int64_t per = (T + g - 1) / g;
  p.grid = (int)((T + per - 1) / per);
  p.per = (int)per;
  p.msp = (int)((per + p.nkb - 1) / p.nkb + 1);
  return p;
}
size_t cg_partial_bytes(const CgPlan& p) { return (size_t)p.grid * p.msp * p.bn * p.bm * sizeof(double2); }

template <int CFG>
nat_bem_status cg_launch(const char* nm, const float2* M, int n, int ld, const float2* X, int nrhs,
                         const CgPlan& cp, double2* part, const int* scal, cudaStream_t s) {
  constexpr CgCfg c = kCgCfgs[CFG];
  constexpr int smem = cg_stages(c.cg, c.tn, c.bk, c.minb) * cg_stage_bytes(c.cg, c.tn, c.bk);
  static const cudaError_t ae =
      cudaFuncSetAttribute(k_cgemm_sk<c.cg, c.tn, c.bk, c.minb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (ae != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ae));
    return NAT_BEM_ECUDA;
  }
  NB_LAUNCH(nm, s, k_cgemm_sk<c.cg, c.tn, c.bk, c.minb><<<cp.grid, 256, smem, s>>>(
                       M, n, ld, X, nrhs, cp.ntn, cp.nkb, cp.per, cp.msp, part, scal));
  return NAT_BEM_OK;
}

template <int CFG = 0>
nat_bem_status cg_dispatch(int cfg, const char* nm, const float2* M, int n, int ld, const float2* X, int nrhs,
                           const CgPlan& cp, double2* part, const int* scal, cudaStream_t s) {
  if constexpr (CFG < kCgNumCfgs) {
    if (cfg == CFG) return cg_launch<CFG>(nm, M, n, ld, X, nrhs, cp, part, scal, s);
    return cg_dispatch<CFG + 1>(cfg, nm, M, n, ld, X, nrhs, cp, part, scal, s);
  }
  set_error("no such FP32 GEMM shape");
  return NAT_BEM_EINVAL;
}
}  // namespace

size_t tc_workspace_bytes(int64_t n, int64_t ld, int nrhs, int sms) {
  const int P = (int)round_up(nrhs, 16);  // N = 2P is a multiple of 32: whole TMEM loads
  const int Ng = 2 * P;
  const int64_t Kt = 2 * ld;
  // partial tiles: the largest plan over K blocks of 32 (TF32) or 64 (BF16), row tiles of 128
  // or 256 and one or two CTAs per SM
  size_t floats = 0;
  for (int64_t bk : {32, 64})
    for (int64_t tm : {128, 256})
      for (int cps : {1, 2}) {
        const TcPlan pl = tc_plan(n, tm, (Kt + bk - 1) / bk, cps * sms);
        floats = std::max(floats, (size_t)pl.grid * pl.msp * (size_t)tm);
      }
  const size_t tc = round_up((size_t)Ng * Kt * 4, 256) + floats * Ng * 4 + 64;
  // x6: three BF16 planes of B for at most 64 RHS per call, one-tile plan on one CTA per SM
  const int Ng6 = std::min(Ng, 128);
  const TcPlan p6 = tc_plan(n, kTcRows, (Kt + 63) / 64, sms);
  const size_t x6 = round_up((size_t)3 * Ng6 * Kt * 2, 256) + (size_t)p6.grid * p6.msp * kTcRows * Ng6 * 4 + 64;
  return std::max(std::max(tc, x6), cg_partial_bytes(cg_plan(n, ld, nrhs, sms)) + 64);
}

bool x6_enabled() { return std::getenv("NATBEM_NO_X6") == nullptr; }

// The x6 kernel's shared-memory opt-in, set once (first from ensure_split, outside any capture).
static cudaError_t x6_attr() {
  static const cudaError_t e =
      cudaFuncSetAttribute(k_tc_gemm_x6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
  return e;
}

nat_bem_status ensure_split(nat_bem_op* op, cudaStream_t s) {
  if (op->views || op->bstride > 0 || !op->L) return NAT_BEM_OK;  // batches run GEMVs
  const int64_t Kt = 2 * op->geo.ld;
  const int64_t count = op->n * Kt;  // floats of L (a multiple of 64)
  if (!op->Ls) NB_TRY(dev_alloc_n(&op->Ls, 3 * (size_t)count, s));
  if (!op->split_ok) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    NB_LAUNCH("split3", s, k_split3<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const float4*>(op->L), count / 4,
                                                           reinterpret_cast<__nv_bfloat16*>(op->Ls), count));
    NB_CHECK_LAUNCH();
    op->split_ok = true;
  }
  if (x6_attr() != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(x6_attr()));
    return NAT_BEM_ECUDA;
  }
  return NAT_BEM_OK;
}

// Y = L X for nrhs <= 64 with the x6 kernel (the caller checked op->split_ok).
static nat_bem_status product_x6(nat_bem_op* op, const float2* X, int nrhs, double2* Y, const int* done,
                                 const int* scal, void* scratch, size_t scratch_bytes, int* err, cudaStream_t s,
                                 int sms) {
  const int n = (int)op->n, ld = (int)op->geo.ld;
  const int P = (int)round_up(nrhs, 16);
  const int Ng = 2 * P;
  const int64_t Kt = 2 * (int64_t)ld;
  const int nkb = (int)((Kt + 63) / 64);
  const TcPlan pl = tc_plan(n, kTcRows, nkb, sms);
  const size_t bplane = (size_t)Ng * Kt;
  const size_t bbytes = round_up(3 * bplane * 2, 256);
  const size_t pbytes = (size_t)pl.grid * pl.msp * Ng * kTcRows * 4;
  if (Ng > 128 || bbytes + pbytes > scratch_bytes) {
    set_error("x6 product: more than 64 RHS or scratch too small");
    return NAT_BEM_ECUDA;
  }
  __nv_bfloat16* B = static_cast<__nv_bfloat16*>(scratch);
  float* part = reinterpret_cast<float*>(static_cast<uint8_t*>(scratch) + bbytes);
  {
    const int64_t tot = (int64_t)P * ld;
    NB_LAUNCH("tc_pack", s, k_pack_b3<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, nrhs, P, B, (int64_t)bplane, scal));
    NB_CHECK_LAUNCH();
  }
  CUtensorMap ta[3], tb[3];
  for (int q = 0; q < 3; ++q) {
    NB_TRY(make_map(&ta[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, op->Ls + (size_t)q * n * Kt, (uint64_t)Kt, (uint64_t)n,
                    (uint64_t)Kt * 2, 64u, (uint32_t)kTcRows));
    NB_TRY(make_map(&tb[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B + (size_t)q * bplane, (uint64_t)Kt, (uint64_t)Ng,
                    (uint64_t)Kt * 2, 64u, (uint32_t)Ng));
  }
  const uint32_t stage_bytes = 3u * (uint32_t)(kTcRows * 128 + Ng * 128);
  const int stages = std::min(kTcMaxStages, (int)((kTcSmemMax - tc_fixed_bytes()) / stage_bytes));
  if (stages < 2) {
    set_error("x6 product: shared memory too small");
    return NAT_BEM_ECUDA;
  }
  const size_t smem = tc_fixed_bytes() + (size_t)stages * stage_bytes;
  if (x6_attr() != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(x6_attr()));
    return NAT_BEM_ECUDA;
  }
  NB_LAUNCH("tc_gemm_x6", s, k_tc_gemm_x6<<<pl.grid, kX6Threads, smem, s>>>(ta[0], ta[1], ta[2], tb[0], tb[1], tb[2], n, nkb,
                                                                          pl.per, pl.msp, Ng, stages, part, err, scal));
  NB_CHECK_LAUNCH();
  const int64_t tot = (int64_t)nrhs * n;
  NB_LAUNCH("tc_reduce", s, k_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      part, n, kTcRows, Ng, P, nrhs, nkb, pl.per, pl.msp, Y, done, scal, nullptr));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

static nat_bem_status product_shaped(nat_bem_op* op, int which, int engine, const float2* X, int nrhs,
                                     double2* Y, const int* done, const int* scal, void* scratch,
                                     size_t scratch_bytes, int* err, cudaStream_t s,
                                     const TcShape* force) {
  const int n = (int)op->n, ld = which == 1 ? (int)op->ldr : (int)op->geo.ld;
  const float2* M = which == 0 ? op->L : op->R;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (engine == kEngineFp32 && which == 0 && nrhs >= kX6MinRhs && op->Ls && op->split_ok && x6_enabled() &&
      ((uintptr_t)scratch & 255u) == 0) {
    for (int c0 = 0; c0 < nrhs; c0 += 64)  // at most 64 RHS per launch (Ng <= 128 TMEM columns)
      NB_TRY(product_x6(op, X + (size_t)c0 * ld, std::min(64, nrhs - c0), Y + (size_t)c0 * n, done ? done + c0 : nullptr,
                        scal, scratch, scratch_bytes, err, s, sms));
    return NAT_BEM_OK;
  }
  if (engine == kEngineFp32) {
    const CgPlan cp = cg_plan(n, ld, nrhs, sms);
    const bool aligned = ld % 2 == 0 && ((uintptr_t)M & 15u) == 0 && ((uintptr_t)X & 15u) == 0 &&
                         ((uintptr_t)scratch & 15u) == 0;
    if (aligned && scratch && cg_partial_bytes(cp) <= scratch_bytes && !std::getenv("NATBEM_CGEMM_TILED")) {
      double2* part = static_cast<double2*>(scratch);
      NB_TRY(cg_dispatch(cp.cfg, which == 0 ? "cgemm_fp32_L" : "cgemm_fp32_R", M, n, ld, X, nrhs, cp, part, scal, s));
      NB_CHECK_LAUNCH();
      const int64_t tot = (int64_t)nrhs * n;
      NB_LAUNCH("cgemm_reduce", s, k_cgemm_sk_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
          part, n, nrhs, cp.bm, cp.bn, cp.ntn, cp.nkb, cp.per, cp.msp, Y, done, scal));
      NB_CHECK_LAUNCH();
      return NAT_BEM_OK;
    }
    dim3 grid((n + kGmRows - 1) / kGmRows, (nrhs + kGmRhs - 1) / kGmRhs);
    NB_LAUNCH(which == 0 ? "cgemm_fp32_L" : "cgemm_fp32_R", s,
              k_cgemm_fp32<<<grid, 256, 0, s>>>(M, n, ld, X, nrhs, Y, done, scal));
    NB_CHECK_LAUNCH();
    return NAT_BEM_OK;
  }
  if (which != 0 || ((engine == kEngineBf16 || engine == kEngineFp16) && !op->Lb) ||
      (engine == kEngineBf16 && op->copy_fp16) || (engine == kEngineFp16 && !op->copy_fp16)) {
    set_error("tensor-core product needs L (and its BF16 or FP16 copy for those engines)");
    return NAT_BEM_EINVAL;
  }
  const int P = (int)round_up(nrhs, 16);  // N = 2P is a multiple of 32: whole TMEM loads
  const int Ng = 2 * P;
  if (Ng > 256) {
    set_error("tensor-core product takes at most 128 right-hand sides per call");
    return NAT_BEM_EINVAL;
  }
  const int64_t Kt = 2 * (int64_t)ld;
  const int BK = engine == kEngineTf32 ? 32 : 64;
  const int nkb = (int)((Kt + BK - 1) / BK);
  const TcShape sh = force ? *force : tc_shape(dev, n, Ng, engine);
  const int TM = kTcRows * sh.tiles;
  const TcPlan pl = tc_plan(n, TM, nkb, sh.cps * sms);
  const size_t esz = engine == kEngineTf32 ? 4 : 2;
  const size_t bbytes = (size_t)Ng * Kt * esz;
  const size_t pbytes = (size_t)pl.grid * pl.msp * Ng * TM * 4;
  if (round_up(bbytes, 256) + pbytes > scratch_bytes) {
    set_error("tensor-core product: scratch too small");
    return NAT_BEM_ECUDA;
  }
  uint8_t* B = static_cast<uint8_t*>(scratch);
  float* part = reinterpret_cast<float*>(B + round_up(bbytes, 256));
  {
    const int64_t tot = (int64_t)P * ld;
    if (engine == kEngineTf32)
      NB_LAUNCH("tc_pack", s, k_pack_b<0><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, nrhs, P, B, scal));
    else if (engine == kEngineBf16)
      NB_LAUNCH("tc_pack", s, k_pack_b<1><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, nrhs, P, B, scal));
    else
      NB_LAUNCH("tc_pack", s, k_pack_b<2><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, nrhs, P, B, scal));
    NB_CHECK_LAUNCH();
  }
  CUtensorMap ta, tb;
  const CUtensorMapDataType dt = engine == kEngineTf32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : engine == kEngineBf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const void* Aptr = engine == kEngineTf32 ? (const void*)op->L : (const void*)op->Lb;
  NB_TRY(make_map(&ta, dt, Aptr, (uint64_t)Kt, (uint64_t)n, (uint64_t)Kt * esz, (uint32_t)BK, (uint32_t)TM));
  NB_TRY(make_map(&tb, dt, B, (uint64_t)Kt, (uint64_t)Ng, (uint64_t)Kt * esz, (uint32_t)BK, (uint32_t)Ng));
  const uint32_t stage_bytes = (uint32_t)(TM * 128 + Ng * 128);
  const size_t smem = tc_fixed_bytes() + (size_t)sh.stages * stage_bytes;
  // opt in to the largest dynamic shared memory any launch uses (per kernel, once)
  static std::mutex attr_mu;
  static bool attr_set = false;
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    if (!attr_set) {
      const int mx = (int)kTcSmemMax;
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      attr_set = true;
    }
  }
  if (engine == kEngineTf32) {
    if (sh.tiles == 2)
      NB_LAUNCH("tc_gemm_tf32", s, k_tc_gemm<0, 2><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
    else
      NB_LAUNCH("tc_gemm_tf32", s, k_tc_gemm<0, 1><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
  } else if (engine == kEngineBf16) {
    if (sh.tiles == 2)
      NB_LAUNCH("tc_gemm_bf16", s, k_tc_gemm<1, 2><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
    else
      NB_LAUNCH("tc_gemm_bf16", s, k_tc_gemm<1, 1><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
  } else {
    if (sh.tiles == 2)
      NB_LAUNCH("tc_gemm_fp16", s, k_tc_gemm<2, 2><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
    else
      NB_LAUNCH("tc_gemm_fp16", s, k_tc_gemm<2, 1><<<pl.grid, kTcThreads, smem, s>>>(ta, tb, n, nkb, pl.per, pl.msp, Ng, sh.stages, part, err, scal));
  }
  NB_CHECK_LAUNCH();
  const int64_t tot = (int64_t)nrhs * n;
  NB_LAUNCH("tc_reduce", s, k_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      part, n, TM, Ng, P, nrhs, nkb, pl.per, pl.msp, Y, done, scal, engine == kEngineFp16 ? op->row_scale : nullptr));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

nat_bem_status product(nat_bem_op* op, int which, int engine, const float2* X, int nrhs,
                       double2* Y, const int* done, const int* scal, void* scratch,
                       size_t scratch_bytes, int* err, cudaStream_t s) {
  return product_shaped(op, which, engine, X, nrhs, Y, done, scal, scratch, scratch_bytes, err, s, nullptr);
}

// The tensor-core product's autotuner, run once per (device, size class, Ng, engine) before the
// first product of a solve (outside any graph capture): each candidate shape is timed on the
// operator itself with CUDA events on the solve's stream, one warm-up round and three
// interleaved rounds, keeping each shape's minimum (other streams' kernels only slow a run
// down); the first candidate wins ties within 2%. X and Y are scratch of the caller.
nat_bem_status tc_tune(nat_bem_op* op, int engine, int nrhs, const float2* X, double2* Y,
                       void* scratch, size_t scratch_bytes, int* err, cudaStream_t s) {
  if (engine != kEngineTf32 && engine != kEngineBf16 && engine != kEngineFp16) return NAT_BEM_OK;
  if (std::getenv("NATBEM_TC_TILES") || std::getenv("NATBEM_TC_CPS")) return NAT_BEM_OK;
  int dev = 0;
  NB_TRY_CUDA(cudaGetDevice(&dev));
  const int Ng = 2 * (int)round_up(nrhs, 16);
  const auto key = std::make_tuple(dev, round_up(op->n, 1024), Ng, engine);
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (g_tc_tuned.count(key)) return NAT_BEM_OK;
  }
  const std::vector<TcShape> cand = tc_candidates(Ng, op->n);
  if (cand.size() < 2) {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    g_tc_tuned[key] = cand.front();
    return NAT_BEM_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NB_TRY_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("cudaEventCreate failed");
    return NAT_BEM_ECUDA;
  }
  std::vector<float> best(cand.size(), 1e30f);
  nat_bem_status st = NAT_BEM_OK;
  for (int round = 0; round < 4 && st == NAT_BEM_OK; ++round)
    for (size_t c = 0; c < cand.size() && st == NAT_BEM_OK; ++c) {
      cudaEventRecord(e0, s);
      st = product_shaped(op, 0, engine, X, nrhs, Y, nullptr, nullptr, scratch, scratch_bytes, err, s, &cand[c]);
      cudaEventRecord(e1, s);
      if (st == NAT_BEM_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        if (round > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best[c] = std::min(best[c], ms);
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NAT_BEM_OK) return st;
  size_t pick = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (best[c] < 0.98f * best[pick]) pick = c;
  std::lock_guard<std::mutex> lk(g_tc_mu);
  g_tc_tuned[key] = cand[pick];
  return NAT_BEM_OK;
}

}  // namespace natbem

extern "C" nat_bem_status nat_bem_selftest_bounded_wait(int32_t timeout_ms, void* cuda_stream) {
  using namespace natbem;
  clear_error();
  if (timeout_ms < 1 || timeout_ms > 10000) {
    set_error("nat_bem_selftest_bounded_wait: timeout_ms must be in [1, 10000]");
    return NAT_BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  NB_TRY(dev_alloc_n(&d, 1, s));
  NB_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(int), s));
  NB_LAUNCH("selftest_wait", s, k_selftest_wait<<<1, 32, 0, s>>>((uint64_t)timeout_ms * 1000000ull, d));
  NB_CHECK_LAUNCH();
  int h = 0;
  NB_TRY_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  NB_TRY_CUDA(cudaStreamSynchronize(s));
  dev_free(d, s);
  if (h == 2) {
    set_error("bounded device wait gave up as intended");
    return NAT_BEM_ETIMEOUT;
  }
  if (h == 1) return NAT_BEM_OK;
  set_error("self-test kernel did not report");
  return NAT_BEM_ECUDA;
}
