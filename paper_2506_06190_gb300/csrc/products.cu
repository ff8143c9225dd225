// Multi-right-hand-side operator products Y = M X (M = L or R, X = nrhs complex vectors).
//
// Two engines:
//  * k_tc_gemm: tensor cores (tcgen05.mma, kind::tf32 on the FP32 operator or kind::f16 on its
//    BF16 copy) for the inner Krylov products of mixed-precision refinement. The complex
//    product is a real GEMM: row i of the complex64 operator read as 2*ld reals
//    [Re M_i0, Im M_i0, Re M_i1, ...] times the real matrix B whose column c < P is
//    (Re x_c0, -Im x_c0, Re x_c1, ...) and column P + c is (Im x_c0, Re x_c0, ...); then
//    Y[i][c] = Re (M x_c)_i and Y[i][P + c] = Im (M x_c)_i. A 128-row tile of the operator and
//    the whole of B (N = 2P <= 256 columns) are staged by TMA with 128-byte swizzling through
//    a ring of shared-memory stages guarded by mbarriers; one thread issues the TMA copies,
//    one thread issues the MMAs into a TMEM accumulator (128 lanes x N columns, FP32), and all
//    four warps read TMEM back (tcgen05.ld) for the epilogue. K is split over blocks; the FP32
//    partials are summed in a fixed order into FP64.
//  * k_cgemm_fp32: FP32 CUDA-core complex GEMM (64 rows x 32 RHS per block, FP32 products
//    summed in FP32 over 128 terms, then FP64) for the products that must carry full FP32
//    accuracy: the right-hand side R G, the refinement residuals and the plain FP32 solve.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets an error flag, the kernel
// skips its remaining work, waits (bounded) for its own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace natbem {

// ------------------------------------------------------------------ PTX wrappers (sm_100+)
namespace {

constexpr int kTcRows = 128;         // M of the MMA (rows of the operator per tile)
constexpr int kTcStages = 3;         // shared-memory ring
constexpr int kTcThreads = 128;
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

}  // namespace

// Y_part[ks][row][c] = sum over this block's K range of A[row][k] B[c][k]. A: n x Kt (tensor map
// ta, box BK x 128), B: Ng x Kt (tensor map tb, box BK x Ng). kKind 0: TF32 (FP32 storage,
// BK = 32), 1: BF16 (BK = 64); either way a stage row is 128 bytes and one MMA covers 32
// bytes of K, four per stage.
template <int kKind>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int n,
          int Kt, int kps, int Ng, float* __restrict__ part, int* __restrict__ err,
          const int* __restrict__ scal) {
  constexpr int BK = kKind == 0 ? 32 : 64;
  if (scal && scal[1]) return;  // every right-hand side has converged
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment of the shared-memory address itself (the 128-byte swizzle atom)
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t a_bytes = kTcRows * 128, b_bytes = (uint32_t)Ng * 128;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTcStages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kTcStages;
  uint64_t* accum = bars + 2 * kTcStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcRows, ks = blockIdx.y;
  const int k_begin = ks * kps;
  const int k_end = min(Kt, k_begin + kps);
  const int nk = k_end > k_begin ? (k_end - k_begin + BK - 1) / BK : 0;
  uint32_t ncols = 32;
  while ((int)ncols < Ng) ncols <<= 1;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accum), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA copies of the A tile and of B into the ring
    int issued = 0;
    for (int it = 0; it < nk && !s_abort; ++it) {
      const int s = it % kTcStages;
      const uint32_t ph = (uint32_t)(it / kTcStages) & 1u;
      if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u)) {
        atomicOr(err, 1);
        s_abort = 1;
        break;
      }
      const uint32_t sa = smem_u32(base + s * stage_bytes);
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, stage_bytes);
      const int k0 = k_begin + it * BK;
      tma_load_2d(sa, &ta, k0, m0, fb);
      tma_load_2d(sa + a_bytes, &tb, k0, 0, fb);
      issued = it + 1;
    }
    if (s_abort) {
      // let the copies already issued land before the block exits
      for (int it = max(0, issued - kTcStages); it < issued; ++it)
        mbar_wait(smem_u32(&full[it % kTcStages]), (uint32_t)(it / kTcStages) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = instr_desc(kKind == 0 ? 2u : 1u, (uint32_t)Ng, (uint32_t)kTcRows);
    for (int it = 0; it < nk && !s_abort; ++it) {
      const int s = it % kTcStages;
      const uint32_t ph = (uint32_t)(it / kTcStages) & 1u;
      if (!mbar_wait(smem_u32(&full[s]), ph)) {
        atomicOr(err, 2);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + s * stage_bytes);
      const uint64_t da = smem_desc(sa), db = smem_desc(sa + a_bytes);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // 32 bytes of K per MMA: +2 in the 16-byte address field
        mma<kKind>(tmem, da + 2 * kk, db + 2 * kk, idesc, (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty[s]));
    }
    mma_commit(smem_u32(accum));
  }
  __syncwarp();
  // epilogue: TMEM lanes 32w..32w+31 hold rows m0 + 32w + lane, 32 columns per load
  const bool ok = mbar_wait(smem_u32(accum), 0);
  if (!ok && lane == 0) atomicOr(err, 4);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (ok && !s_abort) {
    const int row = m0 + warp * 32 + lane;
    float* out = part + ((size_t)ks * n + (size_t)row) * Ng;
    for (int c0 = 0; c0 < Ng; c0 += 32) {  // Ng is a multiple of 32
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      if (row < n && nk > 0) {
#pragma unroll
        for (int q = 0; q < 32; q += 4)
          *reinterpret_cast<float4*>(out + c0 + q) =
              make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                          __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
      } else if (row < n) {
#pragma unroll
        for (int q = 0; q < 32; q += 4) *reinterpret_cast<float4*>(out + c0 + q) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// B for the tensor-core product from nrhs complex64 vectors (x_c at X + c * ld), P = nrhs
// rounded up to 16 (so the epilogue reads whole 32-column TMEM chunks): rows c < P
// (Re, -Im) pairs, rows P + c (Im, Re) pairs; rows of absent RHS are zero. TF32: FP32 storage;
// BF16: round to nearest.
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
  } else {
    __nv_bfloat16* b = static_cast<__nv_bfloat16*>(B);
    b[(size_t)c * Kt + 2 * j] = __float2bfloat16_rn(x.x);
    b[(size_t)c * Kt + 2 * j + 1] = __float2bfloat16_rn(-x.y);
    b[(size_t)(P + c) * Kt + 2 * j] = __float2bfloat16_rn(x.y);
    b[(size_t)(P + c) * Kt + 2 * j + 1] = __float2bfloat16_rn(x.x);
  }
}

// Y[c][row] (complex128, column c at Y + c * n) = sum over splits of the FP32 partials.
__global__ void k_tc_reduce(const float* __restrict__ part, int n, int Ng, int P, int nrhs,
                            int splits, double2* __restrict__ Y, const int* __restrict__ done,
                            const int* __restrict__ scal) {
  if (scal && scal[1]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nrhs * n
  if (i >= (int64_t)nrhs * n) return;
  const int c = (int)(i / n), row = (int)(i % n);
  if (done && done[c]) return;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < splits; ++s) {
    const float* p = part + ((size_t)s * n + row) * Ng;
    re += p[c];
    im += p[P + c];
  }
  Y[(size_t)c * n + row] = make_double2(re, im);
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

size_t tc_workspace_bytes(int64_t n, int64_t ld, int nrhs, int sms) {
  const int P = (int)round_up(nrhs, 16);  // N = 2P is a multiple of 32: whole TMEM loads
  const int Ng = 2 * P;
  const int64_t m_tiles = (n + kTcRows - 1) / kTcRows;
  const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(16, (4 * sms + m_tiles - 1) / m_tiles));
  return (size_t)Ng * 2 * ld * 4 + (size_t)splits * n * Ng * 4 + 64;
}

nat_bem_status product(nat_bem_op* op, int which, int engine, const float2* X, int nrhs,
                       double2* Y, const int* done, const int* scal, void* scratch,
                       size_t scratch_bytes, int* err, cudaStream_t s) {
  const int n = (int)op->n, ld = which == 1 ? (int)op->ldr : (int)op->geo.ld;
  const float2* M = which == 0 ? op->L : op->R;
  if (engine == kEngineFp32) {
    dim3 grid((n + kGmRows - 1) / kGmRows, (nrhs + kGmRhs - 1) / kGmRhs);
    NB_LAUNCH(which == 0 ? "cgemm_fp32_L" : "cgemm_fp32_R", s,
              k_cgemm_fp32<<<grid, 256, 0, s>>>(M, n, ld, X, nrhs, Y, done, scal));
    NB_CHECK_LAUNCH();
    return NAT_BEM_OK;
  }
  if (which != 0 || (engine == kEngineBf16 && !op->Lb)) {
    set_error("tensor-core product needs L (and its BF16 copy for the BF16 engine)");
    return NAT_BEM_EINVAL;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int P = (int)round_up(nrhs, 16);  // N = 2P is a multiple of 32: whole TMEM loads
  const int Ng = 2 * P;
  if (Ng > 256) {
    set_error("tensor-core product takes at most 128 right-hand sides per call");
    return NAT_BEM_EINVAL;
  }
  const int64_t Kt = 2 * (int64_t)ld;
  const int m_tiles = (n + kTcRows - 1) / kTcRows;
  const int splits = std::max(1, std::min(16, (4 * sms + m_tiles - 1) / m_tiles));
  const int BK = engine == kEngineTf32 ? 32 : 64;
  int kps = (int)((Kt + splits - 1) / splits);
  kps = (kps + BK - 1) / BK * BK;
  const int nsplit = (int)((Kt + kps - 1) / kps);
  const size_t esz = engine == kEngineTf32 ? 4 : 2;
  const size_t bbytes = (size_t)Ng * Kt * esz;
  const size_t pbytes = (size_t)nsplit * n * Ng * 4;
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
    else
      NB_LAUNCH("tc_pack", s, k_pack_b<1><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, nrhs, P, B, scal));
    NB_CHECK_LAUNCH();
  }
  CUtensorMap ta, tb;
  const CUtensorMapDataType dt = engine == kEngineTf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const void* Aptr = engine == kEngineTf32 ? (const void*)op->L : (const void*)op->Lb;
  NB_TRY(make_map(&ta, dt, Aptr, (uint64_t)Kt, (uint64_t)n, (uint64_t)Kt * esz, (uint32_t)BK, kTcRows));
  NB_TRY(make_map(&tb, dt, B, (uint64_t)Kt, (uint64_t)Ng, (uint64_t)Kt * esz, (uint32_t)BK, (uint32_t)Ng));
  const size_t smem = 1024 + (size_t)kTcStages * (kTcRows * 128 + (size_t)Ng * 128) + 8 * (2 * kTcStages + 2);
  dim3 grid(m_tiles, nsplit);
  // opt in to the dynamic shared memory this launch needs (once per size increase)
  static size_t attr_set[2] = {0, 0};
  const int ki = engine == kEngineTf32 ? 0 : 1;
  if (smem > attr_set[ki]) {
    if (ki == 0)
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
      NB_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[ki] = smem;
  }
  if (ki == 0)
    NB_LAUNCH("tc_gemm_tf32", s, k_tc_gemm<0><<<grid, kTcThreads, smem, s>>>(ta, tb, n, (int)Kt, kps, Ng, part, err, scal));
  else
    NB_LAUNCH("tc_gemm_bf16", s, k_tc_gemm<1><<<grid, kTcThreads, smem, s>>>(ta, tb, n, (int)Kt, kps, Ng, part, err, scal));
  NB_CHECK_LAUNCH();
  const int64_t tot = (int64_t)nrhs * n;
  NB_LAUNCH("tc_reduce", s, k_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, n, Ng, P, nrhs, nsplit, Y, done, scal));
  NB_CHECK_LAUNCH();
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
