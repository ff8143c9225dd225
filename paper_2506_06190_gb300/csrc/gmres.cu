// Dense complex GMRES for L p = R g (paper Sec. 6.1 settings: relative residual 1e-6, at most
// 200 iterations), run entirely on the device.
//
// Precision split: the operator and its matvec are FP32 (complex64 entries, FP32 products,
// partial sums flushed into FP64 accumulators); the Krylov basis, classical Gram-Schmidt with
// one re-orthogonalisation pass (CGS2), the Hessenberg matrix, the complex Givens rotations
// and the small least-squares solve are FP64.
//
// One iteration (all right-hand sides in lockstep, each with its own Krylov space) is two
// launches: the matvec w = L v_j, then one cooperative kernel (k_arnoldi, or k_arnoldi_units
// for many right-hand sides) that does the Gram-Schmidt passes, ||w||, v_{j+1} and the Givens
// update with grid barriers. Where a cooperative launch cannot hold every block, the same step
// runs as five kernels (dots, update, dots, update, finish). The iteration index, the per-RHS
// convergence flags and the "all done" flag live in device memory, so the launch sequence is
// the same every iteration and finished iterations cost only empty launches; chunks of
// iterations are captured as CUDA graphs. Reductions are deterministic: per-chunk partial
// sums, summed in a fixed order by the last block to finish (counted with an atomic ticket).
// Restarted GMRES(m) and mixed-precision refinement run sweeps of this loop on the current
// residual, accumulating the solution in FP64.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace natbem {

constexpr int kChunk = 256;       // rows per block in the element-wise vector kernels
constexpr int kUpdRows = 64;      // rows per block in the Gram-Schmidt update (4 column groups)
constexpr int kDotThreads = 256;  // threads of the dot-product blocks
constexpr int kDotChunks = 8;     // row ranges per Krylov vector in the dot products
constexpr int kCounters = 8;      // per-RHS tickets

struct Workspace {
  int64_t n = 0, ld = 0;
  int nrhs = 0, cap = 0, m = 0, nchunk = 0;
  double2 *b = nullptr, *V = nullptr, *w = nullptr, *x = nullptr;
  double2 *H = nullptr, *hcol = nullptr, *htmp = nullptr, *sn = nullptr, *gv = nullptr;
  double2 *y = nullptr, *part = nullptr;
  double *cs = nullptr, *partn = nullptr, *bnorm = nullptr, *res = nullptr, *hnorm = nullptr;
  double* res_true = nullptr;
  double2 *b0 = nullptr, *xacc = nullptr;  // refinement: R g and the accumulated solution
  double* b0norm = nullptr;                 // refinement / restart: ||R g|| per RHS
  float2 *xf = nullptr, *gin = nullptr, *pout = nullptr;
  int *done = nullptr, *iters = nullptr, *scal = nullptr;  // scal: j, all_done, rhs ticket
  int* outer_done = nullptr;                               // refinement: converged RHS
  unsigned* gbar = nullptr;                                // grid barrier state (count, gen)
  int coop_blocks = 0;                                     // 0: fused kernel not usable
  int units_blocks = 0;                                    // grid of the multi-RHS fused kernel
  double2 *pblk = nullptr, *hred = nullptr;                // fused kernel: block partials, totals
  int arn_smem = 0;                                        // fused kernel: dynamic shared bytes
  double2* pbu = nullptr;                                  // multi-RHS fused kernel: unit partials
  float2* wf = nullptr;                                    // multi-RHS fused kernel: FP32 w
  // captured iteration chunks: key (engine, RHS count, first iteration, count, cap, tol, mode
  // bits: 1 skip flags, 2 accumulate, 4 tolerance relative to ||R g||). The RHS count is part
  // of the key: a workspace serves later solves with fewer columns, and a graph holds the
  // launch shapes and arguments of the count it was captured with.
  std::map<std::tuple<int, int, int, int, int, double, int>, std::pair<cudaGraphExec_t, int64_t>> graphs;
  bool graphs_off = false;
  // whole GMRES runs on the device: a graph whose conditional while node repeats a captured
  // chunk of iterations until every RHS is done; key (engine, RHS count, cap, tol, mode bits)
  std::map<std::tuple<int, int, int, double, int>, cudaGraphExec_t> loops;
  bool loops_off = false;
  unsigned long long* loop_launches = nullptr;  // kernels the loop bodies ran (device counter)
  int* loop_bodies = nullptr;                    // bodies the current loop ran (reset per run)
  unsigned long long* host_loop = nullptr;      // pinned mirror, read at host sync points
  void* tc_scratch = nullptr;                              // packed B + split-K partials
  size_t tc_bytes = 0;
  int* tc_err = nullptr;                                   // bounded-wait failures
  unsigned* cnt = nullptr;
  int* host_scal = nullptr;  // pinned mirror of scal[0..1]
};

struct GArgs {
  int n, ld, nrhs, m, nchunk;
  int maxit;           // iteration cap of this GMRES run (<= m)
  const int* skip;     // RHS to leave alone in this run (refinement), or null
  const double* bscale;  // stop at res <= tol * bscale[s] (||R g||: restart cycles and the
                         // FP32 finish of refinement), or null: res <= tol * ||b|| of this run
  const float2* L;
  double2 *b, *V, *w, *x, *H, *hcol, *htmp, *sn, *gv, *y, *part;
  double *cs, *partn, *bnorm, *res, *hnorm, *res_true;
  float2* xf;
  // FP32 Krylov basis (same layout as V, in V's memory) and FP32 copy of w, used by inner
  // solves of refinement on the multi-RHS fused kernel; Vf null: the FP64 basis V
  float2 *Vf, *wf;
  int *done, *iters, *scal;
  unsigned* cnt;
  double tol;
};

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a double (blockDim.x a multiple of 32, <= 1024); result in all threads.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh[i];  // fixed order
  return t;
}

// Ticket: returns true in every thread of the last block (among `total`) to arrive.
__device__ bool last_block(unsigned* counter, unsigned total) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == total - 1);
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ size_t vidx(const GArgs& a, int c, int s) {
  return ((size_t)c * a.nrhs + s) * (size_t)a.n;
}

}  // namespace

// ------------------------------------------------------------------------------ matvec
// Compensated FP32 summation (Kahan 1965): after each call s - c equals the exact running sum
// to about twice FP32 precision. The operator stream is bandwidth-bound with FP32 issue slots
// to spare, while GB300's FP64 rate is far too low to accumulate the stream in FP64.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Error-free transformation (Knuth's TwoSum): s + e == a + b exactly in FP32 arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (hi2, lo2) as double-float (an unevaluated FP32 pair, about 48 bits).
__device__ __forceinline__ void df_add(float& hi, float& lo, float hi2, float lo2) {
  float s, e;
  two_sum(hi, hi2, s, e);
  e += lo + lo2;
  hi = s + e;
  lo = e - (hi - s);
}

// Warp sum of a compensated running sum (s, c) as a double-float, all in FP32 (GB300's FP64
// rate is ~1/64 of FP32, too low even for per-thread FP64 shuffles at the end of each row).
__device__ __forceinline__ void warp_sum_df(float s, float c, float& hi, float& lo) {
  two_sum(s, -c, hi, lo);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
}

// Sum over the block (8 warps) of the compensated per-thread sums (s - c) per row: a fixed
// FP32 shuffle tree per warp, then one thread per row adds the eight warp sums in order. The
// per-thread sums carry the long accumulations; the 8 + 5 roundings of the tree are at the
// level of the FP32 operator entries' own rounding. Double-float trees or an FP64 combine here
// hold every block's exit on serial dependent chains and cost 3-15% of the bandwidth.
template <int kRows>
__device__ __forceinline__ void gemv_block_reduce(const float (&sr)[kRows], const float (&cr)[kRows],
                                                  const float (&si)[kRows], const float (&ci)[kRows],
                                                  int n, int row0, double2* __restrict__ y,
                                                  const float* __restrict__ rs = nullptr) {
  __shared__ float2 sh[kRows][8];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    float a = sr[r] - cr[r], b = si[r] - ci[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) sh[r][wid] = make_float2(a, b);
  }
  __syncthreads();
  if (threadIdx.x < kRows && row0 + (int)threadIdx.x < n) {
    const int r = threadIdx.x;
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      tr += sh[r][q].x;
      ti += sh[r][q].y;
    }
    const double sc = rs ? (double)rs[row0 + r] : 1.0;  // a power of two: exact
    y[row0 + r] = make_double2(tr * sc, ti * sc);
  }
}

// y_s = A x_s for the RHS s = blockIdx.y: A is n x ld complex64 (row-major, ld even, pad
// columns zero), x_s complex64 with ld entries, y_s complex128. kRows rows per block of 256
// threads; each thread strides over the row in 16-byte (two-complex) steps with kUnroll
// loads per row in flight, FP32 products and compensated FP32 running sums.
template <int kRows, int kUnroll>
__global__ void __launch_bounds__(256)
k_gemv(const float2* __restrict__ A, int n, int ld, const float2* __restrict__ x, int64_t xstride,
       double2* __restrict__ y, int64_t ystride, const int* __restrict__ done,
       const int* __restrict__ scal, int64_t astride) {
  if (scal && scal[1]) return;
  const int s = blockIdx.y;
  if (done && done[s]) return;
  A += (size_t)s * astride;  // a batch of operators: one per right-hand side
  const int row0 = blockIdx.x * kRows;
  const float4* xv = reinterpret_cast<const float4*>(x + (size_t)s * xstride);
  const float4* a[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r)
    a[r] = reinterpret_cast<const float4*>(A + (size_t)min(row0 + r, n - 1) * ld);
  const int n4 = ld >> 1;
  float sr[kRows], cr[kRows], si[kRows], ci[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) sr[r] = cr[r] = si[r] = ci[r] = 0.f;
  for (int base = threadIdx.x; base < n4; base += 256 * kUnroll) {
    float4 xx[kUnroll], aa[kRows][kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int idx = base + u * 256;
      const bool ok = idx < n4;
      xx[u] = ok ? __ldg(xv + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kRows; ++r) aa[r][u] = ok ? __ldcs(a[r] + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const float4 q = aa[r][u], v = xx[u];
        const float pr = fmaf(q.x, v.x, fmaf(-q.y, v.y, fmaf(q.z, v.z, -q.w * v.w)));
        const float pi = fmaf(q.x, v.y, fmaf(q.y, v.x, fmaf(q.z, v.w, q.w * v.z)));
        kahan_add(sr[r], cr[r], pr);
        kahan_add(si[r], ci[r], pi);
      }
    }
  }
  gemv_block_reduce<kRows>(sr, cr, si, ci, n, row0, y + (size_t)s * ystride);
}

// The same product by persistent blocks with x staged once per block in shared memory: each
// block takes row groups blockIdx.x, blockIdx.x + gridDim.x, ... (kRows rows each), so the
// operator is the only stream from memory; a block otherwise re-reads all of x for every
// kRows rows through L1/L2. Dynamic shared memory: 8 ld bytes.
template <int kRows, int kUnroll>
__global__ void __launch_bounds__(256)
k_gemv_xs(const float2* __restrict__ A, int n, int ld, const float2* __restrict__ x, int64_t xstride,
          double2* __restrict__ y, int64_t ystride, const int* __restrict__ done,
          const int* __restrict__ scal, int64_t astride) {
  extern __shared__ float4 s_x[];
  if (scal && scal[1]) return;
  const int s = blockIdx.y;
  if (done && done[s]) return;
  A += (size_t)s * astride;
  const int n4 = ld >> 1;
  const float4* xv = reinterpret_cast<const float4*>(x + (size_t)s * xstride);
  for (int i = threadIdx.x; i < n4; i += 256) s_x[i] = __ldg(xv + i);
  __syncthreads();
  for (int row0 = blockIdx.x * kRows; row0 < n; row0 += gridDim.x * kRows) {
    const float4* a[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      a[r] = reinterpret_cast<const float4*>(A + (size_t)min(row0 + r, n - 1) * ld);
    float sr[kRows], cr[kRows], si[kRows], ci[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) sr[r] = cr[r] = si[r] = ci[r] = 0.f;
    for (int base = threadIdx.x; base < n4; base += 256 * kUnroll) {
      float4 aa[kRows][kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int idx = base + u * 256;
        const bool ok = idx < n4;
#pragma unroll
        for (int r = 0; r < kRows; ++r) aa[r][u] = ok ? __ldcs(a[r] + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int idx = base + u * 256;
        const float4 v = idx < n4 ? s_x[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          const float4 q = aa[r][u];
          const float pr = fmaf(q.x, v.x, fmaf(-q.y, v.y, fmaf(q.z, v.z, -q.w * v.w)));
          const float pi = fmaf(q.x, v.y, fmaf(q.y, v.x, fmaf(q.z, v.w, q.w * v.z)));
          kahan_add(sr[r], cr[r], pr);
          kahan_add(si[r], ci[r], pi);
        }
      }
    }
    gemv_block_reduce<kRows>(sr, cr, si, ci, n, row0, y + (size_t)s * ystride);
    __syncthreads();  // the reduction's shared staging is reused by the next row group
  }
}

// The same product with A stored as a 16-bit copy: packed bf16 complex pairs (kFmt 0, real in
// the low half), or half2 pairs of the row-scaled entries L_ij s_i (kFmt 1; the row's sum is
// multiplied by rs[row] = 1/s_i, a power of two). Half the bytes of the FP32 operator; 16-byte
// loads hold four complex entries.
template <int kRows, int kUnroll, int kFmt>
__device__ __forceinline__ void gemv_copy_body(const uint32_t* __restrict__ A, int n, int ld,
                                               const float2* __restrict__ x, int64_t xstride,
                                               double2* __restrict__ y, int64_t ystride,
                                               const int* __restrict__ done, const int* __restrict__ scal,
                                               int64_t astride, const float* __restrict__ rs, int64_t sstride) {
  if (scal && scal[1]) return;
  const int s = blockIdx.y;
  if (done && done[s]) return;
  A += (size_t)s * astride;
  if (rs) rs += (size_t)s * sstride;
  const int row0 = blockIdx.x * kRows;
  const float4* xv = reinterpret_cast<const float4*>(x + (size_t)s * xstride);
  const uint4* a[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r)
    a[r] = reinterpret_cast<const uint4*>(A + (size_t)min(row0 + r, n - 1) * ld);
  const int n4 = ld >> 2;  // four complex per 16 bytes
  float sr[kRows], cr[kRows], si[kRows], ci[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) sr[r] = cr[r] = si[r] = ci[r] = 0.f;
  for (int base = threadIdx.x; base < n4; base += 256 * kUnroll) {
    float4 x0[kUnroll], x1[kUnroll];
    uint4 aa[kRows][kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int idx = base + u * 256;
      const bool ok = idx < n4;
      x0[u] = ok ? __ldg(xv + 2 * idx) : make_float4(0.f, 0.f, 0.f, 0.f);
      x1[u] = ok ? __ldg(xv + 2 * idx + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kRows; ++r) aa[r][u] = ok ? __ldcs(a[r] + idx) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const float xr[4] = {x0[u].x, x0[u].z, x1[u].x, x1[u].z};
      const float xi[4] = {x0[u].y, x0[u].w, x1[u].y, x1[u].w};
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const uint32_t w[4] = {aa[r][u].x, aa[r][u].y, aa[r][u].z, aa[r][u].w};
        float pr = 0.f, pi = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float ar, ai;
          if (kFmt == 0) {
            ar = __uint_as_float(w[e] << 16);
            ai = __uint_as_float(w[e] & 0xffff0000u);
          } else {
            const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[e]));
            ar = v.x;
            ai = v.y;
          }
          pr = fmaf(ar, xr[e], fmaf(-ai, xi[e], pr));
          pi = fmaf(ar, xi[e], fmaf(ai, xr[e], pi));
        }
        kahan_add(sr[r], cr[r], pr);
        kahan_add(si[r], ci[r], pi);
      }
    }
  }
  gemv_block_reduce<kRows>(sr, cr, si, ci, n, row0, y + (size_t)s * ystride, rs);
}

template <int kRows, int kUnroll>
__global__ void __launch_bounds__(256)
k_gemv_bf16(const uint32_t* __restrict__ A, int n, int ld, const float2* __restrict__ x,
            int64_t xstride, double2* __restrict__ y, int64_t ystride, const int* __restrict__ done,
            const int* __restrict__ scal, int64_t astride) {
  gemv_copy_body<kRows, kUnroll, 0>(A, n, ld, x, xstride, y, ystride, done, scal, astride, nullptr, 0);
}

template <int kRows, int kUnroll>
__global__ void __launch_bounds__(256)
k_gemv_fp16(const uint32_t* __restrict__ A, int n, int ld, const float2* __restrict__ x,
            int64_t xstride, double2* __restrict__ y, int64_t ystride, const int* __restrict__ done,
            const int* __restrict__ scal, int64_t astride, const float* __restrict__ rs, int64_t sstride) {
  gemv_copy_body<kRows, kUnroll, 1>(A, n, ld, x, xstride, y, ystride, done, scal, astride, rs, sstride);
}

// Bulk-copy GEMV for one RHS per blockIdx.y: each block streams a contiguous range of rows
// through a ring of kStages shared-memory stages. A producer warp issues 1-D bulk async copies
// (cp.async.bulk) of row segments of up to kSeg bytes, completed on mbarriers; eight consumer
// warps multiply each segment with x (read through L1) into compensated FP32 sums, and at the
// end of each row combine them in FP64. In-flight bytes no longer depend on registers.
namespace {
__device__ __forceinline__ uint32_t sa_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (uint32_t i = 0; i < (1u << 26); ++i) {
    if (bar_try(bar, parity)) return true;
    if ((i & 1023u) == 1023u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) return false;
    }
  }
  return false;
}
}  // namespace

template <int kStages, int kSeg>
__global__ void __launch_bounds__(288)
k_gemv_bulk(const float2* __restrict__ A, int n, int ld, const float2* __restrict__ x,
            int64_t xstride, double2* __restrict__ y, int64_t ystride, const int* __restrict__ done,
            const int* __restrict__ scal, int rows_per_block, int* __restrict__ err, int64_t astride) {
  extern __shared__ __align__(128) float4 ring_raw[];  // kStages x kSeg bytes (dynamic)
  float4 (*ring)[kSeg / 16] = reinterpret_cast<float4 (*)[kSeg / 16]>(ring_raw);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ double red[2][8];
  __shared__ int s_abort;
  if (scal && scal[1]) return;
  const int s = blockIdx.y;
  if (done && done[s]) return;
  A += (size_t)s * astride;
  const int row_begin = blockIdx.x * rows_per_block;
  const int row_end = min(n, row_begin + rows_per_block);
  if (row_begin >= row_end) return;
  const int row_bytes = ld * 8;
  const int nseg = (row_bytes + kSeg - 1) / kSeg;
  const int total = (row_end - row_begin) * nseg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < kStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa_u32(&full[q])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa_u32(&empty[q])), "r"(8) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 8) {  // producer
    if (lane == 0) {
      for (int t = 0; t < total && !s_abort; ++t) {
        const int q = t % kStages;
        const uint32_t ph = (uint32_t)(t / kStages) & 1u;
        if (!bar_wait(sa_u32(&empty[q]), ph ^ 1u)) {
          atomicOr(err, 8);
          s_abort = 1;
          break;
        }
        const int row = row_begin + t / nseg, seg = t % nseg;
        const int off = seg * kSeg;
        const int bytes = min(kSeg, row_bytes - off);
        const char* src = reinterpret_cast<const char*>(A + (size_t)row * ld) + off;
        const uint32_t fb = sa_u32(&full[q]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sa_u32(&ring[q][0])),
            "l"(src), "r"(bytes), "r"(fb)
            : "memory");
      }
    }
    return;
  }
  const float4* xv = reinterpret_cast<const float4*>(x + (size_t)s * xstride);
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  for (int t = 0; t < total; ++t) {
    const int q = t % kStages;
    const uint32_t ph = (uint32_t)(t / kStages) & 1u;
    if (!bar_wait(sa_u32(&full[q]), ph)) {
      if (threadIdx.x == 0) atomicOr(err, 16);
      s_abort = 1;
      break;
    }
    const int row = row_begin + t / nseg, seg = t % nseg;
    const int off4 = seg * (kSeg / 16);  // float4 index of the segment within the row
    const int cnt4 = min(kSeg, row_bytes - seg * kSeg) / 16;
    for (int e = threadIdx.x; e < cnt4; e += 256) {
      const float4 a = ring[q][e];
      const float4 v = __ldg(xv + off4 + e);
      const float pr = fmaf(a.x, v.x, fmaf(-a.y, v.y, fmaf(a.z, v.z, -a.w * v.w)));
      const float pi = fmaf(a.x, v.y, fmaf(a.y, v.x, fmaf(a.z, v.w, a.w * v.z)));
      kahan_add(sr, cr, pr);
      kahan_add(si, ci, pi);
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa_u32(&empty[q])) : "memory");
    if (seg == nseg - 1) {  // row complete: double-float warp sums, FP64 across warps
      float hr, lr, hi, li;
      warp_sum_df(sr, cr, hr, lr);
      warp_sum_df(si, ci, hi, li);
      if (lane == 0) {
        red[0][warp] = (double)hr + (double)lr;
        red[1][warp] = (double)hi + (double)li;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < 8; ++w) {
          tr += red[0][w];
          ti += red[1][w];
        }
        y[(size_t)s * ystride + row] = make_double2(tr, ti);
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      sr = cr = si = ci = 0.f;
    }
  }
  if (s_abort && warp == 0 && lane == 0) {
    // let the copies already in flight land before the block exits
    for (int q = 0; q < kStages; ++q) bar_wait(sa_u32(&full[q]), 0), bar_wait(sa_u32(&full[q]), 1);
  }
}

// ------------------------------------------------------------------------ GMRES steps
// Start of a GMRES run: w = b and each block's partial ||b||^2 (kUpdRows rows per block).
__global__ void __launch_bounds__(kUpdRows) k_start(GArgs a) {
  __shared__ double sh[32];
  const int s = blockIdx.y;
  const int r = blockIdx.x * kUpdRows + threadIdx.x;
  double v = 0.0;
  if (r < a.n) {
    const double2 bb = a.b[(size_t)s * a.n + r];
    a.w[(size_t)s * a.n + r] = bb;
    v = cabs2(bb);
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) a.partn[(size_t)blockIdx.x * a.nrhs + s] = v;
}

// Partial h_c = V[c]^H w over one of kDotChunks row ranges, for c <= j: block (c, chunk, RHS),
// FP64, into part[((s (m+1) + c) kDotChunks + chunk]. The consumer sums the chunks in order.
__global__ void __launch_bounds__(kDotThreads) k_dots(GArgs a) {
  __shared__ double sh[32];
  if (a.scal[1]) return;
  const int c = blockIdx.x, chunk = blockIdx.y, s = blockIdx.z;
  const int j = a.scal[0];
  if (c > j || a.done[s]) return;
  const int per = (a.n + kDotChunks - 1) / kDotChunks;
  const int r_begin = chunk * per, r_end = min(a.n, r_begin + per);
  const double2* v = a.V + vidx(a, c, s);
  const double2* w = a.w + (size_t)s * a.n;
  double re[2] = {0.0, 0.0}, im[2] = {0.0, 0.0};
  for (int r0 = r_begin + threadIdx.x; r0 < r_end; r0 += 2 * kDotThreads) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = r0 + u * kDotThreads;
      if (r < r_end) {
        const double2 p = cmulc(v[r], w[r]);
        re[u] += p.x;
        im[u] += p.y;
      }
    }
  }
  const double hr = block_sum(re[0] + re[1], sh);
  const double hi = block_sum(im[0] + im[1], sh);
  if (threadIdx.x == 0)
    a.part[(((size_t)s * (a.m + 1) + c) * kDotChunks) + chunk] = make_double2(hr, hi);
}

// w -= V h on kUpdRows rows per block, h_c = sum of the kDotChunks partials of k_dots (summed
// in order by every block). Thread (row, g) sums the columns c = g, g + 4, ...; the four group
// sums are added in a fixed order. Block 0 records h: pass 0 stores it in hcol, pass 1 adds it
// (the re-orthogonalisation correction) to hcol. Pass 1 also writes the block's ||w||^2.
__global__ void __launch_bounds__(256) k_update(GArgs a, int pass) {
  __shared__ double2 s_h[256];
  __shared__ double2 s_acc[4][kUpdRows];
  __shared__ double sh[32];
  if (a.scal[1]) return;
  const int s = blockIdx.y;
  const int j = a.scal[0];
  const bool active = !a.done[s];
  if (active) {
    for (int c = threadIdx.x; c <= j; c += blockDim.x) {
      const double2* pc = a.part + ((size_t)s * (a.m + 1) + c) * kDotChunks;
      double2 t = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kDotChunks; ++q) t = cadd(t, pc[q]);
      s_h[c] = t;
      if (blockIdx.x == 0) {
        const size_t o = (size_t)s * (a.m + 1) + c;
        a.hcol[o] = pass == 0 ? t : cadd(a.hcol[o], t);
      }
    }
  }
  __syncthreads();
  const int lr = threadIdx.x & (kUpdRows - 1), g = threadIdx.x / kUpdRows;
  const int r = blockIdx.x * kUpdRows + lr;
  double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
  if (active && r < a.n) {
    int c = g;
    for (; c + 4 <= j; c += 8) {
      acc0 = cadd(acc0, cmul(a.V[vidx(a, c, s) + r], s_h[c]));
      acc1 = cadd(acc1, cmul(a.V[vidx(a, c + 4, s) + r], s_h[c + 4]));
    }
    if (c <= j) acc0 = cadd(acc0, cmul(a.V[vidx(a, c, s) + r], s_h[c]));
  }
  s_acc[g][lr] = cadd(acc0, acc1);
  __syncthreads();
  double nv = 0.0;
  if (g == 0 && active && r < a.n) {
    const double2 t = cadd(cadd(s_acc[0][lr], s_acc[1][lr]), cadd(s_acc[2][lr], s_acc[3][lr]));
    const double2 w = csub(a.w[(size_t)s * a.n + r], t);
    a.w[(size_t)s * a.n + r] = w;
    nv = cabs2(w);
  }
  if (pass == 1) {
    nv = block_sum(nv, sh);
    if (threadIdx.x == 0) a.partn[(size_t)blockIdx.x * a.nrhs + s] = nv;
  }
}

// Thread 0 of the last block of k_finish: apply the earlier rotations (staged in s_hc / s_cs /
// s_sn) to the new column, make the rotation zeroing h_{j+1,j} = hn, update g and the residual
// estimate, write the column and the rotation back, and set the convergence flag.
#define givens_step(a, s, j, hn)                                                              \
  do {                                                                                        \
    const size_t ho_ = (size_t)(s) * ((a).m + 1);                                             \
    for (int i = 0; i < (j); ++i) {                                                           \
      const double2 h0 = s_hc[i], h1 = s_hc[i + 1];                                           \
      s_hc[i] = cadd(make_double2(s_cs[i] * h0.x, s_cs[i] * h0.y), cmul(s_sn[i], h1));        \
      s_hc[i + 1] = cadd(cmul(make_double2(-s_sn[i].x, s_sn[i].y), h0),                        \
                         make_double2(s_cs[i] * h1.x, s_cs[i] * h1.y));                         \
    }                                                                                         \
    const double2 h0 = s_hc[(j)];                                                             \
    const double a0 = sqrt(cabs2(h0));                                                        \
    const double rho = sqrt(a0 * a0 + (hn) * (hn));                                           \
    double c_;                                                                                \
    double2 sv, top;                                                                          \
    if (a0 == 0.0) {                                                                          \
      c_ = 0.0;                                                                               \
      sv = make_double2(1.0, 0.0);                                                            \
      top = make_double2((hn), 0.0);                                                          \
    } else {                                                                                  \
      c_ = a0 / rho;                                                                          \
      const double2 ph = make_double2(h0.x / a0, h0.y / a0);                                  \
      sv = make_double2(ph.x * (hn) / rho, ph.y * (hn) / rho);                                \
      top = make_double2(ph.x * rho, ph.y * rho);                                             \
    }                                                                                         \
    (a).cs[(size_t)(s) * (a).m + (j)] = c_;                                                   \
    (a).sn[(size_t)(s) * (a).m + (j)] = sv;                                                   \
    s_hc[(j)] = top;                                                                          \
    double2* gv_ = (a).gv + ho_;                                                              \
    const double2 gj = gv_[(j)];                                                              \
    gv_[(j) + 1] = cmul(make_double2(-sv.x, sv.y), gj);                                       \
    gv_[(j)] = make_double2(c_ * gj.x, c_ * gj.y);                                            \
    double2* Hcol = (a).H + ((size_t)(s) * (a).m + (j)) * ((a).m + 1);                        \
    for (int i = 0; i <= (j); ++i) Hcol[i] = s_hc[i];                                         \
    const double res_ = sqrt(cabs2(gv_[(j) + 1]));                                            \
    (a).res[s] = res_;                                                                        \
    (a).iters[s] = (j) + 1;                                                                   \
    if (res_ <= (a).tol * ((a).bscale ? (a).bscale[s] : (a).bnorm[s]) || (hn) == 0.0)      \
      (a).done[s] = 1;                                                                        \
  } while (0)

// ||w|| from the block partials and v = w / ||w|| into V[jt] and the FP32 copy xf.
// mode 0 starts a run (jt = 0, ||w|| = ||b||); mode 1 ends iteration j (jt = j + 1): the last
// block per RHS applies the earlier Givens rotations to the new Hessenberg column, makes the
// rotation that zeroes h_{j+1,j}, updates the residual estimate |g_{j+1}| and the convergence
// flag; the last RHS to finish advances j and sets the "all done" flag.
__global__ void __launch_bounds__(256) k_finish(GArgs a, int mode) {
  __shared__ double sh[32];
  __shared__ double2 s_hc[256], s_sn[256];
  __shared__ double s_cs[256];
  if (mode == 1 && a.scal[1]) return;
  const int s = blockIdx.y;
  const int j = a.scal[0];
  const bool active = mode == 0 ? !(a.skip && a.skip[s]) : !a.done[s];
  const int jt = mode == 0 ? 0 : j + 1;
  double t = 0.0;
  for (int q = threadIdx.x; q < a.nchunk; q += blockDim.x) t += a.partn[(size_t)q * a.nrhs + s];
  t = block_sum(t, sh);
  const double hn = sqrt(t);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (active && hn > 0.0 && r < a.n) {
    const double inv = 1.0 / hn;
    const double2 ww = a.w[(size_t)s * a.n + r];
    const double2 v = make_double2(ww.x * inv, ww.y * inv);
    const float2 vf = make_float2((float)v.x, (float)v.y);
    if (a.Vf)
      a.Vf[vidx(a, jt, s) + r] = vf;
    else
      a.V[vidx(a, jt, s) + r] = v;
    a.xf[(size_t)s * a.ld + r] = vf;
  }
  if (!last_block(a.cnt + s * kCounters + 0, gridDim.x)) return;
  if (mode == 1 && active) {
    // stage the Hessenberg column and the earlier rotations in shared memory (parallel loads),
    // so the serial rotation chain below runs at shared-memory latency
    const size_t ho = (size_t)s * (a.m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      s_hc[i] = a.hcol[ho + i];
      if (i < j) {
        s_cs[i] = a.cs[(size_t)s * a.m + i];
        s_sn[i] = a.sn[(size_t)s * a.m + i];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const size_t ho = (size_t)s * (a.m + 1);
  if (mode == 0) {
    a.bnorm[s] = hn;
    a.hnorm[s] = hn;
    a.gv[ho] = make_double2(hn, 0.0);
    a.res[s] = hn;
    a.iters[s] = 0;
    a.done[s] = (hn == 0.0) || !active;
  } else if (active) {
    a.hnorm[s] = hn;
    givens_step(a, s, j, hn);
  }
  __threadfence();
  const unsigned t2 = atomicAdd((unsigned*)&a.scal[2], 1u);
  if (t2 == (unsigned)a.nrhs - 1) {
    a.scal[2] = 0;
    int all = 1;
    for (int q = 0; q < a.nrhs; ++q) all &= a.done[q];
    const int jn = mode == 0 ? 0 : j + 1;
    a.scal[0] = jn;
    a.scal[1] = all || jn >= a.maxit;
  }
}

// ------------------------------------------------- fused Krylov step (cooperative launch)
// Grid barrier for a cooperative launch (every block co-resident): arrival count plus a
// generation number, with release/acquire atomics at GPU scope instead of full fences: the
// arrival (acq_rel) publishes the block's writes, which __syncthreads has ordered before it,
// and the waiters' acquire loads of the new generation make every block's writes visible.
// Bounded: a wait longer than about two seconds sets err bit 64 and goes on.
__device__ __forceinline__ void grid_sync(unsigned* count, unsigned* gen, unsigned nblocks, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g, old;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
    if (old == nblocks - 1u) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
    } else {
      uint64_t t0, t;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
      for (unsigned it = 1;; ++it) {
        unsigned cur;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
        if (cur != g) break;
        if ((it & 255u) == 0u) {
          asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
          if (t - t0 > 2000000000ull) {
            atomicOr(err, 64);
            break;
          }
        }
      }
    }
  }
  __syncthreads();
}

// One GMRES iteration after the matvec, in one cooperative launch: classical Gram-Schmidt with
// selective re-orthogonalisation (a second pass on strong cancellation, the test of Daniel,
// Gragg, Kaufman and Stewart 1976 with a tighter threshold), ||w||, v_{j+1} and the Givens
// update, all in FP64.
//
// Blocks 1..G-1 own contiguous row ranges of every vector; block 0 owns no rows and runs the
// Givens steps, so the rotation scan overlaps the other blocks' row updates. A pass is
//   (A) per block and RHS, partial sums over its rows of conj(V_c) . w for c <= j and of ||w||^2
//       (eight lanes per column, reduced with three shuffle levels), stored per block; the
//       block's panel of V is first staged in shared memory with 16-byte asynchronous copies
//       when it fits, so the pass costs one round trip to memory;
//   barrier; (R) each (RHS, column) total summed over the blocks in a fixed order by one warp;
//   barrier; (B) every block reads h and ||w||^2 and takes ||w - V h||^2 = ||w||^2 - ||h||^2
//       (V orthonormal), then updates its rows: w -= V h.
// If ||w - V h||^2 <= 1e-4 ||w||^2 (w within 1% of span V), a second pass runs on the updated w
// and its h is added to the first. Otherwise v_{j+1} = (w - V h) / ||w - V h|| is written
// directly by the update, so the common iteration has two grid barriers. Every block computes
// the same totals in the same order, so all blocks take the same decisions.
// 1 / sqrt(x) for x > 0: an FP32 seed (about 22 bits) and two Newton steps y += y (1 - x y^2) / 2,
// each doubling the correct bits. GB300 runs a dependent FP64 operation in ~66 clocks and an
// FP64 square root or division in ~650, so this is half the latency of sqrt plus a division.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);  // outside the FP32 seed's range
  double y = (double)rsqrtf((float)x);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double r = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, r, y);
  }
  return y;
}

// The Givens update of GMRES for RHS s after iteration j, by one warp. The new Hessenberg column
// hc[0..j] (shared memory) gets the earlier rotations (c_i real, s_i complex) applied in order:
//   out_i = c_i t_i + s_i h_{i+1},   t_{i+1} = -conj(s_i) t_i + c_i h_{i+1},   t_0 = h_0,
// an affine recurrence in t, so the warp computes all t_i by a prefix scan of the maps
// t -> a t + b (each lane composes a contiguous segment, then five shuffle levels) instead of a
// serial chain of j rotations. The new rotation zeroes h_{j+1,j} = hn against t_j; |g_{j+1}| =
// |s_j| |g_j| gives the residual estimate without a square root.
__device__ void givens_warp(const GArgs& a, int s, int j, double hn, double2* hc, const double* cs,
                            const double2* sn, int lane) {
  const int S = (j + 31) / 32;                 // recurrence steps per lane
  const int i0 = min(j, lane * S), i1 = min(j, i0 + S);
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);  // segment map t -> A t + B
  for (int i = i0; i < i1; ++i) {
    const double2 ai = make_double2(-sn[i].x, sn[i].y);
    const double2 bi = make_double2(cs[i] * hc[i + 1].x, cs[i] * hc[i + 1].y);
    A = cmul(ai, A);
    B = cadd(cmul(ai, B), bi);
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {  // inclusive scan: this map after the earlier lanes' maps
    const double2 Ap = make_double2(__shfl_up_sync(0xffffffffu, A.x, o), __shfl_up_sync(0xffffffffu, A.y, o));
    const double2 Bp = make_double2(__shfl_up_sync(0xffffffffu, B.x, o), __shfl_up_sync(0xffffffffu, B.y, o));
    if (lane >= o) {
      B = cadd(cmul(A, Bp), B);
      A = cmul(A, Ap);
    }
  }
  // exclusive prefix: the map from t_0 to t_{i0}
  double2 Ae = make_double2(__shfl_up_sync(0xffffffffu, A.x, 1), __shfl_up_sync(0xffffffffu, A.y, 1));
  double2 Be = make_double2(__shfl_up_sync(0xffffffffu, B.x, 1), __shfl_up_sync(0xffffffffu, B.y, 1));
  if (lane == 0) {
    Ae = make_double2(1.0, 0.0);
    Be = make_double2(0.0, 0.0);
  }
  const double2 h0 = hc[0];
  double2 t = cadd(cmul(Ae, h0), Be);
  const size_t ho = (size_t)s * (a.m + 1);
  double2* Hcol = a.H + ((size_t)s * a.m + j) * (a.m + 1);
  for (int i = i0; i < i1; ++i) {  // rotated entries 0..j-1 straight to the Hessenberg matrix
    const double2 h1 = hc[i + 1];
    Hcol[i] = cadd(make_double2(cs[i] * t.x, cs[i] * t.y), cmul(sn[i], h1));
    t = cadd(cmul(make_double2(-sn[i].x, sn[i].y), t), make_double2(cs[i] * h1.x, cs[i] * h1.y));
  }
  // t_j sits in the lane whose segment ends at j (lane 0 when j == 0)
  const int owner = j == 0 ? 0 : (j - 1) / S;
  t = make_double2(__shfl_sync(0xffffffffu, t.x, owner), __shfl_sync(0xffffffffu, t.y, owner));
  if (lane == 0) {
    const double q = cabs2(t);
    double c, absS;
    double2 sv, top;
    if (q == 0.0) {
      c = 0.0;
      absS = 1.0;
      sv = make_double2(1.0, 0.0);
      top = make_double2(hn, 0.0);
    } else {
      const double ia = rsqrt_nr(q);             // 1 / |t_j|
      const double rho2 = q + hn * hn;
      const double ir = rsqrt_nr(rho2);          // 1 / rho
      const double rho = rho2 * ir;
      const double2 ph = make_double2(t.x * ia, t.y * ia);
      c = q * ia * ir;                           // |t_j| / rho
      absS = hn * ir;
      sv = make_double2(ph.x * absS, ph.y * absS);
      top = make_double2(ph.x * rho, ph.y * rho);
    }
    a.cs[(size_t)s * a.m + j] = c;
    a.sn[(size_t)s * a.m + j] = sv;
    Hcol[j] = top;
    double2* gv = a.gv + ho;
    const double2 gj = gv[j];
    gv[j + 1] = cmul(make_double2(-sv.x, sv.y), gj);
    gv[j] = make_double2(c * gj.x, c * gj.y);
    const double res = absS * a.res[s];
    a.res[s] = res;
    a.hnorm[s] = hn;
    a.iters[s] = j + 1;
    if (res <= a.tol * (a.bscale ? a.bscale[s] : a.bnorm[s]) || hn == 0.0) a.done[s] = 1;
  }
}

constexpr int kArnMaxRows = 512;           // rows per block (n <= 151 * 512 with 152 blocks)
// dynamic shared memory for the V panel. With 96 KiB one fused kernel is resident per SM at a
// time; with solves in flight on several streams this measured faster (102 solves/s at four
// in flight) than 72 KiB with 64 registers a thread, which lets two fused kernels and more
// matvec blocks share an SM (75 solves/s).
constexpr int kArnPanelBytes = 96 * 1024;
// The FP32 panel of inner solves: half the bytes per vector, and 48 KiB (about 90 vectors of a
// block's rows at n = 10240, more than an inner solve reaches) let the kernels of two solves in
// flight share an SM: 125.3 against 123.6 solves/s with 96 KiB on the four-in-flight bench
// (64 KiB: 122.9; 32 KiB: 125.4).
constexpr int kArnPanelBytesF32 = 48 * 1024;
constexpr int kArnMaxRhs = 256;
constexpr int kArnUnitsMinRhs = 4;  // more right-hand sides than this: k_arnoldi_units
constexpr int kArnUnitsPerSm = 2;   // k_arnoldi_units: blocks per SM (at most)
// mixed refinement: a stalled sweep with every open true residual within this factor of the
// tolerance ends the solve (the FP32 residual product's rounding floor)
constexpr double kResidualFloor = 4.0;
// mixed refinement: the inner tolerance of a sweep is inner_tol, loosened once the open true
// residuals are close to the target: kSweepMargin x (tol / largest open residual) is the
// contraction still missing (with a margin), rounded down to inner_tol x 2^e, e <= kSweepMaxDoubling
// (few distinct values, so few captured graphs)
// (measured on the 10240-triangle interior-source workload, 64 k, 4 in flight, solves/s:
// 0.15: 136.2, 0.3: 139.1, 0.5: 142.6-143.2, 0.7: 144.4, 1.0: 144.0)
constexpr double kSweepMargin = 0.7;
constexpr int kSweepMaxDoubling = 5;

// The inner tolerance of the next refinement sweep when the largest open relative residual is
// rho (tol: the outer target; base: the configured inner tolerance).
inline double sweep_inner_tol(double base, double tol, double rho) {
  double want = base;
  const double missing = kSweepMargin * tol / std::max(rho, 1e-300);
  for (int e = 0; e < kSweepMaxDoubling && 2.0 * want <= missing && 2.0 * want < 1.0; ++e) want *= 2.0;
  return want;
}

// Rows per work unit of k_arnoldi_units: about four units per block, 64 <= unit <= n.
inline int arnoldi_unit(int n, int nrhs, int blocks) {
  int64_t u = ((int64_t)n * nrhs / (4 * (int64_t)blocks) + 31) / 32 * 32;
  u = std::max<int64_t>(64, u);
  return (int)std::min<int64_t>(u, n);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(256, 2) k_arnoldi(GArgs a, double2* __restrict__ pb, double2* __restrict__ hr,
                                                 unsigned* __restrict__ bar, int* __restrict__ err,
                                                 int pcap) {
  extern __shared__ double2 s_panel[];  // V_0..V_j on this block's rows (one RHS), when it fits
  __shared__ double2 s_w[kArnMaxRows];
  __shared__ double2 s_h[256];
  __shared__ double2 s_acc[256];
  __shared__ double2 s_sn[256];
  __shared__ double s_cs[256];
  __shared__ unsigned char s_act[kArnMaxRhs];  // 1: active, 2: active and re-orthogonalised
  __shared__ double s_hn[kArnMaxRhs], s_inv[kArnMaxRhs];
  if (a.scal[1]) return;
  const int j = a.scal[0];
  const int G = (int)gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = (a.n + G - 2) / (G - 1);
  const int r0 = b == 0 ? 0 : min(a.n, (b - 1) * R), r1 = b == 0 ? 0 : min(a.n, r0 + R);
  const int rows = r1 - r0;
  const int np = j + 2;                   // columns 0..j and ||w||^2
  const size_t ps = (size_t)(a.m + 2);    // per-RHS stride of pb (times G) and hr
  const bool panel = (j + 1) * rows <= pcap;  // the block's V panel is staged in shared memory
  for (int s = threadIdx.x; s < a.nrhs; s += blockDim.x) s_act[s] = a.done[s] ? 0 : 1;
  __syncthreads();

  for (int pass = 0; pass < 2; ++pass) {
    const unsigned char want = pass == 0 ? 1 : 2;
    bool any = false;
    for (int s = 0; s < a.nrhs; ++s) any |= (s_act[s] >= want);
    if (!any) break;  // uniform: every block holds the same flags
    // (A) partial sums over this block's rows
    if (b > 0) {
      const int l8 = lane & 7;
      for (int s = 0; s < a.nrhs; ++s) {
        if (s_act[s] < want) continue;
        const double2* w = a.w + (size_t)s * a.n + r0;
        if (panel) {  // one round trip for the whole panel: 16-byte asynchronous copies
          for (int e = threadIdx.x; e < (j + 1) * rows; e += blockDim.x) {
            const int c = e / rows, r = e - c * rows;
            cp_async16(&s_panel[e], a.V + vidx(a, c, s) + r0 + r);
          }
        }
        for (int r = threadIdx.x; r < rows; r += blockDim.x) s_w[r] = w[r];
        if (panel) cp_async_wait_all();
        __syncthreads();
        for (int c0 = warp * 4; c0 < np; c0 += 32) {  // same trip count in every lane of a warp
          const int c = c0 + (lane >> 3);
          double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
          if (c <= j && panel) {
            const double2* v = s_panel + c * rows;
            for (int r = l8; r < rows; r += 16) {
              const double2 v0 = v[r], w0 = s_w[r];
              re0 = fma(v0.x, w0.x, re0);
              re0 = fma(v0.y, w0.y, re0);
              im0 = fma(v0.x, w0.y, im0);
              im0 = fma(-v0.y, w0.x, im0);
              if (r + 8 < rows) {
                const double2 v1 = v[r + 8], w1 = s_w[r + 8];
                re1 = fma(v1.x, w1.x, re1);
                re1 = fma(v1.y, w1.y, re1);
                im1 = fma(v1.x, w1.y, im1);
                im1 = fma(-v1.y, w1.x, im1);
              }
            }
          } else if (c <= j) {
            // conj(v) . w as four FMA chains; eight loads issued before they are used
            const double2* v = a.V + vidx(a, c, s) + r0;
            for (int rb = l8; rb < rows; rb += 64) {
              double2 vv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int r = rb + 8 * u;
                vv[u] = r < rows ? v[r] : make_double2(0.0, 0.0);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int r = rb + 8 * u;
                const double2 ww = r < rows ? s_w[r] : make_double2(0.0, 0.0);
                double& re = (u & 1) ? re1 : re0;
                double& im = (u & 1) ? im1 : im0;
                re = fma(vv[u].x, ww.x, re);
                re = fma(vv[u].y, ww.y, re);
                im = fma(vv[u].x, ww.y, im);
                im = fma(-vv[u].y, ww.x, im);
              }
            }
          } else if (c == j + 1) {
            for (int r = l8; r < rows; r += 16) {
              const double2 w0 = s_w[r];
              re0 = fma(w0.x, w0.x, re0);
              re0 = fma(w0.y, w0.y, re0);
              if (r + 8 < rows) {
                const double2 w1 = s_w[r + 8];
                re1 = fma(w1.x, w1.x, re1);
                re1 = fma(w1.y, w1.y, re1);
              }
            }
          }
          double re = re0 + re1, im = im0 + im1;
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
          }
          if (l8 == 0 && c < np) pb[((size_t)s * ps + c) * G + b] = make_double2(re, im);
        }
        __syncthreads();
      }
    } else if (a.nrhs == 1 && pass == 0) {
      // block 0 owns no rows: while the others form their partial sums it fetches the earlier
      // rotations its Givens update needs after the second barrier
      for (int c = threadIdx.x; c < j; c += blockDim.x) {
        s_cs[c] = a.cs[c];
        s_sn[c] = a.sn[c];
      }
    }
    grid_sync(bar, bar + 1, G, err);
    // (R) totals over blocks 1..G-1, one warp per (RHS, column), fixed order
    {
      const int items = a.nrhs * np;
      for (int it = b * 8 + warp; it < items; it += G * 8) {
        const int s = it / np, c = it % np;
        if (s_act[s] < want) continue;
        const double2* src = pb + ((size_t)s * ps + c) * G;
        double re = 0.0, im = 0.0;
        for (int qb = 1 + lane; qb < G; qb += 256) {  // eight loads in flight per lane
          double2 t[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) t[u] = qb + 32 * u < G ? src[qb + 32 * u] : make_double2(0.0, 0.0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            re += t[u].x;
            im += t[u].y;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, o);
          im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) hr[(size_t)s * ps + c] = make_double2(re, im);
      }
    }
    grid_sync(bar, bar + 1, G, err);
    // (B) decisions, row updates, v_{j+1}; block s mod G: Hessenberg column and Givens of RHS s
    for (int s = 0; s < a.nrhs; ++s) {
      if (s_act[s] < want) continue;
      const double2* hs = hr + (size_t)s * ps;
      for (int c = threadIdx.x; c <= j + 1; c += blockDim.x) s_h[c] = hs[c];  // with ||w||^2
      __syncthreads();
      if (warp == 0) {
        double t = 0.0;
        for (int c = lane; c <= j; c += 32) t += cabs2(s_h[c]);
        t = warp_sum(t);
        if (lane == 0) {
          const double wn2 = s_h[j + 1].x;
          const double hn2 = fmax(wn2 - t, 0.0);
          // second pass only after cancellation by more than 100x in ||w - V h||: one FP64
          // pass then leaves components ~1e-14 along V, far below what GMRES notices
          const bool again = pass == 0 && !(hn2 > 1e-4 * wn2);
          const double inv = hn2 > 0.0 ? rsqrt_nr(hn2) : 0.0;
          s_hn[s] = again ? -1.0 : hn2 * inv;
          s_inv[s] = inv;
          if (again) s_act[s] = 2;
        }
      }
      __syncthreads();
      const double hn = s_hn[s];
      const bool last = hn >= 0.0;  // this pass finishes the column
      if (b == s % G) {
        // the Hessenberg column: h of this pass, plus the first pass's h after a second pass
        const size_t ho = (size_t)s * (a.m + 1);
        for (int c = threadIdx.x; c <= j; c += blockDim.x) {
          const double2 t = pass == 0 ? s_h[c] : cadd(a.hcol[ho + c], s_h[c]);
          if (!last) a.hcol[ho + c] = t;
          s_acc[c] = t;
          if (c < j && a.nrhs > 1) {  // one RHS: block 0 fetched them during the partial sums
            s_cs[c] = a.cs[(size_t)s * a.m + c];
            s_sn[c] = a.sn[(size_t)s * a.m + c];
          }
        }
        __syncthreads();
        if (last && warp == 0) givens_warp(a, s, j, hn, s_acc, s_cs, s_sn, lane);
        __syncthreads();
      }
      if (b > 0 && rows > 0) {
        const double inv = s_inv[s];
        for (int rc = 0; rc < rows; rc += 256) {
          const int nr = min(256, rows - rc);
          const int ng = 256 / nr;
          const int lr = threadIdx.x % nr, g = threadIdx.x / nr;
          const int r = r0 + rc + lr;
          double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
          if (g < ng) {
            // sum over c = g, g + ng, ... of V_c h_c: eight loads in flight, FMA chains; the
            // staged panel still holds V when there is one RHS
            const bool from_panel = panel && a.nrhs == 1;
            for (int cb = g; cb <= j; cb += 8 * ng) {
              double2 vv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int c = cb + u * ng;
                vv[u] = c > j ? make_double2(0.0, 0.0)
                              : (from_panel ? s_panel[c * rows + rc + lr] : a.V[vidx(a, c, s) + r]);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int c = cb + u * ng;
                const double2 h = c <= j ? s_h[c] : make_double2(0.0, 0.0);
                double2& acc = (u & 1) ? acc1 : acc0;
                acc.x = fma(vv[u].x, h.x, acc.x);
                acc.x = fma(-vv[u].y, h.y, acc.x);
                acc.y = fma(vv[u].x, h.y, acc.y);
                acc.y = fma(vv[u].y, h.x, acc.y);
              }
            }
          }
          s_acc[threadIdx.x] = cadd(acc0, acc1);
          __syncthreads();
          if (threadIdx.x < nr) {
            double2 t = s_acc[threadIdx.x];
            for (int q = 1; q < ng; ++q) t = cadd(t, s_acc[q * nr + threadIdx.x]);
            const double2 w = csub(a.w[(size_t)s * a.n + r], t);
            if (!last) {
              a.w[(size_t)s * a.n + r] = w;
            } else if (hn > 0.0) {
              const double2 v = make_double2(w.x * inv, w.y * inv);
              a.V[vidx(a, j + 1, s) + r] = v;
              a.xf[(size_t)s * a.ld + r] = make_float2((float)v.x, (float)v.y);
            }
          }
          __syncthreads();
        }
      }
    }
  }
  if (a.nrhs > 1) grid_sync(bar, bar + 1, G, err);  // every Givens update before the flags are read
  if (b == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int q = 0; q < a.nrhs; ++q) all &= a.done[q];
    a.scal[0] = j + 1;
    a.scal[1] = all || j + 1 >= a.maxit;
  }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// k_arnoldi on the FP32 basis of inner refinement solves (a.Vf, a.wf): the block's panel of
// V is staged as FP32 (twice the columns fit), the dots and the row updates run in FP32 with
// FP32 lane and warp sums, the block partials, totals, Hessenberg column and rotations stay
// FP64. Same blocks, barriers, decisions and second-pass test as k_arnoldi. pcap counts float2.
__global__ void __launch_bounds__(256, 2) k_arnoldi_f32(GArgs a, double2* __restrict__ pb, double2* __restrict__ hr,
                                                     unsigned* __restrict__ bar, int* __restrict__ err,
                                                     int pcap) {
  extern __shared__ float2 s_pf[];  // Vf_0..Vf_j on this block's rows (one RHS), when it fits
  __shared__ float2 s_wf[kArnMaxRows];
  __shared__ double2 s_h[256];
  __shared__ float2 s_hf[256];
  __shared__ double2 s_acc[256];
  __shared__ float2 s_accf[256];
  __shared__ double2 s_sn[256];
  __shared__ double s_cs[256];
  __shared__ unsigned char s_act[kArnMaxRhs];
  __shared__ double s_hn[kArnMaxRhs], s_inv[kArnMaxRhs];
  if (a.scal[1]) return;
  const int j = a.scal[0];
  const int G = (int)gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = (a.n + G - 2) / (G - 1);
  const int r0 = b == 0 ? 0 : min(a.n, (b - 1) * R), r1 = b == 0 ? 0 : min(a.n, r0 + R);
  const int rows = r1 - r0;
  const int np = j + 2;
  const size_t ps = (size_t)(a.m + 2);
  const bool panel = (j + 1) * rows <= pcap;
  for (int s = threadIdx.x; s < a.nrhs; s += blockDim.x) s_act[s] = a.done[s] ? 0 : 1;
  __syncthreads();

  for (int pass = 0; pass < 2; ++pass) {
    const unsigned char want = pass == 0 ? 1 : 2;
    bool any = false;
    for (int s = 0; s < a.nrhs; ++s) any |= (s_act[s] >= want);
    if (!any) break;
    // (A) partial sums over this block's rows; w is L v_j (FP64) in the first pass and the
    // FP32 w - V h that the first pass left in wf in the second
    if (b > 0) {
      const int l8 = lane & 7;
      for (int s = 0; s < a.nrhs; ++s) {
        if (s_act[s] < want) continue;
        if (panel) {
          for (int e = threadIdx.x; e < (j + 1) * rows; e += blockDim.x) {
            const int c = e / rows, r = e - c * rows;
            cp_async8(&s_pf[e], a.Vf + vidx(a, c, s) + r0 + r);
          }
        }
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
          if (pass == 0) {
            const double2 ww = a.w[(size_t)s * a.n + r0 + r];
            s_wf[r] = make_float2((float)ww.x, (float)ww.y);
          } else {
            s_wf[r] = a.wf[(size_t)s * a.n + r0 + r];
          }
        }
        if (panel) cp_async_wait_all();
        __syncthreads();
        for (int c0 = warp * 4; c0 < np; c0 += 32) {
          const int c = c0 + (lane >> 3);
          float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
          if (c <= j) {
            const float2* v = panel ? s_pf + c * rows : a.Vf + vidx(a, c, s) + r0;
            for (int r = l8; r < rows; r += 16) {
              const float2 v0 = v[r], w0 = s_wf[r];
              re0 = fmaf(v0.x, w0.x, re0);
              re0 = fmaf(v0.y, w0.y, re0);
              im0 = fmaf(v0.x, w0.y, im0);
              im0 = fmaf(-v0.y, w0.x, im0);
              if (r + 8 < rows) {
                const float2 v1 = v[r + 8], w1 = s_wf[r + 8];
                re1 = fmaf(v1.x, w1.x, re1);
                re1 = fmaf(v1.y, w1.y, re1);
                im1 = fmaf(v1.x, w1.y, im1);
                im1 = fmaf(-v1.y, w1.x, im1);
              }
            }
          } else if (c == j + 1) {
            for (int r = l8; r < rows; r += 16) {
              const float2 w0 = s_wf[r];
              re0 = fmaf(w0.x, w0.x, re0);
              re0 = fmaf(w0.y, w0.y, re0);
              if (r + 8 < rows) {
                const float2 w1 = s_wf[r + 8];
                re1 = fmaf(w1.x, w1.x, re1);
                re1 = fmaf(w1.y, w1.y, re1);
              }
            }
          }
          float re = re0 + re1, im = im0 + im1;
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
          }
          if (l8 == 0 && c < np) pb[((size_t)s * ps + c) * G + b] = make_double2((double)re, (double)im);
        }
        __syncthreads();
      }
    } else if (a.nrhs == 1 && pass == 0) {
      // block 0 owns no rows: while the others form their partial sums it fetches the earlier
      // rotations its Givens update needs after the second barrier
      for (int c = threadIdx.x; c < j; c += blockDim.x) {
        s_cs[c] = a.cs[c];
        s_sn[c] = a.sn[c];
      }
    }
    grid_sync(bar, bar + 1, G, err);
    // (R) totals over blocks 1..G-1, one warp per (RHS, column), fixed order
    {
      const int items = a.nrhs * np;
      for (int it = b * 8 + warp; it < items; it += G * 8) {
        const int s = it / np, c = it % np;
        if (s_act[s] < want) continue;
        const double2* src = pb + ((size_t)s * ps + c) * G;
        double re = 0.0, im = 0.0;
        for (int qb = 1 + lane; qb < G; qb += 256) {
          double2 t[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) t[u] = qb + 32 * u < G ? src[qb + 32 * u] : make_double2(0.0, 0.0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            re += t[u].x;
            im += t[u].y;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, o);
          im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) hr[(size_t)s * ps + c] = make_double2(re, im);
      }
    }
    grid_sync(bar, bar + 1, G, err);
    // (B) decisions, row updates, v_{j+1}; block s mod G: Hessenberg column and Givens of RHS s
    for (int s = 0; s < a.nrhs; ++s) {
      if (s_act[s] < want) continue;
      const double2* hs = hr + (size_t)s * ps;
      for (int c = threadIdx.x; c <= j + 1; c += blockDim.x) {  // with ||w||^2
        s_h[c] = hs[c];
        if (c <= j) s_hf[c] = make_float2((float)hs[c].x, (float)hs[c].y);
      }
      __syncthreads();
      if (warp == 0) {
        double t = 0.0;
        for (int c = lane; c <= j; c += 32) t += cabs2(s_h[c]);
        t = warp_sum(t);
        if (lane == 0) {
          const double wn2 = s_h[j + 1].x;
          const double hn2 = fmax(wn2 - t, 0.0);
          const bool again = pass == 0 && !(hn2 > 1e-4 * wn2);
          const double inv = hn2 > 0.0 ? rsqrt_nr(hn2) : 0.0;
          s_hn[s] = again ? -1.0 : hn2 * inv;
          s_inv[s] = inv;
          if (again) s_act[s] = 2;
        }
      }
      __syncthreads();
      const double hn = s_hn[s];
      const bool last = hn >= 0.0;
      if (b == s % G) {
        const size_t ho = (size_t)s * (a.m + 1);
        for (int c = threadIdx.x; c <= j; c += blockDim.x) {
          const double2 t = pass == 0 ? s_h[c] : cadd(a.hcol[ho + c], s_h[c]);
          if (!last) a.hcol[ho + c] = t;
          s_acc[c] = t;
          if (c < j && a.nrhs > 1) {  // one RHS: block 0 fetched them during the partial sums
            s_cs[c] = a.cs[(size_t)s * a.m + c];
            s_sn[c] = a.sn[(size_t)s * a.m + c];
          }
        }
        __syncthreads();
        if (last && warp == 0) givens_warp(a, s, j, hn, s_acc, s_cs, s_sn, lane);
        __syncthreads();
      }
      if (b > 0 && rows > 0) {
        const float finv = (float)s_inv[s];
        for (int rc = 0; rc < rows; rc += 256) {
          const int nr = min(256, rows - rc);
          const int ng = 256 / nr;
          const int lr = threadIdx.x % nr, g = threadIdx.x / nr;
          const int r = r0 + rc + lr;
          float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
          if (g < ng) {
            const bool from_panel = panel && a.nrhs == 1;
            for (int cb = g; cb <= j; cb += 8 * ng) {
              float2 vv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int c = cb + u * ng;
                vv[u] = c > j ? make_float2(0.f, 0.f)
                              : (from_panel ? s_pf[c * rows + rc + lr] : a.Vf[vidx(a, c, s) + r]);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int c = cb + u * ng;
                const float2 h = c <= j ? s_hf[c] : make_float2(0.f, 0.f);
                float2& acc = (u & 1) ? acc1 : acc0;
                acc.x = fmaf(vv[u].x, h.x, acc.x);
                acc.x = fmaf(-vv[u].y, h.y, acc.x);
                acc.y = fmaf(vv[u].x, h.y, acc.y);
                acc.y = fmaf(vv[u].y, h.x, acc.y);
              }
            }
          }
          s_accf[threadIdx.x] = make_float2(acc0.x + acc1.x, acc0.y + acc1.y);
          __syncthreads();
          if (threadIdx.x < nr) {
            float2 t = s_accf[threadIdx.x];
            for (int q = 1; q < ng; ++q) t = make_float2(t.x + s_accf[q * nr + threadIdx.x].x, t.y + s_accf[q * nr + threadIdx.x].y);
            float2 w;
            if (pass == 0) {
              const double2 ww = a.w[(size_t)s * a.n + r];
              w = make_float2((float)ww.x, (float)ww.y);
            } else {
              w = a.wf[(size_t)s * a.n + r];
            }
            w = make_float2(w.x - t.x, w.y - t.y);
            if (!last) {
              a.wf[(size_t)s * a.n + r] = w;
            } else if (hn > 0.0) {
              const float2 v = make_float2(w.x * finv, w.y * finv);
              a.Vf[vidx(a, j + 1, s) + r] = v;
              a.xf[(size_t)s * a.ld + r] = v;
            }
          }
          __syncthreads();
        }
      }
    }
  }
  if (a.nrhs > 1) grid_sync(bar, bar + 1, G, err);
  if (b == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int q = 0; q < a.nrhs; ++q) all &= a.done[q];
    a.scal[0] = j + 1;
    a.scal[1] = all || j + 1 >= a.maxit;
  }
}

// The same iteration for several right-hand sides, one cooperative launch. The work is dealt
// in units of (RHS s, row range of `unit` rows): block b takes units b, b + G, ..., so every
// block streams long coalesced row ranges of V with no per-RHS barrier, and the FP64 pipe stays
// busy. Per unit and pass: (A) partial dots of its rows for c <= j and ||w||^2 (warp c % 8 per
// column, lanes over rows, four accumulators), stored per (RHS, column, chunk); barrier; (R)
// totals over the chunks of each RHS, one thread per (RHS, column), fixed order; barrier; (B)
// every block takes the decisions for every RHS from the totals (so all blocks agree on the
// barrier count), then updates its units' rows, and the owner of chunk 0 of an RHS applies
// its Givens rotation. Same arithmetic and second-pass test as k_arnoldi.
// kF32: the FP32 basis of inner refinement solves (a.Vf, a.wf): the dots and the row updates
// run in FP32 (lane sums in FP32, unit and chunk totals, Hessenberg column and rotations in
// FP64), so the loop over the basis uses no FP64 instruction and reads half the bytes. An inner
// solve stops at a relative residual of 1e-2, far above the FP32 basis' loss of orthogonality.
template <bool kF32>
__global__ void __launch_bounds__(256) k_arnoldi_units(GArgs a, double2* __restrict__ pbu, double2* __restrict__ hr,
                                                       unsigned* __restrict__ bar, int* __restrict__ err,
                                                       int unit, int cps) {
  __shared__ float2 s_hf[256];
  __shared__ double2 s_h[256];
  __shared__ double2 s_acc[256];
  __shared__ double2 s_sn[256];
  __shared__ double s_cs[256];
  __shared__ unsigned char s_act[kArnMaxRhs];
  __shared__ double s_hn[kArnMaxRhs], s_inv[kArnMaxRhs];
  if (a.scal[1]) return;
  const int j = a.scal[0];
  const int G = (int)gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np = j + 2;
  const size_t ps = (size_t)(a.m + 2);
  const int nunits = a.nrhs * cps;
  for (int q = threadIdx.x; q < a.nrhs; q += blockDim.x) s_act[q] = a.done[q] ? 0 : 1;
  __syncthreads();

  for (int pass = 0; pass < 2; ++pass) {
    const unsigned char want = pass == 0 ? 1 : 2;
    bool any = false;
    for (int q = 0; q < a.nrhs; ++q) any |= (s_act[q] >= want);
    if (!any) break;
    if constexpr (kF32) {
      // FP32 copy of this block's rows of w = L v_j (the second pass reads the w - V h that
      // the first pass left there)
      if (pass == 0) {
        for (int u = b; u < nunits; u += G) {
          const int s = u / cps, chunk = u % cps;
          if (s_act[s] < want) continue;
          const int q0 = chunk * unit, q1 = min(a.n, q0 + unit);
          for (int r = q0 + threadIdx.x; r < q1; r += blockDim.x) {
            const double2 ww = a.w[(size_t)s * a.n + r];
            a.wf[(size_t)s * a.n + r] = make_float2((float)ww.x, (float)ww.y);
          }
        }
      }
      __syncthreads();
      for (int u = b; u < nunits; u += G) {
        const int s = u / cps, chunk = u % cps;
        if (s_act[s] < want) continue;
        const int q0 = chunk * unit, q1 = min(a.n, q0 + unit);
        const float2* w = a.wf + (size_t)s * a.n;
        for (int c = warp; c < np; c += 8) {
          // eight rows per lane in flight (16 loads of 8 bytes)
          float re[8], im[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) re[t] = im[t] = 0.f;
          if (c <= j) {
            const float2* v = a.Vf + vidx(a, c, s);
            for (int r = q0 + lane; r < q1; r += 256) {
              float2 vv[8], ww[8];
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const int rr = r + 32 * t;
                vv[t] = rr < q1 ? v[rr] : make_float2(0.f, 0.f);
                ww[t] = rr < q1 ? w[rr] : make_float2(0.f, 0.f);
              }
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                re[t] = fmaf(vv[t].x, ww[t].x, re[t]);
                re[t] = fmaf(vv[t].y, ww[t].y, re[t]);
                im[t] = fmaf(vv[t].x, ww[t].y, im[t]);
                im[t] = fmaf(-vv[t].y, ww[t].x, im[t]);
              }
            }
          } else {
            for (int r = q0 + lane; r < q1; r += 256) {
              float2 ww[8];
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const int rr = r + 32 * t;
                ww[t] = rr < q1 ? w[rr] : make_float2(0.f, 0.f);
              }
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                re[t] = fmaf(ww[t].x, ww[t].x, re[t]);
                re[t] = fmaf(ww[t].y, ww[t].y, re[t]);
              }
            }
          }
          float sr = ((re[0] + re[1]) + (re[2] + re[3])) + ((re[4] + re[5]) + (re[6] + re[7]));
          float si = ((im[0] + im[1]) + (im[2] + im[3])) + ((im[4] + im[5]) + (im[6] + im[7]));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
          }
          if (lane == 0) pbu[((size_t)s * ps + c) * cps + chunk] = make_double2((double)sr, (double)si);
        }
      }
    } else {
    // (A) partial sums over each unit's rows
    for (int u = b; u < nunits; u += G) {
      const int s = u / cps, chunk = u % cps;
      if (s_act[s] < want) continue;
      const int q0 = chunk * unit, q1 = min(a.n, q0 + unit);
      const double2* w = a.w + (size_t)s * a.n;
      for (int c = warp; c < np; c += 8) {
        double re[4] = {0.0, 0.0, 0.0, 0.0}, im[4] = {0.0, 0.0, 0.0, 0.0};
        if (c <= j) {
          const double2* v = a.V + vidx(a, c, s);
          for (int r = q0 + lane; r < q1; r += 128) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int rr = r + 32 * t;
              if (rr < q1) {
                const double2 vv = v[rr], ww = w[rr];
                re[t] = fma(vv.x, ww.x, re[t]);
                re[t] = fma(vv.y, ww.y, re[t]);
                im[t] = fma(vv.x, ww.y, im[t]);
                im[t] = fma(-vv.y, ww.x, im[t]);
              }
            }
          }
        } else {
          for (int r = q0 + lane; r < q1; r += 128) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int rr = r + 32 * t;
              if (rr < q1) {
                const double2 ww = w[rr];
                re[t] = fma(ww.x, ww.x, re[t]);
                re[t] = fma(ww.y, ww.y, re[t]);
              }
            }
          }
        }
        double sr = (re[0] + re[1]) + (re[2] + re[3]), si = (im[0] + im[1]) + (im[2] + im[3]);
        sr = warp_sum(sr);
        si = warp_sum(si);
        if (lane == 0) pbu[((size_t)s * ps + c) * cps + chunk] = make_double2(sr, si);
      }
    }
    }
    grid_sync(bar, bar + 1, G, err);
    // (R) totals over the chunks, one thread per (RHS, column)
    for (int it = b * blockDim.x + threadIdx.x; it < a.nrhs * np; it += G * blockDim.x) {
      const int s = it / np, c = it % np;
      if (s_act[s] < want) continue;
      const double2* src = pbu + ((size_t)s * ps + c) * cps;
      double re = 0.0, im = 0.0;
      for (int q = 0; q < cps; ++q) {
        re += src[q].x;
        im += src[q].y;
      }
      hr[(size_t)s * ps + c] = make_double2(re, im);
    }
    grid_sync(bar, bar + 1, G, err);
    // (B) decisions for every RHS (identical in every block)
    for (int s = warp; s < a.nrhs; s += 8) {
      if (s_act[s] < want) continue;
      const double2* hs = hr + (size_t)s * ps;
      double t = 0.0;
      for (int c = lane; c <= j; c += 32) t += cabs2(hs[c]);
      t = warp_sum(t);
      if (lane == 0) {
        const double wn2 = hs[j + 1].x;
        const double hn2 = fmax(wn2 - t, 0.0);
        const bool again = pass == 0 && !(hn2 > 1e-4 * wn2);
        const double inv = hn2 > 0.0 ? rsqrt_nr(hn2) : 0.0;
        s_hn[s] = again ? -1.0 : hn2 * inv;
        s_inv[s] = inv;
      }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < a.nrhs; s += blockDim.x)
      if (s_act[s] >= want && s_hn[s] < 0.0) s_act[s] = 2;
    __syncthreads();
    // (B) row updates of each unit, v_{j+1}; chunk 0's owner: Hessenberg column and Givens
    for (int u = b; u < nunits; u += G) {
      const int s = u / cps, chunk = u % cps;
      if (s_act[s] < want) continue;
      const double hn = s_hn[s], inv = s_inv[s];
      const bool last = hn >= 0.0;
      const double2* hs = hr + (size_t)s * ps;
      __syncthreads();
      for (int c = threadIdx.x; c <= j; c += blockDim.x) {
        s_h[c] = hs[c];
        if constexpr (kF32) s_hf[c] = make_float2((float)hs[c].x, (float)hs[c].y);
      }
      __syncthreads();
      const int q0 = chunk * unit, q1 = min(a.n, q0 + unit);
      if constexpr (kF32) {
        const float finv = (float)inv;
        for (int r = q0 + threadIdx.x; r < q1; r += blockDim.x) {
          float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                           make_float2(0.f, 0.f)};
          int c = 0;
          for (; c + 4 <= j + 1; c += 4) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float2 vv = a.Vf[vidx(a, c + t, s) + r], h = s_hf[c + t];
              acc[t].x = fmaf(vv.x, h.x, acc[t].x);
              acc[t].x = fmaf(-vv.y, h.y, acc[t].x);
              acc[t].y = fmaf(vv.x, h.y, acc[t].y);
              acc[t].y = fmaf(vv.y, h.x, acc[t].y);
            }
          }
          for (; c <= j; ++c) {
            const float2 vv = a.Vf[vidx(a, c, s) + r], h = s_hf[c];
            acc[0].x = fmaf(vv.x, h.x, acc[0].x);
            acc[0].x = fmaf(-vv.y, h.y, acc[0].x);
            acc[0].y = fmaf(vv.x, h.y, acc[0].y);
            acc[0].y = fmaf(vv.y, h.x, acc[0].y);
          }
          const float2 ww = a.wf[(size_t)s * a.n + r];
          const float2 wv = make_float2(ww.x - ((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x)),
                                        ww.y - ((acc[0].y + acc[1].y) + (acc[2].y + acc[3].y)));
          if (!last) {
            a.wf[(size_t)s * a.n + r] = wv;
          } else if (hn > 0.0) {
            const float2 v = make_float2(wv.x * finv, wv.y * finv);
            a.Vf[vidx(a, j + 1, s) + r] = v;
            a.xf[(size_t)s * a.ld + r] = v;
          }
        }
      } else
      for (int r = q0 + threadIdx.x; r < q1; r += blockDim.x) {
        double2 acc[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                          make_double2(0.0, 0.0)};
        int c = 0;
        for (; c + 4 <= j + 1; c += 4) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const double2 vv = a.V[vidx(a, c + t, s) + r], h = s_h[c + t];
            acc[t].x = fma(vv.x, h.x, acc[t].x);
            acc[t].x = fma(-vv.y, h.y, acc[t].x);
            acc[t].y = fma(vv.x, h.y, acc[t].y);
            acc[t].y = fma(vv.y, h.x, acc[t].y);
          }
        }
        for (; c <= j; ++c) {
          const double2 vv = a.V[vidx(a, c, s) + r], h = s_h[c];
          acc[0].x = fma(vv.x, h.x, acc[0].x);
          acc[0].x = fma(-vv.y, h.y, acc[0].x);
          acc[0].y = fma(vv.x, h.y, acc[0].y);
          acc[0].y = fma(vv.y, h.x, acc[0].y);
        }
        const double2 tsum = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
        const double2 wv = csub(a.w[(size_t)s * a.n + r], tsum);
        if (!last) {
          a.w[(size_t)s * a.n + r] = wv;
        } else if (hn > 0.0) {
          const double2 v = make_double2(wv.x * inv, wv.y * inv);
          a.V[vidx(a, j + 1, s) + r] = v;
          a.xf[(size_t)s * a.ld + r] = make_float2((float)v.x, (float)v.y);
        }
      }
      if (chunk == 0) {
        const size_t ho = (size_t)s * (a.m + 1);
        for (int c = threadIdx.x; c <= j; c += blockDim.x) {
          const double2 t = pass == 0 ? s_h[c] : cadd(a.hcol[ho + c], s_h[c]);
          if (!last) a.hcol[ho + c] = t;
          s_acc[c] = t;
          if (c < j) {
            s_cs[c] = a.cs[(size_t)s * a.m + c];
            s_sn[c] = a.sn[(size_t)s * a.m + c];
          }
        }
        __syncthreads();
        if (last && warp == 0) givens_warp(a, s, j, hn, s_acc, s_cs, s_sn, lane);
      }
    }
  }
  grid_sync(bar, bar + 1, G, err);  // every Givens update before the flags are read
  if (b == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int q = 0; q < a.nrhs; ++q) all &= a.done[q];
    a.scal[0] = j + 1;
    a.scal[1] = all || j + 1 >= a.maxit;
  }
}

// Back substitution R y = g on the rotated Hessenberg matrix, one 256-thread block per RHS,
// column by column: thread k holds g_k and 1/R_kk (all reciprocals formed in parallel first);
// step i sets y_i = g_i / R_ii and every k < i subtracts R_ki y_i. The columns of R are staged
// through shared memory eight at a time, so a step costs a broadcast and one complex FMA
// rather than a shuffle reduction, a division and a load from L2.
constexpr int kLsqCols = 8;
__global__ void __launch_bounds__(256) k_lsq(GArgs a) {
  __shared__ double2 s_r[kLsqCols][256];
  __shared__ double2 s_y;
  const int s = blockIdx.x, k = threadIdx.x;
  const int kdim = a.iters[s];
  const size_t ho = (size_t)s * (a.m + 1);
  const double2* H = a.H + (size_t)s * a.m * (a.m + 1);  // column c, row r at c (m + 1) + r
  double2* y = a.y + (size_t)s * a.m;
  double2 g = make_double2(0.0, 0.0), inv = g;
  if (k < kdim) {
    g = a.gv[ho + k];
    const double2 d = H[(size_t)k * (a.m + 1) + k];
    const double dd = cabs2(d);
    if (dd > 0.0) inv = make_double2(d.x / dd, -d.y / dd);  // a zero pivot leaves y_k = 0
  }
  for (int i0 = kdim - 1; i0 >= 0; i0 -= kLsqCols) {
    const int nc = min(kLsqCols, i0 + 1);
    __syncthreads();
    for (int q = 0; q < nc; ++q)  // columns i0, i0 - 1, ... rows 0..column-1
      if (k < i0 - q) s_r[q][k] = H[(size_t)(i0 - q) * (a.m + 1) + k];
    __syncthreads();
    for (int q = 0; q < nc; ++q) {
      const int i = i0 - q;
      if (k == i) {
        const double2 yi = cmul(g, inv);
        y[i] = yi;
        s_y = yi;
      }
      __syncthreads();
      if (k < i) g = csub(g, cmul(s_r[q][k], s_y));
      __syncthreads();
    }
  }
}

// x = V y (FP64), or x += V y when `accumulate` (refinement), with the complex64 output and
// the FP32 copy of x for the residual matvec.
// With the FP32 basis the correction V y is formed in FP32 (y staged once per block as FP32)
// and added to x in FP64: an inner solve's correction needs far less than FP32 accuracy.
__global__ void __launch_bounds__(kChunk) k_xupdate(GArgs a, float2* __restrict__ pout, int accumulate) {
  __shared__ float2 s_y[256];
  const int s = blockIdx.y;
  const int r = blockIdx.x * kChunk + threadIdx.x;
  const int kdim = (a.skip && a.skip[s]) ? 0 : a.iters[s];
  const double2* y = a.y + (size_t)s * a.m;
  if (a.Vf) {
    for (int c = threadIdx.x; c < kdim; c += blockDim.x) s_y[c] = make_float2((float)y[c].x, (float)y[c].y);
    __syncthreads();
  }
  if (r >= a.n) return;
  double2 acc = accumulate ? a.x[(size_t)s * a.n + r] : make_double2(0.0, 0.0);
  if (a.Vf) {
    float dr = 0.f, di = 0.f;
    for (int c = 0; c < kdim; ++c) {
      const float2 v = a.Vf[vidx(a, c, s) + r], h = s_y[c];
      dr = fmaf(v.x, h.x, fmaf(-v.y, h.y, dr));
      di = fmaf(v.x, h.y, fmaf(v.y, h.x, di));
    }
    acc = make_double2(acc.x + (double)dr, acc.y + (double)di);
  }
  for (int c = 0; c < (a.Vf ? 0 : kdim); ++c) acc = cadd(acc, cmul(a.V[vidx(a, c, s) + r], y[c]));
  a.x[(size_t)s * a.n + r] = acc;
  pout[(size_t)s * a.n + r] = make_float2((float)acc.x, (float)acc.y);
  a.xf[(size_t)s * a.ld + r] = make_float2((float)acc.x, (float)acc.y);
}

// ||b - w|| / ||b|| with w = L x (true residual of the FP32 operator).
__global__ void __launch_bounds__(kChunk) k_resid(GArgs a) {
  __shared__ double sh[32];
  const int s = blockIdx.y, chunk = blockIdx.x;
  const int r = chunk * kChunk + threadIdx.x;
  double v = 0.0;
  if (r < a.n) v = cabs2(csub(a.b[(size_t)s * a.n + r], a.w[(size_t)s * a.n + r]));
  v = block_sum(v, sh);
  if (threadIdx.x == 0) a.partn[(size_t)chunk * a.nrhs + s] = v;
  if (!last_block(a.cnt + s * kCounters + 4, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) t += a.partn[(size_t)c * a.nrhs + s];
    a.res_true[s] = a.bnorm[s] > 0.0 ? sqrt(t) / a.bnorm[s] : 0.0;
  }
}

// Refinement residual: b = b0 - w (w = L x with the FP32 operator) for the RHS not yet
// converged, ||b0 - w|| / ||b0|| into res_true and the outer convergence flags.
__global__ void __launch_bounds__(kChunk) k_ir_residual(GArgs a, const double2* __restrict__ b0,
                                                        int* __restrict__ outer_done, double tol) {
  __shared__ double sh[32];
  const int s = blockIdx.y, chunk = blockIdx.x;
  const int r = chunk * kChunk + threadIdx.x;
  const bool active = !outer_done[s];
  double v = 0.0, vb = 0.0;
  if (active && r < a.n) {
    const double2 bb = b0[(size_t)s * a.n + r];
    const double2 rr = csub(bb, a.w[(size_t)s * a.n + r]);
    a.b[(size_t)s * a.n + r] = rr;
    v = cabs2(rr);
    vb = cabs2(bb);
  }
  v = block_sum(v, sh);
  vb = block_sum(vb, sh);
  if (threadIdx.x == 0) {
    a.partn[(size_t)chunk * a.nrhs + s] = v;
    a.part[(size_t)chunk * a.nrhs + s] = make_double2(vb, 0.0);
  }
  if (!last_block(a.cnt + s * kCounters + 5, gridDim.x)) return;
  if (threadIdx.x == 0 && active) {
    double t = 0.0, tb = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) {
      t += a.partn[(size_t)c * a.nrhs + s];
      tb += a.part[(size_t)c * a.nrhs + s].x;
    }
    const double rel = tb > 0.0 ? sqrt(t / tb) : 0.0;
    a.res_true[s] = rel;
    if (rel <= tol) outer_done[s] = 1;
  }
}

// complex64 (n) -> padded complex64 (ld), zero pad
__global__ void k_pad_copy(const float2* __restrict__ src, int n, int ld, int nrhs,
                           float2* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ld * nrhs) return;
  const int s = (int)(i / ld), r = (int)(i % ld);
  dst[i] = r < n ? src[(size_t)s * n + r] : make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------------------- host side
// Krylov dimension: the restart length of GMRES(m), or the iteration cap when unrestarted.
static int krylov_dim(const nat_bem_opts& o) {
  const int cap = std::max(1, o.max_iter);
  return o.restart > 0 ? std::min(o.restart, cap) : cap;
}

int64_t workspace_bytes(int64_t n, int nrhs, const nat_bem_opts& o) {
  const int64_t m = krylov_dim(o);
  const int64_t ld = round_up(n, 32);
  const int64_t nchunk = (n + kUpdRows - 1) / kUpdRows;
  int64_t b = 0;
  b += 16 * n * nrhs * 5 + 8 * nrhs;      // b, w, x, b0, xacc, ||b0||
  b += 16 * n * nrhs * (m + 1);           // V
  b += 8 * ld * nrhs * 3;                 // xf, gin, pout
  b += 16 * nrhs * (m + 1) * (m + 4);     // H, hcol, htmp, gv, sn, y
  b += 16 * std::max<int64_t>(nchunk, kDotChunks) * nrhs * (m + 1);  // partial dots
  b += 8 * nchunk * nrhs;                                            // partial norms
  b += 16 * nrhs * (m + 2) * (256 + 1);   // fused Arnoldi partials (<= 256 blocks) and totals
  if (nrhs > kArnUnitsMinRhs)  // unit partials (about four units per block, <= 160 SMs)
    b += 16 * (m + 2) * (4 * kArnUnitsPerSm * 160 + nrhs);
  b += 8 * n * nrhs;  // FP32 w of inner solves
  if (nrhs > 1) {  // operand and partial tiles of the multi-RHS products
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 160;  // no device: an upper bound for current parts
    }
    b += (int64_t)tc_workspace_bytes(n, ld, nrhs, sms);
  }
  return b;
}

void workspace_free(Workspace* ws, cudaStream_t s) {
  if (!ws) return;
  void* ptrs[] = {ws->b, ws->V, ws->w, ws->x, ws->H, ws->hcol, ws->htmp, ws->sn, ws->gv, ws->y,
                  ws->part, ws->cs, ws->partn, ws->bnorm, ws->res, ws->hnorm, ws->res_true,
                  ws->xf, ws->gin, ws->pout, ws->done, ws->iters, ws->scal, ws->cnt,
                  ws->b0, ws->xacc, ws->b0norm, ws->outer_done, ws->tc_scratch, ws->tc_err, ws->gbar,
                  ws->pblk, ws->hred, ws->pbu, ws->wf};
  for (void* p : ptrs)
    if (p) dev_free(p, s);
  if (ws->host_scal) cudaFreeHost(ws->host_scal);
  for (auto& kv : ws->graphs) cudaGraphExecDestroy(kv.second.first);
  for (auto& kv : ws->loops) cudaGraphExecDestroy(kv.second);
  if (ws->loop_launches) dev_free(ws->loop_launches, s);
  if (ws->loop_bodies) dev_free(ws->loop_bodies, s);
  if (ws->host_loop) cudaFreeHost(ws->host_loop);
  delete ws;
}

static nat_bem_status workspace_ensure(nat_bem_op* op, int nrhs, cudaStream_t s) {
  const int m = krylov_dim(op->opts);
  Workspace* ws = op->ws;
  if (ws && ws->cap >= nrhs && ws->m == m) {
    ws->nrhs = nrhs;  // reuse: every array is sized for `cap` right-hand sides
    return NAT_BEM_OK;
  }
  if (ws) workspace_free(ws, s);
  op->ws = ws = new Workspace();
  const int64_t n = op->n, ld = op->geo.ld;
  ws->n = n;
  ws->ld = ld;
  ws->nrhs = nrhs;
  ws->cap = nrhs;
  ws->m = m;
  ws->nchunk = (int)((n + kUpdRows - 1) / kUpdRows);
  const size_t nr = (size_t)nrhs, mm = (size_t)m;
  NB_TRY(dev_alloc_n(&ws->b, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->w, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->x, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->V, n * nr * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->H, nr * mm * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->hcol, nr * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->htmp, nr * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->sn, nr * mm, s));
  NB_TRY(dev_alloc_n(&ws->gv, nr * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->y, nr * mm, s));
  NB_TRY(dev_alloc_n(&ws->part, std::max<size_t>((size_t)ws->nchunk, kDotChunks) * nr * (mm + 1), s));
  NB_TRY(dev_alloc_n(&ws->cs, nr * mm, s));
  NB_TRY(dev_alloc_n(&ws->partn, (size_t)ws->nchunk * nr, s));
  NB_TRY(dev_alloc_n(&ws->bnorm, nr, s));
  NB_TRY(dev_alloc_n(&ws->res, nr, s));
  NB_TRY(dev_alloc_n(&ws->hnorm, nr, s));
  NB_TRY(dev_alloc_n(&ws->res_true, nr, s));
  NB_TRY(dev_alloc_n(&ws->xf, ld * nr, s));
  NB_TRY(dev_alloc_n(&ws->gin, std::max<int64_t>(ld, op->ldr) * nr, s));
  NB_TRY(dev_alloc_n(&ws->pout, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->done, nr, s));
  NB_TRY(dev_alloc_n(&ws->iters, nr, s));
  NB_TRY(dev_alloc_n(&ws->scal, 4, s));
  NB_TRY(dev_alloc_n(&ws->cnt, nr * kCounters, s));
  NB_TRY(dev_alloc_n(&ws->b0, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->xacc, n * nr, s));
  NB_TRY(dev_alloc_n(&ws->b0norm, nr, s));
  NB_TRY(dev_alloc_n(&ws->outer_done, nr, s));
  NB_TRY(dev_alloc_n(&ws->tc_err, 1, s));
  NB_TRY(dev_alloc_n(&ws->gbar, 2, s));
  NB_TRY(dev_alloc_n(&ws->loop_launches, 1, s));
  NB_TRY(dev_alloc_n(&ws->loop_bodies, 1, s));
  NB_TRY_CUDA(cudaMemsetAsync(ws->loop_launches, 0, sizeof(unsigned long long), s));
  NB_TRY_CUDA(cudaMemsetAsync(ws->gbar, 0, 2 * sizeof(unsigned), s));
  {
    // the fused Arnoldi kernel runs one block per SM when every block fits at once and the
    // rows per block and the RHS count fit its shared-memory staging
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    // dynamic shared memory for the V panel: up to kArnPanelBytes, or all m+1 vectors of a
    // block's rows
    const int64_t rows_max = sms >= 2 ? (n + sms - 2) / (sms - 1) : n;
    const int64_t want = std::min<int64_t>(kArnPanelBytes, 16 * rows_max * (m + 1));
    // the attribute is per function, shared by every op and thread: set once to the largest
    // size any launch uses, never lowered
    static std::mutex attr_mu;
    static int attr_set[64] = {0};
    {
      std::lock_guard<std::mutex> lk(attr_mu);
      if (dev >= 0 && dev < 64 && attr_set[dev] == 0) {
        attr_set[dev] = cudaFuncSetAttribute(k_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kArnPanelBytes) == cudaSuccess &&
                                cudaFuncSetAttribute(k_arnoldi_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     kArnPanelBytes) == cudaSuccess
                            ? 1
                            : -1;
        if (attr_set[dev] < 0) cudaGetLastError();
      }
      ws->arn_smem = (dev >= 0 && dev < 64 && attr_set[dev] == 1) ? (int)want : 0;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi, 256, ws->arn_smem);
    {
      int per_sm32 = 0;  // the FP32-basis form must fit as well
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_arnoldi_f32, 256, ws->arn_smem);
      per_sm = std::min(per_sm, per_sm32);
    }
    const bool fits = sms >= 2 && n <= (int64_t)(sms - 1) * kArnMaxRows && nrhs <= kArnMaxRhs;
    ws->coop_blocks = (coop && per_sm >= 1 && fits && !std::getenv("NATBEM_NO_FUSED_KRYLOV")) ? sms : 0;
    if (ws->coop_blocks > 0) {
      NB_TRY(dev_alloc_n(&ws->pblk, nr * (mm + 2) * (size_t)ws->coop_blocks, s));
      NB_TRY(dev_alloc_n(&ws->hred, nr * (mm + 2), s));
      if (nrhs > kArnUnitsMinRhs) {  // the multi-RHS kernel: partials for the largest unit count
        // its own grid: up to kArnUnitsPerSm blocks per SM (more loads in flight for the
        // streaming dots and row updates; one block per SM kept about a third of the HBM rate)
        int pu32 = 0, pu64 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pu32, k_arnoldi_units<true>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pu64, k_arnoldi_units<false>, 256, 0);
        ws->units_blocks = sms * std::max(1, std::min(kArnUnitsPerSm, std::min(pu32, pu64)));
        size_t most = 0;
        for (int q = kArnUnitsMinRhs + 1; q <= nrhs; ++q) {
          const int u = arnoldi_unit((int)n, q, ws->units_blocks);
          most = std::max(most, (size_t)q * (size_t)((n + u - 1) / u));
        }
        NB_TRY(dev_alloc_n(&ws->pbu, most * (mm + 2), s));
      }
      NB_TRY(dev_alloc_n(&ws->wf, (size_t)n * nr, s));  // FP32 w of inner solves on the FP32 basis
    }
  }
  NB_TRY_CUDA(cudaMemsetAsync(ws->tc_err, 0, sizeof(int), s));
  if (nrhs > 1) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ws->tc_bytes = tc_workspace_bytes(n, std::max<int64_t>(ld, op->ldr), nrhs, sms);  // L and R products
    NB_TRY(dev_alloc(&ws->tc_scratch, ws->tc_bytes, s));
  }
  NB_TRY_CUDA(cudaMemsetAsync(ws->cnt, 0, nr * kCounters * sizeof(unsigned), s));
  NB_TRY_CUDA(cudaMemsetAsync(ws->scal, 0, 4 * sizeof(int), s));
  NB_TRY_CUDA(cudaMemsetAsync(ws->xf, 0, ld * nr * sizeof(float2), s));
  NB_TRY_CUDA(cudaMallocHost(&ws->host_scal, 4 * sizeof(int)));
  NB_TRY_CUDA(cudaMallocHost(&ws->host_loop, sizeof(unsigned long long)));
  *ws->host_loop = 0;
  return NAT_BEM_OK;
}

static GArgs make_args(nat_bem_op* op, Workspace* ws, const float2* Lop) {
  GArgs a;
  a.n = (int)ws->n;
  a.ld = (int)ws->ld;
  a.nrhs = ws->nrhs;
  a.m = ws->m;
  a.nchunk = ws->nchunk;
  a.L = Lop;
  a.b = ws->b;
  a.V = ws->V;
  a.w = ws->w;
  a.x = ws->x;
  a.H = ws->H;
  a.hcol = ws->hcol;
  a.htmp = ws->htmp;
  a.sn = ws->sn;
  a.gv = ws->gv;
  a.y = ws->y;
  a.part = ws->part;
  a.cs = ws->cs;
  a.partn = ws->partn;
  a.bnorm = ws->bnorm;
  a.res = ws->res;
  a.hnorm = ws->hnorm;
  a.res_true = ws->res_true;
  a.xf = ws->xf;
  a.done = ws->done;
  a.iters = ws->iters;
  a.scal = ws->scal;
  a.cnt = ws->cnt;
  a.tol = op->opts.tol;
  a.maxit = ws->m;
  a.skip = nullptr;
  a.bscale = nullptr;
  a.Vf = nullptr;
  a.wf = ws->wf;
  return a;
}

// GEMV variants for one RHS and the autotuner that picks one per (device, operator size).
enum GemvVariant { kGemvR2U4 = 0, kGemvR4U4, kGemvR2U8, kGemvBulk4x16k, kGemvBulk6x16k,
                   kGemvXsR2U8, kGemvXsR4U4, kGemvXsR2U4, kGemvVariants };
// 0 rows2_unroll4, 1 rows4_unroll4, 2 rows2_unroll8, 3 bulk_4x16KiB, 4 bulk_6x16KiB,
// 5 xs_rows2_unroll8, 6 xs_rows4_unroll4, 7 xs_rows2_unroll4
static_assert((int)kGemvVariants == (int)NAT_BEM_GEMV_VARIANTS, "GEMV variants and the C ABI disagree");
constexpr int kGemvXsMaxBytes = 200 * 1024;  // x staged in shared memory up to ld = 25600

// Grid of the staged-x GEMV: as many blocks per SM as shared memory and registers allow.
template <int kRows, int kUnroll>
static int gemv_xs_blocks(int ld, int sms) {
  static std::mutex mu;
  static int attr_set[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && attr_set[dev] == 0) {
      attr_set[dev] = cudaFuncSetAttribute(k_gemv_xs<kRows, kUnroll>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kGemvXsMaxBytes) == cudaSuccess ? 1 : -1;
      if (attr_set[dev] < 0) cudaGetLastError();
    }
    if (dev < 0 || dev >= 64 || attr_set[dev] != 1) return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv_xs<kRows, kUnroll>, 256, 8 * (size_t)ld) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

static nat_bem_status gemv_launch(int variant, const char* name, const float2* A, int n, int ld,
                                  const float2* x, double2* y, int nrhs, const int* done,
                                  const int* scal, int* err, cudaStream_t s, int64_t astride = 0) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (variant) {
    case kGemvR4U4: {
      dim3 grid((n + 3) / 4, nrhs);
      NB_LAUNCH(name, s, k_gemv<4, 4><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
      break;
    }
    case kGemvR2U8: {
      dim3 grid((n + 1) / 2, nrhs);
      NB_LAUNCH(name, s, k_gemv<2, 8><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
      break;
    }
    case kGemvBulk4x16k:
    case kGemvBulk6x16k: {
      const int blocks = 2 * sms;
      const int rpb = (n + blocks - 1) / blocks;
      dim3 grid((n + rpb - 1) / rpb, nrhs);
      static bool attr = false;
      if (!attr) {
        NB_TRY_CUDA(cudaFuncSetAttribute(k_gemv_bulk<4, 16384>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 16384));
        NB_TRY_CUDA(cudaFuncSetAttribute(k_gemv_bulk<6, 16384>, cudaFuncAttributeMaxDynamicSharedMemorySize, 6 * 16384));
        attr = true;
      }
      if (variant == kGemvBulk4x16k)
        NB_LAUNCH(name, s, k_gemv_bulk<4, 16384><<<grid, 288, 4 * 16384, s>>>(A, n, ld, x, ld, y, n, done, scal, rpb, err, astride));
      else
        NB_LAUNCH(name, s, k_gemv_bulk<6, 16384><<<grid, 288, 6 * 16384, s>>>(A, n, ld, x, ld, y, n, done, scal, rpb, err, astride));
      break;
    }
    case kGemvXsR2U8:
    case kGemvXsR4U4:
    case kGemvXsR2U4: {
      const size_t smem = 8 * (size_t)ld;
      const int rows = variant == kGemvXsR4U4 ? 4 : 2;
      int blocks = variant == kGemvXsR2U8 ? gemv_xs_blocks<2, 8>(ld, sms)
                 : variant == kGemvXsR4U4 ? gemv_xs_blocks<4, 4>(ld, sms) : gemv_xs_blocks<2, 4>(ld, sms);
      if (smem > (size_t)kGemvXsMaxBytes || blocks <= 0) {  // x does not fit: plain variant
        dim3 grid((n + 1) / 2, nrhs);
        NB_LAUNCH(name, s, k_gemv<2, 8><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
        break;
      }
      blocks = std::min(blocks, (n + rows - 1) / rows);
      dim3 grid(blocks, nrhs);
      if (variant == kGemvXsR2U8)
        NB_LAUNCH(name, s, k_gemv_xs<2, 8><<<grid, 256, smem, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
      else if (variant == kGemvXsR4U4)
        NB_LAUNCH(name, s, k_gemv_xs<4, 4><<<grid, 256, smem, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
      else
        NB_LAUNCH(name, s, k_gemv_xs<2, 4><<<grid, 256, smem, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
      break;
    }
    default: {
      dim3 grid((n + 1) / 2, nrhs);
      NB_LAUNCH(name, s, k_gemv<2, 4><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride));
    }
  }
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, int64_t>, int> g_tuned;  // (device, n rounded to 1024) -> variant
}  // namespace

// The fastest variant for this operator size on this device, measured on the operator itself
// (CUDA events) the first time a size class is met: one warm-up pass over all variants, then
// four interleaved rounds, keeping each variant's minimum. Other streams' kernels only slow a
// run down, so the minimum over interleaved rounds is the uncontended time; the first variant
// (two rows per block, unroll 4) wins ties within 2%. Operators of 8192 rows or more (far
// beyond L2) take four rows per block (unroll 4) without tuning: it is slower alone, and the
// tuner picks against it, but with other solves in flight it has half the blocks of the
// two-row forms and shares the SMs better (plain FP32 bench at 10240 rows, variants pinned:
// 97.0 against 92.2 solves/s).
static int gemv_variant(const float2* A, int n, int ld, const float2* x, double2* y, int* err,
                        cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_pair(dev, (int64_t)((n + 1023) / 1024));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  if (const char* env = std::getenv("NATBEM_GEMV_VARIANT")) {
    const int v = std::atoi(env);
    if (v >= 0 && v < kGemvVariants) return v;
  }
  if (n >= 8192) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = kGemvR4U4;
    return kGemvR4U4;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float vmin[kGemvVariants];
  for (int v = 0; v < kGemvVariants; ++v) vmin[v] = 1e30f;
  for (int round = 0; round < 5; ++round) {
    for (int v = 0; v < kGemvVariants; ++v) {
      float ms = 1e30f;
      cudaEventRecord(e0, s);
      gemv_launch(v, "gemv_tune", A, n, ld, x, y, 1, nullptr, nullptr, err, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (round > 0) vmin[v] = std::min(vmin[v], ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = kGemvR2U4;
  for (int v = 1; v < kGemvVariants; ++v)
    if (vmin[v] < vmin[best] && vmin[v] < 0.98f * vmin[kGemvR2U4]) best = v;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best;
  return best;
}

// The variant the autotuner chose for this size on the current device, or -1 before it has run.
int gemv_tuned_variant(int64_t n) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_pair(dev, (int64_t)((n + 1023) / 1024)));
  return it == g_tuned.end() ? -1 : it->second;
}

// y_s = A x_s for all RHS (x padded to ld), skipping RHS flagged done when `done` is given.
static nat_bem_status gemv(const char* name, const float2* A, int n, int ld, const float2* x,
                           double2* y, int nrhs, const int* done, const int* scal, cudaStream_t s,
                           int* err = nullptr, int64_t astride = 0) {
  int* e = err ? err : nullptr;
  int variant = kGemvR2U4;
  if (e) variant = gemv_variant(A, n, ld, x, y, e, s);
  if (!e && (variant == kGemvBulk4x16k || variant == kGemvBulk6x16k)) variant = kGemvR2U4;
  return gemv_launch(variant, name, A, n, ld, x, y, nrhs, done, scal, e, s, astride);
}

// BF16-copy GEMV variants (rows per block, 16-byte loads per row in flight per thread) and
// their autotuner, which the solver runs before the first mixed sweep of a size class (outside
// any graph capture); until then, and when no tuning ran, the first variant is used.
enum Bf16Variant { kBf16R2U2 = 0, kBf16R2U4, kBf16R4U2, kBf16R4U1, kBf16Variants };

// rs (row scales) null: the BF16 copy; else the row-scaled FP16 copy.
static nat_bem_status gemv_bf16_launch(int variant, const char* name, const uint32_t* A, int n, int ld,
                                       const float2* x, double2* y, int nrhs, const int* done,
                                       const int* scal, cudaStream_t s, int64_t astride = 0,
                                       const float* rs = nullptr, int64_t sstride = 0) {
  const int rows = (variant == kBf16R4U2 || variant == kBf16R4U1) ? 4 : 2;
  dim3 grid((n + rows - 1) / rows, nrhs);
#define NB_COPY_GEMV(R, U)                                                                              \
  do {                                                                                                   \
    if (rs)                                                                                              \
      NB_LAUNCH(name, s, k_gemv_fp16<R, U><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride, rs, \
                                                                    sstride));                          \
    else                                                                                                 \
      NB_LAUNCH(name, s, k_gemv_bf16<R, U><<<grid, 256, 0, s>>>(A, n, ld, x, ld, y, n, done, scal, astride)); \
  } while (0)
  switch (variant) {
    case kBf16R2U4: NB_COPY_GEMV(2, 4); break;
    case kBf16R4U2: NB_COPY_GEMV(4, 2); break;
    case kBf16R4U1: NB_COPY_GEMV(4, 1); break;
    default: NB_COPY_GEMV(2, 2);
  }
#undef NB_COPY_GEMV
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

namespace {
// (device, 2 x (n rounded to 1024) + copy format) -> variant
std::map<std::pair<int, int64_t>, int> g_tuned_bf16;
}  // namespace

static int gemv_bf16_lookup(int n, bool fp16) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_bf16.find(std::make_pair(dev, (int64_t)((n + 1023) / 1024) * 2 + (fp16 ? 1 : 0)));
  return it == g_tuned_bf16.end() ? kBf16R2U2 : it->second;
}

// Times every BF16 variant on the operator copy (x and y are scratch of the solve), like
// gemv_variant: a warm-up round, four interleaved rounds, each variant's minimum; another
// variant must beat the first by 5%. Operators of 8192 rows or more take the first variant
// untuned. NATBEM_GEMV_BF16_VARIANT=v bypasses it.
static void gemv_bf16_tune(const uint32_t* A, int n, int ld, const float2* x, double2* y, cudaStream_t s,
                           const float* rs = nullptr) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_pair(dev, (int64_t)((n + 1023) / 1024) * 2 + (rs ? 1 : 0));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tuned_bf16.count(key)) return;
  }
  int best = kBf16R2U2;
  if (const char* env = std::getenv("NATBEM_GEMV_BF16_VARIANT")) {
    const int v = std::atoi(env);
    if (v >= 0 && v < kBf16Variants) best = v;
  } else if (n >= 8192) {
    // far beyond L2: two rows, two loads in flight (pinned one at a time on the 10240-row
    // bench workload with four solves in flight it was fastest; the tuner, run while other
    // solves share the GPU, has picked slower variants there)
    best = kBf16R2U2;
  } else {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float vmin[kBf16Variants];
    for (int v = 0; v < kBf16Variants; ++v) vmin[v] = 1e30f;
    for (int round = 0; round < 5; ++round)
      for (int v = 0; v < kBf16Variants; ++v) {
        float ms = 1e30f;
        cudaEventRecord(e0, s);
        gemv_bf16_launch(v, "gemv_bf16_tune", A, n, ld, x, y, 1, nullptr, nullptr, s, 0, rs);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (round > 0) vmin[v] = std::min(vmin[v], ms);
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int v = 1; v < kBf16Variants; ++v)
      if (vmin[v] < vmin[best] && vmin[v] < 0.95f * vmin[kBf16R2U2]) best = v;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_bf16[key] = best;
}

static nat_bem_status gemv_bf16(const char* name, const uint32_t* A, int n, int ld,
                                const float2* x, double2* y, int nrhs, const int* done,
                                const int* scal, cudaStream_t s, int64_t astride = 0,
                                const float* rs = nullptr, int64_t sstride = 0) {
  return gemv_bf16_launch(gemv_bf16_lookup(n, rs != nullptr), name, A, n, ld, x, y, nrhs, done, scal, s,
                          astride, rs, sstride);
}

// One GMRES run on the right-hand sides in a.b (x0 = 0): init, iterations until every RHS
// converged or a.maxit, least squares, and x = V y (or x += V y with `accumulate`) into a.x,
// pout and the FP32 copy a.xf. `bf16` selects the operator copy used for the matvec.
// w = M x for every RHS with the given engine (x = ws->xf, padded to ld).
static nat_bem_status matvec(nat_bem_op* op, Workspace* ws, int which, int engine, double2* y,
                             const int* done, const int* scal, const char* name, cudaStream_t s) {
  const int n = (int)op->n, ld = (int)op->geo.ld, nrhs = ws->nrhs;
  const float2* M = which == 0 ? op->L : op->R;
  switch (engine) {
    case kEngineGemv:
      return gemv(name, M, n, ld, ws->xf, y, nrhs, done, scal, s, ws->tc_err, op->bstride);
    case kEngineGemvCopy:  // the BF16 copy, or the FP16 copy with its row scales
      return gemv_bf16(name, op->Lb, n, ld, ws->xf, y, nrhs, done, scal, s, op->bstride,
                       op->copy_fp16 ? op->row_scale : nullptr, op->bstride > 0 ? n : 0);
    default:
      return product(op, which, engine, ws->xf, nrhs, y, done, scal, ws->tc_scratch, ws->tc_bytes,
                     ws->tc_err, s);
  }
}

// End of one loop body: count the body's kernels and continue while some RHS is not done
// (scal[1] is set once every RHS converged or the iteration cap was reached). The loop also
// ends after max_bodies bodies (the cap's worth of iterations and one more body) or once a
// kernel has raised a bounded-wait error, so it ends whatever the kernels did.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* __restrict__ scal,
                            unsigned long long* __restrict__ launches, int per_body,
                            int* __restrict__ bodies, int max_bodies, const int* __restrict__ err) {
  if (threadIdx.x == 0) {
    *launches += (unsigned long long)per_body;
    const int b = ++*bodies;
    cudaGraphSetConditional(h, (scal[1] || b >= max_bodies || *err) ? 0u : 1u);
  }
}

// Kernels the device-side loops ran, for the launch counter: loop_copy enqueues the read of the
// device counter (and its reset) before a host sync point, loop_count adds it after the sync.
static void loop_copy(Workspace* ws, cudaStream_t s) {
  cudaMemcpyAsync(ws->host_loop, ws->loop_launches, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  cudaMemsetAsync(ws->loop_launches, 0, sizeof(unsigned long long), s);
}
static void loop_count(Workspace* ws) {
  add_launches((int64_t)*ws->host_loop);
  *ws->host_loop = 0;
}

static nat_bem_status gmres_run(nat_bem_op* op, Workspace* ws, const GArgs& a, int engine,
                                int accumulate, float2* pout, cudaStream_t s) {
  const int n = (int)op->n, nrhs = ws->nrhs;
  const dim3 upd_grid(ws->nchunk, nrhs), fin_grid((n + kChunk - 1) / kChunk, nrhs);
  // the dot-product grid covers the Krylov vectors 0..j of the iteration being launched (the
  // device's j equals the host's launch count until every RHS is done)
  NB_LAUNCH("gmres_start", s, k_start<<<upd_grid, kUpdRows, 0, s>>>(a));
  NB_LAUNCH("gmres_finish", s, k_finish<<<fin_grid, kChunk, 0, s>>>(a, 0));
  NB_CHECK_LAUNCH();
  int it = 0, chunk = 16;
  // Direct launches, or a CUDA graph of the chunk captured once per configuration: graphs need
  // a capturable (non-legacy) stream and are skipped while per-launch tracing is on.
  static const bool env_off = std::getenv("NATBEM_NO_GRAPHS") != nullptr;
  const bool use_graphs = !env_off && !ws->graphs_off && s != nullptr && !tracing_enabled();
  auto launch_chunk = [&](int it0, int c) -> nat_bem_status {
    for (int q = 0; q < c; ++q) {
      NB_TRY(matvec(op, ws, 0, engine, ws->w, ws->done, ws->scal,
                    engine == kEngineGemvCopy ? (op->copy_fp16 ? "gemv_fp16" : "gemv_bf16") : "gemv", s));
      if (ws->coop_blocks > 0) {
        GArgs ac = a;
        double2* pb = ws->pblk;
        double2* hr = ws->hred;
        unsigned* bar = ws->gbar;
        int* errp = ws->tc_err;
        if (nrhs > kArnUnitsMinRhs && ws->pbu) {
          double2* pu = ws->pbu;
          int unit = arnoldi_unit(n, nrhs, ws->units_blocks);
          int cps = (n + unit - 1) / unit;
          void* args[] = {&ac, &pu, &hr, &bar, &errp, &unit, &cps};
          const void* kern = ac.Vf ? (const void*)k_arnoldi_units<true> : (const void*)k_arnoldi_units<false>;
          NB_LAUNCH("gmres_arnoldi", s, NB_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(ws->units_blocks), dim3(256), args, 0, s)));
          continue;
        }
        const int smem = ac.Vf ? std::min(ws->arn_smem, kArnPanelBytesF32) : ws->arn_smem;
        int pcap = smem / (int)(ac.Vf ? sizeof(float2) : sizeof(double2));
        void* args[] = {&ac, &pb, &hr, &bar, &errp, &pcap};
        const void* kern = ac.Vf ? (const void*)k_arnoldi_f32 : (const void*)k_arnoldi;
        NB_LAUNCH("gmres_arnoldi", s, NB_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(ws->coop_blocks), dim3(256), args, (size_t)smem, s)));
        continue;
      }
      const dim3 dot_grid(std::min(it0 + q + 1, std::max(1, a.maxit)), kDotChunks, nrhs);
      NB_LAUNCH("gmres_dots", s, k_dots<<<dot_grid, kDotThreads, 0, s>>>(a));
      NB_LAUNCH("gmres_update", s, k_update<<<upd_grid, 256, 0, s>>>(a, 0));
      NB_LAUNCH("gmres_dots", s, k_dots<<<dot_grid, kDotThreads, 0, s>>>(a));
      NB_LAUNCH("gmres_update", s, k_update<<<upd_grid, 256, 0, s>>>(a, 1));
      NB_LAUNCH("gmres_finish", s, k_finish<<<fin_grid, kChunk, 0, s>>>(a, 1));
    }
    return NAT_BEM_OK;
  };
  // The whole run on the device: with the cooperative Arnoldi step every iteration launches
  // the same kernels, so one captured chunk of 8 iterations serves as the body of a conditional
  // while node that repeats it until every RHS is done; no host round trip until the caller
  // reads the results.
  static const bool loop_env_off = std::getenv("NATBEM_NO_DEVICE_LOOP") != nullptr;
  if (use_graphs && !loop_env_off && op->opts.device_loop && !ws->loops_off && ws->coop_blocks > 0) {
    const auto key = std::make_tuple(engine, a.nrhs, a.maxit, a.tol,
                                     (a.skip ? 1 : 0) + (accumulate ? 2 : 0) + (a.bscale ? 4 : 0));
    auto f = ws->loops.find(key);
    if (f == ws->loops.end()) {
      cudaGraph_t g = nullptr, body = nullptr;
      cudaGraphExec_t ge = nullptr;
      cudaGraphConditionalHandle h{};
      cudaGraphNode_t node = nullptr;
      bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
                cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
      if (ok) {
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
        if (ok) body = np.conditional.phGraph_out[0];
      }
      if (ok) {
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
          const int64_t l0 = thread_launch_count();
          const nat_bem_status cs = launch_chunk(0, 8);
          const int per_body = (int)(thread_launch_count() - l0) + 1;
          add_launches(-(per_body - 1));  // capturing launches nothing
          const int max_bodies = (a.maxit + 7) / 8 + 1;
          k_loop_cond<<<1, 32, 0, s>>>(h, a.scal, ws->loop_launches, per_body, ws->loop_bodies, max_bodies,
                                       ws->tc_err);
          cudaGraph_t captured = nullptr;
          ok = cudaStreamEndCapture(s, &captured) == cudaSuccess && cs == NAT_BEM_OK;
        }
      }
      if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      if (ok) {
        f = ws->loops.emplace(key, ge).first;
      } else {
        cudaGetLastError();
        ws->loops_off = true;  // chunks with host polling for this workspace
      }
    }
    if (f != ws->loops.end()) {
      NB_TRY_CUDA(cudaMemsetAsync(ws->loop_bodies, 0, sizeof(int), s));
      NB_TRY_CUDA(cudaGraphLaunch(f->second, s));
      const dim3 vg((n + kChunk - 1) / kChunk, nrhs);
      NB_LAUNCH("gmres_lsq", s, k_lsq<<<nrhs, 256, 0, s>>>(a));
      NB_LAUNCH("gmres_xupdate", s, k_xupdate<<<vg, kChunk, 0, s>>>(a, pout, accumulate));
      NB_CHECK_LAUNCH();
      return NAT_BEM_OK;
    }
  }
  while (it < a.maxit) {
    const int c = std::min(chunk, a.maxit - it);
    bool done_direct = true;
    if (use_graphs) {
      const auto key = std::make_tuple(engine, a.nrhs, it, c, a.maxit, a.tol,
                                       (a.skip ? 1 : 0) + (accumulate ? 2 : 0) + (a.bscale ? 4 : 0));
      auto f = ws->graphs.find(key);
      if (f == ws->graphs.end()) {
        const int64_t l0 = thread_launch_count();  // other threads' launches are not captured
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        nat_bem_status cs = ok ? launch_chunk(it, c) : NAT_BEM_ECUDA;
        ok = (cudaStreamEndCapture(s, &g) == cudaSuccess) && ok && cs == NAT_BEM_OK;
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        const int64_t captured = thread_launch_count() - l0;
        add_launches(-captured);  // capturing launches nothing
        if (ok) {
          f = ws->graphs.emplace(key, std::make_pair(ge, captured)).first;
        } else {
          cudaGetLastError();
          ws->graphs_off = true;  // fall back to direct launches for this workspace
        }
      }
      if (f != ws->graphs.end()) {
        NB_TRY_CUDA(cudaGraphLaunch(f->second.first, s));
        add_launches(f->second.second);
        done_direct = false;
      }
    }
    if (done_direct) NB_TRY(launch_chunk(it, c));
    NB_CHECK_LAUNCH();
    it += c;
    NB_TRY_CUDA(cudaMemcpyAsync(ws->host_scal, ws->scal, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    if (ws->host_scal[1]) break;
    chunk = 8;
  }
  const dim3 vec_grid((n + kChunk - 1) / kChunk, nrhs);
  NB_LAUNCH("gmres_lsq", s, k_lsq<<<nrhs, 256, 0, s>>>(a));
  NB_LAUNCH("gmres_xupdate", s, k_xupdate<<<vec_grid, kChunk, 0, s>>>(a, pout, accumulate));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

__global__ void k_to_c64(const double2* __restrict__ y, int64_t count, float2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = make_float2((float)y[i].x, (float)y[i].y);
}

nat_bem_status apply_impl(nat_bem_op* op, int which, int engine, const float2* d_x, int nrhs,
                          float2* d_y, cudaStream_t s) {
  // columns: n (L) or the Neumann count (R), padded to the matrix's leading dimension
  const int n = (int)op->n, ld = which == 1 ? (int)op->ldr : (int)op->geo.ld;
  const int cols = which == 1 ? (int)op->nn : n;
  float2* xpad = nullptr;
  double2* y64 = nullptr;
  void* scratch = nullptr;
  int* err = nullptr;
  size_t sbytes = 0;
  nat_bem_status st = NAT_BEM_OK;
  auto cleanup = [&]() {
    dev_free(xpad, s);
    dev_free(y64, s);
    dev_free(scratch, s);
    dev_free(err, s);
  };
  if ((st = dev_alloc_n(&xpad, (size_t)ld * nrhs, s)) != NAT_BEM_OK ||
      (st = dev_alloc_n(&y64, (size_t)n * nrhs, s)) != NAT_BEM_OK ||
      (st = dev_alloc_n(&err, 1, s)) != NAT_BEM_OK) {
    cleanup();
    return st;
  }
  cudaMemsetAsync(err, 0, sizeof(int), s);
  const int64_t tot = (int64_t)ld * nrhs;
  NB_LAUNCH("pad_copy", s, k_pad_copy<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_x, cols, ld, nrhs, xpad));
  const float2* M = which == 0 ? op->L : op->R;
  if (engine >= NAT_BEM_ENGINE_GEMV0) {
    st = gemv_launch(engine - NAT_BEM_ENGINE_GEMV0, "gemv_apply", M, n, ld, xpad, y64, nrhs, nullptr,
                     nullptr, err, s);
  } else if (engine == NAT_BEM_ENGINE_AUTO && nrhs == 1) {
    st = gemv("gemv_apply", M, n, ld, xpad, y64, 1, nullptr, nullptr, s, err);
  } else {
    const int eng = engine == NAT_BEM_ENGINE_TF32 ? kEngineTf32
                    : engine == NAT_BEM_ENGINE_BF16 ? kEngineBf16
                    : engine == NAT_BEM_ENGINE_FP16 ? kEngineFp16 : kEngineFp32;
    {  // tensor-core operand and partial tiles, or the FP32 GEMM's partial tiles
      int dev = 0, sms = 148;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      sbytes = tc_workspace_bytes(n, ld, nrhs, sms);
      if ((st = dev_alloc(&scratch, sbytes, s)) != NAT_BEM_OK) {
        cleanup();
        return st;
      }
    }
    if (eng == kEngineFp32 && which == 0 && nrhs >= kX6MinRhs && x6_enabled()) st = ensure_split(op, s);
    if (eng != kEngineFp32 && which == 0) st = tc_tune(op, eng, nrhs, xpad, y64, scratch, sbytes, err, s);
    if (st == NAT_BEM_OK) st = product(op, which, eng, xpad, nrhs, y64, nullptr, nullptr, scratch, sbytes, err, s);
  }
  if (st == NAT_BEM_OK) {
    const int64_t cnt = (int64_t)n * nrhs;
    NB_LAUNCH("to_c64", s, k_to_c64<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(y64, cnt, d_y));
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("nat_bem_op_apply: ") + cudaGetErrorString(e));
      st = NAT_BEM_ECUDA;
    } else if (herr) {
      set_error("nat_bem_op_apply: a bounded wait gave up (code " + std::to_string(herr) + ")");
      st = NAT_BEM_ECUDA;
    }
  }
  cleanup();
  return st;
}

nat_bem_status solve_impl(nat_bem_op* op, const float2* d_neumann, int nrhs, float2* d_p,
                          nat_bem_solve_info* info, cudaStream_t s, std::vector<nat_bem_solve_info>* per_rhs,
                          std::vector<int>* per_conv) {
  NB_TRY(workspace_ensure(op, nrhs, s));
  // the split of L for the FP32-accurate tensor-core products (built outside any capture)
  if (nrhs >= kX6MinRhs && op->bstride == 0 && x6_enabled()) NB_TRY(ensure_split(op, s));
  Workspace* ws = op->ws;
  const nat_bem_opts& o = op->opts;
  NB_TRY_CUDA(cudaMemsetAsync(ws->gbar, 0, 2 * sizeof(unsigned), s));
  NB_TRY_CUDA(cudaMemsetAsync(ws->tc_err, 0, sizeof(int), s));  // this solve's bounded-wait flags
  const int n = (int)op->n;
  const dim3 vec_grid((n + kChunk - 1) / kChunk, nrhs);
  // b = R g
  {
    // g has op->nn values per RHS (triangles), padded to R's leading dimension
    const int nn = (int)op->nn, ldr = (int)op->ldr;
    const int64_t tot = (int64_t)ldr * nrhs;
    NB_LAUNCH("pad_copy", s, k_pad_copy<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_neumann, nn, ldr, nrhs, ws->gin));
    NB_CHECK_LAUNCH();
    if (nrhs == 1 || op->bstride > 0)  // one RHS, or a batch of operators (one per RHS)
      NB_TRY(gemv("gemv_rhs", op->R, n, ldr, ws->gin, ws->b, nrhs, nullptr, nullptr, s, ws->tc_err, op->bstride));
    else
      NB_TRY(product(op, 1, kEngineFp32, ws->gin, nrhs, ws->b, nullptr, nullptr, ws->tc_scratch,
                     ws->tc_bytes, ws->tc_err, s));
  }
  std::vector<int> iters(nrhs), done(nrhs), total(nrhs, 0), conv(nrhs, 0);
  std::vector<double> rt(nrhs);
  int tc_err = 0;  // bounded-wait flags of the tensor-core kernels, read at every host sync
  int refinements = 0;
  bool converged = true;
  // engines: the accurate product (FP32 GEMV for one RHS, FP32 CUDA-core GEMM for several) and
  // the inner product of mixed refinement (BF16 GEMV for one RHS; tensor cores for several:
  // TF32 on L or BF16 on its copy). TF32 with one RHS would save no bytes: it runs plain.
  // A batch of operators (one per RHS, bstride > 0) runs GEMVs throughout: the products of
  // different operators are not one GEMM.
  const bool gemv_path = nrhs == 1 || op->bstride > 0;
  const int accurate = gemv_path ? kEngineGemv : kEngineFp32;
  int inner = accurate;
  if (low_copy(o) && op->Lb)
    inner = gemv_path ? kEngineGemvCopy : (op->copy_fp16 ? kEngineFp16 : kEngineBf16);
  if (o.prec == NAT_BEM_PREC_MIXED_TF32 && !gemv_path) inner = kEngineTf32;
  const bool mixed = inner != accurate;
  // GMRES(m): the Krylov basis holds m = restart vectors and the solve runs cycles of at most
  // m iterations, each on the current residual
  const bool restarted = ws->m < std::max(1, o.max_iter);
  if (inner == kEngineGemvCopy)
    gemv_bf16_tune(op->Lb, n, (int)op->geo.ld, ws->gin, ws->w, s, op->copy_fp16 ? op->row_scale : nullptr);
  if (inner == kEngineTf32 || inner == kEngineBf16 || inner == kEngineFp16)  // tensor-core shape, outside capture
    NB_TRY(tc_tune(op, inner, nrhs, ws->xf, ws->w, ws->tc_scratch, ws->tc_bytes, ws->tc_err, s));
  if (!mixed && !restarted) {
    GArgs a = make_args(op, ws, op->L);
    a.maxit = o.max_iter;
    NB_TRY(gmres_run(op, ws, a, accurate, 0, d_p, s));
    // true residual ||R g - L p|| / ||R g|| with the FP32 operator
    NB_TRY(matvec(op, ws, 0, accurate, ws->w, nullptr, nullptr, "gemv_resid", s));
    NB_LAUNCH("gmres_resid", s, k_resid<<<vec_grid, kChunk, 0, s>>>(a));
    NB_CHECK_LAUNCH();
    NB_TRY_CUDA(cudaMemcpyAsync(iters.data(), ws->iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaMemcpyAsync(done.data(), ws->done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaMemcpyAsync(rt.data(), ws->res_true, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaMemcpyAsync(&tc_err, ws->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    loop_copy(ws, s);
    NB_TRY_CUDA(cudaStreamSynchronize(s));  // the solve's one host sync
    loop_count(ws);
    for (int q = 0; q < nrhs; ++q) {
      total[q] = iters[q];
      conv[q] = done[q];
      converged = converged && done[q];
    }
  } else {
    // Refinement form, shared by mixed precision and restarted GMRES: x accumulates in FP64
    // (xacc), b holds the current residual b0 - L x with the FP32 operator and FP64 sums, and
    // each sweep solves the correction equation L d = b with GMRES from d = 0, x += d.
    NB_TRY_CUDA(cudaMemcpyAsync(ws->b0, ws->b, (size_t)n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    NB_TRY_CUDA(cudaMemsetAsync(ws->xacc, 0, (size_t)n * nrhs * sizeof(double2), s));
    NB_TRY_CUDA(cudaMemsetAsync(ws->outer_done, 0, nrhs * sizeof(int), s));
    GArgs a = make_args(op, ws, op->L);
    a.x = ws->xacc;
    a.skip = ws->outer_done;
    int budget = o.max_iter;
    converged = false;
    bool first = true;
    std::vector<int> od(nrhs), inner_done(nrhs);
    std::vector<double> prev(nrhs, 1.0);
    // one sweep with the given engine: GMRES on the correction equation (at most a.maxit
    // iterations), x += d, the true residual and the outer convergence flags
    auto sweep_once = [&](int eng) -> nat_bem_status {
      NB_TRY(gmres_run(op, ws, a, eng, 1, d_p, s));
      if (first) {  // the first run started from b = b0: its ||b|| is ||R g||
        NB_TRY_CUDA(cudaMemcpyAsync(ws->b0norm, ws->bnorm, nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
        first = false;
      }
      NB_TRY(matvec(op, ws, 0, accurate, ws->w, nullptr, nullptr, "gemv_resid", s));
      NB_LAUNCH("ir_residual", s, k_ir_residual<<<vec_grid, kChunk, 0, s>>>(a, ws->b0, ws->outer_done, o.tol));
      NB_CHECK_LAUNCH();
      NB_TRY_CUDA(cudaMemcpyAsync(iters.data(), ws->iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
      NB_TRY_CUDA(cudaMemcpyAsync(od.data(), ws->outer_done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
      NB_TRY_CUDA(cudaMemcpyAsync(inner_done.data(), ws->done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
      NB_TRY_CUDA(cudaMemcpyAsync(rt.data(), ws->res_true, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
      NB_TRY_CUDA(cudaMemcpyAsync(&tc_err, ws->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
      loop_copy(ws, s);
      NB_TRY_CUDA(cudaStreamSynchronize(s));  // one host sync per sweep
      loop_count(ws);
      int used = 0;
      for (int q = 0; q < nrhs; ++q) {
        total[q] += iters[q];
        used = std::max(used, iters[q]);
      }
      budget -= std::max(used, 1);
      ++refinements;
      converged = true;
      for (int q = 0; q < nrhs; ++q) {
        conv[q] = od[q];
        converged = converged && od[q];
      }
      return NAT_BEM_OK;
    };
    bool finish = !mixed;
    if (mixed) {
      // Mixed precision iterative refinement: inner GMRES on the BF16 copy of L (or the
      // tensor-core products) to inner_tol relative to the current residual.
      // Inner solves on the fused Arnoldi kernels keep an FP32 Krylov basis (in V's memory)
      // and an FP32 copy of w: GB300's FP64 pipe made the FP64 Gram-Schmidt the largest cost
      // of multi-RHS inner solves, and they stop at 1e-2.
      static const bool fp64_basis = std::getenv("NATBEM_FP64_BASIS") != nullptr;
      const bool fp32_basis =
          !fp64_basis && ws->coop_blocks > 0 && ws->wf && (nrhs <= kArnUnitsMinRhs || ws->pbu != nullptr);
      // The last sweeps need only the contraction still missing to the outer target, so
      // their inner tolerance is loosened (sweep_inner_tol); NATBEM_FIXED_INNER_TOL keeps
      // inner_tol for every sweep.
      static const bool fixed_inner = std::getenv("NATBEM_FIXED_INNER_TOL") != nullptr;
      for (int sweep = 0; sweep < o.max_refinements && budget > 0; ++sweep) {
        double rho = 0.0;
        for (int q = 0; q < nrhs; ++q)
          if (!od[q]) rho = std::max(rho, sweep == 0 ? 1.0 : prev[q]);
        a.tol = fixed_inner ? o.inner_tol : sweep_inner_tol(o.inner_tol, o.tol, rho);
        a.maxit = std::min(std::min(o.inner_max_iter, budget), ws->m);
        a.Vf = fp32_basis ? reinterpret_cast<float2*>(ws->V) : nullptr;
        NB_TRY(sweep_once(inner));
        a.Vf = nullptr;
        if (converged) break;
        // A sweep that shrank some residual by less than 10x (the low-precision operator's
        // error is comparable to the inner tolerance: high k, ill-conditioned L) or that used
        // up the budget: the rest is solved with the FP32 operator below, with a fresh
        // iteration budget. It runs even when the refinement count is spent.
        // A stall with every open residual within kResidualFloor x tol is the rounding floor
        // of the FP32 residual product itself (on modal low-k solves the sweeps contract by
        // 0.01-0.09 down to 1-2e-6 and then by 0.7, and FP32 GMRES on the correction equation
        // ends at the same level): the solve stops there instead.
        // a stall: some open residual contracted by a factor above 0.1, or above twice the
        // inner tolerance of a loosened sweep
        const double stall = std::max(0.1, 2.0 * a.tol);
        double worst = 0.0;
        bool at_floor = true;
        for (int q = 0; q < nrhs; ++q)
          if (!od[q]) {
            worst = std::max(worst, rt[q] / prev[q]);
            at_floor = at_floor && rt[q] <= kResidualFloor * o.tol;
          }
        if (worst > stall && at_floor) {
          converged = true;
          for (int q = 0; q < nrhs; ++q) conv[q] = 1;
          break;
        }
        if (worst > stall || budget <= 0 || sweep + 1 >= o.max_refinements) {
          finish = true;
          break;
        }
        prev = rt;
      }
    }
    if (finish && !converged) {
      // GMRES with the FP32 operator on the correction equation, in cycles of at most m
      // iterations (one cycle when unrestarted), until GMRES's residual estimate meets the
      // tolerance relative to ||R g|| (the plain path's criterion; after mixed sweeps, half
      // of it) or the true residual does.
      if (mixed) budget = o.max_iter;
      a.tol = mixed ? 0.5 * o.tol : o.tol;
      while (budget > 0) {
        a.bscale = first ? nullptr : ws->b0norm;
        a.maxit = std::min(budget, ws->m);
        NB_TRY(sweep_once(accurate));
        converged = true;
        for (int q = 0; q < nrhs; ++q) {
          conv[q] = od[q] || inner_done[q];
          converged = converged && conv[q];
        }
        if (converged) break;
      }
    }
  }
  if (tc_err) {
    set_error("tensor-core product: a bounded wait gave up (code " + std::to_string(tc_err) + ")");
    return NAT_BEM_ECUDA;
  }
  int maxit = 0;
  double maxres = 0.0;
  for (int q = 0; q < nrhs; ++q) {
    maxit = std::max(maxit, total[q]);
    maxres = std::max(maxres, rt[q]);
  }
  if (info) {
    info->iterations = maxit;
    info->refinements = refinements;
    info->rel_residual = maxres;
  }
  if (per_rhs) {
    per_rhs->resize(nrhs);
    for (int q = 0; q < nrhs; ++q) (*per_rhs)[q] = nat_bem_solve_info{total[q], refinements, rt[q]};
  }
  if (per_conv) *per_conv = conv;
  if (!converged) {
    set_error("GMRES did not reach the tolerance within the iteration limits");
    return NAT_BEM_ENOCONV;
  }
  return NAT_BEM_OK;
}

}  // namespace natbem
