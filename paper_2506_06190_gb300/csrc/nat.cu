// Forward pass of the neural acoustic transfer field (paper Sec. 3.3, Eq. 3 and 4; Sec. 3.4):
// grid encoding over the spherical coordinates, positional encoding of the condition variables
// and the frequency, and a 4 x 128 MLP with ReLU and a linear output layer, fused in one
// persistent kernel on the tensor cores.
//
// A block runs two or three independent groups of four warps; each group owns a tile of 128
// queries (one thread per query), an activation tile A in shared memory and 128 TMEM columns,
// so one group's epilogues overlap the other groups' MMAs. Per tile:
//   encode   each thread forms its query's input row (16 trilinear grid features, then sin and
//            cos of 2^l pi x_d, l = 0..5, for the condition variables and the frequency, zero
//            padding), rounds it to BF16 and writes it as row t of A in the 128-byte-swizzled
//            K-major layout the tensor cores read (only the K steps layer 0 reads);
//   layer l  one thread issues the tcgen05.mma (kind::f16, BF16 A and W_l, M = 128, N = 128,
//            K = 16 each) into the group's FP32 TMEM accumulator and commits them to the
//            group's mbarrier; after the bounded wait each warp reads its 32 TMEM lanes
//            (tcgen05.ld), adds the bias, applies ReLU while rounding to BF16 and writes the next
//            layer's input back into A;
//   output   the last layer (N = n_out rounded up to 16) plus bias goes to global memory (FP32).
// The encoding of the next tile runs in pieces while each layer's MMAs are in flight (grid level
// l during layer l from rows requested two layers earlier, the positional encoding spread over
// the later layers) and collects in TMEM columns next to the accumulators, so the table gathers'
// latency hides behind the tensor cores instead of adding to the tile's critical path.
// The weights stay in shared memory for the kernel's lifetime (at most 160 KB) and the biases
// live in the kernel's parameter space (uniform reads through the constant cache), so HBM only
// carries the queries, the grid tables (through L2) and the outputs. The tables are half
// precision (as tiny-cuda-nn stores its grid parameters); a dense level is laid out so that the
// four vertices of a cell face at one z share a 32-byte sector.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace natbem {
namespace {
constexpr int kNatLevels[4] = {8, 16, 32, 64};
constexpr int kNatWidth = 128;
constexpr int kNatHidden = 4;
constexpr uint32_t kNatTile = 128 * 128 * 2;             // one 128 x 128 BF16 operand
constexpr uint32_t kNatRegion = 128 * 128;               // 128 rows x 64 K values (128 B)
constexpr uint32_t kNatSmemLimit = 227 * 1024;

// Shared memory of a block with G groups: layer 0's weights (the regions its K steps read),
// three hidden layers, the output layer (n16 rows), G activation tiles, barriers, alignment.
__host__ __device__ constexpr uint32_t nat_w0_bytes(int k0) { return (uint32_t)((k0 + 3) / 4) * kNatRegion; }
__host__ __device__ constexpr uint32_t nat_smem_bytes(int k0, int n16, int groups) {
  return nat_w0_bytes(k0) + 3 * kNatTile + (uint32_t)n16 * 256u + (uint32_t)groups * kNatTile + 64 + 1024;
}
__host__ __device__ constexpr int nat_k0(int d) { return (16 + 12 * (d - 3) + 15) / 16; }  // layer-0 K steps
constexpr uint32_t kPrime1 = 2654435761u, kPrime2 = 805459861u;

struct NatBias {
  float b[(kNatHidden + 1) * kNatWidth];  // hidden layers 128 each, then the output layer
};
}  // namespace
}  // namespace natbem

struct nat_field {
  int32_t n_cond = 0, n_out = 0, n16 = 0, table_log2 = 0;
  uint2* tables = nullptr;      // the four levels in half precision (4 features = 8 bytes per
                                // vertex): a dense level as quads of the (i, j), (i+1, j), (i, j+1),
                                // (i+1, j+1) vertices at each z (32 bytes, one sector); a hashed
                                // level as its rows
  int64_t level_off[4] = {0, 0, 0, 0};  // in 8-byte units, multiples of 4
  uint16_t* weights = nullptr;  // BF16 [out][in]: 4 x 128 x 128, then n16 x 128 (rows >= n_out zero)
  natbem::NatBias bias{};       // host copy, passed by value to the kernel
  int device = 0;
  cudaStream_t stream = nullptr;
  int* err = nullptr;           // bounded-wait failures
  // host buffers: upload and download streams, created on first use
  cudaStream_t up = nullptr, down = nullptr;
};

namespace natbem {

namespace {

__device__ __forceinline__ uint32_t nat_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of 16-byte chunk c (0..15, eight K values each) of row r in a rows x 128 BF16
// K-major operand: two regions of 128-byte rows (K 0..63, then K 64..127), the 16-byte chunks
// of a row permuted by r mod 8 (the 128-byte swizzle; regions are 1024-byte aligned).
__device__ __forceinline__ uint32_t swz(int r, int c, int rows) {
  return (uint32_t)((c >> 3) * (rows * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// max(lo, 0) and max(hi, 0) rounded to nearest-even BF16, lo in the low half
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ uint64_t nat_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// FP32 accumulator, BF16 A and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t nat_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ bool nat_bar_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (uint32_t i = 0; i < (1u << 26); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if ((i & 1023u) == 1023u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) return false;
    }
  }
  return false;
}

// Barriers of one group of four warps (named barriers 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ bool group_all(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r) : "r"((uint32_t)v), "r"(id) : "memory");
  return r != 0;
}

// 32 columns of this warp's 32 TMEM lanes into registers; completes at the next
// tcgen05.wait::ld of the thread.
__device__ __forceinline__ void nat_tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
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
}

// Waits for this thread's TMEM loads; r is passed through the asm so that no use of the
// loaded registers can be scheduled before the wait.
__device__ __forceinline__ void nat_tmem_wait(uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

__device__ __forceinline__ void nat_tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  nat_tmem_ld32_async(taddr, r);
  nat_tmem_wait(r);
}

// Two or four 32-bit values of this thread into its TMEM lane at consecutive columns (the
// warp's 32 lanes together); complete at the thread's next tcgen05.wait::st.
__device__ __forceinline__ void nat_tmem_st2(uint32_t taddr, uint32_t a, uint32_t b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void nat_tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(a), "r"(b),
               "r"(c), "r"(d)
               : "memory");
}


// The D inputs of query q (zeros past the end).
template <int D>
__device__ __forceinline__ void nat_load_x(const float* __restrict__ x, int64_t q, int64_t n, float (&xv)[D]) {
#pragma unroll
  for (int d = 0; d < D; ++d) xv[d] = q < n ? __ldg(x + q * D + d) : 0.f;
}

// The four features of a vertex: two half2 in 8 bytes.
__device__ __forceinline__ float4 nat_h4(uint32_t lo, uint32_t hi) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  return make_float4(a.x, a.y, b.x, b.y);
}

// The table rows of one grid level for one query: the eight corners' features (FP16, 8 bytes
// each), requested by nat_fetch and used by nat_finish a pipeline stage later.
struct NatRows {
  uint4 r[4];  // corners 2c and 2c + 1 in r[c]
};

// Grid level lvl (8 << lvl cells per axis) of the query at xv: the cell and the trilinear
// weights along each axis.
template <int D>
__device__ __forceinline__ void nat_cell(int lvl, const float (&xv)[D], int (&i0)[3], float (&w1)[3]) {
  const int N = 8 << lvl;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = fminf(fmaxf(xv[a], 0.f), 1.f) * (float)N;
    i0[a] = min((int)p, N - 1);  // p >= 0: truncation is the floor
    w1[a] = p - (float)i0[a];
  }
}

// Requests the eight corner rows of level lvl. dense_mask bit lvl: the level is stored densely
// (the quads at z = k and z = k + 1: four 16-byte loads from two 32-byte sectors), else hashed.
template <int D>
__device__ __forceinline__ void nat_fetch(int lvl, const float (&xv)[D], const uint2* __restrict__ tables,
                                          const int (&offs)[4], uint32_t hmask, int dense_mask, NatRows& rows) {
  const int N = 8 << lvl;
  int i0[3];
  float w1[3];
  nat_cell<D>(lvl, xv, i0, w1);
  if (dense_mask & (1 << lvl)) {
    const uint4* tq = reinterpret_cast<const uint4*>(tables + offs[lvl]);
    const uint32_t q0 = (uint32_t)i0[0] + (uint32_t)N * ((uint32_t)i0[1] + (uint32_t)N * (uint32_t)i0[2]);
    const uint32_t q1 = q0 + (uint32_t)(N * N);
    rows.r[0] = __ldg(tq + 2 * q0);
    rows.r[1] = __ldg(tq + 2 * q0 + 1);
    rows.r[2] = __ldg(tq + 2 * q1);
    rows.r[3] = __ldg(tq + 2 * q1 + 1);
  } else {
    const uint2* tl = tables + offs[lvl];
    const uint32_t hx[2] = {(uint32_t)i0[0], (uint32_t)i0[0] + 1u};
    const uint32_t hy[2] = {(uint32_t)i0[1] * kPrime1, ((uint32_t)i0[1] + 1u) * kPrime1};
    const uint32_t hz[2] = {(uint32_t)i0[2] * kPrime2, ((uint32_t)i0[2] + 1u) * kPrime2};
    uint2 u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) u[c] = __ldg(tl + ((hx[c & 1] ^ hy[(c >> 1) & 1] ^ hz[c >> 2]) & hmask));
#pragma unroll
    for (int c = 0; c < 4; ++c) rows.r[c] = make_uint4(u[2 * c].x, u[2 * c].y, u[2 * c + 1].x, u[2 * c + 1].y);
  }
}

// The four trilinear features of level lvl from its fetched rows, as two BF16 pairs.
template <int D>
__device__ __forceinline__ void nat_finish(int lvl, const float (&xv)[D], const NatRows& rows, uint32_t& lo,
                                           uint32_t& hi) {
  int i0[3];
  float w1[3], w0[3];
  nat_cell<D>(lvl, xv, i0, w1);
#pragma unroll
  for (int a = 0; a < 3; ++a) w0[a] = 1.f - w1[a];
  const float wxy[4] = {w0[0] * w0[1], w1[0] * w0[1], w0[0] * w1[1], w1[0] * w1[1]};
  float4 v[8];  // corner c = di + 2 dj + 4 dk
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    v[2 * c] = nat_h4(rows.r[c].x, rows.r[c].y);
    v[2 * c + 1] = nat_h4(rows.r[c].z, rows.r[c].w);
  }
  float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float wt = wxy[c & 3] * (c >> 2 ? w1[2] : w0[2]);
    f0 = fmaf(wt, v[c].x, f0);
    f1 = fmaf(wt, v[c].y, f1);
    f2 = fmaf(wt, v[c].z, f2);
    f3 = fmaf(wt, v[c].w, f3);
  }
  lo = pack2(f0, f1);
  hi = pack2(f2, f3);
}

// The positional encoding of the condition variables and the frequency (inputs 3..D-1):
// sin and cos of 2^l pi x_d, l = 0..5, as BF16 pairs after the 16 grid features.
// Input d's six pairs, as BF16 pairs.
__device__ __forceinline__ void nat_pe_input(float xd, uint32_t (&o)[6]) {
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    float s, c;
    sincospif(ldexpf(xd, l), &s, &c);  // sin, cos of 2^l pi x_d
    o[l] = pack2(s, c);
  }
}

// The encoded row of query q as row t of A: the K steps layer 0 reads (2 K0 chunks of 16
// bytes), zero past the end of the queries and in the padding.
template <int K0>
__device__ __forceinline__ void nat_store_row(const uint32_t (&pk)[8 * K0], int64_t q, int64_t n, uint8_t* sA, int t) {
  const bool live = q < n;
#pragma unroll
  for (int c = 0; c < 2 * K0; ++c)
    *reinterpret_cast<uint4*>(sA + swz(t, c, 128)) =
        live ? make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]) : make_uint4(0u, 0u, 0u, 0u);
}
}  // namespace

// x: n x D float32 inputs in [0, 1] (D = 4 + n_cond <= 12); out: n x n_out float32.
// G groups of four warps per block, each with its own 128-query tile.
template <int D, int G>
__global__ void __launch_bounds__(G * 128, 1)
k_nat_forward(const float* __restrict__ x, int64_t n, const uint2* __restrict__ tables, int off1, int off2,
              int off3, int log2, int dense_mask, const uint16_t* __restrict__ weights, int n_out, int n16,
              float* __restrict__ out, int* __restrict__ err, const __grid_constant__ NatBias P) {
  constexpr int K0 = nat_k0(D);
  constexpr uint32_t kW0 = nat_w0_bytes(K0);
  extern __shared__ uint8_t nat_raw[];
  const uint32_t raw = nat_smem_u32(nat_raw);
  uint8_t* base = nat_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* sW = base;                                        // W0, W1..W3 at kW0 + (l-1) tiles, Wout
  uint8_t* sWout = base + kW0 + 3 * kNatTile;
  uint8_t* sA0 = sWout + (uint32_t)n16 * 256u;               // G activation tiles
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA0 + G * kNatTile);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + G);
  const int g = threadIdx.x >> 7, t = threadIdx.x & 127, warp = threadIdx.x >> 5;
  uint8_t* sA = sA0 + g * kNatTile;

  // weights into the swizzled operand layout, once per block
  for (int i = threadIdx.x; i < (int)(kW0 / 16); i += G * 128) {  // layer 0: its K regions only
    const int o = (i >> 3) & 127, c = (i >> 10) * 8 + (i & 7);
    const uint4 v = *reinterpret_cast<const uint4*>(weights + ((size_t)o * 128 + c * 8));
    *reinterpret_cast<uint4*>(sW + swz(o, c, 128)) = v;
  }
  for (int i = threadIdx.x; i < 3 * 128 * 16; i += G * 128) {
    const int l = i >> 11, o = (i >> 4) & 127, c = i & 15;
    const uint4 v = *reinterpret_cast<const uint4*>(weights + ((size_t)((l + 1) * 128 + o) * 128 + c * 8));
    *reinterpret_cast<uint4*>(sW + kW0 + l * kNatTile + swz(o, c, 128)) = v;
  }
  for (int i = threadIdx.x; i < n16 * 16; i += G * 128) {
    const int o = i >> 4, c = i & 15;
    const uint4 v = *reinterpret_cast<const uint4*>(weights + ((size_t)(kNatHidden * 128 + o) * 128 + c * 8));
    *reinterpret_cast<uint4*>(sWout + swz(o, c, n16)) = v;
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < G; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(nat_smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // G groups x 128 accumulator columns, then each group's staging columns for the next
  // tile's encoded row (8 K0 <= 64 each; G K0 <= 16 since three groups only run with K0 <= 4)
  constexpr uint32_t kCols = 512u;
  static_assert(G * 128 + G * 8 * K0 <= 512, "TMEM columns");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nat_smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot + (uint32_t)(g * 128);                 // the group's columns
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);      // this warp's lanes
  const uint32_t stage = *tmem_slot + (uint32_t)(G * 128 + g * 8 * K0) + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t bar = nat_smem_u32(&bars[g]);
  const int offs[4] = {0, off1, off2, off3};
  const uint32_t hmask = (1u << log2) - 1u;
  const uint32_t a0 = nat_smem_u32(sA);
  uint32_t phase = 0;
  bool ok_all = true;

  // Software pipeline over the group's tiles: while the MMAs of layer l of tile i run, the
  // group encodes one piece of tile i + 1 into its TMEM staging columns (grid level l for l < 4
  // from rows requested two layers earlier; a share of the positional encoding from layer 1
  // on); the row goes into A once the output layer's MMA has read it.
  const int64_t tstride = (int64_t)gridDim.x * G;
  int64_t tile = (int64_t)blockIdx.x * G + g;
  float xn[D], xnn[D];  // inputs of tiles i + 1 and i + 2
  NatRows rb[2];        // requested rows of the levels nat_finish uses next (level l in rb[l & 1])
  {
    uint32_t pk[8 * K0];
#pragma unroll
    for (int i = 0; i < 8 * K0; ++i) pk[i] = 0u;
    float xv[D];
    nat_load_x<D>(x, tile * 128 + t, n, xv);
#pragma unroll
    for (int lvl = 0; lvl < 4; ++lvl) {
      nat_fetch<D>(lvl, xv, tables, offs, hmask, dense_mask, rb[0]);
      nat_finish<D>(lvl, xv, rb[0], pk[2 * lvl], pk[2 * lvl + 1]);
    }
#pragma unroll
    for (int d = 3; d < D; ++d) {
      uint32_t o[6];
      nat_pe_input(xv[d], o);
#pragma unroll
      for (int l = 0; l < 6; ++l) pk[8 + (d - 3) * 6 + l] = o[l];
    }
    nat_store_row<K0>(pk, tile * 128 + t, n, sA, t);
#pragma unroll
    for (int c = 0; c < 8 * K0; c += 2) nat_tmem_st2(stage + (uint32_t)c, 0u, 0u);  // the padding stays zero
  }
  nat_load_x<D>(x, (tile + tstride) * 128 + t, n, xn);
  nat_fetch<D>(0, xn, tables, offs, hmask, dense_mask, rb[0]);
  nat_fetch<D>(1, xn, tables, offs, hmask, dense_mask, rb[1]);
  for (;; tile += tstride) {
    const int64_t q0 = tile * 128;
    if (q0 >= n) break;  // uniform over the group
    const int64_t q = q0 + t;
    nat_load_x<D>(x, q + 2 * tstride * 128, n, xnn);
#pragma unroll
    for (int l = 0; l <= kNatHidden; ++l) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A visible to the tensor cores
      group_sync(1 + g);
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool last = l == kNatHidden;
        const uint32_t b0 = nat_smem_u32(l == 0 ? sW : last ? sWout : sW + kW0 + (l - 1) * kNatTile);
        const uint32_t bregion = last ? (uint32_t)n16 * 128u : kNatRegion;
        const uint32_t idesc = nat_idesc(last ? (uint32_t)n16 : 128u);
        const int ksteps = l == 0 ? K0 : 8;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {  // K = 16 per MMA: 32 bytes, 4 per 128-byte region
          if (kk < ksteps) {
            const uint64_t da = nat_desc(a0 + (uint32_t)(kk >> 2) * kNatRegion + (uint32_t)(kk & 3) * 32u);
            const uint64_t db = nat_desc(b0 + (uint32_t)(kk >> 2) * bregion + (uint32_t)(kk & 3) * 32u);
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(da), "l"(db), "r"(idesc), "r"(kk > 0 ? 1u : 0u));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
      }
      // the next tile's piece while the MMAs run: level l from the rows requested two layers
      // earlier into the staging columns, then the request of level l + 2 (of levels 0 and 1 of
      // the tile after it during layers 2 and 3); input d's positional encoding during layer
      // 1 + (d - 3) mod 4
      if (l < 4) {
        uint32_t lo, hi;
        nat_finish<D>(l, xn, rb[l & 1], lo, hi);
        nat_tmem_st2(stage + (uint32_t)(2 * l), lo, hi);
        if (l < 2) nat_fetch<D>(l + 2, xn, tables, offs, hmask, dense_mask, rb[l & 1]);
        else nat_fetch<D>(l - 2, xnn, tables, offs, hmask, dense_mask, rb[l & 1]);
      }
      if (l >= 1) {
#pragma unroll
        for (int d = 3; d < D; ++d)
          if ((d - 3) % 4 == l - 1) {  // input d during layer 1 + (d - 3) mod 4
            uint32_t o[6];
            nat_pe_input(xn[d], o);
            const uint32_t c = stage + (uint32_t)(8 + (d - 3) * 6);
            nat_tmem_st4(c, o[0], o[1], o[2], o[3]);
            nat_tmem_st2(c + 4u, o[4], o[5]);
          }
      }
      // one warp polls the mbarrier; the others wait at the group barrier without issuing
      bool ok = true;
      if (t < 32) ok = nat_bar_wait(bar, phase);
      ok = group_all(1 + g, ok);
      phase ^= 1u;
      if (!ok) {
        if (t == 0) atomicOr(err, 1);
        ok_all = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (l < kNatHidden) {
        // bias, ReLU, BF16: the next layer's input, row t of A
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
          uint32_t v[32];
          nat_tmem_ld32(tlane + (uint32_t)(cb * 32), v);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t p4[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int col = cb * 32 + c * 8 + 2 * h;
              p4[h] = pack2_relu(__uint_as_float(v[c * 8 + 2 * h]) + P.b[l * 128 + col],
                                 __uint_as_float(v[c * 8 + 2 * h + 1]) + P.b[l * 128 + col + 1]);
            }
            *reinterpret_cast<uint4*>(sA + swz(t, cb * 4 + c, 128)) = make_uint4(p4[0], p4[1], p4[2], p4[3]);
          }
        }
      } else {
        const bool vec = (n_out & 3) == 0;
        for (int cb = 0; cb < n16; cb += 32) {
          uint32_t v[32];
          nat_tmem_ld32(tlane + (uint32_t)cb, v);
          if (q < n) {
            float* o = out + q * n_out;
            if (vec) {
#pragma unroll
              for (int c = 0; c < 32; c += 4)
                if (cb + c < n_out)
                  *reinterpret_cast<float4*>(o + cb + c) = make_float4(
                      __uint_as_float(v[c]) + P.b[kNatHidden * 128 + cb + c],
                      __uint_as_float(v[c + 1]) + P.b[kNatHidden * 128 + cb + c + 1],
                      __uint_as_float(v[c + 2]) + P.b[kNatHidden * 128 + cb + c + 2],
                      __uint_as_float(v[c + 3]) + P.b[kNatHidden * 128 + cb + c + 3]);
            } else {
#pragma unroll
              for (int c = 0; c < 32; ++c)
                if (cb + c < n_out) o[cb + c] = __uint_as_float(v[c]) + P.b[kNatHidden * 128 + cb + c];
            }
          }
        }
        // the output layer's MMAs have read A: the next tile's row goes in
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        uint32_t pk[8 * K0];
#pragma unroll
        for (int c = 0; c < 8 * K0; c += 32) {
          uint32_t v[32];
          nat_tmem_ld32(stage + (uint32_t)c, v);
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (c + i < 8 * K0) pk[c + i] = v[i];
        }
        nat_store_row<K0>(pk, q + tstride * 128, n, sA, t);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
#pragma unroll
    for (int d = 0; d < D; ++d) xn[d] = xnn[d];
    if (!ok_all) break;
  }
  if (!ok_all && t < 32) nat_bar_wait(bar, phase ^ 1u);  // MMAs still in flight: bounded wait
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot), "r"(kCols));
}

// The caller's FP32 table rows (level after level, min((N+1)^3, 2^log2) rows each) to the
// half-precision device layout (round to nearest): a dense level as quads, one thread per quad
// (i, j, k), i, j < N, k <= N; a hashed level row by row.
__global__ void k_nat_pack(const float4* __restrict__ in, int N, int dense, int64_t rows, uint2* __restrict__ out) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto h4 = [](float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
  };
  if (!dense) {
    if (u < rows) out[u] = h4(in[u]);
    return;
  }
  const int64_t quads = (int64_t)N * N * (N + 1);
  if (u >= quads) return;
  const int i = (int)(u % N), j = (int)((u / N) % N), k = (int)(u / ((int64_t)N * N));
  const int64_t S1 = N + 1;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t r = (i + (c & 1)) + S1 * ((j + (c >> 1)) + S1 * k);
    out[4 * u + c] = h4(in[r]);
  }
}

// The caller's FP32 weights (w_in values: four 128 x 128 layers, then n_out x 128) to BF16
// rounded to nearest-even, with the output layer's padding rows (up to n16) zero.
__global__ void k_nat_weights_bf16(const float* __restrict__ in, int64_t w_in, int64_t w_out,
                                   uint16_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w_out) return;
  const __nv_bfloat16 v = __float2bfloat16_rn(i < w_in ? in[i] : 0.0f);
  out[i] = *reinterpret_cast<const uint16_t*>(&v);
}

template <int D>
static nat_bem_status nat_launch_d(const nat_field* f, const float* dx, int64_t n, float* dout, cudaStream_t s,
                                   int sms, bool& attr_done) {
  constexpr int K0 = nat_k0(D);
  const int64_t tiles = (n + 127) / 128;
  int dense_mask = 0;
  for (int l = 0; l < 4; ++l) {
    const int64_t v = (int64_t)(kNatLevels[l] + 1) * (kNatLevels[l] + 1) * (kNatLevels[l] + 1);
    if (v <= ((int64_t)1 << f->table_log2)) dense_mask |= 1 << l;
  }
  constexpr bool kThreeFit = nat_smem_bytes(K0, 16, 3) <= kNatSmemLimit;  // three groups possible at all
  if (!attr_done) {
    NB_TRY_CUDA(cudaFuncSetAttribute(k_nat_forward<D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)nat_smem_bytes(K0, 128, 2)));
    if constexpr (kThreeFit)
      NB_TRY_CUDA(cudaFuncSetAttribute(k_nat_forward<D, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kNatSmemLimit));
    attr_done = true;
  }
  const int off1 = (int)f->level_off[1], off2 = (int)f->level_off[2], off3 = (int)f->level_off[3];
  bool launched = false;
  if constexpr (kThreeFit) {
    if (nat_smem_bytes(K0, f->n16, 3) <= kNatSmemLimit) {
      const int blocks = (int)std::min<int64_t>((tiles + 2) / 3, (int64_t)sms);
      NB_LAUNCH("nat_forward", s, k_nat_forward<D, 3><<<blocks, 384, nat_smem_bytes(K0, f->n16, 3), s>>>(
          dx, n, f->tables, off1, off2, off3, f->table_log2, dense_mask, f->weights, f->n_out, f->n16, dout,
          f->err, f->bias));
      launched = true;
    }
  }
  if (!launched) {
    const int blocks = (int)std::min<int64_t>((tiles + 1) / 2, (int64_t)sms);
    NB_LAUNCH("nat_forward", s, k_nat_forward<D, 2><<<blocks, 256, nat_smem_bytes(K0, f->n16, 2), s>>>(
        dx, n, f->tables, off1, off2, off3, f->table_log2, dense_mask, f->weights, f->n_out, f->n16, dout,
        f->err, f->bias));
  }
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

static nat_bem_status nat_launch(const nat_field* f, const float* dx, int64_t n, float* dout, cudaStream_t s) {
  static std::mutex mu;
  static bool attr_set[64][13] = {};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    set_error("nat_field_forward: device ordinal out of range");
    return NAT_BEM_ECUDA;
  }
  std::lock_guard<std::mutex> lk(mu);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  bool* attr = attr_set[dev];
  switch (4 + f->n_cond) {
    case 4: return nat_launch_d<4>(f, dx, n, dout, s, sms, attr[4]);
    case 5: return nat_launch_d<5>(f, dx, n, dout, s, sms, attr[5]);
    case 6: return nat_launch_d<6>(f, dx, n, dout, s, sms, attr[6]);
    case 7: return nat_launch_d<7>(f, dx, n, dout, s, sms, attr[7]);
    case 8: return nat_launch_d<8>(f, dx, n, dout, s, sms, attr[8]);
    case 9: return nat_launch_d<9>(f, dx, n, dout, s, sms, attr[9]);
    case 10: return nat_launch_d<10>(f, dx, n, dout, s, sms, attr[10]);
    case 11: return nat_launch_d<11>(f, dx, n, dout, s, sms, attr[11]);
    case 12: return nat_launch_d<12>(f, dx, n, dout, s, sms, attr[12]);
    default:
      set_error("nat_field_forward: 0 <= n_cond <= 8");
      return NAT_BEM_EINVAL;
  }
}

}  // namespace natbem

using namespace natbem;

namespace natbem {
namespace {
constexpr int64_t kNatChunk = int64_t(1) << 20;  // queries per chunk on the host-buffer path

// Host inputs or outputs: chunks of kNatChunk queries in two device buffers each, uploads on
// one stream, the kernels on the caller's, downloads on another, so that chunk c + 1's upload
// and chunk c - 1's download run during chunk c's kernel. Queries are independent: the results
// are the same as one call on device buffers.
nat_bem_status nat_forward_pipelined(nat_field* f, const float* x, bool xdev, int64_t n, float* out, bool odev,
                                     cudaStream_t s) {
  const int D = 4 + f->n_cond;
  if (!f->up) {
    if (cudaStreamCreateWithFlags(&f->up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&f->down, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      set_error("nat_field_forward: could not create copy streams");
      return NAT_BEM_ECUDA;
    }
  }
  float *bx[2] = {nullptr, nullptr}, *bo[2] = {nullptr, nullptr};
  cudaEvent_t ev[7] = {};  // start, uploaded x2, computed x2, downloaded x2
  auto cleanup = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
      dev_free(bx[b], s);
      dev_free(bo[b], s);
    }
  };
  nat_bem_status st = NAT_BEM_OK;
  for (int b = 0; b < 2 && st == NAT_BEM_OK; ++b) {
    if (!xdev) st = dev_alloc_n(&bx[b], (size_t)kNatChunk * D, s);
    if (st == NAT_BEM_OK && !odev) st = dev_alloc_n(&bo[b], (size_t)kNatChunk * f->n_out, s);
  }
  if (st != NAT_BEM_OK) {
    cleanup();
    return st;
  }
  cudaError_t e = cudaMemsetAsync(f->err, 0, sizeof(int), s);  // this call's bounded-wait flag
  for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  // the buffers were allocated on s; the copy streams start after that
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f->up, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f->down, ev[0], 0);
  cudaEvent_t *uploaded = ev + 1, *computed = ev + 3, *downloaded = ev + 5;
  const int64_t chunks = (n + kNatChunk - 1) / kNatChunk;
  for (int64_t c = 0; c < chunks && e == cudaSuccess && st == NAT_BEM_OK; ++c) {
    const int b = (int)(c & 1);
    const int64_t q0 = c * kNatChunk, cnt = std::min(kNatChunk, n - q0);
    const float* cx = x + q0 * D;
    float* co = out + q0 * f->n_out;
    if (!xdev) {
      if (c >= 2) e = cudaStreamWaitEvent(f->up, computed[b], 0);  // chunk c - 2 has read bx[b]
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bx[b], cx, (size_t)cnt * D * sizeof(float), cudaMemcpyHostToDevice, f->up);
      if (e == cudaSuccess) e = cudaEventRecord(uploaded[b], f->up);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, uploaded[b], 0);
      cx = bx[b];
    }
    if (!odev) {
      if (c >= 2 && e == cudaSuccess) e = cudaStreamWaitEvent(s, downloaded[b], 0);  // bo[b] is free
      co = bo[b];
    }
    if (e != cudaSuccess) break;
    st = nat_launch(f, cx, cnt, co, s);
    if (st != NAT_BEM_OK) break;
    e = cudaEventRecord(computed[b], s);
    if (!odev) {
      if (e == cudaSuccess) e = cudaStreamWaitEvent(f->down, computed[b], 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + q0 * f->n_out, bo[b], (size_t)cnt * f->n_out * sizeof(float),
                            cudaMemcpyDeviceToHost, f->down);
      if (e == cudaSuccess) e = cudaEventRecord(downloaded[b], f->down);
    }
  }
  int err = 0;
  if (e == cudaSuccess && st == NAT_BEM_OK) {
    // the caller's stream ends after the last download; the buffers are freed on it
    e = cudaEventRecord(ev[0], f->down);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[0], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  } else {
    cudaStreamSynchronize(f->up);
    cudaStreamSynchronize(f->down);
    cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    set_error(std::string("nat_field_forward: ") + cudaGetErrorString(e));
    st = NAT_BEM_ECUDA;
  } else if (st == NAT_BEM_OK && err) {
    set_error("nat_field_forward: a bounded wait on the tensor cores gave up");
    st = NAT_BEM_ETIMEOUT;
  }
  cleanup();
  return st;
}
}  // namespace
}  // namespace natbem

extern "C" {

nat_bem_status nat_field_create(int32_t n_cond, int32_t n_out, int32_t table_log2, const float* tables,
                                const float* weights, const float* biases, void* cuda_stream,
                                nat_field** out) {
  try {
    clear_error();
    if (!out || !tables || !weights || !biases) {
      set_error("nat_field_create: NULL argument");
      return NAT_BEM_EINVAL;
    }
    *out = nullptr;
    if (n_cond < 0 || n_cond > 8 || n_out < 1 || n_out > 128 || table_log2 < 12 || table_log2 > 24) {
      set_error("nat_field_create: need 0 <= n_cond <= 8, 1 <= n_out <= 128, 12 <= table_log2 <= 24");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    nat_field* f = new nat_field();
    f->n_cond = n_cond;
    f->n_out = n_out;
    f->table_log2 = table_log2;
    f->stream = s;
    cudaGetDevice(&f->device);
    // input rows per level, and the device layout's size per level (8-byte units)
    int64_t rows = 0, units = 0;
    int64_t in_off[4], in_rows[4];
    bool dense[4];
    for (int l = 0; l < 4; ++l) {
      const int64_t N = kNatLevels[l];
      const int64_t v = (N + 1) * (N + 1) * (N + 1);
      dense[l] = v <= ((int64_t)1 << table_log2);
      in_off[l] = rows;
      in_rows[l] = std::min<int64_t>(v, (int64_t)1 << table_log2);
      rows += in_rows[l];
      f->level_off[l] = units;
      units += dense[l] ? 4 * N * N * (N + 1) : in_rows[l];
      units = (units + 3) / 4 * 4;
    }
    auto fail = [&](nat_bem_status st) {
      nat_field_destroy(f);
      return st;
    };
    f->n16 = (n_out + 15) / 16 * 16;
    const size_t w_rows = (size_t)4 * 128 + (size_t)f->n16;
    // weights: four 128 x 128 layers, then n_out x 128; the output layer is padded to n16 rows
    const size_t w_in = (size_t)4 * 128 * 128 + (size_t)n_out * 128;
    const float4* din = nullptr;
    float4* tin = nullptr;
    const float* dw = nullptr;
    float* tw = nullptr;
    nat_bem_status st = to_device(reinterpret_cast<const float4*>(tables), (size_t)rows, s, &din, &tin);
    if (st == NAT_BEM_OK) st = to_device(weights, w_in, s, &dw, &tw);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&f->tables, (size_t)units, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&f->weights, w_rows * 128, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&f->err, 1, s);
    if (st != NAT_BEM_OK) {
      dev_free(tin, s);
      dev_free(tw, s);
      return fail(st);
    }
    for (int l = 0; l < 4; ++l) {
      const int N = kNatLevels[l];
      const int64_t work = dense[l] ? (int64_t)N * N * (N + 1) : in_rows[l];
      k_nat_pack<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(din + in_off[l], N, dense[l] ? 1 : 0, in_rows[l],
                                                                f->tables + f->level_off[l]);
    }
    const int64_t w_out = (int64_t)w_rows * 128;
    k_nat_weights_bf16<<<(unsigned)((w_out + 255) / 256), 256, 0, s>>>(dw, (int64_t)w_in, w_out, f->weights);
    cudaError_t e = cudaMemsetAsync(f->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f->bias.b, biases, ((size_t)4 * 128 + n_out) * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(tin, s);
    dev_free(tw, s);
    if (e != cudaSuccess) {
      set_error(std::string("nat_field_create: copy failed: ") + cudaGetErrorString(e));
      return fail(NAT_BEM_ECUDA);
    }
    *out = f;
    return NAT_BEM_OK;
  } catch (...) {
    set_error("internal error in nat_field_create");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_field_forward(const nat_field* f, const float* x, int64_t n, float* out, void* cuda_stream) {
  try {
    clear_error();
    if (!f || n < 0 || (n > 0 && (!x || !out))) {
      set_error("nat_field_forward: bad arguments");
      return NAT_BEM_EINVAL;
    }
    if (n == 0) return NAT_BEM_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int D = 4 + f->n_cond;
    const bool xdev = is_device_pointer(x), odev_ = is_device_pointer(out);
    if ((!xdev || !odev_) && n > kNatChunk)
      return nat_forward_pipelined(const_cast<nat_field*>(f), x, xdev, n, out, odev_, s);
    const float* dx = nullptr;
    float* tx = nullptr;
    NB_TRY(to_device(x, (size_t)n * D, s, &dx, &tx));
    const bool odev = is_device_pointer(out);
    float* dout = out;
    float* tout = nullptr;
    nat_bem_status st = NAT_BEM_OK;
    if (!odev) {
      st = dev_alloc_n(&tout, (size_t)n * f->n_out, s);
      dout = tout;
    }
    if (st == NAT_BEM_OK && cudaMemsetAsync(f->err, 0, sizeof(int), s) != cudaSuccess) {  // this call's flag
      set_error("nat_field_forward: could not reset the wait flag");
      st = NAT_BEM_ECUDA;
    }
    if (st == NAT_BEM_OK) st = nat_launch(f, dx, n, dout, s);
    int err = 0;
    if (st == NAT_BEM_OK) {
      cudaError_t e = cudaSuccess;
      if (!odev) e = cudaMemcpyAsync(out, tout, (size_t)n * f->n_out * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&err, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("nat_field_forward: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      } else if (err) {
        set_error("nat_field_forward: a bounded wait on the tensor cores gave up");
        st = NAT_BEM_ETIMEOUT;
      }
    }
    dev_free(tx, s);
    dev_free(tout, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_field_forward");
    return NAT_BEM_ECUDA;
  }
}

void nat_field_destroy(nat_field* f) {
  if (!f) return;
  if (f->up) cudaStreamDestroy(f->up);
  if (f->down) cudaStreamDestroy(f->down);
  dev_free(f->tables, f->stream);
  dev_free(f->weights, f->stream);
  dev_free(f->err, f->stream);
  delete f;
}

}  // extern "C"
