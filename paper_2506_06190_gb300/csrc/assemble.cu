// Assembly of the Burton-Miller collocation operators L and R (paper Sec. 4, Eq. 6; the two
// combined matrices are built directly in one pass, Sec. 4.1).
//
//   L_ij = 1/2 d_ij - int_j [dG/dn_y + beta d2G/dn_x dn_y] dS_y
//   R_ij = -int_j [G + beta dG/dn_x] dS_y - (beta/2) d_ij,     G = e^{ikr}/(4 pi r), beta = i/k
//
// Four kernels:
//   k_geometry           per element: centroid (as a float hi/lo pair), normal, area, the 7
//                        quadrature points as offsets from the centroid with their weights, and
//                        the FP64 copies used by the near-pair kernels.
//   k_assemble_regular   every pair (i, j) that shares no vertex, in FP32: one thread per source
//                        column j holding that element's rule in registers, collocation rows
//                        staged through shared memory and read as broadcasts, coalesced row
//                        stores of L and R. Pairs that share a vertex are skipped.
//   k_assemble_adjacent  vertex-sharing pairs (j != i), 16 lanes per pair over the subdivided
//                        rule: d = x - y formed in float-float arithmetic (where it cancels)
//                        from per-pair FP64 differences, everything after it in FP32 with
//                        compensated sums.
//   k_assemble_self      the self pair, one warp per element: the vertices relative to the
//                        centroid in FP64, the edge geometry and the angular integrals in FP32
//                        with cancellation-free forms.
//
// With d = x - y, r = |d|, rho = k r, q = (d.n_x)(d.n_y)/r^2 the integrands reduce to
//   dG/dn_y + beta H = G/r^2 [ (d.n_y - b/k) + i (a/k - rho d.n_y) ],
//       a = (rho^2 - 3) q + n_x.n_y,   b = rho (3 q - n_x.n_y),
//   G + beta dG/dn_x = G [ 1 - d.n_x / r - i d.n_x / (k r^2) ].
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "internal.h"

namespace natbem {

// ------------------------------------------------------------------------ rule tables
// 7-point degree-5 triangle rule (Radon 1948): centroid weight 9/40, then the orbits of
// (a, a, 1-2a) with a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200.
__constant__ double c_rule7[7][4];          // barycentric l0, l1, l2 and weight (sum 1)
constexpr int kMaxAdjPts = 7 * 64;          // 4^3 sub-triangles
constexpr int kMaxSelfPts = 64;
__device__ double4 g_adj_rule[kMaxAdjPts];  // parent barycentrics and weight (sum 1)
__device__ float4 g_adj_ab[kMaxAdjPts];     // barycentrics l1, l2 as FP32 (hi, lo) pairs
__device__ float g_adj_w[kMaxAdjPts];       // the weight in FP32
__device__ float2 g_glf[kMaxSelfPts];       // Gauss-Legendre nodes / weights on [-1, 1]
__constant__ int c_adj_npts;
__constant__ int c_self_pts;

namespace {

void rule7_host(double out[7][4]) {
  const double s = std::sqrt(15.0);
  const double a = (6.0 - s) / 21.0, wa = (155.0 - s) / 1200.0;
  const double b = (6.0 + s) / 21.0, wb = (155.0 + s) / 1200.0;
  const double t[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40},
                          {a, a, 1 - 2 * a, wa},
                          {a, 1 - 2 * a, a, wa},
                          {1 - 2 * a, a, a, wa},
                          {b, b, 1 - 2 * b, wb},
                          {b, 1 - 2 * b, b, wb},
                          {1 - 2 * b, b, b, wb}};
  for (int i = 0; i < 7; ++i)
    for (int c = 0; c < 4; ++c) out[i][c] = t[i][c];
}

// The 4^levels congruent sub-triangles of the reference triangle, as barycentric corners.
void split(const double tri[3][3], int levels, std::vector<std::array<double, 9>>& out) {
  if (levels == 0) {
    std::array<double, 9> t;
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 3; ++c) t[3 * v + c] = tri[v][c];
    out.push_back(t);
    return;
  }
  double m[3][3];  // midpoints of edges (0,1), (1,2), (2,0)
  for (int c = 0; c < 3; ++c) {
    m[0][c] = 0.5 * (tri[0][c] + tri[1][c]);
    m[1][c] = 0.5 * (tri[1][c] + tri[2][c]);
    m[2][c] = 0.5 * (tri[2][c] + tri[0][c]);
  }
  const double* corner[4][3] = {{tri[0], m[0], m[2]}, {m[0], tri[1], m[1]},
                                {m[2], m[1], tri[2]}, {m[0], m[1], m[2]}};
  for (int s = 0; s < 4; ++s) {
    double sub[3][3];
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 3; ++c) sub[v][c] = corner[s][v][c];
    split(sub, levels - 1, out);
  }
}

void gauss_legendre_host(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), d = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2 * m - 1) * z * p1 - (m - 1) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      d = n * (z * p1 - p0) / (z * z - 1.0);
      double step = p1 / d;
      z -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * d * d);
  }
}

}  // namespace

nat_bem_status upload_rules(int adj_levels, int self_pts) {
  double r7[7][4];
  rule7_host(r7);
  NB_TRY_CUDA(cudaMemcpyToSymbol(c_rule7, r7, sizeof(r7)));
  // vertex-sharing pairs: the 7-point rule on each of the 4^levels sub-triangles
  const double ref[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  std::vector<std::array<double, 9>> subs;
  split(ref, adj_levels, subs);
  std::vector<double4> pts;
  const double wsub = 1.0 / (double)subs.size();
  for (const auto& t : subs)
    for (int q = 0; q < 7; ++q) {
      double l[3];
      for (int c = 0; c < 3; ++c) l[c] = r7[q][0] * t[c] + r7[q][1] * t[3 + c] + r7[q][2] * t[6 + c];
      pts.push_back(make_double4(l[0], l[1], l[2], r7[q][3] * wsub));
    }
  int np = (int)pts.size();
  NB_TRY_CUDA(cudaMemcpyToSymbol(g_adj_rule, pts.data(), np * sizeof(double4)));
  std::vector<float4> ab(np);
  std::vector<float> wf(np);
  for (int i = 0; i < np; ++i) {
    const float ah = (float)pts[i].y, bh = (float)pts[i].z;
    ab[i] = make_float4(ah, (float)(pts[i].y - (double)ah), bh, (float)(pts[i].z - (double)bh));
    wf[i] = (float)pts[i].w;
  }
  NB_TRY_CUDA(cudaMemcpyToSymbol(g_adj_ab, ab.data(), np * sizeof(float4)));
  NB_TRY_CUDA(cudaMemcpyToSymbol(g_adj_w, wf.data(), np * sizeof(float)));
  NB_TRY_CUDA(cudaMemcpyToSymbol(c_adj_npts, &np, sizeof(int)));
  std::vector<double> gx, gw;
  gauss_legendre_host(self_pts, gx, gw);
  std::vector<float2> glf(self_pts);
  for (int i = 0; i < self_pts; ++i) glf[i] = make_float2((float)gx[i], (float)gw[i]);
  NB_TRY_CUDA(cudaMemcpyToSymbol(g_glf, glf.data(), self_pts * sizeof(float2)));
  NB_TRY_CUDA(cudaMemcpyToSymbol(c_self_pts, &self_pts, sizeof(int)));
  return NAT_BEM_OK;
}

// ------------------------------------------------------------------------- geometry
__global__ void k_geometry(const double* __restrict__ V, const int32_t* __restrict__ T, int n,
                           float4* c_hi, float4* c_lo, float4* nrm, float4* qp, int4* vid,
                           double* tri, double* cen, double* nrm64, double* area) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int ia = T[3 * t], ib = T[3 * t + 1], ic = T[3 * t + 2];
  double a[3], b[3], c[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = V[3 * ia + d];
    b[d] = V[3 * ib + d];
    c[d] = V[3 * ic + d];
  }
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                  e1[0] * e2[1] - e1[1] * e2[0]};
  double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double A = 0.5 * len;
  double nn[3] = {cr[0] / len, cr[1] / len, cr[2] / len};
  double cc[3];
  for (int d = 0; d < 3; ++d) cc[d] = (a[d] + b[d] + c[d]) / 3.0;
  float hi[3], lo[3];
  for (int d = 0; d < 3; ++d) {
    hi[d] = (float)cc[d];
    lo[d] = (float)(cc[d] - (double)hi[d]);
  }
  c_hi[t] = make_float4(hi[0], hi[1], hi[2], (float)A);
  c_lo[t] = make_float4(lo[0], lo[1], lo[2], 0.f);
  nrm[t] = make_float4((float)nn[0], (float)nn[1], (float)nn[2], 0.f);
  vid[t] = make_int4(ia, ib, ic, 0);
  const double inv4pi = 0.25 / 3.14159265358979323846;
  for (int q = 0; q < 7; ++q) {
    double y[3];
    for (int d = 0; d < 3; ++d)
      y[d] = c_rule7[q][0] * a[d] + c_rule7[q][1] * b[d] + c_rule7[q][2] * c[d] - cc[d];
    qp[7 * t + q] = make_float4((float)y[0], (float)y[1], (float)y[2],
                                (float)(c_rule7[q][3] * A * inv4pi));
  }
  for (int d = 0; d < 3; ++d) {
    tri[9 * t + d] = a[d];
    tri[9 * t + 3 + d] = b[d];
    tri[9 * t + 6 + d] = c[d];
    cen[3 * t + d] = cc[d];
    nrm64[3 * t + d] = nn[d];
  }
  area[t] = A;
}

// -------------------------------------------------------------- regular pairs (FP32)
namespace {

// 2 pi split for Cody-Waite reduction (Cody & Waite 1980): hi = 2 pi rounded to float,
// lo = float(2 pi - hi); rho - n hi - n lo with n = rint(rho / 2 pi) keeps |t| <= pi.
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.7484555314695172e-7f;
constexpr float kInvTwoPi = 0.159154943091895336f;

__device__ __forceinline__ bool shares_vertex(int4 a, int4 b) {
  return a.x == b.x || a.x == b.y || a.x == b.z || a.y == b.x || a.y == b.y || a.y == b.z ||
         a.z == b.x || a.z == b.y || a.z == b.z;
}

// complex value as two bf16 (real in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16(float re, float im) {
  __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
  return *reinterpret_cast<uint32_t*>(&v);
}

constexpr int kRegThreads = 256;  // source columns per block
constexpr int kRowStage = 64;     // collocation rows staged in shared memory at a time

}  // namespace

__global__ void __launch_bounds__(kRegThreads)
k_assemble_regular(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo,
                   const float4* __restrict__ nrm, const float4* __restrict__ qp,
                   const int4* __restrict__ vid, int n, int ld, int rows_per_block, float k,
                   float2* __restrict__ L, float2* __restrict__ R, uint32_t* __restrict__ Lb) {
  __shared__ float4 s_hi[kRowStage], s_lo[kRowStage], s_n[kRowStage];
  __shared__ int4 s_v[kRowStage];
  const int j = blockIdx.x * kRegThreads + threadIdx.x;
  const bool col_ok = j < n, col_pad = j >= n && j < ld;
  // the source element's rule stays in registers for the whole row range
  float3 chi = make_float3(0.f, 0.f, 0.f), clo = chi, nj = chi;
  float4 q[7];
  int4 vj = make_int4(-1, -1, -1, 0);
  if (col_ok) {
    float4 t = c_hi[j];
    chi = make_float3(t.x, t.y, t.z);
    t = c_lo[j];
    clo = make_float3(t.x, t.y, t.z);
    t = nrm[j];
    nj = make_float3(t.x, t.y, t.z);
#pragma unroll
    for (int p = 0; p < 7; ++p) q[p] = qp[7 * j + p];
    vj = vid[j];
  } else {
#pragma unroll
    for (int p = 0; p < 7; ++p) q[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const float kinv = 1.0f / k;
  const int i_begin = blockIdx.y * rows_per_block;
  const int i_end = min(n, i_begin + rows_per_block);
  for (int ib = i_begin; ib < i_end; ib += kRowStage) {
    const int cnt = min(kRowStage, i_end - ib);
    __syncthreads();
    if (threadIdx.x < cnt) {
      int i = ib + threadIdx.x;
      s_hi[threadIdx.x] = c_hi[i];
      s_lo[threadIdx.x] = c_lo[i];
      s_n[threadIdx.x] = nrm[i];
      s_v[threadIdx.x] = vid[i];
    }
    __syncthreads();
    for (int t = 0; t < cnt; ++t) {
      const int i = ib + t;
      const size_t off = (size_t)i * ld + j;
      if (col_pad) {
        L[off] = make_float2(0.f, 0.f);
        R[off] = make_float2(0.f, 0.f);
        if (Lb) Lb[off] = 0u;
        continue;
      }
      if (!col_ok) continue;
      const int4 vi = s_v[t];
      if (shares_vertex(vi, vj)) continue;  // self and vertex-sharing pairs: FP64 kernel
      const float4 xh = s_hi[t], xl = s_lo[t], ni4 = s_n[t];
      // centroid difference from the hi/lo pairs: exact-ish even for close elements
      const float Dx = (xh.x - chi.x) + (xl.x - clo.x);
      const float Dy = (xh.y - chi.y) + (xl.y - clo.y);
      const float Dz = (xh.z - chi.z) + (xl.z - clo.z);
      const float dny = Dx * nj.x + Dy * nj.y + Dz * nj.z;  // quadrature offsets lie in the plane
      const float Dni = Dx * ni4.x + Dy * ni4.y + Dz * ni4.z;
      const float nxny = ni4.x * nj.x + ni4.y * nj.y + ni4.z * nj.z;
      float Lr = 0.f, Li = 0.f, Rr = 0.f, Ri = 0.f;
#pragma unroll
      for (int p = 0; p < 7; ++p) {
        const float dx = Dx - q[p].x, dy = Dy - q[p].y, dz = Dz - q[p].z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float dnx = Dni - fmaf(q[p].x, ni4.x, fmaf(q[p].y, ni4.y, q[p].z * ni4.z));
        const float rho = k * r;
        const float nq = rintf(rho * kInvTwoPi);
        float th = fmaf(-nq, kTwoPiHi, rho);
        th = fmaf(-nq, kTwoPiLo, th);
        float sn, cs;
        __sincosf(th, &sn, &cs);
        const float gw = rinv * q[p].w;  // w A / (4 pi r)
        const float Gr = cs * gw, Gi = sn * gw;
        const float rinv2 = rinv * rinv;
        const float qq = dnx * dny * rinv2;
        const float a = fmaf(fmaf(rho, rho, -3.0f), qq, nxny);
        const float b = rho * fmaf(3.0f, qq, -nxny);
        const float lr = fmaf(-b, kinv, dny);
        const float li = fmaf(a, kinv, -rho * dny);
        const float Hr = Gr * rinv2, Hi = Gi * rinv2;
        Lr = fmaf(Hr, lr, fmaf(-Hi, li, Lr));
        Li = fmaf(Hr, li, fmaf(Hi, lr, Li));
        const float t1 = fmaf(-dnx, rinv, 1.0f);
        const float t2 = -dnx * rinv2 * kinv;
        Rr = fmaf(Gr, t1, fmaf(-Gi, t2, Rr));
        Ri = fmaf(Gr, t2, fmaf(Gi, t1, Ri));
      }
      __stcs(L + off, make_float2(-Lr, -Li));
      __stcs(R + off, make_float2(-Rr, -Ri));
      if (Lb) __stcs(Lb + off, pack_bf16(-Lr, -Li));
    }
  }
}

// ---------------------------------------------------- regular pairs, paired FP32 (f32x2)
// The same arithmetic as k_assemble_regular for two adjacent source columns per thread, with
// the FP32 operations issued as sm_100 paired instructions (add/sub/mul/fma .rn.f32x2): one
// instruction does the operation for both columns. The kernel is issue-bound, so this halves
// the cost of everything except the MUFU operations (rsqrt, sin, cos), which stay scalar.
namespace {
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 bc(float x) { return pk(x, x); }
constexpr int kX2Threads = 128;  // 256 source columns per block, two per thread
}  // namespace

// Four blocks per SM (128 registers, no spills): 1.192 ms against 1.222 ms at three blocks (164
// registers) on the 10240-triangle operator; five blocks spill and took 1.283 ms.
__global__ void __launch_bounds__(kX2Threads, 4)
k_assemble_regular_x2(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo,
                      const float4* __restrict__ nrm, const float4* __restrict__ qp,
                      const int4* __restrict__ vid, int n, int ld, int rows_per_block, float k,
                      float2* __restrict__ L, float2* __restrict__ R, uint32_t* __restrict__ Lb) {
  __shared__ float4 s_hi[kRowStage], s_lo[kRowStage], s_n[kRowStage];
  __shared__ int4 s_v[kRowStage];
  const int j0 = (blockIdx.x * kX2Threads + threadIdx.x) * 2;  // columns j0, j0 + 1
  const bool ok0 = j0 < n, ok1 = j0 + 1 < n;
  const bool pad0 = !ok0 && j0 < ld, pad1 = !ok1 && j0 + 1 < ld;
  // column records as pairs (column j0 in the low half, j0 + 1 in the high half)
  u64 chx, chy, chz, clx, cly, clz, njx, njy, njz, qx[7], qy[7], qz[7], qw[7];
  int4 v0 = make_int4(-1, -1, -1, 0), v1 = v0;
  {
    const int ja = ok0 ? j0 : 0, jb = ok1 ? j0 + 1 : ja;
    const float4 a = c_hi[ja], b = c_hi[jb];
    chx = pk(a.x, b.x), chy = pk(a.y, b.y), chz = pk(a.z, b.z);
    const float4 al = c_lo[ja], bl = c_lo[jb];
    clx = pk(al.x, bl.x), cly = pk(al.y, bl.y), clz = pk(al.z, bl.z);
    const float4 an = nrm[ja], bn = nrm[jb];
    njx = pk(an.x, bn.x), njy = pk(an.y, bn.y), njz = pk(an.z, bn.z);
#pragma unroll
    for (int p = 0; p < 7; ++p) {
      const float4 qa = qp[7 * ja + p], qb = qp[7 * jb + p];
      qx[p] = pk(qa.x, qb.x), qy[p] = pk(qa.y, qb.y), qz[p] = pk(qa.z, qb.z), qw[p] = pk(qa.w, qb.w);
    }
    if (ok0) v0 = vid[j0];
    if (ok1) v1 = vid[j0 + 1];
  }
  const float kinv = 1.0f / k;
  const u64 k2 = bc(k), kinv2 = bc(kinv), mkinv2 = bc(-kinv), inv2pi2 = bc(kInvTwoPi);
  const u64 m2pihi = bc(-kTwoPiHi), m2pilo = bc(-kTwoPiLo), one2 = bc(1.0f), m3 = bc(-3.0f), three2 = bc(3.0f);
  const int i_begin = blockIdx.y * rows_per_block;
  const int i_end = min(n, i_begin + rows_per_block);
  for (int ib = i_begin; ib < i_end; ib += kRowStage) {
    const int cnt = min(kRowStage, i_end - ib);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const int i = ib + threadIdx.x;
      s_hi[threadIdx.x] = c_hi[i];
      s_lo[threadIdx.x] = c_lo[i];
      s_n[threadIdx.x] = nrm[i];
      s_v[threadIdx.x] = vid[i];
    }
    __syncthreads();
    for (int t = 0; t < cnt; ++t) {
      const int i = ib + t;
      const size_t off = (size_t)i * ld + j0;
      if (pad0 || pad1) {  // zero the padding columns (ld > n)
        if (pad0) {
          L[off] = make_float2(0.f, 0.f);
          R[off] = make_float2(0.f, 0.f);
          if (Lb) Lb[off] = 0u;
        }
        if (pad1) {
          L[off + 1] = make_float2(0.f, 0.f);
          R[off + 1] = make_float2(0.f, 0.f);
          if (Lb) Lb[off + 1] = 0u;
        }
      }
      if (!ok0) continue;
      const int4 vi = s_v[t];
      const bool w0 = !shares_vertex(vi, v0), w1 = ok1 && !shares_vertex(vi, v1);
      if (!w0 && !w1) continue;
      const float4 xh = s_hi[t], xl = s_lo[t], ni = s_n[t];
      const u64 nix = bc(ni.x), niy = bc(ni.y), niz = bc(ni.z);
      const u64 Dx = add2(sub2(bc(xh.x), chx), sub2(bc(xl.x), clx));
      const u64 Dy = add2(sub2(bc(xh.y), chy), sub2(bc(xl.y), cly));
      const u64 Dz = add2(sub2(bc(xh.z), chz), sub2(bc(xl.z), clz));
      const u64 dny = fma2(Dx, njx, fma2(Dy, njy, mul2(Dz, njz)));
      const u64 Dni = fma2(Dx, nix, fma2(Dy, niy, mul2(Dz, niz)));
      const u64 nxny = fma2(nix, njx, fma2(niy, njy, mul2(niz, njz)));
      const u64 mnxny = sub2(bc(0.f), nxny);
      u64 Lr = bc(0.f), Li = Lr, Rr = Lr, Ri = Lr;
#pragma unroll
      for (int p = 0; p < 7; ++p) {
        const u64 dx = sub2(Dx, qx[p]), dy = sub2(Dy, qy[p]), dz = sub2(Dz, qz[p]);
        const u64 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float r2a, r2b;
        upk(r2, r2a, r2b);
        const u64 rinv = pk(rsqrtf(r2a), rsqrtf(r2b));
        const u64 r = mul2(r2, rinv);
        const u64 dnx = sub2(Dni, fma2(qx[p], nix, fma2(qy[p], niy, mul2(qz[p], niz))));
        const u64 rho = mul2(k2, r);
        float ua, ub;
        upk(mul2(rho, inv2pi2), ua, ub);
        const u64 nq = pk(rintf(ua), rintf(ub));
        const u64 th = fma2(nq, m2pilo, fma2(nq, m2pihi, rho));
        float tha, thb, sa, ca, sb, cb;
        upk(th, tha, thb);
        __sincosf(tha, &sa, &ca);
        __sincosf(thb, &sb, &cb);
        const u64 gw = mul2(rinv, qw[p]);
        const u64 Gr = mul2(pk(ca, cb), gw), Gi = mul2(pk(sa, sb), gw);
        const u64 ri2 = mul2(rinv, rinv);
        const u64 qq = mul2(mul2(dnx, dny), ri2);
        const u64 a = fma2(fma2(rho, rho, m3), qq, nxny);
        const u64 b = mul2(rho, fma2(three2, qq, mnxny));
        const u64 lr = fma2(b, mkinv2, dny);                 // dny - b/k
        const u64 nli = fma2(a, mkinv2, mul2(rho, dny));     // -(a/k - rho dny)
        const u64 Hr = mul2(Gr, ri2), Hi = mul2(Gi, ri2);
        Lr = fma2(Hr, lr, fma2(Hi, nli, Lr));                // += Hr lr - Hi li
        Li = sub2(fma2(Hi, lr, Li), mul2(Hr, nli));          // += Hr li + Hi lr
        const u64 t1 = sub2(one2, mul2(dnx, rinv));          // 1 - dnx/r
        const u64 nt2 = mul2(mul2(dnx, ri2), kinv2);         // -t2 = dnx/(k r^2)
        Rr = fma2(Gr, t1, fma2(Gi, nt2, Rr));                // += Gr t1 - Gi t2
        Ri = sub2(fma2(Gi, t1, Ri), mul2(Gr, nt2));          // += Gr t2 + Gi t1
      }
      float lr0, lr1, li0, li1, rr0, rr1, ri0, ri1;
      upk(Lr, lr0, lr1);
      upk(Li, li0, li1);
      upk(Rr, rr0, rr1);
      upk(Ri, ri0, ri1);
      if (w0 && w1) {
        __stcs(reinterpret_cast<float4*>(L + off), make_float4(-lr0, -li0, -lr1, -li1));
        __stcs(reinterpret_cast<float4*>(R + off), make_float4(-rr0, -ri0, -rr1, -ri1));
        if (Lb) __stcs(reinterpret_cast<uint2*>(Lb + off), make_uint2(pack_bf16(-lr0, -li0), pack_bf16(-lr1, -li1)));
      } else {
        if (w0) {
          __stcs(L + off, make_float2(-lr0, -li0));
          __stcs(R + off, make_float2(-rr0, -ri0));
          if (Lb) __stcs(Lb + off, pack_bf16(-lr0, -li0));
        }
        if (w1) {
          __stcs(L + off + 1, make_float2(-lr1, -li1));
          __stcs(R + off + 1, make_float2(-rr1, -ri1));
          if (Lb) __stcs(Lb + off + 1, pack_bf16(-lr1, -li1));
        }
      }
    }
  }
}

// ------------------------------------------------------------- near pairs and self terms
namespace {

// Compensated FP32 running sum (Kahan 1965): s - c is the exact sum to about twice FP32 precision.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Sum over the 16 lanes of a half warp of the compensated sums (s, c), as a double-float
// (hi, lo); every lane of the warp must call it.
__device__ __forceinline__ void half_warp_sum_df(float s, float c, float& hi, float& lo) {
  two_sum(s, -c, hi, lo);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float t, e;
    two_sum(hi, h2, t, e);
    e += lo + l2;
    hi = t + e;
    lo = e - (hi - t);
  }
}

}  // namespace

// D - (a e + b f) for float-float D, e, f and barycentrics a = (ab.x, ab.y), b = (ab.z, ab.w):
// error-free products and sums (Dekker, Knuth) in round-to-nearest FP32 intrinsics (never
// contracted), rounded to FP32 once at the end.
__device__ __forceinline__ float ff_offset(float Dh, float Dl, float4 ab, float eh, float el, float fh, float fl) {
  const float p = __fmul_rn(ab.x, eh);
  const float pe = __fmaf_rn(ab.x, el, __fmaf_rn(ab.y, eh, __fmaf_rn(ab.x, eh, -p)));
  const float q = __fmul_rn(ab.z, fh);
  const float qe = __fmaf_rn(ab.z, fl, __fmaf_rn(ab.w, fh, __fmaf_rn(ab.z, fh, -q)));
  const float s = __fadd_rn(p, q);
  const float sb = __fsub_rn(s, p);
  const float se = __fadd_rn(__fadd_rn(__fsub_rn(p, __fsub_rn(s, sb)), __fsub_rn(q, sb)), __fadd_rn(pe, qe));
  const float d = __fsub_rn(Dh, s);
  const float db = __fsub_rn(d, Dh);
  const float de = __fadd_rn(__fsub_rn(Dh, __fsub_rn(d, db)), __fsub_rn(-s, db));
  return __fadd_rn(d, __fadd_rn(de, __fsub_rn(Dl, se)));
}

// Vertex-sharing pairs (i, j != i): the 7-point rule on the 4^levels sub-triangles of element j,
// 16 lanes per pair (two pairs per warp; 112 points at levels = 2 is seven per lane). The
// quadrature point and x_i are close compared with their distance from the origin, so
// d = x_i - y is formed from x_i - v0 and the edges of j (taken in FP64 from the FP64 vertices,
// once per pair) in float-float arithmetic (ff_offset, about 48 bits); d is then exact to FP32
// rounding. The normal components d.n_i and d.n_j come from per-pair FP64 dot products (they
// cancel for nearly coplanar neighbours). Everything after that (r, the phase, G and the
// hypersingular combination) runs on the FP32 pipe, which GB300 issues ~60x faster than FP64.
// Per-lane sums are compensated (Kahan) and the 16 lanes are added as double-float.
__global__ void __launch_bounds__(256)
k_assemble_adjacent(const int2* __restrict__ pairs, int64_t n_pairs, const double* __restrict__ tri,
                    const double* __restrict__ cen, const double* __restrict__ nrm64,
                    const double* __restrict__ area, int ld, float kf, float kinvf, float2* __restrict__ L,
                    float2* __restrict__ R, uint32_t* __restrict__ Lb) {
  const int64_t pr_idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  const bool valid = pr_idx < n_pairs;  // no early exit: the lane sums use full-warp shuffles
  int i = 0, j = 0;
  if (valid) {
    const int2 pr = pairs[pr_idx];
    i = pr.x;
    j = pr.y;
  }
  const double* t = tri + 9 * j;
  // D = x_i - v0 and the edges e1 = v1 - v0, e2 = v2 - v0 of triangle j as float-float pairs:
  // d = D - (l1 e1 + l2 e2) then keeps about 48 bits on the FP32 pipe (GB300's FP64 rate is
  // about 1/76 of its FP32 rate; this kernel was FP64-pipe-bound). The FP64 prologue is dealt
  // over the pair's 16 lanes (lane c < 9: component c % 3 of D, e1 or e2; lanes 9-14: the two
  // normals; lane 15: the area factor) and broadcast by shuffles.
  float vh = 0.f, vl = 0.f;
  double pi = 0.0, pj = 0.0;  // lanes 0..8: component c of D, e1 or e2 times n_i,c and n_j,c
  if (l16 < 9) {
    const int w = l16 / 3, c = l16 % 3;
    const double v = (w == 0 ? cen[3 * i + c] : t[3 * w + c]) - t[c];
    vh = (float)v;
    vl = (float)(v - (double)vh);
    pi = v * nrm64[3 * i + c];
    pj = v * nrm64[3 * j + c];
  } else if (l16 < 12) {
    vh = (float)nrm64[3 * i + (l16 - 9)];
  } else if (l16 < 15) {
    vh = (float)nrm64[3 * j + (l16 - 12)];
  } else {
    vh = (float)(area[j] * (0.25 / 3.14159265358979323846));
  }
  float Dh[3], Dl[3], e1h[3], e1l[3], e2h[3], e2l[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Dh[c] = __shfl_sync(0xffffffffu, vh, c, 16);
    Dl[c] = __shfl_sync(0xffffffffu, vl, c, 16);
    e1h[c] = __shfl_sync(0xffffffffu, vh, 3 + c, 16);
    e1l[c] = __shfl_sync(0xffffffffu, vl, 3 + c, 16);
    e2h[c] = __shfl_sync(0xffffffffu, vh, 6 + c, 16);
    e2l[c] = __shfl_sync(0xffffffffu, vl, 6 + c, 16);
  }
  const float ni0 = __shfl_sync(0xffffffffu, vh, 9, 16), ni1 = __shfl_sync(0xffffffffu, vh, 10, 16),
              ni2 = __shfl_sync(0xffffffffu, vh, 11, 16);
  const float nj0 = __shfl_sync(0xffffffffu, vh, 12, 16), nj1 = __shfl_sync(0xffffffffu, vh, 13, 16),
              nj2 = __shfl_sync(0xffffffffu, vh, 14, 16);
  const float scale = __shfl_sync(0xffffffffu, vh, 15, 16);
  // d.n_i and d.n_j are O(theta |d|) for nearly coplanar neighbours (theta the angle between
  // them): as FP32 dot products with FP32-rounded normals they carry an absolute error of about
  // 6e-8 |d|, which at low k (beta = i/k weights d.n_i in R) reached 2e-6 of an entry. So the
  // pair's D.n_i, e1.n_i, e2.n_i and D.n_j are FP64 dot products with the FP64 normals (summed
  // over the three lanes of each vector), and per point d.n_i = D.n_i - a e1.n_i - b e2.n_i has
  // no cancellation; d.n_j = D.n_j on the whole flat element j (its edges are normal to n_j).
  const int g3 = (l16 / 3) * 3;  // first lane of this lane's vector (lanes 9..15: unused values)
  const double si = __shfl_sync(0xffffffffu, pi, g3, 16) + __shfl_sync(0xffffffffu, pi, g3 + 1, 16) +
                    __shfl_sync(0xffffffffu, pi, g3 + 2, 16);
  const double sj = __shfl_sync(0xffffffffu, pj, g3, 16) + __shfl_sync(0xffffffffu, pj, g3 + 1, 16) +
                    __shfl_sync(0xffffffffu, pj, g3 + 2, 16);
  const float fi = (float)si, fj = (float)sj;
  const float Dni = __shfl_sync(0xffffffffu, fi, 0, 16), E1i = __shfl_sync(0xffffffffu, fi, 3, 16),
              E2i = __shfl_sync(0xffffffffu, fi, 6, 16);
  const float dny = __shfl_sync(0xffffffffu, fj, 0, 16);
  const float nxny = ni0 * nj0 + ni1 * nj1 + ni2 * nj2;
  float Lr = 0.f, Li = 0.f, Rr = 0.f, Ri = 0.f, cLr = 0.f, cLi = 0.f, cRr = 0.f, cRi = 0.f;
  const int np = valid ? c_adj_npts : 0;
  for (int p = l16; p < np; p += 16) {
    const float4 ab = g_adj_ab[p];
    const float d0 = ff_offset(Dh[0], Dl[0], ab, e1h[0], e1l[0], e2h[0], e2l[0]);
    const float d1 = ff_offset(Dh[1], Dl[1], ab, e1h[1], e1l[1], e2h[1], e2l[1]);
    const float d2 = ff_offset(Dh[2], Dl[2], ab, e1h[2], e1l[2], e2h[2], e2l[2]);
    const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float dnx = fmaf(-ab.x, E1i, fmaf(-ab.z, E2i, Dni));
    const float rho = kf * r;
    const float nq = rintf(rho * kInvTwoPi);
    const float th = fmaf(-nq, kTwoPiLo, fmaf(-nq, kTwoPiHi, rho));
    float sn, cs;
    sincosf(th, &sn, &cs);
    const float gw = g_adj_w[p] * scale * rinv;
    const float Gr = cs * gw, Gi = sn * gw;
    const float rinv2 = rinv * rinv;
    const float qq = dnx * dny * rinv2;
    const float a = fmaf(fmaf(rho, rho, -3.0f), qq, nxny);
    const float b = rho * fmaf(3.0f, qq, -nxny);
    const float lr = fmaf(-b, kinvf, dny), li = fmaf(a, kinvf, -rho * dny);
    const float Hr = Gr * rinv2, Hi = Gi * rinv2;
    const float t1 = fmaf(-dnx, rinv, 1.0f), t2 = -dnx * rinv2 * kinvf;
    kahan_add(Lr, cLr, fmaf(Hr, lr, -Hi * li));
    kahan_add(Li, cLi, fmaf(Hr, li, Hi * lr));
    kahan_add(Rr, cRr, fmaf(Gr, t1, -Gi * t2));
    kahan_add(Ri, cRi, fmaf(Gr, t2, Gi * t1));
  }
  float hLr, lLr, hLi, lLi, hRr, lRr, hRi, lRi;
  half_warp_sum_df(Lr, cLr, hLr, lLr);
  half_warp_sum_df(Li, cLi, hLi, lLi);
  half_warp_sum_df(Rr, cRr, hRr, lRr);
  half_warp_sum_df(Ri, cRi, hRi, lRi);
  if (valid && l16 == 0) {
    const float2 lv = make_float2(-(hLr + lLr), -(hLi + lLi));
    const float2 rv = make_float2(-(hRr + lRr), -(hRi + lRi));
    L[(size_t)i * ld + j] = lv;
    R[(size_t)i * ld + j] = rv;
    if (Lb) Lb[(size_t)i * ld + j] = pack_bf16(lv.x, lv.y);
  }
}

// Self terms (flat element, collocation at the centroid), one warp per element (the vertices
// relative to the centroid in FP64, everything after them in FP32):
//   S = (1/4pi) sum_e int (e^{ikR} - 1)/(ik) dpsi,   FP = (1/4pi) sum_e int (ik - e^{ikR}/R) dpsi,
// with R = d_e / cos(psi) the distance from the centroid to edge e along the ray (radial part
// analytic, Hadamard finite part of the hypersingular term); L_ii = 1/2 - beta FP and
// R_ii = -S - beta/2 with beta = i/k.
__global__ void __launch_bounds__(256)
k_assemble_self(int n, const double* __restrict__ tri, const double* __restrict__ cen, int ld,
                float kf, float kinvf, float2* __restrict__ L, float2* __restrict__ R, uint32_t* __restrict__ Lb) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // whole warps
  const float inv4pi = (float)(0.25 / 3.14159265358979323846);
  const double* t = tri + 9 * i;
  const int ns = c_self_pts;
  // per edge e (lanes 0..2): the distance d_e from the centroid to the edge line and the
  // angles of the edge's end points seen from the centroid, measured from the perpendicular.
  // The end points relative to the centroid are formed in FP64 (the coordinates are far larger
  // than the element) and the rest in FP32 on those element-sized vectors.
  float de = 0.f, mid = 0.f, half = 0.f;
  if (lane < 3) {
    const double* P = t + 3 * lane;
    const double* Q = t + 3 * ((lane + 1) % 3);
    float p[3], q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double xc = cen[3 * i + c];
      p[c] = (float)(P[c] - xc);
      q[c] = (float)(Q[c] - xc);
    }
    float u0 = q[0] - p[0], u1 = q[1] - p[1], u2 = q[2] - p[2];
    const float ul = rsqrtf(fmaf(u0, u0, fmaf(u1, u1, u2 * u2)));
    u0 *= ul;
    u1 *= ul;
    u2 *= ul;
    // positions of P and Q along the edge line, relative to the foot of the perpendicular
    const float sP = fmaf(p[0], u0, fmaf(p[1], u1, p[2] * u2));
    const float sQ = fmaf(q[0], u0, fmaf(q[1], u1, q[2] * u2));
    const float f0 = fmaf(-sP, u0, p[0]), f1 = fmaf(-sP, u1, p[1]), f2 = fmaf(-sP, u2, p[2]);
    de = sqrtf(fmaf(f0, f0, fmaf(f1, f1, f2 * f2)));
    const float psiP = atan2f(sP, de), psiQ = atan2f(sQ, de);
    half = 0.5f * (psiQ - psiP);
    mid = 0.5f * (psiQ + psiP);
  }
  float dEf[3], mEf[3], hEf[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    dEf[e] = __shfl_sync(0xffffffffu, de, e);
    mEf[e] = __shfl_sync(0xffffffffu, mid, e);
    hEf[e] = __shfl_sync(0xffffffffu, half, e);
  }
  // The angular points in FP32 (GB300's FP64 rate is about 1/76 of its FP32 rate), with
  // cancellation-free forms: with x = kR and h = x/2, (e^{ikR} - 1)/(ik) = (sin x + 2i sin^2 h)/k,
  // cos x = cos^2 h - sin^2 h, and k - sin(kR)/R = k (1 - sinc x) from its Taylor series
  // sum_{n>=1} (-1)^(n+1) x^(2n) / (2n+1)! below x = 1.5 (six terms: below 2e-8 of the value)
  // and 1 - sin(x)/x above (where 1 - sinc x >= 0.33).
  float Sre = 0.f, Sim = 0.f, Fre = 0.f, Fim = 0.f;
  for (int p = lane; p < 3 * ns; p += 32) {
    const int e = p / ns, g = p - e * ns;
    const float dE = e == 0 ? dEf[0] : (e == 1 ? dEf[1] : dEf[2]);
    const float mE = e == 0 ? mEf[0] : (e == 1 ? mEf[1] : mEf[2]);
    const float hE = e == 0 ? hEf[0] : (e == 1 ? hEf[1] : hEf[2]);
    const float2 gl = g_glf[g];
    const float psi = fmaf(hE, gl.x, mE);
    const float cpsi = cosf(psi);
    const float Rr = dE / cpsi;
    const float invR = cpsi / dE;
    const float wq = hE * gl.y;
    const float x = kf * Rr;
    float s2, c2;
    sincosf(0.5f * x, &s2, &c2);
    const float sn = 2.0f * s2 * c2, omc = 2.0f * s2 * s2, cs = (c2 - s2) * (c2 + s2);
    float omsinc;  // 1 - sin(x)/x
    if (x < 1.5f) {
      const float x2 = x * x;
      omsinc = x2 * (1.0f / 6.0f -
                     x2 * (1.0f / 120.0f -
                           x2 * (1.0f / 5040.0f -
                                 x2 * (1.0f / 362880.0f - x2 * (1.0f / 39916800.0f - x2 * (1.0f / 6227020800.0f))))));
    } else {
      omsinc = 1.0f - sn / x;
    }
    Sre = fmaf(wq, sn * kinvf, Sre);
    Sim = fmaf(wq, omc * kinvf, Sim);
    Fre = fmaf(-wq, cs * invR, Fre);
    Fim = fmaf(wq, kf * omsinc, Fim);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Sre += __shfl_xor_sync(0xffffffffu, Sre, o);
    Sim += __shfl_xor_sync(0xffffffffu, Sim, o);
    Fre += __shfl_xor_sync(0xffffffffu, Fre, o);
    Fim += __shfl_xor_sync(0xffffffffu, Fim, o);
  }
  Sre *= inv4pi;
  Sim *= inv4pi;
  Fre *= inv4pi;
  Fim *= inv4pi;
  if (lane == 0) {
    const float2 lv = make_float2(fmaf(Fim, kinvf, 0.5f), -Fre * kinvf);
    L[(size_t)i * ld + i] = lv;
    R[(size_t)i * ld + i] = make_float2(-Sre, fmaf(-0.5f, kinvf, -Sim));
    if (Lb) Lb[(size_t)i * ld + i] = pack_bf16(lv.x, lv.y);
  }
}

// ----------------------------------------------------------------------- drivers
nat_bem_status geometry_build(nat_bem_op* op, const double* dV, const int32_t* dT, int64_t nv,
                              const std::vector<int2>& near_pairs, cudaStream_t s) {
  Geometry& g = op->geo;
  const int64_t n = g.n;  // elements
  (void)nv;
  NB_TRY(dev_alloc_n(&g.c_hi, n, s));
  NB_TRY(dev_alloc_n(&g.c_lo, n, s));
  NB_TRY(dev_alloc_n(&g.nrm, n, s));
  NB_TRY(dev_alloc_n(&g.qp, 7 * n, s));
  NB_TRY(dev_alloc_n(&g.vid, n, s));
  NB_TRY(dev_alloc_n(&g.tri, 9 * n, s));
  NB_TRY(dev_alloc_n(&g.cen, 3 * n, s));
  NB_TRY(dev_alloc_n(&g.nrm64, 3 * n, s));
  NB_TRY(dev_alloc_n(&g.area, n, s));
  g.n_near = (int64_t)near_pairs.size();
  NB_TRY(dev_alloc_n(&g.near_pairs, g.n_near, s));
  NB_TRY_CUDA(cudaMemcpyAsync(g.near_pairs, near_pairs.data(), g.n_near * sizeof(int2),
                              cudaMemcpyHostToDevice, s));
  const int threads = 128;
  NB_LAUNCH("geometry", s, k_geometry<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
      dV, dT, (int)n, g.c_hi, g.c_lo, g.nrm, g.qp, g.vid, g.tri, g.cen, g.nrm64, g.area));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

nat_bem_status assemble_operators(nat_bem_op* op, cudaStream_t s) {
  const Geometry& g = op->geo;
  const int n = (int)op->n, ld = (int)g.ld;
  // The near pairs write exactly the entries the regular kernel skips. The three kernels run in
  // order on the solve's stream: beside the FP32 regular kernel on a second stream the FP64
  // kernels saved ~0.3 ms per solve with one solve in flight and nothing with several, and
  // they slowed the regular kernel they shared the SMs with.
  {
    const int64_t threads = 256;
    const int64_t adj_blocks = (g.n_near * 16 + threads - 1) / threads;
    if (adj_blocks > 0)
      NB_LAUNCH("assemble_near", s, k_assemble_adjacent<<<(unsigned)adj_blocks, (unsigned)threads, 0, s>>>(
          g.near_pairs, g.n_near, g.tri, g.cen, g.nrm64, g.area, ld, (float)op->k, (float)(1.0 / op->k), op->L,
          op->R, bf16_target(op)));
    const int64_t self_blocks = ((int64_t)n * 32 + threads - 1) / threads;
    NB_LAUNCH("assemble_self", s, k_assemble_self<<<(unsigned)self_blocks, (unsigned)threads, 0, s>>>(
        n, g.tri, g.cen, ld, (float)op->k, (float)(1.0 / op->k), op->L, op->R, bf16_target(op)));
    NB_CHECK_LAUNCH();
  }
  // regular pairs: columns in blocks of 256 (two columns a thread in the paired form), rows
  // split in blocks of rows_per_block. Every entry is computed the same way whatever the split,
  // so the autotuner (rows per block 64, 32, 128 or 16, per size class) changes no result.
  const int col_blocks = (ld + kRegThreads - 1) / kRegThreads;
  static const bool scalar = std::getenv("NATBEM_ASSEMBLY_SCALAR") != nullptr;
  auto launch = [&](int rows_per_block) -> nat_bem_status {
    const int row_blocks = (n + rows_per_block - 1) / rows_per_block;
    dim3 grid(col_blocks, row_blocks);
    if (scalar)
      NB_LAUNCH("assemble_regular", s, k_assemble_regular<<<grid, kRegThreads, 0, s>>>(
          g.c_hi, g.c_lo, g.nrm, g.qp, g.vid, n, ld, rows_per_block, (float)op->k, op->L, op->R, bf16_target(op)));
    else
      NB_LAUNCH("assemble_regular", s, k_assemble_regular_x2<<<grid, kX2Threads, 0, s>>>(
          g.c_hi, g.c_lo, g.nrm, g.qp, g.vid, n, ld, rows_per_block, (float)op->k, op->L, op->R, bf16_target(op)));
    NB_CHECK_LAUNCH();
    return NAT_BEM_OK;
  };
  static const int kRows[4] = {64, 32, 128, 16};
  const int pick = autotune("assemble_rows", (n + 1023) / 1024, 4, [&](int c) { return launch(kRows[c]); }, s);
  NB_TRY(launch(kRows[pick]));
  return finish_low_copy(op, s);
}

// The row-scaled FP16 copy of L: one block per row finds the row's largest real or imaginary
// magnitude m = f 2^E (f in [0.5, 1)), takes s = 2^(15 - E) so that the scaled entries stay
// below 2^15 (FP16's largest finite value is 65504) and keep FP16's full 11 significant bits
// down to 2^-29 of m, writes half2(L_ij s) rounded to nearest, and 1/s (exact) as the row scale.
__global__ void __launch_bounds__(256) k_copy_fp16_rows(const float2* __restrict__ L, int ld,
                                                        uint32_t* __restrict__ Lh, float* __restrict__ row_scale) {
  __shared__ float red[8];
  const size_t row = blockIdx.x;
  const float2* src = L + row * ld;
  float m = 0.f;
  for (int j = threadIdx.x; j < ld; j += 256) {
    const float2 v = src[j];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);
  const float scale = m > 0.f ? ldexpf(1.0f, 15 - e) : 1.0f;
  for (int j = threadIdx.x; j < ld; j += 256) {
    const float2 v = src[j];
    __half2 h = __floats2half2_rn(v.x * scale, v.y * scale);
    Lh[row * ld + j] = *reinterpret_cast<uint32_t*>(&h);
  }
  if (threadIdx.x == 0) row_scale[row] = m > 0.f ? ldexpf(1.0f, e - 15) : 1.0f;
}

nat_bem_status finish_low_copy(nat_bem_op* op, cudaStream_t s) {
  op->split_ok = false;  // L changed: its three-way split is rebuilt before the next use
  if (!op->copy_fp16 || !op->Lb) return NAT_BEM_OK;
  NB_LAUNCH("copy_fp16", s, k_copy_fp16_rows<<<(unsigned)op->n, 256, 0, s>>>(op->L, (int)op->geo.ld, op->Lb,
                                                                              op->row_scale));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

}  // namespace natbem
