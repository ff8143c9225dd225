// Monte-Carlo BEM (paper Sec. 4.1.1 and 4.2): the conventional boundary integral equation
// (beta = 0 in Eq. 6) with the surface integral replaced by a Monte-Carlo sum over M sample
// points y_j of uniform density on the surface (1/q = |Gamma|), collocated at the samples:
//
//   1/2 p_i = sum_{j != i} w [ dG/dn_y(y_i, y_j) p_j - G(y_i, y_j) g_j ] - (eps/2) g_i,
//
// w = |Gamma| / M and pi eps^2 = |Gamma| / M: the sample's own disk of radius eps contributes
// (eps/2) g_i through the single layer (one sample at its centre, Sec. 4.2) and nothing through
// the double layer (d is perpendicular to the normal on the flat disk). In the L p = R g form
// the solver, the mixed precision, the batching and the serving paths use unchanged:
//
//   L_ij = 1/2 delta_ij - w dG/dn_y(y_i, y_j) (1 - delta_ij)
//   R_ij = -w G(y_i, y_j) (1 - delta_ij) - (eps/2) delta_ij
//
// dG/dn_y = G (1 - i k r) (d . n_y) / r^2 with d = y_i - y_j. One thread per source column, the
// collocation samples staged through shared memory, FP32 with the sample positions as float
// hi/lo pairs (d keeps FP32 relative accuracy for close samples), Cody-Waite phase reduction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace natbem {

namespace {
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.7484555314695172e-7f;
constexpr float kInvTwoPi = 0.159154943091895336f;
constexpr float kInvFourPi = 0.0795774715459476679f;
constexpr int kMcThreads = 256;  // source columns per block
constexpr int kMcStage = 64;     // collocation samples staged at a time

__device__ __forceinline__ uint32_t pack_bf16(float re, float im) {
  __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
  return *reinterpret_cast<uint32_t*>(&v);
}
}  // namespace

// Sample records: position as a float hi/lo pair, unit normal, and the one-point "rule" of the
// field evaluation (offset 0, weight w / (4 pi)).
__global__ void k_mc_geometry(const double* __restrict__ Y, const double* __restrict__ N, int m,
                              float w, float4* __restrict__ c_hi, float4* __restrict__ c_lo,
                              float4* __restrict__ nrm, float4* __restrict__ qp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  float h[3], l[3];
  for (int d = 0; d < 3; ++d) {
    const double v = Y[3 * (size_t)j + d];
    h[d] = (float)v;
    l[d] = (float)(v - (double)h[d]);
  }
  c_hi[j] = make_float4(h[0], h[1], h[2], 0.f);
  c_lo[j] = make_float4(l[0], l[1], l[2], 0.f);
  nrm[j] = make_float4((float)N[3 * (size_t)j], (float)N[3 * (size_t)j + 1], (float)N[3 * (size_t)j + 2], 0.f);
  qp[j] = make_float4(0.f, 0.f, 0.f, w * kInvFourPi);
}

__global__ void __launch_bounds__(kMcThreads)
k_mc_assemble(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo,
              const float4* __restrict__ nrm, int m, int ld, int rows_per_block, float k, float w,
              float eps, float2* __restrict__ L, float2* __restrict__ R, uint32_t* __restrict__ Lb) {
  __shared__ float4 s_hi[kMcStage], s_lo[kMcStage];
  const int j = blockIdx.x * kMcThreads + threadIdx.x;
  const bool col_ok = j < m, col_pad = j >= m && j < ld;
  float3 chi = make_float3(0.f, 0.f, 0.f), clo = chi, nj = chi;
  if (col_ok) {
    float4 t = c_hi[j];
    chi = make_float3(t.x, t.y, t.z);
    t = c_lo[j];
    clo = make_float3(t.x, t.y, t.z);
    t = nrm[j];
    nj = make_float3(t.x, t.y, t.z);
  }
  const float wg = w * kInvFourPi;
  const int i_begin = blockIdx.y * rows_per_block;
  const int i_end = min(m, i_begin + rows_per_block);
  for (int ib = i_begin; ib < i_end; ib += kMcStage) {
    const int cnt = min(kMcStage, i_end - ib);
    __syncthreads();
    if (threadIdx.x < cnt) {
      s_hi[threadIdx.x] = c_hi[ib + threadIdx.x];
      s_lo[threadIdx.x] = c_lo[ib + threadIdx.x];
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
      float2 lv, rv;
      if (i == j) {
        lv = make_float2(0.5f, 0.f);
        rv = make_float2(-0.5f * eps, 0.f);
      } else {
        const float4 xh = s_hi[t], xl = s_lo[t];
        const float dx = (xh.x - chi.x) + (xl.x - clo.x);
        const float dy = (xh.y - chi.y) + (xl.y - clo.y);
        const float dz = (xh.z - chi.z) + (xl.z - clo.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float rho = k * (r2 * rinv);
        const float nq = rintf(rho * kInvTwoPi);
        float th = fmaf(-nq, kTwoPiHi, rho);
        th = fmaf(-nq, kTwoPiLo, th);
        float sn, cs;
        __sincosf(th, &sn, &cs);
        const float gw = rinv * wg;        // w / (4 pi r)
        const float Gr = cs * gw, Gi = sn * gw;
        const float f = (dx * nj.x + dy * nj.y + dz * nj.z) * rinv * rinv;  // (d . n_y) / r^2
        // w dG/dn_y = w G (1 - i rho) f
        const float Dr = f * fmaf(rho, Gi, Gr), Di = f * fmaf(-rho, Gr, Gi);
        lv = make_float2(-Dr, -Di);
        rv = make_float2(-Gr, -Gi);
      }
      __stcs(L + off, lv);
      __stcs(R + off, rv);
      if (Lb) __stcs(Lb + off, pack_bf16(lv.x, lv.y));
    }
  }
}

nat_bem_status mc_geometry_build(nat_bem_op* op, const double* dY, const double* dN, cudaStream_t s) {
  Geometry& g = op->geo;
  const int64_t m = op->n;
  NB_TRY(dev_alloc_n(&g.c_hi, m, s));
  NB_TRY(dev_alloc_n(&g.c_lo, m, s));
  NB_TRY(dev_alloc_n(&g.nrm, m, s));
  NB_TRY(dev_alloc_n(&g.qp, m, s));
  const int threads = 128;
  NB_LAUNCH("geometry", s, k_mc_geometry<<<(unsigned)((m + threads - 1) / threads), threads, 0, s>>>(
      dY, dN, (int)m, (float)(op->mc_area / (double)m), g.c_hi, g.c_lo, g.nrm, g.qp));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

nat_bem_status mc_assemble_operators(nat_bem_op* op, cudaStream_t s) {
  const Geometry& g = op->geo;
  const int m = (int)op->n, ld = (int)g.ld;
  const double w = op->mc_area / (double)m;
  const double eps = std::sqrt(op->mc_area / (3.14159265358979323846 * (double)m));
  const int rows_per_block = 64;
  dim3 grid((ld + kMcThreads - 1) / kMcThreads, (m + rows_per_block - 1) / rows_per_block);
  NB_LAUNCH("assemble_mc", s, k_mc_assemble<<<grid, kMcThreads, 0, s>>>(
      g.c_hi, g.c_lo, g.nrm, m, ld, rows_per_block, (float)op->k, (float)w, (float)eps, op->L, op->R, bf16_target(op)));
  NB_CHECK_LAUNCH();
  return finish_low_copy(op, s);
}

}  // namespace natbem
