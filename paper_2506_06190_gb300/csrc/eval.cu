// Field evaluation: the exterior representation p(x) = int [p dG/dn_y - G g] dS_y with the
// piecewise-constant surface data (pressure anywhere from the Neumann and Dirichlet data,
// paper Sec. 3.4; its surface limit is the first line of Sec. 4, Eq. 6). For a Monte-Carlo op
// (Sec. 4.1.1) the same sum runs over the samples with weight |Gamma| / M each, one point per
// sample. Otherwise the 7-point rule is applied on every element:
//
//   field(x_q) = sum_j [ p_j sum_p w_p A_j dG/dn_y(x_q, y_jp) - g_j sum_p w_p A_j G(x_q, y_jp) ]
//
// FP32 kernel generation, one thread per field point, elements split over blocks and staged in
// shared memory (broadcast reads); per-split FP64 partial sums are reduced in a fixed order.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace natbem {

namespace {
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.7484555314695172e-7f;
constexpr float kInvTwoPi = 0.159154943091895336f;
constexpr int kEvalThreads = 128;  // field points per block
constexpr int kElemStage = 32;     // elements staged per shared-memory round
constexpr int kMaxRhsPass = 16;    // far field: right-hand sides per pass (kernel values reused)
constexpr int kEvalRhsPass = 32;   // field: right-hand sides per pass
constexpr int kNoAllocRhsPass = 4; // the allocation-free path: passes of four (scratch sizing)
}  // namespace

template <int NR, int NQ>
__global__ void __launch_bounds__(kEvalThreads)
k_eval(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo,
       const float4* __restrict__ nrm, const float4* __restrict__ qp, int n,
       const double* __restrict__ pts, int m, float k, const float2* __restrict__ p,
       const float2* __restrict__ g, int rhs0, int nr, int elems_per_split, double2* __restrict__ part) {
  __shared__ float4 s_hi[kElemStage], s_lo[kElemStage], s_n[kElemStage];
  __shared__ float4 s_q[kElemStage * NQ];
  __shared__ float2 s_p[kElemStage * NR], s_g[kElemStage * NR];
  const int qi = blockIdx.x * kEvalThreads + threadIdx.x;
  const bool ok = qi < m;
  float xh[3] = {0.f, 0.f, 0.f}, xl[3] = {0.f, 0.f, 0.f};
  if (ok)
    for (int d = 0; d < 3; ++d) {
      const double v = pts[3 * (size_t)qi + d];
      xh[d] = (float)v;
      xl[d] = (float)(v - (double)xh[d]);
    }
  const int j_begin = blockIdx.y * elems_per_split;
  const int j_end = min(n, j_begin + elems_per_split);
  float accr[NR], acci[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) accr[s] = acci[s] = 0.f;
  for (int jb = j_begin; jb < j_end; jb += kElemStage) {
    const int cnt = min(kElemStage, j_end - jb);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt * NQ; t += kEvalThreads) s_q[t] = qp[NQ * (size_t)jb + t];
    if (threadIdx.x < cnt) {
      const int j = jb + threadIdx.x;
      s_hi[threadIdx.x] = c_hi[j];
      s_lo[threadIdx.x] = c_lo[j];
      s_n[threadIdx.x] = nrm[j];
#pragma unroll
      for (int s = 0; s < NR; ++s) {  // right-hand sides past nr read as zero
        s_p[threadIdx.x * NR + s] = s < nr ? p[(size_t)(rhs0 + s) * n + j] : make_float2(0.f, 0.f);
        s_g[threadIdx.x * NR + s] = s < nr ? g[(size_t)(rhs0 + s) * n + j] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    if (!ok) continue;
    for (int t = 0; t < cnt; ++t) {
      const float4 ch = s_hi[t], cl = s_lo[t], nj = s_n[t];
      const float Dx = (xh[0] - ch.x) + (xl[0] - cl.x);
      const float Dy = (xh[1] - ch.y) + (xl[1] - cl.y);
      const float Dz = (xh[2] - ch.z) + (xl[2] - cl.z);
      const float dny = Dx * nj.x + Dy * nj.y + Dz * nj.z;
      float Gr = 0.f, Gi = 0.f, Dr = 0.f, Di = 0.f;  // sums of w A G and w A dG/dn_y
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 o = s_q[NQ * t + q];
        const float dx = Dx - o.x, dy = Dy - o.y, dz = Dz - o.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float rho = k * (r2 * rinv);
        const float nq = rintf(rho * kInvTwoPi);
        float th = fmaf(-nq, kTwoPiHi, rho);
        th = fmaf(-nq, kTwoPiLo, th);
        float sn, cs;
        __sincosf(th, &sn, &cs);
        const float gw = rinv * o.w;
        const float er = cs * gw, ei = sn * gw;  // w A G
        Gr += er;
        Gi += ei;
        // dG/dn_y = G (1 - i rho) (d.n_y) / r^2
        const float f = dny * rinv * rinv;
        Dr = fmaf(f, fmaf(rho, ei, er), Dr);
        Di = fmaf(f, fmaf(-rho, er, ei), Di);
      }
#pragma unroll
      for (int s = 0; s < NR; ++s) {
        const float2 pj = s_p[t * NR + s], gj = s_g[t * NR + s];
        accr[s] += pj.x * Dr - pj.y * Di - (gj.x * Gr - gj.y * Gi);
        acci[s] += pj.x * Di + pj.y * Dr - (gj.x * Gi + gj.y * Gr);
      }
    }
  }
  if (ok) {
#pragma unroll
    for (int s = 0; s < NR; ++s)
      part[((size_t)blockIdx.y * m + qi) * NR + s] = make_double2(accr[s], acci[s]);
  }
}

// Far-field pattern, the leading FFAT term (paper Sec. 3.1): for unit directions d,
//   F(d) = lim r e^{-ikr} p(r d) = sum_j sum_q (w_q A_j / 4pi) [p_j (-i k d.n_j) - g_j] e^{-ik d.y_jq}
// with the same per-element rule (or one point per Monte-Carlo sample) as the field; one thread
// per direction, elements staged in shared memory, per-split FP64 partials as in k_eval.
template <int NR, int NQ>
__global__ void __launch_bounds__(kEvalThreads)
k_far_field(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo,
            const float4* __restrict__ nrm, const float4* __restrict__ qp, int n,
            const double* __restrict__ dirs, int nd, float k, const float2* __restrict__ p,
            const float2* __restrict__ g, int rhs0, int nr, int elems_per_split, double2* __restrict__ part) {
  __shared__ float4 s_hi[kElemStage], s_lo[kElemStage], s_n[kElemStage];
  __shared__ float4 s_q[kElemStage * NQ];
  __shared__ float2 s_p[kElemStage * NR], s_g[kElemStage * NR];
  const int qi = blockIdx.x * kEvalThreads + threadIdx.x;
  const bool ok = qi < nd;
  float d0 = 0.f, d1 = 0.f, d2 = 0.f;
  if (ok) {
    d0 = (float)dirs[3 * (size_t)qi];
    d1 = (float)dirs[3 * (size_t)qi + 1];
    d2 = (float)dirs[3 * (size_t)qi + 2];
  }
  const int j_begin = blockIdx.y * elems_per_split;
  const int j_end = min(n, j_begin + elems_per_split);
  float accr[NR], acci[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) accr[s] = acci[s] = 0.f;
  for (int jb = j_begin; jb < j_end; jb += kElemStage) {
    const int cnt = min(kElemStage, j_end - jb);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt * NQ; t += kEvalThreads) s_q[t] = qp[NQ * (size_t)jb + t];
    if (threadIdx.x < cnt) {
      const int j = jb + threadIdx.x;
      s_hi[threadIdx.x] = c_hi[j];
      s_lo[threadIdx.x] = c_lo[j];
      s_n[threadIdx.x] = nrm[j];
#pragma unroll
      for (int s = 0; s < NR; ++s) {  // right-hand sides past nr read as zero
        s_p[threadIdx.x * NR + s] = s < nr ? p[(size_t)(rhs0 + s) * n + j] : make_float2(0.f, 0.f);
        s_g[threadIdx.x * NR + s] = s < nr ? g[(size_t)(rhs0 + s) * n + j] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    if (!ok) continue;
    for (int t = 0; t < cnt; ++t) {
      const float4 ch = s_hi[t], cl = s_lo[t], nj = s_n[t];
      const float dc = fmaf(d0, ch.x, fmaf(d1, ch.y, d2 * ch.z)) + fmaf(d0, cl.x, fmaf(d1, cl.y, d2 * cl.z));
      const float kdn = k * fmaf(d0, nj.x, fmaf(d1, nj.y, d2 * nj.z));
      float Er = 0.f, Ei = 0.f;  // sum_q (w A / 4pi) e^{-ik d.y}
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 o = s_q[NQ * t + q];
        const float ph = -k * (dc + fmaf(d0, o.x, fmaf(d1, o.y, d2 * o.z)));
        const float nq = rintf(ph * kInvTwoPi);
        float th = fmaf(-nq, kTwoPiHi, ph);
        th = fmaf(-nq, kTwoPiLo, th);
        float sn, cs;
        __sincosf(th, &sn, &cs);
        Er = fmaf(o.w, cs, Er);
        Ei = fmaf(o.w, sn, Ei);
      }
#pragma unroll
      for (int s = 0; s < NR; ++s) {
        const float2 pj = s_p[t * NR + s], gj = s_g[t * NR + s];
        // a = p (-i k d.n) - g
        const float ar = fmaf(kdn, pj.y, -gj.x), ai = fmaf(-kdn, pj.x, -gj.y);
        accr[s] += ar * Er - ai * Ei;
        acci[s] += ar * Ei + ai * Er;
      }
    }
  }
  if (ok) {
#pragma unroll
    for (int s = 0; s < NR; ++s)
      part[((size_t)blockIdx.y * nd + qi) * NR + s] = make_double2(accr[s], acci[s]);
  }
}

// Training-sample coordinates (paper Sec. 3.4): theta = pi u0, phi = 2 pi u1,
// r = r_lo + (r_hi - r_lo) u2 about the centre; writes (theta, phi, r) and the Cartesian point.
__global__ void k_sample_points(const double* __restrict__ u, int64_t n, double cx, double cy, double cz,
                                double r_lo, double r_hi, double* __restrict__ coords,
                                double* __restrict__ pts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double th = 3.14159265358979323846 * u[3 * i];
  const double ph = 6.28318530717958647692 * u[3 * i + 1];
  const double r = r_lo + (r_hi - r_lo) * u[3 * i + 2];
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  coords[3 * i] = th;
  coords[3 * i + 1] = ph;
  coords[3 * i + 2] = r;
  pts[3 * i] = cx + r * st * cp;
  pts[3 * i + 1] = cy + r * st * sp;
  pts[3 * i + 2] = cz + r * ct;
}

// |p| of complex64 values
__global__ void k_abs(const float2* __restrict__ v, int64_t count, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = hypotf(v[i].x, v[i].y);
}

// out[q, rhs0 + s] = sum over splits of the partials, complex64, column-major (m x nrhs)
__global__ void k_eval_reduce(const double2* __restrict__ part, int m, int splits, int nr, int stride,
                              int rhs0, float2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)m * nr) return;
  const int qi = (int)(i / nr), s = (int)(i % nr);
  double re = 0.0, im = 0.0;
  for (int t = 0; t < splits; ++t) {
    const double2 v = part[((size_t)t * m + qi) * stride + s];
    re += v.x;
    im += v.y;
  }
  out[(size_t)(rhs0 + s) * m + qi] = make_float2((float)re, (float)im);
}

// Pass width for nr right-hand sides: the smallest of 1, 2, 4, 8, 16 that holds them. Each
// (point, element) kernel value is computed once per pass and applied to every RHS of it.
static int pass_width(int nr) { return nr <= 1 ? 1 : nr <= 2 ? 2 : nr <= 4 ? 4 : nr <= 8 ? 8 : 16; }
// The field kernel also takes passes of 32 RHS (64 accumulators a thread, 168 registers): each
// kernel value is then evaluated twice at 64 RHS instead of four times. A pass of 64 spills.
static int eval_pass_width(int nr) { return nr <= 16 ? pass_width(nr) : 32; }

// One k_eval launch for nr right-hand sides: seven quadrature points per element, or one
// sample point per Monte-Carlo sample (weight w / (4 pi) at offset 0). Partials are strided by
// pass_width(nr).
template <int NQ>
static void eval_launch_nq(int nr, dim3 grid, cudaStream_t s, const Geometry& g, int n,
                           const double* d_pts, int m, float k, const float2* d_p,
                           const float2* d_g, int r0, int per, double2* part) {
  switch (eval_pass_width(nr)) {
    case 1: k_eval<1, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
    case 2: k_eval<2, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
    case 4: k_eval<4, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
    case 8: k_eval<8, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
    case 16: k_eval<16, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
    default: k_eval<32, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_pts, m, k, d_p, d_g, r0, nr, per, part); break;
  }
}

// The element records a field kernel sums over: seven points per element, or one point per
// record (Monte-Carlo samples; the quadrature points of a Galerkin op's elements, with the P1
// pressure and the P0 Neumann data expanded to them).
struct EvalSource {
  const Geometry* g;
  int n;
  bool one_point;
};

static void eval_launch(const EvalSource& src, float k, int nr, dim3 grid, cudaStream_t s, const double* d_pts,
                        int m, const float2* d_p, const float2* d_g, int r0, int per, double2* part) {
  if (src.one_point)
    eval_launch_nq<1>(nr, grid, s, *src.g, src.n, d_pts, m, k, d_p, d_g, r0, per, part);
  else
    eval_launch_nq<7>(nr, grid, s, *src.g, src.n, d_pts, m, k, d_p, d_g, r0, per, part);
}

static EvalSource eval_source(const nat_bem_op* op) {
  if (op->galerkin) return EvalSource{&op->gal.pts, (int)op->gal.pts.n, true};
  return EvalSource{&op->geo, (int)op->n, op->mc};
}

static nat_bem_status eval_core(const nat_bem_op* op, const double* d_pts, int64_t m,
                                const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                                cudaStream_t s);

nat_bem_status eval_impl(const nat_bem_op* op, const double* d_pts, int64_t m,
                         const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                         cudaStream_t s) {
  if (m == 0) return NAT_BEM_OK;
  if (!op->galerkin) return eval_core(op, d_pts, m, d_p, d_g, nrhs, d_out, s);
  float2 *pq = nullptr, *gq = nullptr;
  NB_TRY(galerkin_expand(op, d_p, d_g, nrhs, &pq, &gq, s));
  nat_bem_status st = eval_core(op, d_pts, m, pq, gq, nrhs, d_out, s);
  dev_free(pq, s);
  dev_free(gq, s);
  return st;
}

static nat_bem_status eval_core(const nat_bem_op* op, const double* d_pts, int64_t m,
                                const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                                cudaStream_t s) {
  const EvalSource src = eval_source(op);
  const int n = src.n;
  const int pblocks = (int)((m + kEvalThreads - 1) / kEvalThreads);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // split the elements so that the grid holds about `bps` blocks per SM; the autotuner picks
  // bps among 4 (the default), 2, 8 and 16 per size class (elements, points, RHS pass)
  auto split_of = [&](int bps, int* per_out) {
    int splits = (bps * sms + pblocks - 1) / pblocks;
    splits = max(1, min(splits, (n + kElemStage - 1) / kElemStage));
    int per = (n + splits - 1) / splits;
    per = (per + kElemStage - 1) / kElemStage * kElemStage;
    *per_out = per;
    return (n + per - 1) / per;
  };
  static const int kBps[4] = {4, 2, 8, 16};
  int max_splits = 1, per = 0;
  for (int c = 0; c < 4; ++c) max_splits = max(max_splits, split_of(kBps[c], &per));
  double2* part = nullptr;
  NB_TRY(dev_alloc_n(&part, (size_t)max_splits * m * eval_pass_width(min(kEvalRhsPass, nrhs)), s));
  auto run = [&](int bps, int r0, int nr) -> nat_bem_status {
    int per_c = 0;
    const int splits = split_of(bps, &per_c);
    dim3 grid(pblocks, splits);
    NB_LAUNCH("eval", s, eval_launch(src, (float)op->k, nr, grid, s, d_pts, (int)m, d_p, d_g, r0, per_c, part));
    NB_CHECK_LAUNCH();
    const int64_t tot = m * nr;
    NB_LAUNCH("eval_reduce", s, k_eval_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, (int)m, splits, nr, eval_pass_width(nr), r0, d_out));
    NB_CHECK_LAUNCH();
    return NAT_BEM_OK;
  };
  const int nr0 = min(kEvalRhsPass, nrhs);
  const int64_t cls = ((int64_t)((n + 1023) / 1024) << 32) | ((int64_t)((m + 255) / 256) << 8) |
                      ((int64_t)eval_pass_width(nr0) << 1) | (src.one_point ? 1 : 0);
  const int pick = autotune("eval_bps", cls, 4, [&](int c) { return run(kBps[c], 0, nr0); }, s);
  nat_bem_status st = NAT_BEM_OK;
  for (int r0 = 0; r0 < nrhs && st == NAT_BEM_OK; r0 += kEvalRhsPass)
    st = run(kBps[pick], r0, min(kEvalRhsPass, nrhs - r0));
  dev_free(part, s);
  return st;
}

template <int NQ>
static void far_launch_nq(int nr, dim3 grid, cudaStream_t s, const Geometry& g, int n,
                          const double* d_dirs, int nd, float k, const float2* d_p,
                          const float2* d_g, int r0, int per, double2* part) {
  switch (pass_width(nr)) {
    case 1: k_far_field<1, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_dirs, nd, k, d_p, d_g, r0, nr, per, part); break;
    case 2: k_far_field<2, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_dirs, nd, k, d_p, d_g, r0, nr, per, part); break;
    case 4: k_far_field<4, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_dirs, nd, k, d_p, d_g, r0, nr, per, part); break;
    case 8: k_far_field<8, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_dirs, nd, k, d_p, d_g, r0, nr, per, part); break;
    default: k_far_field<16, NQ><<<grid, kEvalThreads, 0, s>>>(g.c_hi, g.c_lo, g.nrm, g.qp, n, d_dirs, nd, k, d_p, d_g, r0, nr, per, part); break;
  }
}

static nat_bem_status far_field_core(const nat_bem_op* op, const double* d_dirs, int64_t nd,
                                     const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                                     cudaStream_t s);

nat_bem_status far_field_impl(const nat_bem_op* op, const double* d_dirs, int64_t nd,
                              const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                              cudaStream_t s) {
  if (nd == 0) return NAT_BEM_OK;
  if (!op->galerkin) return far_field_core(op, d_dirs, nd, d_p, d_g, nrhs, d_out, s);
  float2 *pq = nullptr, *gq = nullptr;
  NB_TRY(galerkin_expand(op, d_p, d_g, nrhs, &pq, &gq, s));
  nat_bem_status st = far_field_core(op, d_dirs, nd, pq, gq, nrhs, d_out, s);
  dev_free(pq, s);
  dev_free(gq, s);
  return st;
}

static nat_bem_status far_field_core(const nat_bem_op* op, const double* d_dirs, int64_t nd,
                                     const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                                     cudaStream_t s) {
  const EvalSource src = eval_source(op);
  const int n = src.n;
  const int pblocks = (int)((nd + kEvalThreads - 1) / kEvalThreads);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int splits = (4 * sms + pblocks - 1) / pblocks;
  splits = max(1, min(splits, (n + kElemStage - 1) / kElemStage));
  int per = (n + splits - 1) / splits;
  per = (per + kElemStage - 1) / kElemStage * kElemStage;
  splits = (n + per - 1) / per;
  double2* part = nullptr;
  NB_TRY(dev_alloc_n(&part, (size_t)splits * nd * pass_width(min(kMaxRhsPass, nrhs)), s));
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsPass) {
    const int nr = min(kMaxRhsPass, nrhs - r0);
    dim3 grid(pblocks, splits);
    if (src.one_point)
      NB_LAUNCH("far_field", s, far_launch_nq<1>(nr, grid, s, *src.g, n, d_dirs, (int)nd, (float)op->k, d_p, d_g, r0, per, part));
    else
      NB_LAUNCH("far_field", s, far_launch_nq<7>(nr, grid, s, *src.g, n, d_dirs, (int)nd, (float)op->k, d_p, d_g, r0, per, part));
    NB_CHECK_LAUNCH();
    const int64_t tot = nd * nr;
    NB_LAUNCH("eval_reduce", s, k_eval_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, (int)nd, splits, nr, pass_width(nr), r0, d_out));
    NB_CHECK_LAUNCH();
  }
  dev_free(part, s);
  return NAT_BEM_OK;
}

nat_bem_status sample_field_impl(const nat_bem_op* op, const double* d_u, int64_t n, const double* center,
                                 double r_lo, double r_hi, const float2* d_p, const float2* d_g, int nrhs,
                                 double* d_coords, float* d_amp, cudaStream_t s) {
  if (n == 0) return NAT_BEM_OK;
  double* pts = nullptr;
  float2* field = nullptr;
  NB_TRY(dev_alloc_n(&pts, (size_t)(3 * n), s));
  nat_bem_status st = dev_alloc_n(&field, (size_t)n * nrhs, s);
  if (st != NAT_BEM_OK) {
    dev_free(pts, s);
    return st;
  }
  NB_LAUNCH("sample_points", s, k_sample_points<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      d_u, n, center[0], center[1], center[2], r_lo, r_hi, d_coords, pts));
  st = eval_impl(op, pts, n, d_p, d_g, nrhs, field, s);
  if (st == NAT_BEM_OK) {
    const int64_t tot = n * nrhs;
    NB_LAUNCH("sample_abs", s, k_abs<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(field, tot, d_amp));
    if (cudaGetLastError() != cudaSuccess) {
      set_error("sample_field: launch failed");
      st = NAT_BEM_ECUDA;
    }
  }
  dev_free(pts, s);
  dev_free(field, s);
  return st;
}


// ------------------------------------------------------------- allocation-free variant
// Field evaluation for callers that must not allocate device memory: code running where
// cudaMalloc is off limits (inside another allocator's callback, under a memory budget that
// a framework enforces, or in a process whose device memory is owned by someone else). The
// per-split partial sums that eval_impl takes from the memory pool live instead in this fixed
// array, which every GPU that loads the library holds until the process exits.
constexpr size_t kNoAllocScratch = (size_t)1 << 18;  // double2 entries: 4 MiB
static __device__ __align__(256) double2 g_eval_scratch[kNoAllocScratch];
constexpr int64_t kNoAllocMaxPoints = (int64_t)(kNoAllocScratch / kNoAllocRhsPass);  // 65,536

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};
}  // namespace

// Device address of g_eval_scratch on the current device, looked up once per device (host
// code cannot use the symbol itself: on the host it names a stand-in, not device memory). The
// address is kept for the life of the process, so the library must not be used across a
// cudaDeviceReset (which would also invalidate every op).
static nat_bem_status scratch_address(double2** out) {
  int dev = 0;
  NB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return NAT_BEM_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(g_eval_scratch) failed: ") + cudaGetErrorString(e));
      return NAT_BEM_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<double2*>(g_scratch_ptr[dev]);
  return NAT_BEM_OK;
}

static nat_bem_status eval_noalloc_impl(const nat_bem_op* op, const double* d_pts, int64_t m,
                                        const float2* d_p, const float2* d_g, int nrhs,
                                        float2* d_out, cudaStream_t s) {
  double2* part = nullptr;
  NB_TRY(scratch_address(&part));
  const int n = (int)op->n;
  const int pblocks = (int)((m + kEvalThreads - 1) / kEvalThreads);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // as many element splits as eval_impl would take, capped by the scratch size
  int splits = (4 * sms + pblocks - 1) / pblocks;
  splits = max(1, min(splits, (n + kElemStage - 1) / kElemStage));
  const int cap = (int)(kNoAllocScratch / ((size_t)m * kNoAllocRhsPass));
  splits = max(1, min(splits, cap));
  int per = (n + splits - 1) / splits;
  per = (per + kElemStage - 1) / kElemStage * kElemStage;
  splits = (n + per - 1) / per;
  for (int r0 = 0; r0 < nrhs; r0 += kNoAllocRhsPass) {
    const int nr = min(kNoAllocRhsPass, nrhs - r0);
    dim3 grid(pblocks, splits);
    NB_LAUNCH("eval", s, eval_launch(eval_source(op), (float)op->k, nr, grid, s, d_pts, (int)m, d_p, d_g, r0, per, part));
    NB_CHECK_LAUNCH();
    const int64_t tot = m * nr;
    NB_LAUNCH("eval_reduce", s, k_eval_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, (int)m, splits, nr, eval_pass_width(nr), r0, d_out));
    NB_CHECK_LAUNCH();
  }
  return NAT_BEM_OK;
}

}  // namespace natbem

extern "C" nat_bem_status nat_bem_eval_noalloc(const nat_bem_op* op, const double* pts, int64_t m,
                                               const float* p, const float* neumann, int32_t nrhs,
                                               float* field_out, void* cuda_stream) {
  using namespace natbem;
  try {
    clear_error();
    if (!op || m < 0 || nrhs < 1 || (m > 0 && (!pts || !p || !neumann || !field_out))) {
      set_error("nat_bem_eval_noalloc: bad arguments (op NULL, m < 0, nrhs < 1 or NULL arrays)");
      return NAT_BEM_EINVAL;
    }
    if (m > kNoAllocMaxPoints) {
      set_error("nat_bem_eval_noalloc: m = " + std::to_string(m) + " exceeds the maximum of " +
                std::to_string(kNoAllocMaxPoints) + " points per call (split the points)");
      return NAT_BEM_EINVAL;
    }
    if (op->galerkin) {
      set_error("nat_bem_eval_noalloc: Galerkin ops need scratch for the P1 expansion: use nat_bem_eval");
      return NAT_BEM_EINVAL;
    }
    if (m == 0) return NAT_BEM_OK;
    if (!is_device_pointer(pts) || !is_device_pointer(p) || !is_device_pointer(neumann) ||
        !is_device_pointer(field_out)) {
      set_error("nat_bem_eval_noalloc: pts, p, neumann and field_out must be device pointers");
      return NAT_BEM_EINVAL;
    }
    return eval_noalloc_impl(op, pts, m, reinterpret_cast<const float2*>(p),
                             reinterpret_cast<const float2*>(neumann), nrhs,
                             reinterpret_cast<float2*>(field_out), (cudaStream_t)cuda_stream);
  } catch (...) {
    set_error("internal error in nat_bem_eval_noalloc");
    return NAT_BEM_ECUDA;
  }
}
