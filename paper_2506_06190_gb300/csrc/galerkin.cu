// Galerkin form of the Burton-Miller equation (paper Sec. 4, Eq. 6 tested with P1 hat functions;
// the element-to-element integration of Sec. 4.1): P1 Dirichlet data at the vertices, P0
// Neumann data per triangle,
//
//   L p = R g,  L = 1/2 M11 - K - beta H,  R = -V - beta K' - (beta/2) M10,
//   H_ij = int int G [k^2 (n_x . n_y) phi_j psi_i - curl phi_j . curl psi_i]   (Maue's form).
//
// Every entry is a sum over element pairs (tau test, sigma trial). The kernels compute, per
// pair, the 3 x 3 block of L and the 3 entries of R that the pair contributes (k_gal_regular for
// pairs sharing no vertex, 7 x 7 points; k_gal_singular for pairs sharing a vertex, an edge, or
// identical, a warp each over 4^4 Gauss points per region of the transformed 4-cube), into
// scratch arrays of pair blocks. The gathers then sum, for every vertex i and column (vertex j,
// or triangle s), the blocks of the triangles around i (and around j) in a fixed order, so the
// result does not depend on scheduling: k_gal_rowsum_L first sums each test triangle's row over
// the triangles around every column vertex (reading each pair block once), k_gal_gather_L and
// k_gal_gather_R then sum over the triangles around each row vertex. FP32 arithmetic throughout: near the
// singularity x - y is formed from the transformed coordinates (a radius times a bounded
// vector), and for regular pairs from the centroid difference (hi/lo pairs) plus the points'
// offsets, so no cancellation occurs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace natbem {

namespace {
constexpr int kGalSing = 4;          // Gauss-Legendre points per dimension on singular pairs
constexpr int kGalVals = 12;         // per pair: L block (a, b) at 3a + b, then R entries (a)
constexpr double kGalScratch = 4e9;  // bytes of pair blocks per round of test triangles
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.7484555314695172e-7f;
constexpr float kInvTwoPi = 0.159154943091895336f;
constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr float kFourPi = 12.5663706143591730f;

__constant__ float c_gal_b7[7][4];           // barycentric l0, l1, l2 and weight (sum 1)
__constant__ float c_gal_gl[kGalSing][2];    // Gauss-Legendre nodes and weights on [0, 1]

__device__ __forceinline__ uint32_t gal_pack_bf16(float re, float im) {
  __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Weighted kernels at x - y = d: w G, w dG/dn_y, w dG/dn_x (w includes 1 / (4 pi)).
struct GalK {
  float gr, gi, yr, yi, xr, xi;
};

// dny = d . n_y and dnx = d . n_x, given by the caller.
__device__ __forceinline__ GalK gal_kernels_dn(float dx, float dy, float dz, float k, float w, float dny,
                                               float dnx) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(r2);
  const float rho = k * (r2 * rinv);
  const float nq = rintf(rho * kInvTwoPi);
  float th = fmaf(-nq, kTwoPiHi, rho);
  th = fmaf(-nq, kTwoPiLo, th);
  float sn, cs;
  __sincosf(th, &sn, &cs);
  const float gw = rinv * w;
  GalK o;
  o.gr = cs * gw;
  o.gi = sn * gw;
  const float r2inv = rinv * rinv;
  const float fr = fmaf(rho, o.gi, o.gr) * r2inv, fi = fmaf(-rho, o.gr, o.gi) * r2inv;
  o.yr = fr * dny;
  o.yi = fi * dny;
  o.xr = -fr * dnx;
  o.xi = -fi * dnx;
  return o;
}

__device__ __forceinline__ GalK gal_kernels(float dx, float dy, float dz, float k, float w, float3 nx,
                                            float3 ny) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(r2);
  const float rho = k * (r2 * rinv);
  const float nq = rintf(rho * kInvTwoPi);
  float th = fmaf(-nq, kTwoPiHi, rho);
  th = fmaf(-nq, kTwoPiLo, th);
  float sn, cs;
  __sincosf(th, &sn, &cs);
  const float gw = rinv * w;
  GalK o;
  o.gr = cs * gw;
  o.gi = sn * gw;
  // G (1 - i rho) / r^2, times d.n_y (dG/dn_y) and -d.n_x (dG/dn_x)
  const float r2inv = rinv * rinv;
  const float fr = fmaf(rho, o.gi, o.gr) * r2inv, fi = fmaf(-rho, o.gr, o.gi) * r2inv;
  const float dny = fmaf(dx, ny.x, fmaf(dy, ny.y, dz * ny.z));
  const float dnx = fmaf(dx, nx.x, fmaf(dy, nx.y, dz * nx.z));
  o.yr = fr * dny;
  o.yi = fi * dny;
  o.xr = -fr * dnx;
  o.xi = -fi * dnx;
  return o;
}

// Per-pair sums: Kb[a][b] = sum w lam_a mu_b dG/dn_y, Gb[a][b] = sum w lam_a mu_b G,
// Kp[a] = sum w lam_a dG/dn_x (complex, interleaved re/im).
struct GalAcc {
  float kb[18], gb[18], kp[6];
};

__device__ __forceinline__ void gal_acc_zero(GalAcc& A) {
#pragma unroll
  for (int i = 0; i < 18; ++i) A.kb[i] = A.gb[i] = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) A.kp[i] = 0.f;
}

__device__ __forceinline__ void gal_acc_point(GalAcc& A, const float (&lam)[3], const float (&mu)[3],
                                              const GalK& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float lm = lam[a] * mu[b];
      A.kb[2 * (3 * a + b)] = fmaf(lm, v.yr, A.kb[2 * (3 * a + b)]);
      A.kb[2 * (3 * a + b) + 1] = fmaf(lm, v.yi, A.kb[2 * (3 * a + b) + 1]);
      A.gb[2 * (3 * a + b)] = fmaf(lm, v.gr, A.gb[2 * (3 * a + b)]);
      A.gb[2 * (3 * a + b) + 1] = fmaf(lm, v.gi, A.gb[2 * (3 * a + b) + 1]);
    }
    A.kp[2 * a] = fmaf(lam[a], v.xr, A.kp[2 * a]);
    A.kp[2 * a + 1] = fmaf(lam[a], v.xi, A.kp[2 * a + 1]);
  }
}

// The pair's 12 values: L block -Kb - beta H and R entries -Vb - beta Kp (beta = i / k), with
// H = k^2 (n_t . n_s) Gb - (curl_a^t . curl_b^s) G0, Vb[a] = sum_b Gb[a][b], G0 = sum Gb.
__device__ __forceinline__ void gal_finish(const GalAcc& A, float k, float nn, const float (&cc)[9],
                                           float2 (&out)[kGalVals]) {
  const float kinv = 1.f / k, k2 = k * k;
  float g0r = 0.f, g0i = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    g0r += A.gb[2 * i];
    g0i += A.gb[2 * i + 1];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float hr = k2 * nn * A.gb[2 * i] - cc[i] * g0r;
    const float hi = k2 * nn * A.gb[2 * i + 1] - cc[i] * g0i;
    // -Kb - (i/k) H = (-Kb_r + H_i / k, -Kb_i - H_r / k)
    out[i] = make_float2(-A.kb[2 * i] + hi * kinv, -A.kb[2 * i + 1] - hr * kinv);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float vr = A.gb[2 * (3 * a)] + A.gb[2 * (3 * a + 1)] + A.gb[2 * (3 * a + 2)];
    const float vi = A.gb[2 * (3 * a) + 1] + A.gb[2 * (3 * a + 1) + 1] + A.gb[2 * (3 * a + 2) + 1];
    out[9 + a] = make_float2(-vr + A.kp[2 * a + 1] * kinv, -vi - A.kp[2 * a] * kinv);
  }
}

// Pair (t, s) of the round starting at t0: the L block at partL[((t - t0) nt + s) 9 + 3a + b],
// the R entries at partR[((t - t0) 3 + a) nt + s] (contiguous over s for the R gather).
__device__ __forceinline__ void gal_store(float2* partL, float2* partR, int nt, int tr, int s,
                                          const float2 (&v)[kGalVals]) {
  float2* pl = partL + ((size_t)tr * nt + s) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) pl[i] = v[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) partR[((size_t)tr * 3 + a) * nt + s] = v[9 + a];
}
}  // namespace

// Per element: the three P1 curls (P_{a+1} - P_{a+2}) / (2A); per quadrature point (7 per
// element): a point record for the field kernels (position hi/lo, normal, weight w A / (4 pi)).
__global__ void k_gal_geometry(const double* __restrict__ tri, const double* __restrict__ nrm64,
                               const double* __restrict__ area, int nt, float4* __restrict__ curl,
                               float4* __restrict__ p_hi, float4* __restrict__ p_lo, float4* __restrict__ p_n,
                               float4* __restrict__ p_q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* P = tri + 9 * (size_t)t;
  const double A = area[t];
  for (int a = 0; a < 3; ++a) {
    const double* p1 = P + 3 * ((a + 1) % 3);
    const double* p2 = P + 3 * ((a + 2) % 3);
    curl[3 * (size_t)t + a] = make_float4((float)((p1[0] - p2[0]) / (2 * A)), (float)((p1[1] - p2[1]) / (2 * A)),
                                          (float)((p1[2] - p2[2]) / (2 * A)), 0.f);
  }
  for (int q = 0; q < 7; ++q) {
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
      const double y = (double)c_gal_b7[q][0] * P[d] + (double)c_gal_b7[q][1] * P[3 + d] + (double)c_gal_b7[q][2] * P[6 + d];
      hi[d] = (float)y;
      lo[d] = (float)(y - (double)hi[d]);
    }
    const size_t i = 7 * (size_t)t + q;
    p_hi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
    p_lo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    p_n[i] = make_float4((float)nrm64[3 * t], (float)nrm64[3 * t + 1], (float)nrm64[3 * t + 2], 0.f);
    p_q[i] = make_float4(0.f, 0.f, 0.f, (float)((double)c_gal_b7[q][3] * A * 0.25 / 3.14159265358979323846));
  }
}

// Pairs sharing no vertex: block row tau = t0 + blockIdx.y, one thread per trial triangle.
__global__ void __launch_bounds__(256, 2)
k_gal_regular(const float4* __restrict__ c_hi, const float4* __restrict__ c_lo, const float4* __restrict__ nrm,
              const float4* __restrict__ qp, const int4* __restrict__ vid, const float4* __restrict__ curl,
              int nt, int t0, float k, float2* __restrict__ partL, float2* __restrict__ partR) {
  const int t = t0 + blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nt) return;
  const int4 vt = vid[t], vs = vid[s];
  const int va[3] = {vt.x, vt.y, vt.z}, vb[3] = {vs.x, vs.y, vs.z};
  bool touch = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) touch |= va[a] == vb[b];
  if (touch) return;  // k_gal_singular writes this pair
  const float4 th = c_hi[t], tl = c_lo[t], sh = c_hi[s], sl = c_lo[s];
  const float Dx = (th.x - sh.x) + (tl.x - sl.x);
  const float Dy = (th.y - sh.y) + (tl.y - sl.y);
  const float Dz = (th.z - sh.z) + (tl.z - sl.z);
  const float4 nt4 = nrm[t], ns4 = nrm[s];
  const float3 nx = make_float3(nt4.x, nt4.y, nt4.z), ny = make_float3(ns4.x, ns4.y, ns4.z);
  float4 qs[7];
  float qny[7], qnx[7];  // y_q . n_y and y_q . n_x of the trial points' offsets
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    qs[q] = qp[7 * (size_t)s + q];
    qny[q] = fmaf(qs[q].x, ny.x, fmaf(qs[q].y, ny.y, qs[q].z * ny.z));
    qnx[q] = fmaf(qs[q].x, nx.x, fmaf(qs[q].y, nx.y, qs[q].z * nx.z));
  }
  GalAcc A;
  gal_acc_zero(A);
#pragma unroll 1
  for (int p = 0; p < 7; ++p) {
    const float4 qt = qp[7 * (size_t)t + p];
    const float wx = qt.w * kFourPi;  // w_p A_tau (the 1 / (4 pi) is in the trial weights)
    // x_p - y_q = (D + x_p offset) - y_q offset; its projections likewise
    const float px = Dx + qt.x, py = Dy + qt.y, pz = Dz + qt.z;
    const float pny = fmaf(px, ny.x, fmaf(py, ny.y, pz * ny.z)), pnx = fmaf(px, nx.x, fmaf(py, nx.y, pz * nx.z));
    // inner sums over the trial points, then the test basis functions. The rule's points are
    // the centroid (weights 1/3 on every basis function) and two orbits whose barycentric
    // coordinates permute (e, e, 1 - 2e): on an orbit, sum_q mu_b(q) v_q = e S + (1 - 3e) v_q*,
    // S the orbit's sum and q* its point with 1 - 2e on vertex b.
    float sg[6], sy[6], sx[2];
    {
      const GalK v = gal_kernels_dn(px - qs[0].x, py - qs[0].y, pz - qs[0].z, k, qs[0].w, pny - qny[0], pnx - qnx[0]);
      const float third = c_gal_b7[0][0];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        sg[2 * b] = third * v.gr;
        sg[2 * b + 1] = third * v.gi;
        sy[2 * b] = third * v.yr;
        sy[2 * b + 1] = third * v.yi;
      }
      sx[0] = v.xr;
      sx[1] = v.xi;
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int q0 = 1 + 3 * o;  // points q0, q0 + 1, q0 + 2 carry 1 - 2e on vertex 2, 1, 0
      float vg[3][4];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int q = q0 + i;
        const GalK v = gal_kernels_dn(px - qs[q].x, py - qs[q].y, pz - qs[q].z, k, qs[q].w, pny - qny[q], pnx - qnx[q]);
        vg[i][0] = v.gr;
        vg[i][1] = v.gi;
        vg[i][2] = v.yr;
        vg[i][3] = v.yi;
        sx[0] += v.xr;
        sx[1] += v.xi;
      }
      const float e = c_gal_b7[q0][0], f = c_gal_b7[q0][2] - e;  // e and 1 - 3e
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float S = e * ((vg[0][c] + vg[1][c]) + vg[2][c]);
        float* acc = c < 2 ? sg : sy;
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[2 * b + (c & 1)] += fmaf(f, vg[2 - b][c], S);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float la = c_gal_b7[p][a] * wx;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        A.kb[2 * (3 * a + b)] = fmaf(la, sy[2 * b], A.kb[2 * (3 * a + b)]);
        A.kb[2 * (3 * a + b) + 1] = fmaf(la, sy[2 * b + 1], A.kb[2 * (3 * a + b) + 1]);
        A.gb[2 * (3 * a + b)] = fmaf(la, sg[2 * b], A.gb[2 * (3 * a + b)]);
        A.gb[2 * (3 * a + b) + 1] = fmaf(la, sg[2 * b + 1], A.gb[2 * (3 * a + b) + 1]);
      }
      A.kp[2 * a] = fmaf(la, sx[0], A.kp[2 * a]);
      A.kp[2 * a + 1] = fmaf(la, sx[1], A.kp[2 * a + 1]);
    }
  }
  float cc[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float4 ca = curl[3 * (size_t)t + a];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 cb = curl[3 * (size_t)s + b];
      cc[3 * a + b] = ca.x * cb.x + ca.y * cb.y + ca.z * cb.z;
    }
  }
  float2 out[kGalVals];
  gal_finish(A, k, nx.x * ny.x + nx.y * ny.y + nx.z * ny.z, cc, out);
  gal_store(partL, partR, nt, blockIdx.y, s, out);
}

namespace {
// Barycentric coordinates placed at local vertices (i0, i1, i2).
__device__ __forceinline__ void gal_place(float (&l)[3], int i0, int i1, float v0, float v1, float v2) {
#pragma unroll
  for (int v = 0; v < 3; ++v) l[v] = v == i0 ? v0 : v == i1 ? v1 : v2;
}

__device__ __forceinline__ float3 f3sub(const double* a, const double* b) {
  return make_float3((float)(a[0] - b[0]), (float)(a[1] - b[1]), (float)(a[2] - b[2]));
}
}  // namespace

// Pairs sharing a vertex or an edge (the near-pair list), then the identical pairs: one warp
// per pair, the rule's points dealt over the lanes, a fixed shuffle tree, lane 0 writes.
__global__ void __launch_bounds__(256)
k_gal_singular(const int2* __restrict__ near_pairs, int64_t n_near, const double* __restrict__ tri,
               const double* __restrict__ nrm64, const double* __restrict__ area, const int4* __restrict__ vid,
               const float4* __restrict__ curl, int nt, int t0, int t1, float k, float2* __restrict__ partL,
               float2* __restrict__ partR) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_near + nt) return;
  int t, s;
  if (w < n_near) {
    const int2 pr = near_pairs[w];
    t = pr.x;
    s = pr.y;
  } else {
    t = s = (int)(w - n_near);
  }
  if (t < t0 || t >= t1) return;
  const double* Pt = tri + 9 * (size_t)t;
  const double* Ps = tri + 9 * (size_t)s;
  const double At = area[t], As = area[s];
  const float3 nx = make_float3((float)nrm64[3 * t], (float)nrm64[3 * t + 1], (float)nrm64[3 * t + 2]);
  const float3 ny = make_float3((float)nrm64[3 * s], (float)nrm64[3 * s + 1], (float)nrm64[3 * s + 2]);
  const int4 vt4 = vid[t], vs4 = vid[s];
  const int vt[3] = {vt4.x, vt4.y, vt4.z}, vs[3] = {vs4.x, vs4.y, vs4.z};
  // shared vertices in the order (a over tau, b over sigma)
  int sh_a[2] = {0, 0}, sh_b[2] = {0, 0}, nsh = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (vt[a] == vs[b] && nsh < 2) {
        sh_a[nsh] = a;
        sh_b[nsh] = b;
        ++nsh;
      }
  const int kind = t == s ? 3 : nsh;  // 1 vertex, 2 edge, 3 identical
  const int regions = kind == 1 ? 2 : 6;
  const int npts = regions * kGalSing * kGalSing * kGalSing * kGalSing;
  const float jac_area = (float)(4.0 * At * As) * kInv4Pi;
  GalAcc A;
  gal_acc_zero(A);
  // geometry of the rule in FP32 (differences of FP64 vertices)
  float3 e1, e2, e3, e4;
  int ia = 0, ib = 0, ic = 0, ja = 0, jb = 0, jc = 0;
  if (kind == 3) {
    e1 = f3sub(Pt + 3, Pt);      // B - A
    e2 = f3sub(Pt + 6, Pt + 3);  // C - B
    e3 = e4 = e1;
  } else if (kind == 2) {
    ia = sh_a[0];
    ib = sh_a[1];
    ja = sh_b[0];
    jb = sh_b[1];
    ic = 3 - ia - ib;
    jc = 3 - ja - jb;
    e1 = f3sub(Pt + 3 * ib, Pt + 3 * ia);  // Pb - Pa
    e2 = f3sub(Pt + 3 * ic, Pt + 3 * ia);  // Ct - Pa
    e3 = f3sub(Ps + 3 * jc, Pt + 3 * ia);  // Cs - Pa
    e4 = e1;
  } else {
    ia = sh_a[0];
    ja = sh_b[0];
    e1 = f3sub(Pt + 3 * ((ia + 1) % 3), Pt + 3 * ia);
    e2 = f3sub(Pt + 3 * ((ia + 2) % 3), Pt + 3 * ia);
    e3 = f3sub(Ps + 3 * ((ja + 1) % 3), Pt + 3 * ia);
    e4 = f3sub(Ps + 3 * ((ja + 2) % 3), Pt + 3 * ia);
  }
  for (int idx = lane; idx < npts; idx += 32) {
    const int region = idx >> 8, g = idx & 255;
    const float2 n0 = make_float2(c_gal_gl[g >> 6][0], c_gal_gl[g >> 6][1]);
    const float2 n1 = make_float2(c_gal_gl[(g >> 4) & 3][0], c_gal_gl[(g >> 4) & 3][1]);
    const float2 n2 = make_float2(c_gal_gl[(g >> 2) & 3][0], c_gal_gl[(g >> 2) & 3][1]);
    const float2 n3 = make_float2(c_gal_gl[g & 3][0], c_gal_gl[g & 3][1]);
    const float gw = n0.y * n1.y * n2.y * n3.y;
    float lam[3], mu[3], dx, dy, dz, jac;
    if (kind == 3) {
      // relative coordinate z on the hexagon T - T, sector `region`, Duffy (rho, w); x in the
      // homothetic triangle of scale 1 - rho by collapsed coordinates (a1, a1 a2)
      // hexagon vertices (1,0), (1,1), (0,1), (-1,0), (-1,-1), (0,-1), by selects (no local array)
      const int r1 = region == 5 ? 0 : region + 1;
      const float hx0 = region < 2 ? 1.f : (region == 2 || region == 5) ? 0.f : -1.f;
      const float hy0 = (region == 0 || region == 3) ? 0.f : region < 3 ? 1.f : -1.f;
      const float hx1 = r1 < 2 ? 1.f : (r1 == 2 || r1 == 5) ? 0.f : -1.f;
      const float hy1 = (r1 == 0 || r1 == 3) ? 0.f : r1 < 3 ? 1.f : -1.f;
      const float rho = n0.x, wv = n1.x, a1 = n2.x, a2 = n3.x;
      const float z1 = rho * fmaf(wv, hx1 - hx0, hx0);
      const float z2 = rho * fmaf(wv, hy1 - hy0, hy0);
      const float ca = fmaxf(0.f, -z2), cb = fmaxf(0.f, z2 - z1);
      const float scale = 1.f - rho;
      const float xs = ca + cb + scale * a1, xt = ca + scale * (a1 * a2);
      const float ys = xs + z1, yt = xt + z2;
      jac = rho * scale * scale * a1;
      dx = -(z1 * e1.x + z2 * e2.x);
      dy = -(z1 * e1.y + z2 * e2.y);
      dz = -(z1 * e1.z + z2 * e2.z);
      lam[0] = 1.f - xs;
      lam[1] = xs - xt;
      lam[2] = xt;
      mu[0] = 1.f - ys;
      mu[1] = ys - yt;
      mu[2] = yt;
    } else if (kind == 2) {
      // along the shared edge (xi on tau, xs on sigma = xi + delta) and towards the opposite
      // vertices (et, es); regions: sign of delta, then which of et, es, |delta| is largest
      const float tt = n0.x, u = n1.x, v = n2.x, wv = n3.x;
      const int sgn = region < 3 ? 1 : -1, reg = region % 3;
      const float et = reg == 0 ? tt : tt * u;
      const float es = reg == 0 ? tt * u : reg == 1 ? tt : tt * v;
      const float dd = reg == 2 ? tt : tt * v;
      const float delta = sgn > 0 ? dd : -dd;
      const float xi = sgn > 0 ? (1.f - dd) * wv : fmaf(1.f - dd, wv, dd);
      const float xs = xi + delta;
      jac = tt * tt * (1.f - dd) * (1.f - et) * (1.f - es);
      // d = -delta e + et (Ct - Et) - es (Cs - Es), Et - Pa = xi e, Es - Pa = xs e
      dx = -delta * e1.x + et * (e2.x - xi * e1.x) - es * (e3.x - xs * e1.x);
      dy = -delta * e1.y + et * (e2.y - xi * e1.y) - es * (e3.y - xs * e1.y);
      dz = -delta * e1.z + et * (e2.z - xi * e1.z) - es * (e3.z - xs * e1.z);
      gal_place(lam, ia, ib, (1.f - et) * (1.f - xi), (1.f - et) * xi, et);
      gal_place(mu, ja, jb, (1.f - es) * (1.f - xs), (1.f - es) * xs, es);
    } else {
      // polar coordinates about the shared vertex on both triangles, the smaller radius as a
      // fraction of the larger
      const float tt = n0.x, u = n1.x, thv = n2.x, ths = n3.x;
      const float rt = region == 0 ? tt : tt * u, rs = region == 0 ? tt * u : tt;
      jac = tt * tt * tt * u;
      const float etx = fmaf(thv, e2.x - e1.x, e1.x), ety = fmaf(thv, e2.y - e1.y, e1.y), etz = fmaf(thv, e2.z - e1.z, e1.z);
      const float esx = fmaf(ths, e4.x - e3.x, e3.x), esy = fmaf(ths, e4.y - e3.y, e3.y), esz = fmaf(ths, e4.z - e3.z, e3.z);
      dx = rt * etx - rs * esx;
      dy = rt * ety - rs * esy;
      dz = rt * etz - rs * esz;
      gal_place(lam, ia, (ia + 1) % 3, 1.f - rt, rt * (1.f - thv), rt * thv);
      gal_place(mu, ja, (ja + 1) % 3, 1.f - rs, rs * (1.f - ths), rs * ths);
    }
    const GalK v = gal_kernels(dx, dy, dz, k, gw * jac * jac_area, nx, ny);
    gal_acc_point(A, lam, mu, v);
  }
  // fixed-order reduction over the warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int i = 0; i < 18; ++i) {
      A.kb[i] += __shfl_xor_sync(0xffffffffu, A.kb[i], off);
      A.gb[i] += __shfl_xor_sync(0xffffffffu, A.gb[i], off);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) A.kp[i] += __shfl_xor_sync(0xffffffffu, A.kp[i], off);
  }
  if (lane != 0) return;
  float cc[9];
  for (int a = 0; a < 3; ++a) {
    const float4 ca = curl[3 * (size_t)t + a];
    for (int b = 0; b < 3; ++b) {
      const float4 cb = curl[3 * (size_t)s + b];
      cc[3 * a + b] = ca.x * cb.x + ca.y * cb.y + ca.z * cb.z;
    }
  }
  float2 out[kGalVals];
  gal_finish(A, k, nx.x * ny.x + nx.y * ny.y + nx.z * ny.z, cc, out);
  if (kind == 3) {
    // mass terms: 1/2 M11 (A / 12 (1 + delta_ab)) and -(beta / 2) M10 (A / 3), beta = i / k
    const float m = (float)(At / 24.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) out[3 * a + b].x += a == b ? 2.f * m : m;
    for (int a = 0; a < 3; ++a) out[9 + a].y -= (float)(At / 6.0) / k;
  }
  gal_store(partL, partR, nt, t - t0, s, out);
}

// First stage of the L gather, one block row per test triangle tau of the round: for every
// column vertex j and local test index a, P2[(tau - t0) 3 + a][j] = sum over the triangles sigma
// around j (local index b) of the pair blocks (tau, sigma)[a][b]. Each block reads its own row
// of pair blocks, so every pair block is read from memory once.
__global__ void __launch_bounds__(256)
k_gal_rowsum_L(const float2* __restrict__ partL, int nt, const int* __restrict__ adj_ptr,
               const int2* __restrict__ adj, int nv, int ldv, float2* __restrict__ P2) {
  const int tr = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const float2* row = partL + (size_t)tr * nt * 9;
  float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int v = adj_ptr[j]; v < adj_ptr[j + 1]; ++v) {
    const int2 sb = adj[v];
    const float2* blk = row + (size_t)sb.x * 9 + sb.y;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 x = blk[3 * a];
      acc[a].x += x.x;
      acc[a].y += x.y;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) P2[((size_t)tr * 3 + a) * ldv + j] = acc[a];
}

// L[i][j] (+)= sum over the triangles tau around i (local index a) in the round of
// P2[(tau - t0) 3 + a][j]; adjacency lists in increasing triangle order. Columns past nv are
// zero. With Lb, the BF16 copy is written too (on the last round).
__global__ void __launch_bounds__(256)
k_gal_gather_L(const float2* __restrict__ P2, int t0, int t1, const int* __restrict__ adj_ptr,
               const int2* __restrict__ adj, int nv, int ldv, int accumulate, float2* __restrict__ L,
               uint32_t* __restrict__ Lb) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ldv) return;
  const size_t off = (size_t)i * ldv + j;
  float2 acc = accumulate ? L[off] : make_float2(0.f, 0.f);
  if (j < nv) {
    for (int u = adj_ptr[i]; u < adj_ptr[i + 1]; ++u) {
      const int2 ta = adj[u];
      if (ta.x < t0 || ta.x >= t1) continue;
      const float2 x = P2[((size_t)(ta.x - t0) * 3 + ta.y) * ldv + j];
      acc.x += x.x;
      acc.y += x.y;
    }
  }
  L[off] = acc;
  if (Lb) Lb[off] = gal_pack_bf16(acc.x, acc.y);
}

// R[i][s] (+)= sum over the triangles tau around i in the round of partR[(tau - t0) 3 + a][s].
__global__ void __launch_bounds__(256)
k_gal_gather_R(const float2* __restrict__ partR, int nt, int t0, int t1, const int* __restrict__ adj_ptr,
               const int2* __restrict__ adj, int ldr, int accumulate, float2* __restrict__ R) {
  const int i = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ldr) return;
  const size_t off = (size_t)i * ldr + s;
  float2 acc = accumulate ? R[off] : make_float2(0.f, 0.f);
  if (s < nt) {
    for (int u = adj_ptr[i]; u < adj_ptr[i + 1]; ++u) {
      const int2 ta = adj[u];
      if (ta.x < t0 || ta.x >= t1) continue;
      const float2 x = partR[((size_t)(ta.x - t0) * 3 + ta.y) * nt + s];
      acc.x += x.x;
      acc.y += x.y;
    }
  }
  R[off] = acc;
}

// P1 data at the vertices and P0 data per triangle, expanded to the 7 points of every triangle:
// pq[r][7 t + q] = sum_b lam_qb p[r][vid_tb], gq[r][7 t + q] = g[r][t].
__global__ void k_gal_expand(const int4* __restrict__ vid, int nt, int nv, int nrhs, const float2* __restrict__ p,
                             const float2* __restrict__ g, float2* __restrict__ pq, float2* __restrict__ gq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = 7 * (int64_t)nt;
  if (i >= per * nrhs) return;
  const int r = (int)(i / per);
  const int64_t e = i % per;
  const int t = (int)(e / 7), q = (int)(e % 7);
  const int4 v = vid[t];
  const float2* pr = p + (size_t)r * nv;
  const float2 a = pr[v.x], b = pr[v.y], c = pr[v.z];
  const float l0 = c_gal_b7[q][0], l1 = c_gal_b7[q][1], l2 = c_gal_b7[q][2];
  pq[i] = make_float2(l0 * a.x + l1 * b.x + l2 * c.x, l0 * a.y + l1 * b.y + l2 * c.y);
  gq[i] = g[(size_t)r * nt + t];
}

namespace {
nat_bem_status gal_upload_rules() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && done[dev]) return NAT_BEM_OK;
  const double s15 = std::sqrt(15.0);
  const double a = (6.0 - s15) / 21.0, wa = (155.0 - s15) / 1200.0;
  const double b = (6.0 + s15) / 21.0, wb = (155.0 + s15) / 1200.0;
  const double r[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40}, {a, a, 1 - 2 * a, wa}, {a, 1 - 2 * a, a, wa},
                          {1 - 2 * a, a, a, wa}, {b, b, 1 - 2 * b, wb}, {b, 1 - 2 * b, b, wb},
                          {1 - 2 * b, b, b, wb}};
  float rf[7][4];
  for (int i = 0; i < 7; ++i)
    for (int c = 0; c < 4; ++c) rf[i][c] = (float)r[i][c];
  NB_TRY_CUDA(cudaMemcpyToSymbol(c_gal_b7, rf, sizeof(rf)));
  // 4-point Gauss-Legendre on [0, 1] (nodes (1 -+ x) / 2, weights w / 2)
  const double x1 = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double x2 = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double w1 = (18.0 + std::sqrt(30.0)) / 36.0, w2 = (18.0 - std::sqrt(30.0)) / 36.0;
  const double gl[4][2] = {{0.5 * (1 - x2), 0.5 * w2}, {0.5 * (1 - x1), 0.5 * w1}, {0.5 * (1 + x1), 0.5 * w1},
                           {0.5 * (1 + x2), 0.5 * w2}};
  float glf[4][2];
  for (int i = 0; i < 4; ++i) {
    glf[i][0] = (float)gl[i][0];
    glf[i][1] = (float)gl[i][1];
  }
  NB_TRY_CUDA(cudaMemcpyToSymbol(c_gal_gl, glf, sizeof(glf)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return NAT_BEM_OK;
}
}  // namespace

nat_bem_status galerkin_geometry_build(nat_bem_op* op, const int32_t* T, int64_t nv, cudaStream_t s) {
  NB_TRY(gal_upload_rules());
  Geometry& g = op->geo;
  const int64_t nt = g.n;
  // vertex -> (triangle, local index) lists in increasing triangle order
  std::vector<int> ptr(nv + 1, 0);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) ++ptr[T[3 * t + a] + 1];
  for (int64_t v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
  std::vector<int2> adj(3 * nt);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) adj[fill[T[3 * t + a]]++] = make_int2((int)t, a);
  Galerkin& G = op->gal;
  NB_TRY(dev_alloc_n(&G.adj_ptr, (size_t)nv + 1, s));
  NB_TRY(dev_alloc_n(&G.adj, (size_t)3 * nt, s));
  NB_TRY(dev_alloc_n(&G.curl, (size_t)3 * nt, s));
  NB_TRY(dev_alloc_n(&G.pts.c_hi, (size_t)7 * nt, s));
  NB_TRY(dev_alloc_n(&G.pts.c_lo, (size_t)7 * nt, s));
  NB_TRY(dev_alloc_n(&G.pts.nrm, (size_t)7 * nt, s));
  NB_TRY(dev_alloc_n(&G.pts.qp, (size_t)7 * nt, s));
  G.pts.n = 7 * nt;
  NB_TRY_CUDA(cudaMemcpyAsync(G.adj_ptr, ptr.data(), (nv + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  NB_TRY_CUDA(cudaMemcpyAsync(G.adj, adj.data(), 3 * nt * sizeof(int2), cudaMemcpyHostToDevice, s));
  NB_TRY_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  NB_LAUNCH("gal_geometry", s, k_gal_geometry<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(
      g.tri, g.nrm64, g.area, (int)nt, G.curl, G.pts.c_hi, G.pts.c_lo, G.pts.nrm, G.pts.qp));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

nat_bem_status galerkin_assemble_operators(nat_bem_op* op, cudaStream_t s) {
  NB_TRY(gal_upload_rules());
  const Geometry& g = op->geo;
  const Galerkin& G = op->gal;
  const int nt = (int)g.n, nv = (int)op->n, ldv = (int)g.ld, ldr = (int)op->ldr;
  const float k = (float)op->k;
  // rounds of test triangles: pair blocks (9 + 3 values) and first-stage row sums (3 ldv)
  const double per_row = (double)nt * kGalVals * sizeof(float2) + 3.0 * ldv * sizeof(float2);
  const int chunk = std::max(1, std::min(nt, std::max(512, (int)(kGalScratch / per_row))));
  float2 *partL = nullptr, *partR = nullptr, *P2 = nullptr;
  nat_bem_status st = dev_alloc_n(&partL, (size_t)chunk * nt * 9, s);
  if (st == NAT_BEM_OK) st = dev_alloc_n(&partR, (size_t)chunk * nt * 3, s);
  if (st == NAT_BEM_OK) st = dev_alloc_n(&P2, (size_t)chunk * 3 * ldv, s);
  for (int t0 = 0; t0 < nt && st == NAT_BEM_OK; t0 += chunk) {
    const int t1 = std::min(nt, t0 + chunk);
    const bool last = t1 == nt;
    NB_LAUNCH("gal_regular", s, k_gal_regular<<<dim3((unsigned)((nt + 255) / 256), (unsigned)(t1 - t0)), 256, 0, s>>>(
        g.c_hi, g.c_lo, g.nrm, g.qp, g.vid, G.curl, nt, t0, k, partL, partR));
    const int64_t warps = g.n_near + nt;
    NB_LAUNCH("gal_singular", s, k_gal_singular<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
        g.near_pairs, g.n_near, g.tri, g.nrm64, g.area, g.vid, G.curl, nt, t0, t1, k, partL, partR));
    NB_LAUNCH("gal_rowsum_L", s, k_gal_rowsum_L<<<dim3((unsigned)((nv + 255) / 256), (unsigned)(t1 - t0)), 256, 0, s>>>(
        partL, nt, G.adj_ptr, G.adj, nv, ldv, P2));
    NB_LAUNCH("gal_gather_L", s, k_gal_gather_L<<<dim3((unsigned)((ldv + 255) / 256), (unsigned)nv), 256, 0, s>>>(
        P2, t0, t1, G.adj_ptr, G.adj, nv, ldv, t0 > 0 ? 1 : 0, op->L, last ? bf16_target(op) : nullptr));
    NB_LAUNCH("gal_gather_R", s, k_gal_gather_R<<<dim3((unsigned)((ldr + 255) / 256), (unsigned)nv), 256, 0, s>>>(
        partR, nt, t0, t1, G.adj_ptr, G.adj, ldr, t0 > 0 ? 1 : 0, op->R));
    if (cudaGetLastError() != cudaSuccess) {
      set_error("Galerkin assembly: launch failed");
      st = NAT_BEM_ECUDA;
    }
  }
  dev_free(partL, s);
  dev_free(partR, s);
  dev_free(P2, s);
  if (st == NAT_BEM_OK) st = finish_low_copy(op, s);
  return st;
}

nat_bem_status galerkin_expand(const nat_bem_op* op, const float2* d_p, const float2* d_g, int nrhs,
                               float2** pq, float2** gq, cudaStream_t s) {
  const int64_t nt = op->geo.n, tot = 7 * nt * nrhs;
  *pq = *gq = nullptr;
  NB_TRY(dev_alloc_n(pq, (size_t)tot, s));
  nat_bem_status st = dev_alloc_n(gq, (size_t)tot, s);
  if (st != NAT_BEM_OK) {
    dev_free(*pq, s);
    *pq = nullptr;
    return st;
  }
  NB_LAUNCH("gal_expand", s, k_gal_expand<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      op->geo.vid, (int)nt, (int)op->n, nrhs, d_p, d_g, *pq, *gq));
  NB_CHECK_LAUNCH();
  return NAT_BEM_OK;
}

void galerkin_free(nat_bem_op* op, cudaStream_t s) {
  Galerkin& G = op->gal;
  void* ptrs[] = {G.adj_ptr, G.adj, G.curl, G.pts.c_hi, G.pts.c_lo, G.pts.nrm, G.pts.qp};
  for (void* p : ptrs) dev_free(p, s);
  G = Galerkin{};
}

}  // namespace natbem
