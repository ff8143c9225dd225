// FP64 CPU oracle for the exterior Helmholtz Burton-Miller boundary element solve.
//
// TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct statement of what
// the GPU path computes; it is used by the tests, the smoke check and the bench's CPU
// baseline leg, and by nothing else. The product library never links, loads or calls it,
// and it shares no source, header, table or helper with the CUDA path.
//
// Method (paper Sec. 4, Eq. 6, the Burton-Miller combined boundary integral equation with
// G(x,y) = e^{ikr}/(4 pi r) from Sec. 4.2 and beta = i/k), discretised with piecewise-
// constant (P0) elements and collocation at element centroids (the Neumann data are
// constant per triangle, Sec. 3.4). For collocation element i and source element j:
//
//   L_ij = 1/2 delta_ij - int_j [ dG/dn_y + beta d2G/dn_x dn_y ] dS_y
//   R_ij = -int_j [ G + beta dG/dn_x ] dS_y - (beta/2) delta_ij
//
// and the system is L p = R g (p = surface Dirichlet data, g = Neumann data). This is the
// "A g = B p" system of Sec. 4.1, assembled directly as the two combined matrices.
//
// Integration rules (the paper says only "Gaussian quadrature", Sec. 4.1):
//   * regular pairs: the 7-point degree-5 triangle rule (Radon 1948);
//   * pairs sharing at least one vertex: the same rule on each of the 4^levels congruent
//     sub-triangles of element j;
//   * the self pair: polar coordinates about the centroid, exact radial integration, and
//     Gauss-Legendre in the angle on each edge; the hypersingular term is the Hadamard
//     finite part. On a flat element dG/dn_y = dG/dn_x = 0 on the element itself.
// The linear solve is GMRES (Saad & Schultz 1986) from x0 = 0 with modified Gram-Schmidt
// and complex Givens rotations, stopping on ||b - A x|| / ||b|| (Sec. 6.1 gives tolerance
// 1e-6 and at most 200 iterations for the paper's solver). Field values use the exterior
// representation p(x) = int [ p dG/dn_y - G dp/dn ] dS_y whose surface limit is the first
// line of Eq. 6 (Sec. 3.4: pressure anywhere follows from the Neumann and Dirichlet data).
//
// Normals point out of the body into the fluid (counter-clockwise winding seen from
// outside), which is the orientation the signs of Eq. 6 require.

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <utility>
#include <vector>

// ORACLE_PLANT selects a deliberate mistake for the mutation tests (0 = none). Only a test
// that checks the pins catch it compiles a variant with a nonzero value.
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

namespace {

using cplx = std::complex<double>;
using vec3 = std::array<double, 3>;

const double kPi = 3.14159265358979323846264338327950288;
const cplx kI(0.0, 1.0);

vec3 sub(const vec3& a, const vec3& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
vec3 add(const vec3& a, const vec3& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
vec3 scale(const vec3& a, double s) { return {a[0] * s, a[1] * s, a[2] * s}; }
double dot(const vec3& a, const vec3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
vec3 cross(const vec3& a, const vec3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double norm(const vec3& a) { return std::sqrt(dot(a, a)); }

vec3 load3(const double* p) { return {p[0], p[1], p[2]}; }

struct Tri {
  vec3 a, b, c;
};

Tri triangle_of(const double* V, const int32_t* T, int64_t t) {
  return {load3(V + 3 * T[3 * t]), load3(V + 3 * T[3 * t + 1]), load3(V + 3 * T[3 * t + 2])};
}

// Unit normal (b-a) x (c-a) / |.|, area |.|/2, centroid (a+b+c)/3.
vec3 tri_normal(const Tri& t) {
  vec3 n = cross(sub(t.b, t.a), sub(t.c, t.a));
  return scale(n, 1.0 / norm(n));
}
double tri_area(const Tri& t) { return 0.5 * norm(cross(sub(t.b, t.a), sub(t.c, t.a))); }
vec3 tri_centroid(const Tri& t) { return scale(add(add(t.a, t.b), t.c), 1.0 / 3.0); }

// ---------------------------------------------------------------------------------------
// 7-point degree-5 rule on a triangle (Radon 1948; tabulated by Strang & Fix 1973 and
// Dunavant 1985). Barycentric points and weights that sum to 1 (they multiply the area).
struct QuadPoint {
  double l0, l1, l2, w;
};

std::vector<QuadPoint> radon7() {
  const double s15 = std::sqrt(15.0);
  const double a = (6.0 - s15) / 21.0, wa = (155.0 - s15) / 1200.0;
  const double b = (6.0 + s15) / 21.0, wb = (155.0 + s15) / 1200.0;
  return {
      {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 9.0 / 40.0},
      {a, a, 1.0 - 2.0 * a, wa},
      {a, 1.0 - 2.0 * a, a, wa},
      {1.0 - 2.0 * a, a, a, wa},
      {b, b, 1.0 - 2.0 * b, wb},
      {b, 1.0 - 2.0 * b, b, wb},
      {1.0 - 2.0 * b, b, b, wb},
  };
}

// Uniform midpoint subdivision into 4^levels congruent sub-triangles.
void subdivide(const Tri& t, int levels, std::vector<Tri>& out) {
  if (levels == 0) {
    out.push_back(t);
    return;
  }
  vec3 ab = scale(add(t.a, t.b), 0.5), bc = scale(add(t.b, t.c), 0.5), ca = scale(add(t.c, t.a), 0.5);
  subdivide({t.a, ab, ca}, levels - 1, out);
  subdivide({ab, t.b, bc}, levels - 1, out);
  subdivide({ca, bc, t.c}, levels - 1, out);
  subdivide({ab, bc, ca}, levels - 1, out);
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      // p1 = P_n(z), p0 = P_{n-1}(z); P_n' = n (z P_n - P_{n-1}) / (z^2 - 1)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ---------------------------------------------------------------------------------------
// The four kernels of Eq. 6 at one pair of points (x with normal nx, y with normal ny):
// G = e^{ikr}/(4 pi r) (Sec. 4.2), dG/dn_y, dG/dn_x and d2G/dn_x dn_y, with d = x - y,
// r = |d|, dG/dr = G (ik - 1/r), d2G/dr2 = G (2 - 2ikr - k^2 r^2)/r^2, r_x = d.nx/r,
// r_y = -d.ny/r, dG/dn_y = dG/dr r_y, dG/dn_x = dG/dr r_x and
// d2G/dn_x dn_y = d2G/dr2 r_x r_y - dG/dr (nx.ny + r_x r_y)/r.
struct Kernels {
  cplx G, dGdny, dGdnx, H;
};

Kernels kernels(double k, const vec3& x, const vec3& nx, const vec3& y, const vec3& ny) {
  vec3 d = sub(x, y);
  double r = norm(d);
  cplx G = std::exp(kI * (k * r)) / (4.0 * kPi * r);
  cplx dG = G * (kI * k - 1.0 / r);
  cplx d2G = G * (2.0 - 2.0 * kI * (k * r) - k * k * r * r) / (r * r);
  double rx = dot(d, nx) / r;
  double ry = (ORACLE_PLANT == 2 ? 1.0 : -1.0) * dot(d, ny) / r;
  Kernels out;
  out.G = G;
  out.dGdny = dG * ry;
  out.dGdnx = dG * rx;
  out.H = d2G * rx * ry - dG * (dot(nx, ny) + (ORACLE_PLANT == 3 ? 0.0 : rx * ry)) / r;
  return out;
}

// Integrals over triangle tri (normal ny) of the four kernels at the point x (normal nx),
// with the 7-point rule on each of the 4^levels sub-triangles.
Kernels element_integrals(double k, const vec3& x, const vec3& nx, const Tri& tri, int levels) {
  static const std::vector<QuadPoint> rule = radon7();
  vec3 ny = tri_normal(tri);
  std::vector<Tri> parts;
  subdivide(tri, levels, parts);
  Kernels sum{0.0, 0.0, 0.0, 0.0};
  for (const Tri& s : parts) {
    double area = tri_area(s);
    for (const QuadPoint& q : rule) {
      vec3 y = add(add(scale(s.a, q.l0), scale(s.b, q.l1)), scale(s.c, q.l2));
      Kernels kv = kernels(k, x, nx, y, ny);
      double wa = q.w * area;
      sum.G += wa * kv.G;
      sum.dGdny += wa * kv.dGdny;
      sum.dGdnx += wa * kv.dGdnx;
      sum.H += wa * kv.H;
    }
  }
  return sum;
}

// Self integrals of a flat triangle at its own centroid x, in polar coordinates (rho, theta)
// about x. For each edge at perpendicular distance d_e the boundary is R = d_e / cos(psi),
// psi measured from the perpendicular. With the radial integrals done exactly:
//   S  = int G dS            = (1/4pi) sum_e int (e^{ikR} - 1)/(ik) dpsi
//   FP = f.p. int H dS       = (1/4pi) sum_e int (ik - e^{ikR}/R) dpsi
// On the flat element d.n = 0, so H = -(dG/dr)/r, whose radial integrand
// e^{ik rho}(1 - ik rho)/rho^2 is the derivative of -e^{ik rho}/rho; the Hadamard finite
// part drops the 1/eps term of the lower limit and keeps ik. The angular integral per edge
// is Gauss-Legendre with npts nodes.
void self_integrals(double k, const Tri& tri, int npts, cplx& S, cplx& FP) {
  vec3 x = tri_centroid(tri);
  vec3 n = tri_normal(tri);
  std::vector<double> gx, gw;
  gauss_legendre(npts, gx, gw);
  const vec3 verts[3] = {tri.a, tri.b, tri.c};
  S = 0.0;
  FP = 0.0;
  for (int e = 0; e < 3; ++e) {
    const vec3& P = verts[e];
    const vec3& Q = verts[(e + 1) % 3];
    vec3 u = scale(sub(Q, P), 1.0 / norm(sub(Q, P)));  // edge direction
    vec3 xp = sub(x, P);
    vec3 foot = add(P, scale(u, dot(xp, u)));           // foot of the perpendicular
    vec3 e_dir = sub(foot, x);
    double de = norm(e_dir);
    e_dir = scale(e_dir, 1.0 / de);
    vec3 t_dir = cross(n, e_dir);  // in-plane, 90 degrees counter-clockwise from e_dir
    double psiP = std::atan2(dot(sub(P, x), t_dir), dot(sub(P, x), e_dir));
    double psiQ = std::atan2(dot(sub(Q, x), t_dir), dot(sub(Q, x), e_dir));
    double half = 0.5 * (psiQ - psiP), mid = 0.5 * (psiQ + psiP);
    for (int q = 0; q < npts; ++q) {
      double psi = mid + half * gx[q];
      double R = de / std::cos(psi);
      cplx eikR = std::exp(kI * (k * R));
      double w = half * gw[q];
      S += w * (eikR - 1.0) / (kI * k);
      FP += w * ((ORACLE_PLANT == 4 ? 0.0 : 1.0) * kI * k - eikR / R);
    }
  }
  S /= 4.0 * kPi;
  FP /= 4.0 * kPi;
}

bool shares_vertex(const int32_t* T, int64_t i, int64_t j) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (T[3 * i + a] == T[3 * j + b]) return true;
  return false;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (nthreads == 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> pool;
  std::atomic_int64_t next(0);
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& th : pool) th.join();
}

// One row of the two Burton-Miller matrices (collocation element i).
void assemble_row(const double* V, const int32_t* T, int64_t nt, double k, int adj_levels,
                  int self_pts, int64_t i, cplx* Lrow, cplx* Rrow) {
  const cplx beta = kI / k;
  Tri ti = triangle_of(V, T, i);
  vec3 x = tri_centroid(ti), nx = tri_normal(ti);
  for (int64_t j = 0; j < nt; ++j) {
    if (j == i) {
      cplx S, FP;
      self_integrals(k, ti, self_pts, S, FP);
      Lrow[j] = 0.5 - beta * FP;
      Rrow[j] = -S - (ORACLE_PLANT == 1 ? 0.0 : 0.5) * beta;
      continue;
    }
    int levels = shares_vertex(T, i, j) ? adj_levels : 0;
    Kernels I = element_integrals(k, x, nx, triangle_of(V, T, j), levels);
    Lrow[j] = -(I.dGdny + beta * I.H);
    Rrow[j] = -(I.G + beta * I.dGdnx);
  }
}

}  // namespace

extern "C" {

// Mesh checks: indices in range, finite coordinates, no zero-area triangle, closed and
// consistently oriented (every directed edge used once and its reverse once), positive
// enclosed volume (outward normals). Returns 0 when valid, else a nonzero code.
int oracle_validate_mesh(const double* V, int64_t nv, const int32_t* T, int64_t nt) {
  if (nv <= 0 || nt <= 0) return 1;
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(V[i])) return 2;
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (T[i] < 0 || T[i] >= nv) return 3;
  std::map<std::pair<int32_t, int32_t>, int> directed;
  double vol6 = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    Tri tr = triangle_of(V, T, t);
    if (!(tri_area(tr) > 0.0)) return 4;
    for (int e = 0; e < 3; ++e) directed[{T[3 * t + e], T[3 * t + (e + 1) % 3]}] += 1;
    vol6 += dot(tr.a, cross(tr.b, tr.c));
  }
  for (const auto& kv : directed) {
    if (kv.second != 1) return 5;
    auto rev = directed.find({kv.first.second, kv.first.first});
    if (rev == directed.end() || rev->second != 1) return 5;
  }
  if (!(vol6 > 0.0)) return 6;
  return 0;
}

void oracle_geometry(const double* V, const int32_t* T, int64_t nt, double* cen, double* nrm,
                     double* area) {
  for (int64_t t = 0; t < nt; ++t) {
    Tri tr = triangle_of(V, T, t);
    vec3 c = tri_centroid(tr), n = tri_normal(tr);
    for (int d = 0; d < 3; ++d) {
      cen[3 * t + d] = c[d];
      nrm[3 * t + d] = n[d];
    }
    area[t] = tri_area(tr);
  }
}

void oracle_quad_rule(double* bary, double* w) {
  std::vector<QuadPoint> r = radon7();
  for (int q = 0; q < 7; ++q) {
    bary[3 * q] = r[q].l0;
    bary[3 * q + 1] = r[q].l1;
    bary[3 * q + 2] = r[q].l2;
    w[q] = r[q].w;
  }
}

void oracle_gauss_legendre(int n, double* x, double* w) {
  std::vector<double> gx, gw;
  gauss_legendre(n, gx, gw);
  for (int i = 0; i < n; ++i) {
    x[i] = gx[i];
    w[i] = gw[i];
  }
}

// out: 4 complex (interleaved re, im): G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y.
void oracle_kernels(double k, const double* x, const double* nx, const double* y,
                    const double* ny, double* out) {
  Kernels kv = kernels(k, load3(x), load3(nx), load3(y), load3(ny));
  const cplx v[4] = {kv.G, kv.dGdny, kv.dGdnx, kv.H};
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = v[i].real();
    out[2 * i + 1] = v[i].imag();
  }
}

// out: 4 complex: the integrals of G, dG/dn_y, dG/dn_x, H over triangle tri (3x3, rows are
// vertices) at the point x with normal nx, using 4^levels sub-triangles.
void oracle_element_integrals(double k, const double* x, const double* nx, const double* tri,
                              int levels, double* out) {
  Tri t{load3(tri), load3(tri + 3), load3(tri + 6)};
  Kernels I = element_integrals(k, load3(x), load3(nx), t, levels);
  const cplx v[4] = {I.G, I.dGdny, I.dGdnx, I.H};
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = v[i].real();
    out[2 * i + 1] = v[i].imag();
  }
}

// out: 2 complex: S (self single layer) and FP (finite-part self hypersingular integral).
void oracle_self_integrals(double k, const double* tri, int npts, double* out) {
  Tri t{load3(tri), load3(tri + 3), load3(tri + 6)};
  cplx S, FP;
  self_integrals(k, t, npts, S, FP);
  out[0] = S.real();
  out[1] = S.imag();
  out[2] = FP.real();
  out[3] = FP.imag();
}

// Rows `rows[0..nrows)` of L and R, each nt complex (interleaved), row after row.
int oracle_assemble_rows(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k,
                         int adj_levels, int self_pts, const int64_t* rows, int64_t nrows,
                         double* L, double* R, int nthreads) {
  if (!(k > 0.0) || nt <= 0 || nv <= 0) return 1;
  parallel_for(nrows, nthreads, [&](int64_t r) {
    assemble_row(V, T, nt, k, adj_levels, self_pts, rows[r],
                 reinterpret_cast<cplx*>(L) + r * nt, reinterpret_cast<cplx*>(R) + r * nt);
  });
  return 0;
}

// Full L and R (nt x nt complex, row-major, interleaved re/im).
int oracle_assemble(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k,
                    int adj_levels, int self_pts, double* L, double* R, int nthreads) {
  if (!(k > 0.0) || nt <= 0 || nv <= 0) return 1;
  parallel_for(nt, nthreads, [&](int64_t i) {
    assemble_row(V, T, nt, k, adj_levels, self_pts, i, reinterpret_cast<cplx*>(L) + i * nt,
                 reinterpret_cast<cplx*>(R) + i * nt);
  });
  return 0;
}

// y = A x for a dense n x n complex matrix (row-major).
void oracle_matvec(const double* A, int64_t n, const double* x, double* y, int nthreads) {
  const cplx* a = reinterpret_cast<const cplx*>(A);
  const cplx* xv = reinterpret_cast<const cplx*>(x);
  cplx* yv = reinterpret_cast<cplx*>(y);
  parallel_for(n, nthreads, [&](int64_t i) {
    cplx s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += a[i * n + j] * xv[j];
    yv[i] = s;
  });
}

// GMRES from x0 = 0, modified Gram-Schmidt Arnoldi, complex Givens rotations, unrestarted.
// Stops when the Arnoldi residual estimate |g_{j+1}| <= tol ||b|| or after maxit steps.
// Returns 0 on convergence, 3 when maxit was reached (x holds the last iterate).
int oracle_gmres(const double* A, int64_t n, const double* b, double tol, int maxit, double* x,
                 int* iters, double* relres, int nthreads) {
  const cplx* bv = reinterpret_cast<const cplx*>(b);
  cplx* xv = reinterpret_cast<cplx*>(x);
  double bnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) bnorm += std::norm(bv[i]);
  bnorm = std::sqrt(bnorm);
  for (int64_t i = 0; i < n; ++i) xv[i] = 0.0;
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) return 0;
  const int m = maxit;
  std::vector<std::vector<cplx>> Vb;
  Vb.emplace_back(n);
  for (int64_t i = 0; i < n; ++i) Vb[0][i] = bv[i] / bnorm;
  std::vector<std::vector<cplx>> H(m + 1, std::vector<cplx>(m, 0.0));
  std::vector<double> cs(m, 0.0);
  std::vector<cplx> sn(m, 0.0), g(m + 1, 0.0);
  g[0] = bnorm;
  int j = 0;
  double res = bnorm;
  std::vector<cplx> w(n);
  for (j = 0; j < m; ++j) {
    oracle_matvec(A, n, reinterpret_cast<const double*>(Vb[j].data()),
                  reinterpret_cast<double*>(w.data()), nthreads);
    for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
      cplx h = 0.0;
      for (int64_t r = 0; r < n; ++r) h += std::conj(Vb[i][r]) * w[r];
      H[i][j] = h;
      for (int64_t r = 0; r < n; ++r) w[r] -= h * Vb[i][r];
    }
    double hn = 0.0;
    for (int64_t r = 0; r < n; ++r) hn += std::norm(w[r]);
    hn = std::sqrt(hn);
    H[j + 1][j] = hn;
    for (int i = 0; i < j; ++i) {  // previous rotations on the new column
      cplx t = cs[i] * H[i][j] + sn[i] * H[i + 1][j];
      H[i + 1][j] = -std::conj(sn[i]) * H[i][j] + cs[i] * H[i + 1][j];
      H[i][j] = t;
    }
    cplx h1 = H[j][j], h2 = H[j + 1][j];
    double rho = std::sqrt(std::norm(h1) + std::norm(h2));
    if (std::abs(h1) == 0.0) {
      cs[j] = 0.0;
      sn[j] = 1.0;
    } else {
      cs[j] = std::abs(h1) / rho;
      sn[j] = (h1 / std::abs(h1)) * std::conj(h2) / rho;
    }
    H[j][j] = cs[j] * h1 + sn[j] * h2;
    H[j + 1][j] = 0.0;
    g[j + 1] = -std::conj(sn[j]) * g[j];
    g[j] = cs[j] * g[j];
    res = std::abs(g[j + 1]);
    bool done = res <= tol * bnorm || hn == 0.0;
    if (!done && j + 1 < m) {
      Vb.emplace_back(n);
      for (int64_t r = 0; r < n; ++r) Vb[j + 1][r] = w[r] / hn;
    }
    if (done) {
      ++j;
      break;
    }
  }
  int kdim = std::min(j, m);
  std::vector<cplx> y(kdim);
  for (int i = kdim - 1; i >= 0; --i) {  // back substitution on the rotated Hessenberg
    cplx s = g[i];
    for (int c = i + 1; c < kdim; ++c) s -= H[i][c] * y[c];
    y[i] = s / H[i][i];
  }
  for (int i = 0; i < kdim; ++i)
    for (int64_t r = 0; r < n; ++r) xv[r] += y[i] * Vb[i][r];
  *iters = kdim;
  *relres = res / bnorm;
  return res <= tol * bnorm ? 0 : 3;
}

// Field at points pts (m x 3): out[q] = sum_j int_j [ p_j dG/dn_y - g_j G ](pts_q, y) dS_y
// with the 7-point rule on each element.
int oracle_eval(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k,
                const double* pts, int64_t m, const double* p, const double* g, double* out,
                int nthreads) {
  if (!(k > 0.0) || nt <= 0 || nv <= 0 || m < 0) return 1;
  const cplx* pv = reinterpret_cast<const cplx*>(p);
  const cplx* gv = reinterpret_cast<const cplx*>(g);
  cplx* o = reinterpret_cast<cplx*>(out);
  const vec3 zero = {0.0, 0.0, 0.0};
  parallel_for(m, nthreads, [&](int64_t q) {
    vec3 x = load3(pts + 3 * q);
    cplx s = 0.0;
    for (int64_t j = 0; j < nt; ++j) {
      Kernels I = element_integrals(k, x, zero, triangle_of(V, T, j), 0);
      s += pv[j] * I.dGdny - gv[j] * I.G;
    }
    o[q] = s;
  });
  return 0;
}

// One whole solve as the CPU baseline runs it: assemble L and R, b = R g, GMRES, field.
// times[0..3] = seconds spent in assembly, right-hand side, solve and field evaluation.
int oracle_bem_solve(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k,
                     int adj_levels, int self_pts, const double* g, const double* pts,
                     int64_t m, double tol, int maxit, int nthreads, double* p_out,
                     double* field_out, int* iters, double* relres, double* times) {
  auto now = []() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
  };
  std::vector<double> L(2 * nt * nt), R(2 * nt * nt), b(2 * nt);
  double t0 = now();
  int rc = oracle_assemble(V, nv, T, nt, k, adj_levels, self_pts, L.data(), R.data(), nthreads);
  if (rc) return rc;
  double t1 = now();
  oracle_matvec(R.data(), nt, g, b.data(), nthreads);
  double t2 = now();
  int st = oracle_gmres(L.data(), nt, b.data(), tol, maxit, p_out, iters, relres, nthreads);
  double t3 = now();
  oracle_eval(V, nv, T, nt, k, pts, m, p_out, g, field_out, nthreads);
  double t4 = now();
  times[0] = t1 - t0;
  times[1] = t2 - t1;
  times[2] = t3 - t2;
  times[3] = t4 - t3;
  return st;
}

// ---------------------------------------------------------------------------------------
// BEM-MC (paper Sec. 4.1.1 and 4.2): the conventional boundary integral equation (beta = 0 in
// Eq. 6) with the surface integral replaced by a Monte-Carlo sum over M sample points y_j of
// uniform density on the surface (1/q = |Gamma|), and collocated at the same samples:
//   1/2 p_i = sum_{j != i} w [ dG/dn_y(y_i, y_j) p_j - G(y_i, y_j) g_j ] - (eps/2) g_i.
// The sample's own neighbourhood is the disk of radius eps about y_i: with one sample at its
// centre, the single layer over the disk is 2 pi eps/(4 pi) g_i = (eps/2) g_i, and the double
// layer vanishes there (d is perpendicular to the normal on the flat disk). The paper gives no
// value for eps; the reading taken is the sample's share of the surface, pi eps^2 = |Gamma|/M,
// so the other samples share |Gamma| - pi eps^2 and each weighs
// w = (|Gamma| - pi eps^2)/(M - 1) = |Gamma|/M. Normals are outward (the paper's equation is
// written with the opposite normal, which flips both terms). In the L p = R g form:
//   L_ij = 1/2 delta_ij - w dG/dn_y(y_i, y_j) (1 - delta_ij)
//   R_ij = -w G(y_i, y_j) (1 - delta_ij) - (eps/2) delta_ij.
// The field at x off the surface is the same Monte-Carlo sum of the exterior representation:
//   p(x) = sum_j w [ p_j dG/dn_y(x, y_j) - g_j G(x, y_j) ].

// L and R (M x M complex, row-major, interleaved re/im) for samples Y (M x 3) with unit
// outward normals N (M x 3) on a surface of area `area`.
int oracle_mc_assemble(const double* Y, const double* N, int64_t M, double area, double k,
                       double* L, double* R, int nthreads) {
  if (!(k > 0.0) || M < 2 || !(area > 0.0)) return 1;
  const double w = area / (double)M;
  const double eps = std::sqrt(area / (kPi * (double)M));
  cplx* Lc = reinterpret_cast<cplx*>(L);
  cplx* Rc = reinterpret_cast<cplx*>(R);
  parallel_for(M, nthreads, [&](int64_t i) {
    const vec3 x = load3(Y + 3 * i), nx = load3(N + 3 * i);
    for (int64_t j = 0; j < M; ++j) {
      if (j == i) {
        Lc[i * M + j] = 0.5;
        Rc[i * M + j] = ORACLE_PLANT == 5 ? 0.5 * eps : (ORACLE_PLANT == 7 ? 0.0 : -0.5 * eps);
        continue;
      }
      Kernels kv = kernels(k, x, nx, load3(Y + 3 * j), load3(N + 3 * j));
      Lc[i * M + j] = -w * (ORACLE_PLANT == 6 ? kv.dGdnx : kv.dGdny);
      Rc[i * M + j] = -w * kv.G;
    }
  });
  return 0;
}

// Field at points pts (Q x 3) from the samples' Dirichlet (p) and Neumann (g) values.
int oracle_mc_eval(const double* Y, const double* N, int64_t M, double area, double k,
                   const double* pts, int64_t Q, const double* p, const double* g, double* out,
                   int nthreads) {
  if (!(k > 0.0) || M < 1 || !(area > 0.0) || Q < 0) return 1;
  const double w = area / (double)M;
  const cplx* pv = reinterpret_cast<const cplx*>(p);
  const cplx* gv = reinterpret_cast<const cplx*>(g);
  cplx* o = reinterpret_cast<cplx*>(out);
  const vec3 zero = {0.0, 0.0, 0.0};
  parallel_for(Q, nthreads, [&](int64_t q) {
    const vec3 x = load3(pts + 3 * q);
    cplx s = 0.0;
    for (int64_t j = 0; j < M; ++j) {
      Kernels kv = kernels(k, x, zero, load3(Y + 3 * j), load3(N + 3 * j));
      s += w * (pv[j] * kv.dGdny + (ORACLE_PLANT == 8 ? 1.0 : -1.0) * gv[j] * kv.G);
    }
    o[q] = s;
  });
  return 0;
}

// ---------------------------------------------------------------------------------------
// Far-field pattern, the leading term Phi_1 of the FFAT expansion |p(x)| = sum_i Phi_i / r^i
// (paper Sec. 3.1, the equation after the FFAT citation): as |x| = r -> infinity along the unit
// direction d, G(x, y) -> e^{ikr}/(4 pi r) e^{-ik d.y} and dG/dn_y -> that times (-ik d.n_y),
// so F(d) = lim r e^{-ikr} p(r d) = (1/4pi) int [ p (-ik d.n_y) - g ] e^{-ik d.y} dS_y,
// with the 7-point rule on every element (the rule of the field evaluation).
int oracle_far_field(const double* V, int64_t nv, const int32_t* T, int64_t nt, double k,
                     const double* dirs, int64_t nd, const double* p, const double* g, double* out,
                     int nthreads) {
  if (!(k > 0.0) || nt <= 0 || nv <= 0 || nd < 0) return 1;
  const cplx* pv = reinterpret_cast<const cplx*>(p);
  const cplx* gv = reinterpret_cast<const cplx*>(g);
  cplx* o = reinterpret_cast<cplx*>(out);
  const std::vector<QuadPoint> rule = radon7();
  parallel_for(nd, nthreads, [&](int64_t q) {
    const vec3 d = load3(dirs + 3 * q);
    cplx s = 0.0;
    for (int64_t j = 0; j < nt; ++j) {
      const Tri t = triangle_of(V, T, j);
      const vec3 n = tri_normal(t);
      const double A = tri_area(t);
      cplx e = 0.0;
      for (const QuadPoint& qp : rule) {
        const vec3 y = add(add(scale(t.a, qp.l0), scale(t.b, qp.l1)), scale(t.c, qp.l2));
        e += qp.w * A * std::exp(-kI * (k * dot(d, y)));
      }
      s += (pv[j] * ((ORACLE_PLANT == 9 ? kI : -kI) * k * dot(d, n)) - gv[j]) * e;
    }
    o[q] = s / (4.0 * kPi);
  });
  return 0;
}

// The same far field for a Monte-Carlo op: samples Y with normals N, each of weight area/M.
int oracle_mc_far_field(const double* Y, const double* N, int64_t M, double area, double k,
                        const double* dirs, int64_t nd, const double* p, const double* g,
                        double* out, int nthreads) {
  if (!(k > 0.0) || M < 1 || !(area > 0.0) || nd < 0) return 1;
  const double w = area / (double)M;
  const cplx* pv = reinterpret_cast<const cplx*>(p);
  const cplx* gv = reinterpret_cast<const cplx*>(g);
  cplx* o = reinterpret_cast<cplx*>(out);
  parallel_for(nd, nthreads, [&](int64_t q) {
    const vec3 d = load3(dirs + 3 * q);
    cplx s = 0.0;
    for (int64_t j = 0; j < M; ++j) {
      const vec3 y = load3(Y + 3 * j), n = load3(N + 3 * j);
      s += w * (pv[j] * (-kI * k * dot(d, n)) - gv[j]) * std::exp(-kI * (k * dot(d, y)));
    }
    o[q] = s / (4.0 * kPi);
  });
  return 0;
}

int oracle_hardware_threads(void) { return (int)std::thread::hardware_concurrency(); }

}  // extern "C"
