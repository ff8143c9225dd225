// Poisson-disk surface sampling for the Monte-Carlo BEM (paper Sec. 4.2: samples that cover the
// surface evenly, drawn in parallel on the GPU after Bowers et al. 2010).
//
//   candidates  per draw (u0, u1, u2): the triangle whose cumulative-area interval holds
//               u0 * A, the point with barycentric (1 - sqrt(u1), sqrt(u1)(1 - u2), sqrt(u1) u2);
//               pushed onto its grid cell's list (cell size h = r / sqrt(3): one sample per cell)
//   27 phases   (i, j, k) mod 3; every cell of a phase accepts its lowest-index candidate with
//               no accepted sample closer than r in the 5 x 5 x 5 cells around it. Cells of one
//               phase are three or more cells apart, so a phase runs its cells in parallel and
//               the result equals the sequential definition, whatever the list order.
// FP64 throughout; products and sums with explicit round-to-nearest intrinsics (no contraction),
// so candidate positions and the distance tests are the same on every machine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace natbem {

namespace {
constexpr int64_t kPsMaxCells = (int64_t)1 << 28;

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
}  // namespace

struct PsGrid {
  double lox, loy, loz, h;
  int nx, ny, nz;
};

__device__ __forceinline__ int ps_clamp(int v, int n) { return v < 0 ? 0 : v >= n ? n - 1 : v; }

// Candidate i: position, normal, and the push onto its cell's list.
__global__ void k_ps_candidates(const double* __restrict__ V, const int32_t* __restrict__ T,
                                const double* __restrict__ cum, int nt, const double* __restrict__ u, int m,
                                PsGrid g, double* __restrict__ x, double* __restrict__ nrm,
                                int* __restrict__ head, int* __restrict__ next, int64_t* __restrict__ occ,
                                int* __restrict__ n_occ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double u0 = u[3 * (size_t)i], u1 = u[3 * (size_t)i + 1], u2 = u[3 * (size_t)i + 2];
  // first triangle with cumulative area > u0 * A
  const double v = dm(u0, cum[nt - 1]);
  int lo = 0, hi = nt;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cum[mid] > v) hi = mid;
    else lo = mid + 1;
  }
  const int t = min(lo, nt - 1);
  const double* a = V + 3 * (size_t)T[3 * (size_t)t];
  const double* b = V + 3 * (size_t)T[3 * (size_t)t + 1];
  const double* c = V + 3 * (size_t)T[3 * (size_t)t + 2];
  const double s = __dsqrt_rn(u1);
  const double b0 = ds(1.0, s), b1 = dm(s, ds(1.0, u2)), b2 = dm(s, u2);
  double p[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) p[d] = da(da(dm(b0, a[d]), dm(b1, b[d])), dm(b2, c[d]));
  const double e1[3] = {ds(b[0], a[0]), ds(b[1], a[1]), ds(b[2], a[2])};
  const double e2[3] = {ds(c[0], a[0]), ds(c[1], a[1]), ds(c[2], a[2])};
  const double cr[3] = {ds(dm(e1[1], e2[2]), dm(e1[2], e2[1])), ds(dm(e1[2], e2[0]), dm(e1[0], e2[2])),
                        ds(dm(e1[0], e2[1]), dm(e1[1], e2[0]))};
  const double len = __dsqrt_rn(da(da(dm(cr[0], cr[0]), dm(cr[1], cr[1])), dm(cr[2], cr[2])));
  const double twoA = dm(2.0, dm(0.5, len));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[3 * (size_t)i + d] = p[d];
    nrm[3 * (size_t)i + d] = __ddiv_rn(cr[d], twoA);
  }
  const int ci = ps_clamp((int)floor(__ddiv_rn(ds(p[0], g.lox), g.h)), g.nx);
  const int cj = ps_clamp((int)floor(__ddiv_rn(ds(p[1], g.loy), g.h)), g.ny);
  const int ck = ps_clamp((int)floor(__ddiv_rn(ds(p[2], g.loz), g.h)), g.nz);
  const int64_t cell = ((int64_t)ci * g.ny + cj) * g.nz + ck;
  const int prev = atomicExch(&head[cell], i);
  next[i] = prev;
  if (prev < 0) occ[atomicAdd(n_occ, 1)] = cell;  // first candidate of the cell: list the cell once
}

// One phase: a warp per occupied cell of the phase. Lane l holds the accepted samples of the
// neighbour cells l, l + 32, l + 64, l + 96 of the 5 x 5 x 5 block (none of them changes during
// the phase: same-phase cells are three or more cells apart); the warp walks the cell's list
// and keeps the lowest index that every lane finds at distance >= r from its samples.
__global__ void __launch_bounds__(256) k_ps_phase(PsGrid g, int phase, double r2, const double* __restrict__ x,
                                                  const int* __restrict__ head, const int* __restrict__ next,
                                                  const int64_t* __restrict__ occ, const int* __restrict__ n_occ,
                                                  int* __restrict__ taken) {
  const int lane = threadIdx.x & 31;
  const int n = *n_occ;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int64_t base = (int64_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
       base += (int64_t)warps * 32) {
    int64_t mine = -1;
    int ci = 0, cj = 0, ck = 0;
    if (base + lane < n) {
      const int64_t c = occ[base + lane];
      ck = (int)(c % g.nz);
      cj = (int)((c / g.nz) % g.ny);
      ci = (int)(c / ((int64_t)g.ny * g.nz));
      if ((ci % 3) * 9 + (cj % 3) * 3 + (ck % 3) == phase) mine = c;
    }
    unsigned todo = __ballot_sync(0xffffffffu, mine >= 0);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t cell = __shfl_sync(0xffffffffu, mine, src);
      const int cx = __shfl_sync(0xffffffffu, ci, src), cy = __shfl_sync(0xffffffffu, cj, src),
                cz = __shfl_sync(0xffffffffu, ck, src);
      double nx[4], ny[4], nz[4];
      bool has[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = lane + 32 * q;
        has[q] = false;
        nx[q] = ny[q] = nz[q] = 0.0;
        if (t < 125) {
          const int a = cx + t / 25 - 2, b = cy + (t / 5) % 5 - 2, c = cz + t % 5 - 2;
          if (a >= 0 && a < g.nx && b >= 0 && b < g.ny && c >= 0 && c < g.nz) {
            const int sidx = taken[((int64_t)a * g.ny + b) * g.nz + c];
            if (sidx >= 0) {
              has[q] = true;
              nx[q] = x[3 * (size_t)sidx];
              ny[q] = x[3 * (size_t)sidx + 1];
              nz[q] = x[3 * (size_t)sidx + 2];
            }
          }
        }
      }
      int best = -1;
      for (int i = head[cell]; i >= 0; i = next[i]) {
        if (best >= 0 && i > best) continue;
        const double xi = x[3 * (size_t)i], yi = x[3 * (size_t)i + 1], zi = x[3 * (size_t)i + 2];
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (has[q]) {
            const double dx = ds(xi, nx[q]), dy = ds(yi, ny[q]), dz = ds(zi, nz[q]);
            if (da(da(dm(dx, dx), dm(dy, dy)), dm(dz, dz)) < r2) ok = false;
          }
        }
        if (__all_sync(0xffffffffu, ok)) best = i;
      }
      if (lane == 0 && best >= 0) taken[cell] = best;
    }
  }
}

__global__ void k_ps_flags(const int* __restrict__ taken, const int64_t* __restrict__ occ,
                           const int* __restrict__ n_occ, unsigned char* __restrict__ flag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < *n_occ) {
    const int s = taken[occ[j]];
    if (s >= 0) flag[s] = 1;
  }
}

__global__ void k_ps_gather(const int* __restrict__ idx, int count, const double* __restrict__ x,
                            const double* __restrict__ nrm, double* __restrict__ pts, double* __restrict__ nout) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const int i = idx[j];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    pts[3 * (size_t)j + d] = x[3 * (size_t)i + d];
    nout[3 * (size_t)j + d] = nrm[3 * (size_t)i + d];
  }
}

}  // namespace natbem

using namespace natbem;

extern "C" nat_bem_status nat_bem_poisson_sample(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                                                 double radius, const double* u, int64_t m, int64_t cap,
                                                 int64_t* idx_out, double* pts_out, double* normals_out,
                                                 int64_t* count, void* cuda_stream) {
  try {
    clear_error();
    if (!verts || !tris || !u || !count || nv <= 0 || nt <= 0 || m < 0 || cap < 0 ||
        m > ((int64_t)1 << 31) - 1 || nt > ((int64_t)1 << 31) - 1 || !(radius > 0.0) || !std::isfinite(radius) ||
        (cap > 0 && (!pts_out || !normals_out))) {
      set_error("nat_bem_poisson_sample: bad arguments");
      return NAT_BEM_EINVAL;
    }
    *count = 0;
    if (m == 0) return NAT_BEM_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<double> hV(3 * nv);
    std::vector<int32_t> hT(3 * nt);
    NB_TRY_CUDA(cudaMemcpyAsync(hV.data(), verts, 3 * nv * sizeof(double), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaMemcpyAsync(hT.data(), tris, 3 * nt * sizeof(int32_t), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < 3 * nt; ++i)
      if (hT[i] < 0 || hT[i] >= nv) {
        set_error("nat_bem_poisson_sample: triangle index out of range");
        return NAT_BEM_EINVAL;
      }
    // cumulative areas (sequential, FP64), the bounding box and the grid
    std::vector<double> cum(nt);
    double acc = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
      const double* a = &hV[3 * hT[3 * t]];
      const double* b = &hV[3 * hT[3 * t + 1]];
      const double* c = &hV[3 * hT[3 * t + 2]];
      const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      const double cx = e1[1] * e2[2] - e1[2] * e2[1];
      const double cy = e1[2] * e2[0] - e1[0] * e2[2];
      const double cz = e1[0] * e2[1] - e1[1] * e2[0];
      const double area = 0.5 * std::sqrt((cx * cx + cy * cy) + cz * cz);
      if (!(area > 0.0) || !std::isfinite(area)) {
        set_error("nat_bem_poisson_sample: degenerate or non-finite triangle " + std::to_string(t));
        return NAT_BEM_EINVAL;
      }
      acc = acc + area;
      cum[t] = acc;
    }
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = hV[d];
    for (int64_t v = 0; v < nv; ++v)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], hV[3 * v + d]);
        hi[d] = std::max(hi[d], hV[3 * v + d]);
      }
    PsGrid g;
    g.lox = lo[0];
    g.loy = lo[1];
    g.loz = lo[2];
    g.h = radius / std::sqrt(3.0);
    double fd[3];
    for (int d = 0; d < 3; ++d) fd[d] = std::floor((hi[d] - lo[d]) / g.h) + 1.0;
    if (!(fd[0] * fd[1] * fd[2] <= (double)kPsMaxCells)) {
      set_error("nat_bem_poisson_sample: radius too small for the mesh's extent (more than 2^28 grid cells)");
      return NAT_BEM_EINVAL;
    }
    g.nx = (int)fd[0];
    g.ny = (int)fd[1];
    g.nz = (int)fd[2];
    const int64_t cells = (int64_t)g.nx * g.ny * g.nz;

    double *dV = nullptr, *dcum = nullptr, *dx = nullptr, *dn = nullptr;
    int32_t* dT = nullptr;
    const double* du = nullptr;
    double* tu = nullptr;
    int *head = nullptr, *next = nullptr, *taken = nullptr, *didx = nullptr, *n_occ = nullptr;
    int64_t* occ = nullptr;
    unsigned char* flag = nullptr;
    double *tp = nullptr, *tn = nullptr;
    auto cleanup = [&]() {
      void* ptrs[] = {dV, dcum, dx, dn, dT, tu, head, next, taken, didx, flag, tp, tn, occ, n_occ};
      for (void* p : ptrs) dev_free(p, s);
    };
    nat_bem_status st = NAT_BEM_OK;
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dV, (size_t)(3 * nv), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dT, (size_t)(3 * nt), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dcum, (size_t)nt, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dx, (size_t)(3 * m), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dn, (size_t)(3 * m), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&head, (size_t)cells, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&taken, (size_t)cells, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&next, (size_t)m, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&flag, (size_t)m, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&occ, (size_t)m, s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&n_occ, 1, s);
    if (st == NAT_BEM_OK) st = to_device(u, (size_t)(3 * m), s, &du, &tu);
    if (st != NAT_BEM_OK) {
      cleanup();
      return st;
    }
    cudaError_t e = cudaMemcpyAsync(dV, hV.data(), 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, hT.data(), 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dcum, cum.data(), nt * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(head, 0xff, (size_t)cells * sizeof(int), s);   // -1
    if (e == cudaSuccess) e = cudaMemsetAsync(taken, 0xff, (size_t)cells * sizeof(int), s);  // -1
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, (size_t)m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_occ, 0, sizeof(int), s);
    if (e != cudaSuccess) {
      set_error(std::string("nat_bem_poisson_sample: ") + cudaGetErrorString(e));
      cleanup();
      return NAT_BEM_ECUDA;
    }
    NB_LAUNCH("ps_candidates", s, k_ps_candidates<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
        dV, dT, dcum, (int)nt, du, (int)m, g, dx, dn, head, next, occ, n_occ));
    const double r2 = radius * radius;
    // the occupied cells number at most m: 8 warps of 32 cells per block, at most 8 blocks per SM
    const unsigned pblocks = (unsigned)std::min<int64_t>((m + 255) / 256, 152 * 8);
    for (int ph = 0; ph < 27; ++ph)
      NB_LAUNCH("ps_phase", s, k_ps_phase<<<pblocks, 256, 0, s>>>(g, ph, r2, dx, head, next, occ, n_occ, taken));
    NB_LAUNCH("ps_flags", s, k_ps_flags<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(taken, occ, n_occ, flag));
    std::vector<unsigned char> hflag(m);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag.data(), flag, (size_t)m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("nat_bem_poisson_sample: ") + cudaGetErrorString(e));
      cleanup();
      return NAT_BEM_ECUDA;
    }
    std::vector<int> order;
    for (int64_t i = 0; i < m; ++i)
      if (hflag[i]) order.push_back((int)i);
    *count = (int64_t)order.size();
    if (idx_out) {
      const int64_t k = std::min<int64_t>(cap, (int64_t)order.size());
      for (int64_t j = 0; j < k; ++j) idx_out[j] = order[j];
    }
    if ((int64_t)order.size() > cap) {
      set_error("nat_bem_poisson_sample: " + std::to_string(order.size()) + " samples exceed cap " + std::to_string(cap));
      cleanup();
      return NAT_BEM_EINVAL;
    }
    if (!order.empty()) {
      const int k = (int)order.size();
      const bool pdev = is_device_pointer(pts_out), ndev = is_device_pointer(normals_out);
      double* dp = pts_out;
      double* dnout = normals_out;
      st = dev_alloc_n(&didx, (size_t)k, s);
      if (st == NAT_BEM_OK && !pdev) st = dev_alloc_n(&tp, (size_t)(3 * k), s);
      if (st == NAT_BEM_OK && !ndev) st = dev_alloc_n(&tn, (size_t)(3 * k), s);
      if (st != NAT_BEM_OK) {
        cleanup();
        return st;
      }
      if (!pdev) dp = tp;
      if (!ndev) dnout = tn;
      e = cudaMemcpyAsync(didx, order.data(), (size_t)k * sizeof(int), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        NB_LAUNCH("ps_gather", s, k_ps_gather<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(didx, k, dx, dn, dp, dnout));
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && !pdev) e = cudaMemcpyAsync(pts_out, tp, (size_t)(3 * k) * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && !ndev)
        e = cudaMemcpyAsync(normals_out, tn, (size_t)(3 * k) * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("nat_bem_poisson_sample: ") + cudaGetErrorString(e));
        cleanup();
        return NAT_BEM_ECUDA;
      }
    }
    cleanup();
    return NAT_BEM_OK;
  } catch (...) {
    set_error("internal error in nat_bem_poisson_sample");
    return NAT_BEM_ECUDA;
  }
}
