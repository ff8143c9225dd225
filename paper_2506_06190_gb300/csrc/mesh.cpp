// Host-side mesh checks and the list of element pairs integrated in FP64 (self pairs and
// pairs that share a vertex). The boundary integral equation of Sec. 4, Eq. 6 needs a closed
// surface with outward normals; this file rejects anything else before device work starts.
#include <algorithm>
#include <cmath>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace natbem {

namespace {

struct V3 {
  double x, y, z;
};
V3 vget(const double* V, int32_t i) { return {V[3 * i], V[3 * i + 1], V[3 * i + 2]}; }
V3 vsub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 vcross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

}  // namespace

nat_bem_status validate_mesh_host(const double* V, int64_t nv, const int32_t* T, int64_t nt) {
  if (nv <= 0 || nt <= 0) {
    set_error("mesh: need nv > 0 and nt > 0");
    return NAT_BEM_EINVAL;
  }
  if (nt > (int64_t)1 << 30 || nv > (int64_t)1 << 30) {
    set_error("mesh: too many vertices or triangles");
    return NAT_BEM_EINVAL;
  }
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(V[i])) {
      set_error("mesh: non-finite vertex coordinate at vertex " + std::to_string(i / 3));
      return NAT_BEM_EINVAL;
    }
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (T[i] < 0 || T[i] >= nv) {
      set_error("mesh: vertex index out of range in triangle " + std::to_string(i / 3));
      return NAT_BEM_EINVAL;
    }
  // every directed edge exactly once, and its reverse exactly once (closed, consistently
  // oriented, two triangles per edge)
  std::unordered_map<uint64_t, int32_t> edges;
  edges.reserve((size_t)(3 * nt * 2));
  double vol6 = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* f = T + 3 * t;
    V3 a = vget(V, f[0]), b = vget(V, f[1]), c = vget(V, f[2]);
    V3 cr = vcross(vsub(b, a), vsub(c, a));
    if (!(vdot(cr, cr) > 0.0)) {
      set_error("mesh: zero-area triangle " + std::to_string(t));
      return NAT_BEM_EINVAL;
    }
    vol6 += vdot(a, vcross(b, c));
    for (int e = 0; e < 3; ++e) {
      uint64_t key = ((uint64_t)(uint32_t)f[e] << 32) | (uint32_t)f[(e + 1) % 3];
      if (++edges[key] > 1) {
        set_error("mesh: directed edge used twice (inconsistent orientation or non-manifold) "
                  "at triangle " + std::to_string(t));
        return NAT_BEM_EINVAL;
      }
    }
  }
  for (const auto& kv : edges) {
    uint64_t rev = (kv.first << 32) | (kv.first >> 32);
    if (edges.find(rev) == edges.end()) {
      set_error("mesh: not closed (an edge has a single triangle)");
      return NAT_BEM_EINVAL;
    }
  }
  if (!(vol6 > 0.0)) {
    set_error("mesh: enclosed volume is not positive (inward winding)");
    return NAT_BEM_EINVAL;
  }
  return NAT_BEM_OK;
}

void build_near_pairs(const int32_t* T, int64_t nv, int64_t nt, std::vector<int2>& pairs) {
  // vertex -> incident triangles (CSR)
  std::vector<int32_t> deg(nv + 1, 0);
  for (int64_t i = 0; i < 3 * nt; ++i) deg[T[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) deg[v + 1] += deg[v];
  std::vector<int32_t> inc(3 * nt), fill(deg.begin(), deg.end() - 1);
  for (int64_t t = 0; t < nt; ++t)
    for (int e = 0; e < 3; ++e) inc[fill[T[3 * t + e]]++] = (int32_t)t;
  pairs.clear();
  pairs.reserve((size_t)nt * 14);
  std::vector<int32_t> row;
  for (int64_t t = 0; t < nt; ++t) {
    row.clear();
    for (int e = 0; e < 3; ++e) {
      int32_t v = T[3 * t + e];
      for (int32_t q = deg[v]; q < deg[v + 1]; ++q) row.push_back(inc[q]);
    }
    std::sort(row.begin(), row.end());
    row.erase(std::unique(row.begin(), row.end()), row.end());
    for (int32_t j : row)
      if (j != t) pairs.push_back(make_int2((int)t, j));  // the self pair has its own kernel
  }
}

}  // namespace natbem
