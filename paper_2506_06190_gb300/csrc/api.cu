// C ABI entry points (include/nat_bem.h): argument checks, host/device staging, memory pool,
// and the order of the device stages. No function lets a C++ exception or abort cross the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace natbem {

namespace {
thread_local std::string g_last_error;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
bool g_rules_ready[64] = {};
int g_rules_levels[64] = {};
int g_rules_self[64] = {};
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

static cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

nat_bem_status dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) {
    set_error("could not create the device memory pool");
    return NAT_BEM_ECUDA;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " +
              cudaGetErrorString(e));
    *p = nullptr;
    return NAT_BEM_ENOMEM;
  }
  return NAT_BEM_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static nat_bem_status ensure_rules(int levels, int self_pts) {
  int dev = 0;
  NB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return NAT_BEM_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_rules_ready[dev] && g_rules_levels[dev] == levels && g_rules_self[dev] == self_pts)
    return NAT_BEM_OK;
  NB_TRY(upload_rules(levels, self_pts));
  g_rules_ready[dev] = true;
  g_rules_levels[dev] = levels;
  g_rules_self[dev] = self_pts;
  return NAT_BEM_OK;
}

nat_bem_status check_opts(const nat_bem_opts& o) {
  if (o.adj_subdiv_levels < 0 || o.adj_subdiv_levels > 3) {
    set_error("opts.adj_subdiv_levels must be in [0, 3]");
    return NAT_BEM_EINVAL;
  }
  if (o.self_theta_pts < 1 || o.self_theta_pts > 64) {
    set_error("opts.self_theta_pts must be in [1, 64]");
    return NAT_BEM_EINVAL;
  }
  if (!(o.tol > 0.0) || !std::isfinite(o.tol)) {
    set_error("opts.tol must be positive and finite");
    return NAT_BEM_EINVAL;
  }
  if (o.restart < 0 || o.restart > 255) {
    set_error("opts.restart must be in [0, 255] (0 = unrestarted GMRES)");
    return NAT_BEM_EINVAL;
  }
  if (o.max_iter < 1 || o.max_iter > (o.restart > 0 ? 100000 : 255)) {
    set_error("opts.max_iter must be in [1, 255] (unrestarted) or [1, 100000] (restart > 0)");
    return NAT_BEM_EINVAL;
  }
  if (o.device_loop != 0 && o.device_loop != 1) {
    set_error("opts.device_loop must be 0 or 1");
    return NAT_BEM_EINVAL;
  }
  if (o.quad_regular != 7) {
    set_error("opts.quad_regular must be 7 (the 7-point degree-5 rule is the only regular rule)");
    return NAT_BEM_EINVAL;
  }
  if (o.prec != NAT_BEM_PREC_FP32 && o.prec != NAT_BEM_PREC_MIXED_TF32 &&
      o.prec != NAT_BEM_PREC_MIXED_BF16 && o.prec != NAT_BEM_PREC_MIXED_FP16) {
    set_error("opts.prec is not a nat_bem_precision value");
    return NAT_BEM_EINVAL;
  }
  if (o.inner_max_iter < 1 || o.inner_max_iter > 255 || !(o.inner_tol > 0.0) ||
      o.max_refinements < 1) {
    set_error("opts: inner_max_iter in [1, 255], inner_tol > 0, max_refinements >= 1");
    return NAT_BEM_EINVAL;
  }
  return NAT_BEM_OK;
}

}  // namespace natbem

using namespace natbem;

namespace {
// Galerkin assembly keeps element-pair blocks of at least 512 test triangles x nt trial
// triangles (96 bytes each) as scratch: 3.2 GB at this size.
constexpr int64_t kGalerkinMaxTriangles = 65536;
}  // namespace

extern "C" {

void nat_bem_opts_default(nat_bem_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->adj_subdiv_levels = 2;
  o->self_theta_pts = 16;
  o->tol = 1e-6;
  o->max_iter = 200;
  o->prec = NAT_BEM_PREC_FP32;
  o->inner_max_iter = 60;
  o->inner_tol = 1e-2;
  o->max_refinements = 10;
  o->restart = 0;
  o->quad_regular = 7;
  o->device_loop = 1;
}

const char* nat_bem_last_error(void) { return g_last_error.c_str(); }

int32_t nat_bem_gemv_variant(int64_t nt) { return nt > 0 ? gemv_tuned_variant(nt) : -1; }

int64_t nat_bem_op_size(const nat_bem_op* op) { return op ? op->n : 0; }

int64_t nat_bem_required_bytes(int64_t nt, int32_t nrhs, const nat_bem_opts* opts) {
  nat_bem_opts o;
  nat_bem_opts_default(&o);
  if (opts) o = *opts;
  if (nt <= 0 || nrhs < 1) return 0;
  const int64_t ld = round_up(nt, 32);
  int64_t b = 2 * 8 * nt * ld;                                     // L and R
  if (low_copy(o)) b += 4 * nt * ld;                               // BF16 or FP16 copy of L
  if (o.prec == NAT_BEM_PREC_MIXED_FP16) b += 4 * nt;               // its row scales
  b += nt * (7 * 16 + 5 * 16 + 9 * 8 + 7 * 8 + 8 * 14);             // geometry + near pairs
  b += workspace_bytes(nt, nrhs, o);
  if (nrhs >= kX6MinRhs) b += 12 * nt * ld;  // three BF16 planes of L for the accurate products
  return b;
}

}  // extern "C"

namespace natbem {

nat_bem_status build_mesh_op(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double k,
                             const nat_bem_opts& o, cudaStream_t s, int64_t ld, float2* L, float2* R,
                             uint32_t* Lb, float* row_scale, nat_bem_op** out) {
  *out = nullptr;
  // host copies for the mesh checks and the near-pair list
  const bool vdev = is_device_pointer(verts), tdev = is_device_pointer(tris);
  std::vector<double> hV;
  std::vector<int32_t> hT;
  const double* V = verts;
  const int32_t* T = tris;
  if (vdev) {
    hV.resize(3 * nv);
    NB_TRY_CUDA(cudaMemcpyAsync(hV.data(), verts, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    V = hV.data();
  }
  if (tdev) {
    hT.resize(3 * nt);
    NB_TRY_CUDA(cudaMemcpyAsync(hT.data(), tris, 3 * nt * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    T = hT.data();
  }
  NB_TRY(validate_mesh_host(V, nv, T, nt));
  std::vector<int2> near;
  build_near_pairs(T, nv, nt, near);
  NB_TRY(ensure_rules(o.adj_subdiv_levels, o.self_theta_pts));

  nat_bem_op* op = new (std::nothrow) nat_bem_op();
  if (!op) {
    set_error("host allocation failed");
    return NAT_BEM_ENOMEM;
  }
  op->n = nt;
  op->k = k;
  op->opts = o;
  op->copy_fp16 = o.prec == NAT_BEM_PREC_MIXED_FP16;
  op->stream = s;
  cudaGetDevice(&op->device);
  op->geo.n = nt;
  op->geo.ld = std::max<int64_t>(ld, round_up(nt, 32));
  op->nn = nt;
  op->ldr = op->geo.ld;
  auto fail = [&](nat_bem_status st) {
    nat_bem_destroy(op);
    return st;
  };
  const double* dV = nullptr;
  const int32_t* dT = nullptr;
  double* tV = nullptr;
  int32_t* tT = nullptr;
  nat_bem_status st = to_device(verts, (size_t)(3 * nv), s, &dV, &tV);
  if (st != NAT_BEM_OK) return fail(st);
  st = to_device(tris, (size_t)(3 * nt), s, &dT, &tT);
  if (st != NAT_BEM_OK) return fail(st);
  st = geometry_build(op, dV, dT, nv, near, s);
  dev_free(tV, s);
  dev_free(tT, s);
  if (st != NAT_BEM_OK) return fail(st);
  if (L) {  // the caller's memory
    op->views = true;
    op->L = L;
    op->R = R;
    op->Lb = low_copy(o) ? Lb : nullptr;
    op->row_scale = op->copy_fp16 ? row_scale : nullptr;
  } else {
    const size_t mat = (size_t)nt * (size_t)op->geo.ld;
    if ((st = dev_alloc_n(&op->L, mat, s)) != NAT_BEM_OK) return fail(st);
    if ((st = dev_alloc_n(&op->R, mat, s)) != NAT_BEM_OK) return fail(st);
    if (low_copy(o) && (st = dev_alloc_n(&op->Lb, mat, s)) != NAT_BEM_OK) return fail(st);
    if (op->copy_fp16 && (st = dev_alloc_n(&op->row_scale, (size_t)nt, s)) != NAT_BEM_OK) return fail(st);
  }
  if ((st = assemble_operators(op, s)) != NAT_BEM_OK) return fail(st);
  *out = op;
  return NAT_BEM_OK;
}

}  // namespace natbem

extern "C" {

nat_bem_status nat_bem_assemble(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                                double k, const nat_bem_opts* opts, void* cuda_stream,
                                nat_bem_op** out) {
  try {
    clear_error();
    if (!out) {
      set_error("out is NULL");
      return NAT_BEM_EINVAL;
    }
    *out = nullptr;
    if (!verts || !tris) {
      set_error("verts and tris must not be NULL");
      return NAT_BEM_EINVAL;
    }
    if (!(k > 0.0) || !std::isfinite(k)) {
      set_error("k must be positive and finite");
      return NAT_BEM_EINVAL;
    }
    if (nv <= 0 || nt <= 0) {
      set_error("mesh: need nv > 0 and nt > 0");
      return NAT_BEM_EINVAL;
    }
    nat_bem_opts o;
    nat_bem_opts_default(&o);
    if (opts) o = *opts;
    NB_TRY(check_opts(o));
    return build_mesh_op(verts, nv, tris, nt, k, o, (cudaStream_t)cuda_stream, 0, nullptr, nullptr,
                         nullptr, nullptr, out);
  } catch (...) {
    set_error("internal error in nat_bem_assemble");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_assemble_galerkin(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                                         double k, const nat_bem_opts* opts, void* cuda_stream,
                                         nat_bem_op** out) {
  try {
    clear_error();
    if (!out) {
      set_error("out is NULL");
      return NAT_BEM_EINVAL;
    }
    *out = nullptr;
    if (!verts || !tris) {
      set_error("verts and tris must not be NULL");
      return NAT_BEM_EINVAL;
    }
    if (!(k > 0.0) || !std::isfinite(k)) {
      set_error("k must be positive and finite");
      return NAT_BEM_EINVAL;
    }
    if (nv <= 0 || nt <= 0 || nt > kGalerkinMaxTriangles) {
      set_error("nat_bem_assemble_galerkin: need nv > 0 and 0 < nt <= 65536");
      return NAT_BEM_EINVAL;
    }
    nat_bem_opts o;
    nat_bem_opts_default(&o);
    if (opts) o = *opts;
    NB_TRY(check_opts(o));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<double> hV(3 * nv);
    std::vector<int32_t> hT(3 * nt);
    NB_TRY_CUDA(cudaMemcpyAsync(hV.data(), verts, 3 * nv * sizeof(double), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaMemcpyAsync(hT.data(), tris, 3 * nt * sizeof(int32_t), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    NB_TRY(validate_mesh_host(hV.data(), nv, hT.data(), nt));
    {
      // every vertex must carry a P1 unknown: each one belongs to some triangle
      std::vector<char> used(nv, 0);
      for (int64_t i = 0; i < 3 * nt; ++i) used[hT[i]] = 1;
      for (int64_t v = 0; v < nv; ++v)
        if (!used[v]) {
          set_error("nat_bem_assemble_galerkin: vertex " + std::to_string(v) + " belongs to no triangle");
          return NAT_BEM_EINVAL;
        }
    }
    std::vector<int2> near;
    build_near_pairs(hT.data(), nv, nt, near);
    NB_TRY(ensure_rules(o.adj_subdiv_levels, o.self_theta_pts));
    nat_bem_op* op = new (std::nothrow) nat_bem_op();
    if (!op) {
      set_error("host allocation failed");
      return NAT_BEM_ENOMEM;
    }
    op->n = nv;
    op->k = k;
    op->opts = o;
    op->stream = s;
    op->galerkin = true;
    cudaGetDevice(&op->device);
    op->geo.n = nt;
    op->geo.ld = round_up(nv, 32);
    op->nn = nt;
    op->ldr = round_up(nt, 32);
    auto fail = [&](nat_bem_status st) {
      nat_bem_destroy(op);
      return st;
    };
    double* dV = nullptr;
    int32_t* dT = nullptr;
    nat_bem_status st = dev_alloc_n(&dV, (size_t)(3 * nv), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dT, (size_t)(3 * nt), s);
    if (st == NAT_BEM_OK &&
        (cudaMemcpyAsync(dV, hV.data(), 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(dT, hT.data(), 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)) {
      set_error("nat_bem_assemble_galerkin: mesh copy failed");
      st = NAT_BEM_ECUDA;
    }
    if (st == NAT_BEM_OK) st = geometry_build(op, dV, dT, nv, near, s);
    if (st == NAT_BEM_OK) st = galerkin_geometry_build(op, hT.data(), nv, s);
    dev_free(dV, s);
    dev_free(dT, s);
    if (st != NAT_BEM_OK) return fail(st);
    if ((st = dev_alloc_n(&op->L, (size_t)nv * op->geo.ld, s)) != NAT_BEM_OK) return fail(st);
    if ((st = dev_alloc_n(&op->R, (size_t)nv * op->ldr, s)) != NAT_BEM_OK) return fail(st);
    op->copy_fp16 = o.prec == NAT_BEM_PREC_MIXED_FP16;
    if (op->copy_fp16 && (st = dev_alloc_n(&op->row_scale, (size_t)nv, s)) != NAT_BEM_OK) return fail(st);
    if (low_copy(o) && (st = dev_alloc_n(&op->Lb, (size_t)nv * op->geo.ld, s)) != NAT_BEM_OK)
      return fail(st);
    if ((st = galerkin_assemble_operators(op, s)) != NAT_BEM_OK) return fail(st);
    *out = op;
    return NAT_BEM_OK;
  } catch (...) {
    set_error("internal error in nat_bem_assemble_galerkin");
    return NAT_BEM_ECUDA;
  }
}

int64_t nat_bem_op_neumann_size(const nat_bem_op* op) { return op ? op->nn : 0; }

nat_bem_status nat_bem_assemble_mc(const double* pts, const double* normals, int64_t m, double area,
                                   double k, const nat_bem_opts* opts, void* cuda_stream,
                                   nat_bem_op** out) {
  try {
    clear_error();
    if (!out) {
      set_error("out is NULL");
      return NAT_BEM_EINVAL;
    }
    *out = nullptr;
    if (!pts || !normals) {
      set_error("pts and normals must not be NULL");
      return NAT_BEM_EINVAL;
    }
    if (!(k > 0.0) || !std::isfinite(k)) {
      set_error("k must be positive and finite");
      return NAT_BEM_EINVAL;
    }
    if (m < 2 || m > ((int64_t)1 << 30)) {
      set_error("nat_bem_assemble_mc: need 2 <= m < 2^30 samples");
      return NAT_BEM_EINVAL;
    }
    if (!(area > 0.0) || !std::isfinite(area)) {
      set_error("nat_bem_assemble_mc: area must be positive and finite");
      return NAT_BEM_EINVAL;
    }
    nat_bem_opts o;
    nat_bem_opts_default(&o);
    if (opts) o = *opts;
    NB_TRY(check_opts(o));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // host copies for the checks: finite positions, unit normals
    std::vector<double> hY(3 * m), hN(3 * m);
    NB_TRY_CUDA(cudaMemcpyAsync(hY.data(), pts, 3 * m * sizeof(double), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaMemcpyAsync(hN.data(), normals, 3 * m * sizeof(double), cudaMemcpyDefault, s));
    NB_TRY_CUDA(cudaStreamSynchronize(s));
    for (int64_t j = 0; j < m; ++j) {
      const double* y = &hY[3 * j];
      const double* nv = &hN[3 * j];
      if (!std::isfinite(y[0]) || !std::isfinite(y[1]) || !std::isfinite(y[2])) {
        set_error("nat_bem_assemble_mc: sample " + std::to_string(j) + " is not finite");
        return NAT_BEM_EINVAL;
      }
      const double nn = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
      if (!(std::fabs(nn - 1.0) < 1e-6)) {
        set_error("nat_bem_assemble_mc: normal " + std::to_string(j) + " is not a unit vector");
        return NAT_BEM_EINVAL;
      }
    }
    nat_bem_op* op = new (std::nothrow) nat_bem_op();
    if (!op) {
      set_error("host allocation failed");
      return NAT_BEM_ENOMEM;
    }
    op->n = m;
    op->k = k;
    op->opts = o;
    op->stream = s;
    op->mc = true;
    op->mc_area = area;
    cudaGetDevice(&op->device);
    op->geo.n = m;
    op->geo.ld = round_up(m, 32);
    op->nn = m;
    op->ldr = op->geo.ld;
    auto fail = [&](nat_bem_status st) {
      nat_bem_destroy(op);
      return st;
    };
    double *dY = nullptr, *dN = nullptr;
    nat_bem_status st = dev_alloc_n(&dY, (size_t)(3 * m), s);
    if (st == NAT_BEM_OK) st = dev_alloc_n(&dN, (size_t)(3 * m), s);
    if (st != NAT_BEM_OK) {
      dev_free(dY, s);
      return fail(st);
    }
    if (cudaMemcpyAsync(dY, hY.data(), 3 * m * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dN, hN.data(), 3 * m * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      dev_free(dY, s);
      dev_free(dN, s);
      set_error("nat_bem_assemble_mc: copy of the samples failed");
      return fail(NAT_BEM_ECUDA);
    }
    st = mc_geometry_build(op, dY, dN, s);
    if (st == NAT_BEM_OK) NB_TRY_CUDA(cudaStreamSynchronize(s));  // hY, hN are the copies' sources
    dev_free(dY, s);
    dev_free(dN, s);
    if (st != NAT_BEM_OK) return fail(st);
    const size_t mat = (size_t)m * (size_t)op->geo.ld;
    if ((st = dev_alloc_n(&op->L, mat, s)) != NAT_BEM_OK) return fail(st);
    if ((st = dev_alloc_n(&op->R, mat, s)) != NAT_BEM_OK) return fail(st);
    op->copy_fp16 = o.prec == NAT_BEM_PREC_MIXED_FP16;
    if (op->copy_fp16 && (st = dev_alloc_n(&op->row_scale, (size_t)m, s)) != NAT_BEM_OK) return fail(st);
    if (low_copy(o) && (st = dev_alloc_n(&op->Lb, mat, s)) != NAT_BEM_OK)
      return fail(st);
    if ((st = mc_assemble_operators(op, s)) != NAT_BEM_OK) return fail(st);
    *out = op;
    return NAT_BEM_OK;
  } catch (...) {
    set_error("internal error in nat_bem_assemble_mc");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_solve(nat_bem_op* op, const float* neumann, int32_t nrhs, float* p_out,
                             nat_bem_solve_info* info, void* cuda_stream) {
  try {
    clear_error();
    if (!op || !neumann || !p_out || nrhs < 1) {
      set_error("nat_bem_solve: op, neumann and p_out must be non-NULL and nrhs >= 1");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (s == nullptr || s == cudaStreamLegacy) {
      // the legacy default stream cannot be captured: run on the op's own stream, after the
      // caller's earlier work on the legacy stream (the solve ends with a host sync, so later
      // work there sees its results)
      if (!op->solve_stream) {
        NB_TRY_CUDA(cudaStreamCreateWithFlags(&op->solve_stream, cudaStreamNonBlocking));
        NB_TRY_CUDA(cudaEventCreateWithFlags(&op->solve_event, cudaEventDisableTiming));
      }
      NB_TRY_CUDA(cudaEventRecord(op->solve_event, cudaStreamLegacy));
      NB_TRY_CUDA(cudaStreamWaitEvent(op->solve_stream, op->solve_event, 0));
      s = op->solve_stream;
    }
    const size_t cnt = (size_t)op->n * nrhs;
    const float2* dg = nullptr;
    float2* tg = nullptr;
    NB_TRY(to_device(reinterpret_cast<const float2*>(neumann), (size_t)op->nn * nrhs, s, &dg, &tg));
    const bool pdev = is_device_pointer(p_out);
    float2* dp = reinterpret_cast<float2*>(p_out);
    float2* tp = nullptr;
    if (!pdev) {
      NB_TRY(dev_alloc_n(&tp, cnt, s));
      dp = tp;
    }
    nat_bem_status st = solve_impl(op, dg, nrhs, dp, info, s);
    if ((st == NAT_BEM_OK || st == NAT_BEM_ENOCONV) && !pdev) {
      cudaError_t e = cudaMemcpyAsync(p_out, tp, cnt * sizeof(float2), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("copy of p to the host failed: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      }
    }
    dev_free(tg, s);
    dev_free(tp, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_bem_solve");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_eval(const nat_bem_op* op, const double* pts, int64_t m, const float* p,
                            const float* neumann, int32_t nrhs, float* field_out,
                            void* cuda_stream) {
  try {
    clear_error();
    if (!op || m < 0 || nrhs < 1 || (m > 0 && (!pts || !p || !neumann || !field_out))) {
      set_error("nat_bem_eval: bad arguments (op NULL, m < 0, nrhs < 1 or NULL arrays)");
      return NAT_BEM_EINVAL;
    }
    if (m == 0) return NAT_BEM_OK;
    if (m > ((int64_t)1 << 31) - 1) {
      set_error("nat_bem_eval: too many points");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t cnt = (size_t)op->n * nrhs;
    const double* dpts = nullptr;
    double* tpts = nullptr;
    const float2 *dp = nullptr, *dg = nullptr;
    float2 *tp = nullptr, *tg = nullptr;
    NB_TRY(to_device(pts, (size_t)(3 * m), s, &dpts, &tpts));
    NB_TRY(to_device(reinterpret_cast<const float2*>(p), cnt, s, &dp, &tp));
    NB_TRY(to_device(reinterpret_cast<const float2*>(neumann), (size_t)op->nn * nrhs, s, &dg, &tg));
    const bool odev = is_device_pointer(field_out);
    float2* dout = reinterpret_cast<float2*>(field_out);
    float2* tout = nullptr;
    if (!odev) {
      NB_TRY(dev_alloc_n(&tout, (size_t)m * nrhs, s));
      dout = tout;
    }
    nat_bem_status st = eval_impl(op, dpts, m, dp, dg, nrhs, dout, s);
    if (st == NAT_BEM_OK && !odev) {
      cudaError_t e = cudaMemcpyAsync(field_out, tout, (size_t)m * nrhs * sizeof(float2),
                                      cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("copy of the field to the host failed: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      }
    }
    dev_free(tpts, s);
    dev_free(tp, s);
    dev_free(tg, s);
    dev_free(tout, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_bem_eval");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_far_field(const nat_bem_op* op, const double* dirs, int64_t nd, const float* p,
                                 const float* neumann, int32_t nrhs, float* out, void* cuda_stream) {
  try {
    clear_error();
    if (!op || nd < 0 || nrhs < 1 || (nd > 0 && (!dirs || !p || !neumann || !out))) {
      set_error("nat_bem_far_field: bad arguments (op NULL, nd < 0, nrhs < 1 or NULL arrays)");
      return NAT_BEM_EINVAL;
    }
    if (nd == 0) return NAT_BEM_OK;
    if (nd > ((int64_t)1 << 31) - 1) {
      set_error("nat_bem_far_field: too many directions");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t cnt = (size_t)op->n * nrhs;
    const double* dd = nullptr;
    double* td = nullptr;
    const float2 *dp = nullptr, *dg = nullptr;
    float2 *tp = nullptr, *tg = nullptr;
    NB_TRY(to_device(dirs, (size_t)(3 * nd), s, &dd, &td));
    NB_TRY(to_device(reinterpret_cast<const float2*>(p), cnt, s, &dp, &tp));
    NB_TRY(to_device(reinterpret_cast<const float2*>(neumann), (size_t)op->nn * nrhs, s, &dg, &tg));
    const bool odev = is_device_pointer(out);
    float2* dout = reinterpret_cast<float2*>(out);
    float2* tout = nullptr;
    if (!odev) {
      NB_TRY(dev_alloc_n(&tout, (size_t)nd * nrhs, s));
      dout = tout;
    }
    nat_bem_status st = far_field_impl(op, dd, nd, dp, dg, nrhs, dout, s);
    if (st == NAT_BEM_OK && !odev) {
      cudaError_t e = cudaMemcpyAsync(out, tout, (size_t)nd * nrhs * sizeof(float2), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("copy of the far field to the host failed: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      }
    }
    dev_free(td, s);
    dev_free(tp, s);
    dev_free(tg, s);
    dev_free(tout, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_bem_far_field");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_sample_field(const nat_bem_op* op, const double* u, int64_t n, const double* center,
                                    double r_lo, double r_hi, const float* p, const float* neumann,
                                    int32_t nrhs, double* coords_out, float* amp_out, void* cuda_stream) {
  try {
    clear_error();
    if (!op || n < 0 || nrhs < 1 || !center ||
        (n > 0 && (!u || !p || !neumann || !coords_out || !amp_out))) {
      set_error("nat_bem_sample_field: bad arguments (op or center NULL, n < 0, nrhs < 1, NULL arrays)");
      return NAT_BEM_EINVAL;
    }
    if (!(r_lo > 0.0) || !(r_hi >= r_lo) || !std::isfinite(r_hi) || !std::isfinite(center[0]) ||
        !std::isfinite(center[1]) || !std::isfinite(center[2])) {
      set_error("nat_bem_sample_field: need 0 < r_lo <= r_hi, finite, and a finite centre");
      return NAT_BEM_EINVAL;
    }
    if (n == 0) return NAT_BEM_OK;
    if (n > ((int64_t)1 << 31) - 1) {
      set_error("nat_bem_sample_field: too many samples");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t cnt = (size_t)op->n * nrhs;
    const double* du = nullptr;
    double* tu = nullptr;
    const float2 *dp = nullptr, *dg = nullptr;
    float2 *tp = nullptr, *tg = nullptr;
    NB_TRY(to_device(u, (size_t)(3 * n), s, &du, &tu));
    NB_TRY(to_device(reinterpret_cast<const float2*>(p), cnt, s, &dp, &tp));
    NB_TRY(to_device(reinterpret_cast<const float2*>(neumann), (size_t)op->nn * nrhs, s, &dg, &tg));
    const bool cdev = is_device_pointer(coords_out), adev = is_device_pointer(amp_out);
    double* dco = coords_out;
    float* dam = amp_out;
    double* tco = nullptr;
    float* tam = nullptr;
    if (!cdev) {
      NB_TRY(dev_alloc_n(&tco, (size_t)(3 * n), s));
      dco = tco;
    }
    if (!adev) {
      NB_TRY(dev_alloc_n(&tam, (size_t)n * nrhs, s));
      dam = tam;
    }
    nat_bem_status st = sample_field_impl(op, du, n, center, r_lo, r_hi, dp, dg, nrhs, dco, dam, s);
    if (st == NAT_BEM_OK && (!cdev || !adev)) {
      cudaError_t e = cudaSuccess;
      if (!cdev) e = cudaMemcpyAsync(coords_out, tco, (size_t)(3 * n) * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && !adev)
        e = cudaMemcpyAsync(amp_out, tam, (size_t)n * nrhs * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("copy of the samples to the host failed: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      }
    }
    dev_free(tu, s);
    dev_free(tp, s);
    dev_free(tg, s);
    dev_free(tco, s);
    dev_free(tam, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_bem_sample_field");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_op_apply(const nat_bem_op* op, int32_t which, int32_t engine,
                                const float* X, int32_t nrhs, float* Y, void* cuda_stream) {
  try {
    clear_error();
    const bool gemv_engine = engine >= NAT_BEM_ENGINE_GEMV0 && engine < NAT_BEM_ENGINE_GEMV0 + NAT_BEM_GEMV_VARIANTS;
    if (!op || !X || !Y || nrhs < 1 || which < 0 || which > 1 ||
        !(engine == NAT_BEM_ENGINE_AUTO || engine == NAT_BEM_ENGINE_FP32 ||
          engine == NAT_BEM_ENGINE_TF32 || engine == NAT_BEM_ENGINE_BF16 || engine == NAT_BEM_ENGINE_FP16 ||
          gemv_engine) ||
        (gemv_engine && nrhs != 1) ||
        ((engine == NAT_BEM_ENGINE_TF32 || engine == NAT_BEM_ENGINE_BF16 || engine == NAT_BEM_ENGINE_FP16) &&
         (which != 0 || nrhs > 128)) ||
        (engine == NAT_BEM_ENGINE_BF16 && (!op->Lb || op->copy_fp16)) ||
        (engine == NAT_BEM_ENGINE_FP16 && (!op->Lb || !op->copy_fp16))) {
      set_error("nat_bem_op_apply: bad arguments or engine not usable for this op");
      return NAT_BEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t cnt = (size_t)op->n * nrhs;
    const float2* dx = nullptr;
    float2* tx = nullptr;
    NB_TRY(to_device(reinterpret_cast<const float2*>(X), (size_t)(which == 1 ? op->nn : op->n) * nrhs, s, &dx, &tx));
    const bool ydev = is_device_pointer(Y);
    float2* dy = reinterpret_cast<float2*>(Y);
    float2* ty = nullptr;
    if (!ydev) {
      NB_TRY(dev_alloc_n(&ty, cnt, s));
      dy = ty;
    }
    nat_bem_status st = apply_impl(const_cast<nat_bem_op*>(op), which, engine, dx, nrhs, dy, s);
    if (st == NAT_BEM_OK && !ydev) {
      cudaError_t e = cudaMemcpyAsync(Y, ty, cnt * sizeof(float2), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("copy of Y to the host failed: ") + cudaGetErrorString(e));
        st = NAT_BEM_ECUDA;
      }
    }
    dev_free(tx, s);
    dev_free(ty, s);
    return st;
  } catch (...) {
    set_error("internal error in nat_bem_op_apply");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_op_rows(const nat_bem_op* op, int32_t which, int64_t row0, int64_t nrows,
                               float* out, void* cuda_stream) {
  clear_error();
  if (!op || !out || which < 0 || which > 1 || row0 < 0 || nrows < 0 || row0 + nrows > op->n) {
    set_error("nat_bem_op_rows: bad arguments");
    return NAT_BEM_EINVAL;
  }
  const float2* M = which == 0 ? op->L : op->R;
  if (!M) {
    set_error("nat_bem_op_rows: matrix not stored");
    return NAT_BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t cols = which == 1 ? op->nn : op->n, ld = which == 1 ? op->ldr : op->geo.ld;
  NB_TRY_CUDA(cudaMemcpy2DAsync(out, cols * sizeof(float2), M + row0 * ld, ld * sizeof(float2),
                                cols * sizeof(float2), nrows, cudaMemcpyDefault, s));
  NB_TRY_CUDA(cudaStreamSynchronize(s));
  return NAT_BEM_OK;
}

void nat_bem_destroy(nat_bem_op* op) {
  if (!op) return;
  cudaStream_t s = op->stream;
  Geometry& g = op->geo;
  if (!op->geo_view) {
    void* gp[] = {g.c_hi, g.c_lo, g.nrm, g.qp, g.vid, g.tri, g.cen, g.nrm64, g.area, g.near_pairs};
    for (void* p : gp) dev_free(p, s);
  }
  if (!op->views) {
    void* mp[] = {op->L, op->R, op->Lb, op->row_scale};
    for (void* p : mp) dev_free(p, s);
  }
  if (op->Ls) dev_free(op->Ls, s);
  galerkin_free(op, s);
  workspace_free(op->ws, s);
  if (op->solve_stream) {
    cudaStreamSynchronize(op->solve_stream);
    cudaStreamDestroy(op->solve_stream);
  }
  if (op->solve_event) cudaEventDestroy(op->solve_event);
  delete op;
}

nat_bem_status nat_bem_reassemble(nat_bem_op* op, double k, void* cuda_stream) {
  try {
    clear_error();
    if (!op) {
      set_error("nat_bem_reassemble: op is NULL");
      return NAT_BEM_EINVAL;
    }
    if (!(k > 0.0) || !std::isfinite(k)) {
      set_error("k must be positive and finite");
      return NAT_BEM_EINVAL;
    }
    op->k = k;
    op->split_ok = false;
    if (op->mc) return mc_assemble_operators(op, (cudaStream_t)cuda_stream);
    if (op->galerkin) return galerkin_assemble_operators(op, (cudaStream_t)cuda_stream);
    NB_TRY(ensure_rules(op->opts.adj_subdiv_levels, op->opts.self_theta_pts));
    return assemble_operators(op, (cudaStream_t)cuda_stream);
  } catch (...) {
    set_error("internal error in nat_bem_reassemble");
    return NAT_BEM_ECUDA;
  }
}

}  // extern "C"
