// Internal declarations of the natbem library (CUDA path). Nothing here is shared with the
// FP64 oracle; this header is only included by the library's own translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/nat_bem.h"

namespace natbem {

// ----------------------------------------------------------------------------- errors
void set_error(const std::string& msg);
void clear_error();

#define NB_TRY_CUDA(call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::natbem::set_error(std::string(#call) + " failed: " + cudaGetErrorString(e_));       \
      return (e_ == cudaErrorMemoryAllocation) ? NAT_BEM_ENOMEM : NAT_BEM_ECUDA;            \
    }                                                                                       \
  } while (0)

#define NB_CHECK_LAUNCH() NB_TRY_CUDA(cudaGetLastError())

#define NB_TRY(expr)                                                                        \
  do {                                                                                      \
    nat_bem_status s_ = (expr);                                                             \
    if (s_ != NAT_BEM_OK) return s_;                                                        \
  } while (0)

// ---------------------------------------------------------------------------- tracing
// Counts one kernel launch and, when tracing is on, brackets it with CUDA events on its
// stream. Construct it immediately before the launch, in the same scope:
//   { TraceScope t("gemv", s); k_gemv<<<g, b, 0, s>>>(...); }
class TraceScope {
 public:
  TraceScope(const char* name, cudaStream_t s);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  void* a_ = nullptr;
  void* b_ = nullptr;
};

bool tracing_enabled();
int64_t launch_count();
int64_t thread_launch_count();  // launches from the calling thread only
void add_launches(int64_t n);  // kernels launched through a replayed CUDA graph

#define NB_LAUNCH(name, stream, ...)            \
  do {                                          \
    ::natbem::TraceScope nb_trace_(name, stream); \
    __VA_ARGS__;                                \
  } while (0)

// ------------------------------------------------------------------------ device memory
// Stream-ordered allocations from a library-owned pool per device that keeps freed blocks
// cached (release threshold = unlimited), so repeated operators of the same size reuse memory
// without going back to the driver.
nat_bem_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
nat_bem_status dev_alloc_n(T** p, size_t count, cudaStream_t s) {
  return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// Whether p is a device (or managed) pointer the GPU can read directly.
bool is_device_pointer(const void* p);

// A device copy of `count` elements of p (which may be a host pointer). Sets *tmp when it
// allocated one; the caller frees it on the same stream.
template <class T>
inline nat_bem_status to_device(const T* p, size_t count, cudaStream_t s, const T** dp, T** tmp) {
  *tmp = nullptr;
  if (is_device_pointer(p)) {
    *dp = p;
    return NAT_BEM_OK;
  }
  NB_TRY(dev_alloc_n(tmp, count, s));
  NB_TRY_CUDA(cudaMemcpyAsync(*tmp, p, count * sizeof(T), cudaMemcpyHostToDevice, s));
  *dp = *tmp;
  return NAT_BEM_OK;
}


// -------------------------------------------------------------------------- geometry
// Device-resident mesh records. Single-precision records serve the regular (FP32) pairs and
// the field evaluation; double-precision arrays serve the self and vertex-sharing pairs.
struct Geometry {
  int64_t n = 0;              // triangles
  int64_t ld = 0;             // leading dimension of the n x n operators (n rounded up to 32)
  // FP32 records, one per element
  float4* c_hi = nullptr;     // centroid, high part (x, y, z, 0)
  float4* c_lo = nullptr;     // centroid, low part: c = hi + lo to ~2^-48 relative
  float4* nrm = nullptr;      // unit outward normal (x, y, z, 0)
  float4* qp = nullptr;       // 7 per element: (y_q - c, w_q A / (4 pi)); 1 per Monte-Carlo sample
  int4* vid = nullptr;        // vertex indices (a, b, c, 0)
  // FP64 records
  double* tri = nullptr;      // 9 per element: vertices a, b, c
  double* cen = nullptr;      // 3 per element
  double* nrm64 = nullptr;    // 3 per element
  double* area = nullptr;     // 1 per element
  // vertex-sharing pairs (i, j != i), grouped by row; the self pairs (i, i) are implicit
  int2* near_pairs = nullptr;
  int64_t n_near = 0;
};

// Galerkin op (galerkin.cu): vertex -> triangle lists, P1 curls, and the 7 quadrature points
// of every element as one-point records for the field kernels.
struct Galerkin {
  int* adj_ptr = nullptr;  // nv + 1 offsets into adj
  int2* adj = nullptr;     // per vertex: (triangle, local index), increasing triangle order
  float4* curl = nullptr;  // 3 per element: curl of the P1 hat of local vertex a
  Geometry pts;            // 7 nt point records (position hi/lo, normal, weight w A / (4 pi))
};

// Host-side mesh check and near-pair list (mesh.cpp). Returns NAT_BEM_EINVAL with a message
// for an invalid mesh.
nat_bem_status validate_mesh_host(const double* V, int64_t nv, const int32_t* T, int64_t nt);
void build_near_pairs(const int32_t* T, int64_t nv, int64_t nt, std::vector<int2>& pairs);

// Quadrature tables the kernels read from constant memory (assemble.cu).
nat_bem_status upload_rules(int adj_levels, int self_pts);

// ------------------------------------------------------------------------------- op
struct Workspace;  // GMRES state (gmres.cu)

}  // namespace natbem

struct nat_bem_op {
  int64_t n = 0;
  double k = 0.0;
  nat_bem_opts opts{};
  int device = 0;
  cudaStream_t stream = nullptr;       // stream the op was built on (frees are ordered there)
  cudaStream_t solve_stream = nullptr; // solves called on the legacy default stream run here
  cudaEvent_t solve_event = nullptr;   // (captured graphs need a non-legacy stream)
  natbem::Geometry geo;
  float2* L = nullptr;                 // n x ld complex64, row-major
  float2* R = nullptr;                 // n x ld complex64, row-major (store_r)
  uint32_t* Lb = nullptr;              // n x ld complex as packed bf16 pairs (mixed BF16) or, with
                                       // copy_fp16, packed half2 of the row-scaled entries
  bool copy_fp16 = false;              // mixed FP16: Lb holds L_ij s_i in half precision
  float* row_scale = nullptr;          // mixed FP16: 1 / s_i per row (a power of two)
  uint16_t* Ls = nullptr;              // FP32-accurate multi-RHS products: L split into three
                                       // BF16 planes (n x 2 ld each), built on first use
  bool split_ok = false;               // Ls holds the split of the current L
  bool views = false;                  // L, R and Lb belong to someone else (not freed here)
  bool geo_view = false;               // geo belongs to another op of the same mesh
  int64_t bstride = 0;                 // > 0: a batch of operators, RHS s uses L + s bstride
                                       // (and R, Lb likewise); 0: one operator for every RHS
  natbem::Workspace* ws = nullptr;     // solver workspace, grown on demand
  bool mc = false;                     // Monte-Carlo op (nat_bem_assemble_mc): n samples
  double mc_area = 0.0;                // Monte-Carlo op: total surface area
  bool galerkin = false;               // Galerkin op: n = vertices, geo.n = triangles
  int64_t nn = 0;                      // Neumann values per RHS (triangles; n except Galerkin)
  int64_t ldr = 0;                     // leading dimension of R (geo.ld except Galerkin)
  natbem::Galerkin gal;                // Galerkin op only
};

namespace natbem {

// api.cu: a mesh op as nat_bem_assemble builds it, with leading dimension ld (>= nt rounded up
// to 32) and, when L is given, its operators written into the caller's memory (views: L, R and,
// for mixed BF16, Lb of nt x ld each) instead of owned allocations.
nat_bem_status build_mesh_op(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double k,
                             const nat_bem_opts& o, cudaStream_t s, int64_t ld, float2* L, float2* R,
                             uint32_t* Lb, float* row_scale, nat_bem_op** out);
inline bool low_copy(const nat_bem_opts& o) {
  return o.prec == NAT_BEM_PREC_MIXED_BF16 || o.prec == NAT_BEM_PREC_MIXED_FP16;
}
nat_bem_status check_opts(const nat_bem_opts& o);

// assemble.cu
nat_bem_status geometry_build(nat_bem_op* op, const double* dV, const int32_t* dT, int64_t nv,
                              const std::vector<int2>& near_pairs, cudaStream_t s);
nat_bem_status assemble_operators(nat_bem_op* op, cudaStream_t s);
// The BF16 copy is written by the assembly kernels; this writes the row-scaled FP16 copy from
// the assembled L (mixed FP16; nothing otherwise). Every assembly ends with it.
nat_bem_status finish_low_copy(nat_bem_op* op, cudaStream_t s);
// The pointer the assembly kernels write the BF16 copy to (null for an FP16 or no copy).
inline uint32_t* bf16_target(const nat_bem_op* op) { return op->copy_fp16 ? nullptr : op->Lb; }

// mc.cu
nat_bem_status mc_geometry_build(nat_bem_op* op, const double* dY, const double* dN, cudaStream_t s);
nat_bem_status mc_assemble_operators(nat_bem_op* op, cudaStream_t s);

// galerkin.cu
nat_bem_status galerkin_geometry_build(nat_bem_op* op, const int32_t* T, int64_t nv, cudaStream_t s);
nat_bem_status galerkin_assemble_operators(nat_bem_op* op, cudaStream_t s);
// P1 p (nv per RHS) and P0 g (nt per RHS) at the 7 points of every triangle (7 nt per RHS)
nat_bem_status galerkin_expand(const nat_bem_op* op, const float2* d_p, const float2* d_g, int nrhs,
                               float2** pq, float2** gq, cudaStream_t s);
void galerkin_free(nat_bem_op* op, cudaStream_t s);

// gmres.cu
// per_rhs / per_conv (may be null): each RHS's iterations and true residual, and whether it
// met the tolerance.
nat_bem_status solve_impl(nat_bem_op* op, const float2* d_neumann, int nrhs, float2* d_p,
                          nat_bem_solve_info* info, cudaStream_t s,
                          std::vector<nat_bem_solve_info>* per_rhs = nullptr,
                          std::vector<int>* per_conv = nullptr);
void workspace_free(Workspace* ws, cudaStream_t s);
nat_bem_status apply_impl(nat_bem_op* op, int which, int engine, const float2* d_x, int nrhs,
                          float2* d_y, cudaStream_t s);
int64_t workspace_bytes(int64_t n, int nrhs, const nat_bem_opts& o);
int gemv_tuned_variant(int64_t n);  // -1 before the autotuner met this size

// products.cu: Y = M X for nrhs right-hand sides (M = L for which == 0, R for 1).
// kEngineFp32: FP32 CUDA-core complex GEMM; kEngineTf32 / kEngineBf16: tcgen05 tensor cores
// on L (TF32) or its BF16 copy, using `scratch` for the packed B and the split-K partials.
// kEngineGemvCopy: the GEMV on the low-precision copy (BF16 or row-scaled FP16, by the op).
enum Engine { kEngineGemv = 0, kEngineGemvCopy = 1, kEngineFp32 = 2, kEngineTf32 = 3, kEngineBf16 = 4,
              kEngineFp16 = 5 };
nat_bem_status product(nat_bem_op* op, int which, int engine, const float2* X, int nrhs,
                       double2* Y, const int* done, const int* scal, void* scratch,
                       size_t scratch_bytes, int* err, cudaStream_t s);
size_t tc_workspace_bytes(int64_t n, int64_t ld, int nrhs, int sms);
// The FP32-accurate multi-RHS product on tensor cores (three-way BF16 split of L and X) runs for
// products with L and at least kX6MinRhs RHS once ensure_split has built the split of L.
constexpr int kX6MinRhs = 8;
bool x6_enabled();
nat_bem_status ensure_split(nat_bem_op* op, cudaStream_t s);
// Picks the tensor-core product's launch shape for this operator size and RHS count by timing
// the candidates once per size class (outside graph capture); X, Y and scratch are the caller's.
nat_bem_status tc_tune(nat_bem_op* op, int engine, int nrhs, const float2* X, double2* Y,
                       void* scratch, size_t scratch_bytes, int* err, cudaStream_t s);

// eval.cu
nat_bem_status eval_impl(const nat_bem_op* op, const double* d_pts, int64_t m,
                         const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                         cudaStream_t s);
nat_bem_status far_field_impl(const nat_bem_op* op, const double* d_dirs, int64_t nd,
                              const float2* d_p, const float2* d_g, int nrhs, float2* d_out,
                              cudaStream_t s);
nat_bem_status sample_field_impl(const nat_bem_op* op, const double* d_u, int64_t n, const double* center,
                                 double r_lo, double r_hi, const float2* d_p, const float2* d_g, int nrhs,
                                 double* d_coords, float* d_amp, cudaStream_t s);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// tune.cu: index of the fastest of `ncand` launch shapes of `kind` for this size class on the
// current device; run(c) enqueues shape c on s (timed once per class, outside graph capture).
int autotune(const char* kind, int64_t size_class, int ncand, const std::function<nat_bem_status(int)>& run,
             cudaStream_t s);

}  // namespace natbem
