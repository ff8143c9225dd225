// Fused batched solves over meshes of uneven size: instead of one op, stream and launch
// sequence per job, jobs of similar size are grouped into size buckets and each bucket is
// solved as one system of B independent operators in lockstep. The bucket's operators are
// padded to its largest triangle count N (rows past a mesh's own n are the identity in L and
// zero in R, with zero right-hand side entries, so the padded solution is the mesh's own one
// followed by zeros) and stored back to back in one allocation, N x ld per operator. Every
// GMRES iteration of the bucket is then one GEMV launch over all B operators (right-hand side
// s reads operator s) and one cooperative Arnoldi launch over all B Krylov spaces, captured in
// CUDA graphs, with per-mesh convergence flags so finished meshes drop out of the launches.
// Assembly writes each mesh's operators straight into its slice (per-mesh geometry, the same
// kernels as a single assembly); the field is evaluated per mesh.
//
// Buckets: meshes sorted by size, largest first; a bucket takes meshes down to N / 2^(1/4)
// (so padding costs at most 41% more operator bytes, 15% on average over log-uniform sizes),
// up to max_batch meshes and a device-memory cap for the operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace natbem {
namespace {

constexpr double kBucketRatio = 1.189207115002721;       // 2^(1/4)
constexpr int64_t kBucketBytes = (int64_t)24 << 30;     // operators of one bucket (L, R, BF16 copy)

// Rows n..N-1 of one padded operator: L the identity, R zero (the low-precision copy: the
// identity too, bf16(1) = 0x3F80 or fp16(1) = 0x3C00 in the low half, row scale 1). One thread
// per (row, column).
__global__ void k_pad_rows(float2* __restrict__ L, float2* __restrict__ R, uint32_t* __restrict__ Lb,
                           uint32_t one, float* __restrict__ row_scale, int n, int N, int ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)(N - n) * ld;
  if (i >= total) return;
  const int row = n + (int)(i / ld), col = (int)(i % ld);
  const size_t off = (size_t)row * ld + col;
  const bool diag = row == col;
  L[off] = make_float2(diag ? 1.f : 0.f, 0.f);
  R[off] = make_float2(0.f, 0.f);
  if (Lb) Lb[off] = diag ? one : 0u;
  if (row_scale && col == 0) row_scale[row] = 1.0f;
}

// Column s of the bucket's right-hand sides: the mesh's n Neumann values, zeros up to N.
__global__ void k_pad_column(const float2* __restrict__ g, int n, int N, float2* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) G[i] = i < n ? g[i] : make_float2(0.f, 0.f);
}

struct Bucket {
  std::vector<int32_t> jobs;  // indices into the job array
  int64_t N = 0;
};

int64_t op_bytes(int64_t N, bool bf16) {
  const int64_t ld = round_up(N, 32);
  return N * ld * (16 + (bf16 ? 4 : 0));
}

// One bucket: assemble every mesh into its slice, pad, solve all in lockstep, evaluate fields.
nat_bem_status run_bucket(nat_bem_job* jobs, const Bucket& bk, const nat_bem_opts& o, cudaStream_t s,
                          std::string& first_error) {
  const int B = (int)bk.jobs.size();
  const int64_t N = bk.N, ld = round_up(N, 32);
  const bool bf16 = low_copy(o);  // a low-precision copy (BF16, or FP16 with row scales)
  const bool fp16 = o.prec == NAT_BEM_PREC_MIXED_FP16;
  const size_t slice = (size_t)N * (size_t)ld;
  float2 *L = nullptr, *R = nullptr, *G = nullptr, *P = nullptr;
  uint32_t* Lb = nullptr;
  float* RS = nullptr;
  std::vector<nat_bem_op*> ops(B, nullptr);
  nat_bem_op* batch = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  auto cleanup = [&]() {
    for (nat_bem_op* op : ops) nat_bem_destroy(op);
    nat_bem_destroy(batch);
    dev_free(L, s);
    dev_free(R, s);
    dev_free(Lb, s);
    dev_free(RS, s);
    dev_free(G, s);
    dev_free(P, s);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  };
  auto fail_all = [&](nat_bem_status st) {
    for (int32_t q : bk.jobs) jobs[q].status = st;
    if (first_error.empty()) first_error = nat_bem_last_error();
    cleanup();
    return st;
  };
  nat_bem_status st = NAT_BEM_OK;
  if ((st = dev_alloc_n(&L, slice * B, s)) != NAT_BEM_OK || (st = dev_alloc_n(&R, slice * B, s)) != NAT_BEM_OK ||
      (bf16 && (st = dev_alloc_n(&Lb, slice * B, s)) != NAT_BEM_OK) ||
      (fp16 && (st = dev_alloc_n(&RS, (size_t)N * B, s)) != NAT_BEM_OK) ||
      (st = dev_alloc_n(&G, (size_t)N * B, s)) != NAT_BEM_OK || (st = dev_alloc_n(&P, (size_t)N * B, s)) != NAT_BEM_OK)
    return fail_all(st);
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
    set_error("run_batch_fused: cudaEventCreate failed");
    return fail_all(NAT_BEM_ECUDA);
  }
  cudaEventRecord(t0, s);
  // per-mesh assembly into the slices; a mesh that fails its checks leaves the bucket (its
  // slice is then padded to the identity and its right-hand side to zero)
  std::vector<int> ok(B, 0);
  for (int b = 0; b < B; ++b) {
    nat_bem_job& j = jobs[bk.jobs[b]];
    const size_t off = slice * (size_t)b;
    // a mesh met earlier in the bucket (same arrays): its checks and geometry are reused, only
    // the element-pair kernels run again at this job's wavenumber
    int same = -1;
    for (int c = 0; c < b && same < 0; ++c) {
      const nat_bem_job& jc = jobs[bk.jobs[c]];
      if (ok[c] && jc.verts == j.verts && jc.tris == j.tris && jc.nv == j.nv && jc.nt == j.nt) same = c;
    }
    if (same >= 0) {
      nat_bem_op* op = new (std::nothrow) nat_bem_op(*ops[same]);
      if (!op) {
        set_error("host allocation failed");
        return fail_all(NAT_BEM_ENOMEM);
      }
      op->ws = nullptr;
      op->geo_view = true;
      op->views = true;
      op->k = j.k;
      op->stream = s;
      op->L = L + off;
      op->R = R + off;
      op->Lb = bf16 ? Lb + off : nullptr;
      op->row_scale = fp16 ? RS + (size_t)b * N : nullptr;
      ops[b] = op;
      st = assemble_operators(op, s);
    } else {
      st = build_mesh_op(j.verts, j.nv, j.tris, j.nt, j.k, o, s, ld, L + off, R + off, bf16 ? Lb + off : nullptr,
                         fp16 ? RS + (size_t)b * N : nullptr, &ops[b]);
    }
    int n_b = (int)j.nt;
    if (st != NAT_BEM_OK) {
      j.status = st;
      if (first_error.empty()) first_error = "job: " + std::string(nat_bem_last_error());
      n_b = 0;
    } else {
      ok[b] = 1;
    }
    if (n_b < N) {
      const int64_t tot = (int64_t)(N - n_b) * ld;
      NB_LAUNCH("pad_rows", s, k_pad_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
          L + off, R + off, bf16 ? Lb + off : nullptr, fp16 ? 0x3C00u : 0x3F80u,
          fp16 ? RS + (size_t)b * N : nullptr, n_b, (int)N, (int)ld));
    }
    // right-hand side column b (zero for a mesh that left the bucket)
    const float2* dg = nullptr;
    float2* tg = nullptr;
    if (ok[b]) {
      if ((st = to_device(reinterpret_cast<const float2*>(j.neumann), (size_t)j.nt, s, &dg, &tg)) != NAT_BEM_OK)
        return fail_all(st);
    }
    NB_LAUNCH("pad_column", s, k_pad_column<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
        dg, ok[b] ? n_b : 0, (int)N, G + (size_t)b * N));
    dev_free(tg, s);
    NB_CHECK_LAUNCH();
  }
  // the bucket as one op: B operators of N unknowns back to back
  batch = new (std::nothrow) nat_bem_op();
  if (!batch) {
    set_error("host allocation failed");
    return fail_all(NAT_BEM_ENOMEM);
  }
  batch->n = N;
  batch->opts = o;
  batch->stream = s;
  cudaGetDevice(&batch->device);
  batch->geo.n = N;
  batch->geo.ld = ld;
  batch->nn = N;
  batch->ldr = ld;
  batch->views = true;
  batch->L = L;
  batch->R = R;
  batch->Lb = Lb;
  batch->copy_fp16 = fp16;
  batch->row_scale = RS;
  batch->bstride = (int64_t)slice;
  std::vector<nat_bem_solve_info> per;
  std::vector<int> conv;
  nat_bem_solve_info info{};
  st = solve_impl(batch, G, B, P, &info, s, &per, &conv);
  if (st != NAT_BEM_OK && st != NAT_BEM_ENOCONV) return fail_all(st);
  // per mesh: surface pressure out, field at its points
  for (int b = 0; b < B; ++b) {
    if (!ok[b]) continue;
    nat_bem_job& j = jobs[bk.jobs[b]];
    const float2* pb = P + (size_t)b * N;
    nat_bem_status sj = conv[b] ? NAT_BEM_OK : NAT_BEM_ENOCONV;
    j.info = per[b];
    if (cudaMemcpyAsync(j.p_out, pb, (size_t)j.nt * sizeof(float2), cudaMemcpyDefault, s) != cudaSuccess) {
      set_error("run_batch_fused: copy of the surface pressure failed");
      sj = NAT_BEM_ECUDA;
    }
    if ((sj == NAT_BEM_OK || sj == NAT_BEM_ENOCONV) && j.m > 0) {
      // the field from the device copies of p and g (the job's arrays may be host memory)
      const float2* dg = nullptr;
      float2* tg = nullptr;
      nat_bem_status se = to_device(reinterpret_cast<const float2*>(j.neumann), (size_t)j.nt, s, &dg, &tg);
      if (se == NAT_BEM_OK)
        se = nat_bem_eval(ops[b], j.pts, j.m, reinterpret_cast<const float*>(pb),
                          reinterpret_cast<const float*>(dg), 1, j.field_out, s);
      dev_free(tg, s);
      if (se != NAT_BEM_OK) sj = se;
    }
    j.status = sj;
    if (sj != NAT_BEM_OK && first_error.empty()) first_error = "job: " + std::string(nat_bem_last_error());
  }
  cudaEventRecord(t1, s);
  float ms = 0.f;
  if (cudaEventSynchronize(t1) == cudaSuccess && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess)
    for (int32_t q : bk.jobs) jobs[q].device_ms = ms;
  cleanup();
  return NAT_BEM_OK;
}

}  // namespace
}  // namespace natbem

extern "C" nat_bem_status nat_bem_run_batch_fused(nat_bem_job* jobs, int32_t njobs, const nat_bem_opts* opts,
                                                  int32_t max_batch, int32_t concurrency, void* cuda_stream) {
  using namespace natbem;
  try {
    clear_error();
    if (njobs < 0 || (njobs > 0 && !jobs) || max_batch < 1 || max_batch > 256 || concurrency < 1 ||
        concurrency > 32) {
      set_error("nat_bem_run_batch_fused: need jobs for njobs > 0, 1 <= max_batch <= 256, 1 <= concurrency <= 32");
      return NAT_BEM_EINVAL;
    }
    if (njobs == 0) return NAT_BEM_OK;
    nat_bem_opts o;
    nat_bem_opts_default(&o);
    if (opts) o = *opts;
    NB_TRY(check_opts(o));
    if (concurrency > 1) o.device_loop = 0;  // other workers' streams fill the host round trips
    for (int32_t i = 0; i < njobs; ++i) {
      const nat_bem_job& j = jobs[i];
      if (!j.verts || !j.tris || j.nv <= 0 || j.nt <= 0 || j.nt > (1 << 30) || j.nrhs < 1 || !j.neumann ||
          !j.p_out || j.m < 0 || (j.m > 0 && (!j.pts || !j.field_out)) || !(j.k > 0.0) || !std::isfinite(j.k)) {
        set_error("nat_bem_run_batch_fused: job " + std::to_string(i) + " has a bad argument");
        return NAT_BEM_EINVAL;
      }
    }
    cudaStream_t user = (cudaStream_t)cuda_stream;
    int dev = 0;
    NB_TRY_CUDA(cudaGetDevice(&dev));
    // meshes with several right-hand sides keep their own solve (their products are GEMMs)
    std::vector<int32_t> fused, single;
    for (int32_t i = 0; i < njobs; ++i) (jobs[i].nrhs == 1 ? fused : single).push_back(i);
    std::stable_sort(fused.begin(), fused.end(), [&](int32_t a, int32_t b) { return jobs[a].nt > jobs[b].nt; });
    const bool bf16 = low_copy(o);
    std::vector<Bucket> buckets;
    for (int32_t q : fused) {
      const int64_t nt = jobs[q].nt;
      if (buckets.empty() || (double)nt * kBucketRatio < (double)buckets.back().N ||
          (int)buckets.back().jobs.size() >= max_batch ||
          op_bytes(buckets.back().N, bf16) * (int64_t)(buckets.back().jobs.size() + 1) > kBucketBytes) {
        buckets.push_back(Bucket{});
        buckets.back().N = nt;
      }
      buckets.back().jobs.push_back(q);
    }
    // work items: the buckets (largest first), then the single jobs; `concurrency` workers with
    // their own streams take them in order, so one bucket's host-side mesh checks and assembly
    // overlap another's solve
    const int items = (int)buckets.size() + (int)single.size();
    const int nw = std::max(1, std::min<int>(concurrency, items));
    cudaEvent_t start = nullptr;
    NB_TRY_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    NB_TRY_CUDA(cudaEventRecord(start, user));  // inputs written on the caller's stream
    std::vector<cudaStream_t> streams(nw, nullptr);
    for (auto& st : streams)
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(st, start, 0) != cudaSuccess) {
        cudaGetLastError();
        for (auto& x : streams)
          if (x) cudaStreamDestroy(x);
        cudaEventDestroy(start);
        set_error("nat_bem_run_batch_fused: could not create worker streams");
        return NAT_BEM_ECUDA;
      }
    std::atomic<int> next{0};
    std::mutex err_mu;
    std::string first_error;
    auto work = [&](int wi) {
      cudaSetDevice(dev);
      cudaStream_t s = streams[wi];
      for (;;) {
        const int it = next.fetch_add(1);
        if (it >= items) break;
        std::string err;
        if (it < (int)buckets.size()) {
          run_bucket(jobs, buckets[it], o, s, err);
        } else {
          nat_bem_job& j = jobs[single[it - buckets.size()]];
          nat_bem_op* op = nullptr;
          cudaEvent_t e0 = nullptr, e1 = nullptr;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          cudaEventRecord(e0, s);
          nat_bem_status st =
              build_mesh_op(j.verts, j.nv, j.tris, j.nt, j.k, o, s, 0, nullptr, nullptr, nullptr, nullptr, &op);
          if (st == NAT_BEM_OK) st = nat_bem_solve(op, j.neumann, j.nrhs, j.p_out, &j.info, s);
          if ((st == NAT_BEM_OK || st == NAT_BEM_ENOCONV) && j.m > 0) {
            const nat_bem_status se = nat_bem_eval(op, j.pts, j.m, j.p_out, j.neumann, j.nrhs, j.field_out, s);
            if (se != NAT_BEM_OK) st = se;
          }
          cudaEventRecord(e1, s);
          float ms = 0.f;
          if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            j.device_ms = ms;
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          nat_bem_destroy(op);
          j.status = st;
          if (st != NAT_BEM_OK) err = "job: " + std::string(nat_bem_last_error());
        }
        if (!err.empty()) {
          std::lock_guard<std::mutex> lk(err_mu);
          if (first_error.empty()) first_error = err;
        }
      }
      cudaStreamSynchronize(s);
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nw; ++w) threads.emplace_back(work, w);
    work(0);
    for (auto& t : threads) t.join();
    for (auto& st : streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    cudaEventDestroy(start);
    nat_bem_status worst = NAT_BEM_OK;
    for (int32_t i = 0; i < njobs; ++i)
      if (jobs[i].status != NAT_BEM_OK && (worst == NAT_BEM_OK || worst == NAT_BEM_ENOCONV)) worst = jobs[i].status;
    if (worst != NAT_BEM_OK) set_error(first_error);
    return worst;
  } catch (...) {
    set_error("internal error in nat_bem_run_batch_fused");
    return NAT_BEM_ECUDA;
  }
}
