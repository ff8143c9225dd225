// Batched solves: a pool of workers, each with its own CUDA stream and op, pulls jobs (mesh,
// wavenumber, Neumann data, field points) from a shared queue. A worker whose next job has
// the same mesh as its current op re-assembles that op at the new wavenumber (no mesh checks,
// geometry or allocation), otherwise it builds a new op. The workers' solves overlap on the
// device, so one job's latency-bound Krylov steps run beside another's bandwidth-bound matvecs
// and assembly. Jobs are taken largest mesh first, which keeps uneven batches balanced.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

struct Worker {
  cudaStream_t stream = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  nat_bem_op* op = nullptr;
  const double* verts = nullptr;
  const int32_t* tris = nullptr;
  int64_t nv = 0, nt = 0;
};

bool same_mesh(const Worker& w, const nat_bem_job& j) {
  return w.op && w.verts == j.verts && w.tris == j.tris && w.nv == j.nv && w.nt == j.nt;
}

}  // namespace

extern "C" nat_bem_status nat_bem_run_batch(nat_bem_job* jobs, int32_t njobs,
                                            const nat_bem_opts* opts, int32_t concurrency,
                                            void* cuda_stream) {
  using namespace natbem;
  try {
    clear_error();
    if (njobs < 0 || (njobs > 0 && !jobs) || concurrency < 1 || concurrency > 32) {
      set_error("nat_bem_run_batch: need jobs for njobs > 0 and 1 <= concurrency <= 32");
      return NAT_BEM_EINVAL;
    }
    if (njobs == 0) return NAT_BEM_OK;
    int dev = 0;
    NB_TRY_CUDA(cudaGetDevice(&dev));
    cudaStream_t user = (cudaStream_t)cuda_stream;
    cudaEvent_t start = nullptr;
    NB_TRY_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    NB_TRY_CUDA(cudaEventRecord(start, user));  // inputs written on the caller's stream
    // largest meshes first; jobs on the same mesh stay adjacent
    std::vector<int32_t> order(njobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return jobs[a].nt > jobs[b].nt;
    });
    const int nw = std::min<int32_t>(concurrency, njobs);
    std::vector<Worker> workers(nw);
    for (auto& w : workers) {
      if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreate(&w.t0) != cudaSuccess || cudaEventCreate(&w.t1) != cudaSuccess ||
          cudaStreamWaitEvent(w.stream, start, 0) != cudaSuccess) {
        cudaGetLastError();
        for (auto& x : workers)
          if (x.stream) cudaStreamDestroy(x.stream);
        cudaEventDestroy(start);
        set_error("nat_bem_run_batch: could not create worker streams");
        return NAT_BEM_ECUDA;
      }
    }
    // with several workers, other streams fill the host round trips between GMRES chunks, and
    // the device-side loop measured slower there: host-polled chunks
    nat_bem_opts wo;
    nat_bem_opts_default(&wo);
    if (opts) wo = *opts;
    if (nw > 1) wo.device_loop = 0;
    std::atomic<int32_t> next{0};
    std::mutex err_mu;
    std::string first_error;
    auto run = [&](int wi) {
      cudaSetDevice(dev);
      Worker& w = workers[wi];
      for (;;) {
        const int32_t q = next.fetch_add(1);
        if (q >= njobs) break;
        nat_bem_job& j = jobs[order[q]];
        nat_bem_status st = NAT_BEM_OK;
        cudaEventRecord(w.t0, w.stream);
        if (same_mesh(w, j)) {
          st = nat_bem_reassemble(w.op, j.k, w.stream);
        } else {
          nat_bem_destroy(w.op);
          w.op = nullptr;
          st = nat_bem_assemble(j.verts, j.nv, j.tris, j.nt, j.k, &wo, w.stream, &w.op);
          if (st == NAT_BEM_OK) {
            w.verts = j.verts;
            w.tris = j.tris;
            w.nv = j.nv;
            w.nt = j.nt;
          }
        }
        if (st == NAT_BEM_OK || st == NAT_BEM_ENOCONV)
          st = nat_bem_solve(w.op, j.neumann, j.nrhs, j.p_out, &j.info, w.stream);
        if ((st == NAT_BEM_OK || st == NAT_BEM_ENOCONV) && j.m > 0) {
          const nat_bem_status se = nat_bem_eval(w.op, j.pts, j.m, j.p_out, j.neumann, j.nrhs,
                                                 j.field_out, w.stream);
          if (se != NAT_BEM_OK) st = se;
        }
        cudaEventRecord(w.t1, w.stream);
        float ms = 0.f;
        if (cudaEventSynchronize(w.t1) == cudaSuccess && cudaEventElapsedTime(&ms, w.t0, w.t1) == cudaSuccess)
          j.device_ms = ms;
        j.status = st;
        if (st != NAT_BEM_OK) {
          std::lock_guard<std::mutex> lk(err_mu);
          if (first_error.empty())
            first_error = "job " + std::to_string(order[q]) + ": " + nat_bem_last_error();
        }
      }
      cudaStreamSynchronize(w.stream);
    };
    std::vector<std::thread> threads;
    for (int i = 1; i < nw; ++i) threads.emplace_back(run, i);
    run(0);
    for (auto& t : threads) t.join();
    for (auto& w : workers) {
      nat_bem_destroy(w.op);
      cudaStreamSynchronize(w.stream);
      cudaStreamDestroy(w.stream);
      cudaEventDestroy(w.t0);
      cudaEventDestroy(w.t1);
    }
    cudaEventDestroy(start);
    nat_bem_status worst = NAT_BEM_OK;
    for (int32_t i = 0; i < njobs; ++i)
      if (jobs[i].status != NAT_BEM_OK && (worst == NAT_BEM_OK || worst == NAT_BEM_ENOCONV))
        worst = jobs[i].status;
    if (worst != NAT_BEM_OK) set_error(first_error);
    return worst;
  } catch (...) {
    set_error("internal error in nat_bem_run_batch");
    return NAT_BEM_ECUDA;
  }
}
