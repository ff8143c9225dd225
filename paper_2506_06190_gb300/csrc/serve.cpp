// Serving loop: requests (nat_bem_job) arrive at any time through nat_bem_submit and are
// admitted in arrival order as worker slots and device memory free up. Each admitted request
// reserves the device bytes its op and solver workspace need (nat_bem_required_bytes) against
// the server's budget, runs on its worker's own stream (assemble, GMRES, field) beside the
// other admitted requests, and releases the bytes when its op is destroyed. This is continuous
// batching: a request arriving while others are on the GPU starts as soon as a slot and its
// memory are free, without waiting for a batch boundary. A request larger than the whole
// budget is refused with NAT_BEM_ENOMEM. nat_bem_wait blocks (with a timeout) for one ticket.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

struct nat_bem_server {
  int64_t budget = 0;
  int64_t reserved = 0;
  nat_bem_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // workers: a request or memory became available
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<int64_t> pending;       // tickets in arrival order
  struct Entry {
    nat_bem_job* job;
    bool done;
    double submit_s, start_s, finish_s;
  };
  std::map<int64_t, Entry> entries;
  int64_t next_ticket = 1;
  bool stop = false;
  bool fake = false;                 // host-logic test mode: no device work (see create)
  std::vector<std::thread> workers;
};

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Test mode without a GPU: a request "runs" for nt / 1e5 seconds and succeeds, so admission
// order, budget accounting, refusals and timeouts can be checked on the host.
nat_bem_status fake_run(nat_bem_job* job) {
  std::this_thread::sleep_for(std::chrono::microseconds(job->nt * 10));
  job->info.iterations = 1;
  job->info.refinements = 0;
  job->info.rel_residual = 0.0;
  job->device_ms = (float)(job->nt * 1e-2);
  return NAT_BEM_OK;
}

void worker_loop(nat_bem_server* srv) {
  cudaStream_t stream = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (!srv->fake) {
    cudaSetDevice(srv->device);
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
  }
  for (;;) {
    int64_t ticket = 0;
    nat_bem_job* job = nullptr;
    int64_t need = 0;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      for (;;) {
        if (srv->stop) goto out;
        if (!srv->pending.empty()) {
          const int64_t t = srv->pending.front();
          nat_bem_job* j = srv->entries[t].job;
          need = nat_bem_required_bytes(j->nt, j->nrhs, &srv->opts);
          if (need > srv->budget) {  // can never fit: refuse
            srv->pending.pop_front();
            j->status = NAT_BEM_ENOMEM;
            auto& e = srv->entries[t];
            e.done = true;
            e.start_s = e.finish_s = now_s();
            srv->cv_done.notify_all();
            continue;
          }
          if (srv->reserved + need <= srv->budget) {  // admit in arrival order
            srv->pending.pop_front();
            srv->reserved += need;
            ticket = t;
            job = j;
            srv->entries[t].start_s = now_s();
            break;
          }
        }
        srv->cv_work.wait(lk);
      }
    }
    nat_bem_status st = NAT_BEM_OK;
    if (srv->fake) {
      st = fake_run(job);
    } else {
      nat_bem_op* op = nullptr;
      cudaEventRecord(t0, stream);
      st = nat_bem_assemble(job->verts, job->nv, job->tris, job->nt, job->k, &srv->opts, stream, &op);
      if (st == NAT_BEM_OK)
        st = nat_bem_solve(op, job->neumann, job->nrhs, job->p_out, &job->info, stream);
      if ((st == NAT_BEM_OK || st == NAT_BEM_ENOCONV) && job->m > 0) {
        const nat_bem_status se = nat_bem_eval(op, job->pts, job->m, job->p_out, job->neumann,
                                               job->nrhs, job->field_out, stream);
        if (se != NAT_BEM_OK) st = se;
      }
      cudaEventRecord(t1, stream);
      nat_bem_destroy(op);
      cudaStreamSynchronize(stream);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) job->device_ms = ms;
    }
    job->status = st;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->reserved -= need;
      auto& e = srv->entries[ticket];
      e.done = true;
      e.finish_s = now_s();
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
out:
  if (!srv->fake) {
    cudaStreamDestroy(stream);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
  }
}

}  // namespace

using namespace natbem;

extern "C" {

nat_bem_status nat_bem_server_create(int64_t budget_bytes, const nat_bem_opts* opts, int32_t slots,
                                     nat_bem_server** out) {
  try {
    clear_error();
    if (!out || budget_bytes <= 0 || slots < 1 || slots > 64) {
      set_error("nat_bem_server_create: need out, budget_bytes > 0 and 1 <= slots <= 64");
      return NAT_BEM_EINVAL;
    }
    *out = nullptr;
    nat_bem_server* srv = new nat_bem_server();
    srv->budget = budget_bytes;
    nat_bem_opts_default(&srv->opts);
    if (opts) srv->opts = *opts;
    if (slots > 1) srv->opts.device_loop = 0;  // other slots' streams fill the host round trips
    const char* fake = std::getenv("NATBEM_SERVER_FAKE");
    srv->fake = fake && fake[0] == '1';
    if (!srv->fake && cudaGetDevice(&srv->device) != cudaSuccess) {
      cudaGetLastError();
      delete srv;
      set_error("nat_bem_server_create: no CUDA device");
      return NAT_BEM_ECUDA;
    }
    for (int i = 0; i < slots; ++i) srv->workers.emplace_back(worker_loop, srv);
    *out = srv;
    return NAT_BEM_OK;
  } catch (...) {
    set_error("internal error in nat_bem_server_create");
    return NAT_BEM_ECUDA;
  }
}

nat_bem_status nat_bem_submit(nat_bem_server* srv, nat_bem_job* job, int64_t* ticket) {
  clear_error();
  if (!srv || !job || !ticket || job->nt <= 0 || job->nrhs < 1) {
    set_error("nat_bem_submit: bad arguments");
    return NAT_BEM_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) {
      set_error("nat_bem_submit: server is shutting down");
      return NAT_BEM_EBUSY;
    }
    const int64_t t = srv->next_ticket++;
    job->status = NAT_BEM_EBUSY;  // in flight
    srv->entries[t] = {job, false, now_s(), 0.0, 0.0};
    srv->pending.push_back(t);
    *ticket = t;
  }
  srv->cv_work.notify_all();
  return NAT_BEM_OK;
}

nat_bem_status nat_bem_wait(nat_bem_server* srv, int64_t ticket, int32_t timeout_ms,
                            double* queue_ms, double* total_ms) {
  clear_error();
  if (!srv) {
    set_error("nat_bem_wait: server is NULL");
    return NAT_BEM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->entries.find(ticket);
  if (it == srv->entries.end()) {
    set_error("nat_bem_wait: unknown ticket");
    return NAT_BEM_EINVAL;
  }
  const auto pred = [&] { return srv->entries[ticket].done; };
  if (timeout_ms < 0) {
    srv->cv_done.wait(lk, pred);
  } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    set_error("nat_bem_wait: timed out");
    return NAT_BEM_ETIMEOUT;
  }
  const auto e = srv->entries[ticket];
  srv->entries.erase(ticket);
  if (queue_ms) *queue_ms = 1e3 * (e.start_s - e.submit_s);
  if (total_ms) *total_ms = 1e3 * (e.finish_s - e.submit_s);
  return e.job->status;
}

int64_t nat_bem_server_reserved(nat_bem_server* srv) {
  if (!srv) return 0;
  std::lock_guard<std::mutex> lk(srv->mu);
  return srv->reserved;
}

void nat_bem_server_destroy(nat_bem_server* srv) {
  if (!srv) return;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    // let admitted and queued requests finish
    srv->cv_done.wait(lk, [&] {
      for (const auto& kv : srv->entries)
        if (!kv.second.done) return false;
      return true;
    });
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  delete srv;
}

}  // extern "C"
