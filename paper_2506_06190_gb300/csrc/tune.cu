// Launch-shape autotuning shared by the assembly and the field evaluation: the first time a
// (device, kind, size class) is met, every candidate shape runs on the actual operands, timed
// with CUDA events on the caller's stream (one warm-up round, then three interleaved rounds,
// each candidate's minimum: kernels of other streams only slow a run down). Candidate 0 is the
// untuned default and wins ties within 2%. The choice is kept for the life of the process.
// NATBEM_NO_TUNE in the environment keeps every default.
#include <cuda_runtime.h>

#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace natbem {
namespace {
std::mutex g_mu;
std::map<std::tuple<int, std::string, int64_t>, int> g_choice;
}  // namespace

int autotune(const char* kind, int64_t size_class, int ncand, const std::function<nat_bem_status(int)>& run,
             cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || ncand <= 1 || std::getenv("NATBEM_NO_TUNE")) return 0;
  const auto key = std::make_tuple(dev, std::string(kind), size_class);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto f = g_choice.find(key);
    if (f != g_choice.end()) return f->second;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return 0;
  }
  std::vector<float> best(ncand, 1e30f);
  bool ok = true;
  for (int round = 0; round < 4 && ok; ++round)
    for (int c = 0; c < ncand && ok; ++c) {
      cudaEventRecord(e0, s);
      ok = run(c) == NAT_BEM_OK;
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        if (round > 0) best[c] = std::min(best[c], ms);
      } else {
        ok = false;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int pick = 0;
  if (ok)
    for (int c = 1; c < ncand; ++c)
      if (best[c] < 0.98f * best[pick]) pick = c;
  std::lock_guard<std::mutex> lk(g_mu);
  g_choice[key] = pick;
  return pick;
}

}  // namespace natbem
