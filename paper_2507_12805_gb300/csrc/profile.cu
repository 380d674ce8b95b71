// Sampled per-kernel timing with CUDA events on the launching stream.
//
// When enabled, every `every`-th global step of the compress/decompress loop
// brackets each kernel launch with two events and records the launch's
// algorithmic work (FLOPs of the contraction it performs, or bytes it must
// move), computed on the host from the rows that step actually predicts.
// pmklc_profile_read() synchronises the events and returns per-kernel totals,
// so achieved FLOP/s or bytes/s = work / time over the sampled launches.
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace pmklc {

namespace {
struct Rec {
  const char *name;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct Prof {
  int every = 0;
  bool on = false;  // current step sampled
  StepWork work{};
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};
Prof g_prof;
}  // namespace

void prof_step(int T, const StepWork &w) {
  g_prof.on = g_prof.every > 0 && (T % g_prof.every) == 0;
  g_prof.work = w;
}
void prof_stop_sampling() { g_prof.on = false; }
bool prof_enabled() { return g_prof.every > 0; }
const StepWork &prof_work() { return g_prof.work; }

ProfScope::ProfScope(const char *name, double flops, double bytes, cudaStream_t st)
    : name_(name), flops_(flops), bytes_(bytes), st_(st), active_(g_prof.on) {
  if (!active_) return;
  a_ = g_prof.get();
  cudaEventRecord((cudaEvent_t)a_, st_);
}

ProfScope::~ProfScope() {
  if (!active_) return;
  cudaEvent_t b = g_prof.get();
  cudaEventRecord(b, st_);
  g_prof.recs.push_back(Rec{name_, (cudaEvent_t)a_, b, flops_, bytes_});
}

bool smem_optin(const void *func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> done;  // (kernel, device) -> limit set
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(mu);
  int &have = done[{func, dev}];
  if (have >= bytes) return true;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
  have = bytes;
  return true;
}

}  // namespace pmklc

using namespace pmklc;

extern "C" int pmklc_profile_enable(int every) {
  if (every < 0) return PMKLC_EINVAL;
  g_prof.every = every;
  g_prof.on = false;
  return PMKLC_OK;
}

extern "C" int pmklc_profile_read(pmklc_kernel_prof *out, int max, int *n) {
  if (!n || (max > 0 && !out)) return PMKLC_EINVAL;
  std::vector<pmklc_kernel_prof> agg;
  for (Rec &r : g_prof.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return PMKLC_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    pmklc_kernel_prof *slot = nullptr;
    for (auto &x : agg)
      if (strcmp(x.name, r.name) == 0) slot = &x;
    if (!slot) {
      agg.push_back(pmklc_kernel_prof{});
      slot = &agg.back();
      strncpy(slot->name, r.name, sizeof(slot->name) - 1);
    }
    slot->launches++;
    slot->ms += ms;
    slot->flops += r.flops;
    slot->bytes += r.bytes;
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  *n = (int)agg.size();
  for (int i = 0; i < (int)agg.size() && i < max; ++i) out[i] = agg[i];
  return PMKLC_OK;
}
