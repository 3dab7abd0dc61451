// aot_prof.cu - kernel launch counter and an optional per-kernel event
// profiler.  Every launch site is wrapped in AOT_KERNEL(name, stream); while
// profiling is on, a pair of CUDA events brackets the launch on its stream,
// so the measured time is that kernel's device time on that stream.
#include <cstring>
#include <mutex>
#include <vector>

#include "aot_internal.cuh"

namespace aot {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};
ProfState& state() {
  static ProfState* st = new ProfState();  // never destroyed (events outlive exit order)
  return *st;
}
std::atomic<unsigned long long> g_launches{0};

cudaEvent_t take_event(ProfState& st) {
  if (!st.pool.empty()) {
    cudaEvent_t e = st.pool.back();
    st.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t st) : s(st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ProfState& P = state();
  if (!P.on) return;
  std::lock_guard<std::mutex> lk(P.mu);
  Rec r{name, take_event(P), take_event(P)};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, s);
  P.recs.push_back(r);
  slot = (int)P.recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  ProfState& P = state();
  std::lock_guard<std::mutex> lk(P.mu);
  if (slot < (int)P.recs.size()) cudaEventRecord(P.recs[slot].b, s);
}

}  // namespace aot

using namespace aot;

extern "C" unsigned long long aot_kernel_launches(void) {
  return g_launches.load(std::memory_order_relaxed);
}

extern "C" aot_status aot_profile_begin(void) {
  ProfState& P = state();
  std::lock_guard<std::mutex> lk(P.mu);
  for (auto& r : P.recs) {
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  P.recs.clear();
  P.on = true;
  return AOT_OK;
}

extern "C" aot_status aot_profile_end(aot_profile_entry* out, int32_t cap, int32_t* count) {
  if (!count || (cap > 0 && !out)) return AOT_ERR_INVALID_ARG;
  ProfState& P = state();
  std::lock_guard<std::mutex> lk(P.mu);
  P.on = false;
  std::vector<aot_profile_entry> agg;
  for (auto& r : P.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return AOT_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return AOT_ERR_CUDA;
    aot_profile_entry* e = nullptr;
    for (auto& x : agg)
      if (std::strncmp(x.name, r.name, sizeof(x.name)) == 0) e = &x;
    if (!e) {
      aot_profile_entry z;
      std::memset(&z, 0, sizeof z);
      std::strncpy(z.name, r.name, sizeof(z.name) - 1);
      agg.push_back(z);
      e = &agg.back();
    }
    e->launches += 1;
    e->total_ms += ms;
  }
  *count = (int32_t)agg.size();
  for (int32_t i = 0; i < cap && i < (int32_t)agg.size(); ++i) out[i] = agg[i];
  return AOT_OK;
}
