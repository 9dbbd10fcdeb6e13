// Launch counting and optional CUDA-event timing of the GEMM kernel classes (C ABI in gfcc.h).
#include "gfcc_internal.cuh"

#include <atomic>
#include <mutex>

namespace gfcc {
namespace {
std::atomic<long long> g_launches{0};
struct Rec {
  cudaEvent_t a, b;
  int cls;
  double flops;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
// events are created once and reused by later profiling runs (creating two per region would put
// host work into the timed stream's gaps)
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;
bool take_event(cudaEvent_t* e) {
  if (g_used == g_pool.size()) {
    cudaEvent_t n;
    if (cudaEventCreate(&n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    g_pool.push_back(n);
  }
  *e = g_pool[g_used++];
  return true;
}
std::atomic<bool> g_alloc_on{false};
long long g_alloc_n[2] = {0, 0};
double g_alloc_ms[2] = {0.0, 0.0};
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool alloc_profiling() { return g_alloc_on.load(std::memory_order_relaxed); }
void note_alloc(int cls, double ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int k = cls == PROF_FREE ? 1 : 0;
  ++g_alloc_n[k];
  g_alloc_ms[k] += ms;
}

ProfScope::ProfScope(int c, double f, cudaStream_t st) : cls(c), flops(f), s(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  Rec* r = new Rec{};
  r->cls = c;
  r->flops = f;
  if (!take_event(&r->a) || !take_event(&r->b)) {
    delete r;
    return;
  }
  cudaEventRecord(r->a, s);
  rec = r;
}
ProfScope::~ProfScope() {
  if (!rec) return;
  Rec* r = static_cast<Rec*>(rec);
  cudaEventRecord(r->b, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(*r);
  delete r;
}

}  // namespace gfcc

extern "C" {

long long gfcc_launch_count(void) { return gfcc::g_launches.load(); }

int gfcc_profile(int enable) {
  std::lock_guard<std::mutex> lk(gfcc::g_mu);
  for (auto& r : gfcc::g_recs) {   // the pooled events are reused once their records have completed
    cudaEventSynchronize(r.b);
  }
  cudaGetLastError();
  gfcc::g_recs.clear();
  gfcc::g_used = 0;
  gfcc::g_on = enable != 0;
  gfcc::g_alloc_n[0] = gfcc::g_alloc_n[1] = 0;
  gfcc::g_alloc_ms[0] = gfcc::g_alloc_ms[1] = 0.0;
  gfcc::g_alloc_on.store(enable != 0);
  return GFCC_OK;
}

int gfcc_profile_read(int cls, long long* launches, double* ms, double* flops) {
  if (cls < 0 || cls >= gfcc::PROF_NCLASS) return GFCC_ERR_ARG;
  std::lock_guard<std::mutex> lk(gfcc::g_mu);
  if (cls == gfcc::PROF_ALLOC || cls == gfcc::PROF_FREE) {   // host-side counts, no events
    const int k = cls == gfcc::PROF_FREE ? 1 : 0;
    if (launches) *launches = gfcc::g_alloc_n[k];
    if (ms) *ms = gfcc::g_alloc_ms[k];
    if (flops) *flops = 0.0;
    return GFCC_OK;
  }
  long long n = 0;
  double t = 0.0, f = 0.0;
  for (auto& r : gfcc::g_recs) {
    if (r.cls != cls) continue;
    float e = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return GFCC_ERR_CUDA;
    }
    ++n;
    t += e;
    f += r.flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return GFCC_OK;
}

}  // extern "C"
