// Launch accounting and optional per-kernel-class CUDA-event timing.
// Every launcher in k_*.cu opens a ProfScope around its launches; when
// timing is enabled the scope records an event pair on the launching stream
// (events come from a reusable pool), and nne_prof_collect sums the elapsed
// times per class after synchronising.
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

namespace nne {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_mu;

struct EvRec {
  cudaEvent_t a, b;
  int cls;
};
static std::vector<cudaEvent_t> g_pool;
static std::vector<EvRec> g_recs;
static long long g_prof_counts[PROF_CLASSES];
static double g_prof_work[PROF_CLASSES];

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(cudaStream_t st, int cls, int kernels, double work)
    : st_(st), cls_(cls), on_(false), work_(work) {
  g_launches.fetch_add(kernels, std::memory_order_relaxed);
  if (g_prof_on.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    b_ = take_event();
    cudaEventRecord(a_, st_);
    on_ = true;
  }
}

ProfScope::~ProfScope() {
  if (on_) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(b_, st_);
    g_recs.push_back({a_, b_, cls_});
    if (cls_ >= 0 && cls_ < PROF_CLASSES) {
      g_prof_counts[cls_]++;
      g_prof_work[cls_] += work_;
    }
  }
}

struct AttrKey {
  const void* f;
  int dev;
  bool operator==(const AttrKey& o) const { return f == o.f && dev == o.dev; }
};
struct AttrHash {
  size_t operator()(const AttrKey& k) const { return std::hash<const void*>()(k.f) ^ (size_t)k.dev; }
};
static std::mutex g_attr_mu;
static std::unordered_map<AttrKey, std::pair<int, bool>, AttrHash> g_attr;

cudaError_t ensure_kernel_smem(const void* func, size_t bytes, bool nonportable_cluster) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto& a = g_attr[AttrKey{func, dev}];
  if ((int)bytes > a.first) {
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    a.first = (int)bytes;
  }
  if (nonportable_cluster && !a.second) {
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    a.second = true;
  }
  return cudaSuccess;
}

}  // namespace nne

using namespace nne;

extern "C" {

long long nne_kernel_launches(void) { return g_launches.load(); }

void nne_prof_enable(int on) { g_prof_on.store(on ? 1 : 0); }

int nne_prof_collect(double* ms_out, long long* count_out, double* work_out, int n_classes) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<double> ms(PROF_CLASSES, 0.0);
  for (auto& r : g_recs) {
    cudaEventSynchronize(r.b);
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.cls >= 0 && r.cls < PROF_CLASSES) ms[r.cls] += t;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  const int m = n_classes < PROF_CLASSES ? n_classes : PROF_CLASSES;
  for (int i = 0; i < m; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (count_out) count_out[i] = g_prof_counts[i];
    if (work_out) work_out[i] = g_prof_work[i];
    g_prof_counts[i] = 0;
    g_prof_work[i] = 0;
  }
  return PROF_CLASSES;
}

}  // extern "C"
