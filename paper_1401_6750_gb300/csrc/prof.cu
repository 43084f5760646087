// Per-kernel-class timing with CUDA events (opt-in).  While profiling is on,
// the solver runs one CG iteration per chunk without graphs and brackets each
// kernel with events on the launching stream; every launch adds its measured
// duration and its algorithmic bytes and flops (compulsory traffic of the
// operation, each operand counted once) to the class totals.
#include <string.h>

#include <atomic>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace tsm {

namespace {
struct Entry {
  long long launches = 0;
  double seconds = 0.0, bytes = 0.0, flops = 0.0;
};
std::mutex g_mu;
bool g_on = false;
std::atomic<long long> g_launches{0};
std::map<std::string, Entry> g_tab;
}  // namespace

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool profiling() {
  std::lock_guard<std::mutex> l(g_mu);
  return g_on;
}

void prof_add(const char* name, double seconds, double bytes, double flops) {
  std::lock_guard<std::mutex> l(g_mu);
  if (!g_on) return;
  Entry& e = g_tab[name];
  e.launches += 1;
  e.seconds += seconds;
  e.bytes += bytes;
  e.flops += flops;
}

int EventPair::begin(cudaStream_t s) {
  if (!a) TSM_CUDA(cudaEventCreate(&a));
  if (!b) TSM_CUDA(cudaEventCreate(&b));
  TSM_CUDA(cudaEventRecord(a, s));
  return TSM_OK;
}
int EventPair::end(cudaStream_t s) {
  TSM_CUDA(cudaEventRecord(b, s));
  return TSM_OK;
}
double EventPair::seconds() {
  float ms = 0.f;
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  return 1e-3 * ms;
}
EventPair::~EventPair() {
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
}

}  // namespace tsm

extern "C" {

long long tsm_kernel_launches(void) { return tsm::g_launches.load(); }

int tsm_profile_enable(int on) {
  std::lock_guard<std::mutex> l(tsm::g_mu);
  if (on && !tsm::g_on) tsm::g_tab.clear();
  tsm::g_on = (on != 0);
  return TSM_OK;
}

int tsm_profile_read(tsm_kernel_profile* out, int cap) {
  std::lock_guard<std::mutex> l(tsm::g_mu);
  int k = 0;
  for (auto& kv : tsm::g_tab) {
    if (out && k < cap) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
      out[k].launches = kv.second.launches;
      out[k].seconds = kv.second.seconds;
      out[k].bytes = kv.second.bytes;
      out[k].flops = kv.second.flops;
    }
    ++k;
  }
  return k;
}

}  // extern "C"
