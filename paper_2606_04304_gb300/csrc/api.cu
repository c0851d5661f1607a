// Status codes, error reporting and version of the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace ovro {
static thread_local char g_last_error[256] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void sub_launches(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

void set_last_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

// ---- tracing
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;
struct ProfRec {
  std::vector<cudaEvent_t> begin, end;
};
static std::map<std::string, ProfRec> g_prof;
// times collected from graph event nodes: name -> (ms, launches)
static std::map<std::string, std::pair<double, int>> g_prof_graph;
static thread_local std::vector<GraphTraceEntry>* g_capture_trace = nullptr;

bool profiling() { return g_prof_on.load(std::memory_order_relaxed); }

void set_capture_trace(std::vector<GraphTraceEntry>* list) { g_capture_trace = list; }
bool graph_tracing() { return g_capture_trace != nullptr; }

void graph_mark(const char* name, cudaStream_t st, bool begin) {
  if (!g_capture_trace) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  if (cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) != cudaSuccess) {
    cudaEventDestroy(e);
    return;
  }
  if (begin) {
    g_capture_trace->push_back(GraphTraceEntry{name, e, nullptr});
  } else {
    // pair with the latest open entry of this name
    for (auto it = g_capture_trace->rbegin(); it != g_capture_trace->rend(); ++it)
      if (it->end == nullptr && std::strcmp(it->name, name) == 0) {
        it->end = e;
        return;
      }
    cudaEventDestroy(e);
  }
}

void graph_trace_collect(const std::vector<GraphTraceEntry>& list) {
  if (!profiling()) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const GraphTraceEntry& t : list) {
    if (!t.end) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.begin, t.end) != cudaSuccess) continue;
    auto& a = g_prof_graph[t.name];
    a.first += ms;
    a.second += 1;
  }
}

void graph_trace_free(std::vector<GraphTraceEntry>& list) {
  for (GraphTraceEntry& t : list) {
    if (t.begin) cudaEventDestroy(t.begin);
    if (t.end) cudaEventDestroy(t.end);
  }
  list.clear();
}

void prof_mark(const char* name, cudaStream_t st, bool begin) {
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec& r = g_prof[name];
  (begin ? r.begin : r.end).push_back(e);
}

static void prof_clear() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& kv : g_prof) {
    for (cudaEvent_t e : kv.second.begin) cudaEventDestroy(e);
    for (cudaEvent_t e : kv.second.end) cudaEventDestroy(e);
  }
  g_prof.clear();
  g_prof_graph.clear();
}

void snprintf_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}
}  // namespace ovro

extern "C" {

const char* ovro_status_string(int status) {
  switch (status) {
    case OVRO_OK: return "OVRO_OK";
    case OVRO_ERR_INVALID_ARG: return "OVRO_ERR_INVALID_ARG";
    case OVRO_ERR_UNSUPPORTED: return "OVRO_ERR_UNSUPPORTED";
    case OVRO_ERR_CUDA: return "OVRO_ERR_CUDA";
    case OVRO_ERR_TIMEOUT: return "OVRO_ERR_TIMEOUT";
    case OVRO_ERR_WORKSPACE: return "OVRO_ERR_WORKSPACE";
    case OVRO_ERR_OVERFLOW: return "OVRO_ERR_OVERFLOW";
    case OVRO_ERR_CAPACITY: return "OVRO_ERR_CAPACITY";
    default: return "OVRO_ERR_UNKNOWN";
  }
}

const char* ovro_last_error(void) { return ovro::g_last_error; }

int ovro_version(void) { return (1 << 16) | 0; }

unsigned long long ovro_launch_count(void) { return ovro::g_launches.load(); }

int ovro_profile(int enable) {
  if (enable) ovro::prof_clear();
  ovro::g_prof_on.store(enable != 0);
  return OVRO_OK;
}

int ovro_profile_query(const char* kernel, double* total_ms, int* launches) {
  if (!kernel || !total_ms || !launches) return OVRO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ovro::g_prof_mu);
  *total_ms = 0.0;
  *launches = 0;
  auto g = ovro::g_prof_graph.find(kernel);
  if (g != ovro::g_prof_graph.end()) {
    *total_ms += g->second.first;
    *launches += g->second.second;
  }
  auto it = ovro::g_prof.find(kernel);
  if (it == ovro::g_prof.end()) return OVRO_OK;
  const auto& r = it->second;
  const size_t n = r.begin.size() < r.end.size() ? r.begin.size() : r.end.size();
  for (size_t i = 0; i < n; ++i) {
    if (cudaEventSynchronize(r.end[i]) != cudaSuccess) return OVRO_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.begin[i], r.end[i]) != cudaSuccess) return OVRO_ERR_CUDA;
    *total_ms += ms;
  }
  *launches += static_cast<int>(n);
  return OVRO_OK;
}

}  // extern "C"
