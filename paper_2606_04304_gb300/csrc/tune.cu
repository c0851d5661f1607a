// Launch-shape autotuner.
//
// A tunable launch site names a key (kernel and problem shape) and a short
// list of candidate values (CTAs per SM, channels per launch, ...) that give
// identical results.  While tuning is enabled and the stream is not being
// captured into a graph, the first use of a key runs every candidate once to
// warm up and once timed with CUDA events, and keeps the fastest; later uses
// (and graph captures) read the cached choice.  The cache can be saved to and
// loaded from a text file ("key value" per line).
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "common.cuh"
#include "tune.h"

namespace ovro {
namespace {
std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_on = false;
}  // namespace

bool tuning(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on && !capturing(st);
}

int tuned(const std::string& key, int fallback) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  return it == g_cache.end() ? fallback : it->second;
}

int tune_pick(const std::string& key, const std::vector<int>& cands, const std::function<int(int)>& run,
              cudaStream_t st, int* chosen) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *chosen = it->second;
      return OVRO_OK;
    }
  }
  cudaEvent_t a, b;
  OVRO_CUDA_TRY(cudaEventCreate(&a));
  OVRO_CUDA_TRY(cudaEventCreate(&b));
  int best = cands.empty() ? 0 : cands[0];
  float best_ms = 0.f;
  int err = OVRO_OK;
  for (size_t i = 0; i < cands.size() && !err; ++i) {
    if ((err = run(cands[i]))) break;                 // warm-up
    if (cudaEventRecord(a, st) != cudaSuccess) { err = OVRO_ERR_CUDA; break; }
    if ((err = run(cands[i]))) break;
    if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
      err = OVRO_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best = cands[i];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (err) return err;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best;
  *chosen = best;
  return OVRO_OK;
}

std::string tune_key(const char* kernel, std::initializer_list<long long> shape) {
  std::ostringstream o;
  o << kernel << "/sm" << num_sms();
  for (long long v : shape) o << "/" << v;
  return o.str();
}

}  // namespace ovro

extern "C" {

int ovro_autotune(int enable) {
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  ovro::g_on = enable != 0;
  return OVRO_OK;
}

int ovro_tune_get(const char* key, int* value) {
  if (!key || !value) return OVRO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  auto it = ovro::g_cache.find(key);
  if (it == ovro::g_cache.end()) return OVRO_ERR_INVALID_ARG;
  *value = it->second;
  return OVRO_OK;
}

int ovro_tune_set(const char* key, int value) {
  if (!key || !*key) return OVRO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  ovro::g_cache[key] = value;
  return OVRO_OK;
}

int ovro_tune_count(void) {
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  return static_cast<int>(ovro::g_cache.size());
}

int ovro_tune_clear(void) {
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  ovro::g_cache.clear();
  return OVRO_OK;
}

int ovro_tune_save(const char* path) {
  if (!path) return OVRO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  std::ofstream f(path);
  if (!f) return OVRO_ERR_INVALID_ARG;
  for (const auto& kv : ovro::g_cache) f << kv.first << " " << kv.second << "\n";
  return f ? OVRO_OK : OVRO_ERR_INVALID_ARG;
}

int ovro_tune_load(const char* path) {
  if (!path) return OVRO_ERR_INVALID_ARG;
  std::ifstream f(path);
  if (!f) return OVRO_ERR_INVALID_ARG;
  std::map<std::string, int> got;
  std::string line;
  while (std::getline(f, line)) {
    if (line.empty()) continue;
    std::istringstream in(line);
    std::string k;
    long long v;
    if (!(in >> k >> v) || v < -2147483647LL || v > 2147483647LL) return OVRO_ERR_INVALID_ARG;
    got[k] = static_cast<int>(v);
  }
  std::lock_guard<std::mutex> lk(ovro::g_mu);
  for (const auto& kv : got) ovro::g_cache[kv.first] = kv.second;
  return OVRO_OK;
}

}  // extern "C"
