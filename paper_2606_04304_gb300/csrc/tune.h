// Launch-shape autotuner (tune.cu): cached choices per (kernel, shape) key.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <initializer_list>
#include <string>
#include <vector>

namespace ovro {

// Tuning is enabled (ovro_autotune) and `st` is not being captured.
bool tuning(cudaStream_t st);
// Cached choice for key, or fallback.
int tuned(const std::string& key, int fallback);
// Times run(c) for every candidate c (each run must leave the same results),
// caches and returns the fastest in *chosen.  A cached key is not re-timed.
int tune_pick(const std::string& key, const std::vector<int>& cands, const std::function<int(int)>& run,
              cudaStream_t st, int* chosen);
// "kernel/sm<count>/<shape...>"
std::string tune_key(const char* kernel, std::initializer_list<long long> shape);

}  // namespace ovro
