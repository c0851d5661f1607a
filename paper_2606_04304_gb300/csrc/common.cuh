// Internal helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/ovro.h"

namespace ovro {

// Records the message of a failed CUDA call for ovro_last_error().
void set_last_error(const char* where, cudaError_t e);
// Counts kernel launches made by the library (ovro_launch_count()).
void count_launch();
// printf-style message for ovro_last_error().
void snprintf_last_error(const char* fmt, ...);

// Optional kernel tracing (ovro_profile): when enabled, CUDA events are
// recorded on the launch stream around each traced kernel.
bool profiling();
void prof_mark(const char* name, cudaStream_t st, bool begin);
// Adds n to the launch counter (kernels replayed by a CUDA graph launch).
void add_launches(unsigned long long n);
// Removes n from it (launches recorded into a graph capture, counted at replay).
void sub_launches(unsigned long long n);

// True while `st` is being captured into a CUDA graph (tracing is skipped then).
inline bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Tracing inside a CUDA graph: while a trace list is installed for the
// capturing thread, traced launches record external event nodes into the
// graph (begin/end per launch); graph_trace_collect adds their elapsed times
// to the trace after the graph has run.
struct GraphTraceEntry {
  const char* name;
  cudaEvent_t begin, end;
};
void set_capture_trace(std::vector<GraphTraceEntry>* list);   // nullptr: none
void graph_mark(const char* name, cudaStream_t st, bool begin);
bool graph_tracing();
void graph_trace_collect(const std::vector<GraphTraceEntry>& list);
void graph_trace_free(std::vector<GraphTraceEntry>& list);

struct ProfScope {
  const char* name;
  cudaStream_t st;
  int mode;          // 0 off, 1 stream events, 2 graph event nodes
  ProfScope(const char* n, cudaStream_t s) : name(n), st(s), mode(0) {
    if (!profiling()) return;
    if (!capturing(s)) mode = 1;
    else if (graph_tracing()) mode = 2;
    if (mode == 1) prof_mark(name, st, true);
    if (mode == 2) graph_mark(name, st, true);
  }
  ~ProfScope() {
    if (mode == 1) prof_mark(name, st, false);
    if (mode == 2) graph_mark(name, st, false);
  }
};
#define OVRO_PROF(name, st) ::ovro::ProfScope ovro_prof_scope_(name, st)

#define OVRO_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) {                                  \
      ::ovro::set_last_error(#expr, e_);                      \
      return OVRO_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

#define OVRO_LAUNCH_CHECK()                                   \
  do {                                                        \
    ::ovro::count_launch();                                   \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) {                                  \
      ::ovro::set_last_error("kernel launch", e_);            \
      return OVRO_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
inline int ilog2(long long x) { int r = 0; while ((1LL << r) < x) ++r; return r; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves 256-byte aligned sub-buffers out of a caller workspace.
struct Carver {
  char* base;
  size_t used = 0;
  size_t cap;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count) {
    used = align_up(used, 256);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += count * sizeof(T);
    return p;
  }
  bool ok() const { return used <= cap; }
};

inline int check_workspace(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return OVRO_OK;
  if (ws == nullptr || ws_bytes < need) return OVRO_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return OVRO_ERR_WORKSPACE;
  return OVRO_OK;
}

inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// ---- device helpers ------------------------------------------------------
// Order-preserving map float -> uint32 (total order, -0 < +0 irrelevant here).
__device__ __forceinline__ uint32_t f2key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

}  // namespace ovro
