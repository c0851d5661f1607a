// Status codes, error reporting and version of the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace ovro {
static thread_local char g_last_error[256] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_last_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
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

}  // extern "C"
