// Measured ceiling of the gridder's accumulation (a measurement aid, no
// counterpart in the paper).  k_grid_rows is bound by shared-memory atomic
// throughput, not by FP32 arithmetic or HBM: every kept visibility adds 49
// complex taps into a 32-row band held as two FP32 planes, one record per
// warp, lane (tv, tu) adding taps (tv, tu) and (tv, tu + 4).  k_probe_accumulate
// runs exactly that pattern (same band shape, pitch and lane map) on
// pseudo-random record origins with no other work, so taps per second here is
// the rate the gridder can at most reach on this GPU.
#include <cstdint>

#include "common.cuh"

namespace ovro {
namespace {

constexpr int kBandH = 32, kG = 512, kPitch = kG + 4, kRecs = 16384;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(1024, 1) k_probe_accumulate(float* __restrict__ sink) {
  extern __shared__ float pl[];
  float* re = pl;
  float* im = pl + kBandH * kPitch;
  for (int i = threadIdx.x; i < 2 * kBandH * kPitch; i += blockDim.x) pl[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const int tv = lane >> 2, tu = lane & 3;
  for (int r = warp; r < kRecs; r += n_warps) {
    const uint32_t h = mix32(static_cast<uint32_t>(r) * 7919u + blockIdx.x);
    // origin row <= kBandH - 8 and column <= kG - 9: taps stay inside the band
    const int row0 = static_cast<int>(h % (kBandH - 7)), col0 = static_cast<int>((h >> 8) % (kG - 8));
    if (tv < 7) {
      const int a = (row0 + tv) * kPitch + col0 + tu;
      const float w = 1.0f + 1e-3f * lane;
      atomicAdd(re + a, w);
      atomicAdd(im + a, -w);
      if (tu < 3) {
        atomicAdd(re + a + 4, w);
        atomicAdd(im + a + 4, -w);
      }
    }
  }
  __syncthreads();
  float s = 0.f;
  for (int i = threadIdx.x; i < 2 * kBandH * kPitch; i += blockDim.x) s += pl[i];
  if (s == 12345.678f) sink[0] = s;            // keeps the work; never true in practice
}

}  // namespace
}  // namespace ovro

extern "C" {

int ovro_probe_accumulate(double* h_gtaps_per_s, void* stream) {
  using namespace ovro;
  if (!h_gtaps_per_s) return OVRO_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  float* sink = nullptr;
  OVRO_CUDA_TRY(cudaMalloc(&sink, sizeof(float)));
  const int smem = 2 * kBandH * kPitch * static_cast<int>(sizeof(float));
  int e = OVRO_OK;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaFuncSetAttribute(k_probe_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    e = OVRO_ERR_CUDA;
  } else {
    const int grid = 4 * num_sms();
    float best = 0.f;
    for (int rep = 0; rep < 3 && !e; ++rep) {
      cudaEventRecord(a, st);
      k_probe_accumulate<<<grid, 1024, smem, st>>>(sink);
      count_launch();
      cudaEventRecord(b, st);
      if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        e = OVRO_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (!e) *h_gtaps_per_s = static_cast<double>(grid) * kRecs * 49 / (best * 1e-3) / 1e9;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  return e;
}

}  // extern "C"
