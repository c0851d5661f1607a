// Stage interfaces shared by the public entry points and the pipeline driver.
//
// Every stage is split into host planning (no device work), a one-off upload
// of its tables into the caller's workspace, and enqueue-only calls that
// launch kernels and stream-ordered memsets but never copy from pageable host
// memory or synchronise -- those can be captured into a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/ovro.h"

namespace ovro {

// ---- a4: X-engine (xengine.cu)
// reset_status: clear the device timeout word first (the public call does; the
// pipeline clears it once per run so a timeout in any coarse channel sticks).
int correlate_enqueue(const int8_t* d_fine_q, int n_ant, int n_chan, int n_spec, int mode, int32_t* d_vis,
                      cudaStream_t st, bool reset_status);
int correlate_reset_status(cudaStream_t st);

// ---- a5-a7: gridding and imaging (imaging.cu)
struct GridCtx;
size_t grid_ctx_workspace(int n_ant, int n_chan, int image_size, int storage);
// Plans one call's worth of channels; the workspace must stay bound to the context.
// storage: OVRO_STORE_* format of the half-transformed grid between the passes.
// d_gains: calibration corrections [n_chan][2 n_ant] (complex64) or nullptr;
// baselines kept when uv_min <= length (wavelengths) < uv_max.
int grid_ctx_init(GridCtx** out, int n_ant, int n_chan, int image_size, double cell, int storage, void* d_ws,
                  size_t ws_bytes, const void* d_gains = nullptr, double uv_min = 0.0,
                  double uv_max = HUGE_VAL);
// Host lists and tables (pageable copies): once per geometry and frequency axis.
int grid_ctx_upload(GridCtx* g, const double* h_ant_enu_m, const double* h_chan_freq_hz, cudaStream_t st);
int grid_ctx_enqueue(GridCtx* g, const int32_t* d_vis, float* d_img, int32_t* d_counts_or_null, cudaStream_t st);
// Cross visibilities gridded by the last enqueue (mirrors not counted; synchronises).
int grid_ctx_gridded(GridCtx* g, long long* total, cudaStream_t st);
void grid_ctx_free(GridCtx* g);

// ---- a8-a12: detection (detect.cu)
struct DetectCtx;
size_t detect_ctx_workspace(int n_chan, int image_size, int n_coarse, const int32_t* h_nfft);
int detect_ctx_init(DetectCtx** out, int n_chan, int image_size, double cell, int n_coarse, const int32_t* h_nfft,
                    const ovro_detect_params* params, void* d_ws, size_t ws_bytes);
int detect_ctx_valid_pixels(const DetectCtx* d);
int detect_ctx_upload(DetectCtx* d, cudaStream_t st);
// Clears the histogram and the device status word (start of one search).
int detect_ctx_begin(DetectCtx* d, cudaStream_t st);
// a8-a10 for coarse channel c: d_img_block holds that channel's nfft[c] images.
int detect_ctx_coarse(DetectCtx* d, int c, const float* d_img_block, cudaStream_t st);
// The same, also scattering the high-passed cube z' into d_zp [n_chan][N][N].
int detect_ctx_coarse_zp(DetectCtx* d, int c, const float* d_img_block, float* d_zp, cudaStream_t st);
// a11-a12 (synchronises): candidates in (pixel, coarse, channel) order.
int detect_ctx_finish(DetectCtx* d, const double* h_chan_freq_hz, ovro_candidate* h_out, int max_out, int* n_out,
                      cudaStream_t st);
// The pieces of finish, for a threshold decided across several searches:
// the SNR histogram (synchronises), the values of one bin, and NMS at a cut.
int detect_ctx_histogram(DetectCtx* d, std::vector<unsigned long long>& hist, cudaStream_t st);
int detect_ctx_bin_values(DetectCtx* d, int b, std::vector<float>& v, cudaStream_t st);
int detect_ctx_candidates(DetectCtx* d, float cut, const double* h_chan_freq_hz, ovro_candidate* h_out, int max_out,
                          int* n_out, cudaStream_t st);
void detect_ctx_layout(const DetectCtx* d, uint32_t* key0, int* n_bins, long long* n_tests);
void detect_ctx_free(DetectCtx* d);
// A search handle over an existing context that ovro_search_destroy does not free.
ovro_search* search_view(DetectCtx* d);

}  // namespace ovro
