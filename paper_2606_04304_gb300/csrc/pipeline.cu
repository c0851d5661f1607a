// a14: the batched driver.  Coarse channels stream through one set of device
// buffers (int8 spectra, visibilities, images); the detection filter of each
// coarse channel writes its SNR/width block into the whole-integration search
// workspace, so the threshold and NMS run once over all channels.  The device
// part of a run is captured into a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "stages.h"
#include "tune.h"

namespace ovro {
namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace
}  // namespace ovro

struct ovro_pipeline {
  // configuration
  int n_ant = 0, n_input = 0, n_coarse = 0, image_size = 0, xeng_mode = 0, use_graph = 0;
  long long n_time = 0;
  double cell = 0.0;
  ovro_detect_params prm{};
  std::vector<int32_t> nfft;
  std::vector<int> chan0, n_spec;
  std::vector<double> ant, freq;
  // workspace layout (offsets from the bound base)
  size_t off_q = 0, off_vis = 0, off_img = 0, off_up = 0, off_det = 0, total = 0;
  size_t up_bytes = 0, det_bytes = 0;
  std::vector<size_t> off_grid, grid_bytes;
  // bound state
  unsigned char* ws = nullptr;
  std::vector<ovro::GridCtx*> grid;
  ovro::DetectCtx* det = nullptr;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const uint8_t* graph_volt = nullptr;
  cudaStream_t cap_stream = nullptr;     // private stream for capture (the legacy stream cannot be captured)
  unsigned long long graph_kernels = 0;   // kernel nodes of the captured graph
  std::vector<ovro::GraphTraceEntry> trace;   // event nodes of traced kernels (captured while tracing)
  bool graph_traced = false;
  unsigned long long kernels_per_run = 0;  // kernels of the last run (graph + threshold/NMS)
};

namespace ovro {
namespace {

int8_t* q_buf(ovro_pipeline* pl) { return reinterpret_cast<int8_t*>(pl->ws + pl->off_q); }
int32_t* vis_buf(ovro_pipeline* pl) { return reinterpret_cast<int32_t*>(pl->ws + pl->off_vis); }
float* img_buf(ovro_pipeline* pl) { return reinterpret_cast<float*>(pl->ws + pl->off_img); }

// Everything before the threshold, for one integration: kernels and
// stream-ordered memsets only (capturable).
int enqueue_device(ovro_pipeline* pl, const uint8_t* d_volt, cudaStream_t st) {
  if (int e = detect_ctx_begin(pl->det, st)) return e;
  if (pl->xeng_mode == OVRO_XENG_TC)
    if (int e = correlate_reset_status(st)) return e;
  for (int c = 0; c < pl->n_coarse; ++c) {
    const int32_t nf = pl->nfft[c];
    const uint8_t* v = d_volt + static_cast<long long>(c) * pl->n_time * pl->n_input;
    if (int e = ovro_upchan(v, pl->n_input, 1, pl->n_time, &nf, nullptr, q_buf(pl), nullptr, pl->ws + pl->off_up,
                            pl->up_bytes, st))
      return e;
    if (int e = correlate_enqueue(q_buf(pl), pl->n_ant, nf, pl->n_spec[c], pl->xeng_mode, vis_buf(pl), st, false))
      return e;
    if (int e = grid_ctx_enqueue(pl->grid[c], vis_buf(pl), img_buf(pl), nullptr, st)) return e;
    if (int e = detect_ctx_coarse(pl->det, c, img_buf(pl), st)) return e;
  }
  return OVRO_OK;
}

void drop_graph(ovro_pipeline* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
  pl->graph_volt = nullptr;
  graph_trace_free(pl->trace);
  pl->graph_traced = false;
}

// Records the device work on the private capture stream (nothing executes);
// the graph is then launched on the caller's stream.
int capture(ovro_pipeline* pl, const uint8_t* d_volt) {
  drop_graph(pl);
  cudaStream_t st = pl->cap_stream;
  const unsigned long long l0 = ovro_launch_count();
  const bool traced = profiling();
  OVRO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  if (traced) set_capture_trace(&pl->trace);
  const int e = enqueue_device(pl, d_volt, st);
  set_capture_trace(nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  const unsigned long long n = ovro_launch_count() - l0;
  sub_launches(n);                         // counted when the graph runs
  if (e) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (ce != cudaSuccess) {
    set_last_error("cudaStreamEndCapture", ce);
    return OVRO_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&pl->exec, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    set_last_error("cudaGraphInstantiate", ie);
    return OVRO_ERR_CUDA;
  }
  pl->graph = g;
  pl->graph_volt = d_volt;
  pl->graph_traced = traced;
  pl->graph_kernels = n;
  return OVRO_OK;
}

}  // namespace
}  // namespace ovro

extern "C" {

int ovro_pipeline_create(const ovro_pipeline_config* cfg, ovro_pipeline** out) {
  using namespace ovro;
  if (!cfg || !out) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->n_ant <= 0 || cfg->n_coarse <= 0 || !cfg->h_nfft || !cfg->h_coarse_hz || !cfg->h_ant_enu_m ||
      cfg->n_time <= 0 || !(cfg->cell_dircos > 0.0))
    return OVRO_ERR_INVALID_ARG;
  if (cfg->xeng_mode != OVRO_XENG_TC && cfg->xeng_mode != OVRO_XENG_FP32) return OVRO_ERR_INVALID_ARG;
  ovro_pipeline* pl = new ovro_pipeline;
  pl->n_ant = cfg->n_ant;
  pl->n_input = 2 * cfg->n_ant;
  pl->n_coarse = cfg->n_coarse;
  pl->image_size = cfg->image_size;
  pl->xeng_mode = cfg->xeng_mode;
  pl->use_graph = cfg->use_graph ? 1 : 0;
  pl->n_time = cfg->n_time;
  pl->cell = cfg->cell_dircos;
  pl->prm = cfg->detect;
  pl->ant.assign(cfg->h_ant_enu_m, cfg->h_ant_enu_m + 3 * static_cast<size_t>(cfg->n_ant));
  const double bw = cfg->detect.coarse_bw_hz;
  int c0 = 0, max_nf = 0;
  size_t max_q = 0, max_vis = 0, max_img = 0;
  const long long n_bl = static_cast<long long>(cfg->n_ant) * (cfg->n_ant + 1) / 2;
  for (int c = 0; c < cfg->n_coarse; ++c) {
    const int nf = cfg->h_nfft[c];
    if (nf <= 0 || cfg->n_time < nf) {
      delete pl;
      return OVRO_ERR_INVALID_ARG;
    }
    const long long k = cfg->n_time / nf;
    pl->nfft.push_back(nf);
    pl->chan0.push_back(c0);
    pl->n_spec.push_back(static_cast<int>(k));
    for (int f = 0; f < nf; ++f)
      pl->freq.push_back(cfg->h_coarse_hz[c] + static_cast<double>(f - nf / 2) * bw / nf);
    c0 += nf;
    if (nf > max_nf) max_nf = nf;
    max_q = std::max<size_t>(max_q, static_cast<size_t>(nf) * k * pl->n_input * 2);
    max_vis = std::max<size_t>(max_vis, static_cast<size_t>(nf) * n_bl * 32);
    max_img = std::max<size_t>(max_img, static_cast<size_t>(nf) * cfg->image_size * cfg->image_size * 4);
  }
  // workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + std::max<size_t>(bytes, 1));
    return o;
  };
  pl->up_bytes = ovro_upchan_workspace_size(pl->n_input, 1);
  pl->det_bytes = detect_ctx_workspace(c0, cfg->image_size, cfg->n_coarse, pl->nfft.data());
  if (pl->up_bytes == 0 || pl->det_bytes == 0) {
    delete pl;
    return OVRO_ERR_UNSUPPORTED;
  }
  pl->off_q = take(max_q);
  pl->off_vis = take(max_vis);
  pl->off_img = take(max_img);
  pl->off_up = take(pl->up_bytes);
  pl->off_det = take(pl->det_bytes);
  for (int c = 0; c < cfg->n_coarse; ++c) {
    const size_t gb = grid_ctx_workspace(cfg->n_ant, pl->nfft[c], cfg->image_size, OVRO_STORE_FP32);
    if (gb == 0) {
      delete pl;
      return OVRO_ERR_UNSUPPORTED;
    }
    pl->grid_bytes.push_back(gb);
    pl->off_grid.push_back(take(gb));
  }
  pl->total = off;
  *out = pl;
  return OVRO_OK;
}

size_t ovro_pipeline_workspace_size(const ovro_pipeline* pl) { return pl ? pl->total : 0; }

int ovro_pipeline_channels(const ovro_pipeline* pl, double* h_freq_or_null) {
  if (!pl) return OVRO_ERR_INVALID_ARG;
  if (h_freq_or_null) std::memcpy(h_freq_or_null, pl->freq.data(), pl->freq.size() * sizeof(double));
  return static_cast<int>(pl->freq.size());
}

int ovro_pipeline_bind(ovro_pipeline* pl, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!pl) return OVRO_ERR_INVALID_ARG;
  if (int e = check_workspace(d_ws, ws_bytes, pl->total)) return e;
  cudaStream_t st = as_stream(stream);
  drop_graph(pl);
  for (GridCtx* g : pl->grid) grid_ctx_free(g);
  pl->grid.clear();
  if (pl->det) detect_ctx_free(pl->det);
  pl->det = nullptr;
  pl->ws = static_cast<unsigned char*>(d_ws);
  if (!pl->cap_stream) OVRO_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  for (int c = 0; c < pl->n_coarse; ++c) {
    GridCtx* g = nullptr;
    if (int e = grid_ctx_init(&g, pl->n_ant, pl->nfft[c], pl->image_size, pl->cell, OVRO_STORE_FP32,
                              pl->ws + pl->off_grid[c], pl->grid_bytes[c]))
      return e;
    pl->grid.push_back(g);
    if (int e = grid_ctx_upload(g, pl->ant.data(), pl->freq.data() + pl->chan0[c], st)) return e;
  }
  if (int e = detect_ctx_init(&pl->det, static_cast<int>(pl->freq.size()), pl->image_size, pl->cell, pl->n_coarse,
                              pl->nfft.data(), &pl->prm, pl->ws + pl->off_det, pl->det_bytes))
    return e;
  if (int e = detect_ctx_upload(pl->det, st)) return e;
  // resolves the device status words outside any graph capture
  if (int e = detect_ctx_begin(pl->det, st)) return e;
  if (int e = correlate_reset_status(st)) return e;
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  return OVRO_OK;
}

int ovro_pipeline_run(ovro_pipeline* pl, const uint8_t* d_volt, ovro_candidate* h_out, int max_out, int* n_out,
                      void* stream) {
  using namespace ovro;
  if (!pl || !d_volt || !n_out || (max_out > 0 && !h_out) || max_out < 0) return OVRO_ERR_INVALID_ARG;
  *n_out = 0;
  if (!pl->ws || !pl->det) return OVRO_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  unsigned long long n_dev = 0;
  if (pl->use_graph && !tuning(st)) {
    // (re)capture for a new buffer, or when tracing was switched since
    if (!pl->exec || pl->graph_volt != d_volt || pl->graph_traced != profiling())
      if (int e = capture(pl, d_volt)) return e;
    OVRO_CUDA_TRY(cudaGraphLaunch(pl->exec, st));
    add_launches(pl->graph_kernels);
    n_dev = pl->graph_kernels;
  } else {
    const unsigned long long l0 = ovro_launch_count();
    if (int e = enqueue_device(pl, d_volt, st)) return e;
    n_dev = ovro_launch_count() - l0;
  }
  const unsigned long long l1 = ovro_launch_count();
  const int e = detect_ctx_finish(pl->det, pl->freq.data(), h_out, max_out, n_out, st);
  pl->kernels_per_run = n_dev + (ovro_launch_count() - l1);
  if (pl->exec && pl->graph_traced && pl->use_graph && !tuning(st)) {
    OVRO_CUDA_TRY(cudaStreamSynchronize(st));
    graph_trace_collect(pl->trace);              // per-kernel times of this replay
  }
  if (pl->xeng_mode == OVRO_XENG_TC) {
    const int s = ovro_correlate_status(st);
    if (s) return s;
  }
  return e;
}

int ovro_pipeline_run_device(ovro_pipeline* pl, const uint8_t* d_volt, void* stream) {
  using namespace ovro;
  if (!pl || !d_volt) return OVRO_ERR_INVALID_ARG;
  if (!pl->ws || !pl->det) return OVRO_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  unsigned long long n_dev = 0;
  if (pl->use_graph && !tuning(st)) {
    if (!pl->exec || pl->graph_volt != d_volt || pl->graph_traced != profiling())
      if (int e = capture(pl, d_volt)) return e;
    OVRO_CUDA_TRY(cudaGraphLaunch(pl->exec, st));
    add_launches(pl->graph_kernels);
    n_dev = pl->graph_kernels;
  } else {
    const unsigned long long l0 = ovro_launch_count();
    if (int e = enqueue_device(pl, d_volt, st)) return e;
    n_dev = ovro_launch_count() - l0;
  }
  pl->kernels_per_run = n_dev;
  if (pl->xeng_mode == OVRO_XENG_TC) return ovro_correlate_status(st);   // synchronises
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  return OVRO_OK;
}

int ovro_pipeline_search(ovro_pipeline* pl, ovro_search** out) {
  if (!pl || !out) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!pl->det) return OVRO_ERR_WORKSPACE;
  *out = ovro::search_view(pl->det);
  return OVRO_OK;
}

int ovro_pipeline_stats(const ovro_pipeline* pl, long long* kernels_per_run, int* graph_live) {
  if (!pl) return OVRO_ERR_INVALID_ARG;
  if (kernels_per_run) *kernels_per_run = static_cast<long long>(pl->kernels_per_run);
  if (graph_live) *graph_live = pl->exec ? 1 : 0;
  return OVRO_OK;
}

int ovro_pipeline_gridded(ovro_pipeline* pl, long long* n_gridded, void* stream) {
  if (!pl || !n_gridded) return OVRO_ERR_INVALID_ARG;
  *n_gridded = 0;
  for (ovro::GridCtx* g : pl->grid) {
    long long n = 0;
    if (int e = ovro::grid_ctx_gridded(g, &n, ovro::as_stream(stream))) return e;
    *n_gridded += n;
  }
  return OVRO_OK;
}

void ovro_pipeline_destroy(ovro_pipeline* pl) {
  using namespace ovro;
  if (!pl) return;
  drop_graph(pl);
  for (GridCtx* g : pl->grid) grid_ctx_free(g);
  if (pl->det) detect_ctx_free(pl->det);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  delete pl;
}

}  // extern "C"
