// Internal interface between the upchannelizer's entry points (upchan.cu) and
// its mixed-radix kernel (upchan_mr.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ovro {

struct UpchanArgs {
  const uint8_t* volt;      // this coarse channel, [n_time][n_input]
  const float2* tw;         // omega_{tw_n}^k
  const float* scale;       // [n_input] for this coarse channel
  int8_t* out_q;            // this coarse block, [C][K][n_input][2]
  float* out_f;             // same layout, floats (optional)
  int n_input;
  int n_spec;
  int tw_n;
  int group;                // G inputs per CTA
  // mixed-radix kernel only
  const float* taps;        // P N polyphase-filter coefficients h[p N + n], or null (h = 1)
  int n_tap;                // P
  int chan_lo;              // first fftshifted fine channel written
  int chan_cnt;             // fine channels written (C)
};

constexpr int kMrMaxPass = 8;
constexpr int kMrMaxN = 8192;

struct MrPlan {
  int n;                    // FFT length
  int f;                    // FFTs in flight
  int threads;
  int n_pass;
  int radix[kMrMaxPass];
};

// Plan of the mixed-radix kernel for even N = 2^a 3^b 5^c <= kMrMaxN with P
// taps and C output channels: false if N is not such a length or no CTA shape fits.
bool mr_plan(int n, int n_input, int n_tap, int chan_cnt, MrPlan* plan, int* group, size_t* smem);

// One launch over every spectrum of one coarse channel (a.tw = omega_N table,
// a.tw_n = N); the CTA shape comes from the autotuner, a.group is ignored.
int launch_upchan_mr(const UpchanArgs& a, int n_tap, cudaStream_t st);

}  // namespace ovro
