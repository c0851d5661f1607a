/*
 * ovro.h -- C ABI of the GB300 ultra-narrowband all-sky imaging hot path
 * (OVRO-LWA technosignature search, arXiv 2606.04304).
 *
 * The path: unpack 4+4-bit coarse-channel voltages, upchannelize with an FFT,
 * requantise to 8 bits, cross-correlate every antenna pair and polarisation
 * product (X-engine), grid and image every fine channel, and search every
 * pixel spectrum for narrowband candidates.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers prefixed d_ are device pointers, h_ are host pointers.  The
 *    caller owns every buffer.  The library never allocates or frees device
 *    memory: where a call needs scratch it takes a caller-allocated workspace
 *    (d_ws, ws_bytes) whose size the matching *_workspace_size() returns.
 *    Workspaces must be 256-byte aligned.
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream), except ovro_detect, which
 *    synchronises `stream` once to run its global Benjamini-Hochberg step.
 *  - Every argument is validated on the host before anything is launched; an
 *    invalid call returns a negative ovro_status and launches nothing.
 *    Nothing throws across the ABI.
 *  - A call that launched kernels returns OVRO_ERR_CUDA if a launch failed;
 *    the message of the last failure is available from ovro_last_error().
 *  - Inputs are numbered input = 2 * antenna + polarisation (X = 0, Y = 1).
 *  - Not thread-safe per stream; distinct streams may be used from distinct
 *    host threads.
 */
#ifndef OVRO_H
#define OVRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OVRO_OK = 0,
  OVRO_ERR_INVALID_ARG = -1,   /* null pointer, negative size, bad enum */
  OVRO_ERR_UNSUPPORTED = -2,   /* valid but outside what the kernels implement */
  OVRO_ERR_CUDA = -3,          /* a CUDA call or launch failed */
  OVRO_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up */
  OVRO_ERR_WORKSPACE = -5,     /* workspace missing, too small or misaligned */
  OVRO_ERR_OVERFLOW = -6,      /* an integer accumulation bound would be exceeded */
  OVRO_ERR_CAPACITY = -7       /* output capacity too small (true count reported) */
} ovro_status;

/* Human-readable name of a status code (static storage). */
const char* ovro_status_string(int status);
/* Message of the last CUDA failure seen by this library in this thread. */
const char* ovro_last_error(void);
/* Library ABI version, (major << 16) | minor. */
int ovro_version(void);
/* Number of kernels this library has launched in this process. */
unsigned long long ovro_launch_count(void);
/* Kernel tracing.  ovro_profile(1) clears the trace and starts recording a
 * CUDA event pair on the launch stream around every launch of the main
 * kernels (k_upchan, k_upchan_mr, k_xeng_tc, k_xeng_simt, k_grid_prep, k_grid_tiles, k_fft_rows,
 * k_fft_cols, k_stats, k_ztrans, k_rank, k_walk, k_median_sub, k_mf, k_nms_warp, k_vet_line,
 * k_vet_fit, k_drift, k_scorer_fwd); ovro_profile(0) stops recording.
 * ovro_profile_query waits for the recorded launches of one kernel and
 * returns their summed device time and count. */
int ovro_profile(int enable);
int ovro_profile_query(const char* kernel, double* total_ms, int* launches);

/* -------------------------------------------------------------------------
 * a1-a3  Unpack + FFT upchannelizer + 8-bit requantisation
 *
 * Section 2.1: the offline pipeline upchannelizes each coarse channel by an
 * FFT over its time samples (factor 2400 -> 9.9 Hz in the paper) and feeds
 * 8-bit complex samples to the xGPU correlator.
 *
 * d_volt   uint8 [n_coarse][n_time][n_input]; each byte is one complex sample,
 *          real part in the high nibble, imaginary in the low nibble, both
 *          4-bit two's complement.
 * h_nfft   [n_coarse] FFT length N_c per coarse channel: a power of two in
 *          [2, 16384], or an even 2^a 3^b 5^c up to 8192 such as the paper's
 *          2400 (mixed-radix kernel).  Each coarse channel yields
 *          K_c = n_time / N_c spectra
 *          from non-overlapping blocks (rectangular window, unnormalised
 *          exp(-2 pi i k n / N) transform); leftover samples are ignored.
 *          Fine channel k' = (k + N/2) mod N (fftshift) sits at
 *          nu_c + (k' - N/2) f_c / N.
 * h_scale_or_null  NULL: one scale per (coarse, input),
 *          s = 8 sqrt(2) / sqrt(N_c P) with P the mean |x|^2 of the used
 *          samples (exact integer sum, FP64 arithmetic), s = 0 if P = 0.
 *          Otherwise a host array [n_coarse][n_input] of scales.
 * d_fine_q int8 output, coarse-major blocks; block c is
 *          [N_c][K_c][n_input][2] (re, im), starting at element offset
 *          sum_{c' < c} N_c' K_c' n_input * 2.  Each component is
 *          clamp(rint(s * X), -127, 127), s rounded to FP32, one FP32 multiply,
 *          round half to even.
 * d_fine_f32_or_null  optional FP32 spectra in the same layout (floats).
 * Workspace: ovro_upchan_workspace_size(n_input, n_coarse) bytes.
 * Errors: OVRO_ERR_INVALID_ARG (null pointers, n_* <= 0), OVRO_ERR_UNSUPPORTED
 *          (N_c not one of the lengths above, n_time < N_c).
 * ------------------------------------------------------------------------- */
size_t ovro_upchan_workspace_size(int n_input, int n_coarse);
int ovro_upchan(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                const int32_t* h_nfft, const double* h_scale_or_null,
                int8_t* d_fine_q, float* d_fine_f32_or_null,
                void* d_ws, size_t ws_bytes, void* stream);

/* Upchannelizer options (Section 2.1).
 *
 * Fine-channel batches: the paper cross-correlates 300 fine channels at a
 * time to bound the memory the upchannelized data take.  chan_count > 0 keeps
 * only fine channels [chan_lo, chan_lo + chan_count) of the fftshifted axis
 * of every coarse channel (chan_lo + chan_count <= N_c for all c); 0 keeps all.
 *
 * Polyphase filter bank in place of the bare block FFT: with n_taps = P and
 * h_taps non-NULL, spectrum s of coarse channel c is the FFT of
 * y_n = sum_{p < P} h[p N + n] x[(s + p) N + n], n < N, with h the P N FP32
 * coefficients at h_taps[c] (a device pointer; the prototype filter read row
 * by row), so K_c = n_time / N_c - P + 1 spectra; P = 1 with h = 1 is the
 * plain FFT.  The scale becomes s = 8 sqrt(2) / sqrt(P_mean sum h^2) (sum in
 * FP64), the power still taken over all n_time / N_c whole blocks.
 * h_taps NULL requires n_taps = 1.  Either option runs the mixed-radix kernel,
 * so N_c <= 8192 there. */
typedef struct ovro_upchan_options {
  int32_t n_taps;              /* P >= 1 */
  const float* const* h_taps;  /* host array [n_coarse] of device pointers, or NULL */
  int32_t chan_lo;             /* first fftshifted fine channel written */
  int32_t chan_count;          /* fine channels written per coarse channel; 0 = all N_c */
} ovro_upchan_options;

/* ovro_upchan with options (NULL = ovro_upchan).  Block c of d_fine_q (and of
 * d_fine_f32_or_null) is [C_c][K_c][n_input][2], C_c = chan_count or N_c,
 * at element offset sum_{c' < c} C_c' K_c' n_input * 2; row i of the block is
 * fine channel chan_lo + i.  Same workspace as ovro_upchan.  Errors as
 * ovro_upchan, plus OVRO_ERR_INVALID_ARG for n_taps < 1, n_taps > 1 without
 * taps, a NULL taps pointer, chan_lo < 0, chan_count < 0 or a window past N_c,
 * and OVRO_ERR_UNSUPPORTED when K_c < 1 or a length the kernels do not take. */
int ovro_upchan_ex(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                   const int32_t* h_nfft, const double* h_scale_or_null,
                   const ovro_upchan_options* opt_or_null,
                   int8_t* d_fine_q, float* d_fine_f32_or_null,
                   void* d_ws, size_t ws_bytes, void* stream);

/* Allocation-free ovro_upchan (no counterpart in the paper; an interface
 * convenience).  For callers that cannot allocate device memory at all -- a
 * plugin whose host framework owns the device heap, or a real-time loop where
 * an allocation (which may synchronise the device) would stall other streams.
 * Same arguments and results as ovro_upchan without the workspace: the
 * scratch is a fixed 1 MiB array inside the library, held on every GPU that
 * loads it until the process exits.  Limit: ovro_upchan_workspace_size(
 * n_input, n_coarse) <= 1 MiB (n_input * n_coarse up to about 45,000, e.g.
 * 704 inputs x 64 coarse channels); larger calls return OVRO_ERR_CAPACITY and
 * launch nothing.  Allocates nothing (no cudaMalloc/cudaFree).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  A
 * failed lookup is not kept: the next call on that device tries again.  Every
 * call reuses the same array (what must start at zero is cleared by each
 * call), so calls that overlap on the GPU -- different streams, or different
 * host threads, on one device -- race and must be serialised by the caller. */
int ovro_upchan_noalloc(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                        const int32_t* h_nfft, const double* h_scale_or_null,
                        int8_t* d_fine_q, float* d_fine_f32_or_null, void* stream);

/* -------------------------------------------------------------------------
 * a4  X-engine: per fine channel, every antenna pair and polarisation product
 *
 * Section 2.1: the correlation stage (xGPU) integrates, per fine channel,
 *     V_ij^pq = sum_{s < K} q_ip(s) conj(q_jq(s))        (i <= j, autos kept)
 *
 * d_fine_q  int8 [n_chan][n_spec][2 n_ant][2] (one coarse block of
 *           ovro_upchan's output, or several with the same K).
 * d_vis     int32 output [n_chan][n_bl][4][2], n_bl = n_ant (n_ant + 1) / 2,
 *           baseline (a, b), a <= b, at a n_ant - a (a - 1) / 2 + (b - a);
 *           pol product p = 2 p_a + p_b (XX, XY, YX, YY); (re, im).
 * mode      OVRO_XENG_TC: tensor cores (tcgen05, int8 values carried exactly
 *           in FP16 operands, FP32 accumulation in tensor memory, exact while
 *           every partial sum stays below 2^24);
 *           OVRO_XENG_FP32: plain FP32 SIMT accumulation (same exactness
 *           bound).  Both are bit-exact integer results.
 * Errors:   OVRO_ERR_OVERFLOW if 2 * 128^2 * n_spec >= 2^24 (n_spec > 511):
 *           the bound holds for any int8 input, -128 included,
 *           OVRO_ERR_UNSUPPORTED if n_ant > 4096,
 *           OVRO_ERR_INVALID_ARG if d_fine_q is not 4-byte aligned or d_vis
 *           not 16-byte aligned.
 * ------------------------------------------------------------------------- */
enum { OVRO_XENG_TC = 0, OVRO_XENG_FP32 = 1 };
int ovro_correlate(const int8_t* d_fine_q, int n_ant, int n_chan, int n_spec, int mode,
                   int32_t* d_vis, void* stream);
/* Synchronises `stream` and reports whether the last OVRO_XENG_TC call gave up
 * a bounded wait on the tensor-core completion barrier (OVRO_ERR_TIMEOUT), in
 * which case its output is incomplete. */
int ovro_correlate_status(void* stream);

/* -------------------------------------------------------------------------
 * a5-a7  uvw (FP64), prolate-spheroidal gridding, 2D FFT -> dirty images
 *
 * Section 2.2: every fine channel is imaged over the visible hemisphere
 * (dirty images are the search product).  Stokes I = (XX + YY) / 2 of every
 * cross baseline, natural weights, zenith phase centre (planar array, w = 0).
 * The uv grid is padded by 2 (G = 2N cells a side) and the image is the
 * central N x N of its transform.  u = (x_a - x_b) s_nu cells,
 * s_nu = nu / (c du), du = 1 / (G cell), one FP64 multiply; position rounded
 * to 1/1024 cell; separable 7 x 7 kernel psi_0(7 pi / 2, x / 3.5); a baseline
 * whose footprint (or its mirror's) leaves the grid is dropped.
 * Image = Re sum G exp(+2 pi i (u l + v m)), divided by (gridded visibilities
 * incl. mirrors) and the grid correction; pixel (r, c) <-> l = (c - N/2) cell,
 * m = (r - N/2) cell; pixels with l^2 + m^2 >= 1 are 0.
 *
 * d_vis           int32 [n_chan][n_bl][4][2] as produced by ovro_correlate.
 * h_ant_enu_m     [n_ant][3] antenna positions, metres (only E, N are used).
 * h_chan_freq_hz  [n_chan] sky frequency of each channel.
 * image_size      N, a power of two in [16, 1024].
 * cell_dircos     pixel size in direction cosines (2 / N images the sky to
 *                 the horizon).
 * storage         OVRO_STORE_FP32, or OVRO_STORE_BF16 / OVRO_STORE_FP16 to keep
 *                 the intermediate uv grid in 16-bit storage (FP32 arithmetic).
 *                 The grid lives in shared memory while it is gridded and row
 *                 transformed; what crosses global memory is the half-transformed
 *                 grid (G rows x N central columns per channel), and that is what
 *                 is stored in 16 bits: BF16 as is, FP16 with a power-of-two
 *                 scale per row (largest component in [2^13, 2^14)).  Measured
 *                 errors vs the FP64 oracle: BF16 ~3e-3 of the image maximum
 *                 (L2 ~1.4e-3), FP16 ~4e-4 (L2 ~1.7e-4), FP32 ~2e-7.
 * d_img           float output [n_chan][N][N].
 * d_n_gridded_or_null  optional int32 [n_chan]: gridded visibilities per
 *                 channel (mirrors included).
 * Workspace: ovro_grid_image_workspace_size(...) bytes.
 * ------------------------------------------------------------------------- */
enum { OVRO_STORE_FP32 = 0, OVRO_STORE_BF16 = 1, OVRO_STORE_FP16 = 2 };
size_t ovro_grid_image_workspace_size(int n_ant, int n_chan, int image_size, int storage);
int ovro_grid_image(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m,
                    const double* h_chan_freq_hz, int n_chan, int image_size,
                    double cell_dircos, int storage, float* d_img,
                    int32_t* d_n_gridded_or_null, void* d_ws, size_t ws_bytes, void* stream);

/* Imaging with calibration corrections and a baseline (uv-range) selection.
 *
 * Section 2.2 calibrates the visibilities (per-antenna gains and a bandpass)
 * before imaging, and Section 2.5.1 re-images with baseline-length cuts to
 * test for near-field emitters.  d_gains_or_null: complex64 (float2, 8-byte
 * aligned) [n_chan][2 n_ant] multiplicative corrections c per input and
 * channel (so a bandpass is included): XX' = c_{2a} conj(c_{2b}) XX,
 * YY' = c_{2a+1} conj(c_{2b+1}) YY, Stokes I = (XX' + YY') / 2, in FP32 on the
 * device (NULL: the exact integer Stokes I of ovro_grid_image).  Baselines are
 * kept when uv_min_lambda <= L nu / c < uv_max_lambda, L = sqrt(dx^2 + dy^2)
 * metres, decided in FP64 per channel (uv_max_lambda <= 0: no upper cut);
 * baselines outside are dropped and not counted.  Otherwise as ovro_grid_image
 * (same workspace size). */
typedef struct {
  int storage;                    /* OVRO_STORE_* */
  const void* d_gains_or_null;    /* complex64 [n_chan][2 n_ant] or NULL */
  double uv_min_lambda;           /* >= 0 */
  double uv_max_lambda;           /* <= 0: none */
} ovro_grid_options;
int ovro_grid_image_ex(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m,
                       const double* h_chan_freq_hz, int n_chan, int image_size, double cell_dircos,
                       const ovro_grid_options* options, float* d_img, int32_t* d_n_gridded_or_null,
                       void* d_ws, size_t ws_bytes, void* stream);

/* a5 on its own: p = rint(u Q), Q = 1024, the rounded uv position in 1/1024
 * cell of the padded (2 image_size) grid of every cross baseline (a < b, row-major order) in every channel,
 * int32 [n_chan][n_cross] (saturated at +-2^30).  The FP64 product of the
 * definition is reproduced exactly.  Workspace: ovro_grid_image_workspace_size
 * with the same n_ant, n_chan and image_size. */
int ovro_uvw(const double* h_ant_enu_m, int n_ant, const double* h_chan_freq_hz, int n_chan,
             int image_size, double cell_dircos, int32_t* d_pu, int32_t* d_pv, void* d_ws,
             size_t ws_bytes, void* stream);

/* -------------------------------------------------------------------------
 * a8-a12  Stage I candidate search
 *
 * Section 2.4: standardise each channel image by its median absolute
 * deviation (in-horizon pixels, FP64 statistics, z = (x - med) /
 * (1.482602218505602 MAD)); subtract a running median along frequency per
 * pixel (window: smallest odd W with W df > highpass_hz, centred, clipped at
 * coarse-channel edges); boxcar matched filters of the given widths
 * (unit-normalised 1/sqrt(w), width w at channel k covers
 * k - floor((w-1)/2) .. k + ceil((w-1)/2) inside the coarse channel), keeping
 * the maximum SNR and its width; p = Q(SNR) with Benjamini-Hochberg across
 * all in-horizon pixels x channels, or a fixed n_sigma threshold; then 1D
 * non-maximum suppression along frequency per pixel (half-width
 * max(1, floor(w/2)), within a coarse channel).
 * ------------------------------------------------------------------------- */
enum { OVRO_DETECT_BH = 0, OVRO_DETECT_FIXED = 1 };

typedef struct {
  int mode;               /* OVRO_DETECT_BH or OVRO_DETECT_FIXED */
  double alpha;           /* BH false-discovery level (e.g. 0.01) */
  double nsigma;          /* fixed-mode threshold (the paper quotes 10) */
  double highpass_hz;     /* running-median span: wider than 5 kHz -> 5000 */
  double coarse_bw_hz;    /* coarse-channel width (24000) */
} ovro_detect_params;

typedef struct {
  int32_t coarse;         /* coarse channel */
  int32_t fine;           /* fine channel within the coarse channel */
  int32_t chan;           /* global channel index */
  int32_t row, col;       /* pixel */
  int32_t width;          /* matched-filter width, channels */
  float snr;              /* matched-filter SNR */
  float score;            /* keep probability from the learned scorer (0 without one) */
  double freq_hz;         /* sky frequency of the channel */
  double log10_p;         /* log10 of the one-sided Gaussian p-value */
} ovro_candidate;

/* Number of boxcar widths and their values (the default set used by
 * ovro_detect: 1..10, 13..49 step 3, 50..100 step 10). */
int ovro_default_widths(int32_t* h_out_or_null);

size_t ovro_detect_workspace_size(int n_chan, int image_size, int n_coarse,
                                  const int32_t* h_nfft);
/* The learned candidate scorer as a stage of the search (a13; no
 * counterpart in the paper, which keeps or drops Stage I triggers by
 * threshold alone).  With a scorer, ovro_detect takes its triggers from the
 * fixed threshold trigger_nsigma (the relaxed Stage I cut; NMS included),
 * scores each trigger's cutout of the high-passed cube with the network of
 * ovro_scorer_forward, and returns the triggers whose keep probability
 * sigmoid(logit) is at least keep_prob, that probability in each record's
 * score.  d_ws (ws_bytes >= ovro_scorer_detect_workspace_size(...)) holds the
 * high-passed cube, the triggers and the cutouts: caller-owned scratch, bound
 * for the call only.  OVRO_ERR_CAPACITY when more than max_triggers triggers
 * pass the relaxed cut. */
typedef struct {
  const void* d_w_bf16;   /* ovro_scorer_n_params() BF16 weights (device) */
  double trigger_nsigma;  /* relaxed fixed threshold proposing triggers (e.g. 5) */
  float keep_prob;        /* keep a trigger when its probability >= keep_prob */
  int max_triggers;       /* capacity of the scratch */
  void* d_ws;
  size_t ws_bytes;
} ovro_scorer;
size_t ovro_scorer_detect_workspace_size(int n_chan, int image_size, int n_coarse, int max_triggers);

/* d_img     float [n_chan][N][N] images (ovro_grid_image output layout).
 * h_nfft    [n_coarse] channels per coarse channel (sum = n_chan).
 * h_chan_freq_hz [n_chan] sky frequencies (for the candidate records).
 * scorer_or_null  NULL: the plain threshold detector (params' mode); else
 *           the scorer stage above replaces the threshold.
 * h_out     host array of max_out candidates, ordered by (row, col, chan);
 *           *n_out = number found.  OVRO_ERR_CAPACITY if more than max_out
 *           (the first max_out are written, *n_out holds the true count). */
int ovro_detect(const float* d_img, int n_chan, int image_size, double cell_dircos,
                int n_coarse, const int32_t* h_nfft, const double* h_chan_freq_hz,
                const ovro_detect_params* params, const ovro_scorer* scorer_or_null,
                ovro_candidate* h_out, int max_out, int* n_out, void* d_ws, size_t ws_bytes,
                void* stream);

/* Stage-isolated pieces of ovro_detect (same workspace), for inspection and
 * testing.  Layouts are the caller's:
 *   ovro_detect_stats:  d_stats double [n_chan][2] = (median, MAD).
 *   ovro_detect_filter: d_zp (optional) float [n_chan][N][N] high-passed
 *       standardised cube (0 outside the horizon); d_snr float [n_chan][N][N]
 *       maximum boxcar SNR; d_width int32 [n_chan][N][N] its width (0 outside
 *       the horizon).  Needs d_stats from ovro_detect_stats. */
int ovro_detect_stats(const float* d_img, int n_chan, int image_size, double cell_dircos,
                      double* d_stats, void* d_ws, size_t ws_bytes, void* stream);
int ovro_detect_filter(const float* d_img, const double* d_stats, int n_chan, int image_size,
                       double cell_dircos, int n_coarse, const int32_t* h_nfft,
                       const ovro_detect_params* params, float* d_zp_or_null, float* d_snr,
                       int32_t* d_width, void* d_ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------------------
 * Stage I re-evaluation and Stage II automated cuts (Section 2.4)
 *
 * For each candidate (an ovro_detect record, width w at global channel k,
 * boxcar support S, coarse channel [c_lo, c_hi)):
 *  - re-evaluation: off-line channels O = the offline_half channels on each
 *    side beyond the NMS guard g = max(1, floor(w/2)) around S, clipped to
 *    the coarse channel; at the candidate's pixel b = median z_O,
 *    sigma = 1.482602218505602 median |z_O - b| (1 if |O| < 16 or sigma = 0),
 *    snr_re = sum_S (z - b) / (sigma sqrt(w)); OVRO_VET_REEVAL if < cut.
 *    z is the MAD-standardised image (d_stats from ovro_detect_stats).
 *  - line image over the (2 fit_half + 1)^2 cutout: L_p = sum_S (z_p - b_p) /
 *    sqrt(w), b_p the median over O at pixel p; pixels off the image or below
 *    the horizon are left out.
 *  - centroid: least squares of A exp(-(a dx^2 + 2 b dx dy + c dy^2) / 2),
 *    dx = col - x0, dy = row - y0, started from (L_centre, col, row) and the
 *    beam's (a, b, c); errors from (J^T J)^-1 chi2_red (rescaled by
 *    sqrt(chi2_red)).  The beam is the same fit to the point-spread image
 *    d_psf of the candidate's coarse channel around pixel (N/2, N/2), started
 *    at (peak, N/2, N/2, 1, 0, 1); beam_fwhm = 2 sqrt(2 ln 2) (ac - b^2)^-1/4
 *    pixels and sigma_therm = beam_fwhm / (2 snr), snr the Stage I SNR.
 *  - OVRO_VET_EXTENDED if sqrt(det Q_beam / det Q_fit) > max_area_ratio;
 *    OVRO_VET_FIT if either fit failed (non-finite, A <= 0, Q not positive
 *    definite, centroid more than fit_half pixels off, fewer than 7 pixels).
 *  - OVRO_VET_NOISY if the candidate channel's standardised in-horizon
 *    pixels have a standard deviation above max_noise_std, or its robust
 *    sigma 1.4826 MAD is more than max_sigma_dev times above or below the
 *    median over its coarse channel.
 * keep = (flags == 0).  Pixels are (col, row) with l = (col - N/2) cell,
 * m = (row - N/2) cell.  Fits run in FP64 on the GPU, one warp each.
 * ------------------------------------------------------------------------- */
enum { OVRO_VET_REEVAL = 1, OVRO_VET_EXTENDED = 2, OVRO_VET_NOISY = 4, OVRO_VET_FIT = 8 };

typedef struct {
  int32_t offline_half;    /* off-line channels per side, 1..64 (64) */
  int32_t fit_half;        /* cutout half-size in pixels, 1..7 (3) */
  double max_area_ratio;   /* (2.0) */
  double max_noise_std;    /* (1.5) */
  double max_sigma_dev;    /* (2.0) */
} ovro_vet_params;

typedef struct {
  int32_t keep;            /* 1: survives every cut */
  int32_t flags;           /* OVRO_VET_* bits */
  float snr_re;            /* re-evaluated SNR */
  float area_ratio;        /* fitted area / beam area (NaN if a fit failed) */
  double amp;              /* fitted amplitude */
  double col, row;         /* fitted centroid, pixels */
  double sigma_col, sigma_row;   /* 1-sigma fit errors x sqrt(chi2_red), pixels */
  double chi2_red;
  double beam_fwhm;        /* synthesized-beam FWHM, pixels */
  double sigma_therm;      /* beam_fwhm / (2 snr), pixels */
  double noise_std;        /* std of the candidate channel's standardised image */
  int32_t iterations;      /* Levenberg-Marquardt steps taken */
  int32_t pad_;
} ovro_vet_result;

void ovro_vet_default_params(ovro_vet_params* p);
size_t ovro_vet_workspace_size(int n_cand, int n_coarse);
/* d_img float [n_chan][N][N] images and d_stats double [n_chan][2] (median,
 * MAD) as ovro_detect_stats; d_psf float [n_coarse][N][N] point-spread
 * images (the dirty image of unit visibilities at each coarse channel);
 * h_cand [n_cand] candidates; cut the Stage I decision threshold; params
 * NULL for the defaults.  h_out [n_cand].  Synchronises stream.  Errors:
 * OVRO_ERR_INVALID_ARG (null pointers, sizes, channel counts not summing to
 * n_chan, a candidate outside its coarse channel or the image),
 * OVRO_ERR_UNSUPPORTED (params out of range). */
int ovro_vet(const float* d_img, const double* d_stats, int n_chan, int image_size, double cell_dircos,
             int n_coarse, const int32_t* h_nfft, const float* d_psf, const ovro_candidate* h_cand, int n_cand,
             float cut, const ovro_vet_params* params_or_null, ovro_vet_result* h_out, void* d_ws,
             size_t ws_bytes, void* stream);

/* -------------------------------------------------------------------------
 * Drift-rate search (the paper's future work, Sections 2.3.4 and 4)
 *
 * Sub-integrations: the K spectra of an integration split into T = 2^k
 * equal chunks (ovro_spectra_slice), each correlated, imaged and passed
 * through ovro_detect_filter, give high-passed standardised cubes z'_t.
 * For every in-horizon pixel and start channel f of coarse channel
 * [c_lo, c_hi) the search sums z'_t along the Taylor tree's digital lines of
 * total drift d, |d| < T: shift(d, 1, 0) = 0; shift(d, n, t) =
 * shift(floor(d/2), n/2, t) for t < n/2, ceil(d/2) + shift(floor(d/2), n/2,
 * t - n/2) otherwise; channel f + shift for d >= 0, f - shift for d < 0.
 * A path counts only if its end f + d lies inside the coarse channel.
 * SNR = sum / sqrt(T), the largest over drifts visited 0, +1, -1, +2, ...
 * (strictly larger replaces).  Candidates: Benjamini-Hochberg on p = Q(SNR)
 * over every in-horizon (pixel, channel), m = in-horizon pixels x channels
 * (params->mode OVRO_DETECT_BH, params->alpha; decided bin by bin as Stage
 * I's), or SNR >= params->nsigma (OVRO_DETECT_FIXED); then greedy NMS
 * along frequency per (pixel, coarse channel) with half-width
 * max(1, floor((|d| + 1) / 2)); records as ovro_candidate with width
 * = |d| + 1 (channels the line crosses) and the signed drift in
 * h_drift_out (channels per integration; Hz/s = d * df / integration time),
 * ordered by (pixel, coarse channel, channel).
 * ------------------------------------------------------------------------- */
size_t ovro_drift_workspace_size(int n_chan, int image_size, int n_coarse, const int32_t* h_nfft);
/* d_zp float [T][n_chan][N][N] (T = n_sub in {2, 4, 8, 16}); optional
 * d_snr_or_null float [n_chan][N][N] (-inf below the horizon) and
 * d_drift_or_null int32 [n_chan][N][N] maps.  Synchronises stream.
 * OVRO_ERR_CAPACITY if more than max_out candidates (the first max_out are
 * written, *n_out holds the true count), a (pixel, coarse channel) pair
 * holds more than 256 detections, or an open histogram bin more than 2^22
 * values. */
int ovro_drift_search(const float* d_zp, int n_sub, int n_chan, int image_size, double cell_dircos, int n_coarse,
                      const int32_t* h_nfft, const double* h_chan_freq_hz, const ovro_detect_params* params,
                      float* d_snr_or_null, int32_t* d_drift_or_null, ovro_candidate* h_out, int32_t* h_drift_out,
                      int max_out, int* n_out, void* d_ws, size_t ws_bytes, void* stream);
/* d_out int8 [n_chan][count][n_input][2] = spectra s0 .. s0 + count - 1 of
 * d_q int8 [n_chan][n_spec][n_input][2] (one sub-integration's block). */
int ovro_spectra_slice(const int8_t* d_q, int n_chan, int n_spec, int n_input, int s0, int count, int8_t* d_out,
                       void* stream);

/* -------------------------------------------------------------------------
 * a13  Learned candidate scorer (no counterpart in the paper, which keeps or
 * drops Stage I triggers by threshold alone; the plain detector stays the
 * fallback and the judge of recall and false alarms).
 *
 * Network: 1600 -> 128 -> 32 -> 1, GELU (erf form) hidden units, logit out.
 * Parameters: one flat vector of ovro_scorer_n_params() values, layer by
 * layer, W row-major [out][in] then b.  Served as BF16 (d_w_bf16, uint16 bit
 * patterns); every product is accumulated in FP32.  Training keeps FP32
 * master weights and Adam moments (b1 = 0.9, b2 = 0.999, eps = 1e-8).
 * Input: cutouts of the high-passed standardised cube (ovro_detect_filter's
 * d_zp) -- 64 channels x 5 x 5 pixels centred on a trigger, channel-major,
 * zero outside the trigger's coarse channel or the image.
 * ------------------------------------------------------------------------- */
int ovro_scorer_n_params(void);
/* Workspace for batch cutouts/activations (and n_coarse channel offsets). */
size_t ovro_scorer_workspace_size(int batch, int n_coarse);
/* d_zp float [n_chan][N][N]; d_trig int32 [n_trig][3] = (channel, row, col);
 * d_x float [n_trig][1600]. */
int ovro_scorer_cutouts(const float* d_zp, int n_chan, int image_size, int n_coarse,
                        const int32_t* h_nfft, const int32_t* d_trig, int n_trig, float* d_x,
                        void* d_ws, size_t ws_bytes, void* stream);
/* d_logit float [batch]. */
int ovro_scorer_forward(const void* d_w_bf16, const float* d_x, int batch, float* d_logit,
                        void* d_ws, size_t ws_bytes, void* stream);
/* Gradient of the mean binary cross-entropy (labels d_y in {0, 1}) with
 * respect to all parameters, evaluated at d_w (BF16 if w_is_bf16, else FP32);
 * d_grad float [n_params]; d_loss_or_null float [1]. */
int ovro_scorer_grad(const void* d_w, int w_is_bf16, const float* d_x, const float* d_y, int batch,
                     float* d_grad, float* d_loss_or_null, void* d_ws, size_t ws_bytes, void* stream);
/* One Adam step (step >= 1) on the FP32 master weights; refreshes the BF16
 * copy when d_w_bf16_or_null is given. */
int ovro_scorer_adam(float* d_master, float* d_m, float* d_v, const float* d_grad, int step, float lr,
                     void* d_w_bf16_or_null, void* stream);
/* BF16 copy (round to nearest even) of the FP32 master weights. */
int ovro_scorer_to_bf16(const float* d_master, void* d_w_bf16, void* stream);

/* -------------------------------------------------------------------------
 * Sharded search: the same Stage I search with coarse channels spread over
 * several processes (one GPU each).  a8-a10 and a12 run per shard; a11's
 * Benjamini-Hochberg family spans every shard (m = in-horizon pixels x all
 * fine channels), so the shards' SNR histograms are summed on the host and
 * the cut is decided bin by bin (ovro_bh_bin_verdict): a bin whose verdict the
 * bin edges leave open is resolved from the values every shard holds in it
 * (ovro_search_bin_values, then ovro_bh_resolve on their union, descending).
 * Every shard then runs NMS at the common cut (ovro_search_candidates).
 * With one shard this is exactly ovro_detect.
 *
 * The handle holds host memory only; the workspace (ovro_detect_workspace_size
 * bytes) stays bound until ovro_search_destroy.
 * ------------------------------------------------------------------------- */
typedef struct ovro_search ovro_search;
int ovro_search_create(int n_chan, int image_size, double cell_dircos, int n_coarse, const int32_t* h_nfft,
                       const ovro_detect_params* params, void* d_ws, size_t ws_bytes, void* stream,
                       ovro_search** out);
/* Clears the histogram for a new integration. */
int ovro_search_reset(ovro_search* s, void* stream);
/* a8-a10 for coarse channel `coarse`: d_img_block holds its nfft images [nfft][N][N]. */
int ovro_search_add(ovro_search* s, int coarse, const float* d_img_block, void* stream);
/* Histogram floor key, bin count and this shard's number of tests. */
int ovro_search_layout(const ovro_search* s, uint32_t* key0, int* n_bins, long long* n_tests);
/* This shard's SNR histogram (synchronises). */
int ovro_search_histogram(ovro_search* s, unsigned long long* h_hist, int n_bins, void* stream);
/* SNR values of this shard in histogram bin `bin` (any order; synchronises).
 * *n is the count; OVRO_ERR_CAPACITY if it exceeds cap. */
int ovro_search_bin_values(ovro_search* s, int bin, float* h_vals, long long cap, long long* n, void* stream);
/* NMS at SNR >= cut; candidates as ovro_detect (synchronises). */
int ovro_search_candidates(ovro_search* s, float cut, const double* h_chan_freq_hz, ovro_candidate* h_out,
                           int max_out, int* n_out, void* stream);
void ovro_search_destroy(ovro_search* s);

/* Host-only pieces of the threshold.  Bins are of the order-preserving 32-bit
 * key of the FP32 SNR shifted right by 16 (ovro_snr_bin_key); bin b holds
 * keys key0 + b, the last bin everything above.  ovro_bh_layout gives key0 and
 * the bin count for the parameters.  The verdict of bin b given the summed
 * histogram and the total number of tests: 0 no value in it can pass, 1 every
 * value passes (the cut is *lo_edge), 2 open, 3 empty; *above_next = count of
 * values above the bin.  ovro_bh_resolve: 1 and *cut = the lowest passing
 * value of an open bin (values descending), or 0. */
int ovro_bh_layout(const ovro_detect_params* params, uint32_t* key0, int* n_bins);
int ovro_bh_bin_verdict(const unsigned long long* h_hist, int n_bins, uint32_t key0, double n_tests, double alpha,
                        int bin, float* lo_edge, unsigned long long* above_next);
int ovro_bh_resolve(const float* h_vals_desc, long long n, unsigned long long above_next, double n_tests,
                    double alpha, float* cut);
uint32_t ovro_snr_bin_key(float snr);

/* -------------------------------------------------------------------------
 * a14  Batched pipeline: every coarse channel of an integration, one graph
 *
 * Section 2.1 processes the upchannelised data in batches because the
 * intermediate products are too large to hold at once; this driver streams
 * coarse channels through fixed buffers: for each coarse channel c,
 * a1-a3 (ovro_upchan), a4 (ovro_correlate), a5-a7 (ovro_grid_image) and
 * a8-a10 (the detection filter) run into one set of buffers, and the SNR of
 * every voxel of every coarse channel is kept; a11-a12 then run once over the
 * whole integration (one Benjamini-Hochberg family, m = pixels x all fine
 * channels).  Results equal ovro_upchan + ovro_correlate + ovro_grid_image +
 * ovro_detect over all coarse channels at once.
 *
 * With use_graph, the device work of one integration (everything before the
 * threshold) is captured once into a CUDA graph and replayed by later runs on
 * the same voltage buffer (a new buffer address is captured anew).
 * Launch shapes come from the autotuner's cache (ovro_autotune).
 *
 * The pipeline handle owns host memory only; the device workspace is the
 * caller's (ovro_pipeline_workspace_size bytes, 256-byte aligned, bound with
 * ovro_pipeline_bind and kept until ovro_pipeline_destroy).  A handle is used
 * from one host thread at a time.
 * ------------------------------------------------------------------------- */
typedef struct ovro_pipeline ovro_pipeline;

typedef struct {
  int n_ant;                      /* dual-polarisation antennas (inputs = 2 n_ant) */
  int n_coarse;
  const int32_t* h_nfft;          /* [n_coarse] fine channels per coarse channel */
  const double* h_coarse_hz;      /* [n_coarse] centre sky frequency of each coarse channel */
  int64_t n_time;                 /* complex samples per coarse channel per integration */
  const double* h_ant_enu_m;      /* [n_ant][3] antenna positions, metres */
  int image_size;                 /* N */
  double cell_dircos;             /* pixel size */
  int xeng_mode;                  /* OVRO_XENG_TC or OVRO_XENG_FP32 */
  ovro_detect_params detect;      /* threshold and filter parameters */
  int use_graph;                  /* nonzero: replay the device work as a CUDA graph */
} ovro_pipeline_config;

/* Plans the pipeline (host only; the config's arrays are copied).  Fine
 * channel k of coarse channel c is at h_coarse_hz[c] + (k - nfft/2) *
 * coarse_bw_hz / nfft. */
int ovro_pipeline_create(const ovro_pipeline_config* cfg, ovro_pipeline** out);
size_t ovro_pipeline_workspace_size(const ovro_pipeline* pl);
/* Binds the workspace and uploads the geometry tables (synchronises stream). */
int ovro_pipeline_bind(ovro_pipeline* pl, void* d_ws, size_t ws_bytes, void* stream);
/* One integration: d_volt uint8 [n_coarse][n_time][2 n_ant] packed 4+4-bit
 * samples (as ovro_upchan).  Candidates as ovro_detect (synchronises stream).
 * Returns OVRO_ERR_TIMEOUT if a tensor-core wait gave up in any coarse channel.
 * While the autotuner is enabled, runs launch eagerly (no graph) and tune
 * every site on first use; the graph is captured by the first run after it is
 * disabled. */
int ovro_pipeline_run(ovro_pipeline* pl, const uint8_t* d_volt, ovro_candidate* h_out, int max_out,
                      int* n_out, void* stream);
/* The device part of one integration only (everything before the
 * threshold; graph replay as ovro_pipeline_run; synchronises stream).  The
 * integration's SNR histogram, bin values and NMS at a cut are then read
 * through the search view below -- for a threshold decided across several
 * pipelines, one per GPU (Section 2.4's single Benjamini-Hochberg family over
 * every shard's tests). */
int ovro_pipeline_run_device(ovro_pipeline* pl, const uint8_t* d_volt, void* stream);
/* A search handle over the pipeline's whole-integration search (layout,
 * histogram, bin values, candidates as the ovro_search_* calls).  It borrows
 * the pipeline's workspace: valid while the pipeline stays bound; release it
 * with ovro_search_destroy, which leaves the pipeline untouched. */
int ovro_pipeline_search(ovro_pipeline* pl, ovro_search** out);
/* Fine channels in the integration and their sky frequencies (host array of
 * that length, or NULL to query the count). */
int ovro_pipeline_channels(const ovro_pipeline* pl, double* h_freq_or_null);
/* Kernels the last run launched (graph replay, threshold and NMS included)
 * and whether a graph is live. */
int ovro_pipeline_stats(const ovro_pipeline* pl, long long* kernels_per_run, int* graph_live);
/* Cross visibilities the last run gridded, summed over channels (each
 * baseline once, mirrors not counted; synchronises). */
int ovro_pipeline_gridded(ovro_pipeline* pl, long long* n_gridded, void* stream);
void ovro_pipeline_destroy(ovro_pipeline* pl);

/* -------------------------------------------------------------------------
 * Autotuner: launch shapes (CTAs per SM of k_xeng_tc, k_rank and k_mf;
 * channels per imaging launch) that give identical results are timed on first
 * use while tuning is enabled (never inside a graph capture) and the fastest
 * is cached per key "kernel/sm<SMs>/<shape...>".  Untuned keys use built-in
 * defaults.  The cache is process-wide; save/load use a text file with one
 * "key value" line per entry.
 * ------------------------------------------------------------------------- */
int ovro_autotune(int enable);
int ovro_tune_get(const char* key, int* value);
int ovro_tune_set(const char* key, int value);
int ovro_tune_count(void);
int ovro_tune_clear(void);
int ovro_tune_save(const char* path);
int ovro_tune_load(const char* path);

#ifdef __cplusplus
}
#endif
#endif /* OVRO_H */
