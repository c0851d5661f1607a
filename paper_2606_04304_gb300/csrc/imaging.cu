// a5-a7: uvw, prolate-spheroidal gridding and dirty imaging per fine channel.
//
// Section 2.2 of the paper images every fine channel over the visible
// hemisphere; the dirty images are the search product.  Per channel:
//
//  a5  u = (x_a - x_b) s_nu in grid cells with s_nu = nu / (c du): one
//      correctly rounded FP64 multiply per coordinate, then rounded to 1/Q
//      cell.  GB300's FP64 pipe is narrow, so the kernels evaluate it as a
//      float-float product and only falls back to a real FP64 multiply when
//      the float-float bound cannot decide rint(u Q) (|frac - 1/2| within the
//      error bound) -- the integer result equals the FP64 definition exactly.
//  a6  Stokes I = (XX + YY)/2 of each kept cross baseline is gridded once (the
//      mirror conj(V) at (-u, -v) is accounted for by taking 2 Re of the
//      transform, which is exact because the mirror's footprint is the point
//      reflection), with a separable 7 x 7 prolate-spheroidal kernel.  The uv
//      position of a baseline moves by a fraction of a cell across a call's
//      channels, so the host lists, once per call, the baselines that can
//      touch each 4 x 8-cell tile of the grid; k_grid_tiles gives every tile
//      to one warp whose 32 lanes are 32 adjacent channels: each lane takes
//      the tile's records for its own channel (exact uv, keep test, weights)
//      and accumulates the tile in registers, so no cell is written by two
//      threads and there are no atomics.  k_fft_rows transforms the rows.
//  a7  The uv grid is padded by 2 (G = 2N cells a side, du = 1 / (G cell)) and
//      the image is the central N x N of its transform, as padded imagers do:
//      the horizon then sits where the kernel's transform is still > 0.25, so
//      the grid correction does not amplify FP32 round-off.  The image is
//      the real part of the transform, i.e. the transform of the grid's
//      Hermitian part, whose row transforms come in conjugate pairs: k_fft_rows
//      forms that part, transforms rows 0 .. G/2 only and keeps the N central
//      columns; k_fft_cols
//      transforms those columns, keeps the N central rows, and applies the
//      (-1)^(r+c) centring sign, normalisation, grid correction and horizon
//      mask while writing the image.  The (-1)^(ku+kv) centring sign is
//      applied at gridding time, and the exp(+) transform is a forward
//      transform of the conjugated grid.  Channel batches keep the
//      intermediate half-transformed grids L2-sized.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "fft.cuh"
#include "pswf.h"
#include "stages.h"
#include "tune.h"

namespace ovro {
namespace {

constexpr double kCLight = 299792458.0;
constexpr int kQ = kOversample;
constexpr int kHalfTab = kSupport * kOversample / 2;
constexpr int kTabLen = 2 * kHalfTab + 1;
constexpr int kHalfSup = kSupport / 2;
constexpr int kPad = 2;              // uv grid cells per image pixel, per axis
// storage of the half-transformed grid between the row and column passes
constexpr int kStoreF32 = OVRO_STORE_FP32, kStoreBF16 = OVRO_STORE_BF16, kStoreF16 = OVRO_STORE_FP16;

struct Baseline {
  double dx, dy;
  float dxh, dxl, dyh, dyl;
  long long bl;
};

struct ChanScale {
  double s;          // s_nu * Q
  double nu_c;       // nu / c (wavelengths per metre)
  float sh, sl;      // float-float split of s
};

__host__ __device__ __forceinline__ long long bl_index(int a, int b, int n) {
  return static_cast<long long>(a) * n - static_cast<long long>(a) * (a - 1) / 2 + (b - a);
}

__global__ void k_baselines(const double* __restrict__ ant, int n_ant, Baseline* __restrict__ out) {
  const int a = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_ant || b <= a) return;
  const long long bl = bl_index(a, b, n_ant);
  Baseline B;
  B.dx = ant[3 * a] - ant[3 * b];
  B.dy = ant[3 * a + 1] - ant[3 * b + 1];
  B.dxh = static_cast<float>(B.dx);
  B.dxl = static_cast<float>(B.dx - static_cast<double>(B.dxh));
  B.dyh = static_cast<float>(B.dy);
  B.dyl = static_cast<float>(B.dy - static_cast<double>(B.dyh));
  B.bl = bl;
  out[bl - a - 1] = B;            // cross baselines in (a, b), a < b, row-major order
}

__global__ void k_chan_scale(const double* __restrict__ freq, int n_chan, int n, double cell,
                             ChanScale* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_chan) return;
  const double du = 1.0 / (static_cast<double>(n) * cell);
  const double s = freq[f] / (kCLight * du);
  ChanScale c;
  c.s = s * static_cast<double>(kQ);          // exact: Q is a power of two
  c.nu_c = freq[f] / kCLight;
  c.sh = static_cast<float>(c.s);
  c.sl = static_cast<float>(c.s - static_cast<double>(c.sh));
  out[f] = c;
}

// rint(fl64(x * s)) decided in FP32: a float-float product, exact unless the
// fractional part is within the error bound (1.2e-7) of 1/2 or |x s| >= 2^21;
// returns false in those (rare) cases, where the FP64 product must be taken.
__device__ __forceinline__ bool fast_rint_prod(float xh, float xl, const ChanScale& s, long long* p) {
  const float hi = __fmul_rn(xh, s.sh);
  if (!(fabsf(hi) < 2097152.0f)) return false;
  const float e = __fmaf_rn(xh, s.sh, -hi);           // exact error of hi
  const float t = __fmaf_rn(xh, s.sl, __fmaf_rn(xl, s.sh, e));
  const float n = rintf(hi);
  const float f = __fadd_rn(hi - n, t);              // x s - n, |error| < 1.2e-7
  if (fabsf(fabsf(f) - 0.5f) <= 2.5e-7f) return false;
  long long q = static_cast<long long>(n);
  if (f > 0.5f) ++q;
  else if (f < -0.5f) --q;
  *p = q;
  return true;
}

__device__ __forceinline__ long long exact_rint_prod(double x, float xh, float xl, const ChanScale& s) {
  long long p;
  if (fast_rint_prod(xh, xl, s, &p)) return p;
  return __double2ll_rn(__dmul_rn(x, s.s));
}

// The same decision in 32-bit integers (|x s| < 2^21 is required anyway).
__device__ __forceinline__ bool fast_rint_prod32(float xh, float xl, const ChanScale& s, int* p) {
  const float hi = __fmul_rn(xh, s.sh);
  if (!(fabsf(hi) < 2097152.0f)) return false;
  const float e = __fmaf_rn(xh, s.sh, -hi);
  const float t = __fmaf_rn(xh, s.sl, __fmaf_rn(xl, s.sh, e));
  const float n = rintf(hi);
  const float f = __fadd_rn(hi - n, t);
  if (fabsf(fabsf(f) - 0.5f) <= 2.5e-7f) return false;
  *p = __float2int_rn(n) + (f > 0.5f ? 1 : 0) - (f < -0.5f ? 1 : 0);   // n is integral, |n| < 2^21
  return true;
}

static_assert(kQ == 1024, "centre_cell32 divides by shifting");
__device__ __forceinline__ void centre_cell32(int p, int& c0, int& off) {
  const int c = (abs(p) + kQ / 2) >> 10;
  c0 = p < 0 ? -c : c;
  off = p - c0 * kQ;
}

// a5 on its own: rounded positions p_u, p_v (1/Q cells) of every cross baseline.
__global__ void k_uvw(const Baseline* __restrict__ base, int n_cross, const ChanScale* __restrict__ cs,
                      int32_t* __restrict__ pu, int32_t* __restrict__ pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (i >= n_cross) return;
  const Baseline B = base[i];
  const ChanScale s = cs[f];
  const long long u = exact_rint_prod(B.dx, B.dxh, B.dxl, s);
  const long long v = exact_rint_prod(B.dy, B.dyh, B.dyl, s);
  const long long lim = 1LL << 30;
  const long long o = static_cast<long long>(f) * n_cross + i;
  pu[o] = static_cast<int32_t>(u > lim ? lim : (u < -lim ? -lim : u));
  pv[o] = static_cast<int32_t>(v > lim ? lim : (v < -lim ? -lim : v));
}

struct GridEntry {
  int bl;            // baseline index in the visibility record
  int cross;         // cross-baseline index (FP64 fallback, baseline length)
  int a;             // antennas a < b
  int bf;            // b | kCheckUv when the uv range must be decided per channel
  float dxh, dxl, dyh, dyl;
};
constexpr int kCheckUv = 1 << 16;

// Calibration and baseline-selection options of one gridding call.
struct GridOpts {
  const float2* gains;      // [n_chan][n_input] corrections or nullptr
  int n_input;
  const double* blen;       // [n_cross] baseline lengths, metres (FP64)
  double uv_min, uv_max;    // wavelengths, [uv_min, uv_max)
};

// Row pitch of a shared-memory grid band: G + G/16 pad slots, rounded so the
// pitch is 7 (mod 16) float2 -- consecutive rows then start 14 banks apart and
// 16 consecutive transposed columns hit distinct banks.
__host__ __device__ constexpr int band_pitch(int g) { return (g + g / 16) + ((7 - (g + g / 16) % 16) + 16) % 16; }

// Gridding tiles.  A warp owns a kTileV x kTileU tile of grid cells for 32
// consecutive channels, one channel per lane, and keeps the tile's 32 complex
// accumulators of its channel in registers.  Every lane of a warp takes the
// same visibility record at the same time; across 32 adjacent fine channels a
// baseline's uv position moves by far less than a cell, so the lanes' centre
// cells agree (or differ by one) and their table reads hit the same words.
// No two warps write the same (cell, channel): there are no atomics.
constexpr int kTileV = 4, kTileU = 4;          // cells per warp tile (rows, columns)
constexpr int kLanes = 32;                     // channels per warp

// Tiles cover the rows G/2 .. G-1 (v >= 0) of the grid's Hermitian part only
// (the rows below are the conjugate reflection).
__host__ __device__ constexpr int n_tiles_u(int g) { return g / kTileU; }
__host__ __device__ constexpr int n_tiles(int g) { return (g / 2 / kTileV) * (g / kTileU); }

// Weights of the separable kernel indexed by (d, off): a tap d cells from the
// centre cell of a position whose offset from that cell is off / Q weighs
// C(d - off / Q) when |d| <= 3 and 0 otherwise.  The table holds every d in
// [-kTabD, kTabD] at stride Q + 1, so (d, off) -> (d + kTabD) (Q + 1) + Q / 2 - off
// is one-to-one over off in [-Q/2, Q/2] (d = 3 at off = -Q/2 and d = 4 at
// off = Q/2 land on different entries) and a tile's weights are plain loads at
// fixed strides from one base, with no range tests.  Offsets a tile column
// can take when the footprint touches the tile lie in [-(3 + kTileU - 1), 3];
// the kTabMargin rows beyond them (zeros) let a lane whose centre is up to
// kTabMargin cells from a tile it is listed for read zeros there.
constexpr int kTabMargin = 4;
constexpr int kTabD = kHalfSup + kTileU - 1 + kTabMargin;   // 10
constexpr int kTabStride = kQ + 1;
constexpr int kTabXLen = (2 * kTabD + 1) * kTabStride;

// Per-channel record of one listed baseline, prepared once per channel group
// by k_grid_prep: its exact rounded position p = rint(u Q), rint(v Q) and its
// value in the Hermitian part of the grid, conj(Stokes I) / 2, or V = 0 when
// the visibility is not gridded in that channel.  Layout [group][listed][32].
// With table bases (a call whose footprints move by less than kTabMargin
// cells over its channels), pu and pv hold instead the weight-table offsets
// of the position: column c's weight is tabx[pu + c (Q + 1)], row r's
// tabx[pv + r (Q + 1)] (r, c grid indices), zero beyond the footprint.
struct PrepRec {
  int pu, pv;
  float vr, vi;
};
constexpr int kMirror = 1 << 31;    // tile list flag: grid the record's mirror (-u, -v, conj V)

// Table offset of a position with centre cell c and offset off (1/Q cells)
// on an axis of G cells; the mirror position (-c, -off) has offset
// tab_mirror(G) - tab_base(G, c, off).
__host__ __device__ constexpr int tab_base(int g, int c, int off) {
  return (kTabD - g / 2 - c) * kTabStride + kQ / 2 - off;
}
__host__ __device__ constexpr int tab_mirror(int g) { return 2 * (kTabD - g / 2) * kTabStride + kQ; }

// a5 and the Stokes I of a6 for one channel group and kPrepBl listed
// baselines per CTA: for each (channel, baseline) a thread decides the exact
// rounded position (float-float, FP64 when that cannot decide), the keep test
// (centre cell inside the grid's margin; the uv range when it must be decided
// per channel), reads XX and YY and forms the record -- the image is the real
// part of the transform, i.e. the transform of the grid's Hermitian part
// H = (G + conj G(-u, -v)) / 2, so the record carries half of
// conj(Stokes I) = conj(XX + YY) / 4 (the exp(+) transform is a forward FFT of
// the conjugated grid); calibration corrections c_a conj(c_b) are applied per
// polarisation in FP32 when given.  Lanes are baselines while the
// visibilities are read (a warp reads consecutive baselines of one channel:
// nearly sequential 32-byte records), and the records are turned around in
// shared memory so each baseline's 32 channel records are stored as one
// 512-byte run ([group][listed][lane]).  Kept visibilities are counted per
// channel.
constexpr int kPrepBl = 64;          // listed baselines per CTA of k_grid_prep
constexpr int kPrepCh = kLanes / 8;  // channels per warp (8 warps)

template <int LOG2G, bool CAL, bool BASES>
__global__ void __launch_bounds__(256, CAL ? 1 : 4)
k_grid_prep(const GridEntry* __restrict__ listed, int n_listed, const int32_t* __restrict__ vis, long long n_bl,
            const Baseline* __restrict__ base, const ChanScale* __restrict__ cs, int ch0, int nb,
            int* __restrict__ kept, PrepRec* __restrict__ prep, GridOpts opt) {
  constexpr int G = 1 << LOG2G;
  // [baseline][channel] records, rows padded by one record so that the lanes'
  // 16-byte stores (lanes = baselines) fall in distinct banks
  __shared__ int4 tile[kPrepBl][kLanes + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int group = blockIdx.y;
  const int i0 = blockIdx.x * kPrepBl;
  const int nbl = min(kPrepBl, n_listed - i0);
  const int cmax = G / 2 - kHalfSup - 1;
  const int lim = (cmax + 1) * kQ;                     // < 2^21
  // this lane's two baselines (i0 + lane, i0 + lane + 32)
  GridEntry en[2];
  bool has[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int bi = lane + 32 * h;
    has[h] = bi < nbl;
    en[h] = listed[i0 + (has[h] ? bi : 0)];
  }
  // every visibility read of the thread (kPrepCh channels x 2 baselines) is
  // issued before any is used
  int2 xx[kPrepCh][2], yy[kPrepCh][2];
#pragma unroll
  for (int cc = 0; cc < kPrepCh; ++cc) {
    const int cb = group * kLanes + warp * kPrepCh + cc;
    const long long chan = ch0 + (cb < nb ? cb : nb - 1);
    const int2* vis2 = reinterpret_cast<const int2*>(vis) + chan * n_bl * 4;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      xx[cc][h] = __ldg(vis2 + static_cast<long long>(en[h].bl) * 4);
      yy[cc][h] = __ldg(vis2 + static_cast<long long>(en[h].bl) * 4 + 3);
    }
  }
#pragma unroll
  for (int cc = 0; cc < kPrepCh; ++cc) {
    const int cl = warp * kPrepCh + cc;              // channel within the group
    const int cb = group * kLanes + cl;
    const bool active = cb < nb;
    const long long chan = ch0 + (active ? cb : nb - 1);
    const ChanScale sc = cs[chan];
    const float2* gc = (CAL && opt.gains != nullptr) ? opt.gains + chan * opt.n_input : nullptr;
    int n_kept = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const GridEntry& e = en[h];
      int pu, pv;
      if (!fast_rint_prod32(e.dxh, e.dxl, sc, &pu)) {
        const long long pl = __double2ll_rn(__dmul_rn(base[e.cross].dx, sc.s));
        pu = static_cast<int>(pl > lim ? lim : (pl < -lim ? -lim : pl));
      }
      if (!fast_rint_prod32(e.dyh, e.dyl, sc, &pv)) {
        const long long pl = __double2ll_rn(__dmul_rn(base[e.cross].dy, sc.s));
        pv = static_cast<int>(pl > lim ? lim : (pl < -lim ? -lim : pl));
      }
      bool keep = pu > -lim && pu < lim && pv > -lim && pv < lim;
      if (keep) {
        int cu, cv, o;
        centre_cell32(pu, cu, o);
        centre_cell32(pv, cv, o);
        keep = cu <= cmax && cu >= -cmax && cv <= cmax && cv >= -cmax;
      }
      if (CAL && (e.bf & kCheckUv)) {
        const double lam = __dmul_rn(opt.blen[e.cross], sc.nu_c);
        keep = keep && lam >= opt.uv_min && lam < opt.uv_max;
      }
      PrepRec r{lim, lim, 0.0f, 0.0f};
      if (BASES) {
        // the position's table offsets, kept or not (a record is only read for
        // tiles within kTabMargin cells of its footprint)
        int cu, cv, ou, ov;
        centre_cell32(pu, cu, ou);
        centre_cell32(pv, cv, ov);
        r.pu = tab_base(G, cu, ou);
        r.pv = tab_base(G, cv, ov);
      }
      if (keep) {
        float vr, vi;
        if (!CAL || gc == nullptr) {
          vr = 0.25f * static_cast<float>(xx[cc][h].x + yy[cc][h].x);
          vi = -0.25f * static_cast<float>(xx[cc][h].y + yy[cc][h].y);
        } else {
          const int a = e.a, b = e.bf & 0xffff;
          float pr = 0.f, pi = 0.f;
#pragma unroll
          for (int pol = 0; pol < 2; ++pol) {
            const float2 ca = __ldg(gc + 2 * a + pol), cbv = __ldg(gc + 2 * b + pol);
            const int2 q = pol ? yy[cc][h] : xx[cc][h];
            const float qr = static_cast<float>(q.x), qi = static_cast<float>(q.y);
            const float gr = ca.x * cbv.x + ca.y * cbv.y, gi = ca.y * cbv.x - ca.x * cbv.y;
            pr += gr * qr - gi * qi;
            pi += gr * qi + gi * qr;
          }
          vr = 0.25f * pr;
          vi = -0.25f * pi;
        }
        if (!BASES) {
          r.pu = pu;
          r.pv = pv;
        }
        r.vr = vr;
        r.vi = vi;
        if (has[h]) ++n_kept;
      }
      tile[lane + 32 * h][cl] = make_int4(r.pu, r.pv, __float_as_int(r.vr), __float_as_int(r.vi));
    }
    // the channel's kept visibilities over the warp's 64 baselines
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_kept += __shfl_xor_sync(0xffffffffu, n_kept, o);
    if (lane == 0 && active && n_kept) atomicAdd(kept + chan, n_kept);
  }
  __syncthreads();
  // one baseline's 32 channel records per warp store: 512 contiguous bytes
  int4* out = reinterpret_cast<int4*>(prep) + (static_cast<long long>(group) * n_listed + i0) * kLanes;
  for (int bi = warp; bi < nbl; bi += 8) out[static_cast<long long>(bi) * kLanes + lane] = tile[bi][lane];
}

// Gridding of one channel batch into the Hermitian part of the grid, rows
// G/2 .. G-1 (v >= 0; a record whose footprint lies below is listed as its
// mirror, one straddling row G/2 as both).  Work items are (group of 32
// channels, warp tile) pairs, group-major, the tiles of a group taken from the
// longest list to the shortest; every warp of the persistent grid (one CTA of
// kGridWarps warps per SM) takes items kGridWarps * gridDim.x apart, so each
// warp starts on a heavy tile and ends on light ones.  The gap-indexed weight
// table sits in shared memory, loaded once per CTA.  For every list entry of
// its tile, a lane reads its channel's prepared record (one 16-byte load, the
// warp's 32 lanes contiguous), mirrors it if flagged, reads the tile's 4 row
// and 4 column weights of the separable kernel and adds the products into its
// accumulators; kRing records are in flight per warp and their list entries
// are read 2 kRing ahead.
//   BASES: the record holds the weight-table offsets of its position, so the
//     weights are 8 loads at fixed strides from (offset + tile origin) and a
//     lane off the footprint reads the table's zero rows;
//   otherwise the lane takes the centre cells from the position and adds
//     zeros when its footprint misses the tile.
// The tile is written with the (-1)^(row + col) centring sign as two real
// planes, grid [batch][2][G/2][G] (row j - G/2).
constexpr int kGridWarps = 20;
constexpr int kRing = 4;           // records in flight per warp
constexpr size_t kTileSmem = static_cast<size_t>(kTabXLen) * sizeof(float);

template <int LOG2G, bool BASES>
__global__ void __launch_bounds__(kGridWarps * 32, 1)
k_grid_tiles(const int* __restrict__ tile_idx, const int* __restrict__ tile_off, const int* __restrict__ tile_order,
             const PrepRec* __restrict__ prep, int n_listed, const float* __restrict__ tabx_g, int nb,
             float* __restrict__ grid) {
  constexpr int G = 1 << LOG2G;
  constexpr int NTU = n_tiles_u(G);
  constexpr int NT = n_tiles(G);
  constexpr long long PLANE = static_cast<long long>(G / 2) * G;
  extern __shared__ __align__(16) unsigned char smem[];
  float* tabx = reinterpret_cast<float*>(smem);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kTabXLen / 4; i += blockDim.x)
    reinterpret_cast<float4*>(tabx)[i] = __ldg(reinterpret_cast<const float4*>(tabx_g) + i);
  for (int i = (kTabXLen / 4) * 4 + threadIdx.x; i < kTabXLen; i += blockDim.x) tabx[i] = __ldg(tabx_g + i);
  __syncthreads();
  const int n_groups = (nb + kLanes - 1) / kLanes;
  const long long n_items = static_cast<long long>(n_groups) * NT;
  const int stride = gridDim.x * kGridWarps;
#pragma unroll 1
  for (long long item = static_cast<long long>(blockIdx.x) * kGridWarps + warp; item < n_items; item += stride) {
    const int g = static_cast<int>(item / NT);
    const int tile = __ldg(tile_order + (item - static_cast<long long>(g) * NT));
    const int cb = g * kLanes + lane;                 // channel within the batch
    const PrepRec* pg = prep + static_cast<long long>(g) * n_listed * kLanes + lane;
    const int tv = tile / NTU, tu = tile - tv * NTU;
    const int r0 = G / 2 + tv * kTileV, c0 = tu * kTileU;
    const int e0 = tile_off[tile], e1 = tile_off[tile + 1];
    float acr[kTileV][kTileU], aci[kTileV][kTileU];
#pragma unroll
    for (int i = 0; i < kTileV; ++i)
#pragma unroll
      for (int j = 0; j < kTileU; ++j) acr[i][j] = aci[i][j] = 0.0f;
    auto index = [&](int e) { return e < e1 ? __ldg(tile_idx + e) : 0; };
    auto load_rec = [&](int ent) {
      return __ldg(reinterpret_cast<const int4*>(pg + static_cast<long long>(ent & ~kMirror) * kLanes));
    };
    auto accumulate = [&](const float* bu, const float* bv, float vr, float vi) {
      float wv[kTileV], wu[kTileU];
#pragma unroll
      for (int i = 0; i < kTileV; ++i) wv[i] = bv[i * kTabStride];
#pragma unroll
      for (int j = 0; j < kTileU; ++j) wu[j] = bu[j * kTabStride];
#pragma unroll
      for (int i = 0; i < kTileV; ++i) {
        const float br = wv[i] * vr, bi = wv[i] * vi;
#pragma unroll
        for (int j = 0; j < kTileU; ++j) {
          acr[i][j] = fmaf(br, wu[j], acr[i][j]);
          aci[i][j] = fmaf(bi, wu[j], aci[i][j]);
        }
      }
    };
    // one list entry: the record (mirrored if flagged) decoded here, at its use
    auto grid_one = [&](int4 v, int ent) {
      const bool m = ent & kMirror;
      const float vr = __int_as_float(v.z), vi = m ? -__int_as_float(v.w) : __int_as_float(v.w);
      if (BASES) {
        // the table's zero rows stand for taps off the footprint
        const int bu = m ? tab_mirror(G) - v.x : v.x, bv = m ? tab_mirror(G) - v.y : v.y;
        accumulate(tabx + bu + c0 * kTabStride, tabx + bv + r0 * kTabStride, vr, vi);
        return;
      }
      int cu, offu, cv, offv;
      centre_cell32(m ? -v.x : v.x, cu, offu);
      centre_cell32(m ? -v.y : v.y, cv, offv);
      int dv0 = r0 - (G / 2 + cv), du0 = c0 - (G / 2 + cu);   // offsets of the tile's first row / column
      const bool touch = dv0 <= kHalfSup && dv0 >= -(kHalfSup + kTileV - 1) && du0 <= kHalfSup &&
                         du0 >= -(kHalfSup + kTileU - 1);
      if (__any_sync(full, touch)) {
        float wr = vr, wi = vi;
        if (!touch) {
          // a lane whose footprint misses the tile adds zeros; its table
          // reads stay inside the table
          wr = wi = 0.0f;
          dv0 = du0 = 0;
          offu = offv = 0;
        }
        accumulate(tabx + (du0 + kTabD) * kTabStride + kQ / 2 - offu,
                   tabx + (dv0 + kTabD) * kTabStride + kQ / 2 - offv, wr, wi);
      }
    };
    // a ring of kRing records in flight, each loaded kRing entries ahead of its
    // use into its own slot (no register moves wait on a load), and their list
    // entries, loaded 2 kRing ahead
    int4 q[kRing];
    int en[kRing], nx[kRing];
#pragma unroll
    for (int d = 0; d < kRing; ++d) en[d] = index(e0 + d);
#pragma unroll
    for (int d = 0; d < kRing; ++d) {
      q[d] = load_rec(en[d]);
      nx[d] = index(e0 + kRing + d);
    }
#pragma unroll 1
    for (int e = e0; e < e1; e += kRing) {
#pragma unroll
      for (int d = 0; d < kRing; ++d) {
        if (e + d < e1) grid_one(q[d], en[d]);
        en[d] = nx[d];
        q[d] = load_rec(en[d]);
        nx[d] = index(e + d + 2 * kRing);
      }
    }
    // ---- the tile, with the centring sign (r0 and c0 are even)
    if (cb < nb) {
      float* gr = grid + static_cast<long long>(cb) * 2 * PLANE;
      float* gi = gr + PLANE;
#pragma unroll
      for (int i = 0; i < kTileV; ++i) {
        float vr[kTileU], vi[kTileU];
#pragma unroll
        for (int j = 0; j < kTileU; ++j) {
          const bool neg = (i + j) & 1;
          vr[j] = neg ? -acr[i][j] : acr[i][j];
          vi[j] = neg ? -aci[i][j] : aci[i][j];
        }
        const long long row = r0 + i - G / 2;
        float4* pr = reinterpret_cast<float4*>(gr + row * G + c0);
        float4* pi = reinterpret_cast<float4*>(gi + row * G + c0);
#pragma unroll
        for (int j = 0; j < kTileU / 4; ++j) {
          pr[j] = make_float4(vr[4 * j], vr[4 * j + 1], vr[4 * j + 2], vr[4 * j + 3]);
          pi[j] = make_float4(vi[4 * j], vi[4 * j + 1], vi[4 * j + 2], vi[4 * j + 3]);
        }
      }
    }
  }
}

// The central N columns of the row transforms of a band of rows in shared
// memory, into the half-transformed grid h ([batch][G][N]) in its storage format.
template <int G, int LDP, int S>
__device__ __forceinline__ void store_band(const float2* band, int band_h, int n_img, long long hrow0, void* h,
                                           float* hs) {
  // band_h: the rows to store (the first rows of the band)
  const int offc = G / 2 - n_img / 2;
  if constexpr (S == kStoreF32) {
    float2* hb = static_cast<float2*>(h) + hrow0 * n_img;
    for (int i = threadIdx.x; i < band_h * n_img; i += blockDim.x) {
      const int r = i / n_img, c = i - r * n_img;
      hb[static_cast<long long>(r) * n_img + c] = band[r * LDP + pad16(offc + c)];
    }
  } else if constexpr (S == kStoreBF16) {
    __nv_bfloat162* hb = static_cast<__nv_bfloat162*>(h) + hrow0 * n_img;
    for (int i = threadIdx.x; i < band_h * n_img; i += blockDim.x) {
      const int r = i / n_img, c = i - r * n_img;
      hb[static_cast<long long>(r) * n_img + c] = __float22bfloat162_rn(band[r * LDP + pad16(offc + c)]);
    }
  } else {
    // FP16 with a power-of-two scale per row: the row's largest component
    // lands in [2^13, 2^14), far from FP16 overflow; scaling is exact
    __half2* hb = static_cast<__half2*>(h) + hrow0 * n_img;
    const int lane = threadIdx.x & 31, n_w = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < band_h; r += n_w) {
      float m = 0.f;
      for (int c = lane; c < n_img; c += 32) {
        const float2 v = band[r * LDP + pad16(offc + c)];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      int e = 0;
      if (m > 0.f) frexpf(m, &e);
      const float sc = m > 0.f ? ldexpf(1.0f, 14 - e) : 1.0f;
      if (lane == 0) hs[hrow0 + r] = m > 0.f ? ldexpf(1.0f, e - 14) : 0.0f;
      for (int c = lane; c < n_img; c += 32) {
        const float2 v = band[r * LDP + pad16(offc + c)];
        hb[static_cast<long long>(r) * n_img + c] = __float22half2_rn(make_float2(v.x * sc, v.y * sc));
      }
    }
  }
}

// Row pitch (floats) of the two real planes of a band staged in shared
// memory: G + 4, 16-byte rows (the planes overlap the FFT layout, which the
// first Stockham pass only writes after all its reads).
__host__ __device__ constexpr int planar_pitch(int g) { return g + 4; }

// Rows of the half-transformed grid kept per channel: the gridded plane is the
// Hermitian part H of the grid on its rows j = G/2 .. G-1; the row transforms
// of H satisfy R(G - j, k) = conj R(j, k), and row 0 is empty (no footprint
// reaches it), so these G/2 rows carry everything the column pass needs.
__host__ __device__ constexpr int half_rows(int g) { return g / 2; }

// Row transforms of one band of rows of the gridded half plane of one channel:
// the two real planes are staged in shared memory with 16-byte loads (all in
// flight at once), the first Stockham pass reads them, the rest run in place;
// the central N columns go to h ([batch][G/2][N], row j - G/2).
template <int LOG2G, int S>
__global__ void __launch_bounds__(1024)
k_fft_rows(const float* __restrict__ grid, const float2* __restrict__ tw_g, int n_img, int band_h,
           void* __restrict__ h, float* __restrict__ hs) {
  constexpr int G = 1 << LOG2G;
  constexpr int LDP = band_pitch(G);
  constexpr int P = planar_pitch(G);
  static_assert(2 * P <= 2 * LDP, "planar band fits in the FFT layout");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* band = reinterpret_cast<float2*>(smem);     // [band_h][LDP]
  float* pre = reinterpret_cast<float*>(smem);        // [band_h][P] (staging)
  float* pim = pre + band_h * P;
  float2* tw = band + band_h * LDP;                   // [G]
  const int b = blockIdx.x, cb = blockIdx.y;
  const int row0 = b * band_h;
  for (int i = threadIdx.x; i < G; i += blockDim.x) tw[i] = tw_g[i];
  const long long plane4 = static_cast<long long>(half_rows(G)) * G / 4;
  const float4* src = reinterpret_cast<const float4*>(grid) + static_cast<long long>(cb) * 2 * plane4 +
                      static_cast<long long>(row0) * (G / 4);
  constexpr int RQ = G / 4;                           // float4 per row
  // 2 band_h G / 4 float4 over band_h G / 16 threads: 8 per thread, all
  // issued before the first is stored
  constexpr int PER = 8;
  const int n1 = band_h * RQ;
  float4 q[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = threadIdx.x + u * blockDim.x;
    const int pl = i >= n1 ? 1 : 0, k = i - pl * n1;
    q[u] = __ldg(src + pl * plane4 + k);
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = threadIdx.x + u * blockDim.x;
    const int pl = i >= n1 ? 1 : 0, k = i - pl * n1;
    const int r = k / RQ, c = k - r * RQ;
    *reinterpret_cast<float4*>((pl ? pim : pre) + r * P + 4 * c) = q[u];
  }
  __syncthreads();
  // the first pass reads the planar staging (which the band overlaps)
  fft_rows_inplace_f<LOG2G>(
      band, LDP, [&](int f, int x) { return make_float2(pre[f * P + x], pim[f * P + x]); },
      [&](int i) { return tw[i]; });
  store_band<G, LDP, S>(band, band_h, n_img, static_cast<long long>(cb) * half_rows(G) + row0, h, hs);
}

// Two adjacent values (idx even) of the half-transformed grid in FP32.
template <int S>
__device__ __forceinline__ void load_h2(const void* h, const float* hs, long long row, long long idx, float2& v0,
                                        float2& v1) {
  if constexpr (S == kStoreF32) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(static_cast<const float2*>(h) + idx));
    v0 = make_float2(q.x, q.y);
    v1 = make_float2(q.z, q.w);
  } else {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned*>(h) + idx));
    if constexpr (S == kStoreBF16) {
      __nv_bfloat162 b0, b1;
      memcpy(&b0, &raw.x, sizeof(b0));
      memcpy(&b1, &raw.y, sizeof(b1));
      v0 = __bfloat1622float2(b0);
      v1 = __bfloat1622float2(b1);
    } else {
      __half2 b0, b1;
      memcpy(&b0, &raw.x, sizeof(b0));
      memcpy(&b1, &raw.y, sizeof(b1));
      const float sc = __ldg(hs + row);
      v0 = __half22float2(b0);
      v1 = __half22float2(b1);
      v0 = make_float2(v0.x * sc, v0.y * sc);
      v1 = make_float2(v1.x * sc, v1.y * sc);
    }
  }
}

// Column transforms of the N central columns and the image itself.
//
// The row transforms are of the Hermitian part of the grid, so every column c
// satisfies c(-k) = conj c(k) and its DFT is real: two columns c1, c2 share
// one complex FFT of d = c1 + i c2, whose DFT is DFT(c1) + i DFT(c2).  Rows
// G/2 .. G-1 are read; rows G/2 - r are their conjugates and row 0 is empty.
// d is formed doubled and the output scale takes the factor 1/2 back.  C
// columns per CTA, C / 2 transforms.
template <int LOG2G, int S>
__global__ void __launch_bounds__(512, 2)
k_fft_cols(const void* __restrict__ h, const float* __restrict__ hs, int n_img, int cols_per_cta, int ch0,
           const float2* __restrict__ tw_g, const float* __restrict__ inv_corr,
           const uint8_t* __restrict__ mask, const int* __restrict__ kept, float* __restrict__ img) {
  constexpr int G = 1 << LOG2G;
  constexpr int LDP = band_pitch(G);
  extern __shared__ __align__(16) unsigned char smem[];
  const int C = cols_per_cta, CP = C / 2;             // powers of two
  const int cp_shift = __ffs(CP) - 1;
  float2* A = reinterpret_cast<float2*>(smem);        // [C / 2][LDP]: packed column pairs
  float2* tw = A + CP * LDP;
  const int cb = blockIdx.y;
  const int c0 = blockIdx.x * C;
  const long long hrow0 = static_cast<long long>(cb) * half_rows(G);
  for (int i = threadIdx.x; i < G; i += blockDim.x) tw[i] = tw_g[i];
  // U items per thread in flight: the reads come from L2 and would otherwise
  // wait one round trip each
  constexpr int U = 8;
  const int n_items = half_rows(G) * CP;
  for (int p = threadIdx.x; p < CP; p += blockDim.x) A[p * LDP] = make_float2(0.0f, 0.0f);   // row 0: empty
  for (int i0 = threadIdx.x; i0 < n_items; i0 += U * blockDim.x) {
    float2 a[U], e[U];                                // c1, c2 at row j = G/2 + r
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n_items) {
        const int r = i >> cp_shift, p = i & (CP - 1);
        load_h2<S>(h, hs, hrow0 + r, (hrow0 + r) * n_img + c0 + 2 * p, a[u], e[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n_items) {
        const int r = i >> cp_shift, p = i & (CP - 1);
        const int j = G / 2 + r, jm = G / 2 - r;      // rows j and G - j
        // d = 2 (c1 + i c2); at G - j the columns are conjugated
        A[p * LDP + pad16(j)] = make_float2(2.0f * (a[u].x - e[u].y), 2.0f * (a[u].y + e[u].x));
        if (r > 0) A[p * LDP + pad16(jm)] = make_float2(2.0f * (a[u].x + e[u].y), 2.0f * (e[u].x - a[u].y));
      }
    }
  }
  __syncthreads();
  fft_rows_inplace_f<LOG2G>(
      A, LDP, [&](int f, int x) { return A[f * LDP + pad16(x)]; }, [&](int i) { return tw[i]; });
  const long long chan = ch0 + cb;
  const int k = kept[chan];
  const float norm = k > 0 ? 0.5f / static_cast<float>(k) : 0.0f;
  const int off = G / 2 - n_img / 2;
  float* out = img + chan * n_img * n_img;
#pragma unroll 4
  for (int i = threadIdx.x; i < n_img * C; i += blockDim.x) {
    const int r = i >> (cp_shift + 1), c = i & (C - 1);
    const int col = c0 + c;
    float v = 0.0f;
    if (mask[r * n_img + col]) {
      const float2 z = A[(c >> 1) * LDP + pad16(off + r)];
      v = (c & 1 ? z.y : z.x) * norm * inv_corr[r] * inv_corr[col];
      if ((r + col) & 1) v = -v;
    }
    out[static_cast<long long>(r) * n_img + col] = v;
  }
}

__global__ void k_mask(int n, double cell, uint8_t* __restrict__ mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, c = i - r * n;
  const double l = static_cast<double>(c - n / 2) * cell;
  const double m = static_cast<double>(r - n / 2) * cell;
  mask[i] = (l * l + m * m) < 1.0 ? 1 : 0;
}

__global__ void k_twiddle_img(float2* tw, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi(-2.0 * static_cast<double>(k) / static_cast<double>(n), &s, &c);
  tw[k] = make_float2(static_cast<float>(c), static_cast<float>(s));
}

__global__ void k_counts_out(const int* __restrict__ kept, int n_chan, int32_t* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n_chan) out[f] = 2 * kept[f];
}

// ---------------------------------------------------------------- planning
struct ImgPlan {
  int n, g, log2g, band_h, batch, cols_per_cta, storage;
  long long n_cross;
};

ImgPlan make_plan(int n_ant, int n_chan, int n, int storage) {
  ImgPlan p;
  p.n = n;
  p.storage = storage;
  p.g = kPad * n;
  p.log2g = ilog2(p.g);
  // row transforms: 8192 complex values per band, 512-thread CTAs (several
  // per SM, so one band's loads overlap another's transforms)
  p.band_h = 8192 / p.g < p.g / 2 ? 8192 / p.g : p.g / 2;
  p.n_cross = static_cast<long long>(n_ant) * (n_ant - 1) / 2;
  // channels per launch: whole groups of 32 (one per lane of a tile warp);
  // the gridded half planes, the prepared records and the half-transformed
  // grids of a batch together up to about 256 MB (the autotuner picks among
  // this and its halves down to 32 channels)
  const long long per = 4LL * p.g * p.g + 4LL * p.g * n + 16LL * std::max<long long>(1, p.n_cross);
  long long b = ((256LL << 20) / per) / kLanes * kLanes;
  if (b < kLanes) b = kLanes;
  if (b > 256) b = 256;
  if (b > n_chan) b = n_chan;
  p.batch = static_cast<int>(b);
  // an even number of columns per CTA (the column pass pairs them)
  int c = 8192 / p.g;
  // 16-bit storage: at least 8 columns per CTA, so each row segment the
  // column pass reads is a whole 32-byte sector
  if (storage != kStoreF32 && c < 8 && 8 * p.g / 32 <= 512) c = 8;
  if (c > n) c = n;
  p.cols_per_cta = c;
  return p;
}

struct ImgWs {
  float* tab;
  float* tabx;       // [kTabXLen] weights by (tap offset, position offset)
  float* inv_corr;
  float2* tw;
  uint8_t* mask;
  double* ant;
  double* freq;
  Baseline* base;
  ChanScale* cs;
  int* kept;
  GridEntry* listed; // baselines that can be gridded in some channel of the call
  int* tile_off;     // [n_tiles + 1]
  int* tile_order;   // [n_tiles] tiles by descending list length
  int* tile_idx;     // per tile: indices into listed
  double* blen;      // [n_cross] baseline lengths (metres)
  PrepRec* prep;     // [batch groups][n_cross][32] prepared records
  float* grid;       // [batch][2][G][G] gridded planes (re, im)
  void* h;           // [batch][G][N] complex in the storage format
  float* hs;         // [batch][G] row scales (FP16 storage)
  int n_listed = 0;
  bool bases = false;  // records carry weight-table offsets (footprints move < kTabMargin cells)
};

// Tile list entries: each listed baseline once per warp tile its footprint, or
// its mirror's, can touch in the gridded half plane in some channel of the
// call.  Over a coarse channel a footprint moves by at most a cell, so a
// baseline touches 6 to 9 tiles of 4 x 4 (a footprint straddling row G/2 up to
// as many more through its mirror).
constexpr int kEntriesPerBaseline = 24;
long long entry_capacity(const ImgPlan& p) { return std::max<long long>(1, p.n_cross * kEntriesPerBaseline); }

ImgWs carve_img(void* ws, size_t bytes, const ImgPlan& p, int n_ant, int n_chan, size_t* need) {
  Carver c(ws, bytes);
  ImgWs w;
  const size_t nx = p.n_cross > 0 ? static_cast<size_t>(p.n_cross) : 1;
  w.tab = c.take<float>(kTabLen);
  w.tabx = c.take<float>(kTabXLen);
  w.inv_corr = c.take<float>(p.n);
  w.tw = c.take<float2>(p.g);
  w.mask = c.take<uint8_t>(static_cast<size_t>(p.n) * p.n);
  w.ant = c.take<double>(static_cast<size_t>(n_ant) * 3);
  w.freq = c.take<double>(n_chan);
  w.base = c.take<Baseline>(nx);
  w.cs = c.take<ChanScale>(n_chan);
  w.kept = c.take<int>(n_chan);
  w.listed = c.take<GridEntry>(nx);
  w.tile_off = c.take<int>(n_tiles(p.g) + 1);
  w.tile_order = c.take<int>(n_tiles(p.g));
  w.tile_idx = c.take<int>(entry_capacity(p));
  w.blen = c.take<double>(nx);
  w.prep = c.take<PrepRec>(static_cast<size_t>((p.batch + kLanes - 1) / kLanes) * nx * kLanes);
  w.grid = c.take<float>(static_cast<size_t>(p.batch) * 2 * half_rows(p.g) * p.g);
  w.h = c.take<float2>(static_cast<size_t>(p.batch) * half_rows(p.g) * p.n);
  w.hs = c.take<float>(static_cast<size_t>(p.batch) * half_rows(p.g));
  *need = c.used;
  return w;
}

// Baseline length in metres, sqrt(dx^2 + dy^2) in FP64 (host code is built
// without FMA contraction, so this rounds like the definition).
double baseline_length(const double* ant, int a, int b) {
  const double dx = ant[3 * a] - ant[3 * b], dy = ant[3 * a + 1] - ant[3 * b + 1];
  const double x2 = dx * dx, y2 = dy * dy;
  return std::sqrt(x2 + y2);
}

// Centre cell of a rounded position p (1/Q cells): p / Q rounded half away from zero.
long long centre_cell_host(long long p) {
  const long long c = (std::llabs(p) + kQ / 2) / kQ;
  return p < 0 ? -c : c;
}

// Host: which baselines can touch which warp tile in some channel of the call.
// The channel scales s_nu Q are computed exactly as the device computes them
// (k_chan_scale), and p = rint(dx s) is monotone in s, so the centre cells of
// every channel lie between those at the smallest and the largest scale.
void build_entries(const ImgPlan& p, int n_ant, const double* ant, const double* freq, int n_chan,
                   double cell, double uv_min, double uv_max, std::vector<GridEntry>& listed,
                   std::vector<int>& idx, std::vector<int>& off, long long* spread) {
  const double du = 1.0 / (static_cast<double>(p.g) * cell);
  double s_lo = HUGE_VAL, s_hi = -HUGE_VAL, fmin = freq[0], fmax = freq[0];
  for (int f = 0; f < n_chan; ++f) {
    const double sq = (freq[f] / (kCLight * du)) * static_cast<double>(kQ);
    s_lo = std::min(s_lo, sq);
    s_hi = std::max(s_hi, sq);
    fmin = std::min(fmin, freq[f]);
    fmax = std::max(fmax, freq[f]);
  }
  const bool uv_cut = uv_min > 0.0 || std::isfinite(uv_max);
  const double w_lo = fmin / kCLight, w_hi = fmax / kCLight;                  // wavelengths per metre
  const long long cmax = p.g / 2 - kHalfSup - 1;
  const int ntu = n_tiles_u(p.g), nt = n_tiles(p.g);
  std::vector<std::vector<int>> tiles(nt);
  // the centre cells over the call's channels; *spread: the most any listed
  // footprint moves across them
  *spread = 0;
  long long move = 0;
  auto cells = [&](double d, long long& lo, long long& hi) {
    const long long a = centre_cell_host(std::llrint(d * s_lo)), b = centre_cell_host(std::llrint(d * s_hi));
    lo = std::max(std::min(a, b), -cmax);
    hi = std::min(std::max(a, b), cmax);
    move = std::max(move, a > b ? a - b : b - a);
    return lo <= hi;
  };
  listed.clear();
  long long cross = 0;
  for (int a = 0; a < n_ant; ++a)
    for (int b = a + 1; b < n_ant; ++b, ++cross) {
      const double dx = ant[3 * a] - ant[3 * b], dy = ant[3 * a + 1] - ant[3 * b + 1];
      long long u0, u1, v0, v1;
      move = 0;
      if (!cells(dx, u0, u1) || !cells(dy, v0, v1)) continue;       // never on the grid
      // uv range: decided here when every channel of the call agrees (with a
      // relative margin), per channel on the device otherwise
      bool check = false;
      if (uv_cut) {
        const double L = baseline_length(ant, a, b);
        const double l0 = L * w_lo, l1 = L * w_hi, eps = 1e-9;
        if (l1 < uv_min * (1.0 - eps) || l0 >= uv_max * (1.0 + eps)) continue;      // always outside
        check = !(l0 >= uv_min * (1.0 + eps) && l1 < uv_max * (1.0 - eps));       // not always inside
      }
      GridEntry e;
      e.bl = static_cast<int>(a * static_cast<long long>(n_ant) - static_cast<long long>(a) * (a - 1) / 2 + (b - a));
      e.cross = static_cast<int>(cross);
      e.a = a;
      e.bf = b | (check ? kCheckUv : 0);
      e.dxh = static_cast<float>(dx);
      e.dxl = static_cast<float>(dx - static_cast<double>(e.dxh));
      e.dyh = static_cast<float>(dy);
      e.dyl = static_cast<float>(dy - static_cast<double>(e.dyh));
      const int li = static_cast<int>(listed.size());
      listed.push_back(e);
      *spread = std::max(*spread, move);
      // footprint rows / columns over the call (centre +- 3 cells), of the
      // record and of its mirror, within the gridded rows G/2 .. G-1
      auto add = [&](long long vl, long long vh, long long ul, long long uh, int flag) {
        const int r_lo = static_cast<int>(std::max<long long>(p.g / 2, p.g / 2 + vl - kHalfSup));
        const int r_hi = static_cast<int>(p.g / 2 + vh + kHalfSup);
        if (r_hi < r_lo) return;
        const int c_lo = static_cast<int>(p.g / 2 + ul - kHalfSup), c_hi = static_cast<int>(p.g / 2 + uh + kHalfSup);
        for (int tv = (r_lo - p.g / 2) / kTileV; tv <= (r_hi - p.g / 2) / kTileV; ++tv)
          for (int tu = c_lo / kTileU; tu <= c_hi / kTileU; ++tu) tiles[tv * ntu + tu].push_back(li | flag);
      };
      add(v0, v1, u0, u1, 0);
      add(-v1, -v0, -u1, -u0, kMirror);
    }
  idx.clear();
  off.assign(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    off[t] = static_cast<int>(idx.size());
    idx.insert(idx.end(), tiles[t].begin(), tiles[t].end());
  }
  off[nt] = static_cast<int>(idx.size());
}

template <int L, int S>
int launch_batch(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
                 int nb, float* img, cudaStream_t st) {
  constexpr int G = 1 << L;
  constexpr int LDP = band_pitch(G);
  {
    // calibration corrections or a uv range select the variant that applies them
    const bool cal = o.gains != nullptr || o.uv_min > 0.0 || std::isfinite(o.uv_max);
    const int n_groups = (nb + kLanes - 1) / kLanes;
    if (w.n_listed > 0) {
      dim3 grid((w.n_listed + kPrepBl - 1) / kPrepBl, n_groups);
      OVRO_PROF("k_grid_prep", st);
      auto prep = cal ? (w.bases ? k_grid_prep<L, true, true> : k_grid_prep<L, true, false>)
                      : (w.bases ? k_grid_prep<L, false, true> : k_grid_prep<L, false, false>);
      prep<<<grid, 256, 0, st>>>(w.listed, w.n_listed, vis, n_bl, w.base, w.cs, ch0, nb, w.kept, w.prep, o);
      OVRO_LAUNCH_CHECK();
    }
    auto tiles = w.bases ? k_grid_tiles<L, true> : k_grid_tiles<L, false>;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kTileSmem)));
    const long long items = static_cast<long long>(n_groups) * n_tiles(G);
    const long long ctas = std::min<long long>(num_sms(), (items + kGridWarps - 1) / kGridWarps);
    OVRO_PROF("k_grid_tiles", st);
    tiles<<<static_cast<unsigned>(ctas), kGridWarps * 32, kTileSmem, st>>>(
        w.tile_idx, w.tile_off, w.tile_order, w.prep, w.n_listed, w.tabx, nb, w.grid);
    OVRO_LAUNCH_CHECK();
  }
  {
    const size_t sm = static_cast<size_t>(p.band_h) * LDP * sizeof(float2) + G * sizeof(float2);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<L, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm)));
    const int threads = p.band_h * G / 16;
    dim3 grid(half_rows(G) / p.band_h, nb);
    OVRO_PROF("k_fft_rows", st);
    k_fft_rows<L, S><<<grid, threads, sm, st>>>(w.grid, w.tw, p.n, p.band_h, w.h, w.hs);
    OVRO_LAUNCH_CHECK();
  }
  {
    const size_t sm = static_cast<size_t>(p.cols_per_cta / 2) * LDP * sizeof(float2) + G * sizeof(float2);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<L, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm)));
    const int threads = p.cols_per_cta * G / 32;
    dim3 grid(p.n / p.cols_per_cta, nb);
    OVRO_PROF("k_fft_cols", st);
    k_fft_cols<L, S><<<grid, threads, sm, st>>>(w.h, w.hs, p.n, p.cols_per_cta, ch0, w.tw, w.inv_corr, w.mask,
                                                w.kept, img);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

template <int L>
int launch_storage(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
                   int nb, float* img, cudaStream_t st) {
  switch (p.storage) {
    case kStoreF32: return launch_batch<L, kStoreF32>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case kStoreBF16: return launch_batch<L, kStoreBF16>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case kStoreF16: return launch_batch<L, kStoreF16>(p, w, o, vis, n_bl, ch0, nb, img, st);
    default: return OVRO_ERR_INVALID_ARG;
  }
}

int run_batch(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
              int nb, float* img, cudaStream_t st) {
  switch (p.log2g) {
    case 5: return launch_storage<5>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 6: return launch_storage<6>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 7: return launch_storage<7>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 8: return launch_storage<8>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 9: return launch_storage<9>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 10: return launch_storage<10>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 11: return launch_storage<11>(p, w, o, vis, n_bl, ch0, nb, img, st);
    default: return OVRO_ERR_UNSUPPORTED;
  }
}

int upload_common(const ImgPlan& p, ImgWs& w, int n_ant, const double* h_ant,
                  const double* h_freq, int n_chan, double cell, cudaStream_t st,
                  double uv_min = 0.0, double uv_max = HUGE_VAL) {
  const KernelTables& kt = kernel_tables();
  std::vector<double> corr;
  grid_correction(p.n, p.g, corr);
  std::vector<float> inv(p.n);
  for (int i = 0; i < p.n; ++i) inv[i] = static_cast<float>(1.0 / corr[i]);
  std::vector<GridEntry> listed;
  std::vector<int> idx, off;
  long long spread = 0;
  build_entries(p, n_ant, h_ant, h_freq, n_chan, cell, uv_min, uv_max, listed, idx, off, &spread);
  if (static_cast<long long>(idx.size()) > entry_capacity(p)) return OVRO_ERR_CAPACITY;
  w.n_listed = static_cast<int>(listed.size());
  // one cell of slack for a host rounding of u Q that differs from the exact one
  w.bases = spread + 1 <= kTabMargin;
  std::vector<double> blen(p.n_cross > 0 ? p.n_cross : 1, 0.0);
  {
    long long x = 0;
    for (int a = 0; a < n_ant; ++a)
      for (int b = a + 1; b < n_ant; ++b) blen[x++] = baseline_length(h_ant, a, b);
  }
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.blen, blen.data(), blen.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tab, kt.table32.data(), kTabLen * sizeof(float),
                                cudaMemcpyHostToDevice, st));
  std::vector<float> tabx(kTabXLen, 0.0f);
  for (int d = -kHalfSup; d <= kHalfSup; ++d)
    for (int off = -kQ / 2; off <= kQ / 2; ++off)
      tabx[(d + kTabD) * kTabStride + kQ / 2 - off] = kt.table32[kHalfTab + d * kQ - off];
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tabx, tabx.data(), kTabXLen * sizeof(float), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.inv_corr, inv.data(), p.n * sizeof(float), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.ant, h_ant, static_cast<size_t>(n_ant) * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.freq, h_freq, static_cast<size_t>(n_chan) * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tile_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<int> order(off.size() - 1);
  for (size_t t = 0; t < order.size(); ++t) order[t] = static_cast<int>(t);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tile_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!listed.empty())
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.listed, listed.data(), listed.size() * sizeof(GridEntry),
                                  cudaMemcpyHostToDevice, st));
  if (!idx.empty())
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.tile_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  // host->device copies from pageable memory are staged before cudaMemcpyAsync
  // returns, so the temporaries above may go out of scope
  k_twiddle_img<<<(p.g + 255) / 256, 256, 0, st>>>(w.tw, p.g);
  OVRO_LAUNCH_CHECK();
  k_mask<<<(p.n * p.n + 255) / 256, 256, 0, st>>>(p.n, cell, w.mask);
  OVRO_LAUNCH_CHECK();
  if (p.n_cross > 0) {
    dim3 g((n_ant + 127) / 128, n_ant);
    k_baselines<<<g, 128, 0, st>>>(w.ant, n_ant, w.base);
    OVRO_LAUNCH_CHECK();
  }
  k_chan_scale<<<(n_chan + 255) / 256, 256, 0, st>>>(w.freq, n_chan, p.g, cell, w.cs);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

int validate(int n_ant, const double* h_ant, const double* h_freq, int n_chan, int n, double cell) {
  if (!h_ant || !h_freq || n_ant <= 0 || n_chan <= 0) return OVRO_ERR_INVALID_ARG;
  if (!(cell > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (!is_pow2(n) || n < 16 || n > 1024) return OVRO_ERR_UNSUPPORTED;
  if (n_ant > 4096) return OVRO_ERR_UNSUPPORTED;
  return OVRO_OK;
}

}  // namespace

struct GridCtx {
  ImgPlan p;
  ImgWs w;
  int n_ant = 0, n_chan = 0;
  double cell = 0.0;
  const float2* gains = nullptr;      // calibration corrections [n_chan][2 n_ant]
  double uv_min = 0.0, uv_max = HUGE_VAL;
};

size_t grid_ctx_workspace(int n_ant, int n_chan, int image_size, int storage) {
  if (n_ant <= 0 || n_chan <= 0 || !is_pow2(image_size) || image_size < 16 || image_size > 1024) return 0;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16) return 0;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size, storage);
  size_t need = 0;
  carve_img(nullptr, 0, p, n_ant, n_chan, &need);
  return need;
}

int grid_ctx_init(GridCtx** out, int n_ant, int n_chan, int image_size, double cell, int storage, void* d_ws,
                  size_t ws_bytes, const void* d_gains, double uv_min, double uv_max) {
  if (!out) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_ant <= 0 || n_chan <= 0 || !(cell > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16)
    return OVRO_ERR_INVALID_ARG;
  if (!is_pow2(image_size) || image_size < 16 || image_size > 1024 || n_ant > 4096) return OVRO_ERR_UNSUPPORTED;
  GridCtx* g = new GridCtx;
  g->p = make_plan(n_ant, n_chan, image_size, storage);
  size_t need = 0;
  g->w = carve_img(d_ws, ws_bytes, g->p, n_ant, n_chan, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) {
    delete g;
    return e;
  }
  g->n_ant = n_ant;
  g->n_chan = n_chan;
  g->cell = cell;
  g->gains = static_cast<const float2*>(d_gains);
  g->uv_min = uv_min;
  g->uv_max = uv_max;
  *out = g;
  return OVRO_OK;
}

int grid_ctx_upload(GridCtx* g, const double* h_ant_enu_m, const double* h_chan_freq_hz, cudaStream_t st) {
  if (!g) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(g->n_ant, h_ant_enu_m, h_chan_freq_hz, g->n_chan, g->p.n, g->cell)) return e;
  return upload_common(g->p, g->w, g->n_ant, h_ant_enu_m, h_chan_freq_hz, g->n_chan, g->cell, st, g->uv_min,
                       g->uv_max);
}

int grid_ctx_enqueue(GridCtx* g, const int32_t* d_vis, float* d_img, int32_t* d_counts_or_null, cudaStream_t st) {
  if (!g || !d_vis || !d_img) return OVRO_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0) return OVRO_ERR_INVALID_ARG;
  const ImgPlan& p = g->p;
  const long long n_bl = static_cast<long long>(g->n_ant) * (g->n_ant + 1) / 2;
  GridOpts o;
  o.gains = g->gains;
  o.n_input = 2 * g->n_ant;
  o.blen = g->w.blen;
  o.uv_min = g->uv_min;
  o.uv_max = g->uv_max;
  // channels per launch pair (at most the workspace's batch): every choice
  // gives the same images and counts
  auto all = [&](int batch) -> int {
    OVRO_CUDA_TRY(cudaMemsetAsync(g->w.kept, 0, g->n_chan * sizeof(int), st));
    for (int ch0 = 0; ch0 < g->n_chan; ch0 += batch) {
      const int nb = g->n_chan - ch0 < batch ? g->n_chan - ch0 : batch;
      if (int e = run_batch(p, g->w, o, d_vis, n_bl, ch0, nb, d_img, st)) return e;
    }
    return OVRO_OK;
  };
  const std::string key = tune_key("grid_batch", {g->n_ant, g->n_chan, p.n, p.storage});
  int batch = std::min(p.batch, std::max(1, tuned(key, p.batch)));
  if (tuning(st)) {
    std::vector<int> cands;
    // whole groups of 32 channels (or the call's channels, if fewer)
    for (int b = p.batch; cands.size() < 4; b /= 2) {
      const int c = b >= kLanes ? b / kLanes * kLanes : b;
      if (cands.empty() || c < cands.back()) cands.push_back(c);
      if (c <= kLanes) break;
    }
    if (int e = tune_pick(key, cands, all, st, &batch)) return e;
  }
  if (int e = all(batch)) return e;
  if (d_counts_or_null) {
    k_counts_out<<<(g->n_chan + 255) / 256, 256, 0, st>>>(g->w.kept, g->n_chan, d_counts_or_null);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

int grid_ctx_gridded(GridCtx* g, long long* total, cudaStream_t st) {
  if (!g || !total) return OVRO_ERR_INVALID_ARG;
  std::vector<int> k(g->n_chan);
  OVRO_CUDA_TRY(cudaMemcpyAsync(k.data(), g->w.kept, g->n_chan * sizeof(int), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  long long s = 0;
  for (int v : k) s += v;
  *total = s;
  return OVRO_OK;
}

void grid_ctx_free(GridCtx* g) { delete g; }

}  // namespace ovro

extern "C" {

size_t ovro_grid_image_workspace_size(int n_ant, int n_chan, int image_size, int storage) {
  return ovro::grid_ctx_workspace(n_ant, n_chan, image_size, storage);
}

int ovro_grid_image(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m,
                    const double* h_chan_freq_hz, int n_chan, int image_size, double cell_dircos,
                    int storage, float* d_img, int32_t* d_n_gridded_or_null, void* d_ws,
                    size_t ws_bytes, void* stream) {
  ovro_grid_options o;
  o.storage = storage;
  o.d_gains_or_null = nullptr;
  o.uv_min_lambda = 0.0;
  o.uv_max_lambda = 0.0;
  return ovro_grid_image_ex(d_vis, n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos, &o, d_img,
                            d_n_gridded_or_null, d_ws, ws_bytes, stream);
}

int ovro_grid_image_ex(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m, const double* h_chan_freq_hz,
                       int n_chan, int image_size, double cell_dircos, const ovro_grid_options* opt, float* d_img,
                       int32_t* d_n_gridded_or_null, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_vis || !d_img || !opt) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos)) return e;
  const int storage = opt->storage;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16)
    return OVRO_ERR_INVALID_ARG;
  if (!(opt->uv_min_lambda >= 0.0) || std::isnan(opt->uv_max_lambda)) return OVRO_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0) return OVRO_ERR_INVALID_ARG;
  if (opt->d_gains_or_null && reinterpret_cast<uintptr_t>(opt->d_gains_or_null) % 8 != 0) return OVRO_ERR_INVALID_ARG;
  const double uv_max = opt->uv_max_lambda > 0.0 ? opt->uv_max_lambda : HUGE_VAL;
  GridCtx* g = nullptr;
  if (int e = grid_ctx_init(&g, n_ant, n_chan, image_size, cell_dircos, storage, d_ws, ws_bytes,
                            opt->d_gains_or_null, opt->uv_min_lambda, uv_max))
    return e;
  cudaStream_t st = as_stream(stream);
  int e = grid_ctx_upload(g, h_ant_enu_m, h_chan_freq_hz, st);
  if (!e) e = grid_ctx_enqueue(g, d_vis, d_img, d_n_gridded_or_null, st);
  grid_ctx_free(g);
  return e;
}

// a5 alone: rounded uv positions p = rint(u Q), Q = 1024, of every cross
// baseline (a < b, row-major) in every channel: int32 [n_chan][n_cross]
// (saturated at +-2^30).  Workspace as for ovro_grid_image.
int ovro_uvw(const double* h_ant_enu_m, int n_ant, const double* h_chan_freq_hz, int n_chan,
             int image_size, double cell_dircos, int32_t* d_pu, int32_t* d_pv, void* d_ws,
             size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_pu || !d_pv) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos)) return e;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size, OVRO_STORE_FP32);
  size_t need = 0;
  ImgWs w = carve_img(d_ws, ws_bytes, p, n_ant, n_chan, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  if (int e = upload_common(p, w, n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, cell_dircos, st)) return e;
  if (p.n_cross == 0) return OVRO_OK;
  dim3 g(static_cast<unsigned>((p.n_cross + 255) / 256), n_chan);
  k_uvw<<<g, 256, 0, st>>>(w.base, static_cast<int>(p.n_cross), w.cs, d_pu, d_pv);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

}  // extern "C"
