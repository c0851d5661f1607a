// a4: X-engine.  Section 2.1 of the paper: per fine channel, every antenna pair
// and polarisation product, integrated over the K spectra of the integration:
//     V_ij = sum_s q_i(s) conj(q_j(s)),  i <= j (autos kept).
//
// Two exact paths over the same int8 input [chan][K][n_input][2]:
//
//  * k_xeng_simt: plain FP32 SIMT accumulation, 2x2 antennas x 2x2 pols per
//    thread (exact: every partial sum is an integer below 2^24).
//
//  * k_xeng_tc: 5th-generation tensor cores.  sm_103a has no integer MMA
//    (tcgen05 .kind::i8 is rejected by ptxas for this target), so the int8
//    values are carried exactly in FP16 operands and accumulated in FP32 in
//    tensor memory; every int8 value has |q| <= 128, so each spectrum adds at
//    most 2 * 128^2 = 2^15 to a sum and every partial sum stays an integer
//    below 2^24 for K <= 511: the result is exact.  The Hermitian product becomes
//    one real GEMM: A row i = X_i = (re_i(s), im_i(s))_s, B rows 2j, 2j+1 =
//    X_j and Z_j = (-im_j(s), re_j(s))_s, so D[i][2j] = Re V_ij and
//    D[i][2j+1] = Im V_ij land as adjacent TMEM columns.  One CTA per SM pair
//    slot runs persistently over (channel, 128x128-input tile) work items of
//    the upper triangle; one thread issues tcgen05.mma (M=128, N=256, K=16
//    steps) from no-swizzle K-major shared-memory operands, the MMA completion
//    is signalled through an mbarrier by tcgen05.commit, and all four warps
//    drain their TMEM lane quarter with tcgen05.ld and store int32 records.
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "stages.h"
#include "tune.h"

namespace ovro {
namespace {

__device__ int g_xeng_status;   // nonzero: a bounded wait timed out

__host__ __device__ __forceinline__ long long bl_index(int a, int b, int n) {
  return static_cast<long long>(a) * n - static_cast<long long>(a) * (a - 1) / 2 + (b - a);
}

// ------------------------------------------------------------------ SIMT FP32
constexpr int kSimtTile = 64;      // inputs per tile side (32 antennas)
constexpr int kSimtKc = 32;        // spectra per shared-memory chunk

__global__ void __launch_bounds__(256)
k_xeng_simt(const int8_t* __restrict__ q, int n_ant, int n_spec, int n_tiles,
            int32_t* __restrict__ vis) {
  __shared__ float2 sa[kSimtKc][kSimtTile];
  __shared__ float2 sb[kSimtKc][kSimtTile];
  const int n_input = 2 * n_ant;
  // tile pair (I <= J) from blockIdx.x
  int p = blockIdx.x, I = 0;
  while (p >= n_tiles - I) { p -= n_tiles - I; ++I; }
  const int J = I + p;
  const int ch = blockIdx.y;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int8_t* qc = q + static_cast<long long>(ch) * n_spec * n_input * 2;
  float acc[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c][0] = acc[r][c][1] = 0.f;

  for (int s0 = 0; s0 < n_spec; s0 += kSimtKc) {
    const int ns = min(kSimtKc, n_spec - s0);
    for (int idx = threadIdx.x; idx < kSimtKc * kSimtTile; idx += blockDim.x) {
      const int s = idx / kSimtTile, t = idx - s * kSimtTile;
      float2 va = make_float2(0.f, 0.f), vb = va;
      if (s < ns) {
        const int ia = I * kSimtTile + t, ib = J * kSimtTile + t;
        const char2* row = reinterpret_cast<const char2*>(qc + static_cast<long long>(s0 + s) * n_input * 2);
        if (ia < n_input) { char2 x = row[ia]; va = make_float2(x.x, x.y); }
        if (ib < n_input) { char2 x = row[ib]; vb = make_float2(x.x, x.y); }
      }
      sa[s][t] = va;
      sb[s][t] = vb;
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      float2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sa[s][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = sb[s][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // a * conj(b)
          acc[r][c][0] = fmaf(a[r].x, b[c].x, fmaf(a[r].y, b[c].y, acc[r][c][0]));
          acc[r][c][1] = fmaf(a[r].y, b[c].x, fmaf(-a[r].x, b[c].y, acc[r][c][1]));
        }
    }
    __syncthreads();
  }
  const long long n_bl = static_cast<long long>(n_ant) * (n_ant + 1) / 2;
  int4* out = reinterpret_cast<int4*>(vis + static_cast<long long>(ch) * n_bl * 8);
#pragma unroll
  for (int ar = 0; ar < 2; ++ar)
#pragma unroll
    for (int bc = 0; bc < 2; ++bc) {
      const int a = (I * kSimtTile + ty * 4) / 2 + ar;
      const int b = (J * kSimtTile + tx * 4) / 2 + bc;
      if (a >= n_ant || b >= n_ant || a > b) continue;
      const long long bl = bl_index(a, b, n_ant);
      // pol products p = 2 pa + pb; rows 2ar + pa, cols 2bc + pb
      int4 lo, hi;
      lo.x = __float2int_rn(acc[2 * ar][2 * bc][0]);      lo.y = __float2int_rn(acc[2 * ar][2 * bc][1]);
      lo.z = __float2int_rn(acc[2 * ar][2 * bc + 1][0]);  lo.w = __float2int_rn(acc[2 * ar][2 * bc + 1][1]);
      hi.x = __float2int_rn(acc[2 * ar + 1][2 * bc][0]);  hi.y = __float2int_rn(acc[2 * ar + 1][2 * bc][1]);
      hi.z = __float2int_rn(acc[2 * ar + 1][2 * bc + 1][0]); hi.w = __float2int_rn(acc[2 * ar + 1][2 * bc + 1][1]);
      out[bl * 2] = lo;
      out[bl * 2 + 1] = hi;
    }
}

// --------------------------------------------------------------- tcgen05 path
constexpr int kTcM = 128;                 // A rows (inputs) per tile
constexpr int kTcInputsN = 128;           // column inputs per tile -> N = 256
constexpr int kTcN = 2 * kTcInputsN;
constexpr int kTcKc = 64;                 // FP16 K elements per chunk (32 spectra)
constexpr int kTcSpecPerChunk = kTcKc / 2;
constexpr int kTmemCols = 256;
constexpr int kTcThreads = 128;
constexpr uint32_t kLBO = 128;            // bytes between K-adjacent core matrices
constexpr uint32_t kSBO = (kTcKc / 8) * 128;  // bytes between 8-row groups
constexpr int kTcASmem = kTcM * kTcKc * 2;    // 16 KB
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle K-major operand: element (row, k) of a [rows][kTcKc] FP16 tile
__device__ __forceinline__ uint32_t op_offset(int row, int k) {
  return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(kLBO >> 4) << 16;
  d |= static_cast<uint64_t>(kSBO >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;          // descriptor version for tcgen05
  return d;                                     // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = F16, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) |
                            (static_cast<uint32_t>(kTcN >> 3) << 17) |
                            (static_cast<uint32_t>(kTcM >> 4) << 24);

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

__global__ void __launch_bounds__(kTcThreads)
k_xeng_tc(const int8_t* __restrict__ q, int n_ant, int n_spec, int n_tiles, int n_pairs,
          long long n_items, int32_t* __restrict__ vis) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                       // 16 KB
  unsigned char* sB = smem + kTcASmem;            // 32 KB
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_input = 2 * n_ant;
  const long long n_bl = static_cast<long long>(n_ant) * (n_ant + 1) / 2;
  const uint32_t mbar_a = smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  uint32_t phase = 0;

  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int ch = static_cast<int>(item / n_pairs);
    int p = static_cast<int>(item - static_cast<long long>(ch) * n_pairs), I = 0;
    while (p >= n_tiles - I) { p -= n_tiles - I; ++I; }
    const int J = I + p;
    const int8_t* qc = q + static_cast<long long>(ch) * n_spec * n_input * 2;

    // ---- operands: A row t = X_{I*128+t}; B rows 2t, 2t+1 = X_j, Z_j, j = J*128+t.
    // A chunk's 2 x 32 int8 pairs per thread are read with one round trip, and
    // the next chunk's reads are issued while this chunk's MMAs run.
    const int ia = I * kTcM + tid;
    const int ib = J * kTcInputsN + tid;
    uint32_t va[kTcSpecPerChunk], vb[kTcSpecPerChunk];   // (re, im) int8 pairs, 16 bits used
    auto read_chunk = [&](int s0) {
#pragma unroll
      for (int ss = 0; ss < kTcSpecPerChunk; ++ss) {
        const int s = s0 + ss;
        const uint16_t* row = reinterpret_cast<const uint16_t*>(qc + static_cast<long long>(s) * n_input * 2);
        va[ss] = (s < n_spec && ia < n_input) ? __ldg(row + ia) : 0u;
        vb[ss] = (s < n_spec && ib < n_input) ? __ldg(row + ib) : 0u;
      }
    };
    read_chunk(0);
    for (int s0 = 0; s0 < n_spec; s0 += kTcSpecPerChunk) {
#pragma unroll
      for (int ss = 0; ss < kTcSpecPerChunk; ++ss) {
        const short ar = static_cast<signed char>(va[ss] & 0xffu), ai = static_cast<signed char>(va[ss] >> 8);
        const short br = static_cast<signed char>(vb[ss] & 0xffu), bi = static_cast<signed char>(vb[ss] >> 8);
        const __half2 ha = __halves2half2(__short2half_rn(ar), __short2half_rn(ai));
        const __half2 hx = __halves2half2(__short2half_rn(br), __short2half_rn(bi));
        const __half2 hz = __halves2half2(__short2half_rn(static_cast<short>(-bi)), __short2half_rn(br));
        *reinterpret_cast<__half2*>(sA + op_offset(tid, 2 * ss)) = ha;
        *reinterpret_cast<__half2*>(sB + op_offset(2 * tid, 2 * ss)) = hx;
        *reinterpret_cast<__half2*>(sB + op_offset(2 * tid + 1, 2 * ss)) = hz;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (s0 + kTcSpecPerChunk < n_spec) read_chunk(s0 + kTcSpecPerChunk);
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
        for (int kk = 0; kk < kTcKc / 16; ++kk) {
          const uint64_t ad = make_sdesc(a0 + kk * 2 * kLBO);
          const uint64_t bd = make_sdesc(b0 + kk * 2 * kLBO);
          const uint32_t acc = (s0 > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
              :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mbar_a) : "memory");
      }
      // all threads wait for the MMAs (operand smem is rewritten next chunk)
      if (!mbar_wait(mbar_a, phase)) {
        atomicExch(&g_xeng_status, 1);
        abort_sh = 1;
      }
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (abort_sh) break;
    }
    if (abort_sh) break;

    // ---- epilogue: warp w drains TMEM lanes 32w..32w+31 (rows = inputs)
    const int gi = I * kTcM + warp * 32 + lane;
    const int a = gi >> 1, pa = gi & 1;
    int4* out = reinterpret_cast<int4*>(vis + static_cast<long long>(ch) * n_bl * 8);
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
            "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
            "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (a < n_ant) {
        // columns c0 .. c0+31 = column inputs j0 .. j0+15, (re, im) each
        const int j0 = J * kTcInputsN + c0 / 2;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) {
          const int b = (j0 >> 1) + bb;
          if (b >= n_ant || b < a) continue;
          int4 v;
          v.x = __float2int_rn(__uint_as_float(r[4 * bb + 0]));
          v.y = __float2int_rn(__uint_as_float(r[4 * bb + 1]));
          v.z = __float2int_rn(__uint_as_float(r[4 * bb + 2]));
          v.w = __float2int_rn(__uint_as_float(r[4 * bb + 3]));
          __stcs(out + bl_index(a, b, n_ant) * 2 + pa, v);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------- tcgen05 path, channel-major
// For arrays of at most 768 inputs and at most 32 spectra per integration, a
// persistent CTA per SM takes whole channels: the channel's int8 spectra are
// converted once into FP16 operand tiles in shared memory -- per tile of 128
// inputs, rows 0..127 hold X = (re, im) per spectrum and rows 128..255 hold
// Z = (-im, re) -- so tile J as a 256-row B operand yields Re in TMEM columns
// 0..127 and Im in 128..255 against A = X rows of tile I.  Two 256-column
// accumulators alternate: the MMAs of tile pair t+1 run while the epilogue
// drains pair t.  The next channel's spectra are prefetched into L2.
constexpr int kV2Threads = 256;
constexpr int kV2MaxTiles = 6;
constexpr int kV2TileBytes = 2 * kTcM * kTcKc * 2;        // 32 KB: X rows then Z rows
constexpr uint32_t kV2TmemCols = 512;

__global__ void __launch_bounds__(kV2Threads, 1)
k_xeng_tc2(const int8_t* __restrict__ q, int n_ant, int n_spec, int n_tiles, int n_chan, int prefetch,
           int32_t* __restrict__ vis) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_input = 2 * n_ant;
  const long long n_bl = static_cast<long long>(n_ant) * (n_ant + 1) / 2;
  const int n_pairs = n_tiles * (n_tiles + 1) / 2;
  const int NI = n_tiles * kTcM;
  const long long chan_bytes = static_cast<long long>(n_spec) * n_input * 2;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(kV2TmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  uint32_t par[2] = {0u, 0u};          // next phase parity to wait for, per accumulator
  int inflight[2] = {0, 0};            // a commit on that accumulator's barrier not yet waited for

  // tile pair t -> (I, J), I <= J, row-major over the upper triangle
  auto pair_of = [&](int t, int& I, int& J) {
    I = 0;
    while (t >= n_tiles - I) { t -= n_tiles - I; ++I; }
    J = I + t;
  };
  auto issue = [&](int t) {
    inflight[t & 1] = 1;
    if (tid != 0) return;
    int I, J;
    pair_of(t, I, J);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t a0 = smem_u32(smem + I * kV2TileBytes), b0 = smem_u32(smem + J * kV2TileBytes);
    const uint32_t d = tmem + static_cast<uint32_t>((t & 1) * 256);
#pragma unroll
    for (int kk = 0; kk < kTcKc / 16; ++kk) {
      const uint64_t ad = make_sdesc(a0 + kk * 2 * kLBO);
      const uint64_t bd = make_sdesc(b0 + kk * 2 * kLBO);
      const uint32_t acc = kk > 0 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
          :: "r"(d), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&mbar[t & 1])) : "memory");
  };

  for (int ch = blockIdx.x; ch < n_chan; ch += gridDim.x) {
    const int8_t* qc = q + static_cast<long long>(ch) * chan_bytes;
    if (prefetch && tid == 0 && ch + static_cast<int>(gridDim.x) < n_chan) {
      const int8_t* nx = qc + static_cast<long long>(gridDim.x) * chan_bytes;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                   :: "l"(nx), "r"(static_cast<uint32_t>(chan_bytes)) : "memory");
    }
    // ---- operands: task = (spectrum group of 4, input), inputs fastest
    for (int task = tid; task < NI * (kTcKc / 8); task += kV2Threads) {
      const int i = task % NI, sg = task / NI;
      uint32_t xw[4], zw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int sp = 4 * sg + j;
        char2 v = make_char2(0, 0);
        if (sp < n_spec && i < n_input)
          v = reinterpret_cast<const char2*>(qc + static_cast<long long>(sp) * n_input * 2)[i];
        const __half2 hx = __halves2half2(__short2half_rn(v.x), __short2half_rn(v.y));
        const __half2 hz = __halves2half2(__short2half_rn(static_cast<short>(-v.y)), __short2half_rn(v.x));
        xw[j] = *reinterpret_cast<const uint32_t*>(&hx);
        zw[j] = *reinterpret_cast<const uint32_t*>(&hz);
      }
      const int t = i / kTcM, r = i - t * kTcM;
      unsigned char* base = smem + t * kV2TileBytes + op_offset(r, 8 * sg);
      *reinterpret_cast<uint4*>(base) = make_uint4(xw[0], xw[1], xw[2], xw[3]);
      *reinterpret_cast<uint4*>(base + 16 * kSBO) = make_uint4(zw[0], zw[1], zw[2], zw[3]);   // rows 128 + r
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    issue(0);
    for (int t = 0; t < n_pairs; ++t) {
      if (t + 1 < n_pairs) issue(t + 1);        // its accumulator was drained in step t - 1
      const bool ok = mbar_wait(smem_u32(&mbar[t & 1]), par[t & 1]);
      if (ok) {
        par[t & 1] ^= 1u;
        inflight[t & 1] = 0;
      } else {
        atomicExch(&g_xeng_status, 1);
        abort_sh = 1;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
        int I, J;
        pair_of(t, I, J);
        const int q4 = warp & 3, wg = warp >> 2;
        const int gi = I * kTcM + q4 * 32 + lane;
        const int a = gi >> 1, pa = gi & 1;
        int4* out = reinterpret_cast<int4*>(vis + static_cast<long long>(ch) * n_bl * 8);
        const uint32_t cb = static_cast<uint32_t>((t & 1) * 256);
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
          const int cin0 = wg * 64 + hh * 32;     // column inputs cin0 .. cin0 + 31
          uint32_t re[32], im[32];
          const uint32_t tl = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + cb + cin0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
              "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
                "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]),
                "=r"(re[13]), "=r"(re[14]), "=r"(re[15]), "=r"(re[16]), "=r"(re[17]), "=r"(re[18]),
                "=r"(re[19]), "=r"(re[20]), "=r"(re[21]), "=r"(re[22]), "=r"(re[23]), "=r"(re[24]),
                "=r"(re[25]), "=r"(re[26]), "=r"(re[27]), "=r"(re[28]), "=r"(re[29]), "=r"(re[30]),
                "=r"(re[31])
              : "r"(tl));
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
              "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
                "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]),
                "=r"(im[13]), "=r"(im[14]), "=r"(im[15]), "=r"(im[16]), "=r"(im[17]), "=r"(im[18]),
                "=r"(im[19]), "=r"(im[20]), "=r"(im[21]), "=r"(im[22]), "=r"(im[23]), "=r"(im[24]),
                "=r"(im[25]), "=r"(im[26]), "=r"(im[27]), "=r"(im[28]), "=r"(im[29]), "=r"(im[30]),
                "=r"(im[31])
              : "r"(tl + 128u));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (a < n_ant) {
            const int b0 = (J * kTcInputsN + cin0) >> 1;
#pragma unroll
            for (int bb = 0; bb < 16; ++bb) {
              const int b = b0 + bb;
              if (b >= n_ant || b < a) continue;
              int4 v;
              v.x = __float2int_rn(__uint_as_float(re[2 * bb]));
              v.y = __float2int_rn(__uint_as_float(im[2 * bb]));
              v.z = __float2int_rn(__uint_as_float(re[2 * bb + 1]));
              v.w = __float2int_rn(__uint_as_float(im[2 * bb + 1]));
              __stcs(out + bl_index(a, b, n_ant) * 2 + pa, v);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (abort_sh) break;
    }
    if (abort_sh) break;
  }
  // after a timeout: wait (bounded) for the MMAs still in flight before the
  // accumulators are released
#pragma unroll
  for (int b = 0; b < 2; ++b)
    if (inflight[b]) (void)mbar_wait(smem_u32(&mbar[b]), par[b]);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kV2TmemCols) : "memory");
  }
}

}  // namespace
}  // namespace ovro

namespace ovro {

// Device address of the timeout word (per device), for stream-ordered memsets.
int* xeng_status_ptr() {
  static int* cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_xeng_status) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int*>(p);
  }
  return cache[dev];
}

int correlate_reset_status(cudaStream_t st) {
  int* p = xeng_status_ptr();
  if (!p) return OVRO_ERR_CUDA;
  OVRO_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(int), st));
  return OVRO_OK;
}

int correlate_enqueue(const int8_t* d_fine_q, int n_ant, int n_chan, int n_spec, int mode, int32_t* d_vis,
                      cudaStream_t st, bool reset_status) {
  if (!d_fine_q || !d_vis || n_ant <= 0 || n_chan <= 0 || n_spec <= 0) return OVRO_ERR_INVALID_ARG;
  if (mode != OVRO_XENG_TC && mode != OVRO_XENG_FP32) return OVRO_ERR_INVALID_ARG;
  if (n_ant > 4096) return OVRO_ERR_UNSUPPORTED;
  // any int8 input (-128 included): partial sums below 2 * 128^2 * K < 2^24
  if (2LL * 128 * 128 * n_spec >= (1LL << 24)) return OVRO_ERR_OVERFLOW;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0 || reinterpret_cast<uintptr_t>(d_fine_q) % 2 != 0)
    return OVRO_ERR_INVALID_ARG;
  const int n_input = 2 * n_ant;
  if (mode == OVRO_XENG_FP32) {
    const int n_tiles = (n_input + kSimtTile - 1) / kSimtTile;
    dim3 grid(n_tiles * (n_tiles + 1) / 2, n_chan);
    OVRO_PROF("k_xeng_simt", st);
    k_xeng_simt<<<grid, 256, 0, st>>>(d_fine_q, n_ant, n_spec, n_tiles, d_vis);
    OVRO_LAUNCH_CHECK();
    return OVRO_OK;
  }
  if (reset_status)
    if (int e = correlate_reset_status(st)) return e;
  const int n_tiles = (n_input + kTcM - 1) / kTcM;
  if (n_tiles <= kV2MaxTiles && n_spec <= kTcSpecPerChunk) {
    // channel-major kernel; at least 116 KB of shared memory keeps one CTA
    // (and so one 512-column TMEM allocation) per SM
    const int smem = std::max(n_tiles * kV2TileBytes, 116 * 1024);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_xeng_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const long long cb = static_cast<long long>(n_spec) * n_input * 2;
    const int prefetch = (cb % 16 == 0 && reinterpret_cast<uintptr_t>(d_fine_q) % 16 == 0) ? 1 : 0;
    const int grid = std::min(n_chan, num_sms());
    OVRO_PROF("k_xeng_tc", st);
    k_xeng_tc2<<<grid, kV2Threads, smem, st>>>(d_fine_q, n_ant, n_spec, n_tiles, n_chan, prefetch, d_vis);
    OVRO_LAUNCH_CHECK();
    return OVRO_OK;
  }
  const int n_pairs = n_tiles * (n_tiles + 1) / 2;
  const long long n_items = static_cast<long long>(n_pairs) * n_chan;
  // 96 KB of dynamic shared memory keeps at most two CTAs (2 x 256 TMEM columns) per SM
  const int smem = 96 * 1024;
  OVRO_CUDA_TRY(cudaFuncSetAttribute(k_xeng_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  // persistent CTAs per SM (one or two fit: 256 TMEM columns each)
  auto run = [&](int per_sm) -> int {
    long long grid = static_cast<long long>(per_sm) * num_sms();
    if (grid > n_items) grid = n_items;
    OVRO_PROF("k_xeng_tc", st);
    k_xeng_tc<<<static_cast<unsigned>(grid), kTcThreads, smem, st>>>(d_fine_q, n_ant, n_spec, n_tiles,
                                                                    n_pairs, n_items, d_vis);
    OVRO_LAUNCH_CHECK();
    return OVRO_OK;
  };
  const std::string key = tune_key("k_xeng_tc", {n_ant, n_chan, n_spec});
  int per_sm = tuned(key, 2);
  if (tuning(st))
    if (int e = tune_pick(key, {1, 2}, run, st, &per_sm)) return e;
  return run(per_sm);
}

}  // namespace ovro

extern "C" {

int ovro_correlate(const int8_t* d_fine_q, int n_ant, int n_chan, int n_spec, int mode,
                   int32_t* d_vis, void* stream) {
  return ovro::correlate_enqueue(d_fine_q, n_ant, n_chan, n_spec, mode, d_vis, ovro::as_stream(stream), true);
}

// Device status of the last tensor-core correlation (nonzero: a bounded wait timed out).
int ovro_correlate_status(void* stream) {
  int v = 0;
  cudaStream_t st = ovro::as_stream(stream);
  if (cudaMemcpyFromSymbolAsync(&v, ovro::g_xeng_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return OVRO_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return OVRO_ERR_CUDA;
  return v ? OVRO_ERR_TIMEOUT : OVRO_OK;
}

}  // extern "C"
