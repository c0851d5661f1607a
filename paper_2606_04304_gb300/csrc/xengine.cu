// a4: X-engine.  Section 2.1 of the paper: per fine channel, every antenna pair
// and polarisation product, integrated over the K spectra of the integration:
//     V_ij = sum_s q_i(s) conj(q_j(s)),  i <= j (autos kept).
//
// Two exact paths over the same int8 input [chan][K][n_input][2]:
//
//  * k_xeng_simt: plain FP32 SIMT accumulation, 2x2 antennas x 2x2 pols per
//    thread (exact: every partial sum is an integer below 2^24).
//
//  * tensor cores (5th generation).  sm_103a has no integer MMA (tcgen05
//    .kind::i8 is rejected by ptxas for this target), so the int8 values are
//    carried exactly in FP16 operands and accumulated in FP32 in tensor
//    memory; every int8 value has |q| <= 128, so each spectrum adds at most
//    2 * 128^2 = 2^15 to a sum and every partial sum stays an integer below
//    2^24 for K <= 511: the result is exact.  The Hermitian product becomes one
//    real GEMM: A row i = X_i = (re_i(s), im_i(s))_s, B rows j and 128 + j of
//    a 128-input tile = X_j and Z_j = (-im_j(s), re_j(s))_s, so D[i][j] =
//    Re V_ij and D[i][128 + j] = Im V_ij.  One thread issues tcgen05.mma
//    (M = 128, N = 256, K = 16 steps) from no-swizzle K-major shared-memory
//    operands, completions are signalled through mbarriers by tcgen05.commit,
//    and warps drain TMEM lane quarters with tcgen05.ld into int32 records.
//    k_xeng_tc2 (K <= 32, up to 768 inputs) converts a channel's spectra once
//    and runs all its tile pairs; k_xeng_tc3 streams the spectra of each tile
//    pair through shared memory with warp-specialised roles.
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

// ------------------------------------------- tcgen05 path, streamed spectra
// For more than 32 spectra (or larger arrays) the operands of a tile pair are
// streamed through shared memory in chunks of 32 spectra, with the roles of a
// CTA's warps split so that the tensor pipe never waits on the SIMT work:
//   warps 0-15 (converters): thread t owns operand rows 2 (t % 64) and
//     2 (t % 64) + 1 of the pair and eighth t / 64 of a chunk's spectra; it
//     reads its inputs' int8 spectra four chunks ahead into registers (4-byte
//     loads, 128 contiguous bytes per warp and spectrum) while converting a
//     chunk into FP16 A and [X; Z] B rows of a free stage (exactly: the byte
//     with its sign bit flipped is the low byte of the FP16 number
//     1024 + 128 + q, and one packed subtraction of 1152 leaves q; 16-byte
//     shared stores), then arrives on that stage's full barrier;
//   warp 20 lane 0 (MMA): per chunk waits for a full stage, issues the four
//     K = 16 MMAs into the item's accumulator and commits them to the stage's
//     empty barrier (and, after the item's last chunk, to the accumulator's
//     ready barrier);
//   warps 16-19 (epilogue): drain an item's accumulator (TMEM lane quarter
//     warp % 4) into int32 records and arrive on its free barrier.
// Three operand stages (48 KB each) and two 256-column accumulators, so the
// epilogue of item i runs under the MMAs of item i + 1.  Every wait is bounded
// (1 s); a timeout sets the status word and a shared abort flag that every
// role polls, and the kernel waits (bounded) for its MMAs before freeing TMEM.
constexpr int kT3Stages = 3;
constexpr int kT3StageBytes = kTcASmem + 2 * kTcASmem;     // A 16 KB + B 32 KB
constexpr int kT3ConvThreads = 512;                        // warps 0-15
constexpr int kT3Threads = 672;                            // 21 warps
constexpr int kT3MmaWarp = 20;
constexpr int kT3SpecPerThread = kTcSpecPerChunk / (kT3ConvThreads / 64);   // a converter's eighth of a chunk
constexpr uint32_t kT3TmemCols = 512;

__device__ __forceinline__ bool mbar_wait_abort(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    // the thread may be suspended up to 20 us inside try_wait (woken when the
    // phase completes), so waiting roles take few issue slots
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(mbar), "r"(parity), "r"(20000u) : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      atomicExch(&g_xeng_status, 1);
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

__global__ void __launch_bounds__(kT3Threads, 1)
k_xeng_tc3(const int8_t* __restrict__ q, int n_ant, int n_spec, int n_tiles, int n_pairs, long long n_items,
           int32_t* __restrict__ vis) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full_b[kT3Stages], empty_b[kT3Stages], accf_b[2], acce_b[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int n_input = 2 * n_ant;
  const long long n_bl = static_cast<long long>(n_ant) * (n_ant + 1) / 2;
  const int n_chunks = (n_spec + kTcSpecPerChunk - 1) / kTcSpecPerChunk;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(kT3TmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kT3Stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full_b[s])), "r"(kT3ConvThreads)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty_b[s])) : "memory");
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&accf_b[a])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&acce_b[a])), "r"(kTcM) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  auto pair_of = [&](long long item, int& ch, int& I, int& J) {
    ch = static_cast<int>(item / n_pairs);
    int p = static_cast<int>(item - static_cast<long long>(ch) * n_pairs);
    I = 0;
    while (p >= n_tiles - I) { p -= n_tiles - I; ++I; }
    J = I + p;
  };

  if (warp < kT3ConvThreads / 32) {
    // ---------------------------------------------------------- converters
    const int pr = tid & 63;                           // operand rows 2 pr, 2 pr + 1
    const int qq = tid >> 6;                           // spectra qq kT3SpecPerThread .. of a chunk
    // this CTA's chunks in order (chunk gg is chunk gg % n_chunks of its item
    // gg / n_chunks); the reads run four chunks ahead of the conversion
    // (register sets 0-3), from a read cursor that moves to the next item's
    // rows once per item
    const int my_items = static_cast<int>((n_items - blockIdx.x + gridDim.x - 1) / gridDim.x);
    const int total = my_items * n_chunks;
    const int stride = n_input / 2;                    // 4-byte words per spectrum row
    int rd_it = 0, rd_c = 0;                           // read cursor: item, chunk
    const uint32_t* rd_a = nullptr;                    // word of inputs ia, ia + 1 in spectrum 8 qq of the item
    const uint32_t* rd_b = nullptr;
    bool rd_oka = false, rd_okb = false;
    auto rd_item = [&]() {
      rd_oka = rd_okb = false;
      if (rd_it >= my_items) return;
      int ch, I, J;
      pair_of(blockIdx.x + static_cast<long long>(rd_it) * gridDim.x, ch, I, J);
      const int ia = I * kTcM + 2 * pr, ib = J * kTcInputsN + 2 * pr;
      const uint32_t* base = reinterpret_cast<const uint32_t*>(q + static_cast<long long>(ch) * n_spec * n_input * 2) +
                             static_cast<long long>(qq * kT3SpecPerThread) * stride;
      rd_a = base + ia / 2;
      rd_b = base + ib / 2;
      rd_oka = ia < n_input;
      rd_okb = ib < n_input;
    };
    rd_item();
    uint32_t va0[kT3SpecPerThread], vb0[kT3SpecPerThread], va1[kT3SpecPerThread], vb1[kT3SpecPerThread];
    uint32_t va2[kT3SpecPerThread], vb2[kT3SpecPerThread], va3[kT3SpecPerThread], vb3[kT3SpecPerThread];
    auto read_next = [&](uint32_t (&va)[kT3SpecPerThread], uint32_t (&vb)[kT3SpecPerThread]) {
      // spectra valid in this thread's eighth of the chunk (0 past the last item)
      const int nv = rd_it < my_items ? n_spec - (rd_c * kTcSpecPerChunk + qq * kT3SpecPerThread) : 0;
      const uint32_t* pa = rd_a + static_cast<long long>(rd_c * kTcSpecPerChunk) * stride;
      const uint32_t* pb = rd_b + static_cast<long long>(rd_c * kTcSpecPerChunk) * stride;
#pragma unroll
      for (int ss = 0; ss < kT3SpecPerThread; ++ss) {
        va[ss] = (ss < nv && rd_oka) ? __ldg(pa) : 0u;
        vb[ss] = (ss < nv && rd_okb) ? __ldg(pb) : 0u;
        pa += stride;
        pb += stride;
      }
      if (++rd_c == n_chunks) {
        rd_c = 0;
        ++rd_it;
        rd_item();
      }
    };
    // (re, im) int8 pairs -> FP16 pairs, exact: with the sign bits flipped
    // each byte is the low byte of the FP16 number 1024 + 128 + q (high byte
    // 0x64), and one packed subtraction of 1152 leaves q
    const __half2 k1152 = __float2half2_rn(1152.0f);
    auto to_h2 = [&](uint32_t x, uint32_t sel) {
      const uint32_t w = __byte_perm(x, 0x64646464u, sel);
      const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&w), k1152);
      return *reinterpret_cast<const uint32_t*>(&h);
    };
    // this thread's operand rows: byte offsets within a stage at K = 0
    const uint32_t oa0 = op_offset(2 * pr, 0), oa1 = op_offset(2 * pr + 1, 0);
    // B rows 0..127 hold X, rows 128..255 Z (so a quarter-warp's stores fall
    // on two rows of each 8-row core matrix group: 2-way bank conflicts)
    const uint32_t ob0 = kTcASmem + op_offset(2 * pr, 0), ob1 = kTcASmem + op_offset(kTcInputsN + 2 * pr, 0);
    const uint32_t ob2 = kTcASmem + op_offset(2 * pr + 1, 0), ob3 = kTcASmem + op_offset(kTcInputsN + 2 * pr + 1, 0);
    // convert chunk gg into its stage once the stage is free
    auto convert = [&](int gg, const uint32_t (&va)[kT3SpecPerThread], const uint32_t (&vb)[kT3SpecPerThread]) {
      const int s = gg % kT3Stages;
      const uint32_t use = static_cast<uint32_t>(gg / kT3Stages);
      if (!mbar_wait_abort(smem_u32(&empty_b[s]), (use & 1u) ^ 1u, abort_flag)) return false;
      unsigned char* st = smem + s * kT3StageBytes;
#pragma unroll
      for (int h2 = 0; h2 < kT3SpecPerThread / 4; ++h2) {
        // spectra 4 k .. 4 k + 3 of the chunk are K elements 8 k .. 8 k + 7:
        // one 16-byte core-matrix row per operand row
        uint32_t a0[4], a1[4], x0[4], x1[4], z0[4], z1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ss = 4 * h2 + u;
          const uint32_t xa = va[ss] ^ 0x80808080u, xb = vb[ss] ^ 0x80808080u;
          a0[u] = to_h2(xa, 0x5140u);
          a1[u] = to_h2(xa, 0x5342u);
          x0[u] = to_h2(xb, 0x5140u);
          x1[u] = to_h2(xb, 0x5342u);
          // Z = (-im, re): the halves swapped, the new low one negated
          z0[u] = __byte_perm(x0[u], 0u, 0x1032u) ^ 0x00008000u;
          z1[u] = __byte_perm(x1[u], 0u, 0x1032u) ^ 0x00008000u;
        }
        unsigned char* sk = st + (qq * (kT3SpecPerThread / 4) + h2) * kLBO;
        *reinterpret_cast<uint4*>(sk + oa0) = make_uint4(a0[0], a0[1], a0[2], a0[3]);
        *reinterpret_cast<uint4*>(sk + oa1) = make_uint4(a1[0], a1[1], a1[2], a1[3]);
        *reinterpret_cast<uint4*>(sk + ob0) = make_uint4(x0[0], x0[1], x0[2], x0[3]);
        *reinterpret_cast<uint4*>(sk + ob1) = make_uint4(z0[0], z0[1], z0[2], z0[3]);
        *reinterpret_cast<uint4*>(sk + ob2) = make_uint4(x1[0], x1[1], x1[2], x1[3]);
        *reinterpret_cast<uint4*>(sk + ob3) = make_uint4(z1[0], z1[1], z1[2], z1[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full_b[s]));
      return true;
    };
    read_next(va0, vb0);
    read_next(va1, vb1);
    read_next(va2, vb2);
    read_next(va3, vb3);
    for (int gg = 0; gg < total; gg += 4) {
      // each set is refilled four chunks ahead as soon as it is converted
      if (!convert(gg, va0, vb0)) break;
      read_next(va0, vb0);
      if (gg + 1 >= total) break;
      if (!convert(gg + 1, va1, vb1)) break;
      read_next(va1, vb1);
      if (gg + 2 >= total) break;
      if (!convert(gg + 2, va2, vb2)) break;
      read_next(va2, vb2);
      if (gg + 3 >= total) break;
      if (!convert(gg + 3, va3, vb3)) break;
      read_next(va3, vb3);
    }
  } else if (warp == kT3MmaWarp) {
    // ------------------------------------------------------------------ MMA
    if (lane == 0) {
      long long g = 0;
      int li = 0;                                      // items of this CTA so far
      for (long long item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x, ++li) {
        const int a = li & 1;
        const uint32_t ause = static_cast<uint32_t>(li >> 1);
        if (!mbar_wait_abort(smem_u32(&acce_b[a]), (ause & 1u) ^ 1u, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + static_cast<uint32_t>(a * 256);
        bool ok = true;
        for (int c = 0; c < n_chunks; ++c, ++g) {
          const int s = static_cast<int>(g % kT3Stages);
          const uint32_t use = static_cast<uint32_t>(g / kT3Stages);
          if (!mbar_wait_abort(smem_u32(&full_b[s]), use & 1u, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(smem + s * kT3StageBytes), b0 = a0 + kTcASmem;
#pragma unroll
          for (int kk = 0; kk < kTcKc / 16; ++kk) {
            const uint64_t ad = make_sdesc(a0 + kk * 2 * kLBO);
            const uint64_t bd = make_sdesc(b0 + kk * 2 * kLBO);
            const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                :: "r"(d), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&empty_b[s])) : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&accf_b[a])) : "memory");
      }
      // before TMEM is released, the MMAs this thread issued complete: the
      // commit of its last chunk arrives (a bounded wait that ignores the
      // abort flag, so an aborted run still drains its MMAs)
      if (g > 0) {
        const long long gl = g - 1;
        (void)mbar_wait(smem_u32(&empty_b[gl % kT3Stages]), static_cast<uint32_t>(gl / kT3Stages) & 1u);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp & 3;
    int li = 0;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x, ++li) {
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;    // warp-uniform
      int ch, I, J;
      pair_of(item, ch, I, J);
      const int a = li & 1;
      const uint32_t ause = static_cast<uint32_t>(li >> 1);
      // one lane waits, the warp follows its verdict: tcgen05.ld needs the
      // whole warp converged
      bool ok = true;
      if (lane == 0) ok = mbar_wait_abort(smem_u32(&accf_b[a]), ause & 1u, abort_flag);
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int gi = I * kTcM + q4 * 32 + lane;
      const int an = gi >> 1, pa = gi & 1;
      int4* out = reinterpret_cast<int4*>(vis + static_cast<long long>(ch) * n_bl * 8);
      const uint32_t tl0 = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + static_cast<uint32_t>(a * 256);
#pragma unroll 1
      for (int cin0 = 0; cin0 < kTcInputsN; cin0 += 16) {
        // TMEM columns cin0 .. cin0 + 15: Re of column inputs J 128 + cin0 ..;
        // the same + 128: their Im (16 columns at a time keep the epilogue's
        // registers within the 21-warp CTA's budget)
        uint32_t re[16], im[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
              "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]),
              "=r"(re[14]), "=r"(re[15])
            : "r"(tl0 + cin0));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
              "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]),
              "=r"(im[14]), "=r"(im[15])
            : "r"(tl0 + cin0 + 128u));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (an < n_ant) {
          const int b0 = (J * kTcInputsN + cin0) >> 1;
#pragma unroll
          for (int bb = 0; bb < 8; ++bb) {
            const int b = b0 + bb;
            if (b >= n_ant || b < an) continue;
            int4 v;
            v.x = __float2int_rn(__uint_as_float(re[2 * bb]));
            v.y = __float2int_rn(__uint_as_float(im[2 * bb]));
            v.z = __float2int_rn(__uint_as_float(re[2 * bb + 1]));
            v.w = __float2int_rn(__uint_as_float(im[2 * bb + 1]));
            __stcs(out + bl_index(an, b, n_ant) * 2 + pa, v);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&acce_b[a]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kT3TmemCols) : "memory");
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
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0 || reinterpret_cast<uintptr_t>(d_fine_q) % 4 != 0)
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
  // three 48 KB operand stages: one CTA (and one 512-column TMEM allocation) per SM
  const int smem = kT3Stages * kT3StageBytes;
  OVRO_CUDA_TRY(cudaFuncSetAttribute(k_xeng_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long grid = std::min<long long>(num_sms(), n_items);
  OVRO_PROF("k_xeng_tc", st);
  k_xeng_tc3<<<static_cast<unsigned>(grid), kT3Threads, smem, st>>>(d_fine_q, n_ant, n_spec, n_tiles, n_pairs,
                                                                    n_items, d_vis);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
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
