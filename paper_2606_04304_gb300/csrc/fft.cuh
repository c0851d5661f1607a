// In-register radix-R DFTs and a shared-memory Stockham FFT used by the
// upchannelizer and the imaging kernels.
#pragma once

#include "common.cuh"

namespace ovro {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int R>
struct BitRev {
  static __device__ __forceinline__ constexpr int of(int x) {
    int r = 0;
    for (int b = 1, m = R >> 1; b < R; b <<= 1, m >>= 1)
      if (x & b) r |= m;
    return r;
  }
};

// V[k] = sum_r v[r] exp(-2 pi i r k / R), natural order in and out.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  float2 t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[BitRev<R>::of(i)];
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        float2 x = t[b + j + h];
        if (j != 0) {
          // w = exp(-2 pi i j / (2h)) = exp(-2 pi i (j * 8 / h) / 16)
          const int q = j * (8 / h);
          float cw, sw;
          switch (q) {
            case 1: cw = 0.92387953251128674f; sw = -0.38268343236508977f; break;
            case 2: cw = 0.70710678118654752f; sw = -0.70710678118654752f; break;
            case 3: cw = 0.38268343236508977f; sw = -0.92387953251128674f; break;
            case 4: cw = 0.0f; sw = -1.0f; break;
            case 5: cw = -0.38268343236508977f; sw = -0.92387953251128674f; break;
            case 6: cw = -0.70710678118654752f; sw = -0.70710678118654752f; break;
            default: cw = -0.92387953251128674f; sw = -0.38268343236508977f; break;
          }
          if (q == 4) {
            x = make_float2(x.y, -x.x);           // multiply by -i
          } else {
            x = cmul(x, make_float2(cw, sw));
          }
        }
        const float2 a = t[b + j];
        t[b + j] = make_float2(a.x + x.x, a.y + x.y);
        t[b + j + h] = make_float2(a.x - x.x, a.y - x.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}


// Forward FFTs (exp(-2 pi i k n / N)) of `count` rows of length N = 2^LOG2N
// stored in `a` with row stride `ld` >= N; `b` is a scratch buffer of the same
// shape.  Stockham auto-sort: radix-16 passes, then one radix-2/4/8 pass.
// All threads of the block take part; returns the buffer holding the result.
// tw: omega_{N * tw_stride}^k table.
template <int LOG2N>
__device__ float2* fft_rows_pingpong(float2* a, float2* b, int count, int ld,
                                     const float2* __restrict__ tw, int tw_stride) {
  constexpr int N = 1 << LOG2N;
  constexpr int n16 = LOG2N / 4;
  constexpr int rem = LOG2N % 4;
  constexpr int n_pass = n16 + (rem ? 1 : 0);
  int Ns = 1;
  float2* src = a;
  float2* dst = b;
#pragma unroll 1
  for (int p = 0; p < n_pass; ++p) {
    const int R = (p < n16) ? 16 : (1 << rem);
    const int per = N / R;
    const int total = count * per;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int f = t / per, j = t - f * per;
      const int k = j & (Ns - 1);
      const float2* s = src + f * ld;
      float2* d = dst + f * ld;
      const int o = (j / Ns) * Ns * R + k;
      const int base = k * (N / (Ns * R));
      if (R == 16) {
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = s[j + r * per];
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], __ldg(tw + (r * base) * tw_stride));
        }
        dft_reg<16>(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) d[o + r * Ns] = v[r];
      } else if (R == 8) {
        float2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = s[j + r * per];
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], __ldg(tw + (r * base) * tw_stride));
        }
        dft_reg<8>(v);
#pragma unroll
        for (int r = 0; r < 8; ++r) d[o + r * Ns] = v[r];
      } else if (R == 4) {
        float2 v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = s[j + r * per];
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < 4; ++r) v[r] = cmul(v[r], __ldg(tw + (r * base) * tw_stride));
        }
        dft_reg<4>(v);
#pragma unroll
        for (int r = 0; r < 4; ++r) d[o + r * Ns] = v[r];
      } else {
        float2 v[2];
        v[0] = s[j];
        v[1] = s[j + per];
        if (Ns > 1) v[1] = cmul(v[1], __ldg(tw + base * tw_stride));
        dft_reg<2>(v);
        d[o] = v[0];
        d[o + Ns] = v[1];
      }
    }
    __syncthreads();
    float2* t = src; src = dst; dst = t;
    Ns *= R;
  }
  return src;
}

}  // namespace ovro

namespace ovro {

// Shared-memory index with one pad slot per 16 elements: Stockham writes at
// stride 16 become conflict-free.
__device__ __forceinline__ int pad16(int x) { return x + (x >> 4); }

// One Stockham pass in place over rows of G points, the first NS-point
// transforms already done (G, R and NS are compile-time, so every index split
// is a shift).  load(f, x) gives element x of row f of the pass's input (the
// rows themselves, or another source for a first pass; every read completes
// before the first write, so the source may overlap `a`); tw(i) = omega_G^i.
template <int R, int NS, int G, class Load, class Tw>
__device__ __forceinline__ void stockham_pass(float2* a, int ldp, Load&& load, Tw&& tw) {
  // every thread holds exactly 16 values: 16 / R butterflies of radix R
  constexpr int NB = 16 / R;
  constexpr int per = G / R;
  const int T = blockDim.x;
  float2 v[16];
  int fj[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int gb = threadIdx.x + b * T;
    const int f = gb / per, j = gb - f * per;
    fj[b] = gb;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = load(f, j + r * per);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int f = fj[b] / per, j = fj[b] - f * per;
    const int k = j & (NS - 1);
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[b * R + r];
    if (NS > 1) {
      // twiddles w^r, w = omega_G^base: w^(2^m) read, the others products of
      // those (at most three roundings deep), so a pass reads log2 R of them
      const int base = k * (G / (NS * R));
      float2 t[R];
      t[1] = tw(base);
      if (R >= 4) t[2] = tw(2 * base);
      if (R >= 8) t[4] = tw(4 * base);
      if (R >= 16) t[8] = tw(8 * base);
#pragma unroll
      for (int r = 3; r < R; ++r) {
        if ((r & (r - 1)) == 0) continue;
        const int hb = 1 << (31 - __clz(r));            // highest power of two in r (compile-time)
        t[r] = cmul(t[hb], t[r - hb]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], t[r]);
    }
    dft_reg<R>(x);
    const int o = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) a[f * ldp + pad16(o + r * NS)] = x[r];
  }
  __syncthreads();
}

// In-place forward FFTs of the rows of `a` (row f at a[f * ldp], element x at
// pad16(x)), G = 2^LOG2G with 16 <= G <= 16384, with blockDim.x * 16 == rows * G:
// radix-16 passes, then one of radix 2, 4 or 8.  The first pass reads its
// input through load0(f, x); tw(i) = omega_G^i.
template <int LOG2G, class Load, class Tw>
__device__ void fft_rows_inplace_f(float2* a, int ldp, Load&& load0, Tw&& tw) {
  constexpr int G = 1 << LOG2G;
  constexpr int n16 = LOG2G / 4;
  constexpr int rem = LOG2G % 4;
  constexpr int NSR = 1 << (4 * n16);                 // transforms done before the last radix-2/4/8 pass
  static_assert(n16 >= 1 && n16 <= 3, "16 <= G <= 16384");
  auto rows = [&](int f, int x) { return a[f * ldp + pad16(x)]; };
  stockham_pass<16, 1, G>(a, ldp, load0, tw);
  if constexpr (n16 >= 2) stockham_pass<16, 16, G>(a, ldp, rows, tw);
  if constexpr (n16 >= 3) stockham_pass<16, 256, G>(a, ldp, rows, tw);
  if constexpr (rem == 1) stockham_pass<2, NSR, G>(a, ldp, rows, tw);
  if constexpr (rem == 2) stockham_pass<4, NSR, G>(a, ldp, rows, tw);
  if constexpr (rem == 3) stockham_pass<8, NSR, G>(a, ldp, rows, tw);
}

}  // namespace ovro
