// In-register DFTs of lengths 2, 3, 4, 5 and their coprime products 6, 10,
// 12, 15 (prime-factor algorithm), for the mixed-radix upchannelizer that
// handles N = 2^a 3^b 5^c, such as the paper's N = 2400 (Section 2.1).
//
// All transforms are forward, V[k] = sum_r v[r] exp(-2 pi i r k / R), natural
// order in and out.  Callable from host code too, so that the index maps can be
// checked against a direct DFT on the CPU.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace ovro {
namespace mr {

#define OVRO_HD __host__ __device__ __forceinline__

OVRO_HD float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
OVRO_HD float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
OVRO_HD float2 scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a - i b and a + i b
OVRO_HD float2 sub_i(float2 a, float2 b) { return make_float2(a.x + b.y, a.y - b.x); }
OVRO_HD float2 add_i(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }
OVRO_HD float2 mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

OVRO_HD void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = add(t, b);
  b = sub(t, b);
}

// omega_3 = -1/2 - i sqrt(3)/2:  X1,2 = a - (b + c)/2 -/+ i (sqrt(3)/2) (b - c)
OVRO_HD void dft3(float2& a, float2& b, float2& c) {
  constexpr float h = 0.866025403784438647f;   // sin(2 pi / 3)
  const float2 t1 = add(b, c);
  const float2 t2 = scale(sub(b, c), h);
  const float2 m = sub(a, scale(t1, 0.5f));
  a = add(a, t1);
  b = sub_i(m, t2);
  c = add_i(m, t2);
}

// X0..3 of 4 points: the radix-2 butterflies with the -i rotation.
OVRO_HD void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 s0 = add(a, c), d0 = sub(a, c);
  const float2 s1 = add(b, d), d1 = sub(b, d);
  a = add(s0, s1);
  c = sub(s0, s1);
  b = sub_i(d0, d1);
  d = add_i(d0, d1);
}

// With c1 = cos(2 pi/5), c2 = cos(4 pi/5), s1 = sin(2 pi/5), s2 = sin(4 pi/5),
// a1 = x1 + x4, b1 = x1 - x4, a2 = x2 + x3, b2 = x2 - x3:
// X1,4 = x0 + c1 a1 + c2 a2 -/+ i (s1 b1 + s2 b2)
// X2,3 = x0 + c2 a1 + c1 a2 -/+ i (s2 b1 - s1 b2)
OVRO_HD void dft5(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4) {
  constexpr float c1 = 0.309016994374947424f;
  constexpr float c2 = -0.809016994374947424f;
  constexpr float s1 = 0.951056516295153572f;
  constexpr float s2 = 0.587785252292473129f;
  const float2 a1 = add(x1, x4), b1 = sub(x1, x4);
  const float2 a2 = add(x2, x3), b2 = sub(x2, x3);
  const float2 p1 = add(x0, add(scale(a1, c1), scale(a2, c2)));
  const float2 p2 = add(x0, add(scale(a1, c2), scale(a2, c1)));
  const float2 q1 = add(scale(b1, s1), scale(b2, s2));
  const float2 q2 = sub(scale(b1, s2), scale(b2, s1));
  x0 = add(x0, add(a1, a2));
  x1 = sub_i(p1, q1);
  x4 = add_i(p1, q1);
  x2 = sub_i(p2, q2);
  x3 = add_i(p2, q2);
}

template <int R>
OVRO_HD void dft_prime(float2 (&v)[R]) {
  static_assert(R == 2 || R == 3 || R == 4 || R == 5, "small DFT length");
  if constexpr (R == 2) dft2(v[0], v[1]);
  if constexpr (R == 3) dft3(v[0], v[1], v[2]);
  if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  if constexpr (R == 5) dft5(v[0], v[1], v[2], v[3], v[4]);
}

// Index maps of the prime-factor algorithm for R = R1 R2, gcd(R1, R2) = 1,
// built at compile time: in[n2][n1] = (R2 n1 + R1 n2) mod R, and out[k1][k2]
// the k in [0, R) with k = k1 (mod R1), k = k2 (mod R2).
template <int R1, int R2>
struct PfaMap {
  int in[R2][R1];
  int out[R1][R2];
  constexpr PfaMap() : in(), out() {
    for (int n2 = 0; n2 < R2; ++n2)
      for (int n1 = 0; n1 < R1; ++n1) in[n2][n1] = (R2 * n1 + R1 * n2) % (R1 * R2);
    for (int k = 0; k < R1 * R2; ++k) out[k % R1][k % R2] = k;
  }
};

template <int R1, int R2, int N2, int N1>
struct PfaIn {
  static constexpr int value = PfaMap<R1, R2>().in[N2][N1];
};
template <int R1, int R2, int K1, int K2>
struct PfaOut {
  static constexpr int value = PfaMap<R1, R2>().out[K1][K2];
};

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
OVRO_HD void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Prime-factor (Good-Thomas) DFT of R = R1 R2, gcd(R1, R2) = 1: input index
// n = (R2 n1 + R1 n2) mod R, then R1-point DFTs over n1, R2-point DFTs over
// n2, and the output at the Chinese-remainder index of (k1, k2).  No twiddles.
// Every index is a template constant, so the arrays stay in registers.
template <int R1, int R2>
OVRO_HD void dft_pfa(float2 (&v)[R1 * R2]) {
  float2 t[R1][R2];
  static_for<0, R2>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    float2 u[R1];
    static_for<0, R1>([&](auto n1c) {
      constexpr int n1 = decltype(n1c)::value;
      u[n1] = v[PfaIn<R1, R2, n2, n1>::value];
    });
    dft_prime<R1>(u);
    static_for<0, R1>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      t[k1][n2] = u[k1];
    });
  });
  static_for<0, R1>([&](auto k1c) {
    constexpr int k1 = decltype(k1c)::value;
    float2 u[R2];
    static_for<0, R2>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      u[n2] = t[k1][n2];
    });
    dft_prime<R2>(u);
    static_for<0, R2>([&](auto k2c) {
      constexpr int k2 = decltype(k2c)::value;
      v[PfaOut<R1, R2, k1, k2>::value] = u[k2];
    });
  });
}

// 8- and 16-point DFTs from two radix-2 / radix-4 levels (Cooley-Tukey,
// decimation in time) with the constant twiddles of the 8th / 16th roots.
OVRO_HD float2 rot8(float2 x, int q) {
  // x exp(-2 pi i q / 8), q in [0, 8)
  constexpr float r = 0.707106781186547524f;
  switch (q & 7) {
    case 0: return x;
    case 1: return make_float2(r * (x.x + x.y), r * (x.y - x.x));
    case 2: return make_float2(x.y, -x.x);
    case 3: return make_float2(r * (x.y - x.x), -r * (x.x + x.y));
    case 4: return make_float2(-x.x, -x.y);
    case 5: return make_float2(-r * (x.x + x.y), r * (x.x - x.y));
    case 6: return make_float2(-x.y, x.x);
    default: return make_float2(r * (x.x - x.y), r * (x.x + x.y));
  }
}

OVRO_HD void dft8(float2 (&v)[8]) {
  // two 4-point DFTs over even / odd samples, then 2-point butterflies
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft_prime<4>(e);
  dft_prime<4>(o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 w = rot8(o[k], k);
    v[k] = add(e[k], w);
    v[k + 4] = sub(e[k], w);
  }
}

OVRO_HD float2 rot16(float2 x, int q) {
  // x exp(-2 pi i q / 16), q in [0, 16)
  constexpr float c = 0.923879532511286756f;   // cos(pi / 8)
  constexpr float s = 0.382683432365089772f;   // sin(pi / 8)
  if ((q & 1) == 0) return rot8(x, q >> 1);
  // odd q: exp(-i pi q / 8) = exp(-i pi / 8) exp(-i pi (q - 1) / 8)
  const float2 y = make_float2(c * x.x + s * x.y, c * x.y - s * x.x);
  return rot8(y, (q - 1) >> 1);
}

OVRO_HD void dft16(float2 (&v)[16]) {
  // four 4-point DFTs over n = 4 m + r (m the inner index), twiddle
  // exp(-2 pi i r k1 / 16), then 4-point DFTs over r; output k = k1 + 4 k2
  float2 t[16];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 u[4] = {v[r], v[r + 4], v[r + 8], v[r + 12]};
    dft_prime<4>(u);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) t[k1 * 4 + r] = rot16(u[k1], r * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 u[4] = {t[k1 * 4], t[k1 * 4 + 1], t[k1 * 4 + 2], t[k1 * 4 + 3]};
    dft_prime<4>(u);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = u[k2];
  }
}

// The DFT of every radix the mixed-radix planner uses.
template <int R>
OVRO_HD void dft(float2 (&v)[R]) {
  if constexpr (R == 2 || R == 3 || R == 4 || R == 5) dft_prime<R>(v);
  else if constexpr (R == 6) dft_pfa<2, 3>(v);
  else if constexpr (R == 10) dft_pfa<2, 5>(v);
  else if constexpr (R == 12) dft_pfa<4, 3>(v);
  else if constexpr (R == 15) dft_pfa<3, 5>(v);
  else if constexpr (R == 8) dft8(v);
  else if constexpr (R == 16) dft16(v);
  else static_assert(R == 2, "radix not supported");
}

#undef OVRO_HD

}  // namespace mr
}  // namespace ovro
