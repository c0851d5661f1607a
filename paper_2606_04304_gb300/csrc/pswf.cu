// Prolate-spheroidal gridding kernel for the imaging step (Section 2.2 images
// with WSClean; the 7 x 7 prolate-spheroidal kernel is this build's choice).
//
// psi_0(c, eta), c = 7 pi / 2, is computed here as the eigenfunction of the
// finite Fourier (cosine) operator restricted to even functions,
//     int_{-1}^{1} cos(c eta y) psi(y) dy = lambda psi(eta),
// whose largest positive eigenvalue belongs to psi_0.  The operator is
// discretised with Gauss-Legendre quadrature (Nystrom method), the symmetric
// matrix is diagonalised with cyclic Jacobi rotations, and psi_0 is evaluated
// anywhere through the eigen-equation itself (Nystrom interpolation).
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "pswf.h"

namespace ovro {
namespace {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;                    // P_0, P_1
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);      // P_n'(z)
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix a (row-major).
void jacobi_eig(std::vector<double> a, int n, std::vector<double>& evals, std::vector<double>& v) {
  v.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {           // A <- A J (columns p, q)
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {           // A <- J^T A (rows p, q)
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {           // V <- V J
          const double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  evals.resize(n);
  for (int i = 0; i < n; ++i) evals[i] = a[i * n + i];
}

struct Psi0 {
  std::vector<double> y, wy, f;   // positive nodes, weights, psi values there
  double lam = 0.0, c = 0.0, norm = 1.0;

  double raw(double eta) const {   // Nystrom interpolation through the eigen-equation
    double acc = 0.0;
    for (size_t j = 0; j < y.size(); ++j) acc += 2.0 * wy[j] * std::cos(c * eta * y[j]) * f[j];
    return acc / lam;
  }
  double operator()(double eta) const { return raw(eta) / norm; }
};

Psi0 build_psi0(double c) {
  const int n_full = 96;
  std::vector<double> x, w;
  gauss_legendre(n_full, x, w);
  Psi0 p;
  p.c = c;
  for (int i = 0; i < n_full; ++i)
    if (x[i] > 0) {
      p.y.push_back(x[i]);
      p.wy.push_back(w[i]);
    }
  const int n = static_cast<int>(p.y.size());
  // even part of the operator on [0, 1]: 2 cos(c y_i y_j), symmetrised by sqrt(w)
  std::vector<double> m(static_cast<size_t>(n) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      m[i * n + j] = 2.0 * std::sqrt(p.wy[i] * p.wy[j]) * std::cos(c * p.y[i] * p.y[j]);
  std::vector<double> ev, vec;
  jacobi_eig(m, n, ev, vec);
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (ev[i] > ev[best]) best = i;
  p.lam = ev[best];
  p.f.resize(n);
  for (int i = 0; i < n; ++i) p.f[i] = vec[i * n + best] / std::sqrt(p.wy[i]);
  p.norm = p.raw(0.0);
  return p;
}

}  // namespace

const KernelTables& kernel_tables() {
  static KernelTables t;
  static std::once_flag once;
  std::call_once(once, [] {
    const Psi0 psi = build_psi0(M_PI * kSupport / 2.0);
    const int half = kSupport * kOversample / 2;
    t.table64.resize(2 * half + 1);
    t.table32.resize(2 * half + 1);
    for (int m = -half; m <= half; ++m) {
      const double eta = static_cast<double>(m) / kOversample / (kSupport / 2.0);
      t.table64[m + half] = psi(eta);
      t.table32[m + half] = static_cast<float>(t.table64[m + half]);
    }
  });
  return t;
}

void grid_correction(int n, int g, std::vector<double>& out) {
  // C^(d) = (1/Q) sum_m C(m / Q) cos(2 pi m d / (Q G)), d = -N/2 .. N/2 - 1
  const KernelTables& t = kernel_tables();
  const int half = kSupport * kOversample / 2;
  out.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double d = i - n / 2;
    double acc = 0.0;
    for (int m = -half; m <= half; ++m)
      acc += t.table64[m + half] * std::cos(2.0 * M_PI * m * d / (static_cast<double>(kOversample) * g));
    out[i] = acc / kOversample;
  }
}

}  // namespace ovro
