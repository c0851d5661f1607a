// Library-side prolate-spheroidal gridding kernel tables (host).
#pragma once

#include <vector>

namespace ovro {

constexpr int kSupport = 7;        // kernel support, cells
constexpr int kOversample = 1024;  // table samples per cell

struct KernelTables {
  std::vector<double> table64;     // C(m / Q), m = -S Q / 2 .. S Q / 2
  std::vector<float> table32;
};

// psi_0(7 pi / 2, x / 3.5) normalised to 1 at x = 0, tabulated (computed once).
const KernelTables& kernel_tables();
// Grid correction C^(d), d = -N/2 .. N/2 - 1 of an image whose uv grid has G
// cells a side: Fourier transform of the table at frequency d / G.
void grid_correction(int n, int g, std::vector<double>& out);

}  // namespace ovro
