// Absorption spectrum of computed excited states (paper, Section "Results and
// discussion": oscillator strengths broadened by Gaussians of width 0.1 eV).
// Width is read as the standard deviation sigma, each line of unit area:
//   S(E) = sum_n f_n exp(-(E - omega_n)^2 / (2 sigma^2)) / (sigma sqrt(2 pi)).
// One thread per grid energy, the roots summed in their given order.
#include <cmath>

#include "kernels.h"
#include "prof.h"

namespace xs {

namespace {

__global__ void spectrum_kernel(int n, const double* __restrict__ omega, const double* __restrict__ f,
                                double inv_width, double norm, int ngrid, const double* __restrict__ grid,
                                double* __restrict__ out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrid) return;
  const double E = grid[g];
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = (E - omega[i]) * inv_width;
    s = fma(f[i], exp(-0.5 * x * x), s);
  }
  out[g] = s * norm;
}

}  // namespace

void absorption_spectrum(cudaStream_t s, int n, const double* omega, const double* f, double width, int ngrid,
                         const double* grid, double* out) {
  if (ngrid <= 0) return;
  const double norm = 1.0 / (width * std::sqrt(2.0 * 3.14159265358979323846));
  ProfScope ps(s, "spectrum", 8.0 * (2.0 * n + 2.0 * ngrid), 4.0 * (double)n * ngrid);
  spectrum_kernel<<<grid1(ngrid, 256), 256, 0, s>>>(n, omega, f, 1.0 / width, norm, ngrid, grid, out);
  XS_CHECK_LAUNCH();
}

}  // namespace xs
