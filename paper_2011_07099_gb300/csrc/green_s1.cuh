// G_S1, the approximately optimal periodic Green's function (Sec. 3, n = 1,
// a_1 = -1/8), in FP64 for the table and mesh kernels.
//
//   G(x) = -1/(4 pi |xhat|),  xhat_i = xi(x_i),
//   xi(t) = (9/(8 pi)) sin(pi t) - (1/(24 pi)) sin(3 pi t).
//
// xi is odd-periodic, so |xhat| and G are 1-periodic and the wrap of xhat is a
// no-op.  Gradient by the chain rule: dG/dx_i = xhat_i xi'(x_i) / (4 pi
// |xhat|^3), xi'(t) = (9/8) cos(pi t) - (1/8) cos(3 pi t).
#pragma once

namespace fmm {
namespace green {

constexpr double kPi = 3.14159265358979323846;

// Mean of 1/r over the unit cube: 3 ln(2 + sqrt 3) - pi/2.  The paper does not
// define the self term G(0); the cell-averaged Newtonian value is used.
__device__ inline double cube_mean_inv_r() { return 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * kPi; }

__device__ inline double xi_s1(double t) {
  return (9.0 / (8.0 * kPi)) * sinpi(t) - (1.0 / (24.0 * kPi)) * sinpi(3.0 * t);
}
__device__ inline double dxi_s1(double t) { return 1.125 * cospi(t) - 0.125 * cospi(3.0 * t); }

// (G, -dG/dx, -dG/dy, -dG/dz) at x != 0 (box units); the caller handles x == 0.
__device__ inline void gs1(double x, double y, double z, double out[4]) {
  const double hx = xi_s1(x), hy = xi_s1(y), hz = xi_s1(z);
  const double r2 = hx * hx + hy * hy + hz * hz;
  const double r = sqrt(r2);
  const double inv4pi = 1.0 / (4.0 * kPi);
  out[0] = -inv4pi / r;
  const double c = -inv4pi / (r2 * r);
  out[1] = c * hx * dxi_s1(x);
  out[2] = c * hy * dxi_s1(y);
  out[3] = c * hz * dxi_s1(z);
}

}  // namespace green
}  // namespace fmm
