// Green's functions of the tables, in FP64 for the table and mesh kernels.
//
// G_S1, the approximately optimal periodic Green's function (Sec. 3, n = 1,
// a_1 = -1/8; eq. gfs1):
//   G(x) = -1/(4 pi |xhat|),  xhat_i = xi(x_i),
//   xi(t) = (9/(8 pi)) sin(pi t) - (1/(24 pi)) sin(3 pi t).
// xi is odd-periodic, so |xhat| and G are 1-periodic and the wrap of xhat is a
// no-op.  Gradient by the chain rule: dG/dx_i = xhat_i xi'(x_i) / (4 pi
// |xhat|^3), xi'(t) = (9/8) cos(pi t) - (1/8) cos(3 pi t).
//
// G_S, the ansatz of Sec. 3 with free coefficients a_1..a_n:
//   xi_n(t) = sin(pi t)/pi + sum_k a_k (sin((2k+1) pi t)/((2k+1) pi) - sin(pi t)/pi),
// G_S1 being n = 1, a_1 = -1/8.
//
// G_0 = -1/(4 pi r), the Newtonian Green's function of the isolated
// (non-periodic) problem of Sec. 3's accuracy experiment (eq. gerr).
//
// G_X = -1/(4 pi |x <> L|), the "exact-in-real-space" periodic function of
// Sec. 1 (eq. gfx): the displacement wrapped to its nearest image.  It has a
// kink where a wrapped component is +-L/2 (the aliasing of Fig. errex); there
// the gradient component is taken as the mean of the two one-sided values, 0.
#pragma once

namespace fmm {
namespace green {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxAnsatz = 4;     // coefficients a_1..a_4 of the G_S ansatz

// Which function a plan tabulates (FMM_GREEN_* of fmm.h), with the ansatz
// coefficients of G_S.
struct Spec {
  int kind = 0;                   // 0 G_S1, 1 G_S(a), 2 G_0, 3 G_X, 4 sampled on the mesh
  int na = 0;
  double a[kMaxAnsatz] = {0.0, 0.0, 0.0, 0.0};
};

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

// xi_n of the ansatz and its derivative.
__device__ inline void xi_ansatz(double t, const Spec& g, double& xi, double& dxi) {
  const double s1 = sinpi(t) / kPi, c1 = cospi(t);
  xi = s1;
  dxi = c1;
  for (int k = 1; k <= g.na; ++k) {
    const double m = 2.0 * k + 1.0;
    xi += g.a[k - 1] * (sinpi(m * t) / (m * kPi) - s1);
    dxi += g.a[k - 1] * (cospi(m * t) - c1);
  }
}

// The same four values for G_S(a) (periodic, like G_S1).
__device__ inline void gs_ansatz(double x, double y, double z, const Spec& g, double out[4]) {
  double h[3], d[3];
  xi_ansatz(x, g, h[0], d[0]);
  xi_ansatz(y, g, h[1], d[1]);
  xi_ansatz(z, g, h[2], d[2]);
  const double r2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  const double r = sqrt(r2);
  const double inv4pi = 1.0 / (4.0 * kPi);
  out[0] = -inv4pi / r;
  const double c = -inv4pi / (r2 * r);
  for (int i = 0; i < 3; ++i) out[1 + i] = c * h[i] * d[i];
}

// The same four values for G_0 (no wrap: x is the displacement itself).
__device__ inline void g0(double x, double y, double z, double out[4]) {
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  const double inv4pi = 1.0 / (4.0 * kPi);
  out[0] = -inv4pi / r;
  const double c = -inv4pi / (r2 * r);
  out[1] = c * x;
  out[2] = c * y;
  out[3] = c * z;
}

// The same four values for G_X.
__device__ inline void gx(double x, double y, double z, double out[4]) {
  const double w[3] = {x - rint(x), y - rint(y), z - rint(z)};
  const double r2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double r = sqrt(r2);
  const double inv4pi = 1.0 / (4.0 * kPi);
  out[0] = -inv4pi / r;
  const double c = -inv4pi / (r2 * r);
  for (int i = 0; i < 3; ++i) out[1 + i] = fabs(w[i]) == 0.5 ? 0.0 : c * w[i];
}

// Dispatch on the plan's analytic function; x != 0.  (A function sampled on
// the mesh, kind 4, is looked up by the table kernels instead.)
__device__ inline void eval(const Spec& g, double x, double y, double z, double out[4]) {
  if (g.kind == 1)
    gs_ansatz(x, y, z, g, out);
  else if (g.kind == 2)
    g0(x, y, z, out);
  else if (g.kind == 3)
    gx(x, y, z, out);
  else
    gs1(x, y, z, out);
}

}  // namespace green
}  // namespace fmm
