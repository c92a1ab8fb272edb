// Contact self-energies on the device, always in FP64 (Eq. GR, Sec. 2.2.2).
//
// Every lead is a semi-infinite chain of rings with circulant couplings; in the ring
// Fourier basis each angular mode j is a dimerised chain whose surface Green's function g
// solves  a2 eps g^2 - (eps^2 - a1 + a2) g + eps = 0  (a1 = |lambda_j(T1)|^2,
// a2 = |lambda_j(T2)|^2, from g0 = 1/(eps - a1 g1), g1 = 1/(eps - a2 g0)), and
// sigma_j = |lambda_j(tau)|^2 g.  The retarded root is the one with Im g < 0: for
// Im eps > 0 the roots multiply to 1/a2, so exactly one has a negative imaginary part;
// if both imaginary parts agree to 1e-12 of |g| the root decaying into the lead
// (sqrt(a2)|g| < 1) is taken.
#pragma once
#include "common.cuh"

namespace negf {

// principal square root, branch cut on the negative real axis (Re sqrt >= 0)
__device__ __forceinline__ cd csqrt_principal(cd z) {
  double r = hypot(z.re, z.im);
  if (r == 0.0) return mk(0.0, 0.0);
  if (z.re >= 0.0) {
    double u = sqrt(0.5 * (r + z.re));
    return mk(u, z.im / (2.0 * u));
  }
  double v = copysign(sqrt(0.5 * (r - z.re)), z.im);
  return mk(z.im / (2.0 * v), v);
}

__device__ __forceinline__ cd cdiv(cd a, cd b) {
  double s = 1.0 / fma(b.re, b.re, b.im * b.im);
  return mk(fma(a.re, b.re, a.im * b.im) * s, fma(a.im, b.re, -(a.re * b.im)) * s);
}

// surface Green's function of the dimerised chain at complex energy eps
__device__ __forceinline__ cd surface_gf(cd eps, double a1, double a2) {
  if (a2 == 0.0) {
    cd den = mk(fma(eps.re, eps.re, -(eps.im * eps.im)) - a1, 2.0 * eps.re * eps.im);
    return cdiv(eps, den);
  }
  cd e2 = eps * eps;
  cd B = mk(e2.re - a1 + a2, e2.im);
  const cd BB = B * B;
  cd disc = mk(fma(-e2.re, 4.0 * a2, BB.re), fma(-e2.im, 4.0 * a2, BB.im));
  cd s = csqrt_principal(disc);
  cd qp = B + s, qm = B - s;
  cd q = (abs2(qp) >= abs2(qm)) ? qp : qm;
  cd g1 = cdiv(q, scale(eps, 2.0 * a2));
  cd g2 = cdiv(scale(eps, 2.0), q);
  double sc = sqrt(abs2(g1)) + sqrt(abs2(g2));
  if (fabs(g1.im - g2.im) <= 1e-12 * sc) {
    return (sqrt(a2) * sqrt(abs2(g1)) < 1.0) ? g1 : g2;
  }
  return (g1.im < g2.im) ? g1 : g2;
}

// self-energy of angular mode j of a lead at device energy eps (Im eps > 0)
__device__ __forceinline__ cd mode_sigma(const LeadView& L, int j, cd eps) {
  cd e = mk(eps.re - L.U, eps.im);
  return scale(surface_gf(e, L.a1[j], L.a2[j]), L.at[j]);
}

}  // namespace negf
