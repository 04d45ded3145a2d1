// Model pieces shared by the host tables and the node-table kernel: an FP64
// complex number and the Fresnel transmission coefficients of Eq. 7.
#pragma once

#include <math.h>

#ifndef PSF_HD
#define PSF_HD __host__ __device__ __forceinline__
#endif

namespace psf {

struct dcplx {
  double re, im;
};
PSF_HD dcplx operator+(dcplx a, dcplx b) { return {a.re + b.re, a.im + b.im}; }
PSF_HD dcplx operator-(dcplx a, dcplx b) { return {a.re - b.re, a.im - b.im}; }
PSF_HD dcplx operator*(dcplx a, dcplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
PSF_HD dcplx operator*(double s, dcplx a) { return {s * a.re, s * a.im}; }
PSF_HD dcplx operator/(dcplx a, dcplx b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// cos(theta_m) in medium m for the immersion-side sin(theta): by Snell's law
// n_m sin(theta_m) = n_i sin(theta), principal root (purely imaginary with
// Im >= 0 where the medium is evanescent).
PSF_HD dcplx cos_in_medium(double n_m, double n_i, double sin_t) {
  const double r = n_i * sin_t / n_m;
  const double arg = 1.0 - r * r;
  return arg >= 0.0 ? dcplx{sqrt(arg), 0.0} : dcplx{0.0, sqrt(-arg)};
}

// q_s, q_p of Eq. 7: products over sample -> coverslip -> immersion of
//   q_s^m = 2 n_m c_m / (n_m c_m + n_{m+1} c_{m+1}),
//   q_p^m = 2 n_m c_m / (n_{m+1} c_m + n_m c_{m+1}).
PSF_HD void fresnel_q(double n_s, double n_g, double n_i, double sin_t, dcplx& qs,
                      dcplx& qp) {
  const double n[3] = {n_s, n_g, n_i};
  dcplx c[3];
  for (int m = 0; m < 3; ++m) c[m] = cos_in_medium(n[m], n_i, sin_t);
  qs = {1.0, 0.0};
  qp = {1.0, 0.0};
  for (int m = 0; m < 2; ++m) {
    const dcplx num = (2.0 * n[m]) * c[m];
    qs = qs * (num / (n[m] * c[m] + n[m + 1] * c[m + 1]));
    qp = qp * (num / (n[m + 1] * c[m] + n[m] * c[m + 1]));
  }
}

}  // namespace psf
