// Enrichment-function evaluation shared by the host set-up and the device
// kernels of the library (value and gradient of one cut-off orbital).
//
// Paper, Sec. IV.A (Eqs. KSOrbitalSplit, EnrichedPsi): N_alpha = R_nl(r) Y_lm,
// written here as q(r) h(r) P_lm(x - R) with q = R / r^l and P_lm = r^l Y_lm
// the real solid harmonic; Sec. IV.B (Eq. Moll1): h(r~) = u(r~)/(u(r~)+u(1-r~)),
// u(s) = exp(-1/s) for s > 0, r~ = 1 - t (r - r0)/r0.
#pragma once

#include <math.h>

#include "efe_internal.h"

#ifdef __CUDACC__
#define EFE_HD __host__ __device__ __forceinline__
#else
#define EFE_HD inline
#endif

namespace efe {

EFE_HD double cutoff_u(double s) { return s > 0.0 ? exp(-1.0 / s) : 0.0; }
EFE_HD double cutoff_du(double s) { return s > 0.0 ? exp(-1.0 / s) / (s * s) : 0.0; }

// h(r) and dh/dr of Eq. Moll1
EFE_HD void cutoff_h(double r, double r0, double t, double* h, double* dh) {
  double rt = 1.0 - t * (r - r0) / r0;
  double a = cutoff_u(rt), b = cutoff_u(1.0 - rt);
  double den = a + b;
  *h = a / den;
  *dh = (cutoff_du(rt) * b + a * cutoff_du(1.0 - rt)) / (den * den) * (-t / r0);
}

// q(r) = R(r)/r^l and dq/dr
EFE_HD void radial_q(const DevFunc& f, double r, double* q, double* dq) {
  if (f.kind == 0) {  // hydrogenic, f.zeta holds Z, f.norm the constant in front
    const double Z = f.zeta;
    if (f.n == 1) {
      double v = f.norm * exp(-Z * r);
      *q = v;
      *dq = -Z * v;
    } else if (f.l == 0) {
      double e = exp(-0.5 * Z * r);
      *q = f.norm * (2.0 - Z * r) * e;
      *dq = f.norm * e * (0.5 * Z * Z * r - 2.0 * Z);
    } else {
      double v = f.norm * exp(-0.5 * Z * r);
      *q = v;
      *dq = -0.5 * Z * v;
    }
  } else {  // Slater: norm r^k exp(-zeta r), k = n - 1 - l
    const int k = f.n - 1 - f.l;
    double e = f.norm * exp(-f.zeta * r);
    double rk = 1.0, rk1 = 0.0;
    for (int i = 0; i < k; ++i) { rk1 = (i == 0) ? 1.0 : rk1 * r; rk *= r; }
    *q = rk * e;
    *dq = e * ((k > 0 ? k * rk1 : 0.0) - f.zeta * rk);
  }
}

// value and gradient of the cut-off enrichment function at (x, y, z)
EFE_HD void eval_func(const DevFunc& f, double x, double y, double z, double* val, double* grad) {
  const double dx = x - f.Rx, dy = y - f.Ry, dz = z - f.Rz;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double q, dq, h, dh;
  radial_q(f, r, &q, &dq);
  cutoff_h(r, f.r0, f.t, &h, &dh);
  double P, dP[3] = {0.0, 0.0, 0.0};
  if (f.l == 0) {
    P = 0.28209479177387814;  // 1/sqrt(4 pi)
  } else {
    const double c = 0.48860251190291992;  // sqrt(3/(4 pi))
    const int ax = (f.m == -1) ? 1 : (f.m == 0 ? 2 : 0);
    P = c * (ax == 0 ? dx : (ax == 1 ? dy : dz));
    dP[ax] = c;
  }
  const double qh = q * h;
  const double dqh = dq * h + q * dh;
  *val = qh * P;
  if (grad) {
    const double s = (r > 0.0) ? dqh * P / r : 0.0;
    grad[0] = s * dx + qh * dP[0];
    grad[1] = s * dy + qh * dP[1];
    grad[2] = s * dz + qh * dP[2];
  }
}

// value only
EFE_HD double eval_func_value(const DevFunc& f, double x, double y, double z) {
  double v;
  eval_func(f, x, y, z, &v, nullptr);
  return v;
}

}  // namespace efe
