// sin and cos in FP64 for turning and pulsating shapes (moving-body kernels of 2D and 3D).
#pragma once

namespace lbm {

// sin t and cos t in FP64 with explicitly rounded operations, so that a turned shape is
// placed by the same operations on every device and on the host: t is reduced by
// k = rint(2 t / pi) multiples of pi/2 (Cody and Waite's reduction, pi/2 split in three
// parts whose first two have 30 significant bits: k times them is exact for |k| < 2^23),
// then sin r and cos r on [-pi/4, pi/4] are their Taylor series to r^17 and r^16 by
// Horner's rule in r^2, and k mod 4 picks signs and roles.
__device__ __forceinline__ void turn_sincos(double t, double &sn, double &cs) {
  constexpr double P1 = 0x1.921fb54p+0, P2 = 0x1.10b46118p-30, P3 = 0x1.313198a2e037p-61;
  const double k = rint(__dmul_rn(t, 0x1.45f306dc9c883p-1));
  const double r = __dsub_rn(__dsub_rn(__dsub_rn(t, __dmul_rn(k, P1)), __dmul_rn(k, P2)), __dmul_rn(k, P3));
  const double r2 = __dmul_rn(r, r);
  double ps = __dadd_rn(-1.0 / 1307674368000.0, __dmul_rn(r2, 1.0 / 355687428096000.0));
  ps = __dadd_rn(1.0 / 6227020800.0, __dmul_rn(r2, ps));
  ps = __dadd_rn(-1.0 / 39916800.0, __dmul_rn(r2, ps));
  ps = __dadd_rn(1.0 / 362880.0, __dmul_rn(r2, ps));
  ps = __dadd_rn(-1.0 / 5040.0, __dmul_rn(r2, ps));
  ps = __dadd_rn(1.0 / 120.0, __dmul_rn(r2, ps));
  ps = __dadd_rn(-1.0 / 6.0, __dmul_rn(r2, ps));
  const double sr = __dadd_rn(r, __dmul_rn(__dmul_rn(r, r2), ps));
  double pc = __dadd_rn(-1.0 / 87178291200.0, __dmul_rn(r2, 1.0 / 20922789888000.0));
  pc = __dadd_rn(1.0 / 479001600.0, __dmul_rn(r2, pc));
  pc = __dadd_rn(-1.0 / 3628800.0, __dmul_rn(r2, pc));
  pc = __dadd_rn(1.0 / 40320.0, __dmul_rn(r2, pc));
  pc = __dadd_rn(-1.0 / 720.0, __dmul_rn(r2, pc));
  pc = __dadd_rn(1.0 / 24.0, __dmul_rn(r2, pc));
  pc = __dadd_rn(-0.5, __dmul_rn(r2, pc));
  const double cr = __dadd_rn(1.0, __dmul_rn(r2, pc));
  switch (static_cast<int>(static_cast<long long>(k) & 3)) {
    case 0: sn = sr; cs = cr; break;
    case 1: sn = cr; cs = -sr; break;
    case 2: sn = -sr; cs = -cr; break;
    default: sn = -cr; cs = sr; break;
  }
}

}  // namespace lbm
