// Device building blocks of the |M|^2 kernels: external states (paper task
// U), the vertex eps/ (task V), the propagator (Q/ + m)/D (task S1 and the
// propagation half of S2) and the join dot product (the product half of S2),
// in the Dirac representation with metric (+,-,-,-).
//
// A current is a 4-component complex spinor stored as 8 reals
// (re0, im0, re1, im1, re2, im2, re3, im3).  Column currents grow from u(p),
// row currents from ubar(p').
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qed_types.h"

namespace qed {

// ------------------------------------------------------------ U: states
// Helicity spinor u(p, h) (FP64): u = (sqrt(E+m) chi, h sqrt(E-m) chi), with
// chi_+ = (|p|+pz, px + i py)/sqrt(2|p|(|p|+pz)), chi_- = (-px + i py,
// |p|+pz)/sqrt(2|p|(|p|+pz)); |p| = 0 uses the z axis, |p|+pz = 0 gives
// chi_+ = (0, 1), chi_- = (-1, 0).  bar: ubar = u^dagger gamma^0.
__device__ __forceinline__ void make_spinor(const double* p, int hbit, double m, bool bar,
                                            double out[8]) {
  const double px = p[1], py = p[2], pz = p[3];
  const double ap = sqrt(px * px + py * py + pz * pz);
  double c0r, c0i, c1r, c1i;
  if (ap == 0.0) {
    c0r = hbit ? 0.0 : 1.0; c0i = 0.0; c1r = hbit ? 1.0 : 0.0; c1i = 0.0;
  } else {
    const double apz = ap + pz;
    if (apz == 0.0) {
      c0r = hbit ? -1.0 : 0.0; c0i = 0.0; c1r = hbit ? 0.0 : 1.0; c1i = 0.0;
    } else {
      const double nrm = sqrt(2.0 * ap * apz);
      if (!hbit) { c0r = apz / nrm; c0i = 0.0; c1r = px / nrm; c1i = py / nrm; }
      else       { c0r = -px / nrm; c0i = py / nrm; c1r = apz / nrm; c1i = 0.0; }
    }
  }
  const double a = sqrt(p[0] + m);
  const double bb = p[0] - m;
  double b = bb > 0.0 ? sqrt(bb) : 0.0;
  if (hbit) b = -b;
  double u[8] = {a * c0r, a * c0i, a * c1r, a * c1i, b * c0r, b * c0i, b * c1r, b * c1i};
  if (!bar) {
    for (int i = 0; i < 8; ++i) out[i] = u[i];
  } else {
    // conjugate, then flip the lower two components (gamma^0)
    out[0] = u[0]; out[1] = -u[1]; out[2] = u[2]; out[3] = -u[3];
    out[4] = -u[4]; out[5] = u[5]; out[6] = -u[6]; out[7] = u[7];
  }
}

// Real linear polarisation 3-vector (eps^0 = 0) of a photon with momentum k.
__device__ __forceinline__ void make_pol(const double* k, int pbit, double e[3]) {
  const double kx = k[1], ky = k[2], kz = k[3];
  const double kt2 = kx * kx + ky * ky;
  if (kt2 == 0.0) {
    e[0] = pbit ? 0.0 : 1.0; e[1] = pbit ? 1.0 : 0.0; e[2] = 0.0;
    return;
  }
  const double kt = sqrt(kt2);
  if (!pbit) {
    const double den = sqrt(kt2 + kz * kz) * kt;
    e[0] = kx * kz / den; e[1] = ky * kz / den; e[2] = -kt2 / den;
  } else {
    e[0] = -ky / kt; e[1] = kx / kt; e[2] = 0.0;
  }
}

// Propagator of the line carrying photon set `mask`: Q = p + sum c_j k_j
// over the set in ascending slot order, D = Q0^2 - Qx^2 - Qy^2 - Qz^2 - m^2
// with every product rounded separately.  Writes (Q0+m)/D, (Q0-m)/D, Q/D.
__device__ __forceinline__ void make_prop(const double* mom, int n, unsigned mask, double m,
                                          double out[5]) {
  double q0 = mom[0], q1 = mom[1], q2 = mom[2], q3 = mom[3];
  for (int j = 0; j < n; ++j) {
    if (!(mask & (1u << j))) continue;
    const double* kj = mom + 4 * (j == 0 ? 1 : j + 2);
    if (j == 0) { q0 += kj[0]; q1 += kj[1]; q2 += kj[2]; q3 += kj[3]; }
    else        { q0 -= kj[0]; q1 -= kj[1]; q2 -= kj[2]; q3 -= kj[3]; }
  }
  double D = __dmul_rn(q0, q0);
  D = __dsub_rn(D, __dmul_rn(q1, q1));
  D = __dsub_rn(D, __dmul_rn(q2, q2));
  D = __dsub_rn(D, __dmul_rn(q3, q3));
  D = __dsub_rn(D, __dmul_rn(m, m));
  const double inv = 1.0 / D;
  out[0] = (q0 + m) * inv;
  out[1] = (q0 - m) * inv;
  out[2] = q1 * inv;
  out[3] = q2 * inv;
  out[4] = q3 * inv;
}

// ------------------------------------------------- 2x2 Pauli products
// (sigma . a) x for a real 3-vector a and a complex 2-vector x, column form.
template <typename R>
QED_HD void pauli_col(const R a[3], const R x[4], R y[4]) {
  // y0 = az x0 + (ax - i ay) x1 ; y1 = (ax + i ay) x0 - az x1
  y[0] = a[2] * x[0] + a[0] * x[2] + a[1] * x[3];
  y[1] = a[2] * x[1] + a[0] * x[3] - a[1] * x[2];
  y[2] = a[0] * x[0] - a[1] * x[1] - a[2] * x[2];
  y[3] = a[0] * x[1] + a[1] * x[0] - a[2] * x[3];
}
// x (sigma . a), row form.
template <typename R>
QED_HD void pauli_row(const R a[3], const R x[4], R y[4]) {
  // y0 = x0 az + x1 (ax + i ay) ; y1 = x0 (ax - i ay) - x1 az
  y[0] = a[2] * x[0] + a[0] * x[2] - a[1] * x[3];
  y[1] = a[2] * x[1] + a[0] * x[3] + a[1] * x[2];
  y[2] = a[0] * x[0] + a[1] * x[1] - a[2] * x[2];
  y[3] = a[0] * x[1] - a[1] * x[0] - a[2] * x[3];
}

// eps/ = -gamma.eps (eps^0 = 0) = [[0, -s.e], [s.e, 0]]
template <typename R>
QED_HD void vertex_col(const R e[3], const R x[8], R y[8]) {
  R t[4];
  pauli_col(e, x + 4, t);           // upper = -(s.e) x_lower
  y[0] = -t[0]; y[1] = -t[1]; y[2] = -t[2]; y[3] = -t[3];
  pauli_col(e, x, y + 4);           // lower = (s.e) x_upper
}
template <typename R>
QED_HD void vertex_row(const R e[3], const R x[8], R y[8]) {
  pauli_row(e, x + 4, y);           // upper = x_lower (s.e)
  R t[4];
  pauli_row(e, x, t);               // lower = -x_upper (s.e)
  y[4] = -t[0]; y[5] = -t[1]; y[6] = -t[2]; y[7] = -t[3];
}

// (Q/ + m)/D = [[A, -s.q], [s.q, -B]], A = (Q0+m)/D, B = (Q0-m)/D, q = Q/D
template <typename R>
QED_HD void prop_col(const R* P, const R x[8], R y[8]) {
  const R A = P[0], B = P[1];
  R t[4], s[4];
  pauli_col(P + 2, x + 4, t);
  pauli_col(P + 2, x, s);
  y[0] = A * x[0] - t[0]; y[1] = A * x[1] - t[1]; y[2] = A * x[2] - t[2]; y[3] = A * x[3] - t[3];
  y[4] = s[0] - B * x[4]; y[5] = s[1] - B * x[5]; y[6] = s[2] - B * x[6]; y[7] = s[3] - B * x[7];
}
template <typename R>
QED_HD void prop_row(const R* P, const R x[8], R y[8]) {
  const R A = P[0], B = P[1];
  R t[4], s[4];
  pauli_row(P + 2, x + 4, t);       // x_lower (s.q)
  pauli_row(P + 2, x, s);           // x_upper (s.q)
  y[0] = A * x[0] + t[0]; y[1] = A * x[1] + t[1]; y[2] = A * x[2] + t[2]; y[3] = A * x[3] + t[3];
  y[4] = -s[0] - B * x[4]; y[5] = -s[1] - B * x[5]; y[6] = -s[2] - B * x[6]; y[7] = -s[3] - B * x[7];
}

// acc += sum_c R_c L_c (complex, no conjugation)
template <typename R>
QED_HD void dot_acc(const R* Rw, const R* Lc, R& re, R& im) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    re = fma(Rw[2 * c], Lc[2 * c], re);
    re = fma(-Rw[2 * c + 1], Lc[2 * c + 1], re);
    im = fma(Rw[2 * c], Lc[2 * c + 1], im);
    im = fma(Rw[2 * c + 1], Lc[2 * c], im);
  }
}

// Kahan-compensated add of x into (s, c); the represented value is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// pext: gather the bits of v selected by mask into the low bits.
QED_HD unsigned pext_bits(unsigned v, unsigned mask, int n) {
  unsigned r = 0;
  int o = 0;
  for (int j = 0; j < n; ++j)
    if (mask & (1u << j)) { r |= ((v >> j) & 1u) << o; ++o; }
  return r;
}

}  // namespace qed
