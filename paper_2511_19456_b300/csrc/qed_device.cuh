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
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
// 1/sqrt(x): CUDA's rsqrt (1 ulp in FP64) and rsqrtf (2 ulp)
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// Helicity spinor u(p, h) in precision T:
// u = (sqrt(E+m) chi, h sqrt(E-m) chi), chi_+ = (|p|+pz, px + i py)/N,
// chi_- = (-px + i py, |p|+pz)/N, N = sqrt(2|p|(|p|+pz)); |p| = 0 uses the
// z axis, |p|+pz = 0 gives chi_+ = (0, 1), chi_- = (-1, 0).
// bar: ubar = u^dagger gamma^0.  In FP32, |p|+pz is formed as
// (px^2 + py^2)/(|p| - pz) when pz < 0 (the same quantity without the
// cancellation near the -z axis).  make_spinor_core takes px, py, pz and
// E + m, E - m already in precision T; make_spinor forms them from the FP64
// momentum (E +- m in FP64).  Both helicities take the same three quotients
// by N (in FP64 through one reciprocal square root), so that the lanes of a
// warp that build the two helicities run the same instructions; in FP32 the
// quotients are IEEE divisions by the rounded N.
template <typename T>
__device__ __forceinline__ void make_spinor_core(T px, T py, T pz, T epm, T emm, int hbit, bool bar, T out[8]) {
  const T pt2 = px * px + py * py;
  const T ap = sqrt_t(pt2 + pz * pz);
  T c0r, c0i, c1r, c1i;
  if (ap == (T)0) {
    c0r = hbit ? (T)0 : (T)1; c0i = (T)0; c1r = hbit ? (T)1 : (T)0; c1i = (T)0;
  } else {
    T apz;
    if constexpr (sizeof(T) == 8) apz = ap + pz;
    else apz = pz >= (T)0 ? ap + pz : pt2 / (ap - pz);
    if (apz == (T)0) {
      c0r = hbit ? (T)-1 : (T)0; c0i = (T)0; c1r = hbit ? (T)0 : (T)1; c1i = (T)0;
    } else {
      T za, zx, zy;
      if constexpr (sizeof(T) == 8) {
        const T inv = rsqrt_t((T)2 * ap * apz);
        za = apz * inv; zx = px * inv; zy = py * inv;
      } else {
        const T nrm = sqrt_t((T)2 * ap * apz);
        za = apz / nrm; zx = px / nrm; zy = py / nrm;
      }
      c0r = hbit ? -zx : za;
      c0i = hbit ? zy : (T)0;
      c1r = hbit ? za : zx;
      c1i = hbit ? (T)0 : zy;
    }
  }
  const T a = sqrt_t(epm);
  const T bb = emm;
  T b = bb > (T)0 ? sqrt_t(bb) : (T)0;
  if (hbit) b = -b;
  const T u[8] = {a * c0r, a * c0i, a * c1r, a * c1i, b * c0r, b * c0i, b * c1r, b * c1i};
  if (!bar) {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = u[i];
  } else {
    // conjugate, then flip the lower two components (gamma^0)
    out[0] = u[0]; out[1] = -u[1]; out[2] = u[2]; out[3] = -u[3];
    out[4] = -u[4]; out[5] = u[5]; out[6] = -u[6]; out[7] = u[7];
  }
}
template <typename T>
__device__ __forceinline__ void make_spinor(const double* p, int hbit, double m, bool bar, T out[8]) {
  make_spinor_core<T>((T)p[1], (T)p[2], (T)p[3], (T)(p[0] + m), (T)(p[0] - m), hbit, bar, out);
}

// Real linear polarisation 3-vector (eps^0 = 0) of a photon with momentum
// components (kx, ky, kz) in precision T:
//   eps_1 = (kx kz, ky kz, -kt^2) / (|k| kt),  eps_2 = (-ky, kx, 0) / kt,
// kt^2 = kx^2 + ky^2; both polarisations run the same instructions (in FP64
// 1/kt and 1/|k| as reciprocal square roots; in FP32 IEEE divisions by the
// rounded kt and |k| kt).
template <typename T>
__device__ __forceinline__ void make_pol_core(T kx, T ky, T kz, int pbit, T e[3]) {
  const T kt2 = kx * kx + ky * ky;
  if (kt2 == (T)0) {
    e[0] = pbit ? (T)0 : (T)1; e[1] = pbit ? (T)1 : (T)0; e[2] = (T)0;
    return;
  }
  T e1[3], e2[2];
  if constexpr (sizeof(T) == 8) {
    const T ikt = rsqrt_t(kt2);
    const T inv = rsqrt_t(kt2 + kz * kz) * ikt;   // 1 / (|k| kt)
    e1[0] = kx * kz * inv; e1[1] = ky * kz * inv; e1[2] = -kt2 * inv;
    e2[0] = -ky * ikt; e2[1] = kx * ikt;
  } else {
    const T kt = sqrt_t(kt2);
    const T den = sqrt_t(kt2 + kz * kz) * kt;
    e1[0] = kx * kz / den; e1[1] = ky * kz / den; e1[2] = -kt2 / den;
    e2[0] = -ky / kt; e2[1] = kx / kt;
  }
  e[0] = pbit ? e2[0] : e1[0];
  e[1] = pbit ? e2[1] : e1[1];
  e[2] = pbit ? (T)0 : e1[2];
}
// ... of a photon with FP64 momentum k.
template <typename T>
__device__ __forceinline__ void make_pol(const double* k, int pbit, T e[3]) {
  make_pol_core<T>((T)k[1], (T)k[2], (T)k[3], pbit, e);
}

// Propagator of the line carrying photon set `mask`: Q = p + sum c_j k_j
// over the set in ascending slot order, D = Q0^2 - Qx^2 - Qy^2 - Qz^2 - m^2
// with every product rounded separately, all in FP64.  Writes (Q0+m)/D,
// (Q0-m)/D, Q/D in precision T (for T = float the quotients are formed in
// FP32 from the FP64 numerators and denominator).
template <typename T>
__device__ __forceinline__ void make_prop(const double* mom, int n, unsigned mask, double m, T out[5]) {
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
  if constexpr (sizeof(T) == 8) {
    const double inv = 1.0 / D;
    out[0] = (q0 + m) * inv;
    out[1] = (q0 - m) * inv;
    out[2] = q1 * inv;
    out[3] = q2 * inv;
    out[4] = q3 * inv;
  } else {
    const float inv = 1.0f / (float)D;
    out[0] = (float)(q0 + m) * inv;
    out[1] = (float)(q0 - m) * inv;
    out[2] = (float)q1 * inv;
    out[3] = (float)q2 * inv;
    out[4] = (float)q3 * inv;
  }
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

// -(sigma . a) x and -x (sigma . a): the same products with the sign on the
// coefficients, so that it costs no separate negation (exact either way).
template <typename R>
QED_HD void pauli_col_neg(const R a[3], const R x[4], R y[4]) {
  y[0] = -a[2] * x[0] - a[0] * x[2] - a[1] * x[3];
  y[1] = -a[2] * x[1] - a[0] * x[3] + a[1] * x[2];
  y[2] = -a[0] * x[0] + a[1] * x[1] + a[2] * x[2];
  y[3] = -a[0] * x[1] - a[1] * x[0] + a[2] * x[3];
}
template <typename R>
QED_HD void pauli_row_neg(const R a[3], const R x[4], R y[4]) {
  y[0] = -a[2] * x[0] - a[0] * x[2] + a[1] * x[3];
  y[1] = -a[2] * x[1] - a[0] * x[3] - a[1] * x[2];
  y[2] = -a[0] * x[0] - a[1] * x[1] + a[2] * x[2];
  y[3] = -a[0] * x[1] + a[1] * x[0] + a[2] * x[3];
}

// eps/ = -gamma.eps (eps^0 = 0) = [[0, -s.e], [s.e, 0]]
template <typename R>
QED_HD void vertex_col(const R e[3], const R x[8], R y[8]) {
  pauli_col_neg(e, x + 4, y);       // upper = -(s.e) x_lower
  pauli_col(e, x, y + 4);           // lower = (s.e) x_upper
}
template <typename R>
QED_HD void vertex_row(const R e[3], const R x[8], R y[8]) {
  pauli_row(e, x + 4, y);           // upper = x_lower (s.e)
  pauli_row_neg(e, x, y + 4);       // lower = -x_upper (s.e)
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

// Error-free FP32 transformations (Knuth TwoSum; TwoProd through fma).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// E + m and E - m from the float-float energy (hi, lo) and the FP32 mass:
// TwoSum of the high parts, then the low parts added to its error, so that
// each is rounded about once (where E is close to m, hi - m is exact).
__device__ __forceinline__ void e_pm_m_ff(float hi, float lo, float m, float& epm, float& emm) {
  float s, e;
  two_sum_f(hi, m, s, e);
  epm = __fadd_rn(s, __fadd_rn(e, lo));
  two_sum_f(hi, -m, s, e);
  emm = __fadd_rn(s, __fadd_rn(e, lo));
}

// Adds (hi - c)^2 to the float-float accumulator (acc_hi, acc_lo); hi - c is a
// Kahan-compensated value with |c| far below ulp(hi).
__device__ __forceinline__ void add_square_ff(float hi, float c, float& acc_hi, float& acc_lo) {
  const float p = __fmul_rn(hi, hi);
  const float e = __fmaf_rn(hi, hi, -p);           // hi^2 = p + e exactly
  const float t = __fmaf_rn(-2.0f * hi, c, e);     // + 2 hi (-c); c^2 is below rounding
  float s, err;
  two_sum_f(acc_hi, p, s, err);
  acc_hi = s;
  acc_lo = __fadd_rn(acc_lo, __fadd_rn(err, t));
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
