// Reverse-mode building blocks shared by the adjoint kernels (qed_adj.cu on
// the node-reduced DAG, qed_radj.cu on the rewritten one): the real parts of
// the Dirac bilinears that the propagator and polarisation parameter terms
// need, and the derivative of the linear polarisation vectors.
#pragma once

#include <cuda_runtime.h>

namespace qed {
namespace adjb {

// Real parts of the bilinears s_mu = sum_ab a_a gamma^mu_ab b_b (mu = 0..3,
// Dirac representation) and u = sum_c a_c b_c, for complex 4-vectors a, b
// stored as 8 reals.  Q, D and eps are real, so df = 2 Re(...) needs only
// these.  Each is one FMA chain over its four products:
//   gamma^0 = diag(1, 1, -1, -1):             s_0 = a0 b0 + a1 b1 - a2 b2 - a3 b3
//   gamma^i = [[0, sigma^i], [-sigma^i, 0]]:  s_i = a_u sigma^i b_l - a_l sigma^i b_u
//     x sigma^1 y = x0 y1 + x1 y0   ->  s_1 = a0 b3 + a1 b2 - a2 b1 - a3 b0
//     x sigma^2 y = i (x1 y0 - x0 y1) -> Re s_2 = Im(a0 b3 - a1 b2 + a3 b0 - a2 b1)
//     x sigma^3 y = x0 y0 - x1 y1   ->  s_3 = a0 b2 - a1 b3 - a2 b0 + a3 b1
// acc + g Re(a_i b_j) and acc + g Im(a_i b_j), g = +-1
template <typename Real>
__device__ __forceinline__ Real fre(const Real* a, int i, const Real* b, int j, Real g, Real acc) {
  return fma(g * a[2 * i], b[2 * j], fma(-g * a[2 * i + 1], b[2 * j + 1], acc));
}
template <typename Real>
__device__ __forceinline__ Real fim(const Real* a, int i, const Real* b, int j, Real g, Real acc) {
  return fma(g * a[2 * i], b[2 * j + 1], fma(g * a[2 * i + 1], b[2 * j], acc));
}

template <typename Real>
__device__ __forceinline__ Real bil_s0(const Real* a, const Real* b) {
  const Real one = 1, mone = -1;
  return fre(a, 3, b, 3, mone, fre(a, 2, b, 2, mone, fre(a, 1, b, 1, one, fre(a, 0, b, 0, one, (Real)0))));
}
template <typename Real>
__device__ __forceinline__ Real bil_s1(const Real* a, const Real* b) {
  const Real one = 1, mone = -1;
  return fre(a, 3, b, 0, mone, fre(a, 2, b, 1, mone, fre(a, 1, b, 2, one, fre(a, 0, b, 3, one, (Real)0))));
}
template <typename Real>
__device__ __forceinline__ Real bil_s2(const Real* a, const Real* b) {
  const Real one = 1, mone = -1;
  return fim(a, 2, b, 1, mone, fim(a, 3, b, 0, one, fim(a, 1, b, 2, mone, fim(a, 0, b, 3, one, (Real)0))));
}
template <typename Real>
__device__ __forceinline__ Real bil_s3(const Real* a, const Real* b) {
  const Real one = 1, mone = -1;
  return fre(a, 3, b, 1, one, fre(a, 2, b, 0, mone, fre(a, 1, b, 3, mone, fre(a, 0, b, 2, one, (Real)0))));
}
template <typename Real>
__device__ __forceinline__ Real bil_u(const Real* a, const Real* b) {
  const Real one = 1;
  return fre(a, 3, b, 3, one, fre(a, 2, b, 2, one, fre(a, 1, b, 1, one, fre(a, 0, b, 0, one, (Real)0))));
}

// d eps_pol / d k_a (a = x, y, z) for the real linear polarisations, in
// precision T (the momentum is FP64); zero on the z axis, where the basis is
// fixed by convention.
template <typename T>
__device__ __forceinline__ void dpol(const double* k, int pbit, T d[3][3]) {
  const T kx = (T)k[1], ky = (T)k[2], kz = (T)k[3];
  const T kt2 = kx * kx + ky * ky;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) d[a][i] = (T)0;
  if (kt2 == (T)0) return;
  const T kt = sqrt(kt2);
  if (pbit) {
    // eps_2 = (-ky, kx, 0) / kT
    const T c = (T)1 / (kt2 * kt);
    d[0][0] = kx * ky * c; d[0][1] = ky * ky * c;
    d[1][0] = -kx * kx * c; d[1][1] = -kx * ky * c;
    return;
  }
  // eps_1 = g (kx kz, ky kz, -kT^2), g = 1 / (K kT)
  const T K2 = kt2 + kz * kz;
  const T K = sqrt(K2);
  const T g = (T)1 / (K * kt);
  const T num[3] = {kx * kz, ky * kz, -kt2};
  const T dg[3] = {-g * (kx / K2 + kx / kt2), -g * (ky / K2 + ky / kt2), -g * kz / K2};
  const T dn[3][3] = {{kz, (T)0, (T)-2 * kx}, {(T)0, kz, (T)-2 * ky}, {kx, ky, (T)0}};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) d[a][i] = g * dn[a][i] + num[i] * dg[a];
}

}  // namespace adjb
}  // namespace qed
