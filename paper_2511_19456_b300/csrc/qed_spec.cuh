// Device building blocks of the specialised forward kernels that the DAG
// builder emits at build time (qed_codegen.cpp writes them as straight-line
// code, one kernel per k and precision, spin-summed).
//
// The generated code calls these helpers with every schedule quantity as a
// literal: the photon of a vertex, the rank of its polarisation bit, the
// source and destination currents and the propagator's photon set.  After
// inlining, a vertex (+ propagation) item is its arithmetic plus one load of
// its input, one of its polarisation vector, the propagator entries and two
// stores; nothing is decoded at run time.
//
// Leaf layout.  The leaves of one photon set (the inputs of the S2 joins) are
// stored by chunk: a chunk is 4 reals, components (0, 1) or (2, 3) of one
// current as (re, im) pairs.  Chunk q of leaf a in spin variant (p, s) sits at
//   ((a * 2 + q) * 2 + s) * NP + p,
// with s the electron-helicity bit, p the polarisation pattern of the set's
// photons and NP the number of patterns.  The lanes of a join read one
// pattern each (their own polarisations of the set), so one load of the team
// touches consecutive chunks: no bank conflicts.
#pragma once

#include "qed_team.cuh"

namespace qed {
namespace spec {

// Operands of one photon set S in a specialised kernel's loop over the sets
// (a constant table the generator writes): S and its complement, and for
// each position of the set's sorted left (NL) and right (NR) leaf lists the
// vertex photon and the input current.
template <int NL, int NR>
struct SetTable {
  int mask, comp;
  int lph[NL], lsrc[NL];
  int rph[NR], rsrc[NR];
};

// The bits of lane selected by MASK, packed into the low bits (photon j's
// polarisation is bit j of a spin-summed team's lane).
template <unsigned MASK>
__device__ __forceinline__ int pext_lane(int lane) {
  int r = 0, o = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (MASK & (1u << j)) { r |= ((lane >> j) & 1) << o; ++o; }
  return r;
}

// Spin variant v of a current without the polarisation bit of the photon of
// rank RANK in its set (bit 0 is the electron helicity): the variant of the
// vertex's input current.
template <int RANK>
__device__ __forceinline__ int drop_pol_bit(int v) {
  constexpr int b = 1 + RANK;
  return (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b);
}

__device__ __forceinline__ void ld8(const float* p, float x[8]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void ld8(const double* p, double x[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = reinterpret_cast<const double2*>(p)[i];
    x[2 * i] = a.x; x[2 * i + 1] = a.y;
  }
}
// Four reals (one chunk) to a 16-byte (float) or 32-byte (double) aligned address.
__device__ __forceinline__ void st4(float* d, const float* x) {
  *reinterpret_cast<float4*>(d) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st4(double* d, const double* x) {
  reinterpret_cast<double2*>(d)[0] = make_double2(x[0], x[1]);
  reinterpret_cast<double2*>(d)[1] = make_double2(x[2], x[3]);
}
// One chunk (4 reals) from shared memory.
__device__ __forceinline__ void ld4(const double* s, double x[4]) {
  const double2 a = reinterpret_cast<const double2*>(s)[0], b = reinterpret_cast<const double2*>(s)[1];
  x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ __forceinline__ void ld3(const float* e, float ev[3]) {
  const float4 a = *reinterpret_cast<const float4*>(e);
  ev[0] = a.x; ev[1] = a.y; ev[2] = a.z;
}
__device__ __forceinline__ void ld3(const double* e, double ev[3]) {
  const double2 a = reinterpret_cast<const double2*>(e)[0];
  ev[0] = a.x; ev[1] = a.y; ev[2] = e[2];
}

// One vertex item (task V), optionally followed by its propagation (task S1,
// or the propagation half of S2 that is hoisted onto a right leaf):
//   side 0 (column current):  z = [S(Q)] eps/ x
//   side 1 (row current):     z = x eps/ [S(Q)]
// x: the input current (8 reals), e: the polarisation vector, P: the
// propagator entries (Q0+m)/D, (Q0-m)/D, Q/D of the line (POST only).  The
// two chunks of z go to d0 (components 0, 1) and d1 (components 2, 3).
template <typename Real, int SIDE, bool POST>
__device__ __forceinline__ void vs_item(const Real* xs, const Real* e, const Real* P, Real* d0, Real* d1) {
  Real x[8], ev[3], y[8];
  ld8(xs, x);
  ld3(e, ev);
  if constexpr (SIDE == 0) vertex_col(ev, x, y); else vertex_row(ev, x, y);
  if constexpr (POST) {
    Real z[8];
    if constexpr (SIDE == 0) prop_col(P, y, z); else prop_row(P, y, z);
    st4(d0, z);
    st4(d1, z + 4);
  } else {
    st4(d0, y);
    st4(d1, y + 4);
  }
}

// The S2 joins of one photon set for one lane, FP32 (task S2's product half
// and task Sum): for each of the lane's 2 x 2 electron-helicity states
// (s_in, s_out) and every pair of a left leaf a (NL) and a right leaf b (NR),
//   M[s_in][s_out] += sum_c R_b[s_out]_c L_a[s_in]_c   (complex, unconjugated),
// added to the compensated accumulators in one compensated step per state.
// L, R: the chunk of leaf 0, q = 0, s = 0 in this lane's polarisation pattern
// (leaf layout above; NPL, NPR patterns).
//
// Packed FP32 FMAs (two lanes of arithmetic per instruction): with
// L_c = (lr, li) and R_c = (rr, ri),
//   A += (lr, lr) * (rr, ri),  B += (li, li) * (rr, ri)
// so that A = (sum lr rr, sum lr ri), B = (sum li rr, sum li ri) and
//   Re M = A.x - B.y,  Im M = A.y + B.x.
// A starts from minus the accumulator's compensation (the first step of the
// Kahan update), B from zero.
template <int NL, int NR, int NPL, int NPR>
__device__ __forceinline__ void join_set_f32(const float4* L, const float4* R, Acc<float> acc[4]) {
  float2 r[NR][2][4];
#pragma unroll
  for (int b = 0; b < NR; ++b)
#pragma unroll
    for (int so = 0; so < 2; ++so) {
      const float4 c0 = R[((b * 2 + 0) * 2 + so) * NPR], c1 = R[((b * 2 + 1) * 2 + so) * NPR];
      r[b][so][0] = make_float2(c0.x, c0.y);
      r[b][so][1] = make_float2(c0.z, c0.w);
      r[b][so][2] = make_float2(c1.x, c1.y);
      r[b][so][3] = make_float2(c1.z, c1.w);
    }
  float2 A[2][2], B[2][2];
#pragma unroll
  for (int si = 0; si < 2; ++si)
#pragma unroll
    for (int so = 0; so < 2; ++so) {
      A[si][so] = make_float2(-acc[si * 2 + so].cre, -acc[si * 2 + so].cim);
      B[si][so] = make_float2(0.f, 0.f);
    }
#pragma unroll
  for (int a = 0; a < NL; ++a) {
    float lr[2][4], li[2][4];
#pragma unroll
    for (int si = 0; si < 2; ++si) {
      const float4 c0 = L[((a * 2 + 0) * 2 + si) * NPL], c1 = L[((a * 2 + 1) * 2 + si) * NPL];
      lr[si][0] = c0.x; li[si][0] = c0.y; lr[si][1] = c0.z; li[si][1] = c0.w;
      lr[si][2] = c1.x; li[si][2] = c1.y; lr[si][3] = c1.z; li[si][3] = c1.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int si = 0; si < 2; ++si) {
        const float2 br = make_float2(lr[si][c], lr[si][c]);
        const float2 bi = make_float2(li[si][c], li[si][c]);
#pragma unroll
        for (int b = 0; b < NR; ++b)
#pragma unroll
          for (int so = 0; so < 2; ++so) {
            A[si][so] = __ffma2_rn(br, r[b][so][c], A[si][so]);
            B[si][so] = __ffma2_rn(bi, r[b][so][c], B[si][so]);
          }
      }
  }
#pragma unroll
  for (int si = 0; si < 2; ++si)
#pragma unroll
    for (int so = 0; so < 2; ++so)
      acc[si * 2 + so].commit(__fsub_rn(A[si][so].x, B[si][so].y), __fadd_rn(A[si][so].y, B[si][so].x));
}

// The same in FP64 (scalar FMAs, plain accumulation), chunks of 4 doubles.
template <int NL, int NR, int NPL, int NPR>
__device__ __forceinline__ void join_set_f64(const double* L, const double* R, Acc<double> acc[4]) {
#pragma unroll
  for (int b = 0; b < NR; ++b) {
    double rw[2][8];
#pragma unroll
    for (int so = 0; so < 2; ++so) {
      ld4(R + ((b * 2 + 0) * 2 + so) * NPR * 4, rw[so]);
      ld4(R + ((b * 2 + 1) * 2 + so) * NPR * 4, rw[so] + 4);
    }
#pragma unroll
    for (int a = 0; a < NL; ++a) {
      double lc[2][8];
#pragma unroll
      for (int si = 0; si < 2; ++si) {
        ld4(L + ((a * 2 + 0) * 2 + si) * NPL * 4, lc[si]);
        ld4(L + ((a * 2 + 1) * 2 + si) * NPL * 4, lc[si] + 4);
      }
#pragma unroll
      for (int si = 0; si < 2; ++si)
#pragma unroll
        for (int so = 0; so < 2; ++so) dot_acc(rw[so], lc[si], acc[si * 2 + so].re, acc[si * 2 + so].im);
    }
  }
}

// a8/a9 of a spin-summed team: |M_l|^2 of the lane's four states (the
// compensated FP32 amplitudes squared in float-float), the sum over the team
// in FP64, the coupling, and the store by lane 0.
template <int TEAM>
__device__ __forceinline__ void finish_summed(const KParams& p, const Acc<float> acc[4], int lane, long long pt,
                                              bool valid, double* s_red) {
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    add_square_ff(acc[i].re, acc[i].cre, hi, lo);
    add_square_ff(acc[i].im, acc[i].cim, hi, lo);
  }
  const double m2 = team_sum<TEAM>((double)hi + (double)lo, s_red);
  if (lane == 0 && valid) p.out[pt] = m2 * p.coupling;
}
template <int TEAM>
__device__ __forceinline__ void finish_summed(const KParams& p, const Acc<double> acc[4], int lane, long long pt,
                                              bool valid, double* s_red) {
  double part = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) part = fma(acc[i].re, acc[i].re, fma(acc[i].im, acc[i].im, part));
  const double m2 = team_sum<TEAM>(part, s_red);
  if (lane == 0 && valid) p.out[pt] = m2 * p.coupling;
}

}  // namespace spec
}  // namespace qed
