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

// ------------------------------------------------------------ set-up
// Per point, FP32-mixed (a1-a3 for a team of one lane per photon subset,
// TEAM = 2^n, k <= 4): the momenta, the propagator entries of every subset
// and the external states, with few FP64 instructions (on B300 each warp
// instruction holds the FP64 pipe for many cycles; ncu counts 16 FP64
// arithmetic instructions per point here against 26 for the direct form,
// whose per-photon adds also issue for lanes without the photon).
//   1. each lane loads one FP64 momentum component and splits it into a
//      float-float pair (hi + lo, exact to about 2^-48);
//   2. the Lorentz invariants (setup_invariants): the Minkowski products
//      p.p, p'.p', k_j.k_j, p.k_j, p'.k_j and k_i.k_j (i < j), one per lane,
//      then their signed combinations, one FMA per lane, all in FP64;
//   3. for the subset T of each lane, the FP64 denominator as the same sum
//      as Q_T^2 - m^2 in invariants.  With |T| <= n/2 the line is taken
//      from the incoming electron, Q_T = p + sum_{j in T} sigma_j k_j
//      (sigma_0 = +1, sigma_j = -1); otherwise from the outgoing electron,
//      Q_T = p' - sum_{j not in T} sigma_j k_j, which is the same momentum
//      by momentum conservation.  With U the photons summed (at most two)
//      and tau = sigma (incoming side) or -sigma (outgoing side),
//        D_T = (q.q - m^2) + sum_{j in U} (k_j.k_j + 2 tau_j q.k_j)
//              + sum_{i<j in U} 2 tau_i tau_j k_i.k_j,   q = p or p',
//      three FP64 additions of combinations; the numerator Q_T in
//      float-float (TwoSum on the FP32 pipe), rounded once; the entries
//      (Q0 +- m)/D and Q/D in FP32;
//   4. u(p, +-), ubar(p', +-) and eps_j (pol 1, 2) in FP32 from the
//      float-float momenta (E +- m as float-float sums rounded once).
// Missing photons of U read a zero slot, so every lane runs the same code.

template <int K, int TEAM>
__device__ __forceinline__ void setup_f32(const KParams& p, int lane, long long pt, double* s_mom, float* s_q,
                                          float* s_eps, float* s_spin, double* s_w, float* s_momf) {
  constexpr int N = K + 1, NS = K + 3, NC = NS * 4;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int NPROD = 2 + 3 * N + N * (N - 1) / 2;
  constexpr int ZERO = 2 + 2 * N + N * N;   // the zero slot of the combinations
  static_assert((1 << N) <= TEAM, "a lane for every photon subset");
  static_assert(N / 2 <= 2, "at most two photons per denominator");
  // 1. momenta (FP64) and their float-float split
  for (int i = lane; i < NC; i += TEAM) {
    const double v = __ldg(p.mom + pt * NC + i);
    const float hi = (float)v;
    s_mom[i] = v;
    s_momf[i] = hi;
    s_momf[NC + i] = (float)(v - (double)hi);
  }
  team_sync<TEAM>();
  // 2. the invariants and their combinations c
  setup_invariants<N, TEAM>(lane, p.mass, s_mom, s_w);
  const double* cmb = s_w + NPROD;
  // 3. the subset of this lane (lanes past the 2^n subsets have none)
  if (lane < (1 << N)) {
    const unsigned T = (unsigned)lane;
    float* d = s_q + T * 5;
    const bool out = 2 * __popc(T) > N;
    const unsigned U = out ? ALL & ~T : T;
    const int ja = U ? __ffs(U) - 1 : -1;
    const unsigned U2 = U & (U - 1);
    const int jb = U2 ? __ffs(U2) - 1 : -1;
    const int so = out ? 2 + N : 2;
    double D = cmb[out ? 1 : 0];
    D += cmb[ja < 0 ? ZERO : so + ja];
    D += cmb[jb < 0 ? ZERO : so + jb];
    D += cmb[jb < 0 ? ZERO : 2 + 2 * N + ja * N + jb];
    // the numerator in float-float: q + tau_a k_a + tau_b k_b, with tau_j =
    // sigma_j on the incoming side and -sigma_j on the outgoing side
    const int qs = out ? 2 : 0;
    const int ka = photon_slot_of(ja < 0 ? 0 : ja), kb = photon_slot_of(jb < 0 ? 0 : jb);
    const float ta = ja < 0 ? 0.f : ((ja == 0) != out ? 1.f : -1.f);
    const float tb = jb < 0 ? 0.f : ((jb == 0) != out ? 1.f : -1.f);
    float qh[4], ql[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float sum, err;
      qh[c] = s_momf[qs * 4 + c];
      ql[c] = s_momf[NC + qs * 4 + c];
      two_sum_f(qh[c], ta * s_momf[ka * 4 + c], sum, err);
      qh[c] = sum;
      ql[c] = __fadd_rn(ql[c], __fadd_rn(err, ta * s_momf[NC + ka * 4 + c]));
      two_sum_f(qh[c], tb * s_momf[kb * 4 + c], sum, err);
      qh[c] = sum;
      ql[c] = __fadd_rn(ql[c], __fadd_rn(err, tb * s_momf[NC + kb * 4 + c]));
    }
    const bool used = T != 0 && T != ALL;
    const float inv = used ? 1.0f / (float)D : 0.0f;
    const float mf = (float)p.mass;
    // Q0 -+ m: the high part first (exact where Q0 is close to m)
    d[0] = __fadd_rn(__fadd_rn(qh[0], mf), ql[0]) * inv;
    d[1] = __fadd_rn(__fsub_rn(qh[0], mf), ql[0]) * inv;
    d[2] = __fadd_rn(qh[1], ql[1]) * inv;
    d[3] = __fadd_rn(qh[2], ql[2]) * inv;
    d[4] = __fadd_rn(qh[3], ql[3]) * inv;
  }
  // 4. external states in FP32
  for (int it = lane; it < 4 + 2 * N; it += TEAM) {
    if (it < 4) {
      const int side = it >> 1, e = it & 1;
      const float* h = s_momf + (side ? 8 : 0);
      const float* l = s_momf + NC + (side ? 8 : 0);
      const float mf = (float)p.mass;
      float sp[8];
      float epm, emm;
      e_pm_m_ff(h[0], l[0], mf, epm, emm);
      make_spinor_core<float>(h[1], h[2], h[3], epm, emm, e, side == 1, sp);
      store8(s_spin + (side * 2 + e) * 8, sp);
    } else {
      const int j = (it - 4) >> 1, pb = (it - 4) & 1;
      const float* h = s_momf + 4 * photon_slot_of(j);
      float ev[3];
      make_pol_core<float>(h[1], h[2], h[3], pb, ev);
      float* d = s_eps + (j * 2 + pb) * 4;
      d[0] = ev[0]; d[1] = ev[1]; d[2] = ev[2]; d[3] = 0.f;
    }
  }
  team_sync<TEAM>();
}

// The set-up of a team (a1-a3 and the external states): the FP64-light form
// above for spin-summed mixed teams, whose lanes cover every photon subset
// (k <= 4), else point_setup.
template <int K, typename Real, int TEAM, bool SUMMED>
__device__ __forceinline__ void team_setup(const KParams& p, int lane, long long pt, double* s_mom, Real* s_q,
                                           Real* s_eps, Real* s_spin, double* s_w, float* s_momf) {
  if constexpr (SUMMED && sizeof(Real) == 4 && K <= 4 && (1 << (K + 1)) <= TEAM)
    setup_f32<K, TEAM>(p, lane, pt, s_mom, s_q, s_eps, s_spin, s_w, s_momf);
  else
    point_setup<K, Real, TEAM>(p, lane, pt, s_mom, s_q, s_eps, s_spin, s_w, s_momf);
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
// L_c = (lr, li) and R_c = (rr, ri), the right leaves held in registers as
// (rr, rr) and (ri, ri),
//   A += (rr, rr) * (lr, li),  B += (ri, ri) * (lr, li)
// so that A = (sum rr lr, sum rr li), B = (sum ri lr, sum ri li) and
//   Re M = A.x - B.y,  Im M = A.y + B.x.
// The right leaves are taken BB at a time (all NR where they fit in
// registers); each block is one compensated step per state over its
// NL x BB diagrams: A starts from minus the accumulator's compensation (the
// first step of the Kahan update), B from zero.
template <int NL, int NR, int NPL, int NPR, int BB = NR>
__device__ __forceinline__ void join_set_f32(const float4* L, const float4* R, Acc<float> acc[4]) {
  static_assert(NR % BB == 0, "whole blocks of right leaves");
  // blocks one after another (not unrolled: the registers of one block)
#pragma unroll 1
  for (int b0 = 0; b0 < NR; b0 += BB) {
    float2 rr[BB][2][4], ri[BB][2][4];
#pragma unroll
    for (int bb = 0; bb < BB; ++bb)
#pragma unroll
      for (int so = 0; so < 2; ++so) {
        const int b = b0 + bb;
        const float4 c0 = R[((b * 2 + 0) * 2 + so) * NPR], c1 = R[((b * 2 + 1) * 2 + so) * NPR];
        const float re[4] = {c0.x, c0.z, c1.x, c1.z}, im[4] = {c0.y, c0.w, c1.y, c1.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          rr[bb][so][c] = make_float2(re[c], re[c]);
          ri[bb][so][c] = make_float2(im[c], im[c]);
        }
      }
    float2 A[2][2], B[2][2];
#pragma unroll
    for (int si = 0; si < 2; ++si)
#pragma unroll
      for (int so = 0; so < 2; ++so) {
        A[si][so] = make_float2(-acc[si * 2 + so].cre, -acc[si * 2 + so].cim);
        B[si][so] = make_float2(0.f, 0.f);
      }
    // all left leaves at once where the right leaves fit whole, else two
    // (the registers of the loads in flight)
    constexpr int UA = BB == NR ? NL : 2;
#pragma unroll (UA)
    for (int a = 0; a < NL; ++a) {
      float2 l[2][4];
#pragma unroll
      for (int si = 0; si < 2; ++si) {
        const float4 c0 = L[((a * 2 + 0) * 2 + si) * NPL], c1 = L[((a * 2 + 1) * 2 + si) * NPL];
        l[si][0] = make_float2(c0.x, c0.y);
        l[si][1] = make_float2(c0.z, c0.w);
        l[si][2] = make_float2(c1.x, c1.y);
        l[si][3] = make_float2(c1.z, c1.w);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int si = 0; si < 2; ++si)
#pragma unroll
          for (int bb = 0; bb < BB; ++bb)
#pragma unroll
            for (int so = 0; so < 2; ++so) {
              A[si][so] = __ffma2_rn(rr[bb][so][c], l[si][c], A[si][so]);
              B[si][so] = __ffma2_rn(ri[bb][so][c], l[si][c], B[si][so]);
            }
    }
#pragma unroll
    for (int si = 0; si < 2; ++si)
#pragma unroll
      for (int so = 0; so < 2; ++so)
        acc[si * 2 + so].commit(__fsub_rn(A[si][so].x, B[si][so].y), __fadd_rn(A[si][so].y, B[si][so].x));
  }
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
