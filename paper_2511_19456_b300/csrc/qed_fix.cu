// Forward |M|^2 of one fixed spin state, register-join form (FP32-mixed and FP64).
//
// The same node-reduced DAG and linear schedule as the table kernel of
// qed_fwd.cu (tasks U, V, S1, S2, Sum of the paper, Sec. II-B), with every
// level below the leaves kept for the whole point.  What differs is how a
// team of TEAM lanes (TEAM >= NL + NR, at most one warp) works through one
// photon set S (|S| = h):
//   1. one round of items: lane a < NL builds left leaf a (the vertex of
//      photon a's position in S applied to a kept column current) and keeps
//      it in registers; lanes NL .. NL+NR-1 build the NR right leaves (a
//      vertex on a kept row current, then the hoisted propagation of S2) and
//      store them to shared memory;
//   2. lane a < NL joins its left leaf with every right leaf of the set:
//      NR complex 4-component dots (S2's product half), read as broadcasts,
//      in packed FP32 FMAs, added to the lane's compensated sum in one
//      Kahan step per set (task Sum).
// So a join loads one right leaf (two 16-byte broadcasts) per dot and never
// reloads the left leaf, and the items carry no decode: each is two ints
// (source and destination current, polarisation vector, propagator, side).
// The loop over the sets is software-pipelined: set s + 1's leaves are
// formed while set s is joined (independent instructions for the same
// warp), with one team barrier per set.
//
// One code path for both sides.  For a real 3-vector a, x (sigma.a) =
// (sigma.a') x with a' = (ax, -ay, az), so the row-form vertex x eps/ equals
// the column-form eps~/ x with eps~ = (-ex, ey, -ez), and the row-form
// propagation x (Q/ + m)/D equals the column form with q = Q/D replaced by
// (-qx, qy, -qz).  Sign flips are exact, so a row item is a column item with
// those two components negated, and the lanes of a round run one code path.
//
// Set-up (momenta, FP64 denominators from Lorentz invariants, FP32
// propagator entries, external states) is the table kernel's (point_setup);
// the lanes' compensated amplitudes are summed across the team in
// float-float and squared in FP64.  The fixed spinors u(p, s) and
// ubar(p', s') are copied to currents 0 and 1 so that first-level items read
// them like any other current.
#include <cuda_runtime.h>

#include "qed_plan.hpp"
#include "qed_spec.cuh"

namespace qed {
namespace fix {

constexpr int fact(int m) { return m <= 1 ? 1 : m * fact(m - 1); }

// One vertex + propagation item: z = S(Q_post) eps/ x in column form, or
// its row form (side bit) by the sign flips above.  Items without a
// propagator name photon set 0, whose entries the kernel sets to the
// identity ((Q0+m)/D = 1, (Q0-m)/D = -1, Q/D = 0: z = eps/ x exactly), so
// that every lane of a round runs the same instructions.
//   w.x: source current (bits 0-15), destination current (bits 16-31;
//        0xffff = keep in registers)
//   w.y: polarisation vector (bits 0-7), propagator photon set (bits 8-23),
//        side (bit 24)
template <typename Real>
__device__ __forceinline__ void item(int2 w, const Real* s_q, const Real* s_eps, const Real* s_cur, Real z[8]) {
  const int src = w.x & 0xffff;
  const int eidx = w.y & 0xff;
  const int post = (w.y >> 8) & 0xffff;
  const Real sg = (w.y >> 24) ? (Real)-1 : (Real)1;
  Real x[8], y[8], e3[3];
  spec::ld8(s_cur + src * 8, x);
  spec::ld3(s_eps + eidx * 4, e3);
  const Real ev[3] = {sg * e3[0], e3[1], sg * e3[2]};
  vertex_col(ev, x, y);
  const Real* P = s_q + post * 5;
  const Real Pt[5] = {P[0], P[1], sg * P[2], P[3], sg * P[4]};
  prop_col(Pt, y, z);
}

__device__ __forceinline__ void store_z(float* cur, int dst, const float z[8]) {
  float4* q = reinterpret_cast<float4*>(cur + dst * 8);
  q[0] = make_float4(z[0], z[1], z[2], z[3]);
  q[1] = make_float4(z[4], z[5], z[6], z[7]);
}
__device__ __forceinline__ void store_z(double* cur, int dst, const double z[8]) {
  double2* q = reinterpret_cast<double2*>(cur + dst * 8);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = make_double2(z[2 * i], z[2 * i + 1]);
}

// Task S2 (product half) + Sum for one left leaf z and the NR right leaves at
// Rb: sum_b sum_c R_b,c z_c (complex, unconjugated) in one compensated step,
// scaled by m (1 for a lane that holds a left leaf, 0 for the others, which
// run the same instructions and add nothing).
// Packed FMAs with the left leaf broadcast in pairs, l = (zr, zr), (zi, zi):
//   A += (zr, zr) * (rr, ri),  B += (zi, zi) * (rr, ri)
// so Re = A.x - B.y and Im = A.y + B.x; two accumulator pairs (even and odd
// right leaves) for independent FMA chains.  A[0] starts from minus the
// compensation (the first step of the Kahan update).
template <int NR>
__device__ __forceinline__ void join(const float z[8], const float* Rb, float m, Acc<float>& acc) {
  float2 lr[4], li[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    lr[c] = make_float2(z[2 * c], z[2 * c]);
    li[c] = make_float2(z[2 * c + 1], z[2 * c + 1]);
  }
  float2 A[2], B[2];
  A[0] = make_float2(-acc.cre, -acc.cim);
  A[1] = B[0] = B[1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int b = 0; b < NR; ++b) {
    const float4* q = reinterpret_cast<const float4*>(Rb + b * 8);
    const float4 c0 = q[0], c1 = q[1];
    const float2 r[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                         make_float2(c1.z, c1.w)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A[b & 1] = __ffma2_rn(lr[c], r[c], A[b & 1]);
      B[b & 1] = __ffma2_rn(li[c], r[c], B[b & 1]);
    }
  }
  const float yr = __fadd_rn(__fsub_rn(A[0].x, B[0].y), __fsub_rn(A[1].x, B[1].y));
  const float yi = __fadd_rn(__fadd_rn(A[0].y, B[0].x), __fadd_rn(A[1].y, B[1].x));
  acc.commit(__fmul_rn(m, yr), __fmul_rn(m, yi));
}

// The same in FP64: plain FMA chains (two, for even and odd right leaves)
// and direct accumulation, as in the other FP64 kernels; m as above.
template <int NR>
__device__ __forceinline__ void join(const double z[8], const double* Rb, double m, Acc<double>& acc) {
  double re[2] = {0.0, 0.0}, im[2] = {0.0, 0.0};
#pragma unroll
  for (int b = 0; b < NR; ++b) {
    double r[8];
    spec::ld8(Rb + b * 8, r);
    dot_acc(r, z, re[b & 1], im[b & 1]);
  }
  acc.add(m * (re[0] + re[1]), m * (im[0] + im[1]));
}

// One point (pt; valid = it exists) by the team whose shared memory starts at
// base: a1..a9.  The team has W warps of WL = TEAM / W lanes (W = 1: TEAM
// lanes in one warp, several teams per warp when TEAM < 32); warp w takes
// the photon sets w, w + W, w + 2W, ... with its own two right-leaf buffers,
// so that the warps of a team meet only at the kept levels and at the end.
template <int K, typename Real, int TEAM, int W, bool PIPE>
__device__ __forceinline__ void point(const KParams& p, long long pt, bool valid, int lane, unsigned char* base) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr int NL = fact(H);
  constexpr int NR = fact(R);
  constexpr int WL = TEAM / W;
  static_assert(NL + NR <= WL && WL <= 32 && (W == 1 || WL == 32), "one warp (part) holds a set's leaves");
  const TeamLayout L = team_layout(K, (int)sizeof(Real), p.fix_ncur);
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  Real* s_q = reinterpret_cast<Real*>(base + L.q);
  Real* s_eps = reinterpret_cast<Real*>(base + L.eps);
  Real* s_spin = reinterpret_cast<Real*>(base + L.spin);
  double* s_red = reinterpret_cast<double*>(base + L.red);
  Real* s_cur = reinterpret_cast<Real*>(base + L.cur);

  // a1-a3 and the external states
  point_setup<K, Real, TEAM>(p, lane, pt, s_mom, s_q, s_eps, s_spin, reinterpret_cast<double*>(base + L.w),
                             reinterpret_cast<float*>(base + L.momf));
  for (int i = lane; i < 16; i += TEAM) {
    const int side = i >> 3;
    s_cur[i] = s_spin[(side * 2 + (side ? p.fixed_sout : p.fixed_sin)) * 8 + (i & 7)];
  }
  if (lane == 0) {   // photon set 0: the identity propagator
    s_q[0] = (Real)1; s_q[1] = (Real)-1; s_q[2] = (Real)0; s_q[3] = (Real)0; s_q[4] = (Real)0;
  }
  team_sync<TEAM>();

  // a4/a5: the kept levels, one group of independent items after another
  const int2* items = reinterpret_cast<const int2*>(p.fix_items);
  for (int g = 0; g < p.fix_ngroups; ++g) {
#pragma unroll 2
    for (int it = p.fix_group[g] + lane; it < p.fix_group[g + 1]; it += TEAM) {
      const int2 w = __ldg(items + it);
      Real z[8];
      item(w, s_q, s_eps, s_cur, z);
      store_z(s_cur, (unsigned)w.x >> 16, z);
    }
    team_sync<TEAM>();
  }

  // a4-a7 per photon set: one item per lane (a right leaf goes to position
  // dst of the warp's current buffer), a warp barrier, the joins.  Double
  // buffering: a buffer is rewritten two sets after it was read, past the
  // barrier that follows the joins which read it.
  const int wl = lane % WL, wi = lane / WL;
  const int2* set_items = items + p.fix_set_off + wl;
  const Real m = wl < NL ? (Real)1 : (Real)0;
  Real* rb = s_cur + (p.fix_rbase + wi * 2 * NR) * 8;
  Acc<Real> acc;
  if constexpr (PIPE) {
    // software-pipelined: the items of the warp's next set are formed while
    // it joins the current one (independent instruction streams).  The
    // table ends with W sets of idle items, so the last iteration needs no
    // branch.
    Real zc[8];
    {
      const int2 w = __ldg(set_items + wi * WL);
      item(w, s_q, s_eps, s_cur, zc);
      const int dst = (unsigned)w.x >> 16;
      if (dst != 0xffff) store_z(rb, dst, zc);
    }
    if constexpr (W == 1) team_sync<TEAM>(); else __syncwarp();
    int i = 0;
    for (int s = wi; s < p.n_sets; s += W, ++i) {
      const int2 w = __ldg(set_items + (s + W) * WL);
      Real zn[8];
      item(w, s_q, s_eps, s_cur, zn);
      const int dst = (unsigned)w.x >> 16;
      if (dst != 0xffff) store_z(rb + ((i + 1) & 1) * NR * 8, dst, zn);
      join<NR>(zc, rb + (i & 1) * NR * 8, m, acc);
      if constexpr (W == 1) team_sync<TEAM>(); else __syncwarp();
#pragma unroll
      for (int c = 0; c < 8; ++c) zc[c] = zn[c];
    }
  } else {
    int i = 0;
    for (int s = wi; s < p.n_sets; s += W, ++i) {
      const int2 w = __ldg(set_items + s * WL);
      Real z[8];
      item(w, s_q, s_eps, s_cur, z);
      const int dst = (unsigned)w.x >> 16;
      Real* buf = rb + (i & 1) * NR * 8;
      if (dst != 0xffff) store_z(buf, dst, z);
      if constexpr (W == 1) team_sync<TEAM>(); else __syncwarp();
      join<NR>(z, buf, m, acc);
    }
  }

  // a7 across the team and a8/a9.  Mixed: the lanes' compensated partial
  // amplitudes summed in float-float (the FP64 pipe, 1/64 of the FP32 rate,
  // is kept for the set-up), |M|^2 in FP64 by lane 0.  FP64: an FP64 sum.
  if constexpr (sizeof(Real) == 4) {
    float rh = acc.re, rl = -acc.cre, ih = acc.im, il = -acc.cim;
    team_sum_ff<TEAM, W>(rh, rl, lane, reinterpret_cast<float*>(s_red));
    team_sum_ff<TEAM, W>(ih, il, lane, reinterpret_cast<float*>(s_red) + 2 * W);
    if (lane == 0 && valid) {
      const double re = (double)rh + (double)rl, im = (double)ih + (double)il;
      p.out[pt] = (re * re + im * im) * p.coupling;
    }
  } else {
    const double re = team_sum<TEAM>(acc.vre(), s_red);
    const double im = team_sum<TEAM>(acc.vim(), s_red);
    if (lane == 0 && valid) p.out[pt] = (re * re + im * im) * p.coupling;
  }
  team_sync<TEAM>();
}

}  // namespace fix

// Persistent grid: the CTA's teams take points blockIdx.x * tpc + team, then
// every gridDim.x * tpc further (points past the end are evaluated on a
// clamped index and not stored, so every team of a CTA runs the same
// number of iterations).
template <int K, typename Real, int TEAM, int W, bool PIPE, int MINB>
__global__ void __launch_bounds__(128, MINB) qed_fix_fwd_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tpc = blockDim.x / TEAM;
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const TeamLayout L = team_layout(K, (int)sizeof(Real), p.fix_ncur);
  unsigned char* base = smem + (size_t)team * L.bytes;
  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    fix::point<K, Real, TEAM, W, PIPE>(p, valid ? pt : p.n - 1, valid, lane, base);
  }
}

// Team of the register-join form: the smallest power of two that holds a
// set's NL + NR leaves (k <= 5, one warp or less, software-pipelined), and
// two warps at k = 6 (30 leaves per set; the two warps take alternate sets,
// which doubles the resident warps for the same shared memory).  None at
// k = 7, whose sets need 48 lanes.  The host derives the warps per team as
// team / min(team, 32).
KernelChoice fixed_join_kernel(int k, bool mixed) {
  if (mixed) {
    switch (k) {
      case 1: return {qed_fix_fwd_kernel<1, float, 2, 1, true, 4>, 2};
      case 2: return {qed_fix_fwd_kernel<2, float, 4, 1, true, 4>, 4};
      case 3: return {qed_fix_fwd_kernel<3, float, 4, 1, true, 4>, 4};
      case 4: return {qed_fix_fwd_kernel<4, float, 8, 1, true, 4>, 8};
      case 5: return {qed_fix_fwd_kernel<5, float, 16, 1, true, 4>, 16};
      case 6: return {qed_fix_fwd_kernel<6, float, 64, 2, false, 7>, 64};
      default: return {nullptr, 0};
    }
  }
  switch (k) {
    case 1: return {qed_fix_fwd_kernel<1, double, 2, 1, true, 2>, 2};
    case 2: return {qed_fix_fwd_kernel<2, double, 4, 1, true, 2>, 4};
    case 3: return {qed_fix_fwd_kernel<3, double, 4, 1, true, 2>, 4};
    case 4: return {qed_fix_fwd_kernel<4, double, 8, 1, true, 2>, 8};
    case 5: return {qed_fix_fwd_kernel<5, double, 16, 1, true, 2>, 16};
    case 6: return {qed_fix_fwd_kernel<6, double, 64, 2, false, 2>, 64};
    default: return {nullptr, 0};
  }
}

}  // namespace qed
