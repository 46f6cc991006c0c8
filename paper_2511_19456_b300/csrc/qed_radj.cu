// Adjoint kernels on the distributively rewritten DAG: |M|^2 and
// d|M|^2 / d k_j for the outgoing photons' 3-momenta (slots 3..k+2, energies
// on shell E_j = |k_j|; p, k_0 and p' held fixed) -- the same function and
// outputs as qed_adj.cu, whose reverse pass walks the node-reduced tries.
//
// The rewritten DAG (term rewriting by distributivity, which the paper
// proposes as a further DAG operation, App. C): one current per photon
// subset and side,
//   column:  J_T = sum_{j in T} eps/_j K_{T\j},  K_{} = u(p),
//            K_T = S(Q_T) J_T for |T| < h; J_S (|S| = h) is a left leaf;
//   row:     I_U = sum_{j in U} G_{U\j} eps/_j,   G_{} = ubar(p'),
//            G_U = I_U S(Q_{all\U}) for |U| <= r (for |U| = r the hoisted
//            propagation half of S2);
//   M_l = sum_{|S| = h} G_{all\S}[l_R] . J_S[l_L].
// Expanding the sums gives back every diagram's chain (Sec. I-D, Eq. 1), so
// M_l and all its derivatives are those of the node-reduced DAG; each
// subset is built once per point and kept in shared memory, and the reverse
// pass visits each subset once.
//
// Reverse mode, with f = sum_l |M_l|^2, seeds Mbar_l = conj(M_l) and the
// bilinear adjoints of qed_adj.cu (sum_l conj(M_l) dM_l = sum zbar . dz):
//   1. transposed joins: Jbar_S[vL] = sum_vR Mbar_l G_{S^c}[vR] and
//      Gbar_{S^c}[vR] = sum_vL Mbar_l J_S[vL]; every leaf is in one join;
//   2. the levels, deepest first, both sides in one phase; a node gathers
//      its adjoint from the pre-propagator adjoints of its parents (the
//      subsets one photon larger), so each adjoint has one writer:
//        column node T:  Kbar_T = sum_{j not in T} Jbar_{T+j} eps/_j,
//                        Jbar_T = Kbar_T S(Q_T);
//        row node U:     Gbar_U = sum_{j not in U} eps/_j Ibar_{U+j},
//                        Ibar_U = S(Q_{all\U}) Gbar_U;
//      with the propagator terms Re s_mu = Re(ybar gamma^mu w) (w the
//      node's sum before its propagator, recomputed from its inputs) and
//      Re u = Re(ybar . y), and the polarisation terms -Re(wbar gamma^i x)
//      of the node's own vertices;
//   3. parameter terms -> photon momenta, as in qed_adj.cu.
// The propagator terms of the lanes that share a node are summed by
// shuffles and stored by one lane (each photon subset is the propagator of
// one node); the polarisation terms go to per-lane accumulators, summed at
// the end; no atomics.  In the mixed form the parameter chain to the
// momenta runs on the FP32 pipe (compensated sums), the FP64 pipe (1/64 of
// the FP32 rate on B300) being kept for the set-up and the final steps.
#include <cuda_runtime.h>

#include "qed_adjoint.cuh"
#include "qed_plan.hpp"
#include "qed_spec.cuh"

namespace qed {

namespace {

using adjb::bil_s0;
using adjb::bil_s1;
using adjb::bil_s2;
using adjb::bil_s3;
using adjb::bil_u;
using adjb::dpol;

// y += SIGN (sigma . a) x for a real 3-vector a and a complex 2-vector x
// (column form; the row form x (sigma . a) is the column form of
// (a_x, -a_y, a_z)), as FMA chains.
template <int SIGN, typename R>
__device__ __forceinline__ void pauli_fma(R ax, R ay, R az, const R x[4], R y[4]) {
  ax *= SIGN; ay *= SIGN; az *= SIGN;
  y[0] = fma(az, x[0], fma(ax, x[2], fma(ay, x[3], y[0])));
  y[1] = fma(az, x[1], fma(ax, x[3], fma(-ay, x[2], y[1])));
  y[2] = fma(ax, x[0], fma(-ay, x[1], fma(-az, x[2], y[2])));
  y[3] = fma(ax, x[1], fma(ay, x[0], fma(-az, x[3], y[3])));
}

// acc += eps/ x (column form; a row node uses it with (-ex, ey, -ez))
template <typename R>
__device__ __forceinline__ void vacc_col(const R e[3], const R x[8], R acc[8]) {
  pauli_fma<-1>(e[0], e[1], e[2], x + 4, acc);
  pauli_fma<1>(e[0], e[1], e[2], x, acc + 4);
}

template <typename R>
__device__ __forceinline__ void load_e3(const R* p, R e[3]) {
  e[0] = p[0]; e[1] = p[1]; e[2] = p[2];
}

// The bits of c selected by mask, packed into the low bits, and the inverse.
template <int N>
__device__ __forceinline__ unsigned pext_n(unsigned c, unsigned mask) {
  unsigned r = 0;
  int o = 0;
#pragma unroll
  for (int j = 0; j < N; ++j)
    if ((mask >> j) & 1u) { r |= ((c >> j) & 1u) << o; ++o; }
  return r;
}
template <int N>
__device__ __forceinline__ unsigned pdep_n(unsigned x, unsigned mask) {
  unsigned r = 0;
  int o = 0;
#pragma unroll
  for (int j = 0; j < N; ++j)
    if ((mask >> j) & 1u) { r |= ((x >> o) & 1u) << j; ++o; }
  return r;
}

__device__ __forceinline__ int slot_of(const KParams& p, int n, int side, unsigned mask) {
  return __ldg(p.radj_slot + (side << n) + (int)mask);
}
__device__ __forceinline__ int aslot_of(const KParams& p, int n, int side, unsigned mask) {
  return __ldg(p.radj_aslot + (side << n) + (int)mask);
}

// Currents in planes of 16 bytes: entry i of a buffer of n entries keeps its
// reals [q * P, (q + 1) * P) at plane q (P = 16 / sizeof(Real)), so that the
// lanes of a round, which mostly take consecutive entries, read and write
// consecutive 16-byte words (no shared-memory bank conflicts).
template <typename Real>
struct Planes {
  static constexpr int P = 16 / (int)sizeof(Real), NQ = 8 / P;
  Real* base;
  int n;
  __device__ __forceinline__ void ld(int i, Real x[8]) const {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if constexpr (P == 4) {
        const float4 a = *reinterpret_cast<const float4*>(base + ((size_t)q * n + i) * P);
        x[4 * q] = a.x; x[4 * q + 1] = a.y; x[4 * q + 2] = a.z; x[4 * q + 3] = a.w;
      } else {
        const double2 a = *reinterpret_cast<const double2*>(base + ((size_t)q * n + i) * P);
        x[2 * q] = a.x; x[2 * q + 1] = a.y;
      }
    }
  }
  __device__ __forceinline__ void st(int i, const Real x[8]) const {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if constexpr (P == 4)
        *reinterpret_cast<float4*>(base + ((size_t)q * n + i) * P) =
            make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
      else
        *reinterpret_cast<double2*>(base + ((size_t)q * n + i) * P) = make_double2(x[2 * q], x[2 * q + 1]);
    }
  }
};

// Spin variant of a node without / with the polarisation bit b (bit 0 is the
// electron helicity, bit 1 + r the polarisation of the set's photon of rank r).
__device__ __forceinline__ int drop_bit(int v, int b) { return (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b); }
__device__ __forceinline__ int ins_bit(int v, int b, int pol) {
  return (v & ((1 << b) - 1)) | (pol << b) | ((v >> b) << (b + 1));
}

// Input x_j of the vertex of photon j in node (side, T), variant v: the
// current of T \ j (variant without j's bit) or the external spinor; also
// returns j's polarisation in this variant.
template <int N, bool SUMMED, typename Real>
__device__ __forceinline__ void vertex_input(const KParams& p, int side, unsigned T, int j, int b, int v,
                                             const Real* s_spin, const Planes<Real>& cur, Real x[8], int& pol) {
  int vp;
  if constexpr (SUMMED) {
    pol = (v >> b) & 1;
    vp = drop_bit(v, b);
  } else {
    pol = (int)((p.fixed_pol_bits >> j) & 1u);
    vp = 0;
  }
  const unsigned Tm = T & ~(1u << j);
  if (Tm == 0) {
    const int e = SUMMED ? vp : (side == 0 ? p.fixed_sin : p.fixed_sout);
    load8(s_spin + (side * 2 + e) * 8, x);
  } else {
    cur.ld(slot_of(p, N, side, Tm) + vp, x);
  }
}

// The node's sum of vertex terms before its propagator: J_T (column) or I_U (row).
template <int N, bool SUMMED, typename Real>
__device__ __forceinline__ void vertex_sum(const KParams& p, int side, unsigned T, int v, const Real* s_eps,
                                           const Real* s_spin, const Planes<Real>& cur, Real w[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = (Real)0;
  int t = 0;
  // the photons of T in increasing order (all nodes of a round have as many)
#pragma unroll 1
  for (unsigned m = T; m; m &= m - 1u) {
    const int j = __ffs((int)m) - 1;
    const int b = 1 + t++;
    Real x[8];
    int pol;
    vertex_input<N, SUMMED, Real>(p, side, T, j, b, v, s_spin, cur, x, pol);
    Real ev[3];
    load_e3(s_eps + (j * 2 + pol) * 4, ev);
    // one code path for both sides: the row form is the column form of
    // (-ex, ey, -ez) (exact sign flips)
    const Real sg = side ? (Real)-1 : (Real)1;
    ev[0] *= sg;
    ev[2] *= sg;
    vacc_col(ev, x, w);
  }
}

// The propagator entries of a node's line in column form: a row node's
// x (Q/ + m)/D is the column form with Q/D replaced by (-qx, qy, -qz).
template <typename Real>
__device__ __forceinline__ void prop_entries(const Real* P, bool row, Real Pt[5]) {
  const Real sg = row ? (Real)-1 : (Real)1;
  Pt[0] = P[0]; Pt[1] = P[1]; Pt[2] = sg * P[2]; Pt[3] = P[3]; Pt[4] = sg * P[4];
}

}  // namespace

// Up to 128 registers per thread in FP32, 255 in FP64 (one warp per block
// for teams of up to 32 lanes, one team per block above).
template <int K, bool SUMMED, typename Real, int TEAM>
__global__ void __launch_bounds__(TEAM > 32 ? TEAM : 32,
                                  sizeof(Real) == 8 ? 1 : 65536 / ((TEAM > 32 ? TEAM : 32) * 128))
qed_radj_kernel(const KParams p) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr int NSUB = 1 << N;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int LMAX = H > R ? H : R;
  static_assert(!SUMMED || TEAM == (1 << N), "one lane per polarisation pattern");

  extern __shared__ __align__(16) unsigned char smem[];
  const RadjLayout A = radj_layout(K, (int)sizeof(Real), p.ncur, p.radj_nadj, SUMMED, TEAM);
  const TeamLayout& L = A.fwd;
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const int tpc = blockDim.x / TEAM;
  unsigned char* base = smem + (size_t)team * A.bytes;
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  Real* s_q = reinterpret_cast<Real*>(base + L.q);
  Real* s_eps = reinterpret_cast<Real*>(base + L.eps);
  Real* s_spin = reinterpret_cast<Real*>(base + L.spin);
  double* s_red = reinterpret_cast<double*>(base + L.red);
  // forward currents, and the adjoints of every node but the column leaves,
  // whose adjoints replace their currents once the joins are transposed
  const Planes<Real> cur{reinterpret_cast<Real*>(base + L.cur), p.ncur};
  const Planes<Real> adj{reinterpret_cast<Real*>(base + A.adj), p.radj_nadj};
  Real* s_mbar = reinterpret_cast<Real*>(base + A.mbar);
  // propagator terms (Re s_mu, Re u) of each photon subset, in the working
  // precision: every subset T with 0 < |T| < n is the propagator of exactly
  // one node (column nodes have |T| < h, row nodes |T| >= h), whose lanes
  // sum them and whose first lane stores them, so no accumulation is needed
  Real* s_ps = reinterpret_cast<Real*>(base + A.acc_s);
  double* s_acc_e = reinterpret_cast<double*>(base + A.acc_e);
  double* s_kbar = reinterpret_cast<double*>(base + A.kbar);
  Real* s_el = reinterpret_cast<Real*>(base + A.elane) + lane * N * 6;   // this lane's polarisation terms

  const int* masks = p.radj_masks;
  const int nsets = p.radj_lev[0][H + 1] - p.radj_lev[0][H];
  const int* set_masks = masks + p.radj_lev[0][H];

  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    const long long ptc = valid ? pt : p.n - 1;

    // ---- forward: external states, propagators, then the subset currents
    if constexpr (SUMMED && sizeof(Real) == 4 && K <= 4)
      // FP64-light mixed set-up of the straight-line kernels (one lane per subset)
      spec::setup_f32<K, TEAM>(p, lane, ptc, s_mom, reinterpret_cast<float*>(s_q), reinterpret_cast<float*>(s_eps),
                               reinterpret_cast<float*>(s_spin), reinterpret_cast<double*>(base + L.w),
                               reinterpret_cast<float*>(base + L.momf));
    else
      point_setup<K, Real, TEAM>(p, lane, ptc, s_mom, s_q, s_eps, s_spin,
                                 reinterpret_cast<double*>(base + L.w), reinterpret_cast<float*>(base + L.momf));
    for (int l = 1; l <= LMAX; ++l) {
      const int lg = SUMMED ? l + 1 : 0;
      const int cl = l <= H ? p.radj_lev[0][l + 1] - p.radj_lev[0][l] : 0;
      const int cr = l <= R ? p.radj_lev[1][l + 1] - p.radj_lev[1][l] : 0;
      const int totl = cl << lg, tot = (cl + cr) << lg;
      for (int it = lane; it < tot; it += TEAM) {
        const int side = it < totl ? 0 : 1;
        const int q = side ? it - totl : it;
        const unsigned T = (unsigned)__ldg(masks + p.radj_lev[side][l] + (q >> lg));
        const int v = q & ((1 << lg) - 1);
        Real w[8];
        vertex_sum<N, SUMMED, Real>(p, side, T, v, s_eps, s_spin, cur, w);
        const unsigned post = side == 0 ? (l < H ? T : 0u) : (ALL & ~T);
        const int dst = slot_of(p, N, side, T) + v;
        if (post) {
          Real z[8], Pt[5];
          prop_entries(s_q + post * 5, side == 1, Pt);
          prop_col(Pt, w, z);
          cur.st(dst, z);
        } else {
          cur.st(dst, w);
        }
      }
      team_sync<TEAM>();
    }

    // ---- the joins: M_l = sum_S G_{S^c}[vR] . J_S[vL]
    Acc<Real> acc[SUMMED ? 4 : 1];
    if constexpr (SUMMED) {
      const unsigned c = (unsigned)lane;
      for (int s = 0; s < nsets; ++s) {
        const unsigned S = (unsigned)__ldg(set_masks + s), Sc = ALL & ~S;
        const int vl = (int)pext_n<N>(c, S) << 1, vr = (int)pext_n<N>(c, Sc) << 1;
        const int ls = slot_of(p, N, 0, S), rs = slot_of(p, N, 1, Sc);
        Real lc[2][8], rw[2][8];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          cur.ld(ls + vl + e, lc[e]);
          cur.ld(rs + vr + e, rw[e]);
        }
#pragma unroll
        for (int si = 0; si < 2; ++si)
#pragma unroll
          for (int so = 0; so < 2; ++so) {
            Real yr = (Real)0, yi = (Real)0;
            dot_acc(rw[so], lc[si], yr, yi);
            acc[si * 2 + so].add(yr, yi);
          }
      }
    } else {
      for (int s = lane; s < nsets; s += TEAM) {
        const unsigned S = (unsigned)__ldg(set_masks + s);
        Real lc[8], rw[8];
        cur.ld(slot_of(p, N, 0, S), lc);
        cur.ld(slot_of(p, N, 1, ALL & ~S), rw);
        Real yr = (Real)0, yi = (Real)0;
        dot_acc(rw, lc, yr, yi);
        acc[0].add(yr, yi);
      }
    }

    // ---- |M|^2 and the seeds conj(M)
    double m2;
    if constexpr (SUMMED) {
      double part = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double re = acc[i].vre(), im = acc[i].vim();
        part = fma(re, re, fma(im, im, part));
        const int lam = (i >> 1) | ((i & 1) << 1) | (lane << 2);   // i = 2 si + so
        s_mbar[2 * lam] = (Real)re;
        s_mbar[2 * lam + 1] = (Real)(-im);
      }
      m2 = team_sum<TEAM>(part, s_red);
    } else if constexpr (sizeof(Real) == 8) {
      const double re = team_sum<TEAM>(acc[0].vre(), s_red);
      const double im = team_sum<TEAM>(acc[0].vim(), s_red);
      m2 = re * re + im * im;
      if (lane == 0) { s_mbar[0] = (Real)re; s_mbar[1] = (Real)(-im); }
    } else {
      // the lanes' compensated sums in float-float (FP32 pipe), squared in FP64
      float rh = acc[0].re, rl = -acc[0].cre, ih = acc[0].im, il = -acc[0].cim;
      team_sum_ff<TEAM>(rh, rl, lane, reinterpret_cast<float*>(s_red));
      team_sum_ff<TEAM>(ih, il, lane, reinterpret_cast<float*>(s_red) + 8);
      m2 = 0.0;
      if (lane == 0) {
        const double re = (double)rh + (double)rl, im = (double)ih + (double)il;
        m2 = re * re + im * im;
        s_mbar[0] = (Real)re;
        s_mbar[1] = (Real)(-im);
      }
    }
    if (lane == 0 && valid && p.out) p.out[pt] = m2 * p.coupling;
    for (int i = lane; i < N * 4; i += TEAM) s_kbar[i] = 0.0;
    team_sync<TEAM>();

    // ---- 1. transposed joins.  First the row leaves' adjoints (they read
    // the column leaves), then the column leaves' adjoints, which replace
    // their currents (they read only the row leaves)
    {
      constexpr int NVL = SUMMED ? 2 << H : 1, NVR = SUMMED ? 2 << R : 1;
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        const bool left = pass == 1;
        const int nvm = left ? NVL : NVR;
        const int tot = nsets * nvm;
        for (int it = lane; it < tot; it += TEAM) {
          const int s = it / nvm, v = it % nvm;
          const unsigned S = (unsigned)__ldg(set_masks + s), Sc = ALL & ~S;
          // the other side of the join: the row leaf of S^c for a column
          // leaf's adjoint, the column leaf of S for a row leaf's
          const unsigned mine = left ? S : Sc, other = left ? Sc : S;
          const int os = slot_of(p, N, left ? 1 : 0, other);
          Real o[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) o[c] = (Real)0;
          if constexpr (SUMMED) {
            const unsigned cm = pdep_n<N>((unsigned)v >> 1, mine);
            const int e_mine = v & 1;
            const int nq = left ? (1 << R) : (1 << H);
            unsigned co = 0;   // submasks of `other` in increasing order: pdep(q, other)
#pragma unroll 1
            for (int qq = 0; qq < nq; ++qq) {
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int si = left ? e_mine : e, so = left ? e : e_mine;
                const int lam = si | (so << 1) | (int)((cm | co) << 2);
                const Real mr = s_mbar[2 * lam], mi = s_mbar[2 * lam + 1];
                Real x[8];
                cur.ld(os + ((qq << 1) | e), x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  o[2 * c] = fma(mr, x[2 * c], fma(-mi, x[2 * c + 1], o[2 * c]));
                  o[2 * c + 1] = fma(mr, x[2 * c + 1], fma(mi, x[2 * c], o[2 * c + 1]));
                }
              }
              co = ((co | ~other) + 1u) & other;
            }
          } else {
            const Real mr = s_mbar[0], mi = s_mbar[1];
            Real x[8];
            cur.ld(os, x);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              o[2 * c] = mr * x[2 * c] - mi * x[2 * c + 1];
              o[2 * c + 1] = mr * x[2 * c + 1] + mi * x[2 * c];
            }
          }
          if (left) cur.st(slot_of(p, N, 0, mine) + v, o);
          else adj.st(aslot_of(p, N, 1, mine) + v, o);
        }
        team_sync<TEAM>();
      }
    }
    // the seeds are read: their space takes the per-lane polarisation terms
#pragma unroll
    for (int i = 0; i < N * 6; ++i) s_el[i] = (Real)0;
    team_sync<TEAM>();

    // ---- 2. the levels, deepest first
    for (int l = LMAX; l >= 1; --l) {
      const int lg = SUMMED ? l + 1 : 0;
      const int nv = 1 << lg;
      const int cl = l <= H ? p.radj_lev[0][l + 1] - p.radj_lev[0][l] : 0;
      const int cr = l <= R ? p.radj_lev[1][l + 1] - p.radj_lev[1][l] : 0;
      const int totl = cl << lg, tot = (cl + cr) << lg;
      constexpr int WMAX = TEAM < 32 ? TEAM : 32;
      const int G = nv < WMAX ? nv : WMAX;   // lanes of one round that share a node
      for (int b0 = 0; b0 < tot; b0 += TEAM) {
        // every lane runs the same rounds (the shuffles below)
        const int it = b0 + lane;
        const bool ok = it < tot;
        const int side = it < totl ? 0 : 1;
        const int q = side ? it - totl : it;
        const unsigned T = ok ? (unsigned)__ldg(masks + p.radj_lev[side][l] + (q >> lg)) : 0u;
        const int v = q & (nv - 1);
        const bool leaf_l = side == 0 && l == H;
        const unsigned post = side == 0 ? (l < H ? T : 0u) : (ALL & ~T);
        Real ps[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) ps[c] = (Real)0;
        if (ok) {
          const int my = slot_of(p, N, side, T);
          const int amy = aslot_of(p, N, side, T);
          // the node's output adjoint ybar: from the joins (leaves; a column
          // leaf's in place of its current) or gathered from the parents'
          // pre-propagator adjoints
          Real yb[8];
          if (leaf_l) {
            cur.ld(my + v, yb);
          } else if (side == 1 && l == R) {
            adj.ld(amy + v, yb);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) yb[c] = (Real)0;
            // the photons not in T: one parent each
#pragma unroll 1
            for (unsigned m = ALL & ~T; m; m &= m - 1u) {
              const int j = __ffs((int)m) - 1;
              const unsigned Tp = T | (1u << j);
              const int bp = 1 + __popc(T & ((1u << j) - 1u));
              // a column leaf keeps its adjoint in its current's place
              const bool in_cur = side == 0 && l + 1 == H;
              const int ps_slot = in_cur ? slot_of(p, N, 0, Tp) : aslot_of(p, N, side, Tp);
#pragma unroll
              for (int pol = 0; pol < (SUMMED ? 2 : 1); ++pol) {
                const int pl = SUMMED ? pol : (int)((p.fixed_pol_bits >> j) & 1u);
                const int vpar = SUMMED ? ins_bit(v, bp, pol) : 0;
                Real wb[8], ev[3];
                if (in_cur) cur.ld(ps_slot + vpar, wb); else adj.ld(ps_slot + vpar, wb);
                load_e3(s_eps + (j * 2 + pl) * 4, ev);
                // transposed vertex: column x -> eps/ x gives xbar = wbar eps/
                // (row form, the column form of (-ex, ey, -ez)), and the
                // converse for a row node
                const Real sg = side ? (Real)1 : (Real)-1;
                ev[0] *= sg;
                ev[2] *= sg;
                vacc_col(ev, wb, yb);
              }
            }
          }
          // through the propagator: wbar = ybar S (column) or S ybar (row),
          // and its parameter terms
          Real wb[8];
          if (post) {
            const Real* P = s_q + post * 5;
            Real Pt[5];
            prop_entries(P, side == 0, Pt);   // transposed: row form for a column node
            prop_col(Pt, yb, wb);
            Real w[8], y[8];
            vertex_sum<N, SUMMED, Real>(p, side, T, v, s_eps, s_spin, cur, w);
            cur.ld(my + v, y);
            if (side == 0) {
              ps[0] = bil_s0(yb, w); ps[1] = bil_s1(yb, w); ps[2] = bil_s2(yb, w); ps[3] = bil_s3(yb, w);
              ps[4] = bil_u(yb, y);
            } else {
              ps[0] = bil_s0(w, yb); ps[1] = bil_s1(w, yb); ps[2] = bil_s2(w, yb); ps[3] = bil_s3(w, yb);
              ps[4] = bil_u(y, yb);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) wb[c] = yb[c];
          }
          // polarisation terms of the node's own vertices: -Re(wbar g^i x)
          // (column) or -Re(x g^i wbar) (row), per photon and polarisation
          int t = 0;
#pragma unroll 1
          for (unsigned m = T; m; m &= m - 1u) {
            const int j = __ffs((int)m) - 1;
            const int b = 1 + t++;
            Real x[8];
            int pol;
            vertex_input<N, SUMMED, Real>(p, side, T, j, b, v, s_spin, cur, x, pol);
            Real* E = s_el + j * 6 + pol * 3;
            if (side == 0) {
              E[0] -= bil_s1(wb, x); E[1] -= bil_s2(wb, x); E[2] -= bil_s3(wb, x);
            } else {
              E[0] -= bil_s1(x, wb); E[1] -= bil_s2(x, wb); E[2] -= bil_s3(x, wb);
            }
          }
          if (!leaf_l) adj.st(amy + v, wb);
        }
        // the propagator terms of one node's variants: summed over its lanes,
        // added to the FP64 accumulators by the first
        for (int off = 1; off < G; off <<= 1)
#pragma unroll
          for (int c = 0; c < 5; ++c) ps[c] += __shfl_xor_sync(0xffffffffu, ps[c], off);
        if (ok && post && (v & (G - 1)) == 0) {
#pragma unroll
          for (int c = 0; c < 5; ++c) s_ps[post * 5 + c] = ps[c];
        }
      }
      team_sync<TEAM>();
    }

    // polarisation terms: the lanes' sums (FP64; in the mixed form a
    // Kahan-compensated FP32 sum, which keeps the FP64 pipe free).  One
    // fixed state uses one polarisation per photon.
    {
      const Real* el = reinterpret_cast<const Real*>(base + A.elane);
      for (int i = lane; i < N * 6; i += TEAM) {
        if constexpr (!SUMMED) {
          const int j = i / 6, pol = (i / 3) & 1;
          if (pol != (int)((p.fixed_pol_bits >> j) & 1u)) { s_acc_e[i] = 0.0; continue; }
        }
        if constexpr (sizeof(Real) == 8) {
          double a = 0.0;
          for (int ln = 0; ln < TEAM; ++ln) a += el[ln * N * 6 + i];
          s_acc_e[i] = a;
        } else {
          float a = 0.f, c = 0.f;
          for (int ln = 0; ln < TEAM; ++ln) {
            const float y = __fsub_rn(el[ln * N * 6 + i], c);
            const float t = __fadd_rn(a, y);
            c = __fsub_rn(__fsub_rn(t, a), y);
            a = t;
          }
          s_acc_e[i] = (double)a - (double)c;
        }
      }
    }
    team_sync<TEAM>();

    // ---- 3. parameters -> outgoing photon momenta
    // df/dQ_T^mu = 2 eta_mu (s_mu - 2 Q^mu u) / D, in place of the subset's
    // terms.  FP64: Q_T and D_T formed again in FP64.  Mixed: from the FP32
    // propagator entries of the set-up, Q^mu / D and 1 / D = (A - B) / 2m
    // with A, B = (Q0 +- m) / D (relative error about u32 Q0 / m, far below
    // the FP32 terms' own).
#pragma unroll 1
    for (int mask = lane; mask < NSUB; mask += TEAM) {
      if (mask == 0 || mask == (int)ALL) continue;
      Real* Ac = s_ps + mask * 5;
      if constexpr (sizeof(Real) == 8) {
        double q0 = s_mom[0], q1 = s_mom[1], q2 = s_mom[2], q3 = s_mom[3];
        for (int j = 0; j < N; ++j) {
          if (!(mask & (1 << j))) continue;
          const double* kj = s_mom + 4 * (j == 0 ? 1 : j + 2);
          if (j == 0) { q0 += kj[0]; q1 += kj[1]; q2 += kj[2]; q3 += kj[3]; }
          else        { q0 -= kj[0]; q1 -= kj[1]; q2 -= kj[2]; q3 -= kj[3]; }
        }
        double D = __dmul_rn(q0, q0);
        D = __dsub_rn(D, __dmul_rn(q1, q1));
        D = __dsub_rn(D, __dmul_rn(q2, q2));
        D = __dsub_rn(D, __dmul_rn(q3, q3));
        D = __dsub_rn(D, __dmul_rn(p.mass, p.mass));
        const double Q[4] = {q0, q1, q2, q3};
        const double two_inv_d = 2.0 / D;
        double qb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const double eta = mu == 0 ? 1.0 : -1.0;
          qb[mu] = eta * (Ac[mu] - 2.0 * Q[mu] * Ac[4]) * two_inv_d;
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) Ac[mu] = qb[mu];
      } else {
        const float* P = reinterpret_cast<const float*>(s_q) + mask * 5;
        const float inv_d = __fdiv_rn(__fsub_rn(P[0], P[1]), 2.0f * (float)p.mass);
        const float qd[4] = {0.5f * __fadd_rn(P[0], P[1]), P[2], P[3], P[4]};   // Q^mu / D
        const float u2 = 2.0f * Ac[4];
        float qb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const float t = __fmaf_rn(-u2, qd[mu], Ac[mu] * inv_d);
          qb[mu] = mu == 0 ? 2.0f * t : -2.0f * t;
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) Ac[mu] = qb[mu];
      }
    }
    team_sync<TEAM>();
    // Q_T = p + k_0 - sum_{j in T, j >= 1} k_j: df/dk_j^mu = -sum over the
    // subsets T that contain j of df/dQ_T^mu, one lane per (j, mu); in the
    // mixed form summed in float-float (TwoSum)
    for (int it = lane; it < K * 4; it += TEAM) {
      const int j = 1 + (it >> 2), mu = it & 3;
      const int lo = (1 << j) - 1;
      if constexpr (sizeof(Real) == 8) {
        double a = 0.0;
#pragma unroll 1
        for (int r = 0; r < (1 << (N - 1)) - 1; ++r)   // r = 2^(n-1) - 1 would be the full set
          a += s_ps[(((r >> j) << (j + 1)) | (1 << j) | (r & lo)) * 5 + mu];
        s_kbar[4 * j + mu] = -a;
      } else {
        float hi = 0.f, lo_ = 0.f;
#pragma unroll 1
        for (int r = 0; r < (1 << (N - 1)) - 1; ++r) {
          float sum, err;
          two_sum_f(hi, s_ps[(((r >> j) << (j + 1)) | (1 << j) | (r & lo)) * 5 + mu], sum, err);
          hi = sum;
          lo_ = __fadd_rn(lo_, err);
        }
        s_kbar[4 * j + mu] = -((double)hi + (double)lo_);
      }
    }
    team_sync<TEAM>();
    // polarisation terms through d eps / d k_j (in the working precision),
    // one lane per (photon, component) over both polarisations
    for (int it = lane; it < 3 * K; it += TEAM) {
      const int j = 1 + it / 3, a = it % 3;
      double g = 0.0;
#pragma unroll
      for (int pb = 0; pb < 2; ++pb) {
        const double* E = s_acc_e + (j * 2 + pb) * 3;
        Real d[3][3];
        dpol<Real>(s_mom + 4 * (j + 2), pb, d);
        g += 2.0 * ((double)E[0] * (double)d[a][0] + (double)E[1] * (double)d[a][1] +
                    (double)E[2] * (double)d[a][2]);
      }
      s_kbar[4 * j + 1 + a] += g;
    }
    team_sync<TEAM>();
    for (int it = lane; it < 3 * K; it += TEAM) {
      const int j = 1 + it / 3, a = it % 3;
      const double* kj = s_mom + 4 * (j + 2);
      const double kn = sqrt(kj[1] * kj[1] + kj[2] * kj[2] + kj[3] * kj[3]);
      const double g = s_kbar[4 * j + 1 + a] + s_kbar[4 * j] * kj[1 + a] / kn;
      if (valid) p.grad[(pt * K + (j - 1)) * 3 + a] = g * p.coupling;
    }
    team_sync<TEAM>();
  }
}

// Teams: one lane per polarisation pattern when the spin is summed (the
// joins' layout), one warp for a fixed state.  Spin-summed k <= 5 and every
// fixed-state k; none beyond (their subset currents and adjoints outgrow
// shared memory).
template <int K, bool SUMMED>
KernelChoice pick_radj(bool mixed) {
  constexpr int T = SUMMED ? (1 << (K + 1)) : 32;
  if (mixed) return {qed_radj_kernel<K, SUMMED, float, T>, T};
  return {qed_radj_kernel<K, SUMMED, double, T>, T};
}

KernelChoice radj_kernel(int k, bool summed, bool mixed) {
  if (summed) {
    switch (k) {
      case 1: return pick_radj<1, true>(mixed);
      case 2: return pick_radj<2, true>(mixed);
      case 3: return pick_radj<3, true>(mixed);
      case 4: return pick_radj<4, true>(mixed);
      case 5: return pick_radj<5, true>(mixed);
      default: return KernelChoice{nullptr, 0};
    }
  }
  switch (k) {
    case 1: return pick_radj<1, false>(mixed);
    case 2: return pick_radj<2, false>(mixed);
    case 3: return pick_radj<3, false>(mixed);
    case 4: return pick_radj<4, false>(mixed);
    case 5: return pick_radj<5, false>(mixed);
    case 6: return pick_radj<6, false>(mixed);
    case 7: return pick_radj<7, false>(mixed);
    default: return KernelChoice{nullptr, 0};
  }
}

}  // namespace qed
