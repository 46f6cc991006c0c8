// Forward kernels of the distributively rewritten DAG.
//
// Same team layout and point loop as the plain forward kernel; a node is a
// photon subset T whose current sums one vertex term per photon of T
// (J_T = sum_j eps/_j K_{T \ j}) before its propagation, and every photon set
// S to the left of the join line needs one join, R'_{S^c} . J_S, per spin
// state.  The cost grows exponentially with the number of photons instead of
// factorially.
#include <cuda_runtime.h>

#include "qed_spec.cuh"

namespace qed {

namespace {

__device__ __forceinline__ SumInstr ld_sum_instr(const SumInstr* p) {
  SumInstr in;
  const int4* s = reinterpret_cast<const int4*>(p);
  int4* d = reinterpret_cast<int4*>(&in);
  d[0] = __ldg(s);
  d[1] = __ldg(s + 1);
  d[2] = __ldg(s + 2);
  return in;
}

// y += SIGN (sigma . a) x, column form (SIGN = +-1), as FMA chains.
template <int SIGN, typename R>
__device__ __forceinline__ void pauli_col_acc(const R a[3], const R x[4], R y[4]) {
  const R ax = SIGN * a[0], ay = SIGN * a[1], az = SIGN * a[2];
  y[0] = fma(az, x[0], fma(ax, x[2], fma(ay, x[3], y[0])));
  y[1] = fma(az, x[1], fma(ax, x[3], fma(-ay, x[2], y[1])));
  y[2] = fma(ax, x[0], fma(-ay, x[1], fma(-az, x[2], y[2])));
  y[3] = fma(ax, x[1], fma(ay, x[0], fma(-az, x[3], y[3])));
}
// acc += eps/ x (column form; eps/ as in vertex_col).
template <typename R>
__device__ __forceinline__ void vertex_col_acc(const R e[3], const R x[8], R acc[8]) {
  pauli_col_acc<-1>(e, x + 4, acc);
  pauli_col_acc<1>(e, x, acc + 4);
}

__device__ __forceinline__ void load_eps(const float* p, float e[3]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  e[0] = v.x; e[1] = v.y; e[2] = v.z;
}
__device__ __forceinline__ void load_eps(const double* p, double e[3]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  e[0] = v.x; e[1] = v.y; e[2] = p[2];
}

// One node of the rewritten DAG, variant v: the sum of its NT vertex terms,
// then the propagator of its post set.  One code path for both sides: for a
// real 3-vector a, x (sigma.a) = (sigma.a') x with a' = (ax, -ay, az), so a
// row node's vertex x eps/ is the column form with eps~ = (-ex, ey, -ez) and
// its propagation x (Q/ + m)/D the column form with Q/D replaced by
// (-qx, qy, -qz); sign flips are exact.
template <int NT, bool SUMMED, typename Real>
__device__ __forceinline__ void apply_sum(const SumInstr& in, int v, const KParams& p, const Real* s_q,
                                          const Real* s_eps, const Real* s_spin, Real* s_cur) {
  const Real sg = in.side ? (Real)-1 : (Real)1;
  Real acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (Real)0;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int j = in.photon[t];
    int pol, vp;
    if constexpr (SUMMED) {
      const int b = 1 + in.rank[t];
      pol = (v >> b) & 1;
      vp = (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b);
    } else {
      pol = (int)((p.fixed_pol_bits >> j) & 1u);
      vp = 0;
    }
    Real x[8];
    if (in.src[t] < 0) {
      const int e = SUMMED ? vp : (in.side == 0 ? p.fixed_sin : p.fixed_sout);
      load8(s_spin + (in.side * 2 + e) * 8, x);
    } else {
      load_cur(s_cur, in.src[t], 0, vp, x);
    }
    Real ev[3];
    load_eps(s_eps + (j * 2 + pol) * 4, ev);
    ev[0] *= sg;
    ev[2] *= sg;
    vertex_col_acc(ev, x, acc);
  }
  if (in.post) {
    const Real* P = s_q + in.post * 5;
    const Real Pt[5] = {P[0], P[1], sg * P[2], P[3], sg * P[4]};
    Real z[8];
    prop_col(Pt, acc, z);
    store_cur(s_cur, in.dst, 0, v, z);
  } else {
    store_cur(s_cur, in.dst, 0, v, acc);
  }
}

template <int NT, int TEAM, bool SUMMED, typename Real>
__device__ __forceinline__ void run_slot(int beg, int cnt, int lg, int lane, const KParams& p, const Real* s_q,
                                         const Real* s_eps, const Real* s_spin, Real* s_cur) {
  const int total = cnt << lg;
  for (int it = lane; it < total; it += TEAM) {
    const SumInstr in = ld_sum_instr(p.sinstr + beg + (it >> lg));
    apply_sum<NT, SUMMED, Real>(in, it & ((1 << lg) - 1), p, s_q, s_eps, s_spin, s_cur);
  }
}

// A phase: up to two ranges of nodes of one level each (every node of a
// level sums as many terms as the level).
template <int TEAM, bool SUMMED, typename Real>
__device__ __forceinline__ void run_sum_phase(const Phase& ph, int lane, const KParams& p, const Real* s_q,
                                              const Real* s_eps, const Real* s_spin, Real* s_cur) {
#pragma unroll 1
  for (int slot = 0; slot < 2; ++slot) {
    const int cnt = ph.cnt[slot];
    if (cnt == 0) continue;
    const int lev = ph.level[slot];
    const int lg = SUMMED ? lev + 1 : 0;
    switch (lev) {
      case 1: run_slot<1, TEAM, SUMMED, Real>(ph.beg[slot], cnt, lg, lane, p, s_q, s_eps, s_spin, s_cur); break;
      case 2: run_slot<2, TEAM, SUMMED, Real>(ph.beg[slot], cnt, lg, lane, p, s_q, s_eps, s_spin, s_cur); break;
      case 3: run_slot<3, TEAM, SUMMED, Real>(ph.beg[slot], cnt, lg, lane, p, s_q, s_eps, s_spin, s_cur); break;
      default: run_slot<4, TEAM, SUMMED, Real>(ph.beg[slot], cnt, lg, lane, p, s_q, s_eps, s_spin, s_cur); break;
    }
  }
}

}  // namespace

// Block: one team when TEAM > 32, else 128 threads; FP64 instances may use up
// to about 96 registers per thread, FP32 ones 64 (72 with the FP64-light
// set-up of spin-summed k <= 4).
template <typename Real, int TEAM>
constexpr int rw_block() { return TEAM > 32 ? TEAM : 128; }
template <typename Real, int TEAM, int K, bool SUMMED>
constexpr int rw_min_blocks() {
  constexpr int regs = sizeof(Real) == 8 ? 96 : (SUMMED && K <= 4 ? 72 : 64);
  constexpr int b = 65536 / (rw_block<Real, TEAM>() * regs);
  return b < 1 ? 1 : b;
}

template <int K, bool SUMMED, typename Real, int TEAM>
__global__ void __launch_bounds__(rw_block<Real, TEAM>(), rw_min_blocks<Real, TEAM, K, SUMMED>())
qed_rw_kernel(const KParams p) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int NVL = SUMMED ? (1 << (H + 1)) : 1;
  constexpr int NVR = SUMMED ? (1 << (R + 1)) : 1;
  static_assert(!SUMMED || TEAM == (1 << N), "one thread per polarisation pattern");
  (void)NVL;
  (void)NVR;

  extern __shared__ __align__(16) unsigned char smem[];
  const TeamLayout L = team_layout(K, (int)sizeof(Real), p.ncur);
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const int tpc = blockDim.x / TEAM;
  unsigned char* base = smem + (size_t)team * L.bytes;
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  Real* s_q = reinterpret_cast<Real*>(base + L.q);
  Real* s_eps = reinterpret_cast<Real*>(base + L.eps);
  Real* s_spin = reinterpret_cast<Real*>(base + L.spin);
  double* s_red = reinterpret_cast<double*>(base + L.red);
  Real* s_cur = reinterpret_cast<Real*>(base + L.cur);

  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    spec::team_setup<K, Real, TEAM, SUMMED>(p, lane, valid ? pt : p.n - 1, s_mom, s_q, s_eps, s_spin,
                                            reinterpret_cast<double*>(base + L.w),
                                            reinterpret_cast<float*>(base + L.momf));
    for (int ph = 0; ph < p.n_stored_phases; ++ph) {
      run_sum_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + ph), lane, p, s_q, s_eps, s_spin, s_cur);
      team_sync<TEAM>();
    }
    Acc<Real> acc[SUMMED ? 4 : 1];
    // photon sets in groups: build the group's leaves, then its joins
    for (int g0 = 0, gi = p.n_stored_phases; g0 < p.n_sets; g0 += p.set_group, ++gi) {
      const int g1 = min(p.n_sets, g0 + p.set_group);
      run_sum_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + gi), lane, p, s_q, s_eps, s_spin, s_cur);
      team_sync<TEAM>();
      if constexpr (SUMMED) {
        // state (si, so, c) of lane c: left variant pext(c, S), right
        // variant pext(c, not S), from the plan's lane table
        const unsigned c = (unsigned)lane & ALL;
        Real yr[4], yi[4];
        if constexpr (sizeof(Real) == 4) {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i].start(yr[i], yi[i]);
        }
        for (int s = g0; s < g1; ++s) {
          const SetEntry se = p.sets[s];
          const unsigned tv = __ldg(p.lane_tab + (s << N) + c);
          const int vl = (int)(tv & 0xffu) << 1;
          const int vr = (int)(tv >> 8) << 1;
          Real lc[2][8], rw[2][8];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            load_cur(s_cur, se.leaf_l, 0, vl + q, lc[q]);
            load_cur(s_cur, se.leaf_r, 0, vr + q, rw[q]);
          }
#pragma unroll
          for (int si = 0; si < 2; ++si)
#pragma unroll
            for (int so = 0; so < 2; ++so) {
              if constexpr (sizeof(Real) == 8) dot_acc(rw[so], lc[si], acc[si * 2 + so].re, acc[si * 2 + so].im);
              else dot_acc(rw[so], lc[si], yr[si * 2 + so], yi[si * 2 + so]);
            }
        }
        // the group's joins are one compensated step
        if constexpr (sizeof(Real) == 4) {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i].commit(yr[i], yi[i]);
        }
      } else {
        // one fixed state: the lanes take the group's joins
        for (int s = g0 + lane; s < g1; s += TEAM) {
          const SetEntry se = p.sets[s];
          Real lc[8], rw[8];
          load_cur(s_cur, se.leaf_l, 0, 0, lc);
          load_cur(s_cur, se.leaf_r, 0, 0, rw);
          if constexpr (sizeof(Real) == 8) {
            dot_acc(rw, lc, acc[0].re, acc[0].im);
          } else {
            float yr, yi;
            acc[0].start(yr, yi);
            dot_acc(rw, lc, yr, yi);
            acc[0].commit(yr, yi);
          }
        }
      }
      team_sync<TEAM>();
    }
    double m2;
    if constexpr (SUMMED) {
      double part;
      if constexpr (sizeof(Real) == 8) {
        part = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) part = fma(acc[i].re, acc[i].re, fma(acc[i].im, acc[i].im, part));
      } else {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          add_square_ff(acc[i].re, acc[i].cre, hi, lo);
          add_square_ff(acc[i].im, acc[i].cim, hi, lo);
        }
        part = (double)hi + (double)lo;
      }
      m2 = team_sum<TEAM>(part, s_red);
    } else {
      const double re = team_sum<TEAM>(acc[0].vre(), s_red);
      const double im = team_sum<TEAM>(acc[0].vim(), s_red);
      m2 = re * re + im * im;
    }
    if (lane == 0 && valid) p.out[pt] = m2 * p.coupling;
    team_sync<TEAM>();
  }
}

using KernelFn = void (*)(const KParams);

struct KernelChoice {
  KernelFn fn;
  int team;
};

template <int K, bool SUMMED>
constexpr int rw_team() {
  if constexpr (SUMMED) return 1 << (K + 1);
  else return 32;
}

template <int K, bool SUMMED>
KernelChoice pick_rw(bool mixed) {
  constexpr int T = rw_team<K, SUMMED>();
  if (mixed) return {qed_rw_kernel<K, SUMMED, float, T>, T};
  return {qed_rw_kernel<K, SUMMED, double, T>, T};
}

KernelChoice rewrite_kernel(int k, bool summed, bool mixed) {
#define QED_CASE(KK) \
  case KK: return summed ? pick_rw<KK, true>(mixed) : pick_rw<KK, false>(mixed);
  switch (k) {
    QED_CASE(1) QED_CASE(2) QED_CASE(3) QED_CASE(4) QED_CASE(5) QED_CASE(6) QED_CASE(7)
    default: return KernelChoice{nullptr, 0};
  }
#undef QED_CASE
}

}  // namespace qed
