// Forward kernels of the ABC model (paper App. F): A B -> A + k B through the
// same node-reduced DAG, or the same rewritten DAG, as the QED kernels with
// one spin state, but with scalar building blocks.
//
// A current is one real number.  A vertex multiplies by the coupling g,
// which is taken out of the DAG and applied once as g^(2n) to |M|^2.  A
// propagator of the line after the B's of the set T are attached multiplies
// by 1 / (Q_T^2 - m^2), with m = m_C for odd |T| and m_A for even |T| (the
// line alternates between C and A at every attachment).  The join of a left
// and a right leaf is their product, with the middle propagator already
// applied to the right leaf as in the QED schedule.
//
// One team of TEAM threads per point.  Its shared memory holds the momenta
// (FP64), the table 1/D_T for every subset, the currents, and a reduction
// scratch.  In the FP64 form every product is FP64.  In the mixed form D_T is
// FP64 (the near-on-shell cancellation) and everything after it FP32, with
// one Kahan step per photon set (plain DAG) or per group of sets (rewrite).
#include <cuda_runtime.h>

#include "qed_plan.hpp"
#include "qed_team.cuh"

namespace qed {

namespace {

template <int N>
constexpr int fact() {
  int f = 1;
  for (int i = 2; i <= N; ++i) f *= i;
  return f;
}

// Lanes of the team as a GA x GB grid over the NL x NR (left, right) leaf
// pairs of one photon set; each lane owns a (NL/GA) x (NR/GB) block.
template <int K>
struct AbcShape {
  static constexpr int N = K + 1, H = (N + 1) / 2, R = N - H;
  static constexpr int NL = fact<H>(), NR = fact<R>();
  static constexpr int TEAM = K <= 3 ? 1 : (K == 5 ? 4 : 32);
  static constexpr int GA = K <= 3 ? 1 : (K == 5 ? 2 : 4);
  static constexpr int GB = TEAM / GA;
  static_assert(NL % GA == 0 && NR % GB == 0, "lane grid tiles the leaf pairs");
  static constexpr int BA = NL / GA, BB = NR / GB;
};

// 1/D_T for every subset T (FP64 D_T, same order of operations as the QED
// FP64 propagator table).
template <int N, typename Real, int TEAM>
__device__ __forceinline__ void abc_props(const KParams& p, int lane, const double* s_mom, Real* s_inv) {
  constexpr int NSUB = 1 << N;
  for (int mask = lane; mask < NSUB; mask += TEAM) {
    if (mask == 0 || mask == NSUB - 1) { s_inv[mask] = (Real)0; continue; }
    double q0 = s_mom[0], q1 = s_mom[1], q2 = s_mom[2], q3 = s_mom[3];
    for (int j = 0; j < N; ++j) {
      if (!(mask & (1 << j))) continue;
      const double* kj = s_mom + 4 * (j == 0 ? 1 : j + 2);
      if (j == 0) { q0 += kj[0]; q1 += kj[1]; q2 += kj[2]; q3 += kj[3]; }
      else        { q0 -= kj[0]; q1 -= kj[1]; q2 -= kj[2]; q3 -= kj[3]; }
    }
    const double m = (__popc(mask) & 1) ? p.mass_c : p.mass;
    double D = __dmul_rn(q0, q0);
    D = __dsub_rn(D, __dmul_rn(q1, q1));
    D = __dsub_rn(D, __dmul_rn(q2, q2));
    D = __dsub_rn(D, __dmul_rn(q3, q3));
    D = __dsub_rn(D, __dmul_rn(m, m));
    if constexpr (sizeof(Real) == 8) s_inv[mask] = 1.0 / D;
    else s_inv[mask] = 1.0f / (float)D;
  }
}

// Plain DAG: one node per ordered prefix (left) or suffix (right).
template <typename Real, int TEAM>
__device__ __forceinline__ void abc_phase(const Phase& ph, int lane, const KParams& p, const Real* s_inv,
                                          Real* s_cur) {
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int cnt = ph.cnt[slot];
    for (int it = lane; it < cnt; it += TEAM) {
      const Instr in = ld_instr(p.instr + ph.beg[slot] + it);
      Real x = in.src < 0 ? (Real)1 : s_cur[in.src];
      if (in.post) x *= s_inv[in.post];
      s_cur[in.dst] = x;
    }
  }
}

// Rewritten DAG: one node per subset, the sum over the last attached B.
template <typename Real, int TEAM>
__device__ __forceinline__ void abc_sum_phase(const Phase& ph, int lane, const KParams& p, const Real* s_inv,
                                              Real* s_cur) {
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int cnt = ph.cnt[slot];
    for (int it = lane; it < cnt; it += TEAM) {
      const SumInstr& in = p.sinstr[ph.beg[slot] + it];
      const int nt = __ldg(&in.nterms);
      Real x = (Real)0;
      for (int t = 0; t < nt; ++t) {
        const int src = __ldg(&in.src[t]);
        x += src < 0 ? (Real)1 : s_cur[src];
      }
      const int post = __ldg(&in.post);
      if (post) x *= s_inv[post];
      s_cur[__ldg(&in.dst)] = x;
    }
  }
}

// Real accumulator: plain in FP64, Kahan-compensated in FP32.
template <typename Real> struct AbcAcc;
template <> struct AbcAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ double start() const { return 0.0; }
  __device__ __forceinline__ void commit(double y) { s += y; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct AbcAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ float start() const { return -c; }
  __device__ __forceinline__ void commit(float y) {
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int K, typename Real, bool REWRITE>
__global__ void __launch_bounds__(128, 8) abc_kernel(const KParams p) {
  using Sh = AbcShape<K>;
  constexpr int N = Sh::N;
  constexpr int NS = K + 3;
  constexpr int TEAM = REWRITE ? (K <= 3 ? 1 : 32) : Sh::TEAM;
  extern __shared__ __align__(16) unsigned char smem[];
  const AbcLayout L = abc_layout(K, (int)sizeof(Real), p.ncur);
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const int tpc = blockDim.x / TEAM;
  unsigned char* base = smem + (size_t)team * L.bytes;
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  Real* s_inv = reinterpret_cast<Real*>(base + L.inv);
  double* s_red = reinterpret_cast<double*>(base + L.red);
  Real* s_cur = reinterpret_cast<Real*>(base + L.cur);

  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    const long long ptc = valid ? pt : p.n - 1;
    for (int i = lane; i < NS * 4; i += TEAM) s_mom[i] = __ldg(p.mom + ptc * (NS * 4) + i);
    team_sync<TEAM>();
    abc_props<N, Real, TEAM>(p, lane, s_mom, s_inv);
    team_sync<TEAM>();
    for (int ph = 0; ph < p.n_stored_phases; ++ph) {
      if constexpr (REWRITE) abc_sum_phase<Real, TEAM>(ld_phase(p.phases + ph), lane, p, s_inv, s_cur);
      else abc_phase<Real, TEAM>(ld_phase(p.phases + ph), lane, p, s_inv, s_cur);
      team_sync<TEAM>();
    }
    AbcAcc<Real> acc;
    if constexpr (REWRITE) {
      // groups of photon sets: build the leaves, then one product per set
      for (int g0 = 0, gi = p.n_stored_phases; g0 < p.n_sets; g0 += p.set_group, ++gi) {
        const int g1 = min(p.n_sets, g0 + p.set_group);
        abc_sum_phase<Real, TEAM>(ld_phase(p.phases + gi), lane, p, s_inv, s_cur);
        team_sync<TEAM>();
        Real y = acc.start();
        for (int s = g0 + lane; s < g1; s += TEAM) {
          const SetEntry se = p.sets[s];
          y = fma(s_cur[se.leaf_l], s_cur[se.leaf_r], y);
        }
        acc.commit(y);
        team_sync<TEAM>();
      }
    } else {
      const int la = (lane / Sh::GB) * Sh::BA, lb = (lane % Sh::GB) * Sh::BB;
      for (int s = 0; s < p.n_sets; ++s) {
        const SetEntry se = p.sets[s];
        for (int t = 0; t < p.n_set_phases; ++t) {
          abc_phase<Real, TEAM>(ld_phase(p.phases + se.phase0 + t), lane, p, s_inv, s_cur);
          team_sync<TEAM>();
        }
        // this lane's block of the set's NL x NR S2 nodes
        Real l[Sh::BA], r[Sh::BB];
#pragma unroll
        for (int a = 0; a < Sh::BA; ++a) l[a] = s_cur[se.leaf_l + la + a];
#pragma unroll
        for (int b = 0; b < Sh::BB; ++b) r[b] = s_cur[se.leaf_r + lb + b];
        Real y = acc.start();
#pragma unroll
        for (int a = 0; a < Sh::BA; ++a)
#pragma unroll
          for (int b = 0; b < Sh::BB; ++b) y = fma(l[a], r[b], y);
        acc.commit(y);
        team_sync<TEAM>();
      }
    }
    const double M = team_sum<TEAM>(acc.value(), s_red);
    if (lane == 0 && valid) p.out[pt] = M * M * p.coupling;
    team_sync<TEAM>();
  }
}

template <int K>
KernelChoice pick_abc(bool mixed, bool rewrite) {
  constexpr int TP = AbcShape<K>::TEAM;
  constexpr int TR = K <= 3 ? 1 : 32;
  if (rewrite) return mixed ? KernelChoice{abc_kernel<K, float, true>, TR} : KernelChoice{abc_kernel<K, double, true>, TR};
  return mixed ? KernelChoice{abc_kernel<K, float, false>, TP} : KernelChoice{abc_kernel<K, double, false>, TP};
}

}  // namespace

KernelChoice abc_kernel_for(int k, bool mixed, bool rewrite) {
  switch (k) {
    case 1: return pick_abc<1>(mixed, rewrite);
    case 3: return pick_abc<3>(mixed, rewrite);
    case 5: return pick_abc<5>(mixed, rewrite);
    case 7: return pick_abc<7>(mixed, rewrite);
    default: return KernelChoice{nullptr, 0};
  }
}

}  // namespace qed
