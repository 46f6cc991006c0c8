// Evaluation of one phase-space point by one team, and of a range of points
// by the teams of a CTA; shared by the standalone and the batched forward
// kernels.
#pragma once

#include "qed_spec.cuh"

namespace qed {

// One point (index pt; valid = it exists) evaluated by the team whose shared
// memory starts at base: a1..a9.
template <int K, bool SUMMED, typename Real, int TEAM, int ES>
__device__ __forceinline__ void eval_point(const KParams& p, long long pt, bool valid, int lane,
                                           unsigned char* base) {
  constexpr int N = K + 1;
  constexpr int NSI = ES >= 2 ? 1 : 2;
  constexpr int NSO = ES >= 4 ? 1 : 2;
  static_assert(!SUMMED || TEAM == (1 << N) * ES, "team = polarisation patterns x helicity split");
  const TeamLayout L = team_layout(K, (int)sizeof(Real), p.ncur);
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  Real* s_q = reinterpret_cast<Real*>(base + L.q);
  Real* s_eps = reinterpret_cast<Real*>(base + L.eps);
  Real* s_spin = reinterpret_cast<Real*>(base + L.spin);
  double* s_red = reinterpret_cast<double*>(base + L.red);
  Real* s_cur = reinterpret_cast<Real*>(base + L.cur);

  spec::team_setup<K, Real, TEAM, SUMMED>(p, lane, pt, s_mom, s_q, s_eps, s_spin,
                                          reinterpret_cast<double*>(base + L.w),
                                          reinterpret_cast<float*>(base + L.momf));

  // ---- a4/a5: currents kept for the whole point
  for (int ph = 0; ph < p.n_stored_phases; ++ph) {
    const Phase P = ld_phase(p.phases + ph);
    run_phase<TEAM, SUMMED, Real>(P, lane, p, s_q, s_eps, s_spin, s_cur);
    team_sync<TEAM>();
  }

  Acc<Real> acc[SUMMED ? NSI * NSO : 1];
  for (int s = 0; s < p.n_sets; ++s) {
    const SetEntry se = p.sets[s];
    for (int t = 0; t < p.n_set_phases; ++t) {
      const Phase P = ld_phase(p.phases + se.phase0 + t);
      run_phase<TEAM, SUMMED, Real>(P, lane, p, s_q, s_eps, s_spin, s_cur);
      team_sync<TEAM>();
    }
    join_set<K, SUMMED, Real, TEAM, ES>(se, SUMMED ? p.lane_tab + ((size_t)s << N) : nullptr, lane, s_cur, acc);
    team_sync<TEAM>();
  }

  // ---- a8/a9: square, spin sum in FP64, store
  double m2;
  if constexpr (SUMMED) {
    double part;
    if constexpr (sizeof(Real) == 8) {
      part = 0.0;
#pragma unroll
      for (int i = 0; i < NSI * NSO; ++i) part = fma(acc[i].re, acc[i].re, fma(acc[i].im, acc[i].im, part));
    } else {
      // squares of the compensated amplitudes, exact to ~2^-48 in
      // float-float; the sum over the team's states in FP64
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int i = 0; i < NSI * NSO; ++i) {
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

// The CTA's teams take points pt0 + team for pt0 = p_begin, p_begin + tpc, ...
// below p_end; every team of a warp runs the same number of iterations (points
// past the end are evaluated on a clamped index and not stored).
template <int K, bool SUMMED, typename Real, int TEAM, int ES>
__device__ __forceinline__ void eval_range(const KParams& p, long long p_begin, long long p_end,
                                           long long stride, unsigned char* smem) {
  const TeamLayout L = team_layout(K, (int)sizeof(Real), p.ncur);
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const int tpc = blockDim.x / TEAM;
  unsigned char* base = smem + (size_t)team * L.bytes;
  for (long long pt0 = p_begin; pt0 < p_end; pt0 += stride) {
    const long long pt = pt0 + team;
    const bool valid = pt < p_end;
    eval_point<K, SUMMED, Real, TEAM, ES>(p, valid ? pt : p_end - 1, valid, lane, base);
  }
  (void)tpc;
}

}  // namespace qed
