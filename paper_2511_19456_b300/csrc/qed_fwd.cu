// Forward |M|^2 kernels for sm_103a.
//
// One team of TEAM threads evaluates one phase-space point at a time
// (persistent grid-stride loop).  Per point:
//   1. momenta -> shared memory (coalesced across the teams of a CTA);
//   2. U: spinors u(p, +-), ubar(p', +-) and eps_j(pol 1, 2) in FP64, and the
//      propagator entries of every photon subset (FP64 momenta and
//      denominators), stored in the team's working precision;
//   3. the linear schedule of the node-reduced DAG: phases of V (+S1)
//      instructions, each expanded over its spin variants;
//   4. for every photon set S to the left of the join line: the currents
//      rebuilt for S, then the S2 joins of all its diagrams, accumulated per
//      spin state (Kahan-compensated in the mixed form);
//   5. |M|^2 summed over spin states in FP64 (shuffle reduction), stored.
//
// Summed spin: TEAM = 2^n and thread c owns the photon-polarisation pattern
// c together with its 4 electron-helicity pairs, i.e. 4 of the 2^(n+2)
// states.  Fixed spin: threads split the diagrams of each set and the
// complex amplitude is reduced across the team at the end.
#include <cuda_runtime.h>

#include <cstdio>

#include "qed_team.cuh"

namespace qed {

template <int K, bool SUMMED, typename Real, int TEAM, int ES>
__global__ void __launch_bounds__(TEAM > 32 ? TEAM : 256)
qed_fwd_kernel(const KParams p) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr int NS = K + 3;
  constexpr int NSUB = 1 << N;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int NVL = SUMMED ? (1 << (H + 1)) : 1;
  constexpr int NVR = SUMMED ? (1 << (R + 1)) : 1;
  constexpr int NL = [] { int f = 1; for (int i = 2; i <= H; ++i) f *= i; return f; }();
  constexpr int NR = [] { int f = 1; for (int i = 2; i <= R; ++i) f *= i; return f; }();
  constexpr int BC = NR >= 2 ? 2 : 1;   // right leaves held in registers
  constexpr int GA = NL % 3 == 0 ? 3 : (NL % 2 == 0 ? 2 : 1); // left leaves per compensated step
  // Summed spin: ES threads share one photon-polarisation pattern and split
  // its 4 electron-helicity pairs (ES = 1: all 4; 2: one incoming helicity
  // each; 4: one pair each).
  constexpr int NSI = ES >= 2 ? 1 : 2;
  constexpr int NSO = ES >= 4 ? 1 : 2;
  static_assert(!SUMMED || TEAM == (1 << N) * ES, "team = polarisation patterns x helicity split");

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
    const long long ptc = valid ? pt : p.n - 1;

    point_setup<K, Real, TEAM>(p, lane, ptc, s_mom, s_q, s_eps, s_spin);

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
      join_set<K, SUMMED, Real, TEAM, ES>(se, lane, s_cur, acc);
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
}

// ----------------------------------------------------------- dispatch
// Summed spin: one thread keeps all 4 helicity pairs of a polarisation
// pattern (ES = 1); splitting them over more threads (ES = 2, 4) raises the
// threads per point but halves the FMAs per shared-memory load of the join,
// which measured slower for both precisions.  Fixed spin: a team of up to
// one warp splits the diagrams.
template <int K, bool SUMMED, bool MIXED>
constexpr int es_of() { return 1; }

template <int K, bool SUMMED, bool MIXED>
constexpr int team_of() {
  if constexpr (SUMMED) return (1 << (K + 1)) * es_of<K, SUMMED, MIXED>();
  else return K == 1 ? 2 : (K == 2 ? 4 : (K == 3 ? 8 : (K == 4 ? 16 : 32)));
}

using KernelFn = void (*)(const KParams);

struct KernelChoice {
  KernelFn fn;
  int team;
};

template <int K, bool SUMMED>
KernelChoice pick(bool mixed) {
  if (mixed) {
    constexpr int T = team_of<K, SUMMED, true>();
    return {qed_fwd_kernel<K, SUMMED, float, T, es_of<K, SUMMED, true>()>, T};
  }
  constexpr int T = team_of<K, SUMMED, false>();
  return {qed_fwd_kernel<K, SUMMED, double, T, es_of<K, SUMMED, false>()>, T};
}

KernelChoice forward_kernel(int k, bool summed, bool mixed) {
#define QED_CASE(KK) \
  case KK: return summed ? pick<KK, true>(mixed) : pick<KK, false>(mixed);
  switch (k) {
    QED_CASE(1) QED_CASE(2) QED_CASE(3) QED_CASE(4) QED_CASE(5) QED_CASE(6) QED_CASE(7)
    default: return KernelChoice{nullptr, 0};
  }
#undef QED_CASE
}

cudaError_t launch_forward(KernelFn fn, int grid, int block, size_t smem, cudaStream_t st,
                           const KParams& p) {
  fn<<<grid, block, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace qed
