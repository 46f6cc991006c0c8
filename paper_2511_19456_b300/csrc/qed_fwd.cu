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

#include "qed_eval.cuh"

namespace qed {

template <int K, bool SUMMED, typename Real, int TEAM, int ES>
__global__ void __launch_bounds__(TEAM > 32 ? TEAM : 256)
qed_fwd_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tpc = blockDim.x / TEAM;
  eval_range<K, SUMMED, Real, TEAM, ES>(p, (long long)blockIdx.x * tpc, p.n, (long long)gridDim.x * tpc,
                                        smem);
}

// Spin-summed, k other than 4 (and mixed k = 7): launch bounds that allow
// up to 128 registers per thread (the compiler's own choice under the
// one-argument bounds spilled a few bytes at k = 1, 3, 5, 6 and, with the
// packed joins, at mixed k = 7; k = 4 and FP64 k = 7 keep those bounds).
template <int K, typename Real, int TEAM>
__global__ void __launch_bounds__(TEAM > 32 ? TEAM : 256, 65536 / ((TEAM > 32 ? TEAM : 256) * 128))
qed_fwd_summed_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tpc = blockDim.x / TEAM;
  eval_range<K, true, Real, TEAM, 1>(p, (long long)blockIdx.x * tpc, p.n, (long long)gridDim.x * tpc, smem);
}

// One fixed state, FP64: 128-thread blocks of up to 96 registers per thread.
template <int K, int TEAM>
__global__ void __launch_bounds__(128, 5)
qed_fwd_fixed64_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tpc = blockDim.x / TEAM;
  eval_range<K, false, double, TEAM, 1>(p, (long long)blockIdx.x * tpc, p.n, (long long)gridDim.x * tpc, smem);
}

// One fixed state, mixed: 128-thread blocks of up to 128 registers per
// thread, so that the unrolled rounds of the join do not spill; at k = 6,
// 102 registers (5 blocks per SM), which it fits without spilling.
template <int K, int TEAM>
__global__ void __launch_bounds__(128, K == 6 ? 5 : 4)
qed_fwd_fixed_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tpc = blockDim.x / TEAM;
  eval_range<K, false, float, TEAM, 1>(p, (long long)blockIdx.x * tpc, p.n, (long long)gridDim.x * tpc, smem);
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
  else if constexpr (!MIXED && K >= 5) return 16;   // FP64: fewer idle lanes in partial rounds
  else return K == 1 ? 2 : (K == 2 ? 4 : (K == 3 ? 8 : (K == 4 ? 16 : 32)));
}

using KernelFn = void (*)(const KParams);

struct KernelChoice {
  KernelFn fn;
  int team;
};

template <int K, bool SUMMED>
KernelChoice pick(bool mixed) {
  if constexpr (!SUMMED) {
    constexpr int TM = team_of<K, false, true>();
    constexpr int TD = team_of<K, false, false>();
    if (mixed) return {qed_fwd_fixed_kernel<K, TM>, TM};
    return {qed_fwd_fixed64_kernel<K, TD>, TD};
  } else if constexpr (K != 4 && K != 7) {
    constexpr int T = team_of<K, true, true>();
    if (mixed) return {qed_fwd_summed_kernel<K, float, T>, T};
    return {qed_fwd_summed_kernel<K, double, T>, T};
  } else {
    if (mixed) {
      constexpr int T = team_of<K, SUMMED, true>();
      // k = 7: the packed joins spill under the one-argument bounds (the
      // compiler settles on 80 registers); two 256-thread blocks per SM are
      // all shared memory holds anyway, so allow 128
      if constexpr (K == 7) return {qed_fwd_summed_kernel<K, float, T>, T};
      else return {qed_fwd_kernel<K, SUMMED, float, T, es_of<K, SUMMED, true>()>, T};
    }
    constexpr int T = team_of<K, SUMMED, false>();
    return {qed_fwd_kernel<K, SUMMED, double, T, es_of<K, SUMMED, false>()>, T};
  }
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
