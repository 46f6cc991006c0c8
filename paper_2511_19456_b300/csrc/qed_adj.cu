// Adjoint kernels: |M|^2 and d|M|^2 / d k_j for the outgoing photons' 3-momenta
// (slots 3..k+2, energies on shell E_j = |k_j|; p, k_0 and p' held fixed).
//
// Reverse mode through the same node-reduced DAG as the forward kernels.
// With f = sum_l |M_l|^2, df = 2 Re sum_l conj(M_l) dM_l.  Every complex
// intermediate z gets an adjoint zbar such that sum_l conj(M_l) dM_l =
// sum zbar . dz (bilinear, no conjugation); a linear step z = W x passes
// xbar = W^T zbar and contributes zbar^T dW x for parameters inside W.
//
// Per point:
//   1. forward pass -> M_l, |M|^2: the currents as in the forward kernel;
//      per photon set M_l += (sum_b R'_b) . (sum_a L_a), the distributive
//      form of the set's joins (the same leaf sums as in step 3); one fixed
//      state in mixed precision keeps the per-diagram joins;
//   2. seeds Mbar_l = conj(M_l) in shared memory;
//   3. for every photon set S: rebuild the set's currents (sub-currents are
//      recomputed, not stored), transposed joins give the leaf adjoints
//        Lbar_a = sum_b sum_l Mbar_l R'_b,   R'bar_b = sum_a sum_l Mbar_l L_a
//      (the same for every a, resp. b: the leaf sums are formed first),
//      then the set's instructions in reverse order pass adjoints to their
//      inputs and accumulate the parameter terms;
//   4. the kept inner levels in reverse order;
//   5. parameter adjoints -> photon momenta:
//        propagator of subset T (P = (Q/ + m)/D): with s_mu = ybar gamma^mu w
//        and u = ybar . y summed over its uses,
//          df/dQ^mu = 2 Re[eta_mu (s_mu - 2 Q^mu u) / D],
//        Q_T = p + sum_{j in T} c_j k_j;
//        vertex of photon j (eps/ = -gamma^i eps^i): with e_i = -wbar gamma^i x,
//          df/deps^i = 2 Re e_i, chained through eps_pol(k_j);
//        finally dE_j/dk_j = k_j / |k_j|.
// Q, D and eps are real, so only the real parts of s_mu, u and e_i are
// accumulated.  The accumulators are FP64 in shared memory (atomic adds);
// currents and their adjoints are in the working precision.  In mixed
// precision the terms of one photon set are first summed in FP32 (one slot
// per propagator of the set, one per photon and polarisation), then added
// to the FP64 accumulators once per set, so that the lanes of a team do not
// all contend for the same FP64 words.
#include <cuda_runtime.h>

#include "qed_adjoint.cuh"
#include "qed_team.cuh"

namespace qed {

namespace {

using adjb::bil_s0;
using adjb::bil_s1;
using adjb::bil_s2;
using adjb::bil_s3;
using adjb::bil_u;
using adjb::dpol;

template <typename Real>
__device__ __forceinline__ void atomic_add_cur(Real* p, int nv, const Real x[8]) {
  typedef typename C2<Real>::T T;
  (void)sizeof(T);
#pragma unroll
  for (int i = 0; i < 8; ++i) atomicAdd(p + i, x[i]);
  (void)nv;
}

// Parameter terms of one instruction output: the propagator bilinears
// (s_mu, mu = 0..3, and u) of its post set and the polarisation terms e_i
// (i = 1..3) of its photon, in the working precision.  Q, D and eps are
// real, so df = 2 Re(...) needs only their real parts.
template <typename Real>
struct ParTerms {
  Real s[5];    // Re s_0..s_3, Re u
  Real e[3];    // Re e_1..e_3, already with the sign of eps/ = -gamma.eps
};

// One instruction output variant (polarisation pol): given its adjoint ybar,
// its input x and (when it has a propagator) its output y = P eps/ x as
// stored by the forward pass, add the parameter terms to T and the input's
// adjoint contribution to xbar.
template <typename Real>
__device__ __forceinline__ void backprop_terms(const Instr& in, int pol, const Real x[8], const Real yb[8],
                                               const Real y[8], const Real* s_q, const Real* s_eps,
                                               ParTerms<Real>& T, Real xbar[8]) {
  const Real* e3 = s_eps + (in.photon * 2 + pol) * 4;
  const Real ev[3] = {e3[0], e3[1], e3[2]};
  Real w[8], wb[8], t[8];
  if (in.side == 0) {
    vertex_col(ev, x, w);                       // w = eps/ x
    if (in.post) {
      const Real* P = s_q + in.post * 5;
      prop_row(P, yb, wb);                      // wbar = ybar P
      T.s[0] += bil_s0(yb, w);                  // s_mu = ybar g^mu w
      T.s[1] += bil_s1(yb, w);
      T.s[2] += bil_s2(yb, w);
      T.s[3] += bil_s3(yb, w);
      T.s[4] += bil_u(yb, y);                   // u = ybar . y
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) wb[i] = yb[i];
    }
    vertex_row(ev, wb, t);                      // xbar += wbar eps/
    T.e[0] -= bil_s1(wb, x);                    // e_i = -wbar g^i x
    T.e[1] -= bil_s2(wb, x);
    T.e[2] -= bil_s3(wb, x);
  } else {
    vertex_row(ev, x, w);                       // w = x eps/
    if (in.post) {
      const Real* P = s_q + in.post * 5;
      prop_col(P, yb, wb);                      // wbar = P ybar
      T.s[0] += bil_s0(w, yb);                  // s_mu = w g^mu ybar
      T.s[1] += bil_s1(w, yb);
      T.s[2] += bil_s2(w, yb);
      T.s[3] += bil_s3(w, yb);
      T.s[4] += bil_u(y, yb);                   // u = y . ybar
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) wb[i] = yb[i];
    }
    vertex_col(ev, wb, t);                      // xbar += eps/ wbar
    T.e[0] -= bil_s1(x, wb);                    // e_i = -x g^i wbar
    T.e[1] -= bil_s2(x, wb);
    T.e[2] -= bil_s3(x, wb);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) xbar[i] += t[i];
}

// Reverse of one phase: every instruction passes its outputs' adjoints to its
// input (atomic adds: siblings share inputs) and its parameter terms to the
// FP64 accumulators.  Summed spin: item vp = one input variant and both
// photon polarisations.  The G = min(2^level, TEAM, 32) consecutive lanes
// that work on one instruction share its post set and photon: their
// parameter terms are summed by shuffles first, and one lane of the group
// adds them to the accumulators, so lanes do not contend for the same
// shared-memory words.
template <int TEAM, bool SUMMED, typename Real>
__device__ __forceinline__ void backprop_phase(const Phase& ph, int lane, const KParams& p,
                                               const Real* s_q, const Real* s_eps,
                                               const Real* s_spin, const Real* s_cur, Real* s_adj,
                                               double* s_acc_s, double* s_acc_e, float* s_part) {
  if constexpr (!SUMMED) {
    // one fixed state: both ranges in one loop (as in run_phase)
    const int c0 = ph.cnt[0], total = c0 + ph.cnt[1];
    for (int it = lane; it < total; it += TEAM) {
      const Instr in = ld_instr(p.instr + (it < c0 ? ph.beg[0] + it : ph.beg[1] + (it - c0)));
      const int pol = (int)((p.fixed_pol_bits >> in.photon) & 1u);
      Real x[8], xb[8], yb[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) xb[c] = (Real)0;
      if (in.src < 0) load8(s_spin + (in.side * 2 + (in.side == 0 ? p.fixed_sin : p.fixed_sout)) * 8, x);
      else load_cur(s_cur, in.src, 1, 0, x);
      load_cur(s_adj, in.dst, 1, 0, yb);
      Real y[8];
      if (in.post) load_cur(s_cur, in.dst, 1, 0, y);
      ParTerms<Real> T;
#pragma unroll
      for (int c = 0; c < 5; ++c) T.s[c] = (Real)0;
#pragma unroll
      for (int c = 0; c < 3; ++c) T.e[c] = (Real)0;
      backprop_terms(in, pol, x, yb, y, s_q, s_eps, T, xb);
      if (in.post && !(sizeof(Real) == 4 && in.pad)) {
        double* A = s_acc_s + in.post * 5;
#pragma unroll
        for (int c = 0; c < 5; ++c) atomicAdd(A + c, (double)T.s[c]);
      }
      if constexpr (sizeof(Real) == 4) {
        // mixed: FP32 partial sums of the photon set (flush_partials)
        if (in.pad) {
          float* A = s_part + (in.pad - 1) * 5;
#pragma unroll
          for (int c = 0; c < 5; ++c) atomicAdd(A + c, T.s[c]);
        }
        float* E = s_part + p.n_part * 5 + in.photon * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(E + c, T.e[c]);
      } else {
        double* E = s_acc_e + (in.photon * 2 + pol) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(E + c, (double)T.e[c]);
      }
      if (in.src >= 0) atomic_add_cur(s_adj + (size_t)in.src * 8, 0, xb);
    }
  } else {
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
      const int cnt = ph.cnt[slot];
      if (cnt == 0) continue;
      constexpr int WMAX = TEAM < 32 ? TEAM : 32;
      const int lg = ph.level[slot];
      const int total = cnt << lg;
      const int G = (1 << lg) < WMAX ? (1 << lg) : WMAX;
      for (int base = 0; base < total; base += TEAM) {
        // every lane of the warp runs the same rounds (the shuffles below)
        const int it = base + lane;
        const bool valid = it < total;
        const int i = valid ? it >> lg : 0;
        const int vp = it & ((1 << lg) - 1);
        const Instr in = ld_instr(p.instr + ph.beg[slot] + i);
        ParTerms<Real> T[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
          for (int c = 0; c < 5; ++c) T[q].s[c] = (Real)0;
#pragma unroll
          for (int c = 0; c < 3; ++c) T[q].e[c] = (Real)0;
        }
        if (valid) {
          Real x[8], xb[8], yb[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) xb[c] = (Real)0;
          const int nv = 2 << in.level;
          if (in.src < 0) load8(s_spin + (in.side * 2 + vp) * 8, x);
          else load_cur(s_cur, in.src, nv >> 1, vp, x);
          const int b = 1 + in.rank;
          const int lo = vp & ((1 << b) - 1);
          const int hi = (vp >> b) << (b + 1);
#pragma unroll
          for (int pol = 0; pol < 2; ++pol) {
            const int var = hi | (pol << b) | lo;
            Real y[8];
            load_cur(s_adj, in.dst, nv, var, yb);
            if (in.post) load_cur(s_cur, in.dst, nv, var, y);
            backprop_terms(in, pol, x, yb, y, s_q, s_eps, T[pol], xb);
          }
          if (in.src >= 0) atomic_add_cur(s_adj + (size_t)(in.src + vp) * 8, 0, xb);
        }
        // the propagator terms do not depend on the polarisation
#pragma unroll
        for (int c = 0; c < 5; ++c) T[0].s[c] += T[1].s[c];
        for (int off = 1; off < G; off <<= 1) {
#pragma unroll
          for (int c = 0; c < 5; ++c) T[0].s[c] += __shfl_xor_sync(0xffffffffu, T[0].s[c], off);
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) T[q].e[c] += __shfl_xor_sync(0xffffffffu, T[q].e[c], off);
        }
        if (valid && (vp & (G - 1)) == 0) {
          if constexpr (sizeof(Real) == 4) {
            // mixed: FP32 partial sums of the photon set (flush_partials);
            // the kept levels' propagator terms go to FP64 directly
            if (in.post) {
              if (in.pad) {
                float* A = s_part + (in.pad - 1) * 5;
#pragma unroll
                for (int c = 0; c < 5; ++c) atomicAdd(A + c, T[0].s[c]);
              } else {
                double* A = s_acc_s + in.post * 5;
#pragma unroll
                for (int c = 0; c < 5; ++c) atomicAdd(A + c, (double)T[0].s[c]);
              }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              float* E = s_part + p.n_part * 5 + (in.photon * 2 + q) * 3;
#pragma unroll
              for (int c = 0; c < 3; ++c) atomicAdd(E + c, T[q].e[c]);
            }
          } else {
            if (in.post) {
              double* A = s_acc_s + in.post * 5;
#pragma unroll
              for (int c = 0; c < 5; ++c) atomicAdd(A + c, (double)T[0].s[c]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              double* E = s_acc_e + (in.photon * 2 + q) * 3;
#pragma unroll
              for (int c = 0; c < 3; ++c) atomicAdd(E + c, (double)T[q].e[c]);
            }
          }
        }
      }
    }
  }
}

// Mixed adjoint: adds the FP32 partial sums to the FP64 accumulators and
// clears them; set >= 0 flushes that set's propagator slots and the photon
// terms, set < 0 the photon terms only.  Every slot of a set names a
// different propagator, so no two lanes add to the same word.  One fixed
// state keeps one polarisation per photon, the spin-summed form both.
template <int TEAM, int N, bool SUMMED>
__device__ __forceinline__ void flush_partials(const KParams& p, int set, int lane, float* s_part,
                                               double* s_acc_s, double* s_acc_e) {
  if (set >= 0) {
    const uint16_t* tab = p.part_tab + (size_t)set * p.n_part;
    for (int i = lane; i < p.n_part * 5; i += TEAM) {
      const int mask = __ldg(tab + i / 5);
      if (!mask) continue;
      s_acc_s[mask * 5 + i % 5] += (double)s_part[i];
      s_part[i] = 0.f;
    }
  }
  float* e = s_part + p.n_part * 5;
  if constexpr (SUMMED) {
    for (int i = lane; i < N * 6; i += TEAM) {
      s_acc_e[i] += (double)e[i];
      e[i] = 0.f;
    }
  } else {
    for (int i = lane; i < N * 3; i += TEAM) {
      const int j = i / 3;
      const int pol = (int)((p.fixed_pol_bits >> j) & 1u);
      s_acc_e[(j * 2 + pol) * 3 + i % 3] += (double)e[i];
      e[i] = 0.f;
    }
  }
}

}  // namespace

// Leaf sums of photon set se, Lsum[v] = sum_a L_a[v] and Rsum[v] = sum_b R'_b[v]
// for every variant v, into the adjoint slots of leaf 1 of each side (leaf 0
// when a side has one leaf); returns those slots.  The set's leaf adjoints
// are written only after the sums are read.
template <int TEAM, int NL, int NR, int NVL, int NVR, typename Real>
__device__ __forceinline__ void leaf_sums(const SetEntry& se, int lane, const Real* s_cur, Real* s_adj,
                                          int& sum_l, int& sum_r) {
  sum_l = NL > 1 ? se.leaf_l + NVL : se.leaf_l;
  sum_r = NR > 1 ? se.leaf_r + NVR : se.leaf_r;
  for (int it = lane; it < (NVL + NVR) * 8; it += TEAM) {
    const bool left = it < NVL * 8;
    const int q = left ? it : it - NVL * 8;
    const int cnt = left ? NL : NR, nv = left ? NVL : NVR;
    const Real* src = s_cur + (size_t)(left ? se.leaf_l : se.leaf_r) * 8;
    Real sum = (Real)0;
    for (int a = 0; a < cnt; ++a) sum += src[(size_t)a * nv * 8 + q];
    s_adj[(size_t)(left ? sum_l : sum_r) * 8 + q] = sum;
  }
}

// Up to 256 threads per block (one team when TEAM > 32); up to 255
// registers per thread for the FP64 forms that are spin-summed or have
// k >= 6 (shared memory holds those to a few warps per SM anyway), 128 for
// the others.
template <int K, bool SUMMED, typename Real, int TEAM, bool GMEM>
__global__ void __launch_bounds__(TEAM > 32 ? TEAM : 256,
                                  (sizeof(Real) == 8 && (SUMMED || K >= 6))
                                      ? 1
                                      : 65536 / ((TEAM > 32 ? TEAM : 256) * 128))
qed_adj_kernel(const KParams p) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr int NSUB = 1 << N;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int NVL = SUMMED ? (1 << (H + 1)) : 1;
  constexpr int NVR = SUMMED ? (1 << (R + 1)) : 1;
  constexpr int NL = [] { int f = 1; for (int i = 2; i <= H; ++i) f *= i; return f; }();
  constexpr int NR = [] { int f = 1; for (int i = 2; i <= R; ++i) f *= i; return f; }();
  static_assert(!SUMMED || TEAM == (1 << N), "one thread per polarisation pattern");

  extern __shared__ __align__(16) unsigned char smem[];
  // currents and their adjoints in shared memory, or (GMEM), where they do
  // not fit, in a global scratch slot of the team; the rest stays in shared
  // memory.  A separate instance, so that the shared-memory one addresses
  // its currents as shared memory.
  constexpr bool PART = sizeof(Real) == 4;   // FP32 partial sums per photon set
  const AdjLayout A = adj_layout(K, (int)sizeof(Real), GMEM ? 0 : p.ncur, SUMMED, PART ? p.n_part : 0);
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
  Real* s_cur;
  Real* s_adj;
  if constexpr (GMEM) {
    s_cur = reinterpret_cast<Real*>(static_cast<unsigned char*>(p.adj_scratch) +
                                    ((size_t)blockIdx.x * tpc + team) * (size_t)p.adj_scratch_team);
    s_adj = s_cur + (size_t)p.ncur * 8;
  } else {
    s_cur = reinterpret_cast<Real*>(base + L.cur);
    s_adj = reinterpret_cast<Real*>(base + A.adj);
  }
  Real* s_mbar = reinterpret_cast<Real*>(base + A.mbar);
  double* s_acc_s = reinterpret_cast<double*>(base + A.acc_s);
  double* s_acc_e = reinterpret_cast<double*>(base + A.acc_e);
  double* s_kbar = reinterpret_cast<double*>(base + A.kbar);
  float* s_part = reinterpret_cast<float*>(base + A.part);

  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    const long long ptc = valid ? pt : p.n - 1;

    // ---- 1. forward pass
    point_setup<K, Real, TEAM>(p, lane, ptc, s_mom, s_q, s_eps, s_spin,
                               reinterpret_cast<double*>(base + L.w), reinterpret_cast<float*>(base + L.momf));
    for (int ph = 0; ph < p.n_stored_phases; ++ph) {
      run_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + ph), lane, p, s_q, s_eps, s_spin, s_cur);
      team_sync<TEAM>();
    }
    Acc<Real> acc[SUMMED ? 4 : 1];
    for (int s = 0; s < p.n_sets; ++s) {
      const SetEntry se = p.sets[s];
      for (int t = 0; t < p.n_set_phases; ++t) {
        run_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + se.phase0 + t), lane, p, s_q, s_eps, s_spin,
                                      s_cur);
        team_sync<TEAM>();
      }
      if constexpr (!SUMMED && sizeof(Real) == 4) {
        // one fixed state, mixed: the per-diagram joins.  They are few, and
        // FP32 leaf sums would lose the accuracy of the compensated diagram
        // sum where the diagrams cancel.
        join_set<K, false, Real, TEAM, 1>(se, nullptr, lane, s_cur, acc);
      } else {
        // M_l = sum_{a,b} R'_b . L_a = (sum_b R'_b) . (sum_a L_a): the backward
        // pass needs only M_l, so the set's leaves are summed first and each
        // state takes one dot (one compensated step in the mixed form)
        int sum_l, sum_r;
        leaf_sums<TEAM, NL, NR, NVL, NVR, Real>(se, lane, s_cur, s_adj, sum_l, sum_r);
        team_sync<TEAM>();
        if constexpr (SUMMED) {
          const unsigned tv = __ldg(p.lane_tab + ((size_t)s << N) + ((unsigned)lane & ALL));
          const int vl = (int)(tv & 0xffu) << 1, vr = (int)(tv >> 8) << 1;
#pragma unroll
          for (int si = 0; si < 2; ++si)
#pragma unroll
            for (int so = 0; so < 2; ++so) {
              Real l[8], r[8];
              load_cur(s_adj, sum_l, NVL, vl + si, l);
              load_cur(s_adj, sum_r, NVR, vr + so, r);
              Real yr = (Real)0, yi = (Real)0;
              dot_acc(r, l, yr, yi);
              acc[si * 2 + so].add(yr, yi);
            }
        } else if (lane == 0) {
          Real l[8], r[8];
          load_cur(s_adj, sum_l, 1, 0, l);
          load_cur(s_adj, sum_r, 1, 0, r);
          Real yr = (Real)0, yi = (Real)0;
          dot_acc(r, l, yr, yi);
          acc[0].add(yr, yi);
        }
      }
      team_sync<TEAM>();
    }

    // ---- 2. |M|^2 and the seeds conj(M)
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
    } else {
      const double re = team_sum<TEAM>(acc[0].vre(), s_red);
      const double im = team_sum<TEAM>(acc[0].vim(), s_red);
      m2 = re * re + im * im;
      if (lane == 0) { s_mbar[0] = (Real)re; s_mbar[1] = (Real)(-im); }
    }
    if (lane == 0 && valid && p.out) p.out[pt] = m2 * p.coupling;

    // zero the adjoints of the kept currents and the accumulators
    {
      const int nst = p.ncur_stored * 8;
      for (int i = lane; i < nst; i += TEAM) s_adj[i] = (Real)0;
      for (int i = lane; i < NSUB * 5; i += TEAM) s_acc_s[i] = 0.0;
      for (int i = lane; i < N * 6; i += TEAM) s_acc_e[i] = 0.0;
      for (int i = lane; i < N * 4; i += TEAM) s_kbar[i] = 0.0;
      if constexpr (PART)
        for (int i = lane; i < p.n_part * 5 + N * (SUMMED ? 6 : 3); i += TEAM) s_part[i] = 0.f;
    }
    team_sync<TEAM>();

    // ---- 3. per photon set: rebuild, transposed joins, reverse phases
    for (int s = 0; s < p.n_sets; ++s) {
      const SetEntry se = p.sets[s];
      for (int i = p.ncur_stored * 8 + lane; i < p.ncur * 8; i += TEAM) s_adj[i] = (Real)0;
      for (int t = 0; t < p.n_set_phases; ++t) {
        run_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + se.phase0 + t), lane, p, s_q, s_eps, s_spin,
                                      s_cur);
        team_sync<TEAM>();
      }
      // transposed joins.  M_l = sum_{a,b} R'_b[vR] . L_a[vL], so the adjoint
      // of every left leaf a is the same, Lbar[vL] = sum_vR Mbar_l Rsum[vR]
      // with Rsum = sum_b R'_b, and likewise Rbar[vR] = sum_vL Mbar_l Lsum[vL]:
      // the leaf sums first (into the adjoint slots of leaf 1 of each side,
      // or leaf 0 when a side has one leaf: free until the copies below),
      // then one product per leaf variant into the adjoint slots of leaf 0,
      // then a copy to every other leaf.
      {
        int sum_l, sum_r;
        leaf_sums<TEAM, NL, NR, NVL, NVR, Real>(se, lane, s_cur, s_adj, sum_l, sum_r);
        team_sync<TEAM>();
        constexpr int NITEM = (NVL + NVR) * 4;
        constexpr int PER = (NITEM + TEAM - 1) / TEAM;
        Real br[PER], bi[PER];
#pragma unroll
        for (int k2 = 0; k2 < PER; ++k2) {
          const int it = lane + k2 * TEAM;
          br[k2] = bi[k2] = (Real)0;
          if (it >= NITEM) continue;
          // item (side, variant v, Dirac component c): one complex output
          const bool left = it < NVL * 4;
          const int q = left ? it : it - NVL * 4;
          const int v = q >> 2, c = q & 3;
          const Real* other = s_adj + (size_t)(left ? sum_r : sum_l) * 8;
          const int nvo = left ? NVR : NVL;
          if constexpr (SUMMED) {
            constexpr int ROW = (1 << H) + (1 << R);
            const uint16_t* dep = p.dep_tab + (size_t)s * ROW;
            const unsigned cv = __ldg(dep + (left ? 0 : (1 << H)) + (v >> 1));
            for (int w = 0; w < nvo; ++w) {
              const unsigned cw = __ldg(dep + (left ? (1 << H) : 0) + (w >> 1));
              const int si = left ? (v & 1) : (w & 1), so = left ? (w & 1) : (v & 1);
              const int lam = si | (so << 1) | (int)((cv | cw) << 2);
              const Real mr = s_mbar[2 * lam], mi = s_mbar[2 * lam + 1];
              const Real xr = other[w * 8 + 2 * c], xi = other[w * 8 + 2 * c + 1];
              br[k2] += mr * xr - mi * xi;
              bi[k2] += mr * xi + mi * xr;
            }
          } else {
            const Real mr = s_mbar[0], mi = s_mbar[1];
            const Real xr = other[2 * c], xi = other[2 * c + 1];
            br[k2] = mr * xr - mi * xi;
            bi[k2] = mr * xi + mi * xr;
          }
        }
        team_sync<TEAM>();   // the sums are read; the slots may be overwritten
#pragma unroll
        for (int k2 = 0; k2 < PER; ++k2) {
          const int it = lane + k2 * TEAM;
          if (it >= NITEM) continue;
          const bool left = it < NVL * 4;
          const int q = left ? it : it - NVL * 4;
          const int v = q >> 2, c = q & 3;
          const int cnt = left ? NL : NR, nv = left ? NVL : NVR;
          Real* dst = s_adj + (size_t)(left ? se.leaf_l : se.leaf_r) * 8 + v * 8 + 2 * c;
          for (int a = 0; a < cnt; ++a) {
            dst[(size_t)a * nv * 8] = br[k2];
            dst[(size_t)a * nv * 8 + 1] = bi[k2];
          }
        }
      }
      team_sync<TEAM>();
      for (int t = p.n_set_phases - 1; t >= 0; --t) {
        backprop_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + se.phase0 + t), lane, p, s_q, s_eps, s_spin,
                                           s_cur, s_adj, s_acc_s, s_acc_e, s_part);
        team_sync<TEAM>();
      }
      if constexpr (PART) {
        flush_partials<TEAM, N, SUMMED>(p, s, lane, s_part, s_acc_s, s_acc_e);
        team_sync<TEAM>();
      }
    }

    // ---- 4. kept inner levels, deepest first
    for (int ph = p.n_stored_phases - 1; ph >= 0; --ph) {
      backprop_phase<TEAM, SUMMED, Real>(ld_phase(p.phases + ph), lane, p, s_q, s_eps, s_spin, s_cur, s_adj,
                                         s_acc_s, s_acc_e, s_part);
      team_sync<TEAM>();
    }
    if constexpr (PART) {
      flush_partials<TEAM, N, SUMMED>(p, -1, lane, s_part, s_acc_s, s_acc_e);
      team_sync<TEAM>();
    }

    // ---- 5. parameters -> outgoing photon momenta (FP64)
#pragma unroll 1
    for (int mask = lane; mask < NSUB; mask += TEAM) {
      if (mask == 0 || mask == (int)ALL) continue;
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
      // df/dQ_T^mu, in place of the subset's accumulator
      double* Ac = s_acc_s + mask * 5;
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
    }
    team_sync<TEAM>();
    // Q_T = p + k_0 - sum_{j in T, j >= 1} k_j: d f/d k_j^mu = -sum_{T containing j}
    // df/dQ_T^mu, one lane per (j, mu) over the 2^(n-1) subsets that contain j
    // (plain stores: no two lanes share a word)
    for (int it = lane; it < K * 4; it += TEAM) {
      const int j = 1 + (it >> 2), mu = it & 3;
      const int lo = (1 << j) - 1;
      double a = 0.0;
#pragma unroll 1
      for (int r = 0; r < (1 << (N - 1)) - 1; ++r)   // r = 2^(n-1) - 1 would be the full set
        a += s_acc_s[(((r >> j) << (j + 1)) | (1 << j) | (r & lo)) * 5 + mu];
      s_kbar[4 * j + mu] = -a;
    }
    team_sync<TEAM>();
    for (int it = lane; it < 2 * N; it += TEAM) {
      const int j = it >> 1, pb = it & 1;
      if (j == 0) continue;
      const double* E = s_acc_e + (j * 2 + pb) * 3;
      double d[3][3];
      dpol(s_mom + 4 * (j + 2), pb, d);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double g = 2.0 * (E[0] * d[a][0] + E[1] * d[a][1] + E[2] * d[a][2]);
        atomicAdd(s_kbar + 4 * j + 1 + a, g);
      }
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

// ----------------------------------------------------------- dispatch
using KernelFn = void (*)(const KParams);

struct KernelChoice {
  KernelFn fn;
  int team;
};

template <int K, bool SUMMED>
constexpr int adj_team() {
  if constexpr (SUMMED) return 1 << (K + 1);
  else return K == 1 ? 2 : (K == 2 ? 4 : (K == 3 ? 8 : (K == 4 ? 16 : 32)));
}

template <int K, bool SUMMED>
KernelChoice pick_adj(bool mixed) {
  constexpr int T = adj_team<K, SUMMED>();
  if (mixed) return {qed_adj_kernel<K, SUMMED, float, T, false>, T};
  return {qed_adj_kernel<K, SUMMED, double, T, false>, T};
}

KernelChoice adjoint_kernel(int k, bool summed, bool mixed) {
#define QED_CASE(KK) \
  case KK: return summed ? pick_adj<KK, true>(mixed) : pick_adj<KK, false>(mixed);
  switch (k) {
    QED_CASE(1) QED_CASE(2) QED_CASE(3) QED_CASE(4) QED_CASE(5) QED_CASE(6) QED_CASE(7)
    default: return KernelChoice{nullptr, 0};
  }
#undef QED_CASE
}

// Global-scratch instances: only the spin-summed FP64 k = 6, 7 adjoints can
// miss shared memory.
KernelChoice adjoint_kernel_gmem(int k, bool summed, bool mixed) {
  if (!summed || mixed) return KernelChoice{nullptr, 0};
  if (k == 7) return {qed_adj_kernel<7, true, double, adj_team<7, true>(), true>, adj_team<7, true>()};
  if (k == 6) return {qed_adj_kernel<6, true, double, adj_team<6, true>(), true>, adj_team<6, true>()};
  return KernelChoice{nullptr, 0};
}

}  // namespace qed
