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

#include "qed_device.cuh"

namespace qed {

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM <= 32) __syncwarp();
  else __syncthreads();
}

template <int TEAM>
__device__ __forceinline__ double team_sum(double v, double* red) {
#pragma unroll
  for (int off = (TEAM < 32 ? TEAM : 32) / 2; off > 0; off >>= 1)
    v += __shfl_xor_sync(0xffffffffu, v, off);
  if constexpr (TEAM > 32) {
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < TEAM / 32; ++i) s += red[i];
    v = s;
    __syncthreads();
  }
  return v;
}

template <typename Real>
__device__ __forceinline__ void load8(const Real* p, Real x[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = p[i];
}
template <typename Real>
__device__ __forceinline__ void store8(Real* p, const Real x[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = x[i];
}

__device__ __forceinline__ Instr ld_instr(const Instr* p) {
  int4 v = __ldg(reinterpret_cast<const int4*>(p));
  Instr in;
  static_assert(sizeof(Instr) == sizeof(int4), "Instr size");
  memcpy(&in, &v, sizeof(Instr));
  return in;
}

// One V (+S1) instruction for spin variant v.
template <bool SUMMED, typename Real>
__device__ __forceinline__ void apply_instr(const Instr& in, int v, const KParams& p,
                                            const Real* s_q, const Real* s_eps,
                                            const Real* s_spin, Real* s_cur) {
  int pol, vp;
  if constexpr (SUMMED) {
    const int b = 1 + in.rank;
    pol = (v >> b) & 1;
    vp = (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b);
  } else {
    pol = (int)((p.fixed_pol_bits >> in.photon) & 1u);
    vp = 0;
  }
  Real x[8], y[8];
  if (in.src < 0) {
    const int e = SUMMED ? vp : (in.side == 0 ? p.fixed_sin : p.fixed_sout);
    load8(s_spin + (in.side * 2 + e) * 8, x);
  } else {
    load8(s_cur + (size_t)(in.src + vp) * 8, x);
  }
  const Real* e3 = s_eps + (in.photon * 2 + pol) * 4;
  Real ev[3] = {e3[0], e3[1], e3[2]};
  if (in.side == 0) vertex_col(ev, x, y); else vertex_row(ev, x, y);
  if (in.post) {
    const Real* P = s_q + in.post * 5;
    if (in.side == 0) prop_col(P, y, x); else prop_row(P, y, x);
    store8(s_cur + (size_t)(in.dst + v) * 8, x);
  } else {
    store8(s_cur + (size_t)(in.dst + v) * 8, y);
  }
}

template <int TEAM, bool SUMMED, typename Real>
__device__ __forceinline__ void run_phase(const Phase& ph, int lane, const KParams& p,
                                          const Real* s_q, const Real* s_eps,
                                          const Real* s_spin, Real* s_cur) {
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int cnt = ph.cnt[slot];
    if (cnt == 0) continue;
    const int lg = SUMMED ? ph.level[slot] + 1 : 0;
    const int total = cnt << lg;
    for (int it = lane; it < total; it += TEAM) {
      const int i = it >> lg;
      const int v = it & ((1 << lg) - 1);
      const Instr in = ld_instr(p.instr + ph.beg[slot] + i);
      apply_instr<SUMMED, Real>(in, v, p, s_q, s_eps, s_spin, s_cur);
    }
  }
}

__device__ __forceinline__ Phase ld_phase(const Phase* p) {
  Phase ph;
  const int* s = reinterpret_cast<const int*>(p);
  int* d = reinterpret_cast<int*>(&ph);
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = __ldg(s + i);
  return ph;
}

// Per-state accumulator of the diagram sum.
template <typename Real> struct Acc;
template <> struct Acc<double> {
  double re = 0.0, im = 0.0;
  __device__ __forceinline__ void add(double r, double i) { re += r; im += i; }
  __device__ __forceinline__ double vre() const { return re; }
  __device__ __forceinline__ double vim() const { return im; }
};
template <> struct Acc<float> {
  float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
  __device__ __forceinline__ void add(float r, float i) { kahan_add(re, cre, r); kahan_add(im, cim, i); }
  __device__ __forceinline__ double vre() const { return (double)re - (double)cre; }
  __device__ __forceinline__ double vim() const { return (double)im - (double)cim; }
};

template <int K, bool SUMMED, typename Real, int TEAM>
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
  constexpr int BC = NR >= 2 ? 2 : 1;

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

    // ---- a1: load the point
    for (int i = lane; i < NS * 4; i += TEAM) s_mom[i] = __ldg(p.mom + ptc * (NS * 4) + i);
    team_sync<TEAM>();

    // ---- a2/a3: external states and propagators (FP64)
    for (int it = lane; it < 4 + 2 * N + NSUB; it += TEAM) {
      if (it < 4) {
        const int side = it >> 1, e = it & 1;
        double s[8];
        make_spinor(s_mom + (side ? 8 : 0), e, p.mass, side == 1, s);
#pragma unroll
        for (int c = 0; c < 8; ++c) s_spin[(side * 2 + e) * 8 + c] = (Real)s[c];
      } else if (it < 4 + 2 * N) {
        const int j = (it - 4) >> 1, pb = (it - 4) & 1;
        double e[3];
        make_pol(s_mom + 4 * (j == 0 ? 1 : j + 2), pb, e);
        Real* d = s_eps + (j * 2 + pb) * 4;
        d[0] = (Real)e[0]; d[1] = (Real)e[1]; d[2] = (Real)e[2]; d[3] = (Real)0;
      } else {
        const unsigned mask = (unsigned)(it - 4 - 2 * N);
        Real* d = s_q + mask * 5;
        if (mask == 0 || mask == ALL) {
#pragma unroll
          for (int c = 0; c < 5; ++c) d[c] = (Real)0;
        } else {
          double P[5];
          make_prop(s_mom, N, mask, p.mass, P);
#pragma unroll
          for (int c = 0; c < 5; ++c) d[c] = (Real)P[c];
        }
      }
    }
    team_sync<TEAM>();

    // ---- a4/a5: currents kept for the whole point
    for (int ph = 0; ph < p.n_stored_phases; ++ph) {
      const Phase P = ld_phase(p.phases + ph);
      run_phase<TEAM, SUMMED, Real>(P, lane, p, s_q, s_eps, s_spin, s_cur);
      team_sync<TEAM>();
    }

    Acc<Real> acc[SUMMED ? 4 : 1];
    for (int s = 0; s < p.n_sets; ++s) {
      const SetEntry se = p.sets[s];
      for (int t = 0; t < p.n_set_phases; ++t) {
        const Phase P = ld_phase(p.phases + se.phase0 + t);
        run_phase<TEAM, SUMMED, Real>(P, lane, p, s_q, s_eps, s_spin, s_cur);
        team_sync<TEAM>();
      }
      // ---- a6/a7: S2 joins of every diagram whose left photon set is S
      if constexpr (SUMMED) {
        const unsigned c = (unsigned)lane;
        const int vl = (int)pext_bits(c, se.mask, N) << 1;
        const int vr = (int)pext_bits(c, ALL & ~se.mask, N) << 1;
        const Real* Lb = s_cur + (size_t)(se.leaf_l + vl) * 8;
        const Real* Rb = s_cur + (size_t)(se.leaf_r + vr) * 8;
        for (int b0 = 0; b0 < NR; b0 += BC) {
          Real rw[BC][2][8];
#pragma unroll
          for (int bb = 0; bb < BC; ++bb)
#pragma unroll
            for (int so = 0; so < 2; ++so) load8(Rb + (size_t)((b0 + bb) * NVR + so) * 8, rw[bb][so]);
          for (int a = 0; a < NL; ++a) {
            Real lc[2][8];
#pragma unroll
            for (int si = 0; si < 2; ++si) load8(Lb + (size_t)(a * NVL + si) * 8, lc[si]);
#pragma unroll
            for (int si = 0; si < 2; ++si)
#pragma unroll
              for (int so = 0; so < 2; ++so) {
                Real re = (Real)0, im = (Real)0;
#pragma unroll
                for (int bb = 0; bb < BC; ++bb) {
                  if constexpr (sizeof(Real) == 8) {
                    dot_acc(rw[bb][so], lc[si], acc[si * 2 + so].re, acc[si * 2 + so].im);
                  } else {
                    re = (Real)0; im = (Real)0;
                    dot_acc(rw[bb][so], lc[si], re, im);
                    acc[si * 2 + so].add(re, im);
                  }
                }
              }
          }
        }
      } else {
        for (int q = lane; q < NL * NR; q += TEAM) {
          const int a = q / NR, b = q - a * NR;
          Real lc[8], rw[8];
          load8(s_cur + (size_t)(se.leaf_l + a) * 8, lc);
          load8(s_cur + (size_t)(se.leaf_r + b) * 8, rw);
          if constexpr (sizeof(Real) == 8) {
            dot_acc(rw, lc, acc[0].re, acc[0].im);
          } else {
            Real re = (Real)0, im = (Real)0;
            dot_acc(rw, lc, re, im);
            acc[0].add(re, im);
          }
        }
      }
      team_sync<TEAM>();
    }

    // ---- a8/a9: square, spin sum in FP64, store
    double m2;
    if constexpr (SUMMED) {
      double part = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double re = acc[i].vre(), im = acc[i].vim();
        part = fma(re, re, fma(im, im, part));
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
template <int K, bool SUMMED>
constexpr int team_of() {
  if constexpr (SUMMED) return 1 << (K + 1);
  else return K == 1 ? 2 : (K == 2 ? 4 : (K == 3 ? 8 : (K == 4 ? 16 : 32)));
}

using KernelFn = void (*)(const KParams);

template <int K, bool SUMMED>
KernelFn pick(bool mixed) {
  constexpr int T = team_of<K, SUMMED>();
  return mixed ? qed_fwd_kernel<K, SUMMED, float, T> : qed_fwd_kernel<K, SUMMED, double, T>;
}

struct KernelChoice {
  KernelFn fn;
  int team;
};

KernelChoice forward_kernel(int k, bool summed, bool mixed) {
#define QED_CASE(KK)                                                                  \
  case KK:                                                                            \
    return summed ? KernelChoice{pick<KK, true>(mixed), team_of<KK, true>()}          \
                  : KernelChoice{pick<KK, false>(mixed), team_of<KK, false>()};
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
