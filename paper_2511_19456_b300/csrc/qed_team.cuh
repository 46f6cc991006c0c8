// Team-level building blocks shared by the forward and adjoint kernels: team
// synchronisation and reductions, shared-memory current access, and the
// execution of one phase of the linear schedule (V with optional S1 per spin
// variant).
#pragma once

#include <cuda_runtime.h>

#include "qed_device.cuh"

namespace qed {

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM == 1) return;      // a thread sees its own shared-memory writes
  else if constexpr (TEAM <= 32) __syncwarp();
  else __syncthreads();
}

template <int TEAM>
__device__ __forceinline__ double team_sum(double v, double* red) {
#pragma unroll
  for (int off = (TEAM < 32 ? TEAM : 32) / 2; off > 0; off >>= 1)
    v += __shfl_xor_sync(0xffffffffu, v, off);
  if constexpr (TEAM > 32) {
    const int w = (threadIdx.x & (TEAM - 1)) >> 5;   // warp within the team
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

// Float-float addition (hi, lo) += (bh, bl): Knuth's TwoSum of the high
// parts, the low parts added to its error, then renormalised (Dekker's
// Fast2Sum), about 2^-48 relative; all on the FP32 pipe.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum_f(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// The team's sum of one float-float value per lane (a compensated diagram
// sum re - c as the pair (re, -c)), returned to lane 0 of the team: warp
// shuffles, then through shared memory across the warps of a team of W > 1.
// Every lane of the team must call it.
template <int TEAM, int W = (TEAM > 32 ? TEAM / 32 : 1)>
__device__ __forceinline__ void team_sum_ff(float& hi, float& lo, int lane, float* red) {
  constexpr int WL = TEAM / W;
#pragma unroll
  for (int off = WL / 2; off > 0; off >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, off);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, off);
    ff_add(hi, lo, bh, bl);
  }
  if constexpr (W > 1) {
    const int wi = lane / WL;
    __syncthreads();
    if (lane % WL == 0) { red[2 * wi] = hi; red[2 * wi + 1] = lo; }
    __syncthreads();
    if (lane == 0)
      for (int w = 1; w < W; ++w) ff_add(hi, lo, red[2 * w], red[2 * w + 1]);
  }
}

// Complex pairs of the working precision (the adjoint's accumulators).
template <typename Real> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

// contiguous layout: variant v of node base at 8*(base+v) reals
__device__ __forceinline__ void load_cur(const float* cur, int base, int nv, int v, float x[8]) {
  const float4* q = reinterpret_cast<const float4*>(cur + (size_t)(base + v) * 8);
  const float4 a = q[0], b = q[1];
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void store_cur(float* cur, int base, int nv, int v, const float x[8]) {
  float4* q = reinterpret_cast<float4*>(cur + (size_t)(base + v) * 8);
  q[0] = make_float4(x[0], x[1], x[2], x[3]);
  q[1] = make_float4(x[4], x[5], x[6], x[7]);
}
__device__ __forceinline__ void load_cur(const double* cur, int base, int nv, int v, double x[8]) {
  const double2* q = reinterpret_cast<const double2*>(cur + (size_t)(base + v) * 8);
#pragma unroll
  for (int i = 0; i < 4; ++i) { const double2 a = q[i]; x[2 * i] = a.x; x[2 * i + 1] = a.y; }
}
__device__ __forceinline__ void store_cur(double* cur, int base, int nv, int v, const double x[8]) {
  double2* q = reinterpret_cast<double2*>(cur + (size_t)(base + v) * 8);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = make_double2(x[2 * i], x[2 * i + 1]);
}
// External spinors: 8 contiguous reals.
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

// Vertex (+ propagation) of one input current x for photon polarisation pol,
// stored as variant v of the instruction's node.  One code path for both
// sides, so that lanes of one round with items of both sides run the same
// instructions: for a real 3-vector a, x (sigma.a) = (sigma.a') x with
// a' = (ax, -ay, az), so the row vertex x eps/ is the column form with
// eps~ = (-ex, ey, -ez) and the row propagation x (Q/ + m)/D the column form
// with Q/D replaced by (-qx, qy, -qz); sign flips are exact.
template <typename Real>
__device__ __forceinline__ void vertex_store(const Instr& in, const Real x[8], int pol, int v, int nv,
                                             const Real* s_q, const Real* s_eps, Real* s_cur) {
  const Real* e3 = s_eps + (in.photon * 2 + pol) * 4;
  const Real sg = in.side ? (Real)-1 : (Real)1;
  const Real ev[3] = {sg * e3[0], e3[1], sg * e3[2]};
  Real y[8], z[8];
  vertex_col(ev, x, y);
  if (in.post) {
    const Real* P = s_q + in.post * 5;
    const Real Pt[5] = {P[0], P[1], sg * P[2], P[3], sg * P[4]};
    prop_col(Pt, y, z);
    store_cur(s_cur, in.dst, nv, v, z);
  } else {
    store_cur(s_cur, in.dst, nv, v, y);
  }
}

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
  Real x[8];
  if (in.src < 0) {
    const int e = SUMMED ? vp : (in.side == 0 ? p.fixed_sin : p.fixed_sout);
    load8(s_spin + (in.side * 2 + e) * 8, x);
  } else {
    load_cur(s_cur, in.src, 0, vp, x);
  }
  vertex_store(in, x, pol, v, 0, s_q, s_eps, s_cur);
}

template <int TEAM, bool SUMMED, typename Real>
__device__ __forceinline__ void run_phase(const Phase& ph, int lane, const KParams& p,
                                          const Real* s_q, const Real* s_eps,
                                          const Real* s_spin, Real* s_cur) {
  if constexpr (!SUMMED) {
    // one fixed state: one item per instruction, both ranges in one loop,
    // so that the short range does not take a round of mostly idle lanes
    const int c0 = ph.cnt[0], total = c0 + ph.cnt[1];
    for (int it = lane; it < total; it += TEAM) {
      const int idx = it < c0 ? ph.beg[0] + it : ph.beg[1] + (it - c0);
      apply_instr<false, Real>(ld_instr(p.instr + idx), 0, p, s_q, s_eps, s_spin, s_cur);
    }
  } else {
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
      const int cnt = ph.cnt[slot];
      if (cnt == 0) continue;
      const int lg = ph.level[slot] + 1;
      const int total = cnt << lg;
      for (int it = lane; it < total; it += TEAM) {
        const int i = it >> lg;
        const int v = it & ((1 << lg) - 1);
        const Instr in = ld_instr(p.instr + ph.beg[slot] + i);
        apply_instr<true, Real>(in, v, p, s_q, s_eps, s_spin, s_cur);
      }
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
// Kahan-compensated: the represented value is (re - cre, im - cim).  A group of
// diagrams is accumulated by an FMA chain that starts from -c (the first
// step of a Kahan update), then committed with the remaining two steps.
template <> struct Acc<float> {
  float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
  __device__ __forceinline__ void start(float& yr, float& yi) const { yr = -cre; yi = -cim; }
  __device__ __forceinline__ void commit(float yr, float yi) {
    const float tr = __fadd_rn(re, yr), ti = __fadd_rn(im, yi);
    cre = __fsub_rn(__fsub_rn(tr, re), yr);
    cim = __fsub_rn(__fsub_rn(ti, im), yi);
    re = tr;
    im = ti;
  }
  __device__ __forceinline__ void add(float r, float i) {
    float yr, yi;
    start(yr, yi);
    commit(__fadd_rn(yr, r), __fadd_rn(yi, i));
  }
  __device__ __forceinline__ double vre() const { return (double)re - (double)cre; }
  __device__ __forceinline__ double vim() const { return (double)im - (double)cim; }
};

// Minkowski product in FP64.
__device__ __forceinline__ double mdot(const double* a, const double* b) {
  return fma(a[0], b[0], fma(-a[1], b[1], fma(-a[2], b[2], -a[3] * b[3])));
}

// Momentum slot of photon j (slot 1: the incoming photon, j = 0).
__device__ __forceinline__ int photon_slot_of(int j) { return j == 0 ? 1 : j + 2; }

// The Lorentz invariants of one point from which the mixed form sums every
// propagator denominator, in FP64 (a3).  Photon j sits in momentum slot 1
// (j = 0, incoming) or j + 2; sigma_0 = +1, sigma_j = -1 (j >= 1).
//   1. the Minkowski products, one per lane and item, so that every lane
//      issues the same four FP64 instructions:
//        w[0] = p.p, w[1] = p'.p', w[2 + j] = k_j.k_j, w[2 + N + j] = p.k_j,
//        w[2 + 2N + j] = p'.k_j, w[2 + 3N + r] = k_a.k_b (a < b, r the
//        rank of (a, b) in row order);
//   2. their signed combinations, one FMA per lane and item, at
//      c = w + n_products(N):
//        c[0], c[1] = q.q - m^2 (q = p, p'),
//        c[2 + j] = k_j.k_j + 2 sigma_j p.k_j,
//        c[2 + N + j] = k_j.k_j - 2 sigma_j p'.k_j,
//        c[2 + 2N + a N + b] = 2 sigma_a sigma_b k_a.k_b (a < b),
//        c[2 + 2N + N N] = 0,
//      so that D_T = Q_T^2 - m^2 with Q_T = p + sum_{j in T} sigma_j k_j is
//        c[0] + sum_{j in T} c[2 + j] + sum_{a<b in T} c[2 + 2N + a N + b],
//      and, with Q_T = p' - sum_{j in U} sigma_j k_j (U the complement of T),
//        c[1] + sum_{j in U} c[2 + N + j] + sum_{a<b in U} c[2 + 2N + a N + b].
// Returns after a team barrier, with w and c complete.
template <int N, int TEAM>
__device__ __forceinline__ void setup_invariants(int lane, double mass, const double* s_mom, double* s_w) {
  constexpr int NP = 2 + 3 * N + N * (N - 1) / 2;
  constexpr int NC = 2 + 2 * N + N * (N - 1) / 2;
  for (int it = lane; it < NP; it += TEAM) {
    int a, b;
    if (it < 2) {
      a = b = it == 0 ? 0 : 2;
    } else if (it < 2 + N) {
      a = b = photon_slot_of(it - 2);
    } else if (it < 2 + 3 * N) {
      a = it < 2 + 2 * N ? 0 : 2;
      b = photon_slot_of((it - 2) % N);
    } else {
      int r = it - 2 - 3 * N, i = 0;
      while (r >= N - 1 - i) { r -= N - 1 - i; ++i; }
      a = photon_slot_of(i);
      b = photon_slot_of(i + 1 + r);
    }
    s_w[it] = mdot(s_mom + 4 * a, s_mom + 4 * b);
  }
  team_sync<TEAM>();
  double* c = s_w + NP;
  for (int it = lane; it < NC; it += TEAM) {
    double f, x, y;
    int dst = it;
    if (it < 2) {
      f = -mass; x = mass; y = s_w[it];
    } else if (it < 2 + 2 * N) {
      const int j = (it - 2) % N;
      const bool out = it >= 2 + N;
      f = (j == 0) != out ? 2.0 : -2.0;   // in: 2 sigma_j; out: -2 sigma_j
      x = s_w[(out ? 2 + 2 * N : 2 + N) + j];
      y = s_w[2 + j];
    } else {
      int r = it - 2 - 2 * N, i = 0;
      const int rank = r;
      while (r >= N - 1 - i) { r -= N - 1 - i; ++i; }
      f = i == 0 ? -2.0 : 2.0;            // 2 sigma_i sigma_j (j >= 1)
      x = s_w[2 + 3 * N + rank];
      y = 0.0;
      dst = 2 + 2 * N + i * N + (i + 1 + r);
    }
    c[dst] = fma(f, x, y);
  }
  if (lane == 0) c[2 + 2 * N + N * N] = 0.0;
  team_sync<TEAM>();
}

// Per point: momenta into shared memory, the propagator table (a3) and the
// external states (a2).
//
// FP64 form: Q_T = p + sum_{j in T} sigma_j k_j (sigma = +1 for the incoming
// photon, -1 for the outgoing ones) and D_T = Q_T^2 - m^2, both in FP64.
//
// Mixed form: the same D_T, in FP64, but summed from the Lorentz invariants
// and their signed combinations computed once per point (setup_invariants),
//   D_T = (p^2 - m^2) + sum_{j in T} (k_j^2 + 2 sigma_j p.k_j)
//         + sum_{i<j in T} 2 sigma_i sigma_j k_i.k_j,
// or, for |T| > n/2, from the outgoing electron's side with the complement,
//   Q_T = p' - sum_{j not in T} sigma_j k_j,
// so that no denominator sums more than n/2 photons.  Q_T itself, which only
// enters the FP32 numerator, is summed in float-float arithmetic on the FP32
// pipe (Knuth's TwoSum on the high parts, the low parts added) and rounded
// once, as accurate as rounding an FP64 sum.  This keeps the FP64 pipe (1/64
// of the FP32 rate) off the critical path where a thread builds several
// subsets or subsets of many photons (n >= 7); with one subset of few photons
// per thread the FP64 form is as fast, and it is used there.
// FORCE_INV: take the invariant-based mixed form whatever the team size.
template <int K, typename Real, int TEAM, bool FORCE_INV = false>
__device__ __forceinline__ void point_setup(const KParams& p, int lane, long long ptc, double* s_mom,
                                          Real* s_q, Real* s_eps, Real* s_spin, double* s_w,
                                          float* s_momf) {
  constexpr int N = K + 1;
  constexpr int NS = K + 3;
  constexpr int NSUB = 1 << N;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr bool INV = sizeof(Real) == 4 && (FORCE_INV || NSUB > TEAM || N >= 7);
  // ---- a1: load the point
  for (int i = lane; i < NS * 4; i += TEAM) {
    const double v = __ldg(p.mom + ptc * (NS * 4) + i);
    s_mom[i] = v;
    if constexpr (INV) {
      const float hi = (float)v;
      s_momf[i] = hi;                          // v = hi + lo to about 2^-48
      s_momf[NS * 4 + i] = (float)(v - (double)hi);
    }
  }
  team_sync<TEAM>();

  if constexpr (!INV) {
    // ---- a3: propagator entries of every photon subset, one subset per
    // thread (momenta and denominators in FP64)
    for (int mask = lane; mask < NSUB; mask += TEAM) {
      Real* d = s_q + mask * 5;
      Real P[5];
      if (mask == 0 || mask == (int)ALL) {
#pragma unroll
        for (int c = 0; c < 5; ++c) P[c] = (Real)0;
      } else {
        make_prop<Real>(s_mom, N, (unsigned)mask, p.mass, P);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) d[c] = P[c];
    }
  } else {
    // ---- a3, mixed: the invariants and their signed combinations c, then
    // the subsets of this lane, a fixed number per lane (two at a time, so
    // that their FP64 chains interleave) and the same instructions on every lane:
    // the U photons summed (at most N / 2) read the zero slot where U has
    // fewer, and D_T is summed in four interleaved partial sums (depth 3 for
    // three photons rather than a chain of six additions)
    setup_invariants<N, TEAM>(lane, p.mass, s_mom, s_w);
    const double* cmb = s_w + (2 + 3 * N + N * (N - 1) / 2);
    constexpr int UMAX = N / 2;
    constexpr int NT = 1 + UMAX + UMAX * (UMAX - 1) / 2;   // terms of a denominator
    static_assert(NT >= 1, "at least the electron's own term");
    constexpr int ZERO = 2 + 2 * N + N * N;
    constexpr int ITER = (NSUB + TEAM - 1) / TEAM;
#pragma unroll (ITER < 2 ? ITER : 2)
    for (int t = 0; t < ITER; ++t) {
      const int mask = lane + t * TEAM;
      if (NSUB % TEAM != 0 && mask >= NSUB) break;
      float* d = reinterpret_cast<float*>(s_q) + mask * 5;
      const bool out = 2 * __popc(mask) > N;
      const unsigned U = out ? ALL & ~(unsigned)mask : (unsigned)mask;
      int js[UMAX];
      unsigned rest = U;
#pragma unroll
      for (int i = 0; i < UMAX; ++i) {
        js[i] = rest ? __ffs(rest) - 1 : -1;
        rest &= rest - 1;
      }
      const int so = out ? 2 + N : 2;
      // the NT terms in NA interleaved partial sums, then added as a tree
      constexpr int NA = NT < 4 ? NT : 4;
      double acc[NA];
      acc[0] = cmb[out ? 1 : 0];
      int q = 1;
      auto add = [&](double x) {
        if (q < NA) acc[q] = x; else acc[q % NA] += x;
        ++q;
      };
#pragma unroll
      for (int i = 0; i < UMAX; ++i) add(cmb[js[i] < 0 ? ZERO : so + js[i]]);
#pragma unroll
      for (int i = 0; i < UMAX; ++i)
#pragma unroll
        for (int l = i + 1; l < UMAX; ++l)   // js[l] >= 0 implies js[i] >= 0
          add(cmb[js[l] < 0 ? ZERO : 2 + 2 * N + js[i] * N + js[l]]);
#pragma unroll
      for (int w = 1; w < NA; w *= 2)
#pragma unroll
        for (int i = 0; i + w < NA; i += 2 * w) acc[i] += acc[i + w];
      const double D = acc[0];
      // the numerator in float-float: q + sum_{j in U} tau_j k_j (tau_j =
      // sigma_j on the incoming side, -sigma_j on the outgoing side)
      float qh[4], ql[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        qh[c] = s_momf[(out ? 8 : 0) + c];
        ql[c] = s_momf[NS * 4 + (out ? 8 : 0) + c];
      }
#pragma unroll 1
      for (int i = 0; i < UMAX; ++i) {
        const int j = js[i] < 0 ? 0 : js[i];
        const int o = 4 * (j == 0 ? 1 : j + 2);
        const float sg = js[i] < 0 ? 0.f : ((j == 0) != out ? 1.f : -1.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float sum, err;
          two_sum_f(qh[c], sg * s_momf[o + c], sum, err);
          qh[c] = sum;
          ql[c] = __fadd_rn(ql[c], __fadd_rn(err, sg * s_momf[NS * 4 + o + c]));
        }
      }
      const bool used = mask != 0 && mask != (int)ALL;
      const float inv = used ? 1.0f / (float)D : 0.0f;
      const float m = (float)p.mass;
      // Q0 -+ m: the high part first (exact where Q0 is close to m)
      d[0] = __fadd_rn(__fadd_rn(qh[0], m), ql[0]) * inv;
      d[1] = __fadd_rn(__fsub_rn(qh[0], m), ql[0]) * inv;
      d[2] = __fadd_rn(qh[1], ql[1]) * inv;
      d[3] = __fadd_rn(qh[2], ql[2]) * inv;
      d[4] = __fadd_rn(qh[3], ql[3]) * inv;
    }
  }
  // ---- a2: external states u(p, +-), ubar(p', +-), eps_j(pol 1, 2) in
  // the working precision; the mixed form's from the float-float momenta
  // (E +- m as float-float sums rounded once), with no FP64 instruction
  for (int it = lane; it < 4 + 2 * N; it += TEAM) {
    if constexpr (INV) {
      if (it < 4) {
        const int side = it >> 1, e = it & 1;
        const float* h = s_momf + (side ? 8 : 0);
        const float* l = s_momf + NS * 4 + (side ? 8 : 0);
        const float mf = (float)p.mass;
        float sp[8];
        float epm, emm;
        e_pm_m_ff(h[0], l[0], mf, epm, emm);
        make_spinor_core<float>(h[1], h[2], h[3], epm, emm, e, side == 1, sp);
        store8(reinterpret_cast<float*>(s_spin) + (side * 2 + e) * 8, sp);
      } else {
        const int j = (it - 4) >> 1, pb = (it - 4) & 1;
        const float* h = s_momf + 4 * photon_slot_of(j);
        float ev[3];
        make_pol_core<float>(h[1], h[2], h[3], pb, ev);
        float* d = reinterpret_cast<float*>(s_eps) + (j * 2 + pb) * 4;
        d[0] = ev[0]; d[1] = ev[1]; d[2] = ev[2]; d[3] = 0.f;
      }
      continue;
    }
    if (it < 4) {
      const int side = it >> 1, e = it & 1;
      Real s[8];
      make_spinor<Real>(s_mom + (side ? 8 : 0), e, p.mass, side == 1, s);
      store8(s_spin + (side * 2 + e) * 8, s);
    } else {
      const int j = (it - 4) >> 1, pb = (it - 4) & 1;
      Real e[3];
      make_pol<Real>(s_mom + 4 * (j == 0 ? 1 : j + 2), pb, e);
      Real* d = s_eps + (j * 2 + pb) * 4;
      d[0] = e[0]; d[1] = e[1]; d[2] = e[2]; d[3] = (Real)0;
    }
  }
  team_sync<TEAM>();
}

// The S2 joins of every diagram whose left photon set is se.mask (a6), summed
// per spin state into acc (a7).
// tab: the set's row of the plan's lane table (spin-summed: entry c holds
// pext(c, S) | pext(c, not S) << 8).
template <int K, bool SUMMED, typename Real, int TEAM, int ES>
__device__ __forceinline__ void join_set(const SetEntry& se, const uint16_t* tab, int lane, const Real* s_cur,
                                       Acc<Real>* acc) {
  constexpr int N = K + 1;
  constexpr int H = (N + 1) / 2;
  constexpr int R = N - H;
  constexpr unsigned ALL = (1u << N) - 1;
  constexpr int NVL = SUMMED ? (1 << (H + 1)) : 1;
  constexpr int NVR = SUMMED ? (1 << (R + 1)) : 1;
  constexpr int NL = [] { int f = 1; for (int i = 2; i <= H; ++i) f *= i; return f; }();
  constexpr int NR = [] { int f = 1; for (int i = 2; i <= R; ++i) f *= i; return f; }();
  constexpr int BC = NR >= 2 ? 2 : 1;   // right leaves held in registers
  constexpr int GA = NL % 3 == 0 ? 3 : (NL % 2 == 0 ? 2 : 1); // left leaves per compensated step
  constexpr int NSI = ES >= 2 ? 1 : 2;
  constexpr int NSO = ES >= 4 ? 1 : 2;
  // mixed form: one compensated step for the whole set where it has at most
  // 12 diagrams, else one per GA x BC block
  constexpr bool ONE_STEP = NL * NR <= 12;
    if constexpr (SUMMED && sizeof(Real) == 4 && !ONE_STEP) {
      // mixed, more than 12 diagrams per set: packed FP32 FMAs (two per
      // instruction).  The BC right leaves of a block stay in registers,
      // broadcast once per block to (re, re) and (im, im) pairs; each left
      // leaf variant is loaded once per block as its natural (re, im) pairs:
      //   A += (rr, rr) * (lr, li),  B += (ri, ri) * (lr, li),
      //   Re M = A.x - B.y,  Im M = A.y + B.x,
      // with A starting from minus the state's compensation; the GA x BC
      // diagrams of a block are one compensated step per state, as in the
      // scalar form below.
      const unsigned c = (unsigned)lane & ALL;
      const int ep = lane >> N;
      const unsigned tv = __ldg(tab + c);
      const int vl = ((int)(tv & 0xffu) << 1) + (ES >= 2 ? (ep & 1) : 0);
      const int vr = ((int)(tv >> 8) << 1) + (ES >= 4 ? (ep >> 1) : 0);
      for (int b0 = 0; b0 < NR; b0 += BC) {
        float2 rr[BC][NSO][4], ri[BC][NSO][4];
#pragma unroll
        for (int bb = 0; bb < BC; ++bb)
#pragma unroll
          for (int so = 0; so < NSO; ++so) {
            float x[8];
            load_cur(s_cur, se.leaf_r + (b0 + bb) * NVR, NVR, vr + so, x);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              rr[bb][so][q] = make_float2(x[2 * q], x[2 * q]);
              ri[bb][so][q] = make_float2(x[2 * q + 1], x[2 * q + 1]);
            }
          }
        for (int a0 = 0; a0 < NL; a0 += GA) {
          float2 A[NSI][NSO], B[NSI][NSO];
#pragma unroll
          for (int si = 0; si < NSI; ++si)
#pragma unroll
            for (int so = 0; so < NSO; ++so) {
              A[si][so] = make_float2(-acc[si * NSO + so].cre, -acc[si * NSO + so].cim);
              B[si][so] = make_float2(0.f, 0.f);
            }
#pragma unroll
          for (int ga = 0; ga < GA; ++ga)
#pragma unroll
            for (int si = 0; si < NSI; ++si) {
              float x[8];
              load_cur(s_cur, se.leaf_l + (a0 + ga) * NVL, NVL, vl + si, x);
              float2 l[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) l[q] = make_float2(x[2 * q], x[2 * q + 1]);
#pragma unroll
              for (int so = 0; so < NSO; ++so)
#pragma unroll
                for (int bb = 0; bb < BC; ++bb)
#pragma unroll
                  for (int q = 0; q < 4; ++q) {
                    A[si][so] = __ffma2_rn(rr[bb][so][q], l[q], A[si][so]);
                    B[si][so] = __ffma2_rn(ri[bb][so][q], l[q], B[si][so]);
                  }
            }
#pragma unroll
          for (int si = 0; si < NSI; ++si)
#pragma unroll
            for (int so = 0; so < NSO; ++so)
              acc[si * NSO + so].commit(__fsub_rn(A[si][so].x, B[si][so].y), __fadd_rn(A[si][so].y, B[si][so].x));
        }
      }
    } else if constexpr (SUMMED) {
      const unsigned c = (unsigned)lane & ALL;
      const int ep = lane >> N;
      const unsigned tv = __ldg(tab + c);
      const int vl = ((int)(tv & 0xffu) << 1) + (ES >= 2 ? (ep & 1) : 0);
      const int vr = ((int)(tv >> 8) << 1) + (ES >= 4 ? (ep >> 1) : 0);
      float ys[NSI * NSO][2];
      if constexpr (sizeof(Real) == 4 && ONE_STEP) {
#pragma unroll
        for (int i = 0; i < NSI * NSO; ++i) acc[i].start(ys[i][0], ys[i][1]);
      }

      for (int b0 = 0; b0 < NR; b0 += BC) {
        Real rw[BC][NSO][8];
#pragma unroll
        for (int bb = 0; bb < BC; ++bb)
#pragma unroll
          for (int so = 0; so < NSO; ++so)
            load_cur(s_cur, se.leaf_r + (b0 + bb) * NVR, NVR, vr + so, rw[bb][so]);
        for (int a0 = 0; a0 < NL; a0 += GA) {
          Real lc[GA][NSI][8];
#pragma unroll
          for (int ga = 0; ga < GA; ++ga)
#pragma unroll
            for (int si = 0; si < NSI; ++si)
              load_cur(s_cur, se.leaf_l + (a0 + ga) * NVL, NVL, vl + si, lc[ga][si]);
#pragma unroll
          for (int si = 0; si < NSI; ++si)
#pragma unroll
            for (int so = 0; so < NSO; ++so) {
              if constexpr (sizeof(Real) == 8) {
#pragma unroll
                for (int ga = 0; ga < GA; ++ga)
#pragma unroll
                  for (int bb = 0; bb < BC; ++bb)
                    dot_acc(rw[bb][so], lc[ga][si], acc[si * NSO + so].re, acc[si * NSO + so].im);
              } else if constexpr (ONE_STEP) {
#pragma unroll
                for (int ga = 0; ga < GA; ++ga)
#pragma unroll
                  for (int bb = 0; bb < BC; ++bb)
                    dot_acc(rw[bb][so], lc[ga][si], ys[si * NSO + so][0], ys[si * NSO + so][1]);
              } else {
                // the GA x BC diagrams of this state in one compensated step
                float yr, yi;
                acc[si * NSO + so].start(yr, yi);
#pragma unroll
                for (int ga = 0; ga < GA; ++ga)
#pragma unroll
                  for (int bb = 0; bb < BC; ++bb) dot_acc(rw[bb][so], lc[ga][si], yr, yi);
                acc[si * NSO + so].commit(yr, yi);
              }
            }
        }
      }
      if constexpr (sizeof(Real) == 4 && ONE_STEP) {
#pragma unroll
        for (int i = 0; i < NSI * NSO; ++i) acc[i].commit(ys[i][0], ys[i][1]);
      }
    } else if constexpr (sizeof(Real) == 8) {
      // one fixed state, FP64: the lanes split the NL x NR diagrams
      for (int q = lane; q < NL * NR; q += TEAM) {
        const int a = q / NR, b = q - a * NR;
        Real lc[8], rw[8];
        load_cur(s_cur, se.leaf_l + a, 1, 0, lc);
        load_cur(s_cur, se.leaf_r + b, 1, 0, rw);
        dot_acc(rw, lc, acc[0].re, acc[0].im);
      }
    } else {
      // one fixed state, mixed: every round of the lanes' split has its own
      // partial sums (independent FMA chains), added at the end and
      // committed as one compensated step per set
      constexpr int ROUNDS = (NL * NR + TEAM - 1) / TEAM;
      float pr[ROUNDS], pi[ROUNDS];
#pragma unroll
      for (int t = 0; t < ROUNDS; ++t) {
        pr[t] = pi[t] = 0.f;
        const int q = lane + t * TEAM;
        if (q < NL * NR) {
          const int a = q / NR, b = q - a * NR;
          float lc[8], rw[8];
          load_cur(s_cur, se.leaf_l + a, 1, 0, lc);
          load_cur(s_cur, se.leaf_r + b, 1, 0, rw);
          dot_acc(rw, lc, pr[t], pi[t]);
        }
      }
#pragma unroll
      for (int t = 1; t < ROUNDS; ++t) { pr[0] += pr[t]; pi[0] += pi[t]; }
      float yr, yi;
      acc[0].start(yr, yi);
      acc[0].commit(yr + pr[0], yi + pi[0]);
    }
}

}  // namespace qed
