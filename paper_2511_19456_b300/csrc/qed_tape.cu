// Node-by-node execution of a CDAG in any node-reduction state (the
// node-reduction sweep of Sec. III-D, Fig. f_optimization).
//
// The tape holds every compute node of the DAG, grouped by level (longest
// path from the external states).  A team of 32 threads evaluates one point:
// it runs the levels in order, its lanes taking the nodes of a level, with a
// warp barrier between levels.  Each node does its own work as a task of the
// paper's CDAG would:
//   T_SPINOR / T_POL  the external states of one fixed spin state;
//   T_V               the vertex eps/ times a current;
//   T_S1              the propagator of its own momentum (FP64 Q and D),
//                     applied to a current;
//   T_S2              the propagator of the left photon set applied to the
//                     left current, then contracted with the right current:
//                     one diagram's amplitude.
// The Sum adds the diagrams in the order of the Sum node's parents, which no
// reduction changes, so every reduction state gives bit-identical results.
// FP64 throughout; values live in shared memory slots allocated by liveness.
#include <cuda_runtime.h>

#include "qed_plan.hpp"
#include "qed_team.cuh"

namespace qed {

namespace {

constexpr int kTapeTeam = 32;

__global__ void __launch_bounds__(kTapeTeam) qed_tape_kernel(const KParams p) {
  constexpr int TEAM = kTapeTeam;
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = p.k, n = k + 1, ns = k + 3;
  const TapeLayout L = tape_layout(k, p.n_slots, p.n_diag);
  const int lane = threadIdx.x & (TEAM - 1);
  const int team = threadIdx.x / TEAM;
  const int tpc = blockDim.x / TEAM;
  unsigned char* base = smem + (size_t)team * L.bytes;
  double* s_mom = reinterpret_cast<double*>(base + L.mom);
  double* s_val = reinterpret_cast<double*>(base + L.val);
  double* s_diag = reinterpret_cast<double*>(base + L.diag);

  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {
    const long long pt = pt0 + team;
    const bool valid = pt < p.n;
    const long long ptc = valid ? pt : p.n - 1;
    for (int i = lane; i < ns * 4; i += TEAM) s_mom[i] = __ldg(p.mom + ptc * (ns * 4) + i);
    team_sync<TEAM>();
    for (int lv = 0; lv < p.n_levels; ++lv) {
      const int beg = __ldg(p.tape_levels + lv), end = __ldg(p.tape_levels + lv + 1);
      for (int it = beg + lane; it < end; it += TEAM) {
        int4 raw = __ldg(reinterpret_cast<const int4*>(p.tape + it));
        TapeInstr in;
        memcpy(&in, &raw, sizeof(in));
        double* dst = s_val + 8 * in.dst;
        switch (in.op) {
          case T_SPINOR: {
            double s[8];
            const int e = in.side == 0 ? p.fixed_sin : p.fixed_sout;
            make_spinor<double>(s_mom + (in.side ? 8 : 0), e, p.mass, in.side == 1, s);
            store8(dst, s);
            break;
          }
          case T_POL: {
            const int j = in.arg;
            double e[3];
            make_pol<double>(s_mom + 4 * (j == 0 ? 1 : j + 2), (int)((p.fixed_pol_bits >> j) & 1u), e);
            dst[0] = e[0]; dst[1] = e[1]; dst[2] = e[2]; dst[3] = 0.0;
            break;
          }
          case T_V: {
            double x[8], y[8];
            load8(s_val + 8 * in.src0, x);
            const double* e = s_val + 8 * in.src1;
            const double ev[3] = {e[0], e[1], e[2]};
            if (in.side == 0) vertex_col(ev, x, y); else vertex_row(ev, x, y);
            store8(dst, y);
            break;
          }
          case T_S1: {
            double x[8], y[8], P[5];
            load8(s_val + 8 * in.src0, x);
            make_prop<double>(s_mom, n, in.mask, p.mass, P);
            if (in.side == 0) prop_col(P, x, y); else prop_row(P, x, y);
            store8(dst, y);
            break;
          }
          case T_S2: {
            double l[8], r[8], z[8], P[5];
            load8(s_val + 8 * in.src0, l);
            load8(s_val + 8 * in.src1, r);
            make_prop<double>(s_mom, n, in.mask, p.mass, P);
            prop_col(P, l, z);
            double re = 0.0, im = 0.0;
            dot_acc(r, z, re, im);
            s_diag[2 * in.dst] = re;
            s_diag[2 * in.dst + 1] = im;
            break;
          }
          default:
            break;
        }
      }
      team_sync<TEAM>();
    }
    if (lane == 0 && valid) {
      double re = 0.0, im = 0.0;
      for (int d = 0; d < p.n_diag; ++d) { re += s_diag[2 * d]; im += s_diag[2 * d + 1]; }
      p.out[pt] = (re * re + im * im) * p.coupling;
    }
    team_sync<TEAM>();
  }
}

}  // namespace

KernelChoice tape_kernel() { return KernelChoice{qed_tape_kernel, kTapeTeam}; }

}  // namespace qed
