// Types shared by the host launcher and the CUDA kernels: the shared-memory
// layout of one team and the kernel parameter block.
#pragma once

#include "dag.hpp"

#if defined(__CUDACC__)
#define QED_HD __host__ __device__ __forceinline__
#else
#define QED_HD inline
#endif

namespace qed {


// Shared-memory layout of one team (the threads that evaluate one point).
struct TeamLayout {
  int mom, q, eps, spin, red, cur, bytes;
};

QED_HD int align16(int x) { return (x + 15) & ~15; }

// real_size: 4 (mixed) or 8 (FP64).  ncur: currents kept per team.
QED_HD TeamLayout team_layout(int k, int real_size, int ncur) {
  const int n = k + 1;
  TeamLayout L;
  int off = 0;
  L.mom = off;  off = align16(off + (k + 3) * 4 * 8);
  L.q = off;    off = align16(off + (1 << n) * 5 * real_size);
  L.eps = off;  off = align16(off + n * 2 * 4 * real_size);
  L.spin = off; off = align16(off + 2 * 2 * 8 * real_size);
  L.red = off;  off = align16(off + 16 * 8);
  L.cur = off;  off = align16(off + ncur * 8 * real_size);
  L.bytes = off;
  return L;
}

struct KParams {
  const double* mom;
  double* out;
  long long n;
  const Instr* instr;
  const Phase* phases;
  const SetEntry* sets;
  int n_stored_phases, n_set_phases, n_sets;
  int ncur;          // stored + local currents
  int team_bytes;
  double mass;
  double coupling;   // e^(2n)
  int fixed_sin, fixed_sout;       // helicity bit (0: +1, 1: -1)
  unsigned fixed_pol_bits;         // bit j: polarisation of photon j (0: pol 1, 1: pol 2)
};

}  // namespace qed
