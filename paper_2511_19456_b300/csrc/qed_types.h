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
  int mom, q, eps, spin, red, w, momf, cur, bytes;
};

// Mixed form's set-up scratch (see setup_invariants): the FP64 Minkowski
// products of the point's momenta, the signed combinations from which every
// denominator is summed (pairs at a square index) and a zero slot; then the
// momenta as float-float pairs.
QED_HD int n_products(int n) { return 2 + 3 * n + n * (n - 1) / 2; }
QED_HD int n_invariants(int n) { return n_products(n) + 2 + 2 * n + n * n + 1; }

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
  // the currents; the mixed form's set-up scratch (invariants, float-float
  // momenta) shares their space, as it is dead before the first current
  L.cur = off;
  const int cur_bytes = ncur * 8 * real_size;
  const int scratch = real_size == 4 ? align16(n_invariants(n) * 8) + (k + 3) * 4 * 4 * 2 : 0;
  L.w = off;
  L.momf = off + align16(n_invariants(n) * 8);
  off = align16(off + (cur_bytes > scratch ? cur_bytes : scratch));
  L.bytes = off;
  return L;
}

// Shared memory of one team of the ABC-model kernels: momenta (FP64), 1/D of
// every subset, a reduction scratch and the (scalar) currents.
struct AbcLayout {
  int mom, inv, red, cur, bytes;
};

QED_HD AbcLayout abc_layout(int k, int real_size, int ncur) {
  const int n = k + 1;
  AbcLayout L;
  int off = 0;
  L.mom = off; off = align16(off + (k + 3) * 4 * 8);
  L.inv = off; off = align16(off + (1 << n) * real_size);
  L.red = off; off = align16(off + 16 * 8);
  L.cur = off; off = align16(off + ncur * real_size);
  L.bytes = off;
  return L;
}

// Shared memory of one team of the tape kernel: momenta, the value slots
// (8 FP64 reals each) and the diagram amplitudes (complex FP64).
struct TapeLayout {
  int mom, val, diag, bytes;
};

QED_HD TapeLayout tape_layout(int k, int n_slots, int n_diag) {
  TapeLayout L;
  int off = 0;
  L.mom = off;  off = align16(off + (k + 3) * 4 * 8);
  L.val = off;  off = align16(off + n_slots * 8 * 8);
  L.diag = off; off = align16(off + n_diag * 2 * 8);
  L.bytes = off;
  return L;
}

// Extra shared memory of the adjoint kernel after the forward team layout:
// adjoints of every current, the amplitude seeds conj(M), and FP64
// accumulators of the propagator (4 Dirac components + 1, complex) and
// polarisation (3 components, complex) parameters and of the photon momenta.
struct AdjLayout {
  TeamLayout fwd;
  int adj, mbar, acc_s, acc_e, kbar, part, bytes;
};

// Parameter accumulators: the real parts of 5 propagator terms per photon
// subset and of 3 polarisation terms per photon and polarisation.
// n_part > 0 (mixed precision): FP32 partial sums of one photon set's
// parameter terms, n_part propagator slots of 5 reals and 3 reals per
// photon (6 when the spin is summed: both polarisations), added to the FP64
// accumulators once per set.
QED_HD AdjLayout adj_layout(int k, int real_size, int ncur, bool summed, int n_part = 0) {
  const int n = k + 1;
  AdjLayout A;
  A.fwd = team_layout(k, real_size, ncur);
  int off = A.fwd.bytes;
  A.adj = off;   off = align16(off + ncur * 8 * real_size);
  A.mbar = off;  off = align16(off + (summed ? (1 << (n + 2)) : 1) * 2 * real_size);
  A.acc_s = off; off = align16(off + (1 << n) * 5 * 8);
  A.acc_e = off; off = align16(off + n * 2 * 3 * 8);
  A.kbar = off;  off = align16(off + n * 4 * 8);
  A.part = off;  off = align16(off + (n_part > 0 ? (n_part * 5 + n * (summed ? 6 : 3)) * 4 : 0));
  A.bytes = off;
  return A;
}

// Shared memory of one team of the rewritten-DAG adjoint (qed_radj.cu): the
// forward team layout with ncur currents, then nadj current adjoints, the
// amplitude seeds conj(M) or (later) per-lane accumulators of the
// polarisation parameters in the working precision, the propagator
// parameters of every photon subset (5, working precision), and FP64
// accumulators of the polarisation parameters (3 per photon and
// polarisation) and of the photon momenta.
struct RadjLayout {
  TeamLayout fwd;
  int adj, mbar, acc_s, acc_e, kbar, elane, bytes;
};

QED_HD RadjLayout radj_layout(int k, int real_size, int ncur, int nadj, bool summed, int team) {
  const int n = k + 1;
  RadjLayout A;
  A.fwd = team_layout(k, real_size, ncur);
  int off = A.fwd.bytes;
  A.adj = off;   off = align16(off + nadj * 8 * real_size);
  // the seeds (needed until the joins are transposed) and the per-lane
  // polarisation terms (needed after) share their space
  const int mbar_bytes = (summed ? (1 << (n + 2)) : 1) * 2 * real_size;
  const int elane_bytes = team * n * 2 * 3 * real_size;
  A.mbar = A.elane = off;
  off = align16(off + (mbar_bytes > elane_bytes ? mbar_bytes : elane_bytes));
  A.acc_s = off; off = align16(off + (1 << n) * 5 * real_size);
  A.acc_e = off; off = align16(off + n * 2 * 3 * 8);
  A.kbar = off;  off = align16(off + n * 4 * 8);
  A.bytes = off;
  return A;
}

struct KParams {
  const double* mom;
  double* out;
  double* grad;      // adjoint kernel: d|M|^2/dk_j [N][k][3] (may be null otherwise)
  long long n;
  int k;             // photons out
  const Instr* instr;
  const SumInstr* sinstr;   // rewritten-DAG instructions (rewrite plans)
  const Phase* phases;
  const SetEntry* sets;
  int n_stored_phases, n_set_phases, n_sets;
  int set_group;     // rewrite plans: photon sets per set phase
  // rewrite plans, spin-summed: for set s and photon-polarisation pattern c,
  // entry [s][c] = pext(c, S) | pext(c, not S) << 8 (left and right leaf
  // variant without the helicity bit)
  const uint16_t* lane_tab;
  // spin-summed plans: for set s, entries [s][0 .. 2^h) = pdep(v, S) and
  // [s][2^h .. 2^h + 2^r) = pdep(v, not S) (the adjoint's state index)
  const uint16_t* dep_tab;
  int ncur;          // stored + local currents
  int ncur_stored;   // currents kept for the whole point
  int team_bytes;
  double mass;       // electron mass; the A mass in the ABC model
  double mass_c;     // ABC model: the C mass
  double coupling;   // e^(2n); g^(2n) in the ABC model
  int fixed_sin, fixed_sout;       // helicity bit (0: +1, 1: -1)
  unsigned fixed_pol_bits;         // bit j: polarisation of photon j (0: pol 1, 1: pol 2)
  // adjoint plans whose currents do not fit in shared memory: a global
  // scratch of adj_scratch_team bytes per team (currents, then adjoints)
  void* adj_scratch;
  long long adj_scratch_team;
  // mixed adjoint: for set s, entry [s][i] is the propagator
  // photon set of partial-sum slot i (0: unused); an instruction of the set
  // names its slot as pad - 1 (pad = 0: no slot, direct FP64 accumulation)
  const uint16_t* part_tab;
  int n_part;
  // one fixed state, register-join form (qed_fix.cu): fix_items holds the
  // items (two ints each, 8-byte aligned) of the kept levels, in groups of
  // independent items
  // [fix_group[g], fix_group[g+1]), then one item per lane of a warp (part)
  // per photon set from fix_set_off; the right leaves of a set go to one of
  // its warp's two alternating buffers of NR currents (the warps' buffers
  // follow each other from current fix_rbase); fix_ncur currents per team
  const int* fix_items;
  int fix_ngroups;
  int fix_group[9];
  int fix_set_off;
  int fix_rbase;
  int fix_ncur;
  // adjoint on the rewritten DAG (qed_radj.cu): the photon subsets of every
  // node, side 0 (column currents) then side 1 (row currents), level by
  // level (side s, level l: entries radj_lev[s][l] .. radj_lev[s][l + 1] of
  // radj_masks, l = 1..8), and radj_slot[(s << n) | mask], the node's first
  // current (spin variant 0) or -1
  const int* radj_masks;
  int radj_lev[2][10];
  const int* radj_slot;
  // ... radj_aslot: the node's first adjoint of radj_nadj (-1 for the
  // column leaves, whose adjoints take their currents' place)
  const int* radj_aslot;
  int radj_nadj;
  // tape plans (node-reduction sweep)
  const TapeInstr* tape;
  const int* tape_levels;          // instruction range of each level
  int n_levels, n_slots, n_diag;
};

}  // namespace qed
