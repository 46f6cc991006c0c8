// C-ABI of the |M|^2 engine (declared in include/qed.h): plan creation (DAG
// generation, node reduction, linear schedule, upload), evaluation entry
// points and argument validation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <stdexcept>

#include "../../include/qed.h"
#include "dag.hpp"
#include "qed_types.h"

#include "qed_plan.hpp"

namespace {

// Levels kept for the whole point; deeper levels are rebuilt per photon set.
// All levels below the leaves fit in shared memory except for spin-summed
// k = 6, 7, where only the first levels are kept.  One fixed state in the
// mixed form, k >= 6: one left level fewer.  Its nodes are rebuilt per
// photon set (+24 % FLOPs at k = 6), but a team's shared memory halves and
// more teams are resident, which the latency-bound FP32 kernel turns into
// +12 %; the FP64 kernel, bound by its pipe, keeps all levels.
void default_levels(int k, bool summed, bool mixed, int* ls, int* rs) {
  const int n = k + 1, h = (n + 1) / 2, r = n - h;
  *ls = h - 1;
  *rs = r - 1;
  if (summed && k == 6) { *ls = 2; *rs = 2; }
  if (summed && k == 7) { *ls = 1; *rs = 1; }
  if (!summed && mixed && k >= 6) *ls = h - 2;
}


bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

void free_plan(qed_plan_s* p) {
  if (!p) return;
  cudaFree(p->d_instr);
  cudaFree(p->d_phases);
  cudaFree(p->d_sets);
  cudaFree(p->d_instr_adj);
  cudaFree(p->d_phases_adj);
  cudaFree(p->d_sets_adj);
  cudaFree(p->d_sinstr);
  cudaFree(p->d_tape);
  cudaFree(p->d_adj_scratch);
  cudaFree(p->d_levels);
  cudaFree(p->d_lane_tab);
  cudaFree(p->d_dep_tab);
  cudaFree(p->d_part_tab);
  cudaFree(p->d_fix_items);
  cudaFree(p->d_radj_masks);
  cudaFree(p->d_radj_slot);
  cudaFree(p->d_radj_aslot);
  cudaFree(p->d_stage);
  if (p->ev_scratch) cudaEventDestroy(p->ev_scratch);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_h2d[i]) cudaEventDestroy(p->ev_h2d[i]);
    if (p->ev_k[i]) cudaEventDestroy(p->ev_k[i]);
    if (p->ev_d2h[i]) cudaEventDestroy(p->ev_d2h[i]);
  }
  if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
  if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
  delete p;
}

}  // namespace

namespace {
std::atomic<int> g_alloc_fail_after{-1};   // -1: no injected failure
}  // namespace

cudaError_t qed::device_alloc(void** p, size_t bytes) {
  int left = g_alloc_fail_after.load();
  while (left >= 0) {
    if (g_alloc_fail_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

qed_status qed::cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QED_OK;
  // a failed call that leaves the context usable also leaves its error as
  // the runtime's last error; clear it, so that the caller's next CUDA call
  // does not report it (a sticky error stays in the context regardless)
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return QED_ENOMEM;
  return QED_ECUDA;
}

KParams qed::make_params(const qed_plan_s* P, const double* mom, long long n, double* out) {
  KParams kp{};
  kp.mom = mom;
  kp.out = out;
  kp.n = n;
  kp.k = P->k;
  kp.instr = P->d_instr;
  kp.sinstr = P->d_sinstr;
  kp.lane_tab = P->d_lane_tab;
  kp.dep_tab = P->d_dep_tab;
  kp.phases = P->d_phases;
  kp.sets = P->d_sets;
  if (P->rewrite) {
    kp.n_stored_phases = P->rsc.n_stored_phases;
    kp.n_set_phases = P->rsc.n_set_phases;
    kp.n_sets = (int)P->rsc.sets.size();
    kp.ncur = P->rsc.stored_currents + P->rsc.local_currents;
    kp.ncur_stored = P->rsc.stored_currents;
    kp.set_group = P->rsc.group;
  } else {
    kp.set_group = 1;
    kp.n_stored_phases = P->sc.n_stored_phases;
    kp.n_set_phases = P->sc.n_set_phases;
    kp.n_sets = (int)P->sc.sets.size();
    kp.ncur = P->sc.stored_currents + P->sc.local_currents;
    kp.ncur_stored = P->sc.stored_currents;
  }
  kp.team_bytes = P->team_bytes;
  kp.mass = P->mass;
  kp.mass_c = P->mass_c;
  kp.coupling = std::pow(P->charge, 2.0 * (P->k + 1));
  kp.fixed_sin = P->fixed_sin;
  kp.fixed_sout = P->fixed_sout;
  kp.fixed_pol_bits = 0;
  for (int j = 0; j < 8; ++j) kp.fixed_pol_bits |= (unsigned)(P->fixed_pol[j] & 1) << j;
  kp.fix_items = P->d_fix_items;
  kp.fix_ngroups = P->fix_ngroups;
  for (int g = 0; g < 9; ++g) kp.fix_group[g] = P->fix_group[g];
  kp.fix_set_off = P->fix_set_off;
  kp.fix_rbase = P->fix_rbase;
  kp.fix_ncur = P->fix_ncur;
  if (P->is_tape) {
    kp.tape = P->d_tape;
    kp.tape_levels = P->d_levels;
    kp.n_levels = (int)P->tp.level_beg.size() - 1;
    kp.n_slots = P->tp.n_slots;
    kp.n_diag = P->tp.n_diag;
  }
  return kp;
}

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  cudaError_t e = device_alloc((void**)dst, bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// The adjoint keeps the forward currents and their adjoints in shared
// memory: take the deepest kept levels (ls, rs) whose team fits; if none
// fits, qed_eval_grad reports QED_EUNSUPPORTED for this plan.
// Mixed adjoint: every photon set gets one FP32 partial-sum slot
// per distinct propagator of its instructions.  Sets the slot (plus one) into
// the instructions' pad field, fills tab[set][slot] with the propagator's
// photon set and returns the slots per set.  The kept levels' instructions
// keep pad = 0 (FP64 accumulation).
int assign_partial_slots(Schedule& sc, std::vector<uint16_t>* tab) {
  for (Instr& in : sc.instr) in.pad = 0;
  std::vector<std::vector<uint16_t>> posts(sc.sets.size());
  size_t n_part = 1;
  for (size_t s = 0; s < sc.sets.size(); ++s) {
    for (int t = 0; t < sc.n_set_phases; ++t) {
      const Phase& ph = sc.phases[sc.sets[s].phase0 + t];
      for (int slot = 0; slot < 2; ++slot)
        for (int i = 0; i < ph.cnt[slot]; ++i) {
          Instr& in = sc.instr[ph.beg[slot] + i];
          if (!in.post) continue;
          auto& v = posts[s];
          size_t j = std::find(v.begin(), v.end(), in.post) - v.begin();
          if (j == v.size()) v.push_back(in.post);
          in.pad = (uint16_t)(j + 1);
        }
    }
    n_part = std::max(n_part, posts[s].size());
  }
  tab->assign(sc.sets.size() * n_part, 0);
  for (size_t s = 0; s < sc.sets.size(); ++s)
    std::copy(posts[s].begin(), posts[s].end(), tab->begin() + s * n_part);
  return (int)n_part;
}

// The adjoint on the rewritten DAG (qed_radj.cu): one current per photon
// subset and side, kept for the whole point with its adjoint.  Tables: the
// subsets of every node, column side then row side, level by level in
// increasing mask order, and the first current of each (side, subset).
// Sets *done when the plan takes it; leaves the plan alone where the kernel
// does not exist or a team does not fit in shared memory.
qed_status setup_radj(qed_plan_s* P, bool mixed, int dev_smem, int sms, bool* done) {
  *done = false;
  const KernelChoice kc = radj_kernel(P->k, P->summed, mixed);
  if (!kc.fn) return QED_OK;
  const int k = P->k, n = k + 1, h = (n + 1) / 2, r = n - h;
  std::vector<int> masks, slot(2u << n, -1), aslot(2u << n, -1);
  int lev[2][10] = {{0}};
  int next = 0, anext = 0;
  for (int side = 0; side < 2; ++side) {
    const int top = side == 0 ? h : r;
    for (int l = 1; l <= 9; ++l) {
      lev[side][l] = (int)masks.size();
      if (l > top) continue;
      for (int T = 1; T < (1 << n); ++T) {
        if (__builtin_popcount(T) != l) continue;
        masks.push_back(T);
        const int nv = P->summed ? (2 << l) : 1;
        slot[(side << n) | T] = next;
        next += nv;
        if (side == 1 || l < h) {   // a column leaf's adjoint takes its current's place
          aslot[(side << n) | T] = anext;
          anext += nv;
        }
      }
    }
  }
  const int team = kc.team, block = std::max(team, 32);
  const size_t smem =
      (size_t)(block / team) * radj_layout(k, mixed ? 4 : 8, next, anext, P->summed, team).bytes;
  if (smem > (size_t)dev_smem) return QED_OK;
  cudaError_t e = upload(&P->d_radj_masks, masks);
  if (e == cudaSuccess) e = upload(&P->d_radj_slot, slot);
  if (e == cudaSuccess) e = upload(&P->d_radj_aslot, aslot);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)kc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kc.fn, block, smem);
  if (e != cudaSuccess) return cuda_status(e);
  if (per_sm < 1) return QED_OK;
  std::memcpy(P->radj_lev, lev, sizeof(lev));
  P->radj_ncur = next;
  P->radj_nadj = anext;
  P->radj = true;
  P->kc_adj = kc;
  P->block_adj = block;
  P->smem_adj = smem;
  P->grid_adj = per_sm * sms;
  P->has_adj = true;
  *done = true;
  return QED_OK;
}

qed_status setup_adjoint(qed_plan_s* P, bool mixed, int dev_smem, int sms) {
  {
    bool done = false;
    const qed_status rs = setup_radj(P, mixed, dev_smem, sms, &done);
    if (rs != QED_OK || done) return rs;
  }
  const int k = P->k, n = k + 1, h = (n + 1) / 2, r = n - h;
  P->kc_adj = adjoint_kernel(k, P->summed, mixed);
  if (!P->kc_adj.fn) return QED_OK;
  const int team = P->kc_adj.team;
  const int block = team > 32 ? team : 32;
  // one fixed state, k >= 6: one kept level fewer than fits.  The adjoint
  // holds currents, their adjoints and FP64 accumulators per team, so few
  // teams are resident; rebuilding one more level per set buys more of them
  // (k = 6: +6 % in FP64, +10 % in the mixed form with its per-set FP32
  // partial sums)
  int start = std::max(h - 1, r - 1);
  if (!P->summed && k >= 6) start -= 1;
  for (int lev = start; lev >= 0; --lev) {
    const int ls = std::min(lev, h - 1), rs = std::min(lev, r - 1);
    Schedule sc;
    try {
      sc = build_schedule(k, P->summed, ls, rs);
    } catch (const std::bad_alloc&) {
      return QED_ENOMEM;
    } catch (...) {
      return QED_EUNSUPPORTED;
    }
    const int ncur = sc.stored_currents + sc.local_currents;
    std::vector<uint16_t> part_tab;
    const int n_part = mixed ? assign_partial_slots(sc, &part_tab) : 0;
    AdjLayout A = adj_layout(k, mixed ? 4 : 8, ncur, P->summed, n_part);
    const size_t smem = (size_t)(block / team) * A.bytes;
    if (smem > (size_t)dev_smem) continue;
    cudaError_t e = upload(&P->d_instr_adj, sc.instr);
    if (e == cudaSuccess && n_part > 0) e = upload(&P->d_part_tab, part_tab);
    if (e == cudaSuccess) e = upload(&P->d_phases_adj, sc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets_adj, sc.sets);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)P->kc_adj.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)P->kc_adj.fn, block, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm < 1) return QED_OK;
    P->sc_adj = std::move(sc);
    P->n_part = n_part;
    P->block_adj = block;
    P->smem_adj = smem;
    P->grid_adj = per_sm * sms;
    P->has_adj = true;
    return QED_OK;
  }
  // nothing fits in shared memory (spin-summed k = 7 in FP64): currents and
  // adjoints in a global scratch slot per resident team, with the forward
  // plan's kept levels; the slots stay in the 126 MB L2
  {
    int ls, rs;
    default_levels(k, P->summed, mixed, &ls, &rs);
    Schedule sc;
    try {
      sc = build_schedule(k, P->summed, ls, rs);
    } catch (const std::bad_alloc&) {
      return QED_ENOMEM;
    } catch (...) {
      return QED_EUNSUPPORTED;
    }
    const int ncur = sc.stored_currents + sc.local_currents;
    const KernelChoice kg = adjoint_kernel_gmem(k, P->summed, mixed);
    if (!kg.fn || kg.team != team) return QED_OK;
    AdjLayout A = adj_layout(k, mixed ? 4 : 8, 0, P->summed);
    const size_t smem = (size_t)(block / team) * A.bytes;
    if (smem > (size_t)dev_smem) return QED_OK;
    cudaError_t e = cudaFuncSetAttribute((const void*)kg.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kg.fn, block, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm < 1) return QED_OK;
    const long long team_bytes = (long long)ncur * 8 * (mixed ? 4 : 8) * 2;
    const long long teams = (long long)per_sm * sms * (block / team);
    e = upload(&P->d_instr_adj, sc.instr);
    if (e == cudaSuccess) e = upload(&P->d_phases_adj, sc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets_adj, sc.sets);
    if (e == cudaSuccess) e = device_alloc(&P->d_adj_scratch, (size_t)(teams * team_bytes));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_scratch, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    P->adj_scratch_team = team_bytes;
    P->adj_scratch_bytes = teams * team_bytes;
    P->kc_adj = kg;
    P->sc_adj = std::move(sc);
    P->block_adj = block;
    P->smem_adj = smem;
    P->grid_adj = per_sm * sms;
    P->has_adj = true;
  }
  return QED_OK;
}

qed_status launch_eval(const qed_plan_s* P, const double* d_mom, long long n, double* d_out,
                       cudaStream_t st) {
  if (n == 0) return QED_OK;
  KParams kp = make_params(P, d_mom, n, d_out);
  const qed_plan_s::Form& f = P->forms[P->form.load(std::memory_order_relaxed)];
  const int tpc = f.block / f.kc.team;
  long long need = (n + tpc - 1) / tpc;
  int grid = (int)std::min<long long>(need, f.grid);
  return cuda_status(launch_forward(f.kc.fn, grid, f.block, f.smem, st, kp));
}

// Shared-memory attribute and resident blocks of one forward form.
cudaError_t configure_form(qed_plan_s::Form* f, int sms) {
  cudaError_t e = cudaFuncSetAttribute((const void*)f->kc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)f->kc.fn, f->block, f->smem);
  f->ok = e == cudaSuccess && per_sm >= 1;
  f->grid = per_sm * sms;
  return e;
}

// One fixed state: the register-join form (qed_fix.cu), on the schedule
// that keeps every level below the leaves.  Items are two ints:
//   source current | destination current << 16 (0xffff: kept in registers),
//   polarisation vector | propagator photon set << 8 | side << 24,
// with the fixed spinors u and ubar as currents 0 and 1 and the schedule's
// stored currents from 2.  The kept levels come first, one group per phase;
// then, per photon set, one item per lane of a warp (part): the NL left
// leaves (kept in the lanes' registers), the NR right leaves (destination:
// the position in the warp's current buffer of the set's right leaves), and
// idle lanes (no store, no join); then one set of idle items per warp (a
// software-pipelined kernel forms its next set's items while it joins the
// current one).  Two alternating buffers per warp of a team.  Items without
// a propagator name photon set 0 (the kernel's identity entry).  Leaves the
// plan without the form where the kernel or the schedule's shape does not
// allow it.
qed_status setup_fixed_join(qed_plan_s* P, bool mixed, int dev_smem, int sms) {
  const KernelChoice kc = fixed_join_kernel(P->k, mixed);
  if (!kc.fn) return QED_OK;
  const int k = P->k, n = k + 1, h = (n + 1) / 2, r = n - h;
  const int team = kc.team;
  Schedule sc;
  try {
    sc = build_schedule(k, false, h - 1, r - 1);
  } catch (const std::bad_alloc&) {
    return QED_ENOMEM;
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  const int NL = sc.n_left_leaves, NR = sc.n_right_leaves;
  const int wl = std::min(team, 32), nw = team / wl;   // lanes per warp (part), warps per team
  if (sc.n_set_phases != 1 || NL + NR > wl || sc.n_stored_phases > 8) return QED_OK;
  const int rbase = 2 + sc.stored_currents, ncur = rbase + nw * 2 * NR;
  if (ncur >= 0xffff) return QED_OK;
  std::vector<uint32_t> w;
  auto push = [&](const Instr& in, int dst) {
    const uint32_t src = in.src < 0 ? (uint32_t)in.side : (uint32_t)in.src + 2;
    const uint32_t eps = (uint32_t)in.photon * 2 + (uint32_t)(P->fixed_pol[in.photon] & 1);
    w.push_back(src | ((uint32_t)dst << 16));
    w.push_back(eps | ((uint32_t)in.post << 8) | ((uint32_t)in.side << 24));
  };
  int group[9] = {0};
  for (int g = 0; g < sc.n_stored_phases; ++g) {
    const Phase& ph = sc.phases[g];
    for (int slot = 0; slot < 2; ++slot)
      for (int i = 0; i < ph.cnt[slot]; ++i) {
        const Instr& in = sc.instr[ph.beg[slot] + i];
        push(in, in.dst + 2);
      }
    group[g + 1] = (int)(w.size() / 2);
  }
  const int set_off = (int)(w.size() / 2);
  for (size_t s = 0; s < sc.sets.size(); ++s) {
    const Phase& ph = sc.phases[sc.sets[s].phase0];
    if (ph.cnt[0] != NL || ph.cnt[1] != NR || ph.level[0] != h || ph.level[1] != r) return QED_OK;
    for (int lane = 0; lane < wl; ++lane) {
      if (lane < NL) {
        const Instr& in = sc.instr[ph.beg[0] + lane];
        if (in.post != 0 || in.side != 0) return QED_OK;
        push(in, 0xffff);
      } else if (lane < NL + NR) {
        const Instr& in = sc.instr[ph.beg[1] + lane - NL];
        if (in.side != 1) return QED_OK;
        push(in, lane - NL);
      } else {
        w.push_back(0xffffu << 16);
        w.push_back(0);
      }
    }
  }
  for (int lane = 0; lane < nw * wl; ++lane) {   // idle sets after the last, one per warp
    w.push_back(0xffffu << 16);
    w.push_back(0);
  }
  const int bytes = team_layout(k, mixed ? 4 : 8, ncur).bytes;
  qed_plan_s::Form f{kc, 128, 0, 0, false, bytes};
  f.smem = (size_t)(f.block / team) * bytes;
  while (f.smem > (size_t)dev_smem && f.block > team) {
    f.block /= 2;
    f.smem = (size_t)(f.block / team) * bytes;
  }
  if (f.smem > (size_t)dev_smem) return QED_OK;
  std::vector<int> items(w.begin(), w.end());
  cudaError_t e = upload(&P->d_fix_items, items);
  if (e == cudaSuccess) e = configure_form(&f, sms);
  if (e != cudaSuccess) return cuda_status(e);
  if (!f.ok) return QED_OK;
  P->fix_ngroups = sc.n_stored_phases;
  for (int g = 0; g < 9; ++g) P->fix_group[g] = group[g];
  P->fix_set_off = set_off;
  P->fix_rbase = rbase;
  P->fix_ncur = ncur;
  P->forms[1] = f;
  return QED_OK;
}

// The form a new plan starts with, from measurements on B300: the
// specialised kernel wherever it exists, except one fixed state in FP64,
// where the table kernel (bound by the FP64 pipe; one code path for the
// items of both sides) is faster but at k = 3 and 4: per launch, table
// against register-join, 1.37 / 1.63 ms (k = 1, 1,048,576 points),
// 3.65 / 4.20 (k = 2), 5.40 / 3.90 (k = 3, 524,288), 8.47 / 6.08 (k = 4,
// 262,144), 5.15 / 7.11 (k = 5, 65,536), 5.39 / 6.12 (k = 6, 16,384).
int default_form(const qed_plan_s* P) {
  if (!P->forms[1].ok) return 0;
  if (!P->summed && P->prec == QED_FP64 && P->k != 3 && P->k != 4) return 0;
  return 1;
}

}  // namespace

extern "C" {

qed_status qed_debug_inject_alloc_failure(int after) {
  if (after < -1) return QED_EINVAL;
  g_alloc_fail_after.store(after);
  return QED_OK;
}

const char* qed_status_string(qed_status s) {
  switch (s) {
    case QED_OK: return "ok";
    case QED_EINVAL: return "invalid argument";
    case QED_ENOMEM: return "out of memory";
    case QED_ECUDA: return "CUDA runtime error";
    case QED_EUNSUPPORTED: return "unsupported request";
    case QED_EDEVICE_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

qed_status qed_dag_counts(int k, qed_dag_counts_t* out) {
  if (!out || k < 1 || k > 8) return QED_EINVAL;
  try {
    Counts u = unreduced_counts(k);
    Counts r;
    if (k <= 7) {
      Dag g = generate(k);
      Counts ug = g.counts();
      if (ug.total != u.total) return QED_EUNSUPPORTED;
      r = reduce(g).counts();
    } else {
      r.total = r.data = r.u = r.v = r.s1 = r.s2 = r.sum = -1;
    }
    out->unreduced_total = u.total; out->unreduced_data = u.data; out->unreduced_u = u.u;
    out->unreduced_v = u.v; out->unreduced_s1 = u.s1; out->unreduced_s2 = u.s2;
    out->unreduced_sum = u.sum;
    out->reduced_total = r.total; out->reduced_data = r.data; out->reduced_u = r.u;
    out->reduced_v = r.v; out->reduced_s1 = r.s1; out->reduced_s2 = r.s2; out->reduced_sum = r.sum;
  } catch (const std::bad_alloc&) {
    return QED_ENOMEM;
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  return QED_OK;
}

namespace {
qed_status create_plan(const qed_process* process, const qed_spin_cfg* spin, qed_precision precision,
                       bool rewrite, qed_plan_t* out) {
  if (!process || !spin || !out) return QED_EINVAL;
  const int k = process->k;
  if (k < 1 || k > 7) return QED_EINVAL;
  if (!(process->mass > 0.0) || !std::isfinite(process->mass) || !std::isfinite(process->charge))
    return QED_EINVAL;
  if (precision != QED_FP64 && precision != QED_MIXED) return QED_EINVAL;
  qed_plan_s* P = new (std::nothrow) qed_plan_s();
  if (!P) return QED_ENOMEM;
  P->k = k;
  P->summed = spin->summed != 0;
  P->prec = precision;
  P->mass = process->mass;
  P->charge = process->charge;
  if (!P->summed) {
    for (int s = 0; s < k + 3; ++s) {
      int v = spin->hel[s];
      bool electron = (s == 0 || s == 2);
      if (electron ? (v != 1 && v != -1) : (v != 1 && v != 2)) { delete P; return QED_EINVAL; }
    }
    P->fixed_sin = spin->hel[0] == 1 ? 0 : 1;
    P->fixed_sout = spin->hel[2] == 1 ? 0 : 1;
    P->fixed_pol[0] = spin->hel[1] - 1;
    for (int j = 1; j <= k; ++j) P->fixed_pol[j] = spin->hel[j + 2] - 1;
  }
  int ls, rs;
  default_levels(k, P->summed, precision == QED_MIXED, &ls, &rs);
  P->rewrite = rewrite;
  const bool mixed = precision == QED_MIXED;
  P->kc = rewrite ? rewrite_kernel(k, P->summed, mixed) : forward_kernel(k, P->summed, mixed);
  if (!P->kc.fn) { delete P; return QED_EUNSUPPORTED; }
  int dev_smem = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  if (e != cudaSuccess) { delete P; return cuda_status(e); }
  try {
    P->sc = build_schedule(k, P->summed, ls, rs);
    if (rewrite) {
      // photon sets per set phase: as many as keep a team's shared memory
      // within half the SM's (two resident teams), or within all of it when
      // the stored currents alone exceed that
      const int real = mixed ? 4 : 8;
      int g = rewrite_default_group(k, P->summed, P->kc.team);
      const RwSchedule one = build_rewrite_schedule(k, P->summed, 1);
      const int budget = team_layout(k, real, one.stored_currents + one.local_currents).bytes <= dev_smem / 2
                             ? dev_smem / 2 : dev_smem;
      for (;;) {
        P->rsc = build_rewrite_schedule(k, P->summed, g);
        if (g == 1 || team_layout(k, real, P->rsc.stored_currents + P->rsc.local_currents).bytes <= budget)
          break;
        g = (g + 1) / 2;
      }
    }
  } catch (const std::bad_alloc&) {
    delete P;
    return QED_ENOMEM;
  } catch (...) {
    delete P;
    return QED_EUNSUPPORTED;
  }
  if (P->summed) {
    // lane table: leaf variants of every (photon set, polarisation pattern)
    const int n = k + 1;
    const auto& sets = rewrite ? P->rsc.sets : P->sc.sets;
    std::vector<uint16_t> tab(sets.size() << n);
    for (size_t s = 0; s < sets.size(); ++s) {
      const unsigned S = sets[s].mask, C = ((1u << n) - 1) & ~S;
      for (unsigned c = 0; c < (1u << n); ++c) {
        unsigned l = 0, r = 0;
        int ol = 0, orr = 0;
        for (int j = 0; j < n; ++j) {
          const unsigned b = (c >> j) & 1u;
          if (S & (1u << j)) l |= b << ol++;
          if (C & (1u << j)) r |= b << orr++;
        }
        tab[(s << n) + c] = (uint16_t)(l | (r << 8));
      }
    }
    if (e == cudaSuccess) e = upload(&P->d_lane_tab, tab);
    // inverse: the polarisation pattern of each left / right leaf variant
    const int h = (n + 1) / 2, r = n - h, row = (1 << h) + (1 << r);
    std::vector<uint16_t> dep(sets.size() * row);
    for (size_t s = 0; s < sets.size(); ++s) {
      const unsigned S = sets[s].mask, C = ((1u << n) - 1) & ~S;
      for (int side = 0; side < 2; ++side) {
        const unsigned M = side == 0 ? S : C;
        const int cnt = side == 0 ? (1 << h) : (1 << r);
        for (int v = 0; v < cnt; ++v) {
          unsigned d = 0;
          int o = 0;
          for (int j = 0; j < n; ++j)
            if (M & (1u << j)) d |= (((unsigned)v >> o++) & 1u) << j;
          dep[s * row + (side == 0 ? 0 : (1 << h)) + v] = (uint16_t)d;
        }
      }
    }
    if (e == cudaSuccess) e = upload(&P->d_dep_tab, dep);
  }
  if (rewrite) {
    if (e == cudaSuccess) e = upload(&P->d_sinstr, P->rsc.instr);
    if (e == cudaSuccess) e = upload(&P->d_phases, P->rsc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets, P->rsc.sets);
  } else {
    if (e == cudaSuccess) e = upload(&P->d_instr, P->sc.instr);
    if (e == cudaSuccess) e = upload(&P->d_phases, P->sc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets, P->sc.sets);
  }
  if (e != cudaSuccess) { free_plan(P); return cuda_status(e); }
  const int ncur = rewrite ? P->rsc.stored_currents + P->rsc.local_currents
                           : P->sc.stored_currents + P->sc.local_currents;
  TeamLayout L = team_layout(k, mixed ? 4 : 8, ncur);
  P->team_bytes = L.bytes;
  P->block = P->kc.team > 32 ? P->kc.team : 128;
  P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  while (P->smem > (size_t)dev_smem && P->block > P->kc.team && P->block > 32) {
    P->block /= 2;
    P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  }
  if (P->smem > (size_t)dev_smem) { free_plan(P); return QED_EUNSUPPORTED; }
  e = cudaFuncSetAttribute((const void*)P->kc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)P->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)P->kc.fn, P->block,
                                                      P->smem);
  if (e != cudaSuccess || per_sm < 1) { free_plan(P); return e != cudaSuccess ? cuda_status(e) : QED_EUNSUPPORTED; }
  P->grid = per_sm * sms;
  P->forms[0] = qed_plan_s::Form{P->kc, P->block, P->grid, P->smem, true, L.bytes};
  if (!rewrite && P->summed) {
    const SpecKernel sk = spec_forward_kernel(k, mixed);
    const int spec_ncur = P->sc.stored_currents + P->sc.local_currents;
    if (sk.fn && sk.team == P->kc.team && sk.ncur == spec_ncur &&
        sk.team_bytes == team_layout(k, mixed ? 4 : 8, spec_ncur).bytes) {
      qed_plan_s::Form f{KernelChoice{sk.fn, sk.team}, P->block, 0, 0, false, sk.team_bytes};
      f.smem = (size_t)(f.block / sk.team) * sk.team_bytes;
      while (f.smem > (size_t)dev_smem && f.block > sk.team) {
        f.block /= 2;
        f.smem = (size_t)(f.block / sk.team) * sk.team_bytes;
      }
      if (f.smem <= (size_t)dev_smem) {
        e = configure_form(&f, sms);
        if (e != cudaSuccess) { free_plan(P); return cuda_status(e); }
        P->forms[1] = f;
      }
    }
  }
  if (!rewrite && !P->summed) {
    qed_status fs = setup_fixed_join(P, mixed, dev_smem, sms);
    if (fs != QED_OK) { free_plan(P); return fs; }
  }
  P->form.store(default_form(P));
  if (!rewrite) {
    qed_status as = setup_adjoint(P, mixed, dev_smem, sms);
    if (as != QED_OK) { free_plan(P); return as; }
  }
  *out = P;
  return QED_OK;
}
}  // namespace

qed_status qed_plan_create(const qed_process* process, const qed_spin_cfg* spin,
                           qed_precision precision, qed_plan_t* out) {
  return create_plan(process, spin, precision, false, out);
}

qed_status qed_plan_create_rewrite(const qed_process* process, const qed_spin_cfg* spin,
                                   qed_precision precision, qed_plan_t* out) {
  return create_plan(process, spin, precision, true, out);
}

qed_status qed_abc_plan_create(const qed_abc_process* proc, qed_precision precision, int rewrite,
                               qed_plan_t* out) {
  if (!proc || !out) return QED_EINVAL;
  const int k = proc->k;
  if (k < 1 || k > 7 || k % 2 == 0) return QED_EINVAL;
  for (double m : {proc->mass_a, proc->mass_b, proc->mass_c})
    if (!(m >= 0.0) || !std::isfinite(m)) return QED_EINVAL;
  if (!std::isfinite(proc->coupling)) return QED_EINVAL;
  if (precision != QED_FP64 && precision != QED_MIXED) return QED_EINVAL;
  const bool mixed = precision == QED_MIXED;
  qed_plan_s* P = new (std::nothrow) qed_plan_s();
  if (!P) return QED_ENOMEM;
  P->k = k;
  P->summed = false;
  P->prec = precision;
  P->mass = proc->mass_a;
  P->mass_c = proc->mass_c;
  P->charge = proc->coupling;
  P->abc = true;
  P->rewrite = rewrite != 0;
  P->kc = abc_kernel_for(k, mixed, P->rewrite);
  if (!P->kc.fn) { delete P; return QED_EUNSUPPORTED; }
  int dev_smem = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  if (e != cudaSuccess) { delete P; return cuda_status(e); }
  const int n = k + 1;
  try {
    int ls, rs;
    default_levels(k, false, false, &ls, &rs);
    P->sc = build_schedule(k, false, ls, rs);
    if (P->rewrite) P->rsc = build_rewrite_schedule(k, false, rewrite_default_group(k, false, P->kc.team));
  } catch (const std::bad_alloc&) {
    delete P;
    return QED_ENOMEM;
  } catch (...) {
    delete P;
    return QED_EUNSUPPORTED;
  }
  // algorithmic FLOPs of the scalar DAG, each node once
  long long fl = ((1ll << n) - 2) * FLOP_ABC_SUBSET + 2;
  if (P->rewrite) {
    fl += (P->rsc.terms - P->rsc.nodes) + P->rsc.s1_nodes * FLOP_ABC_S1 + P->rsc.joins * FLOP_ABC_JOIN;
  } else {
    long long right_leaves = 0, fr = 1, c = 1;
    for (int i = 2; i <= P->sc.r; ++i) fr *= i;
    for (int i = 1; i <= P->sc.h; ++i) c = c * (n - P->sc.h + i) / i;
    right_leaves = c * fr;   // the middle propagator, applied to each right leaf
    fl += (P->sc.s1_nodes + right_leaves) * FLOP_ABC_S1 + P->sc.s2_nodes * FLOP_ABC_JOIN;
  }
  P->abc_flops = fl;
  if (P->rewrite) {
    if (e == cudaSuccess) e = upload(&P->d_sinstr, P->rsc.instr);
    if (e == cudaSuccess) e = upload(&P->d_phases, P->rsc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets, P->rsc.sets);
  } else {
    if (e == cudaSuccess) e = upload(&P->d_instr, P->sc.instr);
    if (e == cudaSuccess) e = upload(&P->d_phases, P->sc.phases);
    if (e == cudaSuccess) e = upload(&P->d_sets, P->sc.sets);
  }
  if (e != cudaSuccess) { free_plan(P); return cuda_status(e); }
  const int ncur = P->rewrite ? P->rsc.stored_currents + P->rsc.local_currents
                              : P->sc.stored_currents + P->sc.local_currents;
  const AbcLayout L = abc_layout(k, mixed ? 4 : 8, ncur);
  P->team_bytes = L.bytes;
  P->block = std::max(128, P->kc.team);
  P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  while (P->smem > (size_t)dev_smem && P->block > P->kc.team && P->block > 32) {
    P->block /= 2;
    P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  }
  if (P->smem > (size_t)dev_smem) { free_plan(P); return QED_EUNSUPPORTED; }
  e = cudaFuncSetAttribute((const void*)P->kc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)P->kc.fn, P->block, P->smem);
  if (e != cudaSuccess || per_sm < 1) { free_plan(P); return e != cudaSuccess ? cuda_status(e) : QED_EUNSUPPORTED; }
  P->grid = per_sm * sms;
  P->forms[0] = qed_plan_s::Form{P->kc, P->block, P->grid, P->smem, true, P->team_bytes};
  *out = P;
  return QED_OK;
}

qed_status qed_reduction_steps(int k, int* steps) {
  if (!steps || k < 1 || k > 6) return QED_EINVAL;
  try {
    *steps = reduction_steps(k);
  } catch (const std::bad_alloc&) {
    return QED_ENOMEM;
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  return QED_OK;
}

qed_status qed_tape_export(int k, int steps, qed_tape_desc_t* desc, void* instr, int* levels) {
  if (!desc || k < 1 || k > 5 || steps < 0) return QED_EINVAL;
  Tape t;
  try {
    t = build_tape(k, steps);
  } catch (const std::bad_alloc&) {
    return QED_ENOMEM;
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  desc->k = t.k; desc->n = t.n; desc->steps = t.steps; desc->n_slots = t.n_slots; desc->n_diag = t.n_diag;
  desc->n_instr = (int)t.instr.size();
  desc->n_levels = (int)t.level_beg.size() - 1;
  desc->nodes = t.counts.total;
  desc->compute_nodes = t.counts.total - t.counts.data;
  desc->flops = t.flops;
  if (instr) std::memcpy(instr, t.instr.data(), t.instr.size() * sizeof(TapeInstr));
  if (levels) std::memcpy(levels, t.level_beg.data(), t.level_beg.size() * sizeof(int32_t));
  return QED_OK;
}

qed_status qed_tape_plan_create(const qed_process* process, const qed_spin_cfg* spin, int reduction_steps,
                                qed_plan_t* out) {
  if (!process || !spin || !out || reduction_steps < 0) return QED_EINVAL;
  const int k = process->k;
  if (k < 1 || k > 5 || spin->summed) return QED_EINVAL;
  if (!(process->mass > 0.0) || !std::isfinite(process->mass) || !std::isfinite(process->charge))
    return QED_EINVAL;
  qed_plan_s* P = new (std::nothrow) qed_plan_s();
  if (!P) return QED_ENOMEM;
  P->k = k;
  P->summed = false;
  P->prec = QED_FP64;
  P->mass = process->mass;
  P->charge = process->charge;
  P->is_tape = true;
  for (int s = 0; s < k + 3; ++s) {
    const int h = spin->hel[s];
    const bool electron = s == 0 || s == 2;
    if (electron ? (h != 1 && h != -1) : (h != 1 && h != 2)) { delete P; return QED_EINVAL; }
  }
  P->fixed_sin = spin->hel[0] == 1 ? 0 : 1;
  P->fixed_sout = spin->hel[2] == 1 ? 0 : 1;
  P->fixed_pol[0] = spin->hel[1] - 1;
  for (int j = 1; j <= k; ++j) P->fixed_pol[j] = spin->hel[j + 2] - 1;
  P->kc = tape_kernel();
  int dev_smem = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  if (e != cudaSuccess) { delete P; return cuda_status(e); }
  try {
    int ls, rs;
    default_levels(k, false, false, &ls, &rs);
    P->sc = build_schedule(k, false, ls, rs);
    P->tp = build_tape(k, reduction_steps);
  } catch (const std::bad_alloc&) {
    delete P;
    return QED_ENOMEM;
  } catch (...) {
    delete P;
    return QED_EUNSUPPORTED;
  }
  const TapeLayout L = tape_layout(k, P->tp.n_slots, P->tp.n_diag);
  P->team_bytes = L.bytes;
  P->block = P->kc.team;   // one team per block: the occupancy follows the team's slots
  P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  while (P->smem > (size_t)dev_smem && P->block > P->kc.team) {
    P->block /= 2;
    P->smem = (size_t)(P->block / P->kc.team) * L.bytes;
  }
  if (P->smem > (size_t)dev_smem) { delete P; return QED_EUNSUPPORTED; }
  e = upload(&P->d_tape, P->tp.instr);
  if (e == cudaSuccess) e = upload(&P->d_levels, P->tp.level_beg);
  if (e != cudaSuccess) { free_plan(P); return cuda_status(e); }
  e = cudaFuncSetAttribute((const void*)P->kc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)P->kc.fn, P->block, P->smem);
  if (e != cudaSuccess || per_sm < 1) { free_plan(P); return e != cudaSuccess ? cuda_status(e) : QED_EUNSUPPORTED; }
  P->grid = per_sm * sms;
  P->forms[0] = qed_plan_s::Form{P->kc, P->block, P->grid, P->smem, true, P->team_bytes};
  *out = P;
  return QED_OK;
}

qed_status qed_plan_info(qed_plan_t P, qed_plan_info_t* info) {
  if (!P || !info) return QED_EINVAL;
  std::memset(info, 0, sizeof(*info));
  const Schedule& sc = P->sc;
  info->k = P->k;
  info->n_photons = sc.n;
  long long d = 1;
  for (int i = 2; i <= sc.n; ++i) d *= i;
  info->n_diagrams = d;
  info->n_states = P->summed ? (1ll << (sc.n + 2)) : 1;
  info->nodes_unreduced = sc.unreduced.total;
  info->nodes_reduced = sc.reduced.total;
  info->compute_reduced = sc.reduced.total - sc.reduced.data;
  info->v_nodes = sc.v_nodes;
  info->s1_nodes = sc.s1_nodes;
  info->s2_nodes = sc.s2_nodes;
  info->flops_per_point = P->rewrite ? P->rsc.flops_algorithmic : sc.flops_algorithmic;
  info->flops_executed_per_point = P->rewrite ? P->rsc.flops_algorithmic : sc.flops_executed;
  if (P->rewrite) {
    info->nodes_reduced = P->rsc.nodes;      // subset nodes times spin variants
    info->v_nodes = P->rsc.terms;
    info->s1_nodes = P->rsc.s1_nodes;
    info->s2_nodes = P->rsc.joins;
  }
  info->flops_literal_s2_per_point = sc.flops_literal_s2;
  if (P->abc) {
    info->flops_per_point = info->flops_executed_per_point = P->abc_flops;
    info->flops_literal_s2_per_point = 0;
  }
  if (P->is_tape) {
    const Counts& c = P->tp.counts;
    info->nodes_reduced = c.total;
    info->compute_reduced = c.total - c.data;
    info->v_nodes = c.v;
    info->s1_nodes = c.s1;
    info->s2_nodes = c.s2;
    info->flops_per_point = info->flops_executed_per_point = P->tp.flops;
    info->flops_literal_s2_per_point = P->tp.flops;
    info->reduction_steps = P->tp.steps;
  }
  const int f = P->form.load();
  info->team_threads = P->forms[f].kc.team;
  info->smem_bytes_per_team = P->forms[f].team_bytes;
  info->precision = (int)P->prec;
  info->kernel_form = f;
  info->kernel_forms = (P->forms[0].ok ? 1 : 0) | (P->forms[1].ok ? 2 : 0);
  info->block_threads = P->forms[f].block;
  info->grid_blocks = P->forms[f].grid;
  return QED_OK;
}

qed_status qed_plan_set_kernel_form(qed_plan_t P, int form) {
  if (!P || form < 0 || form > 1) return QED_EINVAL;
  if (!P->forms[form].ok) return QED_EUNSUPPORTED;
  P->form.store(form);
  return QED_OK;
}

qed_status qed_plan_tune(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2, void* stream,
                         int* form, int* block, double* best_ms) {
  if (!P || n <= 0 || !d_momenta || !d_out_m2 || !aligned8(d_momenta) || !aligned8(d_out_m2))
    return QED_EINVAL;
  int sms = 0, dev_smem = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QED_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QED_ECUDA; }
  const int orig = P->form.load();
  const qed_plan_s::Form saved[2] = {P->forms[0], P->forms[1]};
  int best_f = orig;
  qed_plan_s::Form best_cfg = P->forms[orig];
  double best = 1e300;
  qed_status s = QED_OK;
  for (int f = 0; f < 2 && s == QED_OK; ++f) {
    if (!saved[f].ok) continue;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, (const void*)saved[f].kc.fn) != cudaSuccess) { s = QED_ECUDA; break; }
    const int team = saved[f].kc.team;
    for (int blk : {32, 64, 128, 256}) {
      if (blk < team || blk % team || blk > fa.maxThreadsPerBlock) continue;
      qed_plan_s::Form c = saved[f];
      c.block = blk;
      c.smem = (size_t)(blk / team) * c.team_bytes;
      if (c.smem > (size_t)dev_smem) continue;
      if (configure_form(&c, sms) != cudaSuccess) { s = QED_ECUDA; break; }
      if (!c.ok) continue;
      P->forms[f] = c;
      P->form.store(f);
      s = launch_eval(P, d_momenta, n, d_out_m2, st);   // warm-up
      if (s != QED_OK) break;
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && s == QED_OK; ++rep) s = launch_eval(P, d_momenta, n, d_out_m2, st);
      cudaEventRecord(e1, st);
      if (s != QED_OK || cudaEventSynchronize(e1) != cudaSuccess) { s = s != QED_OK ? s : QED_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 3 < best) { best = ms / 3; best_f = f; best_cfg = c; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->forms[0] = saved[0];
  P->forms[1] = saved[1];
  if (s == QED_OK && best < 1e300) {
    P->forms[best_f] = best_cfg;
    if (configure_form(&P->forms[best_f], sms) != cudaSuccess) s = QED_ECUDA;
    P->form.store(best_f);
  } else {
    for (int f = 0; f < 2; ++f)
      if (saved[f].ok) configure_form(&P->forms[f], sms);
    P->form.store(orig);
  }
  if (s == QED_OK) {
    if (form) *form = best_f;
    if (block) *block = P->forms[best_f].block;
    if (best_ms) *best_ms = best;
  }
  return s;
}

qed_status qed_eval(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2,
                    void* stream) {
  if (!P || n < 0) return QED_EINVAL;
  if (n == 0) return QED_OK;
  if (!d_momenta || !d_out_m2 || !aligned8(d_momenta) || !aligned8(d_out_m2)) return QED_EINVAL;
  return launch_eval(P, d_momenta, n, d_out_m2, (cudaStream_t)stream);
}

namespace {
qed_status launch_grad(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2, double* d_grad,
                       void* scratch, cudaStream_t st) {
  KParams kp = make_params(P, d_momenta, n, d_out_m2);
  kp.grad = d_grad;
  kp.instr = P->d_instr_adj;
  kp.phases = P->d_phases_adj;
  kp.sets = P->d_sets_adj;
  kp.n_stored_phases = P->sc_adj.n_stored_phases;
  kp.n_set_phases = P->sc_adj.n_set_phases;
  kp.n_sets = (int)P->sc_adj.sets.size();
  kp.ncur = P->sc_adj.stored_currents + P->sc_adj.local_currents;
  kp.ncur_stored = P->sc_adj.stored_currents;
  kp.adj_scratch = scratch;
  kp.adj_scratch_team = P->adj_scratch_team;
  kp.part_tab = P->d_part_tab;
  kp.n_part = P->n_part;
  if (P->radj) {
    kp.radj_masks = P->d_radj_masks;
    kp.radj_slot = P->d_radj_slot;
    kp.radj_aslot = P->d_radj_aslot;
    kp.radj_nadj = P->radj_nadj;
    std::memcpy(kp.radj_lev, P->radj_lev, sizeof(kp.radj_lev));
    kp.ncur = P->radj_ncur;
  }
  const int tpc = P->block_adj / P->kc_adj.team;
  const long long need = (n + tpc - 1) / tpc;
  const int grid = (int)std::min<long long>(need, P->grid_adj);
  return cuda_status(launch_forward(P->kc_adj.fn, grid, P->block_adj, P->smem_adj, st, kp));
}

qed_status check_grad_args(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2,
                           double* d_grad) {
  if (!P || n < 0) return QED_EINVAL;
  if (n == 0) return QED_OK;
  if (!d_momenta || !d_grad || !aligned8(d_momenta) || !aligned8(d_grad) ||
      (d_out_m2 && !aligned8(d_out_m2)))
    return QED_EINVAL;
  if (!P->has_adj) return QED_EUNSUPPORTED;
  return QED_OK;
}
}  // namespace

qed_status qed_eval_grad(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2,
                         double* d_grad, void* stream) {
  qed_status s = check_grad_args(P, d_momenta, n, d_out_m2, d_grad);
  if (s != QED_OK || n == 0) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (!P->d_adj_scratch) return launch_grad(P, d_momenta, n, d_out_m2, d_grad, nullptr, st);
  // the plan's scratch: order this launch after the previous one that used
  // it, whatever its stream (inside a stream capture the ordering is the
  // capture's own; see qed.h)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return cuda_status(e);
  if (cs != cudaStreamCaptureStatusNone)
    return launch_grad(P, d_momenta, n, d_out_m2, d_grad, P->d_adj_scratch, st);
  std::lock_guard<std::mutex> guard(P->scratch_lock);
  if (P->scratch_used) e = cudaStreamWaitEvent(st, P->ev_scratch, 0);
  if (e != cudaSuccess) return cuda_status(e);
  s = launch_grad(P, d_momenta, n, d_out_m2, d_grad, P->d_adj_scratch, st);
  if (s != QED_OK) return s;
  e = cudaEventRecord(P->ev_scratch, st);
  if (e != cudaSuccess) return cuda_status(e);
  P->scratch_used = true;
  return QED_OK;
}

qed_status qed_grad_workspace_bytes(qed_plan_t P, long long* bytes) {
  if (!P || !bytes) return QED_EINVAL;
  if (!P->has_adj) return QED_EUNSUPPORTED;
  *bytes = P->d_adj_scratch ? P->adj_scratch_bytes : 0;
  return QED_OK;
}

qed_status qed_eval_grad_ws(qed_plan_t P, const double* d_momenta, long long n, double* d_out_m2,
                            double* d_grad, void* d_workspace, long long workspace_bytes, void* stream) {
  qed_status s = check_grad_args(P, d_momenta, n, d_out_m2, d_grad);
  if (s != QED_OK) return s;
  if (workspace_bytes < 0 || ((uintptr_t)d_workspace & 255u)) return QED_EINVAL;
  if (P->d_adj_scratch && (!d_workspace || workspace_bytes < P->adj_scratch_bytes)) return QED_EINVAL;
  if (n == 0) return QED_OK;
  return launch_grad(P, d_momenta, n, d_out_m2, d_grad, P->d_adj_scratch ? d_workspace : nullptr,
                     (cudaStream_t)stream);
}

qed_status qed_eval_host(qed_plan_t P, const double* h_momenta, long long n, double* h_out_m2,
                         void* stream) {
  if (!P || n < 0) return QED_EINVAL;
  if (n == 0) return QED_OK;
  if (!h_momenta || !h_out_m2) return QED_EINVAL;
  std::lock_guard<std::mutex> guard(P->stage_lock);   // the staging is the plan's
  cudaStream_t st = (cudaStream_t)stream;
  const long long stride = (long long)(P->k + 3) * 4;
  // two staging buffers of `chunk` points each: momenta then |M|^2.  The
  // chunks start at chunk / 8 and double up to chunk, so that only the
  // first (small) copy runs before any kernel: each kernel covers the copy
  // of the next, larger chunk.
  const long long chunk = std::min<long long>(n, std::max<long long>(1 << 16, (n + 7) / 8));
  const long long first = std::max<long long>(std::min<long long>(chunk, 8192), chunk / 8);
  cudaError_t e = cudaSuccess;
  if (chunk > P->stage_cap) {
    cudaFree(P->d_stage);
    P->d_stage = nullptr;
    P->stage_cap = 0;
    e = device_alloc((void**)&P->d_stage, (size_t)2 * chunk * (stride + 1) * sizeof(double));
    if (e != cudaSuccess) return cuda_status(e);
    P->stage_cap = chunk;
  }
  if (!P->s_h2d) {
    e = cudaStreamCreateWithFlags(&P->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->s_d2h, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&P->ev_h2d[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_k[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_d2h[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  const long long cap = P->stage_cap;
  double* mom_buf[2] = {P->d_stage, P->d_stage + cap * stride};
  double* out_buf[2] = {P->d_stage + 2 * cap * stride, P->d_stage + 2 * cap * stride + cap};
  // order the staging buffers after earlier work on the caller's stream
  cudaEvent_t start = P->ev_k[0];
  e = cudaEventRecord(start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_h2d, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_d2h, start, 0);
  long long c = 0, size = first, m = 0;
  for (long long off = 0; off < n && e == cudaSuccess; off += m, ++c, size = std::min(chunk, 2 * size)) {
    const int b = (int)(c & 1);
    m = std::min(size, n - off);
    if (c >= 2) e = cudaStreamWaitEvent(P->s_h2d, P->ev_k[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(mom_buf[b], h_momenta + off * stride, (size_t)m * stride * sizeof(double),
                          cudaMemcpyHostToDevice, P->s_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_h2d[b], P->s_h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P->ev_h2d[b], 0);
    if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(st, P->ev_d2h[b], 0);
    if (e == cudaSuccess) {
      qed_status s = launch_eval(P, mom_buf[b], m, out_buf[b], st);
      if (s != QED_OK) {
        // let the copies already queued finish with the caller's buffers
        cudaStreamSynchronize(P->s_h2d);
        cudaStreamSynchronize(P->s_d2h);
        return s;
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_k[b], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_d2h, P->ev_k[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_out_m2 + off, out_buf[b], (size_t)m * sizeof(double),
                          cudaMemcpyDeviceToHost, P->s_d2h);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_d2h[b], P->s_d2h);
  }
  if (e != cudaSuccess) cudaStreamSynchronize(P->s_h2d);   // no copy outlives the call
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->s_d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e);
}

void qed_plan_destroy(qed_plan_t P) { free_plan(P); }

// Export of a schedule's tables for host-side inspection (no GPU needed).
qed_status qed_schedule_export(int k, int summed, qed_schedule_desc_t* desc, void* instr,
                               void* phases, void* sets) {
  if (!desc || k < 1 || k > 7) return QED_EINVAL;
  int ls, rs;
  default_levels(k, summed != 0, false, &ls, &rs);
  Schedule sc;
  try {
    sc = build_schedule(k, summed != 0, ls, rs);
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  desc->k = sc.k; desc->n = sc.n; desc->h = sc.h; desc->r = sc.r;
  desc->ls = sc.ls; desc->rs = sc.rs; desc->summed = sc.summed ? 1 : 0;
  desc->n_left_leaves = sc.n_left_leaves; desc->n_right_leaves = sc.n_right_leaves;
  desc->stored_currents = sc.stored_currents; desc->local_currents = sc.local_currents;
  desc->n_stored_phases = sc.n_stored_phases; desc->n_set_phases = sc.n_set_phases;
  desc->n_sets = (int)sc.sets.size(); desc->n_instr = (int)sc.instr.size();
  desc->n_phases = (int)sc.phases.size();
  desc->flops_algorithmic = sc.flops_algorithmic;
  desc->flops_executed = sc.flops_executed;
  if (instr) std::memcpy(instr, sc.instr.data(), sc.instr.size() * sizeof(Instr));
  if (phases) std::memcpy(phases, sc.phases.data(), sc.phases.size() * sizeof(Phase));
  if (sets) std::memcpy(sets, sc.sets.data(), sc.sets.size() * sizeof(SetEntry));
  return QED_OK;
}

qed_status qed_rewrite_schedule_export(int k, int summed, int group, qed_schedule_desc_t* desc,
                                       void* instr, void* phases, void* sets) {
  if (!desc || k < 1 || k > 7 || group < 0) return QED_EINVAL;
  RwSchedule sc;
  try {
    sc = build_rewrite_schedule(k, summed != 0, group);
  } catch (...) {
    return QED_EUNSUPPORTED;
  }
  std::memset(desc, 0, sizeof(*desc));
  desc->k = sc.k; desc->n = sc.n; desc->h = sc.h; desc->r = sc.r; desc->summed = sc.summed ? 1 : 0;
  desc->n_left_leaves = 1; desc->n_right_leaves = 1;
  desc->stored_currents = sc.stored_currents; desc->local_currents = sc.local_currents;
  desc->n_stored_phases = sc.n_stored_phases; desc->n_set_phases = sc.n_set_phases;
  desc->n_sets = (int)sc.sets.size(); desc->n_instr = (int)sc.instr.size();
  desc->n_phases = (int)sc.phases.size();
  desc->flops_algorithmic = sc.flops_algorithmic;
  desc->flops_executed = sc.flops_algorithmic;
  if (instr) std::memcpy(instr, sc.instr.data(), sc.instr.size() * sizeof(SumInstr));
  if (phases) std::memcpy(phases, sc.phases.data(), sc.phases.size() * sizeof(Phase));
  if (sets) std::memcpy(sets, sc.sets.data(), sc.sets.size() * sizeof(SetEntry));
  return QED_OK;
}

}  // extern "C"
