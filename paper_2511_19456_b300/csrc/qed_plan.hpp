// Internal plan object shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/qed.h"
#include "dag.hpp"
#include "qed_types.h"

namespace qed {
struct KernelChoice {
  void (*fn)(const KParams);
  int team;
};
KernelChoice forward_kernel(int k, bool summed, bool mixed);
KernelChoice adjoint_kernel(int k, bool summed, bool mixed);
KernelChoice adjoint_kernel_gmem(int k, bool summed, bool mixed);
KernelChoice rewrite_kernel(int k, bool summed, bool mixed);
KernelChoice abc_kernel_for(int k, bool mixed, bool rewrite);
KernelChoice tape_kernel();
cudaError_t launch_forward(void (*fn)(const KParams), int grid, int block, size_t smem,
                           cudaStream_t st, const KParams& p);
// Straight-line specialised forward kernel (generated at build time by
// qed_codegen.cpp): spin-summed, k = 1..5; fn == nullptr where none exists.
// ncur and team_bytes: the currents and shared memory per team it expects.
struct SpecKernel {
  void (*fn)(const KParams);
  int team, ncur, team_bytes;
};
SpecKernel spec_forward_kernel(int k, bool mixed);
// One fixed state, register-join form (qed_fix.cu), k = 1..6, FP32-mixed or
// FP64; fn == nullptr otherwise.
KernelChoice fixed_join_kernel(int k, bool mixed);
// Adjoint on the distributively rewritten DAG (qed_radj.cu): spin-summed
// k <= 5 and one fixed state k <= 7; fn == nullptr otherwise.
KernelChoice radj_kernel(int k, bool summed, bool mixed);
const char* spec_version();
}  // namespace qed

using namespace qed;

struct qed_plan_s {
  int k = 0;
  bool summed = true;
  qed_precision prec = QED_FP64;
  double mass = 1.0, charge = 1.0;
  Schedule sc;
  Instr* d_instr = nullptr;
  Phase* d_phases = nullptr;
  SetEntry* d_sets = nullptr;
  KernelChoice kc{nullptr, 0};
  int block = 0, grid = 0;
  size_t smem = 0;
  int team_bytes = 0;
  // Forward kernel forms of a spin-summed plan: [0] the table-driven kernel
  // above (kc, block, grid, smem: the schedule read from device tables at run
  // time), [1] the straight-line specialised kernel generated at build time
  // from the same schedule (with its own shared-memory size per team, which
  // the generator reports).  The evaluation entry points launch
  // forms[form]; form is switched by qed_plan_set_kernel_form and
  // qed_plan_tune.
  struct Form {
    KernelChoice kc{nullptr, 0};
    int block = 0, grid = 0;
    size_t smem = 0;
    bool ok = false;
    int team_bytes = 0;
  };
  Form forms[2];
  std::atomic<int> form{0};
  int fixed_sin = 0, fixed_sout = 0, fixed_pol[8] = {0};
  // adjoint: its own schedule (fewer kept levels where shared memory is short)
  Schedule sc_adj;
  Instr* d_instr_adj = nullptr;
  Phase* d_phases_adj = nullptr;
  SetEntry* d_sets_adj = nullptr;
  KernelChoice kc_adj{nullptr, 0};
  int block_adj = 0, grid_adj = 0;
  size_t smem_adj = 0;
  bool has_adj = false;
  void* d_adj_scratch = nullptr;     // global currents/adjoints of the adjoint teams
  long long adj_scratch_team = 0;    // bytes per team
  long long adj_scratch_bytes = 0;   // the whole scratch (all resident teams)
  // qed_eval_grad's uses of d_adj_scratch, on any stream, run one after the
  // other: each launch waits for ev_scratch, recorded after the previous one
  std::mutex scratch_lock;
  cudaEvent_t ev_scratch = nullptr;
  bool scratch_used = false;
  // distributively rewritten DAG (qed_plan_create_rewrite)
  bool rewrite = false;
  // ABC model (qed_abc_plan_create): scalar currents, A and C masses
  bool abc = false;
  double mass_c = 0.0;
  long long abc_flops = 0;
  // node-by-node tape of a DAG in a given reduction state (qed_tape_plan_create)
  bool is_tape = false;
  Tape tp;
  TapeInstr* d_tape = nullptr;
  int* d_levels = nullptr;
  RwSchedule rsc;
  SumInstr* d_sinstr = nullptr;
  uint16_t* d_lane_tab = nullptr;   // spin-summed plans: leaf variants per (set, lane)
  uint16_t* d_dep_tab = nullptr;    // spin-summed plans: polarisation patterns per (set, leaf variant)
  uint16_t* d_part_tab = nullptr;   // mixed adjoint: propagator of each partial-sum slot per set
  // one fixed state, mixed: the register-join form's items (KParams::fix_*)
  int* d_fix_items = nullptr;
  int fix_ngroups = 0, fix_group[9] = {0}, fix_set_off = 0, fix_rbase = 0, fix_ncur = 0;
  // the adjoint on the rewritten DAG (KParams::radj_*), when kc_adj is it
  bool radj = false;
  int* d_radj_masks = nullptr;
  int* d_radj_slot = nullptr;
  int* d_radj_aslot = nullptr;
  int radj_lev[2][10] = {{0}};
  int radj_ncur = 0, radj_nadj = 0;
  int n_part = 0;
  int device = 0;
  // staging for qed_eval_host (one call at a time per plan: stage_lock)
  std::mutex stage_lock;
  double* d_stage = nullptr;
  long long stage_cap = 0;    // points per buffer
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_h2d[2] = {nullptr, nullptr}, ev_k[2] = {nullptr, nullptr},
              ev_d2h[2] = {nullptr, nullptr};
};


namespace qed {
KParams make_params(const qed_plan_s* P, const double* mom, long long n, double* out);
qed_status cuda_status(cudaError_t e);
// cudaMalloc behind the library's allocation-failure injection (a host-side
// fake of an out-of-memory device, for tests: qed_debug_inject_alloc_failure).
cudaError_t device_alloc(void** p, size_t bytes);
}  // namespace qed
