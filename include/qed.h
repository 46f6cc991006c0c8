/*
 * qed.h - C-ABI of the B300 multi-photon Compton |M|^2 engine.
 *
 * Process: e-(p) gamma(k0) -> e-(p') + gamma(k1) ... gamma(kK), tree level,
 * K = k outgoing photons, n = k + 1 photons on the electron line and (k+1)!
 * Feynman diagrams (paper Sec. III-A).  The amplitude of one diagram follows
 * the QED Feynman rules of paper Sec. I-D (Eq. 1 is the k = 1 case):
 *
 *   A_sigma = ubar(p') eps/_{sigma(n)} S(Q_{n-1}) ... S(Q_1) eps/_{sigma(1)} u(p),
 *   S(Q) = (Q/ + m) / (Q^2 - m^2),  Q_i = p + sum_{l<=i} c_l k_{sigma(l)},
 *
 * with c = +1 for the incoming and -1 for outgoing photons; the constant
 * factor (-ie)^n i^(n-1) (unit modulus for e = 1) is dropped, and
 * |M|^2 = sum over the requested spin/polarisation states of |sum_sigma A|^2.
 * The evaluation goes through the node-reduced computable DAG of paper
 * Sec. II (node reduction: App. C), built and linearised on the host by
 * qed_plan_create.
 *
 * Conventions (units m = e = 1 by default): metric (+,-,-,-), Dirac
 * representation, helicity spinors, real linear photon polarisations with
 * eps^0 = 0 in the frame of the given momenta (polarisation 1 = the state
 * eps_1 = (kx kz, ky kz, -kT^2)/(|k| kT), polarisation 2 = (-ky, kx, 0)/kT).
 *
 * Momentum layout: momenta[N][k+3][4] float64, row-major, slot 0 = e- in,
 * 1 = gamma in, 2 = e- out, 3..k+2 = gamma out; components (E, px, py, pz).
 * Propagator momenta are formed from p and the photon momenta of the photons
 * to the left of the line (p' never enters a propagator).
 *
 * Ownership and errors: the caller owns every buffer it passes; a plan owns
 * its device tables, allocated in qed_plan_create and freed by
 * qed_plan_destroy.  Every function returns a qed_status and never throws;
 * arguments are validated before any launch; N = 0 returns QED_OK without a
 * launch.  Non-finite momenta give non-finite outputs and are not errors.
 * qed_eval and qed_eval_grad allocate nothing and do not synchronise the
 * host.  A plan's tables are immutable after creation, and evaluations of
 * one plan may be issued from several host threads and streams at once;
 * the one exception, the plan-owned gradient scratch of spin-summed k = 7 in
 * FP64, is described at qed_eval_grad.
 */
#ifndef QED_H
#define QED_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qed_plan_s* qed_plan_t;
typedef struct qed_batch_s* qed_batch_t;

typedef enum {
  QED_OK = 0,
  QED_EINVAL = 1,          /* invalid argument (NULL, range, misaligned)   */
  QED_ENOMEM = 2,          /* host or device allocation failed             */
  QED_ECUDA = 3,           /* a CUDA runtime call failed                   */
  QED_EUNSUPPORTED = 4,    /* valid request this build does not provide    */
  QED_EDEVICE_TIMEOUT = 5  /* a bounded device-side wait ran out           */
} qed_status;

typedef enum {
  QED_FP64 = 0,   /* every step in FP64                                    */
  QED_MIXED = 1   /* spinors, currents and diagram sums in FP32 with a
                     compensated (Kahan) diagram sum; momenta, propagator
                     denominators and the spin sum in FP64                 */
} qed_precision;

/* Process e- gamma -> e- + k gamma, k in [1, 7].  mass: electron mass
 * (> 0); charge: the coupling e, |M|^2 is multiplied by e^(2(k+1)). */
typedef struct {
  int k;
  double mass;
  double charge;
} qed_process;

/* Spin / polarisation selection.  summed != 0: all 2^(k+3) states summed.
 * Otherwise one fixed state: hel[slot] for slot 0..k+2 with electrons
 * (slots 0, 2) in {+1, -1} (helicity) and photons in {1, 2}
 * (polarisation). */
typedef struct {
  int summed;
  signed char hel[10];
} qed_spin_cfg;

/* Sizes of a plan's DAG and its counted arithmetic. */
typedef struct {
  int k;
  int n_photons;               /* k + 1                                    */
  long long n_diagrams;        /* (k+1)!                                   */
  long long n_states;          /* spin/polarisation states summed (or 1)   */
  long long nodes_unreduced;   /* per-diagram CDAG, data + compute nodes,
                                  one spin state (paper Table I)           */
  long long nodes_reduced;     /* after node reduction to the fixpoint     */
  long long compute_reduced;   /* compute nodes of the reduced DAG         */
  long long v_nodes, s1_nodes, s2_nodes; /* reduced, times spin variants  */
  long long flops_per_point;   /* algorithmic FLOPs of the reduced DAG
                                  (add/sub/mul 1, fma 2, div/sqrt 1)       */
  long long flops_executed_per_point; /* including recomputed currents     */
  long long flops_literal_s2_per_point; /* if every S2 propagated itself  */
  int team_threads;            /* threads cooperating on one point         */
  int smem_bytes_per_team;
  int precision;               /* qed_precision                            */
  int reduction_steps;         /* tape plans: node reductions applied      */
  int kernel_form;             /* forward kernel in use: qed_kernel_form   */
  int kernel_forms;            /* forms this plan has: bit f set for form f */
  int block_threads;           /* launch shape of that kernel: threads per */
  int grid_blocks;             /* block, and blocks of the persistent grid */
} qed_plan_info_t;

/* Forward kernel forms of a plan.  The DAG builder either linearises the
 * DAG into instruction tables or emits a straight-line specialised kernel
 * at build time (the paper's framework generates straight-line code from
 * the scheduled DAG, Sec. II-A; Sec. III-D measures full inlining).
 *   QED_KERNEL_TABLE: one kernel per (k, spin mode, precision) that reads the
 *     plan's linear schedule (instruction, phase and photon-set tables) from
 *     device memory at run time.  Every plan has it.
 *   QED_KERNEL_SPECIALISED: a kernel shaped for the plan's kind.
 *     Spin-summed plans of the node-reduced DAG with k <= 5: generated from
 *     the same schedule when the library is built (csrc/qed_codegen.cpp),
 *     with every instruction expanded into straight-line code whose
 *     photon, polarisation, source, destination and propagator are
 *     literals.  One fixed state, k <= 6 (both precisions): the
 *     register-join kernel (csrc/qed_fix.cu) on the schedule that keeps
 *     every level below the leaves; per photon set each lane of one warp
 *     builds one leaf, keeps a left leaf in registers and joins it with
 *     every right leaf of the set, from per-lane items of two ints.  A new
 *     plan starts in this form, except one fixed state in FP64 with k other
 *     than 3 and 4, where the table-driven kernel measured faster.
 * Both compute the same DAG; their results agree to rounding. */
typedef enum { QED_KERNEL_TABLE = 0, QED_KERNEL_SPECIALISED = 1 } qed_kernel_form;

/* Counts of the CDAG of one spin state, computed on the host without a GPU
 * (paper Table I and Fig. graph_size).  For k <= 7 the DAG is built node by
 * node and node-reduced to its fixpoint (paper App. C); for k = 8 only the
 * unreduced counts are given (from the same per-diagram construction, in
 * closed form) and the reduced fields are -1. */
typedef struct {
  long long unreduced_total, unreduced_data, unreduced_u, unreduced_v,
            unreduced_s1, unreduced_s2, unreduced_sum;
  long long reduced_total, reduced_data, reduced_u, reduced_v,
            reduced_s1, reduced_s2, reduced_sum;
} qed_dag_counts_t;

/* Build the CDAG for a process on the host (paper Sec. II-A: generator,
 * optimiser by node reduction, linear schedule), upload its tables and
 * pick the kernel for `precision`.  Requires a CUDA device for the upload.
 * Errors: QED_EINVAL for NULL pointers, k outside [1, 7], mass <= 0 or a bad
 * fixed state; QED_ENOMEM; QED_ECUDA.  *out is set only on QED_OK. */
qed_status qed_plan_create(const qed_process* process, const qed_spin_cfg* spin,
                           qed_precision precision, qed_plan_t* out);

/* As qed_plan_create, for the distributively rewritten DAG: the term
 * rewriting the paper proposes as a further node operation (App. C). The
 * joins of a photon set S share their propagator, so
 *   sum_{a,b} R'_b L_a = (sum_b R'_b)(sum_a L_a).
 * Applied recursively, this collapses the currents of all orderings of a
 * photon subset T into one current per subset:
 *   J_T = sum_{j in T} eps/_j S(Q_{T\j}) J_{T\j}.
 * The value is the same |M|^2. The cost grows exponentially with the number
 * of photons instead of factorially. qed_eval and qed_plan_info work on such
 * plans. qed_eval_grad and the batched entry points return
 * QED_EUNSUPPORTED. */
qed_status qed_plan_create_rewrite(const qed_process* process, const qed_spin_cfg* spin,
                                   qed_precision precision, qed_plan_t* out);

/* The ABC model (paper App. F and Sec. I-C). It has three scalar particles
 * A, B and C and one vertex joining one of each.
 *
 * Process: A(p) B(k_0) -> A(p') B(k_1) ... B(k_k), with the momenta laid out
 * as for QED (slot 0 = A in, 1 = B in, 2 = A out, 3.. = B out).
 *
 * The B lines attach in all n! = (k+1)! orders to the A/C line, whose
 * species alternates at each attachment: C after an odd number, A after an
 * even number. Hence
 *   |M|^2 = g^(2n) [sum_orders prod_{i<n} 1/(Q_i^2 - m_{s(i)}^2)]^2.
 * For an odd n (even k) no diagram exists.
 *
 * Fields:
 *   k: odd, in {1, 3, 5, 7};
 *   mass_a, mass_c: A and C masses (>= 0);
 *   mass_b: the B mass, which enters only through the caller's momenta;
 *   coupling: g. */
typedef struct {
  int k;
  double mass_a, mass_b, mass_c;
  double coupling;
} qed_abc_process;

/* Plan for the ABC model through the same node-reduced DAG as QED with one
 * spin state (rewrite = 0), or through the rewritten DAG (rewrite != 0),
 * with scalar currents. The kernels are in csrc/abc_kernel.cu.
 *
 * Accepted: qed_eval, qed_eval_host, qed_plan_info, qed_plan_destroy. The
 * FLOPs are those of the scalar DAG.
 * Returns QED_EUNSUPPORTED: qed_eval_grad and the batched entry points.
 * Returns QED_EINVAL: NULL pointers, an even or out-of-range k, a negative or
 * non-finite mass, a non-finite coupling. */
qed_status qed_abc_plan_create(const qed_abc_process* process, qed_precision precision, int rewrite,
                               qed_plan_t* out);

/* The node-reduction sweep (paper Sec. III-D, Fig. f_optimization).
 *
 * qed_reduction_steps: the number of single node reductions that take the
 * per-diagram CDAG of e- gamma -> e- + k gamma (k in 1..6, one spin state)
 * to its fixpoint. One step merges the first group, in topological order, of
 * compute nodes with the same function and the same parents. The group's
 * output data nodes merge with them (App. C).
 *
 * qed_tape_plan_create: a plan that executes, node by node, the CDAG after
 * `reduction_steps` such steps (or after all of them, if the fixpoint comes
 * first). Each compute node does its own work, its own propagator included,
 * so the FLOPs per point are those of the DAG in that state.
 *   - Arguments: k in 1..5, one fixed spin state (spin->summed == 0), FP64.
 *   - Accepted: qed_eval, qed_eval_host, qed_plan_info. qed_plan_info's
 *     nodes_reduced is the node count of that state, and reduction_steps
 *     the steps applied.
 *   - Every state gives the same |M|^2, bit for bit.
 *   - Errors: QED_EINVAL for bad arguments; QED_EUNSUPPORTED when a team's
 *     value slots exceed shared memory. */
qed_status qed_reduction_steps(int k, int* steps);

/* The tape of a reduction state, for inspection and CPU tests.
 *   - Call it with instr == levels == NULL to get the sizes, then with
 *     buffers of n_instr * 16 bytes (TapeInstr in csrc/dag.hpp) and
 *     n_levels + 1 ints.
 *   - Level l runs instructions levels[l] .. levels[l+1]-1.
 *   - Errors: QED_EINVAL for k outside 1..5 or steps < 0. */
typedef struct {
  int k, n, steps, n_slots, n_diag, n_instr, n_levels;
  long long nodes, compute_nodes, flops;
} qed_tape_desc_t;
qed_status qed_tape_export(int k, int steps, qed_tape_desc_t* desc, void* instr, int* levels);
qed_status qed_tape_plan_create(const qed_process* process, const qed_spin_cfg* spin, int reduction_steps,
                                qed_plan_t* out);

/* Sizes and counted arithmetic of a plan: the per-diagram and node-reduced
 * DAG sizes of Table I (Sec. III-A), (k+1)! diagrams, the spin states, the
 * FLOPs per point, and the kernel in use.  The paper prints the sizes; the
 * counting convention (add/sub/mul 1, fma 2) is this library's.
 * QED_EINVAL for NULL arguments. */
qed_status qed_plan_info(qed_plan_t plan, qed_plan_info_t* info);

/* Selects the forward kernel form (qed_kernel_form) that qed_eval,
 * qed_eval_host and qed_cross_section launch.  A new plan starts with the
 * specialised form where it has one (see qed_kernel_form for the exception).  The switch is atomic: an evaluation
 * running on another stream uses one form or the other.
 * Errors: QED_EINVAL (NULL plan, unknown form), QED_EUNSUPPORTED (the plan
 * has no such form).  The paper has no counterpart: its framework emits
 * only generated code. */
qed_status qed_plan_set_kernel_form(qed_plan_t plan, int form);

/* Autotuner of a plan's forward launch: kernel form and block size picked
 * by measurement.  Times every form the plan has
 * with blocks of 32, 64, 128 and 256 threads (those that hold whole teams,
 * that the kernel's launch bounds and the shared memory allow) on the
 * caller's device buffers d_momenta[n][k+3][4] -> d_out_m2[n] (n > 0; the
 * outputs are overwritten), with CUDA events on `stream`, and keeps the
 * fastest.  Returns it in *form, *block and *best_ms (each may be NULL).
 * Synchronous; the plan must not be evaluated from another thread while it
 * is tuned.  Errors: QED_EINVAL (NULL or misaligned buffers, n <= 0),
 * QED_ECUDA.  Not in the paper. */
qed_status qed_plan_tune(qed_plan_t plan, const double* d_momenta, long long n, double* d_out_m2, void* stream,
                         int* form, int* block, double* best_ms);

/* The evaluation of the computable DAG (Sec. II-B: it takes the
 * four-momenta of all particles and returns one real value; tasks U, V, S1,
 * S2 and Sum, the Feynman rules of Sec. I-D) at N phase-space points:
 * out_m2[i] = |M|^2 at point i.  d_momenta: device pointer to N*(k+3)*4
 * doubles, 8-byte aligned; d_out_m2: device pointer to N doubles; stream: a
 * cudaStream_t (NULL = legacy default stream).  Asynchronous.  QED_EINVAL for
 * a NULL or misaligned buffer or N < 0. */
qed_status qed_eval(qed_plan_t plan, const double* d_momenta, long long n,
                    double* d_out_m2, void* stream);

/* Not in the paper (the adjoint of its DAG): as qed_eval, plus
 * d_grad[N][k][3] = d|M|^2 / d(px, py, pz) of the k
 * outgoing photons (slots 3..k+2), their energies on shell, E_j = |k_j|, and
 * every other momentum held fixed.  d_out_m2 may be NULL.  Reverse mode
 * through the same reduced DAG, sub-currents recomputed per photon set;
 * where a team's currents and adjoints do not fit in shared memory
 * (spin-summed k = 7 in FP64), the plan holds a global scratch for them,
 * allocated at creation.  d_out_m2 comes from the adjoint's own forward
 * pass.  It joins each photon set through its leaf sums,
 * (sum_b R'_b).(sum_a L_a), except for one fixed state in mixed precision,
 * which keeps the per-diagram joins.  It equals qed_eval's result up to
 * rounding.  QED_EUNSUPPORTED for rewrite, ABC and tape plans.
 *
 * Plans whose adjoint uses the global scratch (qed_grad_workspace_bytes
 * reports more than 0): the launches of qed_eval_grad on such a plan run one
 * after another on the device whatever their streams, each waiting for the
 * previous one (an event the plan records; no host synchronisation).  Inside
 * a stream capture no such wait is added, and a graph so captured must not
 * run at the same time as another use of the plan's scratch.  For
 * concurrent gradients on one plan, give each caller its own workspace
 * through qed_eval_grad_ws. */
qed_status qed_eval_grad(qed_plan_t plan, const double* d_momenta, long long n,
                         double* d_out_m2, double* d_grad, void* stream);

/* Bytes of device workspace that qed_eval_grad_ws needs for this plan's
 * adjoint: the currents and adjoints of every resident team when they do
 * not fit in shared memory (spin-summed k = 7 in FP64), else 0.
 * QED_EUNSUPPORTED for plans without an adjoint.  Not in the paper. */
qed_status qed_grad_workspace_bytes(qed_plan_t plan, long long* bytes);

/* As qed_eval_grad with the scratch in a caller-owned device buffer
 * d_workspace of workspace_bytes bytes (256-byte aligned; at least
 * qed_grad_workspace_bytes, and ignored, may be NULL, when that is 0).
 * Calls with different workspaces may run concurrently on any streams;
 * calls that share one race.  QED_EINVAL for a missing, short or misaligned
 * workspace.  Not in the paper. */
qed_status qed_eval_grad_ws(qed_plan_t plan, const double* d_momenta, long long n, double* d_out_m2,
                            double* d_grad, void* d_workspace, long long workspace_bytes, void* stream);

/* Not in the paper.  End-to-end form of qed_eval on HOST buffers: copies the momenta to the
 * device, evaluates and copies |M|^2 back, chunked so that copies overlap
 * the kernels (the chunks grow from an eighth of the largest, max(65536,
 * n/8) points, so that only a small first copy runs before a kernel).  Uses device staging owned by the plan, grown (allocated) on
 * the first call that needs more; synchronises `stream` before returning.
 * Calls on one plan from several host threads run one at a time (the
 * staging is the plan's); no copy outlives the call, also on error.
 * Host buffers should be page-locked for full copy bandwidth. */
qed_status qed_eval_host(qed_plan_t plan, const double* h_momenta, long long n,
                         double* h_out_m2, void* stream);

/* Frees a plan and everything it owns (NULL: no-op). */
void qed_plan_destroy(qed_plan_t plan);

/* Not in the paper.
 * Batched evaluation of n_req requests of different k in ONE persistent
 * launch (spin-summed plans, k <= 5, all of the same precision).  The host
 * cuts request r's n_points[r] points into work items of about equal
 * arithmetic, most expensive k first; persistent CTAs take items from a
 * device counter, which never makes one CTA wait for another.  The counter
 * reset and the launch are captured once in a CUDA graph.  Kernel forms as
 * for a plan (qed_kernel_form): QED_KERNEL_TABLE runs the table-driven point
 * evaluation of every k, QED_KERNEL_SPECIALISED (a new batch's form) the
 * straight-line specialised one of every k.  The batch keeps the plans (they must outlive it), allocates its
 * item list, request table and counter, and is not safe for concurrent use
 * from two streams.
 * Errors: QED_EINVAL (NULL, n < 0, mixed precisions), QED_EUNSUPPORTED
 * (fixed spin, k > 5), QED_ENOMEM, QED_ECUDA. */
qed_status qed_batch_create(const qed_plan_t* plans, int n_req, const long long* n_points,
                            qed_batch_t* out);

/* Not in the paper.  Evaluates every request: d_momenta[r] -> d_out[r] (device pointers, sizes
 * as given at creation).  Copies the request table (pointers) and replays the
 * graph on `stream`; asynchronous. */
qed_status qed_batch_eval(qed_batch_t batch, const double* const* d_momenta, double* const* d_out,
                          void* stream);

/* Not in the paper.  Autotuner: times kernel forms {table, specialised} x block sizes
 * {64, 128, 256} x item sizes {1e8, 4e8, 1.6e9 FLOPs} on the given buffers,
 * keeps the fastest, rebuilds the graph and returns its time per evaluation
 * in *best_ms (may be NULL).  Synchronous. */
qed_status qed_batch_tune(qed_batch_t batch, const double* const* d_momenta, double* const* d_out,
                          void* stream, double* best_ms);

/* Not in the paper.  Current launch shape of a batch. */
qed_status qed_batch_info(qed_batch_t batch, int* block, double* work_target, long long* n_items);

/* Not in the paper.  Selects the batch's kernel form (qed_kernel_form) and
 * rebuilds its graph; synchronous.  Errors: QED_EINVAL (NULL batch,
 * unknown form), QED_EUNSUPPORTED / QED_ECUDA from the rebuild (the old form
 * is kept). */
qed_status qed_batch_set_kernel_form(qed_batch_t batch, int form);

/* Not in the paper.  The batch's kernel form in *form.  QED_EINVAL for NULL. */
qed_status qed_batch_kernel_form(qed_batch_t batch, int* form);

/* Frees a batch (not its plans; NULL: no-op). */
void qed_batch_destroy(qed_batch_t batch);

/* Allocation-free batched evaluation.  The paper has no counterpart; this
 * entry point serves callers that cannot allocate device memory when they
 * evaluate:
 *   - applications whose memory pool owns the device and forbids foreign
 *     cudaMalloc calls;
 *   - latency-critical loops that cannot afford the synchronisation a
 *     cudaMalloc/cudaFree implies.
 *
 * Behaviour:
 *   - It runs the same persistent kernel as qed_batch_eval in a new batch's
 *     form (QED_KERNEL_SPECIALISED), with 128-thread blocks, on the same
 *     kinds of request: spin-summed plans, k <= 5, all of one precision.
 *   - The counter, request table and work items live in a static device
 *     array of about 1.53 MiB, which every GPU that loads the library holds
 *     until the process exits.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine. The
 *     caller owns every input and output buffer.
 *   - At most 256 requests; more return QED_EINVAL. Work items are made
 *     larger until they fit the static table (65,536 items).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing). The first call on a
 *     device may load the library's device code: make it before any stream
 *     capture on that device.
 *   - Every call shares the array and leaves its contents behind. The
 *     counter is cleared on `stream` before each launch. Calls that overlap
 *     on the GPU, on any stream, race with each other.
 *   - Asynchronous on `stream`. */
qed_status qed_batch_eval_static(const qed_plan_t* plans, int n_req, const long long* n_points,
                                 const double* const* d_momenta, double* const* d_out, void* stream);

qed_status qed_dag_counts(int k, qed_dag_counts_t* out);

/* Device-side phase-space points, the step before the |M|^2 path of a Monte
 * Carlo event generator (the paper motivates the method by Monte Carlo
 * sampling, Sec. I-C and III-E).  Writes points offset .. offset+n-1 of the seeded
 * stream into d_momenta[n][k+3][4] (layout as above), with the same recipe
 * and counter-based SplitMix64 draws as the host generator:
 *   - k = 1: flat two-body, uniform in the CM solid angle;
 *   - k >= 2: RAMBO (Kleiss, Stirling, Ellis 1986) with the electron
 *     massive.
 * The lab frame has e- at rest and the photon along +z with energy omega.
 * d_weight[n] (may be NULL) receives the phase-space weight:
 *   - the measure is (2 pi)^4 delta^4 prod d^3p / ((2 pi)^3 2E);
 *   - massless RAMBO weight times the massive correction factor.
 * Errors: QED_EINVAL (k outside [1,7], omega or mass <= 0, offset or
 * n < 0, NULL or misaligned buffers).  Asynchronous. */
qed_status qed_generate(int k, double omega, double mass, unsigned long long seed, long long offset,
                        long long n, double* d_momenta, double* d_weight, void* stream);

/* Monte Carlo estimate of the total cross section
 *   sigma = 1/(4 m omega) * 1/4 * 1/k! * <w * sum|M|^2>
 * for a spin-summed plan. The factors are the flux of an e- at rest, the
 * average over the initial helicity and polarisation states, and the
 * identical outgoing photons.
 * Procedure: generate points offset .. offset+n-1 of stream `seed`, in
 * chunks of `chunk` points, evaluate each chunk, and accumulate
 * sum(w |M|^2) and sum((w |M|^2)^2) on the device in d_acc[2].
 * Caller-owned device buffers:
 *   - d_momenta[chunk][k+3][4];
 *   - d_weight[chunk];
 *   - d_m2[chunk];
 *   - d_acc[2].
 * Outputs: sigma, its standard error sigma_err and the two raw sums (any of
 * them may be NULL). Partial sums from several ranks combine by adding the
 * raw sums. Synchronises `stream`. */
qed_status qed_cross_section(qed_plan_t plan, double omega, unsigned long long seed, long long offset,
                             long long n, long long chunk, double* d_momenta, double* d_weight,
                             double* d_m2, double* d_acc, void* stream, double* sigma, double* sigma_err,
                             double* sum_wm2, double* sum_wm2_sq);

/* Test hook (failure detection without a device fault). Once `after` more
 * device allocations of the library have succeeded, the next one fails as
 * if the device were out of memory. The call that made it then returns
 * QED_ENOMEM and frees what it had allocated. -1 switches the hook off.
 * QED_EINVAL if after < -1. The paper has no counterpart. */
qed_status qed_debug_inject_alloc_failure(int after);

/* A static English description of a status code. */
const char* qed_status_string(qed_status status);

/* Measured FMA-pipe peak of the current device in TFLOP/s: FP64 for
 * QED_FP64 (about 0.3 s of chains per launch), FP32 for QED_MIXED (the
 * larger of scalar and packed two-per-instruction FMA chains, the form of
 * the mixed joins).  Independent chains on every SM, timed with CUDA events
 * on `stream`; allocates a small scratch buffer; synchronises.  The |M|^2
 * kernels are bound by this pipe, so it is their roofline denominator.
 * Not in the paper. */
qed_status qed_measure_fma_peak(qed_precision precision, double* tflops, void* stream);

/* The static schedule of Sec. II-A (the scheduler's topological order,
 * here grouped into phases and photon sets): the linear schedule of the
 * node-reduced DAG, as the kernels execute it: V (+S1)
 * instructions (16 bytes each), phases (24 bytes) and photon-set entries (16
 * bytes); layouts in csrc/dag.hpp.  Host only, no GPU needed.  Call with NULL
 * buffers to get the sizes in *desc, then with buffers of those sizes. */
typedef struct {
  int k, n, h, r, ls, rs, summed;
  int n_left_leaves, n_right_leaves, stored_currents, local_currents;
  int n_stored_phases, n_set_phases, n_sets, n_instr, n_phases;
  long long flops_algorithmic, flops_executed;
} qed_schedule_desc_t;

qed_status qed_schedule_export(int k, int summed, qed_schedule_desc_t* desc, void* instr,
                               void* phases, void* sets);

/* The same for the rewritten DAG. Instructions are 48 bytes (SumInstr in
 * csrc/dag.hpp: one node summing up to 4 vertex terms). group is the number of
 * photon sets whose leaves one set phase builds; 0 picks the default. Each set
 * entry's phase0 names its group's phase. Returns QED_EINVAL when k is
 * outside 1..7 or group < 0. */
qed_status qed_rewrite_schedule_export(int k, int summed, int group, qed_schedule_desc_t* desc,
                                       void* instr, void* phases, void* sets);

#ifdef __cplusplus
}
#endif
#endif /* QED_H */
