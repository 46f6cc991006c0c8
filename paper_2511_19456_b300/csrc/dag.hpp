// Host-side computable-DAG builder for multi-photon Compton |M|^2.
//
// Follows the paper's pipeline (Sec. II-A, Fig. "callstack"): a generator
// emits the complete CDAG of one spin state (one chain per Feynman diagram,
// shared external states, paper Sec. II-B and Table I), an optimiser applies
// node reduction to its fixpoint (App. C: nodes with the same function and the
// same parent set are merged, their children united), and a scheduler
// linearises the reduced DAG into the instruction tables that the CUDA kernels
// execute.  Data nodes carry no work on one device; they are counted but not
// scheduled.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace qed {

enum NodeKind : uint8_t { K_DATA = 0, K_U = 1, K_V = 2, K_S1 = 3, K_S2 = 4, K_SUM = 5 };

struct Counts {
  long long total = 0, data = 0, u = 0, v = 0, s1 = 0, s2 = 0, sum = 0;
};

// Explicit bipartite DAG in creation (= topological) order.
struct Dag {
  std::vector<uint8_t> kind;
  std::vector<int32_t> fn;       // function tag: distinguishes U states, photons of V
  std::vector<int32_t> pbeg;     // CSR offsets into parents (size = nodes + 1)
  std::vector<int32_t> parents;
  int add(NodeKind k, int f, const int32_t* par, int npar);
  int size() const { return (int)kind.size(); }
  Counts counts() const;
};

// Generator: the per-diagram CDAG of one fixed spin state for k outgoing
// photons, with the S2 split after ceil(n/2) photons counted from the
// incoming electron.  photon_of_u[d] gives, for a U node's data node, which
// external slot it belongs to (-1 otherwise).
Dag generate(int k);

// Node reduction to the fixpoint.  Returns the reduced DAG; rep[i] maps each
// node of `in` to its node in the result.
Dag reduce(const Dag& in, std::vector<int32_t>* rep = nullptr);

// Closed-form counts of generate(k) (valid for any k >= 1).
Counts unreduced_counts(int k);

// ------------------------------------------------------- kernel schedule
// One instruction: a vertex (V) optionally followed by a propagation (S1),
// for all spin variants of one current.
//   side 0 (column, from u):  dst = [S(Q_post)] eps/_j src
//   side 1 (row, from ubar):  dst = src eps/_j [S(Q_post)]
// src < 0 means the external spinor of that side.  dst/src are indices of the
// current of spin variant 0; variant v of a current at level l lives at
// index + v (variants: bit 0 = electron helicity, bit 1+r = polarisation of
// the photon of rank r in the current's photon set).
struct Instr {
  int32_t dst;
  int32_t src;
  uint8_t side;
  uint8_t photon;
  uint8_t rank;    // rank of `photon` within the current's photon set
  uint8_t level;   // number of photons in the current
  uint16_t post;   // photon set of the propagator applied after the vertex (0 = none)
  uint16_t pad;
};
static_assert(sizeof(Instr) == 16, "Instr layout");

// A phase is processed completely before the next one starts; it holds up
// to two homogeneous ranges (same level, so same number of spin variants).
struct Phase {
  int32_t beg[2];
  int32_t cnt[2];
  int32_t level[2];
};

struct SetEntry {
  uint32_t mask;     // photon set S to the left of the join line
  int32_t phase0;    // first of this set's phases
  int32_t leaf_l;    // index of the first left leaf (variant 0)
  int32_t leaf_r;    // index of the first right leaf (variant 0)
};

struct Schedule {
  int k = 0, n = 0, h = 0, r = 0;   // photons, left depth, right depth
  int ls = 0, rs = 0;               // levels kept for the whole point
  bool summed = true;
  int n_left_leaves = 0, n_right_leaves = 0;  // h!, r!
  int stored_currents = 0;          // currents kept for the whole point
  int local_currents = 0;           // currents rebuilt per photon set
  int n_stored_phases = 0, n_set_phases = 0;
  std::vector<Instr> instr;
  std::vector<Phase> phases;        // stored phases, then per set its phases
  std::vector<SetEntry> sets;
  // reduced-DAG statistics (one spin state) and spin-variant totals
  Counts unreduced, reduced;
  long long v_nodes = 0, s1_nodes = 0, s2_nodes = 0;  // times spin variants
  long long flops_algorithmic = 0, flops_executed = 0, flops_literal_s2 = 0;
};

int nvar(bool summed, int level);

// ------------------------------------------------ distributive rewrite
// Term rewriting of the reduced DAG (the paper proposes it as a further node
// operation, App. C): the S2 joins of one photon set S share their
// propagator, so by distributivity sum_{a,b} R'_b L_a = (sum_b R'_b)(sum_a L_a);
// applied recursively, the currents of all orderings of a photon subset T
// collapse into one current per subset,
//   J_T = sum_{j in T} eps/_j S(Q_{T \ j}) J_{T \ j}   (column, from u),
// and likewise for row currents from ubar.  A node of the rewritten DAG is a
// subset; it sums one vertex term per photon of the subset and is then
// propagated.  One join per photon set remains.
struct SumInstr {
  int32_t dst;
  int32_t src[4];       // input node of each term (-1: the external spinor)
  uint8_t photon[4];
  uint8_t rank[4];      // rank of the term's photon within the node's set
  uint8_t nterms;
  uint8_t side;
  uint8_t level;
  uint8_t pad0;
  uint16_t post;        // propagator applied to the sum (0 = none)
  uint16_t pad1;
  int32_t pad2[3];
};
static_assert(sizeof(SumInstr) == 48, "SumInstr layout");

struct RwSchedule {
  int k = 0, n = 0, h = 0, r = 0;
  bool summed = true;
  int group = 1;                    // photon sets whose leaves one set phase builds
  int n_groups = 0;
  int stored_currents = 0, local_currents = 0;
  int n_stored_phases = 0, n_set_phases = 0;
  std::vector<SumInstr> instr;
  std::vector<Phase> phases;
  std::vector<SetEntry> sets;
  long long nodes = 0, terms = 0, s1_nodes = 0, joins = 0;   // times spin variants
  long long flops_algorithmic = 0;
};

// group: number of photon sets handled per set phase (their leaves are built
// together, then their joins run without a barrier in between); 0 picks
// rewrite_default_group.
RwSchedule build_rewrite_schedule(int k, bool summed, int group = 0);
// Enough leaf instructions per set phase for about four per thread of a team
// of `team` threads.
int rewrite_default_group(int k, bool summed, int team);

// ------------------------------------------------ node-reduction sweep
// One node reduction (App. C; Sec. III-E): the first group, in topological
// order, of two or more compute nodes with the same function and the same
// parents is merged into one node, together with their output data nodes,
// and the children are rewired.  Returns false at the fixpoint.
bool reduce_step(Dag& g);

// Number of reduction steps from generate(k) to the fixpoint.
int reduction_steps(int k);

// A level-synchronous tape of a DAG (any reduction state) for one fixed spin
// state, executed node by node: every compute node of the DAG does its own
// work, including the propagator of its own momentum.
enum TapeOp : uint8_t { T_SPINOR = 1, T_POL = 2, T_V = 3, T_S1 = 4, T_S2 = 5 };
struct TapeInstr {
  uint8_t op;
  uint8_t side;     // 0: column current (from u), 1: row current (from ubar)
  uint8_t arg;      // T_SPINOR: slot 0 or 2; T_POL, T_V: photon
  uint8_t pad;
  uint16_t mask;    // T_S1, T_S2: photon set of the propagator's momentum
  uint16_t dst;     // value slot (T_S2: diagram index)
  uint16_t src0;    // T_V, T_S1: current; T_S2: left current
  uint16_t src1;    // T_V: polarisation; T_S2: right current
  uint32_t pad2;
};
static_assert(sizeof(TapeInstr) == 16, "TapeInstr layout");

struct Tape {
  int k = 0, n = 0;
  int steps = 0;                   // reductions applied
  int n_slots = 0, n_diag = 0;     // value slots (8 reals each), diagrams
  std::vector<TapeInstr> instr;    // by level
  std::vector<int32_t> level_beg;  // instr range of each level (size levels + 1)
  Counts counts;                   // of the DAG the tape executes
  long long flops = 0;             // per point
};

// The tape of generate(k) after `steps` reduction steps (fewer if the
// fixpoint comes first; Tape::steps says how many).
Tape build_tape(int k, int steps);

// Build the reduced DAG of process k and linearise it.  ls/rs: number of
// left/right levels stored for the whole point (at most h-1 / r-1); deeper
// levels are rebuilt for each photon set.  Throws std::runtime_error when the
// reduced DAG does not have the expected structure.
Schedule build_schedule(int k, bool summed, int ls, int rs);

// FLOP costs of one operation, as the kernels implement it.
constexpr int FLOP_V = 40;      // eps/ times a spinor (real eps, eps^0 = 0)
constexpr int FLOP_S1 = 56;     // (Q/ + m)/D times a spinor, entries pre-scaled
constexpr int FLOP_JOIN = 32;   // 4-component complex dot accumulated into M
constexpr int FLOP_SUBSET = 20; // Q_S, D_S = Q^2 - m^2, 1/D and scaled entries
constexpr int FLOP_SQUARE = 4;  // |M|^2 of one state added to the spin sum
constexpr int FLOP_SPINOR = 30;
constexpr int FLOP_POL = 15;
constexpr int FLOP_SUM = 2;     // one diagram added to M (complex)
// ABC model (scalar currents; the vertex factor g is applied once as g^(2n))
constexpr int FLOP_ABC_SUBSET = 9;  // Q_S^2 - m^2 (4 mul, 4 sub) and 1/D
constexpr int FLOP_ABC_S1 = 1;      // current times 1/D
constexpr int FLOP_ABC_JOIN = 2;    // product of two leaves added to M

}  // namespace qed
