// Build-time code generator: the straight-line specialised forward kernels.
//
// The paper's framework compiles the scheduled CDAG into one function of
// straight-line code, every task inlined (Sec. II-A, the code generation
// step; Sec. III-D measures full inlining against calls).  This program does
// the same for the spin-summed plans of k = 1..5: it builds the node-reduced
// DAG and its linear schedule (dag.cpp: generate, reduce, build_schedule) and
// writes one CUDA kernel per k and precision in which every instruction of the
// schedule is expanded into the items of one round of the team's lanes, with
// the instruction's photon, polarisation rank, source, destination and
// propagator as literals.  The table-driven kernels (qed_fwd.cu) read the same
// schedule from device tables at run time; both compute the same DAG.
//
// Usage: qed_codegen OUT.cu   (writes OUT.cu only when its content changes)
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <fstream>
#include <iterator>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "dag.hpp"
#include "qed_types.h"

using namespace qed;

namespace {

// Version of the generated kernels (layout, rounds, joins); part of the
// benchmark's record of which kernel a counter capture belongs to.
constexpr const char* SPEC_VERSION = "spec-6";

// One vertex (+ propagation) node of a range.  photon, src and post are C++
// expressions: literals for the kept currents, entries of the photon set's
// constant table inside the loop over photon sets.  rank is always a literal
// (the same for every set at a given position); dst is a literal index.
struct Item {
  std::string photon, src, post;
  bool spinor;      // the input is the external spinor (level 1)
  int rank, dst;
  int photon_i, src_i;   // numeric values (kept currents), for sorting and renumbering
  int leaf_base = -1, leaf_pos = -1;   // leaves: buffer and position, if not the range's own
};

bool is_int(const std::string& e) {
  if (e.empty()) return false;
  for (size_t i = 0; i < e.size(); ++i)
    if (!(std::isdigit((unsigned char)e[i]) || (i == 0 && e[i] == '-'))) return false;
  return true;
}

// One expression per lane group g of a round: the common expression when
// every group has the same, an affine form of g for literals in arithmetic
// progression, else a selection on g.
std::string per_group(const std::vector<std::string>& v) {
  const size_t G = v.size();
  bool same = true;
  for (size_t i = 1; i < G; ++i) same = same && v[i] == v[0];
  if (same) return v[0];
  bool ints = true;
  for (const std::string& e : v) ints = ints && is_int(e);
  if (ints) {
    const int d = std::stoi(v[1]) - std::stoi(v[0]);
    bool affine = true;
    for (size_t i = 2; i < G; ++i) affine = affine && std::stoi(v[i]) - std::stoi(v[i - 1]) == d;
    if (affine) return "(" + v[0] + " + " + std::to_string(d) + " * g)";
  }
  std::string s;
  for (size_t i = 0; i + 1 < G; ++i) s += "g == " + std::to_string(i) + " ? " + v[i] + " : ";
  return "(" + s + v[G - 1] + ")";
}
std::string per_group(const std::vector<int>& v) {
  std::vector<std::string> e;
  for (int x : v) e.push_back(std::to_string(x));
  return per_group(e);
}

struct Emitter {
  std::ostringstream o;
  int team = 0;
  const char* real = "float";
  std::string indent = "  ";

  // The code of every round of a range, one string each.
  std::vector<std::string> rounds(const std::vector<Item>& items, int side, int level, bool post, bool planar,
                                  int leaf_base, int np, const char* what) {
    std::ostringstream saved;
    saved << o.str();
    std::vector<std::string> out;
    const int nv = 1 << (level + 1), lg = level + 1;
    const int cnt = (int)items.size();
    auto one = [&](const std::vector<int>& nodes, int v_off) {
      o.str("");
      o << indent << "// " << what << "\n";
      emit_round(items, nodes, side, post, planar, leaf_base, np, nv, lg, v_off);
      out.push_back(o.str());
    };
    if (nv >= team) {
      for (int i = 0; i < cnt; ++i)
        for (int t = 0; t < nv / team; ++t) one({i}, t * team);
    } else {
      const int G = team / nv;
      for (int t = 0; t * G < cnt; ++t) {
        std::vector<int> nodes;
        for (int g = 0; g < G && t * G + g < cnt; ++g) nodes.push_back(t * G + g);
        one(nodes, -1);
      }
    }
    o.str("");
    o << saved.str();
    return out;
  }

  // The rounds of one range of instructions (one level, one side).  planar:
  // the destinations are leaves (position = index in the list) in the chunk
  // layout at leaf_base with np polarisation patterns; otherwise natural
  // currents at items[i].dst.
  void range(const std::vector<Item>& items, int side, int level, bool post, bool planar, int leaf_base,
             int np, const char* what) {
    const int nv = 1 << (level + 1), lg = level + 1;
    const int cnt = (int)items.size();
    if (cnt == 0) return;
    o << "  // " << what << ": " << cnt << " node(s) x " << nv << " spin variants\n";
    if (nv >= team) {
      for (int i = 0; i < cnt; ++i)
        for (int t = 0; t < nv / team; ++t) emit_round(items, {i}, side, post, planar, leaf_base, np, nv, lg, t * team);
    } else {
      const int G = team / nv;
      for (int t = 0; t * G < cnt; ++t) {
        std::vector<int> nodes;
        for (int g = 0; g < G && t * G + g < cnt; ++g) nodes.push_back(t * G + g);
        emit_round(items, nodes, side, post, planar, leaf_base, np, nv, lg, -1);
      }
    }
  }

  void emit_round(const std::vector<Item>& items, const std::vector<int>& nodes, int side, bool post,
                  bool planar, int leaf_base, int np, int nv, int lg, int v_off) {
    const int G = (int)nodes.size();
    const bool grouped = v_off < 0;
    const int G_full = grouped ? team / nv : 1;
    std::vector<std::string> photon, src, pst;
    std::vector<int> rank, dst;
    for (int i : nodes) {
      photon.push_back(items[i].photon);
      rank.push_back(items[i].rank);
      src.push_back(items[i].src);
      pst.push_back(items[i].post);
      // planar: the offset (in reals) of the leaf's chunk (q = 0, s = 0, p = 0)
      const int lb = items[i].leaf_base >= 0 ? items[i].leaf_base : leaf_base;
      const int lp = items[i].leaf_pos >= 0 ? items[i].leaf_pos : i;
      dst.push_back(planar ? lb * 8 + lp * 16 * np : items[i].dst);
      if (items[i].spinor != items[nodes[0]].spinor)
        throw std::runtime_error("spinor and current inputs in one round");
    }
    o << indent << "{\n";
    std::string ind = indent + "  ";
    if (grouped && G_full > 1) o << ind << "const int g = lane >> " << lg << ";\n";
    if (grouped && G < G_full) {
      o << ind << "if (g < " << G << ") {\n";
      ind += "  ";
    }
    if (grouped) o << ind << "const int v = lane & " << (nv - 1) << ";\n";
    else o << ind << "const int v = lane + " << v_off << ";\n";
    const std::string rk = per_group(rank);
    const bool rank_lit = is_int(rk);
    if (rank_lit) {
      o << ind << "const int vp = spec::drop_pol_bit<" << rk << ">(v);\n";
      o << ind << "const int pol = (v >> " << (1 + rank[0]) << ") & 1;\n";
    } else {
      o << ind << "const int rk = " << rk << ";\n";
      o << ind << "const int vp = (v & ((2 << rk) - 1)) | ((v >> (rk + 2)) << (rk + 1));\n";
      o << ind << "const int pol = (v >> (1 + rk)) & 1;\n";
    }
    if (items[nodes[0]].spinor)
      o << ind << "const " << real << "* xs = s_spin + (" << side * 2 << " + vp) * 8;\n";
    else
      o << ind << "const " << real << "* xs = s_cur + (" << per_group(src) << " + vp) * 8;\n";
    o << ind << "const " << real << "* e = s_eps + (" << per_group(photon) << " * 2 + pol) * 4;\n";
    if (post) o << ind << "const " << real << "* P = s_q + " << per_group(pst) << " * 5;\n";
    else o << ind << "const " << real << "* P = nullptr;\n";
    if (planar) {
      o << ind << real << "* d0 = s_cur + " << per_group(dst) << " + ((v & 1) * " << np << " + (v >> 1)) * 4;\n";
      o << ind << real << "* d1 = d0 + " << 2 * np * 4 << ";\n";
    } else {
      o << ind << real << "* d0 = s_cur + (" << per_group(dst) << " + v) * 8;\n";
      o << ind << real << "* d1 = d0 + 4;\n";
    }
    o << ind << "spec::vs_item<" << real << ", " << side << ", " << (post ? "true" : "false")
      << ">(xs, e, P, d0, d1);\n";
    if (grouped && G < G_full) o << indent << "  }\n";
    o << indent << "}\n";
  }
};

int blocks_by_smem(int block_bytes) {
  // 228 KB of shared memory per SM, 1 KB of it reserved per resident block
  const int sm = 228 * 1024;
  return sm / (block_bytes + 1024);
}

struct KernelDesc {
  std::string name;
  int k, mixed, team, ncur, team_bytes, block, min_blocks;
};

// One specialised kernel: spin-summed, k photons out, FP32-mixed or FP64.
KernelDesc emit_kernel(std::ostringstream& out, int k, bool mixed) {
  const int n = k + 1, h = (n + 1) / 2, r = n - h;
  const Schedule sc = build_schedule(k, true, h - 1, r - 1);
  const int team = 1 << n;
  const int NL = sc.n_left_leaves, NR = sc.n_right_leaves;
  const int ncur = sc.stored_currents + sc.local_currents;
  if (sc.local_currents != NL * (1 << (h + 1)) + NR * (1 << (r + 1)))
    throw std::runtime_error("a photon set's local currents are not just its leaves");
  const int NPL = 1 << h, NPR = 1 << r;
  if (sc.n_set_phases != 1) throw std::runtime_error("expected one phase per photon set");
  const TeamLayout L = team_layout(k, mixed ? 4 : 8, ncur);
  const int real_size = mixed ? 4 : 8;
  KernelDesc kd;
  kd.k = k;
  kd.mixed = mixed;
  kd.team = team;
  kd.ncur = ncur;
  kd.team_bytes = L.bytes;
  kd.block = team > 128 ? team : 128;
  // resident blocks to compile for: as many as shared memory allows, but
  // never fewer than 96 registers per thread in FP32 (the joins hold a block
  // of right leaves, a left leaf and 16 accumulators in registers) or 160 in
  // FP64
  const int min_regs = mixed ? 96 : 160;
  kd.min_blocks = std::max(1, std::min(65536 / (kd.block * min_regs), blocks_by_smem((kd.block / team) * L.bytes)));
  kd.name = "qed_spec_fwd_k" + std::to_string(k) + (mixed ? "_f32" : "_f64");

  Emitter em;
  em.team = team;
  em.real = mixed ? "float" : "double";
  const char* R = em.real;
  std::ostringstream& o = em.o;

  // node order inside a range: by rank and photon, so that a round of lane
  // groups shares them; stored currents are renumbered accordingly and their
  // consumers follow the new numbers
  std::vector<int> remap(ncur, -1);
  auto sorted_items = [&](const Phase& ph, int slot, bool renumber) {
    std::vector<Item> v;
    for (int i = 0; i < ph.cnt[slot]; ++i) {
      const Instr& in = sc.instr[ph.beg[slot] + i];
      Item it;
      it.photon_i = in.photon;
      it.rank = in.rank;
      it.spinor = in.src < 0;
      it.src_i = in.src < 0 ? -1 : remap.at(in.src);
      if (in.src >= 0 && it.src_i < 0) throw std::runtime_error("source before its producer");
      it.post = std::to_string(in.post);
      it.dst = in.dst;
      v.push_back(it);
    }
    std::stable_sort(v.begin(), v.end(), [](const Item& a, const Item& b) {
      if (a.rank != b.rank) return a.rank < b.rank;
      if (a.photon_i != b.photon_i) return a.photon_i < b.photon_i;
      return a.src_i < b.src_i;
    });
    if (renumber) {
      const int nv = nvar(true, ph.level[slot]);
      int base = v[0].dst;
      for (const Item& it : v) base = std::min(base, it.dst);
      for (size_t i = 0; i < v.size(); ++i) {
        const int nd = base + (int)i * nv;
        for (int q = 0; q < nv; ++q) remap.at(v[i].dst + q) = nd + q;
        v[i].dst = nd;
      }
    }
    for (Item& it : v) {
      it.photon = std::to_string(it.photon_i);
      it.src = std::to_string(it.src_i);
    }
    return v;
  };
  auto side_of = [&](const Phase& ph, int slot) { return (int)sc.instr[ph.beg[slot]].side; };
  auto post_of = [&](const Phase& ph, int slot) { return sc.instr[ph.beg[slot]].post != 0; };

  o << "// e- gamma -> e- + " << k << " gamma, " << (k + 1) << "! = " << sc.n_left_leaves * sc.n_right_leaves * (int)sc.sets.size()
    << " diagrams, all " << (1 << (n + 2)) << " spin states summed, " << (mixed ? "FP32-mixed" : "FP64")
    << ".\n// Team of " << team << " lanes (lane c = polarisation pattern c, 4 electron-helicity states each); "
    << ncur << " currents, " << L.bytes << " bytes of shared memory per team.\n";

  // the kept currents first: their renumbering fixes the sources the photon
  // sets read
  struct StoredRange { int phase, side, level; bool post; std::vector<Item> items; };
  std::vector<StoredRange> stored;
  for (int ph = 0; ph < sc.n_stored_phases; ++ph) {
    const Phase& P = sc.phases[ph];
    for (int slot = 0; slot < 2; ++slot) {
      if (P.cnt[slot] == 0) continue;
      stored.push_back(StoredRange{ph, side_of(P, slot), P.level[slot], post_of(P, slot), sorted_items(P, slot, true)});
    }
  }

  // ---- the photon sets: their leaf ranges must have one shape (ranks per
  // position, spinor inputs) so that one loop body serves every set; the
  // photons and sources per position go to a constant table
  const Phase& P0 = sc.phases[sc.sets[0].phase0];
  int lslot = -1, rslot = -1;
  for (int slot = 0; slot < 2; ++slot)
    if (P0.cnt[slot]) (side_of(P0, slot) == 0 ? lslot : rslot) = slot;
  if (lslot < 0 || rslot < 0) throw std::runtime_error("a photon set without left or right leaves");
  std::vector<std::vector<Item>> lsets, rsets;
  const std::string tab = "c_sets_" + kd.name.substr(std::string("qed_spec_fwd_").size());
  std::ostringstream t;
  t << "__constant__ spec::SetTable<" << NL << ", " << NR << "> " << tab << "[" << sc.sets.size() << "] = {\n";
  for (size_t s = 0; s < sc.sets.size(); ++s) {
    const SetEntry& se = sc.sets[s];
    const Phase& P = sc.phases[se.phase0];
    if (side_of(P, lslot) != 0 || side_of(P, rslot) != 1) throw std::runtime_error("set phase layout differs");
    lsets.push_back(sorted_items(P, lslot, false));
    rsets.push_back(sorted_items(P, rslot, false));
    if ((int)lsets.back().size() != NL || (int)rsets.back().size() != NR) throw std::runtime_error("leaf count");
    for (int side = 0; side < 2; ++side) {
      const auto& a = side == 0 ? lsets.back() : rsets.back();
      const auto& b = side == 0 ? lsets[0] : rsets[0];
      for (size_t i = 0; i < a.size(); ++i)
        if (a[i].rank != b[i].rank || a[i].spinor != b[i].spinor)
          throw std::runtime_error("photon sets of different shape");
    }
    const unsigned C = ((1u << n) - 1) & ~se.mask;
    t << "  {" << se.mask << ", " << C << ", {";
    for (int i = 0; i < NL; ++i) t << (i ? ", " : "") << lsets.back()[i].photon_i;
    t << "}, {";
    for (int i = 0; i < NL; ++i) t << (i ? ", " : "") << lsets.back()[i].src_i;
    t << "}, {";
    for (int i = 0; i < NR; ++i) t << (i ? ", " : "") << rsets.back()[i].photon_i;
    t << "}, {";
    for (int i = 0; i < NR; ++i) t << (i ? ", " : "") << rsets.back()[i].src_i;
    t << "}},\n";
  }
  t << "};\n\n";
  o << t.str();

  o << "__device__ __forceinline__ void " << kd.name << "_point(const KParams& p, int lane, long long pt, bool valid,\n"
    << "    unsigned char* base) {\n";
  o << "  constexpr int K = " << k << ", TEAM = " << team << ";\n";
  o << "  const TeamLayout L = team_layout(K, " << real_size << ", " << ncur << ");\n";
  o << "  double* s_mom = reinterpret_cast<double*>(base + L.mom);\n";
  o << "  " << R << "* s_q = reinterpret_cast<" << R << "*>(base + L.q);\n";
  o << "  " << R << "* s_eps = reinterpret_cast<" << R << "*>(base + L.eps);\n";
  o << "  " << R << "* s_spin = reinterpret_cast<" << R << "*>(base + L.spin);\n";
  o << "  double* s_red = reinterpret_cast<double*>(base + L.red);\n";
  o << "  " << R << "* s_cur = reinterpret_cast<" << R << "*>(base + L.cur);\n";
  // the FP64-light mixed set-up takes at most two photons per denominator
  // (n <= 5); otherwise, and in FP64, the table kernels' set-up
  if (mixed && n / 2 <= 2)
    o << "  spec::setup_f32<K, TEAM>(p, lane, pt, s_mom, s_q, s_eps, s_spin,\n"
      << "      reinterpret_cast<double*>(base + L.w), reinterpret_cast<float*>(base + L.momf));\n";
  else
    o << "  point_setup<K, " << R << ", TEAM>(p, lane, pt, s_mom, s_q, s_eps, s_spin,\n"
      << "      reinterpret_cast<double*>(base + L.w), reinterpret_cast<float*>(base + L.momf));\n";
  o << "  Acc<" << R << "> acc[4];\n";
  for (int ph = 0; ph < sc.n_stored_phases; ++ph) {
    o << "  // ---- kept currents, phase " << ph << "\n";
    for (const StoredRange& sr : stored)
      if (sr.phase == ph)
        em.range(sr.items, sr.side, sr.level, sr.post, false, 0, 0,
                 sr.side == 0 ? "column currents" : "row currents");
    o << "  team_sync<TEAM>();\n";
  }
  // The loop over the photon sets: position i of a set's leaf lists takes
  // its photon and source from the set's row of the constant table.  (One
  // loop body instead of one copy per set: fully unrolled, the k = 4 kernel
  // was 7.6 K instructions per point but stalled on instruction fetch.)
  //
  // Where one set's right leaves fill at most half a round, the loop takes
  // the sets in pairs and builds both sets' right leaves in one round, the
  // second set's into the currents of the first kept level, which nothing
  // reads once the second level is built (k = 4: ten sets, 16 right leaf
  // variants each on 32 lanes).
  const int nsets = (int)sc.sets.size();
  const int leaf_l = sc.stored_currents, leaf_r = sc.stored_currents + NL * (1 << (h + 1));
  const int nvr = 1 << (r + 1);
  int dead_base = -1, dead_size = 0;   // the first left level, once the second is built
  if (sc.ls >= 2)
    for (const StoredRange& sr : stored)
      if (sr.side == 0 && sr.level == 1) {
        dead_base = sr.items[0].dst;
        for (const Item& it : sr.items) dead_base = std::min(dead_base, it.dst);
        dead_size = (int)sr.items.size() * (1 << 2);
      }
  const bool paired = 2 * NR * nvr <= team && nsets % 2 == 0 && dead_base >= 0 && dead_size >= NR * nvr;
  auto left_body = [&](const std::string& t) {
    std::vector<Item> v = lsets[0];
    for (int i = 0; i < NL; ++i) {
      v[i].photon = t + ".lph[" + std::to_string(i) + "]";
      v[i].src = t + ".lsrc[" + std::to_string(i) + "]";
      v[i].post = "0";
    }
    return v;
  };
  auto right_body = [&](const std::string& t, int base) {
    std::vector<Item> v = rsets[0];
    for (int i = 0; i < NR; ++i) {
      v[i].photon = t + ".rph[" + std::to_string(i) + "]";
      v[i].src = t + ".rsrc[" + std::to_string(i) + "]";
      v[i].post = t + ".mask";
      v[i].leaf_base = base;
      v[i].leaf_pos = i;
    }
    return v;
  };
  auto emit_rounds = [&](const std::vector<std::string>& rs) { for (const std::string& x : rs) o << x; };
  // right leaves per block of the FP32 joins: all of them up to two (k <= 4),
  // else two at a time (k = 5: six right leaves; 64 registers a block)
  const int BB = NR <= 2 ? NR : 2;
  if (NR % BB != 0) throw std::runtime_error("right leaves not in whole blocks");
  // rbase < 0: the right leaves of an even set at leaf_r, of an odd one at
  // dead_base (sets in pairs)
  auto join = [&](const std::string& set_index, int rbase) {
    o << "    {\n";
    o << "      const unsigned tv = __ldg(p.lane_tab + ((" << set_index << ") << " << n
      << ") + lane);   // pext(lane, S) | pext(lane, ~S) << 8\n";
    o << "      const int pl = (int)(tv & 0xffu), pr = (int)(tv >> 8);\n";
    const std::string rb = rbase >= 0 ? std::to_string(rbase * 8)
                                      : "((" + set_index + ") & 1 ? " + std::to_string(dead_base * 8) + " : " +
                                            std::to_string(leaf_r * 8) + ")";
    if (mixed)
      o << "      spec::join_set_f32<" << NL << ", " << NR << ", " << NPL << ", " << NPR << ", " << BB
        << ">(reinterpret_cast<const float4*>(s_cur + " << leaf_l * 8 << ") + pl,\n"
        << "          reinterpret_cast<const float4*>(s_cur + " << rb << ") + pr, acc);\n";
    else
      o << "      spec::join_set_f64<" << NL << ", " << NR << ", " << NPL << ", " << NPR << ">(s_cur + " << leaf_l * 8
        << " + pl * 4, s_cur + " << rb << " + pr * 4, acc);\n";
    o << "    }\n";
    o << "    team_sync<TEAM>();\n";
  };
  const std::string TT = "spec::SetTable<" + std::to_string(NL) + ", " + std::to_string(NR) + ">";
  o << "  // ---- the " << nsets << " photon sets S (|S| = " << h << "): leaves, then the joins of "
    << NL * NR << " diagrams x 4 states per lane" << (paired ? "; sets in pairs" : "") << "\n";
  o << "#pragma unroll 1\n";
  em.indent = "    ";
  if (!paired) {
    o << "  for (int s = 0; s < " << nsets << "; ++s) {\n";
    o << "    const " << TT << "& cs = " << tab << "[s];\n";
    std::vector<Item> lv = left_body("cs"), rv = right_body("cs", leaf_r);
    // a team of two warps (k = 5): where each side's last round fills at
    // most one warp, the first warp takes the left tail and the second the
    // right tail in one round (warp-uniform branches) instead of two half
    // rounds
    const int nvl = 1 << (h + 1);
    const int tl = nvl < team ? NL % (team / nvl) : 0, tr = nvr < team ? NR % (team / nvr) : 0;
    const bool split = team == 64 && tl > 0 && tr > 0 && tl * nvl <= 32 && tr * nvr <= 32;
    std::vector<Item> ltail, rtail;
    if (split) {
      for (int i = NL - tl; i < NL; ++i) {
        ltail.push_back(lv[i]);
        ltail.back().leaf_base = leaf_l;
        ltail.back().leaf_pos = i;
      }
      for (int i = NR - tr; i < NR; ++i) rtail.push_back(rv[i]);   // leaf_base, leaf_pos set
      lv.resize(NL - tl);
      rv.resize(NR - tr);
    }
    emit_rounds(em.rounds(lv, 0, h, false, true, leaf_l, NPL, "left leaves"));
    emit_rounds(em.rounds(rv, 1, r, true, true, leaf_r, NPR, "right leaves (S2 propagation hoisted)"));
    if (split) {
      o << "    if (lane < 32) {\n";
      em.team = 32;
      em.indent = "      ";
      emit_rounds(em.rounds(ltail, 0, h, false, true, leaf_l, NPL, "left leaves, first warp"));
      o << "    } else {\n";
      o << "      const int lane_w1 = lane - 32;\n";
      o << "      {\n";
      o << "        const int lane = lane_w1;\n";
      em.indent = "        ";
      emit_rounds(em.rounds(rtail, 1, r, true, true, leaf_r, NPR,
                            "right leaves, second warp (S2 propagation hoisted)"));
      o << "      }\n";
      o << "    }\n";
      em.team = team;
      em.indent = "    ";
    }
    o << "    team_sync<TEAM>();\n";
    join("s", leaf_r);
  } else {
    // one set per iteration, one copy of the left rounds and of the join: an
    // even set also builds the right leaves of the odd set after it, whose
    // join then reads them from the first kept level
    o << "  for (int s = 0; s < " << nsets << "; ++s) {\n";
    o << "    const " << TT << "& cs = " << tab << "[s];\n";
    o << "    if ((s & 1) == 0) {\n";
    o << "      const " << TT << "& cb = " << tab << "[s + 1];\n";
    std::vector<Item> rr = right_body("cs", leaf_r);
    for (const Item& it : right_body("cb", dead_base)) rr.push_back(it);
    em.indent = "      ";
    emit_rounds(em.rounds(rr, 1, r, true, true, leaf_r, NPR, "right leaves of this set and the next (S2 propagation hoisted)"));
    em.indent = "    ";
    o << "    }\n";
    emit_rounds(em.rounds(left_body("cs"), 0, h, false, true, leaf_l, NPL, "left leaves"));
    o << "    team_sync<TEAM>();\n";
    join("s", -1);
  }
  em.indent = "  ";
  o << "  }\n";
  o << "  spec::finish_summed<TEAM>(p, acc, lane, pt, valid, s_red);\n";
  o << "  team_sync<TEAM>();\n";
  o << "}\n\n";
  o << "__global__ void __launch_bounds__(" << kd.block << ", " << kd.min_blocks << ") " << kd.name
    << "(const KParams p) {\n";
  o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o << "  constexpr int TEAM = " << team << ";\n";
  o << "  const int lane = threadIdx.x & (TEAM - 1), team = threadIdx.x / TEAM, tpc = blockDim.x / TEAM;\n";
  o << "  unsigned char* base = smem + (size_t)team * " << L.bytes << ";\n";
  o << "  for (long long pt0 = (long long)blockIdx.x * tpc; pt0 < p.n; pt0 += (long long)gridDim.x * tpc) {\n";
  o << "    const long long pt = pt0 + team;\n";
  o << "    const bool valid = pt < p.n;\n";
  o << "    " << kd.name << "_point(p, lane, valid ? pt : p.n - 1, valid, base);\n";
  o << "  }\n";
  o << "}\n\n";
  out << o.str();
  return kd;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) {
    std::fprintf(stderr, "usage: %s OUT.cu\n", argv[0]);
    return 2;
  }
  std::ostringstream out;
  out << "// GENERATED by qed_codegen.cpp from the node-reduced DAG and its linear\n"
      << "// schedule (dag.cpp); do not edit.  Kernel version " << SPEC_VERSION << ".\n"
      << "//\n"
      << "// Straight-line specialised forward kernels, spin-summed, k = 1..5: every\n"
      << "// vertex (+ propagation) instruction of the schedule expanded into rounds of\n"
      << "// the team's lanes with literal photon, polarisation rank, source,\n"
      << "// destination and propagator; the S2 joins of each photon set on the leaf\n"
      << "// layout of qed_spec.cuh.\n"
      << "#include \"qed_spec.cuh\"\n#include \"qed_plan.hpp\"\n#include \"qed_batch.cuh\"\n\nnamespace qed {\n\n";
  std::vector<KernelDesc> kds;
  try {
    for (int k = 1; k <= 5; ++k)
      for (int mixed = 1; mixed >= 0; --mixed) kds.push_back(emit_kernel(out, k, mixed != 0));
  } catch (const std::exception& e) {
    std::fprintf(stderr, "qed_codegen: %s\n", e.what());
    return 1;
  }
  // the batched evaluation's specialised form: the persistent work-item loop
  // of qed_batch_kernel (qed_batch.cuh) with the straight-line points; each
  // item kind is a call of its own (not inlined), so that registers are
  // allocated per kind rather than for their union
  out << "// The batched evaluation (requests of k = 1..5 in one persistent launch),\n"
      << "// specialised form: the work-item loop of qed_batch_kernel with the\n"
      << "// straight-line point evaluation above for every k.  One item's points\n"
      << "// per call, each kind of item a function of its own (called, not\n"
      << "// inlined: registers are allocated per kind, not for their union).\n"
      << "template <int K, typename Real>\n"
      << "__device__ __noinline__ void batch_spec_item(const KParams& kp, long long p0, long long p1,\n"
      << "                                             unsigned char* smem) {\n"
      << "  constexpr int TEAM = 1 << (K + 1);\n"
      << "  const int lane = threadIdx.x & (TEAM - 1), team = threadIdx.x / TEAM, tpc = blockDim.x / TEAM;\n";
  for (int k = 1; k <= 5; ++k) {
    int tb32 = 0, tb64 = 0;
    for (const KernelDesc& kd : kds)
      if (kd.k == k) (kd.mixed ? tb32 : tb64) = kd.team_bytes;
    out << "  " << (k == 1 ? "" : "else ") << "if constexpr (K == " << k << ") {\n"
        << "    unsigned char* base = smem + (size_t)team * (sizeof(Real) == 4 ? " << tb32 << " : " << tb64
        << ");\n"
        << "    for (long long pt0 = p0; pt0 < p1; pt0 += tpc) {\n"
        << "      const long long pt = pt0 + team;\n"
        << "      const bool valid = pt < p1;\n"
        << "      if constexpr (sizeof(Real) == 4) qed_spec_fwd_k" << k
        << "_f32_point(kp, lane, valid ? pt : p1 - 1, valid, base);\n"
        << "      else qed_spec_fwd_k" << k << "_f64_point(kp, lane, valid ? pt : p1 - 1, valid, base);\n"
        << "    }\n"
        << "  }\n";
  }
  out << "}\n\n"
      << "template <typename Real>\n"
      << "__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 2 : 1)\n"
      << "qed_batch_spec_kernel(const BatchDesc* __restrict__ reqs, const BatchItem* __restrict__ items,\n"
      << "                      int n_items, unsigned* counter) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem[];\n"
      << "  __shared__ int s_item;\n"
      << "  for (;;) {\n"
      << "    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);\n"
      << "    __syncthreads();\n"
      << "    const int it = s_item;\n"
      << "    __syncthreads();\n"
      << "    if (it >= n_items) break;\n"
      << "    const BatchItem item = items[it];\n"
      << "    const KParams& kp = reqs[item.req].kp;\n"
      << "    switch (item.k) {\n"
      << "      case 1: batch_spec_item<1, Real>(kp, item.p0, item.p1, smem); break;\n"
      << "      case 2: batch_spec_item<2, Real>(kp, item.p0, item.p1, smem); break;\n"
      << "      case 3: batch_spec_item<3, Real>(kp, item.p0, item.p1, smem); break;\n"
      << "      case 4: batch_spec_item<4, Real>(kp, item.p0, item.p1, smem); break;\n"
      << "      case 5: batch_spec_item<5, Real>(kp, item.p0, item.p1, smem); break;\n"
      << "      default: break;\n"
      << "    }\n"
      << "    __syncthreads();\n"
      << "  }\n"
      << "}\n\n"
      << "BatchFn batch_spec_kernel(bool mixed) {\n"
      << "  return mixed ? qed_batch_spec_kernel<float> : qed_batch_spec_kernel<double>;\n"
      << "}\n\n";
  out << "SpecKernel spec_forward_kernel(int k, bool mixed) {\n";
  for (const KernelDesc& kd : kds)
    out << "  if (k == " << kd.k << " && mixed == " << (kd.mixed ? "true" : "false") << ") return {" << kd.name
        << ", " << kd.team << ", " << kd.ncur << ", " << kd.team_bytes << "};\n";
  out << "  return {nullptr, 0, 0, 0};\n}\n\n";
  out << "const char* spec_version() { return \"" << SPEC_VERSION << "\"; }\n\n}  // namespace qed\n";
  const std::string text = out.str();
  std::string old;
  {
    std::ifstream f(argv[1]);
    if (f) old.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
  }
  if (old != text) {
    std::ofstream f(argv[1]);
    f << text;
    if (!f) {
      std::fprintf(stderr, "qed_codegen: cannot write %s\n", argv[1]);
      return 1;
    }
  }
  return 0;
}
