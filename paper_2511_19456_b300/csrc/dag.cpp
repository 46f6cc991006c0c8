// Host-side CDAG generator, node reduction and linear schedule.
// Paper: Sec. II-A (generator, optimiser, scheduler), Sec. II-B (the QED
// tasks U, V, S1, S2, Sum), Table I (node counts), App. C (node reduction).
#include "dag.hpp"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <unordered_map>

namespace qed {

int Dag::add(NodeKind k, int f, const int32_t* par, int npar) {
  if (pbeg.empty()) pbeg.push_back(0);
  kind.push_back(k);
  fn.push_back(f);
  for (int i = 0; i < npar; ++i) parents.push_back(par[i]);
  pbeg.push_back((int32_t)parents.size());
  return (int)kind.size() - 1;
}

Counts Dag::counts() const {
  Counts c;
  for (uint8_t k : kind) {
    ++c.total;
    switch (k) {
      case K_DATA: ++c.data; break;
      case K_U: ++c.u; break;
      case K_V: ++c.v; break;
      case K_S1: ++c.s1; break;
      case K_S2: ++c.s2; break;
      case K_SUM: ++c.sum; break;
    }
  }
  return c;
}

namespace {

inline int photon_slot(int j) { return j == 0 ? 1 : j + 2; }

// compute node followed by its output data node; returns the data node
int emit(Dag& g, NodeKind k, int f, std::initializer_list<int32_t> par) {
  std::vector<int32_t> p(par);
  int c = g.add(k, f, p.data(), (int)p.size());
  int32_t cc = c;
  return g.add(K_DATA, -1, &cc, 1);
}

long long factorial(int n) {
  long long f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

long long falling(int n, int i) {  // n! / (n-i)!
  long long f = 1;
  for (int t = 0; t < i; ++t) f *= (n - t);
  return f;
}

}  // namespace

Dag generate(int k) {
  const int n = k + 1;
  const int nslots = k + 3;
  const int h = (n + 1) / 2;
  Dag g;
  // entry data nodes (one per external particle, tagged by slot), their U
  // tasks and U output data nodes
  std::vector<int32_t> udata(nslots);
  for (int s = 0; s < nslots; ++s) {
    int e = g.add(K_DATA, 1000 + s, nullptr, 0);
    udata[s] = emit(g, K_U, s, {e});
  }
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<int32_t> diagrams;
  do {
    // left half: photons perm[0..h-1] from the incoming electron
    int32_t cur = udata[0];
    for (int i = 0; i < h; ++i) {
      cur = emit(g, K_V, 0, {udata[photon_slot(perm[i])], cur});
      if (i + 1 < h) cur = emit(g, K_S1, 0, {cur});
    }
    int32_t left = cur;
    // right half: photons perm[n-1], perm[n-2], ... from the outgoing electron
    cur = udata[2];
    for (int i = n - 1; i >= h; --i) {
      cur = emit(g, K_V, 0, {udata[photon_slot(perm[i])], cur});
      if (i > h) cur = emit(g, K_S1, 0, {cur});
    }
    diagrams.push_back(emit(g, K_S2, 0, {left, cur}));
  } while (std::next_permutation(perm.begin(), perm.end()));
  int s = g.add(K_SUM, 0, diagrams.data(), (int)diagrams.size());
  int32_t ss = s;
  g.add(K_DATA, -1, &ss, 1);
  return g;
}

Counts unreduced_counts(int k) {
  const long long n = k + 1;
  const long long d = factorial(k + 1);
  Counts c;
  c.u = k + 3;
  c.v = d * n;
  c.s1 = d * (n - 2);
  c.s2 = d;
  c.sum = 1;
  const long long compute = c.u + c.v + c.s1 + c.s2 + c.sum;
  c.data = (k + 3) + compute;
  c.total = c.data + compute;
  return c;
}

namespace {
struct KeyHash {
  size_t operator()(const std::vector<int64_t>& v) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t x : v) {
      h ^= (uint64_t)x + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};
}  // namespace

Dag reduce(const Dag& in, std::vector<int32_t>* rep_out) {
  // Single pass in topological order: a node's parents are already mapped to
  // their representatives, so nodes that agree in function and parent set
  // map to the same key.  This reaches the fixpoint of repeated reductions.
  Dag out;
  std::vector<int32_t> rep(in.size());
  std::unordered_map<std::vector<int64_t>, int32_t, KeyHash> seen;
  seen.reserve(in.size());
  std::vector<int64_t> key;
  std::vector<int32_t> par;
  for (int i = 0; i < in.size(); ++i) {
    par.clear();
    for (int p = in.pbeg[i]; p < in.pbeg[i + 1]; ++p) par.push_back(rep[in.parents[p]]);
    std::sort(par.begin(), par.end());
    par.erase(std::unique(par.begin(), par.end()), par.end());
    key.assign({(int64_t)in.kind[i], (int64_t)in.fn[i]});
    for (int32_t p : par) key.push_back(p);
    auto it = seen.find(key);
    if (it != seen.end()) {
      rep[i] = it->second;
    } else {
      int id = out.add((NodeKind)in.kind[i], in.fn[i], par.data(), (int)par.size());
      seen.emplace(key, id);
      rep[i] = id;
    }
  }
  if (rep_out) *rep_out = std::move(rep);
  return out;
}

int nvar(bool summed, int level) { return summed ? (1 << (level + 1)) : 1; }

bool reduce_step(Dag& g) {
  const int N = g.size();
  // the first group of equal compute nodes (function and parent set)
  std::unordered_map<std::vector<int64_t>, int32_t, KeyHash> first;
  std::vector<int32_t> leader(N, -1);
  std::vector<int> group_size(N, 0);
  std::vector<int64_t> key;
  int chosen = -1;
  for (int i = 0; i < N && chosen < 0; ++i) {
    if (g.kind[i] == K_DATA) continue;
    std::vector<int32_t> par(g.parents.begin() + g.pbeg[i], g.parents.begin() + g.pbeg[i + 1]);
    std::sort(par.begin(), par.end());
    key.assign({(int64_t)g.kind[i], (int64_t)g.fn[i]});
    for (int32_t p : par) key.push_back(p);
    auto it = first.find(key);
    if (it == first.end()) {
      first.emplace(key, i);
    } else {
      chosen = it->second;   // equal to an earlier node: this class is the first one complete
    }
  }
  if (chosen < 0) return false;
  // all members of the chosen class (they may lie after the one found)
  std::vector<int32_t> cpar(g.parents.begin() + g.pbeg[chosen], g.parents.begin() + g.pbeg[chosen + 1]);
  std::sort(cpar.begin(), cpar.end());
  std::vector<char> merged(N, 0);
  for (int i = chosen + 1; i < N; ++i) {
    if (g.kind[i] != g.kind[chosen] || g.fn[i] != g.fn[chosen]) continue;
    std::vector<int32_t> par(g.parents.begin() + g.pbeg[i], g.parents.begin() + g.pbeg[i + 1]);
    std::sort(par.begin(), par.end());
    if (par == cpar) merged[i] = 1;
  }
  // output data node of each compute node
  std::vector<int32_t> out_data(N, -1);
  for (int i = 0; i < N; ++i)
    if (g.kind[i] == K_DATA && g.pbeg[i + 1] - g.pbeg[i] == 1) out_data[g.parents[g.pbeg[i]]] = i;
  const int keep_data = out_data[chosen];
  // rebuild: merged nodes and their data nodes map to the kept ones
  Dag out;
  std::vector<int32_t> rep(N, -1);
  std::vector<int32_t> par;
  for (int i = 0; i < N; ++i) {
    if (merged[i]) { rep[i] = rep[chosen]; continue; }
    if (g.kind[i] == K_DATA && g.pbeg[i + 1] - g.pbeg[i] == 1 && merged[g.parents[g.pbeg[i]]]) {
      rep[i] = rep[keep_data];
      continue;
    }
    par.clear();
    for (int p = g.pbeg[i]; p < g.pbeg[i + 1]; ++p) par.push_back(rep[g.parents[p]]);
    rep[i] = out.add((NodeKind)g.kind[i], g.fn[i], par.data(), (int)par.size());
  }
  g = std::move(out);
  return true;
}

int reduction_steps(int k) {
  Dag g = generate(k);
  int s = 0;
  while (reduce_step(g)) ++s;
  return s;
}

Tape build_tape(int k, int steps) {
  if (k < 1 || k > 6) throw std::runtime_error("k out of range");
  Tape t;
  t.k = k;
  t.n = k + 1;
  const int n = t.n;
  const uint32_t all = (1u << n) - 1;
  Dag g = generate(k);
  while (t.steps < steps && reduce_step(g)) ++t.steps;
  t.counts = g.counts();
  const int N = g.size();
  std::vector<int32_t> producer(N, -1);
  for (int i = 0; i < N; ++i)
    if (g.kind[i] == K_DATA && g.pbeg[i + 1] - g.pbeg[i] == 1) producer[i] = g.parents[g.pbeg[i]];
  // per compute node: op, side, photon set, level
  std::vector<int> op(N, 0), side(N, -1), level(N, -1), photon(N, -1);
  std::vector<uint32_t> set(N, 0);
  int sum_node = -1;
  for (int i = 0; i < N; ++i) {
    const int np = g.pbeg[i + 1] - g.pbeg[i];
    const int32_t* pp = g.parents.data() + g.pbeg[i];
    switch (g.kind[i]) {
      case K_U: {
        const int s = g.fn[i];
        level[i] = 0;
        if (s == 0 || s == 2) { op[i] = T_SPINOR; side[i] = s == 0 ? 0 : 1; }
        else { op[i] = T_POL; photon[i] = s == 1 ? 0 : s - 2; }
        break;
      }
      case K_V: {
        int cur = -1, ph = -1;
        for (int a = 0; a < np; ++a) {
          const int c = producer[pp[a]];
          if (op[c] == T_POL) ph = c; else cur = c;
        }
        if (cur < 0 || ph < 0 || np != 2) throw std::runtime_error("tape: malformed V");
        op[i] = T_V;
        side[i] = side[cur];
        photon[i] = photon[ph];
        set[i] = set[cur] | (1u << photon[ph]);
        level[i] = std::max(level[cur], level[ph]) + 1;
        break;
      }
      case K_S1: {
        const int c = producer[pp[0]];
        op[i] = T_S1;
        side[i] = side[c];
        set[i] = set[c];
        level[i] = level[c] + 1;
        break;
      }
      case K_S2: {
        int a = producer[pp[0]], b = producer[pp[1]];
        if (side[a] == 1) std::swap(a, b);
        op[i] = T_S2;
        set[i] = set[a];
        level[i] = std::max(level[a], level[b]) + 1;
        break;
      }
      case K_SUM:
        sum_node = i;
        break;
      default:
        break;
    }
  }
  if (sum_node < 0) throw std::runtime_error("tape: no Sum node");
  // diagram index of each S2: its position among the Sum's parents
  std::vector<int> diag(N, -1);
  for (int p = g.pbeg[sum_node]; p < g.pbeg[sum_node + 1]; ++p) diag[producer[g.parents[p]]] = t.n_diag++;
  // last level at which each value is read
  std::vector<int> last_use(N, -1);
  int max_level = 0;
  for (int i = 0; i < N; ++i) {
    if (!op[i]) continue;
    max_level = std::max(max_level, level[i]);
    for (int p = g.pbeg[i]; p < g.pbeg[i + 1]; ++p) {
      const int c = producer[g.parents[p]];
      last_use[c] = std::max(last_use[c], level[i]);
    }
  }
  // slots: before level L, free the values last read below L; values made
  // at L get slots not read at L
  std::vector<std::vector<int>> by_level(max_level + 1);
  for (int i = 0; i < N; ++i)
    if (op[i]) by_level[level[i]].push_back(i);
  std::vector<int> slot(N, -1), free_slots;
  std::vector<std::vector<int>> dies(max_level + 2);
  for (int i = 0; i < N; ++i)
    if (op[i] && op[i] != T_S2) dies[std::max(last_use[i], level[i]) + 1].push_back(i);
  t.level_beg.push_back(0);
  for (int L = 0; L <= max_level; ++L) {
    for (int v : dies[L]) free_slots.push_back(slot[v]);
    std::sort(free_slots.begin(), free_slots.end(), std::greater<int>());
    for (int i : by_level[L]) {
      TapeInstr in{};
      in.op = (uint8_t)op[i];
      in.side = (uint8_t)std::max(0, side[i]);
      if (op[i] == T_S2) {
        in.dst = (uint16_t)diag[i];
      } else {
        int sl;
        if (!free_slots.empty()) { sl = free_slots.back(); free_slots.pop_back(); }
        else sl = t.n_slots++;
        slot[i] = sl;
        in.dst = (uint16_t)sl;
      }
      const int32_t* pp = g.parents.data() + g.pbeg[i];
      switch (op[i]) {
        case T_SPINOR: in.arg = (uint8_t)(side[i] == 0 ? 0 : 2); t.flops += FLOP_SPINOR; break;
        case T_POL: in.arg = (uint8_t)photon[i]; t.flops += FLOP_POL; break;
        case T_V: {
          int cur = producer[pp[0]], ph = producer[pp[1]];
          if (op[cur] == T_POL) std::swap(cur, ph);
          in.arg = (uint8_t)photon[i];
          in.src0 = (uint16_t)slot[cur];
          in.src1 = (uint16_t)slot[ph];
          t.flops += FLOP_V;
          break;
        }
        case T_S1:
          in.src0 = (uint16_t)slot[producer[pp[0]]];
          in.mask = (uint16_t)(side[i] == 0 ? set[i] : all & ~set[i]);
          t.flops += FLOP_SUBSET + FLOP_S1;
          break;
        case T_S2: {
          int a = producer[pp[0]], b = producer[pp[1]];
          if (side[a] == 1) std::swap(a, b);
          in.src0 = (uint16_t)slot[a];
          in.src1 = (uint16_t)slot[b];
          in.mask = (uint16_t)set[a];
          t.flops += FLOP_SUBSET + FLOP_S1 + FLOP_JOIN;
          break;
        }
      }
      t.instr.push_back(in);
    }
    t.level_beg.push_back((int32_t)t.instr.size());
  }
  if (t.n_slots > 65535) throw std::runtime_error("tape: too many slots");
  t.flops += (long long)t.n_diag * FLOP_SUM + 3;
  return t;
}

namespace {

struct VInfo {
  int side = -1;        // 0 left (from e- in), 1 right (from e- out)
  int level = 0;
  int photon = -1;
  int parent = -1;      // parent V (reduced DAG id) or -1
  uint32_t set = 0;
  bool has_s1 = false;
  bool in_s2 = false;
};

int rank_in(uint32_t set, int j) { return __builtin_popcount(set & ((1u << j) - 1)); }

}  // namespace

Schedule build_schedule(int k, bool summed, int ls, int rs) {
  if (k < 1 || k > 7) throw std::runtime_error("k out of range");
  Schedule sc;
  sc.k = k;
  sc.n = k + 1;
  sc.h = (sc.n + 1) / 2;
  sc.r = sc.n - sc.h;
  sc.summed = summed;
  sc.ls = std::max(0, std::min(ls, sc.h - 1));
  sc.rs = std::max(0, std::min(rs, sc.r - 1));
  const int n = sc.n, h = sc.h, r = sc.r;
  const uint32_t all = (1u << n) - 1;

  Dag g = generate(k);
  sc.unreduced = g.counts();
  Dag d = reduce(g);
  sc.reduced = d.counts();

  // ---- recover the structure of the reduced DAG
  const int N = d.size();
  std::vector<int> slot_of_udata(N, -1);   // U output data node -> slot
  std::vector<int> producer(N, -1);        // data node -> its compute node
  for (int i = 0; i < N; ++i) {
    if (d.kind[i] == K_DATA && d.pbeg[i + 1] - d.pbeg[i] == 1) {
      int c = d.parents[d.pbeg[i]];
      producer[i] = c;
      if (d.kind[c] == K_U) slot_of_udata[i] = d.fn[c];
    }
  }
  auto photon_of_slot = [](int s) { return s == 1 ? 0 : (s >= 3 ? s - 2 : -1); };
  std::vector<VInfo> vi(N);
  std::vector<std::pair<int, int>> s2list;
  for (int i = 0; i < N; ++i) {
    if (d.kind[i] == K_V) {
      int a = d.parents[d.pbeg[i]], b = d.parents[d.pbeg[i] + 1];
      int ph = -1, cur = -1;
      for (int x : {a, b}) {
        int s = slot_of_udata[x];
        if (s >= 0 && photon_of_slot(s) >= 0) ph = photon_of_slot(s); else cur = x;
      }
      if (ph < 0 || cur < 0 || d.pbeg[i + 1] - d.pbeg[i] != 2)
        throw std::runtime_error("malformed V node");
      VInfo& v = vi[i];
      v.photon = ph;
      int src = producer[cur];
      if (d.kind[src] == K_U) {
        v.side = (d.fn[src] == 0) ? 0 : (d.fn[src] == 2 ? 1 : -1);
        if (v.side < 0) throw std::runtime_error("V attached to a photon state");
        v.level = 1;
        v.set = 1u << ph;
      } else if (d.kind[src] == K_S1) {
        int pv = producer[d.parents[d.pbeg[src]]];
        if (d.kind[pv] != K_V) throw std::runtime_error("S1 not after V");
        v.side = vi[pv].side;
        v.level = vi[pv].level + 1;
        v.parent = pv;
        v.set = vi[pv].set | (1u << ph);
      } else {
        throw std::runtime_error("V input is neither U nor S1");
      }
    } else if (d.kind[i] == K_S1) {
      int pv = producer[d.parents[d.pbeg[i]]];
      vi[pv].has_s1 = true;
    } else if (d.kind[i] == K_S2) {
      int a = producer[d.parents[d.pbeg[i]]], b = producer[d.parents[d.pbeg[i] + 1]];
      if (vi[a].side == 1) std::swap(a, b);
      vi[a].in_s2 = vi[b].in_s2 = true;
      s2list.emplace_back(a, b);
    }
  }
  // ---- check the reduced DAG is the pair of prefix/suffix tries
  std::vector<std::vector<int>> lv(h + 1), rv(r + 1);
  for (int i = 0; i < N; ++i) {
    if (d.kind[i] != K_V) continue;
    const VInfo& v = vi[i];
    if (v.side == 0) lv.at(v.level).push_back(i); else rv.at(v.level).push_back(i);
    bool leaf = (v.side == 0) ? v.level == h : v.level == r;
    if (leaf != v.in_s2 || leaf == v.has_s1) throw std::runtime_error("unexpected trie shape");
  }
  for (int i = 1; i <= h; ++i)
    if ((long long)lv[i].size() != falling(n, i)) throw std::runtime_error("left level size");
  for (int i = 1; i <= r; ++i)
    if ((long long)rv[i].size() != falling(n, i)) throw std::runtime_error("right level size");
  if ((long long)s2list.size() != factorial(n)) throw std::runtime_error("S2 count");
  for (auto& pr : s2list)
    if ((vi[pr.first].set | vi[pr.second].set) != all || (vi[pr.first].set & vi[pr.second].set))
      throw std::runtime_error("S2 halves do not partition the photons");

  // ---- storage and instructions
  std::vector<int> index(N, -1);
  int next = 0;
  auto make_instr = [&](int node, int dst, int src) {
    const VInfo& v = vi[node];
    Instr in{};
    in.dst = dst;
    in.src = src;
    in.side = (uint8_t)v.side;
    in.photon = (uint8_t)v.photon;
    in.rank = (uint8_t)rank_in(v.set, v.photon);
    in.level = (uint8_t)v.level;
    if (v.side == 0) in.post = v.has_s1 ? (uint16_t)v.set : 0;
    else in.post = (uint16_t)(all & ~v.set);  // inner: S1; leaf: hoisted S2 propagation
    return in;
  };
  auto push_range = [&](Phase& ph, int slot, int beg, int cnt, int level) {
    ph.beg[slot] = beg;
    ph.cnt[slot] = cnt;
    ph.level[slot] = level;
  };
  // stored levels
  const int nsp = std::max(sc.ls, sc.rs);
  for (int dlev = 1; dlev <= nsp; ++dlev) {
    Phase ph{};
    int slot = 0;
    for (int side = 0; side < 2; ++side) {
      int lim = side == 0 ? sc.ls : sc.rs;
      if (dlev > lim) continue;
      auto& lst = side == 0 ? lv[dlev] : rv[dlev];
      int beg = (int)sc.instr.size();
      for (int node : lst) {
        index[node] = next;
        int src = vi[node].parent >= 0 ? index[vi[node].parent] : -1;
        sc.instr.push_back(make_instr(node, next, src));
        next += nvar(summed, dlev);
      }
      push_range(ph, slot++, beg, (int)lst.size(), dlev);
    }
    sc.phases.push_back(ph);
  }
  sc.n_stored_phases = (int)sc.phases.size();
  sc.stored_currents = next;

  // per photon set S (|S| = h): local levels
  sc.n_set_phases = std::max(h - sc.ls, r - sc.rs);
  sc.n_left_leaves = (int)factorial(h);
  sc.n_right_leaves = (int)factorial(r);
  std::vector<uint32_t> setmasks;
  for (uint32_t m = 0; m <= all; ++m)
    if (__builtin_popcount(m) == h) setmasks.push_back(m);
  int local_size = -1;
  std::vector<int> lindex(N, -1);
  for (uint32_t S : setmasks) {
    SetEntry se{};
    se.mask = S;
    se.phase0 = (int)sc.phases.size();
    int lnext = sc.stored_currents;
    std::vector<int> touched;
    // assign local indices: left levels ls+1..h, then right levels rs+1..r
    std::vector<std::vector<int>> lloc(h + 1), rloc(r + 1);
    for (int dl = sc.ls + 1; dl <= h; ++dl)
      for (int node : lv[dl])
        if ((vi[node].set & ~S) == 0) lloc[dl].push_back(node);
    for (int dl = sc.rs + 1; dl <= r; ++dl)
      for (int node : rv[dl])
        if ((vi[node].set & S) == 0) rloc[dl].push_back(node);
    if ((int)lloc[h].size() != sc.n_left_leaves || (int)rloc[r].size() != sc.n_right_leaves)
      throw std::runtime_error("leaf count per set");
    for (int dl = sc.ls + 1; dl <= h; ++dl) {
      if (dl == h) se.leaf_l = lnext;
      for (int node : lloc[dl]) { lindex[node] = lnext; touched.push_back(node); lnext += nvar(summed, dl); }
    }
    for (int dl = sc.rs + 1; dl <= r; ++dl) {
      if (dl == r) se.leaf_r = lnext;
      for (int node : rloc[dl]) { lindex[node] = lnext; touched.push_back(node); lnext += nvar(summed, dl); }
    }
    if (local_size < 0) local_size = lnext - sc.stored_currents;
    else if (local_size != lnext - sc.stored_currents) throw std::runtime_error("set size");
    auto src_of = [&](int node) {
      int p = vi[node].parent;
      if (p < 0) return -1;
      return lindex[p] >= 0 ? lindex[p] : index[p];
    };
    for (int t = 1; t <= sc.n_set_phases; ++t) {
      Phase ph{};
      int slot = 0;
      for (int side = 0; side < 2; ++side) {
        int dl = (side == 0 ? sc.ls : sc.rs) + t;
        int lim = side == 0 ? h : r;
        if (dl > lim) continue;
        auto& lst = side == 0 ? lloc[dl] : rloc[dl];
        int beg = (int)sc.instr.size();
        for (int node : lst) {
          int src = src_of(node);
          if (vi[node].parent >= 0 && src < 0) throw std::runtime_error("missing parent");
          sc.instr.push_back(make_instr(node, lindex[node], src));
        }
        push_range(ph, slot++, beg, (int)lst.size(), dl);
      }
      sc.phases.push_back(ph);
    }
    for (int node : touched) lindex[node] = -1;
    sc.sets.push_back(se);
  }
  sc.local_currents = local_size;

  // ---- arithmetic counts
  const long long P = summed ? (1ll << (n + 2)) : 1;
  long long alg = 0, lit = 0;
  for (int i = 0; i < N; ++i) {
    if (d.kind[i] != K_V) continue;
    const VInfo& v = vi[i];
    long long nv = nvar(summed, v.level);
    sc.v_nodes += nv;
    alg += nv * FLOP_V;
    bool post = (v.side == 0) ? v.has_s1 : true;
    bool real_s1 = v.has_s1;
    if (post) alg += nv * FLOP_S1;
    if (real_s1) { sc.s1_nodes += nv; lit += nv * FLOP_S1; }
    lit += nv * FLOP_V;
  }
  sc.s2_nodes = factorial(n) * P;
  long long fixed_cost = ((1ll << n) - 2) * FLOP_SUBSET + 4ll * FLOP_SPINOR + 2ll * n * FLOP_POL +
                         P * FLOP_SQUARE;
  alg += sc.s2_nodes * FLOP_JOIN + fixed_cost;
  lit += sc.s2_nodes * (FLOP_JOIN + FLOP_S1) + fixed_cost;
  long long exec = fixed_cost + sc.s2_nodes * FLOP_JOIN;
  for (const Instr& in : sc.instr) {
    long long nv = nvar(summed, in.level);
    exec += nv * (FLOP_V + (in.post ? FLOP_S1 : 0));
  }
  sc.flops_algorithmic = alg;
  sc.flops_literal_s2 = lit;
  sc.flops_executed = exec;
  return sc;
}

static long long n_choose(int n, int m) {
  long long c = 1;
  for (int i = 1; i <= m; ++i) c = c * (n - m + i) / i;
  return c;
}

int rewrite_default_group(int k, bool summed, int team) {
  const int n = k + 1, h = (n + 1) / 2, r = n - h;
  const int per_set = nvar(summed, h) + nvar(summed, r);
  const int nsets = (int)n_choose(n, h);
  const int g = std::max(1, std::min(nsets, (4 * team + per_set - 1) / per_set));
  const int groups = (nsets + g - 1) / g;
  return (nsets + groups - 1) / groups;   // groups of nearly equal size
}

RwSchedule build_rewrite_schedule(int k, bool summed, int group) {
  if (k < 1 || k > 7) throw std::runtime_error("k out of range");
  if (group <= 0) group = rewrite_default_group(k, summed, summed ? 1 << (k + 1) : 32);
  RwSchedule sc;
  sc.k = k;
  sc.n = k + 1;
  sc.h = (sc.n + 1) / 2;
  sc.r = sc.n - sc.h;
  sc.summed = summed;
  const int n = sc.n, h = sc.h, r = sc.r;
  const uint32_t all = (1u << n) - 1;
  // node index of (side, subset) for the kept levels
  std::vector<int> idx[2];
  idx[0].assign(1u << n, -1);
  idx[1].assign(1u << n, -1);
  int next = 0;
  auto make = [&](int side, uint32_t T, int dst, bool post) {
    SumInstr in{};
    in.dst = dst;
    in.side = (uint8_t)side;
    in.level = (uint8_t)__builtin_popcount(T);
    int t = 0;
    for (int j = 0; j < n; ++j) {
      if (!(T & (1u << j))) continue;
      const uint32_t par = T & ~(1u << j);
      in.src[t] = par ? idx[side][par] : -1;
      if (par && in.src[t] < 0) throw std::runtime_error("rewrite: missing input node");
      in.photon[t] = (uint8_t)j;
      in.rank[t] = (uint8_t)__builtin_popcount(T & ((1u << j) - 1));
      ++t;
    }
    for (; t < 4; ++t) { in.src[t] = -1; in.photon[t] = 0; in.rank[t] = 0; }
    in.nterms = (uint8_t)in.level;
    if (side == 0) in.post = post ? (uint16_t)T : 0;
    else in.post = (uint16_t)(all & ~T);
    return in;
  };
  const int nsp = std::max(h - 1, r - 1);
  for (int lev = 1; lev <= nsp; ++lev) {
    Phase ph{};
    int slot = 0;
    for (int side = 0; side < 2; ++side) {
      const int lim = side == 0 ? h - 1 : r - 1;
      if (lev > lim) continue;
      const int beg = (int)sc.instr.size();
      int cnt = 0;
      for (uint32_t T = 1; T <= all; ++T) {
        if (__builtin_popcount(T) != lev) continue;
        idx[side][T] = next;
        sc.instr.push_back(make(side, T, next, true));
        next += nvar(summed, lev);
        ++cnt;
      }
      ph.beg[slot] = beg;
      ph.cnt[slot] = cnt;
      ph.level[slot] = lev;
      ++slot;
    }
    sc.phases.push_back(ph);
  }
  sc.n_stored_phases = (int)sc.phases.size();
  sc.stored_currents = next;
  sc.n_set_phases = 1;
  std::vector<uint32_t> masks;
  for (uint32_t S = 0; S <= all; ++S)
    if (__builtin_popcount(S) == h) masks.push_back(S);
  const int nsets = (int)masks.size();
  sc.group = std::min(group, nsets);
  const int nvh = nvar(summed, h), nvr = nvar(summed, r);
  for (int g0 = 0; g0 < nsets; g0 += sc.group) {
    const int g1 = std::min(nsets, g0 + sc.group);
    Phase ph{};
    ph.beg[0] = (int)sc.instr.size();
    ph.cnt[0] = g1 - g0;
    ph.level[0] = h;
    for (int i = g0; i < g1; ++i) sc.instr.push_back(make(0, masks[i], next + (i - g0) * nvh, false));
    ph.beg[1] = (int)sc.instr.size();
    ph.cnt[1] = g1 - g0;
    ph.level[1] = r;
    const int rbase = next + (g1 - g0) * nvh;
    for (int i = g0; i < g1; ++i) sc.instr.push_back(make(1, all & ~masks[i], rbase + (i - g0) * nvr, true));
    for (int i = g0; i < g1; ++i) {
      SetEntry se{};
      se.mask = masks[i];
      se.phase0 = (int)sc.phases.size();
      se.leaf_l = next + (i - g0) * nvh;
      se.leaf_r = rbase + (i - g0) * nvr;
      sc.sets.push_back(se);
    }
    sc.phases.push_back(ph);
    ++sc.n_groups;
  }
  sc.local_currents = sc.group * (nvh + nvr);
  // counts and FLOPs of the rewritten DAG (each subset node once; the
  // per-set leaves are the level-h / level-r nodes)
  const long long P = summed ? (1ll << (n + 2)) : 1;
  long long fl = ((1ll << n) - 2) * FLOP_SUBSET + 4ll * FLOP_SPINOR + 2ll * n * FLOP_POL + P * FLOP_SQUARE;
  for (int side = 0; side < 2; ++side) {
    const int top = side == 0 ? h : r;
    for (uint32_t T = 1; T <= all; ++T) {
      const int lev = __builtin_popcount(T);
      if (lev > top) continue;
      const long long nv = nvar(summed, lev);
      sc.nodes += nv;
      sc.terms += nv * lev;
      fl += nv * (lev * FLOP_V + (lev - 1) * 8);
      const bool post = side == 1 || lev < top;
      if (post) { sc.s1_nodes += nv; fl += nv * FLOP_S1; }
    }
  }
  sc.joins = (long long)nsets * P;
  fl += sc.joins * FLOP_JOIN;
  sc.flops_algorithmic = fl;
  return sc;
}

}  // namespace qed
