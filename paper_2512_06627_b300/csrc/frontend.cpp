// frontend.cpp -- host front end of the ES engine.
//
// Steps (paper §2.1 and §3.3):
//   cone     transitive fan-in of the miter output; support = PIs reached,
//            sorted by PI index (support PI k <-> pattern bit k);
//   order    a topological order of the cone's ANDs (DFS post-order with the
//            deeper fanin first, ascending variable, or by level);
//   slots    "registers aggressively reused under reference-count guidance":
//            every value's reference count is its number of fanout edges in
//            the cone (+1 for the output); walking the order, each AND reads
//            its operands, drops their counts, frees operands that reach zero
//            (lowest free slot first), then takes a slot for its result, which
//            may be an operand's just-freed slot.  PIs and the constant are
//            loaded lazily into a slot right before their first reader.
// The peak slot count is the live-set size the kernels must hold per lane.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <vector>

#include "../../include/lec_es.h"
#include "es_internal.h"

namespace lec {

namespace {

struct Cone {
  std::vector<uint32_t> ands;   // cone AND vars, ascending
  std::vector<uint32_t> pis;    // support PI vars (1-based), ascending
  bool uses_const = false;
};

inline const uint32_t *fanin_of(const MiterView &m, uint32_t v) {
  return m.fanins + 2ull * (v - m.num_pis - 1);
}

int extract_cone(const MiterView &m, std::vector<uint8_t> &mark, Cone &c) {
  const uint64_t maxvar = (uint64_t)m.num_pis + m.num_ands;
  const uint32_t root = m.out_lit >> 1;
  if (root > maxvar) return LEC_ES_EINVAL;
  if (m.num_ands && !m.fanins) return LEC_ES_EINVAL;
  // A walk from the output over the cone's own fanins marks its variables
  // (cost: the cone, not the graph it is cut from).  The lists must come out
  // ascending: a cone that fills most of its variable span is collected by
  // one scan of the marks over that span (sequential bytes), a sparse one
  // (a small cone of a large shared graph) by sorting what the walk found.
  // Marks are cleared before returning.
  mark.resize(maxvar + 1, 0);
  thread_local std::vector<uint32_t> stack;
  stack.clear();
  int rc = LEC_ES_OK;
  uint32_t lowest = root;
  auto visit = [&](uint32_t u) {
    if (mark[u]) return;
    mark[u] = 1;
    if (u > m.num_pis) {
      c.ands.push_back(u);
      stack.push_back(u);
      lowest = std::min(lowest, u);
    } else if (u > 0) {
      c.pis.push_back(u);
    }
  };
  visit(root);
  while (!stack.empty()) {
    const uint32_t v = stack.back();
    stack.pop_back();
    const uint32_t *f = fanin_of(m, v);
    const uint32_t a = f[0] >> 1, b = f[1] >> 1;
    if (a >= v || b >= v) {  // fanins must precede their AND
      rc = LEC_ES_EINVAL;
      break;
    }
    visit(a);
    visit(b);
  }
  c.uses_const = mark[0] != 0;
  mark[0] = 0;
  for (uint32_t u : c.pis) mark[u] = 0;
  if (rc) {
    for (uint32_t u : c.ands) mark[u] = 0;
    c.ands.clear();
    c.pis.clear();
    return rc;
  }
  const size_t k = c.ands.size();
  if (k > 1 && (uint64_t)(root - lowest + 1) <= 16ull * k) {
    c.ands.clear();
    for (uint32_t u = lowest; u <= root; u++)
      if (mark[u]) {
        mark[u] = 0;
        c.ands.push_back(u);
      }
  } else {
    for (uint32_t u : c.ands) mark[u] = 0;
    std::sort(c.ands.begin(), c.ands.end());
  }
  std::sort(c.pis.begin(), c.pis.end());
  return LEC_ES_OK;
}

// Dense index of the cone's variables: value id of every cone variable
// (ANDs 0..NA-1 in ascending order, PIs NA.., the constant last), in a
// per-thread array over the whole graph that is reset when the cone is done,
// so many cones of one large graph cost only their own size.
struct ConeIndex {
  const Cone &c;
  std::vector<int32_t> &id;  // variable -> value id, -1 outside the cone
  ConeIndex(const Cone &cc, std::vector<int32_t> &map, uint64_t maxvar) : c(cc), id(map) {
    if (id.size() < maxvar + 1) id.resize(maxvar + 1, -1);
    const size_t NA = c.ands.size(), NP = c.pis.size();
    for (size_t i = 0; i < NA; i++) id[c.ands[i]] = (int32_t)i;
    for (size_t k = 0; k < NP; k++) id[c.pis[k]] = (int32_t)(NA + k);
    id[0] = (int32_t)(NA + NP);
  }
  ~ConeIndex() {
    for (uint32_t v : c.ands) id[v] = -1;
    for (uint32_t v : c.pis) id[v] = -1;
    id[0] = -1;
  }
  int64_t and_pos(uint32_t v) const {
    const int32_t x = id[v];
    return x >= 0 && (size_t)x < c.ands.size() ? x : -1;
  }
  int64_t vid(uint32_t v) const { return id[v]; }
};

void order_levels(const MiterView &m, const Cone &c, const ConeIndex &ix, std::vector<uint32_t> &level) {
  level.assign(c.ands.size(), 0);
  for (size_t i = 0; i < c.ands.size(); i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    uint32_t l = 0;
    for (int e = 0; e < 2; e++) {
      int64_t p = ix.and_pos(f[e] >> 1);
      if (p >= 0) l = std::max(l, level[p] + 1);
    }
    level[i] = l;
  }
}

// Evaluation orders; each returns positions into c.ands.
void order_var(const Cone &c, std::vector<uint32_t> &ord) {
  ord.resize(c.ands.size());
  for (size_t i = 0; i < ord.size(); i++) ord[i] = (uint32_t)i;
}

void order_level(const std::vector<uint32_t> &level, std::vector<uint32_t> &ord) {
  ord.resize(level.size());
  for (size_t i = 0; i < ord.size(); i++) ord[i] = (uint32_t)i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return level[x] < level[y]; });
}

void order_dfs(const MiterView &m, const Cone &c, const ConeIndex &ix, const std::vector<uint32_t> &level,
               uint32_t root_var, std::vector<uint32_t> &ord) {
  ord.clear();
  ord.reserve(c.ands.size());
  std::vector<uint8_t> state(c.ands.size(), 0);  // 0 new, 1 open, 2 done
  int64_t rp = ix.and_pos(root_var);
  if (rp < 0) return;
  std::vector<std::pair<uint32_t, uint8_t>> stack;
  stack.push_back({(uint32_t)rp, 0});
  while (!stack.empty()) {
    auto &top = stack.back();
    uint32_t i = top.first;
    if (top.second == 0) {
      if (state[i]) { stack.pop_back(); continue; }
      state[i] = 1;
      top.second = 1;
      const uint32_t *f = fanin_of(m, c.ands[i]);
      int64_t p0 = ix.and_pos(f[0] >> 1), p1 = ix.and_pos(f[1] >> 1);
      // push so that the deeper fanin is visited (and finished) first
      int64_t first = p0, second = p1;
      uint32_t l0 = p0 >= 0 ? level[p0] + 1 : 0, l1 = p1 >= 0 ? level[p1] + 1 : 0;
      if (l1 > l0) std::swap(first, second);
      if (second >= 0 && !state[second]) stack.push_back({(uint32_t)second, 0});
      if (first >= 0 && !state[first]) stack.push_back({(uint32_t)first, 0});
    } else {
      stack.pop_back();
      if (state[i] == 1) {
        state[i] = 2;
        ord.push_back(i);
      }
    }
  }
}

// Greedy list scheduling for a small live set: among the ANDs whose fanins
// are computed, take the one whose evaluation changes the number of live
// values least (+1 for its result, +1 per PI or constant it loads first,
// -1 per operand it reads for the last time); ties go to the most recently
// readied node, which keeps chains together.
void order_greedy(const MiterView &m, const Cone &c, const ConeIndex &ix, uint32_t root_var,
                  std::vector<uint32_t> &ord) {
  const size_t NA = c.ands.size(), NP = c.pis.size();
  const size_t NV = NA + NP + 1;
  auto vid = [&](uint32_t var) -> int64_t { return ix.vid(var); };
  std::vector<int64_t> f0(NA), f1(NA);
  std::vector<uint32_t> refs(NV, 0), pending(NA, 0);
  std::vector<std::vector<uint32_t>> users(NV);
  for (size_t i = 0; i < NA; i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    f0[i] = vid(f[0] >> 1);
    f1[i] = vid(f[1] >> 1);
    refs[f0[i]]++;
    refs[f1[i]]++;
    users[f0[i]].push_back((uint32_t)i);
    if (f1[i] != f0[i]) users[f1[i]].push_back((uint32_t)i);
    pending[i] = (f0[i] < (int64_t)NA ? 1u : 0u) + (f1[i] < (int64_t)NA && f1[i] != f0[i] ? 1u : 0u);
  }
  refs[vid(root_var)]++;
  std::vector<uint8_t> loaded(NV, 0), done(NA, 0);
  auto delta = [&](uint32_t i) -> int {
    int d = 1;
    const int64_t a = f0[i], b = f1[i];
    if (a >= (int64_t)NA && !loaded[a]) d++;
    if (b != a && b >= (int64_t)NA && !loaded[b]) d++;
    if (a == b) {
      if (refs[a] == 2) d--;
    } else {
      if (refs[a] == 1) d--;
      if (refs[b] == 1) d--;
    }
    return d;
  };
  typedef std::pair<int, int64_t> Key;  // (delta, -stamp)
  std::priority_queue<std::pair<Key, uint32_t>, std::vector<std::pair<Key, uint32_t>>,
                      std::greater<std::pair<Key, uint32_t>>>
      pq;
  int64_t stamp = 0;
  auto push = [&](uint32_t i) { pq.push({{delta(i), -(stamp++)}, i}); };
  for (size_t i = 0; i < NA; i++)
    if (pending[i] == 0) push((uint32_t)i);
  ord.clear();
  ord.reserve(NA);
  while (!pq.empty()) {
    auto top = pq.top();
    pq.pop();
    const uint32_t i = top.second;
    if (done[i]) continue;
    if (top.first.first != delta(i)) {  // stale key
      push(i);
      continue;
    }
    done[i] = 1;
    ord.push_back(i);
    for (int64_t v : {f0[i], f1[i]}) {
      if (v >= (int64_t)NA && !loaded[v]) {
        loaded[v] = 1;
        for (uint32_t u : users[v])
          if (!done[u] && pending[u] == 0) push(u);
      }
    }
    refs[f0[i]]--;
    refs[f1[i]]--;
    for (int64_t v : {f0[i], f1[i]}) {
      if (refs[v] == 1)
        for (uint32_t u : users[v])
          if (!done[u] && pending[u] == 0) push(u);
    }
    loaded[i] = 1;
    for (uint32_t u : users[i]) {
      if (--pending[u] == 0) push(u);
    }
  }
}

// Spread reads away from writes: reorder a topological AND order so that,
// where it can, no AND reads the result of one of the `window` ANDs just
// before it -- list scheduling with the given order as priority, taking the
// first ready AND (looking at most kLook ready ANDs ahead) that reads none of
// them, else the first ready one.  The interpreter evaluates kInterpStep
// records at once and needs no forwarding between records of a step that
// are independent.  Nearby ready ANDs are taken, so the live set barely
// changes.
void separate_reads(const MiterView &m, const Cone &c, const ConeIndex &ix, uint32_t window,
                    std::vector<uint32_t> &ord) {
  constexpr int kLook = 16;
  const size_t NA = c.ands.size();
  if (window == 0 || NA < 3 || ord.size() != NA) return;
  std::vector<uint32_t> prio(NA), pending(NA, 0);
  for (size_t k = 0; k < NA; k++) prio[ord[k]] = (uint32_t)k;
  std::vector<uint32_t> ustart(NA + 1, 0), users;
  std::vector<int64_t> fa(2 * NA);
  for (size_t i = 0; i < NA; i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    for (int e = 0; e < 2; e++) {
      const int64_t p = ix.and_pos(f[e] >> 1);
      fa[2 * i + e] = (e == 1 && p == fa[2 * i]) ? -1 : p;  // a repeated fanin counts once
      if (fa[2 * i + e] >= 0) {
        ustart[p + 1]++;
        pending[i]++;
      }
    }
  }
  for (size_t i = 0; i < NA; i++) ustart[i + 1] += ustart[i];
  users.resize(ustart[NA]);
  {
    std::vector<uint32_t> fill(ustart.begin(), ustart.end() - 1);
    for (size_t i = 0; i < NA; i++)
      for (int e = 0; e < 2; e++)
        if (fa[2 * i + e] >= 0) users[fill[fa[2 * i + e]]++] = (uint32_t)i;
  }
  // ready ANDs by priority (a min-heap of (priority, index))
  std::priority_queue<std::pair<uint32_t, uint32_t>, std::vector<std::pair<uint32_t, uint32_t>>,
                      std::greater<std::pair<uint32_t, uint32_t>>>
      ready;
  for (size_t i = 0; i < NA; i++)
    if (!pending[i]) ready.push({prio[i], (uint32_t)i});
  std::vector<uint32_t> out;
  out.reserve(NA);
  std::vector<uint32_t> recent;  // the last `window` emitted
  std::pair<uint32_t, uint32_t> held[kLook];
  while (!ready.empty()) {
    int nh = 0, pick = -1;
    while (!ready.empty() && nh < kLook) {
      held[nh] = ready.top();
      ready.pop();
      const uint32_t i = held[nh].second;
      bool near = false;
      for (uint32_t r : recent) near |= (int64_t)r == fa[2 * i] || (int64_t)r == fa[2 * i + 1];
      nh++;
      if (!near) {
        pick = nh - 1;
        break;
      }
    }
    if (pick < 0) pick = 0;
    for (int h = 0; h < nh; h++)
      if (h != pick) ready.push(held[h]);
    const uint32_t i = held[pick].second;
    out.push_back(i);
    recent.push_back(i);
    if (recent.size() > window) recent.erase(recent.begin());
    for (uint32_t k = ustart[i]; k < ustart[i + 1]; k++)
      if (--pending[users[k]] == 0) ready.push({prio[users[k]], users[k]});
  }
  if (out.size() == NA) ord.swap(out);
}

// Reference-count slot assignment over a given order.
int assign_slots(const MiterView &m, const Cone &c, const ConeIndex &ix, const std::vector<uint32_t> &ord,
                 uint32_t root_var, uint32_t step, Program &p) {
  const size_t NA = c.ands.size(), NP = c.pis.size();
  // value ids: [0, NA) ANDs, [NA, NA+NP) PIs, NA+NP the constant
  const size_t NV = NA + NP + 1;
  auto vid = [&](uint32_t var) -> int64_t { return ix.vid(var); };
  std::vector<uint32_t> refs(NV, 0);
  std::vector<int64_t> f0v(NA), f1v(NA);
  for (size_t i = 0; i < NA; i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    f0v[i] = vid(f[0] >> 1);
    f1v[i] = vid(f[1] >> 1);
    refs[f0v[i]]++;
    refs[f1v[i]]++;
  }
  int64_t root = vid(root_var);
  refs[root]++;
  std::vector<int32_t> slot(NV, -1);
  std::priority_queue<uint32_t, std::vector<uint32_t>, std::greater<uint32_t>> freel;
  uint32_t high = 0;
  auto alloc = [&]() -> uint32_t {
    if (!freel.empty()) {
      uint32_t s = freel.top();
      freel.pop();
      return s;
    }
    return high++;
  };
  // AND records emitted since the last load record (at most step - 1)
  std::vector<uint16_t> recent;
  auto load = [&](int64_t v) {
    if (slot[v] >= 0) return;
    recent.clear();
    uint32_t s = alloc();
    slot[v] = (int32_t)s;
    Rec r{};
    r.dst = (uint16_t)s;
    if (v == (int64_t)(NA + NP)) {
      r.op = OP_CONST0;
    } else {
      r.op = OP_PI;
      r.a = (uint16_t)(v - NA);   // support index k
    }
    p.recs.push_back(r);
  };
  p.recs.clear();
  p.order_vars.clear();
  for (uint32_t i : ord) {
    int64_t a = f0v[i], b = f1v[i];
    if (a >= (int64_t)NA) load(a);
    if (b >= (int64_t)NA) load(b);
    if (slot[a] < 0 || slot[b] < 0) return LEC_ES_EINVAL;  // order not topological
    Rec r{};
    r.a = (uint16_t)slot[a];
    r.b = (uint16_t)slot[b];
    const uint32_t *f = fanin_of(m, c.ands[i]);
    r.op = (uint8_t)(OP_AND | (f[0] & 1) | ((f[1] & 1) << 1));
    // A step-`step` program is evaluated `step` AND records of a run (records
    // between two loads) at once, all operand loads first: an AND that reads
    // the result of one of the step - 1 ANDs before it in its run starts a
    // new run, behind a load of the constant into a free slot.
    bool near = false;
    for (uint16_t d : recent) near |= d == r.a || d == r.b;
    if (near) {
      Rec z{};
      z.op = OP_CONST0;
      z.pad = kRecBreak;
      if (freel.empty()) freel.push(high++);
      z.dst = (uint16_t)freel.top();
      p.recs.push_back(z);
      recent.clear();
    }
    // when a == b both edges count, so the count reaches zero at most once
    if (--refs[a] == 0) freel.push((uint32_t)slot[a]);
    if (--refs[b] == 0) freel.push((uint32_t)slot[b]);
    uint32_t d = alloc();
    r.dst = (uint16_t)d;
    slot[i] = (int32_t)d;
    p.recs.push_back(r);
    p.order_vars.push_back(c.ands[i]);
    if (step > 1) {
      recent.push_back(r.dst);
      if (recent.size() > (size_t)step - 1) recent.erase(recent.begin());
    }
    if (high > 65535) return LEC_ES_ETOOBIG;
  }
  if (root >= (int64_t)NA) load(root);  // output is a PI or the constant
  p.num_slots = high;
  p.out_slot = (uint32_t)slot[root];
  p.step = step;
  return LEC_ES_OK;
}

// 3-input table cover of the cone and its evaluation order: post-order from
// the output, deeper leaf first; the live count is the peak number of table
// outputs and PIs alive at once (each value dies after its last reader).
// The cone's 3-input table cover (independent of the evaluation order).
void cover_cone(const MiterView &m, const Cone &c, const ConeIndex &ix, uint32_t root_var, LutProgram &lp,
                LutCover &cov) {
  const size_t NA = c.ands.size(), NP = c.pis.size();
  auto vid = [&](uint32_t var) -> int64_t { return ix.vid(var); };
  std::vector<int64_t> f0(NA), f1(NA);
  std::vector<uint8_t> c0(NA), c1(NA);
  for (size_t i = 0; i < NA; i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    f0[i] = vid(f[0] >> 1);
    f1[i] = vid(f[1] >> 1);
    c0[i] = (uint8_t)(f[0] & 1);
    c1[i] = (uint8_t)(f[1] & 1);
  }
  lp.na = (uint32_t)NA;
  lp.np = (uint32_t)NP;
  lp.root = vid(root_var);
  lp.order.clear();
  lp.live = 0;
  if (lp.root >= (int64_t)NA) return;  // output is a PI or the constant
  lut_map(NA, NP, f0, f1, c0, c1, lp.root, cov);
}

// Evaluation order of the tables and its live count.
void order_luts(const Cone &c, const std::vector<uint32_t> &and_order, const LutCover &cov, LutProgram &lp) {
  const size_t NA = c.ands.size(), NP = c.pis.size();
  if (lp.root >= (int64_t)NA || cov.luts.empty()) return;
  // level of each table (leaves at 0)
  std::vector<uint32_t> lev(cov.luts.size(), 0);
  for (size_t i = 0; i < cov.luts.size(); i++) {
    uint32_t l = 0;
    for (int k = 0; k < cov.luts[i].n; k++) {
      const int32_t x = cov.luts[i].leaf[k];
      if (x < (int32_t)NA) l = std::max(l, lev[cov.index[x]] + 1);
    }
    lev[i] = l;
  }
  const size_t NV = NA + NP + 1;
  auto live_of = [&](const std::vector<LutCover::Lut> &ord) -> uint32_t {
    std::vector<uint32_t> uses(NV, 0);
    for (const auto &l : ord)
      for (int k = 0; k < l.n; k++) uses[l.leaf[k]]++;
    uses[lp.root]++;
    std::vector<uint8_t> alive(NV, 0);
    uint32_t live = 0, peak = 0;
    for (const auto &l : ord) {
      for (int k = 0; k < l.n; k++)
        if (!alive[l.leaf[k]]) { alive[l.leaf[k]] = 1; live++; }  // PI / constant first read
      peak = std::max(peak, live + 1);
      for (int k = 0; k < l.n; k++)
        if (--uses[l.leaf[k]] == 0) { alive[l.leaf[k]] = 0; live--; }
      alive[l.node] = 1;
      live++;
      peak = std::max(peak, live);
    }
    return peak;
  };
  std::vector<std::vector<LutCover::Lut>> cands;
  // (1) post-order from the root, deeper leaf first
  {
    std::vector<LutCover::Lut> ord;
    std::vector<uint8_t> st(cov.luts.size(), 0);
    std::vector<std::pair<int32_t, uint8_t>> stack{{cov.index[lp.root], 0}};
    while (!stack.empty()) {
      auto &top = stack.back();
      const int32_t i = top.first;
      if (top.second == 0) {
        if (st[i]) { stack.pop_back(); continue; }
        st[i] = 1;
        top.second = 1;
        std::vector<int32_t> kids;
        for (int k = 0; k < cov.luts[i].n; k++) {
          const int32_t x = cov.luts[i].leaf[k];
          if (x < (int32_t)NA && !st[cov.index[x]]) kids.push_back(cov.index[x]);
        }
        // the deepest child is finished first, so it is pushed last
        std::sort(kids.begin(), kids.end(), [&](int32_t a, int32_t b) { return lev[a] < lev[b]; });
        for (int32_t k : kids) stack.push_back({k, 0});
      } else {
        stack.pop_back();
        if (st[i] == 1) {
          st[i] = 2;
          ord.push_back(cov.luts[i]);
        }
      }
    }
    cands.push_back(std::move(ord));
  }
  // (2) ascending variable order (the AIG's own topological order)
  cands.push_back(cov.luts);
  // (3) the order of the cone's slot program (the AIG order with the fewest slots)
  if (!and_order.empty()) {
    std::vector<LutCover::Lut> ord;
    for (uint32_t i : and_order)
      if (cov.index[i] >= 0) ord.push_back(cov.luts[cov.index[i]]);
    cands.push_back(std::move(ord));
  }
  size_t bi = 0;
  uint32_t bl = UINT32_MAX;
  for (size_t i = 0; i < cands.size(); i++) {
    const uint32_t l = live_of(cands[i]);
    if (l < bl) { bl = l; bi = i; }
  }
  lp.order = std::move(cands[bi]);
  lp.live = bl;
}

uint64_t fnv1a(const void *data, size_t len, uint64_t h) {
  const uint8_t *b = (const uint8_t *)data;
  for (size_t i = 0; i < len; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

namespace {
// The cone facts of a miter whose kernel was found, kept with a copy of its
// fanin array: a later call on byte-identical input skips cone extraction
// and hashing (a sequential compare instead), then asks for the kernel again.
struct ConeMemo {
  const uint32_t *fanins = nullptr;
  uint32_t num_pis = 0, num_ands = 0, out_lit = 0;
  std::vector<uint32_t> copy;  // 2 * num_ands fanin literals
  uint64_t hash = 0, hash2 = 0;
  std::vector<uint32_t> support;  // 0-based PI indices
  uint32_t cone_ands = 0;
  int64_t root_vid = -1;
};
constexpr size_t kConeMemos = 4;

// The elided program of a cone whose kernel the probe found.
void elided_program(uint32_t n, const uint32_t *support, uint32_t cone_ands, uint32_t out_lit, uint64_t hash,
                    uint64_t hash2, int64_t root_vid, const KernelFacts &facts, Program &out) {
  Program p;
  p.n = n;
  p.support.assign(support, support + n);
  p.cone_ands = cone_ands;
  p.out_compl = out_lit & 1;
  p.hash = hash;
  p.hash2 = hash2;
  p.num_slots = facts.num_slots;
  p.order = facts.order;
  p.num_records = facts.num_records;
  p.slots_elided = true;
  p.lut.na = cone_ands;
  p.lut.np = n;
  p.lut.root = root_vid;
  p.lut.count = facts.luts;
  p.lut.live = facts.live;
  p.lut.elided = true;
  out = std::move(p);
}
}  // namespace

int compact_cone(const MiterView &m, uint32_t max_pis, CompactMiter &out) {
  thread_local std::vector<uint8_t> mark;
  thread_local std::vector<int32_t> dense;
  Cone c;
  int rc = extract_cone(m, mark, c);
  if (rc) return rc;
  if (c.pis.size() > max_pis || c.pis.size() > 63) return LEC_ES_ETOOBIG;
  ConeIndex ix(c, dense, (uint64_t)m.num_pis + m.num_ands);
  const uint32_t n = (uint32_t)c.pis.size(), na = (uint32_t)c.ands.size();
  // value id -> compact variable: ANDs (ids 0..na-1) after the PIs (ids
  // na..na+n-1), the constant (id na+n) stays 0
  auto var_of = [&](uint32_t v) -> uint32_t {
    const int64_t id = ix.vid(v);
    if (id < (int64_t)na) return n + 1 + (uint32_t)id;
    if (id < (int64_t)(na + n)) return (uint32_t)(id - na) + 1;
    return 0;
  };
  out.num_pis = n;
  out.support.resize(n);
  for (uint32_t k = 0; k < n; k++) out.support[k] = c.pis[k] - 1;
  out.fanins.resize(2ull * na);
  for (uint32_t i = 0; i < na; i++) {
    const uint32_t *f = fanin_of(m, c.ands[i]);
    out.fanins[2ull * i] = var_of(f[0] >> 1) << 1 | (f[0] & 1u);
    out.fanins[2ull * i + 1] = var_of(f[1] >> 1) << 1 | (f[1] & 1u);
  }
  out.out_lit = var_of(m.out_lit >> 1) << 1 | (m.out_lit & 1u);
  return LEC_ES_OK;
}

int compile_program(const MiterView &m, uint32_t order, uint32_t max_pis, Program &out, const KernelProbe *probe) {
  thread_local std::vector<uint8_t> mark;
  thread_local std::vector<int32_t> dense;
  thread_local std::vector<ConeMemo> memos;
  if (probe && m.fanins) {
    for (size_t i = 0; i < memos.size(); i++) {
      ConeMemo &e = memos[i];
      if (e.fanins != m.fanins || e.num_pis != m.num_pis || e.num_ands != m.num_ands || e.out_lit != m.out_lit ||
          memcmp(e.copy.data(), m.fanins, 8ull * m.num_ands) != 0)
        continue;
      if (e.support.size() > max_pis) return LEC_ES_ETOOBIG;
      KernelFacts facts;
      if (!probe->have_kernel(probe->arg, e.hash, e.hash2, (uint32_t)e.support.size(), e.cone_ands, &facts)) break;
      elided_program((uint32_t)e.support.size(), e.support.data(), e.cone_ands, m.out_lit, e.hash, e.hash2,
                     e.root_vid, facts, out);
      if (i) std::rotate(memos.begin(), memos.begin() + i, memos.begin() + i + 1);  // most recent first
      return LEC_ES_OK;
    }
  }
  Cone c;
  int rc = extract_cone(m, mark, c);
  if (rc) return rc;
  if (c.pis.size() > max_pis || c.pis.size() > 63) return LEC_ES_ETOOBIG;
  ConeIndex ix(c, dense, (uint64_t)m.num_pis + m.num_ands);
  const uint32_t root_var = m.out_lit >> 1;
  // the cone's structure: fanin value ids and complements of its ANDs in
  // ascending order, the output's value id and complement, the support size;
  // hashed twice, by FNV and by a multiply-xorshift chain, so that a kernel
  // or resident program found by the first is used only if the second
  // agrees too
  uint64_t chash = 1469598103934665603ull, chash2 = 0x243F6A8885A308D3ull;
  {
    const uint32_t head[2] = {(uint32_t)c.pis.size(), (uint32_t)c.ands.size()};
    chash = fnv1a(head, sizeof(head), chash);
    std::vector<uint32_t> row(2 * c.ands.size());
    for (size_t i = 0; i < c.ands.size(); i++) {
      const uint32_t *f = fanin_of(m, c.ands[i]);
      row[2 * i] = (uint32_t)ix.vid(f[0] >> 1) << 1 | (f[0] & 1u);
      row[2 * i + 1] = (uint32_t)ix.vid(f[1] >> 1) << 1 | (f[1] & 1u);
    }
    for (uint32_t w : row) chash = (chash ^ w) * 0x100000001B3ull;  // word-wise FNV step
    chash ^= chash >> 29;
    const uint32_t tail[1] = {(uint32_t)ix.vid(root_var) << 1 | (m.out_lit & 1u)};
    chash = fnv1a(tail, sizeof(tail), chash);
    auto mix = [](uint64_t h, uint64_t w) {
      h = (h ^ (w + 0x9E3779B97F4A7C15ull)) * 0xFF51AFD7ED558CCDull;
      return h ^ (h >> 32);
    };
    chash2 = mix(chash2, (uint64_t)head[0] << 32 | head[1]);
    for (size_t i = 0; i + 1 < row.size(); i += 2) chash2 = mix(chash2, (uint64_t)row[i] << 32 | row[i + 1]);
    chash2 = mix(chash2, tail[0]);
    chash2 = (chash2 ^ (chash2 >> 29)) * 0xC4CEB9FE1A85EC53ull;
    chash2 ^= chash2 >> 32;
  }
  KernelFacts facts;
  if (probe && probe->have_kernel(probe->arg, chash, chash2, (uint32_t)c.pis.size(), (uint32_t)c.ands.size(), &facts)) {
    std::vector<uint32_t> sup(c.pis.size());
    for (size_t k = 0; k < c.pis.size(); k++) sup[k] = c.pis[k] - 1;
    const int64_t root_vid = ix.vid(root_var);
    // remember it when the cone is most of the graph (the compare then costs
    // about what extraction would)
    if (m.fanins && m.num_ands <= (1u << 20) && (uint64_t)m.num_ands <= 4ull * c.ands.size() + 64) {
      ConeMemo e;
      e.fanins = m.fanins;
      e.num_pis = m.num_pis;
      e.num_ands = m.num_ands;
      e.out_lit = m.out_lit;
      e.copy.assign(m.fanins, m.fanins + 2ull * m.num_ands);
      e.hash = chash;
      e.hash2 = chash2;
      e.support = sup;
      e.cone_ands = (uint32_t)c.ands.size();
      e.root_vid = root_vid;
      memos.insert(memos.begin(), std::move(e));
      if (memos.size() > kConeMemos) memos.pop_back();
    }
    elided_program((uint32_t)sup.size(), sup.data(), (uint32_t)c.ands.size(), m.out_lit, chash, chash2, root_vid, facts,
                   out);
    return LEC_ES_OK;
  }
  std::vector<uint32_t> level;
  order_levels(m, c, ix, level);

  // level and greedy orders never beat these two on datapath cones; they stay
  // available on request
  const uint32_t cands_auto[2] = {LEC_ES_ORDER_DFS, LEC_ES_ORDER_VAR};
  std::vector<uint32_t> tried;
  if (order == LEC_ES_ORDER_AUTO) tried.assign(cands_auto, cands_auto + 2);
  else if (order <= LEC_ES_ORDER_GREEDY) tried.push_back(order);
  else return LEC_ES_EINVAL;

  std::vector<Program> cand(tried.size());
  std::vector<std::vector<uint32_t>> base(tried.size());  // each order before separate_reads
  std::vector<int> crc(tried.size(), LEC_ES_OK);
  auto run_order = [&](size_t t) {
    const uint32_t o = tried[t];
    std::vector<uint32_t> ord;
    if (o == LEC_ES_ORDER_DFS) order_dfs(m, c, ix, level, root_var, ord);
    else if (o == LEC_ES_ORDER_VAR) order_var(c, ord);
    else if (o == LEC_ES_ORDER_GREEDY) order_greedy(m, c, ix, root_var, ord);
    else order_level(level, ord);
    if (ord.size() != c.ands.size()) {
      crc[t] = LEC_ES_EINVAL;
      return;
    }
    base[t].reserve(ord.size());
    for (uint32_t i : ord) base[t].push_back((uint32_t)i);
    if (c.ands.size() >= kStepMinAnds) {
      separate_reads(m, c, ix, (uint32_t)kInterpStep - 1, ord);
      crc[t] = assign_slots(m, c, ix, ord, root_var, (uint32_t)kInterpStep, cand[t]);
      // a narrow cone that needs many run breaks runs better with forwarding
      const size_t breaks = cand[t].recs.size() - c.ands.size() -
                            (size_t)std::count_if(cand[t].recs.begin(), cand[t].recs.end(),
                                                  [](const Rec &r) { return r.op >= 4 && r.pad != kRecBreak; });
      if (crc[t] || breaks * kMaxBreakShare <= c.ands.size()) {
        cand[t].order = o;
        return;
      }
      cand[t] = Program{};
    }
    crc[t] = assign_slots(m, c, ix, base[t], root_var, 1u, cand[t]);
    cand[t].order = o;
  };
  for (size_t t = 0; t < tried.size(); t++) run_order(t);
  size_t bi = tried.size();
  for (size_t t = 0; t < tried.size(); t++) {
    if (crc[t]) return crc[t];
    if (bi == tried.size() || cand[t].num_slots < cand[bi].num_slots) bi = t;
  }
  Program best = std::move(cand[bi]);
  best.n = (uint32_t)c.pis.size();
  best.support.resize(c.pis.size());
  for (size_t k = 0; k < c.pis.size(); k++) best.support[k] = c.pis[k] - 1;
  best.cone_ands = (uint32_t)c.ands.size();
  best.out_compl = m.out_lit & 1;
  if (best.num_slots == 0) best.num_slots = 1;
  best.hash = chash;
  best.hash2 = chash2;
  best.num_records = (uint32_t)best.recs.size();
  if (!probe || !probe->want_cover || probe->want_cover(probe->arg, best.n, best.cone_ands)) {
    // the table cover (independent of the slot order), then its evaluation
    // order, one candidate of which follows the chosen slot order
    LutProgram lp;
    LutCover cov;
    cover_cone(m, c, ix, root_var, lp, cov);
    order_luts(c, base[bi], cov, lp);
    lp.count = (uint32_t)lp.order.size();
    best.lut = std::move(lp);
  }
  out = std::move(best);
  return LEC_ES_OK;
}

void encode_w(const Program &g, int block, std::vector<XRec> &recs, std::vector<XLoad> &loads, uint32_t &out_off,
              bool breaks) {
  const uint32_t unit = (uint32_t)block * kLaneBytes;  // bytes between consecutive slots of one thread
  recs.clear();
  loads.clear();
  recs.reserve(g.recs.size());
  for (const Rec &r : g.recs) {
    if (r.op < 4) {
      recs.push_back(XRec{r.a * unit, r.b * unit, r.dst * unit, (uint32_t)(r.op & 3u)});
    } else if (breaks || r.pad != kRecBreak) {
      loads.push_back(XLoad{(uint32_t)recs.size(), r.dst * unit, r.op == OP_PI ? (uint32_t)r.a : 63u, 0u});
    }
  }
  out_off = g.out_slot * unit;
}

}  // namespace lec
