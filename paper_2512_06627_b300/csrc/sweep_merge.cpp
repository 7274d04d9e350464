// sweep_merge.cpp -- the sweeping loop with exact simulation as its engine.
//
// The standard sweeping flow (§2.3): (1) random simulation finds potentially
// equivalent node pairs, (2) each pair is checked, here by ES, (3) proven
// pairs are merged, and the process repeats on the smaller circuit.  The
// sub-miter of a pair is local, in the way the paper builds its sub-miters
// (§3.2: the pair's fanin cones with the preceding logic merged): both cones
// are walked down from the pair and stop where they meet, and the meeting
// nodes become free inputs.  A check with free inputs over-approximates, so
// an EQUIVALENT answer is a proof; a counterexample may be spurious and only
// leaves the pair unmerged.  Merging plus structural hashing makes later
// pairs, and finally the miter's output, collapse, which proves miters whose
// output has far too many PIs to enumerate (64-PI multipliers).
//
// Per round, on the working AIG g (the output's cone, structurally hashed)
// (a round after one that refuted at most a tenth of its pairs skips the
// first two steps and takes that round's uncut candidates, mapped into the
// rebuilt graph -- no random words of its own, so no new refutations):
//   * simulate every node on fresh random words (GPU, sweep.cu) with
//     phase-normalised hashes; a nonzero output signature is a real
//     counterexample and ends the sweep;
//   * group nodes (and the constant and PIs) into classes of equal signature
//     up to complement; each member is paired with its class's lowest
//     variable;
//   * cut each pair's local region (highest level first; a node reached
//     from both sides is a meeting point and a leaf) within the node and
//     leaf limits, copy every region into one AIG whose PIs are the leaves,
//     add the XOR of the pair, and check all of them in one batch (GPU);
//   * rebuild g with every proven member replaced by its representative,
//     folding constants and hashing structure.
// When the rounds stop merging, the output is decided by its own ES check if
// its support is small enough, else the verdict is UNDECIDED (SAT and BDD
// engines are not part of this library).
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <queue>
#include <unordered_map>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

namespace lec {
namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
// Consecutive too-wide regions that end a round's cutting: the pairs above
// the merged frontier fail until lower pairs merge.  128, 256 and 1,024 all
// prove the 32x32 array and Booth pairs in the same 35 and 6 rounds; 128
// bounds a round's trailing failed cuts at 128 instead of 1,024.
constexpr uint32_t kMissRun = 128;
constexpr uint32_t kNoMeet = 48;     // region ANDs walked before the two cones must have met

struct Graph {
  uint32_t P = 0;              // PIs are variables 1..P, the constant is 0
  std::vector<uint32_t> fan;   // two literals per AND, ANDs in topological order
  uint32_t out = 0;            // output literal
  std::vector<uint32_t> orig;  // per variable: an input variable with the same function
  uint32_t vars() const { return P + 1 + (uint32_t)(fan.size() / 2); }
  uint32_t ands() const { return (uint32_t)(fan.size() / 2); }
};

// Structural hashing with constant folding: AND(a, b) for literals a, b.
struct Strash {
  Graph &g;
  std::unordered_map<uint64_t, uint32_t> table;
  explicit Strash(Graph &gg) : g(gg) { table.reserve(gg.fan.size()); }
  uint32_t mk(uint32_t a, uint32_t b, uint32_t origin) {
    if (a > b) std::swap(a, b);
    if (a == 0) return 0;          // x & 0
    if (a == 1) return b;          // x & 1
    if (a == b) return a;          // x & x
    if ((a ^ 1u) == b) return 0;   // x & ~x
    const uint64_t key = (uint64_t)a << 32 | b;
    auto it = table.find(key);
    if (it != table.end()) return 2u * it->second;
    const uint32_t v = g.vars();
    g.fan.push_back(a);
    g.fan.push_back(b);
    g.orig.push_back(origin);
    table.emplace(key, v);
    return 2u * v;
  }
};

// g with the substitutions (subst[v] = replacement literal in g's numbering,
// from a lower variable) applied, then only the output's cone kept.  If
// vmap is given, (*vmap)[v] is the literal of g's variable v in the result,
// or kNone if v's function is no longer in the output's cone.
Graph rebuild(const Graph &g, const std::vector<uint32_t> &subst, std::vector<uint32_t> *vmap = nullptr) {
  Graph t;
  t.P = g.P;
  t.orig.assign(g.orig.begin(), g.orig.begin() + g.P + 1);
  const uint32_t V = g.vars();
  std::vector<uint32_t> map(V);
  for (uint32_t v = 0; v <= g.P; v++) map[v] = 2u * v;
  auto lit = [&](uint32_t l) { return map[l >> 1] ^ (l & 1u); };
  {
    Strash sh(t);
    for (uint32_t v = g.P + 1; v < V; v++) {
      if (!subst.empty() && subst[v] != kNone) {
        map[v] = lit(subst[v]);
        continue;
      }
      const uint32_t a = g.fan[2 * (v - g.P - 1)], b = g.fan[2 * (v - g.P - 1) + 1];
      map[v] = sh.mk(lit(a), lit(b), g.orig[v]);
    }
  }
  const uint32_t out = lit(g.out);
  // keep the output's cone, in the same (topological) order
  const uint32_t TV = t.vars();
  std::vector<uint8_t> keep(TV, 0);
  keep[out >> 1] = 1;
  for (uint32_t v = TV; v-- > t.P + 1;) {
    if (!keep[v]) continue;
    keep[t.fan[2 * (v - t.P - 1)] >> 1] = 1;
    keep[t.fan[2 * (v - t.P - 1) + 1] >> 1] = 1;
  }
  Graph r;
  r.P = t.P;
  r.orig.assign(t.orig.begin(), t.orig.begin() + t.P + 1);
  std::vector<uint32_t> ren(TV);
  for (uint32_t v = 0; v <= t.P; v++) ren[v] = v;
  for (uint32_t v = t.P + 1; v < TV; v++) {
    if (!keep[v]) continue;
    ren[v] = r.vars();
    const uint32_t a = t.fan[2 * (v - t.P - 1)], b = t.fan[2 * (v - t.P - 1) + 1];
    r.fan.push_back(2u * ren[a >> 1] | (a & 1u));
    r.fan.push_back(2u * ren[b >> 1] | (b & 1u));
    r.orig.push_back(t.orig[v]);
  }
  r.out = 2u * ren[out >> 1] | (out & 1u);
  if (vmap) {
    vmap->assign(V, kNone);
    for (uint32_t v = 0; v < V; v++) {
      const uint32_t tv = map[v] >> 1;
      if (tv <= t.P || keep[tv]) (*vmap)[v] = 2u * ren[tv] | (map[v] & 1u);
    }
  }
  return r;
}

// splitmix64-seeded xoshiro256** words for the simulation inputs.
struct Rng {
  uint64_t s[4];
  explicit Rng(uint64_t seed) {
    for (int i = 0; i < 4; i++) {
      seed += 0x9E3779B97F4A7C15ull;
      uint64_t z = seed;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      s[i] = z ^ (z >> 31);
    }
  }
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
  }
};

// Local region of a pair: AND variables (ascending) and leaves (ascending).
struct Region {
  uint32_t rep = 0, mem = 0, phase = 0;
  std::vector<uint32_t> ands, leaves;
};

// Walk down from rep and mem, highest level first (a node's fanouts in the
// region are all seen before it); a node reached from both sides or a PI is
// a leaf, the constant stays the constant.  Then leaves are opened, highest
// level first, while that does not add leaves (a leaf whose fanins are in
// the region, or one of them is, becomes internal), so a leaf is not a free
// copy of logic over other leaves -- the main source of spurious
// counterexamples.  False if the region exceeds the limits.
typedef std::vector<std::pair<uint32_t, uint32_t>> Heap;  // (level, var) max-heaps, reused across calls

bool cut_region(const Graph &g, const std::vector<uint32_t> &level, std::vector<uint8_t> &mask,
                std::vector<uint32_t> &touched, Heap &pq, Heap &leafq, Region &r, uint32_t max_nodes,
                uint32_t max_leaves) {
  constexpr uint8_t kIn = 4, kLeaf = 8;  // mask bits beside the two sides
  pq.clear();
  leafq.clear();
  auto push = [](Heap &h, uint32_t l, uint32_t v) {
    h.push_back({l, v});
    std::push_heap(h.begin(), h.end());
  };
  auto pop = [](Heap &h) {
    std::pop_heap(h.begin(), h.end());
    const uint32_t v = h.back().second;
    h.pop_back();
    return v;
  };
  auto reach = [&](uint32_t v, uint8_t side) {
    if (!mask[v]) {
      touched.push_back(v);
      push(pq, level[v], v);
    }
    mask[v] |= side;
  };
  auto fanin = [&](uint32_t v, int e) { return g.fan[2 * (v - g.P - 1) + e] >> 1; };
  reach(r.rep, 1);
  reach(r.mem, 2);
  bool ok = true;
  uint32_t nand = 0, nleaf = 0;
  bool met = r.rep == 0;  // a constant pair has no meeting point to wait for
  while (!pq.empty() && ok) {
    const uint32_t v = pop(pq);
    if (v == 0) continue;  // the constant stays a constant
    if (v <= g.P || (mask[v] & 3) == 3) {
      met = met || (mask[v] & 3) == 3;
      mask[v] |= kLeaf;
      // opening leaves rarely removes many: give up early on wide cones
      if (++nleaf > 2 * max_leaves + 4) ok = false;
      if (v > g.P) push(leafq, level[v], v);
      continue;
    }
    mask[v] |= kIn;
    if (++nand > max_nodes) ok = false;
    // cones that have not met after a few dozen nodes lie above the merged
    // frontier: their region would run to the node limit
    if (!met && nand > kNoMeet) ok = false;
    reach(fanin(v, 0), mask[v] & 3);
    reach(fanin(v, 1), mask[v] & 3);
  }
  // open leaves that cost no new leaf
  while (ok && !leafq.empty()) {
    const uint32_t v = pop(leafq);
    const uint32_t a = fanin(v, 0), b = fanin(v, 1);
    const int fresh = (a != 0 && !(mask[a] & (kIn | kLeaf))) + (b != 0 && a != b && !(mask[b] & (kIn | kLeaf)));
    if (fresh > 1) continue;
    mask[v] = (uint8_t)((mask[v] & ~kLeaf) | kIn);
    nleaf--;
    if (++nand > max_nodes) ok = false;
    for (uint32_t u : {a, b}) {
      if (u == 0 || (mask[u] & (kIn | kLeaf))) continue;
      if (!mask[u]) touched.push_back(u);
      mask[u] |= kLeaf;
      nleaf++;
      if (u > g.P) push(leafq, level[u], u);
    }
  }
  if (ok && nleaf <= max_leaves) {
    for (uint32_t v : touched) {
      if (mask[v] & kIn) r.ands.push_back(v);
      else if (mask[v] & kLeaf) r.leaves.push_back(v);
    }
  } else {
    ok = false;
  }
  for (uint32_t v : touched) mask[v] = 0;
  touched.clear();
  if (!ok) return false;
  std::sort(r.ands.begin(), r.ands.end());
  std::sort(r.leaves.begin(), r.leaves.end());
  return true;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace lec

using namespace lec;

extern "C" int lec_es_sweep(lec_es_ctx *c, const lec_es_miter *m, const lec_es_sweep_options *opt,
                            lec_es_sweep_result *out, uint64_t *cex_bits, uint32_t *merges, uint64_t merges_cap,
                            uint64_t *nmerges) {
  if (!c || !m || !out || (m->num_ands && !m->fanins)) return LEC_ES_EINVAL;
  const uint64_t V0 = (uint64_t)m->num_pis + m->num_ands + 1;
  if (V0 >= (1ull << 31) || (m->out_lit >> 1) >= V0) return LEC_ES_EINVAL;
  for (uint64_t a = 0; a < m->num_ands; a++)
    if ((m->fanins[2 * a] >> 1) >= m->num_pis + 1 + a || (m->fanins[2 * a + 1] >> 1) >= m->num_pis + 1 + a)
      return LEC_ES_EINVAL;
  const uint32_t nwords = opt && opt->sim_words ? opt->sim_words : 64;
  const uint32_t max_rounds = opt && opt->max_rounds ? opt->max_rounds : 512;
  const uint32_t max_leaves = std::min<uint32_t>(opt && opt->max_leaves ? opt->max_leaves : 16, 40);
  const uint32_t max_nodes = opt && opt->max_nodes ? opt->max_nodes : 128;
  const uint32_t final_pis = std::min<uint32_t>(opt && opt->final_max_pis ? opt->final_max_pis : 36, 63);
  const uint64_t seed = opt ? opt->seed : 0;
  const bool log = getenv("LEC_ES_SWEEP_LOG") != nullptr;  // per-round counts and host times
  const auto t_start = std::chrono::steady_clock::now();
  memset(out, 0, sizeof(*out));
  out->verdict = LEC_ES_UNDECIDED;
  const uint32_t cex_words = (m->num_pis + 63) / 64;
  if (cex_bits) memset(cex_bits, 0, 8ull * cex_words);
  uint64_t logged = 0;
  auto log_merge = [&](uint32_t mem, uint32_t rep, uint32_t phase) {
    if (merges && logged < merges_cap) {
      merges[3 * logged] = mem;
      merges[3 * logged + 1] = rep;
      merges[3 * logged + 2] = phase;
    }
    logged++;
  };
  try {
    Graph g;
    g.P = m->num_pis;
    g.fan.assign(m->fanins, m->fanins + 2ull * m->num_ands);
    g.out = m->out_lit;
    g.orig.resize(V0);
    for (uint64_t v = 0; v < V0; v++) g.orig[v] = (uint32_t)v;
    g = rebuild(g, {});
    out->ands_initial = g.ands();
    std::vector<uint64_t> words, sigs, hash;
    std::vector<uint32_t> level;
    std::vector<uint8_t> mask;
    std::vector<uint32_t> touched;
    Heap heap, heap2;
    uint32_t idle = 0;
    // candidates of the previous round that were not cut, in g's numbering;
    // a round that proved nearly all its pairs hands them on instead of
    // simulating again (its classes are still true: nothing was refuted)
    std::vector<Region> pending;
    bool reuse = false;
    for (uint32_t round = 0; round < max_rounds; round++) {
      if ((g.out >> 1) == 0) break;  // the output is a constant
      out->rounds = round + 1;
      const uint32_t V = g.vars();
      auto t0 = std::chrono::steady_clock::now();
      std::vector<Region> cands;
      if (reuse) {
        cands = std::move(pending);
        out->rounds_reused++;
      } else {
      // (1) random simulation
      Rng rng(seed ^ (0xA5A5A5A5ull + round * 0x100000001B3ull));
      words.resize((size_t)g.P * nwords);
      for (auto &w : words) w = rng.next();
      sigs.resize((size_t)V * nwords);
      hash.resize(V);
      int rc = simulate(c, g.P, g.ands(), g.fan.data(), words.data(), nwords, sigs.data(), hash.data(), nullptr, true);
      if (rc) return rc;
      out->sim_ms += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      auto row = [&](uint32_t v) { return &sigs[(size_t)v * nwords]; };
      {  // the output's signature: any 1 is a counterexample
        const uint64_t *o = row(g.out >> 1);
        const uint64_t f = (g.out & 1u) ? ~0ull : 0ull;
        for (uint32_t w = 0; w < nwords; w++) {
          const uint64_t x = o[w] ^ f;
          if (!x) continue;
          const int b = __builtin_ctzll(x);
          if (cex_bits)
            for (uint32_t k = 0; k < g.P; k++)
              if ((words[(size_t)k * nwords + w] >> b) & 1ull) cex_bits[k / 64] |= 1ull << (k % 64);
          out->verdict = LEC_ES_NONEQUIVALENT;
          out->decided_by = 1;
          out->ands_final = g.ands();
          out->host_ms += ms_since(t0);
          out->total_ms = ms_since(t_start);
          if (nmerges) *nmerges = logged;
          return LEC_ES_OK;
        }
      }
      // (2) classes of equal signatures up to complement; pairs with their
      // class's lowest variable
      std::vector<uint32_t> order(V);
      for (uint32_t v = 0; v < V; v++) order[v] = v;
      std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return hash[x] < hash[y]; });
      auto phase_of = [&](uint32_t v) { return (uint32_t)(row(v)[0] & 1ull); };
      auto same = [&](uint32_t x, uint32_t y) {
        const uint64_t f = (phase_of(x) ^ phase_of(y)) ? ~0ull : 0ull;
        const uint64_t *a = row(x), *b = row(y);
        for (uint32_t w = 0; w < nwords; w++)
          if ((a[w] ^ f) != b[w]) return false;
        return true;
      };
      for (size_t i = 0; i < order.size();) {
        size_t j = i + 1;
        while (j < order.size() && hash[order[j]] == hash[order[i]]) j++;
        if (j - i > 1) {
          std::vector<uint32_t> run(order.begin() + i, order.begin() + j);
          std::sort(run.begin(), run.end());
          std::vector<uint8_t> used(run.size(), 0);
          for (size_t p = 0; p < run.size(); p++) {
            if (used[p]) continue;
            for (size_t q = p + 1; q < run.size(); q++) {
              if (used[q] || run[q] <= g.P || !same(run[p], run[q])) continue;
              used[q] = 1;
              Region r;
              r.rep = run[p];
              r.mem = run[q];
              r.phase = phase_of(run[p]) ^ phase_of(run[q]);
              cands.push_back(std::move(r));
            }
          }
        }
        i = j;
      }
      }  // simulation and classes
      pending.clear();
      level.assign(V, 0);
      for (uint32_t v = g.P + 1; v < V; v++)
        level[v] = std::max(level[g.fan[2 * (v - g.P - 1)] >> 1], level[g.fan[2 * (v - g.P - 1) + 1] >> 1]) + 1;
      mask.assign(V, 0);
      // lowest pairs first; a long run of pairs whose regions are too wide
      // means the merged frontier is below them, so the rest wait for the
      // next round
      const double t_class = ms_since(t0);
      std::stable_sort(cands.begin(), cands.end(), [&](const Region &x, const Region &y) {
        return std::max(level[x.rep], level[x.mem]) < std::max(level[y.rep], level[y.mem]);
      });
      // lowest first; a long run of too-wide regions ends the round's cutting
      // (the merged frontier is below them; threads did not pay here: the
      // cuts are allocation-bound)
      std::vector<uint8_t> cut_ok(cands.size(), 0);
      {
        uint32_t misses = 0;
        for (size_t i = 0; i < cands.size() && misses < kMissRun; i++) {
          cut_ok[i] = cut_region(g, level, mask, touched, heap, heap2, cands[i], max_nodes, max_leaves) ? 1 : 0;
          misses = cut_ok[i] ? 0 : misses + 1;
        }
      }
      std::vector<Region> regions;
      for (size_t i = 0; i < cands.size(); i++) {
        if (cut_ok[i]) {
          regions.push_back(std::move(cands[i]));
        } else {
          out->pairs_skipped++;
          pending.push_back(std::move(cands[i]));
        }
      }
      if (regions.empty()) {
        out->host_ms += ms_since(t0);
        if (!reuse) break;
        reuse = false;  // the handed-on candidates all stay too wide: simulate afresh
        pending.clear();
        continue;
      }
      const double t_cut = ms_since(t0) - t_class;
      // (3) one AIG holding every local sub-miter: leaf i of a region is PI
      // i + 1, region ANDs are copied, the pair's XOR is the output
      uint32_t L = 0;
      for (const Region &r : regions) L = std::max<uint32_t>(L, (uint32_t)r.leaves.size());
      std::vector<uint32_t> bfan;
      std::vector<uint32_t> bout(regions.size());
      std::vector<uint32_t> map(V, kNone);
      uint32_t bv = L + 1;
      auto band = [&](uint32_t a, uint32_t b) {
        bfan.push_back(a);
        bfan.push_back(b);
        return 2u * bv++;
      };
      for (size_t i = 0; i < regions.size(); i++) {
        const Region &r = regions[i];
        map[0] = 0;
        for (size_t k = 0; k < r.leaves.size(); k++) map[r.leaves[k]] = 2u * (uint32_t)(k + 1);
        for (uint32_t v : r.ands) {
          const uint32_t a = g.fan[2 * (v - g.P - 1)], b = g.fan[2 * (v - g.P - 1) + 1];
          map[v] = band(map[a >> 1] ^ (a & 1u), map[b >> 1] ^ (b & 1u));
        }
        const uint32_t x = map[r.rep], y = map[r.mem] ^ r.phase;
        // x XOR y = ~(~(x & ~y) & ~(~x & y))
        const uint32_t p = band(x, y ^ 1u), q = band(x ^ 1u, y);
        bout[i] = band(p ^ 1u, q ^ 1u) ^ 1u;
        for (uint32_t v : r.leaves) map[v] = kNone;
        for (uint32_t v : r.ands) map[v] = kNone;
        map[0] = kNone;
      }
      std::vector<lec_es_miter> bm(regions.size());
      for (size_t i = 0; i < regions.size(); i++)
        bm[i] = lec_es_miter{L, (uint32_t)(bfan.size() / 2), bfan.data(), bout[i]};
      out->host_ms += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      std::vector<lec_es_result> br(regions.size());
      const int rc = lec_es_batch(c, bm.data(), bm.size(), br.data());
      if (rc) return rc;
      out->es_ms += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      // (4) merge the proven pairs and rebuild
      std::vector<uint32_t> subst(V, kNone);
      uint32_t proven = 0;
      for (size_t i = 0; i < regions.size(); i++) {
        out->pairs_checked++;
        if (br[i].verdict != LEC_ES_EQUIVALENT) {
          out->pairs_refuted++;
          continue;
        }
        const Region &r = regions[i];
        subst[r.mem] = 2u * r.rep | r.phase;
        log_merge(g.orig[r.mem], g.orig[r.rep], r.phase);
        proven++;
      }
      out->pairs_proven += proven;
      // the next round reuses the uncut candidates if this one refuted
      // (almost) nothing, mapped into the rebuilt graph: a pair whose two
      // sides became one node, or left the output's cone, drops out
      const bool next_reuse = proven && (uint64_t)proven * 10 >= (uint64_t)regions.size() * 9 && !pending.empty();
      if (proven) {
        std::vector<uint32_t> vmap;
        g = rebuild(g, subst, next_reuse ? &vmap : nullptr);
        if (next_reuse) {
          std::vector<uint8_t> taken(g.vars(), 0);  // a member takes one representative
          size_t k = 0;
          for (Region &r : pending) {
            uint32_t a = vmap[r.rep], b = vmap[r.mem];
            if (a == kNone || b == kNone || (a >> 1) == (b >> 1)) continue;
            if ((a >> 1) > (b >> 1)) std::swap(a, b);
            if ((b >> 1) <= g.P || taken[b >> 1]) continue;
            taken[b >> 1] = 1;
            Region nr;
            nr.rep = a >> 1;
            nr.mem = b >> 1;
            nr.phase = r.phase ^ (a & 1u) ^ (b & 1u);
            pending[k++] = std::move(nr);
          }
          pending.resize(k);
        }
      }
      reuse = next_reuse && !pending.empty();
      if (!reuse) pending.clear();
      const double t_merge = ms_since(t0);
      out->host_ms += t_merge;
      if (log)
        fprintf(stderr, "sweep round %u: vars %u candidates %zu regions %zu proven %u | class %.2f cut %.2f merge %.2f ms\n",
                round, V, cands.size(), regions.size(), proven, t_class, t_cut, t_merge);
      idle = proven ? 0 : idle + 1;
      if (idle >= 2) break;  // two rounds (two sets of random words) without a merge
    }
    out->ands_final = g.ands();
    if ((g.out >> 1) == 0) {
      if (g.out == 0) {
        out->verdict = LEC_ES_EQUIVALENT;
      } else {
        out->verdict = LEC_ES_NONEQUIVALENT;  // constant 1: every pattern fails, e.g. all zeros
      }
      out->decided_by = 0;
    } else {
      // the output's own exact check on the reduced circuit
      {  // PIs of the output's cone
        std::vector<uint8_t> in(g.vars(), 0);
        in[g.out >> 1] = 1;
        for (uint32_t v = g.vars(); v-- > g.P + 1;)
          if (in[v]) in[g.fan[2 * (v - g.P - 1)] >> 1] = in[g.fan[2 * (v - g.P - 1) + 1] >> 1] = 1;
        for (uint32_t v = 1; v <= g.P; v++) out->final_support += in[v];
      }
      lec_es_miter fm{g.P, g.ands(), g.fan.data(), g.out};
      lec_es_program_info info;
      int rc = out->final_support <= final_pis ? lec_es_compile(&fm, LEC_ES_ORDER_AUTO, &info, nullptr, 0)
                                                : LEC_ES_ETOOBIG;
      if (rc == LEC_ES_OK && info.n <= final_pis) {
        const auto t0 = std::chrono::steady_clock::now();
        lec_es_result r;
        rc = lec_es_check(c, &fm, &r);
        if (rc) return rc;
        out->es_ms += ms_since(t0);
        out->verdict = r.verdict;
        out->decided_by = 2;
        if (r.verdict == LEC_ES_NONEQUIVALENT && cex_bits)
          for (uint32_t k = 0; k < r.support_n; k++)
            if ((r.cex >> k) & 1ull) cex_bits[r.support[k] / 64] |= 1ull << (r.support[k] % 64);
      } else {
        out->decided_by = 3;
      }
    }
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  out->total_ms = ms_since(t_start);
  if (nmerges) *nmerges = logged;
  return LEC_ES_OK;
}
