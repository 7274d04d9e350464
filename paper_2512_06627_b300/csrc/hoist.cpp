// hoist.cpp -- tables of the specialised kernel evaluated once per grab.
//
// A warp takes grabs of rep passes; grab q covers the chunks [q*G, (q+1)*G),
// G = 32 * rep (a power of two), so within a grab a chunk index differs only
// in its low log2(G) bits: bits 0..4 are the lane (support PIs 5..9, fixed
// per thread), bits 5..log2(G)-1 are the pass (the only PIs that change from
// pass to pass), and every higher bit is the grab's.  A table none of whose
// inputs depends on the pass PIs has the same value in every pass of a grab,
// so it can be evaluated once per grab -- the same Boolean function of the
// same inputs, fewer instructions.  Keeping such a value across the passes
// costs a register (or a shared-memory slot), so only so many hoisted values
// may be read by the per-pass code; a hoisted table whose every reader is
// hoisted costs nothing.  The hoisted set is grown by whole fanin cones of
// invariant tables at the edge of the invariant region, greedily by tables
// removed per value read, while each step removes at least one table per
// value, up to the budget.
//
// The passes of a grab may also run as nested loops, each over a group of
// the pass PIs.  A table that reads no PI of a deeper loop (and only values
// of its own or outer levels) then runs once per iteration of its loop.
// Each level's set is planned the same way, starting from the set of the
// level outside it, against the PIs of the deeper loops; a value stays live
// across the deeper loops if it is read below its own level.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "es_internal.h"

namespace lec {

void plan_hoist(const LutProgram &lp, uint64_t pass_pis, uint32_t budget, std::vector<uint8_t> &hoisted,
                uint32_t *roots_out) {
  plan_hoist_from(lp, pass_pis, budget, std::vector<uint8_t>(), hoisted, roots_out);
}

void plan_hoist_from(const LutProgram &lp, uint64_t pass_pis, uint32_t budget, const std::vector<uint8_t> &base_in,
                     std::vector<uint8_t> &hoisted, uint32_t *roots_out) {
  const uint32_t NA = lp.na, NP = lp.np;
  const size_t NL = lp.order.size();
  std::vector<uint8_t> base = base_in;
  base.resize(NL, 0);
  hoisted = base;
  if (roots_out) *roots_out = 0;
  if (NL == 0 || lp.root < 0 || lp.root >= (int64_t)NA) return;
  std::vector<int32_t> pos(NA, -1);  // AND value id -> table index
  for (size_t i = 0; i < NL; i++) pos[lp.order[i].node] = (int32_t)i;
  // invariant over the passes of a grab: constants, PIs outside the pass
  // range, tables of invariant inputs
  std::vector<uint8_t> inv(NL, 0);
  auto leaf_inv = [&](int32_t v) -> bool {
    if (v < 0) return true;
    if ((uint32_t)v >= NA) {
      const uint32_t k = (uint32_t)v - NA;
      return k >= NP || !((pass_pis >> k) & 1u);  // k == NP is the constant
    }
    return pos[v] >= 0 && inv[pos[v]];
  };
  for (size_t i = 0; i < NL; i++) {
    bool ok = true;
    for (int k = 0; k < lp.order[i].n; k++) ok = ok && leaf_inv(lp.order[i].leaf[k]);
    inv[i] = ok;
  }
  // readers of each table (table indices; the output counts as a reader
  // that is never hoisted)
  std::vector<std::vector<int32_t>> readers(NL);
  for (size_t i = 0; i < NL; i++)
    for (int k = 0; k < lp.order[i].n; k++) {
      const int32_t v = lp.order[i].leaf[k];
      if (v >= 0 && (uint32_t)v < NA && pos[v] >= 0) readers[pos[v]].push_back((int32_t)i);
    }
  const int32_t out_t = pos[lp.root];
  // A hoisted set is the fanin cone of its roots (every table a hoisted
  // table reads is hoisted too); its cost is the number of hoisted values
  // the per-pass code reads (a table outside the set, or the output), plus
  // the base's values read outside the base (live across the loop too).
  std::vector<uint8_t> in = base, trial(NL, 0), base_read(NL, 0);
  for (size_t i = 0; i < NL; i++) {
    if (!base[i]) continue;
    bool read = (int32_t)i == out_t;
    for (int32_t r : readers[i]) read = read || !base[r];
    base_read[i] = read;
  }
  auto grow = [&](std::vector<uint8_t> &h, int32_t r) -> uint32_t {  // add r's cone, return tables added
    uint32_t added = 0;
    std::vector<int32_t> st{r};
    while (!st.empty()) {
      const int32_t i = st.back();
      st.pop_back();
      if (h[i]) continue;
      h[i] = 1;
      added++;
      for (int k = 0; k < lp.order[i].n; k++) {
        const int32_t v = lp.order[i].leaf[k];
        if (v >= 0 && (uint32_t)v < NA && pos[v] >= 0 && !h[pos[v]]) st.push_back(pos[v]);
      }
    }
    return added;
  };
  auto cost = [&](const std::vector<uint8_t> &h) -> uint32_t {
    uint32_t c = 0;
    for (size_t i = 0; i < NL; i++) {
      if (!h[i]) continue;
      bool read = (int32_t)i == out_t || base_read[i];
      for (int32_t r : readers[i]) read = read || !h[r];
      c += read;
    }
    return c;
  };
  // candidate roots: invariant tables read by a table that is not
  // invariant, or the output itself when it is invariant
  std::vector<int32_t> cand;
  for (size_t i = 0; i < NL; i++) {
    if (!inv[i] || base[i]) continue;
    bool edge = (int32_t)i == out_t;
    for (int32_t r : readers[i]) edge = edge || !inv[r];
    if (edge) cand.push_back((int32_t)i);
  }
  uint32_t have_cost = cost(in), roots = 0;
  std::vector<uint8_t> used(cand.size(), 0);
  for (;;) {
    int best = -1;
    uint32_t best_gain = 0, best_cost = 0;
    for (size_t c = 0; c < cand.size(); c++) {
      if (used[c] || in[cand[c]]) continue;
      trial = in;
      const uint32_t gain = grow(trial, cand[c]);
      const uint32_t cc = cost(trial);
      if (cc > budget) continue;
      // at least one table removed from every pass per extra value read per
      // pass (a cone that absorbs earlier roots can lower the count)
      const uint32_t dc = cc > have_cost ? cc - have_cost : 0;
      if (gain < std::max<uint32_t>(1, dc)) continue;
      if (best < 0 || gain * std::max<uint32_t>(1, best_cost) > best_gain * std::max<uint32_t>(1, dc)) {
        best = (int)c;
        best_gain = gain;
        best_cost = dc;
      }
    }
    if (best < 0) break;
    used[best] = 1;
    grow(in, cand[best]);
    have_cost = cost(in);
    roots++;
  }
  hoisted = in;
  if (roots_out) *roots_out = have_cost;
}

// support PIs each table depends on
std::vector<uint64_t> table_support(const LutProgram &lp) {
  const uint32_t NA = lp.na, NP = lp.np;
  const size_t NL = lp.order.size();
  std::vector<int32_t> pos(NA, -1);
  for (size_t i = 0; i < NL; i++) pos[lp.order[i].node] = (int32_t)i;
  std::vector<uint64_t> dep(NL, 0);
  for (size_t i = 0; i < NL; i++)
    for (int q = 0; q < lp.order[i].n; q++) {
      const int32_t v = lp.order[i].leaf[q];
      if (v < 0) continue;
      if ((uint32_t)v >= NA) {
        if ((uint32_t)v - NA < NP && (uint32_t)v - NA < 64) dep[i] |= 1ull << ((uint32_t)v - NA);
      } else if (pos[v] >= 0) {
        dep[i] |= dep[pos[v]];
      }
    }
  return dep;
}

uint64_t least_influential_pis(const LutProgram &lp, uint32_t k) {
  const uint32_t NP = lp.np;
  const size_t NL = lp.order.size();
  if (NP <= 10 || k == 0) return 0;
  const std::vector<uint64_t> dep = table_support(lp);
  std::vector<std::pair<uint64_t, uint32_t>> infl;
  for (uint32_t p = 10; p < NP && p < 64; p++) {
    uint64_t c = 0;
    for (size_t i = 0; i < NL; i++) c += (dep[i] >> p) & 1u;
    infl.push_back({c, p});
  }
  std::sort(infl.begin(), infl.end());
  uint64_t m = 0;
  for (uint32_t i = 0; i < k && i < infl.size(); i++) m |= 1ull << infl[i].second;
  return m;
}

std::vector<uint64_t> choose_pass_groups(const LutProgram &lp, uint64_t pass_pis, int mode, double *score_out) {
  const uint32_t k = (uint32_t)__builtin_popcountll(pass_pis);
  std::vector<uint32_t> bits;  // pass PIs in ascending order
  for (uint32_t p = 0; p < 64; p++)
    if ((pass_pis >> p) & 1u) bits.push_back(p);
  // tables by the pass PIs they depend on
  const std::vector<uint64_t> dep = table_support(lp);
  std::vector<uint64_t> count(1u << k, 0);
  for (uint64_t d : dep) {
    uint32_t m = 0;
    for (uint32_t i = 0; i < k; i++)
      if ((d >> bits[i]) & 1u) m |= 1u << i;
    count[m]++;
  }
  if (score_out) {  // one loop: grab-level tables once, the others 2^k times
    *score_out = 0;
    for (uint32_t m = 0; m < (1u << k); m++) *score_out += (double)count[m] * (m ? (double)(1u << k) : 1.0);
  }
  if (k < 2 || lp.order.empty() || mode == 0) return {pass_pis};
  if (mode == 3) {  // one loop per pass PI, lowest outermost
    std::vector<uint64_t> g;
    for (uint32_t p : bits) g.push_back(1ull << p);
    return g;
  }
  // every ordered partition of the pass PIs into at most four groups (a
  // group index per PI, groups 0..L-1 all used); evaluations per grab: a
  // table runs once per iteration of the loop of its deepest group, 2^(PIs
  // in that group and the groups outside it) times
  const uint32_t G = std::min<uint32_t>(k, 4);
  std::vector<uint32_t> gi(k, 0), best_gi(k, 0), deep(1u << k, 0);
  double best_score = -1;
  uint32_t best_L = 1;
  for (;;) {
    uint32_t L = 0;
    for (uint32_t i = 0; i < k; i++) L = std::max(L, gi[i] + 1);
    uint32_t used[4] = {0, 0, 0, 0}, prefix[5] = {0, 0, 0, 0, 0};
    for (uint32_t i = 0; i < k; i++) used[gi[i]]++;
    bool ok = true;
    for (uint32_t l = 0; l < L; l++) ok = ok && used[l] > 0;
    if (ok && !(mode == 2 && L < 2)) {
      for (uint32_t l = 0; l < L; l++) prefix[l + 1] = prefix[l] + used[l];
      double e = (double)count[0];
      for (uint32_t m = 1; m < (1u << k); m++) {  // deepest group of m from m without its lowest PI
        const uint32_t i = (uint32_t)__builtin_ctz(m);
        deep[m] = std::max(deep[m & (m - 1)], gi[i]);
        if (count[m]) e += (double)count[m] * (double)(1u << prefix[deep[m] + 1]);
      }
      // a loop level costs registers and loop overhead: take one only for
      // a clear saving
      const double score = e * (1.0 + 0.03 * (L - 1));
      if (best_score < 0 || score < best_score) {
        best_score = score;
        best_gi = gi;
        best_L = L;
      }
    }
    uint32_t i = 0;  // next assignment (base-G counter)
    while (i < k && ++gi[i] == G) gi[i++] = 0;
    if (i == k) break;
  }
  std::vector<uint64_t> g(best_L, 0);
  for (uint32_t i = 0; i < k; i++) g[best_gi[i]] |= 1ull << bits[i];
  if (score_out) *score_out = best_score;
  return g;
}

}  // namespace lec
