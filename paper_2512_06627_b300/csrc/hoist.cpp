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
// The passes of a grab may also run as two nested loops: an outer loop over
// some of the pass PIs and an inner loop over the rest.  A table that reads
// only outer pass PIs (and grab-level values) then runs once per outer
// iteration.  Its set is planned the same way, starting from the grab-level
// set, against the inner pass PIs; a value stays live across the inner loop
// if it is read below its own level.
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

namespace {
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
}  // namespace

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

uint64_t choose_outer_pis(const LutProgram &lp, uint64_t pass_pis, bool force) {
  const uint32_t k = (uint32_t)__builtin_popcountll(pass_pis);
  if (k < 2 || lp.order.empty()) return 0;
  const std::vector<uint64_t> dep = table_support(lp);
  std::vector<uint32_t> bits;  // pass PIs in ascending order
  for (uint32_t p = 0; p < 64; p++)
    if ((pass_pis >> p) & 1u) bits.push_back(p);
  // table evaluations per grab: grab-level tables once, outer-level ones
  // 2^|outer| times, the rest 2^k times (hoisting limits ignored)
  auto evals = [&](uint64_t outer) -> uint64_t {
    uint64_t e = 0;
    const uint64_t no = 1ull << __builtin_popcountll(outer), nk = 1ull << k;
    for (uint64_t d : dep) {
      const uint64_t pd = d & pass_pis;
      e += pd == 0 ? 1 : (pd & ~outer) == 0 ? no : nk;
    }
    return e;
  };
  const uint64_t flat = evals(0);
  uint64_t best = 0, best_e = flat;
  for (uint32_t sub = 1; sub + 1 < (1u << k); sub++) {  // proper, non-empty subsets
    uint64_t outer = 0;
    for (uint32_t i = 0; i < k; i++)
      if ((sub >> i) & 1u) outer |= 1ull << bits[i];
    const uint64_t e = evals(outer);
    if (e < best_e) {
      best_e = e;
      best = outer;
    }
  }
  if (force) return best ? best : pass_pis & (~pass_pis + 1);  // else the lowest pass PI alone
  // a second loop level pays only for a clear saving
  return best_e * 100 <= flat * 95 ? best : 0;
}

}  // namespace lec
