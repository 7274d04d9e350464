// lutmap.cpp -- cover a cone with 3-input lookup tables (one LOP3 each).
//
// A 32-bit LOP3 computes any Boolean function of three 32-bit operands, so an
// AND-inverter cone can be evaluated with fewer instructions than ANDs by
// covering it with 3-input cuts: a full adder's sum and carry (nine ANDs in
// an AIG) become two LOP3s.  This is the XOR/majority compaction the paper
// obtains by converting the AIG to an XAG before instructionalising it (§2.1,
// §3.3), generalised to every 3-feasible cut.  Results are the same Boolean
// functions, so verdicts and counterexamples are unchanged.
//
// Method (standard cut-based technology mapping):
//   cuts      every node gets its trivial cut {v} plus the merges of its
//             fanins' cuts with at most three leaves (PIs, the constant or
//             ANDs), each with its 8-bit truth table over the sorted leaves;
//   selection area flow AF(v) = (1 + sum of AF(leaf) over the cut's AND
//             leaves) / fanout(v), best cut per node, then two rounds of
//             exact-area recovery against the current cover's references;
//   cover     the output's node and, recursively, the AND leaves of every
//             chosen cut.
// Truth-table convention: leaf i of a cut is variable x_i with the patterns
// x0 = 0xAA, x1 = 0xCC, x2 = 0xF0, so a table is also LOP3's immediate when
// the operands are passed as (x2, x1, x0).
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "es_internal.h"

namespace lec {

namespace {

struct Cut {
  uint8_t n = 0;
  uint8_t tt = 0;
  int32_t leaf[3] = {-1, -1, -1};  // value ids, ascending
};

// One bit per leaf (id mod 64): a merge whose union has more than three bits
// set has more than three leaves, so it is rejected without merging.
inline uint64_t sig_of(const Cut &c) {
  uint64_t s = 0;
  for (int k = 0; k < c.n; k++) s |= 1ull << (c.leaf[k] & 63);
  return s;
}

// Re-expressing a table over a superset of its leaves depends only on where
// each old leaf lands (3 positions of 0..2 and the old leaf count): 108
// placements x 256 tables, computed once.
struct ExpandTable {
  uint8_t t[4 * 27][256];
  ExpandTable() {
    for (int n = 0; n <= 3; n++)
      for (int code = 0; code < 27; code++) {
        const int pos[3] = {code % 3, (code / 3) % 3, code / 9};
        for (int tt = 0; tt < 256; tt++) {
          uint8_t out = 0;
          for (int m = 0; m < 8; m++) {
            int mm = 0;
            for (int i = 0; i < n; i++) mm |= ((m >> pos[i]) & 1) << i;
            out |= (uint8_t)(((tt >> mm) & 1) << m);
          }
          t[n * 27 + code][tt] = out;
        }
      }
  }
};
const ExpandTable kExpand;

// Truth table of a function over cut `from`, re-expressed over the leaves of
// `to` (from's leaves are a subset of to's).
inline uint8_t expand(uint8_t tt, const Cut &from, const Cut &to) {
  int code = 0, mul = 1;
  for (int i = 0; i < from.n; i++, mul *= 3) {
    int j = 0;
    while (to.leaf[j] != from.leaf[i]) j++;
    code += j * mul;
  }
  return kExpand.t[from.n * 27 + code][tt];
}

bool merge(const Cut &a, const Cut &b, Cut &out) {
  int32_t l[6];
  int n = 0, i = 0, j = 0;
  while (i < a.n || j < b.n) {
    int32_t x;
    if (j >= b.n || (i < a.n && a.leaf[i] < b.leaf[j])) x = a.leaf[i++];
    else if (i >= a.n || b.leaf[j] < a.leaf[i]) x = b.leaf[j++];
    else { x = a.leaf[i++]; j++; }
    if (n == 3) return false;
    l[n++] = x;
  }
  out.n = (uint8_t)n;
  for (int k = 0; k < 3; k++) out.leaf[k] = k < n ? l[k] : -1;
  return true;
}

// Drop leaves the table does not depend on (keeps cuts minimal).
void minimise(Cut &c) {
  static const uint8_t var[3] = {0xAA, 0xCC, 0xF0};
  for (int i = c.n - 1; i >= 0; i--) {
    const int sh = 1 << i;
    const uint8_t hi = c.tt & var[i], lo = (uint8_t)(c.tt & (uint8_t)~var[i]);
    if ((uint8_t)(hi >> sh) == lo) {  // independent of x_i: remove it
      Cut d;
      d.n = (uint8_t)(c.n - 1);
      int k = 0;
      for (int q = 0; q < c.n; q++)
        if (q != i) d.leaf[k++] = c.leaf[q];
      uint8_t t = 0;
      for (int m = 0; m < 8; m++) {
        // minterm m over d -> insert a 0 bit at position i
        const int low = m & ((1 << i) - 1), high = (m >> i) << (i + 1);
        t |= (uint8_t)(((c.tt >> (low | high)) & 1) << m);
      }
      // tables over fewer leaves repeat; normalise to the 3-variable form
      for (int m = 0; m < 8; m++) {
        const int mm = m & ((1 << d.n) - 1);
        t = (uint8_t)((t & ~(1 << m)) | (((t >> mm) & 1) << m));
      }
      d.tt = t;
      c = d;
    }
  }
}

}  // namespace

// values: ids 0..NA-1 are the cone's ANDs (ascending variable), NA..NA+NP-1
// the support PIs, NA+NP the constant.  fanin value ids and complement bits
// per AND come in f0/f1/c0/c1.
void lut_map(size_t NA, size_t NP, const std::vector<int64_t> &f0, const std::vector<int64_t> &f1,
             const std::vector<uint8_t> &c0, const std::vector<uint8_t> &c1, int64_t root, LutCover &out) {
  const size_t NV = NA + NP + 1;
  const int32_t CONST = (int32_t)(NA + NP);
  const size_t kMaxCuts = 8;           // non-trivial cuts kept per node
  const size_t kStride = kMaxCuts + 1;  // + the trivial cut
  // flat per-thread storage, reused across calls (no per-node allocations)
  thread_local std::vector<Cut> store;
  thread_local std::vector<uint8_t> ncut;
  thread_local std::vector<Cut> scratch;
  store.resize(NV * kStride);
  ncut.assign(NV, 0);
  auto cut_at = [&](size_t v, size_t i) -> Cut & { return store[v * kStride + i]; };
  for (size_t v = NA; v < NV; v++) {
    Cut t;
    if ((int32_t)v == CONST) {
      t.n = 0;
      t.tt = 0x00;
    } else {
      t.n = 1;
      t.leaf[0] = (int32_t)v;
      t.tt = 0xAA;
    }
    cut_at(v, 0) = t;
    ncut[v] = 1;
  }
  std::vector<uint32_t> fanout(NV, 0);
  for (size_t i = 0; i < NA; i++) {
    fanout[f0[i]]++;
    fanout[f1[i]]++;
  }
  fanout[root]++;
  std::vector<double> af(NV, 0.0);
  std::vector<int> best(NV, -1);
  thread_local std::vector<uint64_t> sig;
  sig.resize(NV * kStride);
  for (size_t v = NA; v < NV; v++) sig[v * kStride] = sig_of(cut_at(v, 0));
  thread_local std::vector<double> flows;
  thread_local std::vector<uint32_t> rank;
  for (size_t v = 0; v < NA; v++) {
    scratch.clear();
    const size_t na_ = ncut[f0[v]], nb_ = ncut[f1[v]];
    const uint64_t *sa = &sig[f0[v] * kStride], *sb = &sig[f1[v] * kStride];
    for (size_t ia = 0; ia < na_; ia++) {
      const Cut &a = cut_at(f0[v], ia);
      for (size_t ib = 0; ib < nb_; ib++) {
        if (__builtin_popcountll(sa[ia] | sb[ib]) > 3) continue;
        const Cut &b = cut_at(f1[v], ib);
        Cut m;
        if (!merge(a, b, m)) continue;
        const uint8_t ta = (uint8_t)(expand(a.tt, a, m) ^ (c0[v] ? 0xFF : 0x00));
        const uint8_t tb = (uint8_t)(expand(b.tt, b, m) ^ (c1[v] ? 0xFF : 0x00));
        m.tt = ta & tb;
        minimise(m);
        bool dup = false;
        for (const Cut &e : scratch)
          if (e.n == m.n && e.leaf[0] == m.leaf[0] && e.leaf[1] == m.leaf[1] && e.leaf[2] == m.leaf[2]) {
            dup = true;
            break;
          }
        if (!dup) scratch.push_back(m);
      }
    }
    // area flow of each cut; keep the best kMaxCuts, then the trivial cut
    auto flow = [&](const Cut &c) {
      double s = 1.0;
      for (int k = 0; k < c.n; k++)
        if (c.leaf[k] < (int32_t)NA) s += af[c.leaf[k]];
      return s;
    };
    // the kMaxCuts best by (flow, leaves), ties in generation order: a
    // stable insertion into a short ranked list
    flows.resize(scratch.size());
    rank.clear();
    for (size_t i = 0; i < scratch.size(); i++) {
      flows[i] = flow(scratch[i]);
      auto before = [&](uint32_t x, uint32_t y) {
        return flows[x] < flows[y] || (flows[x] == flows[y] && scratch[x].n < scratch[y].n);
      };
      if (rank.size() == kMaxCuts && !before((uint32_t)i, rank.back())) continue;
      size_t pos = rank.size();
      while (pos > 0 && before((uint32_t)i, rank[pos - 1])) pos--;
      rank.insert(rank.begin() + pos, (uint32_t)i);
      if (rank.size() > kMaxCuts) rank.pop_back();
    }
    const size_t keep = rank.size();
    for (size_t i = 0; i < keep; i++) {
      cut_at(v, i) = scratch[rank[i]];
      sig[v * kStride + i] = sig_of(scratch[rank[i]]);
    }
    best[v] = 0;
    af[v] = keep == 0 ? 1.0 : flows[rank[0]] / std::max<uint32_t>(1, fanout[v]);
    Cut t;
    t.n = 1;
    t.leaf[0] = (int32_t)v;
    t.tt = 0xAA;
    cut_at(v, keep) = t;  // trivial cut: used only when v is a leaf of a parent's cut
    sig[v * kStride + keep] = sig_of(t);
    ncut[v] = (uint8_t)(keep + 1);
  }

  // cover with reference counting, then exact-area recovery
  std::vector<uint32_t> refs(NV, 0);
  std::vector<uint8_t> used(NA, 0);
  auto deref = [&](auto &&self, int32_t v) -> uint32_t {  // returns LUTs freed
    if (v >= (int32_t)NA) return 0;
    uint32_t freed = 1;
    const Cut &c = cut_at(v, best[v]);
    for (int k = 0; k < c.n; k++)
      if (c.leaf[k] < (int32_t)NA && --refs[c.leaf[k]] == 0) freed += self(self, c.leaf[k]);
    return freed;
  };
  auto ref = [&](auto &&self, int32_t v) -> uint32_t {  // returns LUTs added
    if (v >= (int32_t)NA) return 0;
    uint32_t added = 1;
    const Cut &c = cut_at(v, best[v]);
    for (int k = 0; k < c.n; k++)
      if (c.leaf[k] < (int32_t)NA && refs[c.leaf[k]]++ == 0) added += self(self, c.leaf[k]);
    return added;
  };
  // LUTs that referencing cut `c` would add: the same count as ref(), taken
  // without touching the reference counts (a node joins once, when its count
  // is zero; the stamp marks the ones already counted)
  std::vector<uint32_t> stamp(NA, 0);
  uint32_t cur = 0;
  auto added = [&](auto &&self, const Cut &c) -> uint32_t {
    uint32_t a = 1;
    for (int k = 0; k < c.n; k++) {
      const int32_t l = c.leaf[k];
      if (l < (int32_t)NA && refs[l] == 0 && stamp[l] != cur) {
        stamp[l] = cur;
        a += self(self, cut_at(l, best[l]));
      }
    }
    return a;
  };
  if (root < (int64_t)NA) {
    refs[root] = 1;
    ref(ref, (int32_t)root);
  }
  for (int round = 0; round < 2; round++) {
    for (size_t v = 0; v < NA; v++) {
      if (refs[v] == 0) continue;
      const int nc = (int)ncut[v] - 1;  // skip the trivial cut
      if (nc <= 1) continue;
      deref(deref, (int32_t)v);
      uint32_t best_area = UINT32_MAX;
      int best_i = best[v];
      for (int i = 0; i < nc; i++) {
        cur++;
        const uint32_t a = added(added, cut_at(v, i));
        if (a < best_area) {
          best_area = a;
          best_i = i;
        }
      }
      best[v] = best_i;
      ref(ref, (int32_t)v);
    }
  }
  out.luts.clear();
  out.index.assign(NA, -1);
  for (size_t v = 0; v < NA; v++) {
    if (refs[v] == 0) continue;
    const Cut &c = cut_at(v, best[v]);
    LutCover::Lut l;
    l.node = (int32_t)v;
    l.n = c.n;
    for (int k = 0; k < 3; k++) l.leaf[k] = c.leaf[k];
    l.tt = c.tt;
    out.index[v] = (int32_t)out.luts.size();
    out.luts.push_back(l);
  }
}

}  // namespace lec
