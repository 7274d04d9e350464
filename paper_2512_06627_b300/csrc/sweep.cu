// sweep.cu -- random-simulation signatures and candidate equivalent pairs.
//
// Step (1) of the sweeping flow (paper §2.3): simulate the whole AIG on a
// batch of random input words and group nodes with equal signatures into
// potentially-equivalent (PE) pairs, which become the sub-miters handed to
// exact simulation (§3.2).  The input words are drawn by the caller.
//
// Device work: the ANDs are bucketed by logic level on the host; one launch
// per level evaluates its nodes, one warp per node: lanes stride over the
// signature words (coalesced 8-byte loads of both fanins' rows), each
// computes (x ^ cx) & (y ^ cy), stores it, and mixes it with its word index
// into a 64-bit hash that the warp XOR-reduces.  When there are at most 64
// PIs, lane 0 also ORs the fanins' PI-support masks.  Memory-bound: 3 x 8
// bytes per node per word.
//
// Host work (lec_es_match_pairs): nodes are sorted by hash, equal hashes are
// split into classes of identical signatures, classes whose signature is
// constant are dropped, and every member is paired with the class's lowest
// variable if the union of their supports has at most max_support PIs.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

namespace lec {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x, uint64_t w) {
  // splitmix64 finaliser over the word and its position
  uint64_t z = x + (w + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// With norm set the hash is of the node's signature complemented when its
// first pattern is 1, so a node and its complement hash alike.
__global__ void __launch_bounds__(256) sim_level(const uint32_t *__restrict__ fanins, const uint32_t *__restrict__ nodes,
                                                 uint32_t count, uint32_t num_pis, uint32_t nwords, uint64_t *sig,
                                                 uint64_t *sup, uint64_t *hash, int norm) {
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (warp >= count) return;  // whole warps exit together
  const uint32_t v = nodes[warp];
  const uint64_t a = (uint64_t)v - num_pis - 1;
  const uint32_t l0 = fanins[2 * a], l1 = fanins[2 * a + 1];
  const uint64_t m0 = (l0 & 1u) ? ~0ull : 0ull, m1 = (l1 & 1u) ? ~0ull : 0ull;
  const uint64_t *s0 = sig + (size_t)(l0 >> 1) * nwords;
  const uint64_t *s1 = sig + (size_t)(l1 >> 1) * nwords;
  uint64_t *d = sig + (size_t)v * nwords;
  // the phase: first pattern of the node (word 0, bit 0), known to every lane
  const uint64_t flip = norm && (((s0[0] ^ m0) & (s1[0] ^ m1)) & 1ull) ? ~0ull : 0ull;
  uint64_t h = 0;
  for (uint32_t w = lane; w < nwords; w += 32) {
    const uint64_t x = (s0[w] ^ m0) & (s1[w] ^ m1);
    d[w] = x;
    h ^= mix64(x ^ flip, w);
  }
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xFFFFFFFFu, h, o);
  if (lane == 0) {
    hash[v] = h;
    if (sup) sup[v] = sup[l0 >> 1] | sup[l1 >> 1];
  }
}

// Hashes (and support masks) of the constant and the PIs.
__global__ void __launch_bounds__(256) sim_leaves(uint32_t num_pis, uint32_t nwords, const uint64_t *sig, uint64_t *sup,
                                                  uint64_t *hash, int norm) {
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (warp > num_pis) return;
  const uint64_t *s = sig + (size_t)warp * nwords;
  const uint64_t flip = norm && (s[0] & 1ull) ? ~0ull : 0ull;
  uint64_t h = 0;
  for (uint32_t w = lane; w < nwords; w += 32) h ^= mix64(s[w] ^ flip, w);
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xFFFFFFFFu, h, o);
  if (lane == 0) {
    hash[warp] = h;
    if (sup) sup[warp] = warp == 0 ? 0ull : (1ull << (warp - 1));
  }
}

struct SimBuffers {
  void *fan = nullptr, *nodes = nullptr;
  uint64_t *sig = nullptr, *sup = nullptr, *hash = nullptr;
  void free_all(lec_es_ctx *c) {
    c->arena.free(fan);
    c->arena.free(nodes);
    c->arena.free(sig);
    c->arena.free(sup);
    c->arena.free(hash);
  }
};

}  // namespace

// Simulate every variable; fills host arrays (sigs may be null).  With norm
// the hashes are of phase-normalised signatures (complemented when the first
// pattern is 1).
int simulate(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, const uint64_t *pi_words,
             uint32_t nwords, uint64_t *h_sigs, uint64_t *h_hash, uint64_t *h_sup, bool norm) {
  if (!c || (num_ands && !fanins) || (num_pis && !pi_words) || nwords == 0 || !h_hash) return LEC_ES_EINVAL;
  const uint64_t V = (uint64_t)num_pis + num_ands + 1;
  // levels (every fanin variable is below its AND: one forward pass)
  std::vector<uint32_t> level(V, 0);
  uint32_t maxl = 0;
  for (uint64_t a = 0; a < num_ands; a++) {
    const uint64_t v = num_pis + 1 + a;
    const uint32_t u0 = fanins[2 * a] >> 1, u1 = fanins[2 * a + 1] >> 1;
    if (u0 >= v || u1 >= v) return LEC_ES_EINVAL;
    level[v] = std::max(level[u0], level[u1]) + 1;
    maxl = std::max(maxl, level[v]);
  }
  std::vector<uint32_t> off(maxl + 2, 0);
  for (uint64_t a = 0; a < num_ands; a++) off[level[num_pis + 1 + a] + 1]++;
  for (uint32_t l = 1; l <= maxl + 1; l++) off[l] += off[l - 1];
  std::vector<uint32_t> nodes(std::max<uint64_t>(1, num_ands));
  {
    std::vector<uint32_t> fill(off.begin(), off.end());
    for (uint64_t a = 0; a < num_ands; a++) {
      const uint32_t v = (uint32_t)(num_pis + 1 + a);
      nodes[fill[level[v]]++] = v;
    }
  }
  cudaSetDevice(c->device);
  SimBuffers b;
  const bool want_sup = h_sup && num_pis <= 64;
  b.fan = c->arena.alloc(std::max<uint64_t>(8, 8ull * num_ands));
  b.nodes = c->arena.alloc(4ull * nodes.size());
  b.sig = (uint64_t *)c->arena.alloc(V * nwords * 8);
  b.hash = (uint64_t *)c->arena.alloc(V * 8);
  b.sup = want_sup ? (uint64_t *)c->arena.alloc(V * 8) : nullptr;
  if (!b.fan || !b.nodes || !b.sig || !b.hash || (want_sup && !b.sup)) {
    b.free_all(c);
    return LEC_ES_ENOMEM;
  }
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  if (num_ands) e = cudaMemcpyAsync(b.fan, fanins, 8ull * num_ands, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.nodes, nodes.data(), 4ull * nodes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.sig, 0, nwords * 8ull, st);  // the constant's row
  if (e == cudaSuccess && num_pis)
    e = cudaMemcpyAsync(b.sig + nwords, pi_words, (uint64_t)num_pis * nwords * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const uint32_t warps = num_pis + 1;
    sim_leaves<<<(warps * 32 + 255) / 256, 256, 0, st>>>(num_pis, nwords, b.sig, b.sup, b.hash, norm ? 1 : 0);
    e = cudaGetLastError();
  }
  for (uint32_t l = 1; l <= maxl && e == cudaSuccess; l++) {
    const uint32_t cnt = off[l + 1] - off[l];
    if (!cnt) continue;
    sim_level<<<(uint32_t)(((uint64_t)cnt * 32 + 255) / 256), 256, 0, st>>>(
        (const uint32_t *)b.fan, (const uint32_t *)b.nodes + off[l], cnt, num_pis, nwords, b.sig, b.sup, b.hash,
        norm ? 1 : 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_hash, b.hash, V * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && h_sigs) e = cudaMemcpyAsync(h_sigs, b.sig, V * nwords * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && want_sup) e = cudaMemcpyAsync(h_sup, b.sup, V * 8, cudaMemcpyDeviceToHost, st);
  const cudaError_t se = cudaStreamSynchronize(st);
  b.free_all(c);
  return (e == cudaSuccess && se == cudaSuccess) ? LEC_ES_OK : LEC_ES_ECUDA;
}

}  // namespace lec

using namespace lec;

extern "C" int lec_es_signatures(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                                 const uint64_t *pi_words, uint32_t nwords, uint64_t *sigs_out, uint64_t *hash_out) {
  if (!hash_out) return LEC_ES_EINVAL;
  return simulate(c, num_pis, num_ands, fanins, pi_words, nwords, sigs_out, hash_out, nullptr, false);
}

extern "C" int lec_es_match_pairs(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                                  const uint64_t *pi_words, uint32_t nwords, uint32_t max_support, uint32_t *pairs,
                                  uint64_t cap, uint64_t *npairs) {
  if (!c || !npairs || num_pis > 64) return LEC_ES_EINVAL;
  const uint64_t V = (uint64_t)num_pis + num_ands + 1;
  std::vector<uint64_t> sigs, hash(V), sup(V);
  try {
    sigs.resize(V * nwords);
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  int rc = simulate(c, num_pis, num_ands, fanins, pi_words, nwords, sigs.data(), hash.data(), sup.data(), false);
  if (rc) return rc;
  auto row = [&](uint64_t v) { return &sigs[v * nwords]; };
  auto constant = [&](uint64_t v) {
    const uint64_t *r = row(v);
    const bool z = r[0] == 0ull, o = r[0] == ~0ull;
    if (!z && !o) return false;
    for (uint32_t w = 1; w < nwords; w++)
      if (r[w] != r[0]) return false;
    return true;
  };
  std::vector<uint32_t> order;
  order.reserve(num_ands);
  for (uint64_t v = num_pis + 1; v < V; v++)
    if (!constant(v)) order.push_back((uint32_t)v);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return hash[x] < hash[y]; });
  std::vector<std::pair<uint32_t, uint32_t>> out;
  size_t i = 0;
  while (i < order.size()) {
    size_t j = i + 1;
    while (j < order.size() && hash[order[j]] == hash[order[i]]) j++;
    if (j - i > 1) {
      // split the hash run into classes of identical signatures
      std::vector<uint32_t> run(order.begin() + i, order.begin() + j);
      std::sort(run.begin(), run.end());
      std::vector<uint8_t> used(run.size(), 0);
      for (size_t p = 0; p < run.size(); p++) {
        if (used[p]) continue;
        const uint32_t rep = run[p];  // lowest variable of its class
        for (size_t q = p + 1; q < run.size(); q++) {
          if (used[q] || memcmp(row(rep), row(run[q]), nwords * 8) != 0) continue;
          used[q] = 1;
          if (__builtin_popcountll(sup[rep] | sup[run[q]]) <= (int)max_support) out.push_back({rep, run[q]});
        }
      }
    }
    i = j;
  }
  std::sort(out.begin(), out.end());
  *npairs = out.size();
  if (pairs)
    for (uint64_t q = 0; q < std::min<uint64_t>(cap, out.size()); q++) {
      pairs[2 * q] = out[q].first;
      pairs[2 * q + 1] = out[q].second;
    }
  return LEC_ES_OK;
}
