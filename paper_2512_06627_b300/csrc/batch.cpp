// batch.cpp -- many miters in one persistent launch.
//
// Sub-miters of the kind a sweeping scheduler hands to exact simulation
// (paper §3.2: one sub-miter per signal pair; ES cost grows with 2^PIs and
// linearly with gates) are uneven: a few PIs and tens of ANDs up to ~30 PIs
// and thousands of ANDs.  One launch per miter leaves the GPU idle on the
// small ones.  Here every miter's slot program is packed into one record
// arena, its pattern space is cut into (miter, chunk range) tiles whose sizes
// follow cost_ES = ANDs x 2^PIs, and a persistent kernel with one block per
// resident slot pulls tiles from a global queue head with atomicAdd.  Tiles of
// a miter are queued in ascending pattern order, so a counterexample found
// early lets the remaining tiles of that miter skip (the minimum is kept
// exact: a tile is skipped only when its first pattern is not below it).
// The reset-launch-readback sequence is captured once in a CUDA graph and
// replayed by every run.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

using namespace lec;

namespace {
constexpr double kBatchJitWork = 5e7;   // records x chunks: about 50 us in the interpreter
constexpr uint32_t kBatchJitLive = 230; // table live set that still fits the register file
}  // namespace

struct lec_es_batch_plan {
  size_t k = 0;
  std::vector<Program> progs;
  std::vector<int> jit_of;                // miter -> index into jit_miters, or -1
  std::vector<uint32_t> jit_miters;       // miters run by their own specialised kernel
  std::vector<JitKernel *> jit_kernels;
  unsigned long long *d_aux = nullptr;    // per JIT miter: {patterns evaluated, chunk-grab counter}
  double jit_ms = 0;
  std::vector<int> fallback_of;           // miter -> index into fallbacks, or -1
  std::vector<lec_es_plan *> fallbacks;   // miters whose live set exceeds the batch kernel's slots
  int block = 0, grid = 0;
  size_t smem = 0;
  uint32_t ring_recs = 512;
  uint32_t max_slots = 0;
  uint32_t num_tiles = 0;
  void *d_recs = nullptr, *d_miters = nullptr, *d_tiles = nullptr;
  unsigned long long *d_cex = nullptr;
  uint32_t *d_head = nullptr;             // [head, status]
  unsigned long long *h_cex = nullptr;    // pinned
  uint32_t *h_status = nullptr;           // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool pending = false;
  double host_ms = 0;
  BatchParams params{};
};

namespace {

void batch_release(lec_es_ctx *c, lec_es_batch_plan *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->h_cex) cudaFreeHost(b->h_cex);
  if (b->h_status) cudaFreeHost(b->h_status);
  c->arena.free(b->d_recs);
  c->arena.free(b->d_miters);
  c->arena.free(b->d_tiles);
  c->arena.free(b->d_cex);
  c->arena.free(b->d_head);
  c->arena.free(b->d_aux);
  for (lec_es_plan *p : b->fallbacks) plan_release(c, p);
  delete b;
}

int compile_all(lec_es_ctx *c, const lec_es_miter *m, size_t k, uint32_t order, std::vector<Program> &progs) {
  progs.assign(k, Program());
  std::vector<int> rcs(k, LEC_ES_OK);
  const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 16u));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; t++) {
    th.emplace_back([&, t]() {
      for (size_t i = t; i < k; i += nt) {
        MiterView v{m[i].num_pis, m[i].num_ands, m[i].fanins, m[i].out_lit};
        try {
          rcs[i] = compile_program(v, order, c->max_pis, progs[i]);
        } catch (const std::bad_alloc &) {
          rcs[i] = LEC_ES_ENOMEM;
        }
      }
    });
  }
  for (auto &x : th) x.join();
  for (int rc : rcs)
    if (rc) return rc;
  return LEC_ES_OK;
}

}  // namespace

extern "C" int lec_es_batch_prepare(lec_es_ctx *c, const lec_es_miter *m, size_t k, const lec_es_options *opt,
                                    lec_es_batch_plan **out) {
  if (!c || !m || !out || k == 0 || k > 0xFFFFFFFFull) return LEC_ES_EINVAL;
  *out = nullptr;
  const double t0 = now_ms();
  std::unique_ptr<lec_es_batch_plan> b(new (std::nothrow) lec_es_batch_plan());
  if (!b) return LEC_ES_ENOMEM;
  b->k = k;
  int rc = compile_all(c, m, k, opt ? opt->order : LEC_ES_ORDER_AUTO, b->progs);
  if (rc) return rc;
  if (cudaSetDevice(c->device) != cudaSuccess) return LEC_ES_ECUDA;

  // block size: the largest that holds the batch's largest live set in shared
  // memory; miters beyond what a 64-thread block holds run on their own
  std::vector<uint32_t> slots(k);
  for (size_t i = 0; i < k; i++) slots[i] = b->progs[i].num_slots;
  const int pref = opt && opt->block_threads ? (int)opt->block_threads : 256;
  uint32_t max_fit64 = (uint32_t)((c->smem_optin - 64 - 4 * 512 * 8) / (64 * 4));
  b->fallback_of.assign(k, -1);
  uint32_t ms = 1;
  for (size_t i = 0; i < k; i++)
    if (slots[i] <= max_fit64) ms = std::max(ms, slots[i]);
  b->max_slots = ms;
  b->block = 0;
  for (int blk : {256, 128, 64}) {
    if (blk > pref) continue;
    if (batch_smem_bytes(ms, blk, b->ring_recs) <= (size_t)c->smem_optin) {
      b->block = blk;
      break;
    }
  }
  if (!b->block) b->block = 64;
  b->smem = batch_smem_bytes(ms, b->block, b->ring_recs);
  if (configure_batch(b->block, b->smem) != 0) return LEC_ES_ECUDA;
  const int bps = std::max(1, batch_blocks_per_sm(b->block, b->smem));
  b->grid = c->sm_count * bps;
  if (opt && opt->grid_blocks) b->grid = (int)opt->grid_blocks;

  // heavy miters (interpreter cost above ~50 us) get their own specialised
  // kernel, compiled in parallel here and launched inside the same graph
  b->jit_of.assign(k, -1);
  const bool allow_jit = !(opt && (opt->tier == LEC_ES_TIER_INTERP || opt->tier == LEC_ES_TIER_SPILL));
  if (allow_jit) {
    for (size_t i = 0; i < k; i++) {
      const Program &g = b->progs[i];
      const double work = (double)g.recs.size() * (double)num_chunks(g.n);
      if (work >= kBatchJitWork && !g.lut.order.empty() && g.lut.live <= kBatchJitLive) {
        b->jit_of[i] = (int)b->jit_miters.size();
        b->jit_miters.push_back((uint32_t)i);
      }
    }
    b->jit_kernels.assign(b->jit_miters.size(), nullptr);
    std::vector<int> jrc(b->jit_miters.size(), LEC_ES_OK);
    const double tj = now_ms();
    const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 16u));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++) {
      th.emplace_back([&, t]() {
        cudaSetDevice(c->device);
        for (size_t j = t; j < b->jit_miters.size(); j += nt)
          jrc[j] = jit_get_kernel(c, b->progs[b->jit_miters[j]], true, &b->jit_kernels[j], nullptr);
      });
    }
    for (auto &x : th) x.join();
    b->jit_ms = now_ms() - tj;
    for (int r : jrc)
      if (r) return r;
  }

  // pack programs
  std::vector<BatchMiter> mt(k);
  size_t total_recs = 0;
  for (size_t i = 0; i < k; i++) {
    const size_t np = std::max<size_t>(2, (b->progs[i].recs.size() + 1) & ~(size_t)1);
    mt[i].rec_off = (uint32_t)total_recs;
    mt[i].nrec = (uint32_t)b->progs[i].recs.size();
    mt[i].nrec_padded = (uint32_t)np;
    mt[i].nslots = b->progs[i].num_slots;
    mt[i].out_slot = b->progs[i].out_slot;
    mt[i].out_compl = b->progs[i].out_compl;
    mt[i].n = b->progs[i].n;
    total_recs += np;
  }
  if (total_recs > 0xFFFFFFFFull) return LEC_ES_ETOOBIG;
  std::vector<Rec> arena_recs(total_recs);
  for (size_t i = 0; i < k; i++)
    memcpy(&arena_recs[mt[i].rec_off], b->progs[i].recs.data(), b->progs[i].recs.size() * sizeof(Rec));

  // tiles sized by cost_ES (records x chunks), big miters first, each miter's
  // tiles in ascending pattern order
  double total_cost = 0;
  std::vector<size_t> idx;
  for (size_t i = 0; i < k; i++) {
    if (slots[i] > ms || b->jit_of[i] >= 0) continue;
    idx.push_back(i);
    total_cost += (double)mt[i].nrec * (double)num_chunks(mt[i].n);
  }
  std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
    return (double)mt[x].nrec * num_chunks(mt[x].n) > (double)mt[y].nrec * num_chunks(mt[y].n);
  });
  const double target = std::max(1.0, total_cost / ((double)b->grid * 16.0));
  std::vector<BatchTile> tiles;
  for (size_t i : idx) {
    const uint64_t C = num_chunks(mt[i].n);
    uint64_t tc = (uint64_t)(target / std::max<uint32_t>(1, mt[i].nrec));
    tc = ((tc + b->block - 1) / b->block) * b->block;
    tc = std::max<uint64_t>(tc, (uint64_t)b->block);
    for (uint64_t c0 = 0; c0 < C; c0 += tc) {
      BatchTile t{};
      t.miter = (uint32_t)i;
      t.chunk_begin = c0;
      t.chunk_end = std::min(C, c0 + tc);
      tiles.push_back(t);
    }
  }
  if (tiles.size() > 0xFFFFFFF0ull) return LEC_ES_ETOOBIG;
  b->num_tiles = (uint32_t)tiles.size();

  // miters too wide for the batch kernel: their own spill-tier plans
  for (size_t i = 0; i < k; i++) {
    if (slots[i] <= ms || b->jit_of[i] >= 0) continue;
    lec_es_options o{};
    o.word_end = UINT64_MAX;
    o.tier = LEC_ES_TIER_SPILL;
    o.order = opt ? opt->order : LEC_ES_ORDER_AUTO;
    lec_es_plan *p = nullptr;
    rc = plan_prepare(c, &m[i], &o, &p);
    if (rc) return rc;
    b->fallback_of[i] = (int)b->fallbacks.size();
    b->fallbacks.push_back(p);
  }

  // device buffers
  const size_t rb = std::max<size_t>(16, arena_recs.size() * sizeof(Rec));
  b->d_recs = c->arena.alloc(rb);
  b->d_miters = c->arena.alloc(std::max<size_t>(16, k * sizeof(BatchMiter)));
  b->d_tiles = c->arena.alloc(std::max<size_t>(16, tiles.size() * sizeof(BatchTile)));
  b->d_cex = (unsigned long long *)c->arena.alloc(k * 8);
  b->d_head = (uint32_t *)c->arena.alloc(16);
  b->d_aux = (unsigned long long *)c->arena.alloc(std::max<size_t>(16, b->jit_miters.size() * 16));
  if (!b->d_recs || !b->d_miters || !b->d_tiles || !b->d_cex || !b->d_head || !b->d_aux) {
    batch_release(c, b.release());
    return LEC_ES_ENOMEM;
  }
  if (cudaMallocHost((void **)&b->h_cex, k * 8) != cudaSuccess ||
      cudaMallocHost((void **)&b->h_status, 16) != cudaSuccess) {
    batch_release(c, b.release());
    return LEC_ES_ENOMEM;
  }
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemcpyAsync(b->d_recs, arena_recs.data(), arena_recs.size() * sizeof(Rec),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_miters, mt.data(), k * sizeof(BatchMiter), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    batch_release(c, b.release());
    return LEC_ES_ECUDA;
  }
  BatchParams &bp = b->params;
  bp.recs = (const Rec *)b->d_recs;
  bp.miters = (const BatchMiter *)b->d_miters;
  bp.tiles = (const BatchTile *)b->d_tiles;
  bp.num_tiles = b->num_tiles;
  bp.max_slots = ms;
  bp.ring_recs = b->ring_recs;
  bp.cex = b->d_cex;
  bp.head = b->d_head;
  bp.status = b->d_head + 1;
  bp.cancel = nullptr;

  // capture reset + kernel + read-back once
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
    batch_release(c, b.release());
    return LEC_ES_ECUDA;
  }
  int lerr = 0;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(b->d_cex, 0xFF, k * 8, st);
    cudaMemsetAsync(b->d_head, 0, 16, st);
    if (!b->jit_miters.empty()) cudaMemsetAsync(b->d_aux, 0, b->jit_miters.size() * 16, st);
    // heavy miters first, each over the whole GPU, then the tile queue
    for (size_t j = 0; j < b->jit_miters.size() && !lerr; j++) {
      const uint32_t i = b->jit_miters[j];
      JitKernel *kk = b->jit_kernels[j];
      uint64_t cb = 0, ce = num_chunks(b->progs[i].n), grabs = ~0ull;
      unsigned long long *cex = b->d_cex + i, *ev = b->d_aux + 2 * j, *next = b->d_aux + 2 * j + 1;
      void *args[] = {&cb, &ce, &cex, &ev, &next, &grabs};
      const uint64_t warps_needed = (ce + 31) / 32;
      const uint64_t grid = std::max<uint64_t>(
          1, std::min<uint64_t>((uint64_t)c->sm_count * kk->blocks_per_sm, (warps_needed * 32 + kk->block - 1) / kk->block));
      if (cudaLaunchKernel((const void *)kk->kern, dim3((unsigned)grid), dim3(kk->block), args, 0, st) !=
          cudaSuccess)
        lerr = 1;
    }
    if (b->num_tiles && !lerr) lerr = launch_batch(bp, b->block, b->grid, b->smem, st);
    cudaMemcpyAsync(b->h_cex, b->d_cex, k * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(b->h_status, b->d_head, 16, cudaMemcpyDeviceToHost, st);
    e = cudaStreamEndCapture(st, &b->graph);
  }
  if (e != cudaSuccess || lerr || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
    batch_release(c, b.release());
    return LEC_ES_ECUDA;
  }
  b->host_ms = now_ms() - t0;
  *out = b.release();
  return LEC_ES_OK;
}

extern "C" int lec_es_batch_run_async(lec_es_ctx *c, lec_es_batch_plan *b) {
  if (!c || !b) return LEC_ES_EINVAL;
  cudaStream_t st = c->stream;
  cudaEventRecord(b->e0, st);
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return LEC_ES_ECUDA;
  cudaEventRecord(b->e1, st);
  for (lec_es_plan *p : b->fallbacks) {
    int rc = plan_run_async(c, p, nullptr);
    if (rc) return rc;
  }
  b->pending = true;
  return LEC_ES_OK;
}

extern "C" int lec_es_batch_results(lec_es_ctx *c, lec_es_batch_plan *b, lec_es_result *out, size_t k) {
  if (!c || !b || !out || k != b->k || !b->pending) return LEC_ES_EINVAL;
  int rc = wait_event(b->e1, c->timeout_s);
  if (rc) return rc;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LEC_ES_ECUDA;
  b->pending = false;
  float ms = 0;
  cudaEventElapsedTime(&ms, b->e0, b->e1);
  const uint32_t status = b->h_status[1];
  for (size_t i = 0; i < k; i++) {
    if (b->fallback_of[i] >= 0) {
      rc = plan_result(c, b->fallbacks[b->fallback_of[i]], &out[i]);
      if (rc) return rc;
      continue;
    }
    const Program &g = b->progs[i];
    lec_es_result &r = out[i];
    memset(&r, 0, sizeof(r));
    r.support_n = g.n;
    for (uint32_t q = 0; q < g.n; q++) r.support[q] = g.support[q];
    r.cone_ands = g.cone_ands;
    r.num_slots = g.num_slots;
    r.tier = b->jit_of[i] >= 0 ? LEC_ES_TIER_JIT : LEC_ES_TIER_INTERP;
    r.order = g.order;
    r.words_checked = num_words(g.n);
    r.device_ms = ms;
    r.host_ms = b->host_ms / (double)k;
    r.jit_ms = b->jit_ms / (double)k;
    r.cex = b->h_cex[i];
    r.verdict = r.cex == UINT64_MAX ? LEC_ES_EQUIVALENT : LEC_ES_NONEQUIVALENT;
  }
  if (status & DEV_WAIT_TIMEOUT) return LEC_ES_EDEVICE_WAIT;
  return status ? LEC_ES_ECUDA : LEC_ES_OK;
}

extern "C" void lec_es_batch_free(lec_es_ctx *c, lec_es_batch_plan *b) {
  if (!c || !b) return;
  if (b->pending) wait_event(b->e1, c->timeout_s);
  cudaStreamSynchronize(c->stream);
  batch_release(c, b);
}

extern "C" int lec_es_batch(lec_es_ctx *c, const lec_es_miter *m, size_t k, lec_es_result *out) {
  if (!c || !m || !out) return LEC_ES_EINVAL;
  lec_es_batch_plan *b = nullptr;
  int rc = lec_es_batch_prepare(c, m, k, nullptr, &b);
  if (rc) return rc;
  rc = lec_es_batch_run_async(c, b);
  if (!rc) rc = lec_es_batch_results(c, b, out, k);
  lec_es_batch_free(c, b);
  return rc;
}
