// batch.cpp -- many miters in one launch sequence, replayed as a CUDA graph.
//
// Sub-miters of the kind a sweeping scheduler hands to exact simulation
// (paper §3.2: one sub-miter per signal pair; ES cost grows with 2^PIs and
// linearly with gates) are uneven: a few PIs and tens of ANDs up to ~30 PIs
// and thousands of ANDs.  One launch per miter leaves the GPU idle on the
// small ones.  Preparation has two stages:
//   programs  every miter is compiled (front end, 16 host threads); miters
//             whose predicted interpreter time exceeds kBatchJitMs (0.02 ms)
//             get their specialised kernel (compiled in parallel); the
//             others' slot programs are packed into one record arena;
//   layout    the light miters' pattern spaces are cut into (miter, chunk
//             range) tiles sized by cost_ES = records x chunks; a persistent
//             kernel pulls tiles from a queue head with atomicAdd; the graph
//             forks into branches so the specialised kernels overlap each
//             other and the tile queue.
// Tiles of a miter are queued in ascending pattern order, so a counterexample
// found early lets the remaining tiles skip (a tile is skipped only when its
// first pattern is not below the current minimum, so the minimum is exact).
// The layout's tunables -- threads per tile pass, tiles per resident block
// (how many 32-pattern words a thread takes per tile) and records per staging
// stage -- can be chosen by timing candidate layouts of the tile queue
// (LEC_ES_FLAG_AUTOTUNE); choices are cached per batch shape in memory and in
// the context's cache directory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

using namespace lec;

namespace {
// Predicted interpreter time above which a miter gets its own kernel; the
// rest share the tile queue, which runs beside the kernels and must not
// outlast them.  On the 4,096 node-pair batch (B300): 0.2 / 0.1 / 0.05 /
// 0.03 / 0.025 / 0.02 / 0.0125 / 0.005 ms -> 25.3 / 10.5 / 5.39 / 4.09 /
// 3.89 / 3.84 / 4.05 / 5.12 ms per batch.
constexpr double kBatchJitMs = 0.02;
constexpr uint32_t kBatchJitLive = 288;  // table live set given an own kernel (as a single check's)
constexpr int kMaxBranches = 64;         // parallel graph branches (at most)
constexpr int kDefaultBranches = 8;  // 4 / 8 / 16 branches: 3.85 / 3.80 / 3.78 ms on the 4,096-pair batch

struct Layout {
  int block = 256;            // threads (64-pattern words) per tile pass
  uint32_t ring_recs = 256;   // 16-byte records per staging stage (4 stages)
  uint32_t granularity = 8;   // tiles per resident block slot (8 / 16 / 32 on the light node pairs at 384 threads: 1.13 / 1.16 / 1.19 ms)
};
}  // namespace

struct lec_es_batch_plan {
  size_t k = 0;
  std::vector<Program> progs;
  std::vector<int> jit_of;                // miter -> index into jit_miters, or -1
  std::vector<uint32_t> jit_miters;       // miters run by their own specialised kernel
  std::vector<JitKernel *> jit_kernels;
  std::vector<int> fallback_of;           // miter -> index into fallbacks, or -1
  std::vector<lec_es_plan *> fallbacks;   // live sets beyond the tile kernel's shared memory
  std::vector<size_t> light;              // miters of the tile queue
  uint32_t max_slots = 1;
  int packed_block = 0;                   // block size the device records are encoded for
  size_t recs_cap = 0, loads_cap = 0;
  void *d_loads = nullptr;
  Layout layout;
  int grid = 0;
  size_t smem = 0;
  uint32_t num_tiles = 0;
  void *d_recs = nullptr, *d_miters = nullptr, *d_tiles = nullptr;
  size_t tiles_cap = 0;
  unsigned long long *d_cex = nullptr;
  uint32_t *d_head = nullptr;             // [head, status]
  unsigned long long *d_aux = nullptr;    // per specialised miter: {patterns evaluated, grab counter}
  unsigned long long *h_cex = nullptr;    // pinned
  uint32_t *h_status = nullptr;           // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int branches = kDefaultBranches;
  cudaStream_t side[kMaxBranches] = {};
  cudaEvent_t fork = nullptr, join[kMaxBranches] = {};
  bool pending = false;
  double host_ms = 0, jit_ms = 0, tune_ms = 0;
  XBatchParams params{};
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::map<uint64_t, Layout>> g_tuned;  // cache file -> shape -> layout

void release_graph(lec_es_batch_plan *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void batch_release(lec_es_ctx *c, lec_es_batch_plan *b) {
  if (!b) return;
  release_graph(b);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int i = 0; i < kMaxBranches; i++) {
    if (b->join[i]) cudaEventDestroy(b->join[i]);
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
  }
  if (b->h_cex) cudaFreeHost(b->h_cex);
  if (b->h_status) cudaFreeHost(b->h_status);
  c->arena.free(b->d_recs);
  c->arena.free(b->d_loads);
  c->arena.free(b->d_miters);
  c->arena.free(b->d_tiles);
  c->arena.free(b->d_cex);
  c->arena.free(b->d_head);
  c->arena.free(b->d_aux);
  for (lec_es_plan *p : b->fallbacks) plan_release(c, p);
  delete b;
}

}  // namespace

namespace {
// The own-kernel threshold of the batch being prepared (the split search of
// lec_es_batch_prepare sets it; otherwise kBatchJitMs).
thread_local double t_split_ms = -1.0;
}  // namespace

bool lec::batch_wants_kernel(lec_es_ctx *c, uint32_t n, uint32_t cone_ands, uint32_t luts, uint32_t live) {
  const double th = t_split_ms >= 0 ? t_split_ms : kBatchJitMs;
  return cost_run_ms(c, LEC_ES_TIER_INTERP, cone_ands, n) >= th && luts && live <= kBatchJitLive;
}

namespace {

int compile_all(lec_es_ctx *c, const lec_es_miter *m, size_t k, uint32_t order, bool allow_jit,
                std::vector<Program> &progs) {
  progs.assign(k, Program());
  std::vector<int> rcs(k, LEC_ES_OK);
  const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 16u));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; t++) {
    th.emplace_back([&, t]() {
      for (size_t i = t; i < k; i += nt) {
        MiterView v{m[i].num_pis, m[i].num_ands, m[i].fanins, m[i].out_lit};
        try {
          JitProbe jp{c, allow_jit ? JitProbe::kBatch : JitProbe::kInfo};
          const KernelProbe probe{jit_probe, &jp};
          rcs[i] = compile_program(v, order, c->max_pis, progs[i], allow_jit ? &probe : nullptr);
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

// Stage 1: programs, specialised kernels, fallbacks, packed records, buffers.
int stage_programs(lec_es_ctx *c, lec_es_batch_plan *b, const lec_es_miter *m, size_t k,
                   const lec_es_options *opt) {
  const bool allow_jit = !(opt && (opt->tier == LEC_ES_TIER_INTERP || opt->tier == LEC_ES_TIER_SPILL));
  int rc = compile_all(c, m, k, opt ? opt->order : LEC_ES_ORDER_AUTO, allow_jit, b->progs);
  if (rc) return rc;
  if (cudaSetDevice(c->device) != cudaSuccess) return LEC_ES_ECUDA;
  // live sets the tile kernel holds in shared memory at 64 threads per block
  // (kLaneBytes per slot per thread, a 4 x 512-record ring)
  const uint32_t max_fit64 = (uint32_t)((c->smem_optin - 64 - 4 * 512 * 16) / (64 * kLaneBytes));
  b->jit_of.assign(k, -1);
  b->fallback_of.assign(k, -1);
  for (size_t i = 0; i < k; i++) {
    const Program &g = b->progs[i];
    if (g.slots_elided || (allow_jit && batch_wants_kernel(c, g.n, g.cone_ands, g.lut.count, g.lut.live))) {
      b->jit_of[i] = (int)b->jit_miters.size();
      b->jit_miters.push_back((uint32_t)i);
    } else if (g.num_slots > max_fit64) {
      b->fallback_of[i] = 0;  // index assigned below
    } else {
      b->light.push_back(i);
      b->max_slots = std::max(b->max_slots, g.num_slots);
    }
  }
  // specialised kernels, compiled in parallel
  b->jit_kernels.assign(b->jit_miters.size(), nullptr);
  std::vector<int> jrc(b->jit_miters.size(), LEC_ES_OK);
  const double tj = now_ms();
  const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 16u));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt && !b->jit_miters.empty(); t++) {
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
  // fallbacks: their own global-memory plans
  for (size_t i = 0; i < k; i++) {
    if (b->fallback_of[i] < 0) continue;
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
  b->d_miters = c->arena.alloc(std::max<size_t>(16, k * sizeof(XMiter)));
  b->d_cex = (unsigned long long *)c->arena.alloc(k * 8);
  b->d_head = (uint32_t *)c->arena.alloc(16);
  b->d_aux = (unsigned long long *)c->arena.alloc(std::max<size_t>(16, b->jit_miters.size() * 16));
  if (!b->d_miters || !b->d_cex || !b->d_head || !b->d_aux) return LEC_ES_ENOMEM;
  if (cudaMallocHost((void **)&b->h_cex, k * 8) != cudaSuccess ||
      cudaMallocHost((void **)&b->h_status, 16) != cudaSuccess)
    return LEC_ES_ENOMEM;
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return LEC_ES_ECUDA;
  if (const char *e = getenv("LEC_ES_BATCH_BRANCHES")) b->branches = std::max(1, std::min(kMaxBranches, atoi(e)));
  for (int i = 0; i < b->branches; i++)
    if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
      return LEC_ES_ECUDA;
  return LEC_ES_OK;
}

// Stage 2: tiles, kernel geometry and the captured graph for one layout.
// With light_only the graph holds just the tile queue (for timing layouts).
int stage_layout(lec_es_ctx *c, lec_es_batch_plan *b, const Layout &L, int grid_override, bool light_only) {
  release_graph(b);
  b->layout = L;
  b->smem = batch_w_smem_bytes(b->max_slots, L.block, L.ring_recs);
  if (b->smem > (size_t)c->smem_optin) return LEC_ES_ETOOBIG;
  // the limit is a property of the kernel function, which the request
  // server's grouped launches set too: both set the device's maximum
  if (configure_batch_w(L.block, (size_t)c->smem_optin) != 0) return LEC_ES_ECUDA;
  const int bps = std::max(1, batch_w_blocks_per_sm(L.block, b->smem));
  b->grid = grid_override > 0 ? grid_override : c->sm_count * bps;
  cudaStream_t st = c->stream;
  const size_t k = b->k;
  // records encoded for this block size (byte offsets depend on it)
  if (b->packed_block != L.block) {
    std::vector<XMiter> mt(k, XMiter{});
    std::vector<XRec> arec;
    std::vector<XLoad> aload;
    std::vector<XRec> xr;
    std::vector<XLoad> xl;
    for (size_t i : b->light) {
      XMiter &x = mt[i];
      encode_w(b->progs[i], L.block, xr, xl, x.out_off, false);  // the tile queue forwards
      x.rec_off = (uint32_t)arec.size();
      x.nrec = (uint32_t)xr.size();
      x.load_off = (uint32_t)aload.size();
      x.nload = (uint32_t)xl.size();
      x.out_compl = b->progs[i].out_compl;
      x.n = b->progs[i].n;
      arec.insert(arec.end(), xr.begin(), xr.end());
      aload.insert(aload.end(), xl.begin(), xl.end());
    }
    if (arec.size() > 0xFFFFFFF0ull || aload.size() > 0xFFFFFFF0ull) return LEC_ES_ETOOBIG;
    if (arec.size() > b->recs_cap) {
      c->arena.free(b->d_recs);
      b->recs_cap = std::max<size_t>(arec.size(), 16);
      b->d_recs = c->arena.alloc(b->recs_cap * sizeof(XRec));
      if (!b->d_recs) return LEC_ES_ENOMEM;
    }
    if (aload.size() > b->loads_cap) {
      c->arena.free(b->d_loads);
      b->loads_cap = std::max<size_t>(aload.size(), 16);
      b->d_loads = c->arena.alloc(b->loads_cap * sizeof(XLoad));
      if (!b->d_loads) return LEC_ES_ENOMEM;
    }
    if (!b->d_recs) {
      b->recs_cap = 16;
      b->d_recs = c->arena.alloc(16 * sizeof(XRec));
    }
    if (!b->d_loads) {
      b->loads_cap = 16;
      b->d_loads = c->arena.alloc(16 * sizeof(XLoad));
    }
    if (!b->d_recs || !b->d_loads) return LEC_ES_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (!arec.empty()) e = cudaMemcpyAsync(b->d_recs, arec.data(), arec.size() * sizeof(XRec), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !aload.empty())
      e = cudaMemcpyAsync(b->d_loads, aload.data(), aload.size() * sizeof(XLoad), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_miters, mt.data(), k * sizeof(XMiter), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LEC_ES_ECUDA;
    b->packed_block = L.block;
  }
  // tiles sized by cost (records x words), big miters first, each miter's
  // tiles in ascending pattern order
  auto cost = [&](size_t i) { return (double)b->progs[i].recs.size() * (double)num_words(b->progs[i].n); };
  double total = 0;
  std::vector<size_t> idx(b->light);
  for (size_t i : idx) total += cost(i);
  std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cost(x) > cost(y); });
  const double target = std::max(1.0, total / ((double)b->grid * (double)L.granularity));
  std::vector<XTile> tiles;
  for (size_t i : idx) {
    const uint64_t W = num_words(b->progs[i].n);
    uint64_t tw = (uint64_t)(target / std::max<size_t>(1, b->progs[i].recs.size()));
    tw = ((tw + L.block - 1) / L.block) * L.block;
    tw = std::max<uint64_t>(tw, (uint64_t)L.block);
    for (uint64_t w0 = 0; w0 < W; w0 += tw) {
      XTile t{};
      t.miter = (uint32_t)i;
      t.word_begin = w0;
      t.word_end = std::min(W, w0 + tw);
      tiles.push_back(t);
    }
  }
  if (tiles.size() > 0xFFFFFFF0ull) return LEC_ES_ETOOBIG;
  b->num_tiles = (uint32_t)tiles.size();
  if (tiles.size() > b->tiles_cap) {
    c->arena.free(b->d_tiles);
    b->tiles_cap = std::max<size_t>(tiles.size(), 16);
    b->d_tiles = c->arena.alloc(b->tiles_cap * sizeof(XTile));
    if (!b->d_tiles) return LEC_ES_ENOMEM;
  }
  if (!tiles.empty() &&
      (cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(XTile), cudaMemcpyHostToDevice, st) !=
           cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return LEC_ES_ECUDA;
  XBatchParams &bp = b->params;
  bp.recs = (const XRec *)b->d_recs;
  bp.loads = (const XLoad *)b->d_loads;
  bp.miters = (const XMiter *)b->d_miters;
  bp.tiles = (const XTile *)b->d_tiles;
  bp.num_tiles = b->num_tiles;
  bp.ring_recs = L.ring_recs;
  bp.cex = b->d_cex;
  bp.head = b->d_head;
  bp.status = b->d_head + 1;
  bp.cancel = nullptr;
  // specialised kernels by descending work, dealt round robin to the branches
  std::vector<size_t> jorder(light_only ? 0 : b->jit_miters.size());
  for (size_t j = 0; j < jorder.size(); j++) jorder[j] = j;
  std::stable_sort(jorder.begin(), jorder.end(), [&](size_t x, size_t y) {
    const Program &gx = b->progs[b->jit_miters[x]], &gy = b->progs[b->jit_miters[y]];
    return (double)gx.lut.count * num_chunks(gx.n) > (double)gy.lut.count * num_chunks(gy.n);
  });
  int lerr = 0;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return LEC_ES_ECUDA;
  cudaMemsetAsync(b->d_cex, 0xFF, k * 8, st);
  cudaMemsetAsync(b->d_head, 0, 16, st);
  if (!b->jit_miters.empty()) cudaMemsetAsync(b->d_aux, 0, b->jit_miters.size() * 16, st);
  // fork: branch 0 runs the tile queue; the specialised kernels are dealt to
  // branches 1, 2, 3, 0, ... so small kernels overlap instead of queueing
  cudaEventRecord(b->fork, st);
  for (int i = 0; i < b->branches; i++) cudaStreamWaitEvent(b->side[i], b->fork, 0);
  if (b->num_tiles) lerr = launch_batch_w(bp, L.block, b->grid, b->smem, b->side[0]);
  for (size_t q = 0; q < jorder.size() && !lerr; q++) {
    const size_t j = jorder[q];
    const uint32_t i = b->jit_miters[j];
    JitKernel *kk = b->jit_kernels[j];
    uint64_t cb = 0, ce = num_chunks(b->progs[i].n), grabs = ~0ull;
    unsigned long long *cex = b->d_cex + i, *ev = b->d_aux + 2 * j, *next = b->d_aux + 2 * j + 1;
    uint64_t grid = 1, rep = 1, q0 = 0, qend = 0;
    bool strided = false;
    jit_geometry(kk, ce - cb, c->sm_count, &grid, &rep, &strided);
    if (strided) next = nullptr;  // grabs by static stride: no counter
    jit_grab_range(kk, rep, cb, ce, &q0, &qend);
    void *args[] = {&cb, &ce, &cex, &ev, &next, &grabs, &rep, &q0, &qend};
    if (cudaLaunchKernel((const void *)kk->kern, dim3((unsigned)grid), dim3(kk->block), args, kk->dyn_smem,
                         b->side[(q + 1) % b->branches]) != cudaSuccess)
      lerr = 1;
  }
  for (int i = 0; i < b->branches; i++) {
    cudaEventRecord(b->join[i], b->side[i]);
    cudaStreamWaitEvent(st, b->join[i], 0);
  }
  cudaMemcpyAsync(b->h_cex, b->d_cex, k * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(b->h_status, b->d_head, 16, cudaMemcpyDeviceToHost, st);
  e = cudaStreamEndCapture(st, &b->graph);
  if (e != cudaSuccess || lerr) return LEC_ES_ECUDA;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return LEC_ES_ECUDA;
  return LEC_ES_OK;
}

// Batch shape for the tuning cache: log2 of light miters and light work,
// largest live set in steps of 16, SM count.
uint64_t shape_key(lec_es_ctx *c, const lec_es_batch_plan *b) {
  double work = 0;
  for (size_t i : b->light) work += (double)b->progs[i].recs.size() * (double)num_words(b->progs[i].n);
  const uint64_t lk = (uint64_t)std::log2((double)b->light.size() + 1.0);
  const uint64_t lw = (uint64_t)std::log2(work + 1.0);
  return (lk << 48) | (lw << 32) | ((uint64_t)(b->max_slots / 16) << 16) | (uint64_t)c->sm_count;
}

std::string tune_file(lec_es_ctx *c) { return c->jit_dir.empty() ? std::string() : c->jit_dir + "/batch_layouts.txt"; }

bool tuned_lookup(lec_es_ctx *c, uint64_t key, Layout &L) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const std::string f = tune_file(c);
  auto &m = g_tuned[f];
  if (m.empty() && !f.empty()) {
    std::ifstream in(f);
    unsigned long long kk;
    int blk;
    unsigned ring, gran;
    while (in >> std::hex >> kk >> std::dec >> blk >> ring >> gran) m[kk] = Layout{blk, ring, gran};
  }
  auto it = m.find(key);
  if (it == m.end()) return false;
  L = it->second;
  return true;
}

void tuned_store(lec_es_ctx *c, uint64_t key, const Layout &L) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const std::string f = tune_file(c);
  g_tuned[f][key] = L;
  if (!f.empty()) {
    std::ofstream out(f, std::ios::app);
    out << std::hex << (unsigned long long)key << std::dec << " " << L.block << " " << L.ring_recs << " "
        << L.granularity << "\n";
  }
}

// Threads per tile pass for the batch's largest live set: the largest power
// of two up to 256 that fits, replaced by a multiple of 128 threads up to
// kMaxWordBlock that keeps at least a quarter more warps on an SM.  Whole
// multiples of 128 give each of the SM's four schedulers the same number of
// warps: on the 3,630 light node-pair miters (62 live slots: one 256-thread
// block of 143 KB per SM) 384 threads ran 1.16 ms against 1.27 ms at 256,
// while 416 threads (13 warps, one scheduler with four) ran 1.22 ms.
int widest_batch_block(lec_es_ctx *c, uint32_t max_slots, uint32_t ring) {
  int base = 256;
  while (base > 64 && batch_w_smem_bytes(max_slots, base, ring) > (size_t)c->smem_optin) base /= 2;
  if (configure_batch_w(base, (size_t)c->smem_optin) != 0) return base;
  auto warps = [&](int blk) { return batch_w_blocks_per_sm(blk, batch_w_smem_bytes(max_slots, blk, ring)) * blk / 32; };
  const int w0 = warps(base);
  int best = base, best_w = w0;
  for (int blk = 128; blk <= kMaxWordBlock; blk += 128) {
    if (batch_w_smem_bytes(max_slots, blk, ring) > (size_t)c->smem_optin) continue;
    const int w = warps(blk);
    if (4 * w >= 5 * w0 && (w > best_w || (w == best_w && blk > best))) {
      best = blk;
      best_w = w;
    }
  }
  return best;
}

// Time each candidate layout on the tile queue alone (graph replays: one
// warm-up, then the median of three) and keep the fastest.
int autotune(lec_es_ctx *c, lec_es_batch_plan *b, int grid_override, Layout &best) {
  const double t0 = now_ms();
  const uint64_t key = shape_key(c, b);
  if (tuned_lookup(c, key, best)) return LEC_ES_OK;
  float best_ms = 1e30f;
  bool have = false;
  cudaStream_t st = c->stream;
  for (uint32_t ring : {128u, 256u, 512u}) {
    std::vector<int> blocks{widest_batch_block(c, b->max_slots, ring)};
    for (int blk : {256, 128, 64})
      if (blk != blocks[0]) blocks.push_back(blk);
    for (int blk : blocks)
      for (uint32_t gran : {4u, 8u, 16u, 64u}) {
        Layout L{blk, ring, gran};
        if (batch_w_smem_bytes(b->max_slots, blk, ring) > (size_t)c->smem_optin) continue;
        if (stage_layout(c, b, L, grid_override, true) != LEC_ES_OK) continue;
        float t[3] = {0, 0, 0};
        bool ok = true;
        for (int r = 0; r < 4 && ok; r++) {
          cudaEventRecord(b->e0, st);
          ok = cudaGraphLaunch(b->exec, st) == cudaSuccess;
          cudaEventRecord(b->e1, st);
          ok = ok && wait_event(b->e1, c->timeout_s) == LEC_ES_OK;
          if (ok && r > 0) cudaEventElapsedTime(&t[r - 1], b->e0, b->e1);
        }
        if (!ok || cudaStreamSynchronize(st) != cudaSuccess || b->h_status[1]) return LEC_ES_ECUDA;
        std::sort(t, t + 3);
        if (!have || t[1] < best_ms) {
          best_ms = t[1];
          best = L;
          have = true;
        }
      }
  }
  if (!have) return LEC_ES_ETOOBIG;
  tuned_store(c, key, best);
  b->tune_ms = now_ms() - t0;
  return LEC_ES_OK;
}

}  // namespace

namespace {
int batch_prepare_one(lec_es_ctx *c, const lec_es_miter *m, size_t k, const lec_es_options *opt,
                      lec_es_batch_plan **out);
}  // namespace

// With LEC_ES_FLAG_AUTOTUNE the split between miters that get their own
// specialised kernel (a node of the CUDA graph each, about 6 us of launch
// overhead) and miters left to the tile queue is searched too: the batch is
// prepared for a few own-kernel thresholds on the predicted interpreter
// time, each replayed and timed, and the fastest is kept.  On the 4,096
// node pairs the base threshold wins; on a batch of heavier miters (10-28
// PIs) thousands of own kernels would make the graph launch-bound.
constexpr double kSplitCandidatesMs[] = {kBatchJitMs, 0.05, 0.12, 0.3};

extern "C" int lec_es_batch_prepare(lec_es_ctx *c, const lec_es_miter *m, size_t k, const lec_es_options *opt,
                                    lec_es_batch_plan **out) {
  if (!c || !m || !out || k == 0 || k > 0xFFFFFFFFull) return LEC_ES_EINVAL;
  *out = nullptr;
  const bool interp_only = opt && (opt->tier == LEC_ES_TIER_INTERP || opt->tier == LEC_ES_TIER_SPILL);
  if (!(opt && (opt->flags & LEC_ES_FLAG_AUTOTUNE)) || interp_only) return batch_prepare_one(c, m, k, opt, out);
  const double t0 = now_ms();
  lec_es_batch_plan *best = nullptr;
  double best_ms = 1e300;
  double jit_ms = 0;
  for (double th : kSplitCandidatesMs) {
    lec_es_batch_plan *b = nullptr;
    t_split_ms = th;
    int rc = batch_prepare_one(c, m, k, opt, &b);
    t_split_ms = -1.0;
    if (rc) {
      if (best) lec_es_batch_free(c, best);
      return rc;
    }
    jit_ms += b->jit_ms;
    double ms = 1e300;
    for (int r = 0; r < 3 && !rc; r++) {  // the least of three replays
      const double ts = now_ms();
      rc = lec_es_batch_run_async(c, b);
      if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LEC_ES_ECUDA;
      ms = std::min(ms, now_ms() - ts);
    }
    if (rc) {
      lec_es_batch_free(c, b);
      if (best) lec_es_batch_free(c, best);
      return rc;
    }
    const bool no_kernels = b->jit_miters.empty();  // a higher threshold cannot change the split
    if (ms < best_ms) {
      if (best) lec_es_batch_free(c, best);
      best = b;
      best_ms = ms;
    } else {
      lec_es_batch_free(c, b);
    }
    if (no_kernels) break;
  }
  best->host_ms = now_ms() - t0;
  best->tune_ms = best->host_ms - jit_ms;
  best->jit_ms = jit_ms;
  *out = best;
  return LEC_ES_OK;
}

namespace {
int batch_prepare_one(lec_es_ctx *c, const lec_es_miter *m, size_t k, const lec_es_options *opt,
                      lec_es_batch_plan **out) {
  *out = nullptr;
  const double t0 = now_ms();
  lec_es_batch_plan *b = new (std::nothrow) lec_es_batch_plan();
  if (!b) return LEC_ES_ENOMEM;
  b->k = k;
  int rc = stage_programs(c, b, m, k, opt);
  const int grid_override = opt && opt->grid_blocks ? (int)opt->grid_blocks : 0;
  Layout L;
  if (!rc) {
    if (opt && (opt->flags & LEC_ES_FLAG_AUTOTUNE) && !b->light.empty()) {
      rc = autotune(c, b, grid_override, L);
    } else {
      if (opt && opt->stage_records) L.ring_recs = opt->stage_records;
      if (opt && opt->tile_granularity) L.granularity = opt->tile_granularity;
      if (L.ring_recs < 2 || (L.ring_recs & 1) || L.ring_recs > 2048) rc = LEC_ES_EINVAL;
      if (opt && opt->block_threads) {
        L.block = (int)opt->block_threads;
        if (L.block < 64 || !word_block_ok(L.block)) rc = LEC_ES_EINVAL;
        // a block that does not fit shared memory falls back to smaller ones
        while (!rc && L.block > 64 && batch_w_smem_bytes(b->max_slots, L.block, L.ring_recs) > (size_t)c->smem_optin)
          L.block -= 32;
      } else if (!rc) {
        L.block = widest_batch_block(c, b->max_slots, L.ring_recs);
      }
    }
  }
  if (!rc) rc = stage_layout(c, b, L, grid_override, false);
  if (rc) {
    cudaStreamSynchronize(c->stream);
    batch_release(c, b);
    return rc;
  }
  b->host_ms = now_ms() - t0;
  *out = b;
  return LEC_ES_OK;
}
}  // namespace

extern "C" int lec_es_batch_info(const lec_es_batch_plan *b, lec_es_batch_layout *info) {
  if (!b || !info) return LEC_ES_EINVAL;
  memset(info, 0, sizeof(*info));
  info->miters = (uint32_t)b->k;
  info->jit_miters = (uint32_t)b->jit_miters.size();
  info->fallback_miters = (uint32_t)b->fallbacks.size();
  info->tile_miters = (uint32_t)b->light.size();
  info->tiles = b->num_tiles;
  info->block_threads = (uint32_t)b->layout.block;
  info->stage_records = b->layout.ring_recs;
  info->tile_granularity = b->layout.granularity;
  info->grid_blocks = (uint32_t)b->grid;
  info->prepare_ms = b->host_ms;
  info->jit_ms = b->jit_ms;
  info->tune_ms = b->tune_ms;
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
