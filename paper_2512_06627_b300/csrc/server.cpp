// server.cpp -- served exact simulation: continuous batching of ES requests.
//
// A request is one miter.  lec_es_submit copies the miter's output cone
// (a self-contained, renumbered AIG of the cone alone) in the caller's
// thread and returns a ticket; a pool of front-end threads then compiles it
// (support, order, reference-count slots, table cover) and queues it for
// admission, so submissions of many small cones are not bound by one host
// thread.  Errors the front end finds later (too many value slots) are
// reported by lec_es_poll / lec_es_wait.  A dispatcher thread
//   * admits queued requests in arrival order while the requests on the GPU
//     hold less than the slot budget (value slots x resident 64-pattern words
//     x 8 bytes: the live set a request keeps per word in flight) and fewer
//     than max_inflight run;
//   * launches each admitted request on one of several CUDA streams, so work
//     of requests that arrive while others run overlaps on the device; small
//     requests go to high-priority streams and every grid is sized so blocks
//     retire after a few passes, letting the block scheduler interleave them;
//   * keeps programs resident: interpreter records are uploaded once per
//     distinct program, and specialised (JIT) kernels are compiled in the
//     background on first sight and used once ready (the interpreter runs a
//     program until then);
//   * groups small interpreter requests: consecutive queued requests whose
//     predicted time is below kGroupMs run together as one launch of the
//     tile-queue kernel (the batch path's es_batch_w) over their (request,
//     word range) tiles, their programs uploaded in one copy -- so a stream
//     of many small cones costs one launch per group, not per request;
//   * retires requests whose completion event has fired, releasing their
//     budget.  Counterexamples end a request early through the same minimum
//     that drives early exit; cancellation writes 0 into that word, which
//     stops the kernel at its next pass.
// Results are identical to lec_es_check: the same kernels over the same
// pattern space, with the exact lowest-counterexample rule.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

namespace lec {

namespace {

constexpr int kStreams = 8;                    // half high priority, half low
constexpr double kSmallMs = 5.0;               // predicted device time below this is "small"

struct Slot {
  unsigned long long *d_res = nullptr;  // kResWords result words
  unsigned long long *h_res = nullptr;  // pinned
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  // recorded on the control stream after a cancellation's zero write into
  // d_res; the slot's next reset copy waits for it, so a late zero can never
  // land on the next request's counterexample word
  cudaEvent_t zeroed = nullptr;
  bool zero_pending = false;
  bool busy = false;
};

struct Resident {  // device copy of one program's records (word-wide kernel)
  void *d_recs = nullptr;
  void *d_loads = nullptr;
  uint32_t nrec = 0, nload = 0, out_off = 0;
  PlanGeom geom;
  bool shared_block = false;   // part of a group's upload block (freed with it)
  cudaEvent_t ready = nullptr; // recorded on the group stream after that upload
};

// Grouped requests (see the header): up to kGroupMax requests and
// kGroupTiles tiles per launch, programs encoded for kGroupBlock threads.
constexpr double kGroupMs = 0.1;
constexpr int kGroupMax = 512;
constexpr int kGroupTiles = 16384;
constexpr int kGroupBlock = 256;
constexpr uint32_t kGroupRing = 256;
constexpr uint64_t kGroupTileWords = (uint64_t)kGroupBlock * 8;  // 8 passes of a block per tile
constexpr size_t kGroupStage = 8u << 20;                         // pinned staging of new programs' records
constexpr int kGroupSlots = 3;

struct Request;
struct GroupSlot {
  // one pinned and one device buffer: [miters | tiles | cex words | head, status]
  uint8_t *h_buf = nullptr, *d_buf = nullptr;
  uint8_t *h_stage = nullptr;  // records and loads of programs uploaded with this group
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  std::vector<Request *> members;
  bool busy = false;
};
constexpr size_t kGroupMiterBytes = (size_t)kGroupMax * sizeof(XMiter);
constexpr size_t kGroupTileBytes = (size_t)kGroupTiles * sizeof(XTile);
constexpr size_t kGroupCexBytes = (size_t)kGroupMax * 8;
constexpr size_t kGroupBufBytes = kGroupMiterBytes + kGroupTileBytes + kGroupCexBytes + 16;

struct Request {
  enum State { PREPARING, QUEUED, RUNNING, DONE, CANCELLED, FAILED };
  uint64_t ticket = 0;
  CompactMiter cone;  // until the front end has run
  Program prog;
  State state = QUEUED;
  int slot = -1;
  int stream = -1;
  int group = -1;          // group slot of a grouped request
  uint32_t group_at = 0;   // its index in the group
  size_t reserve = 0;
  double t_submit = 0, t_done = 0;
  std::atomic<bool> cancel{false};  // set under the server mutex, read by the dispatcher without it
  bool cancel_sent = false;
  int err = 0;
  uint32_t tier = 0;
  lec_es_result res{};
};

}  // namespace

struct Server {
  lec_es_ctx *c = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_prep;
  std::deque<uint64_t> prep;   // tickets waiting for the front end
  int prep_waiting = 0;        // front-end threads asleep on cv_prep
  bool disp_waiting = false;   // the dispatcher asleep on cv_work
  // (a wake-up is sent only to a thread that sleeps: no system call per request in a burst)
  std::vector<std::thread> prep_threads;
  std::deque<uint64_t> queue;  // compiled, waiting for admission
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request *> running;  // launched one by one (the dispatcher's own list)
  std::vector<Slot> slots;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_load;
  cudaStream_t ctl = nullptr;
  unsigned long long *h_zero = nullptr;
  std::map<std::pair<uint64_t, uint64_t>, Resident> resident;  // by both structure hashes
  std::vector<void *> shared_blocks;  // group upload blocks of resident programs
  std::vector<cudaEvent_t> group_events;  // their copies' completion events
  GroupSlot groups[kGroupSlots];
  cudaStream_t group_stream = nullptr;
  size_t group_smem_max = 0;
  size_t used = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
};

namespace {

size_t reserve_bytes(lec_es_ctx *c, const Program &g) {
  const uint64_t words = num_words(g.n);
  const uint64_t in_flight_words = (uint64_t)c->sm_count * 2048 / 2;  // 2048 lanes per SM, 2 lanes a word
  const uint64_t rw = std::min(words, in_flight_words);
  return (size_t)g.num_slots * rw * 8 + (size_t)g.num_records * sizeof(Rec);
}

void finish(Server *s, Request *r, Request::State st) {
  r->state = st;
  r->t_done = now_ms();
  s->cv_done.notify_all();
}

// Launch one admitted request.  Called with s->mu held.
int launch(Server *s, Request *r) {
  lec_es_ctx *c = s->c;
  const Program &g = r->prog;
  const uint64_t C = num_chunks(g.n);
  JitKernel *k = nullptr;
  if (g.slots_elided || jit_auto_tier(c, g, C) == LEC_ES_TIER_JIT) k = jit_lookup_or_schedule(c, g);
  if (g.slots_elided && !k) return LEC_ES_EINVAL;  // found at submission; kernels are never evicted
  // stream: least loaded within the request's priority class, from the ES
  // time model on the tier it will run
  const double predicted = cost_run_ms(c, k ? LEC_ES_TIER_JIT : LEC_ES_TIER_INTERP, g.cone_ands, g.n, k ? k->model_lop3 : 0.0);
  const int half = kStreams / 2;
  const int lo = predicted < kSmallMs ? 0 : half;
  int best = lo;
  for (int i = lo; i < lo + half; i++)
    if (s->stream_load[i] < s->stream_load[best]) best = i;
  cudaStream_t st = s->streams[best];
  // result slot
  int si = -1;
  for (size_t i = 0; i < s->slots.size(); i++)
    if (!s->slots[i].busy) {
      si = (int)i;
      break;
    }
  if (si < 0) return LEC_ES_EBUSY;
  Slot &sl = s->slots[si];

  Resident *res = nullptr;
  if (!k) {
    auto it = s->resident.find({g.hash, g.hash2});
    if (it == s->resident.end()) {
      Resident rr;
      if (!choose_word_geometry(c, g, nullptr, rr.geom)) return LEC_ES_ETOOBIG;  // slots stay on chip
      std::vector<XRec> xr;
      std::vector<XLoad> xl;
      encode_w(g, rr.geom.block, xr, xl, rr.out_off);
      rr.nrec = (uint32_t)xr.size();
      rr.nload = (uint32_t)xl.size();
      rr.d_recs = c->arena.alloc(std::max<size_t>(16, xr.size() * sizeof(XRec)));
      rr.d_loads = c->arena.alloc(std::max<size_t>(16, xl.size() * sizeof(XLoad)));
      if (!rr.d_recs || !rr.d_loads) {
        c->arena.free(rr.d_recs);
        c->arena.free(rr.d_loads);
        return LEC_ES_ENOMEM;
      }
      cudaError_t e = cudaSuccess;
      if (!xr.empty()) e = cudaMemcpyAsync(rr.d_recs, xr.data(), xr.size() * sizeof(XRec), cudaMemcpyHostToDevice, s->ctl);
      if (e == cudaSuccess && !xl.empty())
        e = cudaMemcpyAsync(rr.d_loads, xl.data(), xl.size() * sizeof(XLoad), cudaMemcpyHostToDevice, s->ctl);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctl);
      if (e != cudaSuccess) {
        c->arena.free(rr.d_recs);
        c->arena.free(rr.d_loads);
        return LEC_ES_ECUDA;
      }
      it = s->resident.emplace(std::make_pair(g.hash, g.hash2), rr).first;
    }
    res = &it->second;
    if (res->ready && cudaStreamWaitEvent(st, res->ready, 0) != cudaSuccess) return LEC_ES_ECUDA;
  }
  if (sl.zero_pending) {  // a cancellation's zero write into this slot must land first
    if (cudaStreamWaitEvent(st, sl.zeroed, 0) != cudaSuccess) return LEC_ES_ECUDA;
    sl.zero_pending = false;
  }
  if (cudaMemcpyAsync(sl.d_res, c->h_init, kResWords * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LEC_ES_ECUDA;
  cudaEventRecord(sl.e0, st);
  int err;
  if (k) {
    // each warp grabs at most 8 times, so blocks retire and other requests
    // interleave; enough blocks that the grabs cover every chunk
    uint64_t cb = 0, ce = C, grabs = 8;
    unsigned long long *cex = sl.d_res, *ev = sl.d_res + 1, *next = sl.d_res + 3;
    // passes per grab as for a full-GPU launch of this kernel
    uint64_t rep = jit_reps(k, C, (uint64_t)c->sm_count * k->blocks_per_sm), q0 = 0, qend = 0;
    jit_grab_range(k, rep, cb, ce, &q0, &qend);
    void *args[] = {&cb, &ce, &cex, &ev, &next, &grabs, &rep, &q0, &qend};
    const uint64_t per_block = (uint64_t)(k->block / 32) * 32 * grabs * rep;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((C + per_block - 1) / per_block, 1u << 30));
    err = cudaLaunchKernel((const void *)k->kern, dim3((unsigned)grid), dim3(k->block), args, k->dyn_smem, st) ==
                  cudaSuccess
              ? 0
              : 1;
    r->tier = LEC_ES_TIER_JIT;
  } else {
    XParams xp{};
    xp.recs = (const XRec *)res->d_recs;
    xp.loads = (const XLoad *)res->d_loads;
    xp.nrec = res->geom.nrec_padded;
    xp.nload = res->nload;
    xp.step = g.step;
    xp.out_off = res->out_off;
    xp.out_compl = g.out_compl;
    xp.n = g.n;
    xp.ring_recs = res->geom.ring_recs;
    xp.resident = res->geom.resident;
    xp.word_begin = 0;
    xp.word_end = num_words(g.n);
    xp.cex = sl.d_res;
    xp.evaluated = sl.d_res + 1;
    xp.status = (uint32_t *)(sl.d_res + 2);
    // a few passes per block, so blocks retire and other requests interleave
    const uint64_t lanes = kLaneBytes == 8 ? xp.word_end : num_chunks(g.n);
    const uint64_t passes = (lanes + res->geom.block - 1) / res->geom.block;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((passes + 3) / 4, 1u << 30));
    err = launch_interp_w(xp, res->geom.block, (int)grid, res->geom.smem, st);
    r->tier = LEC_ES_TIER_INTERP;
  }
  if (err) return LEC_ES_ECUDA;
  cudaEventRecord(sl.e1, st);
  cudaMemcpyAsync(sl.h_res, sl.d_res, kResWords * 8, cudaMemcpyDeviceToHost, st);
  cudaEventRecord(sl.e2, st);
  sl.busy = true;
  r->slot = si;
  r->stream = best;
  s->stream_load[best]++;
  return LEC_ES_OK;
}

// The final state of a finished single launch (its result filled in); the
// caller finishes the request under the server mutex.
Request::State retire(Server *s, Request *r) {
  Slot &sl = s->slots[r->slot];
  const Program &g = r->prog;
  lec_es_result &o = r->res;
  memset(&o, 0, sizeof(o));
  o.support_n = g.n;
  for (uint32_t q = 0; q < g.n; q++) o.support[q] = g.support[q];
  o.cone_ands = g.cone_ands;
  o.num_slots = g.num_slots;
  o.tier = r->tier;
  o.order = g.order;
  o.words_checked = num_words(g.n);
  float ms = 0;
  cudaEventElapsedTime(&ms, sl.e0, sl.e1);
  o.device_ms = ms;
  o.cex = sl.h_res[0];
  o.verdict = o.cex == UINT64_MAX ? LEC_ES_EQUIVALENT : LEC_ES_NONEQUIVALENT;
  const uint32_t status = (uint32_t)sl.h_res[2];
  sl.busy = false;
  s->stream_load[r->stream]--;
  s->used -= r->reserve;
  r->t_done = now_ms();
  o.latency_ms = r->t_done - r->t_submit;
  if (r->cancel) return Request::CANCELLED;
  if (status) {
    r->err = (status & DEV_WAIT_TIMEOUT) ? LEC_ES_EDEVICE_WAIT : LEC_ES_ECUDA;
    return Request::FAILED;
  }
  return Request::DONE;
}

// A request the dispatcher is done with, and its final state (applied under
// the server mutex).
struct Finished {
  Request *r;
  Request::State st;
};

// Front-end thread: compiles submitted cones and queues them for admission.
void prep_worker(Server *s) {
  lec_es_ctx *c = s->c;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->prep_waiting++;
    s->cv_prep.wait(lk, [&] { return s->stop || !s->prep.empty(); });
    s->prep_waiting--;
    if (s->stop) return;
    const uint64_t t = s->prep.front();
    s->prep.pop_front();
    auto it = s->reqs.find(t);
    if (it == s->reqs.end()) continue;
    Request *r = it->second.get();  // stays put: a preparing request is never collected
    if (r->cancel) {
      finish(s, r, Request::CANCELLED);
      continue;
    }
    CompactMiter cone = std::move(r->cone);
    lk.unlock();
    const double t0 = now_ms();
    Program g;
    int rc;
    try {
      JitProbe jp{c, JitProbe::kAuto};
      const KernelProbe probe{jit_probe, &jp, jit_want_cover};
      rc = compile_program(cone.view(), LEC_ES_ORDER_AUTO, c->max_pis, g, &probe);
      if (!rc) g.support = cone.support;
    } catch (const std::bad_alloc &) {
      rc = LEC_ES_ENOMEM;
    }
    const double front_ms = now_ms() - t0;
    lk.lock();
    r->res.host_ms += front_ms;
    if (rc) {
      r->err = rc;
      finish(s, r, Request::FAILED);
    } else if (r->cancel) {
      finish(s, r, Request::CANCELLED);
    } else {
      r->prog = std::move(g);
      r->state = Request::QUEUED;
      s->queue.push_back(t);
      if (s->disp_waiting) s->cv_work.notify_one();
    }
  }
}

// Whether r runs in a group: a slot program (the front end built one),
// predicted below kGroupMs on the interpreter, a live set the group kernel
// holds, and a program not already resident in another block size.
bool groupable(Server *s, Request *r) {
  lec_es_ctx *c = s->c;
  const Program &g = r->prog;
  if (g.slots_elided || g.recs.empty()) return false;
  // small on the interpreter: grouped even when a specialised kernel is held
  // (one launch for the whole group costs less than one launch each)
  if (cost_run_ms(c, LEC_ES_TIER_INTERP, g.cone_ands, g.n) >= kGroupMs) return false;
  const size_t fit =
      (s->group_smem_max - batch_w_smem_bytes(0, kGroupBlock, kGroupRing)) / ((size_t)kGroupBlock * kLaneBytes);
  if (g.num_slots > fit || (size_t)g.recs.size() * 32u > kGroupStage) return false;
  if ((num_words(g.n) + kGroupTileWords - 1) / kGroupTileWords > (uint64_t)kGroupTiles) return false;
  auto it = s->resident.find({g.hash, g.hash2});
  if (it != s->resident.end()) return it->second.geom.block == kGroupBlock;
  PlanGeom geom;  // a program uploaded for a group is encoded for kGroupBlock threads
  return choose_word_geometry(c, g, nullptr, geom) && geom.block == kGroupBlock;
}

int free_group(Server *s) {
  for (int i = 0; i < kGroupSlots; i++)
    if (!s->groups[i].busy) return i;
  return -1;
}

// Take the longest run of groupable requests at the head of `staged` (at
// least one) into group slot gi and launch them as one tile-queue kernel:
// programs not yet resident are encoded into the slot's pinned staging and
// uploaded in one copy on the group stream (residents of later launches
// wait for it by its event), then the miter and tile tables, the
// counterexample words, the kernel, and the read-back of the words.
int admit_group(Server *s, int gi, std::deque<Request *> &staged, std::vector<Finished> &finished) {
  lec_es_ctx *c = s->c;
  GroupSlot &G = s->groups[gi];
  cudaStream_t st = s->group_stream;
  XMiter *hm = (XMiter *)G.h_buf;
  XTile *ht = (XTile *)(G.h_buf + kGroupMiterBytes);
  unsigned long long *hc = (unsigned long long *)(G.h_buf + kGroupMiterBytes + kGroupTileBytes);
  struct Fresh {
    std::pair<uint64_t, uint64_t> key;
    size_t rec_at, load_at;
    uint32_t nrec, nload, out_off;
    PlanGeom geom;
  };
  std::vector<Fresh> fresh;
  std::vector<Request *> mem;
  size_t stage = 0, ntiles = 0;
  uint32_t max_slots = 0;
  size_t used = s->used;
  while (!staged.empty() && (int)mem.size() < kGroupMax) {
    Request *r = staged.front();
    if (r->cancel) {
      staged.pop_front();
      finished.push_back({r, Request::CANCELLED});
      continue;
    }
    if (!groupable(s, r)) break;
    const Program &g = r->prog;
    const uint64_t W = num_words(g.n);
    const size_t tiles = (size_t)((W + kGroupTileWords - 1) / kGroupTileWords);
    if (ntiles + tiles > (size_t)kGroupTiles) break;
    r->reserve = reserve_bytes(c, g);
    if (used + r->reserve > c->slot_budget && (!mem.empty() || !s->running.empty())) break;
    const std::pair<uint64_t, uint64_t> key{g.hash, g.hash2};
    bool known = s->resident.count(key) != 0;
    for (const Fresh &f : fresh) known = known || f.key == key;
    if (!known) {
      Fresh f;
      f.key = key;
      if (!choose_word_geometry(c, g, nullptr, f.geom) || f.geom.block != kGroupBlock) break;
      std::vector<XRec> xr;
      std::vector<XLoad> xl;
      encode_w(g, kGroupBlock, xr, xl, f.out_off);
      const size_t rb = (std::max<size_t>(1, xr.size()) * sizeof(XRec) + 255) & ~(size_t)255;
      const size_t lb = (std::max<size_t>(1, xl.size()) * sizeof(XLoad) + 255) & ~(size_t)255;
      if (stage + rb + lb > kGroupStage) break;
      f.rec_at = stage;
      f.load_at = stage + rb;
      f.nrec = (uint32_t)xr.size();
      f.nload = (uint32_t)xl.size();
      memcpy(G.h_stage + f.rec_at, xr.data(), xr.size() * sizeof(XRec));
      memcpy(G.h_stage + f.load_at, xl.data(), xl.size() * sizeof(XLoad));
      stage += rb + lb;
      fresh.push_back(f);
    }
    staged.pop_front();
    used += r->reserve;
    ntiles += tiles;
    max_slots = std::max(max_slots, g.num_slots);
    mem.push_back(r);
  }
  if (mem.empty()) return LEC_ES_EBUSY;
  int rc = LEC_ES_OK;
  if (stage) {
    void *blk = c->arena.alloc(stage);
    cudaEvent_t ready = nullptr;
    if (!blk || cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
      c->arena.free(blk);
      rc = LEC_ES_ENOMEM;
    } else if (cudaMemcpyAsync(blk, G.h_stage, stage, cudaMemcpyHostToDevice, st) != cudaSuccess ||
               cudaEventRecord(ready, st) != cudaSuccess) {
      rc = LEC_ES_ECUDA;
    }
    if (!rc) {
      s->shared_blocks.push_back(blk);
      for (size_t i = 0; i < fresh.size(); i++) {
        Resident rr;
        rr.d_recs = (uint8_t *)blk + fresh[i].rec_at;
        rr.d_loads = (uint8_t *)blk + fresh[i].load_at;
        rr.nrec = fresh[i].nrec;
        rr.nload = fresh[i].nload;
        rr.out_off = fresh[i].out_off;
        rr.geom = fresh[i].geom;
        rr.shared_block = true;
        rr.ready = ready;  // a later single launch of it waits for the copy
        s->resident.emplace(fresh[i].key, rr);
      }
      s->group_events.push_back(ready);
    }
  }
  size_t t = 0;
  for (size_t i = 0; i < mem.size() && !rc; i++) {
    const Program &g = mem[i]->prog;
    const Resident &rr = s->resident.at({g.hash, g.hash2});
    XMiter &x = hm[i];
    x.rec_off = (uint32_t)(((const uint8_t *)rr.d_recs - c->arena.base) / sizeof(XRec));
    x.nrec = rr.nrec;
    x.load_off = (uint32_t)(((const uint8_t *)rr.d_loads - c->arena.base) / sizeof(XLoad));
    x.nload = rr.nload;
    x.out_off = rr.out_off;
    x.out_compl = g.out_compl;
    x.n = g.n;
    x.pad = 0;
    hc[i] = ~0ull;
    const uint64_t W = num_words(g.n);
    for (uint64_t w = 0; w < W; w += kGroupTileWords)
      ht[t++] = XTile{(uint32_t)i, 0u, w, std::min<uint64_t>(W, w + kGroupTileWords)};
  }
  uint32_t *hctl = (uint32_t *)(G.h_buf + kGroupMiterBytes + kGroupTileBytes + kGroupCexBytes);
  hctl[0] = hctl[1] = 0;  // queue head, status
  uint8_t *dm = G.d_buf, *dt = G.d_buf + kGroupMiterBytes, *dc = dt + kGroupTileBytes, *dctl = dc + kGroupCexBytes;
  const size_t nm = mem.size();
  if (!rc && (cudaMemcpyAsync(dm, hm, nm * sizeof(XMiter), cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(dt, ht, t * sizeof(XTile), cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(dc, hc, nm * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(dctl, hctl, 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
    rc = LEC_ES_ECUDA;
  if (!rc) {
    XBatchParams p{};
    p.recs = (const XRec *)c->arena.base;
    p.loads = (const XLoad *)c->arena.base;
    p.miters = (const XMiter *)dm;
    p.tiles = (const XTile *)dt;
    p.num_tiles = (uint32_t)t;
    p.ring_recs = kGroupRing;
    p.cex = (unsigned long long *)dc;
    p.head = (unsigned int *)dctl;
    p.status = (uint32_t *)dctl + 1;
    p.cancel = nullptr;
    const size_t smem = batch_w_smem_bytes(max_slots, kGroupBlock, kGroupRing);
    const int bps = std::max(1, batch_w_blocks_per_sm(kGroupBlock, smem));
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(t, (size_t)c->sm_count * bps));
    // the kernel's shared-memory limit is a property of the function, which
    // batches set too: both set the device's maximum, never less
    if (configure_batch_w(kGroupBlock, (size_t)c->smem_optin) != 0) rc = LEC_ES_ECUDA;
    cudaEventRecord(G.e0, st);
    if (!rc && launch_batch_w(p, kGroupBlock, grid, smem, st) != 0) rc = LEC_ES_ECUDA;
    cudaEventRecord(G.e1, st);
    if (!rc && (cudaMemcpyAsync(hc, dc, nm * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(hctl, dctl, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaEventRecord(G.e2, st) != cudaSuccess))
      rc = LEC_ES_ECUDA;
  }
  if (rc) {
    for (Request *r : mem) {
      r->err = rc;
      finished.push_back({r, Request::FAILED});
    }
    return LEC_ES_OK;  // the members are answered; the queue moves on
  }
  G.busy = true;
  G.members.clear();
  for (size_t i = 0; i < mem.size(); i++) {
    Request *r = mem[i];
    r->group = gi;
    r->group_at = (uint32_t)i;
    r->tier = LEC_ES_TIER_INTERP;
    s->used += r->reserve;
    G.members.push_back(r);
  }
  return LEC_ES_OK;
}

void retire_group(Server *s, int gi, std::vector<Finished> &finished) {
  GroupSlot &G = s->groups[gi];
  const unsigned long long *hc = (const unsigned long long *)(G.h_buf + kGroupMiterBytes + kGroupTileBytes);
  const uint32_t status = ((const uint32_t *)(G.h_buf + kGroupMiterBytes + kGroupTileBytes + kGroupCexBytes))[1];
  float ms = 0;
  cudaEventElapsedTime(&ms, G.e0, G.e1);
  const double now = now_ms();
  for (Request *r : G.members) {
    const Program &g = r->prog;
    lec_es_result &o = r->res;
    const double host_ms = o.host_ms;
    memset(&o, 0, sizeof(o));
    o.support_n = g.n;
    for (uint32_t q = 0; q < g.n; q++) o.support[q] = g.support[q];
    o.cone_ands = g.cone_ands;
    o.num_slots = g.num_slots;
    o.tier = LEC_ES_TIER_INTERP;
    o.order = g.order;
    o.words_checked = num_words(g.n);
    o.device_ms = ms;  // the group's launch
    o.host_ms = host_ms;
    o.cex = hc[r->group_at];
    o.verdict = o.cex == UINT64_MAX ? LEC_ES_EQUIVALENT : LEC_ES_NONEQUIVALENT;
    s->used -= r->reserve;
    r->t_done = now;
    o.latency_ms = r->t_done - r->t_submit;
    if (r->cancel) {
      finished.push_back({r, Request::CANCELLED});
    } else if (status) {
      r->err = (status & DEV_WAIT_TIMEOUT) ? LEC_ES_EDEVICE_WAIT : LEC_ES_ECUDA;
      finished.push_back({r, Request::FAILED});
    } else {
      finished.push_back({r, Request::DONE});
    }
  }
  G.members.clear();
  G.busy = false;
}

// The dispatcher.  The server mutex guards the queue, the request table
// and request states; the dispatcher takes it only to move queued requests
// into its own `staged` list (they become RUNNING: owned by the
// dispatcher) and to finish requests.  Launches, group uploads and event
// polls -- all the CUDA work -- run without it, so submissions and the
// front-end threads are not held up by them.
void dispatcher(Server *s) {
  lec_es_ctx *c = s->c;
  cudaSetDevice(c->device);
  std::deque<Request *> staged;    // taken from the queue, not launched yet (arrival order)
  std::vector<Finished> finished;  // finished here, to be finished under the mutex
  bool busy = false;               // launches or groups in flight
  bool progress = true;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (const Finished &f : finished) finish(s, f.r, f.st);
      if (!finished.empty()) progress = true;
      finished.clear();
      if (s->stop) break;
      if (!progress && s->queue.empty()) {
        // nothing changed last round: wait for a request (at once) or poll
        // the GPU again soon
        s->disp_waiting = true;
        if (!busy && staged.empty()) s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        else s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        s->disp_waiting = false;
        if (s->stop) break;
      }
      while (!s->queue.empty()) {
        Request *r = s->reqs[s->queue.front()].get();
        s->queue.pop_front();
        if (r->state == Request::CANCELLED) continue;
        r->state = Request::RUNNING;
        staged.push_back(r);
      }
    }
    progress = false;
    // completions
    for (size_t i = 0; i < s->running.size();) {
      Request *r = s->running[i];
      Slot &sl = s->slots[r->slot];
      if (r->cancel && !r->cancel_sent && cudaEventQuery(sl.e0) == cudaSuccess) {
        // the request's reset copy has run: zero its counterexample word so
        // every later pass of its kernel sees "nothing lower to find"
        cudaMemcpyAsync(sl.d_res, s->h_zero, 8, cudaMemcpyHostToDevice, s->ctl);
        cudaEventRecord(sl.zeroed, s->ctl);
        sl.zero_pending = true;
        r->cancel_sent = true;
      }
      const cudaError_t q = cudaEventQuery(sl.e2);
      if (q == cudaErrorNotReady) {
        i++;
        continue;
      }
      if (q == cudaSuccess) {
        finished.push_back({r, retire(s, r)});
      } else {
        r->err = LEC_ES_ECUDA;
        sl.busy = false;
        s->stream_load[r->stream]--;
        s->used -= r->reserve;
        finished.push_back({r, Request::FAILED});
      }
      progress = true;
      s->running[i] = s->running.back();
      s->running.pop_back();
    }
    bool groups_busy = false;
    for (int gi = 0; gi < kGroupSlots; gi++) {
      GroupSlot &G = s->groups[gi];
      if (!G.busy) continue;
      const cudaError_t q = cudaEventQuery(G.e2);
      if (q == cudaErrorNotReady) {
        groups_busy = true;
        continue;
      }
      progress = true;
      if (q == cudaSuccess) {
        retire_group(s, gi, finished);
      } else {
        for (Request *r : G.members) {
          r->err = LEC_ES_ECUDA;
          s->used -= r->reserve;
          finished.push_back({r, Request::FAILED});
        }
        G.members.clear();
        G.busy = false;
      }
    }
    // admission in arrival order: small interpreter requests in groups, the
    // others one launch each
    while (!staged.empty()) {
      Request *r = staged.front();
      if (r->cancel) {
        staged.pop_front();
        finished.push_back({r, Request::CANCELLED});
        progress = true;
        continue;
      }
      if (groupable(s, r)) {
        const int gi = free_group(s);
        if (gi < 0 || admit_group(s, gi, staged, finished) != LEC_ES_OK) break;
        groups_busy = true;
        progress = true;
        continue;
      }
      if (s->running.size() >= c->max_inflight) break;
      r->reserve = reserve_bytes(c, r->prog);
      if (s->used + r->reserve > c->slot_budget && !s->running.empty()) break;
      const int rc = launch(s, r);
      if ((rc == LEC_ES_ENOMEM || rc == LEC_ES_EBUSY) && !s->running.empty()) break;  // retry when some finish
      staged.pop_front();
      progress = true;
      if (rc) {
        r->err = rc;
        finished.push_back({r, Request::FAILED});
        continue;
      }
      s->used += r->reserve;
      s->running.push_back(r);
    }
    busy = !s->running.empty() || groups_busy;
    if (progress) std::this_thread::yield();
  }
}

int ensure_server(lec_es_ctx *c) {
  std::lock_guard<std::mutex> g(c->server_mu);
  if (c->server) return LEC_ES_OK;
  cudaSetDevice(c->device);
  std::unique_ptr<Server> s(new (std::nothrow) Server());
  if (!s) return LEC_ES_ENOMEM;
  s->c = c;
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  s->streams.resize(kStreams);
  s->stream_load.assign(kStreams, 0);
  for (int i = 0; i < kStreams; i++) {
    const int prio = i < kStreams / 2 ? greatest : least;
    if (cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, prio) != cudaSuccess)
      return LEC_ES_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking) != cudaSuccess) return LEC_ES_ECUDA;
  if (cudaMallocHost((void **)&s->h_zero, 8) != cudaSuccess) return LEC_ES_ENOMEM;
  *s->h_zero = 0;
  s->slots.resize(c->max_inflight);
  for (Slot &sl : s->slots) {
    sl.d_res = (unsigned long long *)c->arena.alloc(kResWords * 8);
    if (!sl.d_res) return LEC_ES_ENOMEM;
    if (cudaMallocHost((void **)&sl.h_res, kResWords * 8) != cudaSuccess) return LEC_ES_ENOMEM;
    if (cudaEventCreate(&sl.e0) != cudaSuccess || cudaEventCreate(&sl.e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.e2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.zeroed, cudaEventDisableTiming) != cudaSuccess)
      return LEC_ES_ECUDA;
  }
  // grouped requests: one stream, kGroupSlots sets of tables and staging
  if (cudaStreamCreateWithFlags(&s->group_stream, cudaStreamNonBlocking) != cudaSuccess) return LEC_ES_ECUDA;
  {
    const size_t fit = ((size_t)c->smem_optin - batch_w_smem_bytes(0, kGroupBlock, kGroupRing)) /
                       ((size_t)kGroupBlock * kLaneBytes);
    s->group_smem_max = batch_w_smem_bytes((uint32_t)fit, kGroupBlock, kGroupRing);
    if (configure_batch_w(kGroupBlock, (size_t)c->smem_optin) != 0) return LEC_ES_ECUDA;
  }
  for (GroupSlot &G : s->groups) {
    G.d_buf = (uint8_t *)c->arena.alloc(kGroupBufBytes);
    if (!G.d_buf) return LEC_ES_ENOMEM;
    if (cudaMallocHost((void **)&G.h_buf, kGroupBufBytes) != cudaSuccess ||
        cudaMallocHost((void **)&G.h_stage, kGroupStage) != cudaSuccess)
      return LEC_ES_ENOMEM;
    if (cudaEventCreate(&G.e0) != cudaSuccess || cudaEventCreate(&G.e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&G.e2, cudaEventDisableTiming) != cudaSuccess)
      return LEC_ES_ECUDA;
  }
  Server *raw = s.get();
  raw->th = std::thread(dispatcher, raw);
  const unsigned nprep = std::max(2u, std::min(8u, std::thread::hardware_concurrency() / 2));
  for (unsigned i = 0; i < nprep; i++) raw->prep_threads.emplace_back(prep_worker, raw);
  c->server = s.release();
  return LEC_ES_OK;
}

// The ctx's server, read under server_mu (ensure_server and server_shutdown
// write it under the same lock).  lec_es_destroy must not run concurrently
// with other calls on the same ctx.
Server *server_of(lec_es_ctx *c) {
  std::lock_guard<std::mutex> g(c->server_mu);
  return c->server;
}

}  // namespace

void server_shutdown(lec_es_ctx *c) {
  Server *s = nullptr;
  {
    std::lock_guard<std::mutex> g(c->server_mu);
    s = c->server;
    c->server = nullptr;
  }
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_prep.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto &t : s->prep_threads) t.join();
  cudaSetDevice(c->device);
  // the dispatcher has stopped: end the requests still on the GPU early
  for (Request *r : s->running)
    cudaMemcpyAsync(s->slots[r->slot].d_res, s->h_zero, 8, cudaMemcpyHostToDevice, s->ctl);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaStreamSynchronize(s->ctl);
  cudaStreamDestroy(s->ctl);
  for (Slot &sl : s->slots) {
    c->arena.free(sl.d_res);
    if (sl.h_res) cudaFreeHost(sl.h_res);
    if (sl.e0) cudaEventDestroy(sl.e0);
    if (sl.e1) cudaEventDestroy(sl.e1);
    if (sl.e2) cudaEventDestroy(sl.e2);
    if (sl.zeroed) cudaEventDestroy(sl.zeroed);
  }
  if (s->group_stream) {
    cudaStreamSynchronize(s->group_stream);
    cudaStreamDestroy(s->group_stream);
  }
  for (GroupSlot &G : s->groups) {
    c->arena.free(G.d_buf);
    if (G.h_buf) cudaFreeHost(G.h_buf);
    if (G.h_stage) cudaFreeHost(G.h_stage);
    if (G.e0) cudaEventDestroy(G.e0);
    if (G.e1) cudaEventDestroy(G.e1);
    if (G.e2) cudaEventDestroy(G.e2);
  }
  for (auto &kv : s->resident) {
    if (kv.second.shared_block) continue;
    c->arena.free(kv.second.d_recs);
    c->arena.free(kv.second.d_loads);
  }
  for (void *b : s->shared_blocks) c->arena.free(b);
  for (cudaEvent_t e : s->group_events) cudaEventDestroy(e);
  if (s->h_zero) cudaFreeHost(s->h_zero);
  s->cv_done.notify_all();
  delete s;
}

}  // namespace lec

using namespace lec;

extern "C" int lec_es_server_config(lec_es_ctx *c, size_t slot_budget_bytes, uint32_t max_inflight) {
  if (!c || max_inflight == 0 || max_inflight > 4096) return LEC_ES_EINVAL;
  std::lock_guard<std::mutex> g(c->server_mu);
  if (c->server) return LEC_ES_EBUSY;
  c->slot_budget = slot_budget_bytes;
  c->max_inflight = max_inflight;
  return LEC_ES_OK;
}

extern "C" int lec_es_submit(lec_es_ctx *c, const lec_es_miter *m, uint64_t *ticket) {
  if (!c || !m || !ticket) return LEC_ES_EINVAL;
  const double t0 = now_ms();
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return LEC_ES_ENOMEM;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc;
  try {
    rc = compact_cone(v, c->max_pis, r->cone);  // the caller may free m once this returns
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  if (rc) return rc;
  rc = ensure_server(c);
  if (rc) return rc;
  Server *s = server_of(c);
  r->t_submit = t0;
  r->res.host_ms = now_ms() - t0;
  r->state = Request::PREPARING;
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->prep.push_back(r->ticket);
  s->reqs[r->ticket] = std::move(r);
  if (s->prep_waiting > 0) s->cv_prep.notify_one();
  return LEC_ES_OK;
}

extern "C" int lec_es_submit_many(lec_es_ctx *c, const lec_es_miter *m, size_t k, uint64_t *tickets) {
  if (!c || (!m && k) || (!tickets && k)) return LEC_ES_EINVAL;
  if (k == 0) return LEC_ES_OK;
  const double t0 = now_ms();
  // every cone is copied (and checked) before any request is queued, so an
  // error leaves nothing submitted
  std::vector<std::unique_ptr<Request>> rs(k);
  try {
    for (size_t i = 0; i < k; i++) {
      rs[i].reset(new Request());
      MiterView v{m[i].num_pis, m[i].num_ands, m[i].fanins, m[i].out_lit};
      const int rc = compact_cone(v, c->max_pis, rs[i]->cone);
      if (rc) return rc;
    }
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  int rc = ensure_server(c);
  if (rc) return rc;
  Server *s = server_of(c);
  const double per = (now_ms() - t0) / (double)k;
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t i = 0; i < k; i++) {
    Request *r = rs[i].get();
    r->t_submit = t0;
    r->res.host_ms = per;
    r->state = Request::PREPARING;
    r->ticket = s->next_ticket++;
    tickets[i] = r->ticket;
    s->prep.push_back(r->ticket);
    s->reqs[r->ticket] = std::move(rs[i]);
  }
  if (s->prep_waiting > 0) s->cv_prep.notify_all();
  return LEC_ES_OK;
}

namespace {
// Called with s->mu held: result of a finished request (and release).
int collect(Server *s, uint64_t ticket, lec_es_result *out) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LEC_ES_ENOTFOUND;
  Request *r = it->second.get();
  if (r->state == Request::PREPARING || r->state == Request::QUEUED || r->state == Request::RUNNING)
    return LEC_ES_EBUSY;
  int rc = LEC_ES_OK;
  if (r->state == Request::CANCELLED) rc = LEC_ES_ECANCELLED;
  else if (r->state == Request::FAILED) rc = r->err ? r->err : LEC_ES_ECUDA;
  else if (out) *out = r->res;
  s->reqs.erase(it);
  return rc;
}
}  // namespace

extern "C" int lec_es_poll(lec_es_ctx *c, uint64_t ticket, lec_es_result *out) {
  if (!c || !out) return LEC_ES_EINVAL;
  Server *s = server_of(c);
  if (!s) return LEC_ES_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  return collect(s, ticket, out);
}

extern "C" int lec_es_wait(lec_es_ctx *c, uint64_t ticket, double timeout_s, lec_es_result *out) {
  if (!c || !out) return LEC_ES_EINVAL;
  Server *s = server_of(c);
  if (!s) return LEC_ES_ENOTFOUND;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    int rc = collect(s, ticket, out);
    if (rc != LEC_ES_EBUSY) return rc;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      rc = collect(s, ticket, out);
      return rc == LEC_ES_EBUSY ? LEC_ES_ETIMEOUT : rc;
    }
  }
}

extern "C" int lec_es_cancel(lec_es_ctx *c, uint64_t ticket) {
  if (!c) return LEC_ES_EINVAL;
  Server *s = server_of(c);
  if (!s) return LEC_ES_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LEC_ES_ENOTFOUND;
  Request *r = it->second.get();
  if (r->state == Request::QUEUED) {
    finish(s, r, Request::CANCELLED);
  } else if (r->state == Request::RUNNING || r->state == Request::PREPARING) {
    r->cancel = true;  // a preparing request is finished by its front-end thread
  }
  return LEC_ES_OK;
}
