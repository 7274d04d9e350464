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
  uint32_t nload = 0, out_off = 0;
  PlanGeom geom;
};

struct Request {
  enum State { PREPARING, QUEUED, RUNNING, DONE, CANCELLED, FAILED };
  uint64_t ticket = 0;
  CompactMiter cone;  // until the front end has run
  Program prog;
  State state = QUEUED;
  int slot = -1;
  int stream = -1;
  size_t reserve = 0;
  double t_submit = 0, t_done = 0;
  bool cancel = false, cancel_sent = false;
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
  std::vector<std::thread> prep_threads;
  std::deque<uint64_t> queue;  // compiled, waiting for admission
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<uint64_t> running;
  std::vector<Slot> slots;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_load;
  cudaStream_t ctl = nullptr;
  unsigned long long *h_zero = nullptr;
  std::map<std::pair<uint64_t, uint64_t>, Resident> resident;  // by both structure hashes
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
  const double predicted = cost_run_ms(c, k ? LEC_ES_TIER_JIT : LEC_ES_TIER_INTERP, g.cone_ands, g.n, k ? k->lop3_per_pass : 0.0);
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
    err = cudaLaunchKernel((const void *)k->kern, dim3((unsigned)grid), dim3(k->block), args, 0, st) ==
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
    const uint64_t passes = (xp.word_end + res->geom.block - 1) / res->geom.block;
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

void retire(Server *s, Request *r) {
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
  if (r->cancel) {
    finish(s, r, Request::CANCELLED);
  } else if (status) {
    r->err = (status & DEV_WAIT_TIMEOUT) ? LEC_ES_EDEVICE_WAIT : LEC_ES_ECUDA;
    finish(s, r, Request::FAILED);
  } else {
    finish(s, r, Request::DONE);
  }
}

// Front-end thread: compiles submitted cones and queues them for admission.
void prep_worker(Server *s) {
  lec_es_ctx *c = s->c;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_prep.wait(lk, [&] { return s->stop || !s->prep.empty(); });
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
      const KernelProbe probe{jit_probe, &jp};
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
      s->cv_work.notify_one();
    }
  }
}

void dispatcher(Server *s) {
  lec_es_ctx *c = s->c;
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // completions
    for (size_t i = 0; i < s->running.size();) {
      Request *r = s->reqs[s->running[i]].get();
      Slot &sl = s->slots[r->slot];
      if (r->cancel && !r->cancel_sent && cudaEventQuery(sl.e0) == cudaSuccess) {
        // the request's reset copy has run: zero its counterexample word so
        // every later pass of its kernel sees "nothing lower to find"
        cudaMemcpyAsync(sl.d_res, s->h_zero, 8, cudaMemcpyHostToDevice, s->ctl);
        cudaEventRecord(sl.zeroed, s->ctl);
        sl.zero_pending = true;
        r->cancel_sent = true;
      }
      cudaError_t q = cudaEventQuery(sl.e2);
      if (q == cudaSuccess) {
        retire(s, r);
        s->running[i] = s->running.back();
        s->running.pop_back();
      } else {
        if (q != cudaErrorNotReady) {
          r->err = LEC_ES_ECUDA;
          sl.busy = false;
          s->stream_load[r->stream]--;
          s->used -= r->reserve;
          finish(s, r, Request::FAILED);
          s->running[i] = s->running.back();
          s->running.pop_back();
          continue;
        }
        i++;
      }
    }
    // admission in arrival order
    while (!s->queue.empty() && s->running.size() < c->max_inflight) {
      Request *r = s->reqs[s->queue.front()].get();
      if (r->state == Request::CANCELLED) {
        s->queue.pop_front();
        continue;
      }
      r->reserve = reserve_bytes(c, r->prog);
      if (s->used + r->reserve > c->slot_budget && !s->running.empty()) break;
      int rc = launch(s, r);
      if (rc == LEC_ES_ENOMEM || rc == LEC_ES_EBUSY) {
        if (s->running.empty()) {
          r->err = rc;
          s->queue.pop_front();
          finish(s, r, Request::FAILED);
          continue;
        }
        break;
      }
      s->queue.pop_front();
      if (rc) {
        r->err = rc;
        finish(s, r, Request::FAILED);
        continue;
      }
      s->used += r->reserve;
      r->state = Request::RUNNING;
      s->running.push_back(r->ticket);
    }
    if (s->running.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    } else {  // requests in flight: poll again soon (this thread only schedules)
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
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
    for (uint64_t t : s->running) {
      Request *r = s->reqs[t].get();
      cudaMemcpyAsync(s->slots[r->slot].d_res, s->h_zero, 8, cudaMemcpyHostToDevice, s->ctl);
    }
  }
  s->cv_work.notify_all();
  s->cv_prep.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto &t : s->prep_threads) t.join();
  cudaSetDevice(c->device);
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
  for (auto &kv : s->resident) {
    c->arena.free(kv.second.d_recs);
    c->arena.free(kv.second.d_loads);
  }
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
  s->cv_prep.notify_one();
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
