// api.cpp -- C ABI of the ES engine (see include/lec_es.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

using namespace lec;

namespace lec {

// ---- device arena: first-fit over one device allocation -----------------------

int Arena::init(void *base_, size_t bytes_) {
  base = (uint8_t *)base_;
  bytes = bytes_;
  free_list.clear();
  // keep every block 256-byte aligned
  uintptr_t b = (uintptr_t)base;
  size_t skew = (256 - (b & 255)) & 255;
  if (bytes <= skew) return LEC_ES_ENOMEM;
  free_list[skew] = bytes - skew;
  return LEC_ES_OK;
}

void *Arena::alloc(size_t n) {
  std::lock_guard<std::mutex> g(mu);
  n = (n + 255) & ~(size_t)255;
  if (n == 0) n = 256;
  for (auto it = free_list.begin(); it != free_list.end(); ++it) {
    if (it->second >= n) {
      size_t off = it->first, sz = it->second;
      free_list.erase(it);
      if (sz > n) free_list[off + n] = sz - n;
      used[off] = n;
      in_use += n;
      return base + off;
    }
  }
  return nullptr;
}

void Arena::free(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu);
  size_t off = (uint8_t *)p - base;
  auto u = used.find(off);
  if (u == used.end()) return;
  size_t n = u->second;
  used.erase(u);
  in_use -= n;
  auto nx = free_list.lower_bound(off);
  if (nx != free_list.end() && off + n == nx->first) {
    n += nx->second;
    nx = free_list.erase(nx);
  }
  if (nx != free_list.begin()) {
    auto pv = std::prev(nx);
    if (pv->first + pv->second == off) {
      pv->second += n;
      return;
    }
  }
  free_list[off] = n;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LEC_ES_OK : LEC_ES_ECUDA; }

// Per-run pinned words and events come from a pool: pinned allocation and
// its release are slow (and the release can wait for the device), so a
// check-per-call user would otherwise pay them every time.
int run_res_acquire(lec_es_ctx *c, RunRes *out) {
  std::lock_guard<std::mutex> g(c->res_mu);
  if (c->res_free.empty()) {
    const int kSlab = 64;
    void *slab = nullptr;
    if (cudaMallocHost(&slab, (size_t)kSlab * kResWords * sizeof(unsigned long long)) != cudaSuccess)
      return LEC_ES_ENOMEM;
    c->res_slabs.push_back(slab);
    for (int i = 0; i < kSlab; i++) {
      RunRes r;
      r.h_res = (unsigned long long *)slab + (size_t)i * kResWords;
      if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.e2, cudaEventDisableTiming) != cudaSuccess)
        return LEC_ES_ECUDA;
      c->res_events.push_back(r.e0);
      c->res_events.push_back(r.e1);
      c->res_events.push_back(r.e2);
      c->res_free.push_back(r);
    }
  }
  *out = c->res_free.back();
  c->res_free.pop_back();
  return LEC_ES_OK;
}

void run_res_release(lec_es_ctx *c, const RunRes &r) {
  if (!r.h_res) return;
  std::lock_guard<std::mutex> g(c->res_mu);
  c->res_free.push_back(r);
}

void run_res_destroy_all(lec_es_ctx *c) {
  std::lock_guard<std::mutex> g(c->res_mu);
  for (cudaEvent_t e : c->res_events) cudaEventDestroy(e);
  for (void *s : c->res_slabs) cudaFreeHost(s);
  c->res_events.clear();
  c->res_slabs.clear();
  c->res_free.clear();
}

// Wait for an event with a host-side deadline (no unbounded synchronize).
// Polls the event: for the first 20 ms it yields between polls (a check's
// caller is blocked anyway, and a 50 us sleep would add up to its length
// plus the scheduler's slack to every run), then sleeps 50 us per poll.
int wait_event(cudaEvent_t ev, double timeout_s) {
  const double t0 = now_ms();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return LEC_ES_OK;
    if (e != cudaErrorNotReady) return LEC_ES_ECUDA;
    const double waited = now_ms() - t0;
    if (waited > timeout_s * 1e3) return LEC_ES_ETIMEOUT;
    if (waited < 20.0) std::this_thread::yield();
    else std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// ---- tier / launch geometry ---------------------------------------------------

int choose_interp_geometry(lec_es_ctx *c, const Program &prog, uint64_t chunks, const lec_es_options *opt,
                           PlanGeom &g) {
  const uint32_t nrec_p = (uint32_t)((prog.recs.size() + 1) & ~(size_t)1);
  g.nrec_padded = std::max<uint32_t>(2, nrec_p);
  const int pref = opt && opt->block_threads ? (int)opt->block_threads : 256;
  const bool force_spill = opt && opt->tier == LEC_ES_TIER_SPILL;
  g.spill = false;
  if (!force_spill) {
    for (int b = pref; b >= 32; b /= 2) {
      if (b != 32 && b != 64 && b != 128 && b != 256) continue;
      uint32_t ring, res;
      size_t bytes;
      if (interp_smem_bytes(prog.num_slots, g.nrec_padded, b, &ring, &res, &bytes) == 0 &&
          bytes <= (size_t)c->smem_optin) {
        g.block = b;
        g.ring_recs = ring;
        g.resident = res;
        g.smem = bytes;
        break;
      }
      g.block = 0;
    }
  }
  if (force_spill || g.block == 0) {
    g.spill = true;
    g.block = 128;
    uint32_t ring, res;
    size_t bytes;
    interp_smem_bytes(0, g.nrec_padded, g.block, &ring, &res, &bytes);
    g.ring_recs = ring;
    g.resident = res;
    g.smem = bytes;
  }
  // blocks resident per SM by shared memory, capped by the available passes
  const size_t per_sm = 228u * 1024u;
  int bps = (int)std::max<size_t>(1, per_sm / (g.smem + 1024));
  bps = std::min(bps, 2048 / g.block);
  uint64_t passes = (chunks + g.block - 1) / g.block;
  uint64_t grid = (uint64_t)c->sm_count * bps;
  if (opt && opt->grid_blocks) grid = opt->grid_blocks;
  if (g.spill) grid = std::min<uint64_t>(grid, (uint64_t)c->sm_count * 4);
  g.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(grid, passes));
  return LEC_ES_OK;
}

bool choose_word_geometry(lec_es_ctx *c, const Program &prog, const lec_es_options *opt, PlanGeom &g, bool widest) {
  const uint32_t nand = (uint32_t)std::count_if(prog.recs.begin(), prog.recs.end(), [](const Rec &r) { return r.op < 4; });
  const int pref = opt && opt->block_threads ? (int)opt->block_threads : 256;
  g = PlanGeom{};
  for (int b = 256; b >= 32; b /= 2) {
    if (b > pref) continue;
    uint32_t ring, res;
    const size_t bytes = interp_w_smem_bytes(prog.num_slots, nand, b, &ring, &res);
    if (bytes <= (size_t)c->smem_optin) {
      g.block = b;
      g.ring_recs = ring;
      g.resident = res;
      g.smem = bytes;
      g.word = true;
      g.nrec_padded = nand;
      break;
    }
  }
  if (!g.word) return false;
  if (widest && !(opt && opt->block_threads)) {
    const int base = word_warps_per_sm(g.smem, g.block);
    int best = base;
    for (int b = 128; b <= kMaxWordBlock; b += 128)  // whole warps on each of the SM's four schedulers
      for (int allow_res = 1; allow_res >= 0; allow_res--) {
        uint32_t ring, res;
        const size_t bytes = interp_w_smem_bytes(prog.num_slots, nand, b, &ring, &res, allow_res != 0);
        if (bytes > (size_t)c->smem_optin) continue;
        const int w = word_warps_per_sm(bytes, b);
        if (w < best || 4 * w < 5 * base || (w == best && b <= g.block)) continue;
        g.block = b;
        g.ring_recs = ring;
        g.resident = res;
        g.smem = bytes;
        best = w;
      }
  }
  const uint64_t lanes = kLaneBytes == 8 ? num_words(prog.n) : num_chunks(prog.n);
  const size_t per_sm = 228u * 1024u;
  int bps = (int)std::max<size_t>(1, per_sm / (g.smem + 1024));
  bps = std::min(bps, 2048 / g.block);
  const uint64_t passes = (lanes + g.block - 1) / g.block;
  uint64_t grid = (uint64_t)c->sm_count * bps;
  if (opt && opt->grid_blocks) grid = opt->grid_blocks;
  g.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(grid, passes));
  return true;
}

}  // namespace lec

// ---- context -------------------------------------------------------------------

extern "C" const char *lec_es_strerror(int s) {
  switch (s) {
    case LEC_ES_OK: return "ok";
    case LEC_ES_EINVAL: return "invalid argument or malformed AIG";
    case LEC_ES_ETOOBIG: return "support or live set too large";
    case LEC_ES_ENOMEM: return "out of memory";
    case LEC_ES_ECUDA: return "CUDA error";
    case LEC_ES_ETIMEOUT: return "timeout";
    case LEC_ES_EBUSY: return "busy";
    case LEC_ES_ECANCELLED: return "cancelled";
    case LEC_ES_EDEVICE_WAIT: return "device-side wait exceeded its bound";
    case LEC_ES_EJIT: return "run-time compilation failed";
    case LEC_ES_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

extern "C" int lec_es_create(lec_es_ctx **out, const lec_es_config *cfg) {
  if (!out || !cfg) return LEC_ES_EINVAL;
  *out = nullptr;
  if (cfg->max_pis > 63) return LEC_ES_EINVAL;
  std::unique_ptr<lec_es_ctx> c(new (std::nothrow) lec_es_ctx());
  if (!c) return LEC_ES_ENOMEM;
  c->device = cfg->device;
  c->max_pis = cfg->max_pis ? cfg->max_pis : 63;
  c->timeout_s = cfg->timeout_s > 0 ? cfg->timeout_s : 600.0;
  if (cfg->jit_cache_dir) c->jit_dir = cfg->jit_cache_dir;
  if (cudaSetDevice(c->device) != cudaSuccess) return LEC_ES_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return LEC_ES_ECUDA;
  c->sm_count = prop.multiProcessorCount;
  c->smem_optin = max_smem_optin(c->device);
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return LEC_ES_ECUDA;
    c->own_stream = true;
  }
  size_t bytes = cfg->arena_bytes ? cfg->arena_bytes : ((size_t)256 << 20);
  void *base = cfg->arena;
  if (!base) {
    if (cudaMalloc(&base, bytes) != cudaSuccess) return LEC_ES_ENOMEM;
    c->own_arena = true;
  }
  c->arena_base = base;
  if (c->arena.init(base, bytes) != LEC_ES_OK) return LEC_ES_ENOMEM;
  if (cudaMallocHost((void **)&c->h_init, kResWords * sizeof(unsigned long long)) != cudaSuccess)
    return LEC_ES_ENOMEM;
  for (int i = 0; i < kResWords; i++) c->h_init[i] = 0;
  c->h_init[0] = ~0ull;
  c->h_init[4] = ~0ull;
  *out = c.release();
  return LEC_ES_OK;
}

extern "C" void lec_es_destroy(lec_es_ctx *c) {
  if (!c) return;
  lec::server_shutdown(c);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  lec::jit_release_all(c);
  lec::run_res_destroy_all(c);
  if (c->h_init) cudaFreeHost(c->h_init);
  if (c->own_arena && c->arena_base) cudaFree(c->arena_base);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

// ---- front end (host only) ---------------------------------------------------------

extern "C" int lec_es_compile(const lec_es_miter *m, uint32_t order, lec_es_program_info *info, uint64_t *records,
                              uint64_t cap) {
  if (!m || !info) return LEC_ES_EINVAL;
  Program p;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc;
  try {
    rc = compile_program(v, order, 63, p);
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  if (rc) return rc;
  memset(info, 0, sizeof(*info));
  info->n = p.n;
  for (uint32_t k = 0; k < p.n; k++) info->support[k] = p.support[k];
  info->cone_ands = p.cone_ands;
  info->num_slots = p.num_slots;
  info->out_slot = p.out_slot;
  info->out_compl = p.out_compl;
  info->order = p.order;
  info->num_records = p.recs.size();
  info->hash = p.hash;
  info->num_luts = p.lut.count;
  info->lut_live = p.lut.live;
  info->interp_step = p.step;
  if (records && cap) memcpy(records, p.recs.data(), sizeof(Rec) * std::min<uint64_t>(cap, p.recs.size()));
  return LEC_ES_OK;
}

// ---- single-miter plans --------------------------------------------------------------

namespace lec {

void fill_result(const lec_es_plan *p, lec_es_result *out) {
  memset(out, 0, sizeof(*out));
  const Program &g = p->prog;
  out->support_n = g.n;
  for (uint32_t k = 0; k < g.n; k++) out->support[k] = g.support[k];
  out->cone_ands = g.cone_ands;
  out->num_slots = g.num_slots;
  out->tier = p->tier;
  out->order = g.order;
  out->host_ms = p->host_ms;
  out->jit_ms = p->jit_ms;
}

void plan_release(lec_es_ctx *c, lec_es_plan *p) {
  if (!p) return;
  run_res_release(c, p->res);
  c->arena.free(p->d_recs);
  c->arena.free(p->d_loads);
  c->arena.free(p->d_res);
  c->arena.free(p->d_spill);
  delete p;
}

// Set by lec_es_check_ex around its AUTO prepare: a cold kernel is then
// not built synchronously (see check_race).
thread_local bool t_check_race = false;

int plan_prepare(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt, lec_es_plan **out) {
  if (!c || !m || !out) return LEC_ES_EINVAL;
  *out = nullptr;
  const double t0 = now_ms();
  Program prog;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc;
  try {
    const uint32_t want = opt ? opt->tier : LEC_ES_TIER_AUTO;
    JitProbe jp{c, want == LEC_ES_TIER_JIT ? JitProbe::kRun : JitProbe::kAuto};
    // a one-off AUTO check never builds a kernel it does not hold on its own
    // path (check_race): the table cover is left to the background build
    jp.defer = t_check_race;
    const KernelProbe probe{jit_probe, &jp, jit_want_cover};
    // the probe finds table-form kernels only
    const bool may_skip = (want == LEC_ES_TIER_JIT || want == LEC_ES_TIER_AUTO) &&
                          !(opt && (opt->flags & LEC_ES_FLAG_JIT_AND_FORM));
    rc = compile_program(v, opt ? opt->order : LEC_ES_ORDER_AUTO, c->max_pis, prog, may_skip ? &probe : nullptr);
    if (!rc && jp.deferred && !prog.lut.elided && prog.lut.count == 0) prog.lut.deferred = true;
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  if (rc) return rc;
  const double front_ms = now_ms() - t0;
  if (getenv("LEC_ES_FRONT_LOG"))
    fprintf(stderr, "lec_es front end %016llx: %.3f ms, table cover %s\n", (unsigned long long)prog.hash, front_ms,
            prog.lut.elided ? "reused from the kernel" : prog.lut.deferred ? "left to the background build" : "built");
  rc = plan_prepare_program(c, std::move(prog), opt, out);
  if (!rc) (*out)->host_ms += front_ms;
  return rc;
}

// Device side of a plan for an already compiled program.
int plan_prepare_program(lec_es_ctx *c, Program &&prog, const lec_es_options *opt, lec_es_plan **out) {
  *out = nullptr;
  const double t0 = now_ms();
  std::unique_ptr<lec_es_plan> p(new (std::nothrow) lec_es_plan());
  if (!p) return LEC_ES_ENOMEM;
  p->prog = std::move(prog);
  p->stream = c->stream;
  p->flags = opt ? opt->flags : 0;
  p->user_grid = opt && opt->grid_blocks;
  p->jit_lut = !(p->flags & LEC_ES_FLAG_JIT_AND_FORM);
  int rc;
  if (cudaSetDevice(c->device) != cudaSuccess) return LEC_ES_ECUDA;
  const Program &g = p->prog;
  const uint64_t chunks = num_chunks(g.n);
  uint32_t want = opt ? opt->tier : LEC_ES_TIER_AUTO;
  if (g.slots_elided) want = LEC_ES_TIER_JIT;  // the front end found this cone's kernel for this run
  if (want == LEC_ES_TIER_AUTO) {
    want = jit_auto_tier(c, g, chunks);
    // a one-off check does not wait for a kernel build: it races the
    // interpreter against a background build instead (check_race)
    if (want == LEC_ES_TIER_JIT && t_check_race && !jit_held(c, g)) want = LEC_ES_TIER_INTERP;
  }
  const double tj = now_ms();
  if (want == LEC_ES_TIER_JIT) {
    rc = jit_prepare(c, p.get(), opt);
    if (rc) {
      plan_release(c, p.release());
      return rc;
    }
    p->tier = LEC_ES_TIER_JIT;
  } else {
    const bool want_spill = want == LEC_ES_TIER_SPILL;
    if (!want_spill && choose_word_geometry(c, g, opt, p->geom, true)) {
      p->tier = LEC_ES_TIER_INTERP;
    } else {
      rc = choose_interp_geometry(c, g, chunks, opt, p->geom);
      if (rc) return rc;
      p->tier = p->geom.spill ? LEC_ES_TIER_SPILL : LEC_ES_TIER_INTERP;
    }
  }
  const double td = now_ms();
  rc = plan_finish_device(c, p.get());
  if (rc) {
    plan_release(c, p.release());
    return rc;
  }
  p->host_ms = now_ms() - t0 - p->jit_ms;
  if (getenv("LEC_ES_FRONT_LOG"))
    fprintf(stderr, "lec_es plan: set-up %.3f ms, tier choice and kernel %.3f ms, device buffers %.3f ms\n", tj - t0,
            td - tj, now_ms() - td);
  *out = p.release();
  return LEC_ES_OK;
}

// Records upload (interpreter tiers), spill scratch, result words, events.
int plan_finish_device(lec_es_ctx *c, lec_es_plan *p) {
  const Program &g = p->prog;
  if (p->geom.word) {
    std::vector<XRec> xr;
    std::vector<XLoad> xl;
    encode_w(g, p->geom.block, xr, xl, p->out_off);
    p->nload = (uint32_t)xl.size();
    p->d_recs = c->arena.alloc(std::max<size_t>(16, xr.size() * sizeof(XRec)));
    p->d_loads = c->arena.alloc(std::max<size_t>(16, xl.size() * sizeof(XLoad)));
    if (!p->d_recs || !p->d_loads) return LEC_ES_ENOMEM;
    if ((!xr.empty() &&
         cudaMemcpyAsync(p->d_recs, xr.data(), xr.size() * sizeof(XRec), cudaMemcpyHostToDevice, p->stream) !=
             cudaSuccess) ||
        (!xl.empty() &&
         cudaMemcpyAsync(p->d_loads, xl.data(), xl.size() * sizeof(XLoad), cudaMemcpyHostToDevice, p->stream) !=
             cudaSuccess))
      return LEC_ES_ECUDA;
  } else if (p->tier != LEC_ES_TIER_JIT) {
    const size_t rb = (size_t)p->geom.nrec_padded * sizeof(Rec);
    p->d_recs = c->arena.alloc(rb);
    if (!p->d_recs) return LEC_ES_ENOMEM;
    std::vector<Rec> padded(p->geom.nrec_padded);
    memcpy(padded.data(), g.recs.data(), g.recs.size() * sizeof(Rec));
    if (cudaMemcpyAsync(p->d_recs, padded.data(), rb, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
      return LEC_ES_ECUDA;
    if (p->geom.spill) {
      p->spill_bytes = (size_t)g.num_slots * p->geom.grid * p->geom.block * 4u;
      p->d_spill = c->arena.alloc(p->spill_bytes);
      if (!p->d_spill) return LEC_ES_ENOMEM;
    }
  }
  p->d_res = (unsigned long long *)c->arena.alloc(kResWords * sizeof(unsigned long long));
  if (!p->d_res) return LEC_ES_ENOMEM;
  int rc = run_res_acquire(c, &p->res);
  if (rc) return rc;
  p->h_res = p->res.h_res;
  p->e0 = p->res.e0;
  p->e1 = p->res.e1;
  p->e2 = p->res.e2;
  // the record upload reads a host vector that dies with this call
  if (p->tier != LEC_ES_TIER_JIT && cudaStreamSynchronize(p->stream) != cudaSuccess) return LEC_ES_ECUDA;
  return LEC_ES_OK;
}

int plan_run_async(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt) {
  return plan_run_async_grid(c, p, opt, 0);
}

int plan_run_async_grid(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt, int grid_override) {
  if (!c || !p) return LEC_ES_EINVAL;
  const Program &g = p->prog;
  const uint64_t W = num_words(g.n);
  uint64_t wb = opt ? opt->word_begin : 0, we = opt ? opt->word_end : UINT64_MAX;
  if (!opt) we = UINT64_MAX;
  if (we > W) we = W;
  if (wb >= we) return LEC_ES_EINVAL;
  p->last_wb = wb;
  p->last_we = we;
  p->last_default_grid = grid_override <= 0 && !(opt && opt->grid_blocks) && !p->user_grid &&
                         !(p->flags & LEC_ES_FLAG_TEST_WAIT_TIMEOUT);
  const uint64_t C = num_chunks(g.n);
  const uint64_t cb = std::min<uint64_t>(2 * wb, C), ce = std::min<uint64_t>(2 * we, C);
  cudaStream_t st = p->stream;
  if (cudaMemcpyAsync(p->d_res, c->h_init, kResWords * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return LEC_ES_ECUDA;
  cudaEventRecord(p->e0, st);
  int err;
  if (p->tier == LEC_ES_TIER_JIT) {
    err = jit_launch(c, p, cb, ce, grid_override, ~0ull);
  } else if (p->geom.word) {
    XParams xp{};
    xp.recs = (const XRec *)p->d_recs;
    xp.loads = (const XLoad *)p->d_loads;
    xp.nrec = p->geom.nrec_padded;
    xp.nload = p->nload;
    xp.step = g.step;
    xp.out_off = p->out_off;
    xp.out_compl = g.out_compl;
    xp.n = g.n;
    xp.ring_recs = p->geom.ring_recs;
    xp.resident = p->geom.resident;
    xp.extra_tx = (p->flags & LEC_ES_FLAG_TEST_WAIT_TIMEOUT) ? 16u : 0u;
    xp.word_begin = wb;
    xp.word_end = we;
    xp.cex = p->d_res;
    xp.evaluated = p->d_res + 1;
    xp.status = (uint32_t *)(p->d_res + 2);
    const int grid = grid_override > 0 ? grid_override : p->geom.grid;
    err = launch_interp_w(xp, p->geom.block, grid, p->geom.smem, st);
  } else {
    InterpParams ip{};
    ip.recs = (const Rec *)p->d_recs;
    ip.nrec = (uint32_t)g.recs.size();
    ip.nrec_padded = p->geom.nrec_padded;
    ip.nslots = g.num_slots;
    ip.out_slot = g.out_slot;
    ip.out_compl = g.out_compl;
    ip.n = g.n;
    ip.ring_recs = p->geom.ring_recs;
    ip.resident = p->geom.resident;
    ip.chunk_begin = cb;
    ip.chunk_end = ce;
    ip.cex = p->d_res;
    ip.evaluated = p->d_res + 1;
    ip.status = (uint32_t *)(p->d_res + 2);
    ip.spill = (uint32_t *)p->d_spill;
    ip.extra_tx = (p->flags & LEC_ES_FLAG_TEST_WAIT_TIMEOUT) ? 16u : 0u;
    int grid = p->geom.grid;
    if (grid_override > 0 && !p->geom.spill) grid = grid_override;
    err = launch_interp(ip, p->geom.block, grid, p->geom.smem, p->geom.spill, st);
  }
  if (err) return LEC_ES_ECUDA;
  cudaEventRecord(p->e1, st);
  if (cudaMemcpyAsync(p->h_res, p->d_res, kResWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return LEC_ES_ECUDA;
  if (cudaEventRecord(p->e2, st) != cudaSuccess) return LEC_ES_ECUDA;
  p->pending = true;
  return LEC_ES_OK;
}

int plan_result(lec_es_ctx *c, lec_es_plan *p, lec_es_result *out) {
  if (!c || !p || !out) return LEC_ES_EINVAL;
  if (!p->pending) return LEC_ES_EINVAL;
  int rc = wait_event(p->e2, c->timeout_s);
  if (rc) return rc;
  p->pending = false;
  float ms = 0;
  cudaEventElapsedTime(&ms, p->e0, p->e1);
  fill_result(p, out);
  out->device_ms = ms;
  const uint32_t status = (uint32_t)p->h_res[2];
  if (status & DEV_WAIT_TIMEOUT) return LEC_ES_EDEVICE_WAIT;
  if (status) return LEC_ES_ECUDA;
  const uint64_t cex = p->h_res[0];
  const uint64_t W = num_words(p->prog.n);
  out->words_checked = p->last_we - p->last_wb;
  out->cex = cex;
  if (cex != UINT64_MAX) out->verdict = LEC_ES_NONEQUIVALENT;
  else if (p->last_wb == 0 && p->last_we >= W) out->verdict = LEC_ES_EQUIVALENT;
  else out->verdict = LEC_ES_UNDECIDED;
  // a full enumeration on the library's own geometry refines the time model
  if (out->verdict == LEC_ES_EQUIVALENT && p->last_default_grid)
    cost_add_run(c, p->tier, p->prog.cone_ands, p->prog.n, ms,
                 p->tier == LEC_ES_TIER_JIT && p->jit ? p->jit->model_lop3 : 0.0);
  return LEC_ES_OK;
}

}  // namespace lec

extern "C" int lec_es_prepare(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt,
                              lec_es_plan **out) {
  lec_es_plan *p = nullptr;
  int rc = plan_prepare(c, m, opt, &p);
  if (rc) {
    if (p) plan_release(c, p);
    return rc;
  }
  *out = p;
  return LEC_ES_OK;
}

extern "C" int lec_es_run_async(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt) {
  return plan_run_async(c, p, opt);
}

extern "C" int lec_es_plan_result(lec_es_ctx *c, lec_es_plan *p, lec_es_result *out) {
  return plan_result(c, p, out);
}

extern "C" int lec_es_plan_info(const lec_es_plan *p, lec_es_program_info *info) {
  if (!p || !info) return LEC_ES_EINVAL;
  const Program &g = p->prog;
  memset(info, 0, sizeof(*info));
  info->n = g.n;
  for (uint32_t k = 0; k < g.n; k++) info->support[k] = g.support[k];
  info->cone_ands = g.cone_ands;
  info->num_slots = g.num_slots;
  info->out_slot = g.out_slot;
  info->out_compl = g.out_compl;
  info->order = g.order;
  info->num_records = g.num_records;
  info->hash = g.hash;
  info->num_luts = g.lut.count;
  info->lut_live = g.lut.live;
  info->lop3_per_pass = p->tier == LEC_ES_TIER_JIT && p->jit ? p->jit->lop3_per_pass : 0.0;
  info->interp_step = g.step;
  return LEC_ES_OK;
}

extern "C" void lec_es_plan_free(lec_es_ctx *c, lec_es_plan *p) {
  if (!c || !p) return;
  if (p->pending) wait_event(p->e2, c->timeout_s);
  cudaStreamSynchronize(p->stream);
  plan_release(c, p);
}

namespace lec {

// A check the AUTO tier sends to the interpreter while its cone could run
// as a specialised kernel that the context does not hold yet: the kernel's
// build is scheduled in the background at once, and the interpreter runs
// the word range in ascending slices, the first of about kRaceSliceMs, each
// next twice as long up to kRaceSliceMaxMs (fewer slice boundaries, where the
// GPU waits for the host; a landed kernel waits at most that long).  A slice
// that fails ends the check (its counterexample is the lowest: every lower
// word has passed); once the kernel lands, the rest of the range goes to it.
// So a cold check takes about the lesser of the interpreter's time and the
// build's plus the kernel's on what is left, and the next check of the cone
// finds the kernel built.  Worth it only where a build can pay off.
constexpr double kRaceMinMs = 20.0;     // predicted interpreter time below this: no race
constexpr double kRaceSliceMs = 20.0;
constexpr double kRaceSliceMaxMs = 80.0;  // 16x16 miter: 6 slices instead of 17 (cold check 345 -> 339 ms)

bool race_wanted(lec_es_ctx *c, const lec_es_plan *p, const lec_es_options *opt) {
  if (opt && (opt->tier != LEC_ES_TIER_AUTO || opt->grid_blocks || opt->block_threads || opt->flags)) return false;
  if (p->tier == LEC_ES_TIER_JIT || jit_held(c, p->prog)) return false;
  if (!jit_eligible(p->prog) && !p->prog.lut.deferred) return false;
  const Program &g = p->prog;
  const uint64_t W = num_words(g.n);
  uint64_t wb = opt ? opt->word_begin : 0, we = opt ? std::min<uint64_t>(opt->word_end, W) : W;
  if (wb >= we) return false;
  const double t = cost_run_ms(c, LEC_ES_TIER_INTERP, g.cone_ands, g.n) * (double)(we - wb) / (double)W;
  return t >= kRaceMinMs;
}

int check_race(lec_es_ctx *c, lec_es_plan *p, const lec_es_miter *m, const lec_es_options *opt, lec_es_result *out) {
  const Program &g = p->prog;
  const uint64_t W = num_words(g.n);
  const uint64_t wb = opt ? opt->word_begin : 0, we = opt ? std::min<uint64_t>(opt->word_end, W) : W;
  const double t_int = std::max(1e-3, cost_run_ms(c, LEC_ES_TIER_INTERP, g.cone_ands, g.n));
  uint64_t slice = std::max<uint64_t>(1u << 16, (uint64_t)((double)W * kRaceSliceMs / t_int));
  const uint64_t slice_max = std::max<uint64_t>(slice, (uint64_t)((double)W * kRaceSliceMaxMs / t_int));
  std::shared_ptr<CompactMiter> cone;
  if (g.lut.deferred) {  // the build makes the table cover from its own copy of the cone
    cone = std::make_shared<CompactMiter>();
    if (compact_cone(MiterView{m->num_pis, m->num_ands, m->fanins, m->out_lit}, c->max_pis, *cone)) cone.reset();
  }
  jit_lookup_or_schedule(c, g, true, cone);
  lec_es_options o{};
  o.tier = LEC_ES_TIER_AUTO;
  double dev_ms = 0;
  uint64_t w = wb, cex = UINT64_MAX;
  uint32_t tier = p->tier;
  int rc = LEC_ES_OK;
  lec_es_result r{};
  while (w < we && cex == UINT64_MAX) {
    if (jit_lookup_or_schedule(c, g, true)) {  // the kernel has landed: it takes the rest
      lec_es_plan *jp = nullptr;
      lec_es_options oj{};
      oj.tier = LEC_ES_TIER_JIT;
      oj.word_begin = w;
      oj.word_end = we;
      Program copy = g;
      rc = plan_prepare_program(c, std::move(copy), &oj, &jp);
      if (!rc) rc = plan_run_async(c, jp, &oj);
      if (!rc) rc = plan_result(c, jp, &r);
      if (jp) lec_es_plan_free(c, jp);
      if (rc) return rc;
      dev_ms += r.device_ms;
      cex = r.cex;
      tier = LEC_ES_TIER_JIT;
      w = we;
      break;
    }
    o.word_begin = w;
    o.word_end = std::min(we, w + slice);
    slice = std::min(slice_max, 2 * slice);
    rc = plan_run_async(c, p, &o);
    if (!rc) rc = plan_result(c, p, &r);
    if (rc) return rc;
    dev_ms += r.device_ms;
    cex = r.cex;
    w = o.word_end;
  }
  fill_result(p, out);
  out->tier = tier;
  out->cex = cex;
  out->words_checked = we - wb;
  out->device_ms = dev_ms;
  if (cex != UINT64_MAX) out->verdict = LEC_ES_NONEQUIVALENT;
  else if (wb == 0 && we >= W) out->verdict = LEC_ES_EQUIVALENT;
  else out->verdict = LEC_ES_UNDECIDED;
  return LEC_ES_OK;
}

}  // namespace lec

extern "C" int lec_es_check_ex(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt,
                               lec_es_result *out) {
  if (!c || !m || !out) return LEC_ES_EINVAL;
  lec_es_plan *p = nullptr;
  const bool auto_tier = !opt || (opt->tier == LEC_ES_TIER_AUTO && !opt->grid_blocks && !opt->block_threads &&
                                  !opt->flags);
  t_check_race = auto_tier;
  int rc = lec_es_prepare(c, m, opt, &p);
  t_check_race = false;
  if (rc) return rc;
  if (race_wanted(c, p, opt)) {
    rc = check_race(c, p, m, opt, out);
  } else {
    rc = plan_run_async(c, p, opt);
    if (!rc) rc = plan_result(c, p, out);
  }
  lec_es_plan_free(c, p);
  return rc;
}

extern "C" int lec_es_check(lec_es_ctx *c, const lec_es_miter *m, lec_es_result *out) {
  return lec_es_check_ex(c, m, nullptr, out);
}

// ---- truth tables (interpreter with a per-AND store) ---------------------------------

extern "C" int lec_es_truth_tables(lec_es_ctx *c, const lec_es_miter *m, uint64_t word_begin, uint64_t word_end,
                                   uint32_t *vars_out, uint64_t *host_out) {
  if (!c || !m || !vars_out || !host_out) return LEC_ES_EINVAL;
  Program g;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc = compile_program(v, LEC_ES_ORDER_AUTO, c->max_pis, g);
  if (rc) return rc;
  const uint64_t W = num_words(g.n);
  if (word_begin >= word_end || word_end > W) return LEC_ES_EINVAL;
  const uint64_t nw = word_end - word_begin;
  // dump rows in ascending variable order
  std::vector<uint32_t> sorted(g.order_vars);
  std::sort(sorted.begin(), sorted.end());
  std::vector<uint32_t> row(g.recs.size() + 2, 0xFFFFFFFFu);
  {
    size_t j = 0;
    for (size_t r = 0; r < g.recs.size(); r++) {
      if (g.recs[r].op < 4) {
        const uint32_t var = g.order_vars[j++];
        row[r] = (uint32_t)(std::lower_bound(sorted.begin(), sorted.end(), var) - sorted.begin());
      }
    }
  }
  for (size_t j = 0; j < sorted.size(); j++) vars_out[j] = sorted[j];
  const size_t out_bytes = (size_t)sorted.size() * nw * 8u;
  lec_es_options o{};
  o.tier = LEC_ES_TIER_INTERP;
  PlanGeom geom{};
  rc = choose_interp_geometry(c, g, 2 * nw, &o, geom);
  if (rc) return rc;
  cudaSetDevice(c->device);
  void *d_recs = c->arena.alloc((size_t)geom.nrec_padded * sizeof(Rec));
  void *d_row = c->arena.alloc(row.size() * 4);
  void *d_out = c->arena.alloc(std::max<size_t>(out_bytes, 8));
  void *d_res = c->arena.alloc(kResWords * 8);
  void *d_spill = geom.spill ? c->arena.alloc((size_t)g.num_slots * geom.grid * geom.block * 4u) : nullptr;
  auto cleanup = [&]() {
    c->arena.free(d_recs);
    c->arena.free(d_row);
    c->arena.free(d_out);
    c->arena.free(d_res);
    c->arena.free(d_spill);
  };
  if (!d_recs || !d_row || !d_out || !d_res || (geom.spill && !d_spill)) {
    cleanup();
    return LEC_ES_ENOMEM;
  }
  std::vector<Rec> padded(geom.nrec_padded);
  memcpy(padded.data(), g.recs.data(), g.recs.size() * sizeof(Rec));
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemcpyAsync(d_recs, padded.data(), padded.size() * sizeof(Rec), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_row, row.data(), row.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, std::max<size_t>(out_bytes, 8), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_res, c->h_init, kResWords * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    cleanup();
    return LEC_ES_ECUDA;
  }
  InterpParams ip{};
  ip.recs = (const Rec *)d_recs;
  ip.nrec = (uint32_t)g.recs.size();
  ip.nrec_padded = geom.nrec_padded;
  ip.nslots = g.num_slots;
  ip.out_slot = g.out_slot;
  ip.out_compl = g.out_compl;
  ip.n = g.n;
  ip.ring_recs = geom.ring_recs;
  ip.resident = geom.resident;
  ip.chunk_begin = std::min<uint64_t>(2 * word_begin, num_chunks(g.n));
  ip.chunk_end = std::min<uint64_t>(2 * word_end, num_chunks(g.n));
  unsigned long long *res = (unsigned long long *)d_res;
  ip.cex = res + 4;  // a counterexample word nothing lowers: the dump never exits early
  ip.evaluated = res + 1;
  ip.status = (uint32_t *)(res + 2);
  ip.spill = (uint32_t *)d_spill;
  ip.tt_out = (uint64_t *)d_out;
  ip.tt_row = (const uint32_t *)d_row;
  ip.tt_words = nw;
  ip.tt_word_begin = word_begin;
  int err = launch_interp(ip, geom.block, geom.grid, geom.smem, geom.spill, st);
  uint32_t status = 0;
  if (!err) {
    e = cudaMemcpyAsync(host_out, d_out, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, res + 2, 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) err = 1;
  }
  const bool sync_ok = cudaStreamSynchronize(st) == cudaSuccess;
  cleanup();
  if (err || !sync_ok) return LEC_ES_ECUDA;
  if (status & DEV_WAIT_TIMEOUT) return LEC_ES_EDEVICE_WAIT;
  return status ? LEC_ES_ECUDA : LEC_ES_OK;
}

// Per-node values from a chosen kernel tier: SPILL the chunk interpreter
// (lec_es_truth_tables), INTERP the word interpreter es_interp_w with a
// store per AND record, JIT the specialised kernel's dump variant (its
// tables' nodes only; jit_dump_tables).
extern "C" int lec_es_truth_tables_ex(lec_es_ctx *c, const lec_es_miter *m, uint64_t word_begin, uint64_t word_end,
                                      uint32_t tier, uint32_t *vars_out, uint8_t *row_valid, uint64_t *host_out) {
  if (!c || !m || !vars_out || !host_out) return LEC_ES_EINVAL;
  if (tier != LEC_ES_TIER_SPILL && tier != LEC_ES_TIER_INTERP && tier != LEC_ES_TIER_JIT) return LEC_ES_EINVAL;
  Program g;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc = compile_program(v, LEC_ES_ORDER_AUTO, c->max_pis, g);
  if (rc) return rc;
  const uint64_t W = num_words(g.n);
  if (word_begin >= word_end || word_end > W) return LEC_ES_EINVAL;
  if (tier == LEC_ES_TIER_SPILL) {
    rc = lec_es_truth_tables(c, m, word_begin, word_end, vars_out, host_out);
    if (!rc && row_valid) memset(row_valid, 1, g.cone_ands);
    return rc;
  }
  const uint64_t nw = word_end - word_begin;
  std::vector<uint32_t> sorted(g.order_vars);
  std::sort(sorted.begin(), sorted.end());
  for (size_t j = 0; j < sorted.size(); j++) vars_out[j] = sorted[j];
  std::vector<uint8_t> valid(g.cone_ands, 0);
  if (tier == LEC_ES_TIER_JIT) {
    memset(host_out, 0, (size_t)g.cone_ands * nw * 8u);
    rc = jit_dump_tables(c, g, word_begin, word_end, host_out, valid.data());
    if (rc) return rc;
    if (row_valid) memcpy(row_valid, valid.data(), valid.size());
    return LEC_ES_OK;
  }
  PlanGeom geom{};
  if (!choose_word_geometry(c, g, nullptr, geom)) return LEC_ES_ETOOBIG;  // slots beyond shared memory
  std::vector<XRec> xr;
  std::vector<XLoad> xl;
  uint32_t out_off = 0;
  encode_w(g, geom.block, xr, xl, out_off);
  for (size_t j = 0; j < xr.size(); j++) {  // the j-th AND record computes order_vars[j]
    const uint32_t row = (uint32_t)(std::lower_bound(sorted.begin(), sorted.end(), g.order_vars[j]) - sorted.begin());
    xr[j].ctl |= (row + 1u) << kCtlRowShift;
  }
  const size_t out_bytes = (size_t)g.cone_ands * nw * 8u;
  cudaSetDevice(c->device);
  void *d_recs = c->arena.alloc(std::max<size_t>(16, xr.size() * sizeof(XRec)));
  void *d_loads = c->arena.alloc(std::max<size_t>(16, xl.size() * sizeof(XLoad)));
  void *d_out = c->arena.alloc(std::max<size_t>(out_bytes, 8));
  unsigned long long *d_res = (unsigned long long *)c->arena.alloc(kResWords * 8);
  auto cleanup = [&]() {
    c->arena.free(d_recs);
    c->arena.free(d_loads);
    c->arena.free(d_out);
    c->arena.free(d_res);
  };
  if (!d_recs || !d_loads || !d_out || !d_res) {
    cleanup();
    return LEC_ES_ENOMEM;
  }
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  if (!xr.empty()) e = cudaMemcpyAsync(d_recs, xr.data(), xr.size() * sizeof(XRec), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !xl.empty())
    e = cudaMemcpyAsync(d_loads, xl.data(), xl.size() * sizeof(XLoad), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, std::max<size_t>(out_bytes, 8), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_res, c->h_init, kResWords * 8, cudaMemcpyHostToDevice, st);
  int err = e == cudaSuccess ? 0 : 1;
  if (!err) {
    XParams xp{};
    xp.recs = (const XRec *)d_recs;
    xp.loads = (const XLoad *)d_loads;
    xp.nrec = geom.nrec_padded;
    xp.nload = (uint32_t)xl.size();
    xp.step = g.step;
    xp.out_off = out_off;
    xp.out_compl = g.out_compl;
    xp.n = g.n;
    xp.ring_recs = geom.ring_recs;
    xp.resident = geom.resident;
    xp.word_begin = word_begin;
    xp.word_end = word_end;
    xp.cex = d_res + 4;  // never lowered: the dump variant reports nothing
    xp.evaluated = d_res + 1;
    xp.status = (uint32_t *)(d_res + 2);
    xp.tt_out = (uint64_t *)d_out;
    xp.tt_words = nw;
    err = launch_interp_w_tt(xp, geom.block, geom.grid, geom.smem, st);
  }
  uint32_t status = 0;
  if (!err) {
    e = cudaMemcpyAsync(host_out, d_out, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_res + 2, 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) err = 1;
  }
  const bool sync_ok = cudaStreamSynchronize(st) == cudaSuccess;
  cleanup();
  if (err || !sync_ok) return LEC_ES_ECUDA;
  if (status & DEV_WAIT_TIMEOUT) return LEC_ES_EDEVICE_WAIT;
  if (status) return LEC_ES_ECUDA;
  if (row_valid) memset(row_valid, 1, g.cone_ands);
  return LEC_ES_OK;
}

// ---- LOP3 peak microbenchmark ------------------------------------------------------

extern "C" int lec_es_lop3_peak(lec_es_ctx *c, double *per_clk_per_sm, int *sm_count, int *clock_khz,
                                double *lop3_per_s) {
  if (!c) return LEC_ES_EINVAL;
  cudaSetDevice(c->device);
  const int block = 256, grid = c->sm_count * 8, iters = 4096;
  uint32_t *d_out = (uint32_t *)c->arena.alloc((size_t)grid * block * 4);
  unsigned long long *d_cyc = (unsigned long long *)c->arena.alloc(16);
  if (!d_out || !d_cyc) {
    c->arena.free(d_out);
    c->arena.free(d_cyc);
    return LEC_ES_ENOMEM;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int err = launch_lop3_bench(d_out, d_cyc, grid, block, 64, c->stream);  // warm-up
  cudaEventRecord(a, c->stream);
  if (!err) err = launch_lop3_bench(d_out, d_cyc, grid, block, iters, c->stream);
  cudaEventRecord(b, c->stream);
  unsigned long long cyc[2] = {0, 0};
  if (!err) err = (int)cudaMemcpyAsync(cyc, d_cyc, 16, cudaMemcpyDeviceToHost, c->stream);
  const bool ok = cudaStreamSynchronize(c->stream) == cudaSuccess && !err;
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->arena.free(d_out);
  c->arena.free(d_cyc);
  if (!ok || ms <= 0 || cyc[1] == 0) return LEC_ES_ECUDA;
  const double total = (double)grid * block * iters * 16.0 * 8.0;  // LOP3 lanes
  const double khz = (double)cyc[0] / (double)cyc[1] * 1e6;         // cycles per ns -> kHz
  // results per SM per clock over the whole kernel at the measured clock
  if (per_clk_per_sm) *per_clk_per_sm = total / ((double)ms * 1e-3 * khz * 1e3 * c->sm_count);
  if (sm_count) *sm_count = c->sm_count;
  if (clock_khz) *clock_khz = (int)khz;
  if (lop3_per_s) *lop3_per_s = total / (ms * 1e-3);
  return LEC_ES_OK;
}
