// jit.cpp -- specialised exact-simulation kernels compiled at run time.
//
// The slot program of one cone (paper §3.3: a branch-free instruction stream
// over reference-counted registers) is emitted as straight-line CUDA C++ in
// which every AND is one 32-bit expression (one LOP3 after compilation, with
// the complements folded into the LUT) and every value lives in a register.
// The register allocator sees exactly the live ranges the slot program's
// evaluation order creates, so the slot count bounds the register demand.
// NVRTC compiles the source for sm_103a straight to a cubin (cached in
// memory by program hash and optionally on disk); the runtime's library API
// loads it, so the library never links the driver API.
//
// Work split: thread t of the grid takes 32-pattern chunks c = begin + t,
// begin + t + T, ... (T = threads in the grid).  For each chunk it forms the
// support PI words (constant masks for PIs 0..4, all-ones/all-zeros from the
// bits of c for PIs >= 5), runs the body, and reduces the miter output with a
// warp ballot; the lowest failing lane does atomicMin on the counterexample.
// Before every chunk a warp compares its first pattern with the current
// counterexample (loaded one iteration ahead) and stops if it is not lower.
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <fstream>
#include <thread>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "es_ctx.h"
#include "es_internal.h"

namespace lec {

struct JitState {
  std::mutex mu;
  std::map<uint64_t, JitKernel *> cache;
  // background compiles for the server
  std::map<uint64_t, bool> scheduled;
  std::vector<std::thread> workers;
  std::deque<Program> todo;
  std::condition_variable cv;
  bool stop = false;
};

namespace {

constexpr int kJitBlock = 128;
constexpr uint32_t kMaxJitSlots = 240;   // beyond this the register file spills
constexpr uint64_t kJitMinWork = 1ull << 34;  // AND-chunk evaluations that repay a compile

const char *kMask32[5] = {"0xAAAAAAAAu", "0xCCCCCCCCu", "0xF0F0F0F0u", "0xFF00FF00u", "0xFFFF0000u"};

std::string gen_source(const Program &g) {
  std::ostringstream s;
  s << "typedef unsigned int u32; typedef unsigned long long u64;\n"
       "extern \"C\" __global__ void __launch_bounds__("
    << kJitBlock
    << ") es_jit(const u64 cb, const u64 ce, u64 *cex, u64 *evaluated) {\n"
       "  const u64 T = (u64)gridDim.x * "
    << kJitBlock
    << ";\n"
       "  const unsigned lane = threadIdx.x & 31u;\n"
       "  u64 done = 0;\n"
       "  u64 cur = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile u64 *)cex : 0ull, 0);\n"
       "  for (u64 base = cb + (u64)blockIdx.x * "
    << kJitBlock
    << "; base < ce; base += T) {\n"
       "    const u64 wfirst = base + (threadIdx.x & ~31u);\n"
       "    if (wfirst * 32ull >= cur) break;\n"
       "    const u64 nxt = lane == 0 ? *(volatile u64 *)cex : 0ull;\n"
       "    const u64 c = base + threadIdx.x;\n"
       "    const u32 clo = (u32)c, chi = (u32)(c >> 32);\n";
  // value names per slot, rebound as records execute
  std::vector<std::string> slot(g.num_slots);
  auto opnd = [&](uint32_t sl, bool neg) { return neg ? "~" + slot[sl] : slot[sl]; };
  size_t i = 0;
  for (const Rec &r : g.recs) {
    if (r.op == OP_PI) {
      const uint32_t k = r.a;
      std::string nm = "p" + std::to_string(k);
      if (k < 5) {
        s << "    const u32 " << nm << " = " << kMask32[k] << ";\n";
      } else if (k - 5 < 32) {
        s << "    const u32 " << nm << " = 0u - ((clo >> " << (k - 5) << ") & 1u);\n";
      } else {
        s << "    const u32 " << nm << " = 0u - ((chi >> " << (k - 37) << ") & 1u);\n";
      }
      slot[r.dst] = nm;
    } else if (r.op == OP_CONST0) {
      slot[r.dst] = "0u";
    } else {
      std::string nm = "v" + std::to_string(i);
      s << "    const u32 " << nm << " = " << opnd(r.a, r.op & 1) << " & " << opnd(r.b, (r.op >> 1) & 1)
        << ";\n";
      slot[r.dst] = nm;
    }
    i++;
  }
  const uint32_t vmask = g.n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << g.n)) - 1u);
  s << "    u32 out = (" << (g.out_compl ? "~" : "") << slot[g.out_slot] << ") & 0x" << std::hex << vmask
    << std::dec
    << "u;\n"
       "    if (c >= ce) out = 0u;\n"
       "    const unsigned bal = __ballot_sync(0xffffffffu, out != 0u);\n"
       "    if (bal) {\n"
       "      if ((int)lane == __ffs(bal) - 1) atomicMin(cex, c * 32ull + (u64)(__ffs(out) - 1));\n"
       "    }\n"
       "    done += (c < ce) ? 1ull : 0ull;\n"
       "    cur = __shfl_sync(0xffffffffu, nxt, 0);\n"
       "  }\n"
       "  for (int o = 16; o > 0; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);\n"
       "  if (lane == 0 && done) atomicAdd(evaluated, done * 32ull);\n"
       "}\n";
  return s.str();
}

bool read_file(const std::string &path, std::vector<char> &out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  out.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
  return !out.empty();
}

void write_file(const std::string &path, const std::vector<char> &data) {
  std::string tmp = path + ".tmp";
  std::ofstream f(tmp, std::ios::binary);
  if (!f) return;
  f.write(data.data(), (std::streamsize)data.size());
  f.close();
  rename(tmp.c_str(), path.c_str());
}

int compile_cubin(const std::string &src, int major, int minor, std::vector<char> &cubin, std::string &log) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "es_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return LEC_ES_EJIT;
  // sm_103a on B300; the "a" suffix targets this exact architecture
  std::string arch = "-arch=sm_" + std::to_string(major) + std::to_string(minor) + "a";
  // NVRTC optimises by default; -Xptxas -v puts register and spill counts in the log
  const char *opts[] = {arch.c_str(), "--std=c++17", "-lineinfo", "-diag-suppress=177", "-Xptxas", "-v"};
  nvrtcResult rc = nvrtcCompileProgram(prog, 6, opts);
  size_t lsz = 0;
  nvrtcGetProgramLogSize(prog, &lsz);
  if (lsz > 1) {
    log.resize(lsz);
    nvrtcGetProgramLog(prog, &log[0]);
  }
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return LEC_ES_EJIT;
  }
  size_t n = 0;
  if (nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
    nvrtcDestroyProgram(&prog);
    return LEC_ES_EJIT;
  }
  cubin.resize(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return LEC_ES_OK;
}

}  // namespace

uint32_t jit_auto_tier(lec_es_ctx *c, const Program &g, uint64_t chunks) {
  (void)c;
  const uint64_t work = (uint64_t)g.recs.size() * chunks;
  if (g.num_slots <= kMaxJitSlots && work >= kJitMinWork) return LEC_ES_TIER_JIT;
  return LEC_ES_TIER_INTERP;
}

namespace {

// Compile (or read from the disk cache) and load one program's kernel.
int build_kernel(lec_es_ctx *c, const Program &g, JitKernel **out) {
  const double t0 = now_ms();
  std::vector<char> cubin;
  std::string path;
  if (!c->jit_dir.empty()) {
    mkdir(c->jit_dir.c_str(), 0755);
    char name[64];
    snprintf(name, sizeof(name), "/es_%016llx_sm%d%d.cubin", (unsigned long long)g.hash, c->cc_major,
             c->cc_minor);
    path = c->jit_dir + name;
  }
  if (path.empty() || !read_file(path, cubin)) {
    std::string log;
    int rc = compile_cubin(gen_source(g), c->cc_major, c->cc_minor, cubin, log);
    if (rc) {
      if (getenv("LEC_ES_JIT_LOG")) fprintf(stderr, "lec_es JIT failed:\n%s\n", log.c_str());
      return rc;
    }
    if (!path.empty()) write_file(path, cubin);
  }
  cudaSetDevice(c->device);
  JitKernel *k = new JitKernel();
  if (cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&k->kern, k->lib, "es_jit") != cudaSuccess) {
    if (k->lib) cudaLibraryUnload(k->lib);
    delete k;
    return LEC_ES_EJIT;
  }
  cudaFuncAttributes attr;
  if (cudaFuncGetAttributes(&attr, (const void *)k->kern) == cudaSuccess) {
    k->regs = attr.numRegs;
    k->local_bytes = attr.localSizeBytes;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)k->kern, kJitBlock, 0);
  k->blocks_per_sm = std::max(1, bps);
  k->block = kJitBlock;
  k->compile_ms = now_ms() - t0;
  *out = k;
  return LEC_ES_OK;
}

void worker_loop(lec_es_ctx *c) {
  JitState *js = c->jit;
  for (;;) {
    Program g;
    {
      std::unique_lock<std::mutex> lk(js->mu);
      js->cv.wait(lk, [&] { return js->stop || !js->todo.empty(); });
      if (js->stop) return;
      g = std::move(js->todo.front());
      js->todo.pop_front();
    }
    JitKernel *k = nullptr;
    int rc = build_kernel(c, g, &k);
    std::lock_guard<std::mutex> lk(js->mu);
    if (rc == LEC_ES_OK) js->cache[g.hash] = k;
  }
}

JitState *state(lec_es_ctx *c) {
  if (!c->jit) c->jit = new JitState();
  return c->jit;
}

}  // namespace

int jit_attach(lec_es_ctx *c, lec_es_plan *p, JitKernel *k, const lec_es_options *opt) {
  const Program &g = p->prog;
  p->jit = k;
  p->jit_block = k->block;
  const uint64_t chunks = num_chunks(g.n);
  uint64_t grid = (uint64_t)c->sm_count * k->blocks_per_sm;
  if (opt && opt->grid_blocks) grid = opt->grid_blocks;
  grid = std::min<uint64_t>(grid, (chunks + k->block - 1) / k->block);
  p->jit_grid = (int)std::max<uint64_t>(1, grid);
  return LEC_ES_OK;
}

int jit_prepare(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt) {
  const Program &g = p->prog;
  JitState *js = state(c);
  JitKernel *k = nullptr;
  {
    std::lock_guard<std::mutex> lk(js->mu);
    auto it = js->cache.find(g.hash);
    if (it != js->cache.end()) k = it->second;
  }
  if (k) {
    p->jit_ms = 0;
  } else {
    int rc = build_kernel(c, g, &k);
    if (rc) return rc;
    p->jit_ms = k->compile_ms;
    std::lock_guard<std::mutex> lk(js->mu);
    auto it = js->cache.find(g.hash);
    if (it != js->cache.end()) {  // raced with a background compile
      cudaLibraryUnload(k->lib);
      delete k;
      k = it->second;
    } else {
      js->cache[g.hash] = k;
    }
  }
  return jit_attach(c, p, k, opt);
}

JitKernel *jit_lookup_or_schedule(lec_es_ctx *c, const Program &g) {
  JitState *js = state(c);
  std::lock_guard<std::mutex> lk(js->mu);
  auto it = js->cache.find(g.hash);
  if (it != js->cache.end()) return it->second;
  if (!js->scheduled[g.hash]) {
    js->scheduled[g.hash] = true;
    js->todo.push_back(g);
    if (js->workers.empty()) {
      const unsigned nw = std::max(1u, std::min(4u, std::thread::hardware_concurrency() / 2));
      for (unsigned i = 0; i < nw; i++) js->workers.emplace_back(worker_loop, c);
    }
    js->cv.notify_one();
  }
  return nullptr;
}

int jit_launch(lec_es_ctx *c, lec_es_plan *p, uint64_t chunk_begin, uint64_t chunk_end, int grid) {
  (void)c;
  unsigned long long *cex = p->d_res, *evaluated = p->d_res + 1;
  void *args[] = {&chunk_begin, &chunk_end, &cex, &evaluated};
  const int g = grid > 0 ? grid : p->jit_grid;
  cudaError_t e = cudaLaunchKernel((const void *)p->jit->kern, dim3(g), dim3(p->jit_block), args, 0, p->stream);
  return e == cudaSuccess ? 0 : (int)e;
}

void jit_release_all(lec_es_ctx *c) {
  if (!c->jit) return;
  JitState *js = c->jit;
  {
    std::lock_guard<std::mutex> lk(js->mu);
    js->stop = true;
  }
  js->cv.notify_all();
  for (auto &t : js->workers) t.join();
  for (auto &kv : js->cache) {
    if (kv.second->lib) cudaLibraryUnload(kv.second->lib);
    delete kv.second;
  }
  delete js;
  c->jit = nullptr;
}

// Source of the specialised kernel (no GPU needed).
std::string jit_source_for(const Program &g) { return gen_source(g); }

}  // namespace lec

extern "C" int lec_es_jit_compile(const lec_es_miter *m, int cc_major, int cc_minor, char *log, size_t log_cap,
                                  uint64_t *cubin_bytes) {
  if (!m) return LEC_ES_EINVAL;
  lec::Program g;
  lec::MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc = lec::compile_program(v, LEC_ES_ORDER_AUTO, 63, g);
  if (rc) return rc;
  std::vector<char> cubin;
  std::string lg;
  rc = lec::compile_cubin(lec::gen_source(g), cc_major, cc_minor, cubin, lg);
  if (log && log_cap) {
    const size_t n = std::min(log_cap - 1, lg.size());
    memcpy(log, lg.data(), n);
    log[n] = 0;
  }
  if (cubin_bytes) *cubin_bytes = cubin.size();
  return rc;
}
