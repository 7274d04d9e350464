// jit.cpp -- specialised exact-simulation kernels compiled at run time.
//
// The cone of one miter (paper §3.3: a branch-free instruction stream over
// reference-counted registers) becomes straight-line code in which every
// value lives in a register.  Two forms:
//
//   table form (default): the cone's 3-input table cover (lutmap.cpp) is
//     written directly as PTX, one lop3 per table with constants as
//     immediates, and compiled for sm_103a by the PTX compiler library;
//   C++ forms: one expression per AND (LEC_ES_FLAG_JIT_AND_FORM), or the
//     tables as C++ (LEC_ES_JIT_NVRTC), compiled by NVRTC -- kept for the
//     AND option and for comparing the compilation paths.
//
// Cubins are cached in memory by the cone's structural hash and optionally
// on disk; the runtime's library API loads them (no driver API).
//
// Work split of the table form: bits 0..4 of a 32-pattern chunk index are
// the lane (support PIs 5..9, fixed per thread); a few support PIs are pass
// PIs and the rest select the grab.  Warps take grabs from a counter (one
// ahead) or, on small launches, by a static stride; a grab is every chunk
// whose grab bits spell its number, run as passes over the pass PIs in
// nested loops (jit_layout, choose_pass_groups, and dry runs of the
// generator for large cones).  Each table runs once per iteration of the
// loop of its deepest pass PI (plan_hoist decides what survives a loop);
// the innermost levels are unrolled with their PIs folded as constants.
// The miter output is reduced with a warp ballot and the lowest failing
// lane does atomicMin on the counterexample.  Early exit: a warp stops when
// its grab's lowest pattern is not below the counterexample, and inside a
// grab it skips every loop iteration and pass whose first pattern is not
// below it (the poll is refreshed once per iteration of the innermost
// loop), so a counterexample in the high pass PIs prunes the passes above
// it in every later grab, not only the grabs above it.
#include <cuda_runtime.h>
#include <nvPTXCompiler.h>
#include <nvrtc.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/resource.h>
#include <sys/stat.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <fstream>
#include <thread>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "es_ctx.h"
#include "es_internal.h"

namespace lec {

struct JitState {
  std::mutex mu;
  std::map<uint64_t, JitKernel *> cache;  // by cache_key; an entry serves a program only if hash2 matches too
  std::vector<JitKernel *> unshared;      // built for a program whose key another program holds
  // background compiles (the server, and a single check racing the
  // interpreter against its kernel's build); inflight: scheduled and not
  // finished (jit_get_kernel waits for those instead of building twice)
  std::map<uint64_t, bool> scheduled;
  std::set<uint64_t> inflight;
  std::vector<std::thread> workers;
  struct Job {
    Program prog;
    bool urgent;                                // build its chain of layouts at once
    std::shared_ptr<const CompactMiter> cone;   // for a program whose cover is deferred
  };
  std::deque<Job> todo;
  std::condition_variable cv, built;
  bool stop = false;
};

namespace {

constexpr int kJitBlock = 128;
constexpr int kCodegenVersion = 26;  // part of cached cubin names: bump whenever the generated code changes
// Values computed at one loop level and read at a deeper one: at most
// kHoistPlan of them (see plan_hoist), those read by the innermost loop in
// registers, the others in up to kHoistShared shared-memory slots per
// thread.  Up to kStaticShared slots (96 x 128 threads x 4 B = 48 KB, the
// most a kernel may declare statically) are a static array; a kernel with
// more declares them as dynamic shared memory and is launched with that size
// (192 slots = 96 KB per block: two blocks still fit an SM, as the register
// file allows).
constexpr uint32_t kHoistPlan = 224;
constexpr uint32_t kHoistShared = 192;
constexpr uint32_t kStaticShared = 96;
// Dynamic shared memory a kernel with `slots` shared slots per thread is
// launched with (0 when they fit the static array).
size_t jit_dyn_smem(uint32_t slots) { return slots > kStaticShared ? (size_t)slots * kJitBlock * 4u : 0; }
constexpr uint64_t kGrabsWanted = 4 * 148 * 8;  // four grabs per warp at 8 warps on each of 148 SMs
// A kernel takes grabs by a static warp stride only when a launch has at
// most two per resident warp; one whose full range has more grabs than
// twice the most warps that can be resident (148 SMs x 64 warps) never
// does, and is generated without that code (it would hold two registers).
constexpr uint64_t kStrideMaxGrabs = 2 * 148 * 64;
// Cones of at least this many tables build their chain of layouts in
// parallel (see compile_program_kernel), at most kMaxChain layouts at once.
constexpr uint32_t kParallelChainTables = 1000;
constexpr uint32_t kMaxChain = 12;
constexpr int kBuildNice = 10;  // nice value of background build threads
constexpr uint32_t kDryPlan = 160;  // plan of the layout search's dry runs (see jit_layout)
// Set while a single plan's kernel builds on the calling thread (the host is
// otherwise idle): a large cone's first layout and the rest of its chain then
// build at once, instead of the rest only after the first spills.
thread_local bool t_single_build = false;
// Largest table live set given a specialised kernel: values kept across pass
// loops go to registers and up to kHoistShared shared slots, and a layout
// that still spills is kept only if every candidate does (whole multiplier
// miters: 16x16 198 live, 18x18 237, 20x20 265, all built without spills).
constexpr uint32_t kMaxJitLive = 288;
// A cone whose tables keep at most kFewLive values live is not register-bound:
// its innermost pass levels unroll into up to 64 copies, and the passes run
// in straight-line groups of up to kGroupPasses passes and kGroupEvals table
// evaluations (gen_ptx_lut).  Measured on the 4,096-pair batch and the
// 4,096-miter spread batch (batch ms / preparation s): no groups 3.83 / 2.8
// and 24.8 / 19.6; groups of 8 passes with at most 256, 512, 1,024 or any
// number of evaluations 2.61 / 1.8 and 21.0 / 19.0, 2.59 / 1.9 and 20.1 /
// 28.1, 2.59 / 1.9 and 19.7 / 40.1, 2.58 / 1.9 and 19.8 / 45.8 (longer
// straight-line blocks cost the PTX compiler more); groups of 4: 2.72 / 2.6
// and 20.1 / 40.4.
constexpr uint32_t kFewLive = 96;
constexpr uint32_t kGroupPasses = 8;
// A grouped kernel's passes cost about this many lop3-equivalents less
// control than the time model's per-pass allowance (cost.cpp: 40); fitted
// over 225 measured kernels (90th-percentile error 25% -> 21%).
constexpr double kGroupedPassSaving = -20.0;
constexpr uint64_t kGroupEvals = 512;

// The counterexample word (a pattern; UINT64_MAX while none is known) as
// the first 32-pattern chunk it rules out, ceil(cex / 32), kept in %d12
// (a found cex is below 2^63, so the clamp changes only "none").
const std::string kCexToChunk =
    "  min.u64 %d12, %d12, 0x8000000000000000;\n  add.u64 %d12, %d12, 31;\n  shr.u64 %d12, %d12, 5;\n";
// Inside a grab: lane 0's earlier poll (%d17) becomes the warp's %d12 and
// lane 0 polls again for the next refresh, so the load's latency is hidden
// behind the work in between.
const std::string kCexRefresh =
    "  mov.b64 {%t3, %t4}, %d17;\n  shfl.sync.idx.b32 %t3, %t3, 0, 31, -1;\n"
    "  shfl.sync.idx.b32 %t4, %t4, 0, 31, -1;\n  mov.b64 %d12, {%t3, %t4};\n" +
    kCexToChunk + "  @%p1 ld.volatile.global.u64 %d17, [%d3];\n";

const char *kMask32[5] = {"0xAAAAAAAAu", "0xCCCCCCCCu", "0xF0F0F0F0u", "0xFF00FF00u", "0xFFFF0000u"};

// Kernel prologue / epilogue shared by the C++ code forms; the launch
// contract is the PTX form's: a counter hands out grab numbers, grab q is
// chunks [q*G, (q+1)*G) of the whole pattern space (G = 32 * rep, rep a power
// of two) intersected with [cb, ce), taken one ahead, so warps that run
// faster take more and all finish together.  A warp stops at the end of the
// range, when its grab's first pattern is not below the current
// counterexample, or after max_grabs grabs (the server bounds block lifetimes
// this way).
void emit_prologue(std::ostringstream &s) {
  s << "typedef unsigned int u32; typedef unsigned long long u64;\n"
       "extern \"C\" __global__ void __launch_bounds__("
    << kJitBlock
    << ") es_jit(const u64 cb, const u64 ce, u64 *cex, u64 *evaluated, u64 *next, const u64 max_grabs,\n"
       "    const u64 rep, const u64 q0_host, const u64 qend_host) {\n"
       "  (void)q0_host; (void)qend_host;\n"
       "  const unsigned lane = threadIdx.x & 31u;\n"
       "  const u64 G = 32ull * rep, q0 = cb / G, qend = (ce + G - 1) / G;\n"
       "  u64 done = 0;\n"
       "  u64 mine = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(next, 1ull) : 0ull, 0);\n"
       "  u64 cur = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile u64 *)cex : 0ull, 0);\n"
       "  for (u64 g = 1; ; g++) {\n"
       "    const u64 q = q0 + mine;\n"
       "    if (q >= qend) break;\n"
       "    const u64 gfirst = q * G;\n"
       "    if ((gfirst > cb ? gfirst : cb) * 32ull >= cur) break;\n"
       "    const bool more = g < max_grabs;\n"
       "    const u64 ahead = (lane == 0 && more) ? atomicAdd(next, 1ull) : ~0ull;\n"
       "    const u64 nxt = lane == 0 ? *(volatile u64 *)cex : 0ull;\n"
       "    for (u64 r = 0; r < rep; r++) {\n"
       "    const u64 base = gfirst + 32ull * r;\n"
       "    if (base >= ce) break;\n"
       "    if (base * 32ull >= cur) break;\n"
       "    if (base + 32ull <= cb) continue;\n"
       "    const u64 c = base + lane;\n"
       "    const u32 clo = (u32)c, chi = (u32)(c >> 32);\n"
       "    (void)chi;\n";
}

void emit_epilogue(std::ostringstream &s, const std::string &outv, bool compl_, uint32_t n) {
  const uint32_t vmask = n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << n)) - 1u);
  s << "    u32 out = (" << (compl_ ? "~" : "") << outv << ") & 0x" << std::hex << vmask << std::dec
    << "u;\n"
       "    const bool inside = c >= cb && c < ce;\n"
       "    if (!inside) out = 0u;\n"
       "    const unsigned bal = __ballot_sync(0xffffffffu, out != 0u);\n"
       "    if (bal) {\n"
       "      if ((int)lane == __ffs(bal) - 1) atomicMin(cex, c * 32ull + (u64)(__ffs(out) - 1));\n"
       "    }\n"
       "    done += inside ? 1ull : 0ull;\n"
       "    }\n"
       "    mine = __shfl_sync(0xffffffffu, ahead, 0);\n"
       "    cur = __shfl_sync(0xffffffffu, nxt, 0);\n"
       "    if (!more) break;\n"
       "  }\n"
       "  for (int o = 16; o > 0; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);\n"
       "  if (lane == 0 && done) atomicAdd(evaluated, done * 32ull);\n"
       "}\n";
}

std::string pi_expr(uint32_t k) {
  if (k < 5) return kMask32[k];
  if (k - 5 < 32) return "(0u - ((clo >> " + std::to_string(k - 5) + ") & 1u))";
  return "(0u - ((chi >> " + std::to_string(k - 37) + ") & 1u))";
}

// AND form: one C expression per AND of the slot program; the compiler forms
// its own 3-input LOP3s.
std::string gen_source_and(const Program &g) {
  std::ostringstream s;
  emit_prologue(s);
  std::vector<std::string> slot(g.num_slots);
  auto opnd = [&](uint32_t sl, bool neg) { return neg ? "~" + slot[sl] : slot[sl]; };
  size_t i = 0;
  for (const Rec &r : g.recs) {
    if (r.op == OP_PI) {
      const std::string nm = "p" + std::to_string(r.a);
      s << "    const u32 " << nm << " = " << pi_expr(r.a) << ";\n";
      slot[r.dst] = nm;
    } else if (r.op == OP_CONST0) {
      slot[r.dst] = "0u";
    } else {
      const std::string nm = "v" + std::to_string(i);
      s << "    const u32 " << nm << " = " << opnd(r.a, r.op & 1) << " & " << opnd(r.b, (r.op >> 1) & 1)
        << ";\n";
      slot[r.dst] = nm;
    }
    i++;
  }
  emit_epilogue(s, slot[g.out_slot], g.out_compl, g.n);
  return s.str();
}

// Table form: one lop3 per 3-input table of the cover, in the cover's
// evaluation order; tables whose leaves are all constants (the constant and
// PI masks 0..4) are folded here.
std::string gen_source_lut(const Program &g) {
  const LutProgram &lp = g.lut;
  std::ostringstream s;
  emit_prologue(s);
  const uint32_t NA = lp.na, NP = lp.np;
  const size_t NV = NA + NP + 1;
  std::vector<std::string> name(NV);
  std::vector<int8_t> isconst(NV, 0);
  std::vector<uint32_t> cval(NV, 0);
  std::vector<uint8_t> emitted(NV, 0);
  static const uint32_t mask[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
  for (uint32_t k = 0; k < NP; k++) {
    name[NA + k] = "p" + std::to_string(k);
    if (k < 5) {
      isconst[NA + k] = 1;
      cval[NA + k] = mask[k];
    }
  }
  isconst[NA + NP] = 1;
  cval[NA + NP] = 0;
  auto operand = [&](int32_t id) -> std::string {
    if (id < 0) return "0u";
    if (isconst[id]) {
      char b[16];
      snprintf(b, sizeof(b), "0x%08xu", cval[id]);
      return b;
    }
    if (id >= (int32_t)NA && !emitted[id]) {  // PI from the chunk index, at first use
      s << "    const u32 " << name[id] << " = " << pi_expr((uint32_t)(id - NA)) << ";\n";
      emitted[id] = 1;
    }
    return name[id];
  };
  for (const auto &l : lp.order) {
    const int32_t v = l.node;
    name[v] = "v" + std::to_string(v);
    bool allc = true;
    for (int k = 0; k < l.n; k++) allc = allc && isconst[l.leaf[k]];
    if (allc) {
      uint32_t x[3] = {0, 0, 0};
      for (int k = 0; k < l.n; k++) x[k] = cval[l.leaf[k]];
      uint32_t r = 0;
      for (int b = 0; b < 32; b++) {
        const int m = (int)((x[0] >> b) & 1) | (int)(((x[1] >> b) & 1) << 1) | (int)(((x[2] >> b) & 1) << 2);
        r |= (uint32_t)((l.tt >> m) & 1) << b;
      }
      isconst[v] = 1;
      cval[v] = r;
      continue;
    }
    const std::string x0 = operand(l.leaf[0]), x1 = operand(l.n > 1 ? l.leaf[1] : -1),
                      x2 = operand(l.n > 2 ? l.leaf[2] : -1);
    char lut[8];
    snprintf(lut, sizeof(lut), "0x%02x", l.tt);
    // lop3 operands a, b, c carry the patterns 0xF0, 0xCC, 0xAA: (x2, x1, x0)
    s << "    u32 " << name[v] << "; asm(\"lop3.b32 %0, %1, %2, %3, " << lut << ";\" : \"=r\"(" << name[v]
      << ") : \"r\"(" << x2 << "), \"r\"(" << x1 << "), \"r\"(" << x0 << "));\n";
  }
  std::string outv;
  if (lp.root < 0) {
    outv = "0u";
  } else {
    outv = operand((int32_t)lp.root);
  }
  emit_epilogue(s, outv, g.out_compl, g.n);
  return s.str();
}

std::string gen_source(const Program &g, bool lut_form) {
  return lut_form && !g.lut.order.empty() ? gen_source_lut(g) : gen_source_and(g);
}

// The grab layout of a table-form kernel (jit_layout).
struct GrabLayout {
  uint32_t rep = 0;
  uint32_t regs = 0;  // values read below their level that may stay in registers
  uint32_t plan = 0;  // values read below their level, in all (plan_hoist's budget)
  uint64_t pass_pis = 0;
  std::vector<uint64_t> groups;
};
// Slots of one generated kernel: values read below their level, how many in
// registers and how many in shared memory.
struct SlotSplit {
  uint32_t read = 0, in_regs = 0, in_shared = 0;
  uint32_t inner_in_regs = 0;  // of those in registers, values the innermost loop reads
  bool grouped = false;        // passes run in straight-line groups (the same for every budget)
};
// Most straight-line copies of the innermost pass levels (see gen_ptx_lut).
uint32_t unroll_copies(const LutProgram &lp) {
  const char *unroll_env = getenv("LEC_ES_JIT_UNROLL");
  return unroll_env ? (uint32_t)std::max(0, atoi(unroll_env)) : (lp.live <= kFewLive ? 64u : 4u);
}
// shared-memory slots per thread (LEC_ES_JIT_HOIST_SHARED lowers it)
uint32_t shared_slots() {
  const char *sh = getenv("LEC_ES_JIT_HOIST_SHARED");
  return std::min<uint32_t>(sh ? (uint32_t)std::max(0, atoi(sh)) : kHoistShared, kHoistShared);
}

std::string gen_ptx_lut(const Program &g, int major, int minor, uint32_t REP, uint32_t reg_budget,
                        uint32_t plan_budget, uint64_t pass_pis, const std::vector<uint64_t> &groups,
                        SlotSplit *split = nullptr, double *lop3_per_pass = nullptr,
                        std::vector<uint64_t> *dump_clear = nullptr, uint32_t copies_cap = 0);

// Passes per grab (a power of two), the hoisting budget and the pass PIs of
// a table-form kernel.  Long grabs amortise hoisted tables (and the
// counter's atomic): 16 to 32 passes, at least ~4k instructions per grab; but
// a small pattern space keeps enough grabs to fill the GPU, which wins over
// both.  The pass PIs are the support PIs (index >= 10) the fewest tables
// depend on, so the most tables are the same in every pass of a grab.  The
// passes run as nested loops over groups of pass PIs when that saves enough
// table evaluations (choose_pass_groups), with up to two more pass PIs, and
// large cones then pick among candidate layouts by dry runs of the generator.
// LEC_ES_JIT_REP / LEC_ES_JIT_HOIST override passes and budget,
// LEC_ES_JIT_LOWPASS=1 takes PIs 10, 11, ... as the pass PIs,
// LEC_ES_JIT_NEST=0 keeps one pass loop, =2 nests whenever there are two
// pass PIs or more, =3 gives every pass PI its own loop, and
// LEC_ES_JIT_GROUPS gives the loops explicitly (for measurements and tests).
void jit_layout(const Program &g, GrabLayout *out) {
  uint64_t *const pass_pis = &out->pass_pis;
  std::vector<uint64_t> *const groups = &out->groups;
  const uint32_t per = g.lut.count + 40;
  uint32_t r = 16;
  while (r < 32 && r * per < 4096) r <<= 1;
  const uint64_t chunks = num_chunks(g.n);
  while (r > 1 && chunks / (32ull * r) < kGrabsWanted) r >>= 1;
  // LEC_ES_JIT_HOIST=h: at most h values in registers, the plan h plus the
  // shared-memory slots
  uint32_t regs = 255, plan = kHoistPlan;
  if (const char *e = getenv("LEC_ES_JIT_REP")) r = (uint32_t)std::max(1, atoi(e));
  if (const char *e = getenv("LEC_ES_JIT_HOIST")) {
    regs = (uint32_t)std::max(0, atoi(e));
    plan = regs + shared_slots();
  }
  uint32_t npass = 0;
  while ((1u << (npass + 1)) <= r && npass < 10) npass++;
  npass = std::min<uint32_t>(npass, g.n > 10 ? g.n - 10 : 0);  // pass PIs are support PIs 10..n-1
  uint64_t m = 0;
  if (getenv("LEC_ES_JIT_LOWPASS")) {
    for (uint32_t k = 10; k < 10 + npass; k++) m |= 1ull << k;
  } else {
    m = least_influential_pis(g.lut, npass);
  }
  const char *nest = getenv("LEC_ES_JIT_NEST");
  const int nest_mode = nest ? atoi(nest) : 1;
  double score = 0;
  *groups = choose_pass_groups(g.lut, m, nest_mode, &score);
  // With nested loops, a pass PI in a loop of its own outside the others
  // never makes a table run more often and halves the grab-level tables
  // that do not read it: add up to two more pass PIs (six at most), each
  // the best of the next six least influential, while table evaluations
  // per pass fall by 2% and enough grabs remain.
  if (nest_mode != 0 && !getenv("LEC_ES_JIT_REP") && !getenv("LEC_ES_JIT_LOWPASS")) {
    for (uint32_t k = npass + 1; k <= npass + 2 && k <= 6 && g.n > 10 && k <= g.n - 10; k++) {
      if (chunks / (32ull << k) < kGrabsWanted) break;
      const uint64_t cand = least_influential_pis(g.lut, std::min<uint32_t>(k + 5, g.n - 10)) & ~m;
      uint64_t best_m = 0;
      double best_s = 0;
      std::vector<uint64_t> best_g;
      for (uint32_t p = 0; p < 64; p++) {
        if (!((cand >> p) & 1u)) continue;
        double sk = 0;
        std::vector<uint64_t> gk = choose_pass_groups(g.lut, m | (1ull << p), nest_mode, &sk);
        if (!best_m || sk < best_s) {
          best_m = m | (1ull << p);
          best_s = sk;
          best_g = std::move(gk);
        }
      }
      if (!best_m || best_s / (double)(1u << k) >= 0.98 * score / (double)(1u << npass)) break;
      npass = k;
      m = best_m;
      score = best_s;
      *groups = std::move(best_g);
    }
  }
  // Large cones: rank candidate layouts by the lop3 the generated kernel
  // executes per pass (a dry run of the generator, no compile), since the
  // evaluation count above ignores the hoisting limits and the folding in
  // unrolled levels.  Candidates: the layout above; its pass PIs, and those
  // plus each of the next four least influential, with the m = 1, 2 most
  // influential in the outermost loop and the others a level each, least
  // influential (or highest PI) innermost (on the 16x16 miter b10, b11 |
  // b12 | b13 | b14 | b15: 454 lop3 per pass against 471, 3.35 against 3.49
  // ms).
  if (nest_mode == 1 && g.lut.count >= kParallelChainTables && !g.lut.order.empty() && !getenv("LEC_ES_JIT_REP") &&
      !getenv("LEC_ES_JIT_LOWPASS") && !getenv("LEC_ES_JIT_GROUPS") && npass >= 2) {
    const std::vector<uint64_t> dep = table_support(g.lut);
    auto influence = [&](uint32_t p) {
      uint64_t c = 0;
      for (uint64_t d : dep) c += (d >> p) & 1u;
      return c;
    };
    struct Cand {
      uint32_t npass;
      uint64_t m;
      std::vector<uint64_t> groups;
    };
    std::vector<Cand> cands{{npass, m, *groups}};
    auto patterns = [&](uint32_t k, uint64_t mk) {  // most influential m in the outer loop, then one each
      std::vector<uint32_t> ps;
      for (uint32_t p = 0; p < 64; p++)
        if ((mk >> p) & 1u) ps.push_back(p);
      std::stable_sort(ps.begin(), ps.end(), [&](uint32_t a, uint32_t b) { return influence(a) > influence(b); });
      for (uint32_t mo = 1; mo <= 2 && mo < ps.size(); mo++)
        for (int by_index = 0; by_index < 2; by_index++) {  // the single levels by influence or by PI index
          std::vector<uint32_t> rest(ps.begin() + mo, ps.end());
          if (by_index) std::sort(rest.begin(), rest.end());
          std::vector<uint64_t> gs(1, 0);
          for (uint32_t i = 0; i < mo; i++) gs[0] |= 1ull << ps[i];
          for (uint32_t q : rest) gs.push_back(1ull << q);
          cands.push_back({k, mk, gs});
        }
    };
    patterns(npass, m);
    // one more pass PI: each of the next four least influential
    const uint32_t k1 = npass + 1;
    if (k1 <= 6 && g.n > 10 && k1 <= g.n - 10 && chunks / (32ull << k1) >= kGrabsWanted) {
      const uint64_t more = least_influential_pis(g.lut, std::min<uint32_t>(npass + 4, g.n - 10)) & ~m;
      for (uint32_t p = 0; p < 64; p++)
        if ((more >> p) & 1u) patterns(k1, m | (1ull << p));
    }
    // compared at a plan of kDryPlan values kept across loops, about where
    // large cones end after spill retries, so that a layout good only with
    // more of them does not win
    std::vector<double> per(cands.size(), 0.0);
    {  // independent dry runs, on host threads
      std::mutex mu;
      size_t next = 0;
      auto work = [&]() {
        for (;;) {
          size_t i;
          {
            std::lock_guard<std::mutex> lk(mu);
            if (next >= cands.size()) return;
            i = next++;
          }
          gen_ptx_lut(g, 10, 3, 1u << cands[i].npass, regs, std::min(plan, kDryPlan), cands[i].m, cands[i].groups,
                      nullptr, &per[i]);
        }
      };
      const unsigned nt = (unsigned)std::min<size_t>(cands.size(), std::max(1u, std::thread::hardware_concurrency()));
      std::vector<std::thread> pool;
      for (unsigned t = 1; t < nt; t++) pool.emplace_back(work);
      work();
      for (auto &t : pool) t.join();
    }
    size_t bi = 0;
    for (size_t i = 1; i < cands.size(); i++)
      if (per[i] < per[bi]) bi = i;
    npass = cands[bi].npass;
    m = cands[bi].m;
    *groups = cands[bi].groups;
  }
  // LEC_ES_JIT_GROUPS="27,28|29|30|31": the pass loops given explicitly,
  // outermost first, as support PI indices (for measurements)
  if (const char *e = getenv("LEC_ES_JIT_GROUPS")) {
    std::vector<uint64_t> gs(1, 0);
    uint64_t all = 0;
    for (const char *q = e; *q;) {
      if (*q == '|') {
        gs.push_back(0);
        q++;
      } else if (*q >= '0' && *q <= '9') {
        char *endp = nullptr;
        const unsigned long k = strtoul(q, &endp, 10);
        if (k >= 10 && k < g.n && k < 64) {
          gs.back() |= 1ull << k;
          all |= 1ull << k;
        }
        q = endp;
      } else {
        q++;
      }
    }
    gs.erase(std::remove(gs.begin(), gs.end(), 0ull), gs.end());
    if (!gs.empty()) {
      npass = (uint32_t)__builtin_popcountll(all);
      m = all;
      *groups = gs;
    }
  }
  out->rep = 1u << npass;
  out->regs = regs;
  out->plan = plan;
  *pass_pis = m;
}

// 3-input truth tables (bit m = f(x0 = m&1, x1 = m>>1&1, x2 = m>>2&1)):
// input k complemented, fixed to b, or made equal to input a.
uint8_t tt_flip(uint8_t tt, int k) {
  uint8_t r = 0;
  for (int m = 0; m < 8; m++) r |= (uint8_t)(((tt >> (m ^ (1 << k))) & 1) << m);
  return r;
}
uint8_t tt_fix(uint8_t tt, int k, int b) {
  uint8_t r = 0;
  for (int m = 0; m < 8; m++) r |= (uint8_t)(((tt >> ((m & ~(1 << k)) | (b << k))) & 1) << m);
  return r;
}
uint8_t tt_same(uint8_t tt, int a, int k) {  // x_k := x_a
  uint8_t r = 0;
  for (int m = 0; m < 8; m++) r |= (uint8_t)(((tt >> ((m & ~(1 << k)) | (((m >> a) & 1) << k))) & 1) << m);
  return r;
}
bool tt_reads(uint8_t tt, int k) { return tt_flip(tt, k) != tt; }
constexpr uint8_t kVarTT[3] = {0xAA, 0xCC, 0xF0};

// Whether a kernel of n support PIs and rep passes per grab carries the
// static-stride grab code (see kStrideMaxGrabs).
bool jit_stride_ok(uint32_t n, uint32_t rep) {
  return num_chunks(n) / (32ull * std::max<uint32_t>(1, rep)) + 1 <= kStrideMaxGrabs;
}

// Runs of consecutive chunk-index bits: (first bit, source bit, length).
struct BitRun {
  uint32_t at, from, len;
};
std::vector<BitRun> bit_runs(const std::vector<uint32_t> &pos) {  // pos ascending
  std::vector<BitRun> r;
  for (uint32_t i = 0; i < pos.size(); i++) {
    if (!r.empty() && r.back().at + r.back().len == pos[i]) r.back().len++;
    else r.push_back({pos[i], i, 1});
  }
  return r;
}

// PTX of the table form, written directly (no C++ front end), with virtual
// registers left to ptxas; constants (PI masks 0..4, folded tables) are
// immediate operands.
//
// Chunk index bits: 0..4 are the lane (support PIs 5..9, fixed per thread);
// the bits of the pass PIs (k - 5 for PI k) change from pass to pass; the
// others belong to the grab.  Grab q (handed out by a counter, one ahead,
// from [q0, qend), computed on the host) is every chunk whose grab bits spell
// q, REP passes of 32 chunks, masked to [cb, ce).  Tables chosen by
// plan_hoist (no pass PI among their inputs) are evaluated once per grab,
// the others once per pass.  Grabs increase in chunk index, so a warp stops
// at the end of its range or when its grab's lowest pattern is not below
// the current counterexample; it also stops after max_grabs grabs.  Within
// a grab the counterexample (in %d12 as the first chunk it rules out) is
// re-polled at each iteration of the innermost loop, and a loop iteration,
// unrolled copy or pass that starts at or above it is skipped: every chunk
// of it is higher, so none can be the lowest failing one.  Branches whose
// predicate depends only on warp-uniform values (grab, loop, range and skip
// tests) are emitted as bra.uni; the lane-dependent ones (which lane
// reports a failure) stay bra.
//
// Dump variant (dump_clear non-null; a diagnostic, never cached): the same
// kernel with one extra parameter, a buffer of 32-bit values, row i for
// table lp.order[i] with stride 2^max(n-5, 5) chunks.  Every table's value
// is stored where this layout computes it -- once per grab, per loop
// iteration, per unrolled copy or per pass -- at the chunk index of that
// site plus the lane (the chunk bits of deeper pass PIs zero); constant
// tables are stored at grab level.  (*dump_clear)[i] receives those cleared
// chunk bits, so table i's value at chunk c is row i at c & ~clear.  The
// dump variant reports no counterexample (its cex word stays "none"), so no
// early exit skips a site.
std::string gen_ptx_lut(const Program &g, int major, int minor, uint32_t REP, uint32_t reg_budget,
                        uint32_t plan_budget, uint64_t pass_pis, const std::vector<uint64_t> &groups,
                        SlotSplit *split, double *lop3_per_pass, std::vector<uint64_t> *dump_clear,
                        uint32_t copies_cap) {
  const bool dump = dump_clear != nullptr;
  const LutProgram &lp = g.lut;
  const uint32_t NA = lp.na, NP = lp.np;
  const size_t NV = NA + NP + 1;
  // pass loops, outermost first: loop l (level l + 1) runs over the PIs of grp[l]
  const std::vector<uint64_t> grp = groups.empty() ? std::vector<uint64_t>{pass_pis} : groups;
  const uint32_t L = (uint32_t)grp.size();
  const bool stride_ok = jit_stride_ok(g.n, REP);
  uint32_t roots = 0;
  const uint32_t shared_budget = shared_slots();
  // natural level of each table: its deepest pass loop (0: reads no pass PI)
  const size_t NL = lp.order.size();
  std::vector<uint8_t> natural(NL, 0);
  {
    const std::vector<uint64_t> dep = table_support(lp);
    for (size_t i = 0; i < NL; i++)
      for (uint32_t l = 0; l < L; l++)
        if (dep[i] & grp[l]) natural[i] = (uint8_t)(l + 1);
  }
  // The innermost U levels are unrolled: straight-line copies, one per value
  // of their pass PIs (at most max_copies passes and 4,096 table
  // evaluations before folding); levels 1..Lr stay loops.  A cone whose
  // tables keep many values live is register-bound: four copies measured
  // best on the 16x16 miter (live set 198; two: 3.72 ms, four: 3.48 ms,
  // eight: 4.10 ms -- a 90 KB kernel).  One with at most kFewLive live
  // values gets up to 64 (node-pair miters of 26-28 PIs, live sets 30-73:
  // four copies 0.019-0.078 ms, 8-64 copies 0.015-0.045 ms).
  // LEC_ES_JIT_UNROLL sets the most copies (0: none); a build whose
  // unrolled copies spill may cap them lower (copies_cap, see
  // compile_program_kernel).
  const uint32_t max_copies = std::min(unroll_copies(lp), copies_cap ? copies_cap : ~0u);
  uint32_t U = 0;
  {
    uint64_t copies = 1, evals = 0;
    for (uint32_t l = L; l >= 1 && max_copies > 1; l--) {
      const uint64_t c = copies << __builtin_popcountll(grp[l - 1]);
      evals += (uint64_t)std::count(natural.begin(), natural.end(), (uint8_t)l) * c;
      if (c > max_copies || evals > 4096) break;
      copies = c;
      U++;
    }
  }
  const uint32_t Lr = L - U;
  // level of each table: 0 once per grab, l <= Lr once per iteration of
  // pass loop l (tables planned there: reading no PI of a deeper loop),
  // unrolled levels at their natural level, the rest at level Lr
  std::vector<uint8_t> level(NL, (uint8_t)Lr), h, hn;
  if (Lr >= 1) {
    plan_hoist(lp, pass_pis, plan_budget, h, &roots);
    for (size_t i = 0; i < NL; i++)
      if (h[i]) level[i] = 0;
    uint64_t deeper = pass_pis;
    for (uint32_t l = 1; l < Lr; l++) {
      deeper &= ~grp[l - 1];
      plan_hoist_from(lp, deeper, plan_budget, h, hn, &roots);
      for (size_t i = 0; i < NL; i++)
        if (hn[i] && !h[i]) level[i] = (uint8_t)l;
      h.swap(hn);
    }
  }
  for (size_t i = 0; i < NL; i++)
    if (natural[i] > Lr || Lr == 0) level[i] = natural[i];
  // values read below their own level across a loop (computed above level
  // Lr): those read in the innermost loop's iterations stay in registers,
  // the others go to shared memory (thread-private slots, written where
  // they are computed, loaded in each later section before their first
  // reader there)
  std::vector<int32_t> tpos(NA, -1);
  for (size_t i = 0; i < lp.order.size(); i++) tpos[lp.order[i].node] = (int32_t)i;
  auto crosses = [&](int32_t v, uint32_t reader_level) {
    return v >= 0 && (uint32_t)v < NA && tpos[v] >= 0 && level[tpos[v]] < reader_level && level[tpos[v]] < Lr;
  };
  std::vector<uint32_t> pass_readers(lp.order.size(), 0);
  for (size_t i = 0; i < lp.order.size(); i++) {
    for (int k = 0; k < lp.order[i].n; k++)
      if (crosses(lp.order[i].leaf[k], level[i])) pass_readers[tpos[lp.order[i].leaf[k]]]++;
  }
  if (lp.root >= 0 && crosses((int32_t)lp.root, L)) pass_readers[tpos[lp.root]]++;
  // chunk-index bit positions of each pass loop's PIs and of the grab
  const uint32_t cbits = NP > 5 ? NP - 5 : 0;
  std::vector<std::vector<uint32_t>> lpos(L);
  std::vector<uint32_t> gpos;
  std::vector<int32_t> rank(64, -1);  // chunk bit -> rank among its group's bits
  for (uint32_t b = 5; b < cbits; b++) {
    std::vector<uint32_t> *to = &gpos;
    for (uint32_t l = 0; l < L; l++)
      if ((grp[l] >> (b + 5)) & 1u) to = &lpos[l];
    rank[b] = (int32_t)to->size();
    to->push_back(b);
  }
  std::vector<int8_t> isconst(NV, 0);
  std::vector<uint32_t> cval(NV, 0);
  static const uint32_t mask[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
  for (uint32_t k = 0; k < NP && k < 5; k++) {
    isconst[NA + k] = 1;
    cval[NA + k] = mask[k];
  }
  isconst[NA + NP] = 1;
  // fold tables whose leaves are all constant
  for (const auto &l : lp.order) {
    bool allc = true;
    for (int k = 0; k < l.n; k++) allc = allc && isconst[l.leaf[k]];
    if (!allc) continue;
    uint32_t x[3] = {0, 0, 0};
    for (int k = 0; k < l.n; k++) x[k] = cval[l.leaf[k]];
    uint32_t r = 0;
    for (int b = 0; b < 32; b++) {
      const int m = (int)((x[0] >> b) & 1) | (int)(((x[1] >> b) & 1) << 1) | (int)(((x[2] >> b) & 1) << 2);
      r |= (uint32_t)((l.tt >> m) & 1) << b;
    }
    isconst[l.node] = 1;
    cval[l.node] = r;
  }
  // a value in shared memory is loaded once in every run of each section
  // that reads it (runs per grab of a level-l section: 2^(PIs of loops
  // 1..l)): registers go to the values the innermost loop reads, most
  // loaded first, up to reg_budget; the others take shared-memory slots
  std::vector<double> runs(L + 1, 1.0);
  for (uint32_t l = 1; l <= L; l++) runs[l] = runs[l - 1] * (double)(1u << __builtin_popcountll(grp[l - 1]));
  std::vector<double> load_cost(lp.order.size(), 0.0);
  std::vector<uint32_t> read_at(lp.order.size(), 0);  // bit l: read by a level-l section
  {
    for (size_t i = 0; i < lp.order.size(); i++)
      for (int k = 0; k < lp.order[i].n; k++)
        if (crosses(lp.order[i].leaf[k], level[i])) read_at[tpos[lp.order[i].leaf[k]]] |= 1u << level[i];
    if (lp.root >= 0 && crosses((int32_t)lp.root, L)) read_at[tpos[lp.root]] |= 1u << L;
    for (size_t i = 0; i < lp.order.size(); i++)
      for (uint32_t l = 1; l <= L; l++)
        if ((read_at[i] >> l) & 1u) load_cost[i] += runs[l];
  }
  std::vector<int32_t> read_roots;
  for (size_t i = 0; i < lp.order.size(); i++)
    if (pass_readers[i] && !isconst[lp.order[i].node]) read_roots.push_back((int32_t)i);  // constants are immediates
  std::stable_sort(read_roots.begin(), read_roots.end(), [&](int32_t x, int32_t y) {
    return load_cost[x] > load_cost[y] || (load_cost[x] == load_cost[y] && pass_readers[x] > pass_readers[y]);
  });
  uint32_t inner = 0;  // read in the innermost loop's iterations: sorted first (their loads run most often)
  for (int32_t i : read_roots) inner += (read_at[i] >> Lr) != 0;
  const uint32_t in_regs = std::min<uint32_t>(reg_budget, inner);
  std::vector<int32_t> smem_slot(lp.order.size(), -1);
  uint32_t nsmem = 0;
  for (size_t r = in_regs; r < read_roots.size() && nsmem < shared_budget; r++) smem_slot[read_roots[r]] = (int32_t)nsmem++;
  if (split) {
    split->read = (uint32_t)read_roots.size();
    split->in_regs = (uint32_t)read_roots.size() - nsmem;
    split->in_shared = nsmem;
    split->inner_in_regs = in_regs;
  }
  std::ostringstream s;
  char buf[192];
  s << ".version 9.0\n.target sm_" << major << minor << "a\n.address_size 64\n\n";
  // more slots than a static array may hold: dynamic shared memory of
  // nsmem * kJitBlock words, sized at launch (JitKernel::dyn_smem)
  if (nsmem > kStaticShared) s << ".extern .shared .align 16 .b32 hs[];\n\n";
  s << ".visible .entry es_jit(.param .u64 p_cb, .param .u64 p_ce, .param .u64 p_cex, .param .u64 p_ev,\n"
    << "    .param .u64 p_next, .param .u64 p_maxg, .param .u64 p_rep, .param .u64 p_q0, .param .u64 p_qend"
    << (dump ? ", .param .u64 p_tt" : "") << ")\n"
    << ".maxntid " << kJitBlock << ", 1, 1\n{\n"
    << "  .reg .pred %p<16>;\n  .reg .b32 %t<26>;\n  .reg .b64 %d<40>;\n  .reg .b32 %j<" << L << ">;\n"
    << "  .reg .b64 %o<" << L << ">;\n"
    << "  .reg .b32 %v<" << (NA + 1) << ">;\n  .reg .b32 %s<" << (NA + 1) << ">;\n  .reg .b32 %q<" << (NP + 1)
    << ">;\n  .reg .b32 %po<" << kGroupPasses << ">;\n";
  if (nsmem && nsmem <= kStaticShared) s << "  .shared .align 16 .b32 hs[" << nsmem * kJitBlock << "];\n";
  if (dump) s << "  .reg .b32 %z<2>;\n  ld.param.u64 %d38, [p_tt];\n  cvta.to.global.u64 %d38, %d38;\n";
  // parameters; grab range [d8, d9); lane; first grab; first counterexample poll
  s << "  ld.param.u64 %d1, [p_cb];\n  ld.param.u64 %d2, [p_ce];\n  ld.param.u64 %d3, [p_cex];\n"
       "  ld.param.u64 %d4, [p_ev];\n  ld.param.u64 %d5, [p_next];\n  ld.param.u64 %d6, [p_maxg];\n"
       "  ld.param.u64 %d8, [p_q0];\n  ld.param.u64 %d9, [p_qend];\n"
       << (stride_ok ? "  setp.eq.u64 %p14, %d5, 0;\n" : "")
    << "  cvta.to.global.u64 %d3, %d3;\n  cvta.to.global.u64 %d4, %d4;\n  cvta.to.global.u64 %d5, %d5;\n"
       "  mov.u32 %t1, %tid.x;\n  and.b32 %t2, %t1, 31;\n  setp.eq.u32 %p1, %t2, 0;\n";
  if (stride_ok) {
    // p14: no grab counter -- warp w takes grabs w, w + W, w + 2W, ... (W
    // warps in the grid); else lane 0 (p15) takes them from the counter
    s << "  not.pred %p15, %p14;\n  and.pred %p15, %p15, %p1;\n"
         "  mov.u32 %t17, %ctaid.x;\n  mov.u32 %t18, %nctaid.x;\n  shr.u32 %t19, %t1, 5;\n"
         "  mul.wide.u32 %d35, %t17, "
      << (kJitBlock / 32) << ";\n  cvt.u64.u32 %d37, %t19;\n  add.u64 %d35, %d35, %d37;\n"
      << "  mul.wide.u32 %d36, %t18, " << (kJitBlock / 32) << ";\n";
  } else {
    s << "  mov.pred %p15, %p1;\n";
  }
  s << "  mov.u64 %d10, 0;\n  mov.u64 %d11, 0;\n  @%p15 atom.global.add.u64 %d11, [%d5], 1;\n"
       "  mov.b64 {%t3, %t4}, %d11;\n  shfl.sync.idx.b32 %t3, %t3, 0, 31, -1;\n"
       "  shfl.sync.idx.b32 %t4, %t4, 0, 31, -1;\n  mov.b64 %d11, {%t3, %t4};\n"
    << (stride_ok ? "  @%p14 mov.u64 %d11, %d35;\n" : "")
    << "  mov.u64 %d12, 0;\n  @%p1 ld.volatile.global.u64 %d12, [%d3];\n  mov.b64 {%t3, %t4}, %d12;\n"
       "  shfl.sync.idx.b32 %t3, %t3, 0, 31, -1;\n  shfl.sync.idx.b32 %t4, %t4, 0, 31, -1;\n"
       "  mov.b64 %d12, {%t3, %t4};\n"
    << kCexToChunk << "  mov.u64 %d13, 1;\n  cvt.u64.u32 %d18, %t2;\n";
  if (nsmem) s << "  mov.u32 %t21, hs;\n  shl.b32 %t22, %t1, 2;\n  add.u32 %t21, %t21, %t22;\n";
  // constants (PI masks, the constant, folded tables) are lop3 immediates
  std::vector<std::string> name(NV);
  for (size_t v = 0; v < NV; v++) {
    if (!isconst[v]) continue;
    snprintf(buf, sizeof(buf), "0x%08x", cval[v]);
    name[v] = buf;
  }
  for (uint32_t k = 5; k < NP; k++) name[NA + k] = "%q" + std::to_string(k);
  // which PIs are read at all
  std::vector<uint8_t> pi_used(NP, 0);
  for (const auto &l : lp.order) {
    if (isconst[l.node]) continue;
    for (int k = 0; k < l.n; k++)
      if (l.leaf[k] >= (int32_t)NA && l.leaf[k] < (int32_t)(NA + NP)) pi_used[l.leaf[k] - NA] = 1;
  }
  if (lp.root >= (int64_t)NA && lp.root < (int64_t)(NA + NP)) pi_used[lp.root - NA] = 1;
  // PIs 5..9: bits 0..4 of the chunk index are the lane
  for (uint32_t k = 5; k < NP && k < 10; k++) {
    snprintf(buf, sizeof(buf), "  bfe.s32 %%q%u, %%t2, %u, 1;\n", k, k - 5);
    if (pi_used[k]) s << buf;
  }
  auto emit_table = [&](const LutCover::Lut &l) {
    name[l.node] = "%v" + std::to_string(l.node);
    auto op = [&](int32_t id) -> std::string { return id < 0 ? std::string("0") : name[id]; };
    const std::string x0 = op(l.leaf[0]), x1 = op(l.n > 1 ? l.leaf[1] : -1), x2 = op(l.n > 2 ? l.leaf[2] : -1);
    // lop3 operands a, b, c carry the patterns 0xF0, 0xCC, 0xAA: (x2, x1, x0)
    snprintf(buf, sizeof(buf), "  lop3.b32 %s, %s, %s, %s, 0x%02x;\n", name[l.node].c_str(), x2.c_str(), x1.c_str(),
             x0.c_str(), l.tt);
    s << buf;
  };
  // dump variant: store table i's value (a register, its complement, or an
  // immediate) at row i, chunk site + off + lane; clear(lv) = chunk bits of
  // the pass PIs of levels deeper than lv
  const uint64_t dump_stride = 1ull << std::max<uint32_t>(g.n > 5 ? g.n - 5 : 0, 5);
  if (dump) dump_clear->assign(NL, 0);
  auto clear_below = [&](uint32_t lv) {
    uint64_t m = 0;
    for (uint32_t l = lv; l < L; l++) m |= grp[l];
    return m >> 5;
  };
  auto dump_store = [&](size_t i, const std::string &site, uint64_t off, const std::string &val, bool imm, bool inv,
                        uint32_t lv) {
    if (!dump) return;
    (*dump_clear)[i] = clear_below(lv);
    snprintf(buf, sizeof(buf),
             "  add.u64 %%d39, %s, %llu;\n  add.u64 %%d39, %%d39, %%d18;\n  shl.b64 %%d39, %%d39, 2;\n"
             "  add.u64 %%d39, %%d39, %%d38;\n",
             site.c_str(), (unsigned long long)(i * dump_stride + off));
    s << buf;
    if (imm) s << "  mov.b32 %z0, " << val << ";\n";
    else if (inv) s << "  not.b32 %z0, " << val << ";\n";
    s << "  st.global.b32 [%d39], " << (imm || inv ? std::string("%z0") : val) << ";\n";
  };
  // scatter the bits of a 64-bit source register into chunk positions (runs
  // of consecutive positions): dst = sum over runs of field << position
  auto emit_deposit = [&](const char *dst, const char *src, const std::vector<uint32_t> &pos) {
    s << "  mov.u64 " << dst << ", 0;\n";
    for (const BitRun &r : bit_runs(pos)) {
      snprintf(buf, sizeof(buf),
               "  shr.u64 %%d30, %s, %u;\n  and.b64 %%d30, %%d30, 0x%016llx;\n  shl.b64 %%d30, %%d30, %u;\n"
               "  or.b64 %s, %s, %%d30;\n",
               src, r.from, (unsigned long long)((r.len >= 64 ? 0ull : (1ull << r.len)) - 1ull), r.at, dst, dst);
      s << buf;
    }
  };
  // grab loop: d14 grab number, d15 its lowest chunk (the grab bits of q)
  s << "$LOOP:\n"
       "  add.u64 %d14, %d8, %d11;\n  setp.ge.u64 %p2, %d14, %d9;\n  @%p2 bra.uni $DONE;\n";
  emit_deposit("%d15", "%d14", gpos);
  s << "  max.u64 %d20, %d15, %d1;\n  setp.ge.u64 %p2, %d20, %d12;\n  @%p2 bra.uni $DONE;\n"
       "  setp.lt.u64 %p3, %d13, %d6;\n  and.pred %p4, %p15, %p3;\n  mov.u64 %d16, -1;\n"
       "  @%p4 atom.global.add.u64 %d16, [%d5], 1;\n" << (stride_ok ? "  @%p14 add.u64 %d16, %d11, %d36;\n" : "")
    << "  mov.u64 %d17, 0;\n"
       "  @%p1 ld.volatile.global.u64 %d17, [%d3];\n"
       "  cvt.u32.u64 %t5, %d14;\n  shr.u64 %d20, %d14, 32;\n  cvt.u32.u64 %t6, %d20;\n";
  // p12: every chunk of the grab lies in [cb, ce) -- its passes then skip
  // all range work and it counts its chunks at the end
  uint64_t span = 32;
  for (const auto &ps : lpos)
    for (uint32_t b : ps) span += 1ull << b;
  snprintf(buf, sizeof(buf),
           "  add.u64 %%d34, %%d15, %llu;\n  setp.le.u64 %%p13, %%d34, %%d2;\n  setp.ge.u64 %%p12, %%d15, %%d1;\n"
           "  and.pred %%p12, %%p12, %%p13;\n",
           (unsigned long long)span);
  s << buf;
  // the grab's PIs (bit rank of q), then the hoisted tables
  for (uint32_t k = 10; k < NP; k++) {
    if (!pi_used[k] || ((pass_pis >> k) & 1u)) continue;
    const int32_t j = rank[k - 5];
    snprintf(buf, sizeof(buf), "  bfe.s32 %%q%u, %%t%d, %d, 1;\n", k, j < 32 ? 5 : 6, j < 32 ? j : j - 32);
    s << buf;
  }
  // a shared-memory value is loaded in each section before its first
  // reader there
  std::vector<uint8_t> loaded(NA, 0);
  auto load_shared = [&](int32_t v, uint8_t lv) {  // lv: the reading section's level
    if (v < 0 || (uint32_t)v >= NA || tpos[v] < 0 || smem_slot[tpos[v]] < 0 || loaded[v] || level[tpos[v]] >= lv)
      return;
    snprintf(buf, sizeof(buf), "  ld.shared.b32 %%s%d, [%%t21+%u];\n", v, (uint32_t)smem_slot[tpos[v]] * kJitBlock * 4u);
    s << buf;
    name[v] = "%s" + std::to_string(v);
    loaded[v] = 1;
  };
  // pass loops 1..NLOOP ($LV, index j<l>, first chunk of the iteration
  // o<l>); without unrolling the innermost level L is the pass loop ($PASS)
  const uint32_t NLOOP = U > 0 ? Lr : L - 1;
  std::string stubs;  // out-of-line skip paths, emitted after the kernel's ret
  auto emit_level = [&](uint8_t lv) {
    std::fill(loaded.begin(), loaded.end(), (uint8_t)0);
    const std::string site = lv == 0 ? std::string("%d15") : lv <= NLOOP ? "%o" + std::to_string(lv) : "%d27";
    for (size_t i = 0; i < lp.order.size(); i++) {
      if (level[i] != lv || isconst[lp.order[i].node]) continue;
      for (int k = 0; k < lp.order[i].n; k++) load_shared(lp.order[i].leaf[k], lv);
      emit_table(lp.order[i]);
      dump_store(i, site, 0, name[lp.order[i].node], false, false, lv);
      if (smem_slot[i] >= 0) {
        snprintf(buf, sizeof(buf), "  st.shared.b32 [%%t21+%u], %%v%d;\n", (uint32_t)smem_slot[i] * kJitBlock * 4u,
                 lp.order[i].node);
        s << buf;
      }
    }
  };
  auto close_loops = [&]() {  // loop ends of the outer pass loops, innermost first
    std::string c;
    for (uint32_t l = NLOOP; l >= 1; l--) {
      const std::string j = "%j" + std::to_string(l);
      c += "$LE" + std::to_string(l) + ":\n  add.u32 " + j + ", " + j + ", 1;\n  setp.lt.u32 %p9, " + j + ", " +
           std::to_string(1u << __builtin_popcountll(grp[l - 1])) + ";\n  @%p9 bra.uni $LV" + std::to_string(l) + ";\n";
    }
    return c;
  };
  auto emit_pass_pis = [&](uint64_t group, const char *idx) {
    for (uint32_t k = 10; k < NP; k++) {
      if (!pi_used[k] || !((group >> k) & 1u)) continue;
      snprintf(buf, sizeof(buf), "  bfe.s32 %%q%u, %s, %d, 1;\n", k, idx, rank[k - 5]);
      s << buf;
    }
  };
  emit_level(0);
  if (dump)
    for (size_t i = 0; i < lp.order.size(); i++)
      if (isconst[lp.order[i].node]) {
        snprintf(buf, sizeof(buf), "0x%08x", cval[lp.order[i].node]);
        dump_store(i, "%d15", 0, buf, true, false, 0);
      }
  for (uint32_t l = 1; l <= NLOOP; l++) {
    const std::string j = "%j" + std::to_string(l);
    s << "  mov.u32 " << j << ", 0;\n$LV" << l << ":\n  cvt.u64.u32 %d32, " << j << ";\n";
    emit_deposit("%d28", "%d32", lpos[l - 1]);
    s << "  add.u64 %o" << l << ", " << (l == 1 ? std::string("%d15") : "%o" + std::to_string(l - 1)) << ", %d28;\n";
    if (l == NLOOP) s << kCexRefresh;
    // an iteration whose first chunk is not below the counterexample is
    // skipped, and so are the later ones (they start higher)
    s << "  setp.ge.u64 %p9, %o" << l << ", %d12;\n  @%p9 bra.uni $SKL" << l << ";\n";
    stubs += "$SKL" + std::to_string(l) + ":\n  @%p12 sub.u64 %d10, %d10, " +
             std::to_string((uint64_t)REP / (uint64_t)runs[l]) + ";\n  bra.uni $LE" + std::to_string(l) + ";\n";
    emit_pass_pis(grp[l - 1], j.c_str());
    emit_level((uint8_t)l);
  }
  const std::string base = NLOOP == 0 ? std::string("%d15") : "%o" + std::to_string(NLOOP);
  // passes: j in t20, its chunk bits in d29, the pass's first chunk d27;
  // outer passes do not run in chunk order, so a pass past the range is
  // skipped rather than ending the grab
  // this lane's chunk of the pass in d19 (first chunk of the pass in d27)
  auto emit_chunk = [&]() {
    s << "  cvt.u64.u32 %d31, %t20;\n";
    emit_deposit("%d29", "%d31", lpos[L - 1]);
    s << "  add.u64 %d27, " << base << ", %d29;\n";
  };
  const uint32_t vmask = g.n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << g.n)) - 1u);
  uint64_t unrolled_lop3 = 0;  // lop3 of the unrolled levels (one run of level Lr)
  if (U > 0) {
    // Levels Lr+1..L unrolled: nested straight-line copies, one per value of
    // each level's pass PIs, in which those PIs are the constants 0 or
    // all-ones.  Through each copy they propagate: a table reading one is
    // cofactored, complements fold into the readers' tables, a table left
    // with one input becomes an alias and one left with none a constant --
    // the same Boolean functions with fewer instructions.  The innermost
    // copies are the passes.
    struct SVal {
      bool imm = false;  // an immediate (imm_v) or a register (reg, complemented if inv)
      bool inv = false;
      uint32_t imm_v = 0;
      std::string reg;
    };
    std::vector<SVal> sv(NV);
    std::vector<int8_t> pic(NP, -1);  // pass PIs fixed in the current copy: 0 or 1
    uint32_t ncopy = 0;                // pass copies emitted (label numbers)
    uint32_t nouter = 0;               // checked copies of outer unrolled levels (label numbers)
    unrolled_lop3 = 0;
    // Pass groups (a cone with few live values, not the dump): the passes
    // under one copy of level Lg -- at most kGroupPasses -- are one
    // straight-line block, with no skip check or output branch between them
    // (so their independent table chains interleave): each pass's output is
    // kept in %po<k>, and one check after the group looks at them (pass by
    // pass only in a partial grab, or when one of them fails).  The group is
    // skipped or run as a whole.
    uint32_t Lg = L + 1;  // L + 1: no groups
    if (!dump && lp.live <= kFewLive)
      for (uint32_t lv = Lr + 1; lv <= L && Lg == L + 1; lv++) {
        uint64_t per = 1, evals = 0;  // passes and table evaluations in one group
        for (uint32_t l2 = lv; l2 <= L; l2++) {
          per <<= __builtin_popcountll(grp[l2 - 1]);
          evals += (uint64_t)std::count(level.begin(), level.end(), (uint8_t)l2) * per;
        }
        if (per >= 2 && per <= kGroupPasses && evals <= kGroupEvals) Lg = lv;
      }
    struct GroupPass {
      uint64_t o;   // chunk offset of the pass
      bool never;   // its output folds to 0
    };
    if (split) split->grouped = Lg <= L;
    std::vector<GroupPass> gp;  // passes of the open group
    bool in_group = false;
    uint32_t ngroup = 0;
    const uint32_t vmask_g = g.n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << g.n)) - 1u);
    auto flush_group = [&]() {
      const std::string G = std::to_string(ngroup++);
      // a partial grab: lanes outside [cb, ce) neither fail nor count
      s << "  @%p12 bra.uni $GF" << G << ";\n";
      for (size_t k = 0; k < gp.size(); k++) {
        const std::string P = "%po" + std::to_string(k);
        s << "  add.u64 %d27, " << base << ", " << gp[k].o << ";\n  add.u64 %d19, %d27, %d18;\n"
          << "  setp.ge.u64 %p5, %d19, %d2;\n  setp.lt.u64 %p11, %d19, %d1;\n  or.pred %p5, %p5, %p11;\n"
          << "  @%p5 mov.b32 " << P << ", 0;\n  selp.u64 %d24, 0, 1, %p5;\n  add.u64 %d10, %d10, %d24;\n";
      }
      s << "$GF" << G << ":\n  mov.b32 %t7, 0;\n";
      for (size_t k = 0; k < gp.size(); k++)
        if (!gp[k].never) s << "  or.b32 %t7, %t7, %po" << k << ";\n";
      s << "  setp.ne.u32 %p6, %t7, 0;\n  vote.sync.any.pred %p7, %p6, -1;\n  @!%p7 bra.uni $GE" << G << ";\n";
      for (size_t k = 0; k < gp.size(); k++) {  // a failure (rare): each pass's lowest failing lane
        if (gp[k].never) continue;
        const std::string P = "%po" + std::to_string(k), N = "$GN" + G + "_" + std::to_string(k);
        s << "  setp.ne.u32 %p6, " << P << ", 0;\n  vote.sync.ballot.b32 %t8, %p6, -1;\n  setp.eq.u32 %p7, %t8, 0;\n"
          << "  @%p7 bra " << N << ";\n  neg.s32 %t9, %t8;\n  and.b32 %t9, %t9, %t8;\n  bfind.u32 %t10, %t9;\n"
          << "  setp.ne.u32 %p7, %t10, %t2;\n  @%p7 bra " << N << ";\n"
          << "  add.u64 %d27, " << base << ", " << gp[k].o << ";\n  add.u64 %d19, %d27, %d18;\n"
          << "  neg.s32 %t11, " << P << ";\n  and.b32 %t11, %t11, " << P << ";\n  bfind.u32 %t12, %t11;\n"
          << "  cvt.u64.u32 %d21, %t12;\n  shl.b64 %d22, %d19, 5;\n  add.u64 %d22, %d22, %d21;\n"
          << "  atom.global.min.u64 %d23, [%d3], %d22;\n" << N << ":\n";
      }
      s << "$GE" << G << ":\n";
      gp.clear();
    };
    auto value = [&](int32_t v, uint8_t lv) -> SVal {  // a leaf's value in the current copy
      SVal x;
      if (v < 0 || isconst[v]) {
        x.imm = true;
        x.imm_v = v < 0 ? 0u : cval[v];
        return x;
      }
      if ((uint32_t)v >= NA) {
        const uint32_t k = (uint32_t)v - NA;
        if (k < NP && pic[k] >= 0) {
          x.imm = true;
          x.imm_v = pic[k] ? 0xFFFFFFFFu : 0u;
          return x;
        }
        x.reg = name[v];
        return x;
      }
      if (tpos[v] >= 0 && level[tpos[v]] > Lr) return sv[v];
      load_shared(v, lv);
      x.reg = name[v];
      return x;
    };
    auto emit_spec = [&](const LutCover::Lut &l, uint8_t lv) {
      SVal op[3];
      bool live[3] = {false, false, false};
      uint8_t tt = l.tt;
      for (int k = 0; k < 3; k++) {
        op[k] = value(k < l.n ? l.leaf[k] : -1, lv);
        live[k] = true;
        if (!op[k].imm && op[k].inv) tt = tt_flip(tt, k);
        if (op[k].imm && (op[k].imm_v == 0u || op[k].imm_v == 0xFFFFFFFFu)) {
          tt = tt_fix(tt, k, op[k].imm_v != 0);
          live[k] = false;
        }
      }
      for (int a = 0; a < 3; a++)
        for (int k = a + 1; k < 3; k++)
          if (live[a] && live[k] && op[a].imm == op[k].imm &&
              (op[a].imm ? op[a].imm_v == op[k].imm_v : op[a].reg == op[k].reg)) {
            tt = tt_same(tt, a, k);
            live[k] = false;
          }
      int nlive = 0, nreg = 0, last = -1;
      for (int k = 0; k < 3; k++) {
        live[k] = live[k] && tt_reads(tt, k);
        if (live[k]) {
          nlive++;
          nreg += !op[k].imm;
          last = k;
        }
      }
      SVal res;
      if (nreg == 0) {  // every input a constant: evaluate bitwise
        res.imm = true;
        for (int b = 0; b < 32; b++) {
          int m = 0;
          for (int k = 0; k < 3; k++)
            if (live[k]) m |= (int)((op[k].imm_v >> b) & 1u) << k;
          res.imm_v |= (uint32_t)((tt >> m) & 1) << b;
        }
      } else if (nlive == 1 && (tt == kVarTT[last] || tt == (uint8_t)~kVarTT[last])) {
        res.reg = op[last].reg;  // an alias of its input, or of its complement
        res.inv = tt != kVarTT[last];
      } else {
        res.reg = "%v" + std::to_string(l.node);
        std::string x[3];
        for (int k = 0; k < 3; k++) {
          if (!live[k]) {
            x[k] = "0";
          } else if (op[k].imm) {
            snprintf(buf, sizeof(buf), "0x%08x", op[k].imm_v);
            x[k] = buf;
          } else {
            x[k] = op[k].reg;
          }
        }
        unrolled_lop3++;
        snprintf(buf, sizeof(buf), "  lop3.b32 %s, %s, %s, %s, 0x%02x;\n", res.reg.c_str(), x[2].c_str(), x[1].c_str(),
                 x[0].c_str(), tt);
        s << buf;
      }
      sv[l.node] = res;
    };
    auto dump_spec = [&](size_t i, uint64_t o, uint32_t lv) {  // a copy's value of table i (dump variant)
      const SVal &r = sv[lp.order[i].node];
      char imm[16];
      snprintf(imm, sizeof(imm), "0x%08x", r.imm_v);
      dump_store(i, base, o, r.imm ? std::string(imm) : r.reg, r.imm, r.inv, lv);
    };
    auto unrolled = [&](auto &&self, uint32_t lv, uint64_t off) -> void {
      const bool opens = lv == Lg && !in_group;
      if (opens) in_group = true;
      std::vector<uint32_t> pis;  // this level's pass PIs in rank order (ascending)
      for (uint32_t k = 10; k < NP; k++)
        if ((grp[lv - 1] >> k) & 1u) pis.push_back(k);
      for (uint32_t j = 0; j < (1u << pis.size()); j++) {
        uint64_t o = off;  // chunk offset of this copy
        for (uint32_t r = 0; r < pis.size(); r++) {
          if ((j >> r) & 1u) o |= 1ull << lpos[lv - 1][r];
          pic[pis[r]] = (int8_t)((j >> r) & 1u);
        }
        const std::vector<SVal> saved = sv;
        if (lv < L) {
          // a copy that starts at or above the counterexample's chunk
          // (o >= %t23) skips its tables and every pass below it; the
          // first copy (o = off) starts where its parent does, checked there
          const bool chk = o != off && o <= 0xFFFFFFFEull && !in_group;
          const std::string U = std::to_string(nouter);
          if (chk) {
            nouter++;
            s << "  setp.le.u32 %p9, %t23, " << o << ";\n  @%p9 bra.uni $UK" << U << ";\n";
            stubs += "$UK" + U + ":\n  @%p12 sub.u64 %d10, %d10, " +
                     std::to_string((uint64_t)REP / (uint64_t)runs[lv]) + ";\n  bra.uni $UE" + U + ";\n";
          }
          std::fill(loaded.begin(), loaded.end(), (uint8_t)0);
          for (size_t i = 0; i < lp.order.size(); i++)
            if (level[i] == lv && !isconst[lp.order[i].node]) {
              emit_spec(lp.order[i], (uint8_t)lv);
              dump_spec(i, o, lv);
            }
          self(self, lv + 1, o);
          if (chk) s << "$UE" << U << ":\n";
        } else if (in_group) {  // a pass of a group: its tables and its output, kept in %po<k>
          ncopy++;
          std::fill(loaded.begin(), loaded.end(), (uint8_t)0);
          for (size_t i = 0; i < lp.order.size(); i++)
            if (level[i] == L && !isconst[lp.order[i].node]) emit_spec(lp.order[i], (uint8_t)L);
          const SVal out = value(lp.root < 0 ? -1 : (int32_t)lp.root, (uint8_t)L);
          const uint32_t outc = g.out_compl ? 0xFFFFFFFFu : 0u;
          const bool never = out.imm && ((out.imm_v ^ outc) & vmask_g) == 0;
          const std::string P = "%po" + std::to_string(gp.size());
          if (out.imm)
            snprintf(buf, sizeof(buf), "  mov.b32 %s, 0x%08x;\n", P.c_str(), (out.imm_v ^ outc) & vmask_g);
          else
            snprintf(buf, sizeof(buf), "  xor.b32 %s, %s, 0x%08x;\n  and.b32 %s, %s, 0x%08x;\n", P.c_str(),
                     out.reg.c_str(), out.inv ? ~outc : outc, P.c_str(), P.c_str(), vmask_g);
          s << buf;
          gp.push_back(GroupPass{o, never});
        } else {  // a pass: its range work, its tables, its output check
          const std::string J = std::to_string(ncopy++);
          const std::string chunk = "  add.u64 %d27, " + base + ", " + std::to_string(o) + ";\n";
          // a pass whose first chunk (base + o) is not below the
          // counterexample's is skipped: o >= %t23 = min(cex chunk - base,
          // 2^32 - 1); the first copy (o = off) starts where its parent
          // copy does, checked there
          const bool wide = o > 0xFFFFFFFEull;
          if (o != off) {
            if (wide) s << chunk << "  setp.ge.u64 %p9, %d27, %d12;\n";
            else s << "  setp.le.u32 %p9, %t23, " << o << ";\n";
            s << "  @%p9 bra.uni $SKP" << J << ";\n";
            stubs += "$SKP" + J + ":\n  @%p12 sub.u64 %d10, %d10, 1;\n  bra.uni $NX" + J + ";\n";
          }
          s << "  @%p12 bra.uni $PB" << J << ";\n" << (o != off && wide ? std::string() : chunk)
            << "  setp.ge.u64 %p9, %d27, %d2;\n  @%p9 bra.uni $NX" << J
            << ";\n  add.u64 %d22, %d27, 32;\n  setp.le.u64 %p10, %d22, %d1;\n  @%p10 bra.uni $NX" << J
            << ";\n  add.u64 %d19, %d27, %d18;\n$PB" << J << ":\n";
          std::fill(loaded.begin(), loaded.end(), (uint8_t)0);
          for (size_t i = 0; i < lp.order.size(); i++)
            if (level[i] == L && !isconst[lp.order[i].node]) {
              emit_spec(lp.order[i], (uint8_t)L);
              dump_spec(i, o, L);
            }
          const SVal out = value(lp.root < 0 ? -1 : (int32_t)lp.root, (uint8_t)L);
          const uint32_t outc = g.out_compl ? 0xFFFFFFFFu : 0u;
          const bool never = out.imm && ((out.imm_v ^ outc) & vmask) == 0;
          if (out.imm) {
            snprintf(buf, sizeof(buf), "  mov.b32 %%t7, 0x%08x;\n", (out.imm_v ^ outc) & vmask);
          } else {
            snprintf(buf, sizeof(buf), "  xor.b32 %%t7, %s, 0x%08x;\n  and.b32 %%t7, %%t7, 0x%08x;\n",
                     out.reg.c_str(), out.inv ? ~outc : outc, vmask);
          }
          s << buf;
          s << "  @%p12 bra $CK" << J << ";\n"
            << "  setp.ge.u64 %p5, %d19, %d2;\n  setp.lt.u64 %p11, %d19, %d1;\n  or.pred %p5, %p5, %p11;\n"
               "  @%p5 mov.b32 %t7, 0;\n  selp.u64 %d24, 0, 1, %p5;\n  add.u64 %d10, %d10, %d24;\n"
            << "$CK" << J << ":\n";
          if (!never) {  // a pass whose output is the constant 0 cannot fail
            s << "  setp.ne.u32 %p6, %t7, 0;\n  vote.sync.ballot.b32 %t8, %p6, -1;\n  setp.eq.u32 %p7, %t8, 0;\n"
              << "  @%p7 bra $NX" << J << ";\n"
              << "  neg.s32 %t9, %t8;\n  and.b32 %t9, %t9, %t8;\n  bfind.u32 %t10, %t9;\n"
              << "  setp.ne.u32 %p7, %t10, %t2;\n  @%p7 bra $NX" << J << ";\n"
              << chunk
              << "  add.u64 %d19, %d27, %d18;\n"
                 "  neg.s32 %t11, %t7;\n  and.b32 %t11, %t11, %t7;\n  bfind.u32 %t12, %t11;\n"
                 "  cvt.u64.u32 %d21, %t12;\n  shl.b64 %d22, %d19, 5;\n  add.u64 %d22, %d22, %d21;\n"
              << (dump ? "" : "  atom.global.min.u64 %d23, [%d3], %d22;\n");
          }
          s << "$NX" << J << ":\n";
        }
        sv = saved;
        for (uint32_t r = 0; r < pis.size(); r++) pic[pis[r]] = -1;
      }
      if (opens) {
        flush_group();
        in_group = false;
      }
    };
    // %t23: the counterexample's chunk minus base, at most 2^32 - 1 (base is
    // below it here: the innermost loop's iteration, or the grab, was checked)
    s << "  sub.u64 %d33, %d12, " << base << ";\n  min.u64 %d33, %d33, 4294967295;\n  cvt.u32.u64 %t23, %d33;\n";
    unrolled(unrolled, Lr + 1, 0);
  } else {
    s << "  mov.u32 %t20, 0;\n$PASS:\n";
    if (NLOOP == 0) s << kCexRefresh;
    emit_chunk();
    s << "  setp.ge.u64 %p9, %d27, %d12;\n  @%p9 bra.uni $SKPP;\n  @%p12 bra.uni $PBODY;\n";
    stubs += "$SKPP:\n  @%p12 sub.u64 %d10, %d10, 1;\n  bra.uni $NEXTPASS;\n";
    s << "  setp.ge.u64 %p9, %d27, %d2;\n  @%p9 bra.uni " << (L > 1 ? "$NEXTPASS" : "$GRABEND") << ";\n"
      << "  add.u64 %d22, %d27, 32;\n  setp.le.u64 %p10, %d22, %d1;\n  @%p10 bra.uni $NEXTPASS;\n"
         "  add.u64 %d19, %d27, %d18;\n$PBODY:\n";
    emit_pass_pis(grp[L - 1], "%t20");
    emit_level((uint8_t)L);
    if (lp.root >= 0) load_shared((int32_t)lp.root, (uint8_t)L);
    const std::string root = lp.root < 0 ? std::string("0") : name[lp.root];
    snprintf(buf, sizeof(buf), "  xor.b32 %%t7, %s, 0x%08x;\n  and.b32 %%t7, %%t7, 0x%08x;\n", root.c_str(),
             g.out_compl ? 0xFFFFFFFFu : 0u, vmask);
    s << buf;
    // in a partial grab, chunks outside [cb, ce) neither fail nor count
    s << "  @%p12 bra $CHECK;\n"
         "  setp.ge.u64 %p5, %d19, %d2;\n  setp.lt.u64 %p11, %d19, %d1;\n  or.pred %p5, %p5, %p11;\n"
         "  @%p5 mov.b32 %t7, 0;\n  selp.u64 %d24, 0, 1, %p5;\n  add.u64 %d10, %d10, %d24;\n"
         "$CHECK:\n  setp.ne.u32 %p6, %t7, 0;\n"
         "  vote.sync.ballot.b32 %t8, %p6, -1;\n  setp.eq.u32 %p7, %t8, 0;\n  @%p7 bra $NEXTPASS;\n"
         "  neg.s32 %t9, %t8;\n  and.b32 %t9, %t9, %t8;\n  bfind.u32 %t10, %t9;\n"
         "  setp.ne.u32 %p7, %t10, %t2;\n  @%p7 bra $NEXTPASS;\n";
    emit_chunk();  // a failing pass (rare) recomputes its chunk
    s << "  add.u64 %d19, %d27, %d18;\n"
         "  neg.s32 %t11, %t7;\n  and.b32 %t11, %t11, %t7;\n  bfind.u32 %t12, %t11;\n"
         "  cvt.u64.u32 %d21, %t12;\n  shl.b64 %d22, %d19, 5;\n  add.u64 %d22, %d22, %d21;\n";
    if (!dump) s << "  atom.global.min.u64 %d23, [%d3], %d22;\n";
    s << "$NEXTPASS:\n"
         "  add.u32 %t20, %t20, 1;\n  setp.lt.u32 %p9, %t20, " + std::to_string(1u << __builtin_popcountll(grp[L - 1])) + ";\n  @%p9 bra.uni $PASS;\n";
  }
  s << close_loops() + "  @%p12 add.u64 %d10, %d10, " + std::to_string(REP) + ";\n"
       "$GRABEND:\n"
       "  mov.b64 {%t3, %t4}, %d16;\n  shfl.sync.idx.b32 %t3, %t3, 0, 31, -1;\n"
       "  shfl.sync.idx.b32 %t4, %t4, 0, 31, -1;\n  mov.b64 %d11, {%t3, %t4};\n"
       "  mov.b64 {%t3, %t4}, %d17;\n  shfl.sync.idx.b32 %t3, %t3, 0, 31, -1;\n"
       "  shfl.sync.idx.b32 %t4, %t4, 0, 31, -1;\n  mov.b64 %d12, {%t3, %t4};\n" + kCexToChunk +
       "  add.u64 %d13, %d13, 1;\n  @!%p3 bra $DONE;\n  bra $LOOP;\n"
       "$DONE:\n";
  // warp sum of chunks done, then one reduction per warp
  for (int o = 16; o > 0; o >>= 1) {
    const std::string os = std::to_string(o);
    s << "  mov.b64 {%t13, %t14}, %d10;\n  shfl.sync.down.b32 %t15, %t13, " << os << ", 31, -1;\n"
      << "  shfl.sync.down.b32 %t16, %t14, " << os << ", 31, -1;\n  mov.b64 %d25, {%t15, %t16};\n"
      << "  add.u64 %d10, %d10, %d25;\n";
  }
  s << "  setp.ne.u64 %p8, %d10, 0;\n  and.pred %p8, %p8, %p1;\n  shl.b64 %d26, %d10, 5;\n"
       "  @%p8 red.global.add.u64 [%d4], %d26;\n  ret;\n" << stubs << "}\n";
  // lop3 executed per pass: loop levels' tables times their runs, the
  // unrolled levels' lop3 once per run of level Lr
  double per_grab = 0;
  for (size_t i = 0; i < lp.order.size(); i++)
    if (!isconst[lp.order[i].node] && (U == 0 || level[i] <= Lr)) per_grab += runs[level[i]];
  per_grab += (double)unrolled_lop3 * runs[Lr];
  if (lop3_per_pass) *lop3_per_pass = per_grab / REP;
  if (getenv("LEC_ES_JIT_LOG")) {
    std::string lv;
    for (uint32_t l = 0; l <= L; l++) {
      char t[64];
      snprintf(t, sizeof(t), "%s%zu", l ? "/" : "", (size_t)std::count(level.begin(), level.end(), (uint8_t)l));
      lv += t;
      if (l < L) {
        snprintf(t, sizeof(t), " [%llx] ", (unsigned long long)grp[l]);
        lv += t;
      }
    }
    fprintf(stderr,
            "lec_es JIT %016llx: %u tables, rep %u, pass PIs %016llx; tables per level: %s, %u unrolled "
            "(%u read below their level, %u from shared memory); %.1f lop3 per pass\n",
            (unsigned long long)g.hash, lp.count, REP, (unsigned long long)pass_pis, lv.c_str(), U, roots,
            (unsigned)nsmem, per_grab / REP);
  }
  return s.str();
}

int compile_ptx(const std::string &ptx, int major, int minor, std::vector<char> &cubin, std::string &log) {
  if (const char *dump = getenv("LEC_ES_DUMP_PTX")) {  // debugging aid: keep the generated PTX
    std::ofstream f(dump);
    f << ptx;
  }
  nvPTXCompilerHandle h = nullptr;
  if (nvPTXCompilerCreate(&h, ptx.size(), ptx.c_str()) != NVPTXCOMPILE_SUCCESS) return LEC_ES_EJIT;
  const std::string gpu = "--gpu-name=sm_" + std::to_string(major) + std::to_string(minor) + "a";
  const char *opts[] = {gpu.c_str(), "--verbose"};
  const nvPTXCompileResult rc = nvPTXCompilerCompile(h, 2, opts);
  size_t n = 0;
  if (nvPTXCompilerGetInfoLogSize(h, &n) == NVPTXCOMPILE_SUCCESS && n > 1) {
    std::string info(n, 0);
    nvPTXCompilerGetInfoLog(h, &info[0]);
    log += info;
  }
  if (rc != NVPTXCOMPILE_SUCCESS) {
    if (nvPTXCompilerGetErrorLogSize(h, &n) == NVPTXCOMPILE_SUCCESS && n > 1) {
      std::string err(n, 0);
      nvPTXCompilerGetErrorLog(h, &err[0]);
      log += err;
    }
    nvPTXCompilerDestroy(&h);
    return LEC_ES_EJIT;
  }
  n = 0;
  if (nvPTXCompilerGetCompiledProgramSize(h, &n) != NVPTXCOMPILE_SUCCESS || n == 0) {
    nvPTXCompilerDestroy(&h);
    return LEC_ES_EJIT;
  }
  cubin.resize(n);
  nvPTXCompilerGetCompiledProgram(h, cubin.data());
  nvPTXCompilerDestroy(&h);
  return LEC_ES_OK;
}

int compile_cubin(const std::string &src, int major, int minor, std::vector<char> &cubin, std::string &log);

// The table form goes straight to PTX and the PTX compiler; the AND form
// goes through NVRTC.
// built (optional, four entries) receives the register and plan budgets
// and the cap on unrolled copies (0: the default rule) of the layout the
// returned kernel was generated with (the dump variant reuses them), and
// its shared-memory slots per thread (above kStaticShared: dynamic).
int compile_program_kernel(const Program &g, bool lut_form, int major, int minor, std::vector<char> &cubin,
                           std::string &log, const GrabLayout *layout = nullptr, double *lop3_per_pass = nullptr,
                           uint32_t *built = nullptr, bool *grouped = nullptr) {
  bool grouped_sink = false;
  if (!grouped) grouped = &grouped_sink;
  *grouped = false;
  double per_sink = 0;
  uint32_t built_sink[4];
  if (!lop3_per_pass) lop3_per_pass = &per_sink;
  if (!built) built = built_sink;
  *lop3_per_pass = 0;
  built[2] = 0;  // copies cap (0: the default rule)
  built[3] = 0;  // shared-memory slots per thread
  // LEC_ES_JIT_NVRTC=1 compiles the table form from CUDA C++ through NVRTC
  // instead (same tables, for comparing the two compilation paths)
  static const bool via_nvrtc = getenv("LEC_ES_JIT_NVRTC") != nullptr;
  if (lut_form && !g.lut.order.empty() && !via_nvrtc) {
    // values kept across loops live in registers: if ptxas has to spill,
    // move 16 more of them into shared memory while slots remain, else
    // shrink the plan by 16 values, and build again
    GrabLayout own;
    if (!layout) {
      jit_layout(g, &own);
      layout = &own;
    }
    uint32_t regs = layout->regs, plan = layout->plan;
    auto spilled = [](const std::string &lg) {
      return lg.find(" 0 bytes spill stores") == std::string::npos && lg.find("spill stores") != std::string::npos;
    };
    auto next_layout = [&](const SlotSplit &split) {  // the step after a spill
      if (split.inner_in_regs > 0 && split.in_shared < shared_slots()) {
        regs = split.inner_in_regs - std::min<uint32_t>(16, split.inner_in_regs);
      } else {
        plan -= std::min<uint32_t>(16, plan);
        regs = std::min(regs, plan);
      }
    };
    // A large cone may need several builds.  Each step depends only on the
    // previous layout's slot split, so after a first build that spills (or
    // at once, for a single plan's build) the chain of layouts is generated
    // up front and compiled on host threads together.  The spill usually
    // comes from the unrolled copies' working set, which moving values to
    // shared memory or shrinking the plan does not lower predictably, so a
    // second chain halves the copies (from four to two, starting from the
    // search's budgets), at most kMaxChain steps each.  Candidates are tried
    // in order of the lop3 per pass they execute (chain order among equals);
    // the first without spills is kept.  If all spill, the build goes on
    // from the four-copy chain's end, one layout at a time.  (17x17
    // multiplier miter with 96 shared slots: the four-copy chain ended at
    // 726 lop3 per pass and still spilled, the two-copy one reached 631.)
    if (g.lut.count >= kParallelChainTables && !getenv("LEC_ES_JIT_SERIAL_BUILD")) {
      if (!t_single_build) {
        std::string lg;
        SlotSplit split;
        built[0] = regs;
        built[1] = plan;
        const int rc = compile_ptx(gen_ptx_lut(g, major, minor, layout->rep, regs, plan, layout->pass_pis,
                                               layout->groups, &split, lop3_per_pass),
                                   major, minor, cubin, lg);
        *grouped = split.grouped;
        built[3] = split.in_shared;
        if (rc != LEC_ES_OK || !spilled(lg) || plan == 0) {
          log += lg;
          return rc;
        }
        next_layout(split);
      }
      struct Cand {
        std::string ptx;
        double per = 0;
        uint32_t regs = 0, plan = 0, cap = 0, shared = 0;
        bool grouped = false;
      };
      // the two chains are generated on two host threads (each step of a
      // chain depends on the previous step's slot split)
      auto gen_chain = [&](uint32_t cap, uint32_t r, uint32_t pl, std::vector<Cand> &out) {
        for (uint32_t i = 0; i < kMaxChain; i++) {
          SlotSplit split;
          Cand cd;
          cd.ptx = gen_ptx_lut(g, major, minor, layout->rep, r, pl, layout->pass_pis, layout->groups, &split, &cd.per,
                               nullptr, cap);
          cd.regs = r;
          cd.plan = pl;
          cd.cap = cap;
          cd.shared = split.in_shared;
          cd.grouped = split.grouped;
          out.push_back(std::move(cd));
          if (pl == 0) break;
          if (split.inner_in_regs > 0 && split.in_shared < shared_slots()) {
            r = split.inner_in_regs - std::min<uint32_t>(16, split.inner_in_regs);
          } else {
            pl -= std::min<uint32_t>(16, pl);
            r = std::min(r, pl);
          }
        }
        return std::make_pair(r, pl);
      };
      // Waves: the first holds kMaxChain steps of each chain; while the
      // four-copy chain has steps left and its last step's lop3 per pass is
      // still below the best clean candidate's, the next wave continues it
      // (more values in shared memory, then a smaller plan).
      const uint32_t copies = unroll_copies(g.lut);
      std::vector<char> best_bin;
      std::string best_log;
      Cand best;
      bool have_best = false;
      int rc_fail = LEC_ES_OK;
      const double t0 = now_ms();
      for (uint32_t wave = 0; wave < 4; wave++) {
        std::vector<Cand> cands, chain_b;
        std::thread tb;
        if (wave == 0 && copies > 2 && copies <= 4)
          tb = std::thread([&]() { gen_chain(2, layout->regs, layout->plan, chain_b); });
        const auto a_end = gen_chain(0, regs, plan, cands);
        if (tb.joinable()) tb.join();
        const size_t chain_a = cands.size();
        const Cand a_last = cands.back();
        regs = a_end.first;
        plan = a_end.second;
        for (Cand &cd : chain_b) cands.push_back(std::move(cd));
        std::vector<size_t> order(cands.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cands[x].per < cands[y].per; });
        const size_t n = order.size();
        std::vector<int> rcs(n, LEC_ES_EJIT);
        std::vector<std::string> logs(n);
        std::vector<std::vector<char>> bins(n);
        std::vector<uint8_t> done(n, 0);
        std::mutex mu;
        size_t next_i = 0, first_ok = n;
        auto work = [&]() {
          for (;;) {
            size_t i;
            {
              std::lock_guard<std::mutex> lk(mu);
              if (next_i >= n || next_i > first_ok) return;  // a candidate earlier in the order already built clean
              if (have_best && cands[order[next_i]].per >= best.per) return;  // no better than the kept one
              i = next_i++;
            }
            const int rc = compile_ptx(cands[order[i]].ptx, major, minor, bins[i], logs[i]);
            std::lock_guard<std::mutex> lk(mu);
            rcs[i] = rc;
            done[i] = 1;
            if (rc == LEC_ES_OK && !spilled(logs[i])) first_ok = std::min(first_ok, i);
          }
        };
        const unsigned nt = (unsigned)std::min<size_t>(n, std::max(1u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < nt; t++) pool.emplace_back(work);
        work();
        for (auto &t : pool) t.join();
        for (size_t i = 0; i < n && done[i]; i++) {
          if (rcs[i] != LEC_ES_OK) {
            rc_fail = rcs[i];
            break;
          }
          if (spilled(logs[i])) continue;
          if (!have_best || cands[order[i]].per < best.per) {
            best = cands[order[i]];
            best_bin = std::move(bins[i]);
            best_log = logs[i];
            have_best = true;
          }
          break;
        }
        if (rc_fail) break;
        const bool a_done = a_last.plan == 0;
        if (!have_best && a_done) {  // every candidate spilled and the four-copy chain has no plan left: its last
          for (size_t i = 0; i < n; i++)
            if (order[i] == chain_a - 1) {
              if (!done[i]) rcs[i] = compile_ptx(cands[order[i]].ptx, major, minor, bins[i], logs[i]);
              if (rcs[i] != LEC_ES_OK) return rcs[i];
              best = cands[order[i]];
              best_bin = std::move(bins[i]);
              best_log = logs[i];
              have_best = true;
            }
          break;
        }
        if (a_done || (have_best && a_last.per >= best.per)) break;
      }
      if (rc_fail) return rc_fail;
      if (have_best) {
        if (getenv("LEC_ES_JIT_LOG"))
          fprintf(stderr,
                  "lec_es JIT %016llx: kept %.1f lop3 per pass (copies cap %u, %u shared slots, %s) in %.0f ms\n",
                  (unsigned long long)g.hash, best.per, best.cap, best.shared,
                  spilled(best_log) ? "spills" : "no spills", now_ms() - t0);
        log += best_log;
        cubin = std::move(best_bin);
        *lop3_per_pass = best.per;
        *grouped = best.grouped;
        built[0] = best.regs;
        built[1] = best.plan;
        built[2] = best.cap;
        built[3] = best.shared;
        return LEC_ES_OK;
      }
      // every candidate spilled: go on from the four-copy chain's end
    }
    for (;;) {
      std::string lg;
      SlotSplit split;
      built[0] = regs;
      built[1] = plan;
      built[2] = 0;
      const int rc = compile_ptx(gen_ptx_lut(g, major, minor, layout->rep, regs, plan, layout->pass_pis,
                                             layout->groups, &split, lop3_per_pass),
                                 major, minor, cubin, lg);
      *grouped = split.grouped;
      built[3] = split.in_shared;
      if (rc != LEC_ES_OK || !spilled(lg) || plan == 0) {
        log += lg;
        return rc;
      }
      next_layout(split);
    }
  }
  return compile_cubin(gen_source(g, lut_form), major, minor, cubin, log);
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

uint64_t cache_key(const Program &g, bool lut_form);
JitState *state(lec_es_ctx *c);

// The kernel cached for g's structure (both hashes), or null.  Called with
// js->mu held.
JitKernel *cached_kernel(JitState *js, const Program &g, bool lut_form) {
  auto it = js->cache.find(cache_key(g, lut_form));
  return it != js->cache.end() && it->second->hash2 == g.hash2 ? it->second : nullptr;
}

// Executed lop3 per pass of the kernel this context holds for g's cone, or
// 0 if it holds none (or does not know the figure).
double jit_held_lop3(lec_es_ctx *c, const Program &g) {
  if (!c || g.lut.count == 0) return 0.0;
  JitState *js = state(c);
  std::lock_guard<std::mutex> lk(js->mu);
  const JitKernel *k = cached_kernel(js, g, true);
  return k ? k->model_lop3 : 0.0;
}

bool jit_eligible(const Program &g) { return g.lut.count > 0 && !g.lut.order.empty() && g.lut.live <= kMaxJitLive; }

bool jit_held(lec_es_ctx *c, const Program &g) {
  if (g.lut.elided) return true;
  JitState *js = state(c);
  std::lock_guard<std::mutex> lk(js->mu);
  return cached_kernel(js, g, true) != nullptr;
}

// The ES time model (cost.cpp) decides: the specialised kernel when its
// predicted time, plus the predicted build time unless this context already
// holds the kernel, is below the interpreter's.  Cones whose table live set
// does not fit the register file stay on the interpreter.
uint32_t jit_auto_tier(lec_es_ctx *c, const Program &g, uint64_t chunks) {
  (void)chunks;
  if (g.lut.count == 0 || g.lut.live > kMaxJitLive) return LEC_ES_TIER_INTERP;
  bool cached = g.lut.elided;
  if (!cached && c) {
    JitState *js = state(c);
    std::lock_guard<std::mutex> lk(js->mu);
    cached = cached_kernel(js, g, true) != nullptr;
  }
  const double t_int = cost_run_ms(c, LEC_ES_TIER_INTERP, g.cone_ands, g.n);
  const double t_jit = cached ? cost_run_ms(c, LEC_ES_TIER_JIT, g.cone_ands, g.n, c ? jit_held_lop3(c, g) : 0.0)
                              : cost_run_ms(c, LEC_ES_TIER_JIT, g.cone_ands, g.n) + cost_compile_ms(c, g.lut.count);
  return t_jit < t_int ? LEC_ES_TIER_JIT : LEC_ES_TIER_INTERP;
}

namespace {

// Compile (or read from the disk cache) and load one program's kernel.
int build_kernel(lec_es_ctx *c, const Program &g, bool lut_form, JitKernel **out) {
  // an elided cover or slot program means the kernel was found by hash;
  // generating code from it would drop the program
  if ((lut_form && g.lut.elided) || (!lut_form && g.slots_elided)) return LEC_ES_EINVAL;
  const double t0 = now_ms();
  std::vector<char> cubin;
  std::string path;
  // the PTX form's grab layout (computed once: it searches loop nestings)
  const bool ptx_form = lut_form && !g.lut.order.empty() && !getenv("LEC_ES_JIT_NVRTC");
  GrabLayout lay;
  if (ptx_form) jit_layout(g, &lay);
  if (!c->jit_dir.empty()) {
    mkdir(c->jit_dir.c_str(), 0755);
    char name[160];
    uint64_t nest = 1469598103934665603ull;  // FNV-1a over the loop groups
    for (uint64_t m : lay.groups) nest = (nest ^ m) * 1099511628211ull;
    snprintf(name, sizeof(name), "/es_v%d_%016llx%016llx_%s%s_r%u_h%u_p%llx_n%llx_sm%d%d.cubin", kCodegenVersion,
             (unsigned long long)g.hash, (unsigned long long)g.hash2, lut_form ? "lut" : "and",
             getenv("LEC_ES_JIT_NVRTC") ? "_nvrtc" : "",
             lay.rep, lay.regs * 1000 + lay.plan, (unsigned long long)lay.pass_pis, (unsigned long long)nest, c->cc_major,
             c->cc_minor);
    path = c->jit_dir + name;
  }
  double nvrtc_ms = 0;
  double lop3_per_pass = 0;  // of the PTX form's kernel (a sidecar file next to a cached cubin)
  uint32_t budgets[4] = {lay.regs, lay.plan, 0, 0};  // register, plan and copies budgets it was generated with,
                                                     // and its shared-memory slots per thread
  bool grouped = false;                         // its passes run in straight-line groups
  if (path.empty() || !read_file(path, cubin)) {
    std::string log;
    const double tn = now_ms();
    int rc = compile_program_kernel(g, lut_form, c->cc_major, c->cc_minor, cubin, log, ptx_form ? &lay : nullptr,
                                    &lop3_per_pass, budgets, &grouped);
    nvrtc_ms = now_ms() - tn;
    if (rc) {
      if (getenv("LEC_ES_JIT_LOG")) fprintf(stderr, "lec_es JIT failed:\n%s\n", log.c_str());
      return rc;
    }
    if (!path.empty()) {
      write_file(path, cubin);
      const std::string txt =
          std::to_string(lop3_per_pass) + " " + std::to_string(budgets[0]) + " " + std::to_string(budgets[1]) + " " +
          std::to_string(grouped ? 1 : 0) + " " + std::to_string(budgets[2]) + " " + std::to_string(budgets[3]);
      write_file(path + ".lop3", std::vector<char>(txt.begin(), txt.end()));
    }
  } else {
    std::vector<char> txt;
    if (read_file(path + ".lop3", txt)) {
      const std::string t(txt.begin(), txt.end());
      double per = 0;
      unsigned r = budgets[0], pl = budgets[1], gr = 0, cp = 0, sh = 0;
      if (sscanf(t.c_str(), "%lf %u %u %u %u %u", &per, &r, &pl, &gr, &cp, &sh) >= 1) lop3_per_pass = per;
      budgets[0] = r;
      budgets[1] = pl;
      budgets[2] = cp;
      budgets[3] = sh;
      grouped = gr != 0;
    }
  }
  cudaSetDevice(c->device);
  const double tl = now_ms();
  JitKernel *k = new JitKernel();
  if (cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&k->kern, k->lib, "es_jit") != cudaSuccess) {
    if (k->lib) cudaLibraryUnload(k->lib);
    delete k;
    return LEC_ES_EJIT;
  }
  // slots beyond a static array's: dynamic shared memory, allowed once here
  k->dyn_smem = jit_dyn_smem(budgets[3]);
  if (k->dyn_smem && cudaKernelSetAttributeForDevice(k->kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)k->dyn_smem, c->device) != cudaSuccess) {
    cudaLibraryUnload(k->lib);
    delete k;
    return LEC_ES_EJIT;
  }
  cudaFuncAttributes attr;
  if (cudaFuncGetAttributes(&attr, (const void *)k->kern) == cudaSuccess) {
    k->regs = attr.numRegs;
    k->local_bytes = attr.localSizeBytes;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)k->kern, kJitBlock, k->dyn_smem);
  k->blocks_per_sm = std::max(1, bps);
  k->block = kJitBlock;
  k->num_luts = g.lut.count;
  k->lut_live = g.lut.live;
  k->num_slots = g.num_slots;
  k->order = g.order;
  k->num_records = g.num_records;
  k->work_per_chunk = lut_form ? g.lut.count : (uint32_t)g.recs.size();
  k->chunk_bits = g.n > 5 ? g.n - 5 : 0;
  k->hash2 = g.hash2;
  k->built_regs = budgets[0];
  k->built_plan = budgets[1];
  k->built_copies = budgets[2];
  if (ptx_form) {  // the PTX form: its grab layout
    k->rep_fixed = lay.rep;
    k->pass_bits = lay.pass_pis >> 5;
    k->stride_ok = jit_stride_ok(g.n, lay.rep);
    k->lop3_per_pass = lop3_per_pass;
    k->model_lop3 = lop3_per_pass > 0 ? lop3_per_pass + (grouped ? kGroupedPassSaving : 0.0) : 0.0;
  }
  k->load_ms = now_ms() - tl;
  k->nvrtc_ms = nvrtc_ms;
  k->compile_ms = now_ms() - t0;
  if (nvrtc_ms > 0) cost_add_compile(c, g.lut.count, k->compile_ms);  // a build, not a disk-cache read
  if (getenv("LEC_ES_JIT_LOG"))
    fprintf(stderr, "lec_es JIT %016llx: nvrtc %.1f ms, load %.1f ms, %d regs\n", (unsigned long long)g.hash,
            nvrtc_ms, k->load_ms, k->regs);
  *out = k;
  return LEC_ES_OK;
}

void worker_loop(lec_es_ctx *c) {
  // Background builds yield the host to the threads that launch kernels and
  // wait for them: this thread, and the threads it starts for layout dry
  // runs and compiles (they inherit its nice value), run at a lower
  // priority.  (A cold 16x16 check ran its interpreter slices 12 ms slower
  // than one interpreter launch while the build held every host thread.)
  setpriority(PRIO_PROCESS, (id_t)syscall(SYS_gettid), kBuildNice);
  JitState *js = c->jit;
  for (;;) {
    Program g;
    std::shared_ptr<const CompactMiter> cone;
    {
      std::unique_lock<std::mutex> lk(js->mu);
      js->cv.wait(lk, [&] { return js->stop || !js->todo.empty(); });
      if (js->stop) return;
      g = std::move(js->todo.front().prog);
      t_single_build = js->todo.front().urgent;
      cone = std::move(js->todo.front().cone);
      js->todo.pop_front();
    }
    JitKernel *k = nullptr;
    int rc = LEC_ES_OK;
    if (g.lut.deferred) {  // the front end left the table cover to this build
      Program full;
      rc = cone ? compile_program(cone->view(), LEC_ES_ORDER_AUTO, 63, full) : LEC_ES_EINVAL;
      if (!rc && (full.hash != g.hash || full.hash2 != g.hash2)) rc = LEC_ES_EINVAL;
      if (!rc && !jit_eligible(full)) rc = LEC_ES_ETOOBIG;
      if (!rc) g.lut = std::move(full.lut);
    }
    if (!rc) rc = build_kernel(c, g, true, &k);
    t_single_build = false;
    std::lock_guard<std::mutex> lk(js->mu);
    if (rc == LEC_ES_OK) {
      if (!js->cache.count(cache_key(g, true))) js->cache[cache_key(g, true)] = k;
      else js->unshared.push_back(k);  // the key is another structure's: never found by lookup
    }
    js->inflight.erase(cache_key(g, true));
    js->built.notify_all();
  }
}

}  // namespace

uint64_t cache_key(const Program &g, bool lut_form) { return g.hash ^ (lut_form ? 0x9E3779B97F4A7C15ull : 0ull); }

bool jit_want_cover(void *arg, uint32_t n, uint32_t cone_ands) {
  JitProbe *p = (JitProbe *)arg;
  if (p->use != JitProbe::kAuto) return true;
  constexpr double kCoverMinMs = 5.0;
  const bool want = cost_run_ms(p->c, LEC_ES_TIER_INTERP, cone_ands, n) >= kCoverMinMs;
  if (want && p->defer) {
    p->deferred = true;
    return false;
  }
  return want;
}

bool jit_probe(void *arg, uint64_t hash, uint64_t hash2, uint32_t n, uint32_t cone_ands, KernelFacts *f) {
  const JitProbe *p = (const JitProbe *)arg;
  lec_es_ctx *c = p->c;
  if (!c->jit) return false;
  JitKernel *k = nullptr;
  {
    JitState *js = c->jit;
    std::lock_guard<std::mutex> lk(js->mu);
    auto it = js->cache.find(hash ^ 0x9E3779B97F4A7C15ull);
    if (it == js->cache.end() || it->second->num_luts == 0 || it->second->hash2 != hash2) return false;
    k = it->second;
  }
  // will the caller run this kernel?  (else it needs the slot program)
  switch (p->use) {
    case JitProbe::kRun:
    case JitProbe::kInfo:
      break;
    case JitProbe::kAuto:
      if (k->lut_live > kMaxJitLive || !(cost_run_ms(c, LEC_ES_TIER_JIT, cone_ands, n, k->model_lop3) <
                                         cost_run_ms(c, LEC_ES_TIER_INTERP, cone_ands, n)))
        return false;
      break;
    case JitProbe::kBatch:
      if (!batch_wants_kernel(c, n, cone_ands, k->num_luts, k->lut_live)) return false;
      break;
  }
  f->luts = k->num_luts;
  f->live = k->lut_live;
  f->num_slots = k->num_slots;
  f->order = k->order;
  f->num_records = k->num_records;
  return true;
}

JitState *state(lec_es_ctx *c) {
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (!c->jit) c->jit = new JitState();
  return c->jit;
}

int jit_get_kernel(lec_es_ctx *c, const Program &g, bool lut_form, JitKernel **out, double *compile_ms) {
  JitState *js = state(c);
  const uint64_t key = cache_key(g, lut_form);
  {
    std::unique_lock<std::mutex> lk(js->mu);
    // a background build of this program is under way: wait for it
    js->built.wait(lk, [&] { return !js->inflight.count(key) || js->stop; });
    if (JitKernel *k = cached_kernel(js, g, lut_form)) {
      *out = k;
      if (compile_ms) *compile_ms = 0;
      return LEC_ES_OK;
    }
  }
  JitKernel *k = nullptr;
  int rc = build_kernel(c, g, lut_form, &k);
  if (rc) return rc;
  if (compile_ms) *compile_ms = k->compile_ms;
  std::lock_guard<std::mutex> lk(js->mu);
  auto it = js->cache.find(key);
  if (it == js->cache.end()) {
    js->cache[key] = k;
  } else if (it->second->hash2 == g.hash2) {  // another thread built it first
    cudaLibraryUnload(k->lib);
    delete k;
    k = it->second;
  } else {  // the key belongs to another structure: keep this kernel out of the cache
    js->unshared.push_back(k);
  }
  *out = k;
  return LEC_ES_OK;
}

int jit_attach(lec_es_ctx *c, lec_es_plan *p, JitKernel *k, const lec_es_options *opt) {
  const Program &g = p->prog;
  p->jit = k;
  p->jit_block = k->block;
  const uint64_t chunks = num_chunks(g.n);
  // a caller's grid is kept; otherwise each launch sizes its own (jit_geometry)
  p->jit_grid = 0;
  if (opt && opt->grid_blocks)
    p->jit_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(opt->grid_blocks, (chunks + k->block - 1) / k->block));
  (void)c;
  return LEC_ES_OK;
}

int jit_prepare(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt) {
  const Program &g = p->prog;
  JitState *js = state(c);
  (void)js;
  JitKernel *k = nullptr;
  t_single_build = true;
  int rc = jit_get_kernel(c, g, p->jit_lut, &k, &p->jit_ms);
  t_single_build = false;
  if (rc) return rc;
  return jit_attach(c, p, k, opt);
}

JitKernel *jit_lookup_or_schedule(lec_es_ctx *c, const Program &g, bool urgent,
                                  std::shared_ptr<const CompactMiter> cone) {
  JitState *js = state(c);
  std::lock_guard<std::mutex> lk(js->mu);
  const uint64_t key = cache_key(g, true);
  if (JitKernel *k = cached_kernel(js, g, true)) return k;
  if (!js->scheduled[key]) {
    js->scheduled[key] = true;
    js->inflight.insert(key);
    // a single check waiting on it goes first, and builds its chain of
    // layouts at once (the host is otherwise idle then)
    if (urgent) js->todo.push_front(JitState::Job{g, true, std::move(cone)});
    else js->todo.push_back(JitState::Job{g, false, std::move(cone)});
    if (js->workers.empty()) {
      const unsigned nw = std::max(1u, std::min(4u, std::thread::hardware_concurrency() / 2));
      for (unsigned i = 0; i < nw; i++) js->workers.emplace_back(worker_loop, c);
    }
    js->cv.notify_one();
  }
  return nullptr;
}

// Passes per grab: a power of two, compiled into the PTX form; otherwise
// ~4k instructions per warp per grab, but at least four grabs per warp of
// the grid so the counter still balances the load.
uint64_t jit_reps(const JitKernel *k, uint64_t chunks, uint64_t grid) {
  if (k->rep_fixed) return k->rep_fixed;
  const uint64_t per_chunk = std::max<uint64_t>(1, k->work_per_chunk) + 40;
  uint64_t rep = (4096 + per_chunk - 1) / per_chunk;
  const uint64_t warps = std::max<uint64_t>(1, grid * (uint64_t)(k->block / 32));
  rep = std::min<uint64_t>(rep, chunks / (32ull * 4ull * warps));
  rep = std::max<uint64_t>(1, std::min<uint64_t>(rep, 32));
  uint64_t p2 = 1;
  while (p2 * 2 <= rep) p2 <<= 1;
  return p2;
}

void jit_grab_range(const JitKernel *k, uint64_t rep, uint64_t cb, uint64_t ce, uint64_t *q0, uint64_t *qend) {
  if (!k->pass_bits) {  // contiguous grabs of 32 * rep chunks
    const uint64_t G = 32ull * rep;
    *q0 = cb / G;
    *qend = (ce + G - 1) / G;
    return;
  }
  // grab bits: chunk bits from 5 up that are not pass bits; grab q is every
  // chunk whose grab bits spell q.  Lowest chunk of q: its bits deposited;
  // highest: plus every pass bit and the lane bits.  Both grow with q.
  std::vector<uint32_t> pos;
  for (uint32_t b = 5; b < k->chunk_bits && b < 64; b++)
    if (!((k->pass_bits >> b) & 1u)) pos.push_back(b);
  const uint64_t lanes_and_pass = k->pass_bits | 31ull;
  auto lo = [&](uint64_t q) {
    uint64_t c = 0;
    for (size_t i = 0; i < pos.size(); i++) c |= ((q >> i) & 1ull) << pos[i];
    return c;
  };
  const uint64_t nq = pos.size() >= 63 ? ~0ull : (1ull << pos.size());
  auto first = [&](auto pred) {  // smallest q in [0, nq) with pred(q), else nq
    uint64_t a = 0, b = nq;
    while (a < b) {
      const uint64_t m = a + (b - a) / 2;
      if (pred(m)) b = m;
      else a = m + 1;
    }
    return a;
  };
  *q0 = first([&](uint64_t q) { return (lo(q) | lanes_and_pass) >= cb; });
  *qend = first([&](uint64_t q) { return lo(q) >= ce; });
  if (*qend < *q0) *qend = *q0;
}

void jit_geometry(const JitKernel *k, uint64_t chunks, int sm_count, uint64_t *grid, uint64_t *rep,
                  bool *strided) {
  // Every warp grab costs one atomic on a single counter, so a small cone
  // needs both long grabs (rep passes of 32 chunks, ~4k instructions) and a
  // grid no larger than its grabs can keep busy (four grabs per warp); the
  // grid keeps at least 8 warps per SM, shortening grabs if it has to, and
  // at most what is resident at once.  A PTX-form kernel whose grabs fit in
  // two rounds of the resident warps takes them by a static stride instead
  // (every grab is the same work; no counter), about 8 per warp: on a
  // 124-table, 24-PI node-pair miter 29.8 us with the counter, 21 / 15 /
  // 12.6 us at 1 / 4 / 8 grabs per warp; the 4,096-pair batch 5.72 -> 5.40
  // ms.
  const uint64_t wpb = (uint64_t)std::max(1, k->block / 32);
  const uint64_t w_full = (uint64_t)sm_count * (uint64_t)k->blocks_per_sm * wpb;
  const uint64_t w_min = std::min<uint64_t>(w_full, (uint64_t)sm_count * 8ull);
  if (strided) *strided = false;
  if (k->rep_fixed) {
    const uint64_t r = k->rep_fixed;
    const uint64_t grabs = std::max<uint64_t>(1, (chunks + 32ull * r - 1) / (32ull * r)) + 1;  // + an unaligned end
    uint64_t w = std::min<uint64_t>(w_full, std::max(std::min(w_min, grabs), grabs / 4));
    if (strided && k->stride_ok && grabs <= 2 * w_full) {
      *strided = true;
      w = std::min<uint64_t>(w_full, std::max(std::min(w_min, grabs), (grabs + 7) / 8));
    }
    *rep = r;
    *grid = std::max<uint64_t>(1, (w + wpb - 1) / wpb);
    return;
  }
  const uint64_t per_chunk = std::max<uint64_t>(1, k->work_per_chunk) + 40;
  uint64_t r = std::min<uint64_t>(32, (4096 + per_chunk - 1) / per_chunk);
  uint64_t grabs = chunks / (32ull * r);
  uint64_t w = std::min<uint64_t>(w_full, grabs / 4);
  if (w < w_min) {
    r = std::max<uint64_t>(1, std::min<uint64_t>(r, chunks / (32ull * 4ull * w_min)));
    grabs = (chunks + 32ull * r - 1) / (32ull * r);
    w = std::min<uint64_t>(w_full, std::max<uint64_t>(1, grabs / 4));
  }
  uint64_t p2 = 1;  // grabs are aligned to 32 * rep chunks: a power of two
  while (p2 * 2 <= r) p2 <<= 1;
  *rep = p2;
  *grid = std::max<uint64_t>(1, (w + wpb - 1) / wpb);
}

int jit_launch(lec_es_ctx *c, lec_es_plan *p, uint64_t chunk_begin, uint64_t chunk_end, int grid,
               uint64_t max_grabs) {
  unsigned long long *cex = p->d_res, *evaluated = p->d_res + 1, *next = p->d_res + 3;
  uint64_t geo_grid = 1, rep = 1;
  bool strided = false;
  jit_geometry(p->jit, chunk_end - chunk_begin, c->sm_count, &geo_grid, &rep, &strided);
  const int fixed = grid > 0 ? grid : p->jit_grid;
  const int g = fixed > 0 ? fixed : (int)geo_grid;
  if (fixed > 0) rep = jit_reps(p->jit, chunk_end - chunk_begin, (uint64_t)g);
  if (strided && fixed <= 0 && max_grabs == ~0ull) next = nullptr;  // static stride (PTX form only)
  uint64_t q0 = 0, qend = 0;
  jit_grab_range(p->jit, rep, chunk_begin, chunk_end, &q0, &qend);
  void *args[] = {&chunk_begin, &chunk_end, &cex, &evaluated, &next, &max_grabs, &rep, &q0, &qend};
  cudaError_t e =
      cudaLaunchKernel((const void *)p->jit->kern, dim3(g), dim3(p->jit_block), args, p->jit->dyn_smem, p->stream);
  return e == cudaSuccess ? 0 : (int)e;
}

// Per-table values of g's specialised kernel (lec_es_truth_tables_ex, JIT
// tier).  The context's kernel for g is built first if it holds none; the
// dump variant is generated with that kernel's layout and budgets, compiled
// and loaded for this call only, and run over words [wb, we).  rows (host,
// cone_ands x (we - wb) words) receives the row of every table's node (its
// dense AND id: rank in ascending variable order) and valid[row] = 1; other
// rows are left alone.
int jit_dump_tables(lec_es_ctx *c, const Program &g, uint64_t wb, uint64_t we, uint64_t *rows, uint8_t *valid) {
  const LutProgram &lp = g.lut;
  if (lp.elided) return LEC_ES_EINVAL;
  if (lp.order.empty()) return LEC_ES_OK;
  JitKernel *k = nullptr;
  t_single_build = true;
  int rc = jit_get_kernel(c, g, true, &k, nullptr);
  t_single_build = false;
  if (rc) return rc;
  GrabLayout lay;
  jit_layout(g, &lay);
  const bool known = k->built_regs || k->built_plan;
  std::vector<uint64_t> clear;
  const std::string ptx = gen_ptx_lut(g, c->cc_major, c->cc_minor, lay.rep, known ? k->built_regs : lay.regs,
                                      known ? k->built_plan : lay.plan, lay.pass_pis, lay.groups, nullptr, nullptr,
                                      &clear, k->built_copies);
  std::vector<char> cubin;
  std::string log;
  rc = compile_ptx(ptx, c->cc_major, c->cc_minor, cubin, log);
  if (rc) return rc;
  cudaSetDevice(c->device);
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&kern, lib, "es_jit") != cudaSuccess) {
    if (lib) cudaLibraryUnload(lib);
    return LEC_ES_EJIT;
  }
  const size_t NT = lp.order.size();
  const uint64_t NCH = num_chunks(g.n);
  const uint64_t stride = 1ull << std::max<uint32_t>(g.n > 5 ? g.n - 5 : 0, 5);  // as gen_ptx_lut's
  const size_t bytes = NT * stride * 4u;
  void *d_tt = c->arena.alloc(bytes);
  unsigned long long *d_res = (unsigned long long *)c->arena.alloc(kResWords * 8);
  std::vector<uint32_t> h;
  int err = 0;
  if (!d_tt || !d_res) {
    err = LEC_ES_ENOMEM;
  } else {
    cudaStream_t st = c->stream;
    uint64_t cb = std::min<uint64_t>(2 * wb, NCH), ce = std::min<uint64_t>(2 * we, NCH);
    uint64_t rep = lay.rep, q0 = 0, qend = 0, maxg = ~0ull;
    jit_grab_range(k, rep, cb, ce, &q0, &qend);
    cudaError_t e = cudaSuccess;
    if (k->dyn_smem)
      e = cudaKernelSetAttributeForDevice(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k->dyn_smem,
                                          c->device);
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)kern, kJitBlock, k->dyn_smem);
    const unsigned grid = (unsigned)std::max(1, c->sm_count * std::max(1, bps));
    unsigned long long *cex = d_res, *ev = d_res + 1, *next = d_res + 3;  // a counter: no static stride
    void *tt = d_tt;
    void *args[] = {&cb, &ce, &cex, &ev, &next, &maxg, &rep, &q0, &qend, &tt};
    h.resize(NT * stride);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_tt, 0, bytes, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_res, c->h_init, kResWords * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaLaunchKernel((const void *)kern, dim3(grid), dim3(kJitBlock), args, k->dyn_smem, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_tt, bytes, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || e != cudaSuccess) err = LEC_ES_ECUDA;
  }
  c->arena.free(d_tt);
  c->arena.free(d_res);
  cudaLibraryUnload(lib);
  if (err) return err;
  // table i's value at chunk c is row i at c with the chunk bits of deeper
  // pass PIs cleared (where this layout computes it); word w = chunks 2w, 2w+1
  const uint64_t nw = we - wb;
  for (size_t i = 0; i < NT; i++) {
    const uint32_t row = (uint32_t)lp.order[i].node;
    valid[row] = 1;
    const uint32_t *src = h.data() + i * stride;
    for (uint64_t w = wb; w < we; w++) {
      const uint64_t c0 = 2 * w, c1 = 2 * w + 1;
      const uint32_t v0 = src[c0 & ~clear[i]];
      const uint32_t v1 = c1 < NCH ? src[c1 & ~clear[i]] : v0;
      rows[(uint64_t)row * nw + (w - wb)] = (uint64_t)v1 << 32 | v0;
    }
  }
  return LEC_ES_OK;
}

void jit_release_all(lec_es_ctx *c) {
  if (!c->jit) return;
  JitState *js = c->jit;
  {
    std::lock_guard<std::mutex> lk(js->mu);
    js->stop = true;
  }
  js->cv.notify_all();
  js->built.notify_all();
  for (auto &t : js->workers) t.join();
  for (auto &kv : js->cache) {
    if (kv.second->lib) cudaLibraryUnload(kv.second->lib);
    delete kv.second;
  }
  for (JitKernel *k : js->unshared) {
    if (k->lib) cudaLibraryUnload(k->lib);
    delete k;
  }
  delete js;
  c->jit = nullptr;
}

// Source of the specialised kernel (no GPU needed).
std::string jit_source_for(const Program &g) { return gen_source(g, true); }

}  // namespace lec

extern "C" uint32_t lec_es_codegen_version(void) { return (uint32_t)lec::kCodegenVersion; }

extern "C" int lec_es_jit_compile(const lec_es_miter *m, int cc_major, int cc_minor, char *log, size_t log_cap,
                                  uint64_t *cubin_bytes) {
  if (!m) return LEC_ES_EINVAL;
  lec::Program g;
  lec::MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc = lec::compile_program(v, LEC_ES_ORDER_AUTO, 63, g);
  if (rc) return rc;
  std::vector<char> cubin;
  std::string lg;
  rc = lec::compile_program_kernel(g, true, cc_major, cc_minor, cubin, lg);
  if (log && log_cap) {
    const size_t n = std::min(log_cap - 1, lg.size());
    memcpy(log, lg.data(), n);
    log[n] = 0;
  }
  if (cubin_bytes) *cubin_bytes = cubin.size();
  return rc;
}
