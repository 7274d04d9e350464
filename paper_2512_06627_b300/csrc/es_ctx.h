// es_ctx.h -- definitions of the opaque C-ABI handles and the internal
// interfaces between the C ABI, the JIT tier, the batch engine and the server.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lec_es.h"
#include "es_internal.h"

namespace lec {

// First-fit sub-allocator over one device allocation (256-byte blocks).
struct Arena {
  uint8_t *base = nullptr;
  size_t bytes = 0;
  size_t in_use = 0;
  std::mutex mu;
  std::map<size_t, size_t> free_list;  // offset -> size
  std::map<size_t, size_t> used;
  int init(void *base, size_t bytes);
  void *alloc(size_t n);
  void free(void *p);
};

struct PlanGeom {
  int block = 0;
  int grid = 0;
  size_t smem = 0;
  uint32_t ring_recs = 0;
  uint32_t resident = 0;
  uint32_t nrec_padded = 0;
  bool spill = false;
  bool word = false;  // word-wide shared-memory kernel (else the chunk kernel)
};

// Pinned result words and events of one run, recycled by the context.
struct RunRes {
  unsigned long long *h_res = nullptr;  // kResWords pinned words
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
};

struct JitKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  int regs = 0;
  size_t local_bytes = 0;
  int block = 128;
  int blocks_per_sm = 1;
  double compile_ms = 0;   // whole build
  double nvrtc_ms = 0;     // of which NVRTC (0 on a disk-cache hit)
  double load_ms = 0;      // of which loading the cubin and querying the kernel
  uint32_t num_luts = 0;   // the program's table count and live count when built
  uint32_t lut_live = 0;
  uint32_t num_slots = 0, order = 0, num_records = 0;  // its slot program's, for results
  uint32_t work_per_chunk = 0;  // straight-line instructions per 32-pattern chunk (about)
  uint32_t rep_fixed = 0;       // passes per grab compiled into the kernel (0: a launch parameter)
  bool stride_ok = false;       // the kernel can take grabs by static stride (a null counter)
  double lop3_per_pass = 0;     // lop3 it executes per 32-pattern chunk and thread (0: unknown)
  double model_lop3 = 0;        // the figure the time model takes for it: lop3_per_pass, less the
                                // control a kernel with pass groups saves (0: unknown)
  uint64_t pass_bits = 0;       // chunk-index bits of the pass PIs (0: contiguous grabs of 32 * rep chunks)
  uint32_t chunk_bits = 0;      // bits of the chunk index (support PIs - 5)
  uint64_t hash2 = 0;           // the program's second structure hash (checked on every cache hit)
  uint32_t built_regs = 0, built_plan = 0;  // budgets of the layout it was generated with (PTX form)
  uint32_t built_copies = 0;                // its cap on unrolled copies (0: the default rule)
  size_t dyn_smem = 0;                      // dynamic shared memory every launch passes (bytes)
};
struct JitState;
struct Server;

// ES time model of §3.2 refit per tier: t = a + c * gates + alpha * gates *
// 2^(n - 23) (beta fixed at the paper's 23, so alpha is in the paper's
// units; c * gates is one pass over the program, the floor for small
// supports), fitted in relative error from weighted normal-equation sums that
// start from built-in B300 values.
struct CostSums {
  double S[3][3] = {};         // sum of f f^T / t^2 over features f = (1, gates, x)
  double b[3] = {};            // sum of f / t
  uint64_t count = 0;
};
struct CostFit {
  double coef[3] = {0, 0, 0};  // a_ms, c_ms, alpha_ms
  double S[3][3] = {};         // prior (built-in values) sums
  double b[3] = {};
  // measured runs, binned by (n, log2 gates); a bin counts as at most a few
  // samples, so thousands of runs of one size cannot outweigh the others
  std::map<uint32_t, CostSums> bins;
  uint64_t samples = 0;        // measurements added on this context
};
struct CostModel {
  std::mutex mu;
  CostFit tier[4];       // indexed by LEC_ES_TIER_*
  CostFit compile;       // specialised-kernel build: a + c * tables (coef[0], coef[1])
  CostFit kernel;        // specialised kernel by its executed lop3: x = (lop3 + 40) * 2^(n - 23)
  bool ready = false;
};

double now_ms();

// Random simulation of a whole AIG on the GPU (sweep.cu): signatures (host
// rows, may be null), hashes (phase-normalised with norm), PI-support masks
// (num_pis <= 64; may be null).
int simulate(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, const uint64_t *pi_words,
             uint32_t nwords, uint64_t *h_sigs, uint64_t *h_hash, uint64_t *h_sup, bool norm);

// ES time model (cost.cpp).  c may be null (built-in values only).
// lop3 > 0 (the executed lop3 per pass of a built specialised kernel)
// predicts or fits a JIT run by that kernel's work instead of its gates.
double cost_x(uint32_t gates, uint32_t n);
double cost_run_ms(lec_es_ctx *c, uint32_t tier, uint32_t gates, uint32_t n, double lop3 = 0);
double cost_compile_ms(lec_es_ctx *c, uint32_t tables);
void cost_add_run(lec_es_ctx *c, uint32_t tier, uint32_t gates, uint32_t n, double ms, double lop3 = 0);
void cost_add_compile(lec_es_ctx *c, uint32_t tables, double ms);
// Weighted (relative-error) least squares of t = a + c g + alpha x with all
// three coefficients >= 0; coef = (a, c, alpha).
bool cost_fit(const double *g, const double *x, const double *t, size_t k, double coef[3]);
int wait_event(cudaEvent_t ev, double timeout_s);
int choose_interp_geometry(lec_es_ctx *c, const Program &prog, uint64_t chunks, const lec_es_options *opt,
                           PlanGeom &g);
// Geometry of the word-wide kernel; false if the live set does not fit
// shared memory even at 32 threads per block.  The block is the largest
// power of two up to 256 (or opt->block_threads) that fits; with `widest`
// and no block asked for, a block of a multiple of 128 threads up to
// kMaxWordBlock (the same number of warps on each of the SM's four
// schedulers), records resident or in the ring, replaces it when that keeps
// at least a quarter more warps on each SM (a live set that leaves one
// 256-thread block per SM is latency-bound).
bool choose_word_geometry(lec_es_ctx *c, const Program &prog, const lec_es_options *opt, PlanGeom &g,
                          bool widest = false);

// JIT tier (jit.cpp)
uint32_t jit_auto_tier(lec_es_ctx *c, const Program &g, uint64_t chunks);
// Executed lop3 per pass of the held kernel of g's cone (0: none held).
double jit_held_lop3(lec_es_ctx *c, const Program &g);
int jit_prepare(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt);
// Passes of 32 chunks per grab for a launch of `grid` blocks over `chunks`.
uint64_t jit_reps(const JitKernel *k, uint64_t chunks, uint64_t grid);
// Grab numbers [q0, qend) covering chunks [cb, ce) for the kernel's layout.
void jit_grab_range(const JitKernel *k, uint64_t rep, uint64_t cb, uint64_t ce, uint64_t *q0, uint64_t *qend);
// Grid and passes per grab for a launch over `chunks` chunks.
void jit_geometry(const JitKernel *k, uint64_t chunks, int sm_count, uint64_t *grid, uint64_t *rep,
                  bool *strided = nullptr);
int jit_launch(lec_es_ctx *c, lec_es_plan *p, uint64_t chunk_begin, uint64_t chunk_end, int grid,
               uint64_t max_grabs);
// Non-blocking lookup for the server: the compiled kernel if ready, else
// schedules a background compile (once per program) and returns nullptr.
// urgent: a single check races the interpreter against this build (it goes
// to the front of the queue and builds its chain of layouts at once).
// cone: g's cone, needed when g's cover is deferred (the build makes it).
lec::JitKernel *jit_lookup_or_schedule(lec_es_ctx *c, const Program &g, bool urgent = false,
                                       std::shared_ptr<const CompactMiter> cone = nullptr);
// Whether g's cone can run as a specialised kernel (a table cover whose live
// set fits the register file).
bool jit_eligible(const Program &g);
// Whether the context holds g's table-form kernel.
bool jit_held(lec_es_ctx *c, const Program &g);
int jit_attach(lec_es_ctx *c, lec_es_plan *p, JitKernel *k, const lec_es_options *opt);
// Cached kernel for a program (compiled on a miss; thread-safe).
int jit_get_kernel(lec_es_ctx *c, const Program &g, bool lut_form, JitKernel **out, double *compile_ms);
// Per-table values of g's specialised kernel over words [wb, we) (see jit.cpp).
int jit_dump_tables(lec_es_ctx *c, const Program &g, uint64_t wb, uint64_t we, uint64_t *rows, uint8_t *valid);
// KernelProbe callback: the compiled table-form kernel for a program hash,
// if the context holds one and the caller will run it (arg = JitProbe).
struct JitProbe {
  enum Use { kRun, kAuto, kBatch, kInfo };
  lec_es_ctx *c;
  Use use;  // kRun: the kernel tier was asked for; kAuto: the AUTO choice; kBatch: the batch's split; kInfo: facts only
  // kAuto only: a cone that would get a cover gets none, and `deferred` is
  // set (a one-off check builds the kernel in the background from the cone)
  bool defer = false;
  bool deferred = false;
};
bool jit_probe(void *arg, uint64_t hash, uint64_t hash2, uint32_t n, uint32_t cone_ands, KernelFacts *facts);
// KernelProbe::want_cover for an AUTO caller: a cone whose interpreter run
// is predicted below kCoverMinMs never gets a kernel built by AUTO (a build
// takes tens of milliseconds at least), so it needs no table cover.
bool jit_want_cover(void *arg, uint32_t n, uint32_t cone_ands);
// The batch gives a miter its own kernel (else the tile queue).
bool batch_wants_kernel(lec_es_ctx *c, uint32_t n, uint32_t cone_ands, uint32_t luts, uint32_t live);
void jit_release_all(lec_es_ctx *c);

// single-miter plans (api.cpp)
int plan_prepare(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt, lec_es_plan **out);
int plan_prepare_program(lec_es_ctx *c, Program &&prog, const lec_es_options *opt, lec_es_plan **out);
int plan_run_async(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt);
int plan_run_async_grid(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt, int grid_override);
int plan_finish_device(lec_es_ctx *c, lec_es_plan *p);
int run_res_acquire(lec_es_ctx *c, RunRes *out);
void run_res_release(lec_es_ctx *c, const RunRes &r);
void run_res_destroy_all(lec_es_ctx *c);
int plan_result(lec_es_ctx *c, lec_es_plan *p, lec_es_result *out);
void plan_release(lec_es_ctx *c, lec_es_plan *p);
void fill_result(const lec_es_plan *p, lec_es_result *out);

// server (server.cpp)
void server_shutdown(lec_es_ctx *c);

}  // namespace lec

struct lec_es_ctx {
  int device = 0;
  int sm_count = 0;
  int smem_optin = 0;
  int cc_major = 0, cc_minor = 0;
  uint32_t max_pis = 63;
  double timeout_s = 600.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *arena_base = nullptr;
  bool own_arena = false;
  lec::Arena arena;
  unsigned long long *h_init = nullptr;  // pinned result-word initialiser, kResWords words
  std::string jit_dir;
  lec::JitState *jit = nullptr;
  lec::Server *server = nullptr;
  std::mutex server_mu;
  size_t slot_budget = (size_t)32 << 30;
  uint32_t max_inflight = 64;
  // recycled per-run resources (pinned host words are allocated in slabs)
  std::mutex res_mu;
  std::vector<lec::RunRes> res_free;
  std::vector<void *> res_slabs;
  std::vector<cudaEvent_t> res_events;
  lec::CostModel cost;  // ES time model, refined by this context's runs
};

// Result words of a run: [0] lowest failing pattern (init ~0), [1] patterns
// evaluated, [2] status, [3] JIT chunk-grab counter, [4] a second
// counterexample word (init ~0) for runs that must not exit early.
constexpr int kResWords = 8;

struct lec_es_plan {
  lec::Program prog;
  lec::RunRes res;                       // from the context's pool
  lec::PlanGeom geom;
  uint32_t tier = 0;
  void *d_recs = nullptr;
  void *d_loads = nullptr;               // word-wide kernel: PI/constant loads
  uint32_t nload = 0, out_off = 0;
  void *d_spill = nullptr;
  size_t spill_bytes = 0;
  unsigned long long *d_res = nullptr;  // kResWords result words
  unsigned long long *h_res = nullptr;  // pinned copy
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  bool pending = false;
  uint64_t last_wb = 0, last_we = 0;
  bool last_default_grid = false;        // the last run used the library's own launch geometry
  bool user_grid = false;                // prepared with a caller's grid_blocks
  double host_ms = 0, jit_ms = 0;
  lec::JitKernel *jit = nullptr;
  int jit_block = 0, jit_grid = 0;
  bool jit_lut = true;                   // table form (else AND form)
  uint32_t flags = 0;                    // LEC_ES_FLAG_* the plan was prepared with
  cudaStream_t stream = nullptr;         // where runs are enqueued (ctx stream by default)
};
