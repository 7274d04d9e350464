/*
 * lec_es.h -- C ABI of the B300 exact-simulation (ES) engine.
 *
 * Problem (paper §2.1): given a miter AIG -- two combinational circuits with
 * corresponding outputs XORed and the XORs ORed into one output -- prove the
 * output constant 0 (EQUIVALENT) or return an input pattern that sets it
 * (NONEQUIVALENT).  ES (paper §2.2, "Exact Simulation") decides this by
 * evaluating the output's cone under every assignment of its primary-input
 * support.  The cone is compiled into a branch-free instruction stream whose
 * value registers are reused under reference-count guidance (paper §3.3,
 * "Instructionalized ES").
 *
 * Conventions for every entry point:
 *   - returns lec_es_status (0 = LEC_ES_OK); nothing aborts, throws or exits;
 *   - input arrays are caller-owned and only read during the call; the
 *     library copies what it keeps (submit included);
 *   - result structs are caller-allocated and written only on LEC_ES_OK;
 *   - device pointers are marked "device"; everything else is host memory;
 *   - one lec_es_ctx per host thread, except lec_es_submit / poll / wait /
 *     cancel, which are thread-safe on one ctx.
 *
 * Pattern numbering: the support S of the output is the set of PIs in its
 * transitive fan-in cone (§2.1) sorted by PI index, n = |S|.  Pattern p gives
 * bit k of p to PI S[k].  A 64-pattern word w holds patterns 64w..64w+63:
 * PI S[k] is the constant mask with bit b = bit k of b for k < 6, and all ones
 * iff bit (k-6) of w is set for k >= 6.  There are max(1, 2^(n-6)) words.
 * The counterexample reported is the lowest failing p.
 */
#ifndef LEC_ES_H
#define LEC_ES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lec_es_ctx lec_es_ctx;   /* opaque: device state, arena, JIT cache */
typedef struct lec_es_plan lec_es_plan; /* opaque: one compiled, device-resident miter */
typedef struct lec_es_batch_plan lec_es_batch_plan; /* opaque: many miters, one launch */

typedef enum {
  LEC_ES_OK = 0,
  LEC_ES_EINVAL = 1,        /* malformed graph or argument */
  LEC_ES_ETOOBIG = 2,       /* n > max_pis (<= 63) or more than 65535 value slots */
  LEC_ES_ENOMEM = 3,        /* host allocation or device arena exhausted */
  LEC_ES_ECUDA = 4,         /* a CUDA runtime call failed */
  LEC_ES_ETIMEOUT = 5,      /* wait deadline passed */
  LEC_ES_EBUSY = 6,         /* poll: request not finished yet */
  LEC_ES_ECANCELLED = 7,    /* request was cancelled */
  LEC_ES_EDEVICE_WAIT = 8,  /* a bounded device-side wait gave up (kernel returned early) */
  LEC_ES_EJIT = 9,          /* run-time compilation of a specialised kernel failed */
  LEC_ES_ENOTFOUND = 10     /* unknown ticket */
} lec_es_status;

typedef enum {
  LEC_ES_EQUIVALENT = 0,
  LEC_ES_NONEQUIVALENT = 1,
  LEC_ES_UNDECIDED = 2      /* only a word sub-range was checked and it passed */
} lec_es_verdict;

/* Kernel tiers. */
enum {
  LEC_ES_TIER_AUTO = 0,
  LEC_ES_TIER_INTERP = 1,   /* generic interpreter, value slots in shared memory */
  LEC_ES_TIER_JIT = 2,      /* cone compiled to straight-line register code (NVRTC) */
  LEC_ES_TIER_SPILL = 3     /* generic interpreter, value slots in global memory */
};

/* Evaluation orders for the slot compiler (all give identical results). */
enum {
  LEC_ES_ORDER_AUTO = 0,    /* the fewer value slots of DFS and VAR */
  LEC_ES_ORDER_DFS = 1,     /* post-order from the output, deeper fanin first */
  LEC_ES_ORDER_VAR = 2,     /* ascending variable index */
  LEC_ES_ORDER_LEVEL = 3,   /* by logic level, then variable */
  LEC_ES_ORDER_GREEDY = 4   /* list scheduling that keeps the live set small */
};

/* A miter: AIGER numbering.  Variable 0 is FALSE, 1..num_pis are PIs, AND
 * variable num_pis+1+i has fanins fanins[2i], fanins[2i+1] (literals 2*var +
 * complement, each fanin variable below the AND's own).  Only the cone of
 * out_lit is read, so many miters may share one fanins array. */
typedef struct {
  uint32_t num_pis;
  uint32_t num_ands;
  const uint32_t *fanins;   /* host, 2*num_ands literals */
  uint32_t out_lit;
} lec_es_miter;

typedef struct {
  lec_es_verdict verdict;
  uint32_t support_n;       /* n */
  uint64_t cex;             /* lowest failing pattern (UINT64_MAX if none) */
  uint32_t support[64];     /* S[0..n-1]: original PI indices, 0-based */
  uint32_t cone_ands;       /* AND nodes in the cone (the evaluation count unit) */
  uint32_t num_slots;       /* value slots after reference-count reuse */
  uint32_t tier;            /* LEC_ES_TIER_* that ran */
  uint32_t order;           /* LEC_ES_ORDER_* used */
  uint64_t words_checked;   /* 64-pattern words in the requested range */
  double device_ms;         /* kernel time (CUDA events) */
  double host_ms;           /* front end: cone, order, slots, upload */
  double jit_ms;            /* run-time compilation (0 if cached) */
  double latency_ms;        /* served requests: completion minus submission */
} lec_es_result;

typedef struct {
  uint64_t word_begin;      /* first 64-pattern word checked (default 0) */
  uint64_t word_end;        /* one past the last; UINT64_MAX = all words */
  uint32_t tier;            /* LEC_ES_TIER_* (default AUTO) */
  uint32_t order;           /* LEC_ES_ORDER_* (default AUTO) */
  uint32_t block_threads;   /* 0 = library choice; single miter: an upper bound (a power of two
                               32..256 is used); batch: threads per tile pass, a multiple of 32 in
                               64..512 (a smaller multiple of 32 if it does not fit shared memory) */
  uint32_t grid_blocks;     /* 0 = library choice */
  uint32_t flags;           /* LEC_ES_FLAG_* */
  uint32_t tile_granularity;/* batch: tiles per resident block slot (0 = 8) */
  uint32_t stage_records;   /* batch: 16-byte records per staging stage, even, <= 2048 (0 = 256) */
} lec_es_options;

/* Option flags. */
enum {
  LEC_ES_FLAG_JIT_AND_FORM = 1u,     /* JIT tier: one C expression per AND, fused by the
                                        compiler, instead of the 3-input table cover */
  LEC_ES_FLAG_TEST_WAIT_TIMEOUT = 2u,/* test hook (interpreter tier): the kernel waits for
                                        16 bytes more than its record copy delivers, so
                                        its bounded wait must give up and the call must
                                        return LEC_ES_EDEVICE_WAIT */
  LEC_ES_FLAG_AUTOTUNE = 4u          /* batch: time candidate layouts (threads per tile
                                        pass x tiles per block slot x staging depth) on
                                        the tile queue and keep the fastest; cached per
                                        batch shape (and in jit_cache_dir) */
};

typedef struct {
  int device;               /* CUDA device ordinal */
  void *arena;              /* device memory the ctx sub-allocates from, e.g. a
                               torch tensor; NULL = the ctx allocates
                               arena_bytes itself with cudaMalloc */
  size_t arena_bytes;
  void *stream;             /* cudaStream_t for all work; NULL = ctx creates one */
  uint32_t max_pis;         /* <= 63; default 63 when 0 */
  double timeout_s;         /* bound on any host wait; 0 = 600 s */
  const char *jit_cache_dir;/* directory for compiled JIT kernels; NULL = memory only */
} lec_es_config;

/* Host-only view of a compiled slot program (no GPU needed).  Records are
 * 8 bytes: {u16 dst, u16 a, u16 b, u8 op, u8 flags}; op 0..3 = AND of slots a
 * and b, operand a complemented if op&1, b if op&2; op 4 = load support PI a;
 * op 5 = load constant 0.  flags 1 marks a load of the constant into a free
 * slot that only separates an AND from a recent AND whose result it reads
 * (cones of 256 ANDs or more: no AND reads one of the 3 ANDs before it
 * without a load between, so the interpreter can evaluate 4 at once).
 * Caller provides records[cap]. */
typedef struct {
  uint32_t n;
  uint32_t support[64];
  uint32_t cone_ands;
  uint32_t num_slots;
  uint32_t out_slot;
  uint32_t out_compl;
  uint32_t order;
  uint64_t num_records;     /* written even when cap is too small */
  uint64_t hash;            /* structural hash of the program */
  uint32_t num_luts;        /* 3-input tables covering the cone (JIT instructions) */
  uint32_t lut_live;        /* peak live values when evaluating the tables */
  double lop3_per_pass;     /* plan_info of a specialised-kernel plan: lop3 the kernel executes per
                               32-pattern chunk and thread (tables once per loop level that needs them,
                               folded copies); 0 otherwise or when unknown */
  uint32_t interp_step;     /* AND records the interpreter may evaluate at once without forwarding:
                               4 when no AND reads one of the 3 ANDs before it without a load record
                               between (cones of 256+ ANDs that need at most one run-break load per
                               16 ANDs), else 1 */
  uint32_t pad;
} lec_es_program_info;

/* ---- context ---------------------------------------------------------- */

/* Creates a context on cfg->device.  Errors: EINVAL (NULL args, max_pis >
 * 63), ECUDA (device not usable), ENOMEM. */
int lec_es_create(lec_es_ctx **out, const lec_es_config *cfg);
/* Frees everything the ctx owns (not a caller-provided arena or stream).
 * Outstanding submitted requests are cancelled first.  Must not run
 * concurrently with any other call on the same ctx. */
void lec_es_destroy(lec_es_ctx *c);
const char *lec_es_strerror(int status);

/* ---- front end (host only) ------------------------------------------- */

/* Cone extraction, support, evaluation order and reference-count slot
 * assignment (§3.3) without touching a GPU.  Writes min(cap, needed)
 * records; info->num_records is the needed count.  Errors: EINVAL
 * (malformed cone), ETOOBIG (n > 63 or > 65535 slots). */
int lec_es_compile(const lec_es_miter *m, uint32_t order, lec_es_program_info *info,
                   uint64_t *records, uint64_t cap);

/* Generate the specialised straight-line kernel for m and compile it with
 * NVRTC for compute capability cc_major.cc_minor ("a" target), without
 * loading it (no GPU needed).  log receives NVRTC's log, including ptxas'
 * register and spill counts; *cubin_bytes the image size.  Errors: EINVAL,
 * ETOOBIG, EJIT. */
int lec_es_jit_compile(const lec_es_miter *m, int cc_major, int cc_minor, char *log, size_t log_cap,
                       uint64_t *cubin_bytes);

/* ---- single miter ----------------------------------------------------- */

/* Full ES of one miter, synchronous on the ctx stream: the problem of
 * paper §2.1 (is the miter output constant 0?) decided by exact simulation
 * as §2.2 defines it (every assignment of the output's PI support), with the
 * cone compiled to a reference-counted instruction stream (§3.3).  m and its
 * fanins are read during the call only; *out is written on LEC_ES_OK:
 * verdict EQUIVALENT or NONEQUIVALENT with the lowest failing pattern.
 * Tier (AUTO): the ES time model's choice (§3.2, refit), except that a check
 * never waits for a kernel build -- a cone whose specialised kernel would
 * pay off but is not built yet starts on the interpreter in ascending word
 * slices while the kernel builds in the background; a failing slice ends
 * the check, and once the kernel lands it takes the rest of the range.
 * out->tier is the tier that finished the check.
 * Errors: EINVAL (NULL or malformed graph), ETOOBIG (n > max_pis or more
 * than 65535 value slots), ENOMEM, ECUDA, EJIT, EDEVICE_WAIT, ETIMEOUT. */
int lec_es_check(lec_es_ctx *c, const lec_es_miter *m, lec_es_result *out);
/* As lec_es_check over a word sub-range and with explicit options; a
 * passing proper sub-range gives LEC_ES_UNDECIDED. */
int lec_es_check_ex(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt,
                    lec_es_result *out);

/* Compile a miter and keep its program resident on the device (the host
 * copy of m may be freed afterwards).  opt may be NULL. */
int lec_es_prepare(lec_es_ctx *c, const lec_es_miter *m, const lec_es_options *opt,
                   lec_es_plan **out);
/* Enqueue one ES pass of a prepared plan on the ctx stream and return at
 * once (result reset, kernel, 8-byte result copy).  opt may be NULL. */
int lec_es_run_async(lec_es_ctx *c, lec_es_plan *p, const lec_es_options *opt);
/* Wait for the last run of the plan and fill *out. */
int lec_es_plan_result(lec_es_ctx *c, lec_es_plan *p, lec_es_result *out);
/* Program description of a prepared plan (host memory only). */
int lec_es_plan_info(const lec_es_plan *p, lec_es_program_info *info);
void lec_es_plan_free(lec_es_ctx *c, lec_es_plan *p);

/* Per-node values for small cones: row j of host_out (words_per_row words)
 * holds the value of the j-th cone AND in ascending variable order, over words
 * [word_begin, word_end); vars_out[j] (host, cone_ands entries) receives that
 * variable.  Uses the interpreter kernel with an extra store per AND.
 * Errors: EINVAL if the range is empty or outside the cone's words. */
int lec_es_truth_tables(lec_es_ctx *c, const lec_es_miter *m, uint64_t word_begin,
                        uint64_t word_end, uint32_t *vars_out, uint64_t *host_out);

/* Per-node values from a chosen kernel tier, for checking the kernels that
 * carry the work node by node (paper §3.3: every register of the
 * instruction stream holds one node's value over the current patterns).
 * Same row layout as lec_es_truth_tables:
 *   tier       LEC_ES_TIER_SPILL: the chunk interpreter (lec_es_truth_tables);
 *              LEC_ES_TIER_INTERP: the word interpreter with its value slots
 *              in shared memory, a store after every AND record (all rows);
 *              LEC_ES_TIER_JIT: the specialised kernel in the layout it runs
 *              in (its dump variant: the same generated code plus a store of
 *              every 3-input table's value where the layout computes it,
 *              built for this call; the context's kernel is built first if
 *              it holds none) -- the rows of the nodes the tables compute;
 *   vars_out   host, cone_ands entries: row j's AND variable (ascending);
 *   row_valid  host, cone_ands bytes, or NULL: 1 where row j was written;
 *   host_out   host, cone_ands x (word_end - word_begin) words; JIT rows
 *              that no table computes are zero.
 * The JIT dump holds tables x 2^max(n-5, 5) x 4 bytes of the arena during
 * the call.  Errors: EINVAL (bad tier, empty range or outside the cone's
 * words), ETOOBIG (INTERP: the live set does not fit shared memory),
 * ENOMEM, ECUDA, EJIT. */
int lec_es_truth_tables_ex(lec_es_ctx *c, const lec_es_miter *m, uint64_t word_begin, uint64_t word_end,
                           uint32_t tier, uint32_t *vars_out, uint8_t *row_valid, uint64_t *host_out);

/* For callers that cannot allocate device memory (a framework's caching
 * allocator owns it all, or a service may not allocate after start-up).
 * The paper has no counterpart: it is a deployment variant of the
 * global-memory interpreter.  ES of one program compiled by lec_es_compile
 * whose records the caller has copied to device memory:
 *   d_records         device, 16-byte aligned, records_capacity >= num_records
 *                     rounded up to even (the copy engine moves 16-byte pairs);
 *   prog              the lec_es_program_info lec_es_compile returned;
 *   word_begin/end    64-pattern word range (word_end clipped to the cone's);
 *   d_result          device, 4 x u64 written by the call: [0] lowest failing
 *                     pattern or UINT64_MAX, [1] patterns evaluated,
 *                     [2] status (0 ok, 1 a bounded device wait gave up), [3] unused;
 *   stream            cudaStream_t; the call enqueues and returns at once.
 * The value slots live in a fixed 16 MiB device array that every GPU using
 * the library holds until exit; live sets with num_slots * 32 * 4 bytes above
 * that are rejected with LEC_ES_ETOOBIG.  The first call on a device looks up
 * the array's address (make it before any stream capture).  No cudaMalloc,
 * cudaFree or other allocating call is made.  All calls share the array:
 * calls whose kernels overlap on the GPU race and must be serialised.
 * Errors: EINVAL (NULL, misaligned or short buffers, bad program info,
 * empty range), ETOOBIG, ECUDA. */
int lec_es_check_noalloc(const uint64_t *d_records, uint64_t records_capacity,
                         const lec_es_program_info *prog, uint64_t word_begin, uint64_t word_end,
                         unsigned long long *d_result, void *stream);

/* ---- batch: many miters, one persistent launch ------------------------- */

/* ES of many sub-miters at once: the per-pair sub-miters a sweeping
 * scheduler hands to ES (paper §3.2, local sub-miters of candidate pairs;
 * ES cost linear in gates and exponential in PIs), each decided as in
 * lec_es_check (§2.1, §2.2, §3.3).  m[0..k-1] (host; they may share one
 * fanins array) are read during the call only; out[0..k-1] (caller-owned)
 * receive results identical to lec_es_check on each m[i].  Heavy miters run
 * as their own specialised kernels and light ones in one persistent launch
 * over a queue of (miter, word range) tiles, all in one CUDA graph.
 * Errors: as lec_es_check for any miter (the whole call fails; out is then
 * unspecified), EINVAL for k = 0. */
int lec_es_batch(lec_es_ctx *c, const lec_es_miter *m, size_t k, lec_es_result *out);
/* Prepared form: compile and upload k miters once, then run repeatedly
 * (the launch sequence is captured in a CUDA graph and replayed). */
int lec_es_batch_prepare(lec_es_ctx *c, const lec_es_miter *m, size_t k,
                         const lec_es_options *opt, lec_es_batch_plan **out);
/* Layout a prepared batch ended up with. */
typedef struct {
  uint32_t miters;          /* k */
  uint32_t jit_miters;      /* run by their own specialised kernel */
  uint32_t tile_miters;     /* run by the persistent tile-queue kernel */
  uint32_t fallback_miters; /* live set beyond shared memory: global-memory plans */
  uint32_t tiles;           /* (miter, chunk range) tiles in the queue */
  uint32_t block_threads;   /* threads per tile pass */
  uint32_t stage_records;   /* records per staging stage */
  uint32_t tile_granularity;/* tiles per resident block slot */
  uint32_t grid_blocks;     /* persistent blocks */
  double prepare_ms;        /* whole preparation */
  double jit_ms;            /* of which compiling specialised kernels */
  double tune_ms;           /* of which timing candidate layouts */
} lec_es_batch_layout;
int lec_es_batch_info(const lec_es_batch_plan *b, lec_es_batch_layout *info);
int lec_es_batch_run_async(lec_es_ctx *c, lec_es_batch_plan *b);
int lec_es_batch_results(lec_es_ctx *c, lec_es_batch_plan *b, lec_es_result *out, size_t k);
void lec_es_batch_free(lec_es_ctx *c, lec_es_batch_plan *b);

/* ---- serving: asynchronous requests, continuous batching ----------------- */

/* Admit one ES request (the problem of paper §2.1 decided as in §2.2 and
 * §3.3, like lec_es_check) and return a ticket at once; requests that
 * arrive while others run are admitted as device memory and result slots
 * free up, and their kernels overlap on the GPU (continuous batching).  The
 * miter's output cone is copied before the call returns (so the caller may
 * free m at once) and compiled by the server's front-end threads.  The
 * result, identical to lec_es_check on m, comes from lec_es_poll /
 * lec_es_wait.  Thread-safe.
 * Errors: EINVAL (malformed cone), ETOOBIG (n > max_pis), ENOMEM; an error
 * the front end finds later (more than 65535 value slots) is returned by
 * lec_es_poll / lec_es_wait for the ticket. */
int lec_es_submit(lec_es_ctx *c, const lec_es_miter *m, uint64_t *ticket);
/* lec_es_submit for k miters in one call (m[0..k-1], host; they may share
 * one fanins array): every cone is copied before any request is queued, so
 * on an error nothing is submitted; tickets (host, k entries) receive the
 * tickets in order.  Thread-safe.  Errors: as lec_es_submit for any miter;
 * EINVAL for NULL arrays with k > 0. */
int lec_es_submit_many(lec_es_ctx *c, const lec_es_miter *m, size_t k, uint64_t *tickets);
/* EBUSY while the request runs; OK and *out once done (the ticket is then
 * released); ECANCELLED if cancelled; ENOTFOUND for an unknown ticket. */
int lec_es_poll(lec_es_ctx *c, uint64_t ticket, lec_es_result *out);
/* Blocks until done or timeout_s passes (ETIMEOUT). */
int lec_es_wait(lec_es_ctx *c, uint64_t ticket, double timeout_s, lec_es_result *out);
/* Cancels a queued or running request (a running one stops at its next tile). */
int lec_es_cancel(lec_es_ctx *c, uint64_t ticket);
/* Serving limits: bytes of device memory the admitted requests may hold
 * (value slots x resident words x 8 B, plus programs) and the number of
 * requests in flight.  Call before the first submit. */
int lec_es_server_config(lec_es_ctx *c, size_t slot_budget_bytes, uint32_t max_inflight);

/* ---- sweeping step (1): random simulation and candidate pairs ------------ */

/* Simulate the whole graph on caller-drawn random words (sweeping flow step
 * (1), §2.3) on the device.  pi_words: host, num_pis x nwords words (row k =
 * PI k).  hash_out: host, num_pis+num_ands+1 words, a 64-bit hash of every
 * variable's signature (equal signatures give equal hashes).  sigs_out: host,
 * (num_pis+num_ands+1) x nwords words, or NULL.  Errors: EINVAL (a fanin not
 * below its AND, NULL arrays), ENOMEM (arena), ECUDA. */
int lec_es_signatures(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                      const uint64_t *pi_words, uint32_t nwords, uint64_t *sigs_out, uint64_t *hash_out);
/* Potentially-equivalent node pairs from those signatures: AND nodes with
 * identical (not complemented) signatures form classes, constant signatures
 * are dropped, every member is paired with its class's lowest variable, and a
 * pair is kept if the union of the two PI supports has at most max_support
 * PIs (num_pis <= 64).  pairs (host, 2*cap): (representative, member)
 * variables, ascending; *npairs = total found (may exceed cap). */
int lec_es_match_pairs(lec_es_ctx *c, uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                       const uint64_t *pi_words, uint32_t nwords, uint32_t max_support, uint32_t *pairs,
                       uint64_t cap, uint64_t *npairs);

/* ---- device facts ----------------------------------------------------- */

/* Measured 32-bit LOP3 throughput: results per clock per SM, from a
 * dependent-chain-free microbenchmark timed with CUDA events; also SM count
 * and the SM clock (kHz) read during the run. */
int lec_es_lop3_peak(lec_es_ctx *c, double *lop3_per_clk_per_sm, int *sm_count,
                     int *clock_khz, double *lop3_per_s);

/* ---- sweeping with ES as the engine (§2.3, §3.2) ------------------------ */

typedef struct {
  uint32_t sim_words;       /* 64-pattern random-simulation words per round (0 = 64) */
  uint32_t max_rounds;      /* (0 = 512) */
  uint32_t max_leaves;      /* free inputs of a local sub-miter (0 = 16, at most 40) */
  uint32_t max_nodes;       /* ANDs of a local sub-miter (0 = 128) */
  uint32_t final_max_pis;   /* run the output's own ES check if its support is at most this (0 = 36, <= 63) */
  uint32_t pad;
  uint64_t seed;            /* random simulation seed */
} lec_es_sweep_options;

typedef struct {
  lec_es_verdict verdict;   /* UNDECIDED if neither merging, simulation nor the final check decides */
  uint32_t rounds;
  uint64_t pairs_checked;   /* local sub-miters checked by ES */
  uint64_t pairs_proven;    /* of which EQUIVALENT (merged) */
  uint64_t pairs_refuted;   /* of which a counterexample with free cut inputs (left unmerged) */
  uint64_t pairs_skipped;   /* candidate pairs over the leaf or node limit */
  uint32_t ands_initial, ands_final;   /* ANDs of the output's cone before and after */
  uint32_t final_support;   /* PIs of the output's remaining cone */
  uint32_t decided_by;      /* 0 the output became a constant, 1 random simulation, 2 the final ES check, 3 undecided */
  double sim_ms, es_ms, host_ms, total_ms;
  uint32_t rounds_reused;   /* rounds that checked the previous round's uncut candidates without
                               simulating again (it had refuted at most a tenth of its pairs) */
  uint32_t pad;
} lec_es_sweep_result;

/* Sweep a miter (no counterpart entry point in the paper; its flow, §2.3,
 * with ES as the checking engine and local sub-miters as in §3.2): rounds of
 * GPU random simulation, candidate pairs (equal signatures up to
 * complement), local sub-miters whose inputs are the points where the two
 * cones meet (an EQUIVALENT result is a proof; a counterexample with free
 * inputs only leaves the pair unmerged), one batched ES launch per round,
 * and merging with structural hashing.  The miter may have any number of
 * PIs; the output's own ES check (final_max_pis) runs when merging stops
 * short of a constant.
 * cex_bits (optional, (num_pis + 63) / 64 words): for NONEQUIVALENT, a
 *   failing input assignment, bit i = PI i (0-based); not necessarily the
 *   lowest one unless decided_by = 2.
 * merges (optional, 3 * merges_cap words): (member, representative, phase)
 *   variables of the input AIG proven equal (member == representative XOR
 *   phase) by the local checks, in the order proven; *nmerges = total (may
 *   exceed merges_cap).
 * Errors: EINVAL (malformed AIG), ENOMEM, ECUDA. */
int lec_es_sweep(lec_es_ctx *c, const lec_es_miter *m, const lec_es_sweep_options *opt,
                 lec_es_sweep_result *out, uint64_t *cex_bits, uint32_t *merges, uint64_t merges_cap,
                 uint64_t *nmerges);

/* ---- ES time model (§3.2, refit for this GPU) --------------------------- */

/* The paper models ES time as alpha * gates * 2^(n - beta).  alpha * 2^-beta
 * is one factor, so beta stays at the paper's 23 and each tier gets its own
 * alpha, plus a fixed launch cost a and a cost c per gate for one pass over
 * the program (the floor of a small support on a GPU):
 *   t_ms = a_ms + c_ms * gates + alpha_ms * gates * 2^(n - 23),
 * gates = cone ANDs, n = support PIs.  Build time of a specialised kernel:
 * a_ms + c_ms * tables (alpha_ms = 0).  Once a context holds a cone's
 * kernel, its predicted time follows what that kernel executes instead of
 * the gates (hoisting and folded pass PIs make the two differ by up to 4x):
 *   t_ms = a_ms + c_ms * gates + alpha_ms * (lop3_per_pass + 40) * 2^(n - 23),
 * lop3_per_pass as in lec_es_program_info and 40 the per-pass overhead of
 * the kernel's loop and result check in lop3-equivalents (fitted on B300). */
typedef struct {
  double a_ms;              /* fixed cost per run (ms) */
  double c_ms;              /* ms per gate, independent of n */
  double alpha_ms;          /* ms per gate at 2^23 patterns (the paper's alpha, in ms) */
  uint64_t samples;         /* measurements folded in (0: built-in B300 values) */
} lec_es_cost_coeffs;

typedef struct {
  double interp_ms;         /* predicted device time on the interpreter tier */
  double jit_ms;            /* predicted device time of the specialised kernel (by its
                               executed lop3 when the context holds it, else by gates) */
  double jit_compile_ms;    /* predicted build time (0 if the context holds the kernel) */
  double paper_cpu_s;       /* the paper's one-core CPU model: 0.0003 s * gates * 2^(n-23) */
  uint32_t gates, n, num_luts;
  uint32_t tier;            /* tier an AUTO check starts on (LEC_ES_TIER_*): the kernel only
                               if the context holds it; a cone whose kernel would pay off
                               but is not built starts on the interpreter while the kernel
                               builds in the background, and the check's result reports
                               LEC_ES_TIER_JIT if the kernel took over */
  uint32_t gpu_offload;     /* the paper's rule: 1 if paper_cpu_s / cpu_threads > 0.1 s */
  uint32_t pad;
} lec_es_cost;

/* Weighted least-squares fit (relative error; a_ms, c_ms, alpha_ms >= 0) of
 * k measurements (gates[i], n[i], ms[i]) to the model above.  Host only.
 * EINVAL on k = 0, n > 63 or a time <= 0. */
int lec_es_cost_fit(const uint32_t *gates, const uint32_t *n, const double *ms, size_t k,
                    lec_es_cost_coeffs *out);
/* The context's current coefficients for tier (LEC_ES_TIER_INTERP, _JIT,
 * _SPILL), 4 for kernel builds or 5 for the specialised kernel's time by
 * its executed lop3 (the second form above).  Each context starts from
 * built-in B300 values and folds in its own full, equivalent runs (single
 * checks and served requests) and kernel builds.  c may be NULL: built-in
 * values. */
int lec_es_cost_model(lec_es_ctx *c, uint32_t tier, lec_es_cost_coeffs *out);
/* Predicted times of miter m (front end on the host; nothing runs on the
 * GPU) and the tier an AUTO check would take.  c may be NULL: built-in
 * values, no kernel cache.  cpu_threads is the thread count for the paper's
 * GPU-offload rule. */
int lec_es_cost_predict(lec_es_ctx *c, const lec_es_miter *m, uint32_t cpu_threads, lec_es_cost *out);

/* Version of the specialised-kernel code generator (no counterpart in the
 * paper).  It changes whenever the generated kernel's code or interface
 * does, is part of the on-disk kernel cache names, and lets a caller tell
 * whether a profile of a kernel still describes the one this library emits.
 * Never fails. */
uint32_t lec_es_codegen_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LEC_ES_H */
