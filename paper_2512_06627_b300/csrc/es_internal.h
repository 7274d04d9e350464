// es_internal.h -- types shared by the front end, the kernels and the C ABI.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace lec {

// One instruction of the slot program (8 bytes, 16-byte aligned pairs for TMA).
//   op 0..3 : slot[dst] = (slot[a] ^ (op&1 ? ~0 : 0)) & (slot[b] ^ (op&2 ? ~0 : 0))
//   op 4    : slot[dst] = value of support PI a for the current patterns
//   op 5    : slot[dst] = 0
struct Rec {
  uint16_t dst, a, b;
  uint8_t op, pad;
};
static_assert(sizeof(Rec) == 8, "record is 8 bytes");

enum : uint8_t { OP_AND = 0, OP_PI = 4, OP_CONST0 = 5 };
// Rec.pad of a load of the constant into a free slot that only ends a run of
// AND records (see Program::step).
constexpr uint8_t kRecBreak = 1;

// Cover of a cone by 3-input lookup tables (lutmap.cpp).  Value ids: ANDs
// 0..NA-1 (ascending variable), support PIs NA..NA+n-1, the constant NA+n.
struct LutCover {
  struct Lut {
    int32_t node;      // the AND whose function the table computes
    uint8_t n;         // leaves used (0..3)
    int32_t leaf[3];   // value ids, ascending; -1 if unused
    uint8_t tt;        // truth table, leaf i = x_i with x0 = 0xAA, x1 = 0xCC, x2 = 0xF0
  };
  std::vector<Lut> luts;       // ascending node order
  std::vector<int32_t> index;  // AND id -> position in luts, or -1
};

void lut_map(size_t NA, size_t NP, const std::vector<int64_t> &f0, const std::vector<int64_t> &f1,
             const std::vector<uint8_t> &c0, const std::vector<uint8_t> &c1, int64_t root, LutCover &out);

// LUT program: tables in evaluation order over value ids (see LutCover).
struct LutProgram {
  uint32_t na = 0;                       // ANDs of the cone (value ids below this are ANDs)
  uint32_t np = 0;                       // support PIs
  std::vector<LutCover::Lut> order;      // evaluation order (topological)
  int64_t root = -1;                     // value id of the output's node
  uint32_t live = 0;                     // peak number of live values in this order
  uint32_t count = 0;                    // tables in the cover (order.size() unless elided)
  bool elided = false;                   // cover not built: the specialised kernel exists
  bool deferred = false;                 // cover not built: a background build makes it from the cone
};

// Compiled cone (paper §3.3 "Instructionalized ES"): branch-free instruction
// stream over value slots reused by reference count.
struct Program {
  uint32_t n = 0;                   // support size
  std::vector<uint32_t> support;    // original PI indices (0-based), ascending
  std::vector<uint32_t> order_vars; // cone AND variables in evaluation order
  std::vector<Rec> recs;
  uint32_t num_slots = 0;
  uint32_t out_slot = 0;
  uint32_t out_compl = 0;
  uint32_t cone_ands = 0;
  uint32_t order = 0;
  uint64_t hash = 0;                // of the cone's structure (dense ids, complements, output, n)
  uint64_t hash2 = 0;               // a second, independent hash of the same structure: a cached
                                    // kernel or resident program is used only when both match
  LutProgram lut;                   // 3-input table cover (the JIT tier's instructions)
  bool slots_elided = false;        // recs/order_vars not built: the specialised kernel runs this cone
  uint32_t num_records = 0;         // recs.size(), or the kernel's record count when elided
  uint32_t step = 1;                // kInterpStep: no AND reads one of the kInterpStep - 1 ANDs
                                    // before it without a load between (records with pad =
                                    // kRecBreak are such loads); 1: no such rule
};

struct MiterView {
  uint32_t num_pis, num_ands;
  const uint32_t *fanins;
  uint32_t out_lit;
};

// A miter's output cone as a self-contained AIG: its support PIs renumbered
// 1..n in ascending order, its ANDs after them in ascending order, so a
// request can keep the cone (not the caller's whole graph) until its front
// end runs.  compile_program on view() gives the program of the original
// miter (same structure and hashes) except its support, which is `support`.
struct CompactMiter {
  uint32_t num_pis = 0;
  std::vector<uint32_t> fanins;    // 2 literals per AND
  uint32_t out_lit = 0;
  std::vector<uint32_t> support;   // original PI index (0-based) of compact PI k + 1
  MiterView view() const { return MiterView{num_pis, (uint32_t)(fanins.size() / 2), fanins.data(), out_lit}; }
};
// Errors: EINVAL (malformed cone), ETOOBIG (more than max_pis support PIs).
int compact_cone(const MiterView &m, uint32_t max_pis, CompactMiter &out);

// Front end.  Returns an lec_es_status code.
// The program hash depends only on the cone's structure, so it is known right
// after the cone is extracted.  The table cover only feeds code generation
// for the specialised kernel, and the slot program only the interpreter
// tiers.  A caller that already holds the cone's kernel and will run it can
// pass a probe: when have_kernel returns true (filling in what the kernel
// was built from), neither is rebuilt -- the LutProgram is marked elided and
// so is the slot program (no records; slot and record counts come from the
// kernel).
struct KernelFacts {
  uint32_t luts = 0, live = 0;      // table count and live count
  uint32_t num_slots = 0, order = 0, num_records = 0;
};
struct KernelProbe {
  bool (*have_kernel)(void *arg, uint64_t hash, uint64_t hash2, uint32_t n, uint32_t cone_ands, KernelFacts *facts);
  void *arg;
  // optional: whether the caller may build this cone's specialised kernel at
  // all; if not, the table cover (which only feeds code generation, and is
  // most of the front end's time on small cones) is not built: lut.count = 0
  bool (*want_cover)(void *arg, uint32_t n, uint32_t cone_ands) = nullptr;
};

int compile_program(const MiterView &m, uint32_t order, uint32_t max_pis, Program &out,
                    const KernelProbe *probe = nullptr);

// Tables of the specialised kernel evaluated once per grab (hoist.cpp):
// hoisted[i] for lp.order[i]; the support PIs in the mask pass_pis change
// from pass to pass; at most `budget` hoisted values are read by per-pass
// code.
void plan_hoist(const LutProgram &lp, uint64_t pass_pis, uint32_t budget, std::vector<uint8_t> &hoisted,
                uint32_t *roots);
// The same, growing a fanin-closed base set (kept whole); the base's values
// read outside it count against the budget too.
void plan_hoist_from(const LutProgram &lp, uint64_t pass_pis, uint32_t budget, const std::vector<uint8_t> &base,
                     std::vector<uint8_t> &hoisted, uint32_t *roots);
// The k support PIs (index >= 10) that the fewest tables depend on, as a mask.
uint64_t least_influential_pis(const LutProgram &lp, uint32_t k);
// The support PIs (bit k: support PI k, k < 64) each table of lp.order depends on.
std::vector<uint64_t> table_support(const LutProgram &lp);
// Nested pass loops: the pass PIs split into at most four groups, outermost
// loop first, chosen to minimise table evaluations per grab, each extra loop
// level charged 3%.  mode 0: one loop; 1: chosen; 2: chosen among two levels or
// more; 3: one loop per pass PI.  *score: the chosen nesting's table
// evaluations per grab (with the level charge; for modes 0 and 3, those of
// one loop).
std::vector<uint64_t> choose_pass_groups(const LutProgram &lp, uint64_t pass_pis, int mode,
                                         double *score = nullptr);

// Words of 64 patterns for a support of n PIs.
inline uint64_t num_words(uint32_t n) { return n <= 6 ? 1ull : (1ull << (n - 6)); }
// 32-pattern chunks (the kernels' unit: one 32-bit lane per thread).
inline uint64_t num_chunks(uint32_t n) { return n <= 5 ? 1ull : (1ull << (n - 5)); }

// ---- kernel parameter blocks (passed by value) --------------------------------

struct InterpParams {
  const Rec *recs;          // device, padded to an even count, 16-byte aligned
  uint32_t nrec;            // records to execute
  uint32_t nrec_padded;     // even
  uint32_t nslots;
  uint32_t out_slot;
  uint32_t out_compl;
  uint32_t n;               // support size
  uint32_t ring_recs;       // records per staging stage (multiple of 2)
  uint32_t resident;        // 1: whole program staged once
  uint64_t chunk_begin;     // 32-pattern chunks [begin, end)
  uint64_t chunk_end;
  unsigned long long *cex;  // device, initialised to ~0
  unsigned long long *evaluated; // device: patterns evaluated
  uint32_t *status;         // device error word (0 = ok)
  uint32_t *spill;          // global value slots for the spill tier
  uint64_t *tt_out;         // truth-table dump: [cone AND][word] (optional)
  const uint32_t *tt_row;   // record index -> dump row (or 0xffffffff)
  uint64_t tt_words;        // words per dump row
  uint64_t tt_word_begin;
  uint32_t extra_tx;        // test hook: bytes expected beyond the record copy (0 normally)
};

// ---- lane-wide interpreter (interp_w.cu) -------------------------------------
// Patterns per thread of the interpreter: 64 (a word as two 32-bit halves)
// or 32 (one chunk); slots are that many bits wide.
#ifndef LEC_ES_INTERP_LANE
#define LEC_ES_INTERP_LANE 64
#endif
static_assert(LEC_ES_INTERP_LANE == 32 || LEC_ES_INTERP_LANE == 64, "interpreter lane: 32 or 64 patterns");
constexpr uint32_t kLaneBytes = LEC_ES_INTERP_LANE / 8;
// AND records the interpreter evaluates together (operand loads of a step
// issued before any of its stores) in a program whose step is kInterpStep:
// no AND there reads one of the kInterpStep - 1 ANDs before it without a
// load record between.  Other programs run kFwdStep records per step, an
// operand written within the step taken from the writer's register.
#ifndef LEC_ES_INTERP_STEP
#define LEC_ES_INTERP_STEP 4
#endif
constexpr int kInterpStep = LEC_ES_INTERP_STEP;
constexpr int kFwdStep = 2;
// Cones of at least this many ANDs get kInterpStep programs, unless they
// would need more than one run-break load per kMaxBreakShare ANDs.
constexpr uint32_t kStepMinAnds = 256;
constexpr size_t kMaxBreakShare = 16;
// Records pre-decoded for one block size T: byte offsets slot * T * kLaneBytes
// of the two operand slots and the result slot; ctl bit 0/1 complement
// operand a/b; bits 2.. the truth-table row + 1 (dump only).
constexpr uint32_t kCtlRowShift = 2;
struct XRec {
  uint32_t a_off, b_off, d_off, ctl;
};
// A PI (k < 63) or constant (k = 63) load into d_off before AND record `at`.
struct XLoad {
  uint32_t at, d_off, k, pad;
};
static_assert(sizeof(XLoad) == 16, "the kernels read a load as one 16-byte vector");
struct XParams {
  const XRec *recs;
  const XLoad *loads;
  uint32_t nrec, nload;
  uint32_t step;            // Program::step of the encoded program
  uint32_t out_off, out_compl, n;
  uint32_t ring_recs, resident, extra_tx;
  uint64_t word_begin, word_end;  // 64-pattern words
  unsigned long long *cex;
  unsigned long long *evaluated;
  uint32_t *status;
  uint64_t *tt_out;    // truth-table dump only: rows of tt_words words (see interp_w.cu)
  uint64_t tt_words;
};
struct XMiter {
  uint32_t rec_off, nrec, load_off, nload, out_off, out_compl, n, pad;
};
struct XTile {
  uint32_t miter, pad;
  uint64_t word_begin, word_end;
};
struct XBatchParams {
  const XRec *recs;
  const XLoad *loads;
  const XMiter *miters;
  const XTile *tiles;
  uint32_t num_tiles, ring_recs;
  unsigned long long *cex;
  unsigned int *head;
  uint32_t *status;
  const volatile uint32_t *cancel;
};

// Encode a slot program for the word-wide kernels at block size `block`.
// Run-break loads (kRecBreak) are kept when `breaks` (kernels that rely on
// Program::step) and dropped otherwise (forwarding kernels).
void encode_w(const Program &g, int block, std::vector<XRec> &recs, std::vector<XLoad> &loads, uint32_t &out_off,
              bool breaks = true);
// Threads per block of the word-wide kernels: any multiple of 32 up to
// kMaxWordBlock (the record offsets are encoded for the block's size, so the
// block need not be a power of two; wider blocks put more warps on an SM
// whose shared memory one 256-thread block of a large live set leaves half
// empty).
constexpr int kMaxWordBlock = 512;
inline bool word_block_ok(int b) { return b >= 32 && b <= kMaxWordBlock && b % 32 == 0; }
// Shared memory of the single-miter word kernel: the whole record stream
// resident when it fits (and `allow_resident`), else a 4-stage ring.
size_t interp_w_smem_bytes(uint32_t nslots, uint32_t nrec, int block, uint32_t *ring_recs, uint32_t *resident,
                           bool allow_resident = true);
// Warps per SM that blocks of `block` threads holding `bytes` of shared
// memory each keep resident (228 KB per SM, 1 KB reserved per block, at most
// 64 warps).
inline int word_warps_per_sm(size_t bytes, int block) {
  const size_t per_sm = 228u * 1024u;
  const int bps = (int)(per_sm / (bytes + 1024));
  return (bps < 2048 / block ? bps : 2048 / block) * block / 32;
}
size_t batch_w_smem_bytes(uint32_t max_slots, int block, uint32_t ring_recs);
int launch_interp_w(const XParams &p, int block, int grid, size_t smem, void *stream);
// The same kernel with per-record truth-table stores (interp_w.cu, TTSink).
int launch_interp_w_tt(const XParams &p, int block, int grid, size_t smem, void *stream);
int configure_batch_w(int block, size_t smem);
int batch_w_blocks_per_sm(int block, size_t smem);
int launch_batch_w(const XBatchParams &p, int block, int grid, size_t smem, void *stream);

// Status bits written by kernels.
enum : uint32_t {
  DEV_OK = 0,
  DEV_WAIT_TIMEOUT = 1u,    // an mbarrier wait exceeded its iteration bound
  DEV_BAD_PROGRAM = 2u,     // slot index out of range (host bug guard)
};

// Kernel launchers (kernels.cu).  Return cudaError_t as int.
int launch_interp(const InterpParams &p, int block, int grid, size_t smem, bool spill, void *stream);
int interp_smem_bytes(uint32_t nslots, uint32_t nrec_padded, int block, uint32_t *ring_recs,
                      uint32_t *resident, size_t *bytes);
int launch_lop3_bench(uint32_t *out, unsigned long long *cycles, int grid, int block, int iters,
                      void *stream);
int max_smem_optin(int device);
int set_kernel_smem_limits(size_t bytes);

}  // namespace lec
