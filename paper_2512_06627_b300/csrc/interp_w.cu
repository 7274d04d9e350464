// interp_w.cu -- lane-wide interpreter: one lane of patterns per thread,
// pre-decoded records.
//
// The generic tier for cones without a specialised kernel.  Each thread holds
// the value slots of one lane of patterns and evaluates each AND as one LOP3
// per 32 patterns.  The lane is fixed at build time (LEC_ES_INTERP_LANE):
// 64 -- one 64-pattern word as two 32-bit halves (uint2, so a slot access is
// one 8-byte shared-memory operation); 32 -- one 32-pattern chunk (4-byte
// slots, so the same shared memory holds twice the threads).  The record
// stream is prepared on the host for the launch's block size:
//   record  {a_off, b_off, d_off, ctl}: byte offsets of the two operand slots
//           and the result slot from the thread's slot base, complement bits
//           in ctl (bit 0: a, bit 1: b), turned into all-zero/all-one masks
//           with one bit-field extract each -- no branch, no address math;
//   loads   PI and constant loads live in a separate list {before record i,
//           d_off, k}, consumed between runs of AND records, so the record
//           loop has no kind test.
// Records are staged global->shared by the bulk-copy engine (whole program
// when it fits, else a 4-stage ring) and read warp-uniformly.  Both the
// single-miter kernel and the tile-queue batch kernel use this scheme.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "es_internal.h"

namespace lec {
namespace {

constexpr int NSTAGE = 4;
// AND records per interpreter step.  Measured on B300 (12x12 miter, 16x16
// miter, 3,630 light node-pair miters in one tile queue) with forwarding in
// every step: 1 -> 1.11 / 596 / 1.45 ms, 2 -> 0.90 / 427 / 1.42 ms, 3 ->
// 1.17 / 515 / 1.45 ms, 4 -> 1.08 / 525 / 1.61 ms, 8 -> 1.39 / 699 / 2.12 ms;
// without forwarding, on programs whose ANDs never read one of the K - 1
// before them in a run: 2 -> 0.91 / 415 / 1.57 ms, 3 -> 0.82 / 383 / 1.65
// ms, 4 -> 0.78 / 362 / 1.70 ms (the node pairs' small cones need many run
// breaks, so the tile queue keeps forwarding, kFwdStep = 2, and only cones of
// kStepMinAnds ANDs or more get step-kInterpStep programs).
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr uint64_t kWaitNs = 1000000000ull;

__constant__ uint32_t kMaskW[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void expect_and_copy(uint64_t *bar, void *dst, const void *src, uint32_t bytes,
                                                uint32_t extra) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes + extra)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after 1 s of global time (or kWaitLimit polls).
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity) {
  if (try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kWaitLimit; i++) {
    if (try_wait(bar, parity)) return true;
    if ((i & 15u) == 15u && global_ns() - t0 > kWaitNs) return false;
    if (i > 64) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void drain(uint64_t *bar, uint32_t inflight, uint32_t parity) {
  if (threadIdx.x != 0) return;
  for (int s = 0; s < NSTAGE; s++)
    if ((inflight >> s) & 1u) (void)wait(bar + s, (parity >> s) & 1u);
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// The thread's lane: a 64-pattern word (two halves) or a 32-pattern chunk.
using Lane = std::conditional<kLaneBytes == 8, uint2, uint32_t>::type;
constexpr uint32_t kLanePatterns = kLaneBytes * 8;

// Support PI k for 64-pattern word w, as (low half, high half).
__device__ __forceinline__ uint2 pi_lane(uint32_t k, uint64_t w, uint2) {
  if (k < 5) return make_uint2(kMaskW[k], kMaskW[k]);
  if (k == 5) return make_uint2(0u, 0xFFFFFFFFu);
  if (k == 63) return make_uint2(0u, 0u);  // the constant
  const uint32_t v = 0u - (uint32_t)((w >> (k - 6)) & 1ull);
  return make_uint2(v, v);
}

// Support PI k for 32-pattern chunk c.
__device__ __forceinline__ uint32_t pi_lane(uint32_t k, uint64_t c, uint32_t) {
  if (k < 5) return kMaskW[k];
  if (k == 63) return 0u;  // the constant
  return 0u - (uint32_t)((c >> (k - 5)) & 1ull);
}

__device__ __forceinline__ Lane pi_value(uint32_t k, uint64_t u) { return pi_lane(k, u, Lane{}); }

// Shared-memory accesses by 32-bit shared-window address (S: the thread's
// slot base; off: a record's byte offset), written out as ld/st.shared so
// the address arithmetic is one 32-bit add whatever the compiler infers
// about the pointer; volatile keeps them in the order written (a step's
// loads, then its stores), which is the order the record semantics need.
template <typename V>
__device__ __forceinline__ V lds_lane(uint32_t a) {
  if constexpr (sizeof(V) == 8) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
  } else {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
  }
}
template <typename V>
__device__ __forceinline__ void sts_lane(uint32_t a, V v) {
  if constexpr (sizeof(V) == 8)
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
  else
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ Lane ld_slot(uint32_t S, uint32_t off) { return lds_lane<Lane>(S + off); }

__device__ __forceinline__ void st_slot(uint32_t S, uint32_t off, Lane v) { sts_lane<Lane>(S + off, v); }

// One 16-byte record (read by every thread of the warp: a broadcast).
__device__ __forceinline__ uint4 ld_rec(uint32_t a) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(a));
  return r;
}

// One AND; the complement bits of ctl become all-zero / all-one masks by a
// bit-field extract each.
__device__ __forceinline__ void ctl_masks(uint32_t ctl, uint32_t &ma, uint32_t &mb) {
  int a, b;
  asm("bfe.s32 %0, %1, 0, 1;" : "=r"(a) : "r"(ctl));
  asm("bfe.s32 %0, %1, 1, 1;" : "=r"(b) : "r"(ctl));
  ma = (uint32_t)a;
  mb = (uint32_t)b;
}

__device__ __forceinline__ uint2 and_lane(uint2 x, uint2 y, uint32_t ctl) {
  uint32_t ma, mb;
  ctl_masks(ctl, ma, mb);
  return make_uint2((x.x ^ ma) & (y.x ^ mb), (x.y ^ ma) & (y.y ^ mb));
}

__device__ __forceinline__ uint32_t and_lane(uint32_t x, uint32_t y, uint32_t ctl) {
  uint32_t ma, mb;
  ctl_masks(ctl, ma, mb);
  return (x ^ ma) & (y ^ mb);
}

__device__ __forceinline__ uint64_t lane_bits(uint2 v) { return (uint64_t)v.y << 32 | v.x; }
__device__ __forceinline__ uint64_t lane_bits(uint32_t v) { return v; }

// Valid patterns of a lane (bits above the lane's patterns clear): all of
// them unless the support has fewer PIs than the lane has pattern bits.
__device__ __forceinline__ uint64_t lane_valid(uint32_t n) {
  const uint64_t lane = kLanePatterns == 64 ? ~0ull : 0xFFFFFFFFull;
  return n >= 6 ? lane : ((1ull << (1u << n)) - 1ull) & lane;
}

// Lanes covering words [wb, we) of an n-PI support.
__device__ __forceinline__ void lane_range(uint64_t wb, uint64_t we, uint32_t n, uint64_t &ub, uint64_t &ue) {
  if (kLanePatterns == 64) {
    ub = wb;
    ue = we;
    return;
  }
  const uint64_t C = n <= 5 ? 1ull : 1ull << (n - 5);
  ub = min(2 * wb, C);
  ue = min(2 * we, C);
}

// Run AND records [0, cnt) of a staged block.  S is this thread's slot base
// (a byte address in shared memory); record offsets are added to it.
//
// K records per step: all operand loads are issued first, so their
// shared-memory latencies overlap; the stores follow in order.  FWD = false
// (programs of step kInterpStep, K = kInterpStep): no record of a step reads
// what an earlier record of the step writes -- runs end at load records, and
// the slot program puts a load between an AND and any of the K - 1 ANDs
// before it whose result it reads (write-after-read and write-after-write
// within a step are safe: loads come first, stores in order).  FWD = true
// (any program, K = kFwdStep): an operand that an earlier record of the step
// writes is taken from that record's result instead (the nearest earlier
// writer wins, as in sequential order).  The next step's records are read
// before this step's stores.  Record reads may run up to K records past
// cnt; they stay inside the shared-memory allocation (the slot area follows
// the records) and their values are not used.
__device__ __forceinline__ Lane pick(uint32_t off, uint32_t d, Lane v, Lane x) { return off == d ? v : x; }

// Truth-table dump (TT = true, lec_es_truth_tables_ex): a record whose ctl
// carries row + 1 in bits kCtlRowShift.. also stores its value into word
// row x tt_words + (w - word_begin) of tt_out, where w is the lane's word
// (a 32-pattern lane fills its half of it); words outside the range are not
// stored.
struct TTSink {
  uint64_t *out;
  uint64_t words, wb, u;  // u: the thread's lane
};

template <bool TT>
__device__ __forceinline__ void tt_store(const TTSink &k, uint32_t ctl, Lane v) {
  if (!TT) return;
  const uint32_t row = ctl >> kCtlRowShift;
  const uint64_t w = kLanePatterns == 64 ? k.u : k.u >> 1;
  if (!row || w < k.wb || w - k.wb >= k.words) return;
  const uint64_t at = (uint64_t)(row - 1) * k.words + (w - k.wb);
  if (kLanePatterns == 64)
    k.out[at] = lane_bits(v);
  else
    reinterpret_cast<uint32_t *>(k.out)[2 * at + (k.u & 1)] = (uint32_t)lane_bits(v);
}

template <int K, bool FWD, bool TT>
__device__ __forceinline__ void run_ands_k(uint32_t R, uint32_t cnt, uint32_t S, uint32_t &i, const TTSink &tk) {
  uint4 r[K];
#pragma unroll
  for (int j = 0; j < K; j++) r[j] = ld_rec(R + 16u * (i + j));
  for (; i + K <= cnt; i += K) {
    uint4 n[K];
#pragma unroll
    for (int j = 0; j < K; j++) n[j] = ld_rec(R + 16u * (i + K + j));
    Lane x[K], y[K], v[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
      x[j] = ld_slot(S, r[j].x);
      y[j] = ld_slot(S, r[j].y);
    }
#pragma unroll
    for (int j = 0; j < K; j++) {
      if (FWD) {
#pragma unroll
        for (int q = 0; q < j; q++) {  // later writers override earlier ones
          x[j] = pick(r[j].x, r[q].z, v[q], x[j]);
          y[j] = pick(r[j].y, r[q].z, v[q], y[j]);
        }
      }
      v[j] = and_lane(x[j], y[j], r[j].w);
      tt_store<TT>(tk, r[j].w, v[j]);
    }
#pragma unroll
    for (int j = 0; j < K; j++) st_slot(S, r[j].z, v[j]);
#pragma unroll
    for (int j = 0; j < K; j++) r[j] = n[j];
  }
}

template <int K, bool FWD, bool TT>
__device__ __forceinline__ void run_ands(uint32_t R, uint32_t cnt, uint32_t S, const TTSink &tk) {
  uint32_t i = 0;
  if (cnt >= (uint32_t)K) run_ands_k<K, FWD, TT>(R, cnt, S, i, tk);
  // without forwarding, any two records of a run are independent too
  if (!FWD && K > 2 && cnt - i >= 2) run_ands_k<2, false, TT>(R, i + 2, S, i, tk);
  for (; i < cnt; i++) {
    const uint4 r = ld_rec(R + 16u * i);
    const Lane v = and_lane(ld_slot(S, r.x), ld_slot(S, r.y), r.w);
    st_slot(S, r.z, v);
    tt_store<TT>(tk, r.w, v);
  }
}

// Execute one staged block of records [base, base + cnt) of the program,
// applying each load exactly before the record it precedes (a PI may take a
// slot an earlier record has just freed).  li is the next load (updated);
// u is the thread's lane.
template <int K, bool FWD, bool TT = false>
__device__ __forceinline__ void run_block(uint32_t R, uint32_t base, uint32_t cnt, const XLoad *loads,
                                          uint32_t nload, uint32_t &li, uint32_t S, uint64_t u,
                                          const TTSink &tk = TTSink{}) {
  // the next load {at, d_off, k} is held in registers, fetched as soon as the
  // one before it is applied, so its latency hides behind the records between
  const uint4 *l4 = reinterpret_cast<const uint4 *>(loads);
  const uint4 none = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
  uint4 nl = li < nload ? __ldg(l4 + li) : none;
  uint32_t i = 0;
  for (;;) {
    while (nl.x <= base + i) {
      st_slot(S, nl.y, pi_value(nl.z, u));
      li++;
      nl = li < nload ? __ldg(l4 + li) : none;
    }
    if (i >= cnt) break;
    const uint32_t stop = nl.x < base + cnt ? nl.x - base : cnt;
    run_ands<K, FWD, TT>(R + 16u * i, stop - i, S, tk);
    i = stop;
  }
}

// The miter output of the thread's lane: complemented as the output literal
// says, invalid patterns (n below the lane's pattern bits) and lanes outside
// the range cleared.
__device__ __forceinline__ uint64_t out_bits(uint32_t S, uint32_t off, uint32_t compl_out, uint32_t n,
                                             bool in_range) {
  const uint64_t o = lane_bits(ld_slot(S, off)) ^ (compl_out ? ~0ull : 0ull);
  return in_range ? o & lane_valid(n) : 0ull;
}

// Lowest failing pattern of the warp's lanes (thread order = lane order).
__device__ __forceinline__ void report(uint64_t o, uint64_t u, unsigned long long *cex) {
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, o != 0ull);
  if (bal && (int)(threadIdx.x & 31) == __ffs(bal) - 1)
    atomicMin(cex, (unsigned long long)(u * kLanePatterns + (uint64_t)(__ffsll((long long)o) - 1)));
}

// T (threads per block, the lanes of one pass) is the launch's block size,
// any multiple of 32 up to kMaxWordBlock; the records are encoded for it.
// RES: the whole record stream is resident in shared memory (p.resident);
// the two forms are separate instantiations, so each is compiled alone.
template <bool TT, int K, bool FWD, bool RES>
__global__ void __launch_bounds__(kMaxWordBlock, 1) es_interp_w(const XParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t T = blockDim.x;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  volatile unsigned long long *bcast = reinterpret_cast<unsigned long long *>(smem + 48);
  XRec *ring = reinterpret_cast<XRec *>(smem + 64);
  const uint32_t ring_bytes = RES ? p.nrec * 16u : NSTAGE * p.ring_recs * 16u;
  const uint32_t R = smem_u32(ring);  // shared-window address of the records
  const uint32_t S = smem_u32(smem) + 64u + ((ring_bytes + 15u) & ~15u) + threadIdx.x * kLaneBytes;
  const int t = threadIdx.x;
  if (t == 0) {
    for (int s = 0; s < NSTAGE; s++) mbar_init(bar + s);
    fence_init();
  }
  __syncthreads();
  const uint32_t nch = RES ? 1u : (p.nrec + p.ring_recs - 1) / p.ring_recs;
  if (RES && p.nrec) {
    if (t == 0) expect_and_copy(bar, ring, p.recs, p.nrec * 16u, p.extra_tx);
    const bool ok = wait(bar, 0);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
      drain(bar, 1u, 0u);
      return;
    }
  }
  uint32_t parity = 0, inflight = 0;
  uint64_t ub, ue;
  lane_range(p.word_begin, p.word_end, p.n, ub, ue);
  const uint64_t passes = (ue - ub + T - 1) / T;
  if constexpr (RES) {
    // The records stay put for the whole launch, so the warps need no block
    // barrier: each runs its 32 lanes of every pass on its own, reads the
    // counterexample word itself (lane 0, shuffled to the warp) and counts
    // the patterns it evaluated.  The skip test is on the warp's first
    // pattern: a warp skips only lanes at or above the current minimum.
    const uint32_t lane = t & 31u;
    unsigned long long wdone = 0;
    for (uint64_t pass = blockIdx.x; pass < passes; pass += gridDim.x) {
      const uint64_t w0 = ub + pass * T + (t - lane);
      if (w0 >= ue) break;  // this warp's lanes of this pass and of every later one are past the range
      unsigned long long cur = lane == 0 ? ld_volatile(p.cex) : 0ull;
      cur = __shfl_sync(0xFFFFFFFFu, cur, 0);
      if (w0 * kLanePatterns >= cur) break;
      const uint64_t u = w0 + lane;
      const TTSink tk{p.tt_out, p.tt_words, p.word_begin, u};
      uint32_t li = 0;
      run_block<K, FWD, TT>(R, 0, p.nrec, p.loads, p.nload, li, S, u, tk);
      while (li < p.nload) {  // loads after the last record
        st_slot(S, p.loads[li].d_off, pi_value(p.loads[li].k, u));
        li++;
      }
      if (!TT) report(out_bits(S, p.out_off, p.out_compl, p.n, u < ue), u, p.cex);
      wdone += (unsigned long long)min((uint64_t)32, ue - w0);
    }
    if (lane == 0 && wdone) atomicAdd(p.evaluated, wdone * kLanePatterns);
  } else {
    unsigned long long done = 0;
    for (uint64_t pass = blockIdx.x; pass < passes; pass += gridDim.x) {
      const uint64_t u0 = ub + pass * T;
      if (t == 0) *bcast = ld_volatile(p.cex);
      __syncthreads();
      if (u0 * kLanePatterns >= *bcast) break;  // block-uniform early exit
      const uint64_t u = u0 + t;
      const TTSink tk{p.tt_out, p.tt_words, p.word_begin, u};
      uint32_t li = 0;
      for (uint32_t k = 0; k < nch && k < (uint32_t)NSTAGE; k++) {
        if (t == 0) {
          const uint32_t off = k * p.ring_recs;
          expect_and_copy(bar + k, ring + (size_t)k * p.ring_recs, p.recs + off,
                          min(p.ring_recs, p.nrec - off) * 16u, k == 0 ? p.extra_tx : 0u);
        }
        inflight |= 1u << k;
      }
      bool bad = false;
      for (uint32_t k = 0; k < nch; k++) {
        const uint32_t s = k % NSTAGE;
        const bool ok = wait(bar + s, (parity >> s) & 1u);
        if (__syncthreads_or(!ok)) {
          bad = true;
          break;
        }
        parity ^= 1u << s;
        inflight &= ~(1u << s);
        const uint32_t off = k * p.ring_recs;
        run_block<K, FWD, TT>(R + 16u * s * p.ring_recs, off, min(p.ring_recs, p.nrec - off), p.loads, p.nload, li, S, u,
                      tk);
        __syncthreads();
        if (k + NSTAGE < nch) {
          if (t == 0) {
            const uint32_t off2 = (k + NSTAGE) * p.ring_recs;
            expect_and_copy(bar + s, ring + (size_t)s * p.ring_recs, p.recs + off2,
                            min(p.ring_recs, p.nrec - off2) * 16u, 0u);
          }
          inflight |= 1u << s;
        }
      }
      if (bad) {
        if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
        drain(bar, inflight, parity);
        return;
      }
      // loads after the last record (an output that is a PI or the constant)
      while (li < p.nload) {
        st_slot(S, p.loads[li].d_off, pi_value(p.loads[li].k, u));
        li++;
      }
      // a dump checks nothing, so nothing exits early
      if (!TT) report(out_bits(S, p.out_off, p.out_compl, p.n, u < ue), u, p.cex);
      done += (unsigned long long)min((uint64_t)T, ue - u0);
      __syncthreads();
    }
    if (t == 0 && done) atomicAdd(p.evaluated, done * kLanePatterns);
  }
}

// Tile-queue form: blocks pull (miter, word range) tiles.  T as above.
__global__ void __launch_bounds__(kMaxWordBlock, 1) es_batch_w(const XBatchParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t T = blockDim.x;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  volatile unsigned long long *bcast = reinterpret_cast<unsigned long long *>(smem + 40);
  volatile uint32_t *btile = reinterpret_cast<uint32_t *>(smem + 56);
  XRec *ring = reinterpret_cast<XRec *>(smem + 64);
  const uint32_t R = smem_u32(ring);
  const uint32_t S = smem_u32(smem) + 64u + NSTAGE * p.ring_recs * 16u + threadIdx.x * kLaneBytes;
  const int t = threadIdx.x;
  if (t == 0) {
    for (int s = 0; s < NSTAGE; s++) mbar_init(bar + s);
    fence_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  // The miter whose whole program the ring holds: a block's next tile is
  // often another range of the same miter (a miter's tiles are queued
  // together), and then its records are not staged again.
  uint32_t staged = 0xFFFFFFFFu;
  if (t == 0) *btile = atomicAdd(p.head, 1u);
  __syncthreads();
  uint32_t tile = *btile;
  for (;;) {
    __syncthreads();  // every thread has read btile
    if (tile >= p.num_tiles) break;
    // the next tile's index, taken now so that its latency hides behind this tile
    if (t == 0) *btile = atomicAdd(p.head, 1u);
    const XTile bt = p.tiles[tile];
    const XMiter bm = p.miters[bt.miter];
    const XRec *recs = p.recs + bm.rec_off;
    const XLoad *loads = p.loads + bm.load_off;
    const uint32_t nch = (bm.nrec + p.ring_recs - 1) / p.ring_recs;
    const bool resident = nch <= (uint32_t)NSTAGE;  // the whole program fits the ring
    if (resident && bm.nrec && bt.miter != staged) {
      uint32_t inflight = 0;
      for (uint32_t k = 0; k < nch; k++) {
        if (t == 0) {
          const uint32_t off = k * p.ring_recs;
          expect_and_copy(bar + k, ring + (size_t)k * p.ring_recs, recs + off,
                          min(p.ring_recs, bm.nrec - off) * 16u, 0u);
        }
        inflight |= 1u << k;
      }
      bool ok = true;
      for (uint32_t k = 0; k < nch && ok; k++) {
        ok = wait(bar + k, (parity >> k) & 1u);
        if (ok) {
          parity ^= 1u << k;
          inflight &= ~(1u << k);
        }
      }
      if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
        drain(bar, inflight, parity);
        return;
      }
    }
    staged = resident ? bt.miter : 0xFFFFFFFFu;
    uint64_t ub, ue;
    lane_range(bt.word_begin, bt.word_end, bm.n, ub, ue);
    if (resident) {
      // the whole program is staged: warps run the tile's passes on their
      // own, as in es_interp_w (no block barrier per pass)
      const uint32_t lane = t & 31u;
      for (uint64_t w0 = ub + (t - lane); w0 < ue; w0 += T) {
        unsigned long long cur = 0;
        if (lane == 0) {
          cur = ld_volatile(p.cex + bt.miter);
          if (p.cancel && p.cancel[bt.miter]) cur = 0;
        }
        cur = __shfl_sync(0xFFFFFFFFu, cur, 0);
        if (w0 * kLanePatterns >= cur) break;
        const uint64_t u = w0 + lane;
        uint32_t li = 0;
        run_block<kFwdStep, true>(R, 0, bm.nrec, loads, bm.nload, li, S, u);
        while (li < bm.nload) {
          st_slot(S, loads[li].d_off, pi_value(loads[li].k, u));
          li++;
        }
        report(out_bits(S, bm.out_off, bm.out_compl, bm.n, u < ue), u, p.cex + bt.miter);
      }
      __syncthreads();  // ring reuse by the next tile; btile written
      tile = *btile;
      continue;
    }
    for (uint64_t u0 = ub; u0 < ue; u0 += T) {
      if (t == 0) {
        unsigned long long cur = ld_volatile(p.cex + bt.miter);
        if (p.cancel && p.cancel[bt.miter]) cur = 0;
        *bcast = cur;
      }
      __syncthreads();
      const unsigned long long cur = *bcast;
      __syncthreads();
      if (u0 * kLanePatterns >= cur) break;
      const uint64_t u = u0 + t;
      uint32_t li = 0;
      uint32_t inflight = 0;
      for (uint32_t k = 0; k < (uint32_t)NSTAGE; k++) {
        if (t == 0) {
          const uint32_t off = k * p.ring_recs;
          expect_and_copy(bar + k, ring + (size_t)k * p.ring_recs, recs + off,
                          min(p.ring_recs, bm.nrec - off) * 16u, 0u);
        }
        inflight |= 1u << k;
      }
      bool bad = false;
      for (uint32_t k = 0; k < nch; k++) {
        const uint32_t s = k % NSTAGE;
        const bool ok = wait(bar + s, (parity >> s) & 1u);
        if (__syncthreads_or(!ok)) {
          bad = true;
          break;
        }
        parity ^= 1u << s;
        inflight &= ~(1u << s);
        const uint32_t off = k * p.ring_recs;
        run_block<kFwdStep, true>(R + 16u * s * p.ring_recs, off, min(p.ring_recs, bm.nrec - off), loads, bm.nload, li,
                                  S, u);
        __syncthreads();
        if (k + NSTAGE < nch) {
          if (t == 0) {
            const uint32_t off2 = (k + NSTAGE) * p.ring_recs;
            expect_and_copy(bar + s, ring + (size_t)s * p.ring_recs, recs + off2,
                            min(p.ring_recs, bm.nrec - off2) * 16u, 0u);
          }
          inflight |= 1u << s;
        }
      }
      if (bad) {
        if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
        drain(bar, inflight, parity);
        return;
      }
      while (li < bm.nload) {
        st_slot(S, loads[li].d_off, pi_value(loads[li].k, u));
        li++;
      }
      report(out_bits(S, bm.out_off, bm.out_compl, bm.n, u < ue), u, p.cex + bt.miter);
      __syncthreads();
    }
    __syncthreads();  // ring reuse by the next tile; btile written
    tile = *btile;
  }
}

template <bool TT, int K, bool FWD, bool RES>
int launch_wkr(const XParams &p, int block, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(es_interp_w<TT, K, FWD, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  es_interp_w<TT, K, FWD, RES><<<grid, block, smem, st>>>(p);
  return (int)cudaGetLastError();
}

template <bool TT, int K, bool FWD>
int launch_wk(const XParams &p, int block, int grid, size_t smem, cudaStream_t st) {
  return p.resident ? launch_wkr<TT, K, FWD, true>(p, block, grid, smem, st)
                    : launch_wkr<TT, K, FWD, false>(p, block, grid, smem, st);
}

// Programs of step kInterpStep run without forwarding, others with it.
template <bool TT = false>
int launch_w(const XParams &p, int block, int grid, size_t smem, cudaStream_t st) {
  if (!word_block_ok(block)) return (int)cudaErrorInvalidValue;
  if (p.step == (uint32_t)kInterpStep) return launch_wk<TT, kInterpStep, false>(p, block, grid, smem, st);
  return launch_wk<TT, kFwdStep, true>(p, block, grid, smem, st);
}

}  // namespace

size_t interp_w_smem_bytes(uint32_t nslots, uint32_t nrec, int block, uint32_t *ring_recs, uint32_t *resident,
                           bool allow_resident) {
  const size_t limit = 227u * 1024u;
  const size_t slots = (size_t)nslots * block * kLaneBytes;
  const size_t whole = 64 + (size_t)nrec * 16u + slots;
  if (allow_resident && whole <= limit) {
    *resident = 1;
    *ring_recs = nrec;
    return whole;
  }
  *resident = 0;
  *ring_recs = 256;
  return 64 + (size_t)NSTAGE * 256u * 16u + slots;
}

size_t batch_w_smem_bytes(uint32_t max_slots, int block, uint32_t ring_recs) {
  return 64 + (size_t)NSTAGE * ring_recs * 16u + (size_t)max_slots * block * kLaneBytes;
}

int launch_interp_w(const XParams &p, int block, int grid, size_t smem, void *stream) {
  return launch_w<false>(p, block, grid, smem, (cudaStream_t)stream);
}

int launch_interp_w_tt(const XParams &p, int block, int grid, size_t smem, void *stream) {
  return launch_w<true>(p, block, grid, smem, (cudaStream_t)stream);
}

int configure_batch_w(int block, size_t smem) {
  if (!word_block_ok(block)) return (int)cudaErrorInvalidValue;
  return (int)cudaFuncSetAttribute(es_batch_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int batch_w_blocks_per_sm(int block, size_t smem) {
  int n = 0;
  if (!word_block_ok(block)) return 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, es_batch_w, block, smem) == cudaSuccess ? n : 0;
}

int launch_batch_w(const XBatchParams &p, int block, int grid, size_t smem, void *stream) {
  if (!word_block_ok(block)) return (int)cudaErrorInvalidValue;
  es_batch_w<<<grid, block, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace lec
