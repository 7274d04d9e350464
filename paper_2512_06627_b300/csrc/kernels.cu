// kernels.cu -- generic exact-simulation kernels for sm_103a.
//
// Work unit: a 32-pattern chunk.  Chunk c covers patterns 32c .. 32c+31 of
// the cone's pattern space (the low / high half of 64-pattern word c/2), so
// support PI k < 5 is the constant mask kMask32[k] and PI k >= 5 is all ones
// iff bit (k-5) of c is set.  One thread evaluates one chunk per pass through
// the whole instruction stream (paper §3.3: the cone compiled to a branch-free
// instruction stream over reference-counted value slots; each GPU thread
// simulates 32 patterns).
//
// Kernels
//   es_interp   one miter; the instruction stream is copied global->shared by
//               the bulk-copy engine (cp.async.bulk, mbarrier completion) either
//               once (it fits) or through a 4-stage ring; value slots live in
//               shared memory (slot-major, lane-minor: conflict-free) or, for
//               live sets too large for shared memory, in global memory.
//               The single-miter interpreter tier itself runs the word-wide
//               kernel (interp_w.cu); this one serves the spill tier, the
//               truth-table dump and the allocation-free entry point.
//   lop3_bench  throughput microbenchmark of 32-bit LOP3.
//
// Every AND is one LOP3 per 32-bit lane: (x ^ ca) & (y ^ cb) with warp-uniform
// complement masks.  The miter output goes through a warp ballot; the lowest
// failing lane does atomicMin on the 64-bit counterexample.  Before each pass
// a block reads the current counterexample and skips the pass if its first
// pattern is not lower (early exit; a pass below the minimum always finishes,
// so the reported counterexample is the lowest whatever the schedule).
//
// Device-side waits are bounded: an mbarrier wait that exceeds its iteration
// limit sets DEV_WAIT_TIMEOUT in *status and the block returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "es_internal.h"

namespace lec {

namespace {

constexpr int NSTAGE = 4;
constexpr uint32_t kWaitLimit = 1u << 24;           // poll backstop
constexpr uint64_t kWaitNs = 1000000000ull;         // a wait gives up after 1 s

__constant__ uint32_t kMask32[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> this CTA's shared memory, completion counted on bar.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: false once 1 s of global time has passed (or after
// kWaitLimit polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kWaitLimit; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15u) == 15u && global_ns() - t0 > kWaitNs) return false;
    if (i > 64) __nanosleep(128);
  }
  return false;
}

// After a timed-out wait: wait once more (bounded) for every copy this block
// still has in flight, so no bulk copy lands after the block has exited.
__device__ __forceinline__ void drain_inflight(uint64_t *bar, uint32_t inflight, uint32_t parity) {
  if (threadIdx.x != 0) return;
  for (int s = 0; s < NSTAGE; s++)
    if ((inflight >> s) & 1u) (void)mbar_wait(bar + s, (parity >> s) & 1u);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ uint32_t pi_word(uint32_t k, uint64_t chunk) {
  return k < 5 ? kMask32[k] : (0u - (uint32_t)((chunk >> (k - 5)) & 1ull));
}

__device__ __forceinline__ uint32_t valid_mask(uint32_t n) {
  return n >= 5 ? 0xFFFFFFFFu : ((1u << (1u << n)) - 1u);
}

// Execute records [0, cnt) of a staged block on this thread's slots.
// S points at slot 0 of this lane; slot s is S[s * STRIDE].
template <bool TT>
__device__ __forceinline__ void run_records(const Rec *rr, uint32_t cnt, uint32_t *S, uint32_t stride,
                                            uint64_t c, uint32_t rec_base, const InterpParams &p) {
  const uint2 *r2 = reinterpret_cast<const uint2 *>(rr);
#pragma unroll 4
  for (uint32_t i = 0; i < cnt; i++) {
    const uint2 w = r2[i];  // same address in every lane: broadcast
    const uint32_t dst = w.x & 0xFFFFu, a = w.x >> 16, b = w.y & 0xFFFFu, op = (w.y >> 16) & 0xFFu;
    uint32_t v;
    if (op < 4) {
      const uint32_t x = S[a * stride], y = S[b * stride];
      v = (x ^ (0u - (op & 1u))) & (y ^ (0u - ((op >> 1) & 1u)));
    } else if (op == OP_PI) {
      v = pi_word(a, c);
    } else {
      v = 0u;
    }
    S[dst * stride] = v;
    if (TT) {
      const uint32_t row = p.tt_row[rec_base + i];
      if (row != 0xFFFFFFFFu && c < p.chunk_end) {
        uint32_t *o = reinterpret_cast<uint32_t *>(p.tt_out);
        o[(uint64_t)row * 2ull * p.tt_words + (c - 2ull * p.tt_word_begin)] = v;
      }
    }
  }
}

template <int T, bool SPILL, bool TT>
__global__ void __launch_bounds__(T) es_interp(const InterpParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  volatile unsigned long long *bcast = reinterpret_cast<unsigned long long *>(smem + 48);
  Rec *ring = reinterpret_cast<Rec *>(smem + 64);
  const uint32_t ring_bytes = p.resident ? p.nrec_padded * 8u : NSTAGE * p.ring_recs * 8u;
  const int t = threadIdx.x;
  uint32_t *S;
  uint32_t stride;
  if (SPILL) {
    S = p.spill + (size_t)blockIdx.x * T + t;
    stride = gridDim.x * T;
  } else {
    S = reinterpret_cast<uint32_t *>(smem + 64 + ((ring_bytes + 15u) & ~15u)) + t;
    stride = T;
  }
  if (t == 0) {
    for (int s = 0; s < NSTAGE; s++) mbar_init(bar + s, 1);
    fence_mbar_init();
  }
  __syncthreads();

  const uint32_t nch = p.resident ? 1u : (p.nrec + p.ring_recs - 1) / p.ring_recs;
  if (p.resident) {
    if (t == 0) {
      mbar_arrive_expect_tx(bar, p.nrec_padded * 8u + p.extra_tx);
      bulk_g2s(ring, p.recs, p.nrec_padded * 8u, bar);
    }
    const bool ok = mbar_wait(bar, 0);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
      drain_inflight(bar, 1u, 0u);
      return;
    }
  }
  uint32_t parity = 0;
  uint32_t inflight = 0;
  const uint64_t total = p.chunk_end - p.chunk_begin;
  const uint64_t passes = (total + T - 1) / T;
  const uint32_t vmask = valid_mask(p.n);
  const uint32_t ocompl = p.out_compl ? 0xFFFFFFFFu : 0u;
  unsigned long long done = 0;
  for (uint64_t pass = blockIdx.x; pass < passes; pass += gridDim.x) {
    const uint64_t c0 = p.chunk_begin + pass * T;
    if (t == 0) *bcast = ld_volatile_u64(p.cex);
    __syncthreads();
    const unsigned long long cur = *bcast;
    if (c0 * 32ull >= cur) break;  // block-uniform
    const uint64_t c = c0 + t;
    if (p.resident) {
      run_records<TT>(ring, p.nrec, S, stride, c, 0, p);
    } else {
      for (uint32_t k = 0; k < nch && k < (uint32_t)NSTAGE; k++) {
        if (t == 0) {
          const uint32_t off = k * p.ring_recs;
          const uint32_t cnt = min(p.ring_recs, p.nrec_padded - off);
          mbar_arrive_expect_tx(bar + k, cnt * 8u + (k == 0 ? p.extra_tx : 0u));
          bulk_g2s(ring + (size_t)k * p.ring_recs, p.recs + off, cnt * 8u, bar + k);
        }
        inflight |= 1u << k;
      }
      bool bad = false;
      for (uint32_t k = 0; k < nch; k++) {
        const uint32_t s = k % NSTAGE;
        const bool ok = mbar_wait(bar + s, (parity >> s) & 1u);
        if (__syncthreads_or(!ok)) {
          bad = true;
          break;
        }
        parity ^= 1u << s;
        inflight &= ~(1u << s);
        const uint32_t off = k * p.ring_recs;
        run_records<TT>(ring + (size_t)s * p.ring_recs, min(p.ring_recs, p.nrec - off), S, stride, c, off, p);
        __syncthreads();
        if (k + NSTAGE < nch) {
          if (t == 0) {
            const uint32_t off2 = (k + NSTAGE) * p.ring_recs;
            const uint32_t cnt = min(p.ring_recs, p.nrec_padded - off2);
            mbar_arrive_expect_tx(bar + s, cnt * 8u);
            bulk_g2s(ring + (size_t)s * p.ring_recs, p.recs + off2, cnt * 8u, bar + s);
          }
          inflight |= 1u << s;
        }
      }
      if (bad) {
        if (t == 0) atomicOr(p.status, DEV_WAIT_TIMEOUT);
        drain_inflight(bar, inflight, parity);
        return;
      }
    }
    uint32_t out = (S[p.out_slot * stride] ^ ocompl) & vmask;
    if (c >= p.chunk_end) out = 0;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, out != 0u);
    if (bal) {
      const int lane = __ffs(bal) - 1;
      if ((t & 31) == lane) atomicMin(p.cex, (unsigned long long)(c * 32ull + (uint64_t)(__ffs(out) - 1)));
    }
    done += (unsigned long long)min((uint64_t)T, p.chunk_end - c0);
    __syncthreads();
  }
  if (t == 0 && done) atomicAdd(p.evaluated, done * 32ull);
}

// ---------------------------------------------------------------------------
// LOP3 throughput microbenchmark: 8 independent chains per thread.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) lop3_bench(uint32_t *out, unsigned long long *cycles, int iters) {
  uint32_t a0 = threadIdx.x, a1 = a0 * 3u + 1u, a2 = a0 * 5u + 2u, a3 = a0 * 7u + 3u;
  uint32_t a4 = a0 ^ 0x55u, a5 = a0 ^ 0xAAu, a6 = a0 + 9u, a7 = a0 + 11u;
  const uint32_t k1 = blockIdx.x | 0x1234u, k2 = blockIdx.x ^ 0x0F0Fu;
  unsigned long long g0, g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  const unsigned long long t0 = clock64();
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 16; j++) {
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a0) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a1) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a2) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a3) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a4) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a5) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a6) : "r"(k1), "r"(k2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a7) : "r"(k1), "r"(k2));
    }
  }
  const unsigned long long t1 = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
  // SM clock of this block's lifetime: SM cycles over global nanoseconds
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cycles[0] = t1 - t0;
    cycles[1] = g1 - g0;
  }
}

template <int T, bool SPILL, bool TT>
int launch_one(const InterpParams &p, int grid, size_t smem, cudaStream_t st) {
  auto k = es_interp<T, SPILL, TT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k<<<grid, T, smem, st>>>(p);
  return (int)cudaGetLastError();
}

template <bool SPILL, bool TT>
int launch_block(const InterpParams &p, int block, int grid, size_t smem, cudaStream_t st) {
  switch (block) {
    case 32: return launch_one<32, SPILL, TT>(p, grid, smem, st);
    case 64: return launch_one<64, SPILL, TT>(p, grid, smem, st);
    case 128: return launch_one<128, SPILL, TT>(p, grid, smem, st);
    case 256: return launch_one<256, SPILL, TT>(p, grid, smem, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int interp_smem_bytes(uint32_t nslots, uint32_t nrec_padded, int block, uint32_t *ring_recs,
                      uint32_t *resident, size_t *bytes) {
  // resident when the whole program fits beside the slots, else a 4-stage ring
  const size_t limit = 227u * 1024u;
  const size_t slots = (size_t)nslots * block * 4u;
  const size_t whole = 64 + (((size_t)nrec_padded * 8u + 15u) & ~(size_t)15u) + slots;
  if (whole <= limit) {
    *resident = 1;
    *ring_recs = nrec_padded;
    *bytes = whole;
    return 0;
  }
  *resident = 0;
  *ring_recs = 512;
  *bytes = 64 + (size_t)NSTAGE * 512u * 8u + slots;
  return *bytes <= limit ? 0 : 1;
}

int launch_interp(const InterpParams &p, int block, int grid, size_t smem, bool spill, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool tt = p.tt_out != nullptr;
  if (spill) return tt ? launch_block<true, true>(p, block, grid, smem, st)
                       : launch_block<true, false>(p, block, grid, smem, st);
  return tt ? launch_block<false, true>(p, block, grid, smem, st) : launch_block<false, false>(p, block, grid, smem, st);
}

int launch_lop3_bench(uint32_t *out, unsigned long long *cycles, int grid, int block, int iters, void *stream) {
  lop3_bench<<<grid, block, 0, (cudaStream_t)stream>>>(out, cycles, iters);
  return (int)cudaGetLastError();
}

int max_smem_optin(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return v;
}

}  // namespace lec
