// noalloc.cu -- exact simulation without any device allocation by the library.
//
// Some callers cannot call cudaMalloc: code that runs under a framework whose
// caching allocator owns all device memory, or a service that may not
// allocate once it has started.  lec_es_check_noalloc serves them.  It runs
// the global-memory ("spill") variant of the interpreter kernel, whose
// per-lane value slots normally live in scratch memory the context
// allocates; here that scratch is the file-scope array below, a fixed
// kNoAllocScratchBytes that every GPU loading the library keeps until the
// process exits.  The caller passes the inputs (the compiled records, already
// in device memory) and the outputs (four 64-bit result words); the call
// itself allocates nothing on the device or the host.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents.  Nothing in it needs clearing: the kernel writes every
// slot before reading it.  Calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/lec_es.h"
#include "es_internal.h"

namespace lec {
namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB per device
constexpr size_t kScratchWords = kNoAllocScratchBytes / 4;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

struct DeviceSetup {
  uint32_t *scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sm_count = 0;
  bool done = false;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the array's device address (the
// host-side name is only a stand-in) and the SM count.
int setup_device(int dev, DeviceSetup **out) {
  if (dev < 0 || dev >= kMaxDevices) return LEC_ES_EINVAL;
  std::lock_guard<std::mutex> g(g_setup_mu);
  DeviceSetup &s = g_setup[dev];
  if (!s.done) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LEC_ES_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      return LEC_ES_ECUDA;
    s.scratch = (uint32_t *)ptr;
    s.sm_count = sms;
    s.done = true;
  }
  *out = &s;
  return LEC_ES_OK;
}

}  // namespace
}  // namespace lec

using namespace lec;

extern "C" int lec_es_check_noalloc(const uint64_t *d_records, uint64_t records_capacity,
                                    const lec_es_program_info *prog, uint64_t word_begin, uint64_t word_end,
                                    unsigned long long *d_result, void *stream) {
  if (!d_records || !prog || !d_result) return LEC_ES_EINVAL;
  if (((uintptr_t)d_records & 15u) != 0 || ((uintptr_t)d_result & 7u) != 0) return LEC_ES_EINVAL;
  const uint64_t nrec = prog->num_records;
  const uint64_t nrec_padded = nrec < 2 ? 2 : (nrec + 1) & ~1ull;  // the bulk copy moves 16-byte pairs
  if (nrec == 0 || records_capacity < nrec_padded || nrec_padded > 0xFFFFFFFFull) return LEC_ES_EINVAL;
  if (prog->n > 63 || prog->num_slots == 0 || prog->out_slot >= prog->num_slots) return LEC_ES_EINVAL;
  // the largest live set one warp of lanes can hold in the fixed scratch
  if ((uint64_t)prog->num_slots * 32u > kScratchWords) return LEC_ES_ETOOBIG;
  const uint64_t W = num_words(prog->n);
  if (word_end > W) word_end = W;
  if (word_begin >= word_end) return LEC_ES_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LEC_ES_ECUDA;
  DeviceSetup *s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc) return rc;

  // lanes the scratch holds for this live set, as whole blocks
  const uint64_t lanes = kScratchWords / prog->num_slots;
  int block = 128;
  while (block > 32 && (uint64_t)block > lanes) block /= 2;
  const uint64_t C = num_chunks(prog->n);
  const uint64_t cb = std::min<uint64_t>(2 * word_begin, C), ce = std::min<uint64_t>(2 * word_end, C);
  const uint64_t passes = (ce - cb + block - 1) / block;
  uint64_t grid = lanes / block;
  grid = std::min<uint64_t>(grid, (uint64_t)s->sm_count * 8);
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, passes));

  uint32_t ring = 0, resident = 0;
  size_t smem = 0;
  if (interp_smem_bytes(0, (uint32_t)nrec_padded, block, &ring, &resident, &smem) != 0) return LEC_ES_ETOOBIG;

  cudaStream_t st = (cudaStream_t)stream;
  // result words: lowest failing pattern = none, patterns evaluated = 0, status = 0
  if (cudaMemsetAsync(d_result, 0xFF, 8, st) != cudaSuccess) return LEC_ES_ECUDA;
  if (cudaMemsetAsync(d_result + 1, 0, 24, st) != cudaSuccess) return LEC_ES_ECUDA;

  InterpParams ip;
  memset(&ip, 0, sizeof(ip));
  ip.recs = (const Rec *)d_records;
  ip.nrec = (uint32_t)nrec;
  ip.nrec_padded = (uint32_t)nrec_padded;
  ip.nslots = prog->num_slots;
  ip.out_slot = prog->out_slot;
  ip.out_compl = prog->out_compl;
  ip.n = prog->n;
  ip.ring_recs = ring;
  ip.resident = resident;
  ip.chunk_begin = cb;
  ip.chunk_end = ce;
  ip.cex = d_result;
  ip.evaluated = d_result + 1;
  ip.status = (uint32_t *)(d_result + 2);
  ip.spill = s->scratch;  // slot s of grid lane t at spill[s * grid * block + t]
  if (launch_interp(ip, block, (int)grid, smem, true, st) != 0) return LEC_ES_ECUDA;
  return LEC_ES_OK;
}
