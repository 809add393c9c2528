// Rescale without any device allocation, for callers that cannot allocate.
//
// Some callers of this library must not allocate device memory once they are running:
// a host framework that reserved the whole device up front for its own arena (a later
// cudaMalloc would fail or fragment it), or a latency-critical serving thread where an
// allocation could block on the device or fail under memory pressure in the middle of a
// request.  ctl_rescale_static_dev gives them the rescale step with the caller's own
// input and output buffers; the one scratch buffer the operation needs (the rounded last
// limb in coefficient form) lives in a fixed array compiled into this library.
//
// The scratch array is file-scope device memory: every GPU that loads the library holds
// kNoAllocScratchWords 64-bit words (4 MiB) until the process exits.  In host code the
// symbol name stands for a host-side shadow, not a device address, so its device
// address is fetched with cudaGetSymbolAddress, once per device, with that device
// current, on the first call made on that device.
#include <cstdio>
#include <mutex>
#include "ctl_internal.h"

namespace {

constexpr size_t kNoAllocScratchWords = (size_t)1 << 19;  // 4 MiB of 64-bit words
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_rescale_scratch[kNoAllocScratchWords];

std::mutex g_mu;
ctl::u64* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on first use).
int scratch_for_device(int dev, ctl::u64** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    ctl::set_error("ctl_rescale_static_dev: device ordinal %d out of range", dev);
    return CTL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rescale_scratch);
    if (e != cudaSuccess || !p) {
      ctl::set_error("ctl_rescale_static_dev: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return CTL_ECUDA;
    }
    g_scratch_dev[dev] = (ctl::u64*)p;
  }
  *out = g_scratch_dev[dev];
  return CTL_OK;
}

}  // namespace

extern "C" size_t ctl_rescale_static_capacity_words(void) { return kNoAllocScratchWords; }

extern "C" int ctl_rescale_static_dev(ctl_context* c, const uint64_t* in_dev, uint64_t* out_dev, uint32_t count,
                                      uint32_t level) {
  if (!c || !in_dev || !out_dev || count == 0) {
    ctl::set_error("ctl_rescale_static_dev: null argument or empty batch");
    return CTL_EINVAL;
  }
  if (level < 2 || level > c->L) {
    ctl::set_error("ctl_rescale_static_dev: level %u has no prime to drop (need 2..%u)", level, c->L);
    return CTL_ELEVEL;
  }
  const size_t need = (size_t)count * 2 * c->N;  // one coefficient-form limb per poly
  if (need > kNoAllocScratchWords) {
    ctl::set_error("ctl_rescale_static_dev: %u ciphertexts at N=%u need %zu scratch words, the fixed limit is %zu "
                   "(at most %zu ciphertexts per call at this N)",
                   count, c->N, need, kNoAllocScratchWords, kNoAllocScratchWords / (2 * (size_t)c->N));
    return CTL_EINVAL;
  }
  int dev = -1;
  if (int rc = ctl::cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  ctl::u64* scratch = nullptr;
  if (int rc = scratch_for_device(dev, &scratch)) return rc;
  // The scratch limb of every poly is written in full by the first kernel before the
  // second reads it, so nothing in it has to start at zero.
  const size_t LN = (size_t)level * c->N;
  ctl::launch_intt_rescale_last(c, (const ctl::u64*)in_dev, LN, (int)(2 * count), (int)level, scratch);
  ctl::launch_rescale_ntt(c, scratch, (const ctl::u64*)in_dev, LN, (ctl::u64*)out_dev, (size_t)(level - 1) * c->N,
                          (int)(2 * count), (int)level);
  return ctl::cuda_check(cudaGetLastError(), "ctl_rescale_static_dev");
}
