// Throughput microbenchmarks of the integer work units that the kernels' rooflines count:
// the 64-bit Shoup modular multiplication, a Harvey butterfly, the three-high-half Shoup
// product of the small-prime path and the split-half multiply-accumulate.  Each thread
// runs eight independent dependency chains of one unit, so the measured rate is the
// issue-limited throughput of the integer pipes, not their latency.
#include "ctl_internal.h"
#include "modarith.cuh"

namespace ctl {
namespace {

constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_unit_rate(u64* out, u64 q, u64 w, u64 wsh, int iters) {
  u64 x[kChains], y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) {
    x[c] = (threadIdx.x * 977u + blockIdx.x * 131u + c * 7u) % q;
    y[c] = (x[c] * 3 + 1) % q;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) {
      if constexpr (KIND == 0) {  // Shoup product, fully reduced
        x[c] = shoup(x[c], w, wsh, q);
      } else if constexpr (KIND == 1) {  // Harvey butterfly: X below 2q, outputs below 4q
        const u64 q2 = 2 * q;
        u64 X = x[c];
        if (X >= q2) X -= q2;
        const u64 T = shoup_lazy(y[c], w, wsh, q);
        x[c] = X + T;
        y[c] = X - T + q2;
      } else if constexpr (KIND == 2) {  // three-high-half Shoup product (below 4q)
        x[c] = shoup_small(x[c], w, wsh, q);
      } else {  // split-half multiply-accumulate: four 32x32->64 multiply-adds
        const uint32_t a0 = (uint32_t)x[c], a1 = (uint32_t)(x[c] >> 32);
        const uint32_t b0 = (uint32_t)w, b1 = (uint32_t)(w >> 32);
        y[c] += (u64)a0 * b0 + (u64)a1 * b1;
        x[c] += (u64)a0 * b1 + (u64)a1 * b0 + 1;
      }
    }
  }
  u64 s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s ^= x[c] ^ y[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int KIND>
int time_unit(int sms, double* per_clk_sm) {
  const int threads = 256, blocks = sms * 8, iters = 4096;
  u64* out = nullptr;
  if (cudaMalloc(&out, (size_t)threads * blocks * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    set_error("microbench: allocation failed");
    return CTL_ENOMEM;
  }
  const u64 q = 0x1fffffffffe00001ull % (1ull << 61);  // an odd 61-bit modulus
  const u64 w = 0x123456789abcdefull % q;
  const u64 wsh = h_shoup(w, q);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_unit_rate<KIND><<<blocks, threads>>>(out, q, w, wsh, 64);  // warm-up
  cudaEventRecord(e0);
  k_unit_rate<KIND><<<blocks, threads>>>(out, q, w, wsh, iters);
  cudaEventRecord(e1);
  int rc = cuda_check(cudaEventSynchronize(e1), "microbench");
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return rc;
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  const double units = (double)threads * blocks * iters * kChains;
  const double clocks = (double)ms * 1e-3 * (double)khz * 1e3;
  *per_clk_sm = units / clocks / sms;
  return CTL_OK;
}

}  // namespace
}  // namespace ctl

// Units per clock per SM (at the device's maximum SM clock) of the work unit `kind`:
// 0 = Shoup modular multiplication, 1 = Harvey butterfly, 2 = three-high-half Shoup
// product, 3 = split-half multiply-accumulate.  Runs on the current device, synchronously.
extern "C" int ctl_microbench_unit_rate(int kind, double* per_clk_sm) {
  using namespace ctl;
  if (!per_clk_sm || kind < 0 || kind > 3) {
    set_error("ctl_microbench_unit_rate: invalid argument");
    return CTL_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (kind) {
    case 0: return time_unit<0>(sms, per_clk_sm);
    case 1: return time_unit<1>(sms, per_clk_sm);
    case 2: return time_unit<2>(sms, per_clk_sm);
    default: return time_unit<3>(sms, per_clk_sm);
  }
}

namespace ctl {
namespace {

__global__ void k_modarith_eval(int kind, const u64* __restrict__ x, u64* __restrict__ out, size_t n, u64 w, u64 wsh,
                                u64 q, u64 aux) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const u64 v = x[i];
    u64 r;
    switch (kind) {
      case 0: r = shoup(v, w, wsh, q); break;
      case 1: r = shoup_lazy(v, w, wsh, q); break;
      case 2: r = shoup_small(v, w, wsh, q); break;
      case 3: r = reduce_wide(v, q, aux); break;
      case 4: r = mulmod_mont(v, w, q, aux); break;
      default: r = reduce4(v, q); break;
    }
    out[i] = r;
  }
}

}  // namespace
}  // namespace ctl

// Evaluates one modular-arithmetic primitive of the kernels on n host values (copied to
// the device and back, synchronously, on the current device), so that tests can compare
// the device results with exact integer arithmetic.  kind: 0 = shoup(x, w, wsh, q),
// 1 = shoup_lazy, 2 = shoup_small (three-high-half product), 3 = reduce_wide(x, q, bar =
// aux), 4 = mulmod_mont(x, bmont = w, q, qinv = aux), 5 = reduce4(x, q).
extern "C" int ctl_modarith_eval(int kind, const uint64_t* x, size_t n, uint64_t w, uint64_t wsh, uint64_t q,
                                 uint64_t aux, uint64_t* out) {
  using namespace ctl;
  if (kind < 0 || kind > 5 || (n && (!x || !out)) || q < 2) {
    set_error("ctl_modarith_eval: invalid argument");
    return CTL_EINVAL;
  }
  if (!n) return CTL_OK;
  u64 *dx = nullptr, *dy = nullptr;
  if (cudaMalloc(&dx, n * sizeof(u64)) != cudaSuccess || cudaMalloc(&dy, n * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    if (dx) cudaFree(dx);
    set_error("ctl_modarith_eval: allocation failed");
    return CTL_ENOMEM;
  }
  int rc = cuda_check(cudaMemcpy(dx, x, n * sizeof(u64), cudaMemcpyHostToDevice), "modarith copy");
  if (!rc) {
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((n + threads - 1) / threads, 4096);
    k_modarith_eval<<<blocks, threads>>>(kind, dx, dy, n, w, wsh, q, aux);
    rc = cuda_check(cudaGetLastError(), "modarith launch");
  }
  if (!rc) rc = cuda_check(cudaMemcpy(out, dy, n * sizeof(u64), cudaMemcpyDeviceToHost), "modarith copy back");
  cudaFree(dx);
  cudaFree(dy);
  return rc;
}
