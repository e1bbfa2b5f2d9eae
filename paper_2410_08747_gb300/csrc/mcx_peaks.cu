// mcx_peaks.cu -- the library's own microbenchmarks: the measured peak rates
// that the tracer's roofline divides by.  The tracer is not a dense
// contraction: it is bound by instruction issue on the FP32/INT pipes, by the
// FP64 pipe where the binary64 frames run, or by the rate at which global
// atomics reach the monitors in L2/HBM, so each of those units gets a
// measurement of its own:
//   FFMA      binary32 fused multiply-add chains (one lane instruction each);
//   IMAD      32-bit integer multiply-add chains;
//   PHILOX    whole Philox4x32-10 blocks (the per-ray generator, Sec. 2.2.2's
//             re-implemented RNG) from registers, one block per loop trip;
//   DFMA      binary64 fused multiply-add chains;
//   HIT       monitor hits: three global atomic adds (count u64, sum w f64,
//             sum w^2 f64) to one 24-byte bin, bins drawn uniformly at random
//             over an array of a given footprint (the tracer's score pattern);
//   RED_U64   single u64 atomic adds at random positions of a footprint.
// Chains are independent per thread (8 per thread) so that latency hides
// behind issue; every launch runs a persistent grid of 8 blocks of 256
// threads per SM; results are kept alive by a store guarded by a flag the
// host never sets.
#include <cstdint>

#include "mcx_host.h"
#include "mcx_tracer.cuh"

namespace mcx {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) ffma_kernel(int iters, float b, float c, int flag, float* out) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (flag == 1) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) imad_kernel(int iters, uint32_t c, int flag, uint32_t* out) {
  uint32_t a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 2654435761u + j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = a[j] * a[j] + c;   // quadratic: no chain folds
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s ^= a[j];
  if (flag == 1) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_kernel(int iters, double b, double c, int flag, double* out) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (double)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (flag == 1) out[blockIdx.x] = s;
}

// One Philox4x32-10 block per trip, the counter advanced by the previous
// block's output so the trips form a dependent chain (two chains per thread).
__global__ void __launch_bounds__(256) philox_kernel(int iters, uint32_t k0, uint32_t k1, int flag, uint32_t* out) {
  uint32_t c[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    c[j][0] = blockIdx.x * blockDim.x + threadIdx.x;
    c[j][1] = j;
    c[j][2] = 0;
    c[j][3] = 7;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t o0, o1, o2, o3;
      philox4x32_10(c[j][0], c[j][1], c[j][2], c[j][3], k0, k1, o0, o1, o2, o3);
      c[j][0] = o0; c[j][1] = o1; c[j][2] = o2; c[j][3] = o3;
    }
  }
  if (flag == 1) out[blockIdx.x] = c[0][0] ^ c[1][1] ^ c[0][2] ^ c[1][3];
}

// Random bin of [0, n): a per-thread linear congruential sequence, scaled by
// a high multiply (no division).
__device__ __forceinline__ uint32_t next_bin(uint32_t& x, uint32_t n) {
  x = x * 1664525u + 1013904223u;
  return __umulhi(x, n);
}

__global__ void __launch_bounds__(256) hit_kernel(int iters, MonBin* bins, uint32_t n_bins) {
  uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 747796405u + 1u;
  const float w = 0.5f + (float)(threadIdx.x & 31) * (1.0f / 64.f);
  const double wd = (double)w;
  // the tracer's own monitor update (bin_add: three atomic adds, with the L2
  // cache hint a detector that fits the L2 gets)
  for (int it = 0; it < iters; ++it) bin_add(bins + next_bin(x, n_bins), wd, true);
}

__global__ void __launch_bounds__(256) red_u64_kernel(int iters, unsigned long long* a, uint32_t n) {
  uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 747796405u + 1u;
  for (int it = 0; it < iters; ++it) atomicAdd(a + next_bin(x, n), 1ull);
}

}  // namespace
}  // namespace mcx

using namespace mcx;

extern "C" mcx_status mcx_peak_measure(int32_t kind, int32_t device, uint64_t footprint_bytes,
                                       double* ops_per_s) {
  if (!ops_per_s) return fail(MCX_ERR_INVALID, "ops_per_s is NULL");
  if (kind < MCX_PEAK_FFMA || kind > MCX_PEAK_RED_U64) return fail(MCX_ERR_INVALID, "unknown peak kind %d", kind);
  const bool atomic = kind == MCX_PEAK_HIT || kind == MCX_PEAK_RED_U64;
  const size_t elem = kind == MCX_PEAK_HIT ? sizeof(MonBin) : sizeof(unsigned long long);
  if (atomic && (footprint_bytes < 64 * elem || footprint_bytes / elem > 0xFFFFFFFFull))
    return fail(MCX_ERR_INVALID, "footprint must hold 64 .. 2^32 - 1 elements");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", device);
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  const int block = 256, grid = n_sm * 8;
  const double threads = (double)grid * block;
  // loop trips per thread, sized for a few milliseconds per launch at the
  // expected rate; ops per thread per trip
  int iters = 0;
  double per_trip = 0.0;
  switch (kind) {
    case MCX_PEAK_FFMA: iters = 2048; per_trip = kChains * kUnroll; break;
    case MCX_PEAK_IMAD: iters = 1024; per_trip = kChains * kUnroll; break;
    case MCX_PEAK_PHILOX: iters = 1024; per_trip = 2; break;
    case MCX_PEAK_DFMA: iters = 16; per_trip = kChains * kUnroll; break;
    default: iters = 1024; per_trip = 1; break;
  }
  void* scratch = nullptr;
  void* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * grid);
  if (e == cudaSuccess && atomic) e = cudaMalloc(&scratch, footprint_bytes);
  if (e == cudaSuccess && atomic) e = cudaMemset(scratch, 0, footprint_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint32_t n_elem = atomic ? (uint32_t)(footprint_bytes / elem) : 0u;
  auto launch = [&]() {
    switch (kind) {
      case MCX_PEAK_FFMA: ffma_kernel<<<grid, block, 0, s>>>(iters, 0.999f, 1e-3f, 0, (float*)out); break;
      case MCX_PEAK_IMAD: imad_kernel<<<grid, block, 0, s>>>(iters, 1013904223u, 0, (uint32_t*)out); break;
      case MCX_PEAK_PHILOX: philox_kernel<<<grid, block, 0, s>>>(iters, 12345u, 678u, 0, (uint32_t*)out); break;
      case MCX_PEAK_DFMA: dfma_kernel<<<grid, block, 0, s>>>(iters, 0.999, 1e-3, 0, (double*)out); break;
      case MCX_PEAK_HIT: hit_kernel<<<grid, block, 0, s>>>(iters, (MonBin*)scratch, n_elem); break;
      default: red_u64_kernel<<<grid, block, 0, s>>>(iters, (unsigned long long*)scratch, n_elem); break;
    }
    return cudaGetLastError();
  };
  float best_ms = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {   // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(scratch);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "peak measurement");
  if (!(best_ms > 0.f)) return fail(MCX_ERR_CUDA, "peak measurement: no elapsed time");
  *ops_per_s = threads * (double)iters * per_trip / (best_ms * 1e-3);
  return MCX_OK;
}
