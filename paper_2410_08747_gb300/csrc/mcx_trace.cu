// mcx_trace.cu -- the single-instrument tracing kernel and its launchers.
// Compiled with -fmad=false (see mcx_tracer.cuh).
#include "mcx_tracer.cuh"

namespace mcx {

// The generic tracing kernel: any instrument, its component table copied
// into shared memory by each block.  VOX selects the paths the instantiation
// carries (its phantom traversal, kOptics).
template <int MODE, int VOX>
__global__ void __launch_bounds__(256, (VOX & kScatter) ? kScatterMinBlocksGeneric
                                       : ((VOX & kVoxMask) ? vox_min_blocks<MODE>() : kGenericMinBlocks))
    trace_kernel(const DevInstrument I, uint64_t begin,
                                                    uint64_t end, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[64];
  trace_rays<MODE, VOX, SmemTable>(I, begin, end, seed, smem, red);
}

size_t trace_smem_bytes(int n_comp, int n_mat, int block, int precision, bool has_phantom, int n_priv) {
  (void)n_comp;
  return block_smem_bytes(has_phantom ? n_mat : 0, block, precision, true, n_priv);
}

template <typename K>
static int occupancy_of(K kernel, int block, size_t smem) {
  int n = 0;
  // opt in first, as the launch does, so that static plus dynamic shared
  // memory above 48 KB is counted against the real limit
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) == cudaSuccess ? n : 0;
}

// The instantiation for an instrument's path set: its phantom traversal
// alone, the optics alone, or everything when both are present; in the mixed
// form a march phantom that scatters (kScatter given) alone takes the
// refilling kernel.
static int kernel_kind(int precision, int vox_kind) {
  const bool scatter = (vox_kind & kScatter) != 0;
  vox_kind &= ~kScatter;
  if (vox_kind & kOptics) return (vox_kind & kVoxMask) ? (kVoxMask | kOptics) : kOptics;
  if (scatter && precision == 1 && vox_kind == kVoxMarch) return kVoxMarch | kScatter;
  return vox_kind & kVoxMask;
}

template <int MODE>
static int occupancy_mode(int vk, int block, size_t smem) {
  switch (vk) {
    case kVoxWalk: return occupancy_of(trace_kernel<MODE, kVoxWalk>, block, smem);
    case kVoxMarch: return occupancy_of(trace_kernel<MODE, kVoxMarch>, block, smem);
    case kOptics: return occupancy_of(trace_kernel<MODE, kOptics>, block, smem);
    case kVoxMask | kOptics: return occupancy_of(trace_kernel<MODE, kVoxMask | kOptics>, block, smem);
    case kVoxMarch | kScatter:
      if constexpr (MODE == 1) return occupancy_of(trace_kernel<1, kVoxMarch | kScatter>, block, smem);
      return 0;
    default: return occupancy_of(trace_kernel<MODE, kVoxNone>, block, smem);
  }
}

int trace_occupancy(int precision, int vox_kind, int block, size_t smem) {
  const int vk = kernel_kind(precision, vox_kind);
  return precision == 0 ? occupancy_mode<0>(vk, block, smem) : occupancy_mode<1>(vk, block, smem);
}

template <int MODE, int VOX>
static void launch_one(const DevInstrument& inst, uint64_t begin, uint64_t end, uint64_t seed,
                       int grid, const LaunchShape& shape, cudaStream_t stream) {
  // the phantom kernels also hold the ray-ordering buffers in static shared
  // memory, so they opt in above 48 KB of static plus dynamic memory
  if (VOX || shape.smem > 48 * 1024)
    cudaFuncSetAttribute(trace_kernel<MODE, VOX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)shape.smem);
  trace_kernel<MODE, VOX><<<grid, shape.block, shape.smem, stream>>>(inst, begin, end, seed);
}

template <int MODE>
static void launch_mode(int vk, const DevInstrument& inst, uint64_t begin, uint64_t end, uint64_t seed,
                        int grid, const LaunchShape& shape, cudaStream_t stream) {
  switch (vk) {
    case kVoxWalk: launch_one<MODE, kVoxWalk>(inst, begin, end, seed, grid, shape, stream); break;
    case kVoxMarch: launch_one<MODE, kVoxMarch>(inst, begin, end, seed, grid, shape, stream); break;
    case kOptics: launch_one<MODE, kOptics>(inst, begin, end, seed, grid, shape, stream); break;
    case kVoxMask | kOptics:
      launch_one<MODE, kVoxMask | kOptics>(inst, begin, end, seed, grid, shape, stream);
      break;
    case kVoxMarch | kScatter:
      if constexpr (MODE == 1) launch_one<1, kVoxMarch | kScatter>(inst, begin, end, seed, grid, shape, stream);
      break;
    default: launch_one<MODE, kVoxNone>(inst, begin, end, seed, grid, shape, stream); break;
  }
}

cudaError_t launch_trace(const DevInstrument& inst, int precision, uint64_t begin, uint64_t end,
                         uint64_t seed, const LaunchShape& shape, cudaStream_t stream) {
  if (end <= begin) return cudaSuccess;
  const uint64_t n = end - begin;
  const uint64_t need = (n + shape.block - 1) / shape.block;
  const int grid = (int)(need < (uint64_t)shape.grid ? need : (uint64_t)shape.grid);
  const int vk = kernel_kind(precision, inst.vox != nullptr ? (inst.vox_kind | (inst.sc32 ? kScatter : 0))
                                                           : (inst.vox_kind & kOptics));
  if (precision == 0) launch_mode<0>(vk, inst, begin, end, seed, grid, shape, stream);
  else launch_mode<1>(vk, inst, begin, end, seed, grid, shape, stream);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ ray order of a phantom trace
// Counting sort of a chunk's ray ids by aim-point tile: the keys with a
// histogram in global memory (65,536 tiles: 256 KB, more than a block's
// shared memory; 2^24 ids give ~256 adds per counter), one block's
// exclusive scan over the tiles, and a scatter (the order of ids within a
// tile is whatever the atomics give).
template <int MODE>
__global__ void __launch_bounds__(256) tile_key_kernel(const DevInstrument I, uint64_t begin, uint32_t n,
                                                       uint64_t seed, uint16_t* __restrict__ keys,
                                                       uint32_t* __restrict__ hist) {
  __shared__ DevComp S;
  if (threadIdx.x == 0) S = I.comps[0];
  __syncthreads();
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned k = aim_tile<MODE>(I, S, begin + p, seed);
    keys[p] = (uint16_t)k;
    atomicAdd(&hist[k], 1u);
  }
}

// hist[t] becomes the number of keys below tile t (one block of 1024 threads)
__global__ void __launch_bounds__(1024) tile_scan_kernel(uint32_t* __restrict__ hist) {
  constexpr int per = kTiles / 1024;
  __shared__ unsigned part[32];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  unsigned own = 0u;
#pragma unroll
  for (int j = 0; j < per; ++j) own += hist[threadIdx.x * per + j];
  unsigned x = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31u) part[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned v = part[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= (unsigned)o) v += y;
    }
    part[lane] = v;
  }
  __syncthreads();
  unsigned run = x - own + (warp ? part[warp - 1] : 0u);
#pragma unroll
  for (int j = 0; j < per; ++j) {
    const unsigned c = hist[threadIdx.x * per + j];
    hist[threadIdx.x * per + j] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(256) tile_scatter_kernel(const uint16_t* __restrict__ keys, uint32_t n,
                                                           uint32_t* __restrict__ offs,
                                                           uint32_t* __restrict__ perm) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    perm[atomicAdd(&offs[keys[p]], 1u)] = p;
}

cudaError_t launch_ray_order(const DevInstrument& inst, int precision, uint64_t begin, uint64_t end,
                             uint64_t seed, uint16_t* keys, uint32_t* hist, uint32_t* perm,
                             cudaStream_t stream) {
  static_assert(kTiles % 1024 == 0, "tile scan");
  if (end <= begin) return cudaSuccess;
  const uint32_t n = (uint32_t)(end - begin);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned need = (n + 255) / 256;
  const unsigned grid = need < (unsigned)sms * 4 ? need : (unsigned)sms * 4;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kTiles, stream);
  if (e != cudaSuccess) return e;
  if (precision == 0) tile_key_kernel<0><<<grid, 256, 0, stream>>>(inst, begin, n, seed, keys, hist);
  else tile_key_kernel<1><<<grid, 256, 0, stream>>>(inst, begin, n, seed, keys, hist);
  tile_scan_kernel<<<1, 1024, 0, stream>>>(hist);
  tile_scatter_kernel<<<grid, 256, 0, stream>>>(keys, n, hist, perm);
  return cudaGetLastError();
}

__global__ void philox_fill_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                   size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* a = in + 6 * i;
  uint32_t* o = out + 4 * i;
  philox4x32_10(a[0], a[1], a[2], a[3], a[4], a[5], o[0], o[1], o[2], o[3]);
}

cudaError_t launch_philox_fill(const uint32_t* d_in, uint32_t* d_out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  philox_fill_kernel<<<grid, block, 0, s>>>(d_in, d_out, n);
  return cudaGetLastError();
}

}  // namespace mcx

namespace mcx {

__global__ void convert_fill_kernel(const double* __restrict__ in, float* __restrict__ of,
                                    double* __restrict__ od, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = d2f(in[i]);
  of[i] = f;
  od[i] = f2d(f);
}

cudaError_t launch_convert_fill(const double* in, float* of, double* od, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int block = 256;
  convert_fill_kernel<<<(unsigned)((n + block - 1) / block), block, 0, s>>>(in, of, od, n);
  return cudaGetLastError();
}

// Monitor readout: split the 24-byte bins into three contiguous arrays so the
// host copy is three plain DMA transfers (any output may be null).
__global__ void split_bins_kernel(const MonBin* __restrict__ in, size_t nb,
                                  unsigned long long* __restrict__ N, double* __restrict__ sw,
                                  double* __restrict__ sw2) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) {
    const MonBin b = in[i];
    if (N) N[i] = b.N;
    if (sw) sw[i] = b.sw;
    if (sw2) sw2[i] = b.sw2;
  }
}

// Monitor totals: each block sums its grid-stride share of the bins (count
// exactly in 64 bits, the two sums in binary64), reduces over its warps and
// adds the result to out[0..2] (zeroed by the caller) with one atomic each.
__global__ void __launch_bounds__(256) total_bins_kernel(const MonBin* __restrict__ in, size_t nb,
                                                         unsigned long long* __restrict__ outN,
                                                         double* __restrict__ outw) {
  __shared__ unsigned long long sN[8];
  __shared__ double s1[8], s2[8];
  unsigned long long n = 0;
  double a = 0.0, b = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) {
    const MonBin x = in[i];
    n += x.N;
    a += x.sw;
    b += x.sw2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_down_sync(0xffffffffu, n, o);
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sN[warp] = n; s1[warp] = a; s2[warp] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { n += sN[w]; a += s1[w]; b += s2[w]; }
    atomicAdd(outN, n);
    atomicAdd(outw, a);
    atomicAdd(outw + 1, b);
  }
}

cudaError_t launch_total_bins(const MonBin* in, size_t nb, unsigned long long* outN, double* outw,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(outN, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(outw, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess || nb == 0) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t need = (nb + 255) / 256;
  const size_t grid = need < (size_t)sms * 4 ? need : (size_t)sms * 4;
  total_bins_kernel<<<(unsigned)grid, 256, 0, s>>>(in, nb, outN, outw);
  return cudaGetLastError();
}

cudaError_t launch_split_bins(const MonBin* in, size_t nb, unsigned long long* N, double* sw,
                              double* sw2, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 256;
  const size_t need = (nb + block - 1) / block;
  const size_t grid = need < (size_t)sms * 8 ? need : (size_t)sms * 8;
  split_bins_kernel<<<(unsigned)grid, block, 0, s>>>(in, nb, N, sw, sw2);
  return cudaGetLastError();
}

}  // namespace mcx
