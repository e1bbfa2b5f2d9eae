// mcx_starts.cu -- ray-start buffers: the plain source sampler writing starts,
// and tracing from given starts (with each ray's detected weight).  This is
// how training histories are produced and how an external proposal (the
// learned one) feeds the tracer.  Compiled with -fmad=false.
#include "mcx_host.h"
#include "mcx_tracer.cuh"

namespace mcx {

// Starts of rays [begin, begin + n): the draw contract's binary32 source
// point, aim point and energy, and the initial weight (Kramers factor, a
// Gaussian source's divergence weight).
__global__ void __launch_bounds__(256) sample_starts_kernel(const DevInstrument I, uint64_t begin,
                                                            uint64_t n, uint64_t seed,
                                                            float* __restrict__ out) {
  __shared__ DevComp S;
  if (threadIdx.x == 0) S = I.comps[0];
  __syncthreads();
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (uint64_t)gridDim.x * blockDim.x) {
    RayStream rs;
    rs.init(begin + r, (uint32_t)I.instr_id, seed);
    float sx, sy, tx, ty, E;
    sample_start<float>(S, rs, sx, sy, tx, ty, E);
    const float w = source_weight<float>(S, sx, sy, tx, ty, E);
    out[r] = sx;
    out[n + r] = sy;
    out[2 * n + r] = E;
    out[3 * n + r] = tx;
    out[4 * n + r] = ty;
    out[5 * n + r] = w;
  }
}

cudaError_t sample_starts_async(const DevInstrument& d, uint64_t begin, uint64_t n, uint64_t seed,
                                float* d_starts, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int dev = 0, n_sm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t need = (n + 255) / 256;
  const unsigned grid = (unsigned)(need < (uint64_t)n_sm * 8 ? need : (uint64_t)n_sm * 8);
  sample_starts_kernel<<<grid, 256, 0, s>>>(d, begin, n, seed, d_starts);
  return cudaGetLastError();
}

}  // namespace mcx

using namespace mcx;

extern "C" mcx_status mcx_sample_starts(mcx_instrument* I, uint64_t ray_begin, uint64_t n,
                                        uint64_t seed, float* d_starts) {
  if (!I || (!d_starts && n)) return fail(MCX_ERR_INVALID, "NULL argument");
  if (ray_begin + n < ray_begin || ray_begin + n > (1ull << 62))
    return fail(MCX_ERR_INVALID, "ray ids must stay below 2^62");
  if (n == 0) return MCX_OK;
  DeviceGuard guard(I->device);
  cudaError_t e = sample_starts_async(I->dev, ray_begin, n, seed, d_starts, I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sample starts");
  return MCX_OK;
}

extern "C" mcx_status mcx_trace_starts(mcx_instrument* I, const float* d_starts, uint64_t n,
                                       uint64_t ray_base, float* d_det_w) {
  if (!I || (!d_starts && n)) return fail(MCX_ERR_INVALID, "NULL argument");
  if (I->precision != MCX_PREC_MIXED)
    return fail(MCX_ERR_UNSUPPORTED, "tracing given starts needs the mixed precision form");
  if (I->scatter)
    return fail(MCX_ERR_UNSUPPORTED, "a scattering phantom draws from the ray's own stream, which given starts lack");
  if (ray_base + n < ray_base || ray_base + n > (1ull << 62))
    return fail(MCX_ERR_INVALID, "ray ids must stay below 2^62");
  if (n == 0) return MCX_OK;
  DeviceGuard guard(I->device);
  DevInstrument d = I->dev;
  d.ext = d_starts;
  d.ext_base = ray_base;
  d.ext_n = n;
  d.det_w = d_det_w;
  cudaError_t e = trace_dispatch(I, d, ray_base, ray_base + n, 0);
  if (e != cudaSuccess) return cuda_fail(e, "trace starts");
  I->n_emit += n;
  return MCX_OK;
}
