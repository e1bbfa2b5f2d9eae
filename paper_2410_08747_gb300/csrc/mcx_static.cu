// mcx_static.cu -- batched tracing that allocates nothing, for callers that
// cannot call cudaMalloc/cudaFree (see mcx_batch_trace_static in mcx.h).
//
// The work list, the per-instrument device descriptors and the ticket counter
// live in one file-scope __device__ array of fixed size.  Host code reaches it
// only through the address returned by cudaGetSymbolAddress (once per device,
// with that device current); the array's name in host code is a stand-in, not
// a device address.  Compiled with -fmad=false (see mcx_tracer.cuh).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mcx_host.h"
#include "mcx_tracer.cuh"

namespace mcx {

constexpr int kStaticMaxInsts = 512;
constexpr int kStaticMaxDevices = 64;

// Byte layout of the scratch array: ticket counter, per-instrument first work
// item (prefix sums, n + 1 entries), budgets, device descriptors.
struct StaticLayout {
  static constexpr size_t ticket = 0;
  static constexpr size_t item_start = 256;
  static constexpr size_t budgets =
      item_start + (((size_t)(kStaticMaxInsts + 1) * 4 + 255) / 256) * 256;
  static constexpr size_t insts = budgets + (size_t)kStaticMaxInsts * 8;
  static constexpr size_t bytes = insts + (size_t)kStaticMaxInsts * sizeof(DevInstrument);
};

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[StaticLayout::bytes];

// The batched persistent kernel with its work list decoded from the scratch
// array: ticket t belongs to the last instrument i with item_start[i] <= t and
// covers rays [(t - item_start[i]) chunk, min(budget_i, ... + chunk)).
template <int MODE, int VOX>
__global__ void __launch_bounds__(256, (VOX & kVoxMask) ? vox_min_blocks<MODE>() : kGenericMinBlocks)
    static_batch_kernel(unsigned char* __restrict__ scratch, uint32_t n_inst, uint32_t n_items,
                        uint64_t chunk, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[64];
  __shared__ DevInstrument s_inst;
  __shared__ unsigned int s_item, s_wi_inst;
  __shared__ uint64_t s_wi_begin, s_wi_end;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + StaticLayout::ticket);
  const uint32_t* item_start = reinterpret_cast<const uint32_t*>(scratch + StaticLayout::item_start);
  const uint64_t* budgets = reinterpret_cast<const uint64_t*>(scratch + StaticLayout::budgets);
  const DevInstrument* insts = reinterpret_cast<const DevInstrument*>(scratch + StaticLayout::insts);
  const int n_warps = blockDim.x >> 5;
  BlockSmem<MODE> sm;
  sm.carve(smem, n_warps);
  for (int i = threadIdx.x; i < n_warps * kMaxComps; i += blockDim.x) sm.lost[i] = 0.0;
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  typename Prec<MODE>::Acc acc_w0, acc_wend;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(ticket, 1u);
      s_item = t;
      if (t < n_items) {
        uint32_t lo = 0, hi = n_inst;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (item_start[mid] <= t) lo = mid;
          else hi = mid;
        }
        const uint64_t b = (uint64_t)(t - item_start[lo]) * chunk;
        s_wi_inst = lo;
        s_wi_begin = b;
        s_wi_end = min(budgets[lo], b + chunk);
      }
    }
    __syncthreads();
    if (s_item >= n_items) break;
    const unsigned wi_inst = s_wi_inst;
    const uint64_t wi_begin = s_wi_begin, wi_end = s_wi_end;
    if ((int)wi_inst != cur) {
      if (cur >= 0) {
        flush_tallies(s_inst, sm.lost, n_warps, acc_w0.value(), acc_wend.value(), red);
        __syncthreads();
        for (int i = threadIdx.x; i < n_warps * kMaxComps; i += blockDim.x) sm.lost[i] = 0.0;
        acc_w0 = typename Prec<MODE>::Acc();
        acc_wend = typename Prec<MODE>::Acc();
      }
      if (threadIdx.x == 0) s_inst = insts[wi_inst];
      __syncthreads();
      load_comps(sm.comp, s_inst.comps, s_inst.n_comp);
      cur = (int)wi_inst;
    }
    __syncthreads();
    WarpLoss<MODE> loss{sm.lost + warp * kMaxComps};
    for (uint64_t base = wi_begin + warp * 32u; base < wi_end; base += blockDim.x) {
      const uint64_t id = base + lane;
      trace_ray<MODE, VOX>(s_inst, SmemTable{sm.comp, s_inst.n_comp}, PrivBins{},
                           loss,
                           sm.mu + threadIdx.x, blockDim.x, id, seed, id < wi_end, acc_w0, acc_wend);
    }
    __syncthreads();  // the shared work item is rewritten by the next ticket
  }
  if (cur >= 0) flush_tallies(s_inst, sm.lost, n_warps, acc_w0.value(), acc_wend.value(), red);
}

// one kernel per path set (a marching batch takes both traversals, one with
// optics every path)
template <int MODE>
static const void* static_kernel_mode(int vox) {
  if (vox & kOptics) return (const void*)static_batch_kernel<MODE, kVoxMask | kOptics>;
  if (vox & kVoxMarch) return (const void*)static_batch_kernel<MODE, kVoxBoth>;
  return vox ? (const void*)static_batch_kernel<MODE, kVoxWalk> : (const void*)static_batch_kernel<MODE, kVoxNone>;
}
static const void* static_kernel_fn(int precision, int vox) {
  return precision == 0 ? static_kernel_mode<0>(vox) : static_kernel_mode<1>(vox);
}

// Device address of the scratch array per device (set up on first use) and
// the host staging area for one upload; both guarded by one mutex.
static std::mutex g_static_mu;
static unsigned char* g_static_ptr[kStaticMaxDevices] = {};
static unsigned char g_host_stage[StaticLayout::bytes];

}  // namespace mcx

using namespace mcx;

extern "C" mcx_status mcx_batch_trace_static(mcx_instrument* const* insts, const uint64_t* budgets,
                                             int32_t n, uint64_t chunk_rays, uint64_t seed) {
  if (!insts || !budgets || n < 1) return fail(MCX_ERR_INVALID, "need n >= 1 instruments and budgets");
  if (n > kStaticMaxInsts)
    return fail(MCX_ERR_INVALID, "allocation-free batch takes at most %d instruments, got %d",
                kStaticMaxInsts, n);
  const uint64_t chunk = chunk_rays ? chunk_rays : (1ull << 20);
  uint64_t items = 0;
  int vox = kVoxNone;
  int n_mat = 0;
  for (int i = 0; i < n; ++i) {
    const mcx_instrument* I = insts[i];
    if (!I) return fail(MCX_ERR_INVALID, "instrument %d is NULL", i);
    if (I->device != insts[0]->device || I->precision != insts[0]->precision ||
        I->stream != insts[0]->stream)
      return fail(MCX_ERR_INVALID, "instrument %d differs in device, precision or stream", i);
    if (budgets[i] > (1ull << 62)) return fail(MCX_ERR_INVALID, "budget %d above 2^62", i);
    if (I->prop) return fail(MCX_ERR_UNSUPPORTED, "instrument %d draws from an attached proposal; use mcx_batch_trace", i);
    items += (budgets[i] + chunk - 1) / chunk;   // <= 2^32 + 2^62: cannot wrap
    if (items >= 0xFFFFFFFFull) return fail(MCX_ERR_INVALID, "too many work items; raise chunk_rays");
    vox |= I->vox_kind;
    n_mat = std::max(n_mat, I->dev.n_mat * (I->scatter ? 2 : 1));   // column rows (see the batch)
  }
  const int device = insts[0]->device;
  if (device < 0 || device >= kStaticMaxDevices) return fail(MCX_ERR_INVALID, "device ordinal %d out of range", device);
  const int precision = insts[0]->precision;
  cudaStream_t stream = insts[0]->stream;
  DeviceGuard guard(device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", device);

  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "static scratch address");
    g_static_ptr[device] = static_cast<unsigned char*>(p);
  }
  unsigned char* scratch = g_static_ptr[device];

  // stage prefix sums, budgets and descriptors in static host storage, then
  // one upload (a pageable copy returns once the bytes are staged)
  uint32_t* start = reinterpret_cast<uint32_t*>(g_host_stage + StaticLayout::item_start);
  uint64_t* bud = reinterpret_cast<uint64_t*>(g_host_stage + StaticLayout::budgets);
  DevInstrument* di = reinterpret_cast<DevInstrument*>(g_host_stage + StaticLayout::insts);
  uint32_t acc = 0;
  for (int i = 0; i < n; ++i) {
    start[i] = acc;
    acc += (uint32_t)((budgets[i] + chunk - 1) / chunk);
    bud[i] = budgets[i];
    std::memcpy(&di[i], &insts[i]->dev, sizeof(DevInstrument));
  }
  start[n] = acc;
  const size_t lo = StaticLayout::item_start;
  const size_t hi = StaticLayout::insts + (size_t)n * sizeof(DevInstrument);
  cudaError_t e = cudaMemcpyAsync(scratch + lo, g_host_stage + lo, hi - lo, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + StaticLayout::ticket, 0, sizeof(unsigned int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "static batch upload");
  if (items == 0) return MCX_OK;

  int n_sm = 0, bpsm = 0;
  const int block = 256;
  const size_t smem = block_smem_bytes((vox & kVoxMask) ? n_mat : 0, block, precision);
  const void* fn = static_kernel_fn(precision, vox);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "static batch shared memory");
  }
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, fn, block, smem) != cudaSuccess || bpsm < 1)
    bpsm = 1;
  uint32_t n_inst = (uint32_t)n, n_items = (uint32_t)items;
  uint64_t ch = chunk, sd = seed;
  void* args[] = {&scratch, &n_inst, &n_items, &ch, &sd};
  e = cudaLaunchKernel(fn, dim3(n_sm * bpsm), dim3(block), args, smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "static batch launch");
  for (int i = 0; i < n; ++i) insts[i]->n_emit += budgets[i];
  return MCX_OK;
}
