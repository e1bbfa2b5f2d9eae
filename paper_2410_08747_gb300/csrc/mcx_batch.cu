// mcx_batch.cu -- many instruments traced by one persistent launch: the work
// list, the persistent kernel, CUDA-graph capture and replay, and the
// launch-shape autotuner.  Compiled with -fmad=false (see mcx_tracer.cuh).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mcx_host.h"
#include "mcx_tracer.cuh"

namespace mcx {

// The generic batch kernel: every instrument's table from shared memory
// (VOX: the union of the instruments' phantom traversals).
template <int MODE, int VOX>
__global__ void __launch_bounds__(256, (VOX & kVoxMask) ? vox_min_blocks<MODE>() : kGenericMinBlocks)
    batch_kernel(const DevInstrument* __restrict__ insts, const WorkItem* __restrict__ items,
                 uint32_t n_items, unsigned int* __restrict__ ticket, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[64];
  batch_rays<MODE, VOX, GenericFamilies>(insts, items, n_items, ticket, seed, smem, red);
}

// one kernel per path set; a batch that marches takes the kernel that can
// take both traversals, one with optics the kernel with every path
template <int MODE>
static const void* batch_kernel_mode(int vox) {
  if (vox & kOptics) return (const void*)batch_kernel<MODE, kVoxMask | kOptics>;
  if (vox & kVoxMarch) return (const void*)batch_kernel<MODE, kVoxBoth>;
  return vox ? (const void*)batch_kernel<MODE, kVoxWalk> : (const void*)batch_kernel<MODE, kVoxNone>;
}
static const void* batch_kernel_fn(int precision, int vox) {
  return precision == 0 ? batch_kernel_mode<0>(vox) : batch_kernel_mode<1>(vox);
}

// A learned wave's starts of one instrument in aim-tile order:
// out[row][p] = in[row][perm[p]] over the 6 rows of n starts.  Given starts
// carry every ray's randomness, so the order in which they are traced
// changes nothing but the order of the monitors' atomic additions.
__global__ void __launch_bounds__(256) gather_starts_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                            const uint32_t* __restrict__ perm, uint32_t n) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t q = perm[p];
#pragma unroll
    for (int r = 0; r < 6; ++r) out[(size_t)r * n + p] = in[(size_t)r * n + q];
  }
}

}  // namespace mcx

using namespace mcx;

struct mcx_batch {
  std::vector<mcx_instrument*> insts;
  std::vector<uint64_t> budgets;
  int device = 0;
  int precision = 0;
  int vox = kVoxNone;   // union of the instruments' phantom traversals
  int n_mat = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  DevInstrument* d_insts = nullptr;
  WorkItem* d_items = nullptr;
  size_t items_cap = 0;
  uint32_t n_items = 0;
  unsigned int* d_ticket = nullptr;
  mcx_batch_options opt{};
  LaunchShape shape{};
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t knode = nullptr;
  // kernel arguments (the graph node's parameters point here)
  uint64_t arg_seed = 0;
  const void* spec_kernel = nullptr;   // compiled by families, if enabled
  std::vector<int> fam_of;             // each instrument's family (compiled kernel)
  // instruments with an attached proposal: the starts of one wave of their
  // rays, the wave's descriptors and work list
  float* wave_starts = nullptr;
  float* wave_sorted = nullptr;     // a phantom instrument's slice in aim-tile order
  uint16_t* ord_keys = nullptr;     // its tile keys, counters and permutation
  uint32_t* ord_hist = nullptr;
  uint32_t* ord_perm = nullptr;
  DevInstrument* d_insts_wave = nullptr;
  WorkItem* d_items_wave = nullptr;
  size_t items_wave_cap = 0;
};

// The batch's tracing kernel: compiled by families, or the generic one.
static const void* batch_fn(const mcx_batch* B) {
  return B->spec_kernel ? B->spec_kernel : batch_kernel_fn(B->precision, B->vox);
}

static void drop_graph(mcx_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
  B->knode = nullptr;
}

static int occupancy(mcx_batch* B, int block, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_fn(B), block,
                                                    smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// Bytes of instrument I's monitors that live in global memory (those too
// large for a block-private copy).
static uint64_t global_monitor_bytes(const mcx_instrument* I) {
  uint64_t b = 0;
  for (size_t c = 0; c < I->comps.size(); ++c)
    if (I->mon_off[c] >= 0 && I->comps[c].priv < 0) b += (uint64_t)I->mon_bins[c] * sizeof(MonBin);
  return b;
}

constexpr uint64_t kFootprintBytes = 16ull << 20;   // global monitors above this: items cut by the rule below
constexpr uint64_t kMinItemRays = 1ull << 12;       // below this the per-item costs grow

// Rays per work item of instrument i with `budget` rays in this plan.  The
// global atomics of a large detector keep their rate only while the bins
// they hit fit in the L2 (about 2.1e11 atomics/s up to ~128 MB, 2-3x fewer
// beyond), and the items the persistent grid holds at once belong to
// consecutive instruments: an instrument whose global monitors exceed
// kFootprintBytes is cut into items of c rays, c the largest power of two
// with grid x c <= budget (the items in flight then belong to about one
// instrument), at least kMinItemRays and at most `chunk`.  Other instruments
// keep `chunk` (their per-item costs, such as flushing block-private
// monitors, favour long items).  Measured on the 376-instrument batch with
// the L2-hinted monitor updates, compiled (rays/s) by the bound on the rays
// in flight: budget 5.41e10, budget / 2 5.37e10, / 4 5.31e10, / 8 5.24e10,
// / 16 5.16e10 (without the hint / 4 had been best).
static uint64_t item_rays(const mcx_batch* B, size_t i, uint64_t budget, uint64_t chunk) {
  if (global_monitor_bytes(B->insts[i]) <= kFootprintBytes) return chunk;
  const uint64_t grid = B->shape.grid > 0 ? (uint64_t)B->shape.grid : 1;
  const uint64_t m = budget / grid;
  uint64_t p = 1;
  while (p * 2 <= m) p *= 2;
  return std::min(chunk, std::max(p, kMinItemRays));
}

// Cuts every budget into work items (ordered by instrument; item_rays rays
// each) and uploads the list.
static mcx_status plan(mcx_batch* B, const std::vector<uint64_t>& budgets, uint64_t chunk) {
  // count first: a list that would not fit is refused before it is built
  uint64_t count = 0;
  for (size_t i = 0; i < B->insts.size(); ++i) {
    const uint64_t c = item_rays(B, i, budgets[i], chunk);
    count += budgets[i] / c + (budgets[i] % c != 0);
    if (count > 0xFFFFFFF0ull) return fail(MCX_ERR_INVALID, "too many work items; raise chunk_rays");
  }
  std::vector<WorkItem> items;
  items.reserve((size_t)count);
  for (size_t i = 0; i < B->insts.size(); ++i) {
    const uint64_t c = item_rays(B, i, budgets[i], chunk);
    for (uint64_t b = 0; b < budgets[i]; b += c)
      items.push_back(WorkItem{b, std::min(budgets[i], b + c), (uint32_t)i, 0u});
  }
  if (items.size() > 0xFFFFFFF0ull) return fail(MCX_ERR_INVALID, "too many work items; raise chunk_rays");
  if (items.size() > B->items_cap) {
    if (B->d_items) cudaFree(B->d_items);
    B->d_items = nullptr;
    B->items_cap = 0;
    cudaError_t e = cudaMalloc(&B->d_items, sizeof(WorkItem) * std::max<size_t>(items.size(), 1));
    if (e != cudaSuccess) return cuda_fail(e, "work list");
    B->items_cap = items.size();
  }
  if (!items.empty()) {
    cudaError_t e = cudaMemcpyAsync(B->d_items, items.data(), sizeof(WorkItem) * items.size(),
                                    cudaMemcpyHostToDevice, B->stream);
    if (e != cudaSuccess) return cuda_fail(e, "work list upload");
  }
  B->n_items = (uint32_t)items.size();
  drop_graph(B);
  return MCX_OK;
}

static mcx_status set_shape(mcx_batch* B, const mcx_batch_options& o) {
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, B->device);
  const int block = o.block_size ? o.block_size : 256;
  const size_t smem = block_smem_bytes((B->vox & kVoxMask) ? B->n_mat : 0, block, B->precision);
  if (smem > 48 * 1024)   // before the occupancy query, which counts it
    cudaFuncSetAttribute(batch_fn(B), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int bpsm = o.blocks_per_sm ? o.blocks_per_sm : occupancy(B, block, smem);
  B->shape.block = block;
  B->shape.smem = smem;
  B->shape.grid = n_sm * bpsm;
  B->opt = o;
  if (!B->opt.chunk_rays) B->opt.chunk_rays = 1ull << 20;
  drop_graph(B);
  return MCX_OK;
}

static mcx_status launch_direct(mcx_batch* B, uint64_t seed, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(B->d_ticket, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail(e, "ticket reset");
  B->arg_seed = seed;
  void* args[] = {&B->d_insts, &B->d_items, &B->n_items, &B->d_ticket, &B->arg_seed};
  e = cudaLaunchKernel(batch_fn(B), dim3(B->shape.grid),
                       dim3(B->shape.block), args, B->shape.smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return MCX_OK;
}

// Records [ticket reset, persistent kernel] as a CUDA graph on a private
// stream (the legacy default stream cannot be captured).
static mcx_status capture(mcx_batch* B, uint64_t seed) {
  cudaError_t e = cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  mcx_status s = launch_direct(B, seed, B->capture_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(B->capture_stream, &g);
  if (s != MCX_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g, nodes.data(), &n);
  cudaGraphNode_t kn = nullptr;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) kn = nd;
  }
  cudaGraphExec_t ex = nullptr;
  e = kn ? cudaGraphInstantiate(&ex, g, 0) : cudaErrorInvalidValue;
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "graph instantiate");
  }
  B->graph = g;
  B->exec = ex;
  B->knode = kn;
  return MCX_OK;
}

static mcx_status run(mcx_batch* B, uint64_t seed) {
  if (B->n_items == 0) return MCX_OK;
  if (!B->opt.use_graph) return launch_direct(B, seed, B->stream);
  if (!B->exec) {
    mcx_status s = capture(B, seed);
    if (s != MCX_OK) return s;
  }
  B->arg_seed = seed;
  void* args[] = {&B->d_insts, &B->d_items, &B->n_items, &B->d_ticket, &B->arg_seed};
  cudaKernelNodeParams p{};
  p.func = (void*)batch_fn(B);
  p.gridDim = dim3(B->shape.grid);
  p.blockDim = dim3(B->shape.block);
  p.sharedMemBytes = (unsigned)B->shape.smem;
  p.kernelParams = args;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(B->exec, B->knode, &p);
  if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return MCX_OK;
}

// Instruments a batch traces from staged starts: those drawing from an
// attached proposal (mcx_proposal_attach), and in the mixed form those with
// a phantom that does not scatter (their own source sampled into the
// buffer: tracing given starts equals tracing the source, and it lets the
// batch put a phantom's rays in aim-tile order, as a single instrument's
// phantom trace orders its ids).
static bool staged(const mcx_batch* B, const mcx_instrument* I) {
  return I->prop != nullptr || (B->precision == MCX_PREC_MIXED && I->has_phantom && !I->scatter);
}

// A batch with staged instruments: their rays are traced in waves of at
// most kPropChunk: per wave each such instrument's next rays are sampled
// (by its proposal, or by its own source) into its slice of the wave's
// start buffer, behind a phantom the slice is put in aim-tile order (so that
// a block's rays cross one patch of the phantom), and one persistent launch
// traces the wave's work items (the first wave also carries every other
// instrument's whole budget), the staged instruments reading their starts
// from the buffer.  Direct launches, stream-ordered.
static mcx_status run_staged(mcx_batch* B, uint64_t seed) {
  const size_t n = B->insts.size();
  const uint64_t chunk = B->opt.chunk_rays ? B->opt.chunk_rays : (1ull << 20);
  std::vector<int> learned;   // the staged instruments
  for (size_t i = 0; i < n; ++i) {
    if (!staged(B, B->insts[i])) continue;
    if (B->insts[i]->prop) {
      const mcx_status st = proposal_check(B->insts[i]->prop, B->stream);
      if (st != MCX_OK) return st;
    }
    learned.push_back((int)i);
  }
  cudaError_t e = cudaSuccess;
  bool phantom = false;
  for (int i : learned) phantom = phantom || B->insts[i]->has_phantom;
  if (!B->wave_starts) e = cudaMalloc(&B->wave_starts, sizeof(float) * 6 * kPropChunk);
  if (e == cudaSuccess && !B->d_insts_wave) e = cudaMalloc(&B->d_insts_wave, sizeof(DevInstrument) * n);
  if (phantom && e == cudaSuccess && !B->wave_sorted) e = cudaMalloc(&B->wave_sorted, sizeof(float) * 6 * kPropChunk);
  if (phantom && e == cudaSuccess && !B->ord_keys) e = cudaMalloc(&B->ord_keys, sizeof(uint16_t) * kPropChunk);
  if (phantom && e == cudaSuccess && !B->ord_perm) e = cudaMalloc(&B->ord_perm, sizeof(uint32_t) * kPropChunk);
  if (phantom && e == cudaSuccess && !B->ord_hist) e = cudaMalloc(&B->ord_hist, sizeof(uint32_t) * (kTiles + 64));
  if (e != cudaSuccess) return cuda_fail(e, "staged batch buffers");
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, B->device);
  std::vector<uint64_t> next(n, 0);
  for (bool first = true;; first = false) {
    std::vector<DevInstrument> h(n);
    for (size_t i = 0; i < n; ++i) {
      h[i] = B->insts[i]->dev;
      if (B->spec_kernel) h[i].family = B->fam_of[i];
    }
    std::vector<WorkItem> items;
    uint64_t used = 0;
    for (int i : learned) {
      mcx_instrument* I = B->insts[i];
      const uint64_t take = std::min(B->budgets[i] - next[i], kPropChunk - used);
      if (take == 0) continue;
      float* slice = B->wave_starts + 6 * used;   // rows of `take`
      e = I->prop ? proposal_sample_async(I->prop, I->dev, next[i], take, seed, I->prop_angle, slice, B->stream)
                  : sample_starts_async(I->dev, next[i], take, seed, slice, B->stream);
      if (e != cudaSuccess) return cuda_fail(e, "batch sample");
      h[i].ext = slice;
      h[i].ext_base = next[i];
      h[i].ext_n = take;
      h[i].det_w = nullptr;
      if (I->has_phantom) {
        float* sorted = B->wave_sorted + 6 * used;
        e = launch_ray_order(h[i], B->precision, next[i], next[i] + take, seed, B->ord_keys, B->ord_hist,
                             B->ord_perm, B->stream);
        const uint64_t need = (take + 255) / 256;
        const unsigned grid = (unsigned)(need < (uint64_t)n_sm * 8 ? need : (uint64_t)n_sm * 8);
        if (e == cudaSuccess) {
          gather_starts_kernel<<<grid, 256, 0, B->stream>>>(slice, sorted, B->ord_perm, (uint32_t)take);
          e = cudaGetLastError();
        }
        if (e != cudaSuccess) return cuda_fail(e, "staged batch ray order");
        h[i].ext = sorted;
      }
      // a wave holds at most kPropChunk learned rays: cut them into items
      // small enough that every resident block gets several
      const uint64_t per = (take + 4ull * (uint64_t)B->shape.grid - 1) / (4ull * (uint64_t)B->shape.grid);
      const uint64_t lc = std::min(chunk, std::max<uint64_t>(1024, (per + 127) / 128 * 128));
      for (uint64_t b = next[i]; b < next[i] + take; b += lc)
        items.push_back(WorkItem{b, std::min(next[i] + take, b + lc), (uint32_t)i, 0u});
      next[i] += take;
      used += take;
    }
    if (first) {
      uint64_t count = items.size();
      for (size_t i = 0; i < n; ++i)
        if (!staged(B, B->insts[i])) {
          const uint64_t c = item_rays(B, i, B->budgets[i], chunk);
          count += B->budgets[i] / c + (B->budgets[i] % c != 0);
          if (count > 0xFFFFFFF0ull) return fail(MCX_ERR_INVALID, "too many work items; raise chunk_rays");
        }
    }
    if (first)
      for (size_t i = 0; i < n; ++i)
        if (!staged(B, B->insts[i])) {
          const uint64_t c = item_rays(B, i, B->budgets[i], chunk);
          for (uint64_t b = 0; b < B->budgets[i]; b += c)
            items.push_back(WorkItem{b, std::min(B->budgets[i], b + c), (uint32_t)i, 0u});
        }
    if (items.empty()) break;
    if (items.size() > 0xFFFFFFF0ull) return fail(MCX_ERR_INVALID, "too many work items; raise chunk_rays");
    if (items.size() > B->items_wave_cap) {
      if (B->d_items_wave) cudaFree(B->d_items_wave);
      B->d_items_wave = nullptr;
      B->items_wave_cap = 0;
      e = cudaMalloc(&B->d_items_wave, sizeof(WorkItem) * items.size());
      if (e != cudaSuccess) return cuda_fail(e, "staged batch work list");
      B->items_wave_cap = items.size();
    }
    // pageable copies: they return once the host bytes are staged
    e = cudaMemcpyAsync(B->d_insts_wave, h.data(), sizeof(DevInstrument) * n, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B->d_items_wave, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                          B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_ticket, 0, sizeof(unsigned int), B->stream);
    if (e != cudaSuccess) return cuda_fail(e, "staged batch upload");
    uint32_t n_items = (uint32_t)items.size();
    uint64_t sd = seed;
    void* args[] = {&B->d_insts_wave, &B->d_items_wave, &n_items, &B->d_ticket, &sd};
    e = cudaLaunchKernel(batch_fn(B), dim3(B->shape.grid), dim3(B->shape.block), args, B->shape.smem,
                         B->stream);
    if (e != cudaSuccess) return cuda_fail(e, "staged batch launch");
  }
  return MCX_OK;
}

extern "C" mcx_status mcx_batch_create(mcx_instrument* const* insts, const uint64_t* budgets, int32_t n,
                                       const mcx_batch_options* opt, mcx_batch** out) {
  if (!out) return fail(MCX_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!insts || !budgets || n < 1) return fail(MCX_ERR_INVALID, "need n >= 1 instruments and budgets");
  for (int i = 0; i < n; ++i) {
    if (!insts[i]) return fail(MCX_ERR_INVALID, "instrument %d is NULL", i);
    if (insts[i]->device != insts[0]->device || insts[i]->precision != insts[0]->precision ||
        insts[i]->stream != insts[0]->stream)
      return fail(MCX_ERR_INVALID, "instrument %d differs in device, precision or stream", i);
    if (budgets[i] > (1ull << 62)) return fail(MCX_ERR_INVALID, "budget %d above 2^62", i);
  }
  mcx_batch_options o{};
  if (opt) o = *opt;
  else o.use_graph = 1;
  if (o.block_size && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32))
    return fail(MCX_ERR_INVALID, "block_size must be a multiple of 32 in [32, 256]");
  if (o.blocks_per_sm < 0) return fail(MCX_ERR_INVALID, "blocks_per_sm must be >= 0");
  DeviceGuard guard(insts[0]->device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device");
  mcx_batch* B = new mcx_batch();
  B->device = insts[0]->device;
  B->precision = insts[0]->precision;
  B->stream = insts[0]->stream;
  B->insts.assign(insts, insts + n);
  B->budgets.assign(budgets, budgets + n);
  std::vector<DevInstrument> h(n);
  for (int i = 0; i < n; ++i) {
    h[i] = insts[i]->dev;
    B->vox |= insts[i]->vox_kind;
    // rows of the per-thread material column: a scattering phantom adds its sums
    B->n_mat = std::max(B->n_mat, insts[i]->dev.n_mat * (insts[i]->scatter ? 2 : 1));
  }
  cudaError_t e = cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_insts, sizeof(DevInstrument) * n);
  if (e == cudaSuccess) e = cudaMalloc(&B->d_ticket, 256);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_insts, h.data(), sizeof(DevInstrument) * n, cudaMemcpyHostToDevice, B->stream);
  if (e != cudaSuccess) {
    mcx_status s = cuda_fail(e, "batch create");
    mcx_batch_destroy(B);
    return s;
  }
  set_shape(B, o);
  mcx_status s = plan(B, B->budgets, B->opt.chunk_rays);
  if (s == MCX_OK) {
    e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "batch create");
  }
  if (s != MCX_OK) {
    mcx_batch_destroy(B);
    return s;
  }
  *out = B;
  return MCX_OK;
}

extern "C" mcx_status mcx_batch_trace(mcx_batch* B, uint64_t seed) {
  if (!B) return fail(MCX_ERR_INVALID, "batch is NULL");
  DeviceGuard guard(B->device);
  bool any_staged = false;
  for (auto* I : B->insts) any_staged = any_staged || staged(B, I);
  mcx_status s = any_staged ? run_staged(B, seed) : run(B, seed);
  if (s != MCX_OK) return s;
  for (size_t i = 0; i < B->insts.size(); ++i) B->insts[i]->n_emit += B->budgets[i];
  return MCX_OK;
}

extern "C" mcx_status mcx_batch_specialize(mcx_batch* B, int32_t enable) {
  if (!B) return fail(MCX_ERR_INVALID, "batch is NULL");
  DeviceGuard guard(B->device);
  const int n = (int)B->insts.size();
  std::vector<DevInstrument> h(n);
  const void* k = nullptr;
  if (enable) {
    std::vector<int> fam_of;
    const auto fams = batch_families(B->insts, fam_of);
    if (fams.size() > 8) return fail(MCX_ERR_UNSUPPORTED, "%zu instrument families, at most 8", fams.size());
    if (!tables_finite(B->insts)) return fail(MCX_ERR_UNSUPPORTED, "a component parameter is not finite");
    mcx_status st = compile_batch(batch_source(B->insts, fams, B->precision, B->vox), &k);
    if (st != MCX_OK) return st;
    for (int i = 0; i < n; ++i) {
      h[i] = B->insts[i]->dev;
      h[i].family = fam_of[i];
    }
    B->fam_of = fam_of;
  } else {
    for (int i = 0; i < n; ++i) h[i] = B->insts[i]->dev;
    B->fam_of.clear();
  }
  cudaError_t e = cudaMemcpyAsync(B->d_insts, h.data(), sizeof(DevInstrument) * n, cudaMemcpyHostToDevice,
                                  B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch specialize");
  B->spec_kernel = k;
  mcx_status st = set_shape(B, B->opt);
  // the items of large detectors depend on the grid, which may have changed
  if (st == MCX_OK) st = plan(B, B->budgets, B->opt.chunk_rays);
  return st;
}

extern "C" mcx_status mcx_batch_items(const mcx_batch* B, uint64_t* n_items) {
  if (!B || !n_items) return fail(MCX_ERR_INVALID, "NULL argument");
  *n_items = B->n_items;
  return MCX_OK;
}

// Autotuner cache: batch shape -> chosen launch options (process-wide).
static std::mutex g_tune_mu;
static std::map<std::string, mcx_batch_options> g_tune_cache;

static std::string shape_key(const mcx_batch* B, uint64_t sample) {
  uint64_t total = 0;
  for (auto b : B->budgets) total += std::min(b, sample);
  char buf[160];
  snprintf(buf, sizeof buf, "p%d v%d f%d n%zu m%d t%d", B->precision, (int)B->vox, B->spec_kernel ? 1 : 0,
           B->insts.size(), B->n_mat, (int)std::log2((double)std::max<uint64_t>(total, 1)));
  std::string k = buf;
  for (auto* I : B->insts) k += "|" + std::to_string(I->comps.size());
  return k;
}

extern "C" mcx_status mcx_batch_autotune(mcx_batch* B, uint64_t sample_rays, uint64_t seed,
                                         mcx_batch_options* chosen) {
  if (!B) return fail(MCX_ERR_INVALID, "batch is NULL");
  if (sample_rays == 0) return fail(MCX_ERR_INVALID, "sample_rays must be > 0");
  DeviceGuard guard(B->device);
  const std::string key = shape_key(B, sample_rays);
  const int32_t keep_graph = B->opt.use_graph;
  mcx_batch_options best = B->opt;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    std::vector<uint64_t> sample(B->budgets.size());
    for (size_t i = 0; i < sample.size(); ++i) sample[i] = std::min(B->budgets[i], sample_rays);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // every candidate's time (the better of two runs); kept: the smallest
    // chunk within 5 % of the fastest.  A sample of at most sample_rays per
    // instrument cannot show what the chunk size does at full size (on the
    // 376-instrument batch, 2^16-ray chunks ran 1.45x faster than 2^18 ones
    // that had won the sample)
    struct Trial { mcx_batch_options o; float ms; };
    std::vector<Trial> trials;
    const int blocks[] = {128, 256};
    const uint64_t chunks[] = {1ull << 16, 1ull << 18, 1ull << 20};
    for (int blk : blocks) {
      const size_t smem = block_smem_bytes((B->vox & kVoxMask) ? B->n_mat : 0, blk, B->precision);
      const int occ = occupancy(B, blk, smem);
      const int bps[] = {occ, occ > 1 ? occ - 1 : occ};
      for (int bi = 0; bi < (occ > 1 ? 2 : 1); ++bi) {
        for (uint64_t ch : chunks) {
          mcx_batch_options o = B->opt;
          o.block_size = blk;
          o.blocks_per_sm = bps[bi];
          o.chunk_rays = ch;
          o.use_graph = 0;
          set_shape(B, o);
          mcx_status s = plan(B, sample, ch);
          if (s == MCX_OK) s = run(B, seed);  // warm-up
          float ms = 1e30f;
          for (int rep = 0; rep < 2 && s == MCX_OK; ++rep) {
            cudaEventRecord(e0, B->stream);
            s = run(B, seed + 1 + rep);
            cudaEventRecord(e1, B->stream);
            if (s != MCX_OK) break;
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t < ms ? t : ms;
          }
          if (s != MCX_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s;
          }
          trials.push_back({o, ms});
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    float best_ms = 1e30f;
    for (const Trial& t : trials) best_ms = t.ms < best_ms ? t.ms : best_ms;
    const Trial* pick = nullptr;
    for (const Trial& t : trials) {
      if (t.ms > 1.05f * best_ms) continue;
      if (!pick || t.o.chunk_rays < pick->o.chunk_rays ||
          (t.o.chunk_rays == pick->o.chunk_rays && t.ms < pick->ms))
        pick = &t;
    }
    if (pick) best = pick->o;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  best.use_graph = keep_graph;
  set_shape(B, best);
  mcx_status s = plan(B, B->budgets, B->opt.chunk_rays);
  if (s != MCX_OK) return s;
  for (auto* I : B->insts) {
    s = mcx_monitor_reset(I);
    if (s != MCX_OK) return s;
  }
  cudaError_t e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  if (chosen) *chosen = B->opt;
  return MCX_OK;
}

extern "C" void mcx_batch_destroy(mcx_batch* B) {
  if (!B) return;
  DeviceGuard guard(B->device);
  cudaStreamSynchronize(B->stream);
  drop_graph(B);
  if (B->d_items) cudaFree(B->d_items);
  if (B->d_insts) cudaFree(B->d_insts);
  if (B->d_ticket) cudaFree(B->d_ticket);
  if (B->wave_starts) cudaFree(B->wave_starts);
  if (B->wave_sorted) cudaFree(B->wave_sorted);
  if (B->ord_keys) cudaFree(B->ord_keys);
  if (B->ord_perm) cudaFree(B->ord_perm);
  if (B->ord_hist) cudaFree(B->ord_hist);
  if (B->d_insts_wave) cudaFree(B->d_insts_wave);
  if (B->d_items_wave) cudaFree(B->d_items_wave);
  if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
  delete B;
}
