// mcx_host.h -- host-side state shared by the library's translation units:
// the instrument object, error reporting and the device guard.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/mcx.h"
#include "mcx_internal.h"

namespace mcx {

// Records the calling thread's last error message and returns `s`.
mcx_status fail(mcx_status s, const char* fmt, ...);
mcx_status cuda_fail(cudaError_t e, const char* what);

// Makes `device` current for the scope of an API call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace mcx

struct mcx_instrument {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = 0;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<mcx::DevComp> comps;
  std::vector<int64_t> mon_off, mon_bins;
  int64_t n_bins = 0;
  mcx::DevInstrument dev{};
  std::vector<void*> buffers;
  uint64_t n_emit = 0;
  mcx::LaunchShape shape{};
  bool has_phantom = false;
  int vox_kind = 0;              // its phantom's traversal | kOptics
  bool scatter = false;          // the phantom scatters (rays change line inside it)
  void* split = nullptr;   // readout scratch: SoA copy of the largest monitor
  void* totals = nullptr;  // monitor totals scratch (count, sum w, sum w^2)
  int user_blocks_per_sm = 0;          // mcx_options.blocks_per_sm (0 = from occupancy)
  const void* spec_kernel = nullptr;   // specialised tracer (mcx_jit.cu), if enabled
  size_t spec_smem = 0;
  int spec_grid = 0;
  // ray order of a phantom trace (kOrderChunk ids at a time)
  uint16_t* ord_keys = nullptr;
  uint32_t* ord_hist = nullptr;
  uint32_t* ord_perm = nullptr;
  unsigned* ord_ticket = nullptr;
  // learned proposal attached by mcx_proposal_attach: traces draw their
  // starts from it, kPropChunk rays at a time through prop_buf
  mcx_proposal* prop = nullptr;
  float prop_angle = 0.f;
  float* prop_buf = nullptr;
};

namespace mcx {
// Rays per sampling chunk of an instrument with an attached proposal (24
// bytes a ray, a 200 MB start buffer): large enough that the per-chunk
// launches (sampler, the walk's ray order, tracer) cost little next to the
// chunk's work; the buffer's round trip through HBM costs 48 bytes a ray.
constexpr uint64_t kPropChunk = 1ull << 23;

// Device buffer owned by the instrument (its allocator), freed by destroy.
void* instrument_alloc(mcx_instrument* I, size_t bytes);

// Queue the proposal's sampler for rays [begin, begin + n) of the device
// description d (mcx_proposal_sample without its status check) into
// d_starts (rows of n), on stream s.
cudaError_t proposal_sample_async(mcx_proposal* Q, const DevInstrument& d, uint64_t begin, uint64_t n,
                                  uint64_t seed, float angle, float* d_starts, cudaStream_t s);
// Queue the source's own sampler (mcx_sample_starts) for rays
// [begin, begin + n) of the device description d into d_starts (rows of n).
cudaError_t sample_starts_async(const DevInstrument& d, uint64_t begin, uint64_t n, uint64_t seed,
                                float* d_starts, cudaStream_t s);
// MCX_ERR_TIMEOUT if an earlier sampler of Q gave up waiting for the tensor
// cores (synchronises s).
mcx_status proposal_check(mcx_proposal* Q, cudaStream_t s);

// Queue rays [begin, end) through instrument I's specialised kernel, with
// the device description `d` (I->dev, or a copy with given ray starts).
cudaError_t launch_spec(const mcx_instrument* I, const DevInstrument& d, uint64_t begin,
                        uint64_t end, uint64_t seed);

// Batch compilation by families (mcx_jit.cu): each instrument's family and
// the members of each family; the kernel source; its compilation.
std::vector<std::vector<int>> batch_families(const std::vector<mcx_instrument*>& insts, std::vector<int>& fam_of);
std::string batch_source(const std::vector<mcx_instrument*>& insts, const std::vector<std::vector<int>>& fams,
                         int precision, int vox);
mcx_status compile_batch(const std::string& src, const void** kernel);
bool tables_finite(const std::vector<mcx_instrument*>& insts);

// Queue the trace of rays [begin, end) of instrument I with the device
// description `d`: one launch, or, with a phantom, the ray order and a
// launch for each chunk of at most kOrderChunk ids.
cudaError_t trace_dispatch(const mcx_instrument* I, DevInstrument d, uint64_t begin, uint64_t end,
                           uint64_t seed);
}  // namespace mcx
