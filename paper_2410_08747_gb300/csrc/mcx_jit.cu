// mcx_jit.cu -- instrument compilation: a tracing kernel specialised to one
// instrument's component table, generated and compiled at run time.
//
// McXtrace turns every instrument description into its own C program
// (arXiv 2410.08747 Sec. 2.1), so each component's parameters are constants
// of the compiled code.  Here the same idea is applied to the fused GPU
// tracer: the placed component table (types, frames, parameters, binary32
// copies) is written out as a compile-time constant array and the generic
// ray loop (mcx_tracer.cuh) is instantiated over it.  The loop over
// components unrolls, the per-component type dispatch disappears, and every
// parameter becomes an immediate operand instead of a shared-memory load.
//
// The arithmetic is unchanged: the kernel is compiled with --fmad=false like
// the generic one, constants are written as exact hexadecimal literals, and
// the operations are those of the same source, so counts and sums equal the
// generic kernel's (the parity tests run both).
#include <nvrtc.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mcx_embed.h"   // generated by build.py: the device headers as text
#include "mcx_host.h"
#include "mcx_internal.h"
#include "mcx_tracer.cuh"

namespace mcx {

namespace {

void put_d(std::string& o, double v) {
  char b[48];
  std::snprintf(b, sizeof b, "%a", v);
  o += b;
}

void put_f(std::string& o, float v) {
  char b[48];
  std::snprintf(b, sizeof b, "%af", (double)v);
  o += b;
}

template <class T, class P>
void put_list(std::string& o, const T* v, int n, P put) {
  o += '{';
  for (int i = 0; i < n; ++i) {
    if (i) o += ", ";
    put(o, v[i]);
  }
  o += '}';
}

void put_i(std::string& o, int32_t v) { o += std::to_string(v); }

bool finite_comp(const DevComp& c) {
  auto ok = [](const auto* v, int n) {
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(v[i])) return false;
    return true;
  };
  return ok(c.o, 3) && ok(c.R, 9) && ok(c.p, 12) && ok(c.inv, 3) && ok(c.aux, 3) &&
         ok(c.pf, 12) && ok(c.invf, 3) && ok(c.auxf, 3) && ok(c.Rf, 9);
}

// One DevComp as an aggregate initialiser, fields in declaration order.
void put_comp(std::string& o, const DevComp& c) {
  o += "  {";
  put_i(o, c.type); o += ", ";
  put_i(o, c.shape); o += ", ";
  put_i(o, c.spectrum); o += ", ";
  put_i(o, c.material); o += ", ";
  put_list(o, c.n, 3, put_i); o += ", ";
  put_i(o, c.identity); o += ", ";
  o += std::to_string((long long)c.mon_offset) + "LL, ";
  put_i(o, c.zo); o += ", ";
  put_i(o, c.last); o += ",\n   ";
  put_list(o, c.o, 3, put_d); o += ", ";
  put_list(o, c.R, 9, put_d); o += ",\n   ";
  put_list(o, c.p, 12, put_d); o += ",\n   ";
  put_list(o, c.inv, 3, put_d); o += ", ";
  put_list(o, c.aux, 3, put_d); o += ",\n   ";
  put_list(o, c.pf, 12, put_f); o += ",\n   ";
  put_list(o, c.invf, 3, put_f); o += ", ";
  put_list(o, c.auxf, 3, put_f); o += ", ";
  put_list(o, c.Rf, 9, put_f); o += ",\n   ";
  put_list(o, c.vstride, 3, put_i); o += ", ";
  put_i(o, c.priv); o += ", ";
  put_i(o, c.restore); o += ", ";
  put_i(o, c.l2keep);
  o += "}";
}

struct Compiled {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
};

std::mutex g_mu;
std::map<std::string, Compiled> g_cache;   // source text -> loaded kernel

const char* kKernelName = "mcx_spec_trace";

mcx_status compile(const std::string& src, const char* name, Compiled* out) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(src);
    if (it != g_cache.end()) {
      *out = it->second;
      return MCX_OK;
    }
  }
  const char* hdr_src[2] = {kEmbedInternalH, kEmbedTracerCuh};
  const char* hdr_name[2] = {"mcx_internal.h", "mcx_tracer.cuh"};
  nvrtcProgram prog = nullptr;
  if (nvrtcCreateProgram(&prog, src.c_str(), "mcx_spec.cu", 2, hdr_src, hdr_name) != NVRTC_SUCCESS)
    return fail(MCX_ERR_UNSUPPORTED, "nvrtcCreateProgram failed");
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false", "-lineinfo"};
  const nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    if (log.size() > 600) log.resize(600);
    return fail(MCX_ERR_UNSUPPORTED, "specialised kernel did not compile (%s): %s",
                nvrtcGetErrorString(r), log.c_str());
  }
  size_t n = 0;
  std::vector<char> cubin;
  if (nvrtcGetCUBINSize(prog, &n) == NVRTC_SUCCESS && n) {
    cubin.resize(n);
    if (nvrtcGetCUBIN(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
  }
  nvrtcDestroyProgram(&prog);
  if (cubin.empty()) return fail(MCX_ERR_UNSUPPORTED, "no cubin from the run-time compiler");
  Compiled c;
  cudaError_t e = cudaLibraryLoadData(&c.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&c.kernel, c.lib, name);
  if (e != cudaSuccess) {
    if (c.lib) cudaLibraryUnload(c.lib);
    return cuda_fail(e, "loading the specialised kernel");
  }
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(src);
  if (it != g_cache.end()) {      // another thread compiled it meanwhile
    cudaLibraryUnload(c.lib);
    *out = it->second;
    return MCX_OK;
  }
  g_cache.emplace(src, c);
  *out = c;
  return MCX_OK;
}

// The fields of DevComp, in declaration order, as the family generator sees
// them: name, offset, element size and count.
struct Field {
  const char* name;
  size_t off, size;
  int count;
};
#define MCX_FIELD(f, n) Field{#f, offsetof(DevComp, f), sizeof(DevComp::f) / (n), (n)}
const Field kFields[] = {
    MCX_FIELD(type, 1),   MCX_FIELD(shape, 1),  MCX_FIELD(spectrum, 1), MCX_FIELD(material, 1),
    MCX_FIELD(n, 3),      MCX_FIELD(identity, 1), MCX_FIELD(mon_offset, 1), MCX_FIELD(zo, 1),
    MCX_FIELD(last, 1),   MCX_FIELD(o, 3),      MCX_FIELD(R, 9),        MCX_FIELD(p, 12),
    MCX_FIELD(inv, 3),    MCX_FIELD(aux, 3),    MCX_FIELD(pf, 12),      MCX_FIELD(invf, 3),
    MCX_FIELD(auxf, 3),   MCX_FIELD(Rf, 9),     MCX_FIELD(vstride, 3),  MCX_FIELD(priv, 1),
    MCX_FIELD(restore, 1), MCX_FIELD(l2keep, 1)};
#undef MCX_FIELD

}  // namespace

// Instrument families of a batch: instruments with the same component types
// (and precision) share one; returns each instrument's family index and the
// members of each family.
std::vector<std::vector<int>> batch_families(const std::vector<mcx_instrument*>& insts, std::vector<int>& fam_of) {
  std::vector<std::vector<int>> fams;
  std::vector<std::vector<int32_t>> keys;
  fam_of.assign(insts.size(), -1);
  for (size_t i = 0; i < insts.size(); ++i) {
    std::vector<int32_t> key;
    for (const DevComp& c : insts[i]->comps) key.push_back(c.type);
    size_t f = 0;
    while (f < keys.size() && keys[f] != key) ++f;
    if (f == keys.size()) {
      keys.push_back(key);
      fams.emplace_back();
    }
    fams[f].push_back((int)i);
    fam_of[i] = (int)f;
  }
  return fams;
}

// The source text of a batch kernel compiled by families: per family a
// component table whose fields shared by every member are compile-time
// constants (member 0's values) and whose other fields are read from the
// instrument's table in shared memory.
std::string batch_source(const std::vector<mcx_instrument*>& insts, const std::vector<std::vector<int>>& fams,
                         int precision, int vox) {
  // the union of the members' paths; a marching batch takes both traversals
  const int vk = (vox & kVoxMarch) ? (vox | (int)kVoxBoth) : vox;
  std::string o;
  o += "// Batch tracing kernel compiled by instrument families (generated).\n";
  o += "#include \"mcx_tracer.cuh\"\n\n";
  for (size_t f = 0; f < fams.size(); ++f) {
    const mcx_instrument* I0 = insts[fams[f][0]];
    const int n = (int)I0->comps.size();
    o += "namespace mcx_fam" + std::to_string(f) + " {\n";
    o += "__device__ constexpr mcx::DevComp kComps[" + std::to_string(n) + "] = {\n";
    for (int i = 0; i < n; ++i) {
      put_comp(o, I0->comps[i]);
      o += i + 1 < n ? ",\n" : "\n";
    }
    o += "};\n";
    o += "struct Table {\n";
    o += "  static constexpr bool kStatic = true;\n";
    o += "  static constexpr int kN = " + std::to_string(n) + ";\n";
    o += "  const mcx::DevComp* rt;   // this instrument's table (shared memory)\n";
    o += "  __device__ __forceinline__ mcx::DevComp operator[](int i) const {\n";
    o += "    mcx::DevComp c = kComps[i];\n";
    for (int i = 0; i < n; ++i) {
      std::string varying;
      for (const Field& fd : kFields) {
        bool same = true;
        for (int m : fams[f])
          same = same && std::memcmp(reinterpret_cast<const char*>(&insts[m]->comps[i]) + fd.off,
                                     reinterpret_cast<const char*>(&I0->comps[i]) + fd.off,
                                     fd.size * fd.count) == 0;
        if (same) continue;
        if (fd.count == 1)
          varying += std::string("c.") + fd.name + " = rt[" + std::to_string(i) + "]." + fd.name + "; ";
        else
          varying += "for (int k = 0; k < " + std::to_string(fd.count) + "; ++k) c." + fd.name + "[k] = rt[" +
                     std::to_string(i) + "]." + fd.name + "[k]; ";
      }
      if (!varying.empty()) o += "    if (i == " + std::to_string(i) + ") { " + varying + "}\n";
    }
    o += "    return c;\n  }\n";
    o += "  __device__ __forceinline__ int size() const { return kN; }\n";
    o += "};\n}  // namespace mcx_fam" + std::to_string(f) + "\n\n";
  }
  o += "struct Families {\n";
  o += "  template <class F>\n";
  o += "  __device__ __forceinline__ static void with_table(int family, const mcx::DevComp* table, int, const F& f) {\n";
  o += "    switch (family) {\n";
  for (size_t f = 0; f < fams.size(); ++f)
    o += "      case " + std::to_string(f) + ": f(mcx_fam" + std::to_string(f) + "::Table{table}); break;\n";
  o += "      default: break;\n    }\n  }\n};\n\n";
  o += "extern \"C\" __global__ void __launch_bounds__(256, ";
  o += (vox & kVoxMask) ? (precision == 1 ? "mcx::kVoxMinBlocksMixed" : "mcx::kVoxMinBlocks")
                        : "mcx::kFamilyMinBlocks";
  o += ")\n";
  o += "mcx_batch_spec(const mcx::DevInstrument* insts, const mcx::WorkItem* items, unsigned n_items,\n";
  o += "               unsigned* ticket, unsigned long long seed) {\n";
  o += "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o += "  __shared__ double red[64];\n";
  o += "  mcx::batch_rays<" + std::to_string(precision) + ", " + std::to_string(vk) +
       ", Families>(insts, items, n_items, ticket, seed, smem, red);\n";
  o += "}\n";
  return o;
}

bool tables_finite(const std::vector<mcx_instrument*>& insts) {
  for (const mcx_instrument* I : insts)
    for (const DevComp& c : I->comps)
      if (!finite_comp(c)) return false;
  return true;
}

// Compiles the batch kernel of `src` (cached by source text).
mcx_status compile_batch(const std::string& src, const void** kernel) {
  Compiled c;
  mcx_status st = compile(src, "mcx_batch_spec", &c);
  if (st != MCX_OK) return st;
  *kernel = (const void*)c.kernel;
  return MCX_OK;
}

// The source text of the specialised kernel of instrument I.
std::string spec_source(const mcx_instrument* I) {
  const bool vox = I->has_phantom;
  // a scattering march phantom in the mixed form: the refilling kernel
  const bool refill = I->scatter && I->precision == 1 && I->vox_kind == kVoxMarch;
  const int vk = I->vox_kind | (refill ? (int)kScatter : 0);
  const int n = (int)I->comps.size();
  std::string o;
  o += "// Tracing kernel specialised to one instrument (generated).\n";
  o += "#include \"mcx_tracer.cuh\"\n\n";
  o += "namespace mcx_spec {\n";
  o += "__device__ constexpr mcx::DevComp kComps[" + std::to_string(n) + "] = {\n";
  for (int i = 0; i < n; ++i) {
    put_comp(o, I->comps[i]);
    o += i + 1 < n ? ",\n" : "\n";
  }
  o += "};\n";
  o += "struct Table {\n";
  o += "  static constexpr bool kStatic = true;\n";
  o += "  static constexpr int kN = " + std::to_string(n) + ";\n";
  o += "  __device__ __forceinline__ const mcx::DevComp& operator[](int i) const { return kComps[i]; }\n";
  o += "  __device__ __forceinline__ int size() const { return kN; }\n";
  o += "};\n";
  o += "}  // namespace mcx_spec\n\n";
  // Resident blocks per SM: with its constants folded the kernel without a
  // phantom fits in few registers (kSpecMinBlocks blocks of 256 threads).
  o += "extern \"C\" __global__ void __launch_bounds__(256, ";
  o += refill ? "mcx::kScatterMinBlocks"
              : (vox ? (I->precision == 1 ? "mcx::kVoxMinBlocksMixed" : "mcx::kVoxMinBlocks") : "mcx::kSpecMinBlocks");
  o += ")\n";
  o += std::string(kKernelName) + "(const mcx::DevInstrument I, unsigned long long begin,\n";
  o += "               unsigned long long end, unsigned long long seed) {\n";
  o += "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o += "  __shared__ double red[64];\n";
  o += "  mcx::trace_rays<" + std::to_string(I->precision) + ", " + std::to_string(vk) +
       ", mcx_spec::Table>(I, begin, end, seed, smem, red);\n";
  o += "}\n";
  return o;
}

}  // namespace mcx

using namespace mcx;

extern "C" mcx_status mcx_instrument_source(const mcx_instrument* I, char* buf, size_t cap,
                                            size_t* len) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  const std::string s = spec_source(I);
  if (len) *len = s.size() + 1;
  if (buf) {
    if (cap < s.size() + 1) return fail(MCX_ERR_INVALID, "buffer holds %zu bytes, need %zu", cap, s.size() + 1);
    std::memcpy(buf, s.c_str(), s.size() + 1);
  }
  return MCX_OK;
}

extern "C" mcx_status mcx_instrument_specialize(mcx_instrument* I, int32_t enable) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  if (!enable) {
    I->spec_kernel = nullptr;
    return MCX_OK;
  }
  for (const DevComp& c : I->comps)
    if (!finite_comp(c))
      return fail(MCX_ERR_UNSUPPORTED, "a component parameter is not finite");
  DeviceGuard guard(I->device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", I->device);
  Compiled c;
  mcx_status st = compile(spec_source(I), kKernelName, &c);
  if (st != MCX_OK) return st;
  // rows of the per-thread material column: a scattering phantom adds its sums
  const int n_mat = I->has_phantom ? I->dev.n_mat * (I->scatter ? 2 : 1) : 0;
  const size_t smem = block_smem_bytes(n_mat, I->shape.block, I->precision, false, I->dev.n_priv);
  if (I->has_phantom || smem > 48 * 1024) {   // phantom kernels: static ordering buffers too
    cudaError_t e = cudaFuncSetAttribute((const void*)c.kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "specialised kernel shared memory");
  }
  // persistent grid: SMs x resident blocks of this kernel (its own register
  // count decides), unless the caller fixed the blocks per SM
  int n_sm = 0, bpsm = I->user_blocks_per_sm;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, I->device);
  if (bpsm == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, (const void*)c.kernel,
                                                                 I->shape.block, smem) != cudaSuccess) {
    cudaGetLastError();
    bpsm = n_sm > 0 ? I->shape.grid / n_sm : 1;
  }
  I->spec_grid = n_sm * (bpsm > 0 ? bpsm : 1);
  I->spec_kernel = (const void*)c.kernel;
  I->spec_smem = smem;
  return MCX_OK;
}

namespace mcx {

cudaError_t launch_spec(const mcx_instrument* I, const DevInstrument& dev, uint64_t begin,
                        uint64_t end, uint64_t seed) {
  if (end <= begin) return cudaSuccess;
  const uint64_t n = end - begin;
  const uint64_t need = (n + I->shape.block - 1) / I->shape.block;
  const unsigned grid = (unsigned)(need < (uint64_t)I->spec_grid ? need : (uint64_t)I->spec_grid);
  DevInstrument d = dev;
  unsigned long long b = begin, e = end, s = seed;
  void* args[] = {&d, &b, &e, &s};
  return cudaLaunchKernel(I->spec_kernel, dim3(grid), dim3(I->shape.block), args, I->spec_smem,
                          I->stream);
}

}  // namespace mcx
