"""The kernels the library compiles at run time for an instrument (NVRTC,
sm_103a, the options of mcx_jit.cu) are built on the GPU machine only when an
instrument is compiled there.  These tests compile them here, with no GPU:
the two device headers the library embeds, a compile-time component table
of each path kind (analytic absorber and large detector; exact voxel walk;
fixed-step march; march with scattering, whose mixed form refills lanes;
Gaussian source and lens stack) and the entry point the library generates,
in both precisions, and a batch kernel compiled by instrument families.  A header construct that nvcc accepts and NVRTC does
not (run-time compilation has no host functions) fails here, not on the
GPU."""

import ctypes
import ctypes.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_08747_gb300", "csrc")

# component types and path bits (mcx_internal.h)
T_SOURCE, T_ABS_CYL, T_PHANTOM, T_MON_E, T_MON_EPSD, T_LENS = 0, 4, 6, 8, 10, 11
K_WALK, K_MARCH, K_OPTICS, K_SCATTER = 1, 2, 4, 8


def nvrtc():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libnvrtc.so"),
             "libnvrtc.so", "libnvrtc.so.13", ctypes.util.find_library("nvrtc")]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("libnvrtc is not available")


def table_source(kinds, prec, vox, min_blocks):
    """A generated kernel as mcx_jit.cu writes it, its table built by
    constexpr functions (each entry value-initialised, then its type and the
    fields that select paths set), so no field order is assumed."""
    makers = []
    for i, (t, extra) in enumerate(kinds):
        sets = "".join(f" c.{k} = {v};" for k, v in extra.items())
        makers.append(f"__device__ constexpr mcx::DevComp make{i}() {{\n"
                      f"  mcx::DevComp c{{}}; c.type = {t}; c.identity = 1; c.priv = -1;{sets}\n"
                      "  return c;\n}\n")
    n = len(kinds)
    return (
        '#include "mcx_tracer.cuh"\n'
        "namespace mcx_spec {\n" + "".join(makers) +
        f"__device__ constexpr mcx::DevComp kComps[{n}] = {{{', '.join(f'make{i}()' for i in range(n))}}};\n"
        "struct Table {\n"
        "  static constexpr bool kStatic = true;\n"
        f"  static constexpr int kN = {n};\n"
        "  __device__ __forceinline__ const mcx::DevComp& operator[](int i) const { return kComps[i]; }\n"
        "  __device__ __forceinline__ int size() const { return kN; }\n"
        "};\n}\n"
        f'extern "C" __global__ void __launch_bounds__(256, {min_blocks})\n'
        "mcx_spec_trace(const mcx::DevInstrument I, unsigned long long begin, unsigned long long end,\n"
        "               unsigned long long seed) {\n"
        "  extern __shared__ __align__(16) unsigned char smem[];\n"
        "  __shared__ double red[64];\n"
        f"  mcx::trace_rays<{prec}, {vox}, mcx_spec::Table>(I, begin, end, seed, smem, red);\n"
        "}\n")


def compile_nvrtc(lib, src):
    hdrs = [open(os.path.join(CSRC, f), "rb").read() for f in ("mcx_internal.h", "mcx_tracer.cuh")]
    prog = ctypes.c_void_p()
    H = (ctypes.c_char_p * 2)(*hdrs)
    N = (ctypes.c_char_p * 2)(b"mcx_internal.h", b"mcx_tracer.cuh")
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"mcx_spec.cu", 2, H, N) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"--fmad=false", b"-lineinfo"]
    O = (ctypes.c_char_p * len(opts))(*opts)
    rc = lib.nvrtcCompileProgram(prog, len(opts), O)
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(n.value, 1))
    lib.nvrtcGetProgramLog(prog, log)
    size = ctypes.c_size_t()
    cubin_ok = rc == 0 and lib.nvrtcGetCUBINSize(prog, ctypes.byref(size)) == 0 and size.value > 0
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, cubin_ok, log.value.decode(errors="replace")


SOURCE = (T_SOURCE, {})
DETECTOR = (T_MON_EPSD, {"n[0]": 16, "n[1]": 16, "n[2]": 8, "last": 1, "l2keep": 1})
PATHS = {
    "absorber": ([SOURCE, (T_ABS_CYL, {}), DETECTOR], 0),
    "walk": ([SOURCE, (T_PHANTOM, {"n[0]": 8, "n[1]": 8, "n[2]": 8}), DETECTOR], K_WALK),
    "march": ([SOURCE, (T_PHANTOM, {"n[0]": 8, "n[1]": 8, "n[2]": 8, "p[1]": 3.0}), DETECTOR], K_MARCH),
    "scatter": ([SOURCE, (T_PHANTOM, {"n[0]": 8, "n[1]": 8, "n[2]": 8, "p[1]": 3.0, "p[4]": 1.0}),
                 (T_MON_E, {"n[0]": 8}), DETECTOR], K_MARCH),
    "optics": ([(T_SOURCE, {"shape": 3, "spectrum": 2}), (T_LENS, {}), DETECTOR], K_OPTICS),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("path", sorted(PATHS))
def test_generated_kernel_compiles_with_nvrtc(path, prec):
    lib = nvrtc()
    kinds, vox = PATHS[path]
    if path == "scatter" and prec == 1:
        vox |= K_SCATTER   # the mixed form of a scattering march: refilled lanes
    min_blocks = "mcx::kScatterMinBlocks" if vox & K_SCATTER else "4"
    rc, cubin_ok, log = compile_nvrtc(lib, table_source(kinds, prec, vox, min_blocks))
    assert rc == 0 and cubin_ok, log[-2000:]


def batch_source(families, prec, vox):
    """A batch kernel compiled by instrument families, as mcx_jit.cu writes
    it: per family a compile-time table whose entries members may override
    field by field (here the rotation of component 1), a dispatcher over
    the families, and the persistent entry point."""
    vk = vox | 3 if vox & K_MARCH else vox   # a marching batch takes both traversals
    o = '#include "mcx_tracer.cuh"\n'
    for f, kinds in enumerate(families):
        o += f"namespace mcx_fam{f} {{\n"
        for i, (t, extra) in enumerate(kinds):
            sets = "".join(f" c.{k} = {v};" for k, v in extra.items())
            o += (f"__device__ constexpr mcx::DevComp make{i}() {{\n"
                  f"  mcx::DevComp c{{}}; c.type = {t}; c.identity = 1; c.priv = -1;{sets}\n  return c;\n}}\n")
        n = len(kinds)
        o += f"__device__ constexpr mcx::DevComp kComps[{n}] = {{{', '.join(f'make{i}()' for i in range(n))}}};\n"
        o += ("struct Table {\n  static constexpr bool kStatic = true;\n"
              f"  static constexpr int kN = {n};\n"
              "  const mcx::DevComp* rt;\n"
              "  __device__ __forceinline__ mcx::DevComp operator[](int i) const {\n"
              "    mcx::DevComp c = kComps[i];\n"
              "    if (i == 1) { for (int k = 0; k < 9; ++k) c.R[k] = rt[1].R[k]; }\n"
              "    return c;\n  }\n"
              "  __device__ __forceinline__ int size() const { return kN; }\n};\n}\n")
    o += ("struct Families {\n  template <class F>\n"
          "  __device__ __forceinline__ static void with_table(int family, const mcx::DevComp* table, int, const F& f) {\n"
          "    switch (family) {\n")
    for f in range(len(families)):
        o += f"      case {f}: f(mcx_fam{f}::Table{{table}}); break;\n"
    o += "      default: break;\n    }\n  }\n};\n"
    o += ('extern "C" __global__ void __launch_bounds__(256, 4)\n'
          "mcx_batch_spec(const mcx::DevInstrument* insts, const mcx::WorkItem* items, unsigned n_items,\n"
          "               unsigned* ticket, unsigned long long seed) {\n"
          "  extern __shared__ __align__(16) unsigned char smem[];\n"
          "  __shared__ double red[64];\n"
          f"  mcx::batch_rays<{prec}, {vk}, Families>(insts, items, n_items, ticket, seed, smem, red);\n"
          "}\n")
    return o


@pytest.mark.parametrize("prec", [0, 1])
def test_family_batch_kernel_compiles_with_nvrtc(prec):
    lib = nvrtc()
    fams = [PATHS["absorber"][0], PATHS["scatter"][0], PATHS["optics"][0]]
    rc, cubin_ok, log = compile_nvrtc(lib, batch_source(fams, prec, K_MARCH | K_OPTICS))
    assert rc == 0 and cubin_ok, log[-2000:]
