// mcx_internal.h -- device-side data layout shared by the library's own
// translation units (host API, tracer kernel, batched scheduler).
#pragma once

#ifdef __CUDACC_RTC__
// Run-time compilation of a specialised tracer (mcx_jit.cu): the device
// types only, without host headers.
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#endif

namespace mcx {

constexpr int kMaxComps = 32;     // components per instrument
// Block-private monitor copies: a monitor of at most kPrivMonBins bins gets a
// per-block copy in shared memory while the instrument's private bins stay
// within kMaxPrivBins (20 bytes each).
constexpr int kPrivMonBins = 1024;
constexpr int kMaxPrivBins = 1024;
constexpr int kMaxMats = 64;      // materials per instrument
constexpr int kWarp = 32;

// hc in keV * Angstrom (CODATA 2018): wavelength = hc / E.
constexpr double kHcKevAngstrom = 12.398419843320026;

enum CompType : int32_t {
  T_SOURCE = 0, T_SLIT_RECT = 1, T_SLIT_CIRC = 2, T_ABS_BOX = 3, T_ABS_CYL = 4,
  T_ABS_SPHERE = 5, T_PHANTOM = 6, T_MON_PSD = 7, T_MON_E = 8, T_MON_L = 9,
  T_MON_EPSD = 10, T_LENS = 11
};
enum { SHAPE_POINT = 0, SHAPE_DISK = 1, SHAPE_RECT = 2, SHAPE_GAUSS = 3 };
// The paths a kernel is built for (its VOX template parameter, a bit set):
// the phantom traversals (none, the exact voxel-boundary walk, the
// fixed-step march with phantom p1 > 0, both) and kOptics, the Gaussian
// source and the compound refractive lens.  Kernels without a bit carry no
// code or registers for its path.  kScatter selects, for a single instrument
// traced in the mixed form whose march phantom scatters, the kernel whose
// lanes are refilled with new rays (trace_refill); it only ever selects a
// kernel and is never part of an instrument's vox_kind.
enum : int { kVoxNone = 0, kVoxWalk = 1, kVoxMarch = 2, kVoxBoth = 3, kVoxMask = 3, kOptics = 4, kScatter = 8 };
enum { SPEC_FLAT = 0, SPEC_KRAMERS = 1, SPEC_GAUSS = 2 };

// One placed component: x_lab = o + R x_local.  Copied into shared memory by
// every block, so the whole table is read with broadcast loads.
struct alignas(16) DevComp {
  int32_t type, shape, spectrum, material;
  int32_t n[3];
  int32_t identity;        // R is exactly the identity: skip the products
  int64_t mon_offset;      // first bin of this monitor in the bin array
  int32_t zo;              // bit i set when o[i] == 0: skip the add on that axis
  int32_t last;            // last component: the lab position is not needed after it
  double o[3];
  double R[9];             // row-major
  double p[12];            // type parameters (mcx.h)
  double inv[3];           // monitors: n_i / (hi_i - lo_i); phantom: 1/voxel
  double aux[3];           // source: 1/mean(f), mean(f) (Kramers); phantom: half extents
  // binary32 copies (round to nearest) for the mixed form, so the device never
  // converts a parameter per ray
  float pf[12];
  float invf[3];
  float auxf[3];
  float Rf[9];             // rotation rounded to binary32 (weight-only geometry)
  int32_t vstride[3];      // phantom: byte stride of a step along x, y, z in the device layout
  int32_t priv;            // monitors: first bin of a block-private copy, -1 = global atomics only
  int32_t restore;         // monitors: the ray leaves as it entered (p11 != 0)
  int32_t l2keep;          // monitors in global memory: updates carry the L2 evict-last
                           // hint (the instrument's global monitors fit 7/8 of the L2)
};
static_assert(sizeof(DevComp) % 16 == 0, "DevComp must stay 16-byte aligned");

// Monitor bin: count, sum of weights, sum of squared weights (24 bytes, kept
// together so one ray's three updates hit one or two adjacent L2 sectors).
struct MonBin {
  unsigned long long N;
  double sw;
  double sw2;
};

// Everything one trace of one instrument needs on the device.
struct DevInstrument {
  const DevComp* comps;
  int32_t n_comp;
  int32_t instr_id;
  int32_t n_mat;
  int32_t n_cell;
  double e_min;            // mu-table range
  double cell_inv;         // n_cell / (e_max - e_min)
  float e_min_f;           // binary32 copies of the two above
  float cell_inv_f;
  const double2* mu64;     // [n_mat][n_cell] (c0, c1)
  const float2* mu32;
  const uint8_t* vox;      // phantom bytes [nz][ny][nx]
  MonBin* bins;
  double* tallies;         // [n_comp] removed weight, then sum_w0, sum_wend
  // Given ray starts (mixed form only): SoA rows sx, sy, E, u, v, w0 of
  // ext_n rays with ids ext_base.. (null: the tracer samples the source).
  const float* ext;
  uint64_t ext_base;
  uint64_t ext_n;
  float* det_w;            // optional: weight each ray scored at the last monitor
  // Ray order of a phantom trace (null: ids in order): the kernel's range
  // [perm_base, perm_base + n) is a chunk whose position p is traced as ray
  // id perm_base + perm[p - perm_base] (ids grouped by aim-point tile).
  const uint32_t* perm;
  uint64_t perm_base;
  unsigned* ticket;        // batch counter of an ordered launch (zeroed before it)
  int32_t n_priv;          // bins of all block-private monitor copies
  int32_t family;          // batch compiled by families: this instrument's family
  int32_t vox_kind;        // its phantom's traversal (kVoxNone/Walk/March) | kOptics
  int32_t pad;
  // scattering phantom: the Rayleigh and the Compton coefficient tables
  // [2][n_mat][n_cell] of (c0, c1), mu = c0 + c1 E on each cell of the mu
  // tables (1/m); the binary32 copy holds each coefficient rounded once; or null
  const double* sc64;
  const float* sc32;
};

// One work item of a batch: rays [begin, end) of instrument `inst`.
struct WorkItem {
  uint64_t begin, end;
  uint32_t inst;
  uint32_t pad;
};

// Ray ids per ordered chunk of a phantom trace, and aim-point tiles per axis
// of the target (Morton order, kTileBits bits per axis; 16-bit keys).  A
// 256 x 256 grid puts ~256 rays of a 2^24-id chunk in a tile, so the 1024
// ids a block takes at a time cover a few neighbouring tiles; measured on
// the 256^3 CT projection (compiled, 2e8 rays): 32 x 32 tiles 2.39e9, 64 x 64
// 2.69e9, 128 x 128 2.80e9, 256 x 256 2.80e9 rays/s.
constexpr uint32_t kOrderChunk = 1u << 24;
constexpr int kTileBits = 8;
constexpr int kTiles = 1 << (2 * kTileBits);

// Number of float rows of a ray-start buffer: sx, sy, E, u, v, w0.
constexpr int kStartRows = 6;

#ifndef __CUDACC_RTC__

// Launch shape of one trace.
struct LaunchShape {
  int grid;
  int block;
  size_t smem;
};

size_t trace_smem_bytes(int n_comp, int n_mat, int block, int precision, bool has_phantom,
                        int n_priv);

// Queue one fused trace of rays [begin, end) (stream-ordered).
cudaError_t launch_trace(const DevInstrument& inst, int precision, uint64_t begin,
                         uint64_t end, uint64_t seed, const LaunchShape& shape,
                         cudaStream_t stream);

// Device Philox4x32-10 on n (counter, key) sextets -> n output quads.
cudaError_t launch_philox_fill(const uint32_t* d_in, uint32_t* d_out, size_t n, cudaStream_t s);

// Device binary64 -> binary32 rounding and exact widening (diagnostic).
cudaError_t launch_convert_fill(const double* in, float* of, double* od, size_t n, cudaStream_t s);

// Split n_bins MonBins into SoA arrays N, sum w, sum w^2 (each may be null).
// Totals of n_bins MonBins into outN[0] and outw[0..1] (zeroed first).
cudaError_t launch_total_bins(const MonBin* in, size_t n_bins, unsigned long long* outN, double* outw,
                              cudaStream_t s);
cudaError_t launch_split_bins(const MonBin* in, size_t n_bins, unsigned long long* N, double* sw,
                              double* sw2, cudaStream_t s);

// Occupancy of the tracer kernel (blocks per SM) for a block size and smem;
// vox_kind selects the kernel (kVoxNone, kVoxWalk, kVoxMarch, | kOptics,
// | kScatter for a scattering march phantom).
int trace_occupancy(int precision, int vox_kind, int block, size_t smem);

// Ray order of a phantom trace: perm[0 .. end - begin) lists the chunk's
// ray ids (minus begin) grouped by aim-point tile.  keys: end - begin
// 16-bit scratch words; hist: kTiles counters (zeroed here).
cudaError_t launch_ray_order(const DevInstrument& inst, int precision, uint64_t begin, uint64_t end,
                             uint64_t seed, uint16_t* keys, uint32_t* hist, uint32_t* perm,
                             cudaStream_t stream);
#endif  // __CUDACC_RTC__

}  // namespace mcx
