// mcx_api.cu -- host side of the C ABI declared in include/mcx.h: validation,
// placement of components in the lab frame, one-time upload of every table,
// launch planning, monitor readout and error reporting.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mcx_host.h"

using namespace mcx;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

namespace mcx {

mcx_status fail(mcx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

mcx_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(MCX_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(MCX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace mcx

extern "C" const char* mcx_last_error(void) { return g_last_error.c_str(); }

static void* dev_alloc(mcx_instrument* I, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (I->alloc) {
    p = I->alloc(bytes, I->alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) I->buffers.push_back(p);
  return p;
}

void* mcx::instrument_alloc(mcx_instrument* I, size_t bytes) { return dev_alloc(I, bytes); }

static void release(mcx_instrument* I) {
  if (!I) return;
  cudaStreamSynchronize(I->stream);
  for (void* p : I->buffers) {
    if (I->free_fn) I->free_fn(p, I->alloc_ctx);
    else cudaFree(p);
  }
  I->buffers.clear();
  delete I;
}

static bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

static bool is_monitor(int t) { return t >= T_MON_PSD && t <= T_MON_EPSD; }

// A scattering coefficient table [n_mat][n_cell][2] (c0 + c1 E per cell of
// the mu tables) is finite and its line is >= 0 at both ends of every cell,
// so on the whole cell; the first cell's line from E = 0 (lower energies
// take the first cell, and Compton events lower the energy).
static bool scatter_table_ok(const double* t, const mcx_material_tables* mats) {
  const int nc = mats->n_cell;
  const double de = (mats->e_max - mats->e_min) / nc;
  for (int m = 0; m < mats->n_mat; ++m)
    for (int j = 0; j < nc; ++j) {
      const double c0 = t[((size_t)m * nc + j) * 2], c1 = t[((size_t)m * nc + j) * 2 + 1];
      if (!std::isfinite(c0) || !std::isfinite(c1)) return false;
      const double lo = j == 0 ? 0.0 : mats->e_min + j * de, hi = mats->e_min + (j + 1) * de;
      if (!(c0 + c1 * lo >= 0.0) || !(c0 + c1 * hi >= 0.0)) return false;
    }
  return true;
}

// Checks one component description; returns an error message or nullptr.
static const char* check_component(const mcx_component_desc& c, int index,
                                   const mcx_material_tables* mats, const mcx_phantom* ph) {
  if (!finite_all(c.pos, 3) || !finite_all(c.rot, 9) || !finite_all(c.p, 12))
    return "non-finite position, rotation or parameter";
  if (c.relative_to >= index || c.relative_to < -1) return "relative_to must name an earlier component";
  // rotation: orthonormal to 1e-6
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double d = 0.0;
      for (int k = 0; k < 3; ++k) d += c.rot[3 * i + k] * c.rot[3 * j + k];
      if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-6) return "rotation is not orthonormal";
    }
  const double* p = c.p;
  switch (c.type) {
    case MCX_SOURCE:
      if (index != 0) return "only component 0 may be the source";
      if (c.shape < MCX_SHAPE_POINT || c.shape > MCX_SHAPE_GAUSS) return "unknown source shape";
      if (c.spectrum != MCX_SPEC_FLAT && c.spectrum != MCX_SPEC_KRAMERS && c.spectrum != MCX_SPEC_GAUSS)
        return "unknown spectrum";
      if (c.shape == MCX_SHAPE_GAUSS && (p[9] < 0 || p[10] < 0)) return "negative divergence";
      if (c.spectrum == MCX_SPEC_GAUSS && (!(p[4] > 0) || p[8] < 0))
        return "Gaussian spectrum needs e0 > 0 and sigma_e >= 0";
      if (p[0] < 0 || p[1] < 0 || p[6] < 0 || p[7] < 0) return "negative source or target size";
      if (!(p[5] > 0)) return "target distance must be positive";
      if (!(p[2] >= 0) || !(p[3] >= p[2])) return "energy band must satisfy 0 <= e_min <= e_max";
      if (c.spectrum == MCX_SPEC_KRAMERS && (!(p[2] > 0) || !(p[3] > p[2]) || !(p[4] >= p[3])))
        return "Kramers spectrum needs 0 < e_min < e_max <= e0";
      return nullptr;
    case MCX_SLIT_RECT:
      return (p[0] <= p[1] && p[2] <= p[3]) ? nullptr : "slit needs xmin <= xmax and ymin <= ymax";
    case MCX_SLIT_CIRC:
      return p[0] >= 0 ? nullptr : "negative slit radius";
    case MCX_ABS_BOX:
    case MCX_ABS_CYL:
    case MCX_ABS_SPHERE:
      if (!mats || c.material < 0 || c.material >= mats->n_mat) return "absorber material out of range";
      if (c.type == MCX_ABS_BOX && !(p[0] > 0 && p[1] > 0 && p[2] > 0)) return "box widths must be positive";
      if (c.type == MCX_ABS_CYL && !(p[0] > 0 && p[1] > 0)) return "cylinder size must be positive";
      if (c.type == MCX_ABS_SPHERE && !(p[0] > 0)) return "sphere radius must be positive";
      return nullptr;
    case MCX_PHANTOM:
      if (!ph || !ph->vox || !mats) return "phantom needs mcx_phantom bytes and material tables";
      if (c.n[0] != ph->nx || c.n[1] != ph->ny || c.n[2] != ph->nz) return "phantom size mismatch";
      if (c.n[0] < 1 || c.n[1] < 1 || c.n[2] < 1) return "empty phantom";
      if ((double)c.n[0] * c.n[1] * c.n[2] > 2147483647.0) return "phantom larger than 2^31 voxels";
      if (!(p[0] > 0)) return "voxel size must be positive";
      if (!(p[1] >= 0 && p[1] <= 64)) return "march steps per voxel must lie in [0, 64] (0: exact walk)";
      if (p[4] != 0.0) {
        if (!(p[1] > 0)) return "a scattering phantom needs the fixed-step march (p1 > 0)";
        if (!ph->mu_scatter) return "a scattering phantom needs mcx_phantom.mu_scatter";
        if (mats->n_mat > kMaxMats / 2) return "a scattering phantom takes at most 32 materials";
        if (!scatter_table_ok(ph->mu_scatter, mats))
          return "scattering coefficients must be finite and >= 0 on every cell";
        if (ph->mu_compton && !scatter_table_ok(ph->mu_compton, mats))
          return "Compton coefficients must be finite and >= 0 on every cell";
      }
      return nullptr;
    case MCX_MON_PSD:
    case MCX_MON_E:
    case MCX_MON_L:
    case MCX_MON_EPSD: {
      if (!(p[0] < p[1] && p[2] < p[3])) return "monitor extent needs xmin < xmax and ymin < ymax";
      if (c.type != MCX_MON_PSD && !(p[4] < p[5])) return "monitor range needs lo < hi";
      if (c.type == MCX_MON_L && !(p[4] > 0)) return "wavelength range must be positive";
      int nd = c.type == MCX_MON_PSD ? 2 : (c.type == MCX_MON_EPSD ? 3 : 1);
      double total = 1;
      for (int i = 0; i < nd; ++i) {
        if (c.n[i] < 1) return "monitor needs at least one bin per axis";
        total *= c.n[i];
      }
      if (total > 4.0e9) return "monitor larger than 4e9 bins";
      return nullptr;
    }
    case MCX_LENS_PARAB:
      if (!mats || c.material < 0 || c.material >= mats->n_mat) return "lens material out of range";
      if (!(p[0] > 0) || !(p[2] > 0) || p[1] < 0 || !(p[6] > 0))
        return "lens needs R > 0, aperture > 0, d >= 0, pitch > 0";
      if (c.n[0] < 1 || c.n[0] > 4096 || p[3] != (double)c.n[0]) return "lens needs 1 <= N = n0 = p3 <= 4096";
      if (!(p[4] >= 0 && p[4] < 1e-2) || !(p[5] > 0)) return "lens needs 0 <= delta0 < 1e-2 and e_ref > 0";
      return nullptr;
    default:
      return "unknown component type";
  }
}

// Lab frame of every component: placed relative to p at o_p + R_p pos with
// rotation R_p rot.
static void place(const mcx_component_desc* comps, int n, std::vector<DevComp>& out) {
  out.assign(n, DevComp{});
  for (int i = 0; i < n; ++i) {
    const mcx_component_desc& c = comps[i];
    DevComp& d = out[i];
    if (c.relative_to < 0) {
      for (int k = 0; k < 3; ++k) d.o[k] = c.pos[k];
      for (int k = 0; k < 9; ++k) d.R[k] = c.rot[k];
    } else {
      const DevComp& q = out[c.relative_to];
      for (int r = 0; r < 3; ++r) {
        d.o[r] = q.o[r] + (q.R[3 * r] * c.pos[0] + q.R[3 * r + 1] * c.pos[1] + q.R[3 * r + 2] * c.pos[2]);
        for (int col = 0; col < 3; ++col)
          d.R[3 * r + col] = q.R[3 * r] * c.rot[col] + q.R[3 * r + 1] * c.rot[3 + col] +
                             q.R[3 * r + 2] * c.rot[6 + col];
      }
    }
    bool ident = true;
    for (int k = 0; k < 9; ++k) ident = ident && d.R[k] == ((k % 4 == 0) ? 1.0 : 0.0);
    d.identity = ident ? 1 : 0;
  }
}

extern "C" mcx_status mcx_instrument_create(const mcx_component_desc* comps, int32_t n_comps,
                                            const mcx_material_tables* mats, const mcx_phantom* ph,
                                            const mcx_options* opt, mcx_instrument** out) {
  if (!out) return fail(MCX_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!comps || !opt) return fail(MCX_ERR_INVALID, "comps and opt must not be NULL");
  if (n_comps < 1 || n_comps > kMaxComps)
    return fail(MCX_ERR_INVALID, "n_comps must be in [1, %d]", kMaxComps);
  if (opt->precision != MCX_PREC_FP64 && opt->precision != MCX_PREC_MIXED)
    return fail(MCX_ERR_INVALID, "unknown precision %d", opt->precision);
  if (opt->instr_id < 0) return fail(MCX_ERR_INVALID, "instr_id must be >= 0");
  if ((opt->alloc == nullptr) != (opt->free == nullptr))
    return fail(MCX_ERR_INVALID, "alloc and free hooks must be given together");
  if (opt->block_size && (opt->block_size < 32 || opt->block_size > 256 || opt->block_size % 32))
    return fail(MCX_ERR_INVALID, "block_size must be a multiple of 32 in [32, 256]");
  if (opt->blocks_per_sm < 0) return fail(MCX_ERR_INVALID, "blocks_per_sm must be >= 0");
  if (comps[0].type != MCX_SOURCE) return fail(MCX_ERR_INVALID, "component 0 must be the source");
  if (mats) {
    if (mats->n_mat < 1 || mats->n_mat > kMaxMats || mats->n_cell < 1 || !mats->coef ||
        !(mats->e_min < mats->e_max) || !std::isfinite(mats->e_min) || !std::isfinite(mats->e_max))
      return fail(MCX_ERR_INVALID, "material tables need 1..%d materials, cells, coef and e_min < e_max",
                  kMaxMats);
    if (!finite_all(mats->coef, 2 * mats->n_mat * mats->n_cell))
      return fail(MCX_ERR_INVALID, "material table holds a non-finite coefficient");
  }
  int n_phantoms = 0, vox_kind = kVoxNone;
  for (int i = 0; i < n_comps; ++i) {
    if (const char* msg = check_component(comps[i], i, mats, ph))
      return fail(MCX_ERR_INVALID, "component %d: %s", i, msg);
    if (comps[i].type == MCX_PHANTOM) {
      ++n_phantoms;
      vox_kind |= comps[i].p[1] > 0.0 ? kVoxMarch : kVoxWalk;
    }
    if (comps[i].type == MCX_LENS_PARAB ||
        (comps[i].type == MCX_SOURCE &&
         (comps[i].shape == MCX_SHAPE_GAUSS || comps[i].spectrum == MCX_SPEC_GAUSS)))
      vox_kind |= kOptics;
  }
  if (n_phantoms > 1) return fail(MCX_ERR_INVALID, "at most one phantom per instrument");
  if (n_phantoms == 1) {
    const size_t nv = (size_t)ph->nx * ph->ny * ph->nz;
    for (size_t i = 0; i < nv; ++i)
      if (ph->vox[i] >= mats->n_mat) return fail(MCX_ERR_INVALID, "phantom voxel %zu names material %d >= n_mat", i, ph->vox[i]);
  }

  DeviceGuard guard(opt->device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", opt->device);

  mcx_instrument* I = new mcx_instrument();
  I->device = opt->device;
  I->stream = (cudaStream_t)opt->stream;
  I->precision = opt->precision;
  I->alloc = opt->alloc;
  I->free_fn = opt->free;
  I->alloc_ctx = opt->alloc_ctx;
  I->has_phantom = n_phantoms == 1;
  I->vox_kind = vox_kind;

  place(comps, n_comps, I->comps);
  I->mon_off.assign(n_comps, -1);
  I->mon_bins.assign(n_comps, 0);
  int64_t off = 0;
  for (int i = 0; i < n_comps; ++i) {
    const mcx_component_desc& c = comps[i];
    DevComp& d = I->comps[i];
    d.type = c.type;
    d.shape = c.shape;
    d.spectrum = c.spectrum;
    d.material = c.material;
    for (int k = 0; k < 3; ++k) d.n[k] = c.n[k];
    for (int k = 0; k < 12; ++k) d.p[k] = c.p[k];
    if (c.type == MCX_SOURCE && c.spectrum == MCX_SPEC_KRAMERS) {
      // mean of f(E) = (e0 - E)/E over [e_min, e_max]
      const double lo = c.p[2], hi = c.p[3], e0 = c.p[4];
      const double fbar = (e0 * log(hi / lo) - (hi - lo)) / (hi - lo);
      d.aux[0] = 1.0 / fbar;
      d.aux[1] = fbar;
    }
    if (c.type == MCX_SOURCE && c.shape == MCX_SHAPE_GAUSS) {
      // divergence weights: 1 / (D sigma') per axis (0: none)
      d.inv[0] = c.p[9] > 0.0 ? 1.0 / (c.p[5] * c.p[9]) : 0.0;
      d.inv[1] = c.p[10] > 0.0 ? 1.0 / (c.p[5] * c.p[10]) : 0.0;
    }
    if (c.type == MCX_LENS_PARAB) {
      d.inv[0] = 1.0 / c.p[0];     // 1 / R
      d.aux[0] = 0.5 * c.p[1];     // half the apex thickness
    }
    if (c.type == MCX_PHANTOM) {
      d.inv[0] = 1.0 / c.p[0];
      for (int k = 0; k < 3; ++k) d.aux[k] = 0.5 * (double)c.n[k] * c.p[0];
      // fixed-step traversal: p2 = the step, p3 = a bound on the steps of
      // any chord of the grid (diagonal / step + 2)
      d.p[2] = d.p[3] = 0.0;
      if (c.p[1] > 0.0) {
        const double h = c.p[0] / c.p[1];
        double diag2 = 0.0;
        for (int k = 0; k < 3; ++k) diag2 += (2.0 * d.aux[k]) * (2.0 * d.aux[k]);
        d.p[2] = h;
        d.p[3] = std::ceil(std::sqrt(diag2) / h) + 2.0;
      }
    }
    if (is_monitor(c.type)) {
      d.restore = c.p[11] != 0.0 ? 1 : 0;
      int64_t nb;
      if (c.type == MCX_MON_PSD) {
        nb = (int64_t)c.n[0] * c.n[1];
        d.inv[0] = (double)c.n[0] / (c.p[1] - c.p[0]);
        d.inv[1] = (double)c.n[1] / (c.p[3] - c.p[2]);
      } else if (c.type == MCX_MON_EPSD) {
        nb = (int64_t)c.n[0] * c.n[1] * c.n[2];
        d.inv[0] = (double)c.n[0] / (c.p[1] - c.p[0]);
        d.inv[1] = (double)c.n[1] / (c.p[3] - c.p[2]);
        d.inv[2] = (double)c.n[2] / (c.p[5] - c.p[4]);
      } else {
        nb = c.n[0];
        d.inv[2] = (double)c.n[0] / (c.p[5] - c.p[4]);
      }
      d.mon_offset = off;
      I->mon_off[i] = off;
      I->mon_bins[i] = nb;
      off += nb;
    }
  }
  I->n_bins = off;
  // block-private copies for small monitors (their bins take most hits per
  // bin, so global atomics would queue on a few L2 sectors)
  int32_t n_priv = 0;
  for (int i = 0; i < n_comps; ++i) {
    DevComp& d = I->comps[i];
    d.priv = -1;
    if (I->mon_off[i] >= 0 && I->mon_bins[i] <= kPrivMonBins && n_priv + I->mon_bins[i] <= kMaxPrivBins) {
      d.priv = n_priv;
      n_priv += (int32_t)I->mon_bins[i];
    }
  }
  for (int i = 0; i < n_comps; ++i) {
    DevComp& d = I->comps[i];
    for (int k = 0; k < 12; ++k) d.pf[k] = (float)d.p[k];
    for (int k = 0; k < 9; ++k) d.Rf[k] = (float)d.R[k];
    for (int k = 0; k < 3; ++k) {
      d.invf[k] = (float)d.inv[k];
      d.auxf[k] = (float)d.aux[k];
    }
    d.zo = (d.o[0] == 0.0 ? 1 : 0) | (d.o[1] == 0.0 ? 2 : 0) | (d.o[2] == 0.0 ? 4 : 0);
    d.last = i == n_comps - 1 ? 1 : 0;
  }

  {
    // monitor updates keep their lines in the L2 when the global monitors
    // take at most 7/8 of it (a 100 MB detector on a 126 MB L2: yes; a
    // 201 MB one: no, its lines would push the rest, a phantom, out)
    uint64_t gbytes = 0;
    for (int c = 0; c < n_comps; ++c)
      if (I->mon_off[c] >= 0 && I->comps[c].priv < 0) gbytes += (uint64_t)I->mon_bins[c] * sizeof(MonBin);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, I->device);
    const int keep = gbytes > 0 && l2 > 0 && gbytes <= (uint64_t)l2 / 8 * 7 ? 1 : 0;
    for (int c = 0; c < n_comps; ++c) I->comps[c].l2keep = (I->mon_off[c] >= 0 && I->comps[c].priv < 0) ? keep : 0;
  }

  // ---- device buffers (uploaded once, resident until destroy)
  cudaError_t e;
  DevComp* d_comps = (DevComp*)dev_alloc(I, sizeof(DevComp) * kMaxComps);
  MonBin* d_bins = (MonBin*)dev_alloc(I, sizeof(MonBin) * (size_t)(off > 0 ? off : 1));
  double* d_tally = (double*)dev_alloc(I, sizeof(double) * (kMaxComps + 2));
  if (!d_comps || !d_bins || !d_tally) {
    release(I);
    return fail(MCX_ERR_OOM, "device allocation failed");
  }
  e = cudaMemcpyAsync(d_comps, I->comps.data(), sizeof(DevComp) * n_comps, cudaMemcpyHostToDevice, I->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bins, 0, sizeof(MonBin) * (size_t)(off > 0 ? off : 1), I->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tally, 0, sizeof(double) * (kMaxComps + 2), I->stream);
  DevInstrument& D = I->dev;
  D.comps = d_comps;
  D.n_comp = n_comps;
  D.instr_id = opt->instr_id;
  D.bins = d_bins;
  D.tallies = d_tally;
  D.n_priv = n_priv;
  D.vox_kind = vox_kind;
  if (e == cudaSuccess && mats) {
    const size_t nc = (size_t)mats->n_mat * mats->n_cell;
    std::vector<double2> h64(nc);
    std::vector<float2> h32(nc);
    for (size_t i = 0; i < nc; ++i) {
      h64[i] = make_double2(mats->coef[2 * i], mats->coef[2 * i + 1]);
      h32[i] = make_float2((float)mats->coef[2 * i], (float)mats->coef[2 * i + 1]);
    }
    double2* d64 = (double2*)dev_alloc(I, sizeof(double2) * nc);
    float2* d32 = (float2*)dev_alloc(I, sizeof(float2) * nc);
    if (!d64 || !d32) {
      release(I);
      return fail(MCX_ERR_OOM, "device allocation failed");
    }
    e = cudaMemcpy(d64, h64.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d32, h32.data(), sizeof(float2) * nc, cudaMemcpyHostToDevice);
    D.mu64 = d64;
    D.mu32 = d32;
    D.n_mat = mats->n_mat;
    D.n_cell = mats->n_cell;
    D.e_min = mats->e_min;
    D.cell_inv = (double)mats->n_cell / (mats->e_max - mats->e_min);
    D.e_min_f = (float)D.e_min;
    D.cell_inv_f = (float)D.cell_inv;
  }
  if (e == cudaSuccess && I->has_phantom) {
    // Device layout: the phantom axis closest to the source -> phantom
    // direction (in the phantom's frame) becomes the contiguous one, so the
    // voxels a ray walks through in turn share cache lines.
    int pc = 0;
    while (I->comps[pc].type != T_PHANTOM) ++pc;
    DevComp& P = I->comps[pc];
    const DevComp& S = I->comps[0];
    double dl[3];
    for (int i = 0; i < 3; ++i) {
      dl[i] = 0.0;
      for (int j = 0; j < 3; ++j) dl[i] += P.R[3 * j + i] * (P.o[j] - S.o[j]);
    }
    int order[3] = {2, 1, 0};   // fastest first; default z, y, x
    if (std::fabs(dl[0]) + std::fabs(dl[1]) + std::fabs(dl[2]) > 0.0) {
      order[0] = 0; order[1] = 1; order[2] = 2;
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
          if (std::fabs(dl[order[b]]) > std::fabs(dl[order[a]])) std::swap(order[a], order[b]);
    }
    const int n[3] = {ph->nx, ph->ny, ph->nz};
    int64_t stride[3];
    stride[order[0]] = 1;
    stride[order[1]] = n[order[0]];
    stride[order[2]] = (int64_t)n[order[0]] * n[order[1]];
    for (int i = 0; i < 3; ++i) P.vstride[i] = (int32_t)stride[i];
    const size_t nv = (size_t)ph->nx * ph->ny * ph->nz;
    // padded with zero bytes to a whole number of 16-byte words: the walk
    // loads the aligned word that holds a voxel, never past the allocation
    const size_t nv_pad = (nv + 15) & ~(size_t)15;
    std::vector<uint8_t> lay(nv_pad, 0);
    for (int z = 0; z < n[2]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[0]; ++x)
          lay[x * stride[0] + y * stride[1] + z * stride[2]] =
              ph->vox[((size_t)z * n[1] + y) * n[0] + x];
    // The walk is clipped to the bounding box of the voxels whose material
    // attenuates (a table row not all zero): transparent margins contribute
    // exactly zero, so skipping them changes tau only by rounding.  The box
    // sits in p[6..11] as local (lo, hi) pairs per axis; a full axis keeps
    // exactly -/+ the half extent.
    std::vector<char> opaque(mats->n_mat, 0);
    for (int m = 0; m < mats->n_mat; ++m)
      for (int j = 0; j < 2 * mats->n_cell && !opaque[m]; ++j)
        opaque[m] = mats->coef[(size_t)m * 2 * mats->n_cell + j] != 0.0;
    int blo[3] = {n[0], n[1], n[2]}, bhi[3] = {0, 0, 0};
    for (int z = 0; z < n[2]; ++z)
      for (int y = 0; y < n[1]; ++y)
        for (int x = 0; x < n[0]; ++x)
          if (opaque[ph->vox[((size_t)z * n[1] + y) * n[0] + x]]) {
            const int q[3] = {x, y, z};
            for (int i = 0; i < 3; ++i) {
              blo[i] = std::min(blo[i], q[i]);
              bhi[i] = std::max(bhi[i], q[i] + 1);
            }
          }
    for (int i = 0; i < 3; ++i) {
      if (bhi[i] <= blo[i]) blo[i] = bhi[i] = 0;   // nothing attenuates: an empty box
      const double v = P.p[0], h = P.aux[i];
      P.p[6 + 2 * i] = blo[i] == 0 ? -h : (double)blo[i] * v - h;
      P.p[7 + 2 * i] = bhi[i] == n[i] ? h : (double)bhi[i] * v - h;
      P.pf[6 + 2 * i] = (float)P.p[6 + 2 * i];
      P.pf[7 + 2 * i] = (float)P.p[7 + 2 * i];
    }
    uint8_t* dv = (uint8_t*)dev_alloc(I, nv_pad);
    if (!dv) {
      release(I);
      return fail(MCX_ERR_OOM, "device allocation failed");
    }
    e = cudaMemcpy(dv, lay.data(), nv_pad, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d_comps + pc, &P, sizeof(DevComp), cudaMemcpyHostToDevice);
    D.vox = dv;
    if (P.p[4] != 0.0) {
      // scattering coefficient tables [Rayleigh | Compton][n_mat][n_cell]
      // (c0, c1), binary64 and each coefficient rounded once to binary32;
      // no Compton table: zeros
      const size_t nt = (size_t)mats->n_mat * (size_t)mats->n_cell * 2;
      std::vector<double> m64(2 * nt, 0.0);
      std::vector<float> m32(2 * nt, 0.f);
      for (size_t i = 0; i < nt; ++i) {
        m64[i] = ph->mu_scatter[i];
        if (ph->mu_compton) m64[nt + i] = ph->mu_compton[i];
      }
      for (size_t i = 0; i < 2 * nt; ++i) m32[i] = (float)m64[i];
      double* d64 = (double*)dev_alloc(I, sizeof(double) * 2 * nt);
      float* d32 = d64 ? (float*)dev_alloc(I, sizeof(float) * 2 * nt) : nullptr;
      if (!d32) {
        release(I);
        return fail(MCX_ERR_OOM, "device allocation failed");
      }
      if (e == cudaSuccess) e = cudaMemcpy(d64, m64.data(), sizeof(double) * 2 * nt, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(d32, m32.data(), sizeof(float) * 2 * nt, cudaMemcpyHostToDevice);
      D.sc64 = d64;
      D.sc32 = d32;
      I->scatter = true;
    }
    // ray-order scratch: a chunk's tile keys and permutation, the tile counters
    I->ord_keys = (uint16_t*)dev_alloc(I, sizeof(uint16_t) * kOrderChunk);
    I->ord_perm = I->ord_keys ? (uint32_t*)dev_alloc(I, sizeof(uint32_t) * kOrderChunk) : nullptr;
    I->ord_hist = I->ord_perm ? (uint32_t*)dev_alloc(I, sizeof(uint32_t) * (kTiles + 64)) : nullptr;
    I->ord_ticket = I->ord_hist ? I->ord_hist + kTiles : nullptr;
    if (!I->ord_hist) {
      release(I);
      return fail(MCX_ERR_OOM, "device allocation failed");
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) {
    mcx_status s = cuda_fail(e, "upload");
    release(I);
    return s;
  }

  // ---- launch shape: persistent grid of (SMs x resident blocks)
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, I->device);
  const int block = opt->block_size ? opt->block_size : 256;
  // a scattering phantom keeps a second per-thread column (the scattering sums)
  const size_t smem = trace_smem_bytes(n_comps, D.n_mat * (I->scatter ? 2 : 1), block, I->precision,
                                       I->has_phantom, D.n_priv);
  int bpsm = opt->blocks_per_sm ? opt->blocks_per_sm
                                 : trace_occupancy(I->precision, I->vox_kind | (I->scatter ? kScatter : 0), block, smem);
  if (bpsm < 1) bpsm = 1;
  I->shape.block = block;
  I->shape.smem = smem;
  I->shape.grid = n_sm * bpsm;
  I->user_blocks_per_sm = opt->blocks_per_sm;
  *out = I;
  g_last_error.clear();
  return MCX_OK;
}

namespace mcx {

cudaError_t trace_dispatch(const mcx_instrument* I, DevInstrument d, uint64_t begin, uint64_t end,
                           uint64_t seed) {
  if (!I->ord_perm)
    return I->spec_kernel ? launch_spec(I, d, begin, end, seed)
                          : launch_trace(d, I->precision, begin, end, seed, I->shape, I->stream);
  // a phantom: each chunk's ids grouped by aim-point tile, then traced
  cudaError_t e = cudaSuccess;
  for (uint64_t c0 = begin; c0 < end && e == cudaSuccess; c0 += kOrderChunk) {
    const uint64_t c1 = end - c0 < (uint64_t)kOrderChunk ? end : c0 + kOrderChunk;
    e = launch_ray_order(d, I->precision, c0, c1, seed, I->ord_keys, I->ord_hist, I->ord_perm, I->stream);
    d.perm = I->ord_perm;
    d.perm_base = c0;
    d.ticket = I->ord_ticket;
    if (e == cudaSuccess) e = cudaMemsetAsync(I->ord_ticket, 0, sizeof(unsigned), I->stream);
    if (e == cudaSuccess)
      e = I->spec_kernel ? launch_spec(I, d, c0, c1, seed)
                         : launch_trace(d, I->precision, c0, c1, seed, I->shape, I->stream);
  }
  return e;
}

}  // namespace mcx

extern "C" mcx_status mcx_trace_range(mcx_instrument* I, uint64_t ray_begin, uint64_t ray_end,
                                      uint64_t seed) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  if (ray_end < ray_begin) return fail(MCX_ERR_INVALID, "ray_end < ray_begin");
  if (ray_end > (1ull << 62)) return fail(MCX_ERR_INVALID, "ray ids must stay below 2^62");
  if (ray_end == ray_begin) return MCX_OK;
  DeviceGuard guard(I->device);
  cudaError_t e = cudaSuccess;
  if (I->prop) {
    // learned starts: sample a chunk into the instrument's start buffer, trace
    // it, next chunk (stream order keeps the buffer's uses apart)
    const mcx_status st = proposal_check(I->prop, I->stream);
    if (st != MCX_OK) return st;
    for (uint64_t c0 = ray_begin; c0 < ray_end && e == cudaSuccess; c0 += kPropChunk) {
      const uint64_t n = ray_end - c0 < kPropChunk ? ray_end - c0 : kPropChunk;
      e = proposal_sample_async(I->prop, I->dev, c0, n, seed, I->prop_angle, I->prop_buf, I->stream);
      DevInstrument d = I->dev;
      d.ext = I->prop_buf;
      d.ext_base = c0;
      d.ext_n = n;
      d.det_w = nullptr;
      if (e == cudaSuccess) e = trace_dispatch(I, d, c0, c0 + n, 0);
    }
  } else {
    e = trace_dispatch(I, I->dev, ray_begin, ray_end, seed);
  }
  if (e != cudaSuccess) return cuda_fail(e, "trace launch");
  I->n_emit += ray_end - ray_begin;
  return MCX_OK;
}

extern "C" mcx_status mcx_trace(mcx_instrument* I, uint64_t n_rays, uint64_t seed) {
  return mcx_trace_range(I, 0, n_rays, seed);
}

extern "C" mcx_status mcx_monitor_bins(const mcx_instrument* I, int32_t comp, size_t* n_bins) {
  if (!I || !n_bins) return fail(MCX_ERR_INVALID, "NULL argument");
  if (comp < 0 || comp >= (int)I->comps.size() || I->mon_off[comp] < 0)
    return fail(MCX_ERR_INVALID, "component %d is not a monitor", comp);
  *n_bins = (size_t)I->mon_bins[comp];
  return MCX_OK;
}

// The device address of page-locked host memory the device can write
// (cudaHostAlloc'd memory is mapped under unified addressing), else null.
static void* device_view(void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Queues on the instrument's stream: the bins of monitor `comp` split into
// the readout scratch (allocated on first use), then one DMA copy per given
// host array.  Does not synchronise.
static mcx_status queue_split_copies(mcx_instrument* I, int32_t comp, size_t nb, uint64_t* N, double* sw,
                                     double* sw2) {
  if (!I->split) {
    int64_t most = 1;
    for (int64_t b : I->mon_bins) most = b > most ? b : most;
    I->split = dev_alloc(I, sizeof(MonBin) * (size_t)most);
    if (!I->split) return fail(MCX_ERR_OOM, "monitor readout scratch");
  }
  unsigned long long* dN = (unsigned long long*)I->split;
  double* dsw = (double*)(dN + nb);
  double* dsw2 = dsw + nb;
  cudaError_t e = launch_split_bins(I->dev.bins + I->mon_off[comp], nb, N ? dN : nullptr,
                                    sw ? dsw : nullptr, sw2 ? dsw2 : nullptr, I->stream);
  if (e == cudaSuccess && N)
    e = cudaMemcpyAsync(N, dN, sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess && sw)
    e = cudaMemcpyAsync(sw, dsw, sizeof(double) * nb, cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess && sw2)
    e = cudaMemcpyAsync(sw2, dsw2, sizeof(double) * nb, cudaMemcpyDeviceToHost, I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "monitor read");
  return MCX_OK;
}

extern "C" mcx_status mcx_monitor_read(mcx_instrument* I, int32_t comp, uint64_t* N, double* sw,
                                       double* sw2, size_t n_bins) {
  size_t nb = 0;
  mcx_status s = mcx_monitor_bins(I, comp, &nb);
  if (s != MCX_OK) return s;
  if (n_bins != nb) return fail(MCX_ERR_INVALID, "monitor %d has %zu bins, caller gave %zu", comp, nb, n_bins);
  DeviceGuard guard(I->device);
  {
    // page-locked outputs: the split kernel writes them directly over the
    // host link, with no device copy and no DMA step
    void* vN = device_view(N);
    void* vsw = device_view(sw);
    void* vsw2 = device_view(sw2);
    if ((!N || vN) && (!sw || vsw) && (!sw2 || vsw2)) {
      cudaError_t e = launch_split_bins(I->dev.bins + I->mon_off[comp], nb, (unsigned long long*)vN,
                                        (double*)vsw, (double*)vsw2, I->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
      if (e != cudaSuccess) return cuda_fail(e, "monitor read");
      return MCX_OK;
    }
  }
  const mcx_status st = queue_split_copies(I, comp, nb, N, sw, sw2);
  if (st != MCX_OK) return st;
  const cudaError_t e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "monitor read");
  return MCX_OK;
}

extern "C" mcx_status mcx_monitor_read_async(mcx_instrument* I, int32_t comp, uint64_t* N, double* sw,
                                             double* sw2, size_t n_bins) {
  size_t nb = 0;
  mcx_status s = mcx_monitor_bins(I, comp, &nb);
  if (s != MCX_OK) return s;
  if (n_bins != nb) return fail(MCX_ERR_INVALID, "monitor %d has %zu bins, caller gave %zu", comp, nb, n_bins);
  DeviceGuard guard(I->device);
  return queue_split_copies(I, comp, nb, N, sw, sw2);
}

extern "C" mcx_status mcx_monitor_total(mcx_instrument* I, int32_t comp, uint64_t* N, double* sum_w,
                                        double* sum_w2) {
  size_t nb = 0;
  mcx_status s = mcx_monitor_bins(I, comp, &nb);
  if (s != MCX_OK) return s;
  DeviceGuard guard(I->device);
  if (!I->totals) {
    I->totals = dev_alloc(I, 32);
    if (!I->totals) return fail(MCX_ERR_OOM, "monitor totals scratch");
  }
  unsigned long long* dN = (unsigned long long*)I->totals;
  double* dw = (double*)I->totals + 1;
  unsigned long long hN = 0;
  double hw[2] = {0.0, 0.0};
  cudaError_t e = launch_total_bins(I->dev.bins + I->mon_off[comp], nb, dN, dw, I->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hN, dN, sizeof(hN), cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hw, dw, sizeof(hw), cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "monitor total");
  if (N) *N = hN;
  if (sum_w) *sum_w = hw[0];
  if (sum_w2) *sum_w2 = hw[1];
  return MCX_OK;
}

extern "C" mcx_status mcx_tally_read(mcx_instrument* I, double* lost, int32_t n, uint64_t* n_emit,
                                     double* sum_w0, double* sum_wend) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  const int nc = (int)I->comps.size();
  if (lost && n != nc) return fail(MCX_ERR_INVALID, "lost needs %d entries, caller gave %d", nc, n);
  DeviceGuard guard(I->device);
  double h[kMaxComps + 2];
  cudaError_t e = cudaMemcpyAsync(h, I->dev.tallies, sizeof(double) * (nc + 2), cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tally read");
  if (lost)
    for (int i = 0; i < nc; ++i) lost[i] = h[i];
  if (n_emit) *n_emit = I->n_emit;
  if (sum_w0) *sum_w0 = h[nc];
  if (sum_wend) *sum_wend = h[nc + 1];
  return MCX_OK;
}

extern "C" mcx_status mcx_loss_read(mcx_instrument* I, double* per_component_lost_w, int32_t n) {
  if (!per_component_lost_w) return fail(MCX_ERR_INVALID, "per_component_lost_w is NULL");
  return mcx_tally_read(I, per_component_lost_w, n, nullptr, nullptr, nullptr);
}

extern "C" mcx_status mcx_monitor_reset(mcx_instrument* I) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  DeviceGuard guard(I->device);
  cudaError_t e = cudaMemsetAsync(I->dev.bins, 0, sizeof(MonBin) * (size_t)(I->n_bins > 0 ? I->n_bins : 1), I->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(I->dev.tallies, 0, sizeof(double) * (kMaxComps + 2), I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reset");
  I->n_emit = 0;
  return MCX_OK;
}

extern "C" mcx_status mcx_synchronize(mcx_instrument* I) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  DeviceGuard guard(I->device);
  cudaError_t e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  return MCX_OK;
}

extern "C" void mcx_instrument_destroy(mcx_instrument* I) {
  if (!I) return;
  DeviceGuard guard(I->device);
  release(I);
}

extern "C" mcx_status mcx_philox_fill(const uint32_t* ctr_key, uint32_t* out, size_t n,
                                      int32_t device) {
  if ((!ctr_key || !out) && n) return fail(MCX_ERR_INVALID, "NULL buffer");
  if (n == 0) return MCX_OK;
  if (n > ((size_t)1 << 28)) return fail(MCX_ERR_INVALID, "n too large");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", device);
  uint32_t *d_in = nullptr, *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_in, n * 6 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, n * 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, ctr_key, n * 6 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox_fill(d_in, d_out, n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_fail(e, "philox fill");
  return MCX_OK;
}

extern "C" mcx_status mcx_convert_fill(const double* in, float* out_f, double* out_d, size_t n,
                                       int32_t device) {
  if ((!in || !out_f || !out_d) && n) return fail(MCX_ERR_INVALID, "NULL buffer");
  if (n == 0) return MCX_OK;
  if (n > ((size_t)1 << 28)) return fail(MCX_ERR_INVALID, "n too large");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", device);
  double *d_in = nullptr, *d_od = nullptr;
  float* d_of = nullptr;
  cudaError_t e = cudaMalloc(&d_in, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_od, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_of, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_convert_fill(d_in, d_of, d_od, n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out_f, d_of, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(out_d, d_od, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_od);
  cudaFree(d_of);
  if (e != cudaSuccess) return cuda_fail(e, "convert fill");
  return MCX_OK;
}
