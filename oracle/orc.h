/*
 * orc.h -- CPU oracle of the forward Monte Carlo X-ray ray tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is a plain, slow, single-ray-at-a-time
 * FP64 C implementation of what the traced path computes.  Only the test
 * suite, the package's smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never does.  It shares no code, header, table or
 * constant generator with the CUDA library: both follow the same written
 * draw-and-arithmetic contract independently.
 *
 * What it follows (McXtrace model, arXiv 2410.08747):
 *   - rays are independent (Sec. 2.2) and each is generated at the source and
 *     passed through the component list in order, any component may absorb
 *     it (Sec. 1, Sec. 2.1);
 *   - the particle carries position, wavevector (here direction + energy) and
 *     Monte Carlo weight p (Sec. 2.2.2, the _particle list);
 *   - the per-ray random stream is a counter-based Philox4x32-10 (the paper
 *     re-implements the generator for the GPU but does not name it; Philox is
 *     the reading adopted here), Salmon et al., SC'11;
 *   - monitors accumulate count, sum of weights and sum of squared weights
 *     per bin (the McXtrace monitor convention N, I, I^2).
 *
 * Units: metres, keV, 1/m.  All floating point here is IEEE binary64 unless
 * the decision type of mode 32 is used (see orc_trace.c); the file must be
 * compiled with -ffp-contract=off.
 */
#ifndef ORC_H
#define ORC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum orc_type {
  ORC_SOURCE = 0,
  ORC_SLIT_RECT = 1,
  ORC_SLIT_CIRC = 2,
  ORC_ABS_BOX = 3,
  ORC_ABS_CYL = 4,
  ORC_ABS_SPHERE = 5,
  ORC_PHANTOM = 6,
  ORC_MON_PSD = 7,
  ORC_MON_E = 8,
  ORC_MON_L = 9,
  ORC_MON_EPSD = 10,
  ORC_LENS_PARAB = 11
};

enum { ORC_SHAPE_POINT = 0, ORC_SHAPE_DISK = 1, ORC_SHAPE_RECT = 2, ORC_SHAPE_GAUSS = 3 };
enum { ORC_SPEC_FLAT = 0, ORC_SPEC_KRAMERS = 1, ORC_SPEC_GAUSS = 2 };

/* hc in keV * Angstrom (CODATA 2018): lambda = hc / E */
#define ORC_HC_KEV_A 12.398419843320026

/*
 * One component, already placed in the lab frame: x_lab = o + R x_local.
 * Parameters a[] by type:
 *   SOURCE      a0 radius (disk) or spot width (rect), a1 spot height,
 *               a2 e_min, a3 e_max, a4 e0 (Kramers kVp), a5 target distance,
 *               a6 target width, a7 target height.  Gaussian shape (the
 *               undulator source of Sec. 3.2): a0, a1 the standard deviations
 *               of x and y; a9, a10 those of the divergence, each weighting
 *               the ray by exp(-theta^2 / 2 sigma'^2), theta = (t - s) / a5
 *               (0: no weight).  Gaussian spectrum: E = a4 + a8 z.
 *   SLIT_RECT   a0 xmin, a1 xmax, a2 ymin, a3 ymax
 *   SLIT_CIRC   a0 radius
 *   ABS_BOX     a0 wx, a1 wy, a2 wz (full widths, centred)
 *   ABS_CYL     a0 radius, a1 height (axis = local y, centred)
 *   ABS_SPHERE  a0 radius
 *   PHANTOM     a0 voxel size; a1 steps per voxel edge of the fixed-step
 *               traversal (0: the exact line integral); a4 != 0 (with a1 > 0
 *               and the instrument's scattering coefficients): each step may
 *               also scatter the ray (Rayleigh or Compton; at most 8 times);
 *               n = (nx, ny, nz); centred
 *   MON_PSD     a0..a3 xmin, xmax, ymin, ymax; n = (nx, ny)
 *   MON_E       a0..a3 aperture, a4 e_min, a5 e_max; n0 = ne
 *   MON_L       a0..a3 aperture, a4 l_min, a5 l_max (Angstrom); n0 = nl
 *   MON_EPSD    a0..a3 extent, a4 e_min, a5 e_max; n = (nx, ny, ne)
 *   LENS_PARAB  the compound refractive lens of Sec. 3.2: a stack of a3 = N
 *               double-sided parabolic lenses, centred on the origin, lens j
 *               centred at z_j = (j - (N - 1)/2) a6; its two surfaces
 *               z = z_j -/+ (a1/2 + (x^2 + y^2) / (2 a0)) (a0 radius of
 *               curvature at the apex, a1 apex thickness), aperture radius
 *               a2; refractive index 1 - delta, delta = a4 (a5 / E)^2;
 *               the material between the surfaces attenuates (material).
 */
typedef struct {
  int32_t type, shape, spectrum, material;
  int32_t n[3];
  int32_t pad;
  int64_t mon_offset;   /* first bin of this monitor in the output arrays */
  double o[3];
  double R[9];          /* row-major */
  double a[12];
} orc_comp;

typedef struct {
  int32_t n_comp, n_mat, n_cell, instr_id;
  const orc_comp* comp;
  double e_min, e_max;  /* range of the mu tables */
  const double* coef;   /* [n_mat][n_cell][2]: mu = c0 + c1 * E on each cell */
  const uint8_t* vox;   /* phantom material bytes [nz][ny][nx], x fastest */
  const double* mus;    /* [n_mat][n_cell][2] Rayleigh (elastic) scattering coefficient (1/m),
                           c0 + c1 E on each cell of the mu tables, or NULL */
  const double* muc;    /* the same for Compton scattering, or NULL */
} orc_instrument;

typedef struct {
  int64_t* N;           /* all monitor bins, concatenated by mon_offset */
  double* sw;
  double* sw2;
  double* lost;         /* per component: weight absorbed or attenuated there */
  int64_t n_emit;
  double sum_w0;        /* weight emitted */
  double sum_wend;      /* weight alive after the last component */
} orc_out;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Draw j of ray `id` of instrument `instr` under `seed`:
 * binary64 from 53 bits of block j/2, binary32 from 24 bits of block j/4. */
double orc_uniform64(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j);
float orc_uniform32(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j);

/* Chord length of the half-line x + t k (t >= 0) through a solid centred
 * at the origin. */
double orc_chord_box(const double x[3], const double k[3], const double w[3]);
double orc_chord_cyl(const double x[3], const double k[3], double radius, double height);
double orc_chord_sphere(const double x[3], const double k[3], double radius);

/* Line integral sum_voxels mu[m] * length of the half-line through a
 * centred voxel grid, by Siddon's method (Siddon, Med. Phys. 12, 1985). */
double orc_march_tau(const double x[3], const double k[3], int nx, int ny, int nz,
                     double voxel, double step, const uint8_t* vox, const double* mu_mat);
double orc_siddon_tau(const double x[3], const double k[3], int nx, int ny, int nz,
                      double voxel, const uint8_t* vox, const double* mu_mat);

/* [lo, hi] intersected with {t : |x + t k| <= h}; 0 when empty. */
int orc_clip_slab(double x, double k, double h, double* lo, double* hi);

/* Natural logarithm of a positive normal x from IEEE operations only (the
 * contract's Gaussian draws): x = m 2^e with m in [sqrt(1/2), sqrt(2)],
 * f = (m - 1)/(m + 1), ln m = 2 f (1 + f^2/3 + f^4/5 + ...) by Horner to the
 * f^20 (binary64) or f^10 (binary32) term, ln x = e ln 2 + ln m. */
double orc_ln64(double x);
float orc_ln32(float x);

/* One scattering event from draws j, j+1, ... of a ray's stream (the
 * scattering phantom's sampler, mode 64 or 32): coefficients mr, mc of the
 * voxel's material, direction k and energy *E updated; returns the next draw. */
uint32_t orc_scatter_dir(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j, int mode, double mr,
                         double mc, double k[3], double* E);

/* One ray through a LENS_PARAB component in its local frame (mode 64 or 32
 * arithmetic); x and k are updated, *path receives the length inside the
 * lens material.  Returns 1 if the ray passes, 0 if absorbed. */
int orc_lens_ray(const orc_comp* C, double x[3], double k[3], double E, int mode, double* path);

/* The unit direction of a ray from the source point (in[0], in[1], 0) to the
 * aim point (in[2], in[3], in[4]) in the source frame, computed by the ray
 * loop's own routine in `mode`'s type (32: inputs rounded to binary32). */
void orc_aim_direction(int mode, const double in[5], double k[3]);

/* Table attenuation mu_m(E) with the cell index taken in `mode`'s type. */
double orc_mu(const orc_instrument* ins, int m, double E, int mode);

/* Trace rays [ray_begin, ray_end) and add their contributions to `out`.
 * mode 64: every quantity in binary64.  mode 32: the sampled ray and every
 * quantity that decides a count (clip, bin, cell) in binary32 with the same
 * operation sequence as the mixed-precision GPU path; weights in binary64.
 * Returns 0, or -1 for an invalid instrument. */
int orc_trace(const orc_instrument* ins, uint64_t ray_begin, uint64_t ray_end,
              uint64_t seed, int mode, orc_out* out);

/* Ray starts in mode 32 (binary32): for rays [ray_begin, ray_begin + n) the
 * SoA rows sx, sy, E, u, v, w0 (aim point (u, v), Kramers weight w0) of
 * `starts` (6 n floats). */
int orc_sample_starts(const orc_instrument* ins, uint64_t ray_begin, uint64_t n, uint64_t seed,
                      float* starts);

/* Mode-32 trace of n given ray starts (layout as above).  det (n entries,
 * may be NULL) receives the weight each ray scored at the last component. */
int orc_trace_starts(const orc_instrument* ins, const float* starts, uint64_t n, orc_out* out,
                     double* det);

#ifdef __cplusplus
}
#endif
#endif
