/*
 * orc_geom.c -- chord lengths and the voxel line integral of the CPU oracle.
 * TEST INFRASTRUCTURE ONLY (see orc.h).  Plain binary64.
 *
 * Beer-Lambert attenuation (the absorption the paper's sample components
 * model, Sec. 3.3) needs the length L of the ray's half-line inside a solid:
 * the weight becomes p * exp(-mu(E) L).  For a voxel phantom the exponent is
 * the line integral sum_voxels mu_m(E) * l_voxel, computed here with
 * Siddon's method: collect the parameters where the line crosses every grid
 * plane, sort them, and charge each segment to the voxel containing its
 * midpoint (R. L. Siddon, Med. Phys. 12 (1985) 252).  The GPU path uses a
 * different traversal (incremental 3D-DDA), so agreement is a real check.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* Intersect [*lo, *hi] with the parameter interval where |x + t k| <= h on
 * one axis.  Returns 0 when the interval becomes empty. */
static int clip_slab(double x, double k, double h, double* lo, double* hi)
{
  if (k != 0.0) {
    double t1 = (-h - x) / k;
    double t2 = (h - x) / k;
    *lo = dmax(*lo, dmin(t1, t2));
    *hi = dmin(*hi, dmax(t1, t2));
  } else if (x < -h || x > h) {
    return 0;
  }
  return *hi > *lo;
}

double orc_chord_box(const double x[3], const double k[3], const double w[3])
{
  double lo = 0.0, hi = INFINITY;
  for (int i = 0; i < 3; i++)
    if (!clip_slab(x[i], k[i], 0.5 * w[i], &lo, &hi)) return 0.0;
  return hi - lo;
}

/* Roots of a t^2 + 2 b t + c = 0 in the cancellation-free form
 * q = -(b + sign(b) sqrt(b^2 - a c)), t = q / a and t = c / q. */
static int quad_roots(double a, double b, double c, double* t1, double* t2)
{
  double disc = b * b - a * c;
  if (!(disc > 0.0)) return 0;
  double sq = sqrt(disc);
  double q = (b >= 0.0) ? -(b + sq) : -(b - sq);
  double r1 = q / a, r2 = c / q;
  *t1 = dmin(r1, r2);
  *t2 = dmax(r1, r2);
  return 1;
}

double orc_chord_cyl(const double x[3], const double k[3], double radius, double height)
{
  double lo = 0.0, hi = INFINITY;
  double a = k[0] * k[0] + k[2] * k[2];
  double c = x[0] * x[0] + x[2] * x[2] - radius * radius;
  if (a > 0.0) {
    double t1, t2;
    double b = x[0] * k[0] + x[2] * k[2];
    if (!quad_roots(a, b, c, &t1, &t2)) return 0.0;
    lo = dmax(lo, t1);
    hi = dmin(hi, t2);
  } else if (c > 0.0) {
    return 0.0;
  }
  if (!clip_slab(x[1], k[1], 0.5 * height, &lo, &hi)) return 0.0;
  return hi > lo ? hi - lo : 0.0;
}

double orc_chord_sphere(const double x[3], const double k[3], double radius)
{
  double a = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  double b = x[0] * k[0] + x[1] * k[1] + x[2] * k[2];
  double c = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] - radius * radius;
  double t1, t2;
  if (!(a > 0.0) || !quad_roots(a, b, c, &t1, &t2)) return 0.0;
  double lo = dmax(0.0, t1), hi = t2;
  return hi > lo ? hi - lo : 0.0;
}

static int cmp_double(const void* pa, const void* pb)
{
  double a = *(const double*)pa, b = *(const double*)pb;
  return (a > b) - (a < b);
}

static int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

double orc_siddon_tau(const double x[3], const double k[3], int nx, int ny, int nz,
                      double voxel, const uint8_t* vox, const double* mu_mat)
{
  const int n[3] = {nx, ny, nz};
  double h[3];
  for (int i = 0; i < 3; i++) h[i] = 0.5 * (double)n[i] * voxel;

  /* entry and exit parameters of the half-line through the grid's box */
  double a_in = 0.0, a_out = INFINITY;
  for (int i = 0; i < 3; i++)
    if (!clip_slab(x[i], k[i], h[i], &a_in, &a_out)) return 0.0;

  /* all plane crossings strictly inside (a_in, a_out), plus the two ends */
  size_t cap = (size_t)nx + (size_t)ny + (size_t)nz + 8;
  double* al = (double*)malloc(cap * sizeof(double));
  if (!al) return NAN;
  size_t na = 0;
  al[na++] = a_in;
  al[na++] = a_out;
  for (int i = 0; i < 3; i++) {
    if (k[i] == 0.0) continue;
    for (int m = 0; m <= n[i]; m++) {
      double plane = -h[i] + (double)m * voxel;
      double a = (plane - x[i]) / k[i];
      if (a > a_in && a < a_out) al[na++] = a;
    }
  }
  qsort(al, na, sizeof(double), cmp_double);

  double tau = 0.0;
  for (size_t s = 0; s + 1 < na; s++) {
    double len = al[s + 1] - al[s];
    if (!(len > 0.0)) continue;
    double mid = 0.5 * (al[s] + al[s + 1]);
    int idx[3];
    for (int i = 0; i < 3; i++)
      idx[i] = clampi((int)floor((x[i] + mid * k[i] + h[i]) / voxel), n[i]);
    size_t lin = ((size_t)idx[2] * (size_t)ny + (size_t)idx[1]) * (size_t)nx + (size_t)idx[0];
    tau += mu_mat[vox[lin]] * len;
  }
  free(al);
  return tau;
}

int orc_clip_slab(double x, double k, double h, double* lo, double* hi)
{
  return clip_slab(x, k, h, lo, hi);
}

/* The paper's fixed-step traversal of a voxel phantom (Sec. 3.3): from the
   grid entry, steps of `step` along the line; a step's material is that of
   the voxel holding the step's end point (clamped to the grid), and the last
   step ends at the grid exit.  Positions are 32.32 fixed-point voxel
   coordinates: the entry point and the step are rounded to that lattice once
   (binary64, round to nearest even), and every step is an exact integer
   addition, so any implementation of this rule samples the same voxels. */
double orc_march_tau(const double x[3], const double k[3], int nx, int ny, int nz,
                     double voxel, double step, const uint8_t* vox, const double* mu_mat)
{
  const int n[3] = {nx, ny, nz};
  double h[3];
  for (int i = 0; i < 3; i++) h[i] = 0.5 * (double)n[i] * voxel;
  double a_in = 0.0, a_out = INFINITY;
  for (int i = 0; i < 3; i++)
    if (!clip_slab(x[i], k[i], h[i], &a_in, &a_out)) return 0.0;
  const double L = a_out - a_in;
  const double inv = 1.0 / voxel, scale = 4294967296.0;   /* 2^32 */
  int64_t P[3], D[3];
  for (int i = 0; i < 3; i++) {
    P[i] = llrint(((x[i] + a_in * k[i]) + h[i]) * inv * scale);
    D[i] = llrint((step * k[i]) * inv * scale);
  }
  const int64_t steps = (int64_t)ceil(L / step);
  double tau = 0.0;
  for (int64_t s = 1; s <= steps; s++) {
    int idx[3];
    for (int i = 0; i < 3; i++) {
      P[i] += D[i];
      const int64_t v = P[i] >> 32;   /* floor: arithmetic shift */
      idx[i] = v < 0 ? 0 : (v >= n[i] ? n[i] - 1 : (int)v);
    }
    const double len = s < steps ? step : L - (double)(steps - 1) * step;
    const size_t lin = ((size_t)idx[2] * (size_t)ny + (size_t)idx[1]) * (size_t)nx + (size_t)idx[0];
    tau += mu_mat[vox[lin]] * len;
  }
  return tau;
}
