/*
 * orc_trace.c -- the CPU oracle's ray loop (see orc_core.inc) instantiated for
 * the two decision types, plus the table lookup used by the tests.
 * TEST INFRASTRUCTURE ONLY (see orc.h).  Compile with -ffp-contract=off.
 */
#include "orc.h"

#include <math.h>
#include <stddef.h>

#define REAL double
#define SFX(name) name##_d
#define UNI(id, instr, seed, j) orc_uniform64((id), (instr), (seed), (j))
#define SQRTR(x) sqrt(x)
#define LNR(x) orc_ln64(x)
#include "orc_core.inc"
#undef REAL
#undef SFX
#undef UNI
#undef SQRTR
#undef LNR

#define REAL float
#define SFX(name) name##_f
#define UNI(id, instr, seed, j) orc_uniform32((id), (instr), (seed), (j))
#define SQRTR(x) sqrtf(x)
#define LNR(x) orc_ln32(x)
#include "orc_core.inc"
#undef REAL
#undef SFX
#undef UNI
#undef SQRTR
#undef LNR

void orc_aim_direction(int mode, const double in[5], double k[3])
{
  if (mode == 32) {
    float kf[3];
    aim_direction_f((float)in[0], (float)in[1], (float)in[2], (float)in[3], (float)in[4], kf);
    for (int i = 0; i < 3; i++) k[i] = (double)kf[i];
  } else {
    aim_direction_d(in[0], in[1], in[2], in[3], in[4], k);
  }
}

double orc_mu(const orc_instrument* ins, int m, double E, int mode)
{
  return mode == 32 ? mu_table_f(ins, m, (float)E) : mu_table_d(ins, m, E);
}

static int valid(const orc_instrument* ins)
{
  if (!ins || ins->n_comp < 1 || !ins->comp || ins->comp[0].type != ORC_SOURCE) return 0;
  for (int c = 1; c < ins->n_comp; c++) {
    int t = ins->comp[c].type;
    if (t <= ORC_SOURCE || t > ORC_LENS_PARAB) return 0;
    if ((t == ORC_ABS_BOX || t == ORC_ABS_CYL || t == ORC_ABS_SPHERE || t == ORC_LENS_PARAB) &&
        (!ins->coef || ins->comp[c].material < 0 || ins->comp[c].material >= ins->n_mat))
      return 0;
    if (t == ORC_PHANTOM && (!ins->vox || !ins->coef)) return 0;
  }
  if (ins->comp[0].spectrum == ORC_SPEC_KRAMERS &&
      !(ins->comp[0].a[2] > 0.0 && ins->comp[0].a[4] >= ins->comp[0].a[3]))
    return 0;
  return 1;
}

int orc_trace(const orc_instrument* ins, uint64_t ray_begin, uint64_t ray_end,
              uint64_t seed, int mode, orc_out* out)
{
  if (!valid(ins) || (mode != 64 && mode != 32) || ray_end < ray_begin) return -1;
  /* mean of the Kramers shape f(E) = (e0 - E)/E over [e_min, e_max]:
   * (e0 ln(e_max/e_min) - (e_max - e_min)) / (e_max - e_min) */
  const orc_comp* S = &ins->comp[0];
  double fbar = 1.0;
  if (S->spectrum == ORC_SPEC_KRAMERS) {
    const double lo = S->a[2], hi = S->a[3], e0 = S->a[4];
    fbar = (e0 * log(hi / lo) - (hi - lo)) / (hi - lo);
  }
  for (uint64_t id = ray_begin; id < ray_end; id++) {
    if (mode == 64) trace_ray_d(ins, id, seed, fbar, out);
    else trace_ray_f(ins, id, seed, fbar, out);
  }
  return 0;
}

static double kramers_mean(const orc_instrument* ins)
{
  const orc_comp* S = &ins->comp[0];
  if (S->spectrum != ORC_SPEC_KRAMERS) return 1.0;
  const double lo = S->a[2], hi = S->a[3], e0 = S->a[4];
  return (e0 * log(hi / lo) - (hi - lo)) / (hi - lo);
}

int orc_sample_starts(const orc_instrument* ins, uint64_t ray_begin, uint64_t n, uint64_t seed,
                      float* starts)
{
  if (!valid(ins) || !starts) return -1;
  const double fbar = kramers_mean(ins);
  for (uint64_t i = 0; i < n; i++) {
    float sx, sy, tx, ty, E;
    sample_start_f(ins, ray_begin + i, seed, &sx, &sy, &tx, &ty, &E);
    starts[i] = sx;
    starts[n + i] = sy;
    starts[2 * n + i] = E;
    starts[3 * n + i] = tx;
    starts[4 * n + i] = ty;
    starts[5 * n + i] = (float)start_weight_f(ins, sx, sy, tx, ty, E, fbar);
  }
  return 0;
}

int orc_trace_starts(const orc_instrument* ins, const float* starts, uint64_t n, orc_out* out,
                     double* det)
{
  if (!valid(ins) || !starts) return -1;
  /* scattering draws continue the ray's own stream, which given starts do
     not carry */
  for (int c = 1; c < ins->n_comp; c++)
    if (ins->comp[c].type == ORC_PHANTOM && ins->comp[c].a[4] != 0.0 && ins->mus) return -1;
  for (uint64_t i = 0; i < n; i++) {
    double d = 0.0;
    if (starts[5 * n + i] == 0.0f) {
      out->n_emit += 1;   /* a zero-weight start is emitted but not traced */
    } else {
      trace_from_f(ins, starts[i], starts[n + i], starts[3 * n + i], starts[4 * n + i],
                   starts[2 * n + i], (double)starts[5 * n + i], out, &d, 0, 0, NULL);
    }
    if (det) det[i] = d;
  }
  return 0;
}

int orc_lens_ray(const orc_comp* C, double x[3], double k[3], double E, int mode, double* path)
{
  if (!C || C->type != ORC_LENS_PARAB || !path) return -1;
  int ok;
  if (mode == 64) {
    ok = lens_stack_d(C, x, k, E, path);
  } else {
    float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    float kf[3] = {(float)k[0], (float)k[1], (float)k[2]};
    ok = lens_stack_f(C, xf, kf, (float)E, path);
    for (int i = 0; i < 3; i++) { x[i] = xf[i]; k[i] = kf[i]; }
  }
  return ok;
}

uint32_t orc_scatter_dir(uint64_t id, uint32_t instr, uint64_t seed, uint32_t j, int mode, double mr,
                         double mc, double k[3], double* E)
{
  if (mode == 64) {
    scatter_dir_d(id, instr, seed, &j, mr, mc, k, E);
  } else {
    float kf[3] = {(float)k[0], (float)k[1], (float)k[2]};
    float Ef = (float)*E;
    scatter_dir_f(id, instr, seed, &j, (float)mr, (float)mc, kf, &Ef);
    for (int i = 0; i < 3; i++) k[i] = kf[i];
    *E = Ef;
  }
  return j;
}
