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
#include "orc_core.inc"
#undef REAL
#undef SFX
#undef UNI
#undef SQRTR

#define REAL float
#define SFX(name) name##_f
#define UNI(id, instr, seed, j) orc_uniform32((id), (instr), (seed), (j))
#define SQRTR(x) sqrtf(x)
#include "orc_core.inc"
#undef REAL
#undef SFX
#undef UNI
#undef SQRTR

double orc_mu(const orc_instrument* ins, int m, double E, int mode)
{
  return mode == 32 ? mu_table_f(ins, m, (float)E) : mu_table_d(ins, m, E);
}

static int valid(const orc_instrument* ins)
{
  if (!ins || ins->n_comp < 1 || !ins->comp || ins->comp[0].type != ORC_SOURCE) return 0;
  for (int c = 1; c < ins->n_comp; c++) {
    int t = ins->comp[c].type;
    if (t <= ORC_SOURCE || t > ORC_MON_EPSD) return 0;
    if ((t == ORC_ABS_BOX || t == ORC_ABS_CYL || t == ORC_ABS_SPHERE) &&
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
