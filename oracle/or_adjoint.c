/*
 * or_adjoint.c — reverse mode of the oracle's step (test infrastructure only).
 */
#include "or_internal.h"

int or_adjoint(or_ctx *c, const double *I0, const double *ug0, int nsteps, double dt,
               const double *dL_dI_out, const double *dL_dug_out,
               double *dL_dI0, double *dL_dkappa, double *dL_deta) {
    (void)c; (void)I0; (void)ug0; (void)nsteps; (void)dt; (void)dL_dI_out; (void)dL_dug_out;
    (void)dL_dI0; (void)dL_dkappa; (void)dL_deta;
    or_set_err("adjoint not built");
    return -1;
}
