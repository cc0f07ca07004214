// GMRES, preconditioner and Cayley-IRAM entry points.
#include "internal.cuh"

extern "C" stab_status stab_solve(stab_handle h, double, double, const void*, void*, int*) {
  if (h) ((StabHandle*)h)->err = "stab_solve: not built yet";
  return STAB_ERR_UNSUPPORTED;
}
extern "C" stab_status stab_precond_build(stab_handle h, double, double) {
  if (h) ((StabHandle*)h)->err = "not built yet";
  return STAB_ERR_UNSUPPORTED;
}
extern "C" stab_status stab_precond_apply(stab_handle h, const void*, void*) {
  if (h) ((StabHandle*)h)->err = "not built yet";
  return STAB_ERR_UNSUPPORTED;
}
extern "C" stab_status stab_precond_block(stab_handle h, double, double, long long, double*) {
  if (h) ((StabHandle*)h)->err = "not built yet";
  return STAB_ERR_UNSUPPORTED;
}
extern "C" stab_status stab_orthogonalize(stab_handle h, const void*, int, void*, double*, double*) {
  if (h) ((StabHandle*)h)->err = "not built yet";
  return STAB_ERR_UNSUPPORTED;
}
extern "C" stab_status stab_eigs(stab_handle h, double, double, double, double, int, int, double, const void*,
                                 double*, void*, double*, int*, stab_stats*) {
  if (h) ((StabHandle*)h)->err = "not built yet";
  return STAB_ERR_UNSUPPORTED;
}
