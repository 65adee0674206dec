// Solver-side entry points: implicit apply (eq. 11), PCPG (Algorithm 1),
// recovery (eqs. 5, 8) and the adjoint.
#include "context.h"
#include "kernels.h"

using namespace feti;

extern "C" {

feti_status feti_apply_implicit(feti_ctx* ctx, const double*, double*) {
  return set_error(ctx, FETI_ERR_STATE, "feti_apply_implicit: not available in this build");
}

feti_status feti_solve(feti_ctx* ctx, double*, double*, double*, feti_solve_info*) {
  return set_error(ctx, FETI_ERR_STATE, "feti_solve: not available in this build");
}

feti_status feti_adjoint(feti_ctx* ctx, const double*, double*) {
  return set_error(ctx, FETI_ERR_STATE, "feti_adjoint: not available in this build");
}

}  // extern "C"
