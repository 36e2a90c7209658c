// Mixed precision and adjoint entry points (filled in below as they are built).
#include "krylov.cuh"

namespace omss {
om_status solve_mixed(const om_matrix *, const om_ilu *, const int32_t *, const om_solve_opts *, const double *,
                      double *, om_solve_info *, void *) {
    set_error("precision = 1 is not available in this build");
    return OM_EINVAL;
}
}  // namespace omss

extern "C" om_status om_steady_state_adjoint(const om_matrix *, const om_ilu *, const int32_t *, const om_solve_opts *,
                                             const om_params *, const double *, const double *, double *,
                                             om_solve_info *, void *) {
    omss::set_error("the adjoint is not available in this build");
    return OM_EINVAL;
}
