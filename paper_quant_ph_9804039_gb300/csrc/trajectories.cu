// Error trajectories (filled in by the batched kernel).
#include "qsim_internal.h"

using namespace qs;

extern "C" int qsim_run_trajectories(int M, const qsim_gate *ideal, const double *err_axis, size_t n,
                                     const double *eps, int T, const qsim_traj_opts *opts, double *F_out,
                                     double *mean, double *var) {
    (void)M; (void)ideal; (void)err_axis; (void)n; (void)eps; (void)T; (void)opts;
    (void)F_out; (void)mean; (void)var;
    set_error("error trajectories are not available in this build");
    return QSIM_EUNSUPPORTED;
}
