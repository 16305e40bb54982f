// solve.cu -- iterative interpolation solve (placeholder until GMRES lands).
#include "rbf_internal.cuh"

extern "C" int rbf_interp_solve(rbf_tree *t, rbf_kernel kernel, double eps,
                                const rbf_fmm_params *params, const double *u, double *lambda,
                                int nrhs, const rbf_solve_opts *opts, rbf_solve_report *rep,
                                void *stream)
{
    (void)t; (void)kernel; (void)eps; (void)params; (void)u; (void)lambda; (void)nrhs;
    (void)opts; (void)rep; (void)stream;
    rbf_set_error("rbf_interp_solve: not built yet");
    return RBF_ENOTSUP;
}
