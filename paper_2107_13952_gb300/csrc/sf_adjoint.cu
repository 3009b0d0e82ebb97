// Boundary-contracted amplitude and adjoint; mixed-precision shell sum.
#include "sf_internal.cuh"

struct sf_tables;
int sf_adjoint_run(sf_tables* t, const double* const psi[5], double* a_out, double* const grad_psi[5],
                   double* const grad_B[4], cudaStream_t s) {
    (void)t; (void)psi; (void)a_out; (void)grad_psi; (void)grad_B; (void)s;
    return sf_set_error(SF_ERR_ARG, "sf_vertex_adjoint is not available in this build");
}

int sf_shell_mixed_launch(const VtxDev* d_v, int mdi, int mdk, const WorkItem* d_items, int n_items,
                          int* d_counter, double* d_part, ShellFilter filt, int num_sms, cudaStream_t s) {
    (void)d_v; (void)mdi; (void)mdk; (void)d_items; (void)n_items; (void)d_counter; (void)d_part; (void)filt;
    (void)num_sms; (void)s;
    return sf_set_error(SF_ERR_ARG, "the mixed-precision path is not available in this build");
}
