// Nested-dissection multifrontal factorisation of S on the device.
#include "common.cuh"

struct NDFactor {
    int dummy;
};

void spm_factor_free(NDFactor *f) { delete f; }

spm_status spm_factor_impl(spm_problem_s *P, int prec)
{
    (void)P; (void)prec;
    return SPM_OK; // factor not built yet: spm_solve_S reports SPM_ERR_NOT_BUILT
}

spm_status spm_solveS_impl(spm_problem_s *P, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    (void)P; (void)prec; (void)b; (void)x; (void)nrhs; (void)s;
    spm_set_error("sparse factor not available in this build");
    return SPM_ERR_NOT_BUILT;
}
