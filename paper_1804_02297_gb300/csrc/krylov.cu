// Incident fields, BLAS-1 helpers and the preconditioned GMRES driver.
#include "common.cuh"

namespace {

template <typename C>
__global__ void k_plane_wave(C *e, const double *__restrict__ dp, int n, double h, double k, long total)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long n3 = (long)n * n * n;
    long b = gid / n3, i = gid - b * n3;
    int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
    const double *d = dp + b * 6, *pol = d + 3;
    double phase = k * h * (d[0] * (i1 + 1) + d[1] * (i2 + 1) + d[2] * (i3 + 1));
    double sn, cs;
    sincos(phase, &sn, &cs);
    for (int c = 0; c < 3; ++c) {
        C v;
        v.x = pol[c] * cs;
        v.y = pol[c] * sn;
        e[(b * 3 + c) * n3 + i] = v;
    }
}

template <typename C>
__global__ void k_axpby(long count, double a, const C *__restrict__ x, double b, C *y)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= count) return;
    C xv = x[gid], yv = y[gid];
    yv.x = a * xv.x + b * yv.x;
    yv.y = a * xv.y + b * yv.y;
    y[gid] = yv;
}

} // namespace

spm_status spm_plane_wave_impl(spm_problem_s *P, int prec, const double *dir, const double *pol, int nrhs, void *e,
                               cudaStream_t s)
{
    std::vector<double> dp(6 * nrhs);
    for (int b = 0; b < nrhs; ++b)
        for (int c = 0; c < 3; ++c) { dp[6 * b + c] = dir[3 * b + c]; dp[6 * b + 3 + c] = pol[3 * b + c]; }
    DevBuf t;
    SPM_TRY(t.ensure(sizeof(double) * dp.size()));
    SPM_CUDA_TRY(cudaMemcpyAsync(t.ptr, dp.data(), sizeof(double) * dp.size(), cudaMemcpyHostToDevice, s));
    const long total = (long)nrhs * P->n * P->n * P->n;
    unsigned grid = (unsigned)((total + 255) / 256);
    if (prec == SPM_C128)
        k_plane_wave<double2><<<grid, 256, 0, s>>>((double2 *)e, t.as<double>(), P->n, P->h, P->k, total);
    else
        k_plane_wave<float2><<<grid, 256, 0, s>>>((float2 *)e, t.as<double>(), P->n, P->h, P->k, total);
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    t.release();
    return SPM_OK;
}

spm_status spm_axpby_impl(int prec, long count, double a, const void *x, double b, void *y, cudaStream_t s)
{
    unsigned grid = (unsigned)((count + 255) / 256);
    if (prec == SPM_C128)
        k_axpby<double2><<<grid, 256, 0, s>>>(count, a, (const double2 *)x, b, (double2 *)y);
    else
        k_axpby<float2><<<grid, 256, 0, s>>>(count, a, (const float2 *)x, b, (float2 *)y);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

spm_status spm_solve_impl(spm_problem_s *P, int prec, const void *g, void *x, int nrhs, double tol, int maxit,
                          int restart, spm_solve_info *info)
{
    (void)P; (void)prec; (void)g; (void)x; (void)nrhs; (void)tol; (void)maxit; (void)restart; (void)info;
    spm_set_error("solver not available in this build");
    return SPM_ERR_NOT_BUILT;
}
