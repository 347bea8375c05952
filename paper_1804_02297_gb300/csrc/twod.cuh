// The 2-D variant (Section 2: the same integral equation with the 2-D Helmholtz
// kernel; Section 4, Tables 1-3: two unknowns per grid point): the problem
// handle and the internal entry points shared by twod.cu and the factor.
#pragma once
#include "common.cuh"
#include "../../include/spm2d.h"

struct spm2_problem_s {
    int n = 0, L = 0;          // grid n x n, FFT length L = power of two >= 2n - 1
    double k = 0, h = 0;
    int quad = 0;
    double zprime = 0;         // Z'(0) of the Z^2 lattice zeta
    cudaStream_t stream = nullptr;

    DevBuf m128, p128, m64, p64; // m [n^2], p [2][n^2]
    DevBuf spec128, spec64;      // quadrant spectra [3][L/2+1][L/2+1], k^2/L^2 and 1/L^2 folded in
    DevBuf tw128, tw64;          // exp(-2 pi i j/L), j < L
    DevBuf work;                 // apply workspace [chunk][3][n][L]
    DevBuf entries;              // FP64 Toeplitz entries [3][2n-1][2n-1] (stencil fit)
    DevBuf dev_err;

    bool have_stencils = false;
    std::vector<double> alpha_h, beta_h, sv_h; // (9,18,2), (9,27,2) complex; (9,18) real
    DevBuf qtab128, qtab64;      // alpha on all 9 offsets, zeros outside tau: [9 cls][2 c][9 s][2 d]
    bool have_S = false;
    DevBuf S128, S64;            // [n^2][9][2][2]: row component c, column component f

    NDFactor *fac128 = nullptr, *fac64 = nullptr;
    spm_problem_s::FactorInfo fac_info[2];

    DevBuf kry, gmres_ws;
};

spm_status spm2_apply_A_impl(spm2_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s);
spm_status spm2_apply_Q_impl(spm2_problem_s *P, int prec, const void *v, void *y, int nrhs, cudaStream_t s);
spm_status spm2_apply_S_impl(spm2_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s);
