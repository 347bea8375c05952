/*
 * spm2d.h -- C ABI of the 2-D variant in libspm.
 *
 * Section 2 of the paper (F. Liu and L. Ying, "Sparsifying preconditioner for
 * the time-harmonic Maxwell's equations") notes that the integral equation
 * Eq. (Maxwell_int) holds in 2-D with the 2-D Helmholtz kernel and that the
 * method carries over; Section 4 (Tables 1-3) solves 2-D problems with two
 * unknowns per grid point.  This header is that variant:
 *   G(x) = (i/4) H_0^(1)(k|x|),  G^d = dG/dx_d,  d = 1, 2,
 *   E^d_i + k^2 sum_j G_{i-j} m_j E^d_j + sum_j G^d_{i-j} (p.E)_j = g^d_i,
 *   Toeplitz entries h^2 K(t h) off the diagonal.
 * Conventions are those of spm.h (status codes, precisions, streams, ownership,
 * thread rules) with these changes:
 *   grid Omega = (0,1)^2, n points per dimension, h = 1/(n+1), arrays [i2][i1]
 *   with i1 fastest; a field is [d][i2][i1], d = 0, 1 (E^1, E^2); nrhs fields
 *   stacked outermost, 0 <= nrhs <= 65535.
 * Near-diagonal correction (SPM_QUAD_ORDER4; the paper cites, without giving
 * them, fourth-order weights): a locally corrected trapezoidal rule.  With
 * Z(s) = sum'_{j in Z^2} |j|^{-s} = 4 zeta(s/2) beta(s/2) (Z(0) = -1),
 *   G_0 = h^2 [ i/4 - (ln(k h/2) + gamma_E + Z'(0)) / (2 pi) ],
 *   G^d at t = +-e_d shifted by -+h/(8 pi);
 * SPM_QUAD_ORDER2: G_0 = h^2 [ i/4 - (ln(k/2) + gamma_E) / (2 pi) ], no shift.
 * Point classes (Section 3.2 in 2-D): class = c1 + 3 c2 with c_d = 0 (i_d = 1),
 * 1 (interior), 2 (i_d = n); neighbourhood offsets per dimension {0,1},
 * {-1,0,1}, {-1,0} (T = 4, 6 or 9 points), enumerated o2 outer, o1 inner;
 * enlarged complements [0,n-1], [-(n-2),n-2], [-(n-1),0] per dimension.
 */
#ifndef SPM2D_H
#define SPM2D_H

#include "spm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spm2_problem_s *spm2_problem;

/* Create a 2-D problem on an n x n grid, 4 <= n <= 1024 (any n).  omega = k.
 * eps_host: n^2 complex doubles [i2][i1]; grad_eps_host: 2 n^2 complex doubles
 * [d][i2][i1] (the gradient of eps; required).  The library forms m = 1 - eps,
 * p^d = -d_d eps / eps, the three Toeplitz kernels on a circulant of length L =
 * the smallest power of two >= 2n - 1 per dimension, and their spectra (FP64
 * entries from the Bessel functions of the CUDA math library, FP64 FFTs; kept
 * in complex128 and complex64).  Synchronises `stream`. */
spm_status spm2_create_problem(int n, double omega, const double *eps_host, const double *grad_eps_host,
                               spm_quad quad, void *stream, spm2_problem *out);
spm_status spm2_destroy(spm2_problem prob);

/* n, circulant length L and wavenumber k of a problem (any pointer may be NULL). */
spm_status spm2_problem_info(spm2_problem prob, int *n, int *L, double *k);

/* Z'(0) of the Z^2 lattice zeta used by the ORDER4 correction (host arithmetic). */
double spm2_lattice_zeta_prime(void);

/* The FP64 Toeplitz entries the library computed on the device, copied to
 * out_host: 3 x (2n-1)^2 complex doubles [q][t2 + n - 1][t1 + n - 1], q = G,
 * G^1, G^2.  Synchronises. */
spm_status spm2_kernel_entries(spm2_problem prob, double *out_host);

/* y = A x (Eq. discrete in 2-D) for nrhs fields by three passes: pad, contrast
 * weights [m x^1, m x^2, p.x] and row FFTs; column FFTs, the Fourier-side
 * product with the three spectra and inverse column FFTs; inverse row FFTs,
 * crop and + x.  x_dev, y_dev: nrhs x 2 x n^2 complex in `prec` (SPM_C128 or
 * SPM_C64), not aliased.  Asynchronous on `stream`. */
spm_status spm2_apply_A(spm2_problem prob, spm_prec prec, const void *x_dev, void *y_dev, int nrhs,
                        void *stream);

/* (Q v)_{i,c} = sum_{(d,o) in tau_i} alpha_{class(i)}[(d,o),c] v^d_{i+o}, c = 0, 1
 * (Section 3.1, the rows alpha_i^T).  Needs stencils. */
spm_status spm2_apply_Q(spm2_problem prob, spm_prec prec, const void *v_dev, void *y_dev, int nrhs,
                        void *stream);

/* y = Q A x.  Needs stencils. */
spm_status spm2_apply_QA(spm2_problem prob, spm_prec prec, const void *x_dev, void *y_dev, int nrhs,
                         void *stream);

/* Stencil tables (host memory, complex doubles interleaved):
 *   alpha: [9][18][2], rows (d,o) = d*T + o of the class (rows >= 2T zero),
 *          alpha = conj of the eigenvectors of M M^H for its two smallest
 *          eigenvalues (the two smallest left singular vectors of M), M the
 *          off-neighbourhood block (Section 3.1): rows (d,o), columns (f,u) over
 *          the enlarged complement, entries delta_df k^2 G_{o-u} (f < 2) and
 *          G^d_{o-u} (f = 2);
 *   beta:  [9][27][2], rows (f,o) = f*T + o, beta = B^T alpha (Eq. alphabeta)
 *          with B the same block over the neighbourhood columns;
 *   sv:    [9][18] doubles, the 2T singular values of M, ascending (from the
 *          eigenvalues of M M^H). */
/* Fit the stencils of all nine classes on the device (FP64: Gram matrices
 * M M^H summed over the complement, Jacobi eigen-decomposition), assemble S
 * (Eq. nbr_i_block_alpha_approx with "~" replaced by "=") and factor it in
 * factor_prec (SPM_C128, SPM_C64 or SPM_C64H).  Synchronises. */
spm_status spm2_build_stencils(spm2_problem prob, spm_prec factor_prec);
spm_status spm2_set_stencils(spm2_problem prob, const double *alpha_host, const double *beta_host);
spm_status spm2_get_stencils(spm2_problem prob, double *alpha_host, double *beta_host, double *sv_host);

/* y = S x with the assembled S; S row (i,c), column (f,j), j = i + o, o in tau_i:
 * alpha[(f,o),c] + beta[(f,o),c] m_j + beta[(2,o),c] p^f_j. */
spm_status spm2_apply_S(spm2_problem prob, spm_prec prec, const void *x_dev, void *y_dev, int nrhs,
                        void *stream);

/* Factor S by nested dissection (the multifrontal LU of spm_factor_S on the
 * 2-D grid: separators are grid lines), with the same pivot floor, probe and
 * tree retries; SPM_C128, SPM_C64 or SPM_C64H.  Synchronises. */
spm_status spm2_factor_S(spm2_problem prob, spm_prec prec);
spm_status spm2_factor_info(spm2_problem prob, spm_prec prec, spm_factor_report *out);

/* x = S^{-1} b with the factor of matching precision. */
spm_status spm2_solve_S(spm2_problem prob, spm_prec prec, const void *b_dev, void *x_dev, int nrhs,
                        void *stream);

/* g = E^i - A E^i (the right-hand side of Eq. scattter in 2-D), complex128. */
spm_status spm2_rhs_from_incident(spm2_problem prob, const void *einc_dev, void *g_dev, int nrhs,
                                  void *stream);

/* GMRES(restart) on A x = g left-preconditioned with S^{-1} Q, as spm_solve:
 * FP64 true residual ||g - A x||/||g|| <= tol for every right-hand side;
 * SPM_C128, SPM_C64 or SPM_MIXED; g_dev, x_dev complex128 nrhs x 2 x n^2, x_dev
 * the initial guess.  Synchronises. */
spm_status spm2_solve(spm2_problem prob, spm_prec prec, const void *g_dev, void *x_dev, int nrhs, double tol,
                      int maxit, int restart, spm_solve_info *info);

#ifdef __cplusplus
}
#endif

#endif /* SPM2D_H */
