/*
 * spm.h -- C ABI of libspm, a GB300 (sm_103a) implementation of the hot path of
 * the sparsifying preconditioner for the 3-D time-harmonic Maxwell volume
 * integral equation (F. Liu and L. Ying, "Sparsifying preconditioner for the
 * time-harmonic Maxwell's equations").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid (Section 2): Omega = (0,1)^3, n points per dimension, h = 1/(n+1), node
 *   i = (i1,i2,i3), 1 <= i_d <= n, at x = i*h.  Grid arrays are [i3][i2][i1]
 *   with i1 fastest.
 * Fields: a vector field is [d][i3][i2][i1], d = 0,1,2 (the paper's E^1,E^2,E^3);
 *   nrhs fields are stacked outermost: [b][d][i3][i2][i1], 0 <= nrhs <= 65535
 *   (SPM_ERR_INVALID_ARG otherwise).  Complex numbers are
 *   interleaved (re, im).  SPM_C128 buffers hold double pairs, SPM_C64 buffers
 *   float pairs.
 * Memory: arguments named *_host are host pointers, *_dev device pointers.  The
 *   caller owns every buffer it passes; the library owns everything inside an
 *   spm_problem (spectra, stencils, sparse factor, workspaces) until
 *   spm_destroy.  Input and output buffers of one call must not alias.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Device
 *   work is enqueued on it and the call returns without synchronising, except
 *   where stated (set-up calls and spm_solve synchronise).
 * Errors: every function returns spm_status (0 = SPM_OK) and never throws or
 *   aborts; spm_last_error() gives a thread-local message for the last failure.
 *   A handle must not be used from two host threads at once.
 */
#ifndef SPM_H
#define SPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spm_problem_s *spm_problem;

typedef enum {
    SPM_OK = 0,
    SPM_ERR_INVALID_ARG = 1,    /* bad size, pointer or enum value */
    SPM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SPM_ERR_OOM = 3,            /* device allocation failed */
    SPM_ERR_NOT_BUILT = 4,      /* stencils or factor requested before they exist */
    SPM_ERR_NO_CONVERGENCE = 5, /* solver hit maxit; x holds the last iterate */
    SPM_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
    SPM_ERR_NUMERICAL = 7       /* zero pivot, NaN or Inf */
} spm_status;

/* Quadrature for the Toeplitz entries near the diagonal (Section 2, the
 * "fourth-order quadrature correction" after Eq. discrete).  ORDER4: corrected
 * trapezoidal rule, G_0 = h^2 (i k h - Z)/(4 pi) and G^d at t = +-e_d shifted by
 * +-h Z/(24 pi), Z = sum'_{j in Z^3} |j|^{-1} (continued) = -2.8372974794806...
 * ORDER2: punctured trapezoidal rule, G_0 = h^3 i k/(4 pi), no other change. */
typedef enum { SPM_QUAD_ORDER4 = 0, SPM_QUAD_ORDER2 = 1 } spm_quad;

/* Arithmetic of a call: complex128, complex64 (FP32 accumulation), or, for
 * spm_solve only, complex64 inner iterations inside an FP64 outer loop.
 * SPM_C64H (spm_factor_S / spm_build_stencils only): the factor of S is
 * computed in complex64 and its stored blocks are kept as binary16 pairs
 * scaled per column by the column's largest component (half the memory and
 * half the bytes each S^{-1} reads); it serves complex64 solves. */
typedef enum { SPM_C128 = 0, SPM_C64 = 1, SPM_MIXED = 2, SPM_C64H = 3 } spm_prec;

/* ---------------------------------------------------------------- set-up */

/* Create a problem on an n^3 grid (Section 2).  omega is the normalised
 * frequency; with eps0 = mu0 = 1 the wavenumber is k = omega.
 * eps_host: n^3 complex doubles, the relative permittivity eps + i sigma/omega
 *   at the nodes; eps - 1 must vanish smoothly at the boundary of Omega (the
 *   contrast m = 1 - eps is compactly supported, Section 2).
 * grad_eps_host: 3 n^3 complex doubles [d][i3][i2][i1], the gradient of eps, or
 *   NULL to use fourth-order central differences with eps = 1 outside the grid.
 * The library forms m = 1 - eps and p^d = (d_d m)/(1 - m) = -d_d eps/eps
 * (Section 2, definitions before Eq. discrete), the four Toeplitz kernels
 * G, G^1, G^2, G^3 and their spectra on a 2n-periodic grid (circulant embedding;
 * FP64, stored in complex128 and complex64).  n must be in [4, 256] and a
 * power of two, or 48 or 96 (FFT lengths 2n: powers of two up to 512, 96, 192).
 * Synchronises `stream`.  On success *out is a new handle. */
spm_status spm_create_problem(int n, double omega, const double *eps_host,
                              const double *grad_eps_host, spm_quad quad,
                              void *stream, spm_problem *out);

/* Release every device and host resource of the handle. NULL is accepted. */
spm_status spm_destroy(spm_problem prob);

/* Grid size n, wavenumber k and unknown count 3 n^3 of a handle. */
spm_status spm_problem_info(spm_problem prob, int *n, double *k, long long *unknowns);

/* ---------------------------------------------------------- operator A */

/* y = A x, A = I + [k^2 G, G^d] [m; p] (Eq. discrete_block), for nrhs fields.
 * x_dev, y_dev: nrhs x 3 x n^3 complex in `prec` (SPM_C128 or SPM_C64).
 * Evaluated matrix-free by zero-padded FFT convolution with the four kernel
 * spectra (Section 2: the convolutions "can be evaluated efficiently by the
 * FFT").  Uses library-owned workspace sized for the largest nrhs seen. */
spm_status spm_apply_A(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev,
                       int nrhs, void *stream);

/* y = A x exactly as spm_apply_A, but the call allocates no device memory.
 * The paper has no counterpart: this serves callers that cannot allocate when
 * they apply the operator (device memory owned by another allocator or budget,
 * or loops that cannot afford cudaMalloc/cudaFree blocking or synchronising the
 * device).  The pass intermediates live in one fixed 64 MiB device array inside
 * the library (every GPU that loads the library holds it until the process
 * exits); right-hand sides are processed one at a time, so the limit is
 * 24 n^3 complex values per call: n <= 64 in SPM_C64 and n <= 48 in SPM_C128
 * (n = 64 in SPM_C128 needs 96 MiB).  Larger problems return
 * SPM_ERR_INVALID_ARG before any device work.  Every call looks up the array's
 * device address on the current device (cudaGetSymbolAddress, which allocates
 * nothing), so the call stays valid across a device reset; make the first call
 * on a device before any stream capture, since that lookup may initialise the
 * library's module on the device.  All calls share the array: calls whose work
 * overlaps on the GPU (different streams, or different handles at once) race on
 * it and give wrong results.  The problem handle itself is created (and
 * allocated) by spm_create_problem. */
spm_status spm_apply_A_noalloc(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev,
                               int nrhs, void *stream);

/* y = A x exactly as spm_apply_A, computed the textbook way through cuFFT:
 * the four contrast-weighted fields zero-padded to full (2n)^3 arrays, one
 * batched 3-D cuFFT forward transform, the Fourier-side product with the four
 * kernel spectra, one batched inverse transform, crop and + x.  A comparison
 * point for the hand-written passes of spm_apply_A (the paper has no such
 * path; it states only that the convolutions are evaluated by FFT), not used
 * by any other entry point.  The padded arrays (4 (2n)^3 complex values) and
 * the cuFFT plans are allocated on first use and kept by the problem until
 * spm_destroy; right-hand sides are processed one at a time. */
spm_status spm_apply_A_cufft(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev,
                             int nrhs, void *stream);

/* y = Q A x: A as above followed by the sparsifying row combination Q,
 * (Q v)_{i,c} = sum_{(d,o) in tau(class i)} alpha_class[(d,o),c] v^d_{i+o}
 * (Eq. nbr_i_block_alpha; classes of Section 3.2).  Needs stencils
 * (spm_build_stencils or spm_set_stencils), else SPM_ERR_NOT_BUILT. */
spm_status spm_apply_QA(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev,
                        int nrhs, void *stream);

/* y = A x (spm_apply_A_host) or y = Q A x (spm_apply_QA_host) for nrhs fields
 * held in HOST memory (x_host, y_host: nrhs x 3 x n^3 complex in `prec`, the
 * layout of the device calls).  Each field is copied to the device, applied on
 * `stream`, and copied back; the copies of one field overlap the apply of the
 * previous one (two device slots, host-to-device and device-to-host copies on two
 * library streams), so page-locked host memory lets the transfers hide behind the
 * applies (pageable memory works but serialises the copies).  Same arithmetic as
 * the device calls.  Synchronises `stream`: y_host is complete on return.
 * Device scratch of four fields is allocated for the call and freed on return. */
spm_status spm_apply_A_host(spm_problem prob, spm_prec prec, const void *x_host, void *y_host, int nrhs,
                            void *stream);
spm_status spm_apply_QA_host(spm_problem prob, spm_prec prec, const void *x_host, void *y_host, int nrhs,
                             void *stream);

/* y = Q v (the row combination alone), same layout and requirements. */
spm_status spm_apply_Q(spm_problem prob, spm_prec prec, const void *v_dev, void *y_dev,
                       int nrhs, void *stream);

/* ----------------------------------------------------------- stencils */

/* Point classes (Section 3.2): class = c1 + 3 c2 + 9 c3 with c_d = 0 if i_d = 1,
 * 2 if i_d = n, else 1.  The neighbourhood offsets o of a class are, per
 * dimension, {0,1}, {-1,0,1} or {-1,0}; T = |tau| is 27, 18, 12 or 8; offsets
 * are enumerated o3 outer, o2, o1 inner, each ascending.  Stencil tables are
 * packed for all 27 classes:
 *   alpha: [27][81][3] complex double, row (d,o) = d*T + o (rows >= 3T unused),
 *          alpha = conj(the three left singular vectors of M with the smallest
 *          singular values), M the off-neighbourhood block (Section 3.1,
 *          the minimisation of ||alpha^T M||_F with alpha^T alpha = I);
 *   beta:  [27][108][3] complex double, row (f,o) = f*T + o, beta = B^T alpha
 *          with B the in-neighbourhood block (Eq. alphabeta);
 *   sv:    [27][81] double, the 3T singular values of M, ascending.          */

/* Compute alpha, beta for all classes on the device (FP64), assemble the
 * sparse matrix S (Eq. nbr_i_block_alpha_approx with "~" replaced by "="),
 * and factor it by nested dissection in `factor_prec` (SPM_C128 or SPM_C64).
 * Synchronises the problem's creation stream. */
spm_status spm_build_stencils(spm_problem prob, spm_prec factor_prec);

/* Install caller-computed stencil tables (layout above, host memory), then
 * assemble S.  The factor is dropped; spm_factor_S builds it again. */
spm_status spm_set_stencils(spm_problem prob, const double *alpha_host, const double *beta_host);

/* Copy the current stencil tables to host memory; any pointer may be NULL. */
spm_status spm_get_stencils(spm_problem prob, double *alpha_host, double *beta_host, double *sv_host);

/* Factor the assembled S (nested dissection, multifrontal LU on the device) in
 * `prec` (SPM_C128, SPM_C64 or SPM_C64H).  Each front's fully summed block is
 * inverted by the library's own Gauss-Jordan elimination with partial
 * pivoting, and the Schur-complement products are the library's own complex
 * GEMMs (no vendor dense library).  Pivoting stays inside each front, so a box
 * of the dissection whose part of S is nearly singular spoils the factor even
 * when S itself is well conditioned.  Two safeguards: pivots of a front below
 * 1e-8 (SPM_C128) or 1e-4 (complex64) times the largest entry of its fully
 * summed block are raised to that size (the factor is then exact for S plus a
 * perturbation of that rank); and the factor is probed:
 * x = S^{-1} b for a fixed pseudo-random b, and the residual ||S x - b|| / ||b||
 * (S x in complex128) must be at most 1e-6 (SPM_C128), 3e-2 (SPM_C64) or 0.3
 * (SPM_C64H); otherwise up to three other trees (cut planes moved by one) are
 * factored and the most accurate factor is kept.  Synchronises.  SPM_ERR_TIMEOUT
 * if a bounded wait between the blocks of the elimination kernel gave up. */
spm_status spm_factor_S(spm_problem prob, spm_prec prec);

/* Factor S on one tree variant (0 = cuts through the middle planes; 1, 2, 3 =
 * every cut moved one plane down, up, or alternately by depth), without the
 * retry; the probe residual is still recorded for spm_factor_info.
 * SPM_ERR_INVALID_ARG for a variant outside [0, 4). */
spm_status spm_factor_S_tree(spm_problem prob, spm_prec prec, int variant);

/* Report on the current factor in `prec` (SPM_C128, or SPM_C64 / SPM_C64H for
 * the complex64 slot): tree variant kept (0 = middle cuts), factorisations run
 * by the last spm_factor_S, whether blocks are in half storage, the number of
 * raised pivots, and the probe residual described above.  SPM_ERR_NOT_BUILT if there is no such factor. */
typedef struct {
    int variant;
    int attempts;
    int half_store;
    int raised_pivots;      /* pivots raised by the static perturbation in the kept factor */
    double probe_relres;
    long long stored_bytes; /* bytes of the stored blocks; each S^{-1} reads them once */
} spm_factor_report;
spm_status spm_factor_info(spm_problem prob, spm_prec prec, spm_factor_report *out);

/* y = S x for nrhs fields (sparse product with the assembled S). */
spm_status spm_apply_S(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev,
                       int nrhs, void *stream);

/* x = S^{-1} b with the factor of matching precision (forward and backward
 * substitution through the elimination tree). */
spm_status spm_solve_S(spm_problem prob, spm_prec prec, const void *b_dev, void *x_dev,
                       int nrhs, void *stream);

/* Apply plan (process-wide, per FFT length L = 2n or the radix-3 lengths 96
 * and 192, and per apply precision SPM_C128 / SPM_C64): the z-pass kernel.
 *   0  four lines per thread block with all fields in registers (lengths other
 *      than 96 and 192),
 *   1  one field at a time after a cp.async prefetch of all four (L >= 32, 96, 192),
 *   2  persistent, fed by TMA bulk-tensor copies into two shared-memory stages
 *      (L >= 32),
 *   3  16 values per thread (one shared-memory exchange per line at L = 128
 *      and 256), twiddles in registers, all four fields prefetched by cp.async
 *      (L = 128, 256, 512),
 *   4  as 1, with the tile's kernel spectra and the twiddle table also staged
 *      in shared memory by cp.async (L >= 32),
 *   5  each length-2n transform split into two length-n transforms of the
 *      even and odd frequencies, which share their exchanges (L = 64, 128,
 *      256),
 *  -1  not chosen yet: the next apply of that length times the candidates on
 *      its own data (outside stream capture) and keeps the fastest.
 * Plus 8 (L = 64, 128 only): the x- and y-passes of each z-plane run fused in
 * one kernel per direction (the plane's n x L intermediate stays in shared
 * memory); the timing tries it with the fastest z-pass kernel.
 * SPM_ERR_INVALID_ARG for an unknown length or a variant the length lacks. */
spm_status spm_get_apply_plan(spm_prec prec, int L, int *zvariant);
spm_status spm_set_apply_plan(spm_prec prec, int L, int zvariant);

/* Device time of every pass of one apply of A (with_q = 0) or Q A (with_q = 1)
 * to one right-hand side (x_dev, y_dev as in spm_apply_A), averaged over reps
 * applies, in launch order: x-forward, y-forward, z-pass, y-inverse, x-inverse
 * (or, with the plan's fused plane passes: xy-forward, z-pass, yx-inverse),
 * then Q.  An event is recorded after every pass, so the passes run
 * serialised and their sum exceeds the pipelined time of spm_apply_A.
 * pass_ms: at least 7 floats; *npasses receives the count.  The paper has no
 * counterpart (measurement only).  Synchronises `stream`. */
spm_status spm_profile_apply(spm_problem prob, spm_prec prec, const void *x_dev, void *y_dev, int with_q,
                             int reps, float *pass_ms, int *npasses, void *stream);

/* The autotuner's choices persisted as JSON: {"device": name, "plans": [{"prec":
 * "c64" | "c128", "L": length, "variant": v, "ms": [per-apply ms of variants
 * 0..5 when they were timed, else 0], "fused_xy_ms": ms of the best variant with
 * fused x and y passes, else 0}, ...]} for every (precision, length) whose
 * variant is set.  spm_load_apply_plans installs the entries of a file written
 * on a device of the same name (SPM_ERR_INVALID_ARG for another device or an
 * unreadable file); *loaded (may be NULL) receives the number installed.  The
 * first spm_create_problem of a process loads the file named by the
 * environment variable SPM_APPLY_PLANS, if set (a file for another device is
 * ignored).  The paper has no counterpart: this only fixes which of the
 * equivalent kernels runs. */
spm_status spm_save_apply_plans(const char *path);
spm_status spm_load_apply_plans(const char *path, int *loaded);

/* Synchronise the device and report whether any kernel of this problem gave up
 * a bounded wait since the last call (SPM_ERR_TIMEOUT, then cleared): the
 * TMA-fed z-pass waits on its copies with an iteration limit instead of
 * spinning forever, and leaves its output incomplete when the limit is hit. */
spm_status spm_device_status(spm_problem prob);

/* Self-test of that failure path: launches (on the problem's stream) one block
 * that waits, with the same bound, on an mbarrier no copy will complete, and
 * records the expired wait like the z-pass does; the next spm_device_status
 * then returns SPM_ERR_TIMEOUT.  Takes about as long as one bounded wait. */
spm_status spm_selftest_bounded_wait(spm_problem prob);

/* ------------------------------------------------------------- solving */

typedef struct {
    int iterations;         /* preconditioned GMRES iterations of the batch (all RHS advance together) */
    int outer_steps;        /* FP64 outer steps: one GMRES(restart) cycle each */
    double true_relres;     /* max over RHS of ||g - A x|| / ||g|| in FP64 at exit */
    double solve_ms;        /* wall time of the call */
} spm_solve_info;

/* Incident plane waves E^i = pol_b exp(i k dir_b . x) (Section 4), nrhs of them.
 * dir_host, pol_host: nrhs x 3 doubles.  e_dev: nrhs x 3 x n^3 in `prec`. */
spm_status spm_incident_plane_wave(spm_problem prob, spm_prec prec, const double *dir_host,
                                   const double *pol_host, int nrhs, void *e_dev, void *stream);

/* Right-hand side of Eq. (scattter): g = E^i - A E^i (since
 * (A - I) E^i = k^2 G*(m E^i) + grad G*(p.E^i) = -g).  complex128 buffers. */
spm_status spm_rhs_from_incident(spm_problem prob, const void *einc_dev, void *g_dev, int nrhs,
                                 void *stream);

/* Solve A x = g (Eq. discrete_block) for nrhs right-hand sides by GMRES(restart)
 * left-preconditioned with S^{-1} Q (Section 3.1, last paragraph), stopping
 * when every FP64 true relative residual ||g - A x||/||g|| <= tol.
 * prec: SPM_C128 (everything FP64), SPM_C64 or SPM_MIXED (complex64 operator
 * and factor inside FP64 iterative refinement with FP64 residuals).
 * g_dev, x_dev: complex128, nrhs x 3 x n^3; x_dev is the initial guess on entry.
 * restart <= 0 selects 20 (Section 4).  Returns SPM_ERR_NO_CONVERGENCE with the
 * last iterate in x_dev if maxit inner iterations per RHS are exceeded.
 * The GMRES vectors ((restart + 3) x nrhs fields in the inner precision, plus
 * two FP64 fields per RHS) live in a problem-owned buffer that grows to the
 * largest solve and is freed by spm_destroy.  Synchronises. */
spm_status spm_solve(spm_problem prob, spm_prec prec, const void *g_dev, void *x_dev, int nrhs,
                     double tol, int maxit, int restart, spm_solve_info *info);

/* ------------------------------------------------------------- batches */

/* A batch of independent problems of uneven size: problem i has grid n[i],
 * frequency omega[i] and its own medium (eps_host[i], grad_eps_host[i] or a
 * NULL array / NULL entry for finite differences), all as in
 * spm_create_problem.  Each problem gets its own stream, workspaces, stencils
 * and factor; they share nothing, so the batch is embarrassingly parallel.
 * Synchronises.  *out is a new batch handle. */
typedef struct spm_batch_s *spm_batch;
spm_status spm_create_batch(int count, const int *n, const double *omega, const double *const *eps_host,
                            const double *const *grad_eps_host, spm_quad quad, spm_batch *out);
spm_status spm_destroy_batch(spm_batch batch);
spm_status spm_batch_size(spm_batch batch, int *count);
/* Borrowed handle of problem `index` (owned by the batch: do not destroy it). */
spm_status spm_batch_problem(spm_batch batch, int index, spm_problem *out);
/* spm_build_stencils on every problem, concurrently. */
spm_status spm_batch_build_stencils(spm_batch batch, spm_prec factor_prec);
/* y_dev[i] = A_i x_dev[i] (one right-hand side per problem) for every problem,
 * ordered on `stream`.  The problems run as parallel branches; the first call
 * with a given set of buffers also captures the fork/join into a CUDA graph
 * that later calls with the same buffers and precision replay. */
spm_status spm_batch_apply_A(spm_batch batch, spm_prec prec, const void *const *x_dev, void *const *y_dev,
                             void *stream);
/* spm_solve on every problem (one right-hand side each), concurrently from a
 * pool of host threads; infos (count entries) may be NULL.  Returns the first
 * failing status.  Synchronises. */
spm_status spm_batch_solve(spm_batch batch, spm_prec prec, const void *const *g_dev, void *const *x_dev,
                           double tol, int maxit, int restart, spm_solve_info *infos);

/* -------------------------------------------------------- inspection */

/* The library's Toeplitz entries for offsets t in [-(n-1), n-1]^3,
 * out_host: 4 x (2n-1)^3 complex doubles [kern][t3][t2][t1], kern = G,G^1,G^2,G^3
 * (Section 2).  Evaluated on the device in FP64. */
spm_status spm_kernel_entries(spm_problem prob, double *out_host);

/* The lattice constant Z used by SPM_QUAD_ORDER4 (computed by Ewald summation). */
double spm_lattice_constant(void);

/* -------------------------------------------------------- measurement */

/* Measured arithmetic peak of the current device in TFLOP/s (the paper has no
 * counterpart: this gives the denominators of the ALU roofline the applies are
 * reported against).  kind 0: FP32 fused multiply-add (FFMA), kind 1: packed
 * FP32x2 multiply-add (two per instruction), kind 2: FP64 fused multiply-add.
 * Each runs independent register FMA chains on every SM (2048 threads per SM)
 * for a few milliseconds and reports the best of five timed launches; *ms_out
 * (may be NULL) receives that launch's time.  Allocates a small output buffer
 * and a private stream, synchronises the device's work on that stream only.
 * SPM_ERR_INVALID_ARG for another kind or a NULL tflops. */
spm_status spm_measure_peak(int kind, double *tflops, double *ms_out);

/* Thread-local message of the last failing call ("" if none). */
const char *spm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SPM_H */
