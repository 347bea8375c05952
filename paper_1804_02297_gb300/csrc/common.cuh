// Shared device/host helpers of libspm: complex arithmetic on float2/double2,
// error plumbing and the problem handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/spm.h"

// ------------------------------------------------------------ complex types
template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b)
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
// c + a * b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C c)
{
    C r;
    r.x = c.x + a.x * b.x - a.y * b.y;
    r.y = c.y + a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s)
{
    C r;
    r.x = a.x * s;
    r.y = a.y * s;
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C czero()
{
    C r;
    r.x = 0;
    r.y = 0;
    return r;
}
// multiply by -i (forward) or +i (inverse): DIR = -1 -> -i, +1 -> +i
template <int DIR, typename C> __host__ __device__ __forceinline__ C mul_i(C a)
{
    C r;
    if (DIR < 0) { r.x = a.y; r.y = -a.x; }
    else { r.x = -a.y; r.y = a.x; }
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C conj_of(C a)
{
    C r;
    r.x = a.x;
    r.y = -a.y;
    return r;
}
__host__ __device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ------------------------------------------------------------ errors
void spm_set_error(const char *fmt, ...);

#define SPM_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            spm_set_error("%s failed at %s:%d: %s", #expr, __FILE__, __LINE__,                \
                          cudaGetErrorString(_e));                                            \
            return _e == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA;              \
        }                                                                                     \
    } while (0)

#define SPM_TRY(expr)                                                                         \
    do {                                                                                      \
        spm_status _s = (expr);                                                               \
        if (_s != SPM_OK) return _s;                                                          \
    } while (0)

static inline int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// ------------------------------------------------------------ device buffer
// Owned device allocation: freed by release() or when the owner goes out of
// scope (a local work buffer of a call is returned on every exit path).
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    spm_status ensure(size_t want);
    void release();
    template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

// ------------------------------------------------------------ sparse factor
struct NDFactor; // nested-dissection multifrontal factor (sparse.cu)
struct CufftState; // plans and padded arrays of the cuFFT comparison apply (cufft_apply.cu)

// ------------------------------------------------------------ the handle
struct spm_problem_s {
    int n = 0, L = 0, logL = 0;
    double k = 0, h = 0;
    int quad = 0;
    double zconst = 0;
    cudaStream_t stream = nullptr;

    // medium on the grid: m (n^3), p (3 n^3)
    DevBuf m128, p128, m64, p64;
    // kernel spectra, octant [4][n+1]^3 with k^2/L^3 and 1/L^3 folded in
    DevBuf spec128, spec64;
    // twiddles exp(-2 pi i j / L), j < L
    DevBuf tw128, tw64;
    // apply workspace
    DevBuf work;
    DevBuf dev_err; // int: set by a kernel whose bounded wait gave up (SPM_ERR_TIMEOUT)
    int chunk128 = 1, chunk64 = 1; // right-hand sides per pass chunk

    // stencils
    bool have_stencils = false;
    std::vector<double> alpha_h, beta_h, sv_h; // packed host copies (complex interleaved)
    DevBuf alpha128, alpha64, beta128;
    DevBuf qtab128, qtab64; // alpha of every class on all 27 offsets (zeros outside tau): [27][3][27][3]
    std::vector<double> qtab_h; // host copy of the same table (complex interleaved)
    // assembled S (block CSR with 3x3 complex blocks, 27-point pattern)
    bool have_S = false;
    DevBuf S128, S64; // [n^3][27][3][3] complex; absent neighbours hold zeros
    NDFactor *fac128 = nullptr, *fac64 = nullptr;
    struct FactorInfo {
        int variant = -1, attempts = 0, raised_pivots = 0;
        double probe_relres = 0;
        bool half_store = false;
        size_t stored_bytes = 0;
    };
    FactorInfo fac_info[2]; // [0] complex128 factor, [1] complex64 factor

    CufftState *cufft = nullptr; // comparison apply through cuFFT (created on first use)

    // solver workspace
    DevBuf kry;      // A x inside apply_QA
    DevBuf gmres_ws; // GMRES vectors and reductions of spm_solve
};

// ------------------------------------------------------------ sparse system
// What the nested-dissection factor sees: a grid of n1 x n2 x n3 points (point
// index (i3 n2 + i2) n1 + i1), D unknowns per point, couplings between points at
// offsets in {-1,0,1}^3, stored as D x D blocks (row component c, column
// component f, row-major) per point and offset: [point][nsten][D][D] with
// nsten = 27 (offset s = (o1+1) + 3 (o2+1) + 9 (o3+1)) or, for a 2-D grid
// (n3 = 1), nsten = 9 (s = (o1+1) + 3 (o2+1)).  A vector is [b][c][point].
struct SparseSys {
    int dims[3] = {0, 0, 0};
    int D = 3, nsten = 27;
    const void *S128 = nullptr, *S64 = nullptr;
    cudaStream_t stream = nullptr;
    NDFactor **slot128 = nullptr, **slot64 = nullptr;
    spm_problem_s::FactorInfo *info = nullptr; // [0] complex128 factor, [1] complex64 factor
    // y = S x in complex128 for one right-hand side (the factor's probe)
    spm_status (*apply_S128)(void *ctx, const void *x, void *y, cudaStream_t s) = nullptr;
    void *ctx = nullptr;
    long points() const { return (long)dims[0] * dims[1] * dims[2]; }
};
spm_status spm_nd_factor(const SparseSys &S, int prec);
spm_status spm_nd_factor_tree(const SparseSys &S, int prec, int variant);
spm_status spm_nd_solve(NDFactor *F, int prec, const void *b, void *x, int nrhs, cudaStream_t s);

// ------------------------------------------------------------ Krylov operators
// The preconditioned GMRES driver (krylov.cu) sees the problem through these:
// N unknowns per right-hand side, y = A x, y = Q v, x = S^{-1} b in the inner
// precision (SPM_C128 / SPM_C64), and A x in complex128 for the true residual.
struct KrylovOps {
    long N = 0;
    cudaStream_t stream = nullptr;
    DevBuf *ws = nullptr; // GMRES workspace, kept by the problem
    void *ctx = nullptr;
    spm_status (*apply_A)(void *ctx, int prec, const void *x, void *y, int nrhs, cudaStream_t s) = nullptr;
    spm_status (*apply_Q)(void *ctx, int prec, const void *v, void *y, int nrhs, cudaStream_t s) = nullptr;
    spm_status (*solve_S)(void *ctx, int prec, const void *b, void *x, int nrhs, cudaStream_t s) = nullptr;
};
spm_status spm_gmres_solve(const KrylovOps &ops, int prec, const void *g, void *x, int nrhs, double tol, int maxit,
                           int restart, spm_solve_info *info);
spm_status spm_axpby_impl(int prec, long count, double a, const void *x, double b, void *y, cudaStream_t s);

// ------------------------------------------------------------ internal API
spm_status spm_apply_A_impl(spm_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s);
spm_status spm_apply_Q_impl(spm_problem_s *P, int prec, const void *v, void *y, int nrhs, cudaStream_t s);
spm_status spm_apply_plan_impl(int prec, int L, int *get, const int *set);
spm_status spm_profile_apply_impl(spm_problem_s *P, int prec, const void *x, void *y, int with_q, int reps,
                                  float *pass_ms, int *npasses, cudaStream_t s);
spm_status spm_save_plans_impl(const char *path);
spm_status spm_load_plans_impl(const char *path, int *loaded);
spm_status spm_wait_selftest_impl(spm_problem_s *P);
spm_status spm_build_qtable(spm_problem_s *P);
spm_status spm_build_spectra(spm_problem_s *P);
spm_status spm_stencils_device(spm_problem_s *P);
spm_status spm_assemble_S(spm_problem_s *P);
spm_status spm_apply_S_impl(spm_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s);
spm_status spm_factor_impl(spm_problem_s *P, int prec);
spm_status spm_factor_tree_impl(spm_problem_s *P, int prec, int variant);
spm_status spm_solveS_impl(spm_problem_s *P, int prec, const void *b, void *x, int nrhs, cudaStream_t s);
void spm_factor_free(NDFactor *f);
void spm_cufft_free(CufftState *c);
// dense front kernels (dense.cu)
struct DenseWork;
DenseWork *spm_dense_work_new();
void spm_dense_work_free(DenseWork *w);
template <typename C>
spm_status spm_dense_gemm(int m, int n, int k, double alpha, const C *A, long lda, const C *B, long ldb, double beta,
                          C *Cm, long ldc, cudaStream_t s);
template <typename C>
spm_status spm_dense_inverse(int m, C *A, long lda, C *out, long ldo, double tau, int *raised_dev, int *err_dev,
                             DenseWork *W, cudaStream_t s);
spm_status spm_solve_impl(spm_problem_s *P, int prec, const void *g, void *x, int nrhs, double tol,
                          int maxit, int restart, spm_solve_info *info);
