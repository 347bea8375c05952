// Incident fields, BLAS-1 helpers and the preconditioned GMRES driver.
#include <math.h>

#include <complex>
#include <vector>

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


// ====================================================================== GMRES
// Solve A x = g (Eq. discrete_block), left-preconditioned by S^{-1} Q (Section
// 3.1, last paragraph; GMRES with restart 20 as in Section 4).  The outer loop
// is FP64: r = g - A x in complex128, stop when ||r_b||/||g_b|| <= tol for every
// right-hand side b.  Each outer step runs one GMRES(restart) cycle on A d = r
// (preconditioned residual), in complex128 (SPM_C128) or complex64 (SPM_C64,
// SPM_MIXED) with FP64-accumulated dot products and FP64 Givens rotations on the
// host, then x += d in FP64.  Right-hand sides are iterated together: every
// operator and preconditioner application acts on the whole batch.
namespace {

constexpr int DOT_BLOCKS = 304; // 2 x 152 SMs
constexpr int VGROUP = 8;       // basis vectors per dot/axpy pass

// partial[b][blk][i] = sum over this block's k of conj(V_i[b][k]) w[b][k]
template <typename C>
__global__ void k_dots(const C *__restrict__ V, long vstride, int i0, int ni, const C *__restrict__ w, long N,
                       int nrhs, double2 *__restrict__ partial)
{
    __shared__ double2 red[VGROUP][8];
    const int b = blockIdx.y;
    double2 acc[VGROUP];
#pragma unroll
    for (int i = 0; i < VGROUP; ++i) acc[i] = make_double2(0, 0);
    const C *wb = w + (long)b * N;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long)gridDim.x * blockDim.x) {
        C wk = wb[k];
        double wx = wk.x, wy = wk.y;
#pragma unroll
        for (int i = 0; i < VGROUP; ++i) {
            if (i < ni) {
                C v = V[(long)(i0 + i) * vstride + (long)b * N + k];
                acc[i].x += (double)v.x * wx + (double)v.y * wy;
                acc[i].y += (double)v.x * wy - (double)v.y * wx;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < VGROUP; ++i) {
        double x = acc[i].x, y = acc[i].y;
        for (int off = 16; off > 0; off >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, off);
            y += __shfl_down_sync(0xffffffffu, y, off);
        }
        if (lane == 0) red[i][wid] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < ni) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { s.x += red[threadIdx.x][q].x; s.y += red[threadIdx.x][q].y; }
        partial[((long)b * gridDim.x + blockIdx.x) * VGROUP + threadIdx.x] = s;
    }
}

// out[b][i] = sum over blocks of partial[b][blk][i]
__global__ void k_dots_finish(const double2 *__restrict__ partial, int nblk, int ni, int nrhs, double2 *out, int ld,
                              int i0)
{
    int b = blockIdx.x, i = threadIdx.x;
    if (i >= ni) return;
    double2 s = make_double2(0, 0);
    for (int q = 0; q < nblk; ++q) {
        double2 v = partial[((long)b * nblk + q) * VGROUP + i];
        s.x += v.x;
        s.y += v.y;
    }
    out[(long)b * ld + i0 + i] = s;
}

// w[b] -= sum_{i < ni} h[b][i0+i] V_{i0+i}[b]   (coefficients FP64)
template <typename C>
__global__ void k_axpy_multi(const C *__restrict__ V, long vstride, int i0, int ni, const double2 *__restrict__ h,
                             int ld, C *w, long N, int nrhs, double sign)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N * nrhs) return;
    long b = gid / N, k = gid - b * N;
    C wk = w[gid];
    double x = wk.x, y = wk.y;
    for (int i = 0; i < ni; ++i) {
        double2 c = h[b * ld + i0 + i];
        C v = V[(long)(i0 + i) * vstride + gid];
        x += sign * (c.x * v.x - c.y * v.y);
        y += sign * (c.x * v.y + c.y * v.x);
    }
    (void)k;
    wk.x = x;
    wk.y = y;
    w[gid] = wk;
}

// dst[b] = src[b] * scale[b]
template <typename C, typename D>
__global__ void k_scale_copy(D *dst, const C *__restrict__ src, const double *__restrict__ scale, long N, int nrhs)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N * nrhs) return;
    double s = scale[gid / N];
    C v = src[gid];
    D o;
    o.x = s * v.x;
    o.y = s * v.y;
    dst[gid] = o;
}

// x[b] += scale[b] * d[b]   (x complex128)
template <typename C>
__global__ void k_accum(double2 *x, const C *__restrict__ d, const double *__restrict__ scale, long N, int nrhs)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N * nrhs) return;
    double s = scale[gid / N];
    C v = d[gid];
    double2 o = x[gid];
    o.x += s * v.x;
    o.y += s * v.y;
    x[gid] = o;
}

inline unsigned nblocks(long cnt) { return (unsigned)((cnt + 255) / 256); }

template <typename C>
spm_status dots(const C *V, long vstride, int nvec, const C *w, long N, int nrhs, double2 *partial, double2 *out,
                int ld, cudaStream_t s)
{
    for (int i0 = 0; i0 < nvec; i0 += VGROUP) {
        int ni = nvec - i0 < VGROUP ? nvec - i0 : VGROUP;
        k_dots<C><<<dim3(DOT_BLOCKS, nrhs), 256, 0, s>>>(V, vstride, i0, ni, w, N, nrhs, partial);
        k_dots_finish<<<nrhs, VGROUP, 0, s>>>(partial, DOT_BLOCKS, ni, nrhs, out, ld, i0);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

template <typename C>
spm_status axpy_multi(const C *V, long vstride, int nvec, const double2 *h, int ld, C *w, long N, int nrhs,
                      double sign, cudaStream_t s)
{
    for (int i0 = 0; i0 < nvec; i0 += VGROUP) {
        int ni = nvec - i0 < VGROUP ? nvec - i0 : VGROUP;
        k_axpy_multi<C><<<nblocks(N * nrhs), 256, 0, s>>>(V, vstride, i0, ni, h, ld, w, N, nrhs, sign);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

// One preconditioned GMRES(restart) cycle for all right-hand sides, zero initial
// guess: d = argmin over the Krylov space of ||S^{-1} Q (r - A d)||.  Stops
// early when every active RHS reaches relative preconditioned residual rtol[b].
template <typename R>
spm_status gmres_cycle(spm_problem_s *P, int prec, const typename cplx_of<R>::type *r, typename cplx_of<R>::type *d,
                       int nrhs, int restart, const std::vector<double> &rtol, typename cplx_of<R>::type *V,
                       typename cplx_of<R>::type *tmp, double2 *partial, double2 *hdev, double *sdev, int *iters,
                       cudaStream_t s)
{
    using C = typename cplx_of<R>::type;
    typedef std::complex<double> cd;
    const long N = 3L * P->n * P->n * P->n;
    const long vstride = N * nrhs;
    const int ld = restart + 2;
    std::vector<double2> hh((size_t)nrhs * ld);
    std::vector<double> beta(nrhs), scl(nrhs);
    std::vector<std::vector<cd>> H(nrhs, std::vector<cd>((size_t)(restart + 1) * restart));
    std::vector<std::vector<cd>> cs(nrhs, std::vector<cd>(restart)), sn(nrhs, std::vector<cd>(restart));
    std::vector<std::vector<cd>> gv(nrhs, std::vector<cd>(restart + 1));
    std::vector<char> active(nrhs, 1);
    C *w = V + (long)(restart)*vstride; // reuse slot for w until V_{j+1} is formed

    // v0 = S^{-1} Q r / beta
    SPM_TRY(spm_apply_Q_impl(P, prec, r, tmp, nrhs, s));
    SPM_TRY(spm_solveS_impl(P, prec, tmp, V, nrhs, s));
    SPM_TRY(dots<C>(V, vstride, 1, V, N, nrhs, partial, hdev, ld, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(hh.data(), hdev, sizeof(double2) * nrhs * ld, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int b = 0; b < nrhs; ++b) {
        beta[b] = sqrt(fmax(hh[(size_t)b * ld].x, 0.0));
        if (!(beta[b] > 0) || !isfinite(beta[b])) active[b] = 0;
        scl[b] = beta[b] > 0 ? 1.0 / beta[b] : 0.0;
        gv[b][0] = beta[b];
    }
    SPM_CUDA_TRY(cudaMemcpyAsync(sdev, scl.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    k_scale_copy<C, C><<<nblocks(vstride), 256, 0, s>>>(V, V, sdev, N, nrhs);
    int j = 0;
    for (; j < restart; ++j) {
        bool any = false;
        for (int b = 0; b < nrhs; ++b) any |= active[b] != 0;
        if (!any) break;
        C *vj = V + (long)j * vstride;
        w = V + (long)(j + 1) * vstride;
        SPM_TRY(spm_apply_A_impl(P, prec, vj, w, nrhs, s));        // w = A v_j
        SPM_TRY(spm_apply_Q_impl(P, prec, w, tmp, nrhs, s));       // tmp = Q A v_j
        SPM_TRY(spm_solveS_impl(P, prec, tmp, w, nrhs, s));        // w = S^{-1} Q A v_j
        // classical Gram-Schmidt twice
        SPM_TRY(dots<C>(V, vstride, j + 1, w, N, nrhs, partial, hdev, ld, s));
        SPM_TRY(axpy_multi<C>(V, vstride, j + 1, hdev, ld, w, N, nrhs, -1.0, s));
        SPM_CUDA_TRY(cudaMemcpyAsync(hh.data(), hdev, sizeof(double2) * nrhs * ld, cudaMemcpyDeviceToHost, s));
        SPM_TRY(dots<C>(V, vstride, j + 1, w, N, nrhs, partial, hdev, ld, s));
        SPM_TRY(axpy_multi<C>(V, vstride, j + 1, hdev, ld, w, N, nrhs, -1.0, s));
        std::vector<double2> h2((size_t)nrhs * ld);
        SPM_CUDA_TRY(cudaMemcpyAsync(h2.data(), hdev, sizeof(double2) * nrhs * ld, cudaMemcpyDeviceToHost, s));
        // ||w|| after orthogonalisation: dot of w with itself (w sits at slot j+1)
        SPM_TRY(dots<C>(w, vstride, 1, w, N, nrhs, partial, hdev, ld, s));
        std::vector<double2> nn((size_t)nrhs * ld);
        SPM_CUDA_TRY(cudaMemcpyAsync(nn.data(), hdev, sizeof(double2) * nrhs * ld, cudaMemcpyDeviceToHost, s));
        SPM_CUDA_TRY(cudaStreamSynchronize(s));
        ++*iters;
        for (int b = 0; b < nrhs; ++b) {
            std::vector<cd> &Hb = H[b];
            for (int i = 0; i <= j; ++i) {
                double2 a = hh[(size_t)b * ld + i], c2 = h2[(size_t)b * ld + i];
                Hb[(size_t)i * restart + j] = active[b] ? cd(a.x + c2.x, a.y + c2.y) : cd(0, 0);
            }
            double hn = sqrt(fmax(nn[(size_t)b * ld].x, 0.0));
            if (!isfinite(hn)) { spm_set_error("NaN in GMRES"); return SPM_ERR_NUMERICAL; }
            Hb[(size_t)(j + 1) * restart + j] = active[b] ? hn : 0.0;
            scl[b] = (active[b] && hn > 1e-300) ? 1.0 / hn : 0.0;
            if (!active[b]) continue;
            for (int i = 0; i < j; ++i) {
                cd a = Hb[(size_t)i * restart + j], bb = Hb[(size_t)(i + 1) * restart + j];
                Hb[(size_t)i * restart + j] = std::conj(cs[b][i]) * a + std::conj(sn[b][i]) * bb;
                Hb[(size_t)(i + 1) * restart + j] = -sn[b][i] * a + cs[b][i] * bb;
            }
            cd a = Hb[(size_t)j * restart + j], bb = Hb[(size_t)(j + 1) * restart + j];
            double den = sqrt(std::norm(a) + std::norm(bb));
            if (den == 0.0) { cs[b][j] = 1.0; sn[b][j] = 0.0; }
            else { cs[b][j] = a / den; sn[b][j] = bb / den; }
            Hb[(size_t)j * restart + j] = den;
            Hb[(size_t)(j + 1) * restart + j] = 0.0;
            gv[b][j + 1] = -sn[b][j] * gv[b][j];
            gv[b][j] = std::conj(cs[b][j]) * gv[b][j];
            if (std::abs(gv[b][j + 1]) <= rtol[b] * beta[b] || hn <= 1e-300) active[b] = 0;
        }
        SPM_CUDA_TRY(cudaMemcpyAsync(sdev, scl.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        k_scale_copy<C, C><<<nblocks(vstride), 256, 0, s>>>(w, w, sdev, N, nrhs);
    }
    // d = sum_i y_i v_i with H y = g (upper triangular, per RHS)
    const int m = j;
    std::vector<double2> ycoef((size_t)nrhs * ld, make_double2(0, 0));
    for (int b = 0; b < nrhs; ++b) {
        int mb = m;
        // columns beyond the RHS's convergence point are zero rows/cols: solve the leading block
        while (mb > 0 && std::abs(H[b][(size_t)(mb - 1) * restart + (mb - 1)]) == 0.0) --mb;
        std::vector<cd> y(mb);
        for (int i = mb - 1; i >= 0; --i) {
            cd acc = gv[b][i];
            for (int q = i + 1; q < mb; ++q) acc -= H[b][(size_t)i * restart + q] * y[q];
            y[i] = acc / H[b][(size_t)i * restart + i];
        }
        for (int i = 0; i < mb; ++i) ycoef[(size_t)b * ld + i] = make_double2(y[i].real(), y[i].imag());
    }
    SPM_CUDA_TRY(cudaMemcpyAsync(hdev, ycoef.data(), sizeof(double2) * nrhs * ld, cudaMemcpyHostToDevice, s));
    SPM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(C) * vstride, s));
    SPM_TRY(axpy_multi<C>(V, vstride, m, hdev, ld, d, N, nrhs, 1.0, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    return SPM_OK;
}

template <typename C>
spm_status norms(const C *v, long N, int nrhs, double2 *partial, double2 *hdev, int ld, std::vector<double> &out,
                 cudaStream_t s)
{
    SPM_TRY(dots<C>(v, 0, 1, v, N, nrhs, partial, hdev, ld, s));
    std::vector<double2> t((size_t)nrhs * ld);
    SPM_CUDA_TRY(cudaMemcpyAsync(t.data(), hdev, sizeof(double2) * nrhs * ld, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    out.resize(nrhs);
    for (int b = 0; b < nrhs; ++b) out[b] = sqrt(fmax(t[(size_t)b * ld].x, 0.0));
    return SPM_OK;
}

template <typename R>
spm_status solve_typed(spm_problem_s *P, int mode, const double2 *g, double2 *x, int nrhs, double tol, int maxit,
                       int restart, spm_solve_info *info)
{
    using C = typename cplx_of<R>::type;
    const int inner_prec = sizeof(R) == 8 ? SPM_C128 : SPM_C64;
    cudaStream_t s = P->stream;
    const long N = 3L * P->n * P->n * P->n;
    const long vstride = N * nrhs;
    const int ld = restart + 2;
    // workspace: r (c128), Ax (c128), V (restart+1), d, tmp (inner precision), reductions
    size_t bytes = sizeof(double2) * 2 * vstride + sizeof(C) * (size_t)(restart + 3) * vstride +
                   sizeof(double2) * (size_t)nrhs * DOT_BLOCKS * VGROUP + sizeof(double2) * nrhs * ld +
                   sizeof(double) * nrhs + 256 * 8;
    DevBuf &ws = P->gmres_ws; // kept across solves: sized by the largest solve so far
    SPM_TRY(ws.ensure(bytes));
    char *p = ws.as<char>();
    double2 *r = reinterpret_cast<double2 *>(p); p += sizeof(double2) * vstride;
    double2 *Ax = reinterpret_cast<double2 *>(p); p += sizeof(double2) * vstride;
    C *V = reinterpret_cast<C *>(p); p += sizeof(C) * (restart + 1) * vstride;
    C *d = reinterpret_cast<C *>(p); p += sizeof(C) * vstride;
    C *tmp = reinterpret_cast<C *>(p); p += sizeof(C) * vstride;
    double2 *partial = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * DOT_BLOCKS * VGROUP;
    double2 *hdev = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * ld;
    double *sdev = reinterpret_cast<double *>(p);

    std::vector<double> gnorm, rnorm, rtol(nrhs), scl(nrhs);
    SPM_TRY(norms<double2>(g, N, nrhs, partial, hdev, ld, gnorm, s));
    for (int b = 0; b < nrhs; ++b) if (gnorm[b] == 0.0) gnorm[b] = 1.0;
    int iters = 0, outer = 0;
    double worst = 0.0;
    const double floor_rel = sizeof(R) == 8 ? 1e-14 : 2e-6;
    while (true) {
        SPM_TRY(spm_apply_A_impl(P, SPM_C128, x, Ax, nrhs, s));
        SPM_CUDA_TRY(cudaMemcpyAsync(r, g, sizeof(double2) * vstride, cudaMemcpyDeviceToDevice, s));
        SPM_TRY(spm_axpby_impl(SPM_C128, vstride, -1.0, Ax, 1.0, r, s)); // r = g - A x
        SPM_TRY(norms<double2>(r, N, nrhs, partial, hdev, ld, rnorm, s));
        worst = 0.0;
        bool done = true;
        for (int b = 0; b < nrhs; ++b) {
            double rel = rnorm[b] / gnorm[b];
            if (!isfinite(rel)) { spm_set_error("residual is not finite"); return SPM_ERR_NUMERICAL; }
            worst = fmax(worst, rel);
            if (rel > tol) done = false;
            // target for this cycle, relative to ||r_b||, with a safety factor for
            // the gap between preconditioned and true residuals
            rtol[b] = rel > tol ? fmax(0.1 * tol / rel, floor_rel) : 1e300;
            scl[b] = rnorm[b] > 0 ? 1.0 / rnorm[b] : 0.0;
        }
        if (info) { info->true_relres = worst; info->iterations = iters; info->outer_steps = outer; }
        if (done) return SPM_OK;
        if (iters >= maxit) { spm_set_error("no convergence within %d iterations (residual %.3e)", maxit, worst); return SPM_ERR_NO_CONVERGENCE; }
        // inner right-hand side: r / ||r|| in the inner precision
        SPM_CUDA_TRY(cudaMemcpyAsync(sdev, scl.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        k_scale_copy<double2, C><<<nblocks(vstride), 256, 0, s>>>(tmp, r, sdev, N, nrhs);
        C *rin = d; // d is free until the cycle writes its result
        SPM_CUDA_TRY(cudaMemcpyAsync(rin, tmp, sizeof(C) * vstride, cudaMemcpyDeviceToDevice, s));
        int it_cycle = 0;
        int cyc_restart = restart < maxit - iters ? restart : maxit - iters;
        SPM_TRY(gmres_cycle<R>(P, inner_prec, rin, d, nrhs, cyc_restart, rtol, V, tmp, partial, hdev, sdev, &it_cycle, s));
        iters += it_cycle;
        ++outer;
        for (int b = 0; b < nrhs; ++b) scl[b] = rtol[b] < 1e299 ? rnorm[b] : 0.0;
        SPM_CUDA_TRY(cudaMemcpyAsync(sdev, scl.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        k_accum<C><<<nblocks(vstride), 256, 0, s>>>(x, d, sdev, N, nrhs);
        SPM_CUDA_TRY(cudaGetLastError());
    }
}

} // namespace

spm_status spm_solve_impl(spm_problem_s *P, int prec, const void *g, void *x, int nrhs, double tol, int maxit,
                          int restart, spm_solve_info *info)
{
    if (!P->have_S) { spm_set_error("stencils not built (spm_build_stencils)"); return SPM_ERR_NOT_BUILT; }
    const bool inner64 = prec != SPM_C128;
    if ((inner64 && !P->fac64) || (!inner64 && !P->fac128)) {
        spm_set_error("no factor of S in the %s precision (spm_factor_S)", inner64 ? "complex64" : "complex128");
        return SPM_ERR_NOT_BUILT;
    }
    spm_status st = inner64 ? solve_typed<float>(P, prec, (const double2 *)g, (double2 *)x, nrhs, tol, maxit, restart, info)
                            : solve_typed<double>(P, prec, (const double2 *)g, (double2 *)x, nrhs, tol, maxit, restart, info);
    SPM_CUDA_TRY(cudaStreamSynchronize(P->stream));
    return st;
}
