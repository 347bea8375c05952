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

// ---- the small FP64 problem of GMRES on the device, one thread per RHS ----
// Per right-hand side b the cycle keeps, in device memory: the Hessenberg
// matrix H[b] ((restart + 1) x restart, row i column j at i * restart + j), the
// Givens rotations cs[b][i], sn[b][i], the rotated residual vector g[b][i], beta
// = ||v_0||, and whether b is still active.
struct GmresSmall {
    double2 *H, *cs, *sn, *g;
    double *beta, *rtol, *scale;
    int *active, *count; // count[0]: RHS still active; count[1]: non-finite values seen
};

// after v_0 = S^-1 Q r: beta = ||v_0|| (nn[b*ld] holds <v_0, v_0>), g = beta e_1
__global__ void k_cycle_init(GmresSmall gs, const double2 *__restrict__ nn, int ld, int restart, int nrhs)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrhs) return;
    const double beta = sqrt(fmax(nn[(long)b * ld].x, 0.0));
    const bool ok = beta > 0 && isfinite(beta);
    gs.beta[b] = beta;
    gs.active[b] = ok ? 1 : 0;
    gs.scale[b] = ok ? 1.0 / beta : 0.0;
    for (int i = 0; i <= restart; ++i) gs.g[(long)b * (restart + 1) + i] = make_double2(i == 0 ? beta : 0.0, 0.0);
    for (long i = 0; i < (long)(restart + 1) * restart; ++i) gs.H[(long)b * (restart + 1) * restart + i] = make_double2(0, 0);
    if (ok) atomicAdd(&gs.count[0], 1);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Arnoldi step j: column j of H from the two Gram-Schmidt passes (h1, h2) and
// ||w|| (nn), the previous rotations applied, a new rotation that zeroes
// H[j+1][j], g rotated; scale = 1/||w|| for normalising v_{j+1}; a RHS whose
// |g[j+1]| <= rtol beta (or whose ||w|| vanished) becomes inactive.
__global__ void k_arnoldi_givens(GmresSmall gs, const double2 *__restrict__ h1, const double2 *__restrict__ h2,
                                 const double2 *__restrict__ nn, int ld, int j, int restart, int nrhs)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrhs) return;
    if (!gs.active[b]) { gs.scale[b] = 0.0; return; }
    double2 *H = gs.H + (long)b * (restart + 1) * restart;
    double2 *cs = gs.cs + (long)b * restart, *sn = gs.sn + (long)b * restart, *g = gs.g + (long)b * (restart + 1);
    for (int i = 0; i <= j; ++i) H[i * restart + j] = zadd(h1[(long)b * ld + i], h2[(long)b * ld + i]);
    const double hn = sqrt(fmax(nn[(long)b * ld].x, 0.0));
    if (!isfinite(hn)) { atomicAdd(&gs.count[1], 1); gs.active[b] = 0; gs.scale[b] = 0.0; return; }
    H[(j + 1) * restart + j] = make_double2(hn, 0.0);
    gs.scale[b] = hn > 1e-300 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
        const double2 a = H[i * restart + j], c = H[(i + 1) * restart + j];
        H[i * restart + j] = zadd(zmul(zconj(cs[i]), a), zmul(zconj(sn[i]), c));
        const double2 ms = make_double2(-sn[i].x, -sn[i].y);
        H[(i + 1) * restart + j] = zadd(zmul(ms, a), zmul(cs[i], c));
    }
    const double2 a = H[j * restart + j], c = H[(j + 1) * restart + j];
    const double den = sqrt(a.x * a.x + a.y * a.y + c.x * c.x + c.y * c.y);
    if (den == 0.0) { cs[j] = make_double2(1.0, 0.0); sn[j] = make_double2(0.0, 0.0); }
    else { cs[j] = make_double2(a.x / den, a.y / den); sn[j] = make_double2(c.x / den, c.y / den); }
    H[j * restart + j] = make_double2(den, 0.0);
    H[(j + 1) * restart + j] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    const double2 ms = make_double2(-sn[j].x, -sn[j].y);
    g[j + 1] = zmul(ms, gj);
    g[j] = zmul(zconj(cs[j]), gj);
    const double r = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y);
    if (r <= gs.rtol[b] * gs.beta[b] || hn <= 1e-300) gs.active[b] = 0;
    else atomicAdd(&gs.count[0], 1);
}

// back substitution H y = g over the leading m columns (fewer where a RHS
// stopped early: its trailing diagonal entries are zero); y -> coef[b*ld + i]
__global__ void k_backsolve(GmresSmall gs, double2 *coef, int ld, int m, int restart, int nrhs)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrhs) return;
    const double2 *H = gs.H + (long)b * (restart + 1) * restart, *g = gs.g + (long)b * (restart + 1);
    double2 *y = coef + (long)b * ld;
    int mb = m;
    while (mb > 0 && H[(mb - 1) * restart + (mb - 1)].x == 0.0 && H[(mb - 1) * restart + (mb - 1)].y == 0.0) --mb;
    for (int i = 0; i < ld; ++i) y[i] = make_double2(0, 0);
    for (int i = mb - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < mb; ++q) {
            const double2 t = zmul(H[i * restart + q], y[q]);
            acc.x -= t.x;
            acc.y -= t.y;
        }
        const double2 d = H[i * restart + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

// One preconditioned GMRES(restart) cycle for all right-hand sides, zero initial
// guess: d = argmin over the Krylov space of ||S^{-1} Q (r - A d)||.  Stops
// early when every active RHS reaches relative preconditioned residual rtol[b].
template <typename R>
spm_status gmres_cycle(const KrylovOps &ops, int prec, const typename cplx_of<R>::type *r,
                       typename cplx_of<R>::type *d, int nrhs, int restart, typename cplx_of<R>::type *V,
                       typename cplx_of<R>::type *tmp, double2 *partial, double2 *h1, double2 *h2, double2 *nn,
                       const GmresSmall &gs, int *count_host, int *iters, cudaStream_t s)
{
    using C = typename cplx_of<R>::type;
    const long N = ops.N;
    const long vstride = N * nrhs;
    const int ld = restart + 2;
    const unsigned sb = (unsigned)((nrhs + 63) / 64);
    C *w = V + (long)(restart)*vstride;

    // v0 = S^{-1} Q r / beta
    SPM_TRY(ops.apply_Q(ops.ctx, prec, r, tmp, nrhs, s));
    SPM_TRY(ops.solve_S(ops.ctx, prec, tmp, V, nrhs, s));
    SPM_TRY(dots<C>(V, vstride, 1, V, N, nrhs, partial, nn, ld, s));
    SPM_CUDA_TRY(cudaMemsetAsync(gs.count, 0, 2 * sizeof(int), s));
    k_cycle_init<<<sb, 64, 0, s>>>(gs, nn, ld, restart, nrhs);
    k_scale_copy<C, C><<<nblocks(vstride), 256, 0, s>>>(V, V, gs.scale, N, nrhs);
    SPM_CUDA_TRY(cudaMemcpyAsync(count_host, gs.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    int j = 0;
    for (; j < restart && count_host[0] > 0; ++j) {
        C *vj = V + (long)j * vstride;
        w = V + (long)(j + 1) * vstride;
        SPM_TRY(ops.apply_A(ops.ctx, prec, vj, w, nrhs, s));       // w = A v_j
        SPM_TRY(ops.apply_Q(ops.ctx, prec, w, tmp, nrhs, s));      // tmp = Q A v_j
        SPM_TRY(ops.solve_S(ops.ctx, prec, tmp, w, nrhs, s));      // w = S^{-1} Q A v_j
        // classical Gram-Schmidt twice, FP64 coefficients
        SPM_TRY(dots<C>(V, vstride, j + 1, w, N, nrhs, partial, h1, ld, s));
        SPM_TRY(axpy_multi<C>(V, vstride, j + 1, h1, ld, w, N, nrhs, -1.0, s));
        SPM_TRY(dots<C>(V, vstride, j + 1, w, N, nrhs, partial, h2, ld, s));
        SPM_TRY(axpy_multi<C>(V, vstride, j + 1, h2, ld, w, N, nrhs, -1.0, s));
        SPM_TRY(dots<C>(w, vstride, 1, w, N, nrhs, partial, nn, ld, s)); // ||w||^2 (w sits at slot j+1)
        SPM_CUDA_TRY(cudaMemsetAsync(gs.count, 0, sizeof(int), s));
        k_arnoldi_givens<<<sb, 64, 0, s>>>(gs, h1, h2, nn, ld, j, restart, nrhs);
        k_scale_copy<C, C><<<nblocks(vstride), 256, 0, s>>>(w, w, gs.scale, N, nrhs);
        SPM_CUDA_TRY(cudaMemcpyAsync(count_host, gs.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPM_CUDA_TRY(cudaStreamSynchronize(s)); // the only host round trip of an iteration: a convergence count
        ++*iters;
        if (count_host[1]) { spm_set_error("NaN in GMRES"); return SPM_ERR_NUMERICAL; }
    }
    // d = sum_i y_i v_i with H y = g (upper triangular, per RHS, on the device)
    const int m = j;
    k_backsolve<<<sb, 64, 0, s>>>(gs, h1, ld, m, restart, nrhs);
    SPM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(C) * vstride, s));
    SPM_TRY(axpy_multi<C>(V, vstride, m, h1, ld, d, N, nrhs, 1.0, s));
    SPM_CUDA_TRY(cudaGetLastError());
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
spm_status solve_typed(const KrylovOps &ops, const double2 *g, double2 *x, int nrhs, double tol, int maxit,
                       int restart, spm_solve_info *info)
{
    using C = typename cplx_of<R>::type;
    const int inner_prec = sizeof(R) == 8 ? SPM_C128 : SPM_C64;
    cudaStream_t s = ops.stream;
    const long N = ops.N;
    const long vstride = N * nrhs;
    const int ld = restart + 2;
    // workspace: r (c128), Ax (c128), V (restart+1), d, tmp (inner precision), reductions
    const size_t small = sizeof(double2) * (size_t)nrhs * (3 * ld + (restart + 1) * restart + 2 * restart + restart + 1) +
                         sizeof(double) * 3 * (size_t)nrhs + sizeof(int) * ((size_t)nrhs + 2);
    size_t bytes = sizeof(double2) * 2 * vstride + sizeof(C) * (size_t)(restart + 3) * vstride +
                   sizeof(double2) * (size_t)nrhs * DOT_BLOCKS * VGROUP + small + 16 * 256;
    DevBuf &ws = *ops.ws; // kept across solves: sized by the largest solve so far
    SPM_TRY(ws.ensure(bytes));
    char *p = ws.as<char>();
    double2 *r = reinterpret_cast<double2 *>(p); p += sizeof(double2) * vstride;
    double2 *Ax = reinterpret_cast<double2 *>(p); p += sizeof(double2) * vstride;
    C *V = reinterpret_cast<C *>(p); p += sizeof(C) * (restart + 1) * vstride;
    C *d = reinterpret_cast<C *>(p); p += sizeof(C) * vstride;
    C *tmp = reinterpret_cast<C *>(p); p += sizeof(C) * vstride;
    double2 *partial = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * DOT_BLOCKS * VGROUP;
    double2 *hdev = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * ld;
    double2 *h2dev = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * ld;
    double2 *nndev = reinterpret_cast<double2 *>(p); p += sizeof(double2) * nrhs * ld;
    GmresSmall gs;
    gs.H = reinterpret_cast<double2 *>(p); p += sizeof(double2) * (size_t)nrhs * (restart + 1) * restart;
    gs.cs = reinterpret_cast<double2 *>(p); p += sizeof(double2) * (size_t)nrhs * restart;
    gs.sn = reinterpret_cast<double2 *>(p); p += sizeof(double2) * (size_t)nrhs * restart;
    gs.g = reinterpret_cast<double2 *>(p); p += sizeof(double2) * (size_t)nrhs * (restart + 1);
    gs.beta = reinterpret_cast<double *>(p); p += sizeof(double) * nrhs;
    gs.rtol = reinterpret_cast<double *>(p); p += sizeof(double) * nrhs;
    double *sdev = reinterpret_cast<double *>(p); p += sizeof(double) * nrhs;
    gs.scale = sdev;
    gs.active = reinterpret_cast<int *>(p); p += sizeof(int) * nrhs;
    gs.count = reinterpret_cast<int *>(p);
    int count_host[2] = {0, 0};

    std::vector<double> gnorm, rnorm, rtol(nrhs), scl(nrhs);
    SPM_TRY(norms<double2>(g, N, nrhs, partial, hdev, ld, gnorm, s));
    for (int b = 0; b < nrhs; ++b) if (gnorm[b] == 0.0) gnorm[b] = 1.0;
    int iters = 0, outer = 0;
    double worst = 0.0;
    const double floor_rel = sizeof(R) == 8 ? 1e-14 : 2e-6;
    while (true) {
        SPM_TRY(ops.apply_A(ops.ctx, SPM_C128, x, Ax, nrhs, s));
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
        SPM_CUDA_TRY(cudaMemcpyAsync(gs.rtol, rtol.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        SPM_TRY(gmres_cycle<R>(ops, inner_prec, rin, d, nrhs, cyc_restart, V, tmp, partial, hdev, h2dev, nndev, gs,
                               count_host, &it_cycle, s));
        iters += it_cycle;
        ++outer;
        for (int b = 0; b < nrhs; ++b) scl[b] = rtol[b] < 1e299 ? rnorm[b] : 0.0;
        SPM_CUDA_TRY(cudaMemcpyAsync(sdev, scl.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        k_accum<C><<<nblocks(vstride), 256, 0, s>>>(x, d, sdev, N, nrhs);
        SPM_CUDA_TRY(cudaGetLastError());
    }
}

} // namespace

spm_status spm_gmres_solve(const KrylovOps &ops, int prec, const void *g, void *x, int nrhs, double tol, int maxit,
                           int restart, spm_solve_info *info)
{
    const bool inner64 = prec != SPM_C128;
    spm_status st = inner64 ? solve_typed<float>(ops, (const double2 *)g, (double2 *)x, nrhs, tol, maxit, restart, info)
                            : solve_typed<double>(ops, (const double2 *)g, (double2 *)x, nrhs, tol, maxit, restart, info);
    SPM_CUDA_TRY(cudaStreamSynchronize(ops.stream));
    return st;
}

namespace {
spm_status ops3_A(void *c, int prec, const void *x, void *y, int nrhs, cudaStream_t s)
{
    return spm_apply_A_impl(static_cast<spm_problem_s *>(c), prec, x, y, nrhs, s);
}
spm_status ops3_Q(void *c, int prec, const void *v, void *y, int nrhs, cudaStream_t s)
{
    return spm_apply_Q_impl(static_cast<spm_problem_s *>(c), prec, v, y, nrhs, s);
}
spm_status ops3_S(void *c, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    return spm_solveS_impl(static_cast<spm_problem_s *>(c), prec, b, x, nrhs, s);
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
    KrylovOps ops;
    ops.N = 3L * P->n * P->n * P->n;
    ops.stream = P->stream;
    ops.ws = &P->gmres_ws;
    ops.ctx = P;
    ops.apply_A = ops3_A;
    ops.apply_Q = ops3_Q;
    ops.solve_S = ops3_S;
    return spm_gmres_solve(ops, prec, g, x, nrhs, tol, maxit, restart, info);
}
