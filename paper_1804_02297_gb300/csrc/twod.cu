// The 2-D variant (Section 2: the integral equation with the 2-D Helmholtz
// kernel G = (i/4) H_0^(1)(k|x|); Section 4, Tables 1-3: two unknowns per grid
// point), on the device end to end:
//   * FP64 Toeplitz entries h^2 K(t h) with the corrected near-diagonal weights,
//     their circulant embedding on an L x L grid (L = power of two >= 2n - 1),
//     FP64 2-D FFTs, and one quadrant [3][L/2+1]^2 of each spectrum (G is even
//     in both frequencies, G^1 odd in the first, G^2 odd in the second);
//   * the apply A x in three passes, each a register-resident Stockham line FFT
//     (fft_reg.cuh): the n nonzero columns forward (pad, contrast weights
//     [m x^1, m x^2, p.x]), the L rows (forward, Fourier-side product
//     y^d = k^2 Ghat w^d + G^d hat w^3, inverse, crop to n), the n columns
//     inverse (crop, + x);
//   * Q and S on the 9-point pattern; the stencils of the nine point classes by
//     an FP64 Gram matrix M M^H summed over each class's complement and a
//     Jacobi eigen-decomposition; S factored by the nested-dissection LU of
//     sparse.cu on the n x n x 1 grid; GMRES from krylov.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "fft.cuh"
#include "fft_reg.cuh"
#include "twod.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double EULER_GAMMA = 0.57721566490153286061;
constexpr int NT2 = 256;

inline unsigned nb(long cnt, int t = 256) { return (unsigned)((cnt + t - 1) / t); }

// ------------------------------------------------------------------ entries
// G_t = h^2 G(t h), G^d_t = h^2 dG/dx_d(t h), with
//   G = (i/4)(J_0 + i Y_0)(k r),  G^d = -(i/4) k (J_1 + i Y_1)(k r) x_d / r,
// and the ORDER4 corrections at t = 0 (G) and t = +-e_d (G^d).
__device__ void entry2_dev(int t1, int t2, double h, double k, int quad, double zp, double2 out[3])
{
    const double h2 = h * h;
    if (t1 == 0 && t2 == 0) {
        const double lg = quad == 0 ? log(0.5 * k * h) + EULER_GAMMA + zp : log(0.5 * k) + EULER_GAMMA;
        out[0] = make_double2(-h2 * lg / (2.0 * PI), 0.25 * h2);
        out[1] = out[2] = make_double2(0.0, 0.0);
        return;
    }
    const double x1 = t1 * h, x2 = t2 * h;
    const double r = hypot(x1, x2), kr = k * r;
    const double J0 = j0(kr), Y0 = y0(kr), J1 = j1(kr), Y1 = y1(kr);
    out[0] = make_double2(-0.25 * h2 * Y0, 0.25 * h2 * J0);
    const double f = 0.25 * h2 * k / r;
    out[1] = make_double2(f * x1 * Y1, -f * x1 * J1);
    out[2] = make_double2(f * x2 * Y1, -f * x2 * J1);
    if (quad == 0) {
        const double w = h / (8.0 * PI);
        if (t2 == 0 && (t1 == 1 || t1 == -1)) out[1].x -= t1 * w;
        if (t1 == 0 && (t2 == 1 || t2 == -1)) out[2].x -= t2 * w;
    }
}

// E[q][t2 + n - 1][t1 + n - 1], q = G, G^1, G^2
__global__ void k2_entries(double2 *E, int n, double h, double k, int quad, double zp)
{
    const int W = 2 * n - 1;
    const long W2 = (long)W * W;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= W2) return;
    const int a1 = (int)(gid % W), a2 = (int)(gid / W);
    double2 e[3];
    entry2_dev(a1 - (n - 1), a2 - (n - 1), h, k, quad, zp, e);
    for (int q = 0; q < 3; ++q) E[q * W2 + gid] = e[q];
}

// circulant embedding of kernel q: slot v holds offset v (v < n) or v - L (v > L - n), else 0
__global__ void k2_circulant(double2 *F, const double2 *__restrict__ E, int q, int n, int L)
{
    const long L2 = (long)L * L;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= L2) return;
    const int v1 = (int)(gid % L), v2 = (int)(gid / L);
    const int t1 = v1 < n ? v1 : (v1 > L - n ? v1 - L : INT32_MAX);
    const int t2 = v2 < n ? v2 : (v2 > L - n ? v2 - L : INT32_MAX);
    if (t1 == INT32_MAX || t2 == INT32_MAX) { F[gid] = make_double2(0.0, 0.0); return; }
    const int W = 2 * n - 1;
    F[gid] = E[(long)q * W * W + (long)(t2 + n - 1) * W + (t1 + n - 1)];
}

// in-place FP64 FFT of nrows contiguous rows of length L, nl rows per block
__global__ void __launch_bounds__(NT2) k2_rows64(double2 *a, int L, long nrows, int nl, const double2 *__restrict__ tw)
{
    extern __shared__ unsigned char smem_raw[];
    double2 *b0 = reinterpret_cast<double2 *>(smem_raw);
    double2 *b1 = b0 + nl * L;
    const long row0 = (long)blockIdx.x * nl;
    for (int i = threadIdx.x; i < nl * L; i += blockDim.x)
        b0[i] = row0 + i / L < nrows ? a[row0 * L + i] : make_double2(0.0, 0.0);
    __syncthreads();
    double2 *res = smem_fft<-1>(b0, b1, L, 0, nl, L, tw);
    for (int i = threadIdx.x; i < nl * L; i += blockDim.x)
        if (row0 + i / L < nrows) a[row0 * L + i] = res[i];
}

// in-place FP64 FFT of the L columns of an L x L array, tx columns per block
__global__ void __launch_bounds__(NT2) k2_cols64(double2 *a, int L, int tx, const double2 *__restrict__ tw)
{
    extern __shared__ unsigned char smem_raw[];
    double2 *b0 = reinterpret_cast<double2 *>(smem_raw);
    double2 *b1 = b0 + tx * L;
    const int c0 = blockIdx.x * tx;
    for (int i = threadIdx.x; i < tx * L; i += blockDim.x) {
        const int c = i % tx, r = i / tx;
        b0[c * L + r] = a[(long)r * L + c0 + c];
    }
    __syncthreads();
    double2 *res = smem_fft<-1>(b0, b1, L, 0, tx, L, tw);
    for (int i = threadIdx.x; i < tx * L; i += blockDim.x) {
        const int c = i % tx, r = i / tx;
        a[(long)r * L + c0 + c] = res[c * L + r];
    }
}

// quadrant [a2][a1], a in [0, L/2], times scale
__global__ void k2_quadrant(const double2 *__restrict__ F, double2 *s128, float2 *s64, int L, double scale)
{
    const int H = L / 2 + 1;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)H * H) return;
    const int a1 = (int)(gid % H), a2 = (int)(gid / H);
    double2 v = F[(long)a2 * L + a1];
    v.x *= scale;
    v.y *= scale;
    s128[gid] = v;
    s64[gid] = to_c64(v);
}

__global__ void k2_twiddles(double2 *tw128, float2 *tw64, int L)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= L) return;
    double s, c;
    sincospi(-2.0 * j / L, &s, &c);
    tw128[j] = make_double2(c, s);
    tw64[j] = make_float2((float)c, (float)s);
}

// m = 1 - eps, p^d = -d_d eps / eps (Section 2), complex128 and complex64 copies
__global__ void k2_medium(const double2 *__restrict__ eps, const double2 *__restrict__ grad, double2 *m128,
                          double2 *p128, float2 *m64, float2 *p64, long N)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 e = eps[i];
    const double2 m = make_double2(1.0 - e.x, -e.y);
    m128[i] = m;
    m64[i] = to_c64(m);
    const double den = e.x * e.x + e.y * e.y;
    for (int d = 0; d < 2; ++d) {
        const double2 g = grad[d * N + i];
        // -g / e = -g conj(e) / |e|^2
        const double2 p = make_double2(-(g.x * e.x + g.y * e.y) / den, -(g.y * e.x - g.x * e.y) / den);
        p128[d * N + i] = p;
        p64[d * N + i] = to_c64(p);
    }
}

// ------------------------------------------------------------------ apply
// Line FFTs of length L: T = L/8 threads per line, thread t holds positions
// t + T m, m = 0..7; the line's shared buffer is padded one slot per 8.
__device__ __forceinline__ int pad8(int pos) { return pos + (pos >> 3); }

template <int L> struct Geo2 {
    static constexpr int T = L / 8;
    static constexpr int LS = L + L / 8; // padded line stride
};

// Pass 1, one column i1 < n per line, COLS adjacent columns per block: the
// weights w = [m x^1, m x^2, p.x] of the block's columns staged in shared
// memory (coalesced across columns), the three fields transformed along x2
// together (input rows >= n are the zero padding; the three lines share every
// barrier), the L frequencies back through shared memory to W[b][f][v2][i1]
// (rows of length n, coalesced across columns).
template <typename R, int L>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 512 : 256)
    k2d_colfwd(const typename cplx_of<R>::type *__restrict__ x, const typename cplx_of<R>::type *__restrict__ m,
               const typename cplx_of<R>::type *__restrict__ p, typename cplx_of<R>::type *__restrict__ W, int n,
               const typename cplx_of<R>::type *__restrict__ tw, int COLS)
{
    using C = typename cplx_of<R>::type;
    constexpr int T = L / 8, LS = L + L / 8;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw); // [field][column][LS]
    const int c = threadIdx.x / T, t = threadIdx.x % T;
    const int col0 = blockIdx.x * COLS;
    const long b = blockIdx.y, N = (long)n * n;
    const C *xb = x + b * 2 * N;
    const long fsm = (long)COLS * LS;
    auto buf = [&](int k, int pos) -> C & { return sm[k * fsm + c * LS + pad8(pos)]; };
    auto sync = [&]() { __syncthreads(); };
    // every thread stages at most 4 points (COLS * n <= COLS * L / 2 = 4 blockDim.x):
    // all loads first, then the shared-memory stores
    {
        C mm[4], e0[4], e1[4], p0[4], p1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = q * blockDim.x + threadIdx.x;
            const int cc = i & (COLS - 1), r = i / COLS, i1 = col0 + cc;
            mm[q] = e0[q] = e1[q] = p0[q] = p1[q] = czero<C>();
            if (r < n && i1 < n) {
                const long o = (long)r * n + i1;
                mm[q] = m[o];
                e0[q] = xb[o];
                e1[q] = xb[N + o];
                p0[q] = p[o];
                p1[q] = p[N + o];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = q * blockDim.x + threadIdx.x;
            const int cc = i & (COLS - 1), r = i / COLS;
            if (r < n) {
                const int at = cc * LS + pad8(r);
                sm[at] = cmul(mm[q], e0[q]);
                sm[fsm + at] = cmul(mm[q], e1[q]);
                sm[2 * fsm + at] = cfma(p0[q], e0[q], cmul(p1[q], e1[q]));
            }
        }
    }
    __syncthreads();
    C v[3][8];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = t + T * q;
            v[f][q] = r < n ? buf(f, r) : czero<C>();
            v[f][q + 4] = czero<C>();
        }
    __syncthreads();
    fftr::fft_lines<-1, L, true, 3>(v, t, buf, sync, tw);
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int q = 0; q < 8; ++q) buf(f, t + T * q) = v[f][q];
    __syncthreads();
    for (int f = 0; f < 3; ++f) {
        C *Wf = W + (b * 3 + f) * (long)L * n;
#pragma unroll
        for (int q = 0; q < 8; ++q) { // COLS * L = 8 blockDim.x
            const int i = q * blockDim.x + threadIdx.x;
            const int cc = i & (COLS - 1), r = i / COLS, i1 = col0 + cc;
            if (i1 < n) Wf[(long)r * n + i1] = sm[f * fsm + cc * LS + pad8(r)];
        }
    }
}

// Pass 2, one row v2 (an x2 frequency) per line: the three fields' rows (length
// n, zero-padded to L) transformed along x1 together, the Fourier-side product
// y^d = (k^2 Ghat) w^d + (G^d hat) w^3 (spectra with 1/L^2 folded in; the
// quadrant tables are read along a row, so the loads coalesce), the two results
// transformed back, their first n entries written over fields 0, 1 of the row.
template <typename R, int L>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k2d_rowprod(typename cplx_of<R>::type *W,
                                                   const typename cplx_of<R>::type *__restrict__ spec, int n,
                                                   const typename cplx_of<R>::type *__restrict__ tw, int RB)
{
    using C = typename cplx_of<R>::type;
    using G = Geo2<L>;
    constexpr int T = G::T, H = L / 2 + 1;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int v2 = blockIdx.x * RB + line; // L rows: RB divides L
    const long b = blockIdx.y;
    C *lb = sm + line * 3 * G::LS;
    auto buf = [&](int k, int pos) -> C & { return lb[k * G::LS + pad8(pos)]; };
    // a line within one warp of a block of whole warps needs only a warp barrier
    const bool warp_lines = T <= 32 && (blockDim.x & 31) == 0;
    auto sync = [&]() { if (warp_lines) __syncwarp(); else __syncthreads(); };
    C *Wr = W + b * 3 * (long)L * n + (long)v2 * n;
    const long fs = (long)L * n; // field stride
    C v[3][8];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i1 = t + T * q;
            v[f][q] = i1 < n ? Wr[f * fs + i1] : czero<C>();
            v[f][q + 4] = czero<C>();
        }
    fftr::fft_lines<-1, L, true, 3>(v, t, buf, sync, tw);
    const int a2 = v2 <= L / 2 ? v2 : L - v2;
    const R s2 = v2 > L / 2 ? (R)-1 : (R)1;
    const C *K0 = spec + (long)a2 * H, *K1 = K0 + (long)H * H, *K2 = K1 + (long)H * H;
    C y[2][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int v1 = t + T * q;
        const int a1 = v1 <= L / 2 ? v1 : L - v1;
        const R s1 = v1 > L / 2 ? (R)-1 : (R)1;
        const C k0 = K0[a1], k1 = cscale(K1[a1], s1), k2 = cscale(K2[a1], s2);
        y[0][q] = cfma(k0, v[0][q], cmul(k1, v[2][q]));
        y[1][q] = cfma(k0, v[1][q], cmul(k2, v[2][q]));
    }
    fftr::fft_lines<1, L, false, 2>(y, t, buf, sync, tw);
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i1 = t + T * q;
            if (i1 < n) Wr[f * fs + i1] = y[f][q];
        }
}

// Pass 3, one column i1 < n per line, COLS adjacent columns per block: the
// L rows of fields 0, 1 staged in shared memory (coalesced across columns),
// both inverse FFTs along x2 together, rows i2 < n back through shared memory,
// y = x + result.
template <typename R, int L>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 512 : 256)
    k2d_colinv(const typename cplx_of<R>::type *__restrict__ W, const typename cplx_of<R>::type *__restrict__ x,
               typename cplx_of<R>::type *__restrict__ y, int n, const typename cplx_of<R>::type *__restrict__ tw,
               int COLS)
{
    using C = typename cplx_of<R>::type;
    constexpr int T = L / 8, LS = L + L / 8;
    extern __shared__ unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw); // [field][column][LS]
    const int c = threadIdx.x / T, t = threadIdx.x % T;
    const int col0 = blockIdx.x * COLS;
    const long b = blockIdx.y, N = (long)n * n;
    const long fsm = (long)COLS * LS;
    auto buf = [&](int k, int pos) -> C & { return sm[k * fsm + c * LS + pad8(pos)]; };
    auto sync = [&]() { __syncthreads(); };
    {   // COLS * L = 8 blockDim.x elements per field: all 16 loads first
        C t8[2][8];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const C *Wf = W + (b * 3 + f) * (long)L * n;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = q * blockDim.x + threadIdx.x;
                const int cc = i & (COLS - 1), r = i / COLS, i1 = col0 + cc;
                t8[f][q] = i1 < n ? Wf[(long)r * n + i1] : czero<C>();
            }
        }
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = q * blockDim.x + threadIdx.x;
                sm[f * fsm + (i & (COLS - 1)) * LS + pad8(i / COLS)] = t8[f][q];
            }
    }
    __syncthreads();
    C v[2][8];
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int q = 0; q < 8; ++q) v[f][q] = buf(f, t + T * q);
    __syncthreads();
    fftr::fft_lines<1, L, false, 2>(v, t, buf, sync, tw);
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = t + T * q;
            if (r < n) buf(f, r) = v[f][q];
        }
    __syncthreads();
    for (int f = 0; f < 2; ++f) {
        C xv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { // COLS * n <= 4 blockDim.x
            const int i = q * blockDim.x + threadIdx.x;
            const int cc = i & (COLS - 1), r = i / COLS, i1 = col0 + cc;
            xv[q] = r < n && i1 < n ? x[(b * 2 + f) * N + (long)r * n + i1] : czero<C>();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = q * blockDim.x + threadIdx.x;
            const int cc = i & (COLS - 1), r = i / COLS, i1 = col0 + cc;
            if (r < n && i1 < n) y[(b * 2 + f) * N + (long)r * n + i1] = xv[q] + sm[f * fsm + cc * LS + pad8(r)];
        }
    }
}

template <typename K> spm_status allow_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) SPM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return SPM_OK;
}

template <typename R, int L>
spm_status apply_L(spm2_problem_s *P, const void *xv, void *yv, int nrhs, cudaStream_t s)
{
    using C = typename cplx_of<R>::type;
    const bool dbl = sizeof(R) == 8;
    const int n = P->n;
    const long N = (long)n * n;
    const C *m = dbl ? P->m128.as<C>() : P->m64.as<C>();
    const C *p = dbl ? P->p128.as<C>() : P->p64.as<C>();
    const C *spec = dbl ? P->spec128.as<C>() : P->spec64.as<C>();
    const C *tw = dbl ? P->tw128.as<C>() : P->tw64.as<C>();
    const long per = 3L * n * L; // workspace elements per right-hand side: W[3][L][n]
    int chunk = (int)std::max<long>(1, std::min<long>(nrhs, (512L << 20) / (long)(per * sizeof(C))));
    SPM_TRY(P->work.ensure(sizeof(C) * per * chunk));
    C *W = P->work.as<C>();
    using G = Geo2<L>;
    // Columns per block of the column passes and rows per block of the row pass:
    // as many as keep two blocks per SM busy (powers of two, at most 16 columns
    // and 512 (complex64) or 256 (complex128) threads, at most 256 threads per
    // row block).
    auto pow2_floor = [](long v) { int r = 1; while ((long)r * 2 <= v) r *= 2; return r; };
    const int max_cols = std::max(1, (sizeof(R) == 4 ? 512 : 256) / G::T);
    const int cols = std::max(1, std::min({16, max_cols, pow2_floor(std::max(1L, (long)n / 304))}));
    const int rb = std::max(1, std::min({L, std::max(1, 256 / G::T), pow2_floor(std::max(1L, (long)L / 304))}));
    const size_t sm_rows = sizeof(C) * rb * 3 * G::LS, sm_cols = sizeof(C) * 3 * cols * G::LS;
    SPM_TRY(allow_smem(k2d_colfwd<R, L>, sm_cols));
    SPM_TRY(allow_smem(k2d_rowprod<R, L>, sm_rows));
    SPM_TRY(allow_smem(k2d_colinv<R, L>, sm_cols));
    for (int b0 = 0; b0 < nrhs; b0 += chunk) {
        const int nb_ = std::min(chunk, nrhs - b0);
        const C *x = reinterpret_cast<const C *>(xv) + (long)b0 * 2 * N;
        C *y = reinterpret_cast<C *>(yv) + (long)b0 * 2 * N;
        const dim3 gcol((unsigned)((n + cols - 1) / cols), (unsigned)nb_);
        k2d_colfwd<R, L><<<gcol, cols * G::T, sm_cols, s>>>(x, m, p, W, n, tw, cols);
        k2d_rowprod<R, L><<<dim3(L / rb, (unsigned)nb_), rb * G::T, sm_rows, s>>>(W, spec, n, tw, rb);
        k2d_colinv<R, L><<<gcol, cols * G::T, sm_cols, s>>>(W, x, y, n, tw, cols);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

template <typename R>
spm_status apply_typed(spm2_problem_s *P, const void *x, void *y, int nrhs, cudaStream_t s)
{
    switch (P->L) {
    case 8: return apply_L<R, 8>(P, x, y, nrhs, s);
    case 16: return apply_L<R, 16>(P, x, y, nrhs, s);
    case 32: return apply_L<R, 32>(P, x, y, nrhs, s);
    case 64: return apply_L<R, 64>(P, x, y, nrhs, s);
    case 128: return apply_L<R, 128>(P, x, y, nrhs, s);
    case 256: return apply_L<R, 256>(P, x, y, nrhs, s);
    case 512: return apply_L<R, 512>(P, x, y, nrhs, s);
    case 1024: return apply_L<R, 1024>(P, x, y, nrhs, s);
    case 2048: return apply_L<R, 2048>(P, x, y, nrhs, s);
    default: spm_set_error("no FFT length %d", P->L); return SPM_ERR_INVALID_ARG;
    }
}

// ------------------------------------------------------------------ Q and S
// Offsets s = (o1 + 1) + 3 (o2 + 1) of the 9-point pattern; class of a point.
__device__ __forceinline__ int cls_of(int i1, int i2, int n)
{
    const int c1 = i1 == 0 ? 0 : (i1 == n - 1 ? 2 : 1), c2 = i2 == 0 ? 0 : (i2 == n - 1 ? 2 : 1);
    return c1 + 3 * c2;
}

// (Q v)_{i,c} = sum_{s,d} qtab[cls][c][s][d] v^d_{i+o_s}
template <typename C>
__global__ void k2_applyQ(const C *__restrict__ qtab, const C *__restrict__ v, C *__restrict__ y, int n, long total)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long N = (long)n * n, b = gid / N, i = gid - b * N;
    const int i1 = (int)(i % n), i2 = (int)(i / n);
    const int cls = cls_of(i1, i2, n);
    const C *vb = v + b * 2 * N;
    C acc[2] = {czero<C>(), czero<C>()};
    for (int s = 0; s < 9; ++s) {
        const int j1 = i1 + s % 3 - 1, j2 = i2 + s / 3 - 1;
        if (j1 < 0 || j2 < 0 || j1 >= n || j2 >= n) continue;
        const long j = (long)j2 * n + j1;
        const C v0 = vb[j], v1 = vb[N + j];
        for (int c = 0; c < 2; ++c) {
            const C *q = qtab + ((cls * 2 + c) * 9 + s) * 2;
            acc[c] = cfma(q[0], v0, cfma(q[1], v1, acc[c]));
        }
    }
    y[b * 2 * N + i] = acc[0];
    y[b * 2 * N + N + i] = acc[1];
}

// S[i][s][c][f] = alpha[(f,o),c] + beta[(f,o),c] m_j + beta[(2,o),c] p^f_j, j = i + o_s
__global__ void k2_assemble(const double2 *__restrict__ qt, const double2 *__restrict__ bt,
                            const double2 *__restrict__ m, const double2 *__restrict__ p, double2 *S128, float2 *S64,
                            int n)
{
    const long N = (long)n * n;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N * 9) return;
    const long i = gid / 9;
    const int s = (int)(gid % 9);
    const int i1 = (int)(i % n), i2 = (int)(i / n);
    const int j1 = i1 + s % 3 - 1, j2 = i2 + s / 3 - 1;
    const bool in = j1 >= 0 && j2 >= 0 && j1 < n && j2 < n;
    const int cls = cls_of(i1, i2, n);
    const long j = in ? (long)j2 * n + j1 : 0;
    for (int c = 0; c < 2; ++c)
        for (int f = 0; f < 2; ++f) {
            double2 v = make_double2(0.0, 0.0);
            if (in) {
                const double2 a = qt[((cls * 2 + c) * 9 + s) * 2 + f];
                const double2 bf = bt[((cls * 2 + c) * 9 + s) * 3 + f];
                const double2 b3 = bt[((cls * 2 + c) * 9 + s) * 3 + 2];
                v = cfma(b3, p[f * N + j], cfma(bf, m[j], a));
            }
            S128[gid * 4 + c * 2 + f] = v;
            S64[gid * 4 + c * 2 + f] = to_c64(v);
        }
}

template <typename C>
__global__ void k2_applyS(const C *__restrict__ S, const C *__restrict__ x, C *__restrict__ y, int n, long total)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long N = (long)n * n, b = gid / N, i = gid - b * N;
    const int i1 = (int)(i % n), i2 = (int)(i / n);
    const C *xb = x + b * 2 * N;
    C acc[2] = {czero<C>(), czero<C>()};
    for (int s = 0; s < 9; ++s) {
        const int j1 = i1 + s % 3 - 1, j2 = i2 + s / 3 - 1;
        if (j1 < 0 || j2 < 0 || j1 >= n || j2 >= n) continue;
        const long j = (long)j2 * n + j1;
        const C *blk = S + (i * 9 + s) * 4;
        const C x0 = xb[j], x1 = xb[N + j];
        acc[0] = cfma(blk[0], x0, cfma(blk[1], x1, acc[0]));
        acc[1] = cfma(blk[2], x0, cfma(blk[3], x1, acc[1]));
    }
    y[b * 2 * N + i] = acc[0];
    y[b * 2 * N + N + i] = acc[1];
}

// ------------------------------------------------------------------ stencil fit
// Class geometry: neighbourhood offsets per axis {0,1} (c = 0), {-1,0,1} (1),
// {-1,0} (2); complement box per axis [0,n-1], [-(n-2),n-2], [-(n-1),0].
struct Geom2 {
    int T;
    int off[9][2];     // neighbourhood offsets, o2 outer, o1 inner
    int rlo[2], rhi[2]; // complement box
};

Geom2 geom2(int cls, int n)
{
    Geom2 g;
    const int c[2] = {cls % 3, cls / 3};
    int tlo[2], thi[2];
    for (int d = 0; d < 2; ++d) {
        tlo[d] = c[d] == 0 ? 0 : -1;
        thi[d] = c[d] == 2 ? 0 : 1;
        g.rlo[d] = c[d] == 0 ? 0 : (c[d] == 1 ? -(n - 2) : -(n - 1));
        g.rhi[d] = c[d] == 0 ? n - 1 : (c[d] == 1 ? n - 2 : 0);
    }
    g.T = 0;
    for (int o2 = tlo[1]; o2 <= thi[1]; ++o2)
        for (int o1 = tlo[0]; o1 <= thi[0]; ++o1) {
            g.off[g.T][0] = o1;
            g.off[g.T][1] = o2;
            ++g.T;
        }
    return g;
}

constexpr int GRAM_BLOCKS = 608; // 4 x 152 SMs
constexpr int GRAM_UT = 64;      // complement offsets staged per tile

// Partial Gram sums, one block per slice of the complement box: the block
// stages, for a tile of complement offsets u, the entries K_q(o - u) of the
// three kernels at the class's T neighbourhood offsets o (shared memory), and
// thread (o, o') accumulates the four sums C_00, C_11, C_12, C_22 of
// C_ab[o][o'] = sum_u K_a(o - u) conj(K_b(o' - u)), K_0 = G, K_d = G^d, over
// the tile (u in the neighbourhood box itself is skipped).  part[block][kind][pair].
__global__ void __launch_bounds__(128) k2_gram(const double2 *__restrict__ E, Geom2 g, int n, double2 *part)
{
    __shared__ double2 st[GRAM_UT][9][3];
    const int W = 2 * n - 1;
    const long W2 = (long)W * W;
    const int w1 = g.rhi[0] - g.rlo[0] + 1, w2 = g.rhi[1] - g.rlo[1] + 1;
    const long box = (long)w1 * w2;
    const long per = (box + gridDim.x - 1) / gridDim.x;
    const long u0 = (long)blockIdx.x * per, u1 = min(box, u0 + per);
    const int T = g.T, pair = threadIdx.x;
    const bool act = pair < T * T;
    const int o = act ? pair / T : 0, op = act ? pair % T : 0;
    int tlo[2] = {g.off[0][0], g.off[0][1]}, thi[2] = {g.off[T - 1][0], g.off[T - 1][1]};
    double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (long t0 = u0; t0 < u1; t0 += GRAM_UT) {
        const int cnt = (int)min((long)GRAM_UT, u1 - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * T * 3; i += blockDim.x) {
            const int ul = i / (T * 3), rem = i % (T * 3), oo = rem / 3, q = rem % 3;
            const long idx = t0 + ul;
            const int uu1 = g.rlo[0] + (int)(idx % w1), uu2 = g.rlo[1] + (int)(idx / w1);
            const long e = (long)(g.off[oo][1] - uu2 + n - 1) * W + (g.off[oo][0] - uu1 + n - 1);
            st[ul][oo][q] = E[q * W2 + e];
        }
        __syncthreads();
        if (act) {
            for (int ul = 0; ul < cnt; ++ul) {
                const long idx = t0 + ul;
                const int uu1 = g.rlo[0] + (int)(idx % w1), uu2 = g.rlo[1] + (int)(idx / w1);
                if (uu1 >= tlo[0] && uu1 <= thi[0] && uu2 >= tlo[1] && uu2 <= thi[1]) continue; // u in tau
                const double2 a0 = st[ul][o][0], a1 = st[ul][o][1], a2 = st[ul][o][2];
                const double2 b0 = st[ul][op][0], b1 = st[ul][op][1], b2 = st[ul][op][2];
                acc[0] = cfma(a0, conj_of(b0), acc[0]);
                acc[1] = cfma(a1, conj_of(b1), acc[1]);
                acc[2] = cfma(a1, conj_of(b2), acc[2]);
                acc[3] = cfma(a2, conj_of(b2), acc[3]);
            }
        }
    }
    if (act)
        for (int kk = 0; kk < 4; ++kk) part[((long)blockIdx.x * 4 + kk) * 81 + pair] = acc[kk];
}

// sum the per-block partial Gram sums: out[kind][pair]
__global__ void k2_gram_sum(const double2 *__restrict__ part, int nblocks, double2 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * 81) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nblocks; ++b) s = s + part[(long)b * 4 * 81 + i];
    out[i] = s;
}

__device__ __forceinline__ double2 zm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// One thread per class: H = M M^H from the Gram sums, cyclic Jacobi
// eigen-decomposition, alpha = conj(eigenvectors of the two smallest
// eigenvalues), sv = sqrt(eigenvalues) ascending, beta = B^T alpha.
__global__ void k2_eig(const double2 *__restrict__ part, const double2 *__restrict__ E, Geom2 g, int n, double k,
                       double2 *alpha, double2 *beta, double *sv)
{
    // the small dense work sits in shared memory (no large per-thread stack frame)
    __shared__ double2 Cs[4][81], A[18][18], V[18][18];
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int T = g.T, M = 2 * T;
    for (int kk = 0; kk < 4; ++kk)
        for (int pr = 0; pr < T * T; ++pr) Cs[kk][pr] = part[kk * 81 + pr];
    const double k4 = k * k * k * k;
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) {
            const int d = r / T, o = r % T, e = c / T, op = c % T;
            double2 v;
            if (d == 0 && e == 0) v = Cs[1][o * T + op];
            else if (d == 1 && e == 1) v = Cs[3][o * T + op];
            else if (d == 0 && e == 1) v = Cs[2][o * T + op];
            else v = conj_of(Cs[2][op * T + o]); // C_21[o][o'] = conj(C_12[o'][o])
            if (d == e) { v.x += k4 * Cs[0][o * T + op].x; v.y += k4 * Cs[0][o * T + op].y; }
            A[r][c] = v;
            V[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
        }
    for (int r = 0; r < M; ++r) A[r][r].y = 0.0;
    double fro = 0;
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) fro += A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int r = 0; r < M; ++r)
            for (int c = r + 1; c < M; ++c) off += A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
        if (off <= 1e-34 * fro) break;
        for (int pp = 0; pp < M; ++pp)
            for (int q = pp + 1; q < M; ++q) {
                const double2 cpq = A[pp][q];
                const double ab = sqrt(cpq.x * cpq.x + cpq.y * cpq.y);
                if (ab <= 1e-300) continue;
                const double2 e = make_double2(cpq.x / ab, cpq.y / ab); // phase of A_pq
                const double zeta = (A[q][q].x - A[pp][pp].x) / (2.0 * ab);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                // J = diag(1, conj e) * [[cs, sn], [-sn, cs]] on (pp, q): A <- J^H A J, V <- V J
                const double2 ce = conj_of(e);
                for (int r = 0; r < M; ++r) { // columns
                    const double2 ap = A[r][pp], aq = A[r][q];
                    const double2 aqe = zm(aq, ce);
                    A[r][pp] = make_double2(cs * ap.x - sn * aqe.x, cs * ap.y - sn * aqe.y);
                    A[r][q] = make_double2(sn * ap.x + cs * aqe.x, sn * ap.y + cs * aqe.y);
                    const double2 vp = V[r][pp], vq = V[r][q];
                    const double2 vqe = zm(vq, ce);
                    V[r][pp] = make_double2(cs * vp.x - sn * vqe.x, cs * vp.y - sn * vqe.y);
                    V[r][q] = make_double2(sn * vp.x + cs * vqe.x, sn * vp.y + cs * vqe.y);
                }
                for (int c = 0; c < M; ++c) { // rows
                    const double2 ap = A[pp][c], aq = A[q][c];
                    const double2 aqe = zm(aq, e);
                    A[pp][c] = make_double2(cs * ap.x - sn * aqe.x, cs * ap.y - sn * aqe.y);
                    A[q][c] = make_double2(sn * ap.x + cs * aqe.x, sn * ap.y + cs * aqe.y);
                }
                A[pp][q] = A[q][pp] = make_double2(0.0, 0.0);
                A[pp][pp].y = A[q][q].y = 0.0;
            }
    }
    int idx[18];
    for (int i = 0; i < M; ++i) idx[i] = i;
    for (int i = 1; i < M; ++i) { // insertion sort by eigenvalue
        const int v = idx[i];
        int j = i - 1;
        while (j >= 0 && A[idx[j]][idx[j]].x > A[v][v].x) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = v;
    }
    for (int i = 0; i < 18; ++i) sv[i] = i < M ? sqrt(fmax(A[idx[i]][idx[i]].x, 0.0)) : 0.0;
    for (int r = 0; r < 18; ++r)
        for (int c = 0; c < 2; ++c) alpha[r * 2 + c] = r < M ? conj_of(V[r][idx[c]]) : make_double2(0.0, 0.0);
    // beta[(f,o'),c] = sum_{(d,o)} alpha[(d,o),c] K_{(d,o),(f,o')}
    const int W = 2 * n - 1;
    const long W2 = (long)W * W;
    const double k2 = k * k;
    for (int r = 0; r < 27; ++r)
        for (int c = 0; c < 2; ++c) beta[r * 2 + c] = make_double2(0.0, 0.0);
    for (int f = 0; f < 3; ++f)
        for (int op = 0; op < T; ++op)
            for (int c = 0; c < 2; ++c) {
                double2 s = make_double2(0.0, 0.0);
                for (int d = 0; d < 2; ++d)
                    for (int o = 0; o < T; ++o) {
                        const long e = (long)(g.off[o][1] - g.off[op][1] + n - 1) * W + (g.off[o][0] - g.off[op][0] + n - 1);
                        double2 K;
                        if (f < 2) {
                            if (f != d) continue;
                            K = make_double2(k2 * E[e].x, k2 * E[e].y);
                        } else {
                            K = E[(1 + d) * W2 + e];
                        }
                        s = cfma(alpha[(d * T + o) * 2 + c], K, s);
                    }
                beta[(f * T + op) * 2 + c] = s;
            }
}

} // namespace

// ------------------------------------------------------------------ internal API
spm_status spm2_apply_A_impl(spm2_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s)
{
    return prec == SPM_C128 ? apply_typed<double>(P, x, y, nrhs, s) : apply_typed<float>(P, x, y, nrhs, s);
}

spm_status spm2_apply_Q_impl(spm2_problem_s *P, int prec, const void *v, void *y, int nrhs, cudaStream_t s)
{
    const long total = (long)nrhs * P->n * P->n;
    if (prec == SPM_C128)
        k2_applyQ<double2><<<nb(total), 256, 0, s>>>(P->qtab128.as<double2>(), (const double2 *)v, (double2 *)y, P->n, total);
    else
        k2_applyQ<float2><<<nb(total), 256, 0, s>>>(P->qtab64.as<float2>(), (const float2 *)v, (float2 *)y, P->n, total);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

spm_status spm2_apply_S_impl(spm2_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s)
{
    const long total = (long)nrhs * P->n * P->n;
    if (prec == SPM_C128)
        k2_applyS<double2><<<nb(total), 256, 0, s>>>(P->S128.as<double2>(), (const double2 *)x, (double2 *)y, P->n, total);
    else
        k2_applyS<float2><<<nb(total), 256, 0, s>>>(P->S64.as<float2>(), (const float2 *)x, (float2 *)y, P->n, total);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
bool prec_ok(spm_prec p) { return p == SPM_C128 || p == SPM_C64; }

spm_status build_spectra(spm2_problem_s *P)
{
    const int n = P->n, L = P->L, W = 2 * n - 1, H = L / 2 + 1;
    const long L2 = (long)L * L;
    cudaStream_t s = P->stream;
    SPM_TRY(P->entries.ensure(sizeof(double2) * 3 * (size_t)W * W));
    k2_entries<<<nb((long)W * W), 256, 0, s>>>(P->entries.as<double2>(), n, P->h, P->k, P->quad, P->zprime);
    DevBuf full;
    SPM_TRY(full.ensure(sizeof(double2) * L2));
    SPM_TRY(P->spec128.ensure(sizeof(double2) * 3 * (size_t)H * H));
    SPM_TRY(P->spec64.ensure(sizeof(float2) * 3 * (size_t)H * H));
    const int nl = L >= 256 ? 1 : 256 / L;
    const int tx = std::max(1, std::min(std::min(16, L), 4096 / L));
    const size_t sm_r = 2 * sizeof(double2) * nl * L, sm_c = 2 * sizeof(double2) * tx * L;
    SPM_TRY(allow_smem(k2_rows64, sm_r));
    SPM_TRY(allow_smem(k2_cols64, sm_c));
    const double2 *tw = P->tw128.as<double2>();
    for (int q = 0; q < 3; ++q) {
        k2_circulant<<<nb(L2), 256, 0, s>>>(full.as<double2>(), P->entries.as<double2>(), q, n, L);
        k2_rows64<<<(unsigned)((L + nl - 1) / nl), NT2, sm_r, s>>>(full.as<double2>(), L, L, nl, tw);
        k2_cols64<<<(unsigned)(L / tx), NT2, sm_c, s>>>(full.as<double2>(), L, tx, tw);
        const double scale = (q == 0 ? P->k * P->k : 1.0) / (double)L2;
        k2_quadrant<<<nb((long)H * H), 256, 0, s>>>(full.as<double2>(), P->spec128.as<double2>() + (long)q * H * H,
                                                    P->spec64.as<float2>() + (long)q * H * H, L, scale);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    return SPM_OK;
}

// qtab / btab from the host stencil tables: value of (row (f,o), column c) on
// the 9-point offset s of o, zeros for offsets outside the class's neighbourhood
spm_status install_stencils(spm2_problem_s *P)
{
    const int n = P->n;
    std::vector<double2> qt(9 * 2 * 9 * 2), bt(9 * 2 * 9 * 3);
    for (auto &v : qt) v = make_double2(0, 0);
    for (auto &v : bt) v = make_double2(0, 0);
    const double2 *al = reinterpret_cast<const double2 *>(P->alpha_h.data());
    const double2 *be = reinterpret_cast<const double2 *>(P->beta_h.data());
    for (int cls = 0; cls < 9; ++cls) {
        const Geom2 g = geom2(cls, n);
        for (int o = 0; o < g.T; ++o) {
            const int s = (g.off[o][0] + 1) + 3 * (g.off[o][1] + 1);
            for (int c = 0; c < 2; ++c) {
                for (int d = 0; d < 2; ++d) qt[((cls * 2 + c) * 9 + s) * 2 + d] = al[(cls * 18 + d * g.T + o) * 2 + c];
                for (int f = 0; f < 3; ++f) bt[((cls * 2 + c) * 9 + s) * 3 + f] = be[(cls * 27 + f * g.T + o) * 2 + c];
            }
        }
    }
    std::vector<float2> qt64(qt.size());
    for (size_t i = 0; i < qt.size(); ++i) qt64[i] = to_c64(qt[i]);
    cudaStream_t s = P->stream;
    SPM_TRY(P->qtab128.ensure(sizeof(double2) * qt.size()));
    SPM_TRY(P->qtab64.ensure(sizeof(float2) * qt.size()));
    DevBuf btd;
    SPM_TRY(btd.ensure(sizeof(double2) * bt.size()));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->qtab128.ptr, qt.data(), sizeof(double2) * qt.size(), cudaMemcpyHostToDevice, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->qtab64.ptr, qt64.data(), sizeof(float2) * qt.size(), cudaMemcpyHostToDevice, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(btd.ptr, bt.data(), sizeof(double2) * bt.size(), cudaMemcpyHostToDevice, s));
    const long N = (long)n * n;
    SPM_TRY(P->S128.ensure(sizeof(double2) * N * 9 * 4));
    SPM_TRY(P->S64.ensure(sizeof(float2) * N * 9 * 4));
    k2_assemble<<<nb(N * 9), 256, 0, s>>>(P->qtab128.as<double2>(), btd.as<double2>(), P->m128.as<double2>(),
                                          P->p128.as<double2>(), P->S128.as<double2>(), P->S64.as<float2>(), n);
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    P->have_stencils = true;
    P->have_S = true;
    spm_factor_free(P->fac128);
    spm_factor_free(P->fac64);
    P->fac128 = P->fac64 = nullptr;
    return SPM_OK;
}

spm_status fit_stencils(spm2_problem_s *P)
{
    const int n = P->n;
    cudaStream_t s = P->stream;
    DevBuf part, out;
    SPM_TRY(part.ensure(sizeof(double2) * (GRAM_BLOCKS + 1) * 4 * 81));
    double2 *sums = part.as<double2>() + (long)GRAM_BLOCKS * 4 * 81;
    SPM_TRY(out.ensure(sizeof(double2) * 9 * (18 + 27) * 2 + sizeof(double) * 9 * 18));
    double2 *al = out.as<double2>(), *be = al + 9 * 18 * 2;
    double *sv = reinterpret_cast<double *>(be + 9 * 27 * 2);
    for (int cls = 0; cls < 9; ++cls) {
        const Geom2 g = geom2(cls, n);
        k2_gram<<<GRAM_BLOCKS, 128, 0, s>>>(P->entries.as<double2>(), g, n, part.as<double2>());
        k2_gram_sum<<<3, 128, 0, s>>>(part.as<double2>(), GRAM_BLOCKS, sums);
        k2_eig<<<1, 32, 0, s>>>(sums, P->entries.as<double2>(), g, n, P->k, al + cls * 36, be + cls * 54,
                                sv + cls * 18);
        SPM_CUDA_TRY(cudaGetLastError());
    }
    P->alpha_h.resize(9 * 18 * 2 * 2);
    P->beta_h.resize(9 * 27 * 2 * 2);
    P->sv_h.resize(9 * 18);
    SPM_CUDA_TRY(cudaMemcpyAsync(P->alpha_h.data(), al, sizeof(double2) * 9 * 18 * 2, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->beta_h.data(), be, sizeof(double2) * 9 * 27 * 2, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->sv_h.data(), sv, sizeof(double) * 9 * 18, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    return install_stencils(P);
}

spm_status apply_S128_2d(void *ctx, const void *x, void *y, cudaStream_t s)
{
    return spm2_apply_S_impl(static_cast<spm2_problem_s *>(ctx), SPM_C128, x, y, 1, s);
}

SparseSys sys2_of(spm2_problem_s *P)
{
    SparseSys S;
    S.dims[0] = S.dims[1] = P->n;
    S.dims[2] = 1;
    S.D = 2;
    S.nsten = 9;
    S.S128 = P->S128.ptr;
    S.S64 = P->S64.ptr;
    S.stream = P->stream;
    S.slot128 = &P->fac128;
    S.slot64 = &P->fac64;
    S.info = P->fac_info;
    S.apply_S128 = apply_S128_2d;
    S.ctx = P;
    return S;
}

spm_status ops2_A(void *c, int prec, const void *x, void *y, int nrhs, cudaStream_t s)
{
    return spm2_apply_A_impl(static_cast<spm2_problem_s *>(c), prec, x, y, nrhs, s);
}
spm_status ops2_Q(void *c, int prec, const void *v, void *y, int nrhs, cudaStream_t s)
{
    return spm2_apply_Q_impl(static_cast<spm2_problem_s *>(c), prec, v, y, nrhs, s);
}
spm_status ops2_S(void *c, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    spm2_problem_s *P = static_cast<spm2_problem_s *>(c);
    return spm_nd_solve(prec == SPM_C128 ? P->fac128 : P->fac64, prec, b, x, nrhs, s);
}

spm_status check_io(spm2_problem P, spm_prec prec, const void *x, void *y, int nrhs)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(prec)) { spm_set_error("precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    if (nrhs < 0 || nrhs > 65535) { spm_set_error("nrhs must be in [0, 65535]"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && (!x || !y)) { spm_set_error("NULL buffer"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && x == y) { spm_set_error("input and output alias"); return SPM_ERR_INVALID_ARG; }
    return SPM_OK;
}

} // namespace

// ------------------------------------------------------------------ C ABI
// Z'(0) of Z(s) = sum'_{j in Z^2} |j|^{-s} = 4 zeta(s/2) beta(s/2):
// 2 (zeta'(0) beta(0) + zeta(0) beta'(0)) = -ln(2 pi)/2 - ln(Gamma(1/4)^2/(2 pi sqrt 2)).
extern "C" double spm2_lattice_zeta_prime(void)
{
    return -0.5 * log(2.0 * PI) - (2.0 * lgamma(0.25) - log(2.0 * PI * sqrt(2.0)));
}

extern "C" spm_status spm2_create_problem(int n, double omega, const double *eps_host, const double *grad_eps_host,
                                          spm_quad quad, void *stream, spm2_problem *out)
{
    if (!out) { spm_set_error("out is NULL"); return SPM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 4 || n > 1024) { spm_set_error("n = %d outside [4, 1024]", n); return SPM_ERR_INVALID_ARG; }
    if (!(omega > 0.0) || !isfinite(omega)) { spm_set_error("omega must be positive and finite"); return SPM_ERR_INVALID_ARG; }
    if (!eps_host || !grad_eps_host) { spm_set_error("eps_host and grad_eps_host are required"); return SPM_ERR_INVALID_ARG; }
    if (quad != SPM_QUAD_ORDER4 && quad != SPM_QUAD_ORDER2) { spm_set_error("bad quadrature %d", (int)quad); return SPM_ERR_INVALID_ARG; }
    const long N = (long)n * n;
    for (long i = 0; i < N; ++i) {
        const double er = eps_host[2 * i], ei = eps_host[2 * i + 1];
        if (!(er * er + ei * ei > 0.0) || !isfinite(er) || !isfinite(ei)) {
            spm_set_error("eps[%ld] is zero or not finite", i);
            return SPM_ERR_INVALID_ARG;
        }
    }
    spm2_problem_s *P = new spm2_problem_s();
    P->n = n;
    P->L = 8;
    while (P->L < 2 * n - 1) P->L *= 2;
    P->k = omega;
    P->h = 1.0 / (n + 1);
    P->quad = (int)quad;
    P->zprime = spm2_lattice_zeta_prime();
    P->stream = as_stream(stream);
    auto fail = [&](spm_status st) { delete P; return st; };
    cudaStream_t s = P->stream;
    DevBuf host_in;
    spm_status st = host_in.ensure(sizeof(double2) * 3 * N);
    if (st != SPM_OK) return fail(st);
    if (cudaMemcpyAsync(host_in.ptr, eps_host, sizeof(double2) * N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(host_in.as<double2>() + N, grad_eps_host, sizeof(double2) * 2 * N, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
        spm_set_error("copy of the medium failed");
        return fail(SPM_ERR_CUDA);
    }
    if ((st = P->m128.ensure(sizeof(double2) * N)) != SPM_OK || (st = P->p128.ensure(sizeof(double2) * 2 * N)) != SPM_OK ||
        (st = P->m64.ensure(sizeof(float2) * N)) != SPM_OK || (st = P->p64.ensure(sizeof(float2) * 2 * N)) != SPM_OK ||
        (st = P->tw128.ensure(sizeof(double2) * P->L)) != SPM_OK || (st = P->tw64.ensure(sizeof(float2) * P->L)) != SPM_OK)
        return fail(st);
    k2_medium<<<nb(N), 256, 0, s>>>(host_in.as<double2>(), host_in.as<double2>() + N, P->m128.as<double2>(),
                                    P->p128.as<double2>(), P->m64.as<float2>(), P->p64.as<float2>(), N);
    k2_twiddles<<<nb(P->L), 256, 0, s>>>(P->tw128.as<double2>(), P->tw64.as<float2>(), P->L);
    if (cudaGetLastError() != cudaSuccess) { spm_set_error("medium kernels failed to launch"); return fail(SPM_ERR_CUDA); }
    if ((st = build_spectra(P)) != SPM_OK) return fail(st);
    *out = P;
    return SPM_OK;
}

extern "C" spm_status spm2_destroy(spm2_problem P)
{
    if (!P) return SPM_OK;
    cudaStreamSynchronize(P->stream);
    spm_factor_free(P->fac128);
    spm_factor_free(P->fac64);
    delete P;
    return SPM_OK;
}

extern "C" spm_status spm2_problem_info(spm2_problem P, int *n, int *L, double *k)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (n) *n = P->n;
    if (L) *L = P->L;
    if (k) *k = P->k;
    return SPM_OK;
}

extern "C" spm_status spm2_kernel_entries(spm2_problem P, double *out_host)
{
    if (!P || !out_host) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    const long W = 2L * P->n - 1;
    SPM_CUDA_TRY(cudaMemcpyAsync(out_host, P->entries.ptr, sizeof(double2) * 3 * W * W, cudaMemcpyDeviceToHost, P->stream));
    SPM_CUDA_TRY(cudaStreamSynchronize(P->stream));
    return SPM_OK;
}

extern "C" spm_status spm2_apply_A(spm2_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, prec, x, y, nrhs));
    if (nrhs == 0) return SPM_OK;
    return spm2_apply_A_impl(P, prec, x, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm2_apply_Q(spm2_problem P, spm_prec prec, const void *v, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, prec, v, y, nrhs));
    if (!P->have_stencils) { spm_set_error("stencils not built (spm2_build_stencils)"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    return spm2_apply_Q_impl(P, prec, v, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm2_apply_QA(spm2_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, prec, x, y, nrhs));
    if (!P->have_stencils) { spm_set_error("stencils not built (spm2_build_stencils)"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    const size_t el = prec == SPM_C128 ? sizeof(double2) : sizeof(float2);
    SPM_TRY(P->kry.ensure(el * 2 * (size_t)P->n * P->n * nrhs));
    cudaStream_t s = as_stream(stream);
    SPM_TRY(spm2_apply_A_impl(P, prec, x, P->kry.ptr, nrhs, s));
    return spm2_apply_Q_impl(P, prec, P->kry.ptr, y, nrhs, s);
}

extern "C" spm_status spm2_build_stencils(spm2_problem P, spm_prec factor_prec)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (factor_prec != SPM_C128 && factor_prec != SPM_C64 && factor_prec != SPM_C64H) {
        spm_set_error("factor precision must be SPM_C128, SPM_C64 or SPM_C64H");
        return SPM_ERR_INVALID_ARG;
    }
    SPM_TRY(fit_stencils(P));
    return spm_nd_factor(sys2_of(P), factor_prec);
}

extern "C" spm_status spm2_set_stencils(spm2_problem P, const double *alpha_host, const double *beta_host)
{
    if (!P || !alpha_host || !beta_host) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    P->alpha_h.assign(alpha_host, alpha_host + 9 * 18 * 2 * 2);
    P->beta_h.assign(beta_host, beta_host + 9 * 27 * 2 * 2);
    P->sv_h.assign(9 * 18, 0.0);
    return install_stencils(P);
}

extern "C" spm_status spm2_get_stencils(spm2_problem P, double *alpha_host, double *beta_host, double *sv_host)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    if (alpha_host) memcpy(alpha_host, P->alpha_h.data(), sizeof(double) * P->alpha_h.size());
    if (beta_host) memcpy(beta_host, P->beta_h.data(), sizeof(double) * P->beta_h.size());
    if (sv_host) memcpy(sv_host, P->sv_h.data(), sizeof(double) * P->sv_h.size());
    return SPM_OK;
}

extern "C" spm_status spm2_apply_S(spm2_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, prec, x, y, nrhs));
    if (!P->have_S) { spm_set_error("S not assembled"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    return spm2_apply_S_impl(P, prec, x, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm2_factor_S(spm2_problem P, spm_prec prec)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64 && prec != SPM_C64H) { spm_set_error("bad factor precision"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_S) { spm_set_error("S not assembled"); return SPM_ERR_NOT_BUILT; }
    return spm_nd_factor(sys2_of(P), prec);
}

extern "C" spm_status spm2_factor_info(spm2_problem P, spm_prec prec, spm_factor_report *out)
{
    if (!P || !out) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    const int fi = prec == SPM_C128 ? 0 : 1;
    if (!(fi == 0 ? P->fac128 : P->fac64)) { spm_set_error("no factor in that precision"); return SPM_ERR_NOT_BUILT; }
    const spm_problem_s::FactorInfo &f = P->fac_info[fi];
    out->variant = f.variant;
    out->attempts = f.attempts;
    out->half_store = f.half_store ? 1 : 0;
    out->raised_pivots = f.raised_pivots;
    out->probe_relres = f.probe_relres;
    out->stored_bytes = (long long)f.stored_bytes;
    return SPM_OK;
}

extern "C" spm_status spm2_solve_S(spm2_problem P, spm_prec prec, const void *b, void *x, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, prec, b, x, nrhs));
    NDFactor *F = prec == SPM_C128 ? P->fac128 : P->fac64;
    if (!F) { spm_set_error("no factor of S in that precision (spm2_factor_S)"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    return spm_nd_solve(F, prec, b, x, nrhs, as_stream(stream));
}

extern "C" spm_status spm2_rhs_from_incident(spm2_problem P, const void *einc, void *g, int nrhs, void *stream)
{
    SPM_TRY(check_io(P, SPM_C128, einc, g, nrhs));
    if (nrhs == 0) return SPM_OK;
    cudaStream_t s = as_stream(stream);
    SPM_TRY(spm2_apply_A_impl(P, SPM_C128, einc, g, nrhs, s));
    return spm_axpby_impl(SPM_C128, 2L * P->n * P->n * nrhs, 1.0, einc, -1.0, g, s);
}

extern "C" spm_status spm2_solve(spm2_problem P, spm_prec prec, const void *g, void *x, int nrhs, double tol, int maxit,
                                 int restart, spm_solve_info *info)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64 && prec != SPM_MIXED) { spm_set_error("bad solve precision"); return SPM_ERR_INVALID_ARG; }
    if (nrhs < 1 || nrhs > 65535 || !g || !x || g == x) { spm_set_error("bad right-hand sides"); return SPM_ERR_INVALID_ARG; }
    if (!(tol > 0.0) || maxit < 1) { spm_set_error("tol must be positive and maxit >= 1"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_S) { spm_set_error("stencils not built (spm2_build_stencils)"); return SPM_ERR_NOT_BUILT; }
    const bool inner64 = prec != SPM_C128;
    if ((inner64 && !P->fac64) || (!inner64 && !P->fac128)) {
        spm_set_error("no factor of S in the %s precision (spm2_factor_S)", inner64 ? "complex64" : "complex128");
        return SPM_ERR_NOT_BUILT;
    }
    if (restart <= 0) restart = 20;
    KrylovOps ops;
    ops.N = 2L * P->n * P->n;
    ops.stream = P->stream;
    ops.ws = &P->gmres_ws;
    ops.ctx = P;
    ops.apply_A = ops2_A;
    ops.apply_Q = ops2_Q;
    ops.solve_S = ops2_S;
    spm_solve_info local{};
    spm_solve_info *inf = info ? info : &local;
    cudaEvent_t e0, e1;
    SPM_CUDA_TRY(cudaEventCreate(&e0));
    SPM_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, P->stream);
    spm_status st = spm_gmres_solve(ops, prec, g, x, nrhs, tol, maxit, restart, inf);
    cudaEventRecord(e1, P->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    inf->solve_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
