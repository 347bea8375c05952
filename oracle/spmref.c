/*
 * spmref.c -- plain FP64 CPU oracle for the sparsifying-preconditioned Maxwell
 * volume integral equation (Liu & Ying, "Sparsifying preconditioner for the
 * time-harmonic Maxwell's equations").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the library never does,
 * and the two share no code, headers or tables.
 *
 * Every routine follows the paper's definitions in its own notation:
 *   grid (Section 2): n points per dimension, h = 1/(n+1), node i*h, i in {1..n}^3
 *   contrast m = 1 - eps (eps complex, eps0 = 1), p^d = (d m/d x_d)/(1-m) = -d_d eps/eps
 *   Eq. (discrete):  E^d_i + k^2 sum_j G_ij m_j E^d_j + sum_j G^d_ij (p.E)_j = g^d_i
 *   Toeplitz entries G_ij = h^3 G(ih - jh) off the diagonal, G(x) = e^{ik|x|}/(4 pi |x|),
 *   G^d = dG/dx_d, with a fourth-order correction near the diagonal.
 * The paper does not print the correction weights; the reading used here is a
 * locally corrected trapezoidal rule whose single lattice constant is
 * Z = sum'_{j in Z^3} |j|^{-1} (analytically continued):
 *   G_0      = h^2/(4 pi) * (i k h - Z)          (1/r singularity, h^2 term removed)
 *   G^d_{+-e_d} += +-h Z/(24 pi)                  (-x_d/r^3 singularity, h^2 term removed)
 * All other entries are the plain kernel values.  "order 2" drops both corrections
 * (punctured trapezoidal rule, G_0 = h^3 i k/(4 pi)).
 *
 * Layouts: scalar grid arrays [i3][i2][i1] (i1 fastest, 0-based index i-1);
 * vector fields [d][i3][i2][i1]; several right-hand sides are stacked outermost.
 */
#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
#define PI 3.14159265358979323846264338327950288

/* ===================================================================== */
/* Quadrature helpers                                                     */
/* ===================================================================== */

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_m. */
static void gauss_legendre(int m, double *x, double *w)
{
    for (int i = 0; i < (m + 1) / 2; ++i) {
        double z = cos(PI * (i + 0.75) / (m + 0.5));
        double p1 = 0, p2 = 0, pp = 0;
        for (int it = 0; it < 200; ++it) {
            p1 = 1.0; p2 = 0.0;
            for (int j = 1; j <= m; ++j) {
                double p3 = p2; p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = m * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        p1 = 1.0; p2 = 0.0;
        for (int j = 1; j <= m; ++j) {
            double p3 = p2; p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = m * (z * p1 - p2) / (z * z - 1.0);
        x[i] = -z; x[m - 1 - i] = z;
        w[i] = w[m - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

typedef double (*real_fn)(double t, void *ctx);

static double integrate(real_fn f, void *ctx, double a, double b, int panels)
{
    enum { Q = 20 };
    double x[Q], w[Q];
    gauss_legendre(Q, x, w);
    double hp = (b - a) / panels, s = 0.0;
    for (int p = 0; p < panels; ++p) {
        double c = a + (p + 0.5) * hp, r = 0.5 * hp;
        for (int q = 0; q < Q; ++q) s += w[q] * r * f(c + r * x[q], ctx);
    }
    return s;
}

/* ===================================================================== */
/* Lattice sum Z(s) = sum'_{j in Z^3} |j|^{-2s}, analytically continued.   */
/* Mellin form: Gamma(s) Z(s) = int_0^inf t^{s-1} (theta(t)^3 - 1) dt with */
/* theta(t) = sum_m e^{-t m^2}; the part on (0,1) is continued through     */
/* Poisson summation theta(t) = sqrt(pi/t) theta(pi^2/t).                  */
/* ===================================================================== */

static double theta_minus_one(double t)
{
    double s = 0.0;
    for (int m = 1; m < 100000; ++m) {
        double e = exp(-t * (double)m * m);
        s += 2.0 * e;
        if (e < 1e-300 || e < 1e-22 * s) break;
    }
    return s;
}

static double cube_minus_one(double q) { return 3.0 * q + 3.0 * q * q + q * q * q; }

static double zeta_far(double t, void *ctx)
{
    double s = *(double *)ctx;
    return pow(t, s - 1.0) * cube_minus_one(theta_minus_one(t));
}

static double zeta_near(double t, void *ctx)
{
    double s = *(double *)ctx;
    return pow(t, s - 1.0) * pow(PI / t, 1.5) * cube_minus_one(theta_minus_one(PI * PI / t));
}

double spmref_lattice_zeta(double s)
{
    double lam = pow(PI, 1.5) / (s - 1.5) - 1.0 / s;
    lam += integrate(zeta_near, &s, 0.02, 1.0, 200);
    lam += integrate(zeta_far, &s, 1.0, 80.0, 400);
    return lam / tgamma(s);
}

static double zhalf_cache = 0.0;
static int zhalf_ready = 0;

static double zhalf(void)
{
    if (!zhalf_ready) { zhalf_cache = spmref_lattice_zeta(0.5); zhalf_ready = 1; }
    return zhalf_cache;
}

/* ===================================================================== */
/* Toeplitz entries G_t, G^1_t, G^2_t, G^3_t at integer offset t.          */
/* ===================================================================== */

static void kernel_entry(int t1, int t2, int t3, double h, double k, int quad, cplx out[4])
{
    if (t1 == 0 && t2 == 0 && t3 == 0) {
        double z = (quad == 0) ? zhalf() : 0.0;
        out[0] = h * h / (4.0 * PI) * (I * k * h - z);
        out[1] = out[2] = out[3] = 0.0;
        return;
    }
    double x[3] = {t1 * h, t2 * h, t3 * h};
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    cplx e = cexp(I * k * r);
    double h3 = h * h * h;
    out[0] = h3 * e / (4.0 * PI * r);
    for (int d = 0; d < 3; ++d)
        out[1 + d] = h3 * x[d] * (I * k * r - 1.0) * e / (4.0 * PI * r * r * r);
    if (quad == 0) {
        int t[3] = {t1, t2, t3};
        for (int d = 0; d < 3; ++d) {
            int others = 0;
            for (int e2 = 0; e2 < 3; ++e2) if (e2 != d && t[e2] != 0) others = 1;
            if (!others && (t[d] == 1 || t[d] == -1))
                out[1 + d] += t[d] * h * zhalf() / (24.0 * PI);
        }
    }
}

/* Table of all offsets t in [-(n-1), n-1]^3: out[kern][t3][t2][t1], kern = G,G1,G2,G3. */
void spmref_kernel_entries(int n, double k, int quad, cplx *out)
{
    int W = 2 * n - 1;
    long W3 = (long)W * W * W;
    double h = 1.0 / (n + 1);
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b)
            for (int c = 0; c < W; ++c) {
                cplx v[4];
                kernel_entry(c - (n - 1), b - (n - 1), a - (n - 1), h, k, quad, v);
                long idx = ((long)a * W + b) * W + c;
                for (int q = 0; q < 4; ++q) out[q * W3 + idx] = v[q];
            }
}

typedef struct {
    int n, W;
    cplx *tab; /* 4 x W^3 */
} entries_t;

static entries_t make_entries(int n, double k, int quad)
{
    entries_t e;
    e.n = n; e.W = 2 * n - 1;
    e.tab = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)e.W * e.W * e.W);
    spmref_kernel_entries(n, k, quad, e.tab);
    return e;
}

static inline cplx entry(const entries_t *e, int q, int t1, int t2, int t3)
{
    long W = e->W;
    long idx = ((long)(t3 + e->n - 1) * W + (t2 + e->n - 1)) * W + (t1 + e->n - 1);
    return e->tab[(long)q * W * W * W + idx];
}

/* ===================================================================== */
/* Medium: m = 1 - eps, p^d = (d_d m)/(1 - m) = -d_d eps / eps.            */
/* ===================================================================== */

void spmref_medium(int n, const cplx *eps, const cplx *grad_eps, cplx *m, cplx *p)
{
    long N = (long)n * n * n;
    for (long i = 0; i < N; ++i) {
        m[i] = 1.0 - eps[i];
        for (int d = 0; d < 3; ++d) p[d * N + i] = -grad_eps[d * N + i] / eps[i];
    }
}

/* ===================================================================== */
/* Direct O(N^2) apply of Eq. (discrete): y = A x.                        */
/* ===================================================================== */

void spmref_apply_direct(int n, double k, int quad, const cplx *m, const cplx *p,
                         const cplx *x, cplx *y)
{
    long N = (long)n * n * n;
    entries_t e = make_entries(n, k, quad);
    cplx *w = (cplx *)malloc(sizeof(cplx) * 4 * N);
    for (long j = 0; j < N; ++j) {
        for (int d = 0; d < 3; ++d) w[d * N + j] = m[j] * x[d * N + j];
        w[3 * N + j] = p[j] * x[j] + p[N + j] * x[N + j] + p[2 * N + j] * x[2 * N + j];
    }
    double k2 = k * k;
#pragma omp parallel for schedule(dynamic)
    for (long i = 0; i < N; ++i) {
        int i1 = i % n, i2 = (i / n) % n, i3 = i / ((long)n * n);
        cplx acc[3] = {0, 0, 0};
        for (long j = 0; j < N; ++j) {
            int j1 = j % n, j2 = (j / n) % n, j3 = j / ((long)n * n);
            int t1 = i1 - j1, t2 = i2 - j2, t3 = i3 - j3;
            cplx g = entry(&e, 0, t1, t2, t3);
            for (int d = 0; d < 3; ++d)
                acc[d] += k2 * g * w[d * N + j] + entry(&e, 1 + d, t1, t2, t3) * w[3 * N + j];
        }
        for (int d = 0; d < 3; ++d) y[d * N + i] = x[d * N + i] + acc[d];
    }
    free(w);
    free(e.tab);
}

/* (A x) at selected points only: the same direct sum of Eq. (discrete) as
   spmref_apply_direct, term for term and in the same order, with each kernel
   entry evaluated when it is needed instead of from the full (2n-1)^3 table
   (for large n, where the table and the full O(N^2) sum are out of reach).
   idx: npts linear point indices (i1 fastest); out: npts x 3. */
void spmref_apply_direct_points(int n, double k, int quad, const cplx *m, const cplx *p, const cplx *x,
                                int npts, const long *idx, cplx *out)
{
    long N = (long)n * n * n;
    double h = 1.0 / (n + 1), k2 = k * k;
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < npts; ++s) {
        long i = idx[s];
        int i1 = i % n, i2 = (i / n) % n, i3 = i / ((long)n * n);
        cplx acc[3] = {0, 0, 0};
        for (long j = 0; j < N; ++j) {
            int j1 = j % n, j2 = (j / n) % n, j3 = j / ((long)n * n);
            cplx v[4];
            kernel_entry(i1 - j1, i2 - j2, i3 - j3, h, k, quad, v);
            cplx w4 = p[j] * x[j] + p[N + j] * x[N + j] + p[2 * N + j] * x[2 * N + j];
            for (int d = 0; d < 3; ++d) acc[d] += k2 * v[0] * (m[j] * x[d * N + j]) + v[1 + d] * w4;
        }
        for (int d = 0; d < 3; ++d) out[3 * s + d] = x[d * N + i] + acc[d];
    }
}

/* ===================================================================== */
/* Radix-2 FFT (iterative Cooley-Tukey) and 3-D transforms.               */
/* ===================================================================== */

static void fft1d(cplx *a, int L, int sign)
{
    for (int i = 1, j = 0; i < L; ++i) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= L; len <<= 1) {
        double ang = sign * 2.0 * PI / len;
        for (int i = 0; i < L; i += len)
            for (int j = 0; j < len / 2; ++j) {
                cplx w = cexp(I * ang * j);
                cplx u = a[i + j], v = a[i + j + len / 2] * w;
                a[i + j] = u + v;
                a[i + j + len / 2] = u - v;
            }
    }
}

/* In-place 3-D DFT of an L^3 array [z][y][x]; sign -1 forward, +1 inverse (unscaled). */
static void fft3d(cplx *a, int L, int sign)
{
    long L2 = (long)L * L;
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * L);
#pragma omp for
        for (long r = 0; r < L2; ++r) fft1d(a + r * L, L, sign);
#pragma omp for
        for (long r = 0; r < L2; ++r) {
            long z = r / L, x = r % L;
            for (int y = 0; y < L; ++y) line[y] = a[z * L2 + (long)y * L + x];
            fft1d(line, L, sign);
            for (int y = 0; y < L; ++y) a[z * L2 + (long)y * L + x] = line[y];
        }
#pragma omp for
        for (long r = 0; r < L2; ++r) {
            for (int z = 0; z < L; ++z) line[z] = a[z * L2 + r];
            fft1d(line, L, sign);
            for (int z = 0; z < L; ++z) a[z * L2 + r] = line[z];
        }
        free(line);
    }
}

static int pow2_at_least(int v)
{
    int L = 1;
    while (L < v) L <<= 1;
    return L;
}

/* Spectra of the circulant embeddings of the four Toeplitz kernels (length L >= 2n-1). */
static cplx *kernel_spectra(int n, double k, int quad, int L)
{
    long L3 = (long)L * L * L;
    cplx *spec = (cplx *)calloc(4 * L3, sizeof(cplx));
    entries_t e = make_entries(n, k, quad);
    for (int t3 = -(n - 1); t3 <= n - 1; ++t3)
        for (int t2 = -(n - 1); t2 <= n - 1; ++t2)
            for (int t1 = -(n - 1); t1 <= n - 1; ++t1) {
                long idx = (((long)((t3 + L) % L) * L) + (t2 + L) % L) * L + (t1 + L) % L;
                for (int q = 0; q < 4; ++q) spec[q * L3 + idx] = entry(&e, q, t1, t2, t3);
            }
    free(e.tab);
    for (int q = 0; q < 4; ++q) fft3d(spec + q * L3, L, -1);
    return spec;
}

/* FFT apply of Eq. (discrete_block).  A context holds the kernel spectra so
   repeated applies do not recompute them. */
typedef struct {
    int n, L;
    double k;
    cplx *spec; /* 4 x L^3 */
    cplx *work; /* 4 x L^3 */
} fft_ctx_t;

void *spmref_fft_create(int n, double k, int quad)
{
    fft_ctx_t *c = (fft_ctx_t *)calloc(1, sizeof(fft_ctx_t));
    c->n = n; c->k = k;
    c->L = pow2_at_least(2 * n);
    c->spec = kernel_spectra(n, k, quad, c->L);
    c->work = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)c->L * c->L * c->L);
    return c;
}

void spmref_fft_free(void *h)
{
    fft_ctx_t *c = (fft_ctx_t *)h;
    if (!c) return;
    free(c->spec); free(c->work); free(c);
}

void spmref_fft_apply(void *h, const cplx *m, const cplx *p, const cplx *x, cplx *y, int nrhs)
{
    fft_ctx_t *c = (fft_ctx_t *)h;
    int n = c->n, L = c->L;
    long N = (long)n * n * n;
    long L3 = (long)L * L * L;
    cplx *spec = c->spec, *w = c->work;
    double k2 = c->k * c->k;
    for (int b = 0; b < nrhs; ++b) {
        const cplx *xb = x + (long)b * 3 * N;
        cplx *yb = y + (long)b * 3 * N;
        memset(w, 0, sizeof(cplx) * 4 * L3);
        for (int i3 = 0; i3 < n; ++i3)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i1 = 0; i1 < n; ++i1) {
                    long j = ((long)i3 * n + i2) * n + i1;
                    long J = ((long)i3 * L + i2) * L + i1;
                    for (int d = 0; d < 3; ++d) w[d * L3 + J] = m[j] * xb[d * N + j];
                    w[3 * L3 + J] = p[j] * xb[j] + p[N + j] * xb[N + j] + p[2 * N + j] * xb[2 * N + j];
                }
        for (int q = 0; q < 4; ++q) fft3d(w + q * L3, L, -1);
#pragma omp parallel for
        for (long J = 0; J < L3; ++J) {
            cplx w4 = w[3 * L3 + J];
            for (int d = 0; d < 3; ++d)
                w[d * L3 + J] = k2 * spec[J] * w[d * L3 + J] + spec[(1 + d) * L3 + J] * w4;
        }
        for (int d = 0; d < 3; ++d) fft3d(w + d * L3, L, +1);
        for (int i3 = 0; i3 < n; ++i3)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i1 = 0; i1 < n; ++i1) {
                    long j = ((long)i3 * n + i2) * n + i1;
                    long J = ((long)i3 * L + i2) * L + i1;
                    for (int d = 0; d < 3; ++d) yb[d * N + j] = xb[d * N + j] + w[d * L3 + J] / (double)L3;
                }
    }
}

void spmref_apply_fft(int n, double k, int quad, const cplx *m, const cplx *p,
                      const cplx *x, cplx *y, int nrhs)
{
    void *c = spmref_fft_create(n, k, quad);
    spmref_fft_apply(c, m, p, x, y, nrhs);
    spmref_fft_free(c);
}

/* Discrete convolution with one kernel (0: G, 1..3: G^d) of a scalar grid function. */
void spmref_convolve(int n, double k, int quad, int which, const cplx *f, cplx *out)
{
    long N = (long)n * n * n;
    int L = pow2_at_least(2 * n);
    long L3 = (long)L * L * L;
    cplx *spec = kernel_spectra(n, k, quad, L);
    cplx *w = (cplx *)calloc(L3, sizeof(cplx));
    for (int i3 = 0; i3 < n; ++i3)
        for (int i2 = 0; i2 < n; ++i2)
            for (int i1 = 0; i1 < n; ++i1)
                w[((long)i3 * L + i2) * L + i1] = f[((long)i3 * n + i2) * n + i1];
    fft3d(w, L, -1);
    for (long J = 0; J < L3; ++J) w[J] *= spec[which * L3 + J];
    fft3d(w, L, +1);
    for (int i3 = 0; i3 < n; ++i3)
        for (int i2 = 0; i2 < n; ++i2)
            for (int i1 = 0; i1 < n; ++i1)
                out[((long)i3 * n + i2) * n + i1] = w[((long)i3 * L + i2) * L + i1] / (double)L3;
    (void)N;
    free(w);
    free(spec);
}

/* ===================================================================== */
/* Point classes and their neighbourhoods (Section 3.2).                  */
/* class = c1 + 3 c2 + 9 c3 with c_d = 0 (i_d = 1), 1 (interior), 2 (i_d=n)*/
/* tau offsets per dimension: {0,1}, {-1,0,1}, {-1,0}; the enlarged        */
/* complement ranges: [0,n-1], [-(n-2),n-2], [-(n-1),0], minus tau.        */
/* Offsets are enumerated o3 outer, o2, o1 inner, each ascending.          */
/* ===================================================================== */

static void class_dims(int cls, int c[3])
{
    c[0] = cls % 3; c[1] = (cls / 3) % 3; c[2] = cls / 9;
}

static void tau_range(int c, int *lo, int *hi)
{
    if (c == 0) { *lo = 0; *hi = 1; }
    else if (c == 1) { *lo = -1; *hi = 1; }
    else { *lo = -1; *hi = 0; }
}

static void comp_range(int n, int c, int *lo, int *hi)
{
    if (c == 0) { *lo = 0; *hi = n - 1; }
    else if (c == 1) { *lo = -(n - 2); *hi = n - 2; }
    else { *lo = -(n - 1); *hi = 0; }
}

int spmref_class_tau(int cls, int *offs)
{
    int c[3], lo[3], hi[3], T = 0;
    class_dims(cls, c);
    for (int d = 0; d < 3; ++d) tau_range(c[d], &lo[d], &hi[d]);
    for (int o3 = lo[2]; o3 <= hi[2]; ++o3)
        for (int o2 = lo[1]; o2 <= hi[1]; ++o2)
            for (int o1 = lo[0]; o1 <= hi[0]; ++o1) {
                if (offs) { offs[3 * T] = o1; offs[3 * T + 1] = o2; offs[3 * T + 2] = o3; }
                ++T;
            }
    return T;
}

static int in_tau(int cls, int u1, int u2, int u3)
{
    int c[3], u[3] = {u1, u2, u3};
    class_dims(cls, c);
    for (int d = 0; d < 3; ++d) {
        int lo, hi;
        tau_range(c[d], &lo, &hi);
        if (u[d] < lo || u[d] > hi) return 0;
    }
    return 1;
}

/* Householder QR of a column-major (rows x cols) complex matrix; leaves R in the top. */
static void householder_qr(cplx *A, long rows, int cols, long lda)
{
    for (int j = 0; j < cols && j < rows; ++j) {
        cplx *col = A + (long)j * lda;
        double nrm2 = 0.0;
        for (long r = j; r < rows; ++r) nrm2 += creal(col[r] * conj(col[r]));
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) continue;
        cplx x0 = col[j];
        cplx phase = (cabs(x0) > 0) ? x0 / cabs(x0) : 1.0;
        cplx alpha = -phase * nrm;
        /* v = x - alpha e1, stored in place of the column below the diagonal */
        col[j] = x0 - alpha;
        double vn2 = nrm2 - creal(x0 * conj(x0)) + creal((x0 - alpha) * conj(x0 - alpha));
        if (vn2 == 0.0) { col[j] = alpha; continue; }
        for (int c = j + 1; c < cols; ++c) {
            cplx *cc = A + (long)c * lda;
            cplx dot = 0.0;
            for (long r = j; r < rows; ++r) dot += conj(col[r]) * cc[r];
            cplx f = 2.0 * dot / vn2;
            for (long r = j; r < rows; ++r) cc[r] -= f * col[r];
        }
        col[j] = alpha;
        for (long r = j + 1; r < rows; ++r) col[r] = 0.0;
    }
}

/* One-sided (Hestenes) Jacobi on the columns of a C x C column-major R:
   R V = W Sigma; returns V (column-major) and sigma (column norms). */
static void one_sided_jacobi(cplx *R, int C, cplx *V, double *sigma)
{
    for (int i = 0; i < C * C; ++i) V[i] = 0.0;
    for (int i = 0; i < C; ++i) V[(long)i * C + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < C - 1; ++p)
            for (int q = p + 1; q < C; ++q) {
                cplx *cp = R + (long)p * C, *cq = R + (long)q * C;
                double a = 0, b = 0;
                cplx g = 0;
                for (int r = 0; r < C; ++r) {
                    a += creal(cp[r] * conj(cp[r]));
                    b += creal(cq[r] * conj(cq[r]));
                    g += conj(cp[r]) * cq[r];
                }
                double ag = cabs(g);
                if (ag == 0.0 || ag <= 1e-15 * sqrt(a * b)) continue;
                double rel = ag / sqrt(a * b);
                if (rel > off) off = rel;
                cplx ph = conj(g) / ag; /* multiplies column q so that g becomes real */
                double zeta = (b - a) / (2.0 * ag);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                cplx *vp = V + (long)p * C, *vq = V + (long)q * C;
                for (int r = 0; r < C; ++r) {
                    cplx xp = cp[r], xq = ph * cq[r];
                    cp[r] = cs * xp - sn * xq;
                    cq[r] = sn * xp + cs * xq;
                    cplx yp = vp[r], yq = ph * vq[r];
                    vp[r] = cs * yp - sn * yq;
                    vq[r] = sn * yp + cs * yq;
                }
            }
        if (off < 1e-15) break;
    }
    for (int j = 0; j < C; ++j) {
        double s = 0;
        for (int r = 0; r < C; ++r) s += creal(R[(long)j * C + r] * conj(R[(long)j * C + r]));
        sigma[j] = sqrt(s);
    }
}

/* Stencils of one class: alpha (3T x 3, row (d,o) = d*T+o), beta = B^T alpha
   (4T x 3), and all 3T singular values of M in ascending order.
   alpha = conj(three left singular vectors of M with the smallest singular
   values), M the off-neighbourhood block of the paper's minimisation.        */
int spmref_class_stencil(int n, double k, int quad, int cls,
                         cplx *alpha, cplx *beta, double *sv)
{
    int offs[27 * 3];
    int T = spmref_class_tau(cls, offs);
    int C = 3 * T;
    int c[3], lo[3], hi[3];
    class_dims(cls, c);
    for (int d = 0; d < 3; ++d) comp_range(n, c[d], &lo[d], &hi[d]);
    entries_t e = make_entries(n, k, quad);
    double k2 = k * k;

    const long B = 2048;
    long rows = C + B;
    cplx *A = (cplx *)malloc(sizeof(cplx) * rows * C); /* column-major, lda = rows */
    cplx *Rk = (cplx *)calloc((size_t)C * C, sizeof(cplx));
    long filled = 0;
    /* enumerate the columns (f,u) of M; each gives one row of M^H */
    for (int u3 = lo[2]; u3 <= hi[2]; ++u3)
        for (int u2 = lo[1]; u2 <= hi[1]; ++u2)
            for (int u1 = lo[0]; u1 <= hi[0]; ++u1) {
                if (in_tau(cls, u1, u2, u3)) continue;
                for (int f = 0; f < 4; ++f) {
                    long r = C + filled;
                    for (int col = 0; col < C; ++col) A[(long)col * rows + r] = 0.0;
                    for (int o = 0; o < T; ++o) {
                        int v1 = offs[3 * o] - u1, v2 = offs[3 * o + 1] - u2, v3 = offs[3 * o + 2] - u3;
                        if (f < 3) {
                            A[(long)(f * T + o) * rows + r] = conj(k2 * entry(&e, 0, v1, v2, v3));
                        } else {
                            for (int d = 0; d < 3; ++d)
                                A[(long)(d * T + o) * rows + r] = conj(entry(&e, 1 + d, v1, v2, v3));
                        }
                    }
                    ++filled;
                    if (filled == B) {
                        for (int col = 0; col < C; ++col)
                            for (int r2 = 0; r2 < C; ++r2) A[(long)col * rows + r2] = Rk[(long)col * C + r2];
                        householder_qr(A, rows, C, rows);
                        for (int col = 0; col < C; ++col)
                            for (int r2 = 0; r2 < C; ++r2)
                                Rk[(long)col * C + r2] = (r2 <= col) ? A[(long)col * rows + r2] : 0.0;
                        filled = 0;
                    }
                }
            }
    if (filled > 0) {
        long rr = C + filled;
        cplx *A2 = (cplx *)malloc(sizeof(cplx) * rr * C);
        for (int col = 0; col < C; ++col) {
            for (int r2 = 0; r2 < C; ++r2) A2[(long)col * rr + r2] = Rk[(long)col * C + r2];
            for (long r2 = 0; r2 < filled; ++r2) A2[(long)col * rr + C + r2] = A[(long)col * rows + C + r2];
        }
        householder_qr(A2, rr, C, rr);
        for (int col = 0; col < C; ++col)
            for (int r2 = 0; r2 < C; ++r2)
                Rk[(long)col * C + r2] = (r2 <= col) ? A2[(long)col * rr + r2] : 0.0;
        free(A2);
    }
    free(A);

    /* M = R^H Q^H: left singular vectors of M = right singular vectors of R. */
    cplx *V = (cplx *)malloc(sizeof(cplx) * C * C);
    double *sig = (double *)malloc(sizeof(double) * C);
    one_sided_jacobi(Rk, C, V, sig);
    int *idx = (int *)malloc(sizeof(int) * C);
    for (int i = 0; i < C; ++i) idx[i] = i;
    for (int i = 1; i < C; ++i) {
        int v = idx[i], j = i - 1;
        while (j >= 0 && sig[idx[j]] > sig[v]) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = v;
    }
    if (sv) for (int i = 0; i < C; ++i) sv[i] = sig[idx[i]];
    for (int col = 0; col < 3; ++col)
        for (int r = 0; r < C; ++r) alpha[r * 3 + col] = conj(V[(long)idx[col] * C + r]);

    /* beta = B^T alpha with B the in-neighbourhood block (Eq. alphabeta). */
    for (int col = 0; col < 3; ++col)
        for (int f = 0; f < 4; ++f)
            for (int op = 0; op < T; ++op) {
                cplx s = 0.0;
                for (int o = 0; o < T; ++o) {
                    int v1 = offs[3 * o] - offs[3 * op], v2 = offs[3 * o + 1] - offs[3 * op + 1],
                        v3 = offs[3 * o + 2] - offs[3 * op + 2];
                    if (f < 3) s += k2 * entry(&e, 0, v1, v2, v3) * alpha[(f * T + o) * 3 + col];
                    else
                        for (int d = 0; d < 3; ++d) s += entry(&e, 1 + d, v1, v2, v3) * alpha[(d * T + o) * 3 + col];
                }
                beta[(f * T + op) * 3 + col] = s;
            }
    free(idx); free(sig); free(V); free(Rk); free(e.tab);
    return T;
}

static int point_class(int n, int i1, int i2, int i3) /* 0-based indices */
{
    int ii[3] = {i1, i2, i3}, c = 0, mul = 1;
    for (int d = 0; d < 3; ++d) {
        int cd = (ii[d] == 0) ? 0 : (ii[d] == n - 1 ? 2 : 1);
        c += cd * mul;
        mul *= 3;
    }
    return c;
}

/* Q v: y_{i,c} = sum_{(d,o) in class tau} alpha_cls[(d,o),c] v^d_{i+o}.
   alpha_all is packed [27][81][3] (rows d*T+o of the class, T = class size). */
void spmref_apply_Q(int n, const cplx *alpha_all, const cplx *v, cplx *y, int nrhs)
{
    long N = (long)n * n * n;
    for (int b = 0; b < nrhs; ++b) {
        const cplx *vb = v + (long)b * 3 * N;
        cplx *yb = y + (long)b * 3 * N;
        for (int i3 = 0; i3 < n; ++i3)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i1 = 0; i1 < n; ++i1) {
                    int cls = point_class(n, i1, i2, i3);
                    int offs[81];
                    int T = spmref_class_tau(cls, offs);
                    const cplx *al = alpha_all + (long)cls * 81 * 3;
                    long i = ((long)i3 * n + i2) * n + i1;
                    for (int c = 0; c < 3; ++c) {
                        cplx s = 0.0;
                        for (int d = 0; d < 3; ++d)
                            for (int o = 0; o < T; ++o) {
                                long j = ((long)(i3 + offs[3 * o + 2]) * n + (i2 + offs[3 * o + 1])) * n + (i1 + offs[3 * o]);
                                s += al[(d * T + o) * 3 + c] * vb[d * N + j];
                            }
                        yb[c * N + i] = s;
                    }
                }
    }
}

/* ===================================================================== */
/* Dense operators for brute-force checks on tiny grids.                  */
/* Unknown (d, i) has index d*N + i.                                      */
/* ===================================================================== */

void spmref_dense_A(int n, double k, int quad, const cplx *m, const cplx *p, cplx *A)
{
    long N = (long)n * n * n, M3 = 3 * N;
    entries_t e = make_entries(n, k, quad);
    double k2 = k * k;
    for (long i = 0; i < N; ++i) {
        int i1 = i % n, i2 = (i / n) % n, i3 = i / ((long)n * n);
        for (long j = 0; j < N; ++j) {
            int j1 = j % n, j2 = (j / n) % n, j3 = j / ((long)n * n);
            int t1 = i1 - j1, t2 = i2 - j2, t3 = i3 - j3;
            cplx g = entry(&e, 0, t1, t2, t3);
            for (int d = 0; d < 3; ++d) {
                cplx gd = entry(&e, 1 + d, t1, t2, t3);
                for (int f = 0; f < 3; ++f) {
                    cplx v = gd * p[f * N + j];
                    if (f == d) v += k2 * g * m[j] + (i == j ? 1.0 : 0.0);
                    A[(d * N + i) * M3 + f * N + j] = v;
                }
            }
        }
    }
    free(e.tab);
}

/* S row (i,c), column (f,j), j in tau_i:
   alpha[(f,o),c] + beta[(f,o),c] m_j + beta[(3,o),c] p^f_j, o = j - i (Eq. nbr_i_block_alpha_approx). */
void spmref_dense_S(int n, const cplx *m, const cplx *p, const cplx *alpha_all, const cplx *beta_all, cplx *S)
{
    long N = (long)n * n * n, M3 = 3 * N;
    memset(S, 0, sizeof(cplx) * M3 * M3);
    for (int i3 = 0; i3 < n; ++i3)
        for (int i2 = 0; i2 < n; ++i2)
            for (int i1 = 0; i1 < n; ++i1) {
                int cls = point_class(n, i1, i2, i3);
                int offs[81];
                int T = spmref_class_tau(cls, offs);
                const cplx *al = alpha_all + (long)cls * 81 * 3;
                const cplx *be = beta_all + (long)cls * 108 * 3;
                long i = ((long)i3 * n + i2) * n + i1;
                for (int o = 0; o < T; ++o) {
                    long j = ((long)(i3 + offs[3 * o + 2]) * n + (i2 + offs[3 * o + 1])) * n + (i1 + offs[3 * o]);
                    for (int c = 0; c < 3; ++c)
                        for (int f = 0; f < 3; ++f)
                            S[(c * N + i) * M3 + f * N + j] =
                                al[(f * T + o) * 3 + c] + be[(f * T + o) * 3 + c] * m[j] + be[(3 * T + o) * 3 + c] * p[f * N + j];
                }
            }
}

/* Dense LU with partial pivoting; solves A X = B in place (B is N x nrhs row-major). */
int spmref_dense_solve(long N, cplx *A, cplx *B, int nrhs)
{
    for (long c = 0; c < N; ++c) {
        long piv = c;
        double best = cabs(A[c * N + c]);
        for (long r = c + 1; r < N; ++r)
            if (cabs(A[r * N + c]) > best) { best = cabs(A[r * N + c]); piv = r; }
        if (best == 0.0) return 1;
        if (piv != c) {
            for (long j = 0; j < N; ++j) { cplx t = A[c * N + j]; A[c * N + j] = A[piv * N + j]; A[piv * N + j] = t; }
            for (int j = 0; j < nrhs; ++j) { cplx t = B[c * nrhs + j]; B[c * nrhs + j] = B[piv * nrhs + j]; B[piv * nrhs + j] = t; }
        }
        cplx inv = 1.0 / A[c * N + c];
#pragma omp parallel for
        for (long r = c + 1; r < N; ++r) {
            cplx f = A[r * N + c] * inv;
            if (f == 0.0) continue;
            A[r * N + c] = f;
            for (long j = c + 1; j < N; ++j) A[r * N + j] -= f * A[c * N + j];
            for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[c * nrhs + j];
        }
    }
    for (long c = N - 1; c >= 0; --c) {
        for (int j = 0; j < nrhs; ++j) {
            cplx s = B[c * nrhs + j];
            for (long r = c + 1; r < N; ++r) s -= A[c * N + r] * B[r * nrhs + j];
            B[c * nrhs + j] = s / A[c * N + c];
        }
    }
    return 0;
}

/* ===================================================================== */
/* Banded LU of S (unknowns interleaved: 3*i + c) for the preconditioner. */
/* ===================================================================== */

typedef struct {
    long N;     /* 3 n^3 */
    int kl, ku; /* band widths of S */
    int ldab;   /* 2*kl + ku + 1 */
    cplx *ab;   /* LAPACK-style band storage, column-major */
    int *ipiv;
    int n;
} band_lu_t;

#define AB(bl, r, c) ((bl)->ab[(long)(c) * (bl)->ldab + (bl)->kl + (bl)->ku + (r) - (c)])

void *spmref_S_factor(int n, const cplx *m, const cplx *p, const cplx *alpha_all, const cplx *beta_all)
{
    band_lu_t *bl = (band_lu_t *)calloc(1, sizeof(band_lu_t));
    long N = (long)n * n * n;
    bl->n = n;
    bl->N = 3 * N;
    bl->kl = bl->ku = 3 * (n * n + n + 1) + 2;
    bl->ldab = 2 * bl->kl + bl->ku + 1;
    bl->ab = (cplx *)calloc((size_t)bl->ldab * bl->N, sizeof(cplx));
    bl->ipiv = (int *)malloc(sizeof(int) * bl->N);
    for (int i3 = 0; i3 < n; ++i3)
        for (int i2 = 0; i2 < n; ++i2)
            for (int i1 = 0; i1 < n; ++i1) {
                int cls = point_class(n, i1, i2, i3);
                int offs[81];
                int T = spmref_class_tau(cls, offs);
                const cplx *al = alpha_all + (long)cls * 81 * 3;
                const cplx *be = beta_all + (long)cls * 108 * 3;
                long i = ((long)i3 * n + i2) * n + i1;
                for (int o = 0; o < T; ++o) {
                    long j = ((long)(i3 + offs[3 * o + 2]) * n + (i2 + offs[3 * o + 1])) * n + (i1 + offs[3 * o]);
                    for (int c = 0; c < 3; ++c)
                        for (int f = 0; f < 3; ++f)
                            AB(bl, 3 * i + c, 3 * j + f) =
                                al[(f * T + o) * 3 + c] + be[(f * T + o) * 3 + c] * m[j] + be[(3 * T + o) * 3 + c] * p[f * N + j];
                }
            }
    /* Gaussian elimination with partial pivoting within the band (gbtf2 style). */
    long NN = bl->N;
    int kl = bl->kl, ku = bl->ku;
    for (long c = 0; c < NN; ++c) {
        long rmax = c + kl < NN - 1 ? c + kl : NN - 1;
        long piv = c;
        double best = cabs(AB(bl, c, c));
        for (long r = c + 1; r <= rmax; ++r)
            if (cabs(AB(bl, r, c)) > best) { best = cabs(AB(bl, r, c)); piv = r; }
        bl->ipiv[c] = (int)piv;
        long cmax = c + kl + ku < NN - 1 ? c + kl + ku : NN - 1;
        if (best == 0.0) continue;
        if (piv != c)
            for (long j = c; j <= cmax; ++j) { cplx t = AB(bl, c, j); AB(bl, c, j) = AB(bl, piv, j); AB(bl, piv, j) = t; }
        cplx inv = 1.0 / AB(bl, c, c);
        for (long r = c + 1; r <= rmax; ++r) AB(bl, r, c) *= inv;
#pragma omp parallel for
        for (long j = c + 1; j <= cmax; ++j) {
            cplx u = AB(bl, c, j);
            if (u == 0.0) continue;
            for (long r = c + 1; r <= rmax; ++r) AB(bl, r, j) -= AB(bl, r, c) * u;
        }
    }
    return bl;
}

/* x = S^{-1} b for vectors in the [d][i] layout. */
void spmref_S_solve(void *h, const cplx *b, cplx *x)
{
    band_lu_t *bl = (band_lu_t *)h;
    long NN = bl->N, N = NN / 3;
    int kl = bl->kl, ku = bl->ku;
    cplx *z = (cplx *)malloc(sizeof(cplx) * NN);
    for (long i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) z[3 * i + c] = b[c * N + i];
    for (long c = 0; c < NN; ++c) {
        long piv = bl->ipiv[c];
        if (piv != c) { cplx t = z[c]; z[c] = z[piv]; z[piv] = t; }
        long rmax = c + kl < NN - 1 ? c + kl : NN - 1;
        for (long r = c + 1; r <= rmax; ++r) z[r] -= AB(bl, r, c) * z[c];
    }
    for (long c = NN - 1; c >= 0; --c) {
        long cmax = c + kl + ku < NN - 1 ? c + kl + ku : NN - 1;
        cplx s = z[c];
        for (long j = c + 1; j <= cmax; ++j) s -= AB(bl, c, j) * z[j];
        z[c] = s / AB(bl, c, c);
    }
    for (long i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) x[c * N + i] = z[3 * i + c];
    free(z);
}

void spmref_S_free(void *h)
{
    band_lu_t *bl = (band_lu_t *)h;
    if (!bl) return;
    free(bl->ab); free(bl->ipiv); free(bl);
}

/* ===================================================================== */
/* GMRES (restarted, MGS Arnoldi, Givens rotations), optional left        */
/* preconditioner S^{-1} Q.  Stops on the residual of the system it       */
/* iterates on (preconditioned if a preconditioner is given).             */
/* ===================================================================== */

typedef struct {
    int n;
    void *fft;
    const cplx *m, *p;
    void *slu; const cplx *alpha_all;
} gm_ctx;

static void gm_apply(gm_ctx *c, const cplx *x, cplx *y)
{
    long NN = 3L * c->n * c->n * c->n;
    spmref_fft_apply(c->fft, c->m, c->p, x, y, 1);
    if (c->slu) {
        cplx *t = (cplx *)malloc(sizeof(cplx) * NN);
        spmref_apply_Q(c->n, c->alpha_all, y, t, 1);
        spmref_S_solve(c->slu, t, y);
        free(t);
    }
}

static void gm_precond(gm_ctx *c, const cplx *x, cplx *y)
{
    long NN = 3L * c->n * c->n * c->n;
    if (!c->slu) { memcpy(y, x, sizeof(cplx) * NN); return; }
    cplx *t = (cplx *)malloc(sizeof(cplx) * NN);
    spmref_apply_Q(c->n, c->alpha_all, x, t, 1);
    spmref_S_solve(c->slu, t, y);
    free(t);
}

static double vnorm(const cplx *v, long N)
{
    double s = 0;
    for (long i = 0; i < N; ++i) s += creal(v[i] * conj(v[i]));
    return sqrt(s);
}

int spmref_gmres(int n, double k, int quad, const cplx *m, const cplx *p,
                 const cplx *b, cplx *x, double tol, int maxit, int restart,
                 void *slu, const cplx *alpha_all, double *relres_out, double *history)
{
    gm_ctx ctx = {n, spmref_fft_create(n, k, quad), m, p, slu, alpha_all};
    long NN = 3L * n * n * n;
    int R = restart;
    cplx *V = (cplx *)malloc(sizeof(cplx) * NN * (R + 1));
    cplx *H = (cplx *)calloc((size_t)(R + 1) * R, sizeof(cplx));
    cplx *cs = (cplx *)malloc(sizeof(cplx) * R), *sn = (cplx *)malloc(sizeof(cplx) * R);
    cplx *gvec = (cplx *)malloc(sizeof(cplx) * (R + 1));
    cplx *r = (cplx *)malloc(sizeof(cplx) * NN), *t = (cplx *)malloc(sizeof(cplx) * NN);
    gm_precond(&ctx, b, r);
    double bnorm = vnorm(r, NN);
    if (bnorm == 0) bnorm = 1;
    int it = 0;
    double rel = 1.0;
    while (it < maxit) {
        /* r = P^{-1}(b - A x) */
        spmref_fft_apply(ctx.fft, m, p, x, t, 1);
        for (long i = 0; i < NN; ++i) t[i] = b[i] - t[i];
        gm_precond(&ctx, t, r);
        double beta = vnorm(r, NN);
        rel = beta / bnorm;
        if (rel <= tol) break;
        for (long i = 0; i < NN; ++i) V[i] = r[i] / beta;
        memset(gvec, 0, sizeof(cplx) * (R + 1));
        gvec[0] = beta;
        int j;
        for (j = 0; j < R && it < maxit; ++j, ++it) {
            cplx *w = V + (long)(j + 1) * NN;
            gm_apply(&ctx, V + (long)j * NN, w);
            for (int i = 0; i <= j; ++i) {
                cplx h = 0;
                for (long q = 0; q < NN; ++q) h += conj(V[(long)i * NN + q]) * w[q];
                H[i * R + j] = h;
                for (long q = 0; q < NN; ++q) w[q] -= h * V[(long)i * NN + q];
            }
            double hn = vnorm(w, NN);
            H[(j + 1) * R + j] = hn;
            if (hn > 0) for (long q = 0; q < NN; ++q) w[q] /= hn;
            for (int i = 0; i < j; ++i) {
                cplx a = H[i * R + j], bb = H[(i + 1) * R + j];
                H[i * R + j] = conj(cs[i]) * a + conj(sn[i]) * bb;
                H[(i + 1) * R + j] = -sn[i] * a + cs[i] * bb;
            }
            cplx a = H[j * R + j], bb = H[(j + 1) * R + j];
            double den = sqrt(creal(a * conj(a)) + creal(bb * conj(bb)));
            cs[j] = a / den; sn[j] = bb / den;
            H[j * R + j] = den;
            H[(j + 1) * R + j] = 0;
            gvec[j + 1] = -sn[j] * gvec[j];
            gvec[j] = conj(cs[j]) * gvec[j];
            rel = cabs(gvec[j + 1]) / bnorm;
            if (history) history[it] = rel;
            if (rel <= tol) { ++j; ++it; break; }
        }
        /* back substitution and update */
        cplx *yv = (cplx *)malloc(sizeof(cplx) * j);
        for (int i = j - 1; i >= 0; --i) {
            cplx s = gvec[i];
            for (int q = i + 1; q < j; ++q) s -= H[i * R + q] * yv[q];
            yv[i] = s / H[i * R + i];
        }
        for (int i = 0; i < j; ++i)
            for (long q = 0; q < NN; ++q) x[q] += yv[i] * V[(long)i * NN + q];
        free(yv);
        if (rel <= tol) break;
    }
    /* final residual of the iterated system */
    spmref_fft_apply(ctx.fft, m, p, x, t, 1);
    for (long i = 0; i < NN; ++i) t[i] = b[i] - t[i];
    gm_precond(&ctx, t, r);
    if (relres_out) *relres_out = vnorm(r, NN) / bnorm;
    spmref_fft_free(ctx.fft);
    free(V); free(H); free(cs); free(sn); free(gvec); free(r); free(t);
    (void)k; (void)quad;
    return it;
}

/* Thread count of the OpenMP loops above, for timing the oracle: every
   parallel loop writes disjoint outputs, so results do not depend on it. */
void spmref_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
