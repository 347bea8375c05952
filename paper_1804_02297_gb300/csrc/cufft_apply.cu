// The operator apply of Eq. discrete_block through cuFFT: a comparison point
// for the hand-written passes of apply.cu, never used by them.
//
// Same arithmetic, organised the textbook way: the four contrast-weighted
// fields w = [m E^1, m E^2, m E^3, p.E] zero-padded to full L^3 arrays, one
// batched 3-D forward FFT (cuFFT), the Fourier-side product with the four
// kernel spectra (the octant tables of the problem, expanded by the parity of
// each kernel), one batched 3-D inverse FFT, crop to the grid and add x.  The
// padded arrays (7 L^3 complex values per right-hand side at most) and cuFFT's
// plans and work area are owned by the problem and kept between calls.
#include <cufft.h>

#include "common.cuh"

namespace {

// W[f][i3][i2][i1] over L^3: w_f on [0,n)^3, zero elsewhere
template <typename C>
__global__ void k_cf_pad(const C *__restrict__ x, const C *__restrict__ m, const C *__restrict__ p, C *W, int n, int L)
{
    const long L3 = (long)L * L * L, n3 = (long)n * n * n;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= L3) return;
    const int v1 = (int)(gid % L), v2 = (int)((gid / L) % L), v3 = (int)(gid / ((long)L * L));
    C w[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) w[f] = czero<C>();
    if (v1 < n && v2 < n && v3 < n) {
        const long i = ((long)v3 * n + v2) * n + v1;
        const C e0 = x[i], e1 = x[n3 + i], e2 = x[2 * n3 + i], mm = m[i];
        w[0] = cmul(mm, e0);
        w[1] = cmul(mm, e1);
        w[2] = cmul(mm, e2);
        w[3] = cfma(p[i], e0, cfma(p[n3 + i], e1, cmul(p[2 * n3 + i], e2)));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) W[f * L3 + gid] = w[f];
}

// y_d = K0 w_d + K_d w_4 at every frequency (in place into fields 0..2);
// the octant [4][n+1]^3 holds K0 (even in every frequency) and K_d (odd in
// frequency d, even in the others) for frequencies 0..n
template <typename C>
__global__ void k_cf_product(C *W, const C *__restrict__ spec, int n, int L)
{
    const long L3 = (long)L * L * L;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= L3) return;
    const int v[3] = {(int)(gid % L), (int)((gid / L) % L), (int)(gid / ((long)L * L))};
    const int n1 = n + 1;
    const long oct = (long)n1 * n1 * n1;
    int a[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d] = v[d] <= n ? v[d] : L - v[d];
    const long o = ((long)a[2] * n1 + a[1]) * n1 + a[0];
    const C K0 = spec[o], w4 = W[3 * L3 + gid];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        C Kd = spec[(1 + d) * oct + o];
        if (v[d] > n) { Kd.x = -Kd.x; Kd.y = -Kd.y; }
        W[d * L3 + gid] = cfma(K0, W[d * L3 + gid], cmul(Kd, w4));
    }
}

// y = x + W[d] cropped to [0,n)^3
template <typename C>
__global__ void k_cf_crop(const C *__restrict__ W, const C *__restrict__ x, C *y, int n, int L)
{
    const long n3 = (long)n * n * n, L3 = (long)L * L * L;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 3 * n3) return;
    const int d = (int)(gid / n3);
    const long i = gid - d * n3;
    const int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
    y[gid] = x[gid] + W[d * L3 + ((long)i3 * L + i2) * L + i1];
}

inline unsigned nb256(long c) { return (unsigned)((c + 255) / 256); }

} // namespace

struct CufftState {
    cufftHandle fwd = 0, inv = 0;
    int prec = -1;
    bool have = false;
    DevBuf W;
    ~CufftState()
    {
        if (have) {
            cufftDestroy(fwd);
            cufftDestroy(inv);
        }
    }
};

void spm_cufft_free(CufftState *c) { delete c; }

static spm_status cufft_check(cufftResult r, const char *what)
{
    if (r != CUFFT_SUCCESS) {
        spm_set_error("cuFFT %s failed (cufftResult %d)", what, (int)r);
        return r == CUFFT_ALLOC_FAILED ? SPM_ERR_OOM : SPM_ERR_CUDA;
    }
    return SPM_OK;
}

template <typename R>
static spm_status cufft_apply_typed(spm_problem_s *P, const void *xv, void *yv, int nrhs, cudaStream_t s)
{
    using C = typename cplx_of<R>::type;
    const bool dbl = sizeof(R) == 8;
    const int n = P->n, L = P->L, pi = dbl ? 0 : 1;
    const long n3 = (long)n * n * n, L3 = (long)L * L * L;
    if (!P->cufft) P->cufft = new CufftState();
    CufftState *cs = P->cufft;
    if (!cs->have || cs->prec != pi) {
        if (cs->have) {
            cufftDestroy(cs->fwd);
            cufftDestroy(cs->inv);
            cs->have = false;
        }
        int dims[3] = {L, L, L};
        const cufftType t = dbl ? CUFFT_Z2Z : CUFFT_C2C;
        SPM_TRY(cufft_check(cufftPlanMany(&cs->fwd, 3, dims, nullptr, 1, (int)L3, nullptr, 1, (int)L3, t, 4), "plan (4 fields)"));
        if (cufftPlanMany(&cs->inv, 3, dims, nullptr, 1, (int)L3, nullptr, 1, (int)L3, t, 3) != CUFFT_SUCCESS) {
            cufftDestroy(cs->fwd);
            spm_set_error("cuFFT plan (3 fields) failed");
            return SPM_ERR_CUDA;
        }
        cs->prec = pi;
        cs->have = true;
    }
    SPM_TRY(cs->W.ensure(sizeof(C) * 4 * L3));
    SPM_TRY(cufft_check(cufftSetStream(cs->fwd, s), "set stream"));
    SPM_TRY(cufft_check(cufftSetStream(cs->inv, s), "set stream"));
    C *W = cs->W.as<C>();
    const C *m = dbl ? P->m128.as<C>() : P->m64.as<C>();
    const C *p = dbl ? P->p128.as<C>() : P->p64.as<C>();
    const C *spec = dbl ? P->spec128.as<C>() : P->spec64.as<C>();
    for (int b = 0; b < nrhs; ++b) {
        const C *x = reinterpret_cast<const C *>(xv) + (long)b * 3 * n3;
        C *y = reinterpret_cast<C *>(yv) + (long)b * 3 * n3;
        k_cf_pad<C><<<nb256(L3), 256, 0, s>>>(x, m, p, W, n, L);
        if constexpr (sizeof(R) == 8)
            SPM_TRY(cufft_check(cufftExecZ2Z(cs->fwd, (cufftDoubleComplex *)W, (cufftDoubleComplex *)W, CUFFT_FORWARD), "exec"));
        else
            SPM_TRY(cufft_check(cufftExecC2C(cs->fwd, (cufftComplex *)W, (cufftComplex *)W, CUFFT_FORWARD), "exec"));
        k_cf_product<C><<<nb256(L3), 256, 0, s>>>(W, spec, n, L);
        if constexpr (sizeof(R) == 8)
            SPM_TRY(cufft_check(cufftExecZ2Z(cs->inv, (cufftDoubleComplex *)W, (cufftDoubleComplex *)W, CUFFT_INVERSE), "exec"));
        else
            SPM_TRY(cufft_check(cufftExecC2C(cs->inv, (cufftComplex *)W, (cufftComplex *)W, CUFFT_INVERSE), "exec"));
        k_cf_crop<C><<<nb256(3 * n3), 256, 0, s>>>(W, x, y, n, L);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

extern "C" spm_status spm_apply_A_cufft(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64) { spm_set_error("precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    if (nrhs < 0 || nrhs > 65535) { spm_set_error("nrhs must be in [0, 65535]"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && (!x || !y)) { spm_set_error("NULL buffer"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && x == y) { spm_set_error("input and output alias"); return SPM_ERR_INVALID_ARG; }
    if (nrhs == 0) return SPM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return prec == SPM_C128 ? cufft_apply_typed<double>(P, x, y, nrhs, s) : cufft_apply_typed<float>(P, x, y, nrhs, s);
}
