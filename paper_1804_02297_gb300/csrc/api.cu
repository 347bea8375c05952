// C-ABI entry points of libspm (include/spm.h): argument checks, problem
// set-up on the host (medium, twiddles, lattice constant) and dispatch.
#include <math.h>
#include <stdlib.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <complex>
#include <vector>

#include "common.cuh"

static thread_local char g_err[1024] = "";

void spm_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

spm_status DevBuf::ensure(size_t want)
{
    if (want <= bytes && ptr) return SPM_OK;
    release();
    if (want == 0) return SPM_OK;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        spm_set_error("cudaMalloc(%zu bytes) failed: %s", want, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA;
    }
    bytes = want;
    return SPM_OK;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

spm_status spm_apply_init_attributes();
spm_status spm_entries_impl(spm_problem_s *P, double *out_host);
spm_status spm_plane_wave_impl(spm_problem_s *P, int prec, const double *dir, const double *pol, int nrhs,
                               void *e, cudaStream_t s);
spm_status spm_axpby_impl(int prec, long count, double a, const void *x, double b, void *y, cudaStream_t s);

// ------------------------------------------------------------------ lattice
// Z = sum'_{j in Z^3} |j|^{-1}, analytically continued, by Ewald splitting of
// the Epstein zeta function of the self-dual lattice Z^3 at s = 1/2:
//   Z = -3 + sum'_j [ erfc(sqrt(pi)|j|)/|j| + exp(-pi |j|^2)/(pi |j|^2) ].
extern "C" double spm_lattice_constant(void)
{
    static double cached = 0.0;
    if (cached != 0.0) return cached;
    const double pi = 3.14159265358979323846;
    double s = 0.0;
    const int R = 7;
    for (int a = -R; a <= R; ++a)
        for (int b = -R; b <= R; ++b)
            for (int c = -R; c <= R; ++c) {
                if (!a && !b && !c) continue;
                double r2 = (double)a * a + (double)b * b + (double)c * c;
                double r = sqrt(r2);
                s += erfc(sqrt(pi) * r) / r + exp(-pi * r2) / (pi * r2);
            }
    cached = -3.0 + s;
    return cached;
}

extern "C" const char *spm_last_error(void) { return g_err; }

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static bool prec_ok(spm_prec p) { return p == SPM_C128 || p == SPM_C64; }

// ------------------------------------------------------------------ create
extern "C" spm_status spm_create_problem(int n, double omega, const double *eps_host, const double *grad_eps_host,
                                         spm_quad quad, void *stream, spm_problem *out)
{
    if (!out) { spm_set_error("out is NULL"); return SPM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 4 || n > 256) { spm_set_error("n = %d outside [4, 256] (FFT lengths 2n up to 512)", n); return SPM_ERR_INVALID_ARG; }
    if ((n & (n - 1)) != 0 && n != 48 && n != 96) {
        spm_set_error("n = %d: the FFT length 2n must be a power of two or 96, 192 (n = 48, 96)", n);
        return SPM_ERR_INVALID_ARG;
    }
    if (!(omega > 0.0) || !isfinite(omega)) { spm_set_error("omega must be positive and finite"); return SPM_ERR_INVALID_ARG; }
    if (!eps_host) { spm_set_error("eps_host is NULL"); return SPM_ERR_INVALID_ARG; }
    if (quad != SPM_QUAD_ORDER4 && quad != SPM_QUAD_ORDER2) { spm_set_error("bad quadrature %d", (int)quad); return SPM_ERR_INVALID_ARG; }
    static bool attrs = false;
    if (!attrs) {
        SPM_TRY(spm_apply_init_attributes());
        attrs = true;
        // apply plans tuned earlier on this kind of device, if the caller names a file
        const char *plans = getenv("SPM_APPLY_PLANS");
        if (plans && *plans) {
            int loaded = 0;
            if (spm_load_plans_impl(plans, &loaded) != SPM_OK) spm_set_error(""); // a stale or foreign file is ignored
        }
    }

    spm_problem_s *P = new spm_problem_s();
    P->n = n;
    P->L = 2 * n;
    P->logL = ilog2(P->L);
    P->k = omega; // k = sqrt(eps0 mu0) omega with eps0 = mu0 = 1
    P->h = 1.0 / (n + 1);
    P->quad = (int)quad;
    P->zconst = spm_lattice_constant();
    P->stream = as_stream(stream);

    const long n3 = (long)n * n * n;
    typedef std::complex<double> cd;
    const cd *eps = reinterpret_cast<const cd *>(eps_host);
    std::vector<cd> m(n3), p(3 * n3);
    for (long i = 0; i < n3; ++i) {
        if (!(std::abs(eps[i]) > 0.0) || !isfinite(eps[i].real()) || !isfinite(eps[i].imag())) {
            spm_set_error("eps[%ld] is zero or not finite", i);
            delete P;
            return SPM_ERR_INVALID_ARG;
        }
        m[i] = 1.0 - eps[i];
    }
    if (grad_eps_host) {
        const cd *g = reinterpret_cast<const cd *>(grad_eps_host);
        for (int d = 0; d < 3; ++d)
            for (long i = 0; i < n3; ++i) p[d * n3 + i] = -g[d * n3 + i] / eps[i];
    } else {
        // fourth-order central differences, eps = 1 outside the grid
        auto E = [&](int a, int b, int c) -> cd {
            if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) return cd(1.0, 0.0);
            return eps[((long)c * n + b) * n + a];
        };
        const double inv12h = 1.0 / (12.0 * P->h);
        for (int i3 = 0; i3 < n; ++i3)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i1 = 0; i1 < n; ++i1) {
                    long i = ((long)i3 * n + i2) * n + i1;
                    int ii[3] = {i1, i2, i3};
                    for (int d = 0; d < 3; ++d) {
                        int a[3], b[3], c[3], e2[3];
                        for (int q = 0; q < 3; ++q) a[q] = b[q] = c[q] = e2[q] = ii[q];
                        a[d] += 2; b[d] += 1; c[d] -= 1; e2[d] -= 2;
                        cd der = (-E(a[0], a[1], a[2]) + 8.0 * E(b[0], b[1], b[2]) - 8.0 * E(c[0], c[1], c[2]) +
                                  E(e2[0], e2[1], e2[2])) * inv12h;
                        p[d * n3 + i] = -der / eps[i];
                    }
                }
    }
    std::vector<float> m32(2 * n3), p32(6 * n3);
    for (long i = 0; i < n3; ++i) { m32[2 * i] = (float)m[i].real(); m32[2 * i + 1] = (float)m[i].imag(); }
    for (long i = 0; i < 3 * n3; ++i) { p32[2 * i] = (float)p[i].real(); p32[2 * i + 1] = (float)p[i].imag(); }

    spm_status st = SPM_OK;
    auto fail = [&](spm_status s2) { spm_destroy(P); return s2; };
    if ((st = P->m128.ensure(16 * n3)) != SPM_OK) return fail(st);
    if ((st = P->p128.ensure(48 * n3)) != SPM_OK) return fail(st);
    if ((st = P->m64.ensure(8 * n3)) != SPM_OK) return fail(st);
    if ((st = P->p64.ensure(24 * n3)) != SPM_OK) return fail(st);
    if (cudaMemcpy(P->m128.ptr, m.data(), 16 * n3, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->p128.ptr, p.data(), 48 * n3, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->m64.ptr, m32.data(), 8 * n3, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->p64.ptr, p32.data(), 24 * n3, cudaMemcpyHostToDevice) != cudaSuccess) {
        spm_set_error("medium upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SPM_ERR_CUDA);
    }
    // twiddles exp(-2 pi i j / L) from libm in FP64
    {
        const int L = P->L;
        std::vector<double> t128(2 * L);
        std::vector<float> t64(2 * L);
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < L; ++j) {
            double a = -2.0 * pi * j / L;
            t128[2 * j] = cos(a);
            t128[2 * j + 1] = sin(a);
            t64[2 * j] = (float)t128[2 * j];
            t64[2 * j + 1] = (float)t128[2 * j + 1];
        }
        if ((st = P->tw128.ensure(16 * L)) != SPM_OK) return fail(st);
        if ((st = P->tw64.ensure(8 * L)) != SPM_OK) return fail(st);
        if (cudaMemcpy(P->tw128.ptr, t128.data(), 16 * L, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(P->tw64.ptr, t64.data(), 8 * L, cudaMemcpyHostToDevice) != cudaSuccess) {
            spm_set_error("twiddle upload failed");
            return fail(SPM_ERR_CUDA);
        }
    }
    // right-hand sides per pass chunk: the passes are latency-bound at these
    // sizes, so more right-hand sides per launch (larger grids) pay even when a
    // chunk's intermediates (24 n^3 complex per RHS) leave the L2; up to 4 GB of
    // intermediates per chunk (64 RHS at n = 64: 17.9k field applies/s against
    // 14.9k with the chunk kept within half of the L2; 8 RHS at n = 128: +5 %)
    {
        const double per64 = 24.0 * n3 * 8, per128 = 24.0 * n3 * 16;
        const double budget = 4096.0 * 1024 * 1024;
        P->chunk64 = per64 >= budget ? 1 : (int)(budget / per64);
        P->chunk128 = per128 >= budget ? 1 : (int)(budget / per128);
        if (P->chunk64 > 64) P->chunk64 = 64;
        if (P->chunk128 > 64) P->chunk128 = 64;
    }
    if ((st = P->dev_err.ensure(sizeof(int))) != SPM_OK) return fail(st);
    if (cudaMemset(P->dev_err.ptr, 0, sizeof(int)) != cudaSuccess) { spm_set_error("memset failed"); return fail(SPM_ERR_CUDA); }
    if ((st = spm_build_spectra(P)) != SPM_OK) return fail(st);
    *out = P;
    return SPM_OK;
}

extern "C" spm_status spm_destroy(spm_problem P)
{
    if (!P) return SPM_OK;
    P->m128.release(); P->p128.release(); P->m64.release(); P->p64.release();
    P->spec128.release(); P->spec64.release(); P->tw128.release(); P->tw64.release();
    P->work.release(); P->alpha128.release(); P->alpha64.release(); P->beta128.release();
    P->qtab128.release(); P->qtab64.release();
    P->S128.release(); P->S64.release(); P->kry.release(); P->gmres_ws.release(); P->dev_err.release();
    spm_factor_free(P->fac128);
    spm_factor_free(P->fac64);
    spm_cufft_free(P->cufft);
    delete P;
    return SPM_OK;
}

extern "C" spm_status spm_problem_info(spm_problem P, int *n, double *k, long long *unknowns)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (n) *n = P->n;
    if (k) *k = P->k;
    if (unknowns) *unknowns = 3LL * P->n * P->n * P->n;
    return SPM_OK;
}

// ------------------------------------------------------------------ applies
static spm_status check_apply(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(prec)) { spm_set_error("apply precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    if (nrhs < 0 || nrhs > 65535) { spm_set_error("nrhs must be in [0, 65535]"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && (!x || !y)) { spm_set_error("NULL buffer"); return SPM_ERR_INVALID_ARG; }
    if (x == y && nrhs > 0) { spm_set_error("input and output alias"); return SPM_ERR_INVALID_ARG; }
    return SPM_OK;
}

extern "C" spm_status spm_apply_A(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, prec, x, y, nrhs));
    if (nrhs == 0) return SPM_OK;
    return spm_apply_A_impl(P, prec, x, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm_apply_Q(spm_problem P, spm_prec prec, const void *v, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, prec, v, y, nrhs));
    if (!P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    return spm_apply_Q_impl(P, prec, v, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm_apply_QA(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, prec, x, y, nrhs));
    if (!P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    // A x goes to library scratch, then Q gathers into y
    const size_t el = prec == SPM_C128 ? 16 : 8;
    const size_t bytes = el * 3 * (size_t)P->n * P->n * P->n * nrhs;
    SPM_TRY(P->kry.ensure(bytes > P->kry.bytes ? bytes : P->kry.bytes));
    SPM_TRY(spm_apply_A_impl(P, prec, x, P->kry.ptr, nrhs, as_stream(stream)));
    return spm_apply_Q_impl(P, prec, P->kry.ptr, y, nrhs, as_stream(stream));
}

// ------------------------------------------------------------------ stencils
extern "C" spm_status spm_set_stencils(spm_problem P, const double *alpha_host, const double *beta_host)
{
    if (!P || !alpha_host || !beta_host) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    P->alpha_h.assign(alpha_host, alpha_host + 2 * 27 * 81 * 3);
    P->beta_h.assign(beta_host, beta_host + 2 * 27 * 108 * 3);
    P->sv_h.assign(27 * 81, 0.0);
    std::vector<float> a32(2 * 27 * 81 * 3);
    for (size_t i = 0; i < a32.size(); ++i) a32[i] = (float)P->alpha_h[i];
    SPM_TRY(P->alpha128.ensure(16 * 27 * 81 * 3));
    SPM_TRY(P->alpha64.ensure(8 * 27 * 81 * 3));
    SPM_TRY(P->beta128.ensure(16 * 27 * 108 * 3));
    SPM_CUDA_TRY(cudaMemcpy(P->alpha128.ptr, P->alpha_h.data(), 16 * 27 * 81 * 3, cudaMemcpyHostToDevice));
    SPM_CUDA_TRY(cudaMemcpy(P->alpha64.ptr, a32.data(), 8 * 27 * 81 * 3, cudaMemcpyHostToDevice));
    SPM_CUDA_TRY(cudaMemcpy(P->beta128.ptr, P->beta_h.data(), 16 * 27 * 108 * 3, cudaMemcpyHostToDevice));
    P->have_stencils = true;
    SPM_TRY(spm_build_qtable(P));
    spm_factor_free(P->fac128); P->fac128 = nullptr;
    spm_factor_free(P->fac64); P->fac64 = nullptr;
    return spm_assemble_S(P);
}

extern "C" spm_status spm_get_stencils(spm_problem P, double *alpha_host, double *beta_host, double *sv_host)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    if (alpha_host) memcpy(alpha_host, P->alpha_h.data(), sizeof(double) * P->alpha_h.size());
    if (beta_host) memcpy(beta_host, P->beta_h.data(), sizeof(double) * P->beta_h.size());
    if (sv_host) memcpy(sv_host, P->sv_h.data(), sizeof(double) * P->sv_h.size());
    return SPM_OK;
}

extern "C" spm_status spm_build_stencils(spm_problem P, spm_prec factor_prec)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(factor_prec) && factor_prec != SPM_C64H) { spm_set_error("factor precision must be SPM_C128, SPM_C64 or SPM_C64H"); return SPM_ERR_INVALID_ARG; }
    SPM_TRY(spm_stencils_device(P));
    spm_factor_free(P->fac128); P->fac128 = nullptr;
    spm_factor_free(P->fac64); P->fac64 = nullptr;
    SPM_TRY(spm_assemble_S(P));
    return spm_factor_impl(P, factor_prec);
}

extern "C" spm_status spm_factor_S(spm_problem P, spm_prec prec)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(prec) && prec != SPM_C64H) { spm_set_error("factor precision must be SPM_C128, SPM_C64 or SPM_C64H"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_S) { spm_set_error("S not assembled"); return SPM_ERR_NOT_BUILT; }
    return spm_factor_impl(P, prec);
}

extern "C" spm_status spm_get_apply_plan(spm_prec prec, int L, int *zvariant)
{
    if (!zvariant || (prec != SPM_C128 && prec != SPM_C64)) { spm_set_error("bad arguments"); return SPM_ERR_INVALID_ARG; }
    return spm_apply_plan_impl(prec, L, zvariant, nullptr);
}

extern "C" spm_status spm_set_apply_plan(spm_prec prec, int L, int zvariant)
{
    if (prec != SPM_C128 && prec != SPM_C64) { spm_set_error("apply precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    return spm_apply_plan_impl(prec, L, nullptr, &zvariant);
}

extern "C" spm_status spm_profile_apply(spm_problem P, spm_prec prec, const void *x, void *y, int with_q, int reps,
                                        float *pass_ms, int *npasses, void *stream)
{
    SPM_TRY(check_apply(P, prec, x, y, 1));
    if (!pass_ms || !npasses || reps < 1) { spm_set_error("pass_ms, npasses must be non-NULL and reps >= 1"); return SPM_ERR_INVALID_ARG; }
    if (with_q && !P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    return spm_profile_apply_impl(P, prec, x, y, with_q != 0, reps, pass_ms, npasses, as_stream(stream));
}

extern "C" spm_status spm_save_apply_plans(const char *path)
{
    if (!path) { spm_set_error("NULL path"); return SPM_ERR_INVALID_ARG; }
    return spm_save_plans_impl(path);
}

extern "C" spm_status spm_load_apply_plans(const char *path, int *loaded)
{
    if (!path) { spm_set_error("NULL path"); return SPM_ERR_INVALID_ARG; }
    return spm_load_plans_impl(path, loaded);
}

extern "C" spm_status spm_selftest_bounded_wait(spm_problem P)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    return spm_wait_selftest_impl(P);
}

extern "C" spm_status spm_device_status(spm_problem P)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    SPM_CUDA_TRY(cudaDeviceSynchronize());
    int flag = 0;
    SPM_CUDA_TRY(cudaMemcpy(&flag, P->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        SPM_CUDA_TRY(cudaMemset(P->dev_err.ptr, 0, sizeof(int)));
        spm_set_error("a bounded device wait gave up (code %d); the results of that launch are invalid", flag);
        return SPM_ERR_TIMEOUT;
    }
    return SPM_OK;
}

extern "C" spm_status spm_factor_S_tree(spm_problem P, spm_prec prec, int variant)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(prec) && prec != SPM_C64H) { spm_set_error("factor precision must be SPM_C128, SPM_C64 or SPM_C64H"); return SPM_ERR_INVALID_ARG; }
    if (!P->have_S) { spm_set_error("S not assembled"); return SPM_ERR_NOT_BUILT; }
    return spm_factor_tree_impl(P, prec, variant);
}

extern "C" spm_status spm_factor_info(spm_problem P, spm_prec prec, spm_factor_report *out)
{
    if (!P || !out) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64 && prec != SPM_C64H) { spm_set_error("factor precision must be SPM_C128, SPM_C64 or SPM_C64H"); return SPM_ERR_INVALID_ARG; }
    const int fi = prec == SPM_C128 ? 0 : 1;
    if (!(fi == 0 ? P->fac128 : P->fac64)) { spm_set_error("no factor of S in this precision (spm_factor_S)"); return SPM_ERR_NOT_BUILT; }
    out->variant = P->fac_info[fi].variant;
    out->attempts = P->fac_info[fi].attempts;
    out->half_store = P->fac_info[fi].half_store ? 1 : 0;
    out->probe_relres = P->fac_info[fi].probe_relres;
    out->raised_pivots = P->fac_info[fi].raised_pivots;
    out->stored_bytes = (long long)P->fac_info[fi].stored_bytes;
    return SPM_OK;
}

extern "C" spm_status spm_apply_S(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, prec, x, y, nrhs));
    if (!P->have_S) { spm_set_error("S not assembled"); return SPM_ERR_NOT_BUILT; }
    if (nrhs == 0) return SPM_OK;
    return spm_apply_S_impl(P, prec, x, y, nrhs, as_stream(stream));
}

extern "C" spm_status spm_solve_S(spm_problem P, spm_prec prec, const void *b, void *x, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, prec, b, x, nrhs));
    if ((prec == SPM_C128 && !P->fac128) || (prec == SPM_C64 && !P->fac64)) {
        spm_set_error("no factor of S in this precision (spm_factor_S)");
        return SPM_ERR_NOT_BUILT;
    }
    if (nrhs == 0) return SPM_OK;
    return spm_solveS_impl(P, prec, b, x, nrhs, as_stream(stream));
}

// ------------------------------------------------------------------ solving
extern "C" spm_status spm_incident_plane_wave(spm_problem P, spm_prec prec, const double *dir, const double *pol,
                                             int nrhs, void *e, void *stream)
{
    if (!P || !dir || !pol || (!e && nrhs > 0)) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    if (!prec_ok(prec) || nrhs < 0) { spm_set_error("bad precision or nrhs"); return SPM_ERR_INVALID_ARG; }
    if (nrhs == 0) return SPM_OK;
    return spm_plane_wave_impl(P, prec, dir, pol, nrhs, e, as_stream(stream));
}

extern "C" spm_status spm_rhs_from_incident(spm_problem P, const void *einc, void *g, int nrhs, void *stream)
{
    SPM_TRY(check_apply(P, SPM_C128, einc, g, nrhs));
    if (nrhs == 0) return SPM_OK;
    SPM_TRY(spm_apply_A_impl(P, SPM_C128, einc, g, nrhs, as_stream(stream)));
    // g = E^i - A E^i
    return spm_axpby_impl(SPM_C128, 3L * P->n * P->n * P->n * nrhs, 1.0, einc, -1.0, g, as_stream(stream));
}

extern "C" spm_status spm_solve(spm_problem P, spm_prec prec, const void *g, void *x, int nrhs, double tol,
                                int maxit, int restart, spm_solve_info *info)
{
    if (!P || (nrhs > 0 && (!g || !x))) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64 && prec != SPM_MIXED) { spm_set_error("bad precision"); return SPM_ERR_INVALID_ARG; }
    if (!(tol > 0.0) || maxit <= 0 || nrhs < 0) { spm_set_error("bad tol/maxit/nrhs"); return SPM_ERR_INVALID_ARG; }
    if (g == x) { spm_set_error("g and x alias"); return SPM_ERR_INVALID_ARG; }
    if (restart <= 0) restart = 20;
    if (restart > 200) { spm_set_error("restart > 200"); return SPM_ERR_INVALID_ARG; }
    if (info) memset(info, 0, sizeof(*info));
    if (nrhs == 0) return SPM_OK;
    auto t0 = std::chrono::steady_clock::now();
    spm_status st = spm_solve_impl(P, prec, g, x, nrhs, tol, maxit, restart, info);
    auto t1 = std::chrono::steady_clock::now();
    if (info) info->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    return st;
}

// ------------------------------------------------------------------ inspection
extern "C" spm_status spm_kernel_entries(spm_problem P, double *out_host)
{
    if (!P || !out_host) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    return spm_entries_impl(P, out_host);
}
