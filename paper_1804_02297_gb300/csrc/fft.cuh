// Shared-memory Stockham FFT used by every FFT pass of the operator apply.
//
// Lines of length L = 2^logL sit in shared memory with stride `ls` (>= L).
// Stockham autosort: each stage reads from one buffer and writes to the other,
// so no bit reversal is needed.  A stage of radix R with current span Ns maps
// work item j (0 <= j < L/R, k = j mod Ns) to
//     v_r = in[j + r L/R] * w^(r k L/(R Ns)),  r = 0..R-1,   w = exp(DIR 2 pi i / L)
//     out[(j - k) R + k + r Ns] = (R-point DFT of v)_r.
// One radix-2 stage runs first when logL is odd, then radix-4 stages.
// DIR = -1 forward (exp(-2 pi i ...)), +1 inverse (unscaled).
#pragma once
#include "common.cuh"

template <int DIR, typename C>
__device__ __forceinline__ C twiddle(const C *__restrict__ tw, int idx)
{
    C w = tw[idx];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// Returns the buffer (a or b) that holds the result.  All threads of the block
// must call it (it synchronises with __syncthreads between stages).  L = 2^k or
// 3 * 2^k: a radix-3 stage first when 3 divides L, then radix 2 (if needed) and 4.
template <int DIR, typename C>
__device__ C *smem_fft(C *a, C *b, int L, int logL, int nlines, int ls, const C *__restrict__ tw)
{
    (void)logL;
    const int tid = threadIdx.x, nt = blockDim.x;
    C *in = a, *out = b;
    int Ns = 1;
    int rest = L;
    if (L % 3 == 0) { // radix 3, span 1: outputs at 3 j + r
        const int third = L / 3;
        const int total = nlines * third;
        for (int it = tid; it < total; it += nt) {
            int line = it / third, j = it - line * third;
            const C *li = in + line * ls;
            C *lo = out + line * ls;
            C x0 = li[j], x1 = li[j + third], x2 = li[j + 2 * third];
            using R = decltype(x0.x);
            const R h = (R)0.86602540378443864676;
            C t1 = x1 + x2, t2 = x1 - x2, m, sg;
            m.x = x0.x - (R)0.5 * t1.x;
            m.y = x0.y - (R)0.5 * t1.y;
            sg.x = -(R)DIR * h * t2.y;
            sg.y = (R)DIR * h * t2.x;
            lo[3 * j] = x0 + t1;
            lo[3 * j + 1] = m + sg;
            lo[3 * j + 2] = m - sg;
        }
        __syncthreads();
        C *t = in; in = out; out = t;
        Ns = 3;
        rest = third;
    }
    int lg = 0;
    while ((1 << lg) < rest) ++lg;
    if (lg & 1) { // radix 2, span Ns
        const int half = L >> 1;
        const int total = nlines * half;
        const int step = L / (2 * Ns);
        for (int it = tid; it < total; it += nt) {
            int line = it / half, j = it - line * half;
            int k = j % Ns;
            const C *li = in + line * ls;
            C *lo = out + line * ls;
            C a0 = li[j], a1 = li[j + half];
            if (Ns > 1) a1 = cmul(a1, twiddle<DIR>(tw, k * step));
            int idx = (j - k) * 2 + k;
            lo[idx] = a0 + a1;
            lo[idx + Ns] = a0 - a1;
        }
        __syncthreads();
        C *t = in; in = out; out = t;
        Ns *= 2;
    }
    const int q = L >> 2;
    const int total = nlines * q;
    for (; Ns < L; Ns <<= 2) {
        const int step = L / (4 * Ns); // twiddle index stride for r = 1
        for (int it = tid; it < total; it += nt) {
            int line = it / q, j = it - line * q;
            int k = j % Ns;
            const C *li = in + line * ls;
            C *lo = out + line * ls;
            C v0 = li[j], v1 = li[j + q], v2 = li[j + 2 * q], v3 = li[j + 3 * q];
            if (Ns > 1) {
                v1 = cmul(v1, twiddle<DIR>(tw, k * step));
                v2 = cmul(v2, twiddle<DIR>(tw, 2 * k * step));
                v3 = cmul(v3, twiddle<DIR>(tw, 3 * k * step));
            }
            C s02 = v0 + v2, d02 = v0 - v2, s13 = v1 + v3, d13 = mul_i<DIR>(v1 - v3);
            int idx = (j - k) * 4 + k;
            lo[idx] = s02 + s13;
            lo[idx + Ns] = d02 + d13;
            lo[idx + 2 * Ns] = s02 - s13;
            lo[idx + 3 * Ns] = d02 - d13;
        }
        __syncthreads();
        C *t = in; in = out; out = t;
    }
    return in;
}
