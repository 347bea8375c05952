// Register-resident Stockham FFT of one line of length L (a power of two, 8..512).
//
// T = L/8 threads cooperate on a line; thread t holds v[m] = x[t + T m], m = 0..7,
// both on entry and on exit, so loads and stores of a line are strided by T and
// coalesce across the T threads.  Stages (radix r, span Ns):
//   butterfly j (k = j mod Ns): inputs x[j + q L/r] times w^(q k L/(r Ns)),
//   r-point DFT, outputs to (j - k) r + k + q Ns      (w = exp(DIR 2 pi i / L)).
// Stage 1 is radix 8 with Ns = 1 and reads the registers directly; between
// stages the line passes through shared memory once; the last stage's outputs
// are permuted in registers back to the t + T m pattern.
// PRUNE: x[p] = 0 for p >= L/2 (zero padding), so v[4..7] are ignored.
#pragma once
#include "common.cuh"

namespace fftr {

// stage radices: 8 | 8,2 | 8,4 | 8,8 | 8,8,2 | 8,8,4 | 8,8,8 for L = 8 ... 512
__host__ __device__ constexpr int nstages(int L) { return L == 8 ? 1 : (L <= 64 ? 2 : 3); }
__host__ __device__ constexpr int radix_of(int L, int s)
{
    return s == 0 ? 8 : (s == 1 ? (L == 16 ? 2 : (L == 32 ? 4 : 8)) : (L == 128 ? 2 : (L == 256 ? 4 : 8)));
}
__host__ __device__ constexpr int span_of(int L, int s) { return s == 0 ? 1 : radix_of(L, s - 1) * span_of(L, s - 1); }

template <typename C> __device__ __forceinline__ C add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// multiply by exp(DIR i pi/4)^e for e = 1, 2, 3
template <int DIR, int E, typename C> __device__ __forceinline__ C w8(C a)
{
    using R = decltype(a.x);
    const R h = (R)0.70710678118654752440;
    C r;
    if (E == 1) { // (1 + DIR i)/sqrt2
        r.x = h * (a.x - DIR * a.y);
        r.y = h * (a.y + DIR * a.x);
    } else if (E == 2) { // DIR i
        r.x = -DIR * a.y;
        r.y = DIR * a.x;
    } else { // (-1 + DIR i)/sqrt2
        r.x = h * (-a.x - DIR * a.y);
        r.y = h * (-a.y + DIR * a.x);
    }
    return r;
}

// in-place r-point DFT of v[0..r-1] (natural order in and out)
template <int DIR, typename C> __device__ __forceinline__ void dft2(C *v)
{
    C a = v[0], b = v[1];
    v[0] = add(a, b);
    v[1] = sub(a, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C *v)
{
    C c0 = add(v[0], v[2]), c1 = sub(v[0], v[2]);
    C c2 = add(v[1], v[3]), c3 = w8<DIR, 2>(sub(v[1], v[3]));
    v[0] = add(c0, c2);
    v[2] = sub(c0, c2);
    v[1] = add(c1, c3);
    v[3] = sub(c1, c3);
}

template <int DIR, bool PRUNE, typename C> __device__ __forceinline__ void dft8(C *v)
{
    C a[4], b[4];
    if (PRUNE) {
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] = v[q]; b[q] = v[q]; }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] = add(v[q], v[q + 4]); b[q] = sub(v[q], v[q + 4]); }
    }
    b[1] = w8<DIR, 1>(b[1]);
    b[2] = w8<DIR, 2>(b[2]);
    b[3] = w8<DIR, 3>(b[3]);
    dft4<DIR>(a);
    dft4<DIR>(b);
#pragma unroll
    for (int q = 0; q < 4; ++q) { v[2 * q] = a[q]; v[2 * q + 1] = b[q]; }
}

template <int DIR, int R, bool PRUNE, typename C> __device__ __forceinline__ void dft(C *v)
{
    if (R == 8) dft8<DIR, PRUNE>(v);
    else if (R == 4) dft4<DIR>(v);
    else if (R == 2) dft2<DIR>(v);
}

template <int DIR, typename C> __device__ __forceinline__ C tw_at(const C *__restrict__ tw, int idx)
{
    C w = tw[idx];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// Stage S >= 1 of a line: write the previous stage's outputs to shared memory,
// read this stage's butterfly inputs, twiddle, DFT.
template <int DIR, int L, int S, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void stage(C v[8], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    constexpr int T = L / 8;
    constexpr int r = radix_of(L, S), Ns = span_of(L, S);
    constexpr int pr = radix_of(L, S - 1), pNs = span_of(L, S - 1);
    static_assert(pr == 8, "every stage before the last is radix 8");
    {   // previous stage: radix 8, one butterfly j = t per thread, k = t mod pNs
        const int k = t % pNs;
#pragma unroll
        for (int q = 0; q < 8; ++q) buf((t - k) * 8 + k + q * pNs) = v[q];
    }
    sync();
    constexpr int nb = 8 / r;
#pragma unroll
    for (int u = 0; u < nb; ++u)
#pragma unroll
        for (int q = 0; q < r; ++q) v[u * r + q] = buf(t + u * T + q * (L / r));
    sync();
    constexpr int step = L / (r * Ns);
#pragma unroll
    for (int u = 0; u < nb; ++u) {
        const int k = (t + u * T) % Ns;
#pragma unroll
        for (int q = 1; q < r; ++q) v[u * r + q] = cmul(v[u * r + q], tw_at<DIR>(tw, q * k * step));
        dft<DIR, r, false>(v + u * r);
    }
}

// One line.  Buf: callable pos -> C& into this line's shared-memory buffer.
// Sync: callable that synchronises every thread sharing the buffer.
template <int DIR, int L, bool PRUNE, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void fft_line(C v[8], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    constexpr int NS = nstages(L);
    dft<DIR, 8, PRUNE>(v); // stage 0: radix 8, span 1, no twiddles
    if constexpr (NS >= 2) stage<DIR, L, 1>(v, t, buf, sync, tw);
    if constexpr (NS >= 3) stage<DIR, L, 2>(v, t, buf, sync, tw);
    // last stage: v[u r + q] holds position t + T (u + (8/r) q); reorder to v[m]
    constexpr int rl = radix_of(L, NS - 1);
    if constexpr (rl != 8) {
        C o[8];
#pragma unroll
        for (int u = 0; u < 8 / rl; ++u)
#pragma unroll
            for (int q = 0; q < rl; ++q) o[u + (8 / rl) * q] = v[u * rl + q];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = o[m];
    }
}

} // namespace fftr
