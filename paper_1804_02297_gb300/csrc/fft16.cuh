// Register-resident Stockham FFT with 16 values per thread, for the line
// lengths L = 128, 256, 512 (the padded grids n = 64, 128, 256).
//
// T = L/16 threads cooperate on a line; thread t holds v[m] = x[t + T m],
// m = 0..15, on entry and on exit (the same pattern as the 8-per-thread engine
// of fft_reg.cuh, so loads and stores stay strided by T and coalesce across
// columns).  Stages (radix r, span Ns): butterfly j, k = j mod Ns, inputs
// x[j + q L/r] times w^(q k L/(r Ns)), r-point DFT, outputs to
// (j - k) r + k + q Ns, w = exp(DIR 2 pi i / L):
//   L = 128: radix 16 (Ns 1), radix 8 (Ns 16)      one shared-memory exchange
//   L = 256: radix 16 (Ns 1), radix 16 (Ns 16)     one exchange
//   L = 512: radix 16, radix 16 (Ns 16), radix 2 (Ns 256)   two exchanges
// Compared with 8 values per thread this saves one exchange and one twiddle
// pass per line at L = 128 and 256.  The twiddles of the middle stage depend
// only on the thread's position in the line, so a thread computes them once
// (Tw16::init) and keeps them in registers for every line it transforms (the
// inverse uses their conjugates); the radix-2 stage at L = 512 reads its
// twiddles from a shared-memory table.
// PRUNE: x[p] = 0 for p >= L/2 (zero padding), i.e. v[8..15] are ignored.
#pragma once
#include "fft_reg.cuh"

namespace fft16 {

template <typename C> __device__ __forceinline__ C cj(C a) { a.y = -a.y; return a; }

// a * w (DIR < 0) or a * conj(w) (DIR > 0), w a forward twiddle
template <int DIR, typename C> __device__ __forceinline__ C twmul(C a, C w)
{
    C r;
    if (DIR < 0) { r.x = a.x * w.x - a.y * w.y; r.y = a.x * w.y + a.y * w.x; }
    else { r.x = a.x * w.x + a.y * w.y; r.y = a.y * w.x - a.x * w.y; }
    return r;
}

// multiply by exp(DIR 2 pi i e / 16) for e = 1, 3 (e = 2, 4, 6 use fftr::w8)
template <int DIR, int E, typename C> __device__ __forceinline__ C w16(C a)
{
    using R = decltype(a.x);
    const R c = E == 1 ? (R)0.92387953251128675613 : (R)0.38268343236508977173; // cos(pi/8), cos(3 pi/8)
    const R s = E == 1 ? (R)0.38268343236508977173 : (R)0.92387953251128675613; // sin(pi/8), sin(3 pi/8)
    C r;
    r.x = a.x * c - (R)DIR * a.y * s;
    r.y = a.y * c + (R)DIR * a.x * s;
    return r;
}

// in-place 16-point DFT, natural order in and out:
// X[k1 + 4 k2] = sum_n2 w4^(n2 k2) w16^(n2 k1) sum_n1 x[4 n1 + n2] w4^(n1 k1)
template <int DIR, bool PRUNE, typename C> __device__ __forceinline__ void dft16(C *v)
{
    C a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        if (PRUNE) { // x[4 n1 + n2] = 0 for n1 >= 2
            const C x0 = v[n2], x1 = v[n2 + 4];
            const C ix1 = fftr::w8<DIR, 2>(x1); // w4 x1
            a[n2][0] = fftr::add(x0, x1);
            a[n2][1] = fftr::add(x0, ix1);
            a[n2][2] = fftr::sub(x0, x1);
            a[n2][3] = fftr::sub(x0, ix1);
        } else {
            C t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
            fftr::dft4<DIR>(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
        }
    }
    a[1][1] = w16<DIR, 1>(a[1][1]);
    a[1][2] = fftr::w8<DIR, 1>(a[1][2]);
    a[1][3] = w16<DIR, 3>(a[1][3]);
    a[2][1] = fftr::w8<DIR, 1>(a[2][1]);
    a[2][2] = fftr::w8<DIR, 2>(a[2][2]);
    a[2][3] = fftr::w8<DIR, 3>(a[2][3]);
    a[3][1] = w16<DIR, 3>(a[3][1]);
    a[3][2] = fftr::w8<DIR, 3>(a[3][2]);
    { // w16^9 = -w16^1
        C t = w16<DIR, 1>(a[3][3]);
        a[3][3].x = -t.x;
        a[3][3].y = -t.y;
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        fftr::dft4<DIR>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <int L> struct plan {
    static_assert(L == 128 || L == 256 || L == 512, "16-per-thread lines: L = 128, 256, 512");
    static constexpr int T = L / 16;
    static constexpr int r1 = L == 128 ? 8 : 16;          // radix of the middle stage (span 16)
    static constexpr int nb1 = 16 / r1;                    // its butterflies per thread
    static constexpr int step1 = L / (r1 * 16);            // twiddle step of the middle stage
    static constexpr int NTW = nb1 * (r1 - 1);             // middle-stage twiddles per thread
};

// the middle stage's twiddles of thread t, forward direction: w_L^(q k step1),
// butterfly u (k = (t + u T) mod 16), q = 1 .. r1-1; from the L-entry table
template <typename C, int L> struct Tw16 {
    C w[plan<L>::NTW];
    __device__ __forceinline__ void init(int t, const C *__restrict__ tw)
    {
        constexpr int T = plan<L>::T, r1 = plan<L>::r1, nb1 = plan<L>::nb1, st = plan<L>::step1;
#pragma unroll
        for (int u = 0; u < nb1; ++u) {
            const int k = (t + u * T) % 16;
#pragma unroll
            for (int q = 1; q < r1; ++q) w[u * (r1 - 1) + q - 1] = tw[(q * k * st) % L];
        }
    }
};

// One line.  buf(pos) -> C& into the line's shared-memory buffer (L entries);
// sync() synchronises every thread sharing it; stw: the L-entry forward twiddle
// table in shared memory (read only at L = 512).
template <int DIR, int L, bool PRUNE, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void line(C (&v)[16], int t, Buf buf, Sync sync, const Tw16<C, L> &tw,
                                     const C *stw)
{
    using P = plan<L>;
    constexpr int T = P::T, r1 = P::r1, nb1 = P::nb1;
    dft16<DIR, PRUNE>(v); // stage 0: butterfly j = t, outputs at 16 t + q
#pragma unroll
    for (int q = 0; q < 16; ++q) buf(16 * t + q) = v[q];
    sync();
    // stage 1: radix r1, span 16; butterfly j = t + u T reads x[j + q L/r1]
#pragma unroll
    for (int u = 0; u < nb1; ++u)
#pragma unroll
        for (int q = 0; q < r1; ++q) v[u * r1 + q] = buf(t + u * T + q * (L / r1));
    sync();
#pragma unroll
    for (int u = 0; u < nb1; ++u) {
#pragma unroll
        for (int q = 1; q < r1; ++q) v[u * r1 + q] = twmul<DIR>(v[u * r1 + q], tw.w[u * (r1 - 1) + q - 1]);
        if constexpr (r1 == 16) dft16<DIR, false>(v + u * r1);
        else fftr::dft8<DIR, false>(v + u * r1);
    }
    if constexpr (L == 512) {
        // outputs of stage 1 (one butterfly j = t, k = t mod 16) at (j - k) 16 + k + 16 q
        const int k = t % 16;
#pragma unroll
        for (int q = 0; q < 16; ++q) buf((t - k) * 16 + k + 16 * q) = v[q];
        sync();
        // stage 2: radix 2, span 256; butterflies j = t + 32 u (u < 8) read x[j], x[j + 256]
        C o[16];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = t + 32 * u;
            C a = buf(j), b = buf(j + 256);
            b = twmul<DIR>(b, stw[j]);
            o[u] = fftr::add(a, b);     // position j       -> m = u
            o[u + 8] = fftr::sub(a, b); // position j + 256 -> m = u + 8
        }
        sync();
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = o[m];
    } else {
        // last stage outputs of butterfly u, index q, sit at t + T (u + nb1 q)
        C o[16];
#pragma unroll
        for (int u = 0; u < nb1; ++u)
#pragma unroll
            for (int q = 0; q < r1; ++q) o[u + nb1 * q] = v[u * r1 + q];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = o[m];
    }
}

} // namespace fft16
