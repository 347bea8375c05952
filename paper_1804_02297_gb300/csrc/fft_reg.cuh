// Register-resident Stockham FFT of one line of length L (a power of two, 8..2048).
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

// stage radices: 8 | 8,2 | 8,4 | 8,8 | 8,8,2 | 8,8,4 | 8,8,8 for L = 8 ... 512,
// then 8,8,8,2 | 8,8,8,4 for L = 1024, 2048
__host__ __device__ constexpr int nstages(int L) { return L == 8 ? 1 : (L <= 64 ? 2 : (L <= 512 ? 3 : 4)); }
__host__ __device__ constexpr int radix_of(int L, int s)
{
    return s == 0 ? 8
                  : (s == 1 ? (L == 16 ? 2 : (L == 32 ? 4 : 8))
                            : (s == 2 ? (L == 128 ? 2 : (L == 256 ? 4 : 8)) : L / 512));
}
__host__ __device__ constexpr int span_of(int L, int s) { return s == 0 ? 1 : radix_of(L, s - 1) * span_of(L, s - 1); }

template <typename C> __device__ __forceinline__ C add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// complex64: one packed FP32x2 instruction per complex add or subtract
// (a - b = fma(b, -1, a), exact like the subtraction)
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

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
    if constexpr (NS >= 4) stage<DIR, L, 3>(v, t, buf, sync, tw);
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


// K lines at once (E = 8 per thread): the K lines use K shared buffers and
// share every synchronisation, so K transforms cost the barriers of one.
// buf(k, pos) addresses line k's buffer.
template <int DIR, int L, int S, int K, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void stage_k(C (&v)[K][8], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    constexpr int T = L / 8;
    constexpr int r = radix_of(L, S), Ns = span_of(L, S);
    constexpr int pNs = span_of(L, S - 1);
    const int kp = t % pNs;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int q = 0; q < 8; ++q) buf(k, (t - kp) * 8 + kp + q * pNs) = v[k][q];
    sync();
    constexpr int nb = 8 / r;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int u = 0; u < nb; ++u)
#pragma unroll
            for (int q = 0; q < r; ++q) v[k][u * r + q] = buf(k, t + u * T + q * (L / r));
    sync();
    constexpr int step = L / (r * Ns);
#pragma unroll
    for (int u = 0; u < nb; ++u) {
        const int kk = (t + u * T) % Ns;
#pragma unroll
        for (int q = 1; q < r; ++q) {
            const C w = tw_at<DIR>(tw, q * kk * step);
#pragma unroll
            for (int k = 0; k < K; ++k) v[k][u * r + q] = cmul(v[k][u * r + q], w);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) dft<DIR, r, false>(v[k] + u * r);
    }
}

template <int DIR, int L, bool PRUNE, int K, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void fft_lines(C (&v)[K][8], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    constexpr int NS = nstages(L);
#pragma unroll
    for (int k = 0; k < K; ++k) dft<DIR, 8, PRUNE>(v[k]);
    if constexpr (NS >= 2) stage_k<DIR, L, 1, K>(v, t, buf, sync, tw);
    if constexpr (NS >= 3) stage_k<DIR, L, 2, K>(v, t, buf, sync, tw);
    if constexpr (NS >= 4) stage_k<DIR, L, 3, K>(v, t, buf, sync, tw);
    constexpr int rl = radix_of(L, NS - 1);
    if constexpr (rl != 8) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            C o[8];
#pragma unroll
            for (int u = 0; u < 8 / rl; ++u)
#pragma unroll
                for (int q = 0; q < rl; ++q) o[u + (8 / rl) * q] = v[k][u * rl + q];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[k][m] = o[m];
        }
    }
}

} // namespace fftr

// ============================================================ 12 per thread
// L = 96 and 192 (grids n = 48 and 96): E = 12 elements per thread, T = L/12
// threads per line, stages radix 12 (= 3 x 4), then 4 and 2 (L = 96) or 4 and
// 4 (L = 192).  Same t + T m register pattern on entry and exit.
namespace fftr12 {

__host__ __device__ constexpr int radix_of(int L, int s) { return s == 0 ? 12 : (s == 1 ? 4 : (L == 96 ? 2 : 4)); }
__host__ __device__ constexpr int span_of(int L, int s) { return s == 0 ? 1 : radix_of(L, s - 1) * span_of(L, s - 1); }

// 3-point DFT, w = exp(DIR 2 pi i / 3)
template <int DIR, typename C> __device__ __forceinline__ void dft3(C &x0, C &x1, C &x2)
{
    using R = decltype(x0.x);
    const R h = (R)0.86602540378443864676; // sqrt(3)/2
    C t1 = fftr::add(x1, x2), t2 = fftr::sub(x1, x2);
    C m;
    m.x = x0.x - (R)0.5 * t1.x;
    m.y = x0.y - (R)0.5 * t1.y;
    C s; // DIR i h t2
    s.x = -(R)DIR * h * t2.y;
    s.y = (R)DIR * h * t2.x;
    x0 = fftr::add(x0, t1);
    x1 = fftr::add(m, s);
    x2 = fftr::sub(m, s);
}

// a * exp(DIR 2 pi i M / 12)
template <int DIR, int M, typename C> __device__ __forceinline__ C w12(C a)
{
    using R = decltype(a.x);
    if constexpr (M == 0) return a;
    const R cs[7] = {(R)1, (R)0.86602540378443864676, (R)0.5, (R)0, (R)-0.5, (R)-0.86602540378443864676, (R)-1};
    const R sn7[7] = {(R)0, (R)0.5, (R)0.86602540378443864676, (R)1, (R)0.86602540378443864676, (R)0.5, (R)0};
    const R c = cs[M], sn = (R)DIR * sn7[M];
    C r;
    r.x = a.x * c - a.y * sn;
    r.y = a.x * sn + a.y * c;
    return r;
}

// X[k1 + 3 k2] = sum_n2 w4^(n2 k2) w12^(n2 k1) sum_n1 x[4 n1 + n2] w3^(n1 k1)
template <int DIR, bool PRUNE, typename C> __device__ __forceinline__ void dft12(C *v)
{
    C a[4][3];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C x0 = v[n2], x1 = v[n2 + 4], x2 = v[n2 + 8];
        if (PRUNE) { // x[p] = 0 for p >= 6: x2 = 0 always, x1 = 0 for n2 >= 2
            x2.x = 0; x2.y = 0;
            if (n2 >= 2) { x1.x = 0; x1.y = 0; }
        }
        dft3<DIR>(x0, x1, x2);
        a[n2][0] = x0;
        a[n2][1] = x1;
        a[n2][2] = x2;
    }
    a[1][1] = w12<DIR, 1>(a[1][1]);
    a[1][2] = w12<DIR, 2>(a[1][2]);
    a[2][1] = w12<DIR, 2>(a[2][1]);
    a[2][2] = w12<DIR, 4>(a[2][2]);
    a[3][1] = w12<DIR, 3>(a[3][1]);
    a[3][2] = w12<DIR, 6>(a[3][2]);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        fftr::dft4<DIR>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 3 * k2] = t[k2];
    }
}

template <int DIR, int L, int S, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void stage(C v[12], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    constexpr int T = L / 12;
    constexpr int r = radix_of(L, S), Ns = span_of(L, S);
    constexpr int pr = radix_of(L, S - 1), pNs = span_of(L, S - 1);
    constexpr int pnb = 12 / pr, nb = 12 / r;
#pragma unroll
    for (int u = 0; u < pnb; ++u) {
        const int j = t + u * T, k = j % pNs;
#pragma unroll
        for (int q = 0; q < pr; ++q) buf((j - k) * pr + k + q * pNs) = v[u * pr + q];
    }
    sync();
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
        for (int q = 1; q < r; ++q) v[u * r + q] = cmul(v[u * r + q], fftr::tw_at<DIR>(tw, q * k * step));
        if constexpr (r == 4) fftr::dft4<DIR>(v + u * r);
        else fftr::dft2<DIR>(v + u * r);
    }
}

template <int DIR, int L, bool PRUNE, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void fft_line(C v[12], int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    dft12<DIR, PRUNE>(v);
    stage<DIR, L, 1>(v, t, buf, sync, tw);
    stage<DIR, L, 2>(v, t, buf, sync, tw);
    constexpr int rl = radix_of(L, 2);
    C o[12];
#pragma unroll
    for (int u = 0; u < 12 / rl; ++u)
#pragma unroll
        for (int q = 0; q < rl; ++q) o[u + (12 / rl) * q] = v[u * rl + q];
#pragma unroll
    for (int m = 0; m < 12; ++m) v[m] = o[m];
}

} // namespace fftr12

// elements per thread of the register line FFT for length L
__host__ __device__ constexpr int line_elems(int L) { return (L == 96 || L == 192) ? 12 : 8; }

// one line, E = line_elems(L) values per thread at positions t + (L/E) m
template <int DIR, int L, bool PRUNE, typename C, typename Buf, typename Sync>
__device__ __forceinline__ void line_fft(C *v, int t, Buf buf, Sync sync, const C *__restrict__ tw)
{
    if constexpr (line_elems(L) == 12) fftr12::fft_line<DIR, L, PRUNE>(v, t, buf, sync, tw);
    else fftr::fft_line<DIR, L, PRUNE>(v, t, buf, sync, tw);
}
