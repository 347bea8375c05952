// Dense kernels of the multifrontal factor (sparse.cu): a complex GEMM and an
// in-place Gauss-Jordan inversion with partial pivoting, in complex64 (FP32
// arithmetic) and complex128.  All matrices are column-major.
//
// Gauss-Jordan (blocked, right-looking, panels of GJ_NB columns).  Column j is
// eliminated with the pivot row p_j = the row not yet used as a pivot with the
// largest |a_ij| (partial pivoting; rows are never moved).  Written on the
// augmented system [A | I], the row operations turn A into a permutation
// matrix Pi (row p_j has its 1 in column j) and I into B = Pi A^{-1}; the
// in-place form keeps column p_j of B in the storage of column j once that
// column is eliminated, so at the end A^{-1}[j][c] = S[p_j][q_c] with q the
// inverse of p (one gather).  A panel eliminates its columns on every row
// (one cooperative grid, each block holding a slab of rows in shared memory,
// two grid barriers per column); the columns outside the panel receive the
// panel's row operations at once: with T the panel's accumulated operations
// (T = I except in the columns p_j of its pivot rows, which the panel's storage
// holds), Y <- T Y is  tmp = Y[P, :];  Y[P, :] = 0;  Y += panel * tmp  (a GEMM).
// Static pivoting: a pivot below floor = tau * max |a_ij| (of the matrix before
// elimination, computed on the device) is raised to the floor, phase kept, and
// counted.  Nothing of the inversion waits for the host.
#include "common.cuh"

#include <algorithm>
#include <cstdint>
#include <cstring>

namespace {

template <typename C> __device__ __forceinline__ C cdiv_(C a, C b)
{
    using R = decltype(a.x);
    const R d = b.x * b.x + b.y * b.y;
    C r;
    r.x = (a.x * b.x + a.y * b.y) / d;
    r.y = (a.y * b.x - a.x * b.y) / d;
    return r;
}

// ------------------------------------------------------------------ GEMM
// C = beta C + alpha A B (alpha, beta real); A m x k (lda), B k x n (ldb).
// 64 x 64 tile per block of 256 threads, each thread 4 x 4 complex outputs at
// rows tx + 16 i and columns ty + 16 j; k in steps of 8 through two shared
// buffers, the next step's tile loaded into registers while this one is used.
constexpr int GB_M = 64, GB_N = 64, GB_K = 8;

template <typename C>
__global__ void __launch_bounds__(256) k_zgemm(int m, int n, int k, double alpha, const C *__restrict__ A, long lda,
                                               const C *__restrict__ B, long ldb, double beta, C *Cm, long ldc)
{
    using R = decltype(C{}.x);
    __shared__ C As[2][GB_K][GB_M];
    __shared__ C Bs[2][GB_K][GB_N];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    // loader mapping: A rows (tid % 64) at k-columns (tid / 64) and +4; B k-rows
    // (tid % 8) at columns (tid / 8) and +32
    const int la_r = tid % 64, la_k = tid / 64, lb_k = tid % 8, lb_c = tid / 8;
    C ra[2], rb[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = m0 + la_r, kk = k0 + la_k + 4 * h;
            ra[h] = (r < m && kk < k) ? A[(long)kk * lda + r] : czero<C>();
            const int kb = k0 + lb_k, cc = n0 + lb_c + 32 * h;
            rb[h] = (kb < k && cc < n) ? B[(long)cc * ldb + kb] : czero<C>();
        }
    };
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
    const int nk = (k + GB_K - 1) / GB_K;
    if (nk > 0) load(0);
    for (int s = 0; s < nk; ++s) {
        const int buf = s & 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            As[buf][la_k + 4 * h][la_r] = ra[h];
            Bs[buf][lb_k][lb_c + 32 * h] = rb[h];
        }
        __syncthreads();
        if (s + 1 < nk) load((s + 1) * GB_K);
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int cc = n0 + ty + 16 * j;
        if (cc >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = m0 + tx + 16 * i;
            if (r >= m) continue;
            C *dst = Cm + (long)cc * ldc + r;
            C v;
            v.x = (R)alpha * acc[i][j].x;
            v.y = (R)alpha * acc[i][j].y;
            if (beta != 0.0) {
                const C o = *dst;
                v.x += (R)beta * o.x;
                v.y += (R)beta * o.y;
            }
            *dst = v;
        }
    }
}

// ------------------------------------------------------- grid barrier
// Bounded barrier across the blocks of a cooperative launch (all blocks are
// co-resident): the last block to arrive resets the count and advances the
// generation; the others poll the generation with a sleep, up to GJ_SPIN polls,
// after which the barrier records error 4 in *err and reports failure, and the
// caller returns (every later barrier of the other blocks then expires too).
constexpr long GJ_SPIN = 1L << 24;

struct GridBar {
    unsigned *count, *gen;
    int *err;
};

__device__ bool grid_barrier(const GridBar &gb, unsigned nblocks)
{
    __shared__ int ok_s;
    __syncthreads();
    if (nblocks == 1) return true; // one block: the block barrier is the grid barrier
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = *(volatile unsigned *)gb.gen;
        __threadfence();
        if (atomicAdd(gb.count, 1u) == nblocks - 1) {
            *(volatile unsigned *)gb.count = 0;
            __threadfence();
            atomicAdd(gb.gen, 1u);
        } else {
            long it = 0;
            while (*(volatile unsigned *)gb.gen == g) {
                if (++it > GJ_SPIN) { ok = 0; atomicExch(gb.err, 4); break; }
                if (it > 4096) __nanosleep(64); // short waits poll without sleeping
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ------------------------------------------------------------ GJ panel
constexpr int GJ_NB = 32, GJ_THREADS = 512;
static_assert(GJ_NB == 32, "the row operations map one panel column to each lane");

struct GjScratch {
    double *cval; // [2][G] best |a_ij| of each block (-1: no candidate)
    int *cidx;    // [2][G] its row
    void *prow;   // [GJ_NB] the pivot row's panel entries
    int *used;    // [m] 1 once a row has been a pivot
    int *pivrow;  // [m] pivot row of column j
    int *raised;  // pivots raised to the floor
};

// Eliminate columns [k, k + kb) on all m rows of S (ld lds); this block holds
// rows [r0, r0 + nr) of the panel in shared memory.
template <typename C>
__global__ void __launch_bounds__(GJ_THREADS) k_gj_panel(C *S, long lds, int m, int k, int kb, int rows_per_block,
                                                        double tau, const unsigned long long *amax, GjScratch sc,
                                                        GridBar gb)
{
    const double floor_abs = tau * __longlong_as_double((long long)__ldcg(amax));
    using R = decltype(C{}.x);
    extern __shared__ unsigned char smem_raw[];
    C *sp = reinterpret_cast<C *>(smem_raw);                    // [rows_per_block][GJ_NB]
    C *cv = sp + (long)rows_per_block * GJ_NB;                 // [rows_per_block] the column entries
    int *usedl = reinterpret_cast<int *>(cv + rows_per_block); // [rows_per_block]
    __shared__ R rv[GJ_THREADS / 32];
    __shared__ int ri[GJ_THREADS / 32];
    __shared__ int piv_s;
    const int G = gridDim.x, blk = blockIdx.x;
    const int r0 = blk * rows_per_block, nr = max(0, min(rows_per_block, m - r0));
    for (int e = threadIdx.x; e < nr * kb; e += blockDim.x) {
        const int i = e % nr, cc = e / nr; // consecutive threads read consecutive rows
        sp[i * GJ_NB + cc] = S[(long)(k + cc) * lds + r0 + i];
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) usedl[i] = sc.used[r0 + i];
    __syncthreads();
    C *prow = reinterpret_cast<C *>(sc.prow);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ C prs[GJ_NB]; // the pivot row's panel entries, scaled by 1/d (entry jj: 1/d)
    for (int jj = 0; jj < kb; ++jj) {
        // 1. this block's best unused row for column jj (squared magnitudes compared,
        // in the factor's own precision)
        R best = -1;
        int bidx = -1;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            if (usedl[i]) continue;
            const C a = sp[i * GJ_NB + jj];
            const R v = a.x * a.x + a.y * a.y;
            if (v > best || (v == best && r0 + i < bidx)) { best = v; bidx = r0 + i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ov > best || (ov == best && oi >= 0 && (bidx < 0 || oi < bidx))) { best = ov; bidx = oi; }
        }
        if (lane == 0) { rv[wid] = best; ri[wid] = bidx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < GJ_THREADS / 32; ++w)
                if (rv[w] > best || (rv[w] == best && ri[w] >= 0 && (bidx < 0 || ri[w] < bidx))) { best = rv[w]; bidx = ri[w]; }
            if (G == 1) {
                piv_s = bidx;
            } else {
                sc.cval[(jj & 1) * G + blk] = (double)best;
                sc.cidx[(jj & 1) * G + blk] = bidx;
                __threadfence();
            }
        }
        if (G > 1) {
            if (!grid_barrier(gb, G)) return;
            // 2. the pivot row: best over the blocks (warp 0 reads the candidates in parallel)
            if (wid == 0) {
                double bv = -1.0;
                int bi = -1;
                for (int g = lane; g < G; g += 32) {
                    const double v = __ldcg(&sc.cval[(jj & 1) * G + g]);
                    const int ix = __ldcg(&sc.cidx[(jj & 1) * G + g]);
                    if (ix >= 0 && (v > bv || (v == bv && ix < bi))) { bv = v; bi = ix; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (oi >= 0 && (ov > bv || (ov == bv && (bi < 0 || oi < bi)))) { bv = ov; bi = oi; }
                }
                if (lane == 0) piv_s = bi;
            }
        }
        __syncthreads();
        const int p = piv_s; // always >= 0: column j has m - j > 0 unused rows
        const bool own = p >= r0 && p < r0 + nr;
        if (own) {
            for (int cc = threadIdx.x; cc < kb; cc += blockDim.x) {
                const C v = sp[(p - r0) * GJ_NB + cc];
                prs[cc] = v;
                if (G > 1) prow[cc] = v;
            }
            if (threadIdx.x == 0) {
                usedl[p - r0] = 1;
                sc.used[p] = 1;
                sc.pivrow[k + jj] = p;
            }
            if (G > 1) __threadfence();
        }
        if (G > 1) {
            if (!grid_barrier(gb, G)) return;
            if (!own)
                for (int cc = threadIdx.x; cc < kb; cc += blockDim.x) prs[cc] = __ldcg(&prow[cc]);
        }
        __syncthreads();
        // 3. pivot (raised to the floor if tiny), scaled pivot row, row operations
        C d = prs[jj];
        const R ad2 = d.x * d.x + d.y * d.y, fl = (R)floor_abs;
        if (ad2 < fl * fl) { // rare: the static pivot floor
            const R ad = sqrt(ad2);
            const R sx = ad > 0 ? d.x / ad : (R)1, sy = ad > 0 ? d.y / ad : (R)0;
            d.x = fl * sx;
            d.y = fl * sy;
            if (blk == 0 && threadIdx.x == 0) atomicAdd(sc.raised, 1);
        }
        C one;
        one.x = 1;
        one.y = 0;
        const C inv_d = cdiv_(one, d);
        for (int i = threadIdx.x; i < nr; i += blockDim.x) cv[i] = sp[i * GJ_NB + jj];
        __syncthreads();
        if (threadIdx.x < kb) prs[threadIdx.x] = threadIdx.x == jj ? inv_d : cmul(prs[threadIdx.x], inv_d);
        __syncthreads();
        // one warp per row, lane = panel column (kb <= 32)
        if (lane < kb) {
            const C pr = prs[lane];
            for (int i = wid; i < nr; i += GJ_THREADS / 32) {
                if (r0 + i == p) {
                    sp[i * GJ_NB + lane] = pr;
                } else {
                    const C a = lane == jj ? czero<C>() : sp[i * GJ_NB + lane];
                    const C c = cv[i];
                    C r;
                    r.x = a.x - (c.x * pr.x - c.y * pr.y);
                    r.y = a.y - (c.x * pr.y + c.y * pr.x);
                    sp[i * GJ_NB + lane] = r;
                }
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nr * kb; e += blockDim.x) {
        const int i = e % nr, cc = e / nr;
        S[(long)(k + cc) * lds + r0 + i] = sp[i * GJ_NB + cc];
    }
}

// tmp[jj + kb * c'] = S[p_jj][col(c')], then S[p_jj][col(c')] = 0, over the
// columns c' of [0, k) and [k + kb, m) (c' numbering them in order)
template <typename C>
__global__ void k_gj_gather_rows(C *S, long lds, int m, int k, int kb, const int *__restrict__ pivrow, C *tmp)
{
    const long tot = (long)kb * (m - kb);
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= tot) return;
    const int jj = (int)(gid % kb);
    const int cp = (int)(gid / kb);
    const int col = cp < k ? cp : cp + kb;
    C *a = S + (long)col * lds + pivrow[k + jj];
    tmp[gid] = *a;
    *a = czero<C>();
}

// out[j + c ldo] = S[p_j + q_c lds], q the inverse of p (q[p_j] = j)
template <typename C>
__global__ void k_gj_unpermute(const C *__restrict__ S, long lds, int m, const int *__restrict__ pivrow,
                               const int *__restrict__ q, C *out, long ldo)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)m * m) return;
    const int j = (int)(gid % m), c = (int)(gid / m);
    out[(long)c * ldo + j] = S[(long)q[c] * lds + pivrow[j]];
}

__global__ void k_gj_inverse_perm(const int *__restrict__ pivrow, int *q, int m)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) q[pivrow[j]] = j;
}

// max |a_ij| over an m x m block -> *out (as the bits of a non-negative double)
template <typename C>
__global__ void k_absmax(const C *__restrict__ A, long lda, int m, unsigned long long *out)
{
    using R = decltype(C{}.x);
    R mx = 0; // largest |a|^2, in the matrix's precision
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)m * m; e += (long)gridDim.x * blockDim.x) {
        const C a = A[(e / m) * lda + e % m];
        mx = max(mx, a.x * a.x + a.y * a.y);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sqrt((double)mx)));
}

inline unsigned nblk(long c, int t = 256) { return (unsigned)((c + t - 1) / t); }

} // namespace

// -------------------------------------------------------------- host side
struct DenseWork {
    DevBuf ws;
    int max_m = 0, grid = 0, rows = 0;
};

DenseWork *spm_dense_work_new() { return new DenseWork(); }
void spm_dense_work_free(DenseWork *w) { delete w; }

template <typename C>
spm_status spm_dense_gemm(int m, int n, int k, double alpha, const C *A, long lda, const C *B, long ldb, double beta,
                          C *Cm, long ldc, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return SPM_OK;
    dim3 grid((unsigned)((m + GB_M - 1) / GB_M), (unsigned)((n + GB_N - 1) / GB_N));
    k_zgemm<C><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

// out (m x m, ld ldo) = A^{-1}; A (ld lda) is destroyed.  tau: relative pivot
// floor; *raised_dev (device int) accumulates the raised pivots; *err_dev
// (device int) receives 4 when a grid barrier expired.
template <typename C>
spm_status spm_dense_inverse(int m, C *A, long lda, C *out, long ldo, double tau, int *raised_dev, int *err_dev,
                             DenseWork *W, cudaStream_t s)
{
    if (m <= 0) return SPM_OK;
    // grid of the panel kernel: as few blocks as hold the panel's rows in shared
    // memory (up to 768 rows in complex64, 384 in complex128), so that fronts of
    // up to that size need no grid barrier at all; at most one block per SM
    // (cooperative launch: every block co-resident)
    int dev = 0, sms = 0;
    SPM_CUDA_TRY(cudaGetDevice(&dev));
    SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int cap = sizeof(C) == 8 ? 768 : 384;
    int G = (m + cap - 1) / cap;
    if (G > sms) { spm_set_error("Gauss-Jordan: front of %d unknowns is larger than %d blocks of %d rows", m, sms, cap); return SPM_ERR_INVALID_ARG; }
    const int rows = (m + G - 1) / G;
    const size_t smem = sizeof(C) * ((size_t)rows * GJ_NB + rows) + sizeof(int) * rows + 16;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gj_panel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    int per_sm = 0;
    SPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_panel<C>, GJ_THREADS, smem));
    if (per_sm * sms < G) { spm_set_error("Gauss-Jordan panel: %d blocks cannot be co-resident", G); return SPM_ERR_CUDA; }
    // workspace, every piece on a 256-byte boundary: cval[2G] doubles, cidx[2G],
    // prow[NB], used[m], pivrow[m], q[m], barrier words, absmax, tmp[NB x m]
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_cval = up(sizeof(double) * 2 * G), b_cidx = up(sizeof(int) * 2 * G), b_prow = up(sizeof(C) * GJ_NB),
                 b_int = up(sizeof(int) * (size_t)m), b_bar = 256, b_tmp = up(sizeof(C) * (size_t)GJ_NB * m);
    const size_t bytes = b_cval + b_cidx + b_prow + 3 * b_int + b_bar + b_tmp;
    SPM_TRY(W->ws.ensure(bytes));
    char *p = W->ws.as<char>(); // cudaMalloc: 256-byte aligned
    GjScratch sc;
    sc.cval = reinterpret_cast<double *>(p); p += b_cval;
    sc.cidx = reinterpret_cast<int *>(p); p += b_cidx;
    sc.prow = p; p += b_prow;
    sc.used = reinterpret_cast<int *>(p); p += b_int;
    sc.pivrow = reinterpret_cast<int *>(p); p += b_int;
    int *q = reinterpret_cast<int *>(p); p += b_int;
    GridBar gb;
    gb.count = reinterpret_cast<unsigned *>(p);         // bytes 0..3
    gb.gen = gb.count + 1;                              // bytes 4..7
    unsigned long long *amax = reinterpret_cast<unsigned long long *>(p + 64); // 8-byte aligned
    p += b_bar;
    C *tmp = reinterpret_cast<C *>(p);
    gb.err = err_dev;
    sc.raised = raised_dev;
    SPM_CUDA_TRY(cudaMemsetAsync(sc.used, 0, sizeof(int) * (size_t)m, s));
    SPM_CUDA_TRY(cudaMemsetAsync(gb.count, 0, 128, s)); // barrier words and absmax
    k_absmax<C><<<std::min(nblk((long)m * m), 1024u), 256, 0, s>>>(A, lda, m, amax);
    for (int k = 0; k < m; k += GJ_NB) {
        const int kb = std::min(GJ_NB, m - k);
        C *Sarg = A;
        long ldsarg = lda;
        int marg = m, karg = k, kbarg = kb, rowsarg = rows;
        double tauarg = tau;
        const unsigned long long *amaxarg = amax;
        void *args[] = {&Sarg, &ldsarg, &marg, &karg, &kbarg, &rowsarg, &tauarg, &amaxarg, &sc, &gb};
        SPM_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_gj_panel<C>, dim3(G), dim3(GJ_THREADS), args, smem, s));
        if (m > kb) {
            const long tot = (long)kb * (m - kb);
            k_gj_gather_rows<C><<<nblk(tot), 256, 0, s>>>(A, lda, m, k, kb, sc.pivrow, tmp);
            // columns [0, k): tmp columns [0, k); columns [k + kb, m): tmp columns [k, m - kb)
            if (k > 0) SPM_TRY(spm_dense_gemm<C>(m, k, kb, 1.0, A + (long)k * lda, lda, tmp, kb, 1.0, A, lda, s));
            if (k + kb < m)
                SPM_TRY(spm_dense_gemm<C>(m, m - k - kb, kb, 1.0, A + (long)k * lda, lda, tmp + (long)k * kb, kb, 1.0,
                                          A + (long)(k + kb) * lda, lda, s));
        }
    }
    k_gj_inverse_perm<<<nblk(m), 256, 0, s>>>(sc.pivrow, q, m);
    k_gj_unpermute<C><<<nblk((long)m * m), 256, 0, s>>>(A, lda, m, sc.pivrow, q, out, ldo);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

template spm_status spm_dense_gemm<float2>(int, int, int, double, const float2 *, long, const float2 *, long, double,
                                           float2 *, long, cudaStream_t);
template spm_status spm_dense_gemm<double2>(int, int, int, double, const double2 *, long, const double2 *, long, double,
                                            double2 *, long, cudaStream_t);
template spm_status spm_dense_inverse<float2>(int, float2 *, long, float2 *, long, double, int *, int *, DenseWork *,
                                              cudaStream_t);
template spm_status spm_dense_inverse<double2>(int, double2 *, long, double2 *, long, double, int *, int *, DenseWork *,
                                               cudaStream_t);
