// Sparse system S of the sparsifying preconditioner (Section 3.1):
// row (i,c), column (f,j), j in tau_i, o = j - i,
//   S[(i,c),(f,j)] = alpha[(f,o),c] + beta[(f,o),c] m_j + beta[(3,o),c] p^f_j
// (Eq. nbr_i_block_alpha_approx with "approximately equal" replaced by "=").
// Storage: S[i][s][c][f], s = (o3+1)*9 + (o2+1)*3 + (o1+1) over the 27 offsets
// o in [-1,1]^3; slots outside the class neighbourhood hold zeros.
#include "common.cuh"

namespace {

__device__ __forceinline__ int cls_dim(int i, int n) { return i == 0 ? 0 : (i == n - 1 ? 2 : 1); }

// index of offset o within the class neighbourhood enumeration (o3, o2, o1 ascending), or -1
__device__ __forceinline__ int tau_index(int c1, int c2, int c3, int o1, int o2, int o3, int *T)
{
    int lo1 = c1 == 0 ? 0 : -1, hi1 = c1 == 2 ? 0 : 1;
    int lo2 = c2 == 0 ? 0 : -1, hi2 = c2 == 2 ? 0 : 1;
    int lo3 = c3 == 0 ? 0 : -1, hi3 = c3 == 2 ? 0 : 1;
    int w1 = hi1 - lo1 + 1, w2 = hi2 - lo2 + 1, w3 = hi3 - lo3 + 1;
    *T = w1 * w2 * w3;
    if (o1 < lo1 || o1 > hi1 || o2 < lo2 || o2 > hi2 || o3 < lo3 || o3 > hi3) return -1;
    return ((o3 - lo3) * w2 + (o2 - lo2)) * w1 + (o1 - lo1);
}

__global__ void k_assemble(const double2 *__restrict__ alpha, const double2 *__restrict__ beta,
                           const double2 *__restrict__ m, const double2 *__restrict__ p, double2 *S128,
                           float2 *S64, int n)
{
    const long n3 = (long)n * n * n;
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n3 * 27) return;
    long i = gid / 27;
    int s = (int)(gid - i * 27);
    int o1 = s % 3 - 1, o2 = (s / 3) % 3 - 1, o3 = s / 9 - 1;
    int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
    int c1 = cls_dim(i1, n), c2 = cls_dim(i2, n), c3 = cls_dim(i3, n);
    int cls = c1 + 3 * c2 + 9 * c3;
    int T;
    int oi = tau_index(c1, c2, c3, o1, o2, o3, &T);
    double2 *out = S128 + gid * 9;
    float2 *out32 = S64 + gid * 9;
    if (oi < 0) {
        for (int q = 0; q < 9; ++q) { out[q] = make_double2(0, 0); out32[q] = make_float2(0, 0); }
        return;
    }
    long j = ((long)(i3 + o3) * n + (i2 + o2)) * n + (i1 + o1);
    const double2 *al = alpha + (long)cls * 81 * 3;
    const double2 *be = beta + (long)cls * 108 * 3;
    double2 mj = m[j];
    for (int c = 0; c < 3; ++c)
        for (int f = 0; f < 3; ++f) {
            double2 v = al[(f * T + oi) * 3 + c];
            v = cfma(be[(f * T + oi) * 3 + c], mj, v);
            v = cfma(be[(3 * T + oi) * 3 + c], p[f * n3 + j], v);
            out[c * 3 + f] = v;
            out32[c * 3 + f] = to_c64(v);
        }
}

template <typename C>
__global__ void k_apply_S(const C *__restrict__ S, const C *__restrict__ x, C *__restrict__ y, int n, long total)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const long n3 = (long)n * n * n;
    long b = gid / n3, i = gid - b * n3;
    int i1 = (int)(i % n), i2 = (int)((i / n) % n), i3 = (int)(i / ((long)n * n));
    const C *xb = x + b * 3 * n3;
    C a0 = czero<C>(), a1 = czero<C>(), a2 = czero<C>();
    for (int s = 0; s < 27; ++s) {
        int o1 = s % 3 - 1, o2 = (s / 3) % 3 - 1, o3 = s / 9 - 1;
        int j1 = i1 + o1, j2 = i2 + o2, j3 = i3 + o3;
        if (j1 < 0 || j2 < 0 || j3 < 0 || j1 >= n || j2 >= n || j3 >= n) continue;
        long j = ((long)j3 * n + j2) * n + j1;
        const C *blk = S + (i * 27 + s) * 9;
        C x0 = xb[j], x1 = xb[n3 + j], x2 = xb[2 * n3 + j];
        a0 = cfma(blk[0], x0, cfma(blk[1], x1, cfma(blk[2], x2, a0)));
        a1 = cfma(blk[3], x0, cfma(blk[4], x1, cfma(blk[5], x2, a1)));
        a2 = cfma(blk[6], x0, cfma(blk[7], x1, cfma(blk[8], x2, a2)));
    }
    C *yb = y + b * 3 * n3;
    yb[i] = a0;
    yb[n3 + i] = a1;
    yb[2 * n3 + i] = a2;
}

} // namespace

spm_status spm_assemble_S(spm_problem_s *P)
{
    const int n = P->n;
    const long n3 = (long)n * n * n;
    SPM_TRY(P->S128.ensure(sizeof(double2) * n3 * 27 * 9));
    SPM_TRY(P->S64.ensure(sizeof(float2) * n3 * 27 * 9));
    long total = n3 * 27;
    k_assemble<<<(unsigned)((total + 255) / 256), 256, 0, P->stream>>>(
        P->alpha128.as<double2>(), P->beta128.as<double2>(), P->m128.as<double2>(), P->p128.as<double2>(),
        P->S128.as<double2>(), P->S64.as<float2>(), n);
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->have_S = true;
    return SPM_OK;
}

spm_status spm_apply_S_impl(spm_problem_s *P, int prec, const void *x, void *y, int nrhs, cudaStream_t s)
{
    const int n = P->n;
    long total = (long)nrhs * n * n * n;
    unsigned grid = (unsigned)((total + 255) / 256);
    if (prec == SPM_C128)
        k_apply_S<double2><<<grid, 256, 0, s>>>(P->S128.as<double2>(), (const double2 *)x, (double2 *)y, n, total);
    else
        k_apply_S<float2><<<grid, 256, 0, s>>>(P->S64.as<float2>(), (const float2 *)x, (float2 *)y, n, total);
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

