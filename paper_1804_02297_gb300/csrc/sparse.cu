// Nested-dissection multifrontal LU of the sparse system S (Section 3.1: the
// sparse system "can be solved efficiently by the nested dissection
// algorithm"; complexity in Section 3.3).
//
// Geometric dissection: a box of grid points is cut by one plane normal to its
// longest axis (a line on a 2-D grid); one plane separates because S couples
// only points with ||j - i||_inf <= 1.  The grid, the unknowns per point and the
// block layout of S come from a SparseSys (3-D: n^3 points, 3 unknowns, 27
// neighbours; 2-D variant: n^2 points, 2 unknowns, 9 neighbours).  Node = box B.  Its own unknowns are the separator plane
// (or every point of B for a leaf); its boundary unknowns are the points
// outside B within distance 1 of B, which all lie on ancestor separators.  The
// front is [own; boundary] x [own; boundary]:
//   original rows and columns of the own unknowns are assembled from S,
//   children's Schur complements are extend-added,
//   F11 = P L U (partial pivoting inside the own block),
//   X = F11^{-1} F12,   update = F22 - F21 X  -> parent.
// Each node keeps G = [F11^{-1}; F21 F11^{-1}] (front x own) and X = F11^{-1} F12,
// in the factor's precision or (SPM_C64H) as binary16 pairs scaled per column by
// the column's largest component, which halves the bytes every solve reads.
// Solve, one batched pass per tree level:
//   forward (deepest level first): [y; t] = G w_own, w_own = y, w_bnd -= t
//   backward (root first):         w_own -= X w_bnd.
// Nodes of one level have disjoint own unknowns; their boundaries lie on
// shallower separators, so one launch handles a whole level.  Dense front
// work (dense.cu): F11^{-1} by Gauss-Jordan with partial pivoting, then
// X = F11^{-1} F12, F21 F11^{-1} and the update F22 - F21 X as complex GEMMs;
// assembly, extend-add, the batched level GEMVs, gathers and scatters are
// kernels here.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace {

struct Node {
    int lo[3], hi[3];     // box [lo, hi) of grid points
    int axis = -1, cut = -1; // separator plane (axis, coordinate); -1 for a leaf
    int left = -1, right = -1;
    int nown = 0, nbnd = 0;  // points
    long own_off = 0, bnd_off = 0; // offsets into the point lists
    long map_off = 0;        // offset of the local map over the expanded box
    int elo[3], ehi[3];      // expanded box (B grown by 1, clipped)
    long rel_off = 0;        // offset of the child-bnd -> parent-front map (unknowns)
    long fac_off = 0;        // persistent factor storage (elements)
    long piv_off = 0;        // pivots
    long scale_off = 0;      // per-column scales of G then X (half storage)
    int depth = 0;
};

// ---------------------------------------------------------------- kernels

// Assemble the own rows and own columns of S into a zeroed front (column-major,
// ld = f); unknown (point a, component c) of the front is D a + c.
struct GridDesc {
    int n1, n2, n3, D, nsten;
};

template <typename C>
__global__ void k_front_assemble(C *F, int f, const C *__restrict__ S, const int *__restrict__ own_pts, int nown,
                                 const int *__restrict__ lmap, int e0, int e1, int e2, int ew0, int ew1, GridDesc g)
{
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nown * g.nsten) return;
    const int D = g.D, DD = g.D * g.D;
    int a = gid / g.nsten, s = gid % g.nsten;
    int o1 = s % 3 - 1, o2 = (s / 3) % 3 - 1, o3 = g.nsten == 27 ? s / 9 - 1 : 0;
    int i = own_pts[a];
    int i1 = i % g.n1, i2 = (i / g.n1) % g.n2, i3 = i / (g.n1 * g.n2);
    int j1 = i1 + o1, j2 = i2 + o2, j3 = i3 + o3;
    if (j1 < 0 || j2 < 0 || j3 < 0 || j1 >= g.n1 || j2 >= g.n2 || j3 >= g.n3) return;
    int lj = lmap[((j3 - e2) * ew1 + (j2 - e1)) * ew0 + (j1 - e0)];
    if (lj < 0) return; // neighbour eliminated in a child subtree
    long j = ((long)j3 * g.n2 + j2) * g.n1 + j1;
    const C *blk = S + ((long)i * g.nsten + s) * DD; // rows (i,c), columns (j,f)
    for (int c = 0; c < D; ++c)
        for (int q = 0; q < D; ++q) F[(long)(D * lj + q) * f + D * a + c] = blk[c * D + q];
    if (lj >= nown) { // row of a boundary unknown j, column of own unknown i
        int sr = g.nsten - 1 - s; // offset -o
        const C *bj = S + (j * g.nsten + sr) * DD;
        for (int c = 0; c < D; ++c)
            for (int q = 0; q < D; ++q) F[(long)(D * a + q) * f + D * lj + c] = bj[c * D + q];
    }
}

// ---- batched small fronts: one block per front, the whole front in shared memory
// A front of f unknowns (o3 own first) is assembled from S and the children's
// updates, then swept by Gauss-Jordan over its o3 own pivots with partial
// pivoting among the own rows (explicit row swaps) and the static pivot floor:
// after the sweep the front holds [(P F11)^-1, F11^-1 F12; -F21 (P F11)^-1,
// F22 - F21 F11^-1 F12], from which G = [F11^-1; F21 F11^-1] (columns put back
// in place), X = F11^-1 F12 and the update F22 - F21 X are written out.  The
// same quantities as the per-front path (dense inverse + GEMMs), in one launch
// for every small front of a tree level.
struct BatchFront {
    int own_off, nown, map_off, e0, e1, e2, ew0, ew1, f, o3, nch;
    int ch_bc[2], ch_rel[2];
    long fac_off;
    void *upd;
    const void *ch_upd[2];
};

template <typename C> __device__ __forceinline__ C bdiv(C a, C b)
{
    using R = decltype(a.x);
    const R d = b.x * b.x + b.y * b.y;
    C r;
    r.x = (a.x * b.x + a.y * b.y) / d;
    r.y = (a.y * b.x - a.x * b.y) / d;
    return r;
}

template <typename C>
__global__ void __launch_bounds__(256) k_front_batch(const BatchFront *__restrict__ fronts, const C *__restrict__ S,
                                                     const int *__restrict__ pts, const int *__restrict__ maps,
                                                     const int *__restrict__ rels, GridDesc g, C *fac, double tau,
                                                     int *raised, C *gscratch, long gstride)
{
    using R = decltype(C{}.x);
    extern __shared__ unsigned char smem_raw[];
    const BatchFront fr = fronts[blockIdx.x];
    const int f = fr.f, o3 = fr.o3, b3 = f - o3;
    // the front, f x f column-major (row r, column c at c * f + r): in shared memory,
    // or for larger fronts in this block's slice of a global scratch (then only the
    // pivot row, pivot column and permutation sit in shared memory)
    C *F = gscratch ? gscratch + (long)blockIdx.x * gstride : reinterpret_cast<C *>(smem_raw);
    C *prow = gscratch ? reinterpret_cast<C *>(smem_raw) : F + (long)f * f; // the scaled pivot row
    C *pcol = prow + f;                     // the pivot column before the step
    int *perm = reinterpret_cast<int *>(pcol + f);
    __shared__ R red_v[8];
    __shared__ R s_floor;
    __shared__ int s_p;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < f * f; i += nt) F[i] = czero<C>();
    for (int i = tid; i < o3; i += nt) perm[i] = i;
    __syncthreads();
    const int D = g.D, DD = g.D * g.D;
    const int *own_pts = pts + fr.own_off, *lmap = maps + fr.map_off;
    for (int gid = tid; gid < fr.nown * g.nsten; gid += nt) {
        const int a = gid / g.nsten, s = gid % g.nsten;
        const int o1 = s % 3 - 1, o2 = (s / 3) % 3 - 1, oz = g.nsten == 27 ? s / 9 - 1 : 0;
        const int i = own_pts[a];
        const int i1 = i % g.n1, i2 = (i / g.n1) % g.n2, i3 = i / (g.n1 * g.n2);
        const int j1 = i1 + o1, j2 = i2 + o2, j3 = i3 + oz;
        if (j1 < 0 || j2 < 0 || j3 < 0 || j1 >= g.n1 || j2 >= g.n2 || j3 >= g.n3) continue;
        const int lj = lmap[((j3 - fr.e2) * fr.ew1 + (j2 - fr.e1)) * fr.ew0 + (j1 - fr.e0)];
        if (lj < 0) continue;
        const long j = ((long)j3 * g.n2 + j2) * g.n1 + j1;
        const C *blk = S + ((long)i * g.nsten + s) * DD;
        for (int c = 0; c < D; ++c)
            for (int q = 0; q < D; ++q) F[(long)(D * lj + q) * f + D * a + c] = blk[c * D + q];
        if (lj >= fr.nown) {
            const C *bj = S + (j * g.nsten + (g.nsten - 1 - s)) * DD;
            for (int c = 0; c < D; ++c)
                for (int q = 0; q < D; ++q) F[(long)(D * a + q) * f + D * lj + c] = bj[c * D + q];
        }
    }
    __syncthreads();
    for (int ch = 0; ch < fr.nch; ++ch) { // children one after the other: their maps overlap
        const C *U = reinterpret_cast<const C *>(fr.ch_upd[ch]);
        const int bc = fr.ch_bc[ch];
        const int *rel = rels + fr.ch_rel[ch];
        for (int e = tid; e < bc * bc; e += nt) {
            const C u = U[e];
            C &d = F[(long)rel[e / bc] * f + rel[e % bc]];
            d.x += u.x;
            d.y += u.y;
        }
        __syncthreads();
    }
    // pivot floor: tau times the largest |entry| of F11
    R mx = 0;
    for (int e = tid; e < o3 * o3; e += nt) {
        const C a = F[(long)(e / o3) * f + e % o3];
        mx = max(mx, a.x * a.x + a.y * a.y);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red_v[wid] = mx;
    __syncthreads();
    if (tid == 0) {
        R m2 = red_v[0];
        for (int w = 1; w < nt / 32; ++w) m2 = max(m2, red_v[w]);
        s_floor = (R)(tau * sqrt((double)m2));
    }
    __syncthreads();
    const R fl = s_floor;
    C one;
    one.x = 1;
    one.y = 0;
    for (int k = 0; k < o3; ++k) {
        if (wid == 0) { // the largest |F[i][k]| over the unpivoted own rows, lowest row on ties
            R best = -1;
            int bi = -1;
            for (int i = k + lane; i < o3; i += 32) {
                const C a = F[(long)k * f + i];
                const R v = a.x * a.x + a.y * a.y;
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const R ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ov; bi = oi; }
            }
            if (lane == 0) s_p = bi;
        }
        __syncthreads();
        const int p = s_p;
        if (p != k) {
            for (int c = tid; c < f; c += nt) {
                const C t = F[(long)c * f + p];
                F[(long)c * f + p] = F[(long)c * f + k];
                F[(long)c * f + k] = t;
            }
            if (tid == 0) { const int t = perm[p]; perm[p] = perm[k]; perm[k] = t; }
            __syncthreads();
        }
        C d = F[(long)k * f + k];
        const R ad2 = d.x * d.x + d.y * d.y;
        if (ad2 < fl * fl) { // the static pivot floor
            const R ad = sqrt(ad2);
            const R sx = ad > 0 ? d.x / ad : (R)1, sy = ad > 0 ? d.y / ad : (R)0;
            d.x = fl * sx;
            d.y = fl * sy;
            if (tid == 0) atomicAdd(raised, 1);
        }
        const C inv_d = bdiv(one, d);
        for (int j = tid; j < f; j += nt) {
            prow[j] = j == k ? inv_d : cmul(F[(long)j * f + k], inv_d);
            pcol[j] = F[(long)k * f + j];
        }
        __syncthreads();
        for (int e = tid; e < f * f; e += nt) {
            const int i = e % f, j = e / f;
            C v;
            if (i == k) {
                v = prow[j];
            } else if (j == k) {
                v = cmul(pcol[i], inv_d);
                v.x = -v.x;
                v.y = -v.y;
            } else {
                v = F[e];
                const C pc = pcol[i], pr = prow[j];
                v.x -= pc.x * pr.x - pc.y * pr.y;
                v.y -= pc.x * pr.y + pc.y * pr.x;
            }
            F[e] = v;
        }
        __syncthreads();
    }
    C *G = fac + fr.fac_off; // f x o3, ld f
    for (int e = tid; e < f * o3; e += nt) {
        const int r = e % f, j = e / f;
        C v = F[(long)j * f + r];
        if (r >= o3) { v.x = -v.x; v.y = -v.y; }
        G[(long)perm[j] * f + r] = v;
    }
    C *X = G + (long)f * o3; // o3 x b3, ld o3
    for (int e = tid; e < o3 * b3; e += nt) X[e] = F[(long)(o3 + e / o3) * f + e % o3];
    C *U = reinterpret_cast<C *>(fr.upd); // b3 x b3, ld b3
    for (int e = tid; e < b3 * b3; e += nt) U[e] = F[(long)(o3 + e / b3) * f + o3 + e % b3];
}

template <typename C>
__global__ void k_extend_add(C *F, int f, const C *__restrict__ U, int bc, const int *__restrict__ rel)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)bc * bc) return;
    int r = (int)(gid % bc), c = (int)(gid / bc);
    long dst = (long)rel[c] * f + rel[r];
    C u = U[gid], v = F[dst];
    v.x += u.x;
    v.y += u.y;
    F[dst] = v;
}

// copy an (m x n) block between column-major matrices
template <typename C>
__global__ void k_copy_block(C *dst, int ldd, const C *__restrict__ src, int lds, int m, int ncol)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)m * ncol) return;
    int r = (int)(gid % m), c = (int)(gid / m);
    dst[(long)c * ldd + r] = src[(long)c * lds + r];
}

template <typename C> __global__ void k_zero(C *a, long cnt)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < cnt) { a[gid].x = 0; a[gid].y = 0; }
}

inline unsigned blocks(long cnt, int t = 256) { return (unsigned)((cnt + t - 1) / t); }

// n x n identity in a column-major block with leading dimension ld
template <typename C> __global__ void k_identity(C *a, int n, int ld)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)n * n) return;
    int r = (int)(gid % n), c = (int)(gid / n);
    a[(long)c * ld + r].x = r == c ? 1 : 0;
    a[(long)c * ld + r].y = 0;
}

// Level tables.  Per node of a level: its matrix (rows x cols, column-major,
// ld = rows) at mat_off; packed input block (cols x nrhs) at in_unit * nrhs and
// output block (rows x nrhs) at out_unit * nrhs, in_unit / out_unit being prefix
// sums of cols / rows over the level.
struct LevelNode {
    long mat_off, in_unit, out_unit, scale_off;
    int rows, cols;
    int own_pts, bnd_pts; // offsets into the point list
    int nown, nbnd;
};
struct Tile {
    int node, row0, col0;
};
constexpr int GT_ROWS = 256, GT_COLS = 256;

// out[node] += M[node][row0:+256, col0:+256] * in[node][col0:+256, :]; GT_NB
// right-hand sides per pass over the tile (1 for a single RHS; 4, 8 or 16 for
// blocks, by block size and precision).
// S = C: stored as is; S = __half2: binary16 pairs, column c scaled by scale[c].
__device__ __forceinline__ float2 load_as(const float2 *p) { return *p; }
__device__ __forceinline__ double2 load_as(const double2 *p) { return *p; }
__device__ __forceinline__ float2 load_as(const __half2 *p) { return __half22float2(*p); }

template <typename C, int GT_NB, typename S>
__global__ void __launch_bounds__(GT_ROWS) k_level_gemv(const S *__restrict__ M, const float *__restrict__ scales,
                                                        const LevelNode *__restrict__ nodes,
                                                        const Tile *__restrict__ tiles, const C *__restrict__ in,
                                                        C *out, int nrhs)
{
    using R = decltype(C{}.x);
    __shared__ C xs[GT_COLS * GT_NB];
    const Tile tl = tiles[blockIdx.x];
    const LevelNode nd = nodes[tl.node];
    const int r = tl.row0 + threadIdx.x;
    const int ncol = min(GT_COLS, nd.cols - tl.col0);
    const C *inb = in + nd.in_unit * nrhs;
    C *outb = out + nd.out_unit * nrhs;
    constexpr bool SCALED = !std::is_same<S, C>::value;
    for (int b0 = 0; b0 < nrhs; b0 += GT_NB) {
        const int nb = min(GT_NB, nrhs - b0);
        __syncthreads();
        for (int i = threadIdx.x; i < GT_COLS * GT_NB; i += blockDim.x) {
            int c = i % GT_COLS, b = i / GT_COLS;
            C v;
            v.x = 0;
            v.y = 0;
            if (c < ncol && b < nb) {
                v = inb[(long)(b0 + b) * nd.cols + tl.col0 + c];
                if constexpr (SCALED) {
                    const R sc = (R)scales[nd.scale_off + tl.col0 + c];
                    v.x *= sc;
                    v.y *= sc;
                }
            }
            xs[i] = v;
        }
        __syncthreads();
        if (r < nd.rows) {
            R ax[GT_NB], ay[GT_NB];
#pragma unroll
            for (int b = 0; b < GT_NB; ++b) { ax[b] = 0; ay[b] = 0; }
            const S *col = M + nd.mat_off + (long)tl.col0 * nd.rows + r;
            constexpr int UNR = SCALED ? 16 : 4; // 4-byte elements: more loads in flight
#pragma unroll UNR
            for (int c = 0; c < ncol; ++c) {
                const C g = load_as(col + (long)c * nd.rows);
#pragma unroll
                for (int b = 0; b < GT_NB; ++b) {
                    C xv = xs[b * GT_COLS + c];
                    ax[b] += g.x * xv.x - g.y * xv.y;
                    ay[b] += g.x * xv.y + g.y * xv.x;
                }
            }
#pragma unroll
            for (int b = 0; b < GT_NB; ++b) {
                if (b >= nb) break;
                C *o = outb + (long)(b0 + b) * nd.rows + r;
                atomicAdd(&o->x, ax[b]);
                atomicAdd(&o->y, ay[b]);
            }
        }
    }
}

// scale[c] = largest |component| of column c of an (m x ncol, ld m) block (1 if zero)
__global__ void k_col_scales(const float2 *__restrict__ a, int m, int ncol, float *scale)
{
    const int c = blockIdx.x;
    float mx = 0.f;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        float2 v = a[(long)c * m + r];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        scale[c] = t > 0.f ? t : 1.f;
    }
}

// dst = src / scale[column] as binary16 pairs
__global__ void k_to_half(__half2 *dst, const float2 *__restrict__ src, int m, int ncol,
                          const float *__restrict__ scale)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)m * ncol) return;
    const float inv = 1.f / scale[gid / m];
    const float2 v = src[gid];
    dst[gid] = __floats2half2_rn(v.x * inv, v.y * inv);
}

// node whose element range [unit[i] * nrhs, unit[i+1] * nrhs) holds gid
__device__ __forceinline__ int find_node(const long *__restrict__ unit, int nn, long gid, int nrhs)
{
    int lo = 0, hi = nn - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (unit[mid] * nrhs <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// packed input of every node of a level: own (which = 0) or boundary (1) unknowns of w
template <typename C>
__global__ void k_level_gather(C *packed, const C *__restrict__ w, const LevelNode *__restrict__ nodes,
                               const long *__restrict__ in_units, const int *__restrict__ pts, int nn, long npts,
                               int D, int nrhs, int which)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= in_units[nn] * nrhs) return;
    const int id = find_node(in_units, nn, gid, nrhs);
    const LevelNode nd = nodes[id];
    long e = gid - in_units[id] * nrhs;
    long r = e % nd.cols, b = e / nd.cols;
    int pt = pts[(which ? nd.bnd_pts : nd.own_pts) + (int)(r / D)];
    packed[gid] = w[(b * D + (r % D)) * npts + pt];
}

// forward (mode 0): w_own = out[0:o3], w_bnd -= out[o3:] (siblings share
// boundaries: atomic); backward (mode 1): w_own -= out
template <typename C>
__global__ void k_level_scatter(C *w, const C *__restrict__ packed, const LevelNode *__restrict__ nodes,
                                const long *__restrict__ out_units, const int *__restrict__ pts, int nn, long npts,
                                int D, int nrhs, int mode)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= out_units[nn] * nrhs) return;
    const int id = find_node(out_units, nn, gid, nrhs);
    const LevelNode nd = nodes[id];
    long e = gid - out_units[id] * nrhs;
    long r = e % nd.rows, b = e / nd.rows;
    C v = packed[gid];
    const int o3 = D * nd.nown;
    if (r < o3) {
        long g = (b * D + (r % D)) * npts + pts[nd.own_pts + (int)(r / D)];
        if (mode == 0) {
            w[g] = v;
        } else {
            C u = w[g];
            u.x -= v.x;
            u.y -= v.y;
            w[g] = u;
        }
    } else {
        long rb = r - o3;
        long g = (b * D + (rb % D)) * npts + pts[nd.bnd_pts + (int)(rb / D)];
        atomicAdd(&w[g].x, -v.x);
        atomicAdd(&w[g].y, -v.y);
    }
}

} // namespace

// ---------------------------------------------------------------- factor object

struct NDFactor {
    int prec = 0;
    int variant = 0;         // nested-dissection tree variant (cut offsets)
    int raised_pivots = 0;   // pivots raised by the static perturbation
    size_t stored_bytes = 0; // bytes of the stored blocks (G and X, plus half-storage scales)
    bool half_store = false; // blocks as scaled binary16 pairs (complex64 factor only)
    DevBuf scales;           // per-column scales (half storage)
    int D = 3;               // unknowns per point
    long npts = 0;           // grid points
    std::vector<Node> nodes; // post-order
    DevBuf pts, maps, rels;  // int lists
    DevBuf fac;              // persistent: per node [F11;F21] (f x nown3) then X (nown3 x nbnd3)
    DevBuf piv;
    DevBuf front, stack, work, info; // factor scratch (released after factoring)
    DevBuf solve_ws;
    size_t max_front_unknowns = 0, max_own3 = 0, max_bnd3 = 0;
    // level tables for the batched solve; levels[0] is the deepest
    struct Level {
        int nn_f, nn_b;                // nodes in the forward / backward tables
        long nodes_f, nodes_b;         // offsets into the LevelNode table
        long units_f_in, units_f_out, units_b_in, units_b_out; // offsets into the unit table (nn+1 each)
        long tiles_f, tiles_b;         // offsets into the tile table
        int ntiles_f, ntiles_b;
        long pack_f_in, pack_f_out, pack_b_in, pack_b_out; // packed sizes per RHS
    };
    std::vector<Level> levels;
    DevBuf lv_nodes, lv_units, lv_tiles;
    long max_pack_in = 0, max_pack_out = 0;
    DenseWork *dense = nullptr; // Gauss-Jordan workspace
    ~NDFactor()
    {
        spm_dense_work_free(dense);
        pts.release(); maps.release(); rels.release(); fac.release(); piv.release();
        front.release(); stack.release(); work.release(); info.release(); solve_ws.release();
        lv_nodes.release(); lv_units.release(); lv_tiles.release(); scales.release();
    }
};

void spm_factor_free(NDFactor *f) { delete f; }


namespace {

constexpr int LEAF_SIDE = 5;

// Separator offset of tree variant v at a given depth.  Variant 0 cuts every box
// through its middle plane; the others move the cuts by one plane (all down,
// all up, alternating by depth), so that every box of the tree changes.  A box
// whose restriction of S is nearly singular makes its separator's Schur block
// nearly singular too (det S_box = det S_children * det F11), and the pivots of
// the multifrontal LU stay inside each front, so such a box spoils the factor;
// a different tree has different boxes.
constexpr int TREE_VARIANTS = 4;

// relative floor of the pivots of a front (about the square root of the
// precision's unit roundoff: near-singular boxes only, since S itself is well
// conditioned)
template <typename R> constexpr double pivot_floor() { return sizeof(R) == 8 ? 1e-8 : 1e-4; }
inline int cut_offset(int variant, int depth)
{
    switch (variant) {
    case 1: return -1;
    case 2: return 1;
    case 3: return (depth & 1) ? 1 : -1;
    default: return 0;
    }
}

int build_tree(std::vector<Node> &nodes, const int lo[3], const int hi[3], int variant, int depth = 0)
{
    Node nd;
    nd.depth = depth;
    for (int d = 0; d < 3; ++d) { nd.lo[d] = lo[d]; nd.hi[d] = hi[d]; }
    int axis = 0;
    for (int d = 1; d < 3; ++d) if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
    int len = hi[axis] - lo[axis];
    if (len > LEAF_SIDE) {
        nd.axis = axis;
        int cut = lo[axis] + len / 2 + cut_offset(variant, depth);
        cut = std::max(lo[axis] + 1, std::min(hi[axis] - 2, cut)); // both halves non-empty
        nd.cut = cut;
        int lhi[3] = {hi[0], hi[1], hi[2]}, rlo[3] = {lo[0], lo[1], lo[2]};
        lhi[axis] = nd.cut;
        rlo[axis] = nd.cut + 1;
        nd.left = build_tree(nodes, lo, lhi, variant, depth + 1);
        nd.right = build_tree(nodes, rlo, hi, variant, depth + 1);
    }
    nodes.push_back(nd);
    return (int)nodes.size() - 1;
}

} // namespace

template <typename R>
static spm_status factor_typed(const SparseSys &SY, NDFactor *F, bool half_store, int variant)
{
    using C = typename cplx_of<R>::type;
    const int n1 = SY.dims[0], n2 = SY.dims[1], n3d = SY.dims[2], D = SY.D;
    const GridDesc gd{n1, n2, n3d, D, SY.nsten};
    cudaStream_t s = SY.stream;
    F->D = D;
    F->npts = SY.points();
    F->nodes.clear();
    int lo[3] = {0, 0, 0}, hi[3] = {n1, n2, n3d};
    build_tree(F->nodes, lo, hi, variant);
    F->variant = variant;
    std::vector<Node> &nodes = F->nodes;
    const int NN = (int)nodes.size();

    // point lists and local maps (host)
    std::vector<int> pts, maps;
    for (Node &nd : nodes) {
        nd.own_off = pts.size();
        int olo[3], ohi[3];
        for (int d = 0; d < 3; ++d) { olo[d] = nd.lo[d]; ohi[d] = nd.hi[d]; }
        if (nd.axis >= 0) { olo[nd.axis] = nd.cut; ohi[nd.axis] = nd.cut + 1; }
        for (int z = olo[2]; z < ohi[2]; ++z)
            for (int y = olo[1]; y < ohi[1]; ++y)
                for (int x = olo[0]; x < ohi[0]; ++x) pts.push_back((z * n2 + y) * n1 + x);
        nd.nown = (int)(pts.size() - nd.own_off);
        nd.bnd_off = pts.size();
        for (int d = 0; d < 3; ++d) { nd.elo[d] = std::max(nd.lo[d] - 1, 0); nd.ehi[d] = std::min(nd.hi[d] + 1, hi[d]); }
        for (int z = nd.elo[2]; z < nd.ehi[2]; ++z)
            for (int y = nd.elo[1]; y < nd.ehi[1]; ++y)
                for (int x = nd.elo[0]; x < nd.ehi[0]; ++x) {
                    bool inside = x >= nd.lo[0] && x < nd.hi[0] && y >= nd.lo[1] && y < nd.hi[1] && z >= nd.lo[2] &&
                                  z < nd.hi[2];
                    if (!inside) pts.push_back((z * n2 + y) * n1 + x);
                }
        nd.nbnd = (int)(pts.size() - nd.bnd_off);
        // local map over the expanded box: own -> [0,nown), bnd -> nown + rank, else -1
        nd.map_off = maps.size();
        int ew[3] = {nd.ehi[0] - nd.elo[0], nd.ehi[1] - nd.elo[1], nd.ehi[2] - nd.elo[2]};
        size_t base = maps.size();
        maps.resize(base + (size_t)ew[0] * ew[1] * ew[2], -1);
        auto mi = [&](int p) {
            int x = p % n1, y = (p / n1) % n2, z = p / (n1 * n2);
            return base + ((size_t)(z - nd.elo[2]) * ew[1] + (y - nd.elo[1])) * ew[0] + (x - nd.elo[0]);
        };
        for (int a = 0; a < nd.nown; ++a) maps[mi(pts[nd.own_off + a])] = a;
        for (int b = 0; b < nd.nbnd; ++b) maps[mi(pts[nd.bnd_off + b])] = nd.nown + b;
    }
    // child boundary unknowns -> parent front unknowns
    std::vector<int> rels;
    for (Node &nd : nodes) {
        for (int ch : {nd.left, nd.right}) {
            if (ch < 0) continue;
            Node &c = nodes[ch];
            c.rel_off = rels.size();
            int ew[3] = {nd.ehi[0] - nd.elo[0], nd.ehi[1] - nd.elo[1], nd.ehi[2] - nd.elo[2]};
            for (int b = 0; b < c.nbnd; ++b) {
                int p = pts[c.bnd_off + b];
                int x = p % n1, y = (p / n1) % n2, z = p / (n1 * n2);
                int l = maps[nd.map_off + ((size_t)(z - nd.elo[2]) * ew[1] + (y - nd.elo[1])) * ew[0] + (x - nd.elo[0])];
                if (l < 0) { spm_set_error("nested dissection: child boundary point outside the parent front"); return SPM_ERR_NUMERICAL; }
                for (int q = 0; q < D; ++q) rels.push_back(D * l + q);
            }
        }
    }
    // storage
    F->half_store = half_store;
    long fac_total = 0, piv_total = 0, scale_total = 0;
    std::vector<size_t> upd_size(NN, 0);
    for (int id = 0; id < NN; ++id) {
        Node &nd = nodes[id];
        long o3 = (long)D * nd.nown, b3 = (long)D * nd.nbnd, f = o3 + b3;
        nd.fac_off = fac_total;
        fac_total += f * o3 + o3 * b3;
        nd.piv_off = piv_total;
        piv_total += o3;
        nd.scale_off = scale_total;
        scale_total += f;
        F->max_own3 = std::max(F->max_own3, (size_t)o3);
        F->max_bnd3 = std::max(F->max_bnd3, (size_t)b3);
        upd_size[id] = (size_t)(b3 * b3);
    }
    // Concurrency across fronts.  A subtree whose fronts all have a fully summed
    // block of at most GJ_ONE_BLOCK unknowns (inverted by one block, no grid
    // barrier) is a unit of work; the maximal such subtrees are dealt round-robin
    // to a pool of streams, each stream factoring its subtrees in postorder with
    // its own front, update stack and dense workspace.  A subtree root's update
    // goes to a buffer of its own, where its parent (above the subtrees, factored
    // afterwards on the problem's stream) finds it.
    // Small fronts (f <= BATCH_FMAX, whose whole subtree is small) are factored
    // first, level by level, each level in one launch of k_front_batch; their
    // updates go to buffers of their own.  The stream pool below handles the rest.
    const int BATCH_FMAX_SMEM = sizeof(R) == 8 ? 112 : 160; // whole front in shared memory
    const int BATCH_FMAX = 512;                               // larger fronts: global scratch
    std::vector<char> batched(NN, 0);
    for (int id = 0; id < NN; ++id) { // postorder: children before parents
        const Node &nd = nodes[id];
        bool ok = !half_store && D * (nd.nown + nd.nbnd) <= BATCH_FMAX;
        for (int ch : {nd.left, nd.right})
            if (ch >= 0 && !batched[ch]) ok = false;
        batched[id] = ok ? 1 : 0;
    }
    const size_t one_block = sizeof(R) == 4 ? 768 : 384;
    std::vector<size_t> smax(NN, 0);
    std::vector<int> parent(NN, -1);
    for (int id = 0; id < NN; ++id) { // postorder: children before parents
        const Node &nd = nodes[id];
        smax[id] = batched[id] ? 0 : D * (size_t)nd.nown;
        for (int ch : {nd.left, nd.right})
            if (ch >= 0) { smax[id] = std::max(smax[id], smax[ch]); parent[ch] = id; }
    }
    std::vector<int> group(NN, -1);     // stream slot of the node, -1: above the subtrees
    std::vector<char> sub_root(NN, 0);
    const int NSTREAM = 16;
    int nsub = 0;
    for (int id = 0; id < NN; ++id)
        if (!batched[id] && smax[id] <= one_block && (parent[id] < 0 || smax[parent[id]] > one_block)) {
            sub_root[id] = 1;
            ++nsub;
        }
    {   // deal the subtrees (each a contiguous postorder range ending at its root)
        int k = 0;
        for (int id = 0; id < NN; ++id) {
            if (!sub_root[id]) continue;
            int first = id;
            while (true) { // leftmost descendant = first node of the subtree's range
                const Node &nd = nodes[first];
                if (nd.left >= 0) first = nd.left;
                else if (nd.right >= 0) first = nd.right;
                else break;
            }
            for (int j = first; j <= id; ++j)
                if (!batched[j]) group[j] = k % NSTREAM;
            ++k;
        }
    }
    const int ngroups = std::min(NSTREAM, std::max(nsub, 0)) + 1; // + the problem's stream (slot ngroups - 1)
    auto slot = [&](int id) { return group[id] < 0 ? ngroups - 1 : group[id]; };
    // per-slot workspace sizes: front, update stack (postorder within the slot; a
    // subtree root's update lives in its own buffer), half-storage staging
    std::vector<size_t> g_front(ngroups, 1), g_stack(ngroups, 1), g_now(ngroups, 0), g_gx(ngroups, 1);
    std::vector<size_t> root_upd_off(NN, 0);
    size_t root_upd_total = 0;
    std::vector<size_t> batch_upd_off(NN, 0);
    size_t batch_upd_total = 0;
    for (int id = 0; id < NN; ++id) {
        const Node &nd = nodes[id];
        if (batched[id]) {
            batch_upd_off[id] = batch_upd_total;
            batch_upd_total += upd_size[id];
            continue;
        }
        const size_t o3 = D * (size_t)nd.nown, b3 = D * (size_t)nd.nbnd, f = o3 + b3;
        const int g = slot(id);
        g_front[g] = std::max(g_front[g], f * f);
        g_gx[g] = std::max(g_gx[g], f * o3 + o3 * b3);
        for (int ch : {nd.left, nd.right})
            if (ch >= 0 && !sub_root[ch] && !batched[ch]) g_now[g] -= upd_size[ch];
        if (sub_root[id]) {
            root_upd_off[id] = root_upd_total;
            root_upd_total += upd_size[id];
        } else {
            g_now[g] += upd_size[id];
            g_stack[g] = std::max(g_stack[g], g_now[g]);
        }
    }
    F->max_front_unknowns = 0;
    for (const Node &nd : nodes) F->max_front_unknowns = std::max(F->max_front_unknowns, (size_t)(D * (nd.nown + nd.nbnd)));
    SPM_TRY(F->pts.ensure(sizeof(int) * pts.size()));
    SPM_TRY(F->maps.ensure(sizeof(int) * maps.size()));
    SPM_TRY(F->rels.ensure(sizeof(int) * std::max<size_t>(rels.size(), 1)));
    SPM_CUDA_TRY(cudaMemcpy(F->pts.ptr, pts.data(), sizeof(int) * pts.size(), cudaMemcpyHostToDevice));
    SPM_CUDA_TRY(cudaMemcpy(F->maps.ptr, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice));
    if (!rels.empty())
        SPM_CUDA_TRY(cudaMemcpy(F->rels.ptr, rels.data(), sizeof(int) * rels.size(), cudaMemcpyHostToDevice));
    SPM_TRY(F->fac.ensure((half_store ? sizeof(__half2) : sizeof(C)) * fac_total));
    F->stored_bytes = (half_store ? sizeof(__half2) : sizeof(C)) * (size_t)fac_total +
                      (half_store ? sizeof(float) * (size_t)scale_total : 0);
    if (half_store) SPM_TRY(F->scales.ensure(sizeof(float) * scale_total));
    SPM_TRY(F->info.ensure(sizeof(int) * 3)); // expired grid barrier, unused, raised pivots
    SPM_CUDA_TRY(cudaMemsetAsync(F->info.ptr, 0, sizeof(int) * 3, s));
    const C *Sdev = reinterpret_cast<const C *>(sizeof(R) == 8 ? SY.S128 : SY.S64);
    const int *dpts = F->pts.as<int>(), *dmaps = F->maps.as<int>(), *drels = F->rels.as<int>();
    C *fac = F->fac.as<C>();
    int *dinfo = F->info.as<int>();
    std::vector<const C *> upd_ptr(NN, nullptr); // where each node's update sits
    // the batched levels, deepest first, on the problem's stream
    DevBuf batch_upd, batch_desc;
    {
        SPM_TRY(batch_upd.ensure(sizeof(C) * std::max<size_t>(batch_upd_total, 1)));
        C *bu = batch_upd.as<C>();
        int maxd = 0;
        for (const Node &nd : nodes) maxd = std::max(maxd, nd.depth);
        std::vector<std::vector<BatchFront>> lv(maxd + 1);
        size_t nbf = 0;
        for (int id = 0; id < NN; ++id) {
            if (!batched[id]) continue;
            const Node &nd = nodes[id];
            upd_ptr[id] = bu + batch_upd_off[id];
            BatchFront b;
            b.own_off = (int)nd.own_off;
            b.nown = nd.nown;
            b.map_off = (int)nd.map_off;
            b.e0 = nd.elo[0]; b.e1 = nd.elo[1]; b.e2 = nd.elo[2];
            b.ew0 = nd.ehi[0] - nd.elo[0];
            b.ew1 = nd.ehi[1] - nd.elo[1];
            b.o3 = D * nd.nown;
            b.f = b.o3 + D * nd.nbnd;
            b.fac_off = nd.fac_off;
            b.upd = bu + batch_upd_off[id];
            b.nch = 0;
            for (int ch : {nd.left, nd.right}) {
                if (ch < 0 || nodes[ch].nbnd == 0) continue;
                b.ch_bc[b.nch] = D * nodes[ch].nbnd;
                b.ch_rel[b.nch] = (int)nodes[ch].rel_off;
                b.ch_upd[b.nch] = upd_ptr[ch];
                ++b.nch;
            }
            lv[nd.depth].push_back(b);
            ++nbf;
        }
        if (nbf > 0) {
            // per level: the fronts that fit shared memory, then the larger ones
            SPM_TRY(batch_desc.ensure(sizeof(BatchFront) * nbf));
            std::vector<BatchFront> all;
            struct Launch { size_t first, count; int fm; bool global; };
            std::vector<Launch> launches;
            size_t scratch_max = 0;
            for (int d = maxd; d >= 0; --d) {
                for (int pass = 0; pass < 2; ++pass) {
                    Launch ln{all.size(), 0, 1, pass == 1};
                    for (const BatchFront &b : lv[d])
                        if ((b.f > BATCH_FMAX_SMEM) == (pass == 1)) {
                            all.push_back(b);
                            ++ln.count;
                            ln.fm = std::max(ln.fm, b.f);
                        }
                    if (ln.count == 0) continue;
                    if (ln.global) { // chunks of at most 2 GB of scratch
                        const size_t per = (size_t)ln.fm * ln.fm;
                        const size_t chunk = std::max<size_t>(1, ((size_t)2 << 30) / (sizeof(C) * per));
                        for (size_t c0 = 0; c0 < ln.count; c0 += chunk) {
                            Launch part = ln;
                            part.first = ln.first + c0;
                            part.count = std::min(chunk, ln.count - c0);
                            scratch_max = std::max(scratch_max, part.count * per);
                            launches.push_back(part);
                        }
                    } else {
                        launches.push_back(ln);
                    }
                }
            }
            SPM_CUDA_TRY(cudaMemcpy(batch_desc.ptr, all.data(), sizeof(BatchFront) * nbf, cudaMemcpyHostToDevice));
            DevBuf gscratch;
            if (scratch_max > 0) SPM_TRY(gscratch.ensure(sizeof(C) * scratch_max));
            const size_t smem_max = sizeof(C) * ((size_t)BATCH_FMAX_SMEM * BATCH_FMAX_SMEM + 2 * BATCH_FMAX_SMEM) +
                                    sizeof(int) * BATCH_FMAX_SMEM;
            SPM_CUDA_TRY(cudaFuncSetAttribute(k_front_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
            const GridDesc gd2{n1, n2, n3d, D, SY.nsten};
            for (const Launch &ln : launches) {
                const size_t fm = (size_t)ln.fm;
                const size_t smem = ln.global ? sizeof(C) * 2 * fm + sizeof(int) * fm
                                              : sizeof(C) * (fm * fm + 2 * fm) + sizeof(int) * fm;
                k_front_batch<C><<<(unsigned)ln.count, 256, smem, s>>>(
                    batch_desc.as<BatchFront>() + ln.first, Sdev, dpts, dmaps, drels, gd2, fac, pivot_floor<R>(),
                    dinfo + 2, ln.global ? gscratch.as<C>() : nullptr, (long)(fm * fm));
            }
            SPM_CUDA_TRY(cudaGetLastError());
            if (scratch_max > 0) SPM_CUDA_TRY(cudaStreamSynchronize(s)); // before the scratch is freed
        }
    }
    // per-slot buffers and streams (slot ngroups - 1 is the problem's stream)
    struct Slot {
        DevBuf front, stack, gx;
        DenseWork *dense = nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
        ~Slot()
        {
            spm_dense_work_free(dense);
            if (st) cudaStreamDestroy(st);
            if (done) cudaEventDestroy(done);
        }
    };
    std::vector<Slot> slots(ngroups);
    DevBuf root_upd;
    SPM_TRY(root_upd.ensure(sizeof(C) * std::max<size_t>(root_upd_total, 1)));
    cudaEvent_t start_ev = nullptr;
    SPM_CUDA_TRY(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
    SPM_CUDA_TRY(cudaEventRecord(start_ev, s)); // the streams start after the work queued so far
    for (int g = 0; g < ngroups; ++g) {
        Slot &sl = slots[g];
        SPM_TRY(sl.front.ensure(sizeof(C) * g_front[g]));
        SPM_TRY(sl.stack.ensure(sizeof(C) * g_stack[g]));
        if (half_store) SPM_TRY(sl.gx.ensure(sizeof(C) * g_gx[g]));
        sl.dense = spm_dense_work_new();
        if (g == ngroups - 1) {
            sl.st = nullptr; // use s
        } else {
            SPM_CUDA_TRY(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
            SPM_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
            SPM_CUDA_TRY(cudaStreamWaitEvent(sl.st, start_ev, 0));
        }
    }
    cudaEventDestroy(start_ev);

    std::vector<size_t> top(ngroups, 0);
    auto factor_node = [&](int id) -> spm_status {
        Node &nd = nodes[id];
        const int g = slot(id);
        Slot &sl = slots[g];
        cudaStream_t ss = sl.st ? sl.st : s;
        C *front = sl.front.as<C>(), *stack = sl.stack.as<C>();
        const int o3 = D * nd.nown, b3 = D * nd.nbnd, f = o3 + b3;
        k_zero<C><<<blocks((long)f * f), 256, 0, ss>>>(front, (long)f * f);
        int ew0 = nd.ehi[0] - nd.elo[0], ew1 = nd.ehi[1] - nd.elo[1];
        k_front_assemble<C><<<blocks((long)nd.nown * gd.nsten), 256, 0, ss>>>(front, f, Sdev, dpts + nd.own_off,
                                                                               nd.nown, dmaps + nd.map_off, nd.elo[0],
                                                                               nd.elo[1], nd.elo[2], ew0, ew1, gd);
        // extend-add the children's updates
        for (int ch : {nd.left, nd.right}) {
            if (ch < 0) continue;
            Node &c = nodes[ch];
            int bc = D * c.nbnd;
            if (bc == 0) continue;
            k_extend_add<C><<<blocks((long)bc * bc), 256, 0, ss>>>(front, f, upd_ptr[ch], bc, drels + c.rel_off);
        }
        for (int ch : {nd.left, nd.right})
            if (ch >= 0 && !sub_root[ch] && !batched[ch]) top[g] -= upd_size[ch];
        SPM_CUDA_TRY(cudaGetLastError());
        // F11^{-1} by Gauss-Jordan (partial pivoting inside the own block, static
        // pivot floor), then with G = [F11^{-1}; F21 F11^{-1}] (f x o3, ld f) and
        // X = F11^{-1} F12 (o3 x b3, ld o3) stored after it:
        //   X = F11^{-1} F12,  G_bottom = F21 F11^{-1},  update = F22 - F21 X.
        C *G = half_store ? sl.gx.as<C>() : fac + nd.fac_off;
        SPM_TRY(spm_dense_inverse<C>(o3, front, f, G, f, pivot_floor<R>(), dinfo + 2, dinfo, sl.dense, ss));
        if (b3 > 0) {
            C *X = G + (long)f * o3;
            SPM_TRY(spm_dense_gemm<C>(o3, b3, o3, 1.0, G, f, front + (long)o3 * f, f, 0.0, X, o3, ss));
            SPM_TRY(spm_dense_gemm<C>(b3, o3, o3, 1.0, front + o3, f, G, f, 0.0, G + o3, f, ss));
            SPM_TRY(spm_dense_gemm<C>(b3, b3, o3, -1.0, front + o3, f, X, o3, 1.0, front + (long)o3 * f + o3, f, ss));
            // keep the update: on the slot's stack, or in the subtree root's own buffer
            C *dst = sub_root[id] ? root_upd.as<C>() + root_upd_off[id] : stack + top[g];
            if (!sub_root[id]) top[g] += upd_size[id];
            k_copy_block<C><<<blocks((long)b3 * b3), 256, 0, ss>>>(dst, b3, front + (long)o3 * f + o3, f, b3, b3);
            upd_ptr[id] = dst;
        }
        if constexpr (sizeof(R) == 4) {
            if (half_store) {
                float *sc = F->scales.as<float>() + nd.scale_off;
                __half2 *h = F->fac.as<__half2>() + nd.fac_off;
                const float2 *g2 = reinterpret_cast<const float2 *>(G);
                k_col_scales<<<o3, 256, 0, ss>>>(g2, f, o3, sc);
                k_to_half<<<blocks((long)f * o3), 256, 0, ss>>>(h, g2, f, o3, sc);
                if (b3 > 0) {
                    k_col_scales<<<b3, 256, 0, ss>>>(g2 + (long)f * o3, o3, b3, sc + o3);
                    k_to_half<<<blocks((long)o3 * b3), 256, 0, ss>>>(h + (long)f * o3, g2 + (long)f * o3, o3, b3, sc + o3);
                }
            }
        }
        SPM_CUDA_TRY(cudaGetLastError());
        return SPM_OK;
    };
    // the subtrees on the stream pool, then the nodes above them on the problem's stream
    for (int id = 0; id < NN; ++id)
        if (group[id] >= 0) SPM_TRY(factor_node(id));
    for (int g = 0; g < ngroups - 1; ++g) {
        SPM_CUDA_TRY(cudaEventRecord(slots[g].done, slots[g].st));
        SPM_CUDA_TRY(cudaStreamWaitEvent(s, slots[g].done, 0));
    }
    for (int id = 0; id < NN; ++id)
        if (group[id] < 0 && !batched[id]) SPM_TRY(factor_node(id));
    int hinfo[3] = {0, 0, 0};
    SPM_CUDA_TRY(cudaMemcpyAsync(hinfo, dinfo, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    slots.clear();
    root_upd.release();
    F->raised_pivots = hinfo[2];
    if (hinfo[0] != 0) {
        spm_set_error("a grid barrier of the Gauss-Jordan panel expired (code %d)", hinfo[0]);
        return SPM_ERR_TIMEOUT;
    }
    // level tables for the batched solve
    {
        int maxd = 0;
        for (const Node &nd : nodes) maxd = std::max(maxd, nd.depth);
        std::vector<LevelNode> tn;
        std::vector<long> tu;
        std::vector<Tile> tt;
        F->levels.clear();
        F->max_pack_in = F->max_pack_out = 0;
        auto add_table = [&](const std::vector<int> &ids, bool fwd, int &nn, long &nodes_off, long &uin, long &uout,
                             long &tiles_off, int &ntiles, long &pin, long &pout) {
            nodes_off = (long)tn.size();
            tiles_off = (long)tt.size();
            std::vector<long> ui(1, 0), uo(1, 0);
            nn = 0;
            for (int id : ids) {
                const Node &nd = nodes[id];
                const int o3 = D * nd.nown, b3 = D * nd.nbnd, f = o3 + b3;
                LevelNode L;
                L.rows = fwd ? f : o3;
                L.cols = fwd ? o3 : b3;
                if (L.cols == 0) continue;
                L.mat_off = fwd ? nd.fac_off : nd.fac_off + (long)f * o3;
                L.scale_off = fwd ? nd.scale_off : nd.scale_off + o3;
                L.in_unit = ui.back();
                L.out_unit = uo.back();
                L.own_pts = (int)nd.own_off;
                L.bnd_pts = (int)nd.bnd_off;
                L.nown = nd.nown;
                L.nbnd = nd.nbnd;
                for (int r0 = 0; r0 < L.rows; r0 += GT_ROWS)
                    for (int c0 = 0; c0 < L.cols; c0 += GT_COLS) tt.push_back(Tile{nn, r0, c0});
                tn.push_back(L);
                ui.push_back(ui.back() + L.cols);
                uo.push_back(uo.back() + L.rows);
                ++nn;
            }
            uin = (long)tu.size();
            tu.insert(tu.end(), ui.begin(), ui.end());
            uout = (long)tu.size();
            tu.insert(tu.end(), uo.begin(), uo.end());
            ntiles = (int)(tt.size() - tiles_off);
            pin = ui.back();
            pout = uo.back();
            F->max_pack_in = std::max(F->max_pack_in, pin);
            F->max_pack_out = std::max(F->max_pack_out, pout);
        };
        for (int d = maxd; d >= 0; --d) {
            std::vector<int> ids;
            for (int id = 0; id < NN; ++id) if (nodes[id].depth == d) ids.push_back(id);
            NDFactor::Level lv;
            add_table(ids, true, lv.nn_f, lv.nodes_f, lv.units_f_in, lv.units_f_out, lv.tiles_f, lv.ntiles_f,
                      lv.pack_f_in, lv.pack_f_out);
            add_table(ids, false, lv.nn_b, lv.nodes_b, lv.units_b_in, lv.units_b_out, lv.tiles_b, lv.ntiles_b,
                      lv.pack_b_in, lv.pack_b_out);
            F->levels.push_back(lv);
        }
        SPM_TRY(F->lv_nodes.ensure(sizeof(LevelNode) * tn.size()));
        SPM_TRY(F->lv_units.ensure(sizeof(long) * tu.size()));
        SPM_TRY(F->lv_tiles.ensure(sizeof(Tile) * std::max<size_t>(tt.size(), 1)));
        SPM_CUDA_TRY(cudaMemcpy(F->lv_nodes.ptr, tn.data(), sizeof(LevelNode) * tn.size(), cudaMemcpyHostToDevice));
        SPM_CUDA_TRY(cudaMemcpy(F->lv_units.ptr, tu.data(), sizeof(long) * tu.size(), cudaMemcpyHostToDevice));
        if (!tt.empty())
            SPM_CUDA_TRY(cudaMemcpy(F->lv_tiles.ptr, tt.data(), sizeof(Tile) * tt.size(), cudaMemcpyHostToDevice));
    }
    return SPM_OK;
}

template <typename R>
static spm_status solve_typed(NDFactor *F, const void *bv, void *xv, int nrhs, cudaStream_t s)
{
    using C = typename cplx_of<R>::type;
    const long npts = F->npts;
    const int D = F->D;
    C *x = reinterpret_cast<C *>(xv);
    SPM_CUDA_TRY(cudaMemcpyAsync(x, bv, sizeof(C) * D * npts * nrhs, cudaMemcpyDeviceToDevice, s));
    const size_t pin = (size_t)F->max_pack_in * nrhs, pout = (size_t)F->max_pack_out * nrhs;
    SPM_TRY(F->solve_ws.ensure(sizeof(C) * (pin + pout)));
    C *in = F->solve_ws.as<C>();
    C *out = in + pin;
    const int *dpts = F->pts.as<int>();
    const C *fac = F->fac.as<C>();
    const __half2 *fac16 = F->fac.as<__half2>();
    const float *scales = F->scales.as<float>();
    const LevelNode *tn = F->lv_nodes.as<LevelNode>();
    // right-hand sides per pass over a factor tile: the tile is read once per
    // group, so blocks of many RHS read the factor nrhs / GT_NB times
    auto gemv = [&](int ntiles, const LevelNode *nodes, const Tile *tiles) {
        if constexpr (sizeof(R) == 4) {
            if (F->half_store) {
                if (nrhs == 1) k_level_gemv<C, 1, __half2><<<ntiles, GT_ROWS, 0, s>>>(fac16, scales, nodes, tiles, in, out, nrhs);
                else if (nrhs < 8) k_level_gemv<C, 4, __half2><<<ntiles, GT_ROWS, 0, s>>>(fac16, scales, nodes, tiles, in, out, nrhs);
                else if (nrhs < 16) k_level_gemv<C, 8, __half2><<<ntiles, GT_ROWS, 0, s>>>(fac16, scales, nodes, tiles, in, out, nrhs);
                else k_level_gemv<C, 16, __half2><<<ntiles, GT_ROWS, 0, s>>>(fac16, scales, nodes, tiles, in, out, nrhs);
                return;
            }
            if (nrhs >= 16) {
                k_level_gemv<C, 16, C><<<ntiles, GT_ROWS, 0, s>>>(fac, scales, nodes, tiles, in, out, nrhs);
                return;
            }
        }
        if (nrhs == 1) k_level_gemv<C, 1, C><<<ntiles, GT_ROWS, 0, s>>>(fac, scales, nodes, tiles, in, out, nrhs);
        else if (nrhs < 8) k_level_gemv<C, 4, C><<<ntiles, GT_ROWS, 0, s>>>(fac, scales, nodes, tiles, in, out, nrhs);
        else k_level_gemv<C, 8, C><<<ntiles, GT_ROWS, 0, s>>>(fac, scales, nodes, tiles, in, out, nrhs);
    };
    const long *tu = F->lv_units.as<long>();
    const Tile *tt = F->lv_tiles.as<Tile>();
    const int NL = (int)F->levels.size();
    for (int l = 0; l < NL; ++l) { // forward, deepest level first
        const NDFactor::Level &lv = F->levels[l];
        if (lv.nn_f == 0) continue;
        k_level_gather<C><<<blocks(lv.pack_f_in * nrhs), 256, 0, s>>>(in, x, tn + lv.nodes_f, tu + lv.units_f_in, dpts,
                                                                       lv.nn_f, npts, D, nrhs, 0);
        SPM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(C) * lv.pack_f_out * nrhs, s));
        gemv(lv.ntiles_f, tn + lv.nodes_f, tt + lv.tiles_f);
        k_level_scatter<C><<<blocks(lv.pack_f_out * nrhs), 256, 0, s>>>(x, out, tn + lv.nodes_f, tu + lv.units_f_out,
                                                                         dpts, lv.nn_f, npts, D, nrhs, 0);
    }
    for (int l = NL - 1; l >= 0; --l) { // backward, root first
        const NDFactor::Level &lv = F->levels[l];
        if (lv.nn_b == 0) continue;
        k_level_gather<C><<<blocks(lv.pack_b_in * nrhs), 256, 0, s>>>(in, x, tn + lv.nodes_b, tu + lv.units_b_in, dpts,
                                                                       lv.nn_b, npts, D, nrhs, 1);
        SPM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(C) * lv.pack_b_out * nrhs, s));
        gemv(lv.ntiles_b, tn + lv.nodes_b, tt + lv.tiles_b);
        k_level_scatter<C><<<blocks(lv.pack_b_out * nrhs), 256, 0, s>>>(x, out, tn + lv.nodes_b, tu + lv.units_b_out,
                                                                         dpts, lv.nn_b, npts, D, nrhs, 1);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

namespace {

// probe right-hand side: components uniform in [-1, 1] from a splitmix64 hash of the index
__global__ void k_probe_rhs(double2 *b128, float2 *b64, long N)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    double2 v;
    v.x = (double)(z >> 40) * (2.0 / 16777216.0) - 1.0;
    v.y = (double)((z >> 16) & 0xFFFFFF) * (2.0 / 16777216.0) - 1.0;
    b128[i] = v;
    if (b64) b64[i] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_widen(const float2 *a, double2 *b, long N)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_double2(a[i].x, a[i].y);
}

// acc[0] += sum |y - b|^2, acc[1] += sum |b|^2
__global__ void k_resid_norms(const double2 *y, const double2 *b, long N, double *acc)
{
    __shared__ double s0[256], s1[256];
    double r = 0, q = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double dx = y[i].x - b[i].x, dy = y[i].y - b[i].y;
        r += dx * dx + dy * dy;
        q += b[i].x * b[i].x + b[i].y * b[i].y;
    }
    s0[threadIdx.x] = r;
    s1[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { s0[threadIdx.x] += s0[threadIdx.x + w]; s1[threadIdx.x] += s1[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { atomicAdd(acc, s0[0]); atomicAdd(acc + 1, s1[0]); }
}

// ||S x - b|| / ||b|| for x = S^{-1} b through the factor of precision `prec`,
// with b a fixed pseudo-random vector and S x formed in complex128.
spm_status probe_factor(const SparseSys &SY, int prec, double *relres)
{
    const long N = (long)SY.D * SY.points();
    cudaStream_t s = SY.stream;
    DevBuf buf;
    SPM_TRY(buf.ensure(sizeof(double2) * 3 * N + sizeof(float2) * 2 * N + 2 * sizeof(double)));
    double2 *b = buf.as<double2>(), *x = b + N, *y = x + N;
    float2 *b64 = reinterpret_cast<float2 *>(y + N), *x64 = b64 + N;
    double *acc = reinterpret_cast<double *>(x64 + N);
    const bool single = prec != SPM_C128;
    const unsigned g = (unsigned)((N + 255) / 256);
    k_probe_rhs<<<g, 256, 0, s>>>(b, single ? b64 : nullptr, N);
    if (single) {
        SPM_TRY(spm_nd_solve(*SY.slot64, SPM_C64, b64, x64, 1, s));
        k_widen<<<g, 256, 0, s>>>(x64, x, N);
    } else {
        SPM_TRY(spm_nd_solve(*SY.slot128, SPM_C128, b, x, 1, s));
    }
    SPM_TRY(SY.apply_S128(SY.ctx, x, y, s));
    SPM_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
    k_resid_norms<<<1024, 256, 0, s>>>(y, b, N, acc);
    double h[2];
    SPM_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    *relres = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
    if (!(*relres == *relres)) *relres = HUGE_VAL; // NaN: an unusable factor
    return SPM_OK;
}

// probe residual below which a factor is accepted without trying another tree
// (measured on the n = 48 / 64 media: complex64 factors up to 3e-2 and
// half-storage factors up to 0.3 keep GMRES within a few iterations of the
// best tree; factors above 1 stall it)
double probe_accept(int prec)
{
    return prec == SPM_C128 ? 1e-6 : (prec == SPM_C64H ? 3e-1 : 3e-2);
}

spm_status factor_once(const SparseSys &SY, int prec, int variant, NDFactor *&slot)
{
    spm_factor_free(slot);
    slot = nullptr;
    NDFactor *F = new NDFactor();
    F->prec = prec == SPM_C128 ? SPM_C128 : SPM_C64;
    spm_status st = prec == SPM_C128 ? factor_typed<double>(SY, F, false, variant)
                                     : factor_typed<float>(SY, F, prec == SPM_C64H, variant);
    if (st != SPM_OK) {
        delete F;
        return st;
    }
    slot = F;
    return SPM_OK;
}

} // namespace

// Factor, probe the factor's accuracy, and if the probe residual is above the
// acceptance level try the other tree variants, keeping the most accurate.
spm_status spm_nd_factor(const SparseSys &SY, int prec)
{
    const int fi = prec == SPM_C128 ? 0 : 1;
    NDFactor *&slot = fi == 0 ? *SY.slot128 : *SY.slot64;
    int best_v = -1, attempts = 0;
    double best = HUGE_VAL, last = HUGE_VAL;
    for (int v = 0; v < TREE_VARIANTS; ++v) {
        SPM_TRY(factor_once(SY, prec, v, slot));
        ++attempts;
        SPM_TRY(probe_factor(SY, prec, &last));
        if (last < best) { best = last; best_v = v; }
        if (last <= probe_accept(prec)) break;
    }
    if (best_v != slot->variant) { // a later variant was worse: rebuild the best one
        SPM_TRY(factor_once(SY, prec, best_v, slot));
        ++attempts;
    }
    SY.info[fi].variant = best_v;
    SY.info[fi].attempts = attempts;
    SY.info[fi].raised_pivots = slot->raised_pivots;
    SY.info[fi].stored_bytes = slot->stored_bytes;
    SY.info[fi].probe_relres = best;
    SY.info[fi].half_store = prec == SPM_C64H;
    return SPM_OK;
}

// Factor on one given tree variant (no retry); the probe is still recorded.
spm_status spm_nd_factor_tree(const SparseSys &SY, int prec, int variant)
{
    if (variant < 0 || variant >= TREE_VARIANTS) {
        spm_set_error("tree variant must be in [0, %d)", TREE_VARIANTS);
        return SPM_ERR_INVALID_ARG;
    }
    const int fi = prec == SPM_C128 ? 0 : 1;
    NDFactor *&slot = fi == 0 ? *SY.slot128 : *SY.slot64;
    SPM_TRY(factor_once(SY, prec, variant, slot));
    double r = 0;
    SPM_TRY(probe_factor(SY, prec, &r));
    SY.info[fi].variant = variant;
    SY.info[fi].attempts = 1;
    SY.info[fi].raised_pivots = slot->raised_pivots;
    SY.info[fi].stored_bytes = slot->stored_bytes;
    SY.info[fi].probe_relres = r;
    SY.info[fi].half_store = prec == SPM_C64H;
    return SPM_OK;
}

spm_status spm_nd_solve(NDFactor *F, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    if (!F) { spm_set_error("no factor of S in this precision"); return SPM_ERR_NOT_BUILT; }
    return prec == SPM_C128 ? solve_typed<double>(F, b, x, nrhs, s) : solve_typed<float>(F, b, x, nrhs, s);
}

// ---------------------------------------------------------------- 3-D problem
namespace {
spm_status apply_S128_3d(void *ctx, const void *x, void *y, cudaStream_t s)
{
    return spm_apply_S_impl(static_cast<spm_problem_s *>(ctx), SPM_C128, x, y, 1, s);
}

SparseSys sys_of(spm_problem_s *P)
{
    SparseSys S;
    S.dims[0] = S.dims[1] = S.dims[2] = P->n;
    S.D = 3;
    S.nsten = 27;
    S.S128 = P->S128.ptr;
    S.S64 = P->S64.ptr;
    S.stream = P->stream;
    S.slot128 = &P->fac128;
    S.slot64 = &P->fac64;
    S.info = P->fac_info;
    S.apply_S128 = apply_S128_3d;
    S.ctx = P;
    return S;
}
} // namespace

spm_status spm_factor_impl(spm_problem_s *P, int prec) { return spm_nd_factor(sys_of(P), prec); }

spm_status spm_factor_tree_impl(spm_problem_s *P, int prec, int variant)
{
    return spm_nd_factor_tree(sys_of(P), prec, variant);
}

spm_status spm_solveS_impl(spm_problem_s *P, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    return spm_nd_solve(prec == SPM_C128 ? P->fac128 : P->fac64, prec, b, x, nrhs, s);
}
