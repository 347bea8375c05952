// Nested-dissection multifrontal LU of the sparse system S (Section 3.1: the
// sparse system "can be solved efficiently by the nested dissection
// algorithm"; complexity in Section 3.3).
//
// Geometric dissection: a box of grid points is cut by one plane normal to its
// longest axis; one plane separates because S couples only points with
// ||j - i||_inf <= 1.  Node = box B.  Its own unknowns are the separator plane
// (or every point of B for a leaf); its boundary unknowns are the points
// outside B within distance 1 of B, which all lie on ancestor separators.  The
// front is [own; boundary] x [own; boundary]:
//   original rows and columns of the own unknowns are assembled from S,
//   children's Schur complements are extend-added,
//   F11 = P L U (partial pivoting inside the own block),
//   X = F11^{-1} F12,   update = F22 - F21 X  -> parent.
// Solve: forward y_own = F11^{-1} w_own, w_bnd -= F21 y_own (post-order);
//        backward x_own = y_own - X x_bnd (reverse post-order).
// Dense blocks use cuSOLVER getrf/getrs and cuBLAS gemm; assembly, extend-add
// and the gathers/scatters are kernels here.
#include <cublas_v2.h>
#include <cuComplex.h>
#include <cusolverDn.h>

#include <algorithm>
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
};

template <typename R> struct blas_t;
template <> struct blas_t<float> {
    using C = cuComplex;
    static cusolverStatus_t getrf_ws(cusolverDnHandle_t h, int n, C *A, int lda, int *lw)
    { return cusolverDnCgetrf_bufferSize(h, n, n, A, lda, lw); }
    static cusolverStatus_t getrf(cusolverDnHandle_t h, int n, C *A, int lda, C *ws, int *piv, int *info)
    { return cusolverDnCgetrf(h, n, n, A, lda, ws, piv, info); }
    static cusolverStatus_t getrs(cusolverDnHandle_t h, int n, int nrhs, const C *A, int lda, const int *piv, C *B,
                                  int ldb, int *info)
    { return cusolverDnCgetrs(h, CUBLAS_OP_N, n, nrhs, A, lda, piv, B, ldb, info); }
    static cublasStatus_t gemm(cublasHandle_t h, int m, int n, int k, C alpha, const C *A, int lda, const C *B, int ldb,
                               C beta, C *Cm, int ldc)
    { return cublasCgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &alpha, A, lda, B, ldb, &beta, Cm, ldc); }
    static C one() { return make_cuComplex(1.f, 0.f); }
    static C mone() { return make_cuComplex(-1.f, 0.f); }
};
template <> struct blas_t<double> {
    using C = cuDoubleComplex;
    static cusolverStatus_t getrf_ws(cusolverDnHandle_t h, int n, C *A, int lda, int *lw)
    { return cusolverDnZgetrf_bufferSize(h, n, n, A, lda, lw); }
    static cusolverStatus_t getrf(cusolverDnHandle_t h, int n, C *A, int lda, C *ws, int *piv, int *info)
    { return cusolverDnZgetrf(h, n, n, A, lda, ws, piv, info); }
    static cusolverStatus_t getrs(cusolverDnHandle_t h, int n, int nrhs, const C *A, int lda, const int *piv, C *B,
                                  int ldb, int *info)
    { return cusolverDnZgetrs(h, CUBLAS_OP_N, n, nrhs, A, lda, piv, B, ldb, info); }
    static cublasStatus_t gemm(cublasHandle_t h, int m, int n, int k, C alpha, const C *A, int lda, const C *B, int ldb,
                               C beta, C *Cm, int ldc)
    { return cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &alpha, A, lda, B, ldb, &beta, Cm, ldc); }
    static C one() { return make_cuDoubleComplex(1.0, 0.0); }
    static C mone() { return make_cuDoubleComplex(-1.0, 0.0); }
};

// ---------------------------------------------------------------- kernels

// Assemble the own rows and own columns of S into a zeroed front (column-major, ld = f).
template <typename C>
__global__ void k_front_assemble(C *F, int f, const C *__restrict__ S, const int *__restrict__ own_pts, int nown,
                                 const int *__restrict__ lmap, int e0, int e1, int e2, int ew0, int ew1, int n)
{
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nown * 27) return;
    int a = gid / 27, s = gid % 27;
    int o1 = s % 3 - 1, o2 = (s / 3) % 3 - 1, o3 = s / 9 - 1;
    int i = own_pts[a];
    int i1 = i % n, i2 = (i / n) % n, i3 = i / (n * n);
    int j1 = i1 + o1, j2 = i2 + o2, j3 = i3 + o3;
    if (j1 < 0 || j2 < 0 || j3 < 0 || j1 >= n || j2 >= n || j3 >= n) return;
    int lj = lmap[((j3 - e2) * ew1 + (j2 - e1)) * ew0 + (j1 - e0)];
    if (lj < 0) return; // neighbour eliminated in a child subtree
    long j = ((long)j3 * n + j2) * n + j1;
    const C *blk = S + ((long)i * 27 + s) * 9; // rows (i,c), columns (j,f)
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 3; ++q) F[(long)(3 * lj + q) * f + 3 * a + c] = blk[c * 3 + q];
    if (lj >= nown) { // row of a boundary unknown j, column of own unknown i
        int sr = 26 - s; // offset -o
        const C *bj = S + (j * 27 + sr) * 9;
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < 3; ++q) F[(long)(3 * a + q) * f + 3 * lj + c] = bj[c * 3 + q];
    }
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

// gather unknowns of the listed points from the global [b][d][point] vector into a
// column-major (3*npts x nrhs) block; sign = +1 copy, scatter variants below
template <typename C>
__global__ void k_gather(C *dst, const C *__restrict__ w, const int *__restrict__ pts, int npts, long n3, int nrhs)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long rows = 3L * npts;
    if (gid >= rows * nrhs) return;
    long r = gid % rows, b = gid / rows;
    int a = (int)(r / 3), c = (int)(r % 3);
    dst[b * rows + r] = w[(b * 3 + c) * n3 + pts[a]];
}

template <typename C>
__global__ void k_scatter(C *w, const C *__restrict__ src, const int *__restrict__ pts, int npts, long n3, int nrhs,
                          int subtract)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long rows = 3L * npts;
    if (gid >= rows * nrhs) return;
    long r = gid % rows, b = gid / rows;
    int a = (int)(r / 3), c = (int)(r % 3);
    long g = (b * 3 + c) * n3 + pts[a];
    C s = src[b * rows + r];
    if (subtract) {
        C v = w[g];
        v.x -= s.x;
        v.y -= s.y;
        w[g] = v;
    } else {
        w[g] = s;
    }
}

template <typename C> __global__ void k_zero(C *a, long cnt)
{
    long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < cnt) { a[gid].x = 0; a[gid].y = 0; }
}

inline unsigned blocks(long cnt, int t = 256) { return (unsigned)((cnt + t - 1) / t); }

} // namespace

// ---------------------------------------------------------------- factor object

struct NDFactor {
    int prec = 0;
    int n = 0;
    std::vector<Node> nodes; // post-order
    DevBuf pts, maps, rels;  // int lists
    DevBuf fac;              // persistent: per node [F11;F21] (f x nown3) then X (nown3 x nbnd3)
    DevBuf piv;
    DevBuf front, stack, work, info; // factor scratch (released after factoring)
    DevBuf solve_ws;
    size_t max_front_unknowns = 0, max_own3 = 0, max_bnd3 = 0;
    cublasHandle_t cublas = nullptr;
    cusolverDnHandle_t cusolver = nullptr;
    ~NDFactor()
    {
        if (cublas) cublasDestroy(cublas);
        if (cusolver) cusolverDnDestroy(cusolver);
        pts.release(); maps.release(); rels.release(); fac.release(); piv.release();
        front.release(); stack.release(); work.release(); info.release(); solve_ws.release();
    }
};

void spm_factor_free(NDFactor *f) { delete f; }

namespace {

constexpr int LEAF_SIDE = 5;

int build_tree(std::vector<Node> &nodes, const int lo[3], const int hi[3])
{
    Node nd;
    for (int d = 0; d < 3; ++d) { nd.lo[d] = lo[d]; nd.hi[d] = hi[d]; }
    int axis = 0;
    for (int d = 1; d < 3; ++d) if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
    int len = hi[axis] - lo[axis];
    if (len > LEAF_SIDE) {
        nd.axis = axis;
        nd.cut = lo[axis] + len / 2;
        int lhi[3] = {hi[0], hi[1], hi[2]}, rlo[3] = {lo[0], lo[1], lo[2]};
        lhi[axis] = nd.cut;
        rlo[axis] = nd.cut + 1;
        nd.left = build_tree(nodes, lo, lhi);
        nd.right = build_tree(nodes, rlo, hi);
    }
    nodes.push_back(nd);
    return (int)nodes.size() - 1;
}

} // namespace

template <typename R>
static spm_status factor_typed(spm_problem_s *P, NDFactor *F)
{
    using BT = blas_t<R>;
    using C = typename BT::C;
    using CV = typename cplx_of<R>::type;
    const int n = P->n;
    const long n3 = (long)n * n * n;
    cudaStream_t s = P->stream;
    F->n = n;
    F->nodes.clear();
    int lo[3] = {0, 0, 0}, hi[3] = {n, n, n};
    build_tree(F->nodes, lo, hi);
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
                for (int x = olo[0]; x < ohi[0]; ++x) pts.push_back((z * n + y) * n + x);
        nd.nown = (int)(pts.size() - nd.own_off);
        nd.bnd_off = pts.size();
        for (int d = 0; d < 3; ++d) { nd.elo[d] = std::max(nd.lo[d] - 1, 0); nd.ehi[d] = std::min(nd.hi[d] + 1, n); }
        for (int z = nd.elo[2]; z < nd.ehi[2]; ++z)
            for (int y = nd.elo[1]; y < nd.ehi[1]; ++y)
                for (int x = nd.elo[0]; x < nd.ehi[0]; ++x) {
                    bool inside = x >= nd.lo[0] && x < nd.hi[0] && y >= nd.lo[1] && y < nd.hi[1] && z >= nd.lo[2] &&
                                  z < nd.hi[2];
                    if (!inside) pts.push_back((z * n + y) * n + x);
                }
        nd.nbnd = (int)(pts.size() - nd.bnd_off);
        // local map over the expanded box: own -> [0,nown), bnd -> nown + rank, else -1
        nd.map_off = maps.size();
        int ew[3] = {nd.ehi[0] - nd.elo[0], nd.ehi[1] - nd.elo[1], nd.ehi[2] - nd.elo[2]};
        size_t base = maps.size();
        maps.resize(base + (size_t)ew[0] * ew[1] * ew[2], -1);
        auto mi = [&](int p) {
            int x = p % n, y = (p / n) % n, z = p / (n * n);
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
                int x = p % n, y = (p / n) % n, z = p / (n * n);
                int l = maps[nd.map_off + ((size_t)(z - nd.elo[2]) * ew[1] + (y - nd.elo[1])) * ew[0] + (x - nd.elo[0])];
                if (l < 0) { spm_set_error("nested dissection: child boundary point outside the parent front"); return SPM_ERR_NUMERICAL; }
                for (int q = 0; q < 3; ++q) rels.push_back(3 * l + q);
            }
        }
    }
    // storage
    long fac_total = 0, piv_total = 0;
    size_t max_f = 0, max_upd_stack = 0, stack_now = 0;
    std::vector<size_t> upd_size(NN, 0);
    for (int id = 0; id < NN; ++id) {
        Node &nd = nodes[id];
        long o3 = 3L * nd.nown, b3 = 3L * nd.nbnd, f = o3 + b3;
        nd.fac_off = fac_total;
        fac_total += f * o3 + o3 * b3;
        nd.piv_off = piv_total;
        piv_total += o3;
        max_f = std::max(max_f, (size_t)f);
        F->max_own3 = std::max(F->max_own3, (size_t)o3);
        F->max_bnd3 = std::max(F->max_bnd3, (size_t)b3);
        // stack: children's updates are popped, this node's update pushed
        for (int ch : {nd.left, nd.right}) if (ch >= 0) stack_now -= upd_size[ch];
        upd_size[id] = (size_t)(b3 * b3);
        stack_now += upd_size[id];
        max_upd_stack = std::max(max_upd_stack, stack_now);
    }
    F->max_front_unknowns = max_f;
    SPM_TRY(F->pts.ensure(sizeof(int) * pts.size()));
    SPM_TRY(F->maps.ensure(sizeof(int) * maps.size()));
    SPM_TRY(F->rels.ensure(sizeof(int) * std::max<size_t>(rels.size(), 1)));
    SPM_CUDA_TRY(cudaMemcpy(F->pts.ptr, pts.data(), sizeof(int) * pts.size(), cudaMemcpyHostToDevice));
    SPM_CUDA_TRY(cudaMemcpy(F->maps.ptr, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice));
    if (!rels.empty())
        SPM_CUDA_TRY(cudaMemcpy(F->rels.ptr, rels.data(), sizeof(int) * rels.size(), cudaMemcpyHostToDevice));
    SPM_TRY(F->fac.ensure(sizeof(C) * fac_total));
    SPM_TRY(F->piv.ensure(sizeof(int) * std::max<long>(piv_total, 1)));
    SPM_TRY(F->front.ensure(sizeof(C) * max_f * max_f));
    SPM_TRY(F->stack.ensure(sizeof(C) * std::max<size_t>(max_upd_stack, 1)));
    SPM_TRY(F->info.ensure(sizeof(int) * 2));
    if (!F->cublas && cublasCreate(&F->cublas) != CUBLAS_STATUS_SUCCESS) { spm_set_error("cublasCreate failed"); return SPM_ERR_CUDA; }
    if (!F->cusolver && cusolverDnCreate(&F->cusolver) != CUSOLVER_STATUS_SUCCESS) { spm_set_error("cusolverDnCreate failed"); return SPM_ERR_CUDA; }
    cublasSetStream(F->cublas, s);
    cusolverDnSetStream(F->cusolver, s);
    int lwork = 0;
    if (BT::getrf_ws(F->cusolver, (int)F->max_own3, F->front.as<C>(), (int)max_f, &lwork) != CUSOLVER_STATUS_SUCCESS) {
        spm_set_error("getrf buffer size query failed");
        return SPM_ERR_CUDA;
    }
    SPM_TRY(F->work.ensure(sizeof(C) * std::max(lwork, 1)));
    SPM_CUDA_TRY(cudaMemsetAsync(F->info.ptr, 0, sizeof(int) * 2, s));

    const C *Sdev = reinterpret_cast<const C *>(sizeof(R) == 8 ? P->S128.ptr : P->S64.ptr);
    const int *dpts = F->pts.as<int>(), *dmaps = F->maps.as<int>(), *drels = F->rels.as<int>();
    C *front = F->front.as<C>(), *stack = F->stack.as<C>(), *fac = F->fac.as<C>();
    int *dpiv = F->piv.as<int>(), *dinfo = F->info.as<int>();
    std::vector<size_t> upd_pos(NN, 0);
    size_t top = 0;
    for (int id = 0; id < NN; ++id) {
        Node &nd = nodes[id];
        const int o3 = 3 * nd.nown, b3 = 3 * nd.nbnd, f = o3 + b3;
        k_zero<C><<<blocks((long)f * f), 256, 0, s>>>(front, (long)f * f);
        int ew0 = nd.ehi[0] - nd.elo[0], ew1 = nd.ehi[1] - nd.elo[1];
        k_front_assemble<C><<<blocks((long)nd.nown * 27), 256, 0, s>>>(front, f, Sdev, dpts + nd.own_off, nd.nown,
                                                                        dmaps + nd.map_off, nd.elo[0], nd.elo[1],
                                                                        nd.elo[2], ew0, ew1, n);
        // extend-add children's updates (the right child's is on top of the stack)
        for (int ch : {nd.left, nd.right}) {
            if (ch < 0) continue;
            Node &c = nodes[ch];
            int bc = 3 * c.nbnd;
            if (bc == 0) continue;
            k_extend_add<C><<<blocks((long)bc * bc), 256, 0, s>>>(front, f, stack + upd_pos[ch], bc, drels + c.rel_off);
        }
        for (int ch : {nd.left, nd.right}) if (ch >= 0) top -= upd_size[ch];
        SPM_CUDA_TRY(cudaGetLastError());
        // partial factorisation
        if (BT::getrf(F->cusolver, o3, front, f, F->work.as<C>(), dpiv + nd.piv_off, dinfo) != CUSOLVER_STATUS_SUCCESS) {
            spm_set_error("getrf failed at node %d", id);
            return SPM_ERR_CUDA;
        }
        if (b3 > 0) {
            if (BT::getrs(F->cusolver, o3, b3, front, f, dpiv + nd.piv_off, front + (long)o3 * f, f, dinfo + 1) !=
                CUSOLVER_STATUS_SUCCESS) {
                spm_set_error("getrs failed at node %d", id);
                return SPM_ERR_CUDA;
            }
            // update = F22 - F21 X, in place in the front
            if (BT::gemm(F->cublas, b3, b3, o3, BT::mone(), front + o3, f, front + (long)o3 * f, f, BT::one(),
                         front + (long)o3 * f + o3, f) != CUBLAS_STATUS_SUCCESS) {
                spm_set_error("gemm failed at node %d", id);
                return SPM_ERR_CUDA;
            }
            // push the update
            upd_pos[id] = top;
            k_copy_block<C><<<blocks((long)b3 * b3), 256, 0, s>>>(stack + top, b3, front + (long)o3 * f + o3, f, b3, b3);
            top += upd_size[id];
        }
        // persistent: [F11; F21] (f x o3, ld f) then X (o3 x b3, ld o3)
        k_copy_block<C><<<blocks((long)f * o3), 256, 0, s>>>(fac + nd.fac_off, f, front, f, f, o3);
        if (b3 > 0)
            k_copy_block<C><<<blocks((long)o3 * b3), 256, 0, s>>>(fac + nd.fac_off + (long)f * o3, o3,
                                                                  front + (long)o3 * f, f, o3, b3);
        SPM_CUDA_TRY(cudaGetLastError());
    }
    int hinfo[2] = {0, 0};
    SPM_CUDA_TRY(cudaMemcpyAsync(hinfo, dinfo, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    F->front.release();
    F->stack.release();
    F->work.release();
    if (hinfo[0] != 0 || hinfo[1] != 0) {
        spm_set_error("zero pivot in the multifrontal factor (info %d, %d)", hinfo[0], hinfo[1]);
        return SPM_ERR_NUMERICAL;
    }
    (void)n3;
    (void)sizeof(CV);
    return SPM_OK;
}

template <typename R>
static spm_status solve_typed(spm_problem_s *P, NDFactor *F, const void *bv, void *xv, int nrhs, cudaStream_t s)
{
    using BT = blas_t<R>;
    using C = typename BT::C;
    const int n = P->n;
    const long n3 = (long)n * n * n;
    C *x = reinterpret_cast<C *>(xv);
    SPM_CUDA_TRY(cudaMemcpyAsync(x, bv, sizeof(C) * 3 * n3 * nrhs, cudaMemcpyDeviceToDevice, s));
    size_t ws = (F->max_own3 + F->max_bnd3) * (size_t)nrhs;
    SPM_TRY(F->solve_ws.ensure(sizeof(C) * ws));
    C *y = F->solve_ws.as<C>();
    C *t = y + F->max_own3 * nrhs;
    cublasSetStream(F->cublas, s);
    cusolverDnSetStream(F->cusolver, s);
    const int *dpts = F->pts.as<int>();
    const C *fac = F->fac.as<C>();
    const int *dpiv = F->piv.as<int>();
    int *dinfo = F->info.ptr ? F->info.as<int>() : nullptr;
    if (!dinfo) { SPM_TRY(F->info.ensure(sizeof(int) * 2)); dinfo = F->info.as<int>(); }
    const int NN = (int)F->nodes.size();
    for (int id = 0; id < NN; ++id) { // forward, post-order
        const Node &nd = F->nodes[id];
        const int o3 = 3 * nd.nown, b3 = 3 * nd.nbnd, f = o3 + b3;
        const C *LU = fac + nd.fac_off;
        k_gather<C><<<blocks((long)o3 * nrhs), 256, 0, s>>>(y, x, dpts + nd.own_off, nd.nown, n3, nrhs);
        if (BT::getrs(F->cusolver, o3, nrhs, LU, f, dpiv + nd.piv_off, y, o3, dinfo) != CUSOLVER_STATUS_SUCCESS) {
            spm_set_error("getrs failed in the forward solve");
            return SPM_ERR_CUDA;
        }
        k_scatter<C><<<blocks((long)o3 * nrhs), 256, 0, s>>>(x, y, dpts + nd.own_off, nd.nown, n3, nrhs, 0);
        if (b3 > 0) {
            BT::gemm(F->cublas, b3, nrhs, o3, BT::one(), LU + o3, f, y, o3, C{0, 0}, t, b3);
            k_scatter<C><<<blocks((long)b3 * nrhs), 256, 0, s>>>(x, t, dpts + nd.bnd_off, nd.nbnd, n3, nrhs, 1);
        }
    }
    for (int id = NN - 1; id >= 0; --id) { // backward, reverse post-order
        const Node &nd = F->nodes[id];
        const int o3 = 3 * nd.nown, b3 = 3 * nd.nbnd, f = o3 + b3;
        if (b3 == 0) continue;
        const C *X = fac + nd.fac_off + (long)f * o3;
        k_gather<C><<<blocks((long)o3 * nrhs), 256, 0, s>>>(y, x, dpts + nd.own_off, nd.nown, n3, nrhs);
        k_gather<C><<<blocks((long)b3 * nrhs), 256, 0, s>>>(t, x, dpts + nd.bnd_off, nd.nbnd, n3, nrhs);
        BT::gemm(F->cublas, o3, nrhs, b3, BT::mone(), X, o3, t, b3, BT::one(), y, o3);
        k_scatter<C><<<blocks((long)o3 * nrhs), 256, 0, s>>>(x, y, dpts + nd.own_off, nd.nown, n3, nrhs, 0);
    }
    SPM_CUDA_TRY(cudaGetLastError());
    return SPM_OK;
}

spm_status spm_factor_impl(spm_problem_s *P, int prec)
{
    NDFactor *&slot = prec == SPM_C128 ? P->fac128 : P->fac64;
    spm_factor_free(slot);
    slot = nullptr;
    NDFactor *F = new NDFactor();
    F->prec = prec;
    spm_status st = prec == SPM_C128 ? factor_typed<double>(P, F) : factor_typed<float>(P, F);
    if (st != SPM_OK) {
        delete F;
        return st;
    }
    slot = F;
    return SPM_OK;
}

spm_status spm_solveS_impl(spm_problem_s *P, int prec, const void *b, void *x, int nrhs, cudaStream_t s)
{
    NDFactor *F = prec == SPM_C128 ? P->fac128 : P->fac64;
    return prec == SPM_C128 ? solve_typed<double>(P, F, b, x, nrhs, s) : solve_typed<float>(P, F, b, x, nrhs, s);
}
