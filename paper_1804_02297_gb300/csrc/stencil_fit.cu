// Device stencil fit (Section 3.1 minimisation, Section 3.2 point classes), FP64.
//
// For a class with neighbourhood tau and enlarged complement tau^c = R \ tau
// (R a box of offsets), alpha = conj(three smallest-eigenvalue eigenvectors of
// H = M M^H), M the off-neighbourhood block.  Entry-wise
//   H[(d,o),(e,o')] = k^4 delta_de C_{00}[o,o'] + C_{de}[o,o'],
//   C_{ab}[o,o'] = sum_{u in tau^c} K_a(o-u) conj(K_b(o'-u)),  K_0 = G, K_d = G^d.
// With v = o - u and lag delta = o' - o,
//   C_{ab}[o,o'] = sum_{v in o-R} F(v) - sum_{t in tau} F(o-t),  F(v) = K_a(v) conj(K_b(v+delta)).
// The boxes o - R for the few o of a class differ only at their ends, so each
// axis of their union is cut into a common core and single edge points; the
// lag sums are accumulated once per (pair, lag, cell) and every box sum is a
// sum of cells.  This costs (pairs x lags x |R|) instead of (entries x |R|).
//
// Only the four canonical classes (interior, face, edge, vertex) are fitted;
// the other 23 follow from reflections x_d -> -x_d (G even, G^d odd in x_d)
// and axis permutations, which map M to a signed row/column permutation of the
// canonical M and so map its singular vectors the same way.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace {

constexpr int MAXT = 27;
constexpr int MAXC = 81;

struct ClassGeom {
    int c[3];          // 0 low boundary, 1 interior, 2 high boundary
    int tlo[3], thi[3]; // neighbourhood offsets per axis
    int rlo[3], rhi[3]; // complement box per axis
    int ulo[3], uhi[3]; // union of the boxes o - R over o in tau
    int clo[3], chi[3]; // common core
    int np[3];          // parts per axis: low edge points, core, high edge points
    int nd[3];          // lag counts per axis
    int T;
};

ClassGeom make_geom(int cls, int n)
{
    ClassGeom g;
    g.c[0] = cls % 3; g.c[1] = (cls / 3) % 3; g.c[2] = cls / 9;
    g.T = 1;
    for (int d = 0; d < 3; ++d) {
        int c = g.c[d];
        g.tlo[d] = c == 0 ? 0 : -1;
        g.thi[d] = c == 2 ? 0 : 1;
        g.rlo[d] = c == 0 ? 0 : (c == 1 ? -(n - 2) : -(n - 1));
        g.rhi[d] = c == 0 ? n - 1 : (c == 1 ? n - 2 : 0);
        g.ulo[d] = g.tlo[d] - g.rhi[d];
        g.uhi[d] = g.thi[d] - g.rlo[d];
        g.clo[d] = g.thi[d] - g.rhi[d];
        g.chi[d] = g.tlo[d] - g.rlo[d];
        int w = g.thi[d] - g.tlo[d]; // edge points per side
        g.np[d] = 2 * w + 1;
        g.nd[d] = 2 * w + 1;
        g.T *= w + 1;
    }
    return g;
}

// part of an axis coordinate: 0..w-1 low edge points, w core, w+1..2w high edge points
__host__ __device__ __forceinline__ int part_of(int v, int ulo, int clo, int chi, int w)
{
    if (v < clo) return v - ulo;
    if (v > chi) return w + 1 + (v - chi - 1);
    return w;
}

__device__ __forceinline__ double2 entry_at(const double2 *__restrict__ E, int q, int n, int t1, int t2, int t3)
{
    const int lim = n - 1;
    if (t1 < -lim || t1 > lim || t2 < -lim || t2 > lim || t3 < -lim || t3 > lim) return make_double2(0, 0);
    const long W = 2 * n - 1;
    return E[(long)q * W * W * W + ((long)(t3 + lim) * W + (t2 + lim)) * W + (t1 + lim)];
}

__constant__ int c_pair_a[7] = {0, 1, 2, 3, 1, 1, 2};
__constant__ int c_pair_b[7] = {0, 1, 2, 3, 2, 3, 3};

// One block per (v3, lag, pair).  Threads sweep the (v2, v1) plane of the union box.
__global__ void __launch_bounds__(256) k_lag_cells(const double2 *__restrict__ E, double2 *__restrict__ cells, ClassGeom g,
                                                   int n)
{
    __shared__ double2 edge_acc[25];
    __shared__ double2 red[8];
    const int v3 = g.ulo[2] + blockIdx.x;
    const int lag = blockIdx.y;
    const int pair = blockIdx.z;
    const int nd1 = g.nd[0], nd2 = g.nd[1];
    const int w1 = (g.np[0] - 1) / 2, w2 = (g.np[1] - 1) / 2, w3 = (g.np[2] - 1) / 2;
    const int d1 = lag % nd1 - w1, d2 = (lag / nd1) % nd2 - w2, d3 = lag / (nd1 * nd2) - w3;
    const int qa = c_pair_a[pair], qb = c_pair_b[pair];
    const int p3 = part_of(v3, g.ulo[2], g.clo[2], g.chi[2], w3);
    for (int i = threadIdx.x; i < 25; i += blockDim.x) edge_acc[i] = make_double2(0, 0);
    __syncthreads();
    const int U1 = g.uhi[0] - g.ulo[0] + 1, U2 = g.uhi[1] - g.ulo[1] + 1;
    double2 acc = make_double2(0, 0);
    for (int idx = threadIdx.x; idx < U1 * U2; idx += blockDim.x) {
        int v2 = g.ulo[1] + idx / U1, v1 = g.ulo[0] + idx % U1;
        double2 a = entry_at(E, qa, n, v1, v2, v3);
        double2 b = entry_at(E, qb, n, v1 + d1, v2 + d2, v3 + d3);
        double2 f = cmulc(a, b);
        int p1 = part_of(v1, g.ulo[0], g.clo[0], g.chi[0], w1);
        int p2 = part_of(v2, g.ulo[1], g.clo[1], g.chi[1], w2);
        if (p1 == w1 && p2 == w2) {
            acc.x += f.x;
            acc.y += f.y;
        } else {
            int slot = p2 * g.np[0] + p1;
            atomicAdd(&edge_acc[slot].x, f.x);
            atomicAdd(&edge_acc[slot].y, f.y);
        }
    }
    // block reduction of the core accumulator
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    const int ncell = g.np[0] * g.np[1] * g.np[2];
    double2 *out = cells + ((long)pair * (nd1 * nd2 * g.nd[2]) + lag) * ncell;
    if (threadIdx.x == 0) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s.x += red[w].x; s.y += red[w].y; }
        int slot = (p3 * g.np[1] + w2) * g.np[0] + w1;
        atomicAdd(&out[slot].x, s.x);
        atomicAdd(&out[slot].y, s.y);
    }
    for (int i = threadIdx.x; i < g.np[0] * g.np[1]; i += blockDim.x) {
        int p2 = i / g.np[0], p1 = i % g.np[0];
        if (p1 == w1 && p2 == w2) continue;
        int slot = (p3 * g.np[1] + p2) * g.np[0] + p1;
        atomicAdd(&out[slot].x, edge_acc[i].x);
        atomicAdd(&out[slot].y, edge_acc[i].y);
    }
}

// C_{ab}[o, o'] for a <= b from the cell sums (box part) minus the tau part.
__device__ double2 corr_entry(const double2 *__restrict__ E, const double2 *__restrict__ cells, const ClassGeom &g,
                              int n, int pair, int qa, int qb, const int o[3], const int op[3])
{
    int w[3], lagi[3];
    for (int d = 0; d < 3; ++d) {
        w[d] = (g.np[d] - 1) / 2;
        lagi[d] = op[d] - o[d] + w[d];
    }
    const int nlag = g.nd[0] * g.nd[1] * g.nd[2];
    const int lag = (lagi[2] * g.nd[1] + lagi[1]) * g.nd[0] + lagi[0];
    const int ncell = g.np[0] * g.np[1] * g.np[2];
    const double2 *cs = cells + ((long)pair * nlag + lag) * ncell;
    // parts of each axis inside the box [o - rhi, o - rlo]
    bool in[3][5];
    for (int d = 0; d < 3; ++d) {
        int lo = o[d] - g.rhi[d], hi = o[d] - g.rlo[d];
        for (int p = 0; p < g.np[d]; ++p) {
            if (p == w[d]) { in[d][p] = true; continue; }
            int v = p < w[d] ? g.ulo[d] + p : g.chi[d] + 1 + (p - w[d] - 1);
            in[d][p] = v >= lo && v <= hi;
        }
    }
    double2 s = make_double2(0, 0);
    for (int p3 = 0; p3 < g.np[2]; ++p3) {
        if (!in[2][p3]) continue;
        for (int p2 = 0; p2 < g.np[1]; ++p2) {
            if (!in[1][p2]) continue;
            for (int p1 = 0; p1 < g.np[0]; ++p1) {
                if (!in[0][p1]) continue;
                double2 c = cs[(p3 * g.np[1] + p2) * g.np[0] + p1];
                s.x += c.x;
                s.y += c.y;
            }
        }
    }
    // minus the neighbourhood itself: sum_{t in tau} K_a(o - t) conj(K_b(o' - t))
    for (int t3 = g.tlo[2]; t3 <= g.thi[2]; ++t3)
        for (int t2 = g.tlo[1]; t2 <= g.thi[1]; ++t2)
            for (int t1 = g.tlo[0]; t1 <= g.thi[0]; ++t1) {
                double2 a = entry_at(E, qa, n, o[0] - t1, o[1] - t2, o[2] - t3);
                double2 b = entry_at(E, qb, n, op[0] - t1, op[1] - t2, op[2] - t3);
                double2 f = cmulc(a, b);
                s.x -= f.x;
                s.y -= f.y;
            }
    return s;
}

__device__ void tau_offset(const ClassGeom &g, int idx, int o[3])
{
    int w1 = g.thi[0] - g.tlo[0] + 1, w2 = g.thi[1] - g.tlo[1] + 1;
    o[0] = g.tlo[0] + idx % w1;
    o[1] = g.tlo[1] + (idx / w1) % w2;
    o[2] = g.tlo[2] + idx / (w1 * w2);
}

__device__ __forceinline__ int pair_index(int a, int b) // a <= b
{
    if (a == b) return a;
    if (a == 1 && b == 2) return 4;
    if (a == 1 && b == 3) return 5;
    return 6;
}

// Builds H for one class, then cyclic two-sided Jacobi with a parallel
// (round-robin) ordering.  Outputs eigenvalues ascending and alpha = conj of the
// three eigenvectors with the smallest eigenvalues.  One block per class.
__global__ void __launch_bounds__(256) k_gram_eig(const double2 *__restrict__ E, const double2 *__restrict__ cells, ClassGeom g,
                                                  int n, double k4, double2 *alpha_out, double *sv_out, int *status)
{
    extern __shared__ unsigned char smem_raw[];
    const int T = g.T, C = 3 * T;
    double2 *H = reinterpret_cast<double2 *>(smem_raw); // C x C, row-major
    double2 *V = H + C * C;
    __shared__ double rc[MAXC / 2 + 1], rs[MAXC / 2 + 1];
    __shared__ double2 rph[MAXC / 2 + 1];
    __shared__ int rp[MAXC / 2 + 1], rq[MAXC / 2 + 1];
    __shared__ unsigned long long off_bits;

    for (int idx = threadIdx.x; idx < C * C; idx += blockDim.x) {
        int r = idx / C, c = idx % C;
        int d = r / T, e = c / T;
        int o[3], op[3];
        tau_offset(g, r % T, o);
        tau_offset(g, c % T, op);
        double2 h = make_double2(0, 0);
        if (d == e) {
            double2 c0 = corr_entry(E, cells, g, n, 0, 0, 0, o, op);
            h.x = k4 * c0.x;
            h.y = k4 * c0.y;
        }
        double2 cde;
        if (d <= e) cde = corr_entry(E, cells, g, n, pair_index(d + 1, e + 1), d + 1, e + 1, o, op);
        else cde = conj_of(corr_entry(E, cells, g, n, pair_index(e + 1, d + 1), e + 1, d + 1, op, o));
        h.x += cde.x;
        h.y += cde.y;
        H[idx] = h;
        V[idx] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    // enforce exact Hermitian symmetry (the two halves were summed separately)
    for (int idx = threadIdx.x; idx < C * C; idx += blockDim.x) {
        int r = idx / C, c = idx % C;
        if (r < c) {
            double2 a = H[idx], b = H[c * C + r];
            double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            H[idx] = m;
            H[c * C + r] = conj_of(m);
        } else if (r == c) {
            H[idx].y = 0.0;
        }
    }
    __syncthreads();

    // largest diagonal entry: rounding level of the whole matrix
    __shared__ double dmax;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < C; ++i) m = fmax(m, fabs(H[i * C + i].x));
        dmax = m;
    }
    __syncthreads();
    const double floor_abs = 4e-17 * dmax;
    const int NP = (C + 1) & ~1; // players, one dummy if C is odd
    const int npairs = NP / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) off_bits = 0ull;
        __syncthreads();
        for (int round = 0; round < NP - 1; ++round) {
            // rotation parameters for the disjoint pairs of this round
            for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
                int pa = k, pb = NP - 1 - k;
                int p = pa == 0 ? 0 : ((pa - 1 + round) % (NP - 1)) + 1;
                int q = pb == 0 ? 0 : ((pb - 1 + round) % (NP - 1)) + 1;
                if (p > q) { int t = p; p = q; q = t; }
                rp[k] = p;
                rq[k] = q;
                rc[k] = 1.0;
                rs[k] = 0.0;
                rph[k] = make_double2(1.0, 0.0);
                if (q >= C) continue;
                double a = H[p * C + p].x, c = H[q * C + q].x;
                double2 b = H[p * C + q];
                double ab = hypot(b.x, b.y);
                double scale = sqrt(fabs(a * c));
                if (ab == 0.0 || ab <= 1e-16 * scale || ab <= floor_abs) continue;
                double rel = ab / fmax(scale, floor_abs);
                atomicMax(&off_bits, (unsigned long long)__double_as_longlong(rel)); // positive doubles order as integers
                double zeta = (c - a) / (2.0 * ab);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t);
                rc[k] = cs;
                rs[k] = t * cs;
                rph[k] = make_double2(b.x / ab, -b.y / ab); // e^{-i phi}
            }
            __syncthreads();
            // rows: H <- J^H H
            for (int idx = threadIdx.x; idx < npairs * C; idx += blockDim.x) {
                int k = idx / C, col = idx % C;
                int p = rp[k], q = rq[k];
                if (q >= C || rs[k] == 0.0) continue;
                double cs = rc[k], sn = rs[k];
                double2 ep = conj_of(rph[k]); // e^{+i phi}
                double2 hp = H[p * C + col], hq = cmul(ep, H[q * C + col]);
                H[p * C + col] = make_double2(cs * hp.x - sn * hq.x, cs * hp.y - sn * hq.y);
                H[q * C + col] = make_double2(sn * hp.x + cs * hq.x, sn * hp.y + cs * hq.y);
            }
            __syncthreads();
            // columns: H <- H J, V <- V J; the rotated pair is zeroed exactly
            for (int idx = threadIdx.x; idx < npairs * C; idx += blockDim.x) {
                int k = idx / C, row = idx % C;
                int p = rp[k], q = rq[k];
                if (q >= C || rs[k] == 0.0) continue;
                double cs = rc[k], sn = rs[k];
                double2 em = rph[k]; // e^{-i phi}
                double2 hp = H[row * C + p], hq = cmul(em, H[row * C + q]);
                double2 np_ = make_double2(cs * hp.x - sn * hq.x, cs * hp.y - sn * hq.y);
                double2 nq_ = make_double2(sn * hp.x + cs * hq.x, sn * hp.y + cs * hq.y);
                if (row == p) nq_ = make_double2(0.0, 0.0);
                if (row == q) np_ = make_double2(0.0, 0.0);
                if (row == p || row == q) { (row == p ? np_ : nq_).y = 0.0; }
                H[row * C + p] = np_;
                H[row * C + q] = nq_;
                double2 vp = V[row * C + p], vq = cmul(em, V[row * C + q]);
                V[row * C + p] = make_double2(cs * vp.x - sn * vq.x, cs * vp.y - sn * vq.y);
                V[row * C + q] = make_double2(sn * vp.x + cs * vq.x, sn * vp.y + cs * vq.y);
            }
            __syncthreads();
        }
        __syncthreads();
        if (__longlong_as_double((long long)off_bits) < 1e-14) break;
        __syncthreads();
    }
    // sort eigenvalues ascending (selection on one thread; C <= 81)
    if (threadIdx.x == 0) {
        int idx[MAXC];
        for (int i = 0; i < C; ++i) idx[i] = i;
        for (int i = 1; i < C; ++i) {
            int v = idx[i], j = i - 1;
            while (j >= 0 && H[idx[j] * C + idx[j]].x > H[v * C + v].x) { idx[j + 1] = idx[j]; --j; }
            idx[j + 1] = v;
        }
        for (int i = 0; i < C; ++i) {
            double lam = H[idx[i] * C + idx[i]].x;
            sv_out[i] = sqrt(lam > 0 ? lam : 0.0);
        }
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < C; ++r) alpha_out[r * 3 + c] = conj_of(V[r * C + idx[c]]);
        if (__longlong_as_double((long long)off_bits) >= 1e-10) atomicExch(status, 1);
    }
}

// Maps the canonical alpha of each class family to all 27 classes and forms
// beta = B^T alpha (Eq. alphabeta).  One block per target class.
__global__ void k_map_beta(const double2 *__restrict__ E, const double2 *__restrict__ canon_alpha,
                           const double *__restrict__ canon_sv, const int *__restrict__ rowmap, int n, double k2,
                           double2 *alpha_all, double2 *beta_all, double *sv_all)
{
    const int cls = blockIdx.x;
    int c[3] = {cls % 3, (cls / 3) % 3, cls / 9};
    int nb = (c[0] != 1) + (c[1] != 1) + (c[2] != 1);
    int tlo[3], thi[3];
    for (int d = 0; d < 3; ++d) { tlo[d] = c[d] == 0 ? 0 : -1; thi[d] = c[d] == 2 ? 0 : 1; }
    int w1 = thi[0] - tlo[0] + 1, w2 = thi[1] - tlo[1] + 1, w3 = thi[2] - tlo[2] + 1;
    int T = w1 * w2 * w3, C = 3 * T;
    const double2 *ca = canon_alpha + nb * MAXC * 3;
    double2 *al = alpha_all + (long)cls * MAXC * 3;
    double2 *be = beta_all + (long)cls * 4 * MAXT * 3;
    for (int i = threadIdx.x; i < MAXC * 3; i += blockDim.x) al[i] = make_double2(0, 0);
    for (int i = threadIdx.x; i < 4 * MAXT * 3; i += blockDim.x) be[i] = make_double2(0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        int m = rowmap[cls * MAXC + i]; // canonical row with sign: +-(r+1)
        int r = (m > 0 ? m : -m) - 1;
        double s = m > 0 ? 1.0 : -1.0;
        for (int col = 0; col < 3; ++col) {
            double2 v = ca[r * 3 + col];
            al[i * 3 + col] = make_double2(s * v.x, s * v.y);
        }
    }
    for (int i = threadIdx.x; i < MAXC; i += blockDim.x) sv_all[cls * MAXC + i] = i < C ? canon_sv[nb * MAXC + i] : 0.0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 4 * T * 3; idx += blockDim.x) {
        int col = idx % 3, row = idx / 3;
        int f = row / T, opi = row % T;
        int op[3] = {tlo[0] + opi % w1, tlo[1] + (opi / w1) % w2, tlo[2] + opi / (w1 * w2)};
        double2 s = make_double2(0, 0);
        for (int oi = 0; oi < T; ++oi) {
            int o[3] = {tlo[0] + oi % w1, tlo[1] + (oi / w1) % w2, tlo[2] + oi / (w1 * w2)};
            int t1 = o[0] - op[0], t2 = o[1] - op[1], t3 = o[2] - op[2];
            if (f < 3) {
                double2 gv = entry_at(E, 0, n, t1, t2, t3);
                double2 a = al[(f * T + oi) * 3 + col];
                double2 pr = cmul(gv, a);
                s.x += k2 * pr.x;
                s.y += k2 * pr.y;
            } else {
                for (int d = 0; d < 3; ++d) s = cfma(entry_at(E, 1 + d, n, t1, t2, t3), al[(d * T + oi) * 3 + col], s);
            }
        }
        be[row * 3 + col] = s;
    }
}

// Row map from a canonical class (boundary axes first, all at the low side) to
// class `cls`: canonical axis j goes to axis perm[j]; axes with c = 2 are reflected.
void build_rowmap(int cls, int *out)
{
    int c[3] = {cls % 3, (cls / 3) % 3, cls / 9};
    int perm[3], j = 0;
    for (int d = 0; d < 3; ++d) if (c[d] != 1) perm[j++] = d;
    int nb = j;
    for (int d = 0; d < 3; ++d) if (c[d] == 1) perm[j++] = d;
    int cc[3];
    for (int q = 0; q < 3; ++q) cc[q] = q < nb ? 0 : 1;
    int canon = cc[0] + 3 * cc[1] + 9 * cc[2];
    ClassGeom gc = make_geom(canon, 8), gt = make_geom(cls, 8);
    int cw[3], tw[3];
    for (int d = 0; d < 3; ++d) { cw[d] = gc.thi[d] - gc.tlo[d] + 1; tw[d] = gt.thi[d] - gt.tlo[d] + 1; }
    int Tc = gc.T;
    for (int e = 0; e < 3; ++e)
        for (int oi = 0; oi < Tc; ++oi) {
            int o[3] = {gc.tlo[0] + oi % cw[0], gc.tlo[1] + (oi / cw[0]) % cw[1], gc.tlo[2] + oi / (cw[0] * cw[1])};
            int ot[3];
            for (int q = 0; q < 3; ++q) ot[perm[q]] = o[q];
            for (int d = 0; d < 3; ++d) if (c[d] == 2) ot[d] = -ot[d];
            int et = perm[e];
            int ti = ((ot[2] - gt.tlo[2]) * tw[1] + (ot[1] - gt.tlo[1])) * tw[0] + (ot[0] - gt.tlo[0]);
            int sign = c[et] == 2 ? -1 : 1;
            out[cls * MAXC + et * Tc + ti] = sign * (e * Tc + oi + 1);
        }
}

} // namespace

spm_status spm_entries_device(spm_problem_s *P, DevBuf &E); // apply.cu

spm_status spm_stencils_device(spm_problem_s *P)
{
    const int n = P->n;
    cudaStream_t s = P->stream;
    DevBuf E, cells, calpha, csv, rowmap, stat, alpha_all, beta_all, sv_all;
    SPM_TRY(spm_entries_device(P, E));
    const int canon[4] = {13, 12, 9, 0}; // 0..3 boundary axes
    SPM_TRY(calpha.ensure(sizeof(double2) * 4 * MAXC * 3));
    SPM_TRY(csv.ensure(sizeof(double) * 4 * MAXC));
    SPM_TRY(stat.ensure(sizeof(int)));
    SPM_CUDA_TRY(cudaMemsetAsync(stat.ptr, 0, sizeof(int), s));
    static bool attr = false;
    if (!attr) {
        SPM_CUDA_TRY(cudaFuncSetAttribute(k_gram_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * MAXC * MAXC * 16));
        attr = true;
    }
    for (int f = 0; f < 4; ++f) {
        ClassGeom g = make_geom(canon[f], n);
        int nlag = g.nd[0] * g.nd[1] * g.nd[2];
        int ncell = g.np[0] * g.np[1] * g.np[2];
        size_t bytes = sizeof(double2) * 7 * nlag * ncell;
        SPM_TRY(cells.ensure(bytes));
        SPM_CUDA_TRY(cudaMemsetAsync(cells.ptr, 0, bytes, s));
        dim3 grid(g.uhi[2] - g.ulo[2] + 1, nlag, 7);
        k_lag_cells<<<grid, 256, 0, s>>>(E.as<double2>(), cells.as<double2>(), g, n);
        SPM_CUDA_TRY(cudaGetLastError());
        int C = 3 * g.T;
        k_gram_eig<<<1, 256, 2 * C * C * sizeof(double2), s>>>(E.as<double2>(), cells.as<double2>(), g, n,
                                                              P->k * P->k * P->k * P->k,
                                                              calpha.as<double2>() + f * MAXC * 3,
                                                              csv.as<double>() + f * MAXC, stat.as<int>());
        SPM_CUDA_TRY(cudaGetLastError());
    }
    std::vector<int> rm(27 * MAXC, 0);
    for (int cls = 0; cls < 27; ++cls) build_rowmap(cls, rm.data());
    SPM_TRY(rowmap.ensure(sizeof(int) * rm.size()));
    SPM_CUDA_TRY(cudaMemcpyAsync(rowmap.ptr, rm.data(), sizeof(int) * rm.size(), cudaMemcpyHostToDevice, s));
    SPM_TRY(alpha_all.ensure(sizeof(double2) * 27 * MAXC * 3));
    SPM_TRY(beta_all.ensure(sizeof(double2) * 27 * 4 * MAXT * 3));
    SPM_TRY(sv_all.ensure(sizeof(double) * 27 * MAXC));
    k_map_beta<<<27, 128, 0, s>>>(E.as<double2>(), calpha.as<double2>(), csv.as<double>(), rowmap.as<int>(), n,
                                  P->k * P->k, alpha_all.as<double2>(), beta_all.as<double2>(), sv_all.as<double>());
    SPM_CUDA_TRY(cudaGetLastError());
    int status = 0;
    P->alpha_h.resize(2 * 27 * MAXC * 3);
    P->beta_h.resize(2 * 27 * 4 * MAXT * 3);
    P->sv_h.resize(27 * MAXC);
    SPM_CUDA_TRY(cudaMemcpyAsync(P->alpha_h.data(), alpha_all.ptr, alpha_all.bytes, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->beta_h.data(), beta_all.ptr, beta_all.bytes, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(P->sv_h.data(), sv_all.ptr, sv_all.bytes, cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaMemcpyAsync(&status, stat.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (status != 0) {
        spm_set_error("Jacobi eigensolver did not converge");
        return SPM_ERR_NUMERICAL;
    }
    // device copies used by Q and the assembly
    std::vector<float> a32(P->alpha_h.size());
    for (size_t i = 0; i < a32.size(); ++i) a32[i] = (float)P->alpha_h[i];
    SPM_TRY(P->alpha128.ensure(alpha_all.bytes));
    SPM_TRY(P->alpha64.ensure(sizeof(float) * a32.size()));
    SPM_TRY(P->beta128.ensure(beta_all.bytes));
    SPM_CUDA_TRY(cudaMemcpy(P->alpha128.ptr, alpha_all.ptr, alpha_all.bytes, cudaMemcpyDeviceToDevice));
    SPM_CUDA_TRY(cudaMemcpy(P->alpha64.ptr, a32.data(), sizeof(float) * a32.size(), cudaMemcpyHostToDevice));
    SPM_CUDA_TRY(cudaMemcpy(P->beta128.ptr, beta_all.ptr, beta_all.bytes, cudaMemcpyDeviceToDevice));
    P->have_stencils = true;
    return spm_build_qtable(P);
}
