// Three-dimensional operator build of the VIP method (the paper's introduction
// and Sec. 3: the method in three coordinates with the ten-term quadratic basis).
//
// Neighbour search (Sec. 3: nodes strictly inside |x_i - xbar| < rho), the MLS
// derivative weights of every node, VIP and normal point (Eq. fmlsrk:2 with the
// basis [1, xi, eta, zeta, xi^2, xi eta, xi zeta, eta^2, eta zeta, zeta^2]) and
// the operator tables of Eq. vip:1 and Sec. 4.1 (L, the six VIP interpolations,
// the VIP differences Gx, Gy, Gz, and the zero-normal-derivative rows of the
// boundary nodes).  Independent of the 2D context: its own handle (vip_3d),
// buffers and kernels.
//
// Layout: node coordinates, normals and spacing as FP64 structure-of-arrays.
// Points are enumerated as [nodes | 6 VIPs per interior node (E, W, N, S, T, B
// blocks of Ni each) | 2 normal points per boundary node (blocks of Nb)]; each
// point's neighbour list is a CSR row (int64 offsets, int32 node indices sorted
// ascending).  Node points carry 7 weight arrays (the derivative tables), the
// other points one (interpolation).  Tables are assembled as CSR on first use.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/vip.h"

struct vip_3d;

namespace {

constexpr int K3MAX = 160;                 // largest neighbour list per point
constexpr int NB3 = 10;                    // basis size
constexpr int NM3 = NB3 * (NB3 + 1) / 2;   // packed lower triangle of M
constexpr int NDER3 = 7;                   // node derivative tables
// Basis index of each node derivative table: (0,0,0) (1,0,0) (0,1,0) (0,0,1)
// (2,0,0) (0,2,0) (0,0,2) in the order of the basis above.
__constant__ int c_dbasis[NDER3] = {0, 1, 2, 3, 4, 7, 9};

struct Csr {
    int64_t* ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    int64_t nnz = 0;
};

// Device view of the node set, the cell grid and the point enumeration.
struct Pts {
    const double *x, *y, *z, *nx, *ny, *nz, *h;
    const int32_t* interior;   // [Ni] node index of the k-th interior node
    const int32_t* boundary;   // [Nb] node index of the k-th boundary node
    int64_t N, Ni, Nb;
    double L[3];
    double support;
    int weight;
    double lo[3], cs[3];
    int nc[3];
    const int64_t* cell_ptr;   // [ncells + 1]
    const int32_t* cell_nodes; // [N] nodes sorted by cell
};

__device__ __forceinline__ double min_img(double d, double L) {
    if (L <= 0.0) return d;
    double hl = 0.5 * L;
    if (d > hl) d = __dsub_rn(d, L);
    if (d < -hl) d = __dadd_rn(d, L);
    return d;
}

// Coordinates, dilation and owning node of point p (see the layout above).  The
// arithmetic is rounded step by step (no contraction), as the reference
// statement of the points is.
__device__ __forceinline__ void point_of(const Pts& a, int64_t p, double q[3], double& rho,
                                         int64_t& owner) {
    if (p < a.N) {
        owner = p;
        q[0] = a.x[p]; q[1] = a.y[p]; q[2] = a.z[p];
        rho = __dmul_rn(a.support, a.h[p]);
        return;
    }
    int64_t t = p - a.N;
    if (t < 6 * a.Ni) {
        int k = (int)(t / a.Ni);
        int64_t r = a.interior[t - (int64_t)k * a.Ni];
        owner = r;
        q[0] = a.x[r]; q[1] = a.y[r]; q[2] = a.z[r];
        double hh = __dmul_rn(0.5, a.h[r]);
        int ax = k >> 1;
        q[ax] = (k & 1) ? __dsub_rn(q[ax], hh) : __dadd_rn(q[ax], hh);
        rho = __dmul_rn(a.support, a.h[r]);
        return;
    }
    t -= 6 * a.Ni;
    int s = (int)(t / a.Nb);                   // 0: first normal point, 1: second
    int64_t r = a.boundary[t - (int64_t)s * a.Nb];
    owner = r;
    double sh = __dmul_rn((double)(s + 1), a.h[r]);
    q[0] = __dsub_rn(a.x[r], __dmul_rn(sh, a.nx[r]));
    q[1] = __dsub_rn(a.y[r], __dmul_rn(sh, a.ny[r]));
    q[2] = __dsub_rn(a.z[r], __dmul_rn(sh, a.nz[r]));
    rho = __dmul_rn(a.support, a.h[r]);
}

__device__ __forceinline__ int cell_coord(const Pts& a, double v, int ax) {
    double w;
    if (a.L[ax] > 0.0) w = v - floor(v / a.L[ax]) * a.L[ax];
    else w = v - a.lo[ax];
    int c = (int)floor(w / a.cs[ax]);
    return c < 0 ? 0 : (c >= a.nc[ax] ? a.nc[ax] - 1 : c);
}

// Calls f(node, dx, dy, dz) for every node j with |x_j - q|^2 < rho^2 (minimum
// image in periodic sets), in cell order.
template <class F>
__device__ __forceinline__ void for_each_nbr(const Pts& a, const double q[3], double rho, F f) {
    int c[3], lo[3], hi[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        c[ax] = cell_coord(a, q[ax], ax);
        if (a.L[ax] > 0.0 && a.nc[ax] >= 3) { lo[ax] = c[ax] - 1; hi[ax] = c[ax] + 1; }
        else if (a.L[ax] > 0.0) { lo[ax] = 0; hi[ax] = a.nc[ax] - 1; }   // every cell once
        else { lo[ax] = max(c[ax] - 1, 0); hi[ax] = min(c[ax] + 1, a.nc[ax] - 1); }
    }
    const double r2 = __dmul_rn(rho, rho);
    for (int i = lo[0]; i <= hi[0]; ++i) {
        int ci = (i + a.nc[0]) % a.nc[0];
        for (int j = lo[1]; j <= hi[1]; ++j) {
            int cj = (j + a.nc[1]) % a.nc[1];
            for (int k = lo[2]; k <= hi[2]; ++k) {
                int ck = (k + a.nc[2]) % a.nc[2];
                int64_t cell = ((int64_t)ci * a.nc[1] + cj) * a.nc[2] + ck;
                for (int64_t m = a.cell_ptr[cell]; m < a.cell_ptr[cell + 1]; ++m) {
                    int nd = a.cell_nodes[m];
                    double dx = min_img(__dsub_rn(a.x[nd], q[0]), a.L[0]);
                    double dy = min_img(__dsub_rn(a.y[nd], q[1]), a.L[1]);
                    double dz = min_img(__dsub_rn(a.z[nd], q[2]), a.L[2]);
                    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                          __dmul_rn(dz, dz));
                    if (d2 < r2) f(nd, dx, dy, dz);
                }
            }
        }
    }
}

__device__ __forceinline__ void flag(int* status, long long* bad, int code, int64_t p) {
    atomicCAS(status, 0, code);
    atomicMin(bad, (long long)p);
}

__global__ void k3_cell_count(Pts a, int64_t* __restrict__ node_cell, int32_t* __restrict__ cnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.N) return;
    int cx = cell_coord(a, a.x[r], 0), cy = cell_coord(a, a.y[r], 1), cz = cell_coord(a, a.z[r], 2);
    int64_t cell = ((int64_t)cx * a.nc[1] + cy) * a.nc[2] + cz;
    node_cell[r] = cell;
    atomicAdd(&cnt[cell], 1);
}

__global__ void k3_cell_fill(int64_t N, const int64_t* __restrict__ node_cell,
                             const int64_t* __restrict__ cell_ptr, int32_t* __restrict__ cursor,
                             int32_t* __restrict__ cell_nodes) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    int64_t c = node_cell[r];
    int pos = atomicAdd(&cursor[c], 1);
    cell_nodes[cell_ptr[c] + pos] = (int32_t)r;
}

__global__ void k3_nbr_count(Pts a, int64_t P, int32_t* __restrict__ cnt, int* status, long long* bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double q[3], rho;
    int64_t owner;
    point_of(a, p, q, rho, owner);
    int n = 0;
    for_each_nbr(a, q, rho, [&](int, double, double, double) { ++n; });
    if (n > K3MAX) {
        flag(status, bad, VIP_ERR_ARG, p);
        n = 0;
    }
    cnt[p] = n;
}

__global__ void k3_nbr_fill(Pts a, int64_t P, const int64_t* __restrict__ pptr,
                            int32_t* __restrict__ pidx) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int64_t b = pptr[p], e = pptr[p + 1];
    if (e == b) return;
    double q[3], rho;
    int64_t owner;
    point_of(a, p, q, rho, owner);
    int64_t w = b;
    for_each_nbr(a, q, rho, [&](int nd, double, double, double) {
        if (w < e) pidx[w++] = nd;
    });
    for (int64_t i = b + 1; i < e; ++i) {     // ascending node order (lists are short)
        int32_t v = pidx[i];
        int64_t k = i - 1;
        while (k >= b && pidx[k] > v) { pidx[k + 1] = pidx[k]; --k; }
        pidx[k + 1] = v;
    }
}

__device__ __forceinline__ double weight3(double r, int kind) {
    if (kind == VIP_W_PAPER) {
        if (r >= 1.0) return 0.0;
        double t = 1.0 - pow(r, (1.0 - r) * (1.0 - r));
        return (t * t) * (t * t);
    }
    if (r <= 0.5) return 2.0 / 3.0 - 4.0 * r * r + 4.0 * r * r * r;
    if (r < 1.0) return 4.0 / 3.0 - 4.0 * r + 4.0 * r * r - (4.0 / 3.0) * r * r * r;
    return 0.0;
}

__device__ __forceinline__ constexpr int tri3(int i, int j) { return i * (i + 1) / 2 + j; }

// Scaled offset, weight and basis vector of neighbour node nd of point q.
__device__ __forceinline__ double basis_at(const Pts& a, int nd, const double q[3], double rho,
                                           double pv[NB3]) {
    double xi = min_img(a.x[nd] - q[0], a.L[0]) / rho;
    double eta = min_img(a.y[nd] - q[1], a.L[1]) / rho;
    double zeta = min_img(a.z[nd] - q[2], a.L[2]) / rho;
    pv[0] = 1.0; pv[1] = xi; pv[2] = eta; pv[3] = zeta;
    pv[4] = xi * xi; pv[5] = xi * eta; pv[6] = xi * zeta;
    pv[7] = eta * eta; pv[8] = eta * zeta; pv[9] = zeta * zeta;
    return weight3(sqrt(xi * xi + eta * eta + zeta * zeta), a.weight);
}

// MLS weights of every point: M = sum_j Phi_j p_j p_j^T (ten-term basis), its
// Cholesky factor, and for each derivative k wanted the vector z_k = M^{-1} e_k;
// then Psi_k(j) = fac_k Phi_j (z_k . p_j), fac_k = a! b! c! rho^-(a+b+c).
__global__ void __launch_bounds__(128) k3_mls(Pts a, int64_t P, const int64_t* __restrict__ pptr,
                                              const int32_t* __restrict__ pidx,
                                              double* __restrict__ wnode, int64_t nnz_nodes,
                                              double* __restrict__ w0, int* status, long long* bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int64_t b = pptr[p], e = pptr[p + 1];
    double q[3], rho;
    int64_t owner;
    point_of(a, p, q, rho, owner);
    double M[NM3];
#pragma unroll
    for (int i = 0; i < NM3; ++i) M[i] = 0.0;
    for (int64_t s = b; s < e; ++s) {
        double pv[NB3];
        double W = basis_at(a, pidx[s], q, rho, pv);
#pragma unroll
        for (int i = 0; i < NB3; ++i) {
            double wi = W * pv[i];
#pragma unroll
            for (int k = 0; k <= i; ++k) M[tri3(i, k)] = fma(wi, pv[k], M[tri3(i, k)]);
        }
    }
    double trace = 0.0;
#pragma unroll
    for (int i = 0; i < NB3; ++i) trace += M[tri3(i, i)];
    bool ok = e > b;
#pragma unroll
    for (int j = 0; j < NB3; ++j) {
        double d = M[tri3(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= M[tri3(j, k)] * M[tri3(j, k)];
        if (!(d > 1e-13 * trace)) { ok = false; d = 1.0; }
        double lj = sqrt(d);
        M[tri3(j, j)] = lj;
#pragma unroll
        for (int i = j + 1; i < NB3; ++i) {
            double s = M[tri3(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= M[tri3(i, k)] * M[tri3(j, k)];
            M[tri3(i, j)] = s / lj;
        }
    }
    if (!ok) {
        flag(status, bad, VIP_ERR_SINGULAR_STENCIL, p);
        return;
    }
    const bool node = p < a.N;
    const int nk = node ? NDER3 : 1;
    for (int kk = 0; kk < nk; ++kk) {
        const int kb = c_dbasis[kk];
        // L y = e_kb, then L^T z = y
        double z[NB3];
#pragma unroll
        for (int i = 0; i < NB3; ++i) {
            double s = (i == kb) ? 1.0 : 0.0;
#pragma unroll
            for (int m = 0; m < i; ++m) s -= M[tri3(i, m)] * z[m];
            z[i] = s / M[tri3(i, i)];
        }
#pragma unroll
        for (int i = NB3 - 1; i >= 0; --i) {
            double s = z[i];
#pragma unroll
            for (int m = i + 1; m < NB3; ++m) s -= M[tri3(m, i)] * z[m];
            z[i] = s / M[tri3(i, i)];
        }
        double fac = 1.0;
        if (kb >= 1 && kb <= 3) fac = 1.0 / rho;
        else if (kb >= 4) fac = 2.0 / (rho * rho);
        for (int64_t s = b; s < e; ++s) {
            double pv[NB3];
            double W = basis_at(a, pidx[s], q, rho, pv);
            double dot = 0.0;
#pragma unroll
            for (int i = 0; i < NB3; ++i) dot = fma(z[i], pv[i], dot);
            double psi = (fac * W) * dot;
            if (node) wnode[(int64_t)kk * nnz_nodes + s] = psi;
            else w0[s - nnz_nodes] = psi;
        }
    }
}

// ---- table assembly -------------------------------------------------------
struct Asm {
    Pts a;
    const int64_t* pptr;
    const int32_t* pidx;
    const double* wnode;
    const double* w0;
    int64_t nnz_nodes;
    const int32_t* ipos;   // [N] position in the interior list or -1
    const int32_t* bpos;   // [N] position in the boundary list or -1
};

// The two sorted source lists of row r for the merged tables: op GX/GY/GZ (the
// VIP pair of the axis) or NEUMANN (the two normal points).  Returns false for
// rows without entries.
__device__ __forceinline__ bool row_sources(const Asm& A, int op, int64_t r, int64_t& p1, int64_t& p2) {
    if (op == VIP3_OP_NEUMANN) {
        int32_t i = A.bpos[r];
        if (i < 0) return false;
        p1 = A.a.N + 6 * A.a.Ni + i;
        p2 = p1 + A.a.Nb;
        return true;
    }
    int32_t i = A.ipos[r];
    if (i < 0) return false;
    int ax = op - VIP3_OP_GX;
    p1 = A.a.N + (int64_t)(2 * ax) * A.a.Ni + i;
    p2 = p1 + A.a.Ni;
    return true;
}

// Walks the union of the two lists (and, for NEUMANN, the row's own node) in
// ascending column order, calling f(col, value).
template <class F>
__device__ __forceinline__ void merge_row(const Asm& A, int op, int64_t r, F f) {
    int64_t p1, p2;
    if (!row_sources(A, op, r, p1, p2)) return;
    int64_t i1 = A.pptr[p1], e1 = A.pptr[p1 + 1], i2 = A.pptr[p2], e2 = A.pptr[p2 + 1];
    const int64_t off = A.nnz_nodes;
    if (op == VIP3_OP_NEUMANN) {
        // q_r - (4/3) q(probe 1) + (1/3) q(probe 2), summed in that order
        bool diag = false;
        while (i1 < e1 || i2 < e2 || !diag) {
            int32_t c1 = i1 < e1 ? A.pidx[i1] : INT32_MAX;
            int32_t c2 = i2 < e2 ? A.pidx[i2] : INT32_MAX;
            int32_t cd = diag ? INT32_MAX : (int32_t)r;
            int32_t c = min(cd, min(c1, c2));
            double v = (c == cd) ? 1.0 : 0.0;
            if (c == cd) diag = true;
            if (c == c1) { v = __dsub_rn(v, __dmul_rn(4.0 / 3.0, A.w0[i1 - off])); ++i1; }
            else v = __dsub_rn(v, 0.0);
            if (c == c2) { v = __dadd_rn(v, __dmul_rn(1.0 / 3.0, A.w0[i2 - off])); ++i2; }
            f(c, v);
        }
        return;
    }
    const int ax = op - VIP3_OP_GX;
    double qa[3], qb[3], rho;
    int64_t owner;
    point_of(A.a, p1, qa, rho, owner);
    point_of(A.a, p2, qb, rho, owner);
    const double inv = 1.0 / fabs(__dsub_rn(qa[ax], qb[ax]));
    while (i1 < e1 || i2 < e2) {
        int32_t c1 = i1 < e1 ? A.pidx[i1] : INT32_MAX;
        int32_t c2 = i2 < e2 ? A.pidx[i2] : INT32_MAX;
        int32_t c = min(c1, c2);
        double v;
        if (c1 == c2) { v = __dsub_rn(A.w0[i1 - off], A.w0[i2 - off]); ++i1; ++i2; }
        else if (c == c1) { v = A.w0[i1 - off]; ++i1; }
        else { v = -A.w0[i2 - off]; ++i2; }
        f(c, __dmul_rn(v, inv));
    }
}

__global__ void k3_merge_count(Asm A, int op, int32_t* __restrict__ rowlen) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.a.N) return;
    int n = 0;
    merge_row(A, op, r, [&](int32_t, double) { ++n; });
    rowlen[r] = n;
}

__global__ void k3_merge_fill(Asm A, int op, const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                              double* __restrict__ val) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.a.N) return;
    int64_t w = ptr[r];
    const int64_t e = ptr[r + 1];
    merge_row(A, op, r, [&](int32_t c, double v) {
        if (w < e) { col[w] = c; val[w] = v; ++w; }
    });
}

// Rows of the VIP interpolation table k: the VIP's own list at interior rows.
__global__ void k3_vip_count(Asm A, int k, int32_t* __restrict__ rowlen) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.a.N) return;
    int32_t i = A.ipos[r];
    int n = 0;
    if (i >= 0) {
        int64_t p = A.a.N + (int64_t)k * A.a.Ni + i;
        n = (int)(A.pptr[p + 1] - A.pptr[p]);
    }
    rowlen[r] = n;
}

__global__ void k3_vip_fill(Asm A, int k, const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                            double* __restrict__ val) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.a.N) return;
    int32_t i = A.ipos[r];
    if (i < 0) return;
    int64_t p = A.a.N + (int64_t)k * A.a.Ni + i;
    int64_t w = ptr[r];
    for (int64_t s = A.pptr[p]; s < A.pptr[p + 1]; ++s, ++w) {
        col[w] = A.pidx[s];
        val[w] = A.w0[s - A.nnz_nodes];
    }
}

// Node tables: NBR (value 1), D000..D002, LAPLACE = (D200 + D020) + D002.
__global__ void k3_node_vals(Asm A, int op, double* __restrict__ val) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.nnz_nodes) return;
    double v;
    if (op == VIP3_OP_NBR) v = 1.0;
    else if (op == VIP3_OP_LAPLACE)
        v = __dadd_rn(__dadd_rn(A.wnode[4 * A.nnz_nodes + s], A.wnode[5 * A.nnz_nodes + s]),
                      A.wnode[6 * A.nnz_nodes + s]);
    else v = A.wnode[(int64_t)(op - VIP3_OP_D000) * A.nnz_nodes + s];
    val[s] = v;
}

__global__ void k3_csr_apply(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ x,
                             double* __restrict__ y) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s = 0.0;
    for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) s = fma(val[k], x[col[k]], s);
    y[r] = s;
}

// ---- exclusive scan of int32 counts into int64 offsets (out[n] = total) ----
constexpr int SCAN_T = 256, SCAN_E = 4, SCAN_CHUNK = SCAN_T * SCAN_E;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        int64_t add = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int64_t incl = sh[t];
    *total = sh[SCAN_T - 1];
    __syncthreads();
    return incl - v;
}

__global__ void __launch_bounds__(SCAN_T) k3_scan_local(const int32_t* __restrict__ in, int64_t n,
                                                        int64_t* __restrict__ out,
                                                        int64_t* __restrict__ bsum) {
    __shared__ int64_t sh[SCAN_T];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_E;
    int64_t v[SCAN_E], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_E; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t run = block_excl_scan(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_E; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k3_scan_blocks(int64_t* __restrict__ bsum, int64_t nb,
                                                         int64_t* __restrict__ total) {
    __shared__ int64_t sh[SCAN_T];
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += SCAN_T) {
        int64_t i = c0 + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k3_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ boff) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / SCAN_CHUNK];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct vip_3d {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int weight = VIP_W_CUBIC_SPLINE;
    double support = 2.2;
    int64_t N = 0, Ni = 0, Nb = 0;
    double L[3] = {0, 0, 0};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, hmax = 0.0;
    std::vector<void*> node_bufs;     // freed on a new node set
    std::vector<void*> build_bufs;    // freed on a new build
    double *x = nullptr, *y = nullptr, *z = nullptr, *nx = nullptr, *ny = nullptr, *nz = nullptr,
           *h = nullptr;
    int32_t *interior = nullptr, *boundary = nullptr, *ipos = nullptr, *bpos = nullptr;
    bool built = false;
    Pts pts{};
    int64_t P = 0, nnz_all = 0, nnz_nodes = 0;
    int64_t* pptr = nullptr;
    int32_t* pidx = nullptr;
    double* wnode = nullptr;
    double* w0 = nullptr;
    Csr tab[VIP3_OP_COUNT];
    bool have[VIP3_OP_COUNT] = {};
};

namespace {

vip_status fail(vip_3d* b, vip_status st, const std::string& msg) {
    b->err = msg;
    return st;
}

#define V3_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (void)cudaGetLastError();                                                      \
            return fail(b, e_ == cudaErrorMemoryAllocation ? VIP_ERR_OOM : VIP_ERR_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
        }                                                                                  \
    } while (0)

template <class T>
cudaError_t alloc(std::vector<void*>& owner, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) owner.push_back(q);
    *p = static_cast<T*>(q);
    return e;
}

void free_all(std::vector<void*>& v) {
    for (void* p : v) cudaFree(p);
    v.clear();
}

void reset_build(vip_3d* b) {
    free_all(b->build_bufs);
    b->built = false;
    for (int i = 0; i < VIP3_OP_COUNT; ++i) { b->tab[i] = Csr{}; b->have[i] = false; }
    b->pptr = nullptr; b->pidx = nullptr; b->wnode = nullptr; b->w0 = nullptr;
    b->P = b->nnz_all = b->nnz_nodes = 0;
}

struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(d) == cudaSuccess;
    }
    ~DeviceScope() { if (prev >= 0) cudaSetDevice(prev); }
};

// out[0..n] = exclusive scan of in[0..n) (out[n] = total); *total_host gets the total.
vip_status scan_counts(vip_3d* b, const int32_t* in, int64_t n, int64_t* out, int64_t* total_host) {
    const int64_t nb = std::max<int64_t>(1, (n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    std::vector<void*> tmp;
    int64_t* bsum = nullptr;
    cudaError_t e = alloc(tmp, &bsum, nb);
    if (e != cudaSuccess) { free_all(tmp); V3_CUDA(e); }
    k3_scan_local<<<(unsigned)nb, SCAN_T, 0, b->stream>>>(in, n, out, bsum);
    k3_scan_blocks<<<1, SCAN_T, 0, b->stream>>>(bsum, nb, out + n);
    k3_scan_add<<<blocks_for(n, 256), 256, 0, b->stream>>>(out, n, bsum);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(total_host, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    free_all(tmp);
    V3_CUDA(e);
    return VIP_OK;
}

Asm asm_view(const vip_3d* b) {
    Asm A;
    A.a = b->pts;
    A.pptr = b->pptr;
    A.pidx = b->pidx;
    A.wnode = b->wnode;
    A.w0 = b->w0;
    A.nnz_nodes = b->nnz_nodes;
    A.ipos = b->ipos;
    A.bpos = b->bpos;
    return A;
}

vip_status assemble(vip_3d* b, int op) {
    if (b->have[op]) return VIP_OK;
    const int64_t N = b->N;
    Asm A = asm_view(b);
    Csr T;
    if (op <= VIP3_OP_LAPLACE) {
        V3_CUDA(alloc(b->build_bufs, &T.ptr, N + 1));
        V3_CUDA(cudaMemcpyAsync(T.ptr, b->pptr, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, b->stream));
        T.col = b->pidx;          // the node points' lists come first
        T.nnz = b->nnz_nodes;
        V3_CUDA(alloc(b->build_bufs, &T.val, T.nnz));
        k3_node_vals<<<blocks_for(T.nnz, 256), 256, 0, b->stream>>>(A, op, T.val);
        V3_CUDA(cudaGetLastError());
    } else {
        std::vector<void*> tmp;
        int32_t* rowlen = nullptr;
        cudaError_t e = alloc(tmp, &rowlen, N);
        if (e != cudaSuccess) { free_all(tmp); V3_CUDA(e); }
        const bool vip = op <= VIP3_OP_VIP_B;
        if (vip) k3_vip_count<<<blocks_for(N, 256), 256, 0, b->stream>>>(A, op - VIP3_OP_VIP_E, rowlen);
        else k3_merge_count<<<blocks_for(N, 128), 128, 0, b->stream>>>(A, op, rowlen);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = alloc(b->build_bufs, &T.ptr, N + 1);
        if (e != cudaSuccess) { free_all(tmp); V3_CUDA(e); }
        vip_status st = scan_counts(b, rowlen, N, T.ptr, &T.nnz);
        free_all(tmp);
        if (st != VIP_OK) return st;
        V3_CUDA(alloc(b->build_bufs, &T.col, T.nnz));
        V3_CUDA(alloc(b->build_bufs, &T.val, T.nnz));
        if (vip) k3_vip_fill<<<blocks_for(N, 256), 256, 0, b->stream>>>(A, op - VIP3_OP_VIP_E, T.ptr, T.col, T.val);
        else k3_merge_fill<<<blocks_for(N, 128), 128, 0, b->stream>>>(A, op, T.ptr, T.col, T.val);
        V3_CUDA(cudaGetLastError());
    }
    V3_CUDA(cudaStreamSynchronize(b->stream));
    b->tab[op] = T;
    b->have[op] = true;
    return VIP_OK;
}

bool finite_all(const std::vector<double>& v) {
    for (double d : v) if (!std::isfinite(d)) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

vip_status vip_3d_create(vip_3d** out, int device, void* cuda_stream) {
    if (!out) return VIP_ERR_ARG;
    *out = nullptr;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
        (void)cudaGetLastError();
        return VIP_ERR_ARG;
    }
    vip_3d* b = new (std::nothrow) vip_3d();
    if (!b) return VIP_ERR_OOM;
    b->device = device;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    *out = b;
    return VIP_OK;
}

void vip_3d_destroy(vip_3d* b) {
    if (!b) return;
    DeviceScope ds(b->device);
    free_all(b->build_bufs);
    free_all(b->node_bufs);
    delete b;
}

const char* vip_3d_last_error(const vip_3d* b) { return b ? b->err.c_str() : "null handle"; }

vip_status vip_3d_set_mls(vip_3d* b, int weight, double support) {
    if (!b) return VIP_ERR_ARG;
    if (weight != VIP_W_CUBIC_SPLINE && weight != VIP_W_PAPER)
        return fail(b, VIP_ERR_ARG, "weight must be VIP_W_CUBIC_SPLINE or VIP_W_PAPER");
    if (!(support > 1.0) || !std::isfinite(support)) return fail(b, VIP_ERR_ARG, "support must be > 1");
    b->weight = weight;
    b->support = support;
    reset_build(b);
    return VIP_OK;
}

vip_status vip_3d_set_nodes(vip_3d* b, int64_t n, const double* x, const double* y, const double* z,
                            const uint8_t* kind, const double* nx, const double* ny, const double* nz,
                            const double* h, double Lx, double Ly, double Lz) {
    if (!b) return VIP_ERR_ARG;
    if (n < 1 || n >= INT32_MAX) return fail(b, VIP_ERR_ARG, "node count out of range");
    if (!x || !y || !z || !kind || !nx || !ny || !nz || !h) return fail(b, VIP_ERR_ARG, "null array");
    const double Ls[3] = {Lx, Ly, Lz};
    const int nper = (Lx > 0) + (Ly > 0) + (Lz > 0);
    for (double l : Ls)
        if (!std::isfinite(l) || l < 0.0) return fail(b, VIP_ERR_ARG, "periods must be finite and >= 0");
    if (nper != 0 && nper != 3) return fail(b, VIP_ERR_ARG, "periodic in every direction or in none");
    DeviceScope ds(b->device);
    if (!ds.ok) return fail(b, VIP_ERR_CUDA, "cudaSetDevice failed");
    // stage on the host (the inputs may be host or device memory) and check
    std::vector<double> hx(n), hy(n), hz(n), hnx(n), hny(n), hnz(n), hh(n);
    std::vector<uint8_t> hk(n);
    const double* src[7] = {x, y, z, nx, ny, nz, h};
    std::vector<double>* dst[7] = {&hx, &hy, &hz, &hnx, &hny, &hnz, &hh};
    for (int i = 0; i < 7; ++i) V3_CUDA(cudaMemcpy(dst[i]->data(), src[i], n * sizeof(double), cudaMemcpyDefault));
    V3_CUDA(cudaMemcpy(hk.data(), kind, n, cudaMemcpyDefault));
    for (int i = 0; i < 7; ++i)
        if (!finite_all(*dst[i])) return fail(b, VIP_ERR_ARG, "non-finite input");
    std::vector<int32_t> interior, boundary, ipos(n, -1), bpos(n, -1);
    double hmax = 0.0;
    double lo[3] = {hx[0], hy[0], hz[0]}, hi[3] = {hx[0], hy[0], hz[0]};
    for (int64_t i = 0; i < n; ++i) {
        if (!(hh[i] > 0.0)) return fail(b, VIP_ERR_ARG, "h must be > 0");
        if (hk[i] > VIP_NODE_OUTLET) return fail(b, VIP_ERR_ARG, "unknown node kind");
        if (hk[i] == VIP_NODE_INTERIOR) {
            ipos[i] = (int32_t)interior.size();
            interior.push_back((int32_t)i);
        } else {
            if (nper) return fail(b, VIP_ERR_ARG, "a periodic node set has interior nodes only");
            bpos[i] = (int32_t)boundary.size();
            boundary.push_back((int32_t)i);
        }
        hmax = std::max(hmax, hh[i]);
        const double c[3] = {hx[i], hy[i], hz[i]};
        for (int k = 0; k < 3; ++k) {
            if (nper && !(c[k] >= 0.0 && c[k] < Ls[k]))
                return fail(b, VIP_ERR_ARG, "periodic coordinates must lie in [0, L)");
            lo[k] = std::min(lo[k], c[k]);
            hi[k] = std::max(hi[k], c[k]);
        }
    }
    reset_build(b);
    free_all(b->node_bufs);
    b->N = 0;
    double** dptr[7] = {&b->x, &b->y, &b->z, &b->nx, &b->ny, &b->nz, &b->h};
    for (int i = 0; i < 7; ++i) {
        V3_CUDA(alloc(b->node_bufs, dptr[i], n));
        V3_CUDA(cudaMemcpy(*dptr[i], dst[i]->data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    V3_CUDA(alloc(b->node_bufs, &b->interior, interior.size()));
    V3_CUDA(alloc(b->node_bufs, &b->boundary, boundary.size()));
    V3_CUDA(alloc(b->node_bufs, &b->ipos, n));
    V3_CUDA(alloc(b->node_bufs, &b->bpos, n));
    if (!interior.empty())
        V3_CUDA(cudaMemcpy(b->interior, interior.data(), interior.size() * 4, cudaMemcpyHostToDevice));
    if (!boundary.empty())
        V3_CUDA(cudaMemcpy(b->boundary, boundary.data(), boundary.size() * 4, cudaMemcpyHostToDevice));
    V3_CUDA(cudaMemcpy(b->ipos, ipos.data(), n * 4, cudaMemcpyHostToDevice));
    V3_CUDA(cudaMemcpy(b->bpos, bpos.data(), n * 4, cudaMemcpyHostToDevice));
    b->N = n;
    b->Ni = (int64_t)interior.size();
    b->Nb = (int64_t)boundary.size();
    for (int k = 0; k < 3; ++k) { b->L[k] = Ls[k]; b->lo[k] = lo[k]; b->hi[k] = hi[k]; }
    b->hmax = hmax;
    return VIP_OK;
}

vip_status vip_3d_build(vip_3d* b) {
    if (!b) return VIP_ERR_ARG;
    if (b->N < 1) return fail(b, VIP_ERR_ARG, "no node set");
    DeviceScope ds(b->device);
    if (!ds.ok) return fail(b, VIP_ERR_CUDA, "cudaSetDevice failed");
    reset_build(b);
    const int64_t N = b->N;
    const double rmax = b->support * b->hmax;
    // cell grid: cells of side >= the largest rho, at most about 8 N cells
    Pts& a = b->pts;
    a = Pts{};
    a.x = b->x; a.y = b->y; a.z = b->z; a.nx = b->nx; a.ny = b->ny; a.nz = b->nz; a.h = b->h;
    a.interior = b->interior; a.boundary = b->boundary;
    a.N = N; a.Ni = b->Ni; a.Nb = b->Nb;
    a.support = b->support; a.weight = b->weight;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        a.L[k] = b->L[k];
        double ext = a.L[k] > 0.0 ? a.L[k] : b->hi[k] - b->lo[k];
        a.lo[k] = a.L[k] > 0.0 ? 0.0 : b->lo[k];
        a.nc[k] = (int)std::max(1.0, std::min(1.0e6, std::floor(ext / rmax)));
    }
    while ((ncell = (int64_t)a.nc[0] * a.nc[1] * a.nc[2]) > 8 * N + 4096) {
        for (int k = 0; k < 3; ++k)
            if (a.nc[k] > 3) a.nc[k] = std::max(3, (int)(a.nc[k] / 1.26));
    }
    for (int k = 0; k < 3; ++k) {
        double ext = a.L[k] > 0.0 ? a.L[k] : b->hi[k] - b->lo[k];
        a.cs[k] = ext > 0.0 ? ext / a.nc[k] : 1.0;
        if (ext > 0.0 && a.cs[k] < rmax) a.cs[k] = rmax;   // rounding guard
    }
    std::vector<void*> tmp;
    auto tmp_fail = [&](cudaError_t e) { free_all(tmp); return e; };
    int64_t* node_cell = nullptr;
    int32_t *cnt = nullptr, *cursor = nullptr;
    int64_t* cell_ptr = nullptr;
    int32_t* cell_nodes = nullptr;
    int* status = nullptr;
    long long* bad = nullptr;
    cudaError_t e = alloc(tmp, &node_cell, N);
    if (e == cudaSuccess) e = alloc(tmp, &cnt, ncell);
    if (e == cudaSuccess) e = alloc(tmp, &cursor, ncell);
    if (e == cudaSuccess) e = alloc(b->build_bufs, &cell_ptr, ncell + 1);
    if (e == cudaSuccess) e = alloc(b->build_bufs, &cell_nodes, N);
    if (e == cudaSuccess) e = alloc(tmp, &status, 1);
    if (e == cudaSuccess) e = alloc(tmp, &bad, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, ncell * sizeof(int32_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, ncell * sizeof(int32_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), b->stream);
    const long long big = INT64_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, &big, sizeof(long long), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) V3_CUDA(tmp_fail(e));
    a.cell_ptr = cell_ptr;
    a.cell_nodes = cell_nodes;
    k3_cell_count<<<blocks_for(N, 256), 256, 0, b->stream>>>(a, node_cell, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) V3_CUDA(tmp_fail(e));
    int64_t tot = 0;
    vip_status st = scan_counts(b, cnt, ncell, cell_ptr, &tot);
    if (st != VIP_OK) { free_all(tmp); return st; }
    k3_cell_fill<<<blocks_for(N, 256), 256, 0, b->stream>>>(N, node_cell, cell_ptr, cursor, cell_nodes);
    if ((e = cudaGetLastError()) != cudaSuccess) V3_CUDA(tmp_fail(e));
    // points and their neighbour lists
    const int64_t P = N + 6 * b->Ni + 2 * b->Nb;
    int32_t* pcnt = nullptr;
    if ((e = alloc(tmp, &pcnt, P)) != cudaSuccess) V3_CUDA(tmp_fail(e));
    if ((e = alloc(b->build_bufs, &b->pptr, P + 1)) != cudaSuccess) V3_CUDA(tmp_fail(e));
    k3_nbr_count<<<blocks_for(P, 128), 128, 0, b->stream>>>(a, P, pcnt, status, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) V3_CUDA(tmp_fail(e));
    int hst = 0;
    long long hbad = 0;
    if ((e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hbad, bad, sizeof(long long), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        V3_CUDA(tmp_fail(e));
    if (hst != 0) {
        free_all(tmp);
        return fail(b, (vip_status)hst, "point " + std::to_string(hbad) + " has more than " +
                                             std::to_string(K3MAX) + " neighbours");
    }
    int64_t nnz = 0;
    st = scan_counts(b, pcnt, P, b->pptr, &nnz);
    if (st != VIP_OK) { free_all(tmp); return st; }
    int64_t nnz_nodes = 0;
    if ((e = cudaMemcpy(&nnz_nodes, b->pptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        V3_CUDA(tmp_fail(e));
    if ((e = alloc(b->build_bufs, &b->pidx, nnz)) != cudaSuccess) V3_CUDA(tmp_fail(e));
    if ((e = alloc(b->build_bufs, &b->wnode, (size_t)NDER3 * nnz_nodes)) != cudaSuccess) V3_CUDA(tmp_fail(e));
    if ((e = alloc(b->build_bufs, &b->w0, nnz - nnz_nodes)) != cudaSuccess) V3_CUDA(tmp_fail(e));
    k3_nbr_fill<<<blocks_for(P, 128), 128, 0, b->stream>>>(a, P, b->pptr, b->pidx);
    k3_mls<<<blocks_for(P, 128), 128, 0, b->stream>>>(a, P, b->pptr, b->pidx, b->wnode, nnz_nodes, b->w0,
                                                      status, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) V3_CUDA(tmp_fail(e));
    if ((e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hbad, bad, sizeof(long long), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        V3_CUDA(tmp_fail(e));
    free_all(tmp);
    if (hst != 0) return fail(b, (vip_status)hst, "moment matrix of point " + std::to_string(hbad) +
                                                      " failed its Cholesky test");
    b->P = P;
    b->nnz_all = nnz;
    b->nnz_nodes = nnz_nodes;
    b->built = true;
    return VIP_OK;
}

vip_status vip_3d_stencil_size(vip_3d* b, int which, int64_t* nrows, int64_t* nnz) {
    if (!b) return VIP_ERR_ARG;
    if (!b->built) return fail(b, VIP_ERR_ARG, "not built");
    if (which < 0 || which >= VIP3_OP_COUNT) return fail(b, VIP_ERR_ARG, "bad table");
    DeviceScope ds(b->device);
    vip_status st = assemble(b, which);
    if (st != VIP_OK) return st;
    if (nrows) *nrows = b->N;
    if (nnz) *nnz = b->tab[which].nnz;
    return VIP_OK;
}

vip_status vip_3d_get_stencil(vip_3d* b, int which, int64_t* row_ptr, int32_t* col, double* val) {
    vip_status st = vip_3d_stencil_size(b, which, nullptr, nullptr);
    if (st != VIP_OK) return st;
    if (!row_ptr || !col || !val) return fail(b, VIP_ERR_ARG, "null array");
    DeviceScope ds(b->device);
    const Csr& T = b->tab[which];
    V3_CUDA(cudaMemcpyAsync(row_ptr, T.ptr, (b->N + 1) * sizeof(int64_t), cudaMemcpyDefault, b->stream));
    if (T.nnz) {
        V3_CUDA(cudaMemcpyAsync(col, T.col, T.nnz * sizeof(int32_t), cudaMemcpyDefault, b->stream));
        V3_CUDA(cudaMemcpyAsync(val, T.val, T.nnz * sizeof(double), cudaMemcpyDefault, b->stream));
    }
    V3_CUDA(cudaStreamSynchronize(b->stream));
    return VIP_OK;
}

vip_status vip_3d_apply(vip_3d* b, int which, const double* x, double* y) {
    vip_status st = vip_3d_stencil_size(b, which, nullptr, nullptr);
    if (st != VIP_OK) return st;
    if (!x || !y) return fail(b, VIP_ERR_ARG, "null array");
    DeviceScope ds(b->device);
    const int64_t N = b->N;
    std::vector<void*> tmp;
    double *dx = nullptr, *dy = nullptr;
    cudaError_t e = alloc(tmp, &dx, N);
    if (e == cudaSuccess) e = alloc(tmp, &dy, N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, N * sizeof(double), cudaMemcpyDefault, b->stream);
    const Csr& T = b->tab[which];
    if (e == cudaSuccess) {
        k3_csr_apply<<<blocks_for(N, 256), 256, 0, b->stream>>>(N, T.ptr, T.col, T.val, dx, dy);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, dy, N * sizeof(double), cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    free_all(tmp);
    V3_CUDA(e);
    return VIP_OK;
}

}  // extern "C"
