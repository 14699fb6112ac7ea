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

// ---- the fractional step in 3D (Sec. 2, Eqs. 12-15) ----------------------
// Convection at every node (Sec. 4.1 item 1 in three coordinates): the products
// of the six VIP interpolations of (u, v, w), differenced across each VIP pair
// and divided by the pair distance.
__global__ void k3_conv(Asm A, const double* __restrict__ u, const double* __restrict__ v,
                        const double* __restrict__ w, double* __restrict__ Nu,
                        double* __restrict__ Nv, double* __restrict__ Nw) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.a.N) return;
    const int32_t i = A.ipos[r];
    if (i < 0) { Nu[r] = Nv[r] = Nw[r] = 0.0; return; }
    double val[6][3];
    double inv[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int64_t p = A.a.N + (int64_t)k * A.a.Ni + i;
        double su = 0.0, sv = 0.0, sw = 0.0;
        for (int64_t s = A.pptr[p]; s < A.pptr[p + 1]; ++s) {
            const double wt = A.w0[s - A.nnz_nodes];
            const int32_t j = A.pidx[s];
            su = fma(wt, u[j], su);
            sv = fma(wt, v[j], sv);
            sw = fma(wt, w[j], sw);
        }
        val[k][0] = su; val[k][1] = sv; val[k][2] = sw;
    }
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        double qa[3], qb[3], rho;
        int64_t owner;
        point_of(A.a, A.a.N + (int64_t)(2 * ax) * A.a.Ni + i, qa, rho, owner);
        point_of(A.a, A.a.N + (int64_t)(2 * ax + 1) * A.a.Ni + i, qb, rho, owner);
        inv[ax] = 1.0 / fabs(qa[ax] - qb[ax]);
    }
    double out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double f = 0.0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            f += (val[2 * ax][ax] * val[2 * ax][c] - val[2 * ax + 1][ax] * val[2 * ax + 1][c]) * inv[ax];
        out[c] = f;
    }
    Nu[r] = out[0]; Nv[r] = out[1]; Nw[r] = out[2];
}

__device__ __forceinline__ double csr_row(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, int64_t r,
                                          const double* __restrict__ x) {
    double s = 0.0;
    for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) s = fma(val[k], x[col[k]], s);
    return s;
}

struct Tab3 { const int64_t* ptr; const int32_t* col; const double* val; };

// Right-hand side of Eq. (12) times dt for one component at interior rows:
// (I + alpha L) u^n - dt (1.5 N^n - 0.5 N^{n-1} + G p^n); wall rows: the node's
// boundary value.
__global__ void k3_rhs(int64_t N, Tab3 L, Tab3 G, double alpha, double dt, const int32_t* __restrict__ ipos,
                       const double* __restrict__ bc, const double* __restrict__ uc,
                       const double* __restrict__ Ncur, const double* __restrict__ Nprev,
                       const double* __restrict__ p, double* __restrict__ rhs) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    if (ipos[r] < 0) { rhs[r] = bc[r]; return; }      // wall: the boundary value
    const double Lu = csr_row(L.ptr, L.col, L.val, r, uc);
    const double Gp = csr_row(G.ptr, G.col, G.val, r, p);
    const double nab = 1.5 * Ncur[r] - 0.5 * Nprev[r];
    rhs[r] = (uc[r] + alpha * Lu) - dt * (nab + Gp);
}

// Eq. (13) right-hand side, bordered: b_i = (Gx u* + Gy v* + Gz w*)_i / dt at
// interior rows, 0 at wall rows, then b_N = b_k0 and b_k0 = 0 (k0 the first
// interior node).
__global__ void k3_div(int64_t N, Tab3 Gx, Tab3 Gy, Tab3 Gz, double dt, int64_t k0,
                       const int32_t* __restrict__ ipos, const double* __restrict__ us,
                       const double* __restrict__ vs, const double* __restrict__ ws,
                       double* __restrict__ b) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    if (ipos[r] < 0) { b[r] = 0.0; return; }          // wall rows: zero normal derivative = 0
    double d = (csr_row(Gx.ptr, Gx.col, Gx.val, r, us) + csr_row(Gy.ptr, Gy.col, Gy.val, r, vs)
                + csr_row(Gz.ptr, Gz.col, Gz.val, r, ws)) / dt;
    if (r == k0) { b[N] = d; b[r] = 0.0; }
    else b[r] = d;
}

// Eqs. (14)-(15): u = u* - dt G phi at interior rows; p = p + phi - alpha L phi
// at every node.
__global__ void k3_project(int64_t N, Tab3 L, Tab3 Gx, Tab3 Gy, Tab3 Gz, double alpha, double dt,
                           const int32_t* __restrict__ ipos, const double* __restrict__ phi,
                           const double* __restrict__ us, const double* __restrict__ vs,
                           const double* __restrict__ ws, double* __restrict__ u, double* __restrict__ v,
                           double* __restrict__ w, double* __restrict__ p) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    if (ipos[r] >= 0) {
        u[r] = us[r] - dt * csr_row(Gx.ptr, Gx.col, Gx.val, r, phi);
        v[r] = vs[r] - dt * csr_row(Gy.ptr, Gy.col, Gy.val, r, phi);
        w[r] = ws[r] - dt * csr_row(Gz.ptr, Gz.col, Gz.val, r, phi);
    } else {                                          // walls keep their values
        u[r] = us[r]; v[r] = vs[r]; w[r] = ws[r];
    }
    p[r] = (p[r] + phi[r]) - alpha * csr_row(L.ptr, L.col, L.val, r, phi);
}

// The two systems of the step, applied matrix-free from L:
//   HELM: y = x - alpha L x at interior rows, y = x at wall rows      (n = N)
//   POIS: the bordered Poisson system (n = N + 1, x_N = mu): interior rows
//         y_i = (L x)_i + mu, wall rows y_i = (-6/h_i^2) (Nb x)_i, y_k0 =
//         (-6/h_k0^2) x_k0, y_N = (L x)_k0 + mu.
enum { OPK_HELM = 0, OPK_POIS = 1 };
struct Op3 {
    int kind;
    int64_t n, N, k0;
    double alpha;
    Tab3 L, Nb;
    const int32_t* ipos;
    const double* h;
};

__device__ __forceinline__ double op_row(const Op3& o, int64_t r, const double* __restrict__ x) {
    if (o.kind == OPK_HELM)
        return o.ipos[r] >= 0 ? x[r] - o.alpha * csr_row(o.L.ptr, o.L.col, o.L.val, r, x) : x[r];
    if (r == o.k0) return (-6.0 / (o.h[r] * o.h[r])) * x[r];
    if (r < o.N && o.ipos[r] < 0)
        return (-6.0 / (o.h[r] * o.h[r])) * csr_row(o.Nb.ptr, o.Nb.col, o.Nb.val, r, x);
    const int64_t row = r == o.N ? o.k0 : r;
    return csr_row(o.L.ptr, o.L.col, o.L.val, row, x) + x[o.N];
}

__global__ void k3_op(Op3 o, const double* __restrict__ x, double* __restrict__ y) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < o.n) y[r] = op_row(o, r, x);
}

// Sum of two values over a 256-thread block, in a fixed tree; thread 0 writes them.
__device__ __forceinline__ void block_sum2(double a, double b, double* __restrict__ out) {
    __shared__ double s0[256], s1[256];
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s0[0]; out[1] = s1[0]; }
}

// Deterministic dot products: fixed grid, per-thread strided sums, a fixed tree
// in each block, then one block sums the block partials in order.
constexpr int DOT_B = 256, DOT_T = 256;

__global__ void __launch_bounds__(DOT_T) k3_dot2(int64_t n, const double* __restrict__ a,
                                                 const double* __restrict__ b, const double* __restrict__ c,
                                                 const double* __restrict__ d, double* __restrict__ part) {
    __shared__ double s0[DOT_T], s1[DOT_T];
    double x0 = 0.0, x1 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_T + threadIdx.x; i < n; i += (int64_t)DOT_B * DOT_T) {
        x0 = fma(a[i], b[i], x0);
        if (c) x1 = fma(c[i], d[i], x1);
    }
    s0[threadIdx.x] = x0;
    s1[threadIdx.x] = x1;
    __syncthreads();
    for (int o = DOT_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
}

__global__ void __launch_bounds__(DOT_B) k3_dot_final(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double s0[DOT_B], s1[DOT_B];
    s0[threadIdx.x] = part[2 * threadIdx.x];
    s1[threadIdx.x] = part[2 * threadIdx.x + 1];
    __syncthreads();
    for (int o = DOT_B / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s0[0]; out[1] = s1[0]; }
}

// y = a x + b y' (elementwise vector updates of BiCGSTAB)
__global__ void k3_lin2(int64_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// Device-resident scalars of one BiCGSTAB inner loop.  The single-thread kernels
// below apply the same IEEE operations the host would, so the iterates do not
// depend on where the scalars live; every vector kernel does nothing once the
// state has left "running".
enum { KS_RUN = 0, KS_LEAVE = 1, KS_RESTART = 2, KS_ADD_LEAVE = 3 };
struct KS {
    double rho, rho_old, alpha, omega, beta, rhat_norm, tol, brk;
    double d[2];            // results of the last pair of dot products
    int32_t it, max_it, state, pad;
};

// after (r_hat . r, r . r): breakdown test, iteration count, beta
__global__ void ks_top(KS* K) {
    if (K->state != KS_RUN) return;
    if (K->it >= K->max_it) { K->state = KS_LEAVE; return; }
    const double rho = K->d[0];
    if (fabs(rho) <= K->brk * K->rhat_norm * sqrt(K->d[1])) { K->state = KS_RESTART; return; }
    K->rho = rho;
    K->it += 1;
    K->beta = (rho / K->rho_old) * (K->alpha / K->omega);
}

__global__ void ks_added(KS* K) {
    if (K->state == KS_ADD_LEAVE) K->state = KS_LEAVE;
}

__global__ void kd_pupd(int64_t n, const KS* __restrict__ K, const double* __restrict__ r,
                        const double* __restrict__ v, double* __restrict__ p) {
    if (K->state != KS_RUN) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = r[i] + K->beta * (p[i] - K->omega * v[i]);
}

__global__ void kd_axpy_add(int64_t n, const KS* __restrict__ K, const double* __restrict__ p,
                            double* __restrict__ x) {
    if (K->state != KS_ADD_LEAVE) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + K->alpha * p[i];
}

// The fused kernels below write per-block partial sums of two dot products
// (part[2 b], part[2 b + 1]); k3_final reduces them in block order and then takes
// the iteration's scalar step.  All are launched with 256-thread blocks.
// v = A p (mode 0: partials of r_hat . v and v . v) or t = A s (mode 1: t . t and
// s . t); c is r_hat (mode 0) or s (mode 1).
__global__ void __launch_bounds__(256) k3_op_dot(Op3 o, const double* __restrict__ x, double* __restrict__ y,
                                                 const KS* __restrict__ K, const double* __restrict__ c,
                                                 int mode, double* __restrict__ part) {
    if (K->state != KS_RUN) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double p0 = 0.0, p1 = 0.0;
    if (r < o.n) {
        const double yv = op_row(o, r, x);
        y[r] = yv;
        const double cy = c[r] * yv, yy = yv * yv;
        p0 = mode == 0 ? cy : yy;
        p1 = mode == 0 ? yy : cy;
    }
    block_sum2(p0, p1, part + 2 * blockIdx.x);
}

// s = r - alpha v; partials of s . s
__global__ void __launch_bounds__(256) kd_s_dot(int64_t n, const KS* __restrict__ K, const double* __restrict__ r,
                                                const double* __restrict__ v, double* __restrict__ s,
                                                double* __restrict__ part) {
    if (K->state != KS_RUN) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double p0 = 0.0;
    if (i < n) {
        const double sv = r[i] - K->alpha * v[i];
        s[i] = sv;
        p0 = sv * sv;
    }
    block_sum2(p0, 0.0, part + 2 * blockIdx.x);
}

// x = x + alpha p + omega s; r = s - omega t; partials of r_hat . r and r . r
__global__ void __launch_bounds__(256) kd_xr_dot(int64_t n, const KS* __restrict__ K, const double* __restrict__ p,
                                                 const double* __restrict__ s, const double* __restrict__ t,
                                                 const double* __restrict__ rhat, double* __restrict__ x,
                                                 double* __restrict__ r, double* __restrict__ part) {
    if (K->state != KS_RUN) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double p0 = 0.0, p1 = 0.0;
    if (i < n) {
        x[i] = x[i] + K->alpha * p[i] + K->omega * s[i];
        const double rv = s[i] - K->omega * t[i];
        r[i] = rv;
        p0 = rhat[i] * rv;
        p1 = rv * rv;
    }
    block_sum2(p0, p1, part + 2 * blockIdx.x);
}

// Reduce nblk pairs of partials in block order into K->d, then the scalar step:
//   ALPHA  (r_hat . v, v . v): breakdown test, alpha = rho / r_hat . v
//   S      (s . s): converged on s -> x += alpha p, leave
//   OMEGA  (t . t, s . t): omega (t = 0 -> x += alpha p, leave)
//   END    (r_hat . r, r . r): converged or omega = 0 -> leave, else rho_old = rho
// (the next iteration's ks_top reads r_hat . r and r . r from K->d).
enum { FIN_ALPHA = 0, FIN_S = 1, FIN_OMEGA = 2, FIN_END = 3 };
__global__ void __launch_bounds__(256) k3_final(const double* __restrict__ part, int nblk, KS* __restrict__ K,
                                                int which) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 256) { a += part[2 * k]; b += part[2 * k + 1]; }
    __shared__ double d[2];
    block_sum2(a, b, d);
    __syncthreads();
    if (threadIdx.x != 0 || K->state != KS_RUN) return;
    K->d[0] = d[0];
    K->d[1] = d[1];
    if (which == FIN_ALPHA) {
        if (fabs(d[0]) <= K->brk * K->rhat_norm * sqrt(d[1])) { K->state = KS_RESTART; return; }
        K->alpha = K->rho / d[0];
    } else if (which == FIN_S) {
        if (sqrt(d[0]) <= K->tol) K->state = KS_ADD_LEAVE;
    } else if (which == FIN_OMEGA) {
        if (d[0] == 0.0) { K->state = KS_ADD_LEAVE; return; }
        K->omega = d[1] / d[0];
    } else {
        if (sqrt(d[1]) <= K->tol || K->omega == 0.0) { K->state = KS_LEAVE; return; }
        K->rho_old = K->rho;
    }
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
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, hmax = 0.0, h0 = 0.0;
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
    // the 3D step (vip_3d_set_flow, vip_3d_set_state, vip_3d_step)
    bool flow = false, state = false, have_prev = false;
    double Re = 0.0, dt = 0.0, rtol = 1e-8;
    int32_t max_iters = 20000;
    std::vector<void*> state_bufs;    // freed on a new node set
    double* vel[3] = {nullptr, nullptr, nullptr};
    double* star[3] = {nullptr, nullptr, nullptr};
    double* Ncur[3] = {nullptr, nullptr, nullptr};
    double* Nprev[3] = {nullptr, nullptr, nullptr};
    double* bc[3] = {nullptr, nullptr, nullptr};  // wall values (the state set last)
    double *p = nullptr, *phi = nullptr;          // phi: N + 1 (mu last)
    int64_t k0 = -1;                              // first interior node
    bool other_kinds = false;                     // SLIP or OUTLET nodes present
    double* kv[8] = {};                           // Krylov vectors, N + 1 each
    double *dpart = nullptr, *dres = nullptr;     // dot partials and results
    void* ks = nullptr;                           // device BiCGSTAB scalars (KS)
    // one BiCGSTAB inner iteration as a CUDA graph per (system, solution vector),
    // captured on a private stream and replayed on `stream`; dropped whenever a
    // table, the flow parameters or the step's buffers change
    struct IterGraph { int kind; const double* x; cudaGraphExec_t exec; };
    std::vector<IterGraph> graphs;
    cudaStream_t cap = nullptr;
    int64_t steps = 0;
    int32_t last_helm = 0, last_poisson = 0;
    double last_poisson_res = 0.0;
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

void drop_graphs(vip_3d* b) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

void reset_build(vip_3d* b) {
    drop_graphs(b);
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

Tab3 tab3(const vip_3d* b, int op) {
    return Tab3{b->tab[op].ptr, b->tab[op].col, b->tab[op].val};
}

// Two dot products (the second optional) of device vectors, read back to the host.
vip_status dots(vip_3d* b, int64_t n, const double* a1, const double* b1, const double* a2,
                const double* b2, double out[2]) {
    k3_dot2<<<DOT_B, DOT_T, 0, b->stream>>>(n, a1, b1, a2, b2, b->dpart);
    k3_dot_final<<<1, DOT_B, 0, b->stream>>>(b->dpart, b->dres);
    V3_CUDA(cudaGetLastError());
    V3_CUDA(cudaMemcpyAsync(out, b->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    V3_CUDA(cudaStreamSynchronize(b->stream));
    return VIP_OK;
}

#define V3_TRY(call)                          \
    do {                                      \
        vip_status s_ = (call);               \
        if (s_ != VIP_OK) return s_;          \
    } while (0)

// Unpreconditioned BiCGSTAB (van der Vorst 1992) on o to ||rhs - A x|| <= rtol ||rhs||,
// with the oracle's rules: restart with r_hat = r when |r_hat . r| or |r_hat . v|
// falls below 1e-12 of the product of norms, and confirm convergence on the true
// residual.  x holds the initial guess.
vip_status krylov(vip_3d* b, const Op3& o, const double* rhs, double* x, int32_t* iters, double* relres) {
    const int64_t n = o.n;
    double *r = b->kv[0], *rhat = b->kv[1], *pp = b->kv[2], *v = b->kv[3], *sv = b->kv[4],
           *t = b->kv[5], *y = b->kv[6];
    KS* K = static_cast<KS*>(b->ks);
    const unsigned g = blocks_for(n, 256);
    cudaStream_t st = b->stream;
    auto apply = [&](const double* in, double* out) { k3_op<<<g, 256, 0, st>>>(o, in, out); };
    // one inner iteration, enqueued on stream q (captured once into a graph): 14
    // kernels, the dot products fused into the operator and vector kernels
    const int nblk = (int)g;
    double* part = b->dpart;
    auto iteration = [&](cudaStream_t q) {
        ks_top<<<1, 1, 0, q>>>(K);
        kd_pupd<<<g, 256, 0, q>>>(n, K, r, v, pp);
        k3_op_dot<<<g, 256, 0, q>>>(o, pp, v, K, rhat, 0, part);
        k3_final<<<1, 256, 0, q>>>(part, nblk, K, FIN_ALPHA);
        kd_s_dot<<<g, 256, 0, q>>>(n, K, r, v, sv, part);
        k3_final<<<1, 256, 0, q>>>(part, nblk, K, FIN_S);
        kd_axpy_add<<<g, 256, 0, q>>>(n, K, pp, x);
        ks_added<<<1, 1, 0, q>>>(K);
        k3_op_dot<<<g, 256, 0, q>>>(o, sv, t, K, sv, 1, part);
        k3_final<<<1, 256, 0, q>>>(part, nblk, K, FIN_OMEGA);
        kd_axpy_add<<<g, 256, 0, q>>>(n, K, pp, x);
        ks_added<<<1, 1, 0, q>>>(K);
        kd_xr_dot<<<g, 256, 0, q>>>(n, K, pp, sv, t, rhat, x, r, part);
        k3_final<<<1, 256, 0, q>>>(part, nblk, K, FIN_END);
    };
    cudaGraphExec_t exec = nullptr;
    for (const auto& gr : b->graphs)
        if (gr.kind == o.kind && gr.x == x) exec = gr.exec;
    if (!exec) {
        if (!b->cap) V3_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        V3_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        iteration(b->cap);
        cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        V3_CUDA(ce);
        b->graphs.push_back({o.kind, x, exec});
    }
    double d[2];
    V3_TRY(dots(b, n, rhs, rhs, nullptr, nullptr, d));
    const double bnorm = std::sqrt(d[0]);
    *iters = 0;
    *relres = 0.0;
    if (!std::isfinite(bnorm)) return fail(b, VIP_ERR_NONFINITE, "non-finite right-hand side");
    if (bnorm == 0.0) {
        V3_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        return VIP_OK;
    }
    const double tol = b->rtol * bnorm;
    // inner iterations launched between host reads: 1, 2, 4, ... 16, so that a solve
    // of a few iterations (the Helmholtz ones) launches few that do nothing
    constexpr int CHUNK_MAX = 16;
    int32_t it = 0, restarts = 0;
    while (it < b->max_iters) {
        apply(x, y);
        k3_lin2<<<g, 256, 0, st>>>(n, 1.0, rhs, -1.0, y, r);
        V3_TRY(dots(b, n, r, r, nullptr, nullptr, d));
        if (!std::isfinite(d[0])) return fail(b, VIP_ERR_NONFINITE, "non-finite residual");
        if (std::sqrt(d[0]) <= tol) break;
        if (++restarts > 1000) return fail(b, VIP_ERR_BREAKDOWN, "BiCGSTAB: no progress after 1000 restarts");
        V3_CUDA(cudaMemcpyAsync(rhat, r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KS h{};
        h.rho_old = h.alpha = h.omega = 1.0;
        h.rhat_norm = std::sqrt(d[0]);
        h.tol = tol;
        h.brk = 1e-12;
        h.it = it;
        h.max_it = b->max_iters;
        h.state = KS_RUN;
        h.d[0] = h.d[1] = d[0];       // r_hat . r and r . r, with r_hat = r
        V3_CUDA(cudaMemcpyAsync(K, &h, sizeof(KS), cudaMemcpyHostToDevice, st));
        V3_CUDA(cudaMemsetAsync(v, 0, n * sizeof(double), st));
        V3_CUDA(cudaMemsetAsync(pp, 0, n * sizeof(double), st));
        for (int chunk = 1;; chunk = std::min(2 * chunk, CHUNK_MAX)) {
            for (int c = 0; c < chunk; ++c) V3_CUDA(cudaGraphLaunch(exec, st));
            V3_CUDA(cudaGetLastError());
            V3_CUDA(cudaMemcpyAsync(&h, K, sizeof(KS), cudaMemcpyDeviceToHost, st));
            V3_CUDA(cudaStreamSynchronize(st));
            it = h.it;
            if (!std::isfinite(h.d[0])) return fail(b, VIP_ERR_NONFINITE, "non-finite residual");
            if (h.state != KS_RUN) break;
        }
    }
    apply(x, y);
    k3_lin2<<<g, 256, 0, st>>>(n, 1.0, rhs, -1.0, y, r);
    V3_TRY(dots(b, n, r, r, nullptr, nullptr, d));
    *iters = it;
    *relres = std::sqrt(d[0]) / bnorm;
    if (!std::isfinite(*relres)) return fail(b, VIP_ERR_NONFINITE, "non-finite solution");
    if (*relres > b->rtol) return fail(b, VIP_ERR_NOT_CONVERGED, "BiCGSTAB hit its iteration limit");
    return VIP_OK;
}

// One fractional step (Eqs. 12-15) on a built node set of interior and wall nodes.
vip_status step_once(vip_3d* b) {
    const int64_t N = b->N;
    const unsigned g = blocks_for(N, 128);
    cudaStream_t st = b->stream;
    const double alpha = b->dt / (2.0 * b->Re), dt = b->dt;
    const Tab3 L = tab3(b, VIP3_OP_LAPLACE);
    const Tab3 Nb = b->Nb ? tab3(b, VIP3_OP_NEUMANN) : Tab3{nullptr, nullptr, nullptr};
    const Tab3 G[3] = {tab3(b, VIP3_OP_GX), tab3(b, VIP3_OP_GY), tab3(b, VIP3_OP_GZ)};
    k3_conv<<<g, 128, 0, st>>>(asm_view(b), b->vel[0], b->vel[1], b->vel[2], b->Ncur[0], b->Ncur[1],
                               b->Ncur[2]);
    V3_CUDA(cudaGetLastError());
    if (!b->have_prev)
        for (int c = 0; c < 3; ++c)
            V3_CUDA(cudaMemcpyAsync(b->Nprev[c], b->Ncur[c], N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double* rhs = b->kv[7];
    int32_t helm = 0;
    for (int c = 0; c < 3; ++c) {
        k3_rhs<<<g, 128, 0, st>>>(N, L, G[c], alpha, dt, b->ipos, b->bc[c], b->vel[c], b->Ncur[c],
                                  b->Nprev[c], b->p, rhs);
        V3_CUDA(cudaGetLastError());
        V3_CUDA(cudaMemcpyAsync(b->star[c], b->vel[c], N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        const Op3 oh{OPK_HELM, N, N, b->k0, alpha, L, Nb, b->ipos, b->h};
        int32_t it = 0;
        double res = 0.0;
        V3_TRY(krylov(b, oh, rhs, b->star[c], &it, &res));
        helm += it;
    }
    for (int c = 0; c < 3; ++c) std::swap(b->Ncur[c], b->Nprev[c]);
    b->have_prev = true;
    k3_div<<<g, 128, 0, st>>>(N, G[0], G[1], G[2], dt, b->k0, b->ipos, b->star[0], b->star[1], b->star[2],
                              rhs);
    V3_CUDA(cudaGetLastError());
    const Op3 op{OPK_POIS, N + 1, N, b->k0, alpha, L, Nb, b->ipos, b->h};
    int32_t itp = 0;
    double resp = 0.0;
    V3_TRY(krylov(b, op, rhs, b->phi, &itp, &resp));
    k3_project<<<g, 128, 0, st>>>(N, L, G[0], G[1], G[2], alpha, dt, b->ipos, b->phi, b->star[0],
                                  b->star[1], b->star[2], b->vel[0], b->vel[1], b->vel[2], b->p);
    V3_CUDA(cudaGetLastError());
    V3_CUDA(cudaStreamSynchronize(st));
    b->last_helm = helm;
    b->last_poisson = itp;
    b->last_poisson_res = resp;
    ++b->steps;
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
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    free_all(b->build_bufs);
    free_all(b->node_bufs);
    free_all(b->state_bufs);
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
    free_all(b->state_bufs);
    for (int c = 0; c < 3; ++c) b->vel[c] = b->star[c] = b->Ncur[c] = b->Nprev[c] = b->bc[c] = nullptr;
    for (double*& q : b->kv) q = nullptr;
    b->p = b->phi = b->dpart = b->dres = nullptr;
    b->ks = nullptr;
    b->state = b->have_prev = false;
    b->steps = 0;
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
    b->h0 = hh[0];
    b->k0 = interior.empty() ? -1 : interior[0];
    b->other_kinds = false;
    for (int64_t i = 0; i < n; ++i)
        if (hk[i] == VIP_NODE_SLIP || hk[i] == VIP_NODE_OUTLET) b->other_kinds = true;
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

vip_status vip_3d_set_flow(vip_3d* b, double Re, double dt, double rtol, int32_t max_iters) {
    if (!b) return VIP_ERR_ARG;
    if (!(Re > 0.0) || !(dt > 0.0) || !std::isfinite(Re) || !std::isfinite(dt))
        return fail(b, VIP_ERR_ARG, "Re and dt must be finite and > 0");
    if (!(rtol > 0.0 && rtol < 1.0)) return fail(b, VIP_ERR_ARG, "rtol must lie in (0, 1)");
    if (max_iters < 1) return fail(b, VIP_ERR_ARG, "max_iters must be >= 1");
    drop_graphs(b);
    b->Re = Re;
    b->dt = dt;
    b->rtol = rtol;
    b->max_iters = max_iters;
    b->flow = true;
    return VIP_OK;
}

vip_status vip_3d_set_state(vip_3d* b, const double* u, const double* v, const double* w, const double* p) {
    if (!b) return VIP_ERR_ARG;
    if (b->N < 1) return fail(b, VIP_ERR_ARG, "no node set");
    if (!u || !v || !w || !p) return fail(b, VIP_ERR_ARG, "null array");
    DeviceScope ds(b->device);
    const int64_t N = b->N;
    if (!b->p) {
        for (int c = 0; c < 3; ++c) {
            V3_CUDA(alloc(b->state_bufs, &b->vel[c], N));
            V3_CUDA(alloc(b->state_bufs, &b->star[c], N));
            V3_CUDA(alloc(b->state_bufs, &b->Ncur[c], N));
            V3_CUDA(alloc(b->state_bufs, &b->Nprev[c], N));
            V3_CUDA(alloc(b->state_bufs, &b->bc[c], N));
        }
        V3_CUDA(alloc(b->state_bufs, &b->p, N));
        V3_CUDA(alloc(b->state_bufs, &b->phi, N + 1));
        for (int k = 0; k < 8; ++k) V3_CUDA(alloc(b->state_bufs, &b->kv[k], N + 1));
        V3_CUDA(alloc(b->state_bufs, &b->dpart, 2 * std::max<int64_t>(DOT_B, (N + 1 + 255) / 256)));
        V3_CUDA(alloc(b->state_bufs, &b->dres, 2));
        KS* ksp = nullptr;
        V3_CUDA(alloc(b->state_bufs, &ksp, 1));
        b->ks = ksp;
    }
    const double* src[4] = {u, v, w, p};
    double* dst[4] = {b->vel[0], b->vel[1], b->vel[2], b->p};
    for (int k = 0; k < 4; ++k)
        V3_CUDA(cudaMemcpyAsync(dst[k], src[k], N * sizeof(double), cudaMemcpyDefault, b->stream));
    for (int c = 0; c < 3; ++c)
        V3_CUDA(cudaMemcpyAsync(b->bc[c], b->vel[c], N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    V3_CUDA(cudaMemsetAsync(b->phi, 0, (N + 1) * sizeof(double), b->stream));
    V3_CUDA(cudaStreamSynchronize(b->stream));
    b->have_prev = false;
    b->state = true;
    b->steps = 0;
    return VIP_OK;
}

vip_status vip_3d_step(vip_3d* b, int32_t nsteps) {
    if (!b) return VIP_ERR_ARG;
    if (!b->built) return fail(b, VIP_ERR_ARG, "not built");
    if (!b->flow || !b->state) return fail(b, VIP_ERR_ARG, "vip_3d_set_flow and vip_3d_set_state first");
    if (b->other_kinds) return fail(b, VIP_ERR_ARG, "the 3D step takes interior and wall nodes only");
    if (b->k0 < 0) return fail(b, VIP_ERR_ARG, "the 3D step needs an interior node");
    if (nsteps < 0) return fail(b, VIP_ERR_ARG, "nsteps must be >= 0");
    DeviceScope ds(b->device);
    const int need[5] = {VIP3_OP_LAPLACE, VIP3_OP_GX, VIP3_OP_GY, VIP3_OP_GZ, VIP3_OP_NEUMANN};
    for (int op : need) V3_TRY(assemble(b, op));
    for (int k = 0; k < nsteps; ++k) V3_TRY(step_once(b));
    return VIP_OK;
}

vip_status vip_3d_get_state(vip_3d* b, double* u, double* v, double* w, double* p, double* phi) {
    if (!b) return VIP_ERR_ARG;
    if (!b->state) return fail(b, VIP_ERR_ARG, "no state");
    DeviceScope ds(b->device);
    const int64_t N = b->N;
    double* dst[5] = {u, v, w, p, phi};
    const double* src[5] = {b->vel[0], b->vel[1], b->vel[2], b->p, b->phi};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) V3_CUDA(cudaMemcpyAsync(dst[k], src[k], N * sizeof(double), cudaMemcpyDefault, b->stream));
    V3_CUDA(cudaStreamSynchronize(b->stream));
    return VIP_OK;
}

vip_status vip_3d_get_iters(vip_3d* b, int64_t* steps, int32_t* helm_iters, int32_t* poisson_iters,
                            double* poisson_relres) {
    if (!b) return VIP_ERR_ARG;
    if (steps) *steps = b->steps;
    if (helm_iters) *helm_iters = b->last_helm;
    if (poisson_iters) *poisson_iters = b->last_poisson;
    if (poisson_relres) *poisson_relres = b->last_poisson_res;
    return VIP_OK;
}

}  // extern "C"
