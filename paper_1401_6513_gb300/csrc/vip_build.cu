// Setup stage of the VIP solver on the GPU: neighbour search, MLS weights and the
// merged stencil operators (Sec. 3, Sec. 4 of Park, Jo and Choe).
//
// Points: every padded row r owns seven point slots p = type * R + r:
//   node (the node itself), the four VIPs x_i +- (h/2) e_x, x_i +- (h/2) e_y of an
//   interior node (Sec. 4.1), and two auxiliary points x_i - h n, x_i - 2 h n on
//   the inward normal of a boundary node (zero-normal-derivative rows).
// Inactive slots have no neighbours.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "vip_internal.cuh"

namespace vip {

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------
template <class TI>
__global__ void k_scan_block(const TI* __restrict__ in, int64_t* __restrict__ out,
                             int64_t* __restrict__ bsum, int64_t n) {
    __shared__ int64_t warp_tot[32];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t v = (i < n) ? (int64_t)in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t base = (w > 0) ? warp_tot[w - 1] : 0;
    if (i < n) out[i] = base + x - v;  // exclusive
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = base + x;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ boff, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

// Exclusive scan of n counts into out[0..n]; out[n] = total.
template <class TI>
static cudaError_t scan_excl(const TI* in, int64_t* out, int64_t n, cudaStream_t s) {
    const int B = 1024;
    int64_t nb = (n + B - 1) / B;
    if (n == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    }
    int64_t* bsum = nullptr;
    int64_t* boff = nullptr;
    cudaError_t e = cudaMalloc(&bsum, nb * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&boff, (nb + 1) * sizeof(int64_t));
    if (e != cudaSuccess) { cudaFree(bsum); return e; }
    k_scan_block<TI><<<(unsigned)nb, B, 0, s>>>(in, out, bsum, n);
    if (nb > 1) {
        e = scan_excl<int64_t>(bsum, boff, nb, s);
        if (e == cudaSuccess) k_scan_add<<<(unsigned)nb, B, 0, s>>>(out, boff, n);
        // total = last exclusive + last count
        e = (e == cudaSuccess) ? cudaMemcpyAsync(out + n, boff + nb, sizeof(int64_t),
                                                 cudaMemcpyDeviceToDevice, s) : e;
    } else {
        e = cudaMemcpyAsync(out + n, bsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    }
    cudaStreamSynchronize(s);
    cudaFree(bsum);
    cudaFree(boff);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

// ---------------------------------------------------------------------------
// points
// ---------------------------------------------------------------------------
struct BuildArgs {
    int64_t R;
    const double *x, *y, *nx, *ny, *h;
    const uint8_t* kind;
    const int8_t* row_type;
    const int32_t* row_geom;
    const GeomDev* g;
    double support;
    int weight;
    // cell lists (per geometry)
    const int64_t* cell_base;   // [G]
    const int32_t* ncx;         // [G]
    const int32_t* ncy;         // [G]
    const double* cx0;          // [G] origin
    const double* cy0;
    const double* csx;          // [G] cell size
    const double* csy;
    const int64_t* cell_ptr;    // [C+1]
    const int32_t* cell_rows;   // [N]
    // normal-point step of every row (VIP_PROBES_INSIDE), or null: h_local
    const double* pstep;
};

// Coordinates and support radius of point p; returns false for an inactive slot.
// Coordinates use explicitly rounded operations so that they are the same
// numbers as a plain IEEE evaluation of the same formulas.
__device__ __forceinline__ bool point_of(const BuildArgs& a, int64_t p, double& qx, double& qy,
                                         double& rho, int& row) {
    int t = (int)(p / a.R);
    int64_t r = p - (int64_t)t * a.R;
    row = (int)r;
    if (a.row_type[r] != ROW_NODE) return false;
    uint8_t k = a.kind[r];
    double x = a.x[r], y = a.y[r], h = a.h[r];
    rho = __dmul_rn(a.support, h);
    double hh = __dmul_rn(0.5, h);
    switch (t) {
        case PT_NODE: qx = x; qy = y; return true;
        case PT_E: qx = __dadd_rn(x, hh); qy = y; return k == VIP_NODE_INTERIOR;
        case PT_W: qx = __dsub_rn(x, hh); qy = y; return k == VIP_NODE_INTERIOR;
        case PT_N: qx = x; qy = __dadd_rn(y, hh); return k == VIP_NODE_INTERIOR;
        case PT_S: qx = x; qy = __dsub_rn(y, hh); return k == VIP_NODE_INTERIOR;
        case PT_B1: {
            double sb = a.pstep ? a.pstep[r] : h;
            qx = __dsub_rn(x, __dmul_rn(sb, a.nx[r]));
            qy = __dsub_rn(y, __dmul_rn(sb, a.ny[r]));
            return k != VIP_NODE_INTERIOR;
        }
        case PT_B2: {
            double h2 = __dmul_rn(2.0, a.pstep ? a.pstep[r] : h);
            qx = __dsub_rn(x, __dmul_rn(h2, a.nx[r]));
            qy = __dsub_rn(y, __dmul_rn(h2, a.ny[r]));
            return k != VIP_NODE_INTERIOR;
        }
    }
    return false;
}

// Periodic minimum image with one correction by +-L (L = 0: not periodic).
__device__ __forceinline__ double min_image(double d, double L) {
    if (L > 0.0) {
        double hL = __dmul_rn(0.5, L);
        if (d > hL) d = __dsub_rn(d, L);
        else if (d < -hL) d = __dadd_rn(d, L);
    }
    return d;
}

__device__ __forceinline__ int cell_coord(double q, double c0, double cs, int nc, bool periodic) {
    double f = floor((q - c0) / cs);
    int c;
    if (periodic) {
        long long cc = (long long)f;
        cc %= nc;
        if (cc < 0) cc += nc;
        c = (int)cc;
    } else {
        c = (int)fmin(fmax(f, 0.0), (double)(nc - 1));
    }
    return c;
}

// Visit every node within the support of point (qx, qy).
template <class F>
__device__ __forceinline__ void for_each_neighbour(const BuildArgs& a, int gi, double qx, double qy,
                                                   double rho, F&& f) {
    const GeomDev& G = a.g[gi];
    bool px = G.Lx > 0.0, py = G.Ly > 0.0;
    int nx = a.ncx[gi], ny = a.ncy[gi];
    int cx = cell_coord(qx, a.cx0[gi], a.csx[gi], nx, px);
    int cy = cell_coord(qy, a.cy0[gi], a.csy[gi], ny, py);
    double rho2 = __dmul_rn(rho, rho);
    int rx = (nx >= 3 || !px) ? 1 : 0;
    int ry = (ny >= 3 || !py) ? 1 : 0;
    for (int dy = -ry; dy <= ry; ++dy) {
        int yy = cy + dy;
        if (py) { yy %= ny; if (yy < 0) yy += ny; }
        else if (yy < 0 || yy >= ny) continue;
        for (int dx = -rx; dx <= rx; ++dx) {
            int xx = cx + dx;
            if (px) { xx %= nx; if (xx < 0) xx += nx; }
            else if (xx < 0 || xx >= nx) continue;
            int64_t cell = a.cell_base[gi] + (int64_t)yy * nx + xx;
            for (int64_t q = a.cell_ptr[cell]; q < a.cell_ptr[cell + 1]; ++q) {
                int j = a.cell_rows[q];
                double ddx = min_image(__dsub_rn(a.x[j], qx), G.Lx);
                double ddy = min_image(__dsub_rn(a.y[j], qy), G.Ly);
                double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                if (d2 < rho2) f(j, ddx, ddy);
            }
        }
    }
}

// Normal-point step of every row (VIP_PROBES_INSIDE placement): a boundary node of
// an INSIDE geometry starts from h_local and shrinks its step by 0.7, at most 12
// times, while its second normal point x_b2 = x_i - 2 s n_i lies less than 5 % of
// h_j inside the tangent at the boundary node j nearest to x_b2.  The nearest
// node is searched within the support radius of node i, which contains x_b2 (at
// 2 s <= 2 h_local < rho for a support ratio above 2) and hence node i itself.
// Other rows keep h_local.  Explicitly rounded operations, as in point_of.
__global__ void k_probe_steps(BuildArgs a, double* __restrict__ pstep) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    double h = a.h[r];
    double s = h;
    if (a.row_type[r] == ROW_NODE && a.kind[r] != VIP_NODE_INTERIOR) {
        int gi = a.row_geom[r];
        if (a.g[gi].probes == VIP_PROBES_INSIDE) {
            double x = a.x[r], y = a.y[r], nx = a.nx[r], ny = a.ny[r];
            double rho = __dmul_rn(a.support, h);
            for (int it = 0; it < 12; ++it) {
                double s2 = __dmul_rn(2.0, s);
                double qx = __dsub_rn(x, __dmul_rn(s2, nx));
                double qy = __dsub_rn(y, __dmul_rn(s2, ny));
                int best = -1;
                double bx = 0.0, by = 0.0, bd2 = 0.0;
                for_each_neighbour(a, gi, qx, qy, rho, [&](int j, double ddx, double ddy) {
                    if (a.kind[j] == VIP_NODE_INTERIOR) return;
                    double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                    if (best < 0 || d2 < bd2) { best = j; bd2 = d2; bx = ddx; by = ddy; }
                });
                if (best < 0) break;
                // (x_b2 - x_j) . n_j, with x_j - x_b2 = (bx, by) in the minimum image
                double side = __dadd_rn(__dmul_rn(-bx, a.nx[best]), __dmul_rn(-by, a.ny[best]));
                if (!(side > __dmul_rn(-0.05, a.h[best]))) break;
                s = __dmul_rn(0.7, s);
            }
        }
    }
    pstep[r] = s;
}

__global__ void k_cell_count(BuildArgs a, int32_t* __restrict__ cell_cnt, int32_t* __restrict__ node_cell) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    if (a.row_type[r] != ROW_NODE) { node_cell[r] = -1; return; }
    int gi = a.row_geom[r];
    const GeomDev& G = a.g[gi];
    int nx = a.ncx[gi], ny = a.ncy[gi];
    int cx = cell_coord(a.x[r], a.cx0[gi], a.csx[gi], nx, G.Lx > 0.0);
    int cy = cell_coord(a.y[r], a.cy0[gi], a.csy[gi], ny, G.Ly > 0.0);
    int64_t cell = a.cell_base[gi] + (int64_t)cy * nx + cx;
    node_cell[r] = (int32_t)cell;
    atomicAdd(&cell_cnt[cell], 1);
}

__global__ void k_cell_fill(int64_t R, const int32_t* __restrict__ node_cell,
                            const int64_t* __restrict__ cell_ptr, int32_t* __restrict__ cursor,
                            int32_t* __restrict__ cell_rows) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int c = node_cell[r];
    if (c < 0) return;
    int pos = atomicAdd(&cursor[c], 1);
    cell_rows[cell_ptr[c] + pos] = (int32_t)r;
}

__global__ void k_nbr_count(BuildArgs a, int64_t npts, int32_t* __restrict__ cnt, int32_t* status,
                            int32_t* bad_point) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    double qx, qy, rho;
    int row;
    int n = 0;
    if (point_of(a, p, qx, qy, rho, row)) {
        for_each_neighbour(a, a.row_geom[row], qx, qy, rho, [&](int, double, double) { ++n; });
        if (n > KMAX) {
            set_status(status, VIP_ERR_ARG);
            atomicMin(bad_point, (int32_t)(p < 0x7fffffffLL ? p : 0x7fffffffLL));
            n = 0;
        }
    }
    cnt[p] = n;
}

__global__ void k_nbr_fill(BuildArgs a, int64_t npts, const int64_t* __restrict__ pptr,
                           int32_t* __restrict__ pidx) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    double qx, qy, rho;
    int row;
    int64_t b = pptr[p];
    int64_t e = pptr[p + 1];
    if (e == b || !point_of(a, p, qx, qy, rho, row)) return;
    int64_t w = b;
    for_each_neighbour(a, a.row_geom[row], qx, qy, rho, [&](int j, double, double) {
        if (w < e) pidx[w++] = j;
    });
    // ascending node order (insertion sort; lists are short)
    for (int64_t i = b + 1; i < e; ++i) {
        int32_t v = pidx[i];
        int64_t k = i - 1;
        while (k >= b && pidx[k] > v) { pidx[k + 1] = pidx[k]; --k; }
        pidx[k + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// MLS weights (Sec. 3, Eq. fmlsrk:2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double weight_fn(double r, int kind) {
    if (kind == VIP_W_PAPER) {
        if (r >= 1.0) return 0.0;
        double e = (1.0 - r) * (1.0 - r);
        double t = 1.0 - pow(r, e);
        double t2 = t * t;
        return t2 * t2;
    }
    if (r <= 0.5) return 2.0 / 3.0 - 4.0 * r * r + 4.0 * r * r * r;
    if (r < 1.0) return 4.0 / 3.0 - 4.0 * r + 4.0 * r * r - (4.0 / 3.0) * r * r * r;
    return 0.0;
}

// Packed lower triangle index of (i, j), i >= j.
__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void __launch_bounds__(128) k_mls(BuildArgs a, int64_t npts, const int64_t* __restrict__ pptr,
                                             const int32_t* __restrict__ pidx, double* __restrict__ w00,
                                             double* __restrict__ wd, int64_t nnz_nodes,
                                             int32_t* status, int32_t* bad_point) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    int64_t b = pptr[p], e = pptr[p + 1];
    if (e == b) return;
    double qx, qy, rho;
    int row;
    point_of(a, p, qx, qy, rho, row);
    const GeomDev& G = a.g[a.row_geom[row]];
    const bool node = p < a.R;
    const double irho = 1.0 / rho;
    // moment matrix M = sum_i Phi_i p_i p_i^T (packed lower triangle)
    double M[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) M[i] = 0.0;
    for (int64_t q = b; q < e; ++q) {
        int j = pidx[q];
        double xi = min_image(a.x[j] - qx, G.Lx) * irho;
        double eta = min_image(a.y[j] - qy, G.Ly) * irho;
        double W = weight_fn(sqrt(xi * xi + eta * eta), a.weight);
        double pv[6] = {1.0, xi, eta, xi * xi, xi * eta, eta * eta};
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double wi = W * pv[i];
#pragma unroll
            for (int k = 0; k <= i; ++k) M[tri(i, k)] = fma(wi, pv[k], M[tri(i, k)]);
        }
    }
    // Cholesky M = L L^T in place; a pivot below 1e-12 trace(M) marks the stencil singular
    double trace = M[tri(0, 0)] + M[tri(1, 1)] + M[tri(2, 2)] + M[tri(3, 3)] + M[tri(4, 4)] + M[tri(5, 5)];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double d = M[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= M[tri(j, k)] * M[tri(j, k)];
        if (!(d > 1e-12 * trace)) { ok = false; d = 1.0; }
        double lj = sqrt(d);
        M[tri(j, j)] = lj;
        double il = 1.0 / lj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            double s = M[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= M[tri(i, k)] * M[tri(j, k)];
            M[tri(i, j)] = s * il;
        }
    }
    if (!ok) {
        set_status(status, VIP_ERR_SINGULAR_STENCIL);
        atomicMin(bad_point, (int32_t)(p < 0x7fffffffLL ? p : 0x7fffffffLL));
        return;
    }
    // q_k = L^{-1} e_k (lower triangular, nonzero from index k on).
    // Psi_k(j) = fac_k * Phi_j * (q_k . y_j) with y_j = L^{-1} p_j, because
    // e_k^T M^{-1} p_j = (L^{-1} e_k)^T (L^{-1} p_j).
    double Q[21];  // Q[tri(i,k)] = (q_k)_i for i >= k
    const int nk = node ? 6 : 1;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k >= nk) break;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i < k) continue;
            double s = (i == k) ? 1.0 : 0.0;
#pragma unroll
            for (int m = 0; m < i; ++m)
                if (m >= k) s -= M[tri(i, m)] * Q[tri(m, k)];
            Q[tri(i, k)] = s / M[tri(i, i)];
        }
    }
    // a! b! rho^-(a+b) for k = [0,0],[1,0],[0,1],[2,0],[1,1],[0,2]
    const double fac[6] = {1.0, irho, irho, 2.0 * irho * irho, irho * irho, 2.0 * irho * irho};
    for (int64_t q = b; q < e; ++q) {
        int j = pidx[q];
        double xi = min_image(a.x[j] - qx, G.Lx) * irho;
        double eta = min_image(a.y[j] - qy, G.Ly) * irho;
        double W = weight_fn(sqrt(xi * xi + eta * eta), a.weight);
        double pv[6] = {1.0, xi, eta, xi * xi, xi * eta, eta * eta};
        double yv[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double s = pv[i];
#pragma unroll
            for (int m = 0; m < i; ++m) s -= M[tri(i, m)] * yv[m];
            yv[i] = s / M[tri(i, i)];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (k >= nk) break;
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (i >= k) s += Q[tri(i, k)] * yv[i];
            double psi = fac[k] * W * s;
            if (k == 0) w00[q] = psi;
            else wd[(int64_t)(k - 1) * nnz_nodes + q] = psi;
        }
    }
}

// 1/|x_e - x_w| and 1/|x_n - x_s| of interior nodes.
__global__ void k_vip_inv(BuildArgs a, double* __restrict__ inv_ew, double* __restrict__ inv_ns) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    double ie = 0.0, in_ = 0.0;
    if (a.row_type[r] == ROW_NODE && a.kind[r] == VIP_NODE_INTERIOR) {
        double hh = __dmul_rn(0.5, a.h[r]);
        double xe = __dadd_rn(a.x[r], hh), xw = __dsub_rn(a.x[r], hh);
        double yn = __dadd_rn(a.y[r], hh), ys = __dsub_rn(a.y[r], hh);
        ie = 1.0 / fabs(__dsub_rn(xe, xw));
        in_ = 1.0 / fabs(__dsub_rn(yn, ys));
    }
    inv_ew[r] = ie;
    inv_ns[r] = in_;
}

// ---------------------------------------------------------------------------
// operator assembly into SELL-32 tables
// ---------------------------------------------------------------------------
enum TableId { TB_LAP, TB_D00, TB_VE, TB_VW, TB_VN, TB_VS, TB_GX, TB_GY, TB_HELM, TB_POIS };

struct Src {            // one sorted source list with a coefficient
    const int32_t* idx;
    const double* val;  // nullptr: value 1 (diagonal singleton uses idx == nullptr)
    const double* val2; // optional second value array summed with val (D20 + D02)
    int len;
    double coef;
};

struct AsmArgs {
    BuildArgs b;
    const int64_t* pptr;
    const int32_t* pidx;
    const double* w00;
    const double* wd;
    int64_t nnz_nodes;
    const double* inv_ew;
    const double* inv_ns;
    const int32_t* first_row;
    int identity;
};

__device__ __forceinline__ Src point_src(const AsmArgs& A, int type, int64_t r, double coef) {
    int64_t p = (int64_t)type * A.b.R + r;
    int64_t s = A.pptr[p];
    Src o;
    o.idx = A.pidx + s;
    o.val = A.w00 + s;
    o.val2 = nullptr;
    o.len = (int)(A.pptr[p + 1] - s);
    o.coef = coef;
    return o;
}

// Merge up to four ascending lists (plus an optional diagonal entry) into one
// ascending row, summing coefficients of equal columns.  emit(col, value).
template <class F>
__device__ __forceinline__ int merge_rows(const Src* L, int nl, bool diag, double dcoef, int32_t drow,
                                          int32_t col_off, F&& emit) {
    int pos[4] = {0, 0, 0, 0};
    bool dd = diag;
    int n = 0;
    while (true) {
        int32_t m = 0x7fffffff;
        for (int i = 0; i < nl; ++i)
            if (pos[i] < L[i].len) m = min(m, L[i].idx[pos[i]]);
        if (dd) m = min(m, drow);
        if (m == 0x7fffffff) break;
        double v = 0.0;
        for (int i = 0; i < nl; ++i) {
            if (pos[i] < L[i].len && L[i].idx[pos[i]] == m) {
                double w = L[i].val[pos[i]];
                if (L[i].val2) w += L[i].val2[pos[i]];
                v += L[i].coef * w;
                ++pos[i];
            }
        }
        if (dd && drow == m) { v += dcoef; dd = false; }
        emit(m + col_off, v);
        ++n;
    }
    return n;
}

// Produce row r of table tb; with emit == counting lambda in count mode.
template <class F>
__device__ int table_row(const AsmArgs& A, int tb, int64_t r, F&& emit) {
    const BuildArgs& B = A.b;
    const int64_t R = B.R;
    int64_t rr = r;
    int comp = 0;
    if (tb == TB_HELM && r >= R) { rr = r - R; comp = 1; }
    int rt = B.row_type[rr];
    if (rt == ROW_PAD) {
        if (tb == TB_HELM || tb == TB_POIS) { emit((int32_t)r, 1.0); return 1; }
        return 0;
    }
    const GeomDev& G = B.g[B.row_geom[rr]];
    if (rt == ROW_BORDER) {
        if (tb == TB_POIS) {
            // equation of the reference node k plus the mu column (this row)
            int64_t k = G.pin;
            int64_t kp = A.pptr[k];
            Src lk = {A.pidx + kp, A.wd + 2 * A.nnz_nodes + kp, A.wd + 4 * A.nnz_nodes + kp,
                      (int)(A.pptr[k + 1] - kp), 1.0};
            int n = merge_rows(&lk, 1, false, 0, 0, 0, emit);
            emit((int32_t)rr, 1.0);
            return n + 1;
        }
        if (tb == TB_HELM) { emit((int32_t)r, 1.0); return 1; }
        return 0;
    }
    uint8_t k = B.kind[rr];
    bool interior = k == VIP_NODE_INTERIOR;
    int64_t np = A.pptr[rr];
    int nlen = (int)(A.pptr[rr + 1] - np);
    Src node_d00 = {A.pidx + np, A.w00 + np, nullptr, nlen, 1.0};
    Src node_lap = {A.pidx + np, A.wd + 2 * A.nnz_nodes + np, A.wd + 4 * A.nnz_nodes + np, nlen, 1.0};
    Src L[4];
    switch (tb) {
        case TB_LAP: L[0] = node_lap; return merge_rows(L, 1, false, 0, 0, 0, emit);
        case TB_D00: L[0] = node_d00; return merge_rows(L, 1, false, 0, 0, 0, emit);
        case TB_VE: case TB_VW: case TB_VN: case TB_VS:
            if (!interior) return 0;
            L[0] = point_src(A, PT_E + (tb - TB_VE), rr, 1.0);
            return merge_rows(L, 1, false, 0, 0, 0, emit);
        case TB_GX:
            if (!interior) return 0;
            L[0] = point_src(A, PT_E, rr, A.inv_ew[rr]);
            L[1] = point_src(A, PT_W, rr, -A.inv_ew[rr]);
            return merge_rows(L, 2, false, 0, 0, 0, emit);
        case TB_GY:
            if (!interior) return 0;
            L[0] = point_src(A, PT_N, rr, A.inv_ns[rr]);
            L[1] = point_src(A, PT_S, rr, -A.inv_ns[rr]);
            return merge_rows(L, 2, false, 0, 0, 0, emit);
        case TB_HELM: {
            int32_t off = comp ? (int32_t)R : 0;
            bool dir = (k == VIP_NODE_WALL) || (comp == 1 && k == VIP_NODE_SLIP);
            if (interior) {
                // (I - alpha L) or (D00 - alpha L), Eq. (12) times dt
                L[0] = node_lap;
                L[0].coef = -G.alpha;
                if (A.identity == VIP_IDENTITY_MLS) {
                    L[1] = node_d00;
                    return merge_rows(L, 2, false, 0, 0, off, emit);
                }
                return merge_rows(L, 1, true, 1.0, (int32_t)rr, off, emit);
            }
            if (dir) { emit((int32_t)(rr + off), 1.0); return 1; }
            // zero normal derivative: q_i - 4/3 q(x_b1) + 1/3 q(x_b2)
            L[0] = point_src(A, PT_B1, rr, -4.0 / 3.0);
            L[1] = point_src(A, PT_B2, rr, 1.0 / 3.0);
            return merge_rows(L, 2, true, 1.0, (int32_t)rr, off, emit);
        }
        case TB_POIS: {
            double sc = -4.0 / (B.h[rr] * B.h[rr]);
            if (interior) {
                if (G.bordered && rr == G.pin) { emit((int32_t)rr, sc); return 1; }  // phi_k = 0
                L[0] = node_lap;
                int n = merge_rows(L, 1, false, 0, 0, 0, emit);
                if (G.bordered) {  // column of mu: the geometry's border row
                    emit((int32_t)(G.row0 + G.n), 1.0);
                    ++n;
                }
                return n;
            }
            if (k == VIP_NODE_OUTLET) { emit((int32_t)rr, sc); return 1; }
            L[0] = point_src(A, PT_B1, rr, sc * (-4.0 / 3.0));
            L[1] = point_src(A, PT_B2, rr, sc * (1.0 / 3.0));
            return merge_rows(L, 2, true, sc, (int32_t)rr, 0, emit);
        }
    }
    return 0;
}

__global__ void k_table_count(AsmArgs A, int tb, int64_t nrows, int32_t* __restrict__ rowlen) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    rowlen[r] = table_row(A, tb, r, [](int32_t, double) {});
}

__global__ void k_slice_width(const int32_t* __restrict__ rowlen, int64_t nrows, int64_t nslices,
                              int32_t* __restrict__ width, int64_t* __restrict__ ssize) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int l = 0; l < SLICE; ++l) {
        int64_t r = s * SLICE + l;
        if (r < nrows) w = max(w, rowlen[r]);
    }
    width[s] = w;
    ssize[s] = (int64_t)w * SLICE;
}

__global__ void k_table_fill(AsmArgs A, int tb, int64_t nrows, const int64_t* __restrict__ sptr,
                             const int32_t* __restrict__ width, int32_t* __restrict__ col,
                             double* __restrict__ val) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int64_t s = r / SLICE;
    int lane = (int)(r % SLICE);
    int64_t base = sptr[s] + lane;
    int k = 0;
    int n = table_row(A, tb, r, [&](int32_t c, double v) {
        col[base + (int64_t)k * SLICE] = c;
        val[base + (int64_t)k * SLICE] = v;
        ++k;
    });
    for (int q = n; q < width[s]; ++q) {
        col[base + (int64_t)q * SLICE] = (int32_t)r;
        val[base + (int64_t)q * SLICE] = 0.0;
    }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// FP64 row sums of a SELL table (entries in stored order), rounded to FP32: the
// row sums of the FP32 differenced row form (see Sell::rs32).
__global__ void k_sell_rowsum(Sell A, float* __restrict__ rs) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.nrows) return;
    const int64_t base = A.sptr[r >> 5] + (r & 31);
    double s = 0.0;
    for (int k = 0; k < A.rowlen[r]; ++k) s += A.v64[base + (int64_t)k * SLICE];
    rs[r] = (float)s;
}

// Uniform slices of a SELL table (see Sell): one warp per slice decides whether all
// 32 rows hold the same stencil and writes its entry count (0 if not).
__global__ void k_sell_uniform(Sell A, int64_t* __restrict__ usize) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= A.nslices) return;  // whole warps
    const int w = A.width[s];
    const int64_t row = s * SLICE + lane;
    const int64_t base = A.sptr[s] + lane;
    const int64_t lim = (int64_t)1 << 29;  // column codes fit in int32
    bool ok = (s + 1) * SLICE <= A.nrows && w > 0;
    for (int k = 0; ok && k < w; ++k) {
        const int64_t e = base + (int64_t)k * SLICE;
        const long long v = __double_as_longlong(A.v64[e]);
        const int64_t col = A.col[e];
        const long long v0 = __shfl_sync(0xffffffffu, v, 0);
        const int64_t c0 = __shfl_sync(0xffffffffu, col, 0);
        const int64_t d = col - row, d0 = c0 - s * SLICE;
        const bool rel = __all_sync(0xffffffffu, d == d0 && d > -lim && d < lim);
        const bool ab = __all_sync(0xffffffffu, col == c0 && c0 < lim);
        ok = __all_sync(0xffffffffu, v == v0) && (rel || ab);
    }
    if (lane == 0) usize[s] = ok ? w : 0;
}

// Stencil of each uniform slice, taken from its first row.  Entry k's column is
// relative when rows 0 and 1 of the slice differ by one there, absolute when equal
// (exactly one holds in a uniform slice).
__global__ void k_sell_compact(Sell A, const int64_t* __restrict__ usize,
                               const int64_t* __restrict__ uoff) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= A.nslices) return;
    if (usize[s] == 0) {
        if (lane == 0) A.ucptr[s] = -1;
        return;
    }
    const int64_t o = uoff[s];
    const int w = A.width[s];
    for (int k = lane; k < w; k += 32) {
        const int64_t e = A.sptr[s] + (int64_t)k * SLICE;
        const int64_t c0 = A.col[e], c1 = A.col[e + 1];
        A.ucode[o + k] = c1 == c0 ? (int32_t)(2 * c0 + 1) : (int32_t)(2 * (c0 - s * SLICE));
        A.uv64[o + k] = A.v64[e];
        if (A.uv32) A.uv32[o + k] = A.v32[e];
    }
    if (lane == 0) A.ucptr[s] = o;
}

// Uniform slices that hold the same stencil (width, column codes and FP64 values
// all equal) share one stored copy: on a lattice most interior slices carry the
// same stencil, so the distinct stencils are few (the bumpy channel's Poisson
// operator: 1839 entries, 15 KB, instead of one 13-entry copy for each of its
// 63,936 uniform slices) and stay cache-resident.  The values and columns each row
// reads are unchanged, so results are bit-identical.  The shared copies are written
// over the front of the arrays.
static vip_status sell_share_stencils(vip_ctx* c, Sell& S, const std::vector<int32_t>& hw) {
    cudaStream_t st = c->stream;
    if (S.nuentries == 0) return VIP_OK;
    std::vector<int64_t> ucp(S.nslices);
    std::vector<int32_t> code(S.nuentries);
    std::vector<double> v64(S.nuentries);
    VIP_CUDA(cudaMemcpyAsync(ucp.data(), S.ucptr, S.nslices * 8, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(code.data(), S.ucode, S.nuentries * 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(v64.data(), S.uv64, S.nuentries * 8, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    std::unordered_map<std::string, int64_t> seen;
    std::vector<int32_t> ncode;
    std::vector<double> nv64;
    std::string key;
    for (int64_t s = 0; s < S.nslices; ++s) {
        if (ucp[s] < 0) continue;
        const int64_t o = ucp[s];
        const int w = hw[s];
        key.assign(reinterpret_cast<const char*>(&code[o]), (size_t)w * 4);
        key.append(reinterpret_cast<const char*>(&v64[o]), (size_t)w * 8);
        auto it = seen.find(key);
        if (it != seen.end()) {
            ucp[s] = it->second;
        } else {
            const int64_t no = (int64_t)ncode.size();
            ncode.insert(ncode.end(), code.begin() + o, code.begin() + o + w);
            nv64.insert(nv64.end(), v64.begin() + o, v64.begin() + o + w);
            seen.emplace(key, no);
            ucp[s] = no;
        }
    }
    const int64_t nu = (int64_t)ncode.size();
    std::vector<float> nv32(nu);
    for (int64_t k = 0; k < nu; ++k) nv32[k] = (float)nv64[k];
    VIP_CUDA(cudaMemcpyAsync(S.ucptr, ucp.data(), S.nslices * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(S.ucode, ncode.data(), nu * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(S.uv64, nv64.data(), nu * 8, cudaMemcpyHostToDevice, st));
    if (S.uv32) VIP_CUDA(cudaMemcpyAsync(S.uv32, nv32.data(), nu * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    S.nuentries = nu;
    return VIP_OK;
}

static vip_status sell_uniform(vip_ctx* c, Sell& S) {
    cudaStream_t st = c->stream;
    DeviceScratch s_usize, s_uoff;
    VIP_CUDA(cudaMalloc(&s_usize.p, S.nslices * sizeof(int64_t)));
    VIP_CUDA(cudaMalloc(&s_uoff.p, (S.nslices + 1) * sizeof(int64_t)));
    int64_t* usize = static_cast<int64_t*>(s_usize.p);
    int64_t* uoff = static_cast<int64_t*>(s_uoff.p);
    const int TB = 256;
    const unsigned grid = (unsigned)((S.nslices * 32 + TB - 1) / TB);
    k_sell_uniform<<<grid, TB, 0, st>>>(S, usize);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(scan_excl<int64_t>(usize, uoff, S.nslices, st));
    VIP_CUDA(cudaMemcpyAsync(&S.nuentries, uoff + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    std::vector<int64_t> hs(S.nslices);
    std::vector<int32_t> hw(S.nslices);
    VIP_CUDA(cudaMemcpyAsync(hs.data(), usize, S.nslices * 8, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(hw.data(), S.width, S.nslices * 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    S.nuniform = 0;
    S.nstored_other = 0;
    for (int64_t k = 0; k < S.nslices; ++k) {
        if (hs[k]) ++S.nuniform;
        else S.nstored_other += (int64_t)hw[k] * SLICE;
    }
    VIP_CUDA(dalloc(c, &S.ucptr, S.nslices));
    VIP_CUDA(dalloc(c, &S.ucode, S.nuentries));
    VIP_CUDA(dalloc(c, &S.uv64, S.nuentries));
    if (S.v32) VIP_CUDA(dalloc(c, &S.uv32, S.nuentries));
    k_sell_compact<<<grid, TB, 0, st>>>(S, usize, uoff);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(cudaStreamSynchronize(st));
    return sell_share_stencils(c, S, hw);
}

static vip_status build_table(vip_ctx* c, const AsmArgs& A, int tb, int64_t nrows, Sell& S,
                              bool f32) {
    cudaStream_t st = c->stream;
    S.nrows = nrows;
    S.nslices = (nrows + SLICE - 1) / SLICE;
    VIP_CUDA(dalloc(c, &S.rowlen, nrows));
    VIP_CUDA(dalloc(c, &S.width, S.nslices));
    VIP_CUDA(dalloc(c, &S.sptr, S.nslices + 1));
    int64_t* ssize = nullptr;
    VIP_CUDA(cudaMalloc(&ssize, S.nslices * sizeof(int64_t)));
    const int TB = 256;
    k_table_count<<<(unsigned)((nrows + TB - 1) / TB), TB, 0, st>>>(A, tb, nrows, S.rowlen);
    k_slice_width<<<(unsigned)((S.nslices + TB - 1) / TB), TB, 0, st>>>(S.rowlen, nrows, S.nslices,
                                                                        S.width, ssize);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(scan_excl<int64_t>(ssize, S.sptr, S.nslices, st));
    cudaFree(ssize);
    VIP_CUDA(cudaMemcpyAsync(&S.nstored, S.sptr + S.nslices, sizeof(int64_t),
                             cudaMemcpyDeviceToHost, st));
    int64_t* tot = nullptr;
    VIP_CUDA(cudaMalloc(&tot, (nrows + 1) * sizeof(int64_t)));
    VIP_CUDA(scan_excl<int32_t>(S.rowlen, tot, nrows, st));
    VIP_CUDA(cudaMemcpyAsync(&S.nnz, tot + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    cudaFree(tot);
    VIP_CUDA(dalloc(c, &S.col, S.nstored));
    VIP_CUDA(dalloc(c, &S.v64, S.nstored));
    k_table_fill<<<(unsigned)((nrows + TB - 1) / TB), TB, 0, st>>>(A, tb, nrows, S.sptr, S.width,
                                                                   S.col, S.v64);
    VIP_CUDA(cudaGetLastError());
    if (f32) {  // the Krylov operators: FP32 copy and uniform slices
        VIP_CUDA(dalloc(c, &S.v32, S.nstored));
        k_to_f32<<<(unsigned)((S.nstored + TB - 1) / TB), TB, 0, st>>>(S.v64, S.v32, S.nstored);
        VIP_CUDA(dalloc(c, &S.rs32, nrows));
        k_sell_rowsum<<<(unsigned)((nrows + TB - 1) / TB), TB, 0, st>>>(S, S.rs32);
        VIP_CUDA(cudaGetLastError());
        return sell_uniform(c, S);
    }
    return VIP_OK;
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------
vip_status build_all(vip_ctx* c) {
    cudaStream_t st = c->stream;
    const int64_t R = c->R;
    const int G = (int)c->geoms.size();
    // cell lists: one uniform grid per geometry with cells no smaller than the
    // largest support radius of its points
    std::vector<int64_t> cell_base(G);
    std::vector<int32_t> ncx(G), ncy(G);
    std::vector<double> cx0(G), cy0(G), csx(G), csy(G);
    int64_t C = 0;
    for (int g = 0; g < G; ++g) {
        const Geom& gg = c->geoms[g];
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, hmax = 0;
        for (int64_t i = gg.off; i < gg.off + gg.n; ++i) {
            xmin = std::min(xmin, c->hx[i]); xmax = std::max(xmax, c->hx[i]);
            ymin = std::min(ymin, c->hy[i]); ymax = std::max(ymax, c->hy[i]);
            hmax = std::max(hmax, c->hh[i]);
        }
        double cs = c->support * hmax * (1.0 + 1e-9);
        if (gg.Lx > 0) {
            ncx[g] = std::max(1, (int)std::floor(gg.Lx / cs));
            cx0[g] = 0.0;
            csx[g] = gg.Lx / ncx[g];
        } else {
            ncx[g] = std::max(1, (int)std::floor((xmax - xmin) / cs) + 1);
            cx0[g] = xmin;
            csx[g] = cs;
        }
        if (gg.Ly > 0) {
            ncy[g] = std::max(1, (int)std::floor(gg.Ly / cs));
            cy0[g] = 0.0;
            csy[g] = gg.Ly / ncy[g];
        } else {
            ncy[g] = std::max(1, (int)std::floor((ymax - ymin) / cs) + 1);
            cy0[g] = ymin;
            csy[g] = cs;
        }
        // periodic boxes with fewer than 3 cells are searched as one cell
        if (gg.Lx > 0 && ncx[g] < 3) { ncx[g] = 1; csx[g] = gg.Lx; }
        if (gg.Ly > 0 && ncy[g] < 3) { ncy[g] = 1; csy[g] = gg.Ly; }
        cell_base[g] = C;
        C += (int64_t)ncx[g] * ncy[g];
    }
    int64_t* d_cell_base; int32_t *d_ncx, *d_ncy; double *d_cx0, *d_cy0, *d_csx, *d_csy;
    VIP_CUDA(dalloc(c, &d_cell_base, G)); VIP_CUDA(dalloc(c, &d_ncx, G)); VIP_CUDA(dalloc(c, &d_ncy, G));
    VIP_CUDA(dalloc(c, &d_cx0, G)); VIP_CUDA(dalloc(c, &d_cy0, G));
    VIP_CUDA(dalloc(c, &d_csx, G)); VIP_CUDA(dalloc(c, &d_csy, G));
    VIP_CUDA(cudaMemcpyAsync(d_cell_base, cell_base.data(), G * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_ncx, ncx.data(), G * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_ncy, ncy.data(), G * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_cx0, cx0.data(), G * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_cy0, cy0.data(), G * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_csx, csx.data(), G * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(d_csy, csy.data(), G * 8, cudaMemcpyHostToDevice, st));

    BuildArgs a;
    a.R = R; a.x = c->x; a.y = c->y; a.nx = c->nx; a.ny = c->ny; a.h = c->h;
    a.kind = c->kind; a.row_type = c->row_type; a.row_geom = c->row_geom; a.g = c->gdev;
    a.support = c->support; a.weight = c->weight;
    a.cell_base = d_cell_base; a.ncx = d_ncx; a.ncy = d_ncy; a.cx0 = d_cx0; a.cy0 = d_cy0;
    a.csx = d_csx; a.csy = d_csy;
    a.pstep = nullptr;

    int32_t *cell_cnt = nullptr, *node_cell = nullptr, *cursor = nullptr;
    int64_t* cell_ptr = nullptr;
    int32_t* cell_rows = nullptr;
    VIP_CUDA(cudaMalloc(&cell_cnt, C * sizeof(int32_t)));
    VIP_CUDA(cudaMalloc(&cursor, C * sizeof(int32_t)));
    VIP_CUDA(cudaMalloc(&node_cell, R * sizeof(int32_t)));
    VIP_CUDA(dalloc(c, &cell_ptr, C + 1));
    VIP_CUDA(dalloc(c, &cell_rows, std::max<int64_t>(c->N, 1)));
    VIP_CUDA(cudaMemsetAsync(cell_cnt, 0, C * sizeof(int32_t), st));
    VIP_CUDA(cudaMemsetAsync(cursor, 0, C * sizeof(int32_t), st));
    const int TB = 256;
    k_cell_count<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(a, cell_cnt, node_cell);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(scan_excl<int32_t>(cell_cnt, cell_ptr, C, st));
    k_cell_fill<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(R, node_cell, cell_ptr, cursor, cell_rows);
    VIP_CUDA(cudaGetLastError());
    a.cell_ptr = cell_ptr;
    a.cell_rows = cell_rows;
    bool inside = false;
    for (const Geom& gg : c->geoms) inside = inside || gg.probes == VIP_PROBES_INSIDE;
    if (inside) {
        VIP_CUDA(dalloc(c, &c->pstep, R));
        k_probe_steps<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(a, c->pstep);
        VIP_CUDA(cudaGetLastError());
        a.pstep = c->pstep;
    }

    int32_t* bad = nullptr;
    VIP_CUDA(dalloc(c, &bad, 1));
    int32_t big = 0x7fffffff;
    VIP_CUDA(cudaMemcpyAsync(bad, &big, 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));

    // neighbour lists of all points
    Tables& T = c->T;
    T.npts = (int64_t)NPTYPE * R;
    int32_t* cnt = nullptr;
    VIP_CUDA(cudaMalloc(&cnt, T.npts * sizeof(int32_t)));
    VIP_CUDA(dalloc(c, &T.pptr, T.npts + 1));
    k_nbr_count<<<(unsigned)((T.npts + TB - 1) / TB), TB, 0, st>>>(a, T.npts, cnt, c->d_status, bad);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(scan_excl<int32_t>(cnt, T.pptr, T.npts, st));
    cudaFree(cnt);
    VIP_CUDA(cudaMemcpyAsync(&T.nnz_pts, T.pptr + T.npts, 8, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(&T.nnz_nodes, T.pptr + R, 8, cudaMemcpyDeviceToHost, st));
    int32_t hstat = 0, hbad = 0;
    VIP_CUDA(cudaMemcpyAsync(&hstat, c->d_status, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    if (hstat != 0) {
        char buf[160];
        snprintf(buf, sizeof buf, "point %d (type %d, row %lld) has more than %d neighbours",
                 hbad, (int)(hbad / R), (long long)(hbad % R), KMAX);
        c->err = buf;
        return VIP_ERR_ARG;
    }
    VIP_CUDA(dalloc(c, &T.pidx, std::max<int64_t>(T.nnz_pts, 1)));
    k_nbr_fill<<<(unsigned)((T.npts + TB - 1) / TB), TB, 0, st>>>(a, T.npts, T.pptr, T.pidx);
    VIP_CUDA(cudaGetLastError());
    cudaFree(cell_cnt);
    cudaFree(cursor);
    cudaFree(node_cell);

    // MLS weights
    VIP_CUDA(dalloc(c, &T.w00, std::max<int64_t>(T.nnz_pts, 1)));
    VIP_CUDA(dalloc(c, &T.wd, std::max<int64_t>(5 * T.nnz_nodes, 1)));
    k_mls<<<(unsigned)((T.npts + 127) / 128), 128, 0, st>>>(a, T.npts, T.pptr, T.pidx, T.w00, T.wd,
                                                           T.nnz_nodes, c->d_status, bad);
    VIP_CUDA(cudaGetLastError());
    k_vip_inv<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(a, c->inv_ew, c->inv_ns);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(cudaMemcpyAsync(&hstat, c->d_status, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    if (hstat == VIP_ERR_SINGULAR_STENCIL) {
        int t = (int)(hbad / R);
        int64_t r = hbad % R;
        // map the padded row back to the caller's node index
        int64_t node = -1;
        for (const Geom& gg : c->geoms)
            if (r >= gg.row0 && r < gg.row0 + gg.n) node = gg.off + (r - gg.row0);
        static const char* names[] = {"node", "east VIP", "west VIP", "north VIP", "south VIP",
                                      "normal point 1", "normal point 2"};
        char buf[200];
        snprintf(buf, sizeof buf, "singular MLS moment matrix at the %s of node %lld",
                 names[t], (long long)node);
        c->err = buf;
        return VIP_ERR_SINGULAR_STENCIL;
    }
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));

    // merged operators
    AsmArgs A;
    A.b = a; A.pptr = T.pptr; A.pidx = T.pidx; A.w00 = T.w00; A.wd = T.wd; A.nnz_nodes = T.nnz_nodes;
    A.inv_ew = c->inv_ew; A.inv_ns = c->inv_ns; A.first_row = c->first_row; A.identity = c->identity;
    vip_status s;
    if ((s = build_table(c, A, TB_LAP, R, T.lap, false)) != VIP_OK) return s;
    if (c->identity == VIP_IDENTITY_MLS)
        if ((s = build_table(c, A, TB_D00, R, T.d00, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_VE, R, T.ve, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_VW, R, T.vw, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_VN, R, T.vn, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_VS, R, T.vs, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_GX, R, T.gx, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_GY, R, T.gy, false)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_HELM, 2 * R, T.helm, true)) != VIP_OK) return s;
    if ((s = build_table(c, A, TB_POIS, R, T.pois, true)) != VIP_OK) return s;
    VIP_CUDA(cudaStreamSynchronize(st));
    return VIP_OK;
}

}  // namespace vip
