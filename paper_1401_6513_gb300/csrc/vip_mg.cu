// Aggregation multigrid preconditioner for the pressure-increment solve (Eq. 13).
//
// The node sets live on a regular background lattice (plus boundary nodes on
// curves).  Level 1 aggregates the nodes of each 2h x 2h cell of that lattice;
// level l+1 aggregates 2 x 2 cells of level l.  Prolongation is piecewise
// constant, restriction its transpose, and every coarse operator is the Galerkin
// product P^T A P of the level above, so the coarse levels inherit the MLS
// stencils and the boundary rows of the fine operator.  Because the aggregates are
// lattice cells, every coarse operator is a structured 5 x 5 stencil on a cell
// lattice (25 coefficients per cell).  The setup works through neighbour, parent
// and child tables; the V-cycle addresses cells by lattice position instead, with
// rows padded to a multiple of 32 cells and the stencils stored in slices of 32
// cells ([slice][offset][lane]) so that a warp reads one contiguous block per
// slice.  All sums are formed in a fixed order, so the hierarchy is deterministic.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "vip_internal.cuh"
#include "vip_mg.cuh"

namespace vip {

// cell of a fine row at level 1 (-1: not a node)
__global__ void k_mg_agg(int64_t R, const int8_t* __restrict__ rt, const int32_t* __restrict__ rg,
                         const double* __restrict__ x, const double* __restrict__ y,
                         const MgGeom* __restrict__ mg, const int64_t* __restrict__ off1,
                         int32_t* __restrict__ agg) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (rt[r] != ROW_NODE) { agg[r] = -1; return; }
    const MgGeom& G = mg[rg[r]];
    long long ix = llrint((x[r] - G.x0) / G.h);
    long long iy = llrint((y[r] - G.y0) / G.h);
    int cx = (int)(ix >> 1), cy = (int)(iy >> 1);
    const int nx = G.nx[1], ny = G.ny[1];
    if (G.periodic_x) { cx %= nx; if (cx < 0) cx += nx; } else cx = min(max(cx, 0), nx - 1);
    if (G.periodic_y) { cy %= ny; if (cy < 0) cy += ny; } else cy = min(max(cy, 0), ny - 1);
    agg[r] = (int32_t)(off1[rg[r]] + (int64_t)cy * G.sx[1] + cx);
}

// neighbour table, parent and children of the cells of one level
__global__ void k_mg_topology(int64_t ncells, const int32_t* __restrict__ cgeom,
                              const int32_t* __restrict__ cx_, const int32_t* __restrict__ cy_,
                              const MgGeom* __restrict__ mg, const int64_t* __restrict__ offl,
                              const int64_t* __restrict__ offp, int level, int has_parent,
                              int32_t* __restrict__ nbr, int32_t* __restrict__ parent) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int g = cgeom[c];
    const MgGeom& G = mg[g];
    int nx = G.nx[level], ny = G.ny[level], sx = G.sx[level];
    int x = cx_[c], y = cy_[c];
    if (x < 0) {  // padding cell
        for (int o = 0; o < 25; ++o) nbr[(int64_t)o * ncells + c] = -1;
        if (has_parent) parent[c] = -1;
        return;
    }
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            int xx = x + dx, yy = y + dy;
            bool ok = true;
            if (G.periodic_x) { xx %= nx; if (xx < 0) xx += nx; } else ok &= xx >= 0 && xx < nx;
            if (G.periodic_y) { yy %= ny; if (yy < 0) yy += ny; } else ok &= yy >= 0 && yy < ny;
            int o = (dy + 2) * 5 + (dx + 2);
            nbr[(int64_t)o * ncells + c] = ok ? (int32_t)(offl[g] + (int64_t)yy * sx + xx) : -1;
        }
    if (has_parent) {
        int px = x >> 1, py = y >> 1;
        parent[c] = (int32_t)(offp[g] + (int64_t)py * G.sx[level + 1] + px);
    }
}

// canonical 5x5 offset index of target cell t seen from cell c (wrap-aware), -1 if none
__device__ __forceinline__ int offset_of(const int32_t* __restrict__ nbr, int64_t ncells, int64_t c,
                                         int32_t t) {
    for (int o = 0; o < 25; ++o)
        if (nbr[(int64_t)o * ncells + c] == t) return o;
    return -1;
}

// level-1 Galerkin coefficients from the fine SELL operator (rows of a cell in
// ascending order, entries in stored order)
__global__ void k_mg_galerkin1(int64_t ncells, const int64_t* __restrict__ cptr,
                               const int32_t* __restrict__ crow, Sell A,
                               const int32_t* __restrict__ agg, const int32_t* __restrict__ nbr,
                               double* __restrict__ coef) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    double acc[25];
    for (int o = 0; o < 25; ++o) acc[o] = 0.0;
    for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
        int64_t r = crow[q];
        int64_t s = r >> 5;
        int64_t base = A.sptr[s] + (r & 31);
        int len = A.rowlen[r];
        for (int k = 0; k < len; ++k) {
            int64_t e = base + (int64_t)k * SLICE;
            int32_t j = A.col[e];
            int32_t t = agg[j];
            if (t < 0) continue;  // border (mu) and padding columns stay on the fine level
            int o = offset_of(nbr, ncells, c, t);
            if (o >= 0) acc[o] += A.v64[e];
        }
    }
    for (int o = 0; o < 25; ++o) coef[(int64_t)o * ncells + c] = acc[o];
}

// level l+1 from level l: sum over the (up to 4) children in fixed order
__global__ void k_mg_galerkin(int64_t nc, const int64_t* __restrict__ child,  // [4][nc]
                              int64_t nf, const int32_t* __restrict__ fnbr,
                              const double* __restrict__ fcoef, const int32_t* __restrict__ fparent,
                              const int32_t* __restrict__ cnbr, double* __restrict__ ccoef) {
    int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= nc) return;
    double acc[25];
    for (int o = 0; o < 25; ++o) acc[o] = 0.0;
    for (int k = 0; k < 4; ++k) {
        int64_t c = child[(int64_t)k * nc + C];
        if (c < 0) continue;
        for (int o = 0; o < 25; ++o) {
            int32_t j = fnbr[(int64_t)o * nf + c];
            if (j < 0) continue;
            double a = fcoef[(int64_t)o * nf + c];
            if (a == 0.0) continue;
            int oc = offset_of(cnbr, nc, C, fparent[j]);
            if (oc >= 0) acc[oc] += a;
        }
    }
    for (int o = 0; o < 25; ++o) ccoef[(int64_t)o * nc + C] = acc[o];
}

// sliced copy of the stencils ([n/32][25][32]), the l1-Jacobi scaling
// -1 / sum_o |a_co| of the smoother (0 for empty and padding cells), and per
// slice of 32 cells whether any stencil has a nonzero outside the central 3 x 3
// offsets.  Away from boundaries a 2 x 2 aggregate of the 13-point fine stencil, and
// of a 3 x 3 coarse stencil, couples only to the adjacent cells, so most slices
// need 9 of the 25 products.  n is a multiple of 32 and blockDim a multiple of 32,
// so each warp is one slice.
__global__ void k_mg_finish(int64_t n, const double* __restrict__ coef, double* __restrict__ coefs,
                            double* __restrict__ dinv, uint8_t* __restrict__ ring) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0;
    bool outer = false;
    for (int o = 0; o < 25; ++o) {
        const double a = coef[(int64_t)o * n + c];
        coefs[(c >> 5) * 800 + o * 32 + (c & 31)] = a;
        s += fabs(a);
        const int dy = o / 5 - 2, dx = o % 5 - 2;
        if ((dx < -1 || dx > 1 || dy < -1 || dy > 1) && a != 0.0) outer = true;
    }
    // Every row of the Poisson operator that reaches the coarse levels is a node
    // equation with a negative diagonal (Laplacian rows, and boundary rows scaled to
    // match them); a Galerkin cell whose diagonal comes out positive is an artefact
    // of an aggregate cut by the boundary, and smoothing it with the sign of that
    // diagonal would push the error the wrong way.  So the step has the operator's
    // sign on every cell.
    dinv[c] = (s != 0.0) ? -1.0 / s : 0.0;
    const unsigned any = __ballot_sync(0xffffffffu, outer);
    if ((threadIdx.x & 31) == 0) ring[c >> 5] = any ? 1 : 0;
}

// fine-level l1-Jacobi scaling sign(a_rr) / sum_k |a_rk|
__global__ void k_mg_fine_diag(Sell A, double* __restrict__ dinv) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.nrows) return;
    int64_t base = A.sptr[r >> 5] + (r & 31);
    double d = 0.0, s = 0.0;
    for (int k = 0; k < A.rowlen[r]; ++k) {
        int64_t e = base + (int64_t)k * SLICE;
        if (A.col[e] == r) d += A.v64[e];
        s += fabs(A.v64[e]);
    }
    dinv[r] = s != 0.0 ? (d < 0.0 ? -1.0 : 1.0) / s : 0.0;
}

// w[i] = omega * d[i], and its FP32 rounding
__global__ void k_mg_scale(int64_t n, double omega, const double* __restrict__ d, double* __restrict__ w,
                           float* __restrict__ w32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = omega * d[i];
        w[i] = v;
        w32[i] = (float)v;
    }
}

// b[i] = a[i] rounded to FP32
__global__ void k_mg_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

vip_status mg_set_params(vip_ctx* c, Multigrid& M, float omega, float corr) {
    M.corr = corr;
    M.omega = omega;
    if (!M.built || M.scaled_omega == omega) return VIP_OK;
    const int TB = 256;
    cudaStream_t st = c->stream;
    k_mg_scale<<<(unsigned)((c->R + TB - 1) / TB), TB, 0, st>>>(c->R, (double)omega, M.fdinv, M.fwdinv,
                                                                 M.fwdinv32);
    for (int l = 1; l <= M.nlev; ++l) {
        const MgLevel& lv = M.lev[l];
        k_mg_scale<<<(unsigned)((lv.n + TB - 1) / TB), TB, 0, st>>>(lv.n, (double)omega, lv.dinv, lv.wdinv,
                                                                     lv.wdinv32);
    }
    VIP_CUDA(cudaGetLastError());
    M.scaled_omega = omega;
    return VIP_OK;
}

// Dense inverse of one geometry's coarsest operator, A (m x m, row-major), by
// Gauss-Jordan elimination with partial pivoting in FP64 on the host (setup only;
// the row updates of each pivot step run on the host's cores with OpenMP).
// Cells without a row (empty cells) are decoupled: their unknown stays 0.  The
// result is stored row-major, inv[i * m + j] = (A^{-1})_{ij}.
static void coarse_inverse(std::vector<double>& A, int m, double* inv) {
    const int w = 2 * m;
    std::vector<double> T((size_t)m * w, 0.0);
    for (int r = 0; r < m; ++r) {
        bool empty = true;
        for (int j = 0; j < m; ++j) {
            T[(size_t)r * w + j] = A[(size_t)r * m + j];
            if (A[(size_t)r * m + j] != 0.0) empty = false;
        }
        if (empty) T[(size_t)r * w + r] = 1.0;
        T[(size_t)r * w + m + r] = 1.0;
    }
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (std::fabs(T[(size_t)i * w + k]) > std::fabs(T[(size_t)piv * w + k])) piv = i;
        if (piv != k)
            for (int j = 0; j < w; ++j) std::swap(T[(size_t)k * w + j], T[(size_t)piv * w + j]);
        const double d = T[(size_t)k * w + k];
        const double di = std::fabs(d) > 1e-300 ? 1.0 / d : 0.0;
        double* rk = &T[(size_t)k * w];
        for (int j = 0; j < w; ++j) rk[j] *= di;
        double* t0 = T.data();
#pragma omp parallel for schedule(static) if (m >= 256)
        for (int i = 0; i < m; ++i) {
            if (i == k) continue;
            double* ri = t0 + (size_t)i * w;
            const double f = ri[k];
            if (f == 0.0) continue;
            for (int j = k; j < w; ++j) ri[j] -= f * rk[j];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) inv[(size_t)i * m + j] = T[(size_t)i * w + m + j];
}

vip_status mg_build(vip_ctx* c, Multigrid& M) {
    cudaStream_t st = c->stream;
    const int G = (int)c->geoms.size();
    const Sell& A = c->T.pois;
    // lattice of each geometry
    std::vector<MgGeom> hg(G);
    int L = 1;
    bool any_closed = false;
    for (const Geom& gg : c->geoms) any_closed |= gg.bordered;
    const int coarsest = any_closed ? MG_COARSEST_CLOSED : MG_COARSEST_OPEN;
    for (int g = 0; g < G; ++g) {
        const Geom& gg = c->geoms[g];
        double hmin = 1e300, x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
        for (int64_t i = gg.off; i < gg.off + gg.n; ++i) {
            hmin = std::min(hmin, c->hh[i]);
            x0 = std::min(x0, c->hx[i]); x1 = std::max(x1, c->hx[i]);
            y0 = std::min(y0, c->hy[i]); y1 = std::max(y1, c->hy[i]);
        }
        MgGeom& m = hg[g];
        memset(&m, 0, sizeof(m));
        m.h = hmin;
        m.periodic_x = gg.Lx > 0;
        m.periodic_y = gg.Ly > 0;
        // a cell-grid shift moves the lattice origin back by one spacing and adds one
        // lattice column (row), so that lattice index i falls in cell (i + 1) / 2
        const int shx = m.periodic_x ? 0 : gg.mg_shift_x, shy = m.periodic_y ? 0 : gg.mg_shift_y;
        m.x0 = m.periodic_x ? 0.0 : x0 - shx * hmin;
        m.y0 = m.periodic_y ? 0.0 : y0 - shy * hmin;
        int NX = m.periodic_x ? (int)llround(gg.Lx / hmin) : (int)llround((x1 - x0) / hmin) + 1 + shx;
        int NY = m.periodic_y ? (int)llround(gg.Ly / hmin) : (int)llround((y1 - y0) / hmin) + 1 + shy;
        m.nx[0] = NX;
        m.ny[0] = NY;
        int l = 0;
        while (l + 1 < MG_MAXLEV) {
            int nx = (m.nx[l] + 1) / 2, ny = (m.ny[l] + 1) / 2;
            m.nx[l + 1] = nx;
            m.ny[l + 1] = ny;
            ++l;
            if ((int64_t)nx * ny <= coarsest) break;
        }
        L = std::max(L, l);
    }
    // every geometry gets the same number of levels (tiny ones keep halving to 1 x 1)
    for (int g = 0; g < G; ++g)
        for (int l = 1; l <= L; ++l)
            if (hg[g].nx[l] == 0) {
                hg[g].nx[l] = (hg[g].nx[l - 1] + 1) / 2;
                hg[g].ny[l] = (hg[g].ny[l - 1] + 1) / 2;
            }
    M.nlev = L;  // coarse levels 1..L
    // row strides: multiples of 32 on the tiled levels (the coarsest level keeps
    // sx = nx, so its cells are numbered densely for the direct solve)
    for (int g = 0; g < G; ++g)
        for (int l = 1; l <= L; ++l) {
            const int nx = hg[g].nx[l];
            hg[g].sx[l] = (l == L || nx < 32) ? nx : (nx + 31) / 32 * 32;
        }
    VIP_CUDA(dalloc(c, &M.geom, G));
    VIP_CUDA(cudaMemcpyAsync(M.geom, hg.data(), G * sizeof(MgGeom), cudaMemcpyHostToDevice, st));
    // per level: cell offsets (each geometry's block a multiple of 32 cells), coordinates
    std::vector<std::vector<int64_t>> offs(L + 2, std::vector<int64_t>(G));
    for (int l = 1; l <= L; ++l) {
        MgLevel& lv = M.lev[l];
        int64_t n = 0;
        for (int g = 0; g < G; ++g) {
            offs[l][g] = n;
            n += ((int64_t)hg[g].sx[l] * hg[g].ny[l] + 31) / 32 * 32;
        }
        lv.n = n;
        std::vector<int32_t> cg(n), cx(n, -1), cy(n, -1);
        for (int g = 0; g < G; ++g) {
            const int64_t end = (g + 1 < G) ? offs[l][g + 1] : n;
            for (int64_t id = offs[l][g]; id < end; ++id) cg[id] = g;
            for (int yy = 0; yy < hg[g].ny[l]; ++yy)
                for (int xx = 0; xx < hg[g].nx[l]; ++xx) {
                    int64_t id = offs[l][g] + (int64_t)yy * hg[g].sx[l] + xx;
                    cx[id] = xx; cy[id] = yy;
                }
        }
        VIP_CUDA(dalloc(c, &lv.cgeom, n)); VIP_CUDA(dalloc(c, &lv.cx, n)); VIP_CUDA(dalloc(c, &lv.cy, n));
        VIP_CUDA(dalloc(c, &lv.off, G));
        VIP_CUDA(cudaMemcpyAsync(lv.cgeom, cg.data(), n * 4, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(lv.cx, cx.data(), n * 4, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(lv.cy, cy.data(), n * 4, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(lv.off, offs[l].data(), G * 8, cudaMemcpyHostToDevice, st));
        VIP_CUDA(dalloc(c, &lv.nbr, 25 * n));
        VIP_CUDA(dalloc(c, &lv.parent, n));
        VIP_CUDA(dalloc(c, &lv.coef, 25 * n));
        VIP_CUDA(dalloc(c, &lv.coefs, 25 * n));
        VIP_CUDA(dalloc(c, &lv.coefs32, 25 * n));
        VIP_CUDA(dalloc(c, &lv.dinv, n));
        VIP_CUDA(dalloc(c, &lv.wdinv, n));
        VIP_CUDA(dalloc(c, &lv.wdinv32, n));
        VIP_CUDA(dalloc(c, &lv.ring, n / 32));
        {
            // Tile height: a level with few 32 x 32 tiles would keep most SMs idle
            // while a few apply 1024 stencils each on the FP64 pipe, so small levels
            // take shorter tiles.  Cost model per CTA: rounds of tiles x (stencil and
            // staging FP64 work + a fixed latency per tile).
            const int64_t nblk = std::max(1, c->num_sms);
            double best_cost = 1e300;
            for (int h : {32, 16, 8, 4, 2}) {
                int64_t nt = 0;
                for (int g = 0; g < G; ++g)
                    nt += (int64_t)((hg[g].nx[l] + 31) / 32) * ((hg[g].ny[l] + h - 1) / h);
                const double cost = (double)((nt + nblk - 1) / nblk) *
                                    (h * 32 * 12.0 + (h + 4) * 36 * 3.0 + 4000.0);
                if (cost < best_cost) { best_cost = cost; lv.th = h; }
            }
            std::vector<MgLevGeom> lgh(G);
            std::vector<MgTile> th;
            for (int g = 0; g < G; ++g) {
                lgh[g] = {offs[l][g], hg[g].nx[l], hg[g].ny[l], hg[g].sx[l], hg[g].periodic_x,
                          hg[g].periodic_y, 0};
                for (int y0 = 0; y0 < hg[g].ny[l]; y0 += lv.th)
                    for (int x0 = 0; x0 < hg[g].nx[l]; x0 += 32) th.push_back({g, x0, y0, 0});
            }
            VIP_CUDA(dalloc(c, &lv.lg, G));
            VIP_CUDA(cudaMemcpyAsync(lv.lg, lgh.data(), G * sizeof(MgLevGeom), cudaMemcpyHostToDevice, st));
            lv.ntiles = (int64_t)th.size();
            VIP_CUDA(dalloc(c, &lv.tiles, th.size()));
            VIP_CUDA(cudaMemcpyAsync(lv.tiles, th.data(), th.size() * sizeof(MgTile), cudaMemcpyHostToDevice,
                                     st));
        }
        for (void** v : {&lv.x, &lv.b, &lv.y}) {
            char* m = nullptr;
            VIP_CUDA(dalloc(c, &m, n * 8));
            *v = m;
        }
        cudaStreamSynchronize(st);
    }
    const int TB = 256;
    for (int l = 1; l <= L; ++l) {
        MgLevel& lv = M.lev[l];
        k_mg_topology<<<(unsigned)((lv.n + TB - 1) / TB), TB, 0, st>>>(
            lv.n, lv.cgeom, lv.cx, lv.cy, M.geom, lv.off, l < L ? M.lev[l + 1].off : lv.off, l,
            l < L ? 1 : 0, lv.nbr, lv.parent);
        VIP_CUDA(cudaGetLastError());
    }
    // children lists of levels 2..L
    for (int l = 2; l <= L; ++l) {
        MgLevel& lv = M.lev[l];
        std::vector<int32_t> par(M.lev[l - 1].n);
        VIP_CUDA(cudaMemcpy(par.data(), M.lev[l - 1].parent, par.size() * 4, cudaMemcpyDeviceToHost));
        std::vector<int64_t> ch(4 * lv.n, -1);
        std::vector<int> cnt(lv.n, 0);
        for (int64_t f = 0; f < (int64_t)par.size(); ++f) {
            int32_t p = par[f];
            if (p < 0) continue;  // padding cell
            ch[(int64_t)cnt[p] * lv.n + p] = f;
            cnt[p]++;
        }
        VIP_CUDA(dalloc(c, &lv.child, 4 * lv.n));
        VIP_CUDA(cudaMemcpyAsync(lv.child, ch.data(), ch.size() * 8, cudaMemcpyHostToDevice, st));
        cudaStreamSynchronize(st);
    }
    // fine rows -> level-1 cells; rows of each cell in ascending order
    const int64_t R = c->R;
    VIP_CUDA(dalloc(c, &M.agg, R));
    k_mg_agg<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(R, c->row_type, c->row_geom, c->x, c->y,
                                                          M.geom, M.lev[1].off, M.agg);
    VIP_CUDA(cudaGetLastError());
    {
        std::vector<int32_t> agg(R);
        VIP_CUDA(cudaMemcpy(agg.data(), M.agg, R * 4, cudaMemcpyDeviceToHost));
        const int64_t n1 = M.lev[1].n;
        std::vector<int64_t> ptr(n1 + 1, 0);
        for (int64_t r = 0; r < R; ++r)
            if (agg[r] >= 0) ptr[agg[r] + 1]++;
        for (int64_t i = 0; i < n1; ++i) ptr[i + 1] += ptr[i];
        std::vector<int32_t> rows(std::max<int64_t>(ptr[n1], 1));
        std::vector<int64_t> cur(ptr.begin(), ptr.end() - 1);
        for (int64_t r = 0; r < R; ++r)
            if (agg[r] >= 0) rows[cur[agg[r]]++] = (int32_t)r;
        VIP_CUDA(dalloc(c, &M.cptr, n1 + 1));
        VIP_CUDA(dalloc(c, &M.crow, rows.size()));
        VIP_CUDA(cudaMemcpyAsync(M.cptr, ptr.data(), (n1 + 1) * 8, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(M.crow, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, st));
        cudaStreamSynchronize(st);
    }
    // Galerkin coefficients
    {
        MgLevel& l1 = M.lev[1];
        k_mg_galerkin1<<<(unsigned)((l1.n + TB - 1) / TB), TB, 0, st>>>(l1.n, M.cptr, M.crow, A, M.agg,
                                                                       l1.nbr, l1.coef);
        VIP_CUDA(cudaGetLastError());
        for (int l = 2; l <= L; ++l) {
            MgLevel& lc = M.lev[l];
            MgLevel& lf = M.lev[l - 1];
            k_mg_galerkin<<<(unsigned)((lc.n + TB - 1) / TB), TB, 0, st>>>(
                lc.n, lc.child, lf.n, lf.nbr, lf.coef, lf.parent, lc.nbr, lc.coef);
            VIP_CUDA(cudaGetLastError());
        }
        for (int l = 1; l <= L; ++l) {
            MgLevel& lv = M.lev[l];
            k_mg_finish<<<(unsigned)((lv.n + TB - 1) / TB), TB, 0, st>>>(lv.n, lv.coef, lv.coefs, lv.dinv,
                                                                          lv.ring);
            k_mg_f32<<<(unsigned)((25 * lv.n + TB - 1) / TB), TB, 0, st>>>(25 * lv.n, lv.coefs, lv.coefs32);
            VIP_CUDA(cudaGetLastError());
        }
    }
    {   // exact solve on the coarsest level: dense inverses, one per geometry (host)
        MgLevel& lc = M.lev[L];
        std::vector<int64_t> ioff(G);
        int64_t tot = 0;
        for (int g = 0; g < G; ++g) {
            const int m = hg[g].nx[L] * hg[g].ny[L];
            ioff[g] = tot;
            tot += (int64_t)m * m;
        }
        std::vector<double> hcoef((size_t)25 * lc.n);
        std::vector<int32_t> hnbr((size_t)25 * lc.n);
        VIP_CUDA(cudaMemcpyAsync(hcoef.data(), lc.coef, hcoef.size() * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(hnbr.data(), lc.nbr, hnbr.size() * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        std::vector<double> hinv((size_t)tot);
        for (int g = 0; g < G; ++g) {
            const int m = hg[g].nx[L] * hg[g].ny[L];
            const int64_t c0 = offs[L][g];  // cells numbered densely on the coarsest level
            std::vector<double> Ad((size_t)m * m, 0.0);
            for (int r = 0; r < m; ++r)
                for (int o = 0; o < 25; ++o) {
                    const int32_t j = hnbr[(size_t)o * lc.n + c0 + r];
                    if (j >= 0) Ad[(size_t)r * m + (j - c0)] += hcoef[(size_t)o * lc.n + c0 + r];
                }
            coarse_inverse(Ad, m, hinv.data() + ioff[g]);
        }
        M.cinv_entries = tot;
        VIP_CUDA(dalloc(c, &M.cinv, tot));
        VIP_CUDA(dalloc(c, &M.cinv_off, G));
        VIP_CUDA(cudaMemcpyAsync(M.cinv, hinv.data(), tot * 8, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(M.cinv_off, ioff.data(), G * 8, cudaMemcpyHostToDevice, st));
        VIP_CUDA(dalloc(c, &M.cinv32, tot));
        k_mg_f32<<<(unsigned)((tot + TB - 1) / TB), TB, 0, st>>>(tot, M.cinv, M.cinv32);
        VIP_CUDA(cudaGetLastError());
        VIP_CUDA(cudaStreamSynchronize(st));
        M.ngeom = G;
    }
    VIP_CUDA(dalloc(c, &M.fdinv, R));
    VIP_CUDA(dalloc(c, &M.fwdinv, R));
    VIP_CUDA(dalloc(c, &M.fwdinv32, R));
    k_mg_fine_diag<<<(unsigned)((R + TB - 1) / TB), TB, 0, st>>>(A, M.fdinv);
    VIP_CUDA(cudaGetLastError());
    {
        char* m = nullptr;
        VIP_CUDA(dalloc(c, &m, R * 8));
        M.fr = m;
        VIP_CUDA(dalloc(c, &m, R * 8));
        M.fx = m;
    }
    VIP_CUDA(cudaStreamSynchronize(st));
    M.built = true;
    M.scaled_omega = -1.0f;
    vip_status s = mg_set_params(c, M, M.omega, M.corr);
    if (s != VIP_OK) return s;
    VIP_CUDA(cudaStreamSynchronize(st));
    return VIP_OK;
}

}  // namespace vip
