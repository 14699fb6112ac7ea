// Per-step gather-stencil kernels of the fractional step (Sec. 2, Sec. 4.1):
//   conv_rhs : VIP convection (Sec. 4.1 item 1), its Adams-Bashforth extrapolation
//              (Sec. 4) and the right-hand side of Eq. (12) times dt;
//   div      : right-hand side of Eq. (13), VIP divergence of u* over dt;
//   project  : Eq. (14) with the VIP gradient and the pressure update Eq. (15).
// One thread per padded row; a warp covers one 32-row slice, so every table read
// (slice-major SELL-32) is coalesced.  Field values are gathered through the
// read-only path.
#include "vip_internal.cuh"

namespace vip {

struct StepArgs {
    int64_t R;
    const int8_t* row_type;
    const uint8_t* kind;
    const int32_t* row_geom;
    const GeomDev* g;
    const double* inv_ew;
    const double* inv_ns;
    Sell ve, vw, vn, vs, gx, gy, lap, d00;
    int identity;
    int incremental;   // 1: r^n carries -G p^n and p^{n+1} adds p^n (not VIP_PRESSURE_KIM_MOIN)
    int rot_interior;  // 1: the term -(dt/2Re) L phi of Eq. 15 at interior nodes only
    const int64_t* step;
};

__device__ __forceinline__ double gather(const Sell& A, int64_t r, const double* __restrict__ f) {
    int64_t s = r >> 5;
    int64_t base = A.sptr[s] + (r & 31);
    int w = A.width[s];
    double sum = 0.0;
    for (int k = 0; k < w; ++k) {
        int64_t e = base + (int64_t)k * SLICE;
        sum += __ldg(A.v64 + e) * __ldg(f + __ldg(A.col + e));
    }
    return sum;
}

// Two fields through the same stencil (one pass over the table).
__device__ __forceinline__ void gather2(const Sell& A, int64_t r, const double* __restrict__ f1,
                                       const double* __restrict__ f2, double& o1, double& o2) {
    int64_t s = r >> 5;
    int64_t base = A.sptr[s] + (r & 31);
    int w = A.width[s];
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < w; ++k) {
        int64_t e = base + (int64_t)k * SLICE;
        double a = __ldg(A.v64 + e);
        int c = __ldg(A.col + e);
        s1 += a * __ldg(f1 + c);
        s2 += a * __ldg(f2 + c);
    }
    o1 = s1;
    o2 = s2;
}

// Convection term at an interior row: products of VIP values differenced
// across each VIP pair and divided by the pair distance.
__device__ __forceinline__ void convection_row(const StepArgs& a, int64_t r, const double* u,
                                               const double* v, double& Nu, double& Nv) {
    double ue, ve, uw, vw, un, vn, us, vs;
    gather2(a.ve, r, u, v, ue, ve);
    gather2(a.vw, r, u, v, uw, vw);
    gather2(a.vn, r, u, v, un, vn);
    gather2(a.vs, r, u, v, us, vs);
    double iew = a.inv_ew[r], ins = a.inv_ns[r];
    Nu = (ue * ue - uw * uw) * iew + (un * vn - us * vs) * ins;
    Nv = (ue * ve - uw * vw) * iew + (vn * vn - vs * vs) * ins;
}

__global__ void k_conv_rhs(StepArgs a, const double* __restrict__ u, const double* __restrict__ v,
                           const double* __restrict__ p, const double* __restrict__ ubc,
                           const double* __restrict__ vbc, double* __restrict__ nu_prev,
                           double* __restrict__ nv_prev, double* __restrict__ hsol,
                           double* __restrict__ hrhs, const double* __restrict__ uv_prev) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t R = a.R;
    if (r >= R) return;
    // initial guess of the Helmholtz solve: u^n + (u*^n - u^{n-1}) once a step has been
    // taken (hsol still holds the last solve's u*^n: the increment of the intermediate
    // velocity one step later, an O(dt^2) guess), else u^n
    if (*a.step > 0) {
        hsol[r] = u[r] + (hsol[r] - uv_prev[r]);
        hsol[R + r] = v[r] + (hsol[R + r] - uv_prev[R + r]);
    } else {
        hsol[r] = u[r];
        hsol[R + r] = v[r];
    }
    double ru = 0.0, rv = 0.0;
    if (a.row_type[r] == ROW_NODE) {
        uint8_t k = a.kind[r];
        if (k == VIP_NODE_INTERIOR) {
            const GeomDev& G = a.g[a.row_geom[r]];
            double Nu, Nv;
            convection_row(a, r, u, v, Nu, Nv);
            double Nu0 = Nu, Nv0 = Nv;
            if (*a.step > 0) { Nu0 = nu_prev[r]; Nv0 = nv_prev[r]; }
            nu_prev[r] = Nu;
            nv_prev[r] = Nv;
            double gpx = 0.0, gpy = 0.0;
            if (a.incremental) { gpx = gather(a.gx, r, p); gpy = gather(a.gy, r, p); }
            double lu, lv;
            gather2(a.lap, r, u, v, lu, lv);
            double iu, iv;
            if (a.identity == VIP_IDENTITY_MLS) gather2(a.d00, r, u, v, iu, iv);
            else { iu = u[r]; iv = v[r]; }
            // (I + al L) u^n - dt [ (3 N^n - N^{n-1}) / 2 + G p^n ]  (no G p^n: KIM_MOIN)
            ru = iu + G.alpha * lu - G.dt * ((1.5 * Nu - 0.5 * Nu0) + gpx);
            rv = iv + G.alpha * lv - G.dt * ((1.5 * Nv - 0.5 * Nv0) + gpy);
        } else {
            if (k == VIP_NODE_WALL) ru = ubc[r];
            if (k == VIP_NODE_WALL || k == VIP_NODE_SLIP) rv = vbc[r];
        }
    }
    hrhs[r] = ru;
    hrhs[R + r] = rv;
}

__global__ void k_div(StepArgs a, const double* __restrict__ hsol, double* __restrict__ b) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t R = a.R;
    if (r >= R) return;
    double d = 0.0;
    int rt = a.row_type[r];
    const GeomDev& G = a.g[a.row_geom[r]];
    // closed domain: the reference node's equation sits in the border row, its own row is phi_k = 0
    int64_t q = (rt == ROW_BORDER) ? G.pin : r;
    if ((rt == ROW_NODE && a.kind[r] == VIP_NODE_INTERIOR && !(G.bordered && r == G.pin)) ||
        rt == ROW_BORDER)
        d = (gather(a.gx, q, hsol) + gather(a.gy, q, hsol + R)) / G.dt;
    b[r] = d;
}

__global__ void k_project(StepArgs a, const double* __restrict__ hsol, const double* __restrict__ phi,
                          double* __restrict__ u, double* __restrict__ v, double* __restrict__ p,
                          int64_t* step, double* __restrict__ uv_prev) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t R = a.R;
    if (r == 0) atomicAdd((unsigned long long*)step, 1ull);
    if (r >= R) return;
    if (a.row_type[r] != ROW_NODE) return;
    const GeomDev& G = a.g[a.row_geom[r]];
    double us = hsol[r], vs = hsol[R + r];
    uv_prev[r] = u[r];       // u^n, v^n: the next step's u^{n-1}, v^{n-1}
    uv_prev[R + r] = v[r];
    if (a.kind[r] == VIP_NODE_INTERIOR) {
        us -= G.dt * gather(a.gx, r, phi);
        vs -= G.dt * gather(a.gy, r, phi);
    }
    u[r] = us;
    v[r] = vs;
    // Eq. (15): p^{n+1} = p^n + phi - (dt / 2Re) L phi (KIM_MOIN: without p^n;
    // INCREMENTAL_INTERIOR: without the L phi term at boundary nodes)
    double base = a.incremental ? p[r] : 0.0;
    double rot = (a.rot_interior && a.kind[r] != VIP_NODE_INTERIOR) ? 0.0 : G.alpha * gather(a.lap, r, phi);
    p[r] = base + phi[r] - rot;
}

__global__ void k_spmv(Sell A, const double* __restrict__ x, double* __restrict__ y) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.nrows) return;
    y[r] = gather(A, r, x);
}

__global__ void k_convection(StepArgs a, const double* __restrict__ u, const double* __restrict__ v,
                             double* __restrict__ Nu, double* __restrict__ Nv) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    double nu = 0.0, nv = 0.0;
    if (a.row_type[r] == ROW_NODE && a.kind[r] == VIP_NODE_INTERIOR) convection_row(a, r, u, v, nu, nv);
    Nu[r] = nu;
    Nv[r] = nv;
}

static StepArgs step_args(vip_ctx* c) {
    StepArgs a;
    a.R = c->R; a.row_type = c->row_type; a.kind = c->kind; a.row_geom = c->row_geom; a.g = c->gdev;
    a.inv_ew = c->inv_ew; a.inv_ns = c->inv_ns;
    a.ve = c->T.ve; a.vw = c->T.vw; a.vn = c->T.vn; a.vs = c->T.vs;
    a.gx = c->T.gx; a.gy = c->T.gy; a.lap = c->T.lap; a.d00 = c->T.d00;
    a.identity = c->identity;
    a.incremental = c->pressure != VIP_PRESSURE_KIM_MOIN ? 1 : 0;
    a.rot_interior = c->pressure == VIP_PRESSURE_INCREMENTAL_INTERIOR ? 1 : 0;
    a.step = c->d_step;
    return a;
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_conv_rhs(vip_ctx* c, cudaStream_t s) {
    k_conv_rhs<<<nblk(c->R, 256), 256, 0, s>>>(step_args(c), c->u, c->v, c->p, c->ubc, c->vbc,
                                               c->nu_prev, c->nv_prev, c->hsol, c->hrhs, c->uv_prev);
}
void launch_div(vip_ctx* c, cudaStream_t s) {
    k_div<<<nblk(c->R, 256), 256, 0, s>>>(step_args(c), c->hsol, c->prhs);
}
void launch_project(vip_ctx* c, cudaStream_t s) {
    k_project<<<nblk(c->R, 256), 256, 0, s>>>(step_args(c), c->hsol, c->phi, c->u, c->v, c->p,
                                              c->d_step, c->uv_prev);
}
void launch_spmv(const Sell& A, const double* x, double* y, cudaStream_t s) {
    k_spmv<<<nblk(A.nrows, 256), 256, 0, s>>>(A, x, y);
}
void launch_convection(vip_ctx* c, const double* u, const double* v, double* Nu, double* Nv,
                       cudaStream_t s) {
    k_convection<<<nblk(c->R, 256), 256, 0, s>>>(step_args(c), u, v, Nu, Nv);
}

}  // namespace vip
