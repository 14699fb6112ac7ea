// Krylov solves of Eqs. (12) and (13): one persistent cooperative launch solves a
// batch of independent sparse systems (block-diagonal SELL-32 operator, each
// system a contiguous range of slices) with unpreconditioned BiCGSTAB
// (van der Vorst, 1992) inside an FP64 iterative-refinement loop:
//
//   repeat:  r = b - A x   (FP64 operator, FP64 vectors);  stop if ||r|| <= rtol ||b||
//            solve A d = r by BiCGSTAB in precision T from d = 0 with r_hat = r,
//            until ||r_d|| <= tol_in, or until |r_hat.r| or |r_hat.v| falls below
//            1e-12 of its norms (restart);   x += d
//
// T = double gives the plain FP64 form (tol_in = rtol ||b|| / 2); T = float gives
// the mixed form (FP32 operator copy and FP32 vectors inside, tol_in =
// max(inner_rtol ||r||, rtol ||b|| / 2)).
//
// Every system keeps its own scalars; all systems advance in lock step and a
// finished system idles.  Dot products are reduced deterministically: warp
// shuffles, per-warp partials summed in warp order, per-block partials summed in
// block order by every block, so all blocks hold identical scalars.  Blocks
// meet at a grid barrier whose wait is bounded (2 s, then VIP_ERR_TIMEOUT).
#include <cstdio>
#include <cstring>
#include <vector>

#include "vip_internal.cuh"

namespace vip {

constexpr int KTHREADS = 1024;
constexpr int KWARPS = KTHREADS / 32;
constexpr int MAXSYS = 128;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i(const int* p) {
    return *(const volatile int*)p;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for a cooperative launch; returns false after a timeout.
__device__ bool grid_sync(uint32_t* bar, unsigned nblocks, int32_t* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_volatile_i(status) != VIP_ERR_TIMEOUT;
        if (ok) {
            unsigned gen = ld_acquire(bar + 1);
            __threadfence();
            unsigned arrived = atomicAdd(bar, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                uint64_t t0 = gtimer();
                while (ld_acquire(bar + 1) == gen) {
                    if (gtimer() - t0 > 2000000000ull) {
                        set_status(status, VIP_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T>
struct KArgs {
    const int64_t* sptr;
    const int32_t* width;
    const int32_t* col;
    const double* a64;
    const T* aT;
    const int32_t* slice_sys;
    const int32_t* blk_s0;
    const int32_t* blk_s1;
    const int32_t* blk_g0;
    const int32_t* blk_ng;
    const int32_t* sys_b0;
    const int32_t* sys_b1;
    double* partial;     // [nsys][NQ][nblocks], zero where a block has no rows of a system
    uint32_t* bar;
    int nsys;
    const double* b;
    double* x;
    T *r, *rhat, *p, *v, *s, *t, *dx;
    double rtol, inner_rtol;
    int max_iters, max_outer, max_pass;
    int32_t* out_iters;
    int32_t* out_outer;
    double* out_relres;
    int32_t* out_status;
    int32_t* status;
    int use_mg;          // right preconditioning by one multigrid V-cycle
    MgDev<T> mg;
    T *phat, *shat;      // M^{-1} p and M^{-1} s (alias p and s without a preconditioner)
};

struct SysState {
    double bnorm, rnorm, tol, rho, rho_old, alpha, omega, beta, rhat_norm, relres;
    int outer_active;  // still solving
    int inner_active;  // inside a BiCGSTAB pass
    int s_conv;        // ||s|| met the inner tolerance this iteration
    int zero_x;        // b == 0: set x = 0
    int pass_bad;      // the pass produced a non-finite or diverging correction: discard it
    int bad_passes;    // consecutive discarded passes
    double r0_in;      // ||r|| at the start of the pass
    int pass_cap;      // iteration cap of the current pass (halved after a discarded pass)
    int iters, outer, pass_iters, status;
};

// A reduced value is usable if finite.
__device__ __forceinline__ bool fin(double v) { return isfinite(v); }

template <class T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

// warp sum (fixed butterfly order)
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__global__ void __launch_bounds__(KTHREADS) k_bicgstab(KArgs<T> a) {
    // |r_hat . r| below this fraction of ||r_hat|| ||r|| is rounding noise in T
    // (FP32 vectors of ~1e6 rows: ~6e-8 / sqrt(n) relative noise in a dot product)
    const double bd_tol = sizeof(T) == 8 ? 1e-14 : 1e-9;
    __shared__ double sacc[KWARPS][MAXSYS_PB][NQ];
    __shared__ double stot[MAXSYS][NQ];
    __shared__ SysState S[MAXSYS];
    __shared__ int s_any;
    const int bid = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s0 = a.blk_s0[bid], s1 = a.blk_s1[bid], g0 = a.blk_g0[bid];
    const unsigned nb = gridDim.x;
    const int nsys = a.nsys;

    auto clear_acc = [&]() {
        for (int i = threadIdx.x; i < KWARPS * MAXSYS_PB * NQ; i += KTHREADS)
            (&sacc[0][0][0])[i] = 0.0;
        __syncthreads();
    };
    // accumulate a row's contributions q[0..nq) (warp-collective)
    auto acc = [&](int j, int nq, const double* q) {
        for (int k = 0; k < nq; ++k) {
            double w = wsum(q[k]);
            if (lane == 0) sacc[warp][j][k] += w;
        }
    };
    // block partials -> global, barrier, totals of every system -> stot.
    // Layout partial[(g * NQ + k) * nb + block]: the blocks of one system are a
    // contiguous run, summed by one warp (lanes stride over blocks, then a fixed
    // butterfly), so the order is fixed and the loads are independent.
    const int ng_blk = a.blk_ng[bid];
    auto reduce = [&](int nq) -> bool {
        __syncthreads();
        for (int i = threadIdx.x; i < ng_blk * nq; i += KTHREADS) {
            int j = i / nq, k = i % nq;
            double sum = 0.0;
            for (int w = 0; w < KWARPS; ++w) sum += sacc[w][j][k];
            __stcg(&a.partial[((int64_t)(g0 + j) * NQ + k) * nb + bid], sum);
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int i = warp; i < nsys * nq; i += KWARPS) {
            int g = i / nq, k = i % nq;
            const double* src = a.partial + ((int64_t)g * NQ + k) * nb;
            double sum = 0.0;
            for (int bb = a.sys_b0[g] + lane; bb < a.sys_b1[g]; bb += 32) sum += __ldcg(src + bb);
            sum = wsum(sum);
            if (lane == 0) stot[g][k] = sum;
        }
        __syncthreads();
        return true;
    };
    auto any_of = [&](int which) {
        if (threadIdx.x == 0) {
            int any = 0;
            for (int g = 0; g < nsys; ++g) any |= which ? S[g].inner_active : S[g].outer_active;
            s_any = any;
        }
        __syncthreads();
        return s_any != 0;
    };
    // y_row = sum_k A[row,k] * vec[col] for the warp's slice (lane = row)
    auto spmv_row = [&](int64_t sl, const auto* A, const auto* vec) -> double {
        int64_t base = a.sptr[sl] + lane;
        int w = a.width[sl];
        double sum = 0.0;
        for (int k = 0; k < w; ++k) {
            int64_t e = base + (int64_t)k * 32;
            sum += (double)__ldg(A + e) * (double)ldv(vec + __ldg(a.col + e));
        }
        return sum;
    };

    // One V-cycle z = M^{-1} v of the aggregation multigrid: damped Jacobi from zero on
    // the fine rows, fine residual, restriction (sum over the cell's rows), then on each
    // coarse level a Jacobi step from zero, its residual and restriction; Jacobi sweeps
    // on the coarsest level by block 0; back up with piecewise-constant prolongation
    // and one Jacobi post-smoothing step per level.  Only rows of systems still in
    // their inner pass are touched on the fine level.
    const int64_t gtid = (int64_t)blockIdx.x * KTHREADS + threadIdx.x;
    const int64_t gstride = (int64_t)nb * KTHREADS;
    auto coarse_res = [&](int l, int64_t c, const T* xv) -> double {
        const MgDev<T>& M = a.mg;
        const int64_t n = M.n[l];
        double acc = (double)ldv(M.b[l] + c);
        for (int o = 0; o < 25; ++o) {
            int32_t j = __ldg(M.nbr[l] + (int64_t)o * n + c);
            if (j >= 0) acc -= (double)__ldg(M.coef[l] + (int64_t)o * n + c) * (double)ldv(xv + j);
        }
        return acc;
    };
    auto vcycle = [&](const T* in, T* out) -> bool {
        const MgDev<T>& M = a.mg;
        const double w = M.omega;
        const int L = M.nlev;
        for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
            int g = a.slice_sys[sl];
            int64_t row = (int64_t)sl * 32 + lane;
            T z = (T)0;
            if (S[g].inner_active) z = (T)(w * (double)__ldg(M.fdinv + row) * (double)ldv(in + row));
            M.fx[row] = z;
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
            int g = a.slice_sys[sl];
            int64_t row = (int64_t)sl * 32 + lane;
            T res = (T)0;
            if (S[g].inner_active) res = (T)((double)ldv(in + row) - spmv_row(sl, a.aT, M.fx));
            M.fr[row] = res;
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int64_t c = gtid; c < M.n[1]; c += gstride) {
            double sum = 0.0;
            for (int64_t q = __ldg(M.cptr + c); q < __ldg(M.cptr + c + 1); ++q)
                sum += (double)ldv(M.fr + __ldg(M.crow + q));
            M.b[1][c] = (T)sum;
            M.x[1][c] = (T)(w * (double)__ldg(M.dinv[1] + c) * sum);
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int l = 1; l < L; ++l) {
            for (int64_t c = gtid; c < M.n[l]; c += gstride) M.y[l][c] = (T)coarse_res(l, c, M.x[l]);
            if (!grid_sync(a.bar, nb, a.status)) return false;
            const int64_t nc = M.n[l + 1];
            for (int64_t C = gtid; C < nc; C += gstride) {
                double sum = 0.0;
                for (int k = 0; k < 4; ++k) {
                    int64_t ch = __ldg(M.child[l + 1] + (int64_t)k * nc + C);
                    if (ch >= 0) sum += (double)ldv(M.y[l] + ch);
                }
                M.b[l + 1][C] = (T)sum;
                M.x[l + 1][C] = (T)(w * (double)__ldg(M.dinv[l + 1] + C) * sum);
            }
            if (!grid_sync(a.bar, nb, a.status)) return false;
        }
        // coarsest level: exact solve x_L = A_L^{-1} b_L with each geometry's dense FP64
        // inverse (one row per thread of the grid)
        for (int gg = 0; gg < M.ngeom; ++gg) {
            const int64_t c0 = __ldg(M.coff + gg);
            const int64_t m = ((gg + 1 < M.ngeom) ? __ldg(M.coff + gg + 1) : M.n[L]) - c0;
            const double* Ai = M.cinv + __ldg(M.cinv_off + gg);
            for (int64_t i = gtid; i < m; i += gstride) {
                double sum = 0.0;
                for (int64_t j = 0; j < m; ++j) sum += __ldg(Ai + i * m + j) * (double)ldv(M.b[L] + c0 + j);
                M.x[L][c0 + i] = (T)sum;
            }
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        // the corrected solution of level l is x_L on the coarsest level, y_l above it
        for (int l = L - 1; l >= 1; --l) {
            const T* sol = (l + 1 == L) ? M.x[l + 1] : M.y[l + 1];
            for (int64_t c = gtid; c < M.n[l]; c += gstride)
                M.x[l][c] = (T)((double)ldv(M.x[l] + c) +
                                (double)M.corr * (double)ldv(sol + __ldg(M.parent[l] + c)));
            if (!grid_sync(a.bar, nb, a.status)) return false;
            for (int64_t c = gtid; c < M.n[l]; c += gstride)
                M.y[l][c] = (T)((double)ldv(M.x[l] + c) +
                                w * (double)__ldg(M.dinv[l] + c) * coarse_res(l, c, M.x[l]));
            if (!grid_sync(a.bar, nb, a.status)) return false;
        }
        const T* sol1 = (L == 1) ? M.x[1] : M.y[1];
        for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
            int g = a.slice_sys[sl];
            if (!S[g].inner_active) continue;
            int64_t row = (int64_t)sl * 32 + lane;
            int32_t c = __ldg(M.agg + row);
            if (c >= 0) M.fx[row] = (T)((double)ldv(M.fx + row) + (double)M.corr * (double)ldv(sol1 + c));
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
            int g = a.slice_sys[sl];
            if (!S[g].inner_active) continue;
            int64_t row = (int64_t)sl * 32 + lane;
            double r = (double)ldv(in + row) - spmv_row(sl, a.aT, M.fx);
            out[row] = (T)((double)ldv(M.fx + row) + w * (double)__ldg(M.fdinv + row) * r);
        }
        return grid_sync(a.bar, nb, a.status);
    };

    if (threadIdx.x < nsys) {
        SysState& st = S[threadIdx.x];
        st.bnorm = -1.0; st.rnorm = 0; st.tol = 0; st.rho = st.rho_old = st.alpha = st.omega = 1.0;
        st.beta = 0; st.rhat_norm = 0; st.relres = 0;
        st.outer_active = 1; st.inner_active = 0; st.s_conv = 0; st.zero_x = 0;
        st.pass_bad = 0; st.bad_passes = 0; st.r0_in = 0; st.pass_cap = a.max_pass;
        st.iters = 0; st.outer = 0; st.pass_iters = 0; st.status = 0;
    }
    __syncthreads();

    bool alive = true;
    for (int outer = 0; alive; ++outer) {
        // ---- X: apply the correction of the previous pass
        if (outer > 0) {
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                int64_t row = (int64_t)sl * 32 + lane;
                if (S[g].zero_x) a.x[row] = 0.0;
                else if (S[g].outer_active && !S[g].pass_bad)
                    a.x[row] = __ldcg(a.x + row) + (double)ldv(a.dx + row);
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
        }
        // ---- R: FP64 residual, inner initialisation
        clear_acc();
        for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
            int g = a.slice_sys[sl];
            if (!S[g].outer_active) continue;
            int64_t row = (int64_t)sl * 32 + lane;
            double bi = __ldg(a.b + row);
            double ri = bi - spmv_row(sl, a.a64, a.x);
            T rt = (T)ri;
            a.r[row] = rt;
            a.rhat[row] = rt;
            a.p[row] = (T)0;
            a.v[row] = (T)0;
            a.dx[row] = (T)0;
            double q[3] = {ri * ri, bi * bi, (double)rt * (double)rt};
            acc(g - g0, 3, q);
        }
        if (!reduce(3)) { alive = false; break; }
        if (threadIdx.x < nsys) {
            SysState& st = S[threadIdx.x];
            if (st.outer_active) {
                if (st.bnorm < 0) st.bnorm = sqrt(stot[threadIdx.x][1]);
                st.rnorm = sqrt(stot[threadIdx.x][0]);
                st.zero_x = 0;
                st.inner_active = 0;
                if (st.bnorm == 0.0) {
                    st.relres = 0.0;
                    st.zero_x = 1;            // x = 0 solves A x = 0
                    st.outer_active = 0;
                } else {
                    st.relres = st.rnorm / st.bnorm;
                    if (!(st.relres == st.relres) || isinf(st.relres)) {
                        st.status = VIP_ERR_NONFINITE; st.outer_active = 0;
                    } else if (st.relres <= a.rtol) {
                        st.outer_active = 0;
                    } else if (st.iters >= a.max_iters || st.outer >= a.max_outer) {
                        st.status = VIP_ERR_NOT_CONVERGED; st.outer_active = 0;
                    } else if (st.outer > 0 && st.pass_iters == 0 && !st.pass_bad) {
                        st.status = VIP_ERR_BREAKDOWN; st.outer_active = 0;
                    } else if (st.bad_passes >= 3) {
                        st.status = VIP_ERR_NONFINITE; st.outer_active = 0;
                    } else {
                        st.inner_active = 1;
                        st.outer += 1;
                        double t_abs = 0.5 * a.rtol * st.bnorm;
                        st.tol = (sizeof(T) == 8) ? t_abs : fmax(a.inner_rtol * st.rnorm, t_abs);
                        st.rho = stot[threadIdx.x][2];
                        st.rhat_norm = sqrt(st.rho);
                        st.r0_in = st.rhat_norm;
                        st.rho_old = st.alpha = st.omega = 1.0;
                        st.bad_passes = st.pass_bad ? st.bad_passes + 1 : 0;
                        st.pass_cap = st.pass_bad ? max(st.pass_iters / 2, 20)
                                                  : min(2 * st.pass_cap, a.max_pass);
                        st.pass_bad = 0;
                        st.pass_iters = 0;
                    }
                }
            }
        }
        __syncthreads();
        bool any_zero = false;
        if (threadIdx.x == 0) {
            int z = 0;
            for (int g = 0; g < nsys; ++g) z |= S[g].zero_x;
            s_any = z;
        }
        __syncthreads();
        any_zero = s_any != 0;
        if (!any_of(0)) {
            if (any_zero) {  // final zeroing pass
                for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                    int g = a.slice_sys[sl];
                    if (S[g].zero_x) a.x[(int64_t)sl * 32 + lane] = 0.0;
                }
            }
            break;
        }

        // ---- inner BiCGSTAB pass
        while (any_of(1)) {
            // A: beta, p = r + beta (p - omega v)
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                if (st.inner_active) st.beta = (st.rho / st.rho_old) * (st.alpha / st.omega);
            }
            __syncthreads();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                double pn = (double)ldv(a.r + row) +
                            S[g].beta * ((double)ldv(a.p + row) - S[g].omega * (double)ldv(a.v + row));
                a.p[row] = (T)pn;
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
            if (a.use_mg && !vcycle(a.p, a.phat)) { alive = false; break; }
            // B: v = A phat, rhat . v
            clear_acc();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                double vi = spmv_row(sl, a.aT, a.phat);
                a.v[row] = (T)vi;
                double q[2] = {(double)ldv(a.rhat + row) * (double)(T)vi, (double)(T)vi * (double)(T)vi};
                acc(g - g0, 2, q);
            }
            if (!reduce(2)) { alive = false; break; }
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                if (st.inner_active) {
                    double rv = stot[threadIdx.x][0];
                    if (!fin(rv) || !fin(stot[threadIdx.x][1])) {
                        st.inner_active = 0;
                        st.pass_bad = 1;
                    } else if (!(fabs(rv) > bd_tol * st.rhat_norm * sqrt(stot[threadIdx.x][1]))) {
                        st.inner_active = 0;  // restart from the current x
                    } else {
                        st.alpha = st.rho / rv;
                    }
                }
            }
            __syncthreads();
            // C: s = r - alpha v
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                a.s[row] = (T)((double)ldv(a.r + row) - S[g].alpha * (double)ldv(a.v + row));
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
            if (a.use_mg && !vcycle(a.s, a.shat)) { alive = false; break; }
            // D: t = A shat; t.s, t.t, s.s
            clear_acc();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                T ti = (T)spmv_row(sl, a.aT, a.shat);
                a.t[row] = ti;
                double si = (double)ldv(a.s + row);
                double q[3] = {(double)ti * si, (double)ti * (double)ti, si * si};
                acc(g - g0, 3, q);
            }
            if (!reduce(3)) { alive = false; break; }
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                st.s_conv = 0;
                if (st.inner_active) {
                    st.iters += 1;
                    st.pass_iters += 1;
                    double ts = stot[threadIdx.x][0], tt = stot[threadIdx.x][1];
                    if (!fin(ts) || !fin(tt) || !fin(stot[threadIdx.x][2])) {
                        st.s_conv = 1;      // stop the pass after E and discard it
                        st.omega = 0.0;
                        st.pass_bad = 1;
                    } else if (sqrt(stot[threadIdx.x][2]) <= st.tol || tt == 0.0) {
                        st.s_conv = 1;
                        st.omega = 0.0;
                    } else {
                        st.omega = ts / tt;
                    }
                }
            }
            __syncthreads();
            // E: d += alpha p + omega s; r = s - omega t; rhat.r, r.r
            clear_acc();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                double al = S[g].alpha, om = S[g].omega;
                double si = (double)ldv(a.s + row);
                double d = (double)ldv(a.dx + row) + al * (double)ldv(a.phat + row) +
                           om * (double)ldv(a.shat + row);
                a.dx[row] = (T)d;
                T rn = (T)(si - om * (double)ldv(a.t + row));
                a.r[row] = rn;
                double q[2] = {(double)ldv(a.rhat + row) * (double)rn, (double)rn * (double)rn};
                acc(g - g0, 2, q);
            }
            if (!reduce(2)) { alive = false; break; }
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                if (st.inner_active) {
                    double rho = stot[threadIdx.x][0], rr = sqrt(stot[threadIdx.x][1]);
                    if (!fin(rho) || !fin(rr) || rr > 1e8 * st.r0_in) {
                        st.inner_active = 0;  // diverging in precision T: discard the pass
                        st.pass_bad = 1;
                    } else if (st.s_conv || rr <= st.tol || st.omega == 0.0 || st.iters >= a.max_iters ||
                               st.pass_iters >= st.pass_cap) {
                        st.inner_active = 0;
                    } else if (!(fabs(rho) > bd_tol * st.rhat_norm * rr)) {
                        st.inner_active = 0;  // restart
                    } else {
                        st.rho_old = st.rho;
                        st.rho = rho;
                    }
                }
            }
            __syncthreads();
        }
        if (!alive) break;
    }
    if (bid == 0 && threadIdx.x < nsys) {
        SysState& st = S[threadIdx.x];
        a.out_iters[threadIdx.x] = st.iters;
        a.out_outer[threadIdx.x] = st.outer;
        a.out_relres[threadIdx.x] = st.relres;
        a.out_status[threadIdx.x] = st.status;
        if (st.status) set_status(a.status, st.status);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
vip_status krylov_plan(vip_ctx* c, KrylovPlan& P, const Sell& A, const std::vector<int64_t>& row0,
                       const std::vector<int64_t>& rows) {
    const int nsys = (int)row0.size();
    if (nsys > MAXSYS) {
        c->err = "too many systems in one Krylov batch (limit 128)";
        return VIP_ERR_ARG;
    }
    int occ64 = 0, occ32 = 0;
    VIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_bicgstab<double>, KTHREADS, 0));
    VIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_bicgstab<float>, KTHREADS, 0));
    int occ = std::max(1, std::min(std::min(occ64, occ32), 1));
    const int64_t nsl = A.nslices;
    std::vector<int32_t> slice_sys(nsl, -1);
    for (int g = 0; g < nsys; ++g) {
        if (row0[g] % SLICE || rows[g] % SLICE) { c->err = "unaligned system"; return VIP_ERR_ARG; }
        for (int64_t s = row0[g] / SLICE; s < (row0[g] + rows[g]) / SLICE; ++s) slice_sys[s] = g;
    }
    for (int64_t s = 0; s < nsl; ++s)
        if (slice_sys[s] < 0) { c->err = "slice without system"; return VIP_ERR_ARG; }
    // contiguous slice chunks, one per block; a block may touch MAXSYS_PB systems
    int nb = std::max(1, c->num_sms * occ);
    nb = (int)std::min<int64_t>(nb, nsl);
    std::vector<int32_t> bs0(nb), bs1(nb), bg0(nb), bng(nb);
    std::vector<int32_t> sb0(nsys, 1 << 30), sb1(nsys, -1);
    for (int b = 0; b < nb; ++b) {
        bs0[b] = (int32_t)(nsl * b / nb);
        bs1[b] = (int32_t)(nsl * (b + 1) / nb);
        int ga = slice_sys[bs0[b]], gb = slice_sys[bs1[b] - 1];
        bg0[b] = ga;
        bng[b] = gb - ga + 1;
        if (bng[b] > MAXSYS_PB) { c->err = "a block spans too many systems"; return VIP_ERR_ARG; }
        for (int g = ga; g <= gb; ++g) {
            sb0[g] = std::min(sb0[g], b);
            sb1[g] = std::max(sb1[g], b + 1);
        }
    }
    P.nblocks = nb;
    P.nthreads = KTHREADS;
    P.nsys = nsys;
    P.nslices = nsl;
    VIP_CUDA(dalloc(c, &P.slice_sys, nsl));
    VIP_CUDA(dalloc(c, &P.blk_s0, nb)); VIP_CUDA(dalloc(c, &P.blk_s1, nb));
    VIP_CUDA(dalloc(c, &P.blk_g0, nb)); VIP_CUDA(dalloc(c, &P.blk_ng, nb));
    VIP_CUDA(dalloc(c, &P.sys_b0, nsys)); VIP_CUDA(dalloc(c, &P.sys_b1, nsys));
    VIP_CUDA(dalloc(c, &P.partial, (size_t)nb * nsys * NQ));
    VIP_CUDA(cudaMemsetAsync(P.partial, 0, (size_t)nb * nsys * NQ * sizeof(double), c->stream));
    VIP_CUDA(dalloc(c, &P.flags, nb));
    VIP_CUDA(dalloc(c, &P.bar, 2));
    VIP_CUDA(dalloc(c, &P.out_iters, nsys)); VIP_CUDA(dalloc(c, &P.out_outer, nsys));
    VIP_CUDA(dalloc(c, &P.out_relres, nsys)); VIP_CUDA(dalloc(c, &P.out_status, nsys));
    cudaStream_t st = c->stream;
    VIP_CUDA(cudaMemcpyAsync(P.slice_sys, slice_sys.data(), nsl * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.blk_s0, bs0.data(), nb * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.blk_s1, bs1.data(), nb * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.blk_g0, bg0.data(), nb * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.blk_ng, bng.data(), nb * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.sys_b0, sb0.data(), nsys * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(P.sys_b1, sb1.data(), nsys * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    return VIP_OK;
}

template <class T>
static MgDev<T> mg_view(const Multigrid& M) {
    MgDev<T> d;
    memset(&d, 0, sizeof(d));
    const bool f32 = sizeof(T) == 4;
    d.nlev = M.nlev;
    d.agg = M.agg; d.cptr = M.cptr; d.crow = M.crow;
    d.fdinv = f32 ? (const T*)M.fdinv32 : (const T*)M.fdinv;
    d.fr = (T*)M.fr; d.fx = (T*)M.fx;
    for (int l = 1; l <= M.nlev; ++l) {
        const MgLevel& v = M.lev[l];
        d.n[l] = v.n; d.nbr[l] = v.nbr; d.parent[l] = v.parent; d.child[l] = v.child;
        d.coef[l] = f32 ? (const T*)v.coef32 : (const T*)v.coef;
        d.dinv[l] = f32 ? (const T*)v.dinv32 : (const T*)v.dinv;
        d.x[l] = (T*)v.x; d.b[l] = (T*)v.b; d.y[l] = (T*)v.y;
    }
    d.omega = 0.8f;
    d.corr = 1.5f;
    d.cinv = M.cinv;
    d.cinv_off = M.cinv_off;
    d.coff = M.lev[M.nlev].off;
    d.ngeom = M.ngeom;
    return d;
}

template <class T>
static vip_status launch(vip_ctx* c, const KrylovPlan& P, const Sell& A, const double* b, double* x,
                         double rtol, int32_t max_iters, double inner_rtol, const Multigrid* mg) {
    KrylovWork& W = sizeof(T) == 8 ? c->work64 : c->work32;
    if (W.n < A.nrows) { c->err = "Krylov workspace too small"; return VIP_ERR_ARG; }
    KArgs<T> a;
    a.sptr = A.sptr; a.width = A.width; a.col = A.col; a.a64 = A.v64;
    a.aT = sizeof(T) == 8 ? (const T*)A.v64 : (const T*)A.v32;
    a.slice_sys = P.slice_sys; a.blk_s0 = P.blk_s0; a.blk_s1 = P.blk_s1; a.blk_g0 = P.blk_g0;
    a.blk_ng = P.blk_ng;
    a.sys_b0 = P.sys_b0; a.sys_b1 = P.sys_b1; a.partial = P.partial; a.bar = P.bar;
    a.nsys = P.nsys; a.b = b; a.x = x;
    a.r = (T*)W.r; a.rhat = (T*)W.rhat; a.p = (T*)W.p; a.v = (T*)W.v; a.s = (T*)W.s;
    a.t = (T*)W.t; a.dx = (T*)W.dx;
    a.rtol = rtol; a.inner_rtol = inner_rtol; a.max_iters = max_iters;
    // FP32 passes are re-anchored on the FP64 residual at least every 4000 iterations
    a.max_outer = 1000;
    a.max_pass = sizeof(T) == 8 ? max_iters : 4000;
    a.out_iters = P.out_iters; a.out_outer = P.out_outer; a.out_relres = P.out_relres;
    a.out_status = P.out_status; a.status = c->d_status;
    a.use_mg = (mg && mg->built) ? 1 : 0;
    if (a.use_mg) {
        a.mg = mg_view<T>(*mg);
        a.phat = (T*)c->phat;
        a.shat = (T*)c->shat;
    } else {
        memset(&a.mg, 0, sizeof(a.mg));
        a.phat = a.p;
        a.shat = a.s;
    }
    VIP_CUDA(cudaMemsetAsync(P.bar, 0, 2 * sizeof(uint32_t), c->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.nblocks);
    cfg.blockDim = dim3(P.nthreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    VIP_CUDA(cudaLaunchKernelEx(&cfg, k_bicgstab<T>, a));
    return VIP_OK;
}

vip_status krylov_solve(vip_ctx* c, const KrylovPlan& P, const Sell& A, const double* b, double* x,
                        int precision, double rtol, int32_t max_iters, double inner_rtol,
                        const Multigrid* mg) {
    if (precision == VIP_PREC_MIXED)
        return launch<float>(c, P, A, b, x, rtol, max_iters, inner_rtol, mg);
    return launch<double>(c, P, A, b, x, rtol, max_iters, inner_rtol, mg);
}

}  // namespace vip
