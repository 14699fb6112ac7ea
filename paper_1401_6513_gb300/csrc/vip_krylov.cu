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
#include <vector>

#include "vip_internal.cuh"

namespace vip {

constexpr int KTHREADS = 512;
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
    const int32_t* sys_b0;
    const int32_t* sys_b1;
    double* partial;
    uint32_t* bar;
    int nsys;
    const double* b;
    double* x;
    T *r, *rhat, *p, *v, *s, *t, *dx;
    double rtol, inner_rtol;
    int max_iters, max_outer;
    int32_t* out_iters;
    int32_t* out_outer;
    double* out_relres;
    int32_t* out_status;
    int32_t* status;
};

struct SysState {
    double bnorm, rnorm, tol, rho, rho_old, alpha, omega, beta, rhat_norm, relres;
    int outer_active;  // still solving
    int inner_active;  // inside a BiCGSTAB pass
    int s_conv;        // ||s|| met the inner tolerance this iteration
    int zero_x;        // b == 0: set x = 0
    int iters, outer, pass_iters, status;
};

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
    // block partials -> global, barrier, totals of every system -> stot
    auto reduce = [&](int nq) -> bool {
        __syncthreads();
        for (int i = threadIdx.x; i < MAXSYS_PB * nq; i += KTHREADS) {
            int j = i / nq, k = i % nq;
            double sum = 0.0;
            for (int w = 0; w < KWARPS; ++w) sum += sacc[w][j][k];
            __stcg(&a.partial[((int64_t)bid * MAXSYS_PB + j) * NQ + k], sum);
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int i = threadIdx.x; i < nsys * nq; i += KTHREADS) {
            int g = i / nq, k = i % nq;
            double sum = 0.0;
            for (int bb = a.sys_b0[g]; bb < a.sys_b1[g]; ++bb)
                sum += __ldcg(&a.partial[((int64_t)bb * MAXSYS_PB + (g - a.blk_g0[bb])) * NQ + k]);
            stot[g][k] = sum;
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

    if (threadIdx.x < nsys) {
        SysState& st = S[threadIdx.x];
        st.bnorm = -1.0; st.rnorm = 0; st.tol = 0; st.rho = st.rho_old = st.alpha = st.omega = 1.0;
        st.beta = 0; st.rhat_norm = 0; st.relres = 0;
        st.outer_active = 1; st.inner_active = 0; st.s_conv = 0; st.zero_x = 0;
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
                else if (S[g].outer_active) a.x[row] = __ldcg(a.x + row) + (double)ldv(a.dx + row);
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
                    } else if (st.outer > 0 && st.pass_iters == 0) {
                        st.status = VIP_ERR_BREAKDOWN; st.outer_active = 0;
                    } else {
                        st.inner_active = 1;
                        st.outer += 1;
                        st.pass_iters = 0;
                        double t_abs = 0.5 * a.rtol * st.bnorm;
                        st.tol = (sizeof(T) == 8) ? t_abs : fmax(a.inner_rtol * st.rnorm, t_abs);
                        st.rho = stot[threadIdx.x][2];
                        st.rhat_norm = sqrt(st.rho);
                        st.rho_old = st.alpha = st.omega = 1.0;
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
            // B: v = A p, rhat . v
            clear_acc();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                double vi = spmv_row(sl, a.aT, a.p);
                a.v[row] = (T)vi;
                double q[2] = {(double)ldv(a.rhat + row) * (double)(T)vi, (double)(T)vi * (double)(T)vi};
                acc(g - g0, 2, q);
            }
            if (!reduce(2)) { alive = false; break; }
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                if (st.inner_active) {
                    double rv = stot[threadIdx.x][0];
                    if (!(fabs(rv) > 1e-12 * st.rhat_norm * sqrt(stot[threadIdx.x][1]))) {
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
            // D: t = A s; t.s, t.t, s.s
            clear_acc();
            for (int sl = s0 + warp; sl < s1; sl += KWARPS) {
                int g = a.slice_sys[sl];
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                T ti = (T)spmv_row(sl, a.aT, a.s);
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
                    if (sqrt(stot[threadIdx.x][2]) <= st.tol || tt == 0.0) {
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
                double d = (double)ldv(a.dx + row) + al * (double)ldv(a.p + row) + om * si;
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
                    if (st.s_conv || rr <= st.tol || st.omega == 0.0 || st.iters >= a.max_iters) {
                        st.inner_active = 0;
                    } else if (!(fabs(rho) > 1e-12 * st.rhat_norm * rr)) {
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
    int occ = std::max(1, std::min(std::min(occ64, occ32), 2));
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
    VIP_CUDA(dalloc(c, &P.partial, (size_t)nb * MAXSYS_PB * NQ));
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
static vip_status launch(vip_ctx* c, const KrylovPlan& P, const Sell& A, const double* b, double* x,
                         double rtol, int32_t max_iters, double inner_rtol) {
    KrylovWork& W = sizeof(T) == 8 ? c->work64 : c->work32;
    if (W.n < A.nrows) { c->err = "Krylov workspace too small"; return VIP_ERR_ARG; }
    KArgs<T> a;
    a.sptr = A.sptr; a.width = A.width; a.col = A.col; a.a64 = A.v64;
    a.aT = sizeof(T) == 8 ? (const T*)A.v64 : (const T*)A.v32;
    a.slice_sys = P.slice_sys; a.blk_s0 = P.blk_s0; a.blk_s1 = P.blk_s1; a.blk_g0 = P.blk_g0;
    a.sys_b0 = P.sys_b0; a.sys_b1 = P.sys_b1; a.partial = P.partial; a.bar = P.bar;
    a.nsys = P.nsys; a.b = b; a.x = x;
    a.r = (T*)W.r; a.rhat = (T*)W.rhat; a.p = (T*)W.p; a.v = (T*)W.v; a.s = (T*)W.s;
    a.t = (T*)W.t; a.dx = (T*)W.dx;
    a.rtol = rtol; a.inner_rtol = inner_rtol; a.max_iters = max_iters; a.max_outer = 200;
    a.out_iters = P.out_iters; a.out_outer = P.out_outer; a.out_relres = P.out_relres;
    a.out_status = P.out_status; a.status = c->d_status;
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
                        int precision, double rtol, int32_t max_iters, double inner_rtol) {
    if (precision == VIP_PREC_MIXED)
        return launch<float>(c, P, A, b, x, rtol, max_iters, inner_rtol);
    return launch<double>(c, P, A, b, x, rtol, max_iters, inner_rtol);
}

}  // namespace vip
