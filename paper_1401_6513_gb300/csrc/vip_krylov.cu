// Krylov solves of Eqs. (12) and (13): one persistent cooperative launch solves a
// batch of independent sparse systems (block-diagonal SELL-32 operator, each
// system a contiguous range of slices) with BiCGSTAB (van der Vorst, 1992),
// right-preconditioned by one V-cycle of the aggregation multigrid for Eq. (13),
// inside an FP64 iterative-refinement loop:
//
//   repeat:  r = b - A x   (FP64 operator, FP64 vectors);  stop if ||r|| <= rtol ||b||
//            solve A d = r by BiCGSTAB in precision T from d = 0 with r_hat = r,
//            until ||r_d|| <= tol_in, or until |r_hat.r| or |r_hat.v| falls below
//            a small fraction of its norms (restart);   x += d
//
// Two precisions: T for the Krylov vectors, operator applications and vector
// updates, TM for the V-cycle (its vectors, operators and arithmetic).
//   <double, double>  the plain FP64 form (tol_in = rtol ||b|| / 2: one pass);
//   <float, float>    the mixed form: FP32 arithmetic on FP32 copies of the
//                     operators and FP32 vectors inside, tol_in =
//                     max(inner_rtol ||r||, rtol ||b|| / 2), the correction d
//                     accumulated as an FP32 (hi, lo) pair by error-free
//                     transformations (no FP64 operation per row inside);
//   <double, float>   FP64 Krylov iteration with an FP32 V-cycle.
// FP32 applications of the fine operator use the differenced row form
// sum_k a_ik (x_k - x_i) + rowsum_i x_i with the FP64 row sum rounded to FP32: on
// the smooth vectors of a Poisson solve x_k - x_i is small and exact, so the
// large, nearly cancelling products a_ik x_k of the plain form never appear.
//
// Every system keeps its own scalars; all systems advance in lock step, and the
// slices of the systems still iterating are re-spread over all blocks whenever a
// system finishes.  Dot products are reduced deterministically: per-lane sums in
// registers, warp shuffles, per-warp partials summed in warp order, per-block
// partials summed in block order by every block, so all blocks hold identical
// scalars.  Blocks meet at a grid barrier whose wait is bounded (2 s, then
// VIP_ERR_TIMEOUT).
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "vip_internal.cuh"

namespace vip {

constexpr int KTHREADS = 1024;
constexpr int KWARPS = KTHREADS / 32;
constexpr int MAXSYS = 128;
constexpr int KSMEM_DYN = 36 * 36 * (int)sizeof(double);  // a coarse tile and its halo

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

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid barrier for a cooperative launch; returns false after a timeout.
// bar[0] is an arrival counter whose top bit flips once per barrier: thread 0 of
// CTA 0 adds 2^31 - (nblocks - 1), every other CTA adds 1, so the counter moves by
// exactly 2^31 per barrier and its top bit changes precisely when the last CTA has
// arrived (partial sums stay below the next multiple of 2^31).  Each CTA polls the
// same word until its top bit differs from the value it saw when arriving, so no
// separate release store has to travel after the last arrival.  The arrival is an
// acquire-release add and the poll an acquire load: every write before the barrier
// happens before every read after it, for weak loads too.  The counter must start
// at 0.  A wait gives up after 2 s (VIP_ERR_TIMEOUT), or early when another CTA has
// already reported a timeout.
__device__ bool grid_sync(uint32_t* bar, unsigned nblocks, int32_t* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
        const unsigned old = atom_add_acq_rel(bar, add);
        const uint64_t t0 = gtimer();
        for (unsigned k = 1; ((ld_acquire(bar) ^ old) & 0x80000000u) == 0; ++k) {
            if ((k & 63u) == 0 && (ld_volatile_i(status) == VIP_ERR_TIMEOUT || gtimer() - t0 > 2000000000ull)) {
                set_status(status, VIP_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T, class TM>
struct KArgs {
    const int64_t* sptr;
    const int32_t* width;
    const int32_t* col;
    const double* a64;      // FP64 operator (refinement residual)
    const T* aT;            // the operator in T (Krylov applications)
    const TM* aM;           // the operator in TM (the V-cycle's fine level)
    const int64_t* ucptr;   // uniform slices (null: none)
    const int32_t* ucode;
    const double* u64;
    const T* uT;
    const TM* uM;
    const float* rs32;      // FP64 row sums rounded to FP32 (FP32 differenced rows)
    const int32_t* slice_sys;
    const int32_t* blk_s0;
    const int32_t* blk_s1;
    const int32_t* blk_g0;
    const int32_t* blk_ng;
    const int32_t* sys_b0;
    const int32_t* sys_b1;
    const int32_t* sys_s0;   // [nsys] first slice of each system
    const int32_t* sys_s1;   // [nsys] one past its last slice
    double* partial;     // [2][nsys][NQ][nblocks], zero where a block has no rows of a system
    uint32_t* bar;
    int nsys;
    const double* b;
    double* x;
    double* dx;          // the pass's correction: FP64, or an FP32 (hi, lo) pair per row in the
                         // FP32 iteration (the same 8 bytes), accumulated without rounding loss
    T *r, *rhat, *p, *v, *s, *t;
    double rtol, inner_rtol;
    int max_iters, max_outer, max_pass;
    int32_t* out_iters;
    int32_t* out_outer;
    double* out_relres;
    int32_t* out_status;
    int32_t* status;
    int use_mg;          // right preconditioning by one multigrid V-cycle
    MgDev<TM> mg;
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
    float alpha_f, omega_f, beta_f;  // the scalars rounded to FP32 (FP32 vector updates)
};

// the scalar of precision T: the FP64 value, or its FP32 rounding
template <class T>
__device__ __forceinline__ T sc(double d, float f);
template <>
__device__ __forceinline__ double sc<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float sc<float>(double, float f) { return f; }

// A reduced value is usable if finite.
__device__ __forceinline__ bool fin(double v) { return isfinite(v); }

// Loads of vectors that the launch itself writes: plain (weak) global loads, which
// may hit in L1.  They are ordered after the writes of the previous phase by the
// grid barrier (a GPU-scope acquire in thread 0, then a CTA barrier), which the
// memory model requires to make those writes visible to weak loads; the
// non-coherent read-only path (__ldg) is used only for data no phase writes.
template <class T>
__device__ __forceinline__ T ldv(const T* p) { return *p; }

// Operator entries are streamed once per pass: evict-first, so they do not push the
// gathered vectors out of the caches.
template <class T>
__device__ __forceinline__ T ldm(const T* p) { return __ldcs(p); }

// warp sum (fixed butterfly order)
template <class V>
__device__ __forceinline__ V wsum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum_k A[row, k] f(col[row, k]) over the SELL entries of one row (lane of the
// slice's warp), in entry order, in precision TA.  DIFF: the differenced form
// sum_k A[row, k] (f(col) - xi) + rs xi, xi the row's own value and rs its row
// sum (FP32 applications of the fine operator).  The column indices and values of
// U entries are loaded before their U gathers, so each warp keeps several loads in
// flight.  A uniform slice (ucptr[sl] >= 0, warp-uniform) reads its single stored
// stencil instead (the same values and columns, so the same sum): one broadcast
// load per entry for the whole warp in place of 32 value and 32 column loads.
template <int U, bool DIFF, class TA, class F>
__device__ __forceinline__ TA sell_row(const int64_t* __restrict__ sptr,
                                       const int32_t* __restrict__ width,
                                       const int32_t* __restrict__ col, const TA* __restrict__ A,
                                       const int64_t* __restrict__ ucptr,
                                       const int32_t* __restrict__ ucode,
                                       const TA* __restrict__ uA, int64_t sl, int lane, TA xi, TA rs,
                                       F&& f) {
    const int w = __ldg(width + sl);
    TA sum = (TA)0;
    int k = 0;
    const int64_t up = ucptr ? __ldg(ucptr + sl) : -1;
    if (up >= 0) {
        const int32_t row = (int32_t)(sl * SLICE + lane);
        const int32_t* uc = ucode + up;
        const TA* ua = uA + up;
        for (; k + U <= w; k += U) {
            int c[U];
            TA av[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t code = __ldg(uc + k + u);
                c[u] = (code & 1) ? (code >> 1) : row + (code >> 1);
                av[u] = __ldg(ua + k + u);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xv[u] = f(c[u]);
                if (DIFF) xv[u] -= xi;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) sum += av[u] * xv[u];
        }
        for (; k < w; ++k) {
            const int32_t code = __ldg(uc + k);
            TA xk = f((code & 1) ? (code >> 1) : row + (code >> 1));
            if (DIFF) xk -= xi;
            sum += __ldg(ua + k) * xk;
        }
        if (DIFF) sum += rs * xi;
        return sum;
    }
    const int64_t base = __ldg(sptr + sl) + lane;
    for (; k + U <= w; k += U) {
        int c[U];
        TA av[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = base + (int64_t)(k + u) * SLICE;
            c[u] = ldm(col + e);
            av[u] = ldm(A + e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xv[u] = f(c[u]);
            if (DIFF) xv[u] -= xi;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) sum += av[u] * xv[u];
    }
    for (; k < w; ++k) {
        const int64_t e = base + (int64_t)k * SLICE;
        TA xk = f(ldm(col + e));
        if (DIFF) xk -= xi;
        sum += ldm(A + e) * xk;
    }
    if (DIFF) sum += rs * xi;
    return sum;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA; p 16-byte aligned, bytes a multiple
// of 16).  A hint: no register receives data and nothing waits for it.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Error-free FP32 transformations (Knuth's TwoSum; the product's rounding error
// by one fused multiply-add).  The _rn intrinsics are never contracted into a
// fused multiply-add, which would change the rounding these formulas rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += al * ph + om * sh with FP32 operations only: the two products are
// split exactly into rounded value and error, the rounded values are added to hi
// by TwoSum, and every error term goes into lo; the pair is then renormalised.
// The pair carries the sum to about 2^-44 of its size, so the correction of a
// refinement pass keeps the digits an FP64 accumulator would.
__device__ __forceinline__ float2 dd_axpy2(float2 d, float al, float ph, float om, float sh) {
    const float p1 = __fmul_rn(al, ph), e1 = fmaf(al, ph, -p1);
    const float p2 = __fmul_rn(om, sh), e2 = fmaf(om, sh, -p2);
    float s1, t1, s2, t2;
    two_sum(d.x, p1, s1, t1);
    two_sum(s1, p2, s2, t2);
    const float lo = __fadd_rn(d.y, __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(e1, e2)));
    const float hi = __fadd_rn(s2, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s2)));
}

// Work partition of one block of the Krylov launch (see k_bicgstab): this block's
// slices are nv "virtual" slices in nseg segments, segment k being the slices
// segs[k] + [0, segv[k+1] - segv[k]); its dot-product slots j < ng belong to systems
// sys[j] (j[g] = slot of system g, -1 if none); the partials of system g come from
// blocks [b0[g], b1[g]).
struct Partition {
    int nv, nseg, ng, valid;
    int mixed;                     // 1: the static partition (a segment may span systems)
    int segv[MAXSYS_PB + 1], segs[MAXSYS_PB];
    int b0[MAXSYS], b1[MAXSYS], j[MAXSYS], sys[MAXSYS_PB];
    int ss0[MAXSYS], ss1[MAXSYS];  // slices [ss0[g], ss1[g]) of system g
    uint32_t mask[MAXSYS / 32];    // the set the partition was made for
};

// Recomputes block bid's partition for the systems flagged in S (inner: inside a
// BiCGSTAB pass; else solving or to be zeroed) if that set changed.  The slices of
// those systems are spread evenly over all nb blocks; every block computes the
// whole partition from the same states, so all blocks agree without communicating.
// A block holds one segment per active system in its range (finished systems in
// between are passed over) and reduces only for those systems.  A partition in
// which some block would hold more than MAXSYS_PB active systems is replaced by
// the launch's static one (one segment of all the block's slices).  Run by one
// thread; kept out of line, as it runs only when a system finishes.
__device__ __noinline__ void partition_update(Partition& P, const SysState* S, int nsys, int inner,
                                              int nb, int bid, const int32_t* blk_s0,
                                              const int32_t* blk_s1, const int32_t* blk_g0,
                                              const int32_t* blk_ng, const int32_t* sys_b0,
                                              const int32_t* sys_b1) {
    uint32_t m[MAXSYS / 32];
    for (int w = 0; w < MAXSYS / 32; ++w) m[w] = 0;
    for (int g = 0; g < nsys; ++g) {
        const bool on = inner ? S[g].inner_active : (S[g].outer_active || S[g].zero_x);
        if (on) m[g >> 5] |= 1u << (g & 31);
    }
    bool same = P.valid != 0;
    for (int w = 0; w < MAXSYS / 32; ++w) same = same && m[w] == P.mask[w];
    if (!same) {
        auto on = [&](int g) { return ((m[g >> 5] >> (g & 31)) & 1u) != 0; };
        auto len = [&](int g) -> int64_t { return on(g) ? (int64_t)(P.ss1[g] - P.ss0[g]) : 0; };
        int64_t W = 0;
        for (int g = 0; g < nsys; ++g) W += len(g);
        for (int g = 0; g < nsys; ++g) { P.b0[g] = 0; P.b1[g] = 0; P.j[g] = -1; }
        P.nv = P.nseg = P.ng = 0;
        P.segv[0] = 0;
        bool ok = true;
        int gl = 0, gh = 0;
        int64_t cl = 0, ch = 0;  // active slices of the systems before gl, gh
        // block b takes the active slices [W b / nb, W (b + 1) / nb); a block
        // with none (fewer active slices than blocks) holds an empty range
        // of the active system at its position, for which it reduces a zero,
        // so that the blocks listed for a system are exactly those that
        // write its partials
        for (int b = 0; b < nb && ok && W > 0; ++b) {
            const int64_t lo = W * b / nb, hi = W * (b + 1) / nb;
            while (lo >= cl + len(gl)) { cl += len(gl); ++gl; }
            int last = gl;
            if (hi > lo) {
                while (hi - 1 >= ch + len(gh)) { ch += len(gh); ++gh; }
                last = gh;
            }
            int cnt = 0;
            for (int g = gl; g <= last; ++g) cnt += on(g) ? 1 : 0;
            if (cnt > MAXSYS_PB) { ok = false; break; }
            if (b == bid) {
                int64_t cg = cl;  // active slices before system g
                for (int g = gl; g <= last; ++g) {
                    if (!on(g)) continue;
                    P.j[g] = P.ng;
                    P.sys[P.ng] = g;
                    ++P.ng;
                    const int64_t v0 = lo > cg ? lo : cg;
                    const int64_t v1 = hi < cg + len(g) ? hi : cg + len(g);
                    if (v1 > v0) {
                        P.segs[P.nseg] = P.ss0[g] + (int)(v0 - cg);
                        P.segv[P.nseg + 1] = P.segv[P.nseg] + (int)(v1 - v0);
                        ++P.nseg;
                    }
                    cg += len(g);
                }
                P.nv = P.segv[P.nseg];
            }
            for (int g = gl; g <= last; ++g) {
                if (!on(g)) continue;
                if (P.b1[g] == 0) P.b0[g] = b;
                P.b1[g] = b + 1;
            }
        }
        P.mixed = 0;
        if (!ok) {  // the static partition: every system of the block's range
            const int g0 = blk_g0[bid];
            P.mixed = 1;
            P.nseg = 1;
            P.segs[0] = blk_s0[bid];
            P.segv[0] = 0;
            P.segv[1] = blk_s1[bid] - blk_s0[bid];
            P.nv = P.segv[1];
            P.ng = blk_ng[bid];
            for (int g = 0; g < nsys; ++g) {
                P.b0[g] = sys_b0[g];
                P.b1[g] = sys_b1[g];
                P.j[g] = (g >= g0 && g < g0 + P.ng) ? g - g0 : -1;
            }
            for (int j = 0; j < P.ng; ++j) P.sys[j] = g0 + j;
        }
        for (int w = 0; w < MAXSYS / 32; ++w) P.mask[w] = m[w];
        P.valid = 1;
    }
}

template <class T, class TM>
__global__ void __launch_bounds__(KTHREADS, 1) k_bicgstab(KArgs<T, TM> a) {
    // |r_hat . r| below this fraction of ||r_hat|| ||r|| is rounding noise in T
    // (FP32 vectors of ~1e6 rows: ~6e-8 / sqrt(n) relative noise in a dot product)
    const double bd_tol = sizeof(T) == 8 ? 1e-14 : 1e-9;
    constexpr bool K32 = std::is_same_v<T, float>;   // FP32 Krylov iteration
    constexpr bool M32 = std::is_same_v<TM, float>;  // FP32 V-cycle

    __shared__ double sacc[KWARPS][MAXSYS_PB][NQ];
    __shared__ double stot[MAXSYS][NQ];
    __shared__ SysState S[MAXSYS];
    extern __shared__ double s_tile_raw[];  // multigrid: a coarse tile and its halo, 36 x 36
    TM* s_tile = reinterpret_cast<TM*>(s_tile_raw);
    __shared__ int s_any;
    __shared__ Partition P;  // this block's share of the work
    const int bid = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nb = gridDim.x;
    const int nsys = a.nsys;
    for (int g = threadIdx.x; g < nsys; g += KTHREADS) {
        P.ss0[g] = a.sys_s0[g];
        P.ss1[g] = a.sys_s1[g];
    }
    if (threadIdx.x == 0) P.valid = 0;
    int nv = 0, ng_blk = 0, seg0 = 0;
    bool one_seg = true, p_valid_r = false;
    // slice of virtual index v; sg (the segment of the previous call) only advances,
    // as each warp's v increases; a block of one segment needs no lookup
    auto vslice = [&](int v, int& sg) {
        if (one_seg) return seg0 + v;
        while (v >= P.segv[sg + 1]) ++sg;
        return P.segs[sg] + (v - P.segv[sg]);
    };
    // The slices of the systems still being solved (outer set: solving or to be
    // zeroed; inner set: inside a BiCGSTAB pass) are spread evenly over all blocks,
    // recomputed whenever that set changes, so that blocks whose systems have
    // finished take over the work of the others.  Every block computes the whole
    // partition from the same system states, so all blocks agree without
    // communicating.  A block holds one segment of slices per active system in its
    // range (finished systems in between are passed over) and reduces only for
    // those systems.  A partition in which some block would hold more than
    // MAXSYS_PB active systems is replaced by the launch's static one (one segment
    // of all slices, finished systems' rows skipped).
    auto repartition = [&](int inner) {
        if (nsys == 1 && p_valid_r) return;  // one system: the partition never changes
        p_valid_r = true;
        if (threadIdx.x == 0)
            partition_update(P, S, nsys, inner, (int)nb, bid, a.blk_s0, a.blk_s1, a.blk_g0, a.blk_ng,
                             a.sys_b0, a.sys_b1);
        __syncthreads();
        nv = P.nv;
        ng_blk = P.ng;
        one_seg = P.nseg <= 1;
        seg0 = P.nseg >= 1 ? P.segs[0] : 0;
    };

    auto clear_acc = [&]() {
        for (int i = threadIdx.x; i < KWARPS * MAXSYS_PB * NQ; i += KTHREADS)
            (&sacc[0][0][0])[i] = 0.0;
        __syncthreads();
    };
    // Dot-product contributions are summed per lane in registers over all the
    // warp's rows of one system and reduced across the warp once per phase (the
    // FP64 butterfly is costly on this GPU's FP64 pipe); a warp whose slices change
    // system flushes at the change.  The order is fixed, so sums are deterministic.
    // Contributions in T go to qacck (FP32 per-lane sums in the FP32 iteration,
    // widened once per flush), FP64 ones (refinement residual) to qacc.
    double qacc[NQ];
    T qacck[NQ];
    int qj = -1, qg = -1;
    auto flush_acc = [&](int nq) {  // warp-uniform
        if (qj >= 0)
            for (int k = 0; k < nq; ++k) {
                const double w = wsum(qacc[k] + (double)qacck[k]);
                if (lane == 0) sacc[warp][qj][k] += w;
            }
        qj = -1;
        qg = -1;
    };
    // accumulate a row's contributions q[0..nq) for system g (warp-uniform g)
    auto acc = [&](int g, int nq, const auto* q) {
        using Q = std::remove_cv_t<std::remove_pointer_t<decltype(q)>>;
        if (g != qg) {
            flush_acc(nq);
            qg = g;
            qj = P.j[g];
            for (int k = 0; k < nq; ++k) { qacc[k] = 0.0; qacck[k] = (T)0; }
        }
        if constexpr (std::is_same_v<Q, double>) {
            for (int k = 0; k < nq; ++k) qacc[k] += q[k];
        } else {
            for (int k = 0; k < nq; ++k) qacck[k] += q[k];
        }
    };
    // block partials -> global, barrier, totals of every system -> stot.
    // Layout partial[(g * NQ + k) * nb + block]: the blocks of one system are a
    // contiguous run, summed by one warp (lanes stride over blocks, then a fixed
    // butterfly), so the order is fixed and the loads are independent.
    // Two partial sets used by alternate reductions: a block that has read one
    // reduction's totals and runs ahead into the next one writes the other set, so
    // it never overwrites a partial that a slower block is still reading.
    int pset = 0;
    auto reduce = [&](int nq) -> bool {
        flush_acc(nq);
        __syncthreads();
        double* part = a.partial + (int64_t)pset * nsys * NQ * nb;
        pset ^= 1;
        for (int i = threadIdx.x; i < ng_blk * nq; i += KTHREADS) {
            int j = i / nq, k = i % nq;
            double sum = 0.0;
            for (int w = 0; w < KWARPS; ++w) sum += sacc[w][j][k];
            __stcg(&part[((int64_t)P.sys[j] * NQ + k) * nb + bid], sum);
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int i = warp; i < nsys * nq; i += KWARPS) {
            int g = i / nq, k = i % nq;
            const double* src = part + ((int64_t)g * NQ + k) * nb;
            double sum = 0.0;
            for (int bb = P.b0[g] + lane; bb < P.b1[g]; bb += 32) sum += __ldcg(src + bb);
            sum = wsum(sum);
            if (lane == 0) stot[g][k] = sum;
        }
        __syncthreads();
        return true;
    };
    // system of a slice (a launch of one system needs no lookup)
    auto sysof = [&](int sl) -> int { return nsys == 1 ? 0 : __ldg(a.slice_sys + sl); };
    // The FP32 streaming phases take four consecutive rows per thread with 16-byte
    // loads (consecutive threads, consecutive rows: a warp covers four slices).  A
    // warp walks its rows one group after another and each group waits for one
    // round trip to memory, so four rows per trip instead of one cut those phases'
    // latency.  body(row0, g) for row0 a multiple of 4 in a slice of system g still
    // in its pass; segments hold one system each unless the partition is the
    // static one (P.mixed), which the callers handle by slices instead.  Threads of
    // a warp may have rows or not (a segment's last rows), so a phase with dot
    // products first makes every thread register the segment's system (enter(g),
    // all threads together): the warp-wide flush of the per-lane sums then only
    // ever runs with the whole warp.
    auto quads = [&](auto&& enter, auto&& body) {
        for (int k = 0; k < P.nseg; ++k) {
            const int64_t r0 = (int64_t)P.segs[k] * SLICE;
            const int64_t n4 = (int64_t)(P.segv[k + 1] - P.segv[k]) * (SLICE / 4);
            const int g = sysof(P.segs[k]);
            if (!S[g].inner_active) continue;
            enter(g);
            for (int64_t q = threadIdx.x; q < n4; q += KTHREADS) body(r0 + 4 * q, g);
        }
    };
    auto no_enter = [](int) {};
    // L2 prefetch of this block's rows of a row-indexed vector (elem bytes per row)
    // by bulk copies (one thread per segment, chunks of at most 64 KB), so that a
    // phase's streamed inputs are on their way from DRAM while its warps start:
    // each warp walks its slices one after another, and 32 warps per SM alone keep
    // too few loads in flight to cover the DRAM latency.  Slices start on 128-byte
    // boundaries, so every copy is 16-byte aligned with a size that is a multiple
    // of 16, as the bulk copy requires.
    auto prefetch = [&](const void* vec, int elem) {
        const int ns = P.nseg;
        for (int k = threadIdx.x; k < ns; k += KTHREADS) {
            const char* p0 = static_cast<const char*>(vec) + (int64_t)P.segs[k] * SLICE * elem;
            uint64_t left = (uint64_t)(P.segv[k + 1] - P.segv[k]) * SLICE * elem;
            while (left > 0) {
                const uint32_t n = left > 65536u ? 65536u : (uint32_t)left;
                l2_prefetch(p0, n);
                p0 += n;
                left -= n;
            }
        }
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
    // (A vec)_row for the warp's slice (lane = row): FP64 with the FP64 operator; in
    // the Krylov precision T; in the V-cycle's precision TM (FP32: differenced rows)
    auto spmv64 = [&](int64_t sl, const double* vec) -> double {
        return sell_row<4, false, double>(a.sptr, a.width, a.col, a.a64, a.ucptr, a.ucode, a.u64, sl,
                                          lane, 0.0, 0.0, [&](int j) { return ldv(vec + j); });
    };
    auto spmvK = [&](int64_t sl, const T* vec) -> T {
        if constexpr (K32) {
            const int64_t row = sl * 32 + lane;
            return sell_row<4, true, float>(a.sptr, a.width, a.col, a.aT, a.ucptr, a.ucode, a.uT, sl,
                                            lane, ldv(vec + row), __ldg(a.rs32 + row),
                                            [&](int j) { return ldv(vec + j); });
        } else {
            return spmv64(sl, vec);
        }
    };
    auto spmvM = [&](int64_t sl, const TM* vec) -> TM {
        if constexpr (M32) {
            const int64_t row = sl * 32 + lane;
            return sell_row<4, true, float>(a.sptr, a.width, a.col, a.aM, a.ucptr, a.ucode, a.uM, sl,
                                            lane, ldv(vec + row), __ldg(a.rs32 + row),
                                            [&](int j) { return ldv(vec + j); });
        } else {
            return sell_row<4, false, double>(a.sptr, a.width, a.col, a.aM, a.ucptr, a.ucode, a.uM, sl,
                                              lane, 0.0, 0.0, [&](int j) { return ldv(vec + j); });
        }
    };

    // One V-cycle z = M^{-1} v of the aggregation multigrid: a V(1,1)-cycle with
    // l1-Jacobi smoothing from zero (D = sign(a_ii) sum_j |a_ij|, which stays a
    // convergent smoother on boundary rows that are not diagonally dominant),
    // summed restriction, piecewise-constant prolongation and a scaled coarse
    // correction:
    //   fine, down:   f = w Df^{-1} v (written by the Krylov update that produces v),
    //                 fr = v - A f,  b_1 = sum of fr over the rows of each cell
    //   level l+1:    b_{l+1}(C) = sum over the children c of C of (b_l - A_l x_l)(c),
    //                 x_l = w D_l^{-1} b_l
    //   coarsest:     x_L = A_L^{-1} b_L (dense FP64 inverse of each geometry)
    //   level l, up:  y_l = x_l + w D_l^{-1} (b_l - A_l x_l),
    //                 x_l = w D_l^{-1} b_l + corr s_{l+1}(parent),  s = x_L or y_{l+1}
    //   fine, up:     f += corr s_1(agg),  z = f + w Df^{-1} (v - A f)
    // A coarse level is processed in 32 x th tiles of its cell lattice (th = 32 on
    // large levels, down to 2 on small ones so that every SM gets a share of the
    // FP64 stencil work), one CTA per tile: the smoothing iterate x_l of the tile and
    // a two-cell halo is formed once in shared memory, then each thread of the first
    // th warps applies its cell's 5 x 5 stencil (warp = lattice row, coefficients read
    // as one contiguous slice per warp; 3 x 3 where the slice's outer ring is zero).
    // Going down, the tile's residuals are summed over 2 x 2 children straight into
    // b_{l+1}; going up, level 1 adds corr y_1 to the fine rows of each cell directly
    // (y_1 is not stored).  The smoothing steps w D^{-1} are precomputed per omega.
    // Only rows of systems still in their inner pass are touched on the fine level.
    const int64_t gtid = (int64_t)blockIdx.x * KTHREADS + threadIdx.x;
    const int64_t gstride = (int64_t)nb * KTHREADS;
    const TM mcorr = (TM)a.mg.corr;
    // s_tile[36 r + c] = f(cell, x, y) for the 32 x th tile at (x0, y0) and its halo (0
    // outside a non-periodic lattice; periodic directions wrap)
    auto stage = [&](const MgLevGeom& q, int x0, int y0, int th, auto&& f) {
        TM v[2];
        const int nst = 36 * (th + 4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = threadIdx.x + h * KTHREADS;
            v[h] = (TM)0;
            if (k < nst) {
                int xx = x0 - 2 + k % 36, yy = y0 - 2 + k / 36;
                bool ok = true;
                if (q.px) { xx %= q.nx; if (xx < 0) xx += q.nx; } else ok = xx >= 0 && xx < q.nx;
                if (q.py) { yy %= q.ny; if (yy < 0) yy += q.ny; } else ok = ok && yy >= 0 && yy < q.ny;
                if (ok) v[h] = f(q.off + (int64_t)yy * q.sx + xx, xx, yy);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = threadIdx.x + h * KTHREADS;
            if (k < nst) s_tile[k] = v[h];
        }
    };
    // sum_o A_l[c, o] s_tile[36 (warp + dy) + lane + dx] for the thread's cell c, in offset
    // order; a warp whose slices hold no nonzero outside the 3 x 3 core (wide false,
    // warp-uniform) skips the zero products, which leaves the sum unchanged
    auto stencil = [&](int l, int64_t c, bool wide) -> TM {
        const TM* cp = a.mg.coefs[l] + (c >> 5) * 800 + (c & 31);
        TM acc = (TM)0;
        if (wide) {
#pragma unroll
            for (int o = 0; o < 25; ++o) acc += ldm(cp + o * 32) * s_tile[(warp + o / 5) * 36 + lane + o % 5];
        } else {
#pragma unroll
            for (int dy = 1; dy <= 3; ++dy)
#pragma unroll
                for (int dx = 1; dx <= 3; ++dx)
                    acc += ldm(cp + (dy * 5 + dx) * 32) * s_tile[(warp + dy) * 36 + lane + dx];
        }
        return acc;
    };
    // z = M^{-1} v, given v and f = w Df^{-1} v on the rows of active systems
    auto vcycle = [&](const T* v, T* z) -> bool {
        const MgDev<TM>& M = a.mg;
        const int L = M.nlev;
        prefetch(v, sizeof(T));
        prefetch(M.fx, sizeof(TM));
        if constexpr (M32) prefetch(a.rs32, 4);
        for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
            const int sl = vslice(iv, sg);
            const int g = sysof(sl);
            const int64_t row = (int64_t)sl * 32 + lane;
            TM res = (TM)0;
            if (S[g].inner_active) res = (TM)ldv(v + row) - spmvM(sl, M.fx);
            M.fr[row] = res;
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int64_t c = gtid; c < M.n[1]; c += gstride) {
            TM sum = (TM)0;
            const int64_t q1 = __ldg(M.cptr + c + 1);
            for (int64_t q = __ldg(M.cptr + c); q < q1; ++q) sum += ldv(M.fr + __ldg(M.crow + q));
            M.b[1][c] = sum;
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int l = 1; l < L; ++l) {
            const TM* bl = M.b[l];
            const TM* wdl = M.wdinv[l];
            const int th = M.th[l];
            for (int64_t t = blockIdx.x; t < M.ntiles[l]; t += nb) {
                const MgTile tile = M.tiles[l][t];
                if (!S[tile.g].inner_active) continue;  // that geometry's solve is done
                const MgLevGeom q = M.lg[l][tile.g];
                __syncthreads();  // the previous tile's reads of s_tile are done
                stage(q, tile.x0, tile.y0, th, [&](int64_t j, int, int) -> TM {
                    return __ldg(wdl + j) * ldv(bl + j);
                });
                __syncthreads();
                const int x = tile.x0 + lane, y = tile.y0 + warp;
                const bool in = warp < th && x < q.nx && y < q.ny;
                const int64_t c = q.off + (int64_t)y * q.sx + x;
                const bool wide = __any_sync(0xffffffffu, in && __ldg(M.ring[l] + (c >> 5)));
                TM r = (TM)0;
                if (in) r = ldv(bl + c) - stencil(l, c, wide);
                __syncthreads();
                if (warp < th) s_tile[warp * 32 + lane] = r;
                __syncthreads();
                if (threadIdx.x < th * 8) {  // 16 x th/2 cells of level l+1
                    const int px = threadIdx.x & 15, py = threadIdx.x >> 4;
                    const MgLevGeom qp = M.lg[l + 1][tile.g];
                    const int X = (tile.x0 >> 1) + px, Y = (tile.y0 >> 1) + py;
                    if (X < qp.nx && Y < qp.ny) {
                        const TM* rs = s_tile;
                        const int k0 = (2 * py) * 32 + 2 * px;
                        M.b[l + 1][qp.off + (int64_t)Y * qp.sx + X] =
                            (rs[k0] + rs[k0 + 1]) + (rs[k0 + 32] + rs[k0 + 33]);
                    }
                }
            }
            if (!grid_sync(a.bar, nb, a.status)) return false;
        }
        // coarsest level: x_L = A_L^{-1} b_L with each geometry's dense FP64 inverse;
        // one warp per coarsest cell of any geometry (cells numbered densely per
        // geometry on this level, geometry found by bisection on the offsets), lanes
        // over the row, then a fixed-order warp sum
        for (int64_t c = gtid >> 5; c < M.n[L]; c += gstride >> 5) {
            int lo = 0, hi = M.ngeom - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (M.lg[L][mid].off <= c) lo = mid;
                else hi = mid - 1;
            }
            const MgLevGeom q = M.lg[L][lo];
            const int64_t m = (int64_t)q.nx * q.ny;
            const int64_t i = c - q.off;
            if (i >= m || !S[lo].inner_active) continue;  // padding, or a finished geometry (warp-uniform)
            const TM* Ai = M.cinv + __ldg(M.cinv_off + lo) + i * m;
            const TM* bL = M.b[L] + q.off;
            TM sum = (TM)0;
            for (int64_t j = lane; j < m; j += 32) sum += __ldg(Ai + j) * ldv(bL + j);
            sum = wsum(sum);
            if (lane == 0) M.x[L][c] = sum;
        }
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int l = L - 1; l >= 1; --l) {
            const TM* sol = (l + 1 == L) ? M.x[L] : M.y[l + 1];
            const TM* bl = M.b[l];
            const TM* wdl = M.wdinv[l];
            const int th = M.th[l];
            for (int64_t t = blockIdx.x; t < M.ntiles[l]; t += nb) {
                const MgTile tile = M.tiles[l][t];
                if (!S[tile.g].inner_active) continue;
                const MgLevGeom q = M.lg[l][tile.g];
                const MgLevGeom qp = M.lg[l + 1][tile.g];
                __syncthreads();
                stage(q, tile.x0, tile.y0, th, [&](int64_t j, int xx, int yy) -> TM {
                    return __ldg(wdl + j) * ldv(bl + j) +
                           mcorr * ldv(sol + qp.off + (int64_t)(yy >> 1) * qp.sx + (xx >> 1));
                });
                __syncthreads();
                const int x = tile.x0 + lane, y = tile.y0 + warp;
                const bool in = warp < th && x < q.nx && y < q.ny;
                const int64_t c = q.off + (int64_t)y * q.sx + x;
                const bool wide = __any_sync(0xffffffffu, in && __ldg(M.ring[l] + (c >> 5)));
                if (in) {
                    const TM r = ldv(bl + c) - stencil(l, c, wide);
                    const TM y = s_tile[(warp + 2) * 36 + lane + 2] + __ldg(wdl + c) * r;
                    if (l > 1) {
                        M.y[l][c] = y;
                    } else {  // fine prolongation f += corr y_1 over the cell's rows
                        const int64_t q1 = __ldg(M.cptr + c + 1);
                        for (int64_t qq = __ldg(M.cptr + c); qq < q1; ++qq) {
                            const int32_t row = __ldg(M.crow + qq);
                            M.fx[row] = ldv(M.fx + row) + mcorr * y;
                        }
                    }
                }
            }
            if (!grid_sync(a.bar, nb, a.status)) return false;
        }
        // fine prolongation f += corr s_1(agg) when level 1 is the coarsest; otherwise
        // the level-1 pass above did it
        if (L == 1) {
            const TM* sol1 = M.x[1];
            for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                if (!S[sysof(sl)].inner_active) continue;
                const int64_t rw = (int64_t)sl * 32 + lane;
                const int32_t cc = __ldg(M.agg + rw);
                if (cc >= 0) M.fx[rw] = ldv(M.fx + rw) + mcorr * ldv(sol1 + cc);
            }
            if (!grid_sync(a.bar, nb, a.status)) return false;
        }
        prefetch(v, sizeof(T));
        prefetch(M.fx, sizeof(TM));
        prefetch(M.fwdinv, sizeof(TM));
        if constexpr (M32) prefetch(a.rs32, 4);
        for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
            const int sl = vslice(iv, sg);
            const int g = sysof(sl);
            if (!S[g].inner_active) continue;
            const int64_t row = (int64_t)sl * 32 + lane;
            const TM r = (TM)ldv(v + row) - spmvM(sl, M.fx);
            z[row] = (T)(ldv(M.fx + row) + __ldg(M.fwdinv + row) * r);
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
        st.alpha_f = st.omega_f = 1.0f; st.beta_f = 0.0f;
    }
    __syncthreads();

    bool alive = true;
    for (int outer = 0; alive; ++outer) {
        repartition(0);
        // ---- X: apply the correction of the previous pass
        if (outer > 0) {
            for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                int64_t row = (int64_t)sl * 32 + lane;
                if (S[g].zero_x) a.x[row] = 0.0;
                else if (S[g].outer_active && !S[g].pass_bad) {
                    if constexpr (K32) {
                        const float2 d = ldv(reinterpret_cast<const float2*>(a.dx) + row);
                        a.x[row] = __ldcg(a.x + row) + ((double)d.x + (double)d.y);
                    } else {
                        a.x[row] = __ldcg(a.x + row) + ldv(a.dx + row);
                    }
                }
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
        }
        // ---- R: FP64 residual, inner initialisation
        clear_acc();
        for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
            const int sl = vslice(iv, sg);
            int g = sysof(sl);
            if (!S[g].outer_active) continue;
            int64_t row = (int64_t)sl * 32 + lane;
            double bi = __ldg(a.b + row);
            double ri = bi - spmv64(sl, a.x);
            T rt = (T)ri;
            a.r[row] = rt;
            a.rhat[row] = rt;
            a.p[row] = (T)0;
            a.v[row] = (T)0;
            a.dx[row] = 0.0;  // also the pair (0, 0)
            double q[3] = {ri * ri, bi * bi, (double)rt * (double)rt};
            acc(g, 3, q);
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
                        st.alpha_f = st.omega_f = 1.0f;
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
                for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
                    const int sl = vslice(iv, sg);
                    int g = sysof(sl);
                    if (S[g].zero_x) a.x[(int64_t)sl * 32 + lane] = 0.0;
                }
            }
            break;
        }

        // ---- inner BiCGSTAB pass
        while (any_of(1)) {
            repartition(1);
            // the FP32 streaming phases take rows four at a time (quads); their slice
            // loops then have nothing left to do
            const bool by_quads = K32 && M32 && !P.mixed;
            const int nvq = by_quads ? 0 : nv;
            // A: beta, p = r + beta (p - omega v)
            if (threadIdx.x < nsys) {
                SysState& st = S[threadIdx.x];
                if (st.inner_active) {
                    st.beta = (st.rho / st.rho_old) * (st.alpha / st.omega);
                    st.beta_f = (float)st.beta;
                }
            }
            __syncthreads();
            prefetch(a.r, sizeof(T));
            prefetch(a.p, sizeof(T));
            prefetch(a.v, sizeof(T));
            if (a.use_mg) prefetch(a.mg.fwdinv, sizeof(TM));
            if constexpr (K32 && M32) {
                if (by_quads) {
                    quads(no_enter, [&](int64_t r0, int g) {
                        const float be = S[g].beta_f, om = S[g].omega_f;
                        const float4 rr = *reinterpret_cast<const float4*>(a.r + r0);
                        float4 pp = *reinterpret_cast<const float4*>(a.p + r0);
                        const float4 vv = *reinterpret_cast<const float4*>(a.v + r0);
                        pp.x = rr.x + be * (pp.x - om * vv.x);
                        pp.y = rr.y + be * (pp.y - om * vv.y);
                        pp.z = rr.z + be * (pp.z - om * vv.z);
                        pp.w = rr.w + be * (pp.w - om * vv.w);
                        *reinterpret_cast<float4*>(a.p + r0) = pp;
                        if (a.use_mg) {
                            const float4 wd = __ldg(reinterpret_cast<const float4*>(a.mg.fwdinv + r0));
                            *reinterpret_cast<float4*>(a.mg.fx + r0) =
                                make_float4(wd.x * pp.x, wd.y * pp.y, wd.z * pp.z, wd.w * pp.w);
                        }
                    });
                }
            }
            for (int iv = warp, sg = 0; iv < nvq; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                const T be = sc<T>(S[g].beta, S[g].beta_f), om = sc<T>(S[g].omega, S[g].omega_f);
                const T pn = ldv(a.r + row) + be * (ldv(a.p + row) - om * ldv(a.v + row));
                a.p[row] = pn;
                if (a.use_mg) a.mg.fx[row] = __ldg(a.mg.fwdinv + row) * (TM)pn;
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
            if (a.use_mg && !vcycle(a.p, a.phat)) { alive = false; break; }
            // B: v = A phat, rhat . v
            clear_acc();
            prefetch(a.phat, sizeof(T));
            prefetch(a.rhat, sizeof(T));
            if constexpr (K32) prefetch(a.rs32, 4);
            for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                const T vi = spmvK(sl, a.phat);
                a.v[row] = vi;
                const T q[2] = {ldv(a.rhat + row) * vi, vi * vi};
                acc(g, 2, q);
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
                        st.alpha_f = (float)st.alpha;
                    }
                }
            }
            __syncthreads();
            // C: s = r - alpha v
            prefetch(a.r, sizeof(T));
            prefetch(a.v, sizeof(T));
            if (a.use_mg) prefetch(a.mg.fwdinv, sizeof(TM));
            if constexpr (K32 && M32) {
                if (by_quads) {
                    quads(no_enter, [&](int64_t r0, int g) {
                        const float al = S[g].alpha_f;
                        const float4 rr = *reinterpret_cast<const float4*>(a.r + r0);
                        const float4 vv = *reinterpret_cast<const float4*>(a.v + r0);
                        const float4 ss = make_float4(rr.x - al * vv.x, rr.y - al * vv.y, rr.z - al * vv.z,
                                                      rr.w - al * vv.w);
                        *reinterpret_cast<float4*>(a.s + r0) = ss;
                        if (a.use_mg) {
                            const float4 wd = __ldg(reinterpret_cast<const float4*>(a.mg.fwdinv + r0));
                            *reinterpret_cast<float4*>(a.mg.fx + r0) =
                                make_float4(wd.x * ss.x, wd.y * ss.y, wd.z * ss.z, wd.w * ss.w);
                        }
                    });
                }
            }
            for (int iv = warp, sg = 0; iv < nvq; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                const T si = ldv(a.r + row) - sc<T>(S[g].alpha, S[g].alpha_f) * ldv(a.v + row);
                a.s[row] = si;
                if (a.use_mg) a.mg.fx[row] = __ldg(a.mg.fwdinv + row) * (TM)si;
            }
            if (!grid_sync(a.bar, nb, a.status)) { alive = false; break; }
            if (a.use_mg && !vcycle(a.s, a.shat)) { alive = false; break; }
            // D: t = A shat; t.s, t.t, s.s
            clear_acc();
            prefetch(a.shat, sizeof(T));
            prefetch(a.s, sizeof(T));
            if constexpr (K32) prefetch(a.rs32, 4);
            for (int iv = warp, sg = 0; iv < nv; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                const T ti = spmvK(sl, a.shat);
                a.t[row] = ti;
                const T si = ldv(a.s + row);
                const T q[3] = {ti * si, ti * ti, si * si};
                acc(g, 3, q);
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
                    st.omega_f = (float)st.omega;
                }
            }
            __syncthreads();
            // E: d += alpha p + omega s; r = s - omega t; rhat.r, r.r
            clear_acc();
            prefetch(a.dx, 8);
            prefetch(a.phat, sizeof(T));
            prefetch(a.shat, sizeof(T));
            prefetch(a.s, sizeof(T));
            prefetch(a.t, sizeof(T));
            prefetch(a.rhat, sizeof(T));
            if constexpr (K32 && M32) {
                if (!P.mixed) {
                    const float zero2[2] = {0.0f, 0.0f};
                    quads([&](int g) { acc(g, 2, zero2); }, [&](int64_t r0, int g) {
                        const SysState& q = S[g];
                        const float al = q.alpha_f, om = q.omega_f;
                        float4* dx4 = reinterpret_cast<float4*>(a.dx + r0);  // rows r0, r0 + 1 | r0 + 2, r0 + 3
                        float4 d01 = dx4[0], d23 = dx4[1];
                        const float4 ph = *reinterpret_cast<const float4*>(a.phat + r0);
                        const float4 sh = *reinterpret_cast<const float4*>(a.shat + r0);
                        const float4 ss = *reinterpret_cast<const float4*>(a.s + r0);
                        const float4 tt = *reinterpret_cast<const float4*>(a.t + r0);
                        const float4 rh = *reinterpret_cast<const float4*>(a.rhat + r0);
                        float2 d;
                        d = dd_axpy2(make_float2(d01.x, d01.y), al, ph.x, om, sh.x); d01.x = d.x; d01.y = d.y;
                        d = dd_axpy2(make_float2(d01.z, d01.w), al, ph.y, om, sh.y); d01.z = d.x; d01.w = d.y;
                        d = dd_axpy2(make_float2(d23.x, d23.y), al, ph.z, om, sh.z); d23.x = d.x; d23.y = d.y;
                        d = dd_axpy2(make_float2(d23.z, d23.w), al, ph.w, om, sh.w); d23.z = d.x; d23.w = d.y;
                        dx4[0] = d01;
                        dx4[1] = d23;
                        const float4 rn = make_float4(ss.x - om * tt.x, ss.y - om * tt.y, ss.z - om * tt.z,
                                                      ss.w - om * tt.w);
                        *reinterpret_cast<float4*>(a.r + r0) = rn;
                        const float qq[2] = {((rh.x * rn.x + rh.y * rn.y) + (rh.z * rn.z + rh.w * rn.w)),
                                             ((rn.x * rn.x + rn.y * rn.y) + (rn.z * rn.z + rn.w * rn.w))};
                        acc(g, 2, qq);
                    });
                }
            }
            for (int iv = warp, sg = 0; iv < nvq; iv += KWARPS) {
                const int sl = vslice(iv, sg);
                int g = sysof(sl);
                if (!S[g].inner_active) continue;
                int64_t row = (int64_t)sl * 32 + lane;
                if constexpr (K32) {
                    float2* dx2 = reinterpret_cast<float2*>(a.dx);
                    dx2[row] = dd_axpy2(ldv(dx2 + row), S[g].alpha_f, ldv(a.phat + row), S[g].omega_f,
                                        ldv(a.shat + row));
                } else {
                    a.dx[row] = ldv(a.dx + row) + S[g].alpha * (double)ldv(a.phat + row) +
                                S[g].omega * (double)ldv(a.shat + row);
                }
                const T rn = ldv(a.s + row) - sc<T>(S[g].omega, S[g].omega_f) * ldv(a.t + row);
                a.r[row] = rn;
                const T q[2] = {ldv(a.rhat + row) * rn, rn * rn};
                acc(g, 2, q);
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
    // the coarse tile lives in dynamic shared memory (above the static 48 KB limit
    // together with the rest; set here, outside any graph capture); as much L1 as
    // possible for the vector gathers: the smallest shared-memory configuration that
    // holds the block's ~52 KB
    int occ = 1;
    {
        const void* kern[] = {(const void*)k_bicgstab<double, double>, (const void*)k_bicgstab<float, float>,
                              (const void*)k_bicgstab<double, float>};
        for (const void* k : kern) {
            VIP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, KSMEM_DYN));
            VIP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxL1));
            int o = 0;
            VIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, KTHREADS, KSMEM_DYN));
            if (o < 1) { c->err = "the Krylov kernel does not fit on an SM"; return VIP_ERR_CUDA; }
        }
    }
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
    VIP_CUDA(dalloc(c, &P.sys_s0, nsys)); VIP_CUDA(dalloc(c, &P.sys_s1, nsys));
    VIP_CUDA(dalloc(c, &P.partial, (size_t)2 * nb * nsys * NQ));
    VIP_CUDA(cudaMemsetAsync(P.partial, 0, (size_t)2 * nb * nsys * NQ * sizeof(double), c->stream));
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
    {
        std::vector<int32_t> ss0(nsys), ss1(nsys);
        for (int g = 0; g < nsys; ++g) {
            ss0[g] = (int32_t)(row0[g] / SLICE);
            ss1[g] = (int32_t)((row0[g] + rows[g]) / SLICE);
        }
        VIP_CUDA(cudaMemcpyAsync(P.sys_s0, ss0.data(), nsys * 4, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaMemcpyAsync(P.sys_s1, ss1.data(), nsys * 4, cudaMemcpyHostToDevice, st));
        VIP_CUDA(cudaStreamSynchronize(st));
    }
    VIP_CUDA(cudaStreamSynchronize(st));
    return VIP_OK;
}

// the array of precision T: the FP64 one or its FP32 copy
template <class T>
static const T* pick(const double* d, const float* f) {
    if constexpr (std::is_same_v<T, double>) return d;
    else return f;
}

template <class T>
static MgDev<T> mg_view(const Multigrid& M) {
    MgDev<T> d;
    memset(&d, 0, sizeof(d));
    d.nlev = M.nlev;
    d.ngeom = M.ngeom;
    d.agg = M.agg; d.cptr = M.cptr; d.crow = M.crow;
    d.fwdinv = pick<T>(M.fwdinv, M.fwdinv32);
    d.fr = (T*)M.fr; d.fx = (T*)M.fx;
    for (int l = 1; l <= M.nlev; ++l) {
        const MgLevel& v = M.lev[l];
        d.n[l] = v.n;
        d.ntiles[l] = v.ntiles;
        d.lg[l] = v.lg;
        d.tiles[l] = v.tiles;
        d.coefs[l] = pick<T>(v.coefs, v.coefs32);
        d.ring[l] = v.ring;
        d.th[l] = v.th;
        d.wdinv[l] = pick<T>(v.wdinv, v.wdinv32);
        d.x[l] = (T*)v.x; d.b[l] = (T*)v.b; d.y[l] = (T*)v.y;
    }
    d.corr = M.corr;
    d.cinv = pick<T>(M.cinv, M.cinv32);
    d.cinv_off = M.cinv_off;
    return d;
}

template <class T, class TM>
static vip_status launch(vip_ctx* c, const KrylovPlan& P, const Sell& A, const double* b, double* x,
                         double rtol, int32_t max_iters, double inner_rtol, const Multigrid* mg) {
    KrylovWork& W = sizeof(T) == 8 ? c->work64 : c->work32;
    if (W.n < A.nrows || c->work64.n < A.nrows) { c->err = "Krylov workspace too small"; return VIP_ERR_ARG; }
    if ((sizeof(T) == 4 || sizeof(TM) == 4) && (!A.v32 || !A.rs32)) {
        c->err = "operator has no FP32 copy";
        return VIP_ERR_ARG;
    }
    KArgs<T, TM> a;
    a.sptr = A.sptr; a.width = A.width; a.col = A.col; a.a64 = A.v64;
    a.aT = pick<T>(A.v64, A.v32);
    a.aM = pick<TM>(A.v64, A.v32);
    a.ucptr = A.ucptr; a.ucode = A.ucode; a.u64 = A.uv64;
    a.uT = pick<T>(A.uv64, A.uv32);
    a.uM = pick<TM>(A.uv64, A.uv32);
    a.rs32 = A.rs32;
    a.slice_sys = P.slice_sys; a.blk_s0 = P.blk_s0; a.blk_s1 = P.blk_s1; a.blk_g0 = P.blk_g0;
    a.blk_ng = P.blk_ng;
    a.sys_b0 = P.sys_b0; a.sys_b1 = P.sys_b1; a.partial = P.partial; a.bar = P.bar;
    a.sys_s0 = P.sys_s0; a.sys_s1 = P.sys_s1;
    a.nsys = P.nsys; a.b = b; a.x = x;
    a.r = (T*)W.r; a.rhat = (T*)W.rhat; a.p = (T*)W.p; a.v = (T*)W.v; a.s = (T*)W.s;
    a.t = (T*)W.t;
    a.dx = (double*)c->work64.dx;  // the correction is accumulated in FP64 in every form
    a.rtol = rtol; a.inner_rtol = inner_rtol; a.max_iters = max_iters;
    // FP32 passes are re-anchored on the FP64 residual at least every 4000 iterations
    a.max_outer = 1000;
    a.max_pass = sizeof(T) == 8 ? max_iters : 4000;
    a.out_iters = P.out_iters; a.out_outer = P.out_outer; a.out_relres = P.out_relres;
    a.out_status = P.out_status; a.status = c->d_status;
    a.use_mg = (mg && mg->built) ? 1 : 0;
    if (a.use_mg) {
        a.mg = mg_view<TM>(*mg);
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
    cfg.dynamicSmemBytes = a.use_mg ? KSMEM_DYN : 0;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    VIP_CUDA(cudaLaunchKernelEx(&cfg, k_bicgstab<T, TM>, a));
    return VIP_OK;
}

vip_status krylov_solve(vip_ctx* c, const KrylovPlan& P, const Sell& A, const double* b, double* x,
                        int precision, double rtol, int32_t max_iters, double inner_rtol,
                        const Multigrid* mg) {
    if (precision == VIP_PREC_MIXED)
        return launch<float, float>(c, P, A, b, x, rtol, max_iters, inner_rtol, mg);
    if (precision == VIP_PREC_MG32 && mg && mg->built)
        return launch<double, float>(c, P, A, b, x, rtol, max_iters, inner_rtol, mg);
    return launch<double, double>(c, P, A, b, x, rtol, max_iters, inner_rtol, mg);
}

}  // namespace vip
