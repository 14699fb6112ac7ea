// vip_bicgstab_static: a BiCGSTAB solve that allocates no device memory.
//
// For callers that cannot call cudaMalloc while they run -- for example a host
// process whose device memory is owned by another framework's pooling allocator,
// a real-time loop that must not allocate, or code that runs with a fixed device
// memory budget.  The caller passes the matrix (CSR), the right-hand side and the
// solution vector in its own device memory; every other buffer the solver needs
// (Krylov vectors, reduction partials, the grid-barrier words, the result record)
// lives in file-scope static device arrays of fixed size (about 6.3 MB), which a
// device holds from the moment the library's code is loaded on it until the
// process exits.
//
// The solver is the plain FP64 form of the library's persistent BiCGSTAB: one
// cooperative launch, deterministic reductions, a grid barrier whose every wait is
// bounded (2 s, then VIP_ERR_TIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/vip.h"

namespace {

constexpr int64_t MAX_ROWS = VIP_STATIC_MAX_ROWS;
constexpr int NVEC = 6;                      // r, rhat, p, v, s, t
constexpr int MAX_BLOCKS = 1024;
constexpr int NQ = 2;                        // reduced quantities per phase
constexpr int THREADS = 256;
constexpr int64_t OFF_PART = NVEC * MAX_ROWS;
// two sets of block partials, used by alternate reductions: a block that runs
// ahead into the next reduction never overwrites a partial another block is
// still reading
constexpr int64_t OFF_RES = OFF_PART + 2LL * NQ * MAX_BLOCKS;
constexpr int64_t SCRATCH = OFF_RES + 8;     // doubles (about 6.3 MB)

// The shared workspace.  In host code this name is only a stand-in for the
// device object; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_scratch[SCRATCH];
static __device__ __align__(256) unsigned int g_bar[2];

struct Args {
    int64_t n;
    const int64_t* ptr;
    const int32_t* col;
    const double* val;
    const double* b;
    double* x;
    double rtol;
    int max_iters;
    double* ws;          // device address of g_scratch
    unsigned int* bar;   // device address of g_bar
};

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid barrier with a bounded wait; returns false (and flags the timeout) after 2 s
__device__ bool barrier(unsigned* bar, unsigned nb, double* res) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned gen = ld_acq(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == nb - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long t0 = now_ns();
            while (ld_acq(bar + 1) == gen) {
                if (now_ns() - t0 > 2000000000ull) {
                    res[3] = 1.0;  // timeout flag
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ double spmv_row(const Args& a, int64_t i, const double* v) {
    double s = 0.0;
    for (int64_t k = a.ptr[i]; k < a.ptr[i + 1]; ++k) s += a.val[k] * __ldcg(v + a.col[k]);
    return s;
}

__global__ void __launch_bounds__(THREADS) k_bicgstab_static(Args a) {
    __shared__ double red[THREADS / 32][NQ];
    __shared__ double tot[NQ];
    const unsigned nb = gridDim.x;
    const int64_t n = a.n;
    double* r = a.ws;
    double* rh = r + MAX_ROWS;
    double* p = rh + MAX_ROWS;
    double* v = p + MAX_ROWS;
    double* s = v + MAX_ROWS;
    double* t = s + MAX_ROWS;
    double* part = a.ws + OFF_PART;
    double* res = a.ws + OFF_RES;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)nb * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int set = 0;  // partial set of the next reduction

    // block sums of q[0..nq) -> partials, barrier, totals in fixed order
    auto reduce = [&](double q0, double q1) -> bool {
        double q[NQ] = {q0, q1};
        for (int k = 0; k < NQ; ++k) {
            double w = q[k];
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == 0) red[warp][k] = w;
        }
        __syncthreads();
        double* ps = part + (int64_t)set * NQ * MAX_BLOCKS;
        set ^= 1;
        if (threadIdx.x < NQ) {
            double sum = 0.0;
            for (int w = 0; w < THREADS / 32; ++w) sum += red[w][threadIdx.x];
            __stcg(ps + (int64_t)threadIdx.x * MAX_BLOCKS + blockIdx.x, sum);
        }
        if (!barrier(a.bar, nb, res)) return false;
        if (warp < NQ) {
            double sum = 0.0;
            for (unsigned bb = lane; bb < nb; bb += 32) sum += __ldcg(ps + (int64_t)warp * MAX_BLOCKS + bb);
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) tot[warp] = sum;
        }
        __syncthreads();
        return true;
    };

    // r = b - A x, rhat = r; ||b||, ||r||
    double qb = 0.0, qr = 0.0;
    for (int64_t i = g0; i < n; i += gs) {
        double bi = a.b[i];
        double ri = bi - spmv_row(a, i, a.x);
        r[i] = ri;
        rh[i] = ri;
        p[i] = 0.0;
        v[i] = 0.0;
        qb += bi * bi;
        qr += ri * ri;
    }
    if (!reduce(qb, qr)) return;
    const double bnorm = sqrt(tot[0]);
    double rho = tot[1], rho_old = 1.0, alpha = 1.0, omega = 1.0;
    const double tol = a.rtol * bnorm;
    int it = 0;
    int status = 0;
    bool done = bnorm == 0.0 || sqrt(tot[1]) <= tol;
    if (bnorm == 0.0)
        for (int64_t i = g0; i < n; i += gs) a.x[i] = 0.0;
    while (!done) {
        if (it >= a.max_iters) { status = VIP_ERR_NOT_CONVERGED; break; }
        const double beta = (rho / rho_old) * (alpha / omega);
        for (int64_t i = g0; i < n; i += gs) p[i] = __ldcg(r + i) + beta * (__ldcg(p + i) - omega * __ldcg(v + i));
        if (!barrier(a.bar, nb, res)) return;
        double q0 = 0.0;
        for (int64_t i = g0; i < n; i += gs) {
            double vi = spmv_row(a, i, p);
            v[i] = vi;
            q0 += __ldcg(rh + i) * vi;
        }
        if (!reduce(q0, 0.0)) return;
        if (tot[0] == 0.0) { status = VIP_ERR_BREAKDOWN; break; }
        alpha = rho / tot[0];
        double q1 = 0.0;
        for (int64_t i = g0; i < n; i += gs) {
            double si = __ldcg(r + i) - alpha * __ldcg(v + i);
            s[i] = si;
            q1 += si * si;
        }
        if (!reduce(q1, 0.0)) return;
        ++it;
        if (sqrt(tot[0]) <= tol) {
            for (int64_t i = g0; i < n; i += gs) a.x[i] += alpha * __ldcg(p + i);
            break;
        }
        double qts = 0.0, qtt = 0.0;
        for (int64_t i = g0; i < n; i += gs) {
            double ti = spmv_row(a, i, s);
            t[i] = ti;
            double si = __ldcg(s + i);
            qts += ti * si;
            qtt += ti * ti;
        }
        if (!reduce(qts, qtt)) return;
        if (tot[1] == 0.0) { status = VIP_ERR_BREAKDOWN; break; }
        omega = tot[0] / tot[1];
        double qrr = 0.0, qrh = 0.0;
        for (int64_t i = g0; i < n; i += gs) {
            double si = __ldcg(s + i);
            a.x[i] += alpha * __ldcg(p + i) + omega * si;
            double ri = si - omega * __ldcg(t + i);
            r[i] = ri;
            qrr += ri * ri;
            qrh += __ldcg(rh + i) * ri;
        }
        if (!reduce(qrr, qrh)) return;
        rho_old = rho;
        rho = tot[1];
        if (sqrt(tot[0]) <= tol) break;
        if (rho == 0.0 || omega == 0.0) { status = VIP_ERR_BREAKDOWN; break; }
    }
    // true residual of the returned x
    if (!barrier(a.bar, nb, res)) return;
    double qf = 0.0;
    for (int64_t i = g0; i < n; i += gs) {
        double ri = a.b[i] - spmv_row(a, i, a.x);
        qf += ri * ri;
    }
    if (!reduce(qf, 0.0)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        res[0] = (double)it;
        res[1] = bnorm > 0.0 ? sqrt(tot[0]) / bnorm : 0.0;
        res[2] = (double)status;
    }
}

// Device addresses of the workspace, looked up once per device (the first call
// on a device also loads this module's kernels there).
std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
double* g_ws_addr[MAX_DEVICES] = {};
unsigned int* g_bar_addr[MAX_DEVICES] = {};

// makes `device` current for the call and puts the caller's device back
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

vip_status setup(int device, double** ws, unsigned int** bar) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ws_addr[device]) {
        void* p1 = nullptr;
        void* p2 = nullptr;
        if (cudaGetSymbolAddress(&p1, g_scratch) != cudaSuccess) return VIP_ERR_CUDA;
        if (cudaGetSymbolAddress(&p2, g_bar) != cudaSuccess) return VIP_ERR_CUDA;
        g_ws_addr[device] = static_cast<double*>(p1);
        g_bar_addr[device] = static_cast<unsigned int*>(p2);
    }
    *ws = g_ws_addr[device];
    *bar = g_bar_addr[device];
    return VIP_OK;
}

// q is managed memory, or device memory of `device` (memory of another GPU would be
// read as a peer address, which faults without peer access)
bool on_device(const void* q, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == device);
}

}  // namespace

extern "C" vip_status vip_bicgstab_static(int device, void* cuda_stream, int64_t n, const int64_t* row_ptr,
                                          const int32_t* col, const double* val, const double* b, double* x,
                                          double rtol, int32_t max_iters, int32_t* iters, double* relres) {
    if (n < 1 || n > MAX_ROWS) return VIP_ERR_ARG;  // beyond the static workspace
    if (!row_ptr || !col || !val || !b || !x || !(rtol > 0.0) || max_iters < 1) return VIP_ERR_ARG;
    if (device < 0 || device >= MAX_DEVICES) return VIP_ERR_ARG;
    DeviceGuard guard(device);
    if (!guard.ok) return VIP_ERR_CUDA;
    if (!on_device(row_ptr, device) || !on_device(col, device) || !on_device(val, device) ||
        !on_device(b, device) || !on_device(x, device))
        return VIP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {   // the call synchronises its stream and reads results back: it cannot be captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return VIP_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return VIP_ERR_ARG;
    }
    double* ws = nullptr;
    unsigned int* bar = nullptr;
    vip_status st0 = setup(device, &ws, &bar);
    if (st0 != VIP_OK) return st0;
    int nsm = 0, occ = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return VIP_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bicgstab_static, THREADS, 0) != cudaSuccess)
        return VIP_ERR_CUDA;
    const int64_t want = (n + THREADS - 1) / THREADS;
    const int64_t cap = std::min<int64_t>((int64_t)nsm * std::max(occ, 1), MAX_BLOCKS);
    const int grid = (int)std::min<int64_t>(cap, want);
    // the barrier words and the result record start at zero on every call; the
    // Krylov vectors and partials need no clearing (each is written before it is read)
    if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) return VIP_ERR_CUDA;
    if (cudaMemsetAsync(ws + OFF_RES, 0, 8 * sizeof(double), st) != cudaSuccess) return VIP_ERR_CUDA;
    Args a{n, row_ptr, col, val, b, x, rtol, max_iters, ws, bar};
    void* args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void*)k_bicgstab_static, dim3(grid), dim3(THREADS), args, 0, st) !=
        cudaSuccess)
        return VIP_ERR_CUDA;
    double h[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(h, ws + OFF_RES, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return VIP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return VIP_ERR_CUDA;
    if (iters) *iters = (int32_t)h[0];
    if (relres) *relres = h[1];
    if (h[3] != 0.0) return VIP_ERR_TIMEOUT;
    if (h[2] != 0.0) return (vip_status)(int)h[2];
    return VIP_OK;
}
