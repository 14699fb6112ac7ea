// Internal declarations of libvip (the GPU path).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vip.h"
#include "vip_mg.cuh"

namespace vip {

constexpr int SLICE = 32;           // SELL-C slice height = warp size
constexpr int KMAX = 64;            // largest neighbour list per point
constexpr int NPTYPE = 7;           // point types: node, E, W, N, S, probe1, probe2
enum PointType { PT_NODE = 0, PT_E = 1, PT_W = 2, PT_N = 3, PT_S = 4, PT_B1 = 5, PT_B2 = 6 };
constexpr uint8_t KIND_PAD = 255;   // padding row (not a node)

// Row kinds of a padded row.
enum : int { ROW_PAD = 0, ROW_NODE = 1, ROW_BORDER = 2 };

// Device status codes share the values of vip_status.
__device__ __forceinline__ void set_status(int* st, int code) {
    atomicCAS(st, 0, code);
}

// SELL-32 table: row r lives in slice r/32, lane r%32; entry k of row r is at
// sptr[r/32] + k*32 + r%32.  Padding entries carry col = r and value 0.
struct Sell {
    int64_t nrows = 0;
    int64_t nslices = 0;
    int64_t nstored = 0;          // stored entries incl. padding
    int64_t nnz = 0;              // real entries
    int64_t* sptr = nullptr;      // [nslices+1]
    int32_t* width = nullptr;     // [nslices]
    int32_t* rowlen = nullptr;    // [nrows]
    int32_t* col = nullptr;       // [nstored]
    double* v64 = nullptr;        // [nstored]
    float* v32 = nullptr;         // [nstored] (only for Krylov operators)
    // Krylov operators: FP64 row sums sum_k a_rk rounded to FP32, for rows applied
    // in FP32 in differenced form, sum_k a_rk (x_k - x_r) + rowsum_r x_r
    float* rs32 = nullptr;        // [nrows]
    // Uniform slices (Krylov operators only): a slice whose 32 rows hold the same
    // stencil (entry k has the same value, bit for bit, in every row, and a column
    // that is the row plus the same offset in every row or the same column in every
    // row) is also stored once, as `width` entries at ucptr[s]: value uv64/uv32 and
    // column code ucode (2 d: column = row + d; 2 c + 1: column c).  ucptr[s] = -1
    // for the other slices.  Results are the same either way.
    int64_t* ucptr = nullptr;     // [nslices]
    int32_t* ucode = nullptr;     // [nuentries]
    double* uv64 = nullptr;
    float* uv32 = nullptr;
    int64_t nuniform = 0;         // uniform slices
    int64_t nuentries = 0;        // entries of their stored stencils (slices with the same
                                  // stencil share one copy)
    int64_t nstored_other = 0;    // stored entries of the other slices
};

struct Geom {
    int64_t n = 0;          // nodes
    int64_t off = 0;        // global node offset (caller order)
    int64_t row0 = 0;       // first padded row
    int64_t nrows = 0;      // padded rows (multiple of SLICE, >= n + bordered)
    double Lx = 0, Ly = 0;
    double Re = 100.0, dt = 1e-3;
    bool bordered = false;  // closed domain: Poisson bordered by mu
    bool has_outlet = false;
    int64_t pin = -1;       // bordered: caller index (within the geometry) of node k
    // parity of the multigrid's first 2h x 2h cell grid: 1 moves the cell boundaries
    // by one lattice spacing along that axis (non-periodic axes only)
    int32_t mg_shift_x = 0, mg_shift_y = 0;
    int32_t probes = VIP_PROBES_NORMAL;  // normal-point placement (vip_set_probes)
};

// Per-geometry constants visible to kernels.
struct GeomDev {
    int64_t row0, nrows, n;
    double Lx, Ly, Re, dt, alpha;
    int32_t bordered;
    int64_t pin;       // bordered: padded row of the reference node k (first interior node)
    int32_t probes;    // VIP_PROBES_*
};

// Work split of a persistent Krylov launch over a batch of systems.
constexpr int MAXSYS_PB = 16;   // systems a block may touch
constexpr int NQ = 4;           // reduced quantities per phase
struct KrylovPlan {
    int nblocks = 0, nthreads = 0, nsys = 0;
    int64_t nslices = 0;
    // device arrays
    int32_t* slice_sys = nullptr;   // [nslices] system of each slice
    // static partition (equal slice counts), used by the launch only when its own
    // partition of the active systems would give a block too many systems
    int32_t* blk_s0 = nullptr;      // [nblocks] slice range of a block
    int32_t* blk_s1 = nullptr;
    int32_t* blk_g0 = nullptr;      // [nblocks] first system of the block
    int32_t* blk_ng = nullptr;      // [nblocks] number of systems of the block
    int32_t* sys_b0 = nullptr;      // [nsys] block range of a system
    int32_t* sys_b1 = nullptr;
    int32_t* sys_s0 = nullptr;      // [nsys] slice range of a system
    int32_t* sys_s1 = nullptr;
    double* partial = nullptr;      // [2][nsys][NQ][nblocks]: two sets, alternate reductions
    int32_t* flags = nullptr;       // [nblocks]
    uint32_t* bar = nullptr;        // [2] barrier count / generation
    // per-system outputs
    int32_t* out_iters = nullptr;
    int32_t* out_outer = nullptr;
    double* out_relres = nullptr;
    int32_t* out_status = nullptr;
};

struct KrylovWork {
    int64_t n = 0;                 // vector length (rows)
    void* r = nullptr;             // T vectors
    void* rhat = nullptr;
    void* p = nullptr;
    void* v = nullptr;
    void* s = nullptr;
    void* t = nullptr;
    void* dx = nullptr;
    double* r64 = nullptr;
    int tbytes = 0;
};

struct Tables {
    // MLS output (CSR over points; point id = type * R + row)
    int64_t npts = 0, nnz_pts = 0, nnz_nodes = 0;
    int64_t* pptr = nullptr;       // [npts+1]
    int32_t* pidx = nullptr;       // [nnz_pts] neighbour rows (padded row ids)
    double* w00 = nullptr;         // [nnz_pts] Psi^[0,0] of every point
    double* wd = nullptr;          // [5][nnz_nodes] D10, D01, D20, D11, D02 of node points
    Sell lap, d00, gx, gy, helm, pois, ve, vw, vn, vs;
};

}  // namespace vip

struct vip_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<vip::Geom> geoms;
    // host copies of the node sets (caller order)
    std::vector<double> hx, hy, hnx, hny, hh;
    std::vector<uint8_t> hkind;
    int weight = VIP_W_CUBIC_SPLINE;
    double support = 2.2;
    int basis_order = 2;
    int precision = VIP_PREC_FP64;
    double rtol = 1e-8;
    int32_t max_iters = 20000;
    int identity = VIP_IDENTITY_EXACT;
    int pressure = VIP_PRESSURE_INCREMENTAL;  // VIP_PRESSURE_* (vip_set_pressure)
    double inner_rtol = 1e-4;     // FP32 inner solve target relative to the FP64 residual
    double helm_inner_rtol = 1e-6;   // the same for the Helmholtz solves (vip_set_inner_tolerance)
    bool built = false;
    bool use_graph = true;
    int64_t N = 0;                // nodes
    int64_t R = 0;                // padded rows
    int32_t nbordered = 0;
    int num_sms = 0;
    // device node arrays in padded row space [R]
    double *x = nullptr, *y = nullptr, *nx = nullptr, *ny = nullptr, *h = nullptr;
    uint8_t* kind = nullptr;
    int32_t* row_geom = nullptr;   // [R] geometry of a row
    int8_t* row_type = nullptr;    // [R] ROW_PAD / ROW_NODE / ROW_BORDER
    double* inv_ew = nullptr;      // [R] 1/|x_e - x_w|
    double* inv_ns = nullptr;      // [R] 1/|x_n - x_s|
    double* pstep = nullptr;       // [R] normal-point step of boundary rows (INSIDE geometries only)
    vip::GeomDev* gdev = nullptr;  // [G]
    int32_t* first_row = nullptr;  // [G]
    vip::Tables T;
    // state [R] (FP64)
    double *u = nullptr, *v = nullptr, *p = nullptr, *phi = nullptr;
    double* uv_prev = nullptr;     // [2R] u^{n-1}, v^{n-1}: the Helmholtz guess u^n + (u*^n - u^{n-1})
    double *ubc = nullptr, *vbc = nullptr;
    double *nu_prev = nullptr, *nv_prev = nullptr;
    double *hsol = nullptr, *hrhs = nullptr;   // Helmholtz [2R]
    double* prhs = nullptr;                    // Poisson rhs [R]
    double* lphi = nullptr;                    // scratch [R]
    int64_t* d_step = nullptr;
    int32_t* d_status = nullptr;
    // Krylov plans and workspaces
    vip::KrylovPlan plan_helm, plan_pois;
    vip::KrylovWork work64, work32;
    vip::Multigrid mg;             // preconditioner of the pressure-increment solve
    bool use_mg = true;
    void* cnn = nullptr;           // warm-start network state (vip_cnn.cu)
    void* phat = nullptr;          // preconditioned search directions [2R] (FP64 size)
    void* shat = nullptr;
    // per-step statistics on the device
    int64_t* d_stats = nullptr;     // [4] poisson inner iters, steps, poisson outer, helm iters
    int64_t* d_giters = nullptr;    // [G] Poisson inner iterations of each geometry since vip_set_state
    cudaGraphExec_t graph = nullptr;
    int64_t host_steps = 0;
    // phase events recorded inside every step (also inside the graph)
    cudaEvent_t ev[VIP_PHASE_COUNT + 1] = {};
    bool profiling = false;
    double prof_ms[VIP_PHASE_COUNT] = {0, 0, 0, 0, 0};
    int64_t prof_steps = 0;
    std::vector<void*> allocs;
};

namespace vip {
// build stage (vip_build.cu)
vip_status build_all(vip_ctx* c);
// Krylov (vip_krylov.cu)
vip_status krylov_plan(vip_ctx* c, KrylovPlan& plan, const Sell& A,
                       const std::vector<int64_t>& sys_row0, const std::vector<int64_t>& sys_rows);
// Re-partition the plan's slices over its blocks in proportion to rows x the
// iterations each system needed in its last solve (device side, stream-ordered).
vip_status krylov_solve(vip_ctx* c, const KrylovPlan& plan, const Sell& A, const double* b,
                        double* x, int precision, double rtol, int32_t max_iters,
                        double inner_rtol, const Multigrid* mg = nullptr);
// multigrid (vip_mg.cu)
vip_status mg_build(vip_ctx* c, Multigrid& M);
// Sets the smoother damping and the correction scale; rescales omega * dinv on every
// level (stream-ordered) when omega changes.
vip_status mg_set_params(vip_ctx* c, Multigrid& M, float omega, float corr);
// warm-start network (vip_cnn.cu)
vip_status cnn_setup(vip_ctx* c, uint64_t seed);
void cnn_free(vip_ctx* c);
vip_status cnn_warm_start(vip_ctx* c, cudaStream_t s);
vip_status cnn_after_solve(vip_ctx* c, cudaStream_t s);
bool cnn_collecting(vip_ctx* c);
// the warm start's history phi^{n-1}: reset to phi (outside any step), and its buffer
// (saved with checkpoints)
vip_status cnn_reset_history(vip_ctx* c);
double* cnn_history(vip_ctx* c);
// step kernels (vip_step.cu)
void launch_conv_rhs(vip_ctx* c, cudaStream_t s);
void launch_div(vip_ctx* c, cudaStream_t s);
void launch_project(vip_ctx* c, cudaStream_t s);
void launch_spmv(const Sell& A, const double* x, double* y, cudaStream_t s);
void launch_convection(vip_ctx* c, const double* u, const double* v, double* Nu, double* Nv,
                       cudaStream_t s);
// Device scratch that outlives no call: freed on every return path (cudaFree waits
// for the work queued on it).  Not registered with the context.
struct DeviceScratch {
    void* p = nullptr;
    DeviceScratch() = default;
    DeviceScratch(const DeviceScratch&) = delete;
    DeviceScratch& operator=(const DeviceScratch&) = delete;
    ~DeviceScratch() {
        if (p) cudaFree(p);
    }
};
// memory helper: context-owned device memory, freed by vip_destroy
template <class T>
inline cudaError_t dalloc(vip_ctx* c, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e == cudaSuccess) {
        c->allocs.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}
}  // namespace vip

#define VIP_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            c->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
            return e_ == cudaErrorMemoryAllocation ? VIP_ERR_OOM : VIP_ERR_CUDA;    \
        }                                                                           \
    } while (0)
