// C ABI of libvip (declared in include/vip.h).  Host orchestration only: every
// step of the method runs in the kernels of vip_build.cu, vip_step.cu and
// vip_krylov.cu.
//
// Device layout: each geometry occupies a block of padded rows (a multiple of the
// 32-row slice) holding its nodes in caller order, then one border row for a
// closed domain (the extra unknown mu of the bordered Poisson system), then
// padding rows (identity rows of the Krylov operators).  All per-node fields and
// all operator rows and columns use this padded row space.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "vip_internal.cuh"

using namespace vip;

namespace {

__global__ void k_check_finite(const double* __restrict__ a, const int8_t* __restrict__ rt, int64_t n,
                               int32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && rt[i] == ROW_NODE && !isfinite(a[i])) set_status(status, VIP_ERR_NONFINITE);
}

__global__ void k_stats(const int32_t* __restrict__ it, const int32_t* __restrict__ outer, int nsys,
                        const int32_t* __restrict__ hit, int nhsys, int64_t* __restrict__ tot,
                        int64_t* __restrict__ git) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int m = 0, o = 0, hm = 0;
        for (int g = 0; g < nsys; ++g) { m = max(m, it[g]); o = max(o, outer[g]); git[g] += it[g]; }
        for (int g = 0; g < nhsys; ++g) hm = max(hm, hit[g]);
        tot[0] += m;
        tot[1] += 1;
        tot[2] += o;
        tot[3] += hm;
    }
}

// Sum of the 64-bit words of a buffer modulo 2^64 (order-free, so deterministic
// with atomics): the checkpoint's checksum.
__global__ void k_word_sum(const uint64_t* __restrict__ w, int64_t n, unsigned long long* out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += w[i];
    atomicAdd(out, s);
}

// Checkpoint layout: this header, then CKPT_ARRAYS arrays of R doubles each (padded
// row space: u, v, p, phi, N_u^{n-1}, N_v^{n-1}, the two Dirichlet value arrays, the
// last Helmholtz solutions u*, v* and u^{n-1}, v^{n-1} (the next Helmholtz guess), and
// the warm start's phi^{n-1}), then the step counter (int64).
constexpr int CKPT_ARRAYS = 13;
struct CkptHeader {
    uint64_t magic;      // "VIPCKPT3"
    int64_t n_nodes, n_rows, n_geoms;
    int64_t host_steps;
    uint64_t checksum;   // k_word_sum of everything after the header
    uint64_t pad[2];
};
constexpr uint64_t CKPT_MAGIC = 0x3354504B43504956ull;

vip_status fail(vip_ctx* c, vip_status s, const char* msg) {
    if (c) c->err = msg;
    return s;
}

bool finite_host(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// copy caller-order node data (length N) into padded rows, or back
vip_status scatter(vip_ctx* c, const double* src, double* dst_padded) {
    for (const Geom& g : c->geoms)
        VIP_CUDA(cudaMemcpyAsync(dst_padded + g.row0, src + g.off, g.n * sizeof(double),
                                 cudaMemcpyDefault, c->stream));
    return VIP_OK;
}
vip_status gather_out(vip_ctx* c, const double* src_padded, double* dst) {
    for (const Geom& g : c->geoms)
        VIP_CUDA(cudaMemcpyAsync(dst + g.off, src_padded + g.row0, g.n * sizeof(double),
                                 cudaMemcpyDefault, c->stream));
    return VIP_OK;
}

vip_status do_step(vip_ctx* c, cudaStream_t s) {
    VIP_CUDA(cudaEventRecord(c->ev[0], s));
    launch_conv_rhs(c, s);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(cudaEventRecord(c->ev[1], s));
    vip_status st = krylov_solve(c, c->plan_helm, c->T.helm, c->hrhs, c->hsol, c->precision, c->rtol,
                                 c->max_iters, c->helm_inner_rtol);
    if (st != VIP_OK) return st;
    VIP_CUDA(cudaEventRecord(c->ev[2], s));
    launch_div(c, s);
    VIP_CUDA(cudaGetLastError());
    if ((st = cnn_warm_start(c, s)) != VIP_OK) return st;
    VIP_CUDA(cudaEventRecord(c->ev[3], s));
    st = krylov_solve(c, c->plan_pois, c->T.pois, c->prhs, c->phi, c->precision, c->rtol,
                      c->max_iters, c->inner_rtol, c->use_mg ? &c->mg : nullptr);
    if (st != VIP_OK) return st;
    if ((st = cnn_after_solve(c, s)) != VIP_OK) return st;
    VIP_CUDA(cudaEventRecord(c->ev[4], s));
    k_stats<<<1, 32, 0, s>>>(c->plan_pois.out_iters, c->plan_pois.out_outer, c->plan_pois.nsys,
                             c->plan_helm.out_iters, c->plan_helm.nsys, c->d_stats, c->d_giters);
    launch_project(c, s);
    VIP_CUDA(cudaGetLastError());
    VIP_CUDA(cudaEventRecord(c->ev[5], s));
    return VIP_OK;
}

}  // namespace

extern "C" {

vip_status vip_create(vip_ctx** out, int device, void* cuda_stream) {
    if (!out) return VIP_ERR_ARG;
    *out = nullptr;
    vip_ctx* c = new (std::nothrow) vip_ctx();
    if (!c) return VIP_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        *out = c;
        c->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return VIP_ERR_CUDA;
    }
    *out = c;
    VIP_CUDA(dalloc(c, &c->d_status, 1));
    VIP_CUDA(dalloc(c, &c->d_step, 1));
    VIP_CUDA(dalloc(c, &c->d_stats, 4));
    for (int i = 0; i <= VIP_PHASE_COUNT; ++i) VIP_CUDA(cudaEventCreate(&c->ev[i]));
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, c->stream));
    VIP_CUDA(cudaMemsetAsync(c->d_step, 0, 8, c->stream));
    VIP_CUDA(cudaMemsetAsync(c->d_stats, 0, 32, c->stream));
    return VIP_OK;
}

void vip_destroy(vip_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    cudaStreamSynchronize(c->stream);
    for (void* p : c->allocs) cudaFree(p);
    cnn_free(c);
    for (int i = 0; i <= VIP_PHASE_COUNT; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
}

const char* vip_last_error(const vip_ctx* c) { return c ? c->err.c_str() : "null context"; }

vip_status vip_add_nodes(vip_ctx* c, int64_t n, const double* x, const double* y, const uint8_t* kind,
                         const double* nx, const double* ny, const double* h_local, double Lx,
                         double Ly, int32_t* geom_out) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_add_nodes after vip_build");
    if (n < 6 || !x || !y || !kind || !nx || !ny || !h_local)
        return fail(c, VIP_ERR_ARG, "vip_add_nodes: need n >= 6 and non-null arrays");
    if (n > (int64_t)1 << 29) return fail(c, VIP_ERR_ARG, "vip_add_nodes: too many nodes");
    if (!(Lx >= 0.0) || !(Ly >= 0.0)) return fail(c, VIP_ERR_ARG, "vip_add_nodes: negative period");
    std::vector<double> bx(n), by(n), bnx(n), bny(n), bh(n);
    std::vector<uint8_t> bk(n);
    cudaMemcpy(bx.data(), x, n * 8, cudaMemcpyDefault);
    cudaMemcpy(by.data(), y, n * 8, cudaMemcpyDefault);
    cudaMemcpy(bnx.data(), nx, n * 8, cudaMemcpyDefault);
    cudaMemcpy(bny.data(), ny, n * 8, cudaMemcpyDefault);
    cudaMemcpy(bh.data(), h_local, n * 8, cudaMemcpyDefault);
    cudaMemcpy(bk.data(), kind, n, cudaMemcpyDefault);
    if (cudaGetLastError() != cudaSuccess) return fail(c, VIP_ERR_CUDA, "vip_add_nodes: copy failed");
    if (!finite_host(bx.data(), n) || !finite_host(by.data(), n) || !finite_host(bh.data(), n) ||
        !finite_host(bnx.data(), n) || !finite_host(bny.data(), n))
        return fail(c, VIP_ERR_NONFINITE, "vip_add_nodes: non-finite coordinate, normal or spacing");
    Geom g;
    g.n = n;
    g.off = c->N;
    g.Lx = Lx;
    g.Ly = Ly;
    for (int64_t i = 0; i < n; ++i) {
        if (!(bh[i] > 0.0)) return fail(c, VIP_ERR_ARG, "vip_add_nodes: h_local must be > 0");
        if (bk[i] > VIP_NODE_OUTLET) return fail(c, VIP_ERR_ARG, "vip_add_nodes: bad node kind");
        if (bk[i] != VIP_NODE_INTERIOR) {
            double nn = std::hypot(bnx[i], bny[i]);
            if (std::fabs(nn - 1.0) > 1e-6)
                return fail(c, VIP_ERR_ARG, "vip_add_nodes: boundary normal is not a unit vector");
        }
        if (bk[i] == VIP_NODE_OUTLET) g.has_outlet = true;
    }
    c->hx.insert(c->hx.end(), bx.begin(), bx.end());
    c->hy.insert(c->hy.end(), by.begin(), by.end());
    c->hnx.insert(c->hnx.end(), bnx.begin(), bnx.end());
    c->hny.insert(c->hny.end(), bny.begin(), bny.end());
    c->hh.insert(c->hh.end(), bh.begin(), bh.end());
    c->hkind.insert(c->hkind.end(), bk.begin(), bk.end());
    c->N += n;
    c->geoms.push_back(g);
    if (geom_out) *geom_out = (int32_t)(c->geoms.size() - 1);
    return VIP_OK;
}

vip_status vip_set_mls(vip_ctx* c, int basis_order, int weight, double support) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_set_mls after vip_build");
    if (basis_order != 2) return fail(c, VIP_ERR_ARG, "only the quadratic basis (order 2) is supported");
    if (weight != VIP_W_CUBIC_SPLINE && weight != VIP_W_PAPER) return fail(c, VIP_ERR_ARG, "bad weight");
    if (!(support > 1.0) || !(support < 8.0)) return fail(c, VIP_ERR_ARG, "support must be in (1, 8)");
    c->basis_order = basis_order;
    c->weight = weight;
    c->support = support;
    return VIP_OK;
}

vip_status vip_set_flow(vip_ctx* c, int32_t geom, double Re, double dt) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_set_flow after vip_build");
    if (!(Re > 0.0) || !(dt > 0.0) || !std::isfinite(Re) || !std::isfinite(dt))
        return fail(c, VIP_ERR_ARG, "Re and dt must be positive and finite");
    if (geom < -1 || geom >= (int32_t)c->geoms.size()) return fail(c, VIP_ERR_ARG, "bad geometry index");
    for (int32_t g = 0; g < (int32_t)c->geoms.size(); ++g)
        if (geom == -1 || geom == g) { c->geoms[g].Re = Re; c->geoms[g].dt = dt; }
    return VIP_OK;
}

vip_status vip_set_probes(vip_ctx* c, int32_t geom, int mode) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_set_probes after vip_build");
    if (geom < -1 || geom >= (int32_t)c->geoms.size()) return fail(c, VIP_ERR_ARG, "bad geometry index");
    if (mode != VIP_PROBES_NORMAL && mode != VIP_PROBES_INSIDE)
        return fail(c, VIP_ERR_ARG, "vip_set_probes: mode must be VIP_PROBES_NORMAL or VIP_PROBES_INSIDE");
    for (int32_t g = 0; g < (int32_t)c->geoms.size(); ++g)
        if (geom == -1 || geom == g) c->geoms[g].probes = mode;
    return VIP_OK;
}

vip_status vip_set_mg_shift(vip_ctx* c, int32_t geom, int32_t shift_x, int32_t shift_y) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_set_mg_shift after vip_build");
    if (geom < -1 || geom >= (int32_t)c->geoms.size()) return fail(c, VIP_ERR_ARG, "bad geometry index");
    if ((shift_x != 0 && shift_x != 1) || (shift_y != 0 && shift_y != 1))
        return fail(c, VIP_ERR_ARG, "vip_set_mg_shift: shifts must be 0 or 1");
    for (int32_t g = 0; g < (int32_t)c->geoms.size(); ++g) {
        if (geom != -1 && geom != g) continue;
        const Geom& gg = c->geoms[g];
        if ((shift_x && gg.Lx > 0) || (shift_y && gg.Ly > 0))
            return fail(c, VIP_ERR_ARG, "vip_set_mg_shift: a periodic axis keeps shift 0");
    }
    for (int32_t g = 0; g < (int32_t)c->geoms.size(); ++g)
        if (geom == -1 || geom == g) { c->geoms[g].mg_shift_x = shift_x; c->geoms[g].mg_shift_y = shift_y; }
    return VIP_OK;
}

vip_status vip_get_geometry_iters(vip_ctx* c, int64_t* poisson_iters) {
    if (!c || !poisson_iters) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_get_geometry_iters before vip_build");
    VIP_CUDA(cudaMemcpyAsync(poisson_iters, c->d_giters, c->geoms.size() * 8, cudaMemcpyDeviceToHost,
                             c->stream));
    VIP_CUDA(cudaStreamSynchronize(c->stream));
    return VIP_OK;
}

vip_status vip_set_multigrid(vip_ctx* c, float omega, float corr) {
    if (!c) return VIP_ERR_ARG;
    if (!(omega > 0.0f && omega <= 1.5f)) return fail(c, VIP_ERR_ARG, "omega must be in (0, 1.5]");
    if (!(corr > 0.0f && corr <= 3.0f)) return fail(c, VIP_ERR_ARG, "corr must be in (0, 3]");
    if ((omega != c->mg.omega || corr != c->mg.corr) && c->graph) {
        cudaGraphExecDestroy(c->graph);  // the captured launch holds the old values
        c->graph = nullptr;
    }
    return mg_set_params(c, c->mg, omega, corr);
}

vip_status vip_autotune(vip_ctx* c, const float* omegas, int32_t nomega, const float* corrs, int32_t ncorr,
                        vip_tune_result* out) {
    if (!c || !omegas || !corrs || !out) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_autotune before vip_build");
    if (!c->use_mg || !c->mg.built) return fail(c, VIP_ERR_ARG, "vip_autotune: no multigrid");
    if (c->host_steps < 1) return fail(c, VIP_ERR_ARG, "vip_autotune: take a step first");
    if (nomega < 1 || ncorr < 1 || nomega * ncorr > VIP_TUNE_MAX)
        return fail(c, VIP_ERR_ARG, "vip_autotune: 1 to VIP_TUNE_MAX candidate pairs");
    for (int i = 0; i < nomega; ++i)
        if (!(omegas[i] > 0.0f && omegas[i] <= 1.5f)) return fail(c, VIP_ERR_ARG, "omega must be in (0, 1.5]");
    for (int i = 0; i < ncorr; ++i)
        if (!(corrs[i] > 0.0f && corrs[i] <= 3.0f)) return fail(c, VIP_ERR_ARG, "corr must be in (0, 3]");
    cudaStream_t st = c->stream;
    DeviceScratch xs;  // the candidates' solutions
    VIP_CUDA(cudaMalloc(&xs.p, (size_t)c->R * sizeof(double)));
    double* x = static_cast<double*>(xs.p);
    cudaEvent_t e0, e1;
    VIP_CUDA(cudaEventCreate(&e0));
    VIP_CUDA(cudaEventCreate(&e1));
    memset(out, 0, sizeof(*out));
    const float keep_w = c->mg.omega, keep_c = c->mg.corr;
    int best = -1;
    vip_status s = VIP_OK;
    for (int i = 0; i < nomega && s == VIP_OK; ++i)
        for (int j = 0; j < ncorr && s == VIP_OK; ++j) {
            const int k = i * ncorr + j;
            if ((s = mg_set_params(c, c->mg, omegas[i], corrs[j])) != VIP_OK) break;
            out->omega[k] = omegas[i];
            out->corr[k] = corrs[j];
            if (cudaMemsetAsync(x, 0, c->R * sizeof(double), st) != cudaSuccess ||
                cudaMemsetAsync(c->d_status, 0, 4, st) != cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess) { s = VIP_ERR_CUDA; break; }
            s = krylov_solve(c, c->plan_pois, c->T.pois, c->prhs, x, c->precision, c->rtol, c->max_iters,
                             c->inner_rtol, &c->mg);
            if (s != VIP_OK) break;
            std::vector<int32_t> it(c->plan_pois.nsys);
            int32_t hs = 0;
            float ms = 0.0f;
            if (cudaEventRecord(e1, st) != cudaSuccess ||
                cudaMemcpyAsync(it.data(), c->plan_pois.out_iters, it.size() * 4, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(&hs, c->d_status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                s = VIP_ERR_CUDA;
                break;
            }
            out->iters[k] = *std::max_element(it.begin(), it.end());
            out->ms[k] = hs ? -1.0 : (double)ms;  // a candidate that did not converge is out
            if (!hs && (best < 0 || out->ms[k] < out->ms[best])) best = k;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemsetAsync(c->d_status, 0, 4, st);
    out->ncand = nomega * ncorr;
    {
        const vip_status s2 = mg_set_params(c, c->mg, keep_w, keep_c);
        if (s == VIP_OK) s = s2;
    }
    if (s != VIP_OK) return s;
    if (best < 0) return fail(c, VIP_ERR_NOT_CONVERGED, "vip_autotune: no candidate converged");
    out->best = best;
    return vip_set_multigrid(c, out->omega[best], out->corr[best]);
}

vip_status vip_set_solver(vip_ctx* c, int precision, double rtol, int32_t max_iters, int identity) {
    if (!c) return VIP_ERR_ARG;
    if (precision != VIP_PREC_FP64 && precision != VIP_PREC_MIXED && precision != VIP_PREC_MG32)
        return fail(c, VIP_ERR_ARG, "bad precision");
    if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(c, VIP_ERR_ARG, "rtol must be in (0, 1)");
    if (max_iters < 1) return fail(c, VIP_ERR_ARG, "max_iters must be >= 1");
    if (identity != VIP_IDENTITY_EXACT && identity != VIP_IDENTITY_MLS) return fail(c, VIP_ERR_ARG, "bad identity");
    if (c->built && identity != c->identity) return fail(c, VIP_ERR_ARG, "identity mode is fixed at vip_build");
    if (precision != c->precision || rtol != c->rtol || max_iters != c->max_iters) {
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    }
    c->precision = precision;
    c->rtol = rtol;
    c->max_iters = max_iters;
    c->identity = identity;
    return VIP_OK;
}

vip_status vip_set_pressure(vip_ctx* c, int form) {
    if (!c) return VIP_ERR_ARG;
    if (form != VIP_PRESSURE_INCREMENTAL && form != VIP_PRESSURE_KIM_MOIN &&
        form != VIP_PRESSURE_INCREMENTAL_INTERIOR)
        return fail(c, VIP_ERR_ARG, "vip_set_pressure: bad form");
    if (form != c->pressure && c->graph) {  // the step graph holds the launch arguments
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->pressure = form;
    return VIP_OK;
}

vip_status vip_set_inner_tolerance(vip_ctx* c, int which, double inner_rtol) {
    if (!c) return VIP_ERR_ARG;
    if (which != VIP_OP_POISSON && which != VIP_OP_HELM_U)
        return fail(c, VIP_ERR_ARG, "vip_set_inner_tolerance: which must be VIP_OP_POISSON or VIP_OP_HELM_U");
    if (!(inner_rtol > 0.0) || !(inner_rtol < 1.0)) return fail(c, VIP_ERR_ARG, "inner_rtol must be in (0, 1)");
    double& slot = which == VIP_OP_POISSON ? c->inner_rtol : c->helm_inner_rtol;
    if (inner_rtol != slot && c->graph) {  // the step graph holds the launch arguments
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    slot = inner_rtol;
    return VIP_OK;
}

vip_status vip_set_refinement(vip_ctx* c, double inner_rtol) {
    vip_status s = vip_set_inner_tolerance(c, VIP_OP_POISSON, inner_rtol);
    if (s != VIP_OK) return s;
    return vip_set_inner_tolerance(c, VIP_OP_HELM_U, inner_rtol);
}

vip_status vip_build(vip_ctx* c) {
    if (!c) return VIP_ERR_ARG;
    if (c->built) return fail(c, VIP_ERR_ARG, "vip_build called twice");
    if (c->geoms.empty()) return fail(c, VIP_ERR_ARG, "no nodes");
    VIP_CUDA(cudaSetDevice(c->device));
    const int G = (int)c->geoms.size();
    VIP_CUDA(dalloc(c, &c->d_giters, (size_t)G));
    VIP_CUDA(cudaMemsetAsync(c->d_giters, 0, G * sizeof(int64_t), c->stream));
    int64_t R = 0;
    c->nbordered = 0;
    for (Geom& g : c->geoms) {
        g.bordered = !g.has_outlet;
        g.row0 = R;
        g.nrows = ((g.n + (g.bordered ? 1 : 0) + SLICE - 1) / SLICE) * SLICE;
        R += g.nrows;
        if (g.bordered) c->nbordered++;
    }
    if (R >= ((int64_t)1 << 30)) return fail(c, VIP_ERR_ARG, "problem too large");
    c->R = R;
    std::vector<double> px(R, 0.0), py(R, 0.0), pnx(R, 0.0), pny(R, 0.0), ph(R, 1.0);
    std::vector<uint8_t> pk(R, KIND_PAD);
    std::vector<int32_t> prg(R, 0), first(G);
    std::vector<int8_t> prt(R, ROW_PAD);
    std::vector<GeomDev> gd(G);
    for (int gi = 0; gi < G; ++gi) {
        const Geom& g = c->geoms[gi];
        for (int64_t i = 0; i < g.n; ++i) {
            int64_t r = g.row0 + i, s = g.off + i;
            px[r] = c->hx[s]; py[r] = c->hy[s]; pnx[r] = c->hnx[s]; pny[r] = c->hny[s];
            ph[r] = c->hh[s]; pk[r] = c->hkind[s]; prt[r] = ROW_NODE;
        }
        for (int64_t r = g.row0; r < g.row0 + g.nrows; ++r) prg[r] = gi;
        if (g.bordered) prt[g.row0 + g.n] = ROW_BORDER;
        first[gi] = (int32_t)g.row0;
        int64_t pin = -1;
        if (g.bordered) {
            for (int64_t i = 0; i < g.n && pin < 0; ++i)
                if (c->hkind[g.off + i] == VIP_NODE_INTERIOR) pin = g.row0 + i;
            if (pin < 0) return fail(c, VIP_ERR_ARG, "a closed geometry needs an interior node");
        }
        gd[gi] = GeomDev{g.row0, g.nrows, g.n, g.Lx, g.Ly, g.Re, g.dt, g.dt / (2.0 * g.Re),
                         g.bordered ? 1 : 0, pin, g.probes};
        if (g.probes == VIP_PROBES_INSIDE && !(c->support > 2.0))
            return fail(c, VIP_ERR_ARG, "VIP_PROBES_INSIDE needs a support ratio above 2");
    }
    cudaStream_t st = c->stream;
    VIP_CUDA(dalloc(c, &c->x, R)); VIP_CUDA(dalloc(c, &c->y, R)); VIP_CUDA(dalloc(c, &c->nx, R));
    VIP_CUDA(dalloc(c, &c->ny, R)); VIP_CUDA(dalloc(c, &c->h, R)); VIP_CUDA(dalloc(c, &c->kind, R));
    VIP_CUDA(dalloc(c, &c->row_geom, R)); VIP_CUDA(dalloc(c, &c->row_type, R));
    VIP_CUDA(dalloc(c, &c->inv_ew, R)); VIP_CUDA(dalloc(c, &c->inv_ns, R));
    VIP_CUDA(dalloc(c, &c->gdev, G)); VIP_CUDA(dalloc(c, &c->first_row, G));
    VIP_CUDA(cudaMemcpyAsync(c->x, px.data(), R * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->y, py.data(), R * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->nx, pnx.data(), R * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->ny, pny.data(), R * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->h, ph.data(), R * 8, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->kind, pk.data(), R, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->row_geom, prg.data(), R * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->row_type, prt.data(), R, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->gdev, gd.data(), G * sizeof(GeomDev), cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->first_row, first.data(), G * 4, cudaMemcpyHostToDevice, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    vip_status s = build_all(c);
    if (s != VIP_OK) return s;
    // Krylov plans: Helmholtz = u systems then v systems; Poisson = one per geometry
    std::vector<int64_t> r0, nr, r0h, nrh;
    for (const Geom& g : c->geoms) { r0.push_back(g.row0); nr.push_back(g.nrows); }
    r0h = r0; nrh = nr;
    for (const Geom& g : c->geoms) { r0h.push_back(R + g.row0); nrh.push_back(g.nrows); }
    if ((s = krylov_plan(c, c->plan_helm, c->T.helm, r0h, nrh)) != VIP_OK) return s;
    if ((s = krylov_plan(c, c->plan_pois, c->T.pois, r0, nr)) != VIP_OK) return s;
    for (KrylovWork* W : {&c->work64, &c->work32}) {
        int tb = (W == &c->work64) ? 8 : 4;
        W->n = 2 * R;
        W->tbytes = tb;
        void** v[] = {&W->r, &W->rhat, &W->p, &W->v, &W->s, &W->t, &W->dx};
        for (void** q : v) {
            char* m = nullptr;
            VIP_CUDA(dalloc(c, &m, (size_t)2 * R * tb));
            VIP_CUDA(cudaMemsetAsync(m, 0, (size_t)2 * R * tb, st));
            *q = m;
        }
    }
    if ((s = cnn_setup(c, 20140126)) != VIP_OK) return s;
    if (c->use_mg) {
        if ((s = mg_build(c, c->mg)) != VIP_OK) return s;
        char* m = nullptr;
        VIP_CUDA(dalloc(c, &m, (size_t)2 * R * 8));
        c->phat = m;
        VIP_CUDA(dalloc(c, &m, (size_t)2 * R * 8));
        c->shat = m;
    }
    double** fields[] = {&c->u, &c->v, &c->p, &c->phi, &c->ubc, &c->vbc, &c->nu_prev, &c->nv_prev,
                         &c->prhs, &c->lphi};
    for (double** f : fields) {
        VIP_CUDA(dalloc(c, f, R));
        VIP_CUDA(cudaMemsetAsync(*f, 0, R * 8, st));
    }
    VIP_CUDA(dalloc(c, &c->hsol, 2 * R));
    VIP_CUDA(dalloc(c, &c->hrhs, 2 * R));
    VIP_CUDA(dalloc(c, &c->uv_prev, 2 * R));
    VIP_CUDA(cudaMemsetAsync(c->uv_prev, 0, 2 * R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->hsol, 0, 2 * R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->hrhs, 0, 2 * R * 8, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    c->built = true;
    return VIP_OK;
}

vip_status vip_set_state(vip_ctx* c, const double* u, const double* v, const double* p) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_set_state before vip_build");
    if (!u || !v) return fail(c, VIP_ERR_ARG, "vip_set_state: u and v are required");
    cudaStream_t st = c->stream;
    vip_status s;
    if ((s = scatter(c, u, c->u)) != VIP_OK) return s;
    if ((s = scatter(c, v, c->v)) != VIP_OK) return s;
    if (p) { if ((s = scatter(c, p, c->p)) != VIP_OK) return s; }
    else VIP_CUDA(cudaMemsetAsync(c->p, 0, c->R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));
    for (double* f : {c->u, c->v, c->p})
        k_check_finite<<<(unsigned)((c->R + 255) / 256), 256, 0, st>>>(f, c->row_type, c->R, c->d_status);
    VIP_CUDA(cudaMemcpyAsync(c->ubc, c->u, c->R * 8, cudaMemcpyDeviceToDevice, st));
    VIP_CUDA(cudaMemcpyAsync(c->vbc, c->v, c->R * 8, cudaMemcpyDeviceToDevice, st));
    VIP_CUDA(cudaMemsetAsync(c->phi, 0, c->R * 8, st));
    if ((s = cnn_reset_history(c)) != VIP_OK) return s;
    VIP_CUDA(cudaMemsetAsync(c->nu_prev, 0, c->R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->nv_prev, 0, c->R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->d_step, 0, 8, st));
    VIP_CUDA(cudaMemsetAsync(c->d_stats, 0, 32, st));
    VIP_CUDA(cudaMemsetAsync(c->d_giters, 0, c->geoms.size() * 8, st));
    int32_t hs = 0;
    VIP_CUDA(cudaMemcpyAsync(&hs, c->d_status, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    c->host_steps = 0;
    if (hs) return fail(c, (vip_status)hs, "vip_set_state: non-finite value in u, v or p");
    return VIP_OK;
}

vip_status vip_step(vip_ctx* c, int32_t nsteps) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_step before vip_build");
    if (nsteps < 0) return fail(c, VIP_ERR_ARG, "nsteps < 0");
    VIP_CUDA(cudaSetDevice(c->device));
    for (int32_t k = 0; k < nsteps; ++k) {
        const bool direct = cnn_collecting(c);  // sample slots advance every step
        if (c->use_graph && !c->graph && !direct) {
            cudaGraph_t g = nullptr;
            cudaStream_t cs = c->stream;
            bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            vip_status s = VIP_OK;
            if (ok) {
                s = do_step(c, cs);
                ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && s == VIP_OK;
            }
            if (ok) ok = cudaGraphInstantiate(&c->graph, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (!ok) {  // run without a graph from now on
                cudaGetLastError();
                c->graph = nullptr;
                c->use_graph = false;
            }
        }
        if (c->graph && !direct) {
            VIP_CUDA(cudaGraphLaunch(c->graph, c->stream));
        } else {
            vip_status s = do_step(c, c->stream);
            if (s != VIP_OK) return s;
        }
        c->host_steps++;
        if (c->profiling) {
            VIP_CUDA(cudaEventSynchronize(c->ev[VIP_PHASE_COUNT]));
            for (int ph = 0; ph < VIP_PHASE_COUNT; ++ph) {
                float ms = 0.f;
                VIP_CUDA(cudaEventElapsedTime(&ms, c->ev[ph], c->ev[ph + 1]));
                c->prof_ms[ph] += ms;
            }
            c->prof_steps++;
        }
    }
    return VIP_OK;
}

vip_status vip_load_state(vip_ctx* c, const double* u, const double* v, const double* p) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_load_state before vip_build");
    vip_status s;
    if (u && (s = scatter(c, u, c->u)) != VIP_OK) return s;
    if (v && (s = scatter(c, v, c->v)) != VIP_OK) return s;
    if (p && (s = scatter(c, p, c->p)) != VIP_OK) return s;
    return VIP_OK;
}

vip_status vip_set_profiling(vip_ctx* c, int enable) {
    if (!c) return VIP_ERR_ARG;
    c->profiling = enable != 0;
    if (c->profiling) {
        for (double& m : c->prof_ms) m = 0.0;
        c->prof_steps = 0;
    }
    return VIP_OK;
}

vip_status vip_get_profile(vip_ctx* c, double* phase_ms, int64_t* nsteps) {
    if (!c) return VIP_ERR_ARG;
    if (phase_ms)
        for (int i = 0; i < VIP_PHASE_COUNT; ++i) phase_ms[i] = c->prof_ms[i];
    if (nsteps) *nsteps = c->prof_steps;
    return VIP_OK;
}

vip_status vip_get_state(vip_ctx* c, double* u, double* v, double* p, double* phi) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_get_state before vip_build");
    vip_status s;
    if (u && (s = gather_out(c, c->u, u)) != VIP_OK) return s;
    if (v && (s = gather_out(c, c->v, v)) != VIP_OK) return s;
    if (p && (s = gather_out(c, c->p, p)) != VIP_OK) return s;
    if (phi && (s = gather_out(c, c->phi, phi)) != VIP_OK) return s;
    VIP_CUDA(cudaStreamSynchronize(c->stream));
    return VIP_OK;
}

vip_status vip_checkpoint_size(vip_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_checkpoint_size before vip_build");
    *bytes = (int64_t)sizeof(CkptHeader) + CKPT_ARRAYS * c->R * 8 + 8;
    return VIP_OK;
}

vip_status vip_checkpoint(vip_ctx* c, int save, void* buf) {
    if (!c || !buf) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_checkpoint before vip_build");
    VIP_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    double* arrays[CKPT_ARRAYS] = {c->u, c->v, c->p, c->phi, c->nu_prev, c->nv_prev, c->ubc, c->vbc,
                                   c->hsol, c->hsol + c->R, c->uv_prev, c->uv_prev + c->R,
                                   cnn_history(c)};
    if (!arrays[CKPT_ARRAYS - 1]) return fail(c, VIP_ERR_ARG, "vip_checkpoint: no warm-start state");
    char* body = static_cast<char*>(buf) + sizeof(CkptHeader);
    const int64_t nbody = CKPT_ARRAYS * c->R * 8 + 8;
    // checksum of the body as it lies in buf (host or device): summed on the device
    auto checksum = [&](uint64_t* out) -> vip_status {
        DeviceScratch d_body, d_sum;
        cudaPointerAttributes at{};
        const bool on_dev = cudaPointerGetAttributes(&at, buf) == cudaSuccess &&
                            (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        const uint64_t* w = reinterpret_cast<const uint64_t*>(body);
        if (!on_dev) {
            VIP_CUDA(cudaMalloc(&d_body.p, nbody));
            VIP_CUDA(cudaMemcpyAsync(d_body.p, body, nbody, cudaMemcpyDefault, st));
            w = static_cast<const uint64_t*>(d_body.p);
        }
        VIP_CUDA(cudaMalloc(&d_sum.p, 8));
        VIP_CUDA(cudaMemsetAsync(d_sum.p, 0, 8, st));
        k_word_sum<<<152, 256, 0, st>>>(w, nbody / 8, static_cast<unsigned long long*>(d_sum.p));
        VIP_CUDA(cudaGetLastError());
        VIP_CUDA(cudaMemcpyAsync(out, d_sum.p, 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        return VIP_OK;
    };
    vip_status s;
    if (save) {
        for (int k = 0; k < CKPT_ARRAYS; ++k)
            VIP_CUDA(cudaMemcpyAsync(body + (int64_t)k * c->R * 8, arrays[k], c->R * 8, cudaMemcpyDefault, st));
        VIP_CUDA(cudaMemcpyAsync(body + CKPT_ARRAYS * c->R * 8, c->d_step, 8, cudaMemcpyDefault, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        CkptHeader h{};
        h.magic = CKPT_MAGIC;
        h.n_nodes = c->N;
        h.n_rows = c->R;
        h.n_geoms = (int64_t)c->geoms.size();
        h.host_steps = c->host_steps;
        if ((s = checksum(&h.checksum)) != VIP_OK) return s;
        VIP_CUDA(cudaMemcpyAsync(buf, &h, sizeof(h), cudaMemcpyDefault, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        return VIP_OK;
    }
    CkptHeader h{};
    VIP_CUDA(cudaMemcpyAsync(&h, buf, sizeof(h), cudaMemcpyDefault, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    if (h.magic != CKPT_MAGIC || h.n_nodes != c->N || h.n_rows != c->R || h.n_geoms != (int64_t)c->geoms.size())
        return fail(c, VIP_ERR_ARG, "vip_checkpoint: the buffer holds no checkpoint of this context");
    uint64_t sum = 0;
    if ((s = checksum(&sum)) != VIP_OK) return s;
    if (sum != h.checksum) return fail(c, VIP_ERR_ARG, "vip_checkpoint: checksum mismatch");
    for (int k = 0; k < CKPT_ARRAYS; ++k)
        VIP_CUDA(cudaMemcpyAsync(arrays[k], body + (int64_t)k * c->R * 8, c->R * 8, cudaMemcpyDefault, st));
    VIP_CUDA(cudaMemcpyAsync(c->d_step, body + CKPT_ARRAYS * c->R * 8, 8, cudaMemcpyDefault, st));
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    c->host_steps = h.host_steps;
    return VIP_OK;
}

vip_status vip_get_stats(vip_ctx* c, vip_step_stats* out) {
    if (!c || !out) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_get_stats before vip_build");
    cudaStream_t st = c->stream;
    auto rd = [&](const KrylovPlan& P, int32_t* it, int32_t* outer, double* rel) -> vip_status {
        std::vector<int32_t> a(P.nsys), b(P.nsys);
        std::vector<double> d(P.nsys);
        VIP_CUDA(cudaMemcpyAsync(a.data(), P.out_iters, P.nsys * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(b.data(), P.out_outer, P.nsys * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(d.data(), P.out_relres, P.nsys * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        *it = 0; *outer = 0; *rel = 0;
        for (int g = 0; g < P.nsys; ++g) {
            *it = std::max(*it, a[g]);
            *outer = std::max(*outer, b[g]);
            *rel = std::max(*rel, d[g]);
        }
        return VIP_OK;
    };
    memset(out, 0, sizeof(*out));
    int32_t dummy;
    vip_status s;
    if ((s = rd(c->plan_helm, &out->helm_iters, &dummy, &out->helm_relres)) != VIP_OK) return s;
    if ((s = rd(c->plan_pois, &out->poisson_iters, &out->poisson_outer, &out->poisson_relres)) != VIP_OK)
        return s;
    int64_t tot[4];
    int32_t hs = 0;
    VIP_CUDA(cudaMemcpyAsync(tot, c->d_stats, 32, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaMemcpyAsync(&hs, c->d_status, 4, cudaMemcpyDeviceToHost, st));
    VIP_CUDA(cudaStreamSynchronize(st));
    out->total_poisson_iters = tot[0];
    out->steps = tot[1];
    out->total_poisson_outer = tot[2];
    out->total_helm_iters = tot[3];
    out->status = hs;
    if (hs) {
        c->err = "device reported status " + std::to_string(hs);
        return (vip_status)hs;
    }
    return VIP_OK;
}

vip_status vip_get_sizes(vip_ctx* c, int64_t* n_nodes, int32_t* n_geoms) {
    if (!c) return VIP_ERR_ARG;
    if (n_nodes) *n_nodes = c->N;
    if (n_geoms) *n_geoms = (int32_t)c->geoms.size();
    return VIP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// table export / apply / solve (inspection and parity checks)
// ---------------------------------------------------------------------------
namespace {

struct HostCSR {
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
};

// padded row -> caller node index, or N + k for the border row of the k-th bordered geometry
std::vector<int64_t> row_map(vip_ctx* c, int64_t width) {
    std::vector<int64_t> m(width, -1);
    int64_t k = 0;
    for (const Geom& g : c->geoms) {
        for (int64_t i = 0; i < g.n; ++i) m[g.row0 + i] = g.off + i;
        if (g.bordered) m[g.row0 + g.n] = c->N + (k++);
    }
    return m;
}

vip_status export_csr(vip_ctx* c, int which, HostCSR& H) {
    cudaStream_t st = c->stream;
    const int64_t R = c->R;
    std::vector<int64_t> map = row_map(c, R);
    bool pois = which == VIP_OP_POISSON;
    int64_t nrows = c->N + (pois ? c->nbordered : 0);
    std::vector<std::vector<std::pair<int32_t, double>>> rows(nrows);
    if (which >= VIP_OP_NBR && which <= VIP_OP_D02) {
        std::vector<int64_t> pp(R + 1);
        VIP_CUDA(cudaMemcpyAsync(pp.data(), c->T.pptr, (R + 1) * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        int64_t nn = pp[R];
        std::vector<int32_t> idx(nn);
        std::vector<double> w(nn, 1.0);
        VIP_CUDA(cudaMemcpyAsync(idx.data(), c->T.pidx, nn * 4, cudaMemcpyDeviceToHost, st));
        if (which == VIP_OP_D00)
            VIP_CUDA(cudaMemcpyAsync(w.data(), c->T.w00, nn * 8, cudaMemcpyDeviceToHost, st));
        else if (which > VIP_OP_D00)
            VIP_CUDA(cudaMemcpyAsync(w.data(), c->T.wd + (int64_t)(which - VIP_OP_D10) * c->T.nnz_nodes,
                                     nn * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        for (int64_t r = 0; r < R; ++r) {
            if (map[r] < 0 || map[r] >= c->N) continue;
            for (int64_t q = pp[r]; q < pp[r + 1]; ++q) rows[map[r]].push_back({(int32_t)map[idx[q]], w[q]});
        }
    } else {
        const Sell* S = nullptr;
        int64_t r0 = 0, coff = 0;
        switch (which) {
            case VIP_OP_LAPLACE: S = &c->T.lap; break;
            case VIP_OP_VIP_E: S = &c->T.ve; break;
            case VIP_OP_VIP_W: S = &c->T.vw; break;
            case VIP_OP_VIP_N: S = &c->T.vn; break;
            case VIP_OP_VIP_S: S = &c->T.vs; break;
            case VIP_OP_GX: S = &c->T.gx; break;
            case VIP_OP_GY: S = &c->T.gy; break;
            case VIP_OP_HELM_U: S = &c->T.helm; break;
            case VIP_OP_HELM_V: S = &c->T.helm; r0 = R; coff = R; break;
            case VIP_OP_POISSON: S = &c->T.pois; break;
            default: return fail(c, VIP_ERR_ARG, "unknown table");
        }
        std::vector<int64_t> sptr(S->nslices + 1);
        std::vector<int32_t> width(S->nslices), rl(S->nrows), col(S->nstored);
        std::vector<double> val(S->nstored);
        VIP_CUDA(cudaMemcpyAsync(sptr.data(), S->sptr, sptr.size() * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(width.data(), S->width, width.size() * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(rl.data(), S->rowlen, rl.size() * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(col.data(), S->col, col.size() * 4, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaMemcpyAsync(val.data(), S->v64, val.size() * 8, cudaMemcpyDeviceToHost, st));
        VIP_CUDA(cudaStreamSynchronize(st));
        for (int64_t rr = 0; rr < R; ++rr) {
            int64_t r = rr + r0;
            int64_t m = map[rr];
            if (m < 0) continue;
            if (!pois && m >= c->N) continue;
            int64_t s = r / SLICE, lane = r % SLICE;
            for (int k = 0; k < rl[r]; ++k) {
                int64_t e = sptr[s] + (int64_t)k * SLICE + lane;
                int64_t cc = map[col[e] - coff];
                rows[m].push_back({(int32_t)cc, val[e]});
            }
        }
    }
    H.ptr.assign(nrows + 1, 0);
    for (int64_t r = 0; r < nrows; ++r) {
        std::sort(rows[r].begin(), rows[r].end());
        H.ptr[r + 1] = H.ptr[r] + (int64_t)rows[r].size();
        for (auto& e : rows[r]) { H.col.push_back(e.first); H.val.push_back(e.second); }
    }
    return VIP_OK;
}

}  // namespace

extern "C" {

vip_status vip_stencil_info(vip_ctx* c, int which, int64_t* nrows, int64_t* nnz) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_stencil_info before vip_build");
    if (which < 0 || which >= VIP_OP_COUNT) return fail(c, VIP_ERR_ARG, "unknown table");
    HostCSR H;
    vip_status s = export_csr(c, which, H);
    if (s != VIP_OK) return s;
    if (nrows) *nrows = (int64_t)H.ptr.size() - 1;
    if (nnz) *nnz = H.ptr.back();
    return VIP_OK;
}

vip_status vip_operator_layout(vip_ctx* c, int which, int64_t* slices, int64_t* uniform_slices,
                               int64_t* uniform_entries, int64_t* other_entries) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_operator_layout before vip_build");
    const Sell* S = nullptr;
    if (which == VIP_OP_HELM_U || which == VIP_OP_HELM_V) S = &c->T.helm;
    else if (which == VIP_OP_POISSON) S = &c->T.pois;
    else return fail(c, VIP_ERR_ARG, "vip_operator_layout: not a Krylov operator");
    if (slices) *slices = S->nslices;
    if (uniform_slices) *uniform_slices = S->nuniform;
    if (uniform_entries) *uniform_entries = S->nuentries;
    if (other_entries) *other_entries = S->nstored_other;
    return VIP_OK;
}

vip_status vip_multigrid_info(vip_ctx* c, int32_t* levels, int64_t* coarsest_entries) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_multigrid_info before vip_build");
    const bool on = c->use_mg && c->mg.built;
    if (levels) *levels = on ? c->mg.nlev : 0;
    if (coarsest_entries) *coarsest_entries = on ? c->mg.cinv_entries : 0;
    return VIP_OK;
}

vip_status vip_get_stencil(vip_ctx* c, int which, int64_t* row_ptr, int32_t* col, double* val) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_get_stencil before vip_build");
    if (which < 0 || which >= VIP_OP_COUNT) return fail(c, VIP_ERR_ARG, "unknown table");
    HostCSR H;
    vip_status s = export_csr(c, which, H);
    if (s != VIP_OK) return s;
    if (row_ptr) VIP_CUDA(cudaMemcpy(row_ptr, H.ptr.data(), H.ptr.size() * 8, cudaMemcpyDefault));
    if (col && !H.col.empty()) VIP_CUDA(cudaMemcpy(col, H.col.data(), H.col.size() * 4, cudaMemcpyDefault));
    if (val && !H.val.empty()) VIP_CUDA(cudaMemcpy(val, H.val.data(), H.val.size() * 8, cudaMemcpyDefault));
    return VIP_OK;
}

vip_status vip_apply(vip_ctx* c, int which, const double* x, double* y) {
    if (!c || !x || !y) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_apply before vip_build");
    const int64_t R = c->R;
    if (which >= VIP_OP_NBR && which <= VIP_OP_D02)
        return fail(c, VIP_ERR_ARG, "vip_apply: MLS point tables are exported, not applied");
    Sell S;
    int64_t off = 0;
    switch (which) {
        case VIP_OP_LAPLACE: S = c->T.lap; break;
        case VIP_OP_VIP_E: S = c->T.ve; break;
        case VIP_OP_VIP_W: S = c->T.vw; break;
        case VIP_OP_VIP_N: S = c->T.vn; break;
        case VIP_OP_VIP_S: S = c->T.vs; break;
        case VIP_OP_GX: S = c->T.gx; break;
        case VIP_OP_GY: S = c->T.gy; break;
        case VIP_OP_HELM_U: case VIP_OP_HELM_V: S = c->T.helm; break;
        case VIP_OP_POISSON: S = c->T.pois; break;
        default: return fail(c, VIP_ERR_ARG, "unknown table");
    }
    double *xp = nullptr, *yp = nullptr;
    VIP_CUDA(cudaMalloc(&xp, 2 * R * 8));
    VIP_CUDA(cudaMalloc(&yp, 2 * R * 8));
    cudaStream_t st = c->stream;
    VIP_CUDA(cudaMemsetAsync(xp, 0, 2 * R * 8, st));
    if (which == VIP_OP_HELM_V) off = R;
    vip_status s = scatter(c, x, xp + off);
    if (s == VIP_OK && which == VIP_OP_POISSON) {  // mu entries
        int64_t k = 0;
        for (const Geom& g : c->geoms)
            if (g.bordered) {
                cudaMemcpyAsync(xp + g.row0 + g.n, x + c->N + k, 8, cudaMemcpyDefault, st);
                ++k;
            }
    }
    if (s == VIP_OK) {
        launch_spmv(S, xp, yp, st);
        s = gather_out(c, yp + off, y);
        if (s == VIP_OK && which == VIP_OP_POISSON) {
            int64_t k = 0;
            for (const Geom& g : c->geoms)
                if (g.bordered) {
                    cudaMemcpyAsync(y + c->N + k, yp + g.row0 + g.n, 8, cudaMemcpyDefault, st);
                    ++k;
                }
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(xp);
    cudaFree(yp);
    if (s != VIP_OK) return s;
    if (e != cudaSuccess) return fail(c, VIP_ERR_CUDA, cudaGetErrorString(e));
    return VIP_OK;
}

vip_status vip_convection(vip_ctx* c, const double* u, const double* v, double* Nu, double* Nv) {
    if (!c || !u || !v || !Nu || !Nv) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_convection before vip_build");
    const int64_t R = c->R;
    double* buf = nullptr;
    VIP_CUDA(cudaMalloc(&buf, 4 * R * 8));
    cudaStream_t st = c->stream;
    VIP_CUDA(cudaMemsetAsync(buf, 0, 4 * R * 8, st));
    vip_status s = scatter(c, u, buf);
    if (s == VIP_OK) s = scatter(c, v, buf + R);
    if (s == VIP_OK) {
        launch_convection(c, buf, buf + R, buf + 2 * R, buf + 3 * R, st);
        s = gather_out(c, buf + 2 * R, Nu);
        if (s == VIP_OK) s = gather_out(c, buf + 3 * R, Nv);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (s != VIP_OK) return s;
    if (e != cudaSuccess) return fail(c, VIP_ERR_CUDA, cudaGetErrorString(e));
    return VIP_OK;
}

vip_status vip_solve(vip_ctx* c, int which, const double* b, double* x, int precision, double rtol,
                     int32_t max_iters, int32_t* iters, double* relres) {
    if (!c || !b || !x) return VIP_ERR_ARG;
    if (!c->built) return fail(c, VIP_ERR_ARG, "vip_solve before vip_build");
    if (which != VIP_OP_HELM_U && which != VIP_OP_HELM_V && which != VIP_OP_POISSON)
        return fail(c, VIP_ERR_ARG, "vip_solve: system must be HELM_U, HELM_V or POISSON");
    if (precision != VIP_PREC_FP64 && precision != VIP_PREC_MIXED && precision != VIP_PREC_MG32)
        return fail(c, VIP_ERR_ARG, "bad precision");
    if (!(rtol > 0.0)) return fail(c, VIP_ERR_ARG, "bad rtol");
    const int64_t R = c->R;
    bool pois = which == VIP_OP_POISSON;
    double *bp = nullptr, *xp = nullptr;
    VIP_CUDA(cudaMalloc(&bp, 2 * R * 8));
    VIP_CUDA(cudaMalloc(&xp, 2 * R * 8));
    cudaStream_t st = c->stream;
    VIP_CUDA(cudaMemsetAsync(bp, 0, 2 * R * 8, st));
    VIP_CUDA(cudaMemsetAsync(xp, 0, 2 * R * 8, st));
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));
    int64_t off = which == VIP_OP_HELM_V ? R : 0;
    vip_status s = scatter(c, b, bp + off);
    if (s == VIP_OK) s = scatter(c, x, xp + off);
    if (s == VIP_OK && pois) {
        int64_t k = 0;
        for (const Geom& g : c->geoms)
            if (g.bordered) {
                cudaMemcpyAsync(bp + g.row0 + g.n, b + c->N + k, 8, cudaMemcpyDefault, st);
                cudaMemcpyAsync(xp + g.row0 + g.n, x + c->N + k, 8, cudaMemcpyDefault, st);
                ++k;
            }
    }
    const KrylovPlan& P = pois ? c->plan_pois : c->plan_helm;
    if (s == VIP_OK) s = krylov_solve(c, P, pois ? c->T.pois : c->T.helm, bp, xp, precision, rtol,
                                      max_iters, c->inner_rtol,
                                      (pois && c->use_mg) ? &c->mg : nullptr);
    if (s == VIP_OK) s = gather_out(c, xp + off, x);
    if (s == VIP_OK && pois) {
        int64_t k = 0;
        for (const Geom& g : c->geoms)
            if (g.bordered) {
                cudaMemcpyAsync(x + c->N + k, xp + g.row0 + g.n, 8, cudaMemcpyDefault, st);
                ++k;
            }
    }
    std::vector<int32_t> it(P.nsys);
    std::vector<double> rr(P.nsys);
    int32_t hs = 0;
    cudaMemcpyAsync(it.data(), P.out_iters, P.nsys * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(rr.data(), P.out_relres, P.nsys * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, c->d_status, 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(bp);
    cudaFree(xp);
    if (s != VIP_OK) return s;
    if (e != cudaSuccess) return fail(c, VIP_ERR_CUDA, cudaGetErrorString(e));
    int32_t mi = 0;
    double mr = 0;
    for (int g = 0; g < P.nsys; ++g) { mi = std::max(mi, it[g]); mr = std::max(mr, rr[g]); }
    if (iters) *iters = mi;
    if (relres) *relres = mr;
    VIP_CUDA(cudaMemsetAsync(c->d_status, 0, 4, st));
    if (hs) {
        c->err = "solve ended with device status " + std::to_string(hs);
        return (vip_status)hs;
    }
    return VIP_OK;
}

}  // extern "C"
