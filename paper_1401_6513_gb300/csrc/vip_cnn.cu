// Learned warm start of the pressure-increment solve (Eq. 13): a 6-layer 3x3
// convolutional network on the regular background lattice of each geometry
// predicts the change of the increment, phi^{n+1} - phi^n, from the intermediate
// velocity, the divergence right-hand side, the previous increment and node
// masks.  The Krylov solve then runs from phi^n + S * prediction to the same
// residual as without the network.
//
// Inputs per lattice cell (BF16, 16 channels): u*, v*, b / s_b, phi^n / S, 1 at a
// node, 1 at a boundary node, zeros.  s_b = RMS of b over the geometry's interior
// rows, S = RMS of phi^n (s_b h^2 before the first increment exists).
//
// Forward and data-gradient convolutions run on the tensor cores (vip_cnn_conv.cu);
// the weight gradients are reduced in FP32 with fixed-order block partials; Adam
// updates an FP32 master copy from which the BF16 MMA operands are repacked.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "vip_cnn.cuh"

namespace vip {


// parameter offsets of layer l: weights [3][3][cin][cout_real] then bias [cout_real]
struct ParamLayout {
    int64_t w[CNN_LAYERS], b[CNN_LAYERS], total;
    int cin[CNN_LAYERS], cout[CNN_LAYERS], creal[CNN_LAYERS];
};
static ParamLayout param_layout() {
    ParamLayout p;
    int64_t o = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        CnnLayerDims d = cnn_dims(l);
        p.cin[l] = d.cin;
        p.cout[l] = d.cout;
        p.creal[l] = (l == CNN_LAYERS - 1) ? 1 : d.cout;
        p.w[l] = o;
        o += 9LL * d.cin * p.creal[l];
        p.b[l] = o;
        o += p.creal[l];
    }
    p.total = o;
    return p;
}

// pack FP32 weights [3][3][cin][creal] into the MMA layout [tap][cin/8][cout][8]
// (transpose = 1: the data-gradient operator, taps flipped, roles of cin/cout swapped)
__global__ void k_pack(const float* __restrict__ w, int cin, int cout, int creal, int transpose,
                       __nv_bfloat16* __restrict__ out) {
    // forward: K = cin, N = cout; transposed: K = cout, N = cin
    const int K = transpose ? cout : cin;
    const int N = transpose ? cin : cout;
    const int total = 9 * K * N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int tap = i / (K * N);
        int rem = i - tap * K * N;
        int chunk = rem / (N * 8);
        int rem2 = rem - chunk * N * 8;
        int n = rem2 / 8;
        int kk = chunk * 8 + (rem2 % 8);
        float v = 0.0f;
        if (!transpose) {
            if (n < creal) v = w[((int64_t)tap * cin + kk) * creal + n];
        } else {  // W'[tap][co = kk][ci = n] = W[8 - tap][ci][co]
            if (kk < creal) v = w[((int64_t)(8 - tap) * cin + n) * creal + kk];
        }
        out[i] = __float2bfloat16(v);
    }
}

__global__ void k_pack_bias(const float* __restrict__ b, int creal, int cout, float* __restrict__ out) {
    int i = threadIdx.x;
    if (i < cout) out[i] = i < creal ? b[i] : 0.0f;
}

// Per-geometry scales of the network's input, in two fixed-order passes (so the
// same state always gives the same scales).  Pass 1: block (chunk k, geometry g)
// sums, over its share of g's rows, b^2 and 1 at interior nodes, phi^2 at all
// nodes, and (phi - phi_old)^2 at interior nodes; tree sum in shared memory.
constexpr int WS_CHUNKS = 128;   // blocks per geometry in pass 1
__global__ void k_ws_scales_part(const GeomDev* __restrict__ g, const int8_t* __restrict__ rt,
                                 const uint8_t* __restrict__ kind, const double* __restrict__ b,
                                 const double* __restrict__ phi, const double* __restrict__ phi_old,
                                 double* __restrict__ part) {
    __shared__ double sq[4][256];
    const GeomDev& G = g[blockIdx.y];
    const int64_t len = (G.n + WS_CHUNKS - 1) / WS_CHUNKS;
    const int64_t r0 = G.row0 + (int64_t)blockIdx.x * len;
    const int64_t r1 = min(r0 + len, G.row0 + G.n);
    double a = 0, p = 0, n = 0, d = 0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        if (rt[r] != ROW_NODE) continue;
        if (kind[r] == VIP_NODE_INTERIOR) {
            a += b[r] * b[r];
            n += 1.0;
            const double dd = phi[r] - phi_old[r];
            d += dd * dd;
        }
        p += phi[r] * phi[r];
    }
    sq[0][threadIdx.x] = a; sq[1][threadIdx.x] = p; sq[2][threadIdx.x] = n; sq[3][threadIdx.x] = d;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 4; ++q) sq[q][threadIdx.x] += sq[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[((int64_t)blockIdx.y * WS_CHUNKS + blockIdx.x) * 4 + threadIdx.x] = sq[threadIdx.x][0];
}

// Pass 2: one block per geometry sums its chunks' partials (tree sum) and forms
// s_b (RMS of b over interior nodes), S (RMS of phi, or s_b h^2 when phi = 0) and
// D (RMS of (phi - phi_old) / S over interior nodes, 1 when zero).
__global__ void k_ws_scales(const GeomDev* __restrict__ g, const double* __restrict__ part,
                            const double* __restrict__ hlat, double* __restrict__ scales) {
    __shared__ double sq[4][WS_CHUNKS];
    const GeomDev& G = g[blockIdx.x];
    for (int q = 0; q < 4; ++q)
        sq[q][threadIdx.x] = part[((int64_t)blockIdx.x * WS_CHUNKS + threadIdx.x) * 4 + q];
    __syncthreads();
    for (int s = WS_CHUNKS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 4; ++q) sq[q][threadIdx.x] += sq[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double nn = fmax(sq[2][0], 1.0);
        double s_b = sqrt(sq[0][0] / nn) + 1e-300;
        double rp = sqrt(sq[1][0] / (double)G.n);
        double S = rp > 0.0 ? rp : s_b * hlat[blockIdx.x] * hlat[blockIdx.x];
        double D = sqrt(sq[3][0] / nn) / S;
        scales[3 * blockIdx.x] = s_b;
        scales[3 * blockIdx.x + 1] = S;
        scales[3 * blockIdx.x + 2] = D > 0.0 ? D : 1.0;
    }
}

// assemble the network input of every lattice cell (cells without a node stay zero)
__global__ void k_ws_scatter(int64_t R, const int8_t* __restrict__ rt, const uint8_t* __restrict__ kind,
                             const int32_t* __restrict__ rg, const int32_t* __restrict__ node_cell,
                             const double* __restrict__ us, const double* __restrict__ vs,
                             const double* __restrict__ b, const double* __restrict__ phi,
                             const double* __restrict__ phi_old, const double* __restrict__ scales,
                             __nv_bfloat16* __restrict__ x) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int32_t c = node_cell[r];
    if (c < 0 || rt[r] != ROW_NODE) return;
    int g = rg[r];
    double s_b = scales[3 * g], S = scales[3 * g + 1], D = scales[3 * g + 2];
    float v[CNN_CIN];
    for (int i = 0; i < CNN_CIN; ++i) v[i] = 0.0f;
    v[0] = (float)us[r];
    v[1] = (float)vs[r];
    v[2] = (float)(b[r] / s_b);
    v[3] = (float)(phi[r] / S);
    v[4] = 1.0f;
    v[5] = kind[r] != VIP_NODE_INTERIOR ? 1.0f : 0.0f;
    v[6] = (float)((phi[r] - phi_old[r]) / (S * D));
    __nv_bfloat16* dst = x + (int64_t)c * CNN_CIN;
    for (int i = 0; i < CNN_CIN; ++i) dst[i] = __float2bfloat16(v[i]);
}

// phi guess = phi^n + a (phi^n - phi^{n-1}) at every node, + S D * prediction at
// lattice nodes
__global__ void k_ws_gather(int64_t R, const int8_t* __restrict__ rt, const int32_t* __restrict__ rg,
                            const int32_t* __restrict__ node_cell, const uint8_t* __restrict__ deep,
                            const float* __restrict__ y, const double* __restrict__ scales,
                            const double* __restrict__ phi_old, const double* __restrict__ extrap,
                            double* __restrict__ phi) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || rt[r] != ROW_NODE) return;
    double g = phi[r] + extrap[0] * (phi[r] - phi_old[r]);
    const int32_t c = node_cell[r];
    if (c >= 0 && y && deep[c]) g += scales[3 * rg[r] + 1] * scales[3 * rg[r] + 2] * (double)y[c];
    phi[r] = g;
}

// training target (phi^{n+1} - phi^n) / (S D), the history (phi^n - phi^{n-1}) / (S D)
// and the loss mask (interior lattice nodes)
__global__ void k_ws_target(int64_t R, const int8_t* __restrict__ rt, const uint8_t* __restrict__ deep,
                            const int32_t* __restrict__ rg, const int32_t* __restrict__ node_cell,
                            const double* __restrict__ phi_new, const double* __restrict__ phi_n,
                            const double* __restrict__ phi_nm1, const double* __restrict__ scales,
                            float* __restrict__ tgt, float* __restrict__ dprev, float* __restrict__ mask) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int32_t c = node_cell[r];
    if (c < 0 || rt[r] != ROW_NODE) return;
    const double SD = scales[3 * rg[r] + 1] * scales[3 * rg[r] + 2];
    tgt[c] = (float)((phi_new[r] - phi_n[r]) / SD);
    dprev[c] = (float)((phi_n[r] - phi_nm1[r]) / SD);
    mask[c] = deep[c] ? 1.0f : 0.0f;
}

// Block partials of sum m t d and sum m d d over cells (fixed order): the least-squares
// fit of the extrapolation coefficient over the collected samples.
__global__ void k_ws_fit(int64_t n, const float* __restrict__ t, const float* __restrict__ d,
                         const float* __restrict__ m, double* __restrict__ part) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double dm = (double)m[c] * (double)d[c];
        a += dm * (double)t[c];
        b += dm * (double)d[c];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

// MSE loss and its gradient wrt the output channel 0: gy = 2 (y - t) m / count.
// Block partials of the loss in fixed order.
// The target is t - a dp when dp is given (the part of the increment change that the
// extrapolation a (phi^n - phi^{n-1}) leaves), else t.
__global__ void k_loss(int64_t n, const float* __restrict__ y, const float* __restrict__ t,
                       const float* __restrict__ dp, double a, const float* __restrict__ m, double inv_cnt,
                       __nv_bfloat16* __restrict__ gy, double* __restrict__ part) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double tc = dp ? (double)t[c] - a * (double)dp[c] : (double)t[c];
        double d = (double)m[c] * ((double)y[c] - tc);
        acc += d * d;
        __nv_bfloat16* g = gy + c * CNN_COUT;
        g[0] = __float2bfloat16((float)(2.0 * d * inv_cnt));
        for (int k = 1; k < CNN_COUT; ++k) g[k] = __float2bfloat16(0.0f);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Residual-proxy loss (the squared 5-point lattice Laplacian of the error e = m (y -
// (t - a dp)) plus lam e^2, averaged over the active cells; the Poisson residual an
// initial guess leaves is the operator applied to its error, so rough errors cost
// more than smooth ones).  Cells are those of the images img[0..nimg), row-major.
__device__ __forceinline__ int cnn_image_of(const CnnImage* __restrict__ img, int nimg, int64_t c) {
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (img[mid].off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ double cnn_err(int64_t c, const float* __restrict__ y, const float* __restrict__ t,
                                          const float* __restrict__ dp, double a, const float* __restrict__ m) {
    const double tc = dp ? (double)t[c] - a * (double)dp[c] : (double)t[c];
    return (double)m[c] * ((double)y[c] - tc);
}
// sum of f over the four lattice neighbours of cell c (those inside its image)
template <class F>
__device__ __forceinline__ double cnn_nbr_sum(const CnnImage& I, int64_t c, F&& f) {
    const int64_t k = c - I.off;
    const int iy = (int)(k / I.W), ix = (int)(k % I.W);
    double s = 0.0;
    if (ix > 0) s += f(c - 1);
    if (ix + 1 < I.W) s += f(c + 1);
    if (iy > 0) s += f(c - I.W);
    if (iy + 1 < I.H) s += f(c + I.W);
    return s;
}
// pass 1: q(c) = m(c) (Delta e)(c), block partials of q^2 + lam e^2 (fixed order)
__global__ void k_rloss1(int64_t n, const CnnImage* __restrict__ img, int nimg, const float* __restrict__ y,
                         const float* __restrict__ t, const float* __restrict__ dp, double a,
                         const float* __restrict__ m, double lam, float* __restrict__ q,
                         double* __restrict__ part) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const CnnImage I = img[cnn_image_of(img, nimg, c)];
        const double e = cnn_err(c, y, t, dp, a, m);
        const double lap = cnn_nbr_sum(I, c, [&](int64_t j) { return cnn_err(j, y, t, dp, a, m); }) - 4.0 * e;
        const double qc = (double)m[c] * lap;
        q[c] = (float)qc;
        acc += qc * qc + lam * e * e;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}
// pass 2: gradient wrt output channel 0, gy(c) = 2 m(c) ((Delta q)(c) + lam e(c)) / cnt
__global__ void k_rloss2(int64_t n, const CnnImage* __restrict__ img, int nimg, const float* __restrict__ y,
                         const float* __restrict__ t, const float* __restrict__ dp, double a,
                         const float* __restrict__ m, double lam, const float* __restrict__ q,
                         double inv_cnt, __nv_bfloat16* __restrict__ gy) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const CnnImage I = img[cnn_image_of(img, nimg, c)];
    const double lq = cnn_nbr_sum(I, c, [&](int64_t j) { return (double)q[j]; }) - 4.0 * (double)q[c];
    const double g = 2.0 * (double)m[c] * (lq + lam * cnn_err(c, y, t, dp, a, m)) * inv_cnt;
    __nv_bfloat16* o = gy + c * CNN_COUT;
    o[0] = __float2bfloat16((float)g);
    for (int k = 1; k < CNN_COUT; ++k) o[k] = __float2bfloat16(0.0f);
}

// sum block partials in block order into the gradient slots of the layer
__global__ void k_wgrad_sum(const float* __restrict__ part, int nblocks, int cin, int cout, int creal,
                            float* __restrict__ gw, float* __restrict__ gb) {
    const int nent = 9 * cin * cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent + cout; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * (nent + cout) + e];
        if (e < nent) {
            int tap = e / (cin * cout);
            int rem = e - tap * cin * cout;
            int ci = rem / cout, co = rem % cout;
            if (co < creal) gw[((int64_t)tap * cin + ci) * creal + co] = (float)s;
        } else if (e - nent < creal) {
            gb[e - nent] = (float)s;
        }
    }
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct Cnn {
    ParamLayout L;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    int adam_t = 0;
    __nv_bfloat16* wp[CNN_LAYERS] = {};   // forward operands
    __nv_bfloat16* wt[CNN_LAYERS] = {};   // data-gradient operands
    float* bias[CNN_LAYERS] = {};         // padded to the MMA width
    // lattice of the context's geometries
    std::vector<CnnImage> himg;
    CnnImage* img = nullptr;
    int64_t ncells = 0, ntiles = 0;
    int32_t* node_cell = nullptr;
    uint8_t* deep = nullptr;        // [cells] 1: an interior node whose four lattice neighbours are too
    double* hlat = nullptr;
    double* scales = nullptr;
    double* scale_part = nullptr;   // [G][WS_CHUNKS][4] partial sums of the scales
    // activations of one pass: act[0] input, act[1..5] hidden, out (FP32), grads
    __nv_bfloat16* act[CNN_LAYERS] = {};
    float* out = nullptr;
    __nv_bfloat16 *g0 = nullptr, *g1 = nullptr, *gl = nullptr;
    float* wg_part = nullptr;
    int wg_blocks = 0;
    double* loss_part = nullptr;
    int loss_blocks = 0;
    double* phi_prev = nullptr;     // phi^n, kept through the step's solve
    double* phi_old = nullptr;      // phi^{n-1}, the warm start's history
    double* extrap = nullptr;       // [1] the fitted extrapolation coefficient a (device)
    double extrap_host = 0.0;
    // samples
    int max_samples = 0, nsamples = 0;
    int64_t loss_cnt = 0;           // interior lattice nodes (cells of the loss)
    bool collect = false, enable = false;
    bool net = true;                // the guess uses the network (false: extrapolation only)
    int loss_kind = 1;              // 0: mean squared error; 1: residual proxy (k_rloss1/2)
    int32_t fit_window = 0;         // samples of the extrapolation fit: the last ones (0: all)
    double loss_lam = 0.01;         // weight of the squared error in the residual proxy
    float* lq = nullptr;            // [cells] q of the residual proxy
    __nv_bfloat16* s_in = nullptr;
    float *s_tgt = nullptr, *s_mask = nullptr;
    float* s_dprev = nullptr;       // (phi^n - phi^{n-1}) / S of each sample (FP32)
    // test images (vip_cnn_forward / vip_cnn_grads)
    CnnImage* timg = nullptr;
};

}  // namespace vip

using namespace vip;

namespace {

Cnn* cnn_of(vip_ctx* c) { return reinterpret_cast<Cnn*>(c->cnn); }

vip_status fail(vip_ctx* c, vip_status s, const char* m) {
    c->err = m;
    return s;
}

vip_status repack(vip_ctx* c, Cnn& N) {
    for (int l = 0; l < CNN_LAYERS; ++l) {
        k_pack<<<64, 256, 0, c->stream>>>(N.params + N.L.w[l], N.L.cin[l], N.L.cout[l], N.L.creal[l], 0,
                                          N.wp[l]);
        k_pack<<<64, 256, 0, c->stream>>>(N.params + N.L.w[l], N.L.cin[l], N.L.cout[l], N.L.creal[l], 1,
                                          N.wt[l]);
        k_pack_bias<<<1, 32, 0, c->stream>>>(N.params + N.L.b[l], N.L.creal[l], N.L.cout[l], N.bias[l]);
    }
    VIP_CUDA(cudaGetLastError());
    return VIP_OK;
}

// forward over images `img` (ntiles tiles): act[0] holds the input
vip_status forward(vip_ctx* c, Cnn& N, const CnnImage* img, int nimg, int64_t ntiles, __nv_bfloat16* in,
                   cudaStream_t s) {
    const __nv_bfloat16* x = in;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        CnnConvArgs a;
        memset(&a, 0, sizeof(a));
        a.x = x;
        a.wpack = N.wp[l];
        a.bias = N.bias[l];
        a.img = img;
        a.nimg = nimg;
        a.ntiles = ntiles;
        a.cin = N.L.cin[l];
        a.cout = N.L.cout[l];
        a.status = c->d_status;
        if (l == CNN_LAYERS - 1) {
            a.epi = EPI_F32_CH0;
            a.y32 = N.out;
        } else {
            a.epi = EPI_RELU_BF16;
            a.y = N.act[l + 1];
        }
        const char* why = "";
        cudaError_t e = cnn_conv_fwd(a, c->num_sms, s, &why);
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof buf, "network forward, layer %d (cin %d, cout %d, tiles %lld): %s: %s", l,
                     a.cin, a.cout, (long long)a.ntiles, why, cudaGetErrorString(e));
            c->err = buf;
            return VIP_ERR_CUDA;
        }
        if (l + 1 < CNN_LAYERS) x = N.act[l + 1];
    }
    return VIP_OK;
}

// gradients of the loss for the current act[] and out; fills N.grads
vip_status backward(vip_ctx* c, Cnn& N, const CnnImage* img, int nimg, int64_t ntiles, __nv_bfloat16* in,
                    cudaStream_t s) {
    __nv_bfloat16* gy = N.gl;  // [cells][16] gradient wrt the last layer's output
    __nv_bfloat16* bufs[2] = {N.g0, N.g1};
    for (int l = CNN_LAYERS - 1; l >= 0; --l) {
        const __nv_bfloat16* xin = (l == 0) ? in : N.act[l];
        int cin = N.L.cin[l], cout = N.L.cout[l];
        int nb = (int)std::min<int64_t>(ntiles, N.wg_blocks);
        {
            CnnWgradArgs wa;
            wa.x = xin;
            wa.gy = gy;
            wa.img = img;
            wa.nimg = nimg;
            wa.ntiles = ntiles;
            wa.cin = cin;
            wa.cout = cout;
            wa.part = N.wg_part;
            wa.status = c->d_status;
            const char* why = "";
            cudaError_t e = cnn_wgrad_tc(wa, nb, s, &why);
            if (e != cudaSuccess) return fail(c, VIP_ERR_CUDA, why);
        }
        k_wgrad_sum<<<64, 256, 0, s>>>(N.wg_part, nb, cin, cout, N.L.creal[l], N.grads + N.L.w[l],
                                       N.grads + N.L.b[l]);
        VIP_CUDA(cudaGetLastError());
        if (l > 0) {  // gradient wrt the pre-activation of layer l-1
            CnnConvArgs a;
            memset(&a, 0, sizeof(a));
            a.x = gy;
            a.wpack = N.wt[l];
            a.mask = N.act[l];
            a.img = img;
            a.nimg = nimg;
            a.ntiles = ntiles;
            a.cin = cout;
            a.cout = cin;
            a.epi = EPI_MASK_BF16;
            a.y = bufs[l & 1];
            a.status = c->d_status;
            const char* why = "";
            cudaError_t e = cnn_conv_fwd(a, c->num_sms, s, &why);
            if (e != cudaSuccess) {
                c->err = std::string("network data gradient, layer ") + std::to_string(l) + ": " + why +
                         ": " + cudaGetErrorString(e);
                return VIP_ERR_CUDA;
            }
            gy = bufs[l & 1];
        }
    }
    return VIP_OK;
}

vip_status loss_grad(vip_ctx* c, Cnn& N, const CnnImage* img, int nimg, int64_t n, const float* tgt,
                     const float* dprev, double a, const float* mask, double cnt, double* loss_out,
                     cudaStream_t s) {
    int nb = N.loss_blocks;
    if (N.loss_kind == 1) {
        k_rloss1<<<nb, 256, 0, s>>>(n, img, nimg, N.out, tgt, dprev, a, mask, N.loss_lam, N.lq, N.loss_part);
        k_rloss2<<<nblk(n, 256), 256, 0, s>>>(n, img, nimg, N.out, tgt, dprev, a, mask, N.loss_lam, N.lq,
                                              1.0 / std::max(cnt, 1.0), N.gl);
    } else {
        k_loss<<<nb, 256, 0, s>>>(n, N.out, tgt, dprev, a, mask, 1.0 / std::max(cnt, 1.0), N.gl,
                                  N.loss_part);
    }
    VIP_CUDA(cudaGetLastError());
    if (loss_out) {
        std::vector<double> part(nb);
        VIP_CUDA(cudaMemcpyAsync(part.data(), N.loss_part, nb * 8, cudaMemcpyDeviceToHost, s));
        VIP_CUDA(cudaStreamSynchronize(s));
        double L = 0;
        for (double v : part) L += v;
        *loss_out = L / std::max(cnt, 1.0);
    }
    return VIP_OK;
}

vip_status adam(vip_ctx* c, Cnn& N, double lr, cudaStream_t s) {
    N.adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f - powf(b1, (float)N.adam_t), c2 = 1.0f - powf(b2, (float)N.adam_t);
    k_adam<<<nblk(N.L.total, 256), 256, 0, s>>>(N.L.total, N.params, N.grads, N.am, N.av, (float)lr, b1, b2,
                                                1e-8f, c1, c2);
    VIP_CUDA(cudaGetLastError());
    return repack(c, N);
}

vip_status ensure_act(vip_ctx* c, Cnn& N, int64_t ncells) {
    // activation buffers sized for max(ncells of the context, test images)
    static_assert(CNN_CH >= CNN_COUT, "");
    if (N.ncells >= ncells && N.act[0]) return VIP_OK;
    N.ncells = std::max(N.ncells, ncells);
    for (int l = 0; l < CNN_LAYERS; ++l) VIP_CUDA(dalloc(c, &N.act[l], (size_t)N.ncells * CNN_CH));
    VIP_CUDA(dalloc(c, &N.out, N.ncells));
    VIP_CUDA(dalloc(c, &N.g0, (size_t)N.ncells * CNN_CH));
    VIP_CUDA(dalloc(c, &N.g1, (size_t)N.ncells * CNN_CH));
    VIP_CUDA(dalloc(c, &N.gl, (size_t)N.ncells * CNN_COUT));
    VIP_CUDA(dalloc(c, &N.lq, (size_t)N.ncells));
    return VIP_OK;
}

}  // namespace

namespace vip {

// Create the network state (random init with the given seed) and the lattice of
// the context's geometries.  Called from vip_build.
vip_status cnn_setup(vip_ctx* c, uint64_t seed) {
    Cnn* N = new Cnn();
    c->cnn = N;
    N->L = param_layout();
    const int64_t P = N->L.total;
    VIP_CUDA(dalloc(c, &N->params, P));
    VIP_CUDA(dalloc(c, &N->grads, P));
    VIP_CUDA(dalloc(c, &N->am, P));
    VIP_CUDA(dalloc(c, &N->av, P));
    VIP_CUDA(cudaMemsetAsync(N->am, 0, P * 4, c->stream));
    VIP_CUDA(cudaMemsetAsync(N->av, 0, P * 4, c->stream));
    VIP_CUDA(cudaMemsetAsync(N->grads, 0, P * 4, c->stream));
    {   // He-style initialisation, last layer zero so that the untrained network
        // reproduces the previous-increment guess exactly
        std::vector<float> h(P, 0.0f);
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        for (int l = 0; l < CNN_LAYERS - 1; ++l) {
            float sd = sqrtf(2.0f / (9.0f * N->L.cin[l]));
            for (int64_t i = 0; i < 9LL * N->L.cin[l] * N->L.creal[l]; ++i) h[N->L.w[l] + i] = sd * nd(rng);
        }
        VIP_CUDA(cudaMemcpy(N->params, h.data(), P * 4, cudaMemcpyHostToDevice));
    }
    for (int l = 0; l < CNN_LAYERS; ++l) {
        VIP_CUDA(dalloc(c, &N->wp[l], 9 * N->L.cin[l] * N->L.cout[l]));
        VIP_CUDA(dalloc(c, &N->wt[l], 9 * N->L.cin[l] * N->L.cout[l]));
        VIP_CUDA(dalloc(c, &N->bias[l], CNN_CH));
    }
    VIP_CUDA(cnn_conv_init());
    vip_status st = repack(c, *N);
    if (st != VIP_OK) return st;
    // lattice per geometry: spacing = smallest local spacing, origin = lower-left node
    const int G = (int)c->geoms.size();
    int64_t off = 0, tile0 = 0;
    std::vector<double> hl(G);
    std::vector<int32_t> cell(c->R, -1);
    for (int g = 0; g < G; ++g) {
        const Geom& gg = c->geoms[g];
        double h = 1e300, x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
        for (int64_t i = gg.off; i < gg.off + gg.n; ++i) {
            h = std::min(h, c->hh[i]);
            x0 = std::min(x0, c->hx[i]); x1 = std::max(x1, c->hx[i]);
            y0 = std::min(y0, c->hy[i]); y1 = std::max(y1, c->hy[i]);
        }
        int W = (int)llround((x1 - x0) / h) + 1, H = (int)llround((y1 - y0) / h) + 1;
        CnnImage I;
        I.off = off;
        I.H = H;
        I.W = W;
        I.tile0 = tile0;
        N->himg.push_back(I);
        hl[g] = h;
        for (int64_t i = 0; i < gg.n; ++i) {
            double fx = (c->hx[gg.off + i] - x0) / h, fy = (c->hy[gg.off + i] - y0) / h;
            long long ix = llround(fx), iy = llround(fy);
            if (std::fabs(fx - ix) < 1e-6 && std::fabs(fy - iy) < 1e-6 && ix >= 0 && ix < W && iy >= 0 &&
                iy < H) {
                cell[gg.row0 + i] = (int32_t)(off + iy * W + ix);
            }
        }
        off += (int64_t)W * H;
        tile0 += (int64_t)H * ((W + CNN_TILE - 1) / CNN_TILE);
    }
    N->ntiles = tile0;
    VIP_CUDA(dalloc(c, &N->img, G));
    VIP_CUDA(cudaMemcpy(N->img, N->himg.data(), G * sizeof(CnnImage), cudaMemcpyHostToDevice));
    VIP_CUDA(dalloc(c, &N->node_cell, c->R));
    VIP_CUDA(cudaMemcpy(N->node_cell, cell.data(), c->R * 4, cudaMemcpyHostToDevice));
    {   // cells where the network's correction applies (and is trained): interior nodes
        // whose four lattice neighbours are interior nodes too, away from boundary nodes
        // off the lattice, where a correction that stopped short would leave a jump
        std::vector<uint8_t> inner(off, 0), dp(off, 0);
        for (int g = 0; g < G; ++g) {
            const Geom& gg = c->geoms[g];
            for (int64_t i = 0; i < gg.n; ++i) {
                const int32_t cc = cell[gg.row0 + i];
                if (cc >= 0 && c->hkind[gg.off + i] == VIP_NODE_INTERIOR) inner[cc] = 1;
            }
        }
        for (const CnnImage& I : N->himg)
            for (int iy = 1; iy + 1 < I.H; ++iy)
                for (int ix = 1; ix + 1 < I.W; ++ix) {
                    const int64_t cc = I.off + (int64_t)iy * I.W + ix;
                    dp[cc] = inner[cc] && inner[cc - 1] && inner[cc + 1] && inner[cc - I.W] && inner[cc + I.W];
                }
        int64_t nd = 0;
        for (uint8_t v : dp) nd += v;
        N->loss_cnt = nd;
        VIP_CUDA(dalloc(c, &N->deep, off));
        VIP_CUDA(cudaMemcpy(N->deep, dp.data(), off, cudaMemcpyHostToDevice));
    }
    VIP_CUDA(dalloc(c, &N->hlat, G));
    VIP_CUDA(cudaMemcpy(N->hlat, hl.data(), G * 8, cudaMemcpyHostToDevice));
    VIP_CUDA(dalloc(c, &N->scales, 3 * G));
    VIP_CUDA(dalloc(c, &N->scale_part, (size_t)G * WS_CHUNKS * 4));
    VIP_CUDA(dalloc(c, &N->phi_prev, c->R));
    VIP_CUDA(dalloc(c, &N->phi_old, c->R));
    VIP_CUDA(dalloc(c, &N->extrap, 1));
    VIP_CUDA(cudaMemsetAsync(N->phi_old, 0, c->R * 8, c->stream));
    VIP_CUDA(cudaMemsetAsync(N->extrap, 0, 8, c->stream));
    st = ensure_act(c, *N, off);
    if (st != VIP_OK) return st;
    N->ncells = off;
    N->wg_blocks = std::max(1, c->num_sms * 2);
    VIP_CUDA(dalloc(c, &N->wg_part, (size_t)N->wg_blocks * (9 * CNN_CH * CNN_CH + CNN_CH)));
    N->loss_blocks = 256;
    VIP_CUDA(dalloc(c, &N->loss_part, N->loss_blocks));
    VIP_CUDA(dalloc(c, &N->timg, 1));
    VIP_CUDA(cudaStreamSynchronize(c->stream));
    return VIP_OK;
}

void cnn_free(vip_ctx* c) {
    delete cnn_of(c);
    c->cnn = nullptr;
}

// Warm start of the Poisson solve: called inside the step after the divergence.
vip_status cnn_warm_start(vip_ctx* c, cudaStream_t s) {
    Cnn* N = cnn_of(c);
    if (!N || (!N->enable && !N->collect)) return VIP_OK;
    const int64_t R = c->R;
    VIP_CUDA(cudaMemcpyAsync(N->phi_prev, c->phi, R * 8, cudaMemcpyDeviceToDevice, s));
    if (N->collect || (N->enable && N->net)) {  // the network's input (the extrapolation alone needs none)
        k_ws_scales_part<<<dim3(WS_CHUNKS, (unsigned)c->geoms.size()), 256, 0, s>>>(
            c->gdev, c->row_type, c->kind, c->prhs, c->phi, N->phi_old, N->scale_part);
        k_ws_scales<<<(unsigned)c->geoms.size(), WS_CHUNKS, 0, s>>>(c->gdev, N->scale_part, N->hlat,
                                                                    N->scales);
        VIP_CUDA(cudaMemsetAsync(N->act[0], 0, (size_t)N->ncells * CNN_CIN * 2, s));
        k_ws_scatter<<<nblk(R, 256), 256, 0, s>>>(R, c->row_type, c->kind, c->row_geom, N->node_cell, c->hsol,
                                                   c->hsol + R, c->prhs, c->phi, N->phi_old, N->scales,
                                                   N->act[0]);
        VIP_CUDA(cudaGetLastError());
    }
    if (N->enable) {
        if (N->net) {
            vip_status st = forward(c, *N, N->img, (int)N->himg.size(), N->ntiles, N->act[0], s);
            if (st != VIP_OK) return st;
        }
        k_ws_gather<<<nblk(R, 256), 256, 0, s>>>(R, c->row_type, c->row_geom, N->node_cell, N->deep,
                                                  N->net ? N->out : nullptr, N->scales, N->phi_old, N->extrap,
                                                  c->phi);
        VIP_CUDA(cudaGetLastError());
    }
    return VIP_OK;
}

// phi^{n-1} := phi (the next step's history is then no change), outside any step
vip_status cnn_reset_history(vip_ctx* c) {
    Cnn* N = cnn_of(c);
    if (!N) return VIP_OK;
    VIP_CUDA(cudaMemcpyAsync(N->phi_old, c->phi, c->R * 8, cudaMemcpyDeviceToDevice, c->stream));
    return VIP_OK;
}

double* cnn_history(vip_ctx* c) {
    Cnn* N = cnn_of(c);
    return N ? N->phi_old : nullptr;
}

// After the solve: store (input, target, history) when collecting, and move the
// history on: phi^{n-1} := phi^n.
vip_status cnn_after_solve(vip_ctx* c, cudaStream_t s) {
    Cnn* N = cnn_of(c);
    if (!N || (!N->enable && !N->collect)) return VIP_OK;
    if (N->collect && N->nsamples < N->max_samples) {
        const int64_t nc = N->ncells;
        const int k = N->nsamples;
        VIP_CUDA(cudaMemcpyAsync(N->s_in + (int64_t)k * nc * CNN_CIN, N->act[0], nc * CNN_CIN * 2,
                                 cudaMemcpyDeviceToDevice, s));
        VIP_CUDA(cudaMemsetAsync(N->s_tgt + (int64_t)k * nc, 0, nc * 4, s));
        VIP_CUDA(cudaMemsetAsync(N->s_dprev + (int64_t)k * nc, 0, nc * 4, s));
        VIP_CUDA(cudaMemsetAsync(N->s_mask + (int64_t)k * nc, 0, nc * 4, s));
        k_ws_target<<<nblk(c->R, 256), 256, 0, s>>>(c->R, c->row_type, N->deep, c->row_geom, N->node_cell,
                                                     c->phi, N->phi_prev, N->phi_old, N->scales,
                                                     N->s_tgt + (int64_t)k * nc, N->s_dprev + (int64_t)k * nc,
                                                     N->s_mask + (int64_t)k * nc);
        VIP_CUDA(cudaGetLastError());
        N->nsamples++;
    }
    VIP_CUDA(cudaMemcpyAsync(N->phi_old, N->phi_prev, c->R * 8, cudaMemcpyDeviceToDevice, s));
    return VIP_OK;
}

bool cnn_collecting(vip_ctx* c) {
    Cnn* N = cnn_of(c);
    return N && N->collect;
}

}  // namespace vip

extern "C" {

vip_status vip_ws_collect(vip_ctx* c, int enable, int32_t max_samples) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_collect before vip_build");
    Cnn& N = *cnn_of(c);
    if (enable) {
        if (max_samples < 1) return fail(c, VIP_ERR_ARG, "max_samples must be >= 1");
        if (max_samples > N.max_samples) {
            VIP_CUDA(dalloc(c, &N.s_in, (size_t)max_samples * N.ncells * CNN_CIN));
            VIP_CUDA(dalloc(c, &N.s_tgt, (size_t)max_samples * N.ncells));
            VIP_CUDA(dalloc(c, &N.s_dprev, (size_t)max_samples * N.ncells));
            VIP_CUDA(dalloc(c, &N.s_mask, (size_t)max_samples * N.ncells));
            N.max_samples = max_samples;
        }
        N.nsamples = 0;
        if (!N.collect && !N.enable) {
            vip_status st = cnn_reset_history(c);
            if (st != VIP_OK) return st;
        }
    }
    N.collect = enable != 0;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return VIP_OK;
}

vip_status vip_ws_enable(vip_ctx* c, int enable) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_enable before vip_build");
    Cnn& N = *cnn_of(c);
    if (enable && !N.enable && !N.collect) {
        vip_status st = cnn_reset_history(c);
        if (st != VIP_OK) return st;
    }
    if (enable < 0 || enable > 2) return fail(c, VIP_ERR_ARG, "vip_ws_enable: mode must be 0, 1 or 2");
    N.enable = enable != 0;
    N.net = enable != 2;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return VIP_OK;
}

vip_status vip_ws_train(vip_ctx* c, vip_train_cfg* cfg) {
    if (!c || !cfg) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_train before vip_build");
    Cnn& N = *cnn_of(c);
    if (N.nsamples < 1) return fail(c, VIP_ERR_ARG, "no collected samples");
    if (cfg->epochs < 1 || !(cfg->lr > 0)) return fail(c, VIP_ERR_ARG, "bad training settings");
    cudaStream_t s = c->stream;
    std::mt19937_64 rng(cfg->seed);
    std::vector<int> order(N.nsamples);
    for (int i = 0; i < N.nsamples; ++i) order[i] = i;
    const int64_t nc = N.ncells;
    const CnnImage* img = N.img;
    const int nimg = (int)N.himg.size();
    // the extrapolation coefficient: least squares over the collected samples'
    // interior lattice nodes (every sample, or the last fit_window), a = sum t d /
    // sum d d (t the increment change, d the previous one, both / S); the network
    // then learns what a d leaves of t
    {
        const int fb = 256;
        DeviceScratch d_part;
        VIP_CUDA(cudaMalloc(&d_part.p, 2 * fb * sizeof(double)));
        std::vector<double> part(2 * fb);
        double num = 0.0, den = 0.0;
        const int kfirst = N.fit_window > 0 ? std::max(0, N.nsamples - N.fit_window) : 0;
        for (int k = kfirst; k < N.nsamples; ++k) {
            k_ws_fit<<<fb, 256, 0, s>>>(nc, N.s_tgt + (int64_t)k * nc, N.s_dprev + (int64_t)k * nc,
                                        N.s_mask + (int64_t)k * nc, static_cast<double*>(d_part.p));
            VIP_CUDA(cudaGetLastError());
            VIP_CUDA(cudaMemcpyAsync(part.data(), d_part.p, 2 * fb * 8, cudaMemcpyDeviceToHost, s));
            VIP_CUDA(cudaStreamSynchronize(s));
            for (int b = 0; b < fb; ++b) { num += part[2 * b]; den += part[2 * b + 1]; }
        }
        double a = den > 0.0 ? num / den : 0.0;
        a = std::min(2.0, std::max(-1.0, a));  // a guess beyond these is no extrapolation
        N.extrap_host = a;
        VIP_CUDA(cudaMemcpyAsync(N.extrap, &N.extrap_host, 8, cudaMemcpyHostToDevice, s));
        cfg->extrap = a;
    }
    double last = 0.0;
    for (int ep = 0; ep < cfg->epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        double sum = 0.0;
        for (int k : order) {
            __nv_bfloat16* in = N.s_in + (int64_t)k * nc * CNN_CIN;
            vip_status st = forward(c, N, img, nimg, N.ntiles, in, s);
            if (st != VIP_OK) return st;
            double cnt = (double)N.loss_cnt;
            double L = 0.0;
            st = loss_grad(c, N, img, nimg, nc, N.s_tgt + (int64_t)k * nc, N.s_dprev + (int64_t)k * nc,
                           N.extrap_host, N.s_mask + (int64_t)k * nc, cnt, &L, s);
            if (st != VIP_OK) return st;
            st = backward(c, N, img, nimg, N.ntiles, in, s);
            if (st != VIP_OK) return st;
            st = adam(c, N, cfg->lr, s);
            if (st != VIP_OK) return st;
            sum += L;
        }
        last = sum / N.nsamples;
        if (ep == 0) cfg->first_loss = last;
    }
    (void)last;
    // Keep the network only if, on its own samples, it leaves less than the
    // extrapolation alone: the mean loss with the trained network and with its output
    // zero.  Otherwise its last layer is zeroed, so the guess is the extrapolation.
    {
        double net = 0.0, base = 0.0;
        for (int k = 0; k < N.nsamples; ++k) {
            __nv_bfloat16* in = N.s_in + (int64_t)k * nc * CNN_CIN;
            const float* tk = N.s_tgt + (int64_t)k * nc;
            const float* dk = N.s_dprev + (int64_t)k * nc;
            const float* mk = N.s_mask + (int64_t)k * nc;
            double L = 0.0;
            vip_status st = forward(c, N, img, nimg, N.ntiles, in, s);
            if (st != VIP_OK) return st;
            if ((st = loss_grad(c, N, img, nimg, nc, tk, dk, N.extrap_host, mk, (double)N.loss_cnt, &L, s)) != VIP_OK)
                return st;
            net += L;
            VIP_CUDA(cudaMemsetAsync(N.out, 0, nc * sizeof(float), s));
            if ((st = loss_grad(c, N, img, nimg, nc, tk, dk, N.extrap_host, mk, (double)N.loss_cnt, &L, s)) != VIP_OK)
                return st;
            base += L;
        }
        net /= N.nsamples;
        base /= N.nsamples;
        cfg->final_loss = net;
        cfg->base_loss = base;
        cfg->net_kept = net < base ? 1 : 0;
        if (!cfg->net_kept) {
            const int l = CNN_LAYERS - 1;
            VIP_CUDA(cudaMemsetAsync(N.params + N.L.w[l], 0, (N.L.total - N.L.w[l]) * sizeof(float), s));
            vip_status st = repack(c, N);
            if (st != VIP_OK) return st;
        }
    }
    VIP_CUDA(cudaStreamSynchronize(s));
    int32_t hs = 0;
    VIP_CUDA(cudaMemcpy(&hs, c->d_status, 4, cudaMemcpyDeviceToHost));
    if (hs) return fail(c, (vip_status)hs, "device error during training");
    return VIP_OK;
}

vip_status vip_ws_set_loss(vip_ctx* c, int kind, double lam) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_set_loss before vip_build");
    if ((kind != 0 && kind != 1) || !(lam >= 0.0)) return fail(c, VIP_ERR_ARG, "vip_ws_set_loss: bad kind or weight");
    Cnn& N = *cnn_of(c);
    N.loss_kind = kind;
    N.loss_lam = lam;
    return VIP_OK;
}

vip_status vip_ws_set_fit_window(vip_ctx* c, int32_t window) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_set_fit_window before vip_build");
    if (window < 0) return fail(c, VIP_ERR_ARG, "vip_ws_set_fit_window: window must be >= 0");
    cnn_of(c)->fit_window = window;
    return VIP_OK;
}

vip_status vip_ws_extrapolation(vip_ctx* c, int set, double* a) {
    if (!c || !a) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_extrapolation before vip_build");
    Cnn& N = *cnn_of(c);
    if (!set) {
        *a = N.extrap_host;
        return VIP_OK;
    }
    if (!(*a >= -1.0 && *a <= 2.0)) return fail(c, VIP_ERR_ARG, "vip_ws_extrapolation: a must be in [-1, 2]");
    N.extrap_host = *a;
    VIP_CUDA(cudaMemcpyAsync(N.extrap, &N.extrap_host, 8, cudaMemcpyHostToDevice, c->stream));
    VIP_CUDA(cudaStreamSynchronize(c->stream));
    return VIP_OK;
}

vip_status vip_ws_adam(vip_ctx* c, double lr) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_adam before vip_build");
    if (!(lr > 0)) return fail(c, VIP_ERR_ARG, "vip_ws_adam: lr must be > 0");
    Cnn& N = *cnn_of(c);
    vip_status st = adam(c, N, lr, c->stream);
    if (st != VIP_OK) return st;
    VIP_CUDA(cudaStreamSynchronize(c->stream));
    return VIP_OK;
}

vip_status vip_ws_params(vip_ctx* c, int direction, float* buf, int64_t* count) {
    if (!c) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_params before vip_build");
    Cnn& N = *cnn_of(c);
    if (count) *count = N.L.total;
    if (!buf) return VIP_OK;
    if (direction == 0) {
        VIP_CUDA(cudaMemcpy(buf, N.params, N.L.total * 4, cudaMemcpyDefault));
    } else {
        VIP_CUDA(cudaMemcpy(N.params, buf, N.L.total * 4, cudaMemcpyDefault));
        N.adam_t = 0;
        VIP_CUDA(cudaMemset(N.am, 0, N.L.total * 4));
        VIP_CUDA(cudaMemset(N.av, 0, N.L.total * 4));
        vip_status st = repack(c, N);
        if (st != VIP_OK) return st;
        VIP_CUDA(cudaStreamSynchronize(c->stream));
    }
    return VIP_OK;
}

vip_status vip_ws_eval(vip_ctx* c, int32_t H, int32_t W, const float* x, float* y, float* grads,
                       const float* target, const float* mask, double* loss) {
    if (!c || !x || H < 1 || W < 1) return VIP_ERR_ARG;
    if (!c->built || !c->cnn) return fail(c, VIP_ERR_ARG, "vip_ws_eval before vip_build");
    Cnn& N = *cnn_of(c);
    {   // the layer table must be the one built at set-up
        ParamLayout ref = param_layout();
        for (int l = 0; l < CNN_LAYERS; ++l)
            if (N.L.cin[l] != ref.cin[l] || N.L.cout[l] != ref.cout[l]) {
                char buf[256];
                snprintf(buf, sizeof buf, "network state corrupted: layer %d has cin %d cout %d (expected %d %d)",
                         l, N.L.cin[l], N.L.cout[l], ref.cin[l], ref.cout[l]);
                c->err = buf;
                return VIP_ERR_ARG;
            }
    }
    const int64_t n = (int64_t)H * W;
    vip_status st = ensure_act(c, N, n);
    if (st != VIP_OK) return st;
    cudaStream_t s = c->stream;
    CnnImage I;
    I.off = 0; I.H = H; I.W = W; I.tile0 = 0;
    VIP_CUDA(cudaMemcpyAsync(N.timg, &I, sizeof(I), cudaMemcpyHostToDevice, s));
    int64_t ntiles = (int64_t)H * ((W + CNN_TILE - 1) / CNN_TILE);
    // input: FP32 [H][W][16] -> BF16
    std::vector<float> hx(n * CNN_CIN);
    VIP_CUDA(cudaMemcpy(hx.data(), x, n * CNN_CIN * 4, cudaMemcpyDefault));
    std::vector<__nv_bfloat16> hb(n * CNN_CIN);
    for (int64_t i = 0; i < n * CNN_CIN; ++i) hb[i] = __float2bfloat16(hx[i]);
    __nv_bfloat16* in = nullptr;
    VIP_CUDA(cudaMalloc(&in, n * CNN_CIN * 2));
    VIP_CUDA(cudaMemcpyAsync(in, hb.data(), n * CNN_CIN * 2, cudaMemcpyHostToDevice, s));
    st = forward(c, N, N.timg, 1, ntiles, in, s);
    if (st == VIP_OK && y) VIP_CUDA(cudaMemcpyAsync(y, N.out, n * 4, cudaMemcpyDefault, s));
    if (st == VIP_OK && grads && target && mask) {
        float *dt = nullptr, *dm = nullptr;
        VIP_CUDA(cudaMalloc(&dt, n * 4));
        VIP_CUDA(cudaMalloc(&dm, n * 4));
        VIP_CUDA(cudaMemcpyAsync(dt, target, n * 4, cudaMemcpyDefault, s));
        VIP_CUDA(cudaMemcpyAsync(dm, mask, n * 4, cudaMemcpyDefault, s));
        std::vector<float> hmk(n);
        VIP_CUDA(cudaMemcpy(hmk.data(), mask, n * 4, cudaMemcpyDefault));
        double cnt = 0;
        for (float v : hmk) cnt += v != 0.0f;
        st = loss_grad(c, N, N.timg, 1, n, dt, nullptr, 0.0, dm, cnt, loss, s);
        if (st == VIP_OK) st = backward(c, N, N.timg, 1, ntiles, in, s);
        if (st == VIP_OK) VIP_CUDA(cudaMemcpyAsync(grads, N.grads, N.L.total * 4, cudaMemcpyDefault, s));
        VIP_CUDA(cudaStreamSynchronize(s));
        cudaFree(dt);
        cudaFree(dm);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(in);
    if (st != VIP_OK) return st;
    if (e != cudaSuccess) return fail(c, VIP_ERR_CUDA, cudaGetErrorString(e));
    int32_t hs = 0;
    VIP_CUDA(cudaMemcpy(&hs, c->d_status, 4, cudaMemcpyDeviceToHost));
    if (hs) return fail(c, (vip_status)hs, "device error in the network kernels");
    return VIP_OK;
}

}  // extern "C"
