// 3x3 convolution of the warm-start network as an implicit GEMM on the tensor
// cores with warp-level mma.sync (m16n8k16, BF16 x BF16 -> FP32).
//
// A CTA of four warps loops over tiles of 128 consecutive pixels of one lattice
// row (persistent grid).  Per tile it stages the 3 x 130 halo of the input in
// shared memory, channel-chunk planar: plane[c][row][col] holds channels
// 8c..8c+7 (16 bytes) of one pixel, so the nine taps read the same planes at
// shifted pixel offsets (no im2col copy).  The weights stay in shared memory for
// the whole launch as [tap][chunk][cout][8 ci].  Warp w owns pixels 32w..32w+31 of
// the tile (two m16 tiles) and all output channels (Cout/8 n8 tiles); the K loop
// runs over 9 taps x Cin/16.  Fragments are read with 32-bit shared loads
// (two consecutive channels), which are bank-conflict free in this layout.
#include <algorithm>
#include <cstdio>

#include "vip_cnn.cuh"

namespace vip {

constexpr int PLANE_COLS = CNN_TILE + 2;               // 130
constexpr int PLANE_ELEMS = 3 * PLANE_COLS * 8;        // bf16 per chunk plane
constexpr int MAX_CHUNKS = CNN_CH / 8;                 // 4

__device__ __forceinline__ uint32_t ld_s32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int COUT>
__global__ void __launch_bounds__(128) k_conv_mma(CnnConvArgs a) {
    __shared__ __align__(16) __nv_bfloat16 s_in[MAX_CHUNKS * PLANE_ELEMS];
    __shared__ __align__(16) __nv_bfloat16 s_w[9 * MAX_CHUNKS * CNN_CH * 8];
    constexpr int NT = COUT / 8;  // n8 tiles
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 2, tig = lane & 3;
    const int cin = a.cin;
    const int nch = cin / 8;
    // weights [tap][chunk][cout][8]
    const int wvec = 9 * nch * COUT;  // 16-byte vectors
    for (int i = tid; i < wvec; i += blockDim.x)
        reinterpret_cast<uint4*>(s_w)[i] = reinterpret_cast<const uint4*>(a.wpack)[i];

    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        int im = 0;
        while (im + 1 < a.nimg && a.img[im + 1].tile0 <= tile) ++im;
        const CnnImage I = a.img[im];
        const int64_t tloc = tile - I.tile0;
        const int tpr = (I.W + CNN_TILE - 1) / CNN_TILE;
        const int y = (int)(tloc / tpr);
        const int x0 = (int)(tloc % tpr) * CNN_TILE;
        __syncthreads();  // previous tile's reads of s_in are done
        const int nitem = nch * 3 * PLANE_COLS;
        for (int i = tid; i < nitem; i += blockDim.x) {
            int c = i / (3 * PLANE_COLS);
            int rem = i - c * 3 * PLANE_COLS;
            int r = rem / PLANE_COLS;
            int col = rem - r * PLANE_COLS;
            int yy = y - 1 + r, xx = x0 - 1 + col;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < I.H && xx >= 0 && xx < I.W) {
                const int64_t cell = I.off + (int64_t)yy * I.W + xx;
                v = *reinterpret_cast<const uint4*>(a.x + cell * cin + c * 8);
            }
            *reinterpret_cast<uint4*>(s_in + c * PLANE_ELEMS + (r * PLANE_COLS + col) * 8) = v;
        }
        __syncthreads();
        float acc[2][NT][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.0f;
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
            for (int kc = 0; kc < nch / 2; ++kc) {
                const __nv_bfloat16* p0 = s_in + (2 * kc) * PLANE_ELEMS + (dy * PLANE_COLS + dx) * 8;
                const __nv_bfloat16* p1 = p0 + PLANE_ELEMS;
                uint32_t af[2][4];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int px = warp * 32 + m * 16 + grp;
                    af[m][0] = ld_s32(p0 + px * 8 + tig * 2);
                    af[m][1] = ld_s32(p0 + (px + 8) * 8 + tig * 2);
                    af[m][2] = ld_s32(p1 + px * 8 + tig * 2);
                    af[m][3] = ld_s32(p1 + (px + 8) * 8 + tig * 2);
                }
                const __nv_bfloat16* w0 = s_w + ((tap * nch + 2 * kc) * COUT) * 8;
                const __nv_bfloat16* w1 = w0 + COUT * 8;
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int co = n * 8 + grp;
                    uint32_t b0 = ld_s32(w0 + co * 8 + tig * 2);
                    uint32_t b1 = ld_s32(w1 + co * 8 + tig * 2);
#pragma unroll
                    for (int m = 0; m < 2; ++m) mma_bf16_16816(acc[m][n], af[m], b0, b1);
                }
            }
        }
        // epilogue: the thread holds rows grp, grp + 8 and columns 2 tig, 2 tig + 1 of each tile
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int hrow = 0; hrow < 2; ++hrow) {
                const int x = x0 + warp * 32 + m * 16 + grp + hrow * 8;
                if (x >= I.W) continue;
                const int64_t cell = I.off + (int64_t)y * I.W + x;
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int co = n * 8 + tig * 2;
                    float v0 = acc[m][n][2 * hrow], v1 = acc[m][n][2 * hrow + 1];
                    if (a.epi == EPI_F32_CH0) {
                        if (co == 0) a.y32[cell] = v0 + (a.bias ? a.bias[0] : 0.0f);
                        continue;
                    }
                    if (a.epi == EPI_RELU_BF16) {
                        v0 = fmaxf(v0 + a.bias[co], 0.0f);
                        v1 = fmaxf(v1 + a.bias[co + 1], 0.0f);
                    } else {  // gradient through the ReLU of the layer below
                        const __nv_bfloat16* mk = a.mask + cell * COUT + co;
                        v0 = __bfloat162float(mk[0]) > 0.0f ? v0 : 0.0f;
                        v1 = __bfloat162float(mk[1]) > 0.0f ? v1 : 0.0f;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(a.y + cell * COUT + co) =
                        __floats2bfloat162_rn(v0, v1);
                }
            }
    }
}

cudaError_t cnn_conv_init() { return cudaSuccess; }

cudaError_t cnn_conv_fwd(const CnnConvArgs& a, int nsm, cudaStream_t s, const char** why) {
    *why = "";
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *why = "an earlier CUDA call left an error";
        return e;
    }
    if (a.ntiles <= 0) return cudaSuccess;
    if (a.cin % 16 || a.cin > CNN_CH || (a.cout != 16 && a.cout != 32)) {
        *why = "unsupported channel counts";
        return cudaErrorInvalidValue;
    }
    int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)std::max(nsm, 1) * 4);
    if (a.cout == 32) k_conv_mma<32><<<grid, 128, 0, s>>>(a);
    else k_conv_mma<16><<<grid, 128, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) *why = "kernel launch";
    return e;
}

}  // namespace vip
