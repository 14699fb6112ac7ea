// Warm-start network of the pressure-increment solve: internal declarations.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "vip_internal.cuh"

namespace vip {

constexpr int CNN_LAYERS = 6;
constexpr int CNN_CIN = 16;     // input channels (7 used, zero padded)
constexpr int CNN_CH = 32;      // hidden channels
constexpr int CNN_COUT = 16;    // MMA width of the last layer (channel 0 is the output)
constexpr int CNN_TILE = 128;   // pixels of a lattice row per MMA tile (TMEM lanes)

// One lattice image: cells [off, off + H*W) in row-major order.
struct CnnImage {
    int64_t off;
    int32_t H, W;
    int64_t tile0;   // first tile index of the image
};

struct CnnLayerDims {
    int cin, cout;
};

// Layer widths (input, hidden..., output).
__host__ __device__ inline CnnLayerDims cnn_dims(int l) {
    return {l == 0 ? CNN_CIN : CNN_CH, l == CNN_LAYERS - 1 ? CNN_COUT : CNN_CH};
}

// Epilogue of a convolution launch.
enum CnnEpi { EPI_RELU_BF16 = 0, EPI_F32_CH0 = 1, EPI_MASK_BF16 = 2 };

struct CnnConvArgs {
    const __nv_bfloat16* x;      // [cells][cin]
    const __nv_bfloat16* wpack;  // [9][cin/8][cout][8] (MMA layout)
    const float* bias;           // [cout] (may be null)
    const __nv_bfloat16* mask;   // [cells][cout] for EPI_MASK_BF16 (ReLU derivative source)
    __nv_bfloat16* y;            // [cells][cout]
    float* y32;                  // [cells] for EPI_F32_CH0
    const CnnImage* img;
    int nimg;
    int64_t ntiles;
    int cin, cout, epi;
    int32_t* status;
};

// Weight and bias gradients of one layer on the tensor cores (k_wgrad_tc): each block
// accumulates its tiles into one FP32 partial of 9 cin cout + cout entries at
// part + block (9 cin cout + cout), entry (tap cin + ci) cout + co, then the biases.
struct CnnWgradArgs {
    const __nv_bfloat16* x;      // [cells][cin] the layer's input
    const __nv_bfloat16* gy;     // [cells][cout] the gradient wrt its output
    const CnnImage* img;
    int nimg;
    int64_t ntiles;
    int cin, cout;
    float* part;
    int32_t* status;
};

cudaError_t cnn_conv_init();
cudaError_t cnn_wgrad_tc(const CnnWgradArgs& a, int nblocks, cudaStream_t s, const char** why);
cudaError_t cnn_conv_fwd(const CnnConvArgs& a, int nsm, cudaStream_t s, const char** why);

}  // namespace vip
