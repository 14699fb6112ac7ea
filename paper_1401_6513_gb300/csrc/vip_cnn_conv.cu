// 3x3 convolution of the warm-start network as an implicit GEMM on the 5th-generation
// tensor cores (tcgen05, kind::f16: BF16 x BF16 -> FP32 accumulators in TMEM).
//
// A CTA loops over tiles of 128 consecutive pixels of one lattice row (persistent
// grid).  Per tile it stages the 3 x 130 halo of the input in shared memory,
// channel-chunk planar: plane[c][row][col] holds channels 8c..8c+7 (16 bytes) of one
// pixel.  In that layout the 8-pixel x 8-channel core matrices of the MMA operand A
// are 128 contiguous bytes, so every one of the nine taps is the same operand seen
// from a shifted start address -- no im2col copy.  The weights sit in shared memory
// for the whole launch in the same core-matrix layout ([tap][chunk][cout][8 ci]).
// One thread issues 9 * Cin/16 MMAs (K = 16 each) and commits them to an mbarrier;
// the four warps then read their 32 TMEM lanes with tcgen05.ld and run the epilogue.
//
// Pipeline: two halo buffers and two TMEM accumulators.  The halo of a tile is
// fetched with cp.async (16-byte copies, zero-filled outside the image), so all of a
// thread's copies are in flight at once, and the tile after next is fetched while
// the current tile's MMAs run and the previous tile's epilogue drains its
// accumulator: in iteration k the CTA waits for the MMAs of tile k, issues those of
// tile k+1 (whose halo landed during iteration k-1), starts the copies of tile k+2
// into the buffer tile k has released, and then runs tile k's epilogue.  Every
// mbarrier wait is bounded (2 s, then VIP_ERR_TIMEOUT); TMEM is always freed.
#include <algorithm>
#include <cstdio>

#include "vip_cnn.cuh"

namespace vip {

constexpr int PLANE_COLS = CNN_TILE + 2;               // 130
constexpr int PLANE_BYTES = 3 * PLANE_COLS * 16;       // 6240
constexpr int MAX_CHUNKS = CNN_CH / 8;                 // 4
constexpr int SMEM_IN = MAX_CHUNKS * PLANE_BYTES;      // 24960
constexpr int SMEM_W = 9 * MAX_CHUNKS * CNN_CH * 16;   // 18432
// Two halo buffers, the weights, two mbarriers, the TMEM address word and the
// failure flag: three CTAs (3 x 64 TMEM columns) per SM.
constexpr int SMEM_CONV = 2 * SMEM_IN + SMEM_W + 64;
constexpr int CONV_CTAS_PER_SM = 3;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle, K-major operand: start address,
// leading-dimension (K direction) and stride-dimension (M/N direction) byte
// offsets between 8x16-byte core matrices, all >> 4, and the descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and
// B (bits 7-9 = 1, 10-12 = 1), both K-major, N/8 at bit 17, M/16 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false after 2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    uint64_t t0 = gtime();
    while (!mbar_try_wait(bar, parity)) {
        if (gtime() - t0 > 2000000000ull) return false;
    }
    return true;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous copy global -> shared; src_bytes 0 writes zeros (the source
// address is then not read, but is still a valid one).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Where tile t lies: its image, lattice row and first column.
struct ConvTile {
    CnnImage I;
    int y, x0;
};
__device__ __forceinline__ ConvTile conv_tile_of(const CnnImage* img, int nimg, int64_t tile) {
    int im = 0;
    while (im + 1 < nimg && img[im + 1].tile0 <= tile) ++im;
    ConvTile t;
    t.I = img[im];
    const int64_t tloc = tile - t.I.tile0;
    const int tpr = (t.I.W + CNN_TILE - 1) / CNN_TILE;  // tiles per row
    t.y = (int)(tloc / tpr);
    t.x0 = (int)(tloc % tpr) * CNN_TILE;
    return t;
}
__device__ __forceinline__ ConvTile conv_tile(const CnnConvArgs& a, int64_t tile) {
    return conv_tile_of(a.img, a.nimg, tile);
}

// Start the copies of a tile's halo into the planes at buf: [chunk][3][130] x 16
// bytes, zero outside the image.  One commit group per call.
__device__ __forceinline__ void conv_stage(const CnnConvArgs& a, const ConvTile& t, uint32_t buf,
                                           int nch, int tid) {
    const int nitem = nch * 3 * PLANE_COLS;
    for (int i = tid; i < nitem; i += blockDim.x) {
        const int c = i / (3 * PLANE_COLS);
        const int rem = i - c * 3 * PLANE_COLS;
        const int r = rem / PLANE_COLS;
        const int col = rem - r * PLANE_COLS;
        const int yy = t.y - 1 + r, xx = t.x0 - 1 + col;
        const bool in = yy >= 0 && yy < t.I.H && xx >= 0 && xx < t.I.W;
        const __nv_bfloat16* src = a.x;
        if (in) src = a.x + (t.I.off + (int64_t)yy * t.I.W + xx) * a.cin + c * 8;
        cp_async16(buf + c * PLANE_BYTES + (r * PLANE_COLS + col) * 16, src, in ? 16u : 0u);
    }
    cp_async_commit();
}

// The 9 * Cin/16 MMAs of one tile: halo planes at in_addr, accumulator at tmem_d.
__device__ __forceinline__ void conv_mma(uint32_t in_addr, uint32_t w_base, uint32_t tmem_d,
                                         uint32_t idesc, int nch, int cout) {
    uint32_t acc = 0;
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;  // 0..2 = offset + 1
        for (int kc = 0; kc < nch / 2; ++kc) {
            const uint32_t aaddr = in_addr + (2 * kc) * PLANE_BYTES + (dy * PLANE_COLS + dx) * 16;
            const uint32_t baddr = w_base + (tap * nch + 2 * kc) * cout * 16;
            umma_bf16(tmem_d, umma_desc(aaddr, PLANE_BYTES, 128), umma_desc(baddr, cout * 16, 128),
                      idesc, acc);
            acc = 1;
        }
    }
}

__global__ void __launch_bounds__(128) k_conv_tc(CnnConvArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* s_w = smem + 2 * SMEM_IN;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + 2 * SMEM_IN + SMEM_W);  // [2]
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + 2 * SMEM_IN + SMEM_W + 16);
    int* s_fail = reinterpret_cast<int*>(smem + 2 * SMEM_IN + SMEM_W + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin = a.cin, cout = a.cout;
    const int nch = cin / 8;
    const int ncol = 64;  // TMEM columns: two accumulators of 32 (>= cout) columns

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(s_bar, 1);
        mbar_init(s_bar + 1, 1);
        *s_fail = 0;
    }
    // weights, already in [tap][chunk][cout][8] order: one 16-byte copy per thread step
    const int wbytes = 9 * nch * cout * 16;
    for (int i = tid; i < wbytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(s_w)[i] = reinterpret_cast<const uint4*>(a.wpack)[i];
    // this CTA's tiles: blockIdx.x + k gridDim.x, k < nt
    const int64_t nt = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t in_base = smem_u32(smem);
    if (nt > 0) conv_stage(a, conv_tile(a, blockIdx.x), in_base, nch, tid);
    if (nt > 1) conv_stage(a, conv_tile(a, blockIdx.x + gridDim.x), in_base + SMEM_IN, nch, tid);
    cp_async_wait_all();  // tile 0's halo (tile 1's may still be in flight with it; both wait)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = umma_idesc(CNN_TILE, cout);
    const uint32_t w_base = smem_u32(s_w);
    uint32_t phase = 0u;  // bit b: parity of accumulator b's next completion
    int issued = 0;       // bit b: a committed MMA group on accumulator b not yet waited for
    if (nt > 0 && tid == 0) {
        conv_mma(in_base, w_base, tmem, idesc, nch, cout);
        umma_commit(s_bar);
    }
    if (nt > 0) issued = 1;

    for (int64_t k = 0; k < nt; ++k) {
        const int b = (int)(k & 1);
        // the MMAs of tile k
        const bool ok = mbar_wait_bounded(s_bar + b, (phase >> b) & 1u);
        if (ok) {
            phase ^= 1u << b;
            issued &= ~(1 << b);
        } else {  // still in flight: the cleanup below waits for it again
            set_status(a.status, VIP_ERR_TIMEOUT);
            *s_fail = 1;
        }
        // tile k+1's halo (started two iterations ago, or in the prologue)
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*s_fail) break;
        if (k + 1 < nt) {
            if (tid == 0) {
                conv_mma(in_base + (1 - b) * SMEM_IN, w_base, tmem + (uint32_t)((1 - b) * 32), idesc,
                         nch, cout);
                umma_commit(s_bar + (1 - b));
            }
            issued |= 1 << (1 - b);
        }
        // tile k+2's halo into the buffer that tile k has released
        if (k + 2 < nt)
            conv_stage(a, conv_tile(a, blockIdx.x + (k + 2) * gridDim.x), in_base + b * SMEM_IN, nch, tid);
        // epilogue of tile k: warp w reads TMEM lanes 32w..32w+31 = pixels x0 + 32w + lane
        const ConvTile t = conv_tile(a, blockIdx.x + k * gridDim.x);
        float v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 32);
        if (cout == 32) tmem_ld_x32(taddr, v);
        else tmem_ld_x16(taddr, v);
        const int x = t.x0 + warp * 32 + lane;
        if (x < t.I.W) {
            const int64_t cell = t.I.off + (int64_t)t.y * t.I.W + x;
            if (a.epi == EPI_F32_CH0) {
                a.y32[cell] = v[0] + (a.bias ? a.bias[0] : 0.0f);
            } else {
                uint32_t packed[16];
                for (int c2 = 0; c2 < cout / 2; ++c2) {
                    float p0 = v[2 * c2], p1 = v[2 * c2 + 1];
                    if (a.epi == EPI_RELU_BF16) {
                        p0 = fmaxf(p0 + a.bias[2 * c2], 0.0f);
                        p1 = fmaxf(p1 + a.bias[2 * c2 + 1], 0.0f);
                    } else {  // gradient through the ReLU of the layer below
                        const __nv_bfloat16* m = a.mask + cell * cout;
                        p0 = __bfloat162float(m[2 * c2]) > 0.0f ? p0 : 0.0f;
                        p1 = __bfloat162float(m[2 * c2 + 1]) > 0.0f ? p1 : 0.0f;
                    }
                    packed[c2] = pack_bf16(p0, p1);
                }
                uint4* dst = reinterpret_cast<uint4*>(a.y + cell * cout);
                for (int q = 0; q < cout / 8; ++q)
                    dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2],
                                        packed[4 * q + 3]);
            }
        }
        // accumulator b is read out before the MMAs of tile k+2 overwrite it
        tc_fence_before();
        __syncthreads();
    }
    // after a failed wait MMAs may still be in flight: wait for every committed group
    // once more (bounded) before freeing TMEM; no copy is left in flight either
    cp_async_wait_all();
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb)
            if (issued & (1 << bb)) mbar_wait_bounded(s_bar + bb, (phase >> bb) & 1u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol));
}

// Weight gradients dW[tap][ci][co] = sum_p x[p + off(tap)][ci] gy[p][co] as MMAs on the
// tensor cores, K = pixels.  The halo is staged as for the convolution, channel-chunk
// planar, here with four lattice rows: [row][chunk][col] x 16 bytes.  Read with the
// pixel as K, an 8-pixel x 8-channel block (128 contiguous bytes) is a core matrix of
// an MN-major operand, so A (M = 4 rows x 32 channels, the fourth row's products
// discarded) and B (N = cout channels of gy, staged [chunk][pixel] x 16 bytes) need no
// transpose, and the three column offsets of the taps are start addresses 16 bytes
// apart.  Each block accumulates all its tiles in TMEM (three 32-column accumulators,
// one per column offset) and writes one FP32 partial; the bias gradients are summed
// on the side in pixel order.
constexpr int WG_ROWS = 4;
constexpr int WG_PLANE = PLANE_COLS * 16;                     // 2080: one row of one chunk
constexpr int WG_SMEM_X = WG_ROWS * MAX_CHUNKS * WG_PLANE;    // 33280
constexpr int WG_SMEM_G = MAX_CHUNKS * CNN_TILE * 16;         // 8192
constexpr int SMEM_WGRAD = WG_SMEM_X + WG_SMEM_G + 64;
// MN-major core matrices, no swizzle: the descriptor's leading-dimension offset is
// the byte distance between core matrices adjacent along K (8 more pixels: 128 bytes
// in both staged layouts), the stride-dimension offset the distance along M/N (8 more
// channels: one plane row of the halo, one chunk plane of gy).  (Checked against the
// FP64 reference of the gradients; the other assignment gives wrong sums.)
constexpr uint32_t WG_K_STRIDE = 128;

__host__ __device__ constexpr uint32_t umma_idesc_mn(int M, int N) {
    return umma_idesc(M, N) | (1u << 15) | (1u << 16);  // A and B MN-major
}

__global__ void __launch_bounds__(128) k_wgrad_tc(CnnWgradArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* s_x = smem;
    uint8_t* s_g = smem + WG_SMEM_X;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + WG_SMEM_X + WG_SMEM_G);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + WG_SMEM_X + WG_SMEM_G + 8);
    int* s_fail = reinterpret_cast<int*>(smem + WG_SMEM_X + WG_SMEM_G + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin = a.cin, cout = a.cout;
    const int nch = cin / 8, nchg = cout / 8;
    const int ncol = 128;  // three accumulators of 32 columns

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(s_bar, 1);
        *s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = umma_idesc_mn(128, cout);
    const uint32_t xb = smem_u32(s_x), gb = smem_u32(s_g);
    const uint32_t lbo = WG_K_STRIDE, sbo_a = WG_PLANE, sbo_b = CNN_TILE * 16;
    uint32_t phase = 0u;
    bool pending = false;
    float bacc = 0.0f;
    const int64_t nt = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    for (int64_t k = 0; k < nt; ++k) {
        const ConvTile t = conv_tile_of(a.img, a.nimg, blockIdx.x + k * gridDim.x);
        // rows y-1 .. y+2 of the input, columns x0-1 .. x0+128, zero outside the image
        const int nx_items = WG_ROWS * nch * PLANE_COLS;
        for (int i = tid; i < nx_items; i += blockDim.x) {
            const int r = i / (nch * PLANE_COLS);
            const int rem = i - r * nch * PLANE_COLS;
            const int c = rem / PLANE_COLS;
            const int col = rem - c * PLANE_COLS;
            const int yy = t.y - 1 + r, xx = t.x0 - 1 + col;
            const bool in = yy >= 0 && yy < t.I.H && xx >= 0 && xx < t.I.W;
            const __nv_bfloat16* src = a.x;
            if (in) src = a.x + (t.I.off + (int64_t)yy * t.I.W + xx) * cin + c * 8;
            cp_async16(xb + (r * MAX_CHUNKS + c) * WG_PLANE + col * 16, src, in ? 16u : 0u);
        }
        // gy of the tile's 128 pixels, zero beyond the row
        for (int i = tid; i < nchg * CNN_TILE; i += blockDim.x) {
            const int c = i / CNN_TILE, p = i - c * CNN_TILE;
            const int xx = t.x0 + p;
            const bool in = xx < t.I.W;
            const __nv_bfloat16* src = a.gy;
            if (in) src = a.gy + (t.I.off + (int64_t)t.y * t.I.W + xx) * cout + c * 8;
            cp_async16(gb + (c * CNN_TILE + p) * 16, src, in ? 16u : 0u);
        }
        cp_async_commit();
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid < cout) {  // bias gradient, pixel order
            const __nv_bfloat16* g = reinterpret_cast<const __nv_bfloat16*>(s_g) + (tid >> 3) * CNN_TILE * 8 + (tid & 7);
            for (int p = 0; p < CNN_TILE; ++p) bacc += __bfloat162float(g[p * 8]);
        }
        if (tid == 0) {
            for (int dx = 0; dx < 3; ++dx)
                for (int kc = 0; kc < CNN_TILE / 16; ++kc) {
                    const uint32_t aaddr = xb + dx * 16 + kc * 2 * WG_K_STRIDE;
                    const uint32_t baddr = gb + kc * 2 * WG_K_STRIDE;
                    umma_bf16(tmem + (uint32_t)(dx * 32), umma_desc(aaddr, lbo, sbo_a),
                              umma_desc(baddr, lbo, sbo_b), idesc, (k > 0 || kc > 0) ? 1u : 0u);
                }
            umma_commit(s_bar);
        }
        pending = true;
        const bool ok = mbar_wait_bounded(s_bar, phase);
        if (ok) {
            phase ^= 1u;
            pending = false;
        } else {
            set_status(a.status, VIP_ERR_TIMEOUT);
            *s_fail = 1;
        }
        tc_fence_before();
        __syncthreads();  // the buffers are restaged by the next tile
        tc_fence_after();
        if (*s_fail) break;
    }
    const int nent = 9 * cin * cout;
    float* dst = a.part + (int64_t)blockIdx.x * (nent + cout);
    if (nt > 0 && !*s_fail) {
        // warp w holds TMEM lanes 32w..32w+31 = row w of the halo (tap row dy = w), channel = lane
        for (int dx = 0; dx < 3; ++dx) {
            float v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dx * 32);
            if (cout == 32) tmem_ld_x32(taddr, v);
            else tmem_ld_x16(taddr, v);
            if (warp < 3 && lane < cin) {
                float* o = dst + ((int64_t)(warp * 3 + dx) * cin + lane) * cout;
                for (int co = 0; co < cout; ++co) o[co] = v[co];
            }
        }
    } else {
        for (int e = tid; e < nent; e += blockDim.x) dst[e] = 0.0f;
    }
    if (tid < cout) dst[nent + tid] = bacc;
    cp_async_wait_all();
    if (tid == 0 && pending) mbar_wait_bounded(s_bar, phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol));
}

cudaError_t cnn_wgrad_tc(const CnnWgradArgs& a, int nblocks, cudaStream_t s, const char** why) {
    *why = "";
    if (a.ntiles <= 0 || nblocks <= 0) return cudaSuccess;
    if (a.cin % 16 || a.cin > CNN_CH || (a.cout != 16 && a.cout != 32)) {
        *why = "unsupported channel counts";
        return cudaErrorInvalidValue;
    }
    k_wgrad_tc<<<nblocks, 128, SMEM_WGRAD, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) *why = "weight-gradient launch";
    return e;
}

cudaError_t cnn_conv_init() {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_CONV);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_WGRAD);
}

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
    const int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)std::max(nsm, 1) * CONV_CTAS_PER_SM);
    k_conv_tc<<<grid, 128, SMEM_CONV, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) *why = "kernel launch";
    return e;
}

}  // namespace vip
