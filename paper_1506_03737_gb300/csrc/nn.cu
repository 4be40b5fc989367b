// Learned displacement correction: a 3 -> 16 -> 16 -> 16 -> 3 network of periodic 3x3x3
// convolutions with ReLU between layers, trained and applied on the GPU by the kernels in this
// file (BF16 tensor-core products, FP32 accumulation, FP32 master weights, Adam).
//
// The paper has no learned component. The network maps the final displacement field Psi of a
// coarse, few-step COLA run (3 channels on the Lagrangian grid) to a correction dPsi toward a
// fine-mesh, many-step run from the same seed; plain COLA stays the fallback.
//
// Layout
//   activations  bf16 [z][y][x][16] (32 B per voxel; unused channels are zero)
//   weights      bf16 [tap][c_out 16][c_in 16], tap = (dz+1) 9 + (dy+1) 3 + (dx+1)
//   master       fp32 [layer][28][16][16]: taps 0..26 = W[tap][o][i], slot 27 holds the bias in i = 0
//
// Every convolution (forward of each layer, backward-data of layers 2..4) is one implicit GEMM:
// with mma.sync (k_conv, the default) over a 16 x 8 x 8 voxel tile, or on the tcgen05 tensor cores
// (k_conv_tc, engine 1, grid side a multiple of 128). With 16 channels each tcgen05.mma (M = 128
// voxels, N = 16, K = 16) reads a 4 KB operand from shared memory for 65,536 FLOP, which bounds it
// by shared-memory bandwidth; measured at 128^3 it is slower than the mma.sync kernel. mma.sync: M = 16 consecutive x voxels per mma, N = output channels,
// K = 16 input channels per tap, 27 taps. The 18 x 10 x 10 halo tile of the input is staged in
// shared memory with cp.async; each voxel's two 16-byte halves swap places on every other
// group of four voxels so that ldmatrix reads are free of bank conflicts.
//
//   forward        out[v][o]  = b[o] + sum_tap sum_i W[tap][o][i] a[v + d_tap][i]
//   backward-data  da[u][i]   = sum_tap sum_o W[tap][o][i] dz[u - d_tap][o]
//                             = forward with W'[tap][i][o] = W[26 - tap][o][i], no bias
//   weight grad    dW[tap][o][i] = sum_v dz[v][o] a[v + d_tap][i];  db[o] = sum_v dz[v][o]
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/colapm.h"
#include "../../include/colapm_nn.h"
#include "colapm_internal.h"

namespace colapm {
namespace nn {
namespace {

constexpr int C = 16;                          // padded channel count
constexpr int TX = 16, TY = 8, TZ = 8;         // output tile
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HALO = HX * HY * HZ;             // 1800 voxels
constexpr int TILE = TX * TY * TZ;             // 1024 voxels
constexpr int NTHREADS = 256;                  // 8 warps: warp w owns output plane z = w of the tile
constexpr int SLOTS = 28;                      // 27 taps + bias
constexpr int LAYERS = 4;
constexpr int LSIZE = SLOTS * C * C;           // 7168 master slots per layer
constexpr int CIN[LAYERS] = {3, 16, 16, 16};
constexpr int COUT[LAYERS] = {16, 16, 16, 3};

constexpr size_t SMEM_HALO = (size_t)HALO * 32;   // 57600
constexpr size_t SMEM_W = 27 * C * 32;            // 13824
constexpr size_t SMEM_CONV = SMEM_HALO + SMEM_W;
constexpr size_t SMEM_WGRAD = SMEM_HALO + (size_t)TILE * 32;

enum Epi { EPI_RELU = 0, EPI_OUT = 1, EPI_MASK = 2 };

struct ConvArgs {
    const __nv_bfloat16* in;     // [n^3][16]
    const __nv_bfloat16* w;      // [27][16][16]
    const float* bias;           // [16] or null
    int n;
    __nv_bfloat16* out;          // EPI_RELU / EPI_MASK: [n^3][16]; EPI_OUT with target: dz [n^3][16]
    const __nv_bfloat16* mask;   // EPI_MASK: the layer input whose ReLU gates the gradient
    float* y;                    // EPI_OUT: [n^3][3] = base + oscale * net
    const float* base;           // EPI_OUT: optional [n^3][3]
    float oscale;
    const float* target;         // EPI_OUT training: [n^3][3] physical; normalised by tscale
    float tscale, gscale;        // gscale = 2 / (3 n^3)
    double* loss;                // sum of squared normalised errors
    int* err;                    // bit 4: a bounded wait for the tensor cores gave up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Byte offset of half `k` (0: channels 0..7, 1: channels 8..15) of staged voxel `h`.
__device__ __forceinline__ uint32_t vox_off(int h, int k) { return (uint32_t)(h * 32 + ((k ^ ((h >> 2) & 1)) << 4)); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
}

__device__ __forceinline__ void tile_origin(int t, int n, int& x0, int& y0, int& z0) {
    const int tx = n / TX, ty = n / TY;
    x0 = (t % tx) * TX;
    y0 = ((t / tx) % ty) * TY;
    z0 = (t / (tx * ty)) * TZ;
}

// Stage the periodic halo tile of `in` around the output tile at (x0, y0, z0).
__device__ __forceinline__ void stage_halo(uint8_t* sm, const __nv_bfloat16* __restrict__ in, int n, int x0, int y0,
                                           int z0) {
    const uint32_t base = smem_u32(sm);
    for (int j = threadIdx.x; j < 2 * HALO; j += NTHREADS) {
        const int h = j >> 1, k = j & 1;
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        gx += gx < 0 ? n : (gx >= n ? -n : 0);
        gy += gy < 0 ? n : (gy >= n ? -n : 0);
        gz += gz < 0 ? n : (gz >= n ? -n : 0);
        const size_t v = ((size_t)gz * n + gy) * n + gx;
        cp_async16(base + vox_off(h, k), in + v * C + k * 8);
    }
}

template <int NT, int EPI>
__global__ void __launch_bounds__(NTHREADS, 2) k_conv(ConvArgs a) {
    extern __shared__ __align__(128) uint8_t sm[];
    const int n = a.n;
    int x0, y0, z0;
    tile_origin(blockIdx.x, n, x0, y0, z0);
    stage_halo(sm, a.in, n, x0, y0, z0);
    {   // weights, swizzled like voxels with the output channel as the row
        const uint32_t wb = smem_u32(sm + SMEM_HALO);
        for (int j = threadIdx.x; j < 27 * C * 2; j += NTHREADS) {
            const int row = j >> 1, k = j & 1;
            cp_async16(wb + vox_off(row, k), a.w + row * C + k * 8);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    const int lane = threadIdx.x & 31, tz = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const uint32_t hb = smem_u32(sm), wb = smem_u32(sm + SMEM_HALO);
    // ldmatrix roles: A rows (voxels) and halves; B rows (output channels) and halves
    const int ar = (lane & 7) + 8 * ((lane >> 3) & 1), ak = lane >> 4;
    const int bn = (lane & 7) + 8 * (lane >> 4), bk = (lane >> 3) & 1;

    float acc[TY][NT][4];
#pragma unroll
    for (int m = 0; m < TY; ++m)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[m][j][e] = 0.0f;

#pragma unroll 1
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        uint32_t b[4];
        ldsm_x4(wb + vox_off(tap * C + bn, bk), b[0], b[1], b[2], b[3]);
        const int hrow = ((tz + 1 + dz) * HY + (1 + dy)) * HX + 1 + dx + ar;
#pragma unroll
        for (int m = 0; m < TY; ++m) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(hb + vox_off(hrow + m * HX, ak), a0, a1, a2, a3);
            mma_bf16(acc[m][0], a0, a1, a2, a3, b[0], b[1]);
            if (NT == 2) mma_bf16(acc[m][1], a0, a1, a2, a3, b[2], b[3]);
        }
    }

    double lsum = 0.0;
#pragma unroll
    for (int m = 0; m < TY; ++m) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int x = g + 8 * half;
            const size_t v = ((size_t)(z0 + tz) * n + (y0 + m)) * n + x0 + x;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int ch = 8 * j + 2 * q;
                float v0 = acc[m][j][2 * half], v1 = acc[m][j][2 * half + 1];
                if (EPI == EPI_RELU) {
                    v0 = fmaxf(v0 + a.bias[ch], 0.0f);
                    v1 = fmaxf(v1 + a.bias[ch + 1], 0.0f);
                    *reinterpret_cast<__nv_bfloat162*>(a.out + v * C + ch) = __floats2bfloat162_rn(v0, v1);
                } else if (EPI == EPI_MASK) {
                    const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + v * C + ch);
                    v0 = __bfloat162float(mk.x) > 0.0f ? v0 : 0.0f;
                    v1 = __bfloat162float(mk.y) > 0.0f ? v1 : 0.0f;
                    *reinterpret_cast<__nv_bfloat162*>(a.out + v * C + ch) = __floats2bfloat162_rn(v0, v1);
                } else if (j == 0 && q < 2) {   // EPI_OUT: channels 0..2 of n-tile 0
                    v0 += a.bias[ch];
                    v1 += a.bias[ch + 1];
                    const float vv[2] = {v0, v1};
                    float dzv[2] = {0.0f, 0.0f};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int c = ch + e;
                        if (c < 3) {
                            a.y[v * 3 + c] = (a.base ? a.base[v * 3 + c] : 0.0f) + a.oscale * vv[e];
                            if (a.target) {
                                const float d = vv[e] - a.target[v * 3 + c] * a.tscale;
                                lsum += (double)d * d;
                                dzv[e] = a.gscale * d;
                            }
                        }
                    }
                    if (a.target)
                        *reinterpret_cast<__nv_bfloat162*>(a.out + v * C + ch) = __floats2bfloat162_rn(dzv[0], dzv[1]);
                }
            }
        }
    }
    if (EPI == EPI_OUT && a.target) {
#pragma unroll
        for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0 && lsum != 0.0) atomicAdd(a.loss, lsum);
    }
}

// Per-CTA partial weight gradients of one layer over a static round-robin share of the tiles:
// part[blockIdx.x][slot][o][i]. Warp w owns slots {w, w + 8, w + 16, w + 24} below 28.
__global__ void __launch_bounds__(NTHREADS, 2)
    k_wgrad(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ act, int n, float* __restrict__ part) {
    extern __shared__ __align__(128) uint8_t sm[];
    const int ntiles = (n / TX) * (n / TY) * (n / TZ);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const uint32_t hb = smem_u32(sm), db = smem_u32(sm + SMEM_HALO);
    const int av = (lane & 7) + 8 * (lane >> 4), ak = (lane >> 3) & 1;       // dz^T as A
    const int bv = (lane & 7) + 8 * ((lane >> 3) & 1), bk = lane >> 4;      // shifted act as B
    const uint32_t ones = 0x3F803F80u;                                      // bf16 pair (1, 1)

    float acc[4][2][4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[s][j][e] = 0.0f;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int x0, y0, z0;
        tile_origin(t, n, x0, y0, z0);
        stage_halo(sm, act, n, x0, y0, z0);
        for (int j = threadIdx.x; j < 2 * TILE; j += NTHREADS) {
            const int l = j >> 1, k = j & 1;
            const int lx = l % TX, ly = (l / TX) % TY, lz = l / (TX * TY);
            const size_t v = ((size_t)(z0 + lz) * n + (y0 + ly)) * n + x0 + lx;
            cp_async16(db + vox_off(l, k), dz + v * C + k * 8);
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll 1
        for (int row = 0; row < TZ * TY; ++row) {
            const int lz = row / TY, ly = row % TY;
            uint32_t a0, a1, a2, a3;
            ldsm_x4_t(db + vox_off(row * TX + av, ak), a0, a1, a2, a3);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int slot = w + 8 * s;
                if (slot >= SLOTS) break;
                uint32_t b0, b1, b2, b3;
                if (slot == 27) {
                    b0 = b1 = b2 = b3 = ones;
                } else {
                    const int dzz = slot / 9 - 1, dyy = (slot / 3) % 3 - 1, dxx = slot % 3 - 1;
                    const int h = ((lz + 1 + dzz) * HY + (ly + 1 + dyy)) * HX + 1 + dxx + bv;
                    ldsm_x4_t(hb + vox_off(h, bk), b0, b1, b2, b3);
                }
                mma_bf16(acc[s][0], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[s][1], a0, a1, a2, a3, b2, b3);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int slot = w + 8 * s;
        if (slot >= SLOTS) break;
        float* p = part + ((size_t)blockIdx.x * SLOTS + slot) * C * C;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = 8 * j + 2 * q;
            *reinterpret_cast<float2*>(p + g * C + i) = make_float2(acc[s][j][0], acc[s][j][1]);
            *reinterpret_cast<float2*>(p + (g + 8) * C + i) = make_float2(acc[s][j][2], acc[s][j][3]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores (tcgen05), for grids whose side is a
// multiple of 128. A CTA computes TC_ROWS output x-rows of 128 voxels; for each row and tap one
// tcgen05.mma (M = 128 voxels, N = 16 output channels, K = 16 input channels, BF16 x BF16 -> FP32)
// accumulates into the row's 16 TMEM columns. The halo is staged as two K-half planes (channels
// 0..7 and 8..15, 16 bytes per voxel), which is the no-swizzle K-major core-matrix layout: 8
// consecutive voxels x 16 bytes form one 128-byte core matrix, LBO = the plane distance (K),
// SBO = 128 bytes (next 8 voxels). A tap's operand is the row of 128 halo voxels shifted by the
// tap, i.e. a descriptor start offset. Weights: [tap][K half][16 outputs][8 inputs] (512 B a tap).
// One thread issues the MMAs and commits them to an mbarrier; after a bounded wait the four warps
// read their TMEM lanes (lane = voxel) with tcgen05.ld and run the same epilogues as k_conv.
constexpr int TC_TY = 2, TC_TZ = 2, TC_ROWS = TC_TY * TC_TZ;
constexpr int TC_HX = 130, TC_HY = TC_TY + 2, TC_HZ = TC_TZ + 2;
constexpr int TC_HALO = TC_HX * TC_HY * TC_HZ;                    // 2080 voxels
constexpr uint32_t TC_PLANE = TC_HALO * 16;                       // bytes per K-half plane
constexpr uint32_t TC_W = 27 * 512;                               // weight bytes
constexpr size_t TC_SMEM = 2 * (size_t)TC_PLANE + TC_W + 128;     // + mbarrier and TMEM address
constexpr uint32_t TC_COLS = TC_ROWS * 16;                        // TMEM columns (power of two)
constexpr long long TC_SPIN_LIMIT = 1ll << 24;
// kind::f16 instruction descriptor: FP32 D (bits 4-5), BF16 A and B (bits 7-9, 10-12), both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);   // no swizzle, base offset 0
}

// Stage the halo of tile t (periodic) into the two K-half planes with 16-byte cp.async.
__device__ __forceinline__ void tc_stage(uint32_t sbase, const __nv_bfloat16* __restrict__ in, int n, int t) {
    const int txn = n / 128, tyn = n / TC_TY;
    const int x0 = (t % txn) * 128, y0 = ((t / txn) % tyn) * TC_TY, z0 = (t / (txn * tyn)) * TC_TZ;
#pragma unroll 1
    for (int row = 0; row < TC_HY * TC_HZ; ++row) {
        const int hy = row % TC_HY, hz = row / TC_HY;
        int gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        gy += gy < 0 ? n : (gy >= n ? -n : 0);
        gz += gz < 0 ? n : (gz >= n ? -n : 0);
        const __nv_bfloat16* src = in + ((size_t)gz * n + gy) * n * C;
        for (int j = threadIdx.x; j < 2 * TC_HX; j += 128) {
            const int hx = j >> 1, k = j & 1;
            int gx = x0 - 1 + hx;
            gx += gx < 0 ? n : (gx >= n ? -n : 0);
            cp_async16(sbase + k * TC_PLANE + (row * TC_HX + hx) * 16, src + (size_t)gx * C + k * 8);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// Persistent over tiles: weights, TMEM and the mbarrier are set up once per CTA. Per tile: wait for
// the staged halo, issue the 27 x TC_ROWS MMAs (one thread), wait for them, start staging the next
// tile's halo (the MMAs no longer read shared memory), then read TMEM and write the outputs.
template <int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* wsm = sm + 2 * TC_PLANE;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(wsm + TC_W);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int txn = n / 128, tyn = n / TC_TY;
    const int ntiles = txn * tyn * (n / TC_TZ);
    const uint32_t sbase = smem_u32(sm);
    for (int j = tid; j < 27 * C * 2; j += 128) {     // weights [tap][K half][out][8]
        const int tap = j >> 5, o = (j >> 1) & 15, k = j & 1;
        cp_async16(sbase + 2 * TC_PLANE + tap * 512 + k * 256 + o * 16, a.w + (tap * C + o) * C + k * 8);
    }
    if (blockIdx.x < ntiles) tc_stage(sbase, a.in, n, blockIdx.x);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint64_t a_desc0 = tc_desc(sbase, TC_PLANE, 128), b_desc0 = tc_desc(sbase + 2 * TC_PLANE, 256, 128);
    bool ok = true;
    double lsum = 0.0;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the tensor cores read these bytes
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) {
#pragma unroll 1
            for (int r = 0; r < TC_ROWS; ++r) {
                const int ry = r % TC_TY, rz = r / TC_TY;
                // descriptor start addresses count 16-byte units: adding a voxel index moves by one voxel
                const uint64_t arow = a_desc0 + (uint64_t)(((rz + 1) * TC_HY + (ry + 1)) * TC_HX + 1);
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int off = (tap / 9 - 1) * TC_HY * TC_HX + ((tap / 3) % 3 - 1) * TC_HX + (tap % 3 - 1);
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + r * 16),
                        "l"(arow + (uint64_t)(int64_t)off), "l"(b_desc0 + (uint64_t)(tap * 32)), "r"(TC_IDESC), "r"(tap));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(mbar))
                         : "memory");
        }
        uint32_t done = 0;
        for (long long i = 0; i < TC_SPIN_LIMIT && !done; ++i) {
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(mbar)), "r"(it & 1)
                : "memory");
        }
        if (!done) {
            if (tid == 0 && a.err) atomicOr(a.err, 4);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!__syncthreads_and(done)) break;
        if (t + (int)gridDim.x < ntiles) tc_stage(sbase, a.in, n, t + gridDim.x);   // overlaps the epilogue
        const int x0 = (t % txn) * 128, y0 = ((t / txn) % tyn) * TC_TY, z0 = (t / (txn * tyn)) * TC_TZ;
#pragma unroll 1
        for (int r = 0; r < TC_ROWS; ++r) {
            uint32_t q[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                  "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
                : "r"(taddr + ((uint32_t)(32 * warp) << 16) + r * 16));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const int ry = r % TC_TY, rz = r / TC_TY;
            const size_t v = ((size_t)(z0 + rz) * n + (y0 + ry)) * n + x0 + 32 * warp + lane;
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = __uint_as_float(q[c]);
            if (EPI == EPI_RELU || EPI == EPI_MASK) {
                uint32_t pk[8];
                if (EPI == EPI_MASK) {
                    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + v * C);
                    const uint4 m0 = mp[0], m1 = mp[1];
                    const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(&mw[c]);
                        const float v0 = __bfloat162float(mk.x) > 0.0f ? acc[2 * c] : 0.0f;
                        const float v1 = __bfloat162float(mk.y) > 0.0f ? acc[2 * c + 1] : 0.0f;
                        const __nv_bfloat162 b = __floats2bfloat162_rn(v0, v1);
                        pk[c] = *reinterpret_cast<const uint32_t*>(&b);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const __nv_bfloat162 b = __floats2bfloat162_rn(fmaxf(acc[2 * c] + a.bias[2 * c], 0.0f),
                                                                       fmaxf(acc[2 * c + 1] + a.bias[2 * c + 1], 0.0f));
                        pk[c] = *reinterpret_cast<const uint32_t*>(&b);
                    }
                }
                uint4* op = reinterpret_cast<uint4*>(a.out + v * C);
                op[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                op[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else {   // EPI_OUT: channels 0..2
                float dzv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float val = acc[c] + a.bias[c];
                    a.y[v * 3 + c] = (a.base ? a.base[v * 3 + c] : 0.0f) + a.oscale * val;
                    dzv[c] = 0.0f;
                    if (a.target) {
                        const float d = val - a.target[v * 3 + c] * a.tscale;
                        lsum += (double)d * d;
                        dzv[c] = a.gscale * d;
                    }
                }
                if (a.target) {
                    const __nv_bfloat162 b01 = __floats2bfloat162_rn(dzv[0], dzv[1]);
                    const __nv_bfloat162 b2z = __floats2bfloat162_rn(dzv[2], 0.0f);
                    *reinterpret_cast<uint2*>(a.out + v * C) =
                        make_uint2(*reinterpret_cast<const uint32_t*>(&b01), *reinterpret_cast<const uint32_t*>(&b2z));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");   // TMEM reads done before the next MMAs
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (EPI == EPI_OUT && a.target) {
#pragma unroll
        for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0 && lsum != 0.0) atomicAdd(a.loss, lsum);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(TC_COLS));
}

__device__ __forceinline__ bool real_slot(int l, int slot, int o, int i) {
    constexpr int cin[LAYERS] = {3, 16, 16, 16}, cout[LAYERS] = {16, 16, 16, 3};
    if (o >= cout[l]) return false;
    return slot < 27 ? i < cin[l] : i == 0;
}

// Sum the per-CTA partials of every layer in a fixed order: grad[l][slot][o][i].
__global__ void k_reduce_grads(const float* __restrict__ part, int nparts, float* __restrict__ grad) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= LAYERS * LSIZE) return;
    const int l = idx / LSIZE, r = idx % LSIZE;
    const int slot = r / (C * C), o = (r / C) % C, i = r % C;
    float s = 0.0f;
    if (real_slot(l, slot, o, i)) {
        const float* p = part + (size_t)l * nparts * LSIZE + r;
        for (int b = 0; b < nparts; ++b) s += p[(size_t)b * LSIZE];
    }
    grad[idx] = s;
}

// Adam on the FP32 master copy, then the BF16 forward and flipped-transposed weights and the bias.
__global__ void k_adam(float* __restrict__ wm, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2,
                       int update, __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wt,
                       float* __restrict__ bias) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= LAYERS * LSIZE) return;
    const int l = idx / LSIZE, r = idx % LSIZE;
    const int slot = r / (C * C), o = (r / C) % C, i = r % C;
    float w = wm[idx];
    if (update && real_slot(l, slot, o, i)) {
        const float g = grad[idx];
        const float m = b1 * m1[idx] + (1.0f - b1) * g;
        const float v = b2 * m2[idx] + (1.0f - b2) * g * g;
        m1[idx] = m;
        m2[idx] = v;
        w -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        wm[idx] = w;
    }
    if (slot < 27) {
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        wf[((size_t)l * 27 + slot) * C * C + o * C + i] = wb;
        wt[((size_t)l * 27 + (26 - slot)) * C * C + i * C + o] = wb;
    } else if (i == 0) {
        bias[l * C + o] = w;
    }
}

// x[v][c] = bf16(psi[v][c] / s_in) for c < 3, zero for the padded channels.
__global__ void k_pack_input(const float* __restrict__ psi, size_t nv, float inv_s, __nv_bfloat16* __restrict__ x) {
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const __nv_bfloat162 p01 = __floats2bfloat162_rn(psi[3 * v] * inv_s, psi[3 * v + 1] * inv_s);
    const __nv_bfloat162 p2z = __floats2bfloat162_rn(psi[3 * v + 2] * inv_s, 0.0f);
    uint4 lo;
    lo.x = *reinterpret_cast<const uint32_t*>(&p01);
    lo.y = *reinterpret_cast<const uint32_t*>(&p2z);
    lo.z = lo.w = 0u;
    uint4* d = reinterpret_cast<uint4*>(x + v * C);
    d[0] = lo;
    d[1] = make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace
}  // namespace nn
}  // namespace colapm

using namespace colapm::nn;

struct colapm_nn {
    int n = 0;
    size_t nv = 0;
    colapm_nn_config cfg{};
    cudaStream_t stream = nullptr;
    int steps = 0;
    int nparts = 0;
    // device
    __nv_bfloat16* act[LAYERS] = {};   // act[0] = packed input, act[l] = output of layer l (l = 1..3)
    __nv_bfloat16* dz[2] = {};         // gradient ping-pong
    __nv_bfloat16* dz_out = nullptr;   // gradient at the network output (channels 0..2)
    float* y = nullptr;                // scratch output [n^3][3]
    float* wm = nullptr;               // master [4][28][16][16]
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* grad = nullptr;
    float* part = nullptr;             // [4][nparts][28][16][16]
    __nv_bfloat16* wf = nullptr;       // [4][27][16][16]
    __nv_bfloat16* wt = nullptr;
    float* bias = nullptr;             // [4][16]
    double* loss = nullptr;
    int* err = nullptr;                // device error word (bit 4: a tensor-core wait gave up)
    bool use_tc = false;               // tcgen05 convolutions (grid side a multiple of 128)
    int tc_grid = 0;                   // persistent grid of the tcgen05 convolutions
    long long launches = 0;
};

namespace {

#define NN_CK(x)                                  \
    do {                                          \
        if ((x) != cudaSuccess) {                 \
            (void)cudaGetLastError();             \
            return COLAPM_E_CUDA;                 \
        }                                         \
    } while (0)

int conv_grid(int n) { return (n / TX) * (n / TY) * (n / TZ); }

bool configured = false;

cudaError_t configure() {
    if (configured) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_conv<2, EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CONV))) return e;
    if ((e = cudaFuncSetAttribute(k_conv<2, EPI_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CONV))) return e;
    if ((e = cudaFuncSetAttribute(k_conv<1, EPI_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CONV))) return e;
    if ((e = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_WGRAD))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_tc<EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_tc<EPI_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_tc<EPI_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM))) return e;
    configured = true;
    return cudaSuccess;
}

template <int NT, int EPI>
cudaError_t conv(colapm_nn* c, ConvArgs a) {
    a.err = c->err;
    if (c->use_tc) {
        const int tiles = (c->n / 128) * (c->n / TC_TY) * (c->n / TC_TZ);
        k_conv_tc<EPI><<<std::min(tiles, c->tc_grid), 128, TC_SMEM, c->stream>>>(a);
    } else {
        k_conv<NT, EPI><<<conv_grid(c->n), NTHREADS, SMEM_CONV, c->stream>>>(a);
    }
    ++c->launches;
    return cudaGetLastError();
}

// Report (and clear) a device-side error of the network's kernels; synchronises.
int check_err(colapm_nn* c) {
    int h = 0;
    if (cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return COLAPM_E_CUDA;
    }
    if (h) {
        (void)cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
        return COLAPM_E_TIMEOUT;
    }
    return COLAPM_OK;
}

// Weights (padded master layout) -> bf16 copies and bias, with no update.
cudaError_t publish(colapm_nn* c) {
    const int total = LAYERS * LSIZE;
    k_adam<<<(total + 255) / 256, 256, 0, c->stream>>>(c->wm, c->m1, c->m2, c->grad, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0,
                                                       c->wf, c->wt, c->bias);
    ++c->launches;
    return cudaGetLastError();
}

// Forward through all four layers; with `target`, also the output gradient and the loss sum.
cudaError_t forward(colapm_nn* c, const float* psi, float* y, const float* base, const float* target) {
    const size_t nv = c->nv;
    k_pack_input<<<(unsigned)((nv + 255) / 256), 256, 0, c->stream>>>(psi, nv, 1.0f / c->cfg.s_in, c->act[0]);
    ++c->launches;
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    for (int l = 0; l < 3; ++l) {
        ConvArgs a{};
        a.in = c->act[l];
        a.w = c->wf + (size_t)l * 27 * C * C;
        a.bias = c->bias + l * C;
        a.n = c->n;
        a.out = c->act[l + 1];
        if ((e = conv<2, EPI_RELU>(c, a))) return e;
    }
    ConvArgs a{};
    a.in = c->act[3];
    a.w = c->wf + (size_t)3 * 27 * C * C;
    a.bias = c->bias + 3 * C;
    a.n = c->n;
    a.y = y;
    a.base = base;
    a.oscale = c->cfg.s_out;
    if (target) {
        a.target = target;
        a.tscale = 1.0f / c->cfg.s_out;
        a.gscale = (float)(2.0 / (3.0 * (double)nv));
        a.loss = c->loss;
        a.out = c->dz_out;
    }
    return conv<1, EPI_OUT>(c, a);
}

// Backward through all layers into per-CTA partials, then the fixed-order reduction into grad.
cudaError_t backward(colapm_nn* c) {
    cudaError_t e;
    const __nv_bfloat16* g = c->dz_out;
    for (int l = 3; l >= 0; --l) {
        k_wgrad<<<c->nparts, NTHREADS, SMEM_WGRAD, c->stream>>>(g, c->act[l], c->n,
                                                               c->part + (size_t)l * c->nparts * LSIZE);
        ++c->launches;
        if ((e = cudaGetLastError())) return e;
        if (l == 0) break;
        ConvArgs a{};
        a.in = g;
        a.w = c->wt + (size_t)l * 27 * C * C;
        a.n = c->n;
        a.mask = c->act[l];
        a.out = c->dz[l & 1];
        if ((e = conv<2, EPI_MASK>(c, a))) return e;
        g = c->dz[l & 1];
    }
    const int total = LAYERS * LSIZE;
    k_reduce_grads<<<(total + 255) / 256, 256, 0, c->stream>>>(c->part, c->nparts, c->grad);
    ++c->launches;
    return cudaGetLastError();
}

// Flat parameter order: per layer W[27][cout][cin] then b[cout].
template <class F>
void for_each_param(F f) {
    size_t k = 0;
    for (int l = 0; l < LAYERS; ++l) {
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < COUT[l]; ++o)
                for (int i = 0; i < CIN[l]; ++i) f(k++, (size_t)l * LSIZE + (t * C + o) * C + i);
        for (int o = 0; o < COUT[l]; ++o) f(k++, (size_t)l * LSIZE + (27 * C + o) * C);
    }
}

// He-normal initial weights from a host splitmix64 stream and Box-Muller; biases start at zero.
void init_weights(std::vector<float>& flat, unsigned long long seed) {
    unsigned long long s = seed;
    auto next = [&]() {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    size_t k = 0;
    for (int l = 0; l < LAYERS; ++l) {
        const double sd = std::sqrt(2.0 / (27.0 * CIN[l]));
        for (int j = 0; j < 27 * COUT[l] * CIN[l]; ++j) {
            const double r = std::sqrt(-2.0 * std::log(unif())), th = 6.283185307179586 * unif();
            flat[k++] = (float)(sd * r * std::cos(th));
        }
        for (int o = 0; o < COUT[l]; ++o) flat[k++] = 0.0f;
    }
}

int upload_params(colapm_nn* c, const float* flat) {
    std::vector<float> pad((size_t)LAYERS * LSIZE, 0.0f);
    for_each_param([&](size_t k, size_t slot) { pad[slot] = flat[k]; });
    NN_CK(cudaMemcpyAsync(c->wm, pad.data(), pad.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    NN_CK(publish(c));
    NN_CK(cudaStreamSynchronize(c->stream));
    return COLAPM_OK;
}

bool device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void colapm_nn_default_config(colapm_nn_config* cfg) {
    if (!cfg) return;
    cfg->s_in = 1.0f;
    cfg->s_out = 1.0f;
    cfg->lr = 1e-3f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.999f;
    cfg->eps = 1e-8f;
    cfg->engine = 0;
    cfg->seed = 1;
}

int colapm_nn_create(int n, const colapm_nn_config* cfg, void* stream, colapm_nn** out) {
    if (!out) return COLAPM_E_ARG;
    *out = nullptr;
    if (!cfg || n < 16 || n > 1024 || n % 16 != 0 || !(cfg->s_in > 0.0f) || !(cfg->s_out > 0.0f) ||
        !(cfg->lr >= 0.0f) || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps > 0.0f) || cfg->engine < 0 || cfg->engine > 1)
        return COLAPM_E_ARG;
    colapm_nn* c = new (std::nothrow) colapm_nn;
    if (!c) return COLAPM_E_NOMEM;
    c->n = n;
    c->nv = (size_t)n * n * n;
    c->cfg = *cfg;
    c->stream = static_cast<cudaStream_t>(stream);
    auto fail = [&](int code) {
        colapm_nn_destroy(c);
        return code;
    };
    if (configure() != cudaSuccess) return fail(COLAPM_E_CUDA);
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_wgrad, NTHREADS, SMEM_WGRAD))
        return fail(COLAPM_E_CUDA);
    c->nparts = std::max(1, std::min(conv_grid(n), sms * std::max(occ, 1)));
    int occ_tc = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_tc, k_conv_tc<EPI_RELU>, 128, TC_SMEM)) return fail(COLAPM_E_CUDA);
    c->tc_grid = sms * std::max(occ_tc, 1);
    const size_t abytes = c->nv * C * sizeof(__nv_bfloat16);
    bool ok = true;
    for (int l = 0; l < LAYERS; ++l) ok = ok && cudaMalloc(&c->act[l], abytes) == cudaSuccess;
    ok = ok && cudaMalloc(&c->dz[0], abytes) == cudaSuccess && cudaMalloc(&c->dz[1], abytes) == cudaSuccess &&
         cudaMalloc(&c->dz_out, abytes) == cudaSuccess && cudaMalloc(&c->y, c->nv * 3 * sizeof(float)) == cudaSuccess;
    const size_t ps = (size_t)LAYERS * LSIZE * sizeof(float);
    ok = ok && cudaMalloc(&c->wm, ps) == cudaSuccess && cudaMalloc(&c->m1, ps) == cudaSuccess &&
         cudaMalloc(&c->m2, ps) == cudaSuccess && cudaMalloc(&c->grad, ps) == cudaSuccess &&
         cudaMalloc(&c->part, ps * c->nparts) == cudaSuccess &&
         cudaMalloc(&c->wf, (size_t)LAYERS * 27 * C * C * sizeof(__nv_bfloat16)) == cudaSuccess &&
         cudaMalloc(&c->wt, (size_t)LAYERS * 27 * C * C * sizeof(__nv_bfloat16)) == cudaSuccess &&
         cudaMalloc(&c->bias, LAYERS * C * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->loss, sizeof(double)) == cudaSuccess && cudaMalloc(&c->err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return fail(COLAPM_E_NOMEM);
    }
    c->use_tc = cfg->engine == 1 && n % 128 == 0;
    if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) || cudaMemsetAsync(c->dz_out, 0, abytes, c->stream) ||
        cudaMemsetAsync(c->m1, 0, ps, c->stream) ||
        cudaMemsetAsync(c->m2, 0, ps, c->stream) || cudaMemsetAsync(c->grad, 0, ps, c->stream))
        return fail(COLAPM_E_CUDA);
    std::vector<float> flat(COLAPM_NN_PARAMS);
    init_weights(flat, cfg->seed);
    const int r = upload_params(c, flat.data());
    if (r) return fail(r);
    *out = c;
    return COLAPM_OK;
}

int colapm_nn_destroy(colapm_nn* c) {
    if (!c) return COLAPM_OK;
    (void)cudaStreamSynchronize(c->stream);
    for (auto* p : c->act) cudaFree(p);
    cudaFree(c->dz[0]);
    cudaFree(c->dz[1]);
    cudaFree(c->dz_out);
    cudaFree(c->y);
    for (float* p : {c->wm, c->m1, c->m2, c->grad, c->part, c->bias}) cudaFree(p);
    cudaFree(c->wf);
    cudaFree(c->wt);
    cudaFree(c->loss);
    cudaFree(c->err);
    (void)cudaGetLastError();
    delete c;
    return COLAPM_OK;
}

int colapm_nn_set_params(colapm_nn* c, const float* params) {
    if (!c || !params) return COLAPM_E_ARG;
    NN_CK(cudaStreamSynchronize(c->stream));
    return upload_params(c, params);
}

int colapm_nn_get_params(colapm_nn* c, float* params) {
    if (!c || !params) return COLAPM_E_ARG;
    std::vector<float> pad((size_t)LAYERS * LSIZE);
    NN_CK(cudaMemcpyAsync(pad.data(), c->wm, pad.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    NN_CK(cudaStreamSynchronize(c->stream));
    for_each_param([&](size_t k, size_t slot) { params[k] = pad[slot]; });
    return COLAPM_OK;
}

int colapm_nn_forward(colapm_nn* c, const float* psi, float* out, int add) {
    if (!c || !psi || !out || !device_ptr(psi) || !device_ptr(out) || psi == out) return COLAPM_E_ARG;
    NN_CK(forward(c, psi, out, add ? psi : nullptr, nullptr));
    return COLAPM_OK;
}

static int grads_impl(colapm_nn* c, const float* psi, const float* target, double* loss) {
    if (!c || !psi || !target || !device_ptr(psi) || !device_ptr(target)) return COLAPM_E_ARG;
    NN_CK(cudaMemsetAsync(c->loss, 0, sizeof(double), c->stream));
    NN_CK(forward(c, psi, c->y, nullptr, target));
    NN_CK(backward(c));
    if (loss) {
        double h = 0.0;
        NN_CK(cudaMemcpyAsync(&h, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        NN_CK(cudaStreamSynchronize(c->stream));
        *loss = h / (3.0 * (double)c->nv);
        return check_err(c);
    }
    return COLAPM_OK;
}

int colapm_nn_grads(colapm_nn* c, const float* psi, const float* target, float* grads, double* loss) {
    int r = grads_impl(c, psi, target, loss);
    if (r) return r;
    if (grads) {
        std::vector<float> pad((size_t)LAYERS * LSIZE);
        NN_CK(cudaMemcpyAsync(pad.data(), c->grad, pad.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        NN_CK(cudaStreamSynchronize(c->stream));
        for_each_param([&](size_t k, size_t slot) { grads[k] = pad[slot]; });
        return check_err(c);
    }
    return COLAPM_OK;
}

int colapm_nn_train_step(colapm_nn* c, const float* psi, const float* target, double* loss) {
    int r = grads_impl(c, psi, target, nullptr);
    if (r) return r;
    ++c->steps;
    const float c1 = 1.0f - std::pow(c->cfg.beta1, (float)c->steps);
    const float c2 = 1.0f - std::pow(c->cfg.beta2, (float)c->steps);
    const int total = LAYERS * LSIZE;
    k_adam<<<(total + 255) / 256, 256, 0, c->stream>>>(c->wm, c->m1, c->m2, c->grad, c->cfg.lr, c->cfg.beta1,
                                                       c->cfg.beta2, c->cfg.eps, c1, c2, 1, c->wf, c->wt, c->bias);
    ++c->launches;
    NN_CK(cudaGetLastError());
    if (loss) {
        double h = 0.0;
        NN_CK(cudaMemcpyAsync(&h, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        NN_CK(cudaStreamSynchronize(c->stream));
        *loss = h / (3.0 * (double)c->nv);
        return check_err(c);
    }
    return COLAPM_OK;
}

int colapm_nn_steps(colapm_nn* c) { return c ? c->steps : COLAPM_E_ARG; }

long long colapm_nn_launches(colapm_nn* c) { return c ? c->launches : (long long)COLAPM_E_ARG; }

int colapm_nn_sync(colapm_nn* c) {
    if (!c) return COLAPM_E_ARG;
    return check_err(c);
}

}  // extern "C"
