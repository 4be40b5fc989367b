// Paired-lane 32-point transforms for the 1024-point z pass of the force (L = 32 x 32).
//
// The two-stage z pass gives every radix-32 task to one thread, which then holds 32 complex
// values: with the saved base in shared memory that allows 12 warps per SM. Here a task is split
// over a pair of threads (h = 0, 1), each holding 16 values, so that twice as many warps fit.
// A 32-point DFT of a pair is a radix-2 step between the two threads and a 16-point DFT in each:
//
//  - decimation in time (inputs r = 2m + h, thread h; the DIT form): each thread transforms its
//    16 inputs (E = DFT16 of the even inputs in thread 0, O = of the odd ones in thread 1), then
//    X[k] = E[k] + W^k O[k] and X[k + 16] = E[k] - W^k O[k] (W = exp(S 2 pi i / 32)). Thread h
//    finishes k = i + 8h (i < 8): it needs the other thread's E[k] or O[k] for those k, so each
//    sends 8 values. Thread h ends with outputs r = i + 8h + 16e in slot q = i + 8e.
//  - decimation in frequency (inputs in that same distribution, r = i + 8h + 16e): the first
//    butterfly pairs r = k and k + 16, both in the same thread: Y0[k] = x[k] + x[k + 16],
//    Y1[k] = (x[k] - x[k + 16]) W^k. Thread 0 then collects Y0 (k < 16) and thread 1 Y1, 8 values
//    each way, and a 16-point DFT gives X[2m + h] in slot m.
//
// Every branch on h is a select between two values computed by both threads, so a warp never
// diverges. Each exchange is split into a `send` half (what this thread gives its partner) and a
// `finish` half (given what it received) per butterfly index, so that a host program can emulate
// a pair with the kernel's own arithmetic.
#pragma once

#include "fft2.cuh"

namespace colapm {

__host__ __device__ __forceinline__ float2 csel(bool p, float2 a, float2 b) { return p ? a : b; }

// Output r of the DIT form held in slot q by thread h.
__host__ __device__ __forceinline__ int pair_dit_r(int q, int h) { return (q & 7) + 8 * h + 16 * (q >> 3); }

// DIT, one butterfly index i < 8 at a time: v = DFT16 of this thread's 16 inputs (E for h = 0,
// O for h = 1). dit_send gives the partner E[i + 8] (h = 0) or O[i] (h = 1); dit_finish, given the
// partner's value, leaves X[i + 8h] in v[i] and X[i + 8h + 16] in v[i + 8]. Index i touches only
// v[i] and v[i + 8], so the pairs can be exchanged one at a time.
__host__ __device__ __forceinline__ float2 pair_dit_send(const float2* v, int h, int i) {
    return csel(h != 0, v[i], v[i + 8]);
}
template <int S>
__host__ __device__ __forceinline__ void pair_dit_finish(float2* v, int h, int i, float2 recv) {
    const float2 e = csel(h != 0, recv, v[i]);       // E[i + 8h]
    const float2 o = csel(h != 0, v[i + 8], recv);   // O[i + 8h]
    const float2 w = csel(h != 0, root<32, S>(i + 8), root<32, S>(i));
    const float2 t = cmul(o, w);
    v[i] = cadd(e, t);       // X[i + 8h]
    v[i + 8] = csub(e, t);   // X[i + 8h + 16]
}

// DIF, one index i < 8 at a time: v holds x[r] for r = pair_dit_r(q, h) in slot q. dif_send makes
// the butterfly of k = i + 8h (Y0[k] = x[k] + x[k + 16] in v[i], Y1[k] = (x[k] - x[k + 16]) W^k
// in v[i + 8]) and gives the partner Y1[i] (h = 0) or Y0[i + 8] (h = 1); dif_finish puts the
// partner's value in place, so that v holds Y_h[0..15]; pair_dif_dft then leaves X[2m + h] in v[m].
template <int S>
__host__ __device__ __forceinline__ float2 pair_dif_send(float2* v, int h, int i) {
    const float2 a = v[i], b = v[i + 8];
    const float2 w = csel(h != 0, root<32, S>(i + 8), root<32, S>(i));
    v[i] = cadd(a, b);
    v[i + 8] = cmul(csub(a, b), w);
    return csel(h != 0, v[i], v[i + 8]);
}
__host__ __device__ __forceinline__ void pair_dif_finish(float2* v, int h, int i, float2 recv) {
    v[i] = csel(h != 0, recv, v[i]);              // Y_h[i]
    v[i + 8] = csel(h != 0, v[i + 8], recv);      // Y_h[i + 8]
}
template <int S>
__host__ __device__ __forceinline__ void pair_dif_dft(float2* v) { dft<16, S>(v); }

// Twiddles of stage B for task j, inputs r = 2m + h: v[m] *= w^(S j r), w = exp(-2 pi i / L), from
// the tables w^(8 M j) (M = r >> 3 = m >> 2) and w^j (r & 7 = 2 (m & 3) + h).
template <int S>
__host__ __device__ __forceinline__ void pair_twiddle(float2* v, const Tw2* t, int j, int h) {
    float2 w1 = t->w1[j];
    if (S > 0) w1 = cconj(w1);
    const float2 w2 = cmul(w1, w1);
    float2 q[4];
    q[0] = csel(h != 0, w1, make_float2(1.0f, 0.0f));
#pragma unroll
    for (int i = 1; i < 4; ++i) q[i] = cmul(q[i - 1], w2);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        float2 w = q[m & 3];
        if (m >= 4) {
            float2 b = t->w8[m >> 2][j];
            if (S > 0) b = cconj(b);
            w = cmul(b, w);
        }
        v[m] = cmul(v[m], w);
    }
}

#ifdef __CUDACC__
__device__ __forceinline__ float2 pair_swap(float2 a) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, 4), __shfl_xor_sync(0xffffffffu, a.y, 4));
}
// The exchanges on the device: every send first, then the shuffles, then every finish (the same
// arithmetic as index by index; measured faster than interleaving them at 2 CTAs per SM).
template <int S>
__device__ __forceinline__ void pair_dit(float2* v, int h) {
    float2 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = pair_dit_send(v, h, i);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = pair_swap(x[i]);
#pragma unroll
    for (int i = 0; i < 8; ++i) pair_dit_finish<S>(v, h, i, x[i]);
}
template <int S>
__device__ __forceinline__ void pair_dif(float2* v, int h) {
    float2 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = pair_dif_send<S>(v, h, i);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = pair_swap(x[i]);
#pragma unroll
    for (int i = 0; i < 8; ++i) pair_dif_finish(v, h, i, x[i]);
    pair_dif_dft<S>(v);
}

// ---------------------------------------------------------------------------------------------
// Force z pass, 1024-point lines, blocked layout, 4-column tiles, 256 threads: thread
// (c, h, j) = (tid & 3, (tid >> 2) & 1, tid >> 3) is half h of task j of column c (the partner is
// lane ^ 4). The chain is that of k2_fz<1024, Z_FORCE, 4, true>: forward z (stage A DIT from
// global memory, exchange, stage B DIT), the Green's function with CIC deconvolution, the saved
// base B = k_z A in shared memory, and two inverse z transforms (stage A DIF, exchange, stage B
// DIT) written as the bases A' (field 0) and B' (field 2).
constexpr int PZ_T = 256;

template <int MINB>
__global__ void __launch_bounds__(PZ_T, MINB)
    k2_fz_pair(const float2* __restrict__ in, ZOut out, const float2* __restrict__ tw, const float* __restrict__ sinc2,
               int deconv, float gnorm) {
    constexpr int L = 1024, R = 32, n = L / 2, C = 4, NTILE = (n / C) * L;
    using X = Xch<L, R, C>;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    float2* save = xb + X::SIZE;
    Tw2* tws = reinterpret_cast<Tw2*>(save + X::SIZE);
    load_tw2<L, L>(tws, tw, PZ_T);
    __syncthreads();
    const float kf = 6.283185307179586f / (float)L;
    const int tid = threadIdx.x, c = tid & 3, h = (tid >> 2) & 1, j = tid >> 3;
    // tile -> (ky, kx0) as in k2_fz (blocked layout, 4-column tiles)
    auto tile_of = [&](int tt, int& ky_, int& kx0_) {
        const int qq = tt >> 3;
        ky_ = 8 * (qq / (2 * (n / 8))) + (tt & 7);
        kx0_ = ((qq / 2) % (n / 8)) * 8 + (qq % 2) * C;
    };
    auto load_a = [&](int tt, float2* dst) {
        int ky_, kx0_;
        tile_of(tt, ky_, kx0_);
        const size_t b = hs_index<L, true>(kx0_ + c, ky_, 0);
#pragma unroll
        for (int m = 0; m < 16; ++m) dst[m] = __ldcg(in + b + (size_t)(j + R * (2 * m + h)) * 64);
    };
    for (int t = blockIdx.x; t < NTILE; t += gridDim.x) {
        int ky, kx0;
        tile_of(t, ky, kx0);
        const size_t base = hs_index<L, true>(kx0 + c, ky, 0);
        const int ny = sbin(ky, L), nx = kx0 + c;
        const bool nyq_y = ky == L / 2;
        float2 v[16];
        // forward stage A: inputs z = j + 32 r, r = 2m + h
        load_a(t, v);
        dft<16, -1>(v);
        pair_dit<-1>(v, h);
#pragma unroll
        for (int q = 0; q < 16; ++q) xb[X::at(c, j * R + pair_dit_r(q, h))] = v[q];
        __syncthreads();
        // forward stage B: inputs j + 32 r, r = 2m + h; outputs X[j + 32 r], r = pair_dit_r(q, h)
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = xb[X::at(c, j + R * (2 * m + h))];
        pair_twiddle<-1>(v, tws, j, h);
        dft<16, -1>(v);
        pair_dit<-1>(v, h);
        // bases: A = g X, B = k_z A; g = gnorm / (k^2 W^d), 0 on excluded modes
        {
            const int nxy2 = nx * nx + ny * ny;
            const float wxy = deconv ? sinc2[nx] * sinc2[ky] : 1.0f;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int z = j + R * pair_dit_r(q, h);
                const int nz = sbin(z, L);
                const int n2 = nxy2 + nz * nz;
                float w = 1.0f;
                if (deconv) {
                    w = wxy * sinc2[z];
                    if (deconv == 2) w *= w;
                }
                const float g = !nyq_y && z != L / 2 && n2 != 0 ? __fdividef(gnorm, kf * kf * (float)n2 * w) : 0.0f;
                v[q] = cscale(v[q], g);
                save[X::at(c, z)] = cscale(v[q], kf * (float)nz);
            }
        }
        __syncthreads();   // forward exchange buffer free
#pragma unroll 1
        for (int bi = 0; bi < 2; ++bi) {
            if (bi > 0) {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = save[X::at(c, j + R * pair_dit_r(q, h))];
            }
            // inverse stage A (DIF): outputs 2m + h of task j
            pair_dif<+1>(v, h);
#pragma unroll
            for (int m = 0; m < 16; ++m) xb[X::at(c, j * R + 2 * m + h)] = v[m];
            __syncthreads();
            // inverse stage B: inputs j + 32 r, r = 2m + h; outputs z = j + 32 pair_dit_r(q, h)
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = xb[X::at(c, j + R * (2 * m + h))];
            pair_twiddle<+1>(v, tws, j, h);
            dft<16, +1>(v);
            pair_dit<+1>(v, h);
            float2* dst = out.p[bi == 0 ? 0 : 2];
#pragma unroll
            for (int q = 0; q < 16; ++q) dst[base + (size_t)(j + R * pair_dit_r(q, h)) * 64] = v[q];
            __syncthreads();   // exchange buffer free for the next base / tile
        }
    }
}

template <int MINB>
struct PairZ {
    static constexpr size_t SMEM = sizeof(float2) * 2 * (size_t)Xch<1024, 32, 4>::SIZE + sizeof(Tw2);
};
#endif

}  // namespace colapm
