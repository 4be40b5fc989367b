// Mesh FFT passes of the particle-mesh solver (§2.4 steps 2-3) and of the 2LPT initial
// conditions (§5), on an N^3 real mesh stored [z][y][x].
//
// Layout. The real mesh is also viewed as complex rows of n = N/2 values: x pass (r2c) turns
// each row of N reals into the spectrum for k_x in [0, N/2) (the k_x = N/2 Nyquist value is
// dropped: every spectral operator of this library is zero on Nyquist modes), in the same
// memory; y and z passes then transform columns in place, giving the half spectrum
// [k_z][k_y][k_x]. The inverse runs z, y, then x (c2r) and returns N real values per row.
//
// The real-input transform of length N uses one complex FFT of length n on z[m] = x[2m] +
// i x[2m+1] (the row read as complex) and the split X[k] = E[k] + w^k O[k], w = exp(-2 pi i/N),
// E = (Z[k] + conj Z[n-k]) / 2, O = -i (Z[k] - conj Z[n-k]) / 2; the inverse assembles
// Z'[k] = (X[k] + conj X[n-k]) + i (X[k] - conj X[n-k]) w^-k (X[n] = 0) and returns the
// unnormalised inverse. The 1/N^3 of the inverse transform is folded into the z-pass
// multiplier.
#pragma once

#include "colapm_internal.h"
#include "fft_engine.cuh"

namespace colapm {

constexpr int kW = 8;   // columns per strided tile (8 complex = 64 contiguous bytes per row)

__host__ __device__ constexpr int pow2_floor(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

template <int n>
struct XCfg {   // x pass: WX whole rows of n complex per CTA
    static constexpr int N = 2 * n;
    static constexpr int WA = pow2_floor(4096 / n);
    static constexpr int WX = WA < 4 * n * n ? WA : 4 * n * n;
    static constexpr int T = 256;
    using TL = Tile<n, WX, true>;
};

template <int L>
struct YCfg {   // strided passes: kW columns of length L per CTA
    static constexpr int T0 = L * kW / 16;
    static constexpr int T = T0 < 64 ? 64 : (T0 > 512 ? 512 : T0);
    using TL = Tile<L, kW, false>;
    static constexpr size_t SMEM = sizeof(float2) * TL::SIZE;
};

// ---------------------------------------------------------------------------------------
// x pass, forward (r2c). in: int64 density (I64) or float reals; out: n complex per row.
template <int n, bool I64>
__global__ void __launch_bounds__(256) k_fx_fwd(const void* __restrict__ in_, float2* __restrict__ out,
                                                const float2* __restrict__ tw, float scale, int* err) {
    using C = XCfg<n>;
    using TL = typename C::TL;
    __shared__ float2 sm[TL::SIZE];
    const size_t row0 = (size_t)blockIdx.x * C::WX;
    bool over = false;
    for (int e = threadIdx.x; e < C::WX * n; e += C::T) {
        const int line = e / n, m = e % n;
        const size_t g = (row0 + line) * n + m;
        float2 z;
        if constexpr (I64) {
            const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(in_) + g);
            over |= ((v.x | v.y) >> 63) != 0;
            z.x = fmaf((float)(long long)v.x, scale, -1.0f);
            z.y = fmaf((float)(long long)v.y, scale, -1.0f);
        } else {
            z = reinterpret_cast<const float2*>(in_)[g];
        }
        sm[TL::at(line, m)] = z;
    }
    if constexpr (I64) {
        if (over) atomicOr(err, 1);
    }
    __syncthreads();
    tile_fft<n, C::WX, C::T, true, -1, C::N>(sm, tw);
    constexpr int H = n / 2 + 1;
    for (int e = threadIdx.x; e < C::WX * H; e += C::T) {
        const int line = e / H, k = e % H;
        const int k2 = (n - k) % n;
        const float2 a = sm[TL::at(line, k)], b = sm[TL::at(line, k2)];
        float2* o = out + (row0 + line) * n;
        {   // X[k] from Z[k] = a, Z[n-k] = b
            const float2 bc = cconj(b);
            const float2 E = cscale(cadd(a, bc), 0.5f);
            const float2 d = csub(a, bc);
            const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
            o[k] = cadd(E, cmul(tw[k], O));
        }
        if (k != 0 && k2 != k) {   // X[n-k] from Z[n-k] = b, Z[k] = a
            const float2 ac = cconj(a);
            const float2 E = cscale(cadd(b, ac), 0.5f);
            const float2 d = csub(b, ac);
            const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
            o[k2] = cadd(E, cmul(tw[k2], O));
        }
    }
}

// x pass, inverse (c2r) in place: rows of n complex (k_x < N/2) -> N reals (unnormalised).
template <int n>
__global__ void __launch_bounds__(256) k_fx_inv(float2* __restrict__ data, size_t fstride,
                                                const float2* __restrict__ tw) {
    using C = XCfg<n>;
    using TL = typename C::TL;
    __shared__ float2 sm[TL::SIZE];
    float2* d = data + blockIdx.y * fstride + (size_t)blockIdx.x * C::WX * n;
    for (int e = threadIdx.x; e < C::WX * n; e += C::T) sm[TL::at(e / n, e % n)] = d[e];
    __syncthreads();
    constexpr int H = n / 2 + 1;
    for (int e = threadIdx.x; e < C::WX * H; e += C::T) {
        const int line = e / H, k = e % H;
        const float2 xk = sm[TL::at(line, k)];
        if (k == 0) {
            sm[TL::at(line, 0)] = make_float2(xk.x - xk.y, xk.y + xk.x);   // X0 + i X0
            continue;
        }
        const int k2 = n - k;
        const float2 xk2 = sm[TL::at(line, k2)];
        {
            const float2 xc = cconj(xk2);
            const float2 E = cadd(xk, xc);
            const float2 O = cmul(csub(xk, xc), cconj(tw[k]));
            sm[TL::at(line, k)] = make_float2(E.x - O.y, E.y + O.x);
        }
        if (k2 != k) {
            const float2 xc = cconj(xk);
            const float2 E = cadd(xk2, xc);
            const float2 O = cmul(csub(xk2, xc), cconj(tw[k2]));
            sm[TL::at(line, k2)] = make_float2(E.x - O.y, E.y + O.x);
        }
    }
    __syncthreads();
    tile_fft<n, C::WX, C::T, true, +1, C::N>(sm, tw);
    for (int e = threadIdx.x; e < C::WX * n; e += C::T) d[e] = sm[TL::at(e / n, e % n)];
}

// ---------------------------------------------------------------------------------------
// Tile I/O of the strided passes: kW consecutive complex of each of the L lines.
template <int L, int T>
__device__ __forceinline__ void load_cols(float2* sm, const float2* __restrict__ g, size_t stride) {
    using TL = Tile<L, kW, false>;
    for (int e = threadIdx.x; e < L * (kW / 2); e += T) {
        const int pos = e / (kW / 2), c = (e % (kW / 2)) * 2;
        const float4 v = *reinterpret_cast<const float4*>(g + (size_t)pos * stride + c);
        sm[TL::at(c, pos)] = make_float2(v.x, v.y);
        sm[TL::at(c + 1, pos)] = make_float2(v.z, v.w);
    }
}
template <int L, int T>
__device__ __forceinline__ void store_cols(const float2* sm, float2* __restrict__ g, size_t stride) {
    using TL = Tile<L, kW, false>;
    for (int e = threadIdx.x; e < L * (kW / 2); e += T) {
        const int pos = e / (kW / 2), c = (e % (kW / 2)) * 2;
        const float2 a = sm[TL::at(c, pos)], b = sm[TL::at(c + 1, pos)];
        *reinterpret_cast<float4*>(g + (size_t)pos * stride + c) = make_float4(a.x, a.y, b.x, b.y);
    }
}

// y pass in place; grid (n/kW, N planes z, fields).
template <int L, int S>
__global__ void __launch_bounds__(YCfg<L>::T) k_fy(float2* __restrict__ data, size_t fstride,
                                                    const float2* __restrict__ tw) {
    constexpr int n = L / 2;
    constexpr int T = YCfg<L>::T;
    extern __shared__ float2 sm[];
    float2* g = data + blockIdx.z * fstride + (size_t)blockIdx.y * L * n + blockIdx.x * kW;
    load_cols<L, T>(sm, g, n);
    __syncthreads();
    tile_fft<L, kW, T, false, S, L>(sm, tw);
    store_cols<L, T>(sm, g, n);
}

// Signed index and Nyquist test of FFT bin i on an L grid.
__device__ __forceinline__ int signed_bin(int i, int L) { return i < L / 2 ? i : i - L; }

// z pass with the spectral operator fused; grid (n/kW, N values of k_y).
template <int L, int MODE>
__global__ void __launch_bounds__(YCfg<L>::T) k_fz(float2* __restrict__ in, ZOut out,
                                                    const float2* __restrict__ tw,
                                                    const float* __restrict__ sinc2, int deconv,
                                                    float gnorm, PowerArgs pw) {
    constexpr int n = L / 2;
    constexpr int T = YCfg<L>::T;
    using TL = Tile<L, kW, false>;
    extern __shared__ float2 sm[];
    float2* keep = sm + TL::SIZE;
    const int ky = blockIdx.y, kx0 = blockIdx.x * kW;
    const size_t base = (size_t)ky * n + kx0, stride = (size_t)L * n;
    load_cols<L, T>(sm, in + base, stride);
    __syncthreads();
    if constexpr (MODE != Z_LPT1) tile_fft<L, kW, T, false, -1, L>(sm, tw);

    const int ny = signed_bin(ky, L);
    const bool nyq_y = (ky == L / 2);
    const float kf = 6.283185307179586f / (float)L;

    if constexpr (MODE == Z_POWER) {
        double* ksum = reinterpret_cast<double*>(keep);
        double* psum = ksum + pw.nbins;
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(psum + pw.nbins);
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            ksum[b] = 0.0;
            psum[b] = 0.0;
            cnt[b] = 0ull;
        }
        __syncthreads();
        if (!nyq_y) {
            for (int e = threadIdx.x; e < L * kW; e += T) {
                const int z = e / kW, c = e % kW;
                if (z == L / 2) continue;
                const int nx = kx0 + c, nz = signed_bin(z, L);
                const int n2 = nx * nx + ny * ny + nz * nz;
                if (n2 == 0 || n2 > pw.n2max) continue;
                const int b = pw.bin_of_n2[n2];
                if (b < 0) continue;
                const float2 v = sm[TL::at(c, z)];
                const float w = sinc2[nx] * sinc2[ky] * sinc2[z];
                const float p = (v.x * v.x + v.y * v.y) * pw.pnorm / (w * w);
                const double mult = nx == 0 ? 1.0 : 2.0;   // conjugate twin with k_x -> -k_x
                atomicAdd(&psum[b], mult * (double)p);
                atomicAdd(&ksum[b], mult * pw.kmag_of_n2[n2]);
                atomicAdd(&cnt[b], nx == 0 ? 1ull : 2ull);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            if (cnt[b]) {
                atomicAdd(&pw.psum[b], psum[b]);
                atomicAdd(&pw.ksum[b], ksum[b]);
                atomicAdd(&pw.cnt[b], cnt[b]);
            }
        }
        return;
    } else {
        constexpr int NOUT = MODE == Z_LPT1 ? 9 : 3;
        for (int e = threadIdx.x; e < TL::SIZE; e += T) keep[e] = sm[e];
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < NOUT; ++j) {
            for (int e = threadIdx.x; e < L * kW; e += T) {
                const int z = e / kW, c = e % kW;
                const int nx = kx0 + c, nz = signed_bin(z, L);
                const float2 v = keep[TL::at(c, z)];
                float2 r = make_float2(0.0f, 0.0f);
                if (!nyq_y && z != L / 2 && (nx | ny | nz) != 0) {
                    const float k[3] = {kf * nx, kf * ny, kf * nz};
                    const float k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    if constexpr (MODE == Z_FORCE) {
                        float w = 1.0f;
                        if (deconv) {
                            w = sinc2[nx] * sinc2[ky] * sinc2[z];
                            if (deconv == 2) w *= w;
                        }
                        const float g = k[j] * gnorm / (k2 * w);        // F_j = i k_j delta / (k^2 W^d)
                        r = make_float2(-g * v.y, g * v.x);
                    } else if constexpr (MODE == Z_LPT2) {
                        const float g = k[j] * gnorm / k2;               // Psi2_j = -i k_j S / k^2
                        r = make_float2(g * v.y, -g * v.x);
                    } else {
                        if (j < 3) {                                     // Psi1_j = i k_j delta / k^2
                            const float g = k[j] * gnorm / k2;
                            r = make_float2(-g * v.y, g * v.x);
                        } else {                                         // phi_ab = k_a k_b delta / k^2
                            const int a = j == 3 ? 0 : j == 4 ? 1 : j == 5 ? 2 : j == 6 ? 0 : j == 7 ? 0 : 1;
                            const int b = j == 3 ? 0 : j == 4 ? 1 : j == 5 ? 2 : j == 6 ? 1 : j == 7 ? 2 : 2;
                            const float g = k[a] * k[b] * gnorm / k2;
                            r = make_float2(g * v.x, g * v.y);
                        }
                    }
                }
                sm[TL::at(c, z)] = r;
            }
            __syncthreads();
            tile_fft<L, kW, T, false, +1, L>(sm, tw);
            store_cols<L, T>(sm, out.p[j] + base, stride);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------------------
// Launch helpers (host).
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define COLAPM_FOR_MESH_SIZES(X) X(16) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(1024)

}  // namespace colapm
