// Mesh FFT passes of the particle-mesh solver (§2.4 steps 2-3) and of the 2LPT initial
// conditions (§5), on an N^3 real mesh stored [z][y][x].
//
// Layout. The real mesh is also viewed as complex rows of n = N/2 values: the x pass (r2c)
// turns each row of N reals into the spectrum for k_x in [0, N/2) (the k_x = N/2 Nyquist value
// is dropped: every spectral operator of this library is zero on Nyquist modes), in the same
// memory; y and z passes then transform columns in place, giving the half spectrum
// [k_z][k_y][k_x]. The inverse runs z, y, then x (c2r) and returns N real values per row.
//
// The real-input transform of length N uses one complex FFT of length n on z[m] = x[2m] +
// i x[2m+1] (the row read as complex) and the split X[k] = E[k] + w^k O[k], w = exp(-2 pi i/N),
// E = (Z[k] + conj Z[n-k]) / 2, O = -i (Z[k] - conj Z[n-k]) / 2; the inverse assembles
// Z'[k] = (X[k] + conj X[n-k]) + i (X[k] - conj X[n-k]) w^-k (X[n] = 0) and returns the
// unnormalised inverse. The 1/N^3 of the inverse transform is folded into the z-pass
// multiplier.
//
// Strided passes (y, z) run persistent CTAs over column tiles (kW adjacent columns, all L
// positions) with the next tile prefetched by cp.async into a second shared buffer while the
// current one is transformed.
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
struct YCfg {   // strided passes: kW columns of length L per tile
    static constexpr int T0 = L * kW / 16;
    static constexpr int T = T0 < 64 ? 64 : (T0 > 512 ? 512 : T0);
    using TL = Tile<L, kW, false>;
    static constexpr size_t TILE_BYTES = sizeof(float2) * TL::SIZE;
    static constexpr size_t TW_BYTES = sizeof(float2) * L;
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------------------
// x pass, forward (r2c). in: int64 density (I64) or float reals; out: n complex per row.
template <int n, bool I64>
__global__ void __launch_bounds__(256) k_fx_fwd(const void* __restrict__ in_, float2* __restrict__ out,
                                                const float2* __restrict__ tw, float scale, int* err) {
    using C = XCfg<n>;
    using TL = typename C::TL;
    __shared__ float2 sm[TL::SIZE];
    __shared__ float2 stw[C::N];
    for (int e = threadIdx.x; e < C::N; e += C::T) stw[e] = tw[e];
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
    tile_fft<n, C::WX, C::T, true, -1, C::N>(sm, stw);
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
            o[k] = cadd(E, cmul(stw[k], O));
        }
        if (k != 0 && k2 != k) {   // X[n-k] from Z[n-k] = b, Z[k] = a
            const float2 ac = cconj(a);
            const float2 E = cscale(cadd(b, ac), 0.5f);
            const float2 d = csub(b, ac);
            const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);
            o[k2] = cadd(E, cmul(stw[k2], O));
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
    __shared__ float2 stw[C::N];
    for (int e = threadIdx.x; e < C::N; e += C::T) stw[e] = tw[e];
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
            const float2 O = cmul(csub(xk, xc), cconj(stw[k]));
            sm[TL::at(line, k)] = make_float2(E.x - O.y, E.y + O.x);
        }
        if (k2 != k) {
            const float2 xc = cconj(xk);
            const float2 E = cadd(xk2, xc);
            const float2 O = cmul(csub(xk2, xc), cconj(stw[k2]));
            sm[TL::at(line, k2)] = make_float2(E.x - O.y, E.y + O.x);
        }
    }
    __syncthreads();
    tile_fft<n, C::WX, C::T, true, +1, C::N>(sm, stw);
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
__device__ __forceinline__ void load_cols_async(float2* sm, const float2* __restrict__ g, size_t stride) {
    using TL = Tile<L, kW, false>;
    for (int e = threadIdx.x; e < L * kW; e += T) {
        const int pos = e / kW, c = e % kW;
        cp_async8(&sm[TL::at(c, pos)], g + (size_t)pos * stride + c);
    }
}
// Store out[pos][c] = (i s_c) * A[pos][c] (IMAG: multiply by i) or s_c * A[pos][c], where the
// per-column scale s_c = scale_c(c).
template <int L, int T, bool IMAG, typename F>
__device__ __forceinline__ void store_cols_scaled(const float2* sm, float2* __restrict__ g, size_t stride, F scale_c) {
    using TL = Tile<L, kW, false>;
    for (int e = threadIdx.x; e < L * (kW / 2); e += T) {
        const int pos = e / (kW / 2), c = (e % (kW / 2)) * 2;
        const float2 a = sm[TL::at(c, pos)], b = sm[TL::at(c + 1, pos)];
        const float sa = scale_c(c), sb = scale_c(c + 1);
        float4 v;
        if constexpr (IMAG)
            v = make_float4(-sa * a.y, sa * a.x, -sb * b.y, sb * b.x);
        else
            v = make_float4(sa * a.x, sa * a.y, sb * b.x, sb * b.y);
        *reinterpret_cast<float4*>(g + (size_t)pos * stride + c) = v;
    }
}
template <int L, int T>
__device__ __forceinline__ void store_cols(const float2* sm, float2* __restrict__ g, size_t stride) {
    store_cols_scaled<L, T, false>(sm, g, stride, [](int) { return 1.0f; });
}

// y pass in place, persistent over all column tiles of `nfields` arrays.
template <int L, int S>
__global__ void __launch_bounds__(YCfg<L>::T) k_fy(float2* __restrict__ data, size_t fstride,
                                                    const float2* __restrict__ tw, int nfields) {
    constexpr int n = L / 2;
    constexpr int T = YCfg<L>::T;
    constexpr int NG = n / kW;           // column groups per plane
    constexpr int TPF = NG * L;          // tiles per field
    using TL = Tile<L, kW, false>;
    extern __shared__ float2 sm[];
    float2* stw = sm + 2 * TL::SIZE;
    for (int e = threadIdx.x; e < L; e += T) stw[e] = tw[e];
    const int total = TPF * nfields;
    auto tile_ptr = [&](int t) {
        const int f = t / TPF, r = t % TPF;
        return data + (size_t)f * fstride + (size_t)(r / NG) * L * n + (r % NG) * kW;
    };
    int t = blockIdx.x;
    if (t < total) load_cols_async<L, T>(sm, tile_ptr(t), n);
    cp_async_commit();
    for (int it = 0; t < total; t += gridDim.x, ++it) {
        float2* cur = sm + (it & 1) * TL::SIZE;
        float2* nxt = sm + ((it + 1) & 1) * TL::SIZE;
        const int tn = t + gridDim.x;
        if (tn < total) load_cols_async<L, T>(nxt, tile_ptr(tn), n);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        tile_fft<L, kW, T, false, S, L>(cur, stw);
        store_cols<L, T>(cur, tile_ptr(t), n);
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Signed index of FFT bin i on an L grid.
__device__ __forceinline__ int signed_bin(int i, int L) { return i < L / 2 ? i : i - L; }

template <int MODE>
struct ZCfg {
    static constexpr bool FWD = MODE != Z_LPT1;                      // forward z transform first
    static constexpr bool PREFETCH = MODE != Z_LPT1;                 // double-buffered input
    static constexpr int NBASE = MODE == Z_LPT1 ? 3 : (MODE == Z_POWER ? 0 : 2);
    static constexpr int NBUF = (PREFETCH ? 2 : 1) + (NBASE > 1 ? NBASE - 1 : 0);
};

// z pass with the spectral operator fused, persistent over the (k_y, column group) tiles.
//
// Every output of a mode is a column scale (1, i k_x, i k_y, k_x^2, ...) times the inverse z
// transform of one of at most three base spectra, because k_x and k_y are constant along a
// z line: with phi = g delta / (k^2 [W^d]) the bases are phi, k_z phi and k_z^2 phi, so
//   force:  F_x = i k_x A, F_y = i k_y A, F_z = i B            (A = IFFT_z phi, B = IFFT_z k_z phi)
//   LPT2:   Psi2_j = -(the same with S in place of delta)
//   LPT1:   Psi1 as force (d = 0); phi_xx = k_x^2 A, phi_yy = k_y^2 A, phi_zz = C, phi_xy = k_x k_y A,
//           phi_xz = k_x B, phi_yz = k_y B                      (C = IFFT_z k_z^2 phi)
template <int L, int MODE>
__global__ void __launch_bounds__(YCfg<L>::T) k_fz(float2* __restrict__ in, ZOut out,
                                                    const float2* __restrict__ tw,
                                                    const float* __restrict__ sinc2, int deconv,
                                                    float gnorm, PowerArgs pw) {
    constexpr int n = L / 2;
    constexpr int T = YCfg<L>::T;
    constexpr int NG = n / kW;
    constexpr int NTILE = NG * L;
    using TL = Tile<L, kW, false>;
    using Z = ZCfg<MODE>;
    extern __shared__ float2 sm[];
    float2* aux = sm + (Z::PREFETCH ? 2 : 1) * TL::SIZE;   // bases B, C
    float2* stw = sm + Z::NBUF * TL::SIZE;
    for (int e = threadIdx.x; e < L; e += T) stw[e] = tw[e];
    double* ksum = reinterpret_cast<double*>(stw + L);
    double* psum = ksum + pw.nbins;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(psum + pw.nbins);
    if constexpr (MODE == Z_POWER) {
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            ksum[b] = 0.0;
            psum[b] = 0.0;
            cnt[b] = 0ull;
        }
    }
    const float kf = 6.283185307179586f / (float)L;
    const size_t stride = (size_t)L * n;
    auto tile_base = [&](int t) { return (size_t)(t / NG) * n + (t % NG) * kW; };

    int t = blockIdx.x;
    if constexpr (Z::PREFETCH) {
        if (t < NTILE) load_cols_async<L, T>(sm, in + tile_base(t), stride);
        cp_async_commit();
    }
    for (int it = 0; t < NTILE; t += gridDim.x, ++it) {
        float2* cur = sm;
        if constexpr (Z::PREFETCH) {
            cur = sm + (it & 1) * TL::SIZE;
            float2* nxt = sm + ((it + 1) & 1) * TL::SIZE;
            const int tn = t + gridDim.x;
            if (tn < NTILE) load_cols_async<L, T>(nxt, in + tile_base(tn), stride);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            load_cols<L, T>(cur, in + tile_base(t), stride);
        }
        __syncthreads();
        if constexpr (Z::FWD) tile_fft<L, kW, T, false, -1, L>(cur, stw);

        const int ky = t / NG, kx0 = (t % NG) * kW;
        const int ny = signed_bin(ky, L);
        const bool nyq_y = (ky == L / 2);
        const size_t base = tile_base(t);

        if constexpr (MODE == Z_POWER) {
            // Each thread bins a run of consecutive z of one column, flushing when the bin changes.
            constexpr int PER = L * kW / T;
            const int c = threadIdx.x % kW, z0 = (threadIdx.x / kW) * PER;
            const int nx = kx0 + c;
            int rb = -1;
            double rp = 0.0, rk = 0.0;   // FP64 sums of FP32 per-mode values
            unsigned rc = 0;
            const float mult = nx == 0 ? 1.0f : 2.0f;    // conjugate twin with k_x -> -k_x
            if (!nyq_y) {
                for (int zz = 0; zz < PER; ++zz) {
                    const int z = z0 + zz;
                    if (z == L / 2) continue;
                    const int nz = signed_bin(z, L);
                    const int n2 = nx * nx + ny * ny + nz * nz;
                    const int b = (n2 == 0 || n2 > pw.n2max) ? -1 : pw.bin_of_n2[n2];
                    if (b < 0) continue;
                    if (b != rb) {
                        if (rb >= 0) {
                            atomicAdd(&psum[rb], rp);
                            atomicAdd(&ksum[rb], rk);
                            atomicAdd(&cnt[rb], (unsigned long long)rc);
                        }
                        rb = b;
                        rp = 0.0;
                        rk = 0.0;
                        rc = 0;
                    }
                    const float2 v = cur[TL::at(c, z)];
                    const float w = sinc2[nx] * sinc2[ky] * sinc2[z];
                    rp += (double)(mult * (v.x * v.x + v.y * v.y) * pw.pnorm / (w * w));
                    rk += (double)mult * pw.kmag_of_n2[n2];
                    rc += nx == 0 ? 1u : 2u;
                }
            }
            if (rb >= 0) {
                atomicAdd(&psum[rb], rp);
                atomicAdd(&ksum[rb], rk);
                atomicAdd(&cnt[rb], (unsigned long long)rc);
            }
            __syncthreads();
            continue;
        } else {
            // bases
            for (int e = threadIdx.x; e < L * kW; e += T) {
                const int z = e / kW, c = e % kW;
                const int nx = kx0 + c, nz = signed_bin(z, L);
                const int i = TL::at(c, z);
                float g = 0.0f;
                if (!nyq_y && z != L / 2 && (nx | ny | nz) != 0) {
                    const float k2 = kf * kf * (float)(nx * nx + ny * ny + nz * nz);
                    float w = 1.0f;
                    if (MODE == Z_FORCE && deconv) {
                        w = sinc2[nx] * sinc2[ky] * sinc2[z];
                        if (deconv == 2) w *= w;
                    }
                    g = gnorm / (k2 * w);
                }
                const float2 v = cur[i];
                const float2 a = make_float2(g * v.x, g * v.y);
                const float kz = kf * (float)nz;
                cur[i] = a;
                aux[i] = make_float2(kz * a.x, kz * a.y);
                if constexpr (Z::NBASE == 3) aux[TL::SIZE + i] = make_float2(kz * kz * a.x, kz * kz * a.y);
            }
            __syncthreads();
            tile_fft<L, kW, T, false, +1, L>(cur, stw);
            tile_fft<L, kW, T, false, +1, L>(aux, stw);
            if constexpr (Z::NBASE == 3) tile_fft<L, kW, T, false, +1, L>(aux + TL::SIZE, stw);
            const float kyv = kf * (float)ny;
            auto kxv = [&](int c) { return kf * (float)(kx0 + c); };
            constexpr float sg = MODE == Z_LPT2 ? -1.0f : 1.0f;
            store_cols_scaled<L, T, true>(cur, out.p[0] + base, stride, [&](int c) { return sg * kxv(c); });
            store_cols_scaled<L, T, true>(cur, out.p[1] + base, stride, [&](int) { return sg * kyv; });
            store_cols_scaled<L, T, true>(aux, out.p[2] + base, stride, [&](int) { return sg; });
            if constexpr (MODE == Z_LPT1) {
                store_cols_scaled<L, T, false>(cur, out.p[3] + base, stride, [&](int c) { return kxv(c) * kxv(c); });
                store_cols_scaled<L, T, false>(cur, out.p[4] + base, stride, [&](int) { return kyv * kyv; });
                store_cols_scaled<L, T, false>(aux + TL::SIZE, out.p[5] + base, stride, [&](int) { return 1.0f; });
                store_cols_scaled<L, T, false>(cur, out.p[6] + base, stride, [&](int c) { return kxv(c) * kyv; });
                store_cols_scaled<L, T, false>(aux, out.p[7] + base, stride, [&](int c) { return kxv(c); });
                store_cols_scaled<L, T, false>(aux, out.p[8] + base, stride, [&](int) { return kyv; });
            }
            __syncthreads();
        }
    }
    if constexpr (Z::PREFETCH) cp_async_wait<0>();
    if constexpr (MODE == Z_POWER) {
        __syncthreads();
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            if (cnt[b]) {
                atomicAdd(&pw.psum[b], psum[b]);
                atomicAdd(&pw.ksum[b], ksum[b]);
                atomicAdd(&pw.cnt[b], cnt[b]);
            }
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

// Persistent grid: resident CTAs per SM x SMs (computed once per kernel and shared-memory size).
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (per < 1) per = 1;
    return per * sms;
}

#define COLAPM_FOR_MESH_SIZES(X) X(16) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(1024)

}  // namespace colapm
