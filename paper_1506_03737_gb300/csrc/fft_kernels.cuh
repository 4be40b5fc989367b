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
// Every pass is a persistent kernel over tiles of 8 lines (8 mesh rows for x, 8 adjacent
// columns for y and z) that prefetches the next tile with cp.async into a second shared buffer
// while the current one is transformed. Column tiles are copied with 16-byte cp.async.cg
// (L2 only), row tiles with 8-byte cp.async.ca, the int64 density through a 16-byte staging
// tile.
#pragma once

#include "colapm_internal.h"
#include "fft_engine.cuh"
#include "launch_cache.h"

namespace colapm {

template <int L>
struct TCfg {   // threads for a tile of L rows (each butterfly covers a column pair)
    static constexpr int T0 = L / 2;
    static constexpr int T = T0 < 64 ? 64 : (T0 > 512 ? 512 : T0);
    static constexpr size_t TILE = sizeof(float2) * 8 * L;
};

// ---- tile I/O --------------------------------------------------------------------------------
// Column tile: row r <- g[r * stride + 0..7] (complex).
template <int L, int T>
__device__ __forceinline__ void ld_cols(float2* sm, const float2* g, size_t stride) {
    float4* s4 = reinterpret_cast<float4*>(sm);
    for (int e = threadIdx.x; e < L * 4; e += T) {
        const int r = e >> 2, q = e & 3;
        cp_async16_cg(s4 + CT<L>::a4(r, q), g + (size_t)r * stride + 2 * q);
    }
}
// out[r * stride + c] = f(c) * tile[r][c] (IMAG: times i).
template <int L, int T, bool IMAG, typename F>
__device__ __forceinline__ void st_cols_scaled(const float2* sm, float2* g, size_t stride, F f) {
    const float4* s4 = reinterpret_cast<const float4*>(sm);
    for (int e = threadIdx.x; e < L * 4; e += T) {
        const int r = e >> 2, q = e & 3;
        const float4 v = s4[CT<L>::a4(r, q)];
        const float sa = f(2 * q), sb = f(2 * q + 1);
        float4 o;
        if constexpr (IMAG)
            o = make_float4(-sa * v.y, sa * v.x, -sb * v.w, sb * v.z);
        else
            o = make_float4(sa * v.x, sa * v.y, sb * v.z, sb * v.w);
        *reinterpret_cast<float4*>(g + (size_t)r * stride + 2 * q) = o;
    }
}
template <int L, int T>
__device__ __forceinline__ void st_cols(const float2* sm, float2* g, size_t stride) {
    const float4* s4 = reinterpret_cast<const float4*>(sm);
    for (int e = threadIdx.x; e < L * 4; e += T) {
        const int r = e >> 2, q = e & 3;
        *reinterpret_cast<float4*>(g + (size_t)r * stride + 2 * q) = s4[CT<L>::a4(r, q)];
    }
}
// Row staging: 8 lines of n contiguous complex, copied with coalesced 16-byte cp.async into a
// row-major buffer with a pitch of n + 4 elements (8-byte elements; a warp touching 8 lines x 4
// positions then spreads over all banks), and transposed through shared memory into the column
// tile. ESZ is the element size in bytes (8 for complex float, 16 for an int64 pair).
template <int n, int ESZ>
struct RowStage {
    static constexpr int PITCH = n + (ESZ == 8 ? 4 : 2);     // elements per staged line
    static constexpr size_t BYTES = (size_t)8 * PITCH * ESZ;
};
template <int n, int T, int ESZ>
__device__ __forceinline__ void ld_rows_stage(unsigned char* stg, const unsigned char* g) {
    constexpr int CH = n * ESZ / 16;   // 16-byte chunks per line
    for (int e = threadIdx.x; e < 8 * CH; e += T) {
        const int c = e / CH, k = e % CH;
        cp_async16_cg(stg + ((size_t)c * RowStage<n, ESZ>::PITCH * ESZ + (size_t)k * 16), g + ((size_t)c * n * ESZ + (size_t)k * 16));
    }
}
// staged complex rows -> column tile
template <int n, int T>
__device__ __forceinline__ void stage_to_tile(float2* tile, const float2* stg) {
    for (int e = threadIdx.x; e < n * 8; e += T) {
        const int c = e & 7, p = e >> 3;
        tile[CT<n>::a2(p, c)] = stg[c * RowStage<n, 8>::PITCH + p];
    }
}
// column tile -> staged rows -> coalesced 16-byte stores of 8 lines of n complex at g
template <int n, int T>
__device__ __forceinline__ void tile_to_rows(const float2* tile, float2* stg, float2* g) {
    for (int e = threadIdx.x; e < n * 8; e += T) {
        const int c = e & 7, p = e >> 3;
        stg[c * RowStage<n, 8>::PITCH + p] = tile[CT<n>::a2(p, c)];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 8 * (n / 2); e += T) {
        const int c = e / (n / 2), k = e % (n / 2);
        *reinterpret_cast<float4*>(g + (size_t)c * n + 2 * k) =
            *reinterpret_cast<const float4*>(stg + c * RowStage<n, 8>::PITCH + 2 * k);
    }
}


// ---------------------------------------------------------------------------------------------
// x passes: threads per CTA (the stages use n/2 of them; the copies and transposes all).
template <int n>
struct XT {
    static constexpr int T = n < 64 ? 64 : (n > 512 ? 512 : n);
};

// x pass, forward (r2c), persistent over groups of 8 rows. in: int64 density (I64) converted
// to delta = rho * scale - 1 (err bit 0 when a cell has its top bit set), or float reals.
template <int n, bool I64>
struct FxFwd {
    static constexpr int N = 2 * n, T = XT<n>::T;
    using In = RowStage<n, I64 ? 16 : 8>;
    using Out = RowStage<n, 8>;
    static constexpr size_t SMEM = 2 * In::BYTES + TCfg<n>::TILE + sizeof(float2) * N;
};

template <int n, bool I64>
__global__ void __launch_bounds__(XT<n>::T) k_fx_fwd(const void* __restrict__ in_, float2* __restrict__ out,
                                                      const float2* __restrict__ tw, float scale, int* err,
                                                      int nitems, unsigned long long* zero) {
    using C = FxFwd<n, I64>;
    constexpr int T = C::T, N = C::N, ESZ = I64 ? 16 : 8;
    extern __shared__ float4 smem4[];
    unsigned char* base = reinterpret_cast<unsigned char*>(smem4);
    float2* tile = reinterpret_cast<float2*>(base + 2 * C::In::BYTES);
    float2* stw = tile + 8 * n;
    for (int e = threadIdx.x; e < N; e += T) stw[e] = tw[e];
    const unsigned char* src = reinterpret_cast<const unsigned char*>(in_);
    int t = blockIdx.x;
    if (t < nitems) ld_rows_stage<n, T, ESZ>(base, src + (size_t)t * 8 * n * ESZ);
    cp_async_commit();
    bool over = false;
    for (int it = 0; t < nitems; t += gridDim.x, ++it) {
        unsigned char* stg = base + (it & 1) * C::In::BYTES;
        const int tn = t + gridDim.x;
        if (tn < nitems) ld_rows_stage<n, T, ESZ>(base + ((it + 1) & 1) * C::In::BYTES, src + (size_t)tn * 8 * n * ESZ);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if constexpr (I64) {
            if (zero) {   // the staged rows of tile t are in shared memory: clear them in the input
                ulonglong2* z = reinterpret_cast<ulonglong2*>(zero) + (size_t)t * 8 * n;
                for (int e = threadIdx.x; e < n * 8; e += T) __stcs(z + e, make_ulonglong2(0ull, 0ull));
            }
            const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(stg);
            for (int e = threadIdx.x; e < n * 8; e += T) {
                const int c = e & 7, p = e >> 3;
                const ulonglong2 v = s2[c * C::In::PITCH + p];
                over |= ((v.x | v.y) >> 63) != 0;
                tile[CT<n>::a2(p, c)] =
                    make_float2(fmaf((float)(long long)v.x, scale, -1.0f), fmaf((float)(long long)v.y, scale, -1.0f));
            }
        } else {
            stage_to_tile<n, T>(tile, reinterpret_cast<const float2*>(stg));
        }
        __syncthreads();
        tile_fft<n, T, -1, N>(tile, stw);
        constexpr int H = n / 2 + 1;
        for (int e = threadIdx.x; e < 8 * H; e += T) {
            const int c = e & 7, k = e >> 3;
            const int k2 = (n - k) % n;
            const float2 a = tile[CT<n>::a2(k, c)], b = tile[CT<n>::a2(k2, c)];
            {   // X[k] from Z[k] = a, Z[n-k] = b
                const float2 bc = cconj(b);
                const float2 E = cscale(cadd(a, bc), 0.5f);
                const float2 d = csub(a, bc);
                tile[CT<n>::a2(k, c)] = cadd(E, cmul(stw[k], make_float2(0.5f * d.y, -0.5f * d.x)));
            }
            if (k != 0 && k2 != k) {   // X[n-k] from Z[n-k] = b, Z[k] = a
                const float2 ac = cconj(a);
                const float2 E = cscale(cadd(b, ac), 0.5f);
                const float2 d = csub(b, ac);
                tile[CT<n>::a2(k2, c)] = cadd(E, cmul(stw[k2], make_float2(0.5f * d.y, -0.5f * d.x)));
            }
        }
        __syncthreads();
        tile_to_rows<n, T>(tile, reinterpret_cast<float2*>(stg), out + (size_t)t * 8 * n);
        __syncthreads();
    }
    cp_async_wait<0>();
    if constexpr (I64) {
        if (over) atomicOr(err, 1);
    }
}

// x pass, inverse (c2r) in place, persistent over groups of 8 rows of `nfields` arrays.
template <int n>
struct FxInv {
    static constexpr int N = 2 * n, T = XT<n>::T;
    using St = RowStage<n, 8>;
    static constexpr size_t SMEM = 2 * St::BYTES + TCfg<n>::TILE + sizeof(float2) * N;
};

template <int n>
__global__ void __launch_bounds__(XT<n>::T) k_fx_inv(float2* __restrict__ data, size_t fstride,
                                                      const float2* __restrict__ tw, int items_per_field,
                                                      int nfields) {
    using C = FxInv<n>;
    constexpr int T = C::T, N = C::N;
    extern __shared__ float4 smem4[];
    unsigned char* base = reinterpret_cast<unsigned char*>(smem4);
    float2* tile = reinterpret_cast<float2*>(base + 2 * C::St::BYTES);
    float2* stw = tile + 8 * n;
    for (int e = threadIdx.x; e < N; e += T) stw[e] = tw[e];
    const int nitems = items_per_field * nfields;
    auto gptr = [&](int t) { return data + (size_t)(t / items_per_field) * fstride + (size_t)(t % items_per_field) * 8 * n; };
    int t = blockIdx.x;
    if (t < nitems) ld_rows_stage<n, T, 8>(base, reinterpret_cast<const unsigned char*>(gptr(t)));
    cp_async_commit();
    for (int it = 0; t < nitems; t += gridDim.x, ++it) {
        float2* stg = reinterpret_cast<float2*>(base + (it & 1) * C::St::BYTES);
        const int tn = t + gridDim.x;
        if (tn < nitems)
            ld_rows_stage<n, T, 8>(base + ((it + 1) & 1) * C::St::BYTES, reinterpret_cast<const unsigned char*>(gptr(tn)));
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        stage_to_tile<n, T>(tile, stg);
        __syncthreads();
        constexpr int H = n / 2 + 1;
        for (int e = threadIdx.x; e < 8 * H; e += T) {
            const int c = e & 7, k = e >> 3;
            const float2 xk = tile[CT<n>::a2(k, c)];
            if (k == 0) {
                tile[CT<n>::a2(0, c)] = make_float2(xk.x - xk.y, xk.y + xk.x);   // X0 + i X0
                continue;
            }
            const int k2 = n - k;
            const float2 xk2 = tile[CT<n>::a2(k2, c)];
            {
                const float2 xc = cconj(xk2);
                const float2 E = cadd(xk, xc);
                const float2 O = cmul(csub(xk, xc), cconj(stw[k]));
                tile[CT<n>::a2(k, c)] = make_float2(E.x - O.y, E.y + O.x);
            }
            if (k2 != k) {
                const float2 xc = cconj(xk);
                const float2 E = cadd(xk2, xc);
                const float2 O = cmul(csub(xk2, xc), cconj(stw[k2]));
                tile[CT<n>::a2(k2, c)] = make_float2(E.x - O.y, E.y + O.x);
            }
        }
        __syncthreads();
        tile_fft<n, T, +1, N>(tile, stw);
        tile_to_rows<n, T>(tile, stg, gptr(t));
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------------
// y pass in place, persistent over all column tiles of `nfields` arrays.
template <int L>
struct Fy {
    static constexpr int T = TCfg<L>::T;
    static constexpr size_t SMEM = 2 * TCfg<L>::TILE + sizeof(float2) * L;
};

template <int L, int S>
__global__ void __launch_bounds__(TCfg<L>::T) k_fy(float2* __restrict__ data, size_t fstride,
                                                    const float2* __restrict__ tw, int nfields) {
    constexpr int n = L / 2;
    constexpr int T = Fy<L>::T;
    constexpr int NG = n / 8;            // column groups per plane
    constexpr int TPF = NG * L;          // tiles per field
    extern __shared__ float4 smem4[];
    float2* bufs = reinterpret_cast<float2*>(smem4);
    float2* stw = bufs + 2 * 8 * L;
    for (int e = threadIdx.x; e < L; e += T) stw[e] = tw[e];
    const int total = TPF * nfields;
    auto tile_ptr = [&](int t) {
        const int f = t / TPF, r = t % TPF;
        return data + (size_t)f * fstride + (size_t)(r / NG) * L * n + (r % NG) * 8;
    };
    int t = blockIdx.x;
    if (t < total) ld_cols<L, T>(bufs, tile_ptr(t), n);
    cp_async_commit();
    for (int it = 0; t < total; t += gridDim.x, ++it) {
        float2* cur = bufs + (it & 1) * 8 * L;
        const int tn = t + gridDim.x;
        if (tn < total) ld_cols<L, T>(bufs + ((it + 1) & 1) * 8 * L, tile_ptr(tn), n);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        tile_fft<L, T, S, L>(cur, stw);
        st_cols<L, T>(cur, tile_ptr(t), n);
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Signed index of FFT bin i on an L grid.
__device__ __forceinline__ int signed_bin(int i, int L) { return i < L / 2 ? i : i - L; }

template <int MODE>
struct ZCfg {
    static constexpr bool SCALE = MODE == Z_SCALE_FWD || MODE == Z_SCALE_INV;
    static constexpr bool FWD = MODE != Z_LPT1 && MODE != Z_SCALE_INV;   // forward z transform first
    static constexpr bool PREFETCH = FWD;                                // double-buffered input
    static constexpr int NBASE = MODE == Z_LPT1 ? 3 : (MODE == Z_POWER || SCALE ? 0 : 2);
    static constexpr int NBUF = (PREFETCH ? 2 : 1) + (NBASE > 1 ? NBASE - 1 : 0);
};

template <int L, int MODE>
struct Fz {
    static constexpr int T = TCfg<L>::T;
    static constexpr size_t BASE_SMEM = ZCfg<MODE>::NBUF * TCfg<L>::TILE + sizeof(float2) * L;
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
__global__ void __launch_bounds__(TCfg<L>::T) k_fz(float2* __restrict__ in, ZOut out,
                                                    const float2* __restrict__ tw,
                                                    const float* __restrict__ sinc2, int deconv,
                                                    float gnorm, PowerArgs pw) {
    constexpr int n = L / 2;
    constexpr int T = TCfg<L>::T;
    constexpr int NG = n / 8;
    constexpr int NTILE = NG * L;
    constexpr int TS = 8 * L;            // tile size (float2)
    using Z = ZCfg<MODE>;
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    float2* aux = sm + (Z::PREFETCH ? 2 : 1) * TS;   // bases B, C
    float2* stw = sm + Z::NBUF * TS;
    for (int e = threadIdx.x; e < L; e += T) stw[e] = tw[e];
    double* ksum = reinterpret_cast<double*>(stw + L);
    double* psum = ksum + pw.nbins;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(psum + pw.nbins);
    int* lo = reinterpret_cast<int*>(cnt + pw.nbins);
    if constexpr (MODE == Z_POWER) {
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            ksum[b] = 0.0;
            psum[b] = 0.0;
            cnt[b] = 0ull;
        }
        for (int b = threadIdx.x; b <= pw.nbins; b += T) lo[b] = pw.n2_lo[b];
    }
    const float kf = 6.283185307179586f / (float)L;
    const size_t stride = (size_t)L * n;
    auto tile_base = [&](int t) { return (size_t)(t / NG) * n + (t % NG) * 8; };

    int t = blockIdx.x;
    if constexpr (Z::PREFETCH) {
        if (t < NTILE) ld_cols<L, T>(sm, in + tile_base(t), stride);
        cp_async_commit();
    }
    for (int it = 0; t < NTILE; t += gridDim.x, ++it) {
        float2* cur = sm;
        if constexpr (Z::PREFETCH) {
            cur = sm + (it & 1) * TS;
            const int tn = t + gridDim.x;
            if (tn < NTILE) ld_cols<L, T>(sm + ((it + 1) & 1) * TS, in + tile_base(tn), stride);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            ld_cols<L, T>(cur, in + tile_base(t), stride);
            cp_async_commit();
            cp_async_wait<0>();
        }
        __syncthreads();
        if constexpr (Z::FWD) tile_fft<L, T, -1, L>(cur, stw);

        const int ky = t / NG, kx0 = (t % NG) * 8;
        const int ny = signed_bin(ky, L);
        const bool nyq_y = (ky == L / 2);
        const size_t base = tile_base(t);

        if constexpr (MODE == Z_POWER) {
            // Each thread bins a run of consecutive z of one column, flushing when the bin changes.
            if (!nyq_y) {
                constexpr int PER = L * 8 / T;
                const int c = threadIdx.x % 8;
                bin_column_run(kx0 + c, ny, (threadIdx.x / 8) * PER, PER, L, sinc2[kx0 + c] * sinc2[ky], sinc2, lo, pw,
                               psum, ksum, cnt, [&](int z) { return cur[CT<L>::a2(z, c)]; });
            }
            __syncthreads();
            continue;
        } else if constexpr (Z::SCALE) {
            // multiply every mode by the table value of its |n|^2 (sinc2 holds the table), zero on the
            // Nyquist planes; then the inverse z transform (Z_SCALE_INV) or nothing (Z_SCALE_FWD)
            for (int e = threadIdx.x; e < L * 8; e += T) {
                const int z = e >> 3, c = e & 7;
                const int nx = kx0 + c, nz = signed_bin(z, L);
                const float m = nyq_y || z == L / 2 ? 0.0f : sinc2[nx * nx + ny * ny + nz * nz];
                const int i2 = CT<L>::a2(z, c);
                cur[i2] = cscale(cur[i2], m);
            }
            __syncthreads();
            if constexpr (MODE == Z_SCALE_INV) tile_fft<L, T, +1, L>(cur, stw);
            st_cols<L, T>(cur, out.p[0] + base, stride);
            __syncthreads();
        } else {
            // bases: A = g v, B = k_z A (, C = k_z^2 A), g = gnorm / (k^2 [W^d]), 0 on excluded modes
            float4* c4 = reinterpret_cast<float4*>(cur);
            float4* a4p = reinterpret_cast<float4*>(aux);
            for (int e = threadIdx.x; e < L * 4; e += T) {
                const int z = e >> 2, q = e & 3;
                const int nz = signed_bin(z, L);
                const int i4 = CT<L>::a4(z, q);
                float g[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int nx = kx0 + 2 * q + h;
                    g[h] = 0.0f;
                    if (!nyq_y && z != L / 2 && (nx | ny | nz) != 0) {
                        const float k2 = kf * kf * (float)(nx * nx + ny * ny + nz * nz);
                        float w = 1.0f;
                        if (MODE == Z_FORCE && deconv) {
                            w = sinc2[nx] * sinc2[ky] * sinc2[z];
                            if (deconv == 2) w *= w;
                        }
                        g[h] = gnorm / (k2 * w);
                    }
                }
                const float4 v = c4[i4];
                const float4 a = make_float4(g[0] * v.x, g[0] * v.y, g[1] * v.z, g[1] * v.w);
                const float kz = kf * (float)nz;
                c4[i4] = a;
                a4p[i4] = make_float4(kz * a.x, kz * a.y, kz * a.z, kz * a.w);
                if constexpr (Z::NBASE == 3)
                    a4p[TS / 2 + i4] = make_float4(kz * kz * a.x, kz * kz * a.y, kz * kz * a.z, kz * kz * a.w);
            }
            __syncthreads();
            tile_fft<L, T, +1, L>(cur, stw);
            tile_fft<L, T, +1, L>(aux, stw);
            if constexpr (Z::NBASE == 3) tile_fft<L, T, +1, L>(aux + TS, stw);
            const float kyv = kf * (float)ny;
            auto kxv = [&](int c) { return kf * (float)(kx0 + c); };
            constexpr float sg = MODE == Z_LPT2 ? -1.0f : 1.0f;
            st_cols_scaled<L, T, true>(cur, out.p[0] + base, stride, [&](int c) { return sg * kxv(c); });
            st_cols_scaled<L, T, true>(cur, out.p[1] + base, stride, [&](int) { return sg * kyv; });
            st_cols_scaled<L, T, true>(aux, out.p[2] + base, stride, [&](int) { return sg; });
            if constexpr (MODE == Z_LPT1) {
                st_cols_scaled<L, T, false>(cur, out.p[3] + base, stride, [&](int c) { return kxv(c) * kxv(c); });
                st_cols_scaled<L, T, false>(cur, out.p[4] + base, stride, [&](int) { return kyv * kyv; });
                st_cols_scaled<L, T, false>(aux + TS, out.p[5] + base, stride, [&](int) { return 1.0f; });
                st_cols_scaled<L, T, false>(cur, out.p[6] + base, stride, [&](int c) { return kxv(c) * kyv; });
                st_cols_scaled<L, T, false>(aux, out.p[7] + base, stride, [&](int c) { return kxv(c); });
                st_cols_scaled<L, T, false>(aux, out.p[8] + base, stride, [&](int) { return kyv; });
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

#define COLAPM_FOR_MESH_SIZES(X) X(16) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(1024)

}  // namespace colapm
