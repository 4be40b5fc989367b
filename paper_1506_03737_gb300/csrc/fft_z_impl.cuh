// z passes with the fused spectral operators: the per-size launchers, instantiated by the
// translation units fft_z.cu, fft_z_mid.cu and fft_z_big.cu (one group of mesh sizes each, so that
// they compile in parallel).
#pragma once

#include "fft2.cuh"
#include "fft_kernels.cuh"
#include "fft_pair.cuh"


namespace colapm {

template <int N, int MODE, bool BLK>
static cudaError_t fz2(float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv, float gnorm, PowerArgs pw,
                       cudaStream_t s) {
    if constexpr (N == 1024 && MODE == Z_FORCE && BLK) {
        // 1024-point force lines: each radix-32 task on a pair of lanes (16 values per thread),
        // two CTAs of 256 threads per SM (measured at 1024^3: 4.93 ms against 5.50 for the
        // one-thread-per-task kernel at three CTAs of 128 threads, 6.1-6.4 ms with the pair kernel
        // held to 80 registers for three CTAs, 5.32 ms with the next tile's inputs loaded into
        // registers during the inverse transforms)
        constexpr int MINB = 2;
        static GridCache cache;
        int grid = 0;
        cudaError_t e = cached_grid(cache, k2_fz_pair<MINB>, PZ_T, PairZ<MINB>::SMEM, &grid);
        if (e != cudaSuccess) return e;
        const int total = (N / 2 / 4) * N;
        k2_fz_pair<MINB><<<grid < total ? grid : total, PZ_T, PairZ<MINB>::SMEM, s>>>(in, out, tw, sinc2, deconv, gnorm);
        return cudaGetLastError();
    } else {
        // Blocked layout: 4-column tiles (32-byte rows whose 512-byte runs the neighbouring tiles
        // complete), which with the prefetch buffer measured 2% faster than 8-column ones (34% for the
        // power spectrum), and with direct loads fit three CTAs per SM. Standard layout: 8 columns
        // (4-column rows there are 32 bytes 4 MB apart).
        constexpr int CZ = BLK ? 4 : 8;
        constexpr bool DIRECT = BLK;   // blocked layout: loads straight into registers, three CTAs per SM
        using Z = Z2<N, MODE, CZ, DIRECT>;
        const size_t smem = Z::SMEM + (MODE == Z_POWER ? (size_t)pw.nbins * 24 + (size_t)(pw.nbins + 1) * 4 : 0);
        static GridCache cache;
        int grid2 = 0;
        cudaError_t e = cached_grid(cache, k2_fz<N, MODE, CZ, BLK, DIRECT>, Z::T, smem, &grid2);
        if (e != cudaSuccess) return e;
        const int total = (N / 2 / CZ) * N;
        k2_fz<N, MODE, CZ, BLK, DIRECT><<<grid2 < total ? grid2 : total, Z::T, smem, s>>>(in, out, tw, sinc2, deconv, gnorm, pw);
        return cudaGetLastError();
    }
}

template <int N, int MODE>
static cudaError_t fz_mode(float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv, float gnorm,
                           PowerArgs pw, cudaStream_t s, bool two_stage, bool blocked) {
    if constexpr (F2Has<N>::value && MODE != Z_SCALE_FWD && MODE != Z_SCALE_INV) if (two_stage) {
        if constexpr (MODE == Z_FORCE || MODE == Z_POWER) {
            if (blocked) return fz2<N, MODE, true>(in, out, tw, sinc2, deconv, gnorm, pw, s);
        } else {
            if (blocked) return cudaErrorInvalidValue;
        }
        return fz2<N, MODE, false>(in, out, tw, sinc2, deconv, gnorm, pw, s);
    }
    if (blocked) return cudaErrorInvalidValue;
    using C = Fz<N, MODE>;
    const size_t smem = C::BASE_SMEM + (MODE == Z_POWER ? (size_t)pw.nbins * 24 + (size_t)(pw.nbins + 1) * 4 : 0);
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_fz<N, MODE>, C::T, smem, &grid);
    if (e != cudaSuccess) return e;
    const int total = (N / 2 / 8) * N;
    k_fz<N, MODE><<<grid < total ? grid : total, C::T, smem, s>>>(in, out, tw, sinc2, deconv, gnorm, pw);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fz_t(int mode, float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv,
                        float gnorm, const PowerArgs* pwp, cudaStream_t s, bool ts, bool blk) {
    PowerArgs pw{};
    if (pwp) pw = *pwp;
    switch (mode) {
        case Z_FORCE: return fz_mode<N, Z_FORCE>(in, out, tw, sinc2, deconv, gnorm, pw, s, ts, blk);
        case Z_LPT1: return fz_mode<N, Z_LPT1>(in, out, tw, sinc2, deconv, gnorm, pw, s, ts, blk);
        case Z_LPT2: return fz_mode<N, Z_LPT2>(in, out, tw, sinc2, deconv, gnorm, pw, s, ts, blk);
        case Z_POWER: return fz_mode<N, Z_POWER>(in, out, tw, sinc2, deconv, gnorm, pw, s, ts, blk);
        case Z_SCALE_FWD: return fz_mode<N, Z_SCALE_FWD>(in, out, tw, sinc2, deconv, gnorm, pw, s, false, blk);
        case Z_SCALE_INV: return fz_mode<N, Z_SCALE_INV>(in, out, tw, sinc2, deconv, gnorm, pw, s, false, blk);
        default: return cudaErrorInvalidValue;
    }
}

// One group of mesh sizes: the launcher for n_mesh, or cudaErrorInvalidValue if not in the group.
#define COLAPM_FZ_GROUP(NAME, SIZES)                                                                        \
    cudaError_t NAME(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2,      \
                     int deconv, float gnorm, const PowerArgs* pw, cudaStream_t s, bool two_stage,          \
                     bool blocked) {                                                                        \
        switch (n_mesh) {                                                                                   \
            SIZES(COLAPM_FZ_CASE)                                                                           \
            default: return cudaErrorInvalidValue;                                                          \
        }                                                                                                   \
    }
#define COLAPM_FZ_CASE(N) case N: return fz_t<N>(mode, in, out, tw, sinc2, deconv, gnorm, pw, s, two_stage, blocked);

cudaError_t launch_fz_mid(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv,
                          float gnorm, const PowerArgs* pw, cudaStream_t s, bool two_stage, bool blocked);
cudaError_t launch_fz_big(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv,
                          float gnorm, const PowerArgs* pw, cudaStream_t s, bool two_stage, bool blocked);

}  // namespace colapm
