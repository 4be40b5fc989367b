// y passes (strided columns, both directions) for every supported mesh size.
#include "fft2.cuh"
#include "fft_kernels.cuh"

namespace colapm {

template <int N, int S, bool BLK>
static cudaError_t fy2(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s) {
    using K = K2<N>;
    constexpr size_t smem = sizeof(float2) * Xch<N, K::RA>::SIZE + sizeof(Tw2);
    static GridCache cache;
    int grid2 = 0;
    cudaError_t e = cached_grid(cache, k2_fy<N, S, BLK>, K::T, smem, &grid2);
    if (e != cudaSuccess) return e;
    const int total = (N / 2 / 8) * N * nfields;
    k2_fy<N, S, BLK><<<grid2 < total ? grid2 : total, K::T, smem, s>>>(data, fstride, tw, nfields);
    return cudaGetLastError();
}

template <int N, int S>
static cudaError_t fy_sign(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s,
                           bool two_stage, bool blocked) {
    if constexpr (F2Has<N>::value) if (two_stage) {
        return blocked ? fy2<N, S, true>(data, fstride, nfields, tw, s) : fy2<N, S, false>(data, fstride, nfields, tw, s);
    }
    if (blocked) return cudaErrorInvalidValue;
    using C = Fy<N>;
    constexpr size_t smem = C::SMEM;
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_fy<N, S>, C::T, smem, &grid);
    if (e != cudaSuccess) return e;
    const int total = (N / 2 / 8) * N * nfields;
    k_fy<N, S><<<grid < total ? grid : total, C::T, smem, s>>>(data, fstride, tw, nfields);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fy_t(int sign, float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s,
                        bool two_stage, bool blocked) {
    return sign < 0 ? fy_sign<N, -1>(data, fstride, nfields, tw, s, two_stage, blocked)
                    : fy_sign<N, +1>(data, fstride, nfields, tw, s, two_stage, blocked);
}

template <int N>
static cudaError_t fy_force_t(float2* data, size_t fstride, const float2* tw, cudaStream_t s) {
    using K = K2<N>;
    constexpr size_t smem = sizeof(float2) * Xch<N, K::RA>::SIZE + sizeof(Tw2);
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k2_fy_force<N>, K::T, smem, &grid);
    if (e != cudaSuccess) return e;
    const int total = (N / 2 / 8) * N;
    k2_fy_force<N><<<grid < total ? grid : total, K::T, smem, s>>>(data, fstride, tw);
    return cudaGetLastError();
}

cudaError_t launch_fy_force(int n_mesh, float2* data, size_t field_stride, const float2* tw, cudaStream_t s) {
    switch (n_mesh) {
        case 512: return fy_force_t<512>(data, field_stride, tw, s);
        case 1024: return fy_force_t<1024>(data, field_stride, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fy(int n_mesh, int sign, float2* data, size_t field_stride, int nfields, const float2* tw,
                      cudaStream_t s, bool two_stage, bool blocked) {
    switch (n_mesh) {
#define X(N) case N: return fy_t<N>(sign, data, field_stride, nfields, tw, s, two_stage, blocked);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
