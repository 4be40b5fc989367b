// x passes (contiguous rows, r2c / c2r) for every supported mesh size.
#include "fft2.cuh"
#include "fft_kernels.cuh"

namespace colapm {

template <int n, bool I64, bool BLK>
static cudaError_t fx_fwd2(const void* in, float2* out, const float2* tw, float scale, int* err, cudaStream_t s,
                           unsigned long long* zero) {
    using X = X2<n>;
    static GridCache cache;
    int grid2 = 0;
    cudaError_t e = cached_grid(cache, k2_fx_fwd<n, I64, BLK>, X::T, X::SMEM, &grid2);
    if (e != cudaSuccess) return e;
    const int items = 2 * n * 2 * n / 8;
    k2_fx_fwd<n, I64, BLK><<<grid2 < items ? grid2 : items, X::T, X::SMEM, s>>>(in, out, tw, scale, err, items, zero);
    return cudaGetLastError();
}

template <int N, bool I64>
static cudaError_t fx_fwd_t(const void* in, float2* out, const float2* tw, float scale, int* err, cudaStream_t s,
                            bool two_stage, unsigned long long* zero = nullptr, bool blocked = false) {
    constexpr int n = N / 2;
    if constexpr (F2Has<n>::value) if (two_stage) {
        return blocked ? fx_fwd2<n, I64, true>(in, out, tw, scale, err, s, zero)
                       : fx_fwd2<n, I64, false>(in, out, tw, scale, err, s, zero);
    }
    if (blocked) return cudaErrorInvalidValue;
    using C = FxFwd<n, I64>;
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_fx_fwd<n, I64>, C::T, C::SMEM, &grid);
    if (e != cudaSuccess) return e;
    const int items = N * N / 8;
    k_fx_fwd<n, I64><<<grid < items ? grid : items, C::T, C::SMEM, s>>>(in, out, tw, scale, err, items, zero);
    return cudaGetLastError();
}

template <int n, bool BLK>
static cudaError_t fx_inv2(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s, float2* dst) {
    using X = X2<n>;
    static GridCache cache;
    int grid2 = 0;
    cudaError_t e = cached_grid(cache, k2_fx_inv<n, BLK>, X::T, X::SMEM_INV, &grid2);
    if (e != cudaSuccess) return e;
    const int ipf = 2 * n * 2 * n / 8, items = ipf * nfields;
    k2_fx_inv<n, BLK><<<grid2 < items ? grid2 : items, X::T, X::SMEM_INV, s>>>(data, fstride, tw, ipf, nfields, dst);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fx_inv_t(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s,
                            bool two_stage, bool blocked = false, float2* dst = nullptr) {
    constexpr int n = N / 2;
    if constexpr (F2Has<n>::value) if (two_stage) {
        if (blocked) return dst && dst != data ? fx_inv2<n, true>(data, fstride, nfields, tw, s, dst) : cudaErrorInvalidValue;
        return fx_inv2<n, false>(data, fstride, nfields, tw, s, dst ? dst : data);
    }
    if (blocked || (dst && dst != data)) return cudaErrorInvalidValue;
    using C = FxInv<n>;
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_fx_inv<n>, C::T, C::SMEM, &grid);
    if (e != cudaSuccess) return e;
    const int ipf = N * N / 8, items = ipf * nfields;
    k_fx_inv<n><<<grid < items ? grid : items, C::T, C::SMEM, s>>>(data, fstride, tw, ipf, nfields);
    return cudaGetLastError();
}

cudaError_t launch_fx_fwd_i64(int n_mesh, const unsigned long long* in, float2* out, const float2* tw,
                              float scale, int* err, cudaStream_t s, bool two_stage, bool zero_input, bool blocked) {
    unsigned long long* z = zero_input ? const_cast<unsigned long long*>(in) : nullptr;
    switch (n_mesh) {
#define X(N) case N: return fx_fwd_t<N, true>(in, out, tw, scale, err, s, two_stage, z, blocked);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fx_fwd_f32(int n_mesh, const float* in, float2* out, const float2* tw, cudaStream_t s,
                              bool two_stage) {
    switch (n_mesh) {
#define X(N) case N: return fx_fwd_t<N, false>(in, out, tw, 0.0f, nullptr, s, two_stage);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fx_inv(int n_mesh, float2* data, size_t field_stride, int nfields, const float2* tw,
                          cudaStream_t s, bool two_stage, bool blocked, float2* dst) {
    switch (n_mesh) {
#define X(N) case N: return fx_inv_t<N>(data, field_stride, nfields, tw, s, two_stage, blocked, dst);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
