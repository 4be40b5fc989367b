// x passes (contiguous rows, r2c / c2r) for every supported mesh size.
#include "fft2.cuh"
#include "fft_kernels.cuh"

namespace colapm {

template <int N, bool I64>
static cudaError_t fx_fwd_t(const void* in, float2* out, const float2* tw, float scale, int* err, cudaStream_t s,
                            bool two_stage, unsigned long long* zero = nullptr) {
    constexpr int n = N / 2;
    if constexpr (F2Has<n>::value) if (two_stage) {
        using X = X2<n>;
        static int grid2 = 0;
        if (!grid2) {
            cudaError_t e = set_smem(k2_fx_fwd<n, I64>, X::SMEM);
            if (e != cudaSuccess) return e;
            grid2 = persistent_grid(k2_fx_fwd<n, I64>, X::T, X::SMEM);
        }
        const int items = N * N / 8;
        k2_fx_fwd<n, I64><<<grid2 < items ? grid2 : items, X::T, X::SMEM, s>>>(in, out, tw, scale, err, items, zero);
        return cudaGetLastError();
    }
    using C = FxFwd<n, I64>;
    static int grid = 0;
    if (!grid) {
        cudaError_t e = set_smem(k_fx_fwd<n, I64>, C::SMEM);
        if (e != cudaSuccess) return e;
        grid = persistent_grid(k_fx_fwd<n, I64>, C::T, C::SMEM);
    }
    const int items = N * N / 8;
    k_fx_fwd<n, I64><<<grid < items ? grid : items, C::T, C::SMEM, s>>>(in, out, tw, scale, err, items, zero);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fx_inv_t(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s,
                            bool two_stage) {
    constexpr int n = N / 2;
    if constexpr (F2Has<n>::value) if (two_stage) {
        using X = X2<n>;
        static int grid2 = 0;
        if (!grid2) {
            cudaError_t e = set_smem(k2_fx_inv<n>, X::SMEM_INV);
            if (e != cudaSuccess) return e;
            grid2 = persistent_grid(k2_fx_inv<n>, X::T, X::SMEM_INV);
        }
        const int ipf = N * N / 8, items = ipf * nfields;
        k2_fx_inv<n><<<grid2 < items ? grid2 : items, X::T, X::SMEM_INV, s>>>(data, fstride, tw, ipf, nfields);
        return cudaGetLastError();
    }
    using C = FxInv<n>;
    static int grid = 0;
    if (!grid) {
        cudaError_t e = set_smem(k_fx_inv<n>, C::SMEM);
        if (e != cudaSuccess) return e;
        grid = persistent_grid(k_fx_inv<n>, C::T, C::SMEM);
    }
    const int ipf = N * N / 8, items = ipf * nfields;
    k_fx_inv<n><<<grid < items ? grid : items, C::T, C::SMEM, s>>>(data, fstride, tw, ipf, nfields);
    return cudaGetLastError();
}

cudaError_t launch_fx_fwd_i64(int n_mesh, const unsigned long long* in, float2* out, const float2* tw,
                              float scale, int* err, cudaStream_t s, bool two_stage, bool zero_input) {
    unsigned long long* z = zero_input ? const_cast<unsigned long long*>(in) : nullptr;
    switch (n_mesh) {
#define X(N) case N: return fx_fwd_t<N, true>(in, out, tw, scale, err, s, two_stage, z);
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
                          cudaStream_t s, bool two_stage) {
    switch (n_mesh) {
#define X(N) case N: return fx_inv_t<N>(data, field_stride, nfields, tw, s, two_stage);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
