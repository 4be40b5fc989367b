// x passes (contiguous rows, r2c / c2r) for every supported mesh size.
#include "fft_kernels.cuh"

namespace colapm {

template <int N>
static cudaError_t fx_fwd_t(bool i64, const void* in, float2* out, const float2* tw, float scale, int* err,
                            cudaStream_t s) {
    constexpr int n = N / 2;
    using C = XCfg<n>;
    const unsigned grid = (unsigned)((size_t)N * N / C::WX);
    if (i64)
        k_fx_fwd<n, true><<<grid, C::T, 0, s>>>(in, out, tw, scale, err);
    else
        k_fx_fwd<n, false><<<grid, C::T, 0, s>>>(in, out, tw, scale, err);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fx_inv_t(float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s) {
    constexpr int n = N / 2;
    using C = XCfg<n>;
    dim3 grid((unsigned)((size_t)N * N / C::WX), (unsigned)nfields);
    k_fx_inv<n><<<grid, C::T, 0, s>>>(data, fstride, tw);
    return cudaGetLastError();
}

cudaError_t launch_fx_fwd_i64(int n_mesh, const unsigned long long* in, float2* out, const float2* tw,
                              float scale, int* err, cudaStream_t s) {
    switch (n_mesh) {
#define X(N) case N: return fx_fwd_t<N>(true, in, out, tw, scale, err, s);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fx_fwd_f32(int n_mesh, const float* in, float2* out, const float2* tw, cudaStream_t s) {
    switch (n_mesh) {
#define X(N) case N: return fx_fwd_t<N>(false, in, out, tw, 0.0f, nullptr, s);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fx_inv(int n_mesh, float2* data, size_t field_stride, int nfields, const float2* tw,
                          cudaStream_t s) {
    switch (n_mesh) {
#define X(N) case N: return fx_inv_t<N>(data, field_stride, nfields, tw, s);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
