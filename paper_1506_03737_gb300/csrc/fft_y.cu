// y passes (strided columns, both directions) for every supported mesh size.
#include "fft_kernels.cuh"

namespace colapm {

template <int N>
static cudaError_t fy_t(int sign, float2* data, size_t fstride, int nfields, const float2* tw, cudaStream_t s) {
    using C = YCfg<N>;
    dim3 grid(N / 2 / kW, N, (unsigned)nfields);
    cudaError_t e;
    if (sign < 0) {
        static bool init = false;
        if (!init) { e = set_smem(k_fy<N, -1>, C::SMEM); if (e != cudaSuccess) return e; init = true; }
        k_fy<N, -1><<<grid, C::T, C::SMEM, s>>>(data, fstride, tw);
    } else {
        static bool init = false;
        if (!init) { e = set_smem(k_fy<N, +1>, C::SMEM); if (e != cudaSuccess) return e; init = true; }
        k_fy<N, +1><<<grid, C::T, C::SMEM, s>>>(data, fstride, tw);
    }
    return cudaGetLastError();
}

cudaError_t launch_fy(int n_mesh, int sign, float2* data, size_t field_stride, int nfields, const float2* tw,
                      cudaStream_t s) {
    switch (n_mesh) {
#define X(N) case N: return fy_t<N>(sign, data, field_stride, nfields, tw, s);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
