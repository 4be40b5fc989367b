// z passes with the fused spectral operators for every supported mesh size.
#include "fft_kernels.cuh"

namespace colapm {

template <int N, int MODE>
static cudaError_t fz_mode(float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv, float gnorm,
                           PowerArgs pw, size_t smem, cudaStream_t s) {
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = set_smem(k_fz<N, MODE>, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    dim3 grid(N / 2 / kW, N);
    k_fz<N, MODE><<<grid, YCfg<N>::T, smem, s>>>(in, out, tw, sinc2, deconv, gnorm, pw);
    return cudaGetLastError();
}

template <int N>
static cudaError_t fz_t(int mode, float2* in, ZOut out, const float2* tw, const float* sinc2, int deconv,
                        float gnorm, const PowerArgs* pwp, cudaStream_t s) {
    using C = YCfg<N>;
    PowerArgs pw{};
    if (pwp) pw = *pwp;
    switch (mode) {
        case Z_FORCE: return fz_mode<N, Z_FORCE>(in, out, tw, sinc2, deconv, gnorm, pw, 2 * C::SMEM, s);
        case Z_LPT1: return fz_mode<N, Z_LPT1>(in, out, tw, sinc2, deconv, gnorm, pw, 2 * C::SMEM, s);
        case Z_LPT2: return fz_mode<N, Z_LPT2>(in, out, tw, sinc2, deconv, gnorm, pw, 2 * C::SMEM, s);
        case Z_POWER:
            return fz_mode<N, Z_POWER>(in, out, tw, sinc2, deconv, gnorm, pw,
                                       C::SMEM + (size_t)pw.nbins * 24, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fz(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2,
                      int deconv, float gnorm, const PowerArgs* pw, cudaStream_t s) {
    switch (n_mesh) {
#define X(N) case N: return fz_t<N>(mode, in, out, tw, sinc2, deconv, gnorm, pw, s);
        COLAPM_FOR_MESH_SIZES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace colapm
