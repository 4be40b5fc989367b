// z passes, mesh sizes 16 ... 192, and the dispatch over all sizes.
#include "fft_z_impl.cuh"

namespace colapm {

#define COLAPM_FZ_SMALL(X) X(16) X(32) X(64) X(96) X(128) X(160) X(192)
static COLAPM_FZ_GROUP(launch_fz_small, COLAPM_FZ_SMALL)

cudaError_t launch_fz(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2,
                      int deconv, float gnorm, const PowerArgs* pw, cudaStream_t s, bool two_stage, bool blocked) {
    if (n_mesh >= 512) return launch_fz_big(n_mesh, mode, in, out, tw, sinc2, deconv, gnorm, pw, s, two_stage, blocked);
    if (n_mesh >= 256) return launch_fz_mid(n_mesh, mode, in, out, tw, sinc2, deconv, gnorm, pw, s, two_stage, blocked);
    return launch_fz_small(n_mesh, mode, in, out, tw, sinc2, deconv, gnorm, pw, s, two_stage, blocked);
}

}  // namespace colapm
