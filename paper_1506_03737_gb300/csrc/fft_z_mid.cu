// z passes, mesh sizes 256, 320 and 384.
#include "fft_z_impl.cuh"

namespace colapm {

#define COLAPM_FZ_MID(X) X(256) X(320) X(384)
COLAPM_FZ_GROUP(launch_fz_mid, COLAPM_FZ_MID)

}  // namespace colapm
