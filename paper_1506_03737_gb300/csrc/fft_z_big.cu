// z passes, mesh sizes 512 and 1024.
#include "fft_z_impl.cuh"

namespace colapm {

#define COLAPM_FZ_BIG(X) X(512) X(1024)
COLAPM_FZ_GROUP(launch_fz_big, COLAPM_FZ_BIG)

}  // namespace colapm
