// Initial-condition kernels (§5, §2.1): Gaussian field and the 2LPT source term.
#include "colapm_internal.h"

namespace colapm {

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011), from its published definition:
// ten rounds of two 32x32->64 multiplies by fixed constants with the high halves xored into
// the other words and the round key; the key is bumped by two Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += W0;
            k.y += W1;
        }
        const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// (2 (w >> 9) + 1) 2^-24: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float uniform_open(unsigned w) { return (float)(2u * (w >> 9) + 1u) * 5.9604644775390625e-8f; }

__device__ __forceinline__ float2 draw(unsigned long long m, unsigned long long seed) {
    const uint4 r = philox4x32_10(make_uint4((unsigned)m, (unsigned)(m >> 32), 0u, 0u),
                                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float u1 = uniform_open(r.x), u2 = uniform_open(r.y);
    const float a = sqrtf(-2.0f * logf(u1)) * 0.70710678118654752440f;
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(a * c, a * s);
}

// One thread per half-grid mode (iz, iy, ix < N/2): delta_k = amp(|n|^2) g, Hermitian on ix = 0.
__global__ void k_gaussian_field(int n, const unsigned long long* __restrict__ seedp, const float* __restrict__ amp_of_n2,
                                 float2* __restrict__ dk) {
    const unsigned long long seed = *seedp;
    const int h = n / 2;
    const size_t total = (size_t)n * n * h;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int ix = (int)(t % h), iy = (int)((t / h) % n), iz = (int)(t / ((size_t)h * n));
    float2 v = make_float2(0.0f, 0.0f);
    if (iy != h && iz != h) {
        const int nx = ix, ny = iy < h ? iy : iy - n, nz = iz < h ? iz : iz - n;
        const int n2 = nx * nx + ny * ny + nz * nz;
        if (n2 > 0) {
            const unsigned long long m = ((unsigned long long)iz * n + iy) * n + ix;
            unsigned long long src = m;
            bool conj = false;
            if (ix == 0) {   // the larger full-grid index of each conjugate pair mirrors its partner
                const unsigned long long part = ((unsigned long long)((n - iz) % n) * n + (n - iy) % n) * n;
                if (m > part) {
                    src = part;
                    conj = true;
                }
            }
            const float2 g = draw(src, seed);
            const float a = amp_of_n2[n2];
            v = make_float2(a * g.x, conj ? -a * g.y : a * g.y);
        }
    }
    dk[t] = v;
}

// S = phi_xx phi_yy + phi_xx phi_zz + phi_yy phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2
// (the right-hand side of the phi2 Poisson equation, §2.1); phi = [xx, yy, zz, xy, xz, yz].
__global__ void k_lpt2_source(const float* __restrict__ phi, size_t n3, float* __restrict__ src) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const float xx = phi[i], yy = phi[n3 + i], zz = phi[2 * n3 + i];
    const float xy = phi[3 * n3 + i], xz = phi[4 * n3 + i], yz = phi[5 * n3 + i];
    src[i] = xx * yy + xx * zz + yy * zz - xy * xy - xz * xz - yz * yz;
}

__global__ void k_set_u64(unsigned long long* dst, unsigned long long value) { *dst = value; }

// Sum of phi^2 over the field: FP32 per thread over a grid-stride run, a warp sum, then one FP64
// atomic per warp.
__global__ void k_sum_sq(const float* __restrict__ phi, size_t n, double* __restrict__ sum2) {
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = phi[i];
        acc += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum2, acc);
}

// Local non-Gaussianity (§5): Phi = phi + f_NL (phi^2 - <phi^2>).
__global__ void k_local_fnl(float* __restrict__ phi, size_t n, float fnl, const double* __restrict__ sum2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mean = (float)(*sum2 / (double)n);
    const float v = phi[i];
    phi[i] = fmaf(fnl, fmaf(v, v, -mean), v);
}

}  // namespace

cudaError_t launch_local_fnl(float* phi, size_t n, double fnl, double* sum2, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sum2, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_sum_sq<<<1024, 256, 0, s>>>(phi, n, sum2);
    k_local_fnl<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi, n, (float)fnl, sum2);
    return cudaGetLastError();
}

cudaError_t launch_set_u64(unsigned long long* dst, unsigned long long value, cudaStream_t s) {
    k_set_u64<<<1, 1, 0, s>>>(dst, value);
    return cudaGetLastError();
}

cudaError_t launch_gaussian_field(int np, const unsigned long long* seed, const float* amp_of_n2, float2* dk,
                                  cudaStream_t s) {
    const size_t total = (size_t)np * np * (np / 2);
    k_gaussian_field<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(np, seed, amp_of_n2, dk);
    return cudaGetLastError();
}

cudaError_t launch_lpt2_source(const float* phi, size_t np3, float* src, cudaStream_t s) {
    k_lpt2_source<<<(unsigned)((np3 + 255) / 256), 256, 0, s>>>(phi, np3, src);
    return cudaGetLastError();
}

}  // namespace colapm
