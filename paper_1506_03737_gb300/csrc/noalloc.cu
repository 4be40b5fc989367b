// colapm_power_noalloc: the power spectrum of caller-owned device particle positions, with all
// working memory in one fixed, file-scope device array instead of cudaMalloc.
//
// It is the colapm_power pipeline (fixed-point CIC deposit, x/y/z forward transforms, binning)
// run on scratch carved out of g_noalloc_scratch. Every call shares that array, which keeps the
// last call's contents; each call clears what must start at zero (density mesh, accumulators,
// error word). Two calls that overlap on the GPU (different streams, no ordering) race on it.
//
// Set-up: host code cannot use the symbol's name as a device address (in host code it names a
// host-side stand-in). The first call on each device, with that device current, resolves the
// device address with cudaGetSymbolAddress and caches it; later calls on that device reuse it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "colapm_internal.h"

namespace colapm {
namespace {

constexpr int kMaxNm = COLAPM_NOALLOC_MAX_NM;
constexpr int kMaxBins = COLAPM_NOALLOC_MAX_BINS;

// Byte offsets of the scratch regions (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kRho = 0;                                                        // u64 [nm^3]
constexpr size_t kSpec = align256(kRho + sizeof(unsigned long long) * kMaxNm * kMaxNm * kMaxNm);   // float2 [nm^3/2]
constexpr size_t kTw = align256(kSpec + sizeof(float2) * kMaxNm * kMaxNm * kMaxNm / 2);            // float2 [nm]
constexpr size_t kSinc = align256(kTw + sizeof(float2) * kMaxNm);                  // float [nm]
constexpr size_t kEdges = align256(kSinc + sizeof(float) * kMaxNm);                // double [nbins + 1]
constexpr size_t kBin = align256(kEdges + sizeof(double) * (kMaxBins + 1));        // int [nbins + 1] thresholds
constexpr size_t kAcc = align256(kBin + sizeof(int) * (kMaxBins + 1));             // double [3 nbins]
constexpr size_t kOut = align256(kAcc + sizeof(double) * 3 * kMaxBins);            // k, P (double), n (i64)
constexpr size_t kErr = align256(kOut + sizeof(double) * 3 * kMaxBins);            // int [4]
constexpr size_t kBytes = align256(kErr + 4 * sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

// Fixed-point CIC deposit of xyz cell / offset arrays (the definition of pm_kernels.cu).
__global__ void k_deposit_xyz(const int* __restrict__ cell, const float* __restrict__ off, long long n, int nm,
                              unsigned long long* __restrict__ rho, int* err) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c[3], f[3];
    for (int j = 0; j < 3; ++j) {
        c[j] = cell[3 * p + j];
        const float o = off[3 * p + j];
        if (!(c[j] >= 0 && c[j] < nm && o >= 0.0f && o < 1.0f)) {
            atomicOr(err, 2);
            return;
        }
        f[j] = __float2int_rn(o * 32768.0f);
        if (f[j] == 32768) {
            f[j] = 0;
            c[j] = c[j] + 1 == nm ? 0 : c[j] + 1;
        }
    }
    const unsigned long long w[3][2] = {{32768ull - f[0], (unsigned long long)f[0]},
                                        {32768ull - f[1], (unsigned long long)f[1]},
                                        {32768ull - f[2], (unsigned long long)f[2]}};
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const unsigned long long wt = w[0][dx] * w[1][dy] * w[2][dz];
                if (!wt) continue;
                const int x = (c[0] + dx) % nm, y = (c[1] + dy) % nm, z = (c[2] + dz) % nm;
                // n_particles has no upper bound here, so a cell could wrap past 2^64 and come back
                // below 2^63 unseen by the transform's top-bit check: flag it from the old value.
                const unsigned long long old = atomicAdd(rho + ((size_t)z * nm + y) * nm + x, wt);
                if (old + wt < old || old + wt >= (1ull << 63)) atomicOr(err, 1);
            }
}

// Bin thresholds in FP64: n2_lo[b] = smallest integer |n|^2 with kf sqrt(|n|^2) >= edges[b]
// (sqrt correctly rounded), n2max + 1 if none; one thread per edge, binary search over |n|^2.
__global__ void k_bin_thresholds(const double* __restrict__ edges, int nbins, double kf, int n2max,
                                 int* __restrict__ lo) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbins) return;
    int a = 0, z = n2max + 1;   // find the first n2 in [0, n2max + 1) with kf sqrt(n2) >= edges[b]
    while (a < z) {
        const int m = (a + z) >> 1;
        if (kf * sqrt((double)m) >= edges[b]) z = m; else a = m + 1;
    }
    lo[b] = a;
}

__global__ void k_finish(const double* __restrict__ acc, int nbins, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    unsigned long long cnt;
    memcpy(&cnt, &acc[2 * nbins + b], sizeof(cnt));
    out[b] = cnt ? acc[b] / (double)cnt : NAN;
    out[nbins + b] = cnt ? acc[nbins + b] / (double)cnt : NAN;
    const long long n = (long long)cnt;
    memcpy(&out[2 * nbins + b], &n, sizeof(n));
}

std::mutex g_mu;
unsigned char* g_dev_ptr[64] = {};

// Device memory of the current device `dev` (memory of another GPU is rejected: without peer
// access the kernels could not read it), or managed memory.
bool device_resident(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace colapm

using namespace colapm;

extern "C" int colapm_power_noalloc(const int* cell, const float* offset, long long n_particles, int nm, double box,
                                    int nbins, double kmin, double kmax, double* k_out, double* p_out,
                                    long long* nmodes_out, void* stream) {
    static const int sizes[] = {16, 32, 64, 96, 128};
    bool ok_nm = false;
    for (int s : sizes) ok_nm |= (s == nm);
    if (!ok_nm || nm > kMaxNm || nbins < 1 || nbins > kMaxBins || n_particles < 1 || !(box > 0)) return COLAPM_E_ARG;
    if (!cell || !offset || !k_out || !p_out || !nmodes_out) return COLAPM_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return COLAPM_E_CUDA;
    if (!device_resident(cell, dev) || !device_resident(offset, dev)) return COLAPM_E_ARG;
    const double kf = 2.0 * M_PI / box;
    if (kmin <= 0) kmin = kf;
    if (kmax <= 0) kmax = M_PI * nm / box;
    if (!(kmax > kmin)) return COLAPM_E_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return COLAPM_E_CUDA;
            g_dev_ptr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_dev_ptr[dev];
    }
    auto* rho = reinterpret_cast<unsigned long long*>(base + kRho);
    auto* spec = reinterpret_cast<float2*>(base + kSpec);
    auto* tw = reinterpret_cast<float2*>(base + kTw);
    auto* sinc2 = reinterpret_cast<float*>(base + kSinc);
    auto* edges = reinterpret_cast<double*>(base + kEdges);
    auto* bin = reinterpret_cast<int*>(base + kBin);
    auto* acc = reinterpret_cast<double*>(base + kAcc);
    auto* out = reinterpret_cast<double*>(base + kOut);
    auto* err = reinterpret_cast<int*>(base + kErr);

    // Host tables on the stack (copied before this call returns; the call synchronises).
    float2 h_tw[kMaxNm];
    float h_s2[kMaxNm];
    double h_edges[kMaxBins + 1];
    for (int i = 0; i < nm; ++i) {
        const double ang = 2.0 * M_PI * (double)i / nm;
        h_tw[i] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        const int sg = i < nm / 2 ? i : i - nm;
        const double x = M_PI * sg / nm;
        const double v = sg == 0 ? 1.0 : std::sin(x) / x;
        h_s2[i] = (float)(v * v);
    }
    for (int b = 0; b <= nbins; ++b) h_edges[b] = kmin * std::pow(kmax / kmin, (double)b / nbins);
    const int n2max = 3 * (nm / 2) * (nm / 2);
    const size_t nm3 = (size_t)nm * nm * nm;

    // Once work is queued, an error return first waits (best effort) for what was queued, so that no
    // kernel of this call still writes the shared array when the caller retries, even on another stream.
#define NCK(x)                                  \
    do {                                        \
        if ((x) != cudaSuccess) {               \
            cudaStreamSynchronize(s);           \
            return COLAPM_E_CUDA;               \
        }                                       \
    } while (0)
    NCK(cudaMemcpyAsync(tw, h_tw, sizeof(float2) * nm, cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(sinc2, h_s2, sizeof(float) * nm, cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(edges, h_edges, sizeof(double) * (nbins + 1), cudaMemcpyHostToDevice, s));
    NCK(cudaMemsetAsync(rho, 0, sizeof(unsigned long long) * nm3, s));
    NCK(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * nbins, s));
    NCK(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));
    k_bin_thresholds<<<(nbins + 128) / 128, 128, 0, s>>>(edges, nbins, kf, n2max, bin);
    NCK(cudaGetLastError());
    k_deposit_xyz<<<(unsigned)((n_particles + 255) / 256), 256, 0, s>>>(cell, offset, n_particles, nm, rho, err);
    NCK(cudaGetLastError());
    const double ratio = (double)nm3 / (double)n_particles;   // cells per particle
    NCK(launch_fx_fwd_i64(nm, rho, spec, tw, (float)(ratio * std::ldexp(1.0, -45)), err, s));
    NCK(launch_fy(nm, -1, spec, 0, 1, tw, s));
    PowerArgs pw{};
    pw.n2_lo = bin;
    pw.kf = (float)kf;
    pw.ksum = acc;
    pw.psum = acc + nbins;
    pw.cnt = reinterpret_cast<unsigned long long*>(acc + 2 * nbins);
    pw.nbins = nbins;
    pw.pnorm = (float)(box * box * box / ((double)nm3 * (double)nm3));
    pw.lga = (float)(0.5 * nbins / std::log2(h_edges[nbins] / h_edges[0]));
    pw.lgb = (float)(nbins * std::log2(kf / h_edges[0]) / std::log2(h_edges[nbins] / h_edges[0]));
    NCK(launch_fz(nm, Z_POWER, spec, ZOut{}, tw, sinc2, 0, 1.0f, &pw, s));
    k_finish<<<(nbins + 127) / 128, 128, 0, s>>>(acc, nbins, out);
    NCK(cudaGetLastError());
    int h_err = 0;
    NCK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NCK(cudaMemcpyAsync(k_out, out, sizeof(double) * nbins, cudaMemcpyDefault, s));
    NCK(cudaMemcpyAsync(p_out, out + nbins, sizeof(double) * nbins, cudaMemcpyDefault, s));
    NCK(cudaMemcpyAsync(nmodes_out, out + 2 * nbins, sizeof(long long) * nbins, cudaMemcpyDefault, s));
    NCK(cudaStreamSynchronize(s));
#undef NCK
    if (h_err & 2) return COLAPM_E_ARG;
    if (h_err & 1) return COLAPM_E_OVERFLOW;
    return COLAPM_OK;
}
