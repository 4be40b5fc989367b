// Internal declarations shared by the translation units of libcolapm.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/colapm.h"

namespace colapm {

// Coefficients of one Kick-Drift step in mesh units (cells), converted from the FP64 table.
struct StepCoef {
    float kick;    // 1.5 Om times the kick integral (Quinn or modified, §2.3)
    float c1;      // D1(a_i)            (COLA bracket; 0 for plain PM)
    float c2;      // D2(a_i) - D1(a_i)^2 (COLA bracket; 0 for plain PM)
    float drift;   // drift integral (§2.3)
    float e1;      // D1(a_{i+1}) - D1(a_i) (COLA drift; 0 for plain PM)
    float e2;      // D2(a_{i+1}) - D2(a_i)
};

// Output pointers of a z pass (up to 9 spectra: 3 x Psi1 and 6 x phi_ij of the ICs).
struct ZOut {
    float2* p[9];
};

enum ZMode {
    Z_FORCE = 0,   // forward z, F_j = i k_j delta / (k^2 W^d) / N^3, inverse z, 3 outputs
    Z_LPT1 = 1,    // (input already transformed) Psi1_j = i k_j d/k^2, phi_ab = k_a k_b d/k^2, 9 outputs
    Z_LPT2 = 2,    // forward z, Psi2_j = -i k_j S/k^2, 3 outputs
    Z_POWER = 3,   // forward z, bin |delta|^2 / W^2
    // (Stockham engine only) per-mode scaling by a table indexed by |n|^2, passed in place of sinc2:
    Z_SCALE_FWD = 4,   // forward z, then multiply: 1 output in k-space
    Z_SCALE_INV = 5    // (input already transformed) multiply, then inverse z: 1 output
};

// Power-spectrum binning. Bin membership is decided in FP64 on the host (or once per call on
// the device) and handed to the kernel as integer thresholds on |n|^2: a mode is in bin b when
// n2_lo[b] <= |n|^2 < n2_lo[b + 1] (empty bins have equal thresholds); |n|^2 < n2_lo[0] or
// >= n2_lo[nbins] is outside. Per-mode values are FP32, sums FP64.
struct PowerArgs {
    const int* n2_lo;           // [nbins + 1]
    double* ksum;               // [nbins]
    double* psum;               // [nbins]
    unsigned long long* cnt;    // [nbins]
    int nbins;
    float kf;                   // 2 pi / L (h/Mpc)
    float pnorm;                // L^3 / N^6
    // first guess of the bin of |n|^2 for log-spaced bins, floor(lga log2 |n|^2 + lgb), corrected
    // against n2_lo (lga = 0: binary search only)
    float lga, lgb;
};

// Guess from the log-spacing of the bins (at most one or two off near an edge), then a walk to
// the bin whose thresholds hold |n|^2; -1 outside. The same bin as the binary search.
__device__ __forceinline__ int power_bin_guess(int n2, const int* lo, const PowerArgs& pw) {
    const int nb = pw.nbins;
    if (n2 < lo[0] || n2 >= lo[nb]) return -1;
    int b = (int)floorf(fmaf(pw.lga, __log2f((float)n2), pw.lgb));
    b = b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
    while (b > 0 && n2 < lo[b]) --b;
    while (b < nb - 1 && n2 >= lo[b + 1]) ++b;
    return b;
}

// Bin of |n|^2 given the thresholds (binary search; -1 outside).
__device__ __forceinline__ int power_bin(int n2, const int* lo, int nbins) {
    if (n2 < lo[0] || n2 >= lo[nbins]) return -1;
    int a = 0, b = nbins;
    while (b - a > 1) {
        const int m = (a + b) >> 1;
        if (lo[m] <= n2) a = m; else b = m;
    }
    return a;
}

// Bins the modes (nx, ny, nz(z)) of one column for z = z0 ... z0 + per - 1 (ny not on the Nyquist
// plane; z = L/2 skipped) into the FP64 bins: FP32 sums over runs of consecutive modes in one bin
// (a few dozen at most), added to the bin when the run leaves it. The current bin's |n|^2 range
// stays in registers, so a mode of the same bin costs two compares; a new bin comes from the
// log-spacing guess (power_bin_guess) or the binary search. value(z) gives the mode's complex
// amplitude, sinc2[z] the CIC window factor along z (wxy the product of the x and y factors).
template <typename F>
__device__ __forceinline__ void bin_column_run(int nx, int ny, int z0, int per, int L, float wxy,
                                               const float* __restrict__ sinc2, const int* lo, const PowerArgs& pw,
                                               double* psum, double* ksum, unsigned long long* cnt, F value) {
    const float mult = nx == 0 ? 1.0f : 2.0f;
    const float cp = mult * pw.pnorm, ck = mult * pw.kf;
    const unsigned ci = nx == 0 ? 1u : 2u;
    const int nxy2 = nx * nx + ny * ny;
    int rb = -1, blo = 0, bhi = 0;
    float rp = 0.0f, rk = 0.0f;
    unsigned rc = 0;
    for (int zz = 0; zz < per; ++zz) {
        const int z = z0 + zz;
        if (z == L / 2) continue;
        const int nz = z < L / 2 ? z : z - L;
        const int n2 = nxy2 + nz * nz;
        if (n2 < blo || n2 >= bhi) {   // the run leaves its bin
            if (rb >= 0) {
                atomicAdd(&psum[rb], (double)rp);
                atomicAdd(&ksum[rb], (double)rk);
                atomicAdd(&cnt[rb], (unsigned long long)rc);
            }
            rp = 0.0f;
            rk = 0.0f;
            rc = 0;
            rb = n2 == 0 ? -1 : (pw.lga != 0.0f ? power_bin_guess(n2, lo, pw) : power_bin(n2, lo, pw.nbins));
            blo = rb >= 0 ? lo[rb] : n2;        // outside every bin: a range of this |n|^2 alone
            bhi = rb >= 0 ? lo[rb + 1] : n2 + 1;
        }
        if (rb < 0) continue;
        const float2 v = value(z);
        const float w = wxy * sinc2[z];
        rp += __fdividef(cp * (v.x * v.x + v.y * v.y), w * w);
        rk += ck * sqrtf((float)n2);
        rc += ci;
    }
    if (rb >= 0) {
        atomicAdd(&psum[rb], (double)rp);
        atomicAdd(&ksum[rb], (double)rk);
        atomicAdd(&cnt[rb], (unsigned long long)rc);
    }
}

// --- launchers (fft_kernels_*.cu) ----------------------------------------------------------
// Forward x pass (r2c) of N^2 rows of N reals into N^2 rows of N/2 complex (Nyquist dropped).
// in_i64: int64 fixed-point density converted to delta = rho * scale - 1 (flags err[0] bit 0
// when a cell has its top bit set); in_f32: real field.
// `two_stage` selects the two-stage register FFT where it exists (256, 512, 1024 lines); the
// shared-memory Stockham kernels otherwise.
// zero_input: clear the int64 mesh as it is read, so that the next deposit needs no memset.
// blocked: write the half spectrum in the blocked layout [kx/8][z][y][kx%8] (two-stage engine only).
cudaError_t launch_fx_fwd_i64(int n_mesh, const unsigned long long* in, float2* out, const float2* tw,
                              float scale, int* err, cudaStream_t s, bool two_stage = true, bool zero_input = false,
                              bool blocked = false);
cudaError_t launch_fx_fwd_f32(int n_mesh, const float* in, float2* out, const float2* tw, cudaStream_t s,
                              bool two_stage = true);
// Inverse x pass (c2r), in place, for `nfields` arrays spaced `field_stride` complex apart.
cudaError_t launch_fx_inv(int n_mesh, float2* data, size_t field_stride, int nfields, const float2* tw,
                          cudaStream_t s, bool two_stage = true, bool blocked = false, float2* dst = nullptr);
// y pass in place (sign -1 forward, +1 inverse) on `nfields` arrays.
cudaError_t launch_fy(int n_mesh, int sign, float2* data, size_t field_stride, int nfields, const float2* tw,
                      cudaStream_t s, bool two_stage = true, bool blocked = false);
// Inverse y pass of the force in the blocked layout (N = 512, 1024): from the z pass's two bases in
// fields 0 and 2 to the three force spectra in fields 0, 1, 2 (the blocked force z pass writes
// the bases instead of the three spectra).
cudaError_t launch_fy_force(int n_mesh, float2* data, size_t field_stride, const float2* tw, cudaStream_t s);
// z pass with the spectral multiply fused.
// Fused x-y passes (N = 512, 1024): forward r2c x + y of the int64 density into the half
// spectrum `out`; inverse y + c2r x of `nfields` spectra in place. `ring` holds xy_ring_bytes(N)
// and `ctr` xy_ctr_ints(N, nfields) ints (the launch zeroes them); err bit 4 = a bounded wait gave up.
bool xy_supported(int nm);
size_t xy_ring_bytes(int nm);
size_t xy_ctr_ints(int nm, int nfields);
cudaError_t launch_xy_fwd(int nm, const unsigned long long* rho, float2* out, const float2* tw, float scale,
                          float2* ring, int* ctr, int* err, cudaStream_t s, bool zero_input = false);
cudaError_t launch_xy_inv(int nm, float2* data, size_t fstride, int nfields, const float2* tw, float2* ring, int* ctr,
                          int* err, cudaStream_t s);

cudaError_t launch_fz(int n_mesh, int mode, float2* in, ZOut out, const float2* tw, const float* sinc2,
                      int deconv, float gnorm, const PowerArgs* pw, cudaStream_t s, bool two_stage = true, bool blocked = false);

// What the drift of one step needs to record the particle images that leave the past lightcone
// during it (§6). Rows are two float4: (x, y, z, a_L) and (px, py, pz, id bits), Mpc/h.
struct LightconeStep {
    float4* out;
    unsigned long long* count;
    unsigned long long capacity;
    const float* tab;        // K samples over [a_i, a_{i+1}], 5 floats each: S, D1 - D1(a_i), D2 - D2(a_i), P1, P2
    const int* reps;         // 3 * nrep replicate vectors
    const int* id;           // particle id of each slot (null: slot order is id order)
    int nrep, K, pad0, pad1;
    float ox, oy, oz;        // observer, Mpc/h
    float cell, box;         // cell size and box side, Mpc/h
    float a0, da, rl0, rl1;  // step start and width; lightcone radius at both ends, Mpc/h
};

// One mock of a multi-mock particle launch: its particle arrays, force meshes (gather), density
// (deposit), sizes, step coefficients, and the index of its first work item (chunks of particles,
// numbered mock after mock; multi_items gives a mock's count).
struct MockWork {
    float4* pos;
    float* mom;
    const float* psi1;
    const float* psi2;
    const float* force;
    unsigned long long* rho;
    size_t np3;
    long long first;
    int nm;
    StepCoef k;
};

// --- launchers (pm_kernels.cu) --------------------------------------------------------------
long long multi_items(size_t np3);
// Deposit / gather-kick-drift of every mock in w[0..nmock) in one persistent launch; `queue` is two
// zero-initialised u64 counters per kernel that the launch leaves at zero.
cudaError_t launch_multi_deposit(const MockWork* w, int nmock, long long nitems, unsigned long long* queue,
                                 cudaStream_t s);
cudaError_t launch_multi_gather_kick_drift(const MockWork* w, int nmock, long long nitems, unsigned long long* queue,
                                           cudaStream_t s);
cudaError_t launch_deposit(const float4* pos, size_t np3, int nm, unsigned long long* rho, cudaStream_t s,
                           int block = 256);
cudaError_t launch_gather_kick_drift(float4* pos, float* mom, const float* psi1, const float* psi2,
                                     const float* force, size_t np3, int nm, StepCoef c, int drift,
                                     cudaStream_t s, int block = 256, const LightconeStep* lc = nullptr);
cudaError_t launch_init_particles(float4* pos, float* mom, float* psi1, float* psi2, int np, int nm,
                                  float to_mesh, float d1, float d2, float p1, float p2, int cola,
                                  cudaStream_t s);
cudaError_t launch_add_lpt_momentum(float* mom, const float* psi1, const float* psi2, size_t np3, float p1,
                                    float p2, cudaStream_t s);
// Writes particle p's values at its id (id may be NULL: slot order is id order).
cudaError_t launch_export_particles(const float4* pos, const float* mom, const int* id, size_t np3, int nm, float cell,
                                    float* pos_xyz, float* mom_xyz, cudaStream_t s);
cudaError_t launch_export_state(const float4* pos, const float* mom, size_t np3, int nm, int* cell_xyz,
                                float* off_xyz, float* mom_xyz, cudaStream_t s);
cudaError_t launch_import_state(float4* pos, float* mom, size_t np3, int nm, const int* cell_xyz,
                                const float* off_xyz, const float* mom_xyz, int* err, cudaStream_t s);
cudaError_t launch_export_displacement(const float4* pos, int np, int nm, float cell, float* psi, cudaStream_t s);
cudaError_t launch_import_displacement(float4* pos, int np, int nm, float to_mesh, const float* psi, int* err,
                                       cudaStream_t s);
cudaError_t launch_scale(float* dst, const float* src, size_t n, float f, cudaStream_t s);
// Redshift-space positions (cell bits + offsets) of the particles; scale = 1 / (a^2 E(a)).
cudaError_t launch_rsd_positions(const float4* pos, const float* mom, size_t np3, int nm, float scale, int los,
                                 float4* out, cudaStream_t s);

// --- launchers (sort_kernels.cu) ------------------------------------------------------------
// Particle arrays in and out of a reordering, and the bucket counters of the sort.
struct SortBuffers {
    const float4* pos;
    const float* mom;
    const float* psi1;
    const float* psi2;
    const int* id;
    float4* pos_o;
    float* mom_o;
    float* psi1_o;
    float* psi2_o;
    int* id_o;
    unsigned* cnt;        // sort_buckets(nm): counts, then cursors
    unsigned* tile_sum;   // sort_tiles(nm)
    int* err;             // error bits; 8: a scatter slot out of range (an internal inconsistency)
};
int sort_xshift(int nm);
size_t sort_buckets(int nm);
size_t sort_tiles(int nm);
// Counting sort of the particles by bucket (z, y, x >> sort_xshift) of their cell into the _o arrays.
// Tiles of 64 x 2^tshift x 2^tshift cells (tshift 0 ... 3, nm a multiple of 2^tshift); after the
// sort, cnt[b] is the end of bucket b in the new order (tile t = buckets t 4^tshift ... + 4^tshift - 1).
bool sort_tshift_ok(int nm, int tshift);
cudaError_t launch_sort(SortBuffers b, size_t np3, int nm, int tshift, cudaStream_t s);
// Deposit of particles ordered by tile (the last sort with this tshift; bucket ends in `ends`): each
// tile plus its +1 halo accumulated in shared memory, then added to rho; corners outside go straight
// to rho.
cudaError_t launch_deposit_tiles(const float4* pos, int nm, int tshift, const unsigned* ends, unsigned long long* rho,
                                 cudaStream_t s);
// The _o arrays receive the particles in particle-id order (slot id[p] <- slot p), id_o the identity.
cudaError_t launch_unsort(SortBuffers b, size_t np3, cudaStream_t s);
cudaError_t launch_iota(int* id, size_t n, cudaStream_t s);

// --- launchers (ics_kernels.cu) -----------------------------------------------------------
// The seed is read from device memory, so a captured graph can be replayed with new seeds.
cudaError_t launch_gaussian_field(int np, const unsigned long long* seed, const float* amp_of_n2, float2* dk,
                                  cudaStream_t s);
cudaError_t launch_lpt2_source(const float* phi, size_t np3, float* src, cudaStream_t s);
cudaError_t launch_set_u64(unsigned long long* dst, unsigned long long value, cudaStream_t s);
// Local primordial non-Gaussianity on a real field of n values in place: Phi = phi + fnl (phi^2 - <phi^2>),
// <> the mean over the field (FP64 sum into `sum2`, one double of scratch).
cudaError_t launch_local_fnl(float* phi, size_t n, double fnl, double* sum2, cudaStream_t s);

}  // namespace colapm
