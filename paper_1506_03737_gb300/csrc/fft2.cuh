// Two-stage register FFT for the mesh lengths with a two-radix plan (L = 64 ... 1024).
//
// A line of length L = RA * RB (radices 8 to 32) is transformed in two Stockham stages. In
// stage A (stride 1) task j < L/RA takes inputs j + r L/RA (r < RA) straight from global memory
// (or from the caller), applies the RA-point DFT in registers and writes output r to position
// j RA + r of a shared exchange buffer. In stage B (stride RA) task j < RA reads positions
// j + r RA (r < RB), multiplies input r by w^(j r), w = exp(sign 2 pi i / L), applies the RB-point
// DFT and holds output r = X[j + RA r] in registers, which the caller writes out. A line thus
// crosses shared memory once (one 8-byte write and one read per element); the exchange buffer
// pads every RA elements by one and every line to a pitch = 4 (mod 16) elements, so that the
// two access patterns use the minimum number of bank wavefronts for both thread mappings used
// (8 lines x 4 tasks per warp, or 32 tasks of one line per warp).
//
// Because the stage-B output of task j (X[j + RA r], r < RB) is exactly the stage-A input set
// of task j of a transform with the radices swapped (RB, RA), an inverse transform can follow a
// forward one on the same registers (the z pass chains forward, multiply, inverse).
//
// Twiddles w^(j r) come from two small shared tables, w^j (j < 32) and w^(8 m j) (m < 4, j < 32):
// w^(j r) = w^(8 floor(r/8) j) * (w^j)^(r mod 8), at most 7 multiplications from a table value.
#pragma once

#include "fft_engine.cuh"

namespace colapm {

template <int L>
struct F2;
template <> struct F2<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct F2<96> { static constexpr int R1 = 8, R2 = 12; };
template <> struct F2<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct F2<160> { static constexpr int R1 = 16, R2 = 10; };
template <> struct F2<192> { static constexpr int R1 = 16, R2 = 12; };
template <> struct F2<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct F2<320> { static constexpr int R1 = 16, R2 = 20; };
template <> struct F2<384> { static constexpr int R1 = 16, R2 = 24; };
template <> struct F2<512> { static constexpr int R1 = 16, R2 = 32; };
template <> struct F2<1024> { static constexpr int R1 = 32, R2 = 32; };

// Lengths with a two-stage plan. The mixed ones (96, 160, 192, 320, 384) take a composite second
// radix (10, 12, 20, 24), itself split into coprime factors in registers (prime-factor algorithm).
template <int L>
struct F2Has {
    static constexpr bool value = L == 64 || L == 96 || L == 128 || L == 160 || L == 192 || L == 256 || L == 320 ||
                                  L == 384 || L == 512 || L == 1024;
};

// Exchange buffer of LINES lines (8 by default) for a stage-A radix RA.
template <int L, int RA, int LINES = 8>
struct Xch {
    static constexpr int BASE = L + L / RA;
    static constexpr int PITCH = BASE + (((4 - BASE % 16) % 16) + 16) % 16;   // = 4 (mod 16)
    static constexpr int SIZE = LINES * PITCH;     // float2 elements
    __host__ __device__ __forceinline__ static int at(int c, int e) { return c * PITCH + e + e / RA; }
};

// Twiddle tables for length L: w1[j] = w^j, w8[m][j] = w^(8 m j), w = exp(-2 pi i / L).
struct Tw2 {
    float2 w1[32];
    float2 w8[4][32];
};
template <int L, int TWN>
__device__ __forceinline__ void load_tw2(Tw2* t, const float2* __restrict__ g, int T) {
    for (int e = threadIdx.x; e < 32 * 5; e += T) {
        const int m = e / 32, j = e % 32;
        const int idx = m == 0 ? j : ((8 * (m - 1) * j) % L);
        const float2 v = g[idx * (TWN / L)];
        if (m == 0) t->w1[j] = v; else t->w8[m - 1][j] = v;
    }
}

// Multiply v[r] by w^(S j r) for r < R (j < 32).
template <int R, int S>
__host__ __device__ __forceinline__ void twiddle2(float2* v, const Tw2* t, int j) {
    float2 p[8];
    float2 w1 = t->w1[j];
    if (S > 0) w1 = cconj(w1);
    p[0] = make_float2(1.0f, 0.0f);
#pragma unroll
    for (int k = 1; k < 8; ++k) p[k] = cmul(p[k - 1], w1);
#pragma unroll
    for (int r = 1; r < R; ++r) {
        float2 w = p[r & 7];
        if (r >= 8) {
            float2 b = t->w8[r >> 3][j];
            if (S > 0) b = cconj(b);
            w = (r & 7) ? cmul(b, w) : b;
        }
        v[r] = cmul(v[r], w);
    }
}

}  // namespace colapm

#include "colapm_internal.h"

namespace colapm {

template <int L>
struct K2 {   // threads: the larger task count of the two stages (8 lines)
    static constexpr int RA = F2<L>::R1, RB = F2<L>::R2;
    static constexpr int TA = 8 * L / RA, TB = 8 * L / RB;
    static constexpr int T = TA > TB ? TA : TB;
};

__device__ __forceinline__ int sbin(int i, int L) { return i < L / 2 ? i : i - L; }

// Half-spectrum layouts (n = L/2 complex columns kx, rows y, planes z): standard [z][y][kx], or
// blocked [kx/8][y/8][z][y%8][kx%8]. In the blocked layout every tile the passes read is made of
// 512-byte runs: an x-pass tile of 8 rows is one run per 8-column block, a y-pass tile takes one
// run per group of 8 rows, and the rows of a z-pass tile are 512 bytes apart (64 bytes each; the
// 8 tiles of one row group, taken one after the other, complete every run). In the standard layout
// the rows of a z tile are 4 MB apart, every one in a different 2 MB page, which streams at about a
// third of the bandwidth.
template <int L, bool BLK>
__host__ __device__ __forceinline__ size_t hs_index(int kx, int y, int z) {
    if constexpr (BLK)
        return ((((((size_t)(kx >> 3) * (L / 8) + (y >> 3)) * L + z) << 3) + (y & 7)) << 3) + (kx & 7);
    else return ((size_t)z * L + y) * (L / 2) + kx;
}

// Distance between rows y and y + d of one column when d and y are multiples of 8 apart from the
// same residue (d a multiple of 8): what the passes add per register index.
template <int L, bool BLK>
__host__ __device__ __forceinline__ constexpr size_t hs_ystep(int d) {
    return BLK ? (size_t)(d / 8) * L * 64 : (size_t)d * (L / 2);
}

// Stage B of a line held in exchange buffer xb (stage-A radix RA), task j < RA of line c:
// loads j + RA r, twiddles, RB-point DFT. Returns X[j + RA r] in v.
template <int L, int RA, int RB, int S, int LINES = 8>
__host__ __device__ __forceinline__ void stage_b(const float2* xb, const Tw2* tw, int c, int j, float2* v) {
#pragma unroll
    for (int r = 0; r < RB; ++r) v[r] = xb[Xch<L, RA, LINES>::at(c, j + RA * r)];
    twiddle2<RB, S>(v, tw, j);
    dft<RB, S>(v);
}

// ---------------------------------------------------------------------------------------------
// y pass (strided columns, stride n = L/2 complex), persistent over tiles of 8 columns.
template <int L, int S, bool BLK = false>
__global__ void __launch_bounds__(K2<L>::T) k2_fy(float2* __restrict__ data, size_t fstride,
                                                   const float2* __restrict__ tw, int nfields) {
    using K = K2<L>;
    constexpr int RA = K::RA, RB = K::RB, n = L / 2, NG = n / 8, TPF = NG * L;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* tws = reinterpret_cast<Tw2*>(xb + Xch<L, RA>::SIZE);
    load_tw2<L, L>(tws, tw, K::T);
    __syncthreads();
    const int total = TPF * nfields;
    const int tid = threadIdx.x, c = tid & 7, j = tid >> 3;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int f = t / TPF, r0 = t % TPF;
        // rows y = j + r L/RA (stage A) and j + RA r (stage B); L/RA and RA are multiples of 8
        float2* g = data + (size_t)f * fstride + hs_index<L, BLK>((r0 % NG) * 8 + c, j, r0 / NG);
        if (tid < K::TA) {
            float2 v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = __ldcg(g + r * hs_ystep<L, BLK>(L / RA));
            dft<RA, S>(v);
#pragma unroll
            for (int r = 0; r < RA; ++r) xb[Xch<L, RA>::at(c, j * RA + r)] = v[r];
        }
        __syncthreads();
        if (tid < K::TB) {
            float2 v[RB];
            stage_b<L, RA, RB, S>(xb, tws, c, j, v);
#pragma unroll
            for (int r = 0; r < RB; ++r) g[r * hs_ystep<L, BLK>(RA)] = v[r];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// z pass with the spectral operator fused (see k_fz in fft_kernels.cuh for the algebra):
// forward z (radices R1, R2) -> bases in registers -> inverse z (radices R2, R1) per base.
// C columns per tile: 8, or 4 (the blocked layout) to halve the shared memory per CTA.
template <int L, int MODE, int C = 8, bool DIRECT = false>
struct Z2 {
    static constexpr int R1 = F2<L>::R1, R2 = F2<L>::R2;
    static constexpr int XS = Xch<L, R1, C>::SIZE > Xch<L, R2, C>::SIZE ? Xch<L, R1, C>::SIZE : Xch<L, R2, C>::SIZE;
    static constexpr int NSAVE = MODE == Z_LPT1 ? 2 : (MODE == Z_POWER ? 0 : 1);   // saved bases B (, C)
    // next tile via cp.async into a shared buffer, or (DIRECT) straight from global memory into the
    // stage-A registers: the smaller footprint fits three CTAs per SM at C = 4, which hides the load
    // latency better than the prefetch does with two (force z pass at 1024^3: 6.0 against 6.9 ms)
    static constexpr bool PREFETCH = MODE != Z_LPT1 && !DIRECT;
    static constexpr int MINB = DIRECT && C == 4 ? 3 : 1;                         // CTAs per SM
    static constexpr int PF = PREFETCH ? C * L : 0;                               // dense [z][C] buffer
    static constexpr int TA = C * L / R1, TB = C * L / R2, T = TA > TB ? TA : TB;
    static constexpr size_t SMEM = sizeof(float2) * ((size_t)XS * (1 + NSAVE) + PF) + sizeof(Tw2);
};

template <int L, int MODE, int C = 8, bool BLK = false, bool DIRECT = false>
__global__ void __launch_bounds__(Z2<L, MODE, C, DIRECT>::T, Z2<L, MODE, C, DIRECT>::MINB)
    k2_fz(float2* __restrict__ in, ZOut out, const float2* __restrict__ tw, const float* __restrict__ sinc2, int deconv,
          float gnorm, PowerArgs pw) {
    using Z = Z2<L, MODE, C, DIRECT>;
    constexpr int R1 = Z::R1, R2 = Z::R2, n = L / 2, NG = n / C, NTILE = NG * L;
    constexpr int T = Z::T;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    float2* save = xb + Z::XS;                                   // bases B (, C), layout Xch<L,R1>
    float2* pf = xb + Z::XS * (1 + Z::NSAVE);                    // prefetched input tile [z][8]
    Tw2* tws = reinterpret_cast<Tw2*>(pf + Z::PF);
    double* ksum = reinterpret_cast<double*>(tws + 1);
    double* psum = ksum + pw.nbins;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(psum + pw.nbins);
    int* lo = reinterpret_cast<int*>(cnt + pw.nbins);
    load_tw2<L, L>(tws, tw, T);
    if constexpr (MODE == Z_POWER) {
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            ksum[b] = 0.0;
            psum[b] = 0.0;
            cnt[b] = 0ull;
        }
        for (int b = threadIdx.x; b <= pw.nbins; b += T) lo[b] = pw.n2_lo[b];
    }
    __syncthreads();
    const float kf = 6.283185307179586f / (float)L;
    constexpr size_t stride = BLK ? (size_t)64 : (size_t)L * n;   // distance between planes z
    // tile -> (ky, kx0); in the blocked layout the 8 ky of a row group, then the 8 / C column
    // sub-tiles of an 8-column block, are consecutive tiles (together they cover 512-byte runs)
    auto tile_of = [&](int tt, int& ky_, int& kx0_) {
        if constexpr (BLK) {
            constexpr int SUB = 8 / C;
            const int q = tt >> 3;
            ky_ = 8 * (q / (SUB * (n / 8))) + (tt & 7);
            kx0_ = ((q / SUB) % (n / 8)) * 8 + (q % SUB) * C;
        } else {
            ky_ = tt / NG;
            kx0_ = (tt % NG) * C;
        }
    };
    static_assert(!BLK || C == 8 || C == 4, "blocked layout needs 8- or 4-column tiles");
    const int tid = threadIdx.x, c = tid % C, j = tid / C;
    constexpr int TA = Z::TA, TB = Z::TB;   // forward stage-A / stage-B tasks
    auto prefetch = [&](int tt) {   // 16-byte cp.async.cg of rows z = 0..L-1, C columns, into pf
        int pky, pkx0;
        tile_of(tt, pky, pkx0);
        const size_t b = hs_index<L, BLK>(pkx0, pky, 0);
        constexpr int Q = C / 2;    // 16-byte pieces per row
        for (int e = tid; e < L * Q; e += T) {
            const int z = e / Q, q = e % Q;
            cp_async16_cg(pf + z * C + 2 * q, in + b + (size_t)z * stride + 2 * q);
        }
        cp_async_commit();
    };
    if constexpr (Z::PREFETCH) {
        if (blockIdx.x < NTILE) prefetch(blockIdx.x);
    }

    for (int t = blockIdx.x; t < NTILE; t += gridDim.x) {
        int ky, kx0;
        tile_of(t, ky, kx0);
        const int ny = sbin(ky, L);
        const bool nyq_y = (ky == L / 2);
        const size_t base = hs_index<L, BLK>(kx0 + c, ky, 0);
        const int nx = kx0 + c;
        float2 v[R2];   // stage-B results: X[j + R1 r] (j < R1), or the LPT1 input spectrum
        if constexpr (MODE == Z_LPT1) {
            if (tid < TB) {
#pragma unroll
                for (int r = 0; r < R2; ++r) v[r] = __ldcg(in + base + (size_t)(j + R1 * r) * stride);
            }
        } else {
            float2 a[R1];
            if constexpr (Z::PREFETCH) {
                cp_async_wait<0>();
                __syncthreads();
                if (tid < TA) {
#pragma unroll
                    for (int r = 0; r < R1; ++r) a[r] = pf[(j + r * (L / R1)) * C + c];
                }
                __syncthreads();   // prefetch buffer consumed
                if (t + (int)gridDim.x < NTILE) prefetch(t + gridDim.x);
            } else if (tid < TA) {
#pragma unroll
                for (int r = 0; r < R1; ++r) a[r] = __ldcg(in + base + (size_t)(j + r * (L / R1)) * stride);
            }
            if (tid < TA) {
                dft<R1, -1>(a);
#pragma unroll
                for (int r = 0; r < R1; ++r) xb[Xch<L, R1, C>::at(c, j * R1 + r)] = a[r];
            }
            __syncthreads();
            if (tid < TB) stage_b<L, R1, R2, -1, C>(xb, tws, c, j, v);
        }

        if constexpr (MODE == Z_POWER) {
            // Store the spectrum of the C columns in z order, then bin runs of consecutive z.
            if (tid < TB) {
#pragma unroll
                for (int r = 0; r < R2; ++r) xb[Xch<L, R1, C>::at(c, j + R1 * r)] = v[r];
            }
            __syncthreads();

            if (!nyq_y) {   // each thread a run of consecutive z of one column
                constexpr int PER = L * C / T;
                const int pc = tid % C;
                bin_column_run(kx0 + pc, ny, (tid / C) * PER, PER, L, sinc2[kx0 + pc] * sinc2[ky], sinc2, lo, pw, psum,
                               ksum, cnt, [&](int z) { return xb[Xch<L, R1, C>::at(pc, z)]; });
            }
            __syncthreads();
            continue;
        } else {
            // bases: A = g X, B = k_z A (, C = k_z^2 A); g = gnorm / (k^2 [W^d]), 0 on excluded modes
            if (tid < TB) {
                const int nxy2 = nx * nx + ny * ny;                                   // per column
                const float wxy = MODE == Z_FORCE && deconv ? sinc2[nx] * sinc2[ky] : 1.0f;
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const int z = j + R1 * r;
                    const int nz = sbin(z, L);
                    const int n2 = nxy2 + nz * nz;   // 0 only at k = 0
                    float w = 1.0f;
                    if (MODE == Z_FORCE && deconv) {
                        w = wxy * sinc2[z];
                        if (deconv == 2) w *= w;
                    }
                    // fast division (within 2 ulp; k^2 W is far from the range where it flushes)
                    const float g = !nyq_y && z != L / 2 && n2 != 0 ? __fdividef(gnorm, kf * kf * (float)n2 * w) : 0.0f;
                    v[r] = cscale(v[r], g);
                    const float kz = kf * (float)nz;
                    save[Xch<L, R1, C>::at(c, j + R1 * r)] = cscale(v[r], kz);
                    if constexpr (Z::NSAVE == 2) save[Z::XS + Xch<L, R1, C>::at(c, j + R1 * r)] = cscale(v[r], kz * kz);
                }
            }
            __syncthreads();   // forward exchange buffer free
            const float kyv = kf * (float)ny;
            const float kxv = kf * (float)nx;
            constexpr float sg = MODE == Z_LPT2 ? -1.0f : 1.0f;
            constexpr int NB = Z::NSAVE + 1;
#pragma unroll 1
            for (int bi = 0; bi < NB; ++bi) {
                // inverse stage A (radix R2) on base bi held by task j < R1
                if (tid < TB) {
                    if (bi > 0) {
#pragma unroll
                        for (int r = 0; r < R2; ++r) v[r] = save[(bi - 1) * Z::XS + Xch<L, R1, C>::at(c, j + R1 * r)];
                    }
                    dft<R2, +1>(v);
#pragma unroll
                    for (int r = 0; r < R2; ++r) xb[Xch<L, R2, C>::at(c, j * R2 + r)] = v[r];
                }
                __syncthreads();
                if (tid < TA) {   // inverse stage B (radix R1), task j < R2: outputs at j + R2 r
                    float2 u[R1];
                    stage_b<L, R2, R1, +1, C>(xb, tws, c, j, u);
#pragma unroll
                    for (int r = 0; r < R1; ++r) {
                        const size_t o = base + (size_t)(j + R2 * r) * stride;
                        const float2 a = u[r];
                        const float2 ia = make_float2(-a.y, a.x);   // i * a
                        if (MODE == Z_FORCE && BLK) {   // bases only; k2_fy_force applies i k_x, i k_y, i
                            out.p[bi == 0 ? 0 : 2][o] = a;
                        } else if (bi == 0) {
                            out.p[0][o] = cscale(ia, sg * kxv);
                            out.p[1][o] = cscale(ia, sg * kyv);
                            if constexpr (MODE == Z_LPT1) {
                                out.p[3][o] = cscale(a, kxv * kxv);
                                out.p[4][o] = cscale(a, kyv * kyv);
                                out.p[6][o] = cscale(a, kxv * kyv);
                            }
                        } else if (bi == 1) {
                            out.p[2][o] = cscale(ia, sg);
                            if constexpr (MODE == Z_LPT1) {
                                out.p[7][o] = cscale(a, kxv);
                                out.p[8][o] = cscale(a, kyv);
                            }
                        } else {
                            out.p[5][o] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    if constexpr (MODE == Z_POWER) {
        __syncthreads();
        for (int b = threadIdx.x; b < pw.nbins; b += T) {
            if (cnt[b]) {
                atomicAdd(&pw.psum[b], psum[b]);
                atomicAdd(&pw.ksum[b], ksum[b]);
                atomicAdd(&pw.cnt[b], cnt[b]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Inverse y pass of the force in the blocked layout. The z pass leaves the two inverse-z bases
// A' = IFFT_z(g X) in field 0 and B' = IFFT_z(k_z g X) in field 2 (k_x and k_y are constant along
// a z line, so the three force spectra are i k_x A', i k_y A' and i B'). Per 8-column tile this
// kernel makes the three y transforms from the two inputs:
//   F_z = i IFFT_y(B')         -> field 2 (in place)
//   F_y = i IFFT_y(k_y A')     -> field 1
//   F_x = i k_x IFFT_y(A')     -> field 0 (in place; A' is read twice, the second time from L2)
// It reads 8 bytes per cell instead of the 12 of three separate spectra.
template <int L>
__global__ void __launch_bounds__(K2<L>::T) k2_fy_force(float2* __restrict__ data, size_t fstride,
                                                        const float2* __restrict__ tw) {
    using K = K2<L>;
    constexpr int RA = K::RA, RB = K::RB, n = L / 2, NG = n / 8, TPF = NG * L;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* tws = reinterpret_cast<Tw2*>(xb + Xch<L, RA>::SIZE);
    load_tw2<L, L>(tws, tw, K::T);
    __syncthreads();
    const float kf = 6.283185307179586f / (float)L;
    const int tid = threadIdx.x, c = tid & 7, j = tid >> 3;
    for (int t = blockIdx.x; t < TPF; t += gridDim.x) {
        const int kx = (t % NG) * 8 + c;
        const size_t off = hs_index<L, true>(kx, j, t / NG);   // row j; other rows at hs_ystep offsets
        const float kxv = kf * (float)kx;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const float2* src = data + (pass == 0 ? 2 * fstride : 0) + off;
            float2* dst = data + (pass == 0 ? 2 : (pass == 1 ? 1 : 0)) * fstride + off;
            if (tid < K::TA) {
                float2 v[RA];
#pragma unroll
                for (int r = 0; r < RA; ++r) {
                    const int y = j + r * (L / RA);
                    v[r] = __ldcg(src + r * hs_ystep<L, true>(L / RA));
                    if (pass == 1) v[r] = cscale(v[r], kf * (float)sbin(y, L));
                }
                dft<RA, +1>(v);
#pragma unroll
                for (int r = 0; r < RA; ++r) xb[Xch<L, RA>::at(c, j * RA + r)] = v[r];
            }
            __syncthreads();
            if (tid < K::TB) {
                float2 u[RB];
                stage_b<L, RA, RB, +1>(xb, tws, c, j, u);
                const float sc = pass == 2 ? kxv : 1.0f;
#pragma unroll
                for (int r = 0; r < RB; ++r) dst[r * hs_ystep<L, true>(RA)] = make_float2(-sc * u[r].y, sc * u[r].x);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------------------------
// x passes on rows of n complex (the N = 2n real rows), 8 rows per tile.
template <int n>
struct X2 {
    static constexpr int RA = F2<n>::R1, RB = F2<n>::R2;
    static constexpr int TA = 8 * n / RA, TB = 8 * n / RB, T = TA > TB ? TA : TB;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)Xch<n, RA>::SIZE + sizeof(Tw2);
    // inverse: plus a dense [8][n] staging buffer for the cp.async prefetch of the rows
    static constexpr size_t SMEM_INV = SMEM + sizeof(float2) * 8 * (size_t)n;
};

// forward r2c: in = int64 density pairs (I64, converted to rho * scale - 1) or float reals.
// zero (optional): the int64 input itself, cleared as it is read (the next deposit then needs no memset).
template <int n, bool I64, bool BLK = false>
__global__ void __launch_bounds__(X2<n>::T) k2_fx_fwd(const void* __restrict__ in_, float2* __restrict__ out,
                                                       const float2* __restrict__ tw, float scale, int* err,
                                                       int nitems, unsigned long long* zero) {
    using X = X2<n>;
    constexpr int RA = X::RA, RB = X::RB, N = 2 * n;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* tws = reinterpret_cast<Tw2*>(xb + Xch<n, RA>::SIZE);
    load_tw2<n, N>(tws, tw, X::T);
    __syncthreads();
    const int tid = threadIdx.x;
    bool over = false;
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        const size_t row0 = (size_t)t * 8;
        if (tid < X::TA) {   // stage A: line c, task j (j fastest)
            const int c = tid / (n / RA), j = tid % (n / RA);
            float2 v[RA];
            if constexpr (I64) {
                // all loads first: the clearing stores go through another pointer to the same memory
                ulonglong2 q[RA];
#pragma unroll
                for (int r = 0; r < RA; ++r) q[r] = __ldcs(reinterpret_cast<const ulonglong2*>(in_) + (row0 + c) * n + j + r * (n / RA));
                if (zero) {
#pragma unroll
                    for (int r = 0; r < RA; ++r)
                        __stcs(reinterpret_cast<ulonglong2*>(zero) + (row0 + c) * n + j + r * (n / RA), make_ulonglong2(0ull, 0ull));
                }
#pragma unroll
                for (int r = 0; r < RA; ++r) {
                    over |= ((q[r].x | q[r].y) >> 63) != 0;
                    v[r] = make_float2(fmaf((float)(long long)q[r].x, scale, -1.0f),
                                       fmaf((float)(long long)q[r].y, scale, -1.0f));
                }
            } else {
#pragma unroll
                for (int r = 0; r < RA; ++r) v[r] = __ldcg(reinterpret_cast<const float2*>(in_) + (row0 + c) * n + j + r * (n / RA));
            }
            dft<RA, -1>(v);
#pragma unroll
            for (int r = 0; r < RA; ++r) xb[Xch<n, RA>::at(c, j * RA + r)] = v[r];
        }
        __syncthreads();
        // The half spectrum X[k] from Z[k] and Z[n-k]: inside stage B for n >= 512 (partner values by
        // warp shuffle; one barrier and one shared round trip fewer, measured 3.8 -> 3.4 ms at
        // n = 512), or in a separate loop over the exchange buffer (measured faster at n = 256).
        if constexpr (RB == 32) {
            if (tid < X::TB) {   // stage B: Z[j + RA r], then X[k] for the same k = j + RA r
                static_assert(RA == 16 || RA == 32, "the partner of a task must be in its warp");
                const int c = tid / RA, j = tid % RA;
                float2 v[RB];
                stage_b<n, RA, RB, -1>(xb, tws, c, j, v);
                // X[k] needs Z[n - k] too: for j > 0 that is element RB - 1 - r of task RA - j (same
                // line, same warp); for j = 0 it is this task's own element (RB - r) mod RB
                const int lane = threadIdx.x & 31;
                const int partner = (lane & ~(RA - 1)) | ((RA - j) & (RA - 1));
                const int y = (int)((row0 + c) % N), z = (int)((row0 + c) / N);
    #pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const float bx = __shfl_sync(0xffffffffu, v[RB - 1 - r].x, partner);
                    const float by = __shfl_sync(0xffffffffu, v[RB - 1 - r].y, partner);
                    const float2 a = v[r], b = j == 0 ? v[(RB - r) % RB] : make_float2(bx, by);
                    const int k = j + RA * r;
                    // X[k] from Z[k] = a, Z[n-k] = b; w^k = exp(-2 pi i k / N) = tw[k]
                    const float2 bc = cconj(b);
                    const float2 E = cscale(cadd(a, bc), 0.5f);
                    const float2 d = csub(a, bc);
                    out[hs_index<N, BLK>(k, y, z)] = cadd(E, cmul(tw[k], make_float2(0.5f * d.y, -0.5f * d.x)));
                }
            }
            __syncthreads();   // exchange buffer free for the next tile's stage A
        } else {
            if (tid < X::TB) {   // stage B in place: Z[j + RA r]
                const int c = tid / RA, j = tid % RA;
                float2 v[RB];
                stage_b<n, RA, RB, -1>(xb, tws, c, j, v);
    #pragma unroll
                for (int r = 0; r < RB; ++r) xb[Xch<n, RA>::at(c, j + RA * r)] = v[r];
            }
            __syncthreads();
            constexpr int H = n / 2 + 1;
            for (int e = tid; e < 8 * H; e += X::T) {
                const int c = e / H, k = e % H, k2 = (n - k) % n;
                const float2 a = xb[Xch<n, RA>::at(c, k)], b = xb[Xch<n, RA>::at(c, k2)];
                const int y = (int)((row0 + c) % N), z = (int)((row0 + c) / N);
                {   // X[k] from Z[k] = a, Z[n-k] = b; w^k = exp(-2 pi i k / N) = tw[k]
                    const float2 bc = cconj(b);
                    const float2 E = cscale(cadd(a, bc), 0.5f);
                    const float2 d = csub(a, bc);
                    out[hs_index<N, BLK>(k, y, z)] = cadd(E, cmul(tw[k], make_float2(0.5f * d.y, -0.5f * d.x)));
                }
                if (k != 0 && k2 != k) {
                    const float2 ac = cconj(a);
                    const float2 E = cscale(cadd(b, ac), 0.5f);
                    const float2 d = csub(b, ac);
                    out[hs_index<N, BLK>(k2, y, z)] = cadd(E, cmul(tw[k2], make_float2(0.5f * d.y, -0.5f * d.x)));
                }
            }
            __syncthreads();
        }
    }
    if constexpr (I64) {
        if (over) atomicOr(err, 1);
    }
}

// inverse c2r in place on `nfields` arrays; the next tile's rows are prefetched into a dense
// [8][n] staging buffer with 16-byte cp.async as soon as stage A has read the current one, so the
// copy overlaps stage B. With BLK the spectra are read in the blocked layout and the real rows
// written to `dst` (same field stride), a separate array; otherwise dst == data and the pass is in
// place.
template <int n, bool BLK = false>
__global__ void __launch_bounds__(X2<n>::T, 3) k2_fx_inv(float2* __restrict__ data, size_t fstride,
                                                       const float2* __restrict__ tw, int items_per_field,
                                                       int nfields, float2* __restrict__ dst) {
    using X = X2<n>;
    constexpr int RA = X::RA, RB = X::RB, N = 2 * n, T = X::T;
    extern __shared__ float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* tws = reinterpret_cast<Tw2*>(xb + Xch<n, RA>::SIZE);
    float2* stg = reinterpret_cast<float2*>(tws + 1);   // [8][n]
    load_tw2<n, N>(tws, tw, T);
    const int tid = threadIdx.x;
    const int nitems = items_per_field * nfields;
    auto gptr = [&](int t) { return dst + (size_t)(t / items_per_field) * fstride + (size_t)(t % items_per_field) * 8 * n; };
    auto prefetch = [&](int t) {
        float2* d = stg;
        if constexpr (BLK) {   // 8 rows of one plane (one row group): a 512-byte run per 8-column block
            const int row0 = (t % items_per_field) * 8, y0 = row0 % N, z = row0 / N;
            const float2* g = data + (size_t)(t / items_per_field) * fstride;
            for (int e = tid; e < 8 * n / 2; e += T) {
                const int q = e & 3, c = (e >> 2) & 7, kxb = e >> 5;
                cp_async16_cg(d + c * n + kxb * 8 + 2 * q, g + hs_index<N, true>(kxb * 8 + 2 * q, y0 + c, z));
            }
        } else {
            const float2* g = data + (size_t)(t / items_per_field) * fstride + (size_t)(t % items_per_field) * 8 * n;
            for (int e = tid; e < 8 * n / 2; e += T) cp_async16_cg(d + 2 * e, g + 2 * e);
        }
        cp_async_commit();
    };
    if (blockIdx.x < nitems) prefetch(blockIdx.x);
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        float2* d = gptr(t);
        const float2* rows = stg;
        cp_async_wait<0>();
        __syncthreads();
        // stage A reads its inputs Z'[k] = E + i O straight from the staged rows, with
        // E = X[k] + conj X[n-k], O = (X[k] - conj X[n-k]) conj w^k and X[n] = 0
        const int ca = tid / (n / RA), ja = tid % (n / RA);
        if (tid < X::TA) {
            const float2* row = rows + ca * n;
            float2 v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int k = ja + r * (n / RA);
                const float2 xk = row[k];
                const float2 xm = row[k == 0 ? 0 : n - k];
                const float2 xc = k == 0 ? make_float2(0.0f, 0.0f) : cconj(xm);
                const float2 E = cadd(xk, xc);
                const float2 O = cmul(csub(xk, xc), cconj(tw[k]));
                v[r] = make_float2(E.x - O.y, E.y + O.x);
            }
            dft<RA, +1>(v);
#pragma unroll
            for (int r = 0; r < RA; ++r) xb[Xch<n, RA>::at(ca, ja * RA + r)] = v[r];
        }
        __syncthreads();
        if (t + (int)gridDim.x < nitems) prefetch(t + gridDim.x);   // staging free: overlaps stage B
        if (tid < X::TB) {
            const int c = tid / RA, j = tid % RA;
            float2 u[RB];
            stage_b<n, RA, RB, +1>(xb, tws, c, j, u);
#pragma unroll
            for (int r = 0; r < RB; ++r) d[(size_t)c * n + j + RA * r] = u[r];
        }
        // no barrier: the next tile's stage A writes xb only after the wait + barrier at its top
    }
    cp_async_wait<0>();
}

}  // namespace colapm
