// Shared-memory Stockham FFT engine for the mesh transforms of the particle-mesh solver.
//
// The paper computes these transforms with FFTW-3 (§2.4 step 2, §4.3). Here each CTA
// transforms a tile of lines held in shared memory: either W adjacent columns of a strided
// axis ("column-major" tile, element (pos, col) at pos * (W + 1) + col, so that the W
// contiguous complex values of one mesh row arrive in one coalesced load), or W whole
// contiguous rows ("line-major" tile, element (line, pos) at line * LP + pos + pos / 16).
// The paddings keep both the strided butterfly reads and the scattered Stockham writes of
// 8-byte complex values within two shared-memory wavefronts per warp (column-major tiles
// additionally need a first radix of at most 8).
//
// One stage of radix R at stride Ns (the product of the radices before it) takes, for every
// butterfly j < L/R, the inputs j + r L/R, multiplies input r by w^((j mod Ns) r L/(Ns R))
// with w = exp(sign 2 pi i / L), applies the R-point DFT in registers and writes output r
// to (j / Ns) Ns R + (j mod Ns) + r Ns (Stockham autosort: natural order after the last
// stage). Each stage reads all its inputs into registers, synchronises, then writes.
#pragma once

#include <cuda_runtime.h>

namespace colapm {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i (s = +-1)
template <int S>
__device__ __forceinline__ float2 cmul_si(float2 a) { return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

template <int R, int S>
__device__ __forceinline__ float2 root(int k) {   // exp(S 2 pi i k / R), R in {2,4,8,16}, k < R/2
    constexpr int step = 16 / R;
    float c, s;
    switch (k * step) {
        case 0: c = 1.0f; s = 0.0f; break;
        case 1: c = 0.92387953251128675613f; s = 0.38268343236508977173f; break;
        case 2: c = 0.70710678118654752440f; s = 0.70710678118654752440f; break;
        case 3: c = 0.38268343236508977173f; s = 0.92387953251128675613f; break;
        case 4: c = 0.0f; s = 1.0f; break;
        case 5: c = -0.38268343236508977173f; s = 0.92387953251128675613f; break;
        case 6: c = -0.70710678118654752440f; s = 0.70710678118654752440f; break;
        default: c = -0.92387953251128675613f; s = 0.38268343236508977173f; break;
    }
    return make_float2(c, S > 0 ? s : -s);
}

// In-register R-point DFT, X_k = sum_m v_m exp(S 2 pi i m k / R).
template <int R, int S>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        constexpr float h = 0.86602540378443864676f;   // sqrt(3)/2
        float2 a = v[0], b = v[1], c = v[2];
        float2 t1 = cadd(b, c);
        float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
        float2 t3 = cscale(csub(b, c), S > 0 ? h : -h);
        float2 it3 = make_float2(-t3.y, t3.x);
        v[0] = cadd(a, t1);
        v[1] = cadd(t2, it3);
        v[2] = csub(t2, it3);
    } else if constexpr (R == 4) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = cmul_si<S>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 5) {
        constexpr float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        constexpr float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float sg = S > 0 ? 1.0f : -1.0f;
        float2 b1 = make_float2(sg * (s1 * t3.x + s2 * t4.x), sg * (s1 * t3.y + s2 * t4.y));
        float2 b2 = make_float2(sg * (s2 * t3.x - s1 * t4.x), sg * (s2 * t3.y - s1 * t4.y));
        float2 ib1 = make_float2(-b1.y, b1.x), ib2 = make_float2(-b2.y, b2.x);
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, ib1);
        v[4] = csub(a1, ib1);
        v[2] = cadd(a2, ib2);
        v[3] = csub(a2, ib2);
    } else {
        static_assert(R == 8 || R == 16, "unsupported radix");
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            e[m] = v[2 * m];
            o[m] = v[2 * m + 1];
        }
        dft<R / 2, S>(e);
        dft<R / 2, S>(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            float2 t = cmul(o[k], root<R, S>(k));
            v[k] = cadd(e[k], t);
            v[k + R / 2] = csub(e[k], t);
        }
    }
}

template <int... Rs>
struct Radices {};

// Radix plan per transform length; column-major tiles need a first radix <= 8.
template <int L> struct Plan;
template <> struct Plan<8> { using type = Radices<8>; };
template <> struct Plan<16> { using type = Radices<4, 4>; };
template <> struct Plan<32> { using type = Radices<8, 4>; };
template <> struct Plan<48> { using type = Radices<4, 4, 3>; };
template <> struct Plan<64> { using type = Radices<8, 8>; };
template <> struct Plan<80> { using type = Radices<4, 4, 5>; };
template <> struct Plan<96> { using type = Radices<8, 4, 3>; };
template <> struct Plan<128> { using type = Radices<8, 16>; };
template <> struct Plan<160> { using type = Radices<8, 4, 5>; };
template <> struct Plan<192> { using type = Radices<8, 8, 3>; };
template <> struct Plan<256> { using type = Radices<8, 8, 4>; };
template <> struct Plan<320> { using type = Radices<8, 8, 5>; };
template <> struct Plan<384> { using type = Radices<8, 16, 3>; };
template <> struct Plan<512> { using type = Radices<8, 8, 8>; };
template <> struct Plan<1024> { using type = Radices<8, 8, 16>; };

template <int L, int W, bool LINE_MAJOR>
struct Tile {
    static constexpr int LP = L + L / 16 + 1;                 // padded line (line-major)
    static constexpr int PITCH = W + 1;                       // padded row (column-major)
    static constexpr int SIZE = LINE_MAJOR ? W * LP : L * PITCH;
    __device__ __forceinline__ static int at(int line, int pos) {
        return LINE_MAJOR ? line * LP + pos + (pos >> 4) : pos * PITCH + line;
    }
};

// One Stockham stage over a whole tile (all W lines), T threads.
// tw: exp(-2 pi i t / TWN), t < TWN (shared or global memory), TWN a multiple of L.
template <int L, int W, int T, bool LINE_MAJOR, int S, int NS, int R, int TWN>
__device__ __forceinline__ void stockham_stage(float2* sm, const float2* tw) {
    using TL = Tile<L, W, LINE_MAJOR>;
    constexpr int NB = (L / R) * W;             // butterflies in the tile
    constexpr int PER = (NB + T - 1) / T;       // butterflies per thread
    float2 v[PER][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int b = tid + i * T;
        if (NB % T == 0 || b < NB) {
            const int line = LINE_MAJOR ? b / (L / R) : b % W;
            const int j = LINE_MAJOR ? b % (L / R) : b / W;
            const int jm = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = sm[TL::at(line, j + r * (L / R))];
                if (NS > 1 && r > 0) {
                    float2 w = tw[jm * r * (L / (NS * R)) * (TWN / L)];   // index < TWN
                    x = cmul(x, S > 0 ? cconj(w) : w);
                }
                v[i][r] = x;
            }
            dft<R, S>(v[i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int b = tid + i * T;
        if (NB % T == 0 || b < NB) {
            const int line = LINE_MAJOR ? b / (L / R) : b % W;
            const int j = LINE_MAJOR ? b % (L / R) : b / W;
            const int d = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) sm[TL::at(line, d + r * NS)] = v[i][r];
        }
    }
    __syncthreads();
}

template <int L, int W, int T, bool LINE_MAJOR, int S, int NS, int TWN, int R, int... Rest>
__device__ __forceinline__ void stockham_run(float2* sm, const float2* tw, Radices<R, Rest...>) {
    stockham_stage<L, W, T, LINE_MAJOR, S, NS, R, TWN>(sm, tw);
    if constexpr (sizeof...(Rest) > 0) stockham_run<L, W, T, LINE_MAJOR, S, NS * R, TWN>(sm, tw, Radices<Rest...>{});
}

// Transform every line of the tile in place; the caller has synchronised after filling it.
template <int L, int W, int T, bool LINE_MAJOR, int S, int TWN>
__device__ __forceinline__ void tile_fft(float2* sm, const float2* tw) {
    stockham_run<L, W, T, LINE_MAJOR, S, 1, TWN>(sm, tw, typename Plan<L>::type{});
}

}  // namespace colapm
