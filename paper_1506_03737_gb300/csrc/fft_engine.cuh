// Shared-memory Stockham FFT engine for the mesh transforms of the particle-mesh solver.
//
// The paper computes these transforms with FFTW-3 (§2.4 step 2, §4.3). Here each CTA transforms
// a tile of 8 lines held in shared memory as L rows of 8 complex values (64 bytes per row): row
// pos holds element pos of each of the 8 lines. A strided mesh axis maps 8 adjacent mesh columns
// to one tile (each row is one coalesced 64-byte segment); a contiguous axis is transposed into
// the same shape on load. Row r is stored at physical row r ^ (((r >> 2) ^ (r >> 3)) & 1): this
// swaps the two rows of a 128-byte bank line when bits 2 and 3 of r differ, so that rows at
// strides 1, 4 and 8 fall alternately into the two bank halves.
//
// Each thread works on two adjacent columns at once (one 16-byte shared access per element pair).
// One stage of radix R at stride Ns (the product of the radices before it) takes, for every
// butterfly j < L/R, the inputs j + r L/R, multiplies input r by w^((j mod Ns) r L/(Ns R)) with
// w = exp(sign 2 pi i / L), applies the R-point DFT in registers and writes output r to
// (j / Ns) Ns R + (j mod Ns) + r Ns (Stockham autosort: natural order after the last stage).
// With a first radix of 4 or 8 every stage's shared-memory accesses take the minimum number of
// wavefronts. Each stage reads all of its inputs into registers, synchronises, then writes.
#pragma once

#include <cuda_runtime.h>

namespace colapm {

__device__ __forceinline__ void cp_async8_ca(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i (s = +-1)
template <int S>
__host__ __device__ __forceinline__ float2 cmul_si(float2 a) { return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

// cos and sin of 2 pi m / 32, m = 0..15 (mathematical constants rounded to float)
#define COLAPM_C32(m) ((m) == 0 ? 1.0f : (m) == 1 ? 0.98078528040323044913f : (m) == 2 ? 0.92387953251128675613f : \
    (m) == 3 ? 0.83146961230254523708f : (m) == 4 ? 0.70710678118654752440f : (m) == 5 ? 0.55557023301960222474f : \
    (m) == 6 ? 0.38268343236508977173f : (m) == 7 ? 0.19509032201612826785f : (m) == 8 ? 0.0f : \
    (m) == 9 ? -0.19509032201612826785f : (m) == 10 ? -0.38268343236508977173f : (m) == 11 ? -0.55557023301960222474f : \
    (m) == 12 ? -0.70710678118654752440f : (m) == 13 ? -0.83146961230254523708f : (m) == 14 ? -0.92387953251128675613f : \
    -0.98078528040323044913f)
#define COLAPM_S32(m) ((m) == 0 ? 0.0f : COLAPM_C32(8 - (m) < 0 ? (m) - 8 : 8 - (m)))

template <int R, int S>
__host__ __device__ __forceinline__ float2 root(int k) {   // exp(S 2 pi i k / R), R in {2,4,8,16,32}, k < R/2 (unrolled)
    const int m = k * (32 / R);
    const float c = COLAPM_C32(m), s = COLAPM_S32(m);
    return make_float2(c, S > 0 ? s : -s);
}

// Coprime split R = N1 N2 of the composite radices (N1 = 1: none), with the modular inverses
// INV2 = N2^-1 mod N1 and INV1 = N1^-1 mod N2 of the output map.
constexpr int inv_mod(int a, int m) {
    for (int x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return m == 1 ? 0 : -1;
}
template <int R>
struct Pfa {
    static constexpr int N1 = R == 6 ? 2 : R == 10 ? 2 : R == 12 ? 4 : R == 15 ? 3 : R == 20 ? 4 : R == 24 ? 8 :
                              R == 40 ? 8 : R == 48 ? 16 : 1;
    static constexpr int N2 = R / N1;
    static constexpr int INV2 = N1 > 1 ? inv_mod(N2 % N1, N1) : 0;
    static constexpr int INV1 = N1 > 1 ? inv_mod(N1 % N2, N2) : 0;
    static_assert(N1 == 1 || (INV1 > 0 && INV2 > 0), "factors must be coprime");
};

// In-register R-point DFT, X_k = sum_m v_m exp(S 2 pi i m k / R).
template <int R, int S>
__host__ __device__ __forceinline__ void dft(float2* v) {
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
    } else if constexpr (Pfa<R>::N1 > 1) {
        // Good-Thomas prime-factor split R = N1 N2 (coprime): with the input map
        // n = (N2 n1 + N1 n2) mod R and the Chinese-remainder output map k = k1 (mod N1),
        // k = k2 (mod N2), exp(2 pi i n k / R) factors into exp(2 pi i n1 k1 / N1) exp(2 pi i n2 k2 / N2):
        // an N2-point DFT of every row n1, then an N1-point DFT of every column k2, with no twiddles.
        // All indices are compile-time constants, so the maps are register renaming only.
        constexpr int N1 = Pfa<R>::N1, N2 = Pfa<R>::N2;
        float2 a[N1][N2];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1)
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) a[n1][n2] = v[(N2 * n1 + N1 * n2) % R];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) dft<N2, S>(a[n1]);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            float2 col[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) col[n1] = a[n1][k2];
            dft<N1, S>(col);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[(k1 * N2 * Pfa<R>::INV2 + k2 * N1 * Pfa<R>::INV1) % R] = col[k1];
        }
    } else {
        static_assert(R == 8 || R == 16 || R == 32, "unsupported radix");
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

// Radix plan per transform length (first radix 4 or 8).
template <int L> struct Plan;
template <> struct Plan<8> { using type = Radices<8>; };
template <> struct Plan<16> { using type = Radices<4, 4>; };
template <> struct Plan<32> { using type = Radices<8, 4>; };
template <> struct Plan<48> { using type = Radices<4, 4, 3>; };
template <> struct Plan<64> { using type = Radices<8, 8>; };
template <> struct Plan<80> { using type = Radices<4, 4, 5>; };
template <> struct Plan<96> { using type = Radices<8, 4, 3>; };
template <> struct Plan<128> { using type = Radices<8, 4, 4>; };
template <> struct Plan<160> { using type = Radices<8, 4, 5>; };
template <> struct Plan<192> { using type = Radices<8, 8, 3>; };
template <> struct Plan<256> { using type = Radices<8, 8, 4>; };
template <> struct Plan<320> { using type = Radices<8, 8, 5>; };
template <> struct Plan<384> { using type = Radices<8, 4, 4, 3>; };
template <> struct Plan<512> { using type = Radices<8, 8, 8>; };
template <> struct Plan<1024> { using type = Radices<8, 8, 4, 4>; };

// Tile of L rows x 8 complex columns.
template <int L>
struct CT {
    static constexpr int SIZE = 8 * L;   // float2 elements
    __device__ __forceinline__ static int prow(int r) { return r ^ (((r >> 2) ^ (r >> 3)) & 1); }
    __device__ __forceinline__ static int a2(int r, int c) { return prow(r) * 8 + c; }   // float2 index
    __device__ __forceinline__ static int a4(int r, int q) { return prow(r) * 4 + q; }   // float4 index
};

// One Stockham stage over the tile, T threads, each butterfly on a column pair.
// tw: exp(-2 pi i t / TWN), t < TWN (shared or global memory), TWN a multiple of L.
template <int L, int T, int S, int NS, int R, int TWN>
__device__ __forceinline__ void stockham_stage(float2* sm, const float2* tw) {
    constexpr int NB = (L / R) * 4;
    constexpr int PER = (NB + T - 1) / T;
    float4* s4 = reinterpret_cast<float4*>(sm);
    float2 va[PER][R], vb[PER][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int b = tid + i * T;
        if (NB % T == 0 || b < NB) {
            const int q = b & 3, j = b >> 2, jm = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 x = s4[CT<L>::a4(j + r * (L / R), q)];
                float2 a = make_float2(x.x, x.y), c = make_float2(x.z, x.w);
                if (NS > 1 && r > 0) {
                    float2 w = tw[jm * r * (L / (NS * R)) * (TWN / L)];   // index < TWN
                    if (S > 0) w = cconj(w);
                    a = cmul(a, w);
                    c = cmul(c, w);
                }
                va[i][r] = a;
                vb[i][r] = c;
            }
            dft<R, S>(va[i]);
            dft<R, S>(vb[i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int b = tid + i * T;
        if (NB % T == 0 || b < NB) {
            const int q = b & 3, j = b >> 2;
            const int d = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r)
                s4[CT<L>::a4(d + r * NS, q)] = make_float4(va[i][r].x, va[i][r].y, vb[i][r].x, vb[i][r].y);
        }
    }
    __syncthreads();
}

template <int L, int T, int S, int NS, int TWN, int R, int... Rest>
__device__ __forceinline__ void stockham_run(float2* sm, const float2* tw, Radices<R, Rest...>) {
    stockham_stage<L, T, S, NS, R, TWN>(sm, tw);
    if constexpr (sizeof...(Rest) > 0) stockham_run<L, T, S, NS * R, TWN>(sm, tw, Radices<Rest...>{});
}

// Transform the 8 lines of the tile in place; the caller has synchronised after filling it.
template <int L, int T, int S, int TWN>
__device__ __forceinline__ void tile_fft(float2* sm, const float2* tw) {
    stockham_run<L, T, S, 1, TWN>(sm, tw, typename Plan<L>::type{});
}

}  // namespace colapm
