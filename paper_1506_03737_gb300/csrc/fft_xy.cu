// Fused x-y passes for the large power-of-two meshes (N = 512, 1024): the forward x (r2c) and y
// transforms of the density, and the inverse y and x (c2r) transforms of the force spectra, each
// as ONE persistent kernel whose per-plane intermediate never leaves L2.
//
// Work is split into units: one z plane of one field. A unit has two phases. For the inverse,
// phase 1 = y transforms of the plane's column tiles (8 columns each) into a ring slot, phase 2
// = x transforms of the plane's row tiles (8 rows each) from the ring slot back into the field.
// The forward pass is the mirror (x rows into the ring, then y columns out of it). Tickets carry
// one tile each: longer tickets need a longer lag between the phases, hence a ring too large to
// stay in L2.
//
// Scheduling. CTAs take work-item tickets from one atomic counter. Ticket order interleaves the
// phases with a lag: step s holds phase-1 items of unit s and phase-2 items of unit s - LAG. A
// phase-2 item waits until its unit's phase-1 items are all done; a phase-1 item waits until the
// previous user of its ring slot (unit s - RING) has finished phase 2. Every wait is on items
// with smaller tickets, which CTAs already running hold (a CTA takes a ticket only after its
// previous item is done), so the waits end without any co-residency assumption. Each wait is
// still bounded: past the iteration limit the kernel sets the timeout bit in the error word and
// carries on (the result is then wrong, never hung).
//
// Memory ordering: after a barrier one thread fences and adds to the unit's counter with a
// release; the waiter reads the counter with acquire, barriers, and reads the ring with .cg
// loads (L2, never a stale L1 line). Each CTA fetches its next ticket while the current item
// runs; it holds both, and finishes the current item (whose waits are on smaller tickets) first. Ring data uses default stores so it stays in L2; the input
// planes are read and the final planes written with the streaming (.cs) policy.
#include "fft2.cuh"
#include "launch_cache.h"

namespace colapm {

namespace {

constexpr int XY_T = 256;
constexpr int XY_LAG = 4;          // steps between a unit's phase-1 and phase-2 tickets
constexpr int XY_RING = 8;         // ring slots (units)
constexpr int XY_ERR_TIMEOUT = 4;
constexpr long long XY_SPIN_LIMIT = 1ll << 23;   // x >= 64 ns of back-off: about a second at most

template <int L>
struct XY {
    static constexpr int n = L / 2;
    static constexpr int RY = F2<L>::R1, RYB = F2<L>::R2;   // y (length L) radices
    static constexpr int RX = F2<n>::R1, RXB = F2<n>::R2;   // x (n complex points) radices
    static constexpr int XSX = Xch<n, RX>::SIZE + 8 * n;         // x exchange + 8 staged rows
    static constexpr int XS = Xch<L, RY>::SIZE > XSX ? Xch<L, RY>::SIZE : XSX;
    static constexpr int COLS = n / 8;                        // column tiles per plane
    static constexpr int ROWS = L / 8;                        // row tiles per plane
    static constexpr size_t PLANE = (size_t)L * n;            // complex values per plane
    static constexpr size_t SMEM = sizeof(float2) * XS + 2 * sizeof(Tw2);
    static_assert(8 * L / RY <= XY_T && 8 * L / RYB <= XY_T && 8 * n / RX <= XY_T && 8 * n / RXB <= XY_T, "threads");
};

// Block barriers (bar.sync) need each warp converged. Every section run by thread 0 alone is
// therefore closed with __syncwarp() before the next __syncthreads(), and the spin-wait is run by
// the whole of warp 0 with a warp-uniform exit (lane 0 reads, all lanes decide on its value).
//
// End of a work item: every thread's stores are issued before the barrier; thread 0 then fences
// (cumulative over the CTA's writes ordered by the barrier), releases the unit's counter (if any)
// and publishes the ticket it prefetched; the second barrier makes that ticket visible.
__device__ __forceinline__ void end_item(int* done, int* tk, int next) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (done) {
            __threadfence();
            asm volatile("red.release.gpu.global.add.s32 [%0], 1;\n" ::"l"(done) : "memory");
        }
        *tk = next;
    }
    __syncwarp();
    __syncthreads();
}

__device__ __forceinline__ void wait_count(const int* p, int target, int* err) {
    if (threadIdx.x < 32) {
        for (long long i = 0;; ++i) {
            int v = 0;
            if (threadIdx.x == 0) asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
            v = __shfl_sync(0xffffffffu, v, 0);
            if (v >= target) break;
            if (i >= XY_SPIN_LIMIT) {
                if (threadIdx.x == 0) atomicOr(err, XY_ERR_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        __syncwarp();
        __threadfence();
    }
    __syncthreads();
}

// y transform (sign S) of the 8 columns kx0..kx0+7 of one plane: src -> dst (both [y][x], pitch n).
template <int L, int S, bool SRC_RING>
__device__ __forceinline__ void y_tile(const float2* __restrict__ src, float2* __restrict__ dst, int kx0, float2* xb,
                                       const Tw2* tws) {
    constexpr int n = L / 2, RA = F2<L>::R1, RB = F2<L>::R2;
    constexpr int TA = 8 * L / RA, TB = 8 * L / RB;
    const int tid = threadIdx.x, c = tid & 7, j = tid >> 3;
    if (tid < TA) {
        const float2* g = src + kx0 + c;
        float2 v[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const float2* a = g + (size_t)(j + r * (L / RA)) * n;
            v[r] = SRC_RING ? __ldcg(a) : __ldcs(a);
        }
        dft<RA, S>(v);
#pragma unroll
        for (int r = 0; r < RA; ++r) xb[Xch<L, RA>::at(c, j * RA + r)] = v[r];
    }
    __syncthreads();
    if (tid < TB) {
        float2 v[RB];
        stage_b<L, RA, RB, S>(xb, tws, c, j, v);
        float2* o = dst + kx0 + c;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            float2* a = o + (size_t)(j + RA * r) * n;
            if (SRC_RING) __stcs(a, v[r]); else *a = v[r];
        }
    }
    __syncthreads();
}

// Forward r2c of 8 rows of N = 2n int64 density values (converted to rho * scale - 1) into 8 rows
// of n complex (k_x < n; the k_x = n plane is dropped, as every spectral operator zeroes it).
template <int n>
__device__ __forceinline__ bool x_fwd_rows(const unsigned long long* __restrict__ rho, float2* __restrict__ out,
                                           const float2* __restrict__ tw, float scale, float2* xb, const Tw2* tws,
                                           bool zero) {
    constexpr int RA = F2<n>::R1, RB = F2<n>::R2, TA = 8 * n / RA, TB = 8 * n / RB;
    const int tid = threadIdx.x;
    bool over = false;
    if (tid < TA) {
        const int c = tid / (n / RA), j = tid % (n / RA);
        float2 v[RA];
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(rho) + (size_t)c * n + j;
        ulonglong2 q[RA];   // all loads first: the clearing stores alias them
#pragma unroll
        for (int r = 0; r < RA; ++r) q[r] = __ldcs(src + r * (n / RA));
        if (zero) {
#pragma unroll
            for (int r = 0; r < RA; ++r) __stcs(const_cast<ulonglong2*>(src) + r * (n / RA), make_ulonglong2(0ull, 0ull));
        }
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            over |= ((q[r].x | q[r].y) >> 63) != 0;
            v[r] = make_float2(fmaf((float)(long long)q[r].x, scale, -1.0f), fmaf((float)(long long)q[r].y, scale, -1.0f));
        }
        dft<RA, -1>(v);
#pragma unroll
        for (int r = 0; r < RA; ++r) xb[Xch<n, RA>::at(c, j * RA + r)] = v[r];
    }
    __syncthreads();
    if (tid < TB) {
        const int c = tid / RA, j = tid % RA;
        float2 v[RB];
        stage_b<n, RA, RB, -1>(xb, tws, c, j, v);
#pragma unroll
        for (int r = 0; r < RB; ++r) xb[Xch<n, RA>::at(c, j + RA * r)] = v[r];
    }
    __syncthreads();
    constexpr int H = n / 2 + 1;
    for (int e = tid; e < 8 * H; e += XY_T) {
        const int c = e / H, k = e % H, k2 = (n - k) % n;
        const float2 a = xb[Xch<n, RA>::at(c, k)], b = xb[Xch<n, RA>::at(c, k2)];
        float2* o = out + (size_t)c * n;
        {   // X[k] from Z[k] = a, Z[n-k] = b; w^k = exp(-2 pi i k / N) = tw[k]
            const float2 bc = cconj(b);
            const float2 E = cscale(cadd(a, bc), 0.5f);
            const float2 d = csub(a, bc);
            o[k] = cadd(E, cmul(tw[k], make_float2(0.5f * d.y, -0.5f * d.x)));
        }
        if (k != 0 && k2 != k) {
            const float2 ac = cconj(a);
            const float2 E = cscale(cadd(b, ac), 0.5f);
            const float2 d = csub(b, ac);
            o[k2] = cadd(E, cmul(tw[k2], make_float2(0.5f * d.y, -0.5f * d.x)));
        }
    }
    __syncthreads();
    return over;
}

// Inverse c2r of 8 rows of n complex (from the ring) into 8 rows of N reals stored as n pairs.
template <int n>
__device__ __forceinline__ void x_inv_rows(const float2* __restrict__ rows, float2* __restrict__ dst,
                                           const float2* __restrict__ tw, float2* xb, const Tw2* tws) {
    constexpr int RA = F2<n>::R1, RB = F2<n>::R2, TA = 8 * n / RA, TB = 8 * n / RB;
    const int tid = threadIdx.x;
    constexpr int H = n / 2 + 1;
    // One batch of coalesced 16-byte loads of the 8 rows into the space after the exchange buffer.
    float2* raw = xb + Xch<n, RA>::SIZE;
    constexpr int V4 = 8 * n / 2 / XY_T;
    static_assert(V4 * XY_T * 2 == 8 * n, "rows split evenly");
    float4 q[V4];
#pragma unroll
    for (int i = 0; i < V4; ++i) q[i] = __ldcg(reinterpret_cast<const float4*>(rows) + tid + i * XY_T);
#pragma unroll
    for (int i = 0; i < V4; ++i) reinterpret_cast<float4*>(raw)[tid + i * XY_T] = q[i];
    __syncthreads();
    for (int e = tid; e < 8 * H; e += XY_T) {   // Z'[k], Z'[n-k] from X[k], X[n-k] (X[n] = 0)
        const int c = e / H, k = e % H;
        const float2* row = raw + c * n;
        const float2 xk = row[k];
        if (k == 0) {
            xb[Xch<n, RA>::at(c, 0)] = make_float2(xk.x - xk.y, xk.y + xk.x);   // X0 + i X0
            continue;
        }
        const int k2 = n - k;
        const float2 xk2 = row[k2];
        {
            const float2 xc = cconj(xk2);
            const float2 E = cadd(xk, xc);
            const float2 O = cmul(csub(xk, xc), cconj(tw[k]));
            xb[Xch<n, RA>::at(c, k)] = make_float2(E.x - O.y, E.y + O.x);
        }
        if (k2 != k) {
            const float2 xc = cconj(xk);
            const float2 E = cadd(xk2, xc);
            const float2 O = cmul(csub(xk2, xc), cconj(tw[k2]));
            xb[Xch<n, RA>::at(c, k2)] = make_float2(E.x - O.y, E.y + O.x);
        }
    }
    __syncthreads();
    float2 v[RA];
    const int ca = tid / (n / RA), ja = tid % (n / RA);
    if (tid < TA) {
#pragma unroll
        for (int r = 0; r < RA; ++r) v[r] = xb[Xch<n, RA>::at(ca, ja + r * (n / RA))];
        dft<RA, +1>(v);
    }
    __syncthreads();
    if (tid < TA) {
#pragma unroll
        for (int r = 0; r < RA; ++r) xb[Xch<n, RA>::at(ca, ja * RA + r)] = v[r];
    }
    __syncthreads();
    if (tid < TB) {
        const int c = tid / RA, j = tid % RA;
        float2 u[RB];
        stage_b<n, RA, RB, +1>(xb, tws, c, j, u);
#pragma unroll
        for (int r = 0; r < RB; ++r) __stcs(dst + (size_t)c * n + j + RA * r, u[r]);
    }
    __syncthreads();
}

// ctr: [0] ticket, [1, 1 + U) phase-1 counts, [1 + U, 1 + 2U) phase-2 counts (zeroed by the host).
template <int L>
__global__ void __launch_bounds__(XY_T, 2) k_xy_inv(float2* __restrict__ data, size_t fstride, int nfields,
                                                     const float2* __restrict__ tw, float2* __restrict__ ring,
                                                     int* __restrict__ ctr, int* err) {
    using P = XY<L>;
    extern __shared__ float4 smem4[];
    __shared__ int tk;
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* twy = reinterpret_cast<Tw2*>(xb + P::XS);
    Tw2* twx = twy + 1;
    load_tw2<L, L>(twy, tw, XY_T);
    load_tw2<P::n, L>(twx, tw, XY_T);
    const int U = L * nfields, SS = P::COLS + P::ROWS;
    const long long total = (long long)(U + XY_LAG) * SS;
    int* done1 = ctr + 1;
    int* done2 = ctr + 1 + U;
    if (threadIdx.x == 0) tk = atomicAdd(ctr, 1);
    __syncwarp();
    __syncthreads();
    for (;;) {
        const int t = tk;
        if (t >= total) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(ctr, 1);   // the next ticket, fetched while this item runs
        const int s = t / SS, k = t % SS;
        int* done = nullptr;
        if (k < P::COLS) {
            const int u = s;
            if (u < U) {
                if (u >= XY_RING) wait_count(done2 + (u - XY_RING), P::ROWS, err);
                const float2* plane = data + (size_t)(u % nfields) * fstride + (size_t)(u / nfields) * P::PLANE;
                y_tile<L, +1, false>(plane, ring + (size_t)(u % XY_RING) * P::PLANE, 8 * k, xb, twy);
                done = done1 + u;
            }
        } else {
            const int u = s - XY_LAG;
            if (u >= 0) {
                wait_count(done1 + u, P::COLS, err);
                const size_t r0 = (size_t)8 * (k - P::COLS) * P::n;
                float2* plane = data + (size_t)(u % nfields) * fstride + (size_t)(u / nfields) * P::PLANE;
                x_inv_rows<P::n>(ring + (size_t)(u % XY_RING) * P::PLANE + r0, plane + r0, tw, xb, twx);
                done = done2 + u;
            }
        }
        end_item(done, &tk, next);
    }
}

template <int L>
__global__ void __launch_bounds__(XY_T, 2) k_xy_fwd(const unsigned long long* __restrict__ rho, float2* __restrict__ out,
                                                     const float2* __restrict__ tw, float scale,
                                                     float2* __restrict__ ring, int* __restrict__ ctr, int* err,
                                                     bool zero) {
    using P = XY<L>;
    extern __shared__ float4 smem4[];
    __shared__ int tk;
    float2* xb = reinterpret_cast<float2*>(smem4);
    Tw2* twy = reinterpret_cast<Tw2*>(xb + P::XS);
    Tw2* twx = twy + 1;
    load_tw2<L, L>(twy, tw, XY_T);
    load_tw2<P::n, L>(twx, tw, XY_T);
    const int U = L, SS = P::ROWS + P::COLS;
    const long long total = (long long)(U + XY_LAG) * SS;
    int* done1 = ctr + 1;
    int* done2 = ctr + 1 + U;
    bool over = false;
    if (threadIdx.x == 0) tk = atomicAdd(ctr, 1);
    __syncwarp();
    __syncthreads();
    for (;;) {
        const int t = tk;
        if (t >= total) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(ctr, 1);   // the next ticket, fetched while this item runs
        const int s = t / SS, k = t % SS;
        int* done = nullptr;
        if (k < P::ROWS) {
            const int u = s;
            if (u < U) {
                if (u >= XY_RING) wait_count(done2 + (u - XY_RING), P::COLS, err);
                const size_t row0 = (size_t)u * L + 8 * k;   // density rows of N = L values
                over |= x_fwd_rows<P::n>(rho + row0 * L, ring + (size_t)(u % XY_RING) * P::PLANE + (size_t)8 * k * P::n,
                                         tw, scale, xb, twx, zero);
                done = done1 + u;
            }
        } else {
            const int u = s - XY_LAG;
            if (u >= 0) {
                wait_count(done1 + u, P::ROWS, err);
                y_tile<L, -1, true>(ring + (size_t)(u % XY_RING) * P::PLANE, out + (size_t)u * P::PLANE,
                                    8 * (k - P::ROWS), xb, twy);
                done = done2 + u;
            }
        }
        end_item(done, &tk, next);
    }
    if (over) atomicOr(err, 1);
}

GridCache g_fwd512, g_fwd1024, g_inv512, g_inv1024;   // per-device persistent grids

}  // namespace

bool xy_supported(int nm) { return nm == 512 || nm == 1024; }

size_t xy_ring_bytes(int nm) { return xy_supported(nm) ? (size_t)XY_RING * nm * (nm / 2) * sizeof(float2) : 0; }

size_t xy_ctr_ints(int nm, int nfields) { return 1 + 2 * (size_t)nm * nfields; }

cudaError_t launch_xy_fwd(int nm, const unsigned long long* rho, float2* out, const float2* tw, float scale,
                          float2* ring, int* ctr, int* err, cudaStream_t s, bool zero_input) {
    cudaError_t e = cudaMemsetAsync(ctr, 0, xy_ctr_ints(nm, 1) * sizeof(int), s);
    if (e) return e;
    int grid = 0;
    switch (nm) {
    case 512:
        if ((e = cached_grid(g_fwd512, k_xy_fwd<512>, XY_T, XY<512>::SMEM, &grid)) != cudaSuccess) return e;
        k_xy_fwd<512><<<grid, XY_T, XY<512>::SMEM, s>>>(
            rho, out, tw, scale, ring, ctr, err, zero_input);
        break;
    case 1024:
        if ((e = cached_grid(g_fwd1024, k_xy_fwd<1024>, XY_T, XY<1024>::SMEM, &grid)) != cudaSuccess) return e;
        k_xy_fwd<1024><<<grid, XY_T, XY<1024>::SMEM, s>>>(
            rho, out, tw, scale, ring, ctr, err, zero_input);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_xy_inv(int nm, float2* data, size_t fstride, int nfields, const float2* tw, float2* ring, int* ctr,
                          int* err, cudaStream_t s) {
    if (nfields < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ctr, 0, xy_ctr_ints(nm, nfields) * sizeof(int), s);
    if (e) return e;
    int grid = 0;
    switch (nm) {
    case 512:
        if ((e = cached_grid(g_inv512, k_xy_inv<512>, XY_T, XY<512>::SMEM, &grid)) != cudaSuccess) return e;
        k_xy_inv<512><<<grid, XY_T, XY<512>::SMEM, s>>>(
            data, fstride, nfields, tw, ring, ctr, err);
        break;
    case 1024:
        if ((e = cached_grid(g_inv1024, k_xy_inv<1024>, XY_T, XY<1024>::SMEM, &grid)) != cudaSuccess) return e;
        k_xy_inv<1024><<<grid, XY_T, XY<1024>::SMEM, s>>>(
            data, fstride, nfields, tw, ring, ctr, err);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace colapm
