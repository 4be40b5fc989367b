// Ordering of the particle arrays by mesh cell (the analogue, on one GPU, of the particle
// migration of §4 that keeps each rank's particles with its slab of the mesh).
//
// The deposit and the gather read and write the eight CIC corners of every particle. In particle-id
// (Lagrangian) order a warp's particles start out as mesh neighbours, but as structure grows they
// spread over more and more cache lines; with the arrays ordered by cell, a warp's corners are runs
// of one or two mesh rows again. The order is a counting sort of the particles by bucket = one
// x-run of XB = 64 cells (a bucket holds a few particles, and the order inside a bucket, which the
// scatter leaves to its atomics, changes nothing a warp reads). The buckets are numbered tile by
// tile: tiles of XB x T x T cells (T = 2^tshift, 1 by default) in (z, y, x) order, and inside a
// tile its T x T runs by (z, y), so that the particles of one tile are contiguous and the bucket
// ends of the sort delimit them (the tiled deposit accumulates a tile in shared memory).
//
// Every step of the method is per particle or an order-independent integer sum (the fixed-point
// deposit), so the physics does not depend on the order; `id` keeps each slot's particle id for
// the calls that exchange particle data in id order.
#include "colapm_internal.h"

namespace colapm {

namespace {

constexpr int SCAN_T = 1024;           // threads of the scan kernels
constexpr int SCAN_PER = 4;            // elements per thread in the block scan
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

__device__ __forceinline__ unsigned bucket_of(float w, int nm, int xshift, int tshift) {
    const unsigned c = __float_as_uint(w), u = (unsigned)nm;   // linear cell x + nm (y + nm z)
    const unsigned x = c % u, yz = c / u, y = yz % u, z = yz / u, m = (1u << tshift) - 1u;
    const unsigned tile = ((z >> tshift) * (u >> tshift) + (y >> tshift)) * (u >> xshift) + (x >> xshift);
    return (tile << (2 * tshift)) + ((z & m) << tshift) + (y & m);
}

// Block-aggregated increment: the lanes of a warp with the same bucket are grouped (match_any; the
// first lane leads), and the warp groups of the whole block with the same bucket are merged
// through a small hash table in shared memory (keys, counts), so that each distinct bucket of the
// block takes ONE global atomic and its slots are contiguous across the block's warps. With RANK, returns each valid
// thread's slot (the bucket's old cursor + its rank in the block); every thread of the block must
// call it (valid = false for threads without a particle). The table has twice as many slots as the
// block has threads, so the bounded linear probing always finds the key or a free slot.
constexpr int SC_T = 256;              // threads of the block-aggregated sort kernels
constexpr int SC_H = 2 * SC_T;         // hash slots
constexpr unsigned SC_EMPTY = 0xffffffffu;

template <bool RANK>
__device__ __forceinline__ size_t block_bucket_add(unsigned* ctr, unsigned b, bool valid) {
    __shared__ unsigned keys[SC_H], cnt[SC_H], base[SC_H];
    for (int i = threadIdx.x; i < SC_H; i += SC_T) {
        keys[i] = SC_EMPTY;
        cnt[i] = 0u;
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    unsigned peers = 0, off = 0;
    int leader = 0, slot = 0;
    if (valid) {
        peers = __match_any_sync(act, b);
        leader = __ffs(peers) - 1;
        if ((int)lane == leader) {
            unsigned h = (b * 2654435761u) % (unsigned)SC_H;
            for (int i = 0; i < SC_H; ++i) {
                const unsigned k = atomicCAS(&keys[h], SC_EMPTY, b);
                if (k == SC_EMPTY || k == b) break;
                h = h + 1 == (unsigned)SC_H ? 0u : h + 1;
            }
            slot = (int)h;
            off = atomicAdd(&cnt[slot], (unsigned)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SC_H; i += SC_T) {
        const unsigned k = keys[i];
        if (k != SC_EMPTY) {
            const unsigned o = atomicAdd(ctr + k, cnt[i]);
            if (RANK) base[i] = o;
        }
    }
    if (!RANK) return 0;
    __syncthreads();
    size_t d = ~(size_t)0;
    if (valid) {
        unsigned bs = (int)lane == leader ? base[slot] + off : 0u;
        bs = __shfl_sync(peers, bs, leader);
        d = bs + (unsigned)__popc(peers & ((1u << lane) - 1u));
    }
    return d;
}

__global__ void __launch_bounds__(SC_T) k_sort_count(const float4* __restrict__ pos, size_t np3, int nm, int xshift,
                                                     int tshift, unsigned* __restrict__ cnt) {
    const size_t p = (size_t)blockIdx.x * SC_T + threadIdx.x;
    const bool valid = p < np3;
    block_bucket_add<false>(cnt, valid ? bucket_of(__ldg(&pos[p].w), nm, xshift, tshift) : 0u, valid);
}

// Exclusive scan of cnt[0..n) in tiles of SCAN_TILE: tile sums first, then the scan within tiles
// offset by the scanned tile sums (written to both start and cursor).
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const unsigned* __restrict__ cnt, size_t n,
                                                       unsigned* __restrict__ tile_sum) {
    __shared__ unsigned part[SCAN_T / 32];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        const size_t i = base + (size_t)k * SCAN_T + threadIdx.x;
        if (i < n) s += cnt[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned v = part[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
    }
}

// One block scans the tile sums in place (exclusive), SCAN_T at a time with a running carry.
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(unsigned* __restrict__ tile_sum, int ntiles) {
    __shared__ unsigned warp_tot[SCAN_T / 32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = 0; b < ntiles; b += SCAN_T) {
        const int i = b + threadIdx.x;
        const unsigned v = i < ntiles ? tile_sum[i] : 0u;
        unsigned x = v;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned t = warp_tot[lane];
            unsigned ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += y;
            }
            warp_tot[lane] = ti - t;   // exclusive prefix of the warp totals
        }
        __syncthreads();
        const unsigned c0 = carry;
        if (i < ntiles) tile_sum[i] = c0 + warp_tot[wid] + x - v;
        __syncthreads();
        if (threadIdx.x == SCAN_T - 1) carry = c0 + warp_tot[wid] + x;
        __syncthreads();
    }
}

// (cnt and cursor may be the same array: each thread reads its elements before it writes them.)
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const unsigned* cnt, size_t n,
                                                       const unsigned* __restrict__ tile_off, unsigned* cursor) {
    __shared__ unsigned warp_tot[SCAN_T / 32];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // thread t scans elements base + t * SCAN_PER .. + SCAN_PER - 1 (contiguous per thread)
    unsigned v[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        const size_t i = base + (size_t)threadIdx.x * SCAN_PER + k;
        v[k] = i < n ? cnt[i] : 0u;
        s += v[k];
    }
    unsigned x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const unsigned t = warp_tot[lane];
        unsigned ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;
    }
    __syncthreads();
    unsigned run = tile_off[blockIdx.x] + warp_tot[wid] + x - s;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        const size_t i = base + (size_t)threadIdx.x * SCAN_PER + k;
        if (i < n) cursor[i] = run;
        run += v[k];
    }
}

// Move every particle to the next free slot of its bucket (cursor[] starts at the bucket offsets).
// The slots of one bucket taken by one block are contiguous (block-aggregated cursors), so that the
// block's writes to each array come in runs as long as its particles of that bucket.
__global__ void __launch_bounds__(SC_T) k_sort_scatter(const float4* __restrict__ pos, const float* __restrict__ mom,
                                                       const float* __restrict__ psi1, const float* __restrict__ psi2,
                                                       const int* __restrict__ id, size_t np3, int nm, int xshift,
                                                       int tshift, unsigned* __restrict__ cursor,
                                                       float4* __restrict__ pos_o, float* __restrict__ mom_o,
                                                       float* __restrict__ psi1_o, float* __restrict__ psi2_o,
                                                       int* __restrict__ id_o, int* err) {
    const size_t p = (size_t)blockIdx.x * SC_T + threadIdx.x;
    const bool valid = p < np3;
    const float4 P = valid ? __ldcs(pos + p) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const size_t d = block_bucket_add<true>(cursor, valid ? bucket_of(P.w, nm, xshift, tshift) : 0u, valid);
    if (!valid) return;
    if (d >= np3) {   // cannot happen with consistent counts; guards the writes below
        atomicOr(err, 8);
        return;
    }
    __stcs(pos_o + d, P);
    id_o[d] = __ldcs(id + p);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mom_o[j * np3 + d] = __ldcs(mom + j * np3 + p);
        psi1_o[j * np3 + d] = __ldcs(psi1 + j * np3 + p);
        psi2_o[j * np3 + d] = __ldcs(psi2 + j * np3 + p);
    }
}

// Back to particle-id order: slot id[p] receives particle p's data.
__global__ void k_unsort(const float4* __restrict__ pos, const float* __restrict__ mom, const float* __restrict__ psi1,
                         const float* __restrict__ psi2, const int* __restrict__ id, size_t np3,
                         float4* __restrict__ pos_o, float* __restrict__ mom_o, float* __restrict__ psi1_o,
                         float* __restrict__ psi2_o, int* __restrict__ id_o) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const int i = id[p];
    pos_o[i] = pos[p];
    id_o[i] = i;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mom_o[j * np3 + i] = mom[j * np3 + p];
        psi1_o[j * np3 + i] = psi1[j * np3 + p];
        psi2_o[j * np3 + i] = psi2[j * np3 + p];
    }
}

__global__ void k_iota(int* __restrict__ id, size_t n) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) id[p] = (int)p;
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int sort_xshift(int nm) {
    int s = 0;
    while ((nm >> s) > 1 && (1 << s) < 64 && ((nm >> (s + 1)) << (s + 1)) == nm) ++s;
    return s;   // x-block of 2^s cells: 64 where nm allows, else the largest power of two dividing nm
}

size_t sort_buckets(int nm) { return (size_t)nm * nm * (size_t)(nm >> sort_xshift(nm)); }

size_t sort_tiles(int nm) { return (sort_buckets(nm) + SCAN_TILE - 1) / SCAN_TILE; }

bool sort_tshift_ok(int nm, int tshift) { return tshift >= 0 && tshift <= 3 && nm % (1 << tshift) == 0; }

cudaError_t launch_sort(SortBuffers b, size_t np3, int nm, int tshift, cudaStream_t s) {
    if (!sort_tshift_ok(nm, tshift)) return cudaErrorInvalidValue;
    const int xs = sort_xshift(nm);
    const size_t nb = sort_buckets(nm), nt = sort_tiles(nm);
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, nb * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_sort_count<<<blocks(np3, SC_T), SC_T, 0, s>>>(b.pos, np3, nm, xs, tshift, b.cnt);
    k_scan_tiles<<<(unsigned)nt, SCAN_T, 0, s>>>(b.cnt, nb, b.tile_sum);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(b.tile_sum, (int)nt);
    k_scan_apply<<<(unsigned)nt, SCAN_T, 0, s>>>(b.cnt, nb, b.tile_sum, b.cnt);   // counts -> cursors in place
    k_sort_scatter<<<blocks(np3, SC_T), SC_T, 0, s>>>(b.pos, b.mom, b.psi1, b.psi2, b.id, np3, nm, xs, tshift, b.cnt, b.pos_o,
                                                     b.mom_o, b.psi1_o, b.psi2_o, b.id_o, b.err);
    return cudaGetLastError();
}

cudaError_t launch_unsort(SortBuffers b, size_t np3, cudaStream_t s) {
    k_unsort<<<blocks(np3, 256), 256, 0, s>>>(b.pos, b.mom, b.psi1, b.psi2, b.id, np3, b.pos_o, b.mom_o, b.psi1_o,
                                              b.psi2_o, b.id_o);
    return cudaGetLastError();
}

cudaError_t launch_iota(int* id, size_t n, cudaStream_t s) {
    k_iota<<<blocks(n, 256), 256, 0, s>>>(id, n);
    return cudaGetLastError();
}

}  // namespace colapm
