// Particle kernels of the particle-mesh step (§2.3, §2.4 steps 1 and 4).
//
// Particle state (particle-id order): pos[p] = float4(offset_x, offset_y, offset_z, cell bits)
// with the offsets in [0, 1) mesh cells and the linear cell index x + N (y + N z) stored in
// the w word; mom, psi1, psi2 are component-major float arrays in mesh units (cells).
//
// Fixed-point CIC: f_q = rint(offset * 2^15) (round half to even); f_q = 2^15 moves the base
// cell up by one with f_q = 0. Axis weights (2^15 - f_q, f_q); corner weight = their product
// (scale 2^45), accumulated with 64-bit integer atomics, so the mesh is independent of the
// order in which particles arrive. The gather uses the same weights divided by 2^45.
#include "colapm_internal.h"
#include "launch_cache.h"

namespace colapm {

namespace {

constexpr int QONE = 1 << 15;

struct Cic {
    int x0, y0, z0, x1, y1, z1;
    int fx, fy, fz;
};

__device__ __forceinline__ Cic cic_setup(float4 P, int nm) {
    const unsigned c = __float_as_uint(P.w);
    const unsigned unm = (unsigned)nm;
    int cx = (int)(c % unm), cy = (int)((c / unm) % unm), cz = (int)((c / (unm * unm)) % unm);
    int fx = __float2int_rn(P.x * 32768.0f), fy = __float2int_rn(P.y * 32768.0f), fz = __float2int_rn(P.z * 32768.0f);
    if (fx == QONE) { fx = 0; cx = cx + 1 == nm ? 0 : cx + 1; }
    if (fy == QONE) { fy = 0; cy = cy + 1 == nm ? 0 : cy + 1; }
    if (fz == QONE) { fz = 0; cz = cz + 1 == nm ? 0 : cz + 1; }
    Cic r;
    r.x0 = cx; r.y0 = cy; r.z0 = cz;
    r.x1 = cx + 1 == nm ? 0 : cx + 1;
    r.y1 = cy + 1 == nm ? 0 : cy + 1;
    r.z1 = cz + 1 == nm ? 0 : cz + 1;
    r.fx = fx; r.fy = fy; r.fz = fz;
    return r;
}

// Two threads per particle, one per x corner (lane parity): the atomics of one warp instruction then
// hit 16 particles x 2 neighbouring cells, which along the Lagrangian x rows are runs of consecutive
// int64 cells (fully used 32-byte sectors), instead of every other cell of twice as many sectors.
__device__ __forceinline__ void deposit_corner(const float4* __restrict__ pos, size_t p, int dx, int nm,
                                               unsigned long long* __restrict__ rho) {
    const Cic c = cic_setup(pos[p], nm);
    const unsigned long long wx = (unsigned long long)(dx ? c.fx : QONE - c.fx);
    const unsigned long long wy[2] = {(unsigned long long)(QONE - c.fy), (unsigned long long)c.fy};
    const unsigned long long wz[2] = {(unsigned long long)(QONE - c.fz), (unsigned long long)c.fz};
    const int x = dx ? c.x1 : c.x0, ys[2] = {c.y0, c.y1}, zs[2] = {c.z0, c.z1};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const unsigned long long w = wx * wy[dy] * wz[dz];
            if (w) atomicAdd(rho + ((size_t)zs[dz] * nm + ys[dy]) * nm + x, w);
        }
}

__global__ void k_deposit(const float4* __restrict__ pos, size_t np3, int nm, unsigned long long* __restrict__ rho) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t p = t >> 1;
    if (p >= np3) return;
    deposit_corner(pos, p, (int)(t & 1), nm, rho);
}

// Tiled deposit of particles ordered by tile (a sort with the same tile shape): a CTA takes the
// particles that were in tile (x0 .. x0 + TX - 1, y0 .. + T - 1, z0 .. + T - 1) at the last sort
// and adds their corners that fall in the tile or its +1 halo (TX + 1) x (T + 1) x (T + 1) into
// shared memory with 64-bit shared atomics; corners of particles that have moved further since
// go straight to the mesh. The region is then added to the mesh cell by cell (consecutive x per
// warp, zeros skipped), so where several particles share cells one global atomic serves them all.
// Integer sums: the mesh is the same, bit for bit, as the one-atomic-per-corner deposit.
constexpr int DT_T = 256;

template <int TS>
__global__ void __launch_bounds__(DT_T) k_deposit_tiles(const float4* __restrict__ pos, int nm, int xs,
                                                        const unsigned* __restrict__ ends, unsigned ntiles,
                                                        unsigned long long* __restrict__ rho) {
    constexpr int T = 1 << TS, RY = T + 1, RXMAX = 65;
    __shared__ unsigned long long acc[RXMAX * RY * RY];
    const int RX = (1 << xs) + 1, NR = RX * RY * RY;
    const int nbx = nm >> xs, nty = nm >> TS;
    for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = (int)(tile % (unsigned)nbx), ty = (int)((tile / (unsigned)nbx) % (unsigned)nty),
                  tz = (int)(tile / ((unsigned)nbx * (unsigned)nty));
        const int x0 = tx << xs, y0 = ty << TS, z0 = tz << TS;
        const size_t b0 = (size_t)tile << (2 * TS);
        const size_t start = tile == 0 ? 0 : ends[b0 - 1], end = ends[b0 + ((size_t)1 << (2 * TS)) - 1];
        for (int i = threadIdx.x; i < NR; i += DT_T) acc[i] = 0ull;
        __syncthreads();
        for (size_t slot = start * 2 + threadIdx.x; slot < end * 2; slot += DT_T) {
            const size_t p = slot >> 1;
            const int dx = (int)(slot & 1);
            const Cic c = cic_setup(pos[p], nm);
            const unsigned long long wx = (unsigned long long)(dx ? c.fx : QONE - c.fx);
            const unsigned long long wy[2] = {(unsigned long long)(QONE - c.fy), (unsigned long long)c.fy};
            const unsigned long long wz[2] = {(unsigned long long)(QONE - c.fz), (unsigned long long)c.fz};
            const int x = dx ? c.x1 : c.x0, ys[2] = {c.y0, c.y1}, zs[2] = {c.z0, c.z1};
            int rx = x - x0;
            if (rx < 0) rx += nm;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const unsigned long long w = wx * wy[dy] * wz[dz];
                    if (!w) continue;
                    int ry = ys[dy] - y0, rz = zs[dz] - z0;
                    if (ry < 0) ry += nm;
                    if (rz < 0) rz += nm;
                    if (rx < RX && ry < RY && rz < RY)
                        atomicAdd(&acc[(rz * RY + ry) * RX + rx], w);
                    else
                        atomicAdd(rho + ((size_t)zs[dz] * nm + ys[dy]) * nm + x, w);
                }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NR; i += DT_T) {
            const unsigned long long v = acc[i];
            if (!v) continue;
            const int rx = i % RX, ry = (i / RX) % RY, rz = i / (RX * RY);
            int gx = x0 + rx, gy = y0 + ry, gz = z0 + rz;
            if (gx >= nm) gx -= nm;
            if (gy >= nm) gy -= nm;
            if (gz >= nm) gz -= nm;
            atomicAdd(rho + ((size_t)gz * nm + gy) * nm + gx, v);
        }
        __syncthreads();   // the region is read before the next tile clears it
    }
}

// Records the images of one particle that leave the past lightcone during the drift (§6): the image
// x + R L (R in the step's replicate list) leaves when R_p <= R_L at a_i and R_p > R_L at a_{i+1};
// its exit time interpolates both radii linearly (Eq. eq:lightconeinterp) and it is written at the
// position the drift gives at a_L, with the residual momentum of the step plus the LPT frame momentum
// at a_L (the host fills zeros for the LPT columns of plain PM). Units: Mpc/h.
__device__ __forceinline__ void record_lightcone(const LightconeStep& lc, const int* cell, const float* off,
                                                 const float* d, const float* v, const float* s1, const float* s2,
                                                 size_t p) {
    float xi[3], xn[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        xi[j] = ((float)cell[j] + off[j]) * lc.cell;
        xn[j] = xi[j] + d[j] * lc.cell;   // unwrapped: the image's path is continuous within the step
    }
    const float o[3] = {lc.ox, lc.oy, lc.oz};
    for (int r = 0; r < lc.nrep; ++r) {
        float q0 = 0.0f, q1 = 0.0f, sh[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            sh[j] = (float)lc.reps[3 * r + j] * lc.box - o[j];
            const float u0 = xi[j] + sh[j], u1 = xn[j] + sh[j];
            q0 = fmaf(u0, u0, q0);
            q1 = fmaf(u1, u1, q1);
        }
        const float rp0 = sqrtf(q0), rp1 = sqrtf(q1);
        if (!(rp0 <= lc.rl0 && rp1 > lc.rl1)) continue;
        const float aL = lc.a0 + lc.da * (lc.rl0 - rp0) / ((rp1 - rp0) - (lc.rl1 - lc.rl0));
        float f = (aL - lc.a0) / lc.da * (float)(lc.K - 1);
        f = fminf(fmaxf(f, 0.0f), (float)(lc.K - 1));
        const int k = min((int)f, lc.K - 2);
        const float w = f - (float)k;
        float c[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) c[m] = fmaf(w, lc.tab[5 * (k + 1) + m] - lc.tab[5 * k + m], lc.tab[5 * k + m]);
        float x[3], pm[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            x[j] = xi[j] + sh[j] + o[j] + lc.cell * fmaf(c[0], v[j], fmaf(c[1], s1[j], c[2] * s2[j]));
            pm[j] = lc.cell * fmaf(c[3], s1[j], fmaf(c[4], s2[j], v[j]));
        }
        const unsigned long long slot = atomicAdd(lc.count, 1ull);
        if (slot < lc.capacity) {
            const int id = lc.id ? lc.id[p] : (int)p;
            lc.out[2 * slot] = make_float4(x[0], x[1], x[2], aL);
            lc.out[2 * slot + 1] = make_float4(pm[0], pm[1], pm[2], __int_as_float(id));
        }
    }
}

template <bool LC>
__device__ __forceinline__ void gather_kick_drift(float4* __restrict__ pos, float* __restrict__ mom,
                                                  const float* __restrict__ psi1, const float* __restrict__ psi2,
                                                  const float* __restrict__ force, size_t np3, int nm, const StepCoef& k,
                                                  int drift, const LightconeStep& lc, size_t p) {
    // every load of the particle's own data is issued before the force loads that depend on its
    // position, so the two sets are in flight together (streaming: each is used once per step)
    const float4 P = __ldcs(pos + p);
    float s1[3], s2[3], v[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        s1[j] = __ldcs(psi1 + j * np3 + p);
        s2[j] = __ldcs(psi2 + j * np3 + p);
        v[j] = __ldcs(mom + j * np3 + p);
    }
    const Cic c = cic_setup(P, nm);
    const float s = 1.0f / 32768.0f;
    const float wx[2] = {(QONE - c.fx) * s, c.fx * s};
    const float wy[2] = {(QONE - c.fy) * s, c.fy * s};
    const float wz[2] = {(QONE - c.fz) * s, c.fz * s};
    const int xs[2] = {c.x0, c.x1}, ys[2] = {c.y0, c.y1}, zs[2] = {c.z0, c.z1};
    const size_t m3 = (size_t)nm * nm * nm;
    float f[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const size_t row = ((size_t)zs[dz] * nm + ys[dy]) * nm;
            const float wyz = wy[dy] * wz[dz];
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float w = wx[dx] * wyz;
                const size_t i = row + xs[dx];
#pragma unroll
                for (int j = 0; j < 3; ++j) f[j] = fmaf(w, __ldg(force + j * m3 + i), f[j]);
            }
        }
    float d[3];
    const float off[3] = {P.x, P.y, P.z};
    int cell[3] = {(int)(__float_as_uint(P.w) % (unsigned)nm), (int)((__float_as_uint(P.w) / (unsigned)nm) % (unsigned)nm),
                   (int)((__float_as_uint(P.w) / ((unsigned)nm * (unsigned)nm)) % (unsigned)nm)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // kick (Eq. eq:vcola): p += K [F - D1 Psi1 - (D2 - D1^2) Psi2]
        v[j] = fmaf(k.kick, f[j] - k.c1 * s1[j] - k.c2 * s2[j], v[j]);
        __stcs(mom + j * np3 + p, v[j]);
        // drift (Eq. eq:rcola): x += S p + dD1 Psi1 + dD2 Psi2
        d[j] = drift ? fmaf(k.drift, v[j], fmaf(k.e1, s1[j], k.e2 * s2[j])) : 0.0f;
    }
    if (!drift) return;
    if constexpr (LC) record_lightcone(lc, cell, off, d, v, s1, s2, p);
    float o[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float u = off[j] + d[j];
        float fl = floorf(u);
        float r = u - fl;
        if (r >= 1.0f) { r = 0.0f; fl += 1.0f; }
        int cc = (cell[j] + (int)fl) % nm;
        if (cc < 0) cc += nm;
        cell[j] = cc;
        o[j] = r;
    }
    const unsigned lin = (unsigned)cell[0] + (unsigned)nm * ((unsigned)cell[1] + (unsigned)nm * (unsigned)cell[2]);
    __stcs(pos + p, make_float4(o[0], o[1], o[2], __uint_as_float(lin)));
}

template <bool LC>
__global__ void k_gather_kick_drift(float4* __restrict__ pos, float* __restrict__ mom, const float* __restrict__ psi1,
                                    const float* __restrict__ psi2, const float* __restrict__ force, size_t np3, int nm,
                                    StepCoef k, int drift, LightconeStep lc) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    gather_kick_drift<LC>(pos, mom, psi1, psi2, force, np3, nm, k, drift, lc, p);
}

// ---------------------------------------------------------------------------------------------
// Multi-mock particle kernels: one persistent launch for the particles of many mocks (any mix of
// sizes). The work items are chunks of MW_ITEM particles, numbered mock after mock (w[m].first is
// mock m's first item). Each CTA takes the next item from a ticket counter, finds its mock by
// binary search over the `first` column, and runs the single-mock code on that chunk, until the
// tickets run out. The last CTA to leave resets the counter for the next launch (queue[1] counts
// the CTAs that left), so a captured graph can replay the launch without a memset. There is no
// wait of any kind: a CTA only ever takes tickets.
constexpr int MW_ITEM = 256;
constexpr int MW_T = 256;

__device__ __forceinline__ bool next_item(const MockWork* __restrict__ w, int nmock, long long nitems,
                                          unsigned long long* queue, long long& item, int& mock) {
    __shared__ long long s_item;
    __shared__ int s_mock;
    __syncthreads();   // the previous item's values are no longer read
    if (threadIdx.x == 0) {
        const long long it = (long long)atomicAdd(queue, 1ull);
        int lo = 0, hi = nmock - 1;
        while (lo < hi) {   // last mock whose first item is <= it
            const int mid = (lo + hi + 1) >> 1;
            if (w[mid].first <= it) lo = mid; else hi = mid - 1;
        }
        s_item = it;
        s_mock = lo;
    }
    __syncthreads();
    item = s_item;
    mock = s_mock;
    return item < nitems;
}

__device__ __forceinline__ void leave_queue(unsigned long long* queue) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
            queue[0] = 0ull;
            queue[1] = 0ull;
            __threadfence();
        }
    }
}

__global__ void __launch_bounds__(MW_T) k_multi_deposit(const MockWork* __restrict__ w, int nmock, long long nitems,
                                                        unsigned long long* queue) {
    long long item;
    int m;
    while (next_item(w, nmock, nitems, queue, item, m)) {
        const MockWork& mw = w[m];
        const size_t base = (size_t)(item - mw.first) * MW_ITEM;
#pragma unroll
        for (int h = 0; h < 2 * MW_ITEM / MW_T; ++h) {   // two threads per particle, one per x corner
            const int slot = h * MW_T + threadIdx.x;
            const size_t p = base + (slot >> 1);
            if (p < mw.np3) deposit_corner(mw.pos, p, slot & 1, mw.nm, mw.rho);
        }
    }
    leave_queue(queue);
}

__global__ void __launch_bounds__(MW_T) k_multi_gather_kick_drift(const MockWork* __restrict__ w, int nmock,
                                                                  long long nitems, unsigned long long* queue) {
    long long item;
    int m;
    while (next_item(w, nmock, nitems, queue, item, m)) {
        const MockWork& mw = w[m];
        const size_t base = (size_t)(item - mw.first) * MW_ITEM;
#pragma unroll
        for (int h = 0; h < MW_ITEM / MW_T; ++h) {
            const size_t p = base + h * MW_T + threadIdx.x;
            if (p < mw.np3)
                gather_kick_drift<false>(mw.pos, mw.mom, mw.psi1, mw.psi2, mw.force, mw.np3, mw.nm, mw.k, 1,
                                         LightconeStep{}, p);
        }
    }
    leave_queue(queue);
}

// Site i of the Lagrangian lattice sits at mesh coordinate i nm / np + 1/2 (spacing L / np, offset by
// half a PM cell). Integer part of i nm / np and its exact fractional remainder (0 when np divides nm;
// a multiple of nm / np otherwise, i.e. of 1/2 or 1/4 for the coarse meshes).
__device__ __forceinline__ void lattice_site(int i, int np, int nm, int& base, float& frac) {
    const int t = i * nm;   // < 2^20 for the supported sizes (np, nm <= 1024): 32-bit division
    base = t / np;
    frac = (float)(t % np) / (float)np;
}

// Particles on the Lagrangian lattice (offset by half a PM cell), displaced by D1 Psi1 + D2 Psi2.
// psi1 / psi2 arrive in IC-grid cells and leave in PM-mesh cells (factor to_mesh = Nm / Np).
__global__ void k_init_particles(float4* __restrict__ pos, float* __restrict__ mom, float* __restrict__ psi1,
                                 float* __restrict__ psi2, int np, int nm, float to_mesh, float d1, float d2, float p1,
                                 float p2, int cola) {
    const size_t np3 = (size_t)np * np * np;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const unsigned up = (unsigned)p, unp = (unsigned)np;   // np^3 <= 2^30: 32-bit divisions
    const int site[3] = {(int)(up % unp), (int)((up / unp) % unp), (int)(up / (unp * unp))};
    int cell[3];
    float o[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float s1 = psi1[j * np3 + p] * to_mesh, s2 = psi2[j * np3 + p] * to_mesh;
        psi1[j * np3 + p] = s1;
        psi2[j * np3 + p] = s2;
        int base;
        float frac;
        lattice_site(site[j], np, nm, base, frac);
        const float u = (0.5f + frac) + fmaf(d1, s1, d2 * s2);
        float fl = floorf(u);
        float r = u - fl;
        if (r >= 1.0f) { r = 0.0f; fl += 1.0f; }
        int cc = (base + (int)fl) % nm;
        if (cc < 0) cc += nm;
        cell[j] = cc;
        o[j] = r;
        mom[j * np3 + p] = cola ? 0.0f : fmaf(p1, s1, p2 * s2);
    }
    const unsigned lin = (unsigned)cell[0] + (unsigned)nm * ((unsigned)cell[1] + (unsigned)nm * (unsigned)cell[2]);
    pos[p] = make_float4(o[0], o[1], o[2], __uint_as_float(lin));
}

__global__ void k_add_lpt_momentum(float* __restrict__ mom, const float* __restrict__ psi1, const float* __restrict__ psi2,
                                   size_t n3, float p1, float p2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    mom[i] = fmaf(p1, psi1[i], fmaf(p2, psi2[i], mom[i]));
}

__global__ void k_export_particles(const float4* __restrict__ pos, const float* __restrict__ mom,
                                   const int* __restrict__ id, size_t np3, int nm, float cell,
                                   float* __restrict__ pos_xyz, float* __restrict__ mom_xyz) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const size_t q = id ? (size_t)id[p] : p;   // the particle's id: its place in the output
    if (pos_xyz) {
        const float4 P = pos[p];
        const unsigned c = __float_as_uint(P.w), u = (unsigned)nm;
        const unsigned cx = c % u, cy = (c / u) % u, cz = c / (u * u);
        pos_xyz[3 * q + 0] = ((float)cx + P.x) * cell;
        pos_xyz[3 * q + 1] = ((float)cy + P.y) * cell;
        pos_xyz[3 * q + 2] = ((float)cz + P.z) * cell;
    }
    if (mom_xyz) {
#pragma unroll
        for (int j = 0; j < 3; ++j) mom_xyz[3 * q + j] = mom[j * np3 + p] * cell;
    }
}

__global__ void k_export_state(const float4* __restrict__ pos, const float* __restrict__ mom, size_t np3, int nm,
                               int* __restrict__ cell_xyz, float* __restrict__ off_xyz, float* __restrict__ mom_xyz) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const float4 P = pos[p];
    if (cell_xyz) {
        const unsigned c = __float_as_uint(P.w), u = (unsigned)nm;
        cell_xyz[3 * p + 0] = (int)(c % u);
        cell_xyz[3 * p + 1] = (int)((c / u) % u);
        cell_xyz[3 * p + 2] = (int)(c / (u * u));
    }
    if (off_xyz) {
        off_xyz[3 * p + 0] = P.x;
        off_xyz[3 * p + 1] = P.y;
        off_xyz[3 * p + 2] = P.z;
    }
    if (mom_xyz) {
#pragma unroll
        for (int j = 0; j < 3; ++j) mom_xyz[3 * p + j] = mom[j * np3 + p];
    }
}

__global__ void k_import_state(float4* __restrict__ pos, float* __restrict__ mom, size_t np3, int nm,
                               const int* __restrict__ cell_xyz, const float* __restrict__ off_xyz,
                               const float* __restrict__ mom_xyz, int* err) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    if (cell_xyz && off_xyz) {
        int c[3];
        float o[3];
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c[j] = cell_xyz[3 * p + j];
            o[j] = off_xyz[3 * p + j];
            bad |= !(c[j] >= 0 && c[j] < nm && o[j] >= 0.0f && o[j] < 1.0f);
        }
        if (bad) {
            atomicOr(err, 2);
            return;
        }
        const unsigned lin = (unsigned)c[0] + (unsigned)nm * ((unsigned)c[1] + (unsigned)nm * (unsigned)c[2]);
        pos[p] = make_float4(o[0], o[1], o[2], __uint_as_float(lin));
    }
    if (mom_xyz) {
#pragma unroll
        for (int j = 0; j < 3; ++j) mom[j * np3 + p] = mom_xyz[3 * p + j];
    }
}

// Psi = x - q in Mpc/h with the minimum-image convention, q = (site * Nm/Np + 1/2) cells.
__global__ void k_export_displacement(const float4* __restrict__ pos, int np, int nm, float cell,
                                      float* __restrict__ psi) {
    const size_t np3 = (size_t)np * np * np;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const float4 P = pos[p];
    const unsigned c = __float_as_uint(P.w), u = (unsigned)nm;
    const int cc[3] = {(int)(c % u), (int)((c / u) % u), (int)(c / (u * u))};
    const unsigned up = (unsigned)p, unp = (unsigned)np;   // np^3 <= 2^30: 32-bit divisions
    const int site[3] = {(int)(up % unp), (int)((up / unp) % unp), (int)(up / (unp * unp))};
    const float off[3] = {P.x, P.y, P.z};
    const int h = nm / 2;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        int base;
        float frac;
        lattice_site(site[j], np, nm, base, frac);
        int di = cc[j] - base;
        di += di < -h ? nm : (di >= h ? -nm : 0);
        float d = (float)di + (off[j] - (0.5f + frac));
        d += d < -(float)h ? (float)nm : (d >= (float)h ? -(float)nm : 0.0f);
        psi[3 * p + j] = d * cell;
    }
}

// x = q + Psi (Psi in Mpc/h, xyz-interleaved); momenta are left alone.
__global__ void k_import_displacement(float4* __restrict__ pos, int np, int nm, float to_mesh,
                                      const float* __restrict__ psi, int* err) {
    const size_t np3 = (size_t)np * np * np;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const unsigned up = (unsigned)p, unp = (unsigned)np;   // np^3 <= 2^30: 32-bit divisions
    const int site[3] = {(int)(up % unp), (int)((up / unp) % unp), (int)(up / (unp * unp))};
    int cell[3];
    float o[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float s = psi[3 * p + j] * to_mesh;
        if (!(fabsf(s) < (float)nm)) {
            atomicOr(err, 2);
            return;
        }
        int base;
        float frac;
        lattice_site(site[j], np, nm, base, frac);
        const float u = (0.5f + frac) + s;
        float fl = floorf(u);
        float r = u - fl;
        if (r >= 1.0f) { r = 0.0f; fl += 1.0f; }
        int cc = (base + (int)fl) % nm;
        if (cc < 0) cc += nm;
        cell[j] = cc;
        o[j] = r;
    }
    const unsigned lin = (unsigned)cell[0] + (unsigned)nm * ((unsigned)cell[1] + (unsigned)nm * (unsigned)cell[2]);
    pos[p] = make_float4(o[0], o[1], o[2], __uint_as_float(lin));
}

// Redshift-space positions (§7.1): each particle moves by s_los = v_los / (a H) along the line of
// sight. With momenta p in mesh units (the total momentum after finalisation) and H0 = 1, v = p / a and
// H = E(a), so the shift in cells is p_los / (a^2 E) = p_los * scale. los < 0: radial from the box
// centre (mesh coordinate nm/2 on every axis); los = 0, 1, 2: along that axis. The shift is added to
// the offset and the cell renormalised with the periodic wrap, as in the drift.
__global__ void k_rsd_positions(const float4* __restrict__ pos, const float* __restrict__ mom, size_t np3, int nm,
                                float scale, int los, float4* __restrict__ out) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np3) return;
    const float4 P = pos[p];
    const unsigned c = __float_as_uint(P.w), u = (unsigned)nm;
    int cell[3] = {(int)(c % u), (int)((c / u) % u), (int)(c / (u * u))};
    const float off[3] = {P.x, P.y, P.z};
    const float v[3] = {mom[p], mom[np3 + p], mom[2 * np3 + p]};
    float d[3] = {0.0f, 0.0f, 0.0f};
    if (los < 0) {
        float r[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) r[j] = (float)(cell[j] - nm / 2) + off[j];   // exact integer part
        const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        if (rr > 0.0f) {
            const float inv = rsqrtf(rr);
            const float vl = (v[0] * r[0] + v[1] * r[1] + v[2] * r[2]) * inv * scale;
#pragma unroll
            for (int j = 0; j < 3; ++j) d[j] = vl * r[j] * inv;
        }
    } else {
        d[los] = v[los] * scale;
    }
    float o[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float w = off[j] + d[j];
        float fl = floorf(w);
        float rem = w - fl;
        if (rem >= 1.0f) { rem = 0.0f; fl += 1.0f; }
        int cc = (cell[j] + (int)fl) % nm;
        if (cc < 0) cc += nm;
        cell[j] = cc;
        o[j] = rem;
    }
    const unsigned lin = (unsigned)cell[0] + u * ((unsigned)cell[1] + u * (unsigned)cell[2]);
    out[p] = make_float4(o[0], o[1], o[2], __uint_as_float(lin));
}

__global__ void k_scale(float* __restrict__ dst, const float* __restrict__ src, size_t n, float f) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] * f;
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_deposit(const float4* pos, size_t np3, int nm, unsigned long long* rho, cudaStream_t s, int block) {
    k_deposit<<<blocks(2 * np3, block), block, 0, s>>>(pos, np3, nm, rho);
    return cudaGetLastError();
}

cudaError_t launch_gather_kick_drift(float4* pos, float* mom, const float* psi1, const float* psi2, const float* force,
                                     size_t np3, int nm, StepCoef c, int drift, cudaStream_t s, int block,
                                     const LightconeStep* lc) {
    if (lc && drift)
        k_gather_kick_drift<true><<<blocks(np3, block), block, 0, s>>>(pos, mom, psi1, psi2, force, np3, nm, c, drift, *lc);
    else
        k_gather_kick_drift<false><<<blocks(np3, block), block, 0, s>>>(pos, mom, psi1, psi2, force, np3, nm, c, drift,
                                                                        LightconeStep{});
    return cudaGetLastError();
}

cudaError_t launch_deposit_tiles(const float4* pos, int nm, int tshift, const unsigned* ends, unsigned long long* rho,
                                 cudaStream_t s) {
    const int xs = sort_xshift(nm);
    if (!sort_tshift_ok(nm, tshift) || tshift < 1 || xs > 6) return cudaErrorInvalidValue;
    const unsigned ntiles = (unsigned)((size_t)(nm >> tshift) * (nm >> tshift) * (nm >> xs));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)sms * 8u < ntiles ? (unsigned)sms * 8u : ntiles;
    switch (tshift) {
        case 1: k_deposit_tiles<1><<<grid, DT_T, 0, s>>>(pos, nm, xs, ends, ntiles, rho); break;
        case 2: k_deposit_tiles<2><<<grid, DT_T, 0, s>>>(pos, nm, xs, ends, ntiles, rho); break;
        default: k_deposit_tiles<3><<<grid, DT_T, 0, s>>>(pos, nm, xs, ends, ntiles, rho); break;
    }
    return cudaGetLastError();
}

long long multi_items(size_t np3) { return (long long)((np3 + MW_ITEM - 1) / MW_ITEM); }

cudaError_t launch_multi_deposit(const MockWork* w, int nmock, long long nitems, unsigned long long* queue,
                                 cudaStream_t s) {
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_multi_deposit, MW_T, 0, &grid);
    if (e != cudaSuccess) return e;
    if (nitems < 1 || nmock < 1) return cudaSuccess;
    k_multi_deposit<<<nitems < grid ? (int)nitems : grid, MW_T, 0, s>>>(w, nmock, nitems, queue);
    return cudaGetLastError();
}

cudaError_t launch_multi_gather_kick_drift(const MockWork* w, int nmock, long long nitems, unsigned long long* queue,
                                           cudaStream_t s) {
    static GridCache cache;
    int grid = 0;
    cudaError_t e = cached_grid(cache, k_multi_gather_kick_drift, MW_T, 0, &grid);
    if (e != cudaSuccess) return e;
    if (nitems < 1 || nmock < 1) return cudaSuccess;
    k_multi_gather_kick_drift<<<nitems < grid ? (int)nitems : grid, MW_T, 0, s>>>(w, nmock, nitems, queue);
    return cudaGetLastError();
}

cudaError_t launch_init_particles(float4* pos, float* mom, float* psi1, float* psi2, int np, int nm, float to_mesh,
                                  float d1, float d2, float p1, float p2, int cola, cudaStream_t s) {
    const size_t np3 = (size_t)np * np * np;
    k_init_particles<<<blocks(np3, 256), 256, 0, s>>>(pos, mom, psi1, psi2, np, nm, to_mesh, d1, d2, p1, p2, cola);
    return cudaGetLastError();
}

cudaError_t launch_add_lpt_momentum(float* mom, const float* psi1, const float* psi2, size_t np3, float p1, float p2,
                                    cudaStream_t s) {
    k_add_lpt_momentum<<<blocks(3 * np3, 256), 256, 0, s>>>(mom, psi1, psi2, 3 * np3, p1, p2);
    return cudaGetLastError();
}

cudaError_t launch_export_particles(const float4* pos, const float* mom, const int* id, size_t np3, int nm, float cell,
                                    float* pos_xyz, float* mom_xyz, cudaStream_t s) {
    k_export_particles<<<blocks(np3, 256), 256, 0, s>>>(pos, mom, id, np3, nm, cell, pos_xyz, mom_xyz);
    return cudaGetLastError();
}

cudaError_t launch_export_state(const float4* pos, const float* mom, size_t np3, int nm, int* cell_xyz, float* off_xyz,
                                float* mom_xyz, cudaStream_t s) {
    k_export_state<<<blocks(np3, 256), 256, 0, s>>>(pos, mom, np3, nm, cell_xyz, off_xyz, mom_xyz);
    return cudaGetLastError();
}

cudaError_t launch_import_state(float4* pos, float* mom, size_t np3, int nm, const int* cell_xyz, const float* off_xyz,
                                const float* mom_xyz, int* err, cudaStream_t s) {
    k_import_state<<<blocks(np3, 256), 256, 0, s>>>(pos, mom, np3, nm, cell_xyz, off_xyz, mom_xyz, err);
    return cudaGetLastError();
}

cudaError_t launch_export_displacement(const float4* pos, int np, int nm, float cell, float* psi, cudaStream_t s) {
    const size_t np3 = (size_t)np * np * np;
    k_export_displacement<<<blocks(np3, 256), 256, 0, s>>>(pos, np, nm, cell, psi);
    return cudaGetLastError();
}

cudaError_t launch_import_displacement(float4* pos, int np, int nm, float to_mesh, const float* psi, int* err,
                                       cudaStream_t s) {
    const size_t np3 = (size_t)np * np * np;
    k_import_displacement<<<blocks(np3, 256), 256, 0, s>>>(pos, np, nm, to_mesh, psi, err);
    return cudaGetLastError();
}

cudaError_t launch_rsd_positions(const float4* pos, const float* mom, size_t np3, int nm, float scale, int los,
                                 float4* out, cudaStream_t s) {
    k_rsd_positions<<<blocks(np3, 256), 256, 0, s>>>(pos, mom, np3, nm, scale, los, out);
    return cudaGetLastError();
}

cudaError_t launch_scale(float* dst, const float* src, size_t n, float f, cudaStream_t s) {
    k_scale<<<blocks(n, 256), 256, 0, s>>>(dst, src, n, f);
    return cudaGetLastError();
}

}  // namespace colapm
