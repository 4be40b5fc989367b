// C ABI of libcolapm.so (declared in include/colapm.h): context, initial conditions, the
// COLA / PM step loop, finalisation, power spectrum, state I/O and phase timing.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "colapm_internal.h"
#include "cosmology.h"

using namespace colapm;

struct colapm_ctx {
    colapm_params prm{};
    cudaStream_t stream = nullptr;
    int np = 0, nm = 0;
    size_t np3 = 0, nm3 = 0;
    StepTable table;
    // device buffers
    unsigned long long* rho = nullptr;   // nm^3 int64 fixed-point density
    float* F = nullptr;                  // 3 nm^3: density spectrum, then the three force meshes
    float* Freal = nullptr;              // 3 nm^3: the real force meshes when the spectra use the blocked layout
    float4* pos = nullptr;               // np^3 (offsets, cell bits)
    float* mom = nullptr;                // 3 np^3, cells
    float* psi1 = nullptr;               // 3 np^3, cells
    float* psi2 = nullptr;               // 3 np^3, cells
    float* scratch = nullptr;            // 9 np^3 (IC spectra and phi_ij; staging for state I/O)
    int* id = nullptr;                   // np^3: particle id of each slot of pos, mom, psi1, psi2
    float4* pos_alt = nullptr;           // second set of particle arrays: the target of a reordering
    float* mom_alt = nullptr;
    float* psi1_alt = nullptr;
    float* psi2_alt = nullptr;
    int* id_alt = nullptr;
    unsigned* sort_cnt = nullptr;        // bucket counters / cursors of the cell sort
    unsigned* sort_tile = nullptr;       // their tile sums
    int sort_every = 0;                  // reorder by cell every k steps from step sort_first (0: never)
    int sort_first = 0;
    int key_tshift = 0;                  // sort key: tiles of 64 x 2^t x 2^t cells (0: rows of 64)
    bool dep_tiled = false;              // tiled deposit while the particles are in tile order
    int sorted_tshift = -1;              // tile shift of the order the particles are in (-1: id order)
    double fnl = 0.0;                    // local primordial non-Gaussianity of the next ICs
    float* fnl_tab = nullptr;            // per |n|^2 of the IC grid: 1 / (M N^3), then M (colapm_set_fnl)
    double* fnl_sum = nullptr;           // FP64 sum of phi^2
    // past lightcone (colapm_set_lightcone)
    bool lc_on = false;
    colapm_lightcone lc{};
    int lc_first = 0;                    // first step that records
    float4* lc_out = nullptr;            // 2 float4 per output row
    unsigned long long* lc_count = nullptr;
    unsigned long long lc_cap = 0;
    float* lc_tab = nullptr;             // per step: kLcK x 5 coefficient samples
    int* lc_reps = nullptr;              // per step: its replicate vectors, concatenated
    std::vector<int> lc_rep_off, lc_rep_n;
    std::vector<float> lc_rl;            // lightcone radius at every step boundary
    bool id_order = true;                // slots hold the particles in id order
    float* xfer = nullptr;               // 6 np^3: staging of the asynchronous catalogue copy (lazy)
    cudaStream_t xfer_stream = nullptr;  // its copy stream
    cudaEvent_t xfer_ready = nullptr, xfer_done = nullptr;
    bool xfer_pending = false;           // a copy out of xfer may still be running
    float2* tw_m = nullptr;              // exp(-2 pi i t / nm)
    float2* tw_p = nullptr;              // exp(-2 pi i t / np)
    float* sinc2_m = nullptr;            // sinc^2(pi n / nm) per FFT bin, then nm ones (no window)
    float* amp_p = nullptr;              // Gaussian-field amplitude per integer |n|^2 of the IC grid
    int* err = nullptr;                  // device error bits: 1 overflow, 2 bad state import, 4 wait timeout,
                                         // 8 internal (a sort slot out of range)
    // power-spectrum tables (grown on demand)
    int* pw_bin = nullptr;               // |n|^2 thresholds of the bins
    double* pw_acc = nullptr;            // ksum[nb], psum[nb], cnt[nb] (as u64)
    int pw_n2cap = 0, pw_nbcap = 0;
    float pw_lga = 0.0f, pw_lgb = 0.0f;  // log-spacing guess of the bins (PowerArgs)
    unsigned long long* d_seed = nullptr;          // device seed of the Gaussian field
    const unsigned long long* seed_src = nullptr;  // the seed the ICs read (own, or a batch slot)
    unsigned plan = COLAPM_PLAN_ALL;     // passes on the two-stage register FFT, else Stockham (autotuned)
    int fused = 0;                       // fused x-y passes where supported: bit 0 forward, bit 1 inverse (autotuned)
    bool rho_clean = false;              // rho is all zero (the forward x pass clears it as it reads)
    int phase_mute = 0;                  // > 0: phases nested in another phase are not timed
    float2* xy_ring = nullptr;           // L2-resident ring of intermediate planes of the fused passes
    int* xy_ctr = nullptr;               // their work ticket and per-plane completion counters
    int block = 256;                     // particle-kernel block size (autotuned)
    int step = 0;
    long long launches = 0;              // kernels launched by this context
    bool has_ics = false, finalized = false;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[COLAPM_PHASE_COUNT];
};

namespace {

constexpr int kMeshSizes[] = {16, 32, 64, 96, 128, 160, 192, 256, 320, 384, 512, 1024};

bool supported_size(int n) {
    for (int s : kMeshSizes)
        if (s == n) return true;
    return false;
}

#define CK(call)                                \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return COLAPM_E_CUDA; \
    } while (0)

#define CKL(call)                               \
    do {                                        \
        ++c->launches;                          \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return COLAPM_E_CUDA; \
    } while (0)

struct Phase {   // CUDA-event bracket of one phase when timing is on
    colapm_ctx* c;
    int ph;
    cudaEvent_t b = nullptr, e = nullptr;
    Phase(colapm_ctx* ctx, int phase) : c(ctx), ph(phase) {
        if (!c->timing || c->phase_mute) return;
        if (cudaEventCreate(&b) == cudaSuccess && cudaEventCreate(&e) == cudaSuccess) cudaEventRecord(b, c->stream);
    }
    ~Phase() {
        if (!c->timing || !b || !e) return;
        cudaEventRecord(e, c->stream);
        c->ev[ph].emplace_back(b, e);
    }
};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_all(colapm_ctx* c) {
    if (c->xfer_stream) cudaStreamSynchronize(c->xfer_stream);
    void* ptrs[] = {c->rho, c->F, c->Freal, c->pos, c->mom, c->psi1, c->psi2, c->scratch, c->tw_m, c->tw_p,
                    c->sinc2_m, c->amp_p, c->err, c->pw_bin, c->pw_acc, c->d_seed, c->xy_ring, c->xy_ctr, c->xfer,
                    c->id, c->pos_alt, c->mom_alt, c->psi1_alt, c->psi2_alt, c->id_alt, c->sort_cnt, c->sort_tile,
                    c->fnl_tab, c->fnl_sum, c->lc_out, c->lc_count, c->lc_tab, c->lc_reps};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& v : c->ev)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    if (c->xfer_ready) cudaEventDestroy(c->xfer_ready);
    if (c->xfer_done) cudaEventDestroy(c->xfer_done);
    if (c->xfer_stream) cudaStreamDestroy(c->xfer_stream);
}

std::vector<float2> twiddles(int n) {
    std::vector<float2> t(n);
    for (int i = 0; i < n; ++i) {
        const double ang = 2.0 * M_PI * (double)i / n;
        t[i] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    return t;
}

int pending_error(colapm_ctx* c) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h) CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (h & 1) return COLAPM_E_OVERFLOW;
    if (h & 2) return COLAPM_E_ARG;
    if (h & 4) return COLAPM_E_TIMEOUT;
    if (h & 8) return COLAPM_E_CUDA;
    return COLAPM_OK;
}

// Copy `bytes` produced on the device (src) to a caller array that may be host or device.
int copy_out(colapm_ctx* c, void* dst, const void* src, size_t bytes) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return COLAPM_OK;
}

// Particle positions to deposit: up to two arrays (cell bits + offsets on c's mesh) whose masses add.
struct DepositSrc {
    const float4* pos[2] = {nullptr, nullptr};
    size_t n[2] = {0, 0};
};

DepositSrc own_particles(const colapm_ctx* c) {
    DepositSrc d;
    d.pos[0] = c->pos;
    d.n[0] = c->np3;
    return d;
}

// Fixed-point CIC deposit into c's mesh of the given particles (default: c's own).
// Whether the particles are reordered before step `step`: every sort_every steps from sort_first.
bool sort_due(const colapm_ctx* c, int step) {
    return c->sort_every > 0 && step > 0 && step >= c->sort_first && (step - c->sort_first) % c->sort_every == 0;
}

// Whether the own particles are ordered by the tiles of the tiled deposit (the last sort used the
// context's tile shape and nothing has restored id order since).
bool tiles_ready(const colapm_ctx* c) {
    return c->dep_tiled && c->key_tshift > 0 && !c->id_order && c->sorted_tshift == c->key_tshift;
}

int deposit(colapm_ctx* c, const DepositSrc* src = nullptr) {
    Phase ph(c, COLAPM_PHASE_DEPOSIT);
    if (!c->rho_clean) CK(cudaMemsetAsync(c->rho, 0, c->nm3 * sizeof(unsigned long long), c->stream));
    c->rho_clean = false;
    if (!src && tiles_ready(c)) {
        CKL(launch_deposit_tiles(c->pos, c->nm, c->key_tshift, c->sort_cnt, c->rho, c->stream));
        return COLAPM_OK;
    }
    const DepositSrc d = src ? *src : own_particles(c);
    for (int i = 0; i < 2; ++i)
        if (d.pos[i]) CKL(launch_deposit(d.pos[i], d.n[i], c->nm, c->rho, c->stream, c->block));
    return COLAPM_OK;
}

bool use_xy(const colapm_ctx* c, int bit) { return (c->fused & bit) && c->xy_ring != nullptr; }

// Whether pass `bit` (COLAPM_PLAN_*) runs on the two-stage register FFT (where its length has a
// two-radix plan; the launchers fall back to the Stockham plan otherwise).
bool ts(const colapm_ctx* c, unsigned bit) { return (c->plan & bit) != 0; }

// The two-stage engine keeps the half spectra in the blocked layout (see hs_index) when every pass
// runs on it and the fused x-y passes are off; the inverse x pass then writes the real force
// meshes to Freal.
bool use_blocked(const colapm_ctx* c) {
    return c->plan == COLAPM_PLAN_ALL && !(c->fused & 3) && c->Freal != nullptr;
}

// The three real force meshes of the last force computation.
const float* force_mesh(const colapm_ctx* c) { return use_blocked(c) ? c->Freal : c->F; }

SortBuffers sort_buffers(colapm_ctx* c) {
    return SortBuffers{c->pos, c->mom, c->psi1, c->psi2, c->id, c->pos_alt, c->mom_alt, c->psi1_alt, c->psi2_alt,
                       c->id_alt, c->sort_cnt, c->sort_tile, c->err};
}

void swap_particle_arrays(colapm_ctx* c) {
    std::swap(c->pos, c->pos_alt);
    std::swap(c->mom, c->mom_alt);
    std::swap(c->psi1, c->psi1_alt);
    std::swap(c->psi2, c->psi2_alt);
    std::swap(c->id, c->id_alt);
}

// Reorder the particle arrays by mesh cell (counting sort into the second set, then swap).
int sort_particles(colapm_ctx* c) {
    Phase ph(c, COLAPM_PHASE_SORT);
    CKL(launch_sort(sort_buffers(c), c->np3, c->nm, c->key_tshift, c->stream));
    swap_particle_arrays(c);
    c->id_order = false;
    c->sorted_tshift = c->key_tshift;
    return COLAPM_OK;
}

// Put the particles back in id order (for the calls that exchange particle data in id order).
int id_order(colapm_ctx* c) {
    if (c->id_order) return COLAPM_OK;
    CKL(launch_unsort(sort_buffers(c), c->np3, c->stream));
    swap_particle_arrays(c);
    c->id_order = true;
    return COLAPM_OK;
}

float density_scale(const colapm_ctx* c) {
    const double m = (double)c->nm / c->np;
    return (float)(m * m * m * std::ldexp(1.0, -45));
}

// Forward x and y passes of the current density into F (half spectrum, z still in real space).
int density_xy(colapm_ctx* c) {
    Phase ph(c, COLAPM_PHASE_FFT_FWD);
    float2* d = reinterpret_cast<float2*>(c->F);
    c->rho_clean = false;
    if (use_xy(c, 1)) {
        CKL(launch_xy_fwd(c->nm, c->rho, d, c->tw_m, density_scale(c), c->xy_ring, c->xy_ctr, c->err, c->stream, true));
        c->rho_clean = true;
        return COLAPM_OK;
    }
    const bool blk = use_blocked(c);
    CKL(launch_fx_fwd_i64(c->nm, c->rho, d, c->tw_m, density_scale(c), c->err, c->stream, ts(c, COLAPM_PLAN_XF), true,
                          blk));
    c->rho_clean = true;
    CKL(launch_fy(c->nm, -1, d, 0, 1, c->tw_m, c->stream, ts(c, COLAPM_PLAN_Y), blk));
    return COLAPM_OK;
}

// §2.4 steps 2-3 from the deposited density: the three real force meshes in force_mesh(c).
int force_from_density(colapm_ctx* c) {
    int r = density_xy(c);
    if (r) return r;
    float2* d = reinterpret_cast<float2*>(c->F);
    const size_t fs = c->nm3 / 2;   // complex stride between the three meshes
    {
        Phase ph(c, COLAPM_PHASE_POISSON);
        ZOut out{};
        out.p[0] = d;
        out.p[1] = d + fs;
        out.p[2] = d + 2 * fs;
        const float gnorm = (float)(1.0 / ((double)c->nm * c->nm * c->nm));
        CKL(launch_fz(c->nm, Z_FORCE, d, out, c->tw_m, c->sinc2_m, c->prm.deconv, gnorm, nullptr, c->stream,
                      ts(c, COLAPM_PLAN_Z), use_blocked(c)));
    }
    if (use_xy(c, 2)) {
        Phase ph(c, COLAPM_PHASE_FFT_INV);
        CKL(launch_xy_inv(c->nm, d, fs, 3, c->tw_m, c->xy_ring, c->xy_ctr, c->err, c->stream));
        return COLAPM_OK;
    }
    const bool blk = use_blocked(c);
    {
        Phase ph(c, COLAPM_PHASE_FFT_INV);
        if (blk) {
            CKL(launch_fy_force(c->nm, d, fs, c->tw_m, c->stream));   // bases -> three spectra
        } else {
            CKL(launch_fy(c->nm, +1, d, fs, 3, c->tw_m, c->stream, ts(c, COLAPM_PLAN_Y), blk));
        }
    }
    {
        Phase ph(c, COLAPM_PHASE_FFT_INV_X);
        CKL(launch_fx_inv(c->nm, d, fs, 3, c->tw_m, c->stream, ts(c, COLAPM_PLAN_XI), blk,
                          blk ? reinterpret_cast<float2*>(c->Freal) : nullptr));
    }
    return COLAPM_OK;
}

// §2.4 steps 1-3: the three real force meshes F_j = -d psi / dx_j (cells) in force_mesh(c).
int compute_force(colapm_ctx* c) {
    int r = deposit(c);
    if (r) return r;
    return force_from_density(c);
}

StepCoef coef_for(const colapm_ctx* c, int i) {
    const StepTable& t = c->table;
    StepCoef k{};
    k.kick = (float)t.kick[i];
    k.drift = (float)t.drift[i];
    if (c->prm.cola) {
        k.c1 = (float)t.g[i].d1;
        k.c2 = (float)(t.g[i].d2 - t.g[i].d1 * t.g[i].d1);
        k.e1 = (float)(t.g[i + 1].d1 - t.g[i].d1);
        k.e2 = (float)(t.g[i + 1].d2 - t.g[i].d2);
    }
    return k;
}

constexpr int kLcK = 65;   // samples of the drift coefficients across a step for the lightcone exits

LightconeStep lightcone_step(colapm_ctx* c, int i) {
    LightconeStep l{};
    const int j = i - c->lc_first;
    l.out = c->lc_out;
    l.count = c->lc_count;
    l.capacity = c->lc_cap;
    l.tab = c->lc_tab + (size_t)j * kLcK * 5;
    l.reps = c->lc_reps + 3 * c->lc_rep_off[j];
    l.nrep = c->lc_rep_n[j];
    l.id = c->id_order ? nullptr : c->id;
    l.K = kLcK;
    l.ox = (float)c->lc.origin[0];
    l.oy = (float)c->lc.origin[1];
    l.oz = (float)c->lc.origin[2];
    l.cell = (float)(c->prm.box / c->nm);
    l.box = (float)c->prm.box;
    l.a0 = (float)c->table.a[i];
    l.da = (float)(c->table.a[i + 1] - c->table.a[i]);
    l.rl0 = c->lc_rl[i];
    l.rl1 = c->lc_rl[i + 1];
    return l;
}

void lightcone_free(colapm_ctx* c) {
    for (void* p : {(void*)c->lc_out, (void*)c->lc_count, (void*)c->lc_tab, (void*)c->lc_reps})
        if (p) cudaFree(p);
    c->lc_out = nullptr;
    c->lc_count = nullptr;
    c->lc_tab = nullptr;
    c->lc_reps = nullptr;
    c->lc_on = false;
}

// Particles from the LPT fields in psi1/psi2 (units: to_mesh converts them to mesh cells).
int place_particles(colapm_ctx* c, float to_mesh) {
    const Growth& g = c->table.g[0];
    if (c->lc_on) CK(cudaMemsetAsync(c->lc_count, 0, sizeof(unsigned long long), c->stream));   // a new run
    CKL(launch_iota(c->id, c->np3, c->stream));
    c->id_order = true;
    CKL(launch_init_particles(c->pos, c->mom, c->psi1, c->psi2, c->np, c->nm, to_mesh, (float)g.d1, (float)g.d2,
                             (float)g.p1, (float)g.p2, c->prm.cola, c->stream));
    c->step = 0;
    c->has_ics = true;
    c->finalized = false;
    return COLAPM_OK;
}

// The initial density field delta_k at z = 0 on the IC grid's half spectrum (§5): the Gaussian field,
// and, with f_NL != 0, the local transform of its primordial potential (transforms on the
// Stockham engine; `work` holds N_p^3 floats of scratch).
int initial_field(colapm_ctx* c, float2* dk, float2* work) {
    const int np = c->np;
    CKL(launch_gaussian_field(np, c->seed_src, c->amp_p, dk, c->stream));
    if (c->fnl == 0.0) return COLAPM_OK;
    const size_t ntab = (size_t)3 * (np / 2) * (np / 2) + 1;
    ZOut o{};
    o.p[0] = dk;
    CKL(launch_fz(np, Z_SCALE_INV, dk, o, c->tw_p, c->fnl_tab, 0, 1.0f, nullptr, c->stream, false));   // phi_k, z inverse
    CKL(launch_fy(np, +1, dk, 0, 1, c->tw_p, c->stream, false));
    CKL(launch_fx_inv(np, dk, 0, 1, c->tw_p, c->stream, false));                                       // phi(x)
    CKL(launch_local_fnl(reinterpret_cast<float*>(dk), c->np3, c->fnl, c->fnl_sum, c->stream));       // Phi(x)
    CKL(launch_fx_fwd_f32(np, reinterpret_cast<float*>(dk), work, c->tw_p, c->stream, false));
    CKL(launch_fy(np, -1, work, 0, 1, c->tw_p, c->stream, false));
    CKL(launch_fz(np, Z_SCALE_FWD, work, o, c->tw_p, c->fnl_tab + ntab, 0, 1.0f, nullptr, c->stream, false));   // M Phi_k
    return COLAPM_OK;
}

int validate(const colapm_params* p) {
    if (!p) return COLAPM_E_ARG;
    // N_m a multiple of N_p, or a coarser mesh with N_p = 2 N_m or 4 N_m (§7.3's mesh study)
    if (!supported_size(p->np) || !supported_size(p->nm)) return COLAPM_E_ARG;
    if (p->nm % p->np != 0 && p->np != 2 * p->nm && p->np != 4 * p->nm) return COLAPM_E_ARG;
    if (!(p->box > 0) || !(p->cosmo.omega_m > 0 && p->cosmo.omega_m <= 1) || !(p->cosmo.h > 0) ||
        !(p->cosmo.sigma8 > 0))
        return COLAPM_E_ARG;
    if (!(p->z_init > p->z_final) || !(p->z_final >= 0) || p->n_steps < 1 || p->n_steps > 100000) return COLAPM_E_ARG;
    if (p->spacing < 0 || p->spacing > 1 || p->stepping < 0 || p->stepping > 1) return COLAPM_E_ARG;
    if (p->stepping == 0 && p->nlpt == 0.0) return COLAPM_E_ARG;
    if (p->deconv < 0 || p->deconv > 2 || (p->cola != 0 && p->cola != 1)) return COLAPM_E_ARG;
    return COLAPM_OK;
}

}  // namespace

extern "C" {

void colapm_default_params(colapm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->cosmo.omega_m = 0.3;
    p->cosmo.omega_b = 0.05;
    p->cosmo.h = 0.7;
    p->cosmo.n_s = 0.96;
    p->cosmo.sigma8 = 0.8;
    p->box = 256.0;
    p->np = 32;
    p->nm = 64;
    p->z_init = 9.0;
    p->z_final = 0.0;
    p->n_steps = 10;
    p->spacing = 0;
    p->stepping = 0;
    p->nlpt = -2.5;
    p->cola = 1;
    p->deconv = 1;
    p->seed = 1;
}

const char* colapm_strerror(int code) {
    switch (code) {
        case COLAPM_OK: return "ok";
        case COLAPM_E_ARG: return "invalid argument";
        case COLAPM_E_NOMEM: return "out of memory";
        case COLAPM_E_CUDA: return "CUDA error";
        case COLAPM_E_OVERFLOW: return "fixed-point density overflow";
        case COLAPM_E_TIMEOUT: return "device wait timed out";
        case COLAPM_E_STATE: return "call out of order";
        default: return "unknown error";
    }
}

}  // extern "C"

// Configurations chosen by colapm_autotune in this process, applied to every later context (and
// batch mock) of the same size.
static std::mutex g_tune_mu;
struct Tuned {
    unsigned plan;
    int fused, block, key_tshift;
    bool dep_tiled;
};
static std::map<std::pair<int, int>, Tuned> g_tuned;   // (np, nm) -> choice

extern "C" {

int colapm_create(const colapm_params* p, void* stream, colapm_ctx** out) {
    if (!out) return COLAPM_E_ARG;
    *out = nullptr;
    int r = validate(p);
    if (r) return r;
    colapm_ctx* c = new (std::nothrow) colapm_ctx();
    if (!c) return COLAPM_E_NOMEM;
    c->prm = *p;
    c->stream = static_cast<cudaStream_t>(stream);
    c->np = p->np;
    c->nm = p->nm;
    c->np3 = (size_t)p->np * p->np * p->np;
    c->nm3 = (size_t)p->nm * p->nm * p->nm;
    c->table = make_step_table(p->cosmo.omega_m, p->z_init, p->z_final, p->n_steps, p->spacing, p->stepping, p->nlpt);

    bool ok = dalloc(&c->rho, c->nm3) == cudaSuccess && dalloc(&c->F, 3 * c->nm3) == cudaSuccess &&
              dalloc(&c->pos, c->np3) == cudaSuccess && dalloc(&c->mom, 3 * c->np3) == cudaSuccess &&
              dalloc(&c->psi1, 3 * c->np3) == cudaSuccess && dalloc(&c->psi2, 3 * c->np3) == cudaSuccess &&
              dalloc(&c->scratch, 9 * c->np3) == cudaSuccess && dalloc(&c->tw_m, (size_t)c->nm) == cudaSuccess &&
              dalloc(&c->tw_p, (size_t)c->np) == cudaSuccess && dalloc(&c->sinc2_m, 2 * (size_t)c->nm) == cudaSuccess &&
              dalloc(&c->amp_p, (size_t)3 * (c->np / 2) * (c->np / 2) + 1) == cudaSuccess &&
              dalloc(&c->err, 4) == cudaSuccess && dalloc(&c->d_seed, 1) == cudaSuccess &&
              dalloc(&c->id, c->np3) == cudaSuccess && dalloc(&c->pos_alt, c->np3) == cudaSuccess &&
              dalloc(&c->mom_alt, 3 * c->np3) == cudaSuccess && dalloc(&c->psi1_alt, 3 * c->np3) == cudaSuccess &&
              dalloc(&c->psi2_alt, 3 * c->np3) == cudaSuccess && dalloc(&c->id_alt, c->np3) == cudaSuccess &&
              dalloc(&c->sort_cnt, sort_buckets(c->nm)) == cudaSuccess &&
              dalloc(&c->sort_tile, sort_tiles(c->nm)) == cudaSuccess;
    if (ok && xy_supported(c->nm))
        ok = dalloc(reinterpret_cast<char**>(&c->xy_ring), xy_ring_bytes(c->nm)) == cudaSuccess &&
             dalloc(&c->xy_ctr, xy_ctr_ints(c->nm, 3)) == cudaSuccess;
    // blocked spectra where every pass has a two-stage plan (the x passes need N/2 in 256, 512)
    if (ok && (c->nm == 512 || c->nm == 1024)) ok = dalloc(&c->Freal, 3 * c->nm3) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return COLAPM_E_NOMEM;
    }
    std::vector<float2> tm = twiddles(c->nm), tp = twiddles(c->np);
    std::vector<float> s2(2 * c->nm, 1.0f);
    for (int i = 0; i < c->nm; ++i) {
        const int s = i < c->nm / 2 ? i : i - c->nm;
        const double x = M_PI * s / c->nm;
        const double v = s == 0 ? 1.0 : std::sin(x) / x;
        s2[i] = (float)(v * v);
    }
    // Gaussian-field amplitude N^3 sqrt(P(k) / L^3) per integer |n|^2 (FP64, then FP32).
    const int h = c->np / 2, n2max = 3 * h * h;
    std::vector<float> amp(n2max + 1);
    LinearPk pk(p->cosmo.omega_m, p->cosmo.h, p->cosmo.n_s, p->cosmo.sigma8);
    const double n3 = (double)c->np * c->np * c->np, l3 = p->box * p->box * p->box;
    amp[0] = 0.0f;
    for (int n2 = 1; n2 <= n2max; ++n2) amp[n2] = (float)(n3 * std::sqrt(pk(2.0 * M_PI * std::sqrt((double)n2) / p->box) / l3));
    cudaError_t e = cudaMemcpyAsync(c->tw_m, tm.data(), tm.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->tw_p, tp.data(), tp.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->sinc2_m, s2.data(), s2.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->amp_p, amp.data(), amp.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, 4 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // host vectors die at return
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return COLAPM_E_CUDA;
    }
    c->seed_src = c->d_seed;
    // Default reordering by cell: once, before step 2 n / 5, on meshes far larger than L2 (at 1024^3,
    // 10 steps, one sort before step 4 measured 27.76 ms per step against 27.78 and 27.89 before
    // steps 3 and 5; more frequent sorts cost more than they save).
    c->sort_every = c->nm >= 512 && p->n_steps >= 4 ? p->n_steps : 0;
    c->sort_first = 2 * p->n_steps / 5 > 0 ? 2 * p->n_steps / 5 : 1;
    c->key_tshift = c->nm % 2 == 0 ? 1 : 0;   // tiles of 64 x 2 x 2 cells (measured best of 1, 2, 4, 8 at 1024^3)
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find({c->np, c->nm});
        if (it != g_tuned.end()) {
            c->plan = it->second.plan;
            c->fused = it->second.fused;
            c->block = it->second.block;
            c->key_tshift = it->second.key_tshift;
            c->dep_tiled = it->second.dep_tiled;
        }
    }
    *out = c;
    return COLAPM_OK;
}

void colapm_destroy(colapm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    lightcone_free(c);
    free_all(c);
    delete c;
}

int colapm_make_ics(colapm_ctx* c) {
    if (!c) return COLAPM_E_ARG;
    Phase ph(c, COLAPM_PHASE_ICS);
    const int np = c->np;
    const size_t np3 = c->np3, hs = np3 / 2;   // complex elements per IC field
    float2* dk = reinterpret_cast<float2*>(c->scratch);
    float2* phi = reinterpret_cast<float2*>(c->scratch + np3);   // 6 fields
    float2* p1 = reinterpret_cast<float2*>(c->psi1);
    float2* p2 = reinterpret_cast<float2*>(c->psi2);
    const float gnorm = (float)(1.0 / ((double)np * np * np));
    if (c->seed_src == c->d_seed) CKL(launch_set_u64(c->d_seed, c->prm.seed, c->stream));
    if (int r = initial_field(c, dk, phi)) return r;
    ZOut o1{};
    for (int j = 0; j < 3; ++j) o1.p[j] = p1 + j * hs;
    for (int j = 0; j < 6; ++j) o1.p[3 + j] = phi + j * hs;
    CKL(launch_fz(np, Z_LPT1, dk, o1, c->tw_p, nullptr, 0, gnorm, nullptr, c->stream, ts(c, COLAPM_PLAN_Z)));
    CKL(launch_fy(np, +1, p1, hs, 3, c->tw_p, c->stream, ts(c, COLAPM_PLAN_Y)));
    CKL(launch_fy(np, +1, phi, hs, 6, c->tw_p, c->stream, ts(c, COLAPM_PLAN_Y)));
    CKL(launch_fx_inv(np, p1, hs, 3, c->tw_p, c->stream, ts(c, COLAPM_PLAN_XI)));
    CKL(launch_fx_inv(np, phi, hs, 6, c->tw_p, c->stream, ts(c, COLAPM_PLAN_XI)));
    // 2LPT: S from the six phi_ij, then Psi2 = -i k S_k / k^2.
    CKL(launch_lpt2_source(c->scratch + np3, np3, c->scratch, c->stream));
    CKL(launch_fx_fwd_f32(np, c->scratch, phi, c->tw_p, c->stream, ts(c, COLAPM_PLAN_XF)));
    CKL(launch_fy(np, -1, phi, 0, 1, c->tw_p, c->stream, ts(c, COLAPM_PLAN_Y)));
    ZOut o2{};
    for (int j = 0; j < 3; ++j) o2.p[j] = p2 + j * hs;
    CKL(launch_fz(np, Z_LPT2, phi, o2, c->tw_p, nullptr, 0, gnorm, nullptr, c->stream, ts(c, COLAPM_PLAN_Z)));
    CKL(launch_fy(np, +1, p2, hs, 3, c->tw_p, c->stream, ts(c, COLAPM_PLAN_Y)));
    CKL(launch_fx_inv(np, p2, hs, 3, c->tw_p, c->stream, ts(c, COLAPM_PLAN_XI)));
    return place_particles(c, (float)c->nm / np);
}

int colapm_set_displacements(colapm_ctx* c, const float* psi1, const float* psi2) {
    if (!c || !psi1 || !psi2) return COLAPM_E_ARG;
    c->id_order = true;   // the fields arrive in id order; place_particles resets the ids
    CK(cudaMemcpyAsync(c->psi1, psi1, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(c->psi2, psi2, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->stream));
    int r = place_particles(c, (float)(c->nm / c->prm.box));
    if (r) return r;
    CK(cudaStreamSynchronize(c->stream));
    return COLAPM_OK;
}

int colapm_step(colapm_ctx* c, int k) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics || c->finalized) return COLAPM_E_STATE;
    const int left = c->prm.n_steps - c->step;
    if (k < 0) k = left;
    if (k > left) return COLAPM_E_STATE;
    for (int s = 0; s < k; ++s) {
        if (sort_due(c, c->step)) {
            int r = sort_particles(c);
            if (r) return r;
        }
        int r = compute_force(c);
        if (r) return r;
        Phase ph(c, COLAPM_PHASE_GATHER);
        LightconeStep ls{};
        const bool rec = c->lc_on && c->step >= c->lc_first;
        if (rec) ls = lightcone_step(c, c->step);
        CKL(launch_gather_kick_drift(c->pos, c->mom, c->psi1, c->psi2, force_mesh(c), c->np3, c->nm, coef_for(c, c->step), 1,
                                    c->stream, c->block, rec ? &ls : nullptr));
        ++c->step;
    }
    return COLAPM_OK;
}

int colapm_finalize(colapm_ctx* c) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics || c->finalized || c->step != c->prm.n_steps) return COLAPM_E_STATE;
    int r = compute_force(c);
    if (r) return r;
    const int n = c->prm.n_steps;
    const Growth& g = c->table.g[n];
    StepCoef k{};
    k.kick = (float)c->table.kick_final;
    if (c->prm.cola) {
        k.c1 = (float)g.d1;
        k.c2 = (float)(g.d2 - g.d1 * g.d1);
    }
    {
        Phase ph(c, COLAPM_PHASE_GATHER);
        CKL(launch_gather_kick_drift(c->pos, c->mom, c->psi1, c->psi2, force_mesh(c), c->np3, c->nm, k, 0, c->stream, c->block));
    }
    if (c->prm.cola) CKL(launch_add_lpt_momentum(c->mom, c->psi1, c->psi2, c->np3, (float)g.p1, (float)g.p2, c->stream));
    c->finalized = true;
    return COLAPM_OK;
}

}  // extern "C"

namespace {

// Upload the |n|^2 thresholds of the P(k) bins (§7.1 binning; see PowerArgs) and size the
// accumulators. Bin membership of every integer |n|^2 is decided in FP64 with the same
// expressions as the definition: |k| = (2 pi / L) sqrt(n^2), e_b = kmin (kmax / kmin)^(b / nbins),
// e_b <= |k| < e_{b+1}; it is monotone in n^2, so n2_lo[b] = the smallest n^2 with |k| >= e_b.
int power_prepare(colapm_ctx* c, int nbins, double kmin, double kmax) {
    if (nbins < 1 || nbins > 4096) return COLAPM_E_ARG;
    const double box = c->prm.box, kf = 2.0 * M_PI / box;
    if (kmin <= 0) kmin = kf;
    if (kmax <= 0) kmax = M_PI * c->nm / box;
    if (!(kmax > kmin)) return COLAPM_E_ARG;
    const int h = c->nm / 2, n2max = 3 * h * h;
    std::vector<double> edges(nbins + 1);
    for (int b = 0; b <= nbins; ++b) edges[b] = kmin * std::pow(kmax / kmin, (double)b / nbins);
    std::vector<int> lo(nbins + 1, n2max + 1);
    {
        int b = 0;
        for (int n2 = 0; n2 <= n2max && b <= nbins; ++n2) {
            const double km = kf * std::sqrt((double)n2);
            while (b <= nbins && km >= edges[b]) lo[b++] = n2;   // first n^2 at or above edge b
        }
    }
    if (nbins + 1 > c->pw_n2cap) {
        if (c->pw_bin) cudaFree(c->pw_bin);
        c->pw_bin = nullptr;
        if (dalloc(&c->pw_bin, (size_t)nbins + 1) != cudaSuccess) {
            c->pw_n2cap = 0;
            return COLAPM_E_NOMEM;
        }
        c->pw_n2cap = nbins + 1;
    }
    if (nbins > c->pw_nbcap) {
        if (c->pw_acc) cudaFree(c->pw_acc);
        c->pw_acc = nullptr;
        if (dalloc(&c->pw_acc, (size_t)3 * nbins) != cudaSuccess) {
            c->pw_nbcap = 0;
            return COLAPM_E_NOMEM;
        }
        c->pw_nbcap = nbins;
    }
    CK(cudaMemcpyAsync(c->pw_bin, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double lr = std::log2(kmax / kmin);
    c->pw_lga = (float)(0.5 * nbins / lr);
    c->pw_lgb = (float)(nbins * std::log2(kf / kmin) / lr);
    return COLAPM_OK;
}

// Deposit, forward transform and bin into the device accumulators (no host synchronisation).
struct PhaseMute {   // time the nested deposit and forward passes under the enclosing phase
    colapm_ctx* c;
    explicit PhaseMute(colapm_ctx* x) : c(x) { ++c->phase_mute; }
    ~PhaseMute() { --c->phase_mute; }
};

// The density deposited is that of `src` (default: c's own particles); `window` = false bins
// |delta_k|^2 without dividing by the CIC window.
int power_enqueue(colapm_ctx* c, int nbins, const DepositSrc* src = nullptr, bool window = true) {
    const double box = c->prm.box;
    Phase ph(c, COLAPM_PHASE_POWER);   // all of P(k), its deposit and forward passes included
    PhaseMute mute(c);
    CK(cudaMemsetAsync(c->pw_acc, 0, (size_t)3 * nbins * sizeof(double), c->stream));
    int r = deposit(c, src);
    if (r) return r;
    r = density_xy(c);
    if (r) return r;
    PowerArgs pw{};
    pw.n2_lo = c->pw_bin;
    pw.kf = (float)(2.0 * M_PI / box);
    pw.ksum = c->pw_acc;
    pw.psum = c->pw_acc + nbins;
    pw.cnt = reinterpret_cast<unsigned long long*>(c->pw_acc + 2 * nbins);
    pw.nbins = nbins;
    const double nm = c->nm;
    pw.pnorm = (float)(box * box * box / (nm * nm * nm * nm * nm * nm));
    pw.lga = c->pw_lga;
    pw.lgb = c->pw_lgb;
    CKL(launch_fz(c->nm, Z_POWER, reinterpret_cast<float2*>(c->F), ZOut{}, c->tw_m, c->sinc2_m + (window ? 0 : c->nm), 0, 1.0f, &pw,
                  c->stream, ts(c, COLAPM_PLAN_Z), use_blocked(c)));
    return COLAPM_OK;
}

// Means per bin from the accumulators (ksum, psum, cnt as u64).
void power_finish(const double* acc, int nbins, double* ko, double* po, long long* no) {
    for (int b = 0; b < nbins; ++b) {
        unsigned long long cnt;
        std::memcpy(&cnt, &acc[2 * nbins + b], sizeof(cnt));
        no[b] = (long long)cnt;
        ko[b] = cnt ? acc[b] / (double)cnt : NAN;
        po[b] = cnt ? acc[nbins + b] / (double)cnt : NAN;
    }
}

}  // namespace

extern "C" {

int colapm_power(colapm_ctx* c, int nbins, double kmin, double kmax, double* k_out, double* p_out,
                 long long* nmodes_out) {
    if (!c || !k_out || !p_out || !nmodes_out) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    int r = power_prepare(c, nbins, kmin, kmax);
    if (r) return r;
    r = power_enqueue(c, nbins);
    if (r) return r;
    std::vector<double> acc(3 * nbins);
    CK(cudaMemcpyAsync(acc.data(), c->pw_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    r = pending_error(c);   // synchronises
    if (r) return r;
    std::vector<double> ko(nbins), po(nbins);
    std::vector<long long> no(nbins);
    power_finish(acc.data(), nbins, ko.data(), po.data(), no.data());
    CK(cudaMemcpyAsync(k_out, ko.data(), nbins * sizeof(double), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(p_out, po.data(), nbins * sizeof(double), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(nmodes_out, no.data(), nbins * sizeof(long long), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COLAPM_OK;
}

int colapm_cross_correlation(colapm_ctx* a, colapm_ctx* b, int nbins, double kmin, double kmax, double* k_out,
                             double* r_out, long long* nmodes_out) {
    if (!a || !b || !k_out || !r_out || !nmodes_out) return COLAPM_E_ARG;
    if (!a->has_ics || !b->has_ics) return COLAPM_E_STATE;
    if (a->np != b->np || a->nm != b->nm || a->prm.box != b->prm.box) return COLAPM_E_ARG;
    CK(cudaStreamSynchronize(b->stream));   // b's particles are complete before a's stream reads them
    int r = power_prepare(a, nbins, kmin, kmax);
    if (r) return r;
    // Bin sums of |delta_a|^2, |delta_b|^2 and |delta_a + delta_b|^2 (the masses of both deposited
    // into one mesh; the transform is linear), without the window: Re(delta_a delta_b^*) is half of
    // the third minus the first two, mode by mode, so also bin by bin.
    std::vector<double> acc(9 * (size_t)nbins);
    DepositSrc src[3];
    src[0] = own_particles(a);
    src[1] = own_particles(b);
    src[2] = own_particles(a);
    src[2].pos[1] = b->pos;
    src[2].n[1] = b->np3;
    for (int pass = 0; pass < 3; ++pass) {
        r = power_enqueue(a, nbins, &src[pass], false);
        if (r) return r;
        CK(cudaMemcpyAsync(acc.data() + (size_t)pass * 3 * nbins, a->pw_acc, 3 * (size_t)nbins * sizeof(double),
                           cudaMemcpyDeviceToHost, a->stream));
        r = pending_error(a);   // synchronises
        if (r) return r;
    }
    std::vector<double> ko(nbins), ro(nbins), pa(nbins), pb(nbins), pab(nbins);
    std::vector<long long> no(nbins);
    power_finish(acc.data(), nbins, ko.data(), pa.data(), no.data());
    power_finish(acc.data() + 3 * (size_t)nbins, nbins, ko.data(), pb.data(), no.data());
    power_finish(acc.data() + 6 * (size_t)nbins, nbins, ko.data(), pab.data(), no.data());
    for (int i = 0; i < nbins; ++i) ro[i] = no[i] ? 0.5 * (pab[i] - pa[i] - pb[i]) / std::sqrt(pa[i] * pb[i]) : NAN;
    CK(cudaMemcpyAsync(k_out, ko.data(), nbins * sizeof(double), cudaMemcpyDefault, a->stream));
    CK(cudaMemcpyAsync(r_out, ro.data(), nbins * sizeof(double), cudaMemcpyDefault, a->stream));
    CK(cudaMemcpyAsync(nmodes_out, no.data(), nbins * sizeof(long long), cudaMemcpyDefault, a->stream));
    CK(cudaStreamSynchronize(a->stream));
    return COLAPM_OK;
}

int colapm_power_rsd(colapm_ctx* c, int los, int nbins, double kmin, double kmax, double* k_out, double* p_out,
                     long long* nmodes_out) {
    if (!c || !k_out || !p_out || !nmodes_out || los < -1 || los > 2) return COLAPM_E_ARG;
    if (!c->has_ics || !c->finalized) return COLAPM_E_STATE;   // total momenta at a_N
    int r = power_prepare(c, nbins, kmin, kmax);
    if (r) return r;
    const double a = c->table.a[c->prm.n_steps], om = c->prm.cosmo.omega_m;
    const double e = std::sqrt(om / (a * a * a) + 1.0 - om);
    // the redshift-space positions go to the second particle array (free between calls)
    CKL(launch_rsd_positions(c->pos, c->mom, c->np3, c->nm, (float)(1.0 / (a * a * e)), los, c->pos_alt, c->stream));
    DepositSrc src;
    src.pos[0] = c->pos_alt;
    src.n[0] = c->np3;
    r = power_enqueue(c, nbins, &src);
    if (r) return r;
    std::vector<double> acc(3 * nbins);
    CK(cudaMemcpyAsync(acc.data(), c->pw_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    r = pending_error(c);
    if (r) return r;
    std::vector<double> ko(nbins), po(nbins);
    std::vector<long long> no(nbins);
    power_finish(acc.data(), nbins, ko.data(), po.data(), no.data());
    CK(cudaMemcpyAsync(k_out, ko.data(), nbins * sizeof(double), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(p_out, po.data(), nbins * sizeof(double), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(nmodes_out, no.data(), nbins * sizeof(long long), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COLAPM_OK;
}

int colapm_get_particles(colapm_ctx* c, float* pos, float* mom) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    const float cell = (float)(c->prm.box / c->nm);
    float* dp = pos && !is_device_ptr(pos) ? c->scratch : pos;
    float* dm = mom && !is_device_ptr(mom) ? c->scratch + 3 * c->np3 : mom;
    CKL(launch_export_particles(c->pos, c->mom, c->id_order ? nullptr : c->id, c->np3, c->nm, cell, dp, dm, c->stream));
    if (pos && dp != pos) copy_out(c, pos, dp, 3 * c->np3 * sizeof(float));
    if (mom && dm != mom) copy_out(c, mom, dm, 3 * c->np3 * sizeof(float));
    return pending_error(c);
}

int colapm_get_particles_async(colapm_ctx* c, float* pos, float* mom) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (!c->xfer) {
        if (dalloc(&c->xfer, 6 * c->np3) != cudaSuccess) {
            c->xfer = nullptr;
            cudaGetLastError();
            return COLAPM_E_NOMEM;
        }
        CK(cudaStreamCreateWithFlags(&c->xfer_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->xfer_ready, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->xfer_done, cudaEventDisableTiming));
    }
    if (c->xfer_pending) CK(cudaStreamWaitEvent(c->stream, c->xfer_done, 0));   // staging array free
    const float cell = (float)(c->prm.box / c->nm);
    float* dp = c->xfer;
    float* dm = c->xfer + 3 * c->np3;
    CKL(launch_export_particles(c->pos, c->mom, c->id_order ? nullptr : c->id, c->np3, c->nm, cell, dp, dm, c->stream));
    CK(cudaEventRecord(c->xfer_ready, c->stream));
    CK(cudaStreamWaitEvent(c->xfer_stream, c->xfer_ready, 0));
    if (pos) CK(cudaMemcpyAsync(pos, dp, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->xfer_stream));
    if (mom) CK(cudaMemcpyAsync(mom, dm, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->xfer_stream));
    CK(cudaEventRecord(c->xfer_done, c->xfer_stream));
    c->xfer_pending = true;
    return COLAPM_OK;
}

int colapm_wait_particles(colapm_ctx* c) {
    if (!c) return COLAPM_E_ARG;
    if (c->xfer_pending) {
        CK(cudaEventSynchronize(c->xfer_done));
        c->xfer_pending = false;
    }
    return pending_error(c);
}

int colapm_get_state(colapm_ctx* c, int* cell, float* off, float* mom) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (int r = id_order(c)) return r;
    const size_t n = 3 * c->np3;
    int* dc = cell && !is_device_ptr(cell) ? reinterpret_cast<int*>(c->scratch) : cell;
    float* doff = off && !is_device_ptr(off) ? c->scratch + n : off;
    float* dm = mom && !is_device_ptr(mom) ? c->scratch + 2 * n : mom;
    CKL(launch_export_state(c->pos, c->mom, c->np3, c->nm, dc, doff, dm, c->stream));
    if (cell && dc != cell) copy_out(c, cell, dc, n * sizeof(int));
    if (off && doff != off) copy_out(c, off, doff, n * sizeof(float));
    if (mom && dm != mom) copy_out(c, mom, dm, n * sizeof(float));
    return pending_error(c);
}

int colapm_set_state(colapm_ctx* c, const int* cell, const float* off, const float* mom) {
    if (!c || (!cell != !off) || (!cell && !mom)) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (int r = id_order(c)) return r;
    const size_t n = 3 * c->np3;
    const int* dc = cell;
    const float* doff = off;
    const float* dm = mom;
    if (cell && !is_device_ptr(cell)) {
        CK(cudaMemcpyAsync(c->scratch, cell, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        dc = reinterpret_cast<const int*>(c->scratch);
    }
    if (off && !is_device_ptr(off)) {
        CK(cudaMemcpyAsync(c->scratch + n, off, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        doff = c->scratch + n;
    }
    if (mom && !is_device_ptr(mom)) {
        CK(cudaMemcpyAsync(c->scratch + 2 * n, mom, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        dm = c->scratch + 2 * n;
    }
    CKL(launch_import_state(c->pos, c->mom, c->np3, c->nm, dc, doff, dm, c->err, c->stream));
    return pending_error(c);
}

int colapm_get_displacement(colapm_ctx* c, float* psi) {
    if (!c || !psi) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (int r = id_order(c)) return r;
    float* d = is_device_ptr(psi) ? psi : c->scratch;
    CKL(launch_export_displacement(c->pos, c->np, c->nm, (float)(c->prm.box / c->nm), d, c->stream));
    if (d != psi) copy_out(c, psi, d, 3 * c->np3 * sizeof(float));
    return pending_error(c);
}

int colapm_set_displacement(colapm_ctx* c, const float* psi) {
    if (!c || !psi) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (int r = id_order(c)) return r;
    const float* d = psi;
    if (!is_device_ptr(psi)) {
        CK(cudaMemcpyAsync(c->scratch, psi, 3 * c->np3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        d = c->scratch;
    }
    CKL(launch_import_displacement(c->pos, c->np, c->nm, (float)(c->nm / c->prm.box), d, c->err, c->stream));
    return pending_error(c);
}

int colapm_get_density(colapm_ctx* c, long long* mesh) {
    if (!c || !mesh) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    int r = deposit(c);
    if (r) return r;
    copy_out(c, mesh, c->rho, c->nm3 * sizeof(long long));
    return pending_error(c);
}

int colapm_get_force(colapm_ctx* c, float* force) {
    if (!c || !force) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    int r = compute_force(c);
    if (r) return r;
    copy_out(c, force, force_mesh(c), 3 * c->nm3 * sizeof(float));
    return pending_error(c);
}

int colapm_get_lpt(colapm_ctx* c, float* psi1, float* psi2) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (int r = id_order(c)) return r;
    const float f = (float)(c->prm.box / c->nm);
    const size_t n = 3 * c->np3;
    if (psi1) {
        CKL(launch_scale(c->scratch, c->psi1, n, f, c->stream));
        copy_out(c, psi1, c->scratch, n * sizeof(float));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (psi2) {
        CKL(launch_scale(c->scratch, c->psi2, n, f, c->stream));
        copy_out(c, psi2, c->scratch, n * sizeof(float));
    }
    return pending_error(c);
}

int colapm_get_gaussian_field(colapm_ctx* c, float* dk) {
    if (!c || !dk) return COLAPM_E_ARG;
    CKL(launch_set_u64(c->d_seed, c->prm.seed, c->stream));
    const unsigned long long* src = c->seed_src;
    c->seed_src = c->d_seed;
    int r = initial_field(c, reinterpret_cast<float2*>(c->scratch), reinterpret_cast<float2*>(c->scratch + c->np3));
    c->seed_src = src;
    if (r) return r;
    copy_out(c, dk, c->scratch, c->np3 * sizeof(float));
    return pending_error(c);
}

int colapm_set_fnl(colapm_ctx* c, double fnl) {
    if (!c || !std::isfinite(fnl)) return COLAPM_E_ARG;
    if (fnl != 0.0 && !c->fnl_tab) {
        const int h = c->np / 2;
        const size_t ntab = (size_t)3 * h * h + 1;
        if (dalloc(&c->fnl_tab, 2 * ntab) != cudaSuccess || dalloc(&c->fnl_sum, 1) != cudaSuccess) {
            cudaGetLastError();
            return COLAPM_E_NOMEM;
        }
        // M(k) = (2/3) (k c / H0)^2 T(k) D_md / Om per integer |n|^2 (k = 2 pi |n| / L), FP64 then FP32
        const double om = c->prm.cosmo.omega_m, hh = c->prm.cosmo.h, dmd = growth_matter_era(om);
        const double n3 = (double)c->np * c->np * c->np, chub = 2997.92458;
        std::vector<float> tab(2 * ntab, 0.0f);
        for (size_t n2 = 1; n2 < ntab; ++n2) {
            const double k = 2.0 * M_PI * std::sqrt((double)n2) / c->prm.box;
            const double m = 2.0 / 3.0 * (k * chub) * (k * chub) * bbks(k, om, hh) * dmd / om;
            tab[n2] = (float)(1.0 / (m * n3));
            tab[ntab + n2] = (float)m;
        }
        CK(cudaMemcpyAsync(c->fnl_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->fnl = fnl;
    return COLAPM_OK;
}

int colapm_set_lightcone(colapm_ctx* c, const colapm_lightcone* lc, long long capacity) {
    if (!c) return COLAPM_E_ARG;
    CK(cudaStreamSynchronize(c->stream));
    lightcone_free(c);
    if (!lc) return COLAPM_OK;
    if (capacity < 1 || !(lc->z_max > c->prm.z_final)) return COLAPM_E_ARG;
    for (int j = 0; j < 3; ++j)
        if (lc->rep_lo[j] > lc->rep_hi[j] || lc->rep_hi[j] - lc->rep_lo[j] > 32 || !std::isfinite(lc->origin[j]))
            return COLAPM_E_ARG;
    const StepTable& t = c->table;
    const int n = c->prm.n_steps;
    const double om = c->prm.cosmo.omega_m, L = c->prm.box, a_start = 1.0 / (1.0 + lc->z_max);
    int first = 0;
    while (first < n && t.a[first] < a_start - 1e-12) ++first;   // first boundary at or after a(z_max)
    if (first >= n) return COLAPM_E_ARG;
    c->lc_rl.assign(n + 1, 0.0f);
    for (int i = 0; i <= n; ++i) c->lc_rl[i] = (float)comoving_distance(t.a[i], om);
    // per step: drift coefficients sampled across the step, and the replicates whose box can meet the
    // shell between the two radii (a quarter box of margin for the particles' motion within the step)
    std::vector<float> tab;
    std::vector<int> reps;
    c->lc_rep_off.clear();
    c->lc_rep_n.clear();
    for (int i = first; i < n; ++i) {
        const double a0 = t.a[i], a1 = t.a[i + 1], am = 0.5 * (a0 + a1);
        const Growth g0 = t.g[i];
        for (int k = 0; k < kLcK; ++k) {
            const double a = a0 + (a1 - a0) * k / (kLcK - 1);
            const Growth g = growth_at(a, om);
            const double sd = k == 0 ? 0.0 : drift_coef(a0, a, am, om, c->prm.stepping, c->prm.nlpt);
            const bool cola = c->prm.cola != 0;
            tab.push_back((float)sd);   // position change per unit momentum (any consistent length unit)
            tab.push_back(cola ? (float)(g.d1 - g0.d1) : 0.0f);
            tab.push_back(cola ? (float)(g.d2 - g0.d2) : 0.0f);
            tab.push_back(cola ? (float)g.p1 : 0.0f);
            tab.push_back(cola ? (float)g.p2 : 0.0f);
        }
        c->lc_rep_off.push_back((int)(reps.size() / 3));
        int cnt = 0;
        for (int rx = lc->rep_lo[0]; rx <= lc->rep_hi[0]; ++rx)
            for (int ry = lc->rep_lo[1]; ry <= lc->rep_hi[1]; ++ry)
                for (int rz = lc->rep_lo[2]; rz <= lc->rep_hi[2]; ++rz) {
                    const int rr[3] = {rx, ry, rz};
                    double dmin2 = 0.0, dmax2 = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        const double lo = rr[j] * L - lc->origin[j], hi = lo + L;
                        const double near = lo > 0 ? lo : (hi < 0 ? -hi : 0.0);
                        const double far = std::fmax(std::fabs(lo), std::fabs(hi));
                        dmin2 += near * near;
                        dmax2 += far * far;
                    }
                    const double margin = 0.25 * L;
                    if (std::sqrt(dmin2) <= c->lc_rl[i] + margin && std::sqrt(dmax2) >= c->lc_rl[i + 1] - margin) {
                        reps.insert(reps.end(), rr, rr + 3);
                        ++cnt;
                    }
                }
        c->lc_rep_n.push_back(cnt);
    }
    if (reps.empty()) reps.assign(3, 0);
    if (dalloc(&c->lc_out, 2 * (size_t)capacity) != cudaSuccess || dalloc(&c->lc_count, 1) != cudaSuccess ||
        dalloc(&c->lc_tab, tab.size()) != cudaSuccess || dalloc(&c->lc_reps, reps.size()) != cudaSuccess) {
        cudaGetLastError();
        lightcone_free(c);
        return COLAPM_E_NOMEM;
    }
    CK(cudaMemcpyAsync(c->lc_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->lc_reps, reps.data(), reps.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->lc_count, 0, sizeof(unsigned long long), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->lc = *lc;
    c->lc_first = first;
    c->lc_cap = (unsigned long long)capacity;
    c->lc_on = true;
    return COLAPM_OK;
}

int colapm_get_lightcone(colapm_ctx* c, long long* count, colapm_lc_particle* rows, long long max_rows,
                         long long* copied) {
    if (!c || !count || max_rows < 0 || (max_rows > 0 && !rows)) return COLAPM_E_ARG;
    if (copied) *copied = 0;
    if (!c->lc_on) return COLAPM_E_STATE;
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, c->lc_count, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = (long long)n;
    const unsigned long long stored = n < c->lc_cap ? n : c->lc_cap;
    const unsigned long long k = stored < (unsigned long long)max_rows ? stored : (unsigned long long)max_rows;
    static_assert(sizeof(colapm_lc_particle) == 2 * sizeof(float4), "row layout");
    if (k) CK(cudaMemcpyAsync(rows, c->lc_out, k * sizeof(colapm_lc_particle), cudaMemcpyDefault, c->stream));
    int r = pending_error(c);   // synchronises
    if (r) return r;
    if (copied) *copied = (long long)k;
    return n > c->lc_cap ? COLAPM_E_OVERFLOW : COLAPM_OK;
}

int colapm_reseed(colapm_ctx* c, unsigned long long seed) {
    if (!c) return COLAPM_E_ARG;
    c->prm.seed = seed;
    return COLAPM_OK;
}

long long colapm_kernel_launches(const colapm_ctx* c) { return c ? c->launches : COLAPM_E_ARG; }

int colapm_sync(colapm_ctx* c) {
    if (!c) return COLAPM_E_ARG;
    return pending_error(c);
}

int colapm_steps_done(const colapm_ctx* c) { return c ? c->step : COLAPM_E_ARG; }

static const unsigned long long kStateMagic = 0x434f4c41504d3031ull;   // "COLAPM01"

int colapm_save_state(colapm_ctx* c, void* buf, size_t* n) {
    if (!c || !n) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    if (buf) {
        if (int r = id_order(c)) return r;   // the state is saved in id order
    }
    const size_t hdr = 8 * sizeof(long long);
    const size_t need = hdr + c->np3 * sizeof(float4) + 9 * c->np3 * sizeof(float);
    if (!buf) {
        *n = need;
        return COLAPM_OK;
    }
    if (*n < need) return COLAPM_E_ARG;
    long long h[8] = {(long long)kStateMagic, c->np, c->nm, c->step, c->finalized ? 1 : 0, c->prm.n_steps, 0, 0};
    char* b = static_cast<char*>(buf);
    std::memcpy(b, h, hdr);
    size_t o = hdr;
    CK(cudaMemcpyAsync(b + o, c->pos, c->np3 * sizeof(float4), cudaMemcpyDefault, c->stream));
    o += c->np3 * sizeof(float4);
    for (float* src : {c->mom, c->psi1, c->psi2}) {
        CK(cudaMemcpyAsync(b + o, src, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->stream));
        o += 3 * c->np3 * sizeof(float);
    }
    *n = need;
    CK(cudaStreamSynchronize(c->stream));
    return COLAPM_OK;
}

int colapm_load_state(colapm_ctx* c, const void* buf, size_t n) {
    if (!c || !buf) return COLAPM_E_ARG;
    const size_t hdr = 8 * sizeof(long long);
    const size_t need = hdr + c->np3 * sizeof(float4) + 9 * c->np3 * sizeof(float);
    if (n < need) return COLAPM_E_ARG;
    long long h[8];
    std::memcpy(h, buf, hdr);
    if ((unsigned long long)h[0] != kStateMagic || h[1] != c->np || h[2] != c->nm || h[5] != c->prm.n_steps ||
        h[3] < 0 || h[3] > c->prm.n_steps)
        return COLAPM_E_ARG;
    const char* b = static_cast<const char*>(buf);
    size_t o = hdr;
    CK(cudaMemcpyAsync(c->pos, b + o, c->np3 * sizeof(float4), cudaMemcpyDefault, c->stream));
    o += c->np3 * sizeof(float4);
    for (float* dst : {c->mom, c->psi1, c->psi2}) {
        CK(cudaMemcpyAsync(dst, b + o, 3 * c->np3 * sizeof(float), cudaMemcpyDefault, c->stream));
        o += 3 * c->np3 * sizeof(float);
    }
    CKL(launch_iota(c->id, c->np3, c->stream));
    c->id_order = true;
    CK(cudaStreamSynchronize(c->stream));
    c->step = (int)h[3];
    c->finalized = h[4] != 0;
    c->has_ics = true;
    return COLAPM_OK;
}

int colapm_set_timing(colapm_ctx* c, int on) {
    if (!c) return COLAPM_E_ARG;
    c->timing = on != 0;
    return COLAPM_OK;
}

int colapm_get_timing(colapm_ctx* c, double* ms, long long* launches) {
    if (!c) return COLAPM_E_ARG;
    CK(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < COLAPM_PHASE_COUNT; ++p) {
        double sum = 0.0;
        for (auto& pr : c->ev[p]) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) sum += t;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        if (ms) ms[p] = sum;
        if (launches) launches[p] = (long long)c->ev[p].size();
        c->ev[p].clear();
    }
    return COLAPM_OK;
}


// ---------------------------------------------------------------------------------------------
// Autotuning: FFT engine and particle-kernel block size, timed on the context's own state.


int colapm_set_engine(colapm_ctx* c, int fused, int two_stage, int block) {
    if (!c || (block != 128 && block != 256 && block != 512) || fused < 0 || fused > 3) return COLAPM_E_ARG;
    c->fused = fused;
    c->plan = two_stage ? COLAPM_PLAN_ALL : 0u;
    c->block = block;
    return COLAPM_OK;
}

int colapm_set_plan(colapm_ctx* c, int plan) {
    if (!c || plan < 0 || plan > (int)COLAPM_PLAN_ALL) return COLAPM_E_ARG;
    c->plan = (unsigned)plan;
    return COLAPM_OK;
}

int colapm_get_config(const colapm_ctx* c, int* cfg) {
    if (!c || !cfg) return COLAPM_E_ARG;
    cfg[0] = (int)c->plan;
    cfg[1] = c->block;
    cfg[2] = c->xy_ring ? c->fused : 0;
    cfg[3] = c->sort_every;
    cfg[6] = c->sort_first;
    cfg[4] = 1 << c->key_tshift;
    cfg[5] = c->dep_tiled ? 1 : 0;
    return COLAPM_OK;
}

// t = 2^ts with 0 <= ts <= 3 and nm a multiple of t; -1 otherwise.
static int tile_shift_of(const colapm_ctx* c, int t) {
    for (int ts = 0; ts <= 3; ++ts)
        if (t == (1 << ts)) return sort_tshift_ok(c->nm, ts) ? ts : -1;
    return -1;
}

int colapm_set_sort_tiles(colapm_ctx* c, int t) {
    if (!c) return COLAPM_E_ARG;
    const int ts = tile_shift_of(c, t);
    if (ts < 0) return COLAPM_E_ARG;
    c->key_tshift = ts;
    if (ts == 0) c->dep_tiled = false;
    return COLAPM_OK;
}

int colapm_set_deposit_tiles(colapm_ctx* c, int t) {
    if (!c) return COLAPM_E_ARG;
    if (t == 0) {
        c->dep_tiled = false;
        return COLAPM_OK;
    }
    const int ts = tile_shift_of(c, t);
    if (ts < 1) return COLAPM_E_ARG;
    c->key_tshift = ts;
    c->dep_tiled = true;
    return COLAPM_OK;
}

int colapm_set_sort(colapm_ctx* c, int every) {
    if (!c || every < 0) return COLAPM_E_ARG;
    c->sort_every = every;
    c->sort_first = every;
    return COLAPM_OK;
}

int colapm_autotune(colapm_ctx* c, int* choice) {
    if (!c) return COLAPM_E_ARG;
    if (!c->has_ics) return COLAPM_E_STATE;
    // Snapshot of the particle state in the scratch buffer (4 + 3 floats per particle <= 9).
    float* snap = c->scratch;
    CK(cudaMemcpyAsync(snap, c->pos, c->np3 * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(snap + 4 * c->np3, c->mom, 3 * c->np3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    const int step0 = c->step;
    const bool fin0 = c->finalized;
    const unsigned p0 = c->plan;
    const int f0 = c->fused;
    const int b0 = c->block;
    const bool timing0 = c->timing;
    c->timing = false;
    c->finalized = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int ksteps = c->prm.n_steps - 1 < step0 ? 0 : 1;
    int r = COLAPM_OK;
    // One force computation + gather from the snapshot in configuration (plan, fused, block): the
    // fastest of three repetitions after one warm-up, in ms (infinite on an error).
    auto trial = [&](unsigned plan, int fused, int block) -> float {
        c->plan = plan;
        c->fused = fused;
        c->block = block;
        float best_ms = 1e30f;
        for (int rep = 0; rep < 4 && r == COLAPM_OK; ++rep) {
            if (cudaMemcpyAsync(c->pos, snap, c->np3 * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(c->mom, snap + 4 * c->np3, 3 * c->np3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess) {
                r = COLAPM_E_CUDA;
                break;
            }
            c->step = ksteps ? step0 : 0;
            cudaEventRecord(e0, c->stream);
            r = compute_force(c);
            if (r == COLAPM_OK && cudaGetLastError() == cudaSuccess) {
                const int i = c->step < c->prm.n_steps ? c->step : c->prm.n_steps - 1;
                if (launch_gather_kick_drift(c->pos, c->mom, c->psi1, c->psi2, force_mesh(c), c->np3, c->nm, coef_for(c, i), 1,
                                             c->stream, c->block) != cudaSuccess)
                    r = COLAPM_E_CUDA;
            }
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) r = COLAPM_E_CUDA;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best_ms) best_ms = ms;
        }
        return r == COLAPM_OK ? best_ms : 1e30f;
    };
    float best = 1e30f;
    unsigned best_p = p0;
    int best_f = f0;
    int best_b = b0;
    // 1. engines (fused x-y passes where the mesh size has them, all passes two-stage, all
    //    Stockham) x particle-kernel block sizes
    const int blocks[3] = {128, 256, 512};
    for (int eng = c->xy_ring ? 0 : 1; eng < 3 && r == COLAPM_OK; ++eng) {
        for (int bi = 0; bi < 3 && r == COLAPM_OK; ++bi) {
            const unsigned plan = eng < 2 ? COLAPM_PLAN_ALL : 0u;
            const int fused = eng == 0 ? 3 : 0;
            const float ms = trial(plan, fused, blocks[bi]);
            if (ms < best) {
                best = ms;
                best_p = plan;
                best_f = fused;
                best_b = blocks[bi];
            }
        }
    }
    // 2. the radix plan per pass: starting from the best separate-pass engine, switch each pass
    //    (forward x, y both ways, z, inverse x) to the other plan and keep what is faster
    if (best_f == 0) {
        const unsigned bits[4] = {COLAPM_PLAN_XF, COLAPM_PLAN_Y, COLAPM_PLAN_Z, COLAPM_PLAN_XI};
        for (int k = 0; k < 4 && r == COLAPM_OK; ++k) {
            const unsigned plan = best_p ^ bits[k];
            const float ms = trial(plan, 0, best_b);
            if (ms < best) {
                best = ms;
                best_p = plan;
            }
        }
    }
    cudaMemcpyAsync(c->pos, snap, c->np3 * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->mom, snap + 4 * c->np3, 3 * c->np3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    c->step = step0;
    c->finalized = fin0;
    c->timing = timing0;
    if (r != COLAPM_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->plan = p0;
        c->fused = f0;
        c->block = b0;
        return r;
    }
    c->plan = best_p;
    c->fused = best_f;
    c->block = best_b;
    // 3. where the context reorders its particles: the tile shape of the sort key (rows of 64
    //    cells, or tiles of 64 x T x T) and, for tiles, the tiled deposit or the plain one. For each
    //    candidate the particles are sorted with its key (the order changes no result), and one force
    //    computation + gather is timed from that state as in 1 (restored after each repetition);
    //    the particles are left in the order of the candidate kept
    int best_k = c->key_tshift;
    bool best_dt = c->dep_tiled;
    if (c->sort_every > 0 && r == COLAPM_OK) {
        float best3 = 1e30f;
        for (int ts = 0; ts <= 3 && r == COLAPM_OK; ++ts) {
            if (!sort_tshift_ok(c->nm, ts)) continue;
            c->key_tshift = ts;
            c->dep_tiled = false;
            r = sort_particles(c);
            if (r != COLAPM_OK) break;
            if (cudaMemcpyAsync(snap, c->pos, c->np3 * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(snap + 4 * c->np3, c->mom, 3 * c->np3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess) {
                r = COLAPM_E_CUDA;
                break;
            }
            for (int dt = 0; dt < (ts > 0 ? 2 : 1) && r == COLAPM_OK; ++dt) {
                c->dep_tiled = dt == 1;
                const float ms = trial(best_p, best_f, best_b);
                if (ms < best3) {
                    best3 = ms;
                    best_k = ts;
                    best_dt = dt == 1;
                }
            }
            cudaMemcpyAsync(c->pos, snap, c->np3 * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(c->mom, snap + 4 * c->np3, 3 * c->np3 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        }
        c->dep_tiled = best_dt;
        if (r == COLAPM_OK && c->key_tshift != best_k) {
            c->key_tshift = best_k;
            r = sort_particles(c);
        }
        c->step = step0;
        c->finalized = fin0;
        if (r == COLAPM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) r = COLAPM_E_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != COLAPM_OK) return r;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[{c->np, c->nm}] = Tuned{best_p, best_f, best_b, best_k, best_dt};
    }
    if (choice) {
        choice[0] = best_p == COLAPM_PLAN_ALL ? 1 : 0;
        choice[1] = best_b;
        choice[2] = c->xy_ring ? best_f : 0;
    }
    return COLAPM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched mocks.

struct colapm_batch {
    int n = 0;
    int nstreams = 0;                       // 0: not chosen yet
    cudaStream_t caller = nullptr;          // the caller's stream (may be the legacy default stream)
    cudaStream_t user = nullptr;            // internal stream the graph is captured on and launched from
    std::vector<colapm_ctx*> ctx;
    std::vector<cudaStream_t> ws;           // kMaxStreams worker streams
    std::vector<cudaEvent_t> ev;            // fork + one join per worker
    unsigned long long* seeds_h = nullptr;  // pinned [n]
    unsigned long long* seeds_d = nullptr;  // [n]
    double* acc_h = nullptr;                // pinned [n][3 nbins]
    int nbins = 0;
    double kmin = 0.0, kmax = 0.0;
    cudaGraphExec_t exec = nullptr;
    bool lockstep = true;                   // step all mocks together with the multi-mock particle kernels
    int max_steps = 0;                      // the largest n_steps of the batch
    MockWork* work_h = nullptr;             // pinned [max_steps][n]: the multi-mock descriptors of each step
    MockWork* work_d = nullptr;             // device copy
    unsigned long long* queue_d = nullptr;  // work-ticket counters of the two multi-mock kernels (4 u64)
};

namespace {

constexpr int kMaxStreams = 8;

void batch_free(colapm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (colapm_ctx* c : b->ctx)
        if (c) colapm_destroy(c);
    for (cudaStream_t s : b->ws) cudaStreamDestroy(s);
    if (b->user) cudaStreamDestroy(b->user);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->seeds_h) cudaFreeHost(b->seeds_h);
    if (b->seeds_d) cudaFree(b->seeds_d);
    if (b->acc_h) cudaFreeHost(b->acc_h);
    if (b->work_h) cudaFreeHost(b->work_h);
    if (b->work_d) cudaFree(b->work_d);
    if (b->queue_d) cudaFree(b->queue_d);
}

// Lockstep schedule: ICs of every mock (worker stream i mod K), then per step s one multi-mock
// deposit of every mock still running, the mesh passes of each mock (worker streams), one
// multi-mock gather-kick-drift, then the P(k) of every mock. The descriptors of step s are
// written to the pinned buffer when the step is enqueued (with the particle arrays as they are
// then: a reordering swaps them) and copied to the device in stream order.
int batch_enqueue_lockstep(colapm_batch* b, int K) {
    CK(cudaMemcpyAsync(b->seeds_d, b->seeds_h, b->n * sizeof(unsigned long long), cudaMemcpyHostToDevice, b->user));
    auto fork = [&](int e) -> int {
        CK(cudaEventRecord(b->ev[e], b->user));
        for (int w = 0; w < K; ++w) CK(cudaStreamWaitEvent(b->ws[w], b->ev[e], 0));
        return COLAPM_OK;
    };
    auto join = [&]() -> int {
        for (int w = 0; w < K; ++w) {
            CK(cudaEventRecord(b->ev[1 + w], b->ws[w]));
            CK(cudaStreamWaitEvent(b->user, b->ev[1 + w], 0));
        }
        return COLAPM_OK;
    };
    int r = fork(0);
    for (int i = 0; i < b->n && !r; ++i) {
        colapm_ctx* c = b->ctx[i];
        c->stream = b->ws[i % K];
        r = colapm_make_ics(c);
    }
    if (!r) r = join();
    for (int st = 0; st < b->max_steps && !r; ++st) {
        MockWork* wh = b->work_h + (size_t)st * b->n;
        int m = 0;
        long long items = 0;
        for (int i = 0; i < b->n && !r; ++i) {
            colapm_ctx* c = b->ctx[i];
            if (st >= c->prm.n_steps) continue;
            c->stream = b->user;
            if (sort_due(c, st)) r = sort_particles(c);
            if (!c->rho_clean && cudaMemsetAsync(c->rho, 0, c->nm3 * sizeof(unsigned long long), b->user) != cudaSuccess)
                r = COLAPM_E_CUDA;
            c->rho_clean = false;
            MockWork w{};
            w.pos = c->pos;
            w.mom = c->mom;
            w.psi1 = c->psi1;
            w.psi2 = c->psi2;
            w.force = force_mesh(c);
            w.rho = c->rho;
            w.np3 = c->np3;
            w.first = items;
            w.nm = c->nm;
            w.k = coef_for(c, st);
            wh[m++] = w;
            items += multi_items(c->np3);
        }
        if (r) break;
        MockWork* wd = b->work_d + (size_t)st * b->n;
        CK(cudaMemcpyAsync(wd, wh, m * sizeof(MockWork), cudaMemcpyHostToDevice, b->user));
        CK(launch_multi_deposit(wd, m, items, b->queue_d, b->user));
        r = fork(0);
        for (int i = 0; i < b->n && !r; ++i) {
            colapm_ctx* c = b->ctx[i];
            if (st >= c->prm.n_steps) continue;
            c->stream = b->ws[i % K];
            r = force_from_density(c);
        }
        if (!r) r = join();
        if (r) break;
        CK(launch_multi_gather_kick_drift(wd, m, items, b->queue_d + 2, b->user));
        for (int i = 0; i < b->n; ++i)
            if (st < b->ctx[i]->prm.n_steps) ++b->ctx[i]->step;
    }
    if (!r) r = fork(0);
    for (int i = 0; i < b->n && !r; ++i) {
        colapm_ctx* c = b->ctx[i];
        c->stream = b->ws[i % K];
        r = power_enqueue(c, b->nbins);
        if (!r && cudaMemcpyAsync(b->acc_h + (size_t)i * 3 * b->nbins, c->pw_acc, 3 * b->nbins * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            r = COLAPM_E_CUDA;
    }
    if (!r) r = join();
    return r;
}

// Per-mock schedule: seeds, fork, per-mock ICs + steps + P(k) on worker stream i mod K, copies
// of the accumulators to the pinned buffer, join.
int batch_enqueue(colapm_batch* b, int K) {
    if (b->lockstep) return batch_enqueue_lockstep(b, K);
    CK(cudaMemcpyAsync(b->seeds_d, b->seeds_h, b->n * sizeof(unsigned long long), cudaMemcpyHostToDevice, b->user));
    CK(cudaEventRecord(b->ev[0], b->user));
    for (int w = 0; w < K; ++w) CK(cudaStreamWaitEvent(b->ws[w], b->ev[0], 0));
    for (int i = 0; i < b->n; ++i) {
        colapm_ctx* c = b->ctx[i];
        c->stream = b->ws[i % K];
        int r = colapm_make_ics(c);
        if (!r) r = colapm_step(c, -1);
        if (!r) r = power_enqueue(c, b->nbins);
        if (r) return r;
        CK(cudaMemcpyAsync(b->acc_h + (size_t)i * 3 * b->nbins, c->pw_acc, 3 * b->nbins * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    }
    for (int w = 0; w < K; ++w) {
        CK(cudaEventRecord(b->ev[1 + w], b->ws[w]));
        CK(cudaStreamWaitEvent(b->user, b->ev[1 + w], 0));
    }
    return COLAPM_OK;
}

int batch_capture(colapm_batch* b, int K) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    CK(cudaStreamBeginCapture(b->user, cudaStreamCaptureModeRelaxed));
    int r = batch_enqueue(b, K);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->user, &g);
    if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return COLAPM_E_CUDA;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? COLAPM_OK : COLAPM_E_CUDA;
}

float batch_time(colapm_batch* b) {   // one replay, ms
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->user);
    cudaGraphLaunch(b->exec, b->user);
    cudaEventRecord(e1, b->user);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

extern "C" {

int colapm_batch_create(int n, const colapm_params* ps, int nstreams, void* stream, colapm_batch** out) {
    if (!out || n < 1 || !ps || nstreams > kMaxStreams) return COLAPM_E_ARG;
    *out = nullptr;
    colapm_batch* b = new (std::nothrow) colapm_batch();
    if (!b) return COLAPM_E_NOMEM;
    b->n = n;
    b->nstreams = nstreams > 0 ? nstreams : 0;
    b->caller = static_cast<cudaStream_t>(stream);
    b->ctx.assign(n, nullptr);
    int r = COLAPM_OK;
    if (cudaStreamCreateWithFlags(&b->user, cudaStreamNonBlocking) != cudaSuccess) r = COLAPM_E_CUDA;
    for (int w = 0; w < kMaxStreams && !r; ++w) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) r = COLAPM_E_CUDA;
        else b->ws.push_back(s);
    }
    for (int w = 0; w < kMaxStreams + 1 && !r; ++w) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) r = COLAPM_E_CUDA;
        else b->ev.push_back(e);
    }
    if (!r && (cudaMallocHost(&b->seeds_h, n * sizeof(unsigned long long)) != cudaSuccess ||
               cudaMalloc(&b->seeds_d, n * sizeof(unsigned long long)) != cudaSuccess))
        r = COLAPM_E_NOMEM;
    for (int i = 0; i < n; ++i) b->max_steps = ps[i].n_steps > b->max_steps ? ps[i].n_steps : b->max_steps;
    if (!r && b->max_steps > 0 &&
        (cudaMallocHost(&b->work_h, (size_t)b->max_steps * n * sizeof(MockWork)) != cudaSuccess ||
         cudaMalloc(&b->work_d, (size_t)b->max_steps * n * sizeof(MockWork)) != cudaSuccess ||
         cudaMalloc(&b->queue_d, 4 * sizeof(unsigned long long)) != cudaSuccess ||
         cudaMemset(b->queue_d, 0, 4 * sizeof(unsigned long long)) != cudaSuccess))
        r = COLAPM_E_NOMEM;
    for (int i = 0; i < n && !r; ++i) {
        r = colapm_create(&ps[i], b->ws[0], &b->ctx[i]);
        if (!r) {
            b->ctx[i]->seed_src = b->seeds_d + i;
            b->seeds_h[i] = ps[i].seed;
        }
    }
    if (r) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return r;
    }
    *out = b;
    return COLAPM_OK;
}

int colapm_batch_run(colapm_batch* b, const unsigned long long* seeds, int nbins, double kmin, double kmax,
                     double* k_out, double* p_out, long long* nmodes_out) {
    if (!b || !k_out || !p_out || !nmodes_out || nbins < 1 || nbins > 4096) return COLAPM_E_ARG;
    CK(cudaStreamSynchronize(b->caller));   // work the caller issued before this call comes first
    if (!b->exec || nbins != b->nbins || kmin != b->kmin || kmax != b->kmax) {
        for (colapm_ctx* c : b->ctx) {
            c->stream = b->ws[0];
            int r = power_prepare(c, nbins, kmin, kmax);
            if (r) return r;
        }
        if (b->acc_h) cudaFreeHost(b->acc_h);
        b->acc_h = nullptr;
        if (cudaMallocHost(&b->acc_h, (size_t)b->n * 3 * nbins * sizeof(double)) != cudaSuccess) return COLAPM_E_NOMEM;
        b->nbins = nbins;
        b->kmin = kmin;
        b->kmax = kmax;
        // Autotune every (np, nm) of the batch that has no tuned configuration in this process yet,
        // on its first mock (after its ICs), and give the result to every mock of that size.
        for (int i = 0; i < b->n; ++i) {
            colapm_ctx* c = b->ctx[i];
            bool known = false;
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                known = g_tuned.count({c->np, c->nm}) != 0;
            }
            if (!known) {
                c->stream = b->ws[0];
                int r = colapm_make_ics(c);
                if (!r) r = colapm_autotune(c, nullptr);
                if (r) return r;
            }
            Tuned t{};
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                t = g_tuned.at({c->np, c->nm});
            }
            c->plan = t.plan;
            c->fused = t.fused;
            c->block = t.block;
        }
        // One eager pass initialises every kernel's launch configuration before capture.
        int r = batch_enqueue(b, 1);
        if (r) return r;
        CK(cudaStreamSynchronize(b->user));
        if (b->nstreams == 0) {   // choose the number of worker streams by timing replays
            float best = 1e30f;
            int bestk = 1;
            for (int k = 1; k <= kMaxStreams; k *= 2) {
                r = batch_capture(b, k);
                if (r) return r;
                batch_time(b);
                const float ms = batch_time(b);
                if (ms < best) {
                    best = ms;
                    bestk = k;
                }
            }
            b->nstreams = bestk;
        }
        r = batch_capture(b, b->nstreams);
        if (r) return r;
    }
    for (int i = 0; i < b->n; ++i) b->seeds_h[i] = seeds ? seeds[i] : b->ctx[i]->prm.seed;
    CK(cudaGraphLaunch(b->exec, b->user));
    CK(cudaStreamSynchronize(b->user));
    for (int i = 0; i < b->n; ++i) {
        colapm_ctx* c = b->ctx[i];
        int r = pending_error(c);
        if (r) return r;
        power_finish(b->acc_h + (size_t)i * 3 * nbins, nbins, k_out + (size_t)i * nbins, p_out + (size_t)i * nbins,
                     nmodes_out + (size_t)i * nbins);
    }
    return COLAPM_OK;
}

int colapm_batch_streams(const colapm_batch* b) { return b ? b->nstreams : COLAPM_E_ARG; }

int colapm_batch_set_lockstep(colapm_batch* b, int on) {
    if (!b || on < 0 || on > 1) return COLAPM_E_ARG;
    if (b->lockstep != (on == 1)) {
        b->lockstep = on == 1;
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;   // the next run captures the other schedule
    }
    return COLAPM_OK;
}

void colapm_batch_destroy(colapm_batch* b) {
    if (!b) return;
    if (b->user) cudaStreamSynchronize(b->user);
    for (cudaStream_t s : b->ws) cudaStreamSynchronize(s);
    batch_free(b);
    delete b;
}

}  // extern "C"
