/*
 * colapm.h -- C ABI of libcolapm.so, a single-GPU (GB300, sm_103a) implementation of the
 * COLA particle-mesh method of Howlett, Manera & Percival, "L-PICOLA: A parallel code for
 * fast dark matter simulation" (2015).
 *
 * The calls follow the paper's statement of the problem (§3): prepare the initial linear
 * power spectrum, generate an initial particle distribution with that power spectrum,
 * evolve it over a series of user-specified timesteps to a final redshift, and measure
 * the result.
 *
 * Conventions for every call:
 *   - Return COLAPM_OK (0) or a negative COLAPM_E_* code; nothing throws across the ABI.
 *   - A context owns all of its device memory. Arrays passed in are owned by the caller.
 *   - "host or device" arrays may be either (CUDA unified addressing decides); the call
 *     copies with cudaMemcpyAsync on the context's stream.
 *   - Work is issued on the stream given to colapm_create (0 = the legacy default
 *     stream). Calls return before the GPU finishes unless they write host data or say
 *     otherwise; a device-side error (e.g. fixed-point overflow) is reported by the next
 *     call that synchronises (colapm_sync, colapm_power, colapm_get_*).
 *   - Units: lengths in Mpc/h, wavenumbers in h/Mpc, time in 1/H0 (H0 = 1). Momenta are
 *     p = a^3 E(a) dx/da in Mpc/h (peculiar velocity in km/s = 100 p / a).
 *   - Particle arrays are in particle-id order, id = ix + Np (iy + Np iz), where
 *     (ix, iy, iz) is the particle's site on the Lagrangian lattice; xyz-interleaved
 *     ("xyz") arrays hold 3 values per particle, component-major ("c-major") arrays hold
 *     all x, then all y, then all z.
 *   - Meshes are [iz][iy][ix] with ix fastest.
 */
#ifndef COLAPM_H
#define COLAPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    COLAPM_OK = 0,
    COLAPM_E_ARG = -1,      /* invalid argument: null pointer, size out of range, bad enum      */
    COLAPM_E_NOMEM = -2,    /* device or host allocation failed                                 */
    COLAPM_E_CUDA = -3,     /* a CUDA runtime call or kernel launch failed                      */
    COLAPM_E_OVERFLOW = -4, /* a density cell reached 2^63 in the int64 fixed-point deposit     */
    COLAPM_E_TIMEOUT = -5,  /* a bounded device-side wait gave up (result of that call invalid)  */
    COLAPM_E_STATE = -6     /* call out of order (e.g. colapm_step before initial conditions)   */
};

/* Flat LCDM cosmology, Omega_Lambda = 1 - omega_m. omega_b is carried for completeness; the
 * BBKS transfer function uses Gamma = omega_m * h. sigma8 normalises P(k) at z = 0. */
typedef struct {
    double omega_m, omega_b, h, n_s, sigma8;
} colapm_cosmo;

/* Run parameters (§2.3, §2.4, §5, §7.3). */
typedef struct {
    colapm_cosmo cosmo;
    double box;                 /* box side L, Mpc/h                                            */
    int np;                     /* particles per side N_p (even, 8..1024)                       */
    int nm;                     /* PM mesh cells per side N_m (even, 16..1024): a multiple of   */
                                /* N_p, or N_p / 2 or N_p / 4 (coarser force mesh, §7.3)         */
    double z_init, z_final;     /* redshift of the 2LPT initial conditions and of the last step */
    int n_steps;                /* number of Kick-Drift steps (§2.3)                             */
    int spacing;                /* 0: steps linear in a (default), 1: logarithmic in a (§7.3)   */
    int stepping;               /* 0: modified COLA stepping, Eq. eq:modifiedt (default);        */
                                /* 1: Quinn et al. (1997) stepping (§2.3)                        */
    double nlpt;                /* n of the modified stepping (default -2.5, §1 and §7.3)       */
    int cola;                   /* 1: COLA (default); 0: plain PM (§7.1)                         */
    int deconv;                 /* powers of the CIC window divided out of the force: 0, 1, 2   */
    unsigned long long seed;    /* Philox4x32-10 key of the Gaussian field                      */
} colapm_params;

typedef struct colapm_ctx colapm_ctx;   /* opaque; owns all device memory */

/* Fill *p with the defaults above: omega_m 0.3, omega_b 0.05, h 0.7, n_s 0.96, sigma8 0.8,
 * box 256, np 32, nm 64, z_init 9, z_final 0, 10 steps, lin-a, modified, nlpt -2.5, COLA,
 * deconv 1, seed 1. */
void colapm_default_params(colapm_params* p);

/* Create a context on the current CUDA device: validates *p (COLAPM_E_ARG), computes the FP64
 * timestep table and the linear P(k) normalisation on the host, allocates every device buffer
 * (COLAPM_E_NOMEM). `stream` is a cudaStream_t (may be NULL). On success *out owns the memory
 * until colapm_destroy. */
int colapm_create(const colapm_params* p, void* stream, colapm_ctx** out);

/* Synchronise the context's stream and free everything. NULL is allowed. */
void colapm_destroy(colapm_ctx* ctx);

/* §5, §2.1: Gaussian field from Philox4x32-10 (Salmon et al. 2011) keyed by the seed, with
 * BBKS P(k) at z = 0; 1LPT and 2LPT displacements Psi1 = i k delta/k^2 and Psi2 = -i k S/k^2,
 * S = sum_{i>j}(phi_ii phi_jj - phi_ij^2) (Eqs. za, 2lpt and the Lagrangian-potential Poisson
 * equations); particles at x = q + D1(a0) Psi1 + D2(a0) Psi2 on a lattice offset by half a PM
 * cell; residual momentum 0 (COLA, §2.3) or the 2LPT momentum (plain PM). Resets the step
 * counter. */
int colapm_make_ics(colapm_ctx* ctx);

/* Set the seed of the next colapm_make_ics (a new mock realisation from the same context,
 * without reallocating). */
int colapm_reseed(colapm_ctx* ctx, unsigned long long seed);

/* §5: local primordial non-Gaussianity of the initial conditions made by the next colapm_make_ics
 * (and returned by colapm_get_gaussian_field); 0 (the default) gives the Gaussian field. The Gaussian
 * field delta_k = M(k) phi_k defines the primordial potential phi; in real space
 * Phi = phi + f_NL (phi^2 - <phi^2>) (<> the box average), and the initial density is M(k) Phi_k, with
 * M(k) = (2/3) (k c / H0)^2 T(k) D_md / Om (the Poisson equation in matter domination with the BBKS
 * transfer function and D_md the z = 0 growth normalised to a in the matter era; Phi has the sign of
 * the density, so f_NL > 0 skews it positively). The first non-zero call allocates two small tables
 * (COLAPM_E_NOMEM on failure) and synchronises; COLAPM_E_ARG for a non-finite value. */
int colapm_set_fnl(colapm_ctx* ctx, double fnl);

/* Replace the LPT displacements with caller-supplied fields on the N_p^3 Lagrangian lattice
 * (c-major, 3 * Np^3 floats each, Mpc/h, host or device) and place the particles as
 * colapm_make_ics does. Used to start from a known field (parity tests, planted modes). */
int colapm_set_displacements(colapm_ctx* ctx, const float* psi1, const float* psi2);

/* §2.3-§2.4: advance k Kick-Drift steps (k < 0: all remaining). One step at a_i: fixed-point
 * CIC deposit, FFT, Poisson/gradient/deconvolution, inverse FFT x3, CIC gather, COLA kick
 * (Eq. eq:vcola) and drift (Eq. eq:rcola). COLAPM_E_STATE before initial conditions or when
 * k exceeds the remaining steps. */
int colapm_step(colapm_ctx* ctx, int k);

/* §2.3: closing half kick to a_N (force at a_N), then add the LPT momentum back (COLA).
 * Allowed once, after the last step; afterwards colapm_get_particles returns total momenta. */
int colapm_finalize(colapm_ctx* ctx);

/* §7.1: periodic-box power spectrum of the current particles: fixed-point CIC deposit, FFT,
 * P = L^3 |delta_k|^2 / (N_m^6 W^2), W = prod sinc^2(pi n_i / N_m), binned in nbins log bins
 * with edges kmin (kmax/kmin)^(b/nbins); a mode is in bin b when e_b <= |k| < e_{b+1}; modes
 * counted over the full complex grid; k = 0 and modes with any index at N_m/2 excluded. FP64
 * sums. Outputs (caller-owned, host or device, nbins each): mean |k|, mean P, mode count.
 * kmin <= 0 selects 2 pi / L, kmax <= 0 selects pi N_m / L. Synchronises. */
int colapm_power(colapm_ctx* ctx, int nbins, double kmin, double kmax,
                 double* k_out, double* p_out, long long* nmodes_out);

/* ---- past lightcone (§6) ------------------------------------------------------------------- */
/* An observer at `origin` (Mpc/h) sees the past lightcone shrink to it: its radius at scale factor a
 * is the comoving distance R_L(a) = c int_a^1 da' / (a'^2 H(a')). The box is replicated: every
 * particle has images x + R L for integer vectors R with rep_lo <= R <= rep_hi per axis. From the
 * first step boundary at or after a(z_max), the drift of every step records each image that leaves
 * the lightcone during it (R_p <= R_L at a_i and R_p > R_L at a_{i+1}, R_p its distance to the
 * observer): its exit time a_L interpolates both radii linearly across the step
 * (Eq. eq:lightconeinterp), its position is the one the step's drift gives at a_L (Eq. eq:rcola
 * with every coefficient over [a_i, a_L]), and its momentum is the step's residual momentum (at
 * a_{i+1/2}, not interpolated, as in the paper) plus, for COLA, the LPT frame momentum at a_L. */
typedef struct {
    double origin[3];          /* observer position, Mpc/h                                      */
    double z_max;              /* redshift at which the lightcone starts (> z_final)            */
    int rep_lo[3], rep_hi[3];  /* replicate ranges per axis (at most 33 replicates per axis)    */
} colapm_lightcone;

/* One particle image leaving the lightcone: position (replicated box coordinates, Mpc/h), exit scale
 * factor, total momentum p = a^3 E dx/da (Mpc/h; velocity in km/s = 100 p / a) and particle id. */
typedef struct {
    float x, y, z, a;
    float px, py, pz;
    int id;
} colapm_lc_particle;

/* Turn the lightcone on for the steps that follow (NULL: off), with room for `capacity` output rows
 * on the device (allocated here; COLAPM_E_NOMEM if that fails). colapm_make_ics starts a new
 * lightcone (the row count returns to zero). COLAPM_E_ARG for capacity < 1, z_max <= z_final, a
 * lightcone that starts after the last step, or bad replicate ranges. Synchronises. */
int colapm_set_lightcone(colapm_ctx* ctx, const colapm_lightcone* lc, long long capacity);

/* The rows recorded so far: *count receives their number; up to max_rows of them (at most the
 * capacity) are copied to `rows` (host or device, caller-owned; may be NULL when max_rows is 0), in
 * no particular order, and *copied (may be NULL) how many were. Returns COLAPM_E_OVERFLOW when more
 * rows were recorded than the capacity holds (the extra rows are lost, *count still counts them; the
 * stored ones are copied), COLAPM_E_STATE when no lightcone is set. Synchronises. */
int colapm_get_lightcone(colapm_ctx* ctx, long long* count, colapm_lc_particle* rows, long long max_rows,
                         long long* copied);

/* §7.1: power spectrum in redshift space. Every particle is moved along the line of sight by
 * s_los = v_los / (H(a) a), v the total peculiar velocity at a_N (the run must be finalized:
 * COLAPM_E_STATE otherwise), the line of sight radial from an observer at the centre of the box
 * (los = -1, the paper's choice) or along axis los = 0, 1, 2 (plane-parallel); redshift-space
 * positions wrap periodically. Then as colapm_power (same bins, outputs and conventions); the
 * particles themselves are not moved. Synchronises. */
int colapm_power_rsd(colapm_ctx* ctx, int los, int nbins, double kmin, double kmax,
                     double* k_out, double* p_out, long long* nmodes_out);

/* §7.1: cross-correlation coefficient r(k) = <Re delta_a delta_b^*> / sqrt(<|delta_a|^2> <|delta_b|^2>)
 * of the density fields of the current particles of two contexts with the same np, nm and box (the
 * printed formula lacks the square root, without which r is not dimensionless; it is read as
 * intended). Both fields are the fixed-point CIC deposits of colapm_power on a's mesh; the sums run
 * over the modes of each bin as in colapm_power (same bins, exclusions and full-grid mode counts),
 * without the window (it is not part of the definition). Outputs (caller-owned, host or device,
 * nbins each): mean |k|, r, mode count (NaN where a bin is empty). a may equal b (r = 1).
 * COLAPM_E_ARG for mismatched sizes, COLAPM_E_STATE before initial conditions. Runs on a's stream
 * after waiting for b's; synchronises. */
int colapm_cross_correlation(colapm_ctx* a, colapm_ctx* b, int nbins, double kmin, double kmax,
                             double* k_out, double* r_out, long long* nmodes_out);

/* Positions (xyz, Mpc/h, in [0, L)) and momenta (xyz, Mpc/h) of all particles; either pointer
 * may be NULL. Host or device. Synchronises. */
int colapm_get_particles(colapm_ctx* ctx, float* pos, float* mom);

/* The same catalogue into host memory (3 * Np^3 floats each, caller-owned; page-locked memory lets
 * the copy run asynchronously), without waiting for it: the particles are exported on the
 * context's stream into a device staging array of the context (6 * Np^3 floats, allocated on the
 * first call, COLAPM_E_NOMEM if that fails) and copied out on a separate copy stream, so the copy
 * overlaps the work the caller enqueues next (e.g. the next mock). The host arrays must not be
 * read or freed before colapm_wait_particles returns. A later call waits on the device (not the
 * host) for the previous copy to leave the staging array. Either pointer may be NULL. */
int colapm_get_particles_async(colapm_ctx* ctx, float* pos, float* mom);

/* Block the host until the copy of the last colapm_get_particles_async has landed; then report
 * any pending device error like the synchronising calls. */
int colapm_wait_particles(colapm_ctx* ctx);

/* Raw particle state: integer mesh cell (xyz int32), offset in [0,1) cells (xyz float) and
 * momentum in mesh units (xyz float, Mpc/h divided by the cell size). Any pointer may be NULL.
 * Host or device. Synchronises. */
int colapm_get_state(colapm_ctx* ctx, int* cell, float* offset, float* mom_cells);

/* Overwrite positions with integer cells (xyz int32, each in [0, Nm)) and offsets (xyz float,
 * each in [0, 1)); COLAPM_E_ARG if any is out of range (checked on the device, reported by
 * this call, which synchronises). Host or device. */
int colapm_set_state(colapm_ctx* ctx, const int* cell, const float* offset, const float* mom_cells);

/* Displacement Psi = x - q of every particle (xyz-interleaved [Np^3][3], Mpc/h, host or device),
 * with the minimum-image convention and q the particle's site on the Lagrangian lattice (spacing
 * L/Np, offset by half a PM cell). colapm_get_displacement writes it; colapm_set_displacement
 * moves every particle to x = q + Psi (wrapped into the box) and leaves momenta and the step
 * count alone, so that e.g. colapm_power measures a corrected field. |Psi| must stay below L;
 * otherwise COLAPM_E_ARG (reported by this call, which synchronises). */
int colapm_get_displacement(colapm_ctx* ctx, float* psi);
int colapm_set_displacement(colapm_ctx* ctx, const float* psi);

/* Deposit the current particles and copy the int64 fixed-point density (Nm^3, weight of one
 * particle = 2^45) to `mesh` (host or device). Synchronises. */
int colapm_get_density(colapm_ctx* ctx, long long* mesh);

/* Compute the mesh force of the current particles (§2.4 steps 1-3, mesh units: cells) and copy
 * the three real meshes (c-major, 3 * Nm^3 floats) to `force`, host or device. Synchronises. */
int colapm_get_force(colapm_ctx* ctx, float* force);

/* Copy the LPT displacement fields (c-major, 3 * Np^3 floats each, Mpc/h) to psi1 / psi2
 * (either may be NULL). Synchronises. */
int colapm_get_lpt(colapm_ctx* ctx, float* psi1, float* psi2);

/* Copy the initial Gaussian field on the half grid [iz][iy][ix], ix < Np/2, as interleaved
 * (re, im) floats (Np * Np * Np/2 complex) to `dk`, host or device. Synchronises. */
int colapm_get_gaussian_field(colapm_ctx* ctx, float* dk);

/* Wait for the context's stream and report any pending device-side error. */
int colapm_sync(colapm_ctx* ctx);

/* Number of steps taken so far, and the total. */
int colapm_steps_done(const colapm_ctx* ctx);

/* Checkpoint / resume of the particle state, step counter and LPT fields: with buf == NULL,
 * *n receives the byte size; otherwise *n must be at least that size and buf (host) receives
 * the state. colapm_load_state restores a buffer written by a context with the same np, nm.
 * Both synchronise. */
int colapm_save_state(colapm_ctx* ctx, void* buf, size_t* n);
int colapm_load_state(colapm_ctx* ctx, const void* buf, size_t n);

/* Per-phase device timing with CUDA events (off by default). When on, each phase of every
 * call is bracketed by events on the context's stream. colapm_get_timing copies, for each
 * of the COLAPM_PHASE_COUNT phases, the summed milliseconds and the launch count, then
 * clears them (synchronises). */
enum {
    COLAPM_PHASE_DEPOSIT = 0,   /* fixed-point CIC deposit of a force computation   */
    COLAPM_PHASE_FFT_FWD,       /* x and y forward passes of a force computation    */
    COLAPM_PHASE_POISSON,       /* z forward, Green/gradient/deconvolution, z inverse */
    COLAPM_PHASE_FFT_INV,       /* y inverse pass of the forces (both inverse passes
                                   with the fused x-y engine)                       */
    COLAPM_PHASE_GATHER,        /* CIC gather + kick + drift                        */
    COLAPM_PHASE_ICS,           /* initial conditions                               */
    COLAPM_PHASE_POWER,         /* all of colapm_power: its deposit, forward passes,
                                   z transform and binning                          */
    COLAPM_PHASE_FFT_INV_X,     /* x inverse pass of the three forces (c2r)         */
    COLAPM_PHASE_SORT,          /* reordering of the particle arrays by mesh cell   */
    COLAPM_PHASE_COUNT
};
int colapm_set_timing(colapm_ctx* ctx, int on);
int colapm_get_timing(colapm_ctx* ctx, double* ms, long long* launches);

/* Number of CUDA kernels this context has launched so far (memsets and copies excluded). */
long long colapm_kernel_launches(const colapm_ctx* ctx);

/* ---- autotuning ------------------------------------------------------------------------- */
/* The mesh passes of a force computation, each on the two-stage register FFT (bit set) or on the
 * multi-stage shared-memory Stockham FFT (bit clear). A pass whose line length has no two-stage
 * plan (the lengths 64, 96, 128, 160, 192, 256, 320, 384, 512, 1024 have one: two radices in
 * {8, 10, 12, 16, 20, 24, 32}) runs on the Stockham plan either way. The initial-condition
 * transforms on the particle grid take the same choice per kind of pass. */
#define COLAPM_PLAN_XF 1u    /* forward x pass (r2c of the density)                  */
#define COLAPM_PLAN_Y 2u     /* y passes, both directions                             */
#define COLAPM_PLAN_Z 4u     /* z passes (Poisson operator fused; power spectrum)     */
#define COLAPM_PLAN_XI 8u    /* inverse x pass (c2r of the forces)                    */
#define COLAPM_PLAN_ALL 15u  /* the default                                           */

/* Time the candidate configurations of this context on its current state, keep the fastest, and
 * remember it for later contexts (and batches) with the same (np, nm) in this process:
 *   1. the FFT engine -- fused x-y passes through an L2-resident ring (N_m = 512 and 1024), every
 *      pass two-stage, or every pass Stockham -- times the block size of the particle kernels
 *      (128, 256, 512);
 *   2. then, unless the fused passes won, the radix plan of each pass (COLAPM_PLAN_* bits) in
 *      turn: a pass switched to the other plan is kept if the step gets faster;
 *   3. where the context reorders its particles (colapm_set_sort), the tile shape of the sort key
 *      (colapm_set_sort_tiles: 1, 2, 4, 8) and, for tiles, the tiled or the plain deposit
 *      (colapm_set_deposit_tiles): the particles are sorted with each key.
 * Each candidate is one force computation and gather from the same state (fastest of three after a
 * warm-up); the particle state and step counter are then restored, except that step 3 leaves the
 * particles in the order of the key kept (no result depends on the order). Requires initial conditions
 * (COLAPM_E_STATE). Synchronises. `choice` (may be NULL, else 3 ints) receives {1 if every pass is
 * two-stage else 0, block, fused x-y passes (0 or 3)}; colapm_get_config gives the whole choice. */
int colapm_autotune(colapm_ctx* ctx, int* choice);

/* Select the configuration explicitly (e.g. to compare engines or to pin a choice): fused x-y
 * passes as a bit mask (1 forward, 2 inverse, 3 both; default 0; ignored where N_m has none),
 * two-stage register FFT in every pass (else Stockham in every pass) and the particle-kernel
 * block size (128, 256 or 512); COLAPM_E_ARG otherwise. All engines compute the same transforms
 * and agree to FP32 rounding. */
int colapm_set_engine(colapm_ctx* ctx, int fused, int two_stage, int block);

/* Select the plan per pass: a mask of COLAPM_PLAN_* bits (two-stage where set). The blocked
 * half-spectrum layout of the 512^3 and 1024^3 meshes needs every pass two-stage; any other mask
 * uses the plain layout there. COLAPM_E_ARG outside 0 ... COLAPM_PLAN_ALL. */
int colapm_set_plan(colapm_ctx* ctx, int plan);

/* The context's configuration: cfg (7 ints) = {plan mask, particle-kernel block size, fused x-y
 * passes (0 where N_m has none), reordering period (0: never), sort-key tile T (1: rows), tiled
 * deposit (0/1), step of the first reordering}. */
int colapm_get_config(const colapm_ctx* ctx, int* cfg);

/* Reorder the particle arrays by mesh cell before every `every`-th step (0: never). The default is
 * once, before step 2 n_steps / 5 (step 4 of 10), on meshes of 512^3 cells and more, else never. The analogue of the paper's particle migration (§4),
 * which keeps each rank's particles with its slab of the mesh: here it keeps a warp's particles
 * on neighbouring mesh cells, so that the deposit and the gather read and write runs of cells as
 * structure grows. It is a counting sort of all particle arrays by bucket (z, y, x / 64) of the
 * particle's cell; results do not depend on it (every step is per particle or an exact integer
 * sum), and calls that take or return particle arrays still use particle-id order.
 * COLAPM_E_ARG for every < 0. */
int colapm_set_sort(colapm_ctx* ctx, int every);

/* Order of the reordering: runs of 64 cells along x numbered tile by tile, tiles of 64 x T x T
 * cells (T = 1, 2, 4 or 8, N_m a multiple of T; 1 is plain rows; the default is 2, which measured
 * fastest for the gather and the sort itself at 1024^3): the particles of a tile are then
 * contiguous. COLAPM_E_ARG for other T. Takes effect at the next reordering; T = 1
 * also turns the tiled deposit off. */
int colapm_set_sort_tiles(colapm_ctx* ctx, int t);

/* Deposit tiles of 64 x T x T cells (T = 2, 4 or 8, N_m a multiple of T; 0: none, the default).
 * Sets the sort key's tiles to T (colapm_set_sort_tiles), and while the particles are in that
 * order the deposit gives each tile's particles to one CTA, which adds
 * their corners inside the tile and its +1 halo into shared memory with 64-bit shared atomics and
 * then adds the (T + 1)^2 x 65 region to the mesh, one atomic per non-zero cell; corners of
 * particles that moved out of that region since the sort go straight to the mesh. The mesh is the
 * same integer sum bit for bit (the analogue of the paper's per-rank density slab, §4: each tile is
 * summed where its particles are, then added into the global mesh). It pays where many
 * particles share cells; at 1/8 particle per cell (N_m = 2 N_p) it measured slower than the plain
 * deposit. Takes effect at the next reordering; 0 turns it off (the sort key stays). COLAPM_E_ARG
 * for other T. */
int colapm_set_deposit_tiles(colapm_ctx* ctx, int t);

/* ---- batched mocks (many independent realisations of uneven sizes) ----------------------- */
typedef struct colapm_batch colapm_batch;   /* opaque; owns its contexts and graph */

/* Create one context per entry of ps[0..n-1] (any mix of sizes), spread over `nstreams` worker
 * streams (nstreams <= 0: choose by timing 1, 2, 4 and 8 at the first run). The batch captures
 * and launches on streams of its own; each run first waits for the caller's `stream`.
 * Errors as colapm_create; everything created so far is freed on failure. */
int colapm_batch_create(int n, const colapm_params* ps, int nstreams, void* stream, colapm_batch** out);

/* Run every mock: 2LPT initial conditions from seeds[i] (host array of n seeds; NULL: the seeds
 * in ps), all n_steps COLA steps, and the P(k) of each mock in nbins bins (kmin/kmax <= 0: the
 * per-mock defaults of colapm_power). The whole batch is captured once into a CUDA graph (per
 * nbins/kmin/kmax) and replayed; seeds reach the graph through a pinned buffer, so each run is
 * a new set of realisations. Before the first capture, every (np, nm) of the batch without a
 * tuned configuration in this process is autotuned on its first mock (colapm_autotune) and the
 * choice given to all mocks of that size. Outputs are host arrays of n * nbins (mock-major).
 * Synchronises. */
int colapm_batch_run(colapm_batch* b, const unsigned long long* seeds, int nbins, double kmin, double kmax,
                     double* k_out, double* p_out, long long* nmodes_out);

/* Worker streams in use (after the first run when chosen automatically). */
int colapm_batch_streams(const colapm_batch* b);

/* Schedule of the batch's steps. on = 1 (the default): lockstep -- the mocks advance one step at a
 * time together; each step is one multi-mock deposit of every mock still running, the mesh passes
 * of each mock, and one multi-mock gather-kick-drift. The two multi-mock kernels are persistent:
 * their CTAs take work items (mock, chunk of 256 particles) from a ticket counter across all the
 * mocks, whatever their sizes. on = 0: each mock runs its ICs, steps and P(k) in turn (on worker
 * streams). Both give the same particles bit for bit (the per-particle code is the same and the
 * fixed-point deposit does not depend on order), and the same P(k) up to the order of its FP64 bin
 * sums, which are atomic and so not fixed from run to run (about 1e-16 relative). The next run captures the chosen schedule.
 * COLAPM_E_ARG for other values. */
int colapm_batch_set_lockstep(colapm_batch* b, int on);

void colapm_batch_destroy(colapm_batch* b);

/* Power spectrum of caller-owned particle positions without any allocation.
 *
 * The paper has no counterpart: this is a library convenience. It is for callers that cannot
 * call cudaMalloc -- code that runs inside another framework's device-memory budget or custom
 * allocator, or in a loop where cudaMalloc's implicit device synchronisation is not allowed --
 * and so cannot create a context. It computes what colapm_power computes (same deposit,
 * transform, binning and FP64 sums) for `n_particles` positions given as integer mesh cells
 * (`cell`, xyz int32, each in [0, nm)) and offsets (`offset`, xyz float, each in [0, 1)), both
 * DEVICE arrays of the current device (or managed memory), owned by the caller; the mean density
 * is n_particles / nm^3 per cell. Outputs (nbins each, host or device): mean |k|, mean P, mode
 * count. kmin <= 0 selects 2 pi / box, kmax <= 0 selects pi nm / box. A cell whose fixed-point
 * mass reaches 2^63 (2^18 particles) returns COLAPM_E_OVERFLOW.
 *
 * All working memory lives in one fixed device array inside the library, sized for
 * nm <= COLAPM_NOALLOC_MAX_NM (one of 16, 32, 64, 96, 128) and nbins <= COLAPM_NOALLOC_MAX_BINS;
 * larger sizes, host input arrays, arrays on another GPU or positions out of range return
 * COLAPM_E_ARG. Every GPU
 * that loads the library holds that array (about 25 MB) until the process exits. The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine). Every call
 * shares the array and leaves the last call's contents in it; each call clears what must
 * start at zero. Calls that overlap on the GPU (e.g. on two unordered streams) race on the
 * array and must not be issued. The first call on a device looks up the array's device
 * address for that device (once) and should come before any stream capture. Work runs on
 * `stream` (a cudaStream_t, may be NULL); the call synchronises that stream before returning,
 * also when it fails after queueing work. */
#define COLAPM_NOALLOC_MAX_NM 128
#define COLAPM_NOALLOC_MAX_BINS 512
int colapm_power_noalloc(const int* cell, const float* offset, long long n_particles, int nm, double box,
                         int nbins, double kmin, double kmax, double* k_out, double* p_out,
                         long long* nmodes_out, void* stream);

/* Static message for an error code. */
const char* colapm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* COLAPM_H */
