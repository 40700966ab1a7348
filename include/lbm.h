/*
 * lbm.h - C ABI of the GB300 nested-grid lattice Boltzmann library (liblbm.so).
 *
 * The library advances the fused stream-and-collide update of
 *   - D3Q19 MRT with a Smagorinsky eddy viscosity (Section 2: Eqs. MRT,
 *     relaxationTau, eqSmago, eqStrainRate, eqTauTotFinal, EqnQ; Table 1), and
 *   - D3Q27 factorized cascaded (central-moment) collision (Section 2, Table 2),
 * on a block-structured grid of 8^3-cell blocks with time-nested 2:1
 * refinement after Yu et al. (Sections 1 and 3.2).  All arithmetic runs in
 * CUDA kernels on the calling thread's current device.
 *
 * Conventions for every entry point
 *   - Return value: LBM_OK (0) or a negative lbm_status.  Nothing throws.
 *     lbm_last_error() returns a message for the last failure on a context.
 *   - The context owns all device memory it allocates.  The caller owns every
 *     buffer it passes; host buffers may be pageable or pinned.
 *   - Calls are ordered on the context's stream.  lbm_step() only enqueues
 *     work; every call that returns data to the host synchronises the stream.
 *   - Dense per-level arrays are row-major with x fastest: index
 *     x + NX_l * (y + NY_l * z), NX_l = 8 * nbx * 2^l (likewise y, z).
 *     Distribution arrays are [Q][NZ_l][NY_l][NX_l] in the velocity order of
 *     the paper's D3Q19 / D3Q27 tables, vectors [3][NZ_l][NY_l][NX_l].
 *   - Distributions exchanged with the host are float64 and unshifted: the
 *     D3Q19 model stores the incompressible distribution whose sum is
 *     delta rho (Section 2), the D3Q27 model the full distribution (sum rho).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_LEVELS 4
#define LBM_BLOCK 8

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,       /* invalid argument or grid; nothing was changed        */
  LBM_ERR_OOM = -2,       /* device or host allocation failed                      */
  LBM_ERR_CUDA = -3,      /* a CUDA call failed (no device, launch error, ...)     */
  LBM_ERR_TIMEOUT = -4,   /* reserved: a bounded device wait gave up               */
  LBM_ERR_NONFINITE = -5, /* NaN/Inf in an input or in the audited state          */
  LBM_ERR_STATE = -6      /* call not valid in the context's current state        */
} lbm_status;

typedef enum { LBM_D3Q19_MRT_LES = 0, LBM_D3Q27_FCLB = 1 } lbm_model;

/* Storage of the distributions in device memory.  They are stored shifted by
 * the lattice weights (f_i - w_i for D3Q27; the D3Q19 incompressible
 * distribution is already a fluctuation); F16 stores (f_i - w_i)/w_i.
 * Collision arithmetic is float64 for F64 and float32 otherwise. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2 } lbm_storage;

/* Block grid.  Level 0 has nbx*nby*nbz blocks of 8^3 cells; y and z are
 * periodic unless walls says otherwise.  x is periodic when periodic_x != 0;
 * otherwise the face x = 0 is a velocity inflow (lbm_set_inflow; rest
 * velocity until called) and the face x = NX a zero-gradient outflow.
 * refine concatenates, for l = 0..levels-2, one byte per level-l block
 * (nbx*2^l by nby*2^l by nbz*2^l, x fastest): 1 = the block is split into 8
 * level-(l+1) blocks.  Rules (checked): flags only on blocks of level l; each
 * level l < levels-1 refines at least one block; for l >= 1 every block
 * touching a refined block belongs to level l (so interpolation stencils stay
 * inside level l).
 *
 * Walls (Section 3.2: the tank's no-slip walls and free-slip top): walls has
 * bit 0/1 for the low/high y face and bit 2/3 for the low/high z face; the
 * faces of y or z are walls together or not at all.  slip marks the
 * free-slip walls among them (a subset of those bits); the others are
 * no-slip.  With a non-periodic x, bit 4 makes the face x = 0 and bit 5 the
 * face x = NX a no-slip wall (the tank's upstream wall behind the nozzle, a
 * closed box); they replace the inflow / outflow for the populations
 * entering there, and bit 5 excludes the pressure outlet.  A pull that would cross a wall face is reflected: no-slip by
 * half-way bounce-back, f_i(x, t+1) = f~_opp(i)(x, t) (the wall lies half a
 * cell outside the boundary cells); free-slip by specular reflection, the
 * population with its wall-normal components flipped pulled along the other
 * axes, f_i(x, t+1) = f~_m(i)(x - e_i + (e_i . n) n, t).  A no-slip crossing
 * wins over a free-slip one; two free-slip crossings flip both components.
 * Refined level-0 blocks must keep one block away from every wall face
 * (checked).  walls = slip = 0 (a zero-initialised struct) keeps y and z
 * periodic.
 *
 * Outlet (Section 3.2 holds the tank's outflow at a fixed pressure): outlet
 * = 0 keeps the zero-gradient outflow; outlet = 1 (non-periodic x only)
 * makes the face x = NX a pressure outlet whose ghost cells hold the
 * equilibrium at the outlet density (lbm_set_outlet; 1 until called) with
 * the velocity of the cell x = NX - 1 plus that cell's non-equilibrium part,
 * f_ghost = f_eq(rho_out, u_N) + f_N - f_eq(rho_N, u_N).  Refined level-0
 * blocks must keep one block away from that face (checked).
 *
 * Nozzle (Section 3.2: a cylinder along the jet axis with second-order
 * interpolated no-slip walls after Bouzidi et al.; its downstream end emits
 * the jet): nozzle_r > 0 makes the closed cylinder x0 <= x <= x1,
 * (y - y0)^2 + (z - z0)^2 <= r^2 (coarse-cell units; cells whose centre lies
 * in it) solid.  Its surface is a no-slip wall by Bouzidi's linear
 * interpolation: a link from fluid cell f to solid cell f + e_i cut at the
 * fraction q takes 2q f~_i(f) + (1 - 2q) f~_i(f - e_i) for q < 1/2
 * (f~_i(f) if f - e_i is solid) and f~_i(f)/(2q) + (2q - 1)/(2q) f~_ib(f)
 * otherwise.  Links that enter through the downstream cap x = x1 carry the
 * inflow instead: the disc inflow of lbm_set_inflow moves from the face
 * x = 0 onto the cap (the solid cell takes f_eq(rho of the fluid cell
 * downstream, u_bc at its own y, z)) and the face x = 0 holds u = 0.  The
 * body lives on one level: the finest whose blocks cover the cylinder grown
 * by two of its cells, each of them and its 26 neighbours being non-refined
 * blocks of that level (checked; lbm_plan_info.nozzle_level). */
typedef struct {
  int nbx, nby, nbz;
  int periodic_x;
  int levels;
  const uint8_t* refine;
  int walls; /* wall faces, see above; 0 = periodic y and z */
  int slip;  /* free-slip subset of walls */
  int outlet; /* 0 zero-gradient outflow, 1 fixed-pressure outlet */
  double nozzle_y0, nozzle_z0, nozzle_r, nozzle_x0, nozzle_x1; /* nozzle_r <= 0: none */
} lbm_grid;

/* Sizes of a grid, computed on the host without touching a GPU. */
typedef struct {
  int levels;
  int64_t blocks[LBM_MAX_LEVELS];        /* allocated blocks (level + ghost blocks) */
  int64_t level_blocks[LBM_MAX_LEVELS];  /* blocks belonging to the level           */
  int64_t active_cells[LBM_MAX_LEVELS];  /* cells of unrefined level blocks         */
  int64_t updated_cells[LBM_MAX_LEVELS]; /* active + hidden layer 1                 */
  int64_t hidden_cells[LBM_MAX_LEVELS];  /* hidden layers 1 and 2                   */
  int64_t ghost_cells[LBM_MAX_LEVELS];   /* coarse-to-fine ghost cells              */
  int64_t bc_cells[LBM_MAX_LEVELS];      /* inflow (x = -1) and pressure-outlet     */
                                         /* (x = NX) ghost cells                    */
  int64_t updates_per_coarse_step;       /* sum_l updated_cells[l] * 2^l            */
  int64_t active_updates_per_coarse_step;/* sum_l active_cells[l] * 2^l             */
  int64_t device_bytes;                  /* device memory lbm_create would allocate */
  int nozzle_level;                      /* level holding the nozzle, -1 if none    */
  int64_t solid_cells;                   /* cells inside the nozzle                 */
  int64_t nozzle_links;                  /* links of its surface and cap            */
} lbm_plan_info;

/* Plan a grid on the host (no CUDA call).  Validates g like lbm_create.
 * model/storage are lbm_model/lbm_storage values (they set device_bytes). */
int lbm_plan(const lbm_grid* g, int model, int storage, lbm_plan_info* out);

/* Create a solver.  omega = 1/tau_0 of level 0 (viscosity nu = (1/omega - 1/2)/3,
 * Eq. relaxationTau in lattice units); level l uses tau_l - 1/2 = 2^l (tau_0 - 1/2)
 * (constant CFL, Section 3.2).  cs = Smagorinsky constant (Eq. eqSmago; 0 = none;
 * ignored by FCLB).  cuda_stream = a cudaStream_t or NULL (the library then
 * creates its own).  Every cell starts at rest (rho = 1, u = 0).
 * On failure *out is NULL and nothing is leaked; lbm_create_error() describes it. */
int lbm_create(lbm_ctx** out, lbm_model model, lbm_storage storage, const lbm_grid* g,
               double omega, double cs, void* cuda_stream);

/* Message of the last lbm_create or lbm_shard_create failure on this thread ("" if none). */
const char* lbm_create_error(void);

/* Top-hat inflow on the face x = 0 (Section 3.2 names a constant inflow
 * velocity; the disc and perturbation are this library's setup): ghost
 * x = -1 holds f_eq(rho of cell x = 0, u_bc), u_bc = u_in (1 + p xi_x, p xi_y,
 * p xi_z) where the cell centre lies within diameter/2 of (y0, z0) (coarse cell
 * units), else 0; xi in [-1, 1) from SplitMix64 of (seed, coarse step, level,
 * substep, y + NY_l z, component).  LBM_ERR_STATE if x is periodic. */
int lbm_set_inflow(lbm_ctx* ctx, double y0, double z0, double diameter, double u_in,
                   double perturb, uint64_t seed);

/* Density held at the pressure outlet (full density for both models; the
 * D3Q19 model holds delta rho = rho_out - 1).  LBM_ERR_STATE if the grid has
 * no pressure outlet (lbm_grid.outlet = 0); LBM_ERR_ARG unless 0.5 < rho_out
 * < 2; LBM_ERR_NONFINITE on NaN/Inf.  Takes effect at the next lbm_step. */
int lbm_set_outlet(lbm_ctx* ctx, double rho_out);

/* f = f_eq(rho, u) on every in-domain cell of a level (host arrays: rho
 * [NZ][NY][NX], u [3][NZ][NY][NX]; NULL = rest).  rho is the full density for
 * both models.  Hidden cells of coarser levels are refreshed by restriction
 * before the next step.  LBM_ERR_NONFINITE on NaN/Inf input. */
int lbm_init_equilibrium(lbm_ctx* ctx, int level, const double* rho, const double* u);

/* Per-cell body force F (host, [3][NZ][NY][NX], float64) on a single-level D3Q27
 * grid: u = (sum f e + F/2)/rho in the collision frame and the post-collision
 * momentum gains F.  NULL removes the force. */
int lbm_set_force(lbm_ctx* ctx, const double* F);

/* Advance coarse_steps coarse time steps (each level l takes 2^l substeps per
 * coarse step).  Enqueues one CUDA graph per coarse step. */
int lbm_step(lbm_ctx* ctx, int coarse_steps);

/* Wait for all enqueued work; reports launch/runtime errors. */
int lbm_sync(lbm_ctx* ctx);

/* rho and u (host, float64, dense per level) of every cell that holds a value
 * of the level (unrefined cells and hidden layers); NaN elsewhere. */
int lbm_macroscopic(lbm_ctx* ctx, int level, double* rho, double* u);

/* Time statistics of the flow (the paper's jet evaluation quantities are
 * time averages: mean velocity along the centreline, spreading, turbulence
 * intensity, Section 3.3).  lbm_stats_reset allocates (first call) and zeroes
 * float64 sums of rho, u and u_a^2 per cell of every level (56 bytes per
 * allocated cell); lbm_stats_accumulate adds one sample of the current state
 * of every level (enqueued, no synchronisation); lbm_stats_get returns, for
 * one level, the means mean[4][NZ][NY][NX] = (rho, u_x, u_y, u_z) and the
 * variances var[3][NZ][NY][NX] = <u_a^2> - <u_a>^2 over the samples, NaN where
 * a cell holds no value of the level, and the sample count.  u is taken as in
 * lbm_macroscopic without a body force.  LBM_ERR_STATE before any sample. */
int lbm_stats_reset(lbm_ctx* ctx);
int lbm_stats_accumulate(lbm_ctx* ctx);
int lbm_stats_get(lbm_ctx* ctx, int level, double* mean, double* var, int64_t* nsamples);

/* The jet's radial profiles on cross-sections (Section 3.3 evaluates the
 * mean axial velocity, the spreading width, the radial Gaussian profile and
 * the turbulence intensity), computed on the device from the accumulated
 * statistics of one level.  For station s (x[s] in coarse-cell units: the
 * layer of level cells containing it) and ring b (cell centres at distance
 * r in [b dr, (b + 1) dr) from the axis (y0, z0), coarse units), over the
 * cells of the layer that hold a value of the level: counts[s][b],
 * mean_ux[s][b] the average of the time mean of u_x and var_ux[s][b] the
 * average of its time variance (NaN for empty rings).  level = -1 takes
 * every level of a nested grid: the unrefined cells of each level l in its
 * layer containing x, weighted by their cross-section area 4^-l (they tile
 * the plane), the values being area-weighted ring averages.  Arrays are
 * [nstations][nbins].  The ring sums are float64 atomics, so their order
 * (and the last bit of a ring's value) may vary between calls.
 * LBM_ERR_STATE before any sample; LBM_ERR_ARG for a station outside the
 * level or dr <= 0. */
int lbm_stats_radial(lbm_ctx* ctx, int level, double y0, double z0, double dr, int nbins, int nstations,
                     const double* x, double* mean_ux, double* var_ux, int64_t* counts);

/* Jet quantities of one station's ring profile (host arithmetic, no
 * context): out = {u_m, b_e, tI, a, c} with u_m the value of ring 0, b_e the
 * half width where the profile falls to u_m / e (0.368 u_m; linear between
 * the centres (b + 1/2) dr of the first ring at or below it and the ring
 * before), tI = sqrt(max(var_0, 0)) / u_m, and a, c the least-squares fit
 * u / u_m = a exp(-c (r / b_e)^2) of ln(u / u_m) over the rings with cells,
 * u >= 0.05 u_m and r <= 2 b_e (the paper quotes a = 0.938, c = 0.944).
 * Undefined entries are NaN.  LBM_ERR_ARG for NULL or nbins < 1. */
int lbm_jet_fit(int nbins, double dr, const double* mean_ux, const double* var_ux, const int64_t* counts,
                double out[5]);

/* Float64 sums over the unrefined cells of all levels, weighted by the cell
 * volume 8^-l: out = {sum (rho - 1), sum j_x, sum j_y, sum j_z}, j = sum f e.
 * LBM_ERR_NONFINITE if any summed value is NaN/Inf. */
int lbm_mass_momentum(lbm_ctx* ctx, double out[4]);

/* Dense float64 copy of a level's distributions, count = Q*NX*NY*NZ doubles.
 * Cells outside the level's blocks read NaN; cells inside the nozzle hold the
 * values its links last wrote (no fluid state; lbm_macroscopic gives NaN
 * there).  The stored (shifted) values are
 * read exactly; for D3Q27 the unshifted sum f = (f - w) + w can round away
 * the lowest bits of a deviation far below w, so use the raw state below for
 * bit-exact checkpoints. */
int lbm_get_state(lbm_ctx* ctx, int level, double* f, size_t count);

/* Inverse of lbm_get_state (rounds to the storage type).  NaN entries and
 * cells outside the level are ignored.  Clears the pending restriction. */
int lbm_set_state(lbm_ctx* ctx, int level, const double* f, size_t count);

/* Bit-exact checkpoint of a level: the level's device state as stored (the
 * current distribution buffer of the whole level box, then the strain buffer
 * of nested D3Q19 runs).  The layout is the library's and may change between
 * versions; bytes must equal lbm_raw_state_bytes.  Together with
 * lbm_get_step / lbm_set_step it resumes a run bit for bit when the resumed
 * context runs the same stream-collide variant (lbm_get_tuning of the saved
 * context, passed as LBM_LAUNCH_SHAPE): variants compiled for another
 * register cap may round a few operations differently. */
int lbm_raw_state_bytes(const lbm_ctx* ctx, int level, size_t* bytes);
int lbm_get_raw_state(lbm_ctx* ctx, int level, void* buf, size_t bytes);
int lbm_set_raw_state(lbm_ctx* ctx, int level, const void* buf, size_t bytes);

/* Per-cell strain-rate norm |S| (Eq. eqStrainRate) of the last collision,
 * dense float64 [NZ][NY][NX], count = NX*NY*NZ.  It is state only for nested
 * D3Q19 Smagorinsky runs (it sets the relaxation times used by the interface
 * transfer); elsewhere get returns zeros and set does nothing. */
int lbm_get_strain(lbm_ctx* ctx, int level, double* S, size_t count);
int lbm_set_strain(lbm_ctx* ctx, int level, const double* S, size_t count);

/* Distributions of n sampled cells (level-local dense indices) into f[n][Q]. */
int lbm_get_cells(lbm_ctx* ctx, int level, size_t n, const int64_t* cells, double* f);

/* Coarse steps taken so far (drives the inflow random numbers); settable for
 * checkpoint/resume. */
int lbm_get_step(const lbm_ctx* ctx, int64_t* step);
int lbm_set_step(lbm_ctx* ctx, int64_t step);

/* Discrete adjoint of the forced D3Q27 FCLB update (single periodic level,
 * F32 or F64 storage; the paper has no adjoint: this serves gradient-based
 * studies of the same update).  Two phases: lbm_adjoint_forward advances T
 * steps from the current state (with the force of lbm_set_force) and records
 * what the backward sweep needs; the final state is then the context's state.
 * lbm_adjoint_backward takes dL/df_T (host, float64, dense [27][NZ][NY][NX],
 * w.r.t. the distributions after step T) and returns dL/dF (host, float64,
 * dense [3][NZ][NY][NX]) of a force held constant over the T steps, sweeping
 * the steps backwards with the adjoint stream-collide kernel.
 *   checkpoint_every = 1: every step's input state is kept (the forward
 *     writes each step straight into its slot); the backward sweep needs no
 *     recomputation.  Device memory: T + 2 states plus dL/dF.
 *   checkpoint_every = k > 1: sqrt(T)-style checkpointing; a copy of the
 *     state every k steps, each segment recomputed from its checkpoint
 *     before its backward sweep.  Device memory: (T/k + k + 2) states.
 *   checkpoint_every = 0: the library chooses 1 when T + 2 states fit in
 *     half of the free device memory (counting adjoint buffers it already
 *     holds), else ceil(sqrt(T)).
 * lbm_adjoint_forward returns LBM_ERR_OOM, with every adjoint buffer freed,
 * when an allocation fails.  lbm_set_force and a failed forward discard the
 * recorded forward: lbm_adjoint_backward then returns LBM_ERR_STATE, as it
 * does for other grids or models or without a forward. */
int lbm_adjoint_forward(lbm_ctx* ctx, int T, int checkpoint_every);
/* Number of completed lbm_adjoint_forward calls on ctx while the last one's
 * record is valid, else 0; a caller that keeps several forwards apart (an
 * autograd graph) compares it before lbm_adjoint_backward.  checkpoint_every
 * (may be NULL) receives the spacing that forward used (0 if none). */
int lbm_adjoint_generation(const lbm_ctx* ctx, uint64_t* generation, int* checkpoint_every);
int lbm_adjoint_backward(lbm_ctx* ctx, const double* dLdf_T, double* dLdF);

/* Kernel timing: when enabled, lbm_step launches kernels directly (no graph)
 * between CUDA events on the context stream and accumulates per-kind device
 * time.  kinds: 0 update (stream-collide), 1 coarse-to-fine, 2 fine-to-coarse,
 * 3 boundary, 4 other (an lbm_adjoint_backward call adds the device time of
 * its recompute + adjoint sweep here as one entry).  ms[k] total
 * milliseconds, launches[k] launch counts. */
int lbm_set_profiling(lbm_ctx* ctx, int enable);
int lbm_get_profile(lbm_ctx* ctx, double ms[5], int64_t launches[5]);

/* Launch configuration of the stream-collide kernel chosen by the autotuner:
 * threads per CTA, the minimum resident CTAs per SM the kernel was compiled
 * for (1 = no register cap), and CTAs per launch (0 = one CTA per block).
 * lbm_create times the shapes (128,1) (256,1) (128,8) (256,4) (128,7), each
 * with one CTA per block and as a persistent grid, on the largest update
 * launch of the schedule.  Environment: LBM_AUTOTUNE=0 skips the timing and
 * keeps (256,1, one CTA per block); LBM_LAUNCH_SHAPE="threads,min,persistent"
 * fixes one listed shape (lbm_create fails with LBM_ERR_ARG otherwise). */
int lbm_get_tuning(const lbm_ctx* ctx, int* threads, int* min_ctas_per_sm, int* ctas);

/* Mass/momentum audit for callers that cannot let the library allocate
 * device memory: code running under CUDA stream capture (allocation is not
 * capturable), frameworks whose own caching pool owns all device memory, and
 * time-critical loops that must not stall on an allocation.  The paper has no
 * counterpart; it is a service entry point of this library.
 *   f        device array of nblocks blocks in the library's storage layout,
 *            [block][Q][512 cells] (cell x + 8y + 64z), shifted and typed as
 *            described for lbm_storage; every cell is summed with volume 1.
 *   out      device array of 4 doubles the caller owns; receives
 *            {sum (rho - 1), sum j_x, sum j_y, sum j_z} in float64.
 *   cuda_stream  cudaStream_t the work is enqueued on (NULL = legacy stream);
 *            the call does not synchronise.
 * No cudaMalloc/cudaFree: partial sums go to a static device array of
 * LBM_NOALLOC_MAX_BLOCKS * 4 doubles (2 MiB) that every GPU loading the
 * library keeps until exit.  Returns LBM_ERR_ARG for a bad model/storage, a
 * NULL pointer, or nblocks outside 1..LBM_NOALLOC_MAX_BLOCKS (the static
 * array holds one partial sum per block); LBM_ERR_CUDA on a launch error.
 * All calls share the array: calls that overlap on the same GPU race.  A
 * call whose stream is not capturing looks up the array's device address
 * and remembers it per device; a call under stream capture uses the
 * remembered address (LBM_ERR_CUDA if there is none), so make the first call
 * on a device, and the first after a cudaDeviceReset, outside capture. */
#define LBM_NOALLOC_MAX_BLOCKS 65536
int lbm_mass_momentum_noalloc(int model, int storage, const void* f, int64_t nblocks, double* out,
                              void* cuda_stream);

/* Block sharding (Sections 1 and 3.2: the paper partitions its blocks over
 * processes, with a halo exchange of the populations that leave each
 * partition).  The level-0 block columns along x are cut into nparts parts
 * of balanced work (cells times substeps of every level above a column);
 * each part is an ordinary context over its slab whose level-0 box keeps one
 * halo block column beyond each cut.  Before each coarse step every cut
 * exchanges, in both directions, the populations of the boundary cell layer
 * that cross it (e_x = +1 one way, e_x = -1 the other: 9 of 27 or 5 of 19
 * values per face cell): packed on the sender, copied device to device,
 * unpacked into the receiver's halo.  Cuts lie only where no refined
 * level-0 block is within one block of either side, so finer levels stay in
 * one part and only level 0 has halos; a periodic x axis adds the cut
 * between the last part and the first.  The inflow, the x walls, the outlet
 * and the nozzle belong to the end parts (the nozzle, with a margin of 16
 * coarse cells, must lie in part 0).  This build places every part on the
 * calling thread's device.  The results equal the unsharded context's bit
 * for bit when every context runs the same stream-collide variant
 * (LBM_LAUNCH_SHAPE).  Dense arrays of lbm_shard_* calls are those of the
 * whole grid, as for a context.  All return LBM_ERR_ARG for bad arguments,
 * a grid the unsharded lbm_create rejects, or no admissible cuts. */
typedef struct lbm_shard lbm_shard;
/* The cuts (host only): cuts[0] = 0 < ... < cuts[nparts] = nbx, part p owning
 * level-0 block columns [cuts[p], cuts[p + 1]). */
int lbm_shard_plan(const lbm_grid* g, int nparts, int* cuts);
int lbm_shard_create(lbm_shard** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
                     double cs, int nparts, void* cuda_stream);
/* Context of one part (owned by the shard) and its level-0 block columns. */
int lbm_shard_part(lbm_shard* s, int part, lbm_ctx** ctx, int* col0, int* col1);
/* Bytes every coarse step moves across all cuts (both directions). */
int lbm_shard_halo_bytes(const lbm_shard* s, int64_t* bytes_per_coarse_step);
int lbm_shard_set_inflow(lbm_shard* s, double y0, double z0, double diameter, double u_in, double perturb,
                         uint64_t seed);
int lbm_shard_init_equilibrium(lbm_shard* s, int level, const double* rho, const double* u);
/* Each coarse step: the halo exchange of every cut, then each part's step.
 * With more than one part every part steps on a stream of its own (created
 * by the shard, so the parts' launches overlap as on separate devices); the
 * exchange runs on cuda_stream after all work queued on the part streams,
 * each part's step after the exchange, and cuda_stream waits for every part
 * before the call returns, so work queued on cuda_stream afterwards (events,
 * copies) sees the stepped state.  lbm_shard_sync waits for cuda_stream and
 * every part stream. */
int lbm_shard_step(lbm_shard* s, int coarse_steps);
int lbm_shard_sync(lbm_shard* s);
int lbm_shard_get_state(lbm_shard* s, int level, double* f, size_t count);
int lbm_shard_macroscopic(lbm_shard* s, int level, double* rho, double* u);
/* Sum of the parts' float64 audits. */
int lbm_shard_mass_momentum(lbm_shard* s, double out[4]);
const char* lbm_shard_last_error(const lbm_shard* s);
void lbm_shard_destroy(lbm_shard* s);  /* NULL-safe */

/* Message describing the last failure on ctx ("" if none). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Free everything; NULL-safe. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
