/*
 * lbm.h - C ABI of a GB300 (sm_103a) implementation of the time step of the
 * thermodynamically consistent multi-component pseudo-potential lattice Boltzmann model
 * of Peng, Ayala & Ayala, arXiv:1909.12390.
 *
 * One step, for every site x and every component s (Section 3.4):
 *   rho_s = sum_a f_{s,a}                                             (cell-volume densities)
 *   p_EOS = mixture Peng-Robinson pressure at the molar density n = sum rho_i / M_i and
 *           molar composition c_i = (rho_i / M_i) / n       (Eq. MCPengRobinson, Eq. randommixingrule)
 *   psi   = sqrt(2 (p_EOS - cs2 rho) / (G cs2)),  rho = sum_s rho_s            (Eq. psicorrected)
 *   F     = -beta G psi(x) sum_a w_a psi(x+e_a) e_a
 *           - (1-beta)/2 G sum_a w_a psi^2(x+e_a) e_a                          (Eq. coupledMCforce)
 *   F_s   = chi_s F,  chi_s = gamma_s rho_s / sum_j gamma_j rho_j              (Eq. distributionforce)
 *   u     = (sum_s sum_a e_a f_{s,a} + F/2) / rho                 (barycentric, Guo half force)
 *   f_s  <- BGK collision with Guo forcing (Eq. LBE, Eq. equilibrium a, b), or MRT, then
 *           periodic streaming f(x + e_a, t+1) = f*(x, t).
 * Lattice units throughout: dt = dx = 1, cs2 = 1/3, gas constant R (default 1).
 *
 * Conventions for every call:
 *   - Host pointers are owned by the caller; the library copies in and out. Device memory is
 *     owned by the library and freed by lbm_destroy.
 *   - Work runs on the context's stream (its own non-blocking stream unless lbm_set_stream
 *     gave one). Every call that returns data or a status synchronises that stream.
 *   - No exception crosses the ABI. Every call returns an lbm_status; lbm_last_error gives a
 *     one-line description of the last failure of that context.
 *   - Field layout: component-major, then z, y, x with x fastest: rho[s][z][y][x].
 *   - Population layout (lbm_get_f / lbm_set_f): f[s][a][z][y][x], FP64, with the direction
 *     order below (the same order as the oracle's and the tests'):
 *       D2Q9 : (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *       D3Q19: (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1) (1,1,0) (-1,-1,0)
 *              (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1)
 *              (0,1,-1) (0,-1,1)
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,        /* invalid argument; nothing was changed */
  LBM_ERR_CUDA = -2,       /* a CUDA runtime call failed; see lbm_last_error */
  LBM_ERR_OOM = -3,        /* device allocation failed */
  LBM_ERR_PSI_DOMAIN = -4, /* psi^2 < 0 or b_m n >= 1 at some site (EOS out of its domain) */
  LBM_ERR_NONFINITE = -5,  /* a density or psi^2 is NaN or infinite */
  LBM_ERR_TIMEOUT = -6     /* a bounded device-side wait ran out (fused kernel) */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };
enum { LBM_BGK = 0, LBM_MRT = 1 };
enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1 };

typedef struct {
  int nx, ny, nz; /* sites per axis, periodic; nz = 1 for D2Q9; Q * nx * ny * nz < 2^32 */
  int lattice;    /* LBM_D2Q9 or LBM_D3Q19 */
} lbm_grid;

/* One component in lattice units (critical temperature and pressure, Pitzer acentric
 * factor, molar mass); see lbm_scale_to_lattice for the paper's scaling. */
typedef struct {
  double Tc, pc, omega, M;
} lbm_component;

typedef struct {
  double T;                /* temperature, lattice units */
  double R;                /* gas constant; 0 means 1 */
  const double *kij;       /* nc*nc binary interaction coefficients zeta_ij (Eq.
                              randommixingrule), row-major, symmetric; NULL means all 0 */
  const double *gamma;     /* nc volatility coefficients of Eq. distributionforce, > 0;
                              NULL means all 1 */
  double beta;             /* Kupershtokh beta of Eq. coupledMCforce */
  double G;                /* interaction strength; only its sign matters (psi^2 >= 0) */
  int collision;           /* LBM_BGK or LBM_MRT */
  const double *mrt_rates; /* Q relaxation rates, one per moment row (D2Q9: Lallemand-Luo
                              rho e eps jx qx jy qy pxx pxy; D3Q19: d'Humieres rho e eps jx qx
                              jy qy jz qz 3pxx 3pixx pww piww pxy pyz pxz mx my mz). The rows
                              of rho, j and the shear stresses always relax at 1/tau; their
                              entries are ignored. NULL with LBM_MRT is an error. */
  int precision;           /* LBM_FP64, or LBM_FP32_SHIFTED: populations stored in FP32 as
                              f_a - w_a rho_ref_s, moments in FP32, every EOS sum in FP64 */
  const double *rho_ref;   /* nc shift references for LBM_FP32_SHIFTED; NULL means the
                              minimum of each component's density given to lbm_init (the
                              vapour value of a two-phase field: vapour populations are then
                              stored as small deviations, liquid ones at FP32's relative
                              precision) */
  int split;               /* force split factor: LBM_SPLIT_VOLATILITY (0), the paper's
                              chi_i = gamma_i rho_i / sum_j gamma_j rho_j (Eq. distributionforce);
                              or LBM_SPLIT_GONG (1), the comparison model of Eq. Gong with the
                              two pressures under the root in the order that makes their
                              difference non-negative (the paper swaps them to keep the root
                              real, Section 4.2): chi_i = c_i sqrt(|p0 - ph_i|) / sum_j
                              c_j sqrt(|p0 - ph_j|), c_i the molar composition, ph_i the PR
                              pressure of pure i at the mixture's molar density n, p0 = n R T;
                              evaluated in FP64. gamma is ignored with LBM_SPLIT_GONG. */
} lbm_eos;
enum { LBM_SPLIT_VOLATILITY = 0, LBM_SPLIT_GONG = 1 };

/* Creates a context for one periodic lattice with nc components (1..4), relaxation time
 * tau > 1/2 (Eq. LBE). Validates every argument (LBM_ERR_ARG) and allocates the device
 * populations (LBM_ERR_OOM). The populations are undefined until lbm_init or lbm_set_f. */
lbm_status lbm_create(const lbm_grid *grid, int nc, const lbm_component *comps,
                      const lbm_eos *eos, double tau, lbm_ctx **out);

/* Releases every device and host resource of ctx. NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

/* Uses the given cudaStream_t (passed as void*) for all later work; NULL restores the
 * context's own stream. */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *stream);

/* Sets the populations to the equilibrium of Eq. equilibrium(a), f_{s,a} = f_eq(rho_s, u),
 * from host arrays rho[nc][N] and u[3][N] (NULL: u = 0), and the step counter to 0.
 * With LBM_FP32_SHIFTED and rho_ref == NULL the shift references become the component minima
 * of rho. Densities must be finite and positive. Page-locked arrays (cudaHostAlloc,
 * cudaHostRegister) are read in place by the kernels, others through a device copy; the call
 * returns after the last read either way. */
lbm_status lbm_init(lbm_ctx *ctx, const double *rho, const double *u);

/* Advances n >= 0 steps of Section 3.4's implementation list: per step the cell-volume
 * densities (moments of Eq. LBE), the mixture Peng-Robinson pressure (Eq. MCPengRobinson with
 * Eq. randommixingrule), the pseudo-potential (Eq. psicorrected), the total force (Eq.
 * coupledMCforce), its split (Eq. distributionforce, or Eq. Gong) and the forced collision and
 * streaming of every component (Eq. LBE, Eq. equilibrium a, b). On a failing step the kernels
 * of the remaining steps do nothing, the populations hold the state before the failing step
 * and the status of the failure is returned; lbm_time then gives the index of that step (on
 * LBM_PATH_FUSED after a timeout the state is undefined). */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Number of steps taken since the last lbm_init / lbm_set_f. */
int64_t lbm_time(const lbm_ctx *ctx);

/* Macroscopic fields of the current state into host arrays (any may be NULL):
 * rho[nc][N] cell-volume densities, u[3][N] barycentric velocity with the Guo half force,
 * p[N] the EOS pressure (equal to the hydrodynamic pressure of Eq. hydropressure), psi[N].
 * Page-locked arrays are written in place by the kernel, others through a device copy; the
 * call returns after the last write either way. */
lbm_status lbm_fields(lbm_ctx *ctx, double *rho, double *u, double *p, double *psi);

/* Total mass of each component, sum over sites of rho_s, into host mass[nc]: the quantity
 * Eq. LBE conserves for every component (the collision and the Guo force term of Eq.
 * equilibrium b have no zeroth moment, streaming permutes the populations). FP32-shifted storage: each thread sums its populations with a compensated FP32
 * sum (TwoSum, about 2^-48 relative) and the reference shift N rho_ref_s is added once; FP64
 * storage sums in FP64. The grid and every reduction are fixed, so the result is
 * bit-reproducible on a given device. Synchronous: returns after the copy to host. */
lbm_status lbm_mass(lbm_ctx *ctx, double *mass);

/* Current populations f_{s,a}(x) of Eq. LBE (the distribution functions of every component
 * and direction) in the canonical FP64 layout f[nc][Q][N] (shift added back). */
lbm_status lbm_get_f(lbm_ctx *ctx, double *f);

/* Replaces the populations f_{s,a}(x) of Eq. LBE with host f[nc][Q][N] (canonical FP64 layout;
 * rounded to FP32 after subtracting the shift when the context stores FP32) and sets the step
 * counter to 0. */
lbm_status lbm_set_f(lbm_ctx *ctx, const double *f);

/* Size in bytes of the raw population storage (lbm_save / lbm_restore). */
size_t lbm_state_bytes(const lbm_ctx *ctx);

/* Checkpoint and resume: copies the raw device storage and the step counter to / from host
 * memory of lbm_state_bytes(ctx) bytes. A restore followed by the same steps reproduces the
 * original run bit for bit. */
lbm_status lbm_save(lbm_ctx *ctx, void *buf, size_t bytes, int64_t *t);
lbm_status lbm_restore(lbm_ctx *ctx, const void *buf, size_t bytes, int64_t t);

/* Step path. LBM_PATH_FUSED runs one persistent cooperative kernel per step that computes
 * psi once per site, publishes it plane by plane (release flags) and collides a plane once
 * the blocks owning its neighbour sites have published the planes around it; waits are
 * bounded (LBM_ERR_TIMEOUT if one runs out, after which the state is undefined). Two forms:
 *   LBM_FUSED_PLANES (D3Q19, nz >= 3): two blocks per SM, block b owning a contiguous range
 *     of every z plane (sites [b nxy / G, (b + 1) nxy / G) of the x-fastest plane index),
 *     marching z; the populations of a plane are read once from DRAM for psi and the site
 *     moments, and re-read from L2 for the collision;
 *   LBM_FUSED_TILES (D2Q9, and D3Q19 grids the first form does not take): each block marches
 *     a tile column (32 x 8 sites for D3Q19 along z, 128 sites for D2Q9 along y); needs nx
 *     divisible by the tile width (and ny by 8 for D3Q19) and the marched axis divisible
 *     into chunks of at least two groups of planes.
 * Both need all blocks co-resident. LBM_PATH_TWO_KERNEL runs a pseudo-potential pass and a
 * collide-stream pass. LBM_PATH_AUTO (the default at lbm_create) takes the two-kernel path, the
 * faster one on GB300 for both lattices. Setting LBM_PATH_FUSED on a grid it does not fit returns LBM_ERR_ARG and leaves the
 * two-kernel path. All paths compute the same arithmetic in the same order per site, so their
 * results are bit-identical. */
/* LBM_PATH_TRAILING (D3Q19, nz >= 3): one persistent cooperative kernel per step, one CTA per
 * SM, CTA b owning a contiguous range of every z plane and marching z. psi of the step was
 * computed by the previous step (a pseudo-potential pass precedes the first step of an
 * lbm_step call when the state changed in between), so the collisions wait for nothing; a
 * stage a few planes behind the collision computes psi of the NEXT step from the populations
 * just written (re-read from L2), once the CTAs owning neighbour sites have published
 * (release flags, bounded acquire waits) that they collided the planes around it. The
 * populations are read from DRAM once per step and written once; psi of the next step is
 * written to a second psi field. A failing psi (EOS domain, non-finite) ends the step that
 * computed it normally and is reported for the next step, whose index lbm_time then gives,
 * with the populations of the state before it, as on the other paths. */
/* LBM_PATH_QUEUE (D3Q19, nz >= 3): one launch per step whose CTAs take the step's tasks from a
 * ticket counter in a fixed order: the collision of each chunk of 512 consecutive sites of a z
 * plane (psi of the step computed by the previous step, as on the trailing path), and psi of
 * the NEXT step for each chunk, placed a plane or two after the collisions it needs and
 * waiting for them (per-chunk release flags, bounded acquire waits). The populations are read
 * from DRAM once per step and written once; psi of the next step re-reads them from L2. The
 * order puts every task a psi task waits for at a smaller ticket, so the queue cannot deadlock
 * and needs no co-resident launch. Failures are reported as on the trailing path. The same
 * Section 3.4 step as every other path, bit for bit. */
enum { LBM_PATH_AUTO = 0, LBM_PATH_TWO_KERNEL = 1, LBM_PATH_FUSED = 2, LBM_PATH_TRAILING = 3, LBM_PATH_QUEUE = 4 };
/* The schedule LBM_PATH_QUEUE runs on an nx x ny x nz grid (host arithmetic only, no device;
 * exported so that it can be checked without a GPU). The dependency it encodes is that of
 * Section 3.4's step: psi at a site needs the densities of the state after the collisions of
 * its neighbours. Each z plane is cut into nch chunks of `chunk` consecutive sites of the
 * x-fastest plane index (chunk <= 0: the library's 512). Outputs, each skipped when NULL:
 *   nbr[nch * LBM_QUEUE_MAX_NBR]: per chunk, the other chunks that hold in-plane neighbours
 *     (periodic, the 8 of the D3Q19 stencil's plane projection) of its sites, -1 padded;
 *   tasks[2 * nz * nch]: the ticket order. The collision of chunk c of plane z is z*nch + c;
 *     psi of the next step over that chunk is -(z*nch + c) - 1. Every collision appears in
 *     plane order, and each psi task follows the collision of chunk c of plane z + 1 + lag
 *     (lag <= 0: the library's 6). The psi tasks the march does not place come last, plane 0
 *     at the very end. Every collision a psi task needs (planes z - 1 .. z + 1 of the chunk
 *     and its neighbour chunks) has a smaller ticket.
 * Returns nch, or -1 when the grid is not served (nx or ny < 1, nz < 3, a chunk with more
 * than LBM_QUEUE_MAX_NBR neighbour chunks). Call it with NULL outputs first to size them. */
#define LBM_QUEUE_MAX_NBR 16
int lbm_queue_schedule(int nx, int ny, int nz, int chunk, int lag, int *nbr, int *tasks);
lbm_status lbm_set_path(lbm_ctx *ctx, int path);
/* The path lbm_step takes now (LBM_PATH_TWO_KERNEL, LBM_PATH_FUSED, LBM_PATH_TRAILING or
 * LBM_PATH_QUEUE). */
int lbm_get_path(const lbm_ctx *ctx);
/* The form of the fused path: LBM_FUSED_TILES or LBM_FUSED_PLANES; 0 on the other paths or
 * for a NULL ctx. */
enum { LBM_FUSED_TILES = 1, LBM_FUSED_PLANES = 3 };
int lbm_get_fused_kind(const lbm_ctx *ctx);

/* Failure-detection test hook, fused and trailing paths only: from the next step on, fused
 * block `block` (0-based; LBM_FUSED_TILES: x-tile fastest, then y-tile, then chunk;
 * LBM_FUSED_PLANES and LBM_PATH_TRAILING: the plane range index; LBM_PATH_QUEUE: the chunk index
 * of a plane, whose collisions then publish nothing in any plane) computes but never publishes its
 * progress, so every neighbour's bounded wait runs out and lbm_step returns
 * LBM_ERR_TIMEOUT (within about a second per step, without faulting or hanging the GPU); the
 * populations are then undefined. -1 switches the hook off; lbm_init restores a state. */
lbm_status lbm_test_silence_block(lbm_ctx *ctx, int block);

/* Kernel timing. lbm_profile(ctx, 1) clears the record and from then on brackets every
 * kernel launch of lbm_step with CUDA events on the context's stream (graph replay is off
 * while profiling); lbm_profile(ctx, 0) stops recording. lbm_profile_read sums the recorded
 * durations of one kernel kind (0 = pseudo-potential pass, 1 = force + collide + stream
 * pass, 2 = fused step) in milliseconds and gives the number of launches. Both synchronise
 * the stream. */
lbm_status lbm_profile(lbm_ctx *ctx, int on);
lbm_status lbm_profile_read(lbm_ctx *ctx, int kernel, double *total_ms, int64_t *launches);

/* ---- Adjoint (gradients; BGK or MRT collision) ---------------------------------------
 * lbm_record advances n steps from the current state like lbm_step and keeps a copy of the
 * raw state every checkpoint_every steps (the first at the current step). lbm_adjoint then
 * back-propagates dL/drho of the final state (host array drho[nc][N], the loss gradient with
 * respect to the cell-volume densities the recorded run ended with) through every recorded step
 * with the hand-written discrete adjoint of the step (BGK or MRT collision with Guo forcing,
 * split of Eq. distributionforce, force of Eq. coupledMCforce, EOS of Eq. MCPengRobinson),
 * recomputing each segment's states from its checkpoint. Outputs (any may be NULL):
 * dkij[nc*nc] = dL/dzeta_ij per matrix entry (for a symmetric coefficient add the (i,j) and
 * (j,i) entries), dgamma[nc] = dL/dgamma_i, drho0[nc][N] = dL/drho at the recorded start for
 * an equilibrium start at rest (lbm_init with u = NULL). Arithmetic in the storage precision
 * (FP32 for LBM_FP32_SHIFTED) with the EOS derivative and the reductions in FP64. Device
 * memory, allocated for the call: checkpoint_every states and pseudo-potential fields plus
 * the adjoint fields. With full storage (lbm_set_adjoint_memory 0) and more than one segment
 * it also tries a second set of checkpoint_every states and fields, so that the replay of the
 * next segment runs on a stream of its own beside the current segment's reverse sweep; where
 * that set cannot be allocated the two run one after the other (same results bit for bit). */
lbm_status lbm_record(lbm_ctx *ctx, int64_t n, int checkpoint_every);
/* Device memory of lbm_adjoint's reverse sweep. snapshots = 0 (the default) or >=
 * checkpoint_every: each recorded segment's states are recomputed once and all kept
 * (checkpoint_every state slots). 0 < snapshots < checkpoint_every: revolve-style binomial
 * checkpointing inside each segment (Griewank's schedule): with s free slots the reversal of n
 * steps advances m of them into a slot, reverses the last n - m with s - 1 slots, then the first
 * m with s, m chosen so that no step is advanced more than r times, r the least integer with
 * C(s + 1 + r, s + 1) >= n (s + 1 snapshots, the segment's start included), and the total of
 * advanced steps the least such a schedule allows. snapshots + 2 state slots are allocated
 * (two of them scratch for the out-of-place steps); the gradients equal those of the
 * full schedule bit for bit (the recomputed states are identical), at the cost of up to r
 * recomputations per step. */
lbm_status lbm_set_adjoint_memory(lbm_ctx *ctx, int snapshots);
/* Test hook: on = 0 makes lbm_adjoint run each segment's replay and reverse sweep one after
 * the other on the context's stream, as it does when the second set of state slots cannot be
 * allocated; on = 1 (the default) lets the replay run beside the sweep. The gradients are the
 * same bit for bit either way. */
lbm_status lbm_test_adjoint_overlap(lbm_ctx *ctx, int on);
/* Forward steps the reverse sweep recomputes for one segment of n steps with the given state
 * slots (0 or >= n: n - 1, every state once); host arithmetic only, no device. -1 for n < 1 or
 * snapshots < 0. */
int64_t lbm_revolve_steps(int64_t n, int snapshots);
lbm_status lbm_adjoint(lbm_ctx *ctx, const double *drho, double *dkij, double *dgamma, double *drho0);

/* ---- Batched lattices -------------------------------------------------------------------
 * Many small independent D2Q9 cases (each its own grid, components' constants, temperature,
 * kij, gamma, tau) advanced together, as in a sweep of flash conditions. All cases share nc,
 * precision and collision. Each case is owned by one thread block that keeps the case's
 * populations and pseudo-potential in shared memory for a whole chunk of steps (cases too
 * large for shared memory run from global memory); cases are grouped by size, one launch per
 * size class on its own stream, and the step loop replays a captured CUDA graph. Cases are
 * independent: a case that fails (EOS domain, non-finite) stops at its failing step while the
 * others continue. Arrays are indexed by case and concatenated in case order: grids[ncase],
 * comps[ncase * nc], eos[ncase], tau[ncase]; fields rho[sum_c nc N_c] with case c at offset
 * nc * (sites of cases before c), u likewise with 3 per site, p with 1 per site. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(int ncase, const lbm_grid *grids, int nc, const lbm_component *comps,
                            const lbm_eos *eos, const double *tau, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);
/* Equilibrium start of every case from concatenated densities (and velocities or NULL). */
lbm_status lbm_batch_init(lbm_batch *b, const double *rho, const double *u);
/* Advances every case n steps; returns the first failing case's status (others still ran). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t n);
/* Per-case status and step count (either array may be NULL). */
lbm_status lbm_batch_case_status(lbm_batch *b, int *status, int64_t *t);
lbm_status lbm_batch_fields(lbm_batch *b, double *rho, double *u, double *p);
/* Canonical FP64 populations f[nc][9][N_c] of case i. */
lbm_status lbm_batch_get_f(lbm_batch *b, int i, double *f);
/* Autotuner: times trial_steps steps of every feasible block size per size class on the
 * current state (restored afterwards) and keeps the fastest; lbm_batch_tune_report lists the
 * choices. */
lbm_status lbm_batch_tune(lbm_batch *b, int trial_steps);
const char *lbm_batch_tune_report(const lbm_batch *b);
int64_t lbm_batch_sites(const lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

/* Allocation-free step (the paper has no counterpart; this is a library service).
 *
 * Some callers cannot let a library allocate device memory: applications whose device
 * memory is owned by their own pool allocator (a framework or runtime that reserves the GPU's
 * memory up front, where an outside cudaMalloc fails or fragments the pool), and code that
 * must not allocate at a given point because cudaMalloc and cudaFree can synchronise the
 * device and stall other streams. lbm_step_static serves them: it advances n steps of one
 * lattice (two-kernel path) on populations the caller keeps in its own device memory and
 * calls no cudaMalloc, cudaFree or any other allocating routine.
 *
 * f_device holds the populations in the library's storage layout: f[nc][Q][N] structure of
 * arrays, FP64, or FP32 holding f - w_a rho_ref_s when eos->precision is LBM_FP32_SHIFTED
 * (eos->rho_ref gives the shift; NULL means 0), in the in-place streaming layout of step t0
 * (even t0: slot (x, a) holds f_a(x); lbm_save writes this layout). The other arguments are
 * those of lbm_create. On return *t_out (if not NULL) is the step index reached, t0 plus the
 * number of steps completed: t0 + n on success, the index of the failing step otherwise (the
 * populations then hold the state before that step).
 *
 * Scratch: the pseudo-potential, the status word and the step counter live in one fixed
 * device array inside the library, 256 B + LBM_STATIC_MAX_SITES * 8 B (8 MiB + 256 B), which
 * a GPU holds from the moment the library's code is loaded on it until the process exits.
 * Grids with more than LBM_STATIC_MAX_SITES sites are rejected with LBM_ERR_ARG.
 * First use on a device: CUDA loads a library's device code lazily by default
 * (CUDA_MODULE_LOADING=LAZY), so the first call on a device loads the code that holds the
 * array, commits its 8 MiB and looks up its device address (cudaGetSymbolAddress, with that
 * device current), and the first step of each lattice / precision / collision variant loads
 * that variant's kernels. Loading reserves device memory and may synchronise the device. A
 * caller that must not allocate later should therefore make one warm-up call that runs at
 * least one step (n >= 1) of every variant it will use, at a point where allocation is
 * allowed and before any stream capture; setting CUDA_MODULE_LOADING=EAGER before the
 * process starts moves all of this to the loading of the library instead. After that, calls
 * allocate nothing. Every call shares the array and leaves its contents behind; each call
 * resets the status word and counter it uses. Calls whose work overlaps on
 * the GPU (other streams or threads on the same device) race on the array: serialise them.
 * The call synchronises `stream` (a cudaStream_t, NULL = default stream) before returning
 * the first failing step's status. lbm_step_static_error gives this thread's last message. */
#define LBM_STATIC_MAX_SITES 1048576
lbm_status lbm_step_static(const lbm_grid *grid, int nc, const lbm_component *comps, const lbm_eos *eos,
                           double tau, void *f_device, int64_t t0, int64_t n, void *stream, int64_t *t_out);
const char *lbm_step_static_error(void);

/* Batched two-phase flash (Section 3.2): the phase equilibrium of the Peng-Robinson mixture
 * that sets up the multi-component runs of Section 4.2 (initial phase densities and the
 * volatility coefficients gamma of Eq. gamma), for many (T, p, z) cases of one set of nc
 * components, one GPU thread per case in FP64.
 *
 * comps: nc (1..4) components, Tc, pc, omega and M in any units consistent with the cases'
 *   T and p (only T / Tc, p / pc and the ratios of M enter, except through R below);
 * cases: ncase host structs: T, p, feed mole fractions z[0..nc) (each > 0, summing to 1),
 *   kij[nc * nc] row-major symmetric binary interaction coefficients (zeta_ij);
 * R: the gas constant in the units of p / (n T) (1 in lattice units);
 * tol, maxit: successive substitution stops when max_i |d ln K_i| < tol (1e-13 reaches FP64
 *   precision) or after maxit iterations;
 * stream: a cudaStream_t (NULL = default stream); the call copies in, runs, copies out and
 *   synchronises it; device memory is allocated and freed on the stream.
 * out: ncase host structs. status 0: two phases, converged; 1: single phase or trivial
 *   solution (K_i within 1e-4 of 1), only x = y = z, V, K and Z are meaningful; 2: two phases
 *   not converged within maxit. V is the vapour mole fraction of the Rachford-Rice equation
 *   (negative flash: it may leave [0, 1]); x, y the liquid and vapour mole fractions; Zl, Zv
 *   the Gibbs-selected roots (Eq. solutionselection) of the PR cubic; residual Eq. error;
 *   rho_l, rho_v the phase partial densities n x_i M_i with n = p / (Z R T); gamma the
 *   per-component Eq. gamma, 1 for the least volatile component (smallest K).
 * Returns LBM_ERR_ARG for invalid arguments (nothing runs) and LBM_ERR_CUDA for a CUDA
 * failure; lbm_flash_error gives this thread's last message. */
typedef struct {
  double T, p;
  double z[4];
  double kij[16];
} lbm_flash_case;
typedef struct {
  double V;
  double x[4], y[4], K[4];
  double Zl, Zv;
  double residual;
  double rho_l[4], rho_v[4], gamma[4];
  int iterations;
  int status;
} lbm_flash_result;
lbm_status lbm_flash(int nc, const lbm_component *comps, int ncase, const lbm_flash_case *cases, double R,
                     double tol, int maxit, void *stream, lbm_flash_result *out);
const char *lbm_flash_error(void);

/* Diagnostics of the current state (the checks of Sections 4.2 and 4.3), computed on the
 * device from the component densities and the EOS pressure of every site:
 *   * the contour level: params->threshold if > 0, else (rho_max + rho_min) / 2 of the total
 *     density rho = sum_s rho_s;
 *   * the bulk phases: cells whose whole (2 erode + 1)^D box (periodic) lies above the level
 *     (liquid) or below it (vapour), i.e. farther than `erode` cells from the contour in the
 *     L-infinity norm (the paper's bulk cells are those more than 8 cells from the contour);
 *   * their mean component densities rho_l / rho_v, EOS pressures p_l / p_v, molar
 *     compositions x / y and the iso-fugacity residual of Eq. error with f_i = phi_i c_i p,
 *     ln phi_i from Eq. fugacitycoeff2 at Z = p / (n R T) (no cubic solve);
 *   * liquid_cells (cells above the level), the equivalent radius sqrt(cells / pi) in 2-D or
 *     cbrt(3 cells / (4 pi)) in 3-D, and dp = p_l - p_v (Laplace's law: dp = sigma / R in 2-D).
 * Sums use FP64 atomics (their order is not fixed: results agree to rounding between calls).
 * Allocates and frees a device work buffer of ~12 bytes per site on the context's stream;
 * synchronises it. NaN where a phase has no bulk cell. */
typedef struct {
  double threshold;  /* contour level of the total density; <= 0: (rho_max + rho_min) / 2 */
  int erode;         /* bulk cells are farther than this from the contour (>= 0) */
} lbm_diag_params;
typedef struct {
  double threshold, rho_max, rho_min;
  double rho_l[4], rho_v[4], p_l, p_v, x[4], y[4];
  double residual, radius, dp;
  int64_t n_l, n_v, liquid_cells;
} lbm_diag_result;
lbm_status lbm_diagnostics(lbm_ctx *ctx, const lbm_diag_params *params, lbm_diag_result *out);

/* One-line description of the last failure of ctx ("" if none). Valid until the next call
 * on ctx. With ctx == NULL, the last failure of lbm_create. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Section 4.2 scaling of physical constants to lattice units: a_1 = 2/49, b_1 = 2/21,
 * M_1 = 1, R = 1 fix T_c1 = (0.0778 / 0.45724)(a_1 / b_1) and p_c1 = 0.0778 T_c1 / b_1;
 * component i keeps T_ci / T_c1, p_ci / p_c1 and M_i / M_1, so every reduced quantity is
 * unchanged. Writes nc lattice components to out and the lattice-unit temperature and
 * pressure of (T_phys, p_phys) to T_lb and p_lb (either may be NULL). */
lbm_status lbm_scale_to_lattice(int nc, const lbm_component *phys, double T_phys, double p_phys,
                                lbm_component *out, double *T_lb, double *p_lb);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
