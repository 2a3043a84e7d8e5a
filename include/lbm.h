/*
 * liblbm: GB300 (sm_103a) two-population phase-field lattice Boltzmann step.
 *
 * Model: Otomo, Zhang & Chen, "Improved phase-field-based lattice Boltzmann
 * models with a filtered collision operator" (arXiv 1812.00118).
 *   - h_i: Allen-Cahn interface LB with the theta counter-term (Section 2,
 *     Eqs. 1-4), phi = sum_i h_i.
 *   - g_i: pressure/momentum LB with forcing K_i (Eqs. 5-8), relaxation time
 *     interpolated by Eq. 9, filtered collision (Eqs. 10-12), high-order
 *     equilibrium correction delta f^eq (Section 3, Eq. 13).
 *   - grad phi and lap phi by nearest-neighbour central differences (the
 *     unnumbered stencils after Eq. 12).
 *   - P = T sum g + (T rho_dif / 2) u.grad phi and rho u = sum c g +
 *     (mu grad phi + F)/2 (text after Eq. 12).
 *   - pull streaming on D2Q9 / D3Q19, periodic or halfway bounce-back walls.
 *
 * Conventions shared by every call:
 *   - Lattice units (dx = dt = 1), T = 1/3.
 *   - Fields are x-fastest: idx = x + nx*(y + ny*z); a D2Q9 grid has nz = 1.
 *   - Vectors are component-major: v[d*N + idx], d = 0..dim-1, N = nx*ny*nz.
 *   - Every field passed in or out is double precision, whatever the storage
 *     type of the populations.
 *   - Host pointers (on_device = 0) or device pointers (on_device = 1) are
 *     accepted for fields; the caller owns them and the library never keeps
 *     them past the call.
 *   - The library owns its population buffers (two A/B sets of 2*Q*N values).
 *   - All work is ordered on the CUDA stream given to lbm_create (NULL = the
 *     legacy default stream).  Calls that return data to the host synchronise
 *     that stream; lbm_step does not.
 *   - Return value: LBM_OK (0) or a negative LBM_E* code; lbm_strerror gives
 *     its text.  On an error nothing is launched and the state is unchanged,
 *     except LBM_ECUDA, after which the context should be destroyed.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
enum lbm_bc { LBM_PERIODIC = 0, LBM_WALL = 1 };
/* Population storage.  LBM_F64: FP64 storage and arithmetic.  LBM_F32: FP32
 * storage and arithmetic.  LBM_F16S / LBM_BF16S: 16-bit storage of shifted
 * values (h_i - w_i/2, (g_i - w_i P_ref/T) * g_scale) with FP32 arithmetic. */
enum lbm_store { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 };

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* bad argument, size or parameter */
    LBM_ENOMEM = -2,     /* device allocation failed */
    LBM_ECUDA = -3,      /* a CUDA call failed */
    LBM_EDIVERGED = -4,  /* a diagnostic found a non-finite value or |u| > 0.3 */
    LBM_ETIMEOUT = -5,   /* a bounded device wait gave up */
    LBM_ENOTSUP = -6,    /* combination the library does not support */
    LBM_ECHECKED = -7    /* checked builds: a step kernel met an offset outside its arrays */
};

typedef struct lbm_ctx lbm_ctx;   /* opaque, owned by the library */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* Grid: nx, ny, nz >= 1 (nz == 1 for D2Q9).  bc[a] is the boundary type of
 * both ends of axis a (0 = x, 1 = y, 2 = z).  A walled axis has halfway
 * bounce-back walls half a spacing outside its first and last node; there
 * the phi stencil mirrors the adjacent node (zero normal gradient). */
typedef struct {
    int nx, ny, nz;
    int bc[3];
} lbm_grid;

/* Physical parameters (lattice units).
 *   M       mobility (Eq. 1: tau_phi = M/T + 1/2), > 0
 *   W       interface thickness (Eq. 4, Eq. 8), > 0
 *   sigma   surface tension (Eq. 8), >= 0
 *   rho_L   density of the light phase (phi = 0, "air"), > 0
 *   rho_H   density of the heavy phase (phi = 1, "water"), > 0;
 *           rho(phi) = rho_L + phi (rho_H - rho_L), rho_dif = rho_H - rho_L
 *   nu_L, nu_H  kinematic viscosities; tau = nu/T + 1/2 each, and 1/tau_mix
 *           interpolates 1/tau linearly in phi clipped to [0, 1] (Eq. 9)
 *   g[3]    body acceleration; F_ex = rho g (force_mode 0) or
 *           (rho - rho_bar) g (force_mode 1, rho_bar = mean density of the
 *           initial phi, computed by lbm_init_fields / lbm_set_populations)
 *   eps     regulariser of n = grad phi / (|grad phi| + eps) (Section 2), 1e-10
 *   hocorr  1: add delta f^eq of Eq. 13 and read the velocity from
 *           (rho + lap(rho)/4) u = sum c g + (mu grad phi + F)/2;
 *           0: the uncorrected model of Section 2 (rho u = ...)
 *   store   an lbm_store value
 *   P_ref, g_scale  shift and scale of the 16-bit storage types (ignored
 *           otherwise; g_scale = 0 means 1)
 *   C_dtheta  constant C of the diffusion correction of Eq. 14 (Section 3):
 *           theta of Eq. 4 becomes theta + delta theta with
 *           delta theta = C (M/T) F |grad phi|.  The paper leaves F open and
 *           asks only that it vanish on ordinary drops and bubbles; the
 *           library takes F = -W^2 max(0, (2 phi - 1) lap phi), which is 0 on
 *           the tanh interface profile and negative in a dense bubble (a dip
 *           of phi inside the heavy phase) or a rarefied droplet (a bump
 *           inside the light phase), where C > 0 then adds diffusion.
 *           0 (the default) is the model of Section 2; must be finite.
 */
typedef struct {
    double M, W, sigma, rho_L, rho_H, nu_L, nu_H;
    double g[3];
    int force_mode;
    double eps;
    int hocorr;
    int store;
    double P_ref, g_scale;
    double C_dtheta;
} lbm_params;

/* Create a context: validates the grid and parameters, allocates the A/B
 * population buffers on `cuda_stream` (a cudaStream_t, NULL for the default
 * stream) of the current device.  Populations are zero until
 * lbm_init_fields or lbm_set_populations.  `lattice` is an lbm_lattice.
 * Errors: LBM_EINVAL (sizes < 1, nz != 1 for D2Q9, a periodic axis shorter
 * than 1, tau <= 1/2, M <= 0, W <= 0, rho <= 0, a parameter that is not
 * finite, g_scale < 0, unknown store, a padded grid of 2^31 cells or more),
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(const lbm_grid* grid, int lattice, const lbm_params* params,
               void* cuda_stream, lbm_ctx** out);

/* lbm_create with options.  flags = 0: the same call; the population arrays
 * then carry ghost cells along walled axes only (for the bounce-back writes;
 * a periodic axis wraps its pulls and needs none).  LBM_CREATE_GHOST_BAND:
 * a band of ghost cells along the periodic axes too, which the bulk-copy
 * step tile (tile 4 of lbm_set_tile) needs for the periodic images it reads;
 * the other tiles run on either layout and compute the same values.
 * Errors: as lbm_create, LBM_EINVAL for an unknown flag. */
#define LBM_CREATE_GHOST_BAND 1
int lbm_create_ex(const lbm_grid* grid, int lattice, const lbm_params* params,
                  void* cuda_stream, int flags, lbm_ctx** out);

/* Device memory plan of a grid, computed on the host without a GPU (nothing
 * is allocated): the checks of lbm_create_ex, then out[0..2] = padded
 * extents of the population arrays along the internal axes x, y, z (for
 * D2Q9 the user's y is the internal z and out[1] = 1; x rows padded to 32
 * bytes, ghost cells on walled axes, or on every axis with
 * LBM_CREATE_GHOST_BAND), out[3] = cells per population array (their
 * product, < 2^31), out[4] = bytes of the population buffers (h and g, two
 * time levels each: 4 Q out[3] times the storage type's size), out[5] =
 * bytes a context holds once it has been initialised (out[4], the scratch
 * fields of 5 N doubles and the reduction partials).  Errors: as
 * lbm_create_ex (LBM_EINVAL, out untouched). */
int lbm_layout(const lbm_grid* grid, int lattice, const lbm_params* params, int flags, long long out[6]);

/* Initialise the populations from macroscopic fields (Section 4 set-ups
 * start from (phi, u, P)): h = h^eq (Eq. 2) and g = g^eq (Eq. 6 with Eq. 7
 * and Eq. 13) evaluated with the central-difference stencils of the given
 * phi.  phi, P: N doubles; u: dim*N doubles (dim = 2 for D2Q9, 3 for
 * D3Q19).  lbm_macro right after this call returns the same fields to
 * rounding of the storage type.  Synchronises the stream. */
int lbm_init_fields(lbm_ctx* ctx, const double* phi, const double* u, const double* P,
                    int on_device);

/* lbm_init_fields with options.  flags = 0: the same call.  LBM_INIT_NONEQ:
 * g also carries the filtered non-equilibrium part of a state that has
 * relaxed onto the given flow, Phi_i : Pi(1) with Phi_i of Eq. 11 and the
 * Chapman-Enskog estimate Pi(1) = -tau_mix T rho (grad u + grad u^T) of the
 * non-equilibrium momentum flux (grad u by the central differences of the
 * stencils after Eq. 12, tau_mix from Eq. 9); it leaves the zeroth and first
 * moments, so lbm_macro still returns (phi, u, P).  The paper rebuilds no
 * states; this serves the learned warm start (a state predicted as fields
 * continues without the start-up transient an equilibrium start has).
 * Errors: as lbm_init_fields, LBM_EINVAL for an unknown flag. */
#define LBM_INIT_NONEQ 1
int lbm_init_fields_ex(lbm_ctx* ctx, const double* phi, const double* u, const double* P, int on_device,
                       int flags);

/* Advance n >= 0 time steps: each step is one launch of the fused
 * collide-and-pull-stream kernel (Eqs. 1-14) and a buffer swap; the
 * bulk-copy tile (see lbm_set_tile) adds one launch of a small kernel that
 * writes the periodic images into the ghost band of the buffer just written
 * (and one more before its first step on a state another tile wrote).
 * Asynchronous on the context stream; returns LBM_ECUDA if a launch fails,
 * and LBM_EDIVERGED without launching anything if the last lbm_diagnostics
 * found the state diverged (until lbm_init_fields or lbm_set_populations
 * replace it). */
int lbm_step(lbm_ctx* ctx, int n);

/* lbm_step with CUDA events recorded on the context stream around every
 * launch of the fused step kernel; *kernel_ms receives the summed duration of
 * those launches (the ghost-update launches excluded).  Synchronises.  Used
 * to relate the step kernel's own time to its algorithmic traffic. */
int lbm_step_profiled(lbm_ctx* ctx, int n, double* kernel_ms);

/* Macroscopic fields of the current state (time t, before its collision):
 * phi = sum h, P and rho u by the formulas after Eq. 12, where rho u is
 * rho(phi) times the velocity the collision uses.  Any output pointer may be
 * NULL.  Synchronises the stream. */
int lbm_macro(lbm_ctx* ctx, double* phi, double* P, double* rho_u, int on_device);

/* Pre-collision populations of the current state, converted to double:
 * h and g are Q*N each, population-major (h[i*N + idx]) in the velocity
 * order reported by lbm_lattice_info.  Checkpoint/resume: set(get(x))
 * restores x exactly for every storage type.  Synchronises the stream. */
int lbm_get_populations(lbm_ctx* ctx, double* h, double* g, int on_device);
int lbm_set_populations(lbm_ctx* ctx, const double* h, const double* g, int on_device);

/* FP64 diagnostics of the current state, reduced on the device in a fixed
 * order (deterministic): out[0] = sum phi, out[1] = sum rho, out[2] = max |u|,
 * out[3] = number of non-finite phi/u/P values.  Returns LBM_ETIMEOUT if a
 * bounded wait of a bulk-copy step gave up since creation, else
 * LBM_EDIVERGED (after filling out) if out[3] > 0 or out[2] > 0.3.
 * Synchronises. */
int lbm_diagnostics(lbm_ctx* ctx, double out[4]);

/* Laplace-law measurement (Section 4.1) in FP64 on the device:
 * dP = <P>_{r < r_in} - <P>_{r > r_out}, r the minimum-image distance from
 * centre[3] along periodic axes.  Synchronises. */
int lbm_laplace(lbm_ctx* ctx, const double centre[3], double r_in, double r_out, double* dP);

/* Velocity set of a lattice in the library's own order: Q, c[3*Q] (x, y, z
 * components of each velocity, user axes: D2Q9 velocities lie in x-y) and
 * w[Q].  Either array may be NULL. */
int lbm_lattice_info(int lattice, int* Q, int* c, double* w);

/* Number of kernel launches issued by the context since creation. */
long long lbm_launch_count(const lbm_ctx* ctx);

/* The CUDA stream of the context (as given to lbm_create). */
void* lbm_stream(const lbm_ctx* ctx);

/* Re-impose the total of phi every `every` steps (0, the default: never).
 * 16-bit population storage rounds the stored h every step, and the rounding
 * does not sum to zero: over tens of thousands of steps the total of phi
 * drifts (a third of it in FP16 drop relaxations).  The correction sums phi
 * in FP64 on the GPU, compares it with the total the last lbm_init_fields
 * or lbm_set_populations gave, and adds the difference / N to the rest
 * population h_0 of every node (a uniform shift of phi; the paper's Eq. 1
 * conserves phi exactly, so this only undoes storage rounding).  Four
 * stream-ordered launches per correction, no host synchronisation.  Not for
 * the grids of a batch.  Errors: LBM_EINVAL (every < 0, a batch grid),
 * LBM_ENOMEM. */
int lbm_set_phi_correction(lbm_ctx* ctx, int every);

/* Velocity u (user axes; u[2] ignored for D2Q9) of the wall at end `side`
 * (0: below coordinate 0, 1: above n - 1) of walled user axis `axis`; all
 * walls start at rest.  A sliding wall only: the component normal to the wall
 * must be 0.  Halfway bounce-back less the momentum the wall hands over: a
 * population f*_j leaving a node towards the wall returns as
 * f*_j - 2 w_j s (c_j . u) / T, s = phi for h and rho(phi) for g at that node
 * (the paper's Couette flow of Section 3 assigns wall velocities without
 * writing the rule; this is the library's reading).  Takes effect at the next
 * step.  Errors: LBM_EINVAL (bad axis or side, axis not walled, normal
 * component, non-finite). */
int lbm_set_wall_velocity(lbm_ctx* ctx, int axis, int side, const double u[3]);

/* Step kernel configuration.  `tile` indexes the compiled step kernels of
 * the lattice (CTA shapes in nodes: D3Q19 x-y, D2Q9 rows along x):
 *   0     per-thread loads, the g loads of a plane held in registers across
 *         the phi fill; 32x4 / 128, 4 CTAs per SM.
 *   1-3   per-thread loads in phases (phi fill, g moments, collision):
 *         32x4 / 128 at 8 CTAs per SM, 32x8 / 256 at 4, 32x4 / 64 at 6 / 16.
 *   4     bulk tensor copies into a shared-memory pipeline (persistent CTAs
 *         taking work items of `lz` planes; 32x4 / 128).  Needs a context
 *         created with LBM_CREATE_GHOST_BAND.
 *   5, 6  tiles 0 and 1 launched as one wave: every column split into the
 *         same number of chunks, as many as the resident CTAs allow, each at
 *         least `lz` planes long.
 *   7     loads issued one plane ahead as asynchronous copies into shared
 *         memory (FP32 storage only; 32x4 / 128).
 *   8, 9  tile 1 at 7 CTAs per SM (72 registers), and the same as a one-wave
 *         launch.
 * Tiles other than 4 and the one-wave forms take chunks of `lz` >= 1 planes
 * along the march axis (z in 3-D, y in 2-D).  Every tile computes the same
 * arithmetic.  lbm_create picks tile 1 with lz = 16 for D2Q9, and for D3Q19
 * tile 8 with lz = 16, or tile 3 with lz = 32 for FP32 storage on grids of
 * 2^24 nodes or more; lbm_get_tile reports the current choice and its CTA
 * shape.
 * Errors: LBM_EINVAL for an unknown tile or lz < 1, LBM_ENOTSUP for a
 * bulk-copy or asynchronous-copy tile this grid, layout or storage type
 * cannot use. */
int lbm_set_tile(lbm_ctx* ctx, int tile, int lz);
int lbm_get_tile(const lbm_ctx* ctx, int* tile, int* lz, int* tx, int* ty);

/* Poll limit of the bounded waits of the bulk-copy step pipeline (tile 4;
 * the other step kernels do not wait).  A wait whose copies have not landed
 * after `polls` tries gives up: the kernel raises the context's error flag,
 * lets the copies it has in flight land (a separate bounded wait) and
 * returns, so the GPU context stays usable, lbm_diagnostics returns
 * LBM_ETIMEOUT and the state of that step is invalid until the next
 * lbm_init_fields / lbm_set_populations (which also clear the flag).
 * Default 4194304; 0 makes every pipeline wait give up at once (a host-side
 * way to exercise the failure path without any fault).  Errors: LBM_EINVAL
 * (polls < 0). */
int lbm_set_wait_limit(lbm_ctx* ctx, long long polls);

/* Autotuner: times every compiled tile (those the grid supports) with lz in
 * {4, 8, 16, 32} for `steps` steps each on the current state, keeps the
 * fastest configuration, and restores the state it started from (the state
 * is saved to, and copied back from, a temporary device copy).  Reports the
 * choice and its time per step (step kernel plus ghost update) in ms; any
 * output pointer may be NULL.  Synchronises.  If a trial fails, the state is
 * restored all the same, the context keeps the tile it had and the trial's
 * status is returned.  Errors: LBM_EINVAL (steps < 1), LBM_EDIVERGED (the
 * state was found diverged earlier), LBM_ENOMEM, LBM_ECUDA. */
int lbm_autotune(lbm_ctx* ctx, int steps, int* best_tile, int* best_lz, double* best_ms);

/* Field diagnostics without any allocation.  The paper has no counterpart:
 * this is a service of the library, not a step of the method.
 *
 * For callers that cannot call cudaMalloc -- a host framework whose allocator
 * owns all device memory, a loop that must not enter the allocator -- this
 * computes the same FP64 sums as lbm_diagnostics, in a fixed order, from
 * field arrays the caller provides, and allocates nothing: its scratch
 * (per-block partial sums) is a static device array of 256 KB inside the
 * library, held by every GPU that loads the library until the process exits.
 *
 *   phi, P      device arrays of n doubles (required)
 *   v0, v1, v2  device arrays of n doubles, the components of a vector field
 *               (e.g. u); any may be NULL (treated as 0)
 *   n           number of nodes, 0 <= n <= LBM_NOALLOC_MAX_NODES
 *   rho_L, rho_dif  rho = rho_L + phi rho_dif for the mass sum
 *   out         device array of 4 doubles: sum phi, sum rho, max |v|, and the
 *               number of non-finite phi / P / |v| values
 *   cuda_stream the stream to launch on (NULL: default stream)
 *
 * Asynchronous: out is valid once the stream reaches the call.  The first
 * call on a device (and the first after its context was replaced, e.g. by
 * cudaDeviceReset) looks up the scratch array's device address with that
 * device current; make that first call before any stream capture.  Every
 * call on a device shares the one scratch array, so calls whose launches
 * overlap on the GPU (different streams, no ordering) race: order them on
 * one stream.  Errors: LBM_EINVAL (NULL phi, P or out, n < 0 or
 * n > LBM_NOALLOC_MAX_NODES), LBM_ECUDA (an error was pending before the
 * call -- it is left for its owner to read -- or a launch failed). */

#define LBM_NOALLOC_MAX_NODES 33554432
int lbm_field_sums_noalloc(const double* phi, const double* P, const double* v0, const double* v1,
                           const double* v2, long long n, double rho_L, double rho_dif, double* out,
                           void* cuda_stream);

/* Checked builds (compiled with LBM_CHECKED, a debugging option; the default
 * build is not one).  The step kernels then check every plane's pull offsets
 * and every write offset against the population arrays; an offset outside
 * them is replaced by a valid one and recorded.  lbm_checked_status
 * synchronises `stream` (NULL: the default stream) and reports the record
 * since its last call: LBM_ECHECKED if any offset failed, else LBM_OK
 * (always LBM_OK in a default build); LBM_ECUDA if the synchronisation or
 * the read failed.  lbm_is_checked_build returns 1 in a checked build. */
int lbm_checked_status(void* stream);
int lbm_is_checked_build(void);

/* ------------------------------------------------------------------ batches
 * Many independent D2Q9 grids stepped together (the paper runs its 2-D cases
 * one at a time; batching them is a service of the library, the arithmetic
 * of every grid is that of lbm_step).  The grids share one set of population
 * arrays, each grid in its own ghost-padded block.  A step is ONE launch of a
 * persistent kernel whose CTAs take work items (grid, tile column, chunk of
 * planes) from a list in device memory, so that grids of any size mix
 * without idle launches.
 *
 * lbm_batch_create: n >= 1 grids, grids[i] and params[i] as for lbm_create
 * with lattice LBM_D2Q9 (nz = 1).  Every params[i].store must be the same.
 * Arrays are copied; the caller keeps ownership.  Allocates the population
 * arrays of all grids (4 x 9 x sum of padded grid sizes values).  Errors:
 * LBM_EINVAL (n < 1, a bad grid or parameter block, mixed storage, padded
 * total >= 2^31 cells), LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_create(int n, const lbm_grid* grids, const lbm_params* params, void* cuda_stream,
                     lbm_batch** out);

/* The context of grid i of the batch, owned by the batch (NULL if i is out
 * of range).  It accepts every per-grid call: lbm_init_fields,
 * lbm_set_populations, lbm_get_populations, lbm_macro, lbm_diagnostics,
 * lbm_laplace, lbm_get_tile.  lbm_step, lbm_step_profiled, lbm_autotune and
 * lbm_set_tile on it return LBM_EINVAL (the batch steps all its grids), and
 * lbm_destroy on it does nothing. */
lbm_ctx* lbm_batch_grid(lbm_batch* b, int i);

/* Advance every grid by n >= 0 steps: one persistent launch per step, or,
 * after lbm_batch_set_graph(b, k) with k >= 1, replays of a CUDA graph of k
 * steps (and single launches for the remainder).  Stream-ordered.  Errors:
 * LBM_EINVAL, LBM_ECUDA. */
int lbm_batch_step(lbm_batch* b, int n);

/* The same n steps as one launch of the single-grid step kernel (tile 1,
 * lz 16) per grid and step: the reference to compare the batch against.  */
int lbm_batch_step_sequential(lbm_batch* b, int n);

/* Batch step kernel: tile 0-3 = CTAs of 64, 128, 32 threads along x (in
 * phases) and 128 (g loads held across the phi fill); lz >= 1 planes per
 * work item.  Rebuilds the work list.  lbm_batch_get_tile also reports the
 * CTA width and the number of work items (any pointer may be NULL).
 * Errors: LBM_EINVAL. */
int lbm_batch_set_tile(lbm_batch* b, int tile, int lz);
int lbm_batch_get_tile(const lbm_batch* b, int* tile, int* lz, int* tx, int* n_items);

/* k >= 1: lbm_batch_step replays a CUDA graph of k step launches (captured
 * on a private stream on first use for each buffer parity, launched on the
 * batch stream); k = 0: single launches.  Errors: LBM_EINVAL (k < 0). */
int lbm_batch_set_graph(lbm_batch* b, int k);

/* Times every batch tile with lz in {4, 8, 16, 32} for `steps` steps each,
 * keeps the fastest, and restores the state it started from.  Reports the
 * choice and its time per step in ms (any pointer may be NULL).
 * Synchronises.  If a trial fails, the state is restored all the same, the
 * batch keeps the tile it had and the trial's status is returned.  Errors:
 * LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_autotune(lbm_batch* b, int steps, int* best_tile, int* best_lz, double* best_ms);

/* Kernel launches issued by the batch steps (graph replays count their
 * kernels). */
long long lbm_batch_launch_count(const lbm_batch* b);

/* The work list of a batch, computed on the host (no GPU needed): for grids
 * (D2Q9, internal axes x = user x, z = user y), CTA width tx >= 1 and lz >= 1,
 * the items in launch order, 4 ints each: grid index, first x, first z,
 * end z (exclusive); per grid, z chunks in order and within a chunk the
 * tile columns in order.  Writes at most max_items items (items may be NULL
 * with max_items = 0) and returns the total number of items, or LBM_EINVAL. */
int lbm_batch_plan(int n, const lbm_grid* grids, int tx, int lz, int* items, int max_items);

void lbm_batch_destroy(lbm_batch* b);

void lbm_destroy(lbm_ctx* ctx);
const char* lbm_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
