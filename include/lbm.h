/*
 * lbm.h -- C ABI of the GB300-native rectangular central-moment lattice
 * Boltzmann library (liblbm_gb300.so).
 *
 * The library advances the D2Q9 RC-LBM of Yahia & Premnath, "Central Moment
 * Lattice Boltzmann Method on a Rectangular Lattice" (arXiv 2103.02119),
 * Sec. 4: per cell and time step it maps the nine distributions to raw and
 * central moments (Eq. 4, App. B), relaxes the central moments towards the
 * Maxwell-matched equilibria carrying the isotropy and Galilean-invariance
 * corrections (Eq. 23-27, 37-40, 49), maps back (Eq. 55, App. A) and streams
 * along the rectangular links e_i = (+-1, +-a) (Eq. 2), with half-way
 * bounce-back walls (Sec. 5.1, Eq. 57-59) and body forcing in the same pass.
 * Every step runs as hand-written CUDA kernels for sm_103a on one GPU; there
 * is no CPU fallback.
 *
 * Lattice units: dx = dt = 1, dy = a.  Cell (x, y), 0 <= x < nx, 0 <= y < ny,
 * has linear index y*nx + x (x fastest).  Direction order 0..8 is the order
 * of Eq. 2: (0,0) (1,0) (0,a) (-1,0) (0,-a) (1,a) (-1,a) (-1,-a) (1,-a).
 *
 * Conventions of every entry point:
 *   - The return value is an lbm_status; nothing is thrown across the ABI.
 *   - Host arrays are owned by the caller and copied; the library keeps no
 *     pointer to them after the call returns.  Device arrays (on_device != 0)
 *     must be device memory of the handle's device, owned by the caller.
 *   - Work is issued on the CUDA stream given to lbm_create (borrowed, never
 *     destroyed; NULL = the legacy default stream).  lbm_step and the
 *     on_device variants are asynchronous on that stream; calls that read
 *     into host memory synchronise it before returning.
 *   - On an error the handle stays valid and lbm_last_error describes the
 *     failure.  Invalid parameters are rejected on the host before any
 *     device work: a NULL handle, a NULL required pointer or an argument out
 *     of its stated range gives LBM_ERR_INVALID; a failed allocation
 *     LBM_ERR_OOM; a failed CUDA call LBM_ERR_CUDA.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = -1,  /* argument or parameter rejected; nothing was done */
    LBM_ERR_OOM = -2,      /* a device or host allocation failed              */
    LBM_ERR_CUDA = -3,     /* a CUDA call failed (see lbm_last_error)          */
    LBM_ERR_UNSTABLE = -4, /* lbm_diagnostics found non-finite fluid cells     */
    LBM_ERR_TIMEOUT = -5,  /* a step kernel gave up waiting for its staged data
                              (reported by lbm_diagnostics; the state is not
                              valid after it)                                  */
    LBM_ERR_STATE = -6,    /* state buffer of the wrong size                   */
    LBM_ERR_BOUNDS = -7    /* checked build: a device bounds check failed      */
} lbm_status;

/* Number of doubles written by lbm_diagnostics. */
#define LBM_DIAG_COUNT 8

typedef struct {
    int32_t nx, ny;        /* cells along x and y, each >= 3                    */
    double a;              /* grid aspect ratio dy/dx (Sec. 2.1), > 0           */
    double cs2;            /* speed of sound squared, 0 < cs2 < min(1, a^2)     */
    double omega[9];       /* relaxation rates of Eq. 5 (Lambda), each in
                              [0, 2], omega[3] and omega[4] > 0.  Shear
                              viscosity nu = cs2 (1/omega[4] - 1/2) (Eq. 32),
                              omega[5] should equal omega[4]; bulk viscosity
                              from omega[3] (Eq. 33).  omega[0..2] have no
                              effect (conserved moments).                      */
    double Fx, Fy;         /* uniform body-force density (Sec. 4, Phi^c)        */
    double rho0;           /* reference density of the stored deviations
                              f_i - w_i rho0 (w_i: rest equilibrium weights);
                              0 stores raw f_i                                  */
    int32_t precision;     /* 32: FP32 storage and arithmetic, 64: FP64         */
    int32_t periodic_x;    /* 1: periodic along x; 0: walls at x = -1, x = nx   */
    int32_t periodic_y;    /* 1: periodic along y; 0: walls at y = -1, y = ny   */
    double wall_u[4][2];   /* wall velocity (Ux, Uy) of the left, right,
                              bottom and top walls; a node outside the domain
                              in both x and y (a corner) belongs to the bottom
                              or top wall                                        */
    int32_t use_iso_corr;  /* 1: isotropy correction m^{eq,s} (Eq. 23-24)       */
    int32_t use_gi_corr;   /* 1: Galilean-invariance correction (Eq. 25-26)     */
    int32_t block_x;       /* step kernel tuning: threads per block along x,
                              0 = automatic, else one of 32, 64, 128, 256        */
    int32_t bands;         /* step kernel tuning: number of row bands,
                              0 = automatic                                     */
    int32_t scheme;        /* 0: RC-LBM collision (Sec. 4); 1: raw-moment
                              collision (RNR-LBM, Sec. 3: Eq. 10-13 with the
                              same corrections); -1: no collision (streaming
                              and bounce-back only, a test mode in which a
                              step is a permutation of the state)               */
} lbm_params;

/* Build flags of the loaded library (library plumbing): bit 0
 * (LBM_BUILD_CHECKED) is set in the checked build, compiled with
 * LBM_CHECKED, whose step kernels test every computed global, link-mask and
 * shared-memory index; a failed test skips the access, and the next
 * lbm_diagnostics, lbm_diagnostics_noalloc or lbm_batch_residuals returns
 * LBM_ERR_BOUNDS (the state is then not valid).  The normal build has no
 * such tests. */
#define LBM_BUILD_CHECKED 1
int lbm_build_flags(void);

/* Fill *p with defaults: 64 x 64 periodic, a = 1, cs2 = 1/3 (the square
 * lattice, where the corrections of Eq. 23-24 vanish), all omega 1, no
 * force, rho0 = 1, precision 32, both corrections on, automatic tuning,
 * RC-LBM scheme (Sec. 4).  p NULL: LBM_ERR_INVALID. */
lbm_status lbm_params_init(lbm_params* p);

/* Create a lattice.  p: parameters (copied).  solid_mask: nullable, nx*ny
 * bytes in cell order, non-zero = stationary solid node (copied); a fluid
 * cell whose 8 neighbours are all wall or solid nodes is made solid.
 * cuda_stream: a cudaStream_t or NULL (borrowed).  The new handle owns all of
 * its device memory; its state is the rest state rho = 1, u = 0.
 * Errors: LBM_ERR_INVALID (bad parameters, NULL out), LBM_ERR_OOM,
 * LBM_ERR_CUDA.  *out is NULL on failure. */
lbm_status lbm_create(const lbm_params* p, const uint8_t* solid_mask,
                      void* cuda_stream, lbm_handle** out);

/* Destroy a handle and free its device memory.  NULL is ignored. */
void lbm_destroy(lbm_handle* h);

/* Set the state to the equilibrium f_i = f_i^eq(rho, u) of Sec. 4
 * (T^-1 F(-u) applied to the Maxwell-matched central moments) at every fluid
 * cell.  rho, ux, uy: nx*ny doubles each, nullable (rho = 1, u = 0); host
 * memory, or device memory when on_device != 0.  Resets the step counter and
 * the residual reference of lbm_diagnostics. */
lbm_status lbm_init_fields(lbm_handle* h, const double* rho, const double* ux,
                           const double* uy, int on_device);

/* Advance nsteps >= 0 time steps (collide + stream, Sec. 4), one kernel
 * launch per step; runs of 50 steps replay a CUDA graph the handle captures
 * once per starting buffer (on a stream of its own; lbm_set_force drops
 * it).  Small lattices run many steps per launch (lbm_set_small_path).  Asynchronous: the return value reports launch errors only. */
lbm_status lbm_step(lbm_handle* h, int64_t nsteps);

/* Replace the uniform body force density F (Sec. 4: it shifts the velocity
 * to (sum f e + F/2) / rho and enters the collision through the central
 * source moments); takes effect from the next step.  Non-finite values give
 * LBM_ERR_INVALID. */
lbm_status lbm_set_force(lbm_handle* h, double Fx, double Fy);

/* Kernel choice for small lattices (library plumbing; the paper runs one
 * fused step per launch at every size).  A lattice of at most 4096 cells
 * whose cluster fits the device runs the steps of an lbm_step call in
 * launches of up to 1024 steps each, every launch one thread-block cluster
 * of min(ny, 16) CTAs that synchronise twice per step (density field, then
 * collide and stream); the states are bit for bit those of the row-band
 * kernel.  enable = 0 makes the handle use the row-band kernel (one launch
 * per step); enable = 1 (the default where available) brings the cluster
 * back.  enable not 0 or 1, or 1 for a lattice without the cluster path:
 * LBM_ERR_INVALID. */
lbm_status lbm_set_small_path(lbm_handle* h, int enable);

/* Test hook for the failure path of the bounded waits (the paper has no
 * counterpart: this is library plumbing).  A step kernel waits for each row
 * of staged populations on an mbarrier for at most `polls` polls (default
 * and maximum 4194304 = 2^22, far above what a copy takes); when a wait runs
 * out, the block records it in the handle's status word, waits with the full
 * bound for its copies still in flight, and returns, leaving the state
 * invalid; lbm_diagnostics and lbm_diagnostics_noalloc then return
 * LBM_ERR_TIMEOUT until lbm_init_fields, lbm_set_f or lbm_set_state gives
 * the handle a new state.  polls = 0 makes every such wait run out at once.
 * Takes effect from the next lbm_step.  polls outside [0, 2^22]:
 * LBM_ERR_INVALID. */
lbm_status lbm_set_wait_limit(lbm_handle* h, int64_t polls);

/* Test hook for the allocation failure path (library plumbing, process
 * wide, not thread-safe with concurrent allocations): nth >= 1 makes the
 * nth device allocation the library attempts from now on fail as if the
 * device were out of memory (no CUDA call is made for it); the entry point
 * making it returns LBM_ERR_OOM, releases what it had allocated, and
 * lbm_last_error names the allocation.  nth = 0 disarms the hook.  nth < 0:
 * LBM_ERR_INVALID. */
lbm_status lbm_debug_fail_alloc(int64_t nth);

/* Macroscopic fields of the current state: rho = sum_i f_i and
 * u = (sum_i f_i e_i + F/2) / rho (Sec. 4, last step).  Each output is
 * nx*ny doubles, nullable; solid cells give 0.  Host outputs synchronise the
 * stream; device outputs (on_device != 0) are written asynchronously. */
lbm_status lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy,
                       int on_device);

/* Local strain rates and viscous stress of the current state, in FP64, as
 * the next collision sees it (Sec. 2.2): d_x u_x and d_y u_y from the
 * second-order non-equilibrium raw moments (Eq. 34-35, 37-38, 40), the
 * off-diagonal rate d_y u_x + d_x u_y from m5 - rho ux uy over
 * D1 = -rho cs2 / omega[5] (Eq. 36, 39: its left side is read as the
 * off-diagonal rate, as Eq. 21 gives it), with the density gradient of the
 * step (central differences, spacing 2 and 2a, a wall or solid neighbour
 * taking the cell's own density); and the viscous stress of the recovered
 * Navier-Stokes equations (Eq. 30-33):
 *   txx = rho [nu (2 d_x u_x - div u) + zeta div u], tyy likewise,
 *   txy = rho nu' (d_y u_x + d_x u_y),
 * nu = cs2 (1/omega[4] - 1/2), nu' = cs2 (1/omega[5] - 1/2),
 * zeta = cs2 (1/omega[3] - 1/2).  Each output is nx*ny doubles, nullable;
 * solid cells give 0.  Host or device memory as for lbm_moments (host
 * outputs synchronise the stream).  Uses a staging buffer of the handle
 * (7 nx ny doubles for host outputs, nx ny for device outputs). */
lbm_status lbm_stress(lbm_handle* h, double* dxux, double* dyuy, double* sxy,
                      double* txx, double* tyy, double* txy, int on_device);

/* Distributions f_i(x, t) of the current state (after streaming; i in the
 * order of Eq. 2), as doubles, 9*nx*ny in plane-major order
 * f[i*nx*ny + y*nx + x]; solid cells give 0.  Host or device memory as
 * above. */
lbm_status lbm_get_f(lbm_handle* h, double* f, int on_device);

/* Set the current state from distributions in the layout of lbm_get_f
 * (rounded to the handle's precision).  Values at solid cells are ignored.
 * Resets the step counter and the residual reference. */
lbm_status lbm_set_f(lbm_handle* h, const double* f, int on_device);

/* FP64 global diagnostics over the fluid cells, synchronous (rho and u as
 * in Sec. 4's last step; the paper defines no global diagnostics or steady
 * test: the sums and the residual below are this library's):
 *   out[0] mass  = sum rho; the stored values are summed exactly (fixed
 *                  point), so a permutation of the state gives the same bits
 *   out[1] sum rho u_x, out[2] sum rho u_y, out[3] sum rho |u|^2 / 2
 *   out[4] steady residual sqrt(sum |ubar(n) - ubar(m)|^2) / ((n - m)
 *          sqrt(sum |ubar(n)|^2)) against the state m of the previous call,
 *          or -1 when there is no previous call (or n == m), where
 *          ubar(n) = (u(n) + u(n-1)) / 2 is the mean velocity of the last
 *          two steps (u(n) alone before the first step since the state was
 *          set).  The scheme carries two exact invariants besides the mass,
 *          the staggered momenta sum (-1)^(x+n) rho u_x and
 *          sum (-1)^(y+n) rho u_y (streaming with half-way bounce-back moves
 *          their carriers one cell and flips their sign, the collision
 *          conserves momentum): motion along them alternates every step and
 *          never decays, a residual between states an even number of steps
 *          apart is blind to it, and the two-step mean cancels it
 *   out[5] number of fluid cells with a non-finite rho or u
 *   out[6] step counter n
 *   out[7] step-to-step change sqrt(sum |u(n) - u(n-1)|^2) / sqrt(sum
 *          |ubar(n)|^2), which such alternating motion keeps away from zero;
 *          -1 before the first step since the state was set
 * Returns LBM_ERR_UNSTABLE (with out filled) when out[5] > 0, and
 * LBM_ERR_TIMEOUT (out not written) when a step kernel gave up a bounded
 * wait for its staged data since the state was last set (lbm_create,
 * lbm_init_fields, lbm_set_f, lbm_set_state; see lbm_set_wait_limit). */
lbm_status lbm_diagnostics(lbm_handle* h, double out[LBM_DIAG_COUNT]);

/* The values of lbm_diagnostics, for callers that cannot allocate device
 * memory: a process whose free device memory is already reserved by another
 * allocator (a framework's caching allocator, say), so that cudaMalloc would
 * fail, or a monitoring loop that must not pay cudaMalloc's implicit device
 * synchronisation.  lbm_diagnostics allocates its residual reference field
 * on its first call; this entry point allocates nothing.  Its scratch -- the
 * per-block partial sums and the reference velocity field of the residual --
 * is one fixed device array inside the library (about 16.1 MiB) that every
 * GPU loading the library holds until the process exits.
 * Limit: lattices of at most 1048576 (2^20) cells; larger ones get
 * LBM_ERR_INVALID and a message naming the limit.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.
 * All calls on a device share the array: out[4] is measured against the
 * velocity of the previous lbm_diagnostics_noalloc call, and is -1 unless
 * that call was on the same handle at a smaller step count (init and set
 * calls in between are not detected).  Calls that overlap on the GPU (other
 * streams, other threads) race on the array.  Like lbm_diagnostics it
 * returns LBM_ERR_TIMEOUT (out not written, no residual reference taken)
 * after a step kernel gave up a bounded wait.
 * The paper has no counterpart to this entry point: it is library plumbing. */
lbm_status lbm_diagnostics_noalloc(lbm_handle* h, double out[LBM_DIAG_COUNT]);

/* Size in bytes of the raw state (checkpoint) of a handle; 0 for NULL.
 * Checkpointing has no counterpart in the paper (library plumbing). */
size_t lbm_state_bytes(const lbm_handle* h);

/* Copy the raw device state (storage precision, internal layout) to / from
 * host memory of exactly lbm_state_bytes bytes, synchronously.  A state
 * copied out and back continues bit-identically.  LBM_ERR_STATE on a size
 * mismatch. */
lbm_status lbm_get_state(lbm_handle* h, void* host, size_t bytes);
lbm_status lbm_set_state(lbm_handle* h, const void* host, size_t bytes);

/* Time steps taken since the last init / set call; -1 for NULL. */
int64_t lbm_step_count(const lbm_handle* h);

/* Number of kernel launches issued by lbm_step so far on this handle; -1
 * for NULL. */
int64_t lbm_launch_count(const lbm_handle* h);

/* Message of the last error on h (or of the last failed lbm_create when h is
 * NULL); never NULL.  Not thread-safe. */
const char* lbm_last_error(const lbm_handle* h);

/* ------------------------------------------------------------------------
 * Batches: many independent FP32 lattices of uneven size, aspect ratio and
 * parameters advanced together.  Each lattice runs exactly the scheme of
 * lbm_step (Sec. 4, with the walls of Sec. 5.1): a lattice of a batch and an
 * lbm_handle created from the same parameters and mask go through the same
 * states bit for bit.  The paper solves one lattice at a time; batching, the
 * steady-state residual loop and the autotuner are library plumbing with no
 * counterpart there.
 *
 * Every step of a batch is one launch of a persistent kernel per group of
 * lattices, each walking a list of (lattice, column segment, band of rows)
 * work items of its group's active lattices.  When they fit, the active
 * lattices form up to 4 groups of one scheme and at most 180 lattices
 * each, whose parameter tables sit in constant memory (one table per group,
 * shared by every batch of the device: a batch whose tables another batch
 * has replaced re-uploads them after a device synchronisation; batches
 * stepped at the same time from several host threads must not use this
 * path); the groups' kernels run one after another on the batch's stream.
 * Otherwise one kernel per
 * scheme reads the parameters from a table in global memory (slower: they
 * then take vector registers).  Runs of 50 steps replay a captured CUDA
 * graph.  Lattices
 * can be retired (made inactive) and brought back; an inactive lattice keeps
 * its state and is not stepped.  Conventions as for lbm_handle; work is
 * issued on the stream given to lbm_batch_create.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

/* Create `count` (1 .. 2^20) lattices.  params: count parameter sets as for
 * lbm_create, each with precision 32 and fewer than 2^31 stored values per
 * buffer (9 x ny x nx rounded up to 32); block_x and bands are ignored (the
 * batch has one launch shape, see lbm_batch_set_shape).  solid_masks:
 * nullable, else count pointers, each nullable or nx*ny bytes as for
 * lbm_create (copied).  Every lattice starts at rest and active.  Device
 * memory: two population buffers, a link mask and a residual reference field
 * (2 nx ny doubles) per lattice, in one allocation each.
 * Errors: LBM_ERR_INVALID (naming the first bad lattice), LBM_ERR_OOM,
 * LBM_ERR_CUDA; *out is NULL on failure. */
lbm_status lbm_batch_create(const lbm_params* params, int count,
                            const uint8_t* const* solid_masks, void* cuda_stream,
                            lbm_batch** out);

/* Destroy a batch and free its device memory.  NULL is ignored. */
void lbm_batch_destroy(lbm_batch* b);

/* Number of lattices, or -1 for NULL. */
int lbm_batch_count(const lbm_batch* b);

/* lbm_init_fields for lattice k (0 <= k < count): equilibrium state of
 * Sec. 4 from rho, ux, uy (nullable; host or device).  Resets its step
 * counter and residual reference. */
lbm_status lbm_batch_init_fields(lbm_batch* b, int k, const double* rho,
                                 const double* ux, const double* uy, int on_device);

/* Advance every active lattice by nsteps >= 0 steps.  Asynchronous. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Steady residual of every lattice, synchronous: res (count doubles,
 * nullable) gets, for each active lattice, the residual of lbm_diagnostics'
 * out[4] (FP64 sums over its fluid cells, on the two-step mean velocity)
 * against its mean velocity at its previous check, -1 if there was none (or
 * no step since, or u = 0), NaN if
 * it holds non-finite values; inactive lattices keep their last value.
 * Returns LBM_ERR_UNSTABLE when a lattice holds non-finite values and
 * LBM_ERR_TIMEOUT when a step kernel gave up a bounded wait since the
 * previous check: the lattices active in those steps then hold invalid
 * states (re-initialise them), and the report is cleared. */
lbm_status lbm_batch_residuals(lbm_batch* b, double* res);

/* Run to a steady state: check the residuals, then repeat {step
 * check_every (>= 1) steps; check} until every lattice is inactive or
 * max_steps steps have been taken in this call.  A lattice whose residual
 * is in [0, tol] is retired at that check; one that holds non-finite values
 * is retired too and the call returns LBM_ERR_UNSTABLE after the others
 * finish.  Lattices still active at max_steps stay active.  res: nullable,
 * count doubles, the last residual of each lattice. */
lbm_status lbm_batch_run(lbm_batch* b, double tol, int64_t check_every,
                         int64_t max_steps, double* res);

/* Retire (on = 0) or re-activate (on = 1) lattice k. */
lbm_status lbm_batch_set_active(lbm_batch* b, int k, int on);

/* 1 if lattice k is active, 0 if retired, -1 for a bad argument. */
int lbm_batch_is_active(const lbm_batch* b, int k);

/* Launch shape of the batch step: threads per block along x (32, 64 or 128;
 * a block covers 2 x block_x columns) and target rows per band (1 .. 65536;
 * lattice k gets max(1, round(ny_k / rows_per_band)) bands).  The shape
 * changes the schedule only, never the results.  Default 32, 16. */
lbm_status lbm_batch_set_shape(lbm_batch* b, int block_x, int rows_per_band);
lbm_status lbm_batch_get_shape(const lbm_batch* b, int* block_x, int* rows_per_band);

/* Whether the active lattices step from the constant-memory tables when they
 * fit (enable = 1, the default) or always from the global table (0).  The
 * choice changes the schedule only, never the results.  Errors:
 * LBM_ERR_INVALID. */
lbm_status lbm_batch_set_table_path(lbm_batch* b, int enable);

/* The number of constant-memory table groups the active lattices step in
 * (0: the global-table kernel), or -1 for a NULL batch or a failed upload of
 * the work lists. */
int lbm_batch_table_groups(lbm_batch* b);

/* lbm_set_wait_limit for every lattice of the batch (a test hook): from the
 * next step the batch kernel's row waits give up after `polls` polls; a
 * wait that runs out is reported by lbm_batch_residuals / lbm_batch_run as
 * LBM_ERR_TIMEOUT.  polls outside [0, 2^22]: LBM_ERR_INVALID. */
lbm_status lbm_batch_set_wait_limit(lbm_batch* b, int64_t polls);

/* Autotuner: times trial_steps (>= 1) steps of the active lattices at each
 * block_x in {32, 64, 128} and rows_per_band in {1, 2, 4, 8, 16, 32, 64} (one warm-up
 * step each, CUDA events on the batch's stream), keeps the fastest shape and
 * returns it (outputs nullable).  The trial steps are real steps of the
 * active lattices (21 (trial_steps + 1) in all): the shape does not change
 * the results.  Synchronous. */
lbm_status lbm_batch_tune(lbm_batch* b, int trial_steps, int* block_x,
                          int* rows_per_band);

/* lbm_moments, lbm_get_f and lbm_diagnostics for lattice k.  The
 * diagnostics' out[4] is the lattice's last residual of
 * lbm_batch_residuals / lbm_batch_run. */
lbm_status lbm_batch_moments(lbm_batch* b, int k, double* rho, double* ux,
                             double* uy, int on_device);
lbm_status lbm_batch_get_f(lbm_batch* b, int k, double* f, int on_device);
lbm_status lbm_batch_diagnostics(lbm_batch* b, int k, double out[LBM_DIAG_COUNT]);

/* Steps taken by lattice k since its last init (-1 for a bad argument). */
int64_t lbm_batch_step_count(const lbm_batch* b, int k);

/* Batch step kernel launches issued so far: one per step, two when the
 * batch holds lattices of both schemes (one persistent launch each). */
int64_t lbm_batch_launch_count(const lbm_batch* b);

/* Message of the last error on b (or of the last failed lbm_batch_create
 * when b is NULL); never NULL. */
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- Measurement: the roofs the step is reported against ----
 * Neither has a counterpart in the paper; they measure the GPU, not the
 * method.  Both run on the current device, are synchronous, allocate and
 * free their own device buffers, and return LBM_ERR_INVALID for a bad
 * argument (nothing is run), LBM_ERR_OOM or LBM_ERR_CUDA otherwise.
 *
 * Device-to-device copy bandwidth (the HBM roof of FP32 storage, whose step
 * reads and writes each population once): allocates two buffers of `bytes`
 * (a multiple of 16, >= 16), copies one into the other once untimed and
 * `iters` (>= 1) times timed with CUDA events on `stream` (nullable: the
 * default stream), in 16-byte words by 8 blocks of 256 threads per SM;
 * *gbs = 2 bytes iters / time / 1e9 (read plus write). */
lbm_status lbm_peak_copy_gbs(size_t bytes, int iters, void* stream, double* gbs);

/* FP64 fused multiply-add rate (the roof of FP64 storage, whose step is
 * bound by the FP64 pipe): 4 blocks of 256 threads per SM, each thread
 * running 8 independent chains of `iters` (>= 1) FMAs, one untimed and one
 * timed launch on `stream`; *gflops = 2 FMAs / time / 1e9. */
lbm_status lbm_peak_fp64_gflops(int iters, void* stream, double* gflops);

#ifdef __cplusplus
}
#endif
#endif
