/*
 * lbmtau1.h - C ABI of the GB300 (sm_103a) LBMTau1 library.
 *
 * LBMTau1 is the D2Q9 lattice Boltzmann method with the relaxation time
 * fixed at tau = 1 (Matyka & Dzikowski, arXiv:1912.09327).  With tau = 1 the
 * post-collision populations are the equilibria, Eq. (LBMTau1), so a node's
 * new density and momentum are the sums of the equilibria of its nine
 * neighbours, Eqs. (rhotau1) and (utau1).  Only the moments are stored: two
 * copies (ping-pong, Section 2.1) of density and x/y momentum, as in
 * Eq. (LBMTau1memory).
 *
 * Conventions shared by every call:
 *   - A domain is nx * ny nodes.  Host arrays are row-major, idx = y*nx + x.
 *   - Node types (the flag array F of Algorithm 1, widened to three values):
 *       LBM_FLUID  0  updated every step;
 *       LBM_SOLID  1  no-slip wall, never updated; a fluid node pulling from
 *                     it takes the zero-velocity equilibrium of its own
 *                     density, w_k rho(x) (Eq. feqnoslip);
 *       LBM_FIXED  2  fixed-equilibrium node (the moving lid of Section 3 and
 *                     of Appendix A): never updated, pulled from like fluid.
 *   - An axis flagged periodic wraps; on a non-periodic axis a neighbour
 *     outside the domain counts as solid.
 *   - The body force (fx, fy) is added to a neighbour's momentum before its
 *     equilibrium is formed (Algorithm 1): u = (U + fx) / rho.
 *   - Moments cross the ABI as density rho and momentum (jx, jy) = rho*u,
 *     the quantities Eqs. (rhotau1) and (utau1) evolve, in double precision.
 *     Device storage is FP32: rho - 1, jx, jy.  A solid node holds no fluid
 *     state (the wall rule never reads it): the library stores rho - 1 = 0 and
 *     j = -F there, and lbm_moments reports it at rest, rho = 1, j = 0.
 *   - Every call returns LBM_OK (0) or a negative status; nothing aborts or
 *     throws across the ABI.  lbm_last_error() describes the last failure.
 *   - All device work is enqueued on the CUDA stream given to lbm_create.
 *     Calls that hand results to the host (lbm_moments, lbm_residual)
 *     synchronise that stream.  A context is not thread-safe.
 */
#ifndef LBMTAU1_H
#define LBMTAU1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LBM_OK 0
#define LBM_E_INVAL (-1)     /* bad argument (null pointer, size, type) */
#define LBM_E_WORKSPACE (-2) /* workspace missing, too small or misaligned */
#define LBM_E_CUDA (-3)      /* a CUDA runtime call or launch failed */
#define LBM_E_UNSTABLE (-4)  /* a step produced rho <= 0 or a non-finite value */
#define LBM_E_STATE (-5)     /* call out of order (e.g. step before geometry) */

/* Node types. */
#define LBM_FLUID 0
#define LBM_SOLID 1
#define LBM_FIXED 2

/* Device storage formats.  Arithmetic is FP32 in all of them; the residual
 * and mass reductions sum in FP32 per lane (the mass compensated) and in FP64
 * across lanes and tiles. */
#define LBM_STORAGE_F32 0  /* rho - 1, jx, jy as float32 (24 B/node, 2 copies) */
#define LBM_STORAGE_F16 1  /* as IEEE binary16, (rho - 1) * 2^10 and j * 2^6
                              (12 B/node, 2 copies) */
#define LBM_STORAGE_BF16 2 /* as bfloat16, unscaled (12 B/node, 2 copies) */

/* Rounding of the stored moments.
 * Stochastic rounding rounds a stored value up or down with probabilities
 * that make its expected value exact: increments smaller than half a unit in
 * the last place are not lost, and a near-constant increment (a body force
 * accelerating a flow) does not round the same way step after step.  Under
 * round-to-nearest a slowly converging flow stalls far from its steady state
 * in the 16-bit formats, and in FP32 a uniformly accelerated flow drifts by
 * up to half a unit in the last place per step (2e-5 relative after 2000
 * steps of the 754 x 246 channel of the batched mix, where stochastic
 * rounding keeps it at 3e-7).  Its price is noise: a steady state keeps
 * jittering by about one unit in the last place per step, which bounds the
 * residual a solve can reach from below.
 *   - 16-bit formats: every stored value, with random bits from a counter-
 *     based hash of (column, row, field, step count).
 *   - FP32: the momentum (rho - 1 rounds to nearest), by adding to each
 *     momentum increment a dither uniform over one unit in the last place of
 *     the stored value, drawn once per step from the step count.
 * Both are reproducible bit for bit.  The default is stochastic rounding
 * for the 16-bit formats and rounding to nearest for FP32. */
#define LBM_ROUND_DEFAULT 0
#define LBM_ROUND_NEAREST 1
#define LBM_ROUND_STOCHASTIC 2

/* Problem statement.  Zero-initialise before filling in. */
typedef struct lbm_params {
  int64_t nx;         /* nodes along x, 1 .. 2^30 - 1 */
  int64_t ny;         /* nodes along y, 1 .. 2^30 - 1 */
  int32_t periodic_x; /* nonzero: x wraps (e.g. the channel of Section 3) */
  int32_t periodic_y; /* nonzero: y wraps */
  double fx;          /* body force, momentum added per node per step */
  double fy;
  int32_t storage;    /* LBM_STORAGE_F32, _F16 or _BF16 */
  int32_t rounding;   /* LBM_ROUND_DEFAULT (0), _NEAREST or _STOCHASTIC */
  double sc_g;        /* Shan-Chen coupling g of the multiphase step; 0 (the
                         default) is the single-phase step.  See below. */
} lbm_params;

/*
 * Multiphase step (Section 4): with sc_g != 0 every pulled neighbour's
 * momentum also gets the pseudo-potential force of Eq. (f_sc),
 *   F_SC(x) = -g psi(x) sum_i w_i psi(x + e_i) e_i,  psi = 1 - exp(-rho),
 * (Shan and Chen's model: alpha_i = w_i, G(e_i) = -g e_i; psi = 0 at solid
 * nodes and outside non-periodic edges; g < -4 separates a liquid and its
 * vapour), added beside the body force before the division by the density,
 * where Algorithm 1 adds the body force.  At tau = 1 this velocity shift is
 * also Kupershtokh's exact-difference forcing.  The potential of every node
 * is computed once per step from the density the kernel streams, so no
 * potential field is stored.  FP32 storage only; batches take single-phase
 * members only.
 */

typedef struct lbm_ctx lbm_ctx;

/*
 * Device workspace needed for a domain, in bytes; 0 when p is invalid.
 * The storage model is the paper's, Eq. (LBMTau1memory) in Section 5: two
 * copies of N_f = 3 moment fields per node, 2 N_f c bytes (24 B in FP32,
 * against (2Q + N_f) c = 84 B for standard D2Q9, Eq. (lbmmemory)).  The
 * workspace holds both copies of the three moment fields (rows padded to a
 * multiple of 32 nodes), the node-type array (the flag array F of
 * Algorithm 1, 1 B per node), per-warp-tile reduction partials and a
 * bounded staging buffer for host transfers.
 */
size_t lbm_workspace_bytes(const lbm_params *p);

/*
 * Creates a context over a caller-owned device workspace: the two grids
 * R_c, U_c, V_c (c = 0, 1) of Algorithm 1 and the flag array F, laid out as
 * lbm_workspace_bytes describes.
 *   p               problem statement (copied).
 *   dev_workspace   device pointer, 256-byte aligned, >= lbm_workspace_bytes(p)
 *                   bytes; owned by the caller and must outlive the context.
 *   workspace_bytes size of that allocation.
 *   cuda_stream     cudaStream_t to enqueue all work on (NULL = legacy stream).
 *   out             receives the context.
 * The fields start at rest (rho = 1, j = 0) with every node fluid; call
 * lbm_set_geometry before stepping.
 * Errors: LBM_E_INVAL, LBM_E_WORKSPACE.
 */
int lbm_create(const lbm_params *p, void *dev_workspace, size_t workspace_bytes,
               void *cuda_stream, lbm_ctx **out);

/*
 * Sets the node types from a host array of nx*ny bytes (values 0, 1, 2; see
 * above; Algorithm 1, first line) and resets both copies of the fields to
 * rest, rho = 1 and j = 0 (the initial state of Section 2.1).  The array is
 * copied; the caller keeps ownership.
 * Errors: LBM_E_INVAL (null or a value > 2), LBM_E_CUDA.
 */
int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *host_mask);

/*
 * Loads a state: host arrays of nx*ny doubles with density rho (> 0) and
 * momentum jx, jy.  Fixed nodes keep the values given here for every later
 * step (a lid with speed u0 is rho = 1, jx = u0, jy = 0 as in Appendix A).
 * Errors: LBM_E_INVAL, LBM_E_STATE (no geometry yet), LBM_E_CUDA.
 */
int lbm_set_moments(lbm_ctx *ctx, const double *rho, const double *jx,
                    const double *jy);

/*
 * Enqueues nsteps LBMTau1 time steps (Algorithm 1), asynchronously.  The last
 * step of the call also reduces the residual and mass that lbm_residual
 * returns and checks for rho <= 0 or non-finite values.  nsteps = 0 is a
 * no-op.  On a stream that can be captured (not the legacy default stream,
 * and not under a capture of the caller's), runs of 16 inner steps are
 * replayed from a CUDA graph captured at first use (FP32 storage, or 16-bit
 * storage rounded to nearest; stochastic rounding launches every step).
 * Errors: LBM_E_INVAL (nsteps < 0), LBM_E_STATE, LBM_E_CUDA (launch failure).
 */
int lbm_step(lbm_ctx *ctx, int64_t nsteps);

/*
 * Tile variant (block tile shape, 0 .. lbm_variant_count() - 1) of the
 * context's step kernel.  All variants give bit-identical states; they differ
 * in how well their grid fills the device.  By default (variant -1) the first
 * step picks one from the domain size, the SM count and the kernels'
 * occupancy (the environment variable LBMTAU1_STEP_VARIANT, when set to a
 * valid index, overrides that choice).  lbm_set_variant may be called between
 * steps; lbm_variant returns the variant the next step uses, choosing it if
 * that has not happened yet (-1 for a null context).
 * Errors: LBM_E_INVAL (variant < -1 or >= lbm_variant_count()).
 */
int lbm_set_variant(lbm_ctx *ctx, int32_t variant);
int32_t lbm_variant(lbm_ctx *ctx);

/*
 * Failure detection (Section 5 names a crashing solver as the sign of
 * instability; a stalled copy is the other way a step can fail): every time
 * the step kernel waits for a row it has staged into shared memory with a
 * bulk copy, it waits at most `ns` nanoseconds (default 10^9, the maximum).
 * On expiry the warp stops, lets its copies still in flight land (that drain
 * keeps the one-second bound whatever the limit) and raises a flag, which
 * lbm_residual reports as LBM_E_CUDA; the fields are then incomplete, and
 * loading a state (lbm_set_moments / lbm_set_state) clears the flag.  A limit
 * of 0 makes every such wait give up at once without looking, which tests
 * this path without any fault.  Errors: LBM_E_INVAL (ns < 0 or > 10^9).
 */
int lbm_set_copy_wait_ns(lbm_ctx *ctx, int64_t ns);

/*
 * Copies the current state to caller-owned host arrays of nx*ny doubles:
 * density, and momentum jx, jy (velocity = j / rho).  Fixed nodes return the
 * values they hold, solid nodes rho = 1, j = 0.  Synchronises the stream.
 * Errors: LBM_E_INVAL, LBM_E_STATE, LBM_E_CUDA.
 */
int lbm_moments(lbm_ctx *ctx, double *rho, double *jx, double *jy);

/*
 * Exact state transfer in the device storage format, for checkpoint/resume:
 * three caller-owned host arrays of nx*ny elements (float for
 * LBM_STORAGE_F32, 16-bit words for _F16 and _BF16, scaled as stated above)
 * holding rho - 1, jx and jy exactly as stored (solid
 * nodes: 0, -fx, -fy; lbm_set_state writes those there whatever it is
 * given).  A state saved with lbm_get_state and loaded with lbm_set_state
 * into a context with the same parameters and geometry continues bit for bit.  lbm_get_state
 * synchronises; lbm_set_state returns once the host arrays have been read.
 * Errors: LBM_E_INVAL, LBM_E_STATE (no geometry yet), LBM_E_CUDA.
 */
int lbm_get_state(lbm_ctx *ctx, void *drho, void *jx, void *jy);
int lbm_set_state(lbm_ctx *ctx, const void *drho, const void *jx,
                  const void *jy);

/*
 * Steps the context has taken (lbm_step and batch steps), which seeds the
 * stochastic rounding of 16-bit storage: a checkpoint of such a context
 * saves it beside the state and a resume sets it again, so that the resumed
 * run continues bit for bit.  Errors: LBM_E_INVAL (null, steps < 0).
 */
int lbm_step_count(const lbm_ctx *ctx, int64_t *steps);
int lbm_set_step_count(lbm_ctx *ctx, int64_t steps);

/*
 * Residual and mass of the last step run by lbm_step, over fluid nodes, with
 * velocity u = j / rho:
 *   residual = sqrt(sum |u_n - u_{n-1}|^2 / sum |u_n|^2)  (the relative
 *              velocity change between consecutive steps used as the
 *              steady-state test in Section 3, taken over the whole field;
 *              sqrt(sum |u_n - u_{n-1}|^2) when the flow is at rest),
 *   mass     = sum rho_n.
 * Either pointer may be NULL.  Sums are taken in FP64.  Synchronises.
 * Errors: LBM_E_STATE (no step since the state was set), LBM_E_UNSTABLE
 * (the last reduced step saw rho <= 0 or a non-finite value; the values are
 * still written), LBM_E_CUDA.
 */
int lbm_residual(lbm_ctx *ctx, double *residual, double *mass);

/*
 * A termination test that rounding noise cannot hold off.  The residual
 * above compares consecutive steps, so it cannot fall below the noise of
 * the stored values: about one unit in the last place per step, 6e-4 for
 * FP16 and 5e-3 for BF16 stochastic storage, and near 6e-8 for some FP32
 * flows.  Section 3 tests convergence by the change between states
 * Delta t = 1000 steps apart (the cavity's flux check); these calls measure
 * the velocity change over any span:
 *   lbm_snapshot copies the current state into caller-owned device memory
 *   (256-byte aligned, lbm_snapshot_bytes(p) bytes, asynchronous);
 *   lbm_change_since returns, `steps` steps later,
 *     change = sqrt(sum |u_now - u_snap|^2 / sum |u_now|^2) / steps
 *   over fluid nodes (u = j / rho, FP64 sums; the plain sqrt of the first
 *   sum over steps when the flow is at rest): the mean relative velocity
 *   change per step over the span.  Noise of n units in the last place then
 *   adds only about n ulp / steps.  Synchronises the stream.
 * Errors: LBM_E_INVAL (null, misaligned or small buffer, steps < 1),
 * LBM_E_STATE, LBM_E_CUDA.
 */
size_t lbm_snapshot_bytes(const lbm_params *p);
int lbm_snapshot(lbm_ctx *ctx, void *dev_buf, size_t bytes);
int lbm_change_since(lbm_ctx *ctx, const void *dev_buf, int64_t steps,
                     double *change);

/*
 * One step that allocates no memory (the paper has no counterpart; this is
 * an interface for callers that cannot allocate device memory themselves,
 * such as an application that hands all device memory to its own pool
 * allocator and forbids side allocations, or a loop with a hard latency
 * budget where cudaMalloc / cudaFree are not acceptable).
 *
 * Runs one reduced LBMTau1 step, the same kernel as lbm_step, from
 * caller-owned device fields (rho - 1, jx, jy as float32, rows of `pitch`
 * elements) into a second caller-owned set, with the node types in a
 * caller-owned uint8 array of the same pitch.  It calls no cudaMalloc,
 * cudaFree or allocating library routine: the reduction scratch is a
 * file-scope device array of 6 MB (2^16 block tiles x 4 warp tiles x 3
 * doubles, plus the flag) that every GPU loading this library holds until
 * the process exits.
 *   Inputs:  drho_in, jx_in, jy_in, mask (all 16-byte aligned; pitch >= nx,
 *            pitch % 32 == 0; the mask buffer needs 256 bytes of slack after
 *            its last row, which bulk copies of aligned windows may read).
 *            What the fields hold at solid nodes never reaches a fluid node.
 *   Outputs: drho_out, jx_out, jy_out (same layout; columns nx..pitch-1 may be
 *            overwritten; fluid nodes get the step, fixed nodes their input
 *            values, solid nodes an unspecified value), dev_sums = device
 *            array of 3 doubles receiving
 *            sum |u_n - u_{n-1}|^2, sum |u_n|^2 and sum (rho_n - 1) over fluid
 *            nodes, dev_flags = device uint32 receiving 0 or a nonzero flag
 *            (bit 0: rho <= 0 or a non-finite moment; bit 1: a bulk row copy
 *            did not complete within one second).
 * Asynchronous on cuda_stream.  The first call on each device resolves the
 * scratch array's device address (cudaGetSymbolAddress); the first step of
 * the process (through any entry point) configures the kernels once, for the
 * device current then, so the library serves one device per process.  Make
 * the first call before any stream capture.  All calls share
 * the one scratch array, so calls that overlap on the GPU (for instance on
 * two streams) race; the array keeps the last call's contents, and the call
 * clears what must start at zero.
 * Errors: LBM_E_INVAL (null or misaligned pointer, bad size, or a domain
 * needing more than 2^16 thread blocks), LBM_E_CUDA.
 */
int lbm_step_noalloc(const float *drho_in, const float *jx_in,
                     const float *jy_in, float *drho_out, float *jx_out,
                     float *jy_out, const uint8_t *mask, int64_t nx,
                     int64_t ny, int64_t pitch, int32_t periodic_x,
                     int32_t periodic_y, double fx, double fy,
                     double *dev_sums, uint32_t *dev_flags, void *cuda_stream);

/* Frees the context's host state and its captured step graphs; the
 * workspace stays the caller's.  (Host bookkeeping: the paper has no
 * counterpart.) */
void lbm_destroy(lbm_ctx *ctx);

/*
 * Batches: one launch per time step for many independent domains.
 *
 * The paper steps one domain at a time; independent domains (Algorithm 1
 * applied to each) can share a launch.  A batch references existing contexts
 * (each with its own workspace, geometry and state) that use the batch's
 * stream.  lbm_batch_step advances every member by nsteps with one launch per
 * step over a work list of all members' block tiles, taken by a persistent
 * grid through an atomic counter; runs of steps inside a call are replayed
 * from a captured CUDA graph.  Each member ends bit for bit where it would
 * have ended alone, and afterwards lbm_moments / lbm_residual / lbm_step work
 * on it as usual (the last step of the call is reduced for every member).
 */
typedef struct lbm_batch lbm_batch;

/* Device workspace of a batch of up to `capacity` members whose block tiles
 * number at most `max_tiles` in total (< 2^29); 0 when the arguments are
 * invalid. */
size_t lbm_batch_workspace_bytes(int32_t capacity, int64_t max_tiles);

/* Creates a batch over a caller-owned device workspace (256-byte aligned) on
 * cuda_stream.  Errors: LBM_E_INVAL, LBM_E_WORKSPACE. */
int lbm_batch_create(int32_t capacity, int64_t max_tiles, void *dev_workspace,
                     size_t workspace_bytes, void *cuda_stream,
                     lbm_batch **out);

/* Adds a context (same stream and storage format as the other members,
 * geometry set, single phase) and returns its slot; the context must outlive
 * its membership.  Errors: LBM_E_INVAL (also a multiphase context),
 * LBM_E_STATE, LBM_E_WORKSPACE (full). */
int lbm_batch_add(lbm_batch *b, lbm_ctx *ctx, int32_t *slot);

/* Removes the member in `slot` (between steps).  Errors: LBM_E_INVAL. */
int lbm_batch_remove(lbm_batch *b, int32_t slot);

/* Number of members. */
int32_t lbm_batch_members(const lbm_batch *b);

/* Advances every member by nsteps (asynchronous on the batch stream).
 * Errors: LBM_E_INVAL, LBM_E_WORKSPACE (more tiles than the workspace holds),
 * LBM_E_CUDA. */
int lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Tile variants (block tile shapes) of the step kernels: their count, and
 * the one a batch uses (set by hand or by lbm_batch_autotune; the default is
 * variant 0 unless LBMTAU1_STEP_VARIANT names another).  All variants give
 * bit-identical states. */
int32_t lbm_variant_count(void);
int lbm_batch_set_variant(lbm_batch *b, int32_t variant);
int32_t lbm_batch_variant(const lbm_batch *b);

/* Block tiles of an nx x ny domain under tile variant `variant`, or the
 * largest count over all variants for variant -1 (the bound to size a batch
 * workspace with when the autotuner may try every variant); -1 for invalid
 * arguments. */
int64_t lbm_tile_count(int64_t nx, int64_t ny, int32_t variant);

/* Block tile of a variant: tile_x columns (30 lanes of cols_per_lane
 * columns each, plus one halo lane on either side) by tile_y rows (four
 * warps of tile_y / 4 rows, each also reading one row above and below).
 * cols_per_lane may be NULL.  Errors: LBM_E_INVAL. */
int lbm_variant_tile(int32_t variant, int64_t *tile_x, int64_t *tile_y,
                     int32_t *cols_per_lane);

/* 1 when a variant's kernel also carries the code for clean warp tiles
 * (every node of the tile and its one-node halo in the domain and fluid),
 * which the per-tile flags select; its tiles are those of the variant of the
 * same shape without it.  0 when it does not, -1 for an invalid variant. */
int32_t lbm_variant_has_clean_code(int32_t variant);

/* Autotuner: times steps_per_variant (even, >= 2) batch steps, plus two
 * warm-up steps, with every tile variant and keeps the fastest.  These are
 * real steps: every member advances by (steps_per_variant + 2) times the
 * variant count.  ms_per_step (NULL or lbm_variant_count() doubles) receives
 * the measured time per step of each variant.  Synchronises the stream. */
int lbm_batch_autotune(lbm_batch *b, int32_t steps_per_variant,
                       int32_t *chosen, double *ms_per_step);

/* Residual and mass of every member's last step (as lbm_residual), by slot,
 * read with one device-to-host copy: residual, mass and status are host
 * arrays of the batch capacity; status[slot] is LBM_OK, LBM_E_UNSTABLE,
 * LBM_E_CUDA (copy timeout) or LBM_E_STATE (empty slot / no step yet).
 * Synchronises the stream.  Errors: LBM_E_INVAL, LBM_E_CUDA. */
int lbm_batch_residuals(lbm_batch *b, double *residual, double *mass,
                        int32_t *status);

/* Frees the batch's host state (members and workspace stay the caller's). */
void lbm_batch_destroy(lbm_batch *b);

/* Message for the last failed call on the batch. */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Message for the last failed call on ctx ("" when none; static text for a
 * NULL ctx).  Valid until the next call on ctx. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Static name of a status code. */
const char *lbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBMTAU1_H */
