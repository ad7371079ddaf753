/*
 * dvm.h -- C ABI of libdvm, a GB300 (sm_103a) solver for the steady linearized BGK equation by the
 * discrete velocity method (DVM), for small force-driven gas flows through irregular 2D channels.
 *
 * Paper: S. Lindsay, W. Su, H. Liu and L. Wu, "Comparative study of the discrete velocity and
 * lattice Boltzmann methods for rarefied gas flows through irregular channels", arXiv:1704.03126.
 *
 * The problem (Sec. II.A, Eq. BGK with the time derivative dropped):
 *     v . grad h = L(rho, u, tau) - delta h + F v1,   L = delta [rho + 2 u.v + tau (|v|^2 - 1)],
 * f = f_eq (1 + h), f_eq = exp(-|v|^2)/pi, delta = sqrt(pi)/(2 Kn) (Eq. BGK), moments
 * rho = int h f_eq, u = int v h f_eq, tau = int |v|^2 h f_eq - rho, diffuse walls (Eq. diffuse2),
 * staircase geometry on a Cartesian mask, periodic inlet/outlet (Sec. II.A; Sec. III for porous
 * media with both axes periodic), the unit body force F v1 driving Poiseuille flow (Sec. III), a
 * moving top plate for Couette flow (Sec. II, Eq. diffuse1), and the source iteration of Eq.
 * (iteration) with second-order upwind differences (on rows of unequal height if given, Sec. II.A).
 * Extensions beyond the paper: the adjoint gradient dQ/d delta_c, batched solves with an autotuned
 * sweep kernel, FP32 storage with FP64 accumulation, Anderson mixing of the iteration, and a
 * self-test of the bounded device-side waits.
 *
 * Conventions for every call:
 *   - Arrays named [ny][nx] are row-major with the x1 index fastest; row j is at x2 = (j + 1/2) H/ny
 *     (the centre of row j when row heights are given), whatever the storage order (dvm_storage).
 *   - Pointers marked "host" are ordinary host memory; the library never keeps them.
 *   - The library copies every input; outputs are caller-allocated.
 *   - Calls return a dvm_status and never abort; dvm_last_error() describes the last failure on a
 *     context.  A context is not thread-safe: one host thread at a time.
 *   - Work runs on the CUDA stream given to dvm_create (NULL = the library creates its own); calls
 *     that return host data synchronise that stream.
 */
#ifndef DVM_H
#define DVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvm_ctx dvm_ctx; /* opaque; created by dvm_create, released by dvm_destroy */

typedef enum {
  DVM_OK = 0,
  DVM_EINVAL = 1,   /* invalid argument or unsupported configuration */
  DVM_ENOMEM = 2,   /* host or device allocation failed */
  DVM_ECUDA = 3,    /* a CUDA runtime call failed (message in dvm_last_error) */
  DVM_ENOCONV = 4,  /* max_iter reached before the stopping test passed (results are the last iterate) */
  DVM_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  DVM_ENUMERIC = 6, /* a NaN or Inf appeared in the moments */
  DVM_ESTATE = 7    /* call out of order (e.g. results requested before a successful solve) */
} dvm_status;

typedef enum {
  DVM_QUAD_GAUSS_HERMITE = 0, /* n Gauss-Hermite nodes per axis */
  DVM_QUAD_NEWTON_COTES = 1,  /* closed trapezoid rule on n equispaced nodes in [-vmax, vmax] */
  DVM_QUAD_CUBIC = 2          /* Eq. (nonuniform_v): v = 4 s^3/(n-1)^3, s = -n+1, -n+3, ..., n-1 */
} dvm_quad_kind;

/* Velocity grid: the tensor product of one 1D rule on each axis; n must be even (no zero node). */
typedef struct {
  int kind;    /* dvm_quad_kind */
  int n;       /* nodes per axis, 2..64, even */
  double vmax; /* half-width for DVM_QUAD_NEWTON_COTES; ignored otherwise */
} dvm_quad;

typedef enum {
  DVM_FP64 = 0,      /* distribution stored and swept in FP64 */
  DVM_FP32_ACC64 = 1 /* distribution stored and swept in FP32; moments, wall fluxes, residual and Q in FP64 */
} dvm_precision;

/* How the grid is held in device memory.  Both sweep kernels run their wavefront along the stored
 * x2 axis and spread the stored x1 axis over threads (column sweep: one thread per stored column,
 * at most 512; row sweep: rows in flight across the stored x1, at most 256 cells), so a wide, short
 * grid (e.g. the Couette channel of Sec. II, aspect 5) runs faster, and up to 65536 cells long,
 * when stored transposed.  Every argument and result of this API stays in the caller's layout
 * ([ny][nx], x1 along the flow) whatever the storage. */
typedef enum {
  DVM_STORAGE_AUTO = 0,       /* transposed when nx > ny */
  DVM_STORAGE_AS_GIVEN = 1,
  DVM_STORAGE_TRANSPOSED = 2
} dvm_storage;

typedef struct {
  int nx, ny;                 /* cells along x1 (flow) and x2; 2..65536 each, nx ny <= 16,776,960 */
  int periodic_x, periodic_y; /* 1 = periodic axis; a non-periodic axis is closed by diffuse walls */
  double ly;                  /* domain height H along x2 (cells are square, size ly/ny); > 0 */
  double kn;                  /* Knudsen number (> 0, +INFINITY allowed for delta = 0), or <= 0 ... */
  double delta;               /* ... to give delta >= 0 directly instead; exactly one of the two is set */
  dvm_quad quad;
  double accommodation;       /* alpha in [0, 1] of Eq. (diffuse2): the wall value of a reflected velocity
                                 is alpha rho_w + (1 - alpha) h(mirror v) at the face's gas cell (from the
                                 previous iterate).  1 = fully diffuse (the paper's case).  alpha < 1 runs
                                 on the column sweep only; its adjoint reflects the transposed wall reads
                                 specularly with weight 1 - alpha. */
  int precision;              /* dvm_precision */
  double force;               /* body-force source coefficient F along x1 (1 for the paper's Poiseuille flow) */
  int store_distribution;     /* 1 = also keep h in device memory (needed by dvm_distribution) */
  int sweep_warps;            /* row sweep only: upper bound on rows in flight (warps) per sweep block,
                                 1..16; 0 = 16.  The chunk width is the smallest of 1, 2, 4, 8, 16
                                 cells with ceil(nx / width) rows within the bound. */
  double top_wall_u1;         /* speed U along x1 of the plate beyond the last row (x2 = H; needs a
                                 non-periodic x2 axis): Couette flow, Sec. II, Eq. (diffuse1) with
                                 U0/v_m = U: its reflected molecules carry the drift 2 U v1.  0 = at rest
                                 (every other wall is at rest).  A moving plate runs on the column sweep
                                 only; its adjoint is that of a plate at rest (a constant source). */
  int storage;                /* dvm_storage; the width limits of the sweeps (nx <= 256 rows, 512
                                 columns) apply to the stored x1 axis */
  double dx1;                 /* x1 spacing; 0 = square cells (ly / ny).  Cells are dx1 x (ly / ny)
                                 rectangles otherwise.  Q and k_a keep their definitions (Sec. III). */
  const double *row_heights;  /* host double [ny], read by dvm_create only, or NULL: the heights of the
                                 rows along x2 (Sec. II.A: the paper resolves the rough band of its
                                 Couette channel with 60 rows and the rest with 100), all > 0; ly is then
                                 their sum and dx1 must be > 0.  Each upwind difference along x2 becomes
                                 the derivative at the cell centre of the polynomial through the same
                                 points (exact on linear fields, like the equal-row forms).  Needs the
                                 transposed storage (DVM_STORAGE_AS_GIVEN gives DVM_EINVAL) and runs on
                                 the column sweep only.  Its adjoint (the transposed stretched stencil)
                                 needs a non-periodic x2 axis (DVM_EINVAL otherwise). */
  int anderson_depth;         /* 0 = plain source iteration (Eq. iteration, the paper's).  1..8: Anderson
                                 mixing of that depth (Walker & Ni 2011, type II) of the projected state
                                 the sweeps start from -- moments, wall-face fluxes, periodic seam values,
                                 the mass shift -- three more kernels per sweep; same fixed point, far
                                 fewer sweeps where the plain iteration converges slowly (small Kn).
                                 Needs accommodation = 1 and FP64 storage (with FP32 the sweep's rounding,
                                 about 1e-7 relative, pollutes the mixing history and its residual cannot
                                 certify the distance to the fixed point).  Extra memory (2 depth + 3)
                                 doubles per state element (8 per cell plus the seams). */
  int fp32_refine;            /* FP32 storage only: the most passes of mixed-precision refinement that
                                 dvm_solve / dvm_batch_run add after the FP32 iteration has converged
                                 (0 = none; default 3).  A pass takes the residual of the FP32 fixed
                                 point with one FP64 sweep (an FP64 twin of the context, created on first
                                 use), solves the correction equation with the FP32 iteration itself (no
                                 force, no plate drift, the residual as its source) and adds the
                                 correction (solved to 1e-2 relative); passes stop once the error left,
                                 estimated as |d| / |x| (1e-2 + |d_1| / |x|) with d_1 the first pass's
                                 correction (flow velocity, L1 over gas cells), is below tol / 10 --
                                 usually after one pass.  This removes the FP32
                                 rounding that the iteration amplifies by 1 / (1 - r) where it converges
                                 slowly.  Fully diffuse walls only (accommodation = 1); with
                                 accommodation < 1 or a grid too wide for FP64 the FP32 result is returned
                                 unrefined. */
} dvm_params;

/* The transport sweep kernel (both compute the same update; see dvm_set_schedule; nx below is the
 * stored x1 extent, see dvm_storage):
 *   DVM_SWEEP_ROWS     a thread block per group of 32 velocities, lanes = velocities, warps = rows in
 *                      flight of a row wavefront, each advancing `shape` cells (the chunk width: 1, 2,
 *                      4, 8 or 16; 0 = the narrowest with at most 16 rows in flight); nx <= 256.
 *   DVM_SWEEP_COLUMNS  threads = grid columns walking an anti-diagonal wavefront, each with 8 (FP32)
 *                      or 4 (FP64) velocities; `threads_per_column` (1, 2 or 4) threads share a
 *                      column, so a block holds 8, 16 or 32 (FP32) velocities; nx * threads_per_column
 *                      <= 512.
 *   DVM_SWEEP_AUTO     rows (chunk width 0) where they apply (accommodation 1, no moving plate, equal
 *                      rows, nx <= 256) and the launch has velocity groups for at least half the SMs;
 *                      otherwise columns, with the most threads per column that fit. */
typedef enum { DVM_SWEEP_AUTO = 0, DVM_SWEEP_ROWS = 1, DVM_SWEEP_COLUMNS = 2 } dvm_sweep_kind;

/* Fill defaults: periodic_x = 1, periodic_y = 0, ly = 1, kn = 0.1, delta = -1, Gauss-Hermite 12,
 * accommodation 1, FP64, force 1, no stored distribution, automatic sweep shape, plates at rest,
 * automatic storage, square cells, equal rows, no mixing, up to 3 refinement passes for FP32. */
dvm_status dvm_params_init(dvm_params *params);

/* Build a solver for one geometry: the Cartesian staircase approximation of the channel walls or the
 * porous solids (Sec. II.A: rough surfaces are approximated by a staircase of grid cells; Sec. III:
 * the porous media on the same kind of grid), with the collision rate delta = sqrt(pi) / (2 Kn) of
 * Eq. (BGK) and the velocity grid of params->quad.
 *   mask      host, uint8 [ny][nx]; nonzero = solid cell.  At least one gas cell.
 *   params    host; copied.
 *   stream    a cudaStream_t on the current device, or NULL.
 *   out       receives the context; unchanged on failure.
 * Allocates the device state (about 4 * ncell * 64 bytes of tables plus seams, and with
 * store_distribution the full h: ncell * n^2 * (4 or 8) bytes) and sets the state to h = 0. */
dvm_status dvm_create(const uint8_t *mask, const dvm_params *params, void *stream, dvm_ctx **out);

/* Per-cell collision rate delta_c (host, double [ny][nx], >= 0; solid entries ignored), or NULL to
 * return to the uniform value of the parameters: the coefficient delta in front of the collision
 * term of Eq. (BGK), sqrt(pi) / (2 Kn) for a uniform gas (Sec. II.A), here allowed to vary by cell as
 * a wall-distance-dependent relaxation time would make it.  Resets the state to h = 0.  This is the
 * field the adjoint differentiates. */
dvm_status dvm_set_delta_field(dvm_ctx *ctx, const double *delta_c);

/* Restart from h = 0 (the state a new context has). */
dvm_status dvm_reset(dvm_ctx *ctx);

/* Source iteration (Eq. iteration) from the current state until the stopping test passes or
 * max_iter sweeps have run.  After sweep n the test uses eps_n = sum|u1^n - u1^(n-1)| / sum|u1^n|
 * over gas cells and r = (eps_n / eps_(n-4))^(1/4) clipped to [0, 0.9999]; it passes when n >= 5
 * and eps_n / (1 - r) < tol (an estimate of the relative distance to the fixed point; the paper
 * stops on eps_n < 1e-5, Sec. II.A).  With FP32 storage eps_n stalls at the rounding noise floor,
 * where r says nothing, so the test also passes when eps_n < tol and no sweep of the last 16 gave a
 * smaller eps; tol should then stay above about 1e-6.  With FP32 storage and fp32_refine > 0 the
 * converged FP32 state is then refined (see dvm_params.fp32_refine).  iters (may be NULL) receives the
 * FP32 or FP64 sweeps run by this call (refinement: the FP32 sweeps of every phase; the one FP64
 * residual sweep per pass is not counted), est (may be NULL) the last estimate (refinement: the
 * estimated relative error left after the last pass).  Returns DVM_ENOCONV if max_iter is reached. */
dvm_status dvm_solve(dvm_ctx *ctx, double tol, int max_iter, int *iters, double *est);

/* Run exactly n sweeps with no stopping test (timing and warm-up).  Synchronises the stream. */
dvm_status dvm_iterate(dvm_ctx *ctx, int n);

/* Mass flow rate Q = int v1 f dv dx1 dx2 / Lx = sum_gas u1 dA / Lx (Sec. III, Eq. Q) and apparent
 * permeability k_a = sqrt(4/pi) Q Kn (Sec. III, Eq. k_a; NaN when delta is a field or 0).
 * k_a may be NULL.  DVM_ESTATE before the first sweep. */
dvm_status dvm_flowrate(const dvm_ctx *ctx, double *Q, double *k_a);

/* Macroscopic fields of the current state (Sec. II.A): host double [ny][nx] each, NaN in solid
 * cells; any pointer may be NULL.  tau is the temperature perturbation int |v|^2 h f_eq - rho. */
dvm_status dvm_fields(const dvm_ctx *ctx, double *rho, double *u1, double *u2, double *tau);

/* Diagnostics of the current state: sweeps run since the last reset, last eps and estimate, the
 * accumulated mass shift c of the mean-density projection, the stored status of the last solve, and
 * whether the grid is stored transposed (dvm_storage). */
typedef struct {
  int iterations;
  double eps, est, mass_shift, Q;
  int status;
  int transposed;
} dvm_info;
dvm_status dvm_get_info(const dvm_ctx *ctx, dvm_info *info);

/* Gradient of the flow rate with respect to the per-cell collision rate, dQ/d delta_c, at the current
 * (converged) forward state, by the adjoint of the projected source iteration: transposed sweeps
 * (velocities visited in the reverse order, pulling from their forward-downstream cells) until the
 * stopping test of dvm_solve, applied to the relative change of sum_k v1_k z_k, passes.  This is the
 * field a wall-distance-dependent relaxation time would change (the paper's MRT-LBM comparison
 * alters exactly this coefficient).
 *   dQ_ddelta   host double [ny][nx] (output; 0 in solid cells).
 *   q_identity  host, may be NULL: F sum z v1, equal to Q at convergence (a consistency check).
 *   iters       host, may be NULL: adjoint sweeps run.
 * Needs store_distribution = 1 and at least one forward sweep (DVM_ESTATE otherwise).  Every wall
 * accommodation, moving plate, cell shape and row-height set is covered, except unequal rows with a
 * periodic x2 axis (DVM_EINVAL).  Allocates the adjoint state (about as much as the forward state plus
 * one more distribution) on first use. */
dvm_status dvm_adjoint(dvm_ctx *ctx, double tol, int max_iter, double *dQ_ddelta, double *q_identity, int *iters);

/* Choose the sweep kernel of the context's own solves and adjoint (dvm_sweep_kind) and its shape
 * (threads_per_column for DVM_SWEEP_COLUMNS, the chunk width for DVM_SWEEP_ROWS; 0 = automatic).
 * DVM_EINVAL if the grid does not fit the choice.
 * Results agree to rounding; speed differs with the grid width and the number of velocity groups.
 * Default: DVM_SWEEP_AUTO.  Batches created later start from the first member's choice. */
dvm_status dvm_set_schedule(dvm_ctx *ctx, int kind, int shape);
/* The resolved choice (kind is never DVM_SWEEP_AUTO; for rows the second value is the chunk width). */
dvm_status dvm_get_schedule(const dvm_ctx *ctx, int *kind, int *shape);

/* Distribution h of selected velocities (needs store_distribution = 1).  ks: host int [nk] with
 * k = a * n + b for v = (x_a, x_b) on the 1D nodes in ascending order.  out: host double
 * [nk][ny][nx]; solid cells 0. */
dvm_status dvm_distribution(const dvm_ctx *ctx, const int *ks, int nk, double *out);

/* The 1D nodes and weights the context uses (host double [n] each; weights approximate
 * int g(x) exp(-x^2)/sqrt(pi) dx). */
dvm_status dvm_quadrature(const dvm_ctx *ctx, double *nodes, double *weights);

/* The 1D nodes (ascending) and weights of a velocity-grid description, without a context or a GPU
 * (host double [q->n] each).  Gauss-Hermite uses the Golub-Welsch eigenvalue method. */
dvm_status dvm_velocity_grid(const dvm_quad *q, double *nodes, double *weights);

/* Batched solves: several contexts (independent geometries, Kn and velocity grids, one precision and
 * one store_distribution setting, one device) advanced by one launch of each kernel per sweep, on the
 * stream of the first context.  A batch records the contexts' configuration when it is created:
 * re-create it after dvm_set_delta_field on a member.  Destroying a member first releases the batch's
 * device resources (its launches run on a member's stream); the batch then answers DVM_ESTATE to every
 * call and only dvm_batch_destroy remains to be called. */
typedef struct dvm_batch dvm_batch;
dvm_status dvm_batch_create(dvm_ctx *const *ctxs, int n, dvm_batch **out);
/* Source iteration of every member until each passes the stopping test of dvm_solve or has run
 * max_iter sweeps in this call; converged members stop (their blocks return at once).  per (host,
 * [n], may be NULL) receives each member's status; returns DVM_OK when every member converged,
 * else the first failing status. */
dvm_status dvm_batch_run(dvm_batch *batch, double tol, int max_iter, dvm_status *per);
/* Exactly n sweeps of every member, no stopping test.  Synchronises the stream. */
dvm_status dvm_batch_iterate(dvm_batch *batch, int n);
/* Exactly n sweeps of every member, enqueued on the batch stream without waiting (one arming kernel,
 * then the sweep graphs); nothing is read back.  Call dvm_batch_check (or synchronise the stream)
 * before reading results.  Errors of the sweeps themselves surface in dvm_batch_check. */
dvm_status dvm_batch_enqueue(dvm_batch *batch, int n);
/* Wait for the batch stream and report the first failing member status (DVM_ENOCONV is not a failure
 * here: an enqueued run has no stopping test). */
dvm_status dvm_batch_check(dvm_batch *batch);
/* Device time of the last single sweep run by dvm_batch_iterate(batch, 1) or dvm_batch_enqueue(batch,
 * 1): the sweep kernel and the two finalize kernels, in milliseconds (CUDA events recorded around them
 * on the batch stream); read it after the stream has reached them. */
dvm_status dvm_batch_timing(const dvm_batch *batch, float *sweep_ms, float *finalize_ms);
/* Re-plan the batch's sweep launch for another kernel (see dvm_set_schedule); state is kept. */
dvm_status dvm_batch_set_schedule(dvm_batch *batch, int kind, int shape);
dvm_status dvm_batch_get_schedule(const dvm_batch *batch, int *kind, int *shape);
/* Autotuner: time every sweep kernel that fits the batch's grids (rows at three chunk widths; columns
 * with 1, 2, 4 threads per column) over `sweeps` single sweeps each (CUDA events, median), keep the
 * fastest and return it
 * (any output may be NULL; sweep_ms is its median sweep time).  The trial sweeps are ordinary source
 * iterations: they advance every member's state. */
dvm_status dvm_batch_autotune(dvm_batch *batch, int sweeps, int *kind, int *shape, float *sweep_ms);
/* Kernel launches issued per sweep of the batch (sweep + finalize kernels; with the persistent launch,
 * the arming and scheduler kernels of one launch). */
int dvm_batch_kernels_per_sweep(const dvm_batch *batch);
/* The persistent batched launch (on = 1) or one launch of each kernel per sweep (on = 0, the default).
 * Persistent: one kernel runs up to 64 source iterations of every member not yet done, its blocks
 * (as many as the SMs hold) taking work items -- a member's sweep tiles (velocity groups of the row
 * wavefront), then its finalize chunks (mass shift; moments, records, residual and stopping test) --
 * from a device-side scheduler: members advance independently, a converged member drops out at once
 * and one member's finalize overlaps the others' sweeps; the launch (with its arming kernel) is one
 * CUDA graph.  Needs the row sweep (dvm_batch_set_schedule rows), fully diffuse fixed walls, equal rows
 * and the plain iteration (DVM_EINVAL otherwise).  FP32 batches sweep paired velocity groups under the
 * batch's dvm_pairing policy, as the per-kernel launches do.  Same fixed point and stopping test; sums
 * are accumulated in another order (results agree to rounding).  Every wait of the scheduler is bounded:
 * an idle block that finds no work for about a second gives up and the batch reports DVM_ETIMEOUT.
 * dvm_batch_timing then reports the whole launch as the sweep time and 0 for the finalize.  The
 * autotuner returns a batch to per-kernel launches.  The paper has no counterpart (Sec. II.A iterates
 * one geometry at a time). */
dvm_status dvm_batch_set_persistent(dvm_batch *batch, int on);
/* on: 1 when the batch uses the persistent launch; blocks: the blocks of that launch (or 0). */
dvm_status dvm_batch_get_persistent(const dvm_batch *batch, int *on, int *blocks);

/* Paired velocity groups in the FP32 row sweep (an implementation choice, same update as Eq.
 * (iteration)): a warp sweeps two groups of 32 velocities of one quadrant, each lane holding one velocity
 * of each, so the cell records, the waits and the loop control serve 64 velocities and the update runs
 * as packed FP32x2 arithmetic.  Needs FP32 storage, a uniform collision rate, fully diffuse fixed walls,
 * equal rows and a shared-memory layout that fits (up to 256 cells wide at 16 cells per chunk, one pair
 * per block there), with per-kernel or persistent launches; members outside these keep one group per
 * warp.  Pairing halves the blocks of a
 * launch, so DVM_PAIRING_AUTO (the default) pairs only when the launch has at least three waves of
 * single-group blocks, and a solve under AUTO re-plans the launch without pairs once the members still
 * iterating no longer do (the next solve plans them again); DVM_PAIRING_ON pairs wherever eligible,
 * DVM_PAIRING_OFF never.  The batch is re-planned (its graphs rebuilt; the members' state is
 * untouched).  DVM_EINVAL for another mode. */
enum dvm_pairing { DVM_PAIRING_AUTO = 0, DVM_PAIRING_ON = 1, DVM_PAIRING_OFF = 2 };
dvm_status dvm_batch_set_pairing(dvm_batch *batch, int mode);
/* mode: the batch's dvm_pairing policy; paired_blocks: sweep blocks of the launch as currently planned
 * that sweep paired groups (0 when none, e.g. after a solve that dropped them for its tail). */
dvm_status dvm_batch_get_pairing(const dvm_batch *batch, int *mode, int *paired_blocks);
void dvm_batch_destroy(dvm_batch *batch);

/* One-shot batch: create, run, destroy. */
dvm_status dvm_batch_solve(dvm_ctx *const *ctxs, int n, double tol, int max_iter, dvm_status *per);

/* Moments and flow rate of a distribution held by the caller (the plain, unfused form of the moment
 * reduction: Sec. II.A moments, Sec. III Eq. Q).
 *   q         host; the velocity grid of h (n nodes per axis, n even, 2 <= n <= 64).
 *   h         device, double [n*n][ncell]: velocity k = a*n + b (v = (x_a, x_b)) is row k.
 *   mask      device, uint8 [ncell], nonzero = solid (excluded from Q, moments 0), or NULL.
 *   ncell     number of cells (>= 1).
 *   dA_over_L cell area / domain length along x1, the weight of Q = sum_gas u1 dA / L.
 *   mom       device, double [ncell][4]: rho, u1, u2, tau per cell (output).
 *   Q         device, double [1] (output).
 *   stream    cudaStream_t or NULL; the call synchronises it.
 * Allocates and frees a small scratch buffer for the block partial sums of Q on every call. */
dvm_status dvm_moments(const dvm_quad *q, const double *h, const uint8_t *mask, int ncell, double dA_over_L,
                       double *mom, double *Q, void *stream);

/* dvm_moments without any device allocation, for callers that cannot allocate during a call:
 * cudaMalloc and cudaFree synchronise the whole device and can fail under memory pressure, so a
 * caller inside a latency-critical loop, a caller whose device memory is all reserved by its own
 * allocator at start-up, or a caller that must not touch the allocator while other streams run cannot
 * use dvm_moments.  The paper has no counterpart: this is a deployment variant of the reduction above.
 * Arguments and results are those of dvm_moments.  Differences:
 *   - scratch is a fixed device array of about 8.3 KB inside the library, present on every device
 *     that loads it until the process exits;
 *   - ncell may be at most 16,777,216, a maximum this call sets for itself (the scratch would serve
 *     any count): DVM_EINVAL beyond, message in dvm_last_error(NULL);
 *   - the call is asynchronous on `stream` (results are ready when the stream reaches them);
 *   - every call shares the array: calls that overlap on one device (for example on two streams)
 *     race and must be serialised by the caller;
 *   - the first call in a CUDA context looks up the array's address with that context current; make
 *     that first call before any stream capture.  After cudaDeviceReset (or a released and re-created
 *     primary context) the next call looks it up again.
 * Errors are reported through dvm_last_error(NULL), including the reason an argument was rejected. */
dvm_status dvm_moments_noalloc(const dvm_quad *q, const double *h, const uint8_t *mask, int ncell,
                               double dA_over_L, double *mom, double *Q, void *stream);

/* Description of the last error on ctx (or of the last dvm_create failure when ctx is NULL). */
const char *dvm_last_error(const dvm_ctx *ctx);

/* Static name of a status code. */
const char *dvm_status_string(dvm_status status);

/* Failure detection without a fault.  Every wait inside the sweeps is bounded: a row-sweep warp
 * waiting for its neighbour's progress word, or a column-sweep block waiting for a TMA stage, gives
 * up after a fixed spin count, records DVM_ETIMEOUT in the instance state (dvm_solve then returns it)
 * and returns, leaving the context usable.  This entry point runs one of those wait primitives in a
 * one-block kernel on a flag that nothing raises: primitive 0 = the row sweep's progress-word wait,
 * 1 = the column sweep's mbarrier wait, 2 = the persistent launch's scheduler poll on an active
 * instance whose work never appears (its own limit, 2^22 polls, about a second; spin_limit is not
 * used).  spin_limit > 0 replaces the sweeps' limit (2^22 spins) of primitives 0 and 1 to keep the
 * call short.  Returns DVM_ETIMEOUT (the wait gave up, the expected outcome), DVM_OK (the
 * flag was seen: impossible unless the primitive is broken), DVM_EINVAL or DVM_ECUDA; seconds (may be
 * NULL) receives the call's wall time.  The paper has no counterpart. */
dvm_status dvm_selftest_wait(int primitive, int spin_limit, double *seconds);

/* Measured arithmetic ceiling of the current GPU, for the roofline of the sweeps (the fused sweep keeps
 * h on chip, so its bound is the SM's FMA rate): kind 0 = FP32 FMA, 1 = packed FP32x2 FMA, 2 = FP64
 * FMA.  Every thread of a grid of 8 blocks of 256 threads per SM runs 8 independent FMA chains (no
 * memory traffic) for about `seconds` (0 < seconds <= 10); tflops (required) receives 2 x FMAs / the
 * kernel's CUDA-event time in TFLOP/s, l2_bytes and sms (may be NULL) the device's L2 size and SM
 * count.  Runs on the current device's legacy default stream and synchronises it.  Returns DVM_OK,
 * DVM_EINVAL or DVM_ECUDA.  The paper has no counterpart. */
dvm_status dvm_probe_peaks(int kind, double seconds, double *tflops, int *l2_bytes, int *sms);

/* Release the context and its device memory.  NULL is ignored. */
void dvm_destroy(dvm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DVM_H */
