/*
 * protox.h - C ABI of the B300 (sm_103a) fused periodic 2D Poisson relaxation
 * library, after ProtoX (Mankad, Rao, Colella, Van Straalen, Franchetti,
 * "ProtoX: A First Look").
 *
 * The library solves the model problem of Sec. IV, Delta phi = rho on a periodic
 * rectangular grid of cell-centred cells with spacing h, with the 5-point
 * Laplacian L (taps [0,1,0; 1,-4,1; 0,1,0], scaled by 1/h^2) and weighted
 * point-Jacobi relaxation (Eq. "jacobi" with a weight omega):
 *
 *     phi' = phi + (omega h^2 / 4) (L phi - rho)
 *
 * The paper's lambda = h^2/(4D) is omega = 1/D = 1/2 in D = 2 dimensions.
 * One sweep fuses the periodic ghost fill, the Laplacian, the Jacobi update and
 * the max-norm of the residual rho - L phi of the sweep's INPUT state into one
 * pass over memory (the Sigma-OL loop merging of Sec. IV).
 *
 * Conventions shared by every call
 * ---------------------------------
 *  - Fields are row-major, x fastest: cell (i, j) is at element
 *    off + j*ld + i with off = 0 (ghost = 0) or ld + 1 (ghost = 1).
 *    Every field pointer of one call uses the layout of its px_grid.
 *  - Field pointers are DEVICE pointers owned by the caller (e.g. the
 *    data_ptr() of a CUDA tensor). The library never frees them.
 *  - The px_ctx owns its scratch memory (ping-pong buffer, reduction slots),
 *    allocated on first need with cudaMalloc and grown on demand; a call
 *    that grows it synchronises the device.
 *  - Streams are passed as void* (a cudaStream_t); NULL is the legacy
 *    default stream. Work is enqueued asynchronously unless a call says
 *    it synchronises.
 *  - Every call returns a px_status and never aborts or throws across the
 *    ABI. Arguments are validated before any launch; on error nothing is
 *    launched and px_last_error() holds a one-line message. Asynchronous
 *    device errors surface as PX_ECUDA from the next synchronising call.
 *  - A ctx is bound to the device given at creation. It is not thread-safe:
 *    one host thread at a time per ctx. Work enqueued through one ctx must
 *    not overlap on the GPU (several streams at once): calls share its
 *    scratch field, reduction slots and the small array through which the
 *    warps of one relaxation launch balance their work. Use one ctx per
 *    concurrently running stream.
 */
#ifndef PROTOX_H
#define PROTOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PX_OK = 0,
  PX_EINVAL = 1,        /* bad argument (size, pointer, alias, layout, value) */
  PX_ECUDA = 2,         /* a CUDA runtime call failed */
  PX_ENOMEM = 3,        /* device scratch allocation failed */
  PX_ENOCONV = 4,       /* solve hit its sweep limit before the tolerance */
  PX_ETIMEOUT = 5,      /* solve or device wait ran past its time limit */
  PX_EMEAN = 6,         /* rho has a nonzero mean: the periodic problem has no solution */
  PX_ENAN = 7,          /* a residual became NaN or Inf */
  PX_EUNSUPPORTED = 8   /* valid request this build does not implement */
} px_status;

typedef enum { PX_F64 = 0, PX_F32 = 1 } px_dtype;

/* Layout of one periodic field (Sec. III "Proto": Box / BoxData on a periodic
 * rectangular grid; Sec. IV: an n x n box stored as m x m, m = n + 2 with
 * ghosts). */
typedef struct {
  int32_t nx, ny;  /* interior cells along x (fastest) and y; >= 0 (0 = empty, no-op) */
  int64_t ld;      /* elements between row starts; >= nx + 2*ghost */
  int32_t ghost;   /* 0: plain periodic array (ny rows).
                      1: one ghost layer around the interior, (ny + 2) rows;
                         input ghosts are ignored (the kernels wrap periodically
                         while loading) and output ghosts are written with the
                         periodic images of the interior. */
  int32_t dtype;   /* px_dtype of every field of the call */
  double h;        /* mesh spacing, finite and > 0 */
} px_grid;

/* Layout of a 3D periodic field (px_relax3_n): nz planes of ny rows of nx
 * cells, x fastest, no ghost cells. */
typedef struct {
  int32_t nx, ny, nz;  /* cells along x, y, z; >= 0 (a zero extent: empty, no-op) */
  int64_t ld;          /* elements between row starts; >= nx */
  int64_t lp;          /* elements between plane starts; >= (ny - 1) * ld + nx */
  int32_t dtype;       /* px_dtype of every field of the call */
  double h;            /* mesh spacing, finite and > 0 */
} px_grid3;

typedef struct px_ctx px_ctx;

/* Create a context on CUDA device `device`. *out is NULL on failure. */
px_status px_create(px_ctx** out, int device);

/* Synchronise the context's device, free its scratch and the context.
 * NULL is accepted. */
px_status px_destroy(px_ctx* ctx);

/* Message of the last failed call on ctx ("" if none). Valid until the next
 * call on ctx. ctx may be NULL (then the message of the calling thread's last
 * failed px_create or px_relax_n_static). */
const char* px_last_error(const px_ctx* ctx);

/* Static name of a status code. */
const char* px_status_string(px_status s);

/* Checked build (the library compiled with -DPX_CHECKED into
 * libprotox_checked.so; the paper has no counterpart): the relaxation and
 * Euler kernels check every global index they compute against the field's
 * extent before the access; a violation is counted in a device word, the
 * first one recorded as (site << 48 | index), and the access is skipped.
 * px_is_checked_build() is 1 in that build, 0 otherwise.
 * px_checked_faults synchronises ctx's device, returns the count and the
 * first violation (first may be NULL) and clears both; in the normal build it
 * returns PX_EUNSUPPORTED with *count = 0. */
int px_is_checked_build(void);
px_status px_checked_faults(px_ctx* ctx, uint64_t* count, uint64_t* first);

/* Per-context kernel selection (the paper has no counterpart: these pick
 * among kernels that compute the same sweeps, for A/B timing and for tests
 * that compare the kernel families bitwise). Defaults (0) are the fastest
 * measured on B300.
 *  PX_OPT_FP32_FAMILY           FP32 relaxation kernel for depth >= 2:
 *                               0 automatic by size, 1 one-row shared-memory
 *                               wavefront, 2 two-row shared-memory wavefront,
 *                               3 register wavefront at every size, 4 the
 *                               register wavefront with packed-pair (f32x2)
 *                               arithmetic at every size.
 *  PX_OPT_RB_SWEEPS_PER_LAUNCH  red-black sweeps per launch of the FP32
 *                               register wavefront: 0 automatic (3), 1..4.
 *  PX_OPT_BATCH_LAUNCHES        kernels in the graph of a batch plan made
 *                               through ctx: 0 automatic (one persistent
 *                               launch, or for batches mixing FP64 and FP32
 *                               two side by side when that predicts less),
 *                               1 always one persistent launch.
 *  PX_OPT_RB_FP64_PASSES        launches per FP64 red-black sweep on 16-byte
 *                               vector layouts (px_rbsor_n, multigrid
 *                               smoothers): 0 automatic (1), 1 one fused
 *                               launch, 2 a red pass and a black pass.
 *  PX_OPT_MG_PROLONG            multigrid interpolation + correction on levels
 *                               that the FP32 register wavefront smooths:
 *                               0 automatic (inside the first post-smoothing
 *                               launch), 1 a pass of its own.
 * px_set_option returns PX_EINVAL for an unknown option or a value out of
 * range; it affects calls made through ctx afterwards. */
enum {
  PX_OPT_FP32_FAMILY = 1,
  PX_OPT_RB_SWEEPS_PER_LAUNCH = 2,
  PX_OPT_BATCH_LAUNCHES = 3,
  PX_OPT_RB_FP64_PASSES = 4,
  PX_OPT_MG_PROLONG = 5
};
px_status px_set_option(px_ctx* ctx, int option, int value);
px_status px_get_option(const px_ctx* ctx, int option, int* value);

/* Laplacian (Sec. IV, OL rule Laplace): lphi = L phi = s / h^2, s the
 * unscaled 5-point tap sum with periodic wrap. Computed in the grid's dtype.
 * phi and lphi must not overlap. Asynchronous. */
px_status px_apply_stencil(px_ctx* ctx, const px_grid* g, const void* phi,
                           void* lphi, void* stream);

/* nsweeps fused sweeps (Sec. IV: Laplace, Jacobi and max-norm merged into
 * one loop; Eq. "jacobi" with weight omega) from phi_in into phi_out.
 *
 *  phi_in, phi_out  fields of layout g; phi_in == phi_out is allowed (the
 *                   context ping-pongs through scratch); any other overlap
 *                   is PX_EINVAL. phi_in is not modified unless it is phi_out.
 *  rho              right-hand side, layout g, must not overlap phi_out.
 *  omega            Jacobi weight, finite (2/3 damps the upper half of the
 *                   spectrum by at least 1/3 per sweep; 1/2 is the paper's).
 *  nsweeps          >= 0; 0 copies phi_in to phi_out.
 *  tblock           sweeps fused per launch (temporal blocking), 0 = choose
 *                   automatically, else 1..8. A depth the layout cannot use
 *                   (ghosted, unaligned or x-extent not a multiple of the
 *                   vector width) silently runs at depth 1; results do not
 *                   depend on it beyond rounding.
 *  resid_dev        NULL, or DEVICE array of ceil(nsweeps / report_every)
 *                   doubles: resid_dev[k] = ||rho - L phi^(k*report_every)||_inf,
 *                   the max-norm residual of state k*report_every (state 0 is
 *                   phi_in), computed inside the sweep that reads that state
 *                   (Sec. IV step 3). The call zero-fills the array first.
 *                   FP32 fields report the FP32 residual.
 *  report_every     >= 0; 0 disables reports.
 * Asynchronous. */
px_status px_relax_n(px_ctx* ctx, const px_grid* g, const void* phi_in,
                     void* phi_out, const void* rho, double omega, int nsweeps,
                     int tblock, double* resid_dev, int report_every,
                     void* stream);

/* px_relax_n for callers that cannot allocate device memory. The paper has
 * no counterpart: this is a deployment variant of the same fused sweeps.
 *
 * Some callers may not call cudaMalloc at all: a latency-bound loop that
 * must never block on the allocator, an application whose own memory pool
 * owns the device, or a plug-in that may not create library contexts
 * (px_create allocates). This call needs no
 * px_ctx and allocates nothing. The caller still passes phi_in, phi_out, rho
 * and resid_dev, with exactly the meaning, layout and results of px_relax_n
 * (same kernels, same launch plan). The one working buffer of a multi-launch
 * relax, the ping-pong field, is a fixed 16 MiB device array inside the
 * library: every GPU that loads the library holds it until the process
 * exits.
 *
 *  - Limit: the field's span, ((rows - 1) * ld + width) * element size, must
 *    be at most 16 MiB (e.g. 2048 x 2048 FP32, 1448 x 1448 FP64); larger
 *    fields are rejected with PX_EINVAL before anything is launched.
 *  - Runs on the CURRENT CUDA device. The first call on each device (and
 *    again the first call after that device's primary context was
 *    recreated, e.g. after cudaDeviceReset) looks up the array's device
 *    address (cudaGetSymbolAddress) and caches it for that context; make
 *    that first call before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents
 *    (nothing in it needs to start at zero; resid_dev is zero-filled by the
 *    call as in px_relax_n). Calls whose work overlaps on the GPU (other
 *    streams, other host threads) race on it: serialise them.
 *  - Errors return a px_status; the message is px_last_error(NULL) on the
 *    calling thread. */
px_status px_relax_n_static(const px_grid* g, const void* phi_in, void* phi_out,
                            const void* rho, double omega, int nsweeps, int tblock,
                            double* resid_dev, int report_every, void* stream);

/* nsweeps red-black SOR sweeps from phi_in into phi_out: the relaxation the
 * paper names as the smoother of Proto's multigrid (Sec. VI, future work), in
 * its standard definition. One sweep updates, in place, first every red cell
 * ((x + y) even) and then every black cell, each with the per-point update of
 * px_relax_n, phi <- phi + (omega h^2 / 4)(L phi - rho), L phi taken from the
 * current state (black neighbours old during the red half, red neighbours new
 * during the black half). omega = 1 is red-black Gauss-Seidel; 0 < omega < 2
 * converges on the mean-zero problem.
 *
 *  g                unghosted layout (PX_EUNSUPPORTED otherwise), nx and ny
 *                   even (the colouring must agree across the periodic wrap;
 *                   PX_EINVAL otherwise), FP64 or FP32.
 *  phi_in, phi_out, rho, omega, nsweeps, resid_dev, report_every, stream
 *                   as in px_relax_n; resid_dev[k] is the residual of the
 *                   INPUT state of sweep k * report_every, over all cells.
 * Launches: FP32 16-byte vector layouts run several sweeps per launch of a
 * register wavefront (PX_OPT_RB_SWEEPS_PER_LAUNCH); FP64 vector layouts one
 * fused launch per sweep, out of place (PX_OPT_RB_FP64_PASSES); other layouts
 * two launches per sweep (red pass out of place with the residual, black pass
 * in place). All give the same bits. The context's scratch field is used when
 * in place or for two launches or more. Asynchronous. */
px_status px_rbsor_n(px_ctx* ctx, const px_grid* g, const void* phi_in, void* phi_out,
                     const void* rho, double omega, int nsweeps, double* resid_dev,
                     int report_every, void* stream);

/* ncycles geometric multigrid V-cycles on phi, in place: the multigrid with a
 * red-black SOR smoother that the paper builds on Proto's operators (Sec. VI,
 * future work), as the textbook cell-centred V-cycle. On level l (cells of
 * width 2^l h) one cycle is: nu1 red-black SOR sweeps (px_rbsor_n's sweep);
 * r = rho_l - L phi_l; rho_{l+1} = mean of each 2 x 2 block of r; a cycle on
 * level l+1 from e = 0; phi_l += bilinear interpolation of e between cell
 * centres (weights 9/16, 3/16, 3/16, 1/16, periodic); nu2 sweeps. The
 * coarsest level runs coarse_sweeps sweeps instead. Levels halve both extents
 * while both halves stay even (a 2^k x 2^k grid goes down to 2 x 2), up to
 * max_levels levels (0: no limit).
 *
 *  g              unghosted layout (PX_EUNSUPPORTED otherwise), nx and ny even
 *                 (PX_EINVAL otherwise), FP64 or FP32; level 0 keeps g's pitch,
 *                 coarser levels are contiguous.
 *  phi            device field, read and overwritten (the cycle's state).
 *  rho            device field, same layout; must not overlap phi. For the
 *                 periodic problem it should have zero mean (the constant
 *                 mode of phi is left free).
 *  ncycles        >= 0. nu1, nu2 >= 0 smoothing sweeps per level.
 *  omega          the smoother's relaxation factor (1: Gauss-Seidel).
 *  coarse_sweeps  sweeps on the coarsest level; 0 picks 1 for a 2 x 2 level
 *                 (solved exactly) and 2 n^2 otherwise (n its larger extent).
 *  max_levels     >= 0; 0 = as many as the extents allow.
 *  resid_dev      NULL, or ncycles + 1 device doubles: [k] = ||rho - L phi_k||
 *                 (max-norm) of the state after k cycles, evaluated in the
 *                 storage precision (FMA form): [k < ncycles] by the cycle's
 *                 first kernel, [ncycles] by a residual pass over the final
 *                 state (in FP64 when the grid has a single level).
 * On FP32 levels with 16-byte aligned rows the interpolation and correction
 * are done by the first post-smoothing launch as it loads its input (the same
 * operations, so the same bits; PX_OPT_MG_PROLONG = 1 keeps a pass of their
 * own). Working memory: the context's scratch field (phi's span) and one allocation
 * of three fields per coarser level (a field's size in all), kept by the
 * context; PX_ENOMEM when it cannot be had. Asynchronous. */
px_status px_mg_solve(px_ctx* ctx, const px_grid* g, void* phi, const void* rho, int ncycles,
                      int nu1, int nu2, double omega, int coarse_sweeps, int max_levels,
                      double* resid_dev, void* stream);

/* nsweeps fused sweeps of the 3D periodic Poisson problem, phi_in -> phi_out:
 * Eq. "jacobi" in D = 3 dimensions. Per cell, the 7-point Laplacian
 * L phi = (W + E + S + N + B + T - 6 C) / h^2 of the periodic neighbours, the
 * update phi' = phi + (omega h^2 / 6)(L phi - rho) (the paper's
 * lambda = h^2 / (4 D) = h^2 / 12 is omega = 1/2; 0 < omega <= 1 converges on
 * the mean-zero problem), and the residual max-norm of the input state, in one
 * pass per sweep.
 *
 *  g            px_grid3 layout, FP64 or FP32.
 *  phi_in, phi_out, rho, omega, nsweeps, resid_dev, report_every, stream
 *               as in px_relax_n (resid_dev[k] is the residual of the input
 *               state of sweep k * report_every); phi_in == phi_out runs in
 *               place through the context's scratch field.
 * 16-byte vectors when nx, ld and lp are multiples of 16 / element size and
 * the three pointers are 16-byte aligned; a scalar path otherwise.
 * Asynchronous. */
px_status px_relax3_n(px_ctx* ctx, const px_grid3* g, const void* phi_in, void* phi_out,
                      const void* rho, double omega, int nsweeps, double* resid_dev,
                      int report_every, void* stream);

/* The launch plan px_relax_n would use for these arguments, without running
 * it: *tblock_used = sweeps fused per launch (after auto choice and layout
 * fallback), *launches = relax kernel launches (excluding the zero-fill of
 * resid_dev and a staging copy). Either output may be NULL. Pure host call. */
px_status px_relax_plan(px_ctx* ctx, const px_grid* g, const void* phi_in,
                        const void* phi_out, const void* rho, int nsweeps,
                        int tblock, int* tblock_used, int* launches);

/* ----------------------------------------------------------------------------
 * Solve to a tolerance (Sec. IV: relax, then check the max-norm against the
 * convergence criterion, repeated). Two modes:
 *  PX_SOLVE_PLAIN   sweeps in the grid's dtype (FP64 or FP32 storage), an FP64
 *                   residual check every check_every sweeps.
 *  PX_SOLVE_REFINE  FP64 phi and rho; an FP64 outer loop of iterative
 *                   refinement around FP32-storage sweeps: r = rho - L phi in
 *                   FP64, scaled by an exact power of two and stored as FP32;
 *                   inner_sweeps FP32 sweeps solve L e = r from e = 0; then
 *                   phi += e in FP64. The residual, the correction and the
 *                   final norm are the only FP64 steps.
 * Convergence: ||rho - L phi||_inf <= rtol * ||rho||_inf, evaluated in FP64 on
 * the current state (px_residual_norm), one host synchronisation per check.
 */
typedef enum { PX_SOLVE_PLAIN = 0, PX_SOLVE_REFINE = 1 } px_solve_mode;

typedef struct {
  int32_t mode;          /* px_solve_mode */
  int32_t tblock;        /* sweeps per launch of the sweeps, 0 = automatic */
  double omega;          /* Jacobi weight, finite */
  double rtol;           /* relative max-norm target, >= 0 */
  int64_t max_sweeps;    /* sweep budget (inner sweeps count), >= 0 */
  int32_t check_every;   /* PLAIN: sweeps between checks, > 0 */
  int32_t inner_sweeps;  /* REFINE: FP32 sweeps per outer cycle, > 0 */
  int64_t timeout_ms;    /* host wall-clock limit checked at each check, 0 = none */
  int32_t check_mean;    /* nonzero: PX_EMEAN if |mean rho| > 1e-12 ||rho||_inf */
  int32_t reserved;      /* must be 0 */
} px_solve_opts;

typedef struct {
  int64_t sweeps;        /* sweeps performed (inner sweeps in REFINE) */
  int64_t cycles;        /* REFINE outer cycles (0 in PLAIN) */
  int64_t checks;        /* FP64 residual evaluations */
  double rel_resid;      /* ||rho - L phi||_inf / ||rho||_inf of the returned phi */
  double wall_ms;        /* host wall time of the call */
} px_solve_info;

/* Solve L phi = rho in place from the phi given (the initial guess). Returns
 * PX_OK when converged, PX_ENOCONV when max_sweeps ran out, PX_ETIMEOUT past
 * timeout_ms, PX_ENAN for a NaN/Inf residual, PX_EMEAN (check_mean), PX_EINVAL
 * for bad options (REFINE needs PX_F64). info may be NULL; it is filled on
 * every return after validation. Synchronises the stream at each check. */
px_status px_solve(px_ctx* ctx, const px_grid* g, void* phi, const void* rho,
                   const px_solve_opts* opts, px_solve_info* info, void* stream);

/* ----------------------------------------------------------------------------
 * Batched relaxation: many independent periodic instances of uneven sizes and
 * mixed dtypes, nsweeps fused sweeps each (the same sweep as px_relax_n), in
 * persistent kernel launches replayed from one CUDA graph (one graph launch
 * per run). Instances are independent problems, so the batch needs no
 * exchange between them.
 *
 * Execution per size class (dtype, nx, ny), chosen by an autotuner:
 *  WHOLE     one CTA keeps the instance in shared memory for all sweeps
 *            (fits when 2 * nx * ny * element size <= 200 KiB);
 *  BANDED    a cluster of 2, 4 or 8 CTAs shares the instance, one band of
 *            rows each, sweeping from global memory with a cluster barrier
 *            per sweep;
 *  BANDED_T  (FP32) BANDED with tb = 4 or 8 sweeps per cluster barrier in
 *            shared-memory tiles with a tb-cell halo.
 * The tuner times the modes (and the rows per warp task) with one copy per
 * cluster running at once and keeps the fastest rate per SM; the results are
 * cached as JSON keyed by GPU name. The schedule assigns instances
 * longest-first to the least loaded cluster / CTA. The graph holds ONE
 * persistent launch, or, for a batch mixing FP64 and FP32 instances when
 * that predicts less, two launched side by side (FP64 instances in one, FP32
 * in the other, one CTA of each per SM, at most 100 KiB of shared memory a
 * CTA); PX_OPT_BATCH_LAUNCHES = 1 on the context keeps one launch.
 *
 * px_batch_plan   grids[n]: layouts (unghosted; nx, ld multiples of 4 for FP32,
 *                 2 for FP64; PX_EUNSUPPORTED otherwise). nsweeps, omega,
 *                 report_every as in px_relax_n. tune_cache: JSON path or NULL.
 *                 tune: nonzero = measure classes missing from the cache
 *                 (synchronises the device; allocates temporary buffers).
 *                 Allocates the plan's device tables, BANDED scratch fields and
 *                 captures the graph. *out is NULL on failure.
 * px_batch_run    phis[i], rhos[i]: DEVICE fields of instance i (16-byte aligned,
 *                 phi and rho must not overlap); phi is relaxed in place.
 *                 resid_dev: NULL or DEVICE array of n * nrep doubles, instance
 *                 i's reports at i * nrep (nrep = ceil(nsweeps / report_every)),
 *                 zero-filled by the call. Waits for the plan's previous run,
 *                 then enqueues on `stream` and returns.
 * px_batch_describe  JSON text of the plan (classes, modes, rates, clusters,
 *                 launches, predicted time); valid until px_batch_destroy.
 * px_batch_destroy   synchronises the device and frees the plan.
 */
typedef struct px_batch px_batch;

px_status px_batch_plan(px_ctx* ctx, int n, const px_grid* grids, int nsweeps, double omega,
                        int report_every, const char* tune_cache, int tune, px_batch** out);
px_status px_batch_run(px_batch* plan, void* const* phis, const void* const* rhos,
                       double* resid_dev, void* stream);
const char* px_batch_describe(const px_batch* plan);
px_status px_batch_destroy(px_batch* plan);

/* ----------------------------------------------------------------------------
 * Learned initial guess (the paper has no network; this supplies the starting
 * state of the Sec. IV iteration). A 6-layer CNN of periodic 3x3 convolutions
 * (cross-correlation, circular padding), widths 1-32-32-32-32-32-1, exact (erf)
 * GELU after every layer but the last. BF16 weights and activations, FP32
 * accumulation; the 32 -> 32 layers run on the tensor cores. Trained by MSE
 * with Adam (beta 0.9 / 0.999, eps 1e-8) on FP32 master weights.
 *
 * Scaling: for an image rho with spacing h, s = max|rho h^2|, the network input
 * is x = rho h^2 / s and its target is t = phi 4 pi^2 h^2 / s (phi the mean-zero
 * solution; the factor makes the lowest mode of a unit-square field order one);
 * the guess is phi0 = s / (4 pi^2 h^2) (y - mean(y)). The map rho -> phi is
 * linear, so the scaling is exact.
 *
 * Images are B x H x W, row-major, x fastest; H a multiple of 4 and W a multiple
 * of 64 (PX_EUNSUPPORTED otherwise). All image pointers are DEVICE pointers.
 * Parameters (px_cnn_get/set_params) are the FP32 master weights in the order
 * W1, b1, ..., W6, b6 with W_l of shape (Cout, Cin, 3, 3); px_cnn_param_count()
 * floats. The network owns its weights, Adam state and activation workspace
 * (grown on demand; a call that grows it synchronises the device).
 */
typedef struct px_cnn px_cnn;

size_t px_cnn_param_count(void);
/* He-normal weights (std sqrt(2 / (9 Cin))), zero biases, from `seed`.
 * dilations: NULL (plain 3x3 layers) or 6 per-layer dilations d in 1..4096; a
 * layer of dilation d reads x[p + d (dy - 1, dx - 1)], so dilations 1, 3, 9,
 * 27, 81, 1 give a receptive field of 245 cells instead of 13. */
px_status px_cnn_create(px_ctx* ctx, uint64_t seed, const int32_t* dilations, px_cnn** out);
px_status px_cnn_destroy(px_cnn* net);
px_status px_cnn_get_params(px_cnn* net, float* host, size_t count);
px_status px_cnn_set_params(px_cnn* net, const float* host, size_t count);
/* Checkpoint state: parameters, Adam first and second moments (3 x
 * px_cnn_param_count() floats, px_cnn_state_count()) and the Adam step count.
 * Restoring a state and continuing training reproduces an uninterrupted run
 * bit for bit (every reduction of the training step has a fixed order). */
size_t px_cnn_state_count(void);
px_status px_cnn_get_state(px_cnn* net, float* host, size_t count, int64_t* step);
px_status px_cnn_set_state(px_cnn* net, const float* host, size_t count, int64_t step);
/* y (FP32, B x H x W) = network(x) for scaled inputs x (FP32). Asynchronous. */
px_status px_cnn_forward(px_cnn* net, const float* x, float* y, int B, int H, int W, void* stream);
/* Forward + backward of the MSE loss against t; gradients (FP32, parameter
 * order) to grads_host and the loss to loss_host when not NULL (synchronises). */
px_status px_cnn_grads(px_cnn* net, const float* x, const float* t, int B, int H, int W,
                       float* grads_host, double* loss_host, void* stream);
/* One Adam step of learning rate lr on the batch (x, t); loss_host as above. */
px_status px_cnn_train_step(px_cnn* net, const float* x, const float* t, int B, int H, int W,
                            float lr, double* loss_host, void* stream);
/* Training pair from FP64 images: x = rho h^2 / s and, if phi is not NULL,
 * t = phi 4 pi^2 h^2 / s; per-image s to scales_host when not NULL (synchronises). */
px_status px_cnn_prepare(px_cnn* net, const double* rho, const double* phi, float* x, float* t,
                         int B, int H, int W, double h, double* scales_host, void* stream);
/* Initial guess phi0 (FP64) for FP64 right-hand sides rho: scale, network,
 * unscale, subtract the mean. Asynchronous. */
px_status px_cnn_guess(px_cnn* net, const double* rho, double* phi0, int B, int H, int W,
                       double h, void* stream);
/* Hidden tensors of the last forward pass, for inspection and tests (the
 * paper has no counterpart): which = 0 the activation a_l = gelu(z_l), 1 the
 * pre-activation z_l (kept only by px_cnn_grads and px_cnn_train_step), of
 * hidden layer l = 1..5, as BF16 bit patterns in the library's chunk-planar
 * order (B, 4, H, W, 8), natural pixel order (a relabelled tensor is gathered
 * back through the network's gradient scratch): channel 8 k + c of pixel (y, x) of image b at
 * (((b * 4 + k) * H + y) * W + x) * 8 + c; B x H x W x 32 values of the last
 * call's shape (count may be smaller). Synchronises the stream. */
px_status px_cnn_get_hidden(px_cnn* net, int layer, int which, uint16_t* host, size_t count,
                            void* stream);
/* Polls per handshake wait (producer, MMA issuer, epilogue) of the
 * tensor-core kernels; 0 restores the default 2^24. A poll suspends the
 * waiting thread for at most 1 us (it resumes as soon as the awaited phase
 * completes), so a wait lasts at most polls x 1 us. A wait that runs out
 * makes its CTA stop, drain the MMAs it already issued (that wait keeps the
 * default limit), free its tensor memory and raise a device fault word; the
 * next call that reads the loss returns PX_ETIMEOUT and clears the word.
 * The network stays usable: later calls recompute everything they return.
 * (Failure detection; the paper has no counterpart.) */
px_status px_cnn_set_wait_limit(px_cnn* net, uint32_t polls);
/* How the tensor-core convolutions stage each tap's shifted input tile into
 * shared memory: mode 1 (the default) with one tensor-memory-accelerator box
 * for tiles that lie inside the image and per-pixel copies for tiles that
 * wrap around the periodic edge; mode 0 with per-pixel copies only. Both
 * stage the same bytes, so results are bitwise equal. PX_EINVAL for other
 * modes. (An implementation choice; the paper has no counterpart.) */
px_status px_cnn_set_staging(px_cnn* net, int mode);
/* How the dilated 32 -> 32 layers address their taps. on = 1 (the default):
 * where a layer's dilation d is invertible modulo H and W (d odd and the
 * sides powers of two, for instance), its input is stored relabelled (natural
 * pixel p at position p d^-1 modulo the sides), which makes the taps p +
 * (dy, dx) d unit offsets q + (dy, dx) over positions; the layer then stages
 * one (4 + 2)-row patch per column offset instead of nine tap tiles. Every
 * producer stores its output in the positions its consumer wants; the output
 * y, the loss, the gradients and px_cnn_get_hidden stay in natural order.
 * on = 0: natural order everywhere, nine offset tap tiles per output tile.
 * The two forms sum the same products in different orders (results agree to
 * FP32 rounding). PX_EINVAL for other values. (An implementation choice; the
 * paper has no counterpart.) */
px_status px_cnn_set_relabel(px_cnn* net, int on);

/* ----------------------------------------------------------------------------
 * 2D Euler equations of gas dynamics by the finite-volume method: the paper's
 * second workload (Sec. IV, the Euler result of Fig. "Euler"; Sec. V), whose
 * many stencil and pointwise operations ProtoX fuses. The paper names no
 * scheme; this is the textbook second-order one:
 *   cell averages U = (rho, rho u, rho v, E) of an ideal gas,
 *     p = (gamma - 1) (E - rho (u^2 + v^2) / 2), c = sqrt(gamma p / rho);
 *   minmod-limited linear reconstruction of (rho, u, v, p) per direction,
 *     slope_i = minmod(W_i - W_{i-1}, W_{i+1} - W_i), minmod(a, b) = 0 if
 *     ab <= 0 else the argument of smaller magnitude;
 *   Rusanov flux F = (F(W_L) + F(W_R)) / 2 - a (U_R - U_L) / 2,
 *     a = max(|u_n| + c) of the two face states;
 *   L(U) = -(F_{i+1/2} - F_{i-1/2}) / dx - (G_{j+1/2} - G_{j-1/2}) / dy;
 *   SSP-RK2: U1 = U + dt L(U), U' = (U + (U1 + dt L(U1))) / 2;
 *   dt = cfl / max over cells of (|u| + c) / dx + (|v| + c) / dy, from the
 *     state the step starts from.
 * Periodic in x and y. Each Runge-Kutta stage is one fused kernel (loads,
 * primitives, slopes, face states, fluxes, divergence, update, and in the
 * second stage the next step's max wave speed, all in one pass).
 *
 * Layout: four planes (rho, rho u, rho v, E) in this order, each ny rows of
 * nx cells, x fastest, row pitch ld, the planes cs elements apart. */
typedef struct {
  int32_t nx, ny;  /* cells along x and y; >= 0 (0: empty, no-op) */
  int64_t ld;      /* elements between row starts; >= nx */
  int64_t cs;      /* elements between component planes; >= (ny - 1) * ld + nx */
  int32_t dtype;   /* px_dtype of every plane (arithmetic in that precision) */
  double dx, dy;   /* cell sizes, finite and > 0 */
} px_euler_grid;

/* nsteps SSP-RK2 steps from u_in into u_out (device pointers; u_out may equal
 * u_in, otherwise they must not overlap). gamma > 1. dt_fixed > 0 fixes every
 * step's dt; dt_fixed = 0 takes dt = cfl / (max wave speed) of each step's
 * starting state (cfl > 0). dt_dev: NULL or nsteps doubles (device) that
 * receive each step's dt. A non-physical state (rho <= 0 or p < 0) yields NaN
 * there and in the state. The stage field lives in the context's scratch
 * (grown on demand: such a call synchronises). Asynchronous. */
px_status px_euler_step(px_ctx* ctx, const px_euler_grid* g, const void* u_in, void* u_out,
                        double gamma, double cfl, int nsteps, double dt_fixed, double* dt_dev,
                        void* stream);

/* Conserved planes u = (rho, rho u, rho v, E) from primitive planes
 * w = (rho, u, v, p), same layout; w and u must not overlap. Asynchronous. */
px_status px_euler_conserved(px_ctx* ctx, const px_euler_grid* g, const void* w, void* u,
                             double gamma, void* stream);

/* Max-norm residual check (Sec. IV step 3, OL rule ||.||_inf with a = h):
 * *out_host = ||rho - L phi||_inf and, if rho_norm_host is not NULL,
 * *rho_norm_host = ||rho||_inf. Evaluated in FP64 for both dtypes (FP32 fields
 * are widened exactly). NaN anywhere gives NaN. SYNCHRONISES the stream. */
px_status px_residual_norm(px_ctx* ctx, const px_grid* g, const void* phi,
                           const void* rho, double* out_host,
                           double* rho_norm_host, void* stream);

/* Asynchronous form of px_residual_norm: out_dev (DEVICE, 2 doubles) receives
 * {||rho - L phi||_inf, ||rho||_inf}. out_dev is overwritten, not maxed into. */
px_status px_residual_norm_async(px_ctx* ctx, const px_grid* g, const void* phi,
                                 const void* rho, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PROTOX_H */
