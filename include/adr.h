/*
 * adr.h -- C ABI of the GB300 (sm_103a) directional diffusion splitting
 * solver for 2D advection-diffusion-reaction problems
 * (Drebotiy & Shynkarenko, arXiv 2411.11041).
 *
 * Problem (§2, eqs. BVP1 and Parabolic1):
 *     u_t - mu Lap u + beta . grad u + sigma u = f   in Omega,  u = 0 on its boundary,
 * and its stationary limit.  The library reduces every split substep
 * (§5, eq. SemiDiscrSplit) to independent 1D linear-FEM problems along the
 * integral curves of beta (family B) and of gamma = (beta2, -beta1) (family G)
 * (§6, eqs. SemiDiscrSplit1Dbeta / SemiDiscrSplit1Dgamma).  It carries values
 * between the two families through the grid: curve -> grid by the
 * min/max-crossing rule of §6, grid -> curve by bilinear interpolation (§6.1).
 *
 * Conventions used by every call below:
 *  - Grids are row-major [ny][nx] arrays over the NODES of a uniform grid on
 *    [x0,x1] x [y0,y1], boundary nodes included (spacing hx = (x1-x0)/(nx-1)).
 *  - Every array argument is a DEVICE pointer (CUDA global memory) unless it
 *    is documented as a host pointer.  The caller owns it.  The library never
 *    frees or retains caller memory past the call, except that a handle keeps
 *    private copies of what adr_create derives from its inputs.
 *  - `stream` is a cudaStream_t passed as void*; all device work of a handle is
 *    ordered on it.  NULL means the legacy default stream.
 *  - Functions never abort and never throw across the ABI.  They return an
 *    adr_status; adr_last_error() gives a message for the calling thread.
 *  - Domain: a grid cell is active when its 4 corner nodes have mask != 0;
 *    Omega_h is the union of active cells.  A node is interior when its 4
 *    cells are active; every other node of Omega_h carries u = 0.
 */
#ifndef ADR_H
#define ADR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADR_OK = 0,
    ADR_EINVAL = 1,   /* invalid argument (sizes, mu/sigma <= 0, |beta| = 0, empty mask ...) */
    ADR_ENOMEM = 2,   /* device or host allocation failed */
    ADR_ECUDA = 3,    /* a CUDA call failed (message in adr_last_error) */
    ADR_ENOCONV = 4,  /* max_iter reached before tol, or the iteration diverged (a norm
                         stopped being finite); outputs hold the last iterate */
    ADR_EGEOM = 5,    /* the curve families do not cover the domain (§3, §6): tracing failed
                         (closed integral curve, |beta| = 0 on a curve), a family has no
                         inflow boundary, or an interior node meets no curve of a family */
    ADR_ETIMEOUT = 6  /* a bounded device wait gave up (tensor-core network kernels) */
} adr_status;

typedef enum {
    ADR_FP64 = 0,        /* every step in FP64 */
    ADR_FP32_REFINE = 1  /* line solves in FP32 as one step of mixed-precision iterative
                            refinement: from the current curve values x0 = u the residual
                            dt (F - S u) of the substep system is formed in FP64, the
                            correction is solved in FP32, and v = u + dt d, the grid map,
                            the norms and the convergence test stay in FP64.  The FP32
                            rounding of d does not vanish at the fixed point (d != 0
                            there), so once the relative update reaches 100 tol the
                            iteration solves its corrections in FP64 (adr_stats.fp32_steps
                            counts the steps before that) */
} adr_precision;

typedef enum {
    ADR_INIT_ZERO = 0,     /* u_0 = 0 */
    ADR_INIT_USER = 1,     /* u_0 = caller array (non-interior nodes ignored) */
    ADR_INIT_PAPER_U0 = 2, /* s(u_0, v) = <l, v>  (§5, eq. u0stationary) */
    ADR_INIT_LEARNED = 3   /* the learned warm start: the network attached with
                              adr_set_warm_start corrects the paper's u_0 (256 x 256 grids) */
} adr_init;

/* Grid of nx x ny nodes on [x0,x1] x [y0,y1]; nx, ny >= 3. */
typedef struct {
    int nx, ny;
    double x0, y0, x1, y1;
} adr_grid;

/* Options of a handle.  theta: time-scheme weight, (0,1] (§4 eq. SemiDiscr;
 * 0.5 = Crank-Nicolson).  dt: pseudo-time step of the stationary iteration
 * (<= 0 selects 2/sqrt(lmin*lmax), lmin = sigma, lmax = 12 mu/h^2 +
 * 2 sqrt(3) max|beta|/h).  tol: stop when |u_{j+1}-u_j|_2/|u_{j+1}|_2 <= tol over
 * interior nodes (tol <= 0 runs exactly max_iter steps and succeeds).
 * max_iter: cap (>= 0). */
typedef struct {
    int prec;        /* adr_precision */
    double theta;
    double dt;
    double tol;
    int max_iter;
    int init;        /* adr_init */
    int rows_per_thread;    /* launch shape of the curve solve: 2, 4, 8 or 16 rows per
                               thread (0 = 16); a curve of m unknowns gets blocks of the
                               smallest power-of-two T >= 32 with T * rows_per_thread >= m,
                               at most 1024 (longer curves take up to 16 rows per thread;
                               curves of more than 16384 unknowns are refused) */
    int map_blocks_per_sm;  /* blocks per SM of the curve -> grid map: 1..8 (0 = 4) */
    int interp_weights;     /* curve -> grid: 0 = average of the row and column values (§6);
                               1 = weights by the opposite direction's crossing gap, for
                               flow nearly parallel to a grid axis */
    int stabilize;          /* the 1D problems on the B curves: 0 = Galerkin (§6, the paper);
                               1 = SUPG, the per-line stabilisation the paper's conclusions
                               propose for singularly perturbed problems (test function
                               w + tau |beta| w', tau = h/(2|beta|)(coth Pe - 1/Pe) per element);
                               FP64 mode only */
    int transfer;           /* how values pass from one curve family to the other:
                               0 = through the grid (§6: curve values -> grid nodes, then
                               bilinear samples at the other family's nodes);
                               1 = directly, the transfer the paper's conclusions propose:
                               a node takes the value interpolated linearly, along its own
                               curve, between the nearest crossings with the other family
                               before and after it (each crossing's value linear along the
                               crossed segment; no crossing on a side: the curve's end, value
                               0).  The iteration state then lives at the B curve nodes, the
                               relative update is taken over them, and the grid is touched only
                               by the initial state (bilinear samples) and the output (the
                               curve -> grid map of §6).  FP64 mode only; not in batches */
    int anderson;           /* acceleration of the stationary iteration: 0 = none; m = 1..8 =
                               Anderson extrapolation over the last m split steps (the
                               multi-parameter pseudo-steps read as per-step weights: a cycle of
                               pseudo steps Δt does not keep the split step's fixed point, these
                               weights do).  With g_k the split step's output from u_k and
                               f_k = g_k - u_k, u_{k+1} = g_k - Σ_i γ_i (g_{k-i+1} - g_{k-i}),
                               γ minimising |f_k - Σ_i γ_i (f_{k-i+1} - f_{k-i})|.  The relative
                               update (tol) is |f_k| / |g_k|, as without it.  Applies to the
                               stationary solves (also the slices of adr_step_parabolic mode 1),
                               not to the time steps of mode 0.  FP64 mode only; not in batches */
} adr_opts;

/* Result statistics (host struct filled by the solve calls). */
typedef struct {
    int iters;          /* split steps performed */
    double rel_update;  /* last relative update */
    double ms;          /* device time of the solve (CUDA events on the stream) */
    double line_dofs;   /* line unknowns solved in total (both families, all steps) */
    double dt;          /* pseudo step used */
    double min_pivot;   /* smallest |pivot| that Thomas elimination of the curve systems
                           (M + theta dt S per curve, §6; both families) meets, computed on
                           the device when the systems are factored; +inf when nothing was
                           factored */
    double max_correction; /* ADR_FP32_REFINE: largest |dt d| over the curve nodes of the last
                           split step, d the FP32 correction solved from the FP64 residual;
                           its FP32 rounding bounds what the mode loses against FP64.
                           0 in FP64 mode */
    int fp32_steps;     /* ADR_FP32_REFINE: split steps whose corrections were solved in
                           FP32 (the rest in FP64); 0 in FP64 mode */
} adr_stats;

typedef struct adr_problem adr_problem; /* opaque handle */

/* Fill opts with the defaults: FP64, theta 0.5, dt auto, tol 1e-10,
 * max_iter 100000, zero initial state, default launch shapes. */
void adr_default_opts(adr_opts* opts);

/*
 * adr_create -- build a problem handle (§2 eq. BVP1 data; §6 geometry).
 * grid:  host pointer.  mask: device uint8 [ny][nx].  mu, sigma > 0
 * (constants, §2).  beta1, beta2, f: device double [ny][nx] nodal values.  A
 * field that is the same at every node of Omega_h gives straight line
 * families; any other field gives RK4-traced curves seeded on the inflow
 * boundary (eqs. cauchyStartSets, CauchyBeta, CauchyGamma).  opts: host
 * pointer (copied).  On success *out owns its device buffers until
 * adr_destroy.  They come from the library's stream-ordered memory pool on
 * the current device, allocated in the order of `stream` (and setup's
 * temporaries too).  Inputs may be freed after the call returns.
 * Errors: ADR_EINVAL (bad sizes/coefficients, |beta| = 0 or non-finite data on
 * Omega_h, empty mask), ADR_EGEOM, ADR_ENOMEM, ADR_ECUDA.
 */
adr_status adr_create(const adr_grid* grid, const uint8_t* mask, double mu, double sigma,
                      const double* beta1, const double* beta2, const double* f,
                      const adr_opts* opts, void* stream, adr_problem** out);

/*
 * adr_solve_stationary -- solve BVP1 as the large-time limit of Parabolic1
 * (§2) with the split scheme (§5 eq. SemiDiscrSplit, reduced to the curves as
 * in §6) until the relative update is <= opts.tol or opts.max_iter steps ran.
 * u_init: device [ny][nx], read only when opts.init == ADR_INIT_USER (else may
 * be NULL).  u_out: device [ny][nx] <- the solution: for theta = 0.5 the
 * midpoint (u_j + u_{j+1/2})/2 of the last step, else u_{j+1}.
 * u_iter_out: nullable device [ny][nx] <- u_{j+1}.  stats: nullable host.
 * The call returns after the solve has finished on the stream.
 * Errors: ADR_ENOCONV (outputs written), ADR_EINVAL, ADR_ECUDA.
 */
adr_status adr_solve_stationary(adr_problem* prob, const double* u_init, double* u_out,
                                double* u_iter_out, adr_stats* stats);

/*
 * adr_step_parabolic -- advance Parabolic1 (§2) by nsteps steps of dt.
 * mode 0: the paper's scheme, one split step per time step (§5 eq.
 *         SemiDiscrSplit with dt and opts.theta).
 * mode 1: implicit Euler in time; each slice
 *         -mu Lap u + beta.grad u + (sigma + 1/dt) u = f + u_n/dt
 *         is solved by the stationary iteration (opts.theta, opts.dt as the
 *         pseudo step, opts.tol, opts.max_iter), warm-started from u_n.
 * u_inout: device [ny][nx], the state, overwritten (non-interior nodes set
 * to 0).  stats: nullable host (iters = split steps over all slices).
 * Errors: ADR_EINVAL, ADR_ENOCONV (a slice hit max_iter; stepping continues),
 * ADR_ECUDA.
 */
adr_status adr_step_parabolic(adr_problem* prob, double dt, int nsteps, int mode,
                              double* u_inout, adr_stats* stats);

/* Release a handle and its device buffers (NULL is a no-op).  The device is
 * synchronised first (a batch may still use the buffers on its stream); the
 * buffers go back to the library's pool, which keeps up to 8 GB of freed
 * device memory mapped for later handles and returns the rest to the driver. */
void adr_destroy(adr_problem* prob);

/* Message of the last failing call on this thread ("" if none). */
const char* adr_last_error(void);

/*
 * Geometry inspection (setup results, for tests and tools).  Host outputs.
 * adr_num_lines / adr_num_line_nodes: counts of family fam (0 = B, 1 = G).
 * adr_get_lines: off[n_lines+1] (int32), xi/eta[n_nodes] index coordinates
 * (x = x0 + xi*hx), h[n_lines] element length; any pointer may be NULL.
 * adr_get_crossings: per grid node the 4 crossings used by the curve->grid map
 * (row left, row right, column down, column up): seg[4*nx*ny] global index of
 * the segment's first curve node (-1 boundary, -2 non-interior node),
 * t[4*nx*ny] position in the segment, pos[4*nx*ny] coordinate along the grid
 * line.  Errors: ADR_EINVAL.
 */
int adr_num_lines(const adr_problem* prob, int fam);
int adr_num_line_nodes(const adr_problem* prob, int fam);
adr_status adr_get_lines(const adr_problem* prob, int fam, int* off, double* xi, double* eta,
                         double* h);
adr_status adr_get_crossings(const adr_problem* prob, int fam, int* seg, double* t, double* pos);
/* adr_get_transfer: the direct transfer's crossings (handles created with
 * opts.transfer == 1): per node k of family fam, entries 2k (the nearest
 * crossing at or before the node along its curve) and 2k+1 (at or after it):
 * seg = global index of the first node of the other family's crossed segment
 * (-1 none on that side: the curve's end; -2 the node is a curve end), t =
 * position in that segment, pos = position along the node's own curve in
 * element units (0 .. n).  Errors: ADR_EINVAL (also for opts.transfer == 0). */
adr_status adr_get_transfer(const adr_problem* prob, int fam, int* seg, double* t, double* pos);

/*
 * adr_split_step -- one split step u -> (u_half, u_next) of eq. SemiDiscrSplit
 * with the handle's theta and the given dt (device arrays [ny][nx]; u_half
 * may be NULL).  The building block of both solve calls, exported so that
 * callers can drive their own time loop.  Errors: ADR_EINVAL, ADR_ECUDA.
 */
adr_status adr_split_step(adr_problem* prob, double dt, const double* u, double* u_half,
                          double* u_next);

/*
 * adr_paper_u0 -- the paper's initial state for advection-dominated problems
 * (§5 eq. u0stationary): one steady solve s_i(u0, w) = <l_i, w> on every B
 * curve, mapped to the grid.  u0: device [ny][nx].  The work is enqueued on
 * the handle's stream and the call returns without waiting for it (many
 * handles' states can then be formed back to back).  Errors: ADR_ECUDA.
 */
adr_status adr_paper_u0(adr_problem* prob, double* u0);

/*
 * adr_time_kernels -- device time of the sweep kernels of one split step, each
 * launched reps times back to back on the handle's stream in the launch
 * configuration of the solve, timed with CUDA events on that stream: B gather,
 * B curve solve, B curve->grid map, G gather, G curve solve, G map (+ norms).
 * The gathers are passes of their own through the grid (both precision
 * modes, single handles and batches).  With
 * opts.transfer = 1: 0, B solve, B -> G transfer, 0, G solve,
 * G -> B transfer (+ norms).  They run on the handle's current state (work
 * buffers only; no caller memory is touched).  ms_out: host double[6],
 * average milliseconds per launch.  Errors: ADR_EINVAL, ADR_ECUDA.
 */
adr_status adr_time_kernels(adr_problem* prob, int reps, double* ms_out);

/*
 * adr_autotune -- choose the launch shapes of a handle by measurement (no
 * counterpart in the paper; the result does not change the solution).  Each
 * candidate (rows_per_thread in {4, 8, 16}, map_blocks_per_sm in {2, 4, 8}) is
 * applied and one split step's kernels are timed reps times with CUDA events
 * on the handle's stream; the fastest is kept.  Outputs (host, nullable): the
 * chosen rows_per_thread and map_blocks_per_sm and its ms per split step.
 * The handle's curve groups are rebuilt for every candidate, so a batch built
 * over the handle before the call must be destroyed and built again (or
 * tuned with adr_batch_autotune, which rebuilds its own).  Errors:
 * ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA.
 */
adr_status adr_autotune(adr_problem* prob, int reps, int* rows_per_thread,
                        int* map_blocks_per_sm, double* ms_per_step);

/*
 * Batches (many independent problems of uneven size and shape): every split
 * step of all active problems runs as one persistent launch per sweep stage,
 * over one list of work items (curves of all problems, longest first), and the
 * whole outer loop of the batch is one CUDA graph whose WHILE condition stays
 * set while any problem is active.  Each problem keeps its own options (dt,
 * theta, tol, max_iter, init) and convergence test; a converged problem drops
 * out of the later launches.  All handles must share the precision mode;
 * handles with opts.transfer == 1 are refused; opts.anderson may differ per
 * handle (0: that problem is not extrapolated).
 *
 * adr_batch_create: probs (host array of n handles, not owned; they must
 * outlive the batch and must not be used concurrently with it).  stream: the
 * batch's cudaStream_t (or NULL).  Errors: ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA.
 * adr_batch_solve: u_init (nullable host array of n device grids, read for
 * handles with init == ADR_INIT_USER), u_out (host array of n device grids
 * [ny][nx] of the respective handles), u_iter_out (nullable host array of n
 * nullable device grids <- u_{j+1}, the iterate, as in adr_solve_stationary),
 * stats (nullable host array of n; ms = device time of the whole batch).  Returns ADR_ENOCONV if a problem hit
 * max_iter (all outputs written).
 * adr_batch_autotune: times reps batched split steps from u = 0 for 4, 8 and
 * 16 rows per thread (every handle of the batch regrouped each time: the
 * handles' own cached solve graphs are dropped) and keeps the fastest; the
 * batch is then rebuilt with its handles' options.  rows_out, ms_out
 * (nullable): the choice and its device time per split step.  Errors:
 * ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA.
 * adr_solve_batch: create, solve from the handles' initial states, destroy.
 */
typedef struct adr_batch adr_batch;
adr_status adr_batch_create(adr_problem* const* probs, int n, void* stream, adr_batch** out);
adr_status adr_batch_solve(adr_batch* batch, const double* const* u_init, double* const* u_out,
                           double* const* u_iter_out, adr_stats* stats);
void adr_batch_destroy(adr_batch* batch);
adr_status adr_batch_autotune(adr_batch* batch, int reps, int* rows_out, double* ms_out);
adr_status adr_solve_batch(adr_problem* const* probs, int n, double* const* u_out,
                           adr_stats* stats);

/*
 * adr_cross_substep_noalloc -- one cross-flow substep (G family: curve solve
 * with m_i and the curve -> grid map) that allocates nothing.  The paper has no
 * counterpart; this call exists for callers that cannot call cudaMalloc: code
 * running under a memory pool or caching allocator owned by someone else
 * (a host framework that forbids raw device allocations), and latency-bound
 * callers that must not let an allocation synchronise the device mid-loop.
 * They keep the curve data and crossings in their own memory (for example
 * copies of adr_get_lines / adr_get_crossings of family 1, made once by a
 * setup step that could allocate) and pass them in with the input and output.
 *
 * u_in -> u_out (device double [ny][nx]): u_out = G_G(u^i + dt d) where on
 * every G curve (M + theta dt mu K) d = -mu K u^i, u^i the bilinear samples of
 * u_in.  off[n_lines+1] (device int32, non-decreasing from off[0] = 0 to
 * off[n_lines] == n_nodes), h[n_lines], xi/eta[n_nodes]: the family-1 curves
 * as adr_get_lines reports them.  seg/t/pos[4*nx*ny]: the family-1 crossings
 * as adr_get_crossings reports them (seg = -2 marks a non-interior node, which
 * gets 0).  G_G is the paper's curve -> grid rule with the plain average of
 * the row and the column value (opts.interp_weights does not apply here).
 * stream: cudaStream_t or NULL.  The call only launches work; it returns
 * before the kernels finish.
 *
 * Work space: a fixed array of 4 x 524288 doubles (16 MiB) in device memory,
 * reserved by every GPU that loads the library until the process exits.
 * n_nodes > 524288 is rejected with ADR_EINVAL.  Every call looks up the
 * array's device address on the current device (cudaGetSymbolAddress, no
 * allocation); the first call on a device also loads the library's module
 * there, so make that first call before any stream capture.  Every call on a
 * device shares the one array and it keeps the last call's contents; a call
 * writes every entry it reads (a curve whose offsets fall outside
 * [0, n_nodes], or that has fewer than 2 nodes, is skipped and its nodes in
 * range read as 0), so nothing needs clearing, but calls whose kernels may
 * overlap on the GPU (different streams, no ordering between them) race on it
 * and must be serialised by the caller.  Errors: ADR_EINVAL, ADR_ECUDA.
 */
adr_status adr_cross_substep_noalloc(int nx, int ny, double mu, double theta, double dt,
                                     const double* u_in, int n_lines, int n_nodes, const int* off,
                                     const double* h, const double* xi, const double* eta,
                                     const int* seg, const double* t, const double* pos,
                                     double* u_out, void* stream);

/*
 * Learned warm start (no counterpart in the paper; the paper's iteration stays
 * the solver and alone decides convergence; the network only supplies u_0).
 *
 * A convolutional network maps a problem on a 256 x 256 node grid, and a
 * first initial state u0 of it (normally the state of eq. u0stationary, from
 * adr_paper_u0), to the smooth part of the correction u - u0, u the iterate
 * the stationary solve converges to; adr_cnn_initial_state turns it into an
 * initial state for ADR_INIT_USER.  The grid is read as 64 x 64 cells of 4 x 4
 * nodes, cell (r, c) holding nodes (4 r + a, 4 c + b), a, b in 0..3.  Every
 * problem is scaled by s = max |u0| (1 when u0 is NULL or zero).
 * Features (NHWC, [batch][64][64][40], BF16): channel 4 a + b = f at node
 * (4 r + a, 4 c + b); 16 + 4 a + b = u0 / s there; 32, 33: cell means of
 * beta1, beta2; 34: (log10 mu + 2.5)/1.5; 35: sigma - 1; 36: cell mean of the
 * mask; 37..39: 0.
 * Network: eight 3 x 3 convolutions with zero padding, dilations
 * 1 2 4 8 16 32 1 1, channels 40 64 64 128 128 128 64 64 8, bias, ReLU after
 * all but the last (544 k parameters).  Output ([batch][64][64][8], FP32):
 * channel 0 predicts the cell mean of (u - u0) / s; channels 1..7 are not used.
 * Parameters are one FP32 vector packed as W_0, b_0, W_1, b_1, ... with
 * W_l[(tap * Cin + ci) * Cout + co], tap = 3 ky + kx.  Convolutions (forward,
 * data and weight gradients) run on the BF16 tensor cores with FP32
 * accumulation; Adam keeps FP32 master parameters.  Loss: 1/2 of the mean
 * squared error of channel 0 over all cells of a batch.
 */
typedef struct adr_cnn adr_cnn; /* opaque network handle */

/* Number of parameters (host call, no GPU needed). */
long adr_cnn_num_params(void);

/* adr_cnn_create: params (host float[adr_cnn_num_params()], copied) are the
 * initial parameters; max_batch bounds the batch of every later call; stream is
 * the handle's cudaStream_t (or NULL).  Errors: ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA. */
adr_status adr_cnn_create(int max_batch, const float* params, void* stream, adr_cnn** out);
void adr_cnn_destroy(adr_cnn* cnn);
/* Host copies of the FP32 parameters; set also clears the Adam moments. */
adr_status adr_cnn_set_params(adr_cnn* cnn, const float* params);
adr_status adr_cnn_get_params(adr_cnn* cnn, float* params);

/* adr_cnn_features: batch problems on n x n nodes, n = 256 (device arrays,
 * problem b at offset b n n): f, beta1, beta2 double, mask uint8, u0 double
 * (nullable: zeros); mu, sigma device double[batch].  x: device BF16 (uint16
 * storage) [batch][64][64][40]; scale: device double[batch] <- s of each
 * problem.  Launch only.  Errors: ADR_EINVAL (n != 256, NULL pointer). */
adr_status adr_cnn_features(int batch, int n, const double* f, const double* beta1,
                            const double* beta2, const uint8_t* mask, const double* mu,
                            const double* sigma, const double* u0, uint16_t* x, double* scale,
                            void* stream);
/* adr_cnn_targets: t (device float [batch][64][64]) <- the cell means of
 * (u_b - u0_b) / s_b; u, u0 (nullable: zeros) device double [batch][n][n],
 * n = 256; scale: device double[batch] from adr_cnn_features.  Launch only. */
adr_status adr_cnn_targets(int batch, int n, const double* u, const double* u0,
                           const double* scale, float* t, void* stream);
/* adr_cnn_forward: y (device float [batch][64][64][8]) <- the network's output.
 * Launch only, on the handle's stream.  Errors: ADR_EINVAL, ADR_ECUDA. */
adr_status adr_cnn_forward(adr_cnn* cnn, int batch, const uint16_t* x, float* y);
/* adr_cnn_loss_grad: forward and backward without an update.  grad (nullable
 * device float[num_params]) <- d loss / d params; loss (nullable host) <- the
 * loss (the call then waits for the stream). */
adr_status adr_cnn_loss_grad(adr_cnn* cnn, int batch, const uint16_t* x, const float* t,
                             float* grad, double* loss);
/* adr_cnn_train_step: forward, backward and one Adam step (beta1 0.9, beta2
 * 0.999, eps 1e-8, learning rate lr > 0).  loss: nullable host, the loss before
 * the update (the call then waits for the stream). */
adr_status adr_cnn_train_step(adr_cnn* cnn, int batch, const uint16_t* x, const float* t,
                              float lr, double* loss);
/* adr_cnn_set_wait_limit: bound of the tensor-core kernels' mbarrier waits:
 * spins > 0 non-blocking polls, or spins = 0 the default bound (about a second
 * of blocking polls).  A wait that reaches its bound gives up: the kernel lets
 * the loads and MMAs it issued finish, frees its tensor memory, skips its
 * output and flags the handle; adr_cnn_sync, or a call that returns the loss,
 * then reports ADR_ETIMEOUT and clears the flag.  Outputs of the calls since
 * the last report are then not valid.  A bound of a few polls makes the waits
 * give up, which is how the timeout path is tested.  Errors: ADR_EINVAL. */
adr_status adr_cnn_set_wait_limit(adr_cnn* cnn, long long spins);
/* adr_cnn_sync: wait for the handle's stream; ADR_ETIMEOUT (flag cleared) if a
 * bounded wait gave up since the last report, else ADR_OK. */
adr_status adr_cnn_sync(adr_cnn* cnn);
/* adr_cnn_initial_state: u_out (device double [256][256]) <- u0 + s * v at the
 * interior nodes, 0 elsewhere, v the bilinear interpolation of channel 0 of one
 * prediction y (device float [64][64][8]) with cell centres at node
 * 4 k + 1.5 (clamped at the outer half cells); u0 device double [256][256]
 * (nullable: zeros); scale: device pointer to s (nullable: 1).  Pass u_out as
 * u_init with ADR_INIT_USER.  Launch only, on the problem's stream.
 * Errors: ADR_EINVAL (grid not 256 x 256). */
adr_status adr_cnn_initial_state(adr_problem* prob, const float* y, const double* u0,
                                 const double* scale, double* u_out);

/* adr_set_warm_start -- attach a warm-start network to a problem on a 256 x 256
 * grid, so that opts.init == ADR_INIT_LEARNED starts adr_solve_stationary (and
 * adr_batch_solve) from the network's state: the paper's initial state u0 of
 * §5 eq. u0stationary, the features of the problem and u0 (adr_cnn_features,
 * with the problem's own mask, mu and sigma), one forward pass, and
 * adr_cnn_initial_state -- the chain a caller can also run by hand and pass
 * with ADR_INIT_USER.  The iteration that follows is the paper's, to the same
 * tolerance.  cnn: a handle from adr_cnn_create, not owned: it must outlive
 * every solve that uses it; NULL detaches.  The forward pass runs on the
 * problem's stream, ordered after the network's pending work and before its
 * later work.  The first attach allocates the chain's buffers (about 0.9 MB)
 * from the library's pool.  A solve with ADR_INIT_LEARNED and no network
 * returns ADR_EINVAL.  Errors: ADR_EINVAL (grid not 256 x 256), ADR_ENOMEM,
 * ADR_ECUDA. */
adr_status adr_set_warm_start(adr_problem* prob, adr_cnn* cnn);

#ifdef __cplusplus
}
#endif
#endif /* ADR_H */
