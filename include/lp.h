/*
 * lp.h -- C ABI of the GB300 evaluator of 2D log-kernel volume and layer
 * potentials by heat-kernel splitting (Fryklund, Greengard, Jiang, Potter,
 * "A lightweight, geometrically flexible fast algorithm for the evaluation
 * of layer and volume potentials", arXiv 2409.11998).
 *
 * The library evaluates, at arbitrary target points x,
 *
 *   V[f](x) = int_Omega      G(x - x') f(x')  dx'                 (Sec. 1, eq. volpotposgreen)
 *   S[s](x) = int_dOmega     G(x - x') s(x')  ds_x'               (Sec. 1, eq. slpot)
 *   D[m](x) = int_dOmega  dG/dnu_x'(x - x') m(x') ds_x'           (Sec. 1, eq. dlpot)
 *
 * with G(x) = -log|x| / (2 pi) (eq. GreenPoisson) and nu the outward normal
 * (so D[1] = -1 in Omega, -1/2 on dOmega, 0 outside).  Each potential is the
 * sum of
 *   - a smooth part: the kernel G_H[delta_1] = G - E1(|x|^2/(4 delta_1))/(4 pi)
 *     (eq. splitting2) summed over quadrature-weighted sources, computed as
 *     the near-history plus far-history Fourier sums of Sec. 3 (type-1 NUFFT,
 *     diagonal multiplier of eq. vnearkspace / eq. vfarkspace, type-2 NUFFT),
 *   - a local part: the asymptotic expansions of Sec. 4 (single-layer,
 *     double-layer and volume lemmas), evaluated per target after a
 *     closest-point search on the boundary panels.
 *
 * Discretisation (Sec. 2.2): volume sources are quadrature nodes x_j with
 * weights w_j (any smooth rule on any triangulation, gaps allowed); the
 * boundary is a single closed counter-clockwise curve given as n_panels
 * consecutive panels of panel_order Gauss-Legendre nodes each, with
 * quadrature weights (|gamma'| times the scaled Gauss weights) and outward
 * normals.  Densities sigma, mu are given at the boundary nodes.
 *
 * Memory: every pointer argument may be DEVICE memory (cudaMalloc, managed)
 * or HOST memory (pageable or pinned).  Device pointers are used in place;
 * host inputs are copied to plan-owned device buffers and host outputs are
 * copied back, on the plan's stream.  Caller-owned buffers must stay valid
 * until the call's work on the stream has completed (lp_sync).  All work of
 * a plan runs on the stream given in lp_domain (0 = legacy default stream).
 *
 * Errors: every call returns an lp_status.  No call launches work when it
 * returns LP_ERR_ARG.  Problems detected on the device (a point outside the
 * box, a band target outside the domain where V_L is undefined, a closest-
 * point search that did not converge) set bits of a plan status word that
 * lp_sync returns.  No kernel waits on another kernel or on the host, so no
 * device-side wait can hang; lp_sync_timeout bounds the host's wait.  Calls
 * on one plan must not be made concurrently from several host threads.
 */
#ifndef LP_H_
#define LP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_plan_s* lp_plan_t;
typedef struct lp_batch_s* lp_batch_t;

typedef enum {
  LP_OK = 0,
  LP_ERR_ARG = 1,            /* invalid argument; nothing was launched */
  LP_ERR_OUT_OF_BOX = 2,     /* a source or target lies outside the plan's box, or a
                                coordinate or source strength is not finite */
  LP_ERR_NOMEM = 3,          /* device allocation failed */
  LP_ERR_CUDA = 4,           /* a CUDA runtime or cuFFT call failed */
  LP_ERR_UNSUPPORTED = 5,    /* V requested at an exterior target within 12 sqrt(delta_1)
                                of the boundary, where Sec. 4 gives no expansion; or a
                                refined plan passed to lp_batch_execute */
  LP_ERR_STATE = 6,          /* call order violated (e.g. execute before lp_volume) */
  LP_ERR_NEWTON = 7,         /* the closest-point search (Sec. 2.2: nearest node, then
                                Newton on the panel polynomial) failed for some target of
                                the local band: 20 double-precision Newton steps ended with
                                a Newton step of 1e-6 or more in the panel parameter (the
                                slow gradient steps taken where the distance is flat along
                                the boundary, near a centre of curvature, do not count),
                                the foot ran
                                past the far end of the adjacent panel as well, or the foot
                                lies where the panel's speed |gamma'| is below 1e-9 of the
                                box side, so that the tangent frame of Sec. 4 is undefined
                                (a cusp, or a panel of nearly coincident nodes); the local
                                terms of those targets are unreliable */
  LP_ERR_TIMEOUT = 8         /* lp_sync_timeout: the plan's work did not complete within
                                the given time (it keeps running; nothing is cancelled) */
} lp_status;

enum { LP_FP64 = 0, LP_FP32 = 1 };

/* lp_domain.refine_levels: choose the number of refinement levels from the
 * plan's tolerance and expansion order (Sec. 4.4). */
#define LP_REFINE_AUTO (-1)

/* lp_domain.levels: one history level when its grid is small (at most
 * LP_SINGLE_LEVEL_MAX_GRID points per side), else two. */
#define LP_LEVELS_AUTO (-1)
#define LP_SINGLE_LEVEL_MAX_GRID 1536

/* lp_domain.autotune */
#define LP_AUTOTUNE_BINS 1
#define LP_AUTOTUNE_FULL 2

typedef struct {
  int precision;        /* LP_FP64: tolerances down to ~1e-12.  The volume spread,
                           FFTs, multiplier and interpolation run in double-float
                           arithmetic (pairs of floats, ~48 bits); the boundary
                           spread, the local expansions and all outputs in double.
                           LP_FP32: spread, FFT, interpolation and local
                           expansions in float; the multiplier table is built in
                           double and the zero-mode (log-constant) term is summed
                           and added in double. */
  int order;            /* asymptotic order p in {3,4,5}: local terms through
                           delta^{(p-1)/2} are kept (error O(delta^{p/2})); 0 -> 5 */
  double box_lo[2];     /* box containing every source and target; the plan adds */
  double box_hi[2];     /* its own margins for the periodic grids */
  int64_t n_panels;     /* boundary panels (0: no boundary: free-space V only) */
  int panel_order;      /* Gauss-Legendre nodes per panel (2..32) */
  const double* bnd_xy;     /* [n_panels*panel_order][2] nodes, panel after panel */
  const double* bnd_w;      /* [n_panels*panel_order] arc-length quadrature weights */
  const double* bnd_normal; /* [n_panels*panel_order][2] outward unit normals */
  void* stream;         /* cudaStream_t for all work of the plan */
  int refine_levels;    /* dyadic refinement of the local layer potentials
                           (Sec. 4.4): J in 0..6, or LP_REFINE_AUTO.  0: S_L,
                           D_L from the expansions at delta.  J > 0: expansions
                           at delta/4^J plus direct sums of the difference
                           kernels G_H[delta/4^j] - G_H[delta/4^(j-1)],
                           j = 1..J, over the panels split into 2^j
                           Gauss-Legendre intervals; the expansion error falls
                           by 4^(order/2) per level.  LP_REFINE_AUTO: the
                           smallest J with (delta/4^J)^(order/2) <= tol (the
                           selection rule of Sec. 4.4), at most 6.  V_L keeps
                           delta.  Plans with J > 0 are not accepted by
                           lp_batch_execute. */
  int levels;           /* history levels (Sec. 3): 0 or 2 = near history on
                           [delta_1, delta_2] plus far history from delta_2 =
                           32 delta_1; 1 = one level, the truncated-kernel
                           representation of G_H[delta_1] on one grid (the
                           paper's one-level alternative, delta_2 = delta_1);
                           LP_LEVELS_AUTO = one level if its grid side is at
                           most LP_SINGLE_LEVEL_MAX_GRID, else two. */
  double upsampling;    /* grid upsampling sigma (g >= sigma (2K+1)): 0 = the
                           default (FP64 1.5, FP32 2), else 1.25 .. 3; the
                           kernel width follows from tol and sigma (LP_ERR_ARG
                           when it would exceed 16) */
  int autotune;         /* LP_AUTOTUNE_BINS: the first lp_volume that binds
                           sources times the binned volume spread for three
                           bin sides (FP64 16/24/32, FP32 16/32/48
                           near-history cells) on those sources and keeps the
                           fastest (it synchronises the plan's stream once).
                           LP_AUTOTUNE_FULL: before that, the same lp_volume
                           builds a plan for each upsampling sigma in {1.25,
                           1.5, 2} with one and with two history levels (the
                           trade-off of Sec. 3's one-level remark), each with
                           the kernel width its sigma needs for tol, binds the
                           sources and unit layer densities, times one V, S, D
                           evaluation at the sources (median of three), and
                           keeps the fastest in place of the plan's grids --
                           the upsampling and levels fields are then only the
                           starting point.  Every configuration meets tol, so
                           the choice changes speed, not accuracy beyond
                           rounding.  0: no tuning. */
  int64_t max_device_bytes; /* device-memory budget of the plan (0: none): an
                           allocation that would take the plan's device
                           footprint (lp_plan_info's device bytes) beyond it
                           fails with LP_ERR_NOMEM before cudaMalloc is
                           called, whether in lp_plan, lp_volume or
                           lp_execute; a server uses it to keep a plan within
                           the memory it admitted the plan for */
} lp_domain;

/* Create a plan: chooses the near/far-history grids (Sec. 3: delta_2 =
 * 32 delta_1, Fourier truncation k e^{-k^2 delta} < tol, periods that exclude
 * aliasing for the box), builds the multiplier tables and the boundary
 * search structures, and allocates all device workspace.
 *   delta: delta_1 (> 0); the paper's choice is 3 * mean(w) (Sec. 6).
 *   tol:   target accuracy of the smooth part, 1e-3 .. 1e-13 (FP32: >= 1e-6).
 * On success *plan owns all workspace until lp_destroy. */
lp_status lp_plan(const lp_domain* domain, double delta, double tol, lp_plan_t* plan);

/* Bind volume sources: n nodes xy[n][2], quadrature weights w[n] and density
 * f[n] (Sec. 3, input of the history algorithm: strengths f_j w_j).  The plan
 * copies what it needs; the caller's buffers may be reused once the stream
 * has passed this call.  n may be 0. */
lp_status lp_volume(lp_plan_t plan, int64_t n, const double* xy, const double* w, const double* f);

/* Bind the single-layer density sigma at the boundary nodes (strengths
 * sigma_b w_b).  sigma: [n_panels*panel_order]. */
lp_status lp_single_layer(lp_plan_t plan, const double* sigma);

/* Bind the double-layer density mu at the boundary nodes (dipole strengths
 * mu_b w_b nu_b).  mu: [n_panels*panel_order]. */
lp_status lp_double_layer(lp_plan_t plan, const double* mu);

/* Evaluate at n_t targets t_xy[n_t][2]:
 *   V[i] = V[f](t_i)  (requires lp_volume and f_jet)
 *   S[i] = S[sigma](t_i) (requires lp_single_layer)
 *   D[i] = D[mu](t_i) (requires lp_double_layer)
 * Any of V, S, D may be NULL (not requested).  f_jet[n_t][6] holds
 * (f, f_x, f_y, f_xx, f_xy, f_yy) at each target (zero outside Omega); it
 * feeds the volume expansion of Sec. 4 and may be NULL when V is NULL.
 * Targets may coincide with sources or lie on the boundary (classified as
 * on-surface when within 1e-12 * box side of it).  Asynchronous on the plan's
 * stream; call lp_sync for completion and device-side status. */
lp_status lp_execute(lp_plan_t plan, int64_t n_t, const double* t_xy, const double* f_jet,
                     double* V, double* S, double* D);

/* lp_execute without any allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc at evaluation time -- code running
 * while another allocator has reserved the device's memory, loops that must
 * not take the implicit device synchronisation cudaMalloc/cudaFree can
 * cause, or hosts where allocation after start-up is forbidden.  Such a
 * caller creates the plan and binds sources and densities during set-up;
 * this call then runs the same kernels as lp_execute on the same data, but
 * it stages nothing (every pointer must be device memory, else LP_ERR_ARG)
 * and keeps its per-call scratch -- the list of targets near the boundary
 * -- in a static device array sized for at most 2,097,152 targets (16 MiB
 * per device, held until the process exits); larger n_t is rejected with
 * LP_ERR_ARG before anything is launched.  The call must be made with the
 * plan's device current (LP_ERR_ARG otherwise: the array is per device).
 * The first call on each device looks up that array's device address (with
 * the device current); the CUDA driver loads modules lazily, so that lookup
 * is when it loads the module holding the array and takes the array's 16
 * MiB.  Make the first call on a device during set-up, before any stream
 * capture and before the point from which nothing may be allocated.  All calls share the one array: calls
 * whose work overlaps on the GPU (two plans on different streams, say) race,
 * so serialise them.  No cudaMalloc, cudaFree or allocating library routine
 * is called. */
lp_status lp_execute_noalloc(lp_plan_t plan, int64_t n_t, const double* t_xy, const double* f_jet,
                             double* V, double* S, double* D);

/* lp_execute replayed from a CUDA graph (same arguments and results): the
 * first call for an argument signature -- the pointers, n_t, the bound
 * source count, and no reallocation or bin change in the plan since --
 * runs lp_execute and captures the same call into a graph; later calls with
 * that signature launch the graph (one launch for the whole chain).  Bound
 * densities and sources may change between calls (their buffers are
 * reused).  Device pointers only (LP_ERR_ARG otherwise).  Plans whose
 * transforms run on cuFFT run lp_execute directly.  The replay is ordered
 * after the work already queued on the plan's stream, and later work on
 * that stream after the replay. */
lp_status lp_execute_graph(lp_plan_t plan, int64_t n_t, const double* t_xy, const double* f_jet, double* V,
                           double* S, double* D);

/* Batched evaluation of a wave of independent problems (many uneven
 * problems, one launch per kernel per wave).  A batch owns only the
 * wave's argument records, candidate list and worker streams; the member
 * plans are ordinary plans (each bound with lp_volume / lp_single_layer /
 * lp_double_layer on a stream the batch stream is ordered after, e.g. the
 * same stream).
 *   lp_batch_create(stream, &b): the batch's work runs on stream.
 *   lp_batch_execute(b, n, plans, n_t, t_xy, f_jet, V, S, D): evaluates, for
 *     every member i, exactly what lp_execute(plans[i], n_t[i], t_xy[i],
 *     f_jet[i], V[i], S[i], D[i]) evaluates (Sec. 3 and Sec. 4 per problem),
 *     with one zeroing launch, one point-parallel spread launch (boundary
 *     nodes of FP32 members, volume nodes of plans without bins), one launch
 *     for the binned volume spreads of every member and level, one for the
 *     binned layer spreads of FP64 members (their boundary nodes sorted into
 *     the bins at plan time), one interpolation launch
 *     per arithmetic (df64, and the cuFFT path's), and one local classify +
 *     near launch for the whole wave; each member's transform chain is
 *     issued on one of 8 worker streams that fork from the batch stream
 *     after the spreads and join it before the interpolation (plans on
 *     cuFFT: on the batch stream, with one multiplier launch for them all).
 *     Arrays have n entries; V, S, D (and their entries) may be NULL; all
 *     buffers must be device memory (LP_ERR_ARG otherwise); all members must
 *     share precision and kernel width (one kernel shape per wave) and be
 *     distinct.  Asynchronous: lp_batch_sync waits, lp_sync(member) returns
 *     that member's device status.
 *   lp_batch_stage_times(b, out[9]): {zeroing+record copy, spread, forward
 *     FFTs, multiplier, inverse FFTs, interpolation, local, total} in ms of
 *     the last wave, and the launches issued so far.  With the library's
 *     FFT chain the transforms are timed as forward FFTs. */
lp_status lp_batch_create(void* stream, lp_batch_t* batch);
lp_status lp_batch_execute(lp_batch_t batch, int n, const lp_plan_t* plans, const int64_t* n_t,
                           const double* const* t_xy, const double* const* f_jet, double* const* V,
                           double* const* S, double* const* D);
lp_status lp_batch_sync(lp_batch_t batch);
lp_status lp_batch_stage_times(lp_batch_t batch, float* out);
lp_status lp_batch_destroy(lp_batch_t batch);

/* Interior Dirichlet problem (Sec. 5): with u = V[f] + D[mu] in the domain,
 * solve -mu/2 + D[mu] = g - V[f] at the plan's boundary nodes
 * (eq. dir_inteq) by restarted GMRES, D applied by this library's evaluator at
 * the boundary nodes (on-surface targets; refined when the plan refines).
 *   g:        [n_b] boundary values at the nodes given to lp_plan
 *             (host or device).
 *   f_jet_b:  [n_b][6] f-jet at the boundary nodes, or NULL for f = 0; with it
 *             the sources bound by lp_volume give V[f] at the nodes.
 *   mu:       [n_b] out, the density (host or device).
 *   tol:      relative residual |b - A mu| / |b| to reach.
 *   max_iter: total GMRES iterations (each one D evaluation); restart: Krylov
 *             dimension per cycle, 1..64 (0: 30).
 *   iterations, residual: out (host; may be NULL): iterations taken and the
 *             true relative residual of the returned mu (one more D
 *             evaluation), which the caller compares with tol.
 * On return the plan's double-layer density is mu (lp_execute then gives
 * D[mu] anywhere).  LP_ERR_STATE if the plan has no boundary, or f_jet_b is
 * given without lp_volume.  Synchronises the plan's stream.  FP32 plans
 * stall near 1e-4 on large boundaries (single-precision D, summed with
 * atomics in varying order). */
lp_status lp_solve_dirichlet(lp_plan_t plan, const double* g, const double* f_jet_b, double* mu, double tol,
                             int max_iter, int restart, int* iterations, double* residual);

/* Interior Neumann problem (Sec. 5): for -lap u = f in the domain and
 * du/dnu = g on the boundary (outward normal), Green's representation
 * u = V[f] + S[g] - D[u] gives u/2 + D[u] = V[f] + S[g] at the boundary
 * nodes, solved by restarted GMRES like lp_solve_dirichlet.  Constants are in
 * the null space (D[1] = -1/2 on the boundary); the operator carries the
 * rank-one term (sum_i w_i u_i / |Gamma|) 1 (w the boundary weights), so the
 * returned u has zero weighted boundary mean.  The data should satisfy the
 * compatibility condition int f + int g = 0.
 *   g:        [n_b] normal derivative at the boundary nodes (host or device);
 *   f_jet_b, tol, max_iter, restart, iterations, residual: as for
 *             lp_solve_dirichlet;
 *   u:        [n_b] out, the boundary values (host or device).
 * On return the plan's single-layer density is g and its double-layer
 * density u, so lp_execute with V, S and D gives u = V + S - D anywhere in
 * the domain. */
lp_status lp_solve_neumann(lp_plan_t plan, const double* g, const double* f_jet_b, double* u, double tol,
                           int max_iter, int restart, int* iterations, double* residual);

/* Source sharding across GPUs with one exchange step (one process per GPU).
 * Every rank holds a plan of the same domain, delta, tol, precision and
 * options -- hence the same grids -- binds its own share of the volume nodes
 * with lp_volume and the full layer densities with lp_single_layer /
 * lp_double_layer (the local part of its targets needs them), and then:
 *   lp_spread(plan, outputs, spread_layers): zero the grids of the outputs
 *     (bit mask: 1 V, 2 S, 4 D) and spread the bound volume nodes into them,
 *     and the boundary nodes too when spread_layers is nonzero (on exactly
 *     one rank, so that the sum counts them once) -- Sec. 3, steps 2-3;
 *   lp_grid_buffers(plan, ptrs, bytes, dtypes, n): the device buffers whose
 *     elementwise sum over the ranks (an all-reduce) makes every rank's grids
 *     those of all the sources: per history level the spread channels (V;
 *     S; D as two dipole channels) in the plan's padded layout, dtype 0 for
 *     double, 1 for float; and, last, two doubles of zero-mode strength sums
 *     (used by FP32 plans).  *n: in, the capacity of the arrays; out, the
 *     count (LP_ERR_ARG with *n set when the capacity is short; at most 9).
 *     The buffers belong to the plan; reduce them in place on the plan's
 *     stream (or after lp_sync).  LP_ERR_STATE before lp_spread;
 *   lp_finish(plan, n_t, t_xy, f_jet, V, S, D): transforms, multiplier,
 *     interpolation and local part from the grids as they stand (step 4 and
 *     Sec. 4), for this rank's targets; outputs must be among the spread
 *     ones (LP_ERR_STATE otherwise); device pointers only (LP_ERR_ARG).
 * Without the all-reduce, lp_spread + lp_finish on one plan is lp_execute.
 * The spread is linear in the sources, so the sum of the ranks' grids is the
 * grid of all of them; only the volume and boundary spreads are sharded. */
lp_status lp_spread(lp_plan_t plan, int outputs, int spread_layers);
lp_status lp_grid_buffers(lp_plan_t plan, void** ptrs, int64_t* bytes, int* dtypes, int* n);
lp_status lp_finish(lp_plan_t plan, int64_t n_t, const double* t_xy, const double* f_jet, double* V, double* S,
                    double* D);

/* f-jets at targets estimated from the bound node values, for callers that
 * have f only at the quadrature nodes (the paper computes the jets of
 * Sec. 4's volume expansion analytically, Sec. 6.1).  At each target t_xy[i]:
 * weighted least squares of the nodes' f over the nodes within
 * rho = sqrt(3 delta_1) (three mean node spacings for the paper's delta_1 =
 * 3 x mean weight), weights (1 - r^2/rho^2)^2, on a quadratic in the offset
 * when at least 10 nodes are that close, a linear function with 4 to 9, the
 * weighted mean with 1 to 3, and zero with none (targets away from every
 * node, e.g. outside the domain); at a target within 1e-12 of the box side
 * of a node, the value is that node's f.  The normal equations are summed
 * in single precision and solved in double.
 *   f_jet: [n_t][6] out, (f, f_x, f_y, f_xx, f_xy, f_yy), ready for
 *          lp_execute.
 * Requires lp_volume (LP_ERR_STATE); host or device pointers.  Allocates
 * scratch for the call (a cell index of the nodes) and frees it before
 * returning; synchronises the plan's stream.  LP_ERR_UNSUPPORTED when the
 * box holds more than 6.4e7 cells of side rho. */
lp_status lp_volume_jets(lp_plan_t plan, int64_t n_t, const double* t_xy, double* f_jet);

/* Wait for the plan's stream; return and clear the device status word. */
lp_status lp_sync(lp_plan_t plan);

/* lp_sync with a bounded wait: polls the plan's stream for at most
 * timeout_ms milliseconds of host time (timeout_ms < 0: wait without bound,
 * as lp_sync).  Returns LP_ERR_TIMEOUT if the work queued on the plan's
 * stream has not completed by then -- the work keeps running, and the device
 * status word is left for a later lp_sync / lp_sync_timeout -- otherwise what
 * lp_sync returns. */
lp_status lp_sync_timeout(lp_plan_t plan, double timeout_ms);

/* Release all plan resources (synchronises the plan's stream first). */
lp_status lp_destroy(lp_plan_t plan);

/* Static description of a status code. */
const char* lp_status_string(lp_status status);

/* Plan parameters, for diagnostics and benchmarks:
 * out[0..30] = {delta_1, delta_2, kernel width w, beta, g_NH, K_NH, P_NH, g_FH, K_FH,
 *               P_FH, L_FH, band 12 sqrt(delta_1), node-gap margin, device bytes,
 *               precision, order, kernels launched by this plan so far,
 *               max error of the kernel's polynomial form, its coefficient count,
 *               realised upsampling min g/(2K+1), 1 if the transforms run in
 *               the library's own FFT kernels (for FP64 plans in double-float
 *               arithmetic, with the double-float interpolation), 0 for cuFFT,
 *               1 if volume sources are spread through bins, bin side in
 *               near-history cells, dyadic refinement levels, largest error
 *               of the refinement's kernel tables, refinement subnodes,
 *               history levels in use (2 or 1), upsampling sigma, the
 *               autotuner's spread times in ms of its three bin sides
 *               (0 if it has not run, -1 for a side that does not fit), and
 *               the grid autotuner's evaluation times in ms of sigma 1.25,
 *               1.5, 2 with one and two levels, in that order (0 if it has
 *               not run, -1 for a configuration it could not build)}; the
 *               near-history entries are 0 for single-level plans.
 *               out must hold 37 doubles. */
lp_status lp_plan_info(lp_plan_t plan, double* out);

/* Per-stage device times of the last lp_execute in milliseconds (CUDA events
 * on the plan's stream; valid after lp_sync): out[0..10] = {spread, forward
 * FFT, multiplier, inverse FFT, interpolation, local, total, copies, grid
 * zeroing, spread of the volume sources alone (part of out[0]), difference
 * sums of the dyadic refinement (0 without refinement)}.  With the
 * double-float transforms, "forward FFT" is the row transforms, "multiplier"
 * the fused column pass (forward transform, multiplier, inverse transform)
 * and "inverse FFT" the inverse row transforms.  out must hold 11 floats. */
lp_status lp_stage_times(lp_plan_t plan, float* out);

#ifdef __cplusplus
}
#endif

#endif /* LP_H_ */
