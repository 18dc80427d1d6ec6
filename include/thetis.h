/*
 * thetis.h -- C ABI of the GB300 (sm_103a) solver for LP relaxations by
 * projected stochastic coordinate descent on a quadratic penalty, followed by
 * LP rounding ("An Approximate, Efficient LP Solver for LP Rounding",
 * Sridhar et al., arXiv 1311.2661).
 *
 * The problem is the paper's standard form (Sec. 3.1, eq. LP)
 *      min c^T x   s.t.  A x = b,   lo <= x <= hi,
 * where every inequality row (GE / LE) receives one slack column with
 * coefficient -1 / +1 and bounds [0, +inf) (App. C.2 / C.3 slack forms).
 * The solver minimises the regularised penalty of eq. QP (Sec. 3.2)
 *      f(x) = c^T x - ubar^T (Ax-b) + beta/2 ||Ax-b||^2 + 1/(2 beta) ||x-xbar||^2
 * by coordinate steps x_j <- Proj(x_j - grad_j f / L_j) (Algorithm 1, Sec. 3.3),
 * with simplex-constrained blocks stepped and projected as a whole (App. E,
 * multiway cut).
 *
 * Conventions for every call:
 *  - Every call returns a thetis_status; nothing aborts.  On an error the
 *    thread-local thetis_last_error() names the cause.  A CUDA error is
 *    reported as THETIS_E_CUDA after the handle's stream is synchronised.
 *  - Array arguments are plain pointers.  `mem` says where they live:
 *    THETIS_MEM_HOST (pageable or pinned host memory) or THETIS_MEM_DEVICE
 *    (device memory of the current device).  Inputs are deep-copied before
 *    the call returns, so the caller may free them afterwards.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work of
 *    a handle is ordered on that stream.
 *  - A handle is used by one host thread at a time.
 */
#ifndef THETIS_H
#define THETIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  THETIS_OK = 0,
  THETIS_E_INVALID = 1,  /* bad argument, malformed sparse matrix, size overflow */
  THETIS_E_NOMEM = 2,    /* device allocation failed */
  THETIS_E_BUDGET = 3,   /* request exceeds the server's memory budget */
  THETIS_E_CUDA = 4,     /* CUDA runtime or kernel error */
  THETIS_E_TIMEOUT = 5,  /* a bounded device wait ran out */
  THETIS_E_REPAIR = 6,   /* covering repair impossible: eps >= 1 */
  THETIS_PENDING = 7,    /* server request not finished yet */
  THETIS_NOT_CONVERGED = 8 /* informational: epochs ran out before rho <= tol */
} thetis_status;

typedef enum { THETIS_MEM_HOST = 0, THETIS_MEM_DEVICE = 1 } thetis_mem;
typedef enum { THETIS_ROW_EQ = 0, THETIS_ROW_GE = 1, THETIS_ROW_LE = 2 } thetis_row_kind;
typedef enum {
  THETIS_ROUND_VC = 0,      /* vertex cover threshold (Sec. 2) */
  THETIS_ROUND_IS = 1,      /* independent set, Bansal et al. with alterations (App. B.2) */
  THETIS_ROUND_MC = 2,      /* multiway cut, CKR (App. B.3) */
  THETIS_ROUND_SC = 3,      /* set cover, f-threshold (App. B.1) */
  THETIS_ROUND_SC_RAND = 4, /* set cover, randomized rounding + fix-up (App. B.1) */
  THETIS_ROUND_MAP = 5      /* pairwise MAP, node rounding (Sec. 4.1) */
} thetis_round_kind;
typedef enum { THETIS_MODE_COLORED = 0, THETIS_MODE_ASYNC = 1 } thetis_mode;

typedef struct thetis_handle thetis_handle;
typedef struct thetis_server thetis_server;

/*
 * General sparse LP in the standard form of Sec. 3.1 (eq. LP), structural
 * columns only; slacks are appended per GE/LE row.
 *   m, n          rows and structural columns (n >= 1, m >= 0, both < 2^31)
 *   csc_ptr[n+1]  int64 column pointers, csc_ptr[0] = 0, non-decreasing
 *   csc_row[nnz]  int32 row indices in [0, m); no repeated row inside a column
 *   csc_val[nnz]  coefficients, or NULL for all +1
 *   b[m], c[n], lo[n], hi[n]   lo <= hi; lo == hi marks a fixed column
 *   row_kind[m]   thetis_row_kind per row
 *   block_k, n_blocks, block_first[n_blocks]: simplex blocks of block_k
 *                 consecutive columns starting at block_first[t]; each block's
 *                 coordinates stay on the probability simplex (App. E).  A
 *                 block whose lo == hi everywhere is fixed.  block_k = 1 and
 *                 n_blocks = 0 when there are none.
 */
typedef struct {
  int64_t m, n;
  const int64_t* csc_ptr;
  const int32_t* csc_row;
  const float* csc_val;
  const float *b, *c, *lo, *hi;
  const uint8_t* row_kind;
  int32_t block_k;
  int64_t n_blocks;
  const int64_t* block_first;
} thetis_problem_desc;

/* Solve parameters (eq. QP, Algorithm 1).
 *   beta          penalty parameter (> 0)
 *   epochs        maximum epochs; one epoch = one step of every free coordinate
 *   tol           stop once rho <= tol at a check (0: run all epochs)
 *   refresh_every R: every R epochs (and after the last) r = Ax - b is
 *                 recomputed in FP64 and the FP64 checks run
 *   step_rule     0: L_j = beta ||a_j||^2 + 1/beta per coordinate (block: max
 *                 over the block); 1: the global L_max of eq. Lmax
 *   mode          THETIS_MODE_COLORED (colour classes in order: the iterates
 *                 equal a serial sweep in that order) or THETIS_MODE_ASYNC
 *                 (all coordinates at once with atomic residual updates, the
 *                 asynchronous parallel scheme of Sec. 3.4)
 *   ubar[m], xbar[n + n_slack]  eq. QP centres, NULL = 0; xbar lists the
 *                 structural columns then the slacks in row order
 *   x0[n]         structural starting point (NULL: 0 clipped to the bounds,
 *                 barycentre for simplex blocks); slacks start at 0
 *   mem           where ubar / xbar / x0 live
 *   engine        colored mode only: 0 = default: for a single problem one
 *                 persistent cooperative launch per refresh interval with a
 *                 grid barrier between colours (falls back to 1 where
 *                 cooperative launch is unavailable); for a batch of
 *                 thetis_build_batch without ubar / xbar, the instance-resident
 *                 engine (every instance solved, checked and stopped on its own
 *                 by one CTA or thread-block cluster that keeps its residual
 *                 and iterate in shared memory; see thetis_build_batch);
 *                 1 = one launch per colour, replayed as a CUDA graph;
 *                 2 = the persistent sweep of engine 0 for batches too (the
 *                 whole block-diagonal LP swept colour by colour).  All give
 *                 the same iterates up to FP32 summation order (0 and 1
 *                 bit-identical on single problems).
 *   async_ctas    async mode only: at most this many CTAs (256 threads) step
 *                 coordinates at once, each taking tiles in turn (0 = one CTA
 *                 per tile, as many as the GPU runs); the concurrency of the
 *                 asynchronous scheme. */
typedef struct {
  double beta;
  int32_t epochs;
  double tol;
  int32_t refresh_every;
  int32_t step_rule;
  int32_t mode;
  const float* ubar;
  const float* xbar;
  const float* x0;
  int32_t mem;
  int32_t engine;
  int32_t async_ctas;
} thetis_params;

/* Result of a solve; all checks in FP64 on the final iterate.
 *   rho     max over coordinates of |x_j - Proj(x_j - grad_j / L_j)| with the
 *           per-coordinate L_j, r recomputed exactly (the stopping residual)
 *   obj     c^T x;  infeas  ||Ax - b||_inf;  fbeta  f(x) of eq. QP */
typedef struct {
  int32_t epochs_run;
  int32_t converged;
  int32_t ncolors;
  double rho, obj, infeas, fbeta;
  int64_t updates; /* coordinate updates performed (blocks count k) */
  double solve_ms; /* device time of the solve (CUDA events on the handle's stream) */
  double epoch_ms; /* device time inside the epoch sweeps only (no refresh / checks) */
  int32_t launches_per_epoch; /* kernels one epoch launches */
} thetis_solve_info;

/* Result of a rounding.
 *   obj        objective of the integral solution in the problem's own sense
 *              (VC: cover weight, IS: set weight, MC: cut cost)
 *   repair     eps (VC, Lemma 1), alpha (IS, App. C.3) or 0 (MC)
 *   best_rep   repetition that won (ties to the lowest)
 *   near       VC: vertices with |x~ - 1/2| < 1e-4; IS: vertices whose
 *              Bernoulli draw is within 1e-4 of x~ in the winning rep; MC: 0
 *   valid      1 if the exact validity check passed */
typedef struct {
  double obj;
  double repair;
  int32_t best_rep;
  int64_t near;
  int32_t valid;
} thetis_round_info;

/* Library-wide: message of the last failed call on this thread. */
const char* thetis_last_error(void);
/* Library-wide: number of kernels this library has launched so far. */
uint64_t thetis_launch_count(void);

/*
 * thetis_create -- build the standard form of `desc` on the device, colour
 * the column-intersection graph (greedy in the order (nnz desc,
 * splitmix64(seed, unit) desc, unit asc); Jones-Plassmann rounds that give
 * the same colouring as the sequential greedy) and lay the problem out in
 * colour order.  Sec. 3.1 eq. LP with the slack forms of App. C.
 * Errors: THETIS_E_INVALID on malformed input, THETIS_E_NOMEM, THETIS_E_CUDA.
 * *out owns all device state until thetis_destroy.
 */
thetis_status thetis_create(const thetis_problem_desc* desc, int32_t mem, uint64_t seed,
                            void* stream, thetis_handle** out);

/*
 * Graph builders (mem applies to all arrays):
 *  thetis_build_vc: vertex cover LP of Sec. 2 (eq. lp_vertex_cover): min w^T x,
 *    x_u + x_v >= 1 per edge, 0 <= x <= 1.  Row e: x_u + x_v - s_e = 1.
 *  thetis_build_is: independent set as set packing (App. B.2): max w^T x,
 *    x_u + x_v <= 1, 0 <= x <= 1, stored as min -w^T x, row x_u + x_v + s_e = 1.
 *  thetis_build_mc: multiway cut, linearised form of App. B.3: x_v on the
 *    k-simplex, z_{e,i} in [0,1] with cost ce_e/2, rows
 *    z - x_{u,i} + x_{v,i} - s = 0 and z + x_{u,i} - x_{v,i} - s = 0;
 *    terminals[i] is fixed at the unit vector e_i.  2 <= k <= 32.
 *  eu[m], ev[m]: edge endpoints in [0, n), eu != ev, no repeated edge.
 *  w[n]: vertex weights (> 0); ce[m]: edge weights (>= 0).
 */
thetis_status thetis_build_vc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                              const float* w, int32_t mem, uint64_t seed, void* stream,
                              thetis_handle** out);
thetis_status thetis_build_is(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                              const float* w, int32_t mem, uint64_t seed, void* stream,
                              thetis_handle** out);
thetis_status thetis_build_mc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                              const float* ce, int32_t k, const int32_t* terminals, int32_t mem,
                              uint64_t seed, void* stream, thetis_handle** out);

/*
 * thetis_build_sc -- set cover (App. B.1) as the covering LP
 *   min sum_s c_s x_s  s.t.  sum_{s holds a} x_s - z_a = 1 (z_a >= 0) for every
 *   element a,  0 <= x_s <= 1.
 * Sets are the columns, elements the rows.  set_ptr[n_sets + 1] (int64,
 * set_ptr[0] = 0, non-decreasing) and set_elems[set_ptr[n_sets]] (int32,
 * element ids in [0, n_elements), strictly increasing inside a set) list the
 * sets; cost[n_sets] > 0.  Every element must lie in some set (else the LP is
 * infeasible: THETIS_E_INVALID).  Round with THETIS_ROUND_SC (take every set
 * with x~_s >= 1/f, f = the largest number of sets holding one element) or
 * THETIS_ROUND_SC_RAND (best of `reps` randomized roundings, each completed so
 * that it covers); labels_out[n_sets] marks the chosen sets.  Both first apply
 * the covering repair x~ = min(1, x / (1 - eps)), eps = max_a (1 - sum x)_+
 * (App. C.2; THETIS_E_REPAIR if eps >= 1).  Arrays live in `mem`.
 */
thetis_status thetis_build_sc(int64_t n_elements, int64_t n_sets, const int64_t* set_ptr, const int32_t* set_elems,
                              const float* cost, int32_t mem, uint64_t seed, void* stream, thetis_handle** out);

/*
 * thetis_build_map -- MAP inference on a pairwise factor graph (Sec. 4.1) as
 * the local-polytope LP (the relaxation whose rounding the paper takes from
 * Ravikumar et al.): n variables with k labels each (2 <= k <= 32), m pairwise
 * factors eu[e] -- ev[e] (0-based, no loops), scores theta_node[n*k] (row-major
 * by variable) and theta_edge[m*k*k] (factor e, label of eu[e], label of
 * ev[e]).  Columns: node marginals mu_i(a) at i*k + a (one simplex block per
 * variable) then edge marginals mu_e(a, b) at n*k + e*k*k + a*k + b in [0, 1];
 * rows 2*e*k + a: sum_b mu_e(a, b) - mu_u(a) = 0 and 2*e*k + k + b:
 * sum_a mu_e(a, b) - mu_v(b) = 0; costs -theta (the score is maximised).
 * Round with THETIS_ROUND_MAP: labels_out[n] = argmax_a mu_i(a) (ties: lowest
 * label); info.obj = -(score of the labelling).  Arrays live in `mem`.
 */
thetis_status thetis_build_map(int64_t n, int64_t m, int32_t k, const int32_t* eu, const int32_t* ev,
                               const float* theta_node, const float* theta_edge, int32_t mem, uint64_t seed,
                               void* stream, thetis_handle** out);

/* Sizes of a built problem (any pointer may be NULL): rows m, structural
 * columns n, slack columns (one per GE/LE row), free coordinates (what one
 * epoch updates; simplex blocks count k), non-zeros of A including the slack
 * entries, and the number of colours. */
thetis_status thetis_get_sizes(const thetis_handle* h, int64_t* rows, int64_t* struct_cols,
                               int64_t* slack_cols, int64_t* free_coords, int64_t* nnz,
                               int32_t* ncolors);

/*
 * thetis_solve -- coordinate descent on eq. QP (Algorithm 1 re-ordered as a
 * colour-class sweep, or the asynchronous scheme of Sec. 3.4), FP32 iterate
 * and residual, FP64 refresh of r = Ax - b every refresh_every epochs, FP64
 * checks (Def. 2 infeasibility, objective, eq. QP value, projected-gradient
 * step rho).  Continues from the handle's current iterate (set by create, by
 * x0, or left by a previous solve).  Returns THETIS_OK, THETIS_NOT_CONVERGED
 * (valid iterate, tol not reached), or an error.  info may be NULL.
 */
thetis_status thetis_solve(thetis_handle* h, const thetis_params* p, thetis_solve_info* info);

/*
 * thetis_solve_al -- the augmented-Lagrangian outer loop of Sec. 3.4 (a
 * proximal method of multipliers around eq. QP): `outer` times, solve eq. QP
 * at (ubar, xbar, beta) as thetis_solve does (same p: epochs, tol,
 * refresh_every, step_rule, mode, engine), continuing from the current
 * iterate, then ubar <- ubar - beta (A x - b) (A x - b from the FP64 refresh
 * that ended the solve), xbar <- x (slacks included) and beta <- beta *
 * beta_growth.  p->ubar / p->xbar (original row / column order, slacks after
 * the structural columns, p->mem) give the starting multiplier and centre, or
 * zero when NULL; p->x0 as in thetis_solve.  The multiplier estimate after
 * the last update is read with thetis_get_duals.
 *   outer >= 1, beta_growth >= 1 (1 keeps beta); a batch handle is refused.
 *   info: the last inner solve (epochs_run, updates and epoch_ms summed over all);
 *   infeas_out / obj_out / rho_out[outer]: HOST arrays (each may be NULL) with
 *   ||Ax - b||_inf, c'x and rho at the end of every inner solve.
 * Returns the last inner solve's THETIS_OK / THETIS_NOT_CONVERGED, or an error.
 */
thetis_status thetis_solve_al(thetis_handle* h, const thetis_params* p, int32_t outer, double beta_growth,
                              thetis_solve_info* info, double* infeas_out, double* obj_out, double* rho_out);

/*
 * thetis_get_duals -- the multiplier estimate ubar (FP32, original row order,
 * m entries) held by the handle: after thetis_solve_al, the estimate after its
 * last update; after thetis_solve with p->ubar, that ubar.  out_mem says where
 * `out` lives.  THETIS_E_INVALID if the handle holds no multiplier.
 */
thetis_status thetis_get_duals(thetis_handle* h, float* out, int32_t out_mem);

/*
 * thetis_round -- repair + round the current iterate (structural part).
 *  VC: eps = max_e (1 - x_u - x_v)_+, x~ = min(1, x/(1-eps)) (Lemma
 *      lem:infeasible:rounded:vc), label = [x~ >= 1/2] (Sec. 2); reps ignored.
 *      THETIS_E_REPAIR if eps >= 1.
 *  IS: alpha = max_e (x_u + x_v - 1)_+, x~ = x/(1+alpha) (App. C.3), then
 *      Algorithm 2 of App. B.2 with theta = 1/k: pick v iff U < x~_v, drop the
 *      larger-id end of every picked edge; best of `reps` by weight.
 *  MC: CKR region growing (App. B.3) with radius rho ~ U[0,1) and a random
 *      terminal order; best of `reps` by cut cost.
 *  SC / SC_RAND (handles of thetis_build_sc): covering repair, then the
 *      f-threshold or the randomized rounding (see thetis_build_sc).
 *  MAP (handles of thetis_build_map): node rounding; reps ignored.
 * Random draws: U(seed, rep, stream, index) from splitmix64.
 * labels_out[n] (uint8, vertex order): VC/IS membership, MC label in [0,k);
 * for SC one byte per set (chosen), for MAP the label of every variable.
 * out_mem says where labels_out lives.  info may be NULL.
 */
thetis_status thetis_round(thetis_handle* h, int32_t kind, uint64_t seed, int32_t reps,
                           uint8_t* labels_out, int32_t out_mem, thetis_round_info* info);

/*
 * thetis_check_labels -- exact validity and objective of an integral solution
 * given by the caller (the checks every rounding ends with; Sec. 2 for vertex
 * cover, App. B.1-B.3 for set cover, independent set and multiway cut, Sec. 4.1
 * for MAP), e.g. a rounding kept from earlier or produced elsewhere.
 *   kind          the rounding kind of the handle's problem (as for thetis_round)
 *   labels[n]     uint8 in vertex order (VC / IS / SC: 1 = chosen, 0 = not;
 *                 MC / MAP: the label in [0, k)); `mem` says where it lives
 *   valid_out     1 if VC: every edge has a chosen end; IS: no edge has both
 *                 ends chosen; MC: terminal i has label i; SC: every element
 *                 lies in a chosen set; and every label is in range (0/1, or
 *                 < k); else 0.  May be NULL.
 *   obj_out       cover / set weight, cut cost, set cost or MAP energy (FP64);
 *                 NaN when a label is out of range.  May be NULL.
 * THETIS_E_INVALID for a batch or general-LP handle or a kind that does not
 * match the problem.
 */
thetis_status thetis_check_labels(thetis_handle* h, int32_t kind, const uint8_t* labels, int32_t mem,
                                  int32_t* valid_out, double* obj_out);

/*
 * thetis_round_is_static -- the independent-set branch of thetis_round (repair,
 * best-of-reps rounding with alterations, exact validity) for callers that
 * cannot allocate device memory when they round: serving loops that must not
 * block on cudaMalloc / cudaFree (either can stall every stream of the
 * device), and processes whose free device memory is already owned by another
 * allocator.  The paper has no counterpart; this is a deployment variant of the
 * same kernels.
 *   n, m, eu[m], ev[m], w[n]   the graph and vertex weights, as for
 *                              thetis_build_is (DEVICE pointers of the current
 *                              device; endpoints are checked on the device
 *                              before use: out of [0, n) or a loop gives
 *                              THETIS_E_INVALID, as does a host pointer)
 *   x[n]                       the fractional point in vertex order (DEVICE),
 *                              e.g. from thetis_get_x
 *   labels_out[n]              DEVICE output, 1 = in the independent set
 *   info                       HOST output (may be NULL)
 * Scratch: one file-scope device array of 64 MiB, held by every GPU that loads
 * the library until the process exits.  Requires 2*n*reps + 131,616 bytes <=
 * 64 MiB (n * reps <= 33,488,624); larger sizes return THETIS_E_INVALID.
 * Calls no cudaMalloc / cudaFree and no allocating library routine.  It does
 * synchronise `stream` (after the endpoint check, to pick the best repetition,
 * and at the end) and copies a few words to host stack memory.  The first
 * call on a device looks the array up with cudaGetSymbolAddress (once per
 * device): make that first call before any stream capture.  All calls share the
 * array, so calls that overlap on the GPU (different streams, or different
 * threads) race; serialise them.  Same random streams as thetis_round: equal
 * inputs give equal outputs.
 */
thetis_status thetis_round_is_static(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                                     const float* w, const float* x, uint64_t seed, int32_t reps,
                                     uint8_t* labels_out, thetis_round_info* info, void* stream);

/*
 * thetis_autotune -- choose the launch shape of the colour sweep for this
 * problem: the number of lanes that serve one small column (1, 2, 4 or 8; "warps
 * per column") and the CTAs per SM of the persistent sweep (all that fit, 2 or
 * 1; the size of the colour chunk each CTA takes).  For a batch handle served
 * by the instance-resident engine: one of (1 lane, clusters), (1 lane, no
 * clusters), (8 lanes, clusters) (see thetis_set_batch_shape), returned as
 * *small_group_out and *ctas_per_sm_out (1 = clusters).  Every choice is timed over
 * trial_epochs epochs of the real problem (beta and step_rule from p); the
 * iterate is saved before and restored after each trial, so the result of later
 * solves does not depend on tuning.  The choice is cached in the process per
 * problem shape (kind, size, mean column length, colour count) and applied to
 * the handle; later handles of the same shape reuse it without trials.
 * small_group_out / ctas_per_sm_out (0 = all that fit) may be NULL.
 * This is a performance tool with no counterpart in the paper.
 */
thetis_status thetis_autotune(thetis_handle* h, const thetis_params* p, int32_t trial_epochs,
                              int32_t* small_group_out, int32_t* ctas_per_sm_out);
/*
 * thetis_set_wait_limit -- the time limit of every bounded device wait of this
 * handle's persistent colour sweep (the grid barriers between colours; 2000 ms
 * by default).  A wait that runs out ends the launch and the solve returns
 * THETIS_E_TIMEOUT; the handle stays usable (its iterate is then partly swept).
 * missing_ctas > 0 is a test hook for that path: the barriers then wait for
 * that many CTAs beyond the launch, which never arrive, so the first wait runs
 * out after limit_ms.  limit_ms in (0, 600000], missing_ctas in [0, 1024].
 * No counterpart in the paper (failure handling of the deployment).
 */
thetis_status thetis_set_wait_limit(thetis_handle* h, double limit_ms, int32_t missing_ctas);
/*
 * thetis_set_batch_shape -- the launch shape of the instance-resident engine
 * of a batch handle (what thetis_autotune picks for it): lanes_per_column 1
 * (one thread per short column through 32-column ELL panels, one warp per
 * column longer than 32), 4 or 8 (that many lanes per column through the
 * CSR); clusters 0 (an instance too large for one CTA's shared memory keeps
 * x and the rows beyond it in global memory, i.e. L2) or 1 (such instances
 * span a thread-block cluster of 2, 3 or 4 CTAs whose shared memory holds r --
 * and x, unless keeping x in global memory lets fewer CTAs hold r -- the ranks
 * exchanging the rows their short columns share as contiguous halo copies
 * between colours; a cluster's short columns always take one lane each).
 * Every shape gives the same iterates up to FP32 summation order.  THETIS_E_INVALID for other handles or
 * values.  No counterpart in the paper (a launch-shape knob).
 */
thetis_status thetis_set_batch_shape(thetis_handle* h, int32_t lanes_per_column, int32_t clusters);
/* Set the launch shape by hand: small_group in {1, 2, 4, 8}, ctas_per_sm >= 0
 * (0 = all that fit).  THETIS_E_INVALID otherwise. */
thetis_status thetis_set_launch_shape(thetis_handle* h, int32_t small_group, int32_t ctas_per_sm);

/*
 * thetis_build_batch -- `count` independent vertex-cover / independent-set LPs
 * (Sec. 2; App. B.2) as one block-diagonal LP.  Instance t has kind kinds[t]
 * (THETIS_ROUND_VC or THETIS_ROUND_IS), vertices [vertex_offset[t],
 * vertex_offset[t+1]) of w and edges [edge_offset[t], edge_offset[t+1]) of
 * eu/ev, whose endpoints are LOCAL vertex ids in [0, n_t).  vertex_offset and
 * edge_offset have count+1 entries, start at 0 and do not decrease (n_t >= 1).
 * The colouring hashes instance-local ids, so every instance is coloured, swept
 * and rounded exactly as thetis_build_vc / _is + thetis_solve + thetis_round
 * would treat it alone (up to FP32 summation order).  The handle is solved with
 * thetis_solve: one sweep advances every unfinished instance.  tol applies to
 * each instance separately: at every check (every refresh_every epochs) an
 * instance whose own rho <= tol stops -- it is no longer swept -- which is
 * exactly where a solve of it alone stops; the solve ends when every instance
 * has stopped or after `epochs`.  The returned rho is the largest rho any
 * instance stopped at; thetis_batch_info gives each instance's epochs and rho.
 * thetis_get_x returns the concatenated vertex values.  mem applies to every
 * array.
 */
thetis_status thetis_build_batch(int32_t count, const uint8_t* kinds, const int64_t* vertex_offset,
                                 const int64_t* edge_offset, const int32_t* eu, const int32_t* ev,
                                 const float* w, int32_t mem, uint64_t seed, void* stream,
                                 thetis_handle** out);

/*
 * thetis_batch_info -- per-instance outcome of the last thetis_solve of a batch
 * handle: epochs_out[count] (epochs the instance was swept) and rho_out[count]
 * (its residual when it stopped), HOST arrays, each may be NULL.
 * THETIS_E_INVALID for a handle that is not a batch.
 */
thetis_status thetis_batch_info(const thetis_handle* h, int32_t* epochs_out, double* rho_out);

/*
 * thetis_solve_round_batch -- thetis_solve followed by the repair, rounding
 * and exact validity of every instance, with the results of
 * thetis_round_batch (same random streams, same FP64 decisions: VC threshold
 * after the eps repair of Sec. 2; IS best of `reps` after the alpha repair of
 * App. C.3, Algorithm 2 of App. B.2).  With the instance-resident engine
 * every instance is rounded by its own CTA / cluster the moment it stops, so
 * its result is final then (thetis_batch_latency); other engines round the
 * whole batch after the solve.  Arguments as thetis_solve and
 * thetis_round_batch (labels_out[sum n_t] in out_mem; obj_out, status_out,
 * best_rep_out[count] HOST, each may be NULL; info may be NULL).  Returns the
 * solve's status (THETIS_OK / THETIS_NOT_CONVERGED) or an error.
 */
thetis_status thetis_solve_round_batch(thetis_handle* h, const thetis_params* p, uint64_t seed, int32_t reps,
                                       uint8_t* labels_out, int32_t out_mem, double* obj_out, int32_t* status_out,
                                       int32_t* best_rep_out, thetis_solve_info* info);

/*
 * thetis_batch_latency -- per instance, the device time in ms from the start of
 * the last thetis_solve of a batch handle until the instance's result was
 * final: with the instance-resident engine, when its CTA / cluster finished
 * (instances finish independently); with the union sweep (engine 1 / 2), the
 * check at which it stopped.  done_ms_out[count] is a HOST array.
 */
thetis_status thetis_batch_latency(const thetis_handle* h, double* done_ms_out);

/*
 * thetis_batch_placement -- where the last thetis_solve of a batch handle ran
 * every instance.  start_ms_out[count] (HOST, may be NULL): with the
 * instance-resident engine, the device time in ms from the start of the solve
 * until the instance's CTA / cluster began (with thetis_batch_latency, the
 * span it held its SMs); 0 with the union sweep.  ctas_out[count] (HOST, may
 * be NULL): the CTAs of the CTA / thread-block cluster that solved it (1-4;
 * one SM each), 0 with the union sweep.
 */
thetis_status thetis_batch_placement(const thetis_handle* h, double* start_ms_out, int32_t* ctas_out);

/*
 * thetis_round_batch -- repair + rounding of every instance of a batch handle,
 * exactly as thetis_round does for one instance (VC threshold, IS best of `reps`
 * with the instance-local vertex ids in the random streams).
 *   labels_out[sum n_t]   concatenated labels (out_mem: host or device)
 *   obj_out[count], status_out[count], best_rep_out[count]: HOST arrays (each may
 *   be NULL); status 1 = valid, 0 = validity check failed, -1 = VC repair
 *   impossible (eps >= 1).
 */
thetis_status thetis_round_batch(thetis_handle* h, uint64_t seed, int32_t reps, uint8_t* labels_out,
                                 int32_t out_mem, double* obj_out, int32_t* status_out,
                                 int32_t* best_rep_out);

/*
 * Request server with continuous batching (deployment layer; the paper solves
 * one LP at a time).  Worker threads each own a CUDA stream; a free worker
 * takes the smallest queued request (by estimated device bytes; the oldest
 * instead once it has waited 10 s) and every other queued VC / IS request with
 * the same solve parameters and a size within a factor 4 (up to max_batch,
 * within the memory budget) and solves them together through
 * thetis_build_batch, so requests arriving while
 * others run join the next batch and different workers' work overlaps on the
 * GPU.  MC requests are solved one per worker.  Admission: a request is started
 * only while the estimated device bytes of the running requests plus its own
 * stay within hbm_budget_bytes; a request larger than the whole budget is
 * refused at submit time with THETIS_E_BUDGET.
 * Within a batch, tol applies to every member separately: a request stops at
 * the check where its own rho <= tol, the check where it stops when solved
 * alone, and its result equals the result alone up to FP32 summation order.
 */
typedef struct {
  int32_t kind;            /* THETIS_ROUND_VC, THETIS_ROUND_IS or THETIS_ROUND_MC */
  int64_t n, m;            /* vertices, edges */
  const int32_t *eu, *ev;  /* HOST edge endpoints [m], copied at submit */
  const float* w;          /* VC / IS vertex weights [n] */
  const float* ce;         /* MC edge weights [m] */
  int32_t k;               /* MC labels */
  const int32_t* terminals;/* MC terminals [k] */
  double beta;             /* solve parameters as in thetis_params */
  int32_t epochs;
  double tol;
  int32_t refresh_every;
  uint64_t seed;           /* colouring and rounding seed */
  int32_t reps;            /* rounding repetitions (IS, MC) */
} thetis_request;

typedef struct {
  int32_t status;          /* THETIS_OK, THETIS_NOT_CONVERGED or an error of build / solve / round */
  double obj;              /* objective of the rounded solution */
  int32_t valid;           /* exact validity check passed */
  int32_t epochs_run;
  double rho;              /* residual where this request stopped (its own, also in a batch) */
  double queue_ms, service_ms, latency_ms; /* submit->start, start->done, submit->done (host clock) */
  int32_t batch_size;      /* requests solved together with this one */
  char message[160];       /* error text when status is an error, else empty */
} thetis_result;

thetis_status thetis_server_create(size_t hbm_budget_bytes, int32_t workers, int32_t max_batch,
                                   thetis_server** out);
/* Queue a request; *id identifies it.  The arrays are copied before return. */
thetis_status thetis_submit(thetis_server* sv, const thetis_request* req, uint64_t* id);
/* THETIS_PENDING while the request runs; then THETIS_OK with the result, the
 * labels (host, n bytes) and the fractional point (host, n floats; n*k for MC)
 * copied to the non-NULL outputs.  A request's result is returned once. */
thetis_status thetis_poll(thetis_server* sv, uint64_t id, uint8_t* labels_out, float* x_out,
                          thetis_result* out);
thetis_status thetis_server_stats(thetis_server* sv, int64_t* submitted, int64_t* completed,
                                  int64_t* queued, int64_t* in_flight_bytes);
/* Load shedding: at most max_queued requests wait (0 = no limit); a submit
 * beyond it returns THETIS_E_BUDGET ("queue full") at once.  refused_out (may
 * be NULL) receives the number of submits refused so far. */
thetis_status thetis_server_set_queue_limit(thetis_server* sv, int64_t max_queued, int64_t* refused_out);
/* Finishes every queued request, then stops the workers. */
thetis_status thetis_server_destroy(thetis_server* sv);

/* Copy the structural part of the iterate, original column order, as FP32. */
thetis_status thetis_get_x(thetis_handle* h, float* out, int32_t out_mem);
/* Copy the slack part of the iterate (one value per GE/LE row, row order). */
thetis_status thetis_get_slack(thetis_handle* h, float* out, int32_t out_mem);
/* The colour of every coordinate unit (structural units in column order, then
 * slack units in row order); fixed columns have no unit.  out[n_units]. */
thetis_status thetis_get_colors(thetis_handle* h, int32_t* out, int64_t* n_units);
/* Synchronise the handle's stream (surfaces asynchronous errors). */
thetis_status thetis_sync(thetis_handle* h);
thetis_status thetis_destroy(thetis_handle* h);

/*
 * Library-wide, current device: the library allocates its device memory from
 * its own stream-ordered pool, and memory that builds and destroyed handles
 * free stays reserved there for the next build instead of going back to the
 * device (no new mappings per build).  thetis_cache_info reports the pool's
 * reserved and in-use bytes (either pointer may be NULL; 0 and 0 before the
 * first allocation).  thetis_trim_cache gives unused reserve back until at
 * most keep_bytes stay reserved (memory in use is never touched); an
 * allocation that fails also trims the pool once and retries.
 * Errors: THETIS_E_CUDA.
 */
thetis_status thetis_cache_info(uint64_t* reserved_bytes, uint64_t* used_bytes);
thetis_status thetis_trim_cache(uint64_t keep_bytes);

#ifdef __cplusplus
}
#endif

#endif /* THETIS_H */
