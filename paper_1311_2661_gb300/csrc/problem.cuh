// Internal, colour-ordered device layout of one LP and the kernels' views of it.
#pragma once
#include <memory>
#include <vector>

#include "common.cuh"

namespace thetis {

enum ProbKind { KIND_GENERAL = 0, KIND_VC = 1, KIND_IS = 2, KIND_MC = 3, KIND_BATCH = 4, KIND_SC = 5, KIND_MAP = 6 };

// Classes of coordinate units inside one colour.  Units of a colour are stored
// class by class, so that every class is a contiguous range of units and of
// internal columns.  Singleton columns with at most 32 non-zeros form the
// small classes S32 ... S2 by their row-slot width W (the smallest power of two
// >= nnz, at least 2); their row ids are also kept in ELL form.
enum UnitClass {
  UC_BLOCK = 0, UC_HUGE = 1, UC_LARGE = 2, UC_MED = 3,
  UC_S32 = 4, UC_S16 = 5, UC_S8 = 6, UC_S4 = 7, UC_S2 = 8,
  UC_COUNT = 9
};
// non-zero thresholds of the singleton classes (more than T_HUGE: HUGE, ...)
constexpr int64_t T_HUGE = 1024, T_LARGE = 128, T_MED = 32;
__host__ __device__ constexpr bool is_small_class(int cls) { return cls >= UC_S32 && cls <= UC_S2; }
__host__ __device__ constexpr int small_width(int cls) { return 32 >> (cls - UC_S32); }
// ELL form of a small class of width W: column p of the segment keeps its row
// slot q at e0 + (p / 32) * 32 * W + q * 32 + p % 32 (32-column panels, slot
// major), unused slots hold ELL_PAD
constexpr uint32_t ELL_PAD = 0xffffffffu;

struct Seg {
  int cls;        // UnitClass
  int64_t u0, u1; // units [u0, u1) (positions in colour order)
  int64_t c0;     // first internal column of unit u0
  int32_t len;    // columns per unit (k for blocks, 1 otherwise)
  int64_t e0 = 0; // small classes: first ELL slot of the segment
};

struct ColorPlan {
  std::vector<Seg> segs;   // non-empty classes of this colour
  int64_t srow0 = 0, srow1 = 0; // internal rows whose slack has this colour
  int64_t nnz = 0;          // structural non-zeros of this colour
};

// Original-order input held on the device while the layout is built.
struct RawLP {
  int64_t M = 0, Ns = 0, nnz = 0;
  int64_t* colptr = nullptr;   // Ns+1
  int32_t* rowidx = nullptr;   // nnz
  float* val = nullptr;        // nnz or null (+1)
  float *b = nullptr, *c = nullptr, *lo = nullptr, *hi = nullptr;
  uint8_t* row_kind = nullptr;
  int32_t block_k = 1;
  int64_t n_blocks = 0;
  int64_t* block_first = nullptr;
  // uniform-bounds hint (set by the graph builders)
  bool bounds_uniform = false;
  float lo_u = 0.f, hi_u = 1.f;
  int slack_sign_uniform = 0;  // -1 / +1 if every row has a slack of that sign
  // optional ids hashed into the colouring priority instead of the unit id
  // (a batch of instances passes instance-local ids, so every instance is
  // coloured exactly as it would be alone)
  const uint32_t* prio_col = nullptr;  // per structural column
  const uint32_t* prio_row = nullptr;  // per row (for its slack)
};

struct Problem {
  explicit Problem(cudaStream_t s) : stream(s), mem(s) {}
  cudaStream_t stream;
  Arena mem;  // lives as long as the handle

  int kind = KIND_GENERAL;
  int64_t M = 0;      // rows
  int64_t Ns = 0;     // structural columns (original)
  int64_t nnz = 0;    // structural non-zeros
  int32_t k = 1;      // simplex block size
  bool has_val = false;
  bool bounds_uniform = false;
  float lo_u = 0.f, hi_u = 1.f;
  int slack_sign_uniform = 0;
  bool blk_shared = false;  // some simplex block has two columns in one row

  // batch meta (thetis_build_batch): instance t owns vertices [bnoff[t], bnoff[t+1])
  // and edges [beoff[t], beoff[t+1]) of the union
  int64_t nbatch = 0;
  int64_t *bnoff = nullptr, *beoff = nullptr;
  uint8_t* bkind = nullptr;
  std::vector<uint8_t> h_bkind;
  std::vector<int64_t> h_bnoff, h_beoff;
  // per-instance convergence: the instance of every internal column and row;
  // an instance whose rho reaches tol at a check is frozen (no longer swept),
  // so it ends exactly where a solve of it alone stops
  int32_t* binst_col = nullptr;        // Ns
  int32_t* binst_row = nullptr;        // M
  uint8_t* bfrozen = nullptr;          // nbatch
  unsigned long long* brho = nullptr;  // nbatch: rho of the last check (FP64 bits, >= 0)
  int32_t* bmaxdeg = nullptr;          // nbatch: longest column of every instance
  float* blfix = nullptr;              // nbatch: step rule 1's L_max of every instance (for blfix_beta)
  double blfix_beta = 0.0;
  std::vector<uint8_t> h_bfrozen;
  std::vector<int32_t> h_bepochs;      // epochs each instance ran in the last solve
  std::vector<double> h_brho;          // its rho when it stopped
  std::vector<double> h_bdone;         // ms from the start of the solve to its stop
  std::vector<double> h_bstart;        // instance engine: ms from the start of the solve to its CTA's start
  std::vector<int32_t> h_bctas;        // instance engine: CTAs of the CTA / cluster that solved it (0: union sweep)
  double batch_check_ms = 0.0;         // union sweep: time of the current check since the solve started
  // active tiles: per colour, the sweep tiles holding a unit of an unfinished
  // instance (built for launch shape act_g; recomputed when instances stop)
  int32_t* act_tiles = nullptr;
  int64_t* act_off = nullptr;
  int64_t* act_n = nullptr;
  int64_t* act_cnt = nullptr;     // per flat tile: 1 if active (scan input)
  int64_t* act_pos = nullptr;     // its exclusive scan
  int64_t* tile_start = nullptr;  // per colour: first flat tile (C + 1)
  int64_t tiles_total = 0;
  int act_g = -1;

  // instance-resident engine of batches (inst.cu): every instance's columns,
  // rows and non-zeros in instance-major order ("IML": instance, then colour),
  // built once from the union layout above
  bool iml_built = false;
  int iml_C = 0;                    // colour-table stride (union colours + 1)
  uint32_t* i_col = nullptr;        // Ns: union internal column of IML column k
  uint32_t* i_row = nullptr;        // M: union internal row of IML row k
  uint32_t* i_end = nullptr;        // Ns: end of column k's entries, local to its instance
  uint32_t* i_ent = nullptr;        // 2M: local row of every entry
  uint32_t* i_nb = nullptr;         // 2M: local column of the entry's other endpoint
  uint32_t *i_ru = nullptr, *i_rv = nullptr;  // M: local columns of every row
  int32_t* i_coff = nullptr;        // count * iml_C: first local column of every colour
  int32_t* i_roff = nullptr;        // count * 4 * iml_C: first local slack row of every (rank, colour)
  int32_t* i_qoff = nullptr;        // count * 5: first local row of every cluster rank (and the end)
  uint8_t* i_K = nullptr;           // count: cluster size of every instance (1: one CTA)
  uint32_t* i_vid = nullptr;        // Ns: instance-local vertex id of every IML column
  // rounding inside the instance kernel (thetis_solve_round_batch)
  bool iround_on = false;
  bool iround_done = false;         // the last solve rounded in the kernel
  uint64_t iround_seed = 0;
  int iround_reps = 1;
  uint8_t* i_lab = nullptr;         // Ns: labels by union vertex
  double *i_robj = nullptr, *i_rrep = nullptr;      // count: objective, repair value
  int32_t *i_rbest = nullptr, *i_rstatus = nullptr; // count: winning repetition, status
  float* i_xout = nullptr;          // Ns: final x by union vertex (rounding on)
  float* i_rhoout = nullptr;        // count: rho at the last check
  int* i_done = nullptr;            // count or null: host-mapped completion flags (set by the caller)
  std::vector<uint8_t> h_iK;
  int32_t* i_ncol = nullptr;        // count: colours of the instance
  int32_t* i_cwide = nullptr;       // count * iml_C: first short column (<= 32 entries) of every colour
  int64_t* i_pfirst = nullptr;      // count * iml_C + 1: first ELL panel of every colour
  int64_t* i_pbase = nullptr;       // per panel: first ELL slot
  uint8_t* i_pw = nullptr;          // per panel: slots per column
  uint32_t* i_ell = nullptr;        // ELL slots of the short columns (local rows)
  int64_t i_npanels = 0;
  int64_t i_pcap = 0, i_scap = 0;  // allocated panels / ELL slots
  // cluster instances: rows of a rank in halo-group order and the halo segments
  uint32_t* i_rpos = nullptr;       // M: place of every IML row in its rank's block of r
  uint32_t* i_rrow = nullptr;       // M: the IML row at every place
  int32_t* i_hs = nullptr;          // count * 16 * iml_C: start of segment R(q, A, c) in rank q's block
  int32_t* i_hl = nullptr;          // count * 16 * iml_C: its length
  int32_t* i_hoff = nullptr;        // count * 4 * iml_C * 4: where R(A, q, c) sits in q's halo buffer
  int32_t* i_hH = nullptr;          // count: halo buffer length
  uint8_t* i_hnb = nullptr;         // count: halo buffers (1 or 2)
  std::vector<int32_t> h_iH;        // host copy of i_hH
  std::vector<uint8_t> h_ihnb;      // host copy of i_hnb
  uint8_t* i_xg = nullptr;          // count: 1 when a cluster instance keeps x in global memory
  std::vector<uint8_t> h_ixg;       // host copy of i_xg
  std::vector<uint8_t> h_iKmin;     // count: lowest cluster level an instance may take (2 (K - 2) + x in
                                    // global memory; 6: the spill class)
  int32_t* i_deg = nullptr;         // count: largest column length of the instance
  float *i_c = nullptr, *i_x = nullptr, *i_s = nullptr;  // c, x (Ns) and s (M) in IML order
  float* i_rg = nullptr;            // M: residual rows kept in global memory (instances too large for one CTA)
  bool iml_clusters = true;         // large instances on thread-block clusters (else one CTA + L2)
  bool iml_classes_ok = false;      // launch classes computed for the current iml_clusters
  int32_t* i_ep = nullptr;          // count: epochs the instance ran
  int32_t* i_conv = nullptr;        // count: 1 if it stopped at rho <= tol
  unsigned long long* i_t = nullptr;  // count: [start, done] globaltimer per instance (2 * count)
  int32_t* i_order = nullptr;       // instances grouped by launch class, largest first
  std::vector<int64_t> h_icls_off;  // per class: range of i_order
  std::vector<int64_t> h_icls_smem; // per class: dynamic shared memory per CTA
  std::vector<int32_t> h_iep;       // host copies after a solve
  std::vector<int32_t> h_iconv;
  std::vector<unsigned long long> h_it;
  int iml_G = 0;                    // lanes per column of the instance kernel (1: ELL thread per column; 0: default)
  cudaStream_t i_streams[8] = {};
  cudaEvent_t i_events[10] = {};

  // set cover meta: the sets holding each element, in increasing set id
  // (elements = rows, sets = columns, original order), and f = max frequency
  int64_t* sc_eptr = nullptr;
  int32_t* sc_esets = nullptr;
  int32_t sc_f = 0;

  // pairwise MAP meta: node and edge scores (n*k, m*k*k)
  float* map_tn = nullptr;
  float* map_te = nullptr;

  // graph meta (builders)
  int64_t nv = 0, ne = 0;
  int32_t *eu = nullptr, *ev = nullptr, *term = nullptr;
  float *w = nullptr, *ce = nullptr;

  // units
  int64_t U = 0;        // all units (structural free units then slack units)
  int64_t Us = 0;       // free structural units
  int64_t Nfree = 0;    // free structural columns
  int64_t Nfix = 0;     // fixed structural columns
  int64_t Msl = 0;      // rows with a slack (= slack units)
  int32_t ncolors = 0;
  int64_t free_coords = 0;  // Nfree + Msl
  std::vector<ColorPlan> plan;

  // ELL row ids (and values, if has_val) of the small classes
  uint32_t* ell = nullptr;
  float* ellv = nullptr;
  int64_t ell_size = 0;
  // segment tables for the checks: small segments (start in the flat index of
  // all small columns, first column, first ELL slot, width) and the other
  // singleton segments (start, first column)
  int64_t nss = 0, nsmall = 0, nbs = 0, nbig = 0;
  int64_t *ss_start = nullptr, *ss_c0 = nullptr, *ss_e0 = nullptr;
  int32_t* ss_w = nullptr;
  int64_t *bs_start = nullptr, *bs_c0 = nullptr;

  // internal CSC over internal structural columns [0, Nfree + Nfix)
  int64_t* colptr = nullptr;
  uint32_t* rowidx = nullptr;  // internal row | NEG_BIT
  float* val = nullptr;        // if has_val
  // internal CSR (structural entries only) for the FP64 refresh
  int64_t* rowptr = nullptr;
  uint32_t* colidx = nullptr;  // internal column | NEG_BIT
  float* rval = nullptr;

  // per internal structural column
  float* x = nullptr;
  float* c = nullptr;
  float* lo = nullptr;  // null if bounds_uniform
  float* hi = nullptr;
  float* csq = nullptr; // ||a_j||^2 if has_val (else nnz)
  // per internal row
  float* r = nullptr;
  float* b = nullptr;
  float* s = nullptr;     // slack values, internal rows [0, Msl)
  int8_t* sig = nullptr;  // slack sign per internal row (0: EQ)

  // maps
  uint32_t* col_of_orig = nullptr;  // Ns
  uint32_t* row_of_orig = nullptr;  // M
  uint32_t* orig_of_row = nullptr;  // M
  int32_t* unit_color = nullptr;    // U (original unit numbering)
  uint32_t* unit_of_pos = nullptr;  // Us: original unit id at colour position
  uint32_t* slack_orig = nullptr;   // Msl: original slack index of internal slack row
  int64_t* blk_start = nullptr;     // internal first column of every free simplex block
  int64_t nblk = 0;
  uint8_t* in_block = nullptr;      // per internal column: part of a simplex block

  // solve scratch (allocated once)
  double* r64 = nullptr;      // M
  double* red = nullptr;      // reduction partials
  double* red_out = nullptr;  // final check values
  double* h_red = nullptr;    // pinned host mirror
  float* ctil = nullptr;      // c - A^T ubar (internal order) when ubar given
  float* cs = nullptr;        // slack linear term -sig*ubar when ubar given
  float* ubar_int = nullptr;  // ubar in internal row order
  float* xbar = nullptr;      // Nfree+Nfix, when given
  float* sbar = nullptr;      // Msl, when given
  float* xorig = nullptr;     // rounding scratch: x in vertex order (n*k)
  double lmax_sq = 0.0;       // max ||a_j||^2 over free structural columns
  int64_t max_unit_nnz = 0;

  // persistent sweep (cooperative launch)
  void* d_plan = nullptr;       // per-colour launch descriptors
  int64_t* d_ntiles = nullptr;  // tiles per colour
  unsigned* bar = nullptr;      // grid barrier state
  int* err = nullptr;           // barrier timeout flag
  long long wait_ns = 2000000000LL;  // limit of every bounded grid-barrier wait
  unsigned wait_phantom = 0;    // CTAs the barriers wait for that never arrive (timeout test)
  int sweep_grid = -1;
  // launch shape (set by thetis_autotune): lanes per SMALL unit, CTAs per SM
  int small_g = 8;
  int plan_g = -1;
  int sweep_per_sm = 0;  // 0: as many as fit
  bool force_full = false;  // use the full sweep even where the lean one applies

  // tail colours: the last colours, holding only a few singleton columns each,
  // run as three phases (tail_T = first tail colour, tail_n units in colour
  // order, tail_coff per tail colour); every tail unit's entries are split into
  // rows shared with another tail unit (tptr / trow) and the rest (hptr / hrow)
  int tail_T = -1;            // -1: not built yet; == ncolors: no tail
  int64_t tail_n = 0;
  int tail_ncol = 0;
  int tail_ctas = 0;          // CTAs of the tail colour chain (one per unit)
  int64_t* tail_col = nullptr;
  int64_t* tail_coff = nullptr;
  int64_t *tail_hptr = nullptr, *tail_tptr = nullptr;
  uint32_t *tail_hrow = nullptr, *tail_trow = nullptr;
  float *tail_h = nullptr, *tail_d = nullptr;

  // CUDA graph of one epoch
  cudaGraphExec_t epoch_graph = nullptr;
  int graph_key = -1;
  ~Problem();
};

// build.cu
std::unique_ptr<Problem> build_problem(RawLP& raw, int kind, uint64_t seed, cudaStream_t s,
                                       Arena& tmp);
void build_vc_is_raw(int kind, int64_t n, int64_t m, const int32_t* d_eu, const int32_t* d_ev,
                     const float* d_w, RawLP& raw, Arena& tmp, cudaStream_t s);
void build_mc_raw(int64_t n, int64_t m, const int32_t* d_eu, const int32_t* d_ev,
                  const float* d_ce, int32_t k, const int32_t* d_term, RawLP& raw, Arena& tmp,
                  cudaStream_t s);

// set cover (App. B.1): covering LP of a set system (sets = columns, elements
// = rows, sum_{s holds a} x_s - z_a = 1, 0 <= x <= 1), plus the element lists
void build_sc_raw(int64_t n_elem, int64_t n_sets, int64_t nnz, const int64_t* d_ptr, const int32_t* d_elems,
                  const float* d_cost, RawLP& raw, int64_t*& eptr, int32_t*& esets, int32_t& f, Arena& keep,
                  Arena& tmp, cudaStream_t s);

// pairwise MAP (Sec. 4.1): the local-polytope LP of an MRF with k labels per
// variable (node marginals on simplex blocks, edge marginals in [0, 1],
// marginalisation rows), costs -theta
void build_map_raw(int64_t n, int64_t m, int32_t k, const int32_t* d_eu, const int32_t* d_ev, const float* d_tn,
                   const float* d_te, RawLP& raw, Arena& tmp, cudaStream_t s);

// batch.cu
void build_batch_raw(int64_t count, const uint8_t* d_kind, const int64_t* d_noff, const int64_t* d_eoff, int64_t Nv,
                     int64_t Ne, const int32_t* d_eu, const int32_t* d_ev, const float* d_w, RawLP& raw,
                     int32_t*& geu, int32_t*& gev, bool& mixed, Arena& tmp, cudaStream_t s);
void round_batch(Problem& P, uint64_t seed, int reps, uint8_t* d_labels, std::vector<double>& obj,
                 std::vector<int32_t>& status, std::vector<int32_t>& best_rep, std::vector<double>& repair,
                 std::vector<int64_t>& near);
// per-instance convergence of a batch: index columns / rows by instance (after
// the layout is built), clear the frozen flags at the start of a solve, and
// after each check freeze every instance whose rho <= tol (true: all frozen)
void batch_index(Problem& P);
void batch_begin_solve(Problem& P);
bool batch_after_check(Problem& P, double tol, int epoch);
void batch_end_solve(Problem& P, int epoch);
// the same around an instance-resident solve (inst.cu): clear the frozen flags;
// after the final FP64 check, every instance's epochs, rho and convergence,
// the largest epoch count, whether all converged, and the updates made
void batch_inst_begin(Problem& P);
void batch_inst_end(Problem& P, int& ep_max, bool& all_converged, int64_t& updates);
// (scd.cu) rebuild the active-tile lists from the frozen flags
void batch_active_tiles(Problem& P);
// (inst.cu) instance-resident solve of a batch: every instance in the shared
// memory of one CTA or thread-block cluster, swept colour by colour, checked
// and stopped on its own; returns false when the batch does not fit (then the
// union sweep serves it).  The union iterate (x, s) is read before and
// written after.
bool inst_eligible(Problem& P);
struct SolveArgs;
void inst_solve(Problem& P, const SolveArgs& a, double& sweep_ms);
void inst_release(Problem& P);
// large instances on 2- or 4-CTA clusters (distributed shared memory) or on one
// CTA with the rows beyond its shared memory in L2 (the default)
void inst_set_clusters(Problem& P, bool on);
// launch classes and layout now (before any solve), so callers may read the
// per-instance outputs while a solve runs
void inst_prepare(Problem& P);
// (api.cu) the problem behind a handle
Problem* problem_of(thetis_handle* h);

// scd.cu
struct SolveArgs {
  double beta;
  int32_t epochs;
  double tol;
  int32_t refresh_every;
  int32_t step_rule;
  int32_t mode;
  int32_t async_ctas = 0;  // async mode: CTA cap (0: one per tile)
};
struct CheckOut {
  double rho, obj, infeas, fbeta;
};
void prepare_solve(Problem& P, const float* d_ubar, const float* d_xbar, const float* d_x0);
// batches with step rule 1: the instances' own L_max (before any capture)
void batch_step_rule(Problem& P, const SolveArgs& a);
void run_epoch(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar);
// FP64 refresh of r (unless refresh is false: r is already exact) and the
// check: rho (per instance for batches), and with full also the objective,
// the infeasibility and f_beta (intermediate checks need only rho)
void refresh_and_check(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar, CheckOut& out, bool full = true,
                       bool refresh = true);
void refresh_only(Problem& P);
// Sec. 3.4 multiplier step: ubar <- ubar - beta (A x - b) from the last FP64
// refresh, xbar <- x (slacks included); c - A'ubar and the slack terms follow
void al_update(Problem& P, double beta);
// the multiplier estimate ubar in original row order
void gather_duals(Problem& P, float* out);
void init_iterate(Problem& P);
int sweep_grid(Problem& P);
bool sweep_lean_possible(Problem& P);
// select the tail colours and split their columns' rows (once per problem;
// before any stream capture of an epoch)
void ensure_tail(Problem& P);
void run_sweep(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar, int epochs);
int sweep_error(Problem& P);
void reset_sweep_flags(Problem& P);

// round.cu
struct RoundOut {
  double obj, repair;
  int32_t best_rep;
  int64_t near;
  int32_t valid;
  int status;
};
void round_problem(Problem& P, int kind, uint64_t seed, int reps, uint8_t* d_labels, RoundOut& out);
void gather_x_orig(Problem& P, float* d_out);
// exact validity (1 / 0) and objective of a caller's labels (device memory)
void check_labels(Problem& P, int kind, const uint8_t* d_labels, int& valid, double& obj);

}  // namespace thetis
