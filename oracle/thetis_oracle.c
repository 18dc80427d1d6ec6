/*
 * thetis_oracle.c -- plain, slow, serial FP64 oracle of the SCD + LP-rounding
 * method of "An Approximate, Efficient LP Solver for LP Rounding"
 * (Sridhar et al., arXiv 1311.2661).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference leg may load this code.  It shares no
 * code, header, table or constant generator with the CUDA library: every
 * formula below is written out again from the paper.
 *
 * What it computes, in the paper's order:
 *   1. the standard form  min c^T x  s.t.  Ax = b,  lo <= x <= hi  (Sec. 3.1,
 *      eq. LP), with one slack column per inequality row (App. C.2 covering
 *      form z = max(Ax-b,0); App. C.3 packing form), for vertex cover
 *      (Sec. 2 eq. lp_vertex_cover), independent set (App. B.2 set packing)
 *      and multiway cut (App. B.3, linearised l1 form);
 *   2. a greedy colouring of the column-intersection graph in a fixed total
 *      priority order (not in the paper; it fixes the sweep order);
 *   3. coordinate descent on the quadratic-penalty QP (Sec. 3.2 eq. QP)
 *        f(x) = c^T x - ubar^T(Ax-b) + beta/2 ||Ax-b||^2 + 1/(2 beta)||x-xbar||^2
 *      with the step of Algorithm 1 (x_i <- Proj(x_i - grad_i f / L)), the
 *      gradient being F_beta of App. A (eq. lpb.lcp), L either the global
 *      L_max of eq. Lmax or the per-coordinate beta||a_j||^2 + 1/beta; simplex
 *      blocks (multiway cut, App. E) take one projected step of the whole block
 *      onto the probability simplex;
 *   4. exact FP64 recomputation of r = Ax - b and the checks: objective c^T x,
 *      ||Ax-b||_inf, f_beta(x) and the projected-gradient step length rho;
 *   5. infeasibility repair (Lemma lem:infeasible:rounded:vc and App. C.2 for
 *      covering; App. C.3 packing lemma with the tighter alpha) and rounding:
 *      vertex-cover threshold x >= 1/2 (Sec. 2), Bansal et al. randomized
 *      packing rounding with alterations (App. B.2, Algorithm 2, theta = 1/k),
 *      and CKR region growing for multiway cut (App. B.3), best of R reps
 *      (Sec. 4.2);
 *   6. exact validity and objective of the integral solutions.
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014; public
 * reference implementation by S. Vigna), used as a counter-based generator.
 *
 * Parity pins for each function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ROW_EQ 0
#define ROW_GE 1
#define ROW_LE 2

#define KIND_GENERAL 0
#define KIND_VC 1
#define KIND_IS 2
#define KIND_MC 3

/* ------------------------------------------------------------------------ */
/* splitmix64                                                               */
/* ------------------------------------------------------------------------ */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* i-th output (i = 0, 1, ...) of a splitmix64 generator whose state starts at seed. */
uint64_t or_splitmix64_at(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * SM_GAMMA); }

/* Counter-based stream: three nested splitmix64 draws keyed by (rep, stream, idx). */
uint64_t or_rng_u64(uint64_t seed, uint64_t rep, uint64_t stream, uint64_t idx) {
  uint64_t a = or_splitmix64_at(seed, rep);
  uint64_t b = or_splitmix64_at(a, stream);
  return or_splitmix64_at(b, idx);
}

/* Uniform double in [0,1) from the top 53 bits. */
double or_rng_uniform(uint64_t seed, uint64_t rep, uint64_t stream, uint64_t idx) {
  return (double)(or_rng_u64(seed, rep, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}

#define STREAM_IS_PICK 1
#define STREAM_CKR_RADIUS 2
#define STREAM_CKR_PERM 3
#define STREAM_SC_PICK 4

/* ------------------------------------------------------------------------ */
/* The standard-form LP                                                     */
/* ------------------------------------------------------------------------ */
typedef struct orlp {
  int64_t M;   /* rows */
  int64_t Ns;  /* structural columns */
  int64_t N;   /* all columns: structural then one slack per non-EQ row */
  int64_t *cp; /* CSC, N+1 */
  int64_t *ri;
  double *av;
  int64_t *rp; /* CSR twin, M+1 */
  int64_t *ci;
  double *rv;
  double *b, *c, *lo, *hi;
  int32_t *row_kind;
  int64_t *slack_of_row; /* column index of the row's slack or -1 */
  /* coordinate units: a single free column, or a simplex block of k columns */
  int64_t U;
  int64_t *ustart;
  int32_t *ulen;
  int32_t *usimplex;
  int64_t *unit_of_col; /* -1 for fixed columns */
  /* problem meta used by the rounding step */
  int32_t kind;
  int64_t n, m;
  int32_t k;
  int32_t *eu, *ev;
  double *w;  /* vertex weights (VC, IS) */
  double *ce; /* edge weights (MC) */
  int32_t *term;
} orlp;

static void *xcalloc(size_t n, size_t s) {
  void *p = calloc(n ? n : 1, s);
  return p;
}

void or_free(orlp *P) {
  if (!P) return;
  free(P->cp); free(P->ri); free(P->av);
  free(P->rp); free(P->ci); free(P->rv);
  free(P->b); free(P->c); free(P->lo); free(P->hi);
  free(P->row_kind); free(P->slack_of_row);
  free(P->ustart); free(P->ulen); free(P->usimplex); free(P->unit_of_col);
  free(P->eu); free(P->ev); free(P->w); free(P->ce); free(P->term);
  free(P);
}

int64_t or_num_rows(const orlp *P) { return P->M; }
int64_t or_num_cols(const orlp *P) { return P->N; }
int64_t or_num_struct(const orlp *P) { return P->Ns; }
int64_t or_num_units(const orlp *P) { return P->U; }
int64_t or_nnz(const orlp *P) { return P->cp[P->N]; }

/* Number of free coordinates (what one epoch updates). */
int64_t or_num_free_coords(const orlp *P) {
  int64_t s = 0;
  for (int64_t u = 0; u < P->U; ++u) s += P->ulen[u];
  return s;
}

/*
 * General constructor.  Structural part in CSC (val may be NULL = all +1),
 * bounds per structural column, one slack appended per GE (coefficient -1) or
 * LE (coefficient +1) row, slack bounds [0, +inf), slack cost 0.
 * Simplex blocks: block_first[0..nblocks) are the first columns of blocks of
 * block_k consecutive columns whose coordinates must lie on the probability
 * simplex.  A block (or single column) whose lo == hi everywhere is fixed.
 */
orlp *or_create(int64_t M, int64_t Ns, const int64_t *colptr, const int32_t *rowidx,
                const double *val, const double *b, const double *c, const double *lo,
                const double *hi, const int32_t *row_kind, int32_t block_k,
                int64_t nblocks, const int64_t *block_first) {
  orlp *P = (orlp *)xcalloc(1, sizeof(orlp));
  P->M = M;
  P->Ns = Ns;
  int64_t nslack = 0;
  for (int64_t i = 0; i < M; ++i) nslack += (row_kind[i] != ROW_EQ);
  P->N = Ns + nslack;
  int64_t N = P->N;
  int64_t nnz_s = colptr[Ns];
  int64_t nnz = nnz_s + nslack;
  P->cp = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
  P->ri = (int64_t *)xcalloc(nnz, sizeof(int64_t));
  P->av = (double *)xcalloc(nnz, sizeof(double));
  P->b = (double *)xcalloc(M, sizeof(double));
  P->c = (double *)xcalloc(N, sizeof(double));
  P->lo = (double *)xcalloc(N, sizeof(double));
  P->hi = (double *)xcalloc(N, sizeof(double));
  P->row_kind = (int32_t *)xcalloc(M, sizeof(int32_t));
  P->slack_of_row = (int64_t *)xcalloc(M, sizeof(int64_t));
  for (int64_t j = 0; j <= Ns; ++j) P->cp[j] = colptr[j];
  for (int64_t p = 0; p < nnz_s; ++p) {
    P->ri[p] = rowidx[p];
    P->av[p] = val ? val[p] : 1.0;
  }
  for (int64_t j = 0; j < Ns; ++j) {
    P->c[j] = c[j];
    P->lo[j] = lo[j];
    P->hi[j] = hi[j];
  }
  int64_t col = Ns, p = nnz_s;
  for (int64_t i = 0; i < M; ++i) {
    P->b[i] = b[i];
    P->row_kind[i] = row_kind[i];
    P->slack_of_row[i] = -1;
    if (row_kind[i] == ROW_EQ) continue;
    P->ri[p] = i;
    P->av[p] = (row_kind[i] == ROW_GE) ? -1.0 : 1.0;
    ++p;
    P->c[col] = 0.0;
    P->lo[col] = 0.0;
    P->hi[col] = INFINITY;
    P->slack_of_row[i] = col;
    P->cp[col + 1] = p;
    ++col;
  }
  /* CSR twin by counting sort of the CSC. */
  P->rp = (int64_t *)xcalloc(M + 1, sizeof(int64_t));
  P->ci = (int64_t *)xcalloc(nnz, sizeof(int64_t));
  P->rv = (double *)xcalloc(nnz, sizeof(double));
  for (int64_t q = 0; q < nnz; ++q) P->rp[P->ri[q] + 1]++;
  for (int64_t i = 0; i < M; ++i) P->rp[i + 1] += P->rp[i];
  int64_t *fill = (int64_t *)xcalloc(M, sizeof(int64_t));
  for (int64_t j = 0; j < N; ++j)
    for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q) {
      int64_t i = P->ri[q];
      int64_t at = P->rp[i] + fill[i]++;
      P->ci[at] = j;
      P->rv[at] = P->av[q];
    }
  free(fill);
  /* Units. */
  int32_t *in_block = (int32_t *)xcalloc(N, sizeof(int32_t)); /* 0 none, 1 first, 2 member */
  for (int64_t t = 0; t < nblocks; ++t) {
    in_block[block_first[t]] = 1;
    for (int32_t q = 1; q < block_k; ++q) in_block[block_first[t] + q] = 2;
  }
  P->ustart = (int64_t *)xcalloc(N, sizeof(int64_t));
  P->ulen = (int32_t *)xcalloc(N, sizeof(int32_t));
  P->usimplex = (int32_t *)xcalloc(N, sizeof(int32_t));
  P->unit_of_col = (int64_t *)xcalloc(N, sizeof(int64_t));
  for (int64_t j = 0; j < N; ++j) P->unit_of_col[j] = -1;
  int64_t U = 0;
  for (int64_t j = 0; j < N; ++j) {
    if (in_block[j] == 2) continue;
    int32_t len = (in_block[j] == 1) ? block_k : 1;
    int fixed = 1;
    for (int32_t q = 0; q < len; ++q)
      if (P->lo[j + q] < P->hi[j + q]) fixed = 0;
    if (fixed) continue;
    P->ustart[U] = j;
    P->ulen[U] = len;
    P->usimplex[U] = (in_block[j] == 1);
    for (int32_t q = 0; q < len; ++q) P->unit_of_col[j + q] = U;
    ++U;
  }
  P->U = U;
  free(in_block);
  P->kind = KIND_GENERAL;
  return P;
}

static void copy_graph_meta(orlp *P, int kind, int64_t n, int64_t m, const int32_t *eu,
                            const int32_t *ev) {
  P->kind = kind;
  P->n = n;
  P->m = m;
  P->eu = (int32_t *)xcalloc(m, sizeof(int32_t));
  P->ev = (int32_t *)xcalloc(m, sizeof(int32_t));
  memcpy(P->eu, eu, (size_t)m * sizeof(int32_t));
  memcpy(P->ev, ev, (size_t)m * sizeof(int32_t));
}

/*
 * Vertex cover LP (Sec. 2): min sum_v w_v x_v, x_u + x_v >= 1 per edge,
 * 0 <= x <= 1.  Row e: x_u + x_v - s_e = 1 (GE row, covering slack of App. C.2).
 * Independent set (App. B.2 set packing with the edge as element):
 * max sum w_v x_v  <=>  min -w^T x, row e: x_u + x_v + s_e = 1 (LE row).
 */
static orlp *build_edge_lp(int kind, int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                           const double *w) {
  int64_t *colptr = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    colptr[eu[e] + 1]++;
    colptr[ev[e] + 1]++;
  }
  for (int64_t v = 0; v < n; ++v) colptr[v + 1] += colptr[v];
  int32_t *rowidx = (int32_t *)xcalloc(2 * m, sizeof(int32_t));
  int64_t *fill = (int64_t *)xcalloc(n, sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    rowidx[colptr[eu[e]] + fill[eu[e]]++] = (int32_t)e;
    rowidx[colptr[ev[e]] + fill[ev[e]]++] = (int32_t)e;
  }
  double *b = (double *)xcalloc(m, sizeof(double));
  int32_t *rk = (int32_t *)xcalloc(m, sizeof(int32_t));
  for (int64_t e = 0; e < m; ++e) {
    b[e] = 1.0;
    rk[e] = (kind == KIND_VC) ? ROW_GE : ROW_LE;
  }
  double *c = (double *)xcalloc(n, sizeof(double));
  double *lo = (double *)xcalloc(n, sizeof(double));
  double *hi = (double *)xcalloc(n, sizeof(double));
  for (int64_t v = 0; v < n; ++v) {
    c[v] = (kind == KIND_VC) ? w[v] : -w[v];
    lo[v] = 0.0;
    hi[v] = 1.0;
  }
  orlp *P = or_create(m, n, colptr, rowidx, NULL, b, c, lo, hi, rk, 1, 0, NULL);
  copy_graph_meta(P, kind, n, m, eu, ev);
  P->w = (double *)xcalloc(n, sizeof(double));
  memcpy(P->w, w, (size_t)n * sizeof(double));
  free(colptr); free(rowidx); free(fill); free(b); free(rk); free(c); free(lo); free(hi);
  return P;
}

orlp *or_build_vc(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *w) {
  return build_edge_lp(KIND_VC, n, m, eu, ev, w);
}

orlp *or_build_is(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *w) {
  return build_edge_lp(KIND_IS, n, m, eu, ev, w);
}

/*
 * Multiway cut (App. B.3, linearised form): variables x_{v,i} (v in V, i < k)
 * on the simplex, z_{e,i} in [0,1] with cost c_e/2, and for each edge e=(u,v)
 * and label i the two rows
 *     z_{e,i} - x_{u,i} + x_{v,i} - s+ = 0     (z >= x_u - x_v)
 *     z_{e,i} + x_{u,i} - x_{v,i} - s- = 0     (z >= x_v - x_u)
 * Terminal t_i is fixed at the unit vector e_i (lo = hi), so it keeps label i.
 * Column layout: x_{v,i} at v*k+i, z_{e,i} at n*k + e*k + i.
 * Row layout: 2*(e*k+i) (+ row), 2*(e*k+i)+1 (- row).
 */
orlp *or_build_mc(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *ce,
                  int32_t k, const int32_t *terminals) {
  int64_t Ns = n * k + m * k;
  int64_t M = 2 * m * k;
  int64_t *deg = (int64_t *)xcalloc(n, sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    deg[eu[e]]++;
    deg[ev[e]]++;
  }
  int64_t *colptr = (int64_t *)xcalloc(Ns + 1, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v)
    for (int32_t i = 0; i < k; ++i) colptr[v * k + i + 1] = 2 * deg[v];
  for (int64_t e = 0; e < m; ++e)
    for (int32_t i = 0; i < k; ++i) colptr[n * k + e * k + i + 1] = 2;
  for (int64_t j = 0; j < Ns; ++j) colptr[j + 1] += colptr[j];
  int64_t nnz = colptr[Ns];
  int32_t *rowidx = (int32_t *)xcalloc(nnz, sizeof(int32_t));
  double *val = (double *)xcalloc(nnz, sizeof(double));
  int64_t *fill = (int64_t *)xcalloc(Ns, sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    int64_t u = eu[e], v = ev[e];
    for (int32_t i = 0; i < k; ++i) {
      int64_t rplus = 2 * (e * k + i), rminus = rplus + 1;
      int64_t zc = n * k + e * k + i, xu = u * k + i, xv = v * k + i;
      int64_t q;
      q = colptr[zc] + fill[zc]++; rowidx[q] = (int32_t)rplus; val[q] = 1.0;
      q = colptr[zc] + fill[zc]++; rowidx[q] = (int32_t)rminus; val[q] = 1.0;
      q = colptr[xu] + fill[xu]++; rowidx[q] = (int32_t)rplus; val[q] = -1.0;
      q = colptr[xu] + fill[xu]++; rowidx[q] = (int32_t)rminus; val[q] = 1.0;
      q = colptr[xv] + fill[xv]++; rowidx[q] = (int32_t)rplus; val[q] = 1.0;
      q = colptr[xv] + fill[xv]++; rowidx[q] = (int32_t)rminus; val[q] = -1.0;
    }
  }
  double *b = (double *)xcalloc(M, sizeof(double));
  int32_t *rk = (int32_t *)xcalloc(M, sizeof(int32_t));
  for (int64_t r = 0; r < M; ++r) rk[r] = ROW_GE;
  double *c = (double *)xcalloc(Ns, sizeof(double));
  double *lo = (double *)xcalloc(Ns, sizeof(double));
  double *hi = (double *)xcalloc(Ns, sizeof(double));
  for (int64_t j = 0; j < Ns; ++j) hi[j] = 1.0;
  for (int64_t e = 0; e < m; ++e)
    for (int32_t i = 0; i < k; ++i) c[n * k + e * k + i] = 0.5 * ce[e];
  for (int32_t t = 0; t < k; ++t) {
    int64_t v = terminals[t];
    for (int32_t i = 0; i < k; ++i) {
      lo[v * k + i] = (i == t) ? 1.0 : 0.0;
      hi[v * k + i] = lo[v * k + i];
    }
  }
  int64_t *bf = (int64_t *)xcalloc(n, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) bf[v] = v * k;
  orlp *P = or_create(M, Ns, colptr, rowidx, val, b, c, lo, hi, rk, k, n, bf);
  copy_graph_meta(P, KIND_MC, n, m, eu, ev);
  P->k = k;
  P->ce = (double *)xcalloc(m, sizeof(double));
  memcpy(P->ce, ce, (size_t)m * sizeof(double));
  P->term = (int32_t *)xcalloc(k, sizeof(int32_t));
  memcpy(P->term, terminals, (size_t)k * sizeof(int32_t));
  free(deg); free(colptr); free(rowidx); free(val); free(fill); free(b); free(rk);
  free(c); free(lo); free(hi); free(bf);
  return P;
}

/* Copy out the oracle's standard form (for tests). */
void or_export(const orlp *P, int64_t *cp, int64_t *ri, double *av, double *b, double *c,
               double *lo, double *hi) {
  int64_t nnz = P->cp[P->N];
  if (cp) memcpy(cp, P->cp, (size_t)(P->N + 1) * sizeof(int64_t));
  if (ri) memcpy(ri, P->ri, (size_t)nnz * sizeof(int64_t));
  if (av) memcpy(av, P->av, (size_t)nnz * sizeof(double));
  if (b) memcpy(b, P->b, (size_t)P->M * sizeof(double));
  if (c) memcpy(c, P->c, (size_t)P->N * sizeof(double));
  if (lo) memcpy(lo, P->lo, (size_t)P->N * sizeof(double));
  if (hi) memcpy(hi, P->hi, (size_t)P->N * sizeof(double));
}

void or_export_units(const orlp *P, int64_t *ustart, int32_t *ulen, int32_t *usimplex) {
  if (ustart) memcpy(ustart, P->ustart, (size_t)P->U * sizeof(int64_t));
  if (ulen) memcpy(ulen, P->ulen, (size_t)P->U * sizeof(int32_t));
  if (usimplex) memcpy(usimplex, P->usimplex, (size_t)P->U * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* Colouring of the column-intersection graph                               */
/* ------------------------------------------------------------------------ */
/* Units j and l conflict iff some row holds a column of each.  Units are
 * visited in the total order key(u) = (structural before slack, nnz_u desc,
 * h_u desc, u asc), with h_u the u-th splitmix64 output of `seed`; each takes
 * the smallest colour not held by an already-coloured conflicting unit
 * (sequential greedy colouring). */
static int64_t unit_nnz(const orlp *P, int64_t u) {
  return P->cp[P->ustart[u] + P->ulen[u]] - P->cp[P->ustart[u]];
}

typedef struct {
  int32_t slack;
  int64_t nnz;
  uint64_t h;
  int64_t u;
} prio_key;

static int prio_cmp(const void *a, const void *b) {
  const prio_key *x = (const prio_key *)a, *y = (const prio_key *)b;
  if (x->slack != y->slack) return x->slack < y->slack ? -1 : 1;
  if (x->nnz != y->nnz) return x->nnz > y->nnz ? -1 : 1;
  if (x->h != y->h) return x->h > y->h ? -1 : 1;
  if (x->u != y->u) return x->u < y->u ? -1 : 1;
  return 0;
}

/* Writes the priority order (unit ids, highest first) into order[U]. */
void or_priority_order(const orlp *P, uint64_t seed, int64_t *order) {
  prio_key *keys = (prio_key *)xcalloc(P->U, sizeof(prio_key));
  for (int64_t u = 0; u < P->U; ++u) {
    keys[u].slack = P->ustart[u] >= P->Ns;
    keys[u].nnz = unit_nnz(P, u);
    keys[u].h = or_splitmix64_at(seed, (uint64_t)u);
    keys[u].u = u;
  }
  qsort(keys, (size_t)P->U, sizeof(prio_key), prio_cmp);
  for (int64_t t = 0; t < P->U; ++t) order[t] = keys[t].u;
  free(keys);
}

/* Returns the number of colours; color[u] for every unit. */
int32_t or_color(const orlp *P, uint64_t seed, int32_t *color) {
  int64_t U = P->U;
  int64_t *order = (int64_t *)xcalloc(U, sizeof(int64_t));
  or_priority_order(P, seed, order);
  for (int64_t u = 0; u < U; ++u) color[u] = -1;
  int64_t cap = 64;
  uint8_t *used = (uint8_t *)xcalloc(cap, 1);
  int32_t ncol = 0;
  for (int64_t t = 0; t < U; ++t) {
    int64_t u = order[t];
    /* mark colours of coloured conflicting units */
    int64_t j0 = P->ustart[u], j1 = j0 + P->ulen[u];
    for (int64_t j = j0; j < j1; ++j)
      for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q) {
        int64_t i = P->ri[q];
        for (int64_t s = P->rp[i]; s < P->rp[i + 1]; ++s) {
          int64_t v = P->unit_of_col[P->ci[s]];
          if (v < 0 || v == u || color[v] < 0) continue;
          if (color[v] >= cap) {
            int64_t nc = cap;
            while (nc <= color[v]) nc *= 2;
            used = (uint8_t *)realloc(used, (size_t)nc);
            memset(used + cap, 0, (size_t)(nc - cap));
            cap = nc;
          }
          used[color[v]] = 1;
        }
      }
    int32_t cnew = 0;
    while (cnew < cap && used[cnew]) ++cnew;
    color[u] = cnew;
    if (cnew + 1 > ncol) ncol = cnew + 1;
    if (cnew >= cap - 1) {
      used = (uint8_t *)realloc(used, (size_t)(2 * cap));
      memset(used + cap, 0, (size_t)cap);
      cap *= 2;
    }
    /* clear marks */
    for (int64_t j = j0; j < j1; ++j)
      for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q) {
        int64_t i = P->ri[q];
        for (int64_t s = P->rp[i]; s < P->rp[i + 1]; ++s) {
          int64_t v = P->unit_of_col[P->ci[s]];
          if (v >= 0 && color[v] >= 0 && color[v] < cap) used[color[v]] = 0;
        }
      }
  }
  free(order);
  free(used);
  return ncol;
}

/* ------------------------------------------------------------------------ */
/* Euclidean projection onto the probability simplex                        */
/* ------------------------------------------------------------------------ */
/* Sort-based method (Held, Wolfe & Crowder 1974; as stated by Duchi et al.
 * 2008): sort y descending, find the largest j with
 * u_j - (sum_{i<=j} u_i - 1)/j > 0, shift by theta = (sum_{i<=j} u_i - 1)/j and
 * clip at zero. */
static int dbl_desc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) ? -1 : (x < y) ? 1 : 0;
}

void or_project_simplex(int32_t k, const double *y, double *x) {
  double *u = (double *)xcalloc(k, sizeof(double));
  memcpy(u, y, (size_t)k * sizeof(double));
  qsort(u, (size_t)k, sizeof(double), dbl_desc);
  double cum = 0.0, theta = 0.0;
  for (int32_t j = 0; j < k; ++j) {
    cum += u[j];
    double t = (cum - 1.0) / (double)(j + 1);
    if (u[j] - t > 0.0) theta = t;
  }
  for (int32_t j = 0; j < k; ++j) x[j] = fmax(y[j] - theta, 0.0);
  free(u);
}

/* ------------------------------------------------------------------------ */
/* Coordinate descent on the quadratic-penalty QP                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  double beta;
  int32_t epochs;
  double tol;
  int32_t refresh_every;
  int32_t step_rule; /* 0: per-coordinate L_j, 1: global L_max (eq. Lmax) */
  uint64_t seed;     /* colouring priority seed */
} or_params;

typedef struct {
  int32_t epochs_run;
  int32_t ncolors;
  int32_t converged;
  double rho;
  double obj;
  double infeas;
  double fbeta;
} or_info;

static double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double col_sqnorm(const orlp *P, int64_t j) {
  double s = 0.0;
  for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q) s += P->av[q] * P->av[q];
  return s;
}

/* L of a unit: beta * max_{j in unit} ||a_j||^2 + 1/beta (per-coordinate rule). */
static double unit_L(const orlp *P, int64_t u, double beta) {
  double mx = 0.0;
  for (int32_t q = 0; q < P->ulen[u]; ++q) mx = fmax(mx, col_sqnorm(P, P->ustart[u] + q));
  return beta * mx + 1.0 / beta;
}

/* eq. Lmax: beta * max_i ||A_{:i}||^2 + 1/beta over the free columns. */
static double global_Lmax(const orlp *P, double beta) {
  double mx = 0.0;
  for (int64_t u = 0; u < P->U; ++u)
    for (int32_t q = 0; q < P->ulen[u]; ++q) mx = fmax(mx, col_sqnorm(P, P->ustart[u] + q));
  return beta * mx + 1.0 / beta;
}

/* Partial derivative of f_beta w.r.t. x_j given r = Ax - b (F_beta of App. A). */
static double grad_j(const orlp *P, int64_t j, const double *x, const double *r, double beta,
                     const double *ubar, const double *xbar) {
  double atu = 0.0, atr = 0.0;
  for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q) {
    int64_t i = P->ri[q];
    atr += P->av[q] * r[i];
    if (ubar) atu += P->av[q] * ubar[i];
  }
  double xb = xbar ? xbar[j] : 0.0;
  return P->c[j] - atu + beta * atr + (x[j] - xb) / beta;
}

/* One projected step of unit u; r is updated in place. */
static void update_unit(const orlp *P, int64_t u, double *x, double *r, double beta, double L,
                        const double *ubar, const double *xbar) {
  int64_t j0 = P->ustart[u];
  int32_t len = P->ulen[u];
  if (!P->usimplex[u]) {
    double g = grad_j(P, j0, x, r, beta, ubar, xbar);
    double xn = clip(x[j0] - g / L, P->lo[j0], P->hi[j0]);
    double d = xn - x[j0];
    x[j0] = xn;
    if (d != 0.0)
      for (int64_t q = P->cp[j0]; q < P->cp[j0 + 1]; ++q) r[P->ri[q]] += P->av[q] * d;
    return;
  }
  double *y = (double *)xcalloc(len, sizeof(double));
  double *xn = (double *)xcalloc(len, sizeof(double));
  for (int32_t q = 0; q < len; ++q) y[q] = x[j0 + q] - grad_j(P, j0 + q, x, r, beta, ubar, xbar) / L;
  or_project_simplex(len, y, xn);
  for (int32_t q = 0; q < len; ++q) {
    int64_t j = j0 + q;
    double d = xn[q] - x[j];
    x[j] = xn[q];
    if (d != 0.0)
      for (int64_t s = P->cp[j]; s < P->cp[j + 1]; ++s) r[P->ri[s]] += P->av[s] * d;
  }
  free(y);
  free(xn);
}

/* r = Ax - b, exactly as written (FP64, row by row). */
void or_residual(const orlp *P, const double *x, double *r) {
  for (int64_t i = 0; i < P->M; ++i) {
    double s = 0.0;
    for (int64_t q = P->rp[i]; q < P->rp[i + 1]; ++q) s += P->rv[q] * x[P->ci[q]];
    r[i] = s - P->b[i];
  }
}

/*
 * Checks at x (FP64): rho = max over units of the inf-norm of
 * x_u - Proj(x_u - grad_u / L_u) with the per-coordinate L_u, c^T x,
 * ||Ax - b||_inf and f_beta(x) of eq. QP.
 */
void or_checks(const orlp *P, const double *x, double beta, const double *ubar,
               const double *xbar, or_info *info) {
  double *r = (double *)xcalloc(P->M, sizeof(double));
  or_residual(P, x, r);
  double obj = 0.0, inf = 0.0, rr = 0.0, ur = 0.0, xx = 0.0, rho = 0.0;
  for (int64_t j = 0; j < P->N; ++j) {
    obj += P->c[j] * x[j];
    double xb = xbar ? xbar[j] : 0.0;
    xx += (x[j] - xb) * (x[j] - xb);
  }
  for (int64_t i = 0; i < P->M; ++i) {
    inf = fmax(inf, fabs(r[i]));
    rr += r[i] * r[i];
    if (ubar) ur += ubar[i] * r[i];
  }
  for (int64_t u = 0; u < P->U; ++u) {
    double L = unit_L(P, u, beta);
    int64_t j0 = P->ustart[u];
    if (!P->usimplex[u]) {
      double g = grad_j(P, j0, x, r, beta, ubar, xbar);
      double xn = clip(x[j0] - g / L, P->lo[j0], P->hi[j0]);
      rho = fmax(rho, fabs(xn - x[j0]));
    } else {
      int32_t len = P->ulen[u];
      double *y = (double *)xcalloc(len, sizeof(double));
      double *xn = (double *)xcalloc(len, sizeof(double));
      for (int32_t q = 0; q < len; ++q) y[q] = x[j0 + q] - grad_j(P, j0 + q, x, r, beta, ubar, xbar) / L;
      or_project_simplex(len, y, xn);
      for (int32_t q = 0; q < len; ++q) rho = fmax(rho, fabs(xn[q] - x[j0 + q]));
      free(y);
      free(xn);
    }
  }
  info->rho = rho;
  info->obj = obj;
  info->infeas = inf;
  info->fbeta = obj - ur + 0.5 * beta * rr + 0.5 / beta * xx;
  free(r);
}

/* Initial point: free singletons at clip(0), free simplex blocks at the
 * barycentre 1/k, fixed columns at lo, slacks at 0. */
void or_initial_x(const orlp *P, double *x) {
  for (int64_t j = 0; j < P->N; ++j) x[j] = clip(0.0, P->lo[j], P->hi[j]);
  for (int64_t u = 0; u < P->U; ++u)
    if (P->usimplex[u])
      for (int32_t q = 0; q < P->ulen[u]; ++q) x[P->ustart[u] + q] = 1.0 / P->ulen[u];
}

/*
 * Colour-ordered cyclic sweep: one epoch visits colours 0..C-1 and inside a
 * colour the units in ascending unit index; each unit takes one projected
 * step (Algorithm 1's update, block form for simplex units).  Every
 * refresh_every epochs (and after the last) r is recomputed exactly and the
 * checks are evaluated; the sweep stops once rho <= tol.
 * x must hold the starting point (or_initial_x) on entry; it holds the
 * iterate on exit.  trace (optional, 4 doubles per check: epoch, rho, obj,
 * fbeta) receives every check; ntrace returns how many were written.
 */
int or_solve(const orlp *P, const or_params *prm, const int32_t *color, int32_t ncolors,
             const double *ubar, const double *xbar, double *x, or_info *info, double *trace,
             int32_t *ntrace) {
  double beta = prm->beta;
  int64_t U = P->U;
  /* units grouped by colour, ascending index inside a colour */
  int64_t *cptr = (int64_t *)xcalloc(ncolors + 1, sizeof(int64_t));
  int64_t *clist = (int64_t *)xcalloc(U, sizeof(int64_t));
  for (int64_t u = 0; u < U; ++u) cptr[color[u] + 1]++;
  for (int32_t c = 0; c < ncolors; ++c) cptr[c + 1] += cptr[c];
  int64_t *fill = (int64_t *)xcalloc(ncolors, sizeof(int64_t));
  for (int64_t u = 0; u < U; ++u) clist[cptr[color[u]] + fill[color[u]]++] = u;
  double *L = (double *)xcalloc(U, sizeof(double));
  double Lmax = global_Lmax(P, beta);
  for (int64_t u = 0; u < U; ++u) L[u] = (prm->step_rule == 1) ? Lmax : unit_L(P, u, beta);
  double *r = (double *)xcalloc(P->M, sizeof(double));
  or_residual(P, x, r);
  int32_t nt = 0, ep;
  info->converged = 0;
  info->ncolors = ncolors;
  int R = prm->refresh_every > 0 ? prm->refresh_every : 10;
  for (ep = 0; ep < prm->epochs; ++ep) {
    for (int32_t c = 0; c < ncolors; ++c)
      for (int64_t t = cptr[c]; t < cptr[c + 1]; ++t)
        update_unit(P, clist[t], x, r, beta, L[clist[t]], ubar, xbar);
    if ((ep + 1) % R == 0 || ep + 1 == prm->epochs) {
      or_residual(P, x, r);
      or_checks(P, x, beta, ubar, xbar, info);
      if (trace) {
        trace[4 * nt + 0] = ep + 1;
        trace[4 * nt + 1] = info->rho;
        trace[4 * nt + 2] = info->obj;
        trace[4 * nt + 3] = info->fbeta;
      }
      ++nt;
      if (info->rho <= prm->tol) {
        info->converged = 1;
        ++ep;
        break;
      }
    }
  }
  if (prm->epochs == 0) or_checks(P, x, beta, ubar, xbar, info);
  info->epochs_run = ep;
  if (ntrace) *ntrace = nt;
  free(cptr); free(clist); free(fill); free(L); free(r);
  return 0;
}

/* f_beta after every single unit step of one epoch (monotonicity pin). */
void or_epoch_fbeta_steps(const orlp *P, double beta, int32_t step_rule, const int32_t *color,
                          int32_t ncolors, double *x, double *fsteps) {
  or_params prm = {beta, 1, 0.0, 1, step_rule, 0};
  double Lmax = global_Lmax(P, beta);
  double *r = (double *)xcalloc(P->M, sizeof(double));
  or_residual(P, x, r);
  int64_t t = 0;
  or_info inf;
  for (int32_t c = 0; c < ncolors; ++c)
    for (int64_t u = 0; u < P->U; ++u) {
      if (color[u] != c) continue;
      double L = (prm.step_rule == 1) ? Lmax : unit_L(P, u, beta);
      update_unit(P, u, x, r, beta, L, NULL, NULL);
      or_checks(P, x, beta, NULL, NULL, &inf);
      fsteps[t++] = inf.fbeta;
    }
  free(r);
}

/* ------------------------------------------------------------------------ */
/* Repair and rounding                                                      */
/* ------------------------------------------------------------------------ */
/* Vertex cover: eps = max_e (1 - x_u - x_v)_+ ; x~ = Proj_[0,1](x/(1-eps))
 * (Lemma lem:infeasible:rounded:vc, alpha = eps/q(P) with q(P) = 1);
 * chosen iff x~_v >= 1/2 (Sec. 2).  Returns 0, or 6 if eps >= 1.
 * near counts vertices with |x~_v - 1/2| < band. */
int or_round_vc(const orlp *P, const double *x, uint8_t *label, double *eps_out, double *obj,
                int64_t *near, double band) {
  double eps = 0.0;
  for (int64_t e = 0; e < P->m; ++e) eps = fmax(eps, 1.0 - x[P->eu[e]] - x[P->ev[e]]);
  if (eps_out) *eps_out = eps;
  if (eps >= 1.0) return 6;
  double s = 0.0;
  int64_t nr = 0;
  for (int64_t v = 0; v < P->n; ++v) {
    double xt = fmin(1.0, fmax(0.0, x[v] / (1.0 - eps)));
    label[v] = (xt >= 0.5);
    if (fabs(xt - 0.5) < band) ++nr;
    if (label[v]) s += P->w[v];
  }
  if (obj) *obj = s;
  if (near) *near = nr;
  return 0;
}

/* Independent set, one repetition of Algorithm 2 (App. B.2) with theta = 1/k:
 * pick v with probability x~_v/(k theta) = x~_v, then for every edge with
 * both ends picked mark the end of larger id (elements ordered by
 * (weight desc, id asc); all weights are 1), delete marked vertices. */
void or_round_is_rep(const orlp *P, const double *xt, uint64_t seed, int32_t rep, uint8_t *keep) {
  int64_t n = P->n;
  uint8_t *pick = (uint8_t *)xcalloc(n, 1);
  for (int64_t v = 0; v < n; ++v)
    pick[v] = or_rng_uniform(seed, (uint64_t)rep, STREAM_IS_PICK, (uint64_t)v) < xt[v];
  memcpy(keep, pick, (size_t)n);
  for (int64_t e = 0; e < P->m; ++e) {
    int32_t u = P->eu[e], v = P->ev[e];
    if (pick[u] && pick[v]) keep[u > v ? u : v] = 0;
  }
  free(pick);
}

/* Packing repair (App. C.3, tighter alpha): alpha = max_e (x_u + x_v - 1)_+ ,
 * x~ = x/(1+alpha); best of `reps` repetitions by weight, ties to the lowest rep. */
int or_round_is(const orlp *P, const double *x, uint64_t seed, int32_t reps, uint8_t *label,
                double *alpha_out, double *obj, int32_t *best_rep) {
  double alpha = 0.0;
  for (int64_t e = 0; e < P->m; ++e) alpha = fmax(alpha, x[P->eu[e]] + x[P->ev[e]] - 1.0);
  if (alpha_out) *alpha_out = alpha;
  int64_t n = P->n;
  double *xt = (double *)xcalloc(n, sizeof(double));
  for (int64_t v = 0; v < n; ++v) xt[v] = x[v] / (1.0 + alpha);
  uint8_t *keep = (uint8_t *)xcalloc(n, 1);
  double best = -1.0;
  int32_t br = -1;
  for (int32_t r = 0; r < reps; ++r) {
    or_round_is_rep(P, xt, seed, r, keep);
    double s = 0.0;
    for (int64_t v = 0; v < n; ++v)
      if (keep[v]) s += P->w[v];
    if (s > best) {
      best = s;
      br = r;
      memcpy(label, keep, (size_t)n);
    }
  }
  if (obj) *obj = best;
  if (best_rep) *best_rep = br;
  free(xt);
  free(keep);
  return 0;
}

/* CKR region growing (App. B.3): radius rho ~ U[0,1), a random order sigma of
 * the k terminals (Fisher-Yates, j = floor(U*(i+1)) for i = k-1..1); for
 * t = 0..k-2 every still unlabelled v with x_{v,sigma(t)} >= 1 - rho (the
 * l1/2 ball of radius rho around terminal sigma(t)) takes label sigma(t);
 * the rest take sigma(k-1).  x holds the simplex block of every vertex
 * (x[v*k+i]). */
void or_round_mc_rep(const orlp *P, const double *x, uint64_t seed, int32_t rep, uint8_t *label) {
  int32_t k = P->k;
  double rad = or_rng_uniform(seed, (uint64_t)rep, STREAM_CKR_RADIUS, 0);
  int32_t sigma[256];
  for (int32_t i = 0; i < k; ++i) sigma[i] = i;
  for (int32_t i = k - 1; i >= 1; --i) {
    int32_t j = (int32_t)floor(or_rng_uniform(seed, (uint64_t)rep, STREAM_CKR_PERM, (uint64_t)i) * (double)(i + 1));
    int32_t t = sigma[i];
    sigma[i] = sigma[j];
    sigma[j] = t;
  }
  for (int64_t v = 0; v < P->n; ++v) {
    int32_t lab = sigma[k - 1];
    for (int32_t t = 0; t < k - 1; ++t)
      if (x[v * k + sigma[t]] >= 1.0 - rad) {
        lab = sigma[t];
        break;
      }
    label[v] = (uint8_t)lab;
  }
}

double or_mc_cut_cost(const orlp *P, const uint8_t *label) {
  double s = 0.0;
  for (int64_t e = 0; e < P->m; ++e)
    if (label[P->eu[e]] != label[P->ev[e]]) s += P->ce[e];
  return s;
}

int or_round_mc(const orlp *P, const double *x, uint64_t seed, int32_t reps, uint8_t *label,
                double *obj, int32_t *best_rep) {
  uint8_t *lab = (uint8_t *)xcalloc(P->n, 1);
  double best = INFINITY;
  int32_t br = -1;
  for (int32_t r = 0; r < reps; ++r) {
    or_round_mc_rep(P, x, seed, r, lab);
    double s = or_mc_cut_cost(P, lab);
    if (s < best) {
      best = s;
      br = r;
      memcpy(label, lab, (size_t)P->n);
    }
  }
  if (obj) *obj = best;
  if (best_rep) *best_rep = br;
  free(lab);
  return 0;
}

/* Exact validity of an integral solution: 1 if valid, 0 if not. */
/*
 * Set cover (App. B.1) on a covering LP made by or_create: rows = elements,
 * structural columns = sets (coefficient 1 where the set holds the element),
 * every row sum_{s in a} x_s - z_a = 1 with slack z_a >= 0, costs c.
 * Covering repair (App. C.2 lemma; q(P) = 1 for 0/1 data):
 * eps = max_a (1 - sum_{s in a} x_s)_+ , x~ = min(1, x / (1 - eps)).
 * Returns eps (>= 1: repair impossible).
 */
static double sc_repair(const orlp *P, const double *x, double *xt) {
  double eps = 0.0;
  for (int64_t a = 0; a < P->M; ++a) {
    double cov = 0.0;
    for (int64_t q = P->rp[a]; q < P->rp[a + 1]; ++q)
      if (P->ci[q] < P->Ns) cov += P->rv[q] * x[P->ci[q]];
    eps = fmax(eps, 1.0 - cov);
  }
  for (int64_t j = 0; j < P->Ns; ++j) xt[j] = fmin(1.0, fmax(0.0, x[j] / (1.0 - eps)));
  return eps;
}

/* f = the largest number of sets holding one element */
int32_t or_sc_frequency(const orlp *P) {
  int32_t f = 0;
  for (int64_t a = 0; a < P->M; ++a) {
    int32_t k = 0;
    for (int64_t q = P->rp[a]; q < P->rp[a + 1]; ++q) k += P->ci[q] < P->Ns;
    if (k > f) f = k;
  }
  return f;
}

/* f-threshold rounding (Hochbaum): take every set with x~_s >= 1/f (FP64;
 * |x~_s - 1/f| < band counted as near-threshold). Status 6 if eps >= 1. */
int or_round_sc(const orlp *P, const double *x, uint8_t *label, double *eps_out, double *obj, int64_t *near,
                double band) {
  double *xt = (double *)xcalloc((size_t)P->Ns, sizeof(double));
  double eps = sc_repair(P, x, xt);
  if (eps_out) *eps_out = eps;
  if (eps >= 1.0) {
    free(xt);
    return 6;
  }
  const double thr = 1.0 / (double)or_sc_frequency(P);
  double cost = 0.0;
  int64_t nr = 0;
  for (int64_t j = 0; j < P->Ns; ++j) {
    label[j] = xt[j] >= thr;
    if (fabs(xt[j] - thr) < band) ++nr;
    if (label[j]) cost += P->c[j];
  }
  if (obj) *obj = cost;
  if (near) *near = nr;
  free(xt);
  return 0;
}

/* One repetition of randomized rounding (Srinivasan): set s is taken with
 * probability x~_s; then every element the picks leave uncovered adds its
 * set of largest x~ (ties: lowest set id) -- marks computed on the picks, then
 * added together -- so the result is always a cover. */
void or_round_sc_rand_rep(const orlp *P, const double *xt, uint64_t seed, int32_t rep, uint8_t *take) {
  uint8_t *pick = (uint8_t *)xcalloc((size_t)P->Ns, 1);
  for (int64_t j = 0; j < P->Ns; ++j)
    pick[j] = or_rng_uniform(seed, (uint64_t)rep, STREAM_SC_PICK, (uint64_t)j) < xt[j];
  memcpy(take, pick, (size_t)P->Ns);
  for (int64_t a = 0; a < P->M; ++a) {
    int covered = 0;
    int64_t best = -1;
    for (int64_t q = P->rp[a]; q < P->rp[a + 1]; ++q) {
      const int64_t j = P->ci[q];
      if (j >= P->Ns) continue;
      if (pick[j]) covered = 1;
      if (best < 0 || xt[j] > xt[best] || (xt[j] == xt[best] && j < best)) best = j;
    }
    if (!covered && best >= 0) take[best] = 1;
  }
  free(pick);
}

/* Best of `reps` repetitions by cost, ties to the lowest rep. */
int or_round_sc_rand(const orlp *P, const double *x, uint64_t seed, int32_t reps, uint8_t *label, double *eps_out,
                     double *obj, int32_t *best_rep) {
  double *xt = (double *)xcalloc((size_t)P->Ns, sizeof(double));
  double eps = sc_repair(P, x, xt);
  if (eps_out) *eps_out = eps;
  if (eps >= 1.0) {
    free(xt);
    return 6;
  }
  uint8_t *take = (uint8_t *)xcalloc((size_t)P->Ns, 1);
  double best = INFINITY;
  int32_t br = 0;
  for (int32_t rep = 0; rep < reps; ++rep) {
    or_round_sc_rand_rep(P, xt, seed, rep, take);
    double cost = 0.0;
    for (int64_t j = 0; j < P->Ns; ++j)
      if (take[j]) cost += P->c[j];
    if (cost < best) {
      best = cost;
      br = rep;
      memcpy(label, take, (size_t)P->Ns);
    }
  }
  if (obj) *obj = best;
  if (best_rep) *best_rep = br;
  free(take);
  free(xt);
  return 0;
}

/* every element covered by a taken set */
int or_valid_sc(const orlp *P, const uint8_t *label) {
  for (int64_t a = 0; a < P->M; ++a) {
    int covered = 0;
    for (int64_t q = P->rp[a]; q < P->rp[a + 1]; ++q)
      if (P->ci[q] < P->Ns && label[P->ci[q]]) covered = 1;
    if (!covered) return 0;
  }
  return 1;
}

int or_valid(const orlp *P, const uint8_t *label) {
  if (P->kind == KIND_VC) {
    for (int64_t e = 0; e < P->m; ++e)
      if (!label[P->eu[e]] && !label[P->ev[e]]) return 0;
    return 1;
  }
  if (P->kind == KIND_IS) {
    for (int64_t e = 0; e < P->m; ++e)
      if (label[P->eu[e]] && label[P->ev[e]]) return 0;
    return 1;
  }
  if (P->kind == KIND_MC) {
    for (int64_t v = 0; v < P->n; ++v)
      if (label[v] >= P->k) return 0;
    for (int32_t t = 0; t < P->k; ++t)
      if (label[P->term[t]] != t) return 0;
    return 1;
  }
  return 0;
}
