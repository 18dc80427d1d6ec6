// Coordinate descent on the quadratic-penalty QP (Sec. 3.2 eq. QP), one
// colour class per launch: every unit of a colour touches rows no other unit
// of that colour touches, so the parallel step equals the serial sweep over
// the colour (Algorithm 1's update, re-ordered by colour).  Also the
// asynchronous all-at-once mode of Sec. 3.4 (atomic residual updates), the
// FP64 residual refresh r = Ax - b and the FP64 checks.
#include <algorithm>
#include <cmath>

#include "problem.cuh"

namespace thetis {

constexpr int STEP_T = 256;        // threads per CTA of the step kernels

constexpr int CACHE = 4;           // r values a lane keeps between gather and scatter
constexpr int CHECK_BLOCKS = 2432; // fixed grid of the check kernel (deterministic reduction)
constexpr int NRED = 6;            // rho, obj, infeas, rr, ur, xx

#define GSTRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// segment t of a table of segment starts (start[0] = 0, n segments) holding
// flat index i: the last t with start[t] <= i
__device__ __forceinline__ int64_t seg_find(const int64_t* start, int64_t n, int64_t i) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (start[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

struct StepView {
  const int64_t* colptr;
  const uint32_t* rowidx;
  const float* val;  // null: +-1 encoded in rowidx
  const float* csq;  // ||a_j||^2 when val != null
  float* x;
  const float* ct;   // c - A^T ubar
  const float* xbar; // null: 0
  const float* lo;   // null: uniform bounds
  const float* hi;
  float lo_u, hi_u;
  float* r;
  float* s;
  const int8_t* sig;
  int sig_u;         // uniform slack sign or 0
  const float* cs;   // slack linear term or null
  const float* sbar; // null: 0
  float beta, inv_beta;
  float lfix;        // > 0: global L_max (step_rule 1)
  const float* lfix_i;  // batches with step_rule 1: every instance's own L_max (as its solve alone)
  int k;
  int async;         // 1: atomic residual updates
  int blk_shared;    // 1: a simplex block has two columns in one row (its scatter adds atomically)
  int small_g;       // small classes: 8 / small_g row slots per lane (small_g = 1, 2, 4 or 8, tuned)
  const uint32_t* ell;  // ELL row ids of the small classes
  const float* ellv;    // ELL values (null: +-1 encoded in ell)
  // batches: instance of every internal column / row and the frozen flags
  // (null for a single problem)
  const int32_t* inst_col;
  const int32_t* inst_row;
  const uint8_t* frozen;
  // batches: per colour, the tiles holding a unit of an unfinished instance
  // (act_tiles[act_off[c] .. + act_n[c]]); null for a single problem
  const int32_t* act_tiles;
  const int64_t* act_off;
  const int64_t* act_n;
};

// A column / slack row of a frozen batch instance is not stepped.
__device__ __forceinline__ bool col_frozen(const StepView& V, int64_t j) {
  return V.frozen && V.frozen[V.inst_col[j]];
}
__device__ __forceinline__ bool row_frozen(const StepView& V, int64_t i) {
  return V.frozen && V.frozen[V.inst_row[i]];
}
// step rule 1: the global L_max of column j / slack row i (batches: the instance's own)
__device__ __forceinline__ float lfix_col(const StepView& V, int64_t j) {
  return V.lfix_i ? V.lfix_i[V.inst_col[j]] : V.lfix;
}
__device__ __forceinline__ float lfix_row(const StepView& V, int64_t i) {
  return V.lfix_i ? V.lfix_i[V.inst_row[i]] : V.lfix;
}

struct SegLaunch {
  int cls;        // UnitClass, or UC_COUNT for slacks
  int64_t u0;     // first unit position (slacks: first internal row)
  int64_t n;      // units (slacks: rows)
  int64_t c0;     // first internal column
  int64_t b0;     // first CTA of this segment
  int64_t e0;     // small classes: first ELL slot
};

// Lanes per column of a small class of width W: each lane holds 8 / small_g
// of the W row slots.
__host__ __device__ __forceinline__ int small_lanes(int W, int small_g) {
  const int per = 8 / small_g;
  return W > per ? W / per : 1;
}

struct ColorLaunch {
  SegLaunch seg[UC_COUNT + 1];
  int nseg;
  int color;
  int64_t ntiles;  // tiles of the launch (per-colour engine)
};

__device__ __forceinline__ float coef(const StepView& V, int64_t p, uint32_t e) {
  return V.val ? V.val[p] : sgn_of(e);
}
__device__ __forceinline__ uint32_t rowof(const StepView& V, uint32_t e) {
  return V.val ? e : idx_of(e);
}

// r, x and s are written by other SMs between the colours of one persistent
// launch: read them around L1 (ld.global.cg).
__device__ __forceinline__ float ldr(const StepView& V, uint32_t row) { return __ldcg(V.r + row); }

__device__ __forceinline__ void r_add(const StepView& V, uint32_t row, float cached, float delta) {
  if (V.async) atomicAdd(&V.r[row], delta);
  else V.r[row] = cached + delta;
}

// One projected step of singleton column j by G cooperating lanes (G a power of
// two <= 32) -- or by a whole CTA when G == STEP_T.  Each lane keeps the first
// NC residual values it gathers in registers and writes them back after the
// step; the rest (columns longer than NC*G) are gathered and re-read in
// batches of four independent loads.
template <int G, int NC>
__device__ __forceinline__ void step_column(const StepView& V, int64_t j, int lane, float* red_smem,
                                            bool valid = true) {
  const int64_t p0 = valid ? V.colptr[j] : 0, p1 = valid ? V.colptr[j + 1] : 0;
  // loads that do not depend on r go first
  const float xj = valid ? __ldcg(V.x + j) : 0.f;
  const float ctj = valid ? V.ct[j] : 0.f;
  const float xb = (valid && V.xbar) ? V.xbar[j] : 0.f;
  uint32_t ce[NC];
  float cr[NC];
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    int64_t p = p0 + lane + (int64_t)t * G;
    ce[t] = (p < p1) ? V.rowidx[p] : 0u;
  }
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    int64_t p = p0 + lane + (int64_t)t * G;
    cr[t] = (p < p1) ? ldr(V, rowof(V, ce[t])) : 0.f;
  }
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    int64_t p = p0 + lane + (int64_t)t * G;
    if (p < p1) acc = fmaf(coef(V, p, ce[t]), cr[t], acc);
  }
  for (int64_t pb = p0 + lane + (int64_t)NC * G; pb < p1; pb += 4 * G) {
    uint32_t e4[4];
    float r4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) e4[t] = (pb + t * G < p1) ? V.rowidx[pb + t * G] : 0u;
#pragma unroll
    for (int t = 0; t < 4; ++t) r4[t] = (pb + t * G < p1) ? ldr(V, rowof(V, e4[t])) : 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (pb + t * G < p1) acc = fmaf(coef(V, pb + t * G, e4[t]), r4[t], acc);
  }
  // reduce over the G lanes
  if (G <= 32) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      float v = (threadIdx.x < G / 32) ? red_smem[threadIdx.x] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) red_smem[32] = v;
    }
    __syncthreads();
    acc = red_smem[32];
  }
  if (!valid) {
    if (G > 32) __syncthreads();
    return;
  }
  const float g = ctj + V.beta * acc + (xj - xb) * V.inv_beta;
  const float sq = V.val ? V.csq[j] : (float)(p1 - p0);
  const float L = (V.lfix > 0.f) ? lfix_col(V, j) : fmaf(V.beta, sq, V.inv_beta);
  const float lo = V.lo ? V.lo[j] : V.lo_u;
  const float hi = V.hi ? V.hi[j] : V.hi_u;
  const float xn = fminf(fmaxf(xj - g / L, lo), hi);
  const float d = xn - xj;
  if (lane == 0) V.x[j] = xn;
  if (d != 0.f) {
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      int64_t p = p0 + lane + (int64_t)t * G;
      if (p < p1) r_add(V, rowof(V, ce[t]), cr[t], coef(V, p, ce[t]) * d);
    }
    for (int64_t pb = p0 + lane + (int64_t)NC * G; pb < p1; pb += 4 * G) {
      uint32_t e4[4];
      float r4[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) e4[t] = (pb + t * G < p1) ? V.rowidx[pb + t * G] : 0u;
      if (!V.async) {
#pragma unroll
        for (int t = 0; t < 4; ++t) r4[t] = (pb + t * G < p1) ? ldr(V, rowof(V, e4[t])) : 0.f;
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (pb + t * G < p1) r_add(V, rowof(V, e4[t]), r4[t], coef(V, pb + t * G, e4[t]) * d);
    }
  }
  if (G > 32) __syncthreads();
}

// One projected step of small column j (ELL position p in its segment, first
// slot e0) by G lanes: lane gl holds slots gl, gl + G, ... of the W slots.  The
// slot addresses follow from p alone, and the 32 columns of a panel read one
// slot row as one coalesced line; padding slots are skipped.
template <int W, int G>
__device__ __forceinline__ void step_ell(const StepView& V, int64_t e0, int64_t j, int64_t p, int gl, bool valid) {
  constexpr int E = W / G;
  const int64_t base = e0 + (p >> 5) * (32 * W) + (p & 31);
  const float xj = valid ? __ldcg(V.x + j) : 0.f;
  const float ctj = valid ? V.ct[j] : 0.f;
  const float xb = (valid && V.xbar) ? V.xbar[j] : 0.f;
  uint32_t ce[E];
  float cv[E], cr[E];
#pragma unroll
  for (int i = 0; i < E; ++i) ce[i] = valid ? V.ell[base + (int64_t)(gl + G * i) * 32] : ELL_PAD;
#pragma unroll
  for (int i = 0; i < E; ++i)
    cv[i] = (ce[i] == ELL_PAD) ? 0.f : (V.ellv ? V.ellv[base + (int64_t)(gl + G * i) * 32] : sgn_of(ce[i]));
#pragma unroll
  for (int i = 0; i < E; ++i) cr[i] = (ce[i] != ELL_PAD) ? ldr(V, V.ellv ? ce[i] : idx_of(ce[i])) : 0.f;
  float acc = 0.f, sq = 0.f;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    acc = fmaf(cv[i], cr[i], acc);
    sq = fmaf(cv[i], cv[i], sq);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    sq += __shfl_xor_sync(0xffffffffu, sq, o, G);
  }
  if (!valid) return;
  const float g = ctj + V.beta * acc + (xj - xb) * V.inv_beta;
  const float L = (V.lfix > 0.f) ? lfix_col(V, j) : fmaf(V.beta, V.ellv ? V.csq[j] : sq, V.inv_beta);
  const float lo = V.lo ? V.lo[j] : V.lo_u;
  const float hi = V.hi ? V.hi[j] : V.hi_u;
  const float xn = fminf(fmaxf(xj - g / L, lo), hi);
  const float d = xn - xj;
  if (gl == 0) V.x[j] = xn;
  if (d != 0.f) {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (ce[i] != ELL_PAD) r_add(V, V.ellv ? ce[i] : idx_of(ce[i]), cr[i], cv[i] * d);
  }
}

// Small class of width W: tile b of the segment, G lanes per column.
template <int W, int G>
__device__ __forceinline__ void small_tile(const StepView& V, const SegLaunch& S, int64_t b) {
  const int64_t p = b * (STEP_T / G) + threadIdx.x / G;
  const bool in = p < S.n && !col_frozen(V, S.c0 + p);
  if (__any_sync(0xffffffffu, in)) step_ell<W, G>(V, S.e0, S.c0 + (in ? p : 0), in ? p : 0, threadIdx.x % G, in);
}

template <int W>
__device__ __forceinline__ void small_tile_w(const StepView& V, const SegLaunch& S, int64_t b) {
  switch (small_lanes(W, V.small_g)) {
    case 1: if constexpr (W <= 8) small_tile<W, 1>(V, S, b); break;
    case 2: if constexpr (W >= 2 && W <= 16) small_tile<W, 2>(V, S, b); break;
    case 4: if constexpr (W >= 4) small_tile<W, 4>(V, S, b); break;
    case 8: if constexpr (W >= 8) small_tile<W, 8>(V, S, b); break;
    case 16: if constexpr (W >= 16) small_tile<W, 16>(V, S, b); break;
    default: if constexpr (W >= 32) small_tile<W, 32>(V, S, b); break;
  }
}

// Columns with more than T_HUGE non-zeros: one CTA stages the column's row ids
// and residual values in shared memory with cp.async (every load in flight at
// once, no register staging), then reduces, steps and scatters from there.
// HUGE_CAP entries fit; the rest of a longer column goes through step_column.
constexpr int HUGE_CAP = 5888;  // 8 bytes each: 47,104 bytes of dynamic shared memory
constexpr int STEP_SMEM = HUGE_CAP * 8;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_cg4(void* smem, const void* gmem) {
  // the same copy with a 128-byte L2 prefetch hint (used for r)
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global.L2::128B [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ bool huge_path(const StepView& V, int64_t n) {
  return n <= HUGE_CAP && !V.val && !V.async;
}

// Copy column j's row ids into shared memory and prefetch its r lines into L2
// (used ahead of time, while the CTA waits at a barrier).
__device__ __forceinline__ void stage_huge(const StepView& V, int64_t j, unsigned char* dyn) {
  uint32_t* srow = (uint32_t*)dyn;
  const int64_t p0 = V.colptr[j], p1 = V.colptr[j + 1];
  const int64_t n = p1 - p0;
  if (!huge_path(V, n)) return;
  for (int t = threadIdx.x; t < n; t += STEP_T) cp_async4(srow + t, V.rowidx + p0 + t);
  cp_async_wait_all();
  for (int t = threadIdx.x; t < n; t += STEP_T) prefetch_l2(V.r + idx_of(srow[t]));
}

__device__ __forceinline__ void step_huge(const StepView& V, int64_t j, float* red_smem, unsigned char* dyn,
                                          bool staged = false) {
  uint32_t* srow = (uint32_t*)dyn;
  float* sr = (float*)(dyn + HUGE_CAP * 4);
  const int64_t p0 = V.colptr[j], p1 = V.colptr[j + 1];
  const int64_t n = p1 - p0;
  if (!huge_path(V, n)) {  // long, valued or async columns: register path
    step_column<STEP_T, 8>(V, j, threadIdx.x, red_smem);
    return;
  }
  const float xj = __ldcg(V.x + j);
  const float ctj = V.ct[j];
  const float xb = V.xbar ? V.xbar[j] : 0.f;
  if (!staged) {
    for (int t = threadIdx.x; t < n; t += STEP_T) cp_async4(srow + t, V.rowidx + p0 + t);
    cp_async_wait_all();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += STEP_T) cp_async_cg4(sr + t, V.r + idx_of(srow[t]));
  cp_async_wait_all();
  __syncthreads();
  float acc = 0.f;
  for (int t = threadIdx.x; t < n; t += STEP_T) acc = fmaf(sgn_of(srow[t]), sr[t], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < STEP_T / 32) ? red_smem[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red_smem[32] = v;
  }
  __syncthreads();
  acc = red_smem[32];
  const float g = ctj + V.beta * acc + (xj - xb) * V.inv_beta;
  const float L = (V.lfix > 0.f) ? lfix_col(V, j) : fmaf(V.beta, (float)n, V.inv_beta);
  const float lo = V.lo ? V.lo[j] : V.lo_u;
  const float hi = V.hi ? V.hi[j] : V.hi_u;
  const float xn = fminf(fmaxf(xj - g / L, lo), hi);
  const float d = xn - xj;
  if (threadIdx.x == 0) V.x[j] = xn;
  if (d != 0.f)
    for (int t = threadIdx.x; t < n; t += STEP_T) V.r[idx_of(srow[t])] = sr[t] + sgn_of(srow[t]) * d;
  __syncthreads();
}

// Block step (App. E): the k columns of a simplex block, one warp.  Lanes are
// split into k groups of S lanes (S the largest power of two <= 32/k); group q
// computes grad_q, the block moves to Proj_simplex(x - grad/L), L = beta
// max_q ||a_q||^2 + 1/beta.
__device__ __forceinline__ void step_block(const StepView& V, int64_t j0, int lane) {
  const int k = V.k;
  int S = 1;
  while (S * 2 * k <= 32) S *= 2;
  const int q = lane / S, t = lane % S;
  const bool act = q < k;
  const int64_t jq = j0 + (act ? q : 0);
  const int64_t p0 = act ? V.colptr[jq] : 0, p1 = act ? V.colptr[jq + 1] : 0;
  // lane q < k's own column: loads that do not depend on r go first
  const float xq0 = (lane < k) ? __ldcg(V.x + j0 + lane) : 0.f;
  const float ctq = (lane < k) ? V.ct[j0 + lane] : 0.f;
  const float xbq = (lane < k && V.xbar) ? V.xbar[j0 + lane] : 0.f;
  uint32_t ce[CACHE];
  float cr[CACHE];
  float acc = 0.f;
#pragma unroll
  for (int u = 0; u < CACHE; ++u) {
    int64_t p = p0 + t + (int64_t)u * S;
    ce[u] = 0;
    cr[u] = 0.f;
    if (p < p1) {
      uint32_t e = V.rowidx[p];
      float rr = ldr(V, rowof(V, e));
      ce[u] = e;
      cr[u] = rr;
      acc = fmaf(coef(V, p, e), rr, acc);
    }
  }
  for (int64_t p = p0 + t + (int64_t)CACHE * S; p < p1; p += S) {
    uint32_t e = V.rowidx[p];
    acc = fmaf(coef(V, p, e), ldr(V, rowof(V, e)), acc);
  }
  for (int o = S / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  // per-column ||a||^2 and the block L
  float sq = act ? (V.val ? V.csq[jq] : (float)(p1 - p0)) : 0.f;
  float sqm = sq;
  for (int o = 16; o > 0; o >>= 1) sqm = fmaxf(sqm, __shfl_xor_sync(0xffffffffu, sqm, o));
  const float L = (V.lfix > 0.f) ? V.lfix : fmaf(V.beta, sqm, V.inv_beta);
  // gather y_q into lane q
  float gq = __shfl_sync(0xffffffffu, acc, (lane < k ? lane : 0) * S);
  float xq = 0.f, y = -INFINITY;
  if (lane < k) {
    xq = xq0;
    float g = ctq + V.beta * gq + (xq - xbq) * V.inv_beta;
    y = xq - g / L;
  }
  // simplex projection: for lane j, c_j = #{i: y_i >= y_j}, S_j = sum of those y_i;
  // theta = (S - 1)/c at the largest c whose y_j - (S_j - 1)/c_j > 0.
  float cnt = 0.f, sum = 0.f;
  for (int i = 0; i < k; ++i) {
    float yi = __shfl_sync(0xffffffffu, y, i);
    if (lane < k && yi >= y) {
      cnt += 1.f;
      sum += yi;
    }
  }
  float theta = (lane < k) ? (sum - 1.f) / cnt : 0.f;
  bool ok = (lane < k) && (y - theta > 0.f);
  int key = ok ? (int)cnt : 0;
  int best = key;
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  unsigned who = __ballot_sync(0xffffffffu, key == best && ok);
  float th = __shfl_sync(0xffffffffu, theta, __ffs(who) - 1);
  float xn = fmaxf(y - th, 0.f);
  float d = xn - xq;
  if (lane < k) V.x[j0 + lane] = xn;
  float dq = __shfl_sync(0xffffffffu, d, act ? q : 0);
  if (act && dq != 0.f) {
    // two columns of the block in one row (blk_shared): both changes must
    // land, so the scatter adds atomically
    const bool atom = V.async || V.blk_shared;
#pragma unroll
    for (int u = 0; u < CACHE; ++u) {
      int64_t p = p0 + t + (int64_t)u * S;
      if (p < p1) {
        const uint32_t row = rowof(V, ce[u]);
        const float delta = coef(V, p, ce[u]) * dq;
        if (atom) atomicAdd(&V.r[row], delta);
        else V.r[row] = cr[u] + delta;
      }
    }
    for (int64_t p = p0 + t + (int64_t)CACHE * S; p < p1; p += S) {
      uint32_t e = V.rowidx[p];
      uint32_t row = rowof(V, e);
      float delta = coef(V, p, e) * dq;
      if (atom) atomicAdd(&V.r[row], delta);
      else V.r[row] = ldr(V, row) + delta;
    }
  }
}

constexpr int SLACK_ROWS = 4;  // slack rows per thread (one tile = STEP_T * SLACK_ROWS rows)

// Slack step of rows [i0, i0 + n) handled by this thread: row i0 + t*STEP_T + tid.
__device__ __forceinline__ void step_slacks(const StepView& V, int64_t i0, int64_t n) {
  float sv[SLACK_ROWS], rv[SLACK_ROWS];
  bool on[SLACK_ROWS];
#pragma unroll
  for (int t = 0; t < SLACK_ROWS; ++t) {
    int64_t q = (int64_t)t * STEP_T + threadIdx.x;
    on[t] = q < n && !row_frozen(V, i0 + q);
    sv[t] = on[t] ? __ldcg(V.s + i0 + q) : 0.f;
    rv[t] = on[t] ? __ldcg(V.r + i0 + q) : 0.f;
  }
  const float L0 = (V.lfix > 0.f) ? V.lfix : V.beta + V.inv_beta;
#pragma unroll
  for (int t = 0; t < SLACK_ROWS; ++t) {
    int64_t q = (int64_t)t * STEP_T + threadIdx.x;
    if (!on[t]) continue;
    const int64_t i = i0 + q;
    const float L = (V.lfix > 0.f && V.lfix_i) ? lfix_row(V, i) : L0;
    const float sg = V.sig_u ? (float)V.sig_u : (float)V.sig[i];
    const float sb = V.sbar ? V.sbar[i] : 0.f;
    const float lin = V.cs ? V.cs[i] : 0.f;
    const float g = lin + V.beta * sg * rv[t] + (sv[t] - sb) * V.inv_beta;
    const float sn = fmaxf(sv[t] - g / L, 0.f);
    const float d = sn - sv[t];
    V.s[i] = sn;
    if (d != 0.f) {
      if (V.async) atomicAdd(&V.r[i], sg * d);
      else V.r[i] = rv[t] + sg * d;
    }
  }
}

// One tile of a colour: the CTA serves tile `tile` of the segment it falls in.
// FULL = false compiles the paths of everything but long columns (no shared
// memory staging): fewer registers, more CTAs per SM.
template <bool FULL = true>
__device__ __forceinline__ void process_tile(const StepView& V, const SegLaunch* segs, int nseg, int64_t tile,
                                             float* red_smem, unsigned char* dyn, bool staged = false) {
  int si = 0;
  while (si + 1 < nseg && tile >= segs[si + 1].b0) ++si;
  const SegLaunch S = segs[si];
  const int64_t b = tile - S.b0;
  const int lane = threadIdx.x & 31;
  switch (S.cls) {
    case UC_HUGE:
    case UC_LARGE: {
      if constexpr (FULL) {
        if (b < S.n && !col_frozen(V, S.c0 + b)) step_huge(V, S.c0 + b, red_smem, dyn, staged);
      }
      break;
    }
    case UC_MED: {
      int64_t u = b * (STEP_T / 32) + (threadIdx.x >> 5);
      if (u < S.n && !col_frozen(V, S.c0 + u)) step_column<32, 4>(V, S.c0 + u, lane, red_smem);
      break;
    }
    case UC_S32: small_tile_w<32>(V, S, b); break;
    case UC_S16: small_tile_w<16>(V, S, b); break;
    case UC_S8: small_tile_w<8>(V, S, b); break;
    case UC_S4: small_tile_w<4>(V, S, b); break;
    case UC_S2: small_tile_w<2>(V, S, b); break;
    case UC_BLOCK: {
      int64_t u = b * (STEP_T / 32) + (threadIdx.x >> 5);
      if (u < S.n) step_block(V, S.c0 + u * V.k, lane);
      break;
    }
    default: {  // slacks
      int64_t i0 = S.u0 + b * (STEP_T * SLACK_ROWS);
      int64_t rest = S.n - b * (STEP_T * SLACK_ROWS);
      if (rest > 0) step_slacks(V, i0, rest < STEP_T * SLACK_ROWS ? rest : STEP_T * SLACK_ROWS);
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// Tail colours.  The last colours hold only a few singleton columns each (the
// hubs of a power-law graph); their order is a chain, so each colour costs a
// grid barrier plus one column's latency.  A tail column's rows are split
// into those shared with another tail column (T rows) and the rest (H rows).
// No unit touches an H row between the end of the head colours and that
// column's own step, so the three phases
//   P (all CTAs): h_u = a_u^T r over the H rows,
//   T (one CTA per unit, colours in order, a barrier of those few CTAs
//     between colours): the step of every tail column from h_u plus its T
//     rows, scattering the T rows,
//   S (all CTAs): r += a_u d_u on the H rows,
// leave x and r as the colour-by-colour sweep does (each r entry is updated
// once, from the value it had); only the FP32 order of the dot changes.
// ---------------------------------------------------------------------------
struct TailView {
  int64_t n;           // tail units
  int ncol;            // tail colours
  const int64_t* col;  // internal column of each unit, colour order
  const int64_t* coff; // first unit of each tail colour (ncol + 1)
  const int64_t* hptr;
  const uint32_t* hrow;
  const int64_t* tptr;
  const uint32_t* trow;
  float* h;            // partial dot over the H rows
  float* d;            // step of the unit
  int ctas;            // CTAs of phase T: the most units of any tail colour (one CTA per unit)
};


__device__ __noinline__ void tail_partial(const StepView& V, const TailView& T, int64_t u, float* red_smem) {
  const int64_t q0 = T.hptr[u], q1 = T.hptr[u + 1];
  float acc = 0.f;
  for (int64_t qb = q0 + threadIdx.x; qb < q1; qb += 4 * STEP_T) {
    uint32_t e4[4];
    float r4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) e4[t] = (qb + t * STEP_T < q1) ? T.hrow[qb + t * STEP_T] : 0u;
#pragma unroll
    for (int t = 0; t < 4; ++t) r4[t] = (qb + t * STEP_T < q1) ? ldr(V, idx_of(e4[t])) : 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (qb + t * STEP_T < q1) acc = fmaf(sgn_of(e4[t]), r4[t], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < STEP_T / 32) ? red_smem[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) T.h[u] = v;
  }
  __syncthreads();
}

// The step of tail unit u by the whole CTA: its T rows gathered four at a
// time per thread, block-reduced, added to the H-row partial; the T rows
// scattered.  (The tail functions are not inlined: the sweep's hot loop keeps
// its registers.)
__device__ __noinline__ void tail_unit(const StepView& V, const TailView& T, int64_t u, float* red_smem) {
  const int64_t j = T.col[u];
  const int64_t q0 = T.tptr[u], q1 = T.tptr[u + 1];
  const float xj = __ldcg(V.x + j);
  const float ctj = V.ct[j];
  const float xb = V.xbar ? V.xbar[j] : 0.f;
  const float hj = T.h[u];
  uint32_t ce[4];
  float cr[4];
  const int64_t qf = q0 + threadIdx.x;  // first batch: kept for the scatter
#pragma unroll
  for (int t = 0; t < 4; ++t) ce[t] = (qf + t * STEP_T < q1) ? T.trow[qf + t * STEP_T] : 0u;
#pragma unroll
  for (int t = 0; t < 4; ++t) cr[t] = (qf + t * STEP_T < q1) ? ldr(V, idx_of(ce[t])) : 0.f;
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (qf + t * STEP_T < q1) acc = fmaf(sgn_of(ce[t]), cr[t], acc);
  for (int64_t qb = qf + 4 * STEP_T; qb < q1; qb += 4 * STEP_T) {
    uint32_t e4[4];
    float r4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) e4[t] = (qb + t * STEP_T < q1) ? T.trow[qb + t * STEP_T] : 0u;
#pragma unroll
    for (int t = 0; t < 4; ++t) r4[t] = (qb + t * STEP_T < q1) ? ldr(V, idx_of(e4[t])) : 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (qb + t * STEP_T < q1) acc = fmaf(sgn_of(e4[t]), r4[t], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < STEP_T / 32) ? red_smem[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      const float tot = hj + v;
      const float nnz = (float)((T.hptr[u + 1] - T.hptr[u]) + (q1 - q0));
      const float g = ctj + V.beta * tot + (xj - xb) * V.inv_beta;
      const float L = (V.lfix > 0.f) ? V.lfix : fmaf(V.beta, nnz, V.inv_beta);
      const float lo = V.lo ? V.lo[j] : V.lo_u;
      const float hi = V.hi ? V.hi[j] : V.hi_u;
      const float xn = fminf(fmaxf(xj - g / L, lo), hi);
      V.x[j] = xn;
      T.d[u] = xn - xj;
      red_smem[32] = xn - xj;
    }
  }
  __syncthreads();
  const float d = red_smem[32];
  __syncthreads();  // red_smem is reused by the next unit
  if (d == 0.f) return;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (qf + t * STEP_T < q1) V.r[idx_of(ce[t])] = cr[t] + sgn_of(ce[t]) * d;
  for (int64_t qb = qf + 4 * STEP_T; qb < q1; qb += 4 * STEP_T) {
    uint32_t e4[4];
    float r4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) e4[t] = (qb + t * STEP_T < q1) ? T.trow[qb + t * STEP_T] : 0u;
#pragma unroll
    for (int t = 0; t < 4; ++t) r4[t] = (qb + t * STEP_T < q1) ? ldr(V, idx_of(e4[t])) : 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (qb + t * STEP_T < q1) V.r[idx_of(e4[t])] = r4[t] + sgn_of(e4[t]) * d;
  }
}

__device__ __noinline__ void tail_scatter(const StepView& V, const TailView& T, int64_t u) {
  const float d = T.d[u];
  if (d == 0.f) return;
  for (int64_t q = T.hptr[u] + threadIdx.x; q < T.hptr[u + 1]; q += STEP_T) {
    const uint32_t e = T.hrow[q];
    V.r[idx_of(e)] = ldr(V, idx_of(e)) + sgn_of(e) * d;
  }
}

// the three phases as separate launches (per-colour engine)
__global__ void __launch_bounds__(STEP_T) k_tail_partial(StepView V, TailView T) {
  __shared__ float red_smem[33];
  for (int64_t u = blockIdx.x; u < T.n; u += gridDim.x) tail_partial(V, T, u, red_smem);
}
// one tail colour per launch, one CTA per unit
__global__ void __launch_bounds__(STEP_T) k_tail_colour(StepView V, TailView T, int tc) {
  __shared__ float red_smem[33];
  const int64_t u = T.coff[tc] + blockIdx.x;
  if (u < T.coff[tc + 1]) tail_unit(V, T, u, red_smem);
}
__global__ void __launch_bounds__(STEP_T) k_tail_scatter(StepView V, TailView T) {
  for (int64_t u = blockIdx.x; u < T.n; u += gridDim.x) tail_scatter(V, T, u);
}

// One colour per launch: CTA b serves tile b.
__global__ void __launch_bounds__(STEP_T, 4) k_color_step(StepView V, ColorLaunch CL) {
  __shared__ float red_smem[33];
  extern __shared__ __align__(16) unsigned char dyn[];
  if (V.act_tiles) {  // batches: only the active tiles of the colour (grid sized for all)
    if ((int64_t)blockIdx.x >= V.act_n[CL.color]) return;
    process_tile(V, CL.seg, CL.nseg, V.act_tiles[V.act_off[CL.color] + blockIdx.x], red_smem, dyn);
    return;
  }
  // one tile per CTA, or CTAs taking tiles in turn when the grid is capped (async concurrency)
  for (int64_t t = blockIdx.x; t < CL.ntiles; t += gridDim.x) process_tile(V, CL.seg, CL.nseg, t, red_smem, dyn);
}

// Grid-wide barrier of a cooperative launch, split into arrive and wait so a CTA
// can prefetch the next colour while the others finish.  One 32-bit word: CTA 0
// adds 2^31 - (G - 1), every other CTA adds 1, so the top bit flips exactly once
// per barrier.  The wait is bounded in time (%globaltimer, nanoseconds; 2 s by
// default, set per handle): after the limit the CTA records err = 1 and the
// launch gives up (the host reports THETIS_E_TIMEOUT).  `phantom` adds CTAs
// that never arrive (a test of the timeout path: the wait then always runs
// out).
__device__ __forceinline__ unsigned bar_arrive(unsigned* bar, unsigned participants = 0, unsigned phantom = 0) {
  const unsigned n = (participants ? participants : gridDim.x) + phantom;  // CTAs 0 .. n-1 take part
  unsigned inc = (blockIdx.x == 0) ? (0x80000000u - (n - 1)) : 1u;
  unsigned old;
  asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(inc) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool bar_wait(unsigned* bar, unsigned old, int* err, long long limit_ns) {
  const unsigned long long t0 = global_ns();
  unsigned it = 0, cur;
  while (true) {
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
    if ((cur ^ old) & 0x80000000u) return true;
    if ((++it & 255u) == 0 && (*(volatile int*)err || (long long)(global_ns() - t0) > limit_ns)) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(64);  // keep hundreds of pollers from saturating the line's L2 slice
  }
}

// L2 prefetch of the read-only data of one tile (column pointers, row ids, x, c)
// or, for slack tiles, of the tile's s and r rows.  Only a hint: r lines may be
// rewritten before use, which L2 coherence handles.
__device__ __forceinline__ void prefetch_tile(const StepView& V, const SegLaunch* segs, int nseg, int64_t tile) {
  int si = 0;
  while (si + 1 < nseg && tile >= segs[si + 1].b0) ++si;
  const SegLaunch S = segs[si];
  const int64_t b = tile - S.b0;
  int64_t u0, u1;
  switch (S.cls) {
    case UC_HUGE:
    case UC_LARGE: u0 = b; u1 = b + 1; break;
    case UC_MED:
    case UC_BLOCK: u0 = b * (STEP_T / 32); u1 = u0 + STEP_T / 32; break;
    case UC_S32:
    case UC_S16:
    case UC_S8:
    case UC_S4:
    case UC_S2: {
      // the tile's ELL panels are one contiguous range
      const int W = small_width(S.cls);
      const int per = STEP_T / small_lanes(W, V.small_g);
      const int64_t p0 = b * per, p1 = min(S.n, p0 + per);
      if (p0 >= p1) return;
      const int64_t e1 = S.e0 + ((p1 + 31) >> 5) * 32 * W;
      for (int64_t e = S.e0 + (p0 >> 5) * 32 * W + (int64_t)threadIdx.x * 32; e < e1; e += (int64_t)STEP_T * 32)
        prefetch_l2(V.ell + e);
      if (threadIdx.x == 0) {
        prefetch_l2(V.x + S.c0 + p0);
        prefetch_l2(V.ct + S.c0 + p0);
      }
      return;
    }
    default: {
      const int64_t r0 = S.u0 + b * (STEP_T * SLACK_ROWS);
      const int64_t r1 = min(S.u0 + S.n, r0 + (int64_t)STEP_T * SLACK_ROWS);
      for (int64_t i = r0 + (int64_t)threadIdx.x * 32; i < r1; i += (int64_t)STEP_T * 32) {
        prefetch_l2(V.s + i);
        prefetch_l2(V.r + i);
      }
      return;
    }
  }
  if (u1 > S.n) u1 = S.n;
  if (u0 >= u1) return;
  const int len = (S.cls == UC_BLOCK) ? V.k : 1;
  const int64_t j0 = S.c0 + u0 * len, j1 = S.c0 + u1 * len;
  if (threadIdx.x == 0) {
    prefetch_l2(V.colptr + j0);
    prefetch_l2(V.colptr + j1);
    prefetch_l2(V.x + j0);
    prefetch_l2(V.ct + j0);
  }
  const int64_t p0 = V.colptr[j0], p1 = V.colptr[j1];
  for (int64_t p = p0 + (int64_t)threadIdx.x * 32; p < p1; p += (int64_t)STEP_T * 32) prefetch_l2(V.rowidx + p);
}

// Persistent colour sweep: `epochs` epochs, every colour's tiles spread over all
// CTAs, one grid barrier between colours.  Equivalent to one k_color_step launch
// per colour.  While it waits at a barrier a CTA loads the next colour's launch
// descriptor and prefetches its first tiles into L2.
constexpr int PREFETCH_TILES = 2;

template <bool FULL>
__global__ void __launch_bounds__(STEP_T, FULL ? 4 : 6) k_sweep(StepView V, const ColorLaunch* plan, const int64_t* ntiles,
                                                     int ncolors, int epochs, unsigned* bar, int* err, TailView TV,
                                                     long long wait_ns, unsigned phantom) {
  __shared__ float red_smem[33];
  __shared__ ColorLaunch cl[2];
  __shared__ int ok;
  extern __shared__ __align__(16) unsigned char dyn[];
  constexpr int CLW = (int)(sizeof(ColorLaunch) / 4);
  static_assert(sizeof(ColorLaunch) % 4 == 0, "ColorLaunch copied as words");
  if (threadIdx.x < CLW) ((unsigned*)&cl[0])[threadIdx.x] = ((const unsigned*)&plan[0])[threadIdx.x];
  __syncthreads();
  int cur = 0;
  bool first_staged = false;
  // tile q of colour c (batches: through the active-tile list)
  auto tile_of = [&](int c, int64_t q) -> int64_t { return V.act_tiles ? V.act_tiles[V.act_off[c] + q] : q; };
  auto count_of = [&](int c) -> int64_t { return V.act_tiles ? V.act_n[c] : ntiles[c]; };
  // grid barrier that also loads colour cn's descriptor, stages its first long
  // column and prefetches its first tiles while waiting
  auto advance = [&](int cn) -> bool {
    __syncthreads();
    unsigned old = 0;
    if (threadIdx.x == 0) old = bar_arrive(bar, 0, phantom);
    if (threadIdx.x < CLW) ((unsigned*)&cl[cur ^ 1])[threadIdx.x] = ((const unsigned*)&plan[cn])[threadIdx.x];
    __syncthreads();
    const int64_t ntn = count_of(cn);
    bool staged = false;
    if ((int64_t)blockIdx.x < ntn) {
      // a first tile that is a long column: its row ids go to shared memory now
      const int64_t t0 = tile_of(cn, blockIdx.x);
      const ColorLaunch& nx = cl[cur ^ 1];
      int si = 0;
      while (si + 1 < nx.nseg && t0 >= nx.seg[si + 1].b0) ++si;
      const SegLaunch S = nx.seg[si];
      if (FULL && (S.cls == UC_HUGE || S.cls == UC_LARGE) && t0 - S.b0 < S.n) {
        stage_huge(V, S.c0 + (t0 - S.b0), dyn);
        staged = true;
      }
    }
    for (int q = staged ? 1 : 0; q < PREFETCH_TILES; ++q) {
      const int64_t qq = blockIdx.x + (int64_t)q * gridDim.x;
      if (qq < ntn) prefetch_tile(V, cl[cur ^ 1].seg, cl[cur ^ 1].nseg, tile_of(cn, qq));
    }
    if (threadIdx.x == 0) ok = bar_wait(bar, old, err, wait_ns) ? 1 : 0;
    __syncthreads();
    cur ^= 1;
    first_staged = staged;
    return ok != 0;
  };
  // plain grid barrier (between the tail phases)
  auto sync = [&]() -> bool {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned old = bar_arrive(bar, 0, phantom);
      ok = bar_wait(bar, old, err, wait_ns) ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
  };
  for (int e = 0; e < epochs; ++e) {
    const bool last_epoch = e == epochs - 1;
    for (int c = 0; c < ncolors; ++c) {
      const int64_t nt = count_of(c);
      for (int64_t q = blockIdx.x; q < nt; q += gridDim.x)
        process_tile<FULL>(V, cl[cur].seg, cl[cur].nseg, tile_of(c, q), red_smem, dyn,
                           first_staged && q == blockIdx.x);
      if (c + 1 < ncolors) {
        if (!advance(c + 1)) return;
      } else if (TV.n > 0) {
        if (!sync()) return;
      } else if (!last_epoch) {
        if (!advance(0)) return;
      }
    }
    if (TV.n > 0) {
      for (int64_t u = blockIdx.x; u < TV.n; u += gridDim.x) tail_partial(V, TV, u, red_smem);
      if (!sync()) return;
      const int nT = min(TV.ctas, (int)gridDim.x);
      if ((int)blockIdx.x < nT) {
        // colours in order, one CTA per unit, a barrier of the nT CTAs between colours
        for (int tc = 0; tc < TV.ncol; ++tc) {
          for (int64_t u = TV.coff[tc] + blockIdx.x; u < TV.coff[tc + 1]; u += nT) tail_unit(V, TV, u, red_smem);
          if (tc + 1 < TV.ncol) {
            __syncthreads();
            if (threadIdx.x == 0) {
              const unsigned old = bar_arrive(bar + 32, (unsigned)nT, phantom);
              ok = bar_wait(bar + 32, old, err, wait_ns) ? 1 : 0;
            }
            __syncthreads();
            if (!ok) return;
          }
        }
      }
      if (!sync()) return;
      for (int64_t u = blockIdx.x; u < TV.n; u += gridDim.x) tail_scatter(V, TV, u);
      if (!last_epoch && !advance(0)) return;
    }
  }
}

static int64_t ctas_for(int cls, int64_t n, int small_g) {
  switch (cls) {
    case UC_HUGE:
    case UC_LARGE: return n;
    case UC_MED:
    case UC_BLOCK: return (n + STEP_T / 32 - 1) / (STEP_T / 32);
    case UC_COUNT: return (n + STEP_T * SLACK_ROWS - 1) / (STEP_T * SLACK_ROWS);
    default: {  // small classes
      const int per = STEP_T / small_lanes(small_width(cls), small_g);
      return (n + per - 1) / per;
    }
  }
}

__global__ void k_batch_lfix(const int32_t* maxdeg, const int64_t* eoff, int64_t count, double beta, float* lfix) {
  GSTRIDE(t, count) {
    const int lm = max(maxdeg[t], eoff[t + 1] > eoff[t] ? 1 : 0);
    lfix[t] = (float)(beta * (double)lm + 1.0 / beta);
  }
}

// batches with step rule 1: every instance's own L_max = beta * max(longest
// column, 1 if it has rows) + 1/beta, as its solve alone takes (before any
// stream capture of an epoch)
void batch_step_rule(Problem& P, const SolveArgs& a) {
  if (a.step_rule != 1 || P.nbatch == 0 || !P.bmaxdeg) return;
  if (!P.blfix) P.blfix = P.mem.alloc<float>(P.nbatch);
  if (P.blfix_beta == a.beta) return;
  k_batch_lfix<<<grid_for(P.nbatch, 256), 256, 0, P.stream>>>(P.bmaxdeg, P.beoff, P.nbatch, a.beta, P.blfix);
  TH_LAUNCHED();
  P.blfix_beta = a.beta;
}

static StepView make_view(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar) {
  StepView V;
  V.colptr = P.colptr;
  V.rowidx = P.rowidx;
  V.val = P.has_val ? P.val : nullptr;
  V.csq = P.csq;
  V.x = P.x;
  V.ct = use_ubar ? P.ctil : P.c;
  V.xbar = use_xbar ? P.xbar : nullptr;
  V.lo = P.bounds_uniform ? nullptr : P.lo;
  V.hi = P.bounds_uniform ? nullptr : P.hi;
  V.lo_u = P.lo_u;
  V.hi_u = P.hi_u;
  V.r = P.r;
  V.s = P.s;
  V.sig = P.sig;
  V.sig_u = P.slack_sign_uniform;
  V.cs = use_ubar ? P.cs : nullptr;
  V.sbar = use_xbar ? P.sbar : nullptr;
  V.beta = (float)a.beta;
  V.inv_beta = (float)(1.0 / a.beta);
  V.lfix = (a.step_rule == 1) ? (float)(a.beta * P.lmax_sq + 1.0 / a.beta) : 0.f;
  V.lfix_i = (a.step_rule == 1 && P.nbatch > 0 && P.blfix && P.blfix_beta == a.beta) ? P.blfix : nullptr;
  V.k = P.k;
  V.async = (a.mode == THETIS_MODE_ASYNC) ? 1 : 0;
  V.blk_shared = P.blk_shared ? 1 : 0;
  V.small_g = P.small_g;
  V.ell = P.ell;
  V.ellv = P.has_val ? P.ellv : nullptr;
  const bool batch = P.nbatch > 0 && P.bfrozen;
  V.inst_col = batch ? P.binst_col : nullptr;
  V.inst_row = batch ? P.binst_row : nullptr;
  V.frozen = batch ? P.bfrozen : nullptr;
  const bool act = batch && P.act_tiles && P.act_g == P.small_g;
  V.act_tiles = act ? P.act_tiles : nullptr;
  V.act_off = act ? P.act_off : nullptr;
  V.act_n = act ? P.act_n : nullptr;
  return V;
}

// ---------------------------------------------------------------------------
// tail colours: selection and the split of their columns' rows
// ---------------------------------------------------------------------------
constexpr int TAIL_MIN_COLOURS = 8;    // fewer tail colours: not worth the three phases
constexpr int64_t TAIL_MAX_UNITS = 152; // units a tail colour may hold (one CTA each)

__global__ void k_tail_rowcount(const int64_t* colptr, const uint32_t* rowidx, const int64_t* col, int64_t n,
                                int32_t* rcnt) {
  for (int64_t u = blockIdx.x; u < n; u += gridDim.x) {
    const int64_t j = col[u];
    for (int64_t q = colptr[j] + threadIdx.x; q < colptr[j + 1]; q += blockDim.x) atomicAdd(&rcnt[idx_of(rowidx[q])], 1);
  }
}

// one warp per unit: rows shared with another tail column (T) and the rest (H)
__global__ void k_tail_counts(const int64_t* colptr, const uint32_t* rowidx, const int64_t* col, int64_t n,
                              const int32_t* rcnt, int64_t* hc, int64_t* tc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const int64_t j = col[u], q0 = colptr[j], q1 = colptr[j + 1];
    int t = 0;
    for (int64_t q = q0 + lane; q < q1; q += 32) t += rcnt[idx_of(rowidx[q])] > 1;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      tc[u] = t;
      hc[u] = q1 - q0 - t;
    }
  }
}

// one warp per unit, entries kept in column order (a ballot per 32 entries):
// the same deterministic split as a serial pass
__global__ void k_tail_fill(const int64_t* colptr, const uint32_t* rowidx, const int64_t* col, int64_t n,
                            const int32_t* rcnt, const int64_t* hptr, const int64_t* tptr, uint32_t* hrow,
                            uint32_t* trow) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const int64_t j = col[u], q0 = colptr[j], q1 = colptr[j + 1];
    int64_t h = hptr[u], t = tptr[u];
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane;
      const bool in = q < q1;
      const uint32_t e = in ? rowidx[q] : 0u;
      const bool shared = in && rcnt[idx_of(e)] > 1;
      const unsigned ms = __ballot_sync(0xffffffffu, shared), mh = __ballot_sync(0xffffffffu, in && !shared);
      if (shared) trow[t + __popc(ms & lt)] = e;
      else if (in) hrow[h + __popc(mh & lt)] = e;
      t += __popc(ms);
      h += __popc(mh);
    }
  }
}

// The tail: the longest run of last colours that hold no slack, no simplex
// block and at most TAIL_MAX_UNITS singleton columns each (pattern +-1
// matrices, single problems).
void ensure_tail(Problem& P) {
  if (P.tail_T >= 0) return;
  const int C = P.ncolors;
  P.tail_T = C;
  if (P.nbatch > 0 || P.has_val || C < TAIL_MIN_COLOURS + 1) return;
  int T = C;
  while (T > 1) {
    const ColorPlan& cp = P.plan[T - 1];
    int64_t units = 0;
    bool ok = cp.srow1 == cp.srow0;
    for (auto& sg : cp.segs) {
      ok = ok && sg.cls != UC_BLOCK;
      units += sg.u1 - sg.u0;
    }
    if (!ok || units > TAIL_MAX_UNITS) break;
    --T;
  }
  if (C - T < TAIL_MIN_COLOURS) return;
  std::vector<int64_t> col, coff{0};
  int64_t umax = 1;
  for (int c = T; c < C; ++c) {
    int64_t uc = 0;
    for (auto& sg : P.plan[c].segs) uc += sg.u1 - sg.u0;
    umax = std::max(umax, uc);
  }
  for (int c = T; c < C; ++c) {
    for (auto& sg : P.plan[c].segs)
      for (int64_t u = 0; u < sg.u1 - sg.u0; ++u) col.push_back(sg.c0 + u);
    coff.push_back((int64_t)col.size());
  }
  cudaStream_t s = P.stream;
  const int64_t n = (int64_t)col.size();
  Arena tmp(s);
  P.tail_col = P.mem.alloc<int64_t>(n);
  P.tail_coff = P.mem.alloc<int64_t>(C - T + 1);
  TH_CUDA(cudaMemcpyAsync(P.tail_col, col.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaMemcpyAsync(P.tail_coff, coff.data(), (C - T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  int32_t* rcnt = tmp.alloc<int32_t>(P.M + 1);
  TH_CUDA(cudaMemsetAsync(rcnt, 0, (P.M + 1) * sizeof(int32_t), s));
  k_tail_rowcount<<<grid_for(n * 256, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.tail_col, n, rcnt);
  TH_LAUNCHED();
  int64_t* hc = tmp.alloc<int64_t>(n + 1);
  int64_t* tc = tmp.alloc<int64_t>(n + 1);
  k_tail_counts<<<grid_for(n * 32, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.tail_col, n, rcnt, hc, tc);
  TH_LAUNCHED();
  P.tail_hptr = P.mem.alloc<int64_t>(n + 1);
  P.tail_tptr = P.mem.alloc<int64_t>(n + 1);
  exclusive_scan_i64(hc, P.tail_hptr, n, tmp, s);
  exclusive_scan_i64(tc, P.tail_tptr, n, tmp, s);
  int64_t tot[2];
  TH_CUDA(cudaMemcpyAsync(&tot[0], P.tail_hptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(&tot[1], P.tail_tptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  P.tail_hrow = P.mem.alloc<uint32_t>(tot[0] + 1);
  P.tail_trow = P.mem.alloc<uint32_t>(tot[1] + 1);
  k_tail_fill<<<grid_for(n * 32, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.tail_col, n, rcnt, P.tail_hptr,
                                                   P.tail_tptr, P.tail_hrow, P.tail_trow);
  TH_LAUNCHED();
  P.tail_h = P.mem.alloc<float>(n);
  P.tail_d = P.mem.alloc<float>(n);
  TH_CUDA(cudaStreamSynchronize(s));  // col / coff must outlive their copies
  P.tail_T = T;
  P.tail_n = n;
  P.tail_ncol = C - T;
  P.tail_ctas = (int)umax;
}

static TailView make_tail_view(const Problem& P) {
  TailView T{};
  if (P.tail_T < 0 || P.tail_T >= P.ncolors) return T;
  T.n = P.tail_n;
  T.ncol = P.tail_ncol;
  T.col = P.tail_col;
  T.coff = P.tail_coff;
  T.hptr = P.tail_hptr;
  T.hrow = P.tail_hrow;
  T.tptr = P.tail_tptr;
  T.trow = P.tail_trow;
  T.h = P.tail_h;
  T.d = P.tail_d;
  T.ctas = P.tail_ctas;
  return T;
}

// colours the colour-by-colour sweep runs (the rest, if any, are the tail)
static int head_colours(const Problem& P) { return (P.tail_T >= 0 && P.tail_T < P.ncolors) ? P.tail_T : P.ncolors; }

// Launches of one epoch in colour order (colored) or one launch over all
// units (async).
void run_epoch(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar) {
  StepView V = make_view(P, a, use_ubar, use_xbar);
  cudaStream_t s = P.stream;
  auto launch = [&](ColorLaunch& CL, int64_t total) {
    if (total <= 0) return;
    TH_CHECK(total < (int64_t(1) << 31), THETIS_E_INVALID, "colour class too large for one launch");
    CL.ntiles = total;
    const int64_t grid = (a.mode == THETIS_MODE_ASYNC && a.async_ctas > 0) ? std::min<int64_t>(total, a.async_ctas)
                                                                         : total;
    k_color_step<<<(unsigned)grid, STEP_T, STEP_SMEM, s>>>(V, CL);
    TH_LAUNCHED();
  };
  if (a.mode == THETIS_MODE_ASYNC) {
    V.act_tiles = nullptr;  // the launches below merge colours: no per-colour tile lists
    V.act_off = nullptr;
    V.act_n = nullptr;
    // every class of every colour in one launch; slack rows as one range
    // (per-class launches keep the CTA shapes; they run back to back)
    for (int cls = 0; cls < UC_COUNT; ++cls) {
      ColorLaunch CL{};
      int64_t tot = 0;
      for (auto& cp : P.plan)
        for (auto& sg : cp.segs)
          if (sg.cls == cls) {
            if (CL.nseg == UC_COUNT + 1) {
              launch(CL, tot);
              CL = ColorLaunch{};
              tot = 0;
            }
            CL.seg[CL.nseg++] = SegLaunch{cls, sg.u0, sg.u1 - sg.u0, sg.c0, tot, sg.e0};
            tot += ctas_for(cls, sg.u1 - sg.u0, P.small_g);
          }
      launch(CL, tot);
    }
    if (P.Msl > 0) {
      ColorLaunch CL{};
      CL.seg[0] = SegLaunch{UC_COUNT, 0, P.Msl, 0, 0, 0};
      CL.nseg = 1;
      launch(CL, ctas_for(UC_COUNT, P.Msl, P.small_g));
    }
    TH_CUDA(cudaGetLastError());
    return;
  }
  ensure_tail(P);
  const int Ch = head_colours(P);
  for (int c = 0; c < Ch; ++c) {
    const ColorPlan& cp = P.plan[c];
    ColorLaunch CL{};
    CL.color = c;
    int64_t tot = 0;
    for (auto& sg : cp.segs) {
      CL.seg[CL.nseg++] = SegLaunch{sg.cls, sg.u0, sg.u1 - sg.u0, sg.c0, tot, sg.e0};
      tot += ctas_for(sg.cls, sg.u1 - sg.u0, P.small_g);
    }
    if (cp.srow1 > cp.srow0) {
      CL.seg[CL.nseg++] = SegLaunch{UC_COUNT, cp.srow0, cp.srow1 - cp.srow0, 0, tot, 0};
      tot += ctas_for(UC_COUNT, cp.srow1 - cp.srow0, P.small_g);
    }
    launch(CL, tot);
  }
  const TailView TV = make_tail_view(P);
  if (TV.n > 0) {
    const unsigned g = (unsigned)std::min<int64_t>(TV.n, 152 * 8);
    k_tail_partial<<<g, STEP_T, 0, s>>>(V, TV);
    TH_LAUNCHED();
    for (int tc = 0; tc < TV.ncol; ++tc) {
      k_tail_colour<<<TV.ctas, STEP_T, 0, s>>>(V, TV, tc);
      TH_LAUNCHED();
    }
    k_tail_scatter<<<g, STEP_T, 0, s>>>(V, TV);
    TH_LAUNCHED();
  }
  TH_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// persistent sweep: device plan, cooperative launch
// ---------------------------------------------------------------------------
static void ensure_sweep_plan(Problem& P) {
  if (P.d_plan && P.plan_g == P.small_g) return;
  const int C = P.ncolors;
  std::vector<ColorLaunch> h(C > 0 ? C : 1);
  std::vector<int64_t> nt(C > 0 ? C : 1, 0);
  for (int c = 0; c < C; ++c) {
    const ColorPlan& cp = P.plan[c];
    ColorLaunch CL{};
    CL.color = c;
    int64_t tot = 0;
    for (auto& sg : cp.segs) {
      CL.seg[CL.nseg++] = SegLaunch{sg.cls, sg.u0, sg.u1 - sg.u0, sg.c0, tot, sg.e0};
      tot += ctas_for(sg.cls, sg.u1 - sg.u0, P.small_g);
    }
    if (cp.srow1 > cp.srow0) {
      CL.seg[CL.nseg++] = SegLaunch{UC_COUNT, cp.srow0, cp.srow1 - cp.srow0, 0, tot, 0};
      tot += ctas_for(UC_COUNT, cp.srow1 - cp.srow0, P.small_g);
    }
    h[c] = CL;
    nt[c] = tot;
  }
  ColorLaunch* dp = P.mem.alloc<ColorLaunch>(h.size());
  int64_t* dn = P.mem.alloc<int64_t>(nt.size());
  TH_CUDA(cudaMemcpyAsync(dp, h.data(), h.size() * sizeof(ColorLaunch), cudaMemcpyHostToDevice, P.stream));
  TH_CUDA(cudaMemcpyAsync(dn, nt.data(), nt.size() * sizeof(int64_t), cudaMemcpyHostToDevice, P.stream));
  if (!P.bar) {
    P.bar = P.mem.alloc<unsigned>(64);  // [0]: grid barrier, [32]: tail-phase barrier (its own 128-byte line)
    P.err = P.mem.alloc<int>(1);
  }
  TH_CUDA(cudaMemsetAsync(P.bar, 0, 64 * sizeof(unsigned), P.stream));
  TH_CUDA(cudaMemsetAsync(P.err, 0, sizeof(int), P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  P.d_plan = dp;
  P.plan_g = P.small_g;
  P.d_ntiles = dn;
}

// The lean sweep serves problems whose head colours hold no long column (no
// shared-memory staging).
// (the tail colours run outside the colour loop: only the head colours count)
bool sweep_lean_possible(Problem& P) {
  ensure_tail(P);
  const int Ch = head_colours(P);
  for (int c = 0; c < Ch; ++c)
    for (auto& sg : P.plan[c].segs)
      if (sg.cls == UC_HUGE || sg.cls == UC_LARGE) return false;
  return true;
}

static bool sweep_lean(Problem& P) { return !P.force_full && sweep_lean_possible(P); }

// Grid of the cooperative sweep (0: not available on this device).
int sweep_grid(Problem& P) {
  if (P.sweep_grid >= 0) return P.sweep_grid;
  int dev = 0, coop = 0, sms = 0, per = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  TH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (sweep_lean(P)) TH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<false>, STEP_T, 0));
  else TH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<true>, STEP_T, STEP_SMEM));
  if (P.sweep_per_sm > 0 && P.sweep_per_sm < per) per = P.sweep_per_sm;
  P.sweep_grid = (coop && per > 0) ? sms * per : 0;
  return P.sweep_grid;
}

void reset_sweep_flags(Problem& P) {
  if (!P.bar) return;
  TH_CUDA(cudaMemsetAsync(P.bar, 0, 64 * sizeof(unsigned), P.stream));
  TH_CUDA(cudaMemsetAsync(P.err, 0, sizeof(int), P.stream));
}

// ---------------------------------------------------------------------------
// active tiles of a batch
// ---------------------------------------------------------------------------
// One warp per flat tile: 1 if any unit of the tile belongs to an unfinished
// instance (simplex blocks, absent from batches, always count as active).
__global__ void k_tile_flags(StepView V, const ColorLaunch* plan, const int64_t* tstart, int C, int64_t T,
                             int64_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = warp; f < T; f += nwarps) {
    const int c = (int)seg_find(tstart, C, f);
    const int64_t t = f - tstart[c];
    const ColorLaunch& CL = plan[c];
    int si = 0;
    while (si + 1 < CL.nseg && t >= CL.seg[si + 1].b0) ++si;
    const SegLaunch& S = CL.seg[si];
    const int64_t b = t - S.b0;
    int64_t u0 = 0, u1 = 0;
    bool rows = false, always = false;
    switch (S.cls) {
      case UC_HUGE:
      case UC_LARGE: u0 = b; u1 = b + 1; break;
      case UC_MED: u0 = b * (STEP_T / 32); u1 = u0 + STEP_T / 32; break;
      case UC_BLOCK: always = true; break;
      case UC_COUNT: u0 = b * (STEP_T * SLACK_ROWS); u1 = u0 + STEP_T * SLACK_ROWS; rows = true; break;
      default: {
        const int per = STEP_T / small_lanes(small_width(S.cls), V.small_g);
        u0 = b * per;
        u1 = u0 + per;
      }
    }
    if (u1 > S.n) u1 = S.n;
    bool any = always;
    for (int64_t u = u0 + lane; u < u1 && !any; u += 32) {
      const int32_t inst = rows ? V.inst_row[S.u0 + u] : V.inst_col[S.c0 + u];
      any = !V.frozen[inst];
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) cnt[f] = any ? 1 : 0;
  }
}

__global__ void k_tile_compact(const int64_t* cnt, const int64_t* pos, const int64_t* tstart, int C, int64_t T,
                               int32_t* act_tiles, int64_t* act_off, int64_t* act_n) {
  GSTRIDE(f, T) {
    if (cnt[f]) {
      const int c = (int)seg_find(tstart, C, f);
      act_tiles[pos[f]] = (int32_t)(f - tstart[c]);
    }
  }
  GSTRIDE(c, C) {
    act_off[c] = pos[tstart[c]];
    act_n[c] = pos[tstart[c + 1]] - pos[tstart[c]];
  }
}

void batch_active_tiles(Problem& P) {
  if (P.nbatch == 0 || P.ncolors == 0) return;
  ensure_sweep_plan(P);
  cudaStream_t s = P.stream;
  const int C = P.ncolors;
  if (P.act_g != P.small_g || !P.act_tiles) {
    std::vector<int64_t> nt(C), ts(C + 1, 0);
    TH_CUDA(cudaMemcpyAsync(nt.data(), P.d_ntiles, C * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < C; ++c) ts[c + 1] = ts[c] + nt[c];
    TH_CHECK(ts[C] < (int64_t(1) << 31), THETIS_E_INVALID, "too many tiles for the active-tile lists");
    P.tiles_total = ts[C];
    P.tile_start = P.mem.alloc<int64_t>(C + 1);
    P.act_tiles = P.mem.alloc<int32_t>(P.tiles_total + 1);
    P.act_off = P.mem.alloc<int64_t>(C);
    P.act_n = P.mem.alloc<int64_t>(C);
    P.act_cnt = P.mem.alloc<int64_t>(P.tiles_total + 1);
    P.act_pos = P.mem.alloc<int64_t>(P.tiles_total + 1);
    TH_CUDA(cudaMemcpyAsync(P.tile_start, ts.data(), (C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaStreamSynchronize(s));  // ts must outlive the copy
    P.act_g = P.small_g;
  }
  // the view's instance arrays (the step parameters do not matter here)
  StepView V{};
  V.inst_col = P.binst_col;
  V.inst_row = P.binst_row;
  V.frozen = P.bfrozen;
  V.small_g = P.small_g;
  const int64_t T = P.tiles_total;
  if (T > 0) {
    k_tile_flags<<<grid_for(T * 32, 256), 256, 0, s>>>(V, (const ColorLaunch*)P.d_plan, P.tile_start, C, T,
                                                       P.act_cnt);
    TH_LAUNCHED();
  }
  Arena tmp(s);
  exclusive_scan_i64(P.act_cnt, P.act_pos, T, tmp, s);
  k_tile_compact<<<grid_for(std::max<int64_t>(T, C), 256), 256, 0, s>>>(P.act_cnt, P.act_pos, P.tile_start, C, T,
                                                                        P.act_tiles, P.act_off, P.act_n);
  TH_LAUNCHED();
}

void run_sweep(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar, int epochs) {
  ensure_sweep_plan(P);
  const int grid = sweep_grid(P);
  TH_CHECK(grid > 0, THETIS_E_CUDA, "cooperative launch not available");
  ensure_tail(P);
  StepView V = make_view(P, a, use_ubar, use_xbar);
  const ColorLaunch* plan = (const ColorLaunch*)P.d_plan;
  const int64_t* nt = P.d_ntiles;
  int C = head_colours(P);
  TailView TV = make_tail_view(P);
  long long wait_ns = P.wait_ns;
  unsigned phantom = P.wait_phantom;
  void* args[] = {(void*)&V,      (void*)&plan,  (void*)&nt,    (void*)&C,       (void*)&epochs,
                  (void*)&P.bar, (void*)&P.err, (void*)&TV,    (void*)&wait_ns, (void*)&phantom};
  if (sweep_lean(P))
    TH_CUDA(cudaLaunchCooperativeKernel((const void*)k_sweep<false>, dim3(grid), dim3(STEP_T), args, 0, P.stream));
  else
    TH_CUDA(cudaLaunchCooperativeKernel((const void*)k_sweep<true>, dim3(grid), dim3(STEP_T), args, STEP_SMEM,
                                        P.stream));
  TH_LAUNCHED();
}

int sweep_error(Problem& P) {
  if (!P.err) return 0;
  int h = 0;
  TH_CUDA(cudaMemcpyAsync(&h, P.err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  return h;
}

// ---------------------------------------------------------------------------
// FP64 refresh and checks
// ---------------------------------------------------------------------------

// r = A x - b in FP64 (row by row over the internal CSR, plus the slack)
__global__ void k_refresh(const int64_t* rowptr, const uint32_t* colidx, const float* rval, const float* x,
                          const float* s, const int8_t* sig, const float* b, int64_t M, int64_t Msl,
                          double* r64, float* r) {
  GSTRIDE(i, M) {
    double acc = 0.0;
    if (rval) {
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) acc += (double)rval[q] * (double)x[colidx[q]];
    } else {
      // +-1 coefficients: a sign flip instead of a product
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const uint32_t e = colidx[q];
        const double xj = x[idx_of(e)];
        acc += (e & NEG_BIT) ? -xj : xj;
      }
    }
    if (i < Msl) acc += sig[i] > 0 ? (double)s[i] : -(double)s[i];
    acc -= (double)b[i];
    r64[i] = acc;
    r[i] = (float)acc;
  }
}

struct CheckView {
  const int64_t* colptr;
  const uint32_t* rowidx;
  const float* val;
  const float* csq;
  const float* x;
  const float* c;   // original c
  const float* ct;  // c - A^T ubar
  const float* xbar;
  const float* lo;
  const float* hi;
  float lo_u, hi_u;
  const double* r64;
  const float* s;
  const int8_t* sig;
  const float* cs;
  const float* sbar;
  const float* ubar;  // internal row order, or null
  double beta;
  int full;           // 0: rho only (an intermediate check); 1: also the objective, infeasibility and f_beta terms
  int k;
  int64_t Ncol;   // all internal structural columns
  int64_t Nfree;
  int64_t M, Msl;
  const int64_t* blk_start;  // internal column where a block starts (per block), or null
  int64_t nblk;
  const uint8_t* in_block;   // per free internal column: 1 if part of a block
  // batches: per-instance rho (FP64 bit patterns, atomic max); frozen
  // instances are skipped (their iterate no longer changes)
  const int32_t* inst_col;
  const int32_t* inst_row;
  const uint8_t* frozen;
  unsigned long long* inst_rho;
  // small columns through the ELL (thread per column), the other singleton
  // columns by segment (warp per column)
  const uint32_t* ell;
  const float* ellv;
  const int64_t* ss_start;
  const int64_t* ss_c0;
  const int64_t* ss_e0;
  const int32_t* ss_w;
  int64_t nss, nsmall;
  const int64_t* bs_start;
  const int64_t* bs_c0;
  int64_t nbs, nbig;
};



// max of non-negative doubles through their bit patterns (same order)
__device__ __forceinline__ void rho_max(unsigned long long* p, double v) {
  if (!(v > 0.0)) return;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (b > __ldcg(p)) atomicMax(p, b);
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// a_j^T r in FP64 (warp-wide) and ||a_j||^2 (= the non-zero count for +-1 columns)
__device__ __forceinline__ double col_dot64(const CheckView& V, int64_t j, int lane, double* sq) {
  const int64_t p0 = V.colptr[j], p1 = V.colptr[j + 1];
  double acc = 0.0, s2 = 0.0;
  if (V.val) {
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const double a = (double)V.val[p];
      acc += a * V.r64[V.rowidx[p]];
      s2 += a * a;
    }
    *sq = warp_sum_d(s2);
  } else {
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const uint32_t e = V.rowidx[p];
      const double rv = V.r64[idx_of(e)];
      acc += (e & NEG_BIT) ? -rv : rv;
    }
    *sq = (double)(p1 - p0);
  }
  return warp_sum_d(acc);
}

__global__ void __launch_bounds__(256) k_check(CheckView V, double* red) {
  // per-thread partials: rho(max), obj, infeas(max), rr, ur, xx
  double rho = 0.0, obj = 0.0, inf = 0.0, rr = 0.0, ur = 0.0, xx = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double beta = V.beta, ib = 1.0 / beta;
  const double inv_ls = 1.0 / (beta + ib);  // 1 / L of every slack column
  // (a1) small columns, thread per column through the ELL; a warp's columns
  // are consecutive (nearly always one batch instance: one atomic per warp)
  {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t tb = gt - lane; tb < V.nsmall; tb += gs) {
      const int64_t t = tb + lane;
      bool act = t < V.nsmall;
      double d = 0.0;
      int32_t inst = -1;
      if (act) {
        const int64_t k = seg_find(V.ss_start, V.nss, t);
        const int64_t p = t - V.ss_start[k], j = V.ss_c0[k] + p;
        const int W = V.ss_w[k];
        inst = V.frozen ? V.inst_col[j] : 0;
        if (V.frozen && V.frozen[inst]) {
          act = false;
          inst = -1;
        } else {
          const int64_t base = V.ss_e0[k] + (p >> 5) * 32 * W + (p & 31);
          double acc = 0.0, sq = 0.0;
          int nslot = 0;
          // four slots at a time (their loads overlap), summed in slot order;
          // slots fill from the front
          for (int qb = 0; qb < W; qb += 4) {
            uint32_t e[4];
            double a[4], rv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) e[t] = (qb + t < W) ? V.ell[base + (int64_t)(qb + t) * 32] : ELL_PAD;
            if (V.ellv) {
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (e[t] != ELL_PAD) {
                  a[t] = (double)V.ellv[base + (int64_t)(qb + t) * 32];
                  rv[t] = V.r64[e[t]];
                }
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (e[t] != ELL_PAD) {
                  acc += a[t] * rv[t];
                  sq += a[t] * a[t];
                }
            } else {
              // +-1 coefficients: a sign flip instead of a product, ||a||^2 =
              // the slot count (FP64 instructions are scarce on this part)
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (e[t] != ELL_PAD) rv[t] = V.r64[idx_of(e[t])];
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (e[t] != ELL_PAD) {
                  acc += (e[t] & NEG_BIT) ? -rv[t] : rv[t];
                  ++nslot;
                }
            }
            if (e[3] == ELL_PAD) break;
          }
          if (!V.ellv) sq = (double)nslot;
          const double xj = V.x[j], xb = V.xbar ? V.xbar[j] : 0.0;
          const double g = (double)V.ct[j] + beta * acc + (xj - xb) * ib;
          const double L = beta * sq + ib;
          const double lo = V.lo ? V.lo[j] : V.lo_u, hi = V.hi ? V.hi[j] : V.hi_u;
          d = fabs(fmin(fmax(xj - g / L, lo), hi) - xj);
          rho = fmax(rho, d);
        }
      }
      if (V.frozen) {
        const int32_t i0 = __shfl_sync(0xffffffffu, inst, 0);
        if (__all_sync(0xffffffffu, inst == i0)) {
          const double m = warp_max_d(d);
          if (lane == 0 && i0 >= 0) rho_max(V.inst_rho + i0, m);
        } else if (act) {
          rho_max(V.inst_rho + inst, d);
        }
      }
    }
  }
  // (a2) the other singleton columns, warp per column
  for (int64_t t = warp; t < V.nbig; t += nwarps) {
    const int64_t k = seg_find(V.bs_start, V.nbs, t);
    const int64_t j = V.bs_c0[k] + (t - V.bs_start[k]);
    const int32_t inst = V.frozen ? V.inst_col[j] : 0;
    if (V.frozen && V.frozen[inst]) continue;
    double sq;
    double atr = col_dot64(V, j, lane, &sq);
    double xj = V.x[j], xb = V.xbar ? V.xbar[j] : 0.0;
    double g = (double)V.ct[j] + beta * atr + (xj - xb) * ib;
    double L = beta * sq + ib;
    double lo = V.lo ? V.lo[j] : V.lo_u, hi = V.hi ? V.hi[j] : V.hi_u;
    double xn = fmin(fmax(xj - g / L, lo), hi);
    if (lane == 0) {
      rho = fmax(rho, fabs(xn - xj));
      if (V.frozen) rho_max(V.inst_rho + inst, fabs(xn - xj));
    }
  }
  // (b) simplex blocks, warp per block
  for (int64_t t = warp; t < V.nblk; t += nwarps) {
    int64_t j0 = V.blk_start[t];
    double yq = -INFINITY, xq = 0.0, sqmax = 0.0;
    double gl = 0.0;
    for (int q = 0; q < V.k; ++q) {
      double sq;
      double atr = col_dot64(V, j0 + q, lane, &sq);
      sqmax = fmax(sqmax, sq);
      if (lane == q) gl = atr;
    }
    double L = beta * sqmax + ib;
    if (lane < V.k) {
      xq = V.x[j0 + lane];
      double xb = V.xbar ? V.xbar[j0 + lane] : 0.0;
      double g = (double)V.ct[j0 + lane] + beta * gl + (xq - xb) * ib;
      yq = xq - g / L;
    }
    double cnt = 0.0, sum = 0.0;
    for (int i = 0; i < V.k; ++i) {
      double yi = __shfl_sync(0xffffffffu, yq, i);
      if (lane < V.k && yi >= yq) {
        cnt += 1.0;
        sum += yi;
      }
    }
    double theta = (lane < V.k) ? (sum - 1.0) / cnt : 0.0;
    bool ok = (lane < V.k) && (yq - theta > 0.0);
    int key = ok ? (int)cnt : 0;
    int best = key;
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    unsigned who = __ballot_sync(0xffffffffu, key == best && ok);
    double th = __shfl_sync(0xffffffffu, theta, __ffs(who) - 1);
    if (lane < V.k) rho = fmax(rho, fabs(fmax(yq - th, 0.0) - xq));
  }
  // (c) objective and proximal term over all structural columns
  if (V.full) GSTRIDE(j, V.Ncol) {
    double xj = V.x[j], xb = (V.xbar) ? V.xbar[j] : 0.0;
    obj += (double)V.c[j] * xj;
    xx += (xj - xb) * (xj - xb);
  }
  // (d) rows and slacks.  FP64 instructions are scarce on this part (a few
  // per clock per SM): maxima of non-negative values are taken on their bit
  // patterns (the same order), and the slack step without cs / sbar takes one
  // fused multiply-add for its gradient.
  {
    unsigned long long rho_b = 0, inf_b = 0;
    const bool plain = !V.cs && !V.sbar;
    GSTRIDE(i, V.M) {
      const double ri = V.r64[i];
      if (V.full) {
        inf_b = max(inf_b, (unsigned long long)__double_as_longlong(ri) & 0x7fffffffffffffffull);
        rr = fma(ri, ri, rr);
        if (V.ubar) ur += (double)V.ubar[i] * ri;
      }
      if (i < V.Msl) {
        const double sv = V.s[i];
        const double bsr = V.sig[i] > 0 ? beta * ri : -(beta * ri);  // beta * sign * r, sign = +-1
        double ds, g;
        if (plain) {
          ds = sv;
          g = fma(sv, ib, bsr);
        } else {
          ds = sv - (V.sbar ? (double)V.sbar[i] : 0.0);
          g = fma(ds, ib, (V.cs ? (double)V.cs[i] : 0.0) + bsr);
        }
        double sn = fma(-g, inv_ls, sv);
        if (__double_as_longlong(sn) < 0) sn = 0.0;  // max(., 0)
        const unsigned long long db = (unsigned long long)__double_as_longlong(sn - sv) & 0x7fffffffffffffffull;
        if (!V.frozen) {
          rho_b = max(rho_b, db);
        } else if (!V.frozen[V.inst_row[i]]) {
          rho_b = max(rho_b, db);
          rho_max(V.inst_rho + V.inst_row[i], __longlong_as_double((long long)db));
        }
        if (V.full) xx = fma(ds, ds, xx);
      }
    }
    rho = fmax(rho, __longlong_as_double((long long)rho_b));
    inf = fmax(inf, __longlong_as_double((long long)inf_b));
  }
  // block reduction, fixed order
  __shared__ double sm[NRED][8];
  double vals[NRED] = {warp_max_d(rho), warp_sum_d(obj), warp_max_d(inf), warp_sum_d(rr), warp_sum_d(ur),
                       warp_sum_d(xx)};
  const int w = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < NRED; ++q) sm[q][w] = vals[q];
  __syncthreads();
  if (threadIdx.x < NRED) {
    int q = threadIdx.x;
    double a = sm[q][0];
    for (int t = 1; t < 8; ++t) a = (q == 0 || q == 2) ? fmax(a, sm[q][t]) : a + sm[q][t];
    red[(int64_t)q * CHECK_BLOCKS + blockIdx.x] = a;
  }
}

// one warp per quantity: lane l folds partials l, l + 32, ... in order, then a
// fixed shuffle tree (the same order every call: deterministic)
__global__ void k_check_final(const double* red, double* out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= NRED) return;
  const bool mx = q == 0 || q == 2;
  double a = 0.0;  // maxima are of non-negative values
  for (int t = lane; t < CHECK_BLOCKS; t += 32) {
    const double v = red[(int64_t)q * CHECK_BLOCKS + t];
    a = mx ? fmax(a, v) : a + v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double b = __shfl_xor_sync(0xffffffffu, a, o);
    a = mx ? fmax(a, b) : a + b;
  }
  if (lane == 0) out[q] = a;
}

// ---------------------------------------------------------------------------
// solve preparation: ubar / xbar / x0 into internal order
// ---------------------------------------------------------------------------
__global__ void k_perm_rows_f(const float* src, const uint32_t* orig_of_row, int64_t M, float* dst) {
  GSTRIDE(i, M) dst[i] = src[orig_of_row[i]];
}

__global__ void k_ctil(const int64_t* colptr, const uint32_t* rowidx, const float* val, const float* c,
                       const float* ubar_int, int64_t N, float* ct) {
  GSTRIDE(j, N) {
    float acc = 0.f;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      uint32_t e = rowidx[p];
      float a = val ? val[p] : sgn_of(e);
      uint32_t row = val ? e : idx_of(e);
      acc = fmaf(a, ubar_int[row], acc);
    }
    ct[j] = c[j] - acc;
  }
}

__global__ void k_cs(const float* ubar_int, const int8_t* sig, int64_t Msl, float* cs) {
  GSTRIDE(i, Msl) cs[i] = -(float)sig[i] * ubar_int[i];
}

__global__ void k_xbar(const float* xbar, const uint32_t* col_of_orig, int64_t Ns, const uint32_t* slack_orig,
                       int64_t Msl, float* xb, float* sb) {
  GSTRIDE(j, Ns) xb[col_of_orig[j]] = xbar[j];
  GSTRIDE(t, Msl) sb[t] = xbar[Ns + slack_orig[t]];
}

__global__ void k_x0(const float* x0, const uint32_t* col_of_orig, int64_t Ns, int64_t Nfree, const float* lo,
                     const float* hi, float lo_u, float hi_u, const uint8_t* in_block, float* x) {
  GSTRIDE(j, Ns) {
    int64_t jj = col_of_orig[j];
    if (jj >= Nfree) continue;  // fixed columns keep their value
    float v = x0[j];
    if (!(in_block && in_block[jj])) {
      float l = lo ? lo[jj] : lo_u, h = hi ? hi[jj] : hi_u;
      v = fminf(fmaxf(v, l), h);
    }
    x[jj] = v;
  }
}

// initial point: singletons clip(0), blocks barycentre, fixed at lo; slacks 0
__global__ void k_init_x(int64_t Ncol, int64_t Nfree, const float* lo, const float* hi, float lo_u, float hi_u,
                         const uint8_t* in_block, int k, float* x) {
  GSTRIDE(j, Ncol) {
    float l = lo ? lo[j] : lo_u, h = hi ? hi[j] : hi_u;
    float v;
    if (j >= Nfree) v = l;
    else if (in_block && in_block[j]) v = 1.f / (float)k;
    else v = fminf(fmaxf(0.f, l), h);
    x[j] = v;
  }
}

__global__ void k_mark_blocks(const int64_t* blk_start, int64_t nblk, int k, uint8_t* in_block) {
  GSTRIDE(t, nblk)
  for (int q = 0; q < k; ++q) in_block[blk_start[t] + q] = 1;
}

static CheckView make_check_view(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar) {
  CheckView V;
  V.colptr = P.colptr;
  V.rowidx = P.rowidx;
  V.val = P.has_val ? P.val : nullptr;
  V.csq = P.csq;
  V.x = P.x;
  V.c = P.c;
  V.ct = use_ubar ? P.ctil : P.c;
  V.xbar = use_xbar ? P.xbar : nullptr;
  V.lo = P.bounds_uniform ? nullptr : P.lo;
  V.hi = P.bounds_uniform ? nullptr : P.hi;
  V.lo_u = P.lo_u;
  V.hi_u = P.hi_u;
  V.r64 = P.r64;
  V.s = P.s;
  V.sig = P.sig;
  V.cs = use_ubar ? P.cs : nullptr;
  V.sbar = use_xbar ? P.sbar : nullptr;
  V.ubar = use_ubar ? P.ubar_int : nullptr;
  V.beta = a.beta;
  V.k = P.k;
  V.Ncol = P.Ns;
  V.Nfree = P.Nfree;
  V.M = P.M;
  V.Msl = P.Msl;
  V.blk_start = P.blk_start;
  V.nblk = P.nblk;
  V.in_block = P.in_block;
  const bool batch = P.nbatch > 0 && P.bfrozen;
  V.inst_col = batch ? P.binst_col : nullptr;
  V.inst_row = batch ? P.binst_row : nullptr;
  V.frozen = batch ? P.bfrozen : nullptr;
  V.inst_rho = batch ? P.brho : nullptr;
  V.ell = P.ell;
  V.ellv = P.has_val ? P.ellv : nullptr;
  V.ss_start = P.ss_start;
  V.ss_c0 = P.ss_c0;
  V.ss_e0 = P.ss_e0;
  V.ss_w = P.ss_w;
  V.nss = P.nss;
  V.nsmall = P.nsmall;
  V.bs_start = P.bs_start;
  V.bs_c0 = P.bs_c0;
  V.nbs = P.nbs;
  V.nbig = P.nbig;
  return V;
}

void refresh_and_check(Problem& P, const SolveArgs& a, bool use_ubar, bool use_xbar, CheckOut& out, bool full,
                       bool refresh) {
  cudaStream_t s = P.stream;
  if (refresh && P.M > 0) {
    k_refresh<<<grid_for(P.M, 256, 152 * 64), 256, 0, s>>>(P.rowptr, P.colidx, P.has_val ? P.rval : nullptr, P.x,
                                                          P.s, P.sig, P.b, P.M, P.Msl, P.r64, P.r);
    TH_LAUNCHED();
  }
  if (refresh && P.nbatch > 0 && P.brho)
    TH_CUDA(cudaMemsetAsync(P.brho, 0, P.nbatch * sizeof(unsigned long long), s));
  CheckView V = make_check_view(P, a, use_ubar, use_xbar);
  V.full = full ? 1 : 0;
  k_check<<<CHECK_BLOCKS, 256, 0, s>>>(V, P.red);
  TH_LAUNCHED();
  k_check_final<<<1, 32 * NRED, 0, s>>>(P.red, P.red_out);
  TH_LAUNCHED();
  TH_CUDA(cudaMemcpyAsync(P.h_red, P.red_out, NRED * sizeof(double), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  const double* h = P.h_red;
  out.rho = h[0];
  if (full) {
    out.obj = h[1];
    out.infeas = h[2];
    out.fbeta = h[1] - h[4] + 0.5 * a.beta * h[3] + 0.5 / a.beta * h[5];
  }
}

// FP64 recompute of r only (start of a solve)
void refresh_only(Problem& P) {
  if (P.M <= 0) return;
  k_refresh<<<grid_for(P.M, 256, 152 * 64), 256, 0, P.stream>>>(P.rowptr, P.colidx, P.has_val ? P.rval : nullptr,
                                                                 P.x, P.s, P.sig, P.b, P.M, P.Msl, P.r64, P.r);
  TH_LAUNCHED();
  TH_CUDA(cudaGetLastError());
}

void prepare_solve(Problem& P, const float* d_ubar, const float* d_xbar, const float* d_x0) {
  cudaStream_t s = P.stream;
  if (d_ubar) {
    if (!P.ubar_int) {
      P.ubar_int = P.mem.alloc<float>(P.M);
      P.ctil = P.mem.alloc<float>(P.Ns);
      P.cs = P.mem.alloc<float>(P.Msl);
    }
    if (P.M > 0) {
      k_perm_rows_f<<<grid_for(P.M, 256), 256, 0, s>>>(d_ubar, P.orig_of_row, P.M, P.ubar_int);
      TH_LAUNCHED();
    }
    k_ctil<<<grid_for(P.Ns, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.has_val ? P.val : nullptr, P.c, P.ubar_int,
                                               P.Ns, P.ctil);
    TH_LAUNCHED();
    if (P.Msl > 0) {
      k_cs<<<grid_for(P.Msl, 256), 256, 0, s>>>(P.ubar_int, P.sig, P.Msl, P.cs);
      TH_LAUNCHED();
    }
  }
  if (d_xbar) {
    if (!P.xbar) {
      P.xbar = P.mem.alloc<float>(P.Ns);
      P.sbar = P.mem.alloc<float>(P.Msl);
    }
    k_xbar<<<grid_for(std::max(P.Ns, P.Msl), 256), 256, 0, s>>>(d_xbar, P.col_of_orig, P.Ns, P.slack_orig, P.Msl,
                                                                P.xbar, P.sbar);
    TH_LAUNCHED();
  }
  if (d_x0) {
    k_x0<<<grid_for(P.Ns, 256), 256, 0, s>>>(d_x0, P.col_of_orig, P.Ns, P.Nfree, P.bounds_uniform ? nullptr : P.lo,
                                             P.bounds_uniform ? nullptr : P.hi, P.lo_u, P.hi_u, P.in_block, P.x);
    TH_LAUNCHED();
  }
  TH_CUDA(cudaGetLastError());
}

__global__ void k_al_update(float* ubar, const double* r64, int64_t M, double beta, float* xbar, const float* x,
                            int64_t Ns, float* sbar, const float* s, int64_t Msl) {
  GSTRIDE(i, M > Ns ? M : Ns) {
    if (i < M) ubar[i] = (float)((double)ubar[i] - beta * r64[i]);
    if (i < Ns) xbar[i] = x[i];
    if (i < Msl) sbar[i] = s[i];
  }
}

void al_update(Problem& P, double beta) {
  cudaStream_t s = P.stream;
  TH_CHECK(P.ubar_int && P.xbar, THETIS_E_INVALID, "multiplier step without ubar / xbar state");
  const int64_t n = std::max(P.M, P.Ns);
  if (n > 0) {
    k_al_update<<<grid_for(n, 256), 256, 0, s>>>(P.ubar_int, P.r64, P.M, beta, P.xbar, P.x, P.Ns, P.sbar, P.s,
                                                 P.Msl);
    TH_LAUNCHED();
  }
  k_ctil<<<grid_for(P.Ns, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.has_val ? P.val : nullptr, P.c, P.ubar_int, P.Ns,
                                             P.ctil);
  TH_LAUNCHED();
  if (P.Msl > 0) {
    k_cs<<<grid_for(P.Msl, 256), 256, 0, s>>>(P.ubar_int, P.sig, P.Msl, P.cs);
    TH_LAUNCHED();
  }
}

__global__ void k_gather_rows_f(const float* src_int, const uint32_t* row_of_orig, int64_t M, float* dst) {
  GSTRIDE(i, M) dst[i] = src_int[row_of_orig[i]];
}

void gather_duals(Problem& P, float* out) {
  if (P.M <= 0) return;
  k_gather_rows_f<<<grid_for(P.M, 256), 256, 0, P.stream>>>(P.ubar_int, P.row_of_orig, P.M, out);
  TH_LAUNCHED();
}

void init_iterate(Problem& P) {
  cudaStream_t s = P.stream;
  if (P.nblk > 0 && !P.in_block) {
    P.in_block = P.mem.alloc<uint8_t>(P.Ns);
    TH_CUDA(cudaMemsetAsync(P.in_block, 0, P.Ns, s));
    k_mark_blocks<<<grid_for(P.nblk, 256), 256, 0, s>>>(P.blk_start, P.nblk, P.k, P.in_block);
    TH_LAUNCHED();
  }
  k_init_x<<<grid_for(P.Ns, 256), 256, 0, s>>>(P.Ns, P.Nfree, P.bounds_uniform ? nullptr : P.lo,
                                               P.bounds_uniform ? nullptr : P.hi, P.lo_u, P.hi_u, P.in_block, P.k,
                                               P.x);
  TH_LAUNCHED();
  if (P.Msl > 0) TH_CUDA(cudaMemsetAsync(P.s, 0, P.Msl * sizeof(float), s));
  refresh_only(P);
}

}  // namespace thetis
