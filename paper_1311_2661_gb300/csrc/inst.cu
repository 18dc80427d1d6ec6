// Instance-resident solve of a batch of vertex-cover / independent-set LPs
// (thetis_build_batch).
//
// The union sweep (scd.cu) advances every unfinished instance once per epoch,
// so each epoch streams the residual r of the whole batch (gigabytes) through
// HBM with scattered 4-byte accesses.  Here every instance is solved from
// start to stop by one CTA, or by one thread-block cluster of 2, 3 or 4 CTAs,
// that keeps the instance's residual r and iterate x in shared memory
// (distributed over the cluster's CTAs, reached with ld/st.shared::cluster):
//
//   * the colour classes of the instance are swept in order (Algorithm 1's
//     coordinate step, re-ordered by colour as in the union sweep: no two
//     units of a colour share a row), one CTA / cluster barrier per colour;
//   * every R epochs the residual is recomputed exactly from x and s and the
//     stopping test rho <= tol is made inside the kernel, so an instance stops
//     at the same check as its solve alone and frees its SM for the next
//     instance -- no host round trip, no grid barrier;
//   * only the instance's non-zero structure, c and the slack values stream
//     from memory (they stay in L2 while the instance runs).
//
// The exact recomputation r = Ax - b of a row x_u + x_v + sig s - 1 is done in
// 64-bit fixed point (2^-58 units: exact for every |value| < 8 down to 2^-58,
// with a plain FP64 fallback outside that range), then rounded once to FP32:
// the GB300 issues about two FP64 instructions per clock per SM, the integer
// pipes sixty-four.  The stopping test evaluates rho in FP32 from those exact
// sums with a rigorous error bound, and only units whose bound straddles tol
// are re-evaluated in FP64, so the decision is the FP64 decision.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <type_traits>

#include "problem.cuh"

namespace cg = cooperative_groups;

namespace thetis {

#define GSTRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

namespace {

constexpr uint32_t NO_ENTRY = 0xffffffffu;

// ELL slots of 16 bits, two a word, holding a shared-memory index: every
// cluster instance, and a one-CTA instance with m < 65535 (every instance
// that fits one CTA's shared memory is one); 32-bit local rows otherwise
__host__ __device__ __forceinline__ bool inst_ell16(int64_t K, int64_t m) { return K > 1 || m < 65535; }
constexpr int FIX = 58;                              // fixed point: value * 2^58
constexpr long long FIX_ONE = 1LL << FIX;
constexpr int FIX_SPLIT = 18;                        // column sums: high part in 2^-40 units, low 18 bits apart

// ---------------------------------------------------------------------------
// exact arithmetic helpers
// ---------------------------------------------------------------------------
// |f| < 8 (exponent below 130); false for inf / nan
__device__ __forceinline__ bool fix_ok(float f) { return ((__float_as_uint(f) >> 23) & 0xffu) < 130u; }

// f * 2^58 truncated toward zero, for |f| < 8 (exact when f's lowest mantissa
// bit is >= 2^-58, i.e. |f| >= 2^-35 or f a multiple of 2^-58)
__device__ __forceinline__ long long fix58(float f) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;  // zero or subnormal (< 2^-126)
  const long long mnt = (long long)((b & 0x7fffffu) | 0x800000u);  // f = mnt * 2^(e - 150)
  const int sh = e - 150 + FIX;
  long long v;
  if (sh >= 0) v = mnt << sh;
  else v = (-sh < 24) ? (mnt >> (-sh)) : 0;
  return (b >> 31) ? -v : v;
}

// the row value x_u + x_v + sig s - 1 in 2^-58 units (exact for |terms| < 8)
__device__ __forceinline__ long long row_fix(float xu, float xv, float s, float sig) {
  const long long fs = fix58(s);
  return fix58(xu) + fix58(xv) + (sig > 0.f ? fs : -fs) - FIX_ONE;
}
__device__ __forceinline__ double row_f64(float xu, float xv, float s, float sig) {
  return (((double)xu + (double)xv) + (double)sig * (double)s) - 1.0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// distributed shared memory of a cluster
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t dsm_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));  // pure: the compiler may reuse it
  return r;
}
__device__ __forceinline__ float dsm_ld(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ int dsm_ld_i(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

__device__ __forceinline__ double dsm_ld_d(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t dsm_ld_u(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void dsm_and(uint32_t a, uint32_t mask) {
  asm volatile("red.shared::cluster.and.b32 [%0], %1;" ::"r"(a), "r"(mask) : "memory");
}

// element b[i] of a small register array without dynamic indexing
template <int K>
__device__ __forceinline__ uint32_t pick(const uint32_t (&b)[K], uint32_t i) {
  uint32_t v = b[0];
#pragma unroll
  for (int r = 1; r < K; ++r) v = (i == (uint32_t)r) ? b[r] : v;
  return v;
}

struct InstView {
  const int64_t* noff;   // count + 1: first union vertex (= IML column) of every instance
  const int64_t* eoff;   // count + 1: first union edge (= IML row) of every instance
  const uint32_t* iend;  // per IML column: end of its entries, local to the instance
  const uint32_t* ient;  // per entry: local row
  const uint32_t* inb;   // per entry: local column of the other endpoint
  const uint32_t* iru;   // per IML row: its two local columns
  const uint32_t* irv;
  const int32_t* coff;   // count * C: first local column of every colour
  const int32_t* roff;   // count * 4 * C: first local slack row of every (rank, colour)
  const int32_t* qoff;   // count * 5: first local row of every rank (rows of rank q: [qoff[q], qoff[q + 1]))
  const int32_t* ncol;   // count: colours of the instance
  const int32_t* cwide;  // count * C: first local column of every colour with at most 32 entries
                         // (a colour's columns are sorted by length, longest first)
  const int64_t* pfirst; // count * C + 1: first ELL panel of every colour (panels of 32 short columns)
  const int64_t* pbase;  // per panel: first ELL slot (slot s of lane l at pbase + 32 s + l)
  const uint8_t* pw;     // per panel: slots (its longest column)
  const uint32_t* ell;   // ELL slots: shared-memory index of the row (16 bits, two a word; a cluster
                         // instance's rows of other ranks: their halo copies), or all ones; 32-bit local
                         // rows for a one-CTA instance of 65535 rows or more
  // cluster instances (K > 1): rank q keeps its rows in halo-group order --
  // first those no other rank's short column reads, then per (accessor rank
  // A, accessor colour c) the contiguous segment R(q, A, c)
  const uint32_t* rpos;  // per local row: its place in its rank's block of r
  const uint32_t* rrow;  // per place (rank block starts at qoff[q]): the local row
  const int32_t* hs;     // count * 4 * 4 * C: start of R(q, A, c) in rank q's block
  const int32_t* hl;     // count * 4 * 4 * C: its length
  const int32_t* hoff;   // count * 4 * C * 4: where R(A, q, c) sits in rank q's halo buffer of colour c
  const int32_t* hH;     // count: halo buffer length
  const uint8_t* hnb;    // count: halo buffers (2: colour parity, one barrier a colour; 1: two barriers)
  const uint8_t* xg;     // count: 1 when a cluster instance keeps x in global memory (so fewer CTAs hold r)
  const int32_t* ideg;   // count: longest column of the instance
  const uint8_t* kind;   // count: THETIS_ROUND_VC / _IS
  const float* c;        // IML column costs
  float* x;              // IML iterate (read at start, written at the end)
  float* s;              // IML slack values (updated in place)
  float* rg;             // IML rows: residual of the rows that do not fit in shared memory (one CTA)
  int C;                 // colour-table stride
  float beta, inv_beta, lo, hi;
  double beta_d;
  int step_rule;
  int epochs, R;
  double tol;
  int32_t* ep_out;
  int32_t* conv_out;
  unsigned long long* t_out;  // 2 per instance: start, done (globaltimer ns)
  // rounding inside the kernel (round != 0): repair + VC threshold / IS best
  // of reps with alterations + exact validity, as thetis_round_batch
  int round;
  uint64_t seed;
  int reps;
  const uint32_t* vid;   // per IML column: instance-local vertex id (the random streams' index)
  uint8_t* lab;          // labels by union vertex
  double* r_obj;         // count: objective of the rounded solution
  double* r_rep;         // count: repair value (eps or alpha)
  int32_t* r_best;       // count: winning repetition
  int32_t* r_status;     // count: 1 valid, 0 validity check failed, -1 VC repair impossible
  float* xout;           // union vertex order: the final x (rounding on)
  float* rho_out;        // count: rho at the last check (the largest unit value, FP32 from exact sums)
  int* done;             // count or null: set to 1 (system scope) once the instance's results are written
};

// ---------------------------------------------------------------------------
// the kernel: one instance per CTA (K = 1) or per cluster of K CTAs
// ---------------------------------------------------------------------------
// Rank q of the cluster holds the residual of its block of local rows
// [qoff[q], qoff[q + 1]) (each row kept by a rank that steps one of its two
// columns; in halo-group order, V.rpos) and the iterate of local columns k
// with k % K == q at x[k / K]; CSR entries name a row as (rank << 28) |
// place in the rank's block.  It steps its slack rows (local) and, per
// colour, either
//   G = 1: every K-th ELL panel of the colour's short columns (its own ones,
//          in stride K), one thread per column (slot addresses follow from the
//          panel; no index chain), and the colour's long columns one warp
//          each, or
//   G = 4 / 8 (one CTA only): its columns, G lanes each, through the CSR.
// A cluster's short columns read other ranks' rows from halo copies that the
// ranks exchange between colours (see halo); its long columns and the checks
// reach other ranks' r and x through distributed shared memory.
template <int K, int NT, int G, bool SPILL>
__global__ void __launch_bounds__(NT, (NT >= 1024) ? 1 : 1024 / NT) k_inst(InstView V, const int32_t* order) {
  static_assert(K == 1 || (G == 1 && !SPILL), "a cluster steps its short columns through ELL panels and halos");
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_over[2];
  __shared__ unsigned s_rho[2];  // the largest rho of the check (FP32 bits, non-negative)
  __shared__ int s_q[2];         // work counters of the colour sweep (colour parity)
  // the instance's colour table in shared memory (up to CM colours): first
  // panel (relative), first short column, first column, this rank's first
  // slack row
  constexpr int CM = 64;
  __shared__ int s_cm[4][CM + 1];
  __shared__ long long s_pf0;
  // a cluster rank's halo copies of the coming exchange: per direction (0:
  // changed copies back to their keepers, 1: the next colour's copies out)
  // and other rank, (length, source index, destination index)
  __shared__ int s_hd[2][4][3];
  constexpr int GC = (G == 1) ? 8 : G;  // lanes per column of the stopping test
  const int q = (K > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int t = order[blockIdx.x / K];
  const int64_t col0 = V.noff[t], row0 = V.eoff[t], ent0 = 2 * row0;
  const int n = (int)(V.noff[t + 1] - col0), m = (int)(V.eoff[t + 1] - row0);
  const bool ell16 = inst_ell16(K, m);
  // shared memory: r of the own rows, then x of the own columns.  SPILL (one
  // CTA, an instance that does not fit): x in global memory and the first rs
  // rows of r in shared memory, the rest in V.rg (L2)
  int cap = 0;
  if constexpr (SPILL) {
    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    cap = (int)(dyn_bytes / 4);
  }
  // this rank's block of rows, and the largest block (where x starts)
  int qv[5] = {0, m, m, m, m};
  int rch = m;
  if constexpr (K > 1) {
    rch = 0;
#pragma unroll
    for (int r = 0; r <= K; ++r) qv[r] = V.qoff[(int64_t)t * 5 + r];
#pragma unroll
    for (int r = 0; r < K; ++r) rch = max(rch, qv[r + 1] - qv[r]);
  }
  const int qlo = qv[q], qhi = qv[q + 1];
  // the r region also holds the rounding's two bit words per 32 own columns
  const int rr = max(rch, 2 * (((n + K - 1) / K + 31) / 32));
  const bool xs = SPILL ? (rr + n <= cap) : (K == 1 || V.xg[t] == 0);  // x in shared memory
  const int rs = SPILL ? min(m, cap) : rch;        // rows of r in shared memory (K = 1)
  float* sr = smem;
  float* sx = smem + rr;
  float* rgl = V.rg + row0;
  // cluster: the halo buffer(s) after x (after r when x is in global memory)
  const int hb = rr + (xs ? (n + K - 1) / K : 0);
  const int H = (K > 1) ? V.hH[t] : 0;
  const int nbuf = (K > 1) ? V.hnb[t] : 0;  // the halo buffer of colour c: hb + (nbuf == 2 ? (c & 1) H : 0)
  const uint32_t* Rpos = V.rpos + row0;
  // the instance's arrays (32-bit local indices from here on)
  float* Sx = V.x + col0;
  const float* Cc = V.c + col0;
  float* Ss = V.s + row0;
  const uint32_t* Iend = V.iend + col0;
  const uint32_t* Ient = V.ient + ent0;
  const uint32_t* Inb = V.inb + ent0;
  const uint32_t* Iru = V.iru + row0;
  const uint32_t* Irv = V.irv + row0;
  const int nc = V.ncol[t];
  const int32_t* coff = V.coff + (int64_t)t * V.C;
  const int32_t* roff = V.roff + ((int64_t)t * 4 + q) * V.C;
  const bool cm_ok = nc < CM;
  const float sig = (V.kind[t] == THETIS_ROUND_VC) ? -1.f : 1.f;
  // step rule 1: the instance's own global L_max (as its solve alone uses)
  float lfix = 0.f;
  if (V.step_rule == 1) {
    const int lm = max(V.ideg[t], m > 0 ? 1 : 0);
    lfix = (float)(V.beta_d * (double)lm + 1.0 / V.beta_d);
  }
  const float beta = V.beta, ib = V.inv_beta;
  const float tol32 = (float)V.tol;
  const float bsig = beta * sig;
  // 1 / L of a slack and of a column of every length up to 32 (the ELL path
  // multiplies by it instead of dividing: within one rounding of the quotient)
  __shared__ float s_invL[33];
  const float inv_ls = 1.f / ((lfix > 0.f) ? lfix : beta + ib);
  if (threadIdx.x <= 32) s_invL[threadIdx.x] = 1.f / ((lfix > 0.f) ? lfix : fmaf(beta, (float)threadIdx.x, ib));
  // rank r's copy of a shared-memory word of this CTA (mapped on use: no
  // registers held for the other ranks' bases)
  const uint32_t ra = smem_u32(sr), xa = smem_u32(sx);
  auto rget = [&](uint32_t e) -> float {
    if constexpr (SPILL) return ((int)e < rs) ? sr[e] : rgl[e];
    else if constexpr (K == 1) return sr[e];
    else return dsm_ld(dsm_map(ra + 4u * (e & 0x0fffffffu), e >> 28));
  };
  auto rset = [&](uint32_t e, float v) {
    if constexpr (SPILL) {
      if ((int)e < rs) sr[e] = v;
      else rgl[e] = v;
    } else if constexpr (K == 1) {
      sr[e] = v;
    } else {
      dsm_st(dsm_map(ra + 4u * (e & 0x0fffffffu), e >> 28), v);
    }
  };
  // local row of an entry's encoded row id
  auto row_of = [&](uint32_t e) -> uint32_t {
    if constexpr (K == 1) return e;
    else return V.rrow[row0 + V.qoff[(int64_t)t * 5 + (e >> 28)] + (e & 0x0fffffffu)];
  };
  auto xget = [&](uint32_t k) -> float {
    if constexpr (SPILL) return xs ? sx[k] : Sx[k];
    else if constexpr (K == 1) return sx[k];
    else return xs ? dsm_ld(dsm_map(xa + 4u * (k / K), k % K)) : __ldcg(Sx + k);  // L2: other ranks write it
  };
  auto xset = [&](uint32_t k, float v) {
    if constexpr (SPILL) {
      if (xs) sx[k] = v;
      else Sx[k] = v;
    } else if constexpr (K == 1) {
      sx[k] = v;
    } else {
      if (xs) dsm_st(dsm_map(xa + 4u * (k / K), k % K), v);
      else Sx[k] = v;
    }
  };
  // an own row e (local id in [qlo, qhi)) / own column k (k % K == q)
  auto rown_get = [&](int e) -> float {
    if constexpr (K == 1) return rget((uint32_t)e);
    else return sr[Rpos[e]];
  };
  auto rown_set = [&](int e, float v) {
    if constexpr (K == 1) rset((uint32_t)e, v);
    else sr[Rpos[e]] = v;
  };
  auto xown_get = [&](int k) -> float {
    if constexpr (K == 1) return xget((uint32_t)k);
    else return xs ? sx[k / K] : Sx[k];
  };
  auto xown_set = [&](int k, float v) {
    if constexpr (K == 1) {
      xset((uint32_t)k, v);
    } else {
      if (xs) sx[k / K] = v;
      else Sx[k] = v;
    }
  };
  auto sync = [&]() {
    if constexpr (K == 1) __syncthreads();
    else cg::this_cluster().sync();
  };

  // -- start: x chunk into shared memory, exact residual of the own rows -----
  if (xs)
    for (int i = threadIdx.x; i * K + q < n; i += NT) sx[i] = Sx[i * K + q];
  if (threadIdx.x < 2) {
    s_over[threadIdx.x] = 0;
    s_rho[threadIdx.x] = 0u;
    s_q[threadIdx.x] = 0;
  }
  if (cm_ok && threadIdx.x <= nc) {
    const int c = threadIdx.x;
    const int64_t f = (int64_t)t * V.C;
    if (c == 0) s_pf0 = V.pfirst[f];
    s_cm[0][c] = (int)(V.pfirst[f + c] - V.pfirst[f]);
    s_cm[1][c] = V.cwide[f + c];
    s_cm[2][c] = coff[c];
    s_cm[3][c] = roff[c];
  }
  if (threadIdx.x == 0 && q == 0) V.t_out[2 * t] = global_ns();
  sync();

  // refresh of the own rows (and, when chk, the slack part of the stopping
  // test into s_over[slot])
  auto rows_pass = [&](bool chk, int slot) {
    bool over = false;
    float rmax = 0.f;
#pragma unroll 2
    for (int e = qlo + (int)threadIdx.x; e < qhi; e += NT) {
      const float xu = xget(Iru[e]), xv = xget(Irv[e]);
      const float sv = Ss[e];
      const bool ex = fix_ok(xu) && fix_ok(xv) && fix_ok(sv);
      long long rf = 0;
      float r32;
      if (ex) {
        rf = row_fix(xu, xv, sv, sig);
        r32 = __ll2float_rn(rf) * 0x1p-58f;
      } else {
        r32 = (float)row_f64(xu, xv, sv, sig);
      }
      rown_set(e, r32);
      if (!chk) continue;
      // slack unit: rho = |max(0, s - grad / L) - s|, L = beta + 1/beta
      const float ls = beta + ib;
      const float g = fmaf(beta * sig, r32, sv * ib);
      const float qv = g / ls;
      const float rho = fabsf(fmaxf(sv - qv, 0.f) - sv);
      rmax = fmaxf(rmax, rho);
      if (over) continue;
      const float del = 0x1p-19f * ((beta * fabsf(r32) + sv * ib) / ls + fabsf(sv) + fabsf(qv)) + 0x1p-23f * tol32 +
                        1e-30f;
      if (!(rho - del <= tol32)) {  // over tol (or not finite)
        over = true;
      } else if (rho + del > tol32) {  // too close to tol for FP32: decide in FP64
        const double r64 = ex ? (double)rf * 0x1p-58 : row_f64(xu, xv, sv, sig);
        const double bd = V.beta_d, ibd = 1.0 / bd;
        const double bsr = sig > 0.f ? bd * r64 : -(bd * r64);
        const double g64 = fma((double)sv, ibd, bsr);
        double sn = fma(-g64, 1.0 / (bd + ibd), (double)sv);
        if (sn < 0.0) sn = 0.0;
        if (fabs(sn - (double)sv) > V.tol) over = true;
      }
    }
    if (over) atomicOr(&s_over[slot], 1);
    if (chk && rmax > 0.f) atomicMax(&s_rho[slot], __float_as_uint(rmax));
  };

  // the column part of the stopping test.  a_j^T r is summed in FP32 from
  // the refreshed row values (each the exact row value rounded once), so
  // |sum - a_j^T r| <= 2^-23 (deg + 2) sum |r_i| bounds it; rho is decided
  // from that estimate unless it lies within the bound of tol, and then from
  // the exact sum (2^-58 fixed point) in FP64.
  auto col_decide = [&](int k, float xk, float ck, float sum, float sabs, int deg, bool& over, float& rmax) {
    const float L = fmaf(beta, (float)deg, ib);
    const float g = ck + beta * sum + xk * ib;
    const float qv = g / L;
    const float rho = fabsf(fminf(fmaxf(xk - qv, V.lo), V.hi) - xk);
    rmax = fmaxf(rmax, rho);
    if (over) return;
    const float esum = 0x1p-22f * (float)(deg + 2) * sabs;  // twice the bound above
    const float del = 0x1p-19f * ((fabsf(ck) + beta * fabsf(sum) + fabsf(xk) * ib) / L + fabsf(xk) + fabsf(qv)) +
                      beta * esum / L + 0x1p-23f * tol32 + 1e-30f;
    if (!(rho - del <= tol32)) {  // over tol (or not finite)
      over = true;
    } else if (rho + del > tol32) {  // too close to tol for FP32: the exact sum, FP64
      const uint32_t p0 = (k == 0) ? 0u : Iend[k - 1], p1 = Iend[k];
      long long hi = 0, lo = 0;
      bool bad = !fix_ok(xk);
      const long long fk = fix58(xk);
      double sum64 = 0.0;
      for (uint32_t p = p0; p < p1; ++p) {
        const uint32_t e = row_of(Ient[p]);
        const float xw = xget(Inb[p]);
        const float sv = __ldcg(Ss + e);
        sum64 += row_f64(xk, xw, sv, sig);  // used when some value is outside the fixed-point range
        if (!(fix_ok(xw) && fix_ok(sv))) bad = true;
        const long long fs = fix58(sv);
        const long long rf = fk + fix58(xw) + (sig > 0.f ? fs : -fs) - FIX_ONE;
        hi += rf >> FIX_SPLIT;
        lo += rf & ((1LL << FIX_SPLIT) - 1);
      }
      if (!bad) sum64 = (double)hi * 0x1p-40 + (double)lo * 0x1p-58;
      const double bd = V.beta_d, ibd = 1.0 / bd;
      const double g64 = (double)ck + bd * sum64 + (double)xk * ibd;
      const double L64 = bd * (double)deg + ibd;
      const double xn = fmin(fmax((double)xk - g64 / L64, (double)V.lo), (double)V.hi);
      if (fabs(xn - (double)xk) > V.tol) over = true;
    }
  };
  // the columns [ka, kb) of this rank through the CSR, GC lanes each
  auto cols_csr = [&](int ka, int kb, bool& over, float& rmax) {
    const int first = ka + ((q - ka % K) % K + K) % K;
    const int cnt = (first < kb) ? (kb - first + K - 1) / K : 0;
    constexpr int PW = 32 / GC;
    const int warp = threadIdx.x >> 5, lw = (threadIdx.x & 31) / GC, gl = threadIdx.x % GC;
    for (int ib0 = warp * PW; ib0 < cnt; ib0 += (NT / 32) * PW) {
      const int i = ib0 + lw;
      const bool valid = i < cnt;
      const int k = first + i * K;
      uint32_t p0 = 0, p1 = 0;
      float xk = 0.f, ck = 0.f;
      if (valid) {
        p0 = (k == 0) ? 0u : Iend[k - 1];
        p1 = Iend[k];
        xk = xown_get(k);
        ck = Cc[k];
      }
      float sum = 0.f, sabs = 0.f;
      for (uint32_t p = p0 + gl; p < p1; p += 4 * GC) {
        uint32_t et[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) et[v] = (p + v * GC < p1) ? Ient[p + v * GC] : NO_ENTRY;
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (et[v] != NO_ENTRY) {
            const float rv = rget(et[v]);
            sum += rv;
            sabs += fabsf(rv);
          }
      }
#pragma unroll
      for (int o = GC / 2; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o, GC);
        sabs += __shfl_xor_sync(0xffffffffu, sabs, o, GC);
      }
      if (!valid || gl != 0) continue;
      col_decide(k, xk, ck, sum, sabs, (int)(p1 - p0), over, rmax);
    }
  };
  // one CTA with 16-bit ELL panels: per colour its long columns through the
  // CSR and its short ones a thread each through the panels (the sweep's
  // gather without the step; a cluster reads the other ranks' rows through
  // the CSR, its halo copies being stale here)
  auto cols_check = [&](int slot) {
    bool over = false;
    float rmax = 0.f;
    if constexpr (K == 1 && G == 1) {
      if (!ell16) {
        cols_csr(0, n, over, rmax);
      } else {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        constexpr uint32_t NO16 = 0xffffu;
        for (int c = 0; c < nc; ++c) {
          int64_t pf;
          int np, cw, cend, cst;
          if (cm_ok) {
            pf = s_pf0 + s_cm[0][c];
            np = s_cm[0][c + 1] - s_cm[0][c];
            cw = s_cm[1][c];
            cst = s_cm[2][c];
            cend = s_cm[2][c + 1];
          } else {
            pf = V.pfirst[(int64_t)t * V.C + c];
            np = (int)(V.pfirst[(int64_t)t * V.C + c + 1] - pf);
            cw = V.cwide[(int64_t)t * V.C + c];
            cst = coff[c];
            cend = coff[c + 1];
          }
          if (cw > cst) cols_csr(cst, cw, over, rmax);
          for (int j = warp; j < np; j += NT / 32) {
            const uint32_t* pe = V.ell + V.pbase[pf + j] + lane;
            const int WW = (V.pw[pf + j] + 1) >> 1;
            const int k = cw + 32 * j + lane;
            float sum = 0.f, sabs = 0.f;
            int deg = 0;
            auto take = [&](uint32_t e) {
              if (e != NO16) {
                const float rv = rget(e);
                sum += rv;
                sabs += fabsf(rv);
                ++deg;
              }
            };
            for (int u0 = 0; u0 < WW; u0 += 4) {
              uint32_t et[4];
#pragma unroll
              for (int v = 0; v < 4; ++v) et[v] = (u0 + v < WW) ? pe[32 * (u0 + v)] : NO_ENTRY;
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                take(et[v] & 0xffffu);
                take(et[v] >> 16);
              }
            }
            if (k < cend) col_decide(k, xget((uint32_t)k), Cc[k], sum, sabs, deg, over, rmax);
          }
        }
      }
    } else {
      cols_csr(0, n, over, rmax);
    }
    if (over) atomicOr(&s_over[slot], 1);
    if (rmax > 0.f) atomicMax(&s_rho[slot], __float_as_uint(rmax));
  };

  // columns [ka, kb) of this rank (k % K == q) through the CSR, GG lanes each
  auto csr_columns = [&](auto gg, int ka, int kb) {
    constexpr int GG = decltype(gg)::value;
    constexpr int NC = 32 / GG;  // entries a lane keeps in registers between gather and scatter
    const int first = ka + ((q - ka % K) % K + K) % K;
    const int cnt = (first < kb) ? (kb - first + K - 1) / K : 0;
    constexpr int PW = 32 / GG;
    const int warp = threadIdx.x >> 5, lw = (threadIdx.x & 31) / GG, gl = threadIdx.x % GG;
    for (int ib0 = warp * PW; ib0 < cnt; ib0 += (NT / 32) * PW) {
      const int i = ib0 + lw;
      const bool valid = i < cnt;
      const int k = first + i * K;
      uint32_t p0 = 0, p1 = 0;
      float xk = 0.f, ck = 0.f;
      if (valid) {
        p0 = (k == 0) ? 0u : Iend[k - 1];
        p1 = Iend[k];
        xk = xown_get(k);
        ck = Cc[k];
      }
      uint32_t ce[NC];
      float cr[NC];
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const uint32_t p = p0 + gl + (uint32_t)(u * GG);
        ce[u] = (p < p1) ? Ient[p] : NO_ENTRY;
      }
#pragma unroll
      for (int u = 0; u < NC; ++u) cr[u] = (ce[u] != NO_ENTRY) ? rget(ce[u]) : 0.f;
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < NC; ++u) acc += cr[u];
      for (uint32_t p = p0 + gl + NC * GG; p < p1; p += 4 * GG) {
        uint32_t et[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) et[v] = (p + v * GG < p1) ? Ient[p + v * GG] : NO_ENTRY;
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (et[v] != NO_ENTRY) acc += rget(et[v]);
      }
#pragma unroll
      for (int o = GG / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, GG);
      if (!valid) continue;
      const float g = ck + beta * acc + xk * ib;
      const float L = (lfix > 0.f) ? lfix : fmaf(beta, (float)(p1 - p0), ib);
      const float xn = fminf(fmaxf(xk - g / L, V.lo), V.hi);
      const float d = xn - xk;
      if (gl == 0) xown_set(k, xn);
      if (d != 0.f) {
#pragma unroll
        for (int u = 0; u < NC; ++u)
          if (ce[u] != NO_ENTRY) rset(ce[u], cr[u] + d);
        for (uint32_t p = p0 + gl + NC * GG; p < p1; p += 4 * GG) {
          uint32_t et[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) et[v] = (p + v * GG < p1) ? Ient[p + v * GG] : NO_ENTRY;
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (et[v] != NO_ENTRY) rset(et[v], rget(et[v]) + d);
        }
      }
    }
  };

  // the short columns of colour c in ELL panels, one panel per warp, one
  // column per lane.  Rank q's panels (every K-th) hold its own columns of the
  // colour (k % K == q) in stride K, so x and the rows kept by k's rank are
  // local to it.
  auto ell_columns = [&](int c) {
    constexpr int NE = (K > 1) ? 4 : 8;  // slots kept in registers between gather and scatter
    constexpr int NB = 4;  // slots beyond NE: loaded NB at a time (independent loads in flight)
    const int64_t pf = V.pfirst[(int64_t)t * V.C + c];
    const int np = (int)(V.pfirst[(int64_t)t * V.C + c + 1] - pf);
    const int cw = V.cwide[(int64_t)t * V.C + c], cend = coff[c + 1];
    const int first = cw + ((q - cw % K) % K + K) % K;  // this rank's first short column
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = q + K * warp; j < np; j += K * (NT / 32)) {
      const uint32_t* pe = V.ell + V.pbase[pf + j] + lane;
      const int W = V.pw[pf + j];
      const int k = first + K * (32 * (j / K) + lane);
      uint32_t ce[NE];
      float cr[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) ce[u] = (u < W) ? pe[32 * u] : NO_ENTRY;
      const bool valid = k < cend;
      const float xk = valid ? xown_get(k) : 0.f;
      const float ck = valid ? Cc[k] : 0.f;
#pragma unroll
      for (int u = 0; u < NE; ++u) cr[u] = (ce[u] != NO_ENTRY) ? rget(ce[u]) : 0.f;
      float acc = 0.f;
      int deg = 0;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        acc += cr[u];
        deg += (ce[u] != NO_ENTRY) ? 1 : 0;
      }
      for (int u0 = NE; u0 < W; u0 += NB) {
        uint32_t et[NB];
#pragma unroll
        for (int v = 0; v < NB; ++v) et[v] = (u0 + v < W) ? pe[32 * (u0 + v)] : NO_ENTRY;
#pragma unroll
        for (int v = 0; v < NB; ++v)
          if (et[v] != NO_ENTRY) {
            acc += rget(et[v]);
            ++deg;
          }
      }
      if (!valid) continue;
      const float g = ck + beta * acc + xk * ib;
      const float xn = fminf(fmaxf(xk - g * s_invL[deg], V.lo), V.hi);
      const float d = xn - xk;
      xown_set(k, xn);
      if (d != 0.f) {
#pragma unroll
        for (int u = 0; u < NE; ++u)
          if (ce[u] != NO_ENTRY) rset(ce[u], cr[u] + d);
        for (int u0 = NE; u0 < W; u0 += NB) {
          uint32_t et[NB];
#pragma unroll
          for (int v = 0; v < NB; ++v) et[v] = (u0 + v < W) ? pe[32 * (u0 + v)] : NO_ENTRY;
#pragma unroll
          for (int v = 0; v < NB; ++v)
            if (et[v] != NO_ENTRY) rset(et[v], rget(et[v]) + d);
        }
      }
    }
  };

  // one slack row: its projected step (the row is this rank's)
  auto slack_row = [&](int e, float sv, float rv) {
    const float g = bsig * rv + sv * ib;
    const float sn = fmaxf(sv - g * inv_ls, 0.f);
    const float d = sn - sv;
    Ss[e] = sn;
    if (d != 0.f) rown_set(e, rv + sig * d);
  };
  // the slack rows [ra, rb2) of a colour, four per thread at a time
  auto slack_rows = [&](int ra, int rb2) {
    constexpr int SR = 4;
    for (int e0 = ra + (int)threadIdx.x; e0 < rb2; e0 += SR * NT) {
      float sv[SR], rv[SR];
#pragma unroll
      for (int u = 0; u < SR; ++u) {
        const int e = e0 + u * NT;
        sv[u] = (e < rb2) ? Ss[e] : 0.f;
        rv[u] = (e < rb2) ? rown_get(e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < SR; ++u)
        if (e0 + u * NT < rb2) slack_row(e0 + u * NT, sv[u], rv[u]);
    }
  };

  // a colour through 16-bit ELL panels, two slots a word, so twice the slots
  // per load and per register (the scatter re-reads r: no other column of the
  // colour touches the row).  A slot is the row's index in shared memory: for
  // a cluster rank its own row or the halo copy of another rank's row, so the
  // sweep makes no remote access.  The warps pull the work -- this rank's
  // panels (widest first), then chunks of 128 slack rows -- from a counter in
  // shared memory, so a warp with a narrow panel goes on to the next item
  // instead of waiting at the colour's barrier.
  int seq = 0;  // colours swept so far: the counter of colour step seq is s_q[seq & 1]
  auto colour16 = [&](int c) {
    constexpr int NW = 5;  // words (10 slots) kept in registers between gather and scatter
    constexpr int NB = 4;  // words beyond NW: loaded NB at a time
    constexpr int CH = 128;  // slack rows an item
    constexpr uint32_t NO16 = 0xffffu;
    int64_t pf;
    int np, cw, cend, ra, rb2;
    if (cm_ok) {
      pf = s_pf0 + s_cm[0][c];
      np = s_cm[0][c + 1] - s_cm[0][c];
      cw = s_cm[1][c];
      cend = s_cm[2][c + 1];
      ra = s_cm[3][c];
      rb2 = s_cm[3][c + 1];
    } else {
      pf = V.pfirst[(int64_t)t * V.C + c];
      np = (int)(V.pfirst[(int64_t)t * V.C + c + 1] - pf);
      cw = V.cwide[(int64_t)t * V.C + c];
      cend = coff[c + 1];
      ra = roff[c];
      rb2 = roff[c + 1];
    }
    const int first = cw + ((q - cw % K) % K + K) % K;  // this rank's first short column
    const int npq = (np > q) ? (np - q + K - 1) / K : 0;  // this rank's panels: q + K jj
    const int nit = npq + (rb2 - ra + CH - 1) / CH;
    const int lane = threadIdx.x & 31;
    int* ctr = &s_q[seq & 1];
    if (threadIdx.x == 0) s_q[(seq + 1) & 1] = 0;  // the next colour's counter (last used a barrier ago)
    ++seq;
    auto lr = [&](uint32_t e) -> float {
      if constexpr (SPILL) return rget(e);
      else return smem[e];
    };
    auto lw = [&](uint32_t e, float v) {
      if constexpr (SPILL) rset(e, v);
      else smem[e] = v;
    };
    // a warp holds the next item it will take, and that panel's slot base
    // and width, while it works on the current one
    auto pull = [&]() {
      int v = 0;
      if (lane == 0) v = atomicAdd(ctr, 1);
      return __shfl_sync(0xffffffffu, v, 0);
    };
    int nx = pull();
    int64_t nx_base = 0;
    int nx_w = 0;
    if (nx < npq) {
      nx_base = V.pbase[pf + q + K * nx];
      nx_w = V.pw[pf + q + K * nx];
    }
    for (;;) {
      const int it = nx;
      if (it >= nit) break;
      const int64_t pbase = nx_base;
      const int pw = nx_w;
      nx = pull();
      if (nx < npq) {
        nx_base = V.pbase[pf + q + K * nx];
        nx_w = V.pw[pf + q + K * nx];
      }
      if (it >= npq) {  // slack rows
        const int e0 = ra + (it - npq) * CH + lane;
        float sv[CH / 32], rv[CH / 32];
#pragma unroll
        for (int u = 0; u < CH / 32; ++u) {
          const int e = e0 + 32 * u;
          sv[u] = (e < rb2) ? Ss[e] : 0.f;
          rv[u] = (e < rb2) ? rown_get(e) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < CH / 32; ++u)
          if (e0 + 32 * u < rb2) slack_row(e0 + 32 * u, sv[u], rv[u]);
        continue;
      }
      const uint32_t* pe = V.ell + pbase + lane;
      const int WW = (pw + 1) >> 1;
      const int k = first + K * (32 * it + lane);
      uint32_t ce[NW];
#pragma unroll
      for (int u = 0; u < NW; ++u) ce[u] = (u < WW) ? pe[32 * u] : NO_ENTRY;
      const bool valid = k < cend;
      const float xk = valid ? xown_get(k) : 0.f;
      const float ck = valid ? Cc[k] : 0.f;
      float acc = 0.f;
      int deg = 0;
      auto take = [&](uint32_t e) {
        if (e != NO16) {
          acc += lr(e);
          ++deg;
        }
      };
#pragma unroll
      for (int u = 0; u < NW; ++u) {
        take(ce[u] & 0xffffu);
        take(ce[u] >> 16);
      }
      for (int u0 = NW; u0 < WW; u0 += NB) {
        uint32_t et[NB];
#pragma unroll
        for (int v = 0; v < NB; ++v) et[v] = (u0 + v < WW) ? pe[32 * (u0 + v)] : NO_ENTRY;
#pragma unroll
        for (int v = 0; v < NB; ++v) {
          take(et[v] & 0xffffu);
          take(et[v] >> 16);
        }
      }
      if (!valid) continue;
      const float g = ck + beta * acc + xk * ib;
      const float xn = fminf(fmaxf(xk - g * s_invL[deg], V.lo), V.hi);
      const float d = xn - xk;
      xown_set(k, xn);
      if (d != 0.f) {
        auto put = [&](uint32_t e) {
          if (e != NO16) lw(e, lr(e) + d);
        };
#pragma unroll
        for (int u = 0; u < NW; ++u) {
          put(ce[u] & 0xffffu);
          put(ce[u] >> 16);
        }
        for (int u0 = NW; u0 < WW; u0 += NB) {
          uint32_t et[NB];
#pragma unroll
          for (int v = 0; v < NB; ++v) et[v] = (u0 + v < WW) ? pe[32 * (u0 + v)] : NO_ENTRY;
#pragma unroll
          for (int v = 0; v < NB; ++v) {
            put(et[v] & 0xffffu);
            put(et[v] >> 16);
          }
        }
      }
    }
  };

  // one colour: its long columns (a warp each), then its short columns and
  // slack rows
  auto sweep_colour = [&](int c) {
    if constexpr (G == 1) {
      const int cw = V.cwide[(int64_t)t * V.C + c];
      if (cw > coff[c]) csr_columns(std::integral_constant<int, 32>{}, coff[c], cw);
      if (SPILL && !ell16) {
        ell_columns(c);
        slack_rows(roff[c], roff[c + 1]);
      } else {
        colour16(c);
      }
    } else {
      csr_columns(std::integral_constant<int, G>{}, coff[c], coff[c + 1]);
      slack_rows(roff[c], roff[c + 1]);
    }
  };

  // halo exchange of a cluster instance, between the colour's sweep and its
  // cluster barrier: the halo copies of other ranks' rows that this rank's
  // colour-c short columns changed go back to their keepers (c >= 0), and
  // this rank's rows that other ranks' colour-cin short columns read go to
  // their halo buffers (cin >= 0).  Each is one contiguous segment per pair
  // of ranks (distributed shared memory moves those an order of magnitude
  // faster than scattered words).  Neither touches a row any rank steps in
  // colour c, so the copies overlap the other ranks' sweeps.
  // The descriptors are read from global memory into s_hd by halo_desc at
  // the start of the colour, so their latency hides behind the sweep (the
  // barrier before the exchange publishes them).
  auto halo_desc = [&](int c, int cin) {
    if constexpr (K > 1) {
      if (threadIdx.x < 8) {
        const int dir = threadIdx.x >> 2, A = threadIdx.x & 3;
        const int64_t C1 = V.C;
        int len = 0, src = 0, dst = 0;
        if (A < K && A != q) {
          if (dir == 0 && c >= 0) {
            len = V.hl[(((int64_t)t * 4 + A) * 4 + q) * C1 + c];
            src = hb + ((nbuf == 2) ? (c & 1) * H : 0) + V.hoff[(((int64_t)t * 4 + q) * C1 + c) * 4 + A];
            dst = V.hs[(((int64_t)t * 4 + A) * 4 + q) * C1 + c];
          } else if (dir == 1 && cin >= 0) {
            len = V.hl[(((int64_t)t * 4 + q) * 4 + A) * C1 + cin];
            src = V.hs[(((int64_t)t * 4 + q) * 4 + A) * C1 + cin];
            dst = hb + ((nbuf == 2) ? (cin & 1) * H : 0) + V.hoff[(((int64_t)t * 4 + A) * C1 + cin) * 4 + q];
          }
        }
        s_hd[dir][A][0] = len;
        s_hd[dir][A][1] = src;
        s_hd[dir][A][2] = dst;
      }
    }
  };
  auto halo = [&](bool out, bool in) {
    if constexpr (K > 1) {
#pragma unroll
      for (int A = 0; A < K; ++A) {
        if (A == q) continue;
        if (out) {  // halo copies (after r and x) -> rank A's rows
          const int len = s_hd[0][A][0];
          const float* src = smem + s_hd[0][A][1];
          const uint32_t dst = dsm_map(ra + 4u * (uint32_t)s_hd[0][A][2], (uint32_t)A);
          for (int i = threadIdx.x; i < len; i += NT) dsm_st(dst + 4u * i, src[i]);
        }
        if (in) {  // own rows -> rank A's halo buffer
          const int len = s_hd[1][A][0];
          const float* src = sr + s_hd[1][A][1];
          const uint32_t dst = dsm_map(smem_u32(smem + s_hd[1][A][2]), (uint32_t)A);
          for (int i = threadIdx.x; i < len; i += NT) dsm_st(dst + 4u * i, src[i]);
        }
      }
    }
  };

  // a check: exact refresh + stopping test; true when some unit has rho > tol
  int nchk = 0;
  float last_rho = 0.f;
  // (last: no epoch follows, so rho itself is reported; otherwise the column
  // part is skipped once a slack row is over tol)
  auto check = [&](bool last) -> bool {
    const int slot = nchk & 1;
    ++nchk;
    rows_pass(true, slot);
    sync();  // every rank's rows refreshed before the columns read them
    bool skip = false;
    if constexpr (K == 1) {
      skip = !last && s_over[slot] != 0;
    } else if (!last) {
#pragma unroll
      for (int r = 0; r < K; ++r) skip |= dsm_ld_i(dsm_map(smem_u32(&s_over[slot]), (uint32_t)r)) != 0;
    }
    if (!skip) cols_check(slot);
    sync();
    int over = 0;
    unsigned rb_ = 0;
    if constexpr (K == 1) {
      over = s_over[slot];
      rb_ = s_rho[slot];
    } else {
      const uint32_t fa = smem_u32(&s_over[slot]), ra_ = smem_u32(&s_rho[slot]);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        over |= dsm_ld_i(dsm_map(fa, (uint32_t)r));
        rb_ = max(rb_, (unsigned)dsm_ld_i(dsm_map(ra_, (uint32_t)r)));
      }
    }
    last_rho = __uint_as_float(rb_);
    if (threadIdx.x == 0) {  // the next check's slot (no reader left: see the barriers between)
      s_over[slot ^ 1] = 0;
      s_rho[slot ^ 1] = 0u;
    }
    return over != 0;
  };

  rows_pass(false, 0);
  sync();
  if constexpr (K > 1) {  // the first colour's halo
    halo_desc(-1, 0);
    __syncthreads();
    halo(false, true);
    sync();
  }
  int ep = 0;
  bool conv = false, checked_last = false;
  while (ep < V.epochs) {
    for (int c = 0; c < nc; ++c) {
      const bool more = c + 1 < nc;
      halo_desc(c, more ? c + 1 : -1);
      sweep_colour(c);
      if constexpr (K > 1) {
        __syncthreads();  // this rank's writes of colour c (and the descriptors) done
        if (nbuf == 2) {  // the next colour's halo goes to the other buffer at once
          halo(true, more);
        } else {  // one buffer: emptied before it is filled again
          halo(true, false);
          sync();
          if (more) halo(false, true);
        }
      }
      sync();
    }
    ++ep;
    checked_last = false;
    if (ep % V.R == 0 || ep == V.epochs) {
      checked_last = true;
      if (!check(ep == V.epochs)) {
        conv = true;
        break;
      }
    }
    if constexpr (K > 1) {  // the next epoch's first colour reads the rows as they are now (refreshed by a check)
      halo_desc(-1, 0);
      __syncthreads();
      halo(false, true);
      sync();
    }
  }
  if (!checked_last) conv = !check(true);
  sync();
  if (V.round) {
    // -- repair and rounding of the final iterate (Sec. 2, App. B.2, App. C) --
    // scratch over the r region: pick and keep bits of this rank's columns
    // (own index i = k / K of column k, k % K == q)
    __shared__ double s_wred[32];
    __shared__ double s_ctot;
    const int xch = (n + K - 1) / K;
    const int nw = (xch + 31) / 32;
    uint32_t* pickw = reinterpret_cast<uint32_t*>(smem);
    uint32_t* keepw = pickw + nw;
    uint32_t pb[K], kb[K];
    if constexpr (K > 1) {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        pb[r] = dsm_map(smem_u32(pickw), (uint32_t)r);
        kb[r] = dsm_map(smem_u32(keepw), (uint32_t)r);
      }
    }
    const uint32_t* Vid = V.vid + col0;
    uint8_t* Lab = V.lab + col0;
    const bool vc = sig < 0.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fixed-order reduction over the CTA, then over the cluster's ranks
    auto reduce = [&](double v, bool mx) -> double {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = mx ? fmax(v, u) : v + u;
      }
      if (lane == 0) s_wred[warp] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = s_wred[0];
        for (int w = 1; w < NT / 32; ++w) a = mx ? fmax(a, s_wred[w]) : a + s_wred[w];
        s_ctot = a;
      }
      sync();
      double tot = s_ctot;
      if constexpr (K > 1) {
        tot = dsm_ld_d(dsm_map(smem_u32(&s_ctot), 0));
        for (int r = 1; r < K; ++r) {
          const double u = dsm_ld_d(dsm_map(smem_u32(&s_ctot), (uint32_t)r));
          tot = mx ? fmax(tot, u) : tot + u;
        }
      }
      sync();
      return tot;
    };
    auto bit_of = [&](const uint32_t* w, const uint32_t (&wb)[K], uint32_t k) -> uint32_t {
      if constexpr (K == 1) return (w[k >> 5] >> (k & 31)) & 1u;
      else {
        const uint32_t i = k / K;
        return (dsm_ld_u(pick<K>(wb, k % K) + 4u * (i >> 5)) >> (i & 31)) & 1u;
      }
    };
    auto clear_keep = [&](uint32_t k) {
      if constexpr (K == 1) atomicAnd(&keepw[k >> 5], ~(1u << (k & 31)));
      else {
        const uint32_t i = k / K;
        dsm_and(pick<K>(kb, k % K) + 4u * (i >> 5), ~(1u << (i & 31)));
      }
    };
    // repair value: VC eps = max (1 - x_u - x_v)_+, IS alpha = max (x_u + x_v - 1)_+
    double vmax = 0.0;
    for (int e = qlo + (int)threadIdx.x; e < qhi; e += NT) {
      const double xu = (double)xget(Iru[e]), xv = (double)xget(Irv[e]);
      const double v = vc ? (1.0 - xu) - xv : (xu + xv) - 1.0;
      if (v > vmax) vmax = v;
    }
    const double a = reduce(vmax, true);
    // the labels of this rank's columns, in bit words (and the objective)
    auto label_words = [&](int rep, bool store) -> double {
      double wsum = 0.0;
      for (int i0 = warp * 32; i0 < xch; i0 += NT) {
        const int i = i0 + lane;
        const int k = q + i * K;
        bool b = false;
        if (i < xch && k < n) {
          const double xv = (double)xown_get(k);
          if (vc) {
            if (a < 1.0) b = fmin(1.0, fmax(0.0, xv / (1.0 - a))) >= 0.5;
          } else {
            b = rng_unif(V.seed, (uint64_t)rep, STREAM_IS_PICK, Vid[k]) < xv / (1.0 + a);
          }
          if (store && vc) Lab[Vid[k]] = b ? 1 : 0;
          if (b && vc) wsum += (double)Cc[k];
        }
        const uint32_t w = __ballot_sync(0xffffffffu, b);
        if (lane == 0) {
          pickw[i0 >> 5] = w;
          keepw[i0 >> 5] = w;
        }
      }
      return wsum;
    };
    // IS alterations: of every edge with both ends picked, the end with the
    // larger vertex id leaves; then the kept weight
    auto alter_weight = [&](bool store) -> double {
      sync();
      for (int e = qlo + (int)threadIdx.x; e < qhi; e += NT) {
        const uint32_t u = Iru[e], v = Irv[e];
        if (bit_of(pickw, pb, u) && bit_of(pickw, pb, v)) clear_keep(Vid[u] > Vid[v] ? u : v);
      }
      sync();
      double wsum = 0.0;
      for (int i = threadIdx.x; i < xch; i += NT) {
        const int k = q + i * K;
        if (k >= n) continue;
        const uint32_t kb1 = (keepw[i >> 5] >> (i & 31)) & 1u;
        if (store) Lab[Vid[k]] = (uint8_t)kb1;
        if (kb1) wsum -= (double)Cc[k];  // IS costs are -w
      }
      return wsum;
    };
    double obj;
    int best = 0;
    if (vc) {
      obj = reduce(label_words(0, true), false);
    } else {
      double bw = 0.0;
      for (int rep = 0; rep < V.reps; ++rep) {
        label_words(rep, false);
        const double w = reduce(alter_weight(false), false);
        if (rep == 0 || w > bw) {
          bw = w;
          best = rep;
        }
      }
      label_words(best, false);
      obj = reduce(alter_weight(true), false);
    }
    // exact validity over this rank's rows (labels are in the keep bits; for VC
    // the pick and keep words are equal)
    sync();
    double bad = 0.0;
    for (int e = qlo + (int)threadIdx.x; e < qhi; e += NT) {
      const uint32_t bu = bit_of(keepw, kb, Iru[e]), bv = bit_of(keepw, kb, Irv[e]);
      if (vc ? !(bu | bv) : (bu & bv)) bad = 1.0;
    }
    bad = reduce(bad, true);
    for (int i = threadIdx.x; i < xch; i += NT) {
      const int k = q + i * K;
      if (k < n) V.xout[col0 + Vid[k]] = xown_get(k);
    }
    if (threadIdx.x == 0 && q == 0) {
      V.r_obj[t] = obj;
      V.r_rep[t] = a;
      V.r_best[t] = best;
      V.r_status[t] = (vc && a >= 1.0) ? -1 : (bad != 0.0 ? 0 : 1);
    }
  }
  sync();  // no rank may leave while another still reads its shared memory
  if (xs)
    for (int i = threadIdx.x; i * K + q < n; i += NT) Sx[i * K + q] = sx[i];
  if (threadIdx.x == 0 && q == 0) {
    V.ep_out[t] = ep;
    V.conv_out[t] = conv ? 1 : 0;
    V.rho_out[t] = last_rho;
    V.t_out[2 * t + 1] = global_ns();
  }
  if (V.done) {
    // every rank's results are written (the barrier above orders them within
    // the cluster): publish the instance to the host
    sync();
    if (threadIdx.x == 0 && q == 0) {
      __threadfence_system();
      *(volatile int*)(V.done + t) = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// instance-major layout, built once from the union layout
// ---------------------------------------------------------------------------
// sort keys of the union columns: length (longest first), colour, instance
__global__ void k_inst_key_len(const int64_t* colptr, int64_t Ns, uint32_t* keys, uint32_t* vals) {
  GSTRIDE(j, Ns) {
    const int64_t len = colptr[j + 1] - colptr[j];
    keys[j] = 1023u - (uint32_t)(len < 1023 ? len : 1023);
    vals[j] = (uint32_t)j;
  }
}
__global__ void k_inst_key_of(const uint32_t* vals, const uint32_t* table, int64_t n, uint32_t* keys) {
  GSTRIDE(k, n) keys[k] = table[vals[k]];
}
// colour of every union column: the colours' columns are consecutive ranges
// cstart[c] .. cstart[c + 1] (the last c with cstart[c] <= j)
__global__ void k_inst_ucolour(const int64_t* cstart, int C1, int64_t Ns, uint32_t* colour) {
  GSTRIDE(j, Ns) {
    int lo = 0, hi = C1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (cstart[mid] <= j) lo = mid;
      else hi = mid;
    }
    colour[j] = (uint32_t)lo;
  }
}

// first short column (at most 32 entries) of every colour of every instance,
// and the ELL panels of 32 short columns each colour takes
// ELL panels of a colour's short columns [cw, end) on K ranks: rank r's
// columns (k % K == r) in order, 32 to a panel; panel jj of rank r is panel
// jj * K + r of the colour, and every rank gets the same panel count (the
// last ones may be empty).
__device__ __forceinline__ int64_t ell_rank_first(int64_t cw, int64_t r, int64_t K) {
  return cw + ((r - cw % K) % K + K) % K;
}

__global__ void k_inst_wide(const uint32_t* i_col, const int64_t* colptr, const int64_t* noff, const int32_t* coff,
                            const uint8_t* iK, int64_t count, int C1, int32_t* cwide, int64_t* npan) {
  GSTRIDE(f, count * C1) {
    const int64_t t = f / C1;
    const int c = (int)(f % C1);
    if (c == C1 - 1) {
      cwide[f] = coff[f];
      npan[f] = 0;
      continue;
    }
    int64_t lo = noff[t] + coff[f], hi = noff[t] + coff[f + 1];
    const int64_t end = hi;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const uint32_t j = i_col[mid];
      if (colptr[j + 1] - colptr[j] > 32) lo = mid + 1;
      else hi = mid;
    }
    cwide[f] = (int32_t)(lo - noff[t]);
    const int64_t K = iK[t], per_rank = (end - lo + K - 1) / K;
    npan[f] = K * ((per_rank + 31) / 32);
  }
}

// per panel: its width (the length of its first, longest column; 0 for an
// empty one) and its slot count
__global__ void k_inst_panels(const int64_t* pfirst, const int32_t* cwide, const int32_t* coff, const uint8_t* iK,
                              const uint32_t* i_col, const int64_t* colptr, const int64_t* noff, const int64_t* eoff,
                              int64_t nf, int C1, int64_t npanels, uint8_t* pw, int64_t* pslots) {
  GSTRIDE(p, npanels) {
    int64_t lo = 0, hi = nf;  // the last f with pfirst[f] <= p (f with panels)
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (pfirst[mid] <= p) lo = mid;
      else hi = mid;
    }
    while (lo + 1 < nf && pfirst[lo + 1] <= p) ++lo;
    const int64_t t = lo / C1, K = iK[t], jp = p - pfirst[lo];
    const int64_t k0 = ell_rank_first(cwide[lo], jp % K, K) + K * 32 * (jp / K);
    int w = 0;
    if (k0 < coff[lo + 1]) {
      const uint32_t j = i_col[noff[t] + k0];
      w = (int)(colptr[j + 1] - colptr[j]);
    }
    pw[p] = (uint8_t)w;
    pslots[p] = 32 * (int64_t)(inst_ell16(K, eoff[t + 1] - eoff[t]) ? (w + 1) / 2 : w);  // in 32-bit words
  }
}

// ELL slots of every short column (CSR entries of the IML column, in order)
__global__ void k_inst_ell(const uint32_t* i_col, const int32_t* inst_col, const uint32_t* ucolour,
                           const uint8_t* iK, const int64_t* noff, const int64_t* eoff, const uint32_t* iend,
                           const uint32_t* ient, const int32_t* cwide, const int64_t* pfirst, const int64_t* pbase,
                           const int32_t* qoff, const int32_t* hs, const int32_t* hoff, const int32_t* hH,
                           const uint8_t* hnb, const uint8_t* xg, int64_t Ns, int C1, uint32_t* ell, int* err) {
  GSTRIDE(k, Ns) {
    const uint32_t j = i_col[k];
    const int64_t t = inst_col[j];
    const int c = (int)ucolour[j];
    const int64_t f = t * C1 + c;
    const int64_t loc = k - noff[t];
    if (loc < cwide[f]) continue;  // a long column: served through the CSR
    const int64_t K = iK[t], r = loc % K;
    const int64_t i = (loc - ell_rank_first(cwide[f], r, K)) / K;  // its place among rank r's short columns
    const int64_t p = pfirst[f] + (i / 32) * K + r;
    const int lane = (int)(i % 32);
    const uint32_t e1 = iend[k];
    const uint32_t e0 = (loc == 0) ? 0u : iend[k - 1];
    const int64_t src = 2 * eoff[t];
    if (inst_ell16(K, eoff[t + 1] - eoff[t])) {  // slots 2w, 2w + 1 in word w (low half first)
      // the shared-memory index of an entry's row: for a cluster rank, its own
      // row, or the halo copy of another rank's row (after r and x)
      int64_t hb = 0, H = 0;
      if (K > 1) {
        int64_t rch = 0;
        for (int a = 0; a < K; ++a) rch = max(rch, (int64_t)(qoff[t * 5 + a + 1] - qoff[t * 5 + a]));
        const int64_t xch = (noff[t + 1] - noff[t] + K - 1) / K;
        hb = max(rch, 2 * ((xch + 31) / 32)) + (xg[t] ? 0 : xch);
        H = (hnb[t] == 2) ? hH[t] : 0;  // the buffer of colour c at hb + (c & 1) H
      }
      auto slot = [&](uint32_t e) -> uint32_t {
        if (K == 1) return e;
        const int64_t er = e >> 28, pos = e & 0x0fffffffu;
        const int64_t a = (er == r) ? pos
                                    : hb + (c & 1) * H + hoff[((t * 4 + r) * C1 + c) * 4 + er] +
                                          (pos - hs[((t * 4 + er) * 4 + r) * C1 + c]);
        if (a >= 0xffff) atomicExch(err + 1, 1);
        return (uint32_t)a & 0xffffu;
      };
      for (uint32_t q = e0; q < e1; q += 2) {
        const uint32_t lo = slot(ient[src + q]), hi = (q + 1 < e1) ? slot(ient[src + q + 1]) : 0xffffu;
        ell[pbase[p] + 32 * (int64_t)((q - e0) / 2) + lane] = lo | (hi << 16);
      }
    } else {
      for (uint32_t q = e0; q < e1; ++q) ell[pbase[p] + 32 * (int64_t)(q - e0) + lane] = ient[src + q];
    }
  }
}

__global__ void k_inst_lcol(const uint32_t* i_col, const int32_t* inst_col, const int64_t* noff, int64_t Ns,
                            uint32_t* lcol) {
  GSTRIDE(k, Ns) {
    const uint32_t j = i_col[k];
    lcol[j] = (uint32_t)(k - noff[inst_col[j]]);
  }
}

// instance-local vertex id of every IML column (the rounding streams' index)
__global__ void k_inst_vid(const uint32_t* col_of_orig, const int32_t* inst_col, const int64_t* noff,
                           const uint32_t* lcol, int64_t Ns, uint32_t* vid) {
  GSTRIDE(j, Ns) {
    const uint32_t ci = col_of_orig[j];
    const int64_t t = inst_col[ci];
    vid[noff[t] + lcol[ci]] = (uint32_t)(j - noff[t]);
  }
}

// Rank of the cluster that keeps row i in its shared memory: one of the two
// ranks that step its columns (column k is stepped by rank k % K), chosen by a
// hash of the row for balance -- so that column's access to the row is local.
// 0 for instances on one CTA.
__global__ void k_inst_rowrank(const int64_t* rowptr, const uint32_t* colidx, const uint32_t* lcol,
                               const int32_t* inst_row, const uint8_t* iK, int64_t M, uint32_t* rank,
                               uint32_t* vals) {
  GSTRIDE(i, M) {
    const uint32_t K = iK[inst_row[i]];
    uint32_t r = 0;
    if (K > 1) {
      const int64_t q0 = rowptr[i];
      const uint32_t a = lcol[idx_of(colidx[q0])], b = lcol[idx_of(colidx[q0 + 1])];
      const uint32_t h = (uint32_t)((uint64_t)i * 0x9E3779B97F4A7C15ull >> 40);
      r = ((h & 1u) ? a : b) % K;
    }
    rank[i] = r;
    vals[i] = (uint32_t)i;
  }
}

// local row of every union row, and its encoded id: (rank << 28) | (position
// inside the rank's block)
__global__ void k_inst_lrow(const uint32_t* i_row, const int32_t* inst_row, const int64_t* eoff, const uint32_t* rank,
                            const uint32_t* rpos, int64_t M, uint32_t* lrow, uint32_t* erow) {
  GSTRIDE(k, M) {
    const uint32_t i = i_row[k];
    const int32_t t = inst_row[i];
    lrow[i] = (uint32_t)(k - eoff[t]);
    erow[i] = (rank[i] << 28) | rpos[k];
  }
}

// halo group of every row (at its place k in the rows' (instance, rank)
// order): 0 unless the row's other endpoint is a short column stepped by
// another rank A, then 1 + A * C1 + that column's colour
__global__ void k_inst_hkey(const uint32_t* i_row, const int32_t* inst_row, const uint8_t* iK, const uint32_t* rank,
                            const int64_t* rowptr, const uint32_t* colidx, const int64_t* colptr,
                            const uint32_t* lcol, const uint32_t* ucolour, int C1, int64_t M, uint32_t* keys,
                            uint32_t* vals, uint32_t* hkey) {
  GSTRIDE(k, M) {
    const uint32_t i = i_row[k];
    const uint32_t K = iK[inst_row[i]];
    uint32_t key = 0;
    if (K > 1) {
      const uint32_t r = rank[i];
      const int64_t q0 = rowptr[i];
      const uint32_t a = idx_of(colidx[q0]), b = idx_of(colidx[q0 + 1]);
      const uint32_t w = (lcol[a] % K == r) ? b : a;  // the endpoint the keeper does not step, if any
      const uint32_t A = lcol[w] % K;
      if (A != r && colptr[w + 1] - colptr[w] <= 32) key = 1 + A * (uint32_t)C1 + ucolour[w];
    }
    keys[k] = key;
    vals[k] = (uint32_t)k;
    hkey[k] = key;
  }
}

// sort key of the rows' (instance, rank) block
__global__ void k_inst_hblock(const uint32_t* perm, const uint32_t* i_row, const int32_t* inst_row,
                              const uint32_t* rank, int64_t M, uint32_t* keys) {
  GSTRIDE(p, M) {
    const uint32_t i = i_row[perm[p]];
    keys[p] = (uint32_t)inst_row[i] * 4u + rank[i];
  }
}

// place of every row in its rank's block of r (perm: the rows by (instance,
// rank, halo group), as places k of the (instance, rank) order; null: that
// order itself), the inverse, and the halo groups in the new order
__global__ void k_inst_rpos(const uint32_t* perm, const uint32_t* i_row, const int32_t* inst_row,
                            const uint32_t* rank, const int64_t* eoff, const int32_t* qoff, const uint32_t* hkey,
                            int64_t M, uint32_t* rpos, uint32_t* rrow, uint32_t* hsorted) {
  GSTRIDE(p, M) {
    const uint32_t k = perm ? perm[p] : (uint32_t)p;
    const uint32_t i = i_row[k];
    const int64_t t = inst_row[i];
    const int64_t base = eoff[t] + qoff[t * 5 + rank[i]];
    rpos[k] = (uint32_t)(p - base);
    rrow[p] = (uint32_t)(k - eoff[t]);
    if (hsorted) hsorted[p] = hkey[k];
  }
}

// the segment R(q, A, c) of rank q's block: its rows read by rank A's short
// columns of colour c (f = ((t * 4 + q) * 4 + A) * C1 + c)
__global__ void k_inst_hseg(const uint32_t* hsorted, const int64_t* eoff, const int32_t* qoff, const uint8_t* iK,
                            int64_t count, int C1, int32_t* hs, int32_t* hl) {
  GSTRIDE(f, count * 16 * C1) {
    const int64_t t = f / (16 * C1);
    const int qa = (int)((f / C1) % 16), c = (int)(f % C1);
    const int q = qa / 4, A = qa % 4, K = iK[t];
    int32_t start = 0, len = 0;
    if (q < K && A < K && q != A && hsorted) {
      const int64_t b0 = eoff[t] + qoff[t * 5 + q], b1 = eoff[t] + qoff[t * 5 + q + 1];
      const uint32_t key = 1u + (uint32_t)A * (uint32_t)C1 + (uint32_t)c;
      auto lower = [&](uint32_t v) {
        int64_t lo = b0, hi = b1;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (hsorted[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        return lo;
      };
      const int64_t a = lower(key), b = lower(key + 1);
      start = (int32_t)(a - b0);
      len = (int32_t)(b - a);
    }
    hs[f] = start;
    hl[f] = len;
  }
}

// rank q's halo buffer of colour c: R(A, q, c) for A = 0, 1, ... one after
// another (hoff[((t * 4 + q) * C1 + c) * 4 + A]); hH[t]: the largest buffer
__global__ void k_inst_hoff(const int32_t* hl, int64_t count, int C1, int32_t* hoff, int32_t* hH) {
  GSTRIDE(f, count * 4 * C1) {
    const int64_t t = f / (4 * C1);
    const int q = (int)((f / C1) % 4), c = (int)(f % C1);
    int32_t acc = 0;
    for (int A = 0; A < 4; ++A) {
      hoff[f * 4 + A] = acc;
      acc += hl[((t * 4 + A) * 4 + q) * C1 + c];
    }
    atomicMax(&hH[t], acc);
  }
}

// first local row of every rank (5 per instance: ranks 0..3 and the end)
__global__ void k_inst_qoff(const uint32_t* i_row, const uint32_t* rank, const int64_t* eoff, int64_t count,
                            int32_t* qoff) {
  GSTRIDE(f, count * 5) {
    const int64_t t = f / 5;
    const uint32_t q = (uint32_t)(f % 5);
    int64_t lo = eoff[t], hi = eoff[t + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rank[i_row[mid]] < q) lo = mid + 1;
      else hi = mid;
    }
    qoff[f] = (int32_t)(lo - eoff[t]);
  }
}

__global__ void k_inst_deg(const uint32_t* i_col, const int64_t* colptr, int64_t Ns, int64_t* deg) {
  GSTRIDE(k, Ns) {
    const uint32_t j = i_col[k];
    deg[k] = colptr[j + 1] - colptr[j];
  }
}

// per union row: its two columns, their local ids and the row's encoded id
// (x = 0xffffffff: the row has not exactly two structural entries), so the
// fill below reads one 16-byte record per entry instead of four scattered words
__global__ void k_inst_rowinfo(const int64_t* rowptr, const uint32_t* colidx, const uint32_t* lcol, const uint32_t* erow,
                               int64_t M, uint4* rinfo) {
  GSTRIDE(i, M) {
    const int64_t q0 = rowptr[i];
    uint4 v = make_uint4(0xffffffffu, 0u, 0u, 0u);
    if (rowptr[i + 1] - q0 == 2) {
      const uint32_t a = idx_of(colidx[q0]), b = idx_of(colidx[q0 + 1]);
      v = make_uint4(a, lcol[a], lcol[b], erow[i]);
    }
    rinfo[i] = v;
  }
}

// local end offsets, entries (encoded row, other endpoint) and the longest
// column of every instance; err: a row without exactly two structural entries
__global__ void k_inst_fill(const uint32_t* i_col, const int32_t* inst_col, const int64_t* pos, const int64_t* eoff,
                            const int64_t* colptr, const uint32_t* rowidx, const uint4* rinfo, int64_t Ns,
                            uint32_t* iend, uint32_t* ient, uint32_t* inb, int32_t* ideg, int* err) {
  GSTRIDE(k, Ns) {
    const uint32_t j = i_col[k];
    const int32_t t = inst_col[j];
    const int64_t base = pos[k];
    const int64_t p0 = colptr[j], p1 = colptr[j + 1];
    iend[k] = (uint32_t)(pos[k + 1] - 2 * eoff[t]);
    // the longest column: one atomic per warp where its lanes share the instance
    const unsigned act = __activemask();
    const int leader = __ffs(act) - 1;
    const int32_t t0 = __shfl_sync(act, t, leader);
    const int32_t d = (int32_t)(p1 - p0);
    if (__all_sync(act, t == t0)) {
      const int32_t dmax = __reduce_max_sync(act, d);
      if ((int)(threadIdx.x & 31) == leader) atomicMax(&ideg[t], dmax);
    } else {
      atomicMax(&ideg[t], d);
    }
    for (int64_t p = p0; p < p1; ++p) {
      const uint4 ri = rinfo[idx_of(rowidx[p])];
      if (ri.x == 0xffffffffu) {
        atomicExch(err, 1);
        ient[base + (p - p0)] = 0;
        inb[base + (p - p0)] = 0;
        continue;
      }
      ient[base + (p - p0)] = ri.w;
      inb[base + (p - p0)] = (ri.x == j) ? ri.z : ri.y;
    }
  }
}

__global__ void k_inst_rows(const uint32_t* i_row, const uint4* rinfo, int64_t M, uint32_t* iru, uint32_t* irv) {
  GSTRIDE(k, M) {
    const uint4 ri = rinfo[i_row[k]];
    iru[k] = ri.y;
    irv[k] = ri.z;
  }
}

// first local column / slack row of every colour: the instance's columns are
// in union order, which is colour-major, so a colour starts at the first
// column whose union position reaches the colour's first union column
__global__ void k_inst_colours(const uint32_t* i_col, const uint32_t* i_row, const int64_t* noff, const int64_t* eoff,
                               const int32_t* qoff, const int64_t* cstart, const int64_t* rstart, int64_t count,
                               int C1, int32_t* coff, int32_t* roff) {
  GSTRIDE(f, count * C1 * 5) {
    const int64_t tq = f / C1;  // (instance, q) with q = 0 for the columns' table
    const int c = (int)(f % C1);
    const int64_t t = tq / 5;
    const int q = (int)(tq % 5);
    if (q == 4) {
      int64_t lo = noff[t], hi = noff[t + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)i_col[mid] < cstart[c]) lo = mid + 1;
        else hi = mid;
      }
      coff[t * C1 + c] = (int32_t)(lo - noff[t]);
      continue;
    }
    // the rank's block of rows keeps the union's colour-major order
    int64_t lo = eoff[t] + qoff[t * 5 + q], hi = eoff[t] + qoff[t * 5 + q + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)i_row[mid] < rstart[c]) lo = mid + 1;
      else hi = mid;
    }
    roff[(t * 4 + q) * C1 + c] = (int32_t)(lo - eoff[t]);
  }
}

// colours an instance uses: one past the last colour holding a column or a
// slack row of any rank
__global__ void k_inst_ncol(const int32_t* coff, const int32_t* roff, int64_t count, int C1, int32_t* ncol) {
  GSTRIDE(t, count) {
    int nc = 1;
    for (int c = 0; c + 1 < C1; ++c) {
      bool any = coff[t * C1 + c + 1] > coff[t * C1 + c];
      for (int q = 0; q < 4; ++q) {
        const int32_t* ro = roff + (t * 4 + q) * C1;
        any = any || ro[c + 1] > ro[c];
      }
      if (any) nc = c + 1;
    }
    ncol[t] = nc;
  }
}

__global__ void k_inst_gather(const uint32_t* i_col, const uint32_t* i_row, const float* x, const float* c,
                              const float* s, int64_t Ns, int64_t M, float* ix, float* ic, float* is) {
  GSTRIDE(k, Ns > M ? Ns : M) {
    if (k < Ns) {
      const uint32_t j = i_col[k];
      ix[k] = x[j];
      ic[k] = c[j];
    }
    if (k < M) is[k] = s[i_row[k]];
  }
}

__global__ void k_inst_scatter(const uint32_t* i_col, const uint32_t* i_row, const float* ix, const float* is,
                               int64_t Ns, int64_t M, float* x, float* s) {
  GSTRIDE(k, Ns > M ? Ns : M) {
    if (k < Ns) x[i_col[k]] = ix[k];
    if (k < M) s[i_row[k]] = is[k];
  }
}

__global__ void k_inst_stamp(unsigned long long* t) { *t = global_ns(); }

int bits_for_count(int64_t n) {
  int b = 1;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

// launch classes: (cluster size, threads per CTA).  An instance takes one CTA
// of 256, 512 or 1024 threads when its r and x fit that CTA's shared memory,
// else one CTA with x in global memory when r alone fits, else the smallest
// cluster of 2, 3 or 4 CTAs whose shared memory holds its rows and halo
// buffers -- with x there too, or in global memory where that saves a CTA
// (on by default, the autotuner may switch clusters off) -- else the last
// class: one CTA of 1024 threads with x and the rows beyond its shared memory
// in global memory (L2), measured slower than the clusters.
struct Cls {
  int K, NT;
};
constexpr Cls CLASSES[] = {{1, 256}, {1, 512}, {1, 1024}, {2, 1024}, {3, 1024}, {4, 1024}, {1, 1024}};
constexpr int NCLS = 7;
constexpr int CLS_SPILL = 6;

// shared memory of an instance on K CTAs: its r region (at least the
// rounding's two bit words per 32 columns) and its x
int64_t inst_smem(int64_t n, int64_t m, int K) {
  const int64_t xch = (n + K - 1) / K;
  return 4 * (std::max<int64_t>((m + K - 1) / K, 2 * ((xch + 31) / 32)) + xch);
}

struct DevLimits {
  int64_t optin = 0, per_sm = 0;
  bool cluster = false;
};
DevLimits dev_limits() {
  DevLimits L;
  int dev = 0, v = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  L.optin = v;
  TH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  L.per_sm = v;
  TH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrClusterLaunch, dev));
  L.cluster = v != 0;
  return L;
}

// dynamic shared memory a CTA of class c may take (1 KB per CTA stays with the
// system; the kernel's static shared memory -- flags, 1/L table, colour
// table, rounding scratch -- stays below 2 KB)
constexpr int64_t INST_STATIC_SMEM = 2048;
int64_t class_cap(const DevLimits& L, int c) {
  const int per = (CLASSES[c].K == 1) ? 1024 / CLASSES[c].NT : 1;
  return std::min<int64_t>(L.optin, L.per_sm / per - 1024) - INST_STATIC_SMEM;
}

template <int K, int NT, int G, bool SPILL = false>
void launch_one(const InstView& V, const int32_t* order, int64_t count, size_t smem, int64_t optin, cudaStream_t st) {
  auto kern = k_inst<K, NT, G, SPILL>;
  cudaFuncAttributes fa;
  TH_CUDA(cudaFuncGetAttributes(&fa, kern));
  TH_CHECK((int64_t)fa.sharedSizeBytes <= INST_STATIC_SMEM && (int64_t)smem + (int64_t)fa.sharedSizeBytes <= optin,
           THETIS_E_INVALID, "instance engine: shared memory of a launch class exceeds the device limit");
  TH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(optin - (int64_t)fa.sharedSizeBytes)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * K));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (K > 1) ? 1 : 0;
  TH_CUDA(cudaLaunchKernelEx(&cfg, kern, V, order));
  TH_LAUNCHED();
}

template <int G>
void launch_class(int c, const InstView& V, const int32_t* order, int64_t count, size_t smem, int64_t optin,
                  cudaStream_t st) {
  switch (c) {
    case 0: launch_one<1, 256, G>(V, order, count, smem, optin, st); break;
    case 1: launch_one<1, 512, G>(V, order, count, smem, optin, st); break;
    case 2: launch_one<1, 1024, G>(V, order, count, smem, optin, st); break;
    // clusters: one column per lane through ELL panels and halo buffers
    case 3: launch_one<2, 1024, 1>(V, order, count, smem, optin, st); break;
    case 4: launch_one<3, 1024, 1>(V, order, count, smem, optin, st); break;
    case 5: launch_one<4, 1024, 1>(V, order, count, smem, optin, st); break;
    default: launch_one<1, 1024, G, true>(V, order, count, smem, optin, st); break;
  }
}

// launch classes and the order of instances in them (largest first); the
// cluster size K of every instance (1 unless it takes a cluster) and whether
// a cluster instance keeps x in global memory
void inst_classes(Problem& P) {
  cudaStream_t s = P.stream;
  const int64_t count = P.nbatch;
  const DevLimits L = dev_limits();
  std::vector<std::vector<int32_t>> members(NCLS);
  std::vector<uint8_t> iK(count, 1), xg(count, 0);
  const bool clusters = P.iml_clusters && L.cluster;
  if ((int64_t)P.h_iKmin.size() != count) P.h_iKmin.assign(count, 0);
  for (int64_t t = 0; t < count; ++t) {
    const int64_t n = P.h_bnoff[t + 1] - P.h_bnoff[t], m = P.h_beoff[t + 1] - P.h_beoff[t];
    // one CTA with everything in shared memory; else one CTA with x in global
    // memory when r alone fits; else a cluster (if asked for; rows are split
    // between ranks by a hash, so the estimate leaves 5 % + 256 rows of slack);
    // else one CTA whose r spills to L2
    const int lmin = P.h_iKmin[t];
    int c = 0;
    uint8_t g = 0;
    while (c < 3 && inst_smem(n, m, 1) > class_cap(L, c)) ++c;
    if (c == 3) {
      // a rank: its rows, x (unless in global memory), and a halo buffer of
      // (at a guess) a fifth of the rows the other ranks keep and its short
      // columns read (the layout measures it, takes a second buffer where
      // that fits, and moves an instance that misses to the next level).
      // Levels: 2 CTAs with x in shared memory, 2 CTAs with x in global
      // memory (measured cheaper than a third CTA), 3, 3 global, 4, 4 global.
      auto est = [&](int K, int xg) {
        const int64_t halo = (m * (K - 1)) / (5 * K * K) + 64;
        return 4 * ((m * 102 / 100) / K + 512 + (xg ? 0 : (n + K - 1) / K) + halo);
      };
      c = CLS_SPILL;
      if (4 * m > class_cap(L, CLS_SPILL) && clusters) {
        for (int lv = lmin; lv < 6; ++lv) {
          const int K = 2 + lv / 2, xg = lv & 1;
          if (est(K, xg) <= class_cap(L, K + 1)) {
            c = K + 1;
            g = (uint8_t)xg;
            break;
          }
        }
      }
    }
    TH_CHECK(c != CLS_SPILL || 4 * 2 * ((n + 31) / 32) <= class_cap(L, CLS_SPILL), THETIS_E_INVALID,
             "instance engine: an instance with more vertices than one CTA's rounding scratch holds");
    // the kernels of classes 0-2 read 16-bit ELL slots only
    TH_CHECK(c > 2 || inst_ell16(1, m), THETIS_E_INVALID, "instance engine: a one-CTA instance with 65535 rows or more");
    members[c].push_back((int32_t)t);
    iK[t] = (uint8_t)CLASSES[c].K;
    xg[t] = g;
  }
  std::vector<int32_t> order;
  P.h_icls_off.assign(NCLS + 1, 0);
  for (int c = 0; c < NCLS; ++c) {
    auto& v = members[c];
    std::stable_sort(v.begin(), v.end(), [&](int32_t a, int32_t b) {
      const int64_t wa = (P.h_bnoff[a + 1] - P.h_bnoff[a]) + (P.h_beoff[a + 1] - P.h_beoff[a]);
      const int64_t wb = (P.h_bnoff[b + 1] - P.h_bnoff[b]) + (P.h_beoff[b + 1] - P.h_beoff[b]);
      return wa > wb;
    });
    P.h_icls_off[c] = (int64_t)order.size();
    order.insert(order.end(), v.begin(), v.end());
  }
  P.h_icls_off[NCLS] = (int64_t)order.size();
  if (!P.i_order) P.i_order = P.mem.alloc<int32_t>(count);
  if (!P.i_K) P.i_K = P.mem.alloc<uint8_t>(count);
  TH_CUDA(cudaMemcpyAsync(P.i_order, order.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaMemcpyAsync(P.i_K, iK.data(), count, cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaStreamSynchronize(s));
  if (iK != P.h_iK || xg != P.h_ixg) P.iml_built = false;  // the rows' placement depends on K, the halo on x
  P.h_iK = iK;
  P.h_ixg = xg;
  if (!P.i_xg) P.i_xg = P.mem.alloc<uint8_t>(count);
  TH_CUDA(cudaMemcpyAsync(P.i_xg, xg.data(), count, cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaStreamSynchronize(s));
  P.iml_classes_ok = true;
}

// dynamic shared memory of every launch class from the built layout:
// everything in shared memory (K = 1); the largest rank's rows, the rank's
// columns and its halo buffers (clusters); the whole budget (spill).  False
// (with the minimum cluster size of the instances at fault raised) when a
// cluster instance does not fit its class even with one halo buffer.
bool inst_class_smem(Problem& P) {
  const int64_t count = P.nbatch;
  const DevLimits L = dev_limits();
  std::vector<int32_t> qo((size_t)count * 5);
  TH_CUDA(cudaMemcpyAsync(qo.data(), P.i_qoff, qo.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  std::vector<int32_t> order((size_t)count);
  TH_CUDA(cudaMemcpyAsync(order.data(), P.i_order, count * sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  P.h_icls_smem.assign(NCLS, 0);
  bool fits = true;
  for (int c = 0; c < NCLS; ++c) {
    int64_t need = (c == CLS_SPILL) ? class_cap(L, c) : 0;
    for (int64_t i = P.h_icls_off[c]; i < P.h_icls_off[c + 1] && c != CLS_SPILL; ++i) {
      const int64_t t = order[i];
      const int K = CLASSES[c].K;
      const int64_t n = P.h_bnoff[t + 1] - P.h_bnoff[t];
      int64_t rows = 0;
      for (int q = 0; q < K; ++q) rows = std::max<int64_t>(rows, qo[t * 5 + q + 1] - qo[t * 5 + q]);
      const int64_t xch = (n + K - 1) / K;
      const bool xsm = K == 1 || P.h_ixg[t] == 0;
      const int64_t halo = (K > 1) ? (int64_t)std::max<uint8_t>(P.h_ihnb[t], 1) * P.h_iH[t] : 0;
      const int64_t own = 4 * (std::max<int64_t>(rows, 2 * ((xch + 31) / 32)) + (xsm ? xch : 0) + halo);
      if (K > 1 && own > class_cap(L, c)) {
        P.h_iKmin[t] = (uint8_t)(2 * (K - 2) + P.h_ixg[t] + 1);  // the next level (6: the spill class)
        fits = false;
      }
      need = std::max(need, own);
    }
    if (!fits) continue;
    TH_CHECK(need <= class_cap(L, c), THETIS_E_INVALID, "instance engine: a rank's rows exceed its shared memory");
    P.h_icls_smem[c] = (need + 15) / 16 * 16;
  }
  return fits;
}

void inst_layout(Problem& P) {
  cudaStream_t s = P.stream;
  const int64_t count = P.nbatch, Ns = P.Ns, M = P.M;
  TH_CHECK(P.kind == KIND_BATCH && count > 0 && P.Nfree == Ns && P.Msl == M, THETIS_E_INVALID,
           "instance engine: not a VC / IS batch");
  Arena tmp(s);
  const int C = P.ncolors, C1 = C + 1;
  auto once = [&](auto*& p, int64_t n) {
    using T = std::remove_reference_t<decltype(*p)>;
    if (!p) p = P.mem.alloc<T>(n);
  };
  once(P.i_col, Ns + 1);
  once(P.i_row, M + 1);
  uint32_t* keys = tmp.alloc<uint32_t>(std::max(Ns, M) + 1);
  // colour boundaries of the union layout (colour-major columns and slack rows)
  std::vector<int64_t> cst(C1), rst(C1);
  {
    int64_t col = 0;
    for (int c = 0; c < C; ++c) {
      cst[c] = col;
      rst[c] = P.plan[c].srow0;
      for (auto& sg : P.plan[c].segs) col += (sg.u1 - sg.u0) * sg.len;
    }
    cst[C] = col;
    rst[C] = P.Msl;
  }
  int64_t* dcst = tmp.alloc<int64_t>(C1);
  int64_t* drst = tmp.alloc<int64_t>(C1);
  TH_CUDA(cudaMemcpyAsync(dcst, cst.data(), C1 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaMemcpyAsync(drst, rst.data(), C1 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  uint32_t* ucolour = tmp.alloc<uint32_t>(Ns + 1);
  k_inst_ucolour<<<grid_for(Ns, 256), 256, 0, s>>>(dcst, C1, Ns, ucolour);
  TH_LAUNCHED();
  // columns by (instance, colour, length descending): stable LSD passes from
  // the least significant key
  k_inst_key_len<<<grid_for(Ns, 256), 256, 0, s>>>(P.colptr, Ns, keys, P.i_col);
  TH_LAUNCHED();
  radix_sort_pairs(keys, P.i_col, Ns, 10, tmp, s);
  k_inst_key_of<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, ucolour, Ns, keys);
  TH_LAUNCHED();
  radix_sort_pairs(keys, P.i_col, Ns, bits_for_count(C1), tmp, s);
  k_inst_key_of<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, (const uint32_t*)P.binst_col, Ns, keys);
  TH_LAUNCHED();
  radix_sort_pairs(keys, P.i_col, Ns, bits_for_count(count), tmp, s);
  uint32_t* lcol = tmp.alloc<uint32_t>(Ns + 1);
  k_inst_lcol<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, P.binst_col, P.bnoff, Ns, lcol);
  TH_LAUNCHED();
  once(P.i_vid, Ns + 1);
  k_inst_vid<<<grid_for(Ns, 256), 256, 0, s>>>(P.col_of_orig, P.binst_col, P.bnoff, lcol, Ns, P.i_vid);
  TH_LAUNCHED();
  // rows by (instance, rank of the cluster that keeps them, union order --
  // which is slack-colour major)
  uint32_t* rank = tmp.alloc<uint32_t>(M + 1);
  uint32_t* lrow = tmp.alloc<uint32_t>(M + 1);
  uint32_t* erow = tmp.alloc<uint32_t>(M + 1);
  once(P.i_qoff, count * 5);
  if (M > 0) {
    k_inst_rowrank<<<grid_for(M, 256), 256, 0, s>>>(P.rowptr, P.colidx, lcol, P.binst_row, P.i_K, M, keys, P.i_row);
    TH_LAUNCHED();
    TH_CUDA(cudaMemcpyAsync(rank, keys, M * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    radix_sort_pairs(keys, P.i_row, M, 2, tmp, s);
    k_inst_key_of<<<grid_for(M, 256), 256, 0, s>>>(P.i_row, (const uint32_t*)P.binst_row, M, keys);
    TH_LAUNCHED();
    radix_sort_pairs(keys, P.i_row, M, bits_for_count(count), tmp, s);
  }
  k_inst_qoff<<<grid_for(count * 5, 256), 256, 0, s>>>(P.i_row, rank, P.beoff, count, P.i_qoff);
  TH_LAUNCHED();
  // a cluster rank's block of r in halo-group order: first the rows no other
  // rank's short column reads, then the segments R(q, A, c) by (A, c)
  const bool any_cluster = std::any_of(P.h_iK.begin(), P.h_iK.end(), [](uint8_t k) { return k > 1; });
  once(P.i_rpos, M + 1);
  once(P.i_rrow, M + 1);
  uint32_t* hsorted = nullptr;
  if (M > 0) {
    if (any_cluster) {
      uint32_t* perm = tmp.alloc<uint32_t>(M + 1);
      uint32_t* hkey = tmp.alloc<uint32_t>(M + 1);
      hsorted = tmp.alloc<uint32_t>(M + 1);
      k_inst_hkey<<<grid_for(M, 256), 256, 0, s>>>(P.i_row, P.binst_row, P.i_K, rank, P.rowptr, P.colidx, P.colptr,
                                                   lcol, ucolour, C1, M, keys, perm, hkey);
      TH_LAUNCHED();
      radix_sort_pairs(keys, perm, M, bits_for_count(4 * (int64_t)C1 + 2), tmp, s);
      k_inst_hblock<<<grid_for(M, 256), 256, 0, s>>>(perm, P.i_row, P.binst_row, rank, M, keys);
      TH_LAUNCHED();
      radix_sort_pairs(keys, perm, M, bits_for_count(count * 4), tmp, s);
      k_inst_rpos<<<grid_for(M, 256), 256, 0, s>>>(perm, P.i_row, P.binst_row, rank, P.beoff, P.i_qoff, hkey, M,
                                                   P.i_rpos, P.i_rrow, hsorted);
    } else {
      k_inst_rpos<<<grid_for(M, 256), 256, 0, s>>>(nullptr, P.i_row, P.binst_row, rank, P.beoff, P.i_qoff, nullptr, M,
                                                   P.i_rpos, P.i_rrow, nullptr);
    }
    TH_LAUNCHED();
    k_inst_lrow<<<grid_for(M, 256), 256, 0, s>>>(P.i_row, P.binst_row, P.beoff, rank, P.i_rpos, M, lrow, erow);
    TH_LAUNCHED();
  }
  // the segments, where they sit in the halo buffers, and each instance's
  // buffer length
  once(P.i_hs, count * 16 * C1);
  once(P.i_hl, count * 16 * C1);
  once(P.i_hoff, count * 16 * C1);
  once(P.i_hH, count);
  k_inst_hseg<<<grid_for(count * 16 * C1, 256), 256, 0, s>>>(hsorted, P.beoff, P.i_qoff, P.i_K, count, C1, P.i_hs,
                                                             P.i_hl);
  TH_LAUNCHED();
  TH_CUDA(cudaMemsetAsync(P.i_hH, 0, count * sizeof(int32_t), s));
  k_inst_hoff<<<grid_for(count * 4 * C1, 256), 256, 0, s>>>(P.i_hl, count, C1, P.i_hoff, P.i_hH);
  TH_LAUNCHED();
  // halo buffers of a cluster instance: two (colour parity, one cluster
  // barrier a colour) when they fit its class beside r and x, else one (two
  // barriers a colour)
  {
    std::vector<int32_t> qo((size_t)count * 5);
    P.h_iH.resize(count);
    TH_CUDA(cudaMemcpyAsync(qo.data(), P.i_qoff, qo.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaMemcpyAsync(P.h_iH.data(), P.i_hH, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    const DevLimits L = dev_limits();
    P.h_ihnb.assign(count, 0);
    for (int64_t t = 0; t < count; ++t) {
      const int K = P.h_iK[t];
      if (K == 1) continue;
      int64_t rch = 0;
      for (int q = 0; q < K; ++q) rch = std::max<int64_t>(rch, qo[t * 5 + q + 1] - qo[t * 5 + q]);
      const int64_t xch = (P.h_bnoff[t + 1] - P.h_bnoff[t] + K - 1) / K;
      const int64_t own = std::max<int64_t>(rch, 2 * ((xch + 31) / 32)) + (P.h_ixg[t] ? 0 : xch);
      P.h_ihnb[t] = (4 * (own + 2 * (int64_t)P.h_iH[t]) <= class_cap(L, K + 1)) ? 2 : 1;
    }
    once(P.i_hnb, count);
    TH_CUDA(cudaMemcpyAsync(P.i_hnb, P.h_ihnb.data(), count, cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaStreamSynchronize(s));  // the host vector is read by the copy
  }
  int64_t* pos = tmp.alloc<int64_t>(Ns + 1);
  k_inst_deg<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, P.colptr, Ns, pos);
  TH_LAUNCHED();
  exclusive_scan_i64(pos, pos, Ns, tmp, s);
  once(P.i_end, Ns + 1);
  once(P.i_ent, 2 * M + 1);
  once(P.i_nb, 2 * M + 1);
  once(P.i_ru, M + 1);
  once(P.i_rv, M + 1);
  once(P.i_deg, count);
  int* err = tmp.alloc<int>(2);  // [0]: a malformed row; [1]: a halo index past 16 bits
  TH_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
  TH_CUDA(cudaMemsetAsync(P.i_deg, 0, count * sizeof(int32_t), s));
  uint4* rinfo = tmp.alloc<uint4>(M + 1);
  if (M > 0) {
    k_inst_rowinfo<<<grid_for(M, 256), 256, 0, s>>>(P.rowptr, P.colidx, lcol, erow, M, rinfo);
    TH_LAUNCHED();
  }
  k_inst_fill<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, P.binst_col, pos, P.beoff, P.colptr, P.rowidx, rinfo, Ns,
                                                P.i_end, P.i_ent, P.i_nb, P.i_deg, err);
  TH_LAUNCHED();
  if (M > 0) {
    k_inst_rows<<<grid_for(M, 256), 256, 0, s>>>(P.i_row, rinfo, M, P.i_ru, P.i_rv);
    TH_LAUNCHED();
  }
  P.iml_C = C1;
  once(P.i_coff, count * C1);
  once(P.i_roff, count * 4 * C1);
  once(P.i_ncol, count);
  k_inst_colours<<<grid_for(count * C1 * 5, 256), 256, 0, s>>>(P.i_col, P.i_row, P.bnoff, P.beoff, P.i_qoff, dcst,
                                                               drst, count, C1, P.i_coff, P.i_roff);
  TH_LAUNCHED();
  k_inst_ncol<<<grid_for(count, 256), 256, 0, s>>>(P.i_coff, P.i_roff, count, C1, P.i_ncol);
  TH_LAUNCHED();
  // ELL panels of the short columns (thread-per-column sweep)
  {
    const int64_t nf = count * C1;
    once(P.i_cwide, nf);
    int64_t* npan = tmp.alloc<int64_t>(nf + 1);
    k_inst_wide<<<grid_for(nf, 256), 256, 0, s>>>(P.i_col, P.colptr, P.bnoff, P.i_coff, P.i_K, count, C1, P.i_cwide,
                                                  npan);
    TH_LAUNCHED();
    once(P.i_pfirst, nf + 1);
    exclusive_scan_i64(npan, P.i_pfirst, nf, tmp, s);
    int64_t npanels = 0;
    TH_CUDA(cudaMemcpyAsync(&npanels, P.i_pfirst + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    // the panels depend on the cluster sizes: a layout rebuilt for other sizes
    // may need more of them (the handle's arena keeps the smaller arrays until
    // it is closed)
    P.i_npanels = npanels;
    if (npanels + 1 > P.i_pcap) {
      P.i_pw = P.mem.alloc<uint8_t>(npanels + 1);
      P.i_pbase = P.mem.alloc<int64_t>(npanels + 1);
      P.i_pcap = npanels + 1;
    }
    if (npanels > 0) {
      k_inst_panels<<<grid_for(npanels, 256), 256, 0, s>>>(P.i_pfirst, P.i_cwide, P.i_coff, P.i_K, P.i_col, P.colptr,
                                                           P.bnoff, P.beoff, nf, C1, npanels, P.i_pw, P.i_pbase);
      TH_LAUNCHED();
    }
    exclusive_scan_i64(P.i_pbase, P.i_pbase, npanels, tmp, s);
    int64_t nslots = 0;
    TH_CUDA(cudaMemcpyAsync(&nslots, P.i_pbase + npanels, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    if (nslots + 1 > P.i_scap) {
      P.i_ell = P.mem.alloc<uint32_t>(nslots + 1);
      P.i_scap = nslots + 1;
    }
    TH_CUDA(cudaMemsetAsync(P.i_ell, 0xff, (nslots + 1) * sizeof(uint32_t), s));
    k_inst_ell<<<grid_for(Ns, 256), 256, 0, s>>>(P.i_col, P.binst_col, ucolour, P.i_K, P.bnoff, P.beoff, P.i_end,
                                                 P.i_ent, P.i_cwide, P.i_pfirst, P.i_pbase, P.i_qoff, P.i_hs,
                                                 P.i_hoff, P.i_hH, P.i_hnb, P.i_xg, Ns, C1, P.i_ell, err);
    TH_LAUNCHED();
  }
  once(P.i_c, Ns + 1);
  once(P.i_x, Ns + 1);
  once(P.i_s, M + 1);
  once(P.i_rg, M + 1);
  once(P.i_ep, count);
  once(P.i_conv, count);
  once(P.i_t, 2 * count + 1);
  once(P.i_lab, Ns + 1);
  once(P.i_robj, count);
  once(P.i_rrep, count);
  once(P.i_rbest, count);
  once(P.i_rstatus, count);
  once(P.i_xout, Ns + 1);
  once(P.i_rhoout, count);
  int herr[2] = {0, 0};
  TH_CUDA(cudaMemcpyAsync(herr, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));  // host tables above must outlive their copies
  TH_CHECK(herr[0] == 0, THETIS_E_INVALID, "instance engine: a row without exactly two structural entries");
  if (P.iml_G == 0) P.iml_G = 1;  // ELL panels, one thread per column (the autotuner may pick G lanes)
  P.iml_built = true;
  // an instance whose halo does not fit its class takes a larger cluster (or
  // the spill class) and the layout is built again
  if (!inst_class_smem(P)) {
    P.iml_classes_ok = false;
    P.iml_built = false;
    return;
  }
  TH_CHECK(herr[1] == 0, THETIS_E_CUDA, "instance engine: a halo index past 16 bits in a class that fits");
}

}  // namespace

bool inst_eligible(Problem& P) {
  if (P.kind != KIND_BATCH || P.nbatch <= 0 || P.Nfree != P.Ns || P.Msl != P.M) return false;
  if (!P.bounds_uniform) return false;
  for (int64_t t = 0; t < P.nbatch; ++t) {
    const int64_t n = P.h_bnoff[t + 1] - P.h_bnoff[t], m = P.h_beoff[t + 1] - P.h_beoff[t];
    if (n >= (int64_t(1) << 30) || m >= (int64_t(1) << 30)) return false;
  }
  return true;
}

// launch classes and the layout, again while an instance's halo pushes it
// to the next cluster level (six levels up to the spill class, so at most
// seven rounds)
void inst_ready(Problem& P) {
  for (int it = 0; it < 8; ++it) {
    if (!P.iml_classes_ok) inst_classes(P);
    if (!P.iml_built) inst_layout(P);
    if (P.iml_classes_ok && P.iml_built) return;
  }
  TH_CHECK(false, THETIS_E_CUDA, "instance engine: no launch class settled");
}

void inst_prepare(Problem& P) { inst_ready(P); }

void inst_set_clusters(Problem& P, bool on) {
  if (P.iml_clusters == on) return;
  P.iml_clusters = on;
  P.iml_classes_ok = false;  // the launch classes change on the next solve
}

void inst_solve(Problem& P, const SolveArgs& a, double& sweep_ms) {
  inst_ready(P);
  cudaStream_t s = P.stream;
  const int64_t count = P.nbatch;
  if (!P.i_events[0]) {
    for (int c = 0; c < NCLS; ++c) TH_CUDA(cudaStreamCreateWithFlags(&P.i_streams[c], cudaStreamNonBlocking));
    TH_CUDA(cudaEventCreate(&P.i_events[0]));
    TH_CUDA(cudaEventCreate(&P.i_events[1]));
    for (int c = 0; c <= NCLS; ++c) TH_CUDA(cudaEventCreateWithFlags(&P.i_events[2 + c], cudaEventDisableTiming));
  }
  const int64_t n2 = std::max(P.Ns, P.M);
  k_inst_gather<<<grid_for(n2, 256), 256, 0, s>>>(P.i_col, P.i_row, P.x, P.c, P.s, P.Ns, P.M, P.i_x, P.i_c, P.i_s);
  TH_LAUNCHED();
  InstView V;
  V.noff = P.bnoff;
  V.eoff = P.beoff;
  V.iend = P.i_end;
  V.ient = P.i_ent;
  V.inb = P.i_nb;
  V.iru = P.i_ru;
  V.irv = P.i_rv;
  V.coff = P.i_coff;
  V.roff = P.i_roff;
  V.qoff = P.i_qoff;
  V.ncol = P.i_ncol;
  V.cwide = P.i_cwide;
  V.pfirst = P.i_pfirst;
  V.pbase = P.i_pbase;
  V.pw = P.i_pw;
  V.ell = P.i_ell;
  V.rpos = P.i_rpos;
  V.rrow = P.i_rrow;
  V.hs = P.i_hs;
  V.hl = P.i_hl;
  V.hoff = P.i_hoff;
  V.hH = P.i_hH;
  V.hnb = P.i_hnb;
  V.xg = P.i_xg;
  V.ideg = P.i_deg;
  V.kind = P.bkind;
  V.c = P.i_c;
  V.x = P.i_x;
  V.s = P.i_s;
  V.rg = P.i_rg;
  V.C = P.iml_C;
  V.beta = (float)a.beta;
  V.inv_beta = (float)(1.0 / a.beta);
  V.beta_d = a.beta;
  V.lo = P.lo_u;
  V.hi = P.hi_u;
  V.step_rule = a.step_rule;
  V.epochs = a.epochs;
  V.R = a.refresh_every;
  V.tol = a.tol;
  V.ep_out = P.i_ep;
  V.conv_out = P.i_conv;
  V.t_out = P.i_t;
  V.round = P.iround_on ? 1 : 0;
  P.iround_done = P.iround_on;
  V.seed = P.iround_seed;
  V.reps = P.iround_reps;
  V.vid = P.i_vid;
  V.lab = P.i_lab;
  V.r_obj = P.i_robj;
  V.r_rep = P.i_rrep;
  V.r_best = P.i_rbest;
  V.r_status = P.i_rstatus;
  V.xout = P.i_xout;
  V.rho_out = P.i_rhoout;
  V.done = P.i_done;
  const DevLimits L = dev_limits();
  k_inst_stamp<<<1, 1, 0, s>>>(P.i_t + 2 * count);
  TH_LAUNCHED();
  TH_CUDA(cudaEventRecord(P.i_events[0], s));
  // fork: every class on its own stream, the largest clusters first so they
  // find whole SMs free
  TH_CUDA(cudaEventRecord(P.i_events[2 + NCLS], s));
  for (int c = NCLS - 1; c >= 0; --c) {
    const int64_t cnt = P.h_icls_off[c + 1] - P.h_icls_off[c];
    if (cnt == 0) continue;
    cudaStream_t st = P.i_streams[c];
    TH_CUDA(cudaStreamWaitEvent(st, P.i_events[2 + NCLS], 0));
    const int32_t* ord = P.i_order + P.h_icls_off[c];
    const size_t smem = (size_t)P.h_icls_smem[c];
    // clusters take 8 lanes per column through the CSR (fewer remote
    // round trips per column than one thread per column)
    const int g = (CLASSES[c].K > 1) ? 8 : P.iml_G;
    if (g == 4) launch_class<4>(c, V, ord, cnt, smem, L.optin, st);
    else if (g == 8) launch_class<8>(c, V, ord, cnt, smem, L.optin, st);
    else launch_class<1>(c, V, ord, cnt, smem, L.optin, st);
    TH_CUDA(cudaEventRecord(P.i_events[2 + c], st));
    TH_CUDA(cudaStreamWaitEvent(s, P.i_events[2 + c], 0));
  }
  TH_CUDA(cudaEventRecord(P.i_events[1], s));
  k_inst_scatter<<<grid_for(n2, 256), 256, 0, s>>>(P.i_col, P.i_row, P.i_x, P.i_s, P.Ns, P.M, P.x, P.s);
  TH_LAUNCHED();
  P.h_iep.resize(count);
  P.h_iconv.resize(count);
  P.h_it.resize(2 * count + 1);
  TH_CUDA(cudaMemcpyAsync(P.h_iep.data(), P.i_ep, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(P.h_iconv.data(), P.i_conv, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(P.h_it.data(), P.i_t, (2 * count + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CUDA(cudaGetLastError());
  float ms = 0.f;
  TH_CUDA(cudaEventElapsedTime(&ms, P.i_events[0], P.i_events[1]));
  sweep_ms = ms;
}

void inst_release(Problem& P) {
  for (auto& st : P.i_streams)
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
      st = nullptr;
    }
  for (auto& ev : P.i_events)
    if (ev) {
      cudaEventDestroy(ev);
      ev = nullptr;
    }
}

}  // namespace thetis
