// Building a problem on the device: graph builders (Sec. 2 vertex cover,
// App. B.2 independent set, App. B.3 multiway cut), the CSR twin, the greedy
// colouring of the column-intersection graph (Jones-Plassmann rounds, which
// colour exactly like the sequential greedy in the same total order), and the
// colour-ordered internal layout.
#include <algorithm>
#include <cmath>

#include "problem.cuh"

namespace thetis {


static int bits_for(int64_t n) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) < n) ++b;
  return b;
}

#define GSTRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Colour histograms have only a handful of distinct keys per warp but every
// warp of the grid hits the same few bins, so counts go to per-block shared
// counters when the bins fit (HIST_SMEM_BINS), then one global atomic per bin
// and block; otherwise the lanes of a warp that share a key fold into one
// global atomic.
constexpr int64_t HIST_SMEM_BINS = 8192;
constexpr int HIST_GRID = 304;  // blocks of a shared-counter histogram kernel

__device__ __forceinline__ void hist_init(int* sh, int64_t nbins, bool use_sh) {
  if (use_sh)
    for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
}

__device__ __forceinline__ void hist_add(int64_t* cnt, int* sh, bool use_sh, uint32_t key, bool valid) {
  unsigned act = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  unsigned peers = __match_any_sync(act, key);
  int lane = threadIdx.x & 31;
  if (lane == __ffs(peers) - 1) {
    if (use_sh) atomicAdd(&sh[key], __popc(peers));
    else atomicAdd((unsigned long long*)&cnt[key], (unsigned long long)__popc(peers));
  }
}

__device__ __forceinline__ void hist_flush(int64_t* cnt, const int* sh, int64_t nbins, bool use_sh) {
  if (!use_sh) return;
  __syncthreads();
  for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x)
    if (sh[b]) atomicAdd((unsigned long long*)&cnt[b], (unsigned long long)sh[b]);
}

static void hist_launch_shape(int64_t n, int64_t nbins, int* grid, size_t* smem) {
  const bool use_sh = nbins <= HIST_SMEM_BINS;
  *grid = use_sh ? grid_for(n, 256, HIST_GRID) : grid_for(n, 256);
  *smem = use_sh ? (size_t)nbins * sizeof(int) : 0;
}

// ---------------------------------------------------------------------------
// graph builders
// ---------------------------------------------------------------------------
// the vertex of every endpoint slot: eu of edge e at e, ev at m + e
__global__ void k_slot_vertices(const int32_t* eu, const int32_t* ev, int64_t m, uint32_t* keys) {
  GSTRIDE(e, m) {
    keys[e] = (uint32_t)eu[e];
    keys[m + e] = (uint32_t)ev[e];
  }
}
__global__ void k_slot_edges(uint32_t* slots, int64_t m) {
  GSTRIDE(i, 2 * m) {
    const uint32_t p = slots[i];
    slots[i] = (p >= (uint64_t)m) ? (uint32_t)(p - m) : p;
  }
}

__global__ void k_check_edges(const int32_t* eu, const int32_t* ev, int64_t m, int64_t n, int* err) {
  GSTRIDE(e, m) {
    int32_t a = eu[e], b = ev[e];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) atomicExch(err, 1);
  }
}

__global__ void k_u32_to_i32(const uint32_t* in, int32_t* out, int64_t n) {
  GSTRIDE(i, n) out[i] = (int32_t)in[i];
}

__global__ void k_edge_lp_vectors(int kind, const float* w, int64_t n, int64_t m, float* b, float* c,
                                  float* lo, float* hi, uint8_t* rk, int* err) {
  GSTRIDE(i, n > m ? n : m) {
    if (i < n) {
      float wv = w[i];
      if (!(wv > 0.f) || !isfinite(wv)) atomicExch(err, 2);
      c[i] = (kind == KIND_VC) ? wv : -wv;
      lo[i] = 0.f;
      hi[i] = 1.f;
    }
    if (i < m) {
      b[i] = 1.f;
      rk[i] = (kind == KIND_VC) ? THETIS_ROW_GE : THETIS_ROW_LE;
    }
  }
}

static int read_flag(int* d, cudaStream_t s) {
  int h = 0;
  TH_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  return h;
}

// vertex -> incident edges (stable: edges where v = eu in edge order, then v = ev)
// (the 2m endpoint slots p -- eu of edge p, then ev of edge p - m -- grouped by
// vertex in slot order, then each slot replaced by its edge)
static void incidence(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, int64_t*& ptr,
                      uint32_t*& edges, Arena& tmp, cudaStream_t s) {
  uint32_t* keys = tmp.alloc<uint32_t>(2 * m);
  edges = tmp.alloc<uint32_t>(2 * m);
  if (m > 0) {
    k_slot_vertices<<<grid_for(m, 256), 256, 0, s>>>(eu, ev, m, keys);
    TH_LAUNCHED();
  }
  ptr = tmp.alloc<int64_t>(n + 1);
  group_by_key(keys, nullptr, 2 * m, n, edges, ptr, tmp, s);
  if (m > 0) {
    k_slot_edges<<<grid_for(2 * m, 256), 256, 0, s>>>(edges, m);
    TH_LAUNCHED();
  }
}

// vertex -> incident edges as an int32 CSC (used by the batch builder)
void incidence_csc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, int64_t*& ptr, int32_t*& rows,
                   Arena& tmp, cudaStream_t s) {
  uint32_t* edges;
  incidence(n, m, eu, ev, ptr, edges, tmp, s);
  rows = tmp.alloc<int32_t>(2 * m + 1);
  if (m > 0) {
    k_u32_to_i32<<<grid_for(2 * m, 256), 256, 0, s>>>(edges, rows, 2 * m);
    TH_LAUNCHED();
  }
}

void build_vc_is_raw(int kind, int64_t n, int64_t m, const int32_t* d_eu, const int32_t* d_ev,
                     const float* d_w, RawLP& raw, Arena& tmp, cudaStream_t s) {
  int* err = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (m > 0) {
    k_check_edges<<<grid_for(m, 256), 256, 0, s>>>(d_eu, d_ev, m, n, err);
    TH_LAUNCHED();
  }
  TH_CHECK(read_flag(err, s) == 0, THETIS_E_INVALID, "edge endpoint out of range or a loop");
  int64_t* ptr;
  uint32_t* edges;
  incidence(n, m, d_eu, d_ev, ptr, edges, tmp, s);
  raw.M = m;
  raw.Ns = n;
  raw.nnz = 2 * m;
  raw.colptr = ptr;
  raw.rowidx = tmp.alloc<int32_t>(2 * m);
  if (m > 0) {
    k_u32_to_i32<<<grid_for(2 * m, 256), 256, 0, s>>>(edges, raw.rowidx, 2 * m);
    TH_LAUNCHED();
  }
  raw.val = nullptr;
  raw.b = tmp.alloc<float>(m);
  raw.c = tmp.alloc<float>(n);
  raw.lo = tmp.alloc<float>(n);
  raw.hi = tmp.alloc<float>(n);
  raw.row_kind = tmp.alloc<uint8_t>(m);
  k_edge_lp_vectors<<<grid_for(std::max(n, m), 256), 256, 0, s>>>(kind, d_w, n, m, raw.b, raw.c,
                                                                   raw.lo, raw.hi, raw.row_kind, err);
  TH_LAUNCHED();
  TH_CHECK(read_flag(err, s) == 0, THETIS_E_INVALID, "vertex weights must be finite and > 0");
  raw.block_k = 1;
  raw.n_blocks = 0;
  raw.bounds_uniform = true;
  raw.lo_u = 0.f;
  raw.hi_u = 1.f;
  raw.slack_sign_uniform = (kind == KIND_VC) ? -1 : 1;
}

// Set cover: validate the set lists (elements in range and strictly
// increasing inside a set, costs finite and > 0) and count every element's sets.
__global__ void k_sc_check(const int64_t* ptr, const int32_t* elems, const float* cost, int64_t n_sets,
                           int64_t n_elem, int64_t* ecount, int* err) {
  GSTRIDE(j, n_sets) {
    const int64_t q0 = ptr[j], q1 = ptr[j + 1];
    if (q1 < q0) {
      atomicExch(err, 1);
      continue;
    }
    if (!(cost[j] > 0.f) || !isfinite(cost[j])) atomicExch(err, 2);
    for (int64_t q = q0; q < q1; ++q) {
      const int32_t a = elems[q];
      if (a < 0 || a >= n_elem || (q > q0 && elems[q - 1] >= a)) {
        atomicExch(err, 1);
        break;
      }
      atomicAdd((unsigned long long*)&ecount[a], 1ull);
    }
  }
}

__global__ void k_sc_vectors(const float* cost, int64_t n_sets, int64_t n_elem, float* b, float* c, float* lo,
                             float* hi, uint8_t* rk, const int64_t* ecount, int* err, int* fmax) {
  GSTRIDE(i, n_sets > n_elem ? n_sets : n_elem) {
    if (i < n_sets) {
      c[i] = cost[i];
      lo[i] = 0.f;
      hi[i] = 1.f;
    }
    if (i < n_elem) {
      b[i] = 1.f;
      rk[i] = THETIS_ROW_GE;
      if (ecount[i] == 0) atomicExch(err, 3);
      atomicMax(fmax, (int)min(ecount[i], (int64_t)INT32_MAX));
    }
  }
}

// (element, set) pairs in set-major order, so a stable sort by element keeps
// every element's sets in increasing id
__global__ void k_sc_pairs(const int64_t* ptr, const int32_t* elems, int64_t n_sets, uint32_t* keys, uint32_t* vals) {
  GSTRIDE(j, n_sets)
  for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) {
    keys[q] = (uint32_t)elems[q];
    vals[q] = (uint32_t)j;
  }
}

void build_sc_raw(int64_t n_elem, int64_t n_sets, int64_t nnz, const int64_t* d_ptr, const int32_t* d_elems,
                  const float* d_cost, RawLP& raw, int64_t*& eptr, int32_t*& esets, int32_t& f, Arena& keep,
                  Arena& tmp, cudaStream_t s) {
  int* err = tmp.alloc<int>(2);
  TH_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
  int64_t* ecount = tmp.alloc<int64_t>(n_elem + 1);
  TH_CUDA(cudaMemsetAsync(ecount, 0, (n_elem + 1) * sizeof(int64_t), s));
  k_sc_check<<<grid_for(n_sets, 256), 256, 0, s>>>(d_ptr, d_elems, d_cost, n_sets, n_elem, ecount, err);
  TH_LAUNCHED();
  int e1 = read_flag(err, s);
  TH_CHECK(e1 != 1, THETIS_E_INVALID, "set lists must hold element ids in [0, n_elements), increasing inside a set");
  TH_CHECK(e1 != 2, THETIS_E_INVALID, "set costs must be finite and > 0");
  raw.M = n_elem;
  raw.Ns = n_sets;
  raw.nnz = nnz;
  raw.colptr = const_cast<int64_t*>(d_ptr);
  raw.rowidx = const_cast<int32_t*>(d_elems);
  raw.val = nullptr;
  raw.b = tmp.alloc<float>(n_elem);
  raw.c = tmp.alloc<float>(n_sets);
  raw.lo = tmp.alloc<float>(n_sets);
  raw.hi = tmp.alloc<float>(n_sets);
  raw.row_kind = tmp.alloc<uint8_t>(n_elem);
  k_sc_vectors<<<grid_for(std::max(n_sets, n_elem), 256), 256, 0, s>>>(d_cost, n_sets, n_elem, raw.b, raw.c, raw.lo,
                                                                       raw.hi, raw.row_kind, ecount, err, err + 1);
  TH_LAUNCHED();
  int hf[2];
  TH_CUDA(cudaMemcpyAsync(hf, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CHECK(hf[0] != 3, THETIS_E_INVALID, "an element lies in no set: the covering LP is infeasible");
  f = hf[1];
  raw.block_k = 1;
  raw.n_blocks = 0;
  raw.bounds_uniform = true;
  raw.lo_u = 0.f;
  raw.hi_u = 1.f;
  raw.slack_sign_uniform = -1;
  // element -> sets lists (original ids) for the repair and the rounding
  uint32_t* keys = tmp.alloc<uint32_t>(nnz + 1);
  uint32_t* vals = tmp.alloc<uint32_t>(nnz + 1);
  k_sc_pairs<<<grid_for(n_sets, 256), 256, 0, s>>>(d_ptr, d_elems, n_sets, keys, vals);
  TH_LAUNCHED();
  radix_sort_pairs(keys, vals, nnz, bits_for(n_elem + 1), tmp, s);
  eptr = keep.alloc<int64_t>(n_elem + 1);
  exclusive_scan_i64(ecount, eptr, n_elem, tmp, s);
  esets = keep.alloc<int32_t>(nnz + 1);
  if (nnz > 0) {
    k_u32_to_i32<<<grid_for(nnz, 256), 256, 0, s>>>(vals, esets, nnz);
    TH_LAUNCHED();
  }
}

// Multiway cut: x_{v,i} at v*k+i (2 deg(v) entries), z_{e,i} at n*k+e*k+i.
__global__ void k_mc_counts(const int64_t* iptr, int64_t n, int64_t m, int32_t k, int64_t* cnt) {
  GSTRIDE(j, n * k + m * k) {
    if (j < n * k) {
      int64_t v = j / k;
      cnt[j] = 2 * (iptr[v + 1] - iptr[v]);
    } else {
      cnt[j] = 2;
    }
  }
}

__global__ void k_mc_fill(const int64_t* iptr, const uint32_t* iedge, const int32_t* eu, int64_t n,
                          int64_t m, int32_t k, const int64_t* colptr, int32_t* rowidx, float* val) {
  GSTRIDE(j, n * k + m * k) {
    int64_t q = colptr[j];
    if (j < n * k) {
      int64_t v = j / k;
      int32_t i = (int32_t)(j % k);
      for (int64_t t = iptr[v]; t < iptr[v + 1]; ++t) {
        int64_t e = iedge[t];
        bool is_u = (eu[e] == v);
        int64_t rp = 2 * (e * k + i);
        rowidx[q] = (int32_t)rp;
        val[q] = is_u ? -1.f : 1.f;
        rowidx[q + 1] = (int32_t)(rp + 1);
        val[q + 1] = is_u ? 1.f : -1.f;
        q += 2;
      }
    } else {
      int64_t z = j - n * k;  // e*k + i
      rowidx[q] = (int32_t)(2 * z);
      val[q] = 1.f;
      rowidx[q + 1] = (int32_t)(2 * z + 1);
      val[q + 1] = 1.f;
    }
  }
}

__global__ void k_mc_vectors(const float* ce, const int32_t* term, int64_t n, int64_t m, int32_t k,
                             float* b, float* c, float* lo, float* hi, uint8_t* rk, int64_t* bfirst,
                             int* err) {
  int64_t Ns = n * k + m * k;
  GSTRIDE(i, Ns > 2 * m * k ? Ns : 2 * m * k) {
    if (i < Ns) {
      lo[i] = 0.f;
      hi[i] = 1.f;
      if (i < n * k) {
        c[i] = 0.f;
      } else {
        float w = ce[(i - n * k) / k];
        if (!(w >= 0.f) || !isfinite(w)) atomicExch(err, 2);
        c[i] = 0.5f * w;
      }
    }
    if (i < 2 * m * k) {
      b[i] = 0.f;
      rk[i] = THETIS_ROW_GE;
    }
    if (i < n) bfirst[i] = i * k;
  }
}

__global__ void k_mc_terminals(const int32_t* term, int64_t n, int32_t k, float* lo, float* hi, int* err) {
  int t = threadIdx.x;
  if (t >= k) return;
  int64_t v = term[t];
  if (v < 0 || v >= n) {
    atomicExch(err, 3);
    return;
  }
  for (int i = 0; i < k; ++i) {
    float e = (i == t) ? 1.f : 0.f;
    lo[v * k + i] = e;
    hi[v * k + i] = e;
  }
  for (int q = 0; q < t; ++q)
    if (term[q] == v) atomicExch(err, 4);
}

void build_mc_raw(int64_t n, int64_t m, const int32_t* d_eu, const int32_t* d_ev,
                  const float* d_ce, int32_t k, const int32_t* d_term, RawLP& raw, Arena& tmp,
                  cudaStream_t s) {
  int* err = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (m > 0) {
    k_check_edges<<<grid_for(m, 256), 256, 0, s>>>(d_eu, d_ev, m, n, err);
    TH_LAUNCHED();
  }
  TH_CHECK(read_flag(err, s) == 0, THETIS_E_INVALID, "edge endpoint out of range or a loop");
  int64_t* iptr;
  uint32_t* iedge;
  incidence(n, m, d_eu, d_ev, iptr, iedge, tmp, s);
  int64_t Ns = n * k + m * k;
  raw.M = 2 * m * k;
  raw.Ns = Ns;
  raw.colptr = tmp.alloc<int64_t>(Ns + 1);
  k_mc_counts<<<grid_for(Ns, 256), 256, 0, s>>>(iptr, n, m, k, raw.colptr);
  TH_LAUNCHED();
  exclusive_scan_i64(raw.colptr, raw.colptr, Ns, tmp, s);
  raw.nnz = 4 * m * k + 2 * m * k;
  raw.rowidx = tmp.alloc<int32_t>(raw.nnz);
  raw.val = tmp.alloc<float>(raw.nnz);
  k_mc_fill<<<grid_for(Ns, 256), 256, 0, s>>>(iptr, iedge, d_eu, n, m, k, raw.colptr, raw.rowidx, raw.val);
  TH_LAUNCHED();
  raw.b = tmp.alloc<float>(raw.M);
  raw.c = tmp.alloc<float>(Ns);
  raw.lo = tmp.alloc<float>(Ns);
  raw.hi = tmp.alloc<float>(Ns);
  raw.row_kind = tmp.alloc<uint8_t>(raw.M);
  raw.block_first = tmp.alloc<int64_t>(n);
  k_mc_vectors<<<grid_for(std::max(Ns, 2 * m * k), 256), 256, 0, s>>>(
      d_ce, d_term, n, m, k, raw.b, raw.c, raw.lo, raw.hi, raw.row_kind, raw.block_first, err);
  TH_LAUNCHED();
  k_mc_terminals<<<1, 32, 0, s>>>(d_term, n, k, raw.lo, raw.hi, err);
  TH_LAUNCHED();
  int f = read_flag(err, s);
  TH_CHECK(f != 2, THETIS_E_INVALID, "edge weights must be finite and >= 0");
  TH_CHECK(f != 3, THETIS_E_INVALID, "terminal out of range");
  TH_CHECK(f != 4, THETIS_E_INVALID, "terminals must be distinct");
  raw.block_k = k;
  raw.n_blocks = n;
  raw.bounds_uniform = false;  // terminal blocks are fixed
  raw.slack_sign_uniform = -1;
}

// Pairwise MAP: node column (i, a) at i*k + a holds -1 in row 2*e*k + a of every
// edge e with eu[e] = i and in row 2*e*k + k + a of every edge with ev[e] = i;
// edge column (e, a, b) at n*k + e*k*k + a*k + b holds +1 in rows 2*e*k + a and
// 2*e*k + k + b.
__global__ void k_map_counts(const int64_t* iptr, int64_t n, int64_t m, int32_t k, int64_t* cnt) {
  GSTRIDE(j, n * k + m * (int64_t)k * k) cnt[j] = (j < n * k) ? iptr[j / k + 1] - iptr[j / k] : 2;
}

__global__ void k_map_fill(const int64_t* iptr, const uint32_t* iedge, const int32_t* eu, int64_t n, int64_t m,
                           int32_t k, const int64_t* colptr, int32_t* rowidx, float* val) {
  GSTRIDE(j, n * k + m * (int64_t)k * k) {
    int64_t q = colptr[j];
    if (j < n * k) {
      const int64_t v = j / k;
      const int32_t a = (int32_t)(j % k);
      for (int64_t t = iptr[v]; t < iptr[v + 1]; ++t) {
        const int64_t e = iedge[t];
        rowidx[q] = (int32_t)(2 * e * k + (eu[e] == v ? 0 : k) + a);
        val[q++] = -1.f;
      }
    } else {
      const int64_t t = j - n * k, e = t / ((int64_t)k * k);
      const int32_t a = (int32_t)((t / k) % k), b = (int32_t)(t % k);
      rowidx[q] = (int32_t)(2 * e * k + a);
      val[q] = 1.f;
      rowidx[q + 1] = (int32_t)(2 * e * k + k + b);
      val[q + 1] = 1.f;
    }
  }
}

__global__ void k_map_vectors(const float* tn, const float* te, int64_t n, int64_t m, int32_t k, float* b, float* c,
                              float* lo, float* hi, uint8_t* rk, int64_t* bfirst, int* err) {
  const int64_t Ns = n * k + m * (int64_t)k * k, M = 2 * m * (int64_t)k;
  GSTRIDE(i, Ns > M ? Ns : M) {
    if (i < Ns) {
      const float t = (i < n * k) ? tn[i] : te[i - n * k];
      if (!isfinite(t)) atomicExch(err, 2);
      c[i] = -t;
      lo[i] = 0.f;
      hi[i] = 1.f;
    }
    if (i < M) {
      b[i] = 0.f;
      rk[i] = THETIS_ROW_EQ;
    }
    if (i < n) bfirst[i] = i * k;
  }
}

void build_map_raw(int64_t n, int64_t m, int32_t k, const int32_t* d_eu, const int32_t* d_ev, const float* d_tn,
                   const float* d_te, RawLP& raw, Arena& tmp, cudaStream_t s) {
  int* err = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (m > 0) {
    k_check_edges<<<grid_for(m, 256), 256, 0, s>>>(d_eu, d_ev, m, n, err);
    TH_LAUNCHED();
  }
  TH_CHECK(read_flag(err, s) == 0, THETIS_E_INVALID, "edge endpoint out of range or a loop");
  int64_t* iptr;
  uint32_t* iedge;
  incidence(n, m, d_eu, d_ev, iptr, iedge, tmp, s);
  const int64_t Ns = n * k + m * (int64_t)k * k;
  raw.M = 2 * m * (int64_t)k;
  raw.Ns = Ns;
  raw.colptr = tmp.alloc<int64_t>(Ns + 1);
  k_map_counts<<<grid_for(Ns, 256), 256, 0, s>>>(iptr, n, m, k, raw.colptr);
  TH_LAUNCHED();
  exclusive_scan_i64(raw.colptr, raw.colptr, Ns, tmp, s);
  raw.nnz = 2 * m * (int64_t)k + 2 * m * (int64_t)k * k;
  raw.rowidx = tmp.alloc<int32_t>(raw.nnz + 1);
  raw.val = tmp.alloc<float>(raw.nnz + 1);
  k_map_fill<<<grid_for(Ns, 256), 256, 0, s>>>(iptr, iedge, d_eu, n, m, k, raw.colptr, raw.rowidx, raw.val);
  TH_LAUNCHED();
  raw.b = tmp.alloc<float>(raw.M + 1);
  raw.c = tmp.alloc<float>(Ns);
  raw.lo = tmp.alloc<float>(Ns);
  raw.hi = tmp.alloc<float>(Ns);
  raw.row_kind = tmp.alloc<uint8_t>(raw.M + 1);
  raw.block_first = tmp.alloc<int64_t>(n);
  k_map_vectors<<<grid_for(std::max(Ns, raw.M), 256), 256, 0, s>>>(d_tn, d_te, n, m, k, raw.b, raw.c, raw.lo, raw.hi,
                                                                   raw.row_kind, raw.block_first, err);
  TH_LAUNCHED();
  TH_CHECK(read_flag(err, s) == 0, THETIS_E_INVALID, "scores must be finite");
  raw.block_k = k;
  raw.n_blocks = n;
  raw.bounds_uniform = true;
  raw.lo_u = 0.f;
  raw.hi_u = 1.f;
  raw.slack_sign_uniform = 0;
}

// ---------------------------------------------------------------------------
// general layout
// ---------------------------------------------------------------------------
__global__ void k_validate(const int64_t* colptr, const int32_t* rowidx, const float* val,
                           const float* lo, const float* hi, const uint8_t* rk, int64_t Ns,
                           int64_t M, int64_t nnz, int* err, int* notpm1) {
  GSTRIDE(j, Ns) {
    if (colptr[j + 1] < colptr[j]) atomicExch(err, 1);
    if (!(lo[j] <= hi[j])) atomicExch(err, 2);
  }
  GSTRIDE(p, nnz) {
    int32_t r = rowidx[p];
    if (r < 0 || r >= M) atomicExch(err, 3);
    if (val) {
      float v = val[p];
      if (!isfinite(v)) atomicExch(err, 4);
      if (v != 1.f && v != -1.f) atomicExch(notpm1, 1);
    }
  }
  GSTRIDE(i, M) {
    if (rk[i] > 2) atomicExch(err, 5);
  }
}

__global__ void k_block_claim(const int64_t* bfirst, int64_t nb, int32_t k, int64_t Ns, int32_t* blk,
                              int* err) {
  GSTRIDE(t, nb) {
    int64_t f = bfirst[t];
    if (f < 0 || f + k > Ns) {
      atomicExch(err, 6);
      continue;
    }
    for (int q = 0; q < k; ++q)
      if (atomicCAS(&blk[f + q], -1, (int32_t)t) != -1) atomicExch(err, 7);
  }
}

// Per structural column: is it the first column of a free unit? is it fixed?
__global__ void k_unit_flags(const int32_t* blk, const int64_t* bfirst, int32_t k, const float* lo,
                             const float* hi, int64_t Ns, int64_t* start_flag, int64_t* fixed_flag) {
  GSTRIDE(j, Ns) {
    int32_t t = blk ? blk[j] : -1;
    bool st = false, fx = false;
    if (t < 0) {
      fx = !(lo[j] < hi[j]);
      st = !fx;
    } else {
      int64_t f = bfirst[t];
      bool bfixed = true;
      for (int q = 0; q < k; ++q)
        if (lo[f + q] < hi[f + q]) bfixed = false;
      fx = bfixed;
      st = (j == f) && !bfixed;
    }
    start_flag[j] = st ? 1 : 0;
    fixed_flag[j] = fx ? 1 : 0;
  }
}

// unit_of_col, unit first column, unit length
__global__ void k_unit_ids(const int32_t* blk, const int64_t* bfirst, int32_t k, int64_t Ns,
                           const int64_t* start_scan, const int64_t* fixed_flag, int64_t* unit_of_col,
                           int64_t* ufirst, int32_t* ulen) {
  GSTRIDE(j, Ns) {
    if (fixed_flag[j]) {
      unit_of_col[j] = -1;
      continue;
    }
    int32_t t = blk ? blk[j] : -1;
    int64_t f = (t < 0) ? j : bfirst[t];
    int64_t u = start_scan[f];
    unit_of_col[j] = u;
    if (j == f) {
      ufirst[u] = f;
      ulen[u] = (t < 0) ? 1 : k;
    }
  }
}

__global__ void k_slack_flags(const uint8_t* rk, int64_t M, int64_t* has) {
  GSTRIDE(i, M) has[i] = (rk[i] != THETIS_ROW_EQ) ? 1 : 0;
}

// the segment of every position (the column of a CSC entry, the row of a CSR
// entry): a segment of up to 32 positions written by its thread, a longer one
// by its whole warp
__global__ void k_seg_ids(const int64_t* colptr, int64_t Ns, uint32_t* colof) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < Ns; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = base + threadIdx.x;
    int64_t p0 = 0, p1 = 0;
    if (j < Ns) {
      p0 = colptr[j];
      p1 = colptr[j + 1];
    }
    const bool longc = p1 - p0 > 32;
    if (!longc)
      for (int64_t p = p0; p < p1; ++p) colof[p] = (uint32_t)j;
    unsigned mb = __ballot_sync(0xffffffffu, longc);
    while (mb) {
      const int l = __ffs(mb) - 1;
      mb &= mb - 1;
      const int64_t a = __shfl_sync(0xffffffffu, p0, l), e = __shfl_sync(0xffffffffu, p1, l);
      const uint32_t jj = (uint32_t)__shfl_sync(0xffffffffu, j, l);
      for (int64_t p = a + lane; p < e; p += 32) colof[p] = jj;
    }
  }
}

// csr_p: positions p sorted by row (stable); check for a repeated (row, col)
__global__ void k_csr_dupcheck(const int64_t* rowptr, const uint32_t* csr_p, const uint32_t* colof,
                               int64_t M, int* err) {
  GSTRIDE(i, M) {
    for (int64_t q = rowptr[i] + 1; q < rowptr[i + 1]; ++q)
      if (colof[csr_p[q]] == colof[csr_p[q - 1]]) atomicExch(err, 8);
  }
}

__global__ void k_unit_keys(const int64_t* colptr, const int64_t* ufirst, const int32_t* ulen, int64_t Us,
                            int64_t U, uint64_t seed, const uint32_t* prio_col, const uint32_t* prio_row,
                            const int64_t* slack_row, int64_t* unnz, uint64_t* uh) {
  GSTRIDE(u, U) {
    uint64_t pid = (uint64_t)u;
    if (u < Us) {
      int64_t f = ufirst[u];
      unnz[u] = colptr[f + ulen[u]] - colptr[f];
      if (prio_col) pid = prio_col[f];
    } else {
      unnz[u] = 1;
      if (prio_row) pid = prio_row[slack_row[u - Us]];
    }
    uh[u] = sm64_at(seed, pid);
  }
}

struct JPView {
  const int64_t* colptr;
  const int32_t* rowidx;
  const int64_t* rowptr;
  const uint32_t* csr_p;
  const uint32_t* colof;
  const int64_t* unit_of_col;
  const int64_t* slack_unit;  // per row: unit id or -1
  const int64_t* ufirst;
  const int32_t* ulen;
  const int64_t* unnz;
  const uint64_t* uh;
  int64_t Us;
  const int64_t* slack_row;   // slack unit s -> row
};

// Priority order of the colouring: structural units before slack units, then
// (non-zeros desc, splitmix64(seed, unit) desc, unit id asc).
__device__ __forceinline__ bool higher(const JPView& V, int64_t a, int64_t b) {
  const bool sa = a >= V.Us, sb = b >= V.Us;
  if (sa != sb) return !sa;
  int64_t na = V.unnz[a], nb = V.unnz[b];
  if (na != nb) return na > nb;
  uint64_t ha = V.uh[a], hb = V.uh[b];
  if (ha != hb) return ha > hb;
  return a < b;
}

// Jones-Plassmann over the structural units, driven by data flow, with the
// rows as the dependency structure.  Every row is a clique of the
// column-intersection graph, so in the sequential greedy order the units of a
// row are coloured one after the other: a unit is ready once, in each of its
// rows, the unit just before it is coloured (cnt[u] = rows in which u has a
// predecessor), and the colours it must avoid are those of the row prefixes
// before it.  Per row a 128-bit mask holds the colours of the coloured prefix
// (bit RC_OVF: some colour >= RC_OVF is among them; then, or when colours
// 0..RC_OVF-1 are all taken, the colour is found from the prefixes
// themselves).  Per unit a list of (row, successor) entries, the rows where
// it has a predecessor first (npred[u] of them).  A row of exactly two units
// needs no mask: the second reads the first one's colour directly.  Units of
// one frontier share no row.  Slack units come last in the priority order and
// never conflict with one another, so each takes, after all structural units
// are coloured, the smallest colour its row does not hold (k_slack_color) --
// the sequential greedy result.
constexpr int64_t JP_BIG = 1024;           // list length above which a whole CTA serves a unit
constexpr uint32_t RC_BIG = 0x80000000u;   // successor flag: that unit's own list is long
constexpr uint32_t RC_NONE = 0xffffffffu;  // no unit
constexpr int RC_OVF = 127;                // mask bit: a colour >= RC_OVF in the prefix
constexpr uint32_t RC_TWO = 0x80000000u;   // list-entry flag for a row of exactly two units (see k_row_links)

// Per CSR entry: the structural unit of its column, RC_NONE for a fixed column.
__global__ void k_row_units(JPView V, int64_t nnz, uint32_t* rowunit) {
  GSTRIDE(q, nnz) {
    const int64_t w = V.unit_of_col[V.colof[V.csr_p[q]]];
    rowunit[q] = w >= 0 ? (uint32_t)w : RC_NONE;
  }
}

// Per structural unit its priority key (non-zeros, hash) as one 16-byte word.
__global__ void k_unit_prio(JPView V, int64_t Us, ulonglong2* key) {
  GSTRIDE(u, Us) key[u] = make_ulonglong2((unsigned long long)V.unnz[u], (unsigned long long)V.uh[u]);
}

// Structural unit a before structural unit b in the colouring order.
__device__ __forceinline__ bool ahead(ulonglong2 ka, uint32_t a, ulonglong2 kb, uint32_t b) {
  if (ka.x != kb.x) return ka.x > kb.x;
  if (ka.y != kb.y) return ka.y > kb.y;
  return a < b;
}

// One thread per CSR entry q of row i: the rank of its unit in row i, i.e.
// the occurrences in row i of units ahead of it.  A unit repeated in a row
// (two columns of one block) keeps its first occurrence; later ones, and
// fixed columns, get rank -1.  Distinct units get distinct ranks, so
// sorted[rowptr[i] + rank] lists the row's units in order (with a gap where a
// repeat was counted).
__global__ void k_row_rank(JPView V, const uint32_t* rowof, const uint32_t* rowunit, const ulonglong2* key,
                           int64_t nnz, int32_t* rank, uint32_t* sorted, int32_t* rowcnt, int* repeat) {
  GSTRIDE(q, nnz) {
    const uint32_t u = rowunit[q];
    int32_t r = -1;
    if (u != RC_NONE) {
      const int64_t i = rowof[q];
      const int64_t q0 = V.rowptr[i], q1 = V.rowptr[i + 1];
      const ulonglong2 ku = key[u];
      int32_t c = 0;
      bool rep = false;
      for (int64_t t = q0; t < q1; ++t) {
        const uint32_t w = rowunit[t];
        if (w == RC_NONE) continue;
        if (w == u) {
          rep = rep || t < q;
          continue;
        }
        c += ahead(key[w], w, ku, u);
      }
      if (!rep) {
        r = c;
        sorted[q0 + c] = u;
        atomicAdd(&rowcnt[i], 1);
      } else {
        *repeat = 1;  // a block with two columns in this row
      }
    }
    rank[q] = r;
  }
}

// One thread per CSR entry q: for its column non-zero p = csr_p[q], whether
// the unit has a predecessor in the row (hc[p] = 1) or is the row's first
// (lc[p] = 1) -- both 0 for a fixed column or a repeat --, the unit after it
// in the row (succ[p], RC_NONE if last) and the list entry: the row id, except
// in a row of exactly two units, where the first unit's entry is the row id
// with RC_TWO (no mask needed) and the second unit's entry is the first
// unit's id with RC_TWO (its colour is read directly).
__global__ void k_row_links(JPView V, const uint32_t* rowof, const int32_t* rank, const uint32_t* sorted,
                            const int32_t* rowcnt, int64_t nnz, int64_t* hc, int64_t* lc, uint32_t* succ,
                            uint32_t* lval) {
  GSTRIDE(q, nnz) {
    const int64_t p = V.csr_p[q];
    const int32_t r = rank[q];
    uint32_t sv = RC_NONE, lv = 0;
    if (r >= 0) {
      const int64_t i = rowof[q];
      const int64_t q0 = V.rowptr[i], q1 = V.rowptr[i + 1];
      int64_t t = q0 + r + 1;
      while (t < q1 && sorted[t] == RC_NONE) ++t;
      if (t < q1) sv = sorted[t];
      const bool two = rowcnt[i] == 2;
      lv = !two ? (uint32_t)i : (r == 0 ? ((uint32_t)i | RC_TWO) : (sorted[q0] | RC_TWO));
    }
    hc[p] = r > 0;
    lc[p] = r == 0;
    succ[p] = sv;
    lval[p] = lv;
  }
}

__device__ __forceinline__ int warp_excl(int v, int lane, int* total) {
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  *total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - v;
}

// Push the units flagged by the lanes of one warp onto the next frontier (one
// atomic per list per warp).
__device__ __forceinline__ void warp_push(bool pb, bool ps, uint32_t w, int lane, uint32_t* next_s, int64_t* nnext_s,
                                          uint32_t* next_b, int64_t* nnext_b) {
  unsigned mb = __ballot_sync(0xffffffffu, pb), ms = __ballot_sync(0xffffffffu, ps);
  unsigned long long bb = 0, bs = 0;
  if (lane == 0) {
    if (mb) bb = atomicAdd((unsigned long long*)nnext_b, (unsigned long long)__popc(mb));
    if (ms) bs = atomicAdd((unsigned long long*)nnext_s, (unsigned long long)__popc(ms));
  }
  bb = __shfl_sync(0xffffffffu, bb, 0);
  bs = __shfl_sync(0xffffffffu, bs, 0);
  const unsigned lt = (1u << lane) - 1u;
  if (pb) next_b[bb + __popc(mb & lt)] = w;
  if (ps) next_s[bs + __popc(ms & lt)] = w;
}

// Per unit, from the exclusive scans hc, lc of the per-non-zero flags: list
// start aptr[u] = hc[p0] + lc[p0] (p0, p1 = the unit's non-zero range),
// npred[u] = hc[p1] - hc[p0] (also the initial count), the two bases the fill
// needs, the long-list flag, and the initial frontier (units first in all
// their rows).
__global__ void k_chain_units(JPView V, int64_t Us, int64_t nnz, const int64_t* hc, const int64_t* lc, int64_t* aptr,
                              int32_t* npred, int32_t* cnt, int64_t* lbase, int64_t* hend, uint8_t* ubig,
                              uint32_t* front_s, int64_t* nfront_s, uint32_t* front_b, int64_t* nfront_b) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ub = blockIdx.x * (int64_t)blockDim.x; ub < Us; ub += stride) {  // warp-uniform
    const int64_t u = ub + threadIdx.x;
    bool ready = false, big = false;
    if (u < Us) {
      const int64_t f = V.ufirst[u];
      const int64_t p0 = V.colptr[f], p1 = V.colptr[f + V.ulen[u]];
      const int64_t h0 = hc[p0], l0 = lc[p0], h1 = hc[p1], l1 = lc[p1];
      const int64_t nh = h1 - h0;
      aptr[u] = h0 + l0;
      npred[u] = (int32_t)nh;
      cnt[u] = (int32_t)nh;
      lbase[u] = l0;
      hend[u] = h1;
      big = (h1 + l1) - (h0 + l0) > JP_BIG;
      ubig[u] = big;
      ready = nh == 0;
      if (u == Us - 1) aptr[Us] = hc[nnz] + lc[nnz];
    }
    warp_push(ready && big, ready && !big, (uint32_t)u, lane, front_s, nfront_s, front_b, nfront_b);
  }
}

// One thread per non-zero p of unit u: its (list entry, successor) goes to
// hc[p] + lbase[u] (= aptr[u] + the predecessor rows of u's earlier
// non-zeros) or, for a row u starts, to hend[u] + lc[p] (= aptr[u] + npred[u]
// + ...).  Bit 31 of a successor: that unit's own list is long (a CTA serves
// it).
__global__ void k_chain_fill(JPView V, int64_t nnz, const int64_t* hc, const int64_t* lc, const int64_t* lbase,
                             const int64_t* hend, const uint32_t* succ, const uint32_t* lval, const uint8_t* ubig,
                             uint32_t* lrow, uint32_t* lsucc) {
  GSTRIDE(p, nnz) {
    const bool pred = hc[p + 1] != hc[p], first = lc[p + 1] != lc[p];
    if (!pred && !first) continue;
    const int64_t u = V.unit_of_col[V.colof[p]];
    const int64_t pos = pred ? hc[p] + lbase[u] : hend[u] + lc[p];
    const uint32_t sv = succ[p];
    lrow[pos] = lval[p];
    lsucc[pos] = (sv == RC_NONE) ? RC_NONE : (sv | (ubig[sv] ? RC_BIG : 0u));
  }
}

// grid barrier for the cooperative JP launch (same scheme as the sweep's):
// one word, top bit flips once per barrier, bounded wait.
__device__ __forceinline__ bool jp_barrier(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned inc = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1)) : 1u;
    unsigned old, cur;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(inc) : "memory");
    ok = 1;
    const long long t0 = clock64();
    unsigned it = 0;
    while (true) {
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if ((cur ^ old) & 0x80000000u) break;
      if ((++it & 255u) == 0 && (*(volatile int*)err || clock64() - t0 > 4000000000LL)) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  return ok != 0;
}

struct JPRun {
  const uint32_t* lrow;   // per unit list: rows (RC_TWO entries: see k_row_links), predecessor rows first
  const uint32_t* lsucc;  // successor in that row (RC_NONE: last; RC_BIG flag)
  const int64_t* aptr;
  const int32_t* npred;
  const int64_t* rowptr;  // the rows' units in priority order (slow path)
  const uint32_t* sorted;
  unsigned long long* rmask;  // two words per row
  int32_t* cnt;
  int32_t* color;
  uint32_t* fs[2];
  uint32_t* fb[2];
  int64_t* fc;  // 3 x (small, big) frontier counters
  unsigned long long* done;
  unsigned* bar;
  int* err;
};

// colour c into the mask of row i
__device__ __forceinline__ void mask_add(unsigned long long* rmask, uint32_t i, int c) {
  if (c < 64) atomicOr(rmask + 2 * (int64_t)i, 1ull << c);
  else atomicOr(rmask + 2 * (int64_t)i + 1, 1ull << (c < RC_OVF ? c - 64 : 63));
}

// colour c into a 128-bit accumulator (same bits as mask_add)
__device__ __forceinline__ void mask_set(unsigned long long& m0, unsigned long long& m1, int c) {
  if (c < 64) m0 |= 1ull << c;
  else m1 |= 1ull << (c < RC_OVF ? c - 64 : 63);
}

// the mask a predecessor entry contributes: its row's mask, or for the second
// unit of a two-unit row the first unit's colour
__device__ __forceinline__ void entry_mask(const JPRun& R, uint32_t e, unsigned long long& m0, unsigned long long& m1) {
  if (e & RC_TWO) {
    mask_set(m0, m1, __ldcg(R.color + (e & ~RC_TWO)));
  } else {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(R.rmask) + e);
    m0 |= v.x;
    m1 |= v.y;
  }
}

// the smallest colour free in a 128-bit mask, or -1 when the slow path must
// decide (bit RC_OVF set, or colours 0..RC_OVF-1 all taken)
__device__ __forceinline__ int mask_pick(unsigned long long m0, unsigned long long m1) {
  if (m1 >> 63) return -1;
  if (~m0) return __ffsll((long long)~m0) - 1;
  const unsigned long long f = ~m1 & 0x7fffffffffffffffull;
  return f ? 64 + __ffsll((long long)f) - 1 : -1;
}

// OR of the masks of the rows lrow[a0, ah), strided by `step` from `start`
__device__ __forceinline__ void mask_or(const JPRun& R, int64_t a0, int64_t ah, int64_t start, int step,
                                        unsigned long long& m0, unsigned long long& m1) {
  for (int64_t qb = a0 + start; qb < ah; qb += 4 * (int64_t)step) {
    uint32_t rw[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) rw[t] = (qb + t * step < ah) ? R.lrow[qb + t * step] : RC_NONE;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (rw[t] != RC_NONE) entry_mask(R, rw[t], m0, m1);
  }
}

// slow path: colours in [base, base + 64) of the units before u in the row of
// predecessor entry i
__device__ unsigned long long prefix_mask(const JPRun& R, uint32_t i, uint32_t u, int base) {
  unsigned long long m = 0;
  if (i & RC_TWO) {
    const int c = __ldcg(R.color + (i & ~RC_TWO));
    return (c >= base && c < base + 64) ? 1ull << (c - base) : 0ull;
  }
  for (int64_t t = R.rowptr[i], t1 = R.rowptr[i + 1]; t < t1; ++t) {
    const uint32_t w = R.sorted[t];
    if (w == u) break;
    if (w == RC_NONE) continue;
    const int c = __ldcg(R.color + w);
    if (c >= base && c < base + 64) m |= 1ull << (c - base);
  }
  return m;
}

__device__ __forceinline__ unsigned long long prefix_or(const JPRun& R, uint32_t u, int64_t a0, int64_t ah,
                                                        int64_t start, int step, int base) {
  unsigned long long m = 0;
  for (int64_t q = a0 + start; q < ah; q += step) m |= prefix_mask(R, R.lrow[q], u, base);
  return m;
}

// Colour c into the rows of lrow[a0, a1) that have a successor and count the
// successors down; the loop is uniform over the `step` threads that run it (a
// warp or a CTA).  Four entries per thread at a time; the units released go
// to the next frontier with one reservation per list per warp.
__device__ __forceinline__ void release(const JPRun& R, int c, int64_t a0, int64_t a1, int64_t start, int step,
                                        int lane, uint32_t* next_s, int64_t* nnext_s, uint32_t* next_b,
                                        int64_t* nnext_b) {
  for (int64_t qb = a0; qb < a1; qb += 4 * (int64_t)step) {
    uint32_t sc[4], rw[4];
    bool rel[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t q = qb + start + (int64_t)t * step;
      sc[t] = (q < a1) ? R.lsucc[q] : RC_NONE;
      rw[t] = (q < a1) ? R.lrow[q] : 0u;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (sc[t] != RC_NONE && !(rw[t] & RC_TWO)) mask_add(R.rmask, rw[t], c);
#pragma unroll
    for (int t = 0; t < 4; ++t) rel[t] = sc[t] != RC_NONE && atomicSub(&R.cnt[sc[t] & ~RC_BIG], 1) == 1;
    int nb = 0, ns = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      nb += rel[t] && (sc[t] & RC_BIG);
      ns += rel[t] && !(sc[t] & RC_BIG);
    }
    int tb, ts;
    const int ob = warp_excl(nb, lane, &tb), os = warp_excl(ns, lane, &ts);
    unsigned long long bb = 0, bs = 0;
    if (lane == 0) {
      if (tb) bb = atomicAdd((unsigned long long*)nnext_b, (unsigned long long)tb);
      if (ts) bs = atomicAdd((unsigned long long*)nnext_s, (unsigned long long)ts);
    }
    bb = __shfl_sync(0xffffffffu, bb, 0) + ob;
    bs = __shfl_sync(0xffffffffu, bs, 0) + os;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (rel[t]) {
        if (sc[t] & RC_BIG) next_b[bb++] = sc[t] & ~RC_BIG;
        else next_s[bs++] = sc[t];
      }
  }
}

// The colour of unit u from its predecessor rows lrow[a0, ah), by one warp.
__device__ __forceinline__ int warp_colour(const JPRun& R, uint32_t u, int64_t a0, int64_t ah, int lane) {
  unsigned long long m0 = 0, m1 = 0;
  mask_or(R, a0, ah, lane, 32, m0, m1);
  for (int o = 16; o > 0; o >>= 1) {
    m0 |= __shfl_xor_sync(0xffffffffu, m0, o);
    m1 |= __shfl_xor_sync(0xffffffffu, m1, o);
  }
  int c = mask_pick(m0, m1);
  for (int base = 0; c < 0; base += 64) {  // uniform over the warp
    unsigned long long m = prefix_or(R, u, a0, ah, lane, 32, base);
    for (int o = 16; o > 0; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
    if (~m) c = base + __ffsll((long long)~m) - 1;
  }
  return c;
}

// The same by the whole CTA (sm: two shared words).
__device__ __forceinline__ int cta_colour(const JPRun& R, uint32_t u, int64_t a0, int64_t ah, int lane,
                                          unsigned long long* sm) {
  if (threadIdx.x == 0) {
    sm[0] = 0;
    sm[1] = 0;
  }
  __syncthreads();
  unsigned long long m0 = 0, m1 = 0;
  mask_or(R, a0, ah, threadIdx.x, blockDim.x, m0, m1);
  for (int o = 16; o > 0; o >>= 1) {
    m0 |= __shfl_xor_sync(0xffffffffu, m0, o);
    m1 |= __shfl_xor_sync(0xffffffffu, m1, o);
  }
  if (lane == 0) {
    if (m0) atomicOr(sm, m0);
    if (m1) atomicOr(sm + 1, m1);
  }
  __syncthreads();
  int c = mask_pick(sm[0], sm[1]);
  __syncthreads();
  for (int base = 0; c < 0; base += 64) {  // uniform over the CTA
    if (threadIdx.x == 0) sm[0] = 0;
    __syncthreads();
    unsigned long long m = prefix_or(R, u, a0, ah, threadIdx.x, blockDim.x, base);
    for (int o = 16; o > 0; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
    if (lane == 0 && m) atomicOr(sm, m);
    __syncthreads();
    const unsigned long long all = sm[0];
    if (~all) c = base + __ffsll((long long)~all) - 1;
    __syncthreads();
  }
  return c;
}

constexpr int64_t JP_TINY = 64;    // list length served by 8 lanes (8 entries a lane)
constexpr int64_t JP_SLICE = 512;  // entries of a long list one CTA releases

// Colour and release 32 / TG units whose lists hold at most 8 * TG entries,
// one group of TG lanes per unit (u = RC_NONE: an idle group).  Control flow
// is uniform over the warp: every lane loads its (at most 8) entries at once,
// the masks are OR-reduced inside the group, and the released units are
// reserved on the next frontier once per warp.
template <int TG>
__device__ __forceinline__ void jp_tiny(const JPRun& R, uint32_t u, int lane, uint32_t* next_s, int64_t* nnext_s,
                                        uint32_t* next_b, int64_t* nnext_b) {
  const int sub = lane & (TG - 1);
  int64_t a0 = 0, ah = 0, a1 = 0;
  if (u != RC_NONE) {
    a0 = R.aptr[u];
    ah = a0 + R.npred[u];
    a1 = R.aptr[u + 1];
  }
  uint32_t rw[8], sc[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t q = a0 + sub + t * TG;
    rw[t] = q < a1 ? R.lrow[q] : 0u;
    sc[t] = q < a1 ? R.lsucc[q] : RC_NONE;
  }
  unsigned long long m0 = 0, m1 = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (a0 + sub + t * TG < ah) entry_mask(R, rw[t], m0, m1);
  for (int o = TG / 2; o > 0; o >>= 1) {
    m0 |= __shfl_xor_sync(0xffffffffu, m0, o);
    m1 |= __shfl_xor_sync(0xffffffffu, m1, o);
  }
  int chosen = (u != RC_NONE) ? mask_pick(m0, m1) : 0;
  if (__any_sync(0xffffffffu, chosen < 0)) {
    const bool slow = chosen < 0;  // the same in all lanes of a group
    for (int base = 0;; base += 64) {
      unsigned long long m = 0;
      if (slow)
        for (int t = 0; t < 8; ++t)
          if (a0 + sub + t * TG < ah) m |= prefix_mask(R, rw[t], u, base);
      for (int o = TG / 2; o > 0; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
      if (chosen < 0 && ~m) chosen = base + __ffsll((long long)~m) - 1;
      if (__all_sync(0xffffffffu, chosen >= 0)) break;
    }
  }
  if (u != RC_NONE && sub == 0) R.color[u] = chosen;
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (sc[t] != RC_NONE && !(rw[t] & RC_TWO)) mask_add(R.rmask, rw[t], chosen);
  bool rel[8];
  int nb = 0, ns = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    rel[t] = sc[t] != RC_NONE && atomicSub(&R.cnt[sc[t] & ~RC_BIG], 1) == 1;
    nb += rel[t] && (sc[t] & RC_BIG);
    ns += rel[t] && !(sc[t] & RC_BIG);
  }
  int tb, ts;
  const int ob = warp_excl(nb, lane, &tb), os = warp_excl(ns, lane, &ts);
  unsigned long long bb = 0, bs = 0;
  if (lane == 0) {
    if (tb) bb = atomicAdd((unsigned long long*)nnext_b, (unsigned long long)tb);
    if (ts) bs = atomicAdd((unsigned long long*)nnext_s, (unsigned long long)ts);
  }
  bb = __shfl_sync(0xffffffffu, bb, 0) + ob;
  bs = __shfl_sync(0xffffffffu, bs, 0) + os;
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (rel[t]) {
      if (sc[t] & RC_BIG) next_b[bb++] = sc[t] & ~RC_BIG;
      else next_s[bs++] = sc[t];
    }
}

// Rounds [r0, r0 + nr) of the data-flow colouring; with nr > 1 the launch must
// be cooperative (a grid barrier separates the rounds).
__global__ void __launch_bounds__(256, 4) k_jp(JPRun R, int64_t r0, int64_t nr) {
  __shared__ unsigned long long smask[2];
  __shared__ uint32_t s_u[256];
  __shared__ int s_off[257];
  __shared__ int s_wsum[8];
  __shared__ long long s_fc[2];
  const int lane = threadIdx.x & 31;
  for (int64_t r = r0; r < r0 + nr; ++r) {
    const int in = (int)(r % 3), out = (int)((r + 1) % 3), z = (int)((r + 2) % 3);
    if (threadIdx.x == 0) {  // one read of the frontier sizes per CTA
      s_fc[0] = __ldcg(R.fc + 2 * in);
      s_fc[1] = __ldcg(R.fc + 2 * in + 1);
    }
    __syncthreads();
    const int64_t ns = s_fc[0], nb = s_fc[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // slot z is nobody's input this round; clearing it even when the
      // frontier is empty keeps rounds launched past the end (one launch per
      // round) from reading a stale count three rounds later
      R.fc[2 * z] = 0;
      R.fc[2 * z + 1] = 0;
      if (ns + nb) atomicAdd(R.done, (unsigned long long)(ns + nb));
    }
    if (ns + nb == 0) return;  // every CTA reads the same counts: all stop together
    const uint32_t* front_s = R.fs[r & 1];
    const uint32_t* front_b = R.fb[r & 1];
    uint32_t* next_s = R.fs[(r + 1) & 1];
    uint32_t* next_b = R.fb[(r + 1) & 1];
    int64_t* nnext_s = R.fc + 2 * out;
    int64_t* nnext_b = R.fc + 2 * out + 1;
    if (nb > 0 && nb <= (int64_t)blockDim.x && nb < (int64_t)gridDim.x) {  // uniform
      // few long lists (a chain of hubs): each list is cut into slices of
      // JP_SLICE entries spread over the CTAs; the CTA of a slice finds the
      // unit's colour from its predecessor rows (few for a hub) and releases
      // the slice.  s_off = exclusive scan of the slice counts.
      int nsl = 0;
      if (threadIdx.x < nb) {
        const uint32_t u = __ldcg(front_b + threadIdx.x);
        const int64_t a0 = R.aptr[u], a1 = R.aptr[u + 1];
        nsl = (int)max((int64_t)1, (a1 - a0 + JP_SLICE - 1) / JP_SLICE);
        s_u[threadIdx.x] = u;
      }
      int wt;
      const int wex = warp_excl(nsl, lane, &wt);
      if (lane == 0) s_wsum[threadIdx.x >> 5] = wt;
      __syncthreads();
      int wbase = 0;
      for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += s_wsum[w];
      s_off[threadIdx.x] = wbase + wex;
      if (threadIdx.x == blockDim.x - 1) s_off[blockDim.x] = wbase + wex + nsl;
      __syncthreads();
      const int64_t S = s_off[nb];
      int j = 0;
      for (int64_t g = blockIdx.x; g < S; g += gridDim.x) {
        while (s_off[j + 1] <= g) ++j;  // uniform; g only grows
        const uint32_t u = s_u[j];
        const int64_t sl = g - s_off[j];
        const int64_t a0 = R.aptr[u], ah = a0 + R.npred[u], a1 = R.aptr[u + 1];
        const int chosen = cta_colour(R, u, a0, ah, lane, smask);
        if (sl == 0 && threadIdx.x == 0) R.color[u] = chosen;
        const int64_t b0 = a0 + sl * JP_SLICE, b1 = min(a1, b0 + JP_SLICE);
        release(R, chosen, b0, b1, threadIdx.x, blockDim.x, lane, next_s, nnext_s, next_b, nnext_b);
      }
      __syncthreads();  // s_u / s_off are rewritten next round
    } else {
      // long lists: one CTA each
      for (int64_t t = blockIdx.x; t < nb; t += gridDim.x) {
        const uint32_t u = __ldcg(front_b + t);
        const int64_t a0 = R.aptr[u], ah = a0 + R.npred[u], a1 = R.aptr[u + 1];
        const int chosen = cta_colour(R, u, a0, ah, lane, smask);
        if (threadIdx.x == 0) R.color[u] = chosen;
        release(R, chosen, a0, a1, threadIdx.x, blockDim.x, lane, next_s, nnext_s, next_b, nnext_b);
      }
    }
    // the rest.  A frontier larger than the warps: 16 (or 4) units per warp,
    // 2 (or 8) lanes each when their lists are short enough, else one after
    // the other with the whole warp.  A smaller one: one unit per warp.
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int per = ns > 4 * nwarps ? 16 : (ns > nwarps ? 4 : 1);
    for (int64_t tb = warp * per; tb < ns; tb += nwarps * per) {  // warp-uniform
      uint32_t uu = RC_NONE;
      int64_t len = 0;
      if (lane < per && tb + lane < ns) {
        uu = __ldcg(front_s + tb + lane);
        len = R.aptr[uu + 1] - R.aptr[uu];
      }
      if (per == 16 && __all_sync(0xffffffffu, len <= 16)) {
        jp_tiny<2>(R, __shfl_sync(0xffffffffu, uu, lane / 2), lane, next_s, nnext_s, next_b, nnext_b);
        continue;
      }
      for (int qd = 0; qd < per; qd += 4) {  // uniform
        const int src = qd + (lane & 3);
        const uint32_t uq = __shfl_sync(0xffffffffu, uu, src);  // lanes 0..3: this quad's units
        const int64_t lq = __shfl_sync(0xffffffffu, len, src);
        if (per > 1 && __all_sync(0xffffffffu, lane >= 4 || lq <= JP_TINY)) {
          jp_tiny<8>(R, __shfl_sync(0xffffffffu, uq, lane / 8), lane, next_s, nnext_s, next_b, nnext_b);
          continue;
        }
        for (int j = 0; j < (per > 1 ? 4 : 1); ++j) {
          const uint32_t u = __shfl_sync(0xffffffffu, uq, j);
          if (u == RC_NONE) break;  // uniform
          const int64_t a0 = R.aptr[u], ah = a0 + R.npred[u], a1 = R.aptr[u + 1];
          const int chosen = warp_colour(R, u, a0, ah, lane);
          if (lane == 0) R.color[u] = chosen;
          release(R, chosen, a0, a1, lane, 32, lane, next_s, nnext_s, next_b, nnext_b);
        }
      }
    }
    if (nr > 1 && !jp_barrier(R.bar, R.err)) return;
  }
}

// Slack units, after every structural unit: the smallest colour not held by a
// structural unit of the slack's row.
__global__ void k_slack_color(JPView V, int64_t Msl, int32_t* color) {
  GSTRIDE(t, Msl) {
    const int64_t i = V.slack_row[t];
    int base = 0, chosen = -1;
    while (chosen < 0) {
      unsigned long long m = 0;
      for (int64_t q = V.rowptr[i]; q < V.rowptr[i + 1]; ++q) {
        int64_t w = V.unit_of_col[V.colof[V.csr_p[q]]];
        if (w < 0) continue;
        int cw = color[w];
        if (cw >= base && cw < base + 64) m |= 1ull << (cw - base);
      }
      if (~m) chosen = base + __ffsll((long long)~m) - 1;
      base += 64;
    }
    color[V.Us + t] = chosen;
  }
}

__global__ void k_slack_units(const int64_t* has_scan, const int64_t* has, int64_t M, int64_t Us,
                              int64_t* slack_unit, int64_t* slack_row) {
  GSTRIDE(i, M) {
    if (has[i]) {
      int64_t s = has_scan[i];
      slack_unit[i] = Us + s;
      slack_row[s] = i;
    } else {
      slack_unit[i] = -1;
    }
  }
}

__global__ void k_max_i32(const int32_t* a, int64_t n, int* out) {
  int m = -1;
  GSTRIDE(i, n) m = max(m, a[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// sort keys for structural units: colour * 4 + class
__global__ void k_struct_keys(const int32_t* color, const int32_t* ulen, const int64_t* unnz, int64_t Us,
                              uint32_t* keys, uint32_t* vals, int64_t* cnt, int64_t nbins) {
  extern __shared__ int sh_hist[];
  const bool use_sh = nbins <= HIST_SMEM_BINS;
  hist_init(sh_hist, nbins, use_sh);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ub = blockIdx.x * (int64_t)blockDim.x; ub < Us; ub += stride) {
    const int64_t u = ub + threadIdx.x;
    const bool ok = u < Us;
    uint32_t key = 0;
    if (ok) {
      int cls;
      if (ulen[u] > 1) cls = UC_BLOCK;
      else if (unnz[u] > T_HUGE) cls = UC_HUGE;
      else if (unnz[u] > T_LARGE) cls = UC_LARGE;
      else if (unnz[u] > T_MED) cls = UC_MED;
      else if (unnz[u] > 16) cls = UC_S32;
      else if (unnz[u] > 8) cls = UC_S16;
      else if (unnz[u] > 4) cls = UC_S8;
      else if (unnz[u] > 2) cls = UC_S4;
      else cls = UC_S2;
      key = (uint32_t)color[u] * UC_COUNT + cls;
      keys[u] = key;
      vals[u] = (uint32_t)u;
    }
    hist_add(cnt, sh_hist, use_sh, key, ok);
  }
  hist_flush(cnt, sh_hist, nbins, use_sh);
}

// key = internal column of the row's highest-priority free column (0 if none)
__global__ void k_slack_owner_keys(JPView V, int64_t Msl, const uint32_t* col_of_orig, uint32_t* keys, uint32_t* vals) {
  GSTRIDE(t, Msl) {
    int64_t i = V.slack_row[t];
    int64_t best = -1, bcol = 0;
    for (int64_t q = V.rowptr[i]; q < V.rowptr[i + 1]; ++q) {
      int64_t col = V.colof[V.csr_p[q]];
      int64_t u = V.unit_of_col[col];
      if (u < 0) continue;
      if (best < 0 || higher(V, u, best)) {
        best = u;
        bcol = col;
      }
    }
    keys[t] = best >= 0 ? col_of_orig[bcol] : 0u;
    vals[t] = (uint32_t)i;
  }
}

__global__ void k_slack_color_keys(const uint32_t* rows, int64_t Msl, const int64_t* slack_unit, const int32_t* color,
                                   uint32_t* keys, int64_t* cnt, int64_t nbins) {
  extern __shared__ int sh_hist[];
  const bool use_sh = nbins <= HIST_SMEM_BINS;
  hist_init(sh_hist, nbins, use_sh);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t tb = blockIdx.x * (int64_t)blockDim.x; tb < Msl; tb += stride) {
    const int64_t t = tb + threadIdx.x;
    const bool ok = t < Msl;
    uint32_t c = ok ? (uint32_t)color[slack_unit[rows[t]]] : 0u;
    if (ok) keys[t] = c;
    hist_add(cnt, sh_hist, use_sh, c, ok);
  }
  hist_flush(cnt, sh_hist, nbins, use_sh);
}

__global__ void k_pos_len(const uint32_t* unit_of_pos, const int32_t* ulen, int64_t Us, int64_t* len) {
  GSTRIDE(p, Us) len[p] = ulen[unit_of_pos[p]];
}

__global__ void k_col_maps_free(const uint32_t* unit_of_pos, const int64_t* ufirst, const int32_t* ulen,
                                const int64_t* cstart, int64_t Us, uint32_t* col_of_orig,
                                uint32_t* orig_of_col) {
  GSTRIDE(p, Us) {
    int64_t u = unit_of_pos[p];
    int64_t f = ufirst[u];
    for (int q = 0; q < ulen[u]; ++q) {
      col_of_orig[f + q] = (uint32_t)(cstart[p] + q);
      orig_of_col[cstart[p] + q] = (uint32_t)(f + q);
    }
  }
}

__global__ void k_col_maps_fixed(const int64_t* fixed_flag, const int64_t* fixed_scan, int64_t Ns,
                                 int64_t Nfree, uint32_t* col_of_orig, uint32_t* orig_of_col) {
  GSTRIDE(j, Ns) {
    if (fixed_flag[j]) {
      int64_t jj = Nfree + fixed_scan[j];
      col_of_orig[j] = (uint32_t)jj;
      orig_of_col[jj] = (uint32_t)j;
    }
  }
}

__global__ void k_row_maps(const uint32_t* slack_rows_sorted, int64_t Msl, const int64_t* has,
                           const int64_t* has_scan, int64_t M, uint32_t* row_of_orig, uint32_t* orig_of_row,
                           uint32_t* slack_orig) {
  GSTRIDE(t, Msl) {
    uint32_t i = slack_rows_sorted[t];
    row_of_orig[i] = (uint32_t)t;
    orig_of_row[t] = i;
    slack_orig[t] = (uint32_t)has_scan[i];
  }
  GSTRIDE(i, M) {
    if (!has[i]) {
      int64_t t = Msl + (i - has_scan[i]);
      row_of_orig[i] = (uint32_t)t;
      orig_of_row[t] = (uint32_t)i;
    }
  }
}

__global__ void k_int_col_counts(const uint32_t* orig_of_col, const int64_t* colptr, int64_t N, int64_t* cnt) {
  GSTRIDE(j, N) {
    int64_t o = orig_of_col[j];
    cnt[j] = colptr[o + 1] - colptr[o];
  }
}

// the entries of every internal column at its place, in the original
// column's order: key the internal row, ord the original position.  One
// thread per entry (colof: the original column of every entry) where columns
// are long on average; else one thread per column, a column of more than 32
// entries taken by its whole warp.
__global__ void k_icsc_gather(const uint32_t* colof, const uint32_t* col_of_orig, const int64_t* ocolptr,
                              const int32_t* orow, const uint32_t* row_of_orig, const int64_t* icolptr, int64_t nnz,
                              uint32_t* key, uint32_t* ord) {
  GSTRIDE(p, nnz) {
    const uint32_t o = colof[p];
    const int64_t q = icolptr[col_of_orig[o]] + (p - ocolptr[o]);
    key[q] = row_of_orig[orow[p]];
    ord[q] = (uint32_t)p;
  }
}
__global__ void k_icsc_gather_cols(const uint32_t* orig_of_col, const int64_t* ocolptr, const int32_t* orow,
                                   const uint32_t* row_of_orig, const int64_t* icolptr, int64_t N, uint32_t* key,
                                   uint32_t* ord) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = base + threadIdx.x;
    int64_t p0 = 0, p1 = 0, q0 = 0;
    if (j < N) {
      const int64_t o = orig_of_col[j];
      p0 = ocolptr[o];
      p1 = ocolptr[o + 1];
      q0 = icolptr[j];
    }
    const bool longc = p1 - p0 > 32;
    if (!longc)
      for (int64_t p = p0; p < p1; ++p) {
        key[q0 + (p - p0)] = row_of_orig[orow[p]];
        ord[q0 + (p - p0)] = (uint32_t)p;
      }
    unsigned mb = __ballot_sync(0xffffffffu, longc);
    while (mb) {
      const int l = __ffs(mb) - 1;
      mb &= mb - 1;
      const int64_t a = __shfl_sync(0xffffffffu, p0, l), e = __shfl_sync(0xffffffffu, p1, l);
      const int64_t q = __shfl_sync(0xffffffffu, q0, l);
      for (int64_t p = a + lane; p < e; p += 32) {
        key[q + (p - a)] = row_of_orig[orow[p]];
        ord[q + (p - a)] = (uint32_t)p;
      }
    }
  }
}

__global__ void k_icsc_fill(const uint32_t* ord, const uint32_t* key, const float* oval, int64_t nnz, bool keep_val,
                            uint32_t* irow, float* ival) {
  GSTRIDE(t, nnz) {
    const float v = oval ? oval[ord[t]] : 1.f;
    const uint32_t r = key[t];
    if (keep_val) {
      irow[t] = r;
      ival[t] = v;
    } else {
      irow[t] = r | (v < 0.f ? NEG_BIT : 0u);
    }
  }
}

// ||a_j||^2 per internal column (warp per column)
__global__ void k_csq(const int64_t* colptr, const float* val, int64_t N, float* csq) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < N; j += nwarps) {
    float sq = 0.f;
    for (int64_t p = colptr[j] + lane; p < colptr[j + 1]; p += 32) sq += val[p] * val[p];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) csq[j] = sq;
  }
}

__global__ void k_int_row_counts(const uint32_t* orig_of_row, const int64_t* orowptr, int64_t M, int64_t* cnt) {
  GSTRIDE(i, M) {
    int64_t o = orig_of_row[i];
    cnt[i] = orowptr[o + 1] - orowptr[o];
  }
}

__global__ void k_int_csr_fill(const uint32_t* orig_of_row, const int64_t* orowptr, const uint32_t* csr_p,
                               const uint32_t* colof, const float* oval, const uint32_t* col_of_orig,
                               const int64_t* irowptr, int64_t M, bool keep_val, uint32_t* icol, float* ival) {
  GSTRIDE(i, M) {
    int64_t o = orig_of_row[i];
    int64_t q0 = irowptr[i];
    for (int64_t q = orowptr[o]; q < orowptr[o + 1]; ++q) {
      uint32_t p = csr_p[q];
      float v = oval ? oval[p] : 1.f;
      uint32_t jc = col_of_orig[colof[p]];
      if (keep_val) {
        icol[q0] = jc;
        ival[q0] = v;
      } else {
        icol[q0] = jc | (v < 0.f ? NEG_BIT : 0u);
      }
      ++q0;
    }
  }
}

__global__ void k_col_vectors(const uint32_t* orig_of_col, const float* oc, const float* olo, const float* ohi,
                              int64_t N, bool per_col_bounds, float* c, float* lo, float* hi) {
  GSTRIDE(j, N) {
    int64_t o = orig_of_col[j];
    c[j] = oc[o];
    if (per_col_bounds) {
      lo[j] = olo[o];
      hi[j] = ohi[o];
    }
  }
}

__global__ void k_row_vectors(const uint32_t* orig_of_row, const float* ob, const uint8_t* rk, int64_t M,
                              float* b, int8_t* sig) {
  GSTRIDE(i, M) {
    int64_t o = orig_of_row[i];
    b[i] = ob[o];
    uint8_t k = rk[o];
    sig[i] = (k == THETIS_ROW_GE) ? -1 : (k == THETIS_ROW_LE ? 1 : 0);
  }
}

__global__ void k_unit_color_copy(const int32_t* color, int64_t U, int32_t* out) {
  GSTRIDE(u, U) out[u] = color[u];
}

__global__ void k_max_sq_free(const int64_t* colptr, const float* csq, int64_t Nfree, double* out) {
  double m = 0.0;
  GSTRIDE(j, Nfree) {
    double v = csq ? (double)csq[j] : (double)(colptr[j + 1] - colptr[j]);
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_max_unit_nnz(const int64_t* unnz, int64_t U, unsigned long long* out) {
  unsigned long long m = 0;
  GSTRIDE(u, U) m = max(m, (unsigned long long)unnz[u]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ELL copy of the small classes: column j of small segment t (first column
// c0[t], n[t] columns, width w[t], first slot e0[t]) writes its row slots.
__global__ void k_ell_fill(const int64_t* colptr, const uint32_t* rowidx, const float* val, const int64_t* c0,
                           const int64_t* n, const int64_t* e0, const int32_t* w, int64_t nseg, int64_t Nfree,
                           uint32_t* ell, float* ellv) {
  GSTRIDE(j, Nfree) {
    int64_t lo = 0, hi = nseg;  // last segment with c0 <= j
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (c0[mid] <= j) lo = mid;
      else hi = mid;
    }
    if (j < c0[lo] || j >= c0[lo] + n[lo]) continue;
    const int64_t p = j - c0[lo];
    const int W = w[lo];
    const int64_t base = e0[lo] + (p >> 5) * 32 * W + (p & 31);
    const int64_t q0 = colptr[j], q1 = colptr[j + 1];
    for (int64_t q = q0; q < q1 && q - q0 < W; ++q) {
      ell[base + (q - q0) * 32] = rowidx[q];
      if (ellv) ellv[base + (q - q0) * 32] = val[q];
    }
  }
}

std::unique_ptr<Problem> build_problem(RawLP& raw, int kind, uint64_t seed, cudaStream_t s, Arena& tmp) {
  auto Pp = std::make_unique<Problem>(s);
  Problem& P = *Pp;
  const int64_t M = raw.M, Ns = raw.Ns, nnz = raw.nnz;
  TH_CHECK(Ns >= 1 && M >= 0 && Ns < (int64_t(1) << 31) - 1 && M < (int64_t(1) << 31) - 1 &&
               nnz < (int64_t(1) << 32) - 1,
           THETIS_E_INVALID, "problem too large or empty");
  P.kind = kind;
  P.M = M;
  P.Ns = Ns;
  P.nnz = nnz;
  P.k = raw.block_k;

  // -- validation --------------------------------------------------------
  int* err = tmp.alloc<int>(2);
  TH_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
  k_validate<<<grid_for(std::max(std::max(Ns, M), nnz), 256), 256, 0, s>>>(
      raw.colptr, raw.rowidx, raw.val, raw.lo, raw.hi, raw.row_kind, Ns, M, nnz, err, err + 1);
  TH_LAUNCHED();
  int64_t* d_tmp64 = tmp.alloc<int64_t>(2);
  TH_CUDA(cudaMemcpyAsync(d_tmp64, raw.colptr, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  TH_CUDA(cudaMemcpyAsync(d_tmp64 + 1, raw.colptr + Ns, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int64_t ends[2];
  int flags[2];
  TH_CUDA(cudaMemcpyAsync(ends, d_tmp64, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(flags, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CHECK(ends[0] == 0 && ends[1] == nnz, THETIS_E_INVALID, "csc_ptr must start at 0 and end at nnz");
  TH_CHECK(flags[0] != 1, THETIS_E_INVALID, "csc_ptr is not non-decreasing");
  TH_CHECK(flags[0] != 2, THETIS_E_INVALID, "lo > hi (or NaN) in a bound");
  TH_CHECK(flags[0] != 3, THETIS_E_INVALID, "row index out of range");
  TH_CHECK(flags[0] != 4, THETIS_E_INVALID, "non-finite coefficient");
  TH_CHECK(flags[0] != 5, THETIS_E_INVALID, "invalid row kind");
  P.has_val = (raw.val != nullptr) && flags[1];
  P.bounds_uniform = raw.bounds_uniform;
  P.lo_u = raw.lo_u;
  P.hi_u = raw.hi_u;
  P.slack_sign_uniform = raw.slack_sign_uniform;

  // -- units ---------------------------------------------------------------
  int32_t* blk = nullptr;
  if (raw.n_blocks > 0) {
    TH_CHECK(raw.block_k >= 2 && raw.block_k <= 32, THETIS_E_INVALID, "block_k must be in [2, 32]");
    blk = tmp.alloc<int32_t>(Ns);
    TH_CUDA(cudaMemsetAsync(blk, 0xff, Ns * sizeof(int32_t), s));
    k_block_claim<<<grid_for(raw.n_blocks, 256), 256, 0, s>>>(raw.block_first, raw.n_blocks, raw.block_k, Ns, blk, err);
    TH_LAUNCHED();
    int f = read_flag(err, s);
    TH_CHECK(f != 6, THETIS_E_INVALID, "simplex block out of range");
    TH_CHECK(f != 7, THETIS_E_INVALID, "simplex blocks overlap");
  } else {
    P.k = 1;
  }
  int64_t* start_flag = tmp.alloc<int64_t>(Ns + 1);
  int64_t* fixed_flag = tmp.alloc<int64_t>(Ns + 1);
  k_unit_flags<<<grid_for(Ns, 256), 256, 0, s>>>(blk, raw.block_first, raw.block_k, raw.lo, raw.hi, Ns,
                                                 start_flag, fixed_flag);
  TH_LAUNCHED();
  int64_t* start_scan = tmp.alloc<int64_t>(Ns + 1);
  int64_t* fixed_scan = tmp.alloc<int64_t>(Ns + 1);
  exclusive_scan_i64(start_flag, start_scan, Ns, tmp, s);
  exclusive_scan_i64(fixed_flag, fixed_scan, Ns, tmp, s);
  int64_t* has = tmp.alloc<int64_t>(M + 1);
  int64_t* has_scan = tmp.alloc<int64_t>(M + 1);
  if (M > 0) {
    k_slack_flags<<<grid_for(M, 256), 256, 0, s>>>(raw.row_kind, M, has);
    TH_LAUNCHED();
  }
  exclusive_scan_i64(has, has_scan, M, tmp, s);
  int64_t cnts[3];
  TH_CUDA(cudaMemcpyAsync(&cnts[0], start_scan + Ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(&cnts[1], fixed_scan + Ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(&cnts[2], has_scan + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  const int64_t Us = cnts[0], Nfix = cnts[1], Msl = cnts[2];
  const int64_t U = Us + Msl;
  P.Us = Us;
  P.Nfix = Nfix;
  P.Nfree = Ns - Nfix;
  P.Msl = Msl;
  P.U = U;
  P.free_coords = P.Nfree + Msl;
  TH_CHECK(U < (int64_t(1) << 32) - 1, THETIS_E_INVALID, "too many coordinate units");

  int64_t* unit_of_col = tmp.alloc<int64_t>(Ns);
  int64_t* ufirst = tmp.alloc<int64_t>(Us + 1);
  int32_t* ulen = tmp.alloc<int32_t>(Us + 1);
  k_unit_ids<<<grid_for(Ns, 256), 256, 0, s>>>(blk, raw.block_first, raw.block_k, Ns, start_scan, fixed_flag,
                                               unit_of_col, ufirst, ulen);
  TH_LAUNCHED();
  int64_t* slack_unit = tmp.alloc<int64_t>(M + 1);
  int64_t* slack_row = tmp.alloc<int64_t>(Msl + 1);
  if (M > 0) {
    k_slack_units<<<grid_for(M, 256), 256, 0, s>>>(has_scan, has, M, Us, slack_unit, slack_row);
    TH_LAUNCHED();
  }

  // -- CSR transpose (stable by row, columns ascending inside a row) -------
  // (the entry positions p grouped by row, ascending inside a row; rkeys: the
  // row of every CSR position, colof: the column of every entry)
  uint32_t* csr_p = tmp.alloc<uint32_t>(nnz);
  int64_t* orowptr = tmp.alloc<int64_t>(M + 1);
  group_by_key(reinterpret_cast<const uint32_t*>(raw.rowidx), nullptr, nnz, M, csr_p, orowptr, tmp, s);
  uint32_t* rkeys = tmp.alloc<uint32_t>(nnz);
  uint32_t* colof = tmp.alloc<uint32_t>(nnz);
  if (nnz > 0) {
    k_seg_ids<<<grid_for(M, 256), 256, 0, s>>>(orowptr, M, rkeys);
    TH_LAUNCHED();
    k_seg_ids<<<grid_for(Ns, 256), 256, 0, s>>>(raw.colptr, Ns, colof);
    TH_LAUNCHED();
  }
  if (M > 0) {
    k_csr_dupcheck<<<grid_for(M, 256), 256, 0, s>>>(orowptr, csr_p, colof, M, err);
    TH_LAUNCHED();
    TH_CHECK(read_flag(err, s) != 8, THETIS_E_INVALID, "repeated row index inside a column");
  }

  // -- colouring (Jones-Plassmann, first fit, fixed total order) -----------
  int64_t* unnz = tmp.alloc<int64_t>(U + 1);
  uint64_t* uh = tmp.alloc<uint64_t>(U + 1);
  k_unit_keys<<<grid_for(U, 256), 256, 0, s>>>(raw.colptr, ufirst, ulen, Us, U, seed, raw.prio_col, raw.prio_row,
                                               slack_row, unnz, uh);
  TH_LAUNCHED();
  int32_t* color = tmp.alloc<int32_t>(U + 1);
  TH_CUDA(cudaMemsetAsync(color, 0xff, (U + 1) * sizeof(int32_t), s));
  JPView V{raw.colptr, raw.rowidx, orowptr, csr_p, colof, unit_of_col, slack_unit, ufirst, ulen, unnz, uh, Us, slack_row};
  TH_CHECK(Us < (int64_t)RC_BIG - 1, THETIS_E_INVALID, "too many coordinate units (unit ids are 31-bit)");
  if (Us > 0) {
    int dev = 0, sms = 0, coop = 0, per = 0;
    TH_CUDA(cudaGetDevice(&dev));
    TH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TH_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    TH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_jp, 256, 0));
    // row ranks, successors and per-unit (row, successor) lists; a list holds
    // at most one entry per non-zero
    uint32_t* rowunit = tmp.alloc<uint32_t>(nnz + 1);
    ulonglong2* ukey = tmp.alloc<ulonglong2>(Us);
    int* repeat = nullptr;  // set when a block has two columns in one row
    int32_t* rank = tmp.alloc<int32_t>(nnz + 1);
    uint32_t* sorted = tmp.alloc<uint32_t>(nnz + 1);
    uint32_t* succ = tmp.alloc<uint32_t>(nnz + 1);
    uint32_t* lval = tmp.alloc<uint32_t>(nnz + 1);
    int32_t* rowcnt = tmp.alloc<int32_t>(M + 1);
    int64_t* hc = tmp.alloc<int64_t>(nnz + 1);
    int64_t* lc = tmp.alloc<int64_t>(nnz + 1);
    int64_t* aptr = tmp.alloc<int64_t>(Us + 1);
    int32_t* npred = tmp.alloc<int32_t>(Us + 1);
    int64_t* lbase = tmp.alloc<int64_t>(Us);
    int64_t* hend = tmp.alloc<int64_t>(Us);
    uint8_t* ubig = tmp.alloc<uint8_t>(Us);
    uint32_t* lrow = tmp.alloc<uint32_t>(nnz + 1);
    uint32_t* lsucc = tmp.alloc<uint32_t>(nnz + 1);
    unsigned long long* rmask = tmp.alloc<unsigned long long>(2 * (M + 1));
    TH_CUDA(cudaMemsetAsync(sorted, 0xff, (nnz + 1) * sizeof(uint32_t), s));
    TH_CUDA(cudaMemsetAsync(rmask, 0, 2 * (M + 1) * sizeof(unsigned long long), s));
    TH_CUDA(cudaMemsetAsync(rowcnt, 0, (M + 1) * sizeof(int32_t), s));
    repeat = tmp.alloc<int>(1);
    TH_CUDA(cudaMemsetAsync(repeat, 0, sizeof(int), s));
    if (nnz > 0) {
      k_row_units<<<grid_for(nnz, 256), 256, 0, s>>>(V, nnz, rowunit);
      TH_LAUNCHED();
    }
    k_unit_prio<<<grid_for(Us, 256), 256, 0, s>>>(V, Us, ukey);
    TH_LAUNCHED();
    if (nnz > 0) {
      k_row_rank<<<grid_for(nnz, 256), 256, 0, s>>>(V, rkeys, rowunit, ukey, nnz, rank, sorted, rowcnt, repeat);
      TH_LAUNCHED();
      k_row_links<<<grid_for(nnz, 256), 256, 0, s>>>(V, rkeys, rank, sorted, rowcnt, nnz, hc, lc, succ, lval);
      TH_LAUNCHED();
    }
    exclusive_scan_i64(hc, hc, nnz, tmp, s);
    exclusive_scan_i64(lc, lc, nnz, tmp, s);
    JPRun R;
    R.lrow = lrow;
    R.lsucc = lsucc;
    R.aptr = aptr;
    R.npred = npred;
    R.rowptr = orowptr;
    R.sorted = sorted;
    R.rmask = rmask;
    R.cnt = tmp.alloc<int32_t>(Us + 1);
    R.color = color;
    for (int q = 0; q < 2; ++q) {
      R.fs[q] = tmp.alloc<uint32_t>(Us + 1);
      R.fb[q] = tmp.alloc<uint32_t>(Us + 1);
    }
    R.fc = tmp.alloc<int64_t>(6);
    R.done = tmp.alloc<unsigned long long>(1);
    R.bar = tmp.alloc<unsigned>(1);
    R.err = tmp.alloc<int>(1);
    TH_CUDA(cudaMemsetAsync(R.fc, 0, 6 * sizeof(int64_t), s));
    TH_CUDA(cudaMemsetAsync(R.done, 0, sizeof(unsigned long long), s));
    TH_CUDA(cudaMemsetAsync(R.bar, 0, sizeof(unsigned), s));
    TH_CUDA(cudaMemsetAsync(R.err, 0, sizeof(int), s));
    k_chain_units<<<grid_for(Us, 256), 256, 0, s>>>(V, Us, nnz, hc, lc, aptr, npred, R.cnt, lbase, hend, ubig,
                                                    R.fs[0], R.fc + 0, R.fb[0], R.fc + 1);
    TH_LAUNCHED();
    if (nnz > 0) {
      k_chain_fill<<<grid_for(nnz, 256), 256, 0, s>>>(V, nnz, hc, lc, lbase, hend, succ, lval, ubig, lrow, lsucc);
      TH_LAUNCHED();
    }
    const int64_t max_rounds = Us + 2;
    if (coop && per > 0 && coop_allowed()) {
      // every round in one cooperative launch, a grid barrier between rounds
      int grid = sms * per;
      int64_t r0 = 0, nr = max_rounds;
      void* args[] = {(void*)&R, (void*)&r0, (void*)&nr};
      TH_CUDA(cudaLaunchCooperativeKernel((const void*)k_jp, dim3(grid), dim3(256), args, 0, s));
      TH_LAUNCHED();
    } else {
      // one launch per round; the host looks at the frontier every 16 rounds
      int64_t r = 0;
      while (r < max_rounds) {
        for (int q = 0; q < 16 && r < max_rounds; ++q, ++r) {
          k_jp<<<sms * 8, 256, 0, s>>>(R, r, 1);
          TH_LAUNCHED();
        }
        int64_t hc[2];
        TH_CUDA(cudaMemcpyAsync(hc, R.fc + 2 * (r % 3), 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TH_CUDA(cudaStreamSynchronize(s));
        if (hc[0] + hc[1] == 0) break;
      }
    }
    unsigned long long hdone = 0;
    int herr = 0, hrep = 0;
    TH_CUDA(cudaMemcpyAsync(&hdone, R.done, sizeof(hdone), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaMemcpyAsync(&herr, R.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaMemcpyAsync(&hrep, repeat, sizeof(int), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    P.blk_shared = hrep != 0;
    TH_CHECK(herr == 0, THETIS_E_TIMEOUT, "colouring: grid barrier timed out");
    TH_CHECK((int64_t)hdone == Us, THETIS_E_CUDA, "colouring left units uncoloured");
  }
  if (Msl > 0) {
    k_slack_color<<<grid_for(Msl, 256), 256, 0, s>>>(V, Msl, color);
    TH_LAUNCHED();
  }
  int* dmax = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(dmax, 0xff, sizeof(int), s));
  k_max_i32<<<grid_for(U, 256), 256, 0, s>>>(color, U, dmax);
  TH_LAUNCHED();
  int maxc = read_flag(dmax, s);
  const int32_t C = (U > 0) ? maxc + 1 : 0;
  P.ncolors = C;
  P.unit_color = P.mem.alloc<int32_t>(U);
  if (U > 0) {
    k_unit_color_copy<<<grid_for(U, 256), 256, 0, s>>>(color, U, P.unit_color);
    TH_LAUNCHED();
  }

  // -- colour order --------------------------------------------------------
  uint32_t* skeys = tmp.alloc<uint32_t>(Us + 1);
  uint32_t* unit_of_pos = P.mem.alloc<uint32_t>(Us + 1);
  int64_t* ccnt = tmp.alloc<int64_t>((int64_t)C * UC_COUNT + 1);
  TH_CUDA(cudaMemsetAsync(ccnt, 0, ((int64_t)C * UC_COUNT + 1) * sizeof(int64_t), s));
  if (Us > 0) {
    int hg;
    size_t hsm;
    hist_launch_shape(Us, (int64_t)C * UC_COUNT, &hg, &hsm);
    k_struct_keys<<<hg, 256, hsm, s>>>(color, ulen, unnz, Us, skeys, unit_of_pos, ccnt, (int64_t)C * UC_COUNT);
    TH_LAUNCHED();
  }
  radix_sort_pairs(skeys, unit_of_pos, Us, bits_for((int64_t)C * UC_COUNT + 1), tmp, s);
  P.unit_of_pos = unit_of_pos;
  // internal columns
  int64_t* plen = tmp.alloc<int64_t>(Us + 1);
  int64_t* cstart = tmp.alloc<int64_t>(Us + 1);
  if (Us > 0) {
    k_pos_len<<<grid_for(Us, 256), 256, 0, s>>>(unit_of_pos, ulen, Us, plen);
    TH_LAUNCHED();
  }
  exclusive_scan_i64(plen, cstart, Us, tmp, s);
  P.col_of_orig = P.mem.alloc<uint32_t>(Ns);
  uint32_t* orig_of_col = tmp.alloc<uint32_t>(Ns);
  if (Us > 0) {
    k_col_maps_free<<<grid_for(Us, 256), 256, 0, s>>>(unit_of_pos, ufirst, ulen, cstart, Us, P.col_of_orig, orig_of_col);
    TH_LAUNCHED();
  }
  k_col_maps_fixed<<<grid_for(Ns, 256), 256, 0, s>>>(fixed_flag, fixed_scan, Ns, P.Nfree, P.col_of_orig, orig_of_col);
  TH_LAUNCHED();
  // Slack rows ordered by (slack colour, owner column): the owner of a row is
  // its highest-priority column, so the rows a column owns -- nearly all rows of
  // a hub -- are consecutive and its gather / scatter of r is coalesced.
  uint32_t* slkeys = tmp.alloc<uint32_t>(Msl + 1);
  uint32_t* slrows0 = tmp.alloc<uint32_t>(Msl + 1);
  uint32_t* slrows = tmp.alloc<uint32_t>(Msl + 1);
  int64_t* scnt = tmp.alloc<int64_t>(C + 1);
  TH_CUDA(cudaMemsetAsync(scnt, 0, (C + 1) * sizeof(int64_t), s));
  if (Msl > 0) {
    k_slack_owner_keys<<<grid_for(Msl, 256), 256, 0, s>>>(V, Msl, P.col_of_orig, slkeys, slrows0);
    TH_LAUNCHED();
  }
  {  // by owner column (the rows ascend within an owner's group)
    int64_t* optr = tmp.alloc<int64_t>(Ns + 2);
    group_by_key(slkeys, slrows0, Msl, Ns + 1, slrows, optr, tmp, s);
  }
  if (Msl > 0) {
    int hg;
    size_t hsm;
    hist_launch_shape(Msl, C, &hg, &hsm);
    k_slack_color_keys<<<hg, 256, hsm, s>>>(slrows, Msl, slack_unit, color, slkeys, scnt, C);
    TH_LAUNCHED();
  }
  radix_sort_pairs(slkeys, slrows, Msl, bits_for(C + 1), tmp, s);
  std::vector<int64_t> hc((size_t)C * UC_COUNT + 1), hs((size_t)C + 1);
  TH_CUDA(cudaMemcpyAsync(hc.data(), ccnt, hc.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hs.data(), scnt, hs.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  // internal rows
  P.row_of_orig = P.mem.alloc<uint32_t>(M);
  P.orig_of_row = P.mem.alloc<uint32_t>(M);
  P.slack_orig = P.mem.alloc<uint32_t>(Msl);
  if (M > 0) {
    k_row_maps<<<grid_for(M, 256), 256, 0, s>>>(slrows, Msl, has, has_scan, M, P.row_of_orig, P.orig_of_row,
                                                P.slack_orig);
    TH_LAUNCHED();
  }

  // internal CSC
  int64_t* icnt = tmp.alloc<int64_t>(Ns + 1);
  k_int_col_counts<<<grid_for(Ns, 256), 256, 0, s>>>(orig_of_col, raw.colptr, Ns, icnt);
  TH_LAUNCHED();
  P.colptr = P.mem.alloc<int64_t>(Ns + 1);
  exclusive_scan_i64(icnt, P.colptr, Ns, tmp, s);
  P.rowidx = P.mem.alloc<uint32_t>(nnz);
  if (P.has_val) {
    P.val = P.mem.alloc<float>(nnz);
    P.csq = P.mem.alloc<float>(Ns);
  }
  // entries sorted by (internal column, internal row): every internal
  // column's entries gathered in place, then sorted by internal row
  {
    uint32_t* k1 = tmp.alloc<uint32_t>(nnz + 1);
    uint32_t* ord = tmp.alloc<uint32_t>(nnz + 1);
    if (nnz > 0) {
      if (nnz > 16 * Ns) {
        k_icsc_gather<<<grid_for(nnz, 256), 256, 0, s>>>(colof, P.col_of_orig, raw.colptr, raw.rowidx, P.row_of_orig,
                                                         P.colptr, nnz, k1, ord);
      } else {
        k_icsc_gather_cols<<<grid_for(Ns, 256), 256, 0, s>>>(orig_of_col, raw.colptr, raw.rowidx, P.row_of_orig,
                                                             P.colptr, Ns, k1, ord);
      }
      TH_LAUNCHED();
    }
    segsort_pairs(P.colptr, Ns, k1, ord, nnz, tmp, s);
    if (nnz > 0) {
      k_icsc_fill<<<grid_for(nnz, 256), 256, 0, s>>>(ord, k1, raw.val, nnz, P.has_val, P.rowidx, P.val);
      TH_LAUNCHED();
    }
    if (P.has_val) {
      k_csq<<<grid_for(Ns * 32, 256), 256, 0, s>>>(P.colptr, P.val, Ns, P.csq);
      TH_LAUNCHED();
    }
  }
  // internal CSR (structural entries)
  int64_t* rcnt = tmp.alloc<int64_t>(M + 1);
  P.rowptr = P.mem.alloc<int64_t>(M + 1);
  if (M > 0) {
    k_int_row_counts<<<grid_for(M, 256), 256, 0, s>>>(P.orig_of_row, orowptr, M, rcnt);
    TH_LAUNCHED();
  }
  exclusive_scan_i64(rcnt, P.rowptr, M, tmp, s);
  P.colidx = P.mem.alloc<uint32_t>(nnz);
  if (P.has_val) P.rval = P.mem.alloc<float>(nnz);
  if (M > 0) {
    k_int_csr_fill<<<grid_for(M, 256), 256, 0, s>>>(P.orig_of_row, orowptr, csr_p, colof, raw.val, P.col_of_orig,
                                                    P.rowptr, M, P.has_val, P.colidx, P.rval);
    TH_LAUNCHED();
  }
  // vectors
  P.c = P.mem.alloc<float>(Ns);
  P.x = P.mem.alloc<float>(Ns);
  if (!P.bounds_uniform) {
    P.lo = P.mem.alloc<float>(Ns);
    P.hi = P.mem.alloc<float>(Ns);
  }
  k_col_vectors<<<grid_for(Ns, 256), 256, 0, s>>>(orig_of_col, raw.c, raw.lo, raw.hi, Ns, !P.bounds_uniform,
                                                  P.c, P.lo, P.hi);
  TH_LAUNCHED();
  P.b = P.mem.alloc<float>(M);
  P.sig = P.mem.alloc<int8_t>(M);
  P.r = P.mem.alloc<float>(M);
  P.s = P.mem.alloc<float>(Msl);
  if (M > 0) {
    k_row_vectors<<<grid_for(M, 256), 256, 0, s>>>(P.orig_of_row, raw.b, raw.row_kind, M, P.b, P.sig);
    TH_LAUNCHED();
  }
  // lmax and max unit size
  double* dsq = tmp.alloc<double>(1);
  unsigned long long* dmu = tmp.alloc<unsigned long long>(1);
  TH_CUDA(cudaMemsetAsync(dsq, 0, sizeof(double), s));
  TH_CUDA(cudaMemsetAsync(dmu, 0, sizeof(unsigned long long), s));
  if (P.Nfree > 0) {
    k_max_sq_free<<<grid_for(P.Nfree, 256), 256, 0, s>>>(P.colptr, P.csq, P.Nfree, dsq);
    TH_LAUNCHED();
  }
  k_max_unit_nnz<<<grid_for(U, 256), 256, 0, s>>>(unnz, U, dmu);
  TH_LAUNCHED();
  double hsq = 0.0;
  unsigned long long hmu = 0;
  TH_CUDA(cudaMemcpyAsync(&hsq, dsq, sizeof(double), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(&hmu, dmu, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  P.lmax_sq = std::max(hsq, (P.Msl > 0) ? 1.0 : 0.0);
  P.max_unit_nnz = (int64_t)hmu;

  // colour plan
  P.plan.assign(C, ColorPlan{});
  {
    int64_t u = 0, col = 0, srow = 0;
    for (int c = 0; c < C; ++c) {
      ColorPlan& cp = P.plan[c];
      for (int cls = 0; cls < UC_COUNT; ++cls) {
        int64_t n = hc[(size_t)c * UC_COUNT + cls];
        if (n == 0) continue;
        int32_t len = (cls == UC_BLOCK) ? P.k : 1;
        Seg sg{cls, u, u + n, col, len};
        if (is_small_class(cls)) {
          sg.e0 = P.ell_size;
          P.ell_size += (n + 31) / 32 * 32 * small_width(cls);
        }
        cp.segs.push_back(sg);
        u += n;
        col += n * len;
      }
      cp.srow0 = srow;
      srow += hs[c];
      cp.srow1 = srow;
    }
    TH_CHECK(u == Us && col == P.Nfree && srow == Msl, THETIS_E_CUDA, "colour plan inconsistent");
  }
  // ELL copy of the small classes' row ids, and the segment tables
  {
    std::vector<int64_t> sc0, sstart{0}, se0, bc0, bstart{0};
    std::vector<int32_t> sw;
    for (auto& cp : P.plan)
      for (auto& sg : cp.segs) {
        const int64_t n = sg.u1 - sg.u0;
        if (is_small_class(sg.cls)) {
          sc0.push_back(sg.c0);
          sstart.push_back(sstart.back() + n);
          se0.push_back(sg.e0);
          sw.push_back(small_width(sg.cls));
        } else if (sg.cls != UC_BLOCK) {
          bc0.push_back(sg.c0);
          bstart.push_back(bstart.back() + n);
        }
      }
    const int64_t ns = (int64_t)sc0.size(), nb = (int64_t)bc0.size();
    P.nss = ns;
    P.nsmall = sstart.back();
    P.nbs = nb;
    P.nbig = bstart.back();
    P.ss_start = P.mem.alloc<int64_t>(ns + 1);
    P.ss_c0 = P.mem.alloc<int64_t>(ns + 1);
    P.ss_e0 = P.mem.alloc<int64_t>(ns + 1);
    P.ss_w = P.mem.alloc<int32_t>(ns + 1);
    P.bs_start = P.mem.alloc<int64_t>(nb + 1);
    P.bs_c0 = P.mem.alloc<int64_t>(nb + 1);
    TH_CUDA(cudaMemcpyAsync(P.ss_start, sstart.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(P.bs_start, bstart.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (ns > 0) {
      TH_CUDA(cudaMemcpyAsync(P.ss_c0, sc0.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      TH_CUDA(cudaMemcpyAsync(P.ss_e0, se0.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      TH_CUDA(cudaMemcpyAsync(P.ss_w, sw.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    if (nb > 0) TH_CUDA(cudaMemcpyAsync(P.bs_c0, bc0.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    P.ell = P.mem.alloc<uint32_t>(P.ell_size + 1);
    if (P.has_val) P.ellv = P.mem.alloc<float>(P.ell_size + 1);
    if (ns > 0) {
      TH_CUDA(cudaMemsetAsync(P.ell, 0xff, P.ell_size * sizeof(uint32_t), s));
      std::vector<int64_t> sn(ns);
      for (int64_t t = 0; t < ns; ++t) sn[t] = sstart[t + 1] - sstart[t];
      int64_t* dn = tmp.alloc<int64_t>(ns);
      TH_CUDA(cudaMemcpyAsync(dn, sn.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      k_ell_fill<<<grid_for(P.Nfree, 256), 256, 0, s>>>(P.colptr, P.rowidx, P.has_val ? P.val : nullptr, P.ss_c0,
                                                        dn, P.ss_e0, P.ss_w, ns, P.Nfree, P.ell, P.ellv);
      TH_LAUNCHED();
    }
    TH_CUDA(cudaStreamSynchronize(s));  // the host vectors above must outlive the copies
  }
  // free simplex blocks (internal first columns)
  {
    std::vector<int64_t> bs;
    for (auto& cp : P.plan)
      for (auto& sg : cp.segs)
        if (sg.cls == UC_BLOCK)
          for (int64_t u = sg.u0; u < sg.u1; ++u) bs.push_back(sg.c0 + (u - sg.u0) * sg.len);
    P.nblk = (int64_t)bs.size();
    if (P.nblk > 0) {
      P.blk_start = P.mem.alloc<int64_t>(P.nblk);
      TH_CUDA(cudaMemcpyAsync(P.blk_start, bs.data(), P.nblk * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      TH_CUDA(cudaStreamSynchronize(s));
    }
  }

  // solve scratch
  P.r64 = P.mem.alloc<double>(M);
  P.red = P.mem.alloc<double>(8 * 4096);
  P.red_out = P.mem.alloc<double>(16);
  TH_CUDA(cudaMallocHost((void**)&P.h_red, 16 * sizeof(double)));
  return Pp;
}

Problem::~Problem() {
  inst_release(*this);
  if (epoch_graph) cudaGraphExecDestroy(epoch_graph);
  if (h_red) cudaFreeHost(h_red);
}

}  // namespace thetis
