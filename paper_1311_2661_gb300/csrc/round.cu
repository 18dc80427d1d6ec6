// Repair of the approximate LP point and oblivious rounding (App. C, App. B):
// vertex cover threshold (Sec. 2, Lemma lem:infeasible:rounded:vc), Bansal et
// al. packing rounding with alterations for independent set (App. B.2,
// Algorithm 2, theta = 1/k, tighter alpha of App. C.3), CKR region growing for
// multiway cut (App. B.3), set cover by f-threshold or randomized rounding
// (App. B.1) after the covering repair, best of R repetitions (Sec. 4.2),
// exact validity.
#include <algorithm>
#include <cmath>
#include <vector>

#include "problem.cuh"

namespace thetis {

#define GSTRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

constexpr int RB = 256;       // reduction blocks per repetition (fixed: deterministic sums)
constexpr int MAX_REPS = 64;
constexpr double NEAR_BAND = 1e-4;

__global__ void k_gather_x(const float* x, const uint32_t* col_of_orig, int64_t n, float* out) {
  GSTRIDE(j, n) out[j] = x[col_of_orig[j]];
}

void gather_x_orig(Problem& P, float* d_out) {
  k_gather_x<<<grid_for(P.Ns, 256), 256, 0, P.stream>>>(P.x, P.col_of_orig, P.Ns, d_out);
  TH_LAUNCHED();
  TH_CUDA(cudaGetLastError());
}

// max over edges of f(x_u + x_v), f(t) = (1 - t)_+ (VC) or (t - 1)_+ (IS), exact in FP64
__global__ void k_edge_violation(const float* x, const int32_t* eu, const int32_t* ev, int64_t m, int cover,
                                 unsigned long long* out) {
  double mx = 0.0;
  GSTRIDE(e, m) {
    double xu = (double)x[eu[e]], xv = (double)x[ev[e]];
    double v = cover ? (1.0 - xu) - xv : (xu + xv) - 1.0;
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// VC: x~ = min(1, x/(1-eps)); label = x~ >= 1/2; near-threshold count; weight partials
__global__ void k_vc_label(const float* x, const float* w, int64_t n, const unsigned long long* eps_bits,
                           uint8_t* lab, double* part, unsigned long long* near) {
  double eps = __longlong_as_double((long long)*eps_bits);
  double sum = 0.0;
  unsigned long long nr = 0;
  GSTRIDE(v, n) {
    double xt = fmin(1.0, fmax(0.0, (double)x[v] / (1.0 - eps)));
    uint8_t l = xt >= 0.5;
    lab[v] = l;
    if (fabs(xt - 0.5) < NEAR_BAND) ++nr;
    if (l) sum += (double)w[v];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    nr += __shfl_xor_sync(0xffffffffu, nr, o);
  }
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = sum;
    if (nr) atomicAdd(near, nr);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sm[q];
    part[blockIdx.x] = a;
  }
}

// IS, all repetitions: pick[r][v] = U(seed, r, 1, v) < x~_v
__global__ void k_is_pick(const float* x, int64_t n, int reps, uint64_t seed, const unsigned long long* alpha_bits,
                          uint8_t* pick) {
  double alpha = __longlong_as_double((long long)*alpha_bits);
  GSTRIDE(t, n * reps) {
    int64_t r = t / n, v = t % n;
    double xt = (double)x[v] / (1.0 + alpha);
    pick[t] = rng_unif(seed, (uint64_t)r, STREAM_IS_PICK, (uint64_t)v) < xt;
  }
}

// alteration: for every edge with both ends picked, delete the end of larger id
__global__ void k_is_alter(const int32_t* eu, const int32_t* ev, int64_t m, int64_t n, int reps, const uint8_t* pick,
                           uint8_t* keep) {
  GSTRIDE(t, m * reps) {
    int64_t r = t / m, e = t % m;
    int32_t u = eu[e], v = ev[e];
    const uint8_t* pr = pick + r * n;
    if (pr[u] && pr[v]) keep[r * n + (u > v ? u : v)] = 0;
  }
}

// per-repetition FP64 sums of w over selected vertices (VC/IS) in a fixed order
__global__ void k_rep_weight(const uint8_t* sel, const float* w, int64_t n, double* part) {
  int r = blockIdx.y;
  double sum = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (sel[(int64_t)r * n + v]) sum += (double)w[v];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sm[q];
    part[(int64_t)r * gridDim.x + blockIdx.x] = a;
  }
}

__global__ void k_rep_final(const double* part, int nb, int reps, double* out) {
  int r = threadIdx.x;
  if (r >= reps) return;
  double a = 0.0;
  for (int b = 0; b < nb; ++b) a += part[(int64_t)r * nb + b];
  out[r] = a;
}

// Set cover (App. B.1).  eps = max_a (1 - sum_{s holds a} x_s)_+ with the sum
// over the element's sets in increasing id (FP64, the order of the plain
// definition), the covering repair of App. C.2 (q(P) = 1).
__global__ void k_sc_eps(const float* x, const int64_t* eptr, const int32_t* esets, int64_t n_elem,
                         unsigned long long* out) {
  double mx = 0.0;
  GSTRIDE(a, n_elem) {
    double cov = 0.0;
    for (int64_t q = eptr[a]; q < eptr[a + 1]; ++q) cov += (double)x[esets[q]];
    mx = fmax(mx, 1.0 - cov);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

__device__ __forceinline__ double sc_xt(const float* x, int64_t j, double eps) {
  return fmin(1.0, fmax(0.0, (double)x[j] / (1.0 - eps)));
}

// f-threshold: take s iff x~_s >= 1/f; near-threshold count; cost partials
__global__ void k_sc_threshold(const float* x, const float* c, int64_t n_sets, double thr,
                               const unsigned long long* eps_bits, uint8_t* lab, double* part,
                               unsigned long long* near) {
  const double eps = __longlong_as_double((long long)*eps_bits);
  double sum = 0.0;
  unsigned long long nr = 0;
  GSTRIDE(j, n_sets) {
    const double xt = sc_xt(x, j, eps);
    const uint8_t l = xt >= thr;
    lab[j] = l;
    if (fabs(xt - thr) < NEAR_BAND) ++nr;
    if (l) sum += (double)c[j];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    nr += __shfl_xor_sync(0xffffffffu, nr, o);
  }
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = sum;
    if (nr) atomicAdd(near, nr);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sm[q];
    part[blockIdx.x] = a;
  }
}

// randomized rounding, all repetitions: pick[r][s] = U(seed, r, 4, s) < x~_s
__global__ void k_sc_pick(const float* x, int64_t n_sets, int reps, uint64_t seed, const unsigned long long* eps_bits,
                          uint8_t* pick) {
  const double eps = __longlong_as_double((long long)*eps_bits);
  GSTRIDE(t, n_sets * reps) {
    const int64_t r = t / n_sets, j = t % n_sets;
    pick[t] = rng_unif(seed, (uint64_t)r, STREAM_SC_PICK, (uint64_t)j) < sc_xt(x, j, eps);
  }
}

// fix-up: an element the picks of repetition r leave uncovered adds its set of
// largest x~ (ties: lowest id); marks read only the picks, so their order does
// not matter
__global__ void k_sc_fixup(const float* x, const int64_t* eptr, const int32_t* esets, int64_t n_elem, int64_t n_sets,
                           int reps, const unsigned long long* eps_bits, const uint8_t* pick, uint8_t* take) {
  const double eps = __longlong_as_double((long long)*eps_bits);
  GSTRIDE(t, n_elem * reps) {
    const int64_t r = t / n_elem, a = t % n_elem;
    const uint8_t* pr = pick + r * n_sets;
    bool covered = false;
    int64_t best = -1;
    double bx = 0.0;
    for (int64_t q = eptr[a]; q < eptr[a + 1]; ++q) {
      const int64_t j = esets[q];
      if (pr[j]) {
        covered = true;
        break;
      }
      const double xt = sc_xt(x, j, eps);
      if (best < 0 || xt > bx) {  // sets come in increasing id: ties keep the lowest
        best = j;
        bx = xt;
      }
    }
    if (!covered && best >= 0) take[r * n_sets + best] = 1;
  }
}

// every element covered by a taken set
__global__ void k_sc_valid(const uint8_t* lab, const int64_t* eptr, const int32_t* esets, int64_t n_elem, int* bad) {
  GSTRIDE(a, n_elem) {
    bool covered = false;
    for (int64_t q = eptr[a]; q < eptr[a + 1] && !covered; ++q) covered = lab[esets[q]] != 0;
    if (!covered) atomicExch(bad, 1);
  }
}

// Pairwise MAP node rounding (Sec. 4.1): every variable takes the label of its
// largest node marginal, ties to the lowest label.
__global__ void k_map_label(const float* x, int64_t n, int k, uint8_t* lab) {
  GSTRIDE(i, n) {
    int best = 0;
    float bx = x[i * k];
    for (int a = 1; a < k; ++a)
      if (x[i * k + a] > bx) {
        bx = x[i * k + a];
        best = a;
      }
    lab[i] = (uint8_t)best;
  }
}

// objective of the integral point, -(sum_i theta_i(l_i) + sum_e theta_e(l_u, l_v)),
// in fixed-order FP64 partials
__global__ void k_map_energy(const uint8_t* lab, const float* tn, const float* te, const int32_t* eu,
                             const int32_t* ev, int64_t n, int64_t m, int k, double* part) {
  double sum = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n + m; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < n) {
      sum -= (double)tn[t * k + lab[t]];
    } else {
      const int64_t e = t - n;
      sum -= (double)te[e * k * k + (int64_t)lab[eu[e]] * k + lab[ev[e]]];
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sm[q];
    part[blockIdx.x] = a;
  }
}

// CKR: label of every vertex in every repetition
__global__ void k_ckr_label(const float* x, int64_t n, int k, int reps, const double* rad, const int32_t* sigma,
                            uint8_t* lab) {
  GSTRIDE(t, n * reps) {
    int64_t r = t / n, v = t % n;
    const int32_t* sg = sigma + r * k;
    double thr = 1.0 - rad[r];
    int l = sg[k - 1];
    for (int q = 0; q < k - 1; ++q)
      if ((double)x[v * k + sg[q]] >= thr) {
        l = sg[q];
        break;
      }
    lab[t] = (uint8_t)l;
  }
}

__global__ void k_cut_cost(const uint8_t* lab, const int32_t* eu, const int32_t* ev, const float* ce, int64_t m,
                           int64_t n, double* part) {
  int r = blockIdx.y;
  double sum = 0.0;
  const uint8_t* L = lab + (int64_t)r * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    if (L[eu[e]] != L[ev[e]]) sum += (double)ce[e];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += sm[q];
    part[(int64_t)r * gridDim.x + blockIdx.x] = a;
  }
}

// exact validity: 0 = valid
__global__ void k_valid_edges(const uint8_t* lab, const int32_t* eu, const int32_t* ev, int64_t m, int kind,
                              int* bad) {
  GSTRIDE(e, m) {
    uint8_t a = lab[eu[e]], b = lab[ev[e]];
    if (kind == KIND_VC && !a && !b) atomicExch(bad, 1);
    if (kind == KIND_IS && a && b) atomicExch(bad, 1);
  }
}

__global__ void k_valid_mc(const uint8_t* lab, int64_t n, int k, const int32_t* term, int* bad) {
  GSTRIDE(v, n) if (lab[v] >= k) atomicExch(bad, 1);
  if (blockIdx.x == 0 && threadIdx.x < k)
    if (lab[term[threadIdx.x]] != threadIdx.x) atomicExch(bad, 1);
}

__global__ void k_is_near(const float* x, int64_t n, int rep, uint64_t seed, const unsigned long long* alpha_bits,
                          unsigned long long* near) {
  double alpha = __longlong_as_double((long long)*alpha_bits);
  unsigned long long c = 0;
  GSTRIDE(v, n) {
    double xt = (double)x[v] / (1.0 + alpha);
    if (fabs(rng_unif(seed, (uint64_t)rep, STREAM_IS_PICK, (uint64_t)v) - xt) < NEAR_BAND) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(near, c);
}

// every label below `limit` (VC / IS / SC membership: 2; MC and MAP: k)
__global__ void k_label_range(const uint8_t* lab, int64_t n, int limit, int* bad) {
  GSTRIDE(v, n) if (lab[v] >= limit) atomicExch(bad, 1);
}

// Exact validity and objective of a caller's integral solution (the checks
// the roundings end with): VC every edge covered, IS no edge inside the set,
// MC every label < k with terminal i labelled i, SC every element covered,
// MAP every label < k; labels outside their range make the solution invalid.
// The objective is the cover / set weight, the cut cost, the set cost or the
// MAP energy (-score), in FP64; NaN when a label is out of range.
void check_labels(Problem& P, int kind, const uint8_t* d_labels, int& valid, double& obj) {
  cudaStream_t s = P.stream;
  const bool ok_kind = (kind == THETIS_ROUND_VC && P.kind == KIND_VC) || (kind == THETIS_ROUND_IS && P.kind == KIND_IS) ||
                       (kind == THETIS_ROUND_MC && P.kind == KIND_MC) ||
                       ((kind == THETIS_ROUND_SC || kind == THETIS_ROUND_SC_RAND) && P.kind == KIND_SC) ||
                       (kind == THETIS_ROUND_MAP && P.kind == KIND_MAP);
  TH_CHECK(ok_kind, THETIS_E_INVALID, "label check: kind does not match the problem");
  const bool sc = P.kind == KIND_SC;
  const int64_t n = P.nv, m = P.ne;
  const int limit = (P.kind == KIND_MC || P.kind == KIND_MAP) ? P.k : 2;
  Arena tmp(s);
  int* bad = tmp.alloc<int>(2);  // [0]: range, [1]: validity
  double* part = tmp.alloc<double>(RB);
  double* res = tmp.alloc<double>(1);
  TH_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), s));
  if (n > 0) {
    k_label_range<<<grid_for(n, 256), 256, 0, s>>>(d_labels, n, limit, bad);
    TH_LAUNCHED();
  }
  int hb[2] = {0, 0};
  TH_CUDA(cudaMemcpyAsync(hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  if (hb[0]) {  // the objective kernels index by label: stop here
    valid = 0;
    obj = std::nan("");
    return;
  }
  if (P.kind == KIND_VC || P.kind == KIND_IS) {
    if (m > 0) {
      k_valid_edges<<<grid_for(m, 256), 256, 0, s>>>(d_labels, P.eu, P.ev, m, P.kind, bad + 1);
      TH_LAUNCHED();
    }
    k_rep_weight<<<dim3(RB, 1), 256, 0, s>>>(d_labels, P.w, n, part);
  } else if (P.kind == KIND_MC) {
    k_valid_mc<<<grid_for(n, 256), 256, 0, s>>>(d_labels, n, P.k, P.term, bad + 1);
    TH_LAUNCHED();
    k_cut_cost<<<dim3(RB, 1), 256, 0, s>>>(d_labels, P.eu, P.ev, P.ce, m, n, part);
  } else if (sc) {
    if (P.M > 0) {
      k_sc_valid<<<grid_for(P.M, 256), 256, 0, s>>>(d_labels, P.sc_eptr, P.sc_esets, P.M, bad + 1);
      TH_LAUNCHED();
    }
    k_rep_weight<<<dim3(RB, 1), 256, 0, s>>>(d_labels, P.w, n, part);
  } else {  // MAP: any in-range labelling is feasible
    k_map_energy<<<RB, 256, 0, s>>>(d_labels, P.map_tn, P.map_te, P.eu, P.ev, n, m, P.k, part);
  }
  TH_LAUNCHED();
  k_rep_final<<<1, 32, 0, s>>>(part, RB, 1, res);
  TH_LAUNCHED();
  TH_CUDA(cudaMemcpyAsync(&hb[1], bad + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(&obj, res, sizeof(double), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CUDA(cudaGetLastError());
  valid = hb[1] ? 0 : 1;
}

void round_problem(Problem& P, int kind, uint64_t seed, int reps, uint8_t* d_labels, RoundOut& out) {
  cudaStream_t s = P.stream;
  TH_CHECK(P.kind == KIND_VC || P.kind == KIND_IS || P.kind == KIND_MC || P.kind == KIND_SC || P.kind == KIND_MAP,
           THETIS_E_INVALID, "rounding needs a problem built by thetis_build_vc / _is / _mc / _sc / _map");
  TH_CHECK((kind == THETIS_ROUND_VC && P.kind == KIND_VC) || (kind == THETIS_ROUND_IS && P.kind == KIND_IS) ||
               (kind == THETIS_ROUND_MC && P.kind == KIND_MC) ||
               ((kind == THETIS_ROUND_SC || kind == THETIS_ROUND_SC_RAND) && P.kind == KIND_SC) ||
               (kind == THETIS_ROUND_MAP && P.kind == KIND_MAP),
           THETIS_E_INVALID, "rounding kind does not match the problem");
  if (kind == THETIS_ROUND_VC || kind == THETIS_ROUND_SC || kind == THETIS_ROUND_MAP) reps = 1;
  TH_CHECK(reps >= 1 && reps <= MAX_REPS, THETIS_E_INVALID, "reps must be in [1, 64]");
  const int64_t n = P.nv, m = P.ne;
  Arena tmp(s);
  if (!P.xorig) P.xorig = P.mem.alloc<float>(P.Ns);
  gather_x_orig(P, P.xorig);
  unsigned long long* dbits = tmp.alloc<unsigned long long>(4);
  TH_CUDA(cudaMemsetAsync(dbits, 0, 4 * sizeof(unsigned long long), s));
  int* bad = (int*)(dbits + 3);
  double* part = tmp.alloc<double>((int64_t)RB * reps + 1);
  double* repv = tmp.alloc<double>(reps);
  std::vector<double> hv(reps);
  out.best_rep = 0;
  out.near = 0;
  out.status = THETIS_OK;
  if (kind == THETIS_ROUND_MAP) {
    k_map_label<<<grid_for(n, 256), 256, 0, s>>>(P.xorig, n, P.k, d_labels);
    TH_LAUNCHED();
    k_map_energy<<<RB, 256, 0, s>>>(d_labels, P.map_tn, P.map_te, P.eu, P.ev, n, m, P.k, part);
    TH_LAUNCHED();
    k_rep_final<<<1, 32, 0, s>>>(part, RB, 1, repv);
    TH_LAUNCHED();
    out.repair = 0.0;
  } else if (kind == THETIS_ROUND_SC || kind == THETIS_ROUND_SC_RAND) {
    const int64_t ns = P.Ns, ne_ = P.M;  // sets, elements
    if (ne_ > 0) {
      k_sc_eps<<<grid_for(ne_, 256, 152 * 8), 256, 0, s>>>(P.xorig, P.sc_eptr, P.sc_esets, ne_, dbits);
      TH_LAUNCHED();
    }
    unsigned long long hb = 0;
    TH_CUDA(cudaMemcpyAsync(&hb, dbits, sizeof(hb), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    double eps;
    memcpy(&eps, &hb, sizeof(double));
    out.repair = eps;
    if (eps >= 1.0) {
      out.status = THETIS_E_REPAIR;
      return;
    }
    if (kind == THETIS_ROUND_SC) {
      k_sc_threshold<<<RB, 256, 0, s>>>(P.xorig, P.w, ns, 1.0 / (double)P.sc_f, dbits, d_labels, part, dbits + 1);
      TH_LAUNCHED();
      k_rep_final<<<1, 32, 0, s>>>(part, RB, 1, repv);
      TH_LAUNCHED();
    } else {
      uint8_t* pick = tmp.alloc<uint8_t>(ns * reps);
      uint8_t* take = tmp.alloc<uint8_t>(ns * reps);
      k_sc_pick<<<grid_for(ns * reps, 256), 256, 0, s>>>(P.xorig, ns, reps, seed, dbits, pick);
      TH_LAUNCHED();
      TH_CUDA(cudaMemcpyAsync(take, pick, ns * reps, cudaMemcpyDeviceToDevice, s));
      if (ne_ > 0) {
        k_sc_fixup<<<grid_for(ne_ * reps, 256), 256, 0, s>>>(P.xorig, P.sc_eptr, P.sc_esets, ne_, ns, reps, dbits,
                                                             pick, take);
        TH_LAUNCHED();
      }
      k_rep_weight<<<dim3(RB, reps), 256, 0, s>>>(take, P.w, ns, part);
      TH_LAUNCHED();
      k_rep_final<<<1, MAX_REPS, 0, s>>>(part, RB, reps, repv);
      TH_LAUNCHED();
      TH_CUDA(cudaMemcpyAsync(hv.data(), repv, reps * sizeof(double), cudaMemcpyDeviceToHost, s));
      TH_CUDA(cudaStreamSynchronize(s));
      int best = 0;
      for (int r = 1; r < reps; ++r)
        if (hv[r] < hv[best]) best = r;
      out.best_rep = best;
      TH_CUDA(cudaMemcpyAsync(d_labels, take + (int64_t)best * ns, ns, cudaMemcpyDeviceToDevice, s));
    }
    if (ne_ > 0) {
      k_sc_valid<<<grid_for(ne_, 256), 256, 0, s>>>(d_labels, P.sc_eptr, P.sc_esets, ne_, bad);
      TH_LAUNCHED();
    }
  } else if (kind == THETIS_ROUND_VC || kind == THETIS_ROUND_IS) {
    bool cover = kind == THETIS_ROUND_VC;
    if (m > 0) {
      k_edge_violation<<<grid_for(m, 256, 152 * 8), 256, 0, s>>>(P.xorig, P.eu, P.ev, m, cover ? 1 : 0, dbits);
      TH_LAUNCHED();
    }
    unsigned long long hb = 0;
    TH_CUDA(cudaMemcpyAsync(&hb, dbits, sizeof(hb), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    double viol;
    memcpy(&viol, &hb, sizeof(double));
    out.repair = viol;
    if (cover) {
      if (viol >= 1.0) {
        out.status = THETIS_E_REPAIR;
        return;
      }
      k_vc_label<<<RB, 256, 0, s>>>(P.xorig, P.w, n, dbits, d_labels, part, dbits + 1);
      TH_LAUNCHED();
      k_rep_final<<<1, 32, 0, s>>>(part, RB, 1, repv);
      TH_LAUNCHED();
      if (m > 0) {
        k_valid_edges<<<grid_for(m, 256), 256, 0, s>>>(d_labels, P.eu, P.ev, m, KIND_VC, bad);
        TH_LAUNCHED();
      }
    } else {
      uint8_t* pick = tmp.alloc<uint8_t>(n * reps);
      uint8_t* keep = tmp.alloc<uint8_t>(n * reps);
      k_is_pick<<<grid_for(n * reps, 256), 256, 0, s>>>(P.xorig, n, reps, seed, dbits, pick);
      TH_LAUNCHED();
      TH_CUDA(cudaMemcpyAsync(keep, pick, n * reps, cudaMemcpyDeviceToDevice, s));
      if (m > 0) {
        k_is_alter<<<grid_for(m * reps, 256), 256, 0, s>>>(P.eu, P.ev, m, n, reps, pick, keep);
        TH_LAUNCHED();
      }
      k_rep_weight<<<dim3(RB, reps), 256, 0, s>>>(keep, P.w, n, part);
      TH_LAUNCHED();
      k_rep_final<<<1, MAX_REPS, 0, s>>>(part, RB, reps, repv);
      TH_LAUNCHED();
      TH_CUDA(cudaMemcpyAsync(hv.data(), repv, reps * sizeof(double), cudaMemcpyDeviceToHost, s));
      TH_CUDA(cudaStreamSynchronize(s));
      int best = 0;
      for (int r = 1; r < reps; ++r)
        if (hv[r] > hv[best]) best = r;
      out.best_rep = best;
      TH_CUDA(cudaMemcpyAsync(d_labels, keep + (int64_t)best * n, n, cudaMemcpyDeviceToDevice, s));
      k_is_near<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(P.xorig, n, best, seed, dbits, dbits + 1);
      TH_LAUNCHED();
      if (m > 0) {
        k_valid_edges<<<grid_for(m, 256), 256, 0, s>>>(d_labels, P.eu, P.ev, m, KIND_IS, bad);
        TH_LAUNCHED();
      }
    }
  } else {
    const int k = P.k;
    std::vector<double> rad(reps);
    std::vector<int32_t> sig((size_t)reps * k);
    for (int r = 0; r < reps; ++r) {
      rad[r] = rng_unif(seed, (uint64_t)r, STREAM_CKR_RADIUS, 0);
      int32_t* sg = &sig[(size_t)r * k];
      for (int i = 0; i < k; ++i) sg[i] = i;
      for (int i = k - 1; i >= 1; --i) {
        int j = (int)std::floor(rng_unif(seed, (uint64_t)r, STREAM_CKR_PERM, (uint64_t)i) * (double)(i + 1));
        std::swap(sg[i], sg[j]);
      }
    }
    double* drad = tmp.alloc<double>(reps);
    int32_t* dsig = tmp.alloc<int32_t>((int64_t)reps * k);
    TH_CUDA(cudaMemcpyAsync(drad, rad.data(), reps * sizeof(double), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(dsig, sig.data(), sig.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    uint8_t* lab = tmp.alloc<uint8_t>(n * reps);
    k_ckr_label<<<grid_for(n * reps, 256), 256, 0, s>>>(P.xorig, n, k, reps, drad, dsig, lab);
    TH_LAUNCHED();
    k_cut_cost<<<dim3(RB, reps), 256, 0, s>>>(lab, P.eu, P.ev, P.ce, m, n, part);
    TH_LAUNCHED();
    k_rep_final<<<1, MAX_REPS, 0, s>>>(part, RB, reps, repv);
    TH_LAUNCHED();
    TH_CUDA(cudaMemcpyAsync(hv.data(), repv, reps * sizeof(double), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    int best = 0;
    for (int r = 1; r < reps; ++r)
      if (hv[r] < hv[best]) best = r;
    out.best_rep = best;
    out.repair = 0.0;
    TH_CUDA(cudaMemcpyAsync(d_labels, lab + (int64_t)best * n, n, cudaMemcpyDeviceToDevice, s));
    k_valid_mc<<<grid_for(n, 256), 256, 0, s>>>(d_labels, n, k, P.term, bad);
    TH_LAUNCHED();
  }
  unsigned long long hn[4];
  TH_CUDA(cudaMemcpyAsync(hn, dbits, sizeof(hn), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hv.data(), repv, reps * sizeof(double), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  out.near = (int64_t)hn[1];
  int hbad = (int)(hn[3] & 0xffffffffu);
  out.valid = hbad ? 0 : 1;
  out.obj = hv[out.best_rep];
  TH_CUDA(cudaGetLastError());
}

}  // namespace thetis
