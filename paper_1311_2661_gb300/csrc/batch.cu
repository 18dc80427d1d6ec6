// Batches of independent vertex-cover / independent-set LPs as one
// block-diagonal LP.  The union goes through the single-problem pipeline
// unchanged (device build, colouring, colour-ordered layout, persistent sweep,
// FP64 refresh and checks): the conflict graph of a block-diagonal matrix is
// the disjoint union of the instances' conflict graphs, so every colour class
// of the union is the union of the instances' classes, the number of colours
// is the largest of the instances', and one sweep advances every instance.
// The colouring priority hashes instance-local ids, so each instance is
// coloured -- and therefore swept -- exactly as it would be alone.  Repair and
// rounding (Sec. 2, App. B.2, App. C) are done per instance here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "problem.cuh"

namespace thetis {

#define GSTRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// index t with off[t] <= x < off[t + 1]
__device__ __forceinline__ int64_t seg_of(const int64_t* off, int64_t count, int64_t x) {
  int64_t lo = 0, hi = count;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_batch_edges(const int32_t* eu, const int32_t* ev, const int64_t* noff, const int64_t* eoff,
                              int64_t count, int64_t Ne, int32_t* geu, int32_t* gev, uint32_t* prio_row, int* err) {
  GSTRIDE(e, Ne) {
    const int64_t t = seg_of(eoff, count, e);
    const int64_t nt = noff[t + 1] - noff[t];
    const int32_t a = eu[e], b = ev[e];
    if (a < 0 || b < 0 || a >= nt || b >= nt || a == b) atomicExch(err, 1);
    geu[e] = (int32_t)(noff[t] + a);
    gev[e] = (int32_t)(noff[t] + b);
    prio_row[e] = (uint32_t)(nt + (e - eoff[t]));  // the slack's unit id in the instance alone
  }
}

__global__ void k_batch_vectors(const uint8_t* kind, const int64_t* noff, const int64_t* eoff, int64_t count,
                                const float* w, int64_t Nv, int64_t Ne, float* b, float* c, float* lo, float* hi,
                                uint8_t* rk, uint32_t* prio_col, int* err) {
  GSTRIDE(i, Nv > Ne ? Nv : Ne) {
    if (i < Nv) {
      const int64_t t = seg_of(noff, count, i);
      const float wv = w[i];
      if (!(wv > 0.f) || !isfinite(wv)) atomicExch(err, 2);
      c[i] = (kind[t] == THETIS_ROUND_VC) ? wv : -wv;
      lo[i] = 0.f;
      hi[i] = 1.f;
      prio_col[i] = (uint32_t)(i - noff[t]);
    }
    if (i < Ne) {
      const int64_t t = seg_of(eoff, count, i);
      b[i] = 1.f;
      rk[i] = (kind[t] == THETIS_ROUND_VC) ? THETIS_ROW_GE : THETIS_ROW_LE;
    }
  }
}

__global__ void k_batch_check_kinds(const uint8_t* kind, int64_t count, int* err) {
  GSTRIDE(t, count) if (kind[t] != THETIS_ROUND_VC && kind[t] != THETIS_ROUND_IS) atomicExch(err, 3);
}

// (declared in build.cu)
void incidence_csc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, int64_t*& ptr, int32_t*& rows,
                   Arena& tmp, cudaStream_t s);

void build_batch_raw(int64_t count, const uint8_t* d_kind, const int64_t* d_noff, const int64_t* d_eoff, int64_t Nv,
                     int64_t Ne, const int32_t* d_eu, const int32_t* d_ev, const float* d_w, RawLP& raw,
                     int32_t*& geu, int32_t*& gev, bool& mixed, Arena& tmp, cudaStream_t s) {
  int* err = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_batch_check_kinds<<<grid_for(count, 256), 256, 0, s>>>(d_kind, count, err);
  TH_LAUNCHED();
  geu = tmp.alloc<int32_t>(Ne + 1);
  gev = tmp.alloc<int32_t>(Ne + 1);
  uint32_t* prow = tmp.alloc<uint32_t>(Ne + 1);
  uint32_t* pcol = tmp.alloc<uint32_t>(Nv + 1);
  if (Ne > 0) {
    k_batch_edges<<<grid_for(Ne, 256), 256, 0, s>>>(d_eu, d_ev, d_noff, d_eoff, count, Ne, geu, gev, prow, err);
    TH_LAUNCHED();
  }
  {  // the endpoints index the incidence counters below: checked first
    int h = 0;
    TH_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    TH_CHECK(h != 1, THETIS_E_INVALID, "batch: edge endpoint out of its instance's range, or a loop");
    TH_CHECK(h != 3, THETIS_E_INVALID, "batch: kinds must be THETIS_ROUND_VC or THETIS_ROUND_IS");
  }
  raw.M = Ne;
  raw.Ns = Nv;
  raw.nnz = 2 * Ne;
  incidence_csc(Nv, Ne, geu, gev, raw.colptr, raw.rowidx, tmp, s);
  raw.val = nullptr;
  raw.b = tmp.alloc<float>(Ne + 1);
  raw.c = tmp.alloc<float>(Nv);
  raw.lo = tmp.alloc<float>(Nv);
  raw.hi = tmp.alloc<float>(Nv);
  raw.row_kind = tmp.alloc<uint8_t>(Ne + 1);
  k_batch_vectors<<<grid_for(std::max(Nv, Ne), 256), 256, 0, s>>>(d_kind, d_noff, d_eoff, count, d_w, Nv, Ne, raw.b,
                                                                   raw.c, raw.lo, raw.hi, raw.row_kind, pcol, err);
  TH_LAUNCHED();
  int h = 0;
  TH_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CHECK(h != 1, THETIS_E_INVALID, "batch: edge endpoint out of its instance's range, or a loop");
  TH_CHECK(h != 2, THETIS_E_INVALID, "batch: vertex weights must be finite and > 0");
  TH_CHECK(h != 3, THETIS_E_INVALID, "batch: kinds must be THETIS_ROUND_VC or THETIS_ROUND_IS");
  raw.block_k = 1;
  raw.n_blocks = 0;
  raw.bounds_uniform = true;
  raw.lo_u = 0.f;
  raw.hi_u = 1.f;
  raw.slack_sign_uniform = 0;
  raw.prio_col = pcol;
  raw.prio_row = prow;
  mixed = true;
}

// ---------------------------------------------------------------------------
// per-instance repair and rounding
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  if (v > 0.0) atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// eps (VC) / alpha (IS) per instance, exact FP64 maxima
__global__ void k_bviol(const float* x, const int32_t* eu, const int32_t* ev, const int64_t* eoff,
                        const uint8_t* kind, int64_t count, int64_t Ne, unsigned long long* viol) {
  GSTRIDE(e, Ne) {
    const int64_t t = seg_of(eoff, count, e);
    const double xu = (double)x[eu[e]], xv = (double)x[ev[e]];
    const double v = (kind[t] == THETIS_ROUND_VC) ? (1.0 - xu) - xv : (xu + xv) - 1.0;
    atomic_max_pos(&viol[t], v);
  }
}

// VC instances: threshold labels; IS instances: picks of every repetition
__global__ void k_bpick(const float* x, const float* w, const int64_t* noff, const uint8_t* kind, int64_t count,
                        int64_t Nv, int reps, uint64_t seed, const unsigned long long* viol, uint8_t* lab,
                        uint8_t* pick, double* objs, unsigned long long* near) {
  GSTRIDE(v, Nv) {
    const int64_t t = seg_of(noff, count, v);
    const double a = __longlong_as_double((long long)viol[t]);
    const double xv = (double)x[v];
    if (kind[t] == THETIS_ROUND_VC) {
      if (a >= 1.0) {
        lab[v] = 0;
        continue;
      }
      const double xt = fmin(1.0, fmax(0.0, xv / (1.0 - a)));
      const uint8_t l = xt >= 0.5;
      lab[v] = l;
      if (fabs(xt - 0.5) < 1e-4) atomicAdd(&near[t], 1ull);
      if (l) atomicAdd(&objs[t * reps], (double)w[v]);
    } else {
      const double xt = xv / (1.0 + a);
      const uint64_t local = (uint64_t)(v - noff[t]);
      for (int r = 0; r < reps; ++r) pick[(int64_t)r * Nv + v] = rng_unif(seed, (uint64_t)r, STREAM_IS_PICK, local) < xt;
    }
  }
}

// IS alterations: the larger-id end of every edge with both ends picked goes
__global__ void k_balter(const int32_t* eu, const int32_t* ev, const int64_t* eoff, const uint8_t* kind,
                         int64_t count, int64_t Ne, int64_t Nv, int reps, const uint8_t* pick, uint8_t* keep) {
  GSTRIDE(q, Ne * reps) {
    const int64_t r = q / Ne, e = q % Ne;
    const int64_t t = seg_of(eoff, count, e);
    if (kind[t] != THETIS_ROUND_IS) continue;
    const int32_t u = eu[e], v = ev[e];
    const uint8_t* pr = pick + r * Nv;
    if (pr[u] && pr[v]) keep[r * Nv + (u > v ? u : v)] = 0;
  }
}

__global__ void k_bweight(const uint8_t* keep, const float* w, const int64_t* noff, const uint8_t* kind, int64_t count,
                          int64_t Nv, int reps, double* objs) {
  GSTRIDE(q, Nv * reps) {
    const int64_t r = q / Nv, v = q % Nv;
    const int64_t t = seg_of(noff, count, v);
    if (kind[t] == THETIS_ROUND_IS && keep[q]) atomicAdd(&objs[t * reps + r], (double)w[v]);
  }
}

// best repetition of every IS instance (ties to the lowest)
__global__ void k_bbest(const double* objs, const uint8_t* kind, int64_t count, int reps, int32_t* best) {
  GSTRIDE(t, count) {
    int b = 0;
    if (kind[t] == THETIS_ROUND_IS)
      for (int r = 1; r < reps; ++r)
        if (objs[t * reps + r] > objs[t * reps + b]) b = r;
    best[t] = b;
  }
}

__global__ void k_blabel(const uint8_t* keep, const int64_t* noff, const uint8_t* kind, const int32_t* best,
                         int64_t count, int64_t Nv, uint8_t* lab) {
  GSTRIDE(v, Nv) {
    const int64_t t = seg_of(noff, count, v);
    if (kind[t] == THETIS_ROUND_IS) lab[v] = keep[(int64_t)best[t] * Nv + v];
  }
}

__global__ void k_bvalid(const uint8_t* lab, const int32_t* eu, const int32_t* ev, const int64_t* eoff,
                         const uint8_t* kind, int64_t count, int64_t Ne, int* bad) {
  GSTRIDE(e, Ne) {
    const int64_t t = seg_of(eoff, count, e);
    const uint8_t a = lab[eu[e]], b = lab[ev[e]];
    if (kind[t] == THETIS_ROUND_VC ? (!a && !b) : (a && b)) atomicExch(&bad[t], 1);
  }
}

void round_batch(Problem& P, uint64_t seed, int reps, uint8_t* d_labels, std::vector<double>& obj,
                 std::vector<int32_t>& status, std::vector<int32_t>& best_rep, std::vector<double>& repair,
                 std::vector<int64_t>& near) {
  cudaStream_t s = P.stream;
  TH_CHECK(P.kind == KIND_BATCH, THETIS_E_INVALID, "thetis_round_batch needs a handle from thetis_build_batch");
  TH_CHECK(reps >= 1 && reps <= 64, THETIS_E_INVALID, "reps must be in [1, 64]");
  const int64_t count = P.nbatch, Nv = P.nv, Ne = P.ne;
  Arena tmp(s);
  if (!P.xorig) P.xorig = P.mem.alloc<float>(P.Ns);
  gather_x_orig(P, P.xorig);
  unsigned long long* viol = tmp.alloc<unsigned long long>(count);
  unsigned long long* nr = tmp.alloc<unsigned long long>(count);
  double* objs = tmp.alloc<double>(count * reps);
  int* bad = tmp.alloc<int>(count);
  int32_t* best = tmp.alloc<int32_t>(count);
  TH_CUDA(cudaMemsetAsync(viol, 0, count * sizeof(unsigned long long), s));
  TH_CUDA(cudaMemsetAsync(nr, 0, count * sizeof(unsigned long long), s));
  TH_CUDA(cudaMemsetAsync(objs, 0, count * reps * sizeof(double), s));
  TH_CUDA(cudaMemsetAsync(bad, 0, count * sizeof(int), s));
  uint8_t* pick = tmp.alloc<uint8_t>(Nv * reps);
  uint8_t* keep = tmp.alloc<uint8_t>(Nv * reps);
  if (Ne > 0) {
    k_bviol<<<grid_for(Ne, 256), 256, 0, s>>>(P.xorig, P.eu, P.ev, P.beoff, P.bkind, count, Ne, viol);
    TH_LAUNCHED();
  }
  k_bpick<<<grid_for(Nv, 256), 256, 0, s>>>(P.xorig, P.w, P.bnoff, P.bkind, count, Nv, reps, seed, viol, d_labels,
                                             pick, objs, nr);
  TH_LAUNCHED();
  TH_CUDA(cudaMemcpyAsync(keep, pick, Nv * reps, cudaMemcpyDeviceToDevice, s));
  if (Ne > 0) {
    k_balter<<<grid_for(Ne * reps, 256), 256, 0, s>>>(P.eu, P.ev, P.beoff, P.bkind, count, Ne, Nv, reps, pick, keep);
    TH_LAUNCHED();
  }
  k_bweight<<<grid_for(Nv * reps, 256), 256, 0, s>>>(keep, P.w, P.bnoff, P.bkind, count, Nv, reps, objs);
  TH_LAUNCHED();
  k_bbest<<<grid_for(count, 256), 256, 0, s>>>(objs, P.bkind, count, reps, best);
  TH_LAUNCHED();
  k_blabel<<<grid_for(Nv, 256), 256, 0, s>>>(keep, P.bnoff, P.bkind, best, count, Nv, d_labels);
  TH_LAUNCHED();
  if (Ne > 0) {
    k_bvalid<<<grid_for(Ne, 256), 256, 0, s>>>(d_labels, P.eu, P.ev, P.beoff, P.bkind, count, Ne, bad);
    TH_LAUNCHED();
  }
  std::vector<unsigned long long> hviol(count), hnear(count);
  std::vector<double> hobjs((size_t)count * reps);
  std::vector<int> hbad(count);
  best_rep.assign(count, 0);
  TH_CUDA(cudaMemcpyAsync(hviol.data(), viol, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hnear.data(), nr, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hobjs.data(), objs, hobjs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hbad.data(), bad, count * sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(best_rep.data(), best, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CUDA(cudaGetLastError());
  obj.assign(count, 0.0);
  status.assign(count, 1);
  repair.assign(count, 0.0);
  near.assign(count, 0);
  for (int64_t t = 0; t < count; ++t) {
    double a;
    memcpy(&a, &hviol[t], sizeof(double));
    repair[t] = a;
    near[t] = (int64_t)hnear[t];
    const bool vc = P.h_bkind[t] == THETIS_ROUND_VC;
    obj[t] = hobjs[(size_t)t * reps + (vc ? 0 : best_rep[t])];
    if (vc && a >= 1.0) status[t] = -1;
    else status[t] = hbad[t] ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// per-instance convergence
// ---------------------------------------------------------------------------
__global__ void k_binst(const uint32_t* col_of_orig, const uint32_t* orig_of_row, const int64_t* noff,
                        const int64_t* eoff, int64_t count, int64_t Ns, int64_t M, int32_t* inst_col,
                        int32_t* inst_row) {
  GSTRIDE(i, Ns > M ? Ns : M) {
    if (i < Ns) inst_col[col_of_orig[i]] = (int32_t)seg_of(noff, count, i);
    if (i < M) inst_row[i] = (int32_t)seg_of(eoff, count, (int64_t)orig_of_row[i]);
  }
}

// (one atomic per warp where its lanes share the instance)
__global__ void k_bmaxdeg(const int64_t* colptr, const int32_t* inst_col, int64_t Ns, int32_t* maxdeg) {
  GSTRIDE(j, Ns) {
    const int32_t t = inst_col[j], d = (int32_t)(colptr[j + 1] - colptr[j]);
    const unsigned act = __activemask();
    const int leader = __ffs(act) - 1;
    if (__all_sync(act, t == __shfl_sync(act, t, leader))) {
      const int32_t dmax = __reduce_max_sync(act, d);
      if ((int)(threadIdx.x & 31) == leader) atomicMax(&maxdeg[t], dmax);
    } else {
      atomicMax(&maxdeg[t], d);
    }
  }
}

void batch_index(Problem& P) {
  cudaStream_t s = P.stream;
  const int64_t count = P.nbatch;
  P.binst_col = P.mem.alloc<int32_t>(P.Ns + 1);
  P.binst_row = P.mem.alloc<int32_t>(P.M + 1);
  P.bfrozen = P.mem.alloc<uint8_t>(count);
  P.brho = P.mem.alloc<unsigned long long>(count);
  TH_CUDA(cudaMemsetAsync(P.bfrozen, 0, count, s));
  TH_CUDA(cudaMemsetAsync(P.brho, 0, count * sizeof(unsigned long long), s));
  const int64_t n = std::max(P.Ns, P.M);
  if (n > 0) {
    k_binst<<<grid_for(n, 256), 256, 0, s>>>(P.col_of_orig, P.orig_of_row, P.bnoff, P.beoff, count, P.Ns, P.M,
                                              P.binst_col, P.binst_row);
    TH_LAUNCHED();
  }
  P.bmaxdeg = P.mem.alloc<int32_t>(count);
  TH_CUDA(cudaMemsetAsync(P.bmaxdeg, 0, count * sizeof(int32_t), s));
  if (P.Ns > 0) {
    k_bmaxdeg<<<grid_for(P.Ns, 256), 256, 0, s>>>(P.colptr, P.binst_col, P.Ns, P.bmaxdeg);
    TH_LAUNCHED();
  }
  P.h_bfrozen.assign(count, 0);
  P.h_bepochs.assign(count, 0);
  P.h_brho.assign(count, 0.0);
  P.h_bdone.assign(count, 0.0);
  P.h_bstart.assign(count, 0.0);
  P.h_bctas.assign(count, 0);
}

void batch_begin_solve(Problem& P) {
  if (P.nbatch == 0) return;
  std::fill(P.h_bfrozen.begin(), P.h_bfrozen.end(), 0);
  std::fill(P.h_bepochs.begin(), P.h_bepochs.end(), 0);
  std::fill(P.h_brho.begin(), P.h_brho.end(), 0.0);
  std::fill(P.h_bdone.begin(), P.h_bdone.end(), 0.0);
  std::fill(P.h_bstart.begin(), P.h_bstart.end(), 0.0);
  std::fill(P.h_bctas.begin(), P.h_bctas.end(), 0);
  TH_CUDA(cudaMemsetAsync(P.bfrozen, 0, P.nbatch, P.stream));
  batch_active_tiles(P);
}

// After a check (the stream is synchronised): record every active instance's
// rho and freeze those at or below tol -- the test a solve of the instance
// alone makes at the same check.
bool batch_after_check(Problem& P, double tol, int epoch) {
  const int64_t count = P.nbatch;
  std::vector<unsigned long long> bits(count);
  TH_CUDA(cudaMemcpyAsync(bits.data(), P.brho, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  bool changed = false, all = true;
  for (int64_t t = 0; t < count; ++t) {
    if (P.h_bfrozen[t]) continue;
    double rho;
    memcpy(&rho, &bits[t], sizeof(double));
    P.h_brho[t] = rho;
    P.h_bepochs[t] = epoch;
    if (rho <= tol) {
      P.h_bfrozen[t] = 1;
      P.h_bdone[t] = P.batch_check_ms;
      changed = true;
    } else {
      all = false;
    }
  }
  if (changed) {
    TH_CUDA(cudaMemcpyAsync(P.bfrozen, P.h_bfrozen.data(), count, cudaMemcpyHostToDevice, P.stream));
    if (!all) batch_active_tiles(P);  // later sweeps skip the tiles of finished instances
  }
  // the host vector must outlive the copy
  TH_CUDA(cudaStreamSynchronize(P.stream));
  return all;
}

void batch_end_solve(Problem& P, int epoch) {
  for (int64_t t = 0; t < P.nbatch; ++t)
    if (!P.h_bfrozen[t]) {
      P.h_bepochs[t] = epoch;
      P.h_bdone[t] = P.batch_check_ms;
    }
}

void batch_inst_begin(Problem& P) {
  std::fill(P.h_bfrozen.begin(), P.h_bfrozen.end(), 0);
  std::fill(P.h_bepochs.begin(), P.h_bepochs.end(), 0);
  std::fill(P.h_brho.begin(), P.h_brho.end(), 0.0);
  std::fill(P.h_bdone.begin(), P.h_bdone.end(), 0.0);
  TH_CUDA(cudaMemsetAsync(P.bfrozen, 0, P.nbatch, P.stream));
}

void batch_inst_end(Problem& P, int& ep_max, bool& all_converged, int64_t& updates) {
  const int64_t count = P.nbatch;
  std::vector<unsigned long long> bits(count);
  TH_CUDA(cudaMemcpyAsync(bits.data(), P.brho, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, P.stream));
  TH_CUDA(cudaStreamSynchronize(P.stream));
  ep_max = 0;
  all_converged = true;
  updates = 0;
  for (int64_t t = 0; t < count; ++t) {
    double rho;
    memcpy(&rho, &bits[t], sizeof(double));
    P.h_brho[t] = rho;
    P.h_bepochs[t] = P.h_iep[t];
    P.h_bfrozen[t] = (uint8_t)(P.h_iconv[t] != 0);
    P.h_bdone[t] = (double)(P.h_it[2 * t + 1] - P.h_it[2 * count]) * 1e-6;
    P.h_bstart[t] = (double)(P.h_it[2 * t] - P.h_it[2 * count]) * 1e-6;
    P.h_bctas[t] = (int32_t)P.h_iK[t];
    ep_max = std::max(ep_max, P.h_iep[t]);
    all_converged = all_converged && P.h_iconv[t] != 0;
    updates += (int64_t)P.h_iep[t] * ((P.h_bnoff[t + 1] - P.h_bnoff[t]) + (P.h_beoff[t + 1] - P.h_beoff[t]));
  }
}

}  // namespace thetis
