// C ABI of the library (include/thetis.h).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "problem.cuh"

using namespace thetis;

struct thetis_handle {
  std::unique_ptr<Problem> P;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr, evb = nullptr;
  int64_t graph_launches = 0;  // kernels per epoch graph replay
  // key of the captured epoch graph
  double g_beta = 0;
  int g_rule = -1, g_mode = -1, g_ub = -1, g_xb = -1, g_small = -1, g_async = -1;
  ~thetis_handle() {
    if (P) {
      cudaStreamSynchronize(stream);
      P.reset();
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (ev2) cudaEventDestroy(ev2);
    if (ev3) cudaEventDestroy(ev3);
    if (evb) cudaEventDestroy(evb);
    if (own_stream && stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
  }
};

namespace thetis {
// the problem behind a handle (the request server reads a batch's per-instance
// outputs while its solve runs)
Problem* problem_of(thetis_handle* h) { return h ? h->P.get() : nullptr; }
}  // namespace thetis

namespace {

template <class F>
thetis_status guard(cudaStream_t s, F&& f) {
  try {
    f();
    return THETIS_OK;
  } catch (Error& e) {
    set_error(e.msg);
    if (e.st == THETIS_E_CUDA || e.st == THETIS_E_NOMEM) {
      if (s) cudaStreamSynchronize(s);
      cudaError_t le = cudaGetLastError();
      if (e.st == THETIS_E_CUDA && le == cudaErrorMemoryAllocation) return THETIS_E_NOMEM;
    }
    if (e.st == THETIS_E_CUDA && e.msg.find("out of memory") != std::string::npos) return THETIS_E_NOMEM;
    return e.st;
  } catch (std::bad_alloc&) {
    set_error("host allocation failed");
    return THETIS_E_NOMEM;
  } catch (std::exception& e) {
    set_error(e.what());
    return THETIS_E_INVALID;
  }
}

// Copy n elements to the device if they are on the host; returns a device pointer.
template <class T>
const T* to_dev(const T* p, int64_t n, int32_t mem, Arena& tmp, cudaStream_t s) {
  if (!p) return nullptr;
  if (mem == THETIS_MEM_DEVICE) return p;
  TH_CHECK(mem == THETIS_MEM_HOST, THETIS_E_INVALID, "mem must be THETIS_MEM_HOST or THETIS_MEM_DEVICE");
  T* d = tmp.alloc<T>(n);
  if (n > 0) TH_CUDA(cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

template <class T>
void from_dev(T* dst, const T* src, int64_t n, int32_t mem, cudaStream_t s) {
  if (n <= 0) return;
  TH_CHECK(mem == THETIS_MEM_HOST || mem == THETIS_MEM_DEVICE, THETIS_E_INVALID, "bad out_mem");
  TH_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), mem == THETIS_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                        : cudaMemcpyDeviceToDevice, s));
}

thetis_handle* new_handle(void* stream) {
  auto* h = new thetis_handle();
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      throw Error{THETIS_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)};
    }
    h->own_stream = true;
  }
  return h;
}

template <class T>
T* keep_copy(Arena& mem, const T* src_dev, int64_t n, cudaStream_t s) {
  T* d = mem.alloc<T>(n);
  if (n > 0) TH_CUDA(cudaMemcpyAsync(d, src_dev, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  return d;
}

void finish_create(thetis_handle* h) {
  init_iterate(*h->P);
  TH_CUDA(cudaEventCreate(&h->ev0));
  TH_CUDA(cudaEventCreate(&h->ev1));
  TH_CUDA(cudaEventCreate(&h->ev2));
  TH_CUDA(cudaEventCreate(&h->ev3));
  TH_CUDA(cudaEventCreate(&h->evb));
  TH_CUDA(cudaStreamSynchronize(h->stream));
}

}  // namespace

extern "C" {

const char* thetis_last_error(void) { return get_error(); }
uint64_t thetis_launch_count(void) { return launch_count(); }

thetis_status thetis_create(const thetis_problem_desc* d, int32_t mem, uint64_t seed, void* stream,
                            thetis_handle** out) {
  if (!d || !out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  *out = nullptr;
  thetis_handle* h = nullptr;
  thetis_status st = guard(nullptr, [&] {
    TH_CHECK(d->n >= 1 && d->m >= 0, THETIS_E_INVALID, "need n >= 1 and m >= 0");
    TH_CHECK(d->csc_ptr && d->b && d->c && d->lo && d->hi && d->row_kind, THETIS_E_INVALID, "null array in desc");
    h = new_handle(stream);
    cudaStream_t s = h->stream;
    Arena tmp(s);
    int64_t nnz = 0;
    if (mem == THETIS_MEM_HOST) {
      nnz = d->csc_ptr[d->n];
    } else {
      TH_CUDA(cudaMemcpyAsync(&nnz, d->csc_ptr + d->n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      TH_CUDA(cudaStreamSynchronize(s));
    }
    TH_CHECK(nnz >= 0, THETIS_E_INVALID, "negative nnz");
    TH_CHECK(nnz == 0 || d->csc_row, THETIS_E_INVALID, "csc_row is null");
    RawLP raw;
    raw.M = d->m;
    raw.Ns = d->n;
    raw.nnz = nnz;
    raw.colptr = const_cast<int64_t*>(to_dev(d->csc_ptr, d->n + 1, mem, tmp, s));
    raw.rowidx = const_cast<int32_t*>(to_dev(d->csc_row, nnz, mem, tmp, s));
    raw.val = const_cast<float*>(to_dev(d->csc_val, nnz, mem, tmp, s));
    raw.b = const_cast<float*>(to_dev(d->b, d->m, mem, tmp, s));
    raw.c = const_cast<float*>(to_dev(d->c, d->n, mem, tmp, s));
    raw.lo = const_cast<float*>(to_dev(d->lo, d->n, mem, tmp, s));
    raw.hi = const_cast<float*>(to_dev(d->hi, d->n, mem, tmp, s));
    raw.row_kind = const_cast<uint8_t*>(to_dev(d->row_kind, d->m, mem, tmp, s));
    raw.block_k = d->n_blocks > 0 ? d->block_k : 1;
    raw.n_blocks = d->n_blocks;
    TH_CHECK(d->n_blocks == 0 || d->block_first, THETIS_E_INVALID, "block_first is null");
    raw.block_first = const_cast<int64_t*>(to_dev(d->block_first, d->n_blocks, mem, tmp, s));
    h->P = build_problem(raw, KIND_GENERAL, seed, s, tmp);
    finish_create(h);
  });
  if (st != THETIS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return THETIS_OK;
}

static thetis_status build_graph(int kind, int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                                 const float* wv, const float* ce, int32_t k, const int32_t* term, int32_t mem,
                                 uint64_t seed, void* stream, thetis_handle** out) {
  if (!out) {
    set_error("null out");
    return THETIS_E_INVALID;
  }
  *out = nullptr;
  thetis_handle* h = nullptr;
  thetis_status st = guard(nullptr, [&] {
    TH_CHECK(n >= 1 && m >= 0 && n < (int64_t(1) << 31) && m < (int64_t(1) << 31), THETIS_E_INVALID,
             "need 1 <= n < 2^31 and 0 <= m < 2^31");
    TH_CHECK(m == 0 || (eu && ev), THETIS_E_INVALID, "null edge array");
    if (kind == KIND_MC) {
      TH_CHECK(k >= 2 && k <= 32 && k <= n, THETIS_E_INVALID, "multiway cut needs 2 <= k <= min(32, n)");
      TH_CHECK(term && (m == 0 || ce), THETIS_E_INVALID, "null terminals or edge weights");
      TH_CHECK((n + m) * (int64_t)k < (int64_t(1) << 31) && 2 * m * (int64_t)k < (int64_t(1) << 31),
               THETIS_E_INVALID, "multiway-cut LP too large");
    } else {
      TH_CHECK(wv != nullptr, THETIS_E_INVALID, "null vertex weights");
    }
    h = new_handle(stream);
    cudaStream_t s = h->stream;
    Arena tmp(s);
    const int32_t* deu = to_dev(eu, m, mem, tmp, s);
    const int32_t* dev = to_dev(ev, m, mem, tmp, s);
    RawLP raw;
    const float *dw = nullptr, *dce = nullptr;
    const int32_t* dterm = nullptr;
    if (kind == KIND_MC) {
      dce = to_dev(ce, m, mem, tmp, s);
      dterm = to_dev(term, k, mem, tmp, s);
      build_mc_raw(n, m, deu, dev, dce, k, dterm, raw, tmp, s);
    } else {
      dw = to_dev(wv, n, mem, tmp, s);
      build_vc_is_raw(kind, n, m, deu, dev, dw, raw, tmp, s);
    }
    h->P = build_problem(raw, kind, seed, s, tmp);
    Problem& P = *h->P;
    P.nv = n;
    P.ne = m;
    P.eu = keep_copy(P.mem, deu, m, s);
    P.ev = keep_copy(P.mem, dev, m, s);
    if (kind == KIND_MC) {
      P.ce = keep_copy(P.mem, dce, m, s);
      P.term = keep_copy(P.mem, dterm, k, s);
    } else {
      P.w = keep_copy(P.mem, dw, n, s);
    }
    finish_create(h);
  });
  if (st != THETIS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return THETIS_OK;
}

thetis_status thetis_build_vc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const float* w,
                              int32_t mem, uint64_t seed, void* stream, thetis_handle** out) {
  return build_graph(KIND_VC, n, m, eu, ev, w, nullptr, 0, nullptr, mem, seed, stream, out);
}
thetis_status thetis_build_is(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const float* w,
                              int32_t mem, uint64_t seed, void* stream, thetis_handle** out) {
  return build_graph(KIND_IS, n, m, eu, ev, w, nullptr, 0, nullptr, mem, seed, stream, out);
}
thetis_status thetis_build_mc(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const float* ce,
                              int32_t k, const int32_t* terminals, int32_t mem, uint64_t seed, void* stream,
                              thetis_handle** out) {
  return build_graph(KIND_MC, n, m, eu, ev, nullptr, ce, k, terminals, mem, seed, stream, out);
}

thetis_status thetis_build_sc(int64_t n_elements, int64_t n_sets, const int64_t* set_ptr, const int32_t* set_elems,
                              const float* cost, int32_t mem, uint64_t seed, void* stream, thetis_handle** out) {
  if (!out || !set_ptr || !cost) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  *out = nullptr;
  thetis_handle* h = nullptr;
  thetis_status st = guard(nullptr, [&] {
    TH_CHECK(n_elements >= 1 && n_sets >= 1 && n_elements < (int64_t(1) << 31) && n_sets < (int64_t(1) << 31),
             THETIS_E_INVALID, "need 1 <= n_elements, n_sets < 2^31");
    h = new_handle(stream);
    cudaStream_t s = h->stream;
    Arena tmp(s);
    int64_t ends[2] = {0, 0};
    TH_CUDA(cudaMemcpyAsync(&ends[0], set_ptr, sizeof(int64_t), cudaMemcpyDefault, s));
    TH_CUDA(cudaMemcpyAsync(&ends[1], set_ptr + n_sets, sizeof(int64_t), cudaMemcpyDefault, s));
    TH_CUDA(cudaStreamSynchronize(s));
    const int64_t nnz = ends[1];
    TH_CHECK(ends[0] == 0 && nnz >= 0 && nnz < (int64_t(1) << 31), THETIS_E_INVALID,
             "set_ptr must start at 0 and hold < 2^31 entries");
    TH_CHECK(nnz == 0 || set_elems, THETIS_E_INVALID, "null set_elems");
    const int64_t* dptr = to_dev(set_ptr, n_sets + 1, mem, tmp, s);
    const int32_t* delems = to_dev(set_elems, nnz, mem, tmp, s);
    const float* dcost = to_dev(cost, n_sets, mem, tmp, s);
    RawLP raw;
    int64_t* eptr = nullptr;
    int32_t* esets = nullptr;
    int32_t f = 0;
    build_sc_raw(n_elements, n_sets, nnz, dptr, delems, dcost, raw, eptr, esets, f, tmp, tmp, s);
    h->P = build_problem(raw, KIND_SC, seed, s, tmp);
    Problem& P = *h->P;
    P.nv = n_sets;
    P.ne = n_elements;
    P.sc_f = f;
    P.sc_eptr = keep_copy(P.mem, (const int64_t*)eptr, n_elements + 1, s);
    P.sc_esets = keep_copy(P.mem, (const int32_t*)esets, nnz, s);
    P.w = keep_copy(P.mem, dcost, n_sets, s);
    finish_create(h);
  });
  if (st != THETIS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return THETIS_OK;
}

thetis_status thetis_build_map(int64_t n, int64_t m, int32_t k, const int32_t* eu, const int32_t* ev,
                               const float* theta_node, const float* theta_edge, int32_t mem, uint64_t seed,
                               void* stream, thetis_handle** out) {
  if (!out || !theta_node) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  *out = nullptr;
  thetis_handle* h = nullptr;
  thetis_status st = guard(nullptr, [&] {
    TH_CHECK(n >= 1 && m >= 0 && k >= 2 && k <= 32, THETIS_E_INVALID, "need n >= 1, m >= 0, 2 <= k <= 32");
    TH_CHECK(m == 0 || (eu && ev && theta_edge), THETIS_E_INVALID, "null edge array");
    TH_CHECK(n * (int64_t)k + m * (int64_t)k * k < (int64_t(1) << 31) && 2 * m * (int64_t)k < (int64_t(1) << 31),
             THETIS_E_INVALID, "MAP LP too large");
    h = new_handle(stream);
    cudaStream_t s = h->stream;
    Arena tmp(s);
    const int32_t* deu = to_dev(eu, m, mem, tmp, s);
    const int32_t* dev = to_dev(ev, m, mem, tmp, s);
    const float* dtn = to_dev(theta_node, n * (int64_t)k, mem, tmp, s);
    const float* dte = to_dev(theta_edge, m * (int64_t)k * k, mem, tmp, s);
    RawLP raw;
    build_map_raw(n, m, k, deu, dev, dtn, dte, raw, tmp, s);
    h->P = build_problem(raw, KIND_MAP, seed, s, tmp);
    Problem& P = *h->P;
    P.nv = n;
    P.ne = m;
    P.eu = keep_copy(P.mem, deu, m, s);
    P.ev = keep_copy(P.mem, dev, m, s);
    P.map_tn = keep_copy(P.mem, dtn, n * (int64_t)k, s);
    P.map_te = keep_copy(P.mem, dte, m * (int64_t)k * k, s);
    finish_create(h);
  });
  if (st != THETIS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return THETIS_OK;
}

thetis_status thetis_get_sizes(const thetis_handle* h, int64_t* rows, int64_t* struct_cols, int64_t* slack_cols,
                               int64_t* free_coords, int64_t* nnz, int32_t* ncolors) {
  if (!h || !h->P) {
    set_error("null handle");
    return THETIS_E_INVALID;
  }
  const Problem& P = *h->P;
  if (rows) *rows = P.M;
  if (struct_cols) *struct_cols = P.Ns;
  if (slack_cols) *slack_cols = P.Msl;
  if (free_coords) *free_coords = P.free_coords;
  if (nnz) *nnz = P.nnz + P.Msl;
  if (ncolors) *ncolors = P.ncolors;
  return THETIS_OK;
}

namespace {

// One solve of eq. QP on the handle's current iterate and (ubar, xbar) state:
// sweeps of refresh_every epochs, each followed by the FP64 refresh + checks,
// until rho <= tol (per instance for batches) or the epoch cap.
struct SolveRun {
  bool converged = false;
  int ep = 0;
  double sweep_ms = 0.0;
  int64_t sweep_launches = 0;
  int64_t updates = -1;  // coordinate updates when not epochs * free coordinates (batches)
  CheckOut co{};
};

void solve_run(thetis_handle* h, const SolveArgs& a, bool ub, bool xb, int engine, SolveRun& R) {
  Problem& P = *h->P;
  cudaStream_t s = h->stream;
  if (P.nbatch > 0 && engine == 0 && a.mode == THETIS_MODE_COLORED && !ub && !xb && inst_eligible(P)) {
    // instance-resident engine: every instance solved and stopped on its own
    // (inst.cu); then one FP64 check of the whole batch gives the objective,
    // the infeasibility and every instance's rho at the iterate it stopped at
    batch_inst_begin(P);
    inst_solve(P, a, R.sweep_ms);
    refresh_and_check(P, a, ub, xb, R.co);
    batch_inst_end(P, R.ep, R.converged, R.updates);
    R.sweep_launches = 0;
    for (size_t c = 0; c + 1 < P.h_icls_off.size(); ++c) R.sweep_launches += P.h_icls_off[c + 1] > P.h_icls_off[c];
    R.co.rho = 0.0;  // the largest rho any instance stopped at
    for (double v : P.h_brho) R.co.rho = std::max(R.co.rho, v);
    return;
  }
  if (engine == 2) engine = 0;  // the union sweep, asked for explicitly
  batch_step_rule(P, a);
  if (P.nbatch > 0) {
    TH_CUDA(cudaEventRecord(h->evb, s));
    P.batch_check_ms = 0.0;
  }
  const bool persistent = a.mode == THETIS_MODE_COLORED && engine == 0 && P.ncolors > 0 && coop_allowed() &&
                          sweep_grid(P) > 0;
  if (persistent) reset_sweep_flags(P);
  batch_begin_solve(P);
  if (a.mode == THETIS_MODE_COLORED) ensure_tail(P);
  // per-colour engine: capture one epoch as a CUDA graph (re-captured when its arguments change)
  bool key_ok = P.epoch_graph && h->g_beta == a.beta && h->g_rule == a.step_rule && h->g_mode == a.mode &&
                h->g_ub == (int)ub && h->g_xb == (int)xb && h->g_small == P.small_g && h->g_async == a.async_ctas;
  if (!persistent && !key_ok && a.epochs > 0) {
    if (P.epoch_graph) {
      cudaGraphExecDestroy(P.epoch_graph);
      P.epoch_graph = nullptr;
    }
    cudaGraph_t g;
    TH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    begin_capture_count();
    try {
      run_epoch(P, a, ub, xb);
    } catch (...) {
      end_capture_count();
      cudaStreamEndCapture(s, &g);
      throw;
    }
    h->graph_launches = (int64_t)end_capture_count();  // nothing ran during capture
    TH_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&P.epoch_graph, g, 0);
    cudaGraphDestroy(g);
    TH_CUDA(e);
    h->g_beta = a.beta;
    h->g_rule = a.step_rule;
    h->g_mode = a.mode;
    h->g_ub = ub;
    h->g_xb = xb;
    h->g_small = P.small_g;
    h->g_async = a.async_ctas;
  }
  bool checked_last = false;
  while (R.ep < a.epochs) {
    // epochs up to the next check
    const int chunk = std::min(a.refresh_every - R.ep % a.refresh_every, a.epochs - R.ep);
    TH_CUDA(cudaEventRecord(h->ev2, s));
    if (persistent) {
      run_sweep(P, a, ub, xb, chunk);
      ++R.sweep_launches;
    } else {
      for (int q = 0; q < chunk; ++q) {
        TH_CUDA(cudaGraphLaunch(P.epoch_graph, s));
        count_launch((uint64_t)h->graph_launches);
      }
      R.sweep_launches += (int64_t)chunk * h->graph_launches;
    }
    TH_CUDA(cudaEventRecord(h->ev3, s));
    R.ep += chunk;
    checked_last = false;
    if (R.ep % a.refresh_every == 0 || R.ep == a.epochs) {
      refresh_and_check(P, a, ub, xb, R.co, false);  // rho only; synchronises the stream
      if (persistent && sweep_error(P)) throw Error{THETIS_E_TIMEOUT, "grid barrier of the persistent sweep timed out"};
      float t = 0.f;
      TH_CUDA(cudaEventElapsedTime(&t, h->ev2, h->ev3));
      R.sweep_ms += t;
      checked_last = true;
      if (P.nbatch > 0) {
        float el = 0.f;
        TH_CUDA(cudaEventElapsedTime(&el, h->evb, h->ev3));
        P.batch_check_ms = el;
      }
      // a batch converges instance by instance (each against tol)
      if (P.nbatch > 0 ? batch_after_check(P, a.tol, R.ep) : R.co.rho <= a.tol) {
        R.converged = true;
        break;
      }
    }
  }
  if (!checked_last) {
    refresh_and_check(P, a, ub, xb, R.co);
    R.converged = (P.nbatch > 0) ? batch_after_check(P, a.tol, R.ep) : R.co.rho <= a.tol;
  } else {
    // the last check took rho only: the objective, infeasibility and f_beta
    // of the same (already refreshed) iterate
    CheckOut full{};
    refresh_and_check(P, a, ub, xb, full, true, false);
    R.co.obj = full.obj;
    R.co.infeas = full.infeas;
    R.co.fbeta = full.fbeta;
  }
  if (P.nbatch > 0) {
    batch_end_solve(P, R.ep);
    R.co.rho = 0.0;  // the largest rho any instance stopped at
    for (double v : P.h_brho) R.co.rho = std::max(R.co.rho, v);
  }
}

void check_params(const thetis_params* p) {
  TH_CHECK(p->beta > 0 && std::isfinite(p->beta), THETIS_E_INVALID, "beta must be > 0");
  TH_CHECK(p->epochs >= 0, THETIS_E_INVALID, "epochs must be >= 0");
  TH_CHECK(p->step_rule == 0 || p->step_rule == 1, THETIS_E_INVALID, "step_rule must be 0 or 1");
  TH_CHECK(p->mode == THETIS_MODE_COLORED || p->mode == THETIS_MODE_ASYNC, THETIS_E_INVALID, "bad mode");
  TH_CHECK(p->engine >= 0 && p->engine <= 2, THETIS_E_INVALID, "engine must be 0, 1 or 2");
  TH_CHECK(p->async_ctas >= 0, THETIS_E_INVALID, "async_ctas must be >= 0");
}

void fill_info(const Problem& P, const SolveRun& R, float ms, thetis_solve_info* info) {
  if (!info) return;
  info->epochs_run = R.ep;
  info->converged = R.converged ? 1 : 0;
  info->ncolors = P.ncolors;
  info->rho = R.co.rho;
  info->obj = R.co.obj;
  info->infeas = R.co.infeas;
  info->fbeta = R.co.fbeta;
  info->updates = R.updates >= 0 ? R.updates : (int64_t)R.ep * P.free_coords;
  info->solve_ms = ms;
  info->epoch_ms = R.sweep_ms;
  info->launches_per_epoch = R.ep > 0 ? (int32_t)((R.sweep_launches + R.ep - 1) / R.ep) : 0;
}

}  // namespace

thetis_status thetis_solve(thetis_handle* h, const thetis_params* p, thetis_solve_info* info) {
  if (!h || !h->P || !p) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  SolveRun R;
  thetis_status st = guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    check_params(p);
    SolveArgs a{p->beta, p->epochs, p->tol, p->refresh_every > 0 ? p->refresh_every : 10, p->step_rule, p->mode,
                p->async_ctas};
    Arena tmp(s);
    const float* dub = to_dev(p->ubar, P.M, p->mem, tmp, s);
    const float* dxb = to_dev(p->xbar, P.Ns + P.Msl, p->mem, tmp, s);
    const float* dx0 = to_dev(p->x0, P.Ns, p->mem, tmp, s);
    prepare_solve(P, dub, dxb, dx0);
    refresh_only(P);
    TH_CUDA(cudaEventRecord(h->ev0, s));
    solve_run(h, a, dub != nullptr, dxb != nullptr, p->engine, R);
    TH_CUDA(cudaEventRecord(h->ev1, s));
    TH_CUDA(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    TH_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    fill_info(P, R, ms, info);
  });
  if (st != THETIS_OK) return st;
  return R.converged ? THETIS_OK : THETIS_NOT_CONVERGED;
}

thetis_status thetis_solve_al(thetis_handle* h, const thetis_params* p, int32_t outer, double beta_growth,
                              thetis_solve_info* info, double* infeas_out, double* obj_out, double* rho_out) {
  if (!h || !h->P || !p) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  SolveRun R;
  thetis_status st = guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    check_params(p);
    TH_CHECK(outer >= 1, THETIS_E_INVALID, "outer must be >= 1");
    TH_CHECK(beta_growth >= 1.0 && std::isfinite(beta_growth), THETIS_E_INVALID, "beta_growth must be >= 1");
    TH_CHECK(P.nbatch == 0, THETIS_E_INVALID, "thetis_solve_al takes a single problem");
    SolveArgs a{p->beta, p->epochs, p->tol, p->refresh_every > 0 ? p->refresh_every : 10, p->step_rule, p->mode,
                p->async_ctas};
    Arena tmp(s);
    // ubar and xbar start from the caller's values or from zero
    const float* dub = to_dev(p->ubar, P.M, p->mem, tmp, s);
    const float* dxb = to_dev(p->xbar, P.Ns + P.Msl, p->mem, tmp, s);
    const float* dx0 = to_dev(p->x0, P.Ns, p->mem, tmp, s);
    float* z = nullptr;
    if (!dub || !dxb) {
      z = tmp.alloc<float>(std::max<int64_t>(P.M, P.Ns + P.Msl) + 1);
      TH_CUDA(cudaMemsetAsync(z, 0, (std::max<int64_t>(P.M, P.Ns + P.Msl) + 1) * sizeof(float), s));
    }
    prepare_solve(P, dub ? dub : z, dxb ? dxb : z, dx0);
    refresh_only(P);
    TH_CUDA(cudaEventRecord(h->ev0, s));
    int total = 0;
    double sweep_total = 0.0;
    int64_t launches_total = 0;
    for (int k = 0; k < outer; ++k) {
      R = SolveRun{};
      solve_run(h, a, true, true, p->engine, R);
      total += R.ep;
      sweep_total += R.sweep_ms;
      launches_total += R.sweep_launches;
      if (infeas_out) infeas_out[k] = R.co.infeas;
      if (obj_out) obj_out[k] = R.co.obj;
      if (rho_out) rho_out[k] = R.co.rho;
      al_update(P, a.beta);  // ubar -= beta (Ax - b), xbar <- x, from the last exact refresh
      a.beta *= beta_growth;
    }
    TH_CUDA(cudaEventRecord(h->ev1, s));
    TH_CUDA(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    TH_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    R.ep = total;
    R.sweep_ms = sweep_total;
    R.sweep_launches = launches_total;
    fill_info(P, R, ms, info);
    if (info) info->updates = (int64_t)total * P.free_coords;
  });
  if (st != THETIS_OK) return st;
  return R.converged ? THETIS_OK : THETIS_NOT_CONVERGED;
}

thetis_status thetis_get_duals(thetis_handle* h, float* out, int32_t out_mem) {
  if (!h || !h->P || !out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    TH_CHECK(P.ubar_int != nullptr, THETIS_E_INVALID, "no multiplier estimate: solve with ubar or thetis_solve_al first");
    Arena tmp(h->stream);
    float* d = (out_mem == THETIS_MEM_DEVICE) ? out : tmp.alloc<float>(P.M);
    gather_duals(P, d);
    if (out_mem != THETIS_MEM_DEVICE) from_dev(out, d, P.M, THETIS_MEM_HOST, h->stream);
    TH_CUDA(cudaStreamSynchronize(h->stream));
  });
}

thetis_status thetis_round(thetis_handle* h, int32_t kind, uint64_t seed, int32_t reps, uint8_t* labels_out,
                           int32_t out_mem, thetis_round_info* info) {
  if (!h || !h->P || !labels_out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  RoundOut ro{};
  thetis_status st = guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    Arena tmp(s);
    uint8_t* dl = (out_mem == THETIS_MEM_DEVICE) ? labels_out : tmp.alloc<uint8_t>(P.nv);
    round_problem(P, kind, seed, reps, dl, ro);
    if (ro.status == THETIS_OK && out_mem != THETIS_MEM_DEVICE) from_dev(labels_out, dl, P.nv, THETIS_MEM_HOST, s);
    TH_CUDA(cudaStreamSynchronize(s));
    if (info) {
      info->obj = ro.obj;
      info->repair = ro.repair;
      info->best_rep = ro.best_rep;
      info->near = ro.near;
      info->valid = ro.valid;
    }
  });
  if (st != THETIS_OK) return st;
  if (ro.status != THETIS_OK) {
    set_error("covering repair impossible: eps >= 1");
    if (info) info->repair = ro.repair;
    return (thetis_status)ro.status;
  }
  return THETIS_OK;
}

thetis_status thetis_check_labels(thetis_handle* h, int32_t kind, const uint8_t* labels, int32_t mem,
                                  int32_t* valid_out, double* obj_out) {
  if (!h || !h->P || !labels) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  int valid = 0;
  double obj = 0.0;
  thetis_status st = guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    TH_CHECK(P.kind != KIND_BATCH && P.kind != KIND_GENERAL, THETIS_E_INVALID,
             "thetis_check_labels needs a handle of thetis_build_vc / _is / _mc / _sc / _map");
    Arena tmp(s);
    const uint8_t* dl = to_dev(labels, P.nv, mem, tmp, s);
    check_labels(P, kind, dl, valid, obj);
  });
  if (st != THETIS_OK) return st;
  if (valid_out) *valid_out = valid;
  if (obj_out) *obj_out = obj;
  return THETIS_OK;
}

thetis_status thetis_get_x(thetis_handle* h, float* out, int32_t out_mem) {
  if (!h || !h->P || !out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    Arena tmp(h->stream);
    float* d = (out_mem == THETIS_MEM_DEVICE) ? out : tmp.alloc<float>(P.Ns);
    gather_x_orig(P, d);
    if (out_mem != THETIS_MEM_DEVICE) from_dev(out, d, P.Ns, THETIS_MEM_HOST, h->stream);
    TH_CUDA(cudaStreamSynchronize(h->stream));
  });
}

__global__ void k_gather_slack(const float* s, const uint32_t* slack_orig, int64_t Msl, float* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Msl; t += (int64_t)gridDim.x * blockDim.x)
    out[slack_orig[t]] = s[t];
}

thetis_status thetis_get_slack(thetis_handle* h, float* out, int32_t out_mem) {
  if (!h || !h->P || !out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    if (P.Msl == 0) return;
    Arena tmp(h->stream);
    float* d = (out_mem == THETIS_MEM_DEVICE) ? out : tmp.alloc<float>(P.Msl);
    k_gather_slack<<<grid_for(P.Msl, 256), 256, 0, h->stream>>>(P.s, P.slack_orig, P.Msl, d);
    TH_LAUNCHED();
    if (out_mem != THETIS_MEM_DEVICE) from_dev(out, d, P.Msl, THETIS_MEM_HOST, h->stream);
    TH_CUDA(cudaStreamSynchronize(h->stream));
  });
}

thetis_status thetis_get_colors(thetis_handle* h, int32_t* out, int64_t* n_units) {
  if (!h || !h->P) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    if (n_units) *n_units = P.U;
    if (out && P.U > 0) {
      TH_CUDA(cudaMemcpyAsync(out, P.unit_color, P.U * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
      TH_CUDA(cudaStreamSynchronize(h->stream));
    }
  });
}

thetis_status thetis_sync(thetis_handle* h) {
  if (!h) {
    set_error("null handle");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] { TH_CUDA(cudaStreamSynchronize(h->stream)); });
}

thetis_status thetis_destroy(thetis_handle* h) {
  if (!h) return THETIS_OK;
  delete h;
  return THETIS_OK;
}

thetis_status thetis_cache_info(uint64_t* reserved_bytes, uint64_t* used_bytes) {
  return guard(nullptr, [&] {
    int dev = 0;
    TH_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = lib_pool(dev);
    uint64_t r = 0, u = 0;
    TH_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    TH_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    if (reserved_bytes) *reserved_bytes = r;
    if (used_bytes) *used_bytes = u;
  });
}

thetis_status thetis_trim_cache(uint64_t keep_bytes) {
  return guard(nullptr, [&] {
    int dev = 0;
    TH_CUDA(cudaGetDevice(&dev));
    TH_CUDA(cudaMemPoolTrimTo(lib_pool(dev), (size_t)keep_bytes));
  });
}

namespace {
// In-process cache of tuned launch shapes, keyed by problem shape.
struct TuneKey {
  int kind, log2_coords, avg_nnz, colors_bucket;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, log2_coords, avg_nnz, colors_bucket) <
           std::tie(o.kind, o.log2_coords, o.avg_nnz, o.colors_bucket);
  }
};
std::mutex g_tune_mu;
struct TuneChoice {
  int small_g, per_sm;
  bool full;
};
std::map<TuneKey, TuneChoice> g_tune_cache;

TuneKey tune_key(const Problem& P) {
  int l2 = 0;
  while (l2 < 62 && (int64_t(1) << (l2 + 1)) <= P.free_coords) ++l2;
  int avg = P.Nfree > 0 ? (int)((P.nnz + P.Nfree / 2) / P.Nfree) : 0;
  int cb = 0;
  while (cb < 20 && (1 << (cb + 1)) <= P.ncolors) ++cb;
  return TuneKey{P.kind, l2, avg, cb};
}
}  // namespace

thetis_status thetis_autotune(thetis_handle* h, const thetis_params* p, int32_t trial_epochs,
                              int32_t* small_group_out, int32_t* ctas_per_sm_out) {
  if (!h || !h->P || !p) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    TH_CHECK(p->beta > 0, THETIS_E_INVALID, "beta must be > 0");
    if (P.nbatch > 0 && inst_eligible(P)) {
      // batches: clusters on or off (one thread per short column through ELL
      // panels; the CSR with 8 lanes a column as a third choice), timed on
      // trial_epochs epochs of every instance (no stopping); iterate restored
      TuneKey key = tune_key(P);
      key.kind += 100;
      int G = 0;
      bool clusters = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
          G = it->second.small_g;
          clusters = it->second.full;
        }
      }
      if (G == 0) {
        SolveArgs a{p->beta, std::max(1, trial_epochs), 0.0, 1 << 30, p->step_rule, THETIS_MODE_COLORED};
        Arena tmp(s);
        float* x0 = tmp.alloc<float>(P.Ns);
        float* s0 = tmp.alloc<float>(P.M);
        TH_CUDA(cudaMemcpyAsync(x0, P.x, P.Ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
        if (P.M) TH_CUDA(cudaMemcpyAsync(s0, P.s, P.M * sizeof(float), cudaMemcpyDeviceToDevice, s));
        double best_ms = 1e300;
        const std::pair<int, bool> shapes[3] = {{1, true}, {1, false}, {8, true}};
        for (const auto& sh : shapes) {
          {  // one trial
            const int g = sh.first;
            const bool cl = sh.second;
            P.iml_G = g;
            inst_set_clusters(P, cl);
            double ms = 0.0;
            inst_solve(P, a, ms);
            if (ms < best_ms) {
              best_ms = ms;
              G = g;
              clusters = cl;
            }
            TH_CUDA(cudaMemcpyAsync(P.x, x0, P.Ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
            if (P.M) TH_CUDA(cudaMemcpyAsync(P.s, s0, P.M * sizeof(float), cudaMemcpyDeviceToDevice, s));
          }
        }
        TH_CUDA(cudaStreamSynchronize(s));
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneChoice{G, 0, clusters};
      }
      P.iml_G = G;
      inst_set_clusters(P, clusters);
      if (small_group_out) *small_group_out = G;
      if (ctas_per_sm_out) *ctas_per_sm_out = clusters ? 1 : 0;
      return;
    }
    const TuneKey key = tune_key(P);
    TuneChoice best{P.small_g, P.sweep_per_sm, P.force_full};
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        best = it->second;
        cached = true;
      }
    }
    if (!cached) {
      SolveArgs a{p->beta, std::max(1, trial_epochs), 0.0, 1 << 30, p->step_rule, THETIS_MODE_COLORED};
      Arena tmp(s);
      // the trials move the iterate: keep a copy and put it back after each one
      float* x0 = tmp.alloc<float>(P.Ns);
      float* s0 = tmp.alloc<float>(P.Msl);
      float* r0 = tmp.alloc<float>(P.M);
      TH_CUDA(cudaMemcpyAsync(x0, P.x, P.Ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
      if (P.Msl) TH_CUDA(cudaMemcpyAsync(s0, P.s, P.Msl * sizeof(float), cudaMemcpyDeviceToDevice, s));
      if (P.M) TH_CUDA(cudaMemcpyAsync(r0, P.r, P.M * sizeof(float), cudaMemcpyDeviceToDevice, s));
      prepare_solve(P, nullptr, nullptr, nullptr);
      float best_ms = 1e30f;
      const int groups[4] = {8, 4, 2, 1};
      const int pers[3] = {0, 2, 1};
      const int nvar = sweep_lean_possible(P) ? 2 : 1;
      for (int vi = 0; vi < nvar; ++vi)
      for (int gi = 0; gi < 4; ++gi)
        for (int pi = 0; pi < 3; ++pi) {
          P.force_full = vi == 1;
          P.small_g = groups[gi];
          P.sweep_per_sm = pers[pi];
          P.sweep_grid = -1;
          if (sweep_grid(P) <= 0) continue;
          reset_sweep_flags(P);
          run_sweep(P, a, false, false, 1);  // warm the plan and caches
          TH_CUDA(cudaEventRecord(h->ev2, s));
          run_sweep(P, a, false, false, a.epochs);
          TH_CUDA(cudaEventRecord(h->ev3, s));
          TH_CUDA(cudaEventSynchronize(h->ev3));
          TH_CHECK(sweep_error(P) == 0, THETIS_E_TIMEOUT, "autotune: grid barrier timed out");
          float ms = 0.f;
          TH_CUDA(cudaEventElapsedTime(&ms, h->ev2, h->ev3));
          if (ms < best_ms) {
            best_ms = ms;
            best = {groups[gi], pers[pi], vi == 1};
          }
          TH_CUDA(cudaMemcpyAsync(P.x, x0, P.Ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
          if (P.Msl) TH_CUDA(cudaMemcpyAsync(P.s, s0, P.Msl * sizeof(float), cudaMemcpyDeviceToDevice, s));
          if (P.M) TH_CUDA(cudaMemcpyAsync(P.r, r0, P.M * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
      TH_CUDA(cudaStreamSynchronize(s));
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = best;
    }
    P.small_g = best.small_g;
    P.sweep_per_sm = best.per_sm;
    P.force_full = best.full;
    P.sweep_grid = -1;
    if (small_group_out) *small_group_out = best.small_g;
    if (ctas_per_sm_out) *ctas_per_sm_out = best.per_sm;
  });
}

thetis_status thetis_set_wait_limit(thetis_handle* h, double limit_ms, int32_t missing_ctas) {
  if (!h || !h->P) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  if (!(limit_ms > 0.0 && limit_ms <= 600000.0) || missing_ctas < 0 || missing_ctas > 1024) {
    set_error("limit_ms must be in (0, 600000] and missing_ctas in [0, 1024]");
    return THETIS_E_INVALID;
  }
  h->P->wait_ns = (long long)(limit_ms * 1e6);
  h->P->wait_phantom = (unsigned)missing_ctas;
  return THETIS_OK;
}

thetis_status thetis_set_batch_shape(thetis_handle* h, int32_t lanes_per_column, int32_t clusters) {
  if (!h || !h->P) {
    set_error("null handle");
    return THETIS_E_INVALID;
  }
  if (h->P->kind != KIND_BATCH) {
    set_error("thetis_set_batch_shape needs a handle from thetis_build_batch");
    return THETIS_E_INVALID;
  }
  if (!(lanes_per_column == 1 || lanes_per_column == 4 || lanes_per_column == 8) || clusters < 0 || clusters > 1) {
    set_error("lanes_per_column must be 1, 4 or 8 and clusters 0 or 1");
    return THETIS_E_INVALID;
  }
  h->P->iml_G = lanes_per_column;
  inst_set_clusters(*h->P, clusters != 0);
  return THETIS_OK;
}

thetis_status thetis_set_launch_shape(thetis_handle* h, int32_t small_group, int32_t ctas_per_sm) {
  if (!h || !h->P) {
    set_error("null handle");
    return THETIS_E_INVALID;
  }
  if (!(small_group == 1 || small_group == 2 || small_group == 4 || small_group == 8) || ctas_per_sm < 0) {
    set_error("small_group must be 1, 2, 4 or 8 and ctas_per_sm >= 0");
    return THETIS_E_INVALID;
  }
  h->P->small_g = small_group;
  h->P->sweep_per_sm = ctas_per_sm;
  h->P->sweep_grid = -1;
  return THETIS_OK;
}

thetis_status thetis_build_batch(int32_t count, const uint8_t* kinds, const int64_t* vertex_offset,
                                 const int64_t* edge_offset, const int32_t* eu, const int32_t* ev, const float* w,
                                 int32_t mem, uint64_t seed, void* stream, thetis_handle** out) {
  if (!out || !kinds || !vertex_offset || !edge_offset || !w) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  *out = nullptr;
  thetis_handle* h = nullptr;
  thetis_status st = guard(nullptr, [&] {
    TH_CHECK(count >= 1, THETIS_E_INVALID, "count must be >= 1");
    h = new_handle(stream);
    cudaStream_t s = h->stream;
    Arena tmp(s);
    std::vector<int64_t> hn(count + 1), he(count + 1);
    std::vector<uint8_t> hk(count);
    TH_CUDA(cudaMemcpyAsync(hn.data(), vertex_offset, (count + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
    TH_CUDA(cudaMemcpyAsync(he.data(), edge_offset, (count + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
    TH_CUDA(cudaMemcpyAsync(hk.data(), kinds, count, cudaMemcpyDefault, s));
    TH_CUDA(cudaStreamSynchronize(s));
    TH_CHECK(hn[0] == 0 && he[0] == 0, THETIS_E_INVALID, "offsets must start at 0");
    for (int32_t t = 0; t < count; ++t)
      TH_CHECK(hn[t + 1] > hn[t] && he[t + 1] >= he[t], THETIS_E_INVALID,
               "every instance needs n >= 1 and offsets must not decrease");
    const int64_t Nv = hn[count], Ne = he[count];
    TH_CHECK(Nv < (int64_t(1) << 31) && Ne < (int64_t(1) << 31) && 2 * Ne < (int64_t(1) << 32) - 1,
             THETIS_E_INVALID, "batch too large");
    TH_CHECK(Ne == 0 || (eu && ev), THETIS_E_INVALID, "null edge array");
    const int32_t* deu = to_dev(eu, Ne, mem, tmp, s);
    const int32_t* dev = to_dev(ev, Ne, mem, tmp, s);
    const float* dw = to_dev(w, Nv, mem, tmp, s);
    int64_t* dnoff = tmp.alloc<int64_t>(count + 1);
    int64_t* deoff = tmp.alloc<int64_t>(count + 1);
    uint8_t* dkind = tmp.alloc<uint8_t>(count);
    TH_CUDA(cudaMemcpyAsync(dnoff, hn.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(deoff, he.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(dkind, hk.data(), count, cudaMemcpyHostToDevice, s));
    RawLP raw;
    int32_t *geu = nullptr, *gev = nullptr;
    bool mixed = true;
    build_batch_raw(count, dkind, dnoff, deoff, Nv, Ne, deu, dev, dw, raw, geu, gev, mixed, tmp, s);
    h->P = build_problem(raw, KIND_BATCH, seed, s, tmp);
    Problem& P = *h->P;
    P.nv = Nv;
    P.ne = Ne;
    P.eu = keep_copy(P.mem, (const int32_t*)geu, Ne, s);
    P.ev = keep_copy(P.mem, (const int32_t*)gev, Ne, s);
    P.w = keep_copy(P.mem, dw, Nv, s);
    P.nbatch = count;
    P.bnoff = keep_copy(P.mem, (const int64_t*)dnoff, count + 1, s);
    P.beoff = keep_copy(P.mem, (const int64_t*)deoff, count + 1, s);
    P.bkind = keep_copy(P.mem, (const uint8_t*)dkind, count, s);
    P.h_bkind = hk;
    P.h_bnoff = hn;
    P.h_beoff = he;
    batch_index(P);
    finish_create(h);
  });
  if (st != THETIS_OK) {
    delete h;
    return st;
  }
  *out = h;
  return THETIS_OK;
}

thetis_status thetis_batch_info(const thetis_handle* h, int32_t* epochs_out, double* rho_out) {
  if (!h || !h->P) {
    set_error("null handle");
    return THETIS_E_INVALID;
  }
  const Problem& P = *h->P;
  if (P.kind != KIND_BATCH) {
    set_error("thetis_batch_info needs a handle from thetis_build_batch");
    return THETIS_E_INVALID;
  }
  for (int64_t t = 0; t < P.nbatch; ++t) {
    if (epochs_out) epochs_out[t] = P.h_bepochs[t];
    if (rho_out) rho_out[t] = P.h_brho[t];
  }
  return THETIS_OK;
}

thetis_status thetis_batch_latency(const thetis_handle* h, double* done_ms_out) {
  if (!h || !h->P || !done_ms_out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  const Problem& P = *h->P;
  if (P.kind != KIND_BATCH) {
    set_error("thetis_batch_latency needs a handle from thetis_build_batch");
    return THETIS_E_INVALID;
  }
  for (int64_t t = 0; t < P.nbatch; ++t) done_ms_out[t] = P.h_bdone[t];
  return THETIS_OK;
}

thetis_status thetis_batch_placement(const thetis_handle* h, double* start_ms_out, int32_t* ctas_out) {
  if (!h || !h->P) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  const Problem& P = *h->P;
  if (P.kind != KIND_BATCH) {
    set_error("thetis_batch_placement needs a handle from thetis_build_batch");
    return THETIS_E_INVALID;
  }
  for (int64_t t = 0; t < P.nbatch; ++t) {
    if (start_ms_out) start_ms_out[t] = P.h_bstart[t];
    if (ctas_out) ctas_out[t] = P.h_bctas[t];
  }
  return THETIS_OK;
}

thetis_status thetis_solve_round_batch(thetis_handle* h, const thetis_params* p, uint64_t seed, int32_t reps,
                                       uint8_t* labels_out, int32_t out_mem, double* obj_out, int32_t* status_out,
                                       int32_t* best_rep_out, thetis_solve_info* info) {
  if (!h || !h->P || !p || !labels_out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  Problem& P = *h->P;
  if (P.kind != KIND_BATCH || reps < 1 || reps > 64 || (out_mem != THETIS_MEM_HOST && out_mem != THETIS_MEM_DEVICE)) {
    set_error("thetis_solve_round_batch needs a batch handle, 1 <= reps <= 64 and a valid out_mem");
    return THETIS_E_INVALID;
  }
  // the instance kernels round every instance as it stops; other engines
  // solve, then round the batch as thetis_round_batch
  P.iround_on = true;
  P.iround_done = false;
  P.iround_seed = seed;
  P.iround_reps = reps;
  const thetis_status st = thetis_solve(h, p, info);
  P.iround_on = false;
  if (st != THETIS_OK && st != THETIS_NOT_CONVERGED) return st;
  if (!P.iround_done) {
    const thetis_status rs = thetis_round_batch(h, seed, reps, labels_out, out_mem, obj_out, status_out, best_rep_out);
    return rs != THETIS_OK ? rs : st;
  }
  const thetis_status cs = guard(h->stream, [&] {
    cudaStream_t s = h->stream;
    const int64_t count = P.nbatch;
    from_dev(labels_out, P.i_lab, P.nv, out_mem, s);
    std::vector<double> obj(count);
    std::vector<int32_t> status(count), best(count);
    TH_CUDA(cudaMemcpyAsync(obj.data(), P.i_robj, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaMemcpyAsync(status.data(), P.i_rstatus, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaMemcpyAsync(best.data(), P.i_rbest, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    for (int64_t t = 0; t < count; ++t) {
      if (obj_out) obj_out[t] = obj[t];
      if (status_out) status_out[t] = status[t];
      if (best_rep_out) best_rep_out[t] = best[t];
    }
  });
  return cs != THETIS_OK ? cs : st;
}

thetis_status thetis_round_batch(thetis_handle* h, uint64_t seed, int32_t reps, uint8_t* labels_out,
                                 int32_t out_mem, double* obj_out, int32_t* status_out, int32_t* best_rep_out) {
  if (!h || !h->P || !labels_out) {
    set_error("null argument");
    return THETIS_E_INVALID;
  }
  return guard(h->stream, [&] {
    Problem& P = *h->P;
    cudaStream_t s = h->stream;
    Arena tmp(s);
    uint8_t* dl = (out_mem == THETIS_MEM_DEVICE) ? labels_out : tmp.alloc<uint8_t>(P.nv);
    std::vector<double> obj, repair;
    std::vector<int32_t> status, best;
    std::vector<int64_t> near;
    round_batch(P, seed, reps, dl, obj, status, best, repair, near);
    if (out_mem != THETIS_MEM_DEVICE) from_dev(labels_out, dl, P.nv, THETIS_MEM_HOST, s);
    TH_CUDA(cudaStreamSynchronize(s));
    for (int64_t t = 0; t < P.nbatch; ++t) {
      if (obj_out) obj_out[t] = obj[t];
      if (status_out) status_out[t] = status[t];
      if (best_rep_out) best_rep_out[t] = best[t];
    }
  });
}

}  // extern "C"
