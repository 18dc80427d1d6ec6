// Request server: LP-rounding solves submitted one by one, served with
// continuous batching.  Worker threads ("slots") each own a CUDA stream; a free
// worker takes the smallest queued request (the oldest, once a request has
// waited MAX_WAIT_MS) and every other queued vertex-cover / independent-set
// request with the same solve parameters and a similar size (up to max_batch
// and the memory budget) and solves them as one batch (thetis_build_batch +
// thetis_solve_round_batch) on the instance-resident engine: every request is
// solved, rounded and validated by its own CTA (or cluster), which publishes
// its completion to host-mapped memory the moment it finishes, and the worker
// returns that request's result right away while the rest of the batch runs.
// Finished instances free their SMs at once, which the other workers' batches
// (their own streams) take up, so requests that arrive while others are on the
// GPU start as soon as a worker is free and overlap on the device.  Requests
// too large for one CTA or cluster and multiway-cut requests are solved one
// per worker on the whole GPU.  Admission is by an estimate of the device
// bytes a request needs against a fixed budget.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <string>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "problem.cuh"

namespace {

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
  uint64_t id;
  thetis_request q;  // pointers below are owned copies
  std::vector<int32_t> eu, ev, term;
  std::vector<float> w, ce;
  size_t bytes = 0;
  clk::time_point t_submit, t_start, t_done;
  // result
  bool done = false;
  thetis_result res{};
  std::vector<uint8_t> labels;
  std::vector<float> x;
};

// Device bytes a request is expected to need (layout, scratch and the
// colouring's temporaries), used only for admission.
size_t estimate_bytes(const thetis_request& q) {
  const double n = (double)q.n, m = (double)q.m;
  double cols, rows, nnz;
  if (q.kind == THETIS_ROUND_MC) {
    cols = (n + m) * q.k + 2 * m * q.k;
    rows = 2 * m * q.k;
    nnz = 6 * m * q.k + 2 * m * q.k;
  } else {
    cols = n + m;
    rows = m;
    nnz = 3 * m;
  }
  return (size_t)(64.0 * cols + 48.0 * rows + 40.0 * nnz) + (size_t(8) << 20);
}

// Records an error status and the calling thread's error text on a request.
void fail(Req* r, thetis_status st) {
  if (st == THETIS_OK || st == THETIS_NOT_CONVERGED) return;
  r->res.status = st;
  if (r->res.message[0] == 0) std::snprintf(r->res.message, sizeof(r->res.message), "%s", thetis_last_error());
}

constexpr double MAX_WAIT_MS = 10000.0;  // a request waiting longer goes first
constexpr size_t SIZE_RATIO = 4;         // batched requests differ in size by at most this factor

bool same_params(const thetis_request& a, const thetis_request& b) {
  return a.beta == b.beta && a.epochs == b.epochs && a.tol == b.tol && a.refresh_every == b.refresh_every &&
         a.seed == b.seed && a.reps == b.reps;
}

// small enough for one CTA or cluster of the instance-resident engine
bool batchable(const thetis_request& q) { return q.kind != THETIS_ROUND_MC && q.n + q.m <= 200000; }

// Completion flags of a worker in host-mapped pinned memory (written by the
// instance kernels as instances finish) and a stream for reading finished
// instances back while the batch still runs.
struct Slot {
  int* hflags = nullptr;
  int* dflags = nullptr;
  int cap = 0;
  cudaStream_t copy = nullptr;
  int device = 0;
};

}  // namespace

struct thetis_server {
  size_t budget = 0;
  int max_batch = 64;
  size_t max_queued = 0;  // 0: unbounded; else submits beyond it are refused (load shedding)
  int64_t refused = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> all;
  size_t in_flight = 0;
  uint64_t next_id = 1;
  int64_t submitted = 0, completed = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  void work();
  void run_batch(std::vector<Req*>& batch, cudaStream_t s, Slot& slot);
  void run_single(Req* r, cudaStream_t s);
  void finish(Req* r);
};

// a request's result is ready: its latency ends here
void thetis_server::finish(Req* r) {
  std::lock_guard<std::mutex> lk(mu);
  r->t_done = clk::now();
  r->res.queue_ms = ms_between(r->t_submit, r->t_start);
  r->res.service_ms = ms_between(r->t_start, r->t_done);
  r->res.latency_ms = ms_between(r->t_submit, r->t_done);
  r->done = true;
  ++completed;
}

void thetis_server::run_single(Req* r, cudaStream_t s) {
  const thetis_request& q = r->q;
  thetis_handle* h = nullptr;
  thetis_status st;
  if (q.kind == THETIS_ROUND_VC)
    st = thetis_build_vc(q.n, q.m, r->eu.data(), r->ev.data(), r->w.data(), THETIS_MEM_HOST, q.seed, s, &h);
  else if (q.kind == THETIS_ROUND_IS)
    st = thetis_build_is(q.n, q.m, r->eu.data(), r->ev.data(), r->w.data(), THETIS_MEM_HOST, q.seed, s, &h);
  else
    st = thetis_build_mc(q.n, q.m, r->eu.data(), r->ev.data(), r->ce.data(), q.k, r->term.data(), THETIS_MEM_HOST,
                         q.seed, s, &h);
  r->res.batch_size = 1;
  if (st != THETIS_OK) {
    fail(r, st);
    return;
  }
  thetis_params p{};
  p.beta = q.beta;
  p.epochs = q.epochs;
  p.tol = q.tol;
  p.refresh_every = q.refresh_every;
  p.engine = 1;  // ordinary launches: slots share the GPU
  thetis_solve_info si{};
  st = thetis_solve(h, &p, &si);
  r->res.status = st;
  fail(r, st);
  r->res.epochs_run = si.epochs_run;
  r->res.rho = si.rho;
  if (st == THETIS_OK || st == THETIS_NOT_CONVERGED) {
    r->labels.assign((size_t)q.n, 0);
    thetis_round_info ri{};
    thetis_status rs = thetis_round(h, q.kind, q.seed, q.reps, r->labels.data(), THETIS_MEM_HOST, &ri);
    fail(r, rs);
    r->res.obj = ri.obj;
    r->res.valid = ri.valid;
    const int64_t nx = (q.kind == THETIS_ROUND_MC) ? q.n * q.k : q.n;
    std::vector<float> xs;
    int64_t sc = 0;
    thetis_get_sizes(h, nullptr, &sc, nullptr, nullptr, nullptr, nullptr);
    xs.resize((size_t)sc);
    thetis_get_x(h, xs.data(), THETIS_MEM_HOST);
    r->x.assign(xs.begin(), xs.begin() + nx);
  }
  thetis_destroy(h);
}

void thetis_server::run_batch(std::vector<Req*>& batch, cudaStream_t s, Slot& slot) {
  if (batch.size() == 1 && !batchable(batch[0]->q)) {
    run_single(batch[0], s);
    finish(batch[0]);
    return;
  }
  const int32_t count = (int32_t)batch.size();
  std::vector<uint8_t> kinds(count);
  std::vector<int64_t> noff(count + 1, 0), eoff(count + 1, 0);
  for (int32_t t = 0; t < count; ++t) {
    kinds[t] = (uint8_t)batch[t]->q.kind;
    noff[t + 1] = noff[t] + batch[t]->q.n;
    eoff[t + 1] = eoff[t] + batch[t]->q.m;
  }
  std::vector<int32_t> eu(eoff[count]), ev(eoff[count]);
  std::vector<float> w(noff[count]);
  for (int32_t t = 0; t < count; ++t) {
    Req* r = batch[t];
    std::memcpy(eu.data() + eoff[t], r->eu.data(), r->eu.size() * sizeof(int32_t));
    std::memcpy(ev.data() + eoff[t], r->ev.data(), r->ev.size() * sizeof(int32_t));
    std::memcpy(w.data() + noff[t], r->w.data(), r->w.size() * sizeof(float));
  }
  const thetis_request& q = batch[0]->q;
  thetis_handle* h = nullptr;
  thetis_status st = thetis_build_batch(count, kinds.data(), noff.data(), eoff.data(), eu.data(), ev.data(),
                                        w.data(), THETIS_MEM_HOST, q.seed, s, &h);
  for (Req* r : batch) r->res.batch_size = count;
  if (st != THETIS_OK) {
    for (Req* r : batch) {
      fail(r, st);
      finish(r);
    }
    return;
  }
  thetis_params p{};
  p.beta = q.beta;
  p.epochs = q.epochs;
  p.tol = q.tol;
  p.refresh_every = q.refresh_every;
  p.engine = 0;  // instance-resident engine (ordinary launches on this worker's stream)
  // per-request completion: the kernels publish each finished instance
  thetis::Problem* P = thetis::problem_of(h);
  std::vector<char> fin(count, 0);
  bool early = false;
  if (slot.cap >= count && P && thetis::inst_eligible(*P)) {
    try {
      thetis::inst_prepare(*P);
      std::memset(slot.hflags, 0, count * sizeof(int));
      P->i_done = slot.dflags;
      early = true;
    } catch (thetis::Error&) {
      early = false;
    }
  }
  std::atomic<bool> solving{true};
  std::thread poller;
  if (early) {
    poller = std::thread([&] {
      cudaSetDevice(slot.device);
      volatile int* flags = slot.hflags;
      while (true) {
        bool left = false;
        for (int32_t t = 0; t < count; ++t) {
          if (fin[t]) continue;
          if (!flags[t]) {
            left = true;
            continue;
          }
          Req* r = batch[t];
          const int64_t n = r->q.n;
          r->labels.assign((size_t)n, 0);
          r->x.assign((size_t)n, 0.f);
          double obj = 0.0;
          int32_t status = 0, ep = 0, conv = 0;
          float rho = 0.f;
          cudaStream_t c = slot.copy;
          cudaMemcpyAsync(r->labels.data(), P->i_lab + noff[t], n, cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(r->x.data(), P->i_xout + noff[t], n * sizeof(float), cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(&obj, P->i_robj + t, sizeof(double), cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(&status, P->i_rstatus + t, sizeof(int32_t), cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(&ep, P->i_ep + t, sizeof(int32_t), cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(&conv, P->i_conv + t, sizeof(int32_t), cudaMemcpyDeviceToHost, c);
          cudaMemcpyAsync(&rho, P->i_rhoout + t, sizeof(float), cudaMemcpyDeviceToHost, c);
          if (cudaStreamSynchronize(c) != cudaSuccess) {
            (void)cudaGetLastError();
            left = true;  // read it again after the solve
            continue;
          }
          r->res.status = (status == -1) ? THETIS_E_REPAIR : (conv ? THETIS_OK : THETIS_NOT_CONVERGED);
          if (status == -1) std::snprintf(r->res.message, sizeof(r->res.message), "covering repair impossible");
          r->res.obj = obj;
          r->res.valid = status == 1;
          r->res.epochs_run = ep;
          r->res.rho = rho;
          fin[t] = 1;
          finish(r);
          cv.notify_all();
        }
        if (!left || !solving.load()) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    });
  }
  thetis_solve_info si{};
  std::vector<uint8_t> lab(noff[count]);
  std::vector<double> obj(count);
  std::vector<int32_t> status(count), best(count);
  st = thetis_solve_round_batch(h, &p, q.seed, q.reps, lab.data(), THETIS_MEM_HOST, obj.data(), status.data(),
                                best.data(), &si);
  solving = false;
  if (poller.joinable()) poller.join();
  if (P) P->i_done = nullptr;
  std::vector<float> xs(noff[count]);
  thetis_get_x(h, xs.data(), THETIS_MEM_HOST);
  std::vector<int32_t> iep(count, si.epochs_run);
  std::vector<double> irho(count, si.rho);
  thetis_batch_info(h, iep.data(), irho.data());
  for (int32_t t = 0; t < count; ++t) {
    if (fin[t]) continue;
    Req* r = batch[t];
    fail(r, st);
    if (r->res.message[0] == 0) r->res.status = st;
    if (status[t] == -1) r->res.status = THETIS_E_REPAIR;
    // each instance stops at its own check: its status is its own
    if (r->res.message[0] == 0 && st == THETIS_NOT_CONVERGED && irho[t] <= q.tol) r->res.status = THETIS_OK;
    r->res.epochs_run = iep[t];
    r->res.rho = irho[t];
    r->res.obj = obj[t];
    r->res.valid = status[t] == 1;
    r->labels.assign(lab.begin() + noff[t], lab.begin() + noff[t + 1]);
    r->x.assign(xs.begin() + noff[t], xs.begin() + noff[t + 1]);
    finish(r);
  }
  thetis_destroy(h);
}

void thetis_server::work() {
  thetis::set_coop_allowed(false);
  cudaStream_t s = nullptr;
  const cudaError_t se = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (se != cudaSuccess) {
    s = nullptr;
    thetis::set_error(std::string("server worker: cudaStreamCreateWithFlags: ") + cudaGetErrorString(se));
  }
  // completion flags (host-mapped) and the read-back stream; without them the
  // worker returns a batch's results when the batch ends
  Slot slot;
  cudaGetDevice(&slot.device);
  if (cudaHostAlloc((void**)&slot.hflags, (size_t)max_batch * sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
      cudaHostGetDevicePointer((void**)&slot.dflags, slot.hflags, 0) == cudaSuccess &&
      cudaStreamCreateWithFlags(&slot.copy, cudaStreamNonBlocking) == cudaSuccess) {
    slot.cap = max_batch;
  } else {
    (void)cudaGetLastError();
    slot.cap = 0;
  }
  while (true) {
    std::vector<Req*> batch;
    size_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      // head of the next batch: the smallest queued request (shortest job
      // first), or the oldest once it has waited longer than MAX_WAIT_MS
      auto pick = [&]() {
        auto head = queue.begin();
        if (ms_between(queue.front()->t_submit, clk::now()) < MAX_WAIT_MS)
          for (auto it = queue.begin(); it != queue.end(); ++it)
            if ((*it)->bytes < (*head)->bytes) head = it;
        return head;
      };
      cv.wait(lk, [&] { return stop || (!queue.empty() && in_flight + (*pick())->bytes <= budget); });
      if (stop && queue.empty()) break;
      if (queue.empty()) continue;
      auto hi = pick();
      if (in_flight + (*hi)->bytes > budget) continue;
      Req* r0 = *hi;
      queue.erase(hi);
      batch.push_back(r0);
      bytes = r0->bytes;
      if (batchable(r0->q) && max_batch > 1) {
        // same parameters and a similar size (the worker is busy until its slowest instance ends)
        for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < max_batch;) {
          Req* r = *it;
          if (batchable(r->q) && same_params(r->q, r0->q) && r->bytes <= SIZE_RATIO * r0->bytes &&
              r0->bytes <= SIZE_RATIO * r->bytes && in_flight + bytes + r->bytes <= budget) {
            batch.push_back(r);
            bytes += r->bytes;
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      in_flight += bytes;
    }
    const auto t0 = clk::now();
    for (Req* r : batch) r->t_start = t0;
    if (s) {
      run_batch(batch, s, slot);
    } else {  // no stream of its own: every request fails with the reason
      for (Req* r : batch) {
        fail(r, THETIS_E_CUDA);
        finish(r);
      }
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      in_flight -= bytes;
    }
    cv.notify_all();
  }
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (slot.copy) cudaStreamDestroy(slot.copy);
  if (slot.hflags) cudaFreeHost(slot.hflags);
}

extern "C" {

thetis_status thetis_server_create(size_t hbm_budget_bytes, int32_t workers, int32_t max_batch,
                                   thetis_server** out) {
  if (!out || workers < 1 || workers > 64 || max_batch < 1 || hbm_budget_bytes == 0) {
    thetis::set_error("thetis_server_create: need out, 1 <= workers <= 64, max_batch >= 1, budget > 0");
    return THETIS_E_INVALID;
  }
  auto* sv = new thetis_server();
  sv->budget = hbm_budget_bytes;
  sv->max_batch = max_batch;
  for (int i = 0; i < workers; ++i) sv->workers.emplace_back([sv] { sv->work(); });
  *out = sv;
  return THETIS_OK;
}

thetis_status thetis_submit(thetis_server* sv, const thetis_request* q, uint64_t* id) {
  if (!sv || !q || !id) {
    thetis::set_error("null argument");
    return THETIS_E_INVALID;
  }
  if (!(q->kind == THETIS_ROUND_VC || q->kind == THETIS_ROUND_IS || q->kind == THETIS_ROUND_MC) || q->n < 1 ||
      q->m < 0 || (q->m > 0 && (!q->eu || !q->ev)) || q->beta <= 0 || q->epochs < 0 || q->reps < 1 ||
      (q->kind != THETIS_ROUND_MC && !q->w) ||
      (q->kind == THETIS_ROUND_MC && (!q->terminals || q->k < 2 || (q->m > 0 && !q->ce)))) {
    thetis::set_error("thetis_submit: malformed request");
    return THETIS_E_INVALID;
  }
  auto* r = new Req();
  r->q = *q;
  r->eu.assign(q->eu, q->eu + q->m);
  r->ev.assign(q->ev, q->ev + q->m);
  if (q->kind == THETIS_ROUND_MC) {
    r->ce.assign(q->ce, q->ce + q->m);
    r->term.assign(q->terminals, q->terminals + q->k);
  } else {
    r->w.assign(q->w, q->w + q->n);
  }
  r->q.eu = r->q.ev = nullptr;
  r->q.w = r->q.ce = nullptr;
  r->q.terminals = nullptr;
  r->bytes = estimate_bytes(*q);
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r->bytes > sv->budget) {
      delete r;
      thetis::set_error("thetis_submit: request larger than the server's memory budget");
      return THETIS_E_BUDGET;
    }
    if (sv->max_queued && sv->queue.size() >= sv->max_queued) {
      delete r;
      ++sv->refused;
      thetis::set_error("thetis_submit: queue full (the server's queue limit)");
      return THETIS_E_BUDGET;
    }
    r->id = sv->next_id++;
    sv->all[r->id] = r;
    sv->queue.push_back(r);
    ++sv->submitted;
    *id = r->id;
  }
  sv->cv.notify_all();
  return THETIS_OK;
}

thetis_status thetis_poll(thetis_server* sv, uint64_t id, uint8_t* labels_out, float* x_out, thetis_result* out) {
  if (!sv) {
    thetis::set_error("null server");
    return THETIS_E_INVALID;
  }
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    if (it == sv->all.end()) {
      thetis::set_error("thetis_poll: unknown request id");
      return THETIS_E_INVALID;
    }
    if (!it->second->done) return THETIS_PENDING;
    r = it->second;
    sv->all.erase(it);
  }
  if (labels_out && !r->labels.empty()) std::memcpy(labels_out, r->labels.data(), r->labels.size());
  if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), r->x.size() * sizeof(float));
  if (out) *out = r->res;
  delete r;
  return THETIS_OK;
}

thetis_status thetis_server_stats(thetis_server* sv, int64_t* submitted, int64_t* completed, int64_t* queued,
                                  int64_t* in_flight_bytes) {
  if (!sv) {
    thetis::set_error("null server");
    return THETIS_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (submitted) *submitted = sv->submitted;
  if (completed) *completed = sv->completed;
  if (queued) *queued = (int64_t)sv->queue.size();
  if (in_flight_bytes) *in_flight_bytes = (int64_t)sv->in_flight;
  return THETIS_OK;
}

thetis_status thetis_server_set_queue_limit(thetis_server* sv, int64_t max_queued, int64_t* refused_out) {
  if (!sv || max_queued < 0) {
    thetis::set_error("thetis_server_set_queue_limit: need a server and max_queued >= 0");
    return THETIS_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->max_queued = (size_t)max_queued;
  if (refused_out) *refused_out = sv->refused;
  return THETIS_OK;
}

thetis_status thetis_server_destroy(thetis_server* sv) {
  if (!sv) return THETIS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->all) delete kv.second;
  delete sv;
  return THETIS_OK;
}

}  // extern "C"
