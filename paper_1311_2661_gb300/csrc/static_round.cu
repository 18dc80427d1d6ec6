// Independent-set rounding that performs no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// rounding: a serving loop that must never block on cudaMalloc / cudaFree
// (both can synchronise the whole device), or a process whose memory pool has
// already handed every free byte to another framework's caching allocator.
// thetis_round_is_static serves them: it runs the same kernels as the
// independent-set branch of thetis_round, but every byte of scratch comes from
// one file-scope device array of fixed size.  It still synchronises the
// caller's stream (up to three times) and copies a few words to the host (the
// endpoint check, the best repetition and the info), like thetis_round.
#include <cstring>
#include <mutex>

#include "problem.cuh"

namespace thetis {

// kernels of round.cu (same launch code as thetis_round's independent-set path)
__global__ void k_edge_violation(const float* x, const int32_t* eu, const int32_t* ev, int64_t m, int cover,
                                 unsigned long long* out);
__global__ void k_is_pick(const float* x, int64_t n, int reps, uint64_t seed, const unsigned long long* alpha_bits,
                          uint8_t* pick);
__global__ void k_is_alter(const int32_t* eu, const int32_t* ev, int64_t m, int64_t n, int reps, const uint8_t* pick,
                           uint8_t* keep);
__global__ void k_rep_weight(const uint8_t* sel, const float* w, int64_t n, double* part);
__global__ void k_rep_final(const double* part, int nb, int reps, double* out);
__global__ void k_valid_edges(const uint8_t* lab, const int32_t* eu, const int32_t* ev, int64_t m, int kind, int* bad);
__global__ void k_is_near(const float* x, int64_t n, int rep, uint64_t seed, const unsigned long long* alpha_bits,
                          unsigned long long* near);
// (build.cu) sets *err when an endpoint is outside [0, n) or an edge is a loop
__global__ void k_check_edges(const int32_t* eu, const int32_t* ev, int64_t m, int64_t n, int* err);

namespace {

constexpr int S_RB = 256;      // reduction blocks per repetition (as in round.cu)
constexpr int S_MAX_REPS = 64;
constexpr size_t S_HEADER = 4 * sizeof(unsigned long long) + (size_t)S_RB * S_MAX_REPS * sizeof(double) +
                            S_MAX_REPS * sizeof(double);
constexpr size_t S_BYTES = size_t(64) << 20;  // THETIS_STATIC_SCRATCH_BYTES

// The scratch.  Every GPU that loads the library holds these 64 MiB until the
// process exits.  In host code this name is only a stand-in for the symbol, not
// a device address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[S_BYTES];

std::mutex g_mu;
void* g_addr[64] = {};  // device address of g_scratch per device ordinal

// Looks up the device address of g_scratch on the current device (once per
// device).  The lookup may initialise the module on that device, so the first
// call on a device should not happen inside a stream capture.
void* scratch_on_current_device() {
  int dev = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CHECK(dev >= 0 && dev < 64, THETIS_E_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    TH_CHECK(e == cudaSuccess, THETIS_E_CUDA,
             std::string("cudaGetSymbolAddress(g_scratch): ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

// The arrays must be device memory of the current device (or managed
// memory): the kernels dereference them directly.
void check_device_pointer(const void* p, const char* what) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error{THETIS_E_INVALID, std::string("thetis_round_is_static: ") + what + " is not a CUDA pointer"};
  }
  int dev = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CHECK((a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged, THETIS_E_INVALID,
           std::string("thetis_round_is_static: ") + what + " must be device memory of the current device");
}

}  // namespace
}  // namespace thetis

using namespace thetis;

extern "C" thetis_status thetis_round_is_static(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                                                const float* w, const float* x, uint64_t seed, int32_t reps,
                                                uint8_t* labels_out, thetis_round_info* info, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  try {
    TH_CHECK(n >= 1 && m >= 0 && n < (int64_t(1) << 31) && m < (int64_t(1) << 31), THETIS_E_INVALID,
             "need 1 <= n < 2^31 and 0 <= m < 2^31");
    TH_CHECK(reps >= 1 && reps <= S_MAX_REPS, THETIS_E_INVALID, "reps must be in [1, 64]");
    TH_CHECK(w && x && labels_out && (m == 0 || (eu && ev)), THETIS_E_INVALID, "null array argument");
    check_device_pointer(w, "w");
    check_device_pointer(x, "x");
    check_device_pointer(labels_out, "labels_out");
    if (m > 0) {
      check_device_pointer(eu, "eu");
      check_device_pointer(ev, "ev");
    }
    const size_t need = S_HEADER + 2 * (size_t)n * (size_t)reps;
    TH_CHECK(need <= S_BYTES, THETIS_E_INVALID,
             "thetis_round_is_static: n * reps = " + std::to_string((long long)n * reps) +
                 " exceeds the static scratch limit (2 * n * reps + " + std::to_string(S_HEADER) +
                 " bytes must fit in 64 MiB, i.e. n * reps <= " + std::to_string((S_BYTES - S_HEADER) / 2) + ")");
    unsigned char* base = (unsigned char*)scratch_on_current_device();
    unsigned long long* dbits = (unsigned long long*)base;  // [violation bits, near, edge error, bad]
    int* edge_err = (int*)(dbits + 2);
    int* bad = (int*)(dbits + 3);
    double* part = (double*)(base + 4 * sizeof(unsigned long long));
    double* repv = part + (size_t)S_RB * S_MAX_REPS;
    uint8_t* pick = base + S_HEADER;
    uint8_t* keep = pick + (size_t)n * reps;
    // the scratch keeps the previous call's contents: clear what must start at zero
    TH_CUDA(cudaMemsetAsync(dbits, 0, 4 * sizeof(unsigned long long), s));
    if (m > 0) {
      // every endpoint in [0, n) before any kernel indexes x, keep or labels by it
      k_check_edges<<<grid_for(m, 256), 256, 0, s>>>(eu, ev, m, n, edge_err);
      TH_LAUNCHED();
      int herr = 0;
      TH_CUDA(cudaMemcpyAsync(&herr, edge_err, sizeof(int), cudaMemcpyDeviceToHost, s));
      TH_CUDA(cudaStreamSynchronize(s));
      TH_CHECK(herr == 0, THETIS_E_INVALID, "thetis_round_is_static: edge endpoint outside [0, n), or a loop");
      k_edge_violation<<<grid_for(m, 256, 152 * 8), 256, 0, s>>>(x, eu, ev, m, 0, dbits);
      TH_LAUNCHED();
    }
    k_is_pick<<<grid_for(n * reps, 256), 256, 0, s>>>(x, n, reps, seed, dbits, pick);
    TH_LAUNCHED();
    TH_CUDA(cudaMemcpyAsync(keep, pick, (size_t)n * reps, cudaMemcpyDeviceToDevice, s));
    if (m > 0) {
      k_is_alter<<<grid_for(m * reps, 256), 256, 0, s>>>(eu, ev, m, n, reps, pick, keep);
      TH_LAUNCHED();
    }
    k_rep_weight<<<dim3(S_RB, reps), 256, 0, s>>>(keep, w, n, part);
    TH_LAUNCHED();
    k_rep_final<<<1, S_MAX_REPS, 0, s>>>(part, S_RB, reps, repv);
    TH_LAUNCHED();
    double hv[S_MAX_REPS];
    TH_CUDA(cudaMemcpyAsync(hv, repv, reps * sizeof(double), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    int best = 0;
    for (int r = 1; r < reps; ++r)
      if (hv[r] > hv[best]) best = r;
    TH_CUDA(cudaMemcpyAsync(labels_out, keep + (size_t)best * n, (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_is_near<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(x, n, best, seed, dbits, dbits + 1);
    TH_LAUNCHED();
    if (m > 0) {
      k_valid_edges<<<grid_for(m, 256), 256, 0, s>>>(labels_out, eu, ev, m, KIND_IS, bad);
      TH_LAUNCHED();
    }
    unsigned long long hn[4];
    TH_CUDA(cudaMemcpyAsync(hn, dbits, sizeof(hn), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    TH_CUDA(cudaGetLastError());
    if (info) {
      double alpha;
      std::memcpy(&alpha, &hn[0], sizeof(double));
      info->obj = hv[best];
      info->repair = alpha;
      info->best_rep = best;
      info->near = (int64_t)hn[1];
      info->valid = (hn[3] & 0xffffffffu) ? 0 : 1;
    }
    return THETIS_OK;
  } catch (Error& e) {
    set_error(e.msg);
    if (e.st == THETIS_E_CUDA) {
      cudaStreamSynchronize(s);
      cudaGetLastError();
    }
    return e.st;
  }
}
