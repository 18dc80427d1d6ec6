// Shared definitions of the CUDA library (sm_103a).  Nothing here is shared
// with the FP64 oracle: the random-number generator below is this library's
// own implementation of splitmix64 from its published definition.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/thetis.h"

namespace thetis {

// ---------------------------------------------------------------------------
// error handling: every entry point converts CUDA errors into THETIS_E_CUDA and
// records a thread-local message.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
const char* get_error();

struct Error {
  thetis_status st;
  std::string msg;
};

#define TH_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      throw ::thetis::Error{THETIS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                               " (" __FILE__ ":" + std::to_string(__LINE__) + ")"}; \
    }                                                                                       \
  } while (0)

#define TH_CHECK(cond, status, msg)                       \
  do {                                                    \
    if (!(cond)) throw ::thetis::Error{(status), (msg)};  \
  } while (0)

// Count of kernel launches made by this library (all threads).
void count_launch(uint64_t n = 1);

// Per host thread: when set, this thread's calls use no cooperative launches
// (the server's worker threads share the GPU through several streams, where
// ordinary launches are the safe choice).
bool coop_allowed();
void set_coop_allowed(bool on);
uint64_t launch_count();
// launches recorded into a stream capture by this thread (not counted until
// the graph is replayed)
void begin_capture_count();
uint64_t end_capture_count();

#define TH_LAUNCHED() ::thetis::count_launch(1)

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood 2014): output i of a generator seeded with s is
// mix(s + (i+1) * 0x9E3779B97F4A7C15).  The rounding streams key three nested
// draws by (rep, stream, index).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t i) {
  return sm64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}
__host__ __device__ __forceinline__ uint64_t rng_u64(uint64_t seed, uint64_t rep, uint64_t stream,
                                                     uint64_t idx) {
  return sm64_at(sm64_at(sm64_at(seed, rep), stream), idx);
}
__host__ __device__ __forceinline__ double rng_unif(uint64_t seed, uint64_t rep, uint64_t stream,
                                                   uint64_t idx) {
  return (double)(rng_u64(seed, rep, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}
enum : uint64_t { STREAM_IS_PICK = 1, STREAM_CKR_RADIUS = 2, STREAM_CKR_PERM = 3, STREAM_SC_PICK = 4 };

// Row index encoding in the internal CSC / CSR of +-1 matrices: bit 31 set means
// the coefficient is -1.
constexpr uint32_t NEG_BIT = 0x80000000u;
__host__ __device__ __forceinline__ uint32_t idx_of(uint32_t e) { return e & 0x7fffffffu; }
__host__ __device__ __forceinline__ float sgn_of(uint32_t e) { return (e & NEG_BIT) ? -1.f : 1.f; }

// ---------------------------------------------------------------------------
// device buffers (stream-ordered allocation on the handle's stream)
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// The library's stream-ordered memory pool on device `dev`, created on first
// use.  Freed blocks stay reserved in it (release threshold = unlimited), so a
// build after a build reuses the same physical memory instead of mapping it
// again; thetis_trim_cache gives the unused reserve back.
cudaMemPool_t lib_pool(int dev);

class Arena {
 public:
  explicit Arena(cudaStream_t s) : s_(s) {}
  ~Arena() { release(); }
  template <class T>
  T* alloc(size_t n) {
    void* p = nullptr;
    size_t b = (n ? n : 1) * sizeof(T);
    if (dev_ < 0) TH_CUDA(cudaStreamGetDevice(s_, &dev_));
    cudaMemPool_t pool = lib_pool(dev_);
    if (cudaMallocFromPoolAsync(&p, b, pool, s_) != cudaSuccess) {
      // the reserve may hold the memory in blocks that do not fit: give the
      // unused part back and try once more
      (void)cudaGetLastError();
      TH_CUDA(cudaStreamSynchronize(s_));
      TH_CUDA(cudaMemPoolTrimTo(pool, 0));
      TH_CUDA(cudaMallocFromPoolAsync(&p, b, pool, s_));
    }
    bufs_.push_back({p, b});
    bytes_ += b;
    return (T*)p;
  }
  void release() {
    for (auto& b : bufs_) cudaFreeAsync(b.p, s_);
    bufs_.clear();
    bytes_ = 0;
  }
  size_t bytes() const { return bytes_; }
  cudaStream_t stream() const { return s_; }

 private:
  cudaStream_t s_;
  int dev_ = -1;
  std::vector<DevBuf> bufs_;
  size_t bytes_ = 0;
};

inline int grid_for(int64_t n, int block, int64_t cap = 152 * 32) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---------------------------------------------------------------------------
// primitives (prims.cu)
// ---------------------------------------------------------------------------
// exclusive scan of int64 counts; out may alias in. Returns nothing; total at out[n].
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& tmp, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, Arena& tmp,
                      cudaStream_t s);
// every segment [ptr[i], ptr[i + 1]) of (keys, vals) sorted by key, stably, in
// place (vals may be null); n = ptr[nseg] < 2^32.  Synchronises the stream.
void segsort_pairs(const int64_t* ptr, int64_t nseg, uint32_t* keys, uint32_t* vals, int64_t n, Arena& tmp,
                   cudaStream_t s);
// out_vals: vals grouped by key (keys < nkeys), ascending inside a group (the
// stable sort by key when vals ascend with position; null vals: the positions
// 0..n-1); out_ptr[nkeys + 1] the groups' starts.  Synchronises the stream.
void group_by_key(const uint32_t* keys, const uint32_t* vals, int64_t n, int64_t nkeys, uint32_t* out_vals,
                  int64_t* out_ptr, Arena& tmp, cudaStream_t s);
void fill_iota_u32(uint32_t* p, int64_t n, cudaStream_t s);
void fill_f32(float* p, float v, int64_t n, cudaStream_t s);

}  // namespace thetis
