// Device primitives used while laying a problem out: exclusive scan and a
// stable LSD radix sort of (key, value) pairs.  Both are deterministic.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace thetis {

cudaMemPool_t lib_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  TH_CHECK(dev >= 0 && dev < 64, THETIS_E_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    TH_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = UINT64_MAX;
    TH_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = p;
  }
  return pools[dev];
}

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* get_error() { return g_err.c_str(); }

static thread_local bool g_coop = true;
bool coop_allowed() { return g_coop; }
void set_coop_allowed(bool on) { g_coop = on; }

static std::atomic<uint64_t> g_launches{0};
// while this thread records a stream capture its launches run later (as graph
// replays): they go to a per-thread tally instead of the global count
static thread_local bool g_capturing = false;
static thread_local uint64_t g_captured = 0;
void count_launch(uint64_t n) {
  if (g_capturing) g_captured += n;
  else g_launches.fetch_add(n, std::memory_order_relaxed);
}
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void begin_capture_count() {
  g_capturing = true;
  g_captured = 0;
}
uint64_t end_capture_count() {
  g_capturing = false;
  return g_captured;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_I = 8;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_I;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[SCAN_T / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t s = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
    int64_t si = warp_incl_scan(s);
    if (lane < (int)(blockDim.x >> 5)) wsum[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  int64_t r = inc - v + wsum[w];
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t s = 0;
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + (int64_t)i * SCAN_T + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  __shared__ int64_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                             int64_t* __restrict__ out, int64_t* __restrict__ total_out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_I;
  int64_t v[SCAN_I];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + i;
    v[i] = (idx < n) ? in[idx] : 0;
    s += v[i];
  }
  __shared__ int64_t tot;
  int64_t pre = block_excl_scan(s, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = pre;
    pre += v[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *total_out = pre;
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& tmp, cudaStream_t s) {
  // out must have n+1 entries; out[n] receives the total.
  int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb <= 1) {
    k_scan_apply<<<1, SCAN_T, 0, s>>>(in, n, nullptr, out, out + n);
    TH_LAUNCHED();
    TH_CUDA(cudaGetLastError());
    return;
  }
  int64_t* sums = tmp.alloc<int64_t>(nb + 1);
  k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, sums);
  TH_LAUNCHED();
  exclusive_scan_i64(sums, sums, nb, tmp, s);
  k_scan_apply<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, sums, out, out + n);
  TH_LAUNCHED();
  TH_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 4-bit digits, one item per thread, 512-item tiles
// ---------------------------------------------------------------------------
constexpr int RS_T = 512;
constexpr int RS_W = RS_T / 32;
constexpr int RS_D = 16;

__global__ void k_rs_count(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
                           int64_t* __restrict__ counts) {
  __shared__ int c[RS_D];
  if (threadIdx.x < RS_D) c[threadIdx.x] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * RS_T + threadIdx.x;
  if (i < n) atomicAdd(&c[(keys[i] >> shift) & (RS_D - 1)], 1);
  __syncthreads();
  if (threadIdx.x < RS_D) counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                             int shift, int64_t ntiles, const int64_t* __restrict__ offs) {
  __shared__ int wc[RS_W][RS_D];
  __shared__ int wp[RS_W][RS_D];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < RS_W * RS_D; t += RS_T) (&wc[0][0])[t] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * RS_T + threadIdx.x;
  bool valid = i < n;
  uint32_t k = valid ? kin[i] : 0u;
  uint32_t v = valid ? vin[i] : 0u;
  int d = valid ? (int)((k >> shift) & (RS_D - 1)) : RS_D;
  unsigned peers = __match_any_sync(0xffffffffu, d);
  int rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) wc[w][d] = __popc(peers);
  __syncthreads();
  if (threadIdx.x < RS_D) {
    int acc = 0;
    for (int q = 0; q < RS_W; ++q) {
      wp[q][threadIdx.x] = acc;
      acc += wc[q][threadIdx.x];
    }
  }
  __syncthreads();
  if (valid) {
    int64_t pos = offs[(int64_t)d * ntiles + blockIdx.x] + wp[w][d] + rank;
    kout[pos] = k;
    vout[pos] = v;
  }
}

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, Arena& tmp,
                      cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  int64_t ntiles = (n + RS_T - 1) / RS_T;
  int64_t* counts = tmp.alloc<int64_t>(RS_D * ntiles + 1);
  uint32_t* k2 = tmp.alloc<uint32_t>(n);
  uint32_t* v2 = tmp.alloc<uint32_t>(n);
  uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
  int passes = (bits + 3) / 4;
  for (int p = 0; p < passes; ++p) {
    int shift = 4 * p;
    k_rs_count<<<(unsigned)ntiles, RS_T, 0, s>>>(ka, n, shift, ntiles, counts);
    TH_LAUNCHED();
    exclusive_scan_i64(counts, counts, RS_D * ntiles, tmp, s);
    k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, counts);
    TH_LAUNCHED();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    TH_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    TH_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  TH_CUDA(cudaGetLastError());
}

__global__ void k_iota(uint32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}
__global__ void k_fill_f32(float* p, float v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
void fill_iota_u32(uint32_t* p, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_iota<<<grid_for(n, 256), 256, 0, s>>>(p, n);
  TH_LAUNCHED();
}
void fill_f32(float* p, float v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill_f32<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
  TH_LAUNCHED();
}

}  // namespace thetis
