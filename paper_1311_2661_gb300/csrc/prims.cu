// Device primitives used while laying a problem out: exclusive scan, a stable
// LSD radix sort of (key, value) pairs, a stable segmented sort and a grouping
// by key built on it.  All are deterministic.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace thetis {

#define GSTRIDE_I(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

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
// stable LSD radix sort, 8-bit digits, 4096-item tiles (512 threads x 8):
// per pass a tile histogram, a digit-major scan of all tiles' counts, and a
// scatter in which each tile first sorts itself by the digit in shared memory
// (two stable 4-bit splits) so that its items of one digit leave as one
// contiguous run
// ---------------------------------------------------------------------------
constexpr int R8_T = 512;
constexpr int R8_I = 8;
constexpr int R8_TILE = R8_T * R8_I;
constexpr int R8_D = 256;
constexpr size_t R8_SMEM = (4 * R8_TILE + 16 * R8_T) * sizeof(uint32_t);

__global__ void __launch_bounds__(R8_T) k_r8_count(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                   int64_t ntiles, int64_t* __restrict__ counts) {
  __shared__ int c[R8_D];
  for (int i = threadIdx.x; i < R8_D; i += R8_T) c[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * R8_TILE;
#pragma unroll
  for (int u = 0; u < R8_I; ++u) {
    const int64_t i = base + u * R8_T + threadIdx.x;
    if (i < n) atomicAdd(&c[(keys[i] >> shift) & (R8_D - 1)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < R8_D; d += R8_T) counts[(int64_t)d * ntiles + blockIdx.x] = c[d];
}

__global__ void __launch_bounds__(R8_T) k_r8_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                     int64_t n, int shift, int64_t ntiles,
                                                     const int64_t* __restrict__ offs) {
  extern __shared__ __align__(16) uint32_t r8[];
  uint32_t* ka = r8;                 // the tile's keys and values, two buffers
  uint32_t* va = r8 + R8_TILE;
  uint32_t* kb = r8 + 2 * R8_TILE;
  uint32_t* vb = r8 + 3 * R8_TILE;
  int* cnt = reinterpret_cast<int*>(r8 + 4 * R8_TILE);  // [16][R8_T]: per 4-bit bin and thread
  __shared__ int tstart[R8_D];
  __shared__ int wsum[R8_T / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * R8_TILE;
  const int nv = (n - base < (int64_t)R8_TILE) ? (int)(n - base) : R8_TILE;
  // the tile in its order; the padding past n takes the largest key, so it
  // sorts behind every item of the last digit and is never written
#pragma unroll
  for (int u = 0; u < R8_I; ++u) {
    const int i = u * R8_T + tid;
    ka[i] = (i < nv) ? kin[base + i] : 0xffffffffu;
    va[i] = (i < nv) ? vin[base + i] : 0u;
  }
  __syncthreads();
  for (int half = 0; half < 2; ++half) {
    const int sh = shift + 4 * half;
    uint32_t* kc = half ? kb : ka;
    uint32_t* vc = half ? vb : va;
    uint32_t* kn = half ? ka : kb;
    uint32_t* vn = half ? va : vb;
    // thread t holds items [8t, 8t + 8) of the current order
    uint32_t k[R8_I], v[R8_I];
    {
      const uint4* k4 = reinterpret_cast<const uint4*>(kc) + 2 * tid;
      const uint4* v4 = reinterpret_cast<const uint4*>(vc) + 2 * tid;
      const uint4 k0 = k4[0], k1 = k4[1], v0 = v4[0], v1 = v4[1];
      k[0] = k0.x; k[1] = k0.y; k[2] = k0.z; k[3] = k0.w; k[4] = k1.x; k[5] = k1.y; k[6] = k1.z; k[7] = k1.w;
      v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w; v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
    }
#pragma unroll
    for (int b = 0; b < 16; ++b) cnt[b * R8_T + tid] = 0;
#pragma unroll
    for (int j = 0; j < R8_I; ++j) cnt[((k[j] >> sh) & 15u) * R8_T + tid] += 1;
    __syncthreads();
    // exclusive scan of cnt in (bin, thread) order: thread t takes entries
    // [16 t, 16 t + 16), then a scan over the threads' totals
    int loc[16];
    int tot = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      loc[i] = tot;
      tot += cnt[16 * tid + i];
    }
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int w = (lane < R8_T / 32) ? wsum[lane] : 0;
      int wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < R8_T / 32) wsum[lane] = wi - w;
    }
    __syncthreads();
    const int pre = wsum[warp] + inc - tot;
#pragma unroll
    for (int i = 0; i < 16; ++i) cnt[16 * tid + i] = pre + loc[i];
    __syncthreads();
    // every item to its place in the order by the 4 bits, stably
#pragma unroll
    for (int j = 0; j < R8_I; ++j) {
      int* slot = &cnt[((k[j] >> sh) & 15u) * R8_T + tid];
      const int pos = *slot;
      *slot = pos + 1;
      kn[pos] = k[j];
      vn[pos] = v[j];
    }
    __syncthreads();
  }
  // ka / va: the tile sorted by the digit; where every digit's run starts
#pragma unroll
  for (int u = 0; u < R8_I; ++u) {
    const int p = u * R8_T + tid;
    const uint32_t d = (ka[p] >> shift) & (R8_D - 1);
    if (p == 0 || ((ka[p - 1] >> shift) & (R8_D - 1)) != d) tstart[d] = p;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < R8_I; ++u) {
    const int p = u * R8_T + tid;
    if (p < nv) {
      const uint32_t d = (ka[p] >> shift) & (R8_D - 1);
      const int64_t pos = offs[(int64_t)d * ntiles + blockIdx.x] + (p - tstart[d]);
      kout[pos] = ka[p];
      vout[pos] = va[p];
    }
  }
}

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, Arena& tmp,
                      cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  static thread_local int attr_dev = -1;
  int dev = 0;
  TH_CUDA(cudaGetDevice(&dev));
  if (attr_dev != dev) {
    TH_CUDA(cudaFuncSetAttribute(k_r8_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R8_SMEM));
    attr_dev = dev;
  }
  const int64_t ntiles = (n + R8_TILE - 1) / R8_TILE;
  int64_t* counts = tmp.alloc<int64_t>(R8_D * ntiles + 1);
  uint32_t* k2 = tmp.alloc<uint32_t>(n);
  uint32_t* v2 = tmp.alloc<uint32_t>(n);
  uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_r8_count<<<(unsigned)ntiles, R8_T, 0, s>>>(ka, n, shift, ntiles, counts);
    TH_LAUNCHED();
    exclusive_scan_i64(counts, counts, R8_D * ntiles, tmp, s);
    k_r8_scatter<<<(unsigned)ntiles, R8_T, R8_SMEM, s>>>(ka, va, kb, vb, n, shift, ntiles, counts);
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

// ---------------------------------------------------------------------------
// segmented sort: each segment [ptr[i], ptr[i+1]) of (keys, vals) sorted by key,
// stably (ties keep their order), in place.  A segment of up to 8 items is
// sorted by one thread in registers (odd-even transposition, which swaps only
// strictly greater neighbours and so is stable); up to 128 by a warp (each
// item's rank by shuffles); up to 4096 by a CTA in shared memory (a bitonic
// network over (key, position)); a longer one is gathered with the other long
// ones into one array sorted by two stable radix sorts (by key, then by
// segment).
// ---------------------------------------------------------------------------
constexpr int SEG_A = 8;
constexpr int SEG_B = 128;
constexpr int SEG_C = 4096;
constexpr int SEG_CT = 128;

// per-thread and per-warp tiers; the segments of the CTA and radix tiers are
// appended to listC / listD (cnt[0], cnt[1]; cnt[2]: items in listD's segments)
__global__ void k_seg_small(const int64_t* __restrict__ ptr, int64_t nseg, int64_t n, uint32_t* keys, uint32_t* vals,
                            int64_t* listC, int64_t capC, int64_t* listD, int64_t capD, unsigned long long* cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nseg; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int64_t p0 = 0;
    int64_t len = 0;
    if (i < nseg) {
      p0 = ptr[i];
      len = ptr[i + 1] - p0;
      if (p0 < 0 || len < 0 || p0 + len > n) {  // not a segment of [0, n): reported, left alone
        atomicOr(&cnt[3], 1ull);
        len = 0;
      }
    }
    if (len > 1 && len <= SEG_A) {
      uint32_t k[SEG_A], v[SEG_A];
#pragma unroll
      for (int u = 0; u < SEG_A; ++u) {
        k[u] = (u < len) ? keys[p0 + u] : 0xffffffffu;
        v[u] = (vals && u < len) ? vals[p0 + u] : 0u;
      }
#pragma unroll
      for (int r = 0; r < SEG_A; ++r) {
#pragma unroll
        for (int j = r & 1; j + 1 < SEG_A; j += 2) {
          if (k[j] > k[j + 1]) {
            const uint32_t tk = k[j], tv = v[j];
            k[j] = k[j + 1];
            v[j] = v[j + 1];
            k[j + 1] = tk;
            v[j + 1] = tv;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < SEG_A; ++u)
        if (u < len) {
          keys[p0 + u] = k[u];
          if (vals) vals[p0 + u] = v[u];
        }
    }
    unsigned mb = __ballot_sync(0xffffffffu, len > SEG_A && len <= SEG_B);
    while (mb) {
      const int l = __ffs(mb) - 1;
      mb &= mb - 1;
      const int64_t q0 = __shfl_sync(0xffffffffu, p0, l);
      const int ql = (int)__shfl_sync(0xffffffffu, len, l);
      // item lane + 32 e of the segment in slot e of this lane
      uint32_t kk[SEG_B / 32], vv[SEG_B / 32];
      int rank[SEG_B / 32];
#pragma unroll
      for (int e = 0; e < SEG_B / 32; ++e) {
        const int t = lane + 32 * e;
        kk[e] = (t < ql) ? keys[q0 + t] : 0xffffffffu;
        vv[e] = (vals && t < ql) ? vals[q0 + t] : 0u;
        rank[e] = 0;
      }
      __syncwarp();  // every lane's loads before any lane's stores
      const int ne = (ql + 31) >> 5;  // slots holding items (warp-uniform)
#pragma unroll
      for (int b = 0; b < SEG_B / 32; ++b) {
        if (b >= ne) break;
        for (int j = 0; j < 32; ++j) {
          const uint32_t kj = __shfl_sync(0xffffffffu, kk[b], j);
          const int tj = j + 32 * b;
#pragma unroll
          for (int e = 0; e < SEG_B / 32; ++e) {
            if (e >= ne) break;  // (warp-uniform) only slots that hold items
            const int t = lane + 32 * e;
            rank[e] += (kj < kk[e] || (kj == kk[e] && tj < t)) ? 1 : 0;
          }
        }
      }
#pragma unroll
      for (int e = 0; e < SEG_B / 32; ++e) {
        if (lane + 32 * e < ql) {
          keys[q0 + rank[e]] = kk[e];
          if (vals) vals[q0 + rank[e]] = vv[e];
        }
      }
      __syncwarp();
    }
    if (len > SEG_B) {
      if (len <= SEG_C) {
        const unsigned long long r = atomicAdd(&cnt[0], 1ull);
        if (r < (unsigned long long)capC) listC[r] = i;
        else atomicOr(&cnt[3], 2ull);
      } else {
        const unsigned long long r = atomicAdd(&cnt[1], 1ull);
        if (r < (unsigned long long)capD) listD[r] = i;
        else atomicOr(&cnt[3], 2ull);
        atomicAdd(&cnt[2], (unsigned long long)len);
      }
    }
  }
}

// CTA tier: a bitonic network over (key, index in the segment) in shared
// memory -- distinct composites, so the result is the stable order
__global__ void __launch_bounds__(SEG_CT) k_seg_cta(const int64_t* __restrict__ ptr, const int64_t* __restrict__ listC,
                                                    const unsigned long long* __restrict__ cnt, uint32_t* keys,
                                                    uint32_t* vals) {
  __shared__ unsigned long long sc[SEG_C];
  __shared__ uint32_t sv[SEG_C];
  const int64_t nC = (cnt[3] != 0) ? 0 : (int64_t)cnt[0];  // nothing on a reported fault
  for (int64_t r = blockIdx.x; r < nC; r += gridDim.x) {
    const int64_t i = listC[r];
    const int64_t p0 = ptr[i];
    const int len = (int)min(ptr[i + 1] - p0, (int64_t)SEG_C);
    int P = 64;
    while (P < len) P <<= 1;
    for (int t = threadIdx.x; t < P; t += SEG_CT) {
      sc[t] = (t < len) ? (((unsigned long long)keys[p0 + t] << 32) | (unsigned)t) : ~0ull;
      if (vals && t < len) sv[t] = vals[p0 + t];
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < (P >> 1); t += SEG_CT) {
          const int a = (t / j) * 2 * j + (t % j), b = a + j;
          const unsigned long long x = sc[a], y = sc[b];
          if ((x > y) == ((a & k) == 0)) {
            sc[a] = y;
            sc[b] = x;
          }
        }
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < len; t += SEG_CT) {
      const unsigned long long c = sc[t];
      keys[p0 + t] = (uint32_t)(c >> 32);
      if (vals) vals[p0 + t] = sv[(uint32_t)c];
    }
    __syncthreads();
  }
}

// radix tier: segment r of listD covers items [coff[r], coff[r + 1]) of the
// gathered array and starts at dp0[r] in place
__device__ __forceinline__ int64_t seg_of(const int64_t* coff, int64_t nD, int64_t c) {
  int64_t lo = 0, hi = nD;  // coff[lo] <= c < coff[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (coff[mid] <= c) lo = mid;
    else hi = mid;
  }
  return lo;
}
__global__ void k_seg_gather(const int64_t* dp0, const int64_t* coff, int64_t nD, const uint32_t* keys,
                             uint32_t* ck, uint32_t* ci) {
  for (int64_t r = blockIdx.x; r < nD; r += gridDim.x) {
    const int64_t a = coff[r], len = coff[r + 1] - a;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
      ck[a + t] = keys[dp0[r] + t];
      ci[a + t] = (uint32_t)(a + t);
    }
  }
}
__global__ void k_seg_keyseg(const int64_t* coff, int64_t nD, int64_t total, const uint32_t* ci, uint32_t* ck) {
  GSTRIDE_I(c, total) ck[c] = (uint32_t)seg_of(coff, nD, ci[c]);
}
__global__ void k_seg_take(const int64_t* dp0, const int64_t* coff, int64_t nD, int64_t total, const uint32_t* ci,
                           const uint32_t* keys, const uint32_t* vals, uint32_t* tk, uint32_t* tv) {
  GSTRIDE_I(c, total) {
    const int64_t r = seg_of(coff, nD, c);  // the gathered array is grouped by segment again
    const int64_t src = dp0[r] + ((int64_t)ci[c] - coff[r]);
    tk[c] = keys[src];
    if (vals) tv[c] = vals[src];
  }
}
__global__ void k_seg_put(const int64_t* dp0, const int64_t* coff, int64_t nD, int64_t total, const uint32_t* tk,
                          const uint32_t* tv, uint32_t* keys, uint32_t* vals) {
  GSTRIDE_I(c, total) {
    const int64_t r = seg_of(coff, nD, c);
    const int64_t dst = dp0[r] + (c - coff[r]);
    keys[dst] = tk[c];
    if (vals) vals[dst] = tv[c];
  }
}
__global__ void k_seg_dinfo(const int64_t* ptr, const int64_t* listD, int64_t nD, int64_t* dp0, int64_t* dlen) {
  GSTRIDE_I(r, nD) {
    dp0[r] = ptr[listD[r]];
    dlen[r] = ptr[listD[r] + 1] - dp0[r];
  }
}

void segsort_pairs(const int64_t* ptr, int64_t nseg, uint32_t* keys, uint32_t* vals, int64_t n, Arena& tmp,
                   cudaStream_t s) {
  if (nseg <= 0 || n <= 1) return;
  TH_CHECK(n < (int64_t(1) << 32), THETIS_E_INVALID, "segmented sort of 2^32 items or more");
  const int64_t capC = n / (SEG_B + 1) + 1, capD = n / (SEG_C + 1) + 1;
  int64_t* listC = tmp.alloc<int64_t>(capC);
  int64_t* listD = tmp.alloc<int64_t>(capD);
  unsigned long long* cnt = tmp.alloc<unsigned long long>(4);  // nC, nD, items of D, fault bits
  TH_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s));
  k_seg_small<<<grid_for(nseg, 256), 256, 0, s>>>(ptr, nseg, n, keys, vals, listC, capC, listD, capD, cnt);
  TH_LAUNCHED();
  k_seg_cta<<<152 * 16, SEG_CT, 0, s>>>(ptr, listC, cnt, keys, vals);
  TH_LAUNCHED();
  unsigned long long hc[4];
  TH_CUDA(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CHECK(hc[3] == 0, THETIS_E_CUDA, "segmented sort: segment offsets outside [0, n)");
  const int64_t nD = (int64_t)hc[1], total = (int64_t)hc[2];
  if (nD == 0) return;
  // the radix tier (segments longer than SEG_C): the gathered layout follows
  // listD's order, whatever it is; each segment's result does not depend on it
  int64_t* dp0 = tmp.alloc<int64_t>(nD);
  int64_t* dlen = tmp.alloc<int64_t>(nD + 1);
  int64_t* coff = tmp.alloc<int64_t>(nD + 1);
  k_seg_dinfo<<<grid_for(nD, 256), 256, 0, s>>>(ptr, listD, nD, dp0, dlen);
  TH_LAUNCHED();
  exclusive_scan_i64(dlen, coff, nD, tmp, s);
  uint32_t* ck = tmp.alloc<uint32_t>(total);
  uint32_t* ci = tmp.alloc<uint32_t>(total);
  uint32_t* tk = tmp.alloc<uint32_t>(total);
  uint32_t* tv = vals ? tmp.alloc<uint32_t>(total) : nullptr;
  k_seg_gather<<<grid_for(nD, 1, 152 * 8), 256, 0, s>>>(dp0, coff, nD, keys, ck, ci);
  TH_LAUNCHED();
  radix_sort_pairs(ck, ci, total, 32, tmp, s);
  int nbits = 0;
  while (nbits < 32 && (int64_t(1) << nbits) < nD) ++nbits;
  k_seg_keyseg<<<grid_for(total, 256), 256, 0, s>>>(coff, nD, total, ci, ck);
  TH_LAUNCHED();
  radix_sort_pairs(ck, ci, total, nbits, tmp, s);
  k_seg_take<<<grid_for(total, 256), 256, 0, s>>>(dp0, coff, nD, total, ci, keys, vals, tk, tv);
  TH_LAUNCHED();
  k_seg_put<<<grid_for(total, 256), 256, 0, s>>>(dp0, coff, nD, total, tk, tv, keys, vals);
  TH_LAUNCHED();
  TH_CUDA(cudaGetLastError());
}

// vals grouped by key (0 <= key < nkeys), ascending inside a group: a stable
// sort by key when vals ascend with their position (null vals: the positions
// themselves).  out_ptr[nkeys + 1]: the groups' starts (and n at the end).
__global__ void k_grp_count(const uint32_t* keys, int64_t n, int64_t nkeys, int64_t* cnt, int* err) {
  GSTRIDE_I(i, n) {
    if (keys[i] < (uint64_t)nkeys) atomicAdd((unsigned long long*)&cnt[keys[i]], 1ull);
    else atomicExch(err, 1);
  }
}
__global__ void k_grp_fill(const uint32_t* keys, const uint32_t* vals, int64_t n, int64_t nkeys, int64_t* cur,
                           uint32_t* out) {
  GSTRIDE_I(i, n) {
    if (keys[i] < (uint64_t)nkeys) out[atomicAdd((unsigned long long*)&cur[keys[i]], 1ull)] = vals ? vals[i] : (uint32_t)i;
  }
}
void group_by_key(const uint32_t* keys, const uint32_t* vals, int64_t n, int64_t nkeys, uint32_t* out_vals,
                  int64_t* out_ptr, Arena& tmp, cudaStream_t s) {
  TH_CUDA(cudaMemsetAsync(out_ptr, 0, (nkeys + 1) * sizeof(int64_t), s));
  int* err = tmp.alloc<int>(1);
  TH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (n > 0) {
    k_grp_count<<<grid_for(n, 256), 256, 0, s>>>(keys, n, nkeys, out_ptr, err);
    TH_LAUNCHED();
  }
  exclusive_scan_i64(out_ptr, out_ptr, nkeys, tmp, s);
  if (n <= 0) return;
  int herr = 0;
  TH_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CHECK(herr == 0, THETIS_E_INVALID, "group by key: a key out of range");
  int64_t* cur = tmp.alloc<int64_t>(nkeys + 1);
  TH_CUDA(cudaMemcpyAsync(cur, out_ptr, (nkeys + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  k_grp_fill<<<grid_for(n, 256), 256, 0, s>>>(keys, vals, n, nkeys, cur, out_vals);
  TH_LAUNCHED();
  segsort_pairs(out_ptr, nkeys, out_vals, nullptr, n, tmp, s);
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
