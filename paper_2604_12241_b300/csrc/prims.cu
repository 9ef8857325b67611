// Device primitives: stream-ordered scratch, prefix sums, stable radix sort.
#include <algorithm>
#include <mutex>
#include <set>

#include "aml_internal.cuh"
#include "profile.cuh"

namespace aml {

// ------------------------------------------------------------- allocation

void* dalloc(size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static std::set<int> ready;
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready.count(dev)) {
      // keep freed blocks in the pool so repeated calls do not return memory
      // to the driver between mines
      cudaMemPool_t pool;
      AML_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
      uint64_t thr = UINT64_MAX;
      AML_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
      ready.insert(dev);
    }
  }
  void* p = nullptr;
  AML_CUDA(cudaMallocAsync(&p, bytes ? bytes : 16, s));
  return p;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------------ iota

__global__ void k_iota(int32_t* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)i;
}

void iota_i32(int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  AML_LAUNCH("k_iota", s, k_iota<<<grid_for(n, 256), 256, 0, s>>>(out, n));
}

// ------------------------------------------------------------- prefix sum
//
// Tiles of SCAN_TILE values are staged through shared memory so global loads
// and stores stay coalesced; one tile is scanned by k_tile_scan, more by the
// single-pass k_scan_lookback below.

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

// Shared-memory index of tile element i with one pad element per 128 bytes:
// thread t then reads its SCAN_ITEMS consecutive elements without bank
// conflicts (t * SCAN_ITEMS alone maps a warp onto 4 banks).
template <typename T>
__device__ __forceinline__ int spad(int i) {
  return i + (i >> (sizeof(T) == 8 ? 4 : 5));
}
template <typename T>
constexpr int scan_smem_elems() {
  return SCAN_TILE + SCAN_TILE / (sizeof(T) == 8 ? 16 : 32);
}

template <typename T>
__device__ T block_exclusive_sum(T v, T* total) {
  __shared__ T warp_tot[SCAN_BLOCK / 32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < SCAN_BLOCK / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < SCAN_BLOCK / 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_BLOCK / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  T warp_off = warp ? warp_tot[warp - 1] : T(0);
  *total = warp_tot[SCAN_BLOCK / 32 - 1];
  T r = warp_off + x - v;
  __syncthreads();  // warp_tot may be reused by the caller's next call
  return r;
}

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(SCAN_BLOCK) k_tile_scan(const Tin* __restrict__ in, Tacc* out,
                                                          int64_t n, const Tacc* tile_off,
                                                          bool inclusive) {
  __shared__ Tacc s[scan_smem_elems<Tacc>()];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BLOCK) {
    int64_t j = base + i;
    s[spad<Tacc>(i)] = j < n ? (Tacc)in[j] : Tacc(0);
  }
  __syncthreads();
  Tacc loc[SCAN_ITEMS];
  Tacc sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    loc[k] = s[spad<Tacc>(threadIdx.x * SCAN_ITEMS + k)];
    sum += loc[k];
  }
  Tacc tot;
  Tacc run = block_exclusive_sum<Tacc>(sum, &tot);
  if (tile_off) run += tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    Tacc v = loc[k];
    s[spad<Tacc>(threadIdx.x * SCAN_ITEMS + k)] = inclusive ? run + v : run;
    run += v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BLOCK) {
    int64_t j = base + i;
    if (j < n) out[j] = s[spad<Tacc>(i)];
  }
}

// Larger inputs: reduce-then-scan over one contiguous chunk per block, with
// about as many blocks as the GPU holds at once.  k_chunk_reduce writes each
// chunk's total; k_chunk_scan sums the totals before its chunk (a few
// thousand values, read by every block) and scans its chunk tile by tile,
// carrying the running sum.  Two launches, no inter-block waits; the input
// is read twice.

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(SCAN_BLOCK) k_chunk_reduce(const Tin* __restrict__ in,
                                                             int64_t n, int64_t chunk,
                                                             Tacc* __restrict__ partial) {
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  Tacc sum = 0;
  for (int64_t j = lo + threadIdx.x; j < hi; j += SCAN_BLOCK) sum += (Tacc)in[j];
  Tacc tot;
  block_exclusive_sum<Tacc>(sum, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(SCAN_BLOCK) k_chunk_scan(const Tin* __restrict__ in, Tacc* out,
                                                           int64_t n, int64_t chunk,
                                                           const Tacc* __restrict__ partial,
                                                           bool inclusive) {
  __shared__ Tacc s[scan_smem_elems<Tacc>()];
  // offset of this chunk: the totals of the chunks before it
  Tacc pre = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_BLOCK) pre += partial[b];
  Tacc carry;
  block_exclusive_sum<Tacc>(pre, &carry);
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int64_t base = lo; base < hi; base += SCAN_TILE) {
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BLOCK) {
      const int64_t j = base + i;
      s[spad<Tacc>(i)] = j < hi ? (Tacc)in[j] : Tacc(0);
    }
    __syncthreads();
    Tacc loc[SCAN_ITEMS];
    Tacc sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      loc[k] = s[spad<Tacc>(threadIdx.x * SCAN_ITEMS + k)];
      sum += loc[k];
    }
    Tacc tot;
    Tacc run = carry + block_exclusive_sum<Tacc>(sum, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      const Tacc v = loc[k];
      s[spad<Tacc>(threadIdx.x * SCAN_ITEMS + k)] = inclusive ? run + v : run;
      run += v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BLOCK) {
      const int64_t j = base + i;
      if (j < hi) out[j] = s[spad<Tacc>(i)];
    }
    carry += tot;
    __syncthreads();  // s is refilled by the next tile
  }
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && cached[dev]) return cached[dev];
  int sms = 0;
  AML_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  sms = std::max(sms, 1);
  if (dev < 64) cached[dev] = sms;
  return sms;
}

// blocks the GPU holds at once (8 scan blocks per SM)
static int64_t resident_scan_blocks() { return 8 * (int64_t)sm_count(); }

template <typename Tin, typename Tacc>
static void scan_impl(const Tin* in, Tacc* out, int64_t n, bool inclusive, cudaStream_t s) {
  if (n <= 0) return;
  if (n <= SCAN_TILE) {
    AML_LAUNCH("k_tile_scan", s,
               k_tile_scan<Tin, Tacc><<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr, inclusive));
    return;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  const int64_t nblk0 = std::min<int64_t>(tiles, resident_scan_blocks());
  const int64_t chunk = (tiles + nblk0 - 1) / nblk0 * SCAN_TILE;  // whole tiles per block
  const int64_t nblk = (n + chunk - 1) / chunk;
  DBuf<Tacc> part((size_t)nblk, s);
  AML_LAUNCH("k_chunk_reduce", s,
             k_chunk_reduce<Tin, Tacc><<<(unsigned)nblk, SCAN_BLOCK, 0, s>>>(in, n, chunk,
                                                                             part.p));
  AML_LAUNCH("k_chunk_scan", s,
             k_chunk_scan<Tin, Tacc><<<(unsigned)nblk, SCAN_BLOCK, 0, s>>>(in, out, n, chunk,
                                                                           part.p, inclusive));
}

void scan_i32(const int32_t* in, int32_t* out, int64_t n, bool inclusive, cudaStream_t s) {
  scan_impl<int32_t, int32_t>(in, out, n, inclusive, s);
}
void scan_i64(const int64_t* in, int64_t* out, int64_t n, bool inclusive, cudaStream_t s) {
  scan_impl<int64_t, int64_t>(in, out, n, inclusive, s);
}
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl<int32_t, int64_t>(in, out, n, false, s);
}

// ------------------------------------------------------------ radix sort
//
// LSD radix sort, 8-bit digits.  Per pass: (1) every 4096-element tile
// counts its digits; (2) digit-major exclusive scan of the counts gives each
// (digit, tile) its output offset; (3) every tile re-reads its elements in
// order and ranks equal digits stably: inside a warp with __match_any_sync,
// across the block's warps with per-warp digit counts in shared memory.

constexpr int RS_BLOCK = 256;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;

template <typename K>
__global__ void __launch_bounds__(RS_BLOCK) k_rs_hist(const K* __restrict__ keys, int64_t n,
                                                      int shift, int32_t* __restrict__ hist,
                                                      int nblocks) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_BLOCK) {
    int64_t j = base + i;
    if (j < n) atomicAdd(&h[(uint32_t)(keys[j] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const K* __restrict__ keys,
                                                         const uint32_t* __restrict__ vals,
                                                         int64_t n, int shift,
                                                         const int32_t* __restrict__ offs,
                                                         int nblocks, K* __restrict__ okeys,
                                                         uint32_t* __restrict__ ovals) {
  __shared__ int32_t s_off[256];
  __shared__ int32_t s_w[RS_WARPS][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_off[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) s_w[w][tid] = 0;
    __syncthreads();
    const int64_t j = base + (int64_t)r * RS_BLOCK + tid;
    const bool valid = j < n;
    K key = valid ? keys[j] : K(0);
    uint32_t val = valid ? vals[j] : 0u;
    uint32_t digit = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_w[warp][digit] = __popc(peers);
    __syncthreads();
    int run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      int c = s_w[w][tid];
      s_w[w][tid] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      int dest = s_off[digit] + s_w[warp][digit] + rank;
      okeys[dest] = key;
      ovals[dest] = val;
    }
    __syncthreads();
    s_off[tid] += run;
  }
}

template <typename K>
static void radix_impl(K* keys, uint32_t* vals, K* keys_tmp, uint32_t* vals_tmp, int64_t n,
                       int nbits, cudaStream_t s) {
  if (n <= 1 || nbits <= 0) return;
  int64_t nb64 = (n + RS_TILE - 1) / RS_TILE;
  AML_REQUIRE(nb64 < (1ll << 31) / 256, AML_EINVAL, "radix sort input too large");
  int nb = (int)nb64;
  DBuf<int32_t> hist((size_t)nb * 256, s);
  K* ka = keys;
  uint32_t* va = vals;
  K* kb = keys_tmp;
  uint32_t* vb = vals_tmp;
  for (int shift = 0; shift < nbits; shift += 8) {
    AML_LAUNCH("k_rs_hist", s, k_rs_hist<K><<<nb, RS_BLOCK, 0, s>>>(ka, n, shift, hist.p, nb));
    scan_i32(hist.p, hist.p, (int64_t)nb * 256, false, s);
    AML_LAUNCH("k_rs_scatter", s,
               k_rs_scatter<K><<<nb, RS_BLOCK, 0, s>>>(ka, va, n, shift, hist.p, nb, kb, vb));
    K* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    AML_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, s));
    AML_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
}

void radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                    int64_t n, int nbits, cudaStream_t s) {
  radix_impl<uint32_t>(keys, vals, keys_tmp, vals_tmp, n, nbits, s);
}

void radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_tmp, uint32_t* vals_tmp,
                    int64_t n, int nbits, cudaStream_t s) {
  radix_impl<uint64_t>(keys, vals, keys_tmp, vals_tmp, n, nbits, s);
}

}  // namespace aml
