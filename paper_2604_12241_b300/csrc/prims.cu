// Device primitives: stream-ordered scratch, prefix sums, stable radix sort.
#include <algorithm>
#include <cstring>
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

// ------------------------------------------- copies without the copy engines
//
// The copy engines run transfers one after another, so a cudaMemcpy issued
// on one stream waits behind any bulk transfer another stream has in flight
// (the previous batch's counts on their way back to the host, say).  The
// device-to-device copies of graph building and the few-byte reads the host
// waits for are therefore done by kernels, which do not queue there.

template <typename T>
__global__ void k_copy(const T* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

void copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  const uintptr_t align = (uintptr_t)dst | (uintptr_t)src | (uintptr_t)bytes;
  const unsigned grid = (unsigned)std::min<int64_t>(4 * (int64_t)sm_count(),
                                                    ((int64_t)bytes / 16 + 255) / 256 + 1);
  if (align % 16 == 0) {
    AML_LAUNCH("k_copy", s, k_copy<int4><<<grid, 256, 0, s>>>(
                                static_cast<const int4*>(src), static_cast<int4*>(dst),
                                (int64_t)(bytes / 16)));
  } else if (align % 4 == 0) {
    AML_LAUNCH("k_copy", s, k_copy<int32_t><<<grid, 256, 0, s>>>(
                                static_cast<const int32_t*>(src), static_cast<int32_t*>(dst),
                                (int64_t)(bytes / 4)));
  } else {
    AML_LAUNCH("k_copy", s, k_copy<unsigned char><<<grid, 256, 0, s>>>(
                                static_cast<const unsigned char*>(src),
                                static_cast<unsigned char*>(dst), (int64_t)bytes));
  }
}

struct SmallReadArgs {
  const unsigned char* src[SMALL_READ_MAX];
  uint32_t off[SMALL_READ_MAX];
  uint32_t bytes[SMALL_READ_MAX];
  unsigned char* out;  // device view of mapped host memory
};

__global__ void k_read_small(SmallReadArgs a) {
  const int i = blockIdx.x;
  for (uint32_t b = threadIdx.x; b < a.bytes[i]; b += blockDim.x)
    a.out[a.off[i] + b] = a.src[i][b];
}

void read_small(const SmallRead* r, int n, cudaStream_t s) {
  AML_REQUIRE(n >= 1 && n <= SMALL_READ_MAX, AML_EINTERNAL, "read_small: bad count");
  // one mapped (zero-copy) host buffer per host thread, kept for the process
  thread_local unsigned char* host = nullptr;
  thread_local unsigned char* dev = nullptr;
  if (!host) {
    void* h = nullptr;
    AML_CUDA(cudaHostAlloc(&h, SMALL_READ_BYTES, cudaHostAllocMapped | cudaHostAllocPortable));
    void* d = nullptr;
    AML_CUDA(cudaHostGetDevicePointer(&d, h, 0));
    host = static_cast<unsigned char*>(h);
    dev = static_cast<unsigned char*>(d);
  }
  SmallReadArgs a;
  uint32_t off = 0;
  for (int i = 0; i < n; ++i) {
    a.src[i] = static_cast<const unsigned char*>(r[i].dev);
    a.off[i] = off;
    a.bytes[i] = r[i].bytes;
    off += (r[i].bytes + 15u) & ~15u;
  }
  AML_REQUIRE(off <= SMALL_READ_BYTES, AML_EINTERNAL, "read_small: too many bytes");
  a.out = dev;
  AML_LAUNCH("k_read_small", s, k_read_small<<<n, 32, 0, s>>>(a));
  AML_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) std::memcpy(r[i].host, host + a.off[i], r[i].bytes);
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
// LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.  Per
// pass: (1) every 4096-element tile counts its digits; (2) a digit-major
// exclusive scan of the counts gives each (digit, tile) its output offset;
// (3) every tile ranks its elements stably (inside a warp with
// __match_any_sync, across the block's warps and rounds with digit counts
// in shared memory), places them in shared memory grouped by digit, and
// writes each digit's run out contiguously.

constexpr int RS_BLOCK = 256;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;

__global__ void __launch_bounds__(RS_BLOCK) k_rs_hist(const uint32_t* __restrict__ keys,
                                                      int64_t n, int shift,
                                                      int32_t* __restrict__ hist, int nblocks) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_BLOCK) {
    int64_t j = base + i;
    if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const uint32_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ vals,
                                                         int64_t n, int shift,
                                                         const int32_t* __restrict__ offs,
                                                         int nblocks, uint32_t* __restrict__ okeys,
                                                         uint32_t* __restrict__ ovals) {
  __shared__ uint32_t s_key[RS_TILE];
  __shared__ uint32_t s_val[RS_TILE];
  __shared__ int32_t s_off[256];    // output offset of the tile's run of each digit
  __shared__ int32_t s_start[256];  // start of each digit's run inside the tile
  __shared__ int32_t s_done[256];   // elements of each digit placed so far
  __shared__ int32_t s_w[RS_WARPS][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int tile_n = n - base < RS_TILE ? (int)(n - base) : RS_TILE;
  // the tile's digit counts and run starts (exclusive scan over the digits)
  s_done[tid] = 0;
  __syncthreads();
  for (int i = tid; i < tile_n; i += RS_BLOCK) atomicAdd(&s_done[(keys[base + i] >> shift) & 255u], 1);
  __syncthreads();
  {
    const int c = s_done[tid];
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[0][warp] = x;
    __syncthreads();
    int before = x - c;
    for (int w = 0; w < warp; ++w) before += s_w[0][w];
    s_start[tid] = before;
    s_off[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    __syncthreads();
    s_done[tid] = 0;
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) s_w[w][tid] = 0;
    __syncthreads();
    const int i = r * RS_BLOCK + tid;
    const bool valid = i < tile_n;
    const uint32_t key = valid ? keys[base + i] : 0u;
    const uint32_t val = valid ? vals[base + i] : 0u;
    const uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_w[warp][digit] = __popc(peers);
    __syncthreads();
    int run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const int c = s_w[w][tid];
      s_w[w][tid] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const int at = s_start[digit] + s_done[digit] + s_w[warp][digit] + rank;
      s_key[at] = key;
      s_val[at] = val;
    }
    __syncthreads();
    s_done[tid] += run;
  }
  __syncthreads();
  // consecutive threads write consecutive elements of a digit's run
  for (int i = tid; i < tile_n; i += RS_BLOCK) {
    const uint32_t key = s_key[i];
    const uint32_t digit = (key >> shift) & 255u;
    const int dest = s_off[digit] + (i - s_start[digit]);
    okeys[dest] = key;
    ovals[dest] = s_val[i];
  }
}

void radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                    int64_t n, int nbits, cudaStream_t s) {
  if (n <= 1 || nbits <= 0) return;
  int64_t nb64 = (n + RS_TILE - 1) / RS_TILE;
  AML_REQUIRE(nb64 < (1ll << 31) / 256, AML_EINVAL, "radix sort input too large");
  int nb = (int)nb64;
  DBuf<int32_t> hist((size_t)nb * 256, s);
  uint32_t* ka = keys;
  uint32_t* va = vals;
  uint32_t* kb = keys_tmp;
  uint32_t* vb = vals_tmp;
  for (int shift = 0; shift < nbits; shift += 8) {
    AML_LAUNCH("k_rs_hist", s, k_rs_hist<<<nb, RS_BLOCK, 0, s>>>(ka, n, shift, hist.p, nb));
    scan_i32(hist.p, hist.p, (int64_t)nb * 256, false, s);
    AML_LAUNCH("k_rs_scatter", s,
               k_rs_scatter<<<nb, RS_BLOCK, 0, s>>>(ka, va, n, shift, hist.p, nb, kb, vb));
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    copy_d2d(keys, ka, (size_t)n * sizeof(uint32_t), s);
    copy_d2d(vals, va, (size_t)n * sizeof(uint32_t), s);
  }
}

}  // namespace aml
