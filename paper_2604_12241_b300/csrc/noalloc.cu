// aml_fan_noalloc: the FAN column of one window computed with no device
// allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc (or cudaMallocAsync) at
// the point where they want the feature -- for example code running while a
// CUDA stream capture is active (an allocation there fails or breaks the
// capture), serving processes that reserve their whole device-memory budget
// up front and forbid later allocations, and latency-critical loops that
// cannot afford an allocator call's implicit synchronization.  aml_mine
// allocates its scratch from the stream-ordered pool on every call, so such
// callers use this entry point instead.
//
// The scratch lives in one file-scope __device__ array of fixed size,
// reserved on every GPU that loads the library until the process exits.
#include <cstring>
#include <mutex>

#include "aml_internal.cuh"
#include "mine.cuh"

namespace aml {

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_ITEMS = 8;
constexpr int NA_TILE = NA_BLOCK * NA_ITEMS;                    // 2048 slots per tile
constexpr int64_t NA_MAX_TILES = NA_TILE;                        // partials fit one tile
constexpr int64_t NA_MAX_SLOTS = (int64_t)NA_TILE * NA_MAX_TILES; // 4,194,304 list edges

// [0, MAX_SLOTS): window start per slot; [MAX_SLOTS, 2*MAX_SLOTS): repeat
// deltas, scanned in place; then MAX_TILES tile totals.  32 MiB + 8 KiB.
constexpr int64_t NA_WORDS = 2 * NA_MAX_SLOTS + NA_MAX_TILES;
static __device__ __align__(256) int32_t g_na_scratch[NA_WORDS];

std::mutex g_na_mu;
int32_t* g_na_ptr[64] = {nullptr};  // device address of g_na_scratch, per device

// Resolved once per device, with that device current: in host code the
// array's name is only a host-side stand-in, never a device address.
int32_t* scratch_for_current_device() {
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  AML_REQUIRE(dev >= 0 && dev < 64, AML_EUNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    AML_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    AML_REQUIRE(p != nullptr, AML_ECUDA, "cudaGetSymbolAddress returned NULL");
    g_na_ptr[dev] = static_cast<int32_t*>(p);
  }
  return g_na_ptr[dev];
}

__device__ int32_t na_block_exclusive(int32_t v, int32_t* total) {
  __shared__ int32_t wsum[NA_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < NA_BLOCK / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < NA_BLOCK / 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NA_BLOCK / 32) wsum[lane] = w;
  }
  __syncthreads();
  *total = wsum[NA_BLOCK / 32 - 1];
  int32_t r = (warp ? wsum[warp - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

// tile totals of the deltas
__global__ void __launch_bounds__(NA_BLOCK) k_na_tile_sum(const int32_t* __restrict__ d,
                                                          int64_t n, int32_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * NA_TILE;
  int32_t s = 0;
  for (int i = threadIdx.x; i < NA_TILE; i += NA_BLOCK)
    if (base + i < n) s += d[base + i];
  int32_t tot;
  na_block_exclusive(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// in-place inclusive scan of one tile (nb <= NA_TILE values) seeded with
// `seed` (exclusive prefix of the tiles, or 0) -- used for the tile totals
// (exclusive) and for every data tile (inclusive)
__global__ void __launch_bounds__(NA_BLOCK) k_na_tile_scan(int32_t* __restrict__ d, int64_t n,
                                                           const int32_t* __restrict__ seed,
                                                           int inclusive) {
  __shared__ int32_t s[NA_TILE];
  const int64_t base = (int64_t)blockIdx.x * NA_TILE;
  for (int i = threadIdx.x; i < NA_TILE; i += NA_BLOCK) s[i] = base + i < n ? d[base + i] : 0;
  __syncthreads();
  int32_t loc[NA_ITEMS], sum = 0;
#pragma unroll
  for (int k = 0; k < NA_ITEMS; ++k) {
    loc[k] = s[threadIdx.x * NA_ITEMS + k];
    sum += loc[k];
  }
  int32_t tot;
  int32_t run = na_block_exclusive(sum, &tot) + (seed ? seed[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < NA_ITEMS; ++k) {
    s[threadIdx.x * NA_ITEMS + k] = inclusive ? run + loc[k] : run;
    run += loc[k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NA_TILE; i += NA_BLOCK)
    if (base + i < n) d[base + i] = s[i];
}

// FAN(e) = DEG(e) - repeats(e) for every edge, 0 for self-loops
__global__ void __launch_bounds__(NA_BLOCK) k_na_fan_rows(GraphView g, int dir,
                                                          const int32_t* __restrict__ deg,
                                                          const int32_t* __restrict__ S,
                                                          uint32_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  const int32_t u = g.src[e], v = g.dst[e];
  if (u == v) {
    out[e] = 0u;
    return;
  }
  const int32_t p = dir == AML_DIR_OUT ? g.opos[e] : g.ipos[e];
  const int32_t rs = dir == AML_DIR_OUT ? g.optr[u] : g.iptr[v];
  const int32_t rep = S[p] - (rs > 0 ? S[rs - 1] : 0);
  out[e] = (uint32_t)(deg[p] - rep);
}

}  // namespace

}  // namespace aml

using namespace aml;

extern "C" aml_status aml_fan_noalloc(const aml_graph* g, int32_t delta, int32_t direction,
                                      uint32_t* out, void* stream) {
  try {
    AML_REQUIRE(g != nullptr, AML_EINVAL, "NULL graph");
    AML_REQUIRE(delta >= 0, AML_EINVAL, "delta must be >= 0");
    AML_REQUIRE(direction == AML_DIR_OUT || direction == AML_DIR_IN, AML_EINVAL,
                "direction must be AML_DIR_OUT or AML_DIR_IN");
    AML_REQUIRE(g->E == 0 || out != nullptr, AML_EINVAL, "out is NULL");
    AML_REQUIRE(g->Ev <= NA_MAX_SLOTS, AML_EINVAL,
                "graph has more than 4,194,304 non-loop edges, the scratch limit of "
                "aml_fan_noalloc (use aml_mine)");
    if (g->E == 0) return AML_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* base = scratch_for_current_device();
    int32_t* deg = base;
    int32_t* D = base + NA_MAX_SLOTS;
    int32_t* part = base + 2 * NA_MAX_SLOTS;
    const GraphView gv = view_of(g);
    const Adj& a = direction == AML_DIR_OUT ? g->out : g->in;
    const int64_t Ev = g->Ev;
    // every scratch word read below is first written by this same call, so
    // nothing left over from an earlier call is ever read
    if (Ev > 0) {
      k_window_slots<<<grid_for(Ev, NA_BLOCK), NA_BLOCK, 0, s>>>(
          a.rstart, a.t, a.eid, a.prev, a.next, Ev, delta, deg, D, nullptr);
      AML_CUDA(cudaGetLastError());
      const int64_t nt = (Ev + NA_TILE - 1) / NA_TILE;
      k_na_tile_sum<<<(unsigned)nt, NA_BLOCK, 0, s>>>(D, Ev, part);
      AML_CUDA(cudaGetLastError());
      k_na_tile_scan<<<1, NA_BLOCK, 0, s>>>(part, nt, nullptr, 0);
      AML_CUDA(cudaGetLastError());
      k_na_tile_scan<<<(unsigned)nt, NA_BLOCK, 0, s>>>(D, Ev, part, 1);
      AML_CUDA(cudaGetLastError());
    }
    k_na_fan_rows<<<grid_for(g->E, NA_BLOCK), NA_BLOCK, 0, s>>>(gv, direction, deg, D, out);
    AML_CUDA(cudaGetLastError());
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_fan_noalloc: ") + f.msg);
    return f.status;
  } catch (...) {
    set_error("aml_fan_noalloc: unexpected internal error");
    return AML_EINTERNAL;
  }
}
