// Internal declarations of the B300 AML pattern-counting library.
#pragma once

#include <cuda_runtime.h>

#include <exception>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/aml.h"

namespace aml {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
void clear_error();

struct Failure {
  aml_status status;
  std::string msg;
};

#define AML_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess)                                                          \
      throw ::aml::Failure{_e == cudaErrorMemoryAllocation ? AML_ENOMEM : AML_ECUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(_e)};     \
  } while (0)

#define AML_REQUIRE(cond, st, msg)                         \
  do {                                                     \
    if (!(cond)) throw ::aml::Failure{(st), (msg)};        \
  } while (0)

// Device error word bits (set with atomicOr by kernels, read by aml_sync).
enum : uint32_t {
  ERR_BOUNDS = 1u,    // an index left its buffer (checked builds)
  ERR_TIMEOUT = 2u,   // a bounded wait gave up
  ERR_UNSORTED = 4u,  // timestamps decrease although sorted was promised
  ERR_BAD_ID = 8u,    // a node id outside [0, N)
  ERR_OVERFLOW = 16u, // an internal counter exceeded its range
};

// ------------------------------------------------------- device allocation

// Stream-ordered scratch from the device's default memory pool (kept
// resident by a high release threshold, so steady-state calls reuse it).
void* dalloc(size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t count, cudaStream_t st) : n(count), s(st) {
    p = static_cast<T*>(dalloc(count * sizeof(T) + 16, st));
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    reset();
    p = o.p; n = o.n; s = o.s; o.p = nullptr;
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() {
    // released by an error part-way through enqueueing: work of a side
    // stream may still use it, so wait for the device first
    if (p && std::uncaught_exceptions() > 0) cudaDeviceSynchronize();
    if (p) dfree(p, s);
    p = nullptr;
  }
};

// ----------------------------------------------------------- device graph

// One adjacency direction: rows = accounts, slots sorted by (t, id) inside
// each row; the *n arrays hold the same slots re-sorted by (nbr, t, id).
struct Adj {
  int32_t* ptr = nullptr;   // [N+1] row offsets (row N holds nothing)
  int32_t* rstart = nullptr;  // [Ev] first slot of the slot's row
  int32_t* nbr = nullptr;   // [Ev] counterparty of the slot's edge
  int32_t* t = nullptr;     // [Ev] timestamp
  int32_t* eid = nullptr;   // [Ev] edge id
  int32_t* prev = nullptr;  // [Ev] previous slot of the same row with the same nbr, or -1
  int32_t* next = nullptr;  // [Ev] next such slot, or INT32_MAX
  int32_t* nnbr = nullptr;  // [Ev] (nbr, t, id)-sorted copy: counterparty
  int32_t* nt = nullptr;    //                               timestamp
  int32_t* neid = nullptr;  //                               edge id
  int32_t* pos = nullptr;   // [E] slot of edge e in this direction, -1 for self-loops
};

// Sizes that depend only on the graph and a window, learned on the first
// mine that needs them (one host synchronization) and reused to size the
// buffers of later mines; the contents are recomputed by every mine.
struct LegCache {
  int64_t n_legs = -1;  // temporal 2-paths with s != d in the window (GS instances)
  int64_t n_front[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
                        // cycle-search frontier sizes by level (index = path length)
  int64_t n_wfront[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
                        // the same for the window-cycle search (level 1 = anchors)
  int64_t n_hyb[2][16] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                          {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};
                        // the same for the heavy anchors' legs of the hybrid cycle
                        // search, degree-binned [0] and learned [1]
};

// Runtime tunables of the mining kernels (none changes any count).
struct Tuning {
  int32_t own_max = 32;          // windows up to this long are walked by one lane
  int32_t sg_bucket_mean = 192;  // target leg records per SG bucket
  int32_t close_scan_max = 48;   // closing ranges up to this long are scanned
  int32_t block = 256;           // threads per block of the per-edge kernels
};

// Trained cost model of one window (see mlp.cu / cost.cu).
struct CostModel {
  int32_t delta = -1;
  float* params = nullptr;   // device fp32 parameters, owned by the graph
  float mean[16] = {0};      // feature normalization
  float inv_std[16] = {0};
  float y_mean = 0.f, y_std = 1.f;  // label (log1p cycles) normalization
  float warp_threshold = 0.f;       // predicted cycles at which an item gets a warp
};

// An instantiated CUDA graph of a whole mine, replayed by AML_MINE_GRAPH.
struct MineExec {
  uint32_t flags;     // mining mode it was captured with
  uint64_t ps_id;     // pattern set it was captured for
  uint32_t* counts;   // output pointer baked into it
  int64_t ld;
  uint64_t tune_gen;  // tuning generation it was captured with
  cudaGraphExec_t exec;
  long long n_kernels;  // kernel launches it replays
};

}  // namespace aml

struct aml_graph {
  int64_t E = 0;
  int64_t Ev = 0;  // list edges
  int32_t N = 0;
  int32_t max_out = -1, max_in = -1;  // -1: not read from max_deg yet
  int32_t* max_deg = nullptr;          // device [2]: out, in
  int32_t* src = nullptr;
  int32_t* dst = nullptr;
  int32_t* ts = nullptr;
  float* amount = nullptr;
  int2* dts = nullptr;  // [E] (dst, ts) of every edge: one gather for both
  aml::Adj out, in;
  uint32_t* err = nullptr;  // device error word
  int64_t bytes = 0;
  std::vector<void*> allocs;
  std::map<int32_t, aml::LegCache> legs;  // per window
  cudaStream_t last_stream = nullptr;
  // every caller stream work on this graph was enqueued on (destroy waits
  // for these, not for the whole device)
  std::vector<cudaStream_t> used_streams;
  void note_stream(cudaStream_t s) {
    last_stream = s;
    for (cudaStream_t u : used_streams)
      if (u == s) return;
    used_streams.push_back(s);
  }
  int device = 0;
  // every count above this is reported as this (2^32-1; lowered only by
  // aml_graph_set_count_limit, which tests use to reach the clamp)
  uint32_t count_limit = 0xffffffffu;
  // SM clock cycles a device-side wait of this graph's kernels may take
  // before it gives up (the fused cycle search's grid barriers)
  long long wait_limit = 1ll << 32;
  aml::Tuning tune;
  uint64_t tune_gen = 0;
  std::vector<aml::MineExec> execs;   // captured mines (AML_MINE_GRAPH)
  std::vector<aml::CostModel> cost_models;  // per window (aml_cost_train)
  cudaStream_t capture_stream = nullptr;
  // side streams and fork/join events of a mine's independent branches
  // (created by the first full mine; captured mines use them too)
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t branch_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace aml {

// ------------------------------------------------------------ primitives

// Exclusive (inclusive=false) or inclusive prefix sum of n values.
void scan_i32(const int32_t* in, int32_t* out, int64_t n, bool inclusive, cudaStream_t s);
void scan_i64(const int64_t* in, int64_t* out, int64_t n, bool inclusive, cudaStream_t s);
// Exclusive scan of int32 counts into int64 offsets; total written to *total_dev.
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by key bits [0, nbits).
// Sorted result ends in (keys, vals); tmp buffers must hold n elements.
void radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                    int64_t n, int nbits, cudaStream_t s);

void iota_i32(int32_t* out, int64_t n, cudaStream_t s);
// device-to-device copy by a kernel (no copy engine; see prims.cu)
void copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
// a few small device -> host reads, then waits for `s` (and only `s`): a
// kernel stores the bytes into mapped host memory, so the reads never queue
// behind bulk transfers of other streams on the copy engines
constexpr int SMALL_READ_MAX = 8;
constexpr uint32_t SMALL_READ_BYTES = 512;
struct SmallRead {
  void* host;
  const void* dev;
  uint32_t bytes;
};
void read_small(const SmallRead* r, int n, cudaStream_t s);

// Multiprocessors of the current device (cached per device).
int sm_count();

inline int bits_for(uint64_t max_value) {
  int b = 1;
  while (b < 64 && (max_value >> b) != 0) ++b;
  return b;
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

// ------------------------------------------------------ pattern planning

struct Column {
  int32_t family;  // AML_FAM_*
  int32_t k;       // cycle length
  int32_t delta;
  int32_t prog = -1;  // AML_FAM_PROGRAM: index into the set's programs
};

// A stage program run by the generic interpreter (program.cu): the stages
// of an aml_pattern in a fixed-size form a kernel takes by value.
constexpr int PROG_MAX_STAGES = 8;  // the trigger and up to 7 stages
struct ProgStage {
  int8_t op, a_var, a_dir, b_var, b_dir, out_var, order, window;
  uint32_t skip;
  uint32_t amt;              // AML_AMT_* constraints on the stage's edges
  float amin, amax, rmin, rmax;
};
struct Prog {
  ProgStage st[PROG_MAX_STAGES];
  int32_t n;      // stages, trigger included
  int32_t agg;    // AML_AGG_* (EDGES, DISTINCT or INSTANCES)
  int32_t delta;
  int32_t div;    // INSTANCES counts are divided by it (exactly): the
                  // bindings per instance set of an AML_AGG_SETS column
};

}  // namespace aml

struct aml_pattern_set {
  std::vector<aml::Column> cols;
  std::vector<aml::Prog> progs;  // programs of the AML_FAM_PROGRAM columns
  uint64_t id = 0;  // unique per process, keys captured mines
};

// ---------------------------------------------------------------- helpers

namespace aml {

__device__ __forceinline__ bool before(int32_t tf, int32_t f, int32_t te, int32_t e) {
  return tf < te || (tf == te && f < e);
}

// first i in [lo, hi) with t[i] >= tmin (int64 bound so t - delta cannot wrap)
__device__ __forceinline__ int32_t lower_t(const int32_t* __restrict__ t, int32_t lo, int32_t hi,
                                           int64_t tmin) {
  while (lo < hi) {
    int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    if ((int64_t)__ldg(t + mid) < tmin) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first i in [lo, hi) with t[i] > tmax
__device__ __forceinline__ int32_t upper_t(const int32_t* __restrict__ t, int32_t lo, int32_t hi,
                                           int64_t tmax) {
  while (lo < hi) {
    int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    if ((int64_t)__ldg(t + mid) <= tmax) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first i in [lo, hi) whose edge (t[i], id[i]) comes strictly after (te, e)
__device__ __forceinline__ int32_t after_edge(const int32_t* __restrict__ t,
                                              const int32_t* __restrict__ id, int32_t lo,
                                              int32_t hi, int32_t te, int32_t e) {
  while (lo < hi) {
    int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    int32_t tm = __ldg(t + mid);
    if (tm < te || (tm == te && __ldg(id + mid) <= e)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Paired searches: two bounds of one sorted range found in lockstep.  Each
// step issues both loads before using either, so a pair costs one chain of
// dependent loads instead of two.

// q0 = after_edge(t, id, lo, hi, te, e); q1 = first i in [q0, hi) with
// t[i] > tmax (the window of slots after (te, e) up to tmax)
__device__ __forceinline__ void after_edge_upto(const int32_t* __restrict__ t,
                                                const int32_t* __restrict__ id, int32_t lo,
                                                int32_t hi, int32_t te, int32_t e, int64_t tmax,
                                                int32_t& q0, int32_t& q1) {
  int32_t alo = lo, ahi = hi, blo = lo, bhi = hi;
  while (alo < ahi || blo < bhi) {
    const bool ao = alo < ahi, bo = blo < bhi;
    const int32_t am = (int32_t)(((uint32_t)alo + (uint32_t)ahi) >> 1);
    const int32_t bm = (int32_t)(((uint32_t)blo + (uint32_t)bhi) >> 1);
    const int32_t ta = ao ? __ldg(t + am) : 0;
    const int32_t tb = bo ? __ldg(t + bm) : 0;
    if (ao) {
      if (ta < te || (ta == te && __ldg(id + am) <= e)) alo = am + 1; else ahi = am;
    }
    if (bo) {
      if ((int64_t)tb <= tmax) blo = bm + 1; else bhi = bm;
    }
  }
  q0 = alo;
  q1 = blo > alo ? blo : alo;  // sorted: a later bound below q0 means q0 itself
}

// c0 = lower_t(t, lo, hi, tmin); c1 = first i in [c0, hi) whose edge comes
// strictly after (te, e) (the trailing window up to and including (te, e))
__device__ __forceinline__ void since_upto_edge(const int32_t* __restrict__ t,
                                                const int32_t* __restrict__ id, int32_t lo,
                                                int32_t hi, int64_t tmin, int32_t te, int32_t e,
                                                int32_t& c0, int32_t& c1) {
  int32_t alo = lo, ahi = hi, blo = lo, bhi = hi;
  while (alo < ahi || blo < bhi) {
    const bool ao = alo < ahi, bo = blo < bhi;
    const int32_t am = (int32_t)(((uint32_t)alo + (uint32_t)ahi) >> 1);
    const int32_t bm = (int32_t)(((uint32_t)blo + (uint32_t)bhi) >> 1);
    const int32_t ta = ao ? __ldg(t + am) : 0;
    const int32_t tb = bo ? __ldg(t + bm) : 0;
    if (ao) {
      if ((int64_t)ta < tmin) alo = am + 1; else ahi = am;
    }
    if (bo) {
      if (tb < te || (tb == te && __ldg(id + bm) <= e)) blo = bm + 1; else bhi = bm;
    }
  }
  c0 = alo;
  c1 = blo > alo ? blo : alo;
}

// [r0, r1) = the slots with nbr == x of a range sorted by nbr
__device__ __forceinline__ void nbr_range(const int32_t* __restrict__ nbr, int32_t lo, int32_t hi,
                                          int32_t x, int32_t& r0, int32_t& r1) {
  int32_t alo = lo, ahi = hi, blo = lo, bhi = hi;
  while (alo < ahi || blo < bhi) {
    const bool ao = alo < ahi, bo = blo < bhi;
    const int32_t am = (int32_t)(((uint32_t)alo + (uint32_t)ahi) >> 1);
    const int32_t bm = (int32_t)(((uint32_t)blo + (uint32_t)bhi) >> 1);
    const int32_t na = ao ? __ldg(nbr + am) : 0;
    const int32_t nb = bo ? __ldg(nbr + bm) : 0;
    if (ao) {
      if (na < x) alo = am + 1; else ahi = am;
    }
    if (bo) {
      if (nb <= x) blo = bm + 1; else bhi = bm;
    }
  }
  r0 = alo;
  r1 = blo;
}

// first i in [lo, hi) with nbr[i] >= x
__device__ __forceinline__ int32_t lower_nbr(const int32_t* __restrict__ nbr, int32_t lo,
                                             int32_t hi, int32_t x) {
  while (lo < hi) {
    int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    if (__ldg(nbr + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace aml
