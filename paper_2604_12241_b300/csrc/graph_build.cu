// Device graph construction (aml_graph_create / aml_graph_destroy).
//
// Every list is built with stable radix sorts from the global (t, id) order,
// so each account's out-list (CSR) and in-list (CSC) is sorted by (t, id):
// a time window is a contiguous slot range found by binary search (the
// paper's Find_Starting_Edge, Alg. 1; sorted lists + binary search, Sec. 6).
// A second copy of every row sorted by (counterparty, t, id) answers "edges
// x->y inside a time range" with two nested binary searches, and links each
// slot to the previous / next slot of its row with the same counterparty.
#include <climits>
#include <cstring>

#include "aml_internal.cuh"
#include "profile.cuh"

namespace aml {

__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const int32_t* __restrict__ ts, int64_t E, int32_t N,
                           uint32_t* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  uint32_t bits = 0;
  int32_t s = src[i], d = dst[i];
  if (s < 0 || s >= N || d < 0 || d >= N) bits |= ERR_BAD_ID;
  if (i + 1 < E && ts[i] > ts[i + 1]) bits |= ERR_UNSORTED;
  bits = __reduce_or_sync(0xffffffffu & __activemask(), bits);
  if (bits && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicOr(err, bits);
}

__global__ void k_time_keys(const int32_t* __restrict__ ts, int64_t E,
                            uint32_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) keys[i] = (uint32_t)ts[i] ^ 0x80000000u;  // signed order as unsigned
}

// key of the row holding edge perm[i]: its account, or N for a self-loop
__global__ void k_row_keys(const uint32_t* __restrict__ perm, const int32_t* __restrict__ row_of,
                           const int32_t* __restrict__ other, int64_t E, int32_t N,
                           uint32_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  uint32_t e = perm[i];
  int32_t r = row_of[e], o = other[e];
  keys[i] = (r == o) ? (uint32_t)N : (uint32_t)r;
}

// ptr[u] = first i with keys[i] >= u, for u in [0, N] (one thread per row)
__global__ void k_row_ptr(const uint32_t* __restrict__ keys, int64_t n, int32_t N,
                          int32_t* __restrict__ ptr) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u > N) return;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)keys[mid] < u) lo = mid + 1; else hi = mid;
  }
  ptr[u] = (int32_t)lo;
}

__global__ void k_fill_slots(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ keys,
                             const int32_t* __restrict__ ptr, int64_t Ev,
                             const int32_t* __restrict__ other, const int32_t* __restrict__ ts,
                             int32_t* __restrict__ nbr, int32_t* __restrict__ t,
                             int32_t* __restrict__ eid, int32_t* __restrict__ pos,
                             int32_t* __restrict__ rstart) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ev) return;
  int32_t e = (int32_t)perm[p];
  nbr[p] = other[e];
  t[p] = ts[e];
  eid[p] = e;
  pos[e] = (int32_t)p;
  rstart[p] = ptr[keys[p]];  // keys: the sorted row of every slot
}

// fills the (nbr, t, id) copy and links consecutive same-counterparty slots
__global__ void k_fill_nbr_order(const uint32_t* __restrict__ perm, int64_t Ev,
                                 const int32_t* __restrict__ row_of,
                                 const int32_t* __restrict__ other,
                                 const int32_t* __restrict__ ts, const int32_t* __restrict__ pos,
                                 int32_t* __restrict__ nnbr, int32_t* __restrict__ nt,
                                 int32_t* __restrict__ neid, int32_t* __restrict__ prev,
                                 int32_t* __restrict__ next) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ev) return;
  int32_t e = (int32_t)perm[p];
  nnbr[p] = other[e];
  nt[p] = ts[e];
  neid[p] = e;
  if (p > 0) {
    int32_t f = (int32_t)perm[p - 1];
    if (row_of[f] == row_of[e] && other[f] == other[e]) {
      prev[pos[e]] = pos[f];
      next[pos[f]] = pos[e];
    }
  }
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_max_degree(const int32_t* __restrict__ ptr, int32_t N,
                             int32_t* __restrict__ out) {
  int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t d = (u < N) ? ptr[u + 1] - ptr[u] : 0;
  d = __reduce_max_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(out, d);
}

// The graph's arrays come from the device's stream-ordered pool (no driver
// allocation once the pool holds enough), ordered on the build stream.
struct GraphAlloc {
  aml_graph* g;
  cudaStream_t s;
  template <typename T>
  T* get(size_t n) {
    void* p = dalloc((n ? n : 1) * sizeof(T), s);
    g->allocs.push_back(p);
    g->bytes += (int64_t)((n ? n : 1) * sizeof(T));
    return static_cast<T*>(p);
  }
};

static void free_graph(aml_graph* g) {
  for (void* p : g->allocs) dfree(p, 0);  // callers have synchronized
  g->allocs.clear();
  delete g;
}

// Rows of one direction (row_of/other = src/dst for out-lists, dst/src for
// in-lists): a stable sort of the time order by row gives every row in (t, id)
// order; perm keeps that order for the other direction's second copy.
static void build_rows(aml_graph* g, Adj& a, const int32_t* row_of, const int32_t* other,
                       const uint32_t* time_perm, int64_t E, int32_t N, int nbits,
                       cudaStream_t s, GraphAlloc& ga, uint32_t* perm, int32_t* max_deg_dev) {
  DBuf<uint32_t> keys(E, s), ktmp(E, s), vtmp(E, s);
  const int B = 256;
  copy_d2d(perm, time_perm, E * sizeof(uint32_t), s);
  AML_LAUNCH("k_row_keys", s,
             k_row_keys<<<grid_for(E, B), B, 0, s>>>(perm, row_of, other, E, N, keys.p));
  radix_sort_u32(keys.p, perm, ktmp.p, vtmp.p, E, nbits, s);
  a.ptr = ga.get<int32_t>((size_t)N + 1);
  AML_LAUNCH("k_row_ptr", s,
             k_row_ptr<<<grid_for((int64_t)N + 1, B), B, 0, s>>>(keys.p, E, N, a.ptr));
  const int64_t Ev = g->Ev;
  a.nbr = ga.get<int32_t>(Ev);
  a.t = ga.get<int32_t>(Ev);
  a.eid = ga.get<int32_t>(Ev);
  a.pos = ga.get<int32_t>(E);
  a.rstart = ga.get<int32_t>(Ev);
  AML_CUDA(cudaMemsetAsync(a.pos, 0xff, (E ? E : 1) * sizeof(int32_t), s));
  AML_LAUNCH("k_fill_slots", s,
             k_fill_slots<<<grid_for(Ev, B), B, 0, s>>>(
                 perm, keys.p, a.ptr, Ev, other, g->ts, a.nbr, a.t, a.eid, a.pos, a.rstart));
  AML_LAUNCH("k_max_degree", s, k_max_degree<<<grid_for(N, B), B, 0, s>>>(a.ptr, N, max_deg_dev));
}

// The (counterparty, t, id) copy of one direction's rows, and the links
// between consecutive slots of one counterparty.  `perm` is the other
// direction's row order, sorted by (counterparty, t, id) already: a stable
// sort by this direction's row gives (row, counterparty, t, id).
static void build_nbr_order(aml_graph* g, Adj& a, const int32_t* row_of,
                            const int32_t* other, uint32_t* perm, int64_t E, int32_t N,
                            int nbits, cudaStream_t s, GraphAlloc& ga) {
  DBuf<uint32_t> keys(E, s), ktmp(E, s), vtmp(E, s);
  const int B = 256;
  const int64_t Ev = g->Ev;
  a.prev = ga.get<int32_t>(Ev);
  a.next = ga.get<int32_t>(Ev);
  a.nnbr = ga.get<int32_t>(Ev);
  a.nt = ga.get<int32_t>(Ev);
  a.neid = ga.get<int32_t>(Ev);
  AML_CUDA(cudaMemsetAsync(a.prev, 0xff, (Ev ? Ev : 1) * sizeof(int32_t), s));
  AML_LAUNCH("k_fill_i32", s, k_fill_i32<<<grid_for(Ev, B), B, 0, s>>>(a.next, Ev, INT32_MAX));
  AML_LAUNCH("k_row_keys", s,
             k_row_keys<<<grid_for(E, B), B, 0, s>>>(perm, row_of, other, E, N, keys.p));
  radix_sort_u32(keys.p, perm, ktmp.p, vtmp.p, E, nbits, s);
  AML_LAUNCH("k_fill_nbr_order", s,
             k_fill_nbr_order<<<grid_for(Ev, B), B, 0, s>>>(
                 perm, Ev, row_of, other, g->ts, a.pos, a.nnbr, a.nt, a.neid, a.prev, a.next));
}

__global__ void k_count_loops(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                              int64_t E, unsigned long long* __restrict__ n_loops) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool loop = i < E && src[i] == dst[i];
  unsigned m = __ballot_sync(0xffffffffu, loop);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(n_loops, (unsigned long long)__popc(m));
}

aml_graph* build_graph(const int32_t* src, const int32_t* dst, const int32_t* ts,
                       const float* amount, int64_t E, int32_t N, uint32_t flags,
                       cudaStream_t s) {
  aml_graph* g = new aml_graph();
  GraphAlloc ga{g, s};
  try {
    AML_CUDA(cudaGetDevice(&g->device));
    g->E = E;
    g->N = N;
    g->note_stream(s);
    g->src = ga.get<int32_t>(E);
    g->dst = ga.get<int32_t>(E);
    g->ts = ga.get<int32_t>(E);
    g->amount = ga.get<float>(E);
    g->err = ga.get<uint32_t>(4);
    if (E) {
      // device inputs are copied by a kernel, host inputs by the copy engine
      auto in = [&](void* to, const void* from) {
        if (flags & AML_PTR_DEVICE) copy_d2d(to, from, E * 4, s);
        else AML_CUDA(cudaMemcpyAsync(to, from, E * 4, cudaMemcpyHostToDevice, s));
      };
      in(g->src, src);
      in(g->dst, dst);
      in(g->ts, ts);
      if (amount) in(g->amount, amount);
      else AML_CUDA(cudaMemsetAsync(g->amount, 0, E * 4, s));
    }
    AML_CUDA(cudaMemsetAsync(g->err, 0, 16, s));
    DBuf<unsigned long long> scal(4, s);
    AML_CUDA(cudaMemsetAsync(scal.p, 0, 32, s));
    const int B = 256;
    if (E) {
      AML_LAUNCH("k_validate", s,
                 k_validate<<<grid_for(E, B), B, 0, s>>>(g->src, g->dst, g->ts, E, N, g->err));
      AML_LAUNCH("k_count_loops", s,
                 k_count_loops<<<grid_for(E, B), B, 0, s>>>(g->src, g->dst, E, scal.p));
    }
    uint32_t err = 0;
    unsigned long long hs[4];
    const SmallRead rd[2] = {{&err, g->err, 4}, {hs, scal.p, 32}};
    read_small(rd, 2, s);
    AML_REQUIRE(!(err & ERR_BAD_ID), AML_EINVAL, "a node id is outside [0, n_nodes)");
    AML_REQUIRE(!((flags & AML_ASSUME_SORTED) && (err & ERR_UNSORTED)), AML_EUNSORTED,
                "AML_ASSUME_SORTED given but timestamps decrease");
    AML_CUDA(cudaMemsetAsync(g->err, 0, 16, s));
    g->Ev = E - (int64_t)hs[0];

    // global (t, id) order: identity when already sorted, else a stable sort
    DBuf<uint32_t> tperm(E, s);
    iota_i32(reinterpret_cast<int32_t*>(tperm.p), E, s);
    if (err & ERR_UNSORTED) {
      DBuf<uint32_t> keys(E, s), ktmp(E, s), vtmp(E, s);
      AML_LAUNCH("k_time_keys", s, k_time_keys<<<grid_for(E, B), B, 0, s>>>(g->ts, E, keys.p));
      radix_sort_u32(keys.p, tperm.p, ktmp.p, vtmp.p, E, 32, s);
    }
    int nbits = bits_for((uint64_t)N);  // keys range over [0, N]
    // maximum degrees: read when first asked for (aml_graph_get_info)
    g->max_deg = ga.get<int32_t>(2);
    AML_CUDA(cudaMemsetAsync(g->max_deg, 0, 8, s));
    DBuf<uint32_t> perm_out(E, s), perm_in(E, s);
    build_rows(g, g->out, g->src, g->dst, tperm.p, E, N, nbits, s, ga, perm_out.p, g->max_deg);
    build_rows(g, g->in, g->dst, g->src, tperm.p, E, N, nbits, s, ga, perm_in.p, g->max_deg + 1);
    // (src, dst, t, id) from the in-rows' (dst, t, id) order; (dst, src, t, id)
    // from the out-rows' (src, t, id) order
    build_nbr_order(g, g->out, g->src, g->dst, perm_in.p, E, N, nbits, s, ga);
    build_nbr_order(g, g->in, g->dst, g->src, perm_out.p, E, N, nbits, s, ga);
    return g;
  } catch (...) {
    cudaStreamSynchronize(s);
    free_graph(g);
    throw;
  }
}

void drop_captured_mines(aml_graph* g);

void destroy_graph(aml_graph* g) {
  if (!g) return;
  // wait for the work enqueued on this graph: on every stream a call was
  // given, and on the graph's own side and capture streams (not for other
  // work on the device, so a caller can overlap a graph's teardown with the
  // next graph's transfers); the whole device only if one of them cannot be
  // waited on
  bool ok = true;
  for (cudaStream_t st : g->used_streams) ok &= cudaStreamSynchronize(st) == cudaSuccess;
  for (cudaStream_t st : g->side)
    if (st) ok &= cudaStreamSynchronize(st) == cudaSuccess;
  if (g->capture_stream) ok &= cudaStreamSynchronize(g->capture_stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaDeviceSynchronize();
  }
  drop_captured_mines(g);
  if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
  for (cudaStream_t st : g->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : g->branch_ev)
    if (ev) cudaEventDestroy(ev);
  free_graph(g);
}

}  // namespace aml
