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
#include "mine.cuh"
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
      g->dts = ga.get<int2>(E);
      AML_LAUNCH("k_pack_dst_ts", s,
                 k_pack_dst_ts<<<grid_for(E, 256), 256, 0, s>>>(g->dst, g->ts, E, g->dts));
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

// ------------------------------------------------------------ sliding update
//
// The graph of a sliding window, made from the graph of the window before it
// instead of from scratch.  The new window drops the old one's first `drop`
// edges and appends `n_new` edges that are no earlier than any old edge, so
// local ids shift down by `drop` and every row changes only at its two ends:
// the dropped edges are a prefix of each (t, id)-ordered row (ids follow
// time), and the new edges go after every kept slot.  Kept slots move by a
// per-row offset (one coalesced pass); only the new edges are sorted.  In a
// row's (counterparty, t, id) copy, a kept entry moves up past the new edges
// with a smaller counterparty and a new entry past the kept ones with a
// counterparty no larger than its own.  Same-counterparty links move with
// the kept slots; a new edge is linked to the entry before it in the new
// copy.  The result equals a full build of the new window.

// per row: dropped prefix (first slot with id >= drop) and the new length
__global__ void k_upd_rows(const int32_t* __restrict__ optr, const int32_t* __restrict__ oeid,
                           int32_t drop, const int32_t* __restrict__ bptr, int32_t N,
                           int32_t* __restrict__ cnt, int32_t* __restrict__ kdrop) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N) return;
  if (r == N) {
    cnt[N] = 0;
    return;
  }
  const int32_t lo = optr[r], hi = optr[r + 1];
  int32_t a = lo, b = hi;
  while (a < b) {
    const int32_t mid = (int32_t)(((uint32_t)a + (uint32_t)b) >> 1);
    if (oeid[mid] < drop) a = mid + 1; else b = mid;
  }
  kdrop[r] = a - lo;
  cnt[r] = (hi - a) + (bptr[r + 1] - bptr[r]);
}

// per old row start: {new row start, dropped prefix, new edges' range in the
// sorted batch}, read by every slot of the row through its old row start;
// per row: how far its kept slots move
__global__ void k_upd_rowinfo(const int32_t* __restrict__ optr, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ kdrop, const int32_t* __restrict__ bptr,
                              int32_t N, int4* __restrict__ info, int32_t* __restrict__ shift) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int32_t lo = optr[r];
  shift[r] = ptr[r] - lo - kdrop[r];
  if (optr[r + 1] > lo) info[lo] = make_int4(ptr[r], kdrop[r], bptr[r], bptr[r + 1]);
}

// slot of every kept edge: its old slot moved by its row's shift (edge
// order, so the reads and writes are coalesced; self-loops stay -1)
__global__ void k_upd_pos(const int32_t* __restrict__ opos, const int32_t* __restrict__ row_of,
                          const int32_t* __restrict__ shift, int32_t drop, int64_t n_kept,
                          int32_t* __restrict__ pos) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_kept) return;
  const int32_t p = opos[e + drop];
  pos[e] = p < 0 ? -1 : p + shift[row_of[e]];
}

// kept slots, and their same-counterparty links: the previous slot of the
// counterparty moves with the row unless it was dropped (then no kept slot
// precedes), the next one always moves with it (a new edge that follows is
// linked afterwards by k_upd_new_links)
__global__ void k_upd_keep(const int32_t* __restrict__ oeid, const int32_t* __restrict__ orstart,
                           const int32_t* __restrict__ onbr, const int32_t* __restrict__ ot,
                           const int32_t* __restrict__ oprev, const int32_t* __restrict__ onext,
                           const int4* __restrict__ info, int32_t drop, int64_t oEv,
                           int32_t* __restrict__ nbr, int32_t* __restrict__ t,
                           int32_t* __restrict__ eid, int32_t* __restrict__ rstart,
                           int32_t* __restrict__ prev, int32_t* __restrict__ next) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= oEv) return;
  const int32_t e = oeid[p];
  if (e < drop) return;
  const int32_t rs = orstart[p];
  const int4 ri = info[rs];
  const int32_t off = ri.x - rs - ri.y;  // the row's kept slots move by this
  const int32_t q = (int32_t)p + off;
  nbr[q] = onbr[p];
  t[q] = ot[p];
  eid[q] = e - drop;
  rstart[q] = ri.x;
  const int32_t pv = oprev[p], nx = onext[p];
  prev[q] = (pv < 0 || pv - rs < ri.y) ? -1 : pv + off;
  next[q] = nx == INT32_MAX ? INT32_MAX : nx + off;
}

// new edges in (row, id) order: after the row's kept slots
__global__ void k_upd_new(const uint32_t* __restrict__ bkey, const uint32_t* __restrict__ bperm,
                          const int32_t* __restrict__ bptr, const int32_t* __restrict__ ptr,
                          const int32_t* __restrict__ other, const int32_t* __restrict__ ts,
                          int32_t b0, int64_t n, int32_t N, int32_t* __restrict__ nbr,
                          int32_t* __restrict__ t, int32_t* __restrict__ eid,
                          int32_t* __restrict__ rstart, int32_t* __restrict__ pos,
                          int32_t* __restrict__ prev, int32_t* __restrict__ next) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = (int32_t)bkey[i];
  const int32_t e = b0 + (int32_t)bperm[i];
  if (r >= N) {  // a self-loop: in no row
    pos[e] = -1;
    return;
  }
  const int32_t q = ptr[r + 1] - bptr[r + 1] + (int32_t)i;
  nbr[q] = other[e];
  t[q] = ts[e];
  eid[q] = e;
  rstart[q] = ptr[r];
  pos[e] = q;
  prev[q] = -1;  // linked by k_upd_new_links
  next[q] = INT32_MAX;
}

__global__ void k_upd_kept_flags(const int32_t* __restrict__ oneid, int32_t drop, int64_t oEv,
                                 int32_t* __restrict__ flag) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= oEv) flag[p] = p < oEv && oneid[p] >= drop;
}

__global__ void k_upd_batch_nbr(const uint32_t* __restrict__ bperm,
                                const int32_t* __restrict__ other, int32_t b0, int64_t n,
                                int32_t* __restrict__ bnbr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bnbr[i] = other[b0 + (int32_t)bperm[i]];
}

// kept (counterparty, t, id) entries: past the row's new edges with a smaller
// counterparty (bnbr: counterparties of the batch in (row, counterparty) order)
__global__ void k_upd_nkeep(const int32_t* __restrict__ oneid, const int32_t* __restrict__ onnbr,
                            const int32_t* __restrict__ ont, const int32_t* __restrict__ orstart,
                            const int4* __restrict__ info, const int32_t* __restrict__ kept,
                            const int32_t* __restrict__ bnbr, int32_t drop, int64_t oEv,
                            int32_t* __restrict__ nnbr, int32_t* __restrict__ nt,
                            int32_t* __restrict__ neid) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= oEv) return;
  const int32_t e = oneid[p];
  if (e < drop) return;
  const int32_t rs = orstart[p];
  const int4 ri = info[rs];
  const int32_t x = onnbr[p];
  int32_t a = ri.z, b = ri.w;  // first new edge of the row with counterparty >= x
  while (a < b) {
    const int32_t mid = (int32_t)(((uint32_t)a + (uint32_t)b) >> 1);
    if (bnbr[mid] < x) a = mid + 1; else b = mid;
  }
  const int32_t q = ri.x + (kept[p] - kept[rs]) + (a - ri.z);
  nnbr[q] = x;
  nt[q] = ont[p];
  neid[q] = e - drop;
}

// new (counterparty, t, id) entries: past the row's kept entries with a
// counterparty <= their own
__global__ void k_upd_nnew(const uint32_t* __restrict__ bkey, const uint32_t* __restrict__ bperm,
                           const int32_t* __restrict__ bptr, const int32_t* __restrict__ ptr,
                           const int32_t* __restrict__ optr, const int32_t* __restrict__ onnbr,
                           const int32_t* __restrict__ kept, const int32_t* __restrict__ other,
                           const int32_t* __restrict__ ts, int32_t b0, int64_t n, int32_t N,
                           int32_t* __restrict__ nnbr, int32_t* __restrict__ nt,
                           int32_t* __restrict__ neid, int32_t* __restrict__ nq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = (int32_t)bkey[i];
  nq[i] = -1;
  if (r >= N) return;
  const int32_t e = b0 + (int32_t)bperm[i];
  const int32_t x = other[e];
  const int32_t lo = optr[r];
  int32_t a = lo, b = optr[r + 1];  // first old entry with counterparty > x
  while (a < b) {
    const int32_t mid = (int32_t)(((uint32_t)a + (uint32_t)b) >> 1);
    if (onnbr[mid] <= x) a = mid + 1; else b = mid;
  }
  const int32_t q = ptr[r] + (kept[a] - kept[lo]) + ((int32_t)i - bptr[r]);
  nnbr[q] = x;
  nt[q] = ts[e];
  neid[q] = e;
  nq[i] = q;
}

// a new edge's same-counterparty link: the entry before it in the
// (counterparty, t, id) copy, if of the same row and counterparty, is the
// previous slot of that counterparty (kept or new)
__global__ void k_upd_new_links(const int32_t* __restrict__ nq, int64_t n,
                                const int32_t* __restrict__ nnbr, const int32_t* __restrict__ neid,
                                const int32_t* __restrict__ rstart,
                                const int32_t* __restrict__ pos, int32_t* __restrict__ prev,
                                int32_t* __restrict__ next) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t q = nq[i];
  if (q < 0 || q == rstart[q] || nnbr[q] != nnbr[q - 1]) return;
  const int32_t pe = pos[neid[q]], pf = pos[neid[q - 1]];
  prev[pe] = pf;
  next[pf] = pe;
}

// The sorted new edges of one direction: (row, id) order in (bkey, bperm),
// (row, counterparty, id) order in (nkey, nperm); bptr = row offsets.
struct BatchRows {
  DBuf<uint32_t> bkey, bperm, nkey, nperm;
  DBuf<int32_t> bptr, bnbr, cnt, kdrop;
  BatchRows(int64_t n, int32_t N, cudaStream_t s)
      : bkey(n, s), bperm(n, s), nkey(n, s), nperm(n, s), bptr((size_t)N + 1, s),
        bnbr(n, s), cnt((size_t)N + 1, s), kdrop((size_t)N, s) {}
};

// A batch of up to SMALL_SORT edges is sorted in shared memory: one block
// per (direction, order), all four in one launch, each a bitonic sort of
// 64-bit keys (row << 36 | counterparty << 14 | index), rows as k_row_keys
// gives them (N for a self-loop) and the counterparty 0 when only (row,
// index) order is wanted.  The keys are unique (the index), so the order
// equals the stable radix sorts' order.  It needs N < 2^22 (rows up to N in
// 28 bits, counterparties in 22); a larger batch or graph takes the radix
// passes (three launches each) instead.
constexpr int SMALL_SORT = 16384;
constexpr int SMALL_SORT_THREADS = 1024;
constexpr int32_t SMALL_SORT_MAX_N = 1 << 22;

struct SmallSortJob {
  const int32_t* row_of;
  const int32_t* other;
  uint32_t* key;   // sorted rows
  uint32_t* perm;  // the batch index of each
  int by_nbr;
};
struct SmallSortJobs {
  SmallSortJob job[4];
};

__global__ void __launch_bounds__(SMALL_SORT_THREADS) k_sort_small(SmallSortJobs J, int n, int m,
                                                                   int32_t N) {
  extern __shared__ unsigned long long s_sort[];  // m keys
  const SmallSortJob q = J.job[blockIdx.x];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    unsigned long long k = ~0ull;  // padding sorts last
    if (i < n) {
      const int32_t r = q.row_of[i], o = q.other[i];
      const unsigned long long row = r == o ? (unsigned long long)N : (unsigned long long)r;
      const unsigned long long nbr = q.by_nbr ? (unsigned long long)o : 0ull;
      k = (row << 36) | (nbr << 14) | (unsigned long long)i;
    }
    s_sort[i] = k;
  }
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < m / 2; t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1));  // the lower element of a pair
        const int l = i + j;
        const unsigned long long x = s_sort[i], y = s_sort[l];
        if ((x > y) == ((i & k) == 0)) {
          s_sort[i] = y;
          s_sort[l] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long k = s_sort[i];
    q.key[i] = (uint32_t)(k >> 36);
    q.perm[i] = (uint32_t)(k & 0x3fffull);
  }
}

// Both directions' batch orders at once when the batch and the graph are
// small enough for k_sort_small; false (nothing done) otherwise.
static bool upd_sort_batches_small(BatchRows& bo, BatchRows& bi, const int32_t* src,
                                   const int32_t* dst, int64_t n, int32_t N, cudaStream_t s) {
  if (n > SMALL_SORT || N >= SMALL_SORT_MAX_N) return false;
  const int B = 256;
  int m = 2;
  while (m < n) m <<= 1;
  const int smem = m * (int)sizeof(unsigned long long);
  static bool attr_set[64] = {};  // per device: the large shared-memory opt-in
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  if (smem > 48 * 1024 && (dev >= 64 || !attr_set[dev])) {
    AML_CUDA(cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  SMALL_SORT * (int)sizeof(unsigned long long)));
    if (dev < 64) attr_set[dev] = true;
  }
  SmallSortJobs J;
  J.job[0] = SmallSortJob{src, dst, bo.bkey.p, bo.bperm.p, 0};
  J.job[1] = SmallSortJob{src, dst, bo.nkey.p, bo.nperm.p, 1};
  J.job[2] = SmallSortJob{dst, src, bi.bkey.p, bi.bperm.p, 0};
  J.job[3] = SmallSortJob{dst, src, bi.nkey.p, bi.nperm.p, 1};
  AML_LAUNCH("k_sort_small", s,
             k_sort_small<<<4, SMALL_SORT_THREADS, smem, s>>>(J, (int)n, m, N));
  for (BatchRows* b : {&bo, &bi}) {
    const int32_t* other = b == &bo ? dst : src;
    AML_LAUNCH("k_row_ptr", s,
               k_row_ptr<<<grid_for((int64_t)N + 1, B), B, 0, s>>>(b->bkey.p, n, N, b->bptr.p));
    AML_LAUNCH("k_upd_batch_nbr", s,
               k_upd_batch_nbr<<<grid_for(n, B), B, 0, s>>>(b->nperm.p, other, 0, n, b->bnbr.p));
  }
  return true;
}

static void upd_sort_batch(BatchRows& b, const int32_t* row_of, const int32_t* other, int64_t n,
                           int32_t N, int nbits, cudaStream_t s) {
  const int B = 256;
  DBuf<uint32_t> kt(n, s), vt(n, s);
  iota_i32(reinterpret_cast<int32_t*>(b.bperm.p), n, s);
  AML_LAUNCH("k_row_keys", s,
             k_row_keys<<<grid_for(n, B), B, 0, s>>>(b.bperm.p, row_of, other, n, N, b.bkey.p));
  radix_sort_u32(b.bkey.p, b.bperm.p, kt.p, vt.p, n, nbits, s);
  AML_LAUNCH("k_row_ptr", s,
             k_row_ptr<<<grid_for((int64_t)N + 1, B), B, 0, s>>>(b.bkey.p, n, N, b.bptr.p));
  // by counterparty, then stably by row
  iota_i32(reinterpret_cast<int32_t*>(b.nperm.p), n, s);
  copy_d2d(b.nkey.p, other, (size_t)n * 4, s);
  radix_sort_u32(b.nkey.p, b.nperm.p, kt.p, vt.p, n, nbits, s);
  AML_LAUNCH("k_row_keys", s,
             k_row_keys<<<grid_for(n, B), B, 0, s>>>(b.nperm.p, row_of, other, n, N, b.nkey.p));
  radix_sort_u32(b.nkey.p, b.nperm.p, kt.p, vt.p, n, nbits, s);
  AML_LAUNCH("k_upd_batch_nbr", s,
             k_upd_batch_nbr<<<grid_for(n, B), B, 0, s>>>(b.nperm.p, other, 0, n, b.bnbr.p));
}

static void upd_fill(const aml_graph* o, aml_graph* g, const Adj& ao, Adj& a, BatchRows& b,
                     const int32_t* row_of, const int32_t* other, int32_t drop, int64_t n_new,
                     cudaStream_t s, GraphAlloc& ga, int32_t* max_deg_dev) {
  const int B = 256;
  const int64_t E = g->E, Ev = g->Ev, oEv = o->Ev;
  const int32_t N = g->N, b0 = (int32_t)(E - n_new);
  a.nbr = ga.get<int32_t>(Ev);
  a.t = ga.get<int32_t>(Ev);
  a.eid = ga.get<int32_t>(Ev);
  a.pos = ga.get<int32_t>(E);
  a.rstart = ga.get<int32_t>(Ev);
  a.prev = ga.get<int32_t>(Ev);
  a.next = ga.get<int32_t>(Ev);
  a.nnbr = ga.get<int32_t>(Ev);
  a.nt = ga.get<int32_t>(Ev);
  a.neid = ga.get<int32_t>(Ev);
  DBuf<int4> info(oEv ? oEv : 1, s);
  DBuf<int32_t> nq(n_new ? n_new : 1, s);
  DBuf<int32_t> kept(oEv + 1, s);
  int32_t* shift = b.cnt.p;  // the counts are spent: the scan made the row pointers
  AML_LAUNCH("k_upd_rowinfo", s,
             k_upd_rowinfo<<<grid_for(N, B), B, 0, s>>>(ao.ptr, a.ptr, b.kdrop.p, b.bptr.p, N,
                                                       info.p, shift));
  if (oEv)
    AML_LAUNCH("k_upd_keep", s,
               k_upd_keep<<<grid_for(oEv, B), B, 0, s>>>(ao.eid, ao.rstart, ao.nbr, ao.t, ao.prev,
                                                        ao.next, info.p, drop, oEv, a.nbr, a.t,
                                                        a.eid, a.rstart, a.prev, a.next));
  if (b0 > 0)
    AML_LAUNCH("k_upd_pos", s,
               k_upd_pos<<<grid_for(b0, B), B, 0, s>>>(ao.pos, row_of, shift, drop, b0, a.pos));
  if (n_new)
    AML_LAUNCH("k_upd_new", s,
               k_upd_new<<<grid_for(n_new, B), B, 0, s>>>(b.bkey.p, b.bperm.p, b.bptr.p, a.ptr,
                                                         other, g->ts, b0, n_new, N,
                                                         a.nbr, a.t, a.eid, a.rstart, a.pos,
                                                         a.prev, a.next));
  AML_LAUNCH("k_upd_kept_flags", s,
             k_upd_kept_flags<<<grid_for(oEv + 1, B), B, 0, s>>>(ao.neid, drop, oEv, kept.p));
  scan_i32(kept.p, kept.p, oEv + 1, false, s);
  if (oEv)
    AML_LAUNCH("k_upd_nkeep", s,
               k_upd_nkeep<<<grid_for(oEv, B), B, 0, s>>>(ao.neid, ao.nnbr, ao.nt, ao.rstart,
                                                         info.p, kept.p, b.bnbr.p, drop, oEv,
                                                         a.nnbr, a.nt, a.neid));
  if (n_new)
    AML_LAUNCH("k_upd_nnew", s,
               k_upd_nnew<<<grid_for(n_new, B), B, 0, s>>>(b.nkey.p, b.nperm.p, b.bptr.p, a.ptr,
                                                          ao.ptr, ao.nnbr, kept.p, other, g->ts,
                                                          b0, n_new, N, a.nnbr, a.nt,
                                                          a.neid, nq.p));
  if (n_new)
    AML_LAUNCH("k_upd_new_links", s,
               k_upd_new_links<<<grid_for(n_new, B), B, 0, s>>>(nq.p, n_new, a.nnbr, a.neid,
                                                               a.rstart, a.pos, a.prev, a.next));
  AML_LAUNCH("k_max_degree", s, k_max_degree<<<grid_for(N, B), B, 0, s>>>(a.ptr, N, max_deg_dev));
}

aml_graph* update_graph(const aml_graph* o, int64_t drop, const int32_t* src, const int32_t* dst,
                        const int32_t* ts, const float* amount, int64_t E, cudaStream_t s) {
  AML_REQUIRE(o && drop >= 0 && drop <= o->E && E >= o->E - drop && E < INT32_MAX,
              AML_EINVAL, "bad sliding-window update");
  const int64_t n_new = E - (o->E - drop);
  aml_graph* g = new aml_graph();
  GraphAlloc ga{g, s};
  try {
    AML_CUDA(cudaGetDevice(&g->device));
    g->E = E;
    g->N = o->N;
    g->tune = o->tune;
    g->note_stream(s);
    g->src = ga.get<int32_t>(E);
    g->dst = ga.get<int32_t>(E);
    g->ts = ga.get<int32_t>(E);
    g->amount = ga.get<float>(E);
    g->err = ga.get<uint32_t>(4);
    if (E) {
      copy_d2d(g->src, src, E * 4, s);
      copy_d2d(g->dst, dst, E * 4, s);
      copy_d2d(g->ts, ts, E * 4, s);
      if (amount) copy_d2d(g->amount, amount, E * 4, s);
      else AML_CUDA(cudaMemsetAsync(g->amount, 0, E * 4, s));
      g->dts = ga.get<int2>(E);
      AML_LAUNCH("k_pack_dst_ts", s,
                 k_pack_dst_ts<<<grid_for(E, 256), 256, 0, s>>>(g->dst, g->ts, E, g->dts));
    }
    AML_CUDA(cudaMemsetAsync(g->err, 0, 16, s));
    g->max_deg = ga.get<int32_t>(2);
    AML_CUDA(cudaMemsetAsync(g->max_deg, 0, 8, s));
    const int32_t N = g->N, b0 = (int32_t)(E - n_new);
    const int nbits = bits_for((uint64_t)N);
    const int B = 256;
    const int64_t nb = n_new ? n_new : 1;
    BatchRows bo(nb, N, s), bi(nb, N, s);
    if (n_new) {
      if (!upd_sort_batches_small(bo, bi, g->src + b0, g->dst + b0, n_new, N, s)) {
        upd_sort_batch(bo, g->src + b0, g->dst + b0, n_new, N, nbits, s);
        upd_sort_batch(bi, g->dst + b0, g->src + b0, n_new, N, nbits, s);
      }
    } else {
      AML_CUDA(cudaMemsetAsync(bo.bptr.p, 0, ((size_t)N + 1) * 4, s));
      AML_CUDA(cudaMemsetAsync(bi.bptr.p, 0, ((size_t)N + 1) * 4, s));
    }
    g->out.ptr = ga.get<int32_t>((size_t)N + 1);
    g->in.ptr = ga.get<int32_t>((size_t)N + 1);
    AML_LAUNCH("k_upd_rows", s,
               k_upd_rows<<<grid_for((int64_t)N + 1, B), B, 0, s>>>(
                   o->out.ptr, o->out.eid, (int32_t)drop, bo.bptr.p, N, bo.cnt.p, bo.kdrop.p));
    AML_LAUNCH("k_upd_rows", s,
               k_upd_rows<<<grid_for((int64_t)N + 1, B), B, 0, s>>>(
                   o->in.ptr, o->in.eid, (int32_t)drop, bi.bptr.p, N, bi.cnt.p, bi.kdrop.p));
    scan_i32(bo.cnt.p, g->out.ptr, (int64_t)N + 1, false, s);
    scan_i32(bi.cnt.p, g->in.ptr, (int64_t)N + 1, false, s);
    int32_t ev[2] = {0, 0};
    const SmallRead rd[2] = {{&ev[0], g->out.ptr + N, 4}, {&ev[1], g->in.ptr + N, 4}};
    read_small(rd, 2, s);
    AML_REQUIRE(ev[0] == ev[1], AML_EINTERNAL, "sliding update: out and in lists disagree");
    g->Ev = ev[0];
    upd_fill(o, g, o->out, g->out, bo, g->src, g->dst, (int32_t)drop, n_new, s, ga, g->max_deg);
    upd_fill(o, g, o->in, g->in, bi, g->dst, g->src, (int32_t)drop, n_new, s, ga,
             g->max_deg + 1);
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
