// Streaming recount (aml_stream_*): transactions arrive in time-ordered
// batches; every count of every resident edge stays equal to the count over
// the whole history.  Sec. 5 describes this streaming use: a new edge adds
// one to the counts of every instance it completes, and only the affected
// neighbourhood is re-examined rather than the whole graph.
//
// Why one mine of a window suffices.  A batch B arrives after every resident
// edge in the (t, id) order.  Let W be the resident edges with
// t >= t_min(B) - delta_max.  An instance that contains a batch edge spans at
// most delta_max, so all its edges lie in W u B; and it contains a batch
// edge iff its latest edge is one.  So mining W u B while counting only the
// instances whose latest edge is a batch edge (delta counting: the closing
// edge of a cycle, the later gather edge of a scatter-gather pair, the second
// edge of a gather-scatter pair) yields exactly the instances B creates:
// added to the stored counts of the rows of W, and the full counts of the
// batch rows.  Trailing-window columns (DEG, FAN) of old rows never change:
// later edges are outside their windows.
//
// Each append needs the graph of W u B.  Consecutive windows overlap almost
// entirely, so the stream keeps the last window's graph and updates it (drop
// the rows that left, add the rows that arrived) instead of sorting the whole
// window again.
//
// Resident rows live in device arrays compacted on demand; an append evicts
// the rows older than both t_now - resident_window and t_first(B) -
// delta_max (W must stay resident while B is counted).  resident_window >=
// delta_max keeps every instance of a resident row visible while it is
// counted, so resident rows hold full-history counts.  A batch that would not fit the memory
// budget is refused (AML_EADMIT) before any state changes.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {
aml_graph* build_graph(const int32_t* src, const int32_t* dst, const int32_t* ts,
                       const float* amount, int64_t E, int32_t N, uint32_t flags, cudaStream_t s);
aml_graph* update_graph(const aml_graph* o, int64_t drop, const int32_t* src, const int32_t* dst,
                        const int32_t* ts, const float* amount, int64_t E, cudaStream_t s);
void destroy_graph(aml_graph* g);
}  // namespace aml

struct aml_stream {
  aml_pattern_set ps;
  int32_t P = 0;
  int32_t N = 0;
  int32_t window = 0;        // resident window (s)
  int32_t delta_max = 0;     // largest window of any column
  size_t budget = 0;
  int64_t cap = 0;           // resident edge capacity
  int32_t* src = nullptr;    // device [cap]
  int32_t* dst = nullptr;
  int32_t* ts = nullptr;
  float* amt = nullptr;
  uint32_t* counts = nullptr;  // device [cap * P], row-major
  std::vector<int32_t> hts;    // host copy of ts, slot-indexed
  int64_t lo = 0, hi = 0;      // live slots
  int64_t base = 0;            // global row id of slot 0
  bool any = false;
  int32_t t_max = 0;
  int device = 0;
  // the graph of the last recount window (global rows [g_first, g_first +
  // g->E)), kept so the next window's graph is an update of it
  aml_graph* g = nullptr;
  int64_t g_first = 0;
  uint32_t count_limit = 0xffffffffu;  // saturation bound of the stored counts
};

namespace aml {

// Per-resident-edge working set of one append: the device graph of the
// window (about 90 B/edge) plus the mine's scratch and its output.
static int64_t ws_per_edge(int P) { return 512 + 16 * (int64_t)P; }

static void drop_graph(aml_stream* st) {
  if (st->g) destroy_graph(st->g);
  st->g = nullptr;
}

static void free_stream(aml_stream* st) {
  drop_graph(st);
  cudaFree(st->src);
  cudaFree(st->dst);
  cudaFree(st->ts);
  cudaFree(st->amt);
  cudaFree(st->counts);
  delete st;
}

template <typename T>
static void move_rows(T* p, int64_t from, int64_t n, size_t row_elems, cudaStream_t s) {
  if (n <= 0 || from == 0) return;
  DBuf<T> tmp((size_t)n * row_elems, s);
  AML_CUDA(cudaMemcpyAsync(tmp.p, p + from * row_elems, n * row_elems * sizeof(T),
                           cudaMemcpyDeviceToDevice, s));
  AML_CUDA(cudaMemcpyAsync(p, tmp.p, n * row_elems * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

static void compact(aml_stream* st, cudaStream_t s) {
  const int64_t live = st->hi - st->lo;
  move_rows(st->src, st->lo, live, 1, s);
  move_rows(st->dst, st->lo, live, 1, s);
  move_rows(st->ts, st->lo, live, 1, s);
  move_rows(st->amt, st->lo, live, 1, s);
  move_rows(st->counts, st->lo, live, (size_t)st->P, s);
  std::memmove(st->hts.data(), st->hts.data() + st->lo, (size_t)live * sizeof(int32_t));
  st->base += st->lo;
  st->hi = live;
  st->lo = 0;
}

// mines rows [w0, w0 + n) counting only instances whose latest edge is at
// local id >= new_from (the batch, first edge at time t_new): rows below
// new_from add those to their stored instance columns, the others are
// written outright
//
// The window's graph is the previous window's graph updated (its oldest rows
// dropped, the rows after it added) when that graph starts no later than w0
// and ends inside the new window; otherwise it is built from scratch.  The
// old graph is released once the update is enqueued; on any failure no graph
// is kept, so the next append builds afresh.
static void mine_window(aml_stream* st, int64_t w0, int64_t n, int32_t new_from, int32_t t_new,
                        uint32_t* out, cudaStream_t s) {
  const int64_t first = st->base + w0;
  aml_graph* g = nullptr;
  try {
    aml_graph* o = st->g;
    if (o && st->g_first <= first && first - st->g_first < o->E &&
        st->g_first + o->E <= first + n)
      g = update_graph(o, first - st->g_first, st->src + w0, st->dst + w0, st->ts + w0,
                       st->amt + w0, n, s);
    else
      g = build_graph(st->src + w0, st->dst + w0, st->ts + w0, st->amt + w0, n, st->N,
                      AML_PTR_DEVICE | AML_ASSUME_SORTED, s);
  } catch (...) {
    drop_graph(st);
    throw;
  }
  drop_graph(st);
  try {
    g->count_limit = st->count_limit;
    mine_plain(g, &st->ps, out, st->P, s, 0, new_from, t_new, true);
    AML_CUDA(cudaStreamSynchronize(s));
    uint32_t err = 0;
    AML_CUDA(cudaMemcpy(&err, g->err, 4, cudaMemcpyDeviceToHost));
    AML_REQUIRE(!(err & ERR_TIMEOUT), AML_ETIMEOUT, "a bounded device wait gave up");
    AML_REQUIRE(err == 0, AML_EINTERNAL, "device error word set (" + std::to_string(err) + ")");
  } catch (...) {
    destroy_graph(g);
    throw;
  }
  st->g = g;
  st->g_first = first;
}

__global__ void k_count_diff(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                             int64_t n, unsigned long long* __restrict__ diff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool d = i < n && a[i] != b[i];
  const unsigned m = __ballot_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(diff, (unsigned long long)__popc(m));
}

}  // namespace aml

using namespace aml;

extern "C" {

aml_status aml_stream_open(const aml_pattern_set* ps, int32_t n_nodes, int32_t resident_window_s,
                           size_t mem_budget_bytes, aml_stream** out) {
  aml_stream* st = nullptr;
  try {
    AML_REQUIRE(ps && out, AML_EINVAL, "NULL argument");
    AML_REQUIRE(n_nodes >= 1, AML_EINVAL, "n_nodes must be >= 1");
    st = new aml_stream();
    for (const Column& c : ps->cols) {
      AML_REQUIRE(c.family != AML_FAM_CYCW, AML_EUNSUPPORTED,
                  "window cycles (CYCW) are not counted incrementally");
      AML_REQUIRE(c.family != AML_FAM_PROGRAM, AML_EUNSUPPORTED,
                  "interpreted stage programs are not counted incrementally");
    }
    st->ps = *ps;
    st->P = (int32_t)ps->cols.size();
    st->N = n_nodes;
    for (size_t c = 0; c < ps->cols.size(); ++c)
      st->delta_max = std::max(st->delta_max, ps->cols[c].delta);
    AML_REQUIRE(resident_window_s >= st->delta_max, AML_EINVAL,
                "resident_window_s must be >= the largest pattern window");
    st->window = resident_window_s;
    st->budget = mem_budget_bytes;
    // half of the budget holds resident rows, half the working set of appends
    const int64_t row_bytes = 16 + 4 * (int64_t)st->P;
    st->cap = (int64_t)(mem_budget_bytes / 2) / row_bytes;
    AML_REQUIRE(st->cap >= 1024, AML_EINVAL, "memory budget too small");
    AML_REQUIRE(st->cap < (int64_t)INT32_MAX, AML_EINVAL, "memory budget too large");
    AML_CUDA(cudaGetDevice(&st->device));
    AML_CUDA(cudaMalloc(&st->src, st->cap * 4));
    AML_CUDA(cudaMalloc(&st->dst, st->cap * 4));
    AML_CUDA(cudaMalloc(&st->ts, st->cap * 4));
    AML_CUDA(cudaMalloc(&st->amt, st->cap * 4));
    AML_CUDA(cudaMalloc(&st->counts, st->cap * 4 * (int64_t)st->P));
    st->hts.resize((size_t)st->cap);
    *out = st;
    return AML_OK;
  } catch (const Failure& f) {
    if (st) free_stream(st);
    set_error(std::string("aml_stream_open: ") + f.msg);
    return f.status;
  } catch (...) {
    if (st) free_stream(st);
    set_error("aml_stream_open: unexpected internal error");
    return AML_EINTERNAL;
  }
}

aml_status aml_stream_append(aml_stream* st, const int32_t* src, const int32_t* dst,
                             const int32_t* ts, const float* amount, int64_t n, uint32_t flags,
                             void* stream, aml_stream_batch* info) {
  try {
    AML_REQUIRE(st != nullptr, AML_EINVAL, "NULL stream");
    AML_REQUIRE(n >= 0 && n < (int64_t)INT32_MAX, AML_EINVAL, "bad batch size");
    AML_REQUIRE(n == 0 || (src && dst && ts), AML_EINVAL, "src/dst/ts must not be NULL");
    AML_REQUIRE((flags & ~AML_PTR_DEVICE) == 0, AML_EINVAL, "unknown flag bits");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (info) std::memset(info, 0, sizeof(*info));
    if (n == 0) {
      if (info) info->first_row = st->base + st->hi;
      return AML_OK;
    }
    const bool dev = flags & AML_PTR_DEVICE;
    // host copies for validation and bookkeeping (nothing changes until all checks pass)
    std::vector<int32_t> hs(n), hd(n), ht(n);
    auto fetch = [&](const int32_t* p, std::vector<int32_t>& v) {
      if (dev) AML_CUDA(cudaMemcpy(v.data(), p, n * 4, cudaMemcpyDeviceToHost));
      else std::memcpy(v.data(), p, n * 4);
    };
    fetch(src, hs);
    fetch(dst, hd);
    fetch(ts, ht);
    for (int64_t i = 0; i < n; ++i) {
      AML_REQUIRE(hs[i] >= 0 && hs[i] < st->N && hd[i] >= 0 && hd[i] < st->N, AML_EINVAL,
                  "a node id is outside [0, n_nodes)");
      AML_REQUIRE(i == 0 || ht[i - 1] <= ht[i], AML_EUNSORTED,
                  "batch timestamps must be non-decreasing");
    }
    AML_REQUIRE(!st->any || ht[0] >= st->t_max, AML_ELATE,
                "batch starts before the latest timestamp already appended");
    // eviction and admission plan: rows older than the resident window go,
    // except those the batch's recount window W still needs
    const int32_t t_first = ht[0], t_last = ht[n - 1];
    const int64_t cutoff = std::min((int64_t)t_last - st->window,
                                    (int64_t)t_first - st->delta_max);
    const int64_t new_lo =
        std::lower_bound(st->hts.begin() + st->lo, st->hts.begin() + st->hi, cutoff,
                         [](int32_t a, int64_t b) { return (int64_t)a < b; }) -
        st->hts.begin();
    AML_REQUIRE((st->hi - new_lo) + n <= st->cap, AML_EADMIT,
                "resident rows plus the batch exceed the memory budget");
    const int64_t w_lo =
        std::lower_bound(st->hts.begin() + new_lo, st->hts.begin() + st->hi,
                         (int64_t)t_first - st->delta_max,
                         [](int32_t a, int64_t b) { return (int64_t)a < b; }) -
        st->hts.begin();
    const int64_t n_w = st->hi - w_lo;
    AML_REQUIRE((int64_t)((n_w + n) * ws_per_edge(st->P)) <= (int64_t)(st->budget / 2),
                AML_EADMIT, "the recount window exceeds the working-set half of the budget");
    // commit: evict, compact if needed, store the batch
    st->lo = new_lo;
    int64_t w0 = w_lo;
    if (st->hi + n > st->cap) {
      const int64_t shift = st->lo;
      compact(st, s);
      w0 -= shift;
    }
    const int64_t at = st->hi;
    cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    AML_CUDA(cudaMemcpyAsync(st->src + at, src, n * 4, kind, s));
    AML_CUDA(cudaMemcpyAsync(st->dst + at, dst, n * 4, kind, s));
    AML_CUDA(cudaMemcpyAsync(st->ts + at, ts, n * 4, kind, s));
    if (amount) AML_CUDA(cudaMemcpyAsync(st->amt + at, amount, n * 4, kind, s));
    else AML_CUDA(cudaMemsetAsync(st->amt + at, 0, n * 4, s));
    std::memcpy(st->hts.data() + at, ht.data(), n * 4);
    // recount: one delta-counting mine of W u B; old rows add their new
    // instances, batch rows are written outright
    mine_window(st, w0, n_w + n, (int32_t)n_w, t_first, st->counts + w0 * st->P, s);
    AML_CUDA(cudaStreamSynchronize(s));
    st->hi = at + n;
    st->any = true;
    st->t_max = t_last;
    if (info) {
      info->first_row = st->base + at;
      info->n_rows = n;
      info->rows_recounted = n_w;
      info->resident_first_row = st->base + st->lo;
      info->resident_rows = st->hi - st->lo;
    }
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_stream_append: ") + f.msg);
    return f.status;
  } catch (...) {
    set_error("aml_stream_append: unexpected internal error");
    return AML_EINTERNAL;
  }
}

aml_status aml_stream_read(aml_stream* st, int64_t row0, int64_t n, uint32_t* out, int64_t ld,
                           uint32_t flags, void* stream) {
  try {
    AML_REQUIRE(st != nullptr, AML_EINVAL, "NULL stream");
    AML_REQUIRE((flags & ~AML_MINE_HOST_OUTPUT) == 0, AML_EINVAL, "unknown flag bits");
    AML_REQUIRE(n >= 0 && ld >= st->P, AML_EINVAL, "bad n or ld");
    AML_REQUIRE(n == 0 || out != nullptr, AML_EINVAL, "out is NULL");
    const int64_t first = st->base + st->lo, end = st->base + st->hi;
    AML_REQUIRE(row0 >= first && row0 + n <= end, AML_EINVAL,
                "rows outside the resident range (evicted or not yet appended)");
    if (n == 0) return AML_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t* from = st->counts + (row0 - st->base) * st->P;
    const cudaMemcpyKind kind =
        (flags & AML_MINE_HOST_OUTPUT) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (ld == st->P)  // one contiguous copy (a pitched copy moves row by row)
      AML_CUDA(cudaMemcpyAsync(out, from, (size_t)(n * st->P) * 4, kind, s));
    else
      AML_CUDA(cudaMemcpy2DAsync(out, (size_t)ld * 4, from, (size_t)st->P * 4,
                                 (size_t)st->P * 4, (size_t)n, kind, s));
    if (flags & AML_MINE_HOST_OUTPUT) AML_CUDA(cudaStreamSynchronize(s));
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_stream_read: ") + f.msg);
    return f.status;
  }
}

aml_status aml_stream_get_info(const aml_stream* st, aml_stream_info* info) {
  if (!st || !info) {
    set_error("aml_stream_get_info: NULL argument");
    return AML_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  info->resident_first_row = st->base + st->lo;
  info->resident_rows = st->hi - st->lo;
  info->capacity_rows = st->cap;
  info->t_max = st->t_max;
  info->delta_max = st->delta_max;
  info->device_bytes = st->cap * (16 + 4 * (int64_t)st->P) + (st->g ? st->g->bytes : 0);
  // rows whose every instance window has closed: t_e + delta_max < t_max
  const int64_t lim = (int64_t)st->t_max - st->delta_max;
  int64_t k = std::lower_bound(st->hts.begin() + st->lo, st->hts.begin() + st->hi, lim,
                               [](int32_t a, int64_t b) { return (int64_t)a < b; }) -
              st->hts.begin();
  info->final_end_row = st->any ? st->base + k : st->base + st->lo;
  return AML_OK;
}

aml_status aml_stream_check_graph(aml_stream* st, int64_t* n_mismatch) {
  aml_graph* f = nullptr;
  try {
    AML_REQUIRE(st && n_mismatch, AML_EINVAL, "NULL argument");
    *n_mismatch = 0;
    const aml_graph* g = st->g;
    if (!g) return AML_OK;
    const int64_t w = st->g_first - st->base;
    AML_REQUIRE(w >= st->lo && w + g->E <= st->hi, AML_EINTERNAL,
                "the kept graph's rows are no longer resident");
    cudaStream_t s = nullptr;
    AML_CUDA(cudaDeviceSynchronize());
    f = build_graph(st->src + w, st->dst + w, st->ts + w, st->amt + w, g->E, st->N,
                    AML_PTR_DEVICE | AML_ASSUME_SORTED, s);
    if (f->Ev != g->Ev) {
      *n_mismatch = 1 + std::llabs(f->Ev - g->Ev);
    } else {
      DBuf<unsigned long long> diff(1, s);
      AML_CUDA(cudaMemsetAsync(diff.p, 0, 8, s));
      auto cmp = [&](const int32_t* a, const int32_t* b, int64_t n) {
        if (n > 0)
          AML_LAUNCH("k_count_diff", s,
                     k_count_diff<<<grid_for(n, 256), 256, 0, s>>>(a, b, n, diff.p));
      };
      const int64_t E = g->E, Ev = g->Ev, N1 = (int64_t)g->N + 1;
      cmp(f->src, g->src, E);
      cmp(f->dst, g->dst, E);
      cmp(f->ts, g->ts, E);
      cmp(reinterpret_cast<const int32_t*>(f->dts), reinterpret_cast<const int32_t*>(g->dts),
          2 * E);
      const Adj* fa[2] = {&f->out, &f->in};
      const Adj* ga[2] = {&g->out, &g->in};
      for (int d = 0; d < 2; ++d) {
        cmp(fa[d]->ptr, ga[d]->ptr, N1);
        cmp(fa[d]->pos, ga[d]->pos, E);
        cmp(fa[d]->nbr, ga[d]->nbr, Ev);
        cmp(fa[d]->t, ga[d]->t, Ev);
        cmp(fa[d]->eid, ga[d]->eid, Ev);
        cmp(fa[d]->rstart, ga[d]->rstart, Ev);
        cmp(fa[d]->prev, ga[d]->prev, Ev);
        cmp(fa[d]->next, ga[d]->next, Ev);
        cmp(fa[d]->nnbr, ga[d]->nnbr, Ev);
        cmp(fa[d]->nt, ga[d]->nt, Ev);
        cmp(fa[d]->neid, ga[d]->neid, Ev);
      }
      unsigned long long h = 0;
      AML_CUDA(cudaStreamSynchronize(s));
      AML_CUDA(cudaMemcpy(&h, diff.p, 8, cudaMemcpyDeviceToHost));
      *n_mismatch = (int64_t)h;
    }
    destroy_graph(f);
    return AML_OK;
  } catch (const Failure& e) {
    if (f) destroy_graph(f);
    set_error(std::string("aml_stream_check_graph: ") + e.msg);
    return e.status;
  }
}

aml_status aml_stream_set_count_limit(aml_stream* st, uint32_t limit) {
  if (!st || limit == 0) {
    set_error("aml_stream_set_count_limit: NULL stream or a limit of 0");
    return AML_EINVAL;
  }
  st->count_limit = limit;
  return AML_OK;
}

aml_status aml_stream_close(aml_stream* st) {
  if (st) {
    cudaDeviceSynchronize();
    free_stream(st);
  }
  return AML_OK;
}

}  // extern "C"
