// extern "C" entry points: argument checks, error mapping, dispatch.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aml_internal.cuh"
#include "mine.cuh"

namespace aml {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

aml_graph* build_graph(const int32_t* src, const int32_t* dst, const int32_t* ts,
                       const float* amount, int64_t E, int32_t N, uint32_t flags, cudaStream_t s);
void destroy_graph(aml_graph* g);
std::vector<Column> plan_patterns(const aml_pattern* pats, int n, std::vector<Prog>* progs);

template <typename F>
static aml_status guarded(const char* fn, F&& body) {
  try {
    body();
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string(fn) + ": " + f.msg);
    return f.status;
  } catch (const std::bad_alloc&) {
    set_error(std::string(fn) + ": host allocation failed");
    return AML_ENOMEM;
  } catch (...) {
    set_error(std::string(fn) + ": unexpected internal error");
    return AML_EINTERNAL;
  }
}

static const char* family_name(int f) {
  switch (f) {
    case AML_FAM_DEG_OUT: return "DEG_OUT";
    case AML_FAM_DEG_IN: return "DEG_IN";
    case AML_FAM_FAN_OUT: return "FAN_OUT";
    case AML_FAM_FAN_IN: return "FAN_IN";
    case AML_FAM_GS: return "GS";
    case AML_FAM_SG: return "SG";
    case AML_FAM_CYC: return "CYC";
    case AML_FAM_CYCW: return "CYCW";
    case AML_FAM_PROGRAM: return "PROGRAM";
    default: return "?";
  }
}

// Reads and clears the graph's device error word (the graph's stream must
// be idle or synchronized by the caller).
static void check_device_errors(aml_graph* g) {
  uint32_t err = 0;
  AML_CUDA(cudaMemcpy(&err, g->err, 4, cudaMemcpyDeviceToHost));
  if (!err) return;
  AML_CUDA(cudaMemset(g->err, 0, 4));
  AML_REQUIRE(!(err & ERR_TIMEOUT), AML_ETIMEOUT, "a bounded device wait gave up");
  AML_REQUIRE(false, AML_EINTERNAL, "device error word set (" + std::to_string(err) + ")");
}

}  // namespace aml

using namespace aml;

extern "C" {

const char* aml_status_str(aml_status s) {
  switch (s) {
    case AML_OK: return "AML_OK";
    case AML_EINVAL: return "AML_EINVAL";
    case AML_ENOMEM: return "AML_ENOMEM";
    case AML_ECUDA: return "AML_ECUDA";
    case AML_EUNSUPPORTED: return "AML_EUNSUPPORTED";
    case AML_EUNSORTED: return "AML_EUNSORTED";
    case AML_ELATE: return "AML_ELATE";
    case AML_EADMIT: return "AML_EADMIT";
    case AML_ETIMEOUT: return "AML_ETIMEOUT";
    case AML_EINTERNAL: return "AML_EINTERNAL";
    default: return "AML_UNKNOWN_STATUS";
  }
}

const char* aml_last_error(void) { return g_last_error.c_str(); }

int32_t aml_version(void) { return 10000 * 0 + 100 * 1 + 0; }

aml_status aml_graph_create(const int32_t* src, const int32_t* dst, const int32_t* ts,
                            const float* amount, int64_t n_edges, int32_t n_nodes,
                            uint32_t flags, void* stream, aml_graph** out) {
  return guarded("aml_graph_create", [&] {
    AML_REQUIRE(out != nullptr, AML_EINVAL, "out is NULL");
    AML_REQUIRE(n_edges >= 0 && n_edges < (int64_t)INT32_MAX, AML_EINVAL,
                "n_edges must be in [0, 2^31-1)");
    AML_REQUIRE(n_nodes >= 1 && n_nodes < INT32_MAX, AML_EINVAL, "n_nodes must be in [1, 2^31-1)");
    AML_REQUIRE(n_edges == 0 || (src && dst && ts), AML_EINVAL, "src/dst/ts must not be NULL");
    AML_REQUIRE((flags & ~(AML_PTR_DEVICE | AML_ASSUME_SORTED)) == 0, AML_EINVAL,
                "unknown flag bits");
    *out = build_graph(src, dst, ts, amount, n_edges, n_nodes, flags,
                       static_cast<cudaStream_t>(stream));
  });
}

aml_status aml_graph_destroy(aml_graph* g) {
  return guarded("aml_graph_destroy", [&] { destroy_graph(g); });
}

aml_status aml_graph_get_info(const aml_graph* gc, aml_graph_info* info) {
  return guarded("aml_graph_get_info", [&] {
    AML_REQUIRE(gc && info, AML_EINVAL, "NULL argument");
    aml_graph* g = const_cast<aml_graph*>(gc);  // caches the degree read below
    if (g->max_out < 0) {
      int32_t md[2] = {0, 0};
      AML_CUDA(cudaStreamSynchronize(g->last_stream));
      AML_CUDA(cudaMemcpy(md, g->max_deg, 8, cudaMemcpyDeviceToHost));
      g->max_out = md[0];
      g->max_in = md[1];
    }
    std::memset(info, 0, sizeof(*info));
    info->n_edges = g->E;
    info->n_list_edges = g->Ev;
    info->n_nodes = g->N;
    info->max_out_degree = g->max_out;
    info->max_in_degree = g->max_in;
    info->device_bytes = g->bytes;
  });
}

aml_status aml_graph_window_stats(const aml_graph* g, int32_t delta, int64_t* n_legs,
                                  int64_t* n_front) {
  return guarded("aml_graph_window_stats", [&] {
    AML_REQUIRE(g && n_legs && n_front, AML_EINVAL, "NULL argument");
    static_assert(AML_MAX_CYCLE == MAX_CYCLE, "cycle limit of the ABI and the kernels");
    *n_legs = -1;
    for (int j = 0; j <= MAX_CYCLE; ++j) n_front[j] = -1;
    auto it = g->legs.find(delta);
    if (it == g->legs.end()) return;
    *n_legs = it->second.n_legs;
    for (int j = 2; j <= MAX_CYCLE; ++j) n_front[j] = it->second.n_front[j];
  });
}

aml_status aml_pattern_set_create(const aml_pattern* patterns, int32_t n_patterns,
                                  aml_pattern_set** out) {
  return guarded("aml_pattern_set_create", [&] {
    AML_REQUIRE(out != nullptr, AML_EINVAL, "out is NULL");
    AML_REQUIRE(n_patterns <= MAX_COLS, AML_EUNSUPPORTED, "at most 64 patterns per set");
    std::vector<Prog> progs;
    std::vector<Column> cols = plan_patterns(patterns, n_patterns, &progs);
    static std::atomic<uint64_t> next_id{1};
    aml_pattern_set* ps = new aml_pattern_set();
    ps->cols = std::move(cols);
    ps->progs = std::move(progs);
    ps->id = next_id.fetch_add(1);
    *out = ps;
  });
}

aml_status aml_pattern_set_destroy(aml_pattern_set* ps) {
  delete ps;
  return AML_OK;
}

aml_status aml_pattern_set_num_columns(const aml_pattern_set* ps, int32_t* n_cols) {
  return guarded("aml_pattern_set_num_columns", [&] {
    AML_REQUIRE(ps && n_cols, AML_EINVAL, "NULL argument");
    *n_cols = (int32_t)ps->cols.size();
  });
}

aml_status aml_pattern_set_column(const aml_pattern_set* ps, int32_t col, aml_column_info* info) {
  return guarded("aml_pattern_set_column", [&] {
    AML_REQUIRE(ps && info, AML_EINVAL, "NULL argument");
    AML_REQUIRE(col >= 0 && col < (int32_t)ps->cols.size(), AML_EINVAL, "column out of range");
    const Column& c = ps->cols[col];
    std::memset(info, 0, sizeof(*info));
    info->family = c.family;
    info->k = c.k;
    info->delta = c.delta;
    if (c.family == AML_FAM_CYC || c.family == AML_FAM_CYCW)
      std::snprintf(info->name, sizeof(info->name), "%s%d@%d", family_name(c.family), c.k,
                    c.delta);
    else if (c.family == AML_FAM_PROGRAM)  // numbered by column
      std::snprintf(info->name, sizeof(info->name), "%s%d@%d", family_name(c.family), col,
                    c.delta);
    else
      std::snprintf(info->name, sizeof(info->name), "%s@%d", family_name(c.family), c.delta);
  });
}

aml_status aml_mine(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                    uint32_t flags, void* stream) {
  return guarded("aml_mine", [&] {
    AML_REQUIRE(g && ps, AML_EINVAL, "NULL graph or pattern set");
    AML_REQUIRE((flags & ~(AML_MINE_HOST_OUTPUT | AML_MINE_GRAPH | AML_MINE_PERSISTENT |
                           AML_MINE_LEARNED | AML_MINE_HOST_ASYNC | AML_MINE_FUSED)) == 0,
                AML_EINVAL, "unknown flag bits");
    AML_REQUIRE(!((flags & AML_MINE_FUSED) && (flags & (AML_MINE_PERSISTENT | AML_MINE_LEARNED))),
                AML_EINVAL, "AML_MINE_FUSED excludes AML_MINE_PERSISTENT and AML_MINE_LEARNED");
    AML_REQUIRE(!(flags & AML_MINE_HOST_ASYNC) || (flags & AML_MINE_HOST_OUTPUT), AML_EINVAL,
                "AML_MINE_HOST_ASYNC needs AML_MINE_HOST_OUTPUT");
    const uint32_t mode = flags & (AML_MINE_PERSISTENT | AML_MINE_LEARNED | AML_MINE_FUSED);
    AML_REQUIRE(!((flags & AML_MINE_GRAPH) && (flags & AML_MINE_HOST_OUTPUT)), AML_EINVAL,
                "AML_MINE_GRAPH needs a device output");
    AML_REQUIRE(!(flags & AML_MINE_GRAPH) || ps->progs.empty(), AML_EUNSUPPORTED,
                "interpreted stage programs are not captured (AML_MINE_GRAPH)");
    const int64_t P = (int64_t)ps->cols.size();
    AML_REQUIRE(ld >= P, AML_EINVAL, "ld must be >= the number of columns");
    AML_REQUIRE(g->E == 0 || counts != nullptr, AML_EINVAL, "counts is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->note_stream(s);
    if (flags & AML_MINE_HOST_ASYNC) {  // the copy must not fall back to a synchronous one
      cudaPointerAttributes at;
      AML_CUDA(cudaPointerGetAttributes(&at, counts));
      AML_REQUIRE(at.type == cudaMemoryTypeHost, AML_EINVAL,
                  "AML_MINE_HOST_ASYNC needs page-locked host memory");
    }
    if (flags & AML_MINE_HOST_OUTPUT) {
      DBuf<uint32_t> dev((size_t)(g->E * P), s);
      mine_plain(g, ps, dev.p, P, s, mode);
      if (g->E && ld == P)  // one contiguous copy (a pitched copy moves row by row)
        AML_CUDA(cudaMemcpyAsync(counts, dev.p, (size_t)(g->E * P) * 4, cudaMemcpyDeviceToHost,
                                 s));
      else if (g->E)
        AML_CUDA(cudaMemcpy2DAsync(counts, (size_t)ld * 4, dev.p, (size_t)P * 4, (size_t)P * 4,
                                   (size_t)g->E, cudaMemcpyDeviceToHost, s));
      // the staging buffer is released in stream order after the copy
      if (!(flags & AML_MINE_HOST_ASYNC)) AML_CUDA(cudaStreamSynchronize(s));
    } else if (flags & AML_MINE_GRAPH) {
      mine_graph_mode(g, ps, counts, ld, s, mode);
    } else {
      mine_plain(g, ps, counts, ld, s, mode);
    }
  });
}

aml_status aml_sync(aml_graph* g) {
  return guarded("aml_sync", [&] {
    AML_REQUIRE(g != nullptr, AML_EINVAL, "NULL graph");
    AML_CUDA(cudaStreamSynchronize(g->last_stream));
    AML_CUDA(cudaGetLastError());
    check_device_errors(g);
  });
}

}  // extern "C"
