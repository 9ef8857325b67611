// Whole-mine CUDA graphs (AML_MINE_GRAPH) and the autotuner.
//
// A captured mine is the full kernel sequence of mine_plain recorded once on
// a private stream (its scratch allocations become graph memory nodes) and
// replayed with one cudaGraphLaunch per call.  The autotuner times real mines
// of the caller's graph and pattern set under candidate tunables (coordinate
// descent: one tunable at a time, the others held at their best so far) and
// keeps the fastest; no tunable changes any count.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

void drop_captured_mines(aml_graph* g) {
  for (MineExec& m : g->execs) cudaGraphExecDestroy(m.exec);
  g->execs.clear();
}

void mine_graph_mode(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                     cudaStream_t s, uint32_t mode) {
  for (const MineExec& m : g->execs) {
    if (m.flags == mode && m.ps_id == ps->id && m.counts == counts && m.ld == ld &&
        m.tune_gen == g->tune_gen) {
      AML_CUDA(cudaGraphLaunch(m.exec, s));
      add_launches(m.n_kernels);
      return;
    }
  }
  // this call's result comes from a plain mine, which also learns every
  // buffer size the capture needs (so the captured sequence never waits)
  mine_plain(g, ps, counts, ld, s, mode);
  if (!g->capture_stream)
    AML_CUDA(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = g->capture_stream;
  cudaGraph_t graph = nullptr;
  const long long before = launch_count();
  AML_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  try {
    mine_plain(g, ps, counts, ld, cs, mode);
  } catch (...) {
    cudaStreamEndCapture(cs, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  AML_CUDA(cudaStreamEndCapture(cs, &graph));
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  AML_CUDA(e);
  g->execs.push_back(MineExec{mode, ps->id, counts, ld, g->tune_gen, exec,
                              (long long)(launch_count() - before)});
}

static void check_tuning(const aml_tuning& t) {
  AML_REQUIRE(t.own_max >= 0 && t.own_max <= 4096, AML_EINVAL, "own_max must be in [0, 4096]");
  AML_REQUIRE(t.sg_bucket_mean >= 16 && t.sg_bucket_mean <= 512, AML_EINVAL,
              "sg_bucket_mean must be in [16, 512]");
  AML_REQUIRE(t.close_scan_max >= 0 && t.close_scan_max <= 4096, AML_EINVAL,
              "close_scan_max must be in [0, 4096]");
  AML_REQUIRE(t.block == 64 || t.block == 128 || t.block == 256 || t.block == 512, AML_EINVAL,
              "block must be 64, 128, 256 or 512");
}

static void put_tuning(aml_graph* g, const aml_tuning& t) {
  g->tune.own_max = t.own_max;
  g->tune.sg_bucket_mean = t.sg_bucket_mean;
  g->tune.close_scan_max = t.close_scan_max;
  g->tune.block = t.block;
  ++g->tune_gen;
  drop_captured_mines(g);
}

static aml_tuning get_tuning(const aml_graph* g) {
  aml_tuning t;
  std::memset(&t, 0, sizeof(t));
  t.own_max = g->tune.own_max;
  t.sg_bucket_mean = g->tune.sg_bucket_mean;
  t.close_scan_max = g->tune.close_scan_max;
  t.block = g->tune.block;
  return t;
}

// median device time of `reps` mines (after one untimed mine)
static float time_mines(aml_graph* g, const aml_pattern_set* ps, uint32_t* out, int64_t ld,
                        int reps, cudaStream_t s) {
  mine_plain(g, ps, out, ld, s);
  std::vector<float> ms;
  cudaEvent_t a, b;
  AML_CUDA(cudaEventCreate(&a));
  AML_CUDA(cudaEventCreate(&b));
  for (int r = 0; r < reps; ++r) {
    AML_CUDA(cudaEventRecord(a, s));
    mine_plain(g, ps, out, ld, s);
    AML_CUDA(cudaEventRecord(b, s));
    AML_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    AML_CUDA(cudaEventElapsedTime(&t, a, b));
    ms.push_back(t);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(ms.begin(), ms.end());
  return ms[ms.size() / 2];
}

void autotune(aml_graph* g, const aml_pattern_set* ps, int reps, cudaStream_t s,
              aml_tuning* best_out, float* best_ms_out) {
  const int64_t P = (int64_t)ps->cols.size();
  DBuf<uint32_t> out((size_t)std::max<int64_t>(g->E * P, 1), s);
  aml_tuning best = get_tuning(g);
  float best_ms = time_mines(g, ps, out.p, P, reps, s);
  const std::vector<int> blocks = {128, 256, 512};
  const std::vector<int> owns = {16, 32, 128, 512};
  const std::vector<int> buckets = {96, 128, 192, 256};
  const std::vector<int> scans = {16, 48, 128};
  auto sweep = [&](int aml_tuning::*field, const std::vector<int>& cands) {
    for (int v : cands) {
      aml_tuning t = best;
      if (t.*field == v) continue;
      t.*field = v;
      put_tuning(g, t);
      float ms = time_mines(g, ps, out.p, P, reps, s);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    put_tuning(g, best);
  };
  sweep(&aml_tuning::block, blocks);
  sweep(&aml_tuning::own_max, owns);
  sweep(&aml_tuning::sg_bucket_mean, buckets);
  sweep(&aml_tuning::close_scan_max, scans);
  AML_CUDA(cudaStreamSynchronize(s));
  if (best_out) *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
}

}  // namespace aml

using namespace aml;

extern "C" {

aml_status aml_graph_get_tuning(const aml_graph* g, aml_tuning* out) {
  if (!g || !out) {
    set_error("aml_graph_get_tuning: NULL argument");
    return AML_EINVAL;
  }
  *out = get_tuning(g);
  return AML_OK;
}

aml_status aml_graph_set_tuning(aml_graph* g, const aml_tuning* t) {
  try {
    AML_REQUIRE(g && t, AML_EINVAL, "NULL argument");
    check_tuning(*t);
    put_tuning(g, *t);
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_graph_set_tuning: ") + f.msg);
    return f.status;
  }
}

aml_status aml_graph_set_count_limit(aml_graph* g, uint32_t limit) {
  if (!g || limit == 0) {
    set_error("aml_graph_set_count_limit: NULL graph or a limit of 0");
    return AML_EINVAL;
  }
  if (g->count_limit != limit) {
    g->count_limit = limit;
    drop_captured_mines(g);  // their row assembly holds the old bound
  }
  return AML_OK;
}

aml_status aml_graph_set_wait_limit(aml_graph* g, int64_t cycles) {
  if (!g || cycles < 0) {
    set_error("aml_graph_set_wait_limit: NULL graph or a negative limit");
    return AML_EINVAL;
  }
  if (g->wait_limit != cycles) {
    g->wait_limit = cycles;
    drop_captured_mines(g);  // their launches hold the old bound
  }
  return AML_OK;
}

aml_status aml_autotune(aml_graph* g, const aml_pattern_set* ps, int32_t repeats, void* stream,
                        aml_tuning* best, float* best_ms) {
  try {
    AML_REQUIRE(g && ps, AML_EINVAL, "NULL graph or pattern set");
    AML_REQUIRE(repeats >= 1 && repeats <= 100, AML_EINVAL, "repeats must be in [1, 100]");
    g->note_stream(static_cast<cudaStream_t>(stream));
    autotune(g, ps, repeats, static_cast<cudaStream_t>(stream), best, best_ms);
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_autotune: ") + f.msg);
    return f.status;
  } catch (...) {
    set_error("aml_autotune: unexpected internal error");
    return AML_EINTERNAL;
  }
}

}  // extern "C"
