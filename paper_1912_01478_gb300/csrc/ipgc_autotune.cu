// Schedule autotuner for the single-graph and batched colourings.
//
// The schedule (degree split t1, work-item size, CTA size, team size, the
// size from which a graph of a batch gets a team, and for batches whether
// forbidden colours are pushed into bitmaps or rows rescanned) changes only
// speed, never a colour, so it can be chosen by measurement. The tuner runs a coordinate
// descent from the caller's options: for each knob in turn it times every
// candidate value with the others fixed (best of `reps` launches, CUDA events
// on the caller's stream) and keeps the fastest. The batched tuner times the
// batch's first `sample_graphs` graphs, a contiguous prefix that is itself a
// valid batch, then times its choice and the caller's options on the whole
// batch and keeps the faster (a prefix need not pack like the whole batch).
#include <cfloat>
#include <cstring>
#include <vector>

#include "ipgc_internal.h"

namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  bool ok = false;
  Timer() { ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

template <class Run>
int time_best(Run run, cudaStream_t s, int reps, float* best) {
  Timer t;
  if (!t.ok) return IPGC_ERR_CUDA;
  *best = FLT_MAX;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(t.a, s) != cudaSuccess) return IPGC_ERR_CUDA;
    const int rc = run();
    if (rc != IPGC_OK) return rc;
    if (cudaEventRecord(t.b, s) != cudaSuccess || cudaEventSynchronize(t.b) != cudaSuccess)
      return IPGC_ERR_CUDA;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) return IPGC_ERR_CUDA;
    if (ms < *best) *best = ms;
  }
  return IPGC_OK;
}

// One knob: a setter and its candidate values.
template <class Opt>
struct Knob {
  void (*set)(Opt&, int64_t);
  std::vector<int64_t> values;
};

template <class Opt, class Run>
int descend(Opt* opt, const std::vector<Knob<Opt>>& knobs, Run run, cudaStream_t s, int reps,
            float* best_ms) {
  Opt best = *opt;
  float best_t = FLT_MAX;
  int rc = time_best([&] { return run(best); }, s, reps, &best_t);
  if (rc != IPGC_OK) return rc;
  for (const Knob<Opt>& k : knobs) {
    Opt here = best;
    for (int64_t v : k.values) {
      Opt cand = best;
      k.set(cand, v);
      float t = 0;
      rc = time_best([&] { return run(cand); }, s, reps, &t);
      if (rc != IPGC_OK) return rc;
      if (t < best_t) {
        best_t = t;
        here = cand;
      }
    }
    best = here;
  }
  *opt = best;
  if (best_ms) *best_ms = best_t;
  return IPGC_OK;
}

}  // namespace

extern "C" {

int ipgc_autotune(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                  int32_t* colors_scratch, int32_t reps, ipgc_options* opt, float* best_ms,
                  void* stream) {
  if (!ctx || !opt || reps < 1) return IPGC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  ipgc_options base = *opt;
  base.validate = 0;
  base.trace = nullptr;
  base.fin_round = nullptr;
  base.fault_inject = 0;
  std::vector<Knob<ipgc_options>> knobs = {
      {[](ipgc_options& o, int64_t v) { o.chunk = (int32_t)v; }, {256, 512, 1024, 2048, 4096}},
      {[](ipgc_options& o, int64_t v) { o.t1 = (int32_t)v; }, {16, 32, 64, 128, 255}},
      {[](ipgc_options& o, int64_t v) { o.block_size = (int32_t)v; }, {256, 512}},
  };
  const int rc = descend(
      &base, knobs,
      [&](const ipgc_options& o) {
        return ipgc_color_ex(ctx, rowptr, col, n, nnz, colors_scratch, nullptr, &o, stream);
      },
      s, reps, best_ms);
  if (rc != IPGC_OK) return rc;
  const int validate = opt->validate;
  ipgc_trace_rec* trace = opt->trace;
  int32_t* fin = opt->fin_round;
  *opt = base;
  opt->validate = validate;
  opt->trace = trace;
  opt->fin_round = fin;
  return IPGC_OK;
}

int ipgc_batched_autotune(ipgc_ctx* ctx, int32_t num_graphs, const int64_t* node_off,
                          const int64_t* edge_off, const int32_t* rowptr_cat, const int32_t* col_cat,
                          int32_t* colors_cat, int32_t sample_graphs, int32_t reps,
                          ipgc_batch_options* opt, float* best_ms, void* stream) {
  if (!ctx || !opt || reps < 1 || num_graphs < 0 || !node_off || !edge_off) return IPGC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t G = (sample_graphs > 0 && sample_graphs < num_graphs) ? sample_graphs : num_graphs;
  ipgc_batch_options base = *opt;
  const int validate = base.base.validate;
  base.base.validate = 0;
  std::vector<Knob<ipgc_batch_options>> knobs = {
      {[](ipgc_batch_options& o, int64_t v) { o.base.forbidden = (int32_t)v; },
       {IPGC_FORBIDDEN_AUTO, IPGC_FORBIDDEN_RESCAN}},
      {[](ipgc_batch_options& o, int64_t v) { o.base.chunk = (int32_t)v; }, {512, 1024, 2048}},
      {[](ipgc_batch_options& o, int64_t v) { o.base.t1 = (int32_t)v; }, {16, 32, 64, 128, 255}},
      {[](ipgc_batch_options& o, int64_t v) { o.nnz_per_cta = v; },
       {1 << 14, 1 << 16, 1 << 17, 1 << 18, 1 << 20, (int64_t)1 << 40}},
      {[](ipgc_batch_options& o, int64_t v) { o.max_team = (int32_t)v; }, {0, 4, 16, 64}},
      {[](ipgc_batch_options& o, int64_t v) { o.base.block_size = (int32_t)v; }, {256, 512}},
  };
  const ipgc_batch_options start = base;
  int rc = descend(
      &base, knobs,
      [&](const ipgc_batch_options& o) {
        return ipgc_color_batched(ctx, G, node_off, edge_off, rowptr_cat, col_cat, colors_cat,
                                  nullptr, &o, stream);
      },
      s, reps, best_ms);
  if (rc != IPGC_OK) return rc;
  if (G < num_graphs) {  // the choice against the caller's options, on every graph
    float t_tuned = 0, t_start = 0;
    auto whole = [&](const ipgc_batch_options& o) {
      return [&, o] {
        return ipgc_color_batched(ctx, num_graphs, node_off, edge_off, rowptr_cat, col_cat,
                                  colors_cat, nullptr, &o, stream);
      };
    };
    rc = time_best(whole(base), s, reps, &t_tuned);
    if (rc == IPGC_OK) rc = time_best(whole(start), s, reps, &t_start);
    if (rc != IPGC_OK) return rc;
    if (t_start < t_tuned) base = start;
    if (best_ms) *best_ms = t_start < t_tuned ? t_start : t_tuned;
  }
  base.base.validate = validate;
  *opt = base;
  return IPGC_OK;
}

}  // extern "C"
