// Batched form: many independent systems of very uneven sizes evaluated by one
// persistent work-stealing launch, the whole sequence (every system's metric
// pipeline, then the batched evaluation) captured once in a CUDA graph and
// replayed.  The method-chunk size of the evaluation tiles is chosen by a
// small autotuner (timed trials, cached per batch shape in the process).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mm_internal.cuh"

void build_structures(mm_system *s);
void build_move_precompute(mm_system *s);

struct mm_batch {
  std::vector<mm_system *> sys;
  int32_t n = 0;
  mm_criteria crit{};
  cudaStream_t stream = nullptr;       // the batch's own stream (capture needs a non-default stream)
  cudaStream_t user_stream = nullptr;  // the caller's stream, ordered against ours with events
  cudaEvent_t ev = nullptr;
  // the systems' metric pipelines run as parallel branches on these streams
  static constexpr int kSide = 16;
  cudaStream_t side[kSide] = {};
  cudaEvent_t side_ev[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  int device = 0;
  int64_t kept_cap = 0;
  int32_t mchunk = 256;
  int grid = 0;
  int64_t total_tiles = 0;
  // device memory (one allocation)
  void *mem = nullptr;
  void *d_items = nullptr;
  unsigned long long *d_next = nullptr, *d_digest = nullptr, *d_kcount = nullptr, *d_tmp = nullptr;
  uint32_t *d_fault = nullptr;  // fault word of the bounded waits inside the batch's graph
  mm_move *d_kept = nullptr;
  uint8_t *d_marks = nullptr;
  std::vector<int64_t> mark_off;
  int64_t marks_bytes = 0;
  // graphs of (metrics of every system + batched evaluation + per-system sort),
  // without [0] and with [1] the record digests
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<std::vector<void *>> scratch_at_capture;  // scratch buffers of each system at capture
  bool ran = false;
};

namespace {

std::mutex g_tune_mu;
// per batch shape: {methods per tile, persistent blocks}
std::map<std::tuple<int32_t, int64_t, int64_t, uint32_t, int32_t>, std::pair<int32_t, int32_t>> g_tune_cache;

std::tuple<int32_t, int64_t, int64_t, uint32_t, int32_t> tune_key(const mm_batch *b) {
  int64_t sc = 0, sm = 0;
  for (auto *s : b->sys) { sc += s->c; sm += s->M; }
  return std::make_tuple(b->n, sc, sm, b->crit.metric_mask, b->crit.min_improved);
}

// order: our stream after the caller's work, or the caller's stream after ours
void join(cudaStream_t waiter, cudaStream_t producer, cudaEvent_t ev) {
  if (waiter == producer) return;
  MM_CUDA_TRY(cudaEventRecord(ev, producer));
  MM_CUDA_TRY(cudaStreamWaitEvent(waiter, ev, 0));
}

template <class F>
mm_status guarded(F &&f) {
  try {
    f();
    mm_set_error("");
    return MM_OK;
  } catch (const MmError &e) {
    mm_set_error(e.msg);
    return e.st;
  } catch (...) {
    mm_set_error("unexpected exception");
    return MM_ECUDA;
  }
}

void fill_and_upload_items(mm_batch *b) {
  std::vector<BatchLaunchSpec> specs(b->n);
  for (int32_t i = 0; i < b->n; ++i) {
    specs[i].sys = b->sys[i];
    specs[i].digest = b->d_digest + i;
    specs[i].kept = b->d_kept + (int64_t)i * b->kept_cap;
    specs[i].kept_count = b->d_kcount + i;
    specs[i].kept_mark = b->d_marks + b->mark_off[i];
  }
  std::vector<unsigned char> host(batch_item_bytes() * (size_t)b->n);
  batch_fill_items(specs.data(), b->n, b->crit, b->mchunk, b->kept_cap, host.data(), &b->total_tiles);
  MM_CUDA_TRY(cudaMemcpyAsync(b->d_items, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream));
  MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
}

// Enqueue the evaluation part (counters reset + the persistent launch), then
// sort every system's kept moves that fit one block.
void enqueue_eval(mm_batch *b, bool digest) {
  MM_CUDA_TRY(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), b->stream));
  MM_CUDA_TRY(cudaMemsetAsync(b->d_digest, 0, sizeof(unsigned long long) * b->n, b->stream));
  MM_CUDA_TRY(cudaMemsetAsync(b->d_kcount, 0, sizeof(unsigned long long) * b->n, b->stream));
  if (b->marks_bytes) MM_CUDA_TRY(cudaMemsetAsync(b->d_marks, 0, (size_t)b->marks_bytes, b->stream));
  batch_launch(b->d_items, b->n, b->total_tiles, b->mchunk, b->kept_cap > 0, digest, b->d_next, b->grid,
               b->stream);
  if (b->kept_cap > 0) sort_moves_segments(b->d_kept, b->kept_cap, b->d_kcount, b->n, b->stream);
}

// Enqueue every system's metric pipeline: the systems are independent, so they
// are spread over the side streams (parallel branches when captured) and
// joined back into the batch stream.
void enqueue_metrics(mm_batch *b) {
  MM_CUDA_TRY(cudaEventRecord(b->fork_ev, b->stream));
  for (int j = 0; j < mm_batch::kSide; ++j) MM_CUDA_TRY(cudaStreamWaitEvent(b->side[j], b->fork_ev, 0));
  for (size_t i = 0; i < b->sys.size(); ++i) {
    mm_system *s = b->sys[i];
    cudaStream_t lane = b->side[i % mm_batch::kSide];
    cudaStream_t own = s->stream;
    s->stream = lane;
    s->arena.stream = lane;
    try {
      s->kept_valid = false;
      build_structures(s);
      build_metrics(s);
      build_move_precompute(s);
      s->metrics_ready = true;
    } catch (...) {
      s->stream = own;
      s->arena.stream = own;
      throw;
    }
    s->stream = own;
    s->arena.stream = own;
  }
  for (int j = 0; j < mm_batch::kSide; ++j) {
    MM_CUDA_TRY(cudaEventRecord(b->side_ev[j], b->side[j]));
    MM_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->side_ev[j], 0));
  }
}

// The scratch buffers the metric pipeline uses (their addresses are baked into
// a captured graph).
std::vector<void *> pipeline_scratch(const mm_system *s) {
  return {s->sort_ws.ptr,       s->eval_ws.ptr,       s->union_ws.ptr,      s->side_eval[0].ptr,
          s->side_eval[1].ptr,  s->side_eval[2].ptr,  s->side_sort[0].ptr,  s->side_sort[1].ptr,
          s->side_sort[2].ptr,  s->side_union[0].ptr, s->side_union[1].ptr, s->side_union[2].ptr};
}

bool scratch_moved(const mm_batch *b) {
  if (b->scratch_at_capture.size() != b->sys.size()) return true;
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (b->scratch_at_capture[i] != pipeline_scratch(b->sys[i])) return true;
  return false;
}

void drop_graph(mm_batch *b) {
  for (auto &e : b->exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
}

void capture(mm_batch *b, bool digest) {
  WaitScope wait(b->d_fault, nullptr);  // the graph's scans record into the batch's word
  if (b->exec[digest]) cudaGraphExecDestroy(b->exec[digest]);
  b->exec[digest] = nullptr;
  // run once outside capture so every scratch buffer already has its size; the
  // recorded buffer addresses let a later run notice reallocation
  enqueue_metrics(b);
  MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  cudaGraph_t g = nullptr;
  MM_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue_metrics(b);
    enqueue_eval(b, digest);
  } catch (...) {
    cudaStreamEndCapture(b->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  MM_CUDA_TRY(cudaStreamEndCapture(b->stream, &g));
  cudaError_t e = cudaGraphInstantiate(&b->exec[digest], g, 0);
  cudaGraphDestroy(g);
  MM_CUDA_TRY(e);
  b->scratch_at_capture.clear();
  for (auto *s : b->sys) b->scratch_at_capture.push_back(pipeline_scratch(s));
}

}  // namespace

extern "C" {

MMREF_API mm_status mm_batch_create(mm_system *const *systems, int32_t n, const mm_criteria *crit,
                                    int64_t kept_cap, void *cuda_stream, mm_batch **out) {
  if (out) *out = nullptr;
  mm_batch *b = nullptr;
  mm_status st = guarded([&] {
    if (!systems || n < 1 || !crit || !out || kept_cap < 0)
      throw MmError{MM_EINVAL, "batch_create: bad arguments"};
    check_criteria_public(*crit);
    b = new mm_batch();
    MM_CUDA_TRY(cudaGetDevice(&b->device));
    b->n = n;
    b->crit = *crit;
    b->user_stream = static_cast<cudaStream_t>(cuda_stream);
    MM_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
    for (int j = 0; j < mm_batch::kSide; ++j) {
      MM_CUDA_TRY(cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking));
      MM_CUDA_TRY(cudaEventCreateWithFlags(&b->side_ev[j], cudaEventDisableTiming));
    }
    MM_CUDA_TRY(cudaDeviceSynchronize());  // the systems' loads and earlier work are complete
    b->kept_cap = kept_cap;
    for (int32_t i = 0; i < n; ++i) {
      if (!systems[i]) throw MmError{MM_EINVAL, "batch_create: NULL system"};
      if (systems[i]->device != b->device) throw MmError{MM_EINVAL, "batch_create: systems on another device"};
      use_bitset_coupling(systems[i]);  // the captured dense evaluation reads the bitsets
      b->sys.push_back(systems[i]);
    }
    b->mark_off.resize(n);
    int64_t off = 0;
    for (int32_t i = 0; i < n; ++i) { b->mark_off[i] = off; off += (b->sys[i]->M + 15) / 16 * 16; }
    b->marks_bytes = off;
    size_t items = (batch_item_bytes() * (size_t)n + 255) / 256 * 256;
    size_t ctr = (sizeof(unsigned long long) * (size_t)(4 * n + 8) + 255) / 256 * 256;
    size_t kept = sizeof(mm_move) * (size_t)(kept_cap * n);
    size_t total = items + ctr + kept + (size_t)off + 256;
    MM_CUDA_TRY(cudaMallocAsync(&b->mem, total, b->stream));
    char *p = static_cast<char *>(b->mem);
    b->d_items = p;
    p += items;
    unsigned long long *c = reinterpret_cast<unsigned long long *>(p);
    b->d_next = c;
    b->d_fault = reinterpret_cast<uint32_t *>(c + 7);
    MM_CUDA_TRY(cudaMemsetAsync(b->d_fault, 0, sizeof(uint32_t), b->stream));
    b->d_digest = c + 8;
    b->d_kcount = c + 8 + n;
    b->d_tmp = c + 8 + 2 * n;
    p += ctr;
    b->d_kept = reinterpret_cast<mm_move *>(p);
    p += kept;
    b->d_marks = reinterpret_cast<uint8_t *>(p);
    b->grid = batch_persistent_grid();
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(tune_key(b));
      if (it != g_tune_cache.end()) {
        b->mchunk = it->second.first;
        b->grid = it->second.second;
      }
    }
    fill_and_upload_items(b);
    *out = b;
  });
  if (st != MM_OK && b) {
    if (b->mem) cudaFreeAsync(b->mem, b->stream);
    if (b->stream) { cudaStreamSynchronize(b->stream); cudaStreamDestroy(b->stream); }
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (int j = 0; j < mm_batch::kSide; ++j) {
      if (b->side[j]) cudaStreamDestroy(b->side[j]);
      if (b->side_ev[j]) cudaEventDestroy(b->side_ev[j]);
    }
    delete b;
  }
  return st;
}

MMREF_API mm_status mm_batch_set_tile(mm_batch *b, int32_t mchunk) {
  return guarded([&] {
    if (!b || mchunk < 1) throw MmError{MM_EINVAL, "batch_set_tile: bad arguments"};
    b->mchunk = mchunk;
    fill_and_upload_items(b);
    drop_graph(b);
  });
}

MMREF_API mm_status mm_batch_autotune(mm_batch *b, int32_t *chosen) {
  return guarded([&] {
    if (!b) throw MmError{MM_EINVAL, "batch_autotune: NULL batch"};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(tune_key(b));
      if (it != g_tune_cache.end()) {
        b->mchunk = it->second.first;
        b->grid = it->second.second;
        fill_and_upload_items(b);
        drop_graph(b);
        if (chosen) *chosen = b->mchunk;
        return;
      }
    }
    // metrics must exist for the trial evaluations
    join(b->stream, b->user_stream, b->ev);
    enqueue_metrics(b);
    MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    // two stages: methods per tile with every resident block, then the number
    // of persistent blocks (the launch shape) for the best tile
    const int32_t trials[] = {32, 64, 128, 256, 512, 1024};
    const int32_t full = batch_persistent_grid();
    cudaEvent_t e0, e1;
    MM_CUDA_TRY(cudaEventCreate(&e0));
    MM_CUDA_TRY(cudaEventCreate(&e1));
    auto time_eval = [&]() {
      fill_and_upload_items(b);
      enqueue_eval(b, false);  // warm
      float ms_sum = 0;
      for (int rep = 0; rep < 2; ++rep) {
        MM_CUDA_TRY(cudaEventRecord(e0, b->stream));
        enqueue_eval(b, false);
        MM_CUDA_TRY(cudaEventRecord(e1, b->stream));
        MM_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        MM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        ms_sum += ms;
      }
      return ms_sum;
    };
    float best = 1e30f;
    int32_t best_m = b->mchunk, best_g = full;
    b->grid = full;
    for (int32_t mc : trials) {
      b->mchunk = mc;
      const float ms = time_eval();
      if (ms < best) { best = ms; best_m = mc; }
    }
    b->mchunk = best_m;
    int sms = B300_SMS;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const int32_t per_sm = std::max(1, full / std::max(sms, 1));
    for (int32_t k = 1; k < per_sm; ++k) {  // fewer blocks per SM than the occupancy limit
      b->grid = full / per_sm * k;
      const float ms = time_eval();
      if (ms < best) { best = ms; best_g = b->grid; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->mchunk = best_m;
    b->grid = best_g;
    fill_and_upload_items(b);
    drop_graph(b);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[tune_key(b)] = std::make_pair(best_m, best_g);
    }
    if (chosen) *chosen = best_m;
  });
}

MMREF_API mm_status mm_batch_config_get(const mm_batch *b, int32_t *methods_per_tile, int32_t *blocks) {
  return guarded([&] {
    if (!b) throw MmError{MM_EINVAL, "batch_config_get: NULL batch"};
    if (methods_per_tile) *methods_per_tile = b->mchunk;
    if (blocks) *blocks = b->grid;
  });
}

MMREF_API mm_status mm_batch_run(mm_batch *b, uint64_t *digests, int64_t *n_kept) {
  return guarded([&] {
    if (!b) throw MmError{MM_EINVAL, "batch_run: NULL batch"};
    int cur = -1;
    MM_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != b->device) MM_CUDA_TRY(cudaSetDevice(b->device));
    join(b->stream, b->user_stream, b->ev);
    const bool dg = digests != nullptr;
    if (scratch_moved(b)) drop_graph(b);
    if (!b->exec[dg]) capture(b, dg);
    MM_CUDA_TRY(cudaGraphLaunch(b->exec[dg], b->stream));
    if (digests)
      MM_CUDA_TRY(cudaMemcpyAsync(digests, b->d_digest, sizeof(uint64_t) * b->n, cudaMemcpyDeviceToHost, b->stream));
    std::vector<unsigned long long> kc(b->n);
    MM_CUDA_TRY(cudaMemcpyAsync(kc.data(), b->d_kcount, sizeof(unsigned long long) * b->n, cudaMemcpyDeviceToHost,
                                b->stream));
    uint32_t hfault = 0;
    read_wait_fault(&hfault, b->d_fault, b->stream);
    MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    raise_wait_fault(hfault, b->d_fault, b->stream, "batch_run");
    if (n_kept)
      for (int32_t i = 0; i < b->n; ++i) n_kept[i] = (int64_t)kc[i];
    join(b->user_stream, b->stream, b->ev);
    b->ran = true;
    if (cur != b->device) cudaSetDevice(cur);
  });
}

MMREF_API mm_status mm_batch_suggestions(mm_batch *b, int32_t i, int32_t k, mm_move *out_topk, int32_t out_kind,
                                         int64_t *n_kept) {
  return guarded([&] {
    if (!b || i < 0 || i >= b->n || k < 0 || (k > 0 && !out_topk))
      throw MmError{MM_EINVAL, "batch_suggestions: bad arguments"};
    if (out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE) throw MmError{MM_EINVAL, "batch_suggestions: bad out_kind"};
    if (!b->ran) throw MmError{MM_EINVAL, "batch_suggestions: call mm_batch_run first"};
    WaitScope wait(b->d_fault, nullptr);  // reported by the batch's next run
    join(b->stream, b->user_stream, b->ev);
    unsigned long long K = 0;
    MM_CUDA_TRY(cudaMemcpyAsync(&K, b->d_kcount + i, sizeof(K), cudaMemcpyDeviceToHost, b->stream));
    MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (n_kept) *n_kept = (int64_t)K;
    if ((int64_t)K > b->kept_cap)
      throw MmError{MM_EBUDGET, "batch_suggestions: kept moves exceed the batch's per-system capacity; use "
                                "mm_suggest_moves on that system"};
    mm_system *s = b->sys[i];
    mm_move *kept = b->d_kept + (int64_t)i * b->kept_cap;
    if ((int64_t)K > kSegmentSortMax) {  // not sorted inside the graph
      cudaStream_t own = s->stream;
      s->stream = b->stream;
      try {
        sort_kept_moves(s, kept, (int64_t)K);
      } catch (...) {
        s->stream = own;
        throw;
      }
      s->stream = own;
    }
    int64_t nout = std::min<int64_t>(k, (int64_t)K);
    if (nout > 0)
      MM_CUDA_TRY(cudaMemcpyAsync(out_topk, kept, sizeof(mm_move) * (size_t)nout,
                                  out_kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  b->stream));
    MM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  });
}

MMREF_API void mm_batch_free(mm_batch *b) {
  if (!b) return;
  drop_graph(b);
  if (b->mem) cudaFreeAsync(b->mem, b->stream);
  cudaStreamSynchronize(b->stream);
  cudaStreamDestroy(b->stream);
  cudaEventDestroy(b->ev);
  cudaEventDestroy(b->fork_ev);
  for (int j = 0; j < mm_batch::kSide; ++j) {
    cudaStreamSynchronize(b->side[j]);
    cudaStreamDestroy(b->side[j]);
    cudaEventDestroy(b->side_ev[j]);
  }
  delete b;
}

}  // extern "C"
