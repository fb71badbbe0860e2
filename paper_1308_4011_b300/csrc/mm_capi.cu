// C ABI entry points (include/mmref.h): argument checks, allocation of a
// system's device memory, stream handling and error reporting.  Every step of
// the path itself runs in the kernels of mm_system.cu, mm_metrics.cu and
// mm_moves.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "mm_internal.cuh"

static thread_local std::string g_last_error;

void mm_set_error(const std::string &msg) { g_last_error = msg; }

#include <atomic>
static std::atomic<long long> g_launches{0};
void mm_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

template <class F>
mm_status guarded(F &&f) {
  try {
    f();
    g_last_error.clear();
    return MM_OK;
  } catch (const MmError &e) {
    g_last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return MM_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected exception";
    return MM_ECUDA;
  }
}

void use_device(mm_system *s) {
  int cur = -1;
  MM_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != s->device) MM_CUDA_TRY(cudaSetDevice(s->device));
}

// For the duration of an entry point: the system's device is current and its
// fault word receives the bounded waits that run out.
struct SystemScope {
  explicit SystemScope(mm_system *s) : wait(s->d_fault, &s->test_stall_scans) { use_device(s); }
  WaitScope wait;
};

// Free everything a system holds: device memory in stream order on its stream,
// then its events (released by the runtime once their last use completes).
void release_system(mm_system *s) {
  if (s->lists_staged) cudaStreamWaitEvent(s->stream, s->stage_ev, 0);  // a staged copy may still write lists_ws
  s->arena.release();
  for (Scratch *w : {&s->sort_ws, &s->eval_ws, &s->stage_ws, &s->kept_ws, &s->keyed_ws, &s->edit_ws, &s->sim_ws,
                     &s->sim_keys_ws, &s->sim_val_ws, &s->r1_ws, &s->var_ws, &s->var_keys_ws, &s->adj_ws, &s->lists_ws,
                     &s->union_ws, &s->side_eval[0], &s->side_eval[1], &s->side_eval[2], &s->side_sort[0],
                     &s->side_sort[1], &s->side_sort[2], &s->side_union[0], &s->side_union[1], &s->side_union[2]})
    w->release(s->stream);
  for (cudaEvent_t e : {s->fork_ev, s->join_ev[0], s->join_ev[1], s->join_ev[2], s->mid_ev[0], s->mid_ev[1],
                        s->eval_ev[0], s->eval_ev[1]})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->chunk_ev)
    if (e) cudaEventDestroy(e);
  if (s->stage_ev) cudaEventDestroy(s->stage_ev);
  delete s;
}

void keep_pool_memory(int device) {
  // Serving threads may load their first systems on one device at the same
  // time: one flag per device, set once under call_once.
  static std::once_flag done[64];
  if (device < 0 || device >= 64) return;
  std::call_once(done[device], [device] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

// Up to six device-to-device copies (sizes in bytes, multiples of 4) in one launch.
struct CopySeg {
  void *dst;
  const void *src;
  int64_t bytes;
};
struct CopySegs {
  CopySeg seg[6];
  int n;
};

__global__ void copy_segments_kernel(CopySegs cs) {
  pdl_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < cs.n; ++k) {
    const uint32_t *src = static_cast<const uint32_t *>(cs.seg[k].src);
    uint32_t *dst = static_cast<uint32_t *>(cs.seg[k].dst);
    const int64_t nw = cs.seg[k].bytes / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += stride) dst[i] = src[i];
  }
}

void copy_segments(const CopySegs &cs, cudaStream_t st) {
  int64_t words = 0;
  for (int k = 0; k < cs.n; ++k) words = std::max<int64_t>(words, cs.seg[k].bytes / 4);
  if (words == 0) return;
  pdl_launch(copy_segments_kernel, (unsigned)std::min<int64_t>(ceil_div(words, 256), B300_SMS * 8), 256, 0, st, cs);
  MM_LAUNCH_CHECK();
}

template <class T>
void upload(T *dst, const T *src, int64_t n, int32_t kind, cudaStream_t st) {
  if (n <= 0) return;
  MM_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)n,
                              kind == MM_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
}

void allocate_load_buffers(mm_system *s) {
  DevArena &a = s->arena;
  const int64_t c = s->c, M = s->M, A = s->A;
  s->method_class = a.get<int32_t>(M);
  s->attr_class = a.get<int32_t>(A);
  s->acc_rowptr = a.get<int64_t>(M + 1);
  s->acc_idx = a.get<int32_t>(s->n_acc);
  s->call_rowptr = a.get<int64_t>(M + 1);
  s->call_idx = a.get<int32_t>(s->n_call);
  s->cls_n = a.get<int32_t>(2 * c);  // cls_a follows cls_n: one clear for both
  s->cls_a = s->cls_n ? s->cls_n + c : nullptr;
  s->cm_rowptr = a.get<int64_t>(c + 1);
  s->cm_list = a.get<int32_t>(M);
  s->method_local = a.get<int32_t>(M);
  s->ca_rowptr = a.get<int64_t>(c + 1);
  s->attr_local = a.get<int32_t>(A);
  s->fan_in = a.get<int32_t>(M);
  s->d_u64 = a.get<unsigned long long>(32);
  s->d_err = s->d_u64 ? reinterpret_cast<uint32_t *>(s->d_u64 + 6) : nullptr;  // cleared with the load summary
  s->d_fault = s->d_u64 ? reinterpret_cast<uint32_t *>(s->d_u64 + 9) : nullptr;  // likewise
}

void allocate_compute_buffers(mm_system *s) {
  DevArena &a = s->arena;
  const int64_t c = s->c, M = s->M, nu = s->n_call + s->n_acc;
  s->own_ptr = a.get<int64_t>((int64_t)s->A + 1);
  s->own_list = a.get<int32_t>(std::max<int64_t>(s->n_acc, 1));
  s->cls_P = a.get<int64_t>(c);
  s->cls_Q = a.get<int64_t>(c);
  s->cls_S = a.get<int64_t>(c);
  s->cls_cbo = a.get<int32_t>(c);
  s->own = a.get<int32_t>(M);
  s->q = a.get<int32_t>(M);
  s->mg_rowptr = a.get<int64_t>(c + 1);
  s->mg_dst = a.get<int32_t>(nu);
  s->mg_cnt = a.get<int32_t>(nu);
  s->mg_count = a.get<int64_t>(2);
  s->adj_words = ((c + 127) / 128) * 4;  // rows padded to 16 bytes for vector loads
  if (s->packed_coupling) {  // built on demand from the multigraph rows
    s->out_adj = nullptr;
    s->in_adj = nullptr;
  } else {
    s->out_adj = a.get<uint32_t>(s->adj_words * c);
    s->in_adj = a.get<uint32_t>(s->adj_words * c);
  }
  s->sum_words = (s->adj_words + 31) / 32;
  s->csum = a.get<uint2>(s->sum_words * (2 * c + 1));
  s->cpk = a.get<uint32_t>(2 * nu);
  s->wrank = s->packed_coupling ? a.get<int32_t>(nu) : nullptr;
  s->dest_rec = a.get<int4>(2 * c);
  s->hdr = a.get<MoveHdr>(M);
  s->l_list = a.get<int4>(nu);
  s->l_s = a.get<int32_t>(nu);
  s->l_x = a.get<int32_t>(nu);
  s->r_list = a.get<int4>(s->n_call);
}

std::string describe(uint32_t err) {
  if (err & VE_METHOD_CLASS) return "method_class: class id out of range";
  if (err & VE_ATTR_CLASS) return "attr_class: class id out of range";
  if (err & VE_ACC_ROWPTR) return "acc_rowptr: must start at 0, be non-decreasing and end at n_acc";
  if (err & VE_ACC_IDX_RANGE) return "acc_idx: attribute id out of range";
  if (err & VE_ACC_IDX_ORDER) return "acc_idx: each row must be strictly increasing (sorted, no duplicates)";
  if (err & VE_CALL_ROWPTR) return "call_rowptr: must start at 0, be non-decreasing and end at n_call";
  if (err & VE_CALL_IDX_RANGE) return "call_idx: method id out of range";
  if (err & VE_CALL_IDX_ORDER) return "call_idx: each row must be strictly increasing (sorted, no duplicates)";
  if (err & VE_SELF_CALL) return "call_idx: a method calls itself";
  return "invalid system";
}

__global__ void export_class_kernel(const int32_t *cls_n, const int32_t *cls_a, const int64_t *P, const int64_t *Q,
                                    const int64_t *S, const int32_t *cbo, int32_t c, mm_class_metrics *out) {
  pdl_wait();
  int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= c) return;
  mm_class_metrics r;
  r.n_methods = cls_n[C];
  r.n_attrs = cls_a[C];
  r.P = P[C];
  r.Q = Q[C];
  r.S = S[C];
  r.lcom_ck = r.P > r.Q ? r.P - r.Q : 0;
  int64_t na = (int64_t)r.n_methods * r.n_attrs;
  r.hs_num = na == 0 ? 0 : na - r.S;
  r.hs_den = na == 0 ? 1 : na;
  r.cbo = cbo[C];
  r.reserved = 0;
  out[C] = r;
}

__global__ void export_method_kernel(const int32_t *fan_in, const int64_t *call_rowptr, const int32_t *own,
                                     const int32_t *q, int32_t M, mm_method_metrics *out) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  mm_method_metrics r;
  r.fan_in = fan_in[x];
  r.fan_out = (int32_t)(call_rowptr[x + 1] - call_rowptr[x]);
  r.own = own[x];
  r.q = q[x];
  out[x] = r;
}

}  // namespace

void export_metrics(mm_system *s, mm_class_metrics *out_c, mm_method_metrics *out_m, int32_t kind) {
  cudaStream_t st = s->stream;
  if (out_c && s->c > 0) {
    mm_class_metrics *d = kind == MM_PTR_DEVICE
                              ? out_c
                              : static_cast<mm_class_metrics *>(s->stage_ws.need(sizeof(mm_class_metrics) * s->c, st));
    pdl_launch(export_class_kernel, (unsigned)ceil_div(s->c, 256), 256, 0, st, s->cls_n, s->cls_a, s->cls_P, s->cls_Q,
                                                                      s->cls_S, s->cls_cbo, s->c, d);
    MM_LAUNCH_CHECK();
    if (kind == MM_PTR_HOST)
      MM_CUDA_TRY(cudaMemcpyAsync(out_c, d, sizeof(mm_class_metrics) * s->c, cudaMemcpyDeviceToHost, st));
  }
  if (out_m && s->M > 0) {
    mm_method_metrics *d =
        kind == MM_PTR_DEVICE ? out_m
                              : static_cast<mm_method_metrics *>(s->stage_ws.need(sizeof(mm_method_metrics) * s->M, st));
    pdl_launch(export_method_kernel, (unsigned)ceil_div(s->M, 256), 256, 0, st, s->fan_in, s->call_rowptr, s->own, s->q,
                                                                       s->M, d);
    MM_LAUNCH_CHECK();
    if (kind == MM_PTR_HOST)
      MM_CUDA_TRY(cudaMemcpyAsync(out_m, d, sizeof(mm_method_metrics) * s->M, cudaMemcpyDeviceToHost, st));
  }
  // one synchronisation for both host copies (stream order keeps the shared staging buffer safe)
  if (kind == MM_PTR_HOST && ((out_c && s->c > 0) || (out_m && s->M > 0))) MM_CUDA_TRY(cudaStreamSynchronize(st));
}

extern "C" {

mm_status mm_load_system(const mm_system_desc *desc, void *cuda_stream, mm_system **out) {
  if (out) *out = nullptr;
  mm_system *s = nullptr;
  mm_status st = guarded([&] {
    if (!desc || !out) throw MmError{MM_EINVAL, "load_system: desc and out must be non-NULL"};
    if (desc->n_classes < 1) throw MmError{MM_EINVAL, "load_system: n_classes must be >= 1"};
    if (desc->n_methods < 0 || desc->n_attrs < 0 || desc->n_acc < 0 || desc->n_call < 0)
      throw MmError{MM_EINVAL, "load_system: negative size"};
    if (desc->ptr_kind != MM_PTR_HOST && desc->ptr_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "load_system: bad ptr_kind"};
    if (desc->n_methods == 0 && (desc->n_acc != 0 || desc->n_call != 0))
      throw MmError{MM_EINVAL, "load_system: accesses or calls without methods"};
    if (desc->n_call + desc->n_acc >= (int64_t)0x7fffffff)
      throw MmError{MM_EINVAL, "load_system: more than 2^31-1 calls plus accesses"};
    if (desc->n_methods > 0 && (!desc->method_class || !desc->acc_rowptr || !desc->call_rowptr))
      throw MmError{MM_EINVAL, "load_system: NULL method array"};
    if (desc->n_attrs > 0 && !desc->attr_class) throw MmError{MM_EINVAL, "load_system: NULL attr_class"};
    if ((desc->n_acc > 0 && !desc->acc_idx) || (desc->n_call > 0 && !desc->call_idx))
      throw MmError{MM_EINVAL, "load_system: NULL index array"};
    s = new mm_system();
    MM_CUDA_TRY(cudaGetDevice(&s->device));
    keep_pool_memory(s->device);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->arena.stream = s->stream;
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->join_ev[0], cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->join_ev[1], cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->join_ev[2], cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->mid_ev[0], cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreateWithFlags(&s->mid_ev[1], cudaEventDisableTiming));
    MM_CUDA_TRY(cudaEventCreate(&s->eval_ev[0]));
    MM_CUDA_TRY(cudaEventCreate(&s->eval_ev[1]));
    s->c = desc->n_classes;
    s->M = desc->n_methods;
    s->A = desc->n_attrs;
    s->n_acc = desc->n_acc;
    s->n_call = desc->n_call;
    s->cbo_attrs = desc->cbo_attrs ? 1 : 0;
    if (desc->flags & ~(int32_t)(MM_LOAD_PACKED_COUPLING | MM_LOAD_BITSET_COUPLING))
      throw MmError{MM_EINVAL, "load_system: unknown flags"};
    {
      const double bitset_bytes = 8.0 * (double)((s->c + 127) / 128 * 4) * (double)s->c;
      s->packed_coupling = (desc->flags & MM_LOAD_PACKED_COUPLING) ||
                           (!(desc->flags & MM_LOAD_BITSET_COUPLING) && bitset_bytes > MM_PACKED_COUPLING_BYTES);
    }
    const int64_t M = s->M, A = s->A;
    // size every load-time buffer, reserve one slab, then carve them out of it
    s->arena.sizing = true;
    allocate_load_buffers(s);
    allocate_compute_buffers(s);
    s->arena.sizing = false;
    s->arena.reserve(s->arena.sized);
    allocate_load_buffers(s);
    WaitScope wait(s->d_fault, &s->test_stall_scans);
    cudaStream_t stv = s->stream;
    if (desc->ptr_kind == MM_PTR_DEVICE) {  // one copy kernel for the six device arrays
      CopySegs cs{};
      auto add = [&](void *dst, const void *src, int64_t bytes) {
        if (bytes > 0 && src) cs.seg[cs.n++] = {dst, src, bytes};
      };
      add(s->method_class, desc->method_class, 4 * M);
      add(s->attr_class, desc->attr_class, 4 * A);
      add(s->acc_rowptr, desc->acc_rowptr, 8 * (M + 1));
      add(s->acc_idx, desc->acc_idx, 4 * s->n_acc);
      add(s->call_rowptr, desc->call_rowptr, 8 * (M + 1));
      add(s->call_idx, desc->call_idx, 4 * s->n_call);
      copy_segments(cs, stv);
    } else {
      upload(s->method_class, desc->method_class, M, desc->ptr_kind, stv);
      upload(s->attr_class, desc->attr_class, A, desc->ptr_kind, stv);
      if (M >= 0 && desc->acc_rowptr) upload(s->acc_rowptr, desc->acc_rowptr, M + 1, desc->ptr_kind, stv);
      upload(s->acc_idx, desc->acc_idx, s->n_acc, desc->ptr_kind, stv);
      if (desc->call_rowptr) upload(s->call_rowptr, desc->call_rowptr, M + 1, desc->ptr_kind, stv);
      upload(s->call_idx, desc->call_idx, s->n_call, desc->ptr_kind, stv);
    }
    if (M == 0) {
      MM_CUDA_TRY(cudaMemsetAsync(s->acc_rowptr, 0, sizeof(int64_t), stv));
      MM_CUDA_TRY(cudaMemsetAsync(s->call_rowptr, 0, sizeof(int64_t), stv));
    }
    load_validate_and_summarise(s);
    allocate_compute_buffers(s);  // host allocation calls overlap the checks on the device
    load_finish(s);
    if (s->summary.err) throw MmError{MM_EINVAL, "load_system: " + describe(s->summary.err)};
    *out = s;
  });
  if (st != MM_OK && s) {
    release_system(s);
    if (out) *out = nullptr;
  }
  return st;
}

mm_status mm_set_stream(mm_system *s, void *cuda_stream) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "set_stream: NULL system"};
    SystemScope scope(s);
    // order the new stream after everything queued on the old one
    cudaStream_t ns = static_cast<cudaStream_t>(cuda_stream);
    if (ns != s->stream) {
      cudaEvent_t ev;
      MM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      MM_CUDA_TRY(cudaEventRecord(ev, s->stream));
      MM_CUDA_TRY(cudaStreamWaitEvent(ns, ev, 0));
      MM_CUDA_TRY(cudaEventDestroy(ev));
    }
    s->stream = ns;
    s->arena.stream = ns;
  });
}

mm_status mm_compute_metrics(mm_system *s, mm_class_metrics *out_c, mm_method_metrics *out_m, int32_t out_kind) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "compute_metrics: NULL system"};
    if ((out_c || out_m) && out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "compute_metrics: bad out_kind"};
    SystemScope scope(s);
    s->kept_valid = false;
    build_structures(s);
    build_metrics(s);
    build_move_precompute(s);
    s->metrics_ready = true;
    export_metrics(s, out_c, out_m, out_kind);
    if ((out_c || out_m) && out_kind == MM_PTR_HOST) check_wait_fault(s->d_fault, s->stream, "compute_metrics");
  });
}

mm_status mm_export_metrics(mm_system *s, mm_class_metrics *out_c, mm_method_metrics *out_m, int32_t out_kind) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "export_metrics: NULL system"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "export_metrics: no metrics computed yet"};
    if ((out_c || out_m) && out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "export_metrics: bad out_kind"};
    SystemScope scope(s);
    export_metrics(s, out_c, out_m, out_kind);
    if ((out_c || out_m) && out_kind == MM_PTR_HOST) check_wait_fault(s->d_fault, s->stream, "export_metrics");
  });
}

mm_status mm_evaluate_moves(mm_system *s, const mm_criteria *crit, const mm_candidates *cands,
                            mm_move_eval *records, uint64_t *digest, int32_t out_kind) {
  return guarded([&] {
    if (!s || !crit) throw MmError{MM_EINVAL, "evaluate_moves: NULL system or criteria"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "evaluate_moves: call mm_compute_metrics first"};
    SystemScope scope(s);
    evaluate_moves(s, *crit, cands, records, digest, out_kind);
    if ((records || digest) && out_kind == MM_PTR_HOST) check_wait_fault(s->d_fault, s->stream, "evaluate_moves");
  });
}

mm_status mm_suggest_moves(mm_system *s, const mm_criteria *crit, const mm_candidates *cands, int32_t k,
                           mm_move *out_topk, int32_t out_kind, int64_t *n_kept, int64_t *n_methods_with_kept) {
  return guarded([&] {
    if (!s || !crit) throw MmError{MM_EINVAL, "suggest_moves: NULL system or criteria"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "suggest_moves: call mm_compute_metrics first"};
    SystemScope scope(s);
    suggest_moves(s, *crit, cands, k, out_topk, out_kind, n_kept, n_methods_with_kept);
  });
}

mm_status mm_last_eval_ms(mm_system *s, float *ms) {
  return guarded([&] {
    if (!s || !ms) throw MmError{MM_EINVAL, "last_eval_ms: NULL argument"};
    if (!s->eval_timed) throw MmError{MM_EINVAL, "last_eval_ms: no evaluation kernel has run on this handle"};
    SystemScope scope(s);
    MM_CUDA_TRY(cudaEventSynchronize(s->eval_ev[1]));
    MM_CUDA_TRY(cudaEventElapsedTime(ms, s->eval_ev[0], s->eval_ev[1]));
  });
}

static void fill_similarity_info(const mm_system *s, mm_similarity_info *info, int64_t n_high, int64_t n_cand) {
  if (!info) return;
  info->n_values = s->sim_n;
  info->n_cooccurrences = s->sim_cooc;
  info->n_high = n_high;
  info->n_candidates = n_cand;
  info->average = s->sim_avg;
  info->max_union = s->sim_umax;
  info->reserved = 0;
}

mm_status mm_similarity(mm_system *s, int32_t *x, int32_t *y, int32_t *inter, int32_t *uni, int64_t cap,
                        int32_t out_kind, mm_similarity_info *info) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "similarity: NULL system"};
    if (cap < 0) throw MmError{MM_EINVAL, "similarity: cap < 0"};
    if ((x || y || inter || uni) && out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "similarity: bad out_kind"};
    SystemScope scope(s);
    compute_similarity(s);
    const int64_t n = std::min<int64_t>(cap, s->sim_n);
    const cudaMemcpyKind kind = out_kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int32_t *src[4] = {s->sim_x, s->sim_y, s->sim_i, s->sim_u};
    int32_t *dst[4] = {x, y, inter, uni};
    for (int k = 0; k < 4; ++k)
      if (dst[k] && n > 0) MM_CUDA_TRY(cudaMemcpyAsync(dst[k], src[k], sizeof(int32_t) * (size_t)n, kind, s->stream));
    check_wait_fault(s->d_fault, s->stream, "similarity");
    fill_similarity_info(s, info, 0, 0);
  });
}

mm_status mm_suggest_r1(mm_system *s, const mm_criteria *crit, int32_t k, mm_move *out_topk, int32_t out_kind,
                        int64_t *n_kept, int64_t *n_methods_with_kept, mm_similarity_info *info) {
  return guarded([&] {
    if (!s || !crit) throw MmError{MM_EINVAL, "suggest_r1: NULL system or criteria"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "suggest_r1: call mm_compute_metrics first"};
    SystemScope scope(s);
    compute_similarity(s);
    int64_t n_high = 0, n_cand = 0;
    build_r1_candidates(s, &n_high, &n_cand);
    mm_candidates cands{};
    cands.rowptr = s->r1_rowptr;
    cands.dst = s->r1_dst;
    cands.n_cand = n_cand;
    cands.ptr_kind = MM_PTR_DEVICE;
    suggest_moves(s, *crit, &cands, k, out_topk, out_kind, n_kept, n_methods_with_kept);
    fill_similarity_info(s, info, n_high, n_cand);
  });
}

mm_status mm_system_info_get(mm_system *s, mm_system_info *info) {
  return guarded([&] {
    if (!s || !info) throw MmError{MM_EINVAL, "system_info: NULL argument"};
    SystemScope scope(s);
    info->n_classes = s->c;
    info->n_methods = s->M;
    info->n_attrs = s->A;
    info->cbo_attrs = s->cbo_attrs;
    info->n_acc = s->n_acc;
    info->n_call = s->n_call;
    info->n_class_edges = -1;
    if (s->metrics_ready) {
      int64_t v = 0;
      MM_CUDA_TRY(cudaMemcpyAsync(&v, s->mg_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream));
      MM_CUDA_TRY(cudaStreamSynchronize(s->stream));
      info->n_class_edges = v;
    }
    info->device_bytes =
        s->arena.bytes + (int64_t)(s->sort_ws.cap + s->eval_ws.cap + s->stage_ws.cap + s->kept_ws.cap +
                                   s->keyed_ws.cap + s->edit_ws.cap + s->union_ws.cap + s->side_eval[0].cap +
                                   s->side_eval[1].cap + s->side_eval[2].cap + s->side_sort[0].cap +
                                   s->side_sort[1].cap + s->side_sort[2].cap + s->side_union[0].cap +
                                   s->side_union[1].cap + s->side_union[2].cap);
  });
}

void mm_free_system(mm_system *s) {
  if (!s) return;
  int cur = -1;
  const int dev = s->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  release_system(s);
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
}

mm_status mm_apply_edit(mm_system *s, const mm_edit *e) {
  return guarded([&] {
    if (!s || !e) throw MmError{MM_EINVAL, "apply_edit: NULL argument"};
    SystemScope scope(s);
    apply_edit(s, *e);  // queued: a bounded wait that ran out is reported by the next synchronising call
  });
}

mm_status mm_suggest_r3(mm_system *s, int32_t k, mm_r3_move *out_topk, int64_t *n_kept, int64_t *n_candidates,
                        int32_t *n_high_classes) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "suggest_r3: NULL system"};
    SystemScope scope(s);
    suggest_r3(s, k, out_topk, n_kept, n_candidates, n_high_classes);
    check_wait_fault(s->d_fault, s->stream, "suggest_r3");
  });
}

mm_status mm_apply_sequence(mm_system *s, const mm_criteria *crit, int32_t rounds, int32_t per_round,
                            mm_applied_move *out, int64_t cap, int64_t *n_applied) {
  return guarded([&] {
    if (!s || !crit) throw MmError{MM_EINVAL, "apply_sequence: NULL system or criteria"};
    SystemScope scope(s);
    apply_sequence(s, *crit, rounds, per_round, out, cap, n_applied);
    check_wait_fault(s->d_fault, s->stream, "apply_sequence");
  });
}

mm_status mm_metric_variants(mm_system *s, mm_class_variants *out, int32_t *out_q_all, int32_t out_kind) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "metric_variants: NULL system"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "metric_variants: call mm_compute_metrics first"};
    if ((out || out_q_all) && out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "metric_variants: bad out_kind"};
    SystemScope scope(s);
    mm_class_variants *var = nullptr;
    int32_t *q_all = nullptr;
    compute_variants(s, &var, &q_all);
    const cudaMemcpyKind dir = out_kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (out && s->c > 0)
      MM_CUDA_TRY(cudaMemcpyAsync(out, var, sizeof(mm_class_variants) * (size_t)s->c, dir, s->stream));
    if (out_q_all && s->M > 0)
      MM_CUDA_TRY(cudaMemcpyAsync(out_q_all, q_all, sizeof(int32_t) * (size_t)s->M, dir, s->stream));
    if ((out || out_q_all) && out_kind == MM_PTR_HOST) check_wait_fault(s->d_fault, s->stream, "metric_variants");
  });
}

mm_status mm_rank_classes(mm_system *s, int32_t metric, int32_t k, int32_t *out_ids, int64_t *out_values,
                          int32_t out_kind) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "rank_classes: NULL system"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "rank_classes: call mm_compute_metrics first"};
    if (metric < MM_RANK_LCOM_CK || metric > MM_RANK_CBO_BI) throw MmError{MM_EINVAL, "rank_classes: unknown metric"};
    if (k < 0 || (k > 0 && !out_ids)) throw MmError{MM_EINVAL, "rank_classes: bad k or out_ids"};
    if (out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE) throw MmError{MM_EINVAL, "rank_classes: bad out_kind"};
    SystemScope scope(s);
    rank_classes(s, metric, k, out_ids, out_values, out_kind);
    if (out_kind == MM_PTR_HOST) check_wait_fault(s->d_fault, s->stream, "rank_classes");
  });
}

mm_status mm_stage_candidates(mm_system *s, const mm_candidates *cands) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "stage_candidates: NULL system"};
    SystemScope scope(s);
    stage_candidates(s, cands);
  });
}

mm_status mm_selftest_stall_scans(mm_system *s, int32_t n) {
  return guarded([&] {
    if (!s || n < 0) throw MmError{MM_EINVAL, "selftest_stall_scans: NULL system or n < 0"};
    s->test_stall_scans = n;
  });
}

mm_status mm_export_system(mm_system *s, int32_t *method_class, int32_t *attr_class, int64_t *acc_rowptr,
                           int32_t *acc_idx, int64_t *call_rowptr, int32_t *call_idx) {
  return guarded([&] {
    if (!s) throw MmError{MM_EINVAL, "export_system: NULL system"};
    SystemScope scope(s);
    export_system(s, method_class, attr_class, acc_rowptr, acc_idx, call_rowptr, call_idx);
  });
}

const char *mm_last_error(void) { return g_last_error.c_str(); }

const char *mm_status_string(mm_status st) {
  switch (st) {
    case MM_OK: return "ok";
    case MM_EINVAL: return "invalid argument";
    case MM_ENOMEM: return "out of memory";
    case MM_ECUDA: return "CUDA error";
    case MM_ENOTFOUND: return "not found";
    case MM_EEXIST: return "already exists";
    case MM_ETIMEOUT: return "device wait timed out";
    case MM_EBUDGET: return "memory budget exceeded";
  }
  return "unknown status";
}

int32_t mm_abi_version(void) { return MMREF_ABI_VERSION; }

int64_t mm_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

mm_status mm_selftest_bounded_wait(void) {
  return guarded([&] {
    const uint32_t r = stalled_scan_probe();
    if (r == 2) throw MmError{MM_ECUDA, "selftest: the stalled scan's fallback did not give the exact prefix"};
    if (r) throw MmError{MM_ETIMEOUT, "selftest: the stalled scan's wait gave up as designed; its output is exact"};
  });
}

}  // extern "C"
