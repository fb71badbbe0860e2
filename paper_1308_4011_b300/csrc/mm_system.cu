// Loading a system: upload of the CSR arrays (the paper's cls / dpnd arrays,
// Sec. IV.C), validation on the device, and the class structures every metric
// needs: class -> methods, class -> attributes, and the callers of each method
// (the transpose used for fan-in, Sec. II.A).
#include <cuda_runtime.h>

#include <algorithm>

#include <cstring>

#include "mm_internal.cuh"

// ---------------------------------------------------------------- memory helpers

void DevArena::reserve(size_t n) {
  if (n == 0 || slab) return;
  n = (n + 255) & ~size_t(255);
  void *p = nullptr;
  MM_CUDA_TRY(cudaMallocAsync(&p, n, stream));
  slab = static_cast<char *>(p);
  slab_cap = n;
  slab_used = 0;
  bytes += (int64_t)n;
}

void *DevArena::alloc(size_t n) {
  void *p = nullptr;
  n = (n + 255) & ~size_t(255);
  if (sizing) {
    sized += n;
    return nullptr;
  }
  if (slab && slab_used + n <= slab_cap) {
    p = slab + slab_used;
    slab_used += n;
    return p;
  }
  MM_CUDA_TRY(cudaMallocAsync(&p, n, stream));
  ptrs.push_back(p);
  bytes += (int64_t)n;
  return p;
}

void DevArena::forget(void *p) {
  if (slab && static_cast<char *>(p) >= slab && static_cast<char *>(p) < slab + slab_cap) return;
  for (size_t i = 0; i < ptrs.size(); ++i)
    if (ptrs[i] == p) {
      cudaFreeAsync(p, stream);
      ptrs.erase(ptrs.begin() + (long)i);
      return;
    }
}

void DevArena::release() {
  for (void *p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  if (slab) cudaFreeAsync(slab, stream);
  slab = nullptr;
  slab_cap = slab_used = 0;
  bytes = 0;
}

void *Scratch::need(size_t n, cudaStream_t st) {
  if (n <= cap && ptr) return ptr;
  size_t want = std::max(n, cap + cap / 2);
  if (ptr) MM_CUDA_TRY(cudaFreeAsync(ptr, st));
  ptr = nullptr;
  cap = 0;
  want = (want + 255) & ~size_t(255);
  MM_CUDA_TRY(cudaMallocAsync(&ptr, want, st));
  cap = want;
  return ptr;
}

void Scratch::release(cudaStream_t st) {
  if (ptr) cudaFreeAsync(ptr, st);
  ptr = nullptr;
  cap = 0;
}

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n, int tpb = TPB) {
  int64_t g = ceil_div(n, tpb);
  if (g < 1) g = 1;
  if (g > 0x7fffffffLL) g = 0x7fffffffLL;
  return (unsigned)g;
}

// ---------------------------------------------------------------- validation

__global__ void validate_methods(const int32_t *method_class, const int64_t *acc_rowptr, const int32_t *acc_idx,
                                 const int64_t *call_rowptr, const int32_t *call_idx, int32_t c, int32_t M,
                                 int32_t A, int64_t n_acc, int64_t n_call, uint32_t *err) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  uint32_t e = 0;
  int32_t C = method_class[x];
  if (C < 0 || C >= c) e |= VE_METHOD_CLASS;
  if (x + 1 < M && method_class[x + 1] < C) e |= VI_METHODS_UNSORTED;
  if (x == 0) {
    if (acc_rowptr[0] != 0 || acc_rowptr[M] != n_acc) e |= VE_ACC_ROWPTR;
    if (call_rowptr[0] != 0 || call_rowptr[M] != n_call) e |= VE_CALL_ROWPTR;
  }
  int64_t a0 = acc_rowptr[x], a1 = acc_rowptr[x + 1];
  if (a0 < 0 || a1 < a0 || a1 > n_acc) {
    e |= VE_ACC_ROWPTR;
  } else {
    int32_t prev = -1;
    for (int64_t k = a0; k < a1; ++k) {
      int32_t v = acc_idx[k];
      if (v < 0 || v >= A) e |= VE_ACC_IDX_RANGE;
      if (v <= prev) e |= VE_ACC_IDX_ORDER;
      prev = v;
    }
  }
  int64_t c0 = call_rowptr[x], c1 = call_rowptr[x + 1];
  if (c0 < 0 || c1 < c0 || c1 > n_call) {
    e |= VE_CALL_ROWPTR;
  } else {
    int32_t prev = -1;
    for (int64_t k = c0; k < c1; ++k) {
      int32_t v = call_idx[k];
      if (v < 0 || v >= M) e |= VE_CALL_IDX_RANGE;
      if (v <= prev) e |= VE_CALL_IDX_ORDER;
      if (v == x) e |= VE_SELF_CALL;
      prev = v;
    }
  }
  if (e) atomicOr(err, e);
}

__global__ void validate_attrs(const int32_t *attr_class, int32_t c, int32_t A, uint32_t *err) {
  pdl_wait();
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  int32_t C = attr_class[a];
  uint32_t e = 0;
  if (C < 0 || C >= c) e |= VE_ATTR_CLASS;
  if (a + 1 < A && attr_class[a + 1] < C) e |= VI_ATTRS_UNSORTED;
  if (e) atomicOr(err, e);
}

__global__ void class_histograms(const int32_t *method_class, const int32_t *attr_class, int32_t c, int32_t M,
                                 int32_t A, int32_t *cls_n, int32_t *cls_a) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    int32_t C = method_class[i];
    if (C >= 0 && C < c) atomicAdd(&cls_n[C], 1);
  }
  if (i < A) {
    int32_t C = attr_class[i];
    if (C >= 0 && C < c) atomicAdd(&cls_a[C], 1);
  }
}

__global__ void summarise_classes(const int32_t *cls_n, int32_t c, LoadSummary *sum) {
  pdl_wait();
  int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t nmax = C < c ? cls_n[C] : 0;
  for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_down_sync(0xffffffffu, nmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&sum->max_class_methods, nmax);
}

// ---------------------------------------------------------------- structures

__global__ void iota_u32(uint32_t *v, int64_t n) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

__global__ void copy_i32_to_u32(const int32_t *in, uint32_t *out, int64_t n) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)in[i];
}

// rank of each item inside its class after the stable sort by class
__global__ void local_ranks(const uint32_t *sorted_cls, const uint32_t *sorted_item, const int64_t *rowptr,
                            int64_t n, int32_t *local, int32_t *list) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t C = sorted_cls[i], it = sorted_item[i];
  local[it] = (int32_t)(i - rowptr[C]);
  if (list) list[i] = (int32_t)it;
}

// ids already grouped by class in ascending order: the rank is id - first id of the class
__global__ void local_ranks_sorted(const int32_t *cls, const int64_t *rowptr, int64_t n, int32_t *local,
                                   int32_t *list) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  local[i] = (int32_t)(i - rowptr[cls[i]]);
  if (list) list[i] = (int32_t)i;
}

__global__ void fan_in_hist(const int32_t *call_idx, int64_t n_call, int32_t *fan_in) {
  pdl_wait();
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_call) atomicAdd(&fan_in[call_idx[e]], 1);
}

}  // namespace

// Queue the load checks (validation, class histograms, load summary);
// load_finish reads their results back.
void load_validate_and_summarise(mm_system *s) {
  cudaStream_t st = s->stream;
  LoadSummary *dsum = reinterpret_cast<LoadSummary *>(s->d_u64 + 4);
  // summary, error word, fault word
  MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 4, 0, 6 * sizeof(unsigned long long), st));
  MM_CUDA_TRY(cudaMemsetAsync(s->cls_n, 0, sizeof(int32_t) * 2 * (size_t)s->c, st));  // cls_n, cls_a
  if (s->M > 0)
    pdl_launch(validate_methods, grid_for(s->M), TPB, 0, st, s->method_class, s->acc_rowptr, s->acc_idx, s->call_rowptr,
                                                     s->call_idx, s->c, s->M, s->A, s->n_acc, s->n_call, s->d_err);
  MM_LAUNCH_CHECK();
  if (s->A > 0) pdl_launch(validate_attrs, grid_for(s->A), TPB, 0, st, s->attr_class, s->c, s->A, s->d_err);
  MM_LAUNCH_CHECK();
  int64_t nmax = std::max<int64_t>(s->M, s->A);
  pdl_launch(class_histograms, grid_for(nmax), TPB, 0, st, s->method_class, s->attr_class, s->c, s->M, s->A, s->cls_n,
                                                   s->cls_a);
  MM_LAUNCH_CHECK();
  pdl_launch(summarise_classes, grid_for(s->c), TPB, 0, st, s->cls_n, s->c, dsum);
  MM_LAUNCH_CHECK();
}

// Read back and wait for the load checks queued by load_validate_and_summarise
// (the caller may allocate in between: a read-back into pageable memory blocks
// the host, so it comes last).
namespace {
struct HostStaging {
  void *p = nullptr;
  size_t cap = 0;
  ~HostStaging() {
    if (p) cudaFreeHost(p);  // at process exit the runtime may be gone: errors ignored
  }
};
thread_local HostStaging tl_host;
}  // namespace

void *host_staging(size_t bytes) {
  if (tl_host.p && bytes <= tl_host.cap) return tl_host.p;
  const size_t want = std::max<size_t>(bytes, std::max<size_t>(2 * tl_host.cap, 4096));
  if (tl_host.p) cudaFreeHost(tl_host.p);  // between calls: no copy targets it any more
  tl_host.p = nullptr;
  tl_host.cap = 0;
  MM_CUDA_TRY(cudaMallocHost(&tl_host.p, want));
  tl_host.cap = want;
  return tl_host.p;
}

void load_finish(mm_system *s) {
  cudaStream_t st = s->stream;
  // d_u64[4] = load summary, d_u64[6] = error word: one copy, plus the fault flag
  unsigned char *h = static_cast<unsigned char *>(host_staging(48));
  MM_CUDA_TRY(cudaMemcpyAsync(h, s->d_u64 + 4, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  uint32_t *hfault = reinterpret_cast<uint32_t *>(h + 32);
  *hfault = 0;
  read_wait_fault(hfault, s->d_fault, st);
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  std::memcpy(&s->summary, h, sizeof(LoadSummary));
  std::memcpy(&s->load_err, h + 16, sizeof(uint32_t));
  raise_wait_fault(*hfault, s->d_fault, st, "load");
  const uint32_t err = s->load_err;
  s->summary.err = err & VE_ERRORS;
  s->methods_by_class = !(err & VI_METHODS_UNSORTED);
  s->attrs_by_class = !(err & VI_ATTRS_UNSORTED);
}

void build_structures(mm_system *s) {
  cudaStream_t st = s->stream;
  const int64_t c = s->c, M = s->M, A = s->A, E = s->n_call;
  int64_t n = std::max<int64_t>(std::max<int64_t>(M, A), E);
  n = std::max<int64_t>(n, 1);
  uint32_t *buf = static_cast<uint32_t *>(s->eval_ws.need(sizeof(uint32_t) * 4 * (size_t)n, st));
  uint32_t *k = buf, *ka = buf + n, *v = buf + 2 * n, *va = buf + 3 * n;
  const int cbits = bits_for((uint64_t)(c > 0 ? c - 1 : 0));

  // class -> methods: stable sort of method ids by owner class
  scan_exclusive_i32to64(s->cls_n, s->cm_rowptr, c, s->sort_ws, st, s->cm_rowptr + c);  // total = M
  if (M > 0 && s->methods_by_class) {
    pdl_launch(local_ranks_sorted, grid_for(M), TPB, 0, st, s->method_class, s->cm_rowptr, M, s->method_local, s->cm_list);
    MM_LAUNCH_CHECK();
  } else if (M > 0) {
    pdl_launch(copy_i32_to_u32, grid_for(M), TPB, 0, st, s->method_class, k, M);
    pdl_launch(iota_u32, grid_for(M), TPB, 0, st, v, M);
    MM_LAUNCH_CHECK();
    radix_sort_u32(k, ka, v, va, M, cbits, s->sort_ws, st);
    pdl_launch(local_ranks, grid_for(M), TPB, 0, st, k, v, s->cm_rowptr, M, s->method_local, s->cm_list);
    MM_LAUNCH_CHECK();
  }
  // class -> attributes
  scan_exclusive_i32to64(s->cls_a, s->ca_rowptr, c, s->sort_ws, st, s->ca_rowptr + c);  // total = A
  if (A > 0 && s->attrs_by_class) {
    pdl_launch(local_ranks_sorted, grid_for(A), TPB, 0, st, s->attr_class, s->ca_rowptr, A, s->attr_local, nullptr);
    MM_LAUNCH_CHECK();
  } else if (A > 0) {
    pdl_launch(copy_i32_to_u32, grid_for(A), TPB, 0, st, s->attr_class, k, A);
    pdl_launch(iota_u32, grid_for(A), TPB, 0, st, v, A);
    MM_LAUNCH_CHECK();
    radix_sort_u32(k, ka, v, va, A, cbits, s->sort_ws, st);
    pdl_launch(local_ranks, grid_for(A), TPB, 0, st, k, v, s->ca_rowptr, A, s->attr_local, nullptr);
    MM_LAUNCH_CHECK();
  }
  // fan-in: number of callers of each method (the callers themselves are
  // grouped by class later, from the call edges, by the move precompute's sort)
  MM_CUDA_TRY(cudaMemsetAsync(s->fan_in, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(M, 1), st));
  if (E > 0) {
    pdl_launch(fan_in_hist, grid_for(E), TPB, 0, st, s->call_idx, E, s->fan_in);
    MM_LAUNCH_CHECK();
  }
}

namespace {

// The class -> methods lists after method m moved from class C to class D,
// from the lists before (ascending ids within each class): every member keeps
// its order; m leaves C's segment and enters D's at its rank by id.
__global__ void move_patch_members(const int32_t *old_list, const int64_t *old_ptr, const int64_t *new_ptr,
                                   const int32_t *method_class, int32_t M, int32_t m, int32_t C, int32_t D,
                                   int32_t *cm_list, int32_t *method_local) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = old_list[i];
    int64_t r;
    int32_t Y;
    if (x == m) {  // D's members with a smaller id come first
      int64_t lo = old_ptr[D], hi = old_ptr[D + 1];
      const int64_t base = lo;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (old_list[mid] < m) lo = mid + 1; else hi = mid;
      }
      r = lo - base;
      Y = D;
    } else {
      Y = method_class[x];
      r = i - old_ptr[Y];
      if (Y == C && x > m) r -= 1;
      if (Y == D && x > m) r += 1;
    }
    cm_list[new_ptr[Y] + r] = x;
    method_local[x] = (int32_t)r;
  }
}

__global__ void add_to(int32_t *p, int32_t v) {
  pdl_wait();
  *p += v;
}

}  // namespace

// Class structures after an edit, without the full rebuild: a move patches
// the class -> methods lists and ranks (cls_n and method_class already
// updated); a call added or removed changes one fan-in; an access changes none.
void patch_structures(mm_system *s, int32_t kind, int32_t m, int32_t target, int32_t C) {
  cudaStream_t st = s->stream;
  if (kind == MM_EDIT_ADD_CALL || kind == MM_EDIT_REMOVE_CALL) {
    pdl_launch(add_to, 1, 1, 0, st, s->fan_in + target, kind == MM_EDIT_ADD_CALL ? 1 : -1);
    MM_LAUNCH_CHECK();
    return;
  }
  if (kind != MM_EDIT_MOVE) return;
  const int64_t c = s->c, M = s->M;
  char *b = static_cast<char *>(s->eval_ws.need(sizeof(int64_t) * ((size_t)c + 1) + sizeof(int32_t) * (size_t)M + 512,
                                                st));
  int64_t *old_ptr = reinterpret_cast<int64_t *>(b);
  int32_t *old_list = reinterpret_cast<int32_t *>(b + ((sizeof(int64_t) * ((size_t)c + 1) + 255) & ~size_t(255)));
  MM_CUDA_TRY(cudaMemcpyAsync(old_ptr, s->cm_rowptr, sizeof(int64_t) * ((size_t)c + 1), cudaMemcpyDeviceToDevice, st));
  MM_CUDA_TRY(cudaMemcpyAsync(old_list, s->cm_list, sizeof(int32_t) * (size_t)M, cudaMemcpyDeviceToDevice, st));
  scan_exclusive_i32to64(s->cls_n, s->cm_rowptr, c, s->sort_ws, st, s->cm_rowptr + c);
  pdl_launch(move_patch_members, grid_for(M), TPB, 0, st, static_cast<const int32_t *>(old_list),
             static_cast<const int64_t *>(old_ptr), static_cast<const int64_t *>(s->cm_rowptr),
             static_cast<const int32_t *>(s->method_class), (int32_t)M, m, C, target, s->cm_list, s->method_local);
  MM_LAUNCH_CHECK();
}
