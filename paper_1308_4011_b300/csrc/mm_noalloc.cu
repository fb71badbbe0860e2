// mm_suggest_moves_noalloc: the suggestion list computed without allocating
// any device memory.  Its working memory (kept moves, per-method marks,
// counters, merge-sort buffer) is one file-scope static device array of fixed
// size, shared by every call in the process on a device.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "mm_internal.cuh"

void eval_kept_into(mm_system *s, const mm_criteria &crit, const mm_candidates *cands, mm_move *kept, int64_t cap,
                    unsigned long long *count, uint8_t *mark);
void sort_moves_chunks(mm_move *v, int64_t n, cudaStream_t st);

namespace {

constexpr size_t NA_COUNTERS = 256;
constexpr size_t NA_MARKS = MM_NOALLOC_MAX_METHODS;
constexpr size_t NA_KEPT = sizeof(mm_move) * (size_t)MM_NOALLOC_MAX_KEPT;
constexpr size_t NA_BYTES = NA_COUNTERS + NA_MARKS + 2 * NA_KEPT;  // about 4.2 MB
constexpr int NA_CHUNK = 2048;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_setup_mu;
void *g_scratch_addr[64] = {nullptr};

// Device address of the static array for the current device (looked up once
// per device, with that device current; host code must not use the symbol
// itself, which is only a host-side stand-in).
unsigned char *scratch_for_device(int dev) {
  if (dev < 0 || dev >= 64) throw MmError{MM_EINVAL, "noalloc: device index out of range"};
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) throw MmError{MM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    g_scratch_addr[dev] = p;
  }
  return static_cast<unsigned char *>(g_scratch_addr[dev]);
}

__device__ __forceinline__ bool before(const mm_move &a, const mm_move &b) {
  if (a.n_improved != b.n_improved) return a.n_improved > b.n_improved;
  if (a.d_lcom_ck_sum != b.d_lcom_ck_sum) return a.d_lcom_ck_sum < b.d_lcom_ck_sum;
  if (a.d_cbo_sum != b.d_cbo_sum) return a.d_cbo_sum < b.d_cbo_sum;
  if (a.m != b.m) return a.m < b.m;
  return a.d < b.d;
}

// Merge adjacent sorted runs of length w from src into dst: each element finds
// its output position by a binary search in the partner run (the order is
// total, so no two moves compare equal).
__global__ void merge_runs(const mm_move *src, mm_move *dst, int32_t n, int32_t w) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t run0 = (i / (2 * w)) * (2 * w);
  const bool left = i < run0 + w;
  const int32_t a0 = run0, a1 = min(run0 + w, n);
  const int32_t b0 = a1, b1 = min(run0 + 2 * w, n);
  const mm_move x = src[i];
  int32_t lo, hi;
  if (left) { lo = b0; hi = b1; } else { lo = a0; hi = a1; }
  while (lo < hi) {  // count partner elements that come before x
    int32_t mid = (lo + hi) >> 1;
    if (before(src[mid], x)) lo = mid + 1; else hi = mid;
  }
  const int32_t partner_before = lo - (left ? b0 : a0);
  const int32_t own = left ? i - a0 : i - b0;
  dst[run0 + own + partner_before] = x;
}

__global__ void count_bytes(const uint8_t *mark, int64_t n, unsigned long long *out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += mark[i];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

extern "C" MMREF_API mm_status mm_suggest_moves_noalloc(mm_system *s, const mm_criteria *crit,
                                                        const mm_candidates *cands, int32_t k, mm_move *out_topk,
                                                        int32_t out_kind, int64_t *n_kept,
                                                        int64_t *n_methods_with_kept) {
  try {
    if (!s || !crit) throw MmError{MM_EINVAL, "suggest_moves_noalloc: NULL system or criteria"};
    if (s->M > MM_NOALLOC_MAX_METHODS)
      throw MmError{MM_EBUDGET, "suggest_moves_noalloc: the system has more than MM_NOALLOC_MAX_METHODS (1,048,576) "
                                "methods"};
    if (!s->metrics_ready) throw MmError{MM_EINVAL, "suggest_moves_noalloc: call mm_compute_metrics first"};
    if (k < 0 || (k > 0 && !out_topk)) throw MmError{MM_EINVAL, "suggest_moves_noalloc: bad k or out_topk"};
    if (out_kind != MM_PTR_HOST && out_kind != MM_PTR_DEVICE)
      throw MmError{MM_EINVAL, "suggest_moves_noalloc: bad out_kind"};
    // the caller's current device is restored on every exit, errors included
    struct DeviceGuard {
      int prev = -1;
      ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
      }
    } guard;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) throw MmError{MM_ECUDA, "cudaGetDevice failed"};
    if (cur != s->device) {
      if (cudaSetDevice(s->device) != cudaSuccess) throw MmError{MM_ECUDA, "cudaSetDevice failed"};
      guard.prev = cur;
    }
    if ((!cands || !cands->rowptr) && !s->adj_built)
      throw MmError{MM_EBUDGET, "suggest_moves_noalloc: the full cross product needs the system's adjacency "
                                "bitsets, which are built on demand for systems with packed coupling; use "
                                "mm_suggest_moves"};
    WaitScope wait(s->d_fault, &s->test_stall_scans);
    unsigned char *base = scratch_for_device(s->device);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base);  // [0] kept, [1] methods
    uint8_t *mark = base + NA_COUNTERS;
    mm_move *kept = reinterpret_cast<mm_move *>(base + NA_COUNTERS + NA_MARKS);
    mm_move *tmp = kept + MM_NOALLOC_MAX_KEPT;
    cudaStream_t st = s->stream;
    // the array keeps the previous call's contents: clear what must start at zero
    MM_CUDA_TRY(cudaMemsetAsync(counters, 0, NA_COUNTERS, st));
    if (s->M > 0) MM_CUDA_TRY(cudaMemsetAsync(mark, 0, (size_t)s->M, st));
    eval_kept_into(s, *crit, cands, kept, MM_NOALLOC_MAX_KEPT, &counters[0], mark);
    if (s->M > 0) {
      count_bytes<<<B300_SMS * 4, 256, 0, st>>>(mark, s->M, &counters[1]);
      MM_LAUNCH_CHECK();
    }
    unsigned long long hc[2] = {0, 0};
    uint32_t hfault = 0;
    MM_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
    read_wait_fault(&hfault, s->d_fault, st);
    MM_CUDA_TRY(cudaStreamSynchronize(st));
    raise_wait_fault(hfault, s->d_fault, st, "suggest_moves_noalloc");
    const int64_t K = (int64_t)hc[0];
    if (K > MM_NOALLOC_MAX_KEPT)
      throw MmError{MM_EBUDGET, "suggest_moves_noalloc: " + std::to_string(K) +
                                    " kept moves exceed MM_NOALLOC_MAX_KEPT (65,536); use mm_suggest_moves"};
    // sort: bitonic chunks of 2,048, then pairwise merges between the two halves of the array
    mm_move *cur_buf = kept, *other = tmp;
    if (K > 1) {
      sort_moves_chunks(kept, K, st);  // runs of NA_CHUNK, one block each
      for (int64_t w = NA_CHUNK; w < K; w *= 2) {
        merge_runs<<<(unsigned)ceil_div(K, 256), 256, 0, st>>>(cur_buf, other, (int32_t)K, (int32_t)w);
        MM_LAUNCH_CHECK();
        std::swap(cur_buf, other);
      }
    }
    const int64_t nout = std::min<int64_t>(k, K);
    if (nout > 0)
      MM_CUDA_TRY(cudaMemcpyAsync(out_topk, cur_buf, sizeof(mm_move) * (size_t)nout,
                                  out_kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    MM_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_kept) *n_kept = K;
    if (n_methods_with_kept) *n_methods_with_kept = (int64_t)hc[1];
    mm_set_error("");
    return MM_OK;
  } catch (const MmError &e) {
    mm_set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc &) {
    mm_set_error("host allocation failed");
    return MM_ENOMEM;
  } catch (...) {
    mm_set_error("unexpected exception");
    return MM_ECUDA;
  }
}
