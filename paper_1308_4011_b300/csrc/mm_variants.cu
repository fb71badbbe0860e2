// LCOM and CBO variants (Sec. II.B) and classes ranked by a metric.
//
// Sharing over every accessed attribute.  The methods of class C that share
// an accessed attribute with x (in C) are the union, over x's accesses
// (x, a), of the methods of C that access a.  Sorting all accesses by the key
// (a, class of the accessing method) puts each of those sets in one run of
// equal keys, so q_all(x) is the size of the union of the runs of x's
// accesses minus one (x is in each of them); Q_all(C) = sum of q_all / 2.  A
// method with one access takes its run's length; a method with more takes
// the whole warp, which forms the union in a bitmap over C's method ranks
// (the bitmap of the own-attribute LCOM pass, left zero after each union).
//
// Coupling both ways.  Row Y of the class multigraph lists the classes Y
// uses, ascending.  The classes using E are counted by a histogram over all
// row entries; an entry (Y, E) whose row E also holds Y (a binary search) is
// a pair coupled both ways, so |out u in| = out + in - those pairs.
//
// Ranking.  A class's value is mapped to an unsigned key whose ascending
// order is the value's descending order; a stable LSD radix sort of the keys
// with the class ids (ascending) as values leaves equal values in id order.
#include <cuda_runtime.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, TPB), B300_SMS * 32));
}

// the method of every access (the row of the access CSR)
__global__ void access_rows(const int64_t *acc_rowptr, int32_t M, int32_t *acc_row) {
  pdl_wait();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) acc_row[e] = (int32_t)x;
}

// key of access e = attribute * c + class of the accessing method; value e
__global__ void access_keys(const int32_t *acc_idx, const int32_t *acc_row, const int32_t *method_class,
                            int64_t n_acc, int32_t c, uint64_t *keys, uint32_t *vals) {
  pdl_wait();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_acc; e += (int64_t)gridDim.x * blockDim.x) {
    keys[e] = (uint64_t)(uint32_t)acc_idx[e] * (uint64_t)(uint32_t)c + (uint64_t)(uint32_t)method_class[acc_row[e]];
    vals[e] = (uint32_t)e;
  }
}

// after the sort: the class-local rank of the accessing method at every
// position, and the position of every access
__global__ void access_positions(const uint32_t *vals, const int32_t *acc_row, const int32_t *method_local,
                                 int64_t n_acc, int32_t *sorted_rank, int32_t *pos_of) {
  pdl_wait();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_acc; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = vals[p];
    sorted_rank[p] = method_local[acc_row[e]];
    pos_of[e] = (int32_t)p;
  }
}

// for every access e, the run [lo, hi) of positions whose key equals its own
__global__ void access_runs(const uint64_t *keys, const int32_t *pos_of, int64_t n_acc, int2 *run) {
  pdl_wait();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_acc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = pos_of[e];
    const uint64_t k = keys[p];
    int64_t lo = 0, hi = p;  // first position in [0, p] holding k
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    int64_t lo2 = p + 1, hi2 = n_acc;  // first position after p holding a larger key
    while (lo2 < hi2) {
      const int64_t mid = (lo2 + hi2) >> 1;
      if (keys[mid] <= k) lo2 = mid + 1; else hi2 = mid;
    }
    run[e] = make_int2((int32_t)lo, (int32_t)lo2);
  }
}

// Size of the union of the class-local ranks at sorted_rank[r.x .. r.y) over
// the runs r of one method's accesses, formed in the warp's bitmap bm (zero
// before and after).  Phase 0 sets every bit; phase 1 reads each word back
// with an exchange that clears it, so a bit is counted once.  Every lane
// returns the count.
__device__ int32_t runs_union(const int2 *runs, int64_t len, const int32_t *sorted_rank, uint32_t *bm,
                              uint32_t lane) {
  int32_t cnt = 0;
  for (int phase = 0; phase < 2; ++phase) {
    for (int64_t e0 = 0; e0 < len; e0 += 32) {
      const int2 r = e0 + lane < len ? runs[e0 + lane] : make_int2(0, 0);
      const int32_t n = r.y - r.x;
      int32_t incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
      }
      const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
      for (int32_t k0 = 0; k0 < total; k0 += 32) {
        const int32_t k = k0 + (int32_t)lane;
        int32_t lo = 0, hi = 31;  // the lane whose run holds element k
#pragma unroll
        for (int step = 0; step < 5; ++step) {
          const int32_t mid = (lo + hi) >> 1;
          if (__shfl_sync(0xffffffffu, incl, mid) > k) hi = mid; else lo = mid + 1;
        }
        const int32_t excl = __shfl_sync(0xffffffffu, incl, lo) - __shfl_sync(0xffffffffu, n, lo);
        const int32_t start = __shfl_sync(0xffffffffu, r.x, lo);
        if (k < total) {
          const int32_t j = sorted_rank[start + (k - excl)];
          if (phase == 0) atomicOr(&bm[j >> 5], 1u << (j & 31));
          else cnt += __popc(atomicExch(&bm[j >> 5], 0u));
        }
      }
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  return cnt;
}

// q_all per method and 2 Q_all per class.  A warp owns g consecutive methods
// (one per lane) and takes groups from a counter; methods with two or more
// accesses take the whole warp in turn.
__global__ void __launch_bounds__(256) lcom_all_union(const int32_t *method_class, const int64_t *acc_rowptr,
                                                      const int2 *run, const int32_t *sorted_rank, int32_t M,
                                                      int32_t words, uint32_t *gbm, int32_t *q_all,
                                                      int64_t *cls_twice, int32_t g, unsigned long long *next) {
  pdl_wait();
  extern __shared__ uint32_t va_smem[];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint32_t *bm = gbm ? gbm + ((int64_t)blockIdx.x * (blockDim.x >> 5) + wid) * words : va_smem + wid * words;
  if (!gbm)
    for (int32_t i = (int32_t)lane; i < words; i += 32) bm[i] = 0u;
  __syncwarp();
  auto take = [&]() { return __shfl_sync(0xffffffffu, lane == 0 ? (int64_t)atomicAdd(next, 1ull) : (int64_t)0, 0); };
  for (int64_t wg = take(); wg * g < M; wg = take()) {
    const int64_t base = wg * g, x = base + lane;
    const bool mine = lane < (uint32_t)g && x < M;
    const int64_t a0 = mine ? acc_rowptr[x] : 0;
    const int64_t deg = mine ? acc_rowptr[x + 1] - a0 : 0;
    int32_t u = 0;
    if (deg == 1) {
      const int2 r = run[a0];
      u = r.y - r.x;
    }
    uint32_t multi = __ballot_sync(0xffffffffu, deg >= 2);
    while (multi) {
      const int src = __ffs(multi) - 1;
      multi &= multi - 1u;
      const int64_t as = __shfl_sync(0xffffffffu, a0, src);
      const int64_t ds = __shfl_sync(0xffffffffu, deg, src);
      const int32_t v = runs_union(run + as, ds, sorted_rank, bm, lane);
      if ((int)lane == src) u = v;
    }
    if (mine) {
      const int32_t qx = u > 0 ? u - 1 : 0;
      q_all[x] = qx;
      if (qx) atomicAdd(reinterpret_cast<unsigned long long *>(&cls_twice[method_class[x]]), (unsigned long long)qx);
    }
  }
}

// classes using each class: a histogram over the multigraph's entries
__global__ void cbo_incoming(const int64_t *mg_rowptr, const int32_t *mg_dst, int32_t c, int32_t *cbo_in) {
  pdl_wait();
  const int64_t u = mg_rowptr[c];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cbo_in[mg_dst[k]], 1);
}

// entries (Y, E) whose row E holds Y: pairs coupled both ways, counted at Y
__global__ void cbo_mutual(const int64_t *mg_rowptr, const int32_t *mg_dst, int32_t c, int32_t *mutual) {
  pdl_wait();
  const int64_t u = mg_rowptr[c];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = c;  // the row of entry k: the last Y with mg_rowptr[Y] <= k
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (mg_rowptr[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const int32_t Y = (int32_t)lo, E = mg_dst[k];
    int64_t a = mg_rowptr[E], b = mg_rowptr[E + 1];
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if (mg_dst[mid] < Y) a = mid + 1; else b = mid;
    }
    if (a < mg_rowptr[E + 1] && mg_dst[a] == Y) atomicAdd(&mutual[Y], 1);
  }
}

__global__ void variants_finalize(const int32_t *cls_n, const int64_t *cls_P, const int64_t *cls_Q,
                                  const int64_t *cls_twice, const int32_t *cls_cbo, const int32_t *cbo_in,
                                  const int32_t *mutual, int32_t c, mm_class_variants *out) {
  pdl_wait();
  for (int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; C < c; C += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = cls_n[C];
    mm_class_variants v;
    v.Q_all = cls_twice[C] / 2;
    v.P_all = n * (n - 1) / 2 - v.Q_all;
    v.lcom_ck_all = v.P_all > v.Q_all ? v.P_all - v.Q_all : 0;
    v.lcom_pq = cls_P[C] - cls_Q[C];
    v.lcom_pq_all = v.P_all - v.Q_all;
    v.cbo_out = cls_cbo[C];
    v.cbo_in = cbo_in[C];
    v.cbo_bi = v.cbo_out + v.cbo_in - mutual[C];
    v.reserved = 0;
    out[C] = v;
  }
}

// ascending key order = descending value order
__device__ __forceinline__ uint64_t descending_key(int64_t v) {
  return ~((uint64_t)v ^ 0x8000000000000000ull);
}

__global__ void rank_keys(int32_t metric, const int64_t *cls_P, const int64_t *cls_Q, const int32_t *cls_cbo,
                          const mm_class_variants *var, int32_t c, uint64_t *keys, uint32_t *ids) {
  pdl_wait();
  for (int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; C < c; C += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = 0;
    switch (metric) {
      case MM_RANK_LCOM_CK: v = cls_P[C] > cls_Q[C] ? cls_P[C] - cls_Q[C] : 0; break;
      case MM_RANK_LCOM_PQ: v = cls_P[C] - cls_Q[C]; break;
      case MM_RANK_LCOM_CK_ALL: v = var[C].lcom_ck_all; break;
      case MM_RANK_LCOM_PQ_ALL: v = var[C].lcom_pq_all; break;
      case MM_RANK_CBO: v = cls_cbo[C]; break;
      case MM_RANK_CBO_IN: v = var[C].cbo_in; break;
      default: v = var[C].cbo_bi; break;
    }
    keys[C] = descending_key(v);
    ids[C] = (uint32_t)C;
  }
}

__global__ void rank_values(const uint64_t *keys, int64_t k, int64_t *values) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    values[i] = (int64_t)(~keys[i] ^ 0x8000000000000000ull);
}

}  // namespace

// The variants of every class into s's variant buffers (device); returns
// them (n_classes entries) and q_all (n_methods entries).
void compute_variants(mm_system *s, mm_class_variants **out, int32_t **q_all_out) {
  cudaStream_t st = s->stream;
  const int32_t c = s->c, M = s->M;
  const int64_t n_acc = s->n_acc;
  Carve cv{static_cast<char *>(s->var_ws.need(
      256 * 16 + sizeof(int32_t) * (size_t)(3 * (int64_t)n_acc + M + 2 * (int64_t)c) +
          sizeof(int2) * (size_t)n_acc + sizeof(int64_t) * (size_t)c + sizeof(mm_class_variants) * (size_t)c,
      st))};
  int32_t *acc_row = cv.take<int32_t>(n_acc);
  int32_t *sorted_rank = cv.take<int32_t>(n_acc);
  int32_t *pos_of = cv.take<int32_t>(n_acc);
  int2 *run = cv.take<int2>(n_acc);
  int32_t *q_all = cv.take<int32_t>(M);
  int64_t *twice = cv.take<int64_t>(c);
  int32_t *cbo_in = cv.take<int32_t>(c);
  int32_t *mutual = cv.take<int32_t>(c);
  mm_class_variants *var = cv.take<mm_class_variants>(c);
  MM_CUDA_TRY(cudaMemsetAsync(twice, 0, sizeof(int64_t) * (size_t)c, st));
  MM_CUDA_TRY(cudaMemsetAsync(cbo_in, 0, sizeof(int32_t) * (size_t)c, st));
  MM_CUDA_TRY(cudaMemsetAsync(mutual, 0, sizeof(int32_t) * (size_t)c, st));
  MM_CUDA_TRY(cudaMemsetAsync(q_all, 0, sizeof(int32_t) * (size_t)std::max(M, 1), st));
  if (n_acc > 0) {
    Carve kv{static_cast<char *>(
        s->var_keys_ws.need(256 * 8 + (2 * sizeof(uint64_t) + 2 * sizeof(uint32_t)) * (size_t)n_acc, st))};
    uint64_t *keys = kv.take<uint64_t>(n_acc);
    uint64_t *keys_alt = kv.take<uint64_t>(n_acc);
    uint32_t *vals = kv.take<uint32_t>(n_acc);
    uint32_t *vals_alt = kv.take<uint32_t>(n_acc);
    pdl_launch(access_rows, grid_for(M), TPB, 0, st, s->acc_rowptr, M, acc_row);
    MM_LAUNCH_CHECK();
    pdl_launch(access_keys, grid_for(n_acc), TPB, 0, st, s->acc_idx, static_cast<const int32_t *>(acc_row),
               s->method_class, n_acc, c, keys, vals);
    MM_LAUNCH_CHECK();
    radix_sort_u64(keys, keys_alt, vals, vals_alt, n_acc,
                   bits_for((uint64_t)std::max(s->A, 1) * (uint64_t)c - 1), s->sort_ws, st);
    pdl_launch(access_positions, grid_for(n_acc), TPB, 0, st, static_cast<const uint32_t *>(vals),
               static_cast<const int32_t *>(acc_row), s->method_local, n_acc, sorted_rank, pos_of);
    MM_LAUNCH_CHECK();
    pdl_launch(access_runs, grid_for(n_acc), TPB, 0, st, static_cast<const uint64_t *>(keys),
               static_cast<const int32_t *>(pos_of), n_acc, run);
    MM_LAUNCH_CHECK();
    const int32_t g = M >= B300_SMS * 64 * 32 ? 32 : (M >= B300_SMS * 64 * 16 ? 16 : 8);
    const UnionBitmap ub = union_bitmap(s, ceil_div((int64_t)M, g), s->union_ws, st);
    MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 8, 0, sizeof(unsigned long long), st));
    pdl_launch(lcom_all_union, ub.grid, 256, ub.smem, st, s->method_class, s->acc_rowptr,
               static_cast<const int2 *>(run), static_cast<const int32_t *>(sorted_rank), M, ub.words, ub.gbm, q_all,
               twice, g, s->d_u64 + 8);
    MM_LAUNCH_CHECK();
  }
  pdl_launch(cbo_incoming, B300_SMS * 8, TPB, 0, st, s->mg_rowptr, s->mg_dst, c, cbo_in);
  MM_LAUNCH_CHECK();
  pdl_launch(cbo_mutual, B300_SMS * 8, TPB, 0, st, s->mg_rowptr, s->mg_dst, c, mutual);
  MM_LAUNCH_CHECK();
  pdl_launch(variants_finalize, grid_for(c), TPB, 0, st, s->cls_n, s->cls_P, s->cls_Q,
             static_cast<const int64_t *>(twice), s->cls_cbo, static_cast<const int32_t *>(cbo_in),
             static_cast<const int32_t *>(mutual), c, var);
  MM_LAUNCH_CHECK();
  *out = var;
  *q_all_out = q_all;
}

// The first k classes by `metric` (ids, and values when non-null) into
// device or host memory.
void rank_classes(mm_system *s, int32_t metric, int32_t k, int32_t *out_ids, int64_t *out_values, int32_t kind) {
  cudaStream_t st = s->stream;
  const int32_t c = s->c;
  const mm_class_variants *var = nullptr;
  if (metric == MM_RANK_LCOM_CK_ALL || metric == MM_RANK_LCOM_PQ_ALL || metric == MM_RANK_CBO_IN ||
      metric == MM_RANK_CBO_BI) {
    mm_class_variants *v = nullptr;
    int32_t *q = nullptr;
    compute_variants(s, &v, &q);
    var = v;
  }
  const int64_t n_out = std::min<int64_t>(k, c);
  Carve kv{static_cast<char *>(s->var_keys_ws.need(256 * 8 + (2 * sizeof(uint64_t) + 2 * sizeof(uint32_t) +
                                                                sizeof(int64_t)) * (size_t)c, st))};
  uint64_t *keys = kv.take<uint64_t>(c);
  uint64_t *keys_alt = kv.take<uint64_t>(c);
  uint32_t *ids = kv.take<uint32_t>(c);
  uint32_t *ids_alt = kv.take<uint32_t>(c);
  int64_t *values = kv.take<int64_t>(c);
  pdl_launch(rank_keys, grid_for(c), TPB, 0, st, metric, s->cls_P, s->cls_Q, s->cls_cbo, var, c, keys, ids);
  MM_LAUNCH_CHECK();
  radix_sort_u64(keys, keys_alt, ids, ids_alt, c, 64, s->sort_ws, st);
  if (n_out <= 0) return;
  const cudaMemcpyKind dir = kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  MM_CUDA_TRY(cudaMemcpyAsync(out_ids, ids, sizeof(int32_t) * (size_t)n_out, dir, st));
  if (out_values) {
    pdl_launch(rank_values, grid_for(n_out), TPB, 0, st, static_cast<const uint64_t *>(keys), n_out, values);
    MM_LAUNCH_CHECK();
    MM_CUDA_TRY(cudaMemcpyAsync(out_values, values, sizeof(int64_t) * (size_t)n_out, dir, st));
  }
}
