// Jaccard similarity of method pairs (Sec. II.A) and the suggestions of rule
// R1 (Sec. III.A, first rule, with the average similarity as its threshold).
//
// The properties of a method are the methods it calls and the attributes it
// accesses.  sim(x, y) = |P(x) & P(y)| / |P(x) | P(y)| is kept as the exact
// pair (i, u); only pairs with a common property are values (Sec. IV.C: only
// meaningful, non-zero values are stored).  Instead of the m(m-1)/2 pairs of
// the paper's siml(), the pairs that share a property come from an inverted
// index: for every property, each pair of the methods holding it is one
// co-occurrence (key x * M + y, x < y); sorting the keys and counting equal
// runs gives i for every pair at once, and u = |P(x)| + |P(y)| - i.  Work is
// proportional to the co-occurrences, sum over properties of deg(deg-1)/2.
//
// R1: a pair in different classes whose similarity exceeds the average of
// all similarity values proposes moving either method to the other's class,
// or to another class holding a method it calls.
// The average is taken on the host in double precision in one fixed order
// (sum over u ascending of sum(i)/u, over the number of values), and turned
// into the smallest i per u that exceeds it, so the device decides each pair
// with an integer comparison that equals the double comparison.  The proposed
// moves (distinct, as candidate lists) are then evaluated and filtered like
// any candidate list (mm_suggest_moves).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mm_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, TPB), B300_SMS * 32));
}

// properties per method: |calls(x)| + |acc(x)|
__global__ void property_counts(const int64_t *call_rowptr, const int64_t *acc_rowptr, int32_t M, int32_t *np) {
  pdl_wait();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    np[x] = (int32_t)((call_rowptr[x + 1] - call_rowptr[x]) + (acc_rowptr[x + 1] - acc_rowptr[x]));
}

// holders of each property: property t < M is "calls method t", M + a is
// "accesses attribute a"; deg[p] = number of holders
__global__ void property_degrees(const int32_t *call_idx, int64_t n_call, const int32_t *acc_idx, int64_t n_acc,
                                 int32_t M, int32_t *deg) {
  pdl_wait();
  const int64_t n = n_call + n_acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[e < n_call ? call_idx[e] : M + acc_idx[e - n_call]], 1);
}

// posting lists: the holders of p at post[post_ptr[p] ..] (any order)
__global__ void property_postings(const int64_t *call_rowptr, const int32_t *call_idx, const int64_t *acc_rowptr,
                                  const int32_t *acc_idx, int32_t M, const int64_t *post_ptr, int32_t *cursor,
                                  int32_t *post, int32_t *post_prop) {
  pdl_wait();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = call_rowptr[x]; e < call_rowptr[x + 1]; ++e) {
      const int32_t p = call_idx[e];
      const int64_t q = post_ptr[p] + atomicAdd(&cursor[p], 1);
      post[q] = (int32_t)x;
      post_prop[q] = p;
    }
    for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
      const int32_t p = M + acc_idx[e];
      const int64_t q = post_ptr[p] + atomicAdd(&cursor[p], 1);
      post[q] = (int32_t)x;
      post_prop[q] = p;
    }
  }
}

// co-occurrences of property p: deg(deg - 1) / 2
__global__ void cooccurrence_counts(const int32_t *deg, int64_t n_prop, int64_t *cnt) {
  pdl_wait();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_prop; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = deg[p];
    cnt[p] = d * (d - 1) / 2;
  }
}

__global__ void max_reduce(const int32_t *v, int64_t n, int32_t *out) {
  pdl_wait();
  int32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// One thread per posting entry q (holder a of property p): the keys of the
// pairs (holder a, holder b) for b after a in the list, at the entry's offset.
__global__ void cooccurrence_keys(const int32_t *post, const int32_t *post_prop, int64_t n_post,
                                  const int64_t *post_ptr, const int64_t *pair_off, int32_t M, uint64_t *keys) {
  pdl_wait();
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_post;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = post_prop[q];
    const int64_t b0 = post_ptr[p], d = post_ptr[p + 1] - b0, a = q - b0;
    int64_t o = pair_off[p] + a * (d - 1) - a * (a - 1) / 2;  // pairs of the holders before a
    const uint64_t x = (uint64_t)post[q];
    for (int64_t b = a + 1; b < d; ++b) {
      const uint64_t y = (uint64_t)post[b0 + b];
      keys[o++] = x < y ? x * (uint64_t)M + y : y * (uint64_t)M + x;
    }
  }
}

// first key of each run of equal sorted keys
__global__ void run_heads(const uint64_t *keys, int64_t n, int32_t *flag) {
  pdl_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    flag[k] = (k == 0 || keys[k - 1] != keys[k]) ? 1 : 0;
}

// every run becomes one value (x, y, i, u); the sum of i per u for the average.
// u takes few distinct values, so the sums are gathered per block in shared
// memory (when u's range fits) and added to the global ones once per block.
constexpr int SV_HIST_MAX = 4096;  // u in [0, SV_HIST_MAX): shared-memory sums

__global__ void similarity_values(const uint64_t *keys, int64_t n, const int32_t *flag, const int64_t *pos,
                                  const int32_t *np, int32_t M, int32_t *px, int32_t *py, int32_t *pi, int32_t *pu,
                                  unsigned long long *sum_i, int32_t umax) {
  pdl_wait();
  extern __shared__ unsigned long long sv_sum[];
  const bool local = umax < SV_HIST_MAX;
  if (local) {
    for (int32_t t = threadIdx.x; t <= umax; t += blockDim.x) sv_sum[t] = 0ull;
    __syncthreads();
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[k]) continue;
    const uint64_t key = keys[k];
    int64_t run = 1;
    while (k + run < n && keys[k + run] == key) ++run;
    const int32_t x = (int32_t)(key / (uint64_t)M), y = (int32_t)(key % (uint64_t)M);
    const int32_t i = (int32_t)run, u = np[x] + np[y] - i;
    const int64_t o = pos[k];
    px[o] = x;
    py[o] = y;
    pi[o] = i;
    pu[o] = u;
    atomicAdd(local ? &sv_sum[u] : &sum_i[u], (unsigned long long)i);
  }
  if (local) {
    __syncthreads();
    for (int32_t t = threadIdx.x; t <= umax; t += blockDim.x)
      if (sv_sum[t]) atomicAdd(&sum_i[t], sv_sum[t]);
  }
}

// Moves proposed by the high pairs: x -> cls(y) and y -> cls(x) when the
// classes differ and i >= thr[u]; keys m * c + D.  A warp reserves its output
// slots with one atomicAdd.  Both methods of such a pair are marked as
// proposers.
__global__ void high_pair_moves(const int32_t *px, const int32_t *py, const int32_t *pi, const int32_t *pu,
                                int64_t n, const int32_t *thr, const int32_t *method_class, int32_t c,
                                uint64_t *keys, unsigned long long *count, uint8_t *proposer) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x; k0 < n; k0 += stride) {
    const int64_t k = k0 + threadIdx.x;
    bool high = false;
    int32_t x = 0, y = 0, cx = 0, cy = 0;
    if (k < n) {
      x = px[k];
      y = py[k];
      cx = method_class[x];
      cy = method_class[y];
      high = cx != cy && pi[k] >= thr[pu[k]];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, high);
    if (!bal) continue;
    unsigned long long base = 0;
    const int leader = __ffs(bal) - 1;
    if ((int)lane == leader) base = atomicAdd(count, 2ull * __popc(bal));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (high) {
      const unsigned long long o = base + 2ull * __popc(bal & ((1u << lane) - 1u));
      keys[o] = (uint64_t)x * (uint64_t)c + (uint64_t)cy;
      keys[o + 1] = (uint64_t)y * (uint64_t)c + (uint64_t)cx;
      proposer[x] = 1;
      proposer[y] = 1;
    }
  }
}

// The other moves of a proposer: to the class of each method it calls (when
// not its own); keys appended after the pair moves.
__global__ void called_class_moves(const uint8_t *proposer, const int64_t *call_rowptr, const int32_t *call_idx,
                                   const int32_t *method_class, int32_t M, int32_t c, uint64_t *keys,
                                   unsigned long long *count) {
  pdl_wait();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
    if (!proposer[x]) continue;
    const int32_t C = method_class[x];
    int32_t nk = 0;
    for (int64_t e = call_rowptr[x]; e < call_rowptr[x + 1]; ++e) nk += method_class[call_idx[e]] != C;
    if (!nk) continue;
    unsigned long long o = atomicAdd(count, (unsigned long long)nk);
    for (int64_t e = call_rowptr[x]; e < call_rowptr[x + 1]; ++e) {
      const int32_t D = method_class[call_idx[e]];
      if (D != C) keys[o++] = (uint64_t)x * (uint64_t)c + (uint64_t)D;
    }
  }
}

// distinct sorted move keys -> per-method counts (rows) and the destinations
__global__ void move_lists(const uint64_t *keys, int64_t n, const int32_t *flag, const int64_t *pos, int32_t c,
                           int64_t *row_cnt, int32_t *dst) {
  pdl_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[k]) continue;
    const uint64_t key = keys[k];
    atomicAdd(reinterpret_cast<unsigned long long *>(&row_cnt[key / (uint64_t)c]), 1ull);
    dst[pos[k]] = (int32_t)(key % (uint64_t)c);
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

namespace {

void read_back(void *host, const void *dev, size_t bytes, cudaStream_t st) {
  MM_CUDA_TRY(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace

// The similarity values of the system's current state into s->sim_* (device),
// with their count, the largest union and the average.
void compute_similarity(mm_system *s) {
  cudaStream_t st = s->stream;
  const int32_t M = s->M;
  const int64_t n_call = s->n_call, n_acc = s->n_acc, n_prop = (int64_t)M + s->A, n_post = n_call + n_acc;
  s->sim_n = 0;
  s->sim_cooc = 0;
  s->sim_umax = 0;
  s->sim_avg = 0.0;
  if (M < 2 || n_post == 0) return;
  // posting lists and co-occurrence offsets (sizes known up front)
  const size_t need = 8 * 256 + sizeof(int32_t) * ((size_t)M + 2 * (size_t)n_prop + 2 * (size_t)n_post + 4) +
                      sizeof(int64_t) * 2 * ((size_t)n_prop + 1);
  Carve cv{static_cast<char *>(s->sim_ws.need(need, st))};
  int32_t *np = cv.take<int32_t>(M);
  int32_t *deg = cv.take<int32_t>(n_prop);
  int64_t *post_ptr = cv.take<int64_t>(n_prop + 1);
  int64_t *pair_off = cv.take<int64_t>(n_prop + 1);
  int32_t *post = cv.take<int32_t>(n_post);
  int32_t *post_prop = cv.take<int32_t>(n_post);
  int32_t *ctr = cv.take<int32_t>(4);
  s->sim_np = np;
  MM_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)n_prop, st));
  MM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(int32_t) * 4, st));
  pdl_launch(property_counts, grid_for(M), TPB, 0, st, s->call_rowptr, s->acc_rowptr, M, np);
  MM_LAUNCH_CHECK();
  pdl_launch(max_reduce, grid_for(M), TPB, 0, st, static_cast<const int32_t *>(np), (int64_t)M, ctr);
  MM_LAUNCH_CHECK();
  pdl_launch(property_degrees, grid_for(n_post), TPB, 0, st, s->call_idx, n_call, s->acc_idx, n_acc, M, deg);
  MM_LAUNCH_CHECK();
  scan_exclusive_i32to64(deg, post_ptr, n_prop, s->sort_ws, st, post_ptr + n_prop);
  pdl_launch(cooccurrence_counts, grid_for(n_prop), TPB, 0, st, static_cast<const int32_t *>(deg), n_prop, pair_off);
  MM_LAUNCH_CHECK();
  scan_exclusive_i64(pair_off, pair_off, n_prop, pair_off + n_prop, s->sort_ws, st);  // counts -> offsets
  MM_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)n_prop, st));           // reused as cursors
  pdl_launch(property_postings, grid_for(M), TPB, 0, st, s->call_rowptr, s->call_idx, s->acc_rowptr, s->acc_idx, M,
             static_cast<const int64_t *>(post_ptr), deg, post, post_prop);
  MM_LAUNCH_CHECK();
  // the number of co-occurrences and the largest property count, read back together
  int64_t n_co = 0;
  int32_t max_np = 0;
  MM_CUDA_TRY(cudaMemcpyAsync(&n_co, pair_off + n_prop, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaMemcpyAsync(&max_np, ctr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_co >= ((int64_t)1 << 32)) throw MmError{MM_EBUDGET, "similarity: more than 2^32 co-occurring method pairs"};
  s->sim_umax = 2 * max_np;
  s->sim_cooc = n_co;
  if (n_co == 0) return;
  // keys, sorted, runs counted
  Carve kv{static_cast<char *>(s->sim_keys_ws.need(
      (2 * sizeof(uint64_t) + sizeof(int32_t) + sizeof(int64_t)) * (size_t)n_co + 6 * 256 +
          sizeof(unsigned long long) * (size_t)(s->sim_umax + 2),
      st))};
  uint64_t *keys = kv.take<uint64_t>(n_co);
  uint64_t *keys_alt = kv.take<uint64_t>(n_co);
  int32_t *flag = kv.take<int32_t>(n_co);
  int64_t *pos = kv.take<int64_t>(n_co);
  unsigned long long *sum_i = kv.take<unsigned long long>(s->sim_umax + 1);
  pdl_launch(cooccurrence_keys, grid_for(n_post), TPB, 0, st, static_cast<const int32_t *>(post),
             static_cast<const int32_t *>(post_prop), n_post, static_cast<const int64_t *>(post_ptr),
             static_cast<const int64_t *>(pair_off), M, keys);
  MM_LAUNCH_CHECK();
  radix_sort_u64(keys, keys_alt, nullptr, nullptr, n_co, bits_for((uint64_t)M * (uint64_t)M - 1), s->sort_ws, st);
  pdl_launch(run_heads, grid_for(n_co), TPB, 0, st, static_cast<const uint64_t *>(keys), n_co, flag);
  MM_LAUNCH_CHECK();
  scan_exclusive_i32to64(flag, pos, n_co, s->sort_ws, st);
  int64_t last_pos = 0;
  int32_t last_flag = 0;
  MM_CUDA_TRY(cudaMemcpyAsync(&last_pos, pos + n_co - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaMemcpyAsync(&last_flag, flag + n_co - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t n_val = last_pos + last_flag;
  Carve vv{static_cast<char *>(s->sim_val_ws.need(4 * (sizeof(int32_t) * (size_t)n_val + 256), st))};
  s->sim_x = vv.take<int32_t>(n_val);
  s->sim_y = vv.take<int32_t>(n_val);
  s->sim_i = vv.take<int32_t>(n_val);
  s->sim_u = vv.take<int32_t>(n_val);
  MM_CUDA_TRY(cudaMemsetAsync(sum_i, 0, sizeof(unsigned long long) * (size_t)(s->sim_umax + 1), st));
  const size_t sv_smem = s->sim_umax < SV_HIST_MAX ? sizeof(unsigned long long) * ((size_t)s->sim_umax + 1) : 0;
  pdl_launch(similarity_values, (unsigned)std::min<int64_t>(ceil_div(n_co, TPB), B300_SMS * 8), TPB, sv_smem, st,
             static_cast<const uint64_t *>(keys), n_co, static_cast<const int32_t *>(flag),
             static_cast<const int64_t *>(pos), static_cast<const int32_t *>(np), M, s->sim_x, s->sim_y, s->sim_i,
             s->sim_u, sum_i, s->sim_umax);
  MM_LAUNCH_CHECK();
  // the average over the values, in one fixed order (u ascending), on the host
  std::vector<unsigned long long> hs((size_t)s->sim_umax + 1);
  read_back(hs.data(), sum_i, sizeof(unsigned long long) * hs.size(), st);
  double acc = 0.0;
  for (int32_t u = 1; u <= s->sim_umax; ++u)
    if (hs[(size_t)u]) acc += (double)hs[(size_t)u] / (double)u;
  s->sim_n = n_val;
  s->sim_avg = n_val > 0 ? acc / (double)n_val : 0.0;
}

// Rule R1's candidate lists from the similarity values: device CSR over the
// methods in s->r1_rowptr / s->r1_dst, with their counts.
void build_r1_candidates(mm_system *s, int64_t *n_high, int64_t *n_cand) {
  cudaStream_t st = s->stream;
  const int32_t M = s->M, c = s->c;
  *n_high = 0;
  *n_cand = 0;
  Carve cv{static_cast<char *>(s->r1_ws.need(sizeof(int64_t) * ((size_t)M + 1) + 512, st))};
  s->r1_rowptr = cv.take<int64_t>(M + 1);
  MM_CUDA_TRY(cudaMemsetAsync(s->r1_rowptr, 0, sizeof(int64_t) * ((size_t)M + 1), st));
  s->r1_dst = nullptr;
  if (s->sim_n == 0) return;
  // smallest i per u above the average: the same double comparison as the definition
  const int32_t umax = s->sim_umax;
  std::vector<int32_t> thr((size_t)umax + 1);
  for (int32_t u = 0; u <= umax; ++u) {
    int32_t t = u + 1;
    for (int32_t i = 0; i <= u; ++i)
      if (u > 0 && (double)i / (double)u > s->sim_avg) {
        t = i;
        break;
      }
    thr[(size_t)u] = t;
  }
  const int64_t nv = s->sim_n;
  const int64_t cap = 2 * nv + s->n_call;  // pair moves, then at most one move per call of a proposer
  Carve kv{static_cast<char *>(s->sim_keys_ws.need(((sizeof(uint64_t) * 2 + sizeof(int32_t) + sizeof(int64_t)) *
                                                     (size_t)cap) + 8 * 256 + (size_t)M +
                                                        sizeof(int32_t) * (size_t)(umax + 1) + 64,
                                                    st))};
  uint64_t *keys = kv.take<uint64_t>(cap);
  uint64_t *keys_alt = kv.take<uint64_t>(cap);
  int32_t *flag = kv.take<int32_t>(cap);
  int64_t *pos = kv.take<int64_t>(cap);
  int32_t *dthr = kv.take<int32_t>(umax + 1);
  unsigned long long *count = kv.take<unsigned long long>(2);
  uint8_t *proposer = kv.take<uint8_t>(M);
  MM_CUDA_TRY(cudaMemcpyAsync(dthr, thr.data(), sizeof(int32_t) * thr.size(), cudaMemcpyHostToDevice, st));
  MM_CUDA_TRY(cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), st));
  MM_CUDA_TRY(cudaMemsetAsync(proposer, 0, (size_t)M, st));
  pdl_launch(high_pair_moves, grid_for(nv), TPB, 0, st, static_cast<const int32_t *>(s->sim_x),
             static_cast<const int32_t *>(s->sim_y), static_cast<const int32_t *>(s->sim_i),
             static_cast<const int32_t *>(s->sim_u), nv, static_cast<const int32_t *>(dthr),
             static_cast<const int32_t *>(s->method_class), c, keys, count, proposer);
  MM_LAUNCH_CHECK();
  // count[1] = the pair moves (2 per high pair), kept before the appends
  MM_CUDA_TRY(cudaMemcpyAsync(count + 1, count, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
  pdl_launch(called_class_moves, grid_for(M), TPB, 0, st, static_cast<const uint8_t *>(proposer), s->call_rowptr,
             s->call_idx, static_cast<const int32_t *>(s->method_class), M, c, keys, count);
  MM_LAUNCH_CHECK();
  unsigned long long nk[2] = {0, 0};
  read_back(nk, count, sizeof(nk), st);
  *n_high = (int64_t)(nk[1] / 2);
  if (nk[0] == 0) return;
  const int64_t n = (int64_t)nk[0];
  radix_sort_u64(keys, keys_alt, nullptr, nullptr, n, bits_for((uint64_t)M * (uint64_t)c - 1), s->sort_ws, st);
  pdl_launch(run_heads, grid_for(n), TPB, 0, st, static_cast<const uint64_t *>(keys), n, flag);
  MM_LAUNCH_CHECK();
  scan_exclusive_i32to64(flag, pos, n, s->sort_ws, st);
  int64_t last_pos = 0;
  int32_t last_flag = 0;
  MM_CUDA_TRY(cudaMemcpyAsync(&last_pos, pos + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaMemcpyAsync(&last_flag, flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t nd = last_pos + last_flag;
  Carve dv{static_cast<char *>(s->r1_ws.need(sizeof(int64_t) * ((size_t)M + 1) + sizeof(int32_t) * (size_t)nd + 1024,
                                            st))};
  s->r1_rowptr = dv.take<int64_t>(M + 1);
  s->r1_dst = dv.take<int32_t>(nd);
  int64_t *row_cnt = s->r1_rowptr;  // counts, scanned in place into row pointers
  MM_CUDA_TRY(cudaMemsetAsync(row_cnt, 0, sizeof(int64_t) * ((size_t)M + 1), st));
  pdl_launch(move_lists, grid_for(n), TPB, 0, st, static_cast<const uint64_t *>(keys), n,
             static_cast<const int32_t *>(flag), static_cast<const int64_t *>(pos), c, row_cnt, s->r1_dst);
  MM_LAUNCH_CHECK();
  scan_exclusive_i64(row_cnt, s->r1_rowptr, M, s->r1_rowptr + M, s->sort_ws, st);
  *n_cand = nd;
}
