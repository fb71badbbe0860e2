// Move Method evaluation (Sec. III.A rules, Sec. IV.C re-evaluation), done
// incrementally instead of recomputing the classes for every candidate.
//
// For a method m of class C moved to class D != C:
//   source C:  n' = n - 1, S' = S - own_m, Q' = Q - q_m, P' = P - (n - 1 - q_m)
//   target D:  n' = n + 1, S' = S + t,     Q' = Q + s,   P' = P + (n - s)
//              t = m's accesses to D's attributes, s = methods of D sharing one
//   CBO, through the class-use multigraph cnt[Y][E] (E != Y):
//     row C loses m's use edges and gains C->D for m's callers inside C,
//     row D gains m's use edges and loses D->C for m's callers inside D,
//     row X (any other class calling m) moves its edges from X->C to X->D.
//   Only C, D and the classes of m's callers can change.
//
// Everything that does not depend on D is prepared once per method (header,
// list L of the classes m uses with out_m[E], cnt[C][E], t and s, list R of
// the classes calling m with in_m[X] and cnt[X][C]).  The dense kernel gives
// each thread one destination D and walks a range of methods; the 32 lanes of
// a warp hold 32 consecutive D, so every adjacency probe of a warp is one
// 32-bit word, and the 16-byte records of a warp form one contiguous 512-byte
// store.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "mm_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n, int tpb = TPB) {
  int64_t g = ceil_div(n, tpb);
  if (g < 1) g = 1;
  if (g > 0x7fffffffLL) g = 0x7fffffffLL;
  return (unsigned)g;
}

__device__ __forceinline__ int32_t mg_lookup(const int64_t *rowptr, const int32_t *dst, const int32_t *cnt,
                                             int32_t Y, int32_t E) {
  int64_t lo = rowptr[Y], hi = rowptr[Y + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (dst[mid] < E) lo = mid + 1; else hi = mid;
  }
  return (lo < rowptr[Y + 1] && dst[lo] == E) ? cnt[lo] : 0;
}

// ---------------------------------------------------------------- precompute

// s for list-L entries with t > 0: the methods of D sharing an attribute of D
// with m = the union of the accessor lists of m's accesses into D (m is not in
// D).  One thread per entry: with t = 1 the union is the one accessor list, so
// s is its length; entries with t >= 2 are taken by the whole warp in turn
// (bitmap over D's method ranks, as in the LCOM counts).
__global__ void __launch_bounds__(256) l_entries_s(const int4 *l_list, const int32_t *l_x, const int64_t *n_l,
                                                   const int64_t *acc_rowptr, const int32_t *acc_idx,
                                                   const int32_t *attr_class, const int64_t *own_ptr,
                                                   const int32_t *own_list, int32_t words, uint32_t *gbm,
                                                   int32_t *l_s) {
  pdl_wait();
  extern __shared__ uint32_t ls_smem[];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint32_t *bm = gbm ? gbm + ((int64_t)blockIdx.x * (blockDim.x >> 5) + wid) * words : ls_smem + wid * words;
  if (!gbm)
    for (int32_t i = (int32_t)lane; i < words; i += 32) bm[i] = 0u;
  __syncwarp();
  const int64_t nl = *n_l;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nl; base += stride) {
    const int64_t l = base + threadIdx.x;
    int4 v = make_int4(0, 0, 0, 0);
    int32_t x = 0;
    if (l < nl) {
      v = l_list[l];
      x = l_x[l];
    }
    int32_t sv = 0;
    if (v.w == 1) {
      for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
        const int32_t al = acc_idx[e];
        if (attr_class[al] == v.x) {
          sv = (int32_t)(own_ptr[al + 1] - own_ptr[al]);
          break;
        }
      }
    }
    uint32_t multi = __ballot_sync(0xffffffffu, v.w >= 2);
    while (multi) {
      const int src = __ffs(multi) - 1;
      multi &= multi - 1u;
      const int32_t xs = __shfl_sync(0xffffffffu, x, src), Ds = __shfl_sync(0xffffffffu, v.x, src);
      const int64_t a0 = acc_rowptr[xs];
      const int32_t u = accessor_union(acc_idx + a0, acc_rowptr[xs + 1] - a0, Ds, attr_class, own_ptr, own_list,
                                       bm, lane);
      if ((int)lane == src) sv = u;
    }
    if (l < nl) l_s[l] = sv;
  }
}

// ---- lists L and R without a global sort
//
// Each method's use keys ((E << 1) | kind, kind 1 = an attribute access) are
// written at its segment call_rowptr[x] + acc_rowptr[x]; the class of every
// caller of x at its segment of a counting sort by callee (offsets: exclusive
// scan of fan-in).  One warp sorts each segment (rank by counting, ties by
// position, so the order is deterministic), then walks its runs twice: once to
// count the list entries (and the own-class run), once, after a scan of the
// counts, to write them in method order.

__global__ void method_use_keys32(const int32_t *__restrict__ method_class, const int64_t *__restrict__ call_rowptr,
                                  const int32_t *__restrict__ call_idx, const int64_t *__restrict__ acc_rowptr,
                                  const int32_t *__restrict__ acc_idx, const int32_t *__restrict__ attr_class,
                                  int32_t M, uint32_t *__restrict__ keys) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  const int64_t c0 = call_rowptr[x], c1 = call_rowptr[x + 1], a0 = acc_rowptr[x], a1 = acc_rowptr[x + 1];
  uint32_t *out = keys + c0 + a0;
#pragma unroll 4
  for (int64_t e = c0; e < c1; ++e) *out++ = (uint32_t)method_class[call_idx[e]] << 1;
#pragma unroll 4
  for (int64_t e = a0; e < a1; ++e) *out++ = ((uint32_t)attr_class[acc_idx[e]] << 1) | 1u;
}

// class of every caller y of x, bucketed by callee x (order inside a bucket is arbitrary)
__global__ void caller_classes_scatter(const int32_t *__restrict__ method_class,
                                       const int64_t *__restrict__ call_rowptr, const int32_t *__restrict__ call_idx,
                                       int32_t M, const int64_t *__restrict__ rin_off, int32_t *__restrict__ cursor,
                                       uint32_t *__restrict__ keys) {
  pdl_wait();
  int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= M) return;
  const uint32_t cy = (uint32_t)method_class[y];
  const int64_t e1 = call_rowptr[y + 1];
  for (int64_t e0 = call_rowptr[y]; e0 < e1; e0 += 4) {
    int32_t xs[4];
    int64_t off[4];
    int32_t slot[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xs[u] = e0 + u < e1 ? call_idx[e0 + u] : -1;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      off[u] = xs[u] >= 0 ? rin_off[xs[u]] : 0;
      slot[u] = xs[u] >= 0 ? atomicAdd(&cursor[xs[u]], 1) : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (xs[u] >= 0) keys[off[u] + slot[u]] = cy;
  }
}

// segment of x: [a[x] + (b ? b[x] : 0), a[x + 1] + (b ? b[x + 1] : 0))
__device__ __forceinline__ void segment(const int64_t *a, const int64_t *b, int64_t x, int64_t *p0, int64_t *len) {
  const int64_t s = a[x] + (b ? b[x] : 0), e = a[x + 1] + (b ? b[x + 1] : 0);
  *p0 = s;
  *len = e - s;
}

// Runs of a sorted segment of use keys (L) or caller classes (R).  For each run
// of equal classes, `f(class, n0, n1, index among the runs whose class is not
// C)` is called by one lane; n0/n1 count kind-0/kind-1 keys (R keys are all
// kind 0: the key is the class itself, so `shift` is 0 there).  Returns the
// number of runs whose class is not C.
template <class F>
__device__ __forceinline__ int32_t segment_runs(const uint32_t *keys, int64_t p0, int64_t len, int shift, int32_t C,
                                                uint32_t lane, F f) {
  if (len <= 32) {
    const bool act = (int64_t)lane < len;
    const uint32_t k = act ? keys[p0 + lane] : 0xffffffffu;
    const uint32_t kp = __shfl_up_sync(0xffffffffu, k, 1);
    const int32_t E = (int32_t)(k >> shift);
    const bool head = act && (lane == 0 || (kp >> shift) != (k >> shift));
    const bool acc = act && shift && (k & 1u);
    const uint32_t heads = __ballot_sync(0xffffffffu, head);
    const uint32_t accs = __ballot_sync(0xffffffffu, acc);
    const uint32_t other = __ballot_sync(0xffffffffu, head && E != C);
    if (head) {
      const uint32_t above = heads & ~((2u << lane) - 1u);
      const int32_t end = above ? __ffs(above) - 1 : (int32_t)len;
      const uint32_t run = (end >= 32 ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
      const int32_t n1 = __popc(accs & run), n = end - (int32_t)lane;
      f(E, n - n1, n1, __popc(other & ((1u << lane) - 1u)));
    }
    return __popc(other);
  }
  int32_t idx = 0;
  if (lane == 0) {
    int64_t i = 0;
    while (i < len) {
      const uint32_t E = keys[p0 + i] >> shift;
      int32_t n0 = 0, n1 = 0;
      for (; i < len && (keys[p0 + i] >> shift) == E; ++i) ((shift && (keys[p0 + i] & 1u)) ? n1 : n0)++;
      f((int32_t)E, n0, n1, idx);
      if ((int32_t)E != C) ++idx;
    }
  }
  return __shfl_sync(0xffffffffu, idx, 0);
}

// Sort and count, block version: a block of 256 threads takes 256 consecutive
// segments, whose keys are one contiguous range; it loads the range into shared
// memory (coalesced), each thread sorts its own segment there (insertion sort)
// and walks its runs, and the block writes the sorted range back.  Segments of
// more than SB_SEG keys, and every segment of a block whose range exceeds
// SB_KEYS, are left to the warp version (flag set).
constexpr int SB_KEYS = 6144;
constexpr int SB_SEG = 64;

__global__ void __launch_bounds__(256) segment_sort_count_block(const int64_t *a, const int64_t *b, int32_t M,
                                                                const uint32_t *in, uint32_t *out, int shift,
                                                                const int32_t *method_class, int32_t cbo_attrs,
                                                                int32_t *len_out, int32_t *self_out,
                                                                int32_t *work) {
  pdl_wait();
  __shared__ uint32_t sk[SB_KEYS];
  const int64_t x0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t xl = (x0 + (int64_t)blockDim.x < (int64_t)M ? x0 + (int64_t)blockDim.x : (int64_t)M) - 1;
  int64_t q0, l0, ql, ll;
  segment(a, b, x0, &q0, &l0);
  segment(a, b, xl, &ql, &ll);
  const int64_t K0 = q0, nk = ql + ll - q0;
  const bool fits = nk <= SB_KEYS;
  if (fits)
    for (int64_t k = threadIdx.x; k < nk; k += blockDim.x) sk[k] = in[K0 + k];
  __syncthreads();
  const int64_t x = x0 + threadIdx.x;
  bool warp_sort = false;
  if (x < M) {
    int64_t p0, len;
    segment(a, b, x, &p0, &len);
    if (!fits || len > SB_SEG) {
      warp_sort = true;
    } else {
      uint32_t *v = sk + (p0 - K0);
      for (int32_t i = 1; i < (int32_t)len; ++i) {  // insertion sort (stable)
        const uint32_t key = v[i];
        int32_t j = i - 1;
        while (j >= 0 && v[j] > key) {
          v[j + 1] = v[j];
          --j;
        }
        v[j + 1] = key;
      }
      const int32_t C = method_class[x];
      int32_t n = 0, self = 0;
      for (int32_t i = 0; i < (int32_t)len;) {
        const uint32_t E = v[i] >> shift;
        int32_t n0 = 0, n1 = 0;
        for (; i < (int32_t)len && (v[i] >> shift) == E; ++i) ((shift && (v[i] & 1u)) ? n1 : n0)++;
        if ((int32_t)E == C) self = n0 + (cbo_attrs ? n1 : 0);
        else ++n;
      }
      len_out[x] = n;
      self_out[x] = self;
    }
  }
  // segments left to the warp version go on its list (one atomic per warp)
  const uint32_t wm = __ballot_sync(0xffffffffu, warp_sort);
  if (wm) {
    const uint32_t lane = threadIdx.x & 31u;
    int32_t base = 0;
    if (lane == (uint32_t)(__ffs(wm) - 1)) base = atomicAdd(work, __popc(wm));
    base = __shfl_sync(0xffffffffu, base, __ffs(wm) - 1);
    if (warp_sort) work[1 + base + __popc(wm & ((1u << lane) - 1u))] = (int32_t)x;
  }
  __syncthreads();
  if (fits)
    for (int64_t k = threadIdx.x; k < nk; k += blockDim.x) out[K0 + k] = sk[k];
}

// Sort and count in one pass, warp version (segments the block version left):
// one warp sorts the segment (a segment of at most
// 32 keys also into its shared-memory row, read back for the run walk), then
// counts the runs: l_len / r_len per method and the own-class run (out_self /
// in_self).
__global__ void __launch_bounds__(256) segment_sort_count(const int64_t *a, const int64_t *b, int32_t M,
                                                          const uint32_t *in, uint32_t *out, int shift,
                                                          const int32_t *method_class, int32_t cbo_attrs,
                                                          int32_t *len_out, int32_t *self_out,
                                                          const int32_t *work) {
  pdl_wait();
  __shared__ uint32_t sk[8][32];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nwork = work[0];  // the methods the block version left
  for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nwork; wi += nwarps) {
    const int64_t x = work[1 + wi];
    int64_t p0, len;
    segment(a, b, x, &p0, &len);
    const uint32_t *runs_keys;
    int64_t runs_p0;
    __syncwarp();  // the previous segment's readers are done with the row
    if (len <= 32) {
      const uint32_t k = (int64_t)lane < len ? in[p0 + lane] : 0xffffffffu;
      int32_t rank = 0;
      for (int32_t j = 0; j < (int32_t)len; ++j) {
        const uint32_t kj = __shfl_sync(0xffffffffu, k, j);
        rank += (kj < k) || (kj == k && j < (int32_t)lane);
      }
      if ((int64_t)lane < len) {
        out[p0 + rank] = k;
        sk[wid][rank] = k;
      }
      runs_keys = sk[wid];
      runs_p0 = 0;
    } else {
      for (int64_t i = lane; i < len; i += 32) {
        const uint32_t k = in[p0 + i];
        int64_t rank = 0;
        for (int64_t j = 0; j < len; ++j) {
          const uint32_t kj = in[p0 + j];
          rank += (kj < k) || (kj == k && j < i);
        }
        out[p0 + rank] = k;
      }
      runs_keys = out;
      runs_p0 = p0;
    }
    __syncwarp();  // sorted keys visible to the whole warp
    const int32_t C = method_class[x];
    int32_t self = 0;
    const int32_t n = segment_runs(runs_keys, runs_p0, len, shift, C, lane,
                                   [&](int32_t E, int32_t n0, int32_t n1, int32_t) {
                                     if (E == C) self = n0 + (cbo_attrs ? n1 : 0);
                                   });
    for (int o = 16; o > 0; o >>= 1) self += __shfl_xor_sync(0xffffffffu, self, o);
    if (lane == 0) {
      len_out[x] = n;
      self_out[x] = self;
    }
  }
}

// Fill pass for list L: {E, out, -, t} at l_off[x] + run index, l_x = x; the
// multiplicities cnt(C, E) follow in lists_lookup_l (one thread per entry, so
// the row searches of all entries are in flight together).  A block takes 256
// consecutive methods: their sorted keys are one contiguous range, loaded into
// shared memory when it fits, and each thread walks its own method's runs.
__global__ void __launch_bounds__(256) lists_fill_l(const int64_t *call_rowptr, const int64_t *acc_rowptr, int32_t M,
                                                    const uint32_t *sorted, const int32_t *method_class,
                                                    int32_t cbo_attrs, const int64_t *l_off, int4 *l_list,
                                                    int32_t *l_x) {
  pdl_wait();
  __shared__ uint32_t sk[SB_KEYS];
  const int64_t x0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t xl = (x0 + (int64_t)blockDim.x < (int64_t)M ? x0 + (int64_t)blockDim.x : (int64_t)M) - 1;
  int64_t q0, l0, ql, ll;
  segment(call_rowptr, acc_rowptr, x0, &q0, &l0);
  segment(call_rowptr, acc_rowptr, xl, &ql, &ll);
  const int64_t nk = ql + ll - q0;
  const bool fits = nk <= SB_KEYS;
  if (fits)
    for (int64_t k = threadIdx.x; k < nk; k += blockDim.x) sk[k] = sorted[q0 + k];
  __syncthreads();
  const int64_t x = x0 + threadIdx.x;
  if (x >= M) return;
  int64_t p0, len;
  segment(call_rowptr, acc_rowptr, x, &p0, &len);
  const uint32_t *v = fits ? sk + (p0 - q0) : sorted + p0;
  const int32_t C = method_class[x];
  int64_t o = l_off[x];
  for (int32_t i = 0; i < (int32_t)len;) {
    const int32_t E = (int32_t)(v[i] >> 1);
    int32_t n0 = 0, n1 = 0;
    for (; i < (int32_t)len && (int32_t)(v[i] >> 1) == E; ++i) ((v[i] & 1u) ? n1 : n0)++;
    if (E == C) continue;
    l_list[o] = make_int4(E, n0 + (cbo_attrs ? n1 : 0), 0, n1);
    l_x[o] = (int32_t)x;
    ++o;
  }
}

// cnt(C, E) of every L entry with a use edge (C = class of its method)
// Multigraph look-ups of the list entries: a binary search in the row, or
// (packed coupling form) the row position read off the packed words.
struct MgLookup {
  const int64_t *rowptr;
  const int32_t *dst, *cnt;
  const uint2 *csum;       // packed form (else nullptr)
  const uint32_t *cpk;
  const int32_t *wrank;
  int64_t sw;
  __device__ __forceinline__ int32_t operator()(int32_t Y, int32_t E) const {
    return csum ? mg_lookup_packed(csum, cpk, wrank, sw, rowptr, cnt, Y, E) : mg_lookup(rowptr, dst, cnt, Y, E);
  }
};

__global__ void lists_lookup_l(const int64_t *n_l, const int32_t *l_x, const int32_t *method_class, MgLookup mg,
                               int4 *l_list) {
  pdl_wait();
  const int64_t nl = *n_l;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = l_list[l];
    if (v.y > 0) l_list[l].z = mg(method_class[l_x[l]], v.x);
  }
}

// Fill pass for list R: {X, in, -, C} at r_off[x] + run index (C, the callee's
// class, is replaced by cnt(X, C) in lists_lookup_r); blocks as for list L.
__global__ void __launch_bounds__(256) lists_fill_r(const int64_t *rin_off, int32_t M, const uint32_t *sorted,
                                                    const int32_t *method_class, const int64_t *r_off,
                                                    int4 *r_list) {
  pdl_wait();
  __shared__ uint32_t sk[SB_KEYS];
  const int64_t x0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t xl = (x0 + (int64_t)blockDim.x < (int64_t)M ? x0 + (int64_t)blockDim.x : (int64_t)M) - 1;
  const int64_t q0 = rin_off[x0], nk = rin_off[xl + 1] - q0;
  const bool fits = nk <= SB_KEYS;
  if (fits)
    for (int64_t k = threadIdx.x; k < nk; k += blockDim.x) sk[k] = sorted[q0 + k];
  __syncthreads();
  const int64_t x = x0 + threadIdx.x;
  if (x >= M) return;
  const int64_t p0 = rin_off[x], len = rin_off[x + 1] - p0;
  const uint32_t *v = fits ? sk + (p0 - q0) : sorted + p0;
  const int32_t C = method_class[x];
  int64_t o = r_off[x];
  for (int64_t i = 0; i < len;) {
    const int32_t X = (int32_t)v[i];
    int32_t n0 = 0;
    for (; i < len && (int32_t)v[i] == X; ++i) ++n0;
    if (X == C) continue;
    r_list[o++] = make_int4(X, n0, 0, C);
  }
}

// cnt(X, C) of every R entry: {X, in, cnt(X, C), 0}
__global__ void lists_lookup_r(const int64_t *n_r, MgLookup mg, int4 *r_list) {
  pdl_wait();
  const int64_t nr = *n_r;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = r_list[r];
    r_list[r] = make_int4(v.x, v.y, mg(v.x, v.w), 0);
  }
}

__device__ __forceinline__ int sgn64(int64_t v) { return (v > 0) - (v < 0); }
__device__ __forceinline__ uint32_t enc_sign(int s) { return s < 0 ? 1u : (s > 0 ? 2u : 0u); }

__global__ void build_headers(const int32_t *method_class, const int32_t *cls_n, const int32_t *cls_a,
                              const int64_t *cls_P, const int64_t *cls_Q, const int64_t *cls_S, const int32_t *own,
                              const int32_t *q, const int64_t *l_off, const int32_t *l_len, const int64_t *r_off,
                              const int32_t *r_len, const int32_t *out_self, const int32_t *in_self,
                              const int4 *l_list, int32_t M, MoveHdr *hdr) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  int32_t C = method_class[x];
  int32_t ll = l_len[x], lo = ll ? (int32_t)l_off[x] : 0;
  int32_t rl = r_len[x], ro = rl ? (int32_t)r_off[x] : 0;
  int32_t l_all = 0;
  for (int32_t e = 0; e < ll; ++e) {
    int4 v = l_list[lo + e];
    if (v.y > 0 && v.z == v.y) ++l_all;  // C stops using E after the move
  }
  // source class after the move (independent of the destination)
  int64_t n = cls_n[C], a = cls_a[C], S = cls_S[C];
  int64_t diff = cls_P[C] - cls_Q[C];
  int64_t ck = diff > 0 ? diff : 0;
  int64_t diff2 = diff - (n - 1) + 2 * (int64_t)q[x];
  int64_t ck2 = diff2 > 0 ? diff2 : 0;
  int sck = sgn64(ck2 - ck);
  int shs;
  if (a == 0) shs = 0;
  else if (n == 1) shs = own[x] < a ? -1 : 0;    // after: empty class, LCOM_HS = 0
  else shs = sgn64((int64_t)own[x] * n - S);     // sign(S n' - S' n) with n' = n-1, S' = S - own
  MoveHdr h;
  h.w0 = make_int4(C, lo, ll, ro);
  h.w1 = make_int4(rl, out_self[x], in_self[x], l_all);
  h.w2 = make_int4((int)(enc_sign(sck) | (enc_sign(shs) << 2)), (int)(ck2 - ck), 0, 0);
  hdr[x] = h;
}

}  // namespace

// Scratch of the two list branches: list L in side_eval[1] (side stream 1),
// list R in side_eval[2] (side stream 2).  Both halves of the list build call
// this with the same sizes, so they see the same buffers.
namespace {
struct ListBufs {
  uint32_t *lkeys, *lsorted, *rkeys, *rsorted;
  int64_t *l_off, *rin_off, *r_off;
  int32_t *l_len, *out_self, *r_len, *in_self, *cursor;
  int32_t *lwork, *rwork;
};

ListBufs list_bufs(mm_system *s, cudaStream_t sl, cudaStream_t sr) {
  const int32_t M = s->M;
  const int64_t nu = s->n_call + s->n_acc, nc = s->n_call;
  // L part: keys, sorted keys (u32, nu); l_off (i64, M + 1); l_len, out_self (i32, M)
  // R part: keys, sorted keys (u32, nc); rin_off, r_off (i64, M + 1); r_len, in_self, cursor (i32, M)
  auto part_bytes = [&](int64_t nkeys, int n64, int n32) {
    return (sizeof(uint32_t) * 2 * (size_t)std::max<int64_t>(nkeys, 1) + 15) / 16 * 16 +
           sizeof(int64_t) * (size_t)n64 * ((size_t)M + 1) + sizeof(int32_t) * (size_t)n32 * (size_t)M + 64;
  };
  const size_t work = sizeof(int32_t) * ((size_t)M + 1);
  const size_t lb = part_bytes(nu, 1, 2) + work, rbytes = part_bytes(nc, 2, 3) + work;
  char *lbase = static_cast<char *>(s->side_eval[1].need(lb, sl));
  char *rbase = static_cast<char *>(s->side_eval[2].need(rbytes, sr));
  ListBufs b;
  b.lkeys = reinterpret_cast<uint32_t *>(lbase);
  b.lsorted = b.lkeys + std::max<int64_t>(nu, 1);
  b.l_off = reinterpret_cast<int64_t *>(lbase + (sizeof(uint32_t) * 2 * (size_t)std::max<int64_t>(nu, 1) + 15) / 16 * 16);
  b.l_len = reinterpret_cast<int32_t *>(b.l_off + (M + 1));
  b.out_self = b.l_len + M;
  b.lwork = b.out_self + M;  // [0]: count, then the methods whose segments the warp version sorts
  b.rkeys = reinterpret_cast<uint32_t *>(rbase);
  b.rsorted = b.rkeys + std::max<int64_t>(nc, 1);
  b.rin_off = reinterpret_cast<int64_t *>(rbase + (sizeof(uint32_t) * 2 * (size_t)std::max<int64_t>(nc, 1) + 15) / 16 * 16);
  b.r_off = b.rin_off + (M + 1);
  b.r_len = reinterpret_cast<int32_t *>(b.r_off + (M + 1));
  b.in_self = b.r_len + M;
  b.cursor = b.in_self + M;
  b.rwork = b.cursor + M;
  return b;
}
}  // namespace

// First half of the move lists; needs only the input CSR and the class
// structures, so it runs beside the metric branches.
void begin_move_lists(mm_system *s) {
  const int32_t M = s->M;
  s->side_pending[1] = s->side_pending[2] = s->stream;
  if (M == 0) return;
  const int64_t nu = s->n_call + s->n_acc, nc = s->n_call;
  // the warp sorts take only the segments the block sorts left: a few per system
  const unsigned gw = (unsigned)std::min<int64_t>(ceil_div((int64_t)M * 32, TPB), B300_SMS * 2);
  cudaStream_t sl = fork_side(s, 1), sr = fork_side(s, 2);
  s->side_pending[1] = sl;
  s->side_pending[2] = sr;
  const ListBufs b = list_bufs(s, sl, sr);
  // list L: per-method sort of the use keys, runs counted, scanned, written
  if (nu > 0) {
    pdl_launch(method_use_keys32, grid_for(M), TPB, 0, sl,
               s->method_class, s->call_rowptr, s->call_idx, s->acc_rowptr, s->acc_idx, s->attr_class, M, b.lkeys);
    MM_LAUNCH_CHECK();
  }
  MM_CUDA_TRY(cudaMemsetAsync(b.lwork, 0, sizeof(int32_t), sl));
  pdl_launch(segment_sort_count_block, grid_for(M), 256, 0, sl, s->call_rowptr, s->acc_rowptr, M, b.lkeys, b.lsorted, 1,
                                                        s->method_class, s->cbo_attrs, b.l_len, b.out_self, b.lwork);
  MM_LAUNCH_CHECK();
  pdl_launch(segment_sort_count, gw, TPB, 0, sl, s->call_rowptr, s->acc_rowptr, M, b.lkeys, b.lsorted, 1, s->method_class,
                                         s->cbo_attrs, b.l_len, b.out_self, static_cast<const int32_t *>(b.lwork));
  MM_LAUNCH_CHECK();
  scan_exclusive_i32to64(b.l_len, b.l_off, M, s->side_sort[1], sl, b.l_off + M);
  pdl_launch(lists_fill_l, grid_for(M), 256, 0, sl, s->call_rowptr, s->acc_rowptr, M, b.lsorted, s->method_class,
                                             s->cbo_attrs, b.l_off, s->l_list, s->l_x);
  MM_LAUNCH_CHECK();
  // list R: callers bucketed by callee (counting sort on fan-in), per-callee sort, runs
  scan_exclusive_i32to64(s->fan_in, b.rin_off, M, s->side_sort[2], sr, b.rin_off + M);
  if (nc > 0) {
    MM_CUDA_TRY(cudaMemsetAsync(b.cursor, 0, sizeof(int32_t) * (size_t)M, sr));
    pdl_launch(caller_classes_scatter, grid_for(M), TPB, 0, sr, s->method_class, s->call_rowptr, s->call_idx, M, b.rin_off,
                                                        b.cursor, b.rkeys);
    MM_LAUNCH_CHECK();
  }
  MM_CUDA_TRY(cudaMemsetAsync(b.rwork, 0, sizeof(int32_t), sr));
  pdl_launch(segment_sort_count_block, grid_for(M), 256, 0, sr, b.rin_off, nullptr, M, b.rkeys, b.rsorted, 0,
                                                        s->method_class, s->cbo_attrs, b.r_len, b.in_self, b.rwork);
  MM_LAUNCH_CHECK();
  pdl_launch(segment_sort_count, gw, TPB, 0, sr, b.rin_off, nullptr, M, b.rkeys, b.rsorted, 0, s->method_class,
                                         s->cbo_attrs, b.r_len, b.in_self, static_cast<const int32_t *>(b.rwork));
  MM_LAUNCH_CHECK();
  scan_exclusive_i32to64(b.r_len, b.r_off, M, s->side_sort[2], sr, b.r_off + M);
  if (nc > 0) {
    pdl_launch(lists_fill_r, grid_for(M), 256, 0, sr, b.rin_off, M, b.rsorted, s->method_class, b.r_off, s->r_list);
    MM_LAUNCH_CHECK();
  }
}

static MgLookup mg_lookups(const mm_system *s) {
  MgLookup m;
  m.rowptr = s->mg_rowptr;
  m.dst = s->mg_dst;
  m.cnt = s->mg_cnt;
  const bool packed = s->packed_coupling && s->wrank;
  m.csum = packed ? s->csum : nullptr;
  m.cpk = s->cpk;
  m.wrank = s->wrank;
  m.sw = s->sum_words;
  return m;
}

// Second half: multigraph counts of every entry (after the coupling branch),
// s per L entry (after the own-access lists), then the per-method headers.
void build_move_precompute(mm_system *s) {
  cudaStream_t st = s->stream;
  const int32_t M = s->M;
  if (M == 0) return;
  const int64_t nu = s->n_call + s->n_acc, nc = s->n_call;
  cudaStream_t sl = s->side_pending[1], sr = s->side_pending[2];
  const ListBufs b = list_bufs(s, sl, sr);
  wait_point(s, 0, st, sl);
  if (nu > 0) {
    pdl_launch(lists_lookup_l, (unsigned)std::min<int64_t>(ceil_div(nu, TPB), B300_SMS * 16), TPB, 0, sl,
               static_cast<const int64_t *>(b.l_off + M), static_cast<const int32_t *>(s->l_x),
               static_cast<const int32_t *>(s->method_class), mg_lookups(s), s->l_list);
    MM_LAUNCH_CHECK();
    wait_point(s, 1, s->side_pending[0], sl);
    const UnionBitmap ub = union_bitmap(s, ceil_div(nu, 32), s->side_union[1], sl);
    pdl_launch(l_entries_s, ub.grid, 256, ub.smem, sl, s->l_list, s->l_x, b.l_off + M, s->acc_rowptr, s->acc_idx,
                                                s->attr_class, s->own_ptr, s->own_list, ub.words, ub.gbm, s->l_s);
    MM_LAUNCH_CHECK();
  }
  wait_point(s, 0, st, sr);
  if (nc > 0) {
    pdl_launch(lists_lookup_r, (unsigned)std::min<int64_t>(ceil_div(nc, TPB), B300_SMS * 16), TPB, 0, sr,
               static_cast<const int64_t *>(b.r_off + M), mg_lookups(s), s->r_list);
    MM_LAUNCH_CHECK();
  }
  join_side(s, 1, sl);
  join_side(s, 2, sr);
  pdl_launch(build_headers, grid_for(M), TPB, 0, st, s->method_class, s->cls_n, s->cls_a, s->cls_P, s->cls_Q, s->cls_S,
                                             s->own, s->q, b.l_off, b.l_len, b.r_off, b.r_len, b.out_self, b.in_self,
                                             s->l_list, M, s->hdr);
  MM_LAUNCH_CHECK();
}

// ======================================================================
// evaluation

namespace {

struct DState {
  int32_t D, nD, aD;
  int64_t diffD, SD, ckD;
  // target-side LCOM outcome when m shares nothing with D (t = s = 0), the common case
  int32_t sck0, shs0, dck0;
};

__device__ __forceinline__ DState load_dstate(int32_t D, const int32_t *cls_n, const int32_t *cls_a,
                                              const int64_t *cls_P, const int64_t *cls_Q, const int64_t *cls_S) {
  DState d;
  d.D = D;
  d.nD = cls_n[D];
  d.aD = cls_a[D];
  d.diffD = cls_P[D] - cls_Q[D];
  d.SD = cls_S[D];
  d.ckD = d.diffD > 0 ? d.diffD : 0;
  int64_t diff2 = d.diffD + d.nD;
  int64_t ck2 = diff2 > 0 ? diff2 : 0;
  d.sck0 = sgn64(ck2 - d.ckD);
  d.dck0 = (int32_t)(ck2 - d.ckD);
  d.shs0 = d.aD == 0 ? 0 : (d.nD == 0 ? 1 : (d.SD > 0 ? 1 : 0));
  return d;
}

// destination constants: {P - Q, S} and {n, a, dck0, sck0 | shs0 << 8}
__device__ __forceinline__ DState dstate_rec(const int4 *rec, int32_t D) {
  const int4 a = __ldg(rec + 2 * (int64_t)D), b = __ldg(rec + 2 * (int64_t)D + 1);
  DState d;
  d.D = D;
  d.nD = b.x;
  d.aD = b.y;
  d.dck0 = b.z;
  d.sck0 = (int32_t)(int8_t)(b.w & 0xff);
  d.shs0 = (int32_t)(int8_t)((b.w >> 8) & 0xff);
  d.diffD = (int64_t)(((uint64_t)(uint32_t)a.y << 32) | (uint32_t)a.x);
  d.SD = (int64_t)(((uint64_t)(uint32_t)a.w << 32) | (uint32_t)a.z);
  d.ckD = d.diffD > 0 ? d.diffD : 0;
  return d;
}

struct EvalCtx {
  const MoveHdr *hdr;
  const int4 *l_list;
  const int32_t *l_s;
  const int4 *r_list;
  const uint32_t *in_adj, *out_adj;  // full bitsets (dense evaluation)
  int64_t aw;
  const uint2 *csum;                 // compressed rows (candidate lists): out-rows, then in-rows
  const uint32_t *cpk;
  int64_t sw;
  int32_t c;
  int32_t packed;                    // general-path probes read the compressed rows, not the bitsets
  uint32_t mask;
  int32_t min_improved;
};

// bit col of compressed row r: its summary record, then the packed word if marked
__device__ __forceinline__ int packed_bit(const EvalCtx &cx, int64_t r, int32_t col) {
  const uint2 rec = __ldg(cx.csum + r * cx.sw + (col >> 10));
  const uint32_t b = ((uint32_t)col >> 5) & 31u;
  if (!((rec.x >> b) & 1u)) return 0;
  return (int)((__ldg(cx.cpk + rec.y + __popc(rec.x & ((1u << b) - 1u))) >> (col & 31)) & 1u);
}
// does class D use class E (in-row of E at D)
__device__ __forceinline__ int uses_in(const EvalCtx &cx, int32_t E, int32_t D) {
  if (cx.packed) return packed_bit(cx, (int64_t)cx.c + E, D);
  return (int)((__ldg(cx.in_adj + (int64_t)E * cx.aw + ((uint32_t)D >> 5)) >> ((uint32_t)D & 31u)) & 1u);
}
// does class X use class D (out-row of X at D)
__device__ __forceinline__ int uses_out(const EvalCtx &cx, int32_t X, int32_t D) {
  if (cx.packed) return packed_bit(cx, X, D);
  return (int)((__ldg(cx.out_adj + (int64_t)X * cx.aw + ((uint32_t)D >> 5)) >> ((uint32_t)D & 31u)) & 1u);
}

__device__ __forceinline__ int dec_sign(uint32_t e) { return e == 1u ? -1 : (e == 2u ? 1 : 0); }
__device__ __forceinline__ uint32_t sat_u16(int32_t v) { return v < 0 ? 0u : (v > 65535 ? 65535u : (uint32_t)v); }
__device__ __forceinline__ uint32_t sat_i16(int32_t v) {
  int32_t w = v < -32768 ? -32768 : (v > 32767 ? 32767 : v);
  return (uint32_t)(uint16_t)(int16_t)w;
}

// Everything gathered for one candidate (m -> D) from m's lists and the adjacency bitsets.
struct Gathered {
  int32_t gain;          // classes E used by m (E != C, D) that D does not use yet
  int32_t impX, worX;    // caller classes X != C, D whose CBO drops / rises
  int32_t t, sh;         // m's accesses to D's attributes, methods of D sharing one
  int32_t outD, cntCD;   // m's use edges into D, C's use edges into D (when outD > 0)
  int32_t inD, cntDC;    // m's callers in D, D's use edges into C (when inD > 0)
  int32_t bDC, bCD;      // D uses C / C uses D, before the move (bit probes)
};

// Record of one candidate from the gathered data (shared by every kernel).
__device__ __forceinline__ uint4 finish_move(const MoveHdr &h, const DState &ds, const Gathered &g, uint32_t mk,
                                             int32_t min_improved, int32_t &dck_sum, int32_t &dcbo_sum) {
  const int32_t out_self = h.w1.y, in_self = h.w1.z, l_all = h.w1.w;
  // row D, column C
  int bDC = g.bDC, aDC;
  if (g.inD > 0) {
    bDC = 1;
    aDC = (g.cntDC + out_self - g.inD) > 0;
  } else {
    aDC = bDC | (out_self > 0);
  }
  const int32_t dD = g.gain + aDC - bDC;
  // row C, column D
  int bCD = g.bCD, aCD, corr = 0;
  if (g.outD > 0) {
    bCD = 1;
    aCD = (g.cntCD - g.outD + in_self) > 0;
    corr = g.cntCD == g.outD;
  } else {
    aCD = bCD | (in_self > 0);
  }
  const int32_t dC = -l_all + corr + aCD - bCD;
  // target LCOM
  int sckD, shsD;
  int32_t dckD;
  if (g.t == 0 && g.sh == 0) {
    sckD = ds.sck0;
    shsD = ds.shs0;
    dckD = ds.dck0;
  } else {
    int64_t diff2 = ds.diffD + ds.nD - 2 * (int64_t)g.sh;
    int64_t ck2 = diff2 > 0 ? diff2 : 0;
    sckD = sgn64(ck2 - ds.ckD);
    dckD = (int32_t)(ck2 - ds.ckD);
    if (ds.aD == 0) shsD = 0;
    else if (ds.nD == 0) shsD = g.t < ds.aD ? 1 : 0;
    else shsD = sgn64(ds.SD - (int64_t)g.t * ds.nD);  // sign(S n' - S' n) with n' = n+1, S' = S + t
  }
  const int sckC = dec_sign((uint32_t)h.w2.x & 3u), shsC = dec_sign(((uint32_t)h.w2.x >> 2) & 3u);
  const int scbC = (dC > 0) - (dC < 0), scbD = (dD > 0) - (dD < 0);
  const int upC = ((mk & 1u) && sckC > 0) | ((mk & 2u) && shsC > 0) | ((mk & 4u) && scbC > 0);
  const int dnC = ((mk & 1u) && sckC < 0) | ((mk & 2u) && shsC < 0) | ((mk & 4u) && scbC < 0);
  const int upD = ((mk & 1u) && sckD > 0) | ((mk & 2u) && shsD > 0) | ((mk & 4u) && scbD > 0);
  const int dnD = ((mk & 1u) && sckD < 0) | ((mk & 2u) && shsD < 0) | ((mk & 4u) && scbD < 0);
  int32_t imp = (!upC && dnC) + (!upD && dnD);
  int32_t wor = upC + upD;
  if (mk & 4u) {
    imp += g.impX;
    wor += g.worX;
  }
  uint32_t flags = ((uint32_t)h.w2.x & 15u) | (enc_sign(scbC) << 4) | (enc_sign(sckD) << 6) |
                   (enc_sign(shsD) << 8) | (enc_sign(scbD) << 10);
  if (wor == 0 && imp >= min_improved) flags |= 0x8000u;
  dck_sum = h.w2.y + dckD;
  dcbo_sum = dC + dD;
  uint4 r;
  r.x = (uint32_t)g.sh;
  r.y = sat_u16(g.t) | (sat_i16(dC) << 16);
  r.z = sat_i16(dD) | (sat_u16(imp) << 16);
  r.w = sat_u16(wor) | (flags << 16);
  return r;
}

// Gather for (m -> D) straight from global memory (explicit candidate lists,
// and methods whose lists do not fit the shared-memory stage).
__device__ __forceinline__ uint4 eval_move(const EvalCtx &cx, const MoveHdr &h, const DState &ds, int32_t &dck_sum,
                                           int32_t &dcbo_sum) {
  const int32_t D = ds.D;
  const int32_t C = h.w0.x;
  Gathered g;
  g.gain = 0; g.impX = 0; g.worX = 0; g.t = 0; g.sh = 0; g.outD = 0; g.cntCD = 0; g.inD = 0; g.cntDC = 0;
  const int4 *L = cx.l_list + h.w0.y;
  for (int32_t e = 0; e < h.w0.z; ++e) {
    int4 v = __ldg(L + e);
    if (v.x == D) {
      g.outD = v.y;
      g.cntCD = v.z;
      g.t = v.w;
      g.sh = v.w > 0 ? __ldg(cx.l_s + h.w0.y + e) : 0;
    } else if (v.y > 0) {
      g.gain += 1 - uses_in(cx, v.x, D);
    }
  }
  const int4 *R = cx.r_list + h.w0.w;
  for (int32_t e = 0; e < h.w1.x; ++e) {
    int4 v = __ldg(R + e);
    if (v.x == D) {
      g.inD = v.y;
      g.cntDC = v.z;
    } else {
      int loss = v.z == v.y;
      int gx = 1 - uses_out(cx, v.x, D);
      int dx = gx - loss;
      g.impX += dx < 0;
      g.worX += dx > 0;
    }
  }
  g.bDC = uses_in(cx, C, D);
  g.bCD = uses_out(cx, C, D);
  return finish_move(h, ds, g, cx.mask, cx.min_improved, dck_sum, dcbo_sum);
}

__device__ __forceinline__ uint64_t smix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t record_hash(int32_t m, int32_t D, uint4 r) {
  uint64_t lo = (uint64_t)r.x | ((uint64_t)r.y << 32);
  uint64_t hi = (uint64_t)r.z | ((uint64_t)r.w << 32);
  uint64_t key = ((uint64_t)(uint32_t)m << 32) | (uint32_t)D;
  return smix(key ^ smix(lo ^ smix(hi)));
}

struct OutCtx {
  uint4 *records;                 // nullable
  unsigned long long *digest;     // nullable (device accumulator)
  mm_move *kept;                  // nullable
  unsigned long long *kept_count;
  int64_t kept_cap;
  uint8_t *kept_mark;             // per method
};

__device__ __forceinline__ void emit_kept(const OutCtx &oc, bool kept, int32_t m, int32_t D, uint32_t nimp,
                                          int32_t dck, int32_t dcbo, uint32_t lane) {
  uint32_t bal = __ballot_sync(0xffffffffu, kept);
  if (bal == 0) return;
  unsigned long long base = 0;
  int leader = __ffs(bal) - 1;
  if ((int)lane == leader) base = atomicAdd(oc.kept_count, (unsigned long long)__popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (kept) {
    unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
    if ((int64_t)pos < oc.kept_cap) {
      mm_move mv;
      mv.m = m;
      mv.d = D;
      mv.n_improved = (int32_t)nimp;
      mv.d_lcom_ck_sum = dck;
      mv.d_cbo_sum = dcbo;
      mv.reserved = 0;
      oc.kept[pos] = mv;
    }
    oc.kept_mark[m] = 1;
  }
}

// Dense cross product.  A block owns DB_SPAN = 1024 consecutive destinations;
// thread (warp w, lane l) evaluates D = D0 + 32 w + l + 256 q for q = 0..3, so
// each warp-wide store writes 32 consecutive 16-byte records (512 bytes).
// Methods are walked in batches.  For each batch the block first stages in
// shared memory, cooperatively and with many loads in flight: the headers, the
// list entries and, for every entry, the 32 adjacency words covering the
// block's destinations, already turned into per-destination contributions:
//   L entry E (m uses E):   bit D = 1 iff D does not use E yet (CBO(D) gains E),
//                           0 where D == E or m has no use edge into E;
//   R entry X (X calls m):  bit D = 1 iff CBO(X) drops (X stops using C and
//                           already uses D) or rises (X keeps C, starts using D);
//                           which of the two is the entry's uniform "shift".
// The evaluation then takes a thread's four destinations at once, one byte
// lane each: byte permutes gather the thread's bit of an entry's four words,
// and the counts, the outcome and the record words are packed byte arithmetic
// over per-method and per-destination constants.  A destination that appears
// in m's own lists (D == E or D == X) takes the exact general path, one per
// thread after the batch.
constexpr int DQ = 4;
constexpr int DB_THREADS = 256;
constexpr int DB_WARPS = DB_THREADS / 32;
constexpr int DB_SPAN = DB_THREADS * DQ;
constexpr int DB_MB = 32;
constexpr int DB_ECAP = 192;

static_assert(DB_SPAN == 1024 && DB_MB <= 32, "hit codes (method << 10 | rel) fit 16 bits");

struct DenseStage {
  MoveHdr hdr[DB_MB];
  int32_t lb[DB_MB], rb[DB_MB], hb[DB_MB], hn[DB_MB];
  int4 ent[DB_ECAP];              // L: {E, out, cnt(C,E), t}; R: {X, in, cnt(X,C), shift 0|16}
  int32_t ents[DB_ECAP];          // s of L entries
  uint4 word[DB_ECAP][DB_WARPS];  // [slot][w] = contribution words w, w+8, w+16, w+24
  uint4 cw[DB_MB][2][DB_WARPS];   // adjacency words of row C: [0] = in_adj (D uses C), [1] = out_adj (C uses D)
  int16_t hit[DB_ECAP];           // slots whose class lies in the block's span
  int16_t hl[DB_ECAP];            // distinct listed destinations of the batch: method << 10 | rel
  int8_t sm[DB_ECAP];             // method of each slot
  uint8_t sk[DB_ECAP];            // row of each slot: 1 in-row (else out-row), 2 inverted, 4 counted
  int32_t nhl, ns;
  uint4 hitw[DB_MB][DB_WARPS];    // per method: bit rel set iff D0 + rel is in one of its lists;
                                  // word g = w + 8 q is stored at [w] component q (as word)
  // per method, for b = [m's callers in C make C start using D] (bytes replicated over the four
  // destinations of a thread, plus their change from b = 0 to b = 1):
  //   [0] = {improved of C, worsened of C, change, change},
  //   [1] = {flag bits 0-5 (C's signs), change, record word 1 (dCBO(C) << 16), change},
  //   [2] = {C, 0x01010101 if m uses members of C, 0x01010101 if methods of C call m, 0}
  int4 mc[DB_MB][3];
  int32_t mid[DB_MB];             // method id of each of the batch's methods
  int32_t k, overflow;
};

// Bit `lane` of each word of v as one byte (0 or 1) per word; gsel picks the
// byte of a word that holds the bit, gsh its position there.
__device__ __forceinline__ uint32_t lane_bits4(const uint4 &v, uint32_t gsel, uint32_t gsh) {
  const uint32_t lo = __byte_perm(v.x, v.y, gsel), hi = __byte_perm(v.z, v.w, gsel);
  return (__byte_perm(lo, hi, 0x5410) >> gsh) & 0x01010101u;
}
// 1 in each byte of x that is not zero.
__device__ __forceinline__ uint32_t bytes_nonzero(uint32_t x) {
  return ((((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) >> 7) & 0x01010101u;
}
// 1 in each byte of x that is >= t, given k9 = (256 - t) * 0x00010001 for t in [0, 256]:
// each byte plus 256 - t, in a 16-bit lane, carries into bit 8 exactly when byte >= t.
__device__ __forceinline__ uint32_t bytes_ge(uint32_t x, uint32_t k9) {
  const uint32_t ev = (x & 0x00ff00ffu) + k9, od = ((x >> 8) & 0x00ff00ffu) + k9;
  return ((ev >> 8) & 0x00010001u) | (od & 0x01000100u);
}

__device__ __forceinline__ uint32_t sel4(const uint4 &v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

__device__ __forceinline__ int32_t clamp16(int32_t v) { return max(-32768, min(32767, v)); }
__device__ __forceinline__ uint32_t enc_small(int32_t v) { return (uint32_t)(v < 0) | ((uint32_t)(v > 0) << 1); }

// Word g of method j's hit bitmap (stored so that a warp's four words form one uint4).
__device__ __forceinline__ uint32_t *hit_word(DenseStage &st, int32_t j, int32_t g) {
  return reinterpret_cast<uint32_t *>(&st.hitw[j][0]) + ((g & 7) * 4 + (g >> 3));
}

// Rare paths of the dense kernel, kept out of line so they do not cost the
// common path registers.
__device__ __noinline__ uint4 dense_hit_path(const EvalCtx cx, const DenseStage &st, int32_t j, int32_t D, int q,
                                             uint32_t lane, int warp, const int4 *dest_rec, int32_t *dck,
                                             int32_t *dcbo) {
  const MoveHdr h = st.hdr[j];
  Gathered g;
  g.gain = 0; g.impX = 0; g.worX = 0;
  g.t = 0; g.sh = 0; g.outD = 0; g.cntCD = 0; g.inD = 0; g.cntDC = 0;
  const int32_t lb = st.lb[j], nl = h.w0.z, rb = st.rb[j], nr = h.w1.x;
  for (int32_t e = 0; e < nl; ++e) g.gain += (int32_t)((sel4(st.word[lb + e][warp], q) >> lane) & 1u);
  if (cx.mask & 4u)
    for (int32_t e = 0; e < nr; ++e) {
      const uint32_t bit = (sel4(st.word[rb + e][warp], q) >> lane) & 1u;
      if (st.ent[rb + e].w == 0) g.impX += (int32_t)bit;
      else g.worX += (int32_t)bit;
    }
  const int32_t hb = st.hb[j], hn = st.hn[j];
  for (int32_t i = 0; i < hn; ++i) {
    const int32_t slot = st.hit[hb + i];
    const int4 v = st.ent[slot];
    if (v.x != D) continue;
    if (slot < rb) {
      g.outD = v.y; g.cntCD = v.z; g.t = v.w; g.sh = st.ents[slot];
    } else {
      g.inD = v.y; g.cntDC = v.z;
    }
  }
  g.bDC = (int32_t)((sel4(st.cw[j][0][warp], q) >> lane) & 1u);
  g.bCD = (int32_t)((sel4(st.cw[j][1][warp], q) >> lane) & 1u);
  const DState ds = dstate_rec(dest_rec, D);
  int32_t a = 0, b = 0;
  uint4 r = finish_move(h, ds, g, cx.mask, cx.min_improved, a, b);
  *dck = a;
  *dcbo = b;
  return r;
}

// One method against the block's destinations from global memory (its lists
// do not fit the stage).  Its arguments are values: a reference to a kernel
// parameter would keep the whole parameter block in local memory.
template <bool REC, bool DIG, bool KEEP>
__device__ __noinline__ uint64_t dense_overflow_method(const EvalCtx cx, const OutCtx oc, const MoveHdr h, int32_t m,
                                                       int32_t D0, int32_t c, const int4 *dest_rec) {
  const uint32_t lane = threadIdx.x & 31u;
  const int32_t C = h.w0.x;
  const int64_t rowbase = (int64_t)m * ((int64_t)c - 1);
  uint64_t dig = 0;
  for (int q = 0; q < DQ; ++q) {
    const int32_t D = D0 + (int32_t)threadIdx.x + q * DB_THREADS;
    const bool act = D < c && D != C;
    int32_t dck = 0, dcbo = 0;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (act) r = eval_move(cx, h, dstate_rec(dest_rec, D), dck, dcbo);
    if (REC && act) __stcs(oc.records + rowbase + D - (D > C ? 1 : 0), r);
    if (DIG && act) dig += record_hash(m, D, r);
    if (KEEP) emit_kept(oc, act && (r.w >> 31), m, D, r.z >> 16, dck, dcbo, lane);
  }
  return dig;
}

// Parameters of one system for the dense evaluation (also the unit of the
// batched persistent kernel).
struct DenseSys {
  EvalCtx cx;
  const int4 *dest_rec;  // per class: {P - Q, S}, {n, a, dck0, sck0 | shs0 << 8}
  int32_t c, M;          // M: methods evaluated (the length of mlist when it is set)
  const int32_t *mlist;   // when non-null, position i evaluates method mlist[i] (else method i)
};

// One tile of the dense cross product: destinations [bx*DB_SPAN, +DB_SPAN) x
// methods [m0, m1).  Called by every thread of a block; returns this thread's
// digest partial.
template <bool REC, bool DIG, bool KEEP>
__device__ __forceinline__ uint64_t dense_tile(const DenseSys &sy, const OutCtx &oc, DenseStage &st, int32_t bx,
                                               int32_t m0, int32_t m1) {
  const EvalCtx &cx = sy.cx;
  const int4 *dest_rec = sy.dest_rec;
  const int32_t c = sy.c;
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = (int)(threadIdx.x >> 5);
  const int32_t D0 = bx * DB_SPAN;
  const int64_t dw0 = D0 >> 5;
  const uint32_t mk = cx.mask;
  const int32_t mk4 = (mk & 4u) ? 1 : 0;
  // destination constants of the common path (m shares nothing with D), one
  // byte per destination q of this thread: improved / worsened counts of D for
  // p = [dCBO(D) > 0] = 0 (pdi, pdw) and their change when p = 1 (-negi, +posw;
  // only CBO moves with p), D's sign bits of the flags (bits 6-7 in fdlo, 8-9 in
  // fdhi) and whether D exists
  uint32_t pdi = 0u, pdw = 0u, negi = 0u, posw = 0u, fdlo = 0u, fdhi = 0u, valid = 0u;
#pragma unroll
  for (int q = 0; q < DQ; ++q) {
    const int32_t D = D0 + (int32_t)threadIdx.x + q * DB_THREADS;
    // sign bytes of dLCOM_CK and dLCOM_HS when D gains a method sharing nothing
    const uint32_t sg = (uint32_t)__ldg(&dest_rec[2 * (int64_t)(D < c ? D : 0) + 1].w);
    const int32_t sck0 = (int32_t)(int8_t)(sg & 0xffu), shs0 = (int32_t)(int8_t)((sg >> 8) & 0xffu);
    const uint32_t up = ((mk & 1u) && sck0 > 0) | ((mk & 2u) && shs0 > 0);
    const uint32_t dn = ((mk & 1u) && sck0 < 0) | ((mk & 2u) && shs0 < 0);
    const uint32_t sh = 8u * (uint32_t)q;
    pdi |= (dn & (up ^ 1u)) << sh;
    pdw |= up << sh;
    negi |= (dn & (up ^ 1u) & (uint32_t)mk4) << sh;
    posw |= ((up ^ 1u) & (uint32_t)mk4) << sh;
    fdlo |= (enc_sign(sck0) << 6) << sh;
    fdhi |= enc_sign(shs0) << sh;
    valid |= (uint32_t)(D < c) << sh;
  }
  const uint32_t gsel = (lane >> 3) | (((lane >> 3) + 4u) << 4), gsh = lane & 7u;
  const int32_t mi = min(max(cx.min_improved, 0), 256);
  const uint32_t k9 = (uint32_t)(256 - mi) * 0x00010001u;
  const int64_t row = (int64_t)c - 1;
  const int64_t seg_words = cx.aw - dw0;  // adjacency words left in a row from dw0 (may exceed 32)
  uint64_t dig = 0;
  for (int32_t mb = m0; mb < m1;) {
    for (int32_t i = (int32_t)threadIdx.x; i < DB_MB * DB_WARPS * 4; i += DB_THREADS)
      reinterpret_cast<uint32_t *>(&st.hitw[0][0])[i] = 0u;
    // ---- plan: warp 0 scans the list lengths of up to 32 methods
    if (warp == 0) {
      const int32_t pos = mb + (int32_t)lane;
      const bool ok = pos < m1;
      const int32_t m = ok ? (sy.mlist ? __ldg(sy.mlist + pos) : pos) : 0;
      MoveHdr h;
      h.w0 = make_int4(0, 0, 0, 0);
      h.w1 = make_int4(0, 0, 0, 0);
      h.w2 = make_int4(0, 0, 0, 0);
      if (ok) {
        h.w0 = __ldg(&cx.hdr[m].w0);
        h.w1 = __ldg(&cx.hdr[m].w1);
        h.w2 = __ldg(&cx.hdr[m].w2);
      }
      const int32_t len = ok ? h.w0.z + h.w1.x : 0;
      int32_t incl = len;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const uint32_t fit = __ballot_sync(0xffffffffu, ok && incl <= DB_ECAP);
      int32_t k = __popc(fit);
      int32_t overflow = 0;
      if (k == 0) { k = 1; overflow = 1; }
      if ((int32_t)lane < k) {
        st.hdr[lane] = h;
        st.mid[lane] = m;
        st.lb[lane] = incl - len;
        st.rb[lane] = incl - len + h.w0.z;
        st.hb[lane] = incl - len;  // the method's listed slots are kept from its first slot on
        st.hn[lane] = 0;
        for (int32_t e = incl - len; e < incl; ++e) st.sm[e] = (int8_t)lane;
        const uint32_t sC = (uint32_t)h.w2.x & 15u;
        const int sckC = dec_sign(sC & 3u), shsC = dec_sign(sC >> 2);
        const int32_t upCl = ((mk & 1u) && sckC > 0) | ((mk & 2u) && shsC > 0);
        const int32_t dnCl = ((mk & 1u) && sckC < 0) | ((mk & 2u) && shsC < 0);
        int32_t pci[2], pcw[2], fcb[2], rcb[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int32_t dC = b - h.w1.w;  // -l_all, plus one when C starts using D
          const int32_t upC = upCl | (mk4 & (dC > 0)), dnC = dnCl | (mk4 & (dC < 0));
          pci[b] = dnC & (upC ^ 1);
          pcw[b] = upC;
          fcb[b] = (int32_t)(sC | (enc_small(dC) << 4));
          rcb[b] = (int32_t)((uint32_t)(uint16_t)(int16_t)clamp16(dC) << 16);
        }
        st.mc[lane][0] = make_int4((int32_t)((uint32_t)pci[0] * 0x01010101u), (int32_t)((uint32_t)pcw[0] * 0x01010101u),
                                   pci[1] - pci[0], pcw[1] - pcw[0]);
        st.mc[lane][1] = make_int4((int32_t)((uint32_t)fcb[0] * 0x01010101u), fcb[1] - fcb[0], rcb[0],
                                   (int32_t)((uint32_t)rcb[1] - (uint32_t)rcb[0]));
        st.mc[lane][2] = make_int4(h.w0.x, h.w1.y > 0 ? 0x01010101 : 0, h.w1.z > 0 ? 0x01010101 : 0, 0);
      }
      const int32_t ns = __shfl_sync(0xffffffffu, incl, k - 1);
      if (lane == 0) { st.k = k; st.overflow = overflow; st.nhl = 0; st.ns = overflow ? 0 : ns; }
    }
    __syncthreads();
    const int32_t k = st.k;
    const bool overflow = st.overflow != 0;
    // ---- stage, block-wide: (1) every slot's list entry and the adjacency
    // words of each method's own class C, (2) every slot's 32 row words
    // turned into per-destination contributions
    if (!overflow) {
      const int32_t ns = st.ns;
      for (int32_t slot = (int32_t)threadIdx.x; slot < ns; slot += DB_THREADS) {
        const int32_t j = st.sm[slot];
        const int4 w0 = st.hdr[j].w0;
        const int32_t rb = st.rb[j], lb = st.lb[j];
        const bool isL = slot < rb;
        int4 v;
        uint32_t kind;
        if (isL) {
          v = __ldg(cx.l_list + w0.y + (slot - lb));
          const int32_t sv = __ldg(cx.l_s + w0.y + (slot - lb));
          st.ents[slot] = v.w > 0 ? sv : 0;
          kind = 1u | 2u | (v.y > 0 ? 4u : 0u);  // in-row, inverted: D does not use E yet; only if m uses E
        } else {
          v = __ldg(cx.r_list + w0.w + (slot - rb));
          const bool loss = v.z == v.y;            // X stops using C
          v.w = loss ? 0 : 16;                     // drop -> improved counter, rise -> worsened counter
          kind = (loss ? 0u : 2u) | 4u;            // out-row: loss ? X uses D : X does not use D
        }
        st.ent[slot] = v;
        st.sk[slot] = (uint8_t)kind;
        const int32_t rel = v.x - D0;
        if (rel >= 0 && rel < DB_SPAN) {  // listed destination in this block's span
          st.hit[lb + atomicAdd(&st.hn[j], 1)] = (int16_t)slot;
          const uint32_t hbit = 1u << (rel & 31);
          if (!(atomicOr(hit_word(st, j, rel >> 5), hbit) & hbit))  // first entry of this class
            st.hl[atomicAdd(&st.nhl, 1)] = (int16_t)((j << 10) | rel);
        }
      }
      for (int32_t ci = (int32_t)threadIdx.x; ci < k * 2 * DB_WARPS; ci += DB_THREADS) {
        const int32_t j = ci / (2 * DB_WARPS), which = (ci / DB_WARPS) & 1, w = ci % DB_WARPS;
        const uint32_t *rowp = (which ? cx.out_adj : cx.in_adj) + (int64_t)st.hdr[j].w0.x * cx.aw + dw0;
        uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (w < seg_words) a0 = __ldg(rowp + w);
        if (w + 8 < seg_words) a1 = __ldg(rowp + w + 8);
        if (w + 16 < seg_words) a2 = __ldg(rowp + w + 16);
        if (w + 24 < seg_words) a3 = __ldg(rowp + w + 24);
        st.cw[j][which][w] = make_uint4(a0, a1, a2, a3);
      }
      __syncthreads();
      // four items per slot, each 8 of its 32 words: word g = 8 c4 + w is stored at [w][c4];
      // a thread issues the loads of all its items before storing any
      constexpr int SI = (4 * DB_ECAP + DB_THREADS - 1) / DB_THREADS;
      uint4 ra[SI], rb4[SI];
#pragma unroll
      for (int u = 0; u < SI; ++u) {
        const int32_t it = (int32_t)threadIdx.x + u * DB_THREADS;
        ra[u] = make_uint4(0, 0, 0, 0);
        rb4[u] = make_uint4(0, 0, 0, 0);
        if (it < 4 * ns) {
          const int32_t slot = it >> 2, c4 = it & 3;
          const uint4 *rowp = reinterpret_cast<const uint4 *>(((st.sk[slot] & 1u) ? cx.in_adj : cx.out_adj) +
                                                              (int64_t)st.ent[slot].x * cx.aw + dw0);
          if (8 * c4 < seg_words) ra[u] = __ldg(rowp + 2 * c4);
          if (8 * c4 + 4 < seg_words) rb4[u] = __ldg(rowp + 2 * c4 + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < SI; ++u) {
        const int32_t it = (int32_t)threadIdx.x + u * DB_THREADS;
        if (it < 4 * ns) {
          const int32_t slot = it >> 2, c4 = it & 3;
          const uint32_t kind = st.sk[slot];
          const uint32_t xr = (kind & 2u) ? 0xffffffffu : 0u, am = (kind & 4u) ? 0xffffffffu : 0u;
          const int32_t relv = st.ent[slot].x - D0;
          const int32_t hw = (relv >= 0 && relv < DB_SPAN) ? (relv >> 5) : -1;
          const uint32_t hbit = 1u << (relv & 31);
          const uint32_t wv[8] = {ra[u].x, ra[u].y, ra[u].z, ra[u].w, rb4[u].x, rb4[u].y, rb4[u].z, rb4[u].w};
          uint32_t *dstw = reinterpret_cast<uint32_t *>(&st.word[slot][0]);
#pragma unroll
          for (int w = 0; w < DB_WARPS; ++w) {
            uint32_t x = (wv[w] ^ xr) & am;
            if (hw == 8 * c4 + w) x &= ~hbit;  // D == E or D == X: the listed path counts it
            dstw[4 * w + c4] = x;
          }
        }
      }
    }
    __syncthreads();
    // ---- evaluate the batch (a method whose lists exceed the stage comes alone
    // and takes the general path, called outside the loop so that the loop
    // keeps no call frame)
    if (overflow) dig += dense_overflow_method<REC, DIG, KEEP>(cx, oc, st.hdr[0], st.mid[0], D0, c, dest_rec);
    for (int32_t j = 0; j < k && !overflow; ++j) {
      const int32_t m = st.mid[j];
      const MoveHdr h = st.hdr[j];
      const int32_t C = h.w0.x;
      const int64_t rowbase = (int64_t)m * row;
      // contribution counts of the thread's four destinations, one byte each
      uint32_t gain = 0u, iwl = 0u, iwk = 0u;
      {
        const int32_t lb = st.lb[j], nl = h.w0.z;
        for (int32_t e = 0; e < nl; ++e) gain += lane_bits4(st.word[lb + e][warp], gsel, gsh);
        if (mk4) {  // caller classes only matter when CBO is selected
          const int32_t rb = st.rb[j], nr = h.w1.x;
          for (int32_t e = 0; e < nr; ++e) {
            const uint32_t v = lane_bits4(st.word[rb + e][warp], gsel, gsh);
            if (st.ent[rb + e].w == 0) iwl += v;  // X stops using C: improved
            else iwk += v;                        // X keeps C: worsened
          }
        }
      }
      const int4 mc0 = st.mc[j][0], mc1 = st.mc[j][1], mc2 = st.mc[j][2];
      // hits: destinations of this thread that appear in m's lists (evaluated after the batch)
      const uint32_t hit = lane_bits4(st.hitw[j][warp], gsel, gsh);
      const uint32_t bdc = lane_bits4(st.cw[j][0][warp], gsel, gsh), bcd = lane_bits4(st.cw[j][1][warp], gsel, gsh);
      // common path: m shares nothing with D and D is in neither of m's lists
      const uint32_t dd = gain + (~bdc & (uint32_t)mc2.y);  // dCBO(D) >= 0
      const uint32_t bb = ~bcd & (uint32_t)mc2.z;           // C starts using D
      const uint32_t pb = bytes_nonzero(dd);                // dCBO(D) > 0
      const uint32_t imp = (uint32_t)mc0.x + pdi + bb * (uint32_t)mc0.z - (pb & negi) + iwl;
      const uint32_t wor = (uint32_t)mc0.y + pdw + bb * (uint32_t)mc0.w + (pb & posw) + iwk;
      const uint32_t kb = bytes_ge(imp, k9) & ~bytes_nonzero(wor);
      const uint32_t flo = (uint32_t)mc1.x + fdlo + bb * (uint32_t)mc1.y;  // flag bits 0-7
      const uint32_t fhi = fdhi + pb * 8u + kb * 128u;                     // flag bits 8-15
      const int32_t relC = C - D0;
      const bool cspan = relC >= 0 && relC < DB_SPAN;
      uint32_t act = valid & ~hit;
      if (cspan && (relC & (DB_THREADS - 1)) == (int32_t)threadIdx.x) act &= ~(1u << (8 * (relC / DB_THREADS)));
      // records: {sh = 0, t = 0 | dC << 16, dD | imp << 16, wor | flags << 16}
      const uint32_t dd01 = __byte_perm(dd, 0u, 0x4140), dd23 = __byte_perm(dd, 0u, 0x4342);
      const uint32_t im01 = __byte_perm(imp, 0u, 0x4140), im23 = __byte_perm(imp, 0u, 0x4342);
      const uint32_t wo01 = __byte_perm(wor, 0u, 0x4140), wo23 = __byte_perm(wor, 0u, 0x4342);
      const uint32_t fl01 = __byte_perm(flo, fhi, 0x5140), fl23 = __byte_perm(flo, fhi, 0x7362);
      const uint32_t rc0 = (uint32_t)mc1.z, drc = (uint32_t)mc1.w;
      auto rec = [&](int q) {
        const uint32_t lo = q < 2 ? dd01 : dd23, il = q < 2 ? im01 : im23, wl = q < 2 ? wo01 : wo23,
                       fl = q < 2 ? fl01 : fl23, sel = (q & 1) ? 0x7632u : 0x5410u;
        return make_uint4(0u, rc0 + ((bb >> (8 * q)) & 1u) * drc, __byte_perm(lo, il, sel), __byte_perm(wl, fl, sel));
      };
      uint4 *rp = oc.records + rowbase + D0 + (int32_t)threadIdx.x;
      if (!cspan) {
        if (relC < 0) rp -= 1;  // every destination of the span lies past C
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
          const bool a = (act >> (8 * q)) & 1u;
          const uint4 r = rec(q);
          if (REC && a) __stcs(rp + q * DB_THREADS, r);
          if (DIG && a) dig += record_hash(m, D0 + (int32_t)threadIdx.x + q * DB_THREADS, r);
        }
      } else {
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
          const int32_t D = D0 + (int32_t)threadIdx.x + q * DB_THREADS;
          const bool a = (act >> (8 * q)) & 1u;
          const uint4 r = rec(q);
          if (REC && a) __stcs(rp + q * DB_THREADS - (D > C ? 1 : 0), r);
          if (DIG && a) dig += record_hash(m, D, r);
        }
      }
      // kept moves are rare: one vote per method, the compaction only when a lane has one
      const uint32_t kact = kb & act;
      if (KEEP && __any_sync(0xffffffffu, kact != 0u)) {
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
          const int32_t D = D0 + (int32_t)threadIdx.x + q * DB_THREADS;
          const bool kk = (kact >> (8 * q)) & 1u;
          int32_t dck = 0, dcbo = 0;
          if (kk) {
            dck = h.w2.y + __ldg(&dest_rec[2 * (int64_t)D + 1].z);
            dcbo = (int32_t)((bb >> (8 * q)) & 1u) - h.w1.w + (int32_t)((dd >> (8 * q)) & 0xffu);
          }
          emit_kept(oc, kk, m, D, (imp >> (8 * q)) & 0xffu, dck, dcbo, lane);
        }
      }
    }
    // exact general path for the destinations that appear in the lists of the
    // batch's methods (rare): one listed (method, destination) per thread
    if (!overflow) {
      const int32_t nh = st.nhl;
      for (int32_t i0 = 0; i0 < nh; i0 += DB_THREADS) {
        const int32_t i = i0 + (int32_t)threadIdx.x;
        const bool have = i < nh;
        const int32_t code = have ? (int32_t)st.hl[i] : 0;
        const int32_t j = code >> 10, rel = code & (DB_SPAN - 1);
        const int32_t D = D0 + rel;
        const int32_t m = st.mid[j];
        const int32_t C = have ? st.hdr[j].w0.x : -1;
        const bool act = have && D < c && D != C;
        int32_t dck = 0, dcbo = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (act)
          r = dense_hit_path(cx, st, j, D, rel >> 8, (uint32_t)(rel & 31), (rel & (DB_THREADS - 1)) >> 5, dest_rec,
                             &dck, &dcbo);
        if (REC && act) __stcs(oc.records + (int64_t)m * row + D - (D > C ? 1 : 0), r);
        if (DIG && act) dig += record_hash(m, D, r);
        if (KEEP) emit_kept(oc, act && (r.w >> 31), m, D, r.z >> 16, dck, dcbo, lane);
      }
    }
    mb += k;
    __syncthreads();
  }
  return dig;
}

template <bool REC, bool DIG, bool KEEP>
__global__ void __launch_bounds__(DB_THREADS, 4) eval_dense(DenseSys sy, OutCtx oc, int32_t mchunk) {
  pdl_wait();
  __shared__ __align__(16) DenseStage st;
  const int32_t m0 = blockIdx.y * mchunk;
  const int32_t m1 = min(sy.M, m0 + mchunk);
  uint64_t dig = dense_tile<REC, DIG, KEEP>(sy, oc, st, (int32_t)blockIdx.x, m0, m1);
  if (DIG) {
    for (int o = 16; o > 0; o >>= 1) dig += __shfl_down_sync(0xffffffffu, dig, o);
    if ((threadIdx.x & 31u) == 0 && dig) atomicAdd(oc.digest, (unsigned long long)dig);
  }
}

// Restricted candidates (explicit destination lists, CSR over methods) on the
// compressed adjacency.  A warp owns groups of 8 consecutive methods: one
// coalesced pass loads their row bounds and headers, asynchronous copies bring
// their L and R lists (stored in method order by the list build) into shared
// memory.  For a run of methods whose lists fit, the warp lays out every
// method's probe rows -- the in-row of each class m uses, C's in-row and
// out-row, the out-row of each class calling m -- with three masks per page of
// 32 rows, then walks the run's candidates 32 at a time across method
// boundaries (a lane finds its method by a forward scan), so lanes are not
// left idle at the end of each method.  A lane probes every row of its method
// at its destination D (one 8-byte summary record, plus one packed word only
// when the record marks D's word non-zero; a method's records are re-read from
// L1 by all its candidates, the packed words come from L2), collects the
// answers of a page as a bit mask and reduces it with the page masks:  gain =
// L rows without the bit, impX = R rows of callers that drop C and already use
// D, worX = R rows of callers that keep C and do not use D yet; a row whose
// class is D itself is masked out and supplies the D-specific list fields
// instead.  Methods whose lists exceed the stage take the general
// per-candidate path.
constexpr int CG_M = 8;               // methods per group
constexpr int CG_LCAP = 64;           // staged L entries per warp
constexpr int CG_RCAP = 64;           // staged R entries per warp
constexpr int CG_PMAX = 128;          // probe rows per method (4 pages of 32)
constexpr int CG_TCAP = 256;          // probe rows of a run of methods (each padded to whole batches)
constexpr int CG_WARPS = 8;
constexpr int CG_PB = 4;              // probes per batch

struct CsrGroup {
  MoveHdr hdr[CG_M];
  int64_t rp[CG_M + 2];               // candidate row bounds of the group
  int32_t loff[CG_M], roff[CG_M];     // list offsets in the stage
  int32_t rbase[CG_M + 1];            // first probe row of each method of the current run
  int4 lent[CG_LCAP];
  int4 rent[CG_RCAP];
  int32_t lsh[CG_LCAP];
  uint2 prow[CG_TCAP];                // probe rows of the run: {record offset, class}
  uint4 pmask[CG_M][CG_PMAX / 32];    // per method and page: {L rows with a use edge, R rows dropping C,
                                      //                        R rows keeping C}
};
constexpr int CG_WARP_BYTES = (int)((sizeof(CsrGroup) + 15) / 16 * 16);
static_assert(CG_WARPS * CG_WARP_BYTES <= 48 * 1024, "stage fits the default shared-memory window");

struct CsrSys {
  EvalCtx cx;
  const uint2 *csum;                  // summary records: out-rows, in-rows, zero row
  const uint32_t *cpk;                // packed non-zero words
  const int4 *dest_rec;
  const int32_t *cls_n, *cls_a;
  const int64_t *cls_P, *cls_Q, *cls_S;
  uint32_t sw;                        // records per row
  uint32_t c;
  int32_t M;                          // methods [m0, M) are evaluated (m0 a multiple of CG_M)
  int32_t staged;                     // 0: every method takes the general path
  unsigned long long *next_group;     // counter handing out groups (m0 / CG_M at launch)
  const uint32_t *gate;               // nullable: a nonzero word (failed list check) skips the launch
};

// Asynchronous global -> shared copies (completion awaited by cp_async_wait).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Predicated read-only load: no branch, so a batch of them is in flight together.
__device__ __forceinline__ uint32_t ldg_if(const uint32_t *p, bool pred) {
  uint32_t v = 0;
  asm("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q ld.global.nc.u32 %0, [%1];\n}\n"
      : "+r"(v)
      : "l"(p), "r"((uint32_t)pred));
  return v;
}


// Methods whose lists exceed the stage: the general per-candidate path.  Its
// arguments are values: a reference to a kernel parameter would keep the whole
// parameter block in local memory for the caller's lifetime.
template <bool REC, bool DIG, bool KEEP>
__device__ __noinline__ uint64_t csr_general_row(const EvalCtx cx, const OutCtx oc, const int32_t *cls_n,
                                                 const int32_t *cls_a, const int64_t *cls_P, const int64_t *cls_Q,
                                                 const int64_t *cls_S, const MoveHdr h, int32_t m,
                                                 const int32_t *cand_dst, int64_t b0, int64_t b1, uint32_t lane) {
  uint64_t dig = 0;
  for (int64_t i0 = b0; i0 < b1; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool act = i < b1;
    const int32_t D = act ? __ldg(cand_dst + i) : 0;
    int32_t dck = 0, dcbo = 0;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (act) {
      DState ds = load_dstate(D, cls_n, cls_a, cls_P, cls_Q, cls_S);
      r = eval_move(cx, h, ds, dck, dcbo);
    }
    if (REC && act) __stcs(oc.records + i, r);
    if (DIG && act) dig += record_hash(m, D, r);
    if (KEEP) emit_kept(oc, act && (r.w >> 31), m, D, r.z >> 16, dck, dcbo, lane);
  }
  return dig;
}

// One candidate (m -> D): probe the rows at D, reduce page by page.  Rows are
// m's L entries, C's in-row and out-row, then m's R entries; the R rows only
// matter to the callers' CBO, so without CBO in the mask they are only
// compared with D, not probed.
__device__ __forceinline__ uint4 csr_candidate(const CsrSys &sy, const CsrGroup &w, const MoveHdr &h, int32_t lo,
                                               int32_t ro, const uint2 *prow, const uint4 *pmask, int32_t D,
                                               int32_t &dck, int32_t &dcbo) {
  const DState ds = dstate_rec(sy.dest_rec, D);
  const int32_t nL = h.w0.z, nR = h.w1.x;
  const int32_t nprobe = (sy.cx.mask & 4u) ? nL + nR + 2 : nL + 2;
  const uint32_t rw = (uint32_t)D >> 10, b = ((uint32_t)D >> 5) & 31u, below = (1u << b) - 1u;
  const uint32_t dsh = (uint32_t)D & 31u;
  Gathered g;
  g.gain = 0; g.impX = 0; g.worX = 0; g.bDC = 0; g.bCD = 0;
  g.t = 0; g.sh = 0; g.outD = 0; g.cntCD = 0; g.inD = 0; g.cntDC = 0;
  int32_t ml = -1, mr = -1;  // entries of m's lists whose class is D
  for (int32_t p0 = 0; p0 < nprobe; p0 += 32) {
    const int32_t pend = min(nprobe - p0, 32);
    uint32_t bits = 0, match = 0;
    for (int32_t k0 = 0; k0 < pend; k0 += CG_PB) {
      uint2 rec[CG_PB];
#pragma unroll
      for (int u = 0; u < CG_PB; ++u) {
        const uint2 pw = prow[p0 + k0 + u];  // rows past the probed ones are the zero row
        match |= (uint32_t)((int32_t)pw.y == D) << (k0 + u);
        rec[u] = __ldg(sy.csum + (pw.x + rw));
      }
      uint32_t word[CG_PB];
#pragma unroll
      for (int u = 0; u < CG_PB; ++u)
        word[u] = ldg_if(sy.cpk + rec[u].y + __popc(rec[u].x & below), (rec[u].x >> b) & 1u);
#pragma unroll
      for (int u = 0; u < CG_PB; ++u) bits |= ((word[u] >> dsh) & 1u) << (k0 + u);
    }
    const uint4 pm = pmask[p0 >> 5];
    const uint32_t valid = ~match;
    const uint32_t lv = pm.x & valid;
    g.gain += __popc(lv) - __popc(bits & lv);
    g.impX += __popc(bits & pm.y & valid);
    g.worX += __popc(~bits & pm.z & valid);
    for (uint32_t mm = match; mm; mm &= mm - 1u) {  // D appears at most once among L and once among R
      const int32_t e = p0 + __ffs(mm) - 1;
      if (e < nL) ml = e; else mr = e - nL - 2;
    }
    const int32_t cin = nL - p0;
    if (cin >= 0 && cin < 32) g.bDC = (int32_t)((bits >> cin) & 1u);
    if (cin + 1 >= 0 && cin + 1 < 32) g.bCD = (int32_t)((bits >> (cin + 1)) & 1u);
  }
  if (!(sy.cx.mask & 4u)) {
    for (int32_t e = 0; e < nR; ++e)
      if (w.rent[ro + e].x == D) mr = e;
  }
  if (ml >= 0) {
    const int4 v = w.lent[lo + ml];
    g.outD = v.y;
    g.cntCD = v.z;
    g.t = v.w;
    g.sh = w.lsh[lo + ml];
  }
  if (mr >= 0) {
    const int4 v = w.rent[ro + mr];
    g.inD = v.y;
    g.cntDC = v.z;
  }
  return finish_move(h, ds, g, sy.cx.mask, sy.cx.min_improved, dck, dcbo);
}

__device__ __forceinline__ int32_t warp_scan_incl(int32_t v, uint32_t lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane >= o) v += t;
  }
  return v;
}

template <bool REC, bool DIG, bool KEEP>
__global__ void __launch_bounds__(CG_WARPS * 32, 4) eval_csr_grouped(CsrSys sy, OutCtx oc,
                                                                     const int64_t *cand_rowptr,
                                                                     const int32_t *cand_dst) {
  pdl_wait();
  if (sy.gate && *sy.gate) return;  // the lists of this launch failed their check
  extern __shared__ __align__(16) unsigned char cg_smem[];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  CsrGroup &w = *reinterpret_cast<CsrGroup *>(cg_smem + (size_t)wid * CG_WARP_BYTES);
  const uint32_t sw = sy.sw, zero_row = 2u * sy.c * sw;
  const int64_t ngroups = ((int64_t)sy.M + CG_M - 1) / CG_M;
  uint64_t dig = 0;
  // warps take groups from a counter as they finish (groups differ widely in
  // work: list lengths, big methods), in increasing order
  auto take = [&]() {
    return __shfl_sync(0xffffffffu, lane == 0 ? (int64_t)atomicAdd(sy.next_group, 1ull) : (int64_t)0, 0);
  };
  for (int64_t grp = take(); grp < ngroups; grp = take()) {
    const int32_t ma = (int32_t)(grp * CG_M);
    const int32_t nm = min(CG_M, sy.M - ma);
    __syncwarp();  // the previous group's readers are done with the stage
    MoveHdr h;
    h.w0 = make_int4(0, 0, 0, 0);
    h.w1 = make_int4(0, 0, 0, 0);
    h.w2 = make_int4(0, 0, 0, 0);
    if ((int32_t)lane < nm) {
      h.w0 = __ldg(&sy.cx.hdr[ma + lane].w0);
      h.w1 = __ldg(&sy.cx.hdr[ma + lane].w1);
      h.w2 = __ldg(&sy.cx.hdr[ma + lane].w2);
      w.hdr[lane] = h;
      w.rp[lane + 1] = __ldg(cand_rowptr + ma + lane + 1);
    }
    if (lane == 0) w.rp[0] = __ldg(cand_rowptr + ma);
    const int32_t nl = h.w0.z, nr = h.w1.x;
    const bool big = !sy.staged || nl > CG_LCAP || nr > CG_RCAP || nl + nr + 2 > CG_PMAX;
    const uint32_t bigm = __ballot_sync(0xffffffffu, big);
    __syncwarp();
    int32_t j = 0;
    while (j < nm) {
      if ((bigm >> j) & 1u) {  // lists too long for the stage
        const MoveHdr hj = w.hdr[j];
        dig += csr_general_row<REC, DIG, KEEP>(sy.cx, oc, sy.cls_n, sy.cls_a, sy.cls_P, sy.cls_Q, sy.cls_S, hj,
                                               ma + j, cand_dst, w.rp[j], w.rp[j + 1], lane);
        ++j;
        continue;
      }
      // longest run j..k-1 without a big method whose lists fit together
      const bool inrun = (int32_t)lane >= j && (int32_t)lane < nm;
      const int32_t nalloc = (nl + nr + 2 + CG_PB - 1) / CG_PB * CG_PB;  // probe rows, padded to whole batches
      const int32_t cl = warp_scan_incl(inrun ? nl : 0, lane);
      const int32_t cr = warp_scan_incl(inrun ? nr : 0, lane);
      const int32_t ct = warp_scan_incl(inrun ? nalloc : 0, lane);
      const uint32_t after = bigm & ~((2u << j) - 1u);  // big methods after j
      const int32_t fb = after ? __ffs(after) - 1 : 32;
      const uint32_t fits = __ballot_sync(0xffffffffu, inrun && (int32_t)lane < fb && cl <= CG_LCAP &&
                                                           cr <= CG_RCAP && ct <= CG_TCAP);
      const int32_t k = j + __popc(fits);
      const bool mine = (int32_t)lane >= j && (int32_t)lane < k;
      const int32_t totL = __shfl_sync(0xffffffffu, cl, k - 1);
      const int32_t totR = __shfl_sync(0xffffffffu, cr, k - 1);
      const int32_t totT = __shfl_sync(0xffffffffu, ct, k - 1);
      const uint32_t hasl = __ballot_sync(0xffffffffu, mine && nl > 0);
      const uint32_t hasr = __ballot_sync(0xffffffffu, mine && nr > 0);
      const int32_t l0 = __shfl_sync(0xffffffffu, h.w0.y, hasl ? __ffs(hasl) - 1 : 0);
      const int32_t r0 = __shfl_sync(0xffffffffu, h.w0.w, hasr ? __ffs(hasr) - 1 : 0);
      if (mine) {
        w.loff[lane] = cl - nl;
        w.roff[lane] = cr - nr;
        w.rbase[lane] = ct - nalloc;
#pragma unroll
        for (int pg = 0; pg < CG_PMAX / 32; ++pg) w.pmask[lane][pg] = make_uint4(0u, 0u, 0u, 0u);
      }
      if ((int32_t)lane == k) w.rbase[lane] = totT;
      for (int32_t e = (int32_t)lane; e < totL; e += 32) {
        cp_async16(&w.lent[e], sy.cx.l_list + l0 + e);
        cp_async4(&w.lsh[e], sy.cx.l_s + l0 + e);
      }
      for (int32_t e = (int32_t)lane; e < totR; e += 32) cp_async16(&w.rent[e], sy.cx.r_list + r0 + e);
      cp_async_wait();
      __syncwarp();
      // probe rows of the whole run: row t belongs to method mi with rbase[mi] <= t < rbase[mi + 1];
      // order per method: L entries, C's in-row, C's out-row, R entries, zero rows up to the batch end
      for (int32_t t = (int32_t)lane; t < totT; t += 32) {
        int32_t mi = j;
        while (w.rbase[mi + 1] <= t) ++mi;
        const int32_t kk = t - w.rbase[mi];
        const MoveHdr hm = w.hdr[mi];
        const int32_t nL = hm.w0.z, nR = hm.w1.x, C = hm.w0.x, lo = w.loff[mi], ro = w.roff[mi];
        uint32_t off = zero_row, cls = 0xffffffffu;
        if (kk < nL) {
          const int4 v = w.lent[lo + kk];
          cls = (uint32_t)v.x;
          off = (sy.c + cls) * sw;
          if (v.y > 0) atomicOr(&w.pmask[mi][kk >> 5].x, 1u << (kk & 31));
        } else if (kk < nL + 2) {
          off = (kk == nL ? sy.c + (uint32_t)C : (uint32_t)C) * sw;  // C is never a candidate: no class
        } else if (kk < nL + nR + 2) {
          const int4 v = w.rent[ro + kk - nL - 2];
          cls = (uint32_t)v.x;
          off = cls * sw;
          if (v.z == v.y) atomicOr(&w.pmask[mi][kk >> 5].y, 1u << (kk & 31));
          else atomicOr(&w.pmask[mi][kk >> 5].z, 1u << (kk & 31));
        }
        w.prow[t] = make_uint2(off, cls);
      }
      __syncwarp();
      // the run's candidates, 32 at a time across method boundaries; a lane finds
      // its method by a forward scan from the method of the chunk's first candidate
      {
        const int64_t ce = w.rp[k];
        int32_t k0 = j;
        int64_t i0 = w.rp[j];
        int32_t Dn = i0 + (int64_t)lane < ce ? __ldg(cand_dst + i0 + lane) : 0;
        for (; i0 < ce; i0 += 32) {
          const int64_t i = i0 + lane;
          const bool act = i < ce;
          const int32_t D = Dn;
          if (i0 + 32 + (int64_t)lane < ce) Dn = __ldg(cand_dst + i0 + 32 + lane);  // next chunk in flight
          int32_t mi = k0;
          if (act)
            while (w.rp[mi + 1] <= i) ++mi;
          int32_t dck = 0, dcbo = 0;
          uint4 r = make_uint4(0, 0, 0, 0);
          if (act) {
            const MoveHdr hm = w.hdr[mi];
            r = csr_candidate(sy, w, hm, w.loff[mi], w.roff[mi], &w.prow[w.rbase[mi]], w.pmask[mi], D, dck,
                              dcbo);
          }
          if (REC && act) __stcs(oc.records + i, r);
          if (DIG && act) dig += record_hash(ma + mi, D, r);
          if (KEEP) emit_kept(oc, act && (r.w >> 31), ma + mi, D, r.z >> 16, dck, dcbo, lane);
          k0 = __shfl_sync(0xffffffffu, mi, 31);
        }
      }
      __syncwarp();  // lists and rows reused by the next run
      j = k;
    }
  }
  if (DIG) {
    for (int o = 16; o > 0; o >>= 1) dig += __shfl_down_sync(0xffffffffu, dig, o);
    if (lane == 0 && dig) atomicAdd(oc.digest, (unsigned long long)dig);
  }
}

// Blocks of the grouped kernel resident on the device (occupancy query, cached
// per instantiation).
template <bool REC, bool DIG, bool KEEP>
int64_t grouped_resident_grid() {
  static std::atomic<int64_t> cached{0};
  int64_t v = cached.load(std::memory_order_relaxed);
  if (!v) {
    int dev = 0, sms = B300_SMS, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, eval_csr_grouped<REC, DIG, KEEP>, CG_WARPS * 32,
                                                      CG_WARPS * CG_WARP_BYTES) != cudaSuccess || per < 1)
      per = 1;
    v = (int64_t)sms * per;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

// Candidate lists: row-pointer checks (thread per method) and range / self
// checks streamed over the destinations (a warp per contiguous range of
// entries: one binary search for the range's first method, then each lane
// finds its method by a forward scan), plus a content hash of the lists
// (every (index, destination) and every row end) that keys the cached kept
// moves of a list evaluation.
__device__ __forceinline__ uint64_t cand_mix(uint64_t v) {
  v *= 0x9E3779B97F4A7C15ULL;
  return v ^ (v >> 31);
}

__global__ void validate_cand_rows(const int64_t *rowptr, int32_t M, int64_t n_cand, uint32_t *err,
                                   unsigned long long *hash) {
  pdl_wait();
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t e = 0;
  uint64_t h = 0;
  if (x < M) {
    const int64_t a = rowptr[x], b = rowptr[x + 1];
    if (x == 0 && (a != 0 || rowptr[M] != n_cand)) e |= VE_CAND_ROWPTR;
    if (a < 0 || b < a || b > n_cand) e |= VE_CAND_ROWPTR;
    h = cand_mix((uint64_t)b ^ ((uint64_t)x << 40) ^ 0x6a09e667f3bcc909ULL);
  }
  for (int o = 16; o > 0; o >>= 1) {
    e |= __shfl_xor_sync(0xffffffffu, e, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicOr(err, e);
    if (h) atomicAdd(hash, (unsigned long long)h);
  }
}

// first method whose row ends after entry i (rows are only trusted to be
// in bounds here; a bad row pointer is reported by validate_cand_rows)
__device__ __forceinline__ int32_t owner_of(const int64_t *rowptr, int32_t M, int64_t i) {
  int32_t lo = 0, hi = M;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (rowptr[mid + 1] <= i) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One warp per range of per_warp candidates (a multiple of 128).  For each
// chunk of 128 the warp loads the row ends of the next 32 methods; when they
// cover the chunk, the owner of every candidate comes from a count of the row
// ends at each chunk position and its prefix sum (shared memory, no search),
// else (more than 32 rows end inside the chunk) each lane walks the row
// pointers forward.  The hash is a sum over candidates, so the order of the
// walk does not change it.
__global__ void __launch_bounds__(256) validate_cand_dst(const int64_t *rowptr, const int32_t *dst,
                                                         const int32_t *method_class, int32_t M, int32_t c,
                                                         int64_t i_lo, int64_t n_cand, int64_t per_warp,
                                                         uint32_t *err, unsigned long long *hash) {
  pdl_wait();
  __shared__ int32_t s_cnt[8][128];
  __shared__ int32_t s_cls[8][32];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t i_begin = i_lo + w * per_warp, i_end = min(n_cand, i_begin + per_warp);
  uint32_t e = 0;
  uint64_t h = 0;
  if (i_begin < i_end) {
    int32_t m = owner_of(rowptr, M, i_begin);  // one search per warp
    for (int64_t i0 = i_begin; i0 < i_end; i0 += 128) {
      const int64_t cend = min(i0 + 128, i_end);
      const int32_t mk = m + (int32_t)lane;
      const int64_t ek = mk < M ? rowptr[mk + 1] : INT64_MAX;
      s_cls[wid][lane] = mk < M ? method_class[mk] : -1;
#pragma unroll
      for (int j = 0; j < 4; ++j) s_cnt[wid][4 * lane + j] = 0;
      __syncwarp();
      if (__shfl_sync(0xffffffffu, ek, 31) >= cend) {
        // rows ending at each position of the chunk (ek > i0: method m owns i0)
        if (ek < cend) atomicAdd(&s_cnt[wid][ek - i0], 1);
        __syncwarp();
        int32_t v[4], run = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          run += s_cnt[wid][4 * lane + j];
          v[j] = run;  // rows ended at or before this position
        }
        int32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if ((int)lane >= o) incl += t;
        }
        const int32_t before = incl - run;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t i = i0 + 4 * lane + j;
          if (i < cend) {
            const int32_t D = dst[i];
            const int32_t own = before + v[j];  // rows of m, m+1, ... that ended at or before i
            if (D < 0 || D >= c) e |= VE_CAND_RANGE;
            else if (D == s_cls[wid][own]) e |= VE_CAND_SELF;
            h += cand_mix(((uint64_t)i << 32) | (uint32_t)D);
          }
        }
        m += __shfl_sync(0xffffffffu, incl, 31);
      } else {
        int32_t mi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + 32 * u + lane;
          mi[u] = m;
          if (i < cend) {
            while (mi[u] < M && rowptr[mi[u] + 1] <= i) ++mi[u];
            const int32_t D = dst[i];
            if (D < 0 || D >= c) e |= VE_CAND_RANGE;
            else if (mi[u] < M && D == method_class[mi[u]]) e |= VE_CAND_SELF;
            h += cand_mix(((uint64_t)i << 32) | (uint32_t)D);
          }
        }
        // owner of the chunk's last candidate (or later: rows ending there are empty)
        const int64_t last = cend - 1;
        int32_t ml = m;
        if (lane == 0)
          while (ml < M && rowptr[ml + 1] <= last) ++ml;
        m = __shfl_sync(0xffffffffu, ml, 0);
      }
      __syncwarp();  // s_cnt and s_cls are rewritten by the next chunk
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e |= __shfl_xor_sync(0xffffffffu, e, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
  }
  if (lane == 0) {
    if (e) atomicOr(err, e);
    if (h) atomicAdd(hash, (unsigned long long)h);
  }
}

__global__ void set_counter(unsigned long long *p, unsigned long long v) {
  pdl_wait();
  *p = v;
}

// The restricted kernel over the methods [m0, m1) of candidate lists (m0 a
// multiple of CG_M); gate (nullable) is read at entry: nonzero skips the launch.
template <bool REC, bool DIG, bool KEEP>
void launch_csr_range(mm_system *s, const EvalCtx &cx, const OutCtx &oc, const int64_t *rowptr, const int32_t *dst,
                      int32_t m0, int32_t m1, const uint32_t *gate) {
  cudaStream_t st = s->stream;
  CsrSys sy;
  sy.cx = cx;
  sy.cx.packed = 1;  // every probe reads the compressed rows
  sy.csum = s->csum;
  sy.cpk = s->cpk;
  sy.dest_rec = s->dest_rec;
  sy.cls_n = s->cls_n;
  sy.cls_a = s->cls_a;
  sy.cls_P = s->cls_P;
  sy.cls_Q = s->cls_Q;
  sy.cls_S = s->cls_S;
  sy.sw = (uint32_t)s->sum_words;
  sy.c = (uint32_t)s->c;
  // record offsets are 32-bit: larger systems evaluate every method on the general path
  sy.staged = s->sum_words * (2 * (int64_t)s->c + 1) < (int64_t)UINT32_MAX ? 1 : 0;
  sy.M = m1;
  sy.gate = gate;
  const int64_t groups = ceil_div((int64_t)(m1 - m0), CG_M);
  const int64_t full = grouped_resident_grid<REC, DIG, KEEP>();
  unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(groups, CG_WARPS), full));
  sy.next_group = s->d_u64 + 5;
  if (m0 == 0) {
    MM_CUDA_TRY(cudaMemsetAsync(sy.next_group, 0, sizeof(unsigned long long), st));
  } else {
    pdl_launch(set_counter, 1, 1, 0, st, sy.next_group, (unsigned long long)(m0 / CG_M));
    MM_LAUNCH_CHECK();
  }
  pdl_launch(eval_csr_grouped<REC, DIG, KEEP>, g, CG_WARPS * 32, CG_WARPS * CG_WARP_BYTES, st, sy, oc, rowptr, dst);
  MM_LAUNCH_CHECK();
}

template <bool REC, bool DIG, bool KEEP>
void launch_eval(mm_system *s, const EvalCtx &cx_in, const OutCtx &oc, const int64_t *rowptr, const int32_t *dst) {
  cudaStream_t st = s->stream;
  EvalCtx cx = cx_in;
  if (!rowptr) {  // the dense tiles read the full bitsets
    ensure_adjacency(s);
    cx.in_adj = s->in_adj;
    cx.out_adj = s->out_adj;
    cx.packed = 0;
  } else {  // candidate lists: every probe reads the compressed rows
    cx.packed = 1;
  }
  if (!rowptr) {
    const int32_t c = s->c, M = s->M;
    unsigned gx = (unsigned)ceil_div(c, DB_SPAN);
    // about 90 blocks per SM (4 resident at a time): short method chunks keep
    // the last wave's tail small relative to the whole launch
    int64_t want_y = std::max<int64_t>(1, (B300_SMS * 3 * 30) / gx);
    int32_t mchunk = (int32_t)std::max<int64_t>(1, ceil_div(M, want_y));
    unsigned gy = (unsigned)ceil_div(M, mchunk);
    DenseSys sy{cx, s->dest_rec, c, M};
    pdl_launch(eval_dense<REC, DIG, KEEP>, dim3(gx, gy), DB_THREADS, 0, st, sy, oc, mchunk);
  } else {
    launch_csr_range<REC, DIG, KEEP>(s, cx, oc, rowptr, dst, 0, s->M, nullptr);
    return;
  }
  MM_LAUNCH_CHECK();
}

void dispatch_eval(mm_system *s, const EvalCtx &cx, const OutCtx &oc, const int64_t *rowptr, const int32_t *dst) {
  const int sel = (oc.records ? 4 : 0) | (oc.digest ? 2 : 0) | (oc.kept_count ? 1 : 0);
  struct Timed {  // events around the launch, for mm_last_eval_ms
    mm_system *s;
    explicit Timed(mm_system *sys) : s(sys) {
      if (s->eval_ev[0]) MM_CUDA_TRY(cudaEventRecord(s->eval_ev[0], s->stream));
    }
    ~Timed() {
      if (s->eval_ev[1] && cudaEventRecord(s->eval_ev[1], s->stream) == cudaSuccess) s->eval_timed = true;
    }
  } timed(s);
  switch (sel) {
    case 0: launch_eval<false, false, false>(s, cx, oc, rowptr, dst); break;
    case 1: launch_eval<false, false, true>(s, cx, oc, rowptr, dst); break;
    case 2: launch_eval<false, true, false>(s, cx, oc, rowptr, dst); break;
    case 3: launch_eval<false, true, true>(s, cx, oc, rowptr, dst); break;
    case 4: launch_eval<true, false, false>(s, cx, oc, rowptr, dst); break;
    case 5: launch_eval<true, false, true>(s, cx, oc, rowptr, dst); break;
    case 6: launch_eval<true, true, false>(s, cx, oc, rowptr, dst); break;
    default: launch_eval<true, true, true>(s, cx, oc, rowptr, dst); break;
  }
}

// The restricted kernel over methods [m0, m1) with the output selection of oc.
void dispatch_csr_range(mm_system *s, const EvalCtx &cx, const OutCtx &oc, const int64_t *rowptr, const int32_t *dst,
                        int32_t m0, int32_t m1, const uint32_t *gate) {
  const int sel = (oc.records ? 4 : 0) | (oc.digest ? 2 : 0) | (oc.kept_count ? 1 : 0);
  switch (sel) {
    case 0: launch_csr_range<false, false, false>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 1: launch_csr_range<false, false, true>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 2: launch_csr_range<false, true, false>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 3: launch_csr_range<false, true, true>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 4: launch_csr_range<true, false, false>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 5: launch_csr_range<true, false, true>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    case 6: launch_csr_range<true, true, false>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
    default: launch_csr_range<true, true, true>(s, cx, oc, rowptr, dst, m0, m1, gate); break;
  }
}

// ---------------------------------------------------------------- top-k

__device__ __forceinline__ bool move_before(const mm_move &a, const mm_move &b) {
  if (a.n_improved != b.n_improved) return a.n_improved > b.n_improved;
  if (a.d_lcom_ck_sum != b.d_lcom_ck_sum) return a.d_lcom_ck_sum < b.d_lcom_ck_sum;
  if (a.d_cbo_sum != b.d_cbo_sum) return a.d_cbo_sum < b.d_cbo_sum;
  if (a.m != b.m) return a.m < b.m;
  return a.d < b.d;
}

constexpr int BITONIC_MAX = 2048;

// one block sorts n kept moves through shared memory sm, which holds n rounded up
// to a power of two (bitonic network; padding sorts last)
__device__ __forceinline__ void bitonic_block(mm_move *v, int32_t n, mm_move *sm) {
  int32_t np = 1;
  while (np < n) np <<= 1;
  for (int32_t i = threadIdx.x; i < np; i += blockDim.x) {
    if (i < n) sm[i] = v[i];
    else {
      mm_move z;
      z.m = 0x7fffffff; z.d = 0x7fffffff; z.n_improved = -1; z.d_lcom_ck_sum = 0x7fffffff;
      z.d_cbo_sum = 0x7fffffff; z.reserved = 0;
      sm[i] = z;
    }
  }
  __syncthreads();
  for (int32_t k = 2; k <= np; k <<= 1) {
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = threadIdx.x; i < np; i += blockDim.x) {
        int32_t ixj = i ^ j;
        if (ixj > i) {
          bool asc = (i & k) == 0;
          mm_move a = sm[i], b = sm[ixj];
          bool swap = asc ? move_before(b, a) : move_before(a, b);
          if (swap) { sm[i] = b; sm[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = sm[i];
}

// block b sorts v[b * BITONIC_MAX, min(n, (b + 1) * BITONIC_MAX))
__global__ void __launch_bounds__(1024) bitonic_sort_chunks(mm_move *v, int64_t n) {
  pdl_wait();
  __shared__ mm_move sm[BITONIC_MAX];
  const int64_t b0 = (int64_t)blockIdx.x * BITONIC_MAX;
  const int32_t len = (int32_t)min((int64_t)BITONIC_MAX, n - b0);
  if (len > 1) bitonic_block(v + b0, len, sm);
}

// Kept moves sorted in the suggestion order, up to KEYED_MAX of them, in two
// launches.  Every move gets one 64-bit key (n_improved descending, then dLCOM,
// dCBO, m, d ascending; each field biased by its minimum over the moves and
// given the bits its range needs).  kept_sort_keys (one block) reads the count,
// reduces the fields' ranges and writes the keys and a copy of the moves to
// scratch; kept_sort_rank (many blocks) gives each move its rank -- how many
// moves have a smaller key, or the same key at an earlier position -- and
// writes it there.  The position settles ties (equal keys mean equal moves,
// possible only when a candidate list repeats a destination), so the ranks
// are a permutation.  If the ranges need more than 64 bits, the first launch
// sorts the moves themselves through a bitonic network in shared memory and
// the second does nothing.  The count is read on the device when count is
// given, so a caller needs no round trip first; nothing happens unless
// 2 <= K <= min(cap, KEYED_MAX).
constexpr int KEYED_MAX = 8192;
constexpr size_t KEYED_SMEM = sizeof(mm_move) * KEYED_MAX;  // the bitonic fallback
// scratch: {K to rank (0 = none), pad, keys[KEYED_MAX], moves[KEYED_MAX]}
constexpr size_t KEYED_WS = 16 + (sizeof(uint64_t) + sizeof(mm_move)) * KEYED_MAX;
constexpr int RANK_ITEMS = 32, RANK_PARTS = 8;  // moves per block, key ranges per move
constexpr size_t RANK_SMEM = sizeof(uint64_t) * KEYED_MAX;

__device__ __forceinline__ int bits_dev(uint32_t v) { return v ? 32 - __clz(v) : 0; }  // bits for [0, v]

__global__ void __launch_bounds__(1024) kept_sort_keys(mm_move *v, const unsigned long long *count, int32_t n,
                                                       int64_t cap, int32_t c, int32_t M, unsigned long long *ws) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char ksm[];
  __shared__ int32_t red[6][32];
  const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t K = count ? (int64_t)*count : (int64_t)n;
  if (K < 2 || K > cap || K > KEYED_MAX) {
    if (tid == 0) ws[0] = 0;
    return;
  }
  const int32_t k = (int32_t)K;
  // ranges of n_improved, dLCOM, dCBO
  int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int32_t i = tid; i < k; i += 1024) {
    const mm_move a = v[i];
    const int32_t f[3] = {a.n_improved, a.d_lcom_ck_sum, a.d_cbo_sum};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lo[q] = min(lo[q], f[q]);
      hi[q] = max(hi[q], f[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = min(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = max(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
    if (lane == 0) {
      red[2 * q][warp] = lo[q];
      red[2 * q + 1][warp] = hi[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    lo[q] = red[2 * q][lane];
    hi[q] = red[2 * q + 1][lane];
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = min(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = max(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  }
  const int w_d = bits_dev((uint32_t)max(c - 1, 0)), w_m = bits_dev((uint32_t)max(M - 1, 0));
  const int w_cbo = bits_dev((uint32_t)((int64_t)hi[2] - lo[2])), w_ck = bits_dev((uint32_t)((int64_t)hi[1] - lo[1]));
  const int w_n = bits_dev((uint32_t)((int64_t)hi[0] - lo[0]));
  if (w_d + w_m + w_cbo + w_ck + w_n > 64) {  // every block thread sees the same ranges
    if (tid == 0) ws[0] = 0;
    __syncthreads();
    bitonic_block(v, k, reinterpret_cast<mm_move *>(ksm));
    return;
  }
  const int s_cbo = w_d + w_m, s_ck = s_cbo + w_cbo, s_n = s_ck + w_ck;
  uint64_t *key = reinterpret_cast<uint64_t *>(ws + 2);
  mm_move *mv = reinterpret_cast<mm_move *>(ws + 2 + KEYED_MAX);
  for (int32_t i = tid; i < k; i += 1024) {
    const mm_move a = v[i];
    uint64_t kk = ((uint64_t)(uint32_t)a.m << w_d) | (uint64_t)(uint32_t)a.d;
    if (w_cbo) kk |= (uint64_t)((uint32_t)a.d_cbo_sum - (uint32_t)lo[2]) << s_cbo;
    if (w_ck) kk |= (uint64_t)((uint32_t)a.d_lcom_ck_sum - (uint32_t)lo[1]) << s_ck;
    if (w_n) kk |= (uint64_t)((uint32_t)hi[0] - (uint32_t)a.n_improved) << s_n;
    key[i] = kk;
    mv[i] = a;
  }
  if (tid == 0) ws[0] = (unsigned long long)k;
}

// Block b ranks moves b*RANK_ITEMS .. +RANK_ITEMS-1: lane l of warp q counts,
// for move b*RANK_ITEMS + l, the keys before it among the q-th of RANK_PARTS
// ranges of positions (a warp's lanes read the same key: a broadcast).
__global__ void __launch_bounds__(RANK_ITEMS * RANK_PARTS) kept_sort_rank(mm_move *v,
                                                                          const unsigned long long *ws) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char rsm[];
  __shared__ int32_t part[RANK_PARTS][RANK_ITEMS];
  const int32_t k = (int32_t)ws[0];  // 0 <= k <= KEYED_MAX
  const int32_t i0 = (int32_t)blockIdx.x * RANK_ITEMS;
  if (i0 >= k) return;  // the same for the whole block
  const uint64_t *key = reinterpret_cast<const uint64_t *>(ws + 2);
  const mm_move *mv = reinterpret_cast<const mm_move *>(ws + 2 + KEYED_MAX);
  uint64_t *sk = reinterpret_cast<uint64_t *>(rsm);
  const int tid = (int)threadIdx.x, lane = tid & 31, q = tid >> 5;
  for (int32_t j = tid; j < k; j += RANK_ITEMS * RANK_PARTS) sk[j] = key[j];
  __syncthreads();
  const int32_t i = i0 + lane;
  const uint64_t ki = i < k ? sk[i] : 0ull;
  const int32_t j0 = (int32_t)((int64_t)k * q / RANK_PARTS), j1 = (int32_t)((int64_t)k * (q + 1) / RANK_PARTS);
  int32_t r = 0;
#pragma unroll 4
  for (int32_t j = j0; j < j1; ++j) {
    const uint64_t kj = sk[j];
    r += (int32_t)((kj < ki) | ((kj == ki) & (j < i)));
  }
  part[q][lane] = r;
  __syncthreads();
  if (q == 0 && i < k) {
    int32_t rank = 0;
#pragma unroll
    for (int p = 0; p < RANK_PARTS; ++p) rank += part[p][lane];
    v[rank] = mv[i];
  }
}

static void keyed_sort_launch(mm_system *s, mm_move *v, const unsigned long long *count, int32_t n, int64_t cap,
                              cudaStream_t st) {
  static const cudaError_t attr_keys =
      cudaFuncSetAttribute(kept_sort_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KEYED_SMEM);
  static const cudaError_t attr_rank =
      cudaFuncSetAttribute(kept_sort_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RANK_SMEM);
  MM_CUDA_TRY(attr_keys);
  MM_CUDA_TRY(attr_rank);
  auto *ws = static_cast<unsigned long long *>(s->keyed_ws.need(KEYED_WS, st));
  pdl_launch(kept_sort_keys, 1, 1024, KEYED_SMEM, st, v, count, n, cap, s->c, s->M, ws);
  MM_LAUNCH_CHECK();
  pdl_launch(kept_sort_rank, KEYED_MAX / RANK_ITEMS, RANK_ITEMS * RANK_PARTS, RANK_SMEM, st, v,
             static_cast<const unsigned long long *>(ws));
  MM_LAUNCH_CHECK();
}

// block i sorts segment i (base + i*stride, counts[i] moves) when it fits in one block
__global__ void __launch_bounds__(1024) bitonic_sort_segments(mm_move *base, int64_t stride,
                                                              const unsigned long long *counts) {
  __shared__ mm_move sm[BITONIC_MAX];
  const unsigned long long K = counts[blockIdx.x];
  if (K < 2 || K > (unsigned long long)BITONIC_MAX || (int64_t)K > stride) return;
  bitonic_block(base + (int64_t)blockIdx.x * stride, (int32_t)K, sm);
}

// field-wise LSD radix sort of kept moves through a permutation
__global__ void gather_field(const mm_move *v, const uint32_t *perm, int64_t n, int field, int64_t bias,
                             uint32_t *key) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const mm_move &a = v[perm[i]];
  int64_t f;
  switch (field) {
    case 0: f = a.d; break;
    case 1: f = a.m; break;
    case 2: f = (int64_t)a.d_cbo_sum + bias; break;
    case 3: f = (int64_t)a.d_lcom_ck_sum + bias; break;
    default: f = bias - (int64_t)a.n_improved; break;  // descending: bias = the largest n_improved
  }
  key[i] = (uint32_t)f;
}

// min and max of n_improved, d_lcom_ck_sum and d_cbo_sum over the kept moves
// (mm = {min, max} x 3, initialised to {INT_MAX, INT_MIN})
__global__ void kept_ranges(const mm_move *v, int64_t n, int32_t *mm) {
  pdl_wait();
  int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const mm_move a = v[i];
    const int32_t f[3] = {a.n_improved, a.d_lcom_ck_sum, a.d_cbo_sum};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = min(lo[k], f[k]);
      hi[k] = max(hi[k], f[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&mm[2 * k], lo[k]);
      atomicMax(&mm[2 * k + 1], hi[k]);
    }
  }
}

// One 64-bit key per kept move in the suggestion order: (n_improved desc,
// dLCOM asc, dCBO asc, m asc, d asc), each field biased by its minimum and
// packed into the bits its range needs (field widths from kept_ranges).
struct KeyLayout {
  int32_t nimp_max, ck_min, cbo_min;
  int s_m, s_cbo, s_ck, s_nimp;
};

__global__ void kept_keys(const mm_move *v, int64_t n, KeyLayout kl, uint64_t *key, uint32_t *perm) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const mm_move a = v[i];
  key[i] = ((uint64_t)(uint32_t)(kl.nimp_max - a.n_improved) << kl.s_nimp) |
           ((uint64_t)(uint32_t)(a.d_lcom_ck_sum - kl.ck_min) << kl.s_ck) |
           ((uint64_t)(uint32_t)(a.d_cbo_sum - kl.cbo_min) << kl.s_cbo) | ((uint64_t)(uint32_t)a.m << kl.s_m) |
           (uint64_t)(uint32_t)a.d;
  perm[i] = (uint32_t)i;
}

__global__ void iota_perm(uint32_t *p, int64_t n) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (uint32_t)i;
}

__global__ void permute_moves(const mm_move *in, const uint32_t *perm, int64_t n, mm_move *out) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[perm[i]];
}

__global__ void count_marks(const uint8_t *mark, int64_t n, unsigned long long *out) {
  pdl_wait();
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += mark[i];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

static void check_criteria(const mm_criteria &crit) {
  if ((crit.metric_mask & 7u) == 0 || (crit.metric_mask & ~7u) != 0)
    throw MmError{MM_EINVAL, "criteria: metric_mask must be a non-empty subset of LCOM_CK|LCOM_HS|CBO"};
  if (crit.min_improved < 1) throw MmError{MM_EINVAL, "criteria: min_improved must be >= 1"};
}

// Upload (if host) and validate an explicit candidate list; returns device pointers.
// staging = false: the validation word and hash are read back into host stack
// memory instead of the thread's page-locked staging buffer (which is
// allocated on first use), so nothing is allocated.
static void prepare_candidates(mm_system *s, const mm_candidates *cands, const int64_t **rowptr,
                               const int32_t **dst, int64_t *n_cand, uint64_t *hash = nullptr,
                               bool staging = true) {
  *rowptr = nullptr;
  *dst = nullptr;
  if (!cands || !cands->rowptr) {
    *n_cand = (int64_t)s->M * (int64_t)(s->c - 1);
    if (s->c < 1) *n_cand = 0;
    return;
  }
  if (cands->n_cand < 0) throw MmError{MM_EINVAL, "candidates: n_cand < 0"};
  if (cands->n_cand > 0 && !cands->dst) throw MmError{MM_EINVAL, "candidates: dst is NULL"};
  if (cands->flags & ~(int32_t)MM_CANDS_UNCHANGED) throw MmError{MM_EINVAL, "candidates: unknown flags"};
  *n_cand = cands->n_cand;
  cudaStream_t st = s->stream;
  const bool same = s->lists_kind == cands->ptr_kind && s->lists_rowptr == cands->rowptr &&
                    s->lists_dst == cands->dst && s->lists_n == cands->n_cand && s->lists_edits == s->edits;
  if ((cands->flags & MM_CANDS_UNCHANGED) && same && s->lists_staged) {  // staged: wait for its copy and check
    MM_CUDA_TRY(cudaStreamWaitEvent(st, s->stage_ev, 0));
    unsigned long long words[2] = {0, 0};  // {hash, error word}
    MM_CUDA_TRY(cudaMemcpyAsync(&words[0], s->stage_hash, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaMemcpyAsync(&words[1], s->stage_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaStreamSynchronize(st));
    s->lists_staged = false;
    const uint32_t err = (uint32_t)words[1];
    if (err & VE_CAND_ROWPTR) throw MmError{MM_EINVAL, "candidates: rowptr must start at 0, be non-decreasing and end at n_cand"};
    if (err & VE_CAND_RANGE) throw MmError{MM_EINVAL, "candidates: destination class out of range"};
    if (err & VE_CAND_SELF) throw MmError{MM_EINVAL, "candidates: destination equals the method's own class"};
    s->lists_checked = true;
    s->lists_hash = words[0];
  }
  if ((cands->flags & MM_CANDS_UNCHANGED) && same && s->lists_checked) {
    // checked and hashed by the last list call (host lists: already copied)
    *rowptr = s->lists_dev_rowptr;
    *dst = s->lists_dev_dst;
    if (hash) *hash = s->lists_hash;
    return;
  }
  settle_staged(s);
  s->lists_checked = false;
  if (cands->ptr_kind == MM_PTR_HOST) {  // copied into the handle's list buffer (kept for MM_CANDS_UNCHANGED)
    size_t rb = sizeof(int64_t) * ((size_t)s->M + 1), db = sizeof(int32_t) * (size_t)cands->n_cand;
    char *b = static_cast<char *>(s->lists_ws.need(rb + db + 256, st));
    MM_CUDA_TRY(cudaMemcpyAsync(b, cands->rowptr, rb, cudaMemcpyHostToDevice, st));
    if (db) MM_CUDA_TRY(cudaMemcpyAsync(b + ((rb + 255) & ~size_t(255)), cands->dst, db, cudaMemcpyHostToDevice, st));
    *rowptr = reinterpret_cast<const int64_t *>(b);
    *dst = reinterpret_cast<const int32_t *>(b + ((rb + 255) & ~size_t(255)));
  } else if (cands->ptr_kind == MM_PTR_DEVICE) {
    *rowptr = cands->rowptr;
    *dst = cands->dst;
  } else {
    throw MmError{MM_EINVAL, "candidates: bad ptr_kind"};
  }
  MM_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(uint32_t), st));
  MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 3, 0, sizeof(unsigned long long), st));
  if (s->M > 0) {
    pdl_launch(validate_cand_rows, grid_for(s->M), TPB, 0, st, *rowptr, s->M, *n_cand, s->d_err, s->d_u64 + 3);
    MM_LAUNCH_CHECK();
    if (*n_cand > 0) {
      // one contiguous range per warp (a multiple of 128 entries), at most B300_SMS x 16 blocks of 8 warps
      const int64_t warps = std::min<int64_t>(ceil_div(*n_cand, 128), (int64_t)B300_SMS * 16 * (TPB / 32));
      const int64_t per_warp = ceil_div(ceil_div(*n_cand, warps), 128) * 128;
      const unsigned g = (unsigned)ceil_div(ceil_div(*n_cand, per_warp) * 32, TPB);
      pdl_launch(validate_cand_dst, g, TPB, 0, st, *rowptr, *dst, s->method_class, s->M, s->c, (int64_t)0, *n_cand,
                 per_warp, s->d_err, s->d_u64 + 3);
      MM_LAUNCH_CHECK();
    }
  }
  // d_u64[3] = hash, d_u64[6] = error word: one copy (page-locked staging, or host stack memory)
  unsigned long long local[4] = {0, 0, 0, 0};
  unsigned char *hb = staging ? static_cast<unsigned char *>(host_staging(32)) : reinterpret_cast<unsigned char *>(local);
  MM_CUDA_TRY(cudaMemcpyAsync(hb, s->d_u64 + 3, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  uint32_t err = 0;
  std::memcpy(&err, hb + 24, sizeof(uint32_t));
  uint64_t h = 0;
  std::memcpy(&h, hb, sizeof(uint64_t));
  if (hash) *hash = h;
  if (err & VE_CAND_ROWPTR) throw MmError{MM_EINVAL, "candidates: rowptr must start at 0, be non-decreasing and end at n_cand"};
  if (err & VE_CAND_RANGE) throw MmError{MM_EINVAL, "candidates: destination class out of range"};
  if (err & VE_CAND_SELF) throw MmError{MM_EINVAL, "candidates: destination equals the method's own class"};
  s->lists_checked = true;
  s->lists_kind = cands->ptr_kind;
  s->lists_rowptr = cands->rowptr;
  s->lists_dst = cands->dst;
  s->lists_dev_rowptr = *rowptr;
  s->lists_dev_dst = *dst;
  s->lists_n = cands->n_cand;
  s->lists_edits = s->edits;
  s->lists_hash = h;
}

static EvalCtx make_ctx(mm_system *s, const mm_criteria &crit) {
  EvalCtx cx;
  cx.hdr = s->hdr;
  cx.l_list = s->l_list;
  cx.l_s = s->l_s;
  cx.r_list = s->r_list;
  cx.in_adj = s->in_adj;
  cx.out_adj = s->out_adj;
  cx.aw = s->adj_words;
  cx.csum = s->csum;
  cx.cpk = s->cpk;
  cx.sw = s->sum_words;
  cx.c = s->c;
  cx.packed = 0;
  cx.mask = crit.metric_mask;
  cx.min_improved = crit.min_improved;
  return cx;
}

// Kept-move buffer of the system: [cap] moves followed by one mark byte per method.
static void kept_buffers(mm_system *s, int64_t cap, mm_move **kept, uint8_t **mark) {
  size_t bytes = sizeof(mm_move) * (size_t)cap + (size_t)s->M + 256;
  char *b = static_cast<char *>(s->kept_ws.need(bytes, s->stream));
  *kept = reinterpret_cast<mm_move *>(b);
  *mark = reinterpret_cast<uint8_t *>(b + sizeof(mm_move) * (size_t)cap);
}

static void attach_kept(mm_system *s, OutCtx &oc, int64_t cap) {
  mm_move *kept;
  uint8_t *mark;
  kept_buffers(s, cap, &kept, &mark);
  MM_CUDA_TRY(cudaMemsetAsync(mark, 0, (size_t)s->M, s->stream));
  MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 1, 0, sizeof(unsigned long long), s->stream));
  oc.kept = kept;
  oc.kept_count = s->d_u64 + 1;
  oc.kept_cap = cap;
  oc.kept_mark = mark;
}

static int64_t kept_capacity(mm_system *s) {
  return std::max<int64_t>(65536, s->kept_cap);
}

// Host candidate lists of at least this many entries are copied in chunks of
// methods, each chunk checked and evaluated while the next one is copied.
constexpr int64_t HOST_LISTS_CHUNKED = (int64_t)1 << 24;
constexpr int HOST_LIST_CHUNKS = 8;

// Chunk bounds at multiples of the restricted kernel's method group, from the
// host row pointers (a malformed rowptr is reported by the device check).
static int chunk_bounds(const mm_system *s, const mm_candidates *cands, int32_t *mb, int64_t *lo) {
  const int32_t M = s->M;
  const int64_t n = cands->n_cand;
  const int K = n >= HOST_LISTS_CHUNKED ? HOST_LIST_CHUNKS : 1;
  for (int k = 0; k <= K; ++k) {
    mb[k] = k == K ? M : (int32_t)((int64_t)M * k / K / CG_M * CG_M);
    lo[k] = k == K ? n : std::min<int64_t>(std::max<int64_t>(cands->rowptr[mb[k]], 0), n);
    if (k > 0) lo[k] = std::max(lo[k], lo[k - 1]);
  }
  return K;
}

// Launch the check of destinations [a, e) on stream st.
static void check_dst_range(mm_system *s, const int64_t *rowptr, const int32_t *dst, int64_t a, int64_t e,
                            uint32_t *err, unsigned long long *hash, cudaStream_t st) {
  if (e <= a) return;
  const int64_t warps = std::min<int64_t>(ceil_div(e - a, 128), (int64_t)B300_SMS * 16 * (TPB / 32));
  const int64_t per_warp = ceil_div(ceil_div(e - a, warps), 128) * 128;
  const unsigned g = (unsigned)ceil_div(ceil_div(e - a, per_warp) * 32, TPB);
  pdl_launch(validate_cand_dst, g, TPB, 0, st, rowptr, dst, s->method_class, s->M, s->c, a, e, per_warp, err, hash);
  MM_LAUNCH_CHECK();
}

void settle_staged(mm_system *s) {
  if (s->lists_staged) {
    MM_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->stage_ev, 0));
    s->lists_staged = false;
  }
}

// Copy host lists to the device and check them on the copy stream; the
// system's stream does not wait (see mm_stage_candidates).
void stage_candidates(mm_system *s, const mm_candidates *cands) {
  if (!cands || !cands->rowptr) throw MmError{MM_EINVAL, "stage_candidates: no candidate lists"};
  if (cands->ptr_kind != MM_PTR_HOST) throw MmError{MM_EINVAL, "stage_candidates: the lists must be in host memory"};
  if (cands->n_cand < 0) throw MmError{MM_EINVAL, "candidates: n_cand < 0"};
  if (cands->n_cand > 0 && !cands->dst) throw MmError{MM_EINVAL, "candidates: dst is NULL"};
  if (cands->flags & ~(int32_t)MM_CANDS_UNCHANGED) throw MmError{MM_EINVAL, "candidates: unknown flags"};
  cudaStream_t st = s->stream;
  const int32_t M = s->M;
  const int64_t n = cands->n_cand;
  settle_staged(s);
  s->lists_checked = false;
  if (!s->stage_ev) MM_CUDA_TRY(cudaEventCreateWithFlags(&s->stage_ev, cudaEventDisableTiming));
  const size_t rb = sizeof(int64_t) * ((size_t)M + 1), rb_pad = (rb + 255) & ~size_t(255);
  const size_t db_pad = (sizeof(int32_t) * (size_t)n + 255) & ~size_t(255);
  char *b = static_cast<char *>(s->lists_ws.need(rb_pad + db_pad + 512, st));
  int64_t *rowptr = reinterpret_cast<int64_t *>(b);
  int32_t *dst = reinterpret_cast<int32_t *>(b + rb_pad);
  s->stage_hash = reinterpret_cast<unsigned long long *>(b + rb_pad + db_pad);
  s->stage_err = reinterpret_cast<uint32_t *>(b + rb_pad + db_pad + 256);
  MM_CUDA_TRY(cudaMemsetAsync(b + rb_pad + db_pad, 0, 512, st));
  for (int k = 0; k < HOST_LIST_CHUNKS; ++k)
    if (!s->chunk_ev[k]) MM_CUDA_TRY(cudaEventCreateWithFlags(&s->chunk_ev[k], cudaEventDisableTiming));
  int64_t lo[HOST_LIST_CHUNKS + 1];
  const int K = M > 0 ? chunk_bounds(s, cands, s->stage_mb, lo) : 0;
  s->stage_chunks = K;
  cudaStream_t cp = fork_side(s, 3);  // after the buffer's allocation and the cleared words
  MM_CUDA_TRY(cudaMemcpyAsync(rowptr, cands->rowptr, rb, cudaMemcpyHostToDevice, cp));
  if (M > 0) {
    pdl_launch(validate_cand_rows, grid_for(M), TPB, 0, cp, static_cast<const int64_t *>(rowptr), M, n, s->stage_err,
               s->stage_hash);
    MM_LAUNCH_CHECK();
  }
  for (int k = 0; k < K; ++k) {  // chunk k copied and checked, then its event
    if (lo[k + 1] > lo[k])
      MM_CUDA_TRY(cudaMemcpyAsync(dst + lo[k], cands->dst + lo[k], sizeof(int32_t) * (size_t)(lo[k + 1] - lo[k]),
                                  cudaMemcpyHostToDevice, cp));
    check_dst_range(s, rowptr, dst, lo[k], lo[k + 1], s->stage_err, s->stage_hash, cp);
    MM_CUDA_TRY(cudaEventRecord(s->chunk_ev[k], cp));
  }
  MM_CUDA_TRY(cudaEventRecord(s->stage_ev, cp));
  s->lists_staged = true;
  s->lists_kind = MM_PTR_HOST;
  s->lists_rowptr = cands->rowptr;
  s->lists_dst = cands->dst;
  s->lists_dev_rowptr = rowptr;
  s->lists_dev_dst = dst;
  s->lists_n = n;
  s->lists_edits = s->edits;
}


// evaluate_moves for large host lists (copy of each chunk overlapped with the
// check and evaluation of the previous ones).  Returns the content hash.
static uint64_t evaluate_host_lists(mm_system *s, const mm_candidates *cands, const EvalCtx &cx, const OutCtx &oc) {
  cudaStream_t st = s->stream;
  const int32_t M = s->M;
  const int64_t n = cands->n_cand;
  const size_t rb = sizeof(int64_t) * ((size_t)M + 1), rb_pad = (rb + 255) & ~size_t(255);
  settle_staged(s);
  char *b = static_cast<char *>(s->lists_ws.need(rb_pad + sizeof(int32_t) * (size_t)n + 256, st));
  int64_t *rowptr = reinterpret_cast<int64_t *>(b);
  int32_t *dst = reinterpret_cast<int32_t *>(b + rb_pad);
  s->lists_checked = false;
  int32_t mb[HOST_LIST_CHUNKS + 1];
  int64_t lo[HOST_LIST_CHUNKS + 1];
  const int K = chunk_bounds(s, cands, mb, lo);
  MM_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(uint32_t), st));
  MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 3, 0, sizeof(unsigned long long), st));
  MM_CUDA_TRY(cudaMemcpyAsync(rowptr, cands->rowptr, rb, cudaMemcpyHostToDevice, st));
  pdl_launch(validate_cand_rows, grid_for(M), TPB, 0, st, static_cast<const int64_t *>(rowptr), M, n, s->d_err,
             s->d_u64 + 3);
  MM_LAUNCH_CHECK();
  // the destination chunks on a copy stream, ordered after the buffer's allocation
  static_assert(HOST_LIST_CHUNKS <= (int)(sizeof(s->chunk_ev) / sizeof(s->chunk_ev[0])), "one event per chunk");
  for (int k = 0; k < HOST_LIST_CHUNKS; ++k)
    if (!s->chunk_ev[k]) MM_CUDA_TRY(cudaEventCreateWithFlags(&s->chunk_ev[k], cudaEventDisableTiming));
  cudaStream_t cp = fork_side(s, 1);
  for (int k = 0; k < K; ++k) {
    const int64_t a = lo[k], e = lo[k + 1];
    if (e > a)
      MM_CUDA_TRY(cudaMemcpyAsync(dst + a, cands->dst + a, sizeof(int32_t) * (size_t)(e - a), cudaMemcpyHostToDevice,
                                  cp));
    MM_CUDA_TRY(cudaEventRecord(s->chunk_ev[k], cp));
  }
  if (s->eval_ev[0]) MM_CUDA_TRY(cudaEventRecord(s->eval_ev[0], st));  // mm_last_eval_ms: the pipelined span
  for (int k = 0; k < K; ++k) {
    const int64_t a = lo[k], e = lo[k + 1];
    MM_CUDA_TRY(cudaStreamWaitEvent(st, s->chunk_ev[k], 0));
    check_dst_range(s, rowptr, dst, a, e, s->d_err, s->d_u64 + 3, st);
    if (mb[k + 1] > mb[k])
      dispatch_csr_range(s, cx, oc, rowptr, dst, mb[k], mb[k + 1], s->d_err);  // skipped if a check failed
  }
  if (s->eval_ev[1] && cudaEventRecord(s->eval_ev[1], st) == cudaSuccess) s->eval_timed = true;
  // the check's verdict and the content hash, read back once
  unsigned long long local[4] = {0, 0, 0, 0};
  MM_CUDA_TRY(cudaMemcpyAsync(local, s->d_u64 + 3, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  uint32_t err = 0;
  std::memcpy(&err, reinterpret_cast<unsigned char *>(local) + 24, sizeof(uint32_t));
  const uint64_t h = local[0];
  if (err & VE_CAND_ROWPTR) throw MmError{MM_EINVAL, "candidates: rowptr must start at 0, be non-decreasing and end at n_cand"};
  if (err & VE_CAND_RANGE) throw MmError{MM_EINVAL, "candidates: destination class out of range"};
  if (err & VE_CAND_SELF) throw MmError{MM_EINVAL, "candidates: destination equals the method's own class"};
  s->lists_checked = true;
  s->lists_kind = MM_PTR_HOST;
  s->lists_rowptr = cands->rowptr;
  s->lists_dst = cands->dst;
  s->lists_dev_rowptr = rowptr;
  s->lists_dev_dst = dst;
  s->lists_n = n;
  s->lists_edits = s->edits;
  s->lists_hash = h;
  return h;
}

// evaluate_moves for lists staged by mm_stage_candidates: chunk k is evaluated
// once its copy and check are done (a failed check skips every later launch),
// the verdict and the content hash read back once.  Returns the hash.
static uint64_t evaluate_staged_lists(mm_system *s, const EvalCtx &cx, const OutCtx &oc) {
  cudaStream_t st = s->stream;
  const int64_t *rowptr = s->lists_dev_rowptr;
  const int32_t *dst = s->lists_dev_dst;
  if (s->eval_ev[0]) MM_CUDA_TRY(cudaEventRecord(s->eval_ev[0], st));
  for (int k = 0; k < s->stage_chunks; ++k) {
    MM_CUDA_TRY(cudaStreamWaitEvent(st, s->chunk_ev[k], 0));
    if (s->stage_mb[k + 1] > s->stage_mb[k])
      dispatch_csr_range(s, cx, oc, rowptr, dst, s->stage_mb[k], s->stage_mb[k + 1], s->stage_err);
  }
  if (s->eval_ev[1] && cudaEventRecord(s->eval_ev[1], st) == cudaSuccess) s->eval_timed = true;
  MM_CUDA_TRY(cudaStreamWaitEvent(st, s->stage_ev, 0));
  unsigned long long words[2] = {0, 0};  // {hash, error word}
  MM_CUDA_TRY(cudaMemcpyAsync(&words[0], s->stage_hash, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaMemcpyAsync(&words[1], s->stage_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  s->lists_staged = false;
  const uint32_t err = (uint32_t)words[1];
  if (err & VE_CAND_ROWPTR) throw MmError{MM_EINVAL, "candidates: rowptr must start at 0, be non-decreasing and end at n_cand"};
  if (err & VE_CAND_RANGE) throw MmError{MM_EINVAL, "candidates: destination class out of range"};
  if (err & VE_CAND_SELF) throw MmError{MM_EINVAL, "candidates: destination equals the method's own class"};
  s->lists_checked = true;
  s->lists_hash = words[0];
  return words[0];
}

void evaluate_moves(mm_system *s, const mm_criteria &crit, const mm_candidates *cands, mm_move_eval *records,
                    uint64_t *digest, int32_t kind) {
  check_criteria(crit);
  if (kind != MM_PTR_HOST && kind != MM_PTR_DEVICE) throw MmError{MM_EINVAL, "evaluate: bad out_kind"};
  cudaStream_t st = s->stream;
  const int64_t *rowptr;
  const int32_t *dst;
  int64_t n_cand;
  uint64_t chash = 0;
  const bool chunked = cands && cands->rowptr && cands->ptr_kind == MM_PTR_HOST && cands->dst &&
                       cands->n_cand >= HOST_LISTS_CHUNKED && s->M > 0 && !(cands->flags & ~(int32_t)MM_CANDS_UNCHANGED) &&
                       !((cands->flags & MM_CANDS_UNCHANGED) && (s->lists_checked || s->lists_staged) &&
                         s->lists_kind == MM_PTR_HOST && s->lists_rowptr == cands->rowptr &&
                         s->lists_dst == cands->dst && s->lists_n == cands->n_cand && s->lists_edits == s->edits);
  // lists staged by mm_stage_candidates: each chunk is evaluated as it lands
  const bool staged = cands && cands->rowptr && (cands->flags & MM_CANDS_UNCHANGED) && s->lists_staged &&
                      s->lists_kind == cands->ptr_kind && s->lists_rowptr == cands->rowptr &&
                      s->lists_dst == cands->dst && s->lists_n == cands->n_cand && s->lists_edits == s->edits &&
                      s->stage_chunks > 0 && cands->n_cand > 0;
  if (chunked || staged) {  // pointers filled in below, after the pipelined copy
    rowptr = nullptr;
    dst = nullptr;
    n_cand = cands->n_cand;
  } else {
    prepare_candidates(s, cands, &rowptr, &dst, &n_cand, &chash);
  }
  s->kept_valid = false;
  if (n_cand == 0 || s->M == 0) {
    if (digest) {
      if (kind == MM_PTR_HOST) *digest = 0;
      else MM_CUDA_TRY(cudaMemsetAsync(digest, 0, sizeof(uint64_t), st));
    }
    return;
  }
  EvalCtx cx = make_ctx(s, crit);
  OutCtx oc{};
  uint4 *rec_dev = nullptr;
  if (records) {
    if (kind == MM_PTR_DEVICE) rec_dev = reinterpret_cast<uint4 *>(records);
    else rec_dev = static_cast<uint4 *>(s->eval_ws.need(sizeof(uint4) * (size_t)n_cand, st));
  }
  oc.records = rec_dev;
  if (digest) {
    oc.digest = s->d_u64;
    MM_CUDA_TRY(cudaMemsetAsync(s->d_u64, 0, sizeof(unsigned long long), st));
  }
  // The pass also compacts the kept moves, so a following mm_suggest_moves with
  // the same criteria (and, for explicit lists, lists of the same content hash)
  // needs no second pass.
  const int64_t cap = kept_capacity(s);
  attach_kept(s, oc, cap);
  if (chunked) {
    chash = evaluate_host_lists(s, cands, cx, oc);
    rowptr = s->lists_dev_rowptr;
  } else if (staged) {
    chash = evaluate_staged_lists(s, cx, oc);
    rowptr = s->lists_dev_rowptr;
  } else {
    dispatch_eval(s, cx, oc, rowptr, dst);
  }
  s->kept_valid = true;
  s->kept_mask = crit.metric_mask;
  s->kept_min = crit.min_improved;
  s->kept_cap = cap;
  s->kept_lists = rowptr != nullptr;
  s->kept_hash = chash;
  s->kept_ncand = n_cand;
  if (records && kind == MM_PTR_HOST)
    MM_CUDA_TRY(cudaMemcpyAsync(records, rec_dev, sizeof(uint4) * (size_t)n_cand, cudaMemcpyDeviceToHost, st));
  if (digest) {
    MM_CUDA_TRY(cudaMemcpyAsync(digest, s->d_u64, sizeof(uint64_t),
                                kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  }
  if (kind == MM_PTR_HOST) MM_CUDA_TRY(cudaStreamSynchronize(st));
}

// Sort kept moves in the suggestion order: keys by one block and ranks by many
// up to 8,192, else a radix sort of 64-bit composite keys when the fields' ranges fit,
// else a stable LSD radix sort field by field (d, m, dCBO, dLCOM, n_improved
// desc) through a permutation.
void sort_kept_moves(mm_system *s, mm_move *kept, int64_t K) {
  cudaStream_t st = s->stream;
  if (K > 1 && K <= KEYED_MAX) {
    keyed_sort_launch(s, kept, nullptr, (int32_t)K, K, st);
  } else if (K > KEYED_MAX) {
    // the fields' actual ranges decide whether one 64-bit composite key holds them all
    int32_t *d_mm = reinterpret_cast<int32_t *>(s->d_u64 + 24);
    const int32_t init[6] = {INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN};
    MM_CUDA_TRY(cudaMemcpyAsync(d_mm, init, sizeof(init), cudaMemcpyHostToDevice, st));
    pdl_launch(kept_ranges, (unsigned)std::min<int64_t>(ceil_div(K, TPB), B300_SMS * 4), TPB, 0, st, kept, K, d_mm);
    MM_LAUNCH_CHECK();
    int32_t r[6];
    MM_CUDA_TRY(cudaMemcpyAsync(r, d_mm, sizeof(r), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaStreamSynchronize(st));
    const int w_d = bits_for((uint64_t)std::max(s->c - 1, 0)), w_m = bits_for((uint64_t)std::max(s->M - 1, 0));
    const int w_cbo = bits_for((uint64_t)((int64_t)r[5] - r[4])), w_ck = bits_for((uint64_t)((int64_t)r[3] - r[2]));
    const int w_n = bits_for((uint64_t)((int64_t)r[1] - r[0]));
    const int total = w_d + w_m + w_cbo + w_ck + w_n;
    if (total <= 64) {
      size_t kb = sizeof(uint64_t) * 2 * (size_t)K, pb = sizeof(uint32_t) * 2 * (size_t)K;
      char *base = static_cast<char *>(s->stage_ws.need(kb + pb + sizeof(mm_move) * (size_t)K + 512, st));
      uint64_t *key = reinterpret_cast<uint64_t *>(base), *key_alt = key + K;
      uint32_t *perm = reinterpret_cast<uint32_t *>(key_alt + K), *perm_alt = perm + K;
      mm_move *sorted = reinterpret_cast<mm_move *>((reinterpret_cast<uintptr_t>(perm_alt + K) + 15) & ~uintptr_t(15));
      KeyLayout kl;
      kl.nimp_max = r[1];
      kl.ck_min = r[2];
      kl.cbo_min = r[4];
      kl.s_m = w_d;
      kl.s_cbo = w_d + w_m;
      kl.s_ck = kl.s_cbo + w_cbo;
      kl.s_nimp = kl.s_ck + w_ck;
      pdl_launch(kept_keys, grid_for(K), TPB, 0, st, kept, K, kl, key, perm);
      MM_LAUNCH_CHECK();
      radix_sort_u64(key, key_alt, perm, perm_alt, K, total, s->sort_ws, st);
      pdl_launch(permute_moves, grid_for(K), TPB, 0, st, kept, perm, K, sorted);
      MM_LAUNCH_CHECK();
      MM_CUDA_TRY(cudaMemcpyAsync(kept, sorted, sizeof(mm_move) * (size_t)K, cudaMemcpyDeviceToDevice, st));
      return;
    }
    // else a permutation sort field by field, least significant first (d, m, dCBO, dLCOM, n_improved desc)
    size_t pb = sizeof(uint32_t) * 4 * (size_t)K;
    uint32_t *pw = static_cast<uint32_t *>(s->stage_ws.need(pb + sizeof(mm_move) * (size_t)K + 256, st));
    uint32_t *key = pw, *key_alt = pw + K, *perm = pw + 2 * K, *perm_alt = pw + 3 * K;
    mm_move *sorted = reinterpret_cast<mm_move *>(pw + 4 * K);
    pdl_launch(iota_perm, grid_for(K), TPB, 0, st, perm, K);
    MM_LAUNCH_CHECK();
    const int fbits[5] = {w_d, w_m, w_cbo, w_ck, w_n};
    const int64_t bias[5] = {0, 0, -(int64_t)r[4], -(int64_t)r[2], (int64_t)r[1]};
    for (int f = 0; f < 5; ++f) {
      pdl_launch(gather_field, grid_for(K), TPB, 0, st, kept, perm, K, f, bias[f], key);
      MM_LAUNCH_CHECK();
      radix_sort_u32(key, key_alt, perm, perm_alt, K, fbits[f], s->sort_ws, st);
    }
    pdl_launch(permute_moves, grid_for(K), TPB, 0, st, kept, perm, K, sorted);
    MM_LAUNCH_CHECK();
    MM_CUDA_TRY(cudaMemcpyAsync(kept, sorted, sizeof(mm_move) * (size_t)K, cudaMemcpyDeviceToDevice, st));
  }
}

void suggest_moves(mm_system *s, const mm_criteria &crit, const mm_candidates *cands, int32_t k, mm_move *out,
                   int32_t kind, int64_t *n_kept, int64_t *n_mk) {
  check_criteria(crit);
  if (k < 0) throw MmError{MM_EINVAL, "suggest: k < 0"};
  if (k > 0 && !out) throw MmError{MM_EINVAL, "suggest: out_topk is NULL"};
  if (kind != MM_PTR_HOST && kind != MM_PTR_DEVICE) throw MmError{MM_EINVAL, "suggest: bad out_kind"};
  cudaStream_t st = s->stream;
  const int64_t *rowptr;
  const int32_t *dst;
  int64_t n_cand;
  uint64_t chash = 0;
  prepare_candidates(s, cands, &rowptr, &dst, &n_cand, &chash);
  int64_t K = 0, nm = 0;
  mm_move *kept = nullptr;
  // Host outputs of up to KEYED_MAX kept moves need one round trip: the sort
  // (which checks the count on the device) and the copy of the first moves
  // are queued before the count is read back.
  const mm_move *staged = nullptr;  // the first moves, copied back with the counts
  int64_t nstaged = 0;
  bool sorted_early = false;
  if (n_cand > 0 && s->M > 0) {
    EvalCtx cx = make_ctx(s, crit);
    const bool same_cands = rowptr == nullptr ? !s->kept_lists
                                              : (s->kept_lists && s->kept_hash == chash && s->kept_ncand == n_cand);
    const bool reuse = s->kept_valid && same_cands && s->kept_mask == crit.metric_mask &&
                       s->kept_min == crit.min_improved;
    int64_t cap = reuse ? s->kept_cap : kept_capacity(s);
    if (!reuse) s->kept_valid = false;
    for (int attempt = 0; attempt < 3; ++attempt) {
      uint8_t *mark;
      kept_buffers(s, cap, &kept, &mark);
      if (!(reuse && attempt == 0)) {
        OutCtx oc{};
        attach_kept(s, oc, cap);
        dispatch_eval(s, cx, oc, rowptr, dst);
      }
      MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 2, 0, sizeof(unsigned long long), st));
      pdl_launch(count_marks, B300_SMS * 4, 256, 0, st, mark, s->M, s->d_u64 + 2);
      MM_LAUNCH_CHECK();
      // sorts the kept moves in place when 2 <= K <= min(cap, KEYED_MAX), else leaves them
      keyed_sort_launch(s, kept, s->d_u64 + 1, 0, cap, st);
      const int64_t nstage = kind == MM_PTR_HOST ? std::min<int64_t>({(int64_t)k, cap, (int64_t)KEYED_MAX}) : 0;
      // page-locked staging: {counts (2 x u64), fault flag, pad, moves}
      unsigned char *hb = static_cast<unsigned char *>(host_staging(32 + sizeof(mm_move) * (size_t)nstage));
      unsigned long long *hc = reinterpret_cast<unsigned long long *>(hb);
      uint32_t *hfault = reinterpret_cast<uint32_t *>(hb + 16);
      *hfault = 0;
      if (nstage > 0)
        MM_CUDA_TRY(cudaMemcpyAsync(hb + 32, kept, sizeof(mm_move) * (size_t)nstage, cudaMemcpyDeviceToHost, st));
      MM_CUDA_TRY(cudaMemcpyAsync(hc, s->d_u64 + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      read_wait_fault(hfault, s->d_fault, st);
      MM_CUDA_TRY(cudaStreamSynchronize(st));
      staged = reinterpret_cast<const mm_move *>(hb + 32);
      nstaged = nstage;
      raise_wait_fault(*hfault, s->d_fault, st, "suggest");
      K = (int64_t)hc[0];
      nm = (int64_t)hc[1];
      if (K <= cap) break;
      cap = K + K / 8 + 1024;  // grow and evaluate again
      s->kept_valid = false;
    }
    // the kept moves stay cached for these criteria and candidates
    s->kept_cap = std::max(s->kept_cap, cap);
    s->kept_valid = true;
    s->kept_mask = crit.metric_mask;
    s->kept_min = crit.min_improved;
    s->kept_lists = rowptr != nullptr;
    s->kept_hash = chash;
    s->kept_ncand = n_cand;
    sorted_early = K <= KEYED_MAX;
    if (!sorted_early) sort_kept_moves(s, kept, K);
  }
  const int64_t nout = std::min<int64_t>(k, K);
  if (nout > 0) {
    if (sorted_early && kind == MM_PTR_HOST && staged && nstaged >= nout) {
      std::memcpy(out, staged, sizeof(mm_move) * (size_t)nout);
      if (n_kept) *n_kept = K;
      if (n_mk) *n_mk = nm;
      return;
    }
    MM_CUDA_TRY(cudaMemcpyAsync(out, kept, sizeof(mm_move) * (size_t)nout,
                                kind == MM_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  }
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_kept) *n_kept = K;
  if (n_mk) *n_mk = nm;
}

// ---------------------------------------------------------------- helpers for the allocation-free entry point

// Evaluate the candidates (full cross product or device-resident lists) and
// compact the kept moves into caller-provided device buffers; allocates nothing.
// *count and mark[M] must be zero on entry.
void eval_kept_into(mm_system *s, const mm_criteria &crit, const mm_candidates *cands, mm_move *kept, int64_t cap,
                    unsigned long long *count, uint8_t *mark) {
  check_criteria(crit);
  if (cands && cands->rowptr && cands->ptr_kind != MM_PTR_DEVICE)
    throw MmError{MM_EINVAL, "candidate lists must be in device memory here"};
  const int64_t *rowptr;
  const int32_t *dst;
  int64_t n_cand;
  prepare_candidates(s, cands, &rowptr, &dst, &n_cand, nullptr, false);  // device lists only: nothing allocated
  if (n_cand == 0 || s->M == 0) return;
  EvalCtx cx = make_ctx(s, crit);
  OutCtx oc{};
  oc.kept = kept;
  oc.kept_count = count;
  oc.kept_cap = cap;
  oc.kept_mark = mark;
  dispatch_eval(s, cx, oc, rowptr, dst);
}

// Sort n kept moves in runs of 2,048 in place: one launch, block b sorts run b.
void sort_moves_chunks(mm_move *v, int64_t n, cudaStream_t st) {
  if (n <= 1) return;
  pdl_launch(bitonic_sort_chunks, (unsigned)ceil_div(n, BITONIC_MAX), 1024, 0, st, v, n);
  MM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- batched persistent evaluation

namespace {

struct BatchItem {
  DenseSys sy;
  OutCtx oc;
  int64_t tile0;  // first global tile index of this system
  int32_t gx;     // destination blocks of this system
  int32_t pad;
};

// One persistent launch over every system of a batch: blocks take
// (system, destination block, method chunk) tiles from a global counter and run
// the same dense_tile as the single-system kernel.
template <bool DIG, bool KEEP>
__global__ void __launch_bounds__(DB_THREADS, 4) eval_dense_batched(const BatchItem *items, int32_t n,
                                                                    int64_t total_tiles, int32_t mchunk,
                                                                    unsigned long long *next_tile) {
  __shared__ __align__(16) DenseStage st;
  __shared__ long long s_t;
  __shared__ __align__(16) BatchItem s_it;  // the current tile's system, read by every thread
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(next_tile, 1ull);
      s_t = t;
      if (t < total_tiles) {
        int32_t lo = 0, hi = n - 1;  // last item with tile0 <= t
        while (lo < hi) {
          int32_t mid = (lo + hi + 1) >> 1;
          if (items[mid].tile0 <= t) lo = mid; else hi = mid - 1;
        }
        s_it = items[lo];
      }
    }
    __syncthreads();
    const int64_t t = s_t;
    if (t >= total_tiles) break;
    const BatchItem &it = s_it;
    const int64_t local = t - it.tile0;
    const int32_t bx = (int32_t)(local % it.gx);
    const int32_t m0 = (int32_t)(local / it.gx) * mchunk;
    const int32_t m1 = min(it.sy.M, m0 + mchunk);
    uint64_t dig = dense_tile<false, DIG, KEEP>(it.sy, it.oc, st, bx, m0, m1);
    if (DIG) {
      for (int o = 16; o > 0; o >>= 1) dig += __shfl_down_sync(0xffffffffu, dig, o);
      if ((threadIdx.x & 31u) == 0 && dig) atomicAdd(it.oc.digest, (unsigned long long)dig);
    }
    __syncthreads();  // every thread is done with s_it / s_t before the next tile overwrites them
  }
}

}  // namespace

// Host side of the batched evaluation (see mm_batch.cu).
int64_t batch_tiles(const mm_system *s, int32_t mchunk) {
  if (s->M == 0 || s->c < 2) return 0;
  return ceil_div(s->c, DB_SPAN) * ceil_div(s->M, mchunk);
}

void batch_fill_items(const BatchLaunchSpec *specs, int32_t n, const mm_criteria &crit, int32_t mchunk,
                      int64_t kept_cap, void *items_host, int64_t *total_tiles) {
  BatchItem *items = static_cast<BatchItem *>(items_host);
  int64_t t = 0;
  for (int32_t i = 0; i < n; ++i) {
    mm_system *s = specs[i].sys;
    EvalCtx cx = make_ctx(s, crit);
    BatchItem &it = items[i];
    it.sy = DenseSys{cx, s->dest_rec, s->c, s->M};
    it.oc = OutCtx{};
    it.oc.digest = specs[i].digest;
    it.oc.kept = specs[i].kept;
    it.oc.kept_count = specs[i].kept_count;
    it.oc.kept_cap = kept_cap;
    it.oc.kept_mark = specs[i].kept_mark;
    it.tile0 = t;
    it.gx = (int32_t)std::max<int64_t>(1, ceil_div(s->c, DB_SPAN));
    it.pad = 0;
    t += batch_tiles(s, mchunk);
  }
  *total_tiles = t;
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

void batch_launch(const void *items_dev, int32_t n, int64_t total_tiles, int32_t mchunk, bool keep, bool digest,
                  unsigned long long *next_tile, int grid, cudaStream_t st) {
  if (total_tiles == 0) return;
  const BatchItem *items = static_cast<const BatchItem *>(items_dev);
  if (keep && digest)
    eval_dense_batched<true, true><<<grid, DB_THREADS, 0, st>>>(items, n, total_tiles, mchunk, next_tile);
  else if (keep)
    eval_dense_batched<false, true><<<grid, DB_THREADS, 0, st>>>(items, n, total_tiles, mchunk, next_tile);
  else if (digest)
    eval_dense_batched<true, false><<<grid, DB_THREADS, 0, st>>>(items, n, total_tiles, mchunk, next_tile);
  else
    eval_dense_batched<false, false><<<grid, DB_THREADS, 0, st>>>(items, n, total_tiles, mchunk, next_tile);
  MM_LAUNCH_CHECK();
}

int batch_persistent_grid() {
  int dev = 0, sms = B300_SMS, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_dense_batched<true, true>, DB_THREADS, 0);
  return sms * std::max(per_sm, 1);
}

void check_criteria_public(const mm_criteria &crit) { check_criteria(crit); }

// Sort every segment holding at most 2,048 moves (one block per segment).
void sort_moves_segments(mm_move *base, int64_t stride, const unsigned long long *counts, int32_t n,
                         cudaStream_t st) {
  if (n <= 0) return;
  bitonic_sort_segments<<<n, 1024, 0, st>>>(base, stride, counts);
  MM_LAUNCH_CHECK();
}

// Evaluate an internal (valid by construction) device candidate list and append
// the kept moves to the system's kept buffer (count and marks already set).
void eval_csr_kept_append(mm_system *s, const mm_criteria &crit, const int64_t *rowptr, const int32_t *dst,
                          mm_move *kept, int64_t cap, unsigned long long *count, uint8_t *mark) {
  EvalCtx cx = make_ctx(s, crit);
  OutCtx oc{};
  oc.kept = kept;
  oc.kept_count = count;
  oc.kept_cap = cap;
  oc.kept_mark = mark;
  dispatch_eval(s, cx, oc, rowptr, dst);
}

// Kept moves of the methods mlist[0..n) to every other class (the dense
// tiles over a method list), appended to a kept list.
void eval_dense_kept_subset(mm_system *s, const mm_criteria &crit, const int32_t *mlist, int32_t n, mm_move *kept,
                            int64_t cap, unsigned long long *count, uint8_t *mark) {
  if (n <= 0) return;
  ensure_adjacency(s);
  EvalCtx cx = make_ctx(s, crit);
  OutCtx oc{};
  oc.kept = kept;
  oc.kept_count = count;
  oc.kept_cap = cap;
  oc.kept_mark = mark;
  const int32_t c = s->c;
  const unsigned gx = (unsigned)ceil_div(c, DB_SPAN);
  const int64_t want_y = std::max<int64_t>(1, (B300_SMS * 3 * 30) / gx);
  const int32_t mchunk = (int32_t)std::max<int64_t>(1, ceil_div(n, want_y));
  const unsigned gy = (unsigned)ceil_div(n, mchunk);
  DenseSys sy{cx, s->dest_rec, c, n};
  sy.mlist = mlist;
  pdl_launch(eval_dense<false, false, true>, dim3(gx, gy), DB_THREADS, 0, s->stream, sy, oc, mchunk);
  MM_LAUNCH_CHECK();
}

// Records of internal (valid by construction) device candidate lists; the
// criteria only set the record's kept bit, so CBO alone, one improved, is used.
void eval_lists_records(mm_system *s, const int64_t *rowptr, const int32_t *dst, mm_move_eval *records) {
  const mm_criteria crit{4u, 1};
  EvalCtx cx = make_ctx(s, crit);
  OutCtx oc{};
  oc.records = reinterpret_cast<uint4 *>(records);
  dispatch_eval(s, cx, oc, rowptr, dst);
}

// The system's cached kept list (full cross product) for the edit path.
bool kept_cache(mm_system *s, mm_move **kept, uint8_t **mark, int64_t *cap) {
  if (!s->kept_valid) return false;
  kept_buffers(s, s->kept_cap, kept, mark);
  *cap = s->kept_cap;
  return true;
}
