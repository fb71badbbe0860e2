// Class metrics (Sec. II.B) on the device:
//   * inverted index of own accesses: attribute -> the methods of its class
//     that access it (only attributes owned by the class count);
//   * LCOM pair counts: the methods sharing an attribute with x are the union
//     of the accessor lists of x's own attributes, so q_x = |union| - 1 and
//     Q = sum q_x / 2, P = n(n-1)/2 - Q; the union is counted in a per-warp
//     bitmap over the class's method ranks.  Work is the sum over accesses of
//     the accessor-list length instead of n^2 word ANDs per class;
//   * coupling: every use edge (class of x, class it uses) as a 64-bit key,
//     segmented by source class with the radix sort, run-length encoded into
//     the class-use multigraph cnt[Y][E]; CBO(Y) = number of E != Y with
//     cnt > 0; out/in adjacency bitsets and their compressed two-level form
//     for the move evaluation's probes.
#include <cuda_runtime.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n, int tpb = TPB) {
  int64_t g = ceil_div(n, tpb);
  if (g < 1) g = 1;
  if (g > 0x7fffffffLL) g = 0x7fffffffLL;
  return (unsigned)g;
}

// ---------------------------------------------------------------- LCOM

// Inverted index of own accesses.  One thread per method: count its accesses
// to its own class's attributes per attribute; own_x = their number, S_C += own_x.
__global__ void own_access_count(const int32_t *method_class, const int64_t *acc_rowptr, const int32_t *acc_idx,
                                 const int32_t *attr_class, int32_t M, int64_t *acnt, int32_t *own,
                                 int64_t *cls_S) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  const int32_t C = method_class[x];
  int32_t cnt = 0;
  for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
    const int32_t al = acc_idx[e];
    if (attr_class[al] == C) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&acnt[al]), 1ull);
      ++cnt;
    }
  }
  own[x] = cnt;
  if (cnt) atomicAdd(reinterpret_cast<unsigned long long *>(&cls_S[C]), (unsigned long long)cnt);
}

// accessors of alpha (class-local method ranks) at own_list[own_ptr[alpha] ..], in any order
__global__ void own_access_fill(const int32_t *method_class, const int32_t *method_local, const int64_t *acc_rowptr,
                                const int32_t *acc_idx, const int32_t *attr_class, int32_t M,
                                const int64_t *own_ptr, int32_t *cursor, int32_t *own_list) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  const int32_t C = method_class[x], r = method_local[x];
  for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
    const int32_t al = acc_idx[e];
    if (attr_class[al] == C) own_list[own_ptr[al] + atomicAdd(&cursor[al], 1)] = r;
  }
}

// LCOM pair counts: q_x = methods of x's class sharing an own attribute with x
// = |union of the accessor lists of x's own attributes| - 1 (x itself), and
// sum_x q_x = 2 Q_C.  A warp owns g consecutive methods (one slot each) and
// walks their accesses, which are contiguous, 32 at a time: an own access of
// a method with one own attribute gives q directly (its list length - 1);
// those of methods with two or more have their accessor lists expanded
// across the lanes, and every accessor other than x goes into x's hash table
// of LU_TAB class-local ranks in shared memory (an insert that finds the rank
// already there adds nothing).  The distinct ranks per table are q_x.  A
// method whose table fills up, and every method of a listed subset (edits),
// takes the whole warp for a bitmap union over its class's method ranks
// (bitmap words per warp in shared memory, or in a zeroed global slice when
// the largest class is too big).
constexpr int LU_TAB = 32;
constexpr uint32_t LU_EMPTY = 0xffffffffu;
struct LcomWarp {
  uint32_t tab[32 * LU_TAB];  // per slot: open addressing, linear probing
  int64_t arp[33];            // access row bounds of the group's methods
  int32_t res[32];            // q + 1 of slots with one own attribute
  int32_t full[32];           // slot whose table filled up
};
constexpr size_t LU_WARP_BYTES = (sizeof(LcomWarp) + 15) / 16 * 16;
constexpr size_t LU_RESERVE = LU_WARP_BYTES * 8;  // per block of 8 warps

inline int lcom_group(int64_t M) {
  const int64_t per_warp = M / (B300_SMS * 64);
  return per_warp >= 32 ? 32 : (per_warp >= 16 ? 16 : 8);
}

__device__ __forceinline__ void lu_insert(uint32_t *tab, int32_t *full, int32_t slot, uint32_t j) {
  uint32_t h = (j * 2654435761u) >> 27;  // LU_TAB = 32 buckets
  for (int t = 0; t < LU_TAB; ++t) {
    const uint32_t old = atomicCAS(&tab[slot * LU_TAB + h], LU_EMPTY, j);
    if (old == LU_EMPTY || old == j) return;
    h = (h + 1u) & (LU_TAB - 1);
  }
  full[slot] = 1;
}

__global__ void __launch_bounds__(256) lcom_union(const int32_t *method_class, const int32_t *method_local,
                                                  const int64_t *acc_rowptr, const int32_t *acc_idx,
                                                  const int32_t *attr_class, const int64_t *own_ptr,
                                                  const int32_t *own_list, const int32_t *own, int32_t M,
                                                  int32_t words, uint32_t *gbm, int32_t *q, int64_t *cls_Q,
                                                  int32_t g, unsigned long long *next, const int32_t *mlist) {
  pdl_wait();
  extern __shared__ __align__(16) uint32_t lu_smem[];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  LcomWarp &lw = *reinterpret_cast<LcomWarp *>(reinterpret_cast<unsigned char *>(lu_smem) + wid * LU_WARP_BYTES);
  uint32_t *bm = gbm ? gbm + ((int64_t)blockIdx.x * nw + wid) * words
                     : reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(lu_smem) + nw * LU_WARP_BYTES) +
                           wid * words;
  if (!gbm)
    for (int32_t i = (int32_t)lane; i < words; i += 32) bm[i] = 0u;
  for (int32_t i = (int32_t)lane; i < 32 * LU_TAB; i += 32) lw.tab[i] = LU_EMPTY;
  lw.full[lane] = 0;
  __syncwarp();
  // warps take groups from a counter (unions differ widely in length)
  auto take = [&]() { return __shfl_sync(0xffffffffu, lane == 0 ? (int64_t)atomicAdd(next, 1ull) : (int64_t)0, 0); };
  for (int64_t wg = take(); wg * g < M; wg = take()) {
    const int64_t base = wg * g, pos = base + lane;
    const int32_t nm = (int32_t)min((int64_t)g, (int64_t)M - base);
    const bool mine = (int32_t)lane < nm;
    // with mlist the methods are mlist[0 .. M) (members of the classes an edit changed)
    const int64_t x = mine && mlist ? (int64_t)mlist[pos] : pos;
    const int32_t ox = mine ? own[x] : 0;
    const int32_t C = mine ? method_class[x] : -1;
    int32_t u = 0;
    bool over = false;
    if (mlist) {
      if (ox == 1) {
        for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
          const int32_t al = acc_idx[e];
          if (attr_class[al] == C) {
            u = (int32_t)(own_ptr[al + 1] - own_ptr[al]);
            break;
          }
        }
      }
      over = ox >= 2;
    } else {
      const int32_t r = mine ? method_local[x] : -1;
      if ((int32_t)lane <= nm) lw.arp[lane] = acc_rowptr[base + lane];
      if (lane == 0 && nm == 32) lw.arp[32] = acc_rowptr[base + 32];
      __syncwarp();
      const int64_t a_hi = lw.arp[nm];
      for (int64_t e0 = lw.arp[0]; e0 < a_hi; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool v = e < a_hi;
        int32_t sl = 0;  // slot of access e: the last with arp[sl] <= e
        if (v) {
          int32_t lo = 0, hi = nm - 1;
          while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (lw.arp[mid] <= e) lo = mid; else hi = mid - 1;
          }
          sl = lo;
        }
        const int32_t Cs = __shfl_sync(0xffffffffu, C, sl), oxs = __shfl_sync(0xffffffffu, ox, sl);
        const int32_t rs = __shfl_sync(0xffffffffu, r, sl);
        const int32_t al = v && oxs > 0 ? acc_idx[e] : 0;
        const bool ow = v && oxs > 0 && attr_class[al] == Cs;
        int64_t p0 = 0;
        int32_t n = 0;
        if (ow) {
          p0 = own_ptr[al];
          n = (int32_t)(own_ptr[al + 1] - p0);
          if (oxs == 1) lw.res[sl] = n;
        }
        if (oxs < 2) n = 0;
        // the n accessors of each lane's attribute, 32 at a time across the warp
        int32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if ((int)lane >= o) incl += t;
        }
        const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (int32_t k0 = 0; k0 < total; k0 += 32) {
          const int32_t k = k0 + (int32_t)lane;
          int32_t lo = 0, hi = 31;  // lane holding element k: the first whose inclusive count exceeds k
#pragma unroll
          for (int step = 0; step < 5; ++step) {
            const int32_t mid = (lo + hi) >> 1;
            const int32_t pm = __shfl_sync(0xffffffffu, incl, mid);
            if (pm > k) hi = mid; else lo = mid + 1;
          }
          const int32_t excl = __shfl_sync(0xffffffffu, incl, lo) - __shfl_sync(0xffffffffu, n, lo);
          const int64_t pb = __shfl_sync(0xffffffffu, p0, lo);
          const int32_t ss = __shfl_sync(0xffffffffu, sl, lo), rr = __shfl_sync(0xffffffffu, rs, lo);
          if (k < total) {
            const int32_t j = own_list[pb + (k - excl)];
            if (j != rr) lu_insert(lw.tab, lw.full, ss, (uint32_t)j);
          }
        }
      }
      __syncwarp();
      if (ox == 1) u = lw.res[lane];
      if (ox >= 2) {
        int32_t cnt = 0;
#pragma unroll 8
        for (int t = 0; t < LU_TAB; ++t)  // skewed: lane l reads bank (t + l) mod 32
          cnt += lw.tab[lane * LU_TAB + ((t + (int)lane) & (LU_TAB - 1))] != LU_EMPTY;
        u = cnt + 1;
        over = lw.full[lane] != 0;
      }
      __syncwarp();
      for (int32_t i = (int32_t)lane; i < 32 * LU_TAB; i += 32) lw.tab[i] = LU_EMPTY;
      lw.full[lane] = 0;
      __syncwarp();
    }
    uint32_t multi = __ballot_sync(0xffffffffu, over);
    while (multi) {
      const int src = __ffs(multi) - 1;
      multi &= multi - 1u;
      const int64_t xs = __shfl_sync(0xffffffffu, x, src);  // method of lane src
      const int32_t Cs = __shfl_sync(0xffffffffu, C, src);
      const int64_t a0 = acc_rowptr[xs];
      const int32_t v = accessor_union(acc_idx + a0, acc_rowptr[xs + 1] - a0, Cs, attr_class, own_ptr, own_list,
                                       bm, lane);
      if ((int)lane == src) u = v;
    }
    if (mine) {
      const int32_t qx = u > 0 ? u - 1 : 0;
      q[x] = qx;
      if (qx) atomicAdd(reinterpret_cast<unsigned long long *>(&cls_Q[C]), (unsigned long long)qx);
    }
  }
}

// the members of up to two classes (counts n0, n1 known to the caller), one list
__global__ void class_members_list(const int32_t *cm_list, const int64_t *cm_rowptr, int32_t C0, int64_t n0,
                                   int32_t C1, int64_t n1, int32_t *out) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0 + n1; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < n0 ? cm_list[cm_rowptr[C0] + i] : cm_list[cm_rowptr[C1] + (i - n0)];
}

// P and Q of up to two classes whose pair counts were recomputed
__global__ void finalize_listed(const int32_t *cls_n, int64_t *cls_Q, int64_t *cls_P, int32_t C0, int32_t C1, int ncls) {
  pdl_wait();
  const int k = (int)threadIdx.x;
  if (k >= ncls) return;
  const int32_t C = k == 0 ? C0 : C1;
  const int64_t n = cls_n[C];
  const int64_t Q = cls_Q[C] / 2;
  cls_Q[C] = Q;
  cls_P[C] = n * (n - 1) / 2 - Q;
}

__global__ void finalize_classes(const int32_t *cls_n, int64_t *cls_Q, int32_t c, int64_t *cls_P) {
  pdl_wait();
  int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= c) return;
  const int64_t n = cls_n[C];
  const int64_t Q = cls_Q[C] / 2;  // each sharing pair was counted from both of its methods
  cls_Q[C] = Q;
  cls_P[C] = n * (n - 1) / 2 - Q;
}

// ---------------------------------------------------------------- coupling

// Class-use multigraph without a sort.  Pass 1: every use edge (Y = class of
// x, E = class it uses, E != Y) sets bit E of Y's out-row and the summary bit
// of that word (already-set bits are only read).
__device__ __forceinline__ void mark_use(uint32_t *out_adj, uint2 *csum, int64_t aw, int64_t sw, int32_t Y,
                                         int32_t E) {
  uint32_t *w = &out_adj[(int64_t)Y * aw + (E >> 5)];
  const uint32_t bit = 1u << (E & 31);
  if (!(*w & bit)) atomicOr(w, bit);
  uint32_t *r = &csum[(int64_t)Y * sw + (E >> 10)].x;
  const uint32_t rbit = 1u << ((E >> 5) & 31);
  if (!(*r & rbit)) atomicOr(r, rbit);
}

__global__ void coupling_mark(const int32_t *method_class, const int64_t *call_rowptr, const int32_t *call_idx,
                              const int64_t *acc_rowptr, const int32_t *acc_idx, const int32_t *attr_class,
                              int32_t M, int32_t cbo_attrs, uint32_t *out_adj, int64_t aw, uint2 *csum,
                              int64_t sw, uint64_t *edges) {
  pdl_wait();
  int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  const int32_t Y = method_class[x];
  // edge keys (Y << 32 | E, or ~0 inside the class) at the method's calls, then its accesses
  int64_t pos = call_rowptr[x] + (cbo_attrs ? acc_rowptr[x] : 0);
  for (int64_t e = call_rowptr[x]; e < call_rowptr[x + 1]; ++e) {
    const int32_t E = method_class[call_idx[e]];
    if (E != Y) mark_use(out_adj, csum, aw, sw, Y, E);
    edges[pos++] = E != Y ? ((uint64_t)(uint32_t)Y << 32) | (uint32_t)E : ~0ull;
  }
  if (cbo_attrs)
    for (int64_t e = acc_rowptr[x]; e < acc_rowptr[x + 1]; ++e) {
      const int32_t E = attr_class[acc_idx[e]];
      if (E != Y) mark_use(out_adj, csum, aw, sw, Y, E);
      edges[pos++] = E != Y ? ((uint64_t)(uint32_t)Y << 32) | (uint32_t)E : ~0ull;
    }
}

// Classes marked in the full words that summary record k of out-row Y marks.
__device__ __forceinline__ int32_t record_classes(const uint2 *csum, const uint32_t *out_adj, int64_t aw,
                                                  int64_t sw, int32_t Y, int64_t k) {
  uint32_t bits = csum[(int64_t)Y * sw + k].x;
  int32_t n = 0;
  while (bits) {
    const int j = __ffs(bits) - 1;
    bits &= bits - 1u;
    n += __popc(out_adj[(int64_t)Y * aw + k * 32 + j]);
  }
  return n;
}

// Pass 2: CBO(Y) = number of marked classes of out-row Y (warp per row,
// lanes over its summary records).
// Rows of at most this many words (8,192 classes) are walked word by word with
// every lane busy; longer rows through their summary records.
constexpr int64_t ROW_WORDS_DIRECT = 256;

__global__ void row_distinct(const uint2 *csum, const uint32_t *out_adj, int32_t c, int64_t aw, int64_t sw,
                             int32_t *row_count) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t Y = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; Y < c; Y += nwarps) {
    int32_t n = 0;
    if (aw <= ROW_WORDS_DIRECT)  // short rows: lanes over the words themselves
      for (int64_t k = lane; k < aw; k += 32) n += __popc(out_adj[Y * aw + k]);
    else  // long rows: lanes over the summary records, only marked words read
      for (int64_t k = lane; k < sw; k += 32) n += record_classes(csum, out_adj, aw, sw, (int32_t)Y, k);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) row_count[Y] = n;
  }
}

// Pass 3: write each out-row's classes in ascending order at mg_rowptr[Y]
// (lane k owns record k; records ascend with the lane), zero their counts, and
// set the transposed in-row bits and their summary bits.
__global__ void row_enumerate(uint2 *csum, const uint32_t *out_adj, uint32_t *in_adj, int32_t c, int64_t aw,
                              int64_t sw, const int64_t *mg_rowptr, int32_t *mg_dst, int32_t *mg_cnt) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t Y = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; Y < c; Y += nwarps) {
    int64_t pos = mg_rowptr[Y];
    if (aw <= ROW_WORDS_DIRECT) {  // lane per word: ascending words, ascending bits within a word
      for (int64_t k0 = 0; k0 < aw; k0 += 32) {
        const int64_t wi = k0 + lane;
        uint32_t word = wi < aw ? out_adj[Y * aw + wi] : 0u;
        const int32_t n = __popc(word);
        int32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if ((int)lane >= o) incl += t;
        }
        int64_t p = pos + incl - n;
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1u;
          const int32_t E = (int32_t)(wi * 32 + b);
          mg_dst[p] = E;
          mg_cnt[p] = 0;
          ++p;
          atomicOr(&in_adj[(int64_t)E * aw + (Y >> 5)], 1u << (Y & 31));
          atomicOr(&csum[((int64_t)c + E) * sw + (Y >> 10)].x, 1u << ((Y >> 5) & 31));
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
      }
      continue;
    }
    for (int64_t k0 = 0; k0 < sw; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t n = k < sw ? record_classes(csum, out_adj, aw, sw, (int32_t)Y, k) : 0;
      int32_t incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
      }
      int64_t p = pos + incl - n;
      if (n) {
        uint32_t bits = csum[Y * sw + k].x;
        while (bits) {
          const int j = __ffs(bits) - 1;
          bits &= bits - 1u;
          const int64_t wi = k * 32 + j;
          uint32_t word = out_adj[Y * aw + wi];
          while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            const int32_t E = (int32_t)(wi * 32 + b);
            mg_dst[p] = E;
            mg_cnt[p] = 0;
            ++p;
            atomicOr(&in_adj[(int64_t)E * aw + (Y >> 5)], 1u << (Y & 31));
            atomicOr(&csum[((int64_t)c + E) * sw + (Y >> 10)].x, 1u << ((Y >> 5) & 31));
          }
        }
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// Pass 4: multiplicities cnt[Y][E] = number of use edges, one thread per edge
// (binary search of E in row Y).
__global__ void coupling_count(const uint64_t *edges, int64_t n, const int64_t *mg_rowptr, const int32_t *mg_dst,
                               int32_t *mg_cnt) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = edges[i];
    if (k == ~0ull) continue;
    const int32_t Y = (int32_t)(k >> 32), E = (int32_t)(uint32_t)k;
    int64_t lo = mg_rowptr[Y], hi = mg_rowptr[Y + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (mg_dst[mid] < E) lo = mid + 1; else hi = mid;
    }
    atomicAdd(&mg_cnt[lo], 1);
  }
}

// the same from the packed rows: E's position in out-row Y is the row position
// of its packed word plus the bits below E in that word
__global__ void coupling_count_packed(const uint64_t *__restrict__ edges, int64_t n,
                                      const int64_t *__restrict__ mg_rowptr, const uint2 *__restrict__ csum,
                                      const uint32_t *__restrict__ cpk, const int32_t *__restrict__ wrank, int64_t sw,
                                      int32_t *__restrict__ mg_cnt) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = edges[i];
    if (k == ~0ull) continue;
    const int32_t Y = (int32_t)(k >> 32), E = (int32_t)(uint32_t)k;
    const int64_t row0 = mg_rowptr[Y];
    const uint2 rec = csum[(int64_t)Y * sw + (E >> 10)];
    const uint32_t widx = rec.y + __popc(rec.x & ((1u << ((E >> 5) & 31)) - 1u));
    const int32_t rank = wrank[widx] + __popc(cpk[widx] & ((1u << (E & 31)) - 1u));
    atomicAdd(&mg_cnt[row0 + rank], 1);
  }
}

__global__ void summary_popc(const uint2 *sum, int64_t n, int32_t *cnt) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = __popc(sum[i].x);
}

// record i gets the packed index of its first word; its marked full words are
// copied there (rows below c from the out-bitsets, the next c from the in-bitsets)
__global__ void summary_pack(uint2 *sum, const int64_t *first, const uint32_t *out_adj, const uint32_t *in_adj,
                             int64_t c, int64_t aw, int64_t sw, int64_t n, uint32_t *packed) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / sw, k = i % sw;
    uint32_t bits = sum[i].x;
    const uint32_t f = (uint32_t)first[i];
    sum[i].y = f;
    const uint32_t *row = r < c ? out_adj + r * aw : in_adj + (r - c) * aw;
    uint32_t o = f;
    while (bits) {
      const int j = __ffs(bits) - 1;
      bits &= bits - 1;
      packed[o++] = row[k * 32 + j];
    }
  }
}

// ---------------------------------------------------------------- coupling without the full bitsets
//
// For systems whose full adjacency bitsets would be large, the compressed
// adjacency is built from the use edges themselves and the multigraph is read
// off it: every edge (Y, E), E != Y, sets the summary bits of its out-row
// record (Y, E >> 10) and in-row record (c + E, Y >> 10); the records' first
// packed indices follow by a scan of their popcounts, and each edge ORs its
// bit into the packed word its record points at (a repeated edge sets the
// same bit).  The packed words of an out-row hold its classes in ascending
// order, so counting and enumerating them gives the multigraph rows; the
// multiplicities are counted per edge as in the bitset form.  The full
// bitsets are built from the multigraph rows only when a dense evaluation
// asks for them.

__device__ __forceinline__ void mark_summary(uint2 *csum, int64_t sw, int64_t row, int32_t col) {
  uint32_t *r = &csum[row * sw + (col >> 10)].x;
  const uint32_t bit = 1u << ((col >> 5) & 31);
  if (!(*r & bit)) atomicOr(r, bit);
}

// edge keys (Y << 32 | E, or ~0 inside the class) at the method's calls, then
// its accesses, and the summary bits of both rows of every coupling edge
__global__ void coupling_keys(const int32_t *__restrict__ method_class, const int64_t *__restrict__ call_rowptr,
                              const int32_t *__restrict__ call_idx, const int64_t *__restrict__ acc_rowptr,
                              const int32_t *__restrict__ acc_idx, const int32_t *__restrict__ attr_class, int32_t M,
                              int32_t c, int32_t cbo_attrs, uint2 *__restrict__ csum, int64_t sw,
                              uint64_t *__restrict__ edges) {
  pdl_wait();
  // a warp per 32 methods: their edges are one contiguous range (coalesced
  // index loads and key stores)
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < M; w += nwarps) {
    const int64_t x0 = w * 32;
    const int32_t nm = (int32_t)min((int64_t)32, (int64_t)M - x0);
    const UseGroup u = use_group(call_rowptr, acc_rowptr, cbo_attrs != 0, x0, nm, lane);
    const int32_t Yl = (int32_t)lane < nm ? method_class[x0 + lane] : 0;
    for (int64_t p0 = u.s0; p0 < u.s1; p0 += 32) {
      const int64_t p = p0 + lane;
      int32_t slot;
      bool is_call;
      int64_t idx;
      use_edge_at(u, p, nm, slot, is_call, idx);
      const int32_t Y = __shfl_sync(0xffffffffu, Yl, slot);
      if (p < u.s1) {
        const int32_t E = is_call ? method_class[call_idx[idx]] : attr_class[acc_idx[idx]];
        if (E != Y) {
          mark_summary(csum, sw, Y, E);
          mark_summary(csum, sw, (int64_t)c + E, Y);
          edges[p] = ((uint64_t)(uint32_t)Y << 32) | (uint32_t)E;
        } else {
          edges[p] = ~0ull;
        }
      }
    }
  }
}

__device__ __forceinline__ void pack_bit(const uint2 *csum, int64_t sw, int64_t row, int32_t col, uint32_t *cpk) {
  const uint2 rec = csum[row * sw + (col >> 10)];
  const uint32_t b = ((uint32_t)col >> 5) & 31u;
  atomicOr(&cpk[rec.y + __popc(rec.x & ((1u << b) - 1u))], 1u << (col & 31));
}

// every edge's bit in the packed words of its out-row and in-row
__global__ void coupling_pack(const uint64_t *edges, int64_t n, int32_t c, const uint2 *csum, int64_t sw,
                              uint32_t *cpk) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = edges[i];
    if (k == ~0ull) continue;
    const int32_t Y = (int32_t)(k >> 32), E = (int32_t)(uint32_t)k;
    pack_bit(csum, sw, Y, E, cpk);
    pack_bit(csum, sw, (int64_t)c + E, Y, cpk);
  }
}

// CBO(Y) = classes in out-row Y = the bits of its packed words, which lie
// between its first record's index and the next row's (warp per row)
__global__ void packed_row_counts(const uint2 *csum, const uint32_t *cpk, int32_t c, int64_t sw, int32_t *row_count) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t Y = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; Y < c; Y += nwarps) {
    const uint32_t w0 = csum[Y * sw].y, w1 = csum[(Y + 1) * sw].y;
    int32_t n = 0;
    for (uint32_t w = w0 + lane; w < w1; w += 32) n += __popc(cpk[w]);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) row_count[Y] = n;
  }
}

// the classes of out-row Y in ascending order at mg_rowptr[Y], counts zeroed
// (warp per row, lane per summary record; records ascend with the lane)
__global__ void packed_row_enumerate(const uint2 *csum, const uint32_t *cpk, int32_t c, int64_t sw,
                                     const int64_t *mg_rowptr, int32_t *mg_dst, int32_t *mg_cnt, int32_t *wrank) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t Y = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; Y < c; Y += nwarps) {
    const int64_t row0 = mg_rowptr[Y];
    int64_t pos = row0;
    for (int64_t k0 = 0; k0 < sw; k0 += 32) {
      const int64_t k = k0 + lane;
      uint2 rec = make_uint2(0u, 0u);
      int32_t n = 0;
      if (k < sw) {
        rec = csum[Y * sw + k];
        const int32_t nw = __popc(rec.x);
        for (int32_t j = 0; j < nw; ++j) n += __popc(cpk[rec.y + j]);
      }
      int32_t incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
      }
      int64_t p = pos + incl - n;
      uint32_t bits = rec.x;
      for (uint32_t idx = rec.y; bits; ++idx) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1u;
        uint32_t word = cpk[idx];
        wrank[idx] = (int32_t)(p - row0);  // position of the word's first class in the row
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1u;
          mg_dst[p] = (int32_t)(((k * 32 + j) << 5) + b);
          mg_cnt[p] = 0;
          ++p;
        }
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// full bitsets from the multigraph rows: bit E of out-row Y and bit Y of in-row E
__global__ void adjacency_from_rows(const int64_t *mg_rowptr, const int32_t *mg_dst, int32_t c, int64_t aw,
                                    uint32_t *out_adj, uint32_t *in_adj) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t Y = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; Y < c; Y += nwarps)
    for (int64_t k = mg_rowptr[Y] + lane; k < mg_rowptr[Y + 1]; k += 32) {
      const int32_t E = mg_dst[k];
      atomicOr(&out_adj[Y * aw + (E >> 5)], 1u << (E & 31));
      atomicOr(&in_adj[(int64_t)E * aw + (Y >> 5)], 1u << (Y & 31));
    }
}

// destination record: {P - Q, S} as int64 in the first int4; {n, a, dck0, sck0 | shs0 << 8}
// in the second, where the last three are D's LCOM outcome when m shares nothing with D
__global__ void destination_records(const int32_t *cls_n, const int32_t *cls_a, const int64_t *P, const int64_t *Q,
                                    const int64_t *S, int32_t c, int4 *rec) {
  pdl_wait();
  int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= c) return;
  const int64_t d = P[C] - Q[C], sv = S[C];
  const int32_t n = cls_n[C], a = cls_a[C];
  const int64_t ck = d > 0 ? d : 0, d2 = d + n, ck2 = d2 > 0 ? d2 : 0;
  const int32_t sck0 = (ck2 > ck) - (ck2 < ck);
  const int32_t shs0 = a == 0 ? 0 : (n == 0 ? 1 : (sv > 0 ? 1 : 0));
  rec[2 * C] = make_int4((int32_t)(uint32_t)d, (int32_t)(d >> 32), (int32_t)(uint32_t)sv, (int32_t)(sv >> 32));
  rec[2 * C + 1] = make_int4(n, a, (int32_t)(ck2 - ck), (sck0 & 0xff) | ((shs0 & 0xff) << 8));
}

}  // namespace

UnionBitmap union_bitmap(mm_system *s, int64_t warps_wanted, Scratch &ws, cudaStream_t st, size_t reserve) {
  UnionBitmap ub;
  ub.words = (int32_t)std::max<int64_t>(1, ceil_div(std::max(s->summary.max_class_methods, 1), 32));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps_wanted, 8), B300_SMS * 8));
  ub.grid = (unsigned)blocks;
  const size_t per_block = (size_t)ub.words * 8 * sizeof(uint32_t);
  if (per_block + reserve <= 48 * 1024) {
    ub.smem = per_block + reserve;
    ub.gbm = nullptr;
  } else {
    ub.smem = reserve;
    const size_t bytes = per_block * (size_t)blocks;
    ub.gbm = static_cast<uint32_t *>(ws.need(bytes, st));
    MM_CUDA_TRY(cudaMemsetAsync(ub.gbm, 0, bytes, st));
  }
  return ub;
}

namespace {
// Side streams of one host thread on one device; destroyed with the thread
// (errors ignored: at process exit the runtime may already be gone).
struct SideStreams {
  int device = -1;
  cudaStream_t s[4] = {nullptr, nullptr, nullptr, nullptr};  // [0..2] metric branches, [3] list copies
  ~SideStreams() {
    for (cudaStream_t &x : s)
      if (x) {
        cudaSetDevice(device);
        cudaStreamDestroy(x);
        x = nullptr;
      }
  }
};
thread_local SideStreams tl_side[8];
}  // namespace

cudaStream_t fork_side(mm_system *s, int i) {
  if (!s->fork_ev || s->device < 0 || s->device >= 8) return s->stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MM_CUDA_TRY(cudaStreamIsCapturing(s->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return s->stream;
  SideStreams &ss = tl_side[s->device];
  ss.device = s->device;
  if (!ss.s[i]) MM_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s[i], cudaStreamNonBlocking));
  MM_CUDA_TRY(cudaEventRecord(s->fork_ev, s->stream));
  MM_CUDA_TRY(cudaStreamWaitEvent(ss.s[i], s->fork_ev, 0));
  return ss.s[i];
}

void join_side(mm_system *s, int i, cudaStream_t branch) {
  if (branch == s->stream) return;
  MM_CUDA_TRY(cudaEventRecord(s->join_ev[i], branch));
  MM_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->join_ev[i], 0));
}

void mark_point(mm_system *s, int k, cudaStream_t from) {
  if (s->mid_ev[k]) MM_CUDA_TRY(cudaEventRecord(s->mid_ev[k], from));
}

void wait_point(mm_system *s, int k, cudaStream_t from, cudaStream_t to) {
  if (from != to && s->mid_ev[k]) MM_CUDA_TRY(cudaStreamWaitEvent(to, s->mid_ev[k], 0));
}

void build_metrics(mm_system *s, bool lcom, bool coupling, const LcomClasses *only) {
  cudaStream_t st = s->stream;
  const int32_t c = s->c, M = s->M;

  // branch A (side stream 0): inverted index of own accesses, own, S, LCOM pair
  // counts, P and Q, destination records; lists L and R (side streams 1 and 2,
  // finished by build_move_precompute); branch B (below, on the system's
  // stream): coupling and the adjacency structures.  They share no buffer.
  // An edit that leaves LCOM (or the coupling) unchanged skips its branch: the
  // structures it built stay as they are, and the points the lists wait for
  // were passed long ago.
  if (!lcom) s->side_pending[0] = st;
  if (lcom) {
    cudaStream_t sa = fork_side(s, 0);
    Scratch &ev = s->side_eval[0];  // own scratch whether or not the branch runs concurrently
    Scratch &sw_ = s->side_sort[0];
    Scratch &uw = s->side_union[0];
    const int64_t A = s->A;
    const int64_t nl = only ? only->members[0] + (only->n > 1 ? only->members[1] : 0) : M;
    const size_t acnt_bytes = (sizeof(int64_t) * ((size_t)A + 1) + 255) & ~size_t(255);
    // per-attribute counts, then (edits) the listed classes' members
    char *evb = static_cast<char *>(ev.need(acnt_bytes + (only ? sizeof(int32_t) * (size_t)nl + 256 : 0), sa));
    int64_t *acnt = reinterpret_cast<int64_t *>(evb);
    MM_CUDA_TRY(cudaMemsetAsync(acnt, 0, sizeof(int64_t) * ((size_t)A + 1), sa));
    MM_CUDA_TRY(cudaMemsetAsync(s->cls_S, 0, sizeof(int64_t) * (size_t)c, sa));
    if (only) {  // the pair counts of the listed classes only; the others stay
      for (int k = 0; k < only->n; ++k)
        MM_CUDA_TRY(cudaMemsetAsync(s->cls_Q + only->cls[k], 0, sizeof(int64_t), sa));
    } else {
      MM_CUDA_TRY(cudaMemsetAsync(s->cls_Q, 0, sizeof(int64_t) * (size_t)c, sa));
      MM_CUDA_TRY(cudaMemsetAsync(s->q, 0, sizeof(int32_t) * (size_t)std::max(M, 1), sa));
    }
    if (M > 0) {
      pdl_launch(own_access_count, grid_for(M), TPB, 0, sa, s->method_class, s->acc_rowptr, s->acc_idx, s->attr_class, M,
                                                     acnt, s->own, s->cls_S);
      MM_LAUNCH_CHECK();
    }
    scan_exclusive_i64(acnt, s->own_ptr, A, s->own_ptr + A, sw_, sa);
    if (M > 0 && A > 0) {
      int32_t *cursor = reinterpret_cast<int32_t *>(acnt);  // counts are consumed: reuse as cursors
      MM_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)A, sa));
      pdl_launch(own_access_fill, grid_for(M), TPB, 0, sa, s->method_class, s->method_local, s->acc_rowptr, s->acc_idx,
                                                    s->attr_class, M, s->own_ptr, cursor, s->own_list);
      MM_LAUNCH_CHECK();
    }
    mark_point(s, 1, sa);  // own-access lists built (the s of list L entries needs them)
    if (nl > 0 && A > 0) {
      // LCOM pair counts from accessor unions (all methods, or the listed classes' members)
      const int32_t *mlist = nullptr;
      if (only) {
        int32_t *ml = reinterpret_cast<int32_t *>(evb + acnt_bytes);
        pdl_launch(class_members_list, grid_for(nl), TPB, 0, sa, static_cast<const int32_t *>(s->cm_list),
                   static_cast<const int64_t *>(s->cm_rowptr), only->cls[0], only->members[0],
                   only->n > 1 ? only->cls[1] : only->cls[0], only->n > 1 ? only->members[1] : (int64_t)0, ml);
        MM_LAUNCH_CHECK();
        mlist = ml;
      }
      const int g = lcom_group(nl);
      const UnionBitmap ub = union_bitmap(s, ceil_div(nl, g), uw, sa, LU_RESERVE);
      MM_CUDA_TRY(cudaMemsetAsync(s->d_u64 + 8, 0, sizeof(unsigned long long), sa));
      pdl_launch(lcom_union, ub.grid, 256, ub.smem, sa, s->method_class, s->method_local, s->acc_rowptr, s->acc_idx,
                 s->attr_class, s->own_ptr, s->own_list, s->own, (int32_t)nl, ub.words, ub.gbm, s->q, s->cls_Q, g,
                 s->d_u64 + 8, mlist);
      MM_LAUNCH_CHECK();
    }
    if (only) {
      pdl_launch(finalize_listed, 1, 32, 0, sa, static_cast<const int32_t *>(s->cls_n), s->cls_Q, s->cls_P, only->cls[0],
                 only->n > 1 ? only->cls[1] : only->cls[0], only->n);
    } else {
      pdl_launch(finalize_classes, grid_for(c), TPB, 0, sa, s->cls_n, s->cls_Q, c, s->cls_P);
    }
    MM_LAUNCH_CHECK();
    pdl_launch(destination_records, grid_for(c), TPB, 0, sa, s->cls_n, s->cls_a, s->cls_P, s->cls_Q, s->cls_S, c,
                                                     s->dest_rec);
    MM_LAUNCH_CHECK();
    s->side_pending[0] = sa;
  }
  // lists L and R (first half) on side streams 1 and 2
  begin_move_lists(s);

  const int64_t aw = s->adj_words, sw = s->sum_words;
  const int64_t ns = sw * (2 * (int64_t)c + 1);  // summary records: out-rows, in-rows, the zero row
  int32_t *row_count = s->cls_cbo;
  const int64_t nk = s->n_call + (s->cbo_attrs ? s->n_acc : 0);
  if (!coupling) {
    join_side(s, 0, s->side_pending[0]);
    return;
  }
  if (s->packed_coupling) {
    // coupling from the use edges through the compressed rows; the full
    // bitsets wait for a dense evaluation
    s->adj_built = false;
    Carve cv{static_cast<char *>(s->eval_ws.need(
        256 + sizeof(uint64_t) * (size_t)std::max<int64_t>(nk, 1), st))};
    uint64_t *edges = cv.take<uint64_t>(nk);
    int32_t *wrank = s->wrank;  // out-rows hold at most nk <= n_call + n_acc packed words
    zero_buffers(s->csum, sizeof(uint2) * (size_t)ns, s->cpk, sizeof(uint32_t) * 2 * (size_t)nk, nullptr, 0, st);
    if (M > 0) {
      pdl_launch(coupling_keys, (unsigned)std::min<int64_t>(ceil_div(M, 256), B300_SMS * 16), TPB, 0, st,
                 s->method_class, s->call_rowptr, s->call_idx, s->acc_rowptr,
                 s->acc_idx, s->attr_class, M, c, s->cbo_attrs, s->csum, sw, edges);
      MM_LAUNCH_CHECK();
    }
    scan_summary_first(s->csum, ns, s->sort_ws, st);
    const unsigned grow = (unsigned)std::min<int64_t>(ceil_div((int64_t)c * 32, TPB), B300_SMS * 16);
    if (nk > 0) {
      const unsigned gk = (unsigned)std::min<int64_t>(ceil_div(nk, TPB), B300_SMS * 16);
      pdl_launch(coupling_pack, gk, TPB, 0, st, static_cast<const uint64_t *>(edges), nk, c,
                 static_cast<const uint2 *>(s->csum), sw, s->cpk);
      MM_LAUNCH_CHECK();
    }
    pdl_launch(packed_row_counts, grow, TPB, 0, st, static_cast<const uint2 *>(s->csum),
               static_cast<const uint32_t *>(s->cpk), c, sw, row_count);
    MM_LAUNCH_CHECK();
    scan_exclusive_i32to64(row_count, s->mg_rowptr, c, s->sort_ws, st, s->mg_rowptr + c);
    pdl_launch(packed_row_enumerate, grow, TPB, 0, st, static_cast<const uint2 *>(s->csum),
               static_cast<const uint32_t *>(s->cpk), c, sw, static_cast<const int64_t *>(s->mg_rowptr), s->mg_dst,
               s->mg_cnt, wrank);
    MM_LAUNCH_CHECK();
    if (nk > 0) {
      pdl_launch(coupling_count_packed, (unsigned)std::min<int64_t>(ceil_div(nk, TPB), B300_SMS * 16), TPB, 0, st,
                 static_cast<const uint64_t *>(edges), nk, static_cast<const int64_t *>(s->mg_rowptr),
                 static_cast<const uint2 *>(s->csum), static_cast<const uint32_t *>(s->cpk),
                 static_cast<const int32_t *>(wrank), sw, s->mg_cnt);
      MM_LAUNCH_CHECK();
    }
    MM_CUDA_TRY(cudaMemcpyAsync(s->mg_count, s->mg_rowptr + c, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    mark_point(s, 0, st);  // multigraph rows and counts built (the list look-ups need them)
    join_side(s, 0, s->side_pending[0]);
    return;
  }
  // coupling (bitsets): mark the use edges in the out-rows, count and enumerate
  // the marked classes row by row (ascending, so no sort), then count multiplicities
  zero_buffers(s->out_adj, sizeof(uint32_t) * (size_t)(aw * c), s->in_adj, sizeof(uint32_t) * (size_t)(aw * c),
               s->csum, sizeof(uint2) * (size_t)(sw * (2 * c + 1)), st);
  uint64_t *edges = static_cast<uint64_t *>(s->eval_ws.need(sizeof(uint64_t) * (size_t)std::max<int64_t>(nk, 1), st));
  if (M > 0) {
    pdl_launch(coupling_mark, grid_for(M), TPB, 0, st, s->method_class, s->call_rowptr, s->call_idx, s->acc_rowptr,
                                               s->acc_idx, s->attr_class, M, s->cbo_attrs, s->out_adj, aw,
                                               s->csum, sw, edges);
    MM_LAUNCH_CHECK();
  }
  const unsigned grow = (unsigned)std::min<int64_t>(ceil_div((int64_t)c * 32, TPB), B300_SMS * 16);
  pdl_launch(row_distinct, grow, TPB, 0, st, s->csum, s->out_adj, c, aw, sw, row_count);
  MM_LAUNCH_CHECK();
  // mg_rowptr = exclusive scan of the row counts (CBO); last entry = distinct pairs
  scan_exclusive_i32to64(row_count, s->mg_rowptr, c, s->sort_ws, st, s->mg_rowptr + c);
  pdl_launch(row_enumerate, grow, TPB, 0, st, s->csum, s->out_adj, s->in_adj, c, aw, sw, s->mg_rowptr, s->mg_dst,
                                      s->mg_cnt);
  MM_LAUNCH_CHECK();
  if (M > 0) {
    pdl_launch(coupling_count, (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(nk, 1), TPB), B300_SMS * 16), TPB, 0, st, 
        edges, nk, s->mg_rowptr, s->mg_dst, s->mg_cnt);
    MM_LAUNCH_CHECK();
  }
  MM_CUDA_TRY(cudaMemcpyAsync(s->mg_count, s->mg_rowptr + c, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  mark_point(s, 0, st);  // multigraph rows and counts built (the list look-ups need them)
  // compressed adjacency: record counts -> exclusive scan -> packed non-zero words
  {
    char *b = static_cast<char *>(s->eval_ws.need((sizeof(int32_t) + sizeof(int64_t)) * (size_t)ns + 16, st));
    int64_t *first = reinterpret_cast<int64_t *>(b);
    int32_t *cnt = reinterpret_cast<int32_t *>(first + ns);
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(ns, TPB), B300_SMS * 16);
    pdl_launch(summary_popc, g, TPB, 0, st, s->csum, ns, cnt);
    MM_LAUNCH_CHECK();
    scan_exclusive_i32to64(cnt, first, ns, s->sort_ws, st);
    pdl_launch(summary_pack, g, TPB, 0, st, s->csum, first, s->out_adj, s->in_adj, c, s->adj_words, s->sum_words, ns,
                                    s->cpk);
    MM_LAUNCH_CHECK();
  }
  s->adj_built = true;
  join_side(s, 0, s->side_pending[0]);
}

// The full adjacency bitsets, from the multigraph rows, for a system whose
// coupling was built in the packed form (allocated on first use).
void ensure_adjacency(mm_system *s) {
  if (s->adj_built) return;
  cudaStream_t st = s->stream;
  const int64_t words = s->adj_words * (int64_t)s->c;
  uint32_t *p = static_cast<uint32_t *>(s->adj_ws.need(2 * sizeof(uint32_t) * (size_t)words, st));
  s->out_adj = p;
  s->in_adj = p + words;
  zero_buffers(s->out_adj, sizeof(uint32_t) * (size_t)words, s->in_adj, sizeof(uint32_t) * (size_t)words, nullptr, 0,
               st);
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div((int64_t)s->c * 32, TPB), B300_SMS * 16);
  pdl_launch(adjacency_from_rows, g, TPB, 0, st, static_cast<const int64_t *>(s->mg_rowptr),
             static_cast<const int32_t *>(s->mg_dst), s->c, s->adj_words, s->out_adj, s->in_adj);
  MM_LAUNCH_CHECK();
  s->adj_built = true;
}

// Build the coupling with the full bitsets from now on (for callers that read
// them inside captured work, such as a batch's graph).
void use_bitset_coupling(mm_system *s) {
  if (!s->packed_coupling) return;
  const int64_t words = s->adj_words * (int64_t)s->c;
  uint32_t *p = static_cast<uint32_t *>(s->adj_ws.need(2 * sizeof(uint32_t) * (size_t)words, s->stream));
  s->out_adj = p;
  s->in_adj = p + words;
  s->packed_coupling = false;
  s->adj_built = false;
}
