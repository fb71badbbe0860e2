// Internal declarations of the mmref CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>

#include <string>
#include <vector>

#include "mmref.h"

// ---------------------------------------------------------------- errors

void mm_set_error(const std::string &msg);

struct MmError {
  mm_status st;
  std::string msg;
};

#define MM_CUDA_TRY(expr)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw MmError{e_ == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA,                  \
                    std::string(#expr) + ": " + cudaGetErrorString(e_)};                     \
  } while (0)

// Every kernel launch site is followed by MM_LAUNCH_CHECK(), which also counts
// the launch (mm_launch_count in the C ABI).
void mm_count_launch();
#define MM_LAUNCH_CHECK()      \
  do {                         \
    mm_count_launch();         \
    MM_CUDA_TRY(cudaGetLastError()); \
  } while (0)

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Streaming multiprocessors of a B300 (two dies of 74); grid caps are multiples of it.
constexpr int B300_SMS = 148;

// Programmatic dependent launch: a kernel of the pipeline is launched so that
// the GPU may schedule its blocks while the previous kernel of the stream is
// still finishing; every such kernel first waits (griddepcontrol.wait) until
// that kernel has completed and its writes are visible, so only the launch
// latency overlaps.  Without a preceding kernel the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Carve consecutive, 256-byte aligned pieces out of one scratch buffer (a
// buffer of sum over pieces of round_up(bytes, 256) bytes).
struct Carve {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(int64_t n) {
    T *p = reinterpret_cast<T *>(base + off);
    off += ((sizeof(T) * (size_t)(n > 1 ? n : 1)) + 255) / 256 * 256;
    return p;
  }
};

static inline int bits_for(uint64_t max_value) {  // bits needed to hold [0, max_value]
  int b = 0;
  while (b < 64 && (max_value >> b) != 0) ++b;
  return b;
}

// ---------------------------------------------------------------- device memory

// Stream-ordered allocations owned by a system (freed with the system).
struct DevArena {
  cudaStream_t stream = nullptr;
  std::vector<void *> ptrs;
  int64_t bytes = 0;
  // One slab reserved at load holds the load-time buffers (one allocation and
  // one free instead of dozens); later or larger requests get their own.  In
  // sizing mode alloc() only adds up the sizes and returns null.
  bool sizing = false;
  size_t sized = 0;
  char *slab = nullptr;
  size_t slab_cap = 0, slab_used = 0;
  void reserve(size_t n);
  void *alloc(size_t n);
  void release();
  void forget(void *p);  // free one allocation now (stream-ordered); slab memory stays until release
  template <class T>
  T *get(int64_t count) {
    return static_cast<T *>(alloc(sizeof(T) * (size_t)(count > 0 ? count : 1)));
  }
};

// A grow-only scratch buffer.
struct Scratch {
  void *ptr = nullptr;
  size_t cap = 0;
  void *need(size_t n, cudaStream_t st);
  void release(cudaStream_t st);
};

// Error word written by validation kernels (bit flags).
enum : uint32_t {
  VE_METHOD_CLASS = 1u << 0,
  VE_ATTR_CLASS = 1u << 1,
  VE_ACC_ROWPTR = 1u << 2,
  VE_ACC_IDX_RANGE = 1u << 3,
  VE_ACC_IDX_ORDER = 1u << 4,
  VE_CALL_ROWPTR = 1u << 5,
  VE_CALL_IDX_RANGE = 1u << 6,
  VE_CALL_IDX_ORDER = 1u << 7,
  VE_SELF_CALL = 1u << 8,
  VE_CAND_ROWPTR = 1u << 9,
  VE_CAND_RANGE = 1u << 10,
  VE_CAND_SELF = 1u << 11,
  VE_ERRORS = (1u << 16) - 1,
  // not errors: layout facts found while validating
  VI_METHODS_UNSORTED = 1u << 16,  // method_class is not non-decreasing
  VI_ATTRS_UNSORTED = 1u << 17     // attr_class is not non-decreasing
};

// Summary of a loaded system computed on the device at load time.
struct LoadSummary {
  uint32_t err;
  int32_t max_class_methods;
};

// Per-method header for move evaluation (3 x int4 = 48 bytes):
//   w0 = {C, l_off, l_len, r_off}
//   w1 = {r_len, out_self, in_self, l_all}
//   w2 = {src_signs (2-bit CK | 2-bit HS << 2), dck_src, 0, 0}
// l list entries: int4 {E, out, cnt(C,E), t} plus s in a parallel int32 array.
// r list entries: int4 {X, in, cnt(X,C), 0}.
struct MoveHdr {
  int4 w0, w1, w2;
};

// Host mirror of a system, built on its first edit: the rows (sorted) for edit
// validation and ranks, owners, per-class sizes, and the load-time summary.
struct EditMirror {
  bool ready = false;
  std::vector<std::vector<int32_t>> acc, calls, callers;
  std::vector<int32_t> method_class, attr_class, cls_n, cls_a;
  int64_t acc_cap = 0, call_cap = 0, nu_cap = 0;
};

struct mm_system {
  cudaStream_t stream = nullptr;
  EditMirror mirror;
  int64_t edits = 0;
  int device = 0;
  int32_t c = 0, M = 0, A = 0, cbo_attrs = 1;
  int64_t n_acc = 0, n_call = 0;
  LoadSummary summary{};
  uint32_t load_err = 0;           // validation word read back at load (host)
  bool metrics_ready = false;
  bool methods_by_class = false;   // method ids contiguous by class: no sort needed
  bool attrs_by_class = false;
  int64_t n_class_edges = -1;

  DevArena arena;      // everything sized at load time
  Scratch sort_ws;     // radix-sort / scan scratch
  Scratch eval_ws;     // evaluate/suggest scratch (kept lists, staging)
  Scratch stage_ws;    // host-output staging
  Scratch kept_ws;     // kept moves + per-method marks of the last evaluation
  Scratch keyed_ws;    // keys and a copy of the kept moves while they are ranked
  Scratch edit_ws;     // edit patches and incremental re-evaluation
  Scratch union_ws;    // per-warp bitmaps of accessor unions (largest classes only)
  // independent branches of the metric pipeline run on side streams, each with
  // its own scratch: [0] LCOM (own-access index, pair counts), [1] list L,
  // [2] list R; mid_ev marks points other branches wait for: [0] the multigraph
  // is built (system stream), [1] the own-access lists are built (branch 0)
  Scratch side_eval[3], side_sort[3], side_union[3];
  cudaEvent_t fork_ev = nullptr, join_ev[3] = {nullptr, nullptr, nullptr}, mid_ev[2] = {nullptr, nullptr};
  cudaStream_t side_pending[3] = {nullptr, nullptr, nullptr};  // stream a branch was issued on
  cudaEvent_t eval_ev[2] = {nullptr, nullptr};  // around the last evaluation kernel (timing)
  bool eval_timed = false;
  bool kept_valid = false;   // kept_ws holds the kept moves of the last evaluation for:
  uint32_t kept_mask = 0;    //   this metric mask
  int32_t kept_min = 0;      //   and this min_improved
  bool kept_lists = false;   //   over explicit candidate lists (else the full cross product)
  uint64_t kept_hash = 0;    //   whose content hash was this
  int64_t kept_ncand = 0;    //   and length this
  int64_t kept_cap = 0;
  // the last candidate lists checked on this handle, for MM_CANDS_UNCHANGED:
  // the caller's pointers and kind, and where the lists are on the device
  // (the caller's own device lists, or the copy of host lists in lists_ws)
  bool lists_checked = false;
  int32_t lists_kind = -1;
  const void *lists_rowptr = nullptr, *lists_dst = nullptr;
  const int64_t *lists_dev_rowptr = nullptr;
  const int32_t *lists_dev_dst = nullptr;
  int64_t lists_n = 0, lists_edits = -1;
  uint64_t lists_hash = 0;
  Scratch lists_ws;
  cudaEvent_t chunk_ev[8] = {};  // copies of host-list chunks (created on first use)
  // lists staged by mm_stage_candidates: copied and checked on the copy stream,
  // done when stage_ev completes; their check's words follow the lists in lists_ws
  bool lists_staged = false;
  cudaEvent_t stage_ev = nullptr;
  uint32_t *stage_err = nullptr;
  unsigned long long *stage_hash = nullptr;
  int32_t stage_chunks = 0;                  // method chunks, each copied and checked before chunk_ev[k]
  int32_t stage_mb[9] = {};                  // first method of each chunk (and the end)

  // similarity values (Sec. II.A) of the last mm_similarity / mm_suggest_r1
  Scratch sim_ws, sim_keys_ws, sim_val_ws, r1_ws;
  int32_t *sim_np = nullptr, *sim_x = nullptr, *sim_y = nullptr, *sim_i = nullptr, *sim_u = nullptr;
  int64_t sim_n = 0, sim_cooc = 0;
  int32_t sim_umax = 0;
  double sim_avg = 0.0;
  int64_t *r1_rowptr = nullptr;    // rule R1's candidate lists (device CSR over the methods)
  int32_t *r1_dst = nullptr;
  // metric variants (Sec. II.B) and class ranking
  Scratch var_ws, var_keys_ws;

  // inputs
  int32_t *method_class, *attr_class, *acc_idx, *call_idx;
  int64_t *acc_rowptr, *call_rowptr;

  // class structures
  int32_t *cls_n, *cls_a;          // methods / attributes per class
  int64_t *cm_rowptr;              // class -> methods (ascending ids)
  int32_t *cm_list;
  int32_t *method_local;           // rank of a method inside its class
  int64_t *ca_rowptr;              // class -> attributes (offsets only)
  int32_t *attr_local;             // rank of an attribute inside its class
  int32_t *fan_in;

  // inverted index of own accesses: attribute alpha -> class-local ranks of the
  // methods of own(alpha) that access it, at own_list[own_ptr[alpha] ..]
  int64_t *own_ptr;                // n_attrs + 1
  int32_t *own_list;               // <= n_acc entries

  // metrics
  int64_t *cls_P, *cls_Q, *cls_S;
  int32_t *cls_cbo;
  int32_t *own, *q;

  // class-use multigraph (E != Y) and adjacency bitsets (row-major, adj_words per row)
  int64_t *mg_rowptr;
  int32_t *mg_dst, *mg_cnt;
  int64_t *mg_count;               // device scalar: number of distinct (Y, E)
  uint32_t *out_adj, *in_adj;
  int64_t adj_words;
  // coupling built from the use edges into the compressed rows (large
  // systems): the full bitsets
  // above are then built from the multigraph rows only when a dense
  // evaluation needs them (adj_ws), and adj_built says whether they are current
  bool packed_coupling = false;
  bool adj_built = false;
  Scratch adj_ws;
  // compressed two-level adjacency for the restricted evaluation (L2-resident).
  // Rows 0..c-1 are the out-rows, rows c..2c-1 the in-rows, row 2c is all zero.
  // Record k of a row = {bits, first}: bit j set iff full word 32 k + j of the
  // row is non-zero; `first` = index in cpk of the first non-zero word it marks.
  uint2 *csum;
  uint32_t *cpk;                   // non-zero words, row by row (at most one per distinct pair and side)
  int32_t *wrank;                  // packed form: per out-row word, the row position of its first class
  int64_t sum_words;               // records per row = ceil(adj_words / 32)
  // destination record per class: {P - Q, S, n, a} (32 bytes, one load per candidate)
  int4 *dest_rec;

  // move precompute
  MoveHdr *hdr;
  int4 *l_list;
  int32_t *l_s;
  int4 *r_list;
  int32_t *l_x;                    // method of each L entry (capacity n_acc + n_call)

  // device scalars
  uint32_t *d_err;
  unsigned long long *d_u64;       // [0] digest, [1] kept count, [2] methods with kept, [3] candidate hash,
                                   // [4] load summary, [5] group counter of the restricted evaluation,
                                   // [6..7] error word (d_err), [8] group counter of the LCOM unions,
                                   // [9] fault word of bounded waits (d_fault), [24..] kept field ranges
  uint32_t *d_fault;
  int32_t test_stall_scans = 0;    // test hook: multi-tile scans still to be made to run out
};

// ---------------------------------------------------------------- primitives (mm_prims.cu)

// Exclusive scan of n int64 values (in and out may alias); writes the total to
// *total_dev when non-null.  Uses sys->sort_ws-independent scratch `ws`.
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Scratch &ws,
                        cudaStream_t st);
// Bounded device-side waits (the look-back of the one-pass scan) record that
// they ran out in the fault word of the system or batch whose entry point is
// running on the calling thread, named by a WaitScope for the call's duration
// (a process-wide word when none is).  stall, when non-null, points at the
// test hook's counter: while it is positive, each multi-tile scan decrements
// it and is made to run out of its wait.
struct WaitScope {
  WaitScope(uint32_t *fault, int32_t *stall);
  ~WaitScope();
  WaitScope(const WaitScope &) = delete;
  WaitScope &operator=(const WaitScope &) = delete;
  uint32_t *prev_fault;
  int32_t *prev_stall;
};
uint32_t *current_fault_word();
// Copies a fault word to *host once the stream reaches this point; the caller
// synchronises before reading it.
void read_wait_fault(uint32_t *host, const uint32_t *fault_dev, cudaStream_t st);
// After that synchronisation: a nonzero word is cleared (in stream order) and
// reported as MM_ETIMEOUT naming the call.
void raise_wait_fault(uint32_t host_word, uint32_t *fault_dev, cudaStream_t st, const char *what);
// Both, with a synchronisation between them.
void check_wait_fault(uint32_t *fault_dev, cudaStream_t st, const char *what);
// Page-locked host memory of the calling thread for small read-backs (grow-only,
// freed when the thread exits): copies into it are asynchronous, so a call's
// read-backs need one synchronisation between them, not one each.
void *host_staging(size_t bytes);
// Zeroes three buffers (null or 16-byte aligned starts) in one launch of
// 16-byte stores (faster than cudaMemsetAsync on large buffers here).
void zero_buffers(void *a, size_t na, void *b, size_t nb, void *c, size_t nc, cudaStream_t st);
uint32_t stalled_scan_probe();
void scan_exclusive_i32to64(const int32_t *in, int64_t *out, int64_t n, Scratch &ws, cudaStream_t st,
                            int64_t *total_dev = nullptr);
// Summary records: record k's first packed word = the number of marked words
// in records 0 .. k-1 (an exclusive scan of their popcounts, written into .y).
void scan_summary_first(uint2 *csum, int64_t n, Scratch &ws, cudaStream_t st);

// Stable LSD radix sort of n keys (and optional uint32 values) on bits [0, nbits).
// The result is left in keys/vals; alt buffers are scratch of the same size.
void radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int nbits,
                    Scratch &ws, cudaStream_t st);
void radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                    int nbits, Scratch &ws, cudaStream_t st);
// ---------------------------------------------------------------- pipeline stages

// cnt[Y][E] of the multigraph in the packed form: bit E of out-row Y, and its
// position in the row from the word's row position plus the bits below it
__device__ __forceinline__ int32_t mg_lookup_packed(const uint2 *csum, const uint32_t *cpk, const int32_t *wrank,
                                                    int64_t sw, const int64_t *rowptr, const int32_t *cnt, int32_t Y,
                                                    int32_t E) {
  const uint2 rec = csum[(int64_t)Y * sw + (E >> 10)];
  const uint32_t b = ((uint32_t)E >> 5) & 31u;
  if (!((rec.x >> b) & 1u)) return 0;
  const uint32_t widx = rec.y + __popc(rec.x & ((1u << b) - 1u));
  const uint32_t word = cpk[widx], below = (1u << ((uint32_t)E & 31u)) - 1u;
  if (!((word >> ((uint32_t)E & 31u)) & 1u)) return 0;
  return cnt[rowptr[Y] + wrank[widx] + __popc(word & below)];
}

// Use edges of a warp's group of nm <= 32 consecutive methods x0 .. x0+nm-1:
// each method's calls, then (with_acc) its accesses, are the contiguous range
// [seg(x), seg(x + 1)) with seg(x) = call_rowptr[x] + acc_rowptr[x] (calls
// only: call_rowptr[x]), so the group's edges are [s0, s1) and the warp can
// walk them 32 at a time with coalesced loads and stores.  Lane l holds the
// bounds of method x0 + l.
struct UseGroup {
  int64_t seg, cr, ar;
  int32_t nc;
  int64_t s0, s1;
};
__device__ __forceinline__ UseGroup use_group(const int64_t *call_rowptr, const int64_t *acc_rowptr, bool with_acc,
                                              int64_t x0, int32_t nm, uint32_t lane) {
  UseGroup u;
  const int64_t x = x0 + min((int32_t)lane, nm);  // lanes from nm on hold the group's end
  u.cr = call_rowptr[x];
  u.ar = with_acc ? acc_rowptr[x] : 0;
  u.seg = u.cr + u.ar;
  u.nc = (int32_t)lane < nm ? (int32_t)(call_rowptr[x + 1] - u.cr) : 0;
  u.s0 = __shfl_sync(0xffffffffu, u.seg, 0);
  if (nm < 32) {
    u.s1 = __shfl_sync(0xffffffffu, u.seg, nm);
  } else {
    u.s1 = call_rowptr[x0 + 32] + (with_acc ? acc_rowptr[x0 + 32] : 0);
  }
  return u;
}
// Edge p of the group (every lane calls it, p need not be in range): the
// method's slot, whether it is a call, and its index in call_idx or acc_idx.
__device__ __forceinline__ void use_edge_at(const UseGroup &u, int64_t p, int32_t nm, int32_t &slot, bool &is_call,
                                            int64_t &idx) {
  int32_t lo = 0;  // the last slot whose range starts at or before p
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const int32_t mid = lo + b;
    const int64_t sv = __shfl_sync(0xffffffffu, u.seg, mid & 31);
    if (mid < nm && sv <= p) lo = mid;
  }
  slot = lo;
  const int64_t o = p - __shfl_sync(0xffffffffu, u.seg, lo);
  const int32_t nc = __shfl_sync(0xffffffffu, u.nc, lo);
  const int64_t cr = __shfl_sync(0xffffffffu, u.cr, lo), ar = __shfl_sync(0xffffffffu, u.ar, lo);
  is_call = o < nc;
  idx = is_call ? cr + o : ar + (o - nc);
}

void load_validate_and_summarise(mm_system *s);     // mm_system.cu
void load_finish(mm_system *s);                     // mm_system.cu
void build_structures(mm_system *s);                // mm_system.cu
// Per-warp bitmaps for accessor unions over the methods of one class: words
// per warp (largest class), shared-memory bytes per block of 256 threads, or a
// zeroed global slice per warp of `grid` blocks when the largest class is too
// big for shared memory (then smem = 0 and gbm != nullptr).
struct UnionBitmap {
  int32_t words;
  size_t smem;
  uint32_t *gbm;
  unsigned grid;
};
// reserve: further shared bytes per block of 8 warps that the kernel needs
// beside the bitmaps (the bitmaps go to global memory when both do not fit)
UnionBitmap union_bitmap(mm_system *s, int64_t warps_wanted, Scratch &ws, cudaStream_t st, size_t reserve = 0);
// Side streams of the calling thread on the current device (created on first
// use).  fork_side() returns the stream a branch runs on: side stream i, made
// to wait for the work so far on s->stream, or s->stream itself when the
// stream is being captured into a graph (the batch's graph already runs the
// systems as parallel branches) or the system has no events.
cudaStream_t fork_side(mm_system *s, int i);
// Make s->stream wait for branch i (no-op when the branch ran on s->stream).
void join_side(mm_system *s, int i, cudaStream_t branch);
// Marks point k (mid_ev[k]) on stream from; makes stream to wait for it (no-op
// when both are the same stream, as during capture).
void mark_point(mm_system *s, int k, cudaStream_t from);
void wait_point(mm_system *s, int k, cudaStream_t from, cudaStream_t to);
// The move lists' first half (per-method keys, sorts, offsets, fills), forked
// onto side streams 1 and 2 before the coupling branch; build_move_precompute
// finishes them (multigraph look-ups, s per L entry, headers).
void begin_move_lists(mm_system *s);
// Number of distinct methods of class K that access at least one of the
// attributes of K in acc_row[0 .. len): the union of their accessor lists,
// counted in a per-warp bitmap over K's method ranks.  The accessor elements
// of all the row's attributes are spread over the lanes at once (lane e holds
// attribute e's list; element k goes to the lane whose prefix range holds it),
// set in the bitmap, then read back and cleared word by word, so the bitmap is
// all zero again on return.
__device__ __forceinline__ int32_t accessor_union(const int32_t *acc_row, int64_t len, int32_t K,
                                                  const int32_t *attr_class, const int64_t *own_ptr,
                                                  const int32_t *own_list, uint32_t *bm, uint32_t lane) {
  int32_t cnt = 0;
  // phase 0 sets the bits of every accessor list, phase 1 counts and clears
  // them; each phase walks all of the method's accesses, 32 at a time
  for (int phase = 0; phase < 2; ++phase) {
    for (int64_t e0 = 0; e0 < len; e0 += 32) {
      const int32_t al = e0 + lane < len ? acc_row[e0 + lane] : -1;
      int64_t p0 = 0;
      int32_t n = 0;
      if (al >= 0 && attr_class[al] == K) {
        p0 = own_ptr[al];
        n = (int32_t)(own_ptr[al + 1] - p0);
      }
      int32_t incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
      }
      const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
      for (int32_t k0 = 0; k0 < total; k0 += 32) {
        const int32_t k = k0 + (int32_t)lane;
        // lane holding element k: the first lane whose inclusive prefix exceeds k
        int32_t lo = 0, hi = 31;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
          const int32_t mid = (lo + hi) >> 1;
          const int32_t pm = __shfl_sync(0xffffffffu, incl, mid);
          if (pm > k) hi = mid; else lo = mid + 1;
        }
        const int32_t excl = __shfl_sync(0xffffffffu, incl, lo) - __shfl_sync(0xffffffffu, n, lo);
        const int64_t base = __shfl_sync(0xffffffffu, p0, lo);
        if (k < total) {
          const int32_t j = own_list[base + (k - excl)];
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

// Metric variants of every class and q_all per method into the system's
// variant buffers (mm_variants.cu); the first k classes by a metric.
void compute_variants(mm_system *s, mm_class_variants **out, int32_t **q_all);
void rank_classes(mm_system *s, int32_t metric, int32_t k, int32_t *out_ids, int64_t *out_values, int32_t kind);
// Full adjacency bitsets current for the dense kernels (built from the
// multigraph rows when the coupling was sorted); switch a system to building
// them with its coupling (mm_metrics.cu).
void ensure_adjacency(mm_system *s);
// Class structures after one edit without their full rebuild (mm_system.cu).
void patch_structures(mm_system *s, int32_t kind, int32_t m, int32_t target, int32_t C);
// Host candidate lists copied and checked on a copy stream ahead of their use
// (mm_stage_candidates); settle_staged orders the system's stream after a
// pending staged copy (before lists_ws is reused or freed).
void stage_candidates(mm_system *s, const mm_candidates *cands);
void settle_staged(mm_system *s);
void use_bitset_coupling(mm_system *s);
// Metrics of every class; an edit may skip the LCOM branch or the coupling
// branch when it cannot change them, and recompute the LCOM pair counts of
// only the (at most two) classes whose membership or own accesses it changed
// (mm_metrics.cu).
struct LcomClasses {
  int n = 0;
  int32_t cls[2] = {0, 0};
  int64_t members[2] = {0, 0};  // current method counts of those classes
};
void build_metrics(mm_system *s, bool lcom = true, bool coupling = true, const LcomClasses *only = nullptr);
void build_move_precompute(mm_system *s);           // mm_moves.cu
void export_metrics(mm_system *s, mm_class_metrics *out_c, mm_method_metrics *out_m, int32_t kind);
void evaluate_moves(mm_system *s, const mm_criteria &crit, const mm_candidates *cands,
                    mm_move_eval *records, uint64_t *digest, int32_t kind);
void suggest_moves(mm_system *s, const mm_criteria &crit, const mm_candidates *cands, int32_t k,
                   mm_move *out, int32_t kind, int64_t *n_kept, int64_t *n_mk);

// ---------------------------------------------------------------- batched evaluation (mm_moves.cu)

// One system of a batch and where its results go (all device pointers).
struct BatchLaunchSpec {
  mm_system *sys;
  unsigned long long *digest;      // one per system
  mm_move *kept;                   // kept_cap per system (nullable)
  unsigned long long *kept_count;  // one per system
  uint8_t *kept_mark;              // M bytes per system
};
int64_t batch_tiles(const mm_system *s, int32_t mchunk);
size_t batch_item_bytes();
void batch_fill_items(const BatchLaunchSpec *specs, int32_t n, const mm_criteria &crit, int32_t mchunk,
                      int64_t kept_cap, void *items_host, int64_t *total_tiles);
void batch_launch(const void *items_dev, int32_t n, int64_t total_tiles, int32_t mchunk, bool keep, bool digest,
                  unsigned long long *next_tile, int grid, cudaStream_t st);
void sort_moves_segments(mm_move *base, int64_t stride, const unsigned long long *counts, int32_t n,
                         cudaStream_t st);
constexpr int64_t kSegmentSortMax = 2048;
int batch_persistent_grid();
void sort_kept_moves(mm_system *s, mm_move *kept, int64_t K);
void check_criteria_public(const mm_criteria &crit);

// similarity and rule R1 (mm_similarity.cu)
void compute_similarity(mm_system *s);
void build_r1_candidates(mm_system *s, int64_t *n_high, int64_t *n_cand);

// rule R3 (mm_rules.cu); records of internal (valid) device candidate lists (mm_moves.cu)
void suggest_r3(mm_system *s, int32_t k, mm_r3_move *out, int64_t *n_kept, int64_t *n_cand, int32_t *n_high);
void eval_lists_records(mm_system *s, const int64_t *rowptr, const int32_t *dst, mm_move_eval *records);

// edit path (mm_edit.cu / mm_moves.cu)
void eval_csr_kept_append(mm_system *s, const mm_criteria &crit, const int64_t *rowptr, const int32_t *dst,
                          mm_move *kept, int64_t cap, unsigned long long *count, uint8_t *mark);
void eval_dense_kept_subset(mm_system *s, const mm_criteria &crit, const int32_t *mlist, int32_t n, mm_move *kept,
                            int64_t cap, unsigned long long *count, uint8_t *mark);
bool kept_cache(mm_system *s, mm_move **kept, uint8_t **mark, int64_t *cap);
void apply_edit(mm_system *s, const mm_edit &e);
void export_system(mm_system *s, int32_t *method_class, int32_t *attr_class, int64_t *acc_rowptr,
                   int32_t *acc_idx, int64_t *call_rowptr, int32_t *call_idx);
void ensure_mirror(mm_system *s);
void apply_sequence(mm_system *s, const mm_criteria &crit, int32_t rounds, int32_t per_round, mm_applied_move *out,
                    int64_t cap, int64_t *n_applied);
mm_edit resolve_edit(mm_system *s, int32_t kind, int32_t m, uint64_t sel);
