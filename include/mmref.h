/*
 * mmref -- Move Method metric engine for NVIDIA B300 (sm_103a).
 *
 * C ABI of the library.  It computes, for every class of an object-oriented
 * system, the modularity metrics of Napoli, Pappalardo and Tramontana, "Using
 * Modularity Metrics to assist Move Method Refactoring of Large Systems"
 * (CISIS 2013), and evaluates every candidate Move Method refactoring:
 *
 *   fan-in / fan-out ..... Sec. II.A: methods calling m / methods m calls
 *   CBO .................. Sec. II.B: number of other classes a class uses
 *                          (calls into them; optionally attribute accesses)
 *   LCOM (CK) ............ Sec. II.B: method pairs sharing no attribute minus
 *                          pairs sharing one, reported as max(P - Q, 0); only
 *                          attributes owned by the class count
 *   LCOM (HS) ............ Sec. II.B: 1 - mean over methods of the fraction of
 *                          the class's attributes each uses; exact fraction
 *                          (n*a - S) / (n*a), or 0/1 when n*a == 0
 *   move evaluation ...... Sec. III.A (the three rules) and Sec. IV.C (metrics
 *                          re-evaluated for the source and destination classes
 *                          of each candidate move), done incrementally
 *   suggestions .......... Sec. III.A / Sec. IV.A: keep the moves that improve
 *                          several classes and worsen none, for one selected
 *                          characteristic or the intersection of several
 *
 * Ids are int32: classes [0, n_classes), methods [0, n_methods), attributes
 * [0, n_attrs) (Sec. IV.C: "classes, methods and attributes have been
 * represented by a numerical id").  Everything is integer; no floating point
 * is used anywhere on the path.
 *
 * Conventions for every call:
 *   - Inputs are borrowed: the library copies what it keeps and never frees
 *     caller memory.  Outputs are caller-owned buffers.
 *   - A pointer's kind (host or device memory) is given explicitly.  Device
 *     pointers must be valid on the current CUDA device.
 *   - Work is ordered on the system's CUDA stream.  A call that writes host
 *     memory synchronises that stream before it returns; a call that only
 *     writes device memory may return before the work is done.
 *   - On error the call returns a non-zero mm_status, leaves the outputs and
 *     the system unchanged, and sets a thread-local message (mm_last_error).
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef MMREF_H
#define MMREF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMREF_ABI_VERSION 1

#if defined(__GNUC__)
#define MMREF_API __attribute__((visibility("default")))
#else
#define MMREF_API
#endif

typedef enum {
  MM_OK = 0,
  MM_EINVAL = 1,     /* malformed input (ids out of range, unsorted rows, ...) */
  MM_ENOMEM = 2,     /* device or host allocation failed */
  MM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  MM_ENOTFOUND = 4,  /* edit removes an edge that does not exist */
  MM_EEXIST = 5,     /* edit adds an edge that already exists */
  MM_ETIMEOUT = 6,   /* a bounded device-side wait gave up (see below) */
  MM_EBUDGET = 7     /* admission refused: memory budget exceeded */
} mm_status;

/* Bounded waits.  The one device-side wait of the library is the look-back
 * of its one-pass exclusive scan (Merrill and Garland, 2016), used by load,
 * metrics, lists, similarity and the rules.  It polls at most about a second;
 * when it runs out, the block sums the input before its tile itself, so the
 * scan's output and everything computed from it stay exact, and it sets the
 * fault word of the system (or batch) whose call queued the scan.  Every
 * system and batch has its own word: a give-up is reported to that handle
 * only, as MM_ETIMEOUT from its next call that synchronises (mm_load_system,
 * mm_compute_metrics and mm_export_metrics with host outputs,
 * mm_evaluate_moves with host outputs, mm_suggest_moves,
 * mm_suggest_moves_noalloc, mm_similarity, mm_suggest_r1, mm_suggest_r3,
 * mm_apply_sequence, mm_metric_variants and mm_rank_classes with host
 * outputs, mm_batch_run), which clears it.  The outputs of that call are
 * written before the status is returned. */

enum { MM_PTR_HOST = 0, MM_PTR_DEVICE = 1 };

/* metric selection bits (Sec. IV.A: the developer selects the characteristic
 * to improve, or asks for all of them) */
enum { MM_LCOM_CK = 1, MM_LCOM_HS = 2, MM_CBO = 4 };

typedef struct mm_system mm_system; /* opaque; owns all device memory it allocates */

/*
 * A system in CSR form: the paper's "cls" array (owner class of each method
 * and attribute) and "dpnd" array (per method, the invoked methods and the
 * accessed attributes), Sec. IV.C.
 *   method_class[n_methods]   owner class of each method
 *   attr_class[n_attrs]       owner class of each attribute
 *   acc_rowptr[n_methods+1]   int64, acc_rowptr[0] = 0, non-decreasing,
 *                             acc_rowptr[n_methods] = n_acc
 *   acc_idx[n_acc]            accessed attribute ids, strictly increasing
 *                             within each method's row
 *   call_rowptr/call_idx      called method ids, same rules, and no method
 *                             calls itself
 *   cbo_attrs                 1: an access to another class's attribute is a
 *                             use for CBO (default); 0: only calls count
 *   flags                     0, or one of MM_LOAD_PACKED_COUPLING (build the
 *                             class coupling from the use edges into the
 *                             compressed rows directly; the
 *                             full c x c adjacency bitsets are then built only
 *                             when a full cross-product evaluation needs
 *                             them), MM_LOAD_BITSET_COUPLING (always build the
 *                             bitsets with the coupling).  With 0 the packed
 *                             form is chosen when the two bitsets would take
 *                             more than MM_PACKED_COUPLING_BYTES.  Results
 *                             are the same either way.
 */
enum { MM_LOAD_PACKED_COUPLING = 1, MM_LOAD_BITSET_COUPLING = 2 };
#define MM_PACKED_COUPLING_BYTES (512.0 * 1024.0 * 1024.0)
typedef struct {
  int32_t n_classes, n_methods, n_attrs;
  int32_t ptr_kind; /* MM_PTR_HOST or MM_PTR_DEVICE, for all six arrays */
  int64_t n_acc, n_call;
  const int32_t *method_class;
  const int32_t *attr_class;
  const int64_t *acc_rowptr;
  const int32_t *acc_idx;
  const int64_t *call_rowptr;
  const int32_t *call_idx;
  int32_t cbo_attrs;
  int32_t flags;
} mm_system_desc;

/* Per-class metrics (64 bytes).  P = pairs of methods sharing no attribute of
 * the class, Q = pairs sharing at least one (P + Q = n(n-1)/2), S = sum over
 * methods of the number of the class's attributes they access. */
typedef struct {
  int32_t n_methods, n_attrs;
  int64_t P, Q, S;
  int64_t lcom_ck;          /* max(P - Q, 0) */
  int64_t hs_num, hs_den;   /* LCOM_HS = hs_num / hs_den */
  int32_t cbo, reserved;
} mm_class_metrics;

/* Per-method metrics.  own = accesses to the own class's attributes,
 * q = methods of the own class sharing an attribute of the class with it. */
typedef struct {
  int32_t fan_in, fan_out, own, q;
} mm_method_metrics;

/*
 * Evaluation record of one candidate move (method m from class C to class D),
 * 16 bytes:
 *   s           methods of D sharing an attribute of D with m
 *   t           m's accesses to attributes of D (saturates at 65535)
 *   dcbo_src    CBO(C) after - before (saturates to int16)
 *   dcbo_dst    CBO(D) after - before (saturates to int16)
 *   n_improved  affected classes with no selected metric higher and one lower
 *   n_worsened  affected classes with a selected metric higher
 *               (affected = C, D and the classes of m's callers; both
 *               counts saturate at 65535)
 *   flags       2-bit signs, 0 = unchanged, 1 = lower, 2 = higher:
 *               bits 0-1 LCOM_CK(C), 2-3 LCOM_HS(C), 4-5 CBO(C),
 *               bits 6-7 LCOM_CK(D), 8-9 LCOM_HS(D), 10-11 CBO(D);
 *               bit 15 = kept (n_worsened == 0 and n_improved >= min_improved)
 */
typedef struct {
  int32_t s;
  uint16_t t;
  int16_t dcbo_src, dcbo_dst;
  uint16_t n_improved, n_worsened, flags;
} mm_move_eval;

/* Suggestion criteria (Sec. III.A, Sec. IV.A).  A move is kept when no
 * affected class gets worse in a selected metric and at least min_improved
 * classes get better. */
typedef struct {
  uint32_t metric_mask; /* MM_LCOM_CK | MM_LCOM_HS | MM_CBO subset, non-empty */
  int32_t min_improved; /* >= 1 */
} mm_criteria;

/* One suggested move.  Suggestions are ordered by n_improved (descending),
 * then d_lcom_ck_sum = dLCOM_CK(C) + dLCOM_CK(D) (ascending), then
 * d_cbo_sum = dCBO(C) + dCBO(D) (ascending, not saturated), then m, then d
 * (ascending). */
typedef struct {
  int32_t m, d;
  int32_t n_improved;
  int32_t d_lcom_ck_sum;
  int32_t d_cbo_sum;
  int32_t reserved;
} mm_move;

/*
 * Candidate moves.  rowptr == NULL: the full cross product, every method to
 * every class other than its own, n_methods * (n_classes - 1) candidates; the
 * candidate of (m, D) has index m*(n_classes-1) + D - (D > cls(m)).
 * Otherwise a CSR over methods: rowptr[n_methods+1] (int64, rowptr[0] = 0,
 * non-decreasing, rowptr[n_methods] = n_cand) and dst[n_cand] destination
 * classes, each in range and different from the method's class; index i is
 * the position in dst.  Every call that takes lists checks them on the device
 * and hashes their content (the key of the kept-move cache); host lists are
 * first copied to the device.  flags: 0, or MM_CANDS_UNCHANGED: the caller
 * states that these are the same lists (same memory kind, same rowptr and dst
 * pointers, same n_cand, same content) as in the last call on this handle
 * that took lists, with no edit of the system since; the library then reuses
 * that call's check, hash and, for host lists, its device copy.  When the
 * kind, pointers, length or edit count differ from that call's, the flag is
 * ignored and the lists are checked (and copied) again; lists rewritten in
 * place under the flag are the caller's error (results undefined, no fault).
 */
enum { MM_CANDS_UNCHANGED = 1 };
typedef struct {
  const int64_t *rowptr;
  const int32_t *dst;
  int64_t n_cand;
  int32_t ptr_kind;
  int32_t flags;
} mm_candidates;

/* Start copying host candidate lists (ptr_kind MM_PTR_HOST) to the device and
 * checking them, on a copy stream of the calling thread that first waits for
 * the work already queued on the system's stream; the system's stream does
 * not wait for the copy, so later calls (mm_compute_metrics) overlap it.  A
 * later list call on this handle that passes the same lists with
 * MM_CANDS_UNCHANGED, with no edit between, waits for the copy and check and
 * uses them (it reports their errors); any other list call, or freeing the
 * handle, first waits for the staged copy.  The host arrays must stay
 * unchanged until then; pinned memory lets the copy run asynchronously.
 * Errors: MM_EINVAL (NULL system or lists, device lists, bad n_cand or flags),
 * MM_ENOMEM, MM_ECUDA.  Does not synchronise. */
MMREF_API mm_status mm_stage_candidates(mm_system *sys, const mm_candidates *cands);

typedef struct {
  int32_t n_classes, n_methods, n_attrs, cbo_attrs;
  int64_t n_acc, n_call;
  int64_t n_class_edges;   /* distinct (C, E) class uses, E != C, after compute */
  int64_t device_bytes;    /* device memory held by the system */
} mm_system_info;

/*
 * Load a system (Sec. IV.C: the cls/dpnd arrays are copied to the GPU).
 * Copies the desc's arrays to device memory on `cuda_stream` (a cudaStream_t,
 * NULL = default stream) and validates them on the device.  The stream is
 * kept for every later call on the handle.  Errors: MM_EINVAL for any rule of
 * mm_system_desc broken (the message names the first rule found), MM_ENOMEM,
 * MM_ECUDA, MM_ETIMEOUT if a bounded device-side wait of an earlier queued
 * scan gave up (see mm_selftest_bounded_wait).  Synchronises the stream
 * (validation result).
 */
MMREF_API mm_status mm_load_system(const mm_system_desc *desc, void *cuda_stream, mm_system **out);

/* Use another stream for the later calls on this handle. */
MMREF_API mm_status mm_set_stream(mm_system *sys, void *cuda_stream);

/*
 * Compute every class and method metric (Sec. II.A, II.B) and the per-method
 * data that move evaluation needs.  Builds, on the device: the class->method
 * and class->attribute lists, an inverted index of own-attribute accesses,
 * the LCOM method-pair counts (unions of accessor lists), the class-use
 * multigraph (marked adjacency rows, counted and enumerated per row) with
 * CBO, class adjacency bitsets and their compressed two-level form, and
 * fan-in/out.  Independent parts run on side streams of the calling thread
 * and rejoin the system's stream before the call returns.
 * out_c[n_classes] and out_m[n_methods] are optional (NULL = keep on device);
 * out_kind says where they live.
 */
MMREF_API mm_status mm_compute_metrics(mm_system *sys, mm_class_metrics *out_c, mm_method_metrics *out_m,
                             int32_t out_kind);

/*
 * Copy the system's current class and method metrics (Sec. II.A, II.B) --
 * as the last mm_compute_metrics, batch run (mm_batch_run) or edit
 * (mm_apply_edit) left them -- without computing them again.  Same layouts
 * and out_kind rules as mm_compute_metrics.  MM_EINVAL if no metrics have
 * been computed.  Synchronises the stream when out_kind is MM_PTR_HOST.
 */
MMREF_API mm_status mm_export_metrics(mm_system *sys, mm_class_metrics *out_c, mm_method_metrics *out_m,
                                      int32_t out_kind);

/*
 * Evaluate candidate moves incrementally (Sec. III.A, Sec. IV.C) against the
 * metrics of the last mm_compute_metrics.  cands == NULL means the full cross
 * product.  records[n_cand] (nullable) receives one mm_move_eval per
 * candidate in candidate order.  digest (nullable, one uint64) receives the
 * sum modulo 2^64, over all candidates, of
 *   h = sm(key ^ sm(lo ^ sm(hi))),  key = (uint64)m << 32 | D,
 * where lo/hi are the record's first/last 8 bytes (little endian) and sm is
 * the SplitMix64 output function (Steele, Lea, Flood 2014).  records and
 * digest live in out_kind memory.  The same pass compacts the kept moves for
 * `crit` into the handle, so a following mm_suggest_moves with the same
 * criteria and the same candidates (the full cross product, or lists with the
 * same 64-bit content hash, computed while validating them) does not evaluate
 * again.  Errors: MM_EINVAL (no metrics computed,
 * bad criteria, a candidate out of range or equal to the method's class),
 * MM_ENOMEM, MM_ECUDA.
 */
MMREF_API mm_status mm_evaluate_moves(mm_system *sys, const mm_criteria *crit, const mm_candidates *cands,
                            mm_move_eval *records, uint64_t *digest, int32_t out_kind);

/*
 * Suggest moves (Sec. III.A, IV.A): evaluate the candidates, keep those that
 * pass the criteria (warp-ballot compaction), sort the kept moves in the
 * order given at mm_move and write the first min(k, n_kept) to out_topk
 * (out_kind memory; may be NULL when k == 0).  *n_kept and
 * *n_methods_with_kept (host, nullable) receive the number of kept moves and
 * of distinct methods among them.  Up to 8,192 kept moves are sorted on the
 * device before the one read-back of the counts.  Errors as mm_evaluate_moves,
 * plus MM_ETIMEOUT if a bounded device-side wait (the look-back of a scan in
 * this or an earlier queued call) gave up.  Synchronises the stream.
 */
MMREF_API mm_status mm_suggest_moves(mm_system *sys, const mm_criteria *crit, const mm_candidates *cands,
                           int32_t k, mm_move *out_topk, int32_t out_kind, int64_t *n_kept,
                           int64_t *n_methods_with_kept);

/*
 * Allocation-free variant of mm_suggest_moves.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * the time they ask for suggestions -- a serving process whose device memory
 * is entirely reserved by its own fixed-budget allocator, or a latency-critical
 * loop that must not trigger allocation (which can stall or fail under memory
 * pressure).  It computes the same result as mm_suggest_moves (same criteria,
 * same order) but calls no cudaMalloc, cudaFree or allocating routine: its
 * working memory is a static device array of about 4.2 MB in the library,
 * which every GPU that loads the library holds until the process exits.
 * Limits: the system has at most MM_NOALLOC_MAX_METHODS methods and the
 * criteria keep at most MM_NOALLOC_MAX_KEPT moves; beyond either the call
 * returns MM_EBUDGET with a message naming the limit, and mm_suggest_moves
 * must be used instead.  The same holds for the full cross product of a
 * system with packed coupling (MM_LOAD_PACKED_COUPLING) whose adjacency
 * bitsets no full cross-product call has built yet.  Candidate lists must be
 * NULL (full cross product) or
 * in device memory.  out_topk is in out_kind memory.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls in the process share the one array and
 * each call clears what it needs; calls that overlap on the GPU (from several
 * threads or streams) race on it and must be serialised by the caller.
 * Synchronises the system's stream.
 */
#define MM_NOALLOC_MAX_METHODS 1048576
#define MM_NOALLOC_MAX_KEPT 65536
MMREF_API mm_status mm_suggest_moves_noalloc(mm_system *sys, const mm_criteria *crit, const mm_candidates *cands,
                                             int32_t k, mm_move *out_topk, int32_t out_kind, int64_t *n_kept,
                                             int64_t *n_methods_with_kept);

/*
 * Jaccard similarity of method pairs (Sec. II.A) and rule R1 (Sec. III.A).
 * The properties of a method are the methods it calls and the attributes it
 * accesses; sim(x, y) = |P(x) & P(y)| / |P(x) | P(y)|, kept as the exact
 * integers (i, u).  The values are the pairs with a common property (i > 0;
 * Sec. IV.C keeps only non-zero similarity values); every other pair has
 * similarity 0.
 */
typedef struct {
  int64_t n_values;        /* method pairs with a common property */
  int64_t n_cooccurrences; /* (pair, common property) incidences they were counted from */
  int64_t n_high;          /* R1: values above the average whose methods are in different classes */
  int64_t n_candidates;    /* R1: distinct moves those pairs propose */
  double average;          /* average of the values (footnote of Sec. III.A: R1's threshold) */
  int32_t max_union;       /* upper bound of u: twice the largest property count */
  int32_t reserved;
} mm_similarity_info;

/*
 * Compute every similarity value of the system's current state (its input
 * CSR; metrics need not be computed).  x[], y[], inter[], uni[] (nullable,
 * cap entries each, out_kind memory) receive the first min(cap, n_values)
 * values in (x, y) order, x < y, with inter = i and uni = u.  info
 * (nullable, host) receives the counts and the average (n_high and
 * n_candidates are 0).  Errors: MM_EBUDGET when the pairs sharing a property
 * exceed 2^32, MM_ENOMEM, MM_ECUDA.  Synchronises the stream.
 */
MMREF_API mm_status mm_similarity(mm_system *sys, int32_t *x, int32_t *y, int32_t *inter, int32_t *uni, int64_t cap,
                                  int32_t out_kind, mm_similarity_info *info);

/*
 * Suggestions of rule R1 (Sec. III.A, first rule): every pair of methods in
 * different classes whose similarity is above the average of all similarity
 * values (the average in double precision, summed over u ascending of
 * sum(i)/u and divided by the number of values; a pair is above it when
 * (double)i / (double)u is greater) proposes moving either method to the
 * other's class, or to another class holding a method it calls.  The
 * distinct proposed moves are evaluated and filtered by
 * crit exactly as mm_suggest_moves does with them as candidate lists (R1
 * itself asks for LCOM improved in both the origin and the destination:
 * metric_mask = MM_LCOM_CK | MM_LCOM_HS, min_improved = 2).  Outputs as
 * mm_suggest_moves; info (nullable, host) as mm_similarity plus n_high and
 * n_candidates.  Needs mm_compute_metrics first.  Synchronises the stream.
 */
MMREF_API mm_status mm_suggest_r1(mm_system *sys, const mm_criteria *crit, int32_t k, mm_move *out_topk,
                                  int32_t out_kind, int64_t *n_kept, int64_t *n_methods_with_kept,
                                  mm_similarity_info *info);

/*
 * Suggestions of rule R3 (Sec. III.A, third rule).  Classes whose CBO is
 * above the average CBO of all classes (exactly: CBO(C) * n_classes > sum of
 * CBO) relocate their methods, each to every class it uses (calls into, or
 * reads an attribute of when the system counts attribute uses); a relocation
 * is kept when the origin's CBO drops and the destination's does not rise
 * (dcbo_src < 0, dcbo_dst <= 0, as mm_move_eval computes them).  Kept moves
 * are ordered by fan_in + fan_out of the method (descending: the rule starts
 * with the methods of highest fan-in and fan-out), then dcbo_src + dcbo_dst
 * (ascending), then m, then d.  out_topk (host, k entries) receives the first
 * min(k, n_kept); *n_candidates the relocations evaluated, *n_high_classes
 * the classes above the average (all nullable).  Needs mm_compute_metrics
 * first.  Synchronises the stream.
 */
typedef struct {
  int32_t m, d, fan_in, fan_out, dcbo_src, dcbo_dst;
} mm_r3_move;
MMREF_API mm_status mm_suggest_r3(mm_system *sys, int32_t k, mm_r3_move *out_topk, int64_t *n_kept,
                                  int64_t *n_candidates, int32_t *n_high_classes);

/*
 * Metric variants (Sec. II.B).  The paper defines LCOM as the method pairs
 * sharing no attribute minus the pairs sharing one, without saying whose
 * attributes, and CBO as the classes C uses; the CK suite it cites counts
 * coupling in both directions.  Per class:
 *   P_all, Q_all   pairs of C's methods sharing no accessed attribute / at
 *                  least one, over the attributes of every class (the
 *                  mm_class_metrics P, Q count only C's own attributes);
 *   lcom_ck_all    max(P_all - Q_all, 0);
 *   lcom_pq        P - Q unclamped (negative when sharing pairs dominate);
 *   lcom_pq_all    P_all - Q_all unclamped;
 *   cbo_out        CBO as in mm_class_metrics (other classes C uses);
 *   cbo_in         other classes that use C (same uses: calls, and attribute
 *                  accesses when the system counts them);
 *   cbo_bi         other classes coupled to C either way, |out u in|.
 * out (n_classes entries) and out_q_all (n_methods: methods of m's class
 * sharing an accessed attribute with m) are both in host or both in device
 * memory per out_kind; either may be NULL.  Needs mm_compute_metrics first.
 * Errors: MM_EINVAL (NULL system, metrics not computed, bad out_kind),
 * MM_ENOMEM, MM_ECUDA.  Synchronises the stream when out_kind is host.
 */
typedef struct {
  int64_t P_all, Q_all, lcom_ck_all, lcom_pq, lcom_pq_all;
  int32_t cbo_out, cbo_in, cbo_bi, reserved;
} mm_class_variants; /* 56 bytes */
MMREF_API mm_status mm_metric_variants(mm_system *sys, mm_class_variants *out, int32_t *out_q_all,
                                       int32_t out_kind);

/*
 * Classes ranked by one metric, largest first, equal values by ascending
 * class id (the order in which a rule takes the classes of highest LCOM or
 * CBO, Sec. III.A).  metric is one of MM_RANK_*; out_ids (k entries) and
 * out_values (k entries, nullable) receive the first min(k, n_classes)
 * classes and their values, both in host or both in device memory per
 * out_kind.  Needs mm_compute_metrics first.  Errors: MM_EINVAL (NULL system,
 * metrics not computed, unknown metric, k < 0, out_ids NULL with k > 0, bad
 * out_kind), MM_ENOMEM, MM_ECUDA.  Synchronises the stream when out_kind is
 * host.
 */
enum {
  MM_RANK_LCOM_CK = 1,     /* max(P - Q, 0) */
  MM_RANK_LCOM_PQ = 2,     /* P - Q, unclamped */
  MM_RANK_LCOM_CK_ALL = 3, /* max(P_all - Q_all, 0) */
  MM_RANK_LCOM_PQ_ALL = 4, /* P_all - Q_all, unclamped */
  MM_RANK_CBO = 5,         /* classes used */
  MM_RANK_CBO_IN = 6,      /* classes using it */
  MM_RANK_CBO_BI = 7       /* classes coupled either way */
};
MMREF_API mm_status mm_rank_classes(mm_system *sys, int32_t metric, int32_t k, int32_t *out_ids,
                                    int64_t *out_values, int32_t out_kind);

/*
 * Batched evaluation (no counterpart in the paper; the paper analyses one
 * system at a time, Sec. V).  A batch holds many loaded systems of very
 * uneven sizes.  mm_batch_run computes every system's metrics (as
 * mm_compute_metrics) and evaluates every system's full cross product in one
 * persistent work-stealing launch; the whole sequence is captured once in a
 * CUDA graph and replayed on later runs.  Per system it yields the digest of
 * all its records (as mm_evaluate_moves) and its kept moves for `crit`
 * (as mm_suggest_moves), up to kept_cap moves per system.
 * While a batch exists its systems must not be used by other calls
 * concurrently; results of other calls on them stay valid.
 */
typedef struct mm_batch mm_batch;

/* Create a batch over systems[0..n) (all loaded on the current device; their
 * metrics need not be computed).  The stream orders every batch call. */
MMREF_API mm_status mm_batch_create(mm_system *const *systems, int32_t n, const mm_criteria *crit,
                                    int64_t kept_cap, void *cuda_stream, mm_batch **out);
/* Methods per evaluation tile (default 256, or the autotuned value). */
MMREF_API mm_status mm_batch_set_tile(mm_batch *b, int32_t methods_per_tile);
/* Time a few launch configurations on this batch and keep the fastest (cached
 * in the process per batch shape): first the methods per tile (32 .. 1,024)
 * with every block the device can hold resident, then, for that tile, the
 * number of persistent blocks (1 .. the resident limit per SM, times the SM
 * count).  *chosen (nullable) receives the methods per tile. */
MMREF_API mm_status mm_batch_autotune(mm_batch *b, int32_t *chosen);
/* The batch's launch configuration: methods per tile and persistent blocks
 * (either pointer nullable).  Errors: MM_EINVAL for a NULL batch. */
MMREF_API mm_status mm_batch_config_get(const mm_batch *b, int32_t *methods_per_tile, int32_t *blocks);
/* Run: digests[n] and n_kept[n] (host, nullable) receive each system's digest
 * and kept-move count.  Synchronises the batch stream. */
MMREF_API mm_status mm_batch_run(mm_batch *b, uint64_t *digests, int64_t *n_kept);
/* Sorted suggestions of system i from the last run (order of mm_move);
 * MM_EBUDGET if that system kept more than kept_cap moves. */
MMREF_API mm_status mm_batch_suggestions(mm_batch *b, int32_t i, int32_t k, mm_move *out_topk, int32_t out_kind,
                                         int64_t *n_kept);
MMREF_API void mm_batch_free(mm_batch *b);

/*
 * Edits (the system evolves while it is analysed; abstract, and Sec. IV.C's
 * re-evaluation after a class representation changes).
 *   MM_EDIT_ADD_ACCESS / MM_EDIT_REMOVE_ACCESS   target = attribute id
 *   MM_EDIT_ADD_CALL / MM_EDIT_REMOVE_CALL       target = called method id
 *   MM_EDIT_MOVE                                 target = destination class
 */
enum {
  MM_EDIT_ADD_ACCESS = 1,
  MM_EDIT_REMOVE_ACCESS = 2,
  MM_EDIT_ADD_CALL = 3,
  MM_EDIT_REMOVE_CALL = 4,
  MM_EDIT_MOVE = 5
};
typedef struct {
  int32_t kind, m, target, reserved;
} mm_edit;

/*
 * Apply one edit to a system whose metrics have been computed.  The device
 * CSR is patched in place, every class and method metric is brought up to
 * date (as mm_compute_metrics would compute it on the edited system), and the
 * cached kept moves of the full cross product (left by mm_evaluate_moves or
 * mm_suggest_moves) are updated by evaluating only the candidates whose
 * record can change: every candidate of a method in an affected class and
 * every candidate into an affected class.  Affected classes: the method's
 * class and the attribute's owner (access), the callee's class (call), or
 * the source, destination, the classes the method uses and the classes of
 * its callers (move).  Errors (system unchanged): MM_EINVAL (ids out of
 * range, self-call, move to the own class), MM_EEXIST (adding an existing
 * access or call), MM_ENOTFOUND (removing a missing one).  Does not
 * synchronise the stream except on the first edit of a system (it copies the
 * rows to a host mirror used to validate edits).
 */
MMREF_API mm_status mm_apply_edit(mm_system *sys, const mm_edit *edit);

/*
 * Several moves at once (the "several solutions" of the abstract and Sec. I).
 * In each of up to `rounds` rounds, the kept moves of the full cross product
 * for crit (as mm_suggest_moves orders them) are taken greedily while the
 * classes each one affects -- its source and destination, the classes the
 * method uses and the classes of its callers -- are disjoint from those of the
 * moves already taken, and no method moves twice (at most per_round moves,
 * per_round <= 0: no limit).  Such moves do not change one another's
 * evaluation.  The round's moves are applied to the system (as MM_EDIT_MOVE
 * edits) and its metrics computed again before the next round; rounds stop
 * early when nothing is kept.  out[cap] (host, nullable) receives the
 * applied moves in order: {round, m, from class, to class}; *n_applied their
 * number.  Needs mm_compute_metrics first.  Synchronises the stream.
 */
typedef struct {
  int32_t round, m, from, to;
} mm_applied_move;
MMREF_API mm_status mm_apply_sequence(mm_system *sys, const mm_criteria *crit, int32_t rounds, int32_t per_round,
                                      mm_applied_move *out, int64_t cap, int64_t *n_applied);

/* Copy the system's current arrays (after edits) to host buffers sized from
 * mm_system_info_get (n_acc, n_call); any pointer may be NULL.  Synchronises
 * the stream.  Used to re-admit a served system and to check it. */
MMREF_API mm_status mm_export_system(mm_system *sys, int32_t *method_class, int32_t *attr_class,
                                     int64_t *acc_rowptr, int32_t *acc_idx, int64_t *call_rowptr,
                                     int32_t *call_idx);

/*
 * Serving (no counterpart in the paper beyond "continuously gathered while the
 * system evolves", abstract).  A server keeps many evolving systems, makes
 * them resident on the device on demand under a memory budget (evicting idle
 * systems least recently used first, their current arrays copied back to the
 * host), and answers requests: each request is an intended edit of one
 * system; it is resolved against that system's current state (an addition
 * picks the first absent attribute or callee from a position given by the
 * selector, a removal one of the existing entries or, if there is none, the
 * matching addition, a move one of the other classes), applied with
 * mm_apply_edit, and answered with the system's top-k suggestions for the
 * server's criteria.  n_slots worker threads, each on its own CUDA stream,
 * serve requests concurrently as they arrive (continuous batching: a request
 * that arrives while others run starts as soon as a slot is free, and the
 * kernels of different slots overlap on the device); requests of one system
 * run one at a time in arrival order, so each result is the same whatever
 * else is in flight.
 */
typedef struct mm_server mm_server;
typedef struct {
  int64_t budget_bytes;  /* device memory for resident systems */
  int32_t n_slots;       /* concurrent requests (1..64); about 4 serves most on one B300 */
  int32_t topk;          /* suggestions returned per request */
  mm_criteria crit;
} mm_server_config;
typedef struct {
  int32_t system, kind, m, reserved; /* kind: MM_EDIT_*; m: method of the edit */
  uint64_t selector;                 /* picks the concrete target, see above */
  double arrival_s;                  /* seconds from the start of mm_server_run, non-decreasing */
} mm_request;
typedef struct {
  int32_t status, slot;              /* mm_status of the request, worker slot */
  mm_edit edit;                      /* the resolved edit */
  double arrival_s, start_s, done_s; /* latency = done_s - arrival_s */
  int64_t n_kept, n_methods_with_kept;
} mm_response;
typedef struct {
  int64_t served, failed, loads, evictions, resident_bytes, n_snapshots;
  double wall_s;
} mm_server_stats;
typedef struct {
  int64_t request;
  int32_t system, n_classes, n_methods, n_attrs;
  int64_t n_acc, n_call;
} mm_snapshot_info;

MMREF_API mm_status mm_server_create(const mm_server_config *cfg, mm_server **out);
/* Register a system (host arrays, copied); *id is its index for requests. */
MMREF_API mm_status mm_server_add_system(mm_server *sv, const mm_system_desc *desc, int32_t *id);
/* Serve n requests (open loop: request i is released at arrival_s).  resp[n]
 * receives one response per request; topk (nullable) n * cfg.topk moves.
 * With snapshot_every > 0 the state of the edited system after requests
 * 0, snapshot_every, 2*snapshot_every, ... is kept for mm_server_snapshot. */
MMREF_API mm_status mm_server_run(mm_server *sv, const mm_request *req, int64_t n, mm_response *resp,
                                  mm_move *topk, int64_t snapshot_every);
MMREF_API mm_status mm_server_stats_get(mm_server *sv, mm_server_stats *out);
/* Snapshot k: sizes in *info; arrays (nullable) sized from a first call. */
MMREF_API mm_status mm_server_snapshot(mm_server *sv, int64_t k, mm_snapshot_info *info, int32_t *method_class,
                                       int32_t *attr_class, int64_t *acc_rowptr, int32_t *acc_idx,
                                       int64_t *call_rowptr, int32_t *call_idx);
MMREF_API void mm_server_free(mm_server *sv);

/*
 * GPU time in milliseconds of the evaluation kernel launched by the last
 * mm_evaluate_moves or mm_suggest_moves on this handle that evaluated
 * (events recorded on the system's stream immediately before and after that
 * launch; waits for it to finish).  The paper has no counterpart: it lets a
 * caller relate the evaluation kernel alone -- without the validation of
 * candidate lists or the suggestion sort around it -- to its memory roofline.
 * MM_EINVAL if no evaluation kernel has run on the handle.
 */
MMREF_API mm_status mm_last_eval_ms(mm_system *sys, float *ms);

/* Sizes and device memory of a loaded system (host struct). */
MMREF_API mm_status mm_system_info_get(mm_system *sys, mm_system_info *info);

/* Free the system and all device memory it owns (stream-ordered). */
MMREF_API void mm_free_system(mm_system *sys);

/* Thread-local message of the last failed call on this thread ("" if none). */
MMREF_API const char *mm_last_error(void);

MMREF_API const char *mm_status_string(mm_status st);

MMREF_API int32_t mm_abi_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all systems); for accounting in benchmarks. */
MMREF_API int64_t mm_launch_count(void);

/* Failure-detection self test of the bounded device-side waits (the look-back
 * of the exclusive scan used by load, metrics and lists; Merrill and Garland,
 * 2016).  Runs one scan tile on the current device whose predecessor tile is
 * never processed, so its wait gives up after about a second and its
 * fallback sums the predecessor's input; returns MM_ETIMEOUT when the fault
 * word was set and the output is the exact prefix sum (the designed outcome),
 * MM_OK if the wait did not run out, MM_ECUDA if the output is wrong or on a
 * CUDA error.  Uses its own buffers and fault word.  Needs a GPU. */
MMREF_API mm_status mm_selftest_bounded_wait(void);

/* Test hook for the bounded waits inside a real pipeline: the next n scans of
 * more than 16,384 elements queued by calls on sys hold back their first
 * tile's state until another tile's look-back has run out (polls cut to
 * 4,096), so those tiles take the fallback and set sys's fault word.  The
 * results stay exact; the next synchronising call on sys returns MM_ETIMEOUT
 * (see "Bounded waits" above).  n = 0 ends it.  Errors: MM_EINVAL for a NULL
 * system or n < 0.  No device work. */
MMREF_API mm_status mm_selftest_stall_scans(mm_system *sys, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* MMREF_H */
