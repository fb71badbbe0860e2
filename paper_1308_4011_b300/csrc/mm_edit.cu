// Edits of a loaded system and the incremental re-evaluation that follows
// them (the system "evolves" while metrics are gathered, abstract; candidate
// moves re-evaluated after the class representation changes, Sec. IV.C).
//
// An edit adds or removes one attribute access or one call, or moves one
// method to another class.  The host keeps a mirror of the rows (validation,
// ranks, exact buffer sizes); the device CSR is patched in place by shift
// kernels.  The class metrics are then recomputed by the device pipeline
// (O(edges + method pairs)), and the cached kept-move list of the full cross
// product is updated incrementally: only candidates whose record can change
// are evaluated again, i.e. every candidate of a method in an affected class
// and every candidate whose destination is an affected class, where the
// affected classes are
//   access (m, a):  cls(m), owner(a)
//   call (m, t):    cls(m), cls(t)
//   move (m -> D):  cls(m), D, the classes m uses, the classes of m's callers
// (the classes whose membership, bitset rows, multigraph rows or columns, or
// adjacency bits change).
#include <cuda_runtime.h>

#include <algorithm>
#include <set>
#include <vector>

#include "mm_internal.cuh"

void build_structures(mm_system *s);
void build_move_precompute(mm_system *s);
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Scratch &ws,
                        cudaStream_t st);

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) {
  int64_t g = ceil_div(n, TPB);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 0x7fffffffLL));
}

// ---------------------------------------------------------------- CSR patch kernels

// tmp[j] = arr[start + j] for start + j < n, start = rowptr[m] + rank + from_off
__global__ void csr_save(const int32_t *arr, int64_t n, const int64_t *rowptr, int32_t m, int32_t rank,
                         int32_t from_off, int32_t *tmp) {
  const int64_t start = rowptr[m] + rank + from_off;
  for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    tmp[i - start] = arr[i];
}

// arr[start + j] = tmp[j] for start + j < n_after, start = rowptr[m] + rank + to_off;
// an insertion (to_off = 1) also writes arr[rowptr[m] + rank] = value
__global__ void csr_write(int32_t *arr, int64_t n_after, const int64_t *rowptr, int32_t m, int32_t rank,
                          int32_t to_off, const int32_t *tmp, int32_t value) {
  const int64_t pos = rowptr[m] + rank;
  const int64_t start = pos + to_off;
  if (to_off == 1 && blockIdx.x == 0 && threadIdx.x == 0) arr[pos] = value;
  for (int64_t i = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_after;
       i += (int64_t)gridDim.x * blockDim.x)
    arr[i] = tmp[i - start];
}

__global__ void rowptr_add(int64_t *rowptr, int32_t from, int32_t M, int64_t delta) {
  for (int64_t x = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= M;
       x += (int64_t)gridDim.x * blockDim.x)
    rowptr[x] += delta;
}

__global__ void set_i32(int32_t *p, int32_t v) { *p = v; }

// a move changes the method counts of the source and destination classes
__global__ void move_counts(int32_t *cls_n, int32_t C, int32_t D) {
  cls_n[C] -= 1;
  cls_n[D] += 1;
}

// ---------------------------------------------------------------- incremental re-evaluation kernels

// keep the cached moves whose method and destination are both unaffected
__global__ void kept_filter(const mm_move *in, const unsigned long long *count_in, int64_t cap,
                            const uint8_t *classflag, const int32_t *method_class, mm_move *out,
                            unsigned long long *count_out) {
  const int64_t n = min((int64_t)*count_in, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const mm_move v = in[i];
    const bool drop = classflag[method_class[v.m]] || classflag[v.d];
    if (!drop) out[atomicAdd(count_out, 1ull)] = v;
  }
}

// methods of the affected classes, compacted into a list (any order)
__global__ void affected_methods(const int32_t *method_class, const uint8_t *classflag, int32_t M, int32_t *list,
                                 unsigned long long *n) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    if (classflag[method_class[x]]) list[atomicAdd(n, 1ull)] = (int32_t)x;
}

// candidate rows of the other methods: the affected classes (none for the
// methods of affected classes, whose rows are evaluated in full)
__global__ void candidate_lengths(const int32_t *method_class, const uint8_t *classflag, int32_t M, int32_t nA,
                                  int64_t *len) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    len[x] = classflag[method_class[x]] ? 0 : (int64_t)nA;
}

// one warp per method row
__global__ void candidate_fill(const int32_t *method_class, const uint8_t *classflag, const int64_t *rowptr,
                               const int32_t *alist, int32_t nA, int32_t M, int32_t *dst) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < M; x += nw) {
    if (classflag[method_class[x]]) continue;
    int32_t *row = dst + rowptr[x];
    for (int32_t j = lane; j < nA; j += 32) row[j] = alist[j];
  }
}

__global__ void marks_from_kept(const mm_move *kept, const unsigned long long *count, int64_t cap,
                                uint8_t *mark) {
  const int64_t n = min((int64_t)*count, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mark[kept[i].m] = 1;
}

// ---------------------------------------------------------------- host helpers

void build_mirror(mm_system *s) {
  EditMirror &mr = s->mirror;
  cudaStream_t st = s->stream;
  const int64_t M = s->M;
  std::vector<int64_t> arp(M + 1), crp(M + 1);
  std::vector<int32_t> ai(std::max<int64_t>(s->n_acc, 1)), ci(std::max<int64_t>(s->n_call, 1));
  mr.method_class.resize(M);
  mr.attr_class.resize(s->A);
  if (M) {
    MM_CUDA_TRY(cudaMemcpyAsync(arp.data(), s->acc_rowptr, sizeof(int64_t) * (M + 1), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaMemcpyAsync(crp.data(), s->call_rowptr, sizeof(int64_t) * (M + 1), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaMemcpyAsync(mr.method_class.data(), s->method_class, sizeof(int32_t) * M, cudaMemcpyDeviceToHost,
                                st));
  }
  if (s->A)
    MM_CUDA_TRY(cudaMemcpyAsync(mr.attr_class.data(), s->attr_class, sizeof(int32_t) * s->A, cudaMemcpyDeviceToHost,
                                st));
  if (s->n_acc)
    MM_CUDA_TRY(cudaMemcpyAsync(ai.data(), s->acc_idx, sizeof(int32_t) * s->n_acc, cudaMemcpyDeviceToHost, st));
  if (s->n_call)
    MM_CUDA_TRY(cudaMemcpyAsync(ci.data(), s->call_idx, sizeof(int32_t) * s->n_call, cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  mr.acc.assign(M, {});
  mr.calls.assign(M, {});
  for (int64_t x = 0; x < M; ++x) {
    mr.acc[x].assign(ai.begin() + arp[x], ai.begin() + arp[x + 1]);
    mr.calls[x].assign(ci.begin() + crp[x], ci.begin() + crp[x + 1]);
  }
  mr.callers.assign(M, {});
  for (int64_t y = 0; y < M; ++y)
    for (int32_t t : mr.calls[y]) mr.callers[t].push_back((int32_t)y);
  mr.cls_n.assign(s->c, 0);
  mr.cls_a.assign(s->c, 0);
  for (int32_t C : mr.method_class) mr.cls_n[C]++;
  for (int32_t C : mr.attr_class) mr.cls_a[C]++;
  mr.acc_cap = s->n_acc;
  mr.call_cap = s->n_call;
  mr.nu_cap = s->n_acc + s->n_call;
  mr.ready = true;
}

// Replace a device buffer by a larger one (copying `keep` elements).
template <class T>
T *regrow(mm_system *s, T *old, int64_t keep, int64_t new_count) {
  T *p = s->arena.get<T>(new_count);
  if (keep > 0) MM_CUDA_TRY(cudaMemcpyAsync(p, old, sizeof(T) * keep, cudaMemcpyDeviceToDevice, s->stream));
  s->arena.forget(old);
  return p;
}

// Returns whether a buffer was regrown (its old content is then gone and the
// structures built in it must be rebuilt).
bool ensure_capacity(mm_system *s, int64_t n_acc, int64_t n_call) {
  EditMirror &mr = s->mirror;
  bool regrown = false;
  if (n_acc > mr.acc_cap) {
    regrown = true;
    int64_t cap = n_acc + n_acc / 4 + 1024;
    s->acc_idx = regrow(s, s->acc_idx, s->n_acc, cap);
    s->own_list = regrow(s, s->own_list, (int64_t)0, cap);
    mr.acc_cap = cap;
  }
  if (n_call > mr.call_cap) {
    regrown = true;
    int64_t cap = n_call + n_call / 4 + 1024;
    s->call_idx = regrow(s, s->call_idx, s->n_call, cap);
    s->r_list = regrow(s, s->r_list, (int64_t)0, cap);
    mr.call_cap = cap;
  }
  if (n_acc + n_call > mr.nu_cap) {
    regrown = true;
    int64_t cap = (n_acc + n_call) + (n_acc + n_call) / 4 + 2048;
    s->mg_dst = regrow(s, s->mg_dst, (int64_t)0, cap);
    s->mg_cnt = regrow(s, s->mg_cnt, (int64_t)0, cap);
    s->l_list = regrow(s, s->l_list, (int64_t)0, cap);
    s->l_s = regrow(s, s->l_s, (int64_t)0, cap);
    s->l_x = regrow(s, s->l_x, (int64_t)0, cap);
    s->cpk = regrow(s, s->cpk, (int64_t)0, 2 * cap);
    mr.nu_cap = cap;
  }
  return regrown;
}

// Recompute the load-time summary (largest class) from the per-class sizes of the mirror.
void resummarise(mm_system *s) {
  const EditMirror &mr = s->mirror;
  int32_t nmax = 0;
  for (int32_t C = 0; C < s->c; ++C) nmax = std::max<int32_t>(nmax, mr.cls_n[C]);
  s->summary.max_class_methods = nmax;
}

// Insert (value at rank) into or remove (the element at rank) from row m of a device CSR.
void patch_row(mm_system *s, int32_t *arr, int64_t *rowptr, int64_t n_before, int32_t m, int32_t rank,
               bool insert, int32_t value) {
  cudaStream_t st = s->stream;
  int32_t *tmp = static_cast<int32_t *>(s->edit_ws.need(sizeof(int32_t) * (size_t)(n_before + 1), st));
  const unsigned g = grid_for(n_before + 1);
  if (insert) {
    csr_save<<<g, TPB, 0, st>>>(arr, n_before, rowptr, m, rank, 0, tmp);
    MM_LAUNCH_CHECK();
    csr_write<<<g, TPB, 0, st>>>(arr, n_before + 1, rowptr, m, rank, 1, tmp, value);
    MM_LAUNCH_CHECK();
  } else {
    csr_save<<<g, TPB, 0, st>>>(arr, n_before, rowptr, m, rank, 1, tmp);
    MM_LAUNCH_CHECK();
    csr_write<<<g, TPB, 0, st>>>(arr, n_before - 1, rowptr, m, rank, 0, tmp, 0);
    MM_LAUNCH_CHECK();
  }
  rowptr_add<<<grid_for(s->M), TPB, 0, st>>>(rowptr, m + 1, s->M, insert ? 1 : -1);
  MM_LAUNCH_CHECK();
}

}  // namespace

void apply_edit(mm_system *s, const mm_edit &e) {
  if (!s->metrics_ready) throw MmError{MM_EINVAL, "apply_edit: call mm_compute_metrics first"};
  if (e.m < 0 || e.m >= s->M) throw MmError{MM_EINVAL, "apply_edit: method id out of range"};
  if (!s->mirror.ready) build_mirror(s);
  EditMirror &mr = s->mirror;
  cudaStream_t st = s->stream;
  const int32_t m = e.m, C = mr.method_class[m];
  std::set<int32_t> affected;
  affected.insert(C);
  int64_t n_acc = s->n_acc, n_call = s->n_call;
  // which metric branches the edit can change: LCOM (accesses to own
  // attributes, membership) and the coupling (uses across classes)
  bool lcom_changes = false, coupling_changes = false, regrown = false;
  // ---- validate on the mirror, then patch the device CSR
  switch (e.kind) {
    case MM_EDIT_ADD_ACCESS:
    case MM_EDIT_REMOVE_ACCESS: {
      if (e.target < 0 || e.target >= s->A) throw MmError{MM_EINVAL, "apply_edit: attribute id out of range"};
      auto &row = mr.acc[m];
      auto it = std::lower_bound(row.begin(), row.end(), e.target);
      const bool present = it != row.end() && *it == e.target;
      const int32_t rank = (int32_t)(it - row.begin());
      if (e.kind == MM_EDIT_ADD_ACCESS) {
        if (present) throw MmError{MM_EEXIST, "apply_edit: the method already accesses this attribute"};
        regrown = ensure_capacity(s, n_acc + 1, n_call);
        patch_row(s, s->acc_idx, s->acc_rowptr, n_acc, m, rank, true, e.target);
        row.insert(it, e.target);
        ++n_acc;
      } else {
        if (!present) throw MmError{MM_ENOTFOUND, "apply_edit: the method does not access this attribute"};
        patch_row(s, s->acc_idx, s->acc_rowptr, n_acc, m, rank, false, 0);
        row.erase(it);
        --n_acc;
      }
      affected.insert(mr.attr_class[e.target]);
      lcom_changes = mr.attr_class[e.target] == C;                   // sharing counts own attributes only
      coupling_changes = mr.attr_class[e.target] != C && s->cbo_attrs;  // a foreign access is a use
      break;
    }
    case MM_EDIT_ADD_CALL:
    case MM_EDIT_REMOVE_CALL: {
      if (e.target < 0 || e.target >= s->M) throw MmError{MM_EINVAL, "apply_edit: callee id out of range"};
      if (e.target == m) throw MmError{MM_EINVAL, "apply_edit: a method cannot call itself"};
      auto &row = mr.calls[m];
      auto it = std::lower_bound(row.begin(), row.end(), e.target);
      const bool present = it != row.end() && *it == e.target;
      const int32_t rank = (int32_t)(it - row.begin());
      auto &cr = mr.callers[e.target];
      if (e.kind == MM_EDIT_ADD_CALL) {
        if (present) throw MmError{MM_EEXIST, "apply_edit: the call already exists"};
        regrown = ensure_capacity(s, n_acc, n_call + 1);
        patch_row(s, s->call_idx, s->call_rowptr, n_call, m, rank, true, e.target);
        row.insert(it, e.target);
        cr.insert(std::lower_bound(cr.begin(), cr.end(), m), m);
        ++n_call;
      } else {
        if (!present) throw MmError{MM_ENOTFOUND, "apply_edit: the call does not exist"};
        patch_row(s, s->call_idx, s->call_rowptr, n_call, m, rank, false, 0);
        row.erase(it);
        cr.erase(std::lower_bound(cr.begin(), cr.end(), m));
        --n_call;
      }
      affected.insert(mr.method_class[e.target]);
      coupling_changes = mr.method_class[e.target] != C;  // calls never change LCOM
      break;
    }
    case MM_EDIT_MOVE: {
      const int32_t D = e.target;
      if (D < 0 || D >= s->c) throw MmError{MM_EINVAL, "apply_edit: class id out of range"};
      if (D == C) throw MmError{MM_EINVAL, "apply_edit: the method is already in that class"};
      affected.insert(D);
      for (int32_t t : mr.calls[m]) affected.insert(mr.method_class[t]);
      for (int32_t a : mr.acc[m]) affected.insert(mr.attr_class[a]);
      for (int32_t y : mr.callers[m]) affected.insert(mr.method_class[y]);
      set_i32<<<1, 1, 0, st>>>(s->method_class + m, D);
      MM_LAUNCH_CHECK();
      move_counts<<<1, 1, 0, st>>>(s->cls_n, C, D);
      MM_LAUNCH_CHECK();
      mr.method_class[m] = D;
      s->methods_by_class = false;  // the move breaks the grouping by class
      lcom_changes = coupling_changes = true;
      mr.cls_n[C]--;
      mr.cls_n[D]++;
      break;
    }
    default:
      throw MmError{MM_EINVAL, "apply_edit: unknown edit kind"};
  }
  s->n_acc = n_acc;
  s->n_call = n_call;
  s->edits++;
  resummarise(s);
  // ---- recompute the class metrics and the per-method move data
  const bool had_cache = s->kept_valid && !s->kept_lists;  // only the full cross product is maintained
  s->kept_valid = false;
  const uint32_t kmask = s->kept_mask;
  const int32_t kmin = s->kept_min;
  patch_structures(s, e.kind, m, e.target, C);  // class lists, ranks and fan-in: only what the edit changed
  // the LCOM pair counts of the classes whose membership or own accesses changed
  LcomClasses only;
  only.cls[only.n++] = mr.method_class[m];  // m's class now (D after a move)
  if (e.kind == MM_EDIT_MOVE) only.cls[only.n++] = C;
  for (int k = 0; k < only.n; ++k) only.members[k] = mr.cls_n[only.cls[k]];
  build_metrics(s, lcom_changes || regrown, coupling_changes || regrown, regrown ? nullptr : &only);
  build_move_precompute(s);
  if (!had_cache) return;
  // ---- incremental update of the cached kept moves
  mm_move *kept;
  uint8_t *mark;
  int64_t cap;
  s->kept_valid = true;
  if (!kept_cache(s, &kept, &mark, &cap)) return;
  const int32_t c = s->c, M = s->M;
  const int32_t nA = (int32_t)affected.size();
  int64_t rows = 0;
  for (int32_t Y : affected) rows += mr.cls_n[Y];
  // rows: the methods of the affected classes to every class (dense tiles over
  // a method list); columns: every other method to the affected classes
  // (candidate lists of nA entries)
  const int64_t n_inc = ((int64_t)M - rows) * nA;
  // scratch: classflag[c], alist[nA], len/rowptr[M+1], dst[n_inc], tmp kept[cap], counters, method list[rows]
  size_t off_flag = 0, off_alist = (size_t)(c + 255) / 256 * 256;
  size_t off_rp = off_alist + ((size_t)nA * 4 + 255) / 256 * 256;
  size_t off_dst = off_rp + ((size_t)(M + 1) * 8 + 255) / 256 * 256;
  size_t off_tmp = off_dst + ((size_t)n_inc * 4 + 255) / 256 * 256;
  size_t off_cnt = off_tmp + (size_t)cap * sizeof(mm_move);
  size_t off_ml = off_cnt + 256;
  size_t bytes = off_ml + ((size_t)rows * 4 + 255) / 256 * 256 + 256;
  char *w = static_cast<char *>(s->edit_ws.need(bytes, st));
  uint8_t *classflag = reinterpret_cast<uint8_t *>(w + off_flag);
  int32_t *alist = reinterpret_cast<int32_t *>(w + off_alist);
  int64_t *rowptr = reinterpret_cast<int64_t *>(w + off_rp);
  int32_t *dst = reinterpret_cast<int32_t *>(w + off_dst);
  mm_move *tmp = reinterpret_cast<mm_move *>(w + off_tmp);
  unsigned long long *cnt2 = reinterpret_cast<unsigned long long *>(w + off_cnt);
  unsigned long long *nml = cnt2 + 1;
  int32_t *mlist = reinterpret_cast<int32_t *>(w + off_ml);
  std::vector<uint8_t> hflag(c, 0);
  std::vector<int32_t> hal(affected.begin(), affected.end());
  for (int32_t Y : affected) hflag[Y] = 1;
  MM_CUDA_TRY(cudaMemcpyAsync(classflag, hflag.data(), (size_t)c, cudaMemcpyHostToDevice, st));
  MM_CUDA_TRY(cudaMemcpyAsync(alist, hal.data(), sizeof(int32_t) * (size_t)nA, cudaMemcpyHostToDevice, st));
  // drop the moves whose method or destination is affected
  MM_CUDA_TRY(cudaMemsetAsync(cnt2, 0, sizeof(unsigned long long), st));
  kept_filter<<<grid_for(cap), TPB, 0, st>>>(kept, s->d_u64 + 1, cap, classflag, s->method_class, tmp, cnt2);
  MM_LAUNCH_CHECK();
  MM_CUDA_TRY(cudaMemcpyAsync(kept, tmp, sizeof(mm_move) * (size_t)cap, cudaMemcpyDeviceToDevice, st));
  MM_CUDA_TRY(cudaMemcpyAsync(s->d_u64 + 1, cnt2, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
  // evaluate the affected rows and columns, appending kept moves
  mm_criteria crit{kmask, kmin};
  if (rows > 0) {
    MM_CUDA_TRY(cudaMemsetAsync(nml, 0, sizeof(unsigned long long), st));
    MM_CUDA_TRY(cudaMemsetAsync(mlist, 0, sizeof(int32_t) * (size_t)rows, st));  // every entry a valid id
    affected_methods<<<grid_for(M), TPB, 0, st>>>(s->method_class, classflag, M, mlist, nml);
    MM_LAUNCH_CHECK();
    eval_dense_kept_subset(s, crit, mlist, (int32_t)rows, kept, cap, s->d_u64 + 1, mark);
  }
  if (n_inc > 0) {
    candidate_lengths<<<grid_for(M), TPB, 0, st>>>(s->method_class, classflag, M, nA, rowptr);
    MM_LAUNCH_CHECK();
    scan_exclusive_i64(rowptr, rowptr, M, rowptr + M, s->sort_ws, st);
    candidate_fill<<<grid_for((int64_t)M * 32), TPB, 0, st>>>(s->method_class, classflag, rowptr, alist, nA, M, dst);
    MM_LAUNCH_CHECK();
    eval_csr_kept_append(s, crit, rowptr, dst, kept, cap, s->d_u64 + 1, mark);
  }
  MM_CUDA_TRY(cudaMemsetAsync(mark, 0, (size_t)M, st));
  marks_from_kept<<<grid_for(cap), TPB, 0, st>>>(kept, s->d_u64 + 1, cap, mark);
  MM_LAUNCH_CHECK();
  s->kept_valid = true;
  s->kept_mask = kmask;
  s->kept_min = kmin;
}

namespace {
__global__ void scatter_moves(const int2 *moves, int32_t n, int32_t *method_class) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) method_class[moves[k].x] = moves[k].y;
}
}  // namespace

// Rounds of non-conflicting kept moves (see mm_apply_sequence in mmref.h).
void apply_sequence(mm_system *s, const mm_criteria &crit, int32_t rounds, int32_t per_round, mm_applied_move *out,
                    int64_t cap, int64_t *n_applied) {
  if (!s->metrics_ready) throw MmError{MM_EINVAL, "apply_sequence: call mm_compute_metrics first"};
  check_criteria_public(crit);
  if (rounds < 0) throw MmError{MM_EINVAL, "apply_sequence: rounds < 0"};
  if (cap > 0 && !out) throw MmError{MM_EINVAL, "apply_sequence: out is NULL"};
  ensure_mirror(s);
  EditMirror &mr = s->mirror;
  cudaStream_t st = s->stream;
  int64_t applied = 0;
  std::vector<uint8_t> used((size_t)s->c, 0);
  std::vector<uint8_t> moved((size_t)s->M, 0);
  for (int32_t rnd = 0; rnd < rounds; ++rnd) {
    // the kept moves of the current state, sorted in the suggestion order
    int64_t K = 0, nm = 0;
    suggest_moves(s, crit, nullptr, 0, nullptr, MM_PTR_HOST, &K, &nm);
    if (K == 0) break;
    std::vector<mm_move> kept((size_t)K);
    suggest_moves(s, crit, nullptr, (int32_t)std::min<int64_t>(K, INT32_MAX), kept.data(), MM_PTR_HOST, &K, &nm);
    // greedy: disjoint affected classes, each method once
    std::fill(used.begin(), used.end(), 0);
    std::fill(moved.begin(), moved.end(), 0);
    std::vector<int2> take;
    std::vector<int32_t> aff;
    for (const mm_move &mv : kept) {
      if (per_round > 0 && (int32_t)take.size() >= per_round) break;
      const int32_t m = mv.m, D = mv.d;
      if (moved[(size_t)m]) continue;
      aff.clear();
      aff.push_back(mr.method_class[(size_t)m]);
      aff.push_back(D);
      for (int32_t t : mr.calls[(size_t)m]) aff.push_back(mr.method_class[(size_t)t]);
      for (int32_t a : mr.acc[(size_t)m]) aff.push_back(mr.attr_class[(size_t)a]);
      for (int32_t y : mr.callers[(size_t)m]) aff.push_back(mr.method_class[(size_t)y]);
      bool clash = false;
      for (int32_t Y : aff) clash |= used[(size_t)Y] != 0;
      if (clash) continue;
      for (int32_t Y : aff) used[(size_t)Y] = 1;
      moved[(size_t)m] = 1;
      take.push_back(make_int2(m, D));
    }
    // apply the round: owner classes on the device and in the mirror, class sizes, then the metrics
    for (const int2 &mv : take) {
      const int32_t C = mr.method_class[(size_t)mv.x];
      if (out && applied < cap) out[applied] = mm_applied_move{rnd, mv.x, C, mv.y};
      ++applied;
      mr.method_class[(size_t)mv.x] = mv.y;
      mr.cls_n[(size_t)C]--;
      mr.cls_n[(size_t)mv.y]++;
    }
    int2 *dmv = static_cast<int2 *>(s->edit_ws.need(sizeof(int2) * take.size(), st));
    MM_CUDA_TRY(cudaMemcpyAsync(dmv, take.data(), sizeof(int2) * take.size(), cudaMemcpyHostToDevice, st));
    scatter_moves<<<(unsigned)ceil_div((int64_t)take.size(), 256), 256, 0, st>>>(dmv, (int32_t)take.size(),
                                                                                s->method_class);
    MM_LAUNCH_CHECK();
    MM_CUDA_TRY(cudaMemcpyAsync(s->cls_n, mr.cls_n.data(), sizeof(int32_t) * (size_t)s->c, cudaMemcpyHostToDevice, st));
    s->methods_by_class = false;
    s->edits += (int64_t)take.size();
    resummarise(s);
    s->kept_valid = false;
    build_structures(s);
    build_metrics(s);
    build_move_precompute(s);
    MM_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors copied from go out of scope
  }
  if (n_applied) *n_applied = applied;
}

// Copy the system's current CSR (after edits) to host buffers.
void export_system(mm_system *s, int32_t *method_class, int32_t *attr_class, int64_t *acc_rowptr,
                   int32_t *acc_idx, int64_t *call_rowptr, int32_t *call_idx) {
  cudaStream_t st = s->stream;
  const int64_t M = s->M;
  if (method_class && M) MM_CUDA_TRY(cudaMemcpyAsync(method_class, s->method_class, 4 * M, cudaMemcpyDeviceToHost, st));
  if (attr_class && s->A) MM_CUDA_TRY(cudaMemcpyAsync(attr_class, s->attr_class, 4 * s->A, cudaMemcpyDeviceToHost, st));
  if (acc_rowptr) MM_CUDA_TRY(cudaMemcpyAsync(acc_rowptr, s->acc_rowptr, 8 * (M + 1), cudaMemcpyDeviceToHost, st));
  if (acc_idx && s->n_acc) MM_CUDA_TRY(cudaMemcpyAsync(acc_idx, s->acc_idx, 4 * s->n_acc, cudaMemcpyDeviceToHost, st));
  if (call_rowptr) MM_CUDA_TRY(cudaMemcpyAsync(call_rowptr, s->call_rowptr, 8 * (M + 1), cudaMemcpyDeviceToHost, st));
  if (call_idx && s->n_call)
    MM_CUDA_TRY(cudaMemcpyAsync(call_idx, s->call_idx, 4 * s->n_call, cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- edit resolution for request streams

void ensure_mirror(mm_system *s) {
  if (!s->mirror.ready) build_mirror(s);
}

// Turn an intended edit (kind, method, random selector) into a concrete valid
// edit against the system's current state: an addition picks the first
// absent attribute / callee from a position given by the selector; a removal
// picks one of the existing entries (or becomes the matching addition when
// there is none); a move picks one of the other classes.
mm_edit resolve_edit(mm_system *s, int32_t kind, int32_t m, uint64_t sel) {
  ensure_mirror(s);
  const EditMirror &mr = s->mirror;
  if (m < 0 || m >= s->M) throw MmError{MM_EINVAL, "resolve_edit: method id out of range"};
  mm_edit e{kind, m, 0, 0};
  const auto &acc = mr.acc[m];
  const auto &calls = mr.calls[m];
  if (kind == MM_EDIT_REMOVE_ACCESS && acc.empty()) kind = MM_EDIT_ADD_ACCESS;
  if (kind == MM_EDIT_REMOVE_CALL && calls.empty()) kind = MM_EDIT_ADD_CALL;
  if (kind == MM_EDIT_ADD_ACCESS && (int64_t)acc.size() >= s->A) kind = MM_EDIT_MOVE;
  if (kind == MM_EDIT_ADD_CALL && (int64_t)calls.size() >= (int64_t)s->M - 1) kind = MM_EDIT_MOVE;
  if (kind == MM_EDIT_MOVE && s->c < 2) throw MmError{MM_EINVAL, "resolve_edit: no other class to move to"};
  e.kind = kind;
  switch (kind) {
    case MM_EDIT_ADD_ACCESS: {
      int32_t a = (int32_t)(sel % (uint64_t)s->A);
      while (std::binary_search(acc.begin(), acc.end(), a)) a = (a + 1) % s->A;
      e.target = a;
      break;
    }
    case MM_EDIT_REMOVE_ACCESS:
      e.target = acc[sel % acc.size()];
      break;
    case MM_EDIT_ADD_CALL: {
      int32_t t = (int32_t)(sel % (uint64_t)s->M);
      while (t == m || std::binary_search(calls.begin(), calls.end(), t)) t = (t + 1) % s->M;
      e.target = t;
      break;
    }
    case MM_EDIT_REMOVE_CALL:
      e.target = calls[sel % calls.size()];
      break;
    case MM_EDIT_MOVE: {
      int32_t d = (int32_t)(sel % (uint64_t)(s->c - 1));
      e.target = d + (d >= mr.method_class[m] ? 1 : 0);
      break;
    }
    default:
      throw MmError{MM_EINVAL, "resolve_edit: unknown edit kind"};
  }
  return e;
}
