// Rule R3 (Sec. III.A, third rule): relocations out of classes whose coupling
// is high.  A class is high when its CBO is above the average CBO of all the
// classes (compared exactly: CBO(C) * c > sum of CBO); its methods are moved
// tentatively to every class they use (the L entries with a use edge: calls,
// and attribute reads when those count for CBO), each candidate is evaluated
// by the move kernels (its record holds dCBO of the origin and the
// destination), and a move is kept when the origin's CBO drops and the
// destination's does not rise.  Suggestions are ordered by the method's
// fan-in + fan-out (descending: the rule starts with the methods of highest
// fan-in and fan-out), then dCBO(origin) + dCBO(destination), method, class.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mm_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, TPB), B300_SMS * 32));
}

__global__ void cbo_total(const int32_t *cbo, int32_t c, unsigned long long *sum) {
  unsigned long long v = 0;
  for (int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; C < c; C += (int64_t)gridDim.x * blockDim.x)
    v += (unsigned long long)cbo[C];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(sum, v);
}

// classes used by x when its class is high (else none): row lengths, then the classes
__global__ void r3_rows(const MoveHdr *hdr, const int4 *l_list, const int32_t *cbo, const unsigned long long *sum,
                        int32_t c, int32_t M, int64_t *len, int32_t *high_count) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
    const MoveHdr h = hdr[x];
    int64_t n = 0;
    if ((unsigned long long)cbo[h.w0.x] * (unsigned long long)c > *sum)
      for (int32_t e = 0; e < h.w0.z; ++e) n += l_list[h.w0.y + e].y > 0;
    len[x] = n;
  }
  for (int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; C < c; C += (int64_t)gridDim.x * blockDim.x)
    if ((unsigned long long)cbo[C] * (unsigned long long)c > *sum) atomicAdd(high_count, 1);
}

__global__ void r3_fill(const MoveHdr *hdr, const int4 *l_list, const int64_t *rowptr, int32_t M, int32_t *dst) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rowptr[x], n = rowptr[x + 1] - b;
    if (!n) continue;
    const MoveHdr h = hdr[x];
    int64_t o = b;
    for (int32_t e = 0; e < h.w0.z; ++e) {
      const int4 v = l_list[h.w0.y + e];
      if (v.y > 0) dst[o++] = v.x;  // L entries ascend by class
    }
  }
}

// keep: the origin's CBO drops, the destination's does not rise
__global__ void r3_keep(const int64_t *rowptr, const int32_t *dst, const mm_move_eval *rec, const int32_t *fan_in,
                        const int64_t *call_rowptr, int32_t M, mm_r3_move *out, unsigned long long *count) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    for (int64_t i = rowptr[x]; i < rowptr[x + 1]; ++i) {
      const mm_move_eval r = rec[i];
      if (r.dcbo_src < 0 && r.dcbo_dst <= 0) {
        mm_r3_move v;
        v.m = (int32_t)x;
        v.d = dst[i];
        v.fan_in = fan_in[x];
        v.fan_out = (int32_t)(call_rowptr[x + 1] - call_rowptr[x]);
        v.dcbo_src = r.dcbo_src;
        v.dcbo_dst = r.dcbo_dst;
        out[atomicAdd(count, 1ull)] = v;
      }
    }
}

}  // namespace

void suggest_r3(mm_system *s, int32_t k, mm_r3_move *out, int64_t *n_kept, int64_t *n_cand_out, int32_t *n_high) {
  if (!s->metrics_ready) throw MmError{MM_EINVAL, "suggest_r3: call mm_compute_metrics first"};
  if (k < 0 || (k > 0 && !out)) throw MmError{MM_EINVAL, "suggest_r3: bad k or out_topk"};
  cudaStream_t st = s->stream;
  const int32_t M = s->M, c = s->c;
  if (M == 0) {
    if (n_kept) *n_kept = 0;
    if (n_cand_out) *n_cand_out = 0;
    if (n_high) *n_high = 0;
    return;
  }
  char *w = static_cast<char *>(s->r1_ws.need(sizeof(int64_t) * ((size_t)M + 1) + 1024, st));
  int64_t *rowptr = reinterpret_cast<int64_t *>(w);
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(w + ((sizeof(int64_t) * ((size_t)M + 1) + 255) / 256 * 256));
  MM_CUDA_TRY(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), st));
  cbo_total<<<grid_for(c), TPB, 0, st>>>(s->cls_cbo, c, ctr);
  MM_LAUNCH_CHECK();
  r3_rows<<<grid_for(std::max<int64_t>(M, c)), TPB, 0, st>>>(s->hdr, s->l_list, s->cls_cbo, ctr, c, M, rowptr,
                                                            reinterpret_cast<int32_t *>(ctr + 1));
  MM_LAUNCH_CHECK();
  scan_exclusive_i64(rowptr, rowptr, M, rowptr + M, s->sort_ws, st);
  int64_t n_cand = 0;
  int32_t high = 0;
  MM_CUDA_TRY(cudaMemcpyAsync(&n_cand, rowptr + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaMemcpyAsync(&high, ctr + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_high) *n_high = high;
  if (n_cand_out) *n_cand_out = n_cand;
  std::vector<mm_r3_move> kept;
  if (n_cand > 0) {
    const size_t db = (sizeof(int32_t) * (size_t)n_cand + 255) / 256 * 256;
    const size_t rb = (sizeof(mm_move_eval) * (size_t)n_cand + 255) / 256 * 256;
    char *b = static_cast<char *>(s->sim_keys_ws.need(db + rb + sizeof(mm_r3_move) * (size_t)n_cand + 256, st));
    int32_t *dst = reinterpret_cast<int32_t *>(b);
    mm_move_eval *rec = reinterpret_cast<mm_move_eval *>(b + db);
    mm_r3_move *kv = reinterpret_cast<mm_r3_move *>(b + db + rb);
    r3_fill<<<grid_for(M), TPB, 0, st>>>(s->hdr, s->l_list, rowptr, M, dst);
    MM_LAUNCH_CHECK();
    eval_lists_records(s, rowptr, dst, rec);
    r3_keep<<<grid_for(M), TPB, 0, st>>>(rowptr, dst, rec, s->fan_in, s->call_rowptr, M, kv, ctr + 2);
    MM_LAUNCH_CHECK();
    unsigned long long K = 0;
    MM_CUDA_TRY(cudaMemcpyAsync(&K, ctr + 2, sizeof(K), cudaMemcpyDeviceToHost, st));
    MM_CUDA_TRY(cudaStreamSynchronize(st));
    kept.resize((size_t)K);
    if (K) {
      MM_CUDA_TRY(cudaMemcpyAsync(kept.data(), kv, sizeof(mm_r3_move) * (size_t)K, cudaMemcpyDeviceToHost, st));
      MM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    std::sort(kept.begin(), kept.end(), [](const mm_r3_move &a, const mm_r3_move &b) {
      const int32_t fa = a.fan_in + a.fan_out, fb = b.fan_in + b.fan_out;
      if (fa != fb) return fa > fb;
      const int32_t da = a.dcbo_src + a.dcbo_dst, dbb = b.dcbo_src + b.dcbo_dst;
      if (da != dbb) return da < dbb;
      if (a.m != b.m) return a.m < b.m;
      return a.d < b.d;
    });
  }
  if (n_kept) *n_kept = (int64_t)kept.size();
  const int64_t nout = std::min<int64_t>(k, (int64_t)kept.size());
  if (nout > 0) std::copy(kept.begin(), kept.begin() + nout, out);
}
