// Device-wide primitives: exclusive scan and a stable LSD radix sort.
//
// The sort is the "segmented sort" the coupling metric needs (class-use keys
// (Y, E) sorted by source class, Sec. II.B CBO) and it also builds the
// class -> method lists, the callers of each method and the per-method use
// lists.  Keys are sorted 8 bits per pass; within a 4096-key tile every warp
// ranks its keys with __match_any_sync so equal digits keep their input order,
// which makes every pass, and hence the sort, stable and deterministic.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mm_internal.cuh"

// Set by a bounded device-side wait that ran out (see scan_onepass) when no
// system or batch is named by the calling thread's WaitScope.
__device__ unsigned int g_wait_fault = 0;

namespace {
// The fault word (and the stall counter of the test hook) of the system or
// batch whose entry point is running on this thread.
thread_local uint32_t *t_fault = nullptr;
thread_local int32_t *t_stall = nullptr;
}  // namespace

WaitScope::WaitScope(uint32_t *fault, int32_t *stall) : prev_fault(t_fault), prev_stall(t_stall) {
  t_fault = fault;
  t_stall = stall;
}
WaitScope::~WaitScope() {
  t_fault = prev_fault;
  t_stall = prev_stall;
}

uint32_t *current_fault_word() {
  if (t_fault) return t_fault;
  void *p = nullptr;
  MM_CUDA_TRY(cudaGetSymbolAddress(&p, g_wait_fault));
  return static_cast<uint32_t *>(p);
}

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ T block_exclusive_sum(T v, T *total) {
  __shared__ T warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
    if (lane == SCAN_THREADS / 32 - 1) *total = wi;
  }
  __syncthreads();
  T r = incl - v + warp_sums[warp];
  __syncthreads();
  return r;
}

// Small inputs: one block of 32 warps; thread t scans its own run of
// ceil(n / 1024) <= 16 consecutive elements (so an in-place scan is safe), the
// block scans the 1,024 run totals, then every thread writes its run.
constexpr int SCAN1_THREADS = 1024;
constexpr int SCAN1_ROWS = 16;
constexpr int64_t SCAN1_MAX = (int64_t)SCAN1_THREADS * SCAN1_ROWS;  // larger inputs: the one-pass scan

// Element access of the scans: ld(k) is element k of the input as the sum
// type, st(k, v) writes output k (plain arrays, or fields of records).
template <class Tin, class Tout>
struct ArrLoad {
  const Tin *p;
  __device__ __forceinline__ Tout operator()(int64_t k) const { return (Tout)p[k]; }
};
template <class Tout>
struct ArrStore {
  Tout *p;
  __device__ __forceinline__ void operator()(int64_t k, Tout v) const { p[k] = v; }
};
// summary records: the marked words of record k, and its first packed word
struct SummaryLoad {
  const uint2 *p;
  __device__ __forceinline__ int64_t operator()(int64_t k) const { return (int64_t)__popc(p[k].x); }
};
struct SummaryStore {
  uint2 *p;
  __device__ __forceinline__ void operator()(int64_t k, int64_t v) const { p[k].y = (uint32_t)v; }
};

template <class Tout, class Ld, class St>
__global__ void __launch_bounds__(SCAN1_THREADS) scan_single_block(Ld ld, St st, int64_t n, Tout *total_out) {
  pdl_wait();
  __shared__ Tout wsum[SCAN1_THREADS / 32];
  __shared__ Tout block_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ipt = (int)((n + SCAN1_THREADS - 1) / SCAN1_THREADS);
  const int64_t b0 = (int64_t)threadIdx.x * ipt;
  Tout v[SCAN1_ROWS];
  Tout sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN1_ROWS; ++i) {
    const int64_t k = b0 + i;
    v[i] = (i < ipt && k < n) ? ld(k) : Tout(0);
    sum += v[i];
  }
  Tout incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Tout y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const Tout w = wsum[lane];
    Tout wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Tout y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - w;
    if (lane == 31) block_total = wi;
  }
  __syncthreads();
  Tout run = wsum[warp] + incl - sum;
#pragma unroll
  for (int i = 0; i < SCAN1_ROWS; ++i) {
    const int64_t k = b0 + i;
    if (i < ipt && k < n) st(k, run);
    run += v[i];
  }
  if (threadIdx.x == 0 && total_out) *total_out = block_total;
}

// Larger inputs: one pass over tiles of SCAN_TILE elements with decoupled
// look-back (Merrill and Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", 2016).  Tiles are numbered in the order blocks start,
// so every tile a block waits for belongs to a block that is already running.
// A tile publishes its total (flag 1), then, once the tiles before it are
// summed, its inclusive prefix (flag 2), both as one 64-bit word (sum << 2 |
// flag).  The wait is bounded: past the limit the block records a fault in
// the fault word of the calling system (read back by the host at its next
// synchronisation), sums the input before its tile itself and goes on, so the
// output is exact whether or not the wait ran out.
constexpr unsigned long long SP_AGG = 1ull, SP_INCL = 2ull;
constexpr int SP_WAIT_LIMIT = 1 << 21;  // about a second of polling
constexpr int SP_STALL_LIMIT = 1 << 12;  // the test hook's short limit

// stall != 0 (test hook): tile 0 holds back its state until another tile's
// look-back has run out (or four limits have passed), so the tiles after it
// take the fallback below.
template <class Tout, class Ld, class St>
__global__ void __launch_bounds__(SCAN_THREADS) scan_onepass(Ld ld, St st, int64_t n, Tout *total_out,
                                                              unsigned long long *status, unsigned int *tile_ctr,
                                                              unsigned int *fault, int wait_limit, int stall) {
  pdl_wait();
  static_assert(sizeof(Tout) <= 8, "scan sums are packed with a 2-bit flag");
  __shared__ unsigned int s_tile;
  __shared__ Tout s_prefix;
  __shared__ Tout s_agg;
  __shared__ Tout tot;
  __shared__ int64_t s_j;  // >= 0: the look-back gave up at tile s_j
  __shared__ unsigned long long s_w;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(tile_ctr, 1u);
    s_j = -1;
  }
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tile0 = tile * SCAN_TILE;
  // the tile goes through shared memory: loaded and stored in warp-contiguous
  // order (coalesced), scanned as SCAN_ITEMS consecutive elements per thread
  // (one padding element per 32 keeps both orders free of bank conflicts)
  __shared__ Tout s_x[SCAN_TILE + SCAN_TILE / 32];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int k = i * SCAN_THREADS + (int)threadIdx.x;
    s_x[k + (k >> 5)] = tile0 + k < n ? ld(tile0 + k) : Tout(0);
  }
  __syncthreads();
  Tout v[SCAN_ITEMS];
  Tout sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int k = (int)threadIdx.x * SCAN_ITEMS + i;
    v[i] = s_x[k + (k >> 5)];
    sum += v[i];
  }
  Tout ex = block_exclusive_sum<Tout>(sum, &tot);
  volatile unsigned long long *vs = status;
  if (threadIdx.x < 32) {
    // warp 0 looks back over 32 predecessor states at a time: lane k reads
    // tile j - k; the nearest inclusive state ends the walk, aggregates before
    // it are summed, a state not yet published holds the walk at that tile
    const uint32_t lane = threadIdx.x;
    const Tout agg = tot;
    Tout prefix = 0;
    if (lane == 0) {
      s_agg = agg;
      if (tile == 0 && stall) {
        volatile unsigned int *vf = fault;
        for (int spins = 0; *vf == 0u && spins < 4 * wait_limit; ++spins) __nanosleep(32);
      }
      if (tile > 0) {
        atomicExch(&status[tile], ((unsigned long long)agg << 2) | SP_AGG);
        __threadfence();  // the state is visible before any output of this tile
      }
    }
    __syncwarp();
    int spins = 0;
    for (int64_t j = tile - 1; j >= 0;) {
      const int64_t t = j - (int64_t)lane;
      const unsigned long long w = t >= 0 ? (unsigned long long)vs[t] : (unsigned long long)SP_INCL;  // before tile 0: an inclusive 0
      const unsigned long long f = w & 3ull;
      const uint32_t incl = __ballot_sync(0xffffffffu, f == SP_INCL);
      const uint32_t wait = __ballot_sync(0xffffffffu, f == 0ull);
      const int32_t lim = incl ? __ffs(incl) - 1 : 31;  // lanes 0 .. lim matter
      const uint32_t upto = lim == 31 ? 0xffffffffu : (2u << lim) - 1u;
      const uint32_t held = wait & upto;
      const int32_t take = held ? __ffs(held) - 1 : lim + 1;  // lanes 0 .. take-1 are summed
      Tout part = (int32_t)lane < take ? (Tout)(w >> 2) : Tout(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      prefix += part;
      if (!held) {
        if (incl) break;
        j -= 32;
        continue;
      }
      j -= take;  // the walk resumes at the tile not yet published
      if (++spins > wait_limit) {
        if (lane == 0) {
          atomicOr(fault, 1u);
          s_j = j;
        }
        break;
      }
      if (take == 0) __nanosleep(32);
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  // Fallback after a wait that ran out: the block walks on from tile s_j,
  // taking a published state where there is one and otherwise summing the
  // tile's input itself.  A tile publishes its state before it writes any
  // output, so an input summed while the state still reads 0 afterwards is
  // the original input even when the scan runs in place.
  while (s_j >= 0) {
    const int64_t j = s_j;
    if (threadIdx.x == 0) s_w = vs[j];
    __syncthreads();
    const unsigned long long w = s_w;
    if ((w & 3ull) != 0ull) {
      if (threadIdx.x == 0) {
        s_prefix += (Tout)(w >> 2);
        s_j = (w & 3ull) == SP_INCL ? -1 : j - 1;
      }
    } else {
      Tout part = 0;
      const int64_t lo = j * (int64_t)SCAN_TILE, hi = min(lo + (int64_t)SCAN_TILE, n);
      for (int64_t k = lo + threadIdx.x; k < hi; k += SCAN_THREADS) part += ld(k);
      block_exclusive_sum<Tout>(part, &tot);
      if (threadIdx.x == 0) {
        __threadfence();
        if ((vs[j] & 3ull) == 0ull) {  // still unpublished: the input read was intact
          s_prefix += tot;
          s_j = j - 1;
        }  // else: published meanwhile, take its state on the next pass
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const Tout prefix = s_prefix, agg = s_agg;
    atomicExch(&status[tile], ((unsigned long long)(prefix + agg) << 2) | SP_INCL);
    __threadfence();
    if (total_out && tile0 + SCAN_TILE >= n) *total_out = prefix + agg;  // the last tile
  }
  if (tile == 0) __syncthreads();  // tile 0's first state comes here: publish before writing (in-place scans)
  ex += s_prefix;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int k = (int)threadIdx.x * SCAN_ITEMS + i;
    s_x[k + (k >> 5)] = ex;
    ex += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int k = i * SCAN_THREADS + (int)threadIdx.x;
    if (tile0 + k < n) st(tile0 + k, s_x[k + (k >> 5)]);
  }
}

template <class Tout, class Ld, class St>
void scan_exclusive_with(Ld ld, St sto, int64_t n, Tout *total_dev, Scratch &ws, cudaStream_t st) {
  if (n <= 0) {
    if (total_dev) MM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(Tout), st));
    return;
  }
  if (n <= SCAN1_MAX) {
    pdl_launch(scan_single_block<Tout, Ld, St>, 1, SCAN1_THREADS, 0, st, ld, sto, n, total_dev);
    MM_LAUNCH_CHECK();
    return;
  }
  const int64_t nb = ceil_div(n, SCAN_TILE);
  // tile states and the tile counter, cleared together
  unsigned long long *status = static_cast<unsigned long long *>(ws.need(sizeof(unsigned long long) * (size_t)(nb + 1), st));
  MM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)(nb + 1), st));
  int stall = 0;
  if (t_stall && *t_stall > 0) {  // test hook: this scan's look-back runs out
    --*t_stall;
    stall = 1;
  }
  pdl_launch(scan_onepass<Tout, Ld, St>, (unsigned)nb, SCAN_THREADS, 0, st, ld, sto, n, total_dev, status,
             reinterpret_cast<unsigned int *>(status + nb), current_fault_word(),
             stall ? SP_STALL_LIMIT : SP_WAIT_LIMIT, stall);
  MM_LAUNCH_CHECK();
}

template <class Tin, class Tout>
void scan_exclusive(const Tin *in, Tout *out, int64_t n, Tout *total_dev, Scratch &ws, cudaStream_t st) {
  scan_exclusive_with<Tout>(ArrLoad<Tin, Tout>{in}, ArrStore<Tout>{out}, n, total_dev, ws, st);
}

// ---------------------------------------------------------------- radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys
constexpr int RS_RADIX = 256;

template <class K>
__global__ void radix_upsweep(const K *keys, int64_t n, int shift, uint32_t *hist, int64_t ntiles) {
  pdl_wait();
  __shared__ uint32_t cnt[RS_RADIX];
  for (int i = threadIdx.x; i < RS_RADIX; i += RS_THREADS) cnt[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    int64_t k = base + i;
    if (k < n) atomicAdd(&cnt[(uint32_t)(keys[k] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_RADIX; d += RS_THREADS) hist[(int64_t)d * ntiles + blockIdx.x] = cnt[d];
}

// Scatter pass: every key's rank among the tile's keys of its digit (warps in
// order, then rows, then lanes: the input order, so the pass is stable).  The
// tile is first staged in shared memory in digit order, then written out
// position by position, so that keys of one digit leave as a contiguous run
// (coalesced stores instead of one scattered store per key).
template <class K, bool VALS>
__global__ void __launch_bounds__(RS_THREADS) radix_downsweep(const K *keys_in, const uint32_t *vals_in,
                                                               K *keys_out, uint32_t *vals_out, int64_t n,
                                                               int shift, const uint32_t *offsets,
                                                               int64_t ntiles) {
  static_assert(RS_THREADS == RS_RADIX, "one digit per thread in the per-digit passes");
  pdl_wait();
  __shared__ uint32_t wcnt[RS_WARPS][RS_RADIX];
  __shared__ uint32_t tstart[RS_RADIX];  // first tile-local position of each digit
  __shared__ uint32_t goff[RS_RADIX];    // first output position of each digit for this tile
  __shared__ K skey[RS_TILE];
  __shared__ uint8_t sdig[RS_TILE];
  __shared__ uint32_t ttotal;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
  const int64_t wbase = tbase + (int64_t)warp * (RS_ITEMS * 32);
  const uint32_t lt = (1u << lane) - 1u;
  // per key: its rank among the warp's keys of its digit (< 512) << 8 | digit,
  // or ~0 past the end; the keys themselves are read again when staged
  uint32_t rd[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t idx = wbase + r * 32 + lane;
    bool valid = idx < n;
    const K k = valid ? keys_in[idx] : K(0);
    uint32_t d = (uint32_t)(k >> shift) & 0xffu;
    uint32_t tag = valid ? d : (0x1000u + lane);  // invalid lanes never match
    uint32_t peers = __match_any_sync(0xffffffffu, tag);
    uint32_t before = 0;
    if (valid) before = wcnt[warp][d];
    rd[r] = valid ? ((before + __popc(peers & lt)) << 8) | d : 0xffffffffu;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread d): the warps' prefixes, the tile's count and its output offset
  const int d0 = threadIdx.x;
  uint32_t run = 0;
  for (int w = 0; w < RS_WARPS; ++w) {
    const uint32_t t = wcnt[w][d0];
    wcnt[w][d0] = run;
    run += t;
  }
  goff[d0] = offsets[(int64_t)d0 * ntiles + blockIdx.x];
  const uint32_t ts = block_exclusive_sum<uint32_t>(run, &ttotal);  // synchronises the block
  tstart[d0] = ts;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (rd[r] != 0xffffffffu) {
      const uint32_t d = rd[r] & 0xffu;
      const uint32_t lp = tstart[d] + wcnt[warp][d] + (rd[r] >> 8);
      skey[lp] = keys_in[wbase + r * 32 + lane];
      sdig[lp] = (uint8_t)d;
    }
  }
  __syncthreads();
  const int cnt = (int)min((int64_t)RS_TILE, n - tbase);
  for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
    const uint32_t d = sdig[i];
    keys_out[goff[d] + (uint32_t)i - tstart[d]] = skey[i];
  }
  if (VALS) {
    __syncthreads();  // the keys are out: their stage takes the values
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      if (rd[r] != 0xffffffffu) {
        const uint32_t d = rd[r] & 0xffu;
        sval[tstart[d] + wcnt[warp][d] + (rd[r] >> 8)] = vals_in[wbase + r * 32 + lane];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
      const uint32_t d = sdig[i];
      vals_out[goff[d] + (uint32_t)i - tstart[d]] = sval[i];
    }
  }
}

template <class K>
void radix_sort(K *keys, K *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int nbits, Scratch &ws,
                cudaStream_t st) {
  if (n <= 1 || nbits <= 0) return;
  if (n >= (int64_t)0xffffffffLL) throw MmError{MM_EINVAL, "radix sort: more than 2^32-1 keys"};
  int64_t ntiles = ceil_div(n, RS_TILE);
  int64_t nh = ntiles * RS_RADIX;
  // scratch: hist (uint32 nh) + the scan's tile states and tile counter
  size_t hist_bytes = sizeof(uint32_t) * (size_t)nh;
  size_t part_bytes = sizeof(unsigned long long) * (size_t)(ceil_div(nh, SCAN_TILE) + 2);
  char *base = static_cast<char *>(ws.need(hist_bytes + part_bytes + 256, st));
  uint32_t *hist = reinterpret_cast<uint32_t *>(base);
  Scratch part_ws;  // view into the same allocation for the scan partials
  part_ws.ptr = base + ((hist_bytes + 255) / 256) * 256;
  part_ws.cap = part_bytes + 256 - ((hist_bytes + 255) / 256 * 256 - hist_bytes);
  int passes = (nbits + 7) / 8;
  K *kin = keys, *kout = keys_alt;
  uint32_t *vin = vals, *vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    pdl_launch(radix_upsweep<K>, (unsigned)ntiles, RS_THREADS, 0, st, kin, n, shift, hist, ntiles);
    MM_LAUNCH_CHECK();
    scan_exclusive<uint32_t, uint32_t>(hist, hist, nh, nullptr, part_ws, st);
    if (vals)
      pdl_launch(radix_downsweep<K, true>, (unsigned)ntiles, RS_THREADS, 0, st, kin, vin, kout, vout, n, shift, hist,
                                                                      ntiles);
    else
      pdl_launch(radix_downsweep<K, false>, (unsigned)ntiles, RS_THREADS, 0, st, kin, nullptr, kout, nullptr, n, shift,
                                                                       hist, ntiles);
    MM_LAUNCH_CHECK();
    K *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
  }
  if (kin != keys) {
    MM_CUDA_TRY(cudaMemcpyAsync(keys, kin, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (vals) MM_CUDA_TRY(cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  }
}

}  // namespace

namespace {
// Zero up to three buffers (16-byte aligned) in one launch with 16-byte stores.
struct ZeroSegs {
  void *p[3];
  size_t bytes[3];
};

__global__ void zero_segments_kernel(ZeroSegs z) {
  pdl_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 *q = static_cast<uint4 *>(z.p[k]);
    const int64_t n16 = (int64_t)(z.bytes[k] / 16);
    for (int64_t i = t; i < n16; i += stride) q[i] = make_uint4(0u, 0u, 0u, 0u);
    unsigned char *tail = static_cast<unsigned char *>(z.p[k]) + 16 * n16;
    if (t < (int64_t)(z.bytes[k] % 16)) tail[t] = 0;
  }
}
}  // namespace

void zero_buffers(void *a, size_t na, void *b, size_t nb, void *c, size_t nc, cudaStream_t st) {
  ZeroSegs z{{a, b, c}, {a ? na : 0, b ? nb : 0, c ? nc : 0}};
  const size_t most = std::max(z.bytes[0], std::max(z.bytes[1], z.bytes[2]));
  if (most == 0) return;
  const int64_t blocks = std::min<int64_t>(ceil_div((int64_t)(most / 16) + 1, 256), B300_SMS * 16);
  pdl_launch(zero_segments_kernel, (unsigned)blocks, 256, 0, st, z);
  MM_LAUNCH_CHECK();
}

void read_wait_fault(uint32_t *host, const uint32_t *fault_dev, cudaStream_t st) {
  MM_CUDA_TRY(cudaMemcpyAsync(host, fault_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
}

void raise_wait_fault(uint32_t host_word, uint32_t *fault_dev, cudaStream_t st, const char *what) {
  if (!host_word) return;
  MM_CUDA_TRY(cudaMemsetAsync(fault_dev, 0, sizeof(uint32_t), st));
  throw MmError{MM_ETIMEOUT, std::string(what) + ": a bounded device-side wait gave up (its result was completed "
                                                 "by the fallback and is exact)"};
}

void check_wait_fault(uint32_t *fault_dev, cudaStream_t st, const char *what) {
  uint32_t h = 0;
  read_wait_fault(&h, fault_dev, st);
  MM_CUDA_TRY(cudaStreamSynchronize(st));
  raise_wait_fault(h, fault_dev, st, what);
}

// One block scans tile 1 of a two-tile input while tile 0 is never processed
// (the tile counter starts at 1), so its look-back wait runs out and the
// fallback sums tile 0's input.  Returns the fault word the host reads
// afterwards, or 2 if the output is not the exact prefix sum of the input.
uint32_t stalled_scan_probe() {
  int32_t *in = nullptr;
  int64_t *out = nullptr;
  unsigned long long *status = nullptr;
  const int64_t n = 2 * (int64_t)SCAN_TILE;
  MM_CUDA_TRY(cudaMalloc(&in, sizeof(int32_t) * (size_t)n));
  MM_CUDA_TRY(cudaMalloc(&out, sizeof(int64_t) * (size_t)n));
  MM_CUDA_TRY(cudaMalloc(&status, sizeof(unsigned long long) * 4));
  std::vector<int32_t> h_in((size_t)n);
  for (int64_t k = 0; k < n; ++k) h_in[(size_t)k] = (int32_t)(k % 7);
  MM_CUDA_TRY(cudaMemcpy(in, h_in.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
  MM_CUDA_TRY(cudaMemset(status, 0, sizeof(unsigned long long) * 4));
  const unsigned int first = 1;
  MM_CUDA_TRY(cudaMemcpy(status + 2, &first, sizeof(first), cudaMemcpyHostToDevice));
  uint32_t *fault = reinterpret_cast<uint32_t *>(status + 3);
  pdl_launch(scan_onepass<int64_t, ArrLoad<int32_t, int64_t>, ArrStore<int64_t>>, 1, SCAN_THREADS, 0, 0,
             ArrLoad<int32_t, int64_t>{in}, ArrStore<int64_t>{out}, n, (int64_t *)nullptr, status,
             reinterpret_cast<unsigned int *>(status + 2), fault, SP_WAIT_LIMIT, 0);
  MM_LAUNCH_CHECK();
  MM_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t h_fault = 0;
  MM_CUDA_TRY(cudaMemcpy(&h_fault, fault, sizeof(h_fault), cudaMemcpyDeviceToHost));
  std::vector<int64_t> h_out((size_t)n);
  MM_CUDA_TRY(cudaMemcpy(h_out.data(), out, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost));
  int64_t run = 0;  // tile 1's outputs: the exclusive prefix over both tiles
  for (int64_t k = 0; k < n; ++k) {
    if (k >= SCAN_TILE && h_out[(size_t)k] != run) h_fault = 2;
    run += h_in[(size_t)k];
  }
  cudaFree(in);
  cudaFree(out);
  cudaFree(status);
  return h_fault;
}

void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Scratch &ws,
                        cudaStream_t st) {
  scan_exclusive<int64_t, int64_t>(in, out, n, total_dev, ws, st);
}

void scan_exclusive_i32to64(const int32_t *in, int64_t *out, int64_t n, Scratch &ws, cudaStream_t st,
                            int64_t *total_dev) {
  scan_exclusive<int32_t, int64_t>(in, out, n, total_dev, ws, st);
}

void scan_summary_first(uint2 *csum, int64_t n, Scratch &ws, cudaStream_t st) {
  scan_exclusive_with<int64_t>(SummaryLoad{csum}, SummaryStore{csum}, n, (int64_t *)nullptr, ws, st);
}

void radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int nbits,
                    Scratch &ws, cudaStream_t st) {
  radix_sort<uint64_t>(keys, keys_alt, vals, vals_alt, n, nbits, ws, st);
}

void radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int nbits,
                    Scratch &ws, cudaStream_t st) {
  radix_sort<uint32_t>(keys, keys_alt, vals, vals_alt, n, nbits, ws, st);
}

