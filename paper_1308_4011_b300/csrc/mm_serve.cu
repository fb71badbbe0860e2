// Serving: a request loop that keeps many evolving systems resident on the
// device, applies code edits as they arrive and answers each with the
// system's updated suggestions (the abstract's "continuously gathered while
// the system evolves").
//
// * Continuous batching: n_slots worker threads, each with its own CUDA
//   stream, take requests as they arrive; requests that arrive while others
//   are on the GPU are started as soon as a slot is free, and their kernels
//   overlap on the device.  Requests of one system run one at a time in
//   arrival order (so every result is the same alone and in the mix).
// * Admission by memory footprint: a system is made resident (loaded, metrics
//   computed, suggestions cached) when a request needs it and the resident
//   footprint stays within the budget, evicting idle systems least recently
//   used first (their current arrays are copied back to the host).
// * Each request: resolve the edit against the current state, mm_apply_edit
//   (incremental re-evaluation), then the top-k suggestions back to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "mm_internal.cuh"

namespace {

struct Served {
  int32_t c = 0, M = 0, A = 0, cbo_attrs = 1;
  std::vector<int32_t> method_class, attr_class, acc_idx, call_idx;
  std::vector<int64_t> acc_rowptr, call_rowptr;
  mm_system *dev = nullptr;
  int64_t footprint = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

struct Snapshot {
  int64_t request;
  int32_t system;
  int32_t c, M, A;
  std::vector<int32_t> method_class, attr_class, acc_idx, call_idx;
  std::vector<int64_t> acc_rowptr, call_rowptr;
};

// Device bytes a system will hold once resident (arena + scratch), fitted to
// measured footprints; corrected to the measured value after the load.
int64_t estimate_footprint(const Served &v) {
  const int64_t nu = (int64_t)v.acc_idx.size() + (int64_t)v.call_idx.size();
  const int64_t aw = ((int64_t)v.c + 127) / 128 * 4;
  const int64_t sized = 160 * (int64_t)v.M + 128 * nu + 96 * (int64_t)v.c + 8 * aw * v.c + aw * v.c / 2;
  return sized / 10 * 9 + (2 << 20);
}

}  // namespace

struct mm_server {
  mm_server_config cfg{};
  std::vector<Served> sys;
  std::vector<cudaStream_t> streams;
  int device = 0;
  int64_t resident_bytes = 0;
  uint64_t clock = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Snapshot> snaps;
  mm_server_stats stats{};
};

namespace {

template <class F>
mm_status guarded(F &&f) {
  try {
    f();
    mm_set_error("");
    return MM_OK;
  } catch (const MmError &e) {
    mm_set_error(e.msg);
    return e.st;
  } catch (...) {
    mm_set_error("unexpected exception");
    return MM_ECUDA;
  }
}

void check(mm_status st) {
  if (st != MM_OK) throw MmError{st, mm_last_error()};
}

// Copy a resident system's arrays back to its host copy and free it (caller holds mu).
void evict(mm_server *sv, int32_t i) {
  Served &v = sv->sys[i];
  mm_system_info inf{};
  check(mm_system_info_get(v.dev, &inf));
  v.acc_idx.resize(inf.n_acc);
  v.call_idx.resize(inf.n_call);
  check(mm_export_system(v.dev, v.method_class.data(), v.attr_class.data(), v.acc_rowptr.data(), v.acc_idx.data(),
                         v.call_rowptr.data(), v.call_idx.data()));
  mm_free_system(v.dev);
  v.dev = nullptr;
  sv->resident_bytes -= v.footprint;
  v.footprint = 0;
  sv->stats.evictions++;
}

// Make system i resident for a worker (i is marked busy by the dispatcher).
// Returns MM_EBUDGET if it can never fit.
mm_status admit(mm_server *sv, int32_t i, cudaStream_t st) {
  std::unique_lock<std::mutex> lk(sv->mu);
  Served &v = sv->sys[i];
  if (v.dev) return MM_OK;
  const int64_t need = estimate_footprint(v);
  if (need > sv->cfg.budget_bytes) return MM_EBUDGET;
  for (;;) {
    while (sv->resident_bytes + need > sv->cfg.budget_bytes) {
      int32_t victim = -1;
      for (int32_t j = 0; j < (int32_t)sv->sys.size(); ++j) {
        const Served &u = sv->sys[j];
        if (u.dev && !u.busy && (victim < 0 || u.last_use < sv->sys[victim].last_use)) victim = j;
      }
      if (victim < 0) break;
      evict(sv, victim);
    }
    if (sv->resident_bytes + need <= sv->cfg.budget_bytes) break;
    sv->cv.wait(lk);  // every other resident system is busy: wait for one to finish
  }
  sv->resident_bytes += need;
  v.footprint = need;
  lk.unlock();
  mm_system_desc d{};
  d.n_classes = v.c;
  d.n_methods = v.M;
  d.n_attrs = v.A;
  d.ptr_kind = MM_PTR_HOST;
  d.n_acc = (int64_t)v.acc_idx.size();
  d.n_call = (int64_t)v.call_idx.size();
  d.method_class = v.method_class.data();
  d.attr_class = v.attr_class.data();
  d.acc_rowptr = v.acc_rowptr.data();
  d.acc_idx = v.acc_idx.data();
  d.call_rowptr = v.call_rowptr.data();
  d.call_idx = v.call_idx.data();
  d.cbo_attrs = v.cbo_attrs;
  mm_system *s = nullptr;
  mm_status rc = mm_load_system(&d, st, &s);
  if (rc == MM_OK) rc = mm_compute_metrics(s, nullptr, nullptr, MM_PTR_DEVICE);
  if (rc == MM_OK) rc = mm_suggest_moves(s, &sv->cfg.crit, nullptr, 0, nullptr, MM_PTR_HOST, nullptr, nullptr);
  lk.lock();
  if (rc != MM_OK) {
    if (s) mm_free_system(s);
    sv->resident_bytes -= need;
    v.footprint = 0;
    return rc;
  }
  mm_system_info inf{};
  mm_system_info_get(s, &inf);
  sv->resident_bytes += inf.device_bytes - need;
  v.footprint = inf.device_bytes;
  v.dev = s;
  sv->stats.loads++;
  return MM_OK;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" {

MMREF_API mm_status mm_server_create(const mm_server_config *cfg, mm_server **out) {
  if (out) *out = nullptr;
  mm_server *sv = nullptr;
  mm_status st = guarded([&] {
    if (!cfg || !out || cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->topk < 0 || cfg->budget_bytes <= 0)
      throw MmError{MM_EINVAL, "server_create: bad configuration"};
    check_criteria_public(cfg->crit);
    sv = new mm_server();
    sv->cfg = *cfg;
    MM_CUDA_TRY(cudaGetDevice(&sv->device));
    for (int i = 0; i < cfg->n_slots; ++i) {
      cudaStream_t s;
      MM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      sv->streams.push_back(s);
    }
    *out = sv;
  });
  if (st != MM_OK && sv) {
    for (auto s : sv->streams) cudaStreamDestroy(s);
    delete sv;
  }
  return st;
}

MMREF_API mm_status mm_server_add_system(mm_server *sv, const mm_system_desc *d, int32_t *id) {
  return guarded([&] {
    if (!sv || !d || !id || d->ptr_kind != MM_PTR_HOST) throw MmError{MM_EINVAL, "server_add_system: bad arguments"};
    Served v;
    v.c = d->n_classes;
    v.M = d->n_methods;
    v.A = d->n_attrs;
    v.cbo_attrs = d->cbo_attrs;
    v.method_class.assign(d->method_class, d->method_class + d->n_methods);
    v.attr_class.assign(d->attr_class, d->attr_class + d->n_attrs);
    v.acc_rowptr.assign(d->acc_rowptr, d->acc_rowptr + d->n_methods + 1);
    v.call_rowptr.assign(d->call_rowptr, d->call_rowptr + d->n_methods + 1);
    v.acc_idx.assign(d->acc_idx, d->acc_idx + d->n_acc);
    v.call_idx.assign(d->call_idx, d->call_idx + d->n_call);
    std::lock_guard<std::mutex> lk(sv->mu);
    *id = (int32_t)sv->sys.size();
    sv->sys.push_back(std::move(v));
  });
}

MMREF_API mm_status mm_server_run(mm_server *sv, const mm_request *req, int64_t n, mm_response *resp,
                                  mm_move *topk, int64_t snapshot_every) {
  return guarded([&] {
    if (!sv || (n > 0 && (!req || !resp))) throw MmError{MM_EINVAL, "server_run: bad arguments"};
    for (int64_t i = 0; i < n; ++i) {
      if (req[i].system < 0 || req[i].system >= (int32_t)sv->sys.size())
        throw MmError{MM_EINVAL, "server_run: unknown system"};
      if (i && req[i].arrival_s < req[i - 1].arrival_s) throw MmError{MM_EINVAL, "server_run: arrivals not sorted"};
    }
    const int32_t K = sv->cfg.topk;
    const auto t0 = std::chrono::steady_clock::now();
    std::deque<int64_t> pending;   // arrived, not started (arrival order)
    std::deque<int64_t> work;      // assigned to a slot, waiting for a worker
    int64_t next = 0, done = 0;
    int32_t free_slots = sv->cfg.n_slots;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<char> slot_busy(sv->cfg.n_slots, 0);
    auto worker = [&](int w) {
      cudaStream_t st = sv->streams[w];
      for (;;) {
        int64_t i;
        {
          std::unique_lock<std::mutex> lk(sv->mu);
          sv->cv.wait(lk, [&] { return stop || !work.empty(); });
          if (stop && work.empty()) return;
          i = work.front();
          work.pop_front();
        }
        mm_response &r = resp[i];
        r.slot = w;
        r.start_s = seconds_since(t0);
        const int32_t si = req[i].system;
        mm_status rc = admit(sv, si, st);
        mm_system *s = sv->sys[si].dev;
        if (rc == MM_OK) rc = mm_set_stream(s, st);
        if (rc == MM_OK) {
          try {
            r.edit = resolve_edit(s, req[i].kind, req[i].m, req[i].selector);
            rc = MM_OK;
          } catch (const MmError &e) {
            rc = e.st;
          }
        }
        if (rc == MM_OK) rc = mm_apply_edit(s, &r.edit);
        int64_t nk = 0, nm = 0;
        if (rc == MM_OK)
          rc = mm_suggest_moves(s, &sv->cfg.crit, nullptr, K, topk ? topk + i * (int64_t)K : nullptr, MM_PTR_HOST,
                                &nk, &nm);
        r.n_kept = nk;
        r.n_methods_with_kept = nm;
        if (rc == MM_OK && snapshot_every > 0 && i % snapshot_every == 0) {
          Snapshot sn;
          mm_system_info inf{};
          mm_system_info_get(s, &inf);
          sn.request = i;
          sn.system = si;
          sn.c = inf.n_classes;
          sn.M = inf.n_methods;
          sn.A = inf.n_attrs;
          sn.method_class.resize(sn.M);
          sn.attr_class.resize(sn.A);
          sn.acc_rowptr.resize(sn.M + 1);
          sn.call_rowptr.resize(sn.M + 1);
          sn.acc_idx.resize(inf.n_acc);
          sn.call_idx.resize(inf.n_call);
          rc = mm_export_system(s, sn.method_class.data(), sn.attr_class.data(), sn.acc_rowptr.data(),
                                sn.acc_idx.data(), sn.call_rowptr.data(), sn.call_idx.data());
          std::lock_guard<std::mutex> lk(sv->mu);
          sv->snaps.push_back(std::move(sn));
        }
        r.status = rc;
        r.done_s = seconds_since(t0);
        {
          std::lock_guard<std::mutex> lk(sv->mu);
          sv->sys[si].busy = false;
          sv->sys[si].last_use = ++sv->clock;
          ++free_slots;
          ++done;
          if (rc == MM_OK) sv->stats.served++;
          else sv->stats.failed++;
        }
        sv->cv.notify_all();
      }
    };
    for (int w = 0; w < sv->cfg.n_slots; ++w) workers.emplace_back(worker, w);
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      while (done < n) {
        const double now = seconds_since(t0);
        while (next < n && req[next].arrival_s <= now) {
          resp[next] = mm_response{};
          resp[next].arrival_s = req[next].arrival_s;
          pending.push_back(next++);
        }
        // start what can start: a free slot, and the request's system idle with
        // no earlier request of that system still waiting
        std::vector<char> seen(sv->sys.size(), 0);
        for (auto it = pending.begin(); it != pending.end() && free_slots > 0;) {
          const int32_t si = req[*it].system;
          if (seen[si] || sv->sys[si].busy) {
            seen[si] = 1;
            ++it;
            continue;
          }
          seen[si] = 1;
          sv->sys[si].busy = true;
          --free_slots;
          work.push_back(*it);
          it = pending.erase(it);
          sv->cv.notify_all();
        }
        if (done >= n) break;
        if (next < n) {
          const auto wake = t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                     std::chrono::duration<double>(req[next].arrival_s));
          sv->cv.wait_until(lk, wake);
        } else {
          sv->cv.wait(lk);
        }
      }
      stop = true;
    }
    sv->cv.notify_all();
    for (auto &t : workers) t.join();
    sv->stats.wall_s += seconds_since(t0);
    sv->stats.resident_bytes = sv->resident_bytes;
  });
}

MMREF_API mm_status mm_server_stats_get(mm_server *sv, mm_server_stats *out) {
  return guarded([&] {
    if (!sv || !out) throw MmError{MM_EINVAL, "server_stats: bad arguments"};
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->resident_bytes = sv->resident_bytes;
    out->n_snapshots = (int64_t)sv->snaps.size();
  });
}

MMREF_API mm_status mm_server_snapshot(mm_server *sv, int64_t k, mm_snapshot_info *info, int32_t *method_class,
                                       int32_t *attr_class, int64_t *acc_rowptr, int32_t *acc_idx,
                                       int64_t *call_rowptr, int32_t *call_idx) {
  return guarded([&] {
    if (!sv || !info) throw MmError{MM_EINVAL, "server_snapshot: bad arguments"};
    std::lock_guard<std::mutex> lk(sv->mu);
    if (k < 0 || k >= (int64_t)sv->snaps.size()) throw MmError{MM_EINVAL, "server_snapshot: no such snapshot"};
    const Snapshot &s = sv->snaps[k];
    info->request = s.request;
    info->system = s.system;
    info->n_classes = s.c;
    info->n_methods = s.M;
    info->n_attrs = s.A;
    info->n_acc = (int64_t)s.acc_idx.size();
    info->n_call = (int64_t)s.call_idx.size();
    if (method_class) std::copy(s.method_class.begin(), s.method_class.end(), method_class);
    if (attr_class) std::copy(s.attr_class.begin(), s.attr_class.end(), attr_class);
    if (acc_rowptr) std::copy(s.acc_rowptr.begin(), s.acc_rowptr.end(), acc_rowptr);
    if (acc_idx) std::copy(s.acc_idx.begin(), s.acc_idx.end(), acc_idx);
    if (call_rowptr) std::copy(s.call_rowptr.begin(), s.call_rowptr.end(), call_rowptr);
    if (call_idx) std::copy(s.call_idx.begin(), s.call_idx.end(), call_idx);
  });
}

MMREF_API void mm_server_free(mm_server *sv) {
  if (!sv) return;
  for (auto &v : sv->sys)
    if (v.dev) mm_free_system(v.dev);
  for (auto s : sv->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete sv;
}

}  // extern "C"
