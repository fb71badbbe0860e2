#!/usr/bin/env python3
"""Benchmark of the Move Method metric engine on one B300 (or N replicas).

The bench line is the large workload: a synthetic system of 50,000 classes,
500,000 methods and 250,000 attributes (seed 2) whose candidate moves are
restricted, per method, to the classes it calls into or whose attributes it
reads plus 64 uniformly drawn others (33,448,382 candidates), evaluated with
all three metrics selected (LCOM_CK, LCOM_HS and CBO: source, destination and
the classes of the method's callers).  One step, through the C ABI with the
inputs resident in HBM:

  load_system -> compute_metrics -> evaluate_moves (16-byte records in HBM)
  -> suggest_moves (top-100 read back) -> free.

metric = candidate moves evaluated per second; every record is checked against
the CPU oracle through a digest of all records and the suggestion list.

Measured in the same run and reported as nested keys:
  medium   the 5,000-class, 60,000-method system (seed 1), full cross product
           (299,940,000 candidates), dense evaluation and its roofline;
  batched  256 systems (classes log-uniform in 100..20,000, seeds 100..355):
           one CUDA graph per run against 256 sequential calls;
  serving  64 resident systems (seeds 100..163) answering 100,000 edit
           requests: capacity, p50/p99 latency at half of it, every 1,000th
           state checked against the oracle;
  rules    the similarity values of the large system (values/s, pairs
           assessed/s), the LCOM/CBO variants of the large system, rule R1 on
           the medium system, rule R3 on the large system, four rounds of
           non-conflicting moves on the medium system.
The oracle checks run in a separate low-priority process started before the
first GPU call; its jobs are held until the bench line and the serving section
(both driven by host threads) are timed, and run beside the other nested
sections; the CPU baseline is timed after them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs an independent replica of the bench line
on its own GPU (weak scaling, no data-path collective); value = all ranks'
candidates / the slowest rank's time.  Only rank 0 runs the nested sections.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate moves evaluated/sec (bit-exact vs oracle)"
UNIT = "candidates/s"
WORKLOAD = ("large synthetic system: 50,000 classes, 500,000 methods, 250,000 attributes, seed 2; restricted "
            "candidates (classes each method uses + 64 uniform others); criteria LCOM_CK|LCOM_HS|CBO, 2 improved")
MEDIUM_WORKLOAD = "medium synthetic system: 5,000 classes, 60,000 methods, 30,000 attributes, seed 1; full cross product"
MASK_ALL = 7          # LCOM_CK | LCOM_HS | CBO
MASK_LCOM = 3         # LCOM_CK | LCOM_HS
MIN_IMPROVED = 2
TOPK = 100
L2_FLUSH_BYTES = 512 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant
# kernel of each workload, from a one-pass ncu capture (None once the kernel
# changes, until it is captured again)
EVAL_CSR_TRAFFIC_MASK7 = 986456064   # large restricted, eval_csr_grouped<records, kept>, all three metrics
EVAL_DENSE_TRAFFIC = 4771880448      # medium, eval_dense<records, kept>


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region (clocks + throttle reasons)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mm_bench_clocks_{os.getpid()}_rank{gpu_index}.csv")
        self.window = None  # (t0, t1) wall-clock seconds of the timed region

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(1.0)  # let nvidia-smi finish starting before any timing
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append(dict(t=ts, sm=float(parts[2]), smax=float(parts[3]), power=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], swp=parts[9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = rows
        if self.window:
            t0, t1 = self.window
            inside = [r for r in rows if t0 - 0.1 <= r["t"] <= t1 + 0.1] or rows
        rows = inside
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = sorted({name for r in rows for name, key in (("hw_slowdown", "hw"),
                                                                ("hw_thermal_slowdown", "hwt"),
                                                                ("sw_thermal_slowdown", "swt"),
                                                                ("sw_power_cap", "swp"))
                          if r[key].lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "reasons": reasons,
                "power_w_median": statistics.median(r["power"] for r in rows)}


# ---------------------------------------------------------------- helpers shared with the tests

def max_over_ranks(total_ms, dist, device):
    """The job's time: the slowest rank's (all-reduce MAX); the local time without
    a process group."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_cand, world, steps, total_ms):
    """Whole-job throughput: the candidates every replica evaluated in all
    steps over the job's time (weak scaling: each rank holds its own system)."""
    return n_cand * world * steps / (total_ms / 1e3)


def replica_seed(seed, rank):
    """Each rank evaluates an independent replica of the workload."""
    return seed + 1000 * rank


def metrics_digest(cls_rows, meth_rows) -> str:
    """SHA-256 of class metrics (n, a, P, Q, S, cbo) and method metrics
    (fan_in, fan_out, own, q), as int64 columns, for comparing the GPU's
    arrays with the oracle's in another process."""
    h = hashlib.sha256()
    for col in cls_rows + meth_rows:
        h.update(np.ascontiguousarray(np.asarray(col, dtype=np.int64)).tobytes())
    return h.hexdigest()


def full_rows_lists(system, methods):
    """Candidate lists holding, for each method in `methods`, every class other
    than its own (the full cross product restricted to those rows); other
    methods get no candidates."""
    c, M = system.n_classes, system.n_methods
    lens = np.zeros(M, dtype=np.int64)
    lens[methods] = c - 1
    rowptr = np.zeros(M + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    allc = np.arange(c, dtype=np.int32)
    dst = np.concatenate([np.delete(allc, system.method_class[m]) for m in methods]) if len(methods) else \
        np.zeros(0, dtype=np.int32)
    return rowptr, dst


# ---------------------------------------------------------------- oracle jobs (run in the verifier process)

def _verifier_init():
    try:
        os.nice(19)  # the GPU sections' host threads come first
    except OSError:
        pass


def job_oracle_lists(params, n_extra, cand_seed, mask, mi, topk):
    """O1 over a generated system with restricted candidate lists."""
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.generate(**params)
    rp, dst = synth.candidates(s, n_extra, seed=cand_seed)
    o = oracle.Oracle(s)
    r = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1)
    o.close()
    return {"digest": r.digest, "n_kept": r.n_kept, "n_mk": r.n_methods_with_kept,
            "top": [(int(k["m"]), int(k["d"])) for k in r.kept[:topk]]}


def job_oracle_full(params, mask, mi, topk):
    """O1 over a generated system's full cross product."""
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.generate(**params)
    o = oracle.Oracle(s)
    r = o.evaluate(mask=mask, min_improved=mi, method=1)
    o.close()
    return {"digest": r.digest, "n_kept": r.n_kept, "n_mk": r.n_methods_with_kept,
            "top": [(int(k["m"]), int(k["d"])) for k in r.kept[:topk]]}


def job_oracle_batched(params, rows, mask, mi):
    """One batched system: the digest of its metric arrays and of the
    evaluation of a seeded sample of full candidate rows."""
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.generate(**params)
    o = oracle.Oracle(s)
    cm, mm_ = o.class_metrics(), o.method_metrics()
    md = metrics_digest([cm[f] for f in ("n", "a", "P", "Q", "S", "cbo")],
                        [mm_[f] for f in ("fan_in", "fan_out", "own", "q")])
    rp, dst = full_rows_lists(s, rows)
    r = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1)
    o.close()
    return {"metrics": md, "rows_digest": r.digest, "n_cand": r.n_cand}


def job_oracle_snapshot(c, arrays, mask, mi, topk):
    """One served state: kept-move count and the first suggestions of the
    full cross product, and the digest of its metric arrays."""
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.System(c, len(arrays[0]), len(arrays[1]), *arrays)
    o = oracle.Oracle(s)
    cm, mm_ = o.class_metrics(), o.method_metrics()
    md = metrics_digest([cm[f] for f in ("n", "a", "P", "Q", "S", "cbo")],
                        [mm_[f] for f in ("fan_in", "fan_out", "own", "q")])
    r = o.evaluate(mask=mask, min_improved=mi, method=1)
    o.close()
    return {"n_kept": r.n_kept, "n_mk": r.n_methods_with_kept, "metrics": md,
            "top": [(int(k["m"]), int(k["d"])) for k in r.kept[:topk]], "n_cand": r.n_cand}


class _Deferred:
    """A job held until Verifier.start(); get() waits for its result."""

    def __init__(self, verifier, fn, args):
        self.verifier, self.fn, self.args, self.res = verifier, fn, args, None

    def get(self):
        self.verifier.start()
        return self.res.get()


class Verifier:
    """One spawned worker process (the oracle threads over all host cores),
    started before the first GPU call.  Jobs are held until start() (or the
    first get()), so that the host-driven timed sections do not share the
    host cores with them; after it they run as they are submitted."""

    def __init__(self):
        import multiprocessing as mp
        self.pool = mp.get_context("spawn").Pool(1, initializer=_verifier_init)
        self.held = []
        self.running = False

    def submit(self, fn, *args):
        job = _Deferred(self, fn, args)
        if self.running:
            job.res = self.pool.apply_async(fn, args)
        else:
            self.held.append(job)
        return job

    def start(self):
        self.running = True
        for job in self.held:
            job.res = self.pool.apply_async(job.fn, job.args)
        self.held = []

    def close(self):
        self.start()
        self.pool.close()
        self.pool.join()


# ---------------------------------------------------------------- the bench line: large restricted

def large_inputs(seed):
    from paper_1308_4011_b300 import synth
    params = dict(synth.LARGE)
    params["seed"] = seed
    system = synth.generate(**params, name="large")
    rp, dst = synth.candidates(system, synth.LARGE_EXTRA_CANDIDATES, seed=seed)
    return params, system, rp, dst


def run_large(args, rank, world, local_rank, verifier, dist):
    import torch
    from paper_1308_4011_b300 import mmref, synth

    dev = torch.device("cuda", local_rank)
    seed = replica_seed(synth.LARGE["seed"], rank)
    params, system, rp, dst = large_inputs(seed)
    c, M, n_cand = system.n_classes, system.n_methods, len(dst)
    stream = torch.cuda.current_stream(dev)
    dev_arrs = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
                (system.method_class, system.attr_class, system.acc_rowptr, system.acc_idx,
                 system.call_rowptr, system.call_idx)]
    rpd, dd = torch.from_numpy(rp).to(dev), torch.from_numpy(dst).to(dev)
    records = torch.empty(n_cand * 16, dtype=torch.uint8, device=dev)
    topk = np.zeros(TOPK, dtype=mmref.MOVE_DTYPE)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step(mask, kernel_ms=None):
        s = mmref.load_system(c, *dev_arrs, stream=stream)
        mmref.compute_metrics(s, None, None)
        mmref.evaluate_moves(s, mask, MIN_IMPROVED, rpd, dd, records=records)
        # the same device lists: the suggestion reuses the evaluation's check and hash
        out = mmref.suggest_moves(s, TOPK, mask, MIN_IMPROVED, rpd, dd, out=topk, lists_unchanged=True)
        if kernel_ms is not None:
            kernel_ms.append(s.last_eval_ms())  # the suggestion reused the evaluation's kept moves
        s.free()
        return out

    # correctness: digest of every record and the suggestions, against the oracle
    # (rank 0); the oracle's jobs are queued after the timed steps, so that
    # they do not share the host cores with them
    checks, gpu_side = {}, {}
    if rank == 0 and verifier is not None:
        for mask in (MASK_ALL, MASK_LCOM):
            s = mmref.load_system(c, *dev_arrs, stream=stream)
            mmref.compute_metrics(s, None, None)
            dig = torch.zeros(1, dtype=torch.int64, device=dev)
            mmref.evaluate_moves(s, mask, MIN_IMPROVED, rpd, dd, digest=dig)
            top_g, nk_g, nm_g = mmref.suggest_moves(s, TOPK, mask, MIN_IMPROVED, rpd, dd)
            s.free()
            gpu_side[mask] = (int(dig.cpu().numpy().view(np.uint64)[0]), nk_g, nm_g,
                              [(int(x["m"]), int(x["d"])) for x in top_g])

    def timed(mask, steps):
        step_ms, kern_ms = [], []
        for _ in range(args.warmup):
            step(mask)
        torch.cuda.synchronize(dev)
        launches0 = mmref.launch_count()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.time()
        for _ in range(steps):
            flush.fill_(1)  # L2 flush between steps, outside the timed events
            ev[0].record(stream)
            step(mask, kern_ms)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            step_ms.append(ev[0].elapsed_time(ev[1]))
        if dist:
            dist.barrier()
        return step_ms, kern_ms, mmref.launch_count() - launches0, (t0, time.time())

    with ClockSampler(local_rank) as clk:
        step_ms, kern_ms, launches, window = timed(MASK_ALL, args.steps)
        clk.mark(*window)
        time.sleep(0.3)
    step3_ms, kern3_ms, _, _ = timed(MASK_LCOM, args.steps)
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_value(n_cand, world, args.steps, total_ms)

    peak, peak_kind = _peaks()
    alg_bytes = 20 * n_cand  # 4-byte destination read + 16-byte record written per candidate
    kern_s = statistics.median(kern_ms) / 1e3
    achieved = alg_bytes / kern_s / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": EVAL_CSR_TRAFFIC_MASK7,
            "kernel": "eval_csr_grouped<records, kept>",
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": round(kern_s * 1e3, 4),
            "kernel_ms_source": "CUDA events recorded by the library around the launch on its stream "
                                "(mm_last_eval_ms), median over the timed steps"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/int64", "data": "synthetic (seeded generator; no datasets)",
            "config": {"workload": WORKLOAD, "n_classes": c, "n_methods": M, "n_attrs": system.n_attrs,
                       "candidates_per_step": n_cand,
                       "criteria": {"metric_mask": MASK_ALL, "min_improved": MIN_IMPROVED}, "topk": TOPK,
                       "parallelism": f"replicas x{world}",
                       "l2": "512 MB L2 flush between steps (outside the events)"},
            "roofline": roof, "gpu_launches": launches, "gpu_launches_per_step": launches / max(args.steps, 1),
            "clocks": clk.summary(),
            "step_ms_min_median_max": [round(min(step_ms), 3), round(statistics.median(step_ms), 3),
                                       round(max(step_ms), 3)],
            "lcom_only": {"criteria": {"metric_mask": MASK_LCOM, "min_improved": MIN_IMPROVED},
                          "value": job_value(n_cand, 1, args.steps, sum(step3_ms)),
                          "ms_per_step": sum(step3_ms) / args.steps,
                          "kernel_ms": round(statistics.median(kern3_ms), 4),
                          "roofline_frac": round(alg_bytes / (statistics.median(kern3_ms) / 1e3) / 1e9 / peak, 4)}}
    if rank == 0:
        line["e2e"] = run_large_e2e(args, system, rp, dst, dev, stream)
    for mask, got in gpu_side.items():
        checks[mask] = (verifier.submit(job_oracle_lists, params, synth.LARGE_EXTRA_CANDIDATES, seed, mask,
                                        MIN_IMPROVED, TOPK),) + got
    return line, checks, system


def run_large_e2e(args, system, rp, dst, dev, stream):
    """The same step through the C ABI from pinned host buffers: CSR and
    candidate lists copied in (the lists staged while the metrics are computed,
    then used by the evaluation and the suggestion), class and method metrics
    and the top-100 copied out; records stay in HBM."""
    import torch
    from paper_1308_4011_b300 import mmref

    c, M, n_cand = system.n_classes, system.n_methods, len(dst)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
              (system.method_class, system.attr_class, system.acc_rowptr, system.acc_idx,
               system.call_rowptr, system.call_idx)]
    rp_h, dst_h = torch.from_numpy(rp).pin_memory(), torch.from_numpy(dst).pin_memory()
    cls_h = torch.empty(c * 64, dtype=torch.uint8).pin_memory()
    meth_h = torch.empty(M * 16, dtype=torch.uint8).pin_memory()
    top_h = torch.empty(TOPK * 24, dtype=torch.uint8).pin_memory()
    records = torch.empty(n_cand * 16, dtype=torch.uint8, device=dev)
    h2d = sum(int(p.numel() * p.element_size()) for p in pinned) + rp.nbytes + dst.nbytes
    d2h = c * 64 + M * 16 + TOPK * 24 + 16

    def step():
        s = mmref.load_system(c, *pinned, stream=stream)
        mmref.stage_candidates(s, rp_h.numpy(), dst_h.numpy())  # copied while the metrics are computed
        mmref.compute_metrics(s, cls_h, meth_h)
        mmref.evaluate_moves(s, MASK_ALL, MIN_IMPROVED, rp_h.numpy(), dst_h.numpy(), records=records,
                             lists_unchanged=True)
        mmref.suggest_moves(s, TOPK, MASK_ALL, MIN_IMPROVED, rp_h.numpy(), dst_h.numpy(), out=top_h,
                            lists_unchanged=True)
        s.free()

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    # the bound of this step: its own pinned inputs copied to the device alone
    hosts = pinned + [rp_h, dst_h]
    devs = [torch.empty(h.shape, dtype=h.dtype, device=dev) for h in hosts]
    for _ in range(2):
        for d_, h_ in zip(devs, hosts):
            d_.copy_(h_, non_blocking=True)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for _ in range(5):
        for d_, h_ in zip(devs, hosts):
            d_.copy_(h_, non_blocking=True)
    torch.cuda.synchronize(dev)
    link_s = (time.perf_counter() - t1) / 5
    del devs
    ms = dt * 1e3 / args.steps
    return {"value": n_cand * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms,
            "host_link": {"h2d_gbs": round(h2d / link_s / 1e9, 1), "floor_ms": round(link_s * 1e3, 3),
                          "frac": round(link_s * 1e3 / ms, 3),
                          "note": "the step's pinned inputs copied to the device alone, one stream; "
                                  "frac = that time / the e2e step"},
            "note": "host CSR + candidate lists (pinned) -> device, metrics + top-100 back to host; records in HBM"}


def cpu_baseline_large(system, rp, dst, mask):
    """The CPU oracle as it stands (metrics by definition + incremental
    evaluation of every candidate, all host threads) on the whole bench
    workload."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(system)
    r = o.evaluate(mask=mask, min_improved=MIN_IMPROVED, cand_rowptr=rp, cand_dst=dst, method=1)
    dt = time.perf_counter() - t0
    o.close()
    return {"value": r.n_cand / dt, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"the whole workload: metrics of all classes + all {r.n_cand} candidates",
            "seconds": round(dt, 3)}


# ---------------------------------------------------------------- nested: medium dense

# the dense profiling case: 2,000 classes, 24,000 methods (768 MB of records, above L2)
DENSE_SMALL = dict(n_classes=2000, n_methods=24000, n_attrs=12000, max_class=80, seed=5, zipf_s=1.2, lambda_acc=3.0,
                   lambda_call=4.0, p_loc=0.70)


def run_medium(args, local_rank, verifier, params=None, workload=MEDIUM_WORKLOAD):
    """The full cross product of one system (the medium one by default), dense
    evaluation with records, timed step by step."""
    import torch
    from paper_1308_4011_b300 import mmref, synth

    dev = torch.device("cuda", local_rank)
    params = dict(synth.MEDIUM) if params is None else dict(params)
    system = synth.generate(**params, name="medium")
    c, M = system.n_classes, system.n_methods
    n_cand = M * (c - 1)
    stream = torch.cuda.current_stream(dev)
    job = verifier.submit(job_oracle_full, params, MASK_LCOM, MIN_IMPROVED, TOPK) if verifier else None
    dev_arrs = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
                (system.method_class, system.attr_class, system.acc_rowptr, system.acc_idx,
                 system.call_rowptr, system.call_idx)]
    records = torch.empty(n_cand * 16, dtype=torch.uint8, device=dev)
    topk = np.zeros(TOPK, dtype=mmref.MOVE_DTYPE)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step(kern=None):
        s = mmref.load_system(c, *dev_arrs, stream=stream)
        mmref.compute_metrics(s, None, None)
        mmref.evaluate_moves(s, MASK_LCOM, MIN_IMPROVED, records=records)
        out = mmref.suggest_moves(s, TOPK, MASK_LCOM, MIN_IMPROVED, out=topk)
        if kern is not None:
            kern.append(s.last_eval_ms())
        s.free()
        return out

    s = mmref.load_system(c, *dev_arrs, stream=stream)
    mmref.compute_metrics(s, None, None)
    dig = torch.zeros(1, dtype=torch.int64, device=dev)
    mmref.evaluate_moves(s, MASK_LCOM, MIN_IMPROVED, digest=dig)
    top_g, nk_g, nm_g = mmref.suggest_moves(s, TOPK, MASK_LCOM, MIN_IMPROVED)
    s.free()
    check = (job, int(dig.cpu().numpy().view(np.uint64)[0]), nk_g, nm_g, [(int(x["m"]), int(x["d"])) for x in top_g])
    for _ in range(args.warmup):
        step()
    step_ms, kern = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        ev[0].record(stream)
        step(kern)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(ev[0].elapsed_time(ev[1]))
    peak, peak_kind = _peaks()
    alg = 16 * n_cand
    k = statistics.median(kern) / 1e3
    out = {"workload": workload, "criteria": {"metric_mask": MASK_LCOM, "min_improved": MIN_IMPROVED},
           "candidates_per_step": n_cand, "value": n_cand * args.steps / (sum(step_ms) / 1e3), "unit": UNIT,
           "ms_per_step": sum(step_ms) / args.steps,
           "roofline": {"bound": "hbm", "kernel": "eval_dense<records, kept>", "achieved": round(alg / k / 1e9, 1),
                        "peak": peak, "unit": "GB/s", "frac": round(alg / k / 1e9 / peak, 4),
                        "traffic": EVAL_DENSE_TRAFFIC, "algorithmic_bytes_per_launch": alg,
                        "kernel_ms": round(k * 1e3, 4), "peak_kind": peak_kind}}
    del records
    return out, check


# ---------------------------------------------------------------- nested: batched

BATCH_ROWS = 1000


def run_batched(args, local_rank, verifier):
    """256 independent systems: one persistent launch under a CUDA graph
    (metrics of every system + evaluation of every full cross product + kept
    moves + per-system sorts) against the same systems one after another."""
    import torch
    from paper_1308_4011_b300 import mmref, synth

    dev = torch.device("cuda", local_rank)
    n_sys = args.batch_systems
    params = [synth.batched_params(100 + i) for i in range(n_sys)]
    loaded, systems = [], []
    t0 = time.perf_counter()
    for p in params:
        s = synth.generate(**p)
        systems.append(s)
        loaded.append(mmref.load_synth(s, device=True))
    gen_s = time.perf_counter() - t0
    n_cand = sum(s.n_methods * (s.n_classes - 1) for s in systems)
    rng = np.random.default_rng(2024)
    sample_rows = [np.sort(rng.choice(s.n_methods, size=min(BATCH_ROWS, s.n_methods), replace=False))
                   for s in systems]
    jobs = [verifier.submit(job_oracle_batched, p, rows, MASK_LCOM, MIN_IMPROVED) if verifier else None
            for p, rows in zip(params, sample_rows)]
    mask, mi = MASK_LCOM, MIN_IMPROVED
    stream = torch.cuda.current_stream(dev)
    # kept-move capacity per system: the largest count of a first pass
    b0 = mmref.Batch(loaded, mask=mask, min_improved=mi, kept_cap=1, stream=stream)
    _, counts0 = b0.run(digest=False)
    b0.free()
    cap = int(max(int(counts0.max()), 1) * 1.1) + 64
    b = mmref.Batch(loaded, mask=mask, min_improved=mi, kept_cap=cap, stream=stream)
    tile = b.autotune()
    blocks = b.config()[1]
    dig, nk = b.run(digest=True)
    # what the batch graph computed, per system: metric arrays and a sample of full rows
    gpu_metrics, gpu_rows = [], []
    for g, s, rows in zip(loaded, systems, sample_rows):
        cm, mm_ = mmref.export_metrics(g)
        gpu_metrics.append(metrics_digest([cm[f] for f in ("n_methods", "n_attrs", "P", "Q", "S", "cbo")],
                                          [mm_[f] for f in ("fan_in", "fan_out", "own", "q")]))
        rp, dst = full_rows_lists(s, rows)
        d1 = np.zeros(1, dtype=np.uint64)
        mmref.evaluate_moves(g, mask, mi, rp, dst, digest=d1)
        gpu_rows.append(int(d1[0]))
    # the batch's full digests against single-system evaluations of the same systems
    d1 = torch.zeros(n_sys, dtype=torch.int64, device=dev)
    for i, g in enumerate(loaded):
        mmref.evaluate_moves(g, mask, mi, digest=d1[i:i + 1])
    torch.cuda.synchronize(dev)
    ok_single = bool(np.array_equal(d1.cpu().numpy().view(np.uint64), dig))
    k = TOPK

    def batched():
        _, counts = b.run(digest=False)
        return [b.suggestions(i, k)[0] for i in range(n_sys)], counts

    def sequential():
        out = []
        for g in loaded:
            mmref.compute_metrics(g, None, None)
            out.append(mmref.suggest_moves(g, k, mask, mi)[0])
        return out

    tops_b, counts = batched()
    tops_s = sequential()
    ok_top = all(np.array_equal(x, y) for x, y in zip(tops_b, tops_s))
    times_b, times_s = [], []
    reps = 3
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t = time.perf_counter(); sequential(); torch.cuda.synchronize(dev); times_s.append(time.perf_counter() - t)
    batched()
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t = time.perf_counter(); batched(); torch.cuda.synchronize(dev); times_b.append(time.perf_counter() - t)
    tb, ts = statistics.median(times_b), statistics.median(times_s)
    times_m = []  # the metric phase alone, one system after another
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for g in loaded:
            mmref.compute_metrics(g, None, None)
        torch.cuda.synchronize(dev)
        times_m.append(time.perf_counter() - t)
    b.free()
    for g in loaded:
        g.free()
    out = {"workload": f"{n_sys} systems, classes log-uniform 100..20,000, 12 methods and 6 attributes per class, "
                       f"seeds 100..{99 + n_sys}; full cross products (kept moves + top-100 of each)",
           "criteria": {"metric_mask": mask, "min_improved": mi}, "candidates": n_cand,
           "batched_s": tb, "sequential_s": ts, "speedup_vs_sequential": ts / tb,
           "value": n_cand / tb, "sequential_value": n_cand / ts, "unit": UNIT, "tile_methods": tile,
           "persistent_blocks": blocks, "sequential_metrics_only_s": statistics.median(times_m),
           "kept_cap_per_system": cap, "n_kept_total": int(counts.sum()),
           "batch_digests_equal_single_system": ok_single, "topk_equal_sequential": ok_top,
           "generate_and_load_s": round(gen_s, 2)}
    return out, (jobs, gpu_metrics, gpu_rows)


# ---------------------------------------------------------------- nested: serving

def run_serving(args, local_rank, verifier):
    """64 resident systems answering a Poisson stream of edit requests (each
    kind 1/5, seed 7): a saturating burst for capacity, then an open-loop run
    at half of it for latency with every 1,000th state kept for the oracle;
    a 2 GB budget run in which admission binds."""
    import torch
    from paper_1308_4011_b300 import mmref, synth

    torch.cuda.set_device(local_rank)
    n_req = args.requests
    systems = [synth.generate(**synth.batched_params(100 + i)) for i in range(64)]
    ms = [s.n_methods for s in systems]
    topk = 10

    def serve(budget, req, slots, snap=0):
        sv = mmref.Server(budget, n_slots=slots, topk=topk)
        for s in systems:
            sv.add_system(s)
        resp, top = sv.run(req, snap)
        return sv, resp, top

    warm = mmref.make_requests(ms, 64, rate_per_s=0.0, seed=99)
    warm["system"] = np.arange(64)
    warm["m"] = warm["m"] % np.asarray(ms)[warm["system"]]
    burst = mmref.make_requests(ms, n_req, rate_per_s=0.0, seed=7)
    sv, resp_b, _ = serve(100 << 30, np.concatenate([warm, burst]), args.slots)
    stats_b = sv.stats()
    sv.free()
    rb = resp_b[64:]
    cap_rps = n_req / (rb["done_s"].max() - rb["arrival_s"].min())
    rate = 0.5 * cap_rps
    req = mmref.make_requests(ms, n_req, rate_per_s=rate, seed=7)
    req["arrival_s"] += 2.0  # the warm-up admissions finish first
    sv, resp, top = serve(100 << 30, np.concatenate([warm, req]), args.slots, snap=1000)
    r = resp[64:]
    lat = (r["done_s"] - r["arrival_s"]) * 1e3
    stats = sv.stats()
    ok_req = bool((resp["status"] == 0).all())
    snaps = []
    for kk in range(stats["n_snapshots"]):
        i, si, c, arrs = sv.snapshot(kk)
        if i < 64:
            continue
        # the served answer, and the metric arrays of the same state computed afresh on the GPU
        g = mmref.load_system(c, *arrs)
        cm, mm_ = mmref.compute_metrics(g, "host", "host")
        g.free()
        gm = metrics_digest([cm[f] for f in ("n_methods", "n_attrs", "P", "Q", "S", "cbo")],
                            [mm_[f] for f in ("fan_in", "fan_out", "own", "q")])
        got = (int(resp["n_kept"][i]), int(resp["n_methods_with_kept"][i]),
               [(int(x["m"]), int(x["d"])) for x in top[i][: min(topk, int(resp["n_kept"][i]))]], gm)
        job = verifier.submit(job_oracle_snapshot, c, arrs, MASK_LCOM, MIN_IMPROVED, topk) if verifier else None
        snaps.append((i, si, got, job))
    sv.free()
    n_stress = min(n_req, args.stress_requests)
    req_s = mmref.make_requests(ms, n_stress, rate_per_s=0.0, seed=8)
    sv, resp_s, _ = serve(2 << 30, req_s, args.slots)
    stats_s = sv.stats()
    sv.free()
    rs = resp_s
    out = {"metric": "edit requests/s and latency (bit-exact vs oracle)", "unit": "requests/s",
           "workload": "64 resident systems (classes log-uniform 100..20,000, seeds 100..163), "
                       f"{n_req} Poisson edit requests (each kind 1/5, seed 7), 100 GB budget, "
                       f"{args.slots} worker slots, top-{topk} per request (LCOM_CK|LCOM_HS, 2 improved)",
           "capacity_requests_per_s": cap_rps, "offered_rate_per_s": rate,
           "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
           "latency_ms_mean": float(lat.mean()),
           "achieved_rps_open_loop": n_req / (r["done_s"].max() - r["arrival_s"].min()),
           "all_requests_ok": ok_req, "stats": stats, "burst_stats": stats_b,
           "stress_2GB": {"requests": n_stress, "ok": int((rs["status"] == 0).sum()),
                          "refused_budget": int((rs["status"] == 7).sum()), "evictions": stats_s["evictions"],
                          "loads": stats_s["loads"],
                          "requests_per_s": n_stress / (rs["done_s"].max() - rs["arrival_s"].min()),
                          "latency_ms_p50": float(np.percentile((rs["done_s"] - rs["arrival_s"]) * 1e3, 50)),
                          "latency_ms_p99": float(np.percentile((rs["done_s"] - rs["arrival_s"]) * 1e3, 99))}}
    return out, snaps


# ---------------------------------------------------------------- nested: similarity, rules R1 and R3, sequences

SIM_ROWS = 40
# the same eight per-class values, in the same order, as the oracle and the library name them
VARIANT_FIELDS_ORACLE = ("P_all", "Q_all", "ck_all", "pq", "pq_all", "cbo_out", "cbo_in", "cbo_bi")
VARIANT_FIELDS_GPU = ("P_all", "Q_all", "lcom_ck_all", "lcom_pq", "lcom_pq_all", "cbo_out", "cbo_in", "cbo_bi")


def job_oracle_similarity_rows(params, rows):
    """The oracle's similarity values of sampled methods (every partner)."""
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.generate(**params)
    o = oracle.Oracle(s)
    out = [tuple(a.tolist() for a in o.similarity_row(int(q))) for q in rows]
    o.close()
    return out


def job_oracle_r1(params, mask, mi, topk):
    import oracle
    from paper_1308_4011_b300 import synth
    s = synth.generate(**params)
    o = oracle.Oracle(s)
    res, avg, rp, dst, nv, nh = o.r1(mask=mask, min_improved=mi)
    o.close()
    return {"n_values": nv, "n_high": nh, "n_candidates": len(dst), "average": avg, "n_kept": res.n_kept,
            "top": [(int(k["m"]), int(k["d"])) for k in res.kept[:topk]]}


def job_oracle_r3(params):
    import oracle
    from paper_1308_4011_b300 import synth
    kept, rp, dst, nh = oracle.r3(synth.generate(**params))
    return {"n_kept": len(kept), "n_candidates": len(dst), "n_high": nh,
            "top": [tuple(int(v) for v in k) for k in kept[:TOPK]]}


def job_oracle_variants(params, topk):
    """The oracle's metric variants of every class, q_all of every method, and
    the first topk classes by unclamped LCOM over every accessed attribute
    and by coupling either way."""
    import oracle
    from paper_1308_4011_b300 import synth
    o = oracle.Oracle(synth.generate(**params))
    v, q_all = o.class_variants()
    o.close()
    cols = np.stack([v[f].astype(np.int64) for f in VARIANT_FIELDS_ORACLE], axis=1)
    return {"digest": hashlib.sha256(np.ascontiguousarray(cols).tobytes() + q_all.astype(np.int32).tobytes()).hexdigest(),
            "rank_pq_all": oracle.rank_classes(v["pq_all"], topk).tolist(),
            "rank_cbo_bi": oracle.rank_classes(v["cbo_bi"], topk).tolist()}


def job_oracle_sequence(params, mask, mi, rounds):
    import oracle
    from paper_1308_4011_b300 import synth
    seq, _ = oracle.sequence(synth.generate(**params), mask=mask, min_improved=mi, rounds=rounds)
    return seq


def run_rules(args, local_rank, verifier):
    """Similarity values of the large system (the term that dominates the
    paper's value count and its timed workload), rule R1 on the medium
    system, rule R3 on the large system, four rounds of non-conflicting moves
    on the medium system; each checked against the oracle."""
    import torch
    from paper_1308_4011_b300 import mmref, synth

    dev = torch.device("cuda", local_rank)
    out, jobs = {}, {}
    peak, _ = _peaks()
    large_p, medium_p = dict(synth.LARGE), dict(synth.MEDIUM)
    large, medium = synth.generate(**large_p), synth.generate(**medium_p)
    rows = np.random.default_rng(11).choice(large.n_methods, size=SIM_ROWS, replace=False)
    if verifier:
        jobs["sim"] = verifier.submit(job_oracle_similarity_rows, large_p, rows)
        jobs["r1"] = verifier.submit(job_oracle_r1, medium_p, MASK_LCOM, MIN_IMPROVED, TOPK)
        jobs["r3"] = verifier.submit(job_oracle_r3, large_p)
        jobs["seq"] = verifier.submit(job_oracle_sequence, medium_p, MASK_LCOM, MIN_IMPROVED, 4)
        jobs["var"] = verifier.submit(job_oracle_variants, large_p, TOPK)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize(dev)
            ts.append(time.perf_counter() - t)
        return statistics.median(ts), r

    g = mmref.load_synth(large, device=True)
    t, info = timed(lambda: mmref.similarity_info(g), 5)  # computed on the device, nothing read back
    (x, y, i, u), _ = mmref.similarity(g)
    M = large.n_methods
    n_co, n_val = info["n_cooccurrences"], info["n_values"]
    passes = (int(M * M - 1).bit_length() + 7) // 8
    alg = n_co * 8 * (2 + 2 * passes) + n_val * 16  # keys written, sorted (read + write per pass), read; values
    sim_rows = []
    for q in rows:
        sel = (x == q) | (y == q)
        partner = np.where(x[sel] == q, y[sel], x[sel])
        order = np.argsort(partner)
        sim_rows.append((partner[order].tolist(), i[sel][order].tolist(), u[sel][order].tolist()))
    out["similarity_large"] = {
        "workload": "large system: every method pair sharing a called method or an accessed attribute",
        "seconds": t, "n_values": n_val, "n_cooccurrences": n_co, "average": info["average"],
        "values_per_s": n_val / t, "pairs_assessed_per_s": M * (M - 1) / 2 / t,
        "roofline": {"bound": "hbm", "achieved": round(alg / t / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / t / 1e9 / peak, 4), "algorithmic_bytes": alg,
                     "note": "whole call (posting lists, keys, radix sort, runs, count read-backs) against the "
                             "bytes of its keys and values"}}
    mmref.compute_metrics(g, None, None)
    vd = torch.empty(56 * large.n_classes, dtype=torch.uint8, device=dev)
    qd = torch.empty(4 * large.n_methods, dtype=torch.uint8, device=dev)
    t, _ = timed(lambda: mmref.metric_variants(g, vd, qd), 5)  # device outputs: nothing read back
    v, q_all = mmref.metric_variants(g)
    n_acc = int(large.acc_rowptr[-1])
    out["variants_large"] = {"seconds": t, "classes_per_s": large.n_classes / t, "accesses_per_s": n_acc / t,
                             "note": "LCOM over every accessed attribute, unclamped LCOM, CBO in and either way"}
    cols = np.stack([v[f].astype(np.int64) for f in VARIANT_FIELDS_GPU], axis=1)
    var_got = {"digest": hashlib.sha256(np.ascontiguousarray(cols).tobytes() +
                                        q_all.astype(np.int32).tobytes()).hexdigest(),
               "rank_pq_all": mmref.rank_classes(g, mmref.RANK_LCOM_PQ_ALL, TOPK)[0].tolist(),
               "rank_cbo_bi": mmref.rank_classes(g, mmref.RANK_CBO_BI, TOPK)[0].tolist()}
    t, (top3, nk3, nc3, nh3) = timed(lambda: mmref.suggest_r3(g, TOPK), 5)
    out["r3_large"] = {"seconds": t, "n_candidates": nc3, "n_kept": nk3, "n_high_classes": nh3,
                       "candidates_per_s": nc3 / t}
    r3_got = {"n_kept": nk3, "n_candidates": nc3, "n_high": nh3, "top": [tuple(int(v) for v in k) for k in top3]}
    g.free()
    g = mmref.load_synth(medium, device=True)
    mmref.compute_metrics(g, None, None)
    t, (top1, nk1, nm1, info1) = timed(lambda: mmref.suggest_r1(g, TOPK, MASK_LCOM, MIN_IMPROVED), 5)
    out["r1_medium"] = {"seconds": t, "n_values": info1["n_values"], "n_high": info1["n_high"],
                        "n_candidates": info1["n_candidates"], "n_kept": nk1}
    r1_got = {"n_values": info1["n_values"], "n_high": info1["n_high"], "n_candidates": info1["n_candidates"],
              "average": info1["average"], "n_kept": nk1, "top": [(int(k["m"]), int(k["d"])) for k in top1]}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    seq = mmref.apply_sequence(g, 4, MASK_LCOM, MIN_IMPROVED)
    t = time.perf_counter() - t0
    out["sequence_medium"] = {"seconds": t, "rounds": 4, "moves_applied": len(seq),
                              "per_round": np.bincount(seq["round"], minlength=4).tolist() if len(seq) else []}
    seq_got = [tuple(int(v) for v in r) for r in seq]
    g.free()
    return out, (jobs, sim_rows, r1_got, r3_got, seq_got, var_got)


def collect_rules(check):
    jobs, sim_rows, r1_got, r3_got, seq_got, var_got = check
    if not jobs:
        return None
    ok_sim = jobs["sim"].get() == sim_rows
    ok_r1 = jobs["r1"].get() == r1_got
    ok_r3 = jobs["r3"].get() == r3_got
    ok_seq = jobs["seq"].get() == seq_got
    ok_var = jobs["var"].get() == var_got
    return {"ok": bool(ok_sim and ok_r1 and ok_r3 and ok_seq and ok_var), "similarity_sampled_rows": bool(ok_sim),
            "similarity_rows": SIM_ROWS, "r1": bool(ok_r1), "r3": bool(ok_r3), "sequence": bool(ok_seq),
            "variants": bool(ok_var)}


# ---------------------------------------------------------------- the reference arm

def run_reference(args, rank, world):
    """The CPU oracle timed as the reference arm on the host cores, on the bench
    line's workload and criteria (rank 0 only): each step builds the oracle
    (metrics of every class by definition) and evaluates a quarter of the
    methods' candidate lists."""
    if rank != 0:
        return None
    import oracle
    params, system, rp, dst = large_inputs(2)
    M = system.n_methods
    quarter = M // 4

    def one():
        t0 = time.perf_counter()
        o = oracle.Oracle(system)
        r = o.evaluate(mask=MASK_ALL, min_improved=MIN_IMPROVED, cand_rowptr=rp, cand_dst=dst, method=1,
                       rows=(0, quarter))
        dt = time.perf_counter() - t0
        o.close()
        return r.n_cand, dt

    for _ in range(args.warmup):
        one()
    cands, secs = 0, 0.0
    for _ in range(args.steps):
        n, dt = one()
        cands += n
        secs += dt
    value = cands / secs
    sample = f"per step: metrics of all classes + candidate rows 0..{quarter} of {M} ({cands // args.steps} candidates)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64",
            "data": "synthetic (seeded generator; no datasets)",
            "config": {"workload": WORKLOAD, "n_classes": system.n_classes, "n_methods": M,
                       "candidates_per_step": cands // args.steps,
                       "criteria": {"metric_mask": MASK_ALL, "min_improved": MIN_IMPROVED},
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- checks

def _check_result(kind, check):
    job, dig, nk, nm, top = check
    if job is None:
        return None
    ref = job.get()
    ok = dig == ref["digest"] and nk == ref["n_kept"] and nm == ref["n_mk"] and top == ref["top"][: len(top)]
    return {"ok": bool(ok), "n_kept": nk}


def collect_checks(large_checks, medium_check, batched_check, serving_snaps, rules_check=None):
    out = {"large": {}, "medium": None, "batched": None, "serving": None, "rules": None}
    if rules_check is not None:
        out["rules"] = collect_rules(rules_check)
    for mask, chk in large_checks.items():
        out["large"][f"mask{mask}"] = _check_result("large", chk)
    if medium_check is not None:
        out["medium"] = _check_result("medium", medium_check)
    if batched_check is not None:
        jobs, gpu_metrics, gpu_rows = batched_check
        if jobs and jobs[0] is not None:
            bad_m = bad_r = cands = 0
            for job, gm, gr in zip(jobs, gpu_metrics, gpu_rows):
                ref = job.get()
                bad_m += ref["metrics"] != gm
                bad_r += ref["rows_digest"] != gr
                cands += ref["n_cand"]
            out["batched"] = {"ok": bad_m == 0 and bad_r == 0, "systems": len(jobs), "metrics_mismatched": bad_m,
                              "sampled_rows_mismatched": bad_r, "sampled_candidates": cands,
                              "rows_per_system": BATCH_ROWS}
    if serving_snaps:
        bad = cands = n = 0
        for i, si, got, job in serving_snaps:
            if job is None:
                continue
            ref = job.get()
            n += 1
            cands += ref["n_cand"]
            exp = (ref["n_kept"], ref["n_mk"], ref["top"][: len(got[2])], ref["metrics"])
            bad += got != exp
        out["serving"] = {"ok": bad == 0, "snapshots_checked": n, "mismatched": bad,
                          "candidates_recomputed": cands,
                          "compared": "n_kept, methods with kept, top-10 of the served answer; metric arrays of "
                                      "the state (GPU recompute) -- each against O1 on the exported state"}
    return out


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-verify", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sections", default="medium,batched,serving,rules",
                    help="nested sections measured beside the bench line (comma list; '' for none)")
    ap.add_argument("--requests", type=int, default=100000)
    ap.add_argument("--stress-requests", type=int, default=5000)
    ap.add_argument("--slots", type=int, default=4,
                    help="serving worker slots (4 measured best: 1 slot 2,003, 2: 3,226, 3: 4,056, 4: 4,435, "
                         "5: 4,163, 6: 3,625, 8: 2,049 requests/s)")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--case", choices=["large", "medium", "dense-small"], default="large",
                    help="large: the bench line and its sections; medium / dense-small: only the dense step of "
                         "that system (profiling runs; the JSON line is that step's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    # the oracle's process starts before the first GPU call
    verifier = Verifier() if (rank == 0 and not args.no_verify) else None
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.case != "large":  # one dense step, for profiling
        params = None if args.case == "medium" else DENSE_SMALL
        label = MEDIUM_WORKLOAD if args.case == "medium" else (
            "dense profiling case: 2,000 classes, 24,000 methods, 12,000 attributes, seed 5; full cross product")
        out, check = run_medium(args, local_rank, verifier, params=params, workload=label)
        if verifier:
            out["verified_vs_oracle"] = _check_result("dense", check)
            verifier.close()
        out["case"] = args.case
        print(json.dumps(out), flush=True)
        return
    # the nested sections run on one GPU only (rank 0 of a single-rank job)
    sections = [x for x in args.sections.split(",") if x] if world == 1 else []
    t_start = time.perf_counter()
    nested, serving_snaps, batched_check, medium_check, rules_check = {}, None, None, None, None
    # the bench line first, while the oracle's process is idle
    line, large_checks, system = run_large(args, rank, world, local_rank, verifier, dist)
    if "serving" in sections:
        nested["serving"], serving_snaps = run_serving(args, local_rank, verifier)
    if verifier:
        # the host-driven sections (the bench line, serving) are done: the
        # oracle's jobs run from here on, beside the graph- and kernel-bound ones
        verifier.start()
    if "batched" in sections:
        nested["batched"], batched_check = run_batched(args, local_rank, verifier)
    if "medium" in sections:
        nested["medium"], medium_check = run_medium(args, local_rank, verifier)
    if "rules" in sections:
        nested["rules"], rules_check = run_rules(args, local_rank, verifier)
    if rank == 0:
        checks = collect_checks(large_checks, medium_check, batched_check, serving_snaps,
                                rules_check) if verifier else None
        if verifier:
            verifier.close()
        line["verified_vs_oracle"] = checks
        if not args.no_cpu_baseline:
            _, _, rp, dst = large_inputs(replica_seed(2, rank))
            line["cpu_baseline"] = cpu_baseline_large(system, rp, dst, MASK_ALL)
        line.update(nested)
        line["bench_wall_s"] = round(time.perf_counter() - t_start, 1)
        print(json.dumps(line), flush=True)
        results = []
        if checks is not None:
            results = [r for r in checks["large"].values()] + [checks[k] for k in ("medium", "batched", "serving",
                                                                                      "rules")]
        if any(r is not None and not r["ok"] for r in results):
            print(json.dumps({"error": "GPU results differ from the oracle", "checks": checks}), file=sys.stderr)
            sys.exit(3)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
