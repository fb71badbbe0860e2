"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (the CUDA library and its binding) never calls it and shares no code
with it; the two only share the seeded input generator.

What it computes (Napoli, Pappalardo, Tramontana, CISIS 2013):
  * fan-in / fan-out per method (Sec. II.A);
  * per class: LCOM as Chidamber-Kemerer pair counts (P = pairs sharing no
    owned attribute, Q = pairs sharing one, LCOM_CK = max(P - Q, 0)), LCOM as
    the Henderson-Sellers fraction 1 - S/(n a) kept as the exact pair
    (n a - S, n a), and CBO, the number of other classes used (Sec. II.B);
  * the effect of every candidate Move Method m -> D on the affected classes,
    the improved/worsened tallies and the kept flag (Sec. III.A rules), by
    two independent routes: O0 recomputes the affected classes from the
    definitions after changing cls(m) (the re-evaluation of Sec. IV.C), O1
    applies the incremental update formulas;
  * the sorted suggestion list (top-k) and an order-independent digest;
  * the LCOM and CBO variants of Sec. II.B (sharing over every accessed
    attribute, unclamped differences, coupling in both directions) and the
    ranking of classes by a metric.

``brute.py`` is a third, pure-Python route (whole-system recompute with
Python sets) for tiny systems; ``tables.py`` holds the paper's value-count
model (Sec. III.B) that Table I's ``#values`` column pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RECORD_DTYPE = np.dtype([("s", "<i4"), ("t", "<u2"), ("dcbo_src", "<i2"), ("dcbo_dst", "<i2"),
                         ("n_improved", "<u2"), ("n_worsened", "<u2"), ("flags", "<u2")])
KEPT_DTYPE = np.dtype([("m", "<i4"), ("d", "<i4"), ("n_improved", "<i4"), ("d_ck_sum", "<i4"),
                       ("d_cbo_sum", "<i4"), ("pad", "<i4")])
CLASS_FIELDS = ("n", "a", "P", "Q", "S", "ck", "hs_num", "hs_den", "cbo")
CLASS_DTYPE = np.dtype([(f, "<i8") for f in CLASS_FIELDS])

LCOM_CK, LCOM_HS, CBO = 1, 2, 4
VARIANT_FIELDS = ("P_all", "Q_all", "ck_all", "pq", "pq_all", "cbo_out", "cbo_in", "cbo_bi")
VARIANT_DTYPE = np.dtype([(f, "<i8") for f in VARIANT_FIELDS])


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` to ``liboracle.so`` (gcc -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-o", _LIB, _SRC])
    return _LIB


class _Input(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("n_methods", ctypes.c_int32),
                ("n_attrs", ctypes.c_int32), ("cbo_attrs", ctypes.c_int32),
                ("method_class", ctypes.c_void_p), ("attr_class", ctypes.c_void_p),
                ("acc_rowptr", ctypes.c_void_p), ("call_rowptr", ctypes.c_void_p),
                ("acc_idx", ctypes.c_void_p), ("call_idx", ctypes.c_void_p)]


class _Crit(ctypes.Structure):
    _fields_ = [("metric_mask", ctypes.c_uint32), ("min_improved", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("digest", ctypes.c_uint64), ("n_cand", ctypes.c_int64), ("n_kept", ctypes.c_int64),
                ("n_methods_with_kept", ctypes.c_int64), ("kept", ctypes.c_void_p),
                ("status", ctypes.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_build.argtypes = [ctypes.POINTER(_Input), ctypes.c_int]
        _lib.or_build.restype = ctypes.c_void_p
        _lib.or_free.argtypes = [ctypes.c_void_p]
        _lib.or_class_metrics.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_method_metrics.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4
        _lib.or_multigraph.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 3
        _lib.or_multigraph.restype = ctypes.c_int64
        _lib.or_evaluate.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Crit), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.POINTER(_Result)]
        _lib.or_evaluate.restype = ctypes.c_int
        _lib.or_evaluate_one.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Crit), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64)]
        _lib.or_evaluate_one.restype = ctypes.c_int
        _lib.or_free_kept.argtypes = [ctypes.c_void_p]
        _lib.or_record_hash.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        _lib.or_record_hash.restype = ctypes.c_uint64
        _lib.or_similarity.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4
        _lib.or_similarity.restype = ctypes.c_int64
        _lib.or_similarity_row.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 3
        _lib.or_similarity_row.restype = ctypes.c_int64
        _lib.or_r1_threshold.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_void_p]
        _lib.or_r1_threshold.restype = ctypes.c_double
        _lib.or_class_variants.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_class_variants.restype = ctypes.c_int
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class EvalResult:
    def __init__(self, digest, n_cand, kept, n_methods_with_kept, records=None):
        self.digest = digest
        self.n_cand = n_cand
        self.kept = kept                      # KEPT_DTYPE array, sorted by the suggestion key
        self.n_kept = len(kept)
        self.n_methods_with_kept = n_methods_with_kept
        self.records = records                # RECORD_DTYPE array or None


class Oracle:
    """The oracle's view of one system (metrics by definition at build time)."""

    def __init__(self, system, cbo_attrs: bool = True, threads: int | None = None):
        lib = _load()
        self.sys = system
        self.threads = threads or default_threads()
        self._keep = [np.ascontiguousarray(a) for a in (system.method_class, system.attr_class,
                                                       system.acc_rowptr, system.call_rowptr,
                                                       system.acc_idx, system.call_idx)]
        mc, ac, ar, cr, ai, ci = self._keep
        inp = _Input(system.n_classes, system.n_methods, system.n_attrs, int(bool(cbo_attrs)),
                     mc.ctypes.data, ac.ctypes.data, ar.ctypes.data, cr.ctypes.data,
                     ai.ctypes.data if ai.size else None, ci.ctypes.data if ci.size else None)
        self._inp = inp
        self._h = lib.or_build(ctypes.byref(inp), self.threads)
        if not self._h:
            raise ValueError("oracle: invalid system or out of memory")
        self.n_classes = system.n_classes
        self.n_methods = system.n_methods

    def close(self):
        if self._h:
            _load().or_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def class_metrics(self) -> np.ndarray:
        out = np.zeros(self.n_classes, dtype=CLASS_DTYPE)
        _load().or_class_metrics(self._h, out.ctypes.data)
        return out

    def method_metrics(self) -> dict:
        M = self.n_methods
        arrs = {k: np.zeros(M, dtype=np.int32) for k in ("fan_in", "fan_out", "own", "q")}
        _load().or_method_metrics(self._h, arrs["fan_in"].ctypes.data, arrs["fan_out"].ctypes.data,
                                  arrs["own"].ctypes.data, arrs["q"].ctypes.data)
        return arrs

    def multigraph(self):
        lib = _load()
        u = lib.or_multigraph(self._h, None, None, None)
        rowptr = np.zeros(self.n_classes + 1, dtype=np.int64)
        dst = np.zeros(max(u, 1), dtype=np.int32)
        cnt = np.zeros(max(u, 1), dtype=np.int32)
        lib.or_multigraph(self._h, rowptr.ctypes.data, dst.ctypes.data, cnt.ctypes.data)
        return rowptr, dst[:u], cnt[:u]

    def evaluate(self, mask: int = 7, min_improved: int = 2, cand_rowptr=None, cand_dst=None,
                 rows: tuple[int, int] | None = None, method: int = 1, records: bool = False,
                 threads: int | None = None) -> EvalResult:
        """Evaluate candidate rows (all D != cls(m) when cand_rowptr is None).
        method 0 = recompute (O0), 1 = incremental (O1)."""
        lib = _load()
        r0, r1 = rows if rows is not None else (0, self.n_methods)
        if cand_rowptr is not None:
            cand_rowptr = np.ascontiguousarray(cand_rowptr, dtype=np.int64)
            cand_dst = np.ascontiguousarray(cand_dst, dtype=np.int32)
            n = int(cand_rowptr[r1] - cand_rowptr[r0])
        else:
            n = (r1 - r0) * (self.n_classes - 1)
        rec = np.zeros(n, dtype=RECORD_DTYPE) if records else None
        res = _Result()
        crit = _Crit(mask, min_improved)
        st = lib.or_evaluate(self._h, ctypes.byref(crit),
                             cand_rowptr.ctypes.data if cand_rowptr is not None else None,
                             cand_dst.ctypes.data if cand_dst is not None and cand_dst.size else None,
                             r0, r1, method, threads or self.threads,
                             rec.ctypes.data if rec is not None and n else None, ctypes.byref(res))
        kept = np.zeros(res.n_kept, dtype=KEPT_DTYPE)
        if res.n_kept:
            ctypes.memmove(kept.ctypes.data, res.kept, res.n_kept * KEPT_DTYPE.itemsize)
        lib.or_free_kept(res.kept)
        if st != 0:
            raise ValueError("oracle: invalid candidate (out of range or equal to the source class)")
        return EvalResult(int(res.digest), int(res.n_cand), kept, int(res.n_methods_with_kept), rec)

    def class_variants(self, threads: int | None = None):
        """The LCOM and CBO variants of Sec. II.B for every class (VARIANT_DTYPE):
        LCOM_CK with sharing over every accessed attribute (P_all, Q_all, ck_all),
        the unclamped differences pq = P - Q and pq_all = P_all - Q_all, and
        CBO outgoing (cbo_out), incoming (cbo_in) and either way (cbo_bi).
        Also returns q_all per method (methods of its class sharing an accessed
        attribute with it)."""
        out = np.zeros(self.n_classes, dtype=VARIANT_DTYPE)
        q_all = np.zeros(max(self.n_methods, 1), dtype=np.int32)
        if _load().or_class_variants(self._h, threads or self.threads, out.ctypes.data, q_all.ctypes.data) != 0:
            raise MemoryError("oracle: out of memory")
        return out, q_all[: self.n_methods]

    def similarity(self, threads: int | None = None):
        """Jaccard similarity (Sec. II.A) of every method pair x < y sharing a
        property (called method or accessed attribute): arrays x, y, i =
        |P(x) & P(y)|, u = |P(x) | P(y)|, in (x, y) order."""
        lib = _load()
        n = lib.or_similarity(self._h, threads or self.threads, None, None, None, None)
        out = [np.zeros(max(n, 1), dtype=np.int32) for _ in range(4)]
        lib.or_similarity(self._h, threads or self.threads, *[a.ctypes.data for a in out])
        return tuple(a[:n] for a in out)

    def similarity_row(self, x: int):
        """Every y != x sharing a property with x: arrays y, i, u (ascending y)."""
        lib = _load()
        n = lib.or_similarity_row(self._h, int(x), None, None, None)
        out = [np.zeros(max(n, 1), dtype=np.int32) for _ in range(3)]
        lib.or_similarity_row(self._h, int(x), *[a.ctypes.data for a in out])
        return tuple(a[:n] for a in out)

    def r1(self, mask: int = 3, min_improved: int = 2):
        """Rule R1 (Sec. III.A): every pair of methods in different classes
        whose similarity exceeds the system average (footnote of Sec. III.A)
        proposes moving either method to the other's class or to another
        class holding a method it calls; the candidates
        are evaluated (O1) and the kept ones, with LCOM of both the origin and
        the destination improved under the default criteria, returned.
        Returns (EvalResult, average, candidate rowptr, candidate dst,
        number of similarity values, number of high pairs)."""
        x, y, i, u = self.similarity()
        umax = int(u.max()) if len(u) else 0
        avg, thr = r1_threshold(i, u, umax)
        rowptr, dst, n_high = r1_candidates(self.sys, x, y, i, u, thr)
        res = self.evaluate(mask=mask, min_improved=min_improved, cand_rowptr=rowptr, cand_dst=dst, method=1)
        return res, avg, rowptr, dst, len(x), n_high

    def evaluate_one(self, m: int, d: int, mask: int = 7, min_improved: int = 2, method: int = 1):
        rec = np.zeros(1, dtype=RECORD_DTYPE)
        a, b = ctypes.c_int64(), ctypes.c_int64()
        crit = _Crit(mask, min_improved)
        rc = _load().or_evaluate_one(self._h, ctypes.byref(crit), m, d, method, rec.ctypes.data,
                                     ctypes.byref(a), ctypes.byref(b))
        if rc:
            raise ValueError("oracle: invalid candidate")
        return rec[0], int(a.value), int(b.value)


def rank_classes(values, k: int):
    """Classes ordered by a per-class value, largest first, equal values by
    ascending class id (the order in which a rule takes the classes with the
    highest LCOM or CBO, Sec. III.A); the first k ids."""
    vals = [int(v) for v in values]
    order = sorted(range(len(vals)), key=lambda C: (-vals[C], C))
    return np.asarray(order[:k], dtype=np.int32)


def r1_threshold(i, u, umax: int):
    """The R1 threshold over the similarity values (i, u): their average in
    double precision (sum over u ascending of sum(i)/u, over the count) and,
    per u = 0..umax, the smallest i with i/u above it (u + 1 if none)."""
    i = np.ascontiguousarray(i, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.int32)
    thr = np.zeros(umax + 1, dtype=np.int32)
    avg = _load().or_r1_threshold(i.ctypes.data if len(i) else None, u.ctypes.data if len(u) else None, len(i),
                                  umax, thr.ctypes.data)
    return float(avg), thr


def r1_candidates(system, x, y, i, u, thr):
    """Moves proposed by the high pairs (i >= thr[u]) whose methods are in
    different classes (Sec. III.A, first rule): each method of such a pair to
    the class of the other method, or to another class holding a method it
    calls; each (method, class) once, as candidate lists (rows sorted by
    class).  Returns (rowptr, dst, number of high pairs)."""
    mc = system.method_class
    high = (i >= thr[u]) & (mc[x] != mc[y])
    m = [np.concatenate([x[high], y[high]]).astype(np.int64)]
    d = [np.concatenate([mc[y[high]], mc[x[high]]]).astype(np.int64)]
    for p in np.unique(np.concatenate([x[high], y[high]])):
        called = np.unique(mc[system.calls(int(p))]).astype(np.int64)
        called = called[called != mc[p]]
        m.append(np.full(len(called), int(p), dtype=np.int64))
        d.append(called)
    m, d = np.concatenate(m), np.concatenate(d)
    key = np.unique(m * system.n_classes + d)
    m, d = key // system.n_classes, (key % system.n_classes).astype(np.int32)
    rowptr = np.zeros(system.n_methods + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(m, minlength=system.n_methods))
    return rowptr, d, int(high.sum())


def record_hash(m: int, d: int, rec) -> int:
    arr = np.array([rec], dtype=RECORD_DTYPE) if not isinstance(rec, np.ndarray) else rec.reshape(1)
    return int(_load().or_record_hash(m, d, arr.ctypes.data))


# ---------------------------------------------------------------- move sequences

def affected_classes(system, m: int, d: int) -> set:
    """Classes whose metrics or adjacency a move of m to d can change: its
    class, d, the classes m uses (calls into or reads attributes of) and the
    classes of m's callers (Sec. III.A: the origin and destination classes,
    and through CBO the classes coupled to them)."""
    mc = system.method_class
    aff = {int(mc[m]), int(d)}
    aff |= {int(mc[t]) for t in system.calls(m)}
    aff |= {int(system.attr_class[a]) for a in system.acc(m)}
    rows = np.repeat(np.arange(system.n_methods), np.diff(system.call_rowptr))  # the caller of each call
    aff |= {int(mc[y]) for y in rows[system.call_idx == m]}
    return aff


def sequence(system, mask: int = 3, min_improved: int = 2, rounds: int = 4, per_round: int = 1 << 30,
             cbo_attrs: bool = True):
    """Several moves at once (abstract and Sec. I: several solutions): in each
    round the kept moves of the current state, in suggestion order, are taken
    greedily while their affected classes are disjoint from those of the moves
    already taken (so none changes another's evaluation) and no method moves
    twice; all of them are applied, and the next round starts from the new
    state.  Returns [(round, m, from class, to class), ...] and the final
    method_class array."""
    from paper_1308_4011_b300 import synth as _synth
    mc = system.method_class.copy()
    out = []
    for rnd in range(rounds):
        cur = _synth.System(system.n_classes, system.n_methods, system.n_attrs, mc.copy(), system.attr_class,
                            system.acc_rowptr, system.acc_idx, system.call_rowptr, system.call_idx)
        o = Oracle(cur, cbo_attrs=cbo_attrs)
        kept = o.evaluate(mask=mask, min_improved=min_improved, method=1).kept
        o.close()
        used, moved, taken = set(), set(), []
        for k in kept:
            if len(taken) >= per_round:
                break
            m, d = int(k["m"]), int(k["d"])
            if m in moved:
                continue
            aff = affected_classes(cur, m, d)
            if aff & used:
                continue
            used |= aff
            moved.add(m)
            taken.append((m, d))
        if not taken:
            break
        for m, d in taken:
            out.append((rnd, m, int(mc[m]), d))
            mc[m] = d
    return out, mc


# ---------------------------------------------------------------- rule R3

R3_DTYPE = np.dtype([("m", "<i4"), ("d", "<i4"), ("fan_in", "<i4"), ("fan_out", "<i4"), ("dcbo_src", "<i4"),
                     ("dcbo_dst", "<i4")])


def r3(system, cbo_attrs: bool = True, threads: int | None = None):
    """Rule R3 (Sec. III.A, third rule): for every class whose CBO is above the
    average CBO of all classes (exactly: CBO(C) * c > sum of CBO), relocate
    its methods to the classes each method uses (calls into, or reads
    attributes of when attribute uses count); a move is kept when CBO of the
    origin drops and CBO of the destination does not rise.  Kept moves in
    order of fan-in + fan-out (descending; the rule starts with the methods of
    highest fan-in and fan-out), then dCBO(origin) + dCBO(destination)
    (ascending), method, class.  Returns (kept R3_DTYPE array, candidate
    rowptr, candidate dst, number of high classes)."""
    o = Oracle(system, cbo_attrs=cbo_attrs, threads=threads)
    cm, mm_ = o.class_metrics(), o.method_metrics()
    cbo = cm["cbo"]
    c, M = system.n_classes, system.n_methods
    high = cbo * c > cbo.sum()
    mc = system.method_class
    rows = []
    for m in range(M):
        C = int(mc[m])
        if not high[C]:
            rows.append([])
            continue
        used = {int(mc[t]) for t in system.calls(m)}
        if cbo_attrs:
            used |= {int(system.attr_class[a]) for a in system.acc(m)}
        used.discard(C)
        rows.append(sorted(used))
    rowptr = np.zeros(M + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    dst = np.asarray([d for r in rows for d in r], dtype=np.int32)
    res = o.evaluate(mask=4, min_improved=1, cand_rowptr=rowptr, cand_dst=dst, method=1, records=True)
    o.close()
    mth = np.repeat(np.arange(M), np.diff(rowptr))
    keep = (res.records["dcbo_src"] < 0) & (res.records["dcbo_dst"] <= 0) if len(dst) else np.zeros(0, bool)
    out = np.zeros(int(keep.sum()), dtype=R3_DTYPE)
    out["m"] = mth[keep]
    out["d"] = dst[keep]
    out["fan_in"] = mm_["fan_in"][mth[keep]]
    out["fan_out"] = mm_["fan_out"][mth[keep]]
    out["dcbo_src"] = res.records["dcbo_src"][keep]
    out["dcbo_dst"] = res.records["dcbo_dst"][keep]
    order = np.lexsort((out["d"], out["m"], out["dcbo_src"] + out["dcbo_dst"], -(out["fan_in"] + out["fan_out"])))
    return out[order], rowptr, dst, int(high.sum())
