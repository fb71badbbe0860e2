"""Pure-Python brute force for tiny systems -- TEST INFRASTRUCTURE ONLY.

A third, independent route to every oracle output, used to pin the C oracle.
It recomputes the metrics of EVERY class of the whole system after each
candidate move (no locality assumption), with Python sets and exact
``fractions.Fraction`` arithmetic:

  * fan-in(m): methods calling m; fan-out(m): methods m calls (Sec. II.A);
  * CBO(C): other classes used by C through calls or (optionally) attribute
    accesses (Sec. II.B);
  * LCOM_CK(C) = max(#pairs sharing no owned attribute - #pairs sharing one, 0)
    and LCOM_HS(C) = 1 - mean over methods of |attrs of C used| / |attrs of C|,
    0 when C has no method or no attribute (Sec. II.B);
  * a candidate move m -> D is judged class by class: a class is worsened if
    a selected metric rises, improved if none rises and one drops; the move is
    kept when nothing is worsened and at least ``min_improved`` classes are
    improved (Sec. III.A: improve several components without hindering any).

Only for systems of a few dozen methods: cost is O(candidates * system^2).
"""
from __future__ import annotations

import struct
from fractions import Fraction
from itertools import combinations

MASK64 = (1 << 64) - 1


def _members(cls, n_classes):
    mem = [[] for _ in range(n_classes)]
    for x, c in enumerate(cls):
        mem[c].append(x)
    return mem


def class_metrics(sys, cls, cbo_attrs=True):
    """Per-class dict(n, a, P, Q, S, ck, hs (Fraction), hs_num, hs_den, cbo)."""
    mem = _members(cls, sys.n_classes)
    owned = [set() for _ in range(sys.n_classes)]
    for a, c in enumerate(sys.attr_class):
        owned[int(c)].add(a)
    acc = [set(int(v) for v in sys.acc(x)) for x in range(sys.n_methods)]
    calls = [set(int(v) for v in sys.calls(x)) for x in range(sys.n_methods)]
    out = []
    for Y in range(sys.n_classes):
        ms = mem[Y]
        n, a = len(ms), len(owned[Y])
        P = Q = 0
        for x, y in combinations(ms, 2):
            if acc[x] & acc[y] & owned[Y]:
                Q += 1
            else:
                P += 1
        S = sum(len(acc[x] & owned[Y]) for x in ms)
        used = set()
        for x in ms:
            used |= {cls[t] for t in calls[x]}
            if cbo_attrs:
                used |= {int(sys.attr_class[al]) for al in acc[x]}
        used.discard(Y)
        hs = Fraction(0) if n * a == 0 else 1 - Fraction(S, n * a)
        out.append(dict(n=n, a=a, P=P, Q=Q, S=S, ck=max(P - Q, 0), hs=hs,
                        hs_num=0 if n * a == 0 else n * a - S, hs_den=1 if n * a == 0 else n * a,
                        cbo=len(used)))
    return out


def method_metrics(sys):
    cls = [int(c) for c in sys.method_class]
    owned = [set() for _ in range(sys.n_classes)]
    for a, c in enumerate(sys.attr_class):
        owned[int(c)].add(a)
    acc = [set(int(v) for v in sys.acc(x)) for x in range(sys.n_methods)]
    calls = [set(int(v) for v in sys.calls(x)) for x in range(sys.n_methods)]
    mem = _members(cls, sys.n_classes)
    fan_in = [sum(1 for y in range(sys.n_methods) if x in calls[y]) for x in range(sys.n_methods)]
    fan_out = [len(calls[x]) for x in range(sys.n_methods)]
    own = [len(acc[x] & owned[cls[x]]) for x in range(sys.n_methods)]
    q = [sum(1 for y in mem[cls[x]] if y != x and acc[x] & acc[y] & owned[cls[x]])
         for x in range(sys.n_methods)]
    return dict(fan_in=fan_in, fan_out=fan_out, own=own, q=q)


def _sign(v):
    return (v > 0) - (v < 0)


def _enc(sg):
    return 1 if sg < 0 else (2 if sg > 0 else 0)


def _sat(v, lo, hi):
    return lo if v < lo else (hi if v > hi else v)


def evaluate(sys, mask=7, min_improved=2, cbo_attrs=True, candidates=None):
    """All candidates (m, D), D != cls(m) (or the given list).  Returns a dict
    (m, D) -> dict(record fields..., d_ck_sum, d_cbo_sum)."""
    cls = [int(c) for c in sys.method_class]
    base = class_metrics(sys, cls, cbo_attrs)
    owned = [set() for _ in range(sys.n_classes)]
    for a, c in enumerate(sys.attr_class):
        owned[int(c)].add(a)
    acc = [set(int(v) for v in sys.acc(x)) for x in range(sys.n_methods)]
    mem = _members(cls, sys.n_classes)
    if candidates is None:
        candidates = [(m, D) for m in range(sys.n_methods) for D in range(sys.n_classes) if D != cls[m]]
    out = {}
    for m, D in candidates:
        C = cls[m]
        cls2 = list(cls)
        cls2[m] = D
        after = class_metrics(sys, cls2, cbo_attrs)
        imp = wor = 0
        signs = {}
        for Y in range(sys.n_classes):
            b, a_ = base[Y], after[Y]
            s_ck, s_hs, s_cbo = _sign(a_["ck"] - b["ck"]), _sign(a_["hs"] - b["hs"]), _sign(a_["cbo"] - b["cbo"])
            signs[Y] = (s_ck, s_hs, s_cbo)
            sel = [s for bit, s in ((1, s_ck), (2, s_hs), (4, s_cbo)) if mask & bit]
            if any(s > 0 for s in sel):
                wor += 1
            elif any(s < 0 for s in sel):
                imp += 1
        t = len(acc[m] & owned[D])
        s_ = sum(1 for y in mem[D] if acc[m] & acc[y] & owned[D])
        flags = (_enc(signs[C][0]) | _enc(signs[C][1]) << 2 | _enc(signs[C][2]) << 4 |
                 _enc(signs[D][0]) << 6 | _enc(signs[D][1]) << 8 | _enc(signs[D][2]) << 10)
        if wor == 0 and imp >= min_improved:
            flags |= 1 << 15
        dcs = after[C]["cbo"] - base[C]["cbo"]
        dcd = after[D]["cbo"] - base[D]["cbo"]
        out[(m, D)] = dict(s=s_, t=_sat(t, 0, 65535), dcbo_src=_sat(dcs, -32768, 32767),
                           dcbo_dst=_sat(dcd, -32768, 32767), n_improved=_sat(imp, 0, 65535),
                           n_worsened=_sat(wor, 0, 65535), flags=flags,
                           d_ck_sum=(after[C]["ck"] - base[C]["ck"]) + (after[D]["ck"] - base[D]["ck"]),
                           d_cbo_sum=dcs + dcd,
                           changed=[Y for Y in range(sys.n_classes) if after[Y] != base[Y]])
    return out


def suggestions(evals):
    """Kept moves in suggestion order: more improved classes first, then the
    lower LCOM_CK change sum, lower CBO change sum, method id, class id."""
    kept = [(m, D, r) for (m, D), r in evals.items() if r["flags"] & 0x8000]
    kept.sort(key=lambda k: (-k[2]["n_improved"], k[2]["d_ck_sum"], k[2]["d_cbo_sum"], k[0], k[1]))
    return [(m, D, r["n_improved"], r["d_ck_sum"], r["d_cbo_sum"]) for m, D, r in kept]


def _splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def record_bytes(r):
    return struct.pack("<iHhhHHH", r["s"], r["t"], r["dcbo_src"], r["dcbo_dst"],
                       r["n_improved"], r["n_worsened"], r["flags"])


def record_hash(m, D, r):
    b = record_bytes(r)
    lo, hi = struct.unpack("<QQ", b)
    key = ((m & 0xFFFFFFFF) << 32) | (D & 0xFFFFFFFF)
    return _splitmix64(key ^ _splitmix64(lo ^ _splitmix64(hi)))


def digest(evals):
    return sum(record_hash(m, D, r) for (m, D), r in evals.items()) & MASK64


def variants(sys, cbo_attrs=True):
    """The LCOM and CBO variants of Sec. II.B per class, with Python sets:
    sharing over every accessed attribute (P_all, Q_all, ck_all), the
    unclamped differences pq and pq_all, and coupling outgoing, incoming and
    either way (cbo_out, cbo_in, cbo_bi); and q_all per method."""
    cls = [int(c) for c in sys.method_class]
    mem = _members(cls, sys.n_classes)
    base = class_metrics(sys, cls, cbo_attrs)
    acc = [set(int(v) for v in sys.acc(x)) for x in range(sys.n_methods)]
    calls = [set(int(v) for v in sys.calls(x)) for x in range(sys.n_methods)]
    uses = [set() for _ in range(sys.n_classes)]      # classes each class uses
    for x in range(sys.n_methods):
        uses[cls[x]] |= {cls[t] for t in calls[x]}
        if cbo_attrs:
            uses[cls[x]] |= {int(sys.attr_class[a]) for a in acc[x]}
    for Y in range(sys.n_classes):
        uses[Y].discard(Y)
    used_by = [{Y for Y in range(sys.n_classes) if E in uses[Y]} for E in range(sys.n_classes)]
    q_all = [sum(1 for y in mem[cls[x]] if y != x and acc[x] & acc[y]) for x in range(sys.n_methods)]
    out = []
    for Y in range(sys.n_classes):
        pairs = list(combinations(mem[Y], 2))
        Q_all = sum(1 for x, y in pairs if acc[x] & acc[y])
        P_all = len(pairs) - Q_all
        out.append(dict(P_all=P_all, Q_all=Q_all, ck_all=max(P_all - Q_all, 0),
                        pq=base[Y]["P"] - base[Y]["Q"], pq_all=P_all - Q_all,
                        cbo_out=len(uses[Y]), cbo_in=len(used_by[Y]), cbo_bi=len(uses[Y] | used_by[Y])))
    return out, q_all
