"""Pins of the CPU oracle against things other than itself: the paper's printed
numbers (Table I), hand-worked values, closed forms of the Sec. II definitions,
a pure-Python whole-system brute force, and invariants of the move semantics."""
from __future__ import annotations

import csv
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.tables import count_values, lcom_values
from paper_1308_4011_b300 import synth

from sysutil import GOLDEN, hand_example, make_system, moved, permute, tiny_random

REC_FIELDS = ("s", "t", "dcbo_src", "dcbo_dst", "n_improved", "n_worsened", "flags")


# ---------------------------------------------------------------- Table I

def test_table1_value_counts():
    """#values = 2m + m(m-1)/2 + 2c(m+1) (Sec. III.B) reproduces Table I's
    printed column to its 0.1M precision: rounded for 12 rows, truncated for
    JUnit (1.277M printed as 1.2M)."""
    rows = [r for r in csv.DictReader(l for l in open(os.path.join(GOLDEN, "table1_values.csv"))
                                      if not l.startswith("#"))]
    assert len(rows) == 13
    rounded = 0
    for r in rows:
        v = count_values(int(r["classes"]), int(r["methods"])) / 1e6
        printed = float(r["values_millions"])
        ok_round = abs(round(v, 1) - printed) < 1e-9
        ok_trunc = abs(int(v * 10) / 10 - printed) < 1e-9
        assert ok_round or ok_trunc, (r["system"], v, printed)
        rounded += ok_round
    assert rounded == 12
    # the paper's worked example: JUnit, 1,200 methods and 231 classes -> "1.2 millions"
    assert 1.2e6 <= count_values(231, 1200) < 1.3e6


def test_lcom_values_counts_the_assessed_classes():
    """#LCOM values (Sec. III.B) counted from what the oracle assesses: one LCOM
    per class as it is, plus one per (class, method) pair -- the oracle's own
    candidate count (every method to every other class, m(c-1)) and, for each
    method, its own class after it is moved out (m).  The count is taken from
    the oracle's evaluation, not from the formula."""
    s = tiny_random(3)
    o = oracle.Oracle(s, threads=1)
    n_cand = o.evaluate(mask=3, min_improved=2).n_cand
    c, m = s.n_classes, s.n_methods
    assert n_cand == m * (c - 1)
    assert lcom_values(c, m) == c + n_cand + m
    # and its share of Table I's total: removing it (or the CBO term) breaks the JUnit row
    assert count_values(231, 1200) - lcom_values(231, 1200) < 1.2e6


# ---------------------------------------------------------------- hand-worked

def _rec_tuple(r):
    return tuple(int(r[f]) for f in REC_FIELDS)


def test_hand_example_metrics():
    s, g = hand_example()
    o = oracle.Oracle(s, cbo_attrs=True, threads=1)
    cm = o.class_metrics()
    for f, vals in g["class_metrics_cbo_attrs"].items():
        assert list(cm[f]) == vals, f
    mm = o.method_metrics()
    for f, vals in g["method_metrics"].items():
        assert list(mm[f]) == vals, f
    o2 = oracle.Oracle(s, cbo_attrs=False, threads=1)
    assert list(o2.class_metrics()["cbo"]) == g["cbo_calls_only"]


@pytest.mark.parametrize("method", [0, 1])
def test_hand_example_moves(method):
    s, g = hand_example()
    for mv in g["moves"]:
        o = oracle.Oracle(s, cbo_attrs=bool(mv["cbo_attrs"]), threads=1)
        rec, dck, dcb = o.evaluate_one(mv["m"], mv["d"], mask=mv["mask"], min_improved=mv["min_improved"],
                                       method=method)
        exp = mv["record"]
        assert _rec_tuple(rec) == tuple(exp[f] for f in REC_FIELDS), mv
        assert (dck, dcb) == (mv["d_ck_sum"], mv["d_cbo_sum"]), mv


def test_hand_example_brute():
    s, g = hand_example()
    for mv in g["moves"]:
        ev = brute.evaluate(s, mask=mv["mask"], min_improved=mv["min_improved"],
                            cbo_attrs=bool(mv["cbo_attrs"]), candidates=[(mv["m"], mv["d"])])
        r = ev[(mv["m"], mv["d"])]
        assert tuple(r[f] for f in REC_FIELDS) == tuple(mv["record"][f] for f in REC_FIELDS)


# ---------------------------------------------------------------- closed forms

def _one_class(acc_rows, n_attrs, extra_classes=0):
    n = len(acc_rows)
    return make_system([0] * n, [0] * n_attrs, acc_rows, [[] for _ in range(n)], 1 + extra_classes)


@pytest.mark.parametrize("n", [2, 3, 7, 33, 70])
def test_lcom_all_share_one_attribute(n):
    """Every method uses one common attribute: Q = n(n-1)/2, P = 0, LCOM = 0."""
    rng = np.random.default_rng(n)
    rows = [[0] + [int(v) for v in rng.choice(np.arange(1, 9), size=rng.integers(0, 3), replace=False)]
            for _ in range(n)]
    cm = oracle.Oracle(_one_class(rows, 9), threads=1).class_metrics()
    assert (cm["P"][0], cm["Q"][0], cm["ck"][0]) == (0, n * (n - 1) // 2, 0)


@pytest.mark.parametrize("n", [2, 5, 40])
def test_lcom_disjoint_attributes(n):
    """n methods on disjoint single attributes: P = n(n-1)/2, Q = 0."""
    cm = oracle.Oracle(_one_class([[i] for i in range(n)], n), threads=1).class_metrics()
    assert (cm["P"][0], cm["Q"][0], cm["ck"][0]) == (n * (n - 1) // 2, 0, n * (n - 1) // 2)


def test_lcom_single_and_empty_class():
    s = make_system([0], [0, 1], [[0, 1]], [[]], n_classes=2)
    cm = oracle.Oracle(s, threads=1).class_metrics()
    assert (cm["P"][0], cm["Q"][0], cm["ck"][0]) == (0, 0, 0)
    # class 1 has no method and no attribute
    assert (cm["n"][1], cm["ck"][1], cm["hs_num"][1], cm["hs_den"][1], cm["cbo"][1]) == (0, 0, 0, 1, 0)


@pytest.mark.parametrize("n,a", [(1, 1), (3, 4), (10, 2)])
def test_lcom_hs_closed_forms(n, a):
    """All methods use all a attributes: LCOM_HS = 0/(n a); each uses exactly
    one: (n a - n)/(n a)."""
    cm = oracle.Oracle(_one_class([list(range(a)) for _ in range(n)], a), threads=1).class_metrics()
    assert (cm["hs_num"][0], cm["hs_den"][0]) == (0, n * a)
    cm = oracle.Oracle(_one_class([[i % a] for i in range(n)], a), threads=1).class_metrics()
    assert (cm["hs_num"][0], cm["hs_den"][0]) == (n * a - n, n * a)


def test_lcom_ignores_foreign_attributes():
    """Sharing counts only attributes owned by the class."""
    s = make_system([0, 0, 1], [0, 1, 1], [[1], [1], [2]], [[], [], []], n_classes=2)
    cm = oracle.Oracle(s, threads=1).class_metrics()
    assert (cm["P"][0], cm["Q"][0], cm["S"][0]) == (1, 0, 0)


@pytest.mark.parametrize("k", [0, 1, 5, 12])
def test_cbo_star(k):
    """Class 0 calls one method in each of k other classes: CBO = k; the
    called classes use nothing: CBO = 0."""
    mc = [0] + list(range(1, k + 1))
    s = make_system(mc, [], [[] for _ in mc], [list(range(1, k + 1))] + [[] for _ in range(k)], n_classes=k + 1)
    cm = oracle.Oracle(s, threads=1).class_metrics()
    assert cm["cbo"][0] == k
    assert all(cm["cbo"][1:] == 0)


def test_cbo_attribute_uses():
    """Accessing another class's attribute couples only when attribute uses count."""
    s = make_system([0, 1], [1], [[0], []], [[], []], n_classes=2)
    assert oracle.Oracle(s, cbo_attrs=True, threads=1).class_metrics()["cbo"][0] == 1
    assert oracle.Oracle(s, cbo_attrs=False, threads=1).class_metrics()["cbo"][0] == 0


def test_cbo_equals_distinct_target_classes_on_tiny():
    """CBO(C) = |{cls(t)} U {own(a)}| - own class, computed with numpy sets."""
    s = synth.named("tiny")
    cm = oracle.Oracle(s).class_metrics()
    for Y in range(0, s.n_classes, 7):
        members = np.nonzero(s.method_class == Y)[0]
        used = set()
        for x in members:
            used |= set(s.method_class[s.calls(x)].tolist()) | set(s.attr_class[s.acc(x)].tolist())
        used.discard(Y)
        assert cm["cbo"][Y] == len(used)


def test_fan_sums_and_pair_identity():
    s = synth.named("tiny")
    o = oracle.Oracle(s)
    mm, cm = o.method_metrics(), o.class_metrics()
    assert mm["fan_in"].sum() == mm["fan_out"].sum() == s.n_call
    assert np.array_equal(mm["fan_in"], np.bincount(s.call_idx, minlength=s.n_methods))
    assert np.all(cm["P"] + cm["Q"] == cm["n"] * (cm["n"] - 1) // 2)
    # q_x sums to twice the sharing pairs, own_x sums to S
    q_by_class = np.bincount(s.method_class, weights=mm["q"], minlength=s.n_classes)
    assert np.array_equal(q_by_class.astype(np.int64), 2 * cm["Q"])
    own_by_class = np.bincount(s.method_class, weights=mm["own"], minlength=s.n_classes)
    assert np.array_equal(own_by_class.astype(np.int64), cm["S"])


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(12))
def test_oracle_matches_brute_force(seed):
    """O0 and O1 equal the pure-Python whole-system recompute on every
    candidate of random tiny systems, for several criteria."""
    s = tiny_random(seed)
    for cbo_attrs in (True, False):
        base = brute.class_metrics(s, [int(v) for v in s.method_class], cbo_attrs)
        o = oracle.Oracle(s, cbo_attrs=cbo_attrs, threads=2)
        cm = o.class_metrics()
        for f in oracle.CLASS_FIELDS:
            assert [int(v) for v in cm[f]] == [b[f] for b in base], f
        for mask, mi in ((7, 2), (1, 1), (3, 2), (4, 1), (6, 1)):
            ev = brute.evaluate(s, mask=mask, min_improved=mi, cbo_attrs=cbo_attrs)
            exp = [tuple(ev[(m, D)][f] for f in REC_FIELDS)
                   for m in range(s.n_methods) for D in range(s.n_classes) if D != s.method_class[m]]
            for method in (0, 1):
                r = o.evaluate(mask=mask, min_improved=mi, method=method, records=True)
                got = [tuple(int(x) for x in rec) for rec in r.records]
                assert got == exp, (seed, cbo_attrs, mask, mi, method)
                assert r.digest == brute.digest(ev)
                sug = [tuple(int(k[f]) for f in ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")) for k in r.kept]
                assert sug == brute.suggestions(ev)


def test_brute_force_exercises_kept_moves():
    """The random tiny systems above do produce kept moves (the filter is not vacuous)."""
    kept = 0
    for seed in range(12):
        ev = brute.evaluate(tiny_random(seed), mask=3, min_improved=2)
        kept += sum(1 for r in ev.values() if r["flags"] & 0x8000)
    assert kept > 10


@pytest.mark.parametrize("seed", range(6))
def test_only_source_target_and_caller_classes_change(seed):
    """Whole-system recompute: a move changes only the source, the target and
    the classes of the moved method's callers."""
    s = tiny_random(seed)
    ev = brute.evaluate(s)
    for (m, D), r in ev.items():
        callers = {int(s.method_class[y]) for y in range(s.n_methods) if m in s.calls(y)}
        assert set(r["changed"]) <= {int(s.method_class[m]), D} | callers


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(5))
def test_incremental_delta_equals_recompute_after_move(seed):
    """Metrics of the moved system, computed from scratch, equal the base
    metrics updated by the record (t, s, dCBO) of that move."""
    s = synth.named("tiny") if seed == 0 else tiny_random(seed + 20)
    o = oracle.Oracle(s, threads=2)
    cm = o.class_metrics()
    mm = o.method_metrics()
    rng = np.random.default_rng(seed)
    for _ in range(25 if seed == 0 else 10):
        m = int(rng.integers(s.n_methods))
        C = int(s.method_class[m])
        D = int(rng.integers(s.n_classes - 1))
        D += D >= C
        rec, dck, dcb = o.evaluate_one(m, D, method=0)
        cm2 = oracle.Oracle(moved(s, m, D), threads=2).class_metrics()
        nC, nD = cm["n"][C], cm["n"][D]
        assert cm2["n"][C] == nC - 1 and cm2["n"][D] == nD + 1
        assert cm2["S"][C] == cm["S"][C] - mm["own"][m]
        assert cm2["Q"][C] == cm["Q"][C] - mm["q"][m]
        assert cm2["P"][C] == cm["P"][C] - (nC - 1 - mm["q"][m])
        assert cm2["S"][D] == cm["S"][D] + rec["t"]
        assert cm2["Q"][D] == cm["Q"][D] + rec["s"]
        assert cm2["P"][D] == cm["P"][D] + (nD - rec["s"])
        assert cm2["cbo"][C] == cm["cbo"][C] + rec["dcbo_src"]
        assert cm2["cbo"][D] == cm["cbo"][D] + rec["dcbo_dst"]
        assert dck == (cm2["ck"][C] - cm["ck"][C]) + (cm2["ck"][D] - cm["ck"][D])


@pytest.mark.parametrize("seed", range(4))
def test_move_then_move_back_mirrors(seed):
    """Moving m back from D to C undoes every change: the back move's deltas
    are the forward move's, negated and with source/target swapped."""
    s = tiny_random(seed + 40)
    o = oracle.Oracle(s, threads=1)
    rng = np.random.default_rng(seed)
    for _ in range(10):
        m = int(rng.integers(s.n_methods))
        C = int(s.method_class[m])
        D = int(rng.integers(s.n_classes - 1))
        D += D >= C
        fwd, dck, dcb = o.evaluate_one(m, D, mask=7, min_improved=1, method=1)
        o2 = oracle.Oracle(moved(s, m, D), threads=1)
        back, dck2, dcb2 = o2.evaluate_one(m, C, mask=7, min_improved=1, method=1)
        assert back["dcbo_src"] == -fwd["dcbo_dst"] and back["dcbo_dst"] == -fwd["dcbo_src"]
        assert (dck2, dcb2) == (-dck, -dcb)
        flip = {0: 0, 1: 2, 2: 1}
        for k in range(3):  # sign fields: source of the back move = target of the forward move
            f_src = (int(fwd["flags"]) >> (2 * k)) & 3
            f_dst = (int(fwd["flags"]) >> (6 + 2 * k)) & 3
            b_src = (int(back["flags"]) >> (2 * k)) & 3
            b_dst = (int(back["flags"]) >> (6 + 2 * k)) & 3
            assert b_src == flip[f_dst] and b_dst == flip[f_src]
        assert np.array_equal(oracle.Oracle(moved(moved(s, m, D), m, C), threads=1).class_metrics(),
                              o.class_metrics())


@pytest.mark.parametrize("seed", range(3))
def test_relabelling_invariance(seed):
    s = tiny_random(seed + 60) if seed else synth.named("tiny")
    p, pc, pm, pa = permute(s, seed)
    o, op = oracle.Oracle(s), oracle.Oracle(p)
    cm, cmp_ = o.class_metrics(), op.class_metrics()
    assert np.array_equal(cmp_[pc], cm)
    mm, mmp = o.method_metrics(), op.method_metrics()
    for f in mm:
        assert np.array_equal(mmp[f][pm], mm[f])
    k = o.evaluate(mask=3, min_improved=2).kept
    kp = op.evaluate(mask=3, min_improved=2).kept
    a = sorted((int(pm[r["m"]]), int(pc[r["d"]]), int(r["n_improved"]), int(r["d_ck_sum"]), int(r["d_cbo_sum"]))
               for r in k)
    b = sorted((int(r["m"]), int(r["d"]), int(r["n_improved"]), int(r["d_ck_sum"]), int(r["d_cbo_sum"])) for r in kp)
    assert a == b


@pytest.mark.slow
def test_o0_equals_o1_on_tiny_workload():
    """Recompute (O0) and incremental (O1) agree on all 398,000 candidates of
    the tiny workload (200 classes, 2,000 methods), in two criteria."""
    s = synth.named("tiny")
    o = oracle.Oracle(s)
    for mask, mi in ((7, 2), (3, 2)):
        r0 = o.evaluate(mask=mask, min_improved=mi, method=0)
        r1 = o.evaluate(mask=mask, min_improved=mi, method=1)
        assert r0.n_cand == r1.n_cand == 2000 * 199
        assert r0.digest == r1.digest
        assert np.array_equal(r0.kept, r1.kept)


def test_o0_equals_o1_sampled_medium_restricted():
    """O0 and O1 agree on sampled restricted candidates of a mid-size system."""
    s = synth.generate(1500, 15000, 7500, max_class=400, seed=5, lambda_acc=4, lambda_call=6, p_loc=0.75)
    rowptr, dst = synth.candidates(s, 8, seed=5)
    o = oracle.Oracle(s)
    rng = np.random.default_rng(1)
    rows = rng.choice(s.n_methods, size=12, replace=False)
    for m in rows:
        for D in dst[rowptr[m]:rowptr[m + 1]]:
            a = o.evaluate_one(int(m), int(D), method=0, mask=7, min_improved=1)
            b = o.evaluate_one(int(m), int(D), method=1, mask=7, min_improved=1)
            assert _rec_tuple(a[0]) == _rec_tuple(b[0]) and a[1:] == b[1:]


# ---------------------------------------------------------------- similarity and rule R1 (Sec. II.A, III.A)

def _py_props(s, x):
    return {("m", int(t)) for t in s.calls(x)} | {("a", int(a)) for a in s.acc(x)}


def _py_similarity(s):
    """Jaccard similarity of every pair by Python sets (Sec. II.A)."""
    P = [_py_props(s, x) for x in range(s.n_methods)]
    out = {}
    for x in range(s.n_methods):
        for y in range(x + 1, s.n_methods):
            i = len(P[x] & P[y])
            if i:
                out[(x, y)] = (i, len(P[x] | P[y]))
    return out


def test_similarity_closed_forms():
    """Identical property sets give i = u = |P|; a subset gives i = |small|,
    u = |big|; disjoint sets are no value; a method with no properties shares
    nothing; method 1 (a callee) and attribute 1 are different properties."""
    # P0 = P1 = {a0, a1, m2}, P2 = {a0, m3}, P3 = {a2, m1}, P4 = {}, P5 = {a1, m2}
    s = make_system([0, 0, 1, 1, 2, 2], [0, 1, 2],
                    [[0, 1], [0, 1], [0], [2], [], [1]],
                    [[2], [2], [3], [1], [], [2]], n_classes=3)
    o = oracle.Oracle(s, threads=1)
    x, y, i, u = o.similarity()
    got = {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in zip(x, y, i, u)}
    assert got == {(0, 1): (3, 3), (0, 2): (1, 4), (0, 5): (2, 3), (1, 2): (1, 4), (1, 5): (2, 3)}


@pytest.mark.parametrize("seed", range(8))
def test_similarity_brute_force(seed):
    s = tiny_random(seed)
    o = oracle.Oracle(s, threads=2)
    x, y, i, u = o.similarity()
    got = {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in zip(x, y, i, u)}
    assert got == _py_similarity(s)
    # rows: every partner of x, both sides of the pair
    for q in range(0, s.n_methods, 3):
        ry, ri, ru = o.similarity_row(q)
        exp = sorted((b if a == q else a, v) for (a, b), v in got.items() if q in (a, b))
        assert [(int(a), (int(c), int(d))) for a, c, d in zip(ry, ri, ru)] == exp


def test_r1_threshold_and_candidates_by_hand():
    """The average of three values 1/2, 1/3, 2/3 is 1/2: only 2/3 is above it.
    Pairs in the same class propose nothing; a high pair across classes
    proposes both moves to the partner's class and each method's move to the
    classes of the methods it calls."""
    i = np.array([1, 1, 2], dtype=np.int32)
    u = np.array([2, 3, 3], dtype=np.int32)
    avg, thr = oracle.r1_threshold(i, u, 3)
    assert avg == pytest.approx(0.5)
    assert list(thr) == [1, 1, 2, 2]  # u = 1: 1/1 > 1/2; u = 2: 2/2 (1/2 is not above); u = 3: 2/3
    s = make_system([0, 0, 1, 2], [], [[], [], [], []], [[1], [0], [0], [0]], n_classes=3)
    x = np.array([0, 1, 2], dtype=np.int32)
    y = np.array([1, 2, 3], dtype=np.int32)
    rowptr, dst, nh = oracle.r1_candidates(s, x, y, np.array([1, 1, 2], np.int32), np.array([1, 3, 3], np.int32),
                                           np.array([1, 1, 2, 2], np.int32))
    # (0,1): same class; (1,2): 1/3 below; (2,3): 2/3 above, classes 1 and 2 -> 2 -> class 2, 3 -> class 1;
    # both call method 0 (class 0) -> 2 -> class 0, 3 -> class 0; methods 0, 1 propose nothing
    assert nh == 1 and list(rowptr) == [0, 0, 0, 2, 4] and list(dst) == [0, 2, 0, 1]


@pytest.mark.parametrize("seed", range(6))
def test_r1_suggestions_brute_force(seed):
    """R1 end to end against Python: similarity by sets, the average in the
    same fixed order, the proposed moves, each evaluated by recomputing the
    whole system (brute force), kept when LCOM of origin and destination
    both improve and no LCOM value worsens."""
    s = tiny_random(seed + 20)
    o = oracle.Oracle(s, threads=1)
    res, avg, rowptr, dst, nvals, nhigh = o.r1(mask=3, min_improved=2)
    sims = _py_similarity(s)
    by_u = {}
    for (i, u) in sims.values():
        by_u[u] = by_u.get(u, 0) + i
    tot = 0.0
    for uu in sorted(by_u):
        tot += by_u[uu] / uu
    py_avg = tot / len(sims) if sims else 0.0
    assert avg == py_avg and nvals == len(sims)
    mc = [int(v) for v in s.method_class]
    cand, proposers = set(), set()
    for (x, y), (i, u) in sims.items():
        if i / u > py_avg and mc[x] != mc[y]:
            cand.add((x, mc[y]))
            cand.add((y, mc[x]))
            proposers |= {x, y}
    for p in proposers:
        cand |= {(p, mc[int(t)]) for t in s.calls(p) if mc[int(t)] != mc[p]}
    got = {(m, int(dst[k])) for m in range(s.n_methods) for k in range(rowptr[m], rowptr[m + 1])}
    assert got == cand
    ev = brute.evaluate(s, mask=3, min_improved=2, candidates=sorted(cand))
    assert [tuple(int(v) for v in (k["m"], k["d"], k["n_improved"], k["d_ck_sum"], k["d_cbo_sum"]))
            for k in res.kept] == brute.suggestions(ev)


# ---------------------------------------------------------------- move sequences (abstract, Sec. I)

@pytest.mark.parametrize("seed", range(5))
def test_sequence_rounds_are_non_conflicting_and_additive(seed):
    """Each round's moves: individually kept in the round's state (whole-system
    brute force), pairwise disjoint affected classes, no method twice, and
    maximal (every other kept move conflicts with a taken one).  Applying the
    round changes every class metric by exactly the sum of what each move
    alone changes (recomputed by definition), so the moves do not interact."""
    s = tiny_random(seed + 60)
    seq, final = oracle.sequence(s, mask=3, min_improved=1, rounds=3)
    mc = s.method_class.copy()
    for rnd in sorted({r for r, *_ in seq}):
        moves = [(m, d) for r, m, c_, d in seq if r == rnd]
        cur = synth.System(s.n_classes, s.n_methods, s.n_attrs, mc.copy(), s.attr_class, s.acc_rowptr, s.acc_idx,
                           s.call_rowptr, s.call_idx)
        ev = brute.evaluate(cur, mask=3, min_improved=1)
        kept = brute.suggestions(ev)
        assert all(ev[(m, d)]["flags"] & 0x8000 for m, d in moves)
        affs = [oracle.affected_classes(cur, m, d) for m, d in moves]
        assert all(not (affs[a] & affs[b]) for a in range(len(affs)) for b in range(a))
        assert len({m for m, _ in moves}) == len(moves)
        used = set().union(*affs)
        taken = set(moves)
        for m, d, *_ in kept:
            if (m, d) not in taken:
                assert m in {x for x, _ in moves} or oracle.affected_classes(cur, m, d) & used
        base = brute.class_metrics(cur, [int(v) for v in cur.method_class])
        after_all = mc.copy()
        for m, d in moves:
            after_all[m] = d
        total = brute.class_metrics(cur, [int(v) for v in after_all])
        summed = [dict(b) for b in base]
        for m, d in moves:
            one = mc.copy()
            one[m] = d
            single = brute.class_metrics(cur, [int(v) for v in one])
            for Y in range(s.n_classes):
                for f in ("ck", "cbo"):
                    summed[Y][f] += single[Y][f] - base[Y][f]
        for Y in range(s.n_classes):
            assert (total[Y]["ck"], total[Y]["cbo"]) == (summed[Y]["ck"], summed[Y]["cbo"]), (rnd, Y)
        mc = after_all
    assert np.array_equal(mc, final)


# ---------------------------------------------------------------- rule R3 (Sec. III.A, third rule)

@pytest.mark.parametrize("seed", range(6))
def test_r3_brute_force(seed):
    """R3 against Python: high classes by the exact average, candidates from
    the classes each method uses, CBO changes by whole-system recomputation
    (brute force), kept and ordered by the rule."""
    s = tiny_random(seed + 80)
    kept, rowptr, dst, nhigh = oracle.r3(s)
    base = brute.class_metrics(s, [int(v) for v in s.method_class])
    cbo = [b["cbo"] for b in base]
    high = [v * s.n_classes > sum(cbo) for v in cbo]
    assert nhigh == sum(high)
    mc = [int(v) for v in s.method_class]
    fan_in = [0] * s.n_methods
    for x in range(s.n_methods):
        for t in s.calls(x):
            fan_in[int(t)] += 1
    exp = []
    for m in range(s.n_methods):
        C = mc[m]
        if not high[C]:
            continue
        used = ({mc[int(t)] for t in s.calls(m)} | {int(s.attr_class[a]) for a in s.acc(m)}) - {C}
        for D in sorted(used):
            cls2 = list(mc)
            cls2[m] = D
            after = brute.class_metrics(s, cls2)
            ds, dd = after[C]["cbo"] - cbo[C], after[D]["cbo"] - cbo[D]
            if ds < 0 and dd <= 0:
                exp.append((m, D, fan_in[m], len(s.calls(m)), ds, dd))
    exp.sort(key=lambda t: (-(t[2] + t[3]), t[4] + t[5], t[0], t[1]))
    assert [tuple(int(v) for v in k) for k in kept] == exp


def test_r3_hand_example():
    """m0 (class 0) calls m2 (class 1) and m3 (class 2); m1 (class 0) calls m2;
    m2 calls m3.  CBO = (2, 1, 0): only class 0 is above the average 1.
    m0 -> 1: class 0 keeps only m1 (uses 1): CBO 2 -> 1; class 1 still uses
    only 2: kept.  m0 -> 2: class 2 starts using 1: CBO(2) 0 -> 1, rejected.
    m1 -> 1: class 0 still uses 1 and 2 through m0, rejected."""
    s = make_system([0, 0, 1, 2], [], [[], [], [], []], [[2, 3], [2], [3], []], n_classes=3)
    kept, rowptr, dst, nhigh = oracle.r3(s)
    assert nhigh == 1
    assert list(rowptr) == [0, 2, 3, 3, 3] and list(dst) == [1, 2, 1]
    assert [tuple(int(v) for v in k) for k in kept] == [(0, 1, 0, 2, -1, 0)]


# ---------------------------------------------------------------- metric variants (Sec. II.B)

def _variants(s, cbo_attrs=True):
    v, q_all = oracle.Oracle(s, cbo_attrs=cbo_attrs, threads=2).class_variants()
    return v, q_all


@pytest.mark.parametrize("k", [2, 3, 9])
def test_variants_sharing_only_a_foreign_attribute(k):
    """k methods of class 0 all read one attribute owned by class 1 and nothing
    else: no pair shares an owned attribute (P = k(k-1)/2, Q = 0) but every pair
    shares an accessed one (P_all = 0, Q_all = k(k-1)/2); unclamped
    pq = k(k-1)/2 and pq_all = -k(k-1)/2, clamped ck_all = 0."""
    s = make_system([0] * k + [1], [1], [[0]] * k + [[]], [[] for _ in range(k + 1)], n_classes=2)
    v, q_all = _variants(s)
    pairs = k * (k - 1) // 2
    assert (v["P_all"][0], v["Q_all"][0], v["ck_all"][0]) == (0, pairs, 0)
    assert (v["pq"][0], v["pq_all"][0]) == (pairs, -pairs)
    assert list(q_all[:k]) == [k - 1] * k and q_all[k] == 0


def test_variants_mix_of_own_and_foreign_sharing():
    """Methods 0, 1 share an owned attribute, 1, 2 share a foreign one, 3 shares
    nothing: Q = 1, Q_all = 2 of the 6 pairs; ck = 5 - 1 = 4, ck_all = 4 - 2 = 2."""
    s = make_system([0, 0, 0, 0, 1], [0, 1, 0], [[0], [0, 1], [1], [2], []], [[] for _ in range(5)],
                    n_classes=2)
    cm = oracle.Oracle(s, threads=1).class_metrics()
    v, q_all = _variants(s)
    assert (cm["P"][0], cm["Q"][0], cm["ck"][0]) == (5, 1, 4)
    assert (v["P_all"][0], v["Q_all"][0], v["ck_all"][0], v["pq"][0], v["pq_all"][0]) == (4, 2, 2, 4, 2)
    assert list(q_all[:4]) == [1, 2, 1, 0]


@pytest.mark.parametrize("k", [1, 4, 11])
def test_variants_cbo_star_both_ways(k):
    """k leaf classes each call one method of a hub class: the hub uses nothing
    (cbo_out 0) and is used by k classes (cbo_in = cbo_bi = k); each leaf has
    cbo_out = cbo_bi = 1, cbo_in = 0."""
    mc = [0] + list(range(1, k + 1))
    s = make_system(mc, [], [[] for _ in mc], [[]] + [[0] for _ in range(k)], n_classes=k + 1)
    v, _ = _variants(s)
    assert (v["cbo_out"][0], v["cbo_in"][0], v["cbo_bi"][0]) == (0, k, k)
    assert all(v["cbo_out"][1:] == 1) and all(v["cbo_in"][1:] == 0) and all(v["cbo_bi"][1:] == 1)


def test_variants_mutual_coupling_counts_once():
    """Two classes calling each other: each is coupled to one class in each
    direction and to one class either way (the union, not the sum)."""
    s = make_system([0, 1], [], [[], []], [[1], [0]], n_classes=2)
    v, _ = _variants(s)
    assert list(v["cbo_out"]) == [1, 1] and list(v["cbo_in"]) == [1, 1] and list(v["cbo_bi"]) == [1, 1]


def test_variants_attribute_coupling_switch():
    """Reading another class's attribute couples both ways only when attribute
    uses count (cbo_attrs)."""
    s = make_system([0, 1], [1], [[0], []], [[], []], n_classes=2)
    on, _ = _variants(s, cbo_attrs=True)
    off, _ = _variants(s, cbo_attrs=False)
    assert (on["cbo_out"][0], on["cbo_in"][1], on["cbo_bi"][1]) == (1, 1, 1)
    assert (off["cbo_out"][0], off["cbo_in"][1], off["cbo_bi"][1]) == (0, 0, 0)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("cbo_attrs", [True, False])
def test_variants_match_brute_force(seed, cbo_attrs):
    s = tiny_random(seed)
    v, q_all = _variants(s, cbo_attrs)
    bv, bq = brute.variants(s, cbo_attrs)
    for f in oracle.VARIANT_FIELDS:
        assert [int(x) for x in v[f]] == [r[f] for r in bv], f
    assert [int(x) for x in q_all] == bq


def test_variants_invariants_on_medium_sample():
    """On a generated system: every coupled pair counts once on each side
    (sum cbo_out = sum cbo_in = the multigraph's distinct pairs), max(out, in)
    <= bi <= out + in, cbo_out equals CBO, owned sharing implies sharing
    (Q <= Q_all, q <= q_all), and P_all + Q_all = n(n-1)/2."""
    s = synth.generate(n_classes=400, n_methods=4000, n_attrs=2000, max_class=60, seed=5,
                       lambda_acc=3.0, lambda_call=4.0, p_loc=0.7)
    o = oracle.Oracle(s, threads=4)
    cm, mm_ = o.class_metrics(), o.method_metrics()
    v, q_all = o.class_variants()
    rowptr, _, _ = o.multigraph()
    assert v["cbo_out"].sum() == v["cbo_in"].sum() == rowptr[-1]
    assert np.array_equal(v["cbo_out"], cm["cbo"])
    assert np.all(np.maximum(v["cbo_out"], v["cbo_in"]) <= v["cbo_bi"])
    assert np.all(v["cbo_bi"] <= v["cbo_out"] + v["cbo_in"])
    assert np.all(cm["Q"] <= v["Q_all"]) and np.all(mm_["q"] <= q_all)
    n = cm["n"]
    assert np.array_equal(v["P_all"] + v["Q_all"], n * (n - 1) // 2)
    assert np.array_equal(v["pq"], cm["P"] - cm["Q"])
    assert np.array_equal(np.maximum(v["pq"], 0), cm["ck"])


def test_variants_reduce_to_lcom_when_every_access_is_own():
    """When every accessed attribute belongs to the accessing method's class,
    sharing over accessed attributes is sharing over owned ones: Q_all = Q."""
    s = synth.generate(n_classes=60, n_methods=900, n_attrs=500, max_class=40, seed=8,
                       lambda_acc=3.0, lambda_call=2.0, p_loc=0.7)
    keep = s.attr_class[s.acc_idx] == np.repeat(s.method_class, np.diff(s.acc_rowptr))
    rows = [[int(a) for a, k in zip(s.acc(x), keep[s.acc_rowptr[x]:s.acc_rowptr[x + 1]]) if k]
            for x in range(s.n_methods)]
    own_only = make_system(s.method_class, s.attr_class, rows, [list(map(int, s.calls(x)))
                                                              for x in range(s.n_methods)], s.n_classes)
    o = oracle.Oracle(own_only, threads=2)
    cm = o.class_metrics()
    v, q_all = o.class_variants()
    assert np.array_equal(v["Q_all"], cm["Q"]) and np.array_equal(q_all, o.method_metrics()["q"])
    assert cm["Q"].sum() > 0


def test_rank_classes_by_metric():
    """Largest value first, equal values by ascending class id, first k."""
    vals = np.array([3, -1, 7, 3, 0, 7, -5], dtype=np.int64)
    assert list(oracle.rank_classes(vals, 7)) == [2, 5, 0, 3, 4, 1, 6]
    assert list(oracle.rank_classes(vals, 3)) == [2, 5, 0]
    assert list(oracle.rank_classes(vals, 0)) == []
    s = tiny_random(4)
    bv, _ = brute.variants(s)
    by_pq = sorted(range(s.n_classes), key=lambda C: bv[C]["pq"], reverse=True)  # stable: ids ascending on ties
    v, _ = _variants(s)
    assert list(oracle.rank_classes(v["pq"], s.n_classes)) == by_pq
