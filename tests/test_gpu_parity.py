"""GPU parity: every output of the CUDA path, through the C ABI, equals the
CPU oracle bit for bit (all outputs are integers).  The oracle itself is pinned
by tests/test_oracle_pins.py."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1308_4011_b300 import synth

from sysutil import make_system, moved, permute, tiny_random

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines deselect with -m "not gpu"
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402  (loads libmmref.so; no fallback)

CLASS_MAP = {"n_methods": "n", "n_attrs": "a", "P": "P", "Q": "Q", "S": "S", "lcom_ck": "ck",
             "hs_num": "hs_num", "hs_den": "hs_den", "cbo": "cbo"}
CRITERIA = [(7, 2), (3, 2), (1, 1), (4, 1), (6, 1), (2, 2)]


def gpu_load(sys_, cbo_attrs=True, device=False):
    s = mmref.load_synth(sys_, cbo_attrs=cbo_attrs, device=device)
    cm, mm_ = mmref.compute_metrics(s, "host", "host")
    return s, cm, mm_


def check_metrics(sys_, o, cm, mm_):
    ocm, omm = o.class_metrics(), o.method_metrics()
    for g, f in CLASS_MAP.items():
        assert np.array_equal(cm[g].astype(np.int64), ocm[f]), g
    for f in ("fan_in", "fan_out", "own", "q"):
        assert np.array_equal(mm_[f], omm[f]), f


def gpu_records(s, mask, mi, rowptr=None, dst=None):
    n = s.n_candidates_full if rowptr is None else len(dst)
    rec = torch.empty(max(n, 1) * 16, dtype=torch.uint8, device="cuda")
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    mmref.evaluate_moves(s, mask, mi, rowptr, dst, records=rec, digest=dig)
    torch.cuda.synchronize()
    r = rec[: n * 16].cpu().numpy().view(mmref.MOVE_EVAL_DTYPE)
    return r, int(dig.cpu().numpy().view(np.uint64)[0])


def gpu_digest(s, mask, mi, rowptr=None, dst=None):
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(s, mask, mi, rowptr, dst, digest=dig)
    return int(dig[0])


def kept_tuples(arr, names=("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")):
    return [tuple(int(x[f]) for f in names) for x in arr]


def oracle_kept(res):
    return [tuple(int(x[f]) for f in ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")) for x in res.kept]


def same_records(gpu, orc):
    return np.array_equal(np.ascontiguousarray(gpu).view(np.uint8), np.ascontiguousarray(orc).view(np.uint8))


# ---------------------------------------------------------------- tiny workload

@pytest.fixture(scope="module")
def tiny():
    s = synth.named("tiny")
    return s, oracle.Oracle(s), oracle.Oracle(s, cbo_attrs=False)


@pytest.mark.parametrize("cbo_attrs", [True, False])
def test_tiny_metrics(tiny, cbo_attrs):
    s, o1, o2 = tiny
    g, cm, mm_ = gpu_load(s, cbo_attrs=cbo_attrs)
    check_metrics(s, o1 if cbo_attrs else o2, cm, mm_)
    assert g.info()["n_class_edges"] == len(o1.multigraph()[1] if cbo_attrs else o2.multigraph()[1])


@pytest.mark.parametrize("mask,mi", CRITERIA)
def test_tiny_every_record(tiny, mask, mi):
    """All 398,000 candidates of the tiny workload, record by record."""
    s, o, _ = tiny
    g, _, _ = gpu_load(s)
    rec, dig = gpu_records(g, mask, mi)
    ref = o.evaluate(mask=mask, min_improved=mi, method=1, records=True)
    assert rec.shape[0] == ref.n_cand == 2000 * 199
    assert same_records(rec, ref.records)
    assert dig == ref.digest
    assert gpu_digest(g, mask, mi) == ref.digest


def test_tiny_records_vs_recompute(tiny):
    """Against O0, the recompute-after-move oracle, on every candidate."""
    s, o, _ = tiny
    g, _, _ = gpu_load(s)
    rec, dig = gpu_records(g, 7, 2)
    ref = o.evaluate(mask=7, min_improved=2, method=0, records=True)
    assert same_records(rec, ref.records) and dig == ref.digest


@pytest.mark.parametrize("mask,mi", CRITERIA)
def test_tiny_suggestions(tiny, mask, mi):
    s, o, _ = tiny
    g, _, _ = gpu_load(s)
    ref = o.evaluate(mask=mask, min_improved=mi, method=1)
    top, nk, nm = mmref.suggest_moves(g, k=ref.n_kept + 5, mask=mask, min_improved=mi)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)
    top10, nk2, _ = mmref.suggest_moves(g, k=10, mask=mask, min_improved=mi)
    assert nk2 == nk and kept_tuples(top10) == oracle_kept(ref)[:10]


def test_tiny_device_inputs_and_outputs(tiny):
    s, o, _ = tiny
    g = mmref.load_synth(s, device=True)
    cm = torch.empty(s.n_classes * 64, dtype=torch.uint8, device="cuda")
    mm_ = torch.empty(s.n_methods * 16, dtype=torch.uint8, device="cuda")
    mmref.compute_metrics(g, cm, mm_)
    check_metrics(s, o, cm.cpu().numpy().view(mmref.CLASS_METRICS_DTYPE),
                  mm_.cpu().numpy().view(mmref.METHOD_METRICS_DTYPE))
    out = torch.empty(50 * 24, dtype=torch.uint8, device="cuda")
    _, nk, _ = mmref.suggest_moves(g, k=50, out=out)
    ref = o.evaluate(mask=3, min_improved=2)
    n = min(50, nk)
    assert kept_tuples(out.cpu().numpy().view(mmref.MOVE_DTYPE)[:n]) == oracle_kept(ref)[:n]


def test_tiny_restricted_equals_dense(tiny):
    """The CSR kernel on the full cross product written as a list equals the dense kernel."""
    s, o, _ = tiny
    g, _, _ = gpu_load(s)
    c = s.n_classes
    rowptr = np.arange(s.n_methods + 1, dtype=np.int64) * (c - 1)
    dst = np.concatenate([np.delete(np.arange(c, dtype=np.int32), s.method_class[m]) for m in range(s.n_methods)])
    a, da = gpu_records(g, 7, 1)
    b, db = gpu_records(g, 7, 1, rowptr, dst)
    assert same_records(a, b) and da == db
    # device-resident candidate list too
    b2, db2 = gpu_records(g, 7, 1, torch.from_numpy(rowptr).cuda(), torch.from_numpy(dst).cuda())
    assert same_records(a, b2) and da == db2


# ---------------------------------------------------------------- tiny random systems, brute-force pinned

@pytest.mark.parametrize("seed", range(16))
def test_random_tiny_vs_brute_force(seed):
    s = tiny_random(seed)
    for cbo_attrs in (True, False):
        g, cm, mm_ = gpu_load(s, cbo_attrs=cbo_attrs)
        o = oracle.Oracle(s, cbo_attrs=cbo_attrs, threads=1)
        check_metrics(s, o, cm, mm_)
        for mask, mi in ((7, 2), (3, 2), (7, 1)):
            ev = brute.evaluate(s, mask=mask, min_improved=mi, cbo_attrs=cbo_attrs)
            rec, dig = gpu_records(g, mask, mi)
            assert dig == brute.digest(ev)
            exp = [tuple(ev[(m, D)][f] for f in mmref.MOVE_EVAL_DTYPE.names)
                   for m in range(s.n_methods) for D in range(s.n_classes) if D != s.method_class[m]]
            assert [tuple(int(v) for v in r) for r in rec] == exp
            top, nk, _ = mmref.suggest_moves(g, k=1000, mask=mask, min_improved=mi)
            assert kept_tuples(top) == brute.suggestions(ev)


# ---------------------------------------------------------------- edge cases

def _eval_all_ways(sys_, cbo_attrs=True):
    g, cm, mm_ = gpu_load(sys_, cbo_attrs=cbo_attrs)
    o = oracle.Oracle(sys_, cbo_attrs=cbo_attrs, threads=1)
    check_metrics(sys_, o, cm, mm_)
    for mask, mi in ((7, 2), (7, 1), (3, 1)):
        ref = o.evaluate(mask=mask, min_improved=mi, method=0, records=True)
        if g.n_candidates_full:
            rec, dig = gpu_records(g, mask, mi)
            assert same_records(rec, ref.records) and dig == ref.digest
        top, nk, nm = mmref.suggest_moves(g, k=100000, mask=mask, min_improved=mi)
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert kept_tuples(top) == oracle_kept(ref)


def test_single_class_has_no_candidates():
    s = make_system([0, 0, 0], [0, 0], [[0], [0, 1], []], [[1], [2], []], n_classes=1)
    g, cm, _ = gpu_load(s)
    assert g.n_candidates_full == 0
    assert (cm["P"][0], cm["Q"][0]) == (2, 1)
    _, dig = np.zeros(0), gpu_digest(g, 7, 2)
    assert dig == 0
    top, nk, nm = mmref.suggest_moves(g, k=5)
    assert (len(top), nk, nm) == (0, 0, 0)


def test_empty_classes_and_no_attributes():
    """Classes without methods (moves into an empty class), no attributes at all."""
    s = make_system([0, 0, 2, 2, 2], [], [[], [], [], [], []], [[1, 2], [], [0], [], [1]], n_classes=4)
    _eval_all_ways(s)


def test_emptying_a_class_and_methods_without_accesses():
    s = make_system([0, 1, 1, 2, 3, 3, 3], [1, 1, 3, 0], [[0, 1], [], [1], [2, 3], [2], [], [0]],
                    [[1], [0], [], [4, 5], [], [6], [3]], n_classes=5)
    _eval_all_ways(s)
    _eval_all_ways(s, cbo_attrs=False)


@pytest.mark.parametrize("c", [31, 33, 257, 300])
def test_ragged_class_counts(c):
    """Class counts off the 32-lane and 256-thread grids (ragged D tiles)."""
    s = synth.generate(c, 6 * c, 3 * c, max_class=40, seed=c, lambda_acc=3, lambda_call=3, p_loc=0.6)
    g, cm, mm_ = gpu_load(s)
    o = oracle.Oracle(s)
    check_metrics(s, o, cm, mm_)
    rec, dig = gpu_records(g, 7, 1)
    ref = o.evaluate(mask=7, min_improved=1, method=1, records=True)
    assert same_records(rec, ref.records) and dig == ref.digest


def test_large_class_multi_tile_lcom():
    """A class of 300 methods and 100 attributes (10 x 10 pair tiles, 4 words per row)."""
    rng = np.random.default_rng(7)
    n, a = 300, 100
    acc = [sorted(rng.choice(a, size=rng.integers(0, 6), replace=False).tolist()) for _ in range(n)]
    s = make_system([0] * n + [1] * 5, [0] * a + [1] * 3, acc + [[a], [a + 1], [], [a, a + 2], [0]],
                    [[] for _ in range(n + 5)], n_classes=2)
    g, cm, mm_ = gpu_load(s)
    check_metrics(s, oracle.Oracle(s), cm, mm_)


def test_long_rows_take_the_general_list_paths():
    """A method using 150 classes and one called from 120 classes: its use keys
    and its callers' classes exceed one warp (the per-method sort and run walk
    fall back to their long-segment paths); attributes of many classes, several
    per class (sharing counts from unions of two or more accessor lists); an
    explicit candidate list with long rows (more than 62 list entries: the
    general per-candidate path of the restricted kernel)."""
    rng = np.random.default_rng(11)
    c, per = 160, 3
    method_class = [C for C in range(c) for _ in range(per)]      # methods 3C, 3C+1, 3C+2 in class C
    attr_class = [C for C in range(c) for _ in range(2)]          # attributes 2C, 2C+1
    M = len(method_class)
    acc = [sorted(rng.choice(len(attr_class), size=rng.integers(0, 4), replace=False).tolist()) for _ in range(M)]
    calls = [sorted(set(rng.choice(M, size=rng.integers(0, 4)).tolist()) - {x}) for x in range(M)]
    hub = 0                                                       # uses 150 classes, reads 2 attributes of 70
    calls[hub] = sorted({3 * C + 1 for C in range(1, 151)})
    acc[hub] = sorted({2 * C + k for C in range(1, 71) for k in (0, 1)})
    callee = 4                                                    # called from methods of 120 classes
    for C in range(10, 130):
        y = 3 * C + 2
        calls[y] = sorted(set(calls[y]) | {callee})
    s = make_system(method_class, attr_class, acc, calls, n_classes=c)
    _eval_all_ways(s)
    _eval_all_ways(s, cbo_attrs=False)
    # restricted lists: every other class for the hub and the callee, 5 classes for the rest
    rows = []
    for x in range(M):
        C = method_class[x]
        if x in (hub, callee):
            rows.append([D for D in range(c) if D != C])
        else:
            rows.append(sorted(set(rng.choice(c, size=5).tolist()) - {C}))
    rp = np.zeros(M + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    dst = np.asarray([D for r in rows for D in r], dtype=np.int32)
    g, _, _ = gpu_load(s, device=True)
    o = oracle.Oracle(s, threads=1)
    for mask, mi in ((7, 1), (3, 1)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = gpu_records(g, mask, mi, torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda())
        assert same_records(rec, ref.records) and dig == ref.digest
        top, nk, nm = mmref.suggest_moves(g, k=100000, mask=mask, min_improved=mi,
                                          cand_rowptr=torch.from_numpy(rp).cuda(),
                                          cand_dst=torch.from_numpy(dst).cuda())
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert kept_tuples(top) == oracle_kept(ref)


def test_class_too_big_for_shared_bitmaps():
    """A class of 50,000 methods: the accessor-union bitmaps (one bit per
    method of the class) no longer fit shared memory and live in global
    memory.  Closed forms: a methods read {a0, a1}, b methods read {a1}, k
    methods read {a2}, the rest read nothing, so the sharing pairs are the
    pairs inside the first a + b methods and inside the k methods."""
    n, a, b, k = 50000, 40, 25, 30
    acc = [[0, 1]] * a + [[1]] * b + [[2]] * k + [[]] * (n - a - b - k)
    # class 1: m reads a0 and a2 of class 0 (t = 2: the union of two accessor lists) and its own attribute
    acc = acc + [[0, 2, 3], [3]]
    s = make_system([0] * n + [1, 1], [0, 0, 0, 1], acc, [[] for _ in range(n + 2)], n_classes=2)
    g, cm, mm_ = gpu_load(s, device=True)
    Q = (a + b) * (a + b - 1) // 2 + k * (k - 1) // 2
    assert int(cm["Q"][0]) == Q and int(cm["P"][0]) == n * (n - 1) // 2 - Q
    q = mm_["q"][:n]
    assert (q[: a + b] == a + b - 1).all() and (q[a + b: a + b + k] == k - 1).all() and (q[a + b + k:] == 0).all()
    assert int(cm["Q"][1]) == 1 and int(cm["P"][1]) == 0
    rp = torch.tensor([0] * (n + 1) + [1, 1], dtype=torch.int64, device="cuda")  # one candidate: m = n -> class 0
    dst = torch.tensor([0], dtype=torch.int32, device="cuda")
    rec, _ = gpu_records(g, 7, 1, rp, dst)
    assert int(rec["s"][0]) == a + k and int(rec["t"][0]) == 2


@pytest.mark.parametrize("c,M", [(200, 2500), (300, 5000), (300, 10000)])
def test_kept_sort_regimes(c, M):
    """About 1,900, 4,000 and 32,000 kept moves (CBO, min_improved 1): the
    keyed sort (keys by one block, ranks by a block per 32 moves) at 60 and 125
    rank blocks and the radix sort above 8,192 give the oracle's full
    suggestion order, straight after the metrics and after an evaluation
    cached the kept moves."""
    s = synth.generate(n_classes=c, n_methods=M, n_attrs=M, max_class=max(40, 3 * M // c), seed=7)
    ref = oracle.Oracle(s, threads=4).evaluate(mask=4, min_improved=1)
    g, _, _ = gpu_load(s)
    top, nk, nm = mmref.suggest_moves(g, k=ref.n_kept, mask=4, min_improved=1)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)
    assert gpu_digest(g, 4, 1) == ref.digest
    top2, nk2, _ = mmref.suggest_moves(g, k=100, mask=4, min_improved=1)
    assert nk2 == nk and kept_tuples(top2) == oracle_kept(ref)[:100]
    g.free()


def test_relabelled_system_gives_permuted_results():
    s = tiny_random(5)
    p, pc, pm, pa = permute(s, 3)
    _, cm, mm_ = gpu_load(s)
    _, cmp_, mmp = gpu_load(p)
    assert np.array_equal(cmp_[pc], cm)
    assert np.array_equal(mmp[pm], mm_)


def test_move_then_move_back_on_gpu():
    s = synth.named("tiny")
    g, cm, _ = gpu_load(s)
    rng = np.random.default_rng(0)
    for _ in range(5):
        m = int(rng.integers(s.n_methods))
        C = int(s.method_class[m])
        D = int(rng.integers(s.n_classes - 1))
        D += D >= C
        rp = np.zeros(s.n_methods + 1, dtype=np.int64)
        rp[m + 1:] = 1
        fwd, _ = gpu_records(g, 7, 1, rp, np.array([D], dtype=np.int32))
        g2, cm2, _ = gpu_load(moved(s, m, D))
        assert cm2["cbo"][C] == cm["cbo"][C] + fwd["dcbo_src"][0]
        assert cm2["cbo"][D] == cm["cbo"][D] + fwd["dcbo_dst"][0]
        assert cm2["Q"][D] == cm["Q"][D] + fwd["s"][0]
        assert cm2["S"][D] == cm["S"][D] + fwd["t"][0]
        rp2 = rp.copy()
        back, _ = gpu_records(g2, 7, 1, rp2, np.array([C], dtype=np.int32))
        assert back["dcbo_src"][0] == -fwd["dcbo_dst"][0] and back["dcbo_dst"][0] == -fwd["dcbo_src"][0]


# ---------------------------------------------------------------- invalid input

def _bad(**kw):
    s = synth.generate(10, 40, 20, max_class=10, seed=1)
    arrs = dict(method_class=s.method_class.copy(), attr_class=s.attr_class.copy(),
                acc_rowptr=s.acc_rowptr.copy(), acc_idx=s.acc_idx.copy(), call_rowptr=s.call_rowptr.copy(),
                call_idx=s.call_idx.copy())
    for k, f in kw.items():
        f(arrs[k])
    return arrs


@pytest.mark.parametrize("name,edit,msg", [
    ("method_class", lambda a: a.__setitem__(3, 10), "method_class"),
    ("attr_class", lambda a: a.__setitem__(0, -1), "attr_class"),
    ("acc_idx", lambda a: a.__setitem__(0, 999), "acc_idx"),
    ("call_idx", lambda a: a.__setitem__(0, 4000), "call_idx"),
    ("acc_rowptr", lambda a: a.__setitem__(-1, a[-1] - 1), "acc_rowptr"),
])
def test_invalid_systems_rejected(name, edit, msg):
    arrs = _bad(**{name: edit})
    with pytest.raises(mmref.MMError) as e:
        mmref.load_system(10, **arrs)
    assert e.value.status == mmref.MM_EINVAL and msg in str(e.value)


def test_unsorted_and_self_calls_rejected():
    s = synth.generate(10, 40, 20, max_class=10, seed=1)
    x = int(np.argmax(np.diff(s.call_rowptr) >= 2))
    ci = s.call_idx.copy()
    a, b = s.call_rowptr[x], s.call_rowptr[x] + 1
    ci[a], ci[b] = ci[b], ci[a]
    with pytest.raises(mmref.MMError, match="strictly increasing"):
        mmref.load_system(10, s.method_class, s.attr_class, s.acc_rowptr, s.acc_idx, s.call_rowptr, ci)
    ci = s.call_idx.copy()
    ci[s.call_rowptr[x]] = x
    ci[s.call_rowptr[x]:s.call_rowptr[x + 1]].sort()
    with pytest.raises(mmref.MMError):
        mmref.load_system(10, s.method_class, s.attr_class, s.acc_rowptr, s.acc_idx, s.call_rowptr, ci)


@pytest.mark.parametrize("M,A", [(4097, 4096), (16384, 16385), (16385, 16384)])
def test_scan_size_boundaries(M, A):
    """Method and attribute counts at the edges of the scans: one block up to
    16,384 elements, one pass over tiles of 4,096 above (a last tile of one
    element included).  Metrics and every record's digest equal the oracle."""
    s = synth.generate(n_classes=40, n_methods=M, n_attrs=A, max_class=max(2 * M // 40, 40), seed=M + A)
    o = oracle.Oracle(s, threads=4)
    g, cm, mm_ = gpu_load(s)
    check_metrics(s, o, cm, mm_)
    ref = o.evaluate(mask=7, min_improved=1)
    assert gpu_digest(g, 7, 1) == ref.digest
    g.free()


def _short_row_candidates(s, seed):
    """Candidate lists where most rows hold 0-3 destinations (so a chunk of 128
    candidates spans more than 32 rows) and a few hold 40."""
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 0, 1, 2, 3, 40], size=s.n_methods)
    rows = []
    for m in range(s.n_methods):
        others = np.array([d for d in range(s.n_classes) if d != s.method_class[m]], dtype=np.int32)
        rows.append(np.sort(rng.choice(others, size=min(int(lens[m]), len(others)), replace=False)))
    rowptr = np.zeros(s.n_methods + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    return rowptr, np.concatenate(rows).astype(np.int32)


def test_candidate_validation_with_short_rows():
    """Validation and hashing of lists whose chunks span many rows (the
    per-lane walk) and few rows (the per-position count): results equal the
    oracle, the kept cache is reused, and a self move or an out-of-range class
    deep inside the short rows is rejected."""
    s = synth.generate(n_classes=50, n_methods=3000, n_attrs=1500, max_class=120, seed=5)
    rowptr, dst = _short_row_candidates(s, 5)
    ref = oracle.Oracle(s, threads=4).evaluate(mask=4, min_improved=1, cand_rowptr=rowptr, cand_dst=dst)
    g, _, _ = gpu_load(s)
    assert gpu_digest(g, 4, 1, rowptr, dst) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, k=ref.n_kept, mask=4, min_improved=1, cand_rowptr=rowptr, cand_dst=dst)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)
    lens = np.diff(rowptr)
    m = int(np.nonzero(lens[2000:] >= 1)[0][0]) + 2000
    bad = dst.copy()
    bad[rowptr[m]] = s.method_class[m]
    with pytest.raises(mmref.MMError, match="own class"):
        mmref.evaluate_moves(g, 4, 1, rowptr, bad, digest=np.zeros(1, np.uint64))
    bad = dst.copy()
    bad[rowptr[m]] = s.n_classes
    with pytest.raises(mmref.MMError):
        mmref.evaluate_moves(g, 4, 1, rowptr, bad, digest=np.zeros(1, np.uint64))
    assert gpu_digest(g, 4, 1, rowptr, dst) == ref.digest  # the valid lists still evaluate
    g.free()


@pytest.mark.parametrize("offset", [0, 1, 3])
def test_device_lists_at_any_alignment(offset):
    """Device-resident candidate lists whose destinations start 0, 4 or 12
    bytes past a 16-byte boundary (vector and scalar loads of the validation
    pass), with chunks of 128 entries that span few and many rows: digest and
    kept moves equal the oracle's, and a self move in the middle is found."""
    s = synth.generate(n_classes=60, n_methods=4000, n_attrs=2000, max_class=150, seed=9)
    rowptr, dst = _short_row_candidates(s, 9)
    ref = oracle.Oracle(s, threads=4).evaluate(mask=4, min_improved=1, cand_rowptr=rowptr, cand_dst=dst)
    n = len(dst)
    buf = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    buf[offset: offset + n] = torch.from_numpy(dst).cuda()
    ddst = buf[offset: offset + n]
    drp = torch.from_numpy(rowptr).cuda()
    torch.cuda.synchronize()
    g, _, _ = gpu_load(s)
    assert gpu_digest(g, 4, 1, drp, ddst) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, k=ref.n_kept, mask=4, min_improved=1, cand_rowptr=drp, cand_dst=ddst)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)
    mid = n // 2
    owner = int(np.searchsorted(rowptr, mid, side="right")) - 1
    ddst[mid] = int(s.method_class[owner])
    torch.cuda.synchronize()
    with pytest.raises(mmref.MMError, match="own class"):
        mmref.evaluate_moves(g, 4, 1, drp, ddst, digest=np.zeros(1, np.uint64))
    g.free()


def test_invalid_candidates_and_criteria_rejected():
    s = synth.generate(10, 40, 20, max_class=10, seed=1)
    g, _, _ = gpu_load(s)
    rp = np.zeros(41, dtype=np.int64)
    rp[1:] = 1
    with pytest.raises(mmref.MMError, match="own class"):
        mmref.evaluate_moves(g, 7, 2, rp, np.array([s.method_class[0]], dtype=np.int32), digest=np.zeros(1, np.uint64))
    with pytest.raises(mmref.MMError, match="out of range"):
        mmref.evaluate_moves(g, 7, 2, rp, np.array([10], dtype=np.int32), digest=np.zeros(1, np.uint64))
    with pytest.raises(mmref.MMError, match="metric_mask"):
        mmref.suggest_moves(g, 5, mask=0)
    with pytest.raises(mmref.MMError, match="min_improved"):
        mmref.suggest_moves(g, 5, mask=7, min_improved=0)
    # the system is still usable after the errors
    assert gpu_digest(g, 7, 2) == oracle.Oracle(s).evaluate(mask=7, min_improved=2).digest


# ---------------------------------------------------------------- full-size workloads

@pytest.fixture(scope="module")
def medium():
    s = synth.named("medium")
    return s, oracle.Oracle(s)


def test_medium_metrics(medium):
    s, o = medium
    _, cm, mm_ = gpu_load(s, device=True)
    check_metrics(s, o, cm, mm_)


def test_medium_full_cross_product(medium):
    """299,940,000 candidates: the digest of every record equals the oracle's,
    dense records on the device, in the launch configuration the benchmark uses;
    sampled records equal the recompute oracle one by one."""
    s, o = medium
    g, _, _ = gpu_load(s, device=True)
    n = g.n_candidates_full
    assert n == 60000 * 4999
    rec = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    mmref.evaluate_moves(g, 3, 2, records=rec, digest=dig)
    ref = o.evaluate(mask=3, min_improved=2, method=1)
    assert int(dig.cpu().numpy().view(np.uint64)[0]) == ref.digest
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(n, size=400, replace=False))
    recs = rec.view(-1, 16)[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1).view(mmref.MOVE_EVAL_DTYPE)
    c = s.n_classes
    for i, r in zip(idx, recs):
        m, j = divmod(int(i), c - 1)
        D = j + (j >= s.method_class[m])
        exp, _, _ = o.evaluate_one(m, D, mask=3, min_improved=2, method=0)
        assert same_records(np.array([r]), np.array([exp])), (m, D)
    del rec
    top, nk, nm = mmref.suggest_moves(g, k=ref.n_kept, mask=3, min_improved=2)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)


def test_medium_host_buffers_path(medium):
    """The end-to-end form: host CSR in, host results out."""
    s, o = medium
    g = mmref.load_synth(s)
    cm, _ = mmref.compute_metrics(g, "host", None)
    assert np.array_equal(cm["cbo"].astype(np.int64), o.class_metrics()["cbo"])
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 2, digest=dig)
    assert int(dig[0]) == o.evaluate(mask=7, min_improved=2).digest


@pytest.fixture(scope="module")
def large():
    s = synth.named("large")
    rp, dst = synth.candidates(s, synth.LARGE_EXTRA_CANDIDATES, seed=2)
    return s, rp, dst, oracle.Oracle(s)


def test_large_metrics(large):
    s, _, _, o = large
    _, cm, mm_ = gpu_load(s, device=True)
    check_metrics(s, o, cm, mm_)


def test_large_restricted_candidates(large):
    s, rp, dst, o = large
    g, _, _ = gpu_load(s, device=True)
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    n = len(dst)
    rec = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    mmref.evaluate_moves(g, 7, 1, rpd, dd, records=rec, digest=dig)
    ref = o.evaluate(mask=7, min_improved=1, cand_rowptr=rp, cand_dst=dst, method=1)
    assert int(dig.cpu().numpy().view(np.uint64)[0]) == ref.digest
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, size=300, replace=False))
    recs = rec.view(-1, 16)[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1).view(mmref.MOVE_EVAL_DTYPE)
    rows = np.searchsorted(rp, idx, side="right") - 1
    for i, m, r in zip(idx, rows, recs):
        exp, _, _ = o.evaluate_one(int(m), int(dst[i]), mask=7, min_improved=1, method=0)
        assert same_records(np.array([r]), np.array([exp])), (m, dst[i])
    top, nk, nm = mmref.suggest_moves(g, k=min(ref.n_kept, 5000), mask=7, min_improved=1, cand_rowptr=rpd,
                                      cand_dst=dd)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)[:5000]


# ---------------------------------------------------------------- many classes

def test_forty_thousand_classes_restricted():
    """40,000 classes and 50,000 methods with restricted lists (classes used +
    16 others): adjacency rows of 1,252 words, compressed records over 40
    summary words per row; every record equals the oracle's."""
    s = synth.generate(40000, 50000, 25000, max_class=400, seed=41, lambda_acc=4, lambda_call=6, p_loc=0.75)
    rp, dst = synth.candidates(s, 16, seed=41)
    g, cm, mm_ = gpu_load(s, device=True)
    o = oracle.Oracle(s)
    check_metrics(s, o, cm, mm_)
    assert g.info()["n_class_edges"] == len(o.multigraph()[1])
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    for mask, mi in ((7, 1), (3, 2), (4, 1)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = gpu_records(g, mask, mi, rpd, dd)
        assert same_records(rec, ref.records) and dig == ref.digest, mask
        top, nk, nm = mmref.suggest_moves(g, k=100000, mask=mask, min_improved=mi, cand_rowptr=rpd, cand_dst=dd)
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert kept_tuples(top) == oracle_kept(ref)


def test_many_empty_classes_full_cross_product():
    """33,000 classes of which 32,000 are empty: the full cross product over
    rows of 1,032 words (moves into empty classes everywhere)."""
    base = synth.generate(1000, 3000, 1500, max_class=40, seed=43, lambda_acc=3, lambda_call=4, p_loc=0.7)
    # the same system with its classes spread over 33,000 ids (32,000 empty classes)
    s = synth.System(33000, base.n_methods, base.n_attrs, base.method_class * 33, base.attr_class * 33,
                     base.acc_rowptr, base.acc_idx, base.call_rowptr, base.call_idx, name="spread")
    g, cm, mm_ = gpu_load(s, device=True)
    o = oracle.Oracle(s)
    check_metrics(s, o, cm, mm_)
    ref = o.evaluate(mask=7, min_improved=1, method=1)
    assert gpu_digest(g, 7, 1) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, k=100000, mask=7, min_improved=1)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert kept_tuples(top) == oracle_kept(ref)
    # after the metrics are computed again, restricted lists over the same system agree too
    mmref.compute_metrics(g, None, None)
    rp, dst = synth.candidates(s, 8, seed=43)
    ref = o.evaluate(mask=7, min_improved=1, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
    rec, dig = gpu_records(g, 7, 1, rp, dst)
    assert same_records(rec, ref.records) and dig == ref.digest


def test_repeated_destinations_in_lists(tiny):
    """A list may name a destination twice: both positions get the same record."""
    s, o, _ = tiny
    g, _, _ = gpu_load(s)
    rng = np.random.default_rng(3)
    rows = []
    for m in range(s.n_methods):
        C = int(s.method_class[m])
        r = [int(D) for D in rng.choice(s.n_classes, size=12) if D != C]
        rows.append(r + r[: len(r) // 2])  # repeats, unsorted
    rp = np.zeros(s.n_methods + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    dst = np.asarray([D for r in rows for D in r], dtype=np.int32)
    for mask, mi in ((7, 1), (3, 2)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = gpu_records(g, mask, mi, rp, dst)
        assert same_records(rec, ref.records) and dig == ref.digest
        top, nk, nm = mmref.suggest_moves(g, k=100000, mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst)
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert kept_tuples(top) == oracle_kept(ref)


def test_more_than_65535_classes():
    """70,000 classes (35 ids per class of a 2,000-class system): class ids
    past 16 bits in every key, row and record offset of the restricted path."""
    base = synth.generate(2000, 10000, 5000, max_class=60, seed=47, lambda_acc=3, lambda_call=4, p_loc=0.7)
    s = synth.System(70000, base.n_methods, base.n_attrs, base.method_class * 35, base.attr_class * 35,
                     base.acc_rowptr, base.acc_idx, base.call_rowptr, base.call_idx, name="spread-wide")
    g, cm, mm_ = gpu_load(s, device=True)
    o = oracle.Oracle(s)
    check_metrics(s, o, cm, mm_)
    rp, dst = synth.candidates(s, 8, seed=47)
    for mask, mi in ((7, 1), (3, 2)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = gpu_records(g, mask, mi, rp, dst)
        assert same_records(rec, ref.records) and dig == ref.digest
        top, nk, nm = mmref.suggest_moves(g, k=100000, mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst)
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert kept_tuples(top) == oracle_kept(ref)
