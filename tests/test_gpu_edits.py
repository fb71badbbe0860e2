"""Edits (mm_apply_edit): after every edit the patched system, its metrics and
the incrementally maintained suggestions equal the oracle on the edited
system; invalid edits are rejected and change nothing."""
import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

from edits import ADD_ACCESS, ADD_CALL, MOVE, REMOVE_ACCESS, REMOVE_CALL, Tracked
from sysutil import tiny_random

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

KEPT = ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")
MOVE_F = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")


def _check_state(g, tr, mask, mi, cbo_attrs=True):
    s = tr.system()
    exp = (s.method_class, s.attr_class, s.acc_rowptr, s.acc_idx, s.call_rowptr, s.call_idx)
    for a, b in zip(mmref.export_system(g), exp):
        assert np.array_equal(a, b)
    o = oracle.Oracle(s, cbo_attrs=cbo_attrs, threads=4)
    ref = o.evaluate(mask=mask, min_improved=mi)
    top, nk, nm = mmref.suggest_moves(g, ref.n_kept + 1, mask, mi)  # reuses the maintained kept list
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert [tuple(int(x[f]) for f in MOVE_F) for x in top] == [tuple(int(x[f]) for f in KEPT) for x in ref.kept]
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, mask, mi, digest=dig)
    assert int(dig[0]) == ref.digest
    return o


@pytest.mark.parametrize("seed,mask,mi", [(0, 3, 2), (1, 7, 1), (2, 1, 1), (3, 6, 2)])
def test_random_edit_stream_keeps_everything_exact(seed, mask, mi):
    base = synth.generate(60, 500, 250, max_class=30, seed=seed, lambda_acc=3, lambda_call=4, p_loc=0.7)
    tr = Tracked(base)
    g = mmref.load_synth(base, device=True)
    mmref.compute_metrics(g, None, None)
    mmref.suggest_moves(g, 10, mask, mi)  # establishes the kept-move cache for these criteria
    rng = np.random.default_rng(seed)
    for i in range(40):
        kind, m, t = tr.random_edit(rng)
        mmref.apply_edit(g, kind, m, t)
        tr.apply(kind, m, t)
        if i % 8 == 7:
            _check_state(g, tr, mask, mi)
            mmref.suggest_moves(g, 1, mask, mi)
    o = _check_state(g, tr, mask, mi)
    cm, mm_ = mmref.compute_metrics(g, "host", "host")
    ocm = o.class_metrics()
    for f, of in (("P", "P"), ("Q", "Q"), ("S", "S"), ("cbo", "cbo"), ("n_methods", "n")):
        assert np.array_equal(cm[f].astype(np.int64), ocm[of])
    g.free()


def test_every_edit_kind_on_tiny_systems():
    for seed in range(6):
        base = tiny_random(seed + 3)
        tr = Tracked(base)
        g = mmref.load_synth(base, device=True, cbo_attrs=bool(seed % 2))
        mmref.compute_metrics(g, None, None)
        mmref.suggest_moves(g, 10, 7, 1)
        rng = np.random.default_rng(100 + seed)
        for _ in range(12):
            kind, m, t = tr.random_edit(rng)
            mmref.apply_edit(g, kind, m, t)
            tr.apply(kind, m, t)
            _check_state(g, tr, 7, 1, cbo_attrs=bool(seed % 2))
        g.free()


def test_edits_without_a_kept_cache_and_growth():
    """Many additions grow the device arrays; no cached suggestions exist."""
    base = synth.generate(30, 200, 80, max_class=20, seed=9)
    tr = Tracked(base)
    g = mmref.load_synth(base, device=True)
    mmref.compute_metrics(g, None, None)
    rng = np.random.default_rng(4)
    added = 0
    while added < 600:
        m = int(rng.integers(200))
        if rng.random() < 0.5:
            a = int(rng.integers(80))
            if a in tr.acc[m]:
                continue
            mmref.apply_edit(g, ADD_ACCESS, m, a)
            tr.apply(ADD_ACCESS, m, a)
        else:
            t = int(rng.integers(200))
            if t == m or t in tr.calls[m]:
                continue
            mmref.apply_edit(g, ADD_CALL, m, t)
            tr.apply(ADD_CALL, m, t)
        added += 1
    _check_state(g, tr, 3, 2)
    g.free()


def test_invalid_edits_change_nothing():
    base = tiny_random(5)
    tr = Tracked(base)
    g = mmref.load_synth(base, device=True)
    mmref.compute_metrics(g, None, None)
    mmref.suggest_moves(g, 10, 7, 1)
    dig0 = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 1, digest=dig0)
    m = next(x for x in range(base.n_methods) if tr.acc[x] and tr.calls[x])
    a, t = tr.acc[m][0], tr.calls[m][0]
    missing_a = next(x for x in range(base.n_attrs) if x not in tr.acc[m])
    missing_t = next(x for x in range(base.n_methods) if x != m and x not in tr.calls[m])
    for kind, tgt, status in ((ADD_ACCESS, a, mmref.MM_EEXIST), (REMOVE_ACCESS, missing_a, mmref.MM_ENOTFOUND),
                              (ADD_CALL, t, mmref.MM_EEXIST), (REMOVE_CALL, missing_t, mmref.MM_ENOTFOUND),
                              (ADD_CALL, m, mmref.MM_EINVAL), (MOVE, tr.method_class[m], mmref.MM_EINVAL),
                              (MOVE, base.n_classes, mmref.MM_EINVAL), (ADD_ACCESS, base.n_attrs, mmref.MM_EINVAL)):
        with pytest.raises(mmref.MMError) as e:
            mmref.apply_edit(g, kind, m, tgt)
        assert e.value.status == status
    dig1 = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 1, digest=dig1)
    assert dig0[0] == dig1[0]
    _check_state(g, tr, 7, 1)
    g.free()


# ---------------------------------------------------------------- move sequences

@pytest.mark.parametrize("name,mask,mi,rounds,per_round", [("tiny", 3, 2, 4, 0), ("tiny", 3, 1, 3, 5),
                                                           ("tiny", 7, 1, 2, 0), ("medium", 3, 2, 2, 0)])
def test_sequence_equals_oracle(name, mask, mi, rounds, per_round):
    """Rounds of non-conflicting kept moves applied on the GPU equal the
    oracle's rounds, move for move, and the final state's metrics equal a
    recomputation from the oracle."""
    s = synth.named(name)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    got = mmref.apply_sequence(g, rounds, mask, mi, per_round=per_round)
    exp, final = oracle.sequence(s, mask=mask, min_improved=mi, rounds=rounds,
                                 per_round=per_round if per_round > 0 else 1 << 30)
    assert [tuple(int(v) for v in x) for x in got] == exp
    mc = mmref.export_system(g)[0]
    assert np.array_equal(mc, final)
    cur = synth.System(s.n_classes, s.n_methods, s.n_attrs, final, s.attr_class, s.acc_rowptr, s.acc_idx,
                       s.call_rowptr, s.call_idx)
    cm, mm_ = mmref.export_metrics(g)
    ocm = oracle.Oracle(cur).class_metrics()
    assert np.array_equal(cm["P"], ocm["P"]) and np.array_equal(cm["cbo"].astype(np.int64), ocm["cbo"])
    g.free()
