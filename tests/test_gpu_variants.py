"""GPU parity of the LCOM and CBO variants (Sec. II.B) and of the ranking of
classes by a metric against the CPU oracle, through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

from sysutil import make_system, tiny_random

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

# GPU field -> oracle field
FIELDS = {"P_all": "P_all", "Q_all": "Q_all", "lcom_ck_all": "ck_all", "lcom_pq": "pq", "lcom_pq_all": "pq_all",
          "cbo_out": "cbo_out", "cbo_in": "cbo_in", "cbo_bi": "cbo_bi"}
RANKS = {mmref.RANK_LCOM_CK: lambda cm, v: cm["ck"], mmref.RANK_LCOM_PQ: lambda cm, v: v["pq"],
         mmref.RANK_LCOM_CK_ALL: lambda cm, v: v["ck_all"], mmref.RANK_LCOM_PQ_ALL: lambda cm, v: v["pq_all"],
         mmref.RANK_CBO: lambda cm, v: cm["cbo"], mmref.RANK_CBO_IN: lambda cm, v: v["cbo_in"],
         mmref.RANK_CBO_BI: lambda cm, v: v["cbo_bi"]}


def _check(s, cbo_attrs=True, o=None, device=True):
    o = o or oracle.Oracle(s, cbo_attrs=cbo_attrs)
    g = mmref.load_synth(s, cbo_attrs=cbo_attrs, device=device)
    mmref.compute_metrics(g, None, None)
    v, q_all = mmref.metric_variants(g)
    ov, oq = o.class_variants()
    for gf, of in FIELDS.items():
        assert np.array_equal(v[gf].astype(np.int64), ov[of]), gf
    assert np.array_equal(q_all, oq)
    return g, o, ov


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("cbo_attrs", [True, False])
def test_variants_small_random(seed, cbo_attrs):
    g, _, _ = _check(tiny_random(seed), cbo_attrs)
    g.free()


def test_variants_tiny_and_medium():
    for name in ("tiny", "medium"):
        g, _, _ = _check(synth.named(name))
        g.free()


def test_variants_large():
    g, _, _ = _check(synth.named("large"))
    g.free()


def test_variants_methods_with_many_accesses():
    """Methods with 40 to 90 accesses (own and foreign attributes): the warp
    unions walk several 32-access chunks, for the own-attribute LCOM as for
    the variant, and must count each sharing method once."""
    rng = np.random.default_rng(17)
    c, per, A = 6, 30, 240
    mc = np.repeat(np.arange(c), per)
    ac = np.repeat(np.arange(c), A // c)
    acc = []
    for x in range(c * per):
        k = int(rng.integers(40, 91)) if x % 5 == 0 else int(rng.integers(0, 6))
        acc.append(sorted(rng.choice(A, size=k, replace=False).tolist()))
    calls = [sorted(set(rng.choice(c * per, size=3).tolist()) - {x}) for x in range(c * per)]
    s = make_system(mc, ac, acc, calls, c)
    g, o, _ = _check(s)
    cm, mm_ = mmref.export_metrics(g)
    ocm, omm = o.class_metrics(), o.method_metrics()
    assert np.array_equal(mm_["q"], omm["q"]) and np.array_equal(cm["Q"], ocm["Q"])
    g.free()


def test_variants_after_move_edits():
    """Variants of the edited state equal the oracle's on the moved system."""
    s = synth.named("tiny")
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    mc = s.method_class.copy()
    rng = np.random.default_rng(3)
    for m in rng.choice(s.n_methods, size=6, replace=False):
        d = int((mc[m] + 1 + rng.integers(0, s.n_classes - 1)) % s.n_classes)
        mmref.apply_edit(g, mmref.EDIT_MOVE, int(m), d)
        mc[m] = d
    moved = synth.System(s.n_classes, s.n_methods, s.n_attrs, mc, s.attr_class, s.acc_rowptr, s.acc_idx,
                         s.call_rowptr, s.call_idx)
    v, q_all = mmref.metric_variants(g)
    ov, oq = oracle.Oracle(moved).class_variants()
    for gf, of in FIELDS.items():
        assert np.array_equal(v[gf].astype(np.int64), ov[of]), gf
    assert np.array_equal(q_all, oq)
    g.free()


def test_variants_device_outputs():
    s = synth.named("tiny")
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    vh, qh = mmref.metric_variants(g)
    vd = torch.empty(56 * s.n_classes, dtype=torch.uint8, device="cuda")
    qd = torch.empty(4 * s.n_methods, dtype=torch.uint8, device="cuda")
    mmref.metric_variants(g, vd, qd)
    torch.cuda.synchronize()
    assert np.array_equal(vd.cpu().numpy().view(mmref.VARIANTS_DTYPE), vh)
    assert np.array_equal(qd.cpu().numpy().view(np.int32), qh)
    g.free()


def test_rank_classes_every_metric():
    s = synth.named("medium")
    o = oracle.Oracle(s)
    cm = o.class_metrics()
    ov, _ = o.class_variants()
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    for metric, value in RANKS.items():
        vals = value(cm, ov)
        for k in (0, 1, 37, s.n_classes, s.n_classes + 5):
            ids, got = mmref.rank_classes(g, metric, k)
            want = oracle.rank_classes(vals, k)
            assert np.array_equal(ids, want), (metric, k)
            assert np.array_equal(got, vals[want]), (metric, k)
    g.free()


def test_rank_classes_rejects_bad_arguments():
    s = tiny_random(2)
    g = mmref.load_synth(s)
    with pytest.raises(mmref.MMError):
        mmref.rank_classes(g, mmref.RANK_CBO, 3)  # metrics not computed yet
    mmref.compute_metrics(g, None, None)
    for metric in (0, 8, -1):
        with pytest.raises(mmref.MMError) as e:
            mmref.rank_classes(g, metric, 3)
        assert e.value.status == mmref.MM_EINVAL
    with pytest.raises(mmref.MMError):
        mmref.rank_classes(g, mmref.RANK_CBO, -1)
    g.free()
