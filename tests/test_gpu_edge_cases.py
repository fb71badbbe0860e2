"""Degenerate inputs for the similarity, rules, variants, ranking, coupling
forms, staged lists and move sequences: systems without attributes, without
calls, without any use edge, with one class or empty classes, and empty
candidate lists; every result against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

from sysutil import make_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

FIELDS = {"P_all": "P_all", "Q_all": "Q_all", "lcom_ck_all": "ck_all", "lcom_pq": "pq", "lcom_pq_all": "pq_all",
          "cbo_out": "cbo_out", "cbo_in": "cbo_in", "cbo_bi": "cbo_bi"}
OKEPT = ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")
KEPT = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")


def _kept(a, names):
    return [tuple(int(x[f]) for f in names) for x in a]


def _systems():
    rng = np.random.default_rng(7)
    out = {}
    # no attributes, calls only
    mc = [0, 0, 1, 1, 2, 2]
    out["no_attrs"] = make_system(mc, [], [[] for _ in mc], [[2], [3], [4], [0], [], [1]], n_classes=3)
    # no calls, accesses only (own and foreign)
    out["no_calls"] = make_system(mc, [0, 0, 1, 2], [[0, 1], [1], [2], [0], [3], []], [[] for _ in mc], n_classes=3)
    # no use edge at all: every access own, no calls
    out["no_edges"] = make_system(mc, [0, 1, 2], [[0], [0], [1], [], [2], [2]], [[] for _ in mc], n_classes=3)
    # one class
    out["one_class"] = make_system([0, 0, 0, 0], [0, 0], [[0], [1], [0, 1], []], [[1], [2], [], [0]], n_classes=1)
    # empty classes between used ones
    mc2 = [1, 1, 4, 4, 4, 7]
    out["empty_classes"] = make_system(mc2, [1, 4, 7], [[0], [1], [1], [2], [], [0]],
                                       [[2], [5], [0], [], [1], [3]], n_classes=9)
    # a random small system with many empty classes
    out["sparse"] = synth.generate(n_classes=300, n_methods=400, n_attrs=150, max_class=8, seed=int(rng.integers(99)),
                                   lambda_acc=1.0, lambda_call=1.0, p_loc=0.5)
    return out


SYSTEMS = _systems()


@pytest.mark.parametrize("name", sorted(SYSTEMS))
@pytest.mark.parametrize("flags", [0, 1])
def test_metrics_variants_and_ranks(name, flags):
    s = SYSTEMS[name]
    o = oracle.Oracle(s, threads=1)
    g = mmref.load_synth(s, device=True, flags=flags)
    cm, mm_ = mmref.compute_metrics(g, "host", "host")
    ocm = o.class_metrics()
    for gf, of in (("P", "P"), ("Q", "Q"), ("S", "S"), ("cbo", "cbo"), ("lcom_ck", "ck")):
        assert np.array_equal(cm[gf].astype(np.int64), ocm[of]), gf
    v, q_all = mmref.metric_variants(g)
    ov, oq = o.class_variants()
    for gf, of in FIELDS.items():
        assert np.array_equal(v[gf].astype(np.int64), ov[of]), gf
    assert np.array_equal(q_all, oq)
    for metric, vals in ((mmref.RANK_CBO_BI, ov["cbo_bi"]), (mmref.RANK_LCOM_PQ_ALL, ov["pq_all"]),
                         (mmref.RANK_LCOM_CK, ocm["ck"])):
        ids, got = mmref.rank_classes(g, metric, s.n_classes + 3)
        assert np.array_equal(ids, oracle.rank_classes(vals, s.n_classes)) and np.array_equal(got, vals[ids])
    g.free()


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_similarity_rules_and_sequences(name):
    s = SYSTEMS[name]
    o = oracle.Oracle(s, threads=1)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    (x, y, i, u), info = mmref.similarity(g)
    ox, oy, oi, ou = o.similarity()
    assert info["n_values"] == len(ox)
    for a, b in ((x, ox), (y, oy), (i, oi), (u, ou)):
        assert np.array_equal(a, b)
    res, avg, rp, dst, nv, nh = o.r1(mask=3, min_improved=2)
    top, nk, nm, inf = mmref.suggest_r1(g, 1000, 3, 2)
    assert (nk, nm, inf["n_high"], inf["n_candidates"]) == (res.n_kept, res.n_methods_with_kept, nh, len(dst))
    assert _kept(top, KEPT) == _kept(res.kept, OKEPT)
    kept3, rp3, dst3, nh3 = oracle.r3(s)
    top3, nk3, nc3, nhc = mmref.suggest_r3(g, max(len(kept3), 1))
    assert (nk3, nc3, nhc) == (len(kept3), len(dst3), nh3)
    assert [tuple(int(v) for v in t) for t in top3] == [tuple(int(v) for v in k) for k in kept3]
    seq_o, _ = oracle.sequence(s, mask=3, min_improved=1, rounds=3)
    seq_g = mmref.apply_sequence(g, 3, 3, 1)
    assert [tuple(int(v) for v in r) for r in seq_g] == seq_o
    assert len(mmref.apply_sequence(g, 0, 3, 1)) == 0
    g.free()


def test_empty_candidate_lists_everywhere():
    """Lists with no entry at all: evaluation, suggestion, staging and the
    allocation-free suggestion all return nothing, digest 0."""
    s = SYSTEMS["sparse"]
    rp = np.zeros(s.n_methods + 1, dtype=np.int64)
    dst = np.zeros(0, dtype=np.int32)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    dig = np.ones(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 1, rp, dst, digest=dig)
    assert int(dig[0]) == 0
    top, nk, nm = mmref.suggest_moves(g, 10, 7, 1, rp, dst)
    assert (len(top), nk, nm) == (0, 0, 0)
    mmref.stage_candidates(g, rp, dst)
    top, nk, nm = mmref.suggest_moves(g, 10, 7, 1, rp, dst, lists_unchanged=True)
    assert (len(top), nk, nm) == (0, 0, 0)
    rpd, dd = torch.from_numpy(rp).cuda(), torch.zeros(1, dtype=torch.int32, device="cuda")
    top, nk, nm = mmref.suggest_moves_noalloc(g, 10, 7, 1, rpd, dd[:0])
    assert (len(top), nk, nm) == (0, 0, 0)
    g.free()
