"""GPU parity of the Jaccard similarity values (Sec. II.A) and of rule R1's
suggestions (Sec. III.A) against the CPU oracle, through the C ABI."""
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

KEPT = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")
OKEPT = ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")


def _kept(a, names=KEPT):
    return [tuple(int(x[f]) for f in names) for x in a]


def _check_values(s, o=None):
    o = o or oracle.Oracle(s)
    g = mmref.load_synth(s, device=True)
    (x, y, i, u), info = mmref.similarity(g)
    ox, oy, oi, ou = o.similarity()
    assert info["n_values"] == len(ox)
    for a, b in ((x, ox), (y, oy), (i, oi), (u, ou)):
        assert np.array_equal(a, b)
    avg, _ = oracle.r1_threshold(oi, ou, int(ou.max()) if len(ou) else 0)
    assert info["average"] == avg  # the same double, bit for bit
    return g, o, (ox, oy, oi, ou), info


def test_tiny_every_value_and_r1():
    s = synth.named("tiny")
    g, o, vals, info = _check_values(s)
    mmref.compute_metrics(g, None, None)
    ref, avg, rp, dst, nv, nh = o.r1(mask=3, min_improved=2)
    top, nk, nm, rinfo = mmref.suggest_r1(g, 100000, 3, 2)
    assert (rinfo["n_high"], rinfo["n_candidates"]) == (nh, len(dst))
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert _kept(top) == _kept(ref.kept, OKEPT)
    # other criteria over the same proposed moves
    for mask, mi in ((7, 1), (1, 1)):
        r2 = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1)
        top, nk, nm, _ = mmref.suggest_r1(g, 100000, mask, mi)
        assert (nk, nm) == (r2.n_kept, r2.n_methods_with_kept) and _kept(top) == _kept(r2.kept, OKEPT)
    g.free()


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_values_and_r1(seed):
    s = tiny_random(seed + 40)
    g, o, _, _ = _check_values(s, oracle.Oracle(s, threads=1))
    mmref.compute_metrics(g, None, None)
    ref, *_ = o.r1()
    top, nk, nm, _ = mmref.suggest_r1(g, 1000)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and _kept(top) == _kept(ref.kept, OKEPT)
    g.free()


def test_no_values():
    """Methods without properties, or a single method: no values, average 0, no suggestion."""
    s = make_system([0, 0, 1], [0], [[], [], []], [[], [], []], n_classes=2)
    g = mmref.load_synth(s, device=True)
    (x, y, i, u), info = mmref.similarity(g)
    assert len(x) == 0 and info["n_values"] == 0 and info["average"] == 0.0
    mmref.compute_metrics(g, None, None)
    top, nk, nm, info = mmref.suggest_r1(g, 10)
    assert (len(top), nk, nm, info["n_candidates"]) == (0, 0, 0, 0)
    g.free()
    s = make_system([0], [0], [[0]], [[]], n_classes=1)
    g = mmref.load_synth(s, device=True)
    assert mmref.similarity(g)[1]["n_values"] == 0
    g.free()


def test_medium_every_value_and_r1():
    s = synth.named("medium")
    o = oracle.Oracle(s)
    g, o, (ox, oy, oi, ou), info = _check_values(s, o)
    mmref.compute_metrics(g, None, None)
    avg, thr = oracle.r1_threshold(oi, ou, int(ou.max()))
    rp, dst, nh = oracle.r1_candidates(s, ox, oy, oi, ou, thr)
    ref = o.evaluate(mask=3, min_improved=2, cand_rowptr=rp, cand_dst=dst, method=1)
    top, nk, nm, rinfo = mmref.suggest_r1(g, 100000, 3, 2)
    assert (rinfo["n_high"], rinfo["n_candidates"]) == (nh, len(dst))
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and _kept(top) == _kept(ref.kept, OKEPT)
    g.free()


def test_large_sampled_rows():
    """The large system: every value of 40 sampled methods (both sides of the
    pair) against the oracle's row-by-row definition."""
    s = synth.named("large")
    g = mmref.load_synth(s, device=True)
    (x, y, i, u), info = mmref.similarity(g)
    assert np.all(x < y) and np.all((i > 0) & (i <= u))
    assert np.all(np.diff(x.astype(np.int64) * s.n_methods + y) > 0)  # (x, y) order, no repeats
    o = oracle.Oracle(s)
    rng = np.random.default_rng(9)
    for q in rng.choice(s.n_methods, size=40, replace=False):
        ry, ri, ru = o.similarity_row(int(q))
        sel = (x == q) | (y == q)
        partner = np.where(x[sel] == q, y[sel], x[sel])
        order = np.argsort(partner)
        assert np.array_equal(partner[order], ry)
        assert np.array_equal(i[sel][order], ri) and np.array_equal(u[sel][order], ru)
    g.free()
