"""Failure detection on the GPU without a fault: the bounded look-back wait of
the exclusive scan (one scan tile whose predecessor is never processed) gives
up after its limit, the host reads MM_ETIMEOUT, and the context stays usable:
a system that needs multi-tile scans evaluates bit-exactly afterwards."""
import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402


def test_stalled_wait_times_out_and_context_survives():
    assert mmref.selftest_bounded_wait() == mmref.MM_ETIMEOUT
    # the flag was cleared: a second probe times out again (not a stale flag)
    assert mmref.selftest_bounded_wait() == mmref.MM_ETIMEOUT
    # 20,000 methods and attributes: the offset scans (over methods, attributes)
    # exceed one block and take the multi-tile path with look-back
    s = synth.generate(n_classes=300, n_methods=20000, n_attrs=20000, max_class=150, seed=41)
    g = mmref.load_synth(s, device=False)
    mmref.compute_metrics(g, None, None)
    ref = oracle.Oracle(s, threads=4).evaluate(mask=4, min_improved=1)
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 4, 1, digest=dig)
    assert int(dig[0]) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, 10, 4, 1)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and nk > 0
    assert [(int(x["m"]), int(x["d"])) for x in top] == [(int(k["m"]), int(k["d"])) for k in ref.kept[:10]]
    g.free()


CLASS_MAP = {"n_methods": "n", "n_attrs": "a", "P": "P", "Q": "Q", "S": "S", "lcom_ck": "ck",
             "hs_num": "hs_num", "hs_den": "hs_den", "cbo": "cbo"}


def _same_metrics(o, cm, mm_):
    ocm, omm = o.class_metrics(), o.method_metrics()
    for g, f in CLASS_MAP.items():
        assert np.array_equal(cm[g].astype(np.int64), ocm[f]), g
    for f in ("fan_in", "fan_out", "own", "q"):
        assert np.array_equal(mm_[f], omm[f]), f


def test_give_up_inside_compute_metrics_reaches_its_own_system_only():
    """The look-back of every multi-tile scan of one system's metric pipeline
    is made to run out (test hook): that system's next synchronising call
    reports MM_ETIMEOUT once, its outputs are still exact (the fallback sums
    the input before the tile), another system on another stream sees no
    error, and the following calls are bit-exact."""
    sa = synth.generate(n_classes=300, n_methods=20000, n_attrs=20000, max_class=150, seed=41)
    sb = synth.generate(n_classes=260, n_methods=18000, n_attrs=18000, max_class=150, seed=43)
    oa, ob = oracle.Oracle(sa, threads=4), oracle.Oracle(sb, threads=4)
    other = torch.cuda.Stream()
    a = mmref.load_synth(sa, device=True)
    b = mmref.load_synth(sb, device=True, stream=other)
    mmref.selftest_stall_scans(a, 1000)
    cm = np.zeros(a.n_classes, dtype=mmref.CLASS_METRICS_DTYPE)
    mm_ = np.zeros(a.n_methods, dtype=mmref.METHOD_METRICS_DTYPE)
    with pytest.raises(mmref.MMError) as err:
        mmref.compute_metrics(a, cm, mm_)
    assert err.value.status == mmref.MM_ETIMEOUT
    _same_metrics(oa, cm, mm_)  # written before the status was returned, and exact
    cmb, mmb = mmref.compute_metrics(b, "host", "host")  # no error: the fault word is a's alone
    _same_metrics(ob, cmb, mmb)
    mmref.selftest_stall_scans(a, 0)
    cm2, mm2 = mmref.compute_metrics(a, "host", "host")  # the word was cleared when read
    _same_metrics(oa, cm2, mm2)
    ref = oa.evaluate(mask=7, min_improved=1)
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(a, 7, 1, digest=dig)
    assert int(dig[0]) == ref.digest
    top, nk, nm = mmref.suggest_moves(a, 10, 7, 1)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert [(int(x["m"]), int(x["d"])) for x in top] == [(int(k["m"]), int(k["d"])) for k in ref.kept[:10]]
    oa.close()
    ob.close()
    a.free()
    b.free()


def test_give_up_reported_by_suggest_when_metrics_stay_on_the_device():
    """Metrics computed into device memory do not synchronise: the stalled
    scans' fault is reported by the system's next synchronising call
    (mm_suggest_moves), whose result is still the oracle's."""
    s = synth.generate(n_classes=300, n_methods=20000, n_attrs=20000, max_class=150, seed=41)
    o = oracle.Oracle(s, threads=4)
    g = mmref.load_synth(s, device=True)
    mmref.selftest_stall_scans(g, 1000)
    mmref.compute_metrics(g, None, None)
    mmref.selftest_stall_scans(g, 0)
    ref = o.evaluate(mask=3, min_improved=2)
    with pytest.raises(mmref.MMError) as err:
        mmref.suggest_moves(g, 10, 3, 2)
    assert err.value.status == mmref.MM_ETIMEOUT
    top, nk, nm = mmref.suggest_moves(g, 10, 3, 2)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert [(int(x["m"]), int(x["d"])) for x in top] == [(int(k["m"]), int(k["d"])) for k in ref.kept[:10]]
    o.close()
    g.free()
