"""Serving: requests answered alone (one slot, one at a time) and in the mix
(several slots, overlapping on the device) give identical results; snapshots
of the evolving systems equal the oracle; admission under a small budget
evicts and reloads without changing any result."""
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

SHAPES = [(40, 480, 240), (150, 1800, 900), (90, 1080, 540), (300, 3600, 1800), (25, 300, 150), (120, 1440, 720)]
FIELDS = ("status", "kind", "m", "target", "n_kept", "n_methods_with_kept")


@pytest.fixture(scope="module")
def systems():
    return [synth.generate(c, m, a, max_class=80, seed=200 + i) for i, (c, m, a) in enumerate(SHAPES)]


def _serve(systems, req, n_slots, budget=1 << 36, snapshot_every=0):
    sv = mmref.Server(budget, n_slots=n_slots, topk=5, mask=3, min_improved=2)
    for s in systems:
        sv.add_system(s)
    resp, top = sv.run(req, snapshot_every)
    return sv, resp, top


def test_alone_equals_mix_and_oracle(systems):
    req = mmref.make_requests([s.n_methods for s in systems], 400, rate_per_s=0.0, seed=7)
    _, alone, top_a = _serve(systems, req, 1)
    sv, mix, top_m = _serve(systems, req, 6, snapshot_every=40)
    assert (alone["status"] == 0).all() and (mix["status"] == 0).all()
    for f in FIELDS:
        assert np.array_equal(alone[f], mix[f]), f
    assert np.array_equal(top_a, top_m)
    assert len(set(mix["slot"].tolist())) > 1  # several slots really were used
    # every snapshot equals the oracle on the exported system
    st = sv.stats()
    assert st["n_snapshots"] == 10
    for k in range(st["n_snapshots"]):
        i, si, c, arrs = sv.snapshot(k)
        s = synth.System(c, len(arrs[0]), len(arrs[1]), *arrs)
        ref = oracle.Oracle(s, threads=4).evaluate(mask=3, min_improved=2)
        assert mix["n_kept"][i] == ref.n_kept
        exp = [(int(x["m"]), int(x["d"])) for x in ref.kept[:5]]
        assert [(int(x["m"]), int(x["d"])) for x in top_m[i][: len(exp)]] == exp
    sv.free()


def test_small_budget_evicts_and_reloads_identically(systems):
    req = mmref.make_requests([s.n_methods for s in systems], 200, rate_per_s=0.0, seed=11)
    sv0, ref, top_r = _serve(systems, req, 4)
    everything = sv0.stats()["resident_bytes"]  # all six systems resident
    sv0.free()
    sv, got, top_g = _serve(systems, req, 4, budget=everything // 2)
    st = sv.stats()
    assert (got["status"] == 0).all()
    assert st["evictions"] > 0 and st["loads"] > len(systems)
    for f in FIELDS:
        assert np.array_equal(ref[f], got[f]), f
    assert np.array_equal(top_r, top_g)
    sv.free()


def test_budget_smaller_than_a_system_is_refused(systems):
    req = mmref.make_requests([s.n_methods for s in systems[:1]], 3, rate_per_s=0.0, seed=1)
    sv, resp, _ = _serve(systems[:1], req, 2, budget=1 << 20)
    assert (resp["status"] == mmref.MM_EBUDGET).all()
    sv.free()


def test_open_loop_arrivals_report_latency(systems):
    req = mmref.make_requests([s.n_methods for s in systems], 300, rate_per_s=2000.0, seed=3)
    sv, resp, _ = _serve(systems, req, 4)
    assert (resp["status"] == 0).all()
    lat = resp["done_s"] - resp["arrival_s"]
    assert (lat > 0).all() and (resp["start_s"] >= resp["arrival_s"] - 1e-6).all()
    sv.free()
