"""The class coupling built from the use edges into the compressed rows (MM_LOAD_PACKED_COUPLING:
no full adjacency bitsets until a full cross-product evaluation builds them
from the multigraph rows) gives the same metrics, records, suggestions, edits,
rules and batches as the bitset construction, and both equal the oracle."""
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

PACKED, BITSET = mmref.LOAD_PACKED_COUPLING, mmref.LOAD_BITSET_COUPLING
CLASS_MAP = {"n_methods": "n", "n_attrs": "a", "P": "P", "Q": "Q", "S": "S", "lcom_ck": "ck",
             "hs_num": "hs_num", "hs_den": "hs_den", "cbo": "cbo"}
KEPT = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")
OKEPT = ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")


def _kept(a, names=KEPT):
    return [tuple(int(x[f]) for f in names) for x in a]


def _records(g, mask, mi, rowptr=None, dst=None):
    n = g.n_candidates_full if rowptr is None else len(dst)
    rec = torch.empty(max(n, 1) * 16, dtype=torch.uint8, device="cuda")
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    mmref.evaluate_moves(g, mask, mi, rowptr, dst, records=rec, digest=dig)
    torch.cuda.synchronize()
    return rec[: n * 16].cpu().numpy(), int(dig.cpu().numpy().view(np.uint64)[0])


def _check_metrics(o, cm, mm_):
    ocm, omm = o.class_metrics(), o.method_metrics()
    for gf, of in CLASS_MAP.items():
        assert np.array_equal(cm[gf].astype(np.int64), ocm[of]), gf
    for f in ("fan_in", "fan_out", "own", "q"):
        assert np.array_equal(mm_[f], omm[f]), f


@pytest.mark.parametrize("cbo_attrs", [True, False])
def test_packed_coupling_every_record_on_tiny(cbo_attrs):
    """Metrics and multigraph size; the restricted lists first (compressed rows
    only), then the full cross product (which builds the bitsets from the
    rows), record by record against the oracle."""
    s = synth.named("tiny")
    o = oracle.Oracle(s, cbo_attrs=cbo_attrs)
    g = mmref.load_synth(s, cbo_attrs=cbo_attrs, device=True, flags=PACKED)
    cm, mm_ = mmref.compute_metrics(g, "host", "host")
    _check_metrics(o, cm, mm_)
    assert g.info()["n_class_edges"] == len(o.multigraph()[1])
    rp, dst = synth.candidates(s, 16, 3)
    for mask, mi in ((7, 1), (3, 2)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = _records(g, mask, mi, torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda())
        assert np.array_equal(rec, ref.records.view(np.uint8)) and dig == ref.digest
    for mask, mi in ((7, 1), (3, 2)):
        ref = o.evaluate(mask=mask, min_improved=mi, method=1, records=True)
        rec, dig = _records(g, mask, mi)
        assert np.array_equal(rec, ref.records.view(np.uint8)) and dig == ref.digest
        top, nk, nm = mmref.suggest_moves(g, 100000, mask, mi)
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert _kept(top) == _kept(ref.kept, OKEPT)
    g.free()


@pytest.mark.parametrize("seed", range(4))
def test_packed_and_bitset_forms_agree_on_random_systems(seed):
    s = tiny_random(seed + 40)
    outs = []
    for flags in (PACKED, BITSET):
        g = mmref.load_synth(s, device=True, flags=flags)
        cm, mm_ = mmref.compute_metrics(g, "host", "host")
        rec, dig = _records(g, 7, 1)
        outs.append((cm.tobytes(), mm_.tobytes(), rec.tobytes(), dig))
        g.free()
    assert outs[0] == outs[1]


def test_packed_coupling_long_rows_general_path():
    """Methods with more list entries than the restricted kernel stages take
    its general path, whose probes read the compressed rows."""
    rng = np.random.default_rng(11)
    c, per = 160, 3
    method_class = [C for C in range(c) for _ in range(per)]
    attr_class = [C for C in range(c) for _ in range(2)]
    M = len(method_class)
    acc = [sorted(rng.choice(len(attr_class), size=rng.integers(0, 4), replace=False).tolist()) for _ in range(M)]
    calls = [sorted(set(rng.choice(M, size=rng.integers(0, 4)).tolist()) - {x}) for x in range(M)]
    calls[0] = sorted({3 * C + 1 for C in range(1, 151)})
    acc[0] = sorted({2 * C + k for C in range(1, 71) for k in (0, 1)})
    for C in range(10, 130):
        calls[3 * C + 2] = sorted(set(calls[3 * C + 2]) | {4})
    s = make_system(method_class, attr_class, acc, calls, n_classes=c)
    rows = [[D for D in range(c) if D != method_class[x]] if x in (0, 4)
            else sorted(set(rng.choice(c, size=5).tolist()) - {method_class[x]}) for x in range(M)]
    rp = np.zeros(M + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    dst = np.asarray([D for r in rows for D in r], dtype=np.int32)
    o = oracle.Oracle(s, threads=1)
    g = mmref.load_synth(s, device=True, flags=PACKED)
    mmref.compute_metrics(g, None, None)
    for mask, mi in ((7, 1), (3, 1)):
        ref = o.evaluate(mask=mask, min_improved=mi, cand_rowptr=rp, cand_dst=dst, method=1, records=True)
        rec, dig = _records(g, mask, mi, torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda())
        assert np.array_equal(rec, ref.records.view(np.uint8)) and dig == ref.digest
    g.free()


def test_packed_coupling_medium_digest():
    s = synth.named("medium")
    o = oracle.Oracle(s)
    g = mmref.load_synth(s, device=True, flags=PACKED)
    cm, mm_ = mmref.compute_metrics(g, "host", "host")
    _check_metrics(o, cm, mm_)
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 3, 2, digest=dig)
    assert int(dig[0]) == o.evaluate(mask=3, min_improved=2).digest
    g.free()


def test_large_system_takes_the_packed_form_by_size():
    """50,000 classes: the bitsets would take 626 MB, so the packed form is
    chosen without a flag; the restricted lists evaluate without building them."""
    s = synth.named("large")
    rp, dst = synth.candidates(s, synth.LARGE_EXTRA_CANDIDATES, seed=2)
    o = oracle.Oracle(s)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    assert g.info()["n_class_edges"] == len(o.multigraph()[1])
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 2, torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda(), digest=dig)
    assert int(dig[0]) == o.evaluate(mask=7, min_improved=2, cand_rowptr=rp, cand_dst=dst).digest
    g.free()


def test_edits_on_packed_coupling():
    """Edits rebuild the coupling in the packed form; the kept list kept up to date
    through the dense tiles (bitsets built on demand) equals a fresh oracle."""
    s = synth.generate(60, 500, 250, max_class=30, seed=3, lambda_acc=3, lambda_call=4, p_loc=0.7)
    g = mmref.load_synth(s, device=True, flags=PACKED)
    mmref.compute_metrics(g, None, None)
    mmref.suggest_moves(g, 10, 3, 2)
    rng = np.random.default_rng(2)
    mc = s.method_class.copy()
    for _ in range(5):
        m = int(rng.integers(0, s.n_methods))
        d = int((mc[m] + 1 + rng.integers(0, s.n_classes - 1)) % s.n_classes)
        mmref.apply_edit(g, mmref.EDIT_MOVE, m, d)
        mc[m] = d
    moved = synth.System(s.n_classes, s.n_methods, s.n_attrs, mc, s.attr_class, s.acc_rowptr, s.acc_idx,
                         s.call_rowptr, s.call_idx)
    ref = oracle.Oracle(moved).evaluate(mask=3, min_improved=2)
    top, nk, nm = mmref.suggest_moves(g, 100000, 3, 2)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
    assert _kept(top) == _kept(ref.kept, OKEPT)
    g.free()


def test_noalloc_full_cross_product_needs_the_bitsets():
    """Before any full cross-product call has built the bitsets of a packed
    system, the allocation-free suggestion refuses (MM_EBUDGET); after one, it
    answers like mm_suggest_moves."""
    s = synth.named("tiny")
    g = mmref.load_synth(s, device=True, flags=PACKED)
    mmref.compute_metrics(g, None, None)
    with pytest.raises(mmref.MMError) as e:
        mmref.suggest_moves_noalloc(g, 10, 3, 2)
    assert e.value.status == mmref.MM_EBUDGET
    top, nk, nm = mmref.suggest_moves(g, 10, 3, 2)
    top2, nk2, nm2 = mmref.suggest_moves_noalloc(g, 10, 3, 2)
    assert (nk, nm) == (nk2, nm2) and _kept(top) == _kept(top2)
    g.free()


def test_batch_of_packed_systems():
    """A batch switches its systems to the bitset form (its graph reads them)."""
    systems = [synth.generate(**synth.batched_params(100 + i)) for i in range(3)]
    gs = [mmref.load_synth(x, device=True, flags=PACKED) for x in systems]
    b = mmref.Batch(gs, mask=3, min_improved=2)
    digests, n_kept = b.run()
    for i, x in enumerate(systems):
        ref = oracle.Oracle(x).evaluate(mask=3, min_improved=2)
        assert int(digests[i]) == ref.digest and int(n_kept[i]) == ref.n_kept
    b.free()
    for g in gs:
        g.free()


def test_unknown_load_flags_rejected():
    s = tiny_random(1)
    with pytest.raises(mmref.MMError) as e:
        mmref.load_synth(s, flags=4)
    assert e.value.status == mmref.MM_EINVAL
