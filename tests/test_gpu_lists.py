"""Candidate lists passed again with MM_CANDS_UNCHANGED: the evaluation's check
and content hash are reused only for the same device lists with no edit in
between; otherwise the lists are checked again."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1308_4011_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

KEPT = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")
OKEPT = ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum")


def _kept(a, names=KEPT):
    return [tuple(int(x[f]) for f in names) for x in a]


def test_unchanged_lists_reuse_the_check():
    s = synth.named("tiny")
    rp, dst = synth.candidates(s, 12, 5)
    o = oracle.Oracle(s)
    ref = o.evaluate(mask=3, min_improved=1, cand_rowptr=rp, cand_dst=dst)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 3, 1, rpd, dd, digest=dig)
    assert int(dig[0]) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, 50, 3, 1, rpd, dd, lists_unchanged=True)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and _kept(top) == _kept(ref.kept[:50], OKEPT)
    # the same flag on the next call still answers the same
    top2, nk2, _ = mmref.suggest_moves(g, 50, 3, 1, rpd, dd, lists_unchanged=True)
    assert nk2 == nk and _kept(top2) == _kept(top)
    g.free()


def test_flag_ignored_for_other_lists_and_after_edits():
    s = synth.named("tiny")
    rp, dst = synth.candidates(s, 12, 5)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    mmref.suggest_moves(g, 10, 3, 1, rpd, dd)
    # other lists (a copy holding an invalid destination) are checked despite the flag
    bad = dd.clone()
    bad[0] = int(s.method_class[0])
    with pytest.raises(mmref.MMError) as e:
        mmref.suggest_moves(g, 10, 3, 1, rpd, bad, lists_unchanged=True)
    assert e.value.status == mmref.MM_EINVAL
    mmref.suggest_moves(g, 10, 3, 1, rpd, dd)  # the good lists checked again
    # after an edit the same lists are checked again: moving method 0 to its
    # first listed destination makes that entry its own class
    d0 = int(dst[0])
    mmref.apply_edit(g, mmref.EDIT_MOVE, 0, d0)
    with pytest.raises(mmref.MMError) as e:
        mmref.suggest_moves(g, 10, 3, 1, rpd, dd, lists_unchanged=True)
    assert e.value.status == mmref.MM_EINVAL
    g.free()


def test_unknown_list_flags_rejected():
    s = synth.named("tiny")
    rp, dst = synth.candidates(s, 4, 5)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    cd, keep = mmref._cands(torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda(), flags=6)
    import ctypes
    crit = mmref._Crit(3, 1)
    st = mmref._lib.mm_evaluate_moves(g.handle, ctypes.byref(crit), ctypes.byref(cd), None, None, mmref.PTR_DEVICE)
    assert st == mmref.MM_EINVAL
    del keep
    g.free()


def test_unchanged_host_lists_reuse_the_device_copy():
    """Host lists: the suggestion under the flag reuses the evaluation's device
    copy and check; a different host array is copied and checked again."""
    s = synth.named("tiny")
    rp, dst = synth.candidates(s, 12, 5)
    ref = oracle.Oracle(s).evaluate(mask=7, min_improved=1, cand_rowptr=rp, cand_dst=dst)
    g = mmref.load_synth(s)
    mmref.compute_metrics(g, None, None)
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 1, rp, dst, digest=dig)
    assert int(dig[0]) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, 50, 7, 1, rp, dst, lists_unchanged=True)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and _kept(top) == _kept(ref.kept[:50], OKEPT)
    bad = dst.copy()
    bad[0] = int(s.method_class[0])
    with pytest.raises(mmref.MMError) as e:
        mmref.suggest_moves(g, 10, 7, 1, rp, bad, lists_unchanged=True)
    assert e.value.status == mmref.MM_EINVAL
    g.free()


def test_large_host_lists_take_the_pipelined_copy():
    """Host lists of 2^24 entries or more are copied in chunks overlapped with
    their check and evaluation: records, digest and kept moves equal the
    device-list path, and a bad destination in the last chunk is reported."""
    s = synth.named("medium")
    rp, dst = synth.candidates(s, 300, 9)   # about 2e7 candidates
    assert len(dst) >= 1 << 24
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    n = len(dst)
    rec_h = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    dig_h = torch.zeros(1, dtype=torch.int64, device="cuda")
    mmref.evaluate_moves(g, 7, 1, rp, dst, records=rec_h, digest=dig_h)   # host lists
    top_h, nk_h, nm_h = mmref.suggest_moves(g, 100, 7, 1, rp, dst, lists_unchanged=True)
    rec_d = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    dig_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    mmref.evaluate_moves(g, 7, 1, rpd, dd, records=rec_d, digest=dig_d)  # device lists
    top_d, nk_d, nm_d = mmref.suggest_moves(g, 100, 7, 1, rpd, dd)
    torch.cuda.synchronize()
    assert torch.equal(rec_h, rec_d) and int(dig_h.item()) == int(dig_d.item())
    assert (nk_h, nm_h) == (nk_d, nm_d) and _kept(top_h) == _kept(top_d)
    ref = oracle.Oracle(s).evaluate(mask=7, min_improved=1, cand_rowptr=rp, cand_dst=dst)
    assert int(dig_d.cpu().numpy().view(np.uint64)[0]) == ref.digest
    bad = dst.copy()
    bad[-1] = s.n_classes  # out of range, in the last chunk
    with pytest.raises(mmref.MMError) as e:
        mmref.evaluate_moves(g, 7, 1, rp, bad, digest=np.zeros(1, dtype=np.uint64))
    assert e.value.status == mmref.MM_EINVAL
    g.free()


def test_staged_host_lists():
    """Lists staged before the metrics are computed are used by the evaluation
    and the suggestion that pass them unchanged; a bad staged list is reported
    by the call that uses it; an edit between makes the lists be copied and
    checked again; freeing a handle with a staged copy is safe."""
    s = synth.named("tiny")
    rp, dst = synth.candidates(s, 12, 5)
    ref = oracle.Oracle(s).evaluate(mask=7, min_improved=1, cand_rowptr=rp, cand_dst=dst)
    rp_p = torch.from_numpy(rp).pin_memory().numpy()
    dst_p = torch.from_numpy(dst).pin_memory().numpy()
    g = mmref.load_synth(s, device=True)
    mmref.stage_candidates(g, rp_p, dst_p)
    mmref.compute_metrics(g, None, None)
    dig = np.zeros(1, dtype=np.uint64)
    mmref.evaluate_moves(g, 7, 1, rp_p, dst_p, digest=dig, lists_unchanged=True)
    assert int(dig[0]) == ref.digest
    top, nk, nm = mmref.suggest_moves(g, 50, 7, 1, rp_p, dst_p, lists_unchanged=True)
    assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept) and _kept(top) == _kept(ref.kept[:50], OKEPT)
    # a bad list, staged: the error comes from the call that uses it
    bad = dst_p.copy()
    bad[3] = s.n_classes + 7
    mmref.stage_candidates(g, rp_p, bad)
    with pytest.raises(mmref.MMError) as e:
        mmref.evaluate_moves(g, 7, 1, rp_p, bad, digest=dig, lists_unchanged=True)
    assert e.value.status == mmref.MM_EINVAL
    # staged, then an edit: copied and checked again (moving method 0 into its
    # first listed class makes that entry its own class)
    mmref.stage_candidates(g, rp_p, dst_p)
    mmref.apply_edit(g, mmref.EDIT_MOVE, 0, int(dst[0]))
    with pytest.raises(mmref.MMError) as e:
        mmref.suggest_moves(g, 10, 7, 1, rp_p, dst_p, lists_unchanged=True)
    assert e.value.status == mmref.MM_EINVAL
    mmref.stage_candidates(g, rp_p, dst_p)
    g.free()  # waits for the staged copy
    with pytest.raises(ValueError):
        g2 = mmref.load_synth(s, device=True)
        try:
            mmref.stage_candidates(g2, torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda())
        finally:
            g2.free()
