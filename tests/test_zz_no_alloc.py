"""The allocation-free suggestion entry point (mm_suggest_moves_noalloc).

Some callers cannot allocate device memory when they ask for suggestions:
a serving process whose device memory is all reserved by its own fixed-budget
allocator, or a latency-critical loop that must not allocate.  For them the
library offers a variant of mm_suggest_moves that works in a fixed static
device array.  These tests call it through the C ABI and check, on two calls
in a row, that it returns exactly what mm_suggest_moves returns, and that it
rejects work beyond its stated limits with a clear error.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

from paper_1308_4011_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_4011_b300 import mmref  # noqa: E402

FIELDS = ("m", "d", "n_improved", "d_lcom_ck_sum", "d_cbo_sum")


def _rows(a):
    return [tuple(int(x[f]) for f in FIELDS) for x in a]


def _noalloc_c(g, k, mask, mi, out, kind, rowptr=None, dst=None):
    """Direct C-ABI call of mm_suggest_moves_noalloc (candidate lists: CUDA tensors or None)."""
    crit = mmref._Crit(mask, mi)
    nk, nm = ctypes.c_int64(-1), ctypes.c_int64(-1)
    ptr = out.data_ptr() if kind == mmref.PTR_DEVICE else out.ctypes.data
    cands = None
    if rowptr is not None:
        cands = ctypes.byref(mmref._Cands(rowptr.data_ptr(), dst.data_ptr(), int(dst.numel()), mmref.PTR_DEVICE, 0))
    rc = mmref._lib.mm_suggest_moves_noalloc(g.handle, ctypes.byref(crit), cands, k, ptr, kind, ctypes.byref(nk),
                                             ctypes.byref(nm))
    return rc, nk.value, nm.value


@pytest.fixture(scope="module")
def tiny():
    s = synth.named("tiny")
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    yield g
    g.free()


# (3, 2): a few dozen kept moves (one bitonic chunk); (1, 1): 63,656 kept moves
# (2,048-chunks plus merges); (7, 2): nothing kept
@pytest.mark.parametrize("mask,mi", [(3, 2), (1, 1), (7, 2)])
def test_noalloc_equals_suggest_on_two_calls(tiny, mask, mi):
    ref, ref_nk, ref_nm = mmref.suggest_moves(tiny, 100000, mask, mi)
    assert ref_nk <= mmref.NOALLOC_MAX_KEPT
    k = max(ref_nk, 1)
    for _ in range(2):
        out = np.zeros(k, dtype=mmref.MOVE_DTYPE)
        rc, nk, nm = _noalloc_c(tiny, k, mask, mi, out, mmref.PTR_HOST)
        assert rc == mmref.MM_OK, mmref._lib.mm_last_error()
        assert (nk, nm) == (ref_nk, ref_nm)
        assert _rows(out[:nk]) == _rows(ref)
        dev = torch.zeros(k * 24, dtype=torch.uint8, device="cuda")
        rc, nk2, _ = _noalloc_c(tiny, k, mask, mi, dev, mmref.PTR_DEVICE)
        assert rc == mmref.MM_OK and nk2 == ref_nk
        assert _rows(dev.cpu().numpy().view(mmref.MOVE_DTYPE)[:nk2]) == _rows(ref)


def test_noalloc_top10_after_a_larger_call(tiny):
    """The static array keeps the previous call's contents; a smaller call
    after a larger one must not see them."""
    big, _, _ = mmref.suggest_moves_noalloc(tiny, 70000, 1, 1)
    ref, nk, _ = mmref.suggest_moves(tiny, 10, 3, 2)
    top, nk2, _ = mmref.suggest_moves_noalloc(tiny, 10, 3, 2)
    assert len(big) > 10 and nk2 == nk and _rows(top) == _rows(ref)


def test_noalloc_rejects_more_kept_moves_than_its_limit():
    s = synth.generate(400, 8000, 4000, max_class=80, seed=3)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    _, nk, _ = mmref.suggest_moves(g, 0, 1, 1)
    assert nk > mmref.NOALLOC_MAX_KEPT
    out = np.zeros(10, dtype=mmref.MOVE_DTYPE)
    rc, _, _ = _noalloc_c(g, 10, 1, 1, out, mmref.PTR_HOST)
    assert rc == mmref.MM_EBUDGET and b"MM_NOALLOC_MAX_KEPT" in mmref._lib.mm_last_error()
    # still usable afterwards, and equal to the allocating entry point
    ref, nk, _ = mmref.suggest_moves(g, 50, 3, 2)
    rc, nk2, _ = _noalloc_c(g, 50, 3, 2, out := np.zeros(50, dtype=mmref.MOVE_DTYPE), mmref.PTR_HOST)
    assert rc == mmref.MM_OK and nk2 == nk and _rows(out[:nk2]) == _rows(ref)
    g.free()


def test_noalloc_rejects_systems_above_the_method_limit():
    n = mmref.NOALLOC_MAX_METHODS + 1
    s = synth.generate(20000, n, 1000, max_class=80, seed=5, lambda_acc=0.5, lambda_call=0.5)
    g = mmref.load_synth(s, device=True)
    out = np.zeros(1, dtype=mmref.MOVE_DTYPE)
    rc, _, _ = _noalloc_c(g, 1, 3, 2, out, mmref.PTR_HOST)
    assert rc == mmref.MM_EBUDGET and b"MM_NOALLOC_MAX_METHODS" in mmref._lib.mm_last_error()
    g.free()


def test_noalloc_first_call_on_a_fresh_system_equals_the_oracle():
    """The main use: a system loaded and measured (compute_metrics only), then
    asked for suggestions without allocating -- no earlier evaluation on the
    handle -- gives exactly the oracle's kept list."""
    import oracle
    s = synth.named("tiny")
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    ref = oracle.Oracle(s).evaluate(mask=3, min_improved=2, method=1)
    k = max(ref.n_kept, 1)
    for _ in range(2):
        out = np.zeros(k, dtype=mmref.MOVE_DTYPE)
        rc, nk, nm = _noalloc_c(g, k, 3, 2, out, mmref.PTR_HOST)
        assert rc == mmref.MM_OK, mmref._lib.mm_last_error()
        assert (nk, nm) == (ref.n_kept, ref.n_methods_with_kept)
        assert _rows(out[:nk]) == [tuple(int(x[f]) for f in ("m", "d", "n_improved", "d_ck_sum", "d_cbo_sum"))
                                   for x in ref.kept]
    g.free()


def test_noalloc_with_device_candidate_lists():
    """Candidate lists in device memory (validated on the device, read back
    without allocating host memory) give what mm_suggest_moves gives."""
    s = synth.generate(300, 4000, 2000, max_class=80, seed=12)
    rp, dst = synth.candidates(s, 16, seed=12)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    rpd, dd = torch.from_numpy(rp).cuda(), torch.from_numpy(dst).cuda()
    for mask, mi in ((3, 2), (7, 1)):
        ref, ref_nk, ref_nm = mmref.suggest_moves(g, 100000, mask, mi, rpd, dd)
        k = max(ref_nk, 1)
        for _ in range(2):
            out = np.zeros(k, dtype=mmref.MOVE_DTYPE)
            rc, nk, nm = _noalloc_c(g, k, mask, mi, out, mmref.PTR_HOST, rpd, dd)
            assert rc == mmref.MM_OK, mmref._lib.mm_last_error()
            assert (nk, nm) == (ref_nk, ref_nm)
            assert _rows(out[:nk]) == _rows(ref)
    g.free()
