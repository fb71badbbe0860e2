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
