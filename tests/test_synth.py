"""The seeded generator: determinism, CSR validity, the stated shapes."""
import numpy as np
import pytest

from paper_1308_4011_b300 import synth


def _check_csr(s):
    assert s.method_class.min() >= 0 and s.method_class.max() < s.n_classes
    assert s.attr_class.size == 0 or (s.attr_class.min() >= 0 and s.attr_class.max() < s.n_classes)
    for rp, idx, hi in ((s.acc_rowptr, s.acc_idx, s.n_attrs), (s.call_rowptr, s.call_idx, s.n_methods)):
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == idx.size
        if idx.size:
            assert idx.min() >= 0 and idx.max() < hi
        rows = np.repeat(np.arange(s.n_methods), np.diff(rp))
        same = rows[1:] == rows[:-1]
        assert np.all(idx[1:][same] > idx[:-1][same])  # strictly increasing rows
    rows = np.repeat(np.arange(s.n_methods), np.diff(s.call_rowptr))
    assert not np.any(s.call_idx == rows)  # no self-calls


def test_deterministic():
    a, b = synth.named("tiny"), synth.named("tiny")
    for f in ("method_class", "attr_class", "acc_rowptr", "acc_idx", "call_rowptr", "call_idx"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = synth.generate(**{**synth.TINY, "seed": 9})
    assert not np.array_equal(a.acc_idx[:100], c.acc_idx[:100])


@pytest.mark.parametrize("name,cap,n_at_cap", [("tiny", 80, 7), ("medium", 400, 38)])
def test_shapes(name, cap, n_at_cap):
    s = synth.named(name)
    _check_csr(s)
    sizes = np.bincount(s.method_class, minlength=s.n_classes)
    assert sizes.sum() == s.n_methods and sizes.min() >= 1 and sizes.max() == cap
    assert (sizes == cap).sum() == n_at_cap
    assert np.bincount(s.attr_class, minlength=s.n_classes).sum() == s.n_attrs
    # methods contiguous by class id
    assert np.all(np.diff(s.method_class) >= 0)
    lam_a, lam_c = synth.TINY["lambda_acc"], synth.TINY["lambda_call"]
    if name == "medium":
        lam_a, lam_c = synth.MEDIUM["lambda_acc"], synth.MEDIUM["lambda_call"]
    # dedup only removes a few draws
    assert 0.85 * lam_a < s.n_acc / s.n_methods <= lam_a * 1.05
    assert 0.85 * lam_c < s.n_call / s.n_methods <= lam_c * 1.05


def test_candidates_restricted():
    s = synth.generate(300, 3000, 1500, max_class=80, seed=3)
    rowptr, dst = synth.candidates(s, 64, seed=3)
    for m in range(0, s.n_methods, 37):
        row = dst[rowptr[m]:rowptr[m + 1]]
        assert np.all(np.diff(row) > 0) and s.method_class[m] not in row
        natural = (set(s.attr_class[s.acc(m)].tolist()) | set(s.method_class[s.calls(m)].tolist())) - {int(s.method_class[m])}
        assert natural <= set(row.tolist())
        assert len(row) == len(natural) + 64


def test_batched_class_counts():
    cs = [synth.logu_classes(100 + i) for i in range(256)]
    assert min(cs) >= 100 and max(cs) <= 20000
    assert 300 < np.exp(np.mean(np.log(cs))) < 5000


def test_workload_checksums():
    """Every named workload (tiny, medium, large and its candidate lists, the
    256 batched systems of seeds 100..355, the 64 served systems of seeds
    100..163) hashes to the digest stored in tests/golden/synth_checksums.json:
    a generator change cannot silently change the workloads."""
    import json
    import os
    import sys
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, golden)
    try:
        import make_synth_checksums as mk
    finally:
        sys.path.remove(golden)
    with open(os.path.join(golden, "synth_checksums.json")) as f:
        stored = json.load(f)
    assert mk.compute() == stored
