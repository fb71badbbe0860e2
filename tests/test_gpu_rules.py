"""GPU parity of rule R3 (Sec. III.A, third rule) against the CPU oracle,
through the C ABI."""
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


def _check(s, cbo_attrs=True):
    kept, rowptr, dst, nhigh = oracle.r3(s, cbo_attrs=cbo_attrs)
    g = mmref.load_synth(s, cbo_attrs=cbo_attrs, device=True)
    mmref.compute_metrics(g, None, None)
    top, nk, nc, nh = mmref.suggest_r3(g, max(len(kept), 1))
    assert (nk, nc, nh) == (len(kept), len(dst), nhigh)
    assert [tuple(int(v) for v in x) for x in top] == [tuple(int(v) for v in x) for x in kept]
    g.free()
    return len(kept)


@pytest.mark.parametrize("name", ["tiny", "medium", "large"])
def test_named_workloads(name):
    assert _check(synth.named(name)) > 0


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny(seed):
    s = tiny_random(seed + 100)
    _check(s)
    _check(s, cbo_attrs=False)


def test_hand_example():
    s = make_system([0, 0, 1, 2], [], [[], [], [], []], [[2, 3], [2], [3], []], n_classes=3)
    g = mmref.load_synth(s, device=True)
    mmref.compute_metrics(g, None, None)
    top, nk, nc, nh = mmref.suggest_r3(g, 10)
    assert (nk, nc, nh) == (1, 3, 1) and [tuple(int(v) for v in x) for x in top] == [(0, 1, 0, 2, -1, 0)]
    g.free()
