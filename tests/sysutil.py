"""Helpers for tests: build systems from plain lists, permute ids, tiny randoms."""
from __future__ import annotations

import json
import os

import numpy as np

from paper_1308_4011_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def make_system(method_class, attr_class, acc, calls, n_classes=None, name="hand"):
    n_classes = n_classes if n_classes is not None else (max(list(method_class) + list(attr_class) + [-1]) + 1)
    acc = [sorted(set(int(v) for v in row)) for row in acc]
    calls = [sorted(set(int(v) for v in row)) for row in calls]
    acc_rowptr = np.zeros(len(acc) + 1, dtype=np.int64)
    acc_rowptr[1:] = np.cumsum([len(r) for r in acc])
    call_rowptr = np.zeros(len(calls) + 1, dtype=np.int64)
    call_rowptr[1:] = np.cumsum([len(r) for r in calls])
    return synth.System(
        n_classes=int(n_classes), n_methods=len(method_class), n_attrs=len(attr_class),
        method_class=np.asarray(method_class, dtype=np.int32),
        attr_class=np.asarray(attr_class, dtype=np.int32),
        acc_rowptr=acc_rowptr, acc_idx=np.asarray([v for r in acc for v in r], dtype=np.int32),
        call_rowptr=call_rowptr, call_idx=np.asarray([v for r in calls for v in r], dtype=np.int32),
        name=name)


def hand_example():
    with open(os.path.join(GOLDEN, "hand_example.json")) as f:
        g = json.load(f)
    s = g["system"]
    return make_system(s["method_class"], s["attr_class"], s["acc"], s["calls"], s["n_classes"]), g


def tiny_random(seed: int):
    """A random system of 3..8 classes and up to ~30 methods."""
    c = 3 + seed % 6
    M = c + 4 + (seed * 7) % 18
    A = (seed * 3) % 11
    return synth.generate(c, M, A, max_class=max(2, (M + c - 1) // c + 3), seed=seed,
                          lambda_acc=2.5, lambda_call=2.0, p_loc=0.6)


def permute(sys_, seed: int):
    """Relabel classes, methods and attributes by seeded permutations.
    Returns (new system, pc, pm, pa) with new_id = p[old_id]."""
    rng = np.random.default_rng(seed)
    pc = rng.permutation(sys_.n_classes)
    pm = rng.permutation(sys_.n_methods)
    pa = rng.permutation(sys_.n_attrs)
    mc = np.zeros(sys_.n_methods, dtype=np.int32)
    mc[pm] = pc[sys_.method_class]
    ac = np.zeros(sys_.n_attrs, dtype=np.int32)
    ac[pa] = pc[sys_.attr_class]
    acc = [None] * sys_.n_methods
    calls = [None] * sys_.n_methods
    for x in range(sys_.n_methods):
        acc[pm[x]] = [int(pa[a]) for a in sys_.acc(x)]
        calls[pm[x]] = [int(pm[t]) for t in sys_.calls(x)]
    return make_system(mc, ac, acc, calls, sys_.n_classes, name=sys_.name + "-perm"), pc, pm, pa


def moved(sys_, m: int, d: int):
    """The system after moving method m to class d (attributes stay)."""
    mc = sys_.method_class.copy()
    mc[m] = d
    return synth.System(sys_.n_classes, sys_.n_methods, sys_.n_attrs, mc, sys_.attr_class.copy(),
                        sys_.acc_rowptr.copy(), sys_.acc_idx.copy(), sys_.call_rowptr.copy(),
                        sys_.call_idx.copy(), name=sys_.name + "-moved")
