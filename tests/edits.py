"""Seeded edit streams over a system (shared by the edit and serving tests)."""
from __future__ import annotations

import numpy as np

from sysutil import make_system

ADD_ACCESS, REMOVE_ACCESS, ADD_CALL, REMOVE_CALL, MOVE = 1, 2, 3, 4, 5


class Tracked:
    """A system as plain Python rows, kept in step with the edits applied."""

    def __init__(self, sys_):
        self.n_classes = sys_.n_classes
        self.method_class = [int(v) for v in sys_.method_class]
        self.attr_class = [int(v) for v in sys_.attr_class]
        self.acc = [sorted(int(v) for v in sys_.acc(x)) for x in range(sys_.n_methods)]
        self.calls = [sorted(int(v) for v in sys_.calls(x)) for x in range(sys_.n_methods)]

    def system(self):
        return make_system(self.method_class, self.attr_class, self.acc, self.calls, self.n_classes)

    def apply(self, kind, m, t):
        if kind == ADD_ACCESS:
            self.acc[m] = sorted(self.acc[m] + [t])
        elif kind == REMOVE_ACCESS:
            self.acc[m].remove(t)
        elif kind == ADD_CALL:
            self.calls[m] = sorted(self.calls[m] + [t])
        elif kind == REMOVE_CALL:
            self.calls[m].remove(t)
        else:
            self.method_class[m] = t

    def random_edit(self, rng):
        """A valid edit, each kind with probability 1/5 (falls back to a move)."""
        M, A, c = len(self.method_class), len(self.attr_class), self.n_classes
        kind = int(rng.integers(1, 6))
        m = int(rng.integers(M))
        if kind == ADD_ACCESS and A > len(self.acc[m]):
            while True:
                a = int(rng.integers(A))
                if a not in self.acc[m]:
                    return kind, m, a
        if kind == REMOVE_ACCESS and self.acc[m]:
            return kind, m, int(self.acc[m][int(rng.integers(len(self.acc[m])))])
        if kind == ADD_CALL and M - 1 > len(self.calls[m]):
            while True:
                t = int(rng.integers(M))
                if t != m and t not in self.calls[m]:
                    return kind, m, t
        if kind == REMOVE_CALL and self.calls[m]:
            return kind, m, int(self.calls[m][int(rng.integers(len(self.calls[m])))])
        d = int(rng.integers(c - 1))
        d += d >= self.method_class[m]
        return MOVE, m, d
